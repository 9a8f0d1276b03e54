// Pair counts with no device allocation: the cell-list scratch of the pair
// enumeration lives in one file-scope __device__ array instead of a plan's
// workspace. The same launchers as pg_find_pairs run on it.
#include <math.h>
#include <string.h>

#include <mutex>

#include "pg_internal.cuh"

using namespace pg;

namespace {

constexpr int64_t kMaxGal = 131072;     // galaxies per call
constexpr int kMaxCellsPerSide = 40;    // cell list of at most 40^3 cells
constexpr int64_t kMaxCells = (int64_t)kMaxCellsPerSide * kMaxCellsPerSide * kMaxCellsPerSide;

constexpr size_t up256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kScanTmp = (size_t)((kMaxCells + 1 + 2047) / 2048 + 1);   // int64 values

// byte offsets of each scratch piece
constexpr size_t kOffX = 0;                                      // x, y, z  [kMaxGal] FP64
constexpr size_t kOffXs = kOffX + up256(24 * kMaxGal);           // sorted xs, ys, zs
constexpr size_t kOffCellId = kOffXs + up256(24 * kMaxGal);      // int32 [kMaxGal]
constexpr size_t kOffPerm = kOffCellId + up256(4 * kMaxGal);     // int32 [kMaxGal]
constexpr size_t kOffWs = kOffPerm + up256(4 * kMaxGal);         // float [kMaxGal]
constexpr size_t kOffCount = kOffWs + up256(4 * kMaxGal);        // int32 [kMaxCells + 1]
constexpr size_t kOffStart = kOffCount + up256(4 * (kMaxCells + 1));
constexpr size_t kOffCursor = kOffStart + up256(4 * (kMaxCells + 1));
constexpr size_t kOffTmp = kOffCursor + up256(4 * (kMaxCells + 1));
constexpr size_t kOffTot = kOffTmp + up256(8 * kScanTmp);
constexpr size_t kOffFlag = kOffTot + 256;                       // int32 non-finite flag
constexpr size_t kBytes = kOffFlag + 256;                        // about 8.4 MB

static __device__ __align__(256) unsigned char g_pair_scratch[kBytes];

// Device address of g_pair_scratch on the current device, looked up once per
// device (the symbol's host-side name is not a device address). The address
// is kept for the life of the process: it does not survive a reset of the
// device's primary context (cudaDeviceReset), after which the module and its
// array are loaded anew, so the entry point is not to be called on a device
// after a reset.
pg_status scratch_on_current_device(unsigned char** out) {
  static std::mutex mu;
  static void* addr[256] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return PG_ERR_CUDA;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pair_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      return PG_ERR_CUDA;
    }
    addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(addr[dev]);
  return PG_OK;
}

}  // namespace

extern "C" pg_status pg_pair_counts_static(int64_t n, const double* d_pos, const float* d_w,
                                           double box_L, int32_t n_s, const double* s_edges,
                                           int32_t n_mu, int64_t* d_dd, int64_t* d_ddq,
                                           void* stream) {
  if (n < 0 || !(box_L > 0.0) || !isfinite(box_L) || n_s < 1 || n_s > 64 || n_mu < 1 ||
      n_mu > 64 || !s_edges || !d_dd || !d_ddq || (n > 0 && !d_pos))
    return PG_ERR_INVALID_ARG;
  for (int i = 0; i < n_s; ++i)
    if (!(s_edges[i] < s_edges[i + 1]) || !(s_edges[0] >= 0.0)) return PG_ERR_INVALID_ARG;
  if (!(s_edges[n_s] < 0.5 * box_L)) return PG_ERR_INVALID_ARG;
  if (n > kMaxGal) return PG_ERR_CAPACITY;
  unsigned char* base = nullptr;
  pg_status st = scratch_on_current_device(&base);
  if (st != PG_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  PairGeom g;
  memset(&g, 0, sizeof(g));
  g.L = box_L;
  g.halfL = 0.5 * box_L;
  // cells per side, clamped in FP64 before the conversion (a tiny s_max
  // gives a ratio far above INT_MAX); larger cells stay correct
  const double ncr = floor(box_L / (s_edges[n_s] * (1.0 + 1e-9)));
  int nc = ncr > (double)kMaxCellsPerSide ? kMaxCellsPerSide : (int)ncr;
  if (nc < 3) nc = 1;
  g.nc = nc;
  g.cell_scale = (double)nc / box_L;
  g.n_s = n_s;
  g.n_mu = n_mu;
  for (int i = 0; i <= n_s; ++i) g.e2[i] = s_edges[i] * s_edges[i];

  double* x = reinterpret_cast<double*>(base + kOffX);
  double* xs = reinterpret_cast<double*>(base + kOffXs);
  CellList cl{reinterpret_cast<int32_t*>(base + kOffCellId),
              reinterpret_cast<int32_t*>(base + kOffCount),
              reinterpret_cast<int32_t*>(base + kOffStart),
              reinterpret_cast<int32_t*>(base + kOffCursor),
              reinterpret_cast<int32_t*>(base + kOffPerm),
              xs, xs + kMaxGal, xs + 2 * kMaxGal,
              reinterpret_cast<float*>(base + kOffWs),
              reinterpret_cast<int64_t*>(base + kOffTmp),
              reinterpret_cast<int64_t*>(base + kOffTot)};
  const size_t P = (size_t)n_s * n_mu;
  // positions holding NaN or Inf are refused, as in pg_forward: the flag is
  // read back before anything else is launched (one stream synchronisation)
  int32_t* flag = reinterpret_cast<int32_t*>(base + kOffFlag);
  int32_t hflag = 0;
  cudaError_t e = cudaMemsetAsync(flag, 0, 4, s);
  if (e == cudaSuccess) e = launch_check_finite(n, d_pos, flag, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && hflag) return PG_ERR_INVALID_ARG;
  if (e == cudaSuccess) e = cudaMemsetAsync(d_dd, 0, 8 * P, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_ddq, 0, 8 * P, s);
  if (e == cudaSuccess)
    e = launch_transform(n, box_L, 0.0, d_pos, nullptr, nullptr, x, x + kMaxGal, x + 2 * kMaxGal, s);
  if (e == cudaSuccess) e = launch_cells(g, n, x, x + kMaxGal, x + 2 * kMaxGal, d_w, cl, s);
  if (e == cudaSuccess) {
    PairOut po{};
    po.dd = reinterpret_cast<unsigned long long*>(d_dd);
    po.ddq = reinterpret_cast<unsigned long long*>(d_ddq);
    e = launch_pairs(g, n, cl, d_w != nullptr, false, po, s);
  }
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? PG_ERR_OOM : PG_ERR_CUDA;
  }
  return PG_OK;
}
