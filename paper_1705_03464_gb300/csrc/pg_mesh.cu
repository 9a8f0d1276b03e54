// Mass assignment (Sec. 3.5: NGP, CIC or the paper's TSC) into compact
// x-lines of Q32.32 int64 nodes.
//
// A pair bin touches few mesh lines (Sec. 2.1: a pair field is a sum of
// deltas at the pair midpoints), so each bin's mesh is stored as the list of
// (y, z) lines it touches: the lines are flagged, an exclusive scan of the
// flags numbers them, and the deposit adds llrint(((w*wx)*wy)*wz*2^32) to the
// node with a 64-bit integer atomic. Integer sums make every mesh exact and
// independent of the order of the atomics. Compiled with -fmad=false.
#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBatch = 64;   // bins whose totals are summed in shared memory

struct Foot {
  int ix[3], iy[3], iz[3];
  double wx[3], wy[3], wz[3];
  int n;  // nodes per axis: 1 (NGP), 2 (CIC), 3 (TSC)
};

__device__ __forceinline__ void footprint(const DepGeom& g, double x, double y, double z, Foot& f) {
  f.n = axis_nodes(g, __ddiv_rn(x, g.dx), f.ix, f.wx);
  axis_nodes(g, __ddiv_rn(y, g.dx), f.iy, f.wy);
  axis_nodes(g, __ddiv_rn(z, g.dx), f.iz, f.wz);
}

__device__ __forceinline__ unsigned long long node_q(const DepGeom& g, double w, double wx,
                                                     double wy, double wz) {
  double v = (g.assign == 0) ? w : __dmul_rn(__dmul_rn(__dmul_rn(w, wx), wy), wz);
  return (unsigned long long)__double2ll_rn(__dmul_rn(v, 4294967296.0));
}

// The mesh geometry travels by value as a kernel argument, so plans with
// different meshes can run concurrently on separate streams.

__global__ void __launch_bounds__(kThreads)
k_mark_lines(DepGeom g, int64_t n, const double* __restrict__ x, const double* __restrict__ y,
             const double* __restrict__ z, const int32_t* __restrict__ pbin, int bin0,
             uint8_t* __restrict__ flags) {
  int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p >= n) return;
  Foot f;
  footprint(g, x[p], y[p], z[p], f);
  const int b = pbin ? pbin[p] - bin0 : 0;
  uint8_t* fl = flags + (int64_t)b * g.N * g.N;
  for (int cz = 0; cz < f.n; ++cz)
    for (int cy = 0; cy < f.n; ++cy) fl[(int64_t)f.iz[cz] * g.N + f.iy[cy]] = 1;
}

__global__ void __launch_bounds__(kThreads)
k_line_compact(int N, int nb, const uint8_t* __restrict__ flags, const int32_t* __restrict__ idx,
               const int64_t* __restrict__ line_base, int32_t* __restrict__ line_y,
               int32_t* __restrict__ line_bin, int32_t* __restrict__ line_z) {
  const int64_t NN = (int64_t)N * N;
  int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (t >= NN * nb) return;
  if (!flags[t]) return;
  int b = (int)(t / NN);
  int64_t zy = t - (int64_t)b * NN;
  int64_t l = line_base[b] + idx[t];
  line_y[l] = (int32_t)(zy % N);
  line_bin[l] = b;
  if (line_z) line_z[l] = (int32_t)(zy / N);
}

__global__ void k_line_bases(int nb, const int64_t* __restrict__ seg_total,
                             int64_t* __restrict__ line_base, int64_t* __restrict__ total) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t run = 0;
  for (int b = 0; b < nb; ++b) { line_base[b] = run; run += seg_total[b]; }
  *total = run;
}

__global__ void __launch_bounds__(kThreads)
k_deposit_lines(DepGeom g, int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                const double* __restrict__ z, const double* __restrict__ w,
                const int32_t* __restrict__ pbin, int bin0, const int32_t* __restrict__ idx,
                const int64_t* __restrict__ line_base, unsigned long long* __restrict__ lines_q,
                unsigned long long* __restrict__ qsum) {
  __shared__ unsigned long long sh_q[kMaxBatch];
  for (int t = threadIdx.x; t < kMaxBatch; t += kThreads) sh_q[t] = 0ull;
  __syncthreads();
  int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p < n) {
    Foot f;
    footprint(g, x[p], y[p], z[p], f);
    const int b = pbin ? pbin[p] - bin0 : 0;
    const double wp = w ? w[p] : 1.0;
    const int64_t NN = (int64_t)g.N * g.N;
    unsigned long long mine = 0ull;
    for (int cz = 0; cz < f.n; ++cz)
      for (int cy = 0; cy < f.n; ++cy) {
        int64_t zy = (int64_t)f.iz[cz] * g.N + f.iy[cy];
        int64_t line = line_base[b] + idx[(int64_t)b * NN + zy];
        unsigned long long* row = lines_q + line * g.N;
        for (int cx = 0; cx < f.n; ++cx) {
          unsigned long long q = node_q(g, wp, f.wx[cx], f.wy[cy], f.wz[cz]);
          if (q) atomicAdd(&row[f.ix[cx]], q);
          mine += q;
        }
      }
    // mesh total (rho_bar) per bin: block-local integer sums, then one global add
    if (b < kMaxBatch) atomicAdd(&sh_q[b], mine);
    else atomicAdd(&qsum[b], mine);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kMaxBatch; t += kThreads)
    if (sh_q[t]) atomicAdd(&qsum[t], sh_q[t]);
}

__global__ void __launch_bounds__(kThreads)
k_deposit_dense(DepGeom g, int64_t n, const double* __restrict__ aos, const double* __restrict__ w,
                unsigned long long* __restrict__ mesh) {
  int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p >= n) return;
  Foot f;
  footprint(g, aos[3 * p], aos[3 * p + 1], aos[3 * p + 2], f);
  const double wp = w ? w[p] : 1.0;
  for (int cz = 0; cz < f.n; ++cz)
    for (int cy = 0; cy < f.n; ++cy)
      for (int cx = 0; cx < f.n; ++cx) {
        unsigned long long q = node_q(g, wp, f.wx[cx], f.wy[cy], f.wz[cz]);
        int64_t node = ((int64_t)f.iz[cz] * g.N + f.iy[cy]) * g.N + f.ix[cx];
        if (q) atomicAdd(&mesh[node], q);
      }
}

// Sets *bad when a mesh index lies outside [0, nb) (checked before a deposit
// that takes caller-supplied indices).
__global__ void __launch_bounds__(kThreads)
k_check_bins(int64_t n, const int32_t* __restrict__ bin, int nb, int32_t* bad) {
  int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p < n && (bin[p] < 0 || bin[p] >= nb)) atomicOr(bad, 1);
}

// Compact lines back into dense meshes mesh[bin][z][y][x] (the stage entry
// point that exposes the deposit's own output); one thread per node.
__global__ void __launch_bounds__(kThreads)
k_lines_scatter(int N, int64_t n_lines, const unsigned long long* __restrict__ lines_q,
                const int32_t* __restrict__ line_y, const int32_t* __restrict__ line_z,
                const int32_t* __restrict__ line_bin, unsigned long long* __restrict__ mesh) {
  int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (t >= n_lines * N) return;
  const int64_t l = t / N;
  const int x = (int)(t - l * N);
  const int64_t node = (((int64_t)line_bin[l] * N + line_z[l]) * N + line_y[l]) * N + x;
  mesh[node] = lines_q[t];
}

// f = rho / rho_bar = q * N^3 / Q per mesh (FP64); 0 when the mesh is empty.
__global__ void k_field_scale(int nb, const unsigned long long* __restrict__ qsum, double n3,
                              double* __restrict__ scale) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  long long Q = (long long)qsum[b];
  scale[b] = Q > 0 ? n3 / (double)Q : 0.0;
}

}  // namespace

cudaError_t launch_mark_lines(const DepGeom& g, int64_t n, const double* x, const double* y,
                              const double* z, const int32_t* pbin, int bin0, uint8_t* flags,
                              cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_mark_lines<<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(g, n, x, y, z, pbin, bin0, flags);
  return launched();
}

cudaError_t launch_line_compact(int N, int nb, const uint8_t* flags, const int32_t* idx,
                                const int64_t* line_base, int32_t* line_y, int32_t* line_bin,
                                int32_t* line_z,
                                cudaStream_t s) {
  int64_t tot = (int64_t)N * N * nb;
  k_line_compact<<<(unsigned)cdiv(tot, kThreads), kThreads, 0, s>>>(N, nb, flags, idx, line_base, line_y, line_bin,
                                                                       line_z);
  return launched();
}

cudaError_t launch_line_bases(int nb, const int64_t* seg_total, int64_t* line_base,
                              int64_t* n_lines_total, cudaStream_t s) {
  k_line_bases<<<1, 32, 0, s>>>(nb, seg_total, line_base, n_lines_total);
  return launched();
}

cudaError_t launch_deposit_lines(const DepGeom& g, int64_t n, const double* x, const double* y,
                                 const double* z, const double* w, const int32_t* pbin, int bin0,
                                 const int32_t* idx, const int64_t* line_base,
                                 unsigned long long* lines_q, unsigned long long* qsum,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_deposit_lines<<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(g, n, x, y, z, w, pbin, bin0, idx,
                                                                     line_base, lines_q, qsum);
  return launched();
}

cudaError_t launch_deposit_dense(const DepGeom& g, int64_t n, const double* aos, const double* w,
                                 unsigned long long* mesh, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_deposit_dense<<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(g, n, aos, w, mesh);
  return launched();
}

cudaError_t launch_check_bins(int64_t n, const int32_t* bin, int nb, int32_t* bad, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_check_bins<<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(n, bin, nb, bad);
  return launched();
}

cudaError_t launch_lines_scatter(int N, int64_t n_lines, const unsigned long long* lines_q,
                                const int32_t* line_y, const int32_t* line_z,
                                const int32_t* line_bin, unsigned long long* mesh,
                                cudaStream_t s) {
  if (n_lines <= 0) return cudaSuccess;
  k_lines_scatter<<<(unsigned)cdiv(n_lines * N, kThreads), kThreads, 0, s>>>(
      N, n_lines, lines_q, line_y, line_z, line_bin, mesh);
  return launched();
}

cudaError_t launch_field_scale(int nb, const unsigned long long* qsum, int N, double* scale,
                               cudaStream_t s) {
  double n3 = (double)N * (double)N * (double)N;
  k_field_scale<<<(unsigned)cdiv(nb, 64), 64, 0, s>>>(nb, qsum, n3, scale);
  return launched();
}

}  // namespace pg
