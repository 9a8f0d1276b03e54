// Positions (Sec. 3.2, eq. RSD) and pair enumeration (Sec. 2.1, Sec. 3.3).
//
// Every floating-point operation whose result decides an integer (a bin, a
// mesh node, a Q32.32 weight) is written with explicit round-to-nearest
// intrinsics in a fixed order, and this file is compiled with
// -fmad=false, so the pair lists and counts are bit-identical to any other
// IEEE FP64 evaluation of the same expressions.
#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double wrap_box(double v, double L) {
  // v - L*floor(v/L); a result of exactly L (rounding) becomes 0
  double r = __dsub_rn(v, __dmul_rn(L, floor(__ddiv_rn(v, L))));
  return r >= L ? 0.0 : r;
}

__global__ void __launch_bounds__(kThreads)
k_transform(int64_t n, double L, double rsd, const double* __restrict__ in,
            const float* __restrict__ vel, double* __restrict__ out,
            double* __restrict__ x, double* __restrict__ y, double* __restrict__ z) {
  int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  double a = wrap_box(in[3 * i + 0], L);
  double b = wrap_box(in[3 * i + 1], L);
  double c = wrap_box(in[3 * i + 2], L);
  if (rsd != 0.0 && vel) c = wrap_box(__dadd_rn(c, __dmul_rn(rsd, (double)vel[3 * i + 2])), L);
  if (out) { out[3 * i + 0] = a; out[3 * i + 1] = b; out[3 * i + 2] = c; }
  if (x) { x[i] = a; y[i] = b; z[i] = c; }
}

__global__ void __launch_bounds__(kThreads)
k_widen(int64_t n, const float* __restrict__ in, double* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}

__global__ void __launch_bounds__(kThreads)
k_check_finite(int64_t n, const double* __restrict__ aos, int32_t* flag) {
  int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= 3 * n) return;
  if (!isfinite(aos[i])) atomicOr(flag, 1);
}

// Sum w and sum w^2 in FP64: per-block partials, then one block reduces them.
__global__ void __launch_bounds__(kThreads)
k_wsum_partial(int64_t n, const float* __restrict__ w, double* __restrict__ partial) {
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    double v = w ? (double)w[i] : 1.0;
    s1 = __dadd_rn(s1, v);
    s2 = __dadd_rn(s2, __dmul_rn(v, v));
  }
  __shared__ double sh1[kThreads], sh2[kThreads];
  sh1[threadIdx.x] = s1; sh2[threadIdx.x] = s2;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh1[threadIdx.x] = __dadd_rn(sh1[threadIdx.x], sh1[threadIdx.x + o]);
      sh2[threadIdx.x] = __dadd_rn(sh2[threadIdx.x], sh2[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { partial[2 * blockIdx.x] = sh1[0]; partial[2 * blockIdx.x + 1] = sh2[0]; }
}

__global__ void __launch_bounds__(kThreads)
k_wsum_final(int nblk, const double* __restrict__ partial, double* __restrict__ out2) {
  __shared__ double sh1[kThreads], sh2[kThreads];
  double s1 = 0.0, s2 = 0.0;
  for (int i = threadIdx.x; i < nblk; i += kThreads) {
    s1 = __dadd_rn(s1, partial[2 * i]);
    s2 = __dadd_rn(s2, partial[2 * i + 1]);
  }
  sh1[threadIdx.x] = s1; sh2[threadIdx.x] = s2;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sh1[threadIdx.x] = __dadd_rn(sh1[threadIdx.x], sh1[threadIdx.x + o]);
      sh2[threadIdx.x] = __dadd_rn(sh2[threadIdx.x], sh2[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out2[0] = sh1[0]; out2[1] = sh2[0]; }
}

// ---- cell list: counting sort of galaxies into nc^3 cells of side >= s_max ---

__device__ __forceinline__ int cell_coord(double v, double scale, int nc) {
  int c = (int)floor(__dmul_rn(v, scale));
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void __launch_bounds__(kThreads)
k_cell_count(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
             const double* __restrict__ z, double scale, int nc, int32_t* __restrict__ cell_id,
             int32_t* __restrict__ count) {
  int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  int cx = cell_coord(x[i], scale, nc), cy = cell_coord(y[i], scale, nc), cz = cell_coord(z[i], scale, nc);
  int c = (cz * nc + cy) * nc + cx;
  cell_id[i] = c;
  atomicAdd(&count[c], 1);
}

__global__ void __launch_bounds__(kThreads)
k_cell_scatter(int64_t n, const int32_t* __restrict__ cell_id, int32_t* __restrict__ cursor,
               int32_t* __restrict__ perm) {
  int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (i >= n) return;
  int slot = atomicAdd(&cursor[cell_id[i]], 1);
  perm[slot] = (int32_t)i;
}

__global__ void __launch_bounds__(kThreads)
k_cell_gather(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ x,
              const double* __restrict__ y, const double* __restrict__ z,
              const float* __restrict__ w, double* __restrict__ xs, double* __restrict__ ys,
              double* __restrict__ zs, float* __restrict__ ws) {
  int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p >= n) return;
  int i = perm[p];
  xs[p] = x[i]; ys[p] = y[i]; zs[p] = z[i];
  if (w) ws[p] = w[i];
}

// ---- pair enumeration ---------------------------------------------------------

// The pair geometry (box, cells, squared s edges) travels by value as a kernel
// argument, so plans with different binning can run concurrently.

__device__ __forceinline__ double min_image(double d, double L, double h) {
  if (d > h) d = __dsub_rn(d, L);
  if (d < -h) d = __dadd_rn(d, L);
  return d;
}

struct PairHit {
  int bin;
  double mx, my, mz, wp;
  int i, j;
};

// Evaluates one unordered pair (orientation from input indices i < j).
__device__ __forceinline__ bool eval_pair(const PairGeom& g, const CellList& cl, bool use_w,
                                          int a, int b, PairHit& h) {
  int oa = cl.perm[a], ob = cl.perm[b];
  int pi = a, pj = b;
  if (oa > ob) { pi = b; pj = a; int t = oa; oa = ob; ob = t; }
  double xi = cl.xs[pi], yi = cl.ys[pi], zi = cl.zs[pi];
  double dx = min_image(__dsub_rn(cl.xs[pj], xi), g.L, g.halfL);
  double dy = min_image(__dsub_rn(cl.ys[pj], yi), g.L, g.halfL);
  double dz = min_image(__dsub_rn(cl.zs[pj], zi), g.L, g.halfL);
  int k = 0, m = 0;
  if (g.grid) {
    // (d_perp, d_par) grid: d_perp^2 = dx^2 + dy^2 against the squared
    // d_perp edges, d_par = |dz| against the d_par edges, half-open bins
    const double p2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    const double l = fabs(dz);
    if (p2 < g.e2[0] || !(p2 < g.e2[g.n_s]) || l < g.pe[0] || !(l < g.pe[g.n_mu])) return false;
    while (k + 1 < g.n_s && !(p2 < g.e2[k + 1])) ++k;
    while (m + 1 < g.n_mu && !(l < g.pe[m + 1])) ++m;
  } else {
    double s2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (s2 < g.e2[0] || !(s2 < g.e2[g.n_s])) return false;
    while (k + 1 < g.n_s && !(s2 < g.e2[k + 1])) ++k;
    double s = __dsqrt_rn(s2);
    double mu = s > 0.0 ? __ddiv_rn(fabs(dz), s) : 0.0;
    m = (int)floor(__dmul_rn((double)g.n_mu, mu));
    if (m > g.n_mu - 1) m = g.n_mu - 1;
  }
  h.bin = k * g.n_mu + m;
  h.mx = wrap_box(__dadd_rn(xi, __dmul_rn(0.5, dx)), g.L);
  h.my = wrap_box(__dadd_rn(yi, __dmul_rn(0.5, dy)), g.L);
  h.mz = wrap_box(__dadd_rn(zi, __dmul_rn(0.5, dz)), g.L);
  h.wp = use_w ? __dmul_rn((double)cl.ws[pi], (double)cl.ws[pj]) : 1.0;
  h.i = oa;
  h.j = ob;
  return true;
}

__device__ __forceinline__ unsigned long long q32(double w) {
  return (unsigned long long)__double2ll_rn(__dmul_rn(w, 4294967296.0));
}

// One thread per sorted galaxy a; candidates b > a in the 27 neighbouring
// cells (one cell when nc == 1). FILL: found pairs are compacted per warp
// with a ballot and appended with one atomic per warp and step.
template <bool FILL>
__global__ void __launch_bounds__(kThreads)
k_pairs(const __grid_constant__ PairGeom g, int64_t n, CellList cl, bool use_w, PairOut po,
        int use_smem_hist) {
  extern __shared__ unsigned long long hist[];   // [2 * P] when use_smem_hist
  const int P = g.n_s * g.n_mu;
  if (!FILL && use_smem_hist) {
    for (int t = threadIdx.x; t < 2 * P; t += blockDim.x) hist[t] = 0ull;
    __syncthreads();
  }
  const int64_t a = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool active = a < n;
  int cx = 0, cy = 0, cz = 0;
  if (active) {
    cx = cell_coord(cl.xs[a], g.cell_scale, g.nc);
    cy = cell_coord(cl.ys[a], g.cell_scale, g.nc);
    cz = cell_coord(cl.zs[a], g.cell_scale, g.nc);
  }
  const int nnb = g.nc == 1 ? 1 : 27;
  const int lane = threadIdx.x & 31;
  for (int t = 0; t < nnb; ++t) {
    int b0 = 0, b1 = 0;
    if (active) {
      int ox = 0, oy = 0, oz = 0;
      if (nnb == 27) { ox = t % 3 - 1; oy = (t / 3) % 3 - 1; oz = t / 9 - 1; }
      int nx = cx + ox, ny = cy + oy, nz = cz + oz;
      nx += (nx < 0) ? g.nc : (nx >= g.nc ? -g.nc : 0);
      ny += (ny < 0) ? g.nc : (ny >= g.nc ? -g.nc : 0);
      nz += (nz < 0) ? g.nc : (nz >= g.nc ? -g.nc : 0);
      int c = (nz * g.nc + ny) * g.nc + nx;
      b0 = cl.start[c];
      b1 = cl.start[c + 1];
      if (b0 < (int)a + 1) b0 = (int)a + 1;   // each unordered pair once: b > a
      if (b1 < b0) b1 = b0;
    }
    // iterate in lock step so that the warp can ballot
    int len = b1 - b0;
    int maxlen = len;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxlen = max(maxlen, __shfl_xor_sync(0xffffffffu, maxlen, o));
    for (int u = 0; u < maxlen; ++u) {
      PairHit h;
      bool hit = (u < len) && eval_pair(g, cl, use_w, (int)a, b0 + u, h);
      if (!FILL) {
        if (hit) {
          unsigned long long q = q32(h.wp);
          if (use_smem_hist) {
            atomicAdd(&hist[h.bin], 1ull);
            atomicAdd(&hist[P + h.bin], q);
          } else {
            atomicAdd(&po.dd[h.bin], 1ull);
            atomicAdd(&po.ddq[h.bin], q);
          }
        }
      } else {
        unsigned mask = __ballot_sync(0xffffffffu, hit);
        if (mask) {
          unsigned long long base = 0;
          int leader = __ffs(mask) - 1;
          if (lane == leader) base = atomicAdd(po.cursor, (unsigned long long)__popc(mask));
          base = __shfl_sync(0xffffffffu, base, leader);
          if (hit) {
            unsigned long long slot = base + __popc(mask & ((1u << lane) - 1u));
            if ((int64_t)slot < po.capacity) {
              po.bin[slot] = h.bin; po.i[slot] = h.i; po.j[slot] = h.j;
              po.mx[slot] = h.mx; po.my[slot] = h.my; po.mz[slot] = h.mz; po.wp[slot] = h.wp;
            }
          }
        }
      }
    }
  }
  if (!FILL && use_smem_hist) {
    __syncthreads();
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
      if (hist[t]) atomicAdd(&po.dd[t], hist[t]);
      if (hist[P + t]) atomicAdd(&po.ddq[t], hist[P + t]);
    }
  }
}

__global__ void __launch_bounds__(kThreads)
k_pair_scatter(int64_t np, PairOut po, unsigned long long* __restrict__ bin_cursor,
               int32_t* __restrict__ sbin, int32_t* __restrict__ si, int32_t* __restrict__ sj,
               double* __restrict__ smid, double* __restrict__ sx, double* __restrict__ sy,
               double* __restrict__ sz, double* __restrict__ sw) {
  int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (p >= np) return;
  int b = po.bin[p];
  unsigned long long slot = atomicAdd(&bin_cursor[b], 1ull);
  if (sbin) sbin[slot] = b;
  if (si) { si[slot] = po.i[p]; sj[slot] = po.j[p]; }
  if (smid) { smid[3 * slot] = po.mx[p]; smid[3 * slot + 1] = po.my[p]; smid[3 * slot + 2] = po.mz[p]; }
  if (sx) { sx[slot] = po.mx[p]; sy[slot] = po.my[p]; sz[slot] = po.mz[p]; }
  if (sw) sw[slot] = po.wp[p];
}

}  // namespace

cudaError_t launch_transform(int64_t n, double L, double rsd, const double* in_aos,
                             const float* vel, double* out_aos, double* x, double* y,
                             double* z, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_transform<<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(n, L, rsd, in_aos, vel, out_aos, x, y, z);
  return launched();
}

cudaError_t launch_widen_f32(int64_t n, const float* in, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_widen<<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(n, in, out);
  return launched();
}

cudaError_t launch_check_finite(int64_t n, const double* aos, int32_t* flag, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_check_finite<<<(unsigned)cdiv(3 * n, kThreads), kThreads, 0, s>>>(n, aos, flag);
  return launched();
}

cudaError_t launch_wsum(int64_t n, const float* w, double* partial, double* out2, cudaStream_t s) {
  int nblk = 256;
  k_wsum_partial<<<nblk, kThreads, 0, s>>>(n, w, partial);
  PG_CUDA_TRY(launched());
  k_wsum_final<<<1, kThreads, 0, s>>>(nblk, partial, out2);
  return launched();
}

cudaError_t launch_cells(const PairGeom& g, int64_t n, const double* x, const double* y,
                         const double* z, const float* w, CellList& cl, cudaStream_t s) {
  const int64_t ncell = (int64_t)g.nc * g.nc * g.nc;
  PG_CUDA_TRY(cudaMemsetAsync(cl.count, 0, sizeof(int32_t) * (ncell + 1), s));
  if (n > 0) {
    k_cell_count<<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(n, x, y, z, g.cell_scale, g.nc, cl.cell_id, cl.count);
    PG_CUDA_TRY(launched());
  }
  PG_CUDA_TRY(scan_i32_i32(cl.count, cl.start, ncell + 1, 1, cl.tot, cl.tmp, s));
  if (n > 0) {
    PG_CUDA_TRY(cudaMemcpyAsync(cl.cursor, cl.start, sizeof(int32_t) * ncell, cudaMemcpyDeviceToDevice, s));
    k_cell_scatter<<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(n, cl.cell_id, cl.cursor, cl.perm);
    PG_CUDA_TRY(launched());
    k_cell_gather<<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(n, cl.perm, x, y, z, w, cl.xs, cl.ys, cl.zs, cl.ws);
    PG_CUDA_TRY(launched());
  }
  return cudaSuccess;
}

cudaError_t launch_pairs(const PairGeom& g, int64_t n, const CellList& cl, bool use_w, bool fill,
                         PairOut& po, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  const int P = g.n_s * g.n_mu;
  unsigned grid = (unsigned)cdiv(n, kThreads);
  if (fill) {
    k_pairs<true><<<grid, kThreads, 0, s>>>(g, n, cl, use_w, po, 0);
  } else {
    size_t sm = sizeof(unsigned long long) * 2 * P;
    int use = sm <= 48 * 1024 ? 1 : 0;
    k_pairs<false><<<grid, kThreads, use ? sm : 0, s>>>(g, n, cl, use_w, po, use);
  }
  return launched();
}

cudaError_t launch_pair_scatter(int64_t np, const PairOut& po, unsigned long long* bin_cursor,
                                int32_t* sbin, int32_t* si, int32_t* sj, double* smid_aos,
                                double* sx, double* sy, double* sz, double* sw, cudaStream_t s) {
  if (np <= 0) return cudaSuccess;
  k_pair_scatter<<<(unsigned)cdiv(np, kThreads), kThreads, 0, s>>>(np, po, bin_cursor, sbin, si, sj,
                                                                    smid_aos, sx, sy, sz, sw);
  return launched();
}

}  // namespace pg
