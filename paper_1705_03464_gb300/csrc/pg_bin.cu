// (r, mu_r) binning of the correlation window and the ratio outputs.
//
// Binning (Sec. 2.1, eq. bpg_initial with W the indicator of one shell): every
// window cell belongs to at most one (r, mu_r) bin, and the plan holds, per
// bin, the sorted list of its cells plus one extra list for the aggregate
// support. The lists are cut into chunks of kBinChunk cells; one CTA sums one
// chunk of one mesh in FP64 (sum C and sum C^2) with a fixed warp-shuffle
// tree, and one thread per list adds its chunks in order, so the sums are
// deterministic. Chunking spreads the aggregate list (about half of all
// listed cells) over the whole GPU, whose FP64 rate is low.
//
// Ratios (Sec. 2.2 and Sec. 3.4): xi_pg, xi_gg, b_pg = xi_pg / xi_gg,
// xi(d_w) = sum C_gg^2 / sum C_gg (eq. xi_dw), xi(s, mu) = DD/RR - 1
// (eq. 2PCF_d_collapsed with the exact pair normalisation and the plan's bin
// volumes, (s, mu) shells or (d_perp, d_par) cells), Q_eff (eq. Qeff_notsq),
// the strict-squeezed Q_eff (eq. Qeff) and, on the grid, w(d_perp), all FP64.
#include <math.h>

#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kThreads = 256;

// First chunk index of list l and its chunk count (lists are cut into
// kBinChunk cells; the chunks of one list are consecutive).
__device__ __forceinline__ void chunk_of(const int64_t* __restrict__ list_off, int n_lists, int ci, int& l,
                                         int64_t& lo, int64_t& hi) {
  int first = 0;
  for (l = 0; l < n_lists; ++l) {
    const int64_t a = list_off[l], e = list_off[l + 1];
    const int nch = (int)((e - a + kBinChunk - 1) / kBinChunk);
    if (ci < first + nch) {
      lo = a + (int64_t)(ci - first) * kBinChunk;
      hi = min(e, lo + kBinChunk);
      return;
    }
    first += nch;
  }
  lo = hi = 0;
}

// One CTA per (chunk, mesh): FP64 sums of C and C^2 over the chunk's cells,
// reduced by a fixed warp-shuffle tree.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_bin_chunks(const R* __restrict__ Cwin, int64_t stride, const int32_t* __restrict__ cells,
             const int64_t* __restrict__ list_off, int n_lists, int n_chunks, double* __restrict__ part) {
  const int ci = blockIdx.x, b = blockIdx.y;
  const R* cw = Cwin + (int64_t)b * stride;
  int l;
  int64_t lo, hi;
  chunk_of(list_off, n_lists, ci, l, lo, hi);
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
    const double v = (double)cw[cells[i]];
    s1 += v;
    s2 = fma(v, v, s2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  __shared__ double w1[kThreads / 32], w2[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { w1[wid] = s1; w2[wid] = s2; }
  __syncthreads();
  if (wid == 0) {
    s1 = lane < kThreads / 32 ? w1[lane] : 0.0;
    s2 = lane < kThreads / 32 ? w2[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_down_sync(0xffffffffu, s1, o);
      s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
      part[((int64_t)b * n_chunks + ci) * 2] = s1;
      part[((int64_t)b * n_chunks + ci) * 2 + 1] = s2;
    }
  }
}

// One thread per (list, mesh): the list's chunk partials in chunk order.
__global__ void k_bin_combine(const int64_t* __restrict__ list_off, int n_lists, int n_chunks, int nb,
                              const double* __restrict__ part, double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_lists * nb) return;
  const int l = t % n_lists, b = t / n_lists;
  int first = 0;
  for (int k = 0; k < l; ++k) first += (int)((list_off[k + 1] - list_off[k] + kBinChunk - 1) / kBinChunk);
  const int nch = (int)((list_off[l + 1] - list_off[l] + kBinChunk - 1) / kBinChunk);
  double s1 = 0.0, s2 = 0.0;
  for (int k = 0; k < nch; ++k) {
    s1 += part[((int64_t)b * n_chunks + first + k) * 2];
    s2 += part[((int64_t)b * n_chunks + first + k) * 2 + 1];
  }
  out[((int64_t)b * n_lists + l) * 2] = s1;
  out[((int64_t)b * n_lists + l) * 2 + 1] = s2;
}

__device__ __forceinline__ double q_notsq(double b, double xi, double xw) {
  // eq. Qeff_notsq
  return ((1.0 + xi) * b - 2.0 - xw / (2.0 * xi)) / (2.0 * xi + 1.5 * xw);
}
__device__ __forceinline__ double q_sq(double b, double xi) {
  // eq. Qeff
  return ((1.0 + xi) * b - 2.0) / (2.0 * xi);
}

__global__ void __launch_bounds__(kThreads) k_ratios(RatioArgs a) {
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const int P = a.P, Q = a.Q, L = Q + 1;
  const double sw = a.wsum[0], sw2 = a.wsum[1];
  const double npairs = 0.5 * (sw * sw - sw2);
  const double L3 = a.L * a.L * a.L;
  // per pair bin: counts and xi(s, mu) (or xi(d_perp, d_par))
  for (int p = threadIdx.x; p < P; p += kThreads) {
    const double rr = npairs * a.vbin[p] / L3;
    const double ddw = (double)(long long)a.ddq[p] * (1.0 / 4294967296.0);
    if (a.o_dd) a.o_dd[p] = (int64_t)a.dd[p];
    if (a.dd_w) a.dd_w[p] = ddw;
    if (a.xi_ss) a.xi_ss[p] = rr > 0.0 ? ddw / rr - 1.0 : nan;
  }
  // grid: w(d_perp) = sum over the d_par bins of wcoef * xi, in bin order
  if (a.w_perp) {
    for (int k = threadIdx.x; k < a.n_s; k += kThreads) {
      double wp = a.wcoef ? 0.0 : nan;
      for (int m = 0; m < a.n_mu && a.wcoef; ++m) {
        const int p = k * a.n_mu + m;
        const double rr = npairs * a.vbin[p] / L3;
        const double ddw = (double)(long long)a.ddq[p] * (1.0 / 4294967296.0);
        wp += a.wcoef[p] * (rr > 0.0 ? ddw / rr - 1.0 : nan);
      }
      a.w_perp[k] = wp;
    }
  }
  // per correlation bin: galaxy terms
  for (int q = threadIdx.x; q <= Q; q += kThreads) {
    const int64_t n = a.list_off[q + 1] - a.list_off[q];
    const double s1 = a.gg_valid ? a.sum_gg[2 * q] : nan;
    const double s2 = a.gg_valid ? a.sum_gg[2 * q + 1] : nan;
    if (q < Q) {
      if (a.n_cells) a.n_cells[q] = n;
      if (a.xi_gg) a.xi_gg[q] = n > 0 ? s1 / (double)n : nan;
      if (a.xi_dw) a.xi_dw[q] = s2 / s1;
      if (a.o_sum_gg) a.o_sum_gg[q] = s1;
      if (a.o_sum2_gg) a.o_sum2_gg[q] = s2;
    } else {
      if (a.n_cells_agg) *a.n_cells_agg = n;
      if (a.xi_dw_agg) *a.xi_dw_agg = s2 / s1;
      if (a.o_sum_gg_agg) { a.o_sum_gg_agg[0] = s1; a.o_sum_gg_agg[1] = s2; }
    }
  }
  // per (pair bin, correlation bin)
  for (int t = threadIdx.x; t < P * L; t += kThreads) {
    const int p = t / L, q = t % L;
    const double ddw = (double)(long long)a.ddq[p] * (1.0 / 4294967296.0);
    const double rr = npairs * a.vbin[p] / L3;
    const double xi = rr > 0.0 ? ddw / rr - 1.0 : nan;
    const double sp = a.pg_valid[p] ? a.sum_pg[((int64_t)p * L + q) * 2] : nan;
    const double sg = a.gg_valid ? a.sum_gg[2 * q] : nan;
    const double s2g = a.gg_valid ? a.sum_gg[2 * q + 1] : nan;
    const double xw = s2g / sg;
    if (q < Q) {
      const int64_t n = a.list_off[q + 1] - a.list_off[q];
      const double xpg = n > 0 ? sp / (double)n : nan;
      const double xgg = n > 0 ? sg / (double)n : nan;
      const double b = xpg / xgg;
      const int64_t o = (int64_t)p * Q + q;
      if (a.o_sum_pg) a.o_sum_pg[o] = sp;
      if (a.xi_pg) a.xi_pg[o] = xpg;
      if (a.b_pg) a.b_pg[o] = b;
      if (a.q_eff) a.q_eff[o] = q_notsq(b, xi, xw);
      if (a.q_eff_sq) a.q_eff_sq[o] = q_sq(b, xi);
    } else {
      const double b = sp / sg;
      if (a.o_sum_pg_agg) a.o_sum_pg_agg[p] = sp;
      if (a.b_pg_agg) a.b_pg_agg[p] = b;
      if (a.q_eff_agg) a.q_eff_agg[p] = q_notsq(b, xi, xw);
    }
  }
}

}  // namespace

template <typename R>
cudaError_t launch_bin_sums(int nb, int n_lists, const R* Cwin, int64_t Cwin_stride,
                            const int32_t* cells, const int64_t* list_off, int n_chunks, double* part,
                            double* out, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  if (n_chunks > 0) {
    dim3 g(n_chunks, nb);
    k_bin_chunks<R><<<g, kThreads, 0, s>>>(Cwin, Cwin_stride, cells, list_off, n_lists, n_chunks, part);
    PG_CUDA_TRY(launched());
  }
  const int nt = n_lists * nb;
  k_bin_combine<<<(unsigned)cdiv(nt, 128), 128, 0, s>>>(list_off, n_lists, n_chunks, nb, part, out);
  return launched();
}
template cudaError_t launch_bin_sums<float>(int, int, const float*, int64_t, const int32_t*,
                                            const int64_t*, int, double*, double*, cudaStream_t);
template cudaError_t launch_bin_sums<double>(int, int, const double*, int64_t, const int32_t*,
                                             const int64_t*, int, double*, double*, cudaStream_t);

cudaError_t launch_ratios(const RatioArgs& a, cudaStream_t s) {
  k_ratios<<<1, kThreads, 0, s>>>(a);
  return launched();
}

}  // namespace pg
