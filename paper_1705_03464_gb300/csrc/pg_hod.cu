// HOD-parameter derivatives of the pair-count statistics (Sec. 5, the
// coefficients of the emulators of eqs. 2pf_emulate_1st / 2pf_emulate_2nd).
//
// With soft occupation weights (eq. hod) on fixed candidates, DD_b (the sum
// over the pairs of bin b of w_i w_j) and R = ((sum w)^2 - sum w^2)/2 are
// polynomials in the weights, so their first and second derivatives in theta
// follow exactly from dw/dtheta and d2w/dtheta2 by the product rule, in one
// pass over the pairs and one over the galaxies. xi_b = DD_b / (R V_b/L^3) - 1
// (eq. 2PCF_d_collapsed) follows by the quotient rule and w(d_perp) (eq.
// 2PCF_los_integrated_explicit) by linearity. All sums are FP64 in a fixed
// order (deterministic).
#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kT = 5;          // parameters
constexpr int kT2 = 15;        // second derivatives, j <= k
constexpr int kV = kHodVals;   // 1 + 5 + 15
constexpr int kThr = 128;

__device__ __forceinline__ int tri(int j, int k) {   // j <= k
  return j * kT - (j * (j - 1)) / 2 + (k - j);
}

// Block tree reduction of vals[kNv] over kThr threads in shared memory;
// thread 0 receives the sums in red[v][0].
template <int kNv>
__device__ __forceinline__ void block_sum(double (&vals)[kNv], double (*red)[kThr]) {
  for (int v = 0; v < kNv; ++v) red[v][threadIdx.x] = vals[v];
  __syncthreads();
  for (int o = kThr / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int v = 0; v < kNv; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + o];
    __syncthreads();
  }
}

// sum w and sum w^2 with derivatives; grid-stride over galaxies, one block
// partial per block (fixed grid, so a fixed summation order).
__global__ void __launch_bounds__(kThr)
k_hod_norm_partial(int64_t n, const float* __restrict__ w, const double* __restrict__ dw,
                   const double* __restrict__ d2w, double* __restrict__ partial) {
  __shared__ double red[2 * kV][kThr];
  double a[2 * kV];
  for (int v = 0; v < 2 * kV; ++v) a[v] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kThr + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThr) {
    const double wi = (double)w[i];
    double d[kT];
    for (int j = 0; j < kT; ++j) d[j] = dw[kT * i + j];
    a[0] += wi;
    a[kV] += wi * wi;
    for (int j = 0; j < kT; ++j) {
      a[1 + j] += d[j];
      a[kV + 1 + j] += 2.0 * wi * d[j];
    }
    for (int j = 0; j < kT; ++j)
      for (int k = j; k < kT; ++k) {
        const int t = tri(j, k);
        const double h = d2w[kT2 * i + t];
        a[1 + kT + t] += h;
        a[kV + 1 + kT + t] += 2.0 * (d[j] * d[k] + wi * h);
      }
  }
  block_sum<2 * kV>(a, red);
  if (threadIdx.x < 2 * kV) partial[(int64_t)blockIdx.x * 2 * kV + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_hod_norm_final(int nblk, const double* __restrict__ partial, double* __restrict__ out) {
  const int v = threadIdx.x;
  if (v >= 2 * kV) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * 2 * kV + v];
  out[v] = s;
}

// One block per chunk of a bin's pairs (chunk c covers [cs[c], cs[c] +
// kHodChunk) clipped to its bin's end ce[c]): partial sums of DD = sum w_i w_j
// and its derivatives d_j = w_i' w_j + w_i w_j',
// d_jk = w_i'' w_j + w_i^j w_j^k + w_i^k w_j^j + w_i w_j''.
__global__ void __launch_bounds__(kThr)
k_hod_pair_sums(const int64_t* __restrict__ cs, const int64_t* __restrict__ ce,
                const int32_t* __restrict__ pi, const int32_t* __restrict__ pj,
                const float* __restrict__ w, const double* __restrict__ dw,
                const double* __restrict__ d2w, double* __restrict__ partial) {
  __shared__ double red[kV][kThr];
  const int64_t ch = blockIdx.x;
  const int64_t p0 = cs[ch], p1 = ce[ch];
  double a[kV];
  for (int v = 0; v < kV; ++v) a[v] = 0.0;
  for (int64_t p = p0 + threadIdx.x; p < p1; p += kThr) {
    const int64_t i = pi[p], j = pj[p];
    const double wi = (double)w[i], wj = (double)w[j];
    double di[kT], dj[kT];
    for (int t = 0; t < kT; ++t) { di[t] = dw[kT * i + t]; dj[t] = dw[kT * j + t]; }
    a[0] += wi * wj;
    for (int t = 0; t < kT; ++t) a[1 + t] += di[t] * wj + wi * dj[t];
    for (int t = 0; t < kT; ++t)
      for (int u = t; u < kT; ++u) {
        const int q = tri(t, u);
        a[1 + kT + q] += d2w[kT2 * i + q] * wj + di[t] * dj[u] + di[u] * dj[t] + wi * d2w[kT2 * j + q];
      }
  }
  block_sum<kV>(a, red);
  if (threadIdx.x < kV) partial[ch * kV + threadIdx.x] = red[threadIdx.x][0];
}

// Per bin b, the sum of its chunks [c0[b], c0[b+1]) in order: out[P][21].
__global__ void k_hod_pair_final(int P, const int64_t* __restrict__ c0, const double* __restrict__ partial,
                                 double* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P * kV) return;
  const int b = t / kV, v = t - b * kV;
  double s = 0.0;
  for (int64_t c = c0[b]; c < c0[b + 1]; ++c) s += partial[c * kV + v];
  out[t] = s;
}

// One thread per pair bin: q = DD / E, E = R c with c = V_b / L^3,
// dq_j = (dDD_j - q dE_j) / E, d2q_jk = (d2DD_jk - dq_j dE_k - dq_k dE_j - q d2E_jk) / E.
__global__ void k_hod_xi(int P, const double* __restrict__ dd, const double* __restrict__ norm,
                         const double* __restrict__ vbin, double inv_L3, double* __restrict__ xi) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P) return;
  const double* s1 = norm;        // sum w
  const double* s2 = norm + kV;   // sum w^2
  const double c = vbin[b] * inv_L3;
  double E = 0.5 * (s1[0] * s1[0] - s2[0]) * c;
  double dE[kT], d2E[kT2];
  for (int j = 0; j < kT; ++j) dE[j] = (s1[0] * s1[1 + j] - 0.5 * s2[1 + j]) * c;
  for (int j = 0; j < kT; ++j)
    for (int k = j; k < kT; ++k) {
      const int t = tri(j, k);
      d2E[t] = (s1[1 + j] * s1[1 + k] + s1[0] * s1[1 + kT + t] - 0.5 * s2[1 + kT + t]) * c;
    }
  const double* D = dd + (int64_t)b * kV;
  double* o = xi + (int64_t)b * kV;
  const double q = D[0] / E;
  double dq[kT];
  for (int j = 0; j < kT; ++j) dq[j] = (D[1 + j] - q * dE[j]) / E;
  o[0] = q - 1.0;
  for (int j = 0; j < kT; ++j) o[1 + j] = dq[j];
  for (int j = 0; j < kT; ++j)
    for (int k = j; k < kT; ++k) {
      const int t = tri(j, k);
      o[1 + kT + t] = (D[1 + kT + t] - dq[j] * dE[k] - dq[k] * dE[j] - q * d2E[t]) / E;
    }
}

// w(d_perp)_k and its derivatives: the fixed combination of the d_par bins.
__global__ void k_hod_wperp(int n_s, int n_mu, const double* __restrict__ xi,
                            const double* __restrict__ wcoef, double* __restrict__ wp) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_s * kV) return;
  const int k = t / kV, v = t - k * kV;
  double s = 0.0;
  for (int m = 0; m < n_mu; ++m) s += wcoef[k * n_mu + m] * xi[(int64_t)(k * n_mu + m) * kV + v];
  wp[t] = s;
}

}  // namespace

cudaError_t launch_hod_norm(int64_t n, const float* w, const double* dw, const double* d2w,
                            double* partial, double* out, cudaStream_t s) {
  k_hod_norm_partial<<<kHodNormBlocks, kThr, 0, s>>>(n, w, dw, d2w, partial);
  PG_CUDA_TRY(launched());
  k_hod_norm_final<<<1, 64, 0, s>>>(kHodNormBlocks, partial, out);
  return launched();
}

cudaError_t launch_hod_pair_sums(int P, int64_t n_chunks, const int64_t* chunks, const int32_t* pi,
                                 const int32_t* pj, const float* w, const double* dw,
                                 const double* d2w, double* partial, double* out, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  const int64_t* cs = chunks;
  const int64_t* ce = chunks + n_chunks;
  const int64_t* c0 = chunks + 2 * n_chunks;
  if (n_chunks > 0) {
    k_hod_pair_sums<<<(unsigned)n_chunks, kThr, 0, s>>>(cs, ce, pi, pj, w, dw, d2w, partial);
    PG_CUDA_TRY(launched());
  }
  k_hod_pair_final<<<(unsigned)cdiv(P * kV, 128), 128, 0, s>>>(P, c0, partial, out);
  return launched();
}

cudaError_t launch_hod_xi(int n_s, int n_mu, const double* dd, const double* norm,
                          const double* vbin, const double* wcoef, double inv_L3, double* xi,
                          double* wp, cudaStream_t s) {
  const int P = n_s * n_mu;
  k_hod_xi<<<(unsigned)cdiv(P, 64), 64, 0, s>>>(P, dd, norm, vbin, inv_L3, xi);
  PG_CUDA_TRY(launched());
  if (!wcoef || !wp) return cudaSuccess;
  k_hod_wperp<<<(unsigned)cdiv(n_s * kV, 64), 64, 0, s>>>(n_s, n_mu, xi, wcoef, wp);
  return launched();
}

}  // namespace pg
