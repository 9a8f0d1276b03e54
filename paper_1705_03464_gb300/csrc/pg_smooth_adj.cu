// Adjoint of the smooth-W estimator (reverse sweep of Sec. 2.1 eq. bpg_final
// with the W of Sec. 3.6 eq. weighting, eqs. xi_dw, Qeff_notsq,
// 2PCF_d_collapsed) with respect to the galaxy weights. pg_api.cu orders the
// launches: ratio adjoints -> pair terms and their weight chain -> the
// adjoint weights at the points deposited on a mesh (the transpose of the
// interpolation) -> W convolution and the xi_w term in k space -> the rho / Q
// normalisation at the galaxies.
#include <math.h>

#include <algorithm>

#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float ex(float v) { return expf(v); }
__device__ __forceinline__ double ex(double v) { return exp(v); }
__device__ __forceinline__ float sq(float v) { return sqrtf(v); }
__device__ __forceinline__ double sq(double v) { return sqrt(v); }

__device__ __forceinline__ double fin_or_zero(double g, double v) { return isfinite(v) ? g : 0.0; }

// One block: per-bin adjoints of num, xi and the scalars den, xi_w, npairs,
// each scalar a fixed-order block reduction.
__global__ void __launch_bounds__(kThreads) k_sadj_ratios(SmoothAdjArgs a) {
  __shared__ double r0[kThreads], r1[kThreads], r2[kThreads];
  const int P = a.P;
  const double* xs = a.out;
  const double* num = a.out + P;
  const double* bp = a.out + 2 * P;
  const double* qe = a.out + 3 * P;
  const double den = a.out[4 * P], xw = a.out[4 * P + 1];
  const double* gxs = a.g;
  const double* gnum = a.g + P;
  const double* gb = a.g + 2 * P;
  const double* gq = a.g + 3 * P;
  const double sw = a.wsum[0], sw2 = a.wsum[1];
  const double npairs = 0.5 * (sw * sw - sw2);
  const double L3 = a.L * a.L * a.L;
  double xwc = 0.0, denc = 0.0, npbc = 0.0;
  for (int p = threadIdx.x; p < P; p += kThreads) {
    const double x = xs[p], b = bp[p];
    double bbar = fin_or_zero(gb[p], b);
    double xsbar = fin_or_zero(gxs[p], x);
    const double g_q = fin_or_zero(gq[p], qe[p]);
    if (g_q != 0.0) {   // eq. Qeff_notsq: q = n / D
      const double D = 2.0 * x + 1.5 * xw;
      const double n = (1.0 + x) * b - 2.0 - xw / (2.0 * x);
      bbar += g_q * (1.0 + x) / D;
      xsbar += g_q * ((b + xw / (2.0 * x * x)) / D - 2.0 * n / (D * D));
      xwc += g_q * ((-1.0 / (2.0 * x)) / D - 1.5 * n / (D * D));
    }
    double numbar = 0.0;
    if (isfinite(num[p])) {   // b = num / den
      numbar = fin_or_zero(gnum[p], num[p]) + bbar / den;
      denc += -bbar * num[p] / (den * den);
    }
    const double rr = npairs * a.vbin[p] / L3;
    const double dd = (double)(long long)a.ddq[p] * (1.0 / 4294967296.0);
    if (rr > 0.0) npbc += -xsbar * dd / (rr * rr) * a.vbin[p] / L3;
    a.sa[p] = numbar;
    a.sa[P + p] = xsbar;
    a.sa[2 * P + p] = rr;
  }
  r0[threadIdx.x] = xwc;
  r1[threadIdx.x] = denc;
  r2[threadIdx.x] = npbc;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      r0[threadIdx.x] += r0[threadIdx.x + o];
      r1[threadIdx.x] += r1[threadIdx.x + o];
      r2[threadIdx.x] += r2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.sa[3 * P] = fin_or_zero(a.g[4 * P], den) + r1[0];        // den bar
    a.sa[3 * P + 1] = fin_or_zero(a.g[4 * P + 1], xw) + r0[0];  // xi_w bar
    a.sa[3 * P + 2] = r2[0];                                     // npairs bar
  }
}

// Pair k of bin b: its direct weight adjoint (the bin mean and DD), the
// adjoint weight of its interpolated G, and the chain w_p = w_i w_j.
__global__ void __launch_bounds__(kThreads)
k_sadj_pairs(int64_t np, int P, const int32_t* __restrict__ pbin, const double* __restrict__ pw,
             const double* __restrict__ gp, const int32_t* __restrict__ pi, const int32_t* __restrict__ pj,
             const double* __restrict__ wgal, const double* __restrict__ psums, const double* __restrict__ out,
             const double* __restrict__ sa, double* __restrict__ gpbar, double* __restrict__ wbar) {
  const int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (k >= np) return;
  const int b = pbin[k];
  const double Wb = psums[2 * b + 1], numb = out[P + b];
  const double numbar = sa[b], xsbar = sa[P + b], rr = sa[2 * P + b];
  double wpbar = 0.0, gb = 0.0;
  if (Wb > 0.0) {
    wpbar = numbar * (gp[k] - numb) / Wb;
    gb = numbar * pw[k] / Wb;
  }
  if (rr > 0.0) wpbar += xsbar / rr;
  gpbar[k] = gb;
  const int i = pi[k], j = pj[k];
  const double wi = wgal ? wgal[i] : 1.0, wj = wgal ? wgal[j] : 1.0;
  atomicAdd(&wbar[i], wpbar * wj);
  atomicAdd(&wbar[j], wpbar * wi);
}

// Adjoint weight of G at galaxy k: den bar * w_k / sum w.
__global__ void __launch_bounds__(kThreads)
k_sadj_gbar(int64_t n, int P, const double* __restrict__ sa, const double* __restrict__ gal,
            const double* __restrict__ wgal, double* __restrict__ gjbar) {
  const int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (k >= n) return;
  gjbar[k] = sa[3 * P] * (wgal ? wgal[k] : 1.0) / gal[1];
}

// The transpose of the interpolation: v_k times the assignment weights of
// point k, added to a dense [z][y][x] mesh.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_scatter(DepGeom geo, int64_t n, const double* __restrict__ x, const double* __restrict__ y,
          const double* __restrict__ z, const double* __restrict__ v, R* __restrict__ mesh) {
  const int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (k >= n) return;
  const double vk = v[k];
  if (vk == 0.0) return;
  const int N = geo.N;
  int ix[3], iy[3], iz[3];
  double kx[3], ky[3], kz[3];
  const int nn = axis_nodes(geo, __ddiv_rn(x[k], geo.dx), ix, kx);
  axis_nodes(geo, __ddiv_rn(y[k], geo.dx), iy, ky);
  axis_nodes(geo, __ddiv_rn(z[k], geo.dx), iz, kz);
  for (int cz = 0; cz < nn; ++cz)
    for (int cy = 0; cy < nn; ++cy) {
      R* row = mesh + ((int64_t)iz[cz] * N + iy[cy]) * N;
      for (int cx = 0; cx < nn; ++cx) atomicAdd(&row[ix[cx]], (R)(vk * kx[cx] * ky[cy] * kz[cz]));
    }
}

// Cbar = xi_w bar * W * (2 C / S1 - S2 / S1^2) in place over C (the adjoint
// of xi_w = S2 / S1, S2 = sum W C^2, S1 = sum W C), W in the column form of
// the forward's sums: the (x, y) factor per thread, the z factor from a table.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_cbar(int N, double dx, SmoothW p, const double* __restrict__ wc, const double* __restrict__ sa, int P,
       R* __restrict__ Cm) {
  __shared__ R bz[1024];
  const int xb = (N + kThreads - 1) / kThreads;
  const int y = blockIdx.x / xb, x = (blockIdx.x % xb) * kThreads + threadIdx.x;
  const R inv2s2 = (R)(0.5 / (p.sigma * p.sigma));
  for (int zz = threadIdx.x; zz < N; zz += kThreads) {
    const R rz = (R)((double)(zz <= N / 2 ? zz : zz - N) * dx);
    bz[zz] = ex(-inv2s2 * rz * rz);
  }
  __syncthreads();
  if (x >= N) return;
  const double rx = (double)(x <= N / 2 ? x : x - N) * dx;
  const double ry = (double)(y <= N / 2 ? y : y - N) * dx;
  const double rp2 = rx * rx + ry * ry;
  R axy = 0;
  if (rp2 >= p.r_cut * p.r_cut) {
    const R rp = sq((R)rp2);
    axy = ((R)1 / ((R)1 + ex(-(R)p.s0 * (rp - (R)p.r_s)))) * ex(-inv2s2 * rp * rp);
  }
  const double S2 = wc[0], S1 = wc[1], xwbar = sa[3 * P + 1];
  const R c2 = (R)(2.0 * xwbar / S1), c0 = (R)(-xwbar * S2 / (S1 * S1));
  R* col = Cm + (int64_t)y * N + x;
  const int64_t zs = (int64_t)N * N;
  for (int zz = 0; zz < N; ++zz) {
    const R wv = axy * bz[zz];
    col[zz * zs] = wv * (c2 * col[zz * zs] + c0);
  }
}

// out[kz][ky][kx] (pitch P) = scale * (Wk * A + cs * B * Fg), k = 0 zeroed; the
// spectra in layout L.
template <typename C>
__global__ void __launch_bounds__(kThreads)
k_spec_combine(int N, int P, Lay L, const C* __restrict__ Wk, const C* __restrict__ A, const C* __restrict__ B,
               const C* __restrict__ Fg, double cs, double scale, C* __restrict__ out) {
  using RT = decltype(C::x);
  const int M1 = N / 2 + 1;
  const int64_t total = (int64_t)N * N * M1;
  for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < total; t += (int64_t)gridDim.x * kThreads) {
    const int kx = (int)(t % M1);
    const int ky = (int)((t / M1) % N);
    const int kz = (int)(t / ((int64_t)M1 * N));
    const int64_t src = (int64_t)kz * L.zs + yoff(L, ky) + xoff(L, kx);
    const C w = Wk[src], a = A[src], b = B[src], f = Fg[src];
    C v;
    v.x = (RT)scale * ((w.x * a.x - w.y * a.y) + (RT)cs * (b.x * f.x - b.y * f.y));
    v.y = (RT)scale * ((w.x * a.y + w.y * a.x) + (RT)cs * (b.x * f.y + b.y * f.x));
    if (kx == 0 && ky == 0 && kz == 0) v.x = v.y = 0;
    out[((int64_t)kz * N + ky) * P + kx] = v;
  }
}

// Galaxy k: the rho / Q chain (f = rho N^3 / Q, T = sum_j w_j fbar(x_j)), the
// galaxy mean of den and the npairs term of RR.
__global__ void __launch_bounds__(kThreads)
k_sadj_gal(int64_t n, int P, const double* __restrict__ fj, const double* __restrict__ Tsum,
           const unsigned long long* __restrict__ qsum, double n3, const double* __restrict__ gj,
           const double* __restrict__ gal, const double* __restrict__ sa, const double* __restrict__ wgal,
           double* __restrict__ wbar) {
  const int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (k >= n) return;
  const double Q = (double)(long long)qsum[0] * (1.0 / 4294967296.0);
  const double T = Tsum[0];
  const double sw = gal[1], den = gal[0] / gal[1];
  const double wk = wgal ? wgal[k] : 1.0;
  wbar[k] += (n3 / Q) * (fj[k] - T / Q) + sa[3 * P] * (gj[k] - den) / sw + sa[3 * P + 2] * (sw - wk);
}

unsigned blocks(int64_t n) { return (unsigned)std::max<int64_t>(cdiv(n, kThreads), 1); }

}  // namespace

cudaError_t launch_sadj_ratios(const SmoothAdjArgs& a, cudaStream_t s) {
  k_sadj_ratios<<<1, kThreads, 0, s>>>(a);
  return launched();
}

cudaError_t launch_sadj_pairs(int64_t np, int P, const int32_t* pbin, const double* pw, const double* gp,
                              const int32_t* pi, const int32_t* pj, const double* wgal, const double* psums,
                              const double* out, const double* sa, double* gpbar, double* wbar, cudaStream_t s) {
  if (np <= 0) return cudaSuccess;
  k_sadj_pairs<<<blocks(np), kThreads, 0, s>>>(np, P, pbin, pw, gp, pi, pj, wgal, psums, out, sa, gpbar, wbar);
  return launched();
}

cudaError_t launch_sadj_gbar(int64_t n, int P, const double* sa, const double* gal, const double* wgal,
                             double* gjbar, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_sadj_gbar<<<blocks(n), kThreads, 0, s>>>(n, P, sa, gal, wgal, gjbar);
  return launched();
}

template <typename R>
cudaError_t launch_scatter(const DepGeom& geo, int64_t n, const double* x, const double* y, const double* z,
                           const double* v, R* mesh, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_scatter<R><<<blocks(n), kThreads, 0, s>>>(geo, n, x, y, z, v, mesh);
  return launched();
}

template <typename R>
cudaError_t launch_cbar(int N, double dx, const SmoothW& p, const double* wc, const double* sa, int P, R* Cm,
                        cudaStream_t s) {
  if (N > 1024) return cudaErrorInvalidValue;   // the z-factor table
  k_cbar<R><<<(unsigned)(N * ((N + kThreads - 1) / kThreads)), kThreads, 0, s>>>(N, dx, p, wc, sa, P, Cm);
  return launched();
}

template <typename R>
cudaError_t launch_spec_combine(int N, int P, Lay L, const typename CT<R>::C* Wk, const typename CT<R>::C* A,
                                const typename CT<R>::C* B, const typename CT<R>::C* Fg, double cs, double scale,
                                typename CT<R>::C* out, cudaStream_t s) {
  const int64_t total = (int64_t)N * N * (N / 2 + 1);
  const unsigned g = (unsigned)std::min<int64_t>(cdiv(total, kThreads), 1 << 16);
  k_spec_combine<typename CT<R>::C><<<g, kThreads, 0, s>>>(N, P, L, Wk, A, B, Fg, cs, scale, out);
  return launched();
}

cudaError_t launch_sadj_gal(int64_t n, int P, const double* fj, const double* Tsum, const unsigned long long* qsum,
                            double n3, const double* gj, const double* gal, const double* sa, const double* wgal,
                            double* wbar, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_sadj_gal<<<blocks(n), kThreads, 0, s>>>(n, P, fj, Tsum, qsum, n3, gj, gal, sa, wgal, wbar);
  return launched();
}

template cudaError_t launch_scatter<float>(const DepGeom&, int64_t, const double*, const double*, const double*,
                                           const double*, float*, cudaStream_t);
template cudaError_t launch_scatter<double>(const DepGeom&, int64_t, const double*, const double*, const double*,
                                            const double*, double*, cudaStream_t);
template cudaError_t launch_cbar<float>(int, double, const SmoothW&, const double*, const double*, int, float*,
                                        cudaStream_t);
template cudaError_t launch_cbar<double>(int, double, const SmoothW&, const double*, const double*, int, double*,
                                         cudaStream_t);
template cudaError_t launch_spec_combine<float>(int, int, Lay, const float2*, const float2*, const float2*,
                                                const float2*, double, double, float2*, cudaStream_t);
template cudaError_t launch_spec_combine<double>(int, int, Lay, const double2*, const double2*, const double2*,
                                                 const double2*, double, double, double2*, cudaStream_t);

}  // namespace pg
