// The paper's own estimator with the smooth Gauss-sigmoid W (Sec. 2.1
// eq. bpg_final, Sec. 3.6 eq. weighting): kernels for W on the mesh offsets,
// the spectrum products, interpolation of the convolved field at points,
// deterministic FP64 sums and the final ratios. The FFT passes are the
// forward path's (pg_fft_*.cu); pg_api.cu orders the launches.
#include <math.h>

#include <algorithm>

#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kThreads = 256;

// eq. weighting with normalisation 1: W = 0 inside the line-of-sight cylinder
// r_perp < r_cut, else sigmoid(s0 (r_perp - r_s)) exp(-(r_perp^2 + r_par^2)/(2 sigma^2)).
// Evaluated in the plan's precision R: W only weights the mesh offsets, and
// FP64 exp at every one of N^3 offsets would cost more than the FFTs.
__device__ __forceinline__ float ex(float v) { return expf(v); }
__device__ __forceinline__ double ex(double v) { return exp(v); }
__device__ __forceinline__ float sq(float v) { return sqrtf(v); }
__device__ __forceinline__ double sq(double v) { return sqrt(v); }

template <typename R>
__device__ __forceinline__ R w_of(const SmoothW& p, R r_perp, R r_par) {
  const R sig = (R)1 / ((R)1 + ex(-(R)p.s0 * (r_perp - (R)p.r_s)));
  return sig * ex((R)-0.5 * (r_perp * r_perp + r_par * r_par) / (R)(p.sigma * p.sigma));
}

// W at the mesh offset of node t of a [z][y][x] mesh (line of sight = z);
// offsets are the signed minimum images i (i <= N/2) or i - N times dx. The
// cylinder r_perp < r_cut is decided in FP64 on the squared offset.
template <typename R>
__device__ __forceinline__ R w_at(int64_t t, int N, double dx, const SmoothW& p) {
  const int x = (int)(t % N), y = (int)((t / N) % N), z = (int)(t / ((int64_t)N * N));
  const double rx = (double)(x <= N / 2 ? x : x - N) * dx;
  const double ry = (double)(y <= N / 2 ? y : y - N) * dx;
  const double rz = (double)(z <= N / 2 ? z : z - N) * dx;
  const double rp2 = rx * rx + ry * ry;
  if (!(rp2 >= p.r_cut * p.r_cut)) return (R)0;
  return w_of<R>(p, sq((R)rp2), (R)fabs(rz));
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_w_mesh(int N, double dx, SmoothW p, R* __restrict__ out) {
  const int64_t n3 = (int64_t)N * N * N;
  for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < n3; t += (int64_t)gridDim.x * kThreads)
    out[t] = w_at<R>(t, N, dx, p);
}

// out[kz][ky][kx] (pitch P) = scale * A * B (mode 0) or scale * |B|^2
// (mode 1), k = 0 set to zero; A and B in layout L.
template <typename C>
__global__ void __launch_bounds__(kThreads)
k_spec_mul(int N, int P, Lay L, const C* __restrict__ A, const C* __restrict__ B, int mode, double scale,
           C* __restrict__ out) {
  using RT = decltype(C::x);
  const int M1 = N / 2 + 1;
  const int64_t total = (int64_t)N * N * M1;
  for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * kThreads) {
    const int kx = (int)(t % M1);
    const int ky = (int)((t / M1) % N);
    const int kz = (int)(t / ((int64_t)M1 * N));
    const int64_t src = (int64_t)kz * L.zs + yoff(L, ky) + xoff(L, kx);
    const C b = B[src];
    C v;
    if (mode == 0) {
      const C a = A[src];
      v.x = (RT)scale * (a.x * b.x - a.y * b.y);
      v.y = (RT)scale * (a.x * b.y + a.y * b.x);
    } else {
      v.x = (RT)scale * (b.x * b.x + b.y * b.y);
      v.y = 0;
    }
    if (kx == 0 && ky == 0 && kz == 0) v.x = v.y = 0;
    out[((int64_t)kz * N + ky) * P + kx] = v;
  }
}

// g[k] = the dense real field G [z][y][x] at point k, with the point's
// assignment weights (unrounded).
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_interp(DepGeom geo, int64_t n, const double* __restrict__ x, const double* __restrict__ y,
         const double* __restrict__ z, const R* __restrict__ G, double* __restrict__ g) {
  const int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (k >= n) return;
  const int N = geo.N;
  int ix[3], iy[3], iz[3];
  double kx[3], ky[3], kz[3];
  const int nn = axis_nodes(geo, __ddiv_rn(x[k], geo.dx), ix, kx);
  axis_nodes(geo, __ddiv_rn(y[k], geo.dx), iy, ky);
  axis_nodes(geo, __ddiv_rn(z[k], geo.dx), iz, kz);
  double v = 0.0;
  for (int cz = 0; cz < nn; ++cz)
    for (int cy = 0; cy < nn; ++cy) {
      const R* row = G + ((int64_t)iz[cz] * N + iy[cy]) * N;
      for (int cx = 0; cx < nn; ++cx) v += kx[cx] * ky[cy] * kz[cz] * (double)row[ix[cx]];
    }
  g[k] = v;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// One CTA per segment [off[s], off[s+1]): sums[2s] = sum w g, sums[2s+1] =
// sum w (w null: 1). Fixed order, so the sums are deterministic.
__global__ void __launch_bounds__(kThreads)
k_seg_sums(const int64_t* __restrict__ off, const double* __restrict__ g, const double* __restrict__ w,
           double* __restrict__ sums) {
  __shared__ double red[kThreads];
  const int s = blockIdx.x;
  double a = 0.0, b = 0.0;
  for (int64_t i = off[s] + threadIdx.x; i < off[s + 1]; i += kThreads) {
    const double wi = w ? w[i] : 1.0;
    a += wi * g[i];
    b += wi;
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    sums[2 * s] = a;
    sums[2 * s + 1] = b;
  }
}

// Partial sums of W C^2 and W C over all mesh offsets (C real [z][y][x]).
// sum W C^2 and sum W C over the mesh offsets (eq. xi_dw). W separates into
// an (x, y) factor (the cylinder mask in FP64 on squared offsets, the
// sigmoid and the Gaussian in r_perp) and a z factor (the Gaussian in r_par),
// so one thread owns an (x, y) column, evaluates its factor once, and walks z
// with the z factors from a shared table; the loads of a warp are consecutive
// x. Sums run in the plan precision over chunks of 32 z rows and are added to
// FP64 after each chunk; one partial per block, reduced in block order.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_wc_partial(int N, double dx, SmoothW p, const R* __restrict__ Cm, double* __restrict__ part) {
  __shared__ double red[kThreads];
  __shared__ R bz[1024];
  const int xb = (N + kThreads - 1) / kThreads;
  const int y = blockIdx.x / xb, x = (blockIdx.x % xb) * kThreads + threadIdx.x;
  const R inv2s2 = (R)(0.5 / (p.sigma * p.sigma));
  for (int z = threadIdx.x; z < N; z += kThreads) {
    const R rz = (R)((double)(z <= N / 2 ? z : z - N) * dx);
    bz[z] = ex(-inv2s2 * rz * rz);
  }
  R axy = 0;
  if (x < N) {
    const double rx = (double)(x <= N / 2 ? x : x - N) * dx;
    const double ry = (double)(y <= N / 2 ? y : y - N) * dx;
    const double rp2 = rx * rx + ry * ry;
    if (rp2 >= p.r_cut * p.r_cut) {
      const R rp = sq((R)rp2);
      axy = ((R)1 / ((R)1 + ex(-(R)p.s0 * (rp - (R)p.r_s)))) * ex(-inv2s2 * rp * rp);
    }
  }
  __syncthreads();
  double a = 0.0, b = 0.0;
  if (axy != (R)0) {
    const R* col = Cm + (int64_t)y * N + x;
    const int64_t zs = (int64_t)N * N;
    for (int z0 = 0; z0 < N; z0 += 32) {
      R ca = 0, cb = 0;
      const int z1 = min(N, z0 + 32);
      for (int z = z0; z < z1; ++z) {
        const R c = col[z * zs];
        const R wc = axy * bz[z] * c;
        ca += wc * c;
        cb += wc;
      }
      a += (double)ca;
      b += (double)cb;
    }
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

__global__ void __launch_bounds__(kThreads) k_wc_final(int nblk, const double* __restrict__ part,
                                                       double* __restrict__ out) {
  __shared__ double red[kThreads];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblk; i += kThreads) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = b;
  }
}

__global__ void __launch_bounds__(kThreads) k_smooth_final(SmoothArgs a) {
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const double sw = a.wsum[0], sw2 = a.wsum[1];
  const double npairs = 0.5 * (sw * sw - sw2);
  const double L3 = a.L * a.L * a.L;
  const double den = a.gal[1] > 0.0 ? a.gal[0] / a.gal[1] : nan;
  const double xw = a.wc[0] / a.wc[1];   // eq. xi_dw
  if (threadIdx.x == 0) {
    a.den[0] = den;
    a.xi_dw[0] = xw;
  }
  for (int p = threadIdx.x; p < a.P; p += kThreads) {
    const double vb = a.vbin[p];
    const double rr = npairs * vb / L3;
    const double ddw = (double)(long long)a.ddq[p] * (1.0 / 4294967296.0);
    const double xi = rr > 0.0 ? ddw / rr - 1.0 : nan;
    const double num = a.pairs[2 * p + 1] > 0.0 ? a.pairs[2 * p] / a.pairs[2 * p + 1] : nan;
    const double b = num / den;   // eq. bpg_final
    a.xi_ss[p] = xi;
    a.num[p] = num;
    a.b_pg[p] = b;
    // eq. Qeff_notsq
    a.q_eff[p] = ((1.0 + xi) * b - 2.0 - xw / (2.0 * xi)) / (2.0 * xi + 1.5 * xw);
  }
}

unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>(std::max<int64_t>(cdiv(n, kThreads), 1), 1 << 16); }

}  // namespace

template <typename R>
cudaError_t launch_w_mesh(int N, double dx, const SmoothW& p, R* out, cudaStream_t s) {
  k_w_mesh<R><<<grid_for((int64_t)N * N * N), kThreads, 0, s>>>(N, dx, p, out);
  return launched();
}

template <typename R>
cudaError_t launch_spec_mul(int N, int P, Lay L, const typename CT<R>::C* A, const typename CT<R>::C* B,
                            int mode, double scale, typename CT<R>::C* out, cudaStream_t s) {
  using C = typename CT<R>::C;
  k_spec_mul<C><<<grid_for((int64_t)N * N * (N / 2 + 1)), kThreads, 0, s>>>(N, P, L, A, B, mode, scale, out);
  return launched();
}

template <typename R>
cudaError_t launch_interp(const DepGeom& geo, int64_t n, const double* x, const double* y, const double* z,
                          const R* G, double* g, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_interp<R><<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(geo, n, x, y, z, G, g);
  return launched();
}

cudaError_t launch_seg_sums(int nseg, const int64_t* off, const double* g, const double* w, double* sums,
                            cudaStream_t s) {
  if (nseg <= 0) return cudaSuccess;
  k_seg_sums<<<nseg, kThreads, 0, s>>>(off, g, w, sums);
  return launched();
}

int wc_partials(int N) { return N * ((N + kThreads - 1) / kThreads); }

template <typename R>
cudaError_t launch_wc_sums(int N, double dx, const SmoothW& p, const R* Cm, double* part, double* out,
                           cudaStream_t s) {
  if (N > 1024) return cudaErrorInvalidValue;   // the z-factor table
  const int nblk = wc_partials(N);
  k_wc_partial<R><<<nblk, kThreads, 0, s>>>(N, dx, p, Cm, part);
  PG_CUDA_TRY(launched());
  k_wc_final<<<1, kThreads, 0, s>>>(nblk, part, out);
  return launched();
}

cudaError_t launch_smooth_final(const SmoothArgs& a, cudaStream_t s) {
  k_smooth_final<<<1, kThreads, 0, s>>>(a);
  return launched();
}

template cudaError_t launch_w_mesh<float>(int, double, const SmoothW&, float*, cudaStream_t);
template cudaError_t launch_w_mesh<double>(int, double, const SmoothW&, double*, cudaStream_t);
template cudaError_t launch_spec_mul<float>(int, int, Lay, const float2*, const float2*, int, double, float2*,
                                            cudaStream_t);
template cudaError_t launch_spec_mul<double>(int, int, Lay, const double2*, const double2*, int, double,
                                             double2*, cudaStream_t);
template cudaError_t launch_interp<float>(const DepGeom&, int64_t, const double*, const double*, const double*,
                                          const float*, double*, cudaStream_t);
template cudaError_t launch_interp<double>(const DepGeom&, int64_t, const double*, const double*,
                                           const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_wc_sums<float>(int, double, const SmoothW&, const float*, double*, double*,
                                           cudaStream_t);
template cudaError_t launch_wc_sums<double>(int, double, const SmoothW&, const double*, double*, double*,
                                            cudaStream_t);

}  // namespace pg
