// Adjoint of the forward path with respect to per-galaxy weights w_i.
//
// With w_p = w_i w_j for a pair, rho_b = sum_p w_p K(. - m_p), rho_g =
// sum_j w_j K(. - x_j), f = rho N^3 / Q and C_b(r) = (1/N^3) sum_x f_g(x)
// f_b(x + r) - 1 (Sec. 2.1, eqs. bpg_initial / bpg_intermediate), the
// reverse sweep is: ratio outputs -> bin sums S[b][q], G[q], G2[q], DD, sum w,
// sum w^2 (k_adjoint_ratios) -> a window field Cbar(r) per mesh
// (k_window_field) -> mesh adjoints by FFT correlation (the FFT passes) ->
// rho adjoints (normalisation) -> w_p and w_j by interpolating the mesh
// adjoint at the points with the deposit's node weights (k_gather_*) ->
// w_i = chain through w_p = w_i w_j (k_pair_chain). All scalars are FP64.
#include <math.h>

#include <algorithm>

#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double gate(const double* g, const double* out, int64_t i) {
  // upstream gradient of an output, zero where the forward output is not finite
  if (!g) return 0.0;
  const double v = out[i];
  return isfinite(v) ? g[i] : 0.0;
}

__global__ void __launch_bounds__(kThreads) k_adjoint_ratios(AdjRatioArgs a) {
  const int P = a.P, Q = a.Q, L = Q + 1;
  const double sw = a.wsum[0], sw2 = a.wsum[1];
  const double npairs = 0.5 * (sw * sw - sw2);
  const double L3 = a.L * a.L * a.L;
  auto rr_of = [&](int p) { return npairs * a.vbin[p] / L3; };
  auto ddw_of = [&](int p) { return (double)(long long)a.ddq[p] * (1.0 / 4294967296.0); };
  const double* S = a.sum_pg;   // [P][L][2]
  const double* Gs = a.sum_gg;  // [L][2]
  // per (pair bin, list): contributions
  for (int t = threadIdx.x; t < P * L; t += kThreads) {
    const int p = t / L, q = t % L;
    double sb = 0.0, dg = 0.0, dg2 = 0.0, dx = 0.0;
    const int64_t n = a.list_off[q + 1] - a.list_off[q];
    const double G = Gs[2 * q], G2 = Gs[2 * q + 1];
    if (a.pg_valid[p] && a.gg_valid && n > 0 && G != 0.0) {
      const double s = S[((int64_t)p * L + q) * 2];
      const double x = ddw_of(p) / rr_of(p) - 1.0;
      const double bb = s / G, xw = G2 / G;
      const double den = 2.0 * x + 1.5 * xw;
      const double num = (1.0 + x) * bb - 2.0 - xw / (2.0 * x);
      if (q < Q) {
        const int64_t o = (int64_t)p * Q + q;
        const double gq = gate(a.g.q_eff, a.o.q_eff, o), gs = gate(a.g.q_eff_sq, a.o.q_eff_sq, o);
        // terms of an output whose gradient is zero are skipped (they may be 0 * inf)
        double dbb = gate(a.g.b_pg, a.o.b_pg, o), dxw = 0.0;
        if (gq != 0.0) {
          dbb += gq * (1.0 + x) / den;
          dx += gq * ((bb + xw / (2.0 * x * x)) / den - 2.0 * num / (den * den));
          dxw += gq * (-1.0 / (2.0 * x) / den - 1.5 * num / (den * den));
        }
        if (gs != 0.0) {
          dbb += gs * (1.0 + x) / (2.0 * x);
          dx += gs * (bb / (2.0 * x) - ((1.0 + x) * bb - 2.0) / (2.0 * x * x));
        }
        sb = gate(a.g.xi_pg, a.o.xi_pg, o) / (double)n + dbb / G;
        dg = -dbb * s / (G * G) - dxw * G2 / (G * G);
        dg2 = dxw / G;
      } else {
        const double ga = gate(a.g.q_eff_agg, a.o.q_eff_agg, p);
        double dba = gate(a.g.b_pg_agg, a.o.b_pg_agg, p), dxwa = 0.0;
        if (ga != 0.0) {
          dba += ga * (1.0 + x) / den;
          dx = ga * ((bb + xw / (2.0 * x * x)) / den - 2.0 * num / (den * den));
          dxwa = ga * (-1.0 / (2.0 * x) / den - 1.5 * num / (den * den));
        }
        sb = dba / G;
        dg = -dba * s / (G * G) - dxwa * G2 / (G * G);
        dg2 = dxwa / G;
      }
    }
    a.Sbar[t] = sb;
    a.tmp[3 * (int64_t)t] = dg;
    a.tmp[3 * (int64_t)t + 1] = dg2;
    a.tmp[3 * (int64_t)t + 2] = dx;
  }
  __syncthreads();
  // galaxy sums: reduce over pair bins (fixed order)
  for (int q = threadIdx.x; q < L; q += kThreads) {
    const int64_t n = a.list_off[q + 1] - a.list_off[q];
    const double G = Gs[2 * q], G2 = Gs[2 * q + 1];
    double gb = 0.0, g2b = 0.0;
    for (int p = 0; p < P; ++p) {
      gb += a.tmp[3 * ((int64_t)p * L + q)];
      g2b += a.tmp[3 * ((int64_t)p * L + q) + 1];
    }
    if (a.gg_valid && n > 0 && G != 0.0) {
      if (q < Q) {
        const double gx = gate(a.g.xi_dw, a.o.xi_dw, q);
        gb += gate(a.g.xi_gg, a.o.xi_gg, q) / (double)n - gx * G2 / (G * G);
        g2b += gx / G;
      } else {
        const double gx = gate(a.g.xi_dw_agg, a.o.xi_dw_agg, 0);
        gb += -gx * G2 / (G * G);
        g2b += gx / G;
      }
    }
    a.Gbar[q] = gb;
    a.G2bar[q] = g2b;
  }
  // pair counts and the RR normalisation
  __shared__ double red[kThreads];
  double npb = 0.0;
  for (int p = threadIdx.x; p < P; p += kThreads) {
    double xsb = gate(a.g.xi_ss, a.o.xi_ss, p);
    if (a.wcoef) xsb += a.wcoef[p] * gate(a.g.w_perp, a.o.w_perp, p / a.n_mu);   // w(d_perp)
    for (int q = 0; q < L; ++q) xsb += a.tmp[3 * ((int64_t)p * L + q) + 2];
    const double rr = rr_of(p), ddw = ddw_of(p);
    const double ddb = gate(a.g.dd_w, a.o.dd_w, p) + (rr > 0.0 ? xsb / rr : 0.0);
    a.DDbar[p] = ddb;
    if (rr > 0.0) npb += (-xsb * ddw / (rr * rr)) * a.vbin[p] / L3;
  }
  red[threadIdx.x] = npb;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.wsbar[0] = red[0] * sw;     // d/d(sum w)
    a.wsbar[1] = -0.5 * red[0];   // d/d(sum w^2)
  }
}

// Window adjoint field laid out as the W^2 x-lines of the window, in mesh
// order of (z, y); a line of N reals holds Cbar at x offsets |x| <= w (mesh
// index x mod N) and zeros elsewhere.
//   pair mode:  Cbar(r) = Sbar[q(r)] + agg(r) Sbar[Q]
//   gg mode:    Cbar(r) = Gbar[q] + 2 C_gg(r) G2bar[q] + agg(r) (Gbar[Q] + 2 C_gg(r) G2bar[Q])
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_window_field(int N, int w, const int32_t* __restrict__ cell_bin, const uint8_t* __restrict__ cell_agg,
               int Q, const double* __restrict__ sbar, const double* __restrict__ gbar,
               const double* __restrict__ g2bar, const R* __restrict__ cgg, R* __restrict__ lines) {
  const int W = 2 * w + 1;
  const int64_t total = (int64_t)W * W * N;
  for (int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * kThreads) {
    const int64_t line = t / N;
    const int x = (int)(t % N);
    const int ox = x <= N / 2 ? x : x - N;
    if (ox < -w || ox > w) {   // outside the window: no FP64 work (the GPU's FP64 rate is low)
      lines[t] = R(0);
      continue;
    }
    double v = 0.0;
    {
      // lines are in mesh order (z, then y): rank r <= w is offset r, rank
      // r > w is offset r - W; window coordinate = offset + w
      const int rz = (int)(line / W), ry = (int)(line % W);
      const int zw = rz <= w ? rz + w : rz - w - 1;
      const int yw = ry <= w ? ry + w : ry - w - 1;
      const int64_t cell = ((int64_t)zw * W + yw) * W + (ox + w);
      const int q = cell_bin[cell];
      const bool ag = cell_agg[cell] != 0;
      if (!gbar) {
        if (q >= 0) v += sbar[q];
        if (ag) v += sbar[Q];
      } else {
        const double c = (double)cgg[cell];
        if (q >= 0) v += gbar[q] + 2.0 * c * g2bar[q];
        if (ag) v += gbar[Q] + 2.0 * c * g2bar[Q];
      }
    }
    lines[t] = (R)v;
  }
}

// Interpolation of a mesh adjoint held as compact real lines at points, with
// the deposit's node weights (unrounded): g[k] = sum_nodes K * field(node).
// Also the partial sums of w[k] * g[k] per block.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_gather(DepGeom geo, int64_t n, const double* __restrict__ x, const double* __restrict__ y,
         const double* __restrict__ z, const double* __restrict__ wt,
         const int32_t* __restrict__ idx, const R* __restrict__ lines, double* __restrict__ g,
         double* __restrict__ partial) {
  const int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  double v = 0.0, wv = 0.0;
  if (k < n) {
    const int N = geo.N;
    int ix[3], iy[3], iz[3];
    double kx[3], ky[3], kz[3];
    const int nn = axis_nodes(geo, __ddiv_rn(x[k], geo.dx), ix, kx);
    axis_nodes(geo, __ddiv_rn(y[k], geo.dx), iy, ky);
    axis_nodes(geo, __ddiv_rn(z[k], geo.dx), iz, kz);
    for (int cz = 0; cz < nn; ++cz)
      for (int cy = 0; cy < nn; ++cy) {
        const int64_t line = idx[(int64_t)iz[cz] * N + iy[cy]];
        for (int cx = 0; cx < nn; ++cx) v += kx[cx] * ky[cy] * kz[cz] * (double)lines[line * N + ix[cx]];
      }
    g[k] = v;
    wv = (wt ? wt[k] : 1.0) * v;
  }
  __shared__ double red[kThreads];
  red[threadIdx.x] = wv;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(int nblk, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double red[kThreads];
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += kThreads) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// w_p adjoint of the pairs of one mesh and its chain to the two galaxies:
// wbar_p = (N^3/Q)(g_p - T/Q) + DDbar; wbar[i] += wbar_p w_j, wbar[j] += wbar_p w_i.
__global__ void __launch_bounds__(kThreads)
k_pair_chain(int64_t np, const double* __restrict__ g, const double* __restrict__ T,
             const unsigned long long* __restrict__ qsum, double n3, const double* __restrict__ ddbar,
             const int32_t* __restrict__ pi, const int32_t* __restrict__ pj,
             const double* __restrict__ wgal, double* __restrict__ wbar) {
  const int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (k >= np) return;
  const double Q = (double)(long long)qsum[0] * (1.0 / 4294967296.0);
  const double wp = (n3 / Q) * (g[k] - *T / Q) + *ddbar;
  const int i = pi[k], j = pj[k];
  const double wi = wgal ? wgal[i] : 1.0, wj = wgal ? wgal[j] : 1.0;
  atomicAdd(&wbar[i], wp * wj);
  atomicAdd(&wbar[j], wp * wi);
}

// Galaxy mesh term and the sum-w terms: wbar[j] += (N^3/Q)(g_j - T/Q)
// + d/d(sum w) + 2 w_j d/d(sum w^2).
__global__ void __launch_bounds__(kThreads)
k_gal_final(int64_t n, const double* __restrict__ g, const double* __restrict__ T,
            const unsigned long long* __restrict__ qsum, double n3,
            const double* __restrict__ wsbar, const double* __restrict__ wgal,
            double* __restrict__ wbar) {
  const int64_t k = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (k >= n) return;
  const double Q = (double)(long long)qsum[0] * (1.0 / 4294967296.0);
  const double wk = wgal ? wgal[k] : 1.0;
  wbar[k] += (n3 / Q) * (g[k] - *T / Q) + wsbar[0] + 2.0 * wk * wsbar[1];
}

}  // namespace

cudaError_t launch_adjoint_ratios(const AdjRatioArgs& a, cudaStream_t s) {
  k_adjoint_ratios<<<1, kThreads, 0, s>>>(a);
  return launched();
}

template <typename R>
cudaError_t launch_window_field(int N, int w, const int32_t* cell_bin, const uint8_t* cell_agg, int Q,
                                const double* sbar, const double* gbar, const double* g2bar,
                                const R* cgg, R* lines, cudaStream_t s) {
  const int64_t total = (int64_t)(2 * w + 1) * (2 * w + 1) * N;
  const unsigned grid = (unsigned)std::min<int64_t>(cdiv(total, kThreads), 65536);
  k_window_field<R><<<grid, kThreads, 0, s>>>(N, w, cell_bin, cell_agg, Q, sbar, gbar, g2bar, cgg, lines);
  return launched();
}
template cudaError_t launch_window_field<float>(int, int, const int32_t*, const uint8_t*, int, const double*,
                                                const double*, const double*, const float*, float*, cudaStream_t);
template cudaError_t launch_window_field<double>(int, int, const int32_t*, const uint8_t*, int, const double*,
                                                 const double*, const double*, const double*, double*,
                                                 cudaStream_t);

template <typename R>
cudaError_t launch_gather(const DepGeom& geo, int64_t n, const double* x, const double* y,
                          const double* z, const double* wt, const int32_t* idx, const R* lines,
                          double* g, double* partial, double* T, cudaStream_t s) {
  if (n <= 0) return cudaMemsetAsync(T, 0, sizeof(double), s);
  const unsigned nblk = (unsigned)cdiv(n, kThreads);
  k_gather<R><<<nblk, kThreads, 0, s>>>(geo, n, x, y, z, wt, idx, lines, g, partial);
  PG_CUDA_TRY(launched());
  k_sum_partials<<<1, kThreads, 0, s>>>((int)nblk, partial, T);
  return launched();
}
template cudaError_t launch_gather<float>(const DepGeom&, int64_t, const double*, const double*,
                                          const double*, const double*, const int32_t*, const float*,
                                          double*, double*, double*, cudaStream_t);
template cudaError_t launch_gather<double>(const DepGeom&, int64_t, const double*, const double*,
                                           const double*, const double*, const int32_t*,
                                           const double*, double*, double*, double*, cudaStream_t);

cudaError_t launch_pair_chain(int64_t np, const double* g, const double* T,
                              const unsigned long long* qsum, double n3, const double* ddbar,
                              const int32_t* pi, const int32_t* pj, const double* wgal,
                              double* wbar, cudaStream_t s) {
  if (np <= 0) return cudaSuccess;
  k_pair_chain<<<(unsigned)cdiv(np, kThreads), kThreads, 0, s>>>(np, g, T, qsum, n3, ddbar, pi, pj,
                                                                  wgal, wbar);
  return launched();
}

// Soft HOD occupation weights (Sec. 3.3, eq. hod) of candidate galaxies and
// their derivatives in theta = (log10 M_cut, log10 M_1, sigma, alpha, kappa):
//   central:   w = erfc(u)/2, u = ln(M_cut/M) / (sqrt(2) sigma)
//   satellite: w = ((M - kappa M_cut)/M_1)^alpha / K for M > kappa M_cut, else 0
// (K: the number of satellite candidates of the halo).
// With d2w, also the second derivatives, upper triangle j <= k in row order
// (00 01 02 03 04 11 12 13 14 22 23 24 33 34 44), by the chain rule:
//   central: g = dv/du = -exp(-u^2)/sqrt(pi), dg/du = -2 u g; u_0 =
//     ln10/(sqrt(2) sigma), u_2 = -u/sigma, u_02 = -u_0/sigma, u_22 = 2u/sigma^2;
//     v_jk = -2 u g u_j u_k + g u_jk
//   satellite: f = x^alpha; x_0 = -kappa M_cut ln10/M_1, x_1 = -x ln10,
//     x_4 = -M_cut/M_1, x_00 = x_0 ln10, x_01 = -x_0 ln10, x_04 = x_4 ln10,
//     x_11 = x ln10^2, x_14 = -x_4 ln10; v_jk = (f_xx x_j x_k + f_x x_jk)/K
//     for j, k in {0, 1, 4}, v_j3 = f_xa x_j / K, v_33 = f_aa / K.
__global__ void __launch_bounds__(256)
k_hod_weights(int64_t n, const double* __restrict__ mass, const int32_t* __restrict__ kind,
              const float* __restrict__ kh, double t0, double t1, double sig, double alpha,
              double kappa, float* __restrict__ w, double* __restrict__ dw, double* __restrict__ d2w) {
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= n) return;
  const double ln10 = 2.302585092994045684;
  const double M = mass[i];
  const double mcut = exp(t0 * ln10), m1 = exp(t1 * ln10);
  double v = 0.0, d[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  double h[15];
  for (int k = 0; k < 15; ++k) h[k] = 0.0;
  if (kind[i] == 0) {
    const double u = (t0 * ln10 - log(M)) / (sqrt(2.0) * sig);
    v = 0.5 * erfc(u);
    const double dv_du = -exp(-u * u) / sqrt(M_PI);
    const double u0 = ln10 / (sqrt(2.0) * sig), u2 = -u / sig;
    d[0] = dv_du * u0;
    d[2] = dv_du * u2;
    const double gu = -2.0 * u * dv_du;
    h[0] = gu * u0 * u0;                                   // 00
    h[2] = gu * u0 * u2 + dv_du * (-u0 / sig);             // 02
    h[9] = gu * u2 * u2 + dv_du * (2.0 * u / (sig * sig)); // 22
  } else {
    const double x = (M - kappa * mcut) / m1;
    const double K = (double)kh[i];
    if (x > 0.0) {
      const double xa = pow(x, alpha);
      const double lx = log(x);
      v = xa / K;
      const double fx = alpha * xa / x;
      const double x0 = -kappa * mcut * ln10 / m1, x1 = -x * ln10, x4 = -mcut / m1;
      d[0] = fx * x0 / K;
      d[1] = fx * x1 / K;
      d[3] = xa * lx / K;
      d[4] = fx * x4 / K;
      const double fxx = alpha * (alpha - 1.0) * xa / (x * x);
      const double fxa = xa / x * (1.0 + alpha * lx);
      h[0] = (fxx * x0 * x0 + fx * x0 * ln10) / K;     // 00
      h[1] = (fxx * x0 * x1 - fx * x0 * ln10) / K;     // 01
      h[3] = fxa * x0 / K;                             // 03
      h[4] = (fxx * x0 * x4 + fx * x4 * ln10) / K;     // 04
      h[5] = (fxx * x1 * x1 + fx * x * ln10 * ln10) / K;   // 11
      h[7] = fxa * x1 / K;                             // 13
      h[8] = (fxx * x1 * x4 - fx * x4 * ln10) / K;     // 14
      h[12] = xa * lx * lx / K;                        // 33
      h[13] = fxa * x4 / K;                            // 34
      h[14] = fxx * x4 * x4 / K;                       // 44
    }
  }
  w[i] = (float)v;
  if (dw)
    for (int k = 0; k < 5; ++k) dw[5 * i + k] = d[k];
  if (d2w)
    for (int k = 0; k < 15; ++k) d2w[15 * i + k] = h[k];
}

// dL/dtheta_k = sum_i wbar_i dw_i/dtheta_k, per-block partials then a fixed-order sum.
__global__ void __launch_bounds__(256)
k_hod_chain_partial(int64_t n, const double* __restrict__ wbar, const double* __restrict__ dw,
                    double* __restrict__ partial) {
  __shared__ double red[5][256];
  const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
  for (int k = 0; k < 5; ++k) red[k][threadIdx.x] = i < n ? wbar[i] * dw[5 * i + k] : 0.0;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 5; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 5) partial[5 * (int64_t)blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void k_hod_chain_final(int nblk, const double* __restrict__ partial, double* __restrict__ out) {
  if (threadIdx.x >= 5) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[5 * (int64_t)b + threadIdx.x];
  out[threadIdx.x] = s;
}

cudaError_t launch_hod_weights(int64_t n, const double* mass, const int32_t* kind, const float* kh,
                               const double theta[5], float* w, double* dw, double* d2w,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_hod_weights<<<(unsigned)cdiv(n, 256), 256, 0, s>>>(n, mass, kind, kh, theta[0], theta[1], theta[2],
                                                        theta[3], theta[4], w, dw, d2w);
  return launched();
}

cudaError_t launch_hod_chain(int64_t n, const double* wbar, const double* dw, double* partial,
                             double* out5, cudaStream_t s) {
  const int nblk = (int)std::max<int64_t>(1, cdiv(n, 256));
  k_hod_chain_partial<<<nblk, 256, 0, s>>>(n, wbar, dw, partial);
  PG_CUDA_TRY(launched());
  k_hod_chain_final<<<1, 32, 0, s>>>(nblk, partial, out5);
  return launched();
}

cudaError_t launch_gal_final(int64_t n, const double* g, const double* T,
                             const unsigned long long* qsum, double n3, const double* wsbar,
                             const double* wgal, double* wbar, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_gal_final<<<(unsigned)cdiv(n, kThreads), kThreads, 0, s>>>(n, g, T, qsum, n3, wsbar, wgal, wbar);
  return launched();
}

}  // namespace pg
