// FFT passes of the mesh cross-correlation (Sec. 2.1: F_p conj(F_g) and its
// inverse, eqs. bpg_initial / bpg_intermediate), templated on the real type
// R (float or double) and the mesh size N. Included by pg_fft_f32.cu and
// pg_fft_f64.cu, which instantiate it once per precision.
//
// Layout. A mesh is [z][y][x], x contiguous. After the x pass a half spectrum
// row holds kx = 0..N/2 with pitch P complex elements. The y and z passes work
// on tiles of B consecutive kx columns x all N rows of one axis, staged in
// shared memory as buf[n*B + c]; the x passes stage lines as buf[n*LD + line].
//
// Each length-N 1D transform is one Cooley-Tukey split N = N1*N2 (N1 = 32):
// step 1 does the N1-point DFTs over j1 in registers and applies W_N^(j2 k1)
// in place; step 2 does the N2-point DFTs over j2 in registers and leaves
// X[k1 + N1 k2] in the registers of task (c, k1). The inverse runs the split
// the other way round from registers (step A) back through shared memory
// (step B), so the z pass goes forward -> multiply -> inverse without a
// second round trip. Twiddles W_N^j come from an FP64-generated table.
#pragma once

#include "pg_internal.cuh"
#include "pg_tma.cuh"
#include "pg_twiddle32.cuh"

namespace pg {
namespace fft {

// W_32^j from constant memory on the device, from the same values on the host
// (the host path exists only so that the register DFT can be checked on a CPU).
template <typename C> __host__ __device__ __forceinline__ C w32(int j);
template <> __host__ __device__ __forceinline__ float2 w32<float2>(int j) {
#ifdef __CUDA_ARCH__
  return c_w32f[j];
#else
  return h_w32f[j];
#endif
}
template <> __host__ __device__ __forceinline__ double2 w32<double2>(int j) {
#ifdef __CUDA_ARCH__
  return c_w32d[j];
#else
  return h_w32d[j];
#endif
}

template <typename C> struct Real;
template <> struct Real<float2> { using T = float; };
template <> struct Real<double2> { using T = double; };

template <typename C> __host__ __device__ __forceinline__ C make_c(typename Real<C>::T x, typename Real<C>::T y);
template <> __host__ __device__ __forceinline__ float2 make_c<float2>(float x, float y) { return make_float2(x, y); }
template <> __host__ __device__ __forceinline__ double2 make_c<double2>(double x, double y) { return make_double2(x, y); }

__host__ __device__ constexpr int cbitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr int clog2(int n) { return n <= 1 ? 0 : 1 + clog2(n >> 1); }

template <int V> struct IC { static constexpr int value = V; };

// Compile-time loop: f(IC<I>{}) for I in [B, E).
template <int B, int E, typename F>
__host__ __device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B < E) {
    f(IC<B>{});
    sfor<B + 1, E>(f);
  }
}

// v * W_32^J (forward) or v * conj(W_32^J) (inverse) with J known at compile
// time: multiples of 8 (1, -i, -1, i) cost no multiplication.
template <int J, bool INV, typename C>
__host__ __device__ __forceinline__ C tw32_mul(C v) {
  constexpr int j = J & 31;
  if constexpr (j == 0) {
    return v;
  } else if constexpr (j == 16) {
    return make_c<C>(-v.x, -v.y);
  } else if constexpr ((j == 8 && !INV) || (j == 24 && INV)) {   // times -i
    return make_c<C>(v.y, -v.x);
  } else if constexpr (j == 8 || j == 24) {  // times +i
    return make_c<C>(-v.y, v.x);
  } else {
    C w = w32<C>(j);
    if (INV) w.y = -w.y;
    return cmul(v, w);
  }
}

__host__ __device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }
__host__ __device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }

// One radix-2 butterfly u, v -> u + t, u - t with t = v * W_32^J (conjugated
// for the inverse), J known at compile time; TOP / BOT select the outputs that
// are needed. A general twiddle costs four fused multiply-adds for u + t and
// two more for u - t = 2u - (u + t): six instructions instead of the eight of
// a complex product followed by a sum and a difference.
//
// With PK, on sm_100 and later, FP32 butterflies use the packed two-wide FP32
// arithmetic (__fadd2_rn, __ffma2_rn), which rounds each component exactly as
// the scalar operation: a twiddle of +-1 takes two packed operations instead
// of four, a general twiddle three packed fused multiply-adds (each component
// in the scalar form's order, so the results are bit-identical) instead of six.
// The operand swaps and paired constants cost registers, so only the kernels
// where it measured faster ask for it.
template <int J, bool INV, bool TOP, bool BOT, bool PK, typename C>
__host__ __device__ __forceinline__ void bfly(C& u, C& v) {
  using T = typename Real<C>::T;
  constexpr int j = J & 31;
  constexpr bool triv = j == 0 || j == 8 || j == 16 || j == 24;
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  if constexpr (PK && sizeof(T) == 4) {
    const float2 m1 = make_float2(-1.f, -1.f);
    if constexpr (j == 0 || j == 16) {
      // u + v and u - v (j = 16 swaps them)
      const float2 s = __fadd2_rn(u, v), d = __ffma2_rn(v, m1, u);
      if constexpr (TOP) u = j == 0 ? s : d;
      if constexpr (BOT) v = j == 0 ? d : s;
      return;
    } else if constexpr (!triv) {
      float2 w = w32<float2>(j);
      if (INV) w.y = -w.y;
      const float2 vs = make_float2(v.y, v.x);
      if constexpr (TOP) {
        // (fma(w.x, v.x, fma(-w.y, v.y, u.x)), fma(w.x, v.y, fma(w.y, v.x, u.y)))
        const float2 in = __ffma2_rn(make_float2(-w.y, w.y), vs, u);
        const float2 x = __ffma2_rn(make_float2(w.x, w.x), v, in);
        if constexpr (BOT) v = __ffma2_rn(make_float2(2.f, 2.f), u, make_float2(-x.x, -x.y));
        u = x;
      } else if constexpr (BOT) {
        // (fma(-w.x, v.x, fma(w.y, v.y, u.x)), fma(-w.x, v.y, fma(-w.y, v.x, u.y)))
        const float2 in = __ffma2_rn(make_float2(w.y, -w.y), vs, u);
        v = __ffma2_rn(make_float2(-w.x, -w.x), v, in);
      }
      return;
    }
  }
#endif
  if constexpr (triv) {
    const C t = tw32_mul<j, INV>(v);
    const C x = cadd(u, t), y = csub(u, t);
    if constexpr (TOP) u = x;
    if constexpr (BOT) v = y;
  } else {
    C w = w32<C>(j);
    if (INV) w.y = -w.y;
    if constexpr (TOP) {
      const C x = make_c<C>(fmadd(w.x, v.x, fmadd(-w.y, v.y, u.x)), fmadd(w.x, v.y, fmadd(w.y, v.x, u.y)));
      if constexpr (BOT) v = make_c<C>(fmadd((T)2, u.x, -x.x), fmadd((T)2, u.y, -x.y));
      u = x;
    } else if constexpr (BOT) {
      v = make_c<C>(fmadd(-w.x, v.x, fmadd(w.y, v.y, u.x)), fmadd(-w.x, v.y, fmadd(-w.y, v.x, u.y)));
    }
  }
}

// One radix-2 stage (butterflies of span LEN) of the in-register DFT, then
// the later stages. K prunes the outputs: only X[k] for k < K or k >= RL - K
// are wanted (all when 2K >= RL). A decimation-in-time stage of span LEN then
// needs, within each group of LEN, exactly its outputs k < K and k >= LEN - K
// (the same rule one stage down), so unneeded halves of butterflies are
// dropped at compile time. Unwanted outputs are left undefined.
template <typename C, int RL, bool INV, int LEN, int K, bool PK = false>
__host__ __device__ __forceinline__ void dft_stage(C (&a)[RL]) {
  if constexpr (LEN <= RL) {
    constexpr int half = LEN / 2;
    sfor<0, RL / LEN>([&](auto ii) {
      constexpr int i = decltype(ii)::value * LEN;
      sfor<0, half>([&](auto kk) {
        constexpr int k = decltype(kk)::value;
        constexpr bool all = 2 * K >= LEN;
        constexpr bool top = all || k < K;
        constexpr bool bot = all || k + half >= LEN - K;
        if constexpr (top || bot) bfly<k * (32 / LEN), INV, top, bot, PK>(a[i + k], a[i + k + half]);
      });
    });
    dft_stage<C, RL, INV, LEN * 2, K, PK>(a);
  }
}

// In-register DFT of length RL (1..32), forward (exp(-i...)) or inverse:
// bit-reversal permutation, then radix-2 decimation-in-time stages. With
// K < RL / 2 only the outputs k < K and k >= RL - K are computed.
template <typename C, int RL, bool INV, int K = RL, bool PK = false>
__host__ __device__ __forceinline__ void reg_dft(C (&a)[RL]) {
  if constexpr (RL > 1) {
    constexpr int bits = clog2(RL);
#pragma unroll
    for (int i = 0; i < RL; ++i) {
      const int j = cbitrev(i, bits);
      if (j > i) { C t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    dft_stage<C, RL, INV, 2, K, PK>(a);
  }
}

// Forward DFT of length RL (dividing 32) of an input whose entries m >= NZ
// are zero: y[k] = sum_{m < NZ} b_m W_RL^(m k), k = 0..RL-1. For
// k = (RL / NZ) q + r, W_RL^(m k) = W_NZ^(m q) W_RL^(m r), so the outputs
// with remainder r are the NZ-point DFT of b_m W_RL^(m r) (compile-time
// twiddles, multiples of a quarter turn free).
template <typename C, int RL, int NZ>
__host__ __device__ __forceinline__ void dft_few_inputs(const C (&b)[NZ], C (&y)[RL]) {
  constexpr int R = RL / NZ;
  static_assert(R * NZ == RL && 32 % RL == 0, "NZ divides RL, RL divides 32");
  sfor<0, R>([&](auto rr) {
    constexpr int r = decltype(rr)::value;
    C cc[NZ];
    sfor<0, NZ>([&](auto mm) {
      constexpr int m = decltype(mm)::value;
      cc[m] = tw32_mul<m * r * (32 / RL), false>(b[m]);
    });
    reg_dft<C, NZ, false>(cc);
#pragma unroll
    for (int q = 0; q < NZ; ++q) y[R * q + r] = cc[q];
  });
}

// Copies the twiddle table W_N^j (j < n) into shared memory; the caller's
// next __syncthreads() publishes it.
template <typename C>
__device__ __forceinline__ const C* stage_tw(C* dst, const C* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
  return dst;
}

template <typename C, bool INV>
__device__ __forceinline__ C twid(const C* tw, int j) {
  C w = tw[j];
  if (INV) w.y = -w.y;
  return w;
}

// Rows of the split in shared memory. Tasks of one warp touch rows hi*span +
// lo for consecutive hi; with rows of B complex values (fewer than 128 bytes)
// those rows share banks. Storing row (hi, lo) at lo ^ (hi mod X), X = 128
// bytes / row bytes, spreads them over all banks. X = 1 keeps the natural
// order.
template <int X>
__device__ __forceinline__ int prow(int hi, int lo, int span) { return hi * span + (lo ^ (hi & (X - 1))); }

// Step 1 of the split on B columns held as buf[n*LD + c]: tasks (c, j2). It
// reads rows in natural order and writes row (k1, j2) at prow<X>(k1, j2, N2);
// the tasks j2 ^ m it overwrites belong to the same warp (B * X <= 32), so a
// warp barrier between its reads and writes makes it safe in place.
// tid / nthr: this thread's index in, and the size of, the (warp-aligned)
// group of threads sharing the tile.
template <typename C, int N1, int N2, int B, bool INV, int X = 1, bool PK = false>
__device__ __forceinline__ void step1(C* buf, int LD, const C* tw, int tws, int tid, int nthr) {
  static_assert(X == 1 || (B * X <= 32 && N2 % X == 0 && (B * N2) % 32 == 0), "row permutation");
  for (int t = tid; t < B * N2; t += nthr) {
    const int c = t % B, j2 = t / B;
    C a[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) a[j1] = buf[(N2 * j1 + j2) * LD + c];
    reg_dft<C, N1, INV, N1, PK>(a);
    if (N2 > 1 && j2 > 0) {
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) a[k1] = cmul(a[k1], twid<C, INV>(tw, j2 * k1 * tws));
    }
    if (X > 1) __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) buf[prow<X>(k1, j2, N2) * LD + c] = a[k1];
  }
}

template <typename C, int N1, int N2, int B, bool INV, int X = 1, bool PK = false>
__device__ __forceinline__ void step1(C* buf, int LD, const C* tw, int tws) {
  step1<C, N1, N2, B, INV, X, PK>(buf, LD, tw, tws, (int)threadIdx.x, (int)blockDim.x);
}

// Step 1 on a tile whose rows are present only where msk says so: bit j1 of
// msk[j2] marks row N2 j1 + j2 (msk null: every row). Absent rows are read as
// zero without touching shared memory, so the tile needs no clearing between
// sparse fills.
template <typename C, int N1, int N2, int B, bool INV, int X = 1, bool PK = false>
__device__ __forceinline__ void step1_m(C* buf, int LD, const C* tw, const uint32_t* msk) {
  static_assert(N1 <= 32, "one mask word per task");
  for (int t = threadIdx.x; t < B * N2; t += blockDim.x) {
    const int c = t % B, j2 = t / B;
    const uint32_t m = msk ? msk[j2] : 0xffffffffu;
    C a[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      a[j1].x = 0; a[j1].y = 0;
      if ((m >> j1) & 1u) a[j1] = buf[(N2 * j1 + j2) * LD + c];
    }
    reg_dft<C, N1, INV, N1, PK>(a);
    if (N2 > 1 && j2 > 0) {
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) a[k1] = cmul(a[k1], twid<C, INV>(tw, j2 * k1));
    }
    if (X > 1) __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) buf[prow<X>(k1, j2, N2) * LD + c] = a[k1];
  }
}

// Step 2: task (c, k1) reads its N2 values and leaves X[k1 + N1*k2] in a[k2];
// with K < N2 / 2 only k2 < K and k2 >= N2 - K are computed (see reg_dft).
template <typename C, int N1, int N2, bool INV, int X = 1, int K = N2, bool PK = false>
__device__ __forceinline__ void step2(const C* buf, int LD, int c, int k1, C (&a)[N2]) {
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) a[j2] = buf[prow<X>(k1, j2, N2) * LD + c];
  reg_dft<C, N2, INV, K, PK>(a);
}

// Step A (inverse split from registers): a[k2] = X[k1 + N1*k2] of task
// (c, k1) -> row (n2, k1) = W_N^(-+k1 n2) sum_k2 X W_N2^(-+k2 n2). The row is
// written back into the slot its thread read in step 2, prow<X>(k1, n2, N2)
// (its input j2 = n2). No other thread touches those slots between step 2 and
// step A, so the two need no barrier between them.
// Step B: task (c, n2) reads row (n2, k1) for k1 = 0..N1-1 from
// prow<X>(k1, n2, N2), the access pattern of step 1's stores, and leaves
// out[n1] = x[n2 + N2*n1]; with K < N1 / 2 only n1 < K and n1 >= N1 - K are
// computed (see reg_dft).
template <typename C, int N1, int N2, bool INV, int X = 1, bool PK = false>
__device__ __forceinline__ void stepA_own(C* buf, int LD, int c, int k1, C (&a)[N2], const C* tw, int tws) {
  reg_dft<C, N2, INV, N2, PK>(a);
  if (N2 > 1 && k1 > 0) {
#pragma unroll
    for (int n2 = 1; n2 < N2; ++n2) a[n2] = cmul(a[n2], twid<C, INV>(tw, k1 * n2 * tws));
  }
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) buf[prow<X>(k1, n2, N2) * LD + c] = a[n2];
}

template <typename C, int N1, int N2, bool INV, int X = 1, int K = N1, bool PK = false>
__device__ __forceinline__ void stepB_own(const C* buf, int LD, int c, int n2, C (&a)[N1]) {
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) a[k1] = buf[prow<X>(k1, n2, N2) * LD + c];
  reg_dft<C, N1, INV, K, PK>(a);
}

// Step 1 and step A (own slots) when every thread runs exactly one task and
// N1 = N2: task (c, q) of either step multiplies its outputs by W_N^(q m),
// m < N1, with q = tid / B in both. The caller loads those N1 twiddles into
// registers once (tq[m] = W_N^(q m); conjugated here for the inverse), which
// saves 2 (N1 - 1) shared-memory loads per thread and mesh.
template <typename C, int N1, int N2, int B, bool INV, int X, bool PK = false>
__device__ __forceinline__ void step1_tr(C* buf, int LD, const C (&tq)[N1], int tid) {
  const int c = tid % B, j2 = tid / B;
  C a[N1];
#pragma unroll
  for (int j1 = 0; j1 < N1; ++j1) a[j1] = buf[(N2 * j1 + j2) * LD + c];
  reg_dft<C, N1, INV, N1, PK>(a);
#pragma unroll
  for (int k1 = 1; k1 < N1; ++k1) {
    C w = tq[k1];
    if (INV) w.y = -w.y;
    a[k1] = cmul(a[k1], w);
  }
  if (X > 1) __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) buf[prow<X>(k1, j2, N2) * LD + c] = a[k1];
}
template <typename C, int N1, int N2, bool INV, int X, bool PK = false>
__device__ __forceinline__ void stepA_own_tr(C* buf, int LD, int c, int k1, C (&a)[N2], const C (&tq)[N1]) {
  reg_dft<C, N2, INV, N2, PK>(a);
#pragma unroll
  for (int n2 = 1; n2 < N2; ++n2) {
    C w = tq[n2];
    if (INV) w.y = -w.y;
    a[n2] = cmul(a[n2], w);
  }
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) buf[prow<X>(k1, n2, N2) * LD + c] = a[n2];
}

template <int N> struct Split {
  static constexpr int N1 = N < 32 ? N : 32;
  static constexpr int N2 = N / N1;
};

// Row permutation span for column tiles of B complex values (see prow).
template <typename C, int N, int B>
__host__ __device__ constexpr int xperm() {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  constexpr int row = B * (int)sizeof(C);
  constexpr int X = row >= 128 ? 1 : 128 / row;
  return (N2 % X == 0 && N1 % X == 0 && (B * N2) % 32 == 0 && B * X <= 32) ? X : 1;
}

// Work item of a pass over the z columns (ky, kx tile) of the plan's
// spectra, ordered with the 8 ky rows of a block fastest: the CTAs running at
// once then read the 8 rows of each 512-byte kx-tile block together.
__host__ __device__ __forceinline__ void zcol_item(int64_t item, int T, int& ky, int& kx_tile) {
  const int64_t q = item >> kYBlockShift;
  kx_tile = (int)(q % T);
  ky = (int)(q / T) * (1 << kYBlockShift) + (int)(item & ((1 << kYBlockShift) - 1));
}

__device__ __forceinline__ int win_index(int n, int N, int w) {
  // signed offset of mesh index n in (-N/2, N/2]; returns offset + w, or -1
  if (n <= w) return n + w;
  if (n >= N - w) return n - N + w;
  return -1;
}

// ============================================================================
// X pass, real-to-complex. Lines of N reals become M = N/2 complex values
// z[m] = f[2m] + i f[2m+1]; after the M-point DFT,
// X[k] = (Z[k] + conj Z[M-k])/2 + W_N^k (Z[k] - conj Z[M-k])/(2i), k = 0..M.
// ============================================================================
template <typename C, int N>
struct XPass {
  static constexpr int M = N / 2;
  static constexpr int N1 = Split<M>::N1, N2 = Split<M>::N2;
  static constexpr int LB = (256 / N1) < 8 ? 8 : (256 / N1);   // lines per CTA
  static constexpr int LD = LB + 1;
  static constexpr int THREADS = LB * N1;
  static constexpr size_t smem_bytes() { return sizeof(C) * ((size_t)(M + 1) * LD + N); }
};

template <typename C, int N, typename Loader>
__device__ __forceinline__ void x_r2c_body(C* buf, int64_t l0, int64_t n_lines, C* __restrict__ spec,
                                           int P, const C* tw, Loader load) {
  using X = XPass<C, N>;
  constexpr int M = X::M, LB = X::LB, LD = X::LD, N1 = X::N1, N2 = X::N2;
  for (int idx = threadIdx.x; idx < LB * M; idx += blockDim.x) {
    const int c = idx / M, m = idx % M;
    const int64_t l = l0 + c;
    C v;
    v.x = 0; v.y = 0;
    if (l < n_lines) v = load(l, m);
    buf[m * LD + c] = v;
  }
  __syncthreads();
  step1<C, N1, N2, LB, false>(buf, LD, tw, 2);
  __syncthreads();
  const int c = threadIdx.x % LB, k1 = threadIdx.x / LB;
  C a[N2];
  step2<C, N1, N2, false>(buf, LD, c, k1, a);
  __syncthreads();
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) buf[(k1 + N1 * k2) * LD + c] = a[k2];
  __syncthreads();
  using RT = typename Real<C>::T;
  for (int idx = threadIdx.x; idx < LB * (M + 1); idx += blockDim.x) {
    const int cc = idx / (M + 1), k = idx % (M + 1);
    const int64_t l = l0 + cc;
    if (l >= n_lines) continue;
    C zk = buf[(k % M) * LD + cc];
    C zm = buf[((M - k) % M) * LD + cc];
    C e = make_c<C>((zk.x + zm.x) * RT(0.5), (zk.y - zm.y) * RT(0.5));
    // (Z[k] - conj Z[M-k]) / (2i)
    C d = make_c<C>((zk.y + zm.y) * RT(0.5), -(zk.x - zm.x) * RT(0.5));
    C w = tw[k];   // shared-memory twiddle table
    C o = cmul(d, w);
    spec[l * P + k] = cadd(e, o);
  }
}


template <typename C, int N>
__global__ void __launch_bounds__(XPass<C, N>::THREADS)
k_x_r2c_lines(const int64_t* __restrict__ q, const int32_t* __restrict__ line_bin,
              const double* __restrict__ scale, int64_t n_lines, C* __restrict__ spec, int P,
              const C* __restrict__ tw) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw) + N;        // twiddles W_N^j first, then the tile
  const C* tws = stage_tw(reinterpret_cast<C*>(smem_raw), tw, N);
  using RT = typename Real<C>::T;
  const int64_t l0 = (int64_t)blockIdx.x * XPass<C, N>::LB;
  x_r2c_body<C, N>(buf, l0, n_lines, spec, P, tws, [&](int64_t l, int m) {
    const longlong2 qq = reinterpret_cast<const longlong2*>(q + l * N)[m];
    if constexpr (sizeof(RT) == 4) {
      // FP32 plans convert in FP32: the GPU's FP64 rate would make this
      // load the x pass's limit; the two extra roundings (of q, and of the
      // mesh's scale) are far below the FFT's own
      const float s = (float)scale[line_bin[l]];
      return make_c<C>(__ll2float_rn(qq.x) * s, __ll2float_rn(qq.y) * s);
    } else {
      const double s = scale[line_bin[l]];
      return make_c<C>((RT)((double)qq.x * s), (RT)((double)qq.y * s));
    }
  });
}

template <typename C, int N>
__global__ void __launch_bounds__(XPass<C, N>::THREADS)
k_x_r2c_dense(const typename Real<C>::T* __restrict__ f, int64_t n_lines, C* __restrict__ spec,
              int P, const C* __restrict__ tw) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw) + N;        // twiddles W_N^j first, then the tile
  const C* tws = stage_tw(reinterpret_cast<C*>(smem_raw), tw, N);
  const int64_t l0 = (int64_t)blockIdx.x * XPass<C, N>::LB;
  x_r2c_body<C, N>(buf, l0, n_lines, spec, P, tws, [&](int64_t l, int m) {
    return reinterpret_cast<const C*>(f + l * N)[m];
  });
}

// ============================================================================
// Y pass forward over compact lines. CTA = (kx tile, z plane, mesh).
// ============================================================================
template <typename C, int N, int B>
struct ColPass {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int THREADS = B * N1;
  // two CTAs per SM (registers capped at 128 for 256 threads): these passes
  // wait on strided column loads, and a second CTA covers that latency
  static constexpr int MINB = 2;
  static constexpr size_t smem_bytes() { return sizeof(C) * ((size_t)N * B + N); }
};

template <typename C, int B>
__device__ __forceinline__ void zero_tile(C* buf, int rows) {
  C z;
  z.x = 0; z.y = 0;
  for (int t = threadIdx.x; t < rows * B; t += blockDim.x) buf[t] = z;
}

// Y pass forward, persistent. A work item is (kx tile, z plane, mesh b), kx
// tile fastest, so the CTAs running at once gather the same compact lines of
// one plane. While one item is transformed, the rows of the next are gathered
// by cp.async into the second buffer (their line numbers were loaded at the
// start of the item, the plane's line range one item earlier), so the
// dependent index loads do not stall the pass. The gather marks the rows it
// fills in the buffer's presence mask, and step 1 reads only those (the rows
// a sparse plane lacks are zero without being stored).
// Sparse path (idx != null): the compact lines of plane z of mesh b are
// line_base[b] + [idx_b[z][0], idx_b[z+1][0]) with y = line_y[line]; dense
// path: line z*N + y of one mesh.
// Output (TS, the plan's tiled layout): the item's column goes to a staging
// tile in natural ky order and thread 0 writes it with TMA tensor stores
// (map mO: the spectra map with boxes of YB ky rows of one z) at the next
// item's first barrier, and waits for the store to leave shared memory
// before its second, so the transform threads issue no global stores.
// Otherwise each thread stores its outputs directly.
// Buffers: with TS, two gather tiles and the staging tile (two CTAs per SM
// where that fits); without, two tiles where two CTAs' pairs fit, else one
// (the next item's rows are then gathered into it once step 2 has read it).
template <typename C, int N, int B, bool TS>
struct YFwd {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int THREADS = B * N1;
  static constexpr int TILE = N * B;
  static constexpr int RS = THREADS / B;   // rows gathered per round
  static constexpr int PRE = 4;            // rounds whose line numbers are loaded ahead
  static constexpr int YB = N < 256 ? N : 256;   // ky rows per store box
  static constexpr int NBUF = TS || 2 * sizeof(C) * (2 * (size_t)TILE + N) <= 220 * 1024 ? 2 : 1;
  static constexpr size_t SMEM = sizeof(C) * ((NBUF + (TS ? 1 : 0)) * (size_t)TILE + N) + 4 * NBUF * N2;
  static constexpr int MINB = 2 * SMEM <= 220 * 1024 || !TS ? 2 : 1;
  static constexpr size_t smem_bytes() { return SMEM; }
};

template <typename C, int N, int B, bool TS>
__global__ void __launch_bounds__(YFwd<C, N, B, TS>::THREADS, YFwd<C, N, B, TS>::MINB)
k_y_fwd_p(const __grid_constant__ CUtensorMap mO, const C* __restrict__ spec, int P, int nb,
          const int32_t* __restrict__ idx, const int64_t* __restrict__ seg_total,
          const int64_t* __restrict__ line_base, const int32_t* __restrict__ line_y, C* __restrict__ S,
          int64_t S_stride, Lay L, const C* __restrict__ tw) {
  using Y = YFwd<C, N, B, TS>;
  constexpr int N1 = Y::N1, N2 = Y::N2, TILE = Y::TILE, M1 = N / 2 + 1, RS = Y::RS, PRE = Y::PRE;
  constexpr int NBUF = Y::NBUF;
  constexpr int XP = xperm<C, N, B>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* const tws = reinterpret_cast<C*>(smem_raw);
  C* const buf0 = tws + N;   // buffers buf0 + k * TILE, k < NBUF
  C* const stg = buf0 + NBUF * TILE;   // staging tile (TS)
  // row presence of each buffer (sparse path): bit j1 of msk[k * N2 + j2] = row N2 j1 + j2
  uint32_t* const msk = reinterpret_cast<uint32_t*>(stg + (TS ? TILE : 0));
  const int T = (M1 + B - 1) / B;
  const int64_t n_items = (int64_t)T * N * nb;
  int64_t item = blockIdx.x;
  if (item >= n_items) return;   // whole CTA
  C zc;
  zc.x = 0; zc.y = 0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = tw[i];
  for (int i = threadIdx.x; i < NBUF * N2; i += blockDim.x) msk[i] = 0;
  const int c = threadIdx.x % B, slot = threadIdx.x / B;
  struct Item {
    int kx0, z, b;
    int64_t lo, hi;   // rows (compact lines, or dense lines) of the item's plane
  };
  // an item's line range is loaded raw (fetch) one item before its first use
  // and combined (resolve) after the next barrier, so no arithmetic waits on
  // the loads while they are in flight
  struct Raw {
    int kx0, z, b;
    int64_t base, last;
    int32_t i0, i1;
  };
  auto fetch = [&](int64_t it, Raw& q) {
    q.kx0 = (int)(it % T) * B;
    const int64_t r = it / T;
    q.z = (int)(r % N);
    q.b = (int)(r / N);
    if (idx) {
      const int32_t* ib = idx + (int64_t)q.b * N * N;
      q.base = line_base[q.b];
      q.i0 = ib[(int64_t)q.z * N];
      if (q.z + 1 < N) q.i1 = ib[(int64_t)(q.z + 1) * N];
      else q.last = seg_total[q.b];
    }
  };
  auto resolve = [&](const Raw& q, Item& m) {
    m.kx0 = q.kx0;
    m.z = q.z;
    m.b = q.b;
    if (idx) {
      m.lo = q.base + q.i0;
      m.hi = q.base + ((q.z + 1 < N) ? (int64_t)q.i1 : q.last);
    } else {
      m.lo = (int64_t)q.z * N;
      m.hi = m.lo + N;
    }
  };
  auto meta = [&](int64_t it, Item& m) {
    Raw q;
    fetch(it, q);
    resolve(q, m);
  };
  // rows of item m into buffer dst; y of the first PRE rounds from yv
  auto gather = [&](const Item& m, C* dst, const int (&yv)[PRE], bool have_yv) {
    const bool in = c < min(B, M1 - m.kx0);
    uint32_t* const mk = msk + (int)((dst - buf0) / TILE) * N2;
#pragma unroll
    for (int p = 0; p < PRE; ++p) {
      const int64_t r = m.lo + slot + (int64_t)p * RS;
      if (r < m.hi) {
        const int y = idx ? (have_yv ? yv[p] : line_y[r]) : (int)(r - m.lo);
        if (in) tma::cp_async(dst + y * B + c, spec + r * P + m.kx0 + c);
        if (idx && c == 0) atomicOr(&mk[y % N2], 1u << (y / N2));
      }
    }
    for (int64_t r = m.lo + slot + (int64_t)PRE * RS; r < m.hi; r += RS) {
      const int y = idx ? line_y[r] : (int)(r - m.lo);
      if (in) tma::cp_async(dst + y * B + c, spec + r * P + m.kx0 + c);
      if (idx && c == 0) atomicOr(&mk[y % N2], 1u << (y / N2));
    }
    tma::cp_async_commit();
  };
  Item cur, nxt;
  Raw pn;   // raw line range of the item after next, resolved into nxt one item later
  meta(item, cur);
  __syncthreads();   // twiddles staged, buffers cleared
  {
    int yv[PRE];
    gather(cur, buf0, yv, false);
  }
  int64_t nitem = item + gridDim.x;
  if (nitem < n_items) meta(nitem, nxt);
  bool pend = false;
  // TS: the column in the staging tile (item kx0, z, mesh b), if any
  bool staged = false;
  int skx = 0, sz = 0, sb = 0;
  const uint64_t pol_out = tma::policy_evict_first();
  auto put = [&]() {
#pragma unroll
    for (int y0 = 0; y0 < N; y0 += Y::YB)
      tma::store_5d_hint(&mO, stg + y0 * B, 0, 0, skx / B, sz, (y0 >> kYBlockShift) + sb * (N >> kYBlockShift),
                         pol_out);
    tma::bulk_commit();
  };
  for (int64_t job = 0; item < n_items; ++job) {
    C* buf = buf0 + (NBUF == 2 ? (int)(job & 1) : 0) * TILE;
    tma::cp_async_wait_all();
    __syncthreads();   // this item's rows have landed; the other buffer is clear; [TS] staging written
    if (TS && staged && threadIdx.x == 0) put();
    if (pend) resolve(pn, nxt);
    const int64_t nnitem = nitem + gridDim.x;
    int yv[PRE];
    if (nitem < n_items) {
      if (idx) {
#pragma unroll
        for (int p = 0; p < PRE; ++p) {
          const int64_t r = nxt.lo + slot + (int64_t)p * RS;
          yv[p] = r < nxt.hi ? line_y[r] : 0;
        }
      }
    }
    pend = nitem < n_items && nnitem < n_items;
    if (pend) fetch(nnitem, pn);
    const int cb = NBUF == 2 ? (int)(job & 1) : 0;
    // packed FP32 butterflies (see bfly); absent rows of a sparse plane read as zero
    step1_m<C, N1, N2, B, false, XP, true>(buf, B, tws, idx ? msk + cb * N2 : nullptr);
    if (TS && staged && threadIdx.x == 0) tma::bulk_wait_read_all();   // staging free again
    __syncthreads();
    if (threadIdx.x < N2) msk[cb * N2 + threadIdx.x] = 0;   // read by step 1; clear for the next fill
    if (NBUF == 2 && nitem < n_items) gather(nxt, buf0 + ((job & 1) ^ 1) * TILE, yv, true);
    C a[N2];
    step2<C, N1, N2, false, XP, N2, true>(buf, B, c, slot, a);
    if (NBUF == 1) {
      __syncthreads();   // the tile is read; its mask was cleared after step 1
      if (nitem < n_items) gather(nxt, buf, yv, true);
    }
    if constexpr (TS) {
      // columns past the half spectrum (kx >= M1, the last tile's padding) get zeros
      const bool in = c < min(B, M1 - cur.kx0);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) stg[(slot + N1 * k2) * B + c] = in ? a[k2] : zc;
      tma::fence_async_shared();
      staged = true;
      skx = cur.kx0; sz = cur.z; sb = cur.b;
    } else if (c < min(B, M1 - cur.kx0)) {
      C* out = S + (int64_t)cur.b * S_stride + (int64_t)cur.z * L.zs + xoff(L, cur.kx0) + c;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) tma::st_hint(out + yoff(L, slot + N1 * k2), a[k2], tma::policy_evict_first());
    }
    item = nitem;
    cur = nxt;
    nitem = nnitem;
  }
  if (TS && staged) {
    __syncthreads();   // the last column is in the staging tile
    if (threadIdx.x == 0) {
      put();
      tma::bulk_wait_all();
    }
  }
}

// Column tile load of one (ky, kx tile) z-column: rows z at stride zs.
template <typename C, int N, int B>
__device__ __forceinline__ void load_zcol(C* buf, const C* __restrict__ src, int64_t zs, int ncol) {
  const int c = threadIdx.x % B;
  for (int z = threadIdx.x / B; z < N; z += blockDim.x / B) {
    C v;
    v.x = 0; v.y = 0;
    if (c < ncol) v = src[(int64_t)z * zs + c];
    buf[z * B + c] = v;
  }
}

// Z pass forward in place (galaxy spectrum). CTA = (kx tile, ky).
template <typename C, int N, int B>
__global__ void __launch_bounds__(ColPass<C, N, B>::THREADS, ColPass<C, N, B>::MINB)
k_z_fwd(C* __restrict__ S, Lay L, const C* __restrict__ tw) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw) + N;        // twiddles W_N^j first, then the tile
  const C* tws = stage_tw(reinterpret_cast<C*>(smem_raw), tw, N);
  using CP = ColPass<C, N, B>;
  constexpr int N1 = CP::N1, N2 = CP::N2, M1 = N / 2 + 1;
  constexpr int XP = xperm<C, N, B>();
  int ky, kxt;
  zcol_item((int64_t)blockIdx.y * gridDim.x + blockIdx.x, gridDim.x, ky, kxt);
  const int kx0 = kxt * B;
  const int ncol = min(B, M1 - kx0);
  C* col = S + yoff(L, ky) + xoff(L, kx0);
  load_zcol<C, N, B>(buf, col, L.zs, ncol);
  __syncthreads();
  step1<C, N1, N2, B, false, XP>(buf, B, tws, 1);
  __syncthreads();
  const int c = threadIdx.x % B, k1 = threadIdx.x / B;
  C a[N2];
  step2<C, N1, N2, false, XP>(buf, B, c, k1, a);
  if (c < ncol) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) col[(int64_t)(k1 + N1 * k2) * L.zs + c] = a[k2];
  }
}

// ============================================================================
// X pass, complex-to-real inverse (unnormalised) of half-spectrum lines:
// Z[k] = (X[k] + conj X[M-k]) + i W_N^-k (X[k] - conj X[M-k]), k < M;
// z = IDFT_M(Z) gives x[2m] = Re z[m], x[2m+1] = Im z[m].
// ============================================================================
template <typename C, int N, typename Store>
__device__ __forceinline__ void x_c2r_body(C* buf, int64_t l0, int64_t n_lines, const C* __restrict__ src_of_line0,
                                           int P, const C* tw, Store store);

// C2R of LB lines whose half spectra come from load(line, k), k = 0..N/2.
template <typename C, int N, typename Loader, typename Store>
__device__ __forceinline__ void x_c2r_core(C* buf, int64_t l0, int64_t n_lines, Loader load,
                                           const C* tw, Store store) {
  using X = XPass<C, N>;
  constexpr int M = X::M, LB = X::LB, LD = X::LD, N1 = X::N1, N2 = X::N2;
  for (int idx = threadIdx.x; idx < LB * (M + 1); idx += blockDim.x) {
    const int cc = idx / (M + 1), k = idx % (M + 1);
    const int64_t l = l0 + cc;
    C v;
    v.x = 0; v.y = 0;
    if (l < n_lines) v = load(l, k);
    buf[k * LD + cc] = v;
  }
  __syncthreads();
  // build Z in place: task (line, k) for k in [0, M/2]
  for (int idx = threadIdx.x; idx < LB * (M / 2 + 1); idx += blockDim.x) {
    const int cc = idx / (M / 2 + 1), k = idx % (M / 2 + 1);
    C xk = buf[k * LD + cc];
    C xm = buf[(M - k) * LD + cc];
    // for index k: E = X[k] + conj X[M-k], D = X[k] - conj X[M-k]
    C e1 = make_c<C>(xk.x + xm.x, xk.y - xm.y);
    C d1 = make_c<C>(xk.x - xm.x, xk.y + xm.y);
    C w1 = twid<C, true>(tw, k);
    C o1 = cmul(d1, w1);
    C z1 = make_c<C>(e1.x - o1.y, e1.y + o1.x);   // E + i*O
    // for index M-k: E' = X[M-k] + conj X[k], D' = X[M-k] - conj X[k]
    C e2 = make_c<C>(xm.x + xk.x, xm.y - xk.y);
    C d2 = make_c<C>(xm.x - xk.x, xm.y + xk.y);
    C w2 = twid<C, true>(tw, M - k);
    C o2 = cmul(d2, w2);
    C z2 = make_c<C>(e2.x - o2.y, e2.y + o2.x);
    buf[k * LD + cc] = z1;
    if (k != 0 && k != M - k) buf[(M - k) * LD + cc] = z2;
  }
  __syncthreads();
  step1<C, N1, N2, LB, true>(buf, LD, tw, 2);
  __syncthreads();
  const int c = threadIdx.x % LB, k1 = threadIdx.x / LB;
  C a[N2];
  step2<C, N1, N2, true>(buf, LD, c, k1, a);
  const int64_t l = l0 + c;
  if (l < n_lines) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      const int m = k1 + N1 * k2;
      store(l, 2 * m, a[k2].x);
      store(l, 2 * m + 1, a[k2].y);
    }
  }
}

// Lines l0.. stored contiguously at src_of_line0 with pitch P.
template <typename C, int N, typename Store>
__device__ __forceinline__ void x_c2r_body(C* buf, int64_t l0, int64_t n_lines, const C* __restrict__ src_of_line0,
                                           int P, const C* tw, Store store) {
  x_c2r_core<C, N>(buf, l0, n_lines,
                   [&](int64_t l, int k) { return src_of_line0[(l - l0) * P + k]; }, tw, store);
}

// C2R of scattered lines of a dense half spectrum S[z][y][P]: line l is
// (line_z[l], line_y[l]); out[l][x] = scale * x-line value (the adjoint
// fields at the lines that hold deposited points). line_y == null: the
// lines are compact, line l at S + l * P.
template <typename C, int N>
__global__ void __launch_bounds__(XPass<C, N>::THREADS)
k_x_c2r_lines(const C* __restrict__ S, int P, Lay L, int64_t n_lines, const int32_t* __restrict__ line_y,
              const int32_t* __restrict__ line_z, typename Real<C>::T* __restrict__ out,
              typename Real<C>::T scale, const C* __restrict__ tw) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw) + N;
  const C* tws = stage_tw(reinterpret_cast<C*>(smem_raw), tw, N);
  using RT = typename Real<C>::T;
  const int64_t l0 = (int64_t)blockIdx.x * XPass<C, N>::LB;
  x_c2r_core<C, N>(
      buf, l0, n_lines,
      [&](int64_t l, int k) {
        return line_y ? S[(int64_t)line_z[l] * L.zs + yoff(L, line_y[l]) + xoff(L, k)] : S[l * P + k];
      },
      tws,
      [&](int64_t l, int n, RT v) { out[l * N + n] = v * scale; });
}

// Window lines of one mesh: line = zw*W + yw, output x offsets |x| <= w.
template <typename C, int N>
__global__ void __launch_bounds__(XPass<C, N>::THREADS)
k_x_c2r_win(const C* __restrict__ Wy, int64_t Wy_stride, int w, typename Real<C>::T* __restrict__ Cwin,
            int64_t Cwin_stride, int P, typename Real<C>::T scale, const C* __restrict__ tw) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw) + N;        // twiddles W_N^j first, then the tile
  const C* tws = stage_tw(reinterpret_cast<C*>(smem_raw), tw, N);
  using RT = typename Real<C>::T;
  const int W = 2 * w + 1;
  const int64_t n_lines = (int64_t)W * W;
  const int b = blockIdx.y;
  const int64_t l0 = (int64_t)blockIdx.x * XPass<C, N>::LB;
  const C* src = Wy + (int64_t)b * Wy_stride + l0 * P;
  RT* out = Cwin + (int64_t)b * Cwin_stride;
  x_c2r_body<C, N>(buf, l0, n_lines, src, P, tws, [&](int64_t l, int n, RT v) {
    const int xw = win_index(n, N, w);
    if (xw >= 0) out[l * W + xw] = v * scale;
  });
}

// Full C2R of all N^2 lines (stage entry point).
template <typename C, int N>
__global__ void __launch_bounds__(XPass<C, N>::THREADS)
k_x_c2r_full(const C* __restrict__ S, int P, typename Real<C>::T* __restrict__ out,
             const C* __restrict__ tw) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw) + N;        // twiddles W_N^j first, then the tile
  const C* tws = stage_tw(reinterpret_cast<C*>(smem_raw), tw, N);
  using RT = typename Real<C>::T;
  const int64_t n_lines = (int64_t)N * N;
  const int64_t l0 = (int64_t)blockIdx.x * XPass<C, N>::LB;
  x_c2r_body<C, N>(buf, l0, n_lines, S + l0 * P, P, tws, [&](int64_t l, int n, RT v) {
    out[l * N + n] = v;
  });
}

// Full inverse along z or y in place on a dense half spectrum (stage entry).
template <typename C, int N, int B, bool ALONG_Z>
__global__ void __launch_bounds__(ColPass<C, N, B>::THREADS, ColPass<C, N, B>::MINB)
k_col_inv_full(C* __restrict__ S, Lay L, const C* __restrict__ tw) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw) + N;        // twiddles W_N^j first, then the tile
  const C* tws = stage_tw(reinterpret_cast<C*>(smem_raw), tw, N);
  using CP = ColPass<C, N, B>;
  constexpr int N1 = CP::N1, N2 = CP::N2, M1 = N / 2 + 1;
  constexpr int XP = xperm<C, N, B>();
  int kxt = blockIdx.x, other = blockIdx.y;
  if (ALONG_Z) zcol_item((int64_t)blockIdx.y * gridDim.x + blockIdx.x, gridDim.x, other, kxt);
  const int kx0 = kxt * B;
  const int ncol = min(B, M1 - kx0);
  const int c = threadIdx.x % B;
  // ALONG_Z: column over z at fixed y = other; else over y at fixed z = other
  // row r of the column: z = r (ALONG_Z) or y = r
  auto row = [&](int r) { return ALONG_Z ? (int64_t)r * L.zs : yoff(L, r); };
  C* col = S + (ALONG_Z ? yoff(L, other) : (int64_t)other * L.zs) + xoff(L, kx0);
  for (int r = threadIdx.x / B; r < N; r += blockDim.x / B) {
    C v;
    v.x = 0; v.y = 0;
    if (c < ncol) v = col[row(r) + c];
    buf[r * B + c] = v;
  }
  __syncthreads();
  step1<C, N1, N2, B, true, XP>(buf, B, tws, 1);
  __syncthreads();
  const int k1 = threadIdx.x / B;
  C a[N2];
  step2<C, N1, N2, true, XP>(buf, B, c, k1, a);
  if (c < ncol) {
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) col[row(k1 + N1 * k2) + c] = a[k2];
  }
}

// ============================================================================
// Z pass fused, persistent and TMA fed. A work item is (ky, a tile of B kx
// columns). For each item the CTA loads the galaxy spectrum tile once (and
// scales it by 1/N^3, a power of two, so exactly), then runs every mesh of the
// batch through forward z -> * conj(F_g) / N^3 -> k = 0 zeroed -> inverse z
// -> window rows. While one mesh is transformed the next mesh's tile streams
// into the second shared buffer (TMA + mbarrier), issued by a load warpgroup
// (zc_produce) while the transform warpgroups compute, so HBM reads overlap
// the FFT arithmetic. The inverse's last DFTs compute only the outputs n1 < K and
// n1 >= N1 - K, which hold every window row when K > w / N2 (rows
// n = n2 + N2 n1 with |n| <= w).
// ============================================================================
// Registers per thread for a CTA of CT transform threads (whole warpgroups)
// plus one load warpgroup, MINB CTAs per SM: RLAUNCH is the cap of
// __launch_bounds__(CT + 128, MINB); after the split the load warpgroup keeps
// RP and the transform warpgroups take what it frees, RC, so that
// CT * RC + 128 * RP <= (CT + 128) * RLAUNCH.
template <int CT, int MINB>
struct RegSplit {
  static constexpr int THREADS = CT + 128;
  static constexpr int RLAUNCH_RAW = (65536 / (THREADS * MINB)) & ~7;
  static constexpr int RLAUNCH = RLAUNCH_RAW > 248 ? 248 : RLAUNCH_RAW;
  static constexpr int RP = 24;
  static constexpr int RC_RAW = ((THREADS * RLAUNCH - 128 * RP) / CT) & ~7;
  static constexpr int RC = RC_RAW > 240 ? 240 : RC_RAW;
  static constexpr bool SPLIT = RC > RLAUNCH;   // else every warp keeps the launch count
  static_assert(CT % 128 == 0, "transform threads form whole warpgroups");
  static_assert(!SPLIT || CT * RC + 128 * RP <= THREADS * RLAUNCH, "split exceeds the registers at launch");
};

// Gives the load warpgroup's registers to the transform warpgroups (threads
// below CT); every thread of the CTA calls it once.
template <typename RS>
__device__ __forceinline__ void reg_split(int tid) {
  if constexpr (RS::SPLIT) {
    if (tid >= RS::THREADS - 128) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(RS::RP));
    else asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(RS::RC));
  }
}

template <typename C, int N, int B>
struct ZCorr {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int CTHREADS = B * N1;           // transform warpgroups
  static constexpr int THREADS = CTHREADS + 128;    // + one warpgroup whose first thread issues the loads
  static constexpr int TILE = N * B;
  static constexpr int ZB = N < 256 ? N : 256;   // rows per TMA box
  static constexpr uint32_t TILE_BYTES = TILE * sizeof(C);
  static constexpr int E = sizeof(C) / 8;        // 8-byte TMA elements per complex
  static constexpr size_t SMEM = sizeof(C) * (3 * (size_t)TILE + N) + 64;
  static constexpr int MINB = SMEM <= 110 * 1024 ? 2 : 1;   // resident CTAs per SM
  static constexpr size_t smem_bytes() { return SMEM; }
  using Regs = RegSplit<CTHREADS, MINB>;
};

template <typename C, int N, int B>
__device__ __forceinline__ void zc_issue(C* dst, const CUtensorMap* map, uint64_t* bar, int kx0,
                                         int ky, int b) {
  using Z = ZCorr<C, N, B>;
  tma::mbar_arrive_expect_tx(bar, Z::TILE_BYTES);
  // spectra maps are (kx mod B, y mod 8, kx / B, z, y / 8 + mesh N / 8)
  const uint64_t pol = tma::policy_evict_first();
  constexpr int KM = (1 << kYBlockShift) - 1;
#pragma unroll
  for (int z0 = 0; z0 < N; z0 += Z::ZB)
    tma::load_5d_hint(dst + z0 * B, map, bar, 0, ky & KM, kx0 / B, z0,
                      (ky >> kYBlockShift) + b * (N >> kYBlockShift), pol);
}

// The same column prefetched into L2 (issued one mesh ahead of its load, so
// that the load into shared memory finds it there).
template <typename C, int N, int B>
__device__ __forceinline__ void zc_prefetch(const CUtensorMap* map, int kx0, int ky, int b) {
  using Z = ZCorr<C, N, B>;
  constexpr int KM = (1 << kYBlockShift) - 1;
#pragma unroll
  for (int z0 = 0; z0 < N; z0 += Z::ZB)
    tma::prefetch_5d(map, 0, ky & KM, kx0 / B, z0, (ky >> kYBlockShift) + b * (N >> kYBlockShift));
}

// The load side of the fused z pass, run by one thread of the load
// warpgroup. Barriers: bar[0], bar[1] mesh buffer k loaded; bar[2] galaxy
// tile loaded; bar[3], bar[4] mesh buffer k free again (an arrival from every
// transform warp); bar[5] galaxy tile free again (an arrival from every
// transform thread).
// Per item the order is: first mesh, galaxy tile, remaining meshes, so the
// first mesh of an item streams in while the previous item's last mesh is
// still being transformed. Returns 0, or 1 when a wait for a free buffer ran
// out; copies issued are waited for (bounded) before it returns.
template <typename C, int N, int B>
__device__ int zc_produce(const CUtensorMap* mS, const CUtensorMap* mF, C* sbuf0, C* ftile,
                          uint64_t* bar, int nb, int gg, int64_t n_items, int T, uint64_t limit_ns) {
  using Z = ZCorr<C, N, B>;
  uint32_t issued[3] = {0, 0, 0};
  int64_t job = 0;
  int failed = 0;
  auto mesh = [&](int kx0, int ky, int b) {
    const int s = (int)(job & 1);
    if (job >= 2 && !tma::mbar_wait(&bar[3 + s], (uint32_t)((job >> 1) - 1) & 1, limit_ns)) return false;
    tma::fence_async_shared();
    zc_issue<C, N, B>(sbuf0 + s * Z::TILE, mS, &bar[s], kx0, ky, b);
    ++issued[s];
    ++job;
    return true;
  };
  // the mesh column after the one just issued (the next item's first mesh
  // after an item's last) and the next item's galaxy column go to L2 early
  auto ahead = [&](int64_t item, int kx0, int ky, int b) {
    if (b + 1 < nb) {
      zc_prefetch<C, N, B>(mS, kx0, ky, b + 1);
    } else if (item + gridDim.x < n_items) {
      int ky2, kxt2;
      zcol_item(item + gridDim.x, T, ky2, kxt2);
      zc_prefetch<C, N, B>(mS, kxt2 * B, ky2, 0);
      zc_prefetch<C, N, B>(mF, kxt2 * B, ky2, 0);
    }
  };
  int64_t i = 0;
  for (int64_t item = blockIdx.x; item < n_items && !failed; item += gridDim.x, ++i) {
    int ky, kxt;
    zcol_item(item, T, ky, kxt);
    const int kx0 = kxt * B;
    if (!gg && !mesh(kx0, ky, 0)) { failed = 1; break; }
    if (!gg) ahead(item, kx0, ky, 0);
    if (i > 0 && !tma::mbar_wait(&bar[5], (uint32_t)(i - 1) & 1, limit_ns)) { failed = 1; break; }
    tma::fence_async_shared();
    zc_issue<C, N, B>(ftile, mF, &bar[2], kx0, ky, 0);
    ++issued[2];
    for (int b = 1; b < nb && !gg; ++b) {
      if (!mesh(kx0, ky, b)) { failed = 1; break; }
      ahead(item, kx0, ky, b);
    }
  }
  // every copy issued has landed before the CTA may exit
  for (int k = 0; k < 3; ++k)
    if (issued[k]) tma::mbar_wait(&bar[k], (issued[k] - 1) & 1, failed ? 100000000ull : limit_ns);
  return failed;
}

template <typename C, int N, int B, int K>
__global__ void __launch_bounds__(ZCorr<C, N, B>::THREADS, ZCorr<C, N, B>::MINB)
k_z_corr_tma(const __grid_constant__ CUtensorMap mS, const __grid_constant__ CUtensorMap mF,
             int nb, int gg, int w, C* __restrict__ Wz, int64_t Wz_stride, int P,
             const C* __restrict__ tw, int* __restrict__ err) {
  using Z = ZCorr<C, N, B>;
  using RT = typename Real<C>::T;
  constexpr int N1 = Z::N1, N2 = Z::N2, TILE = Z::TILE, M1 = N / 2 + 1, CT = Z::CTHREADS;
  constexpr int XP = xperm<C, N, B>();
  constexpr uint64_t kLimitNs = 2000000000ull;   // 2 s per wait
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* const sbuf0 = reinterpret_cast<C*>(smem_raw);   // mesh buffers: sbuf0 + k * TILE
  C* ftile = sbuf0 + 2 * TILE;
  C* tws = ftile + TILE;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tws + N);   // see zc_produce
  const int T = (M1 + B - 1) / B;
  const int64_t n_items = (int64_t)T * N;
  int64_t item = blockIdx.x;
  if (item >= n_items) return;   // whole CTA
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += blockDim.x) tws[i] = tw[i];
  if (tid == 0) {
    for (int k = 0; k < 3; ++k) tma::mbar_init(&bar[k], 1);
    for (int k = 3; k < 5; ++k) tma::mbar_init(&bar[k], CT / 32);   // one arrival per transform warp
    tma::mbar_init(&bar[5], CT);   // every transform thread reports its last read of the galaxy tile
    tma::fence_async_shared();
  }
  __syncthreads();
  reg_split<typename Z::Regs>(tid);
  if (tid >= CT) {   // the load warpgroup; the transform warps sync on named barrier 1 from here
    if (tid == CT && zc_produce<C, N, B>(&mS, &mF, sbuf0, ftile, bar, nb, gg, n_items, T, kLimitNs))
      atomicExch(err, tma::kErrTmaTimeout);
    return;
  }
  const int c = tid % B, k1 = tid / B;
  constexpr bool TR = (N1 == N2) && (B * N2 == CT);   // twiddles in registers (step1_tr)
  C tq[N1];
  if constexpr (TR) {
#pragma unroll
    for (int m = 0; m < N1; ++m) tq[m] = tws[(k1 * m) % N];
  }
  const RT inv_n3 = (RT)(1.0 / ((double)N * (double)N * (double)N));
  uint32_t ph[3] = {0, 0, 0};
  int64_t job = 0;
  int failed = 0;
  for (; item < n_items && !failed; item += gridDim.x) {
    int ky, kxt;
    zcol_item(item, T, ky, kxt);
    const int kx0 = kxt * B;
    const int ncol = min(B, M1 - kx0);
    if (tma::bar_or(1, CT, !tma::mbar_wait(&bar[2], ph[2], kLimitNs))) { failed = 1; break; }
    ph[2] ^= 1;
    if (!gg) {   // F_g / N^3 once per item
      for (int i = tid; i < TILE; i += CT) ftile[i] = cscale(ftile[i], inv_n3);
      tma::bar_sync(1, CT);
    }
    const bool dc_col = (kx0 + c == 0) && (ky == 0);
    for (int b = 0; b < nb; ++b, ++job) {
      const int cur = (int)(job & 1);
      C* buf = sbuf0 + cur * TILE;
      C a[N2];
      if (!gg) {
        if (tma::bar_or(1, CT, !tma::mbar_wait(&bar[cur], ph[cur], kLimitNs))) { failed = 1; break; }
        ph[cur] ^= 1;
        if constexpr (TR) step1_tr<C, N1, N2, B, false, XP>(buf, B, tq, tid);
        else step1<C, N1, N2, B, false, XP>(buf, B, tws, 1, tid, CT);
        tma::bar_sync(1, CT);
        step2<C, N1, N2, false, XP>(buf, B, c, k1, a);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) a[k2] = cmulc(a[k2], ftile[(k1 + N1 * k2) * B + c]);
      } else {
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
          const C g = ftile[(k1 + N1 * k2) * B + c];
          a[k2].x = (g.x * g.x + g.y * g.y) * inv_n3;
          a[k2].y = 0;
        }
      }
      if (b == nb - 1) tma::mbar_arrive(&bar[5]);   // this thread is done with the galaxy tile
      if (dc_col && k1 == 0) { a[0].x = 0; a[0].y = 0; }   // k = 0 mode
      C* wbuf = gg ? sbuf0 : buf;
      if constexpr (TR) stepA_own_tr<C, N1, N2, true, XP>(wbuf, B, c, k1, a, tq);
      else stepA_own<C, N1, N2, true, XP>(wbuf, B, c, k1, a, tws, 1);
      tma::bar_sync(1, CT);
      C* wout = Wz + (int64_t)b * Wz_stride + (int64_t)ky * P + kx0;
      for (int t = tid; t < B * N2; t += CT) {
        const int cc = t % B, n2 = t / B;
        C x[N1];
        stepB_own<C, N1, N2, true, XP, K>(wbuf, B, cc, n2, x);
        if (cc < ncol) {
#pragma unroll
          for (int n1 = 0; n1 < N1; ++n1) {
            if (2 * K < N1 && n1 >= K && n1 < N1 - K) continue;   // not computed, not in the window
            const int zw = win_index(n2 + N2 * n1, N, w);
            if (zw >= 0) wout[(int64_t)zw * N * P + cc] = x[n1];
          }
        }
      }
      // each warp frees the mesh buffer once its own reads are done; the next
      // barrier is the next mesh's or item's wait (which also orders the
      // galaxy-only mode's reuse of its single buffer)
      __syncwarp();
      if (!gg && (tid & 31) == 0) tma::mbar_arrive(&bar[3 + cur]);
    }
  }
  if (failed && tid == 0) atomicExch(err, tma::kErrTmaTimeout);
}

// ============================================================================
// Inverse y on the window rows, persistent and TMA fed. A work item is
// (mesh b, window row zw, tile of B kx columns); its column over ky is
// Wz[b][zw][0..N)[kx0..kx0+B). Items alternate between two shared buffers so
// the next column streams in while the current one is transformed; only the
// |y| <= w outputs are stored, to Wy[b][zw][yw][kx]. Those rows y = k1 + N1 k2
// have k2 < K or k2 >= N2 - K for K > w / N1, so step 2 computes only those
// outputs (K is dispatched from w; K >= N2 / 2 computes all).
// ============================================================================
template <typename C, int N, int B>
struct YInv {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int THREADS = B * N1;
  static constexpr int TILE = N * B;
  static constexpr int YB = N < 256 ? N : 256;   // rows per TMA box
  static constexpr uint32_t TILE_BYTES = TILE * sizeof(C);
  static constexpr int E = sizeof(C) / 8;
  static constexpr size_t SMEM = sizeof(C) * (2 * (size_t)TILE + N) + 64;
  static constexpr int MINB = SMEM <= 74 * 1024 ? 3 : SMEM <= 110 * 1024 ? 2 : 1;
  static constexpr size_t smem_bytes() { return SMEM; }
};

template <typename C, int N, int B>
__device__ __forceinline__ void yi_issue(C* dst, const CUtensorMap* map, uint64_t* bar, int kx0,
                                         int zw, int b) {
  using Y = YInv<C, N, B>;
  tma::mbar_arrive_expect_tx(bar, Y::TILE_BYTES);
#pragma unroll
  for (int y0 = 0; y0 < N; y0 += Y::YB) tma::load_4d(dst + y0 * B, map, bar, kx0 * Y::E, y0, zw, b);
}

template <typename C, int N, int B, int K>
__global__ void __launch_bounds__(YInv<C, N, B>::THREADS, YInv<C, N, B>::MINB)
k_y_inv_tma(const __grid_constant__ CUtensorMap mW, int nb, int w, C* __restrict__ Wy,
            int64_t Wy_stride, int P, const C* __restrict__ tw, int* __restrict__ err) {
  using Y = YInv<C, N, B>;
  constexpr int N1 = Y::N1, N2 = Y::N2, TILE = Y::TILE, M1 = N / 2 + 1;
  constexpr int XP = xperm<C, N, B>();
  constexpr uint64_t kLimitNs = 2000000000ull;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* const buf0 = reinterpret_cast<C*>(smem_raw);   // buffers: buf0 + k * TILE
  C* tws = buf0 + 2 * TILE;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tws + N);
  const int W = 2 * w + 1;
  const int T = (M1 + B - 1) / B;
  const int64_t n_items = (int64_t)T * W * nb;
  int64_t item = blockIdx.x;
  if (item >= n_items) return;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = tw[i];
  auto decode = [&](int64_t it, int& kx0, int& zw, int& b) {
    kx0 = (int)(it % T) * B;
    const int64_t r = it / T;
    zw = (int)(r % W);
    b = (int)(r / W);
  };
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::fence_async_shared();
    int kx0, zw, b;
    decode(item, kx0, zw, b);
    yi_issue<C, N, B>(buf0, &mW, &bar[0], kx0, zw, b);
  }
  __syncthreads();
  const int c = threadIdx.x % B, k1 = threadIdx.x / B;
  uint32_t ph[2] = {0, 0};
  int failed = 0;
  for (int64_t job = 0; item < n_items; item += gridDim.x, ++job) {
    const int cur = (int)(job & 1);
    C* buf = buf0 + cur * TILE;
    if (threadIdx.x == 0 && item + gridDim.x < n_items) {
      int kx0n, zwn, bn;
      decode(item + gridDim.x, kx0n, zwn, bn);
      tma::fence_async_shared();
      yi_issue<C, N, B>(buf0 + (cur ^ 1) * TILE, &mW, &bar[cur ^ 1], kx0n, zwn, bn);
    }
    if (__syncthreads_or(!tma::mbar_wait(&bar[cur], ph[cur], kLimitNs))) { failed = 1; break; }
    ph[cur] ^= 1;
    int kx0, zw, b;
    decode(item, kx0, zw, b);
    const int ncol = min(B, M1 - kx0);
    step1<C, N1, N2, B, true, XP>(buf, B, tws, 1);
    __syncthreads();
    C a[N2];
    step2<C, N1, N2, true, XP, K>(buf, B, c, k1, a);
    if (c < ncol) {
      C* out = Wy + (int64_t)b * Wy_stride + (int64_t)zw * W * P + kx0 + c;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int yw = win_index(k1 + N1 * k2, N, w);
        if (yw >= 0) out[(int64_t)yw * P] = a[k2];
      }
    }
    __syncthreads();   // buffer free for the prefetch two items ahead
  }
  if (failed) {
    if (threadIdx.x == 0) {
      atomicExch(err, tma::kErrTmaTimeout);
      for (int k = 0; k < 2; ++k) tma::mbar_wait(&bar[k], ph[k], 100000000ull);
    }
    __syncthreads();
  }
}


// ============================================================================
// Full column transform in place, persistent and TMA fed: every column of a
// dense half spectrum along z (columns (ky, kx tile), rows z) or along y
// (columns (z, kx tile), rows y), forward or inverse (unnormalised). Items
// alternate between two shared buffers, so the next column streams in while
// the current one is transformed; results are stored back in place (each
// column is read and written by the one CTA that owns its item). The tensor
// map covers the plan's tiled layout (tiled = 1; dimensions (kx mod B,
// y mod 8, kx / B, z, y / 8)) or a [z][y][kx] layout whose pitch is a
// multiple of 16 bytes (tiled = 0; dimensions (kx, y, z, 1)).
// ============================================================================
template <typename C, int N, int B>
struct ColT {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int THREADS = B * N1;
  static constexpr int TILE = N * B;
  static constexpr int RB = N < 256 ? N : 256;   // rows per TMA box
  static constexpr uint32_t TILE_BYTES = TILE * sizeof(C);
  static constexpr int E = sizeof(C) / 8;
  static constexpr size_t SMEM = sizeof(C) * (2 * (size_t)TILE + N) + 64;
  static constexpr int MINB = SMEM <= 74 * 1024 ? 3 : SMEM <= 110 * 1024 ? 2 : 1;
  static constexpr size_t smem_bytes() { return SMEM; }
};

template <typename C, int N, int B, bool ALONG_Z>
__device__ __forceinline__ void colt_issue(C* dst, const CUtensorMap* map, uint64_t* bar, int kxt,
                                           int other, int tiled) {
  using Q = ColT<C, N, B>;
  tma::mbar_arrive_expect_tx(bar, Q::TILE_BYTES);
  const uint64_t pol = tma::policy_evict_first();
  constexpr int KM = (1 << kYBlockShift) - 1;
#pragma unroll
  for (int r0 = 0; r0 < N; r0 += Q::RB) {
    if (tiled) {
      if (ALONG_Z) tma::load_5d_hint(dst + r0 * B, map, bar, 0, other & KM, kxt, r0, other >> kYBlockShift, pol);
      else tma::load_5d_hint(dst + r0 * B, map, bar, 0, 0, kxt, other, r0 >> kYBlockShift, pol);
    } else {
      if (ALONG_Z) tma::load_4d(dst + r0 * B, map, bar, kxt * B * Q::E, other, r0, 0);
      else tma::load_4d(dst + r0 * B, map, bar, kxt * B * Q::E, r0, other, 0);
    }
  }
}

template <typename C, int N, int B, bool INV, bool ALONG_Z>
__global__ void __launch_bounds__(ColT<C, N, B>::THREADS, ColT<C, N, B>::MINB)
k_col_tma(const __grid_constant__ CUtensorMap map, int tiled, C* __restrict__ S, Lay L,
          const C* __restrict__ tw, int* __restrict__ err) {
  using Q = ColT<C, N, B>;
  constexpr int N1 = Q::N1, N2 = Q::N2, TILE = Q::TILE, M1 = N / 2 + 1;
  constexpr int XP = xperm<C, N, B>();
  constexpr uint64_t kLimitNs = 2000000000ull;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* const buf0 = reinterpret_cast<C*>(smem_raw);   // buffers: buf0 + k * TILE
  C* tws = buf0 + 2 * TILE;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tws + N);
  const int T = (M1 + B - 1) / B;
  const int64_t n_items = (int64_t)T * N;
  int64_t item = blockIdx.x;
  if (item >= n_items) return;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = tw[i];
  // item -> (kx tile, other): other = ky (along z) or z (along y)
  auto decode = [&](int64_t it, int& kxt, int& other) {
    if (ALONG_Z) {
      zcol_item(it, T, other, kxt);
    } else {
      kxt = (int)(it % T);
      other = (int)(it / T);
    }
  };
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::fence_async_shared();
    int kxt, o;
    decode(item, kxt, o);
    colt_issue<C, N, B, ALONG_Z>(buf0, &map, &bar[0], kxt, o, tiled);
  }
  __syncthreads();
  const int c = threadIdx.x % B, k1 = threadIdx.x / B;
  uint32_t ph[2] = {0, 0};
  int failed = 0;
  for (int64_t job = 0; item < n_items; item += gridDim.x, ++job) {
    const int cur = (int)(job & 1);
    C* buf = buf0 + cur * TILE;
    if (threadIdx.x == 0 && item + gridDim.x < n_items) {
      int kxn, on;
      decode(item + gridDim.x, kxn, on);
      tma::fence_async_shared();
      colt_issue<C, N, B, ALONG_Z>(buf0 + (cur ^ 1) * TILE, &map, &bar[cur ^ 1], kxn, on, tiled);
    }
    if (__syncthreads_or(!tma::mbar_wait(&bar[cur], ph[cur], kLimitNs))) { failed = 1; break; }
    ph[cur] ^= 1;
    int kxt, other;
    decode(item, kxt, other);
    const int kx0 = kxt * B, ncol = min(B, M1 - kx0);
    step1<C, N1, N2, B, INV, XP>(buf, B, tws, 1);
    __syncthreads();
    C a[N2];
    step2<C, N1, N2, INV, XP>(buf, B, c, k1, a);
    if (c < ncol) {
      C* col = S + (ALONG_Z ? yoff(L, other) : (int64_t)other * L.zs) + xoff(L, kx0) + c;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int r = k1 + N1 * k2;
        col[ALONG_Z ? (int64_t)r * L.zs : yoff(L, r)] = a[k2];
      }
    }
    __syncthreads();   // buffer free for the prefetch two items ahead
  }
  if (failed) {
    if (threadIdx.x == 0) {
      atomicExch(err, tma::kErrTmaTimeout);
      for (int k = 0; k < 2; ++k) tma::mbar_wait(&bar[k], ph[k], 100000000ull);
    }
    __syncthreads();
  }
}

// ============================================================================
// Adjoint passes, batched like the forward (reverse sweep of Sec. 2.1's
// correlation through FFTs). A window adjoint field is supported on the
// |r| <= w window, so after its x and y passes only the W = 2w+1 window z
// planes are nonzero; they are held compactly as Xw[b][zr][ky][kx], zr the
// window rank of z (mesh_of_rank). Its z transform zero-pads those rows.
// ============================================================================
__device__ __forceinline__ int mesh_of_rank(int r, int N, int w) { return r <= w ? r : r - (2 * w + 1) + N; }

// Step 1 of the split (see step1) on the zero-padded window column whose
// nonzero rows z <= w and z >= N - w come from the compact slot
// xc[rank * B + c]: reads the slot directly, writes buf like step1.
template <typename C, int N, int B, int X, bool PK = false>
__device__ __forceinline__ void step1_win(C* buf, const C* xc, int w, const C* tw, int tid, int nthr) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  const int W = 2 * w + 1;
  for (int t = tid; t < B * N2; t += nthr) {
    const int c = t % B, j2 = t / B;
    C a[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) {
      const int z = N2 * j1 + j2;
      const int r = z <= w ? z : (z >= N - w ? z - N + W : -1);
      C v;
      v.x = 0; v.y = 0;
      if (r >= 0) v = xc[r * B + c];
      a[j1] = v;
    }
    reg_dft<C, N1, false, N1, PK>(a);
    if (N2 > 1 && j2 > 0) {
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) a[k1] = cmul(a[k1], twid<C, false>(tw, j2 * k1));
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) buf[prow<X>(k1, j2, N2) * B + c] = a[k1];
  }
}

// Step 1 on the same zero-padded window column with the zero inputs pruned.
// Its nonzero rows, signed z = N2 j1 + j2 with |z| <= w, have j1 in [-J, J),
// J = floor(w / N2) + 1. With b_m = a[(m - J) mod N1] for m < NZ (NZ >= 2J a
// power of two, b_m = 0 for m >= 2J):
//   sum_j1 a_j1 W_N1^(j1 k1) = W_N1^(-J k1) Y[k1],  Y[k] = sum_m b_m W_N1^(m k),
// and for k = (N1 / NZ) q + r, W_N1^(m k) = W_NZ^(m q) W_N1^(m r), so Y at
// those k is the NZ-point DFT over m of b_m W_N1^(m r) (compile-time
// twiddles). The factor W_N1^(-J k1) = W_N^(-J N2 k1) joins step 1's twiddle
// W_N^(j2 k1): one table entry W_N^((j2 - J N2) k1 mod N). A task reads NZ
// rows of the compact slot instead of N1, and its DFT costs about half.
// Compact slot rows: signed z >= 0 at z, z < 0 at z + W.
template <typename C, int N, int B, int X, int NZ>
__device__ __forceinline__ void step1_win_p(C* buf, const C* xc, int w, const C* tw, int tid, int nthr) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, R = N1 / NZ;
  static_assert(R * NZ == N1, "NZ divides N1");
  const int W = 2 * w + 1;
  const int J = w / N2 + 1;
  for (int t = tid; t < B * N2; t += nthr) {
    const int c = t % B, j2 = t / B;
    C b[NZ];
#pragma unroll
    for (int m = 0; m < NZ; ++m) {
      const int z = N2 * (m - J) + j2;
      C v;
      v.x = 0; v.y = 0;
      if (m < 2 * J && z >= -w && z <= w) v = xc[(z >= 0 ? z : z + W) * B + c];
      b[m] = v;
    }
    C a[N1];
    dft_few_inputs<C, N1, NZ>(b, a);
    const int base = j2 - J * N2;
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) a[k1] = cmul(a[k1], tw[(base * k1) & (N - 1)]);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) buf[prow<X>(k1, j2, N2) * B + c] = a[k1];
  }
}

// Nonzero-input count of the pruned window step 1 for half-width w (a power
// of two NZ >= 2 (floor(w / N2) + 1)), or 0 where pruning would not pay
// (NZ > N1 / 4) and the full step runs.
template <int N>
__host__ __device__ constexpr int win_nz(int w) {
  constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  int nz = 2;
  while (nz < 2 * (w / N2 + 1)) nz *= 2;
  return nz <= N1 / 4 ? nz : 0;
}

// Y pass forward of the window lines of nb meshes into their W window
// planes. Window line (b, zr, ry) is spec[((b * W + zr) * W + ry) * P] with
// y = mesh_of_rank(ry): the W rows of a column go to a compact slot in
// shared memory (rank ry is slot ry: signed y >= 0 at y, y < 0 at y + W),
// and step 1 reads only them (pruned to its nonzero inputs where that pays).
// CTA = (kx tile, zr, mesh b). The output Xw is [ky / 8][zr][kx / B][ky % 8]
// [kx % B] per mesh (layout XL), so a CTA writes whole 512-byte blocks.
template <typename C, int N, int B>
__global__ void __launch_bounds__(ColPass<C, N, B>::THREADS, ColPass<C, N, B>::MINB)
k_y_fwd_win(const C* __restrict__ spec, int P, int w, C* __restrict__ Xw, int64_t Xw_stride, Lay XL,
            const C* __restrict__ tw) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw) + N;
  const C* tws = stage_tw(reinterpret_cast<C*>(smem_raw), tw, N);
  C* xc = buf + N * B;   // compact slot of the W window rows
  using CP = ColPass<C, N, B>;
  constexpr int N1 = CP::N1, N2 = CP::N2, M1 = N / 2 + 1;
  constexpr int XP = xperm<C, N, B>();
  const int W = 2 * w + 1;
  const int kx0 = blockIdx.x * B, zr = blockIdx.y, b = blockIdx.z;
  const int ncol = min(B, M1 - kx0);
  const int c = threadIdx.x % B;
  const int64_t l0 = ((int64_t)b * W + zr) * W;
  for (int r = threadIdx.x / B; r < W; r += blockDim.x / B) {
    C v;
    v.x = 0; v.y = 0;
    if (c < ncol) v = spec[(l0 + r) * P + kx0 + c];
    xc[r * B + c] = v;
  }
  __syncthreads();
  switch (win_nz<N>(w)) {
    case 2: step1_win_p<C, N, B, XP, 2>(buf, xc, w, tws, threadIdx.x, blockDim.x); break;
    case 4: step1_win_p<C, N, B, XP, 4>(buf, xc, w, tws, threadIdx.x, blockDim.x); break;
    case 8: step1_win_p<C, N, B, XP, 8>(buf, xc, w, tws, threadIdx.x, blockDim.x); break;
    default: step1_win<C, N, B, XP>(buf, xc, w, tws, threadIdx.x, blockDim.x);
  }
  __syncthreads();
  const int k1 = threadIdx.x / B;
  C a[N2];
  step2<C, N1, N2, false, XP>(buf, B, c, k1, a);
  if (c < ncol) {
    C* out = Xw + (int64_t)b * Xw_stride + (int64_t)zr * XL.zs + xoff(XL, kx0) + c;
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) out[yoff(XL, k1 + N1 * k2)] = a[k2];
  }
}

// The same pass, persistent: a work item is (kx tile, zr, mesh b), kx tile
// fastest; its W window rows come by one TMA box (the line spectra as a 2D
// [line][kx] map) into one of two compact slots, so the next item's rows
// stream in while the current one is transformed, and the twiddles are
// staged once per CTA instead of once per item. With ts, the item's output
// column goes back into the tile in natural ky order and thread 0 writes it
// with TMA stores (map mO: boxes of YB ky rows of one zr plane).
template <typename C, int N, int B>
struct YWin {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int THREADS = B * N1;
  static constexpr int TILE = N * B;
  static constexpr int E = sizeof(C) / 8;
  static constexpr int YB = N < 256 ? N : 256;   // ky rows per store box
  // a compact slot of W rows of B values, rounded up to 128 bytes (TMA destination)
  static __host__ __device__ int slot(int W) {
    constexpr int e = 128 / (int)sizeof(C);
    return (W * B + e - 1) / e * e;
  }
  static size_t smem(int W) { return sizeof(C) * (2 * (size_t)slot(W) + TILE + N) + 64; }
};

template <typename C, int N, int B>
__global__ void __launch_bounds__(YWin<C, N, B>::THREADS, 2)
k_y_fwd_win_p(const __grid_constant__ CUtensorMap mL, const __grid_constant__ CUtensorMap mO, int ts, int nb, int w,
              C* __restrict__ Xw, int64_t Xw_stride, Lay XL, const C* __restrict__ tw, int* __restrict__ err) {
  using Y = YWin<C, N, B>;
  constexpr int N1 = Y::N1, N2 = Y::N2, TILE = Y::TILE, M1 = N / 2 + 1;
  constexpr int XP = xperm<C, N, B>();
  constexpr uint64_t kLimitNs = 2000000000ull;
  const int W = 2 * w + 1, WS = Y::slot(W);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* const slot0 = reinterpret_cast<C*>(smem_raw);   // slots: slot0 + k * WS
  C* const buf = slot0 + 2 * WS;
  C* const tws = buf + TILE;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tws + N);
  const int T = (M1 + B - 1) / B;
  const int n_items = T * W * nb;   // the launcher keeps this below 2^31
  int item = blockIdx.x;
  if (item >= n_items) return;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = tw[i];
  const uint32_t slot_bytes = (uint32_t)(W * B * sizeof(C));
  auto issue = [&](int k, int it) {
    const int kxt = it % T, r = it / T;   // r = b W + zr: lines (r W + ry)
    tma::mbar_arrive_expect_tx(&bar[k], slot_bytes);
    tma::load_4d(slot0 + k * WS, &mL, &bar[k], kxt * B * Y::E, r * W, 0, 0);
  };
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::fence_async_shared();
    issue(0, item);
  }
  __syncthreads();
  const uint64_t pol_out = tma::policy_evict_first();
  const int nz = win_nz<N>(w);
  const int c = threadIdx.x % B, k1 = threadIdx.x / B;
  uint32_t ph[2] = {0, 0};
  int failed = 0;
  const int stride = (int)gridDim.x;
  for (int job = 0; item < n_items; item += stride, ++job) {
    const int cur = job & 1;
    if (threadIdx.x == 0 && item < n_items - stride) {
      tma::fence_async_shared();
      issue(cur ^ 1, item + stride);
    }
    if (__syncthreads_or(!tma::mbar_wait(&bar[cur], ph[cur], kLimitNs))) { failed = 1; break; }
    ph[cur] ^= 1;
    const int kx0 = (item % T) * B;
    const int r = item / T;
    const int zr = r % W, b = r / W;
    const int ncol = min(B, M1 - kx0);
    const C* xc = slot0 + cur * WS;
    switch (nz) {
      case 2: step1_win_p<C, N, B, XP, 2>(buf, xc, w, tws, threadIdx.x, blockDim.x); break;
      case 4: step1_win_p<C, N, B, XP, 4>(buf, xc, w, tws, threadIdx.x, blockDim.x); break;
      case 8: step1_win_p<C, N, B, XP, 8>(buf, xc, w, tws, threadIdx.x, blockDim.x); break;
      default: step1_win<C, N, B, XP>(buf, xc, w, tws, threadIdx.x, blockDim.x);
    }
    __syncthreads();
    C a[N2];
    step2<C, N1, N2, false, XP>(buf, B, c, k1, a);
    if (ts) {
      __syncthreads();   // every task has read its step-2 rows
      // the column in natural ky order; past the half spectrum (the last
      // tile's padding columns) zeros
      const bool in = c < ncol;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        C v = a[k2];
        if (!in) { v.x = 0; v.y = 0; }
        buf[(k1 + N1 * k2) * B + c] = v;
      }
      tma::fence_async_shared();
      __syncthreads();   // the column is written; this slot is free again
      if (threadIdx.x == 0) {
#pragma unroll
        for (int y0 = 0; y0 < N; y0 += Y::YB)
          tma::store_5d_hint(&mO, buf + y0 * B, 0, 0, kx0 / B, zr, (y0 >> kYBlockShift) + b * (N >> kYBlockShift),
                             pol_out);
        tma::bulk_commit();
        tma::bulk_wait_read_all();   // the tile may be overwritten after the next barrier
      }
    } else {
      if (c < ncol) {
        C* out = Xw + (int64_t)b * Xw_stride + (int64_t)zr * XL.zs + xoff(XL, kx0) + c;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) out[yoff(XL, k1 + N1 * k2)] = a[k2];
      }
      __syncthreads();   // the tile and this slot are free again
    }
  }
  if (ts && threadIdx.x == 0) tma::bulk_wait_all();
  if (failed) {
    if (threadIdx.x == 0) {
      atomicExch(err, tma::kErrTmaTimeout);
      for (int k = 0; k < 2; ++k) tma::mbar_wait(&bar[k], ph[k], 100000000ull);
    }
    __syncthreads();
  }
}

template <typename C, int N, int B>
struct ZAdj {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int CTHREADS = B * N1;           // transform warpgroups
  static constexpr int THREADS = CTHREADS + 128;    // + one warpgroup whose first thread issues the loads
  using Regs = RegSplit<CTHREADS, 1>;
  static constexpr int TILE = N * B;
  static constexpr int ZB = N < 256 ? N : 256;   // rows per TMA box of a full column
  static constexpr uint32_t TILE_BYTES = TILE * sizeof(C);
  static constexpr int E = sizeof(C) / 8;
  // compact window slot in complex elements: W rows of B, rounded up to 128
  // bytes (a TMA destination in shared memory must be 128-byte aligned)
  static __host__ __device__ int win_slot(int W) {
    constexpr int e = 128 / (int)sizeof(C);
    return (W * B + e - 1) / e * e;
  }
  // two mesh tiles, the A tile, two compact window slots
  static size_t smem(int W) { return sizeof(C) * (3 * (size_t)TILE + 2 * (size_t)win_slot(W) + N) + 64; }
};

// Full z column (N rows) of a spectrum array into dst; the tensor map's
// dimensions are (kx mod B, ky mod 8, kx / B, z, ky / 8 + mesh N / 8).
template <typename C, int N, int B>
__device__ __forceinline__ void za_issue_col(C* dst, const CUtensorMap* map, uint64_t* bar, int kx0,
                                             int ky, int b, uint64_t policy) {
  using Z = ZAdj<C, N, B>;
#pragma unroll
  for (int z0 = 0; z0 < N; z0 += Z::ZB)
    tma::load_5d_hint(dst + z0 * B, map, bar, 0, ky & ((1 << kYBlockShift) - 1), kx0 / B, z0,
                      (ky >> kYBlockShift) + b * (N >> kYBlockShift), policy);
}

// Compact window column (W rows) of Xw into dst; the tensor map's
// dimensions are (kx mod B, ky mod 8, kx / B, zr, ky / 8 + mesh N / 8).
template <typename C, int N, int B>
__device__ __forceinline__ void za_issue_win(C* dst, const CUtensorMap* map, uint64_t* bar, int kx0,
                                             int ky, int b, uint64_t policy) {
  tma::load_5d_hint(dst, map, bar, 0, ky & ((1 << kYBlockShift) - 1), kx0 / B, 0,
                    (ky >> kYBlockShift) + b * (N >> kYBlockShift), policy);
}

// The same column prefetched into L2.
template <typename C, int N, int B>
__device__ __forceinline__ void za_prefetch_col(const CUtensorMap* map, int kx0, int ky, int b) {
  using Z = ZAdj<C, N, B>;
#pragma unroll
  for (int z0 = 0; z0 < N; z0 += Z::ZB)
    tma::prefetch_5d(map, 0, ky & ((1 << kYBlockShift) - 1), kx0 / B, z0,
                     (ky >> kYBlockShift) + b * (N >> kYBlockShift));
}

// Full z column (N rows) from shared memory back to a spectrum array, same
// tensor map and coordinates as za_issue_col.
template <typename C, int N, int B>
__device__ __forceinline__ void za_store_col(const C* src, const CUtensorMap* map, int kx0, int ky, int b,
                                             uint64_t policy) {
  using Z = ZAdj<C, N, B>;
#pragma unroll
  for (int z0 = 0; z0 < N; z0 += Z::ZB)
    tma::store_5d_hint(map, src + z0 * B, 0, ky & ((1 << kYBlockShift) - 1), kx0 / B, z0,
                       (ky >> kYBlockShift) + b * (N >> kYBlockShift), policy);
}

// The load and store side of the adjoint z pass, run by one thread of the
// load warpgroup (barriers as in k_zadj). Per item the order is: first mesh's
// slot, A tile, remaining meshes' slots. Before a slot is refilled, the
// output column the transform warps left in it (Y_b of the job two back) is
// stored over that job's S column; before the A tile is refilled, the
// previous item's A column is stored. Returns 0, or 1 when a wait ran out;
// copies issued are waited for (bounded) before it returns.
template <typename C, int N, int B>
__device__ int za_produce(const CUtensorMap* mS, const CUtensorMap* mX, const CUtensorMap* mA, C* sb0,
                          C* at, C* xb0, int WS, int W, uint64_t* bar, int nb, int64_t n_items, int T,
                          uint64_t limit_ns) {
  using Z = ZAdj<C, N, B>;
  // S, the window columns, A and the outputs pass through once: evict first
  const uint64_t pol = tma::policy_evict_first();
  const uint32_t slot_bytes = Z::TILE_BYTES + (uint32_t)(W * B * sizeof(C));
  uint32_t issued[3] = {0, 0, 0};
  int pkx[2] = {0, 0}, pky[2] = {0, 0}, pb[2] = {0, 0};   // the job each slot holds
  int64_t job = 0, cur_item = 0;
  int failed = 0;
  // the output of job j (in slot j & 1) back to global memory
  auto put = [&](int64_t j) {
    const int k = (int)(j & 1);
    if (!tma::mbar_wait(&bar[3 + k], (uint32_t)(j >> 1) & 1, limit_ns)) return false;
    za_store_col<C, N, B>(sb0 + k * Z::TILE, mS, pkx[k], pky[k], pb[k], pol);
    tma::bulk_commit();
    return true;
  };
  auto slot = [&](int kx0, int ky, int b) {
    const int k = (int)(job & 1);
    if (job >= 2) {
      if (!put(job - 2)) return false;
      tma::bulk_wait_read_all();   // the slot's output has left shared memory
    }
    tma::fence_async_shared();
    tma::mbar_arrive_expect_tx(&bar[k], slot_bytes);
    za_issue_col<C, N, B>(sb0 + k * Z::TILE, mS, &bar[k], kx0, ky, b, pol);
    za_issue_win<C, N, B>(xb0 + k * WS, mX, &bar[k], kx0, ky, b, pol);
    // the next job's S column to L2 (meshes descend within an item; after an
    // item's mesh 0 comes the next item's mesh nb - 1, with its A column)
    if (b > 0) {
      za_prefetch_col<C, N, B>(mS, kx0, ky, b - 1);
    } else if (cur_item + gridDim.x < n_items) {
      int ky2, kxt2;
      zcol_item(cur_item + gridDim.x, T, ky2, kxt2);
      za_prefetch_col<C, N, B>(mS, kxt2 * B, ky2, nb - 1);
      za_prefetch_col<C, N, B>(mA, kxt2 * B, ky2, 0);
    }
    pkx[k] = kx0; pky[k] = ky; pb[k] = b;
    ++issued[k];
    ++job;
    return true;
  };
  // the A column of item number i (tile complete in shared memory) back
  int akx = 0, aky = 0;
  auto put_a = [&](int64_t i) {
    if (!tma::mbar_wait(&bar[5], (uint32_t)i & 1, limit_ns)) return false;
    za_store_col<C, N, B>(at, mA, akx, aky, 0, pol);
    tma::bulk_commit();
    return true;
  };
  int64_t i = 0;
  for (int64_t item = blockIdx.x; item < n_items && !failed; item += gridDim.x, ++i) {
    int ky, kxt;
    zcol_item(item, T, ky, kxt);
    const int kx0 = kxt * B;
    cur_item = item;
    // meshes in descending order (see k_zadj)
    if (nb > 0 && !slot(kx0, ky, nb - 1)) { failed = 1; break; }
    if (i > 0) {
      if (!put_a(i - 1)) { failed = 1; break; }
      tma::bulk_wait_read_all();   // the previous item's A has left shared memory
    }
    tma::fence_async_shared();
    tma::mbar_arrive_expect_tx(&bar[2], Z::TILE_BYTES);
    za_issue_col<C, N, B>(at, mA, &bar[2], kx0, ky, 0, pol);
    akx = kx0; aky = ky;
    ++issued[2];
    for (int j = 1; j < nb; ++j)
      if (!slot(kx0, ky, nb - 1 - j)) { failed = 1; break; }
  }
  // the last two jobs' outputs and the last item's A column
  for (int64_t j = job >= 2 ? job - 2 : 0; j < job && !failed; ++j)
    if (!put(j)) failed = 1;
  if (i > 0 && !failed && !put_a(i - 1)) failed = 1;
  tma::bulk_wait_all();
  for (int k = 0; k < 3; ++k)
    if (issued[k]) tma::mbar_wait(&bar[k], (issued[k] - 1) & 1, failed ? 100000000ull : limit_ns);
  return failed;
}

// Both sides of the adjoint z pass for every mesh b of the batch, per work
// item (ky, kx tile): F_b = z transform of S_b, X_b = z transform of the
// zero-padded window column; A += F_b conj(X_b) accumulates in shared memory
// over the batch (A read and written once per item); then Y_b = inverse z of
// X_b F_g (k = 0 set to zero), left in the slot and stored by TMA over S_b's
// column, which this CTA has already read. Persistent and TMA fed; mesh b's S
// and window tiles share one of two slots so the next mesh streams in during
// the transforms, issued (and the outputs stored) by a load warpgroup
// (za_produce) while the transform warpgroups compute. F_g's column is read
// once per item into registers.
template <typename C, int N, int B>
__global__ void __launch_bounds__(ZAdj<C, N, B>::THREADS, 1)
k_zadj(const __grid_constant__ CUtensorMap mS, const __grid_constant__ CUtensorMap mX,
       const __grid_constant__ CUtensorMap mA, int nb, int w, Lay L, const C* __restrict__ Fg,
       const C* __restrict__ tw, int* __restrict__ err) {
  using Z = ZAdj<C, N, B>;
  static_assert(B * Split<N>::N2 <= Z::CTHREADS, "one step-B task per transform thread");
  constexpr int N1 = Z::N1, N2 = Z::N2, TILE = Z::TILE, M1 = N / 2 + 1, CT = Z::CTHREADS;
  constexpr int XP = xperm<C, N, B>();
  constexpr bool PK = true;   // packed FP32 butterflies (see bfly)
  constexpr uint64_t kLimitNs = 2000000000ull;
  const int W = 2 * w + 1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* const sb0 = reinterpret_cast<C*>(smem_raw);   // slots: sb0 + k * TILE
  C* const at = sb0 + 2 * TILE;                     // A tile
  const int WS = Z::win_slot(W);
  C* const xb0 = at + TILE;                         // compact window slots: xb0 + k * WS
  C* const tws = xb0 + 2 * WS;
  // [0], [1]: slot k loaded; [2]: A tile loaded; [3], [4]: slot k's output
  // ready (one arrival per transform warp); [5]: A tile complete (the same)
  uint64_t* bar = reinterpret_cast<uint64_t*>(tws + N);
  const int T = (M1 + B - 1) / B;
  const int64_t n_items = (int64_t)T * N;
  int64_t item = blockIdx.x;
  if (item >= n_items) return;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += blockDim.x) tws[i] = tw[i];
  if (tid == 0) {
    for (int k = 0; k < 6; ++k) tma::mbar_init(&bar[k], k < 3 ? 1u : (uint32_t)(CT / 32));
    tma::fence_async_shared();
  }
  __syncthreads();
  reg_split<typename Z::Regs>(tid);
  if (tid >= CT) {   // the load warpgroup; the transform warps sync on named barrier 1 from here
    if (tid == CT && za_produce<C, N, B>(&mS, &mX, &mA, sb0, at, xb0, WS, W, bar, nb, n_items, T, kLimitNs))
      atomicExch(err, tma::kErrTmaTimeout);
    return;
  }
  // the item's F_g column is re-read for every mesh of the batch: evict last
  const uint64_t pol_keep = tma::policy_evict_last();
  const int c = tid % B, k1 = tid / B;
  uint32_t ph[3] = {0, 0, 0};
  int64_t job = 0;
  int failed = 0;
  for (; item < n_items && !failed; item += gridDim.x) {
    int ky, kxt;
    zcol_item(item, T, ky, kxt);
    const int kx0 = kxt * B;
    const int ncol = min(B, M1 - kx0);
    const bool dc_col = (kx0 + c == 0) && (ky == 0);
    const C* fcol = Fg + yoff(L, ky) + xoff(L, kx0) + c;
    // the item's galaxy column, the same for every mesh: loaded once per item
    // (its L2 latency overlaps the wait for the item's first tiles)
    C f[N2];
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
      f[k2].x = 0; f[k2].y = 0;
      if (c < ncol) f[k2] = tma::ld_hint(fcol + (int64_t)(k1 + N1 * k2) * L.zs, pol_keep);
    }
    if (tma::bar_or(1, CT, !tma::mbar_wait(&bar[2], ph[2], kLimitNs))) { failed = 1; break; }
    ph[2] ^= 1;
    // meshes in descending order: with the batches also taken last first, A
    // accumulates the pair meshes in descending bin order for any batching
    for (int j = 0; j < nb; ++j, ++job) {   // mesh nb - 1 - j (the load thread's order)
      const int cur = (int)(job & 1);
      C* buf = sb0 + cur * TILE;
      if (tma::bar_or(1, CT, !tma::mbar_wait(&bar[cur], ph[cur], kLimitNs))) { failed = 1; break; }
      ph[cur] ^= 1;
      step1<C, N1, N2, B, false, XP, PK>(buf, B, tws, 1, tid, CT);
      tma::bar_sync(1, CT);
      C a[N2];
      step2<C, N1, N2, false, XP, N2, PK>(buf, B, c, k1, a);
      tma::bar_sync(1, CT);
      // the window column's step 1 (its rows from the compact slot); the
      // pruned form (step1_win_p) needs more registers than this loop has
      // left and measured slower here
      step1_win<C, N, B, XP, PK>(buf, xb0 + cur * WS, w, tws, tid, CT);
      tma::bar_sync(1, CT);
      C x[N2];
      step2<C, N1, N2, false, XP, N2, PK>(buf, B, c, k1, x);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        C* o = &at[(k1 + N1 * k2) * B + c];
        const C t = cmulc(a[k2], x[k2]);   // F_b conj(X_b)
        C v = *o;
        v.x += t.x;
        v.y += t.y;
        *o = v;
      }
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) x[k2] = cmul(x[k2], f[k2]);
      if (dc_col && k1 == 0) { x[0].x = 0; x[0].y = 0; }   // k = 0 mode
      stepA_own<C, N1, N2, true, XP, PK>(buf, B, c, k1, x, tws, 1);
      tma::bar_sync(1, CT);
      {
        // Y_b's column into the slot in natural row order for the TMA store
        // (za_produce). A lane's output rows n2 + N2 n1 were read in step B
        // by lanes whose n2 differs in the bits below X, all in its warp.
        const int cc = tid % B, n2 = tid / B;
        const bool act = tid < B * N2;
        C v[N1];
        if (act) stepB_own<C, N1, N2, true, XP, N1, PK>(buf, B, cc, n2, v);
        __syncwarp();
        if (act) {
#pragma unroll
          for (int n1 = 0; n1 < N1; ++n1) buf[(n2 + N2 * n1) * B + cc] = v[n1];
        }
        tma::fence_async_shared();
      }
      // each warp marks its part of the output column ready for the store
      // (the next barrier is the next mesh's or item's wait)
      __syncwarp();
      if ((tid & 31) == 0) tma::mbar_arrive(&bar[3 + cur]);
    }
    if (failed) break;
    // the item's A column (updated at each task's own positions) is complete:
    // the load thread stores it before the tile is refilled
    tma::fence_async_shared();
    __syncwarp();
    if ((tid & 31) == 0) tma::mbar_arrive(&bar[5]);
  }
  if (failed && tid == 0) atomicExch(err, tma::kErrTmaTimeout);
}

// The galaxy auto-correlation term of the adjoint: A = 2 Re(X) F_g, X the
// z transform of one compact window spectrum (mesh 0 of the window map: the
// y-transformed window field, W nonzero z rows per column), computed per work
// item (ky, kx tile) from the W rows alone (pruned step 1) and combined with
// the F_g column on the way out, so the dense spectrum X never exists.
// Persistent; the W rows of the next item stream into the other compact slot
// by TMA while the current item is transformed.
template <typename C, int N, int B>
__global__ void __launch_bounds__(YWin<C, N, B>::THREADS, 2)
k_zwin_acc(const __grid_constant__ CUtensorMap mX, int w, Lay L, const C* __restrict__ Fg,
           C* __restrict__ A, const C* __restrict__ tw, int* __restrict__ err) {
  using Y = YWin<C, N, B>;
  constexpr int N1 = Y::N1, N2 = Y::N2, TILE = Y::TILE, M1 = N / 2 + 1;
  constexpr int XP = xperm<C, N, B>();
  constexpr uint64_t kLimitNs = 2000000000ull;
  const int W = 2 * w + 1, WS = Y::slot(W);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* const slot0 = reinterpret_cast<C*>(smem_raw);   // slots: slot0 + k * WS
  C* const buf = slot0 + 2 * WS;
  C* const tws = buf + TILE;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tws + N);
  const int T = (M1 + B - 1) / B;
  const int n_items = T * N;
  int item = blockIdx.x;
  if (item >= n_items) return;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = tw[i];
  const uint32_t slot_bytes = (uint32_t)(W * B * sizeof(C));
  const uint64_t pol = tma::policy_evict_first();
  auto issue = [&](int k, int it) {
    int ky, kxt;
    zcol_item(it, T, ky, kxt);
    tma::mbar_arrive_expect_tx(&bar[k], slot_bytes);
    za_issue_win<C, N, B>(slot0 + k * WS, &mX, &bar[k], kxt * B, ky, 0, pol);
  };
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::fence_async_shared();
    issue(0, item);
  }
  __syncthreads();
  const int nz = win_nz<N>(w);
  const int c = threadIdx.x % B, k1 = threadIdx.x / B;
  uint32_t ph[2] = {0, 0};
  int failed = 0;
  const int stride = (int)gridDim.x;
  for (int job = 0; item < n_items; item += stride, ++job) {
    const int cur = job & 1;
    if (threadIdx.x == 0 && item < n_items - stride) {
      tma::fence_async_shared();
      issue(cur ^ 1, item + stride);
    }
    if (__syncthreads_or(!tma::mbar_wait(&bar[cur], ph[cur], kLimitNs))) { failed = 1; break; }
    ph[cur] ^= 1;
    int ky, kxt;
    zcol_item(item, T, ky, kxt);
    const int kx0 = kxt * B;
    const int ncol = min(B, M1 - kx0);
    const C* xc = slot0 + cur * WS;
    switch (nz) {
      case 2: step1_win_p<C, N, B, XP, 2>(buf, xc, w, tws, threadIdx.x, blockDim.x); break;
      case 4: step1_win_p<C, N, B, XP, 4>(buf, xc, w, tws, threadIdx.x, blockDim.x); break;
      case 8: step1_win_p<C, N, B, XP, 8>(buf, xc, w, tws, threadIdx.x, blockDim.x); break;
      default: step1_win<C, N, B, XP>(buf, xc, w, tws, threadIdx.x, blockDim.x);
    }
    __syncthreads();
    typename Real<C>::T r[N2];
    {
      C x[N2];
      step2<C, N1, N2, false, XP>(buf, B, c, k1, x);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) r[k2] = 2 * x[k2].x;
    }
    if (c < ncol) {
      const int64_t o = yoff(L, ky) + xoff(L, kx0) + c;
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        const int64_t zo = o + (int64_t)(k1 + N1 * k2) * L.zs;
        const C g = tma::ld_hint(Fg + zo, pol);
        C v;
        v.x = r[k2] * g.x;
        v.y = r[k2] * g.y;
        tma::st_hint(A + zo, v, pol);
      }
    }
    __syncthreads();   // the tile and this slot are free again
  }
  if (failed) {
    if (threadIdx.x == 0) {
      atomicExch(err, tma::kErrTmaTimeout);
      for (int k = 0; k < 2; ++k) tma::mbar_wait(&bar[k], ph[k], 100000000ull);
    }
    __syncthreads();
  }
}

// Inverse y of Y_b on the z planes that hold lines of mesh b, stored only at
// those lines: hspec[line][kx] for the compact lines of the batch (the
// forward deposit's numbering: idx, seg_total, line_base, line_y). Work item
// = (kx tile, z, mesh b); items whose plane holds no lines are skipped by the
// leader thread, which streams the next item's column into the other buffer.
template <typename C, int N, int B>
struct YLines {
  static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2;
  static constexpr int THREADS = B * N1;
  static constexpr int TILE = N * B;
  static constexpr int YB = N < 256 ? N : 256;   // rows per TMA box
  static constexpr uint32_t TILE_BYTES = TILE * sizeof(C);
  static constexpr int E = sizeof(C) / 8;
  static constexpr size_t SMEM = sizeof(C) * (2 * (size_t)TILE + N) + 128;
  static constexpr int MINB = SMEM <= 74 * 1024 ? 3 : SMEM <= 110 * 1024 ? 2 : 1;
  static constexpr size_t smem_bytes() { return SMEM; }
};

template <typename C, int N, int B>
__global__ void __launch_bounds__(YLines<C, N, B>::THREADS, YLines<C, N, B>::MINB)
k_y_inv_lines(const __grid_constant__ CUtensorMap mY, int nb, int P, const int32_t* __restrict__ idx,
              const int64_t* __restrict__ seg_total, const int64_t* __restrict__ line_base,
              const int32_t* __restrict__ line_y, C* __restrict__ hspec, const C* __restrict__ tw,
              int* __restrict__ err) {
  using Y = YLines<C, N, B>;
  constexpr int N1 = Y::N1, N2 = Y::N2, TILE = Y::TILE, M1 = N / 2 + 1;
  constexpr int XP = xperm<C, N, B>();
  constexpr uint64_t kLimitNs = 2000000000ull;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  C* const buf0 = reinterpret_cast<C*>(smem_raw);   // buffers: buf0 + k * TILE
  C* const tws = buf0 + 2 * TILE;
  uint64_t* bar = reinterpret_cast<uint64_t*>(tws + N);
  int64_t* s_item = reinterpret_cast<int64_t*>(bar + 2);   // [2] item per buffer
  int64_t* s_lo = s_item + 2;                              // [2] line range
  int64_t* s_hi = s_lo + 2;
  int64_t* s_base = s_hi + 2;                              // [2] the mesh's first line
  const int T = (M1 + B - 1) / B;
  const int64_t NN = (int64_t)N * N;
  const int64_t n_items = (int64_t)T * N * nb;
  // first item at or after `it` (stride gridDim.x) whose plane holds lines
  auto find = [&](int64_t it, int64_t& lo, int64_t& hi, int64_t& base) {
    for (; it < n_items; it += gridDim.x) {
      const int64_t r = it / T;
      const int z = (int)(r % N), b = (int)(r / N);
      const int32_t* ib = idx + (int64_t)b * NN;
      lo = ib[(int64_t)z * N];
      hi = (z + 1 < N) ? ib[(int64_t)(z + 1) * N] : seg_total[b];
      if (lo < hi) {
        base = line_base[b];
        return it;
      }
    }
    return n_items;
  };
  const uint64_t pol_stream = tma::policy_evict_first();
  auto issue = [&](int k, int64_t it) {
    const int64_t r = it / T;
    tma::mbar_arrive_expect_tx(&bar[k], Y::TILE_BYTES);
#pragma unroll
    for (int y0 = 0; y0 < N; y0 += Y::YB)
      tma::load_5d_hint(buf0 + k * TILE + y0 * B, &mY, &bar[k], 0, 0, (int)(it % T), (int)(r % N),
                        (y0 >> kYBlockShift) + (int)(r / N) * (N >> kYBlockShift), pol_stream);
  };
  for (int i = threadIdx.x; i < N; i += blockDim.x) tws[i] = tw[i];
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::fence_async_shared();
    for (int k = 0; k < 2; ++k) {
      const int64_t it = find(k == 0 ? (int64_t)blockIdx.x : s_item[0] + gridDim.x, s_lo[k], s_hi[k], s_base[k]);
      s_item[k] = it;
      if (it < n_items) issue(k, it);
      else break;
    }
    if (s_item[0] >= n_items) s_item[1] = n_items;
  }
  __syncthreads();
  const int c = threadIdx.x % B, k1 = threadIdx.x / B;
  uint32_t ph[2] = {0, 0};
  int failed = 0;
  for (int64_t job = 0;; ++job) {
    const int cur = (int)(job & 1);
    const int64_t it = s_item[cur];
    if (it >= n_items) break;
    C* buf = buf0 + cur * TILE;
    if (__syncthreads_or(!tma::mbar_wait(&bar[cur], ph[cur], kLimitNs))) { failed = 1; break; }
    ph[cur] ^= 1;
    const int kx0 = (int)(it % T) * B;
    const int ncol = min(B, M1 - kx0);
    const int64_t lo = s_lo[cur], hi = s_hi[cur], base = s_base[cur];
    // A plane with few lines (at most two outputs per thread) takes each
    // needed output y = k1 + N1 k2 straight from step 1's rows as the N2-point
    // sum over j2 of row (k1, j2) W_N2^(+j2 k2); otherwise step 2 runs whole
    // and the lines are gathered from it.
    constexpr int RSY = Y::THREADS / B, PRE = 2;
    const bool direct = (hi - lo) * B <= 2 * Y::THREADS;
    // line numbers of the first rounds, loaded while the item is transformed
    int yv[PRE];
#pragma unroll
    for (int p = 0; p < PRE; ++p) {
      const int64_t q = direct ? lo + ((int64_t)threadIdx.x + (int64_t)p * Y::THREADS) / B
                               : lo + k1 + (int64_t)p * RSY;
      yv[p] = q < hi ? line_y[base + q] : 0;
    }
    step1<C, N1, N2, B, true, XP>(buf, B, tws, 1);
    __syncthreads();   // every thread has read this buffer's item data
    // the item after next, looked up now so that its index loads overlap the
    // transform; its tile is requested once this buffer is free
    if (threadIdx.x == 0) {
      const int64_t nx = s_item[cur ^ 1];
      s_item[cur] = nx < n_items ? find(nx + gridDim.x, s_lo[cur], s_hi[cur], s_base[cur]) : n_items;
    }
    if (direct) {
#pragma unroll
      for (int p = 0; p < PRE; ++p) {
        const int t = threadIdx.x + p * Y::THREADS;
        const int64_t q = lo + t / B;
        const int cc = t % B;
        if (q < hi && cc < ncol) {
          const int kk1 = yv[p] % N1, kk2 = yv[p] / N1;
          C acc;
          acc.x = 0; acc.y = 0;
#pragma unroll
          for (int j2 = 0; j2 < N2; ++j2) {
            const C v = buf[prow<XP>(kk1, j2, N2) * B + cc];
            const C w = twid<C, true>(tws, ((j2 * kk2) % N2) * N1);   // W_N2^(+j2 k2) = W_N^(+N1 j2 k2)
            acc.x = fmadd(v.x, w.x, fmadd(-v.y, w.y, acc.x));
            acc.y = fmadd(v.x, w.y, fmadd(v.y, w.x, acc.y));
          }
          hspec[(base + q) * P + kx0 + cc] = acc;
        }
      }
    } else {
      C a[N2];
      step2<C, N1, N2, true, XP>(buf, B, c, k1, a);
      __syncthreads();
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) buf[(k1 + N1 * k2) * B + c] = a[k2];   // natural row y
      __syncthreads();
#pragma unroll
      for (int p = 0; p < PRE; ++p) {
        const int64_t q = lo + k1 + (int64_t)p * RSY;
        if (q < hi && c < ncol) hspec[(base + q) * P + kx0 + c] = buf[yv[p] * B + c];
      }
      for (int64_t q = lo + k1 + (int64_t)PRE * RSY; q < hi; q += RSY) {
        const int64_t l = base + q;
        if (c < ncol) hspec[l * P + kx0 + c] = buf[line_y[l] * B + c];
      }
    }
    __syncthreads();   // buffer free: stream in the item after the next
    if (threadIdx.x == 0 && s_item[cur] < n_items) {
      tma::fence_async_shared();
      issue(cur, s_item[cur]);
    }
  }
  if (failed) {
    if (threadIdx.x == 0) {
      atomicExch(err, tma::kErrTmaTimeout);
      for (int k = 0; k < 2; ++k) tma::mbar_wait(&bar[k], ph[k], 100000000ull);
    }
    __syncthreads();
  }
}

}  // namespace fft
}  // namespace pg
