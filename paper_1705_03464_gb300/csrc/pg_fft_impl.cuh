// Host launchers of the FFT passes: dispatch on the mesh size N and set the
// dynamic shared-memory limits. Instantiated per precision.
#pragma once

#include "pg_fft_kernels.cuh"

namespace pg {

template <typename K>
static cudaError_t set_smem(K kern, size_t bytes) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

namespace fft {
template <typename R> struct Cols;
// 64 KB column tiles, 256 threads: two or three CTAs share an SM, so one
// CTA's loads overlap another's arithmetic
template <> struct Cols<float> { static constexpr int B = 8; };
template <> struct Cols<double> { static constexpr int B = 4; };
// Tile width of the persistent TMA passes (fused z pass, windowed y
// inverse): 64 KB tiles.
template <typename R> struct ZCols;
template <> struct ZCols<float> { static constexpr int B = 8; };
template <> struct ZCols<double> { static constexpr int B = 4; };

// Resident CTAs per SM of a persistent kernel, at least one.
template <typename K>
static cudaError_t persistent_grid(K kern, int threads, size_t smem, int64_t items, unsigned* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  PG_CUDA_TRY(cudaGetDevice(&dev));
  PG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  PG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
  *grid = (unsigned)std::min<int64_t>(items, (int64_t)sms * std::max(1, per_sm));
  return cudaSuccess;
}

// A kernel that splits its registers (RegSplit) grows its transform
// warpgroups into the registers its load warpgroup gives back: it may only be
// launched if it was built with the launch cap the split assumes.
template <typename RS, typename K>
static cudaError_t check_reg_split(K kern) {
  if constexpr (RS::SPLIT) {
    cudaFuncAttributes fa;
    PG_CUDA_TRY(cudaFuncGetAttributes(&fa, kern));
    if ((int64_t)fa.numRegs * RS::THREADS < (int64_t)(RS::THREADS - 128) * RS::RC + 128 * RS::RP)
      return cudaErrorInvalidConfiguration;
  }
  return cudaSuccess;
}

// Tensor map over 8-byte elements of nb spectra of the plan layout L (each
// N*N*P complex, kx in tiles of B = 2^L.txs complex values of 64 bytes, ky in
// blocks of K = 2^L.ks rows), dimensions (kx mod B, y mod K, kx / B, z,
// y / K + mesh N / K) (the meshes follow one another, so the last two indices
// of a mesh's blocks merge into one), box (one kx tile, then either bz z rows
// of one y (by = 1) or by y rows of one z (bz = 1)).
template <typename R, int B = ZCols<R>::B>
static bool spec_map(CUtensorMap* m, const void* base, int N, int P, Lay L, int nb, uint32_t bz,
                     uint32_t by) {
  using C = typename CT<R>::C;
  constexpr int E = (int)(sizeof(C) / 8);
  const int K = 1 << L.ks;
  if (K > N || N % K != 0 || (by > 1 && by % K != 0)) return false;
  if ((1 << L.txs) != B || P % B != 0 || L.ys != B || L.ts != (int64_t)K * B ||
      L.zs != (int64_t)K * P || L.hs != (int64_t)N * K * P)
    return false;
  const uint64_t dims[5] = {(uint64_t)B * E, (uint64_t)K, (uint64_t)(P / B), (uint64_t)N,
                            (uint64_t)(N / K) * nb};
  const uint64_t strides[4] = {(uint64_t)L.ys * 8 * E, (uint64_t)L.ts * 8 * E, (uint64_t)L.zs * 8 * E,
                               (uint64_t)L.hs * 8 * E};
  const uint32_t box[5] = {(uint32_t)(B * E), by > 1 ? (uint32_t)K : 1u, 1u, bz, by > 1 ? by / (uint32_t)K : 1u};
  return encode_map_5d(m, base, dims, strides, box);
}
// Tensor map of the persistent column pass over one dense half spectrum in
// layout L: the plan's tiled layout (*tiled = 1, spec_map), or [z][y][kx]
// with a pitch of a multiple of 16 bytes (*tiled = 0; dimensions (kx, y, z,
// 1), box one kx tile by rb rows along the column). False where neither
// applies (the caller then runs the column pass without TMA).
template <typename R>
static bool col_map(CUtensorMap* m, const void* base, int N, int P, Lay L, bool along_z, uint32_t rb,
                    int* tiled) {
  using C = typename CT<R>::C;
  constexpr int B = Cols<R>::B, E = (int)(sizeof(C) / 8);
  if (L.txs > 0) {
    *tiled = 1;
    return spec_map<R, B>(m, base, N, P, L, 1, along_z ? rb : 1u, along_z ? 1u : rb);
  }
  if (L.ks < 30 || L.ys != P || L.zs != (int64_t)N * P || ((int64_t)P * (int64_t)sizeof(C)) % 16 != 0)
    return false;
  *tiled = 0;
  const uint64_t dims[4] = {(uint64_t)P * E, (uint64_t)N, (uint64_t)N, 1u};
  const uint64_t strides[3] = {(uint64_t)P * 8 * E, (uint64_t)N * P * 8 * E, (uint64_t)N * N * P * 8 * E};
  const uint32_t box[4] = {(uint32_t)(B * E), along_z ? 1u : rb, along_z ? rb : 1u, 1u};
  return encode_map_4d(m, base, dims, strides, box);
}

// Runs the persistent TMA column pass when a map of S can be encoded, else
// the plain column kernel `plain`; true when the TMA pass was launched.
template <typename R, int NN, bool INV, bool ALONG_Z>
static cudaError_t col_pass(typename CT<R>::C* S, int P, Lay L, const typename CT<R>::C* tw, int* err,
                            cudaStream_t s, bool* used_tma) {
  using C = typename CT<R>::C;
  constexpr int B = Cols<R>::B;
  using Q = ColT<C, NN, B>;
  CUtensorMap m;
  int tiled = 0;
  *used_tma = false;
  if (!err || !col_map<R>(&m, S, NN, P, L, ALONG_Z, (uint32_t)Q::RB, &tiled)) return cudaSuccess;
  auto k = k_col_tma<C, NN, B, INV, ALONG_Z>;
  PG_CUDA_TRY(set_smem(k, Q::smem_bytes()));
  unsigned grid = 0;
  PG_CUDA_TRY(persistent_grid(k, Q::THREADS, Q::smem_bytes(), cdiv(NN / 2 + 1, B) * (int64_t)NN, &grid));
  k<<<grid, Q::THREADS, Q::smem_bytes(), s>>>(m, tiled, S, L, tw, err);
  *used_tma = true;
  return cudaSuccess;
}
}  // namespace fft

#define PG_DISPATCH_N(N, ...)                               \
  switch (N) {                                              \
    case 32: { constexpr int NN = 32; __VA_ARGS__; break; } \
    case 64: { constexpr int NN = 64; __VA_ARGS__; break; } \
    case 128: { constexpr int NN = 128; __VA_ARGS__; break; } \
    case 256: { constexpr int NN = 256; __VA_ARGS__; break; } \
    case 512: { constexpr int NN = 512; __VA_ARGS__; break; } \
    case 1024: { constexpr int NN = 1024; __VA_ARGS__; break; } \
    default: return cudaErrorInvalidValue;                  \
  }


template <typename R>
int FftPasses<R>::cols() { return fft::Cols<R>::B; }

template <typename R>
cudaError_t FftPasses<R>::x_r2c_lines(int N, const int64_t* q, const int32_t* line_bin,
                                      const double* scale, int64_t n_lines, C* spec, int P,
                                      const C* tw, cudaStream_t s) {
  if (n_lines <= 0) return cudaSuccess;
  PG_DISPATCH_N(N, {
    using X = fft::XPass<C, NN>;
    auto k = fft::k_x_r2c_lines<C, NN>;
    PG_CUDA_TRY(set_smem(k, X::smem_bytes()));
    k<<<(unsigned)cdiv(n_lines, X::LB), X::THREADS, X::smem_bytes(), s>>>(q, line_bin, scale, n_lines, spec, P, tw);
  });
  return launched();
}

template <typename R>
cudaError_t FftPasses<R>::x_r2c_dense(int N, const R* f, C* spec, int P, const C* tw, cudaStream_t s) {
  const int64_t n_lines = (int64_t)N * N;
  PG_DISPATCH_N(N, {
    using X = fft::XPass<C, NN>;
    auto k = fft::k_x_r2c_dense<C, NN>;
    PG_CUDA_TRY(set_smem(k, X::smem_bytes()));
    k<<<(unsigned)cdiv(n_lines, X::LB), X::THREADS, X::smem_bytes(), s>>>(f, n_lines, spec, P, tw);
  });
  return launched();
}

template <typename R>
cudaError_t FftPasses<R>::y_fwd(int N, int nb, const C* spec, int P, const int32_t* idx,
                                const int64_t* seg_total, const int64_t* line_base,
                                const int32_t* line_y, C* S, int64_t S_stride, Lay L,
                                const C* tw, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  constexpr int B = fft::Cols<R>::B;
  static_assert(fft::Cols<R>::B == fft::ZCols<R>::B, "one tile width for the spectra maps");
  // TMA stores where the output is the plan's tiled layout with meshes back to back
  CUtensorMap mO;
  const bool ts = S_stride == (int64_t)N * N * P && spec != S &&
                  fft::spec_map<R>(&mO, S, N, P, L, nb, 1, N < 256 ? (uint32_t)N : 256u);
  if (!ts) memset(&mO, 0, sizeof(mO));
  PG_DISPATCH_N(N, {
    auto run = [&](auto tsc) -> cudaError_t {
      constexpr bool TS = decltype(tsc)::value;
      using Y = fft::YFwd<C, NN, B, TS>;
      auto k = fft::k_y_fwd_p<C, NN, B, TS>;
      PG_CUDA_TRY(set_smem(k, Y::smem_bytes()));
      unsigned grid = 0;
      PG_CUDA_TRY(fft::persistent_grid(k, Y::THREADS, Y::smem_bytes(), cdiv(NN / 2 + 1, B) * (int64_t)NN * nb, &grid));
      k<<<grid, Y::THREADS, Y::smem_bytes(), s>>>(mO, spec, P, nb, idx, seg_total, line_base, line_y, S, S_stride,
                                                  L, tw);
      return launched();
    };
    if (ts) PG_CUDA_TRY(run(std::true_type{}));
    else PG_CUDA_TRY(run(std::false_type{}));
  });
  return launched();
}

template <typename R>
cudaError_t FftPasses<R>::z_fwd(int N, C* S, int P, Lay L, const C* tw, int* err, cudaStream_t s) {
  constexpr int B = fft::Cols<R>::B;
  PG_DISPATCH_N(N, {
    bool tma_used = false;
    PG_CUDA_TRY((fft::col_pass<R, NN, false, true>(S, P, L, tw, err, s, &tma_used)));
    if (tma_used) return launched();
    using CP = fft::ColPass<C, NN, B>;
    auto k = fft::k_z_fwd<C, NN, B>;
    PG_CUDA_TRY(set_smem(k, CP::smem_bytes()));
    dim3 g((unsigned)cdiv(NN / 2 + 1, B), NN);
    k<<<g, CP::THREADS, CP::smem_bytes(), s>>>(S, L, tw);
  });
  return launched();
}

template <typename R>
cudaError_t FftPasses<R>::y_inv_win(int N, int nb, const C* Wz, int64_t Wz_stride, int w, C* Wy,
                                    int64_t Wy_stride, int P, const C* tw, int* err,
                                    cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  constexpr int B = fft::ZCols<R>::B;
  constexpr int E = (int)(sizeof(C) / 8);
  const int W = 2 * w + 1;
  // Wz as [bin][zw][ky][kx] over 8-byte elements
  const uint64_t dims[4] = {(uint64_t)P * E, (uint64_t)N, (uint64_t)W, (uint64_t)nb};
  const uint64_t strides[3] = {(uint64_t)P * 8 * E, (uint64_t)N * P * 8 * E,
                               (uint64_t)Wz_stride * 8 * E};
  const uint32_t box[4] = {(uint32_t)(B * E), N < 256 ? (uint32_t)N : 256u, 1u, 1u};
  CUtensorMap mW;
  if (!encode_map_4d(&mW, Wz, dims, strides, box)) return cudaErrorInvalidValue;
  // outputs y = k1 + N1 k2 with |y| <= w need k2 < K or k2 >= N2 - K, K = floor(w / N1) + 1
  const int kreq = w / (N < 32 ? N : 32) + 1;
  PG_DISPATCH_N(N, {
    auto run = [&](auto kc) -> cudaError_t {
      constexpr int K = decltype(kc)::value;
      using Y = fft::YInv<C, NN, B>;
      auto k = fft::k_y_inv_tma<C, NN, B, K>;
      PG_CUDA_TRY(set_smem(k, Y::smem_bytes()));
      unsigned grid = 0;
      PG_CUDA_TRY(fft::persistent_grid(k, Y::THREADS, Y::smem_bytes(), cdiv(NN / 2 + 1, B) * (int64_t)W * nb, &grid));
      k<<<grid, Y::THREADS, Y::smem_bytes(), s>>>(mW, nb, w, Wy, Wy_stride, P, tw, err);
      return launched();
    };
    if (kreq <= 2) PG_CUDA_TRY(run(std::integral_constant<int, 2>{}));
    else if (kreq <= 4) PG_CUDA_TRY(run(std::integral_constant<int, 4>{}));
    else if (kreq <= 8) PG_CUDA_TRY(run(std::integral_constant<int, 8>{}));
    else PG_CUDA_TRY(run(std::integral_constant<int, 32>{}));
  });
  return launched();
}

template <typename R>
cudaError_t FftPasses<R>::x_c2r_win(int N, int nb, const C* Wy, int64_t Wy_stride, int w, R* Cwin,
                                    int64_t Cwin_stride, int P, double scale, const C* tw,
                                    cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  const int64_t n_lines = (int64_t)(2 * w + 1) * (2 * w + 1);
  PG_DISPATCH_N(N, {
    using X = fft::XPass<C, NN>;
    auto k = fft::k_x_c2r_win<C, NN>;
    PG_CUDA_TRY(set_smem(k, X::smem_bytes()));
    dim3 g((unsigned)cdiv(n_lines, X::LB), nb);
    k<<<g, X::THREADS, X::smem_bytes(), s>>>(Wy, Wy_stride, w, Cwin, Cwin_stride, P, (R)scale, tw);
  });
  return launched();
}

template <typename R>
cudaError_t FftPasses<R>::z_inv_full(int N, C* S, int P, Lay L, const C* tw, int* err, cudaStream_t s) {
  constexpr int B = fft::Cols<R>::B;
  PG_DISPATCH_N(N, {
    bool tma_used = false;
    PG_CUDA_TRY((fft::col_pass<R, NN, true, true>(S, P, L, tw, err, s, &tma_used)));
    if (tma_used) return launched();
    using CP = fft::ColPass<C, NN, B>;
    auto k = fft::k_col_inv_full<C, NN, B, true>;
    PG_CUDA_TRY(set_smem(k, CP::smem_bytes()));
    dim3 g((unsigned)cdiv(NN / 2 + 1, B), NN);
    k<<<g, CP::THREADS, CP::smem_bytes(), s>>>(S, L, tw);
  });
  return launched();
}

template <typename R>
cudaError_t FftPasses<R>::y_inv_full(int N, C* S, int P, Lay L, const C* tw, int* err, cudaStream_t s) {
  constexpr int B = fft::Cols<R>::B;
  PG_DISPATCH_N(N, {
    bool tma_used = false;
    PG_CUDA_TRY((fft::col_pass<R, NN, true, false>(S, P, L, tw, err, s, &tma_used)));
    if (tma_used) return launched();
    using CP = fft::ColPass<C, NN, B>;
    auto k = fft::k_col_inv_full<C, NN, B, false>;
    PG_CUDA_TRY(set_smem(k, CP::smem_bytes()));
    dim3 g((unsigned)cdiv(NN / 2 + 1, B), NN);
    k<<<g, CP::THREADS, CP::smem_bytes(), s>>>(S, L, tw);
  });
  return launched();
}

template <typename R>
cudaError_t FftPasses<R>::x_c2r_full(int N, const C* S, int P, R* out, const C* tw, cudaStream_t s) {
  const int64_t n_lines = (int64_t)N * N;
  PG_DISPATCH_N(N, {
    using X = fft::XPass<C, NN>;
    auto k = fft::k_x_c2r_full<C, NN>;
    PG_CUDA_TRY(set_smem(k, X::smem_bytes()));
    k<<<(unsigned)cdiv(n_lines, X::LB), X::THREADS, X::smem_bytes(), s>>>(S, P, out, tw);
  });
  return launched();
}

template <typename R>
cudaError_t FftPasses<R>::set_smem_limits() { return cudaSuccess; }

template <typename R>
cudaError_t FftPasses<R>::x_r2c_real(int N, const R* f, int64_t n_lines, C* spec, int P, const C* tw,
                                     cudaStream_t s) {
  if (n_lines <= 0) return cudaSuccess;
  PG_DISPATCH_N(N, {
    using X = fft::XPass<C, NN>;
    auto k = fft::k_x_r2c_dense<C, NN>;
    PG_CUDA_TRY(set_smem(k, X::smem_bytes()));
    k<<<(unsigned)cdiv(n_lines, X::LB), X::THREADS, X::smem_bytes(), s>>>(f, n_lines, spec, P, tw);
  });
  return launched();
}

template <typename R>
bool FftPasses<R>::adj_fits(int N, int w) {
  constexpr int B = fft::ZCols<R>::B;
  const int W = 2 * w + 1;
  if (W > 256 || W > N) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  size_t need = 0;
  PG_DISPATCH_N(N, { need = fft::ZAdj<C, NN, B>::smem(W); });
  return need <= (size_t)optin;
}

namespace fft {
// Tensor map of compact window spectra (defined below with its layout).
template <typename R>
static bool adj_win_map(CUtensorMap* m, const void* base, int N, int P, int W, int nb, int64_t stride, Lay XL,
                        uint32_t by = 0);
}  // namespace fft

template <typename R>
cudaError_t FftPasses<R>::y_fwd_win(int N, int nb, const C* spec, int P, int w, C* Xw,
                                    int64_t Xw_stride, Lay XL, const C* tw, int* err, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  constexpr int B = fft::ZCols<R>::B;
  constexpr int E = (int)(sizeof(C) / 8);
  const int W = 2 * w + 1;
  // the line spectra as [line][kx] over 8-byte elements, one box = W rows of one kx tile
  const uint64_t n_lines = (uint64_t)nb * W * W;
  const uint64_t dims[4] = {(uint64_t)P * E, n_lines, 1u, 1u};
  const uint64_t strides[3] = {(uint64_t)P * 8 * E, n_lines * P * 8 * E, n_lines * P * 8 * E};
  const uint32_t box[4] = {(uint32_t)(B * E), (uint32_t)W, 1u, 1u};
  CUtensorMap mL, mO;
  const bool tma_ok = err && W <= 256 && (P * 8 * E) % 16 == 0 &&
                      (int64_t)cdiv(N / 2 + 1, B) * W * nb < INT32_MAX && encode_map_4d(&mL, spec, dims, strides, box);
  // outputs by TMA store where the compact layout has its tensor map
  const bool ts = tma_ok && fft::adj_win_map<R>(&mO, Xw, N, P, W, nb, Xw_stride, XL, N < 256 ? (uint32_t)N : 256u);
  if (!ts) memset(&mO, 0, sizeof(mO));
  PG_DISPATCH_N(N, {
    if (tma_ok) {
      using Y = fft::YWin<C, NN, B>;
      auto k = fft::k_y_fwd_win_p<C, NN, B>;
      const size_t sm = Y::smem(W);
      PG_CUDA_TRY(set_smem(k, sm));
      unsigned grid = 0;
      PG_CUDA_TRY(fft::persistent_grid(k, Y::THREADS, sm, cdiv(NN / 2 + 1, B) * (int64_t)W * nb, &grid));
      k<<<grid, Y::THREADS, sm, s>>>(mL, mO, ts ? 1 : 0, nb, w, Xw, Xw_stride, XL, tw, err);
    } else {
      using CP = fft::ColPass<C, NN, B>;
      auto k = fft::k_y_fwd_win<C, NN, B>;
      const size_t sm = CP::smem_bytes() + sizeof(C) * (size_t)W * B;   // + the compact slot
      PG_CUDA_TRY(set_smem(k, sm));
      dim3 g((unsigned)cdiv(NN / 2 + 1, B), (unsigned)W, (unsigned)nb);
      k<<<g, CP::THREADS, sm, s>>>(spec, P, w, Xw, Xw_stride, XL, tw);
    }
  });
  return launched();
}

namespace fft {
// Tensor map of compact window spectra Xw in layout XL, [ky / 8][zr][kx / B]
// [ky % 8][kx % B] per mesh: dimensions (kx mod B, ky mod 8, kx / B, zr,
// ky / 8 + mesh N / 8), box (one kx tile, one ky, all W rows zr), or with
// by > 0 (one kx tile, by ky rows, one zr).
template <typename R>
static bool adj_win_map(CUtensorMap* m, const void* base, int N, int P, int W, int nb, int64_t stride,
                        Lay XL, uint32_t by) {
  using C = typename CT<R>::C;
  constexpr int B = ZCols<R>::B, E = (int)(sizeof(C) / 8);
  const int K = 1 << kYBlockShift;
  if (XL.ks != kYBlockShift || (1 << XL.txs) != B || XL.ys != B || XL.ts != (int64_t)K * B ||
      XL.zs != (int64_t)K * P || XL.hs != (int64_t)W * K * P || stride != (int64_t)W * N * P || P % B != 0)
    return false;
  const uint64_t dims[5] = {(uint64_t)B * E, (uint64_t)K, (uint64_t)(P / B), (uint64_t)W,
                            (uint64_t)(N / K) * nb};
  const uint64_t strides[4] = {(uint64_t)XL.ys * 8 * E, (uint64_t)XL.ts * 8 * E, (uint64_t)XL.zs * 8 * E,
                               (uint64_t)XL.hs * 8 * E};
  if (by > 0 && (by % K != 0 || by > 256)) return false;
  // box: one kx tile and all W rows zr of one ky, or (by > 0) by ky rows of one zr
  const uint32_t box[5] = {(uint32_t)(B * E), by > 0 ? (uint32_t)K : 1u, 1u, by > 0 ? 1u : (uint32_t)W,
                           by > 0 ? by / (uint32_t)K : 1u};
  return encode_map_5d(m, base, dims, strides, box);
}
}  // namespace fft

template <typename R>
cudaError_t FftPasses<R>::zadj(int N, int nb, C* S, int64_t S_stride, Lay L, const C* Xw,
                               int64_t Xw_stride, Lay XL, const C* Fg, C* A, int w, int P, const C* tw,
                               int* err, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  if (!adj_fits(N, w)) return cudaErrorInvalidValue;
  constexpr int B = fft::ZCols<R>::B;
  const int W = 2 * w + 1;
  const uint32_t zb = N < 256 ? (uint32_t)N : 256u;
  CUtensorMap mS, mX, mA;
  if (!fft::spec_map<R>(&mS, S, N, P, L, nb, zb, 1) ||
      !fft::adj_win_map<R>(&mX, Xw, N, P, W, nb, Xw_stride, XL) || !fft::spec_map<R>(&mA, A, N, P, L, 1, zb, 1))
    return cudaErrorInvalidValue;
  PG_DISPATCH_N(N, {
    using Z = fft::ZAdj<C, NN, B>;
    auto k = fft::k_zadj<C, NN, B>;
    const size_t sm = Z::smem(W);
    PG_CUDA_TRY(set_smem(k, sm));
    PG_CUDA_TRY(fft::check_reg_split<typename Z::Regs>(k));
    unsigned grid = 0;
    PG_CUDA_TRY(fft::persistent_grid(k, Z::THREADS, sm, cdiv(NN / 2 + 1, B) * (int64_t)NN, &grid));
    k<<<grid, Z::THREADS, sm, s>>>(mS, mX, mA, nb, w, L, Fg, tw, err);
  });
  return launched();
}

template <typename R>
cudaError_t FftPasses<R>::zwin_acc(int N, const C* Xw, int64_t Xw_stride, Lay XL, Lay L, int P, int w,
                                   const C* Fg, C* A, const C* tw, int* err, cudaStream_t s) {
  constexpr int B = fft::ZCols<R>::B;
  const int W = 2 * w + 1;
  CUtensorMap mX;
  if (!err || W > 256 || W > N || !fft::adj_win_map<R>(&mX, Xw, N, P, W, 1, Xw_stride, XL))
    return cudaErrorInvalidValue;
  PG_DISPATCH_N(N, {
    using Y = fft::YWin<C, NN, B>;
    auto k = fft::k_zwin_acc<C, NN, B>;
    const size_t sm = Y::smem(W);
    PG_CUDA_TRY(set_smem(k, sm));
    unsigned grid = 0;
    PG_CUDA_TRY(fft::persistent_grid(k, Y::THREADS, sm, cdiv(NN / 2 + 1, B) * (int64_t)NN, &grid));
    k<<<grid, Y::THREADS, sm, s>>>(mX, w, L, Fg, A, tw, err);
  });
  return launched();
}

template <typename R>
cudaError_t FftPasses<R>::y_inv_lines(int N, int nb, const C* Y, int64_t Y_stride, Lay L, int P,
                                      const int32_t* idx, const int64_t* seg_total,
                                      const int64_t* line_base, const int32_t* line_y, C* hspec,
                                      const C* tw, int* err, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  constexpr int B = fft::ZCols<R>::B;
  // a box is one kx tile of up to 256 ky rows of one z plane
  if (Y_stride != (int64_t)N * N * P) return cudaErrorInvalidValue;
  CUtensorMap mY;
  if (!fft::spec_map<R>(&mY, Y, N, P, L, nb, 1, N < 256 ? (uint32_t)N : 256u)) return cudaErrorInvalidValue;
  PG_DISPATCH_N(N, {
    using YL = fft::YLines<C, NN, B>;
    auto k = fft::k_y_inv_lines<C, NN, B>;
    PG_CUDA_TRY(set_smem(k, YL::smem_bytes()));
    unsigned grid = 0;
    PG_CUDA_TRY(fft::persistent_grid(k, YL::THREADS, YL::smem_bytes(),
                                     cdiv(NN / 2 + 1, B) * (int64_t)NN * nb, &grid));
    k<<<grid, YL::THREADS, YL::smem_bytes(), s>>>(mY, nb, P, idx, seg_total, line_base, line_y, hspec, tw, err);
  });
  return launched();
}

template <typename R>
cudaError_t FftPasses<R>::x_c2r_lines(int N, const C* S, int P, Lay L, int64_t n_lines,
                                      const int32_t* line_y, const int32_t* line_z, R* out,
                                      double scale, const C* tw, cudaStream_t s) {
  if (n_lines <= 0) return cudaSuccess;
  PG_DISPATCH_N(N, {
    using X = fft::XPass<C, NN>;
    auto k = fft::k_x_c2r_lines<C, NN>;
    PG_CUDA_TRY(set_smem(k, X::smem_bytes()));
    k<<<(unsigned)cdiv(n_lines, X::LB), X::THREADS, X::smem_bytes(), s>>>(S, P, L, n_lines, line_y,
                                                                        line_z, out, (R)scale, tw);
  });
  return launched();
}

}  // namespace pg
