// Launcher of the fused z pass (its own translation units per precision: the
// pass is instantiated once per mesh size and inverse pruning width K).
#pragma once

#include "pg_fft_impl.cuh"

namespace pg {
namespace fft {

// kx columns per tile of the fused z pass
template <typename R> struct ZCorrCols;
template <> struct ZCorrCols<float> { static constexpr int B = 8; };
template <> struct ZCorrCols<double> { static constexpr int B = 4; };

template <typename R, int N, int K>
static cudaError_t z_corr_launch(const typename CT<R>::C* S, const typename CT<R>::C* Fg, Lay L, int nb,
                                 bool gg, int w, typename CT<R>::C* Wz, int64_t Wz_stride, int P,
                                 const typename CT<R>::C* tw, int* err, cudaStream_t s) {
  using C = typename CT<R>::C;
  constexpr int B = ZCorrCols<R>::B;
  using Z = ZCorr<C, N, B>;
  CUtensorMap mS, mF;
  if (!spec_map<R, B>(&mF, Fg, N, P, L, 1, Z::ZB, 1) ||
      !spec_map<R, B>(&mS, gg ? (const void*)Fg : (const void*)S, N, P, L, gg ? 1 : nb, Z::ZB, 1))
    return cudaErrorInvalidValue;
  auto k = k_z_corr_tma<C, N, B, K>;
  PG_CUDA_TRY(set_smem(k, Z::smem_bytes()));
  PG_CUDA_TRY(check_reg_split<typename Z::Regs>(k));
  unsigned grid = 0;
  PG_CUDA_TRY(persistent_grid(k, Z::THREADS, Z::smem_bytes(), cdiv(N / 2 + 1, B) * (int64_t)N, &grid));
  // the galaxy-only mode is one pass over one buffer (the kernel relies on nb = 1 there)
  k<<<grid, Z::THREADS, Z::smem_bytes(), s>>>(mS, mF, gg ? 1 : nb, gg ? 1 : 0, w, Wz, Wz_stride, P, tw, err);
  return cudaSuccess;
}

}  // namespace fft

template <typename R>
cudaError_t FftPasses<R>::z_corr(int N, int nb, const C* S, const C* Fg, bool gg, int w, C* Wz,
                                 int64_t Wz_stride, int P, Lay L, const C* tw, int* err, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  PG_DISPATCH_N(N, {
    // window rows n = n2 + N2 n1 with |n| <= w have n1 < kreq or n1 >= N1 - kreq
    const int kreq = w / fft::Split<NN>::N2 + 1;
    if constexpr (NN >= 256) {
      if (kreq <= 2) PG_CUDA_TRY((fft::z_corr_launch<R, NN, 2>(S, Fg, L, nb, gg, w, Wz, Wz_stride, P, tw, err, s)));
      else if (kreq <= 4) PG_CUDA_TRY((fft::z_corr_launch<R, NN, 4>(S, Fg, L, nb, gg, w, Wz, Wz_stride, P, tw, err, s)));
      else if (kreq <= 8) PG_CUDA_TRY((fft::z_corr_launch<R, NN, 8>(S, Fg, L, nb, gg, w, Wz, Wz_stride, P, tw, err, s)));
      else PG_CUDA_TRY((fft::z_corr_launch<R, NN, 16>(S, Fg, L, nb, gg, w, Wz, Wz_stride, P, tw, err, s)));
    } else {
      PG_CUDA_TRY((fft::z_corr_launch<R, NN, 16>(S, Fg, L, nb, gg, w, Wz, Wz_stride, P, tw, err, s)));
    }
  });
  return launched();
}

}  // namespace pg
