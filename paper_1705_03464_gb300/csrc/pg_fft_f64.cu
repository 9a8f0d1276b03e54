// FP64 instantiation of the FFT passes (the plain per-bin comparison path).
#include "pg_fft_impl.cuh"
template struct pg::FftPasses<double>;
