// FP32 instantiation of the FFT passes (the batched fast path).
#include "pg_fft_impl.cuh"
template struct pg::FftPasses<float>;
