// FP32 instantiation of the fused z pass.
#include "pg_fft_zcorr.cuh"
template cudaError_t pg::FftPasses<float>::z_corr(int, int, const pg::CT<float>::C*, const pg::CT<float>::C*, bool, int,
                                                pg::CT<float>::C*, int64_t, int, pg::Lay, const pg::CT<float>::C*,
                                                int*, cudaStream_t);
