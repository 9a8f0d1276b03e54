// FP64 instantiation of the fused z pass.
#include "pg_fft_zcorr.cuh"
template cudaError_t pg::FftPasses<double>::z_corr(int, int, const pg::CT<double>::C*, const pg::CT<double>::C*, bool, int,
                                                pg::CT<double>::C*, int64_t, int, pg::Lay, const pg::CT<double>::C*,
                                                int*, cudaStream_t);
