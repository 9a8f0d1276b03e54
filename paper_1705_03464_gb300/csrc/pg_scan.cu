// Segmented exclusive prefix sums (cell-list offsets, compact line indices).
// Three phases: per-block scans with block totals, a scan of the block totals
// per segment, and a final add of the block offsets. Deterministic.
#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;   // elements per block

template <typename Tin>
__global__ void __launch_bounds__(kThreads)
k_scan_tiles(const Tin* __restrict__ in, int32_t* __restrict__ out, int64_t len,
             int64_t nblk, int64_t* __restrict__ block_sum) {
  const int seg = blockIdx.y;
  const int64_t blk = blockIdx.x;
  const int64_t base = (int64_t)seg * len + blk * kTile;
  const int64_t lim = len - blk * kTile;
  int v[kItems];
  int local = 0;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    int64_t i = (int64_t)threadIdx.x * kItems + k;
    v[k] = (i < lim) ? (int)in[base + i] : 0;
    local += v[k];
  }
  // block-wide exclusive scan of `local`
  __shared__ int warp_tot[kThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int t = (lane < kThreads / 32) ? warp_tot[lane] : 0;
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int u = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += u;
    }
    if (lane < kThreads / 32) warp_tot[lane] = ti - t;
    if (lane == kThreads / 32 - 1) block_sum[(int64_t)seg * nblk + blk] = ti;
  }
  __syncthreads();
  int run = warp_tot[wid] + incl - local;
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    int64_t i = (int64_t)threadIdx.x * kItems + k;
    if (i < lim) out[base + i] = run;
    run += v[k];
  }
}

__global__ void __launch_bounds__(kThreads)
k_scan_block_sums(int64_t* __restrict__ block_sum, int64_t nblk, int64_t* __restrict__ seg_total) {
  const int seg = blockIdx.x;
  int64_t* bs = block_sum + (int64_t)seg * nblk;
  __shared__ int64_t sh[kThreads];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t c0 = 0; c0 < nblk; c0 += kThreads) {
    int64_t i = c0 + threadIdx.x;
    int64_t v = (i < nblk) ? bs[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kThreads; o <<= 1) {
      int64_t t = (threadIdx.x >= o) ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nblk) bs[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == kThreads - 1) carry += sh[kThreads - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0 && seg_total) seg_total[seg] = carry;
}

__global__ void __launch_bounds__(kThreads)
k_scan_add(int32_t* __restrict__ out, int64_t len, int64_t nblk, const int64_t* __restrict__ block_sum) {
  const int seg = blockIdx.y;
  const int64_t blk = blockIdx.x;
  const int add = (int)block_sum[(int64_t)seg * nblk + blk];
  if (add == 0) return;
  const int64_t base = (int64_t)seg * len + blk * kTile;
  const int64_t lim = len - blk * kTile;
  for (int i = threadIdx.x; i < kTile && i < lim; i += kThreads) out[base + i] += add;
}

template <typename Tin>
cudaError_t scan_impl(const Tin* in, int32_t* out, int64_t len, int nseg, int64_t* seg_total,
                      int64_t* tmp, cudaStream_t s) {
  if (len <= 0 || nseg <= 0) return cudaSuccess;
  const int64_t nblk = cdiv(len, kTile);
  dim3 g((unsigned)nblk, (unsigned)nseg);
  k_scan_tiles<Tin><<<g, kThreads, 0, s>>>(in, out, len, nblk, tmp);
  PG_CUDA_TRY(launched());
  k_scan_block_sums<<<nseg, kThreads, 0, s>>>(tmp, nblk, seg_total);
  PG_CUDA_TRY(launched());
  k_scan_add<<<g, kThreads, 0, s>>>(out, len, nblk, tmp);
  return launched();
}

}  // namespace

size_t scan_tmp_elems(int64_t len, int nseg) { return (size_t)cdiv(len, kTile) * nseg + 1; }

cudaError_t scan_u8_i32(const uint8_t* in, int32_t* out, int64_t len, int nseg,
                        int64_t* seg_total, int64_t* tmp, cudaStream_t s) {
  return scan_impl<uint8_t>(in, out, len, nseg, seg_total, tmp, s);
}
cudaError_t scan_i32_i32(const int32_t* in, int32_t* out, int64_t len, int nseg,
                         int64_t* seg_total, int64_t* tmp, cudaStream_t s) {
  return scan_impl<int32_t>(in, out, len, nseg, seg_total, tmp, s);
}

}  // namespace pg
