// scan.cuh -- stable stream compaction over index spaces whose length may be
// known only on the device (the kept-domain lists of pools above 2^20
// positions), and the block scan that the other compactions share.
//
// Three launches: per-block counts of the predicate, one block scanning the
// counts, and a scatter that gives every selected element its global rank in
// index order.  Grids are sized for the host-known capacity; elements at or
// beyond the device count are ignored.
#pragma once

#include "fic_common.cuh"

namespace fic {

constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 4;
constexpr int kScanTile = kScanThreads * kScanPerThread;  // elements per block

__device__ inline int block_excl_scan(int v, int* smem_warp, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int w = (lane < (int)(blockDim.x >> 5)) ? smem_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    smem_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  int before = (warp > 0 ? smem_warp[warp - 1] : 0) + x - v;
  if (total) *total = smem_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

// F: struct with  __device__ int64_t size() const;  __device__ bool flag(int64_t i) const;
//                 __device__ void emit(int64_t i, int64_t rank, bool flagged) const;
template <class F>
__global__ void __launch_bounds__(kScanThreads) k_scan_count(F f, int32_t* block_cnt) {
  __shared__ int sw[32];
  const int64_t n = f.size();
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int c = 0;
  if (base < n) {
#pragma unroll
    for (int t = 0; t < kScanPerThread; ++t) {
      int64_t i = base + (int64_t)threadIdx.x * kScanPerThread + t;
      if (i < n && f.flag(i)) ++c;
    }
  }
  int tot;
  block_excl_scan(c, sw, &tot);
  if (threadIdx.x == 0) block_cnt[blockIdx.x] = (base < n) ? tot : 0;
}

// Single block: exclusive scan of nb counts in place; *total = sum.
__global__ void __launch_bounds__(1024) k_scan_blocks(int32_t* cnt, int nb, int64_t* total);

template <class F>
__global__ void __launch_bounds__(kScanThreads) k_scan_scatter(F f, const int32_t* block_off) {
  __shared__ int sw[32];
  const int64_t n = f.size();
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  if (base >= n) return;  // uniform per block
  bool fl[kScanPerThread];
  int c = 0;
#pragma unroll
  for (int t = 0; t < kScanPerThread; ++t) {
    int64_t i = base + (int64_t)threadIdx.x * kScanPerThread + t;
    fl[t] = (i < n) && f.flag(i);
    c += fl[t];
  }
  int before = block_excl_scan(c, sw, nullptr);
  int64_t r = (int64_t)block_off[blockIdx.x] + before;
#pragma unroll
  for (int t = 0; t < kScanPerThread; ++t) {
    int64_t i = base + (int64_t)threadIdx.x * kScanPerThread + t;
    if (i < n) {
      f.emit(i, fl[t] ? r : (i - r), fl[t]);
      r += fl[t];
    }
  }
}

// Host: run the three launches for `cap` elements at most.
template <class F>
inline cudaError_t scan_compact(const F& f, int64_t cap, int32_t* d_block_scratch,
                                int64_t* d_total, cudaStream_t st) {
  int nb = (int)ceil_div64(cap > 0 ? cap : 1, kScanTile);
  k_scan_count<F><<<nb, kScanThreads, 0, st>>>(f, d_block_scratch);
  k_scan_blocks<<<1, 1024, 0, st>>>(d_block_scratch, nb, d_total);
  k_scan_scatter<F><<<nb, kScanThreads, 0, st>>>(f, d_block_scratch);
  return cudaGetLastError();
}

inline int64_t scan_scratch_blocks(int64_t cap) { return ceil_div64(cap > 0 ? cap : 1, kScanTile) + 1; }

}  // namespace fic
