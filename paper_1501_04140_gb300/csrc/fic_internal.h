// fic_internal.h -- host-side structures and launchers shared by the
// translation units of the CUDA encoder (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "fic_common.cuh"

namespace fic {

// A kernel launch with programmatic stream serialisation (see
// grid_dep_sync): the kernel must begin with grid_dep_sync().
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, ((KArgs)args)...);
}

// The same launch without programmatic serialisation (the kernel's
// grid_dep_sync() then returns at once).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_std(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  return cudaLaunchKernelEx(&cfg, kernel, ((KArgs)args)...);
}

// Device buffer owned by a plan; grows, never shrinks.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  int reserve(size_t want);
  void release();
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// Selection state of one image's pool (exact percentile by radix select).
struct SelState {
  int64_t prefix;   // key bits chosen so far
  int64_t rank;     // rank still to find inside the current prefix
  int64_t nlt;      // keys strictly below the prefix region
  int64_t nle;      // after the last pass: keys <= threshold
  int64_t thr;      // threshold key (after the last pass)
  int32_t nkept;    // kept domains
  int32_t fallback; // 1: nothing had key < thr, kept key <= thr
  int64_t base;     // sum of nkept of the images before this one
};

constexpr int kSelBits = 9;
constexpr int kSelBins = 1 << kSelBits;
constexpr int kSelPasses = 5;  // 45 key bits: keys are below 1024 ln(1024) 2^32 < 2^45

// Entropy-filtered domain pool of one level over a batch of images.
struct PoolLevel {
  int B = 0, L = 0, n = 0, Kp = 0, n_images = 0;
  int64_t P_tot = 0;                 // pool positions over all images
  int64_t S_tot = 0;                 // domain slots (each image's rounded up to 128)
  std::vector<int64_t> h_off;        // n_images + 1 position offsets
  std::vector<int64_t> h_slot_off;   // n_images + 1 slot offsets (multiples of 128)
  std::vector<ImgDev> h_img;         // with px, py of this level
  std::vector<int64_t> h_run_off;    // n_images + 1: runs of the sliding statistics
  bool want_tc = false, want_f32 = false;
  SSet sset{};
  double pct = 0.5;                  // entropy percentile of the threshold
  int top_k = 0;                     // > 0: keep the top_k highest entropies instead
  int nsm = 0;                       // SMs of the device (grid sizing)
  // per position: off, keys, sd, sq; per slot: slot_off, kept, bpack, b32, dom, domf
  DevBuf off, slot_off, img, keys, sd, sq, sel, hist, kept, bpack, b32, dom, domf, scan_scratch,
      total, umax, run_off;
};

// Runs of the sliding pool statistics: along a row of pool positions, the
// positions whose 2x2 cell grid shares a phase (every position for even L,
// every other one for odd L), kPoolRun at a time (kPoolRunWarp at B = 16,
// where a warp slides one window).
constexpr int kPoolRun = 4;
constexpr int kPoolRunWarp = 8;
__host__ __device__ inline int pool_run_step(int L) { return (L & 1) ? 2 : 1; }
__host__ __device__ inline int pool_run_len(int B, int L) {
  return pool_run_step(L) * L >= 2 * B ? 1 : B == 16 ? kPoolRunWarp : kPoolRun;
}
// runs of one row of px positions (phase class 0 first)
__host__ __device__ inline int pool_runs_per_row(int px, int B, int L) {
  const int st = pool_run_step(L), R = pool_run_len(B, L);
  int runs = 0;
  for (int c = 0; c < st; ++c) {
    const int nc = px > c ? (px - c + st - 1) / st : 0;
    runs += (nc + R - 1) / R;
  }
  return runs;
}
int pool_prepare();  // per device, before the first pool build

// Launchers (pool.cu)
int pool_build(PoolLevel& pl, const int64_t* d_dT, cudaStream_t st);
void make_sset(int s_mode, int grid_samples, int B, SSet* out);
int host_key_table(int64_t* dT, int nmax);

// scan.cu
__global__ void k_scan_blocks(int32_t* cnt, int nb, int64_t* total);

}  // namespace fic
