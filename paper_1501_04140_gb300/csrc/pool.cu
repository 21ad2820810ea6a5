// pool.cu -- the entropy-filtered domain pool of one quadtree level (Sec. 2
// domain pool, Sec. 3 entropy filter) for a batch of images.
//
//   k_pool_stats_lane, k_pool_stats_warp16
//                   every 2B x 2B square at step L: its entropy key (Eq. 4-5,
//                   fixed point), the sum of its 2x2 sums Ds and of Ds^2,
//                   sliding along runs of positions.
//   k_select_compact  per image in one block: the exact percentile (or top-K)
//                   threshold of the keys and the kept list; pools above 2^20
//                   positions use k_sel_* (radix select, 5 passes of 9 bits)
//                   and the multi-block compaction.
//   compaction      kept = entropy greater than the threshold (key below it),
//                   ascending raster order; "greater or equal" when that keeps
//                   nothing.
//   k_pack_domains  the kept domains as matcher operands: f16 (Ds - 512) in
//                   the tensor cores' K-major core-matrix layout and/or fp32,
//                   plus the per-domain moments the scoring needs.
#include <math.h>

#include <algorithm>

#include "fic_internal.h"
#include "scan.cuh"

namespace fic {

// ---------------------------------------------------------------- S sets
void make_sset(int s_mode, int grid_samples, int B, SSet* o) {
  *o = SSet{};
  if (s_mode == FIC_S_EXACT) {  // one "s" per pair, found from its moments
    o->exact = 1;
    o->m = 1;
    o->q = 1;
    return;
  }
  if (s_mode == FIC_S_GRID) {
    o->grid = 1;
    o->m = grid_samples;
    o->q = grid_samples - 1;
    for (int k = 0; k < grid_samples && k < kMaxS; ++k) o->p[k] = k;
    return;
  }
  // Sec. 3.1: step 1 (B = 16) {0.1}; step 2 (B = 8) {0.2, 0.4};
  // step 3 (B = 4) {0.3, 0.8}; step 4 (B = 2) {0.5, 0.9}.
  o->grid = 0;
  o->q = 10;
  switch (B) {
    case 16: o->m = 1; o->p[0] = 1; break;
    case 8: o->m = 2; o->p[0] = 2; o->p[1] = 4; break;
    case 4: o->m = 2; o->p[0] = 3; o->p[1] = 8; break;
    default: o->m = 2; o->p[0] = 5; o->p[1] = 9; break;
  }
}

// ---------------------------------------------------------------- entropy key table
// Key of a histogram: sum over grey levels of round(c ln c 2^32), c the
// level's count (Eq. 4-5 with the constant ln(#pixels) and the 1/#pixels
// factor dropped: H = ln N - key / (N 2^32), so a larger key is a lower
// entropy).  The device accumulates it per pixel as the increments
// dT[c] = T[c] - T[c - 1] of the running count, so no bin scan is needed.
int host_key_table(int64_t* dT, int nmax) {
  int64_t prev = 0;
  dT[0] = 0;
  for (int c = 1; c <= nmax; ++c) {
    long double v = (long double)c * logl((long double)c) * 4294967296.0L;
    int64_t t = (int64_t)llroundl(v);
    dT[c] = t - prev;
    prev = t;
  }
  return 0;
}

// ---------------------------------------------------------------- pool statistics
// One lane per run of positions along a row (see
// pool_run_len), with a lane-private histogram in shared memory (16-bit
// counts, [grey level][lane], so the lanes of a warp never contend).  The
// first window of a run is built in full; each next position removes the
// d = step L pixel columns that leave and adds the d that enter (d / 2 cell
// columns of 2x2 sums), updating the key by -dT[c] / +dT[c + 1] and the
// moments by the cells' sums and squares -- the same exact integers as a
// full recount.
constexpr int kPoolLaneThreads = 128;

template <int B>
struct PoolLaneSmem {
  static constexpr int N4 = 4 * B * B;
  static constexpr int DT_BYTES = ((N4 + 1) * 8 + 127) / 128 * 128;
  static constexpr int BYTES = DT_BYTES + (kPoolLaneThreads / 32) * 256 * 32 * 2;
};

template <int B>
__global__ void __launch_bounds__(kPoolLaneThreads)
k_pool_stats_lane(const ImgDev* __restrict__ imgs, const int64_t* __restrict__ off,
                  const int64_t* __restrict__ run_off, int n_images, int L,
                  const int64_t* __restrict__ dT_g, int64_t* __restrict__ keys,
                  int32_t* __restrict__ sd, int32_t* __restrict__ sq) {
  using Sm = PoolLaneSmem<B>;
  extern __shared__ __align__(128) uint8_t psm[];
  int64_t* dT = (int64_t*)psm;
  const int lane = threadIdx.x & 31;
  grid_dep_sync();
  uint16_t* h = (uint16_t*)(psm + Sm::DT_BYTES) + (threadIdx.x >> 5) * (256 * 32) + lane;
  for (int i = threadIdx.x; i <= Sm::N4; i += blockDim.x) dT[i] = dT_g[i];
  for (int b = 0; b < 256; ++b) h[b * 32] = 0;
  __syncthreads();
  const int step = pool_run_step(L), R = pool_run_len(B, L), d = step * L;
  const int64_t total = run_off[n_images];
  for (int64_t gr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gr < total;
       gr += (int64_t)gridDim.x * blockDim.x) {
    const int im = find_segment(run_off, n_images, gr);
    const ImgDev I = imgs[im];
    const int rpr = pool_runs_per_row(I.px, B, L);
    const int64_t lr = gr - run_off[im];
    const int row = (int)(lr / rpr);
    int rem = (int)(lr % rpr), cls = 0;
    const int r0 = ((I.px + step - 1) / step + R - 1) / R;  // runs of phase class 0
    if (rem >= r0) {
      cls = 1;
      rem -= r0;
    }
    int i = cls + step * rem * R;  // first position of the run (x index)
    const int y0 = row * L;
    int x0 = i * L;
    const uint8_t* base = I.pix + (int64_t)y0 * I.pitch;
    int64_t key = 0;
    int s = 0, s2 = 0;
    auto add = [&](int v) {
      const int c = h[v * 32] + 1;
      h[v * 32] = (uint16_t)c;
      key += dT[c];
    };
    auto del = [&](int v) {
      const int c = h[v * 32];
      h[v * 32] = (uint16_t)(c - 1);
      key -= dT[c];
    };
    // the run's first window in full
    for (int ci = 0; ci < B; ++ci) {
      const uint8_t* p = base + (int64_t)(2 * ci) * I.pitch + x0;
      for (int cj = 0; cj < B; ++cj) {
        const int v0 = p[2 * cj], v1 = p[2 * cj + 1], v2 = p[I.pitch + 2 * cj],
                  v3 = p[I.pitch + 2 * cj + 1];
        add(v0); add(v1); add(v2); add(v3);
        const int ds = v0 + v1 + v2 + v3;
        s += ds;
        s2 += ds * ds;
      }
    }
    int64_t g = off[im] + (int64_t)row * I.px + i;
    keys[g] = key;
    sd[g] = s;
    sq[g] = s2;
    for (int m = 1; m < R; ++m) {
      i += step;
      if (i >= I.px) break;
      for (int ci = 0; ci < B; ++ci) {
        const uint8_t* p = base + (int64_t)(2 * ci) * I.pitch + x0;
        for (int cc = 0; cc < d; cc += 2) {
          const int o0 = p[cc], o1 = p[cc + 1], o2 = p[I.pitch + cc], o3 = p[I.pitch + cc + 1];
          const int n0 = p[2 * B + cc], n1 = p[2 * B + cc + 1], n2 = p[I.pitch + 2 * B + cc],
                    n3 = p[I.pitch + 2 * B + cc + 1];
          del(o0); del(o1); del(o2); del(o3);
          add(n0); add(n1); add(n2); add(n3);
          const int dso = o0 + o1 + o2 + o3, dsn = n0 + n1 + n2 + n3;
          s += dsn - dso;
          s2 += dsn * dsn - dso * dso;
        }
      }
      x0 += d;
      g += step;
      keys[g] = key;
      sd[g] = s;
      sq[g] = s2;
    }
    for (int b = 0; b < 256; ++b) h[b * 32] = 0;
  }
}

// B = 16: one warp per run, the window's 32 pixel columns (then, sliding,
// its 32 pixel rows) on the 32 lanes and one 256-bin histogram per warp in
// shared memory.  Each atomic returns the bin's count before it, so every
// lane adds the exact key change of its own update (dT[c + 1] on an
// increment from c, -dT[c] on a decrement from c) and the lanes' sums
// telescope to the key of the final counts whatever order the atomics take.
// A cell's 2x2 sum is two lanes' column (row) pairs, joined by a shuffle.
constexpr int kPoolWarpThreads = 256;

__global__ void __launch_bounds__(kPoolWarpThreads)
k_pool_stats_warp16(const ImgDev* __restrict__ imgs, const int64_t* __restrict__ off,
                    const int64_t* __restrict__ run_off, int n_images, int L,
                    const int64_t* __restrict__ dT_g, int64_t* __restrict__ keys,
                    int32_t* __restrict__ sd, int32_t* __restrict__ sq) {
  constexpr int B = 16, W = 2 * B, N4 = 4 * B * B, WARPS = kPoolWarpThreads / 32;
  __shared__ int64_t dT[N4 + 1];
  __shared__ uint32_t hist[WARPS][256];
  grid_dep_sync();
  for (int i = threadIdx.x; i <= N4; i += blockDim.x) dT[i] = dT_g[i];
  for (int i = threadIdx.x; i < WARPS * 256; i += blockDim.x) (&hist[0][0])[i] = 0;
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* h = hist[warp];
  const int step = pool_run_step(L), R = pool_run_len(B, L), d = step * L;
  const int64_t total = run_off[n_images];
  // (warp-uniform loop: every lane takes part in the shuffles)
  for (int64_t gr = (int64_t)blockIdx.x * WARPS + warp; gr < total;
       gr += (int64_t)gridDim.x * WARPS) {
    const int im = find_segment(run_off, n_images, gr);
    const ImgDev I = imgs[im];
    const int rpr = pool_runs_per_row(I.px, B, L);
    const int64_t lr = gr - run_off[im];
    const int row = (int)(lr / rpr);
    int rem = (int)(lr % rpr), cls = 0;
    const int r0 = ((I.px + step - 1) / step + R - 1) / R;  // runs of phase class 0
    if (rem >= r0) {
      cls = 1;
      rem -= r0;
    }
    int i = cls + step * rem * R;  // first position of the run (x index)
    int x0 = i * L;
    const int pitch = I.pitch;
    const uint8_t* base = I.pix + (int64_t)(row * L) * pitch;
    int64_t key = 0;  // this lane's share of the key and moments
    int s = 0, s2 = 0;
    // the warp's sums by hardware reductions of 32-bit values: the key as
    // two digits key = hi 2^24 + lo (lo in [0, 2^24)); a lane's share stays
    // below 2^41 in magnitude, so both digit sums over the 32 lanes fit
    auto emit = [&](int64_t g) {
      const int lo = (int)(key & 0xFFFFFF);
      const int hi = (int)(key >> 24);
      const int slo = __reduce_add_sync(0xffffffffu, lo);
      const int shi = __reduce_add_sync(0xffffffffu, hi);
      const int a = __reduce_add_sync(0xffffffffu, s);
      const int b = __reduce_add_sync(0xffffffffu, s2);
      if (lane == 0) {
        keys[g] = (int64_t)shi * (1LL << 24) + slo;
        sd[g] = a;
        sq[g] = b;
      }
    };
    // the run's first window: lane = pixel column, two rows per step
    for (int r = 0; r < W; r += 2) {
      const uint8_t* p = base + (int64_t)r * pitch + x0 + lane;
      const int a = p[0], b = p[pitch];
      key += dT[atomicAdd(&h[a], 1u) + 1];
      key += dT[atomicAdd(&h[b], 1u) + 1];
      const int col = a + b;
      const int ds = col + __shfl_xor_sync(0xffffffffu, col, 1);
      if (!(lane & 1)) {
        s += ds;
        s2 += ds * ds;
      }
    }
    int64_t g = off[im] + (int64_t)row * I.px + i;
    emit(g);
    // next positions: lane = pixel row; the d columns that leave, the d that enter
    const uint8_t* pr = base + (int64_t)lane * pitch;
    // column pairs as 2-byte loads where they start on even addresses (x0
    // keeps its parity: d is even)
    const bool pairs = ((((uintptr_t)I.pix) | (uintptr_t)pitch | (uintptr_t)x0) & 1) == 0;
    for (int m = 1; m < R; ++m) {
      i += step;
      if (i >= I.px) break;
      for (int cc = 0; cc < d; cc += 2) {
        int o0, o1, n0, n1;
        if (pairs) {
          const uchar2 o = *(const uchar2*)(pr + x0 + cc), nw = *(const uchar2*)(pr + x0 + W + cc);
          o0 = o.x, o1 = o.y, n0 = nw.x, n1 = nw.y;
        } else {
          o0 = pr[x0 + cc], o1 = pr[x0 + cc + 1];
          n0 = pr[x0 + W + cc], n1 = pr[x0 + W + cc + 1];
        }
        key -= dT[atomicSub(&h[o0], 1u)];
        key -= dT[atomicSub(&h[o1], 1u)];
        key += dT[atomicAdd(&h[n0], 1u) + 1];
        key += dT[atomicAdd(&h[n1], 1u) + 1];
        const int ro = o0 + o1, rn = n0 + n1;
        const int dso = ro + __shfl_xor_sync(0xffffffffu, ro, 1);
        const int dsn = rn + __shfl_xor_sync(0xffffffffu, rn, 1);
        if (!(lane & 1)) {
          s += dsn - dso;
          s2 += dsn * dsn - dso * dso;
        }
      }
      x0 += d;
      g += step;
      emit(g);
    }
    __syncwarp();
#pragma unroll
    for (int b = 0; b < 256; b += 32) h[b + lane] = 0;
    __syncwarp();
  }
}

template <int B>
static int prepare_pool_B() {
  return cudaFuncSetAttribute(k_pool_stats_lane<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              PoolLaneSmem<B>::BYTES) == cudaSuccess
             ? 0
             : 1;
}

// The sliding statistics kernels' shared memory.
static int prepare_stats() {
  return prepare_pool_B<16>() | prepare_pool_B<8>() | prepare_pool_B<4>() | prepare_pool_B<2>();
}

// ---------------------------------------------------------------- exact percentile
// Sec. 3 keeps domains whose entropy is greater than a threshold; the
// threshold is the pool's entropy at percentile p: sorted ascending by
// entropy, index floor(p (P - 1)).  Entropy ascending is key descending, so
// the threshold is the key of ascending rank P - 1 - floor(p (P - 1)).
// Rank of the threshold key (ascending key order) and whether the whole pool
// is kept: the percentile p, or Tables 1-2's pool size K (the K lowest keys
// lie below the key of ascending rank K; K >= P keeps everything).
__device__ inline int64_t sel_rank(int64_t P, double pct, int top_k, int* keep_all) {
  *keep_all = 0;
  if (P <= 0) return 0;
  if (top_k > 0) {
    *keep_all = top_k >= P;
    return top_k < P ? top_k : P - 1;
  }
  int64_t ih = (int64_t)floor(pct * (double)(P - 1));
  if (ih < 0) ih = 0;
  if (ih > P - 1) ih = P - 1;
  return P - 1 - ih;
}

__global__ void k_sel_init(const int64_t* __restrict__ off, int n_images, double pct, int top_k,
                           SelState* __restrict__ st, uint32_t* __restrict__ hist) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_images * kSelBins;
       i += gridDim.x * blockDim.x)
    hist[i] = 0;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_images) {
    int64_t P = off[i + 1] - off[i];
    int keep_all;
    SelState s{};
    s.prefix = 0;
    s.rank = sel_rank(P, pct, top_k, &keep_all);
    s.nlt = 0;
    s.fallback = keep_all;  // kept: key <= threshold
    st[i] = s;
  }
}

constexpr int kSelThreads = 256;
constexpr int kSelPerThread = 16;

__global__ void __launch_bounds__(kSelThreads)
k_sel_hist(const int64_t* __restrict__ keys, const int64_t* __restrict__ off, int n_images,
           int shift, const SelState* __restrict__ st, uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[kSelBins];
  for (int i = threadIdx.x; i < kSelBins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int64_t P_tot = off[n_images];
  const int64_t b0 = (int64_t)blockIdx.x * kSelThreads * kSelPerThread;
  const int im0 = b0 < P_tot ? find_segment(off, n_images, b0) : 0;
  const int64_t pre0 = st[im0].prefix;
  for (int t = 0; t < kSelPerThread; ++t) {
    int64_t g = b0 + (int64_t)t * kSelThreads + threadIdx.x;
    if (g >= P_tot) break;
    const int64_t k = keys[g];
    if (g >= off[im0 + 1] || g < off[im0]) {  // block straddles images
      int im = find_segment(off, n_images, g);
      if ((k >> (shift + kSelBits)) == st[im].prefix)
        atomicAdd(&hist[im * kSelBins + ((k >> shift) & (kSelBins - 1))], 1u);
    } else if ((k >> (shift + kSelBits)) == pre0) {
      atomicAdd(&sh[(k >> shift) & (kSelBins - 1)], 1u);
    }
  }
  __syncthreads();
  if (b0 < P_tot)
    for (int i = threadIdx.x; i < kSelBins; i += blockDim.x)
      if (sh[i]) atomicAdd(&hist[im0 * kSelBins + i], sh[i]);
}

// One block of kSelBins threads per image: pick the digit holding the rank.
__global__ void __launch_bounds__(kSelBins)
k_sel_find(SelState* __restrict__ st, uint32_t* __restrict__ hist, int last) {
  __shared__ int sw[32];
  __shared__ int tot;
  const int im = blockIdx.x;
  uint32_t* h = hist + (int64_t)im * kSelBins;
  const int c = (int)h[threadIdx.x];
  const int before = block_excl_scan(c, sw, &tot);
  SelState s = st[im];
  __syncthreads();
  if (tot > 0 && before <= s.rank && s.rank < before + c) {
    s.prefix = (s.prefix << kSelBits) | threadIdx.x;
    s.rank -= before;
    s.nlt += before;
    if (last) {
      s.thr = s.prefix;
      s.nle = s.nlt + c;
      s.fallback = (s.nlt == 0 || s.fallback) ? 1 : 0;
      s.nkept = (int32_t)(s.fallback ? s.nle : s.nlt);
    }
    st[im] = s;
  }
  h[threadIdx.x] = 0;
}

__global__ void k_sel_bases(SelState* st, int n_images) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t b = 0;
    for (int i = 0; i < n_images; ++i) {
      st[i].base = b;
      b += st[i].nkept;
    }
  }
}

// The same selection and the stable compaction of the kept positions in one
// block per image, for pools of at most kSelFusedMax positions.  Digits are
// 12 bits wide (4096 shared-memory bins; keys are below 2^45): the entropy
// keys of a pool crowd into a narrow band, and wide digits spread them so
// the bins' atomics rarely collide.
//
// Candidates.  Pools of up to kSelCand keys are copied to shared memory
// whole.  Pools of up to kSelSampleMax keys first take an evenly strided
// sample of kSelSample keys and bracket the sample keys kSelMargin sample
// ranks below and above the target's estimated sample rank by lo, hi (a
// histogram of the sample over its range); one pass over the keys counts
// those below lo and gathers those in [lo, hi].  When
// the target rank falls among the gathered keys (it does unless the sample
// misjudges it by more than the margin, about four standard deviations) the
// radix passes run on them alone, starting from the count below lo; all keys
// equal to the threshold lie in [lo, hi], so the counts stay exact.
// Otherwise (and for larger pools) two passes read the keys from L2; the
// second also gathers the keys that share the top digit, so the last two
// passes usually run on shared memory alone.  The compaction then gives each
// warp a contiguous run of positions: a counting sweep, a scan of the 32 warp
// totals, and an ordered write with ballot ranks.
constexpr int kSelFusedThreads = 1024;
constexpr int64_t kSelFusedMax = (int64_t)1 << 20;
constexpr int kSelCand = 12288;         // candidate keys (dynamic shared memory)
constexpr int kSelSample = 1024;        // sample keys
constexpr int kSelMargin = 64;          // sample ranks on each side of the estimate
constexpr int64_t kSelSampleMax = 81920;  // about 10300 candidates expected at most
constexpr int kSelDynBytes = (kSelCand + 128) * 8;  // candidates, then a scratch of 128 keys
constexpr int kSelWBits = 12;
constexpr int kSelWBins = 1 << kSelWBits;
constexpr int kSelWPasses = 4;  // 48 >= 45 key bits
// A candidate in shared memory carries, above its key (< 2^45), the warp of
// the compaction whose run of positions it came from.
constexpr int kSelTagShift = 56;
constexpr int64_t kSelKeyMask = ((int64_t)1 << kSelTagShift) - 1;

// Adds 1 to cnt[d] for each lane with d >= 0, one atomic per run of equal d
// over adjacent lanes; lanes with nothing to add pass distinct negative
// values.  All 32 lanes call it.
__device__ inline void warp_run_count(int* cnt, int d, int lane) {
  const int dp = __shfl_up_sync(0xffffffffu, d, 1);
  const bool head = lane == 0 || d != dp;
  const unsigned heads = __ballot_sync(0xffffffffu, head);
  if (head && d >= 0) {
    const unsigned after = heads & ~((2u << lane) - 1u);  // run heads above this lane
    const int end = after ? __ffs(after) - 1 : 32;
    atomicAdd(&cnt[d], end - lane);
  }
}

__global__ void __launch_bounds__(kSelFusedThreads)
k_select_compact(const int64_t* __restrict__ keys, const int64_t* __restrict__ off,
                 const int64_t* __restrict__ slot_off, double pct, int top_k,
                 SelState* __restrict__ st,
                 int32_t* __restrict__ kept, unsigned int* __restrict__ umax) {
  __shared__ uint32_t hist[kSelWBins];
  extern __shared__ int64_t sel_dyn[];
  int64_t* cand = sel_dyn;               // kSelCand keys
  int64_t* samp = sel_dyn + kSelCand;    // scratch: warp minima and maxima, the bracket
  __shared__ int n_cand;
  grid_dep_sync();
  __shared__ unsigned long long n_below;
  __shared__ int sw[32];
  __shared__ int wtot[32];
  __shared__ SelState s_st;
  // compaction runs: warp w of the block owns positions [w seg, (w + 1) seg)
  const int64_t P0 = off[blockIdx.x + 1] - off[blockIdx.x];
  const int64_t seg = ceil_div64(ceil_div64(P0, 32), 32) * 32;  // a multiple of 32
  const int im = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t o0 = off[im], P = off[im + 1] - o0;
  const int64_t* k = keys + o0;
  wtot[lane] = 0;  // (every warp writes the same zeros)
  if (threadIdx.x == 0) {
    int keep_all;
    SelState z{};
    z.rank = sel_rank(P, pct, top_k, &keep_all);
    z.fallback = keep_all;  // kept: key <= threshold
    s_st = z;
    n_cand = 0;
    n_below = 0;
    if (im == 0) *umax = 0;  // the packer's running maximum starts here
  }
  __syncthreads();
  bool in_smem = false;
  if (P <= kSelCand) {  // the whole pool as candidates
    for (int64_t g = threadIdx.x; g < P; g += blockDim.x)
      cand[g] = __ldg(k + g) | ((g / seg) << kSelTagShift);
    if (threadIdx.x == 0) n_cand = (int)P;
    in_smem = true;
  } else if (P <= kSelSampleMax) {
    // the sample's keys of ranks ts -/+ kSelMargin, to the resolution of
    // 4096 bins over the sample's range: lo = the low edge of the bin that
    // holds the first, hi = the high edge of the bin that holds the second
    // (so lo <= that key, hi >= the other: the bracket only widens)
    static_assert(kSelSample == kSelFusedThreads, "one sample key per thread");
    const int64_t sk = __ldg(k + (int64_t)threadIdx.x * P / kSelSample);
    int64_t mn = sk, mx = sk;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = min(mn, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)mn, o));
      mx = max(mx, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)mx, o));
    }
    for (int i = threadIdx.x; i < kSelWBins; i += blockDim.x) hist[i] = 0;
    if (lane == 0) {
      samp[warp] = mn;
      samp[32 + warp] = mx;
    }
    __syncthreads();
    if (warp == 0) {
      mn = samp[lane];
      mx = samp[32 + lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)mn, o));
        mx = max(mx, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)mx, o));
      }
      if (lane == 0) {
        samp[66] = mn;
        samp[67] = mx;
      }
    }
    __syncthreads();
    const int64_t kmin = samp[66], kmax = samp[67];
    int sh = 0;
    while (((kmax - kmin) >> sh) >= kSelWBins) ++sh;
    atomicAdd(&hist[(sk - kmin) >> sh], 1u);
    __syncthreads();
    const int64_t rank0 = s_st.rank;
    const int ts = (int)(rank0 * kSelSample / P);
    const int rlo = ts - kSelMargin, rhi = ts + kSelMargin;
    constexpr int SPT = kSelWBins / kSelFusedThreads;  // bins per thread
    uint32_t c[SPT];
    int csum = 0;
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      c[u] = hist[threadIdx.x * SPT + u];
      csum += (int)c[u];
    }
    int tot;
    int before = block_excl_scan(csum, sw, &tot);
    if (threadIdx.x == 0) {
      samp[64] = INT64_MIN;
      samp[65] = INT64_MAX;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int b = threadIdx.x * SPT + u;
      if (rlo >= 0 && before <= rlo && rlo < before + (int)c[u]) samp[64] = kmin + ((int64_t)b << sh);
      if (rhi < kSelSample && before <= rhi && rhi < before + (int)c[u])
        samp[65] = kmin + ((int64_t)(b + 1) << sh) - 1;
      before += (int)c[u];
    }
    __syncthreads();
    const int64_t lo = samp[64], hi = samp[65];
    // one pass over the warp's compaction run: its keys below lo counted,
    // those in [lo, hi] appended (one atomic per warp and 256 keys) with the
    // warp as their tag
    int below = 0;
    constexpr int U = 8;
    const int64_t g0 = (int64_t)warp * seg, g1 = min(P, g0 + seg);
    for (int64_t gb = g0; gb < g1; gb += U * 32) {  // (warp-uniform)
      int64_t kk[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t g = gb + u * 32 + lane;
        kk[u] = g < g1 ? __ldg(k + g) : -1;
      }
      unsigned m[U];
      int n = 0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const bool in = kk[u] >= 0 && kk[u] >= lo && kk[u] <= hi;  // (-1: past the end)
        below += kk[u] >= 0 && kk[u] < lo;
        m[u] = __ballot_sync(0xffffffffu, in);
        n += __popc(m[u]);
      }
      if (n) {
        int b0 = 0;
        if (lane == 0) b0 = atomicAdd(&n_cand, n);
        b0 = __shfl_sync(0xffffffffu, b0, 0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int i = b0 + __popc(m[u] & ((1u << lane) - 1u));
          if (((m[u] >> lane) & 1u) && i < kSelCand) cand[i] = kk[u] | ((int64_t)warp << kSelTagShift);
          b0 += __popc(m[u]);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
    if (lane == 0) {
      wtot[warp] = below;  // the warp's kept keys so far: all those below lo
      atomicAdd(&n_below, (unsigned long long)below);
    }
    __syncthreads();
    const int64_t nb = (int64_t)n_below, nc = n_cand;
    in_smem = nc <= kSelCand && nb <= rank0 && rank0 < nb + nc;  // uniform
    __syncthreads();
    if (threadIdx.x == 0) {
      if (in_smem) {
        s_st.rank = rank0 - nb;
        s_st.nlt = nb;
      } else {
        n_cand = 0;  // the L2 passes gather afresh
      }
    }
  }
  // candidates that carry their compaction warp: the warps' kept counts come
  // from shared memory, without a counting sweep over the keys
  const bool tagged = in_smem;
  constexpr int BPT = kSelWBins / kSelFusedThreads;  // bins per thread in the scan
  for (int pass = 0; pass < kSelWPasses; ++pass) {
    const int shift = (kSelWPasses - 1 - pass) * kSelWBits;
    for (int i = threadIdx.x; i < kSelWBins; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    // every thread reads the state before the one that owns the digit
    // rewrites it below
    const int64_t prefix = s_st.prefix, rank = s_st.rank;
    if (in_smem) {
      const int nc = n_cand;
      for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        const int64_t kk = cand[i] & kSelKeyMask;
        if ((kk >> (shift + kSelWBits)) == prefix)
          atomicAdd(&hist[(kk >> shift) & (kSelWBins - 1)], 1u);
      }
    } else {
      constexpr int U = 8;
      for (int64_t g0 = threadIdx.x; g0 < P; g0 += (int64_t)U * blockDim.x) {
        int64_t kk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int64_t g = g0 + (int64_t)u * blockDim.x;
          kk[u] = g < P ? __ldg(k + g) : -1;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (kk[u] >= 0 && (kk[u] >> (shift + kSelWBits)) == prefix) {
            atomicAdd(&hist[(kk[u] >> shift) & (kSelWBins - 1)], 1u);
            if (pass == 1) {  // gather the keys that share the top digit
              const int i = atomicAdd(&n_cand, 1);
              if (i < kSelCand) cand[i] = kk[u];
            }
          }
        }
      }
    }
    __syncthreads();
    // exclusive scan of the bins: BPT consecutive bins per thread
    uint32_t c[BPT];
    int csum = 0;
#pragma unroll
    for (int u = 0; u < BPT; ++u) {
      c[u] = hist[threadIdx.x * BPT + u];
      csum += (int)c[u];
    }
    int tot;
    int before = block_excl_scan(csum, sw, &tot);
    if (tot > 0 && before <= rank && rank < before + csum) {
#pragma unroll
      for (int u = 0; u < BPT; ++u) {
        if (before <= rank && rank < before + (int)c[u]) {
          SelState x = s_st;
          x.prefix = (prefix << kSelWBits) | (threadIdx.x * BPT + u);
          x.rank = rank - before;
          x.nlt += before;
          if (pass == kSelWPasses - 1) {
            x.thr = x.prefix;
            x.nle = x.nlt + c[u];
            x.fallback = (x.nlt == 0 || x.fallback) ? 1 : 0;
            x.nkept = (int32_t)(x.fallback ? x.nle : x.nlt);
          }
          s_st = x;
        }
        before += (int)c[u];
      }
    }
    __syncthreads();
    if (pass == 1) in_smem = n_cand <= kSelCand;  // uniform: read after the barrier
  }
  // stable compaction: kept = key below the threshold (or equal, fallback)
  const int64_t thr = s_st.thr;
  const bool fb = s_st.fallback != 0;
  const int64_t g0 = (int64_t)warp * seg, g1 = min(P, g0 + seg);
  if (tagged) {  // the kept candidates of each warp's run, on top of its keys below lo
    const int nc = n_cand;
    for (int ib = warp * 32; ib < nc; ib += blockDim.x) {  // (warp-uniform)
      const int i = ib + lane;
      const int64_t c = i < nc ? cand[i] : -1;
      const int64_t kk = c & kSelKeyMask;
      const bool f = c >= 0 && (fb ? (kk <= thr) : (kk < thr));
      warp_run_count(wtot, f ? (int)(c >> kSelTagShift) : -1 - lane, lane);
    }
  } else {
    int cnt = 0;
    for (int64_t gb = g0; gb < g1; gb += 8 * 32) {
      int64_t kk[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t g = gb + u * 32 + lane;
        kk[u] = g < g1 ? __ldg(k + g) : -1;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) cnt += kk[u] >= 0 && (fb ? (kk[u] <= thr) : (kk[u] < thr));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) wtot[warp] = cnt;
  }
  __syncthreads();
  int base = 0;
  for (int w2 = 0; w2 < warp; ++w2) base += wtot[w2];
  int32_t* out = kept + slot_off[im];
  for (int64_t gb = g0; gb < g1; gb += 8 * 32) {
    int64_t kk[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t g = gb + u * 32 + lane;
      kk[u] = g < g1 ? __ldg(k + g) : -1;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool f = kk[u] >= 0 && (fb ? (kk[u] <= thr) : (kk[u] < thr));
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (f) out[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)(gb + u * 32 + lane);
      base += __popc(bal);
    }
  }
  if (threadIdx.x == 0) st[im] = s_st;
}

// Opt the pool kernels in to their shared memory (once per device, before any
// launch or stream capture).
int pool_prepare() {
  const bool ok = prepare_stats() == 0 &&
                  cudaFuncSetAttribute(k_select_compact, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSelDynBytes) == cudaSuccess;
  return ok ? FIC_OK : FIC_ECUDA;
}

struct KeptCompact {
  const int64_t* keys;
  const int64_t* off;
  const int64_t* slot_off;
  const SelState* st;
  int32_t* kept;
  int n_images;
  __device__ int64_t size() const { return off[n_images]; }
  __device__ bool flag(int64_t g) const {
    const int im = find_segment(off, n_images, g);
    const SelState& s = st[im];
    return s.fallback ? keys[g] <= s.thr : keys[g] < s.thr;
  }
  __device__ void emit(int64_t g, int64_t rank, bool f) const {
    if (!f) return;
    const int im = find_segment(off, n_images, g);
    kept[slot_off[im] + (rank - st[im].base)] = (int32_t)(g - off[im]);
  }
};

// ---------------------------------------------------------------- operand packing
// f16 bits of a small integer (|v| <= 2048, exact in binary16).
__device__ inline uint16_t f16_bits(int v) {
  return __half_as_ushort(__int2half_rn(v));
}

// Tensor operand layout of the kept domains: for each 128-slot tile T and
// K slice kc (one slice of 128 at B = 16, the whole padded K otherwise), the
// tile's 16 groups of 8 domains, each as K/8 core matrices of 8 domains x 8
// f16 (16-byte rows): [T][kc][group][k / 8][slot % 8][k % 8].  A (T, kc)
// slice is contiguous and is copied to shared memory as it is.  At B <= 8
// the tile's operand is followed by its scoring records (tc_tile_bytes).
template <int B>
struct PackGeom {
  static constexpr int n = B * B;
  static constexpr int Kp = n < 16 ? 16 : n;
  static constexpr int NKC = n > 128 ? n / 128 : 1;
  static constexpr int KS = Kp / NKC;
};

template <int B>
__device__ inline int64_t bpack_index(int64_t slot, int e) {
  using P = PackGeom<B>;
  const int64_t T = slot >> 7;
  const int r = (int)(slot & 127);
  const int kc = e / P::KS, ek = e % P::KS;
  return ((((T * P::NKC + kc) * 16 + (r >> 3)) * (P::KS / 8) + (ek >> 3)) * 8 + (r & 7)) * 8 +
         (ek & 7);
}

// One thread per (kept domain, 8-element K group): the group's 8 downsampled
// values Ds - 512 (each the sum of a 2x2 pixel block, read as two pixel
// pairs) go out as one 16-byte store of f16 (at B = 16 the warp of a domain
// reads row by row instead, see below).  Then one thread per domain writes
// its records.
constexpr int kPackThreads = 256;

template <int B>
__global__ void __launch_bounds__(kPackThreads)
k_pack_domains(const ImgDev* __restrict__ imgs, const int64_t* __restrict__ off,
               const int64_t* __restrict__ slot_off, int n_images, int L,
               const SelState* __restrict__ st, const int32_t* __restrict__ kept,
               const int32_t* __restrict__ sd, const int32_t* __restrict__ sq, SSet S,
               uint16_t* __restrict__ bpack, float* __restrict__ b32, DomRec* __restrict__ dom,
               float* __restrict__ domf, unsigned int* __restrict__ umax) {
  constexpr int n = B * B;
  constexpr int Kp = PackGeom<B>::Kp;
  constexpr int NG = Kp / 8;  // 16-byte groups per operand row
  __shared__ unsigned int s_umax;
  grid_dep_sync();
  if (threadIdx.x == 0) s_umax = 0;
  __syncthreads();
  const int64_t S_tot = slot_off[n_images];
  for (int64_t w = (int64_t)blockIdx.x * kPackThreads + threadIdx.x; w < S_tot * NG;
       w += (int64_t)gridDim.x * kPackThreads) {
    const int64_t slot = w / NG;
    const int g = (int)(w % NG);
    const int im = find_segment(slot_off, n_images, slot);
    const int64_t j = slot - slot_off[im];
    if (j >= st[im].nkept) continue;
    const ImgDev I = imgs[im];
    const int32_t pos = kept[slot];
    const int x0 = (pos % I.px) * L, y0 = (pos / I.px) * L;
    // pixel pairs as 2-byte loads where every pair starts on an even address
    const bool pairs = ((((uintptr_t)I.pix) | (uintptr_t)I.pitch | (uintptr_t)x0) & 1) == 0;
    uint8_t* tile_blk = bpack ? (uint8_t*)bpack + (slot >> 7) * (int64_t)tc_tile_bytes(B) : nullptr;
    if constexpr (B == 16) {
      // a warp per domain (NG = 32): lane g takes cell column cj = g % 16 of
      // every other cell row, so that each load of a half-warp reads 32
      // consecutive pixels of one image row; one f16 store per cell
      const int cj = g & 15;
#pragma unroll 2
      for (int ci = g >> 4; ci < B; ci += 2) {
        const uint8_t* p = I.pix + (int64_t)(y0 + 2 * ci) * I.pitch + (x0 + 2 * cj);
        int ds;
        if (pairs) {
          const uchar2 a = *(const uchar2*)p;
          const uchar2 b = *(const uchar2*)(p + I.pitch);
          ds = a.x + a.y + b.x + b.y;
        } else {
          ds = p[0] + p[1] + p[I.pitch] + p[I.pitch + 1];
        }
        const int e = ci * B + cj;
        if (bpack) ((uint16_t*)tile_blk)[bpack_index<B>(slot & 127, e)] = f16_bits(ds - 512);
        if (b32) b32[slot * n + e] = (float)(ds - 512);
      }
    }
    int v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = 8 * g + u;
      v[u] = 0;  // K padding (B = 2: K = 4 of 16)
      if (B < 16 && e < n) {
        const int ci = e / B, cj = e % B;
        const uint8_t* p = I.pix + (int64_t)(y0 + 2 * ci) * I.pitch + (x0 + 2 * cj);
        int ds;
        if (pairs) {
          const uchar2 a = *(const uchar2*)p;
          const uchar2 b = *(const uchar2*)(p + I.pitch);
          ds = a.x + a.y + b.x + b.y;
        } else {
          ds = p[0] + p[1] + p[I.pitch] + p[I.pitch + 1];
        }
        v[u] = ds - 512;
      }
    }
    if (B < 16 && bpack) {
      uint4 q;
      q.x = f16_bits(v[0]) | ((uint32_t)f16_bits(v[1]) << 16);
      q.y = f16_bits(v[2]) | ((uint32_t)f16_bits(v[3]) << 16);
      q.z = f16_bits(v[4]) | ((uint32_t)f16_bits(v[5]) << 16);
      q.w = f16_bits(v[6]) | ((uint32_t)f16_bits(v[7]) << 16);
      *(uint4*)((uint16_t*)tile_blk + bpack_index<B>(slot & 127, 8 * g)) = q;
    }
    if (B < 16 && b32) {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (8 * g + u < n) b32[slot * n + 8 * g + u] = (float)v[u];
    }
  }
  // the domains' records: one thread per slot
  for (int64_t slot = (int64_t)blockIdx.x * kPackThreads + threadIdx.x; slot < S_tot;
       slot += (int64_t)gridDim.x * kPackThreads) {
    const int im = find_segment(slot_off, n_images, slot);
    if (slot - slot_off[im] >= st[im].nkept) continue;
    const int32_t pos = kept[slot];
    uint8_t* tile_blk = bpack ? (uint8_t*)bpack + (slot >> 7) * (int64_t)tc_tile_bytes(B) : nullptr;
    {
      const int64_t gpos = off[im] + pos;
      const int64_t s = sd[gpos], s2 = sq[gpos];
      DomRec r;
      r.v = (int64_t)n * s2 - s * s;
      r.sdp = (int32_t)(s - 512 * n);
      r.pos = pos;
      dom[slot] = r;
      // Scores are E' / (8 q n) with E' = p^2 V - 8 p q C (see the match
      // kernels): explicit sets store p_t^2 V / (8 q n); the grid stores
      // V / (8 q n) and 4 q n / V, the scale of the real minimiser
      // p* = 4 q C / V.  Layout: per 128-slot tile, four planes of 128
      // floats {sum Ds', F0, F1, 0}, so a tile's constants are one
      // contiguous 2 KB block and each plane loads as float4 vectors.
      const double u = (double)r.v / (8.0 * S.q * n);
      // largest u of the level (non-negative floats order as their bits):
      // bounds the scores' rounding errors in the matcher
      atomicMax(&s_umax, __float_as_uint(__double2float_ru(u)));
      float f0, f1, f2 = 0.0f;
      if (S.exact) {
        // exact s: G of the pair is y^2 n^2 / V below the clamp point
        // y = V / (4 n) and n y / 2 - V / 16 above it (y = C / n)
        f0 = r.v > 0 ? (float)((double)n * n / (double)r.v) : 0.0f;
        f1 = (float)((double)r.v / (4.0 * n));
        f2 = (float)((double)r.v / 16.0);
      } else if (S.grid) {
        f0 = (float)u;
        f1 = r.v > 0 ? (float)(4.0 * S.q * n / (double)r.v) : 0.0f;
      } else {
        f0 = (float)(u * S.p[0] * S.p[0]);
        f1 = S.m > 1 ? (float)(u * S.p[1] * S.p[1]) : 0.0f;
      }
      float* ft = domf + (slot >> 7) * (4 * kTileDoms) + (slot & 127);
      ft[0] = (float)r.sdp;
      ft[kTileDoms] = f0;
      ft[2 * kTileDoms] = f1;
      ft[3 * kTileDoms] = f2;
      if (B <= 8 && tile_blk) {  // the same records inside the tile block
        float* fb = (float*)(tile_blk + tc_op_bytes(B)) + (slot & 127);
        fb[0] = (float)r.sdp;
        fb[kTileDoms] = f0;
        fb[2 * kTileDoms] = f1;
        fb[3 * kTileDoms] = f2;
        ((DomRec*)(tile_blk + tc_op_bytes(B) + 4 * kTileDoms * 4))[slot & 127] = r;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_umax) atomicMax(umax, s_umax);
}

// ---------------------------------------------------------------- driver
// The pool kernels run on side streams beside the level chain.  Launched with
// programmatic serialisation (launch_dep) their next kernels' blocks wait on
// the SMs early; measured on a 512 x 512 encode that slows the tensor path's
// level chain (0.9575 against 0.9447 ms per encode) but speeds the FP32 path
// (10.9 against 12.7 ms), so only the FP32 path's pools use it.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pool(const PoolLevel& pl, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                               size_t smem, cudaStream_t st, Args... args) {
  return pl.want_f32 ? launch_dep(kernel, grid, block, smem, st, args...)
                     : launch_std(kernel, grid, block, smem, st, args...);
}

template <int B>
static int pool_build_B(PoolLevel& pl, const int64_t* d_dT, cudaStream_t st) {
  const int ni = pl.n_images;
  const int nsm = pl.nsm > 0 ? pl.nsm : 148;
  const int64_t runs = pl.h_run_off[ni];
  if constexpr (B == 16) {
    const int64_t blocks = ceil_div64(runs > 0 ? runs : 1, kPoolWarpThreads / 32);
    const int grid = (int)(blocks < (int64_t)nsm * 8 ? blocks : (int64_t)nsm * 8);
    FIC_CUDA_TRY(launch_pool(pl, k_pool_stats_warp16, dim3(grid), dim3(kPoolWarpThreads), 0, st,
                            pl.img.as<ImgDev>(), pl.off.as<int64_t>(), pl.run_off.as<int64_t>(),
                            ni, pl.L, d_dT, pl.keys.as<int64_t>(), pl.sd.as<int32_t>(),
                            pl.sq.as<int32_t>()));
    return FIC_OK;
  }
  const int64_t blocks = ceil_div64(runs > 0 ? runs : 1, kPoolLaneThreads);
  const int grid = (int)(blocks < (int64_t)nsm * 3 ? blocks : (int64_t)nsm * 3);
  FIC_CUDA_TRY(launch_pool(pl, k_pool_stats_lane<B>, dim3(grid), dim3(kPoolLaneThreads),
                          PoolLaneSmem<B>::BYTES, st, pl.img.as<ImgDev>(), pl.off.as<int64_t>(),
                          pl.run_off.as<int64_t>(), ni, pl.L, d_dT, pl.keys.as<int64_t>(),
                          pl.sd.as<int32_t>(), pl.sq.as<int32_t>()));
  return FIC_OK;
}

int pool_build(PoolLevel& pl, const int64_t* d_dT, cudaStream_t st) {
  const double pct = pl.pct;
  const int ni = pl.n_images;
  const int64_t P = pl.P_tot;
  int rc = FIC_OK;
  switch (pl.B) {
    case 16: rc = pool_build_B<16>(pl, d_dT, st); break;
    case 8: rc = pool_build_B<8>(pl, d_dT, st); break;
    case 4: rc = pool_build_B<4>(pl, d_dT, st); break;
    case 2: rc = pool_build_B<2>(pl, d_dT, st); break;
    default: return FIC_EINVAL;
  }
  if (rc) return rc;
  SelState* sel = pl.sel.as<SelState>();
  uint32_t* hist = pl.hist.as<uint32_t>();
  const int64_t* off = pl.off.as<int64_t>();
  int64_t pmax = 0;
  for (int i = 0; i < ni; ++i) pmax = std::max(pmax, pl.h_off[i + 1] - pl.h_off[i]);
  if (pmax <= kSelFusedMax) {
    FIC_CUDA_TRY(launch_pool(pl, k_select_compact, dim3(ni), dim3(kSelFusedThreads), kSelDynBytes, st,
                            pl.keys.as<int64_t>(), off, pl.slot_off.as<int64_t>(), pct, pl.top_k,
                            sel, pl.kept.as<int32_t>(), pl.umax.as<unsigned int>()));
  } else {
    k_sel_init<<<ceil_div(ni * kSelBins, 256), 256, 0, st>>>(off, ni, pct, pl.top_k, sel, hist);
    const int nb = (int)ceil_div64(P > 0 ? P : 1, (int64_t)kSelThreads * kSelPerThread);
    for (int pass = 0; pass < kSelPasses; ++pass) {
      const int shift = (kSelPasses - 1 - pass) * kSelBits;
      k_sel_hist<<<nb, kSelThreads, 0, st>>>(pl.keys.as<int64_t>(), off, ni, shift, sel, hist);
      k_sel_find<<<ni, kSelBins, 0, st>>>(sel, hist, pass == kSelPasses - 1);
    }
    k_sel_bases<<<1, 32, 0, st>>>(sel, ni);
    KeptCompact kc{pl.keys.as<int64_t>(), off, pl.slot_off.as<int64_t>(), sel,
                   pl.kept.as<int32_t>(), ni};
    FIC_CUDA_TRY(scan_compact(kc, P, pl.scan_scratch.as<int32_t>(), pl.total.as<int64_t>(), st));
    FIC_CUDA_TRY(cudaMemsetAsync(pl.umax.p, 0, sizeof(unsigned int), st));
  }

  const int nsm = pl.nsm > 0 ? pl.nsm : 148;
  uint16_t* bp = pl.want_tc ? pl.bpack.as<uint16_t>() : nullptr;
  float* b32 = pl.want_f32 ? pl.b32.as<float>() : nullptr;
#define FIC_PACK(BB)                                                                           \
  {                                                                                            \
    const int64_t work = (pl.S_tot > 0 ? pl.S_tot : 1) * (PackGeom<BB>::Kp / 8);              \
    const int64_t blocks = ceil_div64(work, kPackThreads);                                     \
    const int grid = (int)(blocks < (int64_t)nsm * 16 ? blocks : (int64_t)nsm * 16);          \
    FIC_CUDA_TRY(launch_pool(pl, k_pack_domains<BB>, dim3(grid), dim3(kPackThreads), 0, st,       \
                            pl.img.as<ImgDev>(), off, pl.slot_off.as<int64_t>(), ni, pl.L,     \
                            sel, pl.kept.as<int32_t>(), pl.sd.as<int32_t>(),                   \
                            pl.sq.as<int32_t>(), pl.sset, bp, b32, pl.dom.as<DomRec>(),        \
                            pl.domf.as<float>(), pl.umax.as<unsigned int>()));                \
  }
  switch (pl.B) {
    case 16: FIC_PACK(16) break;
    case 8: FIC_PACK(8) break;
    case 4: FIC_PACK(4) break;
    default: FIC_PACK(2) break;
  }
#undef FIC_PACK
  FIC_CUDA_TRY(cudaGetLastError());
  return FIC_OK;
}

}  // namespace fic
