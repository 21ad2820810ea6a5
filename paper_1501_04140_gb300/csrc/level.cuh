// level.cuh -- launchers of the per-level steps and the matcher interface.
#pragma once

#include "fic_internal.h"

namespace fic {

struct PlanMeta {
  int64_t items;        // work items of the level
  int32_t chunk_tiles;  // 128-domain tiles per item (the last chunk may be shorter)
  int32_t overflow;     // 1 if items exceeded the capacity (nothing matched)
};

// Everything a matcher launch needs (device pointers).
// Per pool position (kept or not): sum Ds and sum Ds^2 of the domain's 2x2
// sums, for the V = n sum Ds^2 - (sum Ds)^2 that the exact-s order needs of a
// candidate known only by its key (pos * 8 + iso).
struct PosMoments {
  const int32_t* sd;
  const int32_t* sq;
  const int64_t* off;  // n_images + 1 (positions)
};
__device__ inline int64_t pos_v(const PosMoments& pm, int im, int64_t pos, int n) {
  const int64_t g = pm.off[im] + pos;
  const int64_t s = pm.sd[g], s2 = pm.sq[g];
  return (int64_t)n * s2 - s * s;
}

struct MatchArgs {
  int B, n, Kp, n_images;
  SSet S;
  float delta;                      // screening margin in score units (tensor path)
  const RangeMom* mom;              // per range
  const uint16_t* apack;            // f16 rows, core-matrix layout
  const float* a32;                 // fp32 rows
  const uint16_t* bpack;            // f16 domains, core-matrix layout
  const float* b32;                 // fp32 domains
  const DomRec* dom;                // per domain slot
  const float* domf;                // per 128-slot tile: planes {SD'}, {F0}, {F1}, {0}
  const float* umax;                // largest V / (8 q n) of the level's kept domains
  uint32_t* gthr;                   // per range: best screening threshold found so far
                                    // (order-preserving bits of a float), shared by
                                    // every CTA that scores the range
  const int64_t* act_off;           // n_images + 1 (ranges)
  const int64_t* act_cnt;           // n_images
  const int64_t* pool_off;          // n_images + 1 (domain slots)
  const SelState* sel;              // n_kept per image
  const int64_t* item_off;          // n_images + 1
  const int32_t* chunks;            // per image
  const PlanMeta* meta;
  Cand* part;                       // per item: 16 ranges x 8 isometry rows (FP32 path)
                                    // or 16 ranges (tensor path)
  uint32_t* status;                 // device status word
  PosMoments pm;                    // the exact-s mode's V of a key
  int inject;                       // test hook (kInjectDropTileCopy), 0 normally
  int groups_per_tile;              // tensor path, B <= 8: 1 or 2 epilogue groups per tile
};

// Test hook of the tensor matcher: the producer of CTA 0 leaves the first
// stage of its first work item unfilled, so the waits on it run out after
// kWaitLimitNs; the kernel then records kStatusTimeout and returns.
constexpr int kInjectDropTileCopy = FIC_FAULT_DROP_TILE_COPY;

int launch_range_pack(int B, const ImgDev* imgs, const RangeRec* rec, const int64_t* n_act,
                      int64_t cap, int Kp, RangeMom* mom, uint32_t* gthr, uint16_t* apack,
                      float* a32, int nsm, cudaStream_t st);

// Screening thresholds are shared between CTAs as order-preserving unsigned
// images of floats (atomicMin on the image = min on the float).
constexpr uint32_t kThrInit = 0xFF800000u;  // image of +inf
__device__ inline uint32_t thr_to_ord(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ inline float ord_to_thr(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

// A level's work plan (k_plan): work items from the device-side counts.
struct PlanArgs {
  int n_images;
  const SelState* sel;    // the level's pool: n_kept per image
  int target_items;       // work items wanted (items per CTA x CTAs)
  int64_t item_cap, mt_cap;
  PlanMeta* meta;
  int64_t* item_off;      // n_images + 1
  int32_t* chunks;        // per image
  int32_t* acc_cnt;       // zeroed: the reduction's per-image counts
  int32_t* rej_cnt;
  int32_t* tile_acc;      // zeroed: accepted ranges per kScanTile tile (may be null)
  int n_tiles;
};

__global__ void k_plan(PlanArgs p, const int64_t* act_off, const int64_t* act_cnt);

int launch_reduce_final(int B, const ImgDev* imgs, const RangeRec* rec, const int64_t* n_act,
                        int64_t cap, const int64_t* act_off, const int64_t* pool_off,
                        int n_images, int L, const SelState* sel, const int64_t* item_off,
                        const int32_t* chunks, const Cand* part, int iso_rows, const SSet& S,
                        int level, const PlanMeta* meta, uint32_t* status, fic_transform* res,
                        double rms, int last, uint8_t* acc, int32_t* acc_cnt, int32_t* rej_cnt,
                        int32_t* tile_acc, const PosMoments& pm, const RangeMom* mom, int nsm,
                        cudaStream_t st);

// The saved codes and the next level's ranges of a level whose reducer took
// the split decision (acc, the per-image counts and tile_acc, the accepted
// ranges of every kScanTile-range tile, counted by k_reduce_final).
int launch_split(const fic_transform* res, const RangeRec* rec, const int64_t* n_act, int64_t cap,
                 int B, int n_images, uint8_t* acc, int32_t* acc_cnt,
                 int32_t* rej_cnt, int64_t* code_off, fic_transform* codes, RangeRec* next,
                 int64_t* next_off, int64_t* next_cnt, int64_t* next_n, int32_t* tile_acc,
                 int64_t* total, const PlanArgs* next_plan, cudaStream_t st);

// Matchers: fill args.part for every planned item.  `grid` persistent CTAs.
int launch_match_f32(const MatchArgs& a, int grid, cudaStream_t st);
int launch_match_tc(const MatchArgs& a, int grid, cudaStream_t st);
int match_tc_prepare();  // per device, before the first launch

// Screening margin of the tensor path's float scores (score units, E'/(8qn)).
float screening_delta(int B, const SSet& S);

}  // namespace fic
