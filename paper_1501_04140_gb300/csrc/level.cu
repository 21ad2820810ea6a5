// level.cu -- per-level steps around the matcher (Sec. 2):
//   k_range_pack     active ranges -> exact moments and the 8 isometric copies
//                    T_k^-1(R) as matcher rows (f16 r - 128 and/or fp32);
//   k_plan           work items (image, 16-range M tile, chunk of 128-domain
//                    tiles) over a batch, from device-side counts;
//   k_reduce_final   best candidate of every range over all domain chunks
//                    (and the 8 isometry rows of the FP32 path), then Eq. 1
//                    and Eq. 3 in exact integers for the chosen map, and the
//                    split decision: accept when E <= n T^2 (last level:
//                    always), otherwise four children (16 -> 8 -> 4 -> 2);
//   k_reduce_moments the same on the tensor path, from exact moments;
//   k_split          the saved codes and the next level's ranges, from the
//                    reducer's accepted counts per tile (and the next
//                    level's plan).
#include <math.h>

#include <algorithm>

#include "fic_internal.h"
#include "level.cuh"
#include "scan.cuh"

namespace fic {

// One block: exclusive scan of nb counts in place; *total = their sum.
__device__ void block_scan_counts(int32_t* cnt, int nb, int64_t* total) {
  __shared__ int sw[32];
  __shared__ int tot;
  int64_t carry = 0;
  for (int base = 0; base < nb; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? cnt[i] : 0;
    const int before = block_excl_scan(v, sw, &tot);
    if (i < nb) cnt[i] = (int32_t)(carry + before);
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void __launch_bounds__(1024) k_scan_blocks(int32_t* cnt, int nb, int64_t* total) {
  block_scan_counts(cnt, nb, total);
}

// ---------------------------------------------------------------- range operand
// One thread per range pixel (256 / n ranges per block): the pixel r goes to
// its place in each of the 8 rows T_k^-1(R) (<T_k^-1 R, D> = <R, T_k D>), and
// the block reduces the range's moments in shared memory.  Also resets the
// range's screening threshold for the matcher.
constexpr int kRangePackThreads = 256;

template <int B>
__global__ void __launch_bounds__(kRangePackThreads)
k_range_pack(const ImgDev* __restrict__ imgs, const RangeRec* __restrict__ rec,
             const int64_t* __restrict__ n_act, int Kp, RangeMom* __restrict__ mom,
             uint32_t* __restrict__ gthr, uint16_t* __restrict__ apack,
             float* __restrict__ a32) {
  constexpr int n = B * B;
  constexpr int RPB = kRangePackThreads / n;  // ranges per block step
  __shared__ int s_sr[RPB], s_s2[RPB], s_sa[RPB];
  grid_dep_sync();
  const int64_t N = *n_act;
  const int lr = threadIdx.x / n, e = threadIdx.x % n;
  const int i = e / B, j = e % B;
  for (int64_t g0 = (int64_t)blockIdx.x * RPB; g0 < N; g0 += (int64_t)gridDim.x * RPB) {
    if (threadIdx.x < RPB) s_sr[threadIdx.x] = 0, s_s2[threadIdx.x] = 0, s_sa[threadIdx.x] = 0;
    __syncthreads();
    const int64_t g = g0 + lr;
    if (g < N) {
      const RangeRec r = rec[g];
      const ImgDev I = imgs[r.img];
      const int v = I.pix[(int64_t)(r.y + i) * I.pitch + r.x + j];
      atomicAdd(&s_sr[lr], v);
      atomicAdd(&s_s2[lr], v * v);  // <= 256 * 255^2 < 2^31
      atomicAdd(&s_sa[lr], v >= 128 ? v - 128 : 128 - v);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        int si, sj;
        iso_src(B, k, i, j, &si, &sj);
        const int d = si * B + sj;
        if (apack)
          apack[(((g * (Kp >> 3)) + (d >> 3)) * 8 + k) * 8 + (d & 7)] =
              __half_as_ushort(__int2half_rn(v - 128));
        if (a32) a32[(g * 8 + k) * n + d] = (float)(v - 128);
      }
      if (apack)  // zero the K padding (B = 2: K = 4 of 16)
        for (int d = n + e; d < Kp; d += n)
#pragma unroll
          for (int k = 0; k < 8; ++k) apack[(((g * (Kp >> 3)) + (d >> 3)) * 8 + k) * 8 + (d & 7)] = 0;
    }
    __syncthreads();
    if (g < N && e == 0) {
      const int sr = s_sr[lr];
      RangeMom m;
      m.sr = sr;
      m.srp = sr - 128 * n;
      m.a = (int64_t)n * s_s2[lr] - (int64_t)sr * sr;
      m.sabs = s_sa[lr];
      m.pad = 0;
      mom[g] = m;
      if (gthr) gthr[g] = kThrInit;
    }
    // the sums are read before the next pass clears them
    __syncthreads();
  }
}

int launch_range_pack(int B, const ImgDev* imgs, const RangeRec* rec, const int64_t* n_act,
                      int64_t cap, int Kp, RangeMom* mom, uint32_t* gthr, uint16_t* apack,
                      float* a32, int nsm, cudaStream_t st) {
  const int threads = kRangePackThreads;
  const int64_t rpb = threads / (B * B);
  // grid-stride over the device count: at most 8 resident blocks per SM
  const int64_t gmax = nsm > 0 ? 8 * (int64_t)nsm : 65535;
  const int grid = (int)std::min<int64_t>(ceil_div64(cap > 0 ? cap : 1, rpb), gmax);
  cudaError_t e;
#define FIC_RP(BB) launch_dep(k_range_pack<BB>, dim3(grid), dim3(threads), 0, st, imgs, rec, n_act, \
                              Kp, mom, gthr, apack, a32)
  switch (B) {
    case 16: e = FIC_RP(16); break;
    case 8: e = FIC_RP(8); break;
    case 4: e = FIC_RP(4); break;
    case 2: e = FIC_RP(2); break;
    default: return FIC_EINVAL;
  }
#undef FIC_RP
  return e == cudaSuccess ? FIC_OK : FIC_ECUDA;
}

// ---------------------------------------------------------------- plan
// One thread: images are few (<= kMaxImages) and this runs once per level.
// The block also zeroes the reducer's accepted counts per compaction tile.
// Run by one whole block (k_plan, or block 0 of the previous level's k_split).
__device__ void plan_level(const PlanArgs& p, const int64_t* __restrict__ act_off,
                           const int64_t* __restrict__ act_cnt) {
  if (p.tile_acc)
    for (int i = threadIdx.x; i < p.n_tiles; i += blockDim.x) p.tile_acc[i] = 0;
  if (threadIdx.x != 0) return;
  // the split counters of the level start at zero (the reduction adds)
  for (int i = 0; i < p.n_images; ++i) p.acc_cnt[i] = 0, p.rej_cnt[i] = 0;
  int64_t work = 0;
  for (int i = 0; i < p.n_images; ++i)
    work += ceil_div64(act_cnt[i], kTileRanges) * ceil_div64(p.sel[i].nkept, kTileDoms);
  int64_t ch = ceil_div64(work, p.target_items > 0 ? p.target_items : 1);
  if (ch < 1) ch = 1;
  const int64_t room = p.item_cap - p.mt_cap;
  if (room > 0) {
    const int64_t need = ceil_div64(work, room);
    if (ch < need) ch = need;
  }
  int64_t items = 0;
  for (int i = 0; i < p.n_images; ++i) {
    const int64_t mt = ceil_div64(act_cnt[i], kTileRanges);
    const int64_t nt = ceil_div64(p.sel[i].nkept, kTileDoms);
    const int64_t c = nt > 0 ? ceil_div64(nt, ch) : 0;
    p.item_off[i] = items;
    p.chunks[i] = (int32_t)c;
    items += mt * c;
  }
  p.item_off[p.n_images] = items;
  p.meta->chunk_tiles = (int32_t)ch;
  p.meta->items = items;
  p.meta->overflow = items > p.item_cap ? 1 : 0;
}

__global__ void k_plan(PlanArgs p, const int64_t* __restrict__ act_off,
                       const int64_t* __restrict__ act_cnt) {
  grid_dep_sync();
  if (blockIdx.x == 0) plan_level(p, act_off, act_cnt);
}

// ---------------------------------------------------------------- reduce + exact map
// One warp per range: the lanes share the range's partial candidates (every
// domain chunk, and the isometry rows of the FP32 path) and then the pixels
// of the chosen pair; the exact moments are warp sums.  The split decision of
// the quadtree (accept when E <= n T^2, the last level always) is taken here
// as well, with per-image counts for the compaction that follows.
constexpr int kReduceWarps = 8;

__device__ inline void cand_min(Cand& b, const Cand& x) {
  if (x.score < b.score || (x.score == b.score && x.key < b.key)) b = x;
}

template <int B>
__global__ void __launch_bounds__(32 * kReduceWarps)
k_reduce_final(const ImgDev* __restrict__ imgs, const RangeRec* __restrict__ rec,
               const int64_t* __restrict__ n_act, const int64_t* __restrict__ act_off,
               const int64_t* __restrict__ pool_off, int n_images, int L,
               const SelState* __restrict__ sel, const int64_t* __restrict__ item_off,
               const int32_t* __restrict__ chunks, const Cand* __restrict__ part, int iso_rows,
               SSet S, int level, const PlanMeta* __restrict__ meta, uint32_t* __restrict__ status,
               fic_transform* __restrict__ res, double e_thr, int last, uint8_t* __restrict__ acc,
               int32_t* __restrict__ acc_cnt, int32_t* __restrict__ rej_cnt,
               int32_t* __restrict__ tile_acc, PosMoments pm) {
  constexpr int n = B * B;
  const int lane = threadIdx.x & 31;
  grid_dep_sync();
  const int64_t N = *n_act;
  const bool overflow = meta->overflow != 0;
  if (overflow && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatusOverflow);
  const int64_t w0 = (int64_t)blockIdx.x * kReduceWarps + (threadIdx.x >> 5);
  const int64_t wstep = (int64_t)gridDim.x * kReduceWarps;
  for (int64_t g = w0; g < N; g += wstep) {
    const RangeRec r = rec[g];
    const int im = r.img;
    const int64_t l = g - act_off[im];
    const int64_t m = l / kTileRanges;
    const int rr = (int)(l % kTileRanges);
    const int nc = overflow ? 0 : chunks[im];
    Cand best{INT64_MAX, INT64_MAX};
    int64_t bv = 0;  // exact s: the best's V
    for (int e = lane; e < nc * iso_rows; e += 32) {
      const int c = e / iso_rows, k = e % iso_rows;
      const Cand x = part[((item_off[im] + m * nc + c) * kTileRanges + rr) * iso_rows + k];
      if (S.exact) {
        const int64_t xv = x.key == INT64_MAX ? 0 : pos_v(pm, im, x.key >> 3, n);
        if (exact_better(x.score, xv, x.key, best.score, bv, best.key)) best = x, bv = xv;
      } else {
        cand_min(best, x);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      Cand x;
      x.score = __shfl_xor_sync(0xffffffffu, best.score, o);
      x.key = __shfl_xor_sync(0xffffffffu, best.key, o);
      const int64_t xv = __shfl_xor_sync(0xffffffffu, bv, o);
      if (S.exact) {
        if (exact_better(x.score, xv, x.key, best.score, bv, best.key)) best = x, bv = xv;
      } else {
        cand_min(best, x);
      }
    }
    const ImgDev I = imgs[im];
    const bool bad = best.key == INT64_MAX || best.key < 0 ||
                     best.key / (8 * (int64_t)S.m) >= (int64_t)I.px * I.py;
    fic_transform t{};
    t.level = level;
    t.x = r.x;
    t.y = r.y;
    t.size = B;
    if (!bad) {
      const int s_idx = (int)(best.key % S.m);
      const int iso = (int)((best.key / S.m) % 8);
      const int pos = (int)(best.key / (8 * (int64_t)S.m));
      const int dx = (pos % I.px) * L, dy = (pos / I.px) * L;
      // Exact moments of the chosen pair: Eq. 1 with D = Ds / 4 and s = p / q.
      int64_t sr = 0, sr2 = 0, sdd = 0, sdd2 = 0, cor = 0;
      for (int e = lane; e < n; e += 32) {
        const int i = e / B, j = e % B;
        int si, sj;
        iso_src(B, iso, i, j, &si, &sj);
        const uint8_t* pd = I.pix + (int64_t)(dy + 2 * si) * I.pitch + (dx + 2 * sj);
        const int64_t ds = (int64_t)pd[0] + pd[1] + pd[I.pitch] + pd[I.pitch + 1];
        const int64_t rv = I.pix[(int64_t)(r.y + i) * I.pitch + r.x + j];
        sr += rv;
        sr2 += rv * rv;
        sdd += ds;
        sdd2 += ds * ds;
        cor += rv * ds;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        sr2 += __shfl_xor_sync(0xffffffffu, sr2, o);
        sdd += __shfl_xor_sync(0xffffffffu, sdd, o);
        sdd2 += __shfl_xor_sync(0xffffffffu, sdd2, o);
        cor += __shfl_xor_sync(0xffffffffu, cor, o);
      }
      const int64_t A = n * sr2 - sr * sr;
      const int64_t C = n * cor - sr * sdd;
      const int64_t V = n * sdd2 - sdd * sdd;
      t.dom_index = pos;
      t.dom_x = dx;
      t.dom_y = dy;
      t.iso = iso;
      if (S.exact) {
        // Eq. 2's s clamped to [0, 1] as sn / sd; Eq. 3's o; E in the
        // moment form n E = A - G (double operations in this order)
        int64_t sn = 0, sd = 1;
        if (C > 0 && V > 0) {
          if (4 * C >= V) sn = 1;
          else sn = 4 * C, sd = V;
        }
        t.s_idx = 0;
        t.p = t.q = 0;
        t.e_num = 0;
        t.o_num = 0;
        t.s = __ddiv_rn((double)sn, (double)sd);
        t.o = __ddiv_rn((double)(4 * sd * sr - sn * sdd), __dmul_rn(__dmul_rn(4.0, (double)sd), (double)n));
        if (sn == 0)
          t.e = __ddiv_rn((double)A, (double)n);
        else if (sn == sd)
          t.e = __ddiv_rn((double)(16 * A - 8 * C + V), __dmul_rn(16.0, (double)n));
        else
          t.e = __ddiv_rn(__dsub_rn((double)A, __ddiv_rn(__dmul_rn((double)C, (double)C), (double)V)),
                          (double)n);
      } else {
        const int64_t p = S.p[s_idx], q = S.q;
        // 16 q^2 n^2 E = n (16 q^2 A - 8 p q C + p^2 V)
        const int64_t enum_ = (int64_t)n * (16 * q * q * A - 8 * p * q * C + p * p * V);
        t.s_idx = s_idx;
        t.p = (int32_t)p;
        t.q = (int32_t)q;
        t.e_num = enum_;
        t.o_num = 4 * q * sr - p * sdd;  // Eq. 3 times 4 q n
        t.e = (double)enum_ / (16.0 * (double)(q * q) * (double)n * (double)n);
        t.s = (double)p / (double)q;
        t.o = (double)t.o_num / (4.0 * (double)q * (double)n);
      }
    } else {  // no candidate (plan overflow): flagged, never read as a map
      t.dom_index = -1;
      t.e = INFINITY;
      t.e_num = INT64_MAX;
    }
    if (lane == 0) {
      res[g] = t;
      if (acc) {
        // Sec. 2: keep the map when its error is acceptable, else split
        const bool a = last || (t.e <= e_thr);
        acc[g] = a ? 1 : 0;
        atomicAdd(a ? &acc_cnt[im] : &rej_cnt[im], 1);
        if (a) atomicAdd(&tile_acc[g / kScanTile], 1);
      }
    }
  }
}

// Tensor path: every candidate's score is exact -- E' = p^2 V - 8 p q C of
// the predefined or grid S, or the pair's C in the exact-s mode -- so the
// chosen map follows from exact moments already at hand: the range's A and
// sum r (RangeMom) and the domain's sum Ds and sum Ds^2 (the pool's
// per-position sums, V = n sum Ds^2 - (sum Ds)^2).  One thread per range, no
// pixel reads; the same values as k_reduce_final's sums over the pixels.
// The accept / reject counts are aggregated per warp: a warp's 32 ranges lie
// in one kScanTile-range tile, and usually in one image.
template <int B>
__global__ void __launch_bounds__(256)
k_reduce_moments(const ImgDev* __restrict__ imgs, const RangeRec* __restrict__ rec,
                 const int64_t* __restrict__ n_act, const int64_t* __restrict__ act_off,
                 int n_images, int L, const int64_t* __restrict__ item_off,
                 const int32_t* __restrict__ chunks, const Cand* __restrict__ part, SSet S,
                 int level, const PlanMeta* __restrict__ meta, uint32_t* __restrict__ status,
                 const RangeMom* __restrict__ mom, fic_transform* __restrict__ res, double e_thr,
                 int last, uint8_t* __restrict__ acc, int32_t* __restrict__ acc_cnt,
                 int32_t* __restrict__ rej_cnt, int32_t* __restrict__ tile_acc, PosMoments pm) {
  constexpr int n = B * B;
  grid_dep_sync();
  const int lane = threadIdx.x & 31;
  const int64_t N = *n_act;
  const bool overflow = meta->overflow != 0;
  if (overflow && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, kStatusOverflow);
  // (block-uniform loop: every lane of a warp takes part in its votes)
  for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x; g0 < N;
       g0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = g0 + threadIdx.x;
    const bool valid = g < N;
    int im = -1;
    bool ok_acc = false;
    if (valid) {
      const RangeRec r = rec[g];
      im = r.img;
      const int64_t l = g - act_off[im];
      const int64_t m = l / kTileRanges;
      const int rr = (int)(l % kTileRanges);
      const int nc = overflow ? 0 : chunks[im];
      Cand best{INT64_MAX, INT64_MAX};
      int64_t bv = 0;  // exact s: the best's V
      for (int c = 0; c < nc; ++c) {
        const Cand x = part[(item_off[im] + m * nc + c) * kTileRanges + rr];
        if (S.exact) {
          const int64_t xv = x.key == INT64_MAX ? 0 : pos_v(pm, im, x.key >> 3, n);
          if (exact_better(x.score, xv, x.key, best.score, bv, best.key)) best = x, bv = xv;
        } else {
          cand_min(best, x);
        }
      }
      const ImgDev I = imgs[im];
      const bool bad = best.key == INT64_MAX || best.key < 0 ||
                       best.key / (8 * (int64_t)S.m) >= (int64_t)I.px * I.py;
      fic_transform t{};
      t.level = level;
      t.x = r.x;
      t.y = r.y;
      t.size = B;
      if (!bad) {
        const int s_idx = (int)(best.key % S.m);
        const int iso = (int)((best.key / S.m) % 8);
        const int pos = (int)(best.key / (8 * (int64_t)S.m));
        const RangeMom mo = mom[g];
        const int64_t gp = pm.off[im] + pos;
        const int64_t sdd = pm.sd[gp], sdd2 = pm.sq[gp];
        const int64_t sr = mo.sr, A = mo.a;
        const int64_t V = (int64_t)n * sdd2 - sdd * sdd;
        t.dom_index = pos;
        t.dom_x = (pos % I.px) * L;
        t.dom_y = (pos / I.px) * L;
        t.iso = iso;
        if (S.exact) {
          // Eq. 2's s clamped to [0, 1] as sn / sd; Eq. 3's o; E in the
          // moment form n E = A - G (double operations in this order)
          const int64_t C = best.score;
          int64_t sn = 0, sd = 1;
          if (C > 0 && V > 0) {
            if (4 * C >= V) sn = 1;
            else sn = 4 * C, sd = V;
          }
          t.s_idx = 0;
          t.p = t.q = 0;
          t.e_num = 0;
          t.o_num = 0;
          t.s = __ddiv_rn((double)sn, (double)sd);
          t.o = __ddiv_rn((double)(4 * sd * sr - sn * sdd),
                          __dmul_rn(__dmul_rn(4.0, (double)sd), (double)n));
          if (sn == 0)
            t.e = __ddiv_rn((double)A, (double)n);
          else if (sn == sd)
            t.e = __ddiv_rn((double)(16 * A - 8 * C + V), __dmul_rn(16.0, (double)n));
          else
            t.e = __ddiv_rn(__dsub_rn((double)A, __ddiv_rn(__dmul_rn((double)C, (double)C), (double)V)),
                            (double)n);
        } else {
          const int64_t p = S.p[s_idx], q = S.q;
          // 16 q^2 n^2 E = n (16 q^2 A - 8 p q C + p^2 V) = n (16 q^2 A + E')
          const int64_t enum_ = (int64_t)n * (16 * q * q * A + best.score);
          t.s_idx = s_idx;
          t.p = (int32_t)p;
          t.q = (int32_t)q;
          t.e_num = enum_;
          t.o_num = 4 * q * sr - p * sdd;  // Eq. 3 times 4 q n
          t.e = (double)enum_ / (16.0 * (double)(q * q) * (double)n * (double)n);
          t.s = (double)p / (double)q;
          t.o = (double)t.o_num / (4.0 * (double)q * (double)n);
        }
      } else {  // no candidate (plan overflow): flagged, never read as a map
        t.dom_index = -1;
        t.e = INFINITY;
        t.e_num = INT64_MAX;
      }
      res[g] = t;
      ok_acc = last || (t.e <= e_thr);  // Sec. 2: keep when acceptable, else split
      if (acc) acc[g] = ok_acc ? 1 : 0;
    }
    if (acc) {
      const unsigned am = __ballot_sync(0xffffffffu, valid && ok_acc);
      const unsigned rm = __ballot_sync(0xffffffffu, valid && !ok_acc);
      const int im0 = __shfl_sync(0xffffffffu, im, 0);
      if (__all_sync(0xffffffffu, !valid || im == im0)) {
        if (lane == 0) {
          if (am) atomicAdd(&acc_cnt[im0], __popc(am));
          if (rm) atomicAdd(&rej_cnt[im0], __popc(rm));
        }
      } else if (valid) {
        atomicAdd(ok_acc ? &acc_cnt[im] : &rej_cnt[im], 1);
      }
      if (lane == 0 && am) atomicAdd(&tile_acc[(g0 + (threadIdx.x & ~31)) / kScanTile], __popc(am));
    }
  }
}

int launch_reduce_final(int B, const ImgDev* imgs, const RangeRec* rec, const int64_t* n_act,
                        int64_t cap, const int64_t* act_off, const int64_t* pool_off,
                        int n_images, int L, const SelState* sel, const int64_t* item_off,
                        const int32_t* chunks, const Cand* part, int iso_rows, const SSet& S,
                        int level, const PlanMeta* meta, uint32_t* status, fic_transform* res,
                        double rms, int last, uint8_t* acc, int32_t* acc_cnt, int32_t* rej_cnt,
                        int32_t* tile_acc, const PosMoments& pm, const RangeMom* mom, int nsm,
                        cudaStream_t st) {
  if (acc && !tile_acc) return FIC_EINVAL;
  if (iso_rows == 1 && mom) {  // tensor path: from the exact moments
    const int64_t gmax = nsm > 0 ? 8 * (int64_t)nsm : 65535;
    const int grid = (int)std::min<int64_t>(ceil_div64(cap > 0 ? cap : 1, 256), gmax);
    const double e_thr1 = (double)(B * B) * (rms * rms);
    cudaError_t e;
#define FIC_RM(BB)                                                                             \
  launch_dep(k_reduce_moments<BB>, dim3(grid), dim3(256), 0, st, imgs, rec, n_act, act_off,    \
             n_images, L, item_off, chunks, part, S, level, meta, status, mom, res, e_thr1,     \
             last, acc, acc_cnt, rej_cnt, tile_acc, pm)
    switch (B) {
      case 16: e = FIC_RM(16); break;
      case 8: e = FIC_RM(8); break;
      case 4: e = FIC_RM(4); break;
      case 2: e = FIC_RM(2); break;
      default: return FIC_EINVAL;
    }
#undef FIC_RM
    return e == cudaSuccess ? FIC_OK : FIC_ECUDA;
  }
  const int threads = 32 * kReduceWarps;
  // grid-stride over the device count: at most 8 resident blocks per SM
  const int64_t gmax = nsm > 0 ? 8 * (int64_t)nsm : 65535;
  const int grid = (int)std::min<int64_t>(ceil_div64(cap > 0 ? cap : 1, kReduceWarps), gmax);
  const double e_thr = (double)(B * B) * (rms * rms);
  cudaError_t e;
#define FIC_RF(BB)                                                                             \
  launch_dep(k_reduce_final<BB>, dim3(grid), dim3(threads), 0, st, imgs, rec, n_act, act_off,   \
             pool_off, n_images, L, sel, item_off, chunks, part, iso_rows, S, level, meta,       \
             status, res, e_thr, last, acc, acc_cnt, rej_cnt, tile_acc, pm)
  switch (B) {
    case 16: e = FIC_RF(16); break;
    case 8: e = FIC_RF(8); break;
    case 4: e = FIC_RF(4); break;
    case 2: e = FIC_RF(2); break;
    default: return FIC_EINVAL;
  }
#undef FIC_RF
  return e == cudaSuccess ? FIC_OK : FIC_ECUDA;
}

// ---------------------------------------------------------------- quadtree split
// (The accept / split flags and their per-image counts come from
// k_reduce_final: accept when E <= n T^2, compared in double as
// (double) e_num / (16 q^2 n^2) against n (T T); the last level accepts
// everything.)

struct SplitCompact {
  const int64_t* n_act;
  const uint8_t* acc;
  const fic_transform* res;
  const RangeRec* rec;
  fic_transform* codes;
  RangeRec* next;
  int half;
  __device__ int64_t size() const { return *n_act; }
  __device__ bool flag(int64_t g) const { return acc[g] != 0; }
  __device__ void emit(int64_t g, int64_t rank, bool f) const {
    if (f) {
      codes[rank] = res[g];
    } else if (next) {
      const RangeRec r = rec[g];
      RangeRec* o = next + 4 * rank;
      o[0] = RangeRec{r.img, r.x, r.y, (int32_t)g};
      o[1] = RangeRec{r.img, r.x + half, r.y, (int32_t)g};
      o[2] = RangeRec{r.img, r.x, r.y + half, (int32_t)g};
      o[3] = RangeRec{r.img, r.x + half, r.y + half, (int32_t)g};
    }
  }
};

// One thread per range of a kScanTile-range tile (so that the copies of
// all the tile's ranges are in flight at once): the tile's accepted ranges
// take consecutive code ranks from the accepted counts of the tiles before
// it -- which the block sums itself: only the tiles that hold active ranges
// get past the first check, so this stays small -- the others four children
// each, both in index order.  Block 0 also writes the per-image offsets of
// the codes saved at this level and of the next level's ranges (4 children
// per split range; images stay in order).
__global__ void __launch_bounds__(kScanTile)
k_split(SplitCompact f, const int32_t* __restrict__ tile_cnt, int n_images,
        const int32_t* __restrict__ acc_cnt, const int32_t* __restrict__ rej_cnt,
        int64_t* __restrict__ code_off, int64_t* __restrict__ next_off,
        int64_t* __restrict__ next_cnt, int64_t* __restrict__ next_n,
        int64_t* __restrict__ total, PlanArgs next_plan, int plan_next) {
  __shared__ int sw[32];
  grid_dep_sync();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int64_t a = 0, c = 0;
    for (int i = 0; i < n_images; ++i) {
      code_off[i] = a;
      if (next_off) next_off[i] = c;
      if (next_cnt) next_cnt[i] = 4 * (int64_t)rej_cnt[i];
      a += acc_cnt[i];
      c += 4 * (int64_t)rej_cnt[i];
    }
    code_off[n_images] = a;
    if (next_off) next_off[n_images] = c;
    if (next_n) *next_n = c;
    if (total) *total = a;
  }
  // the next level's work plan, from the counts just written (thread 0
  // wrote them; the other threads only zero the next level's tile counts)
  if (plan_next && blockIdx.x == 0) plan_level(next_plan, next_off, next_cnt);
  const int64_t n = f.size();
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  if (base >= n) return;  // uniform per block
  int part = 0;
  for (int t = threadIdx.x; t < (int)blockIdx.x; t += blockDim.x) part += tile_cnt[t];
  int first = 0;
  block_excl_scan(part, sw, &first);  // the block's sum: codes saved by the tiles before
  const int64_t i = base + threadIdx.x;
  const bool fl = i < n && f.flag(i);
  const int before = block_excl_scan(fl ? 1 : 0, sw, nullptr);
  const int64_t r = (int64_t)first + before;
  if (i < n) f.emit(i, fl ? r : i - r, fl);
}

int launch_split(const fic_transform* res, const RangeRec* rec, const int64_t* n_act, int64_t cap,
                 int B, int n_images, uint8_t* acc, int32_t* acc_cnt,
                 int32_t* rej_cnt, int64_t* code_off, fic_transform* codes, RangeRec* next,
                 int64_t* next_off, int64_t* next_cnt, int64_t* next_n, int32_t* tile_acc,
                 int64_t* total, const PlanArgs* next_plan, cudaStream_t st) {
  const int nb = (int)ceil_div64(cap > 0 ? cap : 1, kScanTile);
  SplitCompact sc{n_act, acc, res, rec, codes, next, B / 2};
  const PlanArgs np = next_plan ? *next_plan : PlanArgs{};
  const cudaError_t e = launch_dep(k_split, dim3(nb), dim3(kScanTile), 0, st, sc,
                                   (const int32_t*)tile_acc, n_images, (const int32_t*)acc_cnt,
                                   (const int32_t*)rej_cnt, code_off, next_off, next_cnt, next_n,
                                   total, np, next_plan && next_off && next_cnt ? 1 : 0);
  return e == cudaSuccess ? FIC_OK : FIC_ECUDA;
}

}  // namespace fic
