// match_tc.cu -- the tensor-core matcher (sm_103a tcgen05).
//
// Sec. 2's search scores every range against every kept domain under the 8
// isometries.  With the isometries applied to the range (<R, T_k D> =
// <T_k^-1 R, D>), the correlations of a level form one dense contraction
//     corr[domain, (range, k)] = sum_i (Ds_i - 512) (T_k^-1 R)_i ,  K = n,
// with columns r - 128 in [-128, 127] and rows Ds - 512 in [-512, 508]: small
// integers, exact in binary16.  Every partial sum, in any order, is an
// integer of magnitude at most n * 128 * 512 <= 2^24 (B = 16, K = 256), so
// the f32 accumulator of tcgen05.mma kind::f16 holds the exact integer
// correlation; one accumulator per tile takes the whole K (at B = 16 both
// K-half stages).
//
// Orientation.  The streamed 128-domain tile is the MMA's A operand (M =
// 128: one TMEM lane per domain) and the resident tile of 16 ranges x 8
// isometries is its B operand (N = 128 columns, the 8 isometries of a range
// adjacent).  An epilogue thread owns one domain: its per-domain constants
// sit in registers, and a range's 8 isometries are 8 of its own columns.
//
// Isometry reduction.  For s = p/q, E of Eq. 1 with o from Eq. 3 is, up to
// the range-only term, E' = p^2 V - 8 p q C with C = n <r', Ds'> - sum r'
// sum Ds' (exact integers).  V and both sums are the same for the 8
// isometric copies, so for p > 0 E' falls strictly as the correlation
// rises: of a (domain, range) pair, the isometry with the largest
// correlation (the lowest k among equals) wins for every s > 0, and for
// p = 0 every isometry gives E' = 0, where k = 0 has the lowest tie-break
// key.  The epilogue therefore reduces the 8 exact correlations to their
// maximum before any scoring: one score per (domain, range) and s.
//
// Warp roles of one persistent CTA per SM:
//   warp 0      producer: bulk copies (TMA engine) of the resident range
//               tile, the streamed 128-domain tiles (one stage per K half at
//               B = 16) and each tile's per-domain scoring planes and exact
//               records;
//   warp 1      allocates tensor memory and issues the MMAs (one thread);
//               at B <= 8 warp 2 issues too, each the MMAs of one of the
//               two tile sets (the tiles whose accumulators one pair of
//               epilogue groups reads);
//   warps 2-3   otherwise idle (they complete the control warpgroup);
//   warps 4-    epilogue, EG groups of four warps (four at B <= 8, two at
//               B = 16): each warp owns the 32 TMEM lanes = 32 domains of its
//               quarter.  At B = 16 the groups take turns on the tiles; at
//               B <= 8 two groups share each tile, one half of its ranges
//               each, and the two pairs take turns.  The groups merge their
//               per-range bests per item.  A warp hands the accumulator back
//               to the MMA as soon as its part of the tile is in registers.
//
// Screening.  The float score E' / (8 q n) = p^2 u - p y, with
// u = V / (8 q n) and y = C / n = cmax - (sum r' / n) sum Ds', screens the
// pairs: a pair is skipped only when its best float score exceeds the
// range's threshold -- the exact score of a candidate already kept plus the
// rounding bound `delta`; every other pair is scored exactly in int64 and
// compared with the tie-break key (pos * 8 + k) * |S| + s_idx.  The result
// therefore equals the exhaustive exact argmin.  A threshold only has to
// bound the exact score of some candidate of the same range that stays in
// the reduction, so the warp's 32 domains share theirs (warp shuffles) and
// every CTA that scores the range shares it through a per-range word in
// global memory (atomicMin on an order-preserving image of the float).
//
// Rounding bound.  cmax is exact, w = sum r' / n is exact (n is a power of
// two) and the FMAs round once each, so y carries at most 2^-24 |y| and a
// score F - p y (F = p^2 u rounded from double) at most
//     2^-23 (F + p |y|) <= 2^-23 (p^2 umax + p Y),   Y = 1024 sum |r'|,
// because |corr| <= 512 sum |r'| and |w sum Ds'| <= 512 |sum r'|; umax is the
// largest u of the level's kept domains.  The kernel uses 4x that bound
// (`delta`), per range.
//
// Grid S (s = p / q, p = 0..q).  E'(p) = V (p - p*)^2 + const with the real
// minimiser p* = 4 q C / V, so the best grid point is the nearest integer to
// p* clamped to [0, q].  The float path takes p^ = clamp(rint(y 4qn / V)); p^
// can miss the exact choice by one only when p* lies within about 2^-22 q of
// a half-integer, where the two neighbours' scores differ by at most
// 2^-21 q umax -- inside the level-wide margin used on the grid (2^-20 times
// the worst-case score bound) -- and the exact pass scores p^ - 1, p^, p^ + 1.
#include <math.h>

#include <type_traits>

#include "level.cuh"
#include "tc_ptx.cuh"

namespace fic {

constexpr int kCtlWarps = 4;  // producer, MMA issuer and two idle warps: one warpgroup

// Epilogue warpgroups and registers.  The block launches with LREGS per
// thread (what 65536 registers give its threads); the control warpgroup
// hands most of its share to the epilogue warpgroups (setmaxnreg).  The host
// checks the launch count before the first launch: an increment that the
// block's total cannot pay for would never complete.
template <int EG>
struct TcWarps {
  static constexpr int EPI_WARPS = 4 * EG;  // EG warps per TMEM lane quarter
  static constexpr int THREADS = 32 * (kCtlWarps + EPI_WARPS);
  static constexpr int LREGS = EG == 2 ? 168 : EG == 3 ? 128 : 96;
  static constexpr int CREGS = EG == 2 ? 40 : 32;
  static constexpr int EREGS = EG == 2 ? 232 : EG == 3 ? 160 : 112;
  static_assert(32 * (kCtlWarps * CREGS + EPI_WARPS * EREGS) <= THREADS * LREGS,
                "register split exceeds the launch budget");
};

// G: epilogue warp groups per tile at B <= 8 (2: a warp scores 8 of the
// tile's 16 ranges per visit; 1: all 16, in two 64-column halves), a shape
// the autotuner chooses per level; B = 16 always takes whole tiles.
template <int B, int G = 2>
struct TcCfg {
  static constexpr int EG = B == 16 ? 2 : 4;          // epilogue warp groups
  using Wp = TcWarps<EG>;
  static constexpr int n = B * B;
  static constexpr int Kp = tc_kp(B);                 // K padded to the MMA K step
  static constexpr int NKC = n > 128 ? n / 128 : 1;   // K-half stages per tile
  static constexpr int KS = Kp / NKC;                 // K per pipeline stage
  static constexpr int KSTEPS = KS / 16;              // MMAs per stage
  // B <= 8: one stage = one whole tile block (operand + scoring records),
  // one bulk copy and one barrier per tile; B = 16: one stage per K half,
  // the scoring records in a ring of their own
  static constexpr bool UNI = B <= 8;
  static constexpr int NA = UNI ? 2 : 1;              // range-tile buffers
  static constexpr int A_BYTES = kTileRows * Kp * 2;
  static constexpr int OP_BYTES = kTileDoms * KS * 2;
  static constexpr int DT_BYTES = 4 * kTileDoms * 4;  // float planes {sum Ds', F0, F1, 0}
  static constexpr int DR_BYTES = kTileDoms * 16;     // DomRec per domain
  static constexpr int D_BYTES = DT_BYTES + DR_BYTES;
  static constexpr int ST_BYTES = UNI ? OP_BYTES + D_BYTES : OP_BYTES;
  static_assert(!UNI || ST_BYTES == tc_tile_bytes(B), "tile block layout");
  static constexpr int NST = B == 16 ? 4 : B == 8 ? 8 : 16;  // stages
  static constexpr int NACC = 4;                              // TMEM accumulators
  static constexpr int ND = UNI ? 0 : 4;                      // scoring-record stages (B = 16)
  static constexpr int TCOLS = 512;
  static constexpr int CW = 32;                       // tile columns per epilogue chunk
  static constexpr int RPC = CW / 8;                  // ranges per chunk
  static constexpr int NCH = kTileRows / CW;
  // B <= 8: two groups score each tile, a warp two of its four chunks; it
  // loads both, hands the accumulator back, then scores them.  B = 16: one
  // group per tile.
  static constexpr int GPT = UNI ? G : 1;             // warp groups per tile
  static constexpr int TSETS = EG / GPT;              // tiles scored at once
  // MMA issuers: at B <= 8 two (warps 1 and 2), each the tiles of every
  // other tile set, so that the refill of one set's accumulators never
  // waits behind the other set's
  static constexpr int NMMA = UNI ? (TSETS < 2 ? TSETS : 2) : 1;
  static_assert(GPT == 1 || (NCH == 2 * GPT && NKC == 1), "two chunks per warp");
  static_assert(!UNI || ((NCH / GPT) % 2 == 0 && (G == 1 || G == 2)), "64-column halves");
  static constexpr int MRG_BYTES = Wp::EPI_WARPS * kTileRanges * 16;  // per-warp range bests
  static constexpr int SCR_BYTES = 3 * kTileRanges * 4;  // per range: w, delta, threshold
  // B <= 4 (the explicit and grid S sets): the exact pass is deferred to a
  // per-warp queue of candidates (see the epilogue); B = 8 and the exact-s
  // mode score candidates in place
  static constexpr bool DEFER = B <= 4;
  static constexpr int QCAP = DEFER ? 64 : 0;
  static constexpr int Q_BYTES = Wp::EPI_WARPS * QCAP * 16;
  static constexpr int OFF_B = NA * A_BYTES;
  static constexpr int OFF_D = OFF_B + NST * ST_BYTES;
  static constexpr int OFF_MRG = OFF_D + ND * D_BYTES;
  static constexpr int OFF_SCR = OFF_MRG + MRG_BYTES;
  static constexpr int OFF_Q = OFF_SCR + SCR_BYTES;
  static constexpr int OFF_BAR = OFF_Q + Q_BYTES;
  static constexpr int NBAR = 2 * NST + 2 * NA + 2 * NACC + 2 * ND + 1;
  static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
  static constexpr int BYTES = OFF_MISC + 16;
  // one CTA per SM: the CTA owns all 512 TMEM columns
  static constexpr int SMEM = BYTES < 120 * 1024 ? 120 * 1024 : BYTES;
  static_assert(NACC * 128 <= TCOLS, "tensor memory");
  static_assert(BYTES + 128 <= 227 * 1024, "shared memory");
};

constexpr int MODE_M1 = 0, MODE_M2 = 1, MODE_GRID = 2, MODE_EXACT = 3;

// A candidate pair queued for exact scoring (B <= 8): the domain's slot in
// the level's kept pool, the pair's largest isometry correlation (an exact
// integer) and the range in the item (grid S: and the nearest grid point of
// the pair's float minimiser).
struct QCand {
  int64_t slot;  // kept-pool slot of the domain
  int32_t cmax;  // largest isometry correlation of the pair
  int32_t rk;    // range in the item (bits 0-7) | grid point << 12
};
static_assert(sizeof(QCand) == 16, "queue entry");

// The 8 isometry correlations of a (domain, range) pair, recomputed by one
// thread from the operands in global memory: the domain's row Ds - 512 in its
// 128-domain tile block and the range's 8 rows T_k^-1 R - 128, both f16 in
// the MMA's core-matrix layouts.  Every product and partial sum is an
// integer below 2^22 (n <= 64), so the float sums are exact: the values the
// MMA accumulated.
template <int B, int KP, int TILE_BYTES>
__device__ inline void pair_corr_global(const uint16_t* __restrict__ bpack,
                                        const uint16_t* __restrict__ apack, int64_t slot,
                                        int64_t range, float (&v)[8]) {
  constexpr int n = B * B;
  const uint16_t* dt =
      (const uint16_t*)((const uint8_t*)bpack + (slot >> 7) * (int64_t)TILE_BYTES);
  const int d = (int)(slot & 127);
  const uint16_t* drow = dt + (d >> 3) * (KP / 8) * 64 + (d & 7) * 8;
  const uint16_t* rrow = apack + range * 8 * KP;
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = 0.f;
#pragma unroll 1
  for (int c = 0; c < (n + 7) / 8; ++c) {
    const uint4 dq = __ldg((const uint4*)(drow + c * 64));
    const uint32_t dw[4] = {dq.x, dq.y, dq.z, dq.w};
    float df[8];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const float2 f = __half22float2(*(const __half2*)&dw[h]);
      df[2 * h] = f.x;
      df[2 * h + 1] = f.y;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint4 rq = __ldg((const uint4*)(rrow + (c * 8 + k) * 8));
      const uint32_t rw[4] = {rq.x, rq.y, rq.z, rq.w};
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const float2 f = __half22float2(*(const __half2*)&rw[h]);
        v[k] = fmaf(df[2 * h], f.x, v[k]);
        v[k] = fmaf(df[2 * h + 1], f.y, v[k]);
      }
    }
  }
}

struct ItemGeo {
  int im, nr, t0, t1, nkept;
  int rot;       // the item's tiles run from t0 + rot, wrapping at t1
  int64_t r0, slot0;
  int64_t pidx;  // index of the item's partials: (range tile) * chunks + chunk
};

// Items run chunk-major within an image: every range tile's first domain
// chunk before any second chunk, so the later chunks of a range tile start
// from the thresholds its earlier chunks published.
__device__ inline ItemGeo item_geo(const MatchArgs& a, int64_t it, int CH) {
  ItemGeo g;
  g.im = find_segment(a.item_off, a.n_images, it);
  const int nc = a.chunks[g.im];
  const int64_t local = it - a.item_off[g.im];
  const int64_t nmt = ceil_div64(a.act_cnt[g.im], kTileRanges);
  const int c = (int)(local / nmt);
  const int64_t mt = local % nmt;
  g.pidx = a.item_off[g.im] + mt * nc + c;
  g.r0 = a.act_off[g.im] + mt * kTileRanges;
  g.nr = (int)min((int64_t)kTileRanges, a.act_cnt[g.im] - mt * kTileRanges);
  g.nkept = a.sel[g.im].nkept;
  const int nt = ceil_div(g.nkept, kTileDoms);
  g.t0 = c * CH;
  g.t1 = min(nt, g.t0 + CH);
  // concurrent items of one chunk start at different tiles, so the CTAs
  // do not all fetch the same tile block from L2 at the same moment
  g.rot = g.t1 > g.t0 ? (int)((mt * 53) % (g.t1 - g.t0)) : 0;
  g.slot0 = a.pool_off[g.im];
  return g;
}

// Tile k (0-based) of an item in its rotated order.
__device__ inline int item_tile(const ItemGeo& g, int k) {
  const int t = g.t0 + g.rot + k;
  return t < g.t1 ? t : t - (g.t1 - g.t0);
}

// Skip a candidate whose float score is above this: an upper bound of the
// exact score E' / (8 q n) plus the margin, in directed-rounding FP32
// (inv_up / inv_dn: 1 / (8 q n) rounded up / down).
__device__ inline float thr_of(int64_t e, float inv_up, float inv_dn, float delta) {
  const float ef = __ll2float_ru(e);
  return __fadd_ru(__fmul_ru(ef, ef >= 0.f ? inv_up : inv_dn), delta);
}

// Exact-s mode.  A pair's y = C / n is the FMA y above, rounded once: |y -
// C / n| <= 2^-24 |y|.  Below the clamp point (4C < V: y < Yc = V / (4 n))
// G = y^2 n^2 / V, computed as (y y) F0 with F0 = n^2 / V rounded: relative
// error < 5 2^-24; at and above it G = n y / 2 - V / 16, as an FMA with
// b = V / 16 rounded: error < 2^-23 (n |y| / 2 + b + G); picking the wrong
// branch next to the clamp point costs (4C - V)^2 / (16 V), below 2^-46 V
// there; y <= 0 gives G = 0 exactly.  So U = g + 2^-18 (g + n |y| / 2 + b)
// bounds G from above (rounding of U included).  The screen's score is -U:
// a pair is skipped only when U stays below a lower bound of the exact G of
// a candidate already kept, i.e. when it can neither beat nor tie it.
constexpr float kExactErr = 0x1p-18f;

// Threshold of an exact-s candidate (C, V): -(a lower bound of its exact G).
__device__ inline float thr_exact(int64_t C, int64_t V) {
  double gd = 0.0;
  if (C > 0 && V > 0) {
    if (4 * C >= V)
      gd = (double)(8 * C - V) / 16.0;                 // exact (< 2^53)
    else
      gd = ((double)C * (double)C) / (double)V;      // within 2 ulps
  }
  return -__double2float_rd(gd * (1.0 - 0x1p-50));
}

template <int B, int MODE, int G>
__global__ void __launch_bounds__(TcCfg<B, G>::Wp::THREADS, 1) k_match_tc(MatchArgs a) {
  using Cf = TcCfg<B, G>;
  constexpr int n = B * B;
  constexpr int LOGN = B == 16 ? 8 : B == 8 ? 6 : B == 4 ? 4 : 2;
  grid_dep_sync();
  constexpr int CW = Cf::CW;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  uint8_t* sA = smem;
  uint8_t* sB = smem + Cf::OFF_B;
  uint64_t* bars = (uint64_t*)(smem + Cf::OFF_BAR);
  uint64_t* full_b = bars;
  uint64_t* empty_b = bars + Cf::NST;
  uint64_t* a_full = bars + 2 * Cf::NST;
  uint64_t* a_empty = a_full + Cf::NA;
  uint64_t* acc_full = a_empty + Cf::NA;
  uint64_t* acc_empty = acc_full + Cf::NACC;
  uint64_t* d_full = acc_empty + Cf::NACC;
  uint64_t* d_empty = d_full + Cf::ND;
  uint64_t* done_bar = d_empty + Cf::ND;
  uint32_t* tmem_slot = (uint32_t*)(smem + Cf::OFF_MISC);
  volatile int* abort_flag = (volatile int*)(smem + Cf::OFF_MISC + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < Cf::NST; ++i) {
      ptx::mbar_init(&full_b[i], 1);
      // a whole-tile stage is released by the four epilogue warps that
      // score it, a K-half stage by the MMA's commit
      ptx::mbar_init(&empty_b[i], Cf::UNI ? 4 * Cf::GPT : 1);
    }
    for (int i = 0; i < Cf::NA; ++i) {
      ptx::mbar_init(&a_full[i], 1);
      ptx::mbar_init(&a_empty[i], Cf::NMMA);  // a commit from every MMA issuer
    }
    for (int i = 0; i < Cf::NACC; ++i) {
      ptx::mbar_init(&acc_full[i], 1);
      ptx::mbar_init(&acc_empty[i], 4 * Cf::GPT);  // the warps that read it
    }
    for (int i = 0; i < Cf::ND; ++i) {
      ptx::mbar_init(&d_full[i], 1);
      ptx::mbar_init(&d_empty[i], 4);
    }
    ptx::mbar_init(done_bar, Cf::NMMA);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, Cf::TCOLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t items = a.meta->overflow ? 0 : a.meta->items;
  const int CH = a.meta->chunk_tiles;
  auto fail = [&]() {
    *abort_flag = 1;
    atomicOr(a.status, kStatusTimeout);
  };

  if (warp < kCtlWarps) {
  ptx::setmaxnreg_dec<Cf::Wp::CREGS>();
  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t si = 0, ai = 0, di = 0;  // stage, range-tile and record fills
      bool ok = true;
      for (int64_t it = blockIdx.x; ok && it < items; it += gridDim.x) {
        const ItemGeo g = item_geo(a, it, CH);
        const int ab = ai % Cf::NA;
        if (!ptx::mbar_spin_abort(&a_empty[ab], ((ai / Cf::NA) & 1) ^ 1, abort_flag)) {
          ok = false;
          break;
        }
        ptx::mbar_expect_tx(&a_full[ab], Cf::A_BYTES);
        ptx::bulk_g2s(sA + ab * Cf::A_BYTES, a.apack + g.r0 * 8 * Cf::Kp, Cf::A_BYTES,
                      &a_full[ab]);
        ++ai;
        for (int kt = 0; ok && kt < g.t1 - g.t0; ++kt) {
          const int t = item_tile(g, kt);
          const int64_t tile_g = g.slot0 / kTileDoms + t;
          if constexpr (!Cf::UNI) {
            // the tile's scoring records: a ring of their own, ND tiles ahead
            const int db = di % Cf::ND;
            if (!ptx::mbar_spin_abort(&d_empty[db], ((di / Cf::ND) & 1) ^ 1, abort_flag)) {
              ok = false;
              break;
            }
            uint8_t* dst = smem + Cf::OFF_D + db * Cf::D_BYTES;
            ptx::mbar_expect_tx(&d_full[db], Cf::D_BYTES);
            ptx::bulk_g2s(dst, a.domf + tile_g * (4 * kTileDoms), Cf::DT_BYTES, &d_full[db]);
            ptx::bulk_g2s(dst + Cf::DT_BYTES, a.dom + tile_g * kTileDoms, Cf::DR_BYTES,
                          &d_full[db]);
            ++di;
          }
          for (int kc = 0; kc < Cf::NKC; ++kc) {
            const int st = si % Cf::NST;
            if (!ptx::mbar_spin_abort(&empty_b[st], ((si / Cf::NST) & 1) ^ 1, abort_flag)) {
              ok = false;
              break;
            }
            if (a.inject == kInjectDropTileCopy && blockIdx.x == 0 && si == 0) {
              ++si;  // test hook: this stage is never filled (see MatchArgs::inject)
              continue;
            }
            ptx::mbar_expect_tx(&full_b[st], Cf::ST_BYTES);
            ptx::bulk_g2s(sB + st * Cf::ST_BYTES,
                          (const uint8_t*)a.bpack + (tile_g * Cf::NKC + kc) * Cf::ST_BYTES,
                          Cf::ST_BYTES, &full_b[st]);
            ++si;
          }
        }
      }
      if (!ok) fail();
      // drain: every copy this thread issued has landed before the CTA exits
      // (the last fill of each buffer, fill f waits for parity (f / N) & 1)
      for (uint32_t i = 0; i < Cf::NST; ++i)
        if (si > i) ptx::mbar_spin(&full_b[i], ((i + (si - 1 - i) / Cf::NST * Cf::NST) / Cf::NST) & 1);
      for (uint32_t i = 0; i < Cf::NA; ++i)
        if (ai > i) ptx::mbar_spin(&a_full[i], ((i + (ai - 1 - i) / Cf::NA * Cf::NA) / Cf::NA) & 1);
      if constexpr (Cf::ND > 0)
        for (uint32_t i = 0; i < Cf::ND; ++i)
          if (di > i) ptx::mbar_spin(&d_full[i], ((i + (di - 1 - i) / Cf::ND * Cf::ND) / Cf::ND) & 1);
    }
  } else if (warp >= 1 && warp <= Cf::NMMA) {
    // ------------------------------------------------------------ MMA issuers
    // issuer `set` takes the tiles ti = set mod NMMA (all of them at B = 16)
    if (lane == 0) {
      constexpr uint32_t IDESC = ptx::idesc_f16_f32(kTileDoms, kTileRows);
      constexpr int NMMA = Cf::NMMA;
      const int set = warp - 1;
      uint32_t ai = 0, tib = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; ok && it < items; it += gridDim.x) {
        const ItemGeo g = item_geo(a, it, CH);
        const int rb = ai % Cf::NA;
        if (!ptx::mbar_spin_abort(&a_full[rb], (ai / Cf::NA) & 1, abort_flag)) {
          ok = false;
          break;
        }
        const uint8_t* sR = sA + rb * Cf::A_BYTES;
        const int len = g.t1 - g.t0;
        for (int kt = (int)((set + NMMA - tib % NMMA) % NMMA); ok && kt < len; kt += NMMA) {
          const uint32_t ti = tib + kt;
          uint32_t si = ti * Cf::NKC;  // stage fills run in tile order, NKC per tile
          const int ab = ti % Cf::NACC;
          const uint32_t pa = ((ti / Cf::NACC) & 1) ^ 1;
          // one stage per tile: the accumulator and the stage are usually
          // both ready, and one round trip tests the two
          const bool ready = Cf::NKC == 1 && ptx::mbar_test_wait2(&acc_empty[ab], pa, &full_b[si % Cf::NST],
                                                                 (si / Cf::NST) & 1);
          if (!ready && !ptx::mbar_spin_abort(&acc_empty[ab], pa, abort_flag)) {
            ok = false;
            break;
          }
          for (int kc = 0; kc < Cf::NKC; ++kc) {
            const int st = si % Cf::NST;
            if (!ready && !ptx::mbar_spin_abort(&full_b[st], (si / Cf::NST) & 1, abort_flag)) {
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            // one accumulator per tile over the whole K (both K halves at
            // B = 16): every partial sum is an integer of magnitude at most
            // n * 128 * 512 <= 2^24, exact in f32
            const uint32_t d = tmem + (uint32_t)(ab * kTileDoms);
#pragma unroll
            for (int s = 0; s < Cf::KSTEPS; ++s) {
              const int kk = (kc * Cf::KSTEPS + s) * 2;  // core-matrix column of the range tile
              // A = the domain stage (one TMEM lane per domain), B = the
              // resident range tile (columns = range x isometry)
              const uint64_t rd = ptx::smem_desc(sR + kk * 128, 128, 16 * Cf::Kp);
              const uint64_t dd = ptx::smem_desc(sB + st * Cf::ST_BYTES + s * 256, 128, 16 * Cf::KS);
              ptx::mma_f16(d, dd, rd, IDESC, (kc > 0 || s > 0) ? 1u : 0u);
            }
            if constexpr (!Cf::UNI) ptx::mma_commit(&empty_b[st]);
            ++si;
          }
          if (!ok) break;
          ptx::mma_commit(&acc_full[ab]);
        }
        tib += len;
        ptx::mma_commit(&a_empty[rb]);
        ++ai;
      }
      if (!ok) fail();
      ptx::mma_commit(done_bar);
      if (!ptx::mbar_spin(done_bar, 0)) atomicOr(a.status, kStatusTimeout);
    }
  }
  } else {
    ptx::setmaxnreg_inc<Cf::Wp::EREGS>();
    // ------------------------------------------------------------ epilogue
    // Warps 4..: quarter qd = warp % 4 of the TMEM lanes = the tile's domains
    // qd * 32 .. qd * 32 + 31; group h belongs to tile set ts = h / GPT, which
    // takes the tiles ti = ts mod TSETS, and scores the chunks of part
    // cp = h mod GPT of those tiles' columns.  Each
    // warp keeps its best candidate per range of the item in shared memory;
    // the warps' bests merge at item end.  Per item the first epilogue warp
    // stages each range's w, rounding bound and starting threshold (the best
    // any CTA has published) in shared memory; the warps share their
    // threshold improvements there (a plain store of a smaller value: a lost
    // race only leaves a looser, still valid, threshold) and publish them to
    // the other CTAs with atomicMin.  The warps read w and the thresholds
    // from shared memory for every chunk.
    constexpr int RPC = Cf::RPC;
    constexpr int REFRESH = 4;               // tiles between reads of the global thresholds
    const int ew = warp - kCtlWarps;
    const int h = ew >> 2;
    const int ts = h / Cf::GPT, cp = h % Cf::GPT;
    const int qd = warp & 3;
    const int dl = qd * 32 + lane;           // tile row = domain slot in the tile
    const uint32_t epi_threads = 32 * Cf::Wp::EPI_WARPS;
    Cand* wbest = (Cand*)(smem + Cf::OFF_MRG);  // [EPI_WARPS][16]
    Cand* mybest = wbest + ew * kTileRanges;
    QCand* myq = (QCand*)(smem + Cf::OFF_Q) + ew * Cf::QCAP;  // B <= 8
    float* sW = (float*)(smem + Cf::OFF_SCR);
    float* sDelta = sW + kTileRanges;
    float* sThr = sW + 2 * kTileRanges;
    const int m_s = a.S.m;
    const int qv = a.S.q;
    const float inv_up = __double2float_ru(1.0 / (8.0 * qv * n));
    const float inv_dn = __double2float_rd(1.0 / (8.0 * qv * n));
    const float p0f = (float)a.S.p[0], p1f = (float)a.S.p[1];
    const float qf = (float)qv;
    const int rl = lane & (kTileRanges - 1);
    uint32_t ti = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
      const ItemGeo g = item_geo(a, it, CH);
      const bool rv = rl < g.nr;
      if (ew == 0 && lane < kTileRanges) {
        float wv = 0.f, dv = 0.f, tv = -INFINITY;
        if (rv) {
          const RangeMom m = a.mom[g.r0 + rl];
          wv = (float)m.srp * (1.0f / n);
          // rounding bound of this range's float scores (score units): 4x
          // the bound derived above; the grid uses the level-wide margin
          if (MODE == MODE_EXACT) {
            dv = 0.f;  // per-pair bounds in the score itself
          } else if (MODE == MODE_GRID) {
            dv = a.delta;
          } else {
            const double pmx = (double)(MODE == MODE_M2 ? max(a.S.p[0], a.S.p[1]) : a.S.p[0]);
            dv = __double2float_ru(
                ldexp(pmx * pmx * (double)*a.umax + pmx * 1024.0 * (double)m.sabs, -21));
          }
          tv = ord_to_thr(__ldcg(a.gthr + g.r0 + rl));
        }
        sW[lane] = wv;
        sDelta[lane] = dv;
        sThr[lane] = tv;
      }
      // (the first epilogue warp has merged the previous item's bests and
      // staged this item's ranges when every warp passes this barrier)
      ptx::named_bar_sync(1, epi_threads);
      if (lane < kTileRanges) mybest[lane] = Cand{INT64_MAX, INT64_MAX};
      __syncwarp();
      uint32_t gpre = rv ? __ldcg(a.gthr + g.r0 + rl) : kThrInit;
      int qn = 0;  // candidates in this warp's queue (warp-uniform)
      int nmine = 0;

      // Exact scoring of the queued candidates (warp-collective): a lane per
      // candidate computes its best exact E' and tie-break key over S (the
      // arithmetic of pair_exact), then per range the warp's best merges
      // into this warp's best of the range and tightens the range's
      // threshold (as an exact pass does).
      auto flush = [&]() {
        if constexpr (Cf::DEFER && MODE != MODE_EXACT) {
          const int m_s2 = a.S.m, qv2 = a.S.q;
          for (int b0 = 0; b0 < qn; b0 += 32) {
            const bool have = b0 + lane < qn;
            int64_t be = INT64_MAX, bk = INT64_MAX;
            int r = 0;
            if (have) {
              const QCand c = myq[b0 + lane];
              r = c.rk & 0xff;
              // the isometry of the largest correlation (lowest k on ties),
              // from the pair's correlations recomputed exactly
              float cv[8];
              pair_corr_global<B, Cf::Kp, Cf::ST_BYTES>(a.bpack, a.apack, c.slot, g.r0 + r, cv);
              const float cmf = (float)c.cmax;
              int kmax = 7;
#pragma unroll
              for (int k = 6; k >= 0; --k)
                if (cv[k] == cmf) kmax = k;
              const DomRec dr = a.dom[c.slot];
              const int64_t srp_r = (int64_t)(int)(sW[r] * (float)n);
              const int64_t C = ((int64_t)c.cmax << LOGN) - srp_r * (int64_t)dr.sdp;
              auto cand = [&](int64_t p, int si) {
                const int64_t e = p * p * dr.v - 8 * p * qv2 * C;
                const int64_t key = ((int64_t)dr.pos * 8 + (p > 0 ? kmax : 0)) * m_s2 + si;
                if (e < be || (e == be && key < bk)) {
                  be = e;
                  bk = key;
                }
              };
              if constexpr (MODE == MODE_GRID) {
                const int pi = c.rk >> 12;
                for (int pp = max(pi - 1, 0); pp <= min(pi + 1, qv2); ++pp) cand(pp, pp);
              } else {
                cand(a.S.p[0], 0);
                if constexpr (MODE == MODE_M2) cand(a.S.p[1], 1);
              }
            }
            for (uint32_t rm = __reduce_or_sync(0xffffffffu, have ? 1u << r : 0u); rm;
                 rm &= rm - 1) {
              const int rr = __ffs(rm) - 1;
              int64_t e2 = have && r == rr ? be : INT64_MAX, k2 = have && r == rr ? bk : INT64_MAX;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) {
                const int64_t eo = __shfl_xor_sync(0xffffffffu, e2, o);
                const int64_t ko = __shfl_xor_sync(0xffffffffu, k2, o);
                if (eo < e2 || (eo == e2 && ko < k2)) {
                  e2 = eo;
                  k2 = ko;
                }
              }
              const Cand cur = mybest[rr];
              if (e2 < cur.score || (e2 == cur.score && k2 < cur.key)) {
                const float to = thr_of(e2, inv_up, inv_dn, sDelta[rr]);
                __syncwarp();
                if (lane == 0) {
                  mybest[rr] = Cand{e2, k2};
                  if (to < sThr[rr]) {
                    sThr[rr] = to;
                    atomicMin(a.gthr + g.r0 + rr, thr_to_ord(to));
                  }
                }
                __syncwarp();
              }
            }
          }
          qn = 0;
        }
      };

      // this group's tiles of the item: ti = tile counter of the CTA
      const uint32_t tib = ti;
      const int len = g.t1 - g.t0;
      ti += len;
      constexpr int TSETS = Cf::TSETS;
      for (int kt = (int)((ts + TSETS - tib % TSETS) % TSETS); kt < len; kt += TSETS) {
        const uint32_t ti = tib + kt;
        const int t = item_tile(g, kt);
        const int ab = ti % Cf::NACC;
        // the tile's scoring records: in its whole-tile stage (B <= 8; one
        // stage per tile, so stage fill = tile), or in the record ring
        constexpr int NREC = Cf::UNI ? Cf::NST : Cf::ND;
        const int db = ti % NREC;
        uint64_t* rec_full = Cf::UNI ? &full_b[db] : &d_full[db];
        uint64_t* rec_empty = Cf::UNI ? &empty_b[db] : &d_empty[db];
        const uint32_t rec_par = (ti / NREC) & 1;
        const bool got = ok && ptx::mbar_wait(&acc_full[ab], (ti / Cf::NACC) & 1) &&
                         ptx::mbar_wait(rec_full, rec_par);
        // the TMEM loads below are warp-collective: the lanes agree on the outcome
        const bool all = __all_sync(0xffffffffu, got);
        if (ok && !all && lane == 0) fail();
        ok = all;
        ptx::tc_fence_after();
        // thresholds of the other CTAs: loaded REFRESH tiles ahead, passed on
        // through shared memory
        if (++nmine % REFRESH == 0) {
          if (lane < kTileRanges && rv) {
            const float tg = ord_to_thr(gpre);
            if (tg < sThr[lane]) sThr[lane] = tg;
          }
          gpre = rv ? __ldcg(a.gthr + g.r0 + rl) : kThrInit;
        }
        const uint8_t* sD = Cf::UNI ? sB + db * Cf::ST_BYTES + Cf::OP_BYTES
                                    : smem + Cf::OFF_D + db * Cf::D_BYTES;
        const float* sX = (const float*)sD;
        const DomRec* sDom = (const DomRec*)(sD + Cf::DT_BYTES);
        const int nv = min(kTileDoms, g.nkept - t * kTileDoms);
        const bool dvalid = dl < nv;
        // this lane's domain constants
        const float nX = -sX[dl];
        const float F0 = sX[kTileDoms + dl];
        const float F1 = sX[2 * kTileDoms + dl];
        const float F2 = MODE == MODE_EXACT ? sX[3 * kTileDoms + dl] : 0.f;
        const uint32_t tb = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(ab * kTileRows);

        // B = 16: one 32-column chunk (4 ranges x 8 isometries) and each
        // range's isometry maximum, from four reducing loads
        auto load = [&](int ch, float (&r)[32], float (&m)[4]) {
          ptx::tmem_ldred32(tb + ch * 32, r, m);
        };

        // exact-s mode: -(upper bound of G), see kExactErr (F0 = n^2 / V,
        // F1 = V / (4 n), F2 = V / 16)
        auto exact_sc = [&](float y) -> float {
          constexpr float hn = 0.5f * n;
          const float gy = y > 0.f ? (y >= F1 ? fmaf(hn, y, -F2) : (y * y) * F0) : 0.f;
          return -fmaf(kExactErr, gy + fmaf(hn, fabsf(y), F2), gy);
        };

        // float score of a pair from its largest correlation and the range's w
        auto score = [&](float cmax, float wr) -> float {
          const float y = fmaf(nX, wr, cmax);
          if constexpr (MODE == MODE_EXACT) {
            return exact_sc(y);
          } else if constexpr (MODE == MODE_GRID) {
            float p = rintf(y * F1);
            p = fminf(fmaxf(p, 0.f), qf);
            return p * fmaf(p, F0, -y);
          } else if constexpr (MODE == MODE_M2) {
            return fminf(fmaf(-p0f, y, F0), fmaf(-p1f, y, F1));
          } else {
            return fmaf(-p0f, y, F0);
          }
        };

        // float screen of one (domain, range) pair from the maximum of the
        // range's 8 isometry correlations: the best score over S against the
        // range's threshold
        auto screen = [&](float cmax, float wr, float tr, float& sc) -> uint32_t {
          const float y = fmaf(nX, wr, cmax);
          if constexpr (MODE == MODE_EXACT) {
            sc = exact_sc(y);
          } else if constexpr (MODE == MODE_GRID) {
            float p = rintf(y * F1);
            p = fminf(fmaxf(p, 0.f), qf);
            sc = p * fmaf(p, F0, -y);
          } else if constexpr (MODE == MODE_M2) {
            sc = fminf(fmaf(-p0f, y, F0), fmaf(-p1f, y, F1));
          } else {
            sc = fmaf(-p0f, y, F0);
          }
          return sc <= tr ? 1u : 0u;
        };

        // exact score of this lane's pair: the isometry with the largest
        // correlation (k = 0 where p = 0), every s that can win
        auto pair_exact = [&](const float* v, float cmax, float wr, const DomRec& dr,
                              int64_t& be, int64_t& bv, int64_t& bk) {
          int kmax = 7;
#pragma unroll
          for (int k = 6; k >= 0; --k)
            if (v[k] == cmax) kmax = k;
          const int64_t srp_r = (int64_t)(int)(wr * (float)n);
          const int64_t C = ((int64_t)(int)cmax << LOGN) - srp_r * (int64_t)dr.sdp;
          if constexpr (MODE == MODE_EXACT) {
            // the isometry of the largest correlation (k = 0 when G = 0)
            const int64_t key = (int64_t)dr.pos * 8 + (C > 0 && dr.v > 0 ? kmax : 0);
            if (exact_better(C, dr.v, key, be, bv, bk)) {
              be = C;
              bv = dr.v;
              bk = key;
            }
            return;
          }
          auto cand = [&](int64_t p, int si) {
            const int64_t e = p * p * dr.v - 8 * p * qv * C;
            const int64_t key = ((int64_t)dr.pos * 8 + (p > 0 ? kmax : 0)) * m_s + si;
            if (e < be || (e == be && key < bk)) {
              be = e;
              bk = key;
            }
          };
          if constexpr (MODE == MODE_GRID) {
            const float y = fmaf(nX, wr, cmax);
            const int pi = (int)fminf(fmaxf(rintf(y * F1), 0.f), qf);
            for (int pp = max(pi - 1, 0); pp <= min(pi + 1, qv); ++pp) cand(pp, pp);
          } else {
            cand(a.S.p[0], 0);
            if constexpr (MODE == MODE_M2) cand(a.S.p[1], 1);
          }
        };

        // the warp's best candidate (every lane ends with it): from the one
        // lane that scored, or a butterfly over all of them
        auto warp_best = [&](int64_t& be, int64_t& bv, int64_t& bk, unsigned bal) {
          if (__popc(bal) == 1) {
            const int src = __ffs(bal) - 1;
            be = __shfl_sync(0xffffffffu, be, src);
            bk = __shfl_sync(0xffffffffu, bk, src);
            if constexpr (MODE == MODE_EXACT) bv = __shfl_sync(0xffffffffu, bv, src);
          } else {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              const int64_t e2 = __shfl_xor_sync(0xffffffffu, be, o);
              const int64_t k2 = __shfl_xor_sync(0xffffffffu, bk, o);
              if constexpr (MODE == MODE_EXACT) {
                const int64_t v2 = __shfl_xor_sync(0xffffffffu, bv, o);
                if (exact_better(e2, v2, k2, be, bv, bk)) {
                  be = e2;
                  bv = v2;
                  bk = k2;
                }
              } else if (e2 < be || (e2 == be && k2 < bk)) {
                be = e2;
                bk = k2;
              }
            }
          }
        };

        // this warp's best of range r and the shared thresholds, from the
        // warp's best candidate (held by every lane)
        auto resolve = [&](int r, int64_t be, int64_t bv, int64_t bk) {
          const Cand cur = mybest[r];
          bool better;
          if constexpr (MODE == MODE_EXACT) {
            const int64_t vc = cur.key == INT64_MAX ? 0 : pos_v(a.pm, g.im, cur.key >> 3, n);
            better = exact_better(be, bv, bk, cur.score, vc, cur.key);
          } else {
            better = be < cur.score || (be == cur.score && bk < cur.key);
          }
          if (better) {
            const float to = MODE == MODE_EXACT ? thr_exact(be, bv)
                                                : thr_of(be, inv_up, inv_dn, sDelta[r]);
            __syncwarp();
            if (lane == 0) {
              mybest[r] = Cand{be, bk};
              if (to < sThr[r]) {
                sThr[r] = to;
                atomicMin(a.gthr + g.r0 + r, thr_to_ord(to));
              }
            }
            __syncwarp();
          }
        };

        // one chunk of CW columns = RPC ranges: the float screen (hot), and
        // for the rare chunk where some lane passes it, the exact pass on a
        // local copy in a rolled loop, which keeps the kernel's code small
        //
        // Of the flagged lanes only those whose float score lies within two
        // margins of the warp's smallest can hold the exact winner (each
        // score is within a quarter margin of its exact value, and the
        // smallest one's pair is scored exactly); usually that is one lane,
        // which scores its pair and broadcasts it.
        auto slow = [&](const float* c, const float* cm, const float* scs, const float* wr, int ch,
                        uint32_t fl) {
          float cl[CW], cml[RPC], sl[RPC], wl[RPC];
#pragma unroll
          for (int j = 0; j < CW; ++j) cl[j] = c[j];
#pragma unroll
          for (int j = 0; j < RPC; ++j) cml[j] = cm[j], sl[j] = scs[j], wl[j] = wr[j];
#pragma unroll 1
          for (int j = 0; j < RPC; ++j) {
            const bool mine = (fl >> j) & 1u;
            if (!__any_sync(0xffffffffu, mine)) continue;
            const int r = ch * RPC + j;
            bool need = mine;  // exact s: every flagged lane (no shared margin)
            if constexpr (MODE != MODE_EXACT) {
              float mn = mine ? sl[j] : INFINITY;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
              const float lim = __fadd_ru(mn, 2.0f * sDelta[r]);
              need = mine && sl[j] <= lim;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, need);
            int64_t be = INT64_MAX, bv = 0, bk = INT64_MAX;
            if (need) pair_exact(cl + 8 * j, cml[j], wl[j], sDom[dl], be, bv, bk);
            warp_best(be, bv, bk, bal);
            resolve(r, be, bv, bk);
          }
        };
        auto chunk = [&](int ch, const float* c, const float* cm) {
          float wr[RPC], tr[RPC];
          if constexpr (RPC == 4) {
            const float4 wv4 = *(const float4*)(sW + 4 * ch);
            const float4 tv4 = *(const float4*)(sThr + 4 * ch);
            wr[0] = wv4.x, wr[1] = wv4.y, wr[2] = wv4.z, wr[3] = wv4.w;
            tr[0] = tv4.x, tr[1] = tv4.y, tr[2] = tv4.z, tr[3] = tv4.w;
          } else {
            const float2 wv2 = *(const float2*)(sW + 2 * ch);
            const float2 tv2 = *(const float2*)(sThr + 2 * ch);
            wr[0] = wv2.x, wr[1] = wv2.y;
            tr[0] = tv2.x, tr[1] = tv2.y;
          }
          float scs[RPC];
          uint32_t fl = 0;
#pragma unroll
          for (int j = 0; j < RPC; ++j) fl |= screen(cm[j], wr[j], tr[j], scs[j]) << j;
          if (!dvalid) fl = 0;
          if (__any_sync(0xffffffffu, fl != 0)) slow(c, cm, scs, wr, ch, fl);
        };

        if constexpr (Cf::UNI) {
          // this warp's chunks: 8 ranges per 64-column half, one or two
          // halves.  Each range's 8 correlations (its isometries) come out of
          // tensor memory already reduced to their maximum -- the reducing
          // load of sm_103a -- and the float screen keeps each range's
          // margin (score - threshold) in a register.
          constexpr int CPW = Cf::NCH / Cf::GPT;  // chunks per warp
          constexpr int NH = CPW / 2;             // 64-column halves
          const int c0 = CPW * cp;
          const DomRec* drp = sDom + dl;
          // the float screen of one half from its 8 maxima: margins dm and
          // their minimum m
          auto screen8 = [&](const float (&cm)[8], int rb0, float (&dm)[8], float& m) {
            const float4 wa = *(const float4*)(sW + rb0), wb = *(const float4*)(sW + rb0 + 4);
            const float4 ta = *(const float4*)(sThr + rb0), tq = *(const float4*)(sThr + rb0 + 4);
            const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
            const float tv[8] = {ta.x, ta.y, ta.z, ta.w, tq.x, tq.y, tq.z, tq.w};
            if constexpr (MODE == MODE_GRID || MODE == MODE_EXACT) {
#pragma unroll
              for (int j = 0; j < 8; j += 2) {
                const float sa = score(cm[j], wv[j]), sb = score(cm[j + 1], wv[j + 1]);
                dm[j] = sa - tv[j];
                dm[j + 1] = sb - tv[j + 1];
                m = ptx::fmin3(m, dm[j], dm[j + 1]);
              }
            } else {
              // two ranges per packed FMA: y = cmax - w sum Ds', the scores
              // F_t - p_t y and the margins (a float difference is <= 0
              // exactly when sc <= thr)
#pragma unroll
              for (int j = 0; j < 8; j += 2) {
                const float2 y2 = __ffma2_rn(make_float2(nX, nX), make_float2(wv[j], wv[j + 1]),
                                             make_float2(cm[j], cm[j + 1]));
                float2 s2 = __ffma2_rn(make_float2(-p0f, -p0f), y2, make_float2(F0, F0));
                if constexpr (MODE == MODE_M2) {
                  const float2 s1 = __ffma2_rn(make_float2(-p1f, -p1f), y2, make_float2(F1, F1));
                  s2 = make_float2(fminf(s2.x, s1.x), fminf(s2.y, s1.y));
                }
                const float2 d2 = __fadd2_rn(s2, make_float2(-tv[j], -tv[j + 1]));
                dm[j] = d2.x;
                dm[j + 1] = d2.y;
                m = ptx::fmin3(m, d2.x, d2.y);
              }
            }
          };
          if constexpr (MODE == MODE_EXACT || !Cf::DEFER) {
            // exact s, and B = 8 (where recomputing a queued pair's 8
            // correlations from the operands costs more than holding the
            // accumulator): the exact pass reads the flagged ranges'
            // correlations from tensor memory again, so the accumulator goes
            // back after the last half
#pragma unroll 1
            for (int h2 = 0; h2 < CPW; h2 += 2) {
              const int cb = c0 + h2;  // first chunk of the half
              const int rb0 = cb * RPC;
              float m = INFINITY;
              float dm[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) dm[j] = INFINITY;
              if (ok) {
                float cm[8];
                ptx::tmem_ldmax8x8_wait(tb + cb * 32, cm);
                screen8(cm, rb0, dm, m);
              }
              if (__any_sync(0xffffffffu, dvalid && m <= 0.f)) {
                const DomRec dr = *drp;
                uint32_t fl = 0;
#pragma unroll
                for (int j = 0; j < 8; ++j) fl |= (dvalid && dm[j] <= 0.f) ? 1u << j : 0u;
                uint32_t wm = __reduce_or_sync(0xffffffffu, fl);
#pragma unroll 1
                for (; wm; wm &= wm - 1) {
                  const int j = __ffs(wm) - 1;
                  const int r = rb0 + j;
                  float v[8];
                  ptx::tmem_ld8_wait(tb + cb * 32 + 8 * j, v);
                  const float cmj = fmaxf(ptx::fmax3(v[0], v[1], v[2]),
                                          ptx::fmax3(v[3], v[4], ptx::fmax3(v[5], v[6], v[7])));
                  const float scj = score(cmj, sW[r]);
                  const bool mine = dvalid && scj <= sThr[r];
                  if (!__any_sync(0xffffffffu, mine)) continue;
                  bool need = mine;  // exact s: every flagged lane (no shared margin)
                  if constexpr (MODE != MODE_EXACT) {
                    float mn = mine ? scj : INFINITY;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                    const float lim = __fadd_ru(mn, 2.0f * sDelta[r]);
                    need = mine && scj <= lim;
                  }
                  const unsigned bal = __ballot_sync(0xffffffffu, need);
                  int64_t be = INT64_MAX, bv = 0, bk = INT64_MAX;
                  if (need) pair_exact(v, cmj, sW[r], dr, be, bv, bk);
                  warp_best(be, bv, bk, bal);
                  resolve(r, be, bv, bk);
                }
              }
            }
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&acc_empty[ab]);
          } else {
            // every correlation the warp needs is reduced to the 8 maxima of
            // each half before the screen, and the accumulator goes back to
            // the MMA at once.  In the rare case that some lane passes, of
            // the lanes that pass a flagged range those within two margins
            // of the warp's smallest float score can hold the range's best
            // (usually one); they queue the pair for exact scoring (flush,
            // which recovers the isometry of the maximum from the operands),
            // and the range's threshold drops at once to that smallest score
            // plus two margins -- an upper bound of the queued pair's exact
            // score plus the margin, so a valid threshold while the pair
            // stays queued.
            // With two halves per warp visit (one group per tile) the first
            // is screened while the accumulator is still held, so that only
            // one half's maxima are live at a time; the accumulator goes
            // back right after the last half's loads.
            const int64_t myslot = g.slot0 + (int64_t)t * kTileDoms + dl;
#pragma unroll
            for (int h = 0; h < NH; ++h) {
              float cmh[8];
              if (ok) ptx::tmem_ldmax8x8_wait(tb + (c0 + 2 * h) * 32, cmh);
              if (h == NH - 1) {
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&acc_empty[ab]);
              }
              const int rb0 = (c0 + 2 * h) * RPC;
              float m = INFINITY;
              float dm[8];
#pragma unroll
              for (int j = 0; j < 8; ++j) dm[j] = INFINITY;
              if (ok) screen8(cmh, rb0, dm, m);
              if (__any_sync(0xffffffffu, dvalid && m <= 0.f)) {
                uint32_t fl = 0;
#pragma unroll
                for (int j = 0; j < 8; ++j) fl |= (dvalid && dm[j] <= 0.f) ? 1u << j : 0u;
#pragma unroll 1
                for (uint32_t wm = __reduce_or_sync(0xffffffffu, fl); wm; wm &= wm - 1) {
                  const int j = __ffs(wm) - 1;
                  const int r = rb0 + j;
                  float cmj = cmh[0];
#pragma unroll
                  for (int jj = 1; jj < 8; ++jj)
                    if (jj == j) cmj = cmh[jj];
                  const float wr = sW[r];
                  const float scj = score(cmj, wr);
                  const bool mine = dvalid && scj <= sThr[r];
                  if (!__any_sync(0xffffffffu, mine)) continue;
                  float mn = mine ? scj : INFINITY;
#pragma unroll
                  for (int o = 16; o > 0; o >>= 1)
                    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                  const float lim = __fadd_ru(mn, 2.0f * sDelta[r]);
                  const bool need = mine && scj <= lim;
                  const unsigned bal = __ballot_sync(0xffffffffu, need);
                  const int cnt = __popc(bal);
                  if (qn + cnt > Cf::QCAP) flush();
                  if (need) {
                    int pi = 0;
                    if constexpr (MODE == MODE_GRID)
                      pi = (int)fminf(fmaxf(rintf(fmaf(nX, wr, cmj) * F1), 0.f), qf);
                    const int slot = qn + __popc(bal & ((1u << lane) - 1u));
                    myq[slot] = QCand{myslot, (int32_t)cmj, r | (pi << 12)};
                  }
                  qn += cnt;
                  __syncwarp();
                  if (lane == 0 && lim < sThr[r]) {
                    sThr[r] = lim;
                    atomicMin(a.gthr + g.r0 + r, thr_to_ord(lim));
                  }
                  __syncwarp();
                }
              }
            }
          }
        } else {
          float ra[32], rb[32], ma[4], mb[4];
          // two TMEM loads in flight; the accumulator goes back to the MMA
          // once the tile's last chunk is in registers
          if (ok) load(0, ra, ma);
#pragma unroll 1
          for (int ch = 0; ch < Cf::NCH; ch += 2) {
            if (ok) {
              ptx::tmem_wait_red(ra, ma);
              load(ch + 1, rb, mb);
              chunk(ch, ra, ma);
              ptx::tmem_wait_red(rb, mb);
              if (ch + 2 < Cf::NCH) load(ch + 2, ra, ma);
            }
            if (ch + 2 >= Cf::NCH) {
              ptx::tc_fence_before();
              __syncwarp();
              if (lane == 0) ptx::mbar_arrive(&acc_empty[ab]);
            }
            if (ok) chunk(ch + 1, rb, mb);
          }
        }
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(rec_empty);
      }
      // the queued candidates' exact scores, then merge the warps' bests per
      // range; one thread per range writes the item's partial
      flush();
      __syncwarp();
      ptx::named_bar_sync(1, epi_threads);
      if (ew == 0 && lane < kTileRanges) {
        Cand best{INT64_MAX, INT64_MAX};
        int64_t bv = 0;
        for (int o = 0; o < Cf::Wp::EPI_WARPS; ++o) {
          const Cand x = wbest[o * kTileRanges + lane];
          if constexpr (MODE == MODE_EXACT) {
            const int64_t xv = x.key == INT64_MAX ? 0 : pos_v(a.pm, g.im, x.key >> 3, n);
            if (exact_better(x.score, xv, x.key, best.score, bv, best.key)) best = x, bv = xv;
          } else if (x.score < best.score || (x.score == best.score && x.key < best.key)) {
            best = x;
          }
        }
        if (lane >= g.nr) best = Cand{INT64_MAX, INT64_MAX};
        a.part[g.pidx * kTileRanges + lane] = best;
      }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, Cf::TCOLS);
  }
}

// ---------------------------------------------------------------- host side
template <int B, int MODE, int G>
static int launch_tc_BMG(const MatchArgs& a, int grid, cudaStream_t st) {
  using Cf = TcCfg<B, G>;
  return launch_dep(k_match_tc<B, MODE, G>, dim3(grid), dim3(Cf::Wp::THREADS), Cf::SMEM + 128, st,
                    a) == cudaSuccess
             ? FIC_OK
             : FIC_ECUDA;
}

template <int B, int MODE, int G>
static int prepare_BMG() {
  using Cf = TcCfg<B, G>;
  if (cudaFuncSetAttribute(k_match_tc<B, MODE, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           Cf::SMEM + 128) != cudaSuccess)
    return 1;
  // the warpgroups' register split is paid for by the launch allocation
  cudaFuncAttributes at{};
  if (cudaFuncGetAttributes(&at, k_match_tc<B, MODE, G>) != cudaSuccess) return 1;
  return at.numRegs >= Cf::Wp::LREGS ? 0 : 1;
}

template <int B, int G>
static int prepare_BG() {
  return prepare_BMG<B, MODE_M1, G>() | prepare_BMG<B, MODE_M2, G>() |
         prepare_BMG<B, MODE_GRID, G>() | prepare_BMG<B, MODE_EXACT, G>();
}

// Opt the matcher kernels in to their shared memory (once per device, before
// any launch or stream capture).
int match_tc_prepare() {
  return (prepare_BG<16, 1>() | prepare_BG<8, 2>() | prepare_BG<8, 1>() | prepare_BG<4, 2>() |
          prepare_BG<4, 1>() | prepare_BG<2, 2>() | prepare_BG<2, 1>())
             ? FIC_ECUDA
             : FIC_OK;
}

template <int B, int G>
static int launch_tc_BG(const MatchArgs& a, int grid, cudaStream_t st) {
  if (a.S.exact) return launch_tc_BMG<B, MODE_EXACT, G>(a, grid, st);
  if (a.S.grid) return launch_tc_BMG<B, MODE_GRID, G>(a, grid, st);
  if (a.S.m > 1) return launch_tc_BMG<B, MODE_M2, G>(a, grid, st);
  return launch_tc_BMG<B, MODE_M1, G>(a, grid, st);
}

int launch_match_tc(const MatchArgs& a, int grid, cudaStream_t st) {
  const bool g1 = a.groups_per_tile == 1;
  switch (a.B) {
    case 16: return launch_tc_BG<16, 1>(a, grid, st);
    case 8: return g1 ? launch_tc_BG<8, 1>(a, grid, st) : launch_tc_BG<8, 2>(a, grid, st);
    case 4: return g1 ? launch_tc_BG<4, 1>(a, grid, st) : launch_tc_BG<4, 2>(a, grid, st);
    case 2: return g1 ? launch_tc_BG<2, 1>(a, grid, st) : launch_tc_BG<2, 2>(a, grid, st);
    default: return FIC_EINVAL;
  }
}

// Rounding bound of the float scores (score units E' / (8 q n)).  With
// |r'| <= 128 and |Ds'| <= 512: |corr| <= 65536 n and |w sum Ds'| <= 65536 n,
// so |y| <= Y = 131072 n; V <= n^2 1020^2 / 4, so u <= U = 260100 n / (8 q).
// One score costs at most three roundings of quantities bounded by
// p^2 U + p Y (explicit S) or q (q U + Y) (grid, plus the choice of the
// nearest grid point); 2^-20 times that bound leaves a margin of 8x or more.
float screening_delta(int B, const SSet& S) {
  const double n = (double)B * B;
  const double Y = 131072.0 * n;
  const double U = 260100.0 * n / (8.0 * S.q);
  double pm = 0;
  if (S.grid) {
    pm = S.q;
  } else {
    for (int i = 0; i < S.m; ++i) pm = pm > S.p[i] ? pm : S.p[i];
  }
  const double bound = pm * pm * U + pm * Y;
  return (float)(ldexp(bound, -20));
}

}  // namespace fic
