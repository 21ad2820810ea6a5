// match_tc.cu -- the tensor-core matcher (sm_103a tcgen05).
//
// Sec. 2's search scores every range against every kept domain under the 8
// isometries.  With the isometries applied to the range (<R, T_k D> =
// <T_k^-1 R, D>), the correlations of a level form one dense contraction
//     corr[(range, k), domain] = sum_i (T_k^-1 R)_i (Ds_i - 512) ,  K = n,
// with rows r - 128 in [-128, 127] and columns Ds - 512 in [-512, 508]: small
// integers, exact in binary16.  Each 128-wide K slice keeps every partial sum
// below 2^23 in magnitude (128 * 512 * 128), so the f32 accumulators of
// tcgen05.mma kind::f16 hold the exact integer correlation; B = 16 (K = 256)
// uses two accumulators, one per K half, added as exact integers.
//
// Warp roles of one persistent CTA per SM:
//   warp 0      producer: bulk copies (TMA engine) of the resident 128-row
//               range tile, the streamed 128-domain tiles (one stage per K
//               half at B = 16) and each tile's per-domain scoring planes
//               and exact records;
//   warp 1      allocates tensor memory and issues the MMAs (one thread);
//   warps 2-3   idle (they complete the control warpgroup);
//   warps 4-    epilogue, EG groups of four warps (EG = 3, or 2 at B = 16
//               where shared memory is short): each warp owns the 32 TMEM
//               lanes = 32 rows (range, isometry) of its quarter; the groups
//               take turns on the tiles and merge their row bests per item.
//
// Epilogue.  For s = p/q, E of Eq. 1 with o from Eq. 3 is, up to the
// range-only term, E' = p^2 V - 8 p q C with C = n <r', Ds'> - sum r' sum Ds'
// (exact integers).  The float score E' / (8 q n) = p^2 u - p y, with
// u = V / (8 q n) and y = C / n = corr - (sum r' / n) sum Ds', screens the
// candidates: a column is skipped only when its float score exceeds the
// row's best exact score by more than the level's rounding bound `delta`;
// every other candidate is scored exactly in int64 and compared with the
// tie-break key (pos * 8 + k) * |S| + s_idx.  The result therefore equals the
// exhaustive exact argmin.  A threshold only has to bound the exact score of
// some candidate of the same range that stays in the reduction, so the 8
// isometry rows of a range share theirs (warp shuffles) and every CTA that
// scores the range shares it through a per-range word in global memory
// (atomicMin on an order-preserving image of the float).  Scores of two
// columns at a time use the packed f32x2 FMA.
//
// Rounding bound.  corr is exact, w = sum r' / n is exact (n is a power of
// two) and the FMAs round once each, so y carries at most 2^-24 |y| and a
// score F - p y (F = p^2 u rounded from double) at most
//     2^-23 (F + p |y|) <= 2^-23 (p^2 umax + p Y),   Y = 1024 sum |r'|,
// because |corr| <= 512 sum |r'| and |w sum Ds'| <= 512 |sum r'|; umax is the
// largest u of the level's kept domains.  The kernel uses 4x that bound
// (`delta`), per range.  A chunk's best float candidate X is scored exactly,
// so any candidate whose float score exceeds X's by more than 2 delta is
// strictly worse than X and is skipped as well.
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
  static constexpr int LREGS = EG == 2 ? 168 : 128;
  static constexpr int CREGS = EG == 2 ? 40 : 32;
  static constexpr int EREGS = EG == 2 ? 232 : 160;
  static_assert(32 * (kCtlWarps * CREGS + EPI_WARPS * EREGS) <= THREADS * LREGS,
                "register split exceeds the launch budget");
};

template <int B>
struct TcCfg {
  static constexpr int EG = B == 16 ? 2 : 3;          // epilogue warp groups
  using Wp = TcWarps<EG>;
  static constexpr int n = B * B;
  static constexpr int Kp = n < 16 ? 16 : n;          // K padded to the MMA K step
  static constexpr int NKC = n > 128 ? n / 128 : 1;   // exact accumulators per tile
  static constexpr int KS = Kp / NKC;                 // K per pipeline stage
  static constexpr int KSTEPS = KS / 16;              // MMAs per stage
  static constexpr int A_BYTES = kTileRows * Kp * 2;
  static constexpr int ST_BYTES = kTileDoms * KS * 2;
  static constexpr int NST = B == 16 ? 4 : B == 8 ? 6 : 8;   // operand stages
  static constexpr int NACC = B == 16 ? 2 : 4;                // TMEM accumulators
  static constexpr int ND = B == 16 ? 4 : B == 8 ? 8 : 16;    // scoring-record stages
  static constexpr int TCOLS = 512;
  static constexpr int CW = NKC == 1 ? 32 : 16;       // tile columns per epilogue chunk
  static constexpr int NCH = kTileDoms / CW;
  static constexpr int DT_BYTES = 4 * kTileDoms * 4;  // float planes {sum Ds', F0, F1, 0}
  static constexpr int DR_BYTES = kTileDoms * 16;     // DomRec per column
  static constexpr int D_BYTES = DT_BYTES + DR_BYTES;
  static constexpr int MRG_BYTES = (EG - 1) * kTileRows * 16;
  static constexpr int SCR_BYTES = Wp::EPI_WARPS * 32 * CW * 4;
  static constexpr int OFF_B = A_BYTES;
  static constexpr int OFF_D = OFF_B + NST * ST_BYTES;
  static constexpr int OFF_MRG = OFF_D + ND * D_BYTES;
  static constexpr int OFF_SCR = OFF_MRG + MRG_BYTES;
  static constexpr int OFF_BAR = OFF_SCR + SCR_BYTES;
  static constexpr int NBAR = 2 * NST + 2 + 2 * NACC + 2 * ND + 1;
  static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
  static constexpr int BYTES = OFF_MISC + 16;
  // one CTA per SM: the CTA owns all 512 TMEM columns
  static constexpr int SMEM = BYTES < 120 * 1024 ? 120 * 1024 : BYTES;
  static_assert(NACC * NKC * 128 <= TCOLS, "tensor memory");
  static_assert(BYTES + 128 <= 227 * 1024, "shared memory");
};

constexpr int MODE_M1 = 0, MODE_M2 = 1, MODE_GRID = 2;

struct ItemGeo {
  int im, nr, t0, t1, nkept;
  int64_t r0, slot0;
};

__device__ inline ItemGeo item_geo(const MatchArgs& a, int64_t it, int CH) {
  ItemGeo g;
  g.im = find_segment(a.item_off, a.n_images, it);
  const int nc = a.chunks[g.im];
  const int64_t local = it - a.item_off[g.im];
  const int64_t mt = local / nc;
  const int c = (int)(local % nc);
  g.r0 = a.act_off[g.im] + mt * kTileRanges;
  g.nr = (int)min((int64_t)kTileRanges, a.act_cnt[g.im] - mt * kTileRanges);
  g.nkept = a.sel[g.im].nkept;
  const int nt = ceil_div(g.nkept, kTileDoms);
  g.t0 = c * CH;
  g.t1 = min(nt, g.t0 + CH);
  g.slot0 = a.pool_off[g.im];
  return g;
}

// Skip a candidate whose float score is above this (exact E' plus the margin).
__device__ inline float thr_of(int64_t e, double inv8qn, float delta) {
  return __double2float_ru(fma((double)e, inv8qn, (double)delta));
}

template <int B, int MODE>
__global__ void __launch_bounds__(TcCfg<B>::Wp::THREADS, 1) k_match_tc(MatchArgs a) {
  using Cf = TcCfg<B>;
  constexpr int EG = Cf::EG;
  constexpr int n = B * B;
  constexpr int LOGN = B == 16 ? 8 : B == 8 ? 6 : B == 4 ? 4 : 2;
  constexpr int CW = Cf::CW;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  uint8_t* sA = smem;
  uint8_t* sB = smem + Cf::OFF_B;
  uint64_t* bars = (uint64_t*)(smem + Cf::OFF_BAR);
  uint64_t* full_b = bars;
  uint64_t* empty_b = bars + Cf::NST;
  uint64_t* a_full = bars + 2 * Cf::NST;
  uint64_t* a_empty = a_full + 1;
  uint64_t* acc_full = a_empty + 1;
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
      ptx::mbar_init(&empty_b[i], 1);
    }
    ptx::mbar_init(a_full, 1);
    ptx::mbar_init(a_empty, 1);
    for (int i = 0; i < Cf::NACC; ++i) {
      ptx::mbar_init(&acc_full[i], 1);
      ptx::mbar_init(&acc_empty[i], 4);  // the four warps of the group that reads it
    }
    for (int i = 0; i < Cf::ND; ++i) {
      ptx::mbar_init(&d_full[i], 1);
      ptx::mbar_init(&d_empty[i], 4);
    }
    ptx::mbar_init(done_bar, 1);
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
      uint32_t bi = 0, ai = 0, ti = 0;
      uint32_t issued_par[Cf::NST], d_par[Cf::ND];
      bool issued[Cf::NST], d_issued[Cf::ND];
      for (int i = 0; i < Cf::NST; ++i) issued[i] = false, issued_par[i] = 0;
      for (int i = 0; i < Cf::ND; ++i) d_issued[i] = false, d_par[i] = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; ok && it < items; it += gridDim.x) {
        const ItemGeo g = item_geo(a, it, CH);
        if (!ptx::mbar_wait(a_empty, (ai & 1) ^ 1) || *abort_flag) { ok = false; break; }
        ptx::mbar_expect_tx(a_full, Cf::A_BYTES);
        ptx::bulk_g2s(sA, a.apack + g.r0 * 8 * Cf::Kp, Cf::A_BYTES, a_full);
        ++ai;
        for (int t = g.t0; ok && t < g.t1; ++t) {
          // the tile's scoring records: a ring of their own, ND tiles ahead
          const int db = ti % Cf::ND;
          if (!ptx::mbar_wait(&d_empty[db], ((ti / Cf::ND) & 1) ^ 1) || *abort_flag) {
            ok = false;
            break;
          }
          const int64_t tile_g = g.slot0 / kTileDoms + t;
          uint8_t* dst = smem + Cf::OFF_D + db * Cf::D_BYTES;
          ptx::mbar_expect_tx(&d_full[db], Cf::D_BYTES);
          ptx::bulk_g2s(dst, a.domf + tile_g * (4 * kTileDoms), Cf::DT_BYTES, &d_full[db]);
          ptx::bulk_g2s(dst + Cf::DT_BYTES, a.dom + tile_g * kTileDoms, Cf::DR_BYTES,
                        &d_full[db]);
          d_issued[db] = true;
          d_par[db] = (ti / Cf::ND) & 1;
          ++ti;
          for (int kc = 0; kc < Cf::NKC; ++kc) {
            const int st = bi % Cf::NST;
            if (!ptx::mbar_wait(&empty_b[st], ((bi / Cf::NST) & 1) ^ 1) || *abort_flag) {
              ok = false;
              break;
            }
            ptx::mbar_expect_tx(&full_b[st], Cf::ST_BYTES);
            ptx::bulk_g2s(sB + st * Cf::ST_BYTES,
                          (const uint8_t*)a.bpack + (tile_g * Cf::NKC + kc) * Cf::ST_BYTES,
                          Cf::ST_BYTES, &full_b[st]);
            issued[st] = true;
            issued_par[st] = (bi / Cf::NST) & 1;
            ++bi;
          }
        }
      }
      if (!ok) fail();
      // drain: every copy this thread issued has landed before the CTA exits
      for (int i = 0; i < Cf::NST; ++i)
        if (issued[i]) ptx::mbar_wait(&full_b[i], issued_par[i]);
      for (int i = 0; i < Cf::ND; ++i)
        if (d_issued[i]) ptx::mbar_wait(&d_full[i], d_par[i]);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t IDESC = ptx::idesc_f16_f32(kTileRows, kTileDoms);
      uint32_t bi = 0, ai = 0, ti = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; ok && it < items; it += gridDim.x) {
        const ItemGeo g = item_geo(a, it, CH);
        if (!ptx::mbar_wait(a_full, ai & 1) || *abort_flag) { ok = false; break; }
        ++ai;
        ptx::tc_fence_after();
        for (int t = g.t0; ok && t < g.t1; ++t) {
          const int ab = ti % Cf::NACC;
          if (!ptx::mbar_wait(&acc_empty[ab], ((ti / Cf::NACC) & 1) ^ 1) || *abort_flag) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          for (int kc = 0; kc < Cf::NKC; ++kc) {
            const int st = bi % Cf::NST;
            if (!ptx::mbar_wait(&full_b[st], (bi / Cf::NST) & 1) || *abort_flag) {
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t d = tmem + (uint32_t)((ab * Cf::NKC + kc) * kTileDoms);
#pragma unroll
            for (int s = 0; s < Cf::KSTEPS; ++s) {
              const int kk = (kc * Cf::KSTEPS + s) * 2;  // core-matrix column of A
              const uint64_t ad = ptx::smem_desc(sA + kk * 128, 128, 16 * Cf::Kp);
              const uint64_t bd = ptx::smem_desc(sB + st * Cf::ST_BYTES + s * 256, 128, 16 * Cf::KS);
              ptx::mma_f16(d, ad, bd, IDESC, s > 0 ? 1u : 0u);
            }
            ptx::mma_commit(&empty_b[st]);
            ++bi;
          }
          if (!ok) break;
          ptx::mma_commit(&acc_full[ab]);
          ++ti;
        }
        ptx::mma_commit(a_empty);
      }
      if (!ok) fail();
      ptx::mma_commit(done_bar);
      if (!ptx::mbar_wait(done_bar, 0)) atomicOr(a.status, kStatusTimeout);
    }
  }
  } else {
    ptx::setmaxnreg_inc<Cf::Wp::EREGS>();
    // ------------------------------------------------------------ epilogue
    // Warps 4..: quarter qd = warp % 4 of the TMEM lanes (rows); group h
    // takes the tiles ti = h mod EG.  The groups' row bests merge at item end.
    const int ew = warp - kCtlWarps;
    const int h = ew >> 2;
    const int qd = warp & 3;
    const int row = qd * 32 + lane;          // tile row = (range, isometry)
    const int k_iso = row & 7;
    float* scr = (float*)(smem + Cf::OFF_SCR) + ew * 32 * CW;
    Cand* mrg = (Cand*)(smem + Cf::OFF_MRG);
    const int m_s = a.S.m;
    const int qv = a.S.q;
    const double inv8qn = 1.0 / (8.0 * qv * n);
    const double umax = (double)*a.umax;
    const double pmx = (double)(MODE == MODE_M2 ? max(a.S.p[0], a.S.p[1]) : a.S.p[0]);
    const float p0f = (float)a.S.p[0], p1f = (float)a.S.p[1];
    const float qf = (float)qv;
    const float2 np0 = make_float2(-p0f, -p0f), np1 = make_float2(-p1f, -p1f);
    uint32_t ti = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
      const ItemGeo g = item_geo(a, it, CH);
      const int rr = row >> 3;
      const bool valid = rr < g.nr;
      int32_t srp = 0, sabs = 0;
      if (valid) {
        const RangeMom m = a.mom[g.r0 + rr];
        srp = m.srp;
        sabs = m.sabs;
      }
      // rounding bound of this range's float scores (score units), the same
      // for its 8 rows in every CTA: 4x the bound derived above
      const float delta =
          MODE == MODE_GRID
              ? a.delta
              : __double2float_ru(ldexp(pmx * pmx * umax + pmx * 1024.0 * (double)sabs, -21));
      const float w = (float)srp / (float)n;
      const float2 nw2 = make_float2(-w, -w);
      uint32_t* gth = a.gthr + (g.r0 + (valid ? rr : 0));
      uint32_t gpre = valid ? __ldcg(gth) : kThrInit;
      int64_t best_e = INT64_MAX, best_key = INT64_MAX;
      float thr = valid ? INFINITY : -INFINITY;
      bool improved = false;

      // exact score of one candidate (tile column col, set index si)
      auto exact = [&](const DomRec* sDom, int col, float cf, int si) {
        const DomRec d = sDom[col];
        const int64_t ci = (int64_t)(int)cf;
        const int64_t C = (ci << LOGN) - (int64_t)srp * (int64_t)d.sdp;
        const int64_t p = (MODE == MODE_GRID) ? si : a.S.p[si];
        const int64_t e = p * p * d.v - 8 * p * qv * C;
        const int64_t key = ((int64_t)d.pos * 8 + k_iso) * m_s + si;
        if (e < best_e || (e == best_e && key < best_key)) {
          best_e = e;
          best_key = key;
          const float to = thr_of(e, inv8qn, delta);
          if (to < thr) {
            thr = to;
            improved = true;
          }
        }
      };

      for (int t = g.t0; t < g.t1; ++t, ++ti) {
        if ((int)(ti % EG) != h) continue;
        const int ab = ti % Cf::NACC;
        const int db = ti % Cf::ND;
        const bool got = ok && ptx::mbar_wait(&acc_full[ab], (ti / Cf::NACC) & 1) &&
                         ptx::mbar_wait(&d_full[db], (ti / Cf::ND) & 1);
        // the TMEM loads below are warp-collective: the lanes agree on the outcome
        const bool all = __all_sync(0xffffffffu, got);
        if (ok && !all && lane == 0) fail();
        ok = all;
        ptx::tc_fence_after();
        // threshold found by any CTA for this range (loaded one tile ahead)
        if (valid) thr = fminf(thr, ord_to_thr(gpre));
        gpre = valid ? __ldcg(gth) : kThrInit;
        const float* sX = (const float*)(smem + Cf::OFF_D + db * Cf::D_BYTES);
        const float* sF0 = sX + kTileDoms;
        const float* sF1 = sX + 2 * kTileDoms;
        const DomRec* sDom = (const DomRec*)(smem + Cf::OFF_D + db * Cf::D_BYTES + Cf::DT_BYTES);
        const int nv = min(kTileDoms, g.nkept - t * kTileDoms);
        const uint32_t tb = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(ab * Cf::NKC * kTileDoms);

        auto load = [&](int ch, uint32_t(&r)[32]) {
          if constexpr (Cf::NKC == 1) {
            ptx::tmem_ld32(tb + ch * 32, r);
          } else {
            ptx::tmem_ld16<0>(tb + ch * 16, r);
            ptx::tmem_ld16<16>(tb + kTileDoms + ch * 16, r);
          }
        };

        // fast screen of one chunk: the minimum float score over its
        // columns and S (masked past the tile's last kept domain)
        auto screen = [&](const float* c, int c0, int nvc, auto masked) {
          constexpr bool MK = decltype(masked)::value;
          float m0 = INFINITY, m1 = INFINITY, m2 = INFINITY, m3 = INFINITY;
#pragma unroll
          for (int j = 0; j < CW; j += 4) {
            const float4 X = *(const float4*)(sX + c0 + j);
            const float2 y01 = __ffma2_rn(nw2, make_float2(X.x, X.y), make_float2(c[j], c[j + 1]));
            const float2 y23 = __ffma2_rn(nw2, make_float2(X.z, X.w), make_float2(c[j + 2], c[j + 3]));
            if constexpr (MODE == MODE_GRID) {
              const float4 U = *(const float4*)(sF0 + c0 + j);
              const float4 G = *(const float4*)(sF1 + c0 + j);
              const float yy[4] = {y01.x, y01.y, y23.x, y23.y};
              const float uu[4] = {U.x, U.y, U.z, U.w};
              const float gg[4] = {G.x, G.y, G.z, G.w};
              float sc[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                float p = rintf(yy[u] * gg[u]);
                p = fminf(fmaxf(p, 0.f), qf);
                sc[u] = p * fmaf(p, uu[u], -yy[u]);
                if constexpr (MK) sc[u] = j + u < nvc ? sc[u] : INFINITY;
              }
              m0 = ptx::fmin3(sc[0], sc[1], m0);
              m1 = ptx::fmin3(sc[2], sc[3], m1);
            } else {
              const float4 F = *(const float4*)(sF0 + c0 + j);
              float2 s01 = __ffma2_rn(np0, y01, make_float2(F.x, F.y));
              float2 s23 = __ffma2_rn(np0, y23, make_float2(F.z, F.w));
              if constexpr (MK) {
                s01.x = j < nvc ? s01.x : INFINITY;
                s01.y = j + 1 < nvc ? s01.y : INFINITY;
                s23.x = j + 2 < nvc ? s23.x : INFINITY;
                s23.y = j + 3 < nvc ? s23.y : INFINITY;
              }
              m0 = ptx::fmin3(s01.x, s01.y, m0);
              m1 = ptx::fmin3(s23.x, s23.y, m1);
              if constexpr (MODE == MODE_M2) {
                const float4 F1 = *(const float4*)(sF1 + c0 + j);
                float2 b01 = __ffma2_rn(np1, y01, make_float2(F1.x, F1.y));
                float2 b23 = __ffma2_rn(np1, y23, make_float2(F1.z, F1.w));
                if constexpr (MK) {
                  b01.x = j < nvc ? b01.x : INFINITY;
                  b01.y = j + 1 < nvc ? b01.y : INFINITY;
                  b23.x = j + 2 < nvc ? b23.x : INFINITY;
                  b23.y = j + 3 < nvc ? b23.y : INFINITY;
                }
                m2 = ptx::fmin3(b01.x, b01.y, m2);
                m3 = ptx::fmin3(b23.x, b23.y, m3);
              }
            }
          }
          return fminf(fminf(m0, m1), fminf(m2, m3));
        };

        // slow path: exact scores of every candidate of the chunk that can win.
        // The lane marks its candidate columns (float score <= threshold) in
        // bit masks, then scores only those exactly, reading their exact
        // correlations back from its own column of the scratch.
        auto slow = [&](const float* c, int c0, int nvc, float mn) {
          if (mn <= thr) {
            // the chunk's best float candidate is scored exactly below, so
            // nothing more than 2 delta above it can win either
            const float cut = fminf(thr, __fadd_ru(mn, 2.f * delta));
            uint32_t mk0 = 0, mk1 = 0;
#pragma unroll
            for (int j = 0; j < CW; j += 2) {
              const float2 X2 = *(const float2*)(sX + c0 + j);
              const float2 y = __ffma2_rn(nw2, X2, make_float2(c[j], c[j + 1]));
              if constexpr (MODE == MODE_GRID) {
                const float2 U = *(const float2*)(sF0 + c0 + j);
                const float2 G = *(const float2*)(sF1 + c0 + j);
                float pa = fminf(fmaxf(rintf(y.x * G.x), 0.f), qf);
                float pb = fminf(fmaxf(rintf(y.y * G.y), 0.f), qf);
                if (pa * fmaf(pa, U.x, -y.x) <= cut) mk0 |= 1u << j;
                if (pb * fmaf(pb, U.y, -y.y) <= cut) mk0 |= 2u << j;
              } else {
                const float2 F = *(const float2*)(sF0 + c0 + j);
                const float2 s0 = __ffma2_rn(np0, y, F);
                if (s0.x <= cut) mk0 |= 1u << j;
                if (s0.y <= cut) mk0 |= 2u << j;
                if constexpr (MODE == MODE_M2) {
                  const float2 F1 = *(const float2*)(sF1 + c0 + j);
                  const float2 s1 = __ffma2_rn(np1, y, F1);
                  if (s1.x <= cut) mk1 |= 1u << j;
                  if (s1.y <= cut) mk1 |= 2u << j;
                }
              }
            }
            const uint32_t lim = nvc >= 32 ? 0xffffffffu : (1u << nvc) - 1u;
            mk0 &= lim;
            mk1 &= lim;
            if (mk0 | mk1) {
#pragma unroll
              for (int j = 0; j < CW; ++j) scr[j * 32 + lane] = c[j];
              while (mk0) {
                const int j = __ffs(mk0) - 1;
                mk0 &= mk0 - 1;
                const int col = c0 + j;
                const float cf = scr[j * 32 + lane];
                if constexpr (MODE == MODE_GRID) {
                  const float y = fmaf(-w, sX[col], cf);
                  const int pi = (int)fminf(fmaxf(rintf(y * sF1[col]), 0.f), qf);
                  for (int pp = max(pi - 1, 0); pp <= min(pi + 1, qv); ++pp)
                    exact(sDom, col, cf, pp);
                } else {
                  exact(sDom, col, cf, 0);
                }
              }
              while (mk1) {
                const int j = __ffs(mk1) - 1;
                mk1 &= mk1 - 1;
                exact(sDom, c0 + j, scr[j * 32 + lane], 1);
              }
            }
          }
          __syncwarp();
          // the 8 isometry rows of a range share the tightest threshold
          float t8 = thr;
          t8 = fminf(t8, __shfl_xor_sync(0xffffffffu, t8, 1));
          t8 = fminf(t8, __shfl_xor_sync(0xffffffffu, t8, 2));
          t8 = fminf(t8, __shfl_xor_sync(0xffffffffu, t8, 4));
          if (valid) {
            thr = t8;
            if (improved) {
              atomicMin(gth, thr_to_ord(thr));
              improved = false;
            }
          }
        };

        auto chunk = [&](int ch, const uint32_t* r) {
          const int c0 = ch * CW;
          float c[CW];
          if constexpr (Cf::NKC == 1) {
#pragma unroll
            for (int j = 0; j < CW; ++j) c[j] = __uint_as_float(r[j]);
          } else {
#pragma unroll
            for (int j = 0; j < CW; j += 2) {
              const float2 s2 =
                  __fadd2_rn(make_float2(__uint_as_float(r[j]), __uint_as_float(r[j + 1])),
                             make_float2(__uint_as_float(r[16 + j]), __uint_as_float(r[17 + j])));
              c[j] = s2.x;
              c[j + 1] = s2.y;
            }
          }
          const int nvc = nv - c0;
          const float mn = nvc >= CW ? screen(c, c0, nvc, std::false_type{})
                                     : screen(c, c0, nvc, std::true_type{});
          if (__any_sync(0xffffffffu, mn <= thr)) slow(c, c0, nvc, mn);
        };

        if (ok) {
          if constexpr (EG == 2) {
            // two warps per sub-partition: overlap the next chunk's TMEM
            // load with this chunk's scoring
            uint32_t ra[32], rb[32];
            load(0, ra);
#pragma unroll
            for (int ch = 0; ch < Cf::NCH; ch += 2) {
              if (ch * CW >= nv) break;
              ptx::tmem_wait(ra);
              if ((ch + 1) * CW < nv) load(ch + 1, rb);
              chunk(ch, ra);
              if ((ch + 1) * CW >= nv) break;
              ptx::tmem_wait(rb);
              if (ch + 2 < Cf::NCH && (ch + 2) * CW < nv) load(ch + 2, ra);
              chunk(ch + 1, rb);
            }
          } else {
            // three warps per sub-partition hide the load latency
#pragma unroll 1
            for (int ch = 0; ch < Cf::NCH; ++ch) {
              if (ch * CW >= nv) break;
              uint32_t ra[32];
              load(ch, ra);
              ptx::tmem_wait(ra);
              chunk(ch, ra);
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          ptx::mbar_arrive(&acc_empty[ab]);
          ptx::mbar_arrive(&d_empty[db]);
        }
      }
      // merge the groups' bests of this row; group 0 writes the partial
      if (h > 0) mrg[(h - 1) * kTileRows + row] = Cand{best_e, best_key};
      ptx::named_bar_sync(1 + qd, 32 * EG);
      if (h == 0) {
#pragma unroll
        for (int o2 = 0; o2 < EG - 1; ++o2) {
          const Cand o = mrg[o2 * kTileRows + row];
          if (o.score < best_e || (o.score == best_e && o.key < best_key)) {
            best_e = o.score;
            best_key = o.key;
          }
        }
        Cand out;
        out.score = valid ? best_e : INT64_MAX;
        out.key = valid ? best_key : INT64_MAX;
        a.part[it * kTileRows + row] = out;
      }
      ptx::named_bar_sync(1 + qd, 32 * EG);
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
template <int B, int MODE>
static int launch_tc_BM(const MatchArgs& a, int grid, cudaStream_t st) {
  k_match_tc<B, MODE><<<grid, TcCfg<B>::Wp::THREADS, TcCfg<B>::SMEM + 128, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? FIC_OK : FIC_ECUDA;
}

template <int B, int MODE>
static int prepare_BM() {
  if (cudaFuncSetAttribute(k_match_tc<B, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           TcCfg<B>::SMEM + 128) != cudaSuccess)
    return 1;
  // the warpgroups' register split is paid for by the launch allocation
  cudaFuncAttributes at{};
  if (cudaFuncGetAttributes(&at, k_match_tc<B, MODE>) != cudaSuccess) return 1;
  return at.numRegs >= TcCfg<B>::Wp::LREGS ? 0 : 1;
}

template <int B>
static int prepare_B() {
  return prepare_BM<B, MODE_M1>() | prepare_BM<B, MODE_M2>() | prepare_BM<B, MODE_GRID>();
}

// Opt the matcher kernels in to their shared memory (once per device, before
// any launch or stream capture).
int match_tc_prepare() {
  return (prepare_B<16>() | prepare_B<8>() | prepare_B<4>() | prepare_B<2>()) ? FIC_ECUDA : FIC_OK;
}

template <int B>
static int launch_tc_B(const MatchArgs& a, int grid, cudaStream_t st) {
  if (a.S.grid) return launch_tc_BM<B, MODE_GRID>(a, grid, st);
  if (a.S.m > 1) return launch_tc_BM<B, MODE_M2>(a, grid, st);
  return launch_tc_BM<B, MODE_M1>(a, grid, st);
}

int launch_match_tc(const MatchArgs& a, int grid, cudaStream_t st) {
  switch (a.B) {
    case 16: return launch_tc_B<16>(a, grid, st);
    case 8: return launch_tc_B<8>(a, grid, st);
    case 4: return launch_tc_B<4>(a, grid, st);
    case 2: return launch_tc_B<2>(a, grid, st);
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
