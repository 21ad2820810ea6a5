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
//               half at B = 16) and the per-domain scoring records;
//   warp 1      allocates tensor memory and issues the MMAs (one thread);
//   warps 2-5   epilogue: each owns 32 TMEM lanes = 32 rows (range, isometry)
//               and reduces the 128 columns of every tile to the row's best
//               (domain, s) candidate.
//
// Epilogue.  For s = p/q, E of Eq. 1 with o from Eq. 3 is, up to the
// range-only term, E' = p^2 V - 8 p q C with C = n <r', Ds'> - sum r' sum Ds'
// (exact integers).  The float score E' / (8 q n) = p^2 u - p y, with
// u = V / (8 q n) and y = C / n = corr - (sum r' / n) sum Ds', screens the
// candidates: a column is skipped only when its float score exceeds the
// row's best exact score by more than the level's rounding bound `delta`;
// every other candidate is scored exactly in int64 and compared with the
// tie-break key (pos * 8 + k) * |S| + s_idx.  The result therefore equals the
// exhaustive exact argmin.
#include <math.h>

#include <type_traits>

#include "level.cuh"
#include "tc_ptx.cuh"

namespace fic {

template <int B>
struct TcCfg {
  static constexpr int n = B * B;
  static constexpr int Kp = n < 16 ? 16 : n;          // K padded to the MMA K step
  static constexpr int NKC = n > 128 ? n / 128 : 1;   // exact accumulators per tile
  static constexpr int KS = Kp / NKC;                 // K per pipeline stage
  static constexpr int KSTEPS = KS / 16;              // MMAs per stage
  static constexpr int A_BYTES = kTileRows * Kp * 2;
  static constexpr int ST_BYTES = kTileDoms * KS * 2;
  static constexpr int NST = B == 16 ? 4 : 8;
  static constexpr int NACC = B == 16 ? 2 : 4;
  static constexpr int TCOLS = 512;
  static constexpr int DF_BYTES = kTileDoms * 16;
  static constexpr int SCR_BYTES = 4 * 32 * 32 * 4;
  static constexpr int OFF_B = A_BYTES;
  static constexpr int OFF_DF = OFF_B + NST * ST_BYTES;
  static constexpr int OFF_SCR = OFF_DF + NACC * DF_BYTES;
  static constexpr int OFF_BAR = OFF_SCR + SCR_BYTES;
  static constexpr int NBAR = 2 * NST + 2 + 3 * NACC + 1;
  static constexpr int OFF_MISC = OFF_BAR + NBAR * 8;
  static constexpr int BYTES = OFF_MISC + 16;
  // one CTA per SM: the CTA owns all 512 TMEM columns
  static constexpr int SMEM = BYTES < 120 * 1024 ? 120 * 1024 : BYTES;
  static_assert(NACC * NKC * 128 <= TCOLS, "tensor memory");
  static_assert(BYTES + 1024 <= 227 * 1024, "shared memory");
};

constexpr int kTcThreads = 192;
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

// Per-row best candidate of the epilogue.
struct RowBest {
  int64_t e;    // exact E'
  int64_t key;
  float thr;    // skip a candidate whose float score is above this
};

__device__ inline float thr_of(int64_t e, double inv8qn, float delta) {
  return __double2float_ru(fma((double)e, inv8qn, (double)delta));
}

template <int B, int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_match_tc(MatchArgs a) {
  using Cf = TcCfg<B>;
  constexpr int n = Cf::n;
  constexpr int LOGN = B == 16 ? 8 : B == 8 ? 6 : B == 4 ? 4 : 2;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + Cf::OFF_B;
  float4* sDf = (float4*)(smem + Cf::OFF_DF);
  float* sScr = (float*)(smem + Cf::OFF_SCR);
  uint64_t* bars = (uint64_t*)(smem + Cf::OFF_BAR);
  uint64_t* full_b = bars;
  uint64_t* empty_b = bars + Cf::NST;
  uint64_t* a_full = bars + 2 * Cf::NST;
  uint64_t* a_empty = a_full + 1;
  uint64_t* acc_full = a_empty + 1;
  uint64_t* acc_empty = acc_full + Cf::NACC;
  uint64_t* df_full = acc_empty + Cf::NACC;
  uint64_t* done_bar = df_full + Cf::NACC;
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
      ptx::mbar_init(&acc_empty[i], 4);
      ptx::mbar_init(&df_full[i], 1);
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

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t bi = 0, ai = 0, ti = 0;
      uint32_t issued_par[Cf::NST];
      bool issued[Cf::NST];
      for (int i = 0; i < Cf::NST; ++i) issued[i] = false, issued_par[i] = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; ok && it < items; it += gridDim.x) {
        const ItemGeo g = item_geo(a, it, CH);
        if (!ptx::mbar_wait(a_empty, (ai & 1) ^ 1) || *abort_flag) { ok = false; break; }
        ptx::mbar_expect_tx(a_full, Cf::A_BYTES);
        ptx::bulk_g2s(sA, a.apack + g.r0 * 8 * Cf::Kp, Cf::A_BYTES, a_full);
        ++ai;
        for (int t = g.t0; ok && t < g.t1; ++t) {
          const int db = ti % Cf::NACC;
          if (!ptx::mbar_wait(&acc_empty[db], ((ti / Cf::NACC) & 1) ^ 1) || *abort_flag) {
            ok = false;
            break;
          }
          ptx::mbar_expect_tx(&df_full[db], Cf::DF_BYTES);
          ptx::bulk_g2s((uint8_t*)sDf + db * Cf::DF_BYTES,
                        a.domf + g.slot0 + (int64_t)t * kTileDoms, Cf::DF_BYTES, &df_full[db]);
          ++ti;
          const int64_t tile_g = g.slot0 / kTileDoms + t;
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
  } else {
    // ------------------------------------------------------------ epilogue
    const int qd = warp & 3;                 // TMEM lane quarter of this warp
    const int row = qd * 32 + lane;          // tile row = (range, isometry)
    const int k_iso = row & 7;
    float* scr = sScr + (warp - 2) * 32 * 32;
    const int m_s = a.S.m;
    const int qv = a.S.q;
    const double inv8qn = 1.0 / (8.0 * qv * n);
    const float delta = a.delta;
    const float p0f = (float)a.S.p[0], p1f = (float)a.S.p[1];
    const float qf = (float)qv;
    uint32_t ti = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
      const ItemGeo g = item_geo(a, it, CH);
      const int rr = row >> 3;
      const bool valid = rr < g.nr;
      int32_t srp = 0;
      if (valid) srp = a.mom[g.r0 + rr].srp;
      const float w = (float)srp / (float)n;
      RowBest best{INT64_MAX, INT64_MAX, valid ? INFINITY : -INFINITY};

      // exact score of one candidate (column col of tile t, set index si)
      auto exact = [&](int t, int col, float cf, int si) {
        const DomRec d = a.dom[g.slot0 + (int64_t)t * kTileDoms + col];
        const int64_t ci = (int64_t)(int)cf;
        const int64_t C = (ci << LOGN) - (int64_t)srp * (int64_t)d.sdp;
        const int64_t p = (MODE == MODE_GRID) ? si : a.S.p[si];
        const int64_t e = p * p * d.v - 8 * p * qv * C;
        const int64_t key = ((int64_t)d.pos * 8 + k_iso) * m_s + si;
        if (e < best.e || (e == best.e && key < best.key)) {
          best.e = e;
          best.key = key;
          best.thr = thr_of(e, inv8qn, delta);
        }
      };

      for (int t = g.t0; t < g.t1; ++t) {
        const int ab = ti % Cf::NACC;
        const uint32_t par = (ti / Cf::NACC) & 1;
        const bool got =
            ok && ptx::mbar_wait(&acc_full[ab], par) && ptx::mbar_wait(&df_full[ab], par);
        // the TMEM loads below are warp-collective: the lanes agree on the outcome
        const bool all = __all_sync(0xffffffffu, got);
        if (ok && !all && lane == 0) fail();
        ok = all;
        ptx::tc_fence_after();
        const float4* Df = sDf + ab * kTileDoms;
        const int nv = min(kTileDoms, g.nkept - t * kTileDoms);
        if (ok) {
#pragma unroll 1
          for (int cc = 0; cc < 4; ++cc) {
            const int nvc = nv - cc * 32;
            if (nvc <= 0) break;
            uint32_t r0[32];
            const uint32_t ta = tmem + ((uint32_t)(qd * 32) << 16) +
                                (uint32_t)(ab * Cf::NKC * kTileDoms + cc * 32);
            ptx::tmem_ld32(ta, r0);
            float c[32];
            if constexpr (Cf::NKC == 2) {
              uint32_t r1[32];
              ptx::tmem_ld32(ta + kTileDoms, r1);
              ptx::tmem_wait(r0);
              ptx::tmem_dep(r1);
#pragma unroll
              for (int j = 0; j < 32; ++j) c[j] = __uint_as_float(r0[j]) + __uint_as_float(r1[j]);
            } else {
              ptx::tmem_wait(r0);
#pragma unroll
              for (int j = 0; j < 32; ++j) c[j] = __uint_as_float(r0[j]);
            }
            // fast screen: the chunk's minimum float score (full chunks
            // unmasked; the ragged last chunk masks columns >= nvc)
            auto screen = [&](auto masked) {
              // two columns per step, four independent running minima
              float mn[4] = {INFINITY, INFINITY, INFINITY, INFINITY};
              auto score1 = [&](int j, float y, const float4& f) {
                float s;
                if constexpr (MODE == MODE_GRID) {
                  float p = rintf(y * f.z);
                  p = fminf(fmaxf(p, 0.f), qf);
                  s = p * fmaf(p, f.y, -y);
                } else {
                  s = fmaf(-p0f, y, f.y);
                }
                if constexpr (decltype(masked)::value) s = j < nvc ? s : INFINITY;
                return s;
              };
#pragma unroll
              for (int j = 0; j < 32; j += 2) {
                const float4 fa = Df[cc * 32 + j], fb = Df[cc * 32 + j + 1];
                const float ya = fmaf(-w, fa.x, c[j]), yb = fmaf(-w, fb.x, c[j + 1]);
                float& m = mn[(j >> 1) & 3];
                if constexpr (MODE == MODE_M2) {
                  float a0 = fmaf(-p0f, ya, fa.y), a1 = fmaf(-p1f, ya, fa.z);
                  float b0 = fmaf(-p0f, yb, fb.y), b1 = fmaf(-p1f, yb, fb.z);
                  if constexpr (decltype(masked)::value) {
                    a0 = j < nvc ? a0 : INFINITY;
                    a1 = j < nvc ? a1 : INFINITY;
                    b0 = j + 1 < nvc ? b0 : INFINITY;
                    b1 = j + 1 < nvc ? b1 : INFINITY;
                  }
                  m = ptx::fmin3(ptx::fmin3(a0, a1, b0), b1, m);
                } else {
                  m = ptx::fmin3(score1(j, ya, fa), score1(j + 1, yb, fb), m);
                }
              }
              return fminf(fminf(mn[0], mn[1]), fminf(mn[2], mn[3]));
            };
            const float mn = nvc >= 32 ? screen(std::false_type{}) : screen(std::true_type{});
            if (__any_sync(0xffffffffu, mn <= best.thr)) {
              // slow path: exact scores of every candidate that can win
#pragma unroll
              for (int j = 0; j < 32; ++j) scr[j * 32 + lane] = c[j];
              __syncwarp();
              if (mn <= best.thr) {
                const int jn = nvc < 32 ? nvc : 32;
#pragma unroll 1
                for (int j = 0; j < jn; ++j) {
                  const float cf = scr[j * 32 + lane];
                  const float4 f = Df[cc * 32 + j];
                  const float y = fmaf(-w, f.x, cf);
                  if constexpr (MODE == MODE_GRID) {
                    float p = rintf(y * f.z);
                    p = fminf(fmaxf(p, 0.f), qf);
                    const float s = p * fmaf(p, f.y, -y);
                    if (s <= best.thr) {
                      const int pi = (int)p;
                      for (int pp = max(pi - 1, 0); pp <= min(pi + 1, qv); ++pp)
                        exact(t, cc * 32 + j, cf, pp);
                    }
                  } else {
                    if (fmaf(-p0f, y, f.y) <= best.thr) exact(t, cc * 32 + j, cf, 0);
                    if constexpr (MODE == MODE_M2)
                      if (fmaf(-p1f, y, f.z) <= best.thr) exact(t, cc * 32 + j, cf, 1);
                  }
                }
              }
              __syncwarp();
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&acc_empty[ab]);
        ++ti;
      }
      Cand out;
      out.score = valid ? best.e : INT64_MAX;
      out.key = valid ? best.key : INT64_MAX;
      a.part[it * kTileRows + row] = out;
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
  k_match_tc<B, MODE><<<grid, kTcThreads, TcCfg<B>::SMEM + 1024, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? FIC_OK : FIC_ECUDA;
}

template <int B, int MODE>
static int prepare_BM() {
  return cudaFuncSetAttribute(k_match_tc<B, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TcCfg<B>::SMEM + 1024) == cudaSuccess
             ? 0
             : 1;
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
