// match_f32.cu -- plain FP32 CUDA-core matcher (the comparison path).
//
// For every work item (16 ranges x 8 isometries = 128 rows, a chunk of
// 128-domain tiles) it computes the correlations <T_k^-1 R, Ds> with FP32
// FMAs (a register-tiled SGEMM, 8 x 8 outputs per thread), scores every
// (domain, isometry, s) in FP32 and keeps each row's best.  Scores are
// E' / (8 q n) with E' = p^2 V - 8 p q C (Eq. 1 after Eq. 3, times 16 q^2 n
// and without the range-only term): for s = p / q and the centred moments
//   y = <r - 128, Ds - 512> - (sum(r - 128) / n) sum(Ds - 512)   (= C / n)
//   score(p) = p^2 V / (8 q n) - p y.
// Explicit S sets evaluate every p; the grid takes the real minimiser
// p* = y / (2 u), u = V / (8 q n), rounded to the nearest grid point (E' is
// a convex quadratic in p).  Ties and near-ties are resolved in FP32 only.
#include <math.h>

#include "level.cuh"

namespace fic {

constexpr int kF32Threads = 256;

__device__ inline int64_t order_bits(float f) {
  int b = __float_as_int(f);
  return (int64_t)(b >= 0 ? b : (b ^ 0x7fffffff));
}

template <int B>
__global__ void __launch_bounds__(kF32Threads)
k_match_f32(MatchArgs a) {
  constexpr int n = B * B;
  constexpr int KC = n < 16 ? n : 16;
  __shared__ float As[KC][kTileRows + 4];
  __shared__ float Bs[KC][kTileDoms + 4];
  __shared__ float4 Df[kTileDoms];
  __shared__ int32_t Dpos[kTileDoms];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t items = a.meta->items;
  const int CH = a.meta->chunk_tiles;
  const int m_s = a.S.m;
  const float qf = (float)a.S.q;

  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int im = find_segment(a.item_off, a.n_images, it);
    const int nc = a.chunks[im];
    const int64_t local = it - a.item_off[im];
    const int64_t mt = local / nc;
    const int c = (int)(local % nc);
    const int64_t r0 = a.act_off[im] + mt * kTileRanges;  // first range of the tile
    const int nr = (int)min((int64_t)kTileRanges, a.act_cnt[im] - mt * kTileRanges);
    const int nkept = a.sel[im].nkept;
    const int nt = ceil_div(nkept, kTileDoms);
    const int t0 = c * CH, t1 = min(nt, t0 + CH);

    // per-row constants of my 8 rows: rows ty + 16 i
    float w[8];
    float best[8];
    int bslot[8], bs[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = ty + 16 * i;
      const int rr = row >> 3;
      w[i] = rr < nr ? (float)a.mom[r0 + rr].srp / (float)n : 0.f;
      best[i] = INFINITY;
      bslot[i] = -1;
      bs[i] = 0;
    }
    const float* Ag = a.a32 + r0 * 8 * n;
    for (int t = t0; t < t1; ++t) {
      const int64_t d0 = a.pool_off[im] + (int64_t)t * kTileDoms;
      const int nv = min(kTileDoms, nkept - t * kTileDoms);
      const float* Bg = a.b32 + d0 * n;
      float acc[8][8];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
      __syncthreads();
      for (int j = tid; j < kTileDoms; j += blockDim.x) {
        const float* ft = a.domf + (d0 >> 7) * (4 * kTileDoms) + j;  // d0: tile start
        Df[j] = make_float4(ft[0], ft[kTileDoms], ft[2 * kTileDoms], ft[3 * kTileDoms]);
        Dpos[j] = a.dom[d0 + j].pos;
      }
      for (int k0 = 0; k0 < n; k0 += KC) {
        __syncthreads();
        for (int e = tid; e < kTileRows * KC; e += blockDim.x) {
          const int row = e / KC, kk = e % KC;
          As[kk][row] = Ag[(int64_t)row * n + k0 + kk];
          Bs[kk][row] = Bg[(int64_t)row * n + k0 + kk];
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
          float av[8], bv[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
          for (int j = 0; j < 8; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
          for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
      }
      // FP32 scoring of my 8 x 8 candidates
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = tx + 16 * j;
        if (col >= nv) continue;
        const float4 f = Df[col];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float y = fmaf(-w[i], f.x, acc[i][j]);
          if (a.S.grid) {
            float p = rintf(y * f.z);
            p = fminf(fmaxf(p, 0.f), qf);
            const float sc = p * fmaf(p, f.y, -y);
            if (sc < best[i]) { best[i] = sc; bslot[i] = col + t * kTileDoms; bs[i] = (int)p; }
          } else {
            const float s0 = fmaf(-(float)a.S.p[0], y, f.y);
            if (s0 < best[i]) { best[i] = s0; bslot[i] = col + t * kTileDoms; bs[i] = 0; }
            if (m_s > 1) {
              const float s1 = fmaf(-(float)a.S.p[1], y, f.z);
              if (s1 < best[i]) { best[i] = s1; bslot[i] = col + t * kTileDoms; bs[i] = 1; }
            }
          }
        }
      }
    }
    // reduce each row over the 16 threads that share it (same half-warp)
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = ty + 16 * i;
      const int k = row & 7;
      int64_t key = INT64_MAX;
      if (bslot[i] >= 0) {
        const int pos = a.dom[a.pool_off[im] + bslot[i]].pos;
        key = ((int64_t)pos * 8 + k) * m_s + bs[i];
      }
      int64_t sc = bslot[i] >= 0 ? order_bits(best[i]) : INT64_MAX;
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        const int64_t sc2 = __shfl_xor_sync(0xffffffffu, sc, o, 16);
        const int64_t k2 = __shfl_xor_sync(0xffffffffu, key, o, 16);
        if (sc2 < sc || (sc2 == sc && k2 < key)) { sc = sc2; key = k2; }
      }
      if (tx == 0) {
        Cand out;
        out.score = ((row >> 3) < nr) ? sc : INT64_MAX;
        out.key = ((row >> 3) < nr) ? key : INT64_MAX;
        a.part[it * kTileRows + row] = out;
      }
    }
  }
}

int launch_match_f32(const MatchArgs& a, int grid, cudaStream_t st) {
  switch (a.B) {
    case 16: k_match_f32<16><<<grid, kF32Threads, 0, st>>>(a); break;
    case 8: k_match_f32<8><<<grid, kF32Threads, 0, st>>>(a); break;
    case 4: k_match_f32<4><<<grid, kF32Threads, 0, st>>>(a); break;
    case 2: k_match_f32<2><<<grid, kF32Threads, 0, st>>>(a); break;
    default: return FIC_EINVAL;
  }
  return cudaGetLastError() == cudaSuccess ? FIC_OK : FIC_ECUDA;
}

}  // namespace fic
