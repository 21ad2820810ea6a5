// fic_common.cuh -- shared definitions of the CUDA encoder (sm_103a).
//
// Notation follows "A Fast Fractal Image Compression Algorithm Using
// Predefined Values for Contrast Scaling" (Miar Naimi, Salarian): B is the
// range side (16 -> 8 -> 4 -> 2, Sec. 2), n = B*B, L the domain step, a domain
// is a 2B x 2B square decimated to B x B (Eq. 1), s = p/q the contrast scale
// and o the offset of Eq. 3.  All integer moments are exact; the decimated
// block is carried as the integer 2x2 sum Ds (the paper's D is Ds / 4).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fic.h"

namespace fic {

// ---------------------------------------------------------------- limits
constexpr int kMaxImages = 4096;      // images per fic_encode call
constexpr int kMaxS = 32;             // |S| of a level
constexpr int kKeyTableN = 1024;      // 4 B^2 for B = 16: pixels of a domain
constexpr int kTileRanges = 16;       // ranges per M tile (x 8 isometries = 128 rows)
constexpr int kTileRows = 128;        // M of the tensor tile
constexpr int kTileDoms = 128;        // N of one domain tile
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // bounded mbarrier waits: 2 s

// device status word bits (ctx->d_status)
constexpr uint32_t kStatusTimeout = 1u;
constexpr uint32_t kStatusOverflow = 2u;

// Tensor-path operand geometry.  K (= n) is padded to the MMA's K step of
// 16.  At B <= 8 each 128-domain tile of the kept pool is one contiguous
// block: the f16 operand (core-matrix layout), four float planes of 128
// scoring constants, then 128 DomRec -- one bulk copy per tile.  At B = 16
// the operand tiles stand alone and the records are separate arrays.
__host__ __device__ constexpr int tc_kp(int B) { return B * B < 16 ? 16 : B * B; }
__host__ __device__ constexpr int tc_op_bytes(int B) { return kTileDoms * tc_kp(B) * 2; }
__host__ __device__ constexpr int tc_rec_bytes() { return 4 * kTileDoms * 4 + kTileDoms * 16; }
__host__ __device__ constexpr int tc_tile_bytes(int B) {
  return B <= 8 ? tc_op_bytes(B) + tc_rec_bytes() : tc_op_bytes(B);
}

// ---------------------------------------------------------------- images
struct ImgDev {
  const uint8_t* pix;  // device pointer, row-major
  int W, H, pitch;
  int px, py;          // pool positions per row / column at the level
};

// Active range of a level: image, top-left corner.
struct RangeRec {
  int32_t img, x, y, parent;  // parent: index in the previous level (-1 at level 0)
};

// Per-range moments used by the scoring epilogues.
struct RangeMom {
  int32_t sr;      // sum of r
  int32_t srp;     // sum of (r - 128)
  int64_t a;       // n sum r^2 - (sum r)^2
  int32_t sabs;    // sum of |r - 128|: bounds the range's correlations
  int32_t pad;
};

// Per kept domain, for the scoring epilogues.
struct DomRec {
  int64_t v;       // n sum Ds^2 - (sum Ds)^2  (= 16 n^2 Var(D) scaled, shift invariant)
  int32_t sdp;     // sum of (Ds - 512)
  int32_t pos;     // raster index in the unfiltered pool of its image
};

// Level-wide constants of the S set (Sec. 2 grid or Sec. 3.1 values).
struct SSet {
  int m;            // |S|
  int q;            // common denominator
  int grid;         // 1: grid k/(M-1) (convex shortcut), 0: explicit list
  int exact;        // 1: Eq. 2's s of every pair, clamped to [0, 1] (m = 1)
  int p[kMaxS];     // numerators
};

// Exact lexicographic candidate: score first, then the tie-break key.  In
// the exact-s mode the score is the pair's C = n <r, Ds> - sum r sum Ds and
// the order is exact_better's (the domain's V comes with it).
struct Cand {
  int64_t score;    // E' (exact, tensor path), C (exact s) or float bits (fp32 path)
  int64_t key;      // (pos * 8 + iso) * |S| + s_idx
};

// Exact-s mode: with the pair's C and the domain's V = n sum Ds^2 - (sum Ds)^2
// the clamped Eq. 2 gives n E = A - G, G = 0 (C <= 0: s = 0), C^2 / V
// (0 < 4C < V: s = 4C / V) or (8C - V) / 16 (4C >= V: s = 1); A is the
// range's, so a larger G is a smaller E.  G as a fraction num / den.
struct GFrac {
  __int128 num;
  int64_t den;
};
__host__ __device__ inline GFrac exact_g(int64_t C, int64_t V) {
  if (C <= 0 || V <= 0) return GFrac{0, 1};
  if (4 * C >= V) return GFrac{(__int128)(8 * C - V), 16};
  return GFrac{(__int128)C * C, V};  // C^2 <= 2^68, times a den <= 2^37 below
}
// a better than b: larger G, then the lower key; INT64_MAX keys are "none".
__host__ __device__ inline bool exact_better(int64_t Ca, int64_t Va, int64_t ka, int64_t Cb,
                                             int64_t Vb, int64_t kb) {
  if (ka == INT64_MAX) return false;
  if (kb == INT64_MAX) return true;
  const GFrac a = exact_g(Ca, Va), b = exact_g(Cb, Vb);
  const __int128 l = a.num * b.den, r = b.num * a.den;
  return l > r || (l == r && ka < kb);
}

// ---------------------------------------------------------------- launches
// Programmatic dependent launch.  The kernels of the level chain and of the
// pool builds are launched with programmatic stream serialisation
// (launch_dep), so the next kernel of a stream is launched -- its blocks
// placed on the SMs -- while the previous one is still running; each such
// kernel starts with grid_dep_sync(), which waits until the kernels before it
// on the stream have completed and their writes are visible, and then lets
// the kernel after it be launched in turn.  Without a programmatic
// predecessor the wait returns at once.
__device__ __forceinline__ void grid_dep_sync() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------- helpers
__host__ __device__ inline int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Upper bound (exclusive) search: index i with off[i] <= x < off[i+1].
__device__ inline int find_segment(const int64_t* off, int n, int64_t x) {
  int lo = 0, hi = n;  // off[0] = 0 <= x < off[n]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// Isometry k of Sec. 2 as a map of block coordinates: output pixel (i, j) of
// T_k(D) is taken from D at iso_src(k, i, j).  k = 0..3 turns the block
// clockwise by 90k degrees, k = 4..7 mirrors left-right after turning by
// 90(k-4) degrees.
__host__ __device__ inline void iso_src(int B, int k, int i, int j, int* si, int* sj) {
  const int m = B - 1;
  int jj = (k & 4) ? m - j : j;       // mirror acts on the turned block
  switch (k & 3) {
    case 0: *si = i;      *sj = jj;     break;
    case 1: *si = m - jj; *sj = i;      break;  // top row -> right column
    case 2: *si = m - i;  *sj = m - jj; break;
    default: *si = jj;    *sj = m - i;  break;  // top row -> left column
  }
}

}  // namespace fic

#define FIC_CUDA_TRY(expr)                                   \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return ::fic::cuda_status(_e);    \
  } while (0)

namespace fic {
inline int cuda_status(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? FIC_ENOMEM : FIC_ECUDA;
}
}  // namespace fic
