/*
 * fic_oracle.c -- plain CPU oracle of the fractal encoder (test
 * infrastructure only: the tests, the smoke check and the benchmark's
 * CPU-baseline leg call it; the CUDA path never does).
 *
 * Written from the paper's definitions, looped the obvious way:
 *   - Sec. 2: non-overlapping B x B range blocks; the domain pool is every
 *     2B x 2B square at integer step L; a domain is decimated to B x B
 *     (Eq. 1's D); the pool is extended by the 4 clockwise rotations and
 *     their mirrors; the best domain minimises E of Eq. 1 with o from Eq. 3;
 *     ranges whose best error is not acceptable are split into four and
 *     matched again (16 -> 8 -> 4 -> 2).
 *   - Sec. 3, Eq. 4-5: block entropy; only domains whose entropy is greater
 *     than a threshold stay in the pool.
 *   - Sec. 3.1: predefined s per step: {0.1}, {0.2, 0.4}, {0.3, 0.8},
 *     {0.5, 0.9}.
 *
 * Readings of what the paper leaves open (each also listed in the design
 * notes of the repository):
 *   - decimation is the 2x2 mean; it is carried as the integer 2x2 sum Ds
 *     and E is scaled so that every quantity stays an exact integer;
 *   - the entropy block is the original 2B x 2B domain, 256 grey levels,
 *     probabilities q / (4 B^2); the filter compares the fixed-point key
 *     sum_q round(q ln q 2^32) so that equal histograms give equal keys;
 *   - the threshold is the pool's entropy percentile:
 *     thr = H_sorted_ascending[floor(p (P - 1))], keep H > thr; if that keeps
 *     nothing, keep H >= thr;
 *   - a pool size K (Tables 1-2) keeps the K highest entropies: thr = the
 *     (K+1)-th highest entropy, keep H > thr (ties at thr dropped); K >= P
 *     keeps the whole pool;
 *   - isometry k = 0..3 rotates clockwise by 90k degrees; k = 4..7 mirrors
 *     left-right after rotation k - 4;
 *   - the grid S set is k / (M - 1), k = 0..M-1; s is never negative and o
 *     is not clamped or quantised;
 *   - ties are broken by the lowest key (dom_index * 8 + iso) * |S| + s_idx,
 *     dom_index being the raster index in the unfiltered pool;
 *   - a range is accepted when E <= n T^2 (compared in double as
 *     (double) e_num / (16 q^2 n^2) <= n * (T * T)); the last level and the
 *     single-level mode accept every range;
 *   - decoding starts from a flat 128 image and iterates all codes at once
 *     (Jacobi) in double, clamping to [0, 255], until max |delta| < tol.
 *
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include "fic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define KEY_SCALE 4294967296.0L /* 2^32 */

/* ------------------------------------------------------------------------ */
/* Sec. 3, Eq. 4-5: entropy                                                  */
/* ------------------------------------------------------------------------ */

static void block_histogram(const uint8_t* img, long pitch, int x, int y, int size,
                            long hist[256]) {
  memset(hist, 0, 256 * sizeof(long));
  for (int i = 0; i < size; ++i)
    for (int j = 0; j < size; ++j) hist[img[(long)(y + i) * pitch + (x + j)]]++;
}

double oracle_entropy(const uint8_t* img, long pitch, int x, int y, int size) {
  long hist[256];
  block_histogram(img, pitch, x, y, size, hist);
  long double total = (long double)size * (long double)size; /* Eq. 4 denominator */
  long double h = 0.0L;
  for (int v = 0; v < 256; ++v) {
    if (hist[v] == 0) continue;
    long double p = (long double)hist[v] / total; /* Eq. 4 */
    h -= p * logl(p);                             /* Eq. 5 */
  }
  return (double)h;
}

void oracle_key_table(int64_t* table, int qmax) {
  table[0] = 0;
  for (int q = 1; q <= qmax; ++q) {
    long double v = (long double)q * logl((long double)q) * KEY_SCALE;
    table[q] = (int64_t)llroundl(v);
  }
}

int64_t oracle_entropy_key(const uint8_t* img, long pitch, int x, int y, int size) {
  long hist[256];
  block_histogram(img, pitch, x, y, size, hist);
  int64_t key = 0;
  for (int v = 0; v < 256; ++v) {
    if (hist[v] == 0) continue;
    long double t = (long double)hist[v] * logl((long double)hist[v]) * KEY_SCALE;
    key += (int64_t)llroundl(t);
  }
  return key;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2: domain pool and its entropy filter (Sec. 3)                       */
/* ------------------------------------------------------------------------ */

int oracle_pool_size(int W, int H, int B, int L, int* px, int* py) {
  if (L < 1 || W < 2 * B || H < 2 * B) {
    if (px) *px = 0;
    if (py) *py = 0;
    return 0;
  }
  int nx = (W - 2 * B) / L + 1;
  int ny = (H - 2 * B) / L + 1;
  if (px) *px = nx;
  if (py) *py = ny;
  return nx * ny;
}

static int cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

int oracle_pool_filter(const uint8_t* img, long pitch, int W, int H, int B, int L,
                       double percentile, int pool_size, int64_t* keys, int32_t* kept,
                       int64_t* thr_key, int* fallback) {
  int nx, ny;
  int P = oracle_pool_size(W, H, B, L, &nx, &ny);
  if (P <= 0) return 0;
  /* each position's key on its own (rows spread over the host's threads;
   * every key is computed alone, in the same operations, in any order) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int iy = 0; iy < ny; ++iy)
    for (int ix = 0; ix < nx; ++ix)
      keys[iy * nx + ix] = oracle_entropy_key(img, pitch, ix * L, iy * L, 2 * B);

  /* Percentile of the entropies: the entropy-ascending order is the
   * key-descending order, so H_sorted[i] is the key at ascending index
   * P - 1 - i. */
  int64_t* sorted = (int64_t*)malloc(sizeof(int64_t) * (size_t)P);
  memcpy(sorted, keys, sizeof(int64_t) * (size_t)P);
  qsort(sorted, (size_t)P, sizeof(int64_t), cmp_i64);
  long rank;  /* ascending key rank of the threshold */
  int keep_all = 0;
  if (pool_size > 0) {
    /* Tables 1-2's pool size K: the K highest entropies are the K lowest
     * keys, all below the key of ascending rank K */
    rank = pool_size < P ? pool_size : P - 1;
    keep_all = pool_size >= P;
  } else {
    long i_h = (long)floor(percentile * (double)(P - 1));
    if (i_h < 0) i_h = 0;
    if (i_h > P - 1) i_h = P - 1;
    rank = P - 1 - i_h;
  }
  int64_t thr = sorted[rank];
  free(sorted);

  /* Keep entropy > threshold, i.e. key < thr_key. */
  int n = 0;
  if (!keep_all)
    for (int d = 0; d < P; ++d)
      if (keys[d] < thr) kept[n++] = d;
  int fb = 0;
  if (n == 0) { /* nothing strictly above (or K >= P): keep H >= thr */
    fb = 1;
    for (int d = 0; d < P; ++d)
      if (keys[d] <= thr) kept[n++] = d;
  }
  if (thr_key) *thr_key = thr;
  if (fallback) *fallback = fb;
  return n;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2: decimation, isometries and the distance of Eq. 1                  */
/* ------------------------------------------------------------------------ */

void oracle_decimate(const uint8_t* img, long pitch, int x, int y, int B, int64_t* Ds) {
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) {
      const uint8_t* p = img + (long)(y + 2 * i) * pitch + (x + 2 * j);
      Ds[i * B + j] = (int64_t)p[0] + p[1] + p[pitch] + p[pitch + 1];
    }
}

/* Source pixel of T_k's output pixel (i, j). */
static void iso_source(int B, int k, int i, int j, int* si, int* sj) {
  if (k >= 4) j = B - 1 - j; /* mirror left-right after the rotation */
  switch (k & 3) {
    case 0: *si = i; *sj = j; break;                 /* identity          */
    case 1: *si = B - 1 - j; *sj = i; break;         /* 90 deg clockwise  */
    case 2: *si = B - 1 - i; *sj = B - 1 - j; break; /* 180 deg           */
    default: *si = j; *sj = B - 1 - i; break;        /* 270 deg clockwise */
  }
}

void oracle_isometry(const int64_t* src, int B, int k, int64_t* dst) {
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) {
      int si, sj;
      iso_source(B, k, i, j, &si, &sj);
      dst[i * B + j] = src[si * B + sj];
    }
}

/* Eq. 1 with d_i = Ds_i / 4, s = p / q and Eq. 3's o = Rbar - s Dbar.
 * Multiplying each term by 4 q n gives the integer
 *   p n Ds_i + 4 q Sr - p Sd - 4 q n r_i,
 * so 16 q^2 n^2 E is a sum of integer squares. */
int64_t oracle_error_num(const int64_t* R, const int64_t* Ds, int n, int p, int q) {
  int64_t Sr = 0, Sd = 0;
  for (int i = 0; i < n; ++i) {
    Sr += R[i];
    Sd += Ds[i];
  }
  __int128 acc = 0;
  for (int i = 0; i < n; ++i) {
    int64_t t = (int64_t)p * n * Ds[i] + 4LL * q * Sr - (int64_t)p * Sd - 4LL * q * n * R[i];
    acc += (__int128)t * t;
  }
  if (acc > (__int128)INT64_MAX) return INT64_MAX;
  return (int64_t)acc;
}

/* Eq. 1 / Eq. 3 of maps chosen elsewhere: each map on its own, with the
 * functions above (decimation, isometry, error numerator). */
void oracle_map_numerators(const uint8_t* img, long pitch, int n_maps, const int32_t* x,
                           const int32_t* y, const int32_t* size, const int32_t* dom_x,
                           const int32_t* dom_y, const int32_t* iso, const int32_t* p,
                           const int32_t* q, int n_threads, int64_t* e_num, int64_t* o_num) {
  if (n_threads < 1) n_threads = 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(n_threads)
#endif
  for (int m = 0; m < n_maps; ++m) {
    const int B = size[m], n = B * B;
    int64_t R[256], Ds[256], T[256];
    for (int i = 0; i < B; ++i)
      for (int j = 0; j < B; ++j) R[i * B + j] = img[(long)(y[m] + i) * pitch + x[m] + j];
    oracle_decimate(img, pitch, dom_x[m], dom_y[m], B, Ds);
    oracle_isometry(Ds, B, iso[m], T);
    e_num[m] = oracle_error_num(R, T, n, p[m], q[m]);
    int64_t Sr = 0, St = 0;
    for (int i = 0; i < n; ++i) {
      Sr += R[i];
      St += T[i];
    }
    o_num[m] = 4LL * q[m] * Sr - (int64_t)p[m] * St;
  }
}

void oracle_error_num128(const int64_t* R, const int64_t* Ds, int n, int64_t p, int64_t q,
                         uint64_t* out) {
  int64_t Sr = 0, Sd = 0;
  for (int i = 0; i < n; ++i) {
    Sr += R[i];
    Sd += Ds[i];
  }
  /* each term is 4 q n times a residual of magnitude <= 510: below 2^57 for
   * q <= 2^37 and n <= 256, so the sum of n squares stays below 2^128 */
  unsigned __int128 acc = 0;
  for (int i = 0; i < n; ++i) {
    int64_t t = p * n * Ds[i] + 4 * q * Sr - p * Sd - 4 * q * n * R[i];
    unsigned __int128 a = (unsigned __int128)(t < 0 ? -t : t);
    acc += a * a;
  }
  out[0] = (uint64_t)acc;
  out[1] = (uint64_t)(acc >> 64);
}

/* Eq. 2 with d = Ds / 4:
 *   s = (n sum r d - sum r sum d) / (n sum d^2 - (sum d)^2)
 *     = 4 (n sum r Ds - sum r sum Ds) / (n sum Ds^2 - (sum Ds)^2). */
void oracle_s_exact(const int64_t* R, const int64_t* Ds, int n, int64_t* s_num, int64_t* s_den) {
  int64_t Sr = 0, Sd = 0, Srd = 0, Sdd = 0;
  for (int i = 0; i < n; ++i) {
    Sr += R[i];
    Sd += Ds[i];
    Srd += R[i] * Ds[i];
    Sdd += Ds[i] * Ds[i];
  }
  const int64_t C = (int64_t)n * Srd - Sr * Sd;
  const int64_t V = (int64_t)n * Sdd - Sd * Sd;
  if (V <= 0 || C <= 0) { /* flat block, or the best s in [0, 1] is 0 */
    *s_num = 0;
    *s_den = 1;
  } else if (4 * C >= V) { /* s >= 1: clamped */
    *s_num = 1;
    *s_den = 1;
  } else {
    *s_num = 4 * C;
    *s_den = V;
  }
}

void oracle_mul_u128(uint64_t a_lo, uint64_t a_hi, uint64_t b_lo, uint64_t b_hi, uint64_t* out) {
  const unsigned __int128 p00 = (unsigned __int128)a_lo * b_lo;
  const unsigned __int128 p01 = (unsigned __int128)a_lo * b_hi;
  const unsigned __int128 p10 = (unsigned __int128)a_hi * b_lo;
  const unsigned __int128 p11 = (unsigned __int128)a_hi * b_hi;
  const unsigned __int128 mid = (p00 >> 64) + (uint64_t)p01 + (uint64_t)p10;
  const unsigned __int128 hi = (mid >> 64) + (p01 >> 64) + (p10 >> 64) + (uint64_t)p11;
  out[0] = (uint64_t)p00;
  out[1] = (uint64_t)mid;
  out[2] = (uint64_t)hi;
  out[3] = (uint64_t)(hi >> 64) + (uint64_t)(p11 >> 64);
}

/* sign of a_num / a_den^2 - b_num / b_den^2 (all non-negative, den > 0) */
static int cmp_ratio(unsigned __int128 a_num, int64_t a_den, unsigned __int128 b_num,
                     int64_t b_den) {
  const unsigned __int128 a2 = (unsigned __int128)a_den * (unsigned __int128)a_den;
  const unsigned __int128 b2 = (unsigned __int128)b_den * (unsigned __int128)b_den;
  uint64_t x[4], y[4];
  oracle_mul_u128((uint64_t)a_num, (uint64_t)(a_num >> 64), (uint64_t)b2, (uint64_t)(b2 >> 64), x);
  oracle_mul_u128((uint64_t)b_num, (uint64_t)(b_num >> 64), (uint64_t)a2, (uint64_t)(a2 >> 64), y);
  for (int i = 3; i >= 0; --i)
    if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
  return 0;
}

double oracle_error_direct(const int64_t* R, const int64_t* Ds, int n, int p, int q) {
  long double s = (long double)p / (long double)q;
  long double rbar = 0.0L, dbar = 0.0L;
  for (int i = 0; i < n; ++i) {
    rbar += (long double)R[i];
    dbar += (long double)Ds[i] / 4.0L;
  }
  rbar /= n;
  dbar /= n;
  long double o = rbar - s * dbar; /* Eq. 3 */
  long double e = 0.0L;
  for (int i = 0; i < n; ++i) {
    long double t = s * ((long double)Ds[i] / 4.0L) + o - (long double)R[i];
    e += t * t; /* Eq. 1 */
  }
  return (double)e;
}

int oracle_s_set(int s_mode, int grid_samples, int B, int32_t* p, int32_t* q) {
  if (s_mode == ORACLE_S_GRID) {
    if (grid_samples < 2) return 0;
    for (int k = 0; k < grid_samples; ++k) p[k] = k;
    *q = grid_samples - 1;
    return grid_samples;
  }
  /* Sec. 3.1: step 1 (16x16) {0.1}, step 2 (8x8) {0.2, 0.4},
   * step 3 (4x4) {0.3, 0.8}, step 4 (2x2) {0.5, 0.9}. */
  *q = 10;
  switch (B) {
    case 16: p[0] = 1; return 1;
    case 8: p[0] = 2; p[1] = 4; return 2;
    case 4: p[0] = 3; p[1] = 8; return 2;
    case 2: p[0] = 5; p[1] = 9; return 2;
    default: return 0;
  }
}

/* ------------------------------------------------------------------------ */
/* Exhaustive matching (Sec. 2)                                              */
/* ------------------------------------------------------------------------ */

void oracle_match(const uint8_t* img, long pitch, int W, int H, int B, int L,
                  const int32_t* kept, int n_kept, const int32_t* range_xy,
                  int n_ranges, const int32_t* s_p, int n_s, int q, int n_threads,
                  oracle_match_result* out) {
  int nx, ny;
  oracle_pool_size(W, H, B, L, &nx, &ny);
  const int n = B * B;
  /* Decimated kept domains, computed once (each on its own). */
  int64_t* Dall = (int64_t*)malloc(sizeof(int64_t) * (size_t)n * (size_t)(n_kept > 0 ? n_kept : 1));
  if (n_threads < 1) n_threads = 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(n_threads)
#endif
  for (int j = 0; j < n_kept; ++j) {
    int d = kept[j];
    oracle_decimate(img, pitch, (d % nx) * L, (d / nx) * L, B, Dall + (size_t)j * n);
  }
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
  for (int r = 0; r < n_ranges; ++r) {
    int64_t R[256], T[256];
    int rx = range_xy[2 * r], ry = range_xy[2 * r + 1];
    for (int i = 0; i < B; ++i)
      for (int jj = 0; jj < B; ++jj) R[i * B + jj] = img[(long)(ry + i) * pitch + rx + jj];
    oracle_match_result best;
    best.e_num = INT64_MAX;
    best.key = INT64_MAX;
    best.dom_index = -1;
    best.iso = -1;
    best.s_idx = -1;
    best.pad = 0;
    for (int j = 0; j < n_kept; ++j) {
      const int64_t* Ds = Dall + (size_t)j * n;
      for (int k = 0; k < 8; ++k) {
        oracle_isometry(Ds, B, k, T);
        for (int si = 0; si < n_s; ++si) {
          int64_t e = oracle_error_num(R, T, n, s_p[si], q);
          /* candidates arrive in increasing key order: strict < keeps the
           * lowest key among equal errors */
          if (e < best.e_num) {
            best.e_num = e;
            best.key = ((int64_t)kept[j] * 8 + k) * n_s + si;
            best.dom_index = kept[j];
            best.iso = k;
            best.s_idx = si;
          }
        }
      }
    }
    out[r] = best;
  }
  free(Dall);
}

void oracle_match_exact(const uint8_t* img, long pitch, int W, int H, int B, int L,
                        const int32_t* kept, int n_kept, const int32_t* range_xy, int n_ranges,
                        int n_threads, oracle_match_exact_result* out) {
  int nx, ny;
  oracle_pool_size(W, H, B, L, &nx, &ny);
  const int n = B * B;
  int64_t* Dall = (int64_t*)malloc(sizeof(int64_t) * (size_t)n * (size_t)(n_kept > 0 ? n_kept : 1));
  for (int j = 0; j < n_kept; ++j) {
    int d = kept[j];
    oracle_decimate(img, pitch, (d % nx) * L, (d / nx) * L, B, Dall + (size_t)j * n);
  }
  if (n_threads < 1) n_threads = 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
  for (int r = 0; r < n_ranges; ++r) {
    int64_t R[256], T[256];
    int rx = range_xy[2 * r], ry = range_xy[2 * r + 1];
    for (int i = 0; i < B; ++i)
      for (int jj = 0; jj < B; ++jj) R[i * B + jj] = img[(long)(ry + i) * pitch + rx + jj];
    oracle_match_exact_result best;
    memset(&best, 0, sizeof(best));
    best.key = INT64_MAX;
    best.dom_index = -1;
    best.iso = -1;
    unsigned __int128 best_num = 0;
    for (int j = 0; j < n_kept; ++j) {
      const int64_t* Ds = Dall + (size_t)j * n;
      for (int k = 0; k < 8; ++k) {
        oracle_isometry(Ds, B, k, T);
        int64_t sn, sd;
        oracle_s_exact(R, T, n, &sn, &sd);      /* Eq. 2 */
        uint64_t e2[2];
        oracle_error_num128(R, T, n, sn, sd, e2); /* Eq. 1 with Eq. 3's o */
        const unsigned __int128 num = ((unsigned __int128)e2[1] << 64) | e2[0];
        /* candidates arrive in increasing key order: strictly smaller E wins */
        if (best.dom_index < 0 || cmp_ratio(num, sd, best_num, best.s_den) < 0) {
          best_num = num;
          best.key = (int64_t)kept[j] * 8 + k;
          best.s_num = sn;
          best.s_den = sd;
          best.dom_index = kept[j];
          best.iso = k;
          best.e_lo = e2[0];
          best.e_hi = e2[1];
        }
      }
    }
    out[r] = best;
  }
  free(Dall);
}

/* E in the moment form n E = A - G of the exact-s search, as the encoder
 * reports it: with A = n sum r^2 - (sum r)^2 and the pair's C, V,
 *   s = 0: A / n;   s = 1: (16 A - 8 C + V) / (16 n);   else (A - C C / V) / n,
 * each operation in double in this order (the same value as Eq. 1's E up to
 * rounding; the tests bound the difference). */
static double exact_s_error(const int64_t* R, const int64_t* Ds, int n, int64_t s_num,
                            int64_t s_den) {
  int64_t Sr = 0, Srr = 0, Sd = 0, Srd = 0, Sdd = 0;
  for (int i = 0; i < n; ++i) {
    Sr += R[i];
    Srr += R[i] * R[i];
    Sd += Ds[i];
    Srd += R[i] * Ds[i];
    Sdd += Ds[i] * Ds[i];
  }
  const int64_t A = (int64_t)n * Srr - Sr * Sr;
  const int64_t C = (int64_t)n * Srd - Sr * Sd;
  const int64_t V = (int64_t)n * Sdd - Sd * Sd;
  if (s_num == 0) return (double)A / (double)n;
  if (s_num == s_den) return (double)(16 * A - 8 * C + V) / (16.0 * (double)n);
  const double g = ((double)C * (double)C) / (double)V;
  return ((double)A - g) / (double)n;
}

/* ------------------------------------------------------------------------ */
/* Quadtree encoder (Sec. 2) and decoder                                     */
/* ------------------------------------------------------------------------ */

int oracle_encode(const uint8_t* img, long pitch, int W, int H, const oracle_params* prm,
                  oracle_code* codes, int cap, oracle_level_stats* stats) {
  const int B0 = prm->range_size0;
  if (B0 != 2 && B0 != 4 && B0 != 8 && B0 != 16) return -2;
  if (prm->n_levels < 1 || (B0 >> (prm->n_levels - 1)) < 2) return -2;
  if (W % B0 || H % B0 || W < 2 * B0 || H < 2 * B0 || prm->domain_step < 1) return -2;
  const int L = prm->domain_step;

  int n_active = (W / B0) * (H / B0);
  int32_t* active = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)W * H);
  int32_t* next = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)W * H);
  for (int by = 0; by < H / B0; ++by)
    for (int bx = 0; bx < W / B0; ++bx) {
      int r = by * (W / B0) + bx;
      active[2 * r] = bx * B0;
      active[2 * r + 1] = by * B0;
    }

  int n_codes = 0, overflow = 0;
  const int n_lv = prm->single_level ? 1 : prm->n_levels;
  for (int lv = 0; lv < n_lv; ++lv) {
    const int B = B0 >> lv;
    const int n = B * B;
    int nx, ny;
    int P = oracle_pool_size(W, H, B, L, &nx, &ny);
    int64_t* keys = (int64_t*)malloc(sizeof(int64_t) * (size_t)P);
    int32_t* kept = (int32_t*)malloc(sizeof(int32_t) * (size_t)P);
    int64_t thr;
    int fb;
    int n_kept = oracle_pool_filter(img, pitch, W, H, B, L, prm->entropy_percentile,
                                    prm->pool_size, keys, kept, &thr, &fb);
    int32_t sp[64], q = 1;
    const int exact = prm->s_mode == ORACLE_S_EXACT;
    int n_s = exact ? 1 : oracle_s_set(prm->s_mode, prm->grid_samples, B, sp, &q);
    oracle_match_result* res =
        (oracle_match_result*)malloc(sizeof(oracle_match_result) * (size_t)(n_active > 0 ? n_active : 1));
    oracle_match_exact_result* rex = NULL;
    if (exact) {
      rex = (oracle_match_exact_result*)malloc(sizeof(oracle_match_exact_result) *
                                               (size_t)(n_active > 0 ? n_active : 1));
      oracle_match_exact(img, pitch, W, H, B, L, kept, n_kept, active, n_active, prm->n_threads,
                         rex);
      for (int r = 0; r < n_active; ++r) {
        res[r].e_num = 0;
        res[r].key = rex[r].key;
        res[r].dom_index = rex[r].dom_index;
        res[r].iso = rex[r].iso;
        res[r].s_idx = 0;
        res[r].pad = 0;
      }
    } else {
      oracle_match(img, pitch, W, H, B, L, kept, n_kept, active, n_active, sp, n_s, q,
                   prm->n_threads, res);
    }

    const int last = (lv == n_lv - 1) || prm->single_level;
    const double den = 16.0 * q * q * (double)n * (double)n;
    const double e_thr = (double)n * (prm->rms_threshold * prm->rms_threshold);
    int n_next = 0, n_acc = 0;
    for (int r = 0; r < n_active; ++r) {
      int rx = active[2 * r], ry = active[2 * r + 1];
      double e = (double)res[r].e_num / den;
      int64_t Rb[256], Tb[256];
      if (exact) { /* E of the chosen pair in the moment form */
        int d = res[r].dom_index;
        int64_t Dd[256];
        for (int i = 0; i < B; ++i)
          for (int j = 0; j < B; ++j) Rb[i * B + j] = img[(long)(ry + i) * pitch + rx + j];
        oracle_decimate(img, pitch, (d % nx) * L, (d / nx) * L, B, Dd);
        oracle_isometry(Dd, B, res[r].iso, Tb);
        e = exact_s_error(Rb, Tb, n, rex[r].s_num, rex[r].s_den);
      }
      if (last || e <= e_thr) {
        n_acc++;
        if (n_codes >= cap) {
          overflow = 1;
          continue;
        }
        oracle_code* c = &codes[n_codes++];
        memset(c, 0, sizeof(*c));
        int d = res[r].dom_index;
        int64_t Sr = 0, Sd = 0, Ds[256];
        for (int i = 0; i < B; ++i)
          for (int j = 0; j < B; ++j) Sr += img[(long)(ry + i) * pitch + rx + j];
        oracle_decimate(img, pitch, (d % nx) * L, (d / nx) * L, B, Ds);
        for (int i = 0; i < n; ++i) Sd += Ds[i];
        int p = exact ? 0 : sp[res[r].s_idx];
        c->level = lv;
        c->x = rx;
        c->y = ry;
        c->size = B;
        c->dom_index = d;
        c->dom_x = (d % nx) * L;
        c->dom_y = (d / nx) * L;
        c->iso = res[r].iso;
        c->s_idx = res[r].s_idx;
        c->e = e;
        if (exact) {
          /* Eq. 3 with s = s_num / s_den: o = (4 s_den Sr - s_num Sd) / (4 s_den n) */
          c->p = c->q = 0;
          c->e_num = 0;
          c->o_num = 0;
          c->s_num = rex[r].s_num;
          c->s_den = rex[r].s_den;
          c->s = (double)c->s_num / (double)c->s_den;
          c->o = (double)(4 * c->s_den * Sr - c->s_num * Sd) / (4.0 * (double)c->s_den * (double)n);
        } else {
          c->p = p;
          c->q = q;
          c->e_num = res[r].e_num;
          c->s_num = p;
          c->s_den = q;
          c->s = (double)p / (double)q;
          /* Eq. 3: o = Sr / n - (p / q) Sd / (4 n) = (4 q Sr - p Sd) / (4 q n) */
          c->o_num = 4LL * q * Sr - (int64_t)p * Sd;
          c->o = (double)c->o_num / (4.0 * q * (double)n);
        }
      } else {
        int h = B / 2;
        int32_t* o = next + 2 * (size_t)n_next;
        o[0] = rx;     o[1] = ry;
        o[2] = rx + h; o[3] = ry;
        o[4] = rx;     o[5] = ry + h;
        o[6] = rx + h; o[7] = ry + h;
        n_next += 4;
      }
    }
    if (stats) {
      stats[lv].size = B;
      stats[lv].pool_size = P;
      stats[lv].n_kept = n_kept;
      stats[lv].fallback = fb;
      stats[lv].thr_key = thr;
      stats[lv].n_active = n_active;
      stats[lv].n_accepted = n_acc;
      stats[lv].matches = (double)n_active * (double)n_kept * 8.0;
    }
    free(res);
    free(rex);
    free(keys);
    free(kept);
    int32_t* t = active;
    active = next;
    next = t;
    n_active = n_next;
  }
  free(active);
  free(next);
  return overflow ? -1 : n_codes;
}

/* ------------------------------------------------------------------------ */
/* Stored form: quantised o and the bit count (readings in the header)       */
/* ------------------------------------------------------------------------ */

void oracle_quantize_o(oracle_code* codes, int n_codes, int o_bits) {
  const double levels = (double)((1L << o_bits) - 1);
  const double step = 510.0 / levels;
  for (int c = 0; c < n_codes; ++c) {
    double u = nearbyint((codes[c].o + 255.0) / step); /* default mode: half to even */
    if (u < 0.0) u = 0.0;
    if (u > levels) u = levels;
    codes[c].o = u * step - 255.0;
  }
}

static int ceil_log2(int64_t v) {
  int b = 0;
  while (((int64_t)1 << b) < v) ++b;
  return b;
}

int64_t oracle_code_bits(const oracle_level_stats* stats, int n_levels, const int* n_s,
                         int o_bits) {
  int64_t bits = 0;
  for (int l = 0; l < n_levels; ++l) {
    if (l < n_levels - 1) bits += stats[l].n_active; /* kept or split */
    bits += (int64_t)stats[l].n_accepted *
            (ceil_log2(stats[l].pool_size) + 3 + ceil_log2(n_s[l]) + o_bits);
  }
  return bits;
}

int oracle_decode(const oracle_code* codes, int n_codes, int W, int H, int max_iters,
                  double tol, double* out) {
  double* cur = out;
  double* nxt = (double*)malloc(sizeof(double) * (size_t)W * H);
  for (long i = 0; i < (long)W * H; ++i) cur[i] = 128.0;
  int it = 0;
  while (it < max_iters) {
    ++it;
    for (int c = 0; c < n_codes; ++c) {
      const oracle_code* k = &codes[c];
      const int B = k->size;
      const double s = k->s; /* p / q, or Eq. 2's s in the exact-s mode */
      for (int i = 0; i < B; ++i)
        for (int j = 0; j < B; ++j) {
          int si, sj;
          iso_source(B, k->iso, i, j, &si, &sj);
          const double* d = cur + (long)(k->dom_y + 2 * si) * W + (k->dom_x + 2 * sj);
          double t = (((d[0] + d[1]) + d[W]) + d[W + 1]) * 0.25;
          double v = s * t + k->o;
          if (v < 0.0) v = 0.0;
          if (v > 255.0) v = 255.0;
          nxt[(long)(k->y + i) * W + (k->x + j)] = v;
        }
    }
    double delta = 0.0;
    for (long i = 0; i < (long)W * H; ++i) {
      double a = fabs(nxt[i] - cur[i]);
      if (a > delta) delta = a;
    }
    memcpy(cur, nxt, sizeof(double) * (size_t)W * H);
    if (delta < tol) break;
  }
  free(nxt);
  return it;
}
