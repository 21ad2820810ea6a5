/*
 * fic_oracle.h -- plain, slow CPU oracle of the fractal encoder's matching
 * search (test infrastructure only).
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may call this library.  It shares no code with the CUDA path.
 *
 * Everything follows "A Fast Fractal Image Compression Algorithm Using
 * Predefined Values for Contrast Scaling" (Miar Naimi, Salarian):
 *   Sec. 2     range partition, domain pool (2B x 2B squares at step L),
 *              the 8 isometries, the distance of Eq. 1, s and o of Eq. 2-3,
 *              the quadtree split 16 -> 8 -> 4 -> 2.
 *   Sec. 3     block entropy (Eq. 4-5) and the "entropy greater than a
 *              threshold" pool filter.
 *   Sec. 3.1   the predefined contrast-scaling sets per step.
 * Readings of points the paper leaves open are stated beside each function.
 */
#ifndef FIC_ORACLE_H
#define FIC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* S-set selection. */
#define ORACLE_S_PREDEFINED 0 /* Sec. 3.1 per-step sets, denominators 10  */
#define ORACLE_S_GRID 1       /* k/(M-1), k = 0..M-1 (Sec. 2 "pre-sampled") */
#define ORACLE_S_EXACT 2      /* Eq. 2's s of every pair, clamped to [0, 1] */

typedef struct {
  int n_levels;              /* 1..4 */
  int range_size0;           /* B at the first level: 16, 8, 4 or 2      */
  int domain_step;           /* L >= 1                                    */
  double rms_threshold;      /* accept when E <= n * T^2                  */
  int single_level;          /* 1: accept every range at the first level  */
  int s_mode;                /* ORACLE_S_PREDEFINED | ORACLE_S_GRID       */
  int grid_samples;          /* M for ORACLE_S_GRID                       */
  double entropy_percentile; /* 0 <= p <= 1                               */
  int n_threads;             /* OpenMP threads for the range loop (>= 1)  */
  int pool_size;             /* K > 0: keep the K highest-entropy domains
                                (Tables 1-2 "pool size"); 0: percentile   */
} oracle_params;

/* One saved affine transformation (Sec. 2). */
typedef struct {
  int32_t level, x, y, size;   /* range block: top-left corner, side B    */
  int32_t dom_index;           /* raster index in the unfiltered pool     */
  int32_t dom_x, dom_y;        /* domain block top-left corner (2B x 2B)  */
  int32_t iso;                 /* isometry 0..7                           */
  int32_t s_idx, p, q;         /* s = p / q, s_idx its index in the set
                                  (exact-s mode: s_idx = p = q = 0)       */
  int32_t pad;
  int64_t e_num;               /* 16 q^2 n^2 E, exact (exact-s mode: 0)   */
  int64_t o_num;               /* 4 q n o, exact (exact-s mode: 0)        */
  double e;                    /* E = e_num / (16 q^2 n^2); exact-s mode:
                                  the moment form below                   */
  double s;                    /* p / q (exact-s mode: s_num / s_den)     */
  double o;                    /* o_num / (4 q n) (exact-s mode: with
                                  s_num, s_den in place of p, q)          */
  int64_t s_num, s_den;        /* s as an exact fraction (every mode)     */
} oracle_code;

typedef struct {
  int64_t e_num;               /* 16 q^2 n^2 E of the best candidate      */
  int64_t key;                 /* (dom_index * 8 + iso) * |S| + s_idx     */
  int32_t dom_index, iso, s_idx, pad;
} oracle_match_result;

typedef struct {
  int32_t size;                /* B                                       */
  int32_t pool_size;           /* P                                       */
  int32_t n_kept;
  int32_t fallback;            /* 1 when the strict filter kept nothing   */
  int64_t thr_key;
  int32_t n_active;            /* ranges matched at this level            */
  int32_t n_accepted;
  double matches;              /* n_active * n_kept * 8                   */
} oracle_level_stats;

/* Eq. 4-5: entropy (natural log) of the size x size block at (x, y). */
double oracle_entropy(const uint8_t* img, long pitch, int x, int y, int size);

/* Fixed-point entropy key of the same block: sum over grey levels of
 * round(q ln q * 2^32), q the level's count.  H = ln(N) - key / (N 2^32), so
 * a larger key means a lower entropy. */
int64_t oracle_entropy_key(const uint8_t* img, long pitch, int x, int y, int size);

/* table[q] = round(q ln q * 2^32), q = 0..qmax. */
void oracle_key_table(int64_t* table, int qmax);

/* Number of pool positions for block size B and step L (Sec. 2). */
int oracle_pool_size(int W, int H, int B, int L, int* px, int* py);

/* Entropy keys of every pool position (raster order), the threshold and the
 * kept list (ascending raster index).  pool_size K > 0 keeps the K highest
 * entropies (threshold = the key of ascending rank min(K, P - 1), keep
 * key < threshold; K >= P keeps the whole pool); pool_size 0 uses the
 * percentile.  Returns n_kept. */
int oracle_pool_filter(const uint8_t* img, long pitch, int W, int H, int B, int L,
                       double percentile, int pool_size, int64_t* keys, int32_t* kept,
                       int64_t* thr_key, int* fallback);

/* 2x2 sums of the 2B x 2B block at (x, y): Ds[i*B+j] (Eq. 1's decimated
 * block is Ds / 4). */
void oracle_decimate(const uint8_t* img, long pitch, int x, int y, int B, int64_t* Ds);

/* dst = T_k(src) for a B x B block, k = 0..7 (Sec. 2). */
void oracle_isometry(const int64_t* src, int B, int k, int64_t* dst);

/* 16 q^2 n^2 E(R, D) of Eq. 1 with s = p/q and o from Eq. 3, computed term
 * by term in exact integers.  R: range pixels; D: decimated sums Ds (already
 * transformed); n = B*B. */
int64_t oracle_error_num(const int64_t* R, const int64_t* Ds, int n, int p, int q);

/* Eq. 1 evaluated in long double with s = p/q and o = Rbar - s Dbar. */
double oracle_error_direct(const int64_t* R, const int64_t* Ds, int n, int p, int q);

/* S set of a level: fills p[] and *q, returns |S|. */
int oracle_s_set(int s_mode, int grid_samples, int B, int32_t* p, int32_t* q);

/* Best (domain, isometry, s) for each listed range (x, y at size B) against
 * the kept pool, exhaustive over the definition (Sec. 2). */
void oracle_match(const uint8_t* img, long pitch, int W, int H, int B, int L,
                  const int32_t* kept, int n_kept, const int32_t* range_xy,
                  int n_ranges, const int32_t* s_p, int n_s, int q, int n_threads,
                  oracle_match_result* out);

/* Eq. 1 and Eq. 3 of given maps, whatever chose them: map i takes the
 * size[i] x size[i] range at (x[i], y[i]), the domain whose 2x2-sum
 * decimation starts at (dom_x[i], dom_y[i]), isometry iso[i] and s =
 * p[i] / q[i]; e_num[i] = 16 q^2 n^2 E (oracle_error_num on the range and the
 * transformed decimated domain T) and o_num[i] = 4 q n o = 4 q sum R -
 * p sum T.  The maps are independent (OpenMP over n_threads). */
void oracle_map_numerators(const uint8_t* img, long pitch, int n_maps, const int32_t* x,
                           const int32_t* y, const int32_t* size, const int32_t* dom_x,
                           const int32_t* dom_y, const int32_t* iso, const int32_t* p,
                           const int32_t* q, int n_threads, int64_t* e_num, int64_t* o_num);

/* 16 q^2 n^2 E of Eq. 1 as oracle_error_num, for 64-bit p and q and as an
 * unsigned 128-bit integer (out[0] = low, out[1] = high 64 bits). */
void oracle_error_num128(const int64_t* R, const int64_t* Ds, int n, int64_t p, int64_t q,
                         uint64_t* out);
/* Eq. 2's least-squares s of a range R and a (transformed) decimated block
 * d = Ds / 4: s = (n sum r d - sum r sum d) / (n sum d^2 - (sum d)^2), in
 * integer moments 4C / V with C = n sum r Ds - sum r sum Ds and
 * V = n sum Ds^2 - (sum Ds)^2.  Reading: s stays in [0, 1] (clamped), and a
 * flat block (V = 0) takes s = 0.  Returned as *s_num / *s_den. */
void oracle_s_exact(const int64_t* R, const int64_t* Ds, int n, int64_t* s_num, int64_t* s_den);
/* a * b of two unsigned 128-bit integers as four 64-bit limbs, low first
 * (the products of the exact-s comparisons). */
void oracle_mul_u128(uint64_t a_lo, uint64_t a_hi, uint64_t b_lo, uint64_t b_hi, uint64_t* out);
typedef struct {
  int64_t key;                 /* dom_index * 8 + iso                     */
  int64_t s_num, s_den;        /* the pair's s (oracle_s_exact)           */
  int32_t dom_index, iso;
  double e;                    /* E, the moment form (oracle_encode)      */
  uint64_t e_lo, e_hi;         /* 16 s_den^2 n^2 E, exact (Eq. 1)         */
} oracle_match_exact_result;
/* The exact-s search: for each listed range, the (domain, isometry) whose
 * Eq. 1 error at its own Eq. 2 s (oracle_s_exact) and Eq. 3 o is smallest,
 * compared exactly (E_a < E_b iff num_a den_b^2 < num_b den_a^2, 256-bit
 * products); ties go to the lowest key dom_index * 8 + iso. */
void oracle_match_exact(const uint8_t* img, long pitch, int W, int H, int B, int L,
                        const int32_t* kept, int n_kept, const int32_t* range_xy, int n_ranges,
                        int n_threads, oracle_match_exact_result* out);
/* Full quadtree encoder.  Returns the number of codes (or -1 if cap is too
 * small, -2 on bad arguments).  stats has n_levels entries. */
int oracle_encode(const uint8_t* img, long pitch, int W, int H, const oracle_params* prm,
                  oracle_code* codes, int cap, oracle_level_stats* stats);

/* Stored form of the maps (the paper reports compression ratios but gives no
 * layout; this is the reading used here):
 *   - o is stored with `o_bits` bits, uniform over [-255, 255] (s is in
 *     [0, 1] and the means in [0, 255]): step = 510 / (2^o_bits - 1),
 *     o' = round((o + 255) / step) * step - 255 (round half to even);
 *   - every range of a level above the last costs one quadtree bit (kept or
 *     split); every saved map costs ceil(log2 P) bits of domain position
 *     (P = the level's pool positions, which a decoder can count),
 *     3 bits of isometry, ceil(log2 |S|) bits of s and o_bits bits of o.
 * oracle_quantize_o replaces each code's o by o'; oracle_code_bits returns
 * the total bits of an encode from its level statistics. */
void oracle_quantize_o(oracle_code* codes, int n_codes, int o_bits);
int64_t oracle_code_bits(const oracle_level_stats* stats, int n_levels, const int* n_s,
                         int o_bits);

/* Fixed-point decoder: Jacobi iteration from a flat 128 image, stopping
 * when max |delta| < tol or after max_iters.  out: W*H doubles.  Returns the
 * number of iterations done. */
int oracle_decode(const oracle_code* codes, int n_codes, int W, int H, int max_iters,
                  double tol, double* out);

#ifdef __cplusplus
}
#endif
#endif
