/*
 * CPU oracle for one Larger-than-Life (LTL) step -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library.  It shares no code, header or constant with the CUDA path.
 *
 * What it computes, straight from the definitions in the CAT paper
 * (Navarro et al., "CAT: Cellular Automata on Tensor cores", arXiv 2406.17284):
 *
 *  1. Box count (Sec. IV, Eqs. 1-2; the band product Pi*Lambda*Pi of ones
 *     reduces every cell's Moore neighbourhood of radius r):
 *        L(y,x) = sum_{dy=-r..r} sum_{dx=-r..r} [ s(y+dy, x+dx) == 1 ]
 *     Cells outside the grid are ghost cells of value 0 (zero boundary, the
 *     global halo of Sec. IV) or wrap around (periodic boundary, Sec. V-A).
 *     Only state 1 ("alive") is counted.  The centre cell is counted ONCE
 *     (reading of the "added twice" remark of Sec. IV: the Moore product with
 *     a unit-diagonal band contains the centre once).
 *  1b. Simplified von Neumann count (Sec. IV, Eq. 3: the second product takes
 *     Lambda instead of H and adds H, R = Pi*Lambda + Lambda*Pi):
 *        L(y,x) = sum_{d=-r..r} [ s(y+d, x) == 1 ] + sum_{d=-r..r} [ s(y, x+d) == 1 ]
 *     the vertical and the horizontal segment through the cell; the centre
 *     lies on both and is counted TWICE, as the paper states for this form.
 *  2. Middle-cell flag M of the LTL notation R C M S B N (Sec. V-A):
 *        Moore:              k = L - (M == 0 ? [s(y,x) == 1] : 0)
 *        simplified v. N.:   k = L - (M == 0 ? 2 : 1) * [s(y,x) == 1]
 *     so that k counts the live neighbours, plus the cell itself when M = 1,
 *     in both neighbourhoods (the paper's "compute R - 2 Lambda" when the
 *     centre is excluded).
 *  3. Transition (Sec. V-A notation; multi-state decay read as the
 *     Generations-style LTL rule, since the paper only runs C = 2):
 *        s == 0      -> 1 if b1 <= k <= b2 else 0
 *        s == 1      -> 1 if s1 <= k <= s2 else (C > 2 ? 2 : 0)
 *        2 <= s < C  -> s + 1, or 0 when s + 1 == C
 *     All cells update synchronously from the previous grid (ping-pong
 *     buffers of Sec. IV-C).
 *
 * No blocking, fusion or reordering: one plain (2r+1)^2 loop per cell (two
 * (2r+1) loops for the simplified von Neumann count).  The
 * only liberty taken is clipping the dy/dx loop ranges to the grid for the
 * zero boundary (the skipped terms are the ghost zeros).  Rows are spread
 * over OpenMP threads; every cell is independent.
 *
 * Built with -DORACLE_MUTATION=<n> (tests only) the file plants one known
 * mistake so the test-suite can show that its pins catch it.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORACLE_MUTATION
#define ORACLE_MUTATION 0
#endif

typedef struct {
  int32_t r, C, M, s1, s2, b1, b2;
  int32_t nbhd; /* 0: Moore box (Eqs. 1-2); 1: simplified von Neumann cross (Eq. 3) */
} oracle_rule;

enum { ORACLE_ZERO = 0, ORACLE_PERIODIC = 1 };

static int64_t wrap(int64_t i, int64_t n) {
  int64_t m = i % n;
  return m < 0 ? m + n : m;
}

/* L(y,x): state-1 cells in the (2r+1)^2 box centred on (y,x), centre included. */
static int32_t box_count(const uint8_t *g, int64_t H, int64_t W, int64_t ld,
                         int64_t y, int64_t x, int r, int boundary) {
  int32_t n = 0;
  int lo = -r, hi = r;
#if ORACLE_MUTATION == 1 /* dropped term: the last column of the box */
  int hix = r - 1;
#else
  int hix = r;
#endif
  if (boundary == ORACLE_PERIODIC) {
    for (int dy = lo; dy <= hi; ++dy) {
      const uint8_t *row = g + wrap(y + dy, H) * ld;
      for (int dx = lo; dx <= hix; ++dx) n += row[wrap(x + dx, W)] == 1;
    }
    return n;
  }
  int64_t y0 = y + lo < 0 ? 0 : y + lo;
  int64_t y1 = y + hi > H - 1 ? H - 1 : y + hi;
  int64_t x0 = x + lo < 0 ? 0 : x + lo;
  int64_t x1 = x + hix > W - 1 ? W - 1 : x + hix;
  for (int64_t yy = y0; yy <= y1; ++yy) {
#if ORACLE_MUTATION == 2 /* transposed index */
    for (int64_t xx = x0; xx <= x1; ++xx) n += (xx < H && yy < W) ? g[xx * ld + yy] == 1 : 0;
#else
    const uint8_t *row = g + yy * ld;
    for (int64_t xx = x0; xx <= x1; ++xx) n += row[xx] == 1;
#endif
  }
  return n;
}

/* L(y,x) of Eq. 3: state-1 cells on the vertical and on the horizontal segment
 * of half-length r through (y,x); the centre is on both and counts twice. */
static int32_t cross_count(const uint8_t *g, int64_t H, int64_t W, int64_t ld,
                           int64_t y, int64_t x, int r, int boundary) {
  int32_t n = 0;
  for (int d = -r; d <= r; ++d) {
    const int64_t yy = y + d, xx = x + d;
    if (boundary == ORACLE_PERIODIC) {
      n += g[wrap(yy, H) * ld + x] == 1;
#if ORACLE_MUTATION == 6 /* the horizontal segment misses the centre */
      if (d != 0)
#endif
      n += g[y * ld + wrap(xx, W)] == 1;
    } else {
      if (yy >= 0 && yy < H) n += g[yy * ld + x] == 1;
#if ORACLE_MUTATION == 6
      if (d != 0)
#endif
      if (xx >= 0 && xx < W) n += g[y * ld + xx] == 1;
    }
  }
  return n;
}

static uint8_t transition(uint8_t s, int32_t L, const oracle_rule *R) {
#if ORACLE_MUTATION == 3 /* centre handling inverted (subtract when M == 1) */
  int32_t k = L - ((R->M == 1) ? (s == 1) : 0);
#elif ORACLE_MUTATION == 7 /* the cross takes the Moore centre handling */
  int32_t k = L - ((R->M == 0) ? (s == 1) : 0);
#else
  int32_t k = R->nbhd == 1 ? L - (R->M == 0 ? 2 : 1) * (s == 1)
                           : L - ((R->M == 0) ? (s == 1) : 0);
#endif
  if (s == 0) {
#if ORACLE_MUTATION == 4 /* off-by-one in the birth range */
    return (uint8_t)(k >= R->b1 && k < R->b2);
#else
    return (uint8_t)(k >= R->b1 && k <= R->b2);
#endif
  }
  if (s == 1) {
    if (k >= R->s1 && k <= R->s2) return 1;
    return (uint8_t)(R->C > 2 ? 2 : 0);
  }
#if ORACLE_MUTATION == 5 /* decay skips the last state */
  return (uint8_t)(s + 2 >= R->C ? 0 : s + 1);
#else
  return (uint8_t)(s + 1 == R->C ? 0 : s + 1);
#endif
}

static int check_args(int64_t H, int64_t W, int64_t ld, int r, int boundary) {
  if (H < 1 || W < 1 || ld < W || r < 0) return -1;
  if (boundary != ORACLE_ZERO && boundary != ORACLE_PERIODIC) return -1;
  return 0;
}

static int check_rule(const oracle_rule *R) {
  if (!R || R->r < 0 || R->C < 2 || R->C > 256 || (R->M != 0 && R->M != 1)) return -1;
  if (R->nbhd != 0 && R->nbhd != 1) return -1;
  return 0;
}

/* S[y*lds + x] = L(y,x) for the whole grid. */
int oracle_box_sums(const uint8_t *g, int64_t H, int64_t W, int64_t ld, int r,
                    int boundary, int32_t *S, int64_t lds) {
  if (!g || !S || check_args(H, W, ld, r, boundary) || lds < W) return -1;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t y = 0; y < H; ++y)
    for (int64_t x = 0; x < W; ++x) S[y * lds + x] = box_count(g, H, W, ld, y, x, r, boundary);
  return 0;
}

/* S[y*lds + x] = the simplified von Neumann count L(y,x) of Eq. 3. */
int oracle_cross_sums(const uint8_t *g, int64_t H, int64_t W, int64_t ld, int r,
                      int boundary, int32_t *S, int64_t lds) {
  if (!g || !S || check_args(H, W, ld, r, boundary) || lds < W) return -1;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t y = 0; y < H; ++y)
    for (int64_t x = 0; x < W; ++x) S[y * lds + x] = cross_count(g, H, W, ld, y, x, r, boundary);
  return 0;
}

/* out = one synchronous LTL step of in. */
int oracle_step(const uint8_t *in, uint8_t *out, int64_t H, int64_t W, int64_t ld,
                const oracle_rule *R, int boundary) {
  if (!in || !out || in == out || check_rule(R) || check_args(H, W, ld, R->r, boundary)) return -1;
  for (int64_t y = 0; y < H; ++y)
    for (int64_t x = 0; x < W; ++x)
      if (in[y * ld + x] >= R->C) return -2; /* state outside [0, C) */
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t y = 0; y < H; ++y)
    for (int64_t x = 0; x < W; ++x) {
      int32_t L = R->nbhd == 1 ? cross_count(in, H, W, ld, y, x, R->r, boundary)
                               : box_count(in, H, W, ld, y, x, R->r, boundary);
      out[y * ld + x] = transition(in[y * ld + x], L, R);
    }
  return 0;
}

/* n_steps synchronous steps, in place on g (ping-pong through a scratch copy). */
int oracle_run(uint8_t *g, int64_t H, int64_t W, int64_t ld, const oracle_rule *R,
               int boundary, int64_t n_steps) {
  if (!g || n_steps < 0) return -1;
  if (n_steps == 0) return 0;
  uint8_t *tmp = (uint8_t *)malloc((size_t)(H * ld));
  if (!tmp) return -3;
  memcpy(tmp, g, (size_t)(H * ld));
  uint8_t *a = g, *b = tmp;
  int rc = 0;
  for (int64_t t = 0; t < n_steps && rc == 0; ++t) {
    rc = oracle_step(a, b, H, W, ld, R, boundary);
    uint8_t *s = a; a = b; b = s;
  }
  if (rc == 0 && a != g) memcpy(g, a, (size_t)(H * ld));
  free(tmp);
  return rc;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
