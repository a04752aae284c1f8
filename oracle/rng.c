/*
 * rng.c -- oracle (test infrastructure only): the random parameters of one
 * SRFT realization, Section 3 of the paper.
 *
 * The paper fixes the distributions, not a generator:
 *   - d_j, zeta_j, zeta~_j i.i.d. uniform on the unit circle (Eqs. SRFT2, Rokhlin_trans);
 *   - Pi, Pi~ independent uniform permutations (Eq. Rokhlin_trans);
 *   - theta_k, theta~_k i.i.d. uniform on [0, 2 pi] (after Eq. big_def);
 *   - s_1..s_l uniform on {1..n}, drawn WITHOUT replacement as in the
 *     paper's own implementation (Section 3), which keeps T's rows orthonormal.
 * The generator is SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a
 * counter-based stream per parameter kind; bounded integers use Lemire's
 * unbiased multiply-shift method (ACM TOMS 2019); permutations use the
 * Fisher-Yates shuffle (Durstenfeld's in-place form). The sampled indices are
 * sorted ascending (their order does not change R, only the row order of Y).
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

static const uint64_t GOLDEN = 0x9E3779B97F4A7C15ULL;

uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t orc_draw(uint64_t seed, uint64_t kind, uint64_t j) {
  return orc_mix64(seed + GOLDEN * ((kind << 40) + j + 1));
}

typedef struct { uint64_t seed, kind, j; } stream;

static uint64_t next(stream *st) { return orc_draw(st->seed, st->kind, st->j++); }

/* uniform double in [0, 1) from the top 53 bits */
static double next_unit(stream *st) { return (double)(next(st) >> 11) * 0x1.0p-53; }

/* Lemire: uniform integer in [0, range), range >= 1, unbiased */
static uint64_t next_below(stream *st, uint64_t range) {
  unsigned __int128 prod = (unsigned __int128)next(st) * range;
  uint64_t low = (uint64_t)prod;
  if (low < range) {
    uint64_t thresh = (0 - range) % range;
    while (low < thresh) {
      prod = (unsigned __int128)next(st) * range;
      low = (uint64_t)prod;
    }
  }
  return (uint64_t)(prod >> 64);
}

static void draw_phases(stream *st, int64_t n, zc *out) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t j = 0; j < n; ++j) {
    double a = two_pi * next_unit(st);
    out[j] = cos(a) + I * sin(a);
  }
}

static void draw_angles(stream *st, int64_t count, double *out) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t k = 0; k < count; ++k) out[k] = two_pi * next_unit(st);
}

static void draw_permutation(stream *st, int64_t n, int64_t *p) {
  for (int64_t j = 0; j < n; ++j) p[j] = j;
  for (int64_t i = n - 1; i >= 1; --i) {
    int64_t j = (int64_t)next_below(st, (uint64_t)(i + 1));
    int64_t t = p[i]; p[i] = p[j]; p[j] = t;
  }
}

static int cmp_i64(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return (x > y) - (x < y);
}

/* l distinct indices of [0, n): the first l steps of a forward Fisher-Yates pass */
static void draw_sample(stream *st, int64_t n, int64_t l, int64_t *s) {
  int64_t *q = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t j = 0; j < n; ++j) q[j] = j;
  for (int64_t i = 0; i < l; ++i) {
    int64_t j = i + (int64_t)next_below(st, (uint64_t)(n - i));
    int64_t t = q[i]; q[i] = q[j]; q[j] = t;
  }
  for (int64_t i = 0; i < l; ++i) s[i] = q[i];
  qsort(s, (size_t)l, sizeof(int64_t), cmp_i64);
  free(q);
}

void orc_draw_params(uint64_t seed, int64_t n, int64_t l,
                     zc *zeta_t, int64_t *pi_t, double *theta_t,
                     zc *zeta, int64_t *pi, double *theta,
                     zc *d, int64_t *s) {
  stream st;
  st = (stream){seed, 0, 0}; draw_phases(&st, n, zeta_t);
  st = (stream){seed, 1, 0}; draw_permutation(&st, n, pi_t);
  st = (stream){seed, 2, 0}; draw_angles(&st, n - 1, theta_t);
  st = (stream){seed, 3, 0}; draw_phases(&st, n, zeta);
  st = (stream){seed, 4, 0}; draw_permutation(&st, n, pi);
  st = (stream){seed, 5, 0}; draw_angles(&st, n - 1, theta);
  st = (stream){seed, 6, 0}; draw_phases(&st, n, d);
  st = (stream){seed, 7, 0}; draw_sample(&st, n, l, s);
}
