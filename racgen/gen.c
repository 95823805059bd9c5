/*
 * racgen: seeded synthetic inputs for binary-CSP arc-consistency runs.
 *
 * This module only draws random networks and domain states.  It holds none
 * of the arc-consistency arithmetic; both the CUDA path and the CPU oracle
 * consume what it writes.
 *
 * Every random decision is a counter-based hash, so any single bit of any
 * instance can be regenerated on its own, independent of thread count:
 *
 *   splitmix64(z): z += 0x9E3779B97F4A7C15;
 *                  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
 *                  z = (z ^ (z >> 27)) * 0x94D049BB133111EB;
 *                  return z ^ (z >> 31);
 *   key(seed, tag, f0, f1, ...) = absorb fields one at a time:
 *                  h = splitmix64(seed); h = splitmix64(h ^ tag);
 *                  h = splitmix64(h ^ f0); h = splitmix64(h ^ f1); ...
 *   u01(h) = (h >> 11) * 2^-53,  Bern(p, h) = u01(h) < p.
 *
 * Random binary CSP (the experiments' benchmark model: every unordered pair
 * of the n variables carries a constraint with probability `density`):
 *   pair x<y constrained  iff Bern(density, key(seed, 1, inst, x, y))
 *   R_xy[a][b] = 0        iff Bern(tightness, splitmix64(P ^ ((a << 8) | b)))
 *                          with P = key(seed, 2, inst, x, y)
 * Constraints are listed in (x, y) lexicographic order with x < y; relation
 * word a of constraint c holds R_xy[a][b] in bit b.
 *
 * Per-instance shape draws for uneven batches use tag 3; assignment states
 * (a few variables reduced to singleton domains, as the search's `assign`
 * step does) use tag 4.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t sm64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline double u01(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

uint64_t racgen_splitmix64(uint64_t z) { return sm64(z); }

uint64_t racgen_key(uint64_t seed, uint64_t tag, int nf, const uint64_t *f) {
  uint64_t h = sm64(seed);
  h = sm64(h ^ tag);
  for (int i = 0; i < nf; ++i) h = sm64(h ^ f[i]);
  return h;
}

static inline uint64_t key3(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, uint64_t c) {
  uint64_t h = sm64(seed);
  h = sm64(h ^ tag);
  h = sm64(h ^ a);
  h = sm64(h ^ b);
  return sm64(h ^ c);
}

static inline int pair_present(uint64_t seed, uint64_t inst, int x, int y, double density) {
  return u01(key3(seed, 1, inst, (uint64_t)x, (uint64_t)y)) < density;
}

/* Number of constraints of instance `inst` (x < y pairs drawn present). */
int64_t racgen_count_constraints(uint64_t seed, uint64_t inst, int32_t n, double density) {
  if (n <= 1) return 0;
  int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
  for (int x = 0; x < n; ++x) {
    int64_t c = 0;
    for (int y = x + 1; y < n; ++y) c += pair_present(seed, inst, x, y, density);
    total += c;
  }
  return total;
}

/* Fill scope (m x 2 int32) and rel (m x d uint32).  `m` must equal
 * racgen_count_constraints(seed, inst, n, density).  Returns 0 on success. */
int racgen_fill_network(uint64_t seed, uint64_t inst, int32_t n, int32_t d, double density,
                        double tightness, int64_t m, int32_t *scope, uint32_t *rel) {
  if (n < 0 || d < 1 || d > 32) return -1;
  int64_t *row_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  if (!row_off) return -2;
#pragma omp parallel for schedule(dynamic, 16)
  for (int x = 0; x < n; ++x) {
    int64_t c = 0;
    for (int y = x + 1; y < n; ++y) c += pair_present(seed, inst, x, y, density);
    row_off[x + 1] = c;
  }
  row_off[0] = 0;
  for (int x = 0; x < n; ++x) row_off[x + 1] += row_off[x];
  if (row_off[n] != m) {
    free(row_off);
    return -3;
  }
#pragma omp parallel for schedule(dynamic, 4)
  for (int x = 0; x < n; ++x) {
    int64_t c = row_off[x];
    for (int y = x + 1; y < n; ++y) {
      if (!pair_present(seed, inst, x, y, density)) continue;
      scope[2 * c] = x;
      scope[2 * c + 1] = y;
      uint64_t P = key3(seed, 2, inst, (uint64_t)x, (uint64_t)y);
      for (int a = 0; a < d; ++a) {
        uint32_t w = 0;
        for (int b = 0; b < d; ++b) {
          uint64_t h = sm64(P ^ (((uint64_t)a << 8) | (uint64_t)b));
          if (!(u01(h) < tightness)) w |= 1u << b;
        }
        rel[c * d + a] = w;
      }
      ++c;
    }
  }
  free(row_off);
  return 0;
}

/* Shape of instance `inst` of an uneven batch: n ~ U{50..800}, d ~ U{8..32},
 * density ~ U[0.3, 1.0], tightness ~ U[0.2, 0.4]. */
void racgen_batch_params(uint64_t seed, uint64_t inst, int32_t *n, int32_t *d, double *density,
                         double *tightness) {
  *n = 50 + (int32_t)(u01(key3(seed, 3, inst, 0, 0)) * 751.0);
  *d = 8 + (int32_t)(u01(key3(seed, 3, inst, 1, 0)) * 25.0);
  *density = 0.3 + 0.7 * u01(key3(seed, 3, inst, 2, 0));
  *tightness = 0.2 + 0.2 * u01(key3(seed, 3, inst, 3, 0));
}

/* Assignment state s of instance inst: k ~ U{1..5} distinct variables (at most
 * n), each reduced to one uniformly drawn value; every other domain full.
 * Writes n words to dom; returns k. */
int32_t racgen_assignment_state(uint64_t seed, uint64_t inst, uint64_t s, int32_t n, int32_t d,
                                uint32_t *dom) {
  uint32_t full = d >= 32 ? 0xFFFFFFFFu : ((1u << d) - 1u);
  for (int x = 0; x < n; ++x) dom[x] = full;
  if (n <= 0) return 0;
  uint64_t f[4];
  f[0] = inst; f[1] = s; f[2] = 0; f[3] = 0;
  int k = 1 + (int)(u01(racgen_key(seed, 4, 4, f)) * 5.0);
  if (k > n) k = n;
  int picked[5];
  int chosen = 0;
  for (uint64_t i = 0; chosen < k; ++i) {
    f[2] = 1; f[3] = i;
    int v = (int)(u01(racgen_key(seed, 4, 4, f)) * (double)n);
    int dup = 0;
    for (int j = 0; j < chosen; ++j) dup |= picked[j] == v;
    if (dup) continue;
    picked[chosen++] = v;
    f[2] = 2; f[3] = (uint64_t)v;
    int a = (int)(u01(racgen_key(seed, 4, 4, f)) * (double)d);
    dom[v] = 1u << a;
  }
  return k;
}
