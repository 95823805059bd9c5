/*
 * CPU oracle for arc-consistency enforcement on binary CSPs.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg use it.  It shares no code with the CUDA
 * library and is deliberately plain and slow.
 *
 * Notation (paper, Sec. 2): D is the set of pairs (x,a) with a in dom(x);
 * c_xy|_(x,a) is the set of supports of (x,a) on the constraint c_xy; C_x is
 * the set of constraints involving x.
 *
 * Input format (the same the library boundary takes): n variables with
 * values 0..d-1 (1 <= d <= 32); m constraints, constraint c has scope
 * (scope[2c], scope[2c+1]) and relation rows rel[c*d + a], bit b of row a set
 * iff the scope's first variable taking a and the second taking b is allowed.
 * A domain is one uint32 word per variable, bit a set iff a is in dom(x).
 *
 * Readings of the paper that this oracle fixes:
 *  - supports are taken inside the input domain D: c_xy|_(x,a) =
 *    { (y,b) in D : (a,b) allowed }  (the listing multiplies the constraint
 *    tensor by the domain mask before counting, Appendix E);
 *  - "exists y" in Eq. 1 ranges over the real constraints C_x only;
 *  - iterations counts every sweep executed, including the final sweep that
 *    removes nothing;
 *  - default mode runs Eq. 1 to its fixpoint and reports a wipe-out when a
 *    domain of the result is empty; stop-on-wipeout mode ends after the first
 *    sweep that leaves some domain empty (Algorithm 1 throws there, the
 *    listing returns None there).
 *
 * Functions:
 *  oracle_rac        Eq. 1 (Sec. 3) swept synchronously, optionally with the
 *                    incremental restriction of Proposition 2; reports D_ac,
 *                    the sweep count, the status and optionally each sweep.
 *  oracle_ac3        AC-3 (Mackworth 1977; the sequential baseline the paper
 *                    compares against in Sec. 5): a propagation queue of arcs.
 *  oracle_bruteforce D_ac straight from its definition in Sec. 3: the union
 *                    of every arc-consistent subset of D (tiny inputs only).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_WIPEOUT 1
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_ETIMEOUT (-4)

typedef struct {
  int n, d;
  int64_t m;
  const int32_t *scope;
  const uint32_t *rel;
  /* C_x as a list of (constraint, side) entries; side 0: x = scope[2c]. */
  int64_t *cx_off;
  int64_t *cx_con;
  unsigned char *cx_side;
} net_t;

/* Is the pair (x = a, y = b) allowed by constraint c, seen from side `side`
 * (x is the scope's first variable when side == 0, its second otherwise)? */
static int allowed(const net_t *N, int64_t c, int side, int a, int b) {
  if (side == 0) return (int)((N->rel[c * N->d + a] >> b) & 1u);
  return (int)((N->rel[c * N->d + b] >> a) & 1u);
}

static int other(const net_t *N, int64_t c, int side) {
  return side == 0 ? N->scope[2 * c + 1] : N->scope[2 * c];
}

static void net_free(net_t *N) {
  free(N->cx_off);
  free(N->cx_con);
  free(N->cx_side);
}

static int net_init(net_t *N, int32_t n, int32_t d, int64_t m, const int32_t *scope,
                    const uint32_t *rel) {
  memset(N, 0, sizeof(*N));
  if (n < 0 || d < 1 || d > 32 || m < 0) return ORACLE_EINVAL;
  N->n = n;
  N->d = d;
  N->m = m;
  N->scope = scope;
  N->rel = rel;
  N->cx_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  N->cx_con = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * m + 1));
  N->cx_side = (unsigned char *)malloc((size_t)(2 * m + 1));
  if (!N->cx_off || !N->cx_con || !N->cx_side) {
    net_free(N);
    return ORACLE_ENOMEM;
  }
  for (int64_t c = 0; c < m; ++c) {
    int x = scope[2 * c], y = scope[2 * c + 1];
    if (x < 0 || x >= n || y < 0 || y >= n || x == y) {
      net_free(N);
      return ORACLE_EINVAL;
    }
    N->cx_off[x + 1]++;
    N->cx_off[y + 1]++;
  }
  for (int x = 0; x < n; ++x) N->cx_off[x + 1] += N->cx_off[x];
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!fill) {
    net_free(N);
    return ORACLE_ENOMEM;
  }
  memcpy(fill, N->cx_off, sizeof(int64_t) * ((size_t)n + 1));
  for (int64_t c = 0; c < m; ++c) {
    int x = scope[2 * c], y = scope[2 * c + 1];
    N->cx_con[fill[x]] = c;
    N->cx_side[fill[x]++] = 0;
    N->cx_con[fill[y]] = c;
    N->cx_side[fill[y]++] = 1;
  }
  free(fill);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* O2: the recurrence of Eq. 1.                                              */
/*                                                                          */
/*   Dt^(0) = {}                                                            */
/*   Dt^(k) = Dt^(k-1) U { (x,a) in D : exists c_xy in C_x with             */
/*                          c_xy|_(x,a) subset of Dt^(k-1) }                */
/*                                                                          */
/* Dt ("D tilde") is the set of values found to have no valid support; the  */
/* enforced domain is D \ Dt^(K) once Dt^(K) = Dt^(K+1).  Every sweep reads */
/* only Dt^(k-1) (all pairs are collected simultaneously).                  */
/*                                                                          */
/* With `incremental`, sweep k >= 2 examines only the constraints c_xy      */
/* whose y lost a value in sweep k-1 (Proposition 2: every value removed in */
/* sweep k lost a support removed in sweep k-1).                            */
/* ------------------------------------------------------------------------ */

/* c_xy|_(x,a) subset of Dt, where supports range over the input domain D. */
static int supports_all_removed(const net_t *N, const unsigned char *inD,
                                const unsigned char *Dt, int64_t c, int side, int a) {
  int y = other(N, c, side);
  for (int b = 0; b < N->d; ++b) {
    int in_support_set = allowed(N, c, side, a, b) && inD[(size_t)y * N->d + b];
    if (in_support_set && !Dt[(size_t)y * N->d + b]) return 0;
  }
  return 1;
}

int oracle_rac(int32_t n, int32_t d, int64_t m, const int32_t *scope, const uint32_t *rel,
               const uint32_t *dom_in, uint32_t *dom_out, int32_t stop_on_wipeout,
               int32_t incremental, int32_t max_sweeps, int32_t n_threads, int32_t *iterations,
               int32_t *status, uint32_t *trace, int32_t trace_cap, int64_t *removed_per_sweep) {
  net_t N;
  int rc = net_init(&N, n, d, m, scope, rel);
  if (rc != ORACLE_OK) return rc;
  size_t nd = (size_t)n * (size_t)d;
  unsigned char *inD = (unsigned char *)calloc(nd + 1, 1);
  unsigned char *Dt_prev = (unsigned char *)calloc(nd + 1, 1); /* Dt^(k-1) */
  unsigned char *Dt = (unsigned char *)calloc(nd + 1, 1);      /* Dt^(k)   */
  unsigned char *lost_prev = (unsigned char *)calloc((size_t)n + 1, 1); /* y lost a value in k-1 */
  unsigned char *lost = (unsigned char *)calloc((size_t)n + 1, 1);
  if (!inD || !Dt_prev || !Dt || !lost_prev || !lost) {
    free(inD); free(Dt_prev); free(Dt); free(lost_prev); free(lost);
    net_free(&N);
    return ORACLE_ENOMEM;
  }
  for (int x = 0; x < n; ++x)
    for (int a = 0; a < d; ++a) inD[(size_t)x * d + a] = (unsigned char)((dom_in[x] >> a) & 1u);

  int k = 0;
  int st = ORACLE_OK;
  for (;;) {
    ++k;
    /* Dt^(k) starts as Dt^(k-1) and collects the newly unsupported pairs. */
    memcpy(Dt, Dt_prev, nd);
    int64_t newly = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : newly) num_threads(n_threads > 0 ? n_threads : 1)
    for (int x = 0; x < n; ++x) {
      unsigned char lost_x = 0;
      for (int a = 0; a < d; ++a) {
        size_t xa = (size_t)x * d + a;
        if (!inD[xa] || Dt_prev[xa]) continue; /* only pairs of D not yet collected */
        int collect = 0;
        for (int64_t e = N.cx_off[x]; e < N.cx_off[x + 1] && !collect; ++e) {
          int64_t c = N.cx_con[e];
          int side = N.cx_side[e];
          if (incremental && k >= 2 && !lost_prev[other(&N, c, side)]) continue;
          collect = supports_all_removed(&N, inD, Dt_prev, c, side, a);
        }
        if (collect) {
          Dt[xa] = 1;
          lost_x = 1;
          ++newly;
        }
      }
      lost[x] = lost_x;
    }
    if (removed_per_sweep && k <= trace_cap) removed_per_sweep[k - 1] = newly;
    if (trace && k <= trace_cap) {
      for (int x = 0; x < n; ++x) {
        uint32_t w = 0;
        for (int a = 0; a < d; ++a)
          if (inD[(size_t)x * d + a] && !Dt[(size_t)x * d + a]) w |= 1u << a;
        trace[(size_t)(k - 1) * n + x] = w;
      }
    }
    int some_empty = 0;
    for (int x = 0; x < n && !some_empty; ++x) {
      int left = 0;
      for (int a = 0; a < d; ++a) left += inD[(size_t)x * d + a] && !Dt[(size_t)x * d + a];
      some_empty = left == 0;
    }
    unsigned char *swap = Dt_prev;
    Dt_prev = Dt; /* Dt_prev now holds Dt^(k) */
    Dt = swap;
    swap = lost_prev;
    lost_prev = lost;
    lost = swap;
    if (stop_on_wipeout && some_empty) {
      st = ORACLE_WIPEOUT;
      break;
    }
    if (newly == 0) { /* Dt^(k) = Dt^(k-1): the fixpoint */
      st = some_empty ? ORACLE_WIPEOUT : ORACLE_OK;
      break;
    }
    if (max_sweeps > 0 && k >= max_sweeps) {
      st = ORACLE_ETIMEOUT;
      break;
    }
  }
  for (int x = 0; x < n; ++x) {
    uint32_t w = 0;
    for (int a = 0; a < d; ++a)
      if (inD[(size_t)x * d + a] && !Dt_prev[(size_t)x * d + a]) w |= 1u << a;
    dom_out[x] = w;
  }
  *iterations = k;
  *status = st;
  free(inD); free(Dt_prev); free(Dt); free(lost_prev); free(lost);
  net_free(&N);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* O1: AC-3.  A queue of arcs (x, c); revising (x, c) deletes every value a */
/* of dom(x) without any b in dom(y) allowed with it; when dom(x) shrinks,  */
/* every arc (z, c') with c' in C_x, z != y, is queued again.  Runs to the   */
/* empty queue (no early exit on an empty domain), so it ends at D_ac.      */
/* ------------------------------------------------------------------------ */

int oracle_ac3(int32_t n, int32_t d, int64_t m, const int32_t *scope, const uint32_t *rel,
               const uint32_t *dom_in, uint32_t *dom_out, int64_t *revisions, int32_t *status) {
  net_t N;
  int rc = net_init(&N, n, d, m, scope, rel);
  if (rc != ORACLE_OK) return rc;
  size_t nd = (size_t)n * (size_t)d;
  unsigned char *D = (unsigned char *)calloc(nd + 1, 1);
  /* arc id 2c + side: the arc from scope[2c + side] through c */
  int64_t n_arcs = 2 * m;
  int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_arcs + 1));
  unsigned char *queued = (unsigned char *)calloc((size_t)n_arcs + 1, 1);
  if (!D || !queue || !queued) {
    free(D); free(queue); free(queued);
    net_free(&N);
    return ORACLE_ENOMEM;
  }
  for (int x = 0; x < n; ++x)
    for (int a = 0; a < d; ++a) D[(size_t)x * d + a] = (unsigned char)((dom_in[x] >> a) & 1u);
  /* circular FIFO of capacity n_arcs: an arc is in it at most once */
  int64_t head = 0, count = 0;
  for (int64_t arc = 0; arc < n_arcs; ++arc) {
    queue[arc] = arc;
    queued[arc] = 1;
  }
  count = n_arcs;
  int64_t revs = 0;
  while (count > 0) {
    int64_t arc = queue[head];
    head = (head + 1) % n_arcs;
    --count;
    queued[arc] = 0;
    int64_t c = arc / 2;
    int side = (int)(arc % 2);
    int x = side == 0 ? scope[2 * c] : scope[2 * c + 1];
    int y = other(&N, c, side);
    ++revs;
    int revised = 0;
    for (int a = 0; a < d; ++a) {
      if (!D[(size_t)x * d + a]) continue;
      int has_support = 0;
      for (int b = 0; b < d && !has_support; ++b)
        has_support = D[(size_t)y * d + b] && allowed(&N, c, side, a, b);
      if (!has_support) {
        D[(size_t)x * d + a] = 0;
        revised = 1;
      }
    }
    if (revised) {
      for (int64_t e = N.cx_off[x]; e < N.cx_off[x + 1]; ++e) {
        int64_t c2 = N.cx_con[e];
        if (c2 == c) continue;
        /* the arc pointing at x: from the other end of c2 */
        int64_t in_arc = 2 * c2 + (1 - N.cx_side[e]);
        if (!queued[in_arc]) {
          queue[(head + count) % n_arcs] = in_arc;
          queued[in_arc] = 1;
          ++count;
        }
      }
    }
  }
  int some_empty = 0;
  for (int x = 0; x < n; ++x) {
    uint32_t w = 0;
    for (int a = 0; a < d; ++a)
      if (D[(size_t)x * d + a]) w |= 1u << a;
    dom_out[x] = w;
    some_empty |= w == 0;
  }
  if (revisions) *revisions = revs;
  *status = some_empty ? ORACLE_WIPEOUT : ORACLE_OK;
  free(D); free(queue); free(queued);
  net_free(&N);
  return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* O3: brute force from the definition in Sec. 3.  A subset S of D is arc    */
/* consistent iff every (x,a) in S has, on every c_xy in C_x, a support      */
/* (y,b) that is also in S; D_ac is the union of all such S.  |D| <= 22.     */
/* ------------------------------------------------------------------------ */

int oracle_bruteforce(int32_t n, int32_t d, int64_t m, const int32_t *scope,
                      const uint32_t *rel, const uint32_t *dom_in, uint32_t *dom_out,
                      int32_t *status) {
  net_t N;
  int rc = net_init(&N, n, d, m, scope, rel);
  if (rc != ORACLE_OK) return rc;
  int vx[32], va[32];
  int nv = 0;
  for (int x = 0; x < n; ++x)
    for (int a = 0; a < d; ++a)
      if ((dom_in[x] >> a) & 1u) {
        if (nv >= 22) {
          net_free(&N);
          return ORACLE_EINVAL;
        }
        vx[nv] = x;
        va[nv] = a;
        ++nv;
      }
  /* index of (x,a) among the listed values, -1 if not in D */
  int *idx = (int *)malloc(sizeof(int) * ((size_t)n * d + 1));
  if (!idx) {
    net_free(&N);
    return ORACLE_ENOMEM;
  }
  for (size_t i = 0; i < (size_t)n * d; ++i) idx[i] = -1;
  for (int i = 0; i < nv; ++i) idx[(size_t)vx[i] * d + va[i]] = i;
  uint32_t union_of_ac = 0;
  for (uint32_t S = 0; S < (1u << nv); ++S) {
    int is_ac = 1;
    for (int i = 0; i < nv && is_ac; ++i) {
      if (!((S >> i) & 1u)) continue;
      int x = vx[i], a = va[i];
      for (int64_t e = N.cx_off[x]; e < N.cx_off[x + 1] && is_ac; ++e) {
        int64_t c = N.cx_con[e];
        int side = N.cx_side[e];
        int y = other(&N, c, side);
        int has_support_in_S = 0;
        for (int b = 0; b < d && !has_support_in_S; ++b) {
          int j = idx[(size_t)y * d + b];
          has_support_in_S = j >= 0 && ((S >> j) & 1u) && allowed(&N, c, side, a, b);
        }
        is_ac = has_support_in_S;
      }
    }
    if (is_ac) union_of_ac |= S;
  }
  int some_empty = 0;
  for (int x = 0; x < n; ++x) dom_out[x] = 0;
  for (int i = 0; i < nv; ++i)
    if ((union_of_ac >> i) & 1u) dom_out[vx[i]] |= 1u << va[i];
  for (int x = 0; x < n; ++x) some_empty |= dom_out[x] == 0;
  *status = some_empty ? ORACLE_WIPEOUT : ORACLE_OK;
  free(idx);
  net_free(&N);
  return ORACLE_OK;
}
