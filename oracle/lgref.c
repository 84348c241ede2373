/*
 * lgref.c -- plain FP64 reference ("the oracle") for the unsmoothed-aggregation
 * multigrid for graph Laplacians of Konolige & Brown, "A Parallel Solver for
 * Graph Laplacians" (PASC'18).
 *
 * TEST INFRASTRUCTURE. Slow, single-threaded, sequential loops in the order
 * the paper states each step. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg use it; the CUDA library never does. It shares
 * no code with the CUDA library.
 *
 * Readings of points the paper leaves open are marked "reading:" where they
 * are taken. Everything is FP64.
 *
 * Parity status of each part (what pins it is in the tests under tests/):
 *   - random streams: SplitMix64 published outputs;
 *   - Laplacian, components: scipy sparse / csgraph, quadratic-form identity;
 *   - elimination: brute-force neighbourhood check, dense Schur complement,
 *     two-level inverse identity, star/path/grid worked cases;
 *   - strength: Jacobi on eigenvectors (closed form), Cauchy-Schwarz bounds,
 *     hand-computed normalisation;
 *   - aggregation: partition/seed/vote invariants, star worked cases;
 *   - Galerkin: dense R L P, energy identity;
 *   - Lanczos: K_n and bipartite closed forms, dense eigenvalues;
 *   - Chebyshev: the degree-k error polynomial on eigenvectors;
 *   - coarsest pseudo-inverse: K_n closed form, dense pseudo-inverse;
 *   - PCG: residual recomputed independently, dense direct solution.
 */
#include "lgref.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct lgref_csr {
  int64_t n, nnz;
  int64_t* rowptr;
  int32_t* col;
  double* w;
};

typedef struct {
  int32_t kind;
  lgref_csr a;     /* off-diagonal weights of L_l */
  double* d;       /* diagonal of L_l (row sums of a) */
  int64_t nc;      /* size of level l+1 */
  int32_t* map;    /* AGG: vertex -> aggregate; ELIM: C vertex -> coarse id, F -> -1 */
  double lambda;   /* AGG: largest-eigenvalue estimate of D^-1 L */
  double* pinv;    /* COARSEST: dense pseudo-inverse, n x n row-major */
} level_t;

#define LGREF_MAX_LEVELS 128

struct lgref_hier {
  int32_t nlev;
  level_t lev[LGREF_MAX_LEVELS];
  lgref_opts o;
};

static void* xmalloc(size_t bytes) {
  void* p = malloc(bytes ? bytes : 1);
  if (!p) abort();
  return p;
}
static void* xcalloc(size_t count, size_t size) {
  void* p = calloc(count ? count : 1, size ? size : 1);
  if (!p) abort();
  return p;
}

void lgref_opts_default(lgref_opts* o) {
  memset(o, 0, sizeof(*o));
  o->coarse_nnz = 1000.0;
  o->elim_min_frac = 0.05;
  o->jacobi_omega = 2.0 / 3.0;
  o->cheb_lo = 0.3;
  o->cheb_hi = 1.1;
  o->stagnation_frac = 0.95;
  o->seed = 0x5eed;
  o->max_levels = 64;
  o->elim_max_degree = 4;
  o->agg_iters = 10;
  o->vote_threshold = 8;
  o->strength_vecs = 4;
  o->strength_sweeps = 3;
  o->cheb_degree = 2;
  o->eig_iters = 10;
  o->max_coarse_n = 4096;
  o->elim_enable = 1;
  o->elim_rounds = 1;
}

/* ------------------------------------------------------------------------ */
/* Random streams: the n-th output of SplitMix64 (Steele, Lea & Flood,       */
/* "Fast splittable pseudorandom number generators", OOPSLA 2014): the state */
/* after n+1 steps is seed + (n+1)*0x9E3779B97F4A7C15, passed through the    */
/* published 64-bit finaliser.                                               */
/* ------------------------------------------------------------------------ */
uint64_t lgref_splitmix64(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Counter layout: stream in bits 56..63, level in bits 40..55, index below. */
static uint64_t stream_counter(int32_t stream, int32_t level, int64_t idx) {
  return ((uint64_t)(uint32_t)stream << 56) | ((uint64_t)(uint32_t)level << 40) | (uint64_t)idx;
}

/* Reading: the hash of a vertex id that Section 3.4 leaves open is the id-th
 * output of stream 0; SplitMix64 is a bijection, so distinct ids never tie.
 * The same hash serves every level (ids are per level). */
uint64_t lgref_vertex_hash(uint64_t seed, int64_t id) {
  return lgref_splitmix64(seed, stream_counter(0, 0, id));
}

/* Uniform in [-1, 1) with 53 random bits. */
double lgref_uniform(uint64_t seed, int32_t stream, int32_t level, int64_t idx) {
  uint64_t z = lgref_splitmix64(seed, stream_counter(stream, level, idx));
  double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  return 2.0 * u - 1.0;
}

/* ------------------------------------------------------------------------ */
/* Laplacian basics (Section 2.1): L = D - A, D_ii = sum_j A_ij.             */
/* ------------------------------------------------------------------------ */
int64_t lgref_components(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t* label) {
  int64_t* queue = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) label[i] = -1;
  int64_t ncomp = 0;
  for (int64_t s = 0; s < n; ++s) {
    if (label[s] >= 0) continue;
    int64_t head = 0, tail = 0;
    queue[tail++] = s;
    label[s] = (int32_t)ncomp;
    while (head < tail) {
      int64_t v = queue[head++];
      for (int64_t k = rowptr[v]; k < rowptr[v + 1]; ++k) {
        int32_t u = col[k];
        if (label[u] < 0) {
          label[u] = (int32_t)ncomp;
          queue[tail++] = u;
        }
      }
    }
    ++ncomp;
  }
  free(queue);
  return ncomp;
}

static int find_in_row(const int64_t* rowptr, const int32_t* col, int64_t row, int32_t key, int64_t* pos) {
  int64_t lo = rowptr[row], hi = rowptr[row + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] == key) { *pos = mid; return 1; }
    if (col[mid] < key) lo = mid + 1; else hi = mid - 1;
  }
  return 0;
}

/* The input contract: a weighted undirected graph with w > 0 (Section 2.1),
 * both directions stored with equal weight, sorted rows, no self-loops or
 * duplicates, and connected. */
int lgref_check_graph(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w) {
  if (n < 1 || rowptr[0] != 0) return LGREF_INVALID;
  for (int64_t i = 0; i < n; ++i) {
    if (rowptr[i + 1] < rowptr[i]) return LGREF_INVALID;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (col[k] < 0 || col[k] >= n || col[k] == i) return LGREF_INVALID;
      if (k > rowptr[i] && col[k] <= col[k - 1]) return LGREF_INVALID;
      if (!(w[k] > 0.0) || !isfinite(w[k])) return LGREF_INVALID;
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      int64_t pos;
      if (!find_in_row(rowptr, col, col[k], (int32_t)i, &pos)) return LGREF_INVALID;
      if (w[pos] != w[k]) return LGREF_INVALID;
    }
  }
  int32_t* label = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)n);
  int64_t ncomp = lgref_components(n, rowptr, col, label);
  free(label);
  return ncomp == 1 ? LGREF_OK : LGREF_DISCONNECTED;
}

void lgref_diag(int64_t n, const int64_t* rowptr, const double* w, double* d) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += w[k];
    d[i] = s;
  }
}

/* y = (D - A) x */
void lgref_apply_L(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                   const double* x, double* y) {
  for (int64_t i = 0; i < n; ++i) {
    double di = 0.0, ax = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      di += w[k];
      ax += w[k] * x[col[k]];
    }
    y[i] = di * x[i] - ax;
  }
}

static lgref_csr* csr_alloc(int64_t n, int64_t nnz) {
  lgref_csr* a = (lgref_csr*)xcalloc(1, sizeof(lgref_csr));
  a->n = n;
  a->nnz = nnz;
  a->rowptr = (int64_t*)xcalloc((size_t)n + 1, sizeof(int64_t));
  a->col = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)nnz);
  a->w = (double*)xmalloc(sizeof(double) * (size_t)nnz);
  return a;
}

int64_t lgref_csr_n(const lgref_csr* a) { return a->n; }
int64_t lgref_csr_nnz(const lgref_csr* a) { return a->nnz; }
void lgref_csr_copy(const lgref_csr* a, int64_t* rowptr, int32_t* col, double* w) {
  memcpy(rowptr, a->rowptr, sizeof(int64_t) * (size_t)(a->n + 1));
  memcpy(col, a->col, sizeof(int32_t) * (size_t)a->nnz);
  memcpy(w, a->w, sizeof(double) * (size_t)a->nnz);
}
static void csr_release(lgref_csr* a) {
  free(a->rowptr);
  free(a->col);
  free(a->w);
}
void lgref_csr_free(lgref_csr* a) {
  if (!a) return;
  csr_release(a);
  free(a);
}

/* ------------------------------------------------------------------------ */
/* Sparse accumulation by sorted triplets: a coarse operator is assembled    */
/* from (row, col, value) contributions; equal (row, col) are summed in the  */
/* order the contributions were generated.                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t r, c;
  int64_t ord;
  double v;
} trip_t;

static int trip_cmp(const void* pa, const void* pb) {
  const trip_t* a = (const trip_t*)pa;
  const trip_t* b = (const trip_t*)pb;
  if (a->r != b->r) return a->r < b->r ? -1 : 1;
  if (a->c != b->c) return a->c < b->c ? -1 : 1;
  if (a->ord != b->ord) return a->ord < b->ord ? -1 : 1;
  return 0;
}

static lgref_csr* csr_from_triplets(int64_t n, trip_t* t, int64_t nt) {
  qsort(t, (size_t)nt, sizeof(trip_t), trip_cmp);
  int64_t nnz = 0;
  for (int64_t k = 0; k < nt; ++k)
    if (k == 0 || t[k].r != t[k - 1].r || t[k].c != t[k - 1].c) ++nnz;
  lgref_csr* a = csr_alloc(n, nnz);
  int64_t o = -1;
  for (int64_t k = 0; k < nt; ++k) {
    if (k == 0 || t[k].r != t[k - 1].r || t[k].c != t[k - 1].c) {
      ++o;
      a->col[o] = t[k].c;
      a->w[o] = t[k].v;
      a->rowptr[t[k].r + 1] += 1;
    } else {
      a->w[o] += t[k].v;
    }
  }
  for (int64_t i = 0; i < n; ++i) a->rowptr[i + 1] += a->rowptr[i];
  return a;
}

/* ------------------------------------------------------------------------ */
/* Low-degree elimination, Section 3.4.                                      */
/* ------------------------------------------------------------------------ */

/* Elimination selection (Section 3.4, Algorithm 2): every vertex with at
 * most max_degree neighbours is a candidate carrying its own id, the others
 * carry nothing. A semiring product of L with this candidate vector gives,
 * for each vertex, the candidate of smallest hash in its neighbourhood (the
 * product passes a candidate through any nonzero entry, and the sum keeps
 * the candidate with the smaller hash; an absent candidate ranks last). A
 * vertex is eliminated when that winner is itself. Readings: a vertex's
 * degree counts its off-diagonal entries, and the neighbourhood is taken
 * from L, so it contains the vertex itself. */
int64_t lgref_elim_select(int64_t n, const int64_t* rowptr, const int32_t* col,
                          int32_t max_degree, uint64_t seed, uint8_t* is_f) {
  int64_t* cand = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) cand[i] = (rowptr[i + 1] - rowptr[i] <= max_degree) ? i : -1;
  int64_t nf = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t z = -1; /* none */
    int self_done = 0;
    int64_t k = rowptr[i], e = rowptr[i + 1];
    while (k < e || !self_done) {
      int64_t j;
      if (!self_done && (k == e || col[k] > i)) {
        j = i; /* the diagonal entry, at its place in column order */
        self_done = 1;
      } else {
        j = col[k++];
      }
      int64_t c = cand[j];
      /* x (+)elim y: keep x unless hash(x) > hash(y) */
      if (c < 0) continue; /* hash(none) = infinity never wins */
      if (z < 0 || lgref_vertex_hash(seed, z) > lgref_vertex_hash(seed, c)) z = c;
    }
    is_f[i] = (uint8_t)(z == i);
    nf += is_f[i];
  }
  free(cand);
  return nf;
}

/* With F the eliminated set and C the rest, the next level is the Schur
 * complement L_{l+1} = L_CC - L_FC^T L_FF^-1 L_FC (Section 3.4). F is an
 * independent set, so L_FF = diag(d_F) and the off-diagonal weight between
 * coarse vertices a != b becomes
 *   W_ab = w_ab + sum_{f in F adjacent to a and b} w_fa w_fb / d_f.
 * C vertices keep their relative order: cmap[c] = rank of c among C, and
 * cmap[f] = -1. */
lgref_csr* lgref_schur(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                       const uint8_t* is_f, int32_t* cmap) {
  int64_t nc = 0;
  for (int64_t i = 0; i < n; ++i) cmap[i] = is_f[i] ? -1 : (int32_t)(nc++);
  int64_t nt = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t deg = rowptr[i + 1] - rowptr[i];
    nt += is_f[i] ? deg * (deg - 1) : deg;
  }
  trip_t* t = (trip_t*)xmalloc(sizeof(trip_t) * (size_t)(nt ? nt : 1));
  int64_t o = 0;
  /* L_CC part */
  for (int64_t i = 0; i < n; ++i) {
    if (is_f[i]) continue;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      if (is_f[col[k]]) continue;
      t[o].r = cmap[i]; t[o].c = cmap[col[k]]; t[o].ord = o; t[o].v = w[k];
      ++o;
    }
  }
  /* - L_FC^T L_FF^-1 L_FC part */
  for (int64_t f = 0; f < n; ++f) {
    if (!is_f[f]) continue;
    double df = 0.0;
    for (int64_t k = rowptr[f]; k < rowptr[f + 1]; ++k) df += w[k];
    for (int64_t ka = rowptr[f]; ka < rowptr[f + 1]; ++ka) {
      for (int64_t kb = rowptr[f]; kb < rowptr[f + 1]; ++kb) {
        if (ka == kb) continue;
        t[o].r = cmap[col[ka]]; t[o].c = cmap[col[kb]]; t[o].ord = o;
        t[o].v = w[ka] * w[kb] / df;
        ++o;
      }
    }
  }
  lgref_csr* a = csr_from_triplets(nc, t, o);
  free(t);
  return a;
}

/* ------------------------------------------------------------------------ */
/* Strength of connection, Section 3.5: m random vectors y, smoothed on      */
/* L y = 0, then the affinity C_ij and its normalisation S_ij.               */
/* ------------------------------------------------------------------------ */

/* Reading: entries uniform in [-1, 1), vector k of level l drawn from
 * stream 1 + k, so both implementations can regenerate them. Layout [n][m]. */
void lgref_strength_vectors(uint64_t seed, int32_t level, int64_t n, int32_t m, double* y) {
  for (int64_t i = 0; i < n; ++i)
    for (int32_t k = 0; k < m; ++k) y[i * m + k] = lgref_uniform(seed, 1 + k, level, i);
}

/* Reading: "Jacobi smoothing" is damped Jacobi on L y = 0,
 * x <- x - omega D^-1 L x, applied `sweeps` times to each of the m columns. */
void lgref_jacobi(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                  int32_t m, int32_t sweeps, double omega, double* x) {
  double* xin = (double*)xmalloc(sizeof(double) * (size_t)(n * m));
  double* lx = (double*)xmalloc(sizeof(double) * (size_t)m);
  for (int32_t s = 0; s < sweeps; ++s) {
    memcpy(xin, x, sizeof(double) * (size_t)(n * m));
    for (int64_t i = 0; i < n; ++i) {
      double di = 0.0;
      for (int32_t k = 0; k < m; ++k) lx[k] = 0.0;
      for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        di += w[p];
        for (int32_t k = 0; k < m; ++k) lx[k] -= w[p] * xin[(int64_t)col[p] * m + k];
      }
      if (di == 0.0) continue;
      for (int32_t k = 0; k < m; ++k) {
        double li = di * xin[i * m + k] + lx[k]; /* (L x)_i */
        x[i * m + k] = xin[i * m + k] - omega * li / di;
      }
    }
  }
  free(lx);
  free(xin);
}

/* C_ij = (sum_k x_ik x_jk)^2 / ((sum_k x_ik^2)(sum_k x_jk^2)) on each edge,
 * S_ij = C_ij / max(max_{s != i} C_is, max_{s != j} C_sj), zero diagonal.
 * Reading: the paper's denominator prints each sum squared; taken unsquared,
 * so that C is the squared cosine of the two test-vector rows and lies in
 * [0, 1] (the affinity of Livne & Brandt that the paper cites). A zero
 * denominator gives C = 0, a zero row maximum gives S = 0. */
void lgref_affinity(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t m,
                    const double* x, double* S) {
  double* rowmax = (double*)xcalloc((size_t)n, sizeof(double));
  for (int64_t i = 0; i < n; ++i) {
    double xi2 = 0.0;
    for (int32_t k = 0; k < m; ++k) xi2 += x[i * m + k] * x[i * m + k];
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      int64_t j = col[p];
      double xj2 = 0.0, xij = 0.0;
      for (int32_t k = 0; k < m; ++k) {
        xj2 += x[j * m + k] * x[j * m + k];
        xij += x[i * m + k] * x[j * m + k];
      }
      double den = xi2 * xj2;
      double c = den > 0.0 ? (xij * xij) / den : 0.0;
      S[p] = c;
      if (c > rowmax[i]) rowmax[i] = c;
    }
  }
  /* C is symmetric, so the column maximum of column j is the row maximum of row j */
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      double mx = rowmax[i] > rowmax[col[p]] ? rowmax[i] : rowmax[col[p]];
      S[p] = mx > 0.0 ? S[p] / mx : 0.0;
    }
  }
  free(rowmax);
}

void lgref_strength(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                    uint64_t seed, int32_t level, int32_t m, int32_t sweeps, double omega, double* S) {
  double* x = (double*)xmalloc(sizeof(double) * (size_t)(n * m));
  lgref_strength_vectors(seed, level, n, m, x);
  lgref_jacobi(n, rowptr, col, w, m, sweeps, omega, x);
  lgref_affinity(n, rowptr, col, m, x, S);
  free(x);
}

/* ------------------------------------------------------------------------ */
/* Aggregation, Section 3.5 (Algorithm 3).  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t state; /* Seed > Undecided > Decided */
  int64_t idx;
  double w;
} agg_trip;

/* (state_a, i_a, w_a) (+)agg (state_b, i_b, w_b): the higher state wins; on
 * equal states the larger weight wins. Reading: equal states and weights go
 * to the smaller index (the paper keeps the left operand, which depends on
 * the order of the reduction). */
static agg_trip agg_oplus(agg_trip a, agg_trip b) {
  if (a.state == b.state) {
    if (a.w > b.w) return a;
    if (a.w < b.w) return b;
    return a.idx <= b.idx ? a : b;
  }
  return a.state > b.state ? a : b;
}

/* Returns the number of aggregates; agg[i] is the aggregate of vertex i,
 * numbered from 0 in ascending order of the aggregate's root vertex.
 * state/votes (may be NULL) receive the final status and vote counts.
 * Readings:
 *  - the filter keeps S_ij >= 0.5^iter (the algorithm's "remove nonzeros <");
 *  - a vertex with votes >= threshold becomes a seed (the prose's "8 or more");
 *  - only Undecided vertices join a seed or vote (the prose); seeds and
 *    decided vertices keep their status;
 *  - every decision of a step reads the status from the start of the step;
 *    votes are tallied, then promotion runs;
 *  - a vertex still Undecided after the last step is its own aggregate. */
int64_t lgref_aggregate(int64_t n, const int64_t* rowptr, const int32_t* col, const double* S,
                        int32_t iters, int32_t threshold, int32_t* agg, int8_t* state_out,
                        int32_t* votes_out) {
  int32_t* st = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)n);
  int64_t* idx = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)n);
  int32_t* nst = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)n);
  int64_t* nidx = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)n);
  int64_t* votes = (int64_t*)xcalloc((size_t)n, sizeof(int64_t));
  int64_t* local_votes = (int64_t*)xcalloc((size_t)n, sizeof(int64_t));
  for (int64_t i = 0; i < n; ++i) { st[i] = LGREF_UNDECIDED; idx[i] = i; }

  double filter = 1.0;
  for (int32_t it = 1; it <= iters; ++it) {
    filter *= 0.5; /* 0.5^iter */
    memcpy(nst, st, sizeof(int32_t) * (size_t)n);
    memcpy(nidx, idx, sizeof(int64_t) * (size_t)n);
    memset(local_votes, 0, sizeof(int64_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
      if (st[i] != LGREF_UNDECIDED) continue;
      /* d_i = (S_filt (+)agg.(x)agg status)_i, starting from (Decided, -1, 0) */
      agg_trip d = {LGREF_DECIDED, -1, 0.0};
      for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        if (!(S[p] >= filter)) continue; /* removed by the filter */
        agg_trip t = {st[col[p]], idx[col[p]], S[p]};
        d = agg_oplus(d, t);
      }
      if (d.state == LGREF_SEED) {
        nst[i] = LGREF_DECIDED; /* joins the neighbouring seed */
        nidx[i] = d.idx;
      } else if (d.state == LGREF_UNDECIDED) {
        local_votes[d.idx] += 1; /* votes for that neighbour */
      }
    }
    for (int64_t i = 0; i < n; ++i) votes[i] += local_votes[i];
    for (int64_t i = 0; i < n; ++i)
      if (votes[i] >= threshold && nst[i] == LGREF_UNDECIDED && nidx[i] == i) nst[i] = LGREF_SEED;
    memcpy(st, nst, sizeof(int32_t) * (size_t)n);
    memcpy(idx, nidx, sizeof(int64_t) * (size_t)n);
  }
  /* aggregates_i = j from status_i = (., j); renumber the roots from 0 in ascending order */
  int64_t* cid = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)n);
  int64_t nc = 0;
  for (int64_t i = 0; i < n; ++i) cid[i] = (idx[i] == i) ? nc++ : -1;
  for (int64_t i = 0; i < n; ++i) agg[i] = (int32_t)cid[idx[i]];
  if (state_out)
    for (int64_t i = 0; i < n; ++i) state_out[i] = (int8_t)st[i];
  if (votes_out)
    for (int64_t i = 0; i < n; ++i) votes_out[i] = (int32_t)votes[i];
  free(cid); free(local_votes); free(votes); free(nidx); free(nst); free(idx); free(st);
  return nc;
}

/* L_{l+1} = R L P with R_{v_j j} = 1 and P = R^T (Section 3.5): the weight
 * between aggregates I != J is the sum of the weights of the edges joining
 * them; edges inside an aggregate drop out of the off-diagonal part. */
lgref_csr* lgref_galerkin(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                          const int32_t* agg, int64_t nc) {
  int64_t nt = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
      if (agg[i] != agg[col[p]]) ++nt;
  trip_t* t = (trip_t*)xmalloc(sizeof(trip_t) * (size_t)(nt ? nt : 1));
  int64_t o = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
      if (agg[i] != agg[col[p]]) {
        t[o].r = agg[i]; t[o].c = agg[col[p]]; t[o].ord = o; t[o].v = w[p];
        ++o;
      }
  lgref_csr* a = csr_from_triplets(nc, t, o);
  free(t);
  return a;
}

/* ------------------------------------------------------------------------ */
/* Smoothing, Section 3.6.                                                   */
/* ------------------------------------------------------------------------ */

/* Number of eigenvalues of the symmetric tridiagonal T(alpha, beta) below x
 * (Sturm sequence of the LDL^T pivots). */
static int32_t sturm_count(int32_t m, const double* a, const double* b, double x) {
  int32_t count = 0;
  double q = 1.0;
  for (int32_t i = 0; i < m; ++i) {
    double off = (i > 0) ? b[i - 1] * b[i - 1] / q : 0.0;
    q = (a[i] - x) - off;
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++count;
  }
  return count;
}

/* Largest eigenvalue of the tridiagonal with diagonal alpha[0..m-1] and
 * off-diagonal beta[0..m-2], by bisection on the Sturm count. */
double lgref_tridiag_max(int32_t m, const double* alpha, const double* beta) {
  double lo = alpha[0], hi = alpha[0];
  for (int32_t i = 0; i < m; ++i) {
    double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i < m - 1 ? fabs(beta[i]) : 0.0);
    if (alpha[i] - r < lo) lo = alpha[i] - r;
    if (alpha[i] + r > hi) hi = alpha[i] + r;
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(m, alpha, beta, mid) == m) hi = mid; /* all eigenvalues below mid */
    else lo = mid;
  }
  return hi;
}

/* Largest eigenvalue of D^-1 L, estimated by `iters` Lanczos steps on the
 * similar symmetric matrix D^-1/2 L D^-1/2 (the paper runs Arnoldi on the
 * Jacobi-preconditioned operator; in the D inner product that operator is
 * symmetric and Arnoldi reduces to Lanczos). Reading: the start vector is
 * uniform in [-1, 1) from stream 8; the recursion stops early once
 * beta_k <= 1e-12 |alpha_k| (invariant subspace found). */
double lgref_lanczos(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                     uint64_t seed, int32_t level, int32_t iters) {
  double* d = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* v = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* vp = (double*)xcalloc((size_t)n, sizeof(double));
  double* t = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* u = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* alpha = (double*)xcalloc((size_t)iters + 1, sizeof(double));
  double* beta = (double*)xcalloc((size_t)iters + 1, sizeof(double));
  lgref_diag(n, rowptr, w, d);
  double nrm = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    v[i] = lgref_uniform(seed, 8, level, i);
    nrm += v[i] * v[i];
  }
  nrm = sqrt(nrm);
  for (int64_t i = 0; i < n; ++i) v[i] /= nrm;
  double bprev = 0.0;
  int32_t m = 0;
  for (int32_t k = 0; k < iters; ++k) {
    /* u = D^-1/2 L D^-1/2 v */
    for (int64_t i = 0; i < n; ++i) t[i] = d[i] > 0.0 ? v[i] / sqrt(d[i]) : 0.0;
    lgref_apply_L(n, rowptr, col, w, t, u);
    for (int64_t i = 0; i < n; ++i) u[i] = d[i] > 0.0 ? u[i] / sqrt(d[i]) : 0.0;
    double a = 0.0;
    for (int64_t i = 0; i < n; ++i) a += v[i] * u[i];
    for (int64_t i = 0; i < n; ++i) u[i] = u[i] - a * v[i] - bprev * vp[i];
    double b = 0.0;
    for (int64_t i = 0; i < n; ++i) b += u[i] * u[i];
    b = sqrt(b);
    alpha[k] = a;
    beta[k] = b;
    m = k + 1;
    if (b <= 1e-12 * fabs(a)) break;
    for (int64_t i = 0; i < n; ++i) {
      vp[i] = v[i];
      v[i] = u[i] / b;
    }
    bprev = b;
  }
  double lam = lgref_tridiag_max(m, alpha, beta);
  free(beta); free(alpha); free(u); free(t); free(vp); free(v); free(d);
  return lam;
}

/* One application of degree-k Chebyshev smoothing on D^-1 L over the
 * interval [lo*lambda, hi*lambda] (Section 3.6; the classical three-term
 * Chebyshev iteration with Jacobi preconditioning), theta and delta the
 * interval's centre and half-width:
 *   d_0 = D^-1 r_0 / theta, rho_0 = delta / theta,
 *   x_{s+1} = x_s + d_s, r_{s+1} = r_s - L d_s,
 *   rho_{s+1} = 1 / (2 theta/delta - rho_s),
 *   d_{s+1} = rho_{s+1} rho_s d_s + (2 rho_{s+1} / delta) D^-1 r_{s+1}.
 * The pre-smoother starts from x = 0 (r_0 = f) and also returns the residual
 * r = f - L x of its result. */
static void cheb_run(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                     const double* dg, double lambda, double lo, double hi, int32_t degree,
                     double* x, double* r, int want_residual) {
  double a = lo * lambda, b = hi * lambda;
  double theta = 0.5 * (b + a), delta = 0.5 * (b - a);
  double sigma = theta / delta;
  double rho = 1.0 / sigma;
  double* d = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* ld = (double*)xmalloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    d[i] = r[i] / (dg[i] * theta);
    x[i] += d[i];
  }
  for (int32_t s = 1; s < degree; ++s) {
    lgref_apply_L(n, rowptr, col, w, d, ld);
    double rho_n = 1.0 / (2.0 * sigma - rho);
    for (int64_t i = 0; i < n; ++i) {
      r[i] -= ld[i];
      d[i] = rho_n * rho * d[i] + (2.0 * rho_n / delta) * r[i] / dg[i];
      x[i] += d[i];
    }
    rho = rho_n;
  }
  if (want_residual) {
    lgref_apply_L(n, rowptr, col, w, d, ld);
    for (int64_t i = 0; i < n; ++i) r[i] -= ld[i];
  }
  free(ld);
  free(d);
}

void lgref_cheb_pre(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                    double lambda, double lo, double hi, int32_t degree,
                    const double* f, double* x, double* r) {
  double* dg = (double*)xmalloc(sizeof(double) * (size_t)n);
  lgref_diag(n, rowptr, w, dg);
  for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = f[i]; }
  cheb_run(n, rowptr, col, w, dg, lambda, lo, hi, degree, x, r, 1);
  free(dg);
}

void lgref_cheb_post(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                     double lambda, double lo, double hi, int32_t degree,
                     const double* f, double* x) {
  double* dg = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* r = (double*)xmalloc(sizeof(double) * (size_t)n);
  lgref_diag(n, rowptr, w, dg);
  lgref_apply_L(n, rowptr, col, w, x, r);
  for (int64_t i = 0; i < n; ++i) r[i] = f[i] - r[i];
  cheb_run(n, rowptr, col, w, dg, lambda, lo, hi, degree, x, r, 0);
  free(r);
  free(dg);
}

/* ------------------------------------------------------------------------ */
/* Coarsest level (Algorithm 1, direct solve): the singular  */
/* Laplacian is inverted on the complement of its null space span(1)        */
/* (Section 2.1), L^+ = (L + 11^T/n)^-1 - 11^T/n, by Cholesky.               */
/* ------------------------------------------------------------------------ */
static int dense_shifted_cholesky(int64_t n, const int64_t* rowptr, const int32_t* col,
                                  const double* w, double* g) {
  /* g = L + 11^T/n, then its lower Cholesky factor in place */
  for (int64_t i = 0; i < n * n; ++i) g[i] = 1.0 / (double)n;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      g[i * n + col[p]] -= w[p];
      g[i * n + i] += w[p];
    }
  }
  for (int64_t j = 0; j < n; ++j) {
    double s = g[j * n + j];
    for (int64_t k = 0; k < j; ++k) s -= g[j * n + k] * g[j * n + k];
    if (!(s > 0.0)) return LGREF_SETUP;
    double gjj = sqrt(s);
    g[j * n + j] = gjj;
    for (int64_t i = j + 1; i < n; ++i) {
      double t = g[i * n + j];
      for (int64_t k = 0; k < j; ++k) t -= g[i * n + k] * g[j * n + k];
      g[i * n + j] = t / gjj;
    }
  }
  return LGREF_OK;
}

static void cholesky_solve(int64_t n, const double* g, double* x) {
  for (int64_t i = 0; i < n; ++i) {
    double t = x[i];
    for (int64_t k = 0; k < i; ++k) t -= g[i * n + k] * x[k];
    x[i] = t / g[i * n + i];
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double t = x[i];
    for (int64_t k = i + 1; k < n; ++k) t -= g[k * n + i] * x[k];
    x[i] = t / g[i * n + i];
  }
}

int lgref_pinv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w, double* out) {
  double* g = (double*)xmalloc(sizeof(double) * (size_t)(n * n));
  double* e = (double*)xmalloc(sizeof(double) * (size_t)n);
  int st = dense_shifted_cholesky(n, rowptr, col, w, g);
  if (st == LGREF_OK) {
    for (int64_t j = 0; j < n; ++j) {
      for (int64_t i = 0; i < n; ++i) e[i] = (i == j) ? 1.0 : 0.0;
      cholesky_solve(n, g, e);
      for (int64_t i = 0; i < n; ++i) out[i * n + j] = e[i] - 1.0 / (double)n;
    }
  }
  free(e);
  free(g);
  return st;
}

/* x = L^+ b (mean-zero), the plain definition of the solve's result. */
int lgref_dense_solve(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                      const double* b, double* x) {
  double* g = (double*)xmalloc(sizeof(double) * (size_t)(n * n));
  double mean = 0.0;
  for (int64_t i = 0; i < n; ++i) mean += b[i];
  mean /= (double)n;
  for (int64_t i = 0; i < n; ++i) x[i] = b[i] - mean;
  int st = dense_shifted_cholesky(n, rowptr, col, w, g);
  if (st == LGREF_OK) {
    cholesky_solve(n, g, x);
    double mx = 0.0;
    for (int64_t i = 0; i < n; ++i) mx += x[i];
    mx /= (double)n;
    for (int64_t i = 0; i < n; ++i) x[i] -= mx;
  }
  free(g);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Hierarchy (Sections 3.4-3.6 and 4).                                       */
/* ------------------------------------------------------------------------ */
static lgref_csr csr_copy_of(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w) {
  lgref_csr a;
  a.n = n;
  a.nnz = rowptr[n];
  a.rowptr = (int64_t*)xmalloc(sizeof(int64_t) * (size_t)(n + 1));
  a.col = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)(a.nnz ? a.nnz : 1));
  a.w = (double*)xmalloc(sizeof(double) * (size_t)(a.nnz ? a.nnz : 1));
  memcpy(a.rowptr, rowptr, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(a.col, col, sizeof(int32_t) * (size_t)a.nnz);
  memcpy(a.w, w, sizeof(double) * (size_t)a.nnz);
  return a;
}

static level_t* push_level(lgref_hier* h, int32_t kind, lgref_csr a) {
  level_t* L = &h->lev[h->nlev++];
  memset(L, 0, sizeof(*L));
  L->kind = kind;
  L->a = a;
  L->d = (double*)xmalloc(sizeof(double) * (size_t)(a.n ? a.n : 1));
  lgref_diag(a.n, a.rowptr, a.w, L->d);
  return L;
}

/* Reading of the level order (the paper: eliminate before every aggregation
 * level when more than 5% of the vertices go, stop at nnz(L) <= 1000):
 * stages alternate [elimination if it passes the gate] then aggregation,
 * the stop test runs before each stage, and nnz(L) counts the diagonal. An
 * aggregation stage that keeps more than stagnation_frac of the vertices, or
 * reaching max_levels, also ends coarsening. A coarsest level larger than
 * max_coarse_n is a setup failure. Random streams use the level's index. */
lgref_hier* lgref_setup(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                        const lgref_opts* o, int* status) {
  int st = lgref_check_graph(n, rowptr, col, w);
  if (st != LGREF_OK) { *status = st; return NULL; }
  lgref_hier* h = (lgref_hier*)xcalloc(1, sizeof(lgref_hier));
  h->o = *o;
  lgref_csr cur = csr_copy_of(n, rowptr, col, w);
  int32_t maxlev = o->max_levels < LGREF_MAX_LEVELS ? o->max_levels : LGREF_MAX_LEVELS;
  for (;;) {
    if ((double)(cur.nnz + cur.n) <= o->coarse_nnz || h->nlev >= maxlev - 1) break;
    /* Reading of the elimination rounds (Section 3.4 finds one round enough;
     * more serve chain-like graphs): up to elim_rounds elimination levels in
     * a row, each while the 5% gate passes, then aggregation. */
    int stop = 0;
    for (int32_t round = 0; o->elim_enable && round < o->elim_rounds; ++round) {
      uint8_t* is_f = (uint8_t*)xmalloc((size_t)cur.n);
      int64_t nf = lgref_elim_select(cur.n, cur.rowptr, cur.col, o->elim_max_degree, o->seed, is_f);
      if (!((double)nf > o->elim_min_frac * (double)cur.n)) {
        free(is_f);
        break;
      }
      int32_t* cmap = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)cur.n);
      lgref_csr* s = lgref_schur(cur.n, cur.rowptr, cur.col, cur.w, is_f, cmap);
      level_t* L = push_level(h, LGREF_LEVEL_ELIM, cur);
      L->map = cmap;
      L->nc = s->n;
      cur = *s;
      free(s);
      free(is_f);
      if ((double)(cur.nnz + cur.n) <= o->coarse_nnz || h->nlev >= maxlev - 1) {
        stop = 1;
        break;
      }
    }
    if (stop) break;
    double* S = (double*)xmalloc(sizeof(double) * (size_t)(cur.nnz ? cur.nnz : 1));
    lgref_strength(cur.n, cur.rowptr, cur.col, cur.w, o->seed, h->nlev, o->strength_vecs,
                   o->strength_sweeps, o->jacobi_omega, S);
    int32_t* agg = (int32_t*)xmalloc(sizeof(int32_t) * (size_t)cur.n);
    int64_t nc = lgref_aggregate(cur.n, cur.rowptr, cur.col, S, o->agg_iters, o->vote_threshold,
                                 agg, NULL, NULL);
    free(S);
    if ((double)nc > o->stagnation_frac * (double)cur.n) {
      free(agg);
      break;
    }
    double lam = lgref_lanczos(cur.n, cur.rowptr, cur.col, cur.w, o->seed, h->nlev, o->eig_iters);
    lgref_csr* c = lgref_galerkin(cur.n, cur.rowptr, cur.col, cur.w, agg, nc);
    level_t* L = push_level(h, LGREF_LEVEL_AGG, cur);
    L->map = agg;
    L->nc = nc;
    L->lambda = lam;
    cur = *c;
    free(c);
  }
  level_t* L = push_level(h, LGREF_LEVEL_COARSEST, cur);
  if (cur.n > o->max_coarse_n) {
    *status = LGREF_SETUP;
    lgref_hier_free(h);
    return NULL;
  }
  L->pinv = (double*)xmalloc(sizeof(double) * (size_t)(cur.n * cur.n));
  st = lgref_pinv(cur.n, cur.rowptr, cur.col, cur.w, L->pinv);
  if (st != LGREF_OK) {
    *status = st;
    lgref_hier_free(h);
    return NULL;
  }
  *status = LGREF_OK;
  return h;
}

void lgref_hier_free(lgref_hier* h) {
  if (!h) return;
  for (int32_t l = 0; l < h->nlev; ++l) {
    csr_release(&h->lev[l].a);
    free(h->lev[l].d);
    free(h->lev[l].map);
    free(h->lev[l].pinv);
  }
  free(h);
}

int32_t lgref_hier_nlevels(const lgref_hier* h) { return h->nlev; }

void lgref_hier_level_info(const lgref_hier* h, int32_t l, int32_t* kind, int64_t* n, int64_t* nnz,
                           int64_t* nc, double* lambda) {
  const level_t* L = &h->lev[l];
  *kind = L->kind;
  *n = L->a.n;
  *nnz = L->a.nnz;
  *nc = L->nc;
  *lambda = L->lambda;
}

void lgref_hier_level_csr(const lgref_hier* h, int32_t l, int64_t* rowptr, int32_t* col, double* w) {
  lgref_csr_copy(&h->lev[l].a, rowptr, col, w);
}

void lgref_hier_level_map(const lgref_hier* h, int32_t l, int32_t* map) {
  const level_t* L = &h->lev[l];
  if (L->map) memcpy(map, L->map, sizeof(int32_t) * (size_t)L->a.n);
}

void lgref_hier_coarsest_pinv(const lgref_hier* h, double* out) {
  const level_t* L = &h->lev[h->nlev - 1];
  memcpy(out, L->pinv, sizeof(double) * (size_t)(L->a.n * L->a.n));
}

/* ------------------------------------------------------------------------ */
/* Multigrid cycle (Algorithm 1, gamma = 1: a V-cycle) with  */
/* x = 0 on entry at every level (it is applied as a preconditioner).        */
/* With the K-cycle (Section 3.7) the system of every aggregation level      */
/* below the first is solved by two FCG iterations preconditioned by that    */
/* level's cycle (so each such level is visited twice per visit of the one   */
/* above: cycle index 2). Readings: the first aggregation level is left to   */
/* the outer Krylov method, and elimination levels, exact, get no Krylov     */
/* (Section 3.7 says so); two iterations, no residual test between them.    */
/* ------------------------------------------------------------------------ */
static void cycle(const lgref_hier* h, int32_t l, const double* f, double* x);

static double dot(int64_t n, const double* a, const double* b);

static int32_t first_agg_level(const lgref_hier* h) {
  for (int32_t l = 0; l < h->nlev; ++l)
    if (h->lev[l].kind == LGREF_LEVEL_AGG) return l;
  return -1;
}

static void cycle_body(const lgref_hier* h, int32_t l, const double* f, double* x);

/* Two FCG iterations on L_l x = f from x = 0, preconditioner B = the level's
 * cycle body (Notay & Vassilevski's K-cycle with two inner iterations):
 *   c1 = B f, v1 = L c1, rho1 = c1.v1, t1 = c1.f / rho1, r1 = f - t1 v1;
 *   c2 = B r1, v2 = L c2, g = c2.v1, rho2 = c2.v2 - g^2 / rho1,
 *   x = (t1 - g (c2.r1) / (rho1 rho2)) c1 + ((c2.r1) / rho2) c2,
 * the second direction being c2 made L-orthogonal to c1. A non-positive
 * rho1 gives x = c1, a non-positive rho2 x = t1 c1. */
static void kcycle_solve(const lgref_hier* h, int32_t l, const double* f, double* x) {
  const level_t* L = &h->lev[l];
  const int64_t n = L->a.n;
  double* c1 = (double*)xcalloc((size_t)n, sizeof(double));
  double* c2 = (double*)xcalloc((size_t)n, sizeof(double));
  double* v1 = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* v2 = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* r1 = (double*)xmalloc(sizeof(double) * (size_t)n);
  cycle_body(h, l, f, c1);
  lgref_apply_L(n, L->a.rowptr, L->a.col, L->a.w, c1, v1);
  const double rho1 = dot(n, c1, v1);
  if (!(rho1 > 0.0)) {
    memcpy(x, c1, sizeof(double) * (size_t)n);
  } else {
    const double t1 = dot(n, c1, f) / rho1;
    for (int64_t i = 0; i < n; ++i) r1[i] = f[i] - t1 * v1[i];
    cycle_body(h, l, r1, c2);
    lgref_apply_L(n, L->a.rowptr, L->a.col, L->a.w, c2, v2);
    const double g = dot(n, c2, v1);
    const double rho2 = dot(n, c2, v2) - g * g / rho1;
    if (!(rho2 > 0.0)) {
      for (int64_t i = 0; i < n; ++i) x[i] = t1 * c1[i];
    } else {
      const double a2 = dot(n, c2, r1);
      const double u1 = t1 - g * a2 / (rho1 * rho2), u2 = a2 / rho2;
      for (int64_t i = 0; i < n; ++i) x[i] = u1 * c1[i] + u2 * c2[i];
    }
  }
  free(r1); free(v2); free(v1); free(c2); free(c1);
}

static void cycle(const lgref_hier* h, int32_t l, const double* f, double* x) {
  if (h->o.kcycle && h->lev[l].kind == LGREF_LEVEL_AGG && l != first_agg_level(h)) {
    kcycle_solve(h, l, f, x);
    return;
  }
  cycle_body(h, l, f, x);
}

static void cycle_body(const lgref_hier* h, int32_t l, const double* f, double* x) {
  const level_t* L = &h->lev[l];
  int64_t n = L->a.n;
  const int64_t* rp = L->a.rowptr;
  const int32_t* cl = L->a.col;
  const double* w = L->a.w;
  if (L->kind == LGREF_LEVEL_COARSEST) {
    for (int64_t i = 0; i < n; ++i) {
      double s = 0.0;
      for (int64_t j = 0; j < n; ++j) s += L->pinv[i * n + j] * f[j];
      x[i] = s;
    }
    return;
  }
  int64_t nc = L->nc;
  double* fc = (double*)xcalloc((size_t)nc, sizeof(double));
  double* xc = (double*)xcalloc((size_t)nc, sizeof(double));
  if (L->kind == LGREF_LEVEL_ELIM) {
    /* Elimination level (Section 3.4): the additive two-level form
     *   x = P x_c + Fsmooth(f),  x_c = cycle(P^T f),
     * P's F rows hold -L_ff^-1 L_fc = w_fc / d_f, its C rows the identity;
     * Fsmooth(f) = f_f / d_f on F and 0 on C. Reading: with x = 0 on entry
     * this equals the multiplicative form, because P^T L Fsmooth(f) = 0. */
    for (int64_t i = 0; i < n; ++i)
      if (L->map[i] >= 0) fc[L->map[i]] += f[i];
    for (int64_t i = 0; i < n; ++i) {
      if (L->map[i] >= 0) continue;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) fc[L->map[cl[p]]] += (w[p] / L->d[i]) * f[i];
    }
    cycle(h, l + 1, fc, xc);
    for (int64_t i = 0; i < n; ++i) {
      if (L->map[i] >= 0) {
        x[i] = xc[L->map[i]];
      } else {
        double s = f[i] / L->d[i];
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += (w[p] / L->d[i]) * xc[L->map[cl[p]]];
        x[i] = s;
      }
    }
  } else {
    /* Aggregation level: pre-smooth, residual, restrict, coarse cycle,
     * prolong, post-smooth. */
    const lgref_opts* o = &h->o;
    double* r = (double*)xmalloc(sizeof(double) * (size_t)n);
    lgref_cheb_pre(n, rp, cl, w, L->lambda, o->cheb_lo, o->cheb_hi, o->cheb_degree, f, x, r);
    for (int64_t i = 0; i < n; ++i) fc[L->map[i]] += r[i]; /* r_c = R r */
    cycle(h, l + 1, fc, xc);
    for (int64_t i = 0; i < n; ++i) x[i] += xc[L->map[i]]; /* x + P x_c */
    lgref_cheb_post(n, rp, cl, w, L->lambda, o->cheb_lo, o->cheb_hi, o->cheb_degree, f, x);
    free(r);
  }
  free(xc);
  free(fc);
}

void lgref_vcycle(const lgref_hier* h, const double* f, double* x) { cycle(h, 0, f, x); }

void lgref_level_cycle(const lgref_hier* h, int32_t l, const double* f, double* x, int32_t body_only) {
  const int64_t n = h->lev[l].a.n;
  for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
  if (body_only) cycle_body(h, l, f, x);
  else cycle(h, l, f, x);
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static void project_mean(int64_t n, double* v) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) m += v[i];
  m /= (double)n;
  for (int64_t i = 0; i < n; ++i) v[i] -= m;
}

/* Conjugate gradients preconditioned by one V-cycle (Section 2.3, 4).
 * Readings: x_0 = 0 with the constant projected out of b (Section 4); the
 * stopping test is ||b - L x||_2 / ||b||_2 <= tol on the recurrence residual,
 * confirmed on the true residual before returning; the true residual
 * replaces the recurrence every 50 iterations; the preconditioned residual
 * has its mean removed; beta takes the Polak-Ribiere form
 * z_new^T (r_new - r_old) / z_old^T r_old, which equals the classical one
 * for a symmetric preconditioner and stays robust when it is not. */
int lgref_pcg(const lgref_hier* h, const double* b, double* x, double tol, int32_t maxit,
              int32_t* iters, double* relres) {
  const level_t* L0 = &h->lev[0];
  int64_t n = L0->a.n;
  const int64_t* rp = L0->a.rowptr;
  const int32_t* cl = L0->a.col;
  const double* w = L0->a.w;
  double* bm = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* r = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* ro = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* z = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* p = (double*)xmalloc(sizeof(double) * (size_t)n);
  double* q = (double*)xmalloc(sizeof(double) * (size_t)n);
  memcpy(bm, b, sizeof(double) * (size_t)n);
  project_mean(n, bm);
  for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = bm[i]; }
  double nb = sqrt(dot(n, bm, bm));
  int st = LGREF_OK;
  int32_t it = 0;
  double rel = 0.0;
  if (nb == 0.0) goto done;
  cycle(h, 0, r, z);
  project_mean(n, z);
  memcpy(p, z, sizeof(double) * (size_t)n);
  double rz = dot(n, r, z);
  rel = 1.0;
  st = LGREF_NOT_CONVERGED;
  for (it = 1; it <= maxit; ++it) {
    lgref_apply_L(n, rp, cl, w, p, q);
    double pq = dot(n, p, q);
    if (!(pq > 0.0) || !isfinite(pq) || !(rz > 0.0)) { st = LGREF_BREAKDOWN; break; }
    double alpha = rz / pq;
    memcpy(ro, r, sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    if (it % 50 == 0) {
      lgref_apply_L(n, rp, cl, w, x, q);
      for (int64_t i = 0; i < n; ++i) r[i] = bm[i] - q[i];
    }
    rel = sqrt(dot(n, r, r)) / nb;
    if (rel <= tol) {
      lgref_apply_L(n, rp, cl, w, x, q);
      for (int64_t i = 0; i < n; ++i) r[i] = bm[i] - q[i];
      rel = sqrt(dot(n, r, r)) / nb;
      if (rel <= tol) { st = LGREF_OK; break; }
    }
    cycle(h, 0, r, z);
    project_mean(n, z);
    double zr_new = dot(n, z, r);
    double zr_old = dot(n, z, ro);
    double beta = (zr_new - zr_old) / rz;
    rz = zr_new;
    for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
  if (it > maxit) it = maxit;
  project_mean(n, x);
done:
  *iters = it;
  *relres = rel;
  free(q); free(p); free(z); free(ro); free(r); free(bm);
  return st;
}
