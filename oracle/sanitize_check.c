/*
 * sanitize_check.c -- drives every entry point of the oracle (lgref.h) on a
 * handful of small graphs, for a build under AddressSanitizer and
 * UndefinedBehaviorSanitizer (tests/test_oracle_sanitized.py compiles and runs
 * it). TEST INFRASTRUCTURE, like the oracle itself.
 *
 * It checks only what needs no reference: valid inputs set up and solve to
 * the requested residual (recomputed here), the dense solve agrees with the
 * iterative one on small graphs, invalid and disconnected inputs are refused,
 * and every object is freed (so that the leak checker sees a clean exit). The
 * sanitizers check the memory accesses and arithmetic on the way. Returns 0
 * when every check passed.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "lgref.h"

static int failures = 0;

#define CHECK(cond, ...)                     \
  do {                                       \
    if (!(cond)) {                           \
      fprintf(stderr, "FAIL: " __VA_ARGS__); \
      fprintf(stderr, "\n");                 \
      ++failures;                            \
    }                                        \
  } while (0)

/* ---- graphs: an edge list made into symmetric CSR (duplicates summed) ---- */
typedef struct {
  int64_t n, nnz;
  int64_t* rowptr;
  int32_t* col;
  double* w;
} graph;

typedef struct {
  int32_t r, c;
  double w;
} entry;

static int entry_cmp(const void* a, const void* b) {
  const entry* x = (const entry*)a;
  const entry* y = (const entry*)b;
  if (x->r != y->r) return x->r < y->r ? -1 : 1;
  if (x->c != y->c) return x->c < y->c ? -1 : 1;
  return 0;
}

static graph from_edges(int64_t n, int64_t m, const int32_t* u, const int32_t* v, const double* w) {
  entry* e = (entry*)malloc(sizeof(entry) * (size_t)(2 * m + 1));
  int64_t ne = 0;
  for (int64_t q = 0; q < m; ++q) {
    if (u[q] == v[q]) continue;
    e[ne++] = (entry){u[q], v[q], w[q]};
    e[ne++] = (entry){v[q], u[q], w[q]};
  }
  qsort(e, (size_t)ne, sizeof(entry), entry_cmp);
  graph g;
  g.n = n;
  g.rowptr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  g.col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ne + 1));
  g.w = (double*)malloc(sizeof(double) * (size_t)(ne + 1));
  int64_t k = 0;
  for (int64_t q = 0; q < ne; ++q) {
    if (k > 0 && q > 0 && e[q].r == e[q - 1].r && e[q].c == e[q - 1].c) {
      g.w[k - 1] += e[q].w;
      continue;
    }
    g.col[k] = e[q].c;
    g.w[k] = e[q].w;
    g.rowptr[e[q].r + 1] += 1;
    ++k;
  }
  for (int64_t i = 0; i < n; ++i) g.rowptr[i + 1] += g.rowptr[i];
  g.nnz = k;
  free(e);
  return g;
}

static void graph_free(graph* g) {
  free(g->rowptr);
  free(g->col);
  free(g->w);
}

static uint64_t lcg_state = 12345;
static double lcg_uniform(void) { /* in [0, 1) */
  lcg_state = lcg_state * 6364136223846793005ull + 1442695040888963407ull;
  return (double)(lcg_state >> 11) * 0x1.0p-53;
}

static graph grid(int nx, int ny, int nz, int spread) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t mmax = 3 * n;
  int32_t* u = (int32_t*)malloc(sizeof(int32_t) * (size_t)mmax);
  int32_t* v = (int32_t*)malloc(sizeof(int32_t) * (size_t)mmax);
  double* w = (double*)malloc(sizeof(double) * (size_t)mmax);
  int64_t m = 0;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const int32_t id = (int32_t)((z * ny + y) * nx + x);
        const int32_t nb[3] = {x + 1 < nx ? id + 1 : -1, y + 1 < ny ? id + nx : -1, z + 1 < nz ? id + nx * ny : -1};
        for (int d = 0; d < 3; ++d) {
          if (nb[d] < 0) continue;
          u[m] = id;
          v[m] = nb[d];
          w[m] = spread ? 0.5 + lcg_uniform() : 1.0;
          ++m;
        }
      }
  graph g = from_edges(n, m, u, v, w);
  free(u);
  free(v);
  free(w);
  return g;
}

static graph random_graph(int64_t n, int64_t extra) { /* a spanning path plus random edges */
  const int64_t m = n - 1 + extra;
  int32_t* u = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  int32_t* v = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  double* w = (double*)malloc(sizeof(double) * (size_t)m);
  for (int64_t q = 0; q < n - 1; ++q) {
    u[q] = (int32_t)q;
    v[q] = (int32_t)(q + 1);
    w[q] = 0.5 + lcg_uniform();
  }
  for (int64_t q = n - 1; q < m; ++q) {
    u[q] = (int32_t)(lcg_uniform() * (double)n);
    v[q] = (int32_t)(lcg_uniform() * (double)n);
    w[q] = 0.5 + lcg_uniform();
  }
  graph g = from_edges(n, m, u, v, w);
  free(u);
  free(v);
  free(w);
  return g;
}

static graph star(int64_t leaves) {
  int32_t* u = (int32_t*)malloc(sizeof(int32_t) * (size_t)leaves);
  int32_t* v = (int32_t*)malloc(sizeof(int32_t) * (size_t)leaves);
  double* w = (double*)malloc(sizeof(double) * (size_t)leaves);
  for (int64_t q = 0; q < leaves; ++q) {
    u[q] = 0;
    v[q] = (int32_t)(q + 1);
    w[q] = 1.0;
  }
  graph g = from_edges(leaves + 1, leaves, u, v, w);
  free(u);
  free(v);
  free(w);
  return g;
}

/* ---- checks ---- */
static double relres(const graph* g, const double* b, const double* x) {
  double* y = (double*)malloc(sizeof(double) * (size_t)g->n);
  lgref_apply_L(g->n, g->rowptr, g->col, g->w, x, y);
  double mean = 0.0;
  for (int64_t i = 0; i < g->n; ++i) mean += b[i];
  mean /= (double)g->n;
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < g->n; ++i) {
    const double bm = b[i] - mean;
    num += (bm - y[i]) * (bm - y[i]);
    den += bm * bm;
  }
  free(y);
  return den > 0.0 ? sqrt(num / den) : 0.0;
}

static void check_steps(const char* name, const graph* g) {
  const int64_t n = g->n;
  int32_t* label = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  CHECK(lgref_components(n, g->rowptr, g->col, label) == 1, "%s: one component", name);
  free(label);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  lgref_diag(n, g->rowptr, g->w, d);
  free(d);
  uint8_t* is_f = (uint8_t*)malloc((size_t)n);
  int32_t* cmap = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  lgref_elim_select(n, g->rowptr, g->col, 4, 0x5eed, is_f);
  lgref_csr* s = lgref_schur(n, g->rowptr, g->col, g->w, is_f, cmap);
  if (s) lgref_csr_free(s);
  free(is_f);
  free(cmap);
  double* S = (double*)malloc(sizeof(double) * (size_t)(g->nnz + 1));
  lgref_strength(n, g->rowptr, g->col, g->w, 0x5eed, 0, 4, 3, 2.0 / 3.0, S);
  int32_t* agg = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int8_t* state = (int8_t*)malloc((size_t)n);
  int32_t* votes = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  const int64_t nc = lgref_aggregate(n, g->rowptr, g->col, S, 10, 8, agg, state, votes);
  CHECK(nc >= 1 && nc <= n, "%s: aggregate count %lld", name, (long long)nc);
  lgref_csr* c = lgref_galerkin(n, g->rowptr, g->col, g->w, agg, nc);
  if (c) lgref_csr_free(c);
  free(S);
  free(agg);
  free(state);
  free(votes);
  const double lam = lgref_lanczos(n, g->rowptr, g->col, g->w, 0x5eed, 0, 10);
  CHECK(lam > 0.0 && lam <= 2.0 + 1e-9, "%s: lambda %g", name, lam);
  double* f = (double*)malloc(sizeof(double) * (size_t)n);
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) f[i] = lcg_uniform() - 0.5;
  lgref_cheb_pre(n, g->rowptr, g->col, g->w, lam, 0.3, 1.1, 2, f, x, r);
  lgref_cheb_post(n, g->rowptr, g->col, g->w, lam, 0.3, 1.1, 2, f, x);
  free(f);
  free(x);
  free(r);
}

static void check_solve(const char* name, const graph* g, const lgref_opts* o) {
  const int64_t n = g->n;
  int st = -1;
  lgref_hier* h = lgref_setup(n, g->rowptr, g->col, g->w, o, &st);
  CHECK(h != NULL && st == LGREF_OK, "%s: setup status %d", name, st);
  if (!h) return;
  const int32_t nl = lgref_hier_nlevels(h);
  for (int32_t l = 0; l < nl; ++l) {
    int32_t kind;
    int64_t ln, lnnz, lnc;
    double lam;
    lgref_hier_level_info(h, l, &kind, &ln, &lnnz, &lnc, &lam);
    int64_t* rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ln + 1));
    int32_t* cl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(lnnz + 1));
    double* w = (double*)malloc(sizeof(double) * (size_t)(lnnz + 1));
    lgref_hier_level_csr(h, l, rp, cl, w);
    if (kind != LGREF_LEVEL_COARSEST) {
      int32_t* map = (int32_t*)malloc(sizeof(int32_t) * (size_t)ln);
      lgref_hier_level_map(h, l, map);
      free(map);
    } else {
      double* p = (double*)malloc(sizeof(double) * (size_t)(ln * ln));
      lgref_hier_coarsest_pinv(h, p);
      free(p);
    }
    double* f = (double*)malloc(sizeof(double) * (size_t)ln);
    double* x = (double*)malloc(sizeof(double) * (size_t)ln);
    for (int64_t i = 0; i < ln; ++i) f[i] = lcg_uniform() - 0.5;
    lgref_level_cycle(h, l, f, x, 0);
    lgref_level_cycle(h, l, f, x, 1);
    free(f);
    free(x);
    free(rp);
    free(cl);
    free(w);
  }
  double* b = (double*)malloc(sizeof(double) * (size_t)n);
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) b[i] = lcg_uniform() - 0.5;
  lgref_vcycle(h, b, x);
  int32_t it = 0;
  double rel = 1.0;
  st = lgref_pcg(h, b, x, 1e-10, 500, &it, &rel);
  CHECK(st == LGREF_OK, "%s: pcg status %d after %d iterations", name, st, it);
  const double rr = relres(g, b, x);
  CHECK(rr <= 1e-10 * 1.0001, "%s: residual %g", name, rr);
  if (n <= 400) {
    double* xd = (double*)malloc(sizeof(double) * (size_t)n);
    CHECK(lgref_dense_solve(n, g->rowptr, g->col, g->w, b, xd) == LGREF_OK, "%s: dense solve", name);
    double mx = 0.0, md = 0.0, num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      mx += x[i];
      md += xd[i];
    }
    mx /= (double)n;
    md /= (double)n;
    for (int64_t i = 0; i < n; ++i) {
      num += ((x[i] - mx) - (xd[i] - md)) * ((x[i] - mx) - (xd[i] - md));
      den += (xd[i] - md) * (xd[i] - md);
    }
    CHECK(num <= 1e-12 * den, "%s: iterative and dense solutions differ (%g)", name, sqrt(num / den));
    double* p = (double*)malloc(sizeof(double) * (size_t)(n * n));
    CHECK(lgref_pinv(n, g->rowptr, g->col, g->w, p) == LGREF_OK, "%s: pinv", name);
    free(p);
    free(xd);
  }
  free(b);
  free(x);
  lgref_hier_free(h);
}

static void check_refusals(void) {
  graph g = grid(4, 4, 1, 0);
  /* an asymmetric weight */
  double* w = (double*)malloc(sizeof(double) * (size_t)g.nnz);
  memcpy(w, g.w, sizeof(double) * (size_t)g.nnz);
  w[0] *= 2.0;
  CHECK(lgref_check_graph(g.n, g.rowptr, g.col, w) != LGREF_OK, "asymmetric weights accepted");
  int st = -1;
  lgref_opts o;
  lgref_opts_default(&o);
  lgref_hier* h = lgref_setup(g.n, g.rowptr, g.col, w, &o, &st);
  CHECK(h == NULL && st == LGREF_INVALID, "asymmetric graph set up (status %d)", st);
  if (h) lgref_hier_free(h);
  free(w);
  graph_free(&g);
  /* two components */
  const int32_t u[2] = {0, 2}, v[2] = {1, 3};
  const double wt[2] = {1.0, 1.0};
  graph two = from_edges(4, 2, u, v, wt);
  h = lgref_setup(two.n, two.rowptr, two.col, two.w, &o, &st);
  CHECK(h == NULL && st == LGREF_DISCONNECTED, "disconnected graph set up (status %d)", st);
  if (h) lgref_hier_free(h);
  graph_free(&two);
}

int main(void) {
  graph gs[6];
  const char* names[6] = {"grid2d_20x17", "grid3d_7", "random_600", "star_40", "path_300", "edge_2"};
  gs[0] = grid(20, 17, 1, 1);
  gs[1] = grid(7, 7, 7, 0);
  gs[2] = random_graph(600, 1500);
  gs[3] = star(40);
  gs[4] = grid(300, 1, 1, 1);
  gs[5] = grid(2, 1, 1, 0);
  for (int q = 0; q < 6; ++q) {
    CHECK(lgref_check_graph(gs[q].n, gs[q].rowptr, gs[q].col, gs[q].w) == LGREF_OK, "%s: check_graph", names[q]);
    check_steps(names[q], &gs[q]);
    lgref_opts o;
    lgref_opts_default(&o);
    o.coarse_nnz = 100.0; /* several levels even on these small graphs */
    check_solve(names[q], &gs[q], &o);
    o.kcycle = 1;
    check_solve(names[q], &gs[q], &o);
    o.kcycle = 0;
    o.elim_rounds = 4;
    o.cheb_degree = 3;
    check_solve(names[q], &gs[q], &o);
    graph_free(&gs[q]);
  }
  check_refusals();
  if (failures) {
    fprintf(stderr, "%d check(s) failed\n", failures);
    return 1;
  }
  printf("all oracle checks passed under the sanitizers\n");
  return 0;
}
