/*
 * lgref.h -- plain FP64 reference ("the oracle") for the unsmoothed-aggregation
 * multigrid for graph Laplacians of Konolige & Brown, "A Parallel Solver for
 * Graph Laplacians" (PASC'18).
 *
 * TEST INFRASTRUCTURE. This library exists to check the CUDA library against
 * a slow, obviously correct restatement of the paper. Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it. It shares no
 * code, header, table or helper with the CUDA library; the two agree only
 * through the paper and through the published SplitMix64 generator, which
 * each side implements on its own.
 *
 * Conventions. A graph is given as CSR adjacency (rowptr int64[n+1], col
 * int32[nnz], w double[nnz]) with both directions of each edge present,
 * columns strictly ascending in each row, no self-loops and w > 0. The
 * Laplacian is L = D - A with D_ii = sum_j w_ij (Section 2.1); only the
 * off-diagonal weights are stored, the diagonal is always the row sum.
 */
#ifndef LGREF_H
#define LGREF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { LGREF_OK = 0, LGREF_INVALID = 1, LGREF_DISCONNECTED = 2, LGREF_SETUP = 3,
       LGREF_NOT_CONVERGED = 4, LGREF_BREAKDOWN = 5 };
enum { LGREF_LEVEL_AGG = 1, LGREF_LEVEL_ELIM = 2, LGREF_LEVEL_COARSEST = 3 };
enum { LGREF_DECIDED = 0, LGREF_UNDECIDED = 1, LGREF_SEED = 2 };

typedef struct lgref_csr lgref_csr;
typedef struct lgref_hier lgref_hier;

/* Solver constants, with the paper's defaults in the comments. */
typedef struct {
  double coarse_nnz;       /* 1000: coarsest level when nnz(L) <= this (Section 4) */
  double elim_min_frac;    /* 0.05: eliminate only if more than 5% (Section 3.4) */
  double jacobi_omega;     /* 2/3: damping of the strength test-vector smoother */
  double cheb_lo, cheb_hi; /* 0.3, 1.1: Chebyshev interval in units of lambda (Section 3.6) */
  double stagnation_frac;  /* 0.95: a stage keeping more than this share of n ends coarsening */
  uint64_t seed;           /* random streams: elimination hash, test vectors, Lanczos start */
  int32_t max_levels;      /* 64 */
  int32_t elim_max_degree; /* 4 (Section 3.4) */
  int32_t agg_iters;       /* 10 voting iterations (Section 3.5) */
  int32_t vote_threshold;  /* 8 votes make a seed (Section 3.5) */
  int32_t strength_vecs;   /* 4 test vectors (Section 3.5) */
  int32_t strength_sweeps; /* 3 Jacobi sweeps (Section 3.5) */
  int32_t cheb_degree;     /* 2 (Section 4) */
  int32_t eig_iters;       /* 10 (Section 3.6) */
  int32_t max_coarse_n;    /* 4096: largest coarsest level for the dense solve */
  int32_t elim_enable;     /* 1 */
  int32_t kcycle;          /* 0: V-cycle (Section 4's default); 1: K-cycle (Section 3.7) */
  int32_t elim_rounds;     /* 1: elimination rounds before each aggregation (Section 3.4) */
} lgref_opts;

void lgref_opts_default(lgref_opts* o);

/* ---- random streams (SplitMix64, Steele, Lea & Flood 2014) ---- */
uint64_t lgref_splitmix64(uint64_t seed, uint64_t counter);
uint64_t lgref_vertex_hash(uint64_t seed, int64_t id);
double lgref_uniform(uint64_t seed, int32_t stream, int32_t level, int64_t idx);

/* ---- Laplacian basics (Section 2.1) ---- */
int lgref_check_graph(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w);
int64_t lgref_components(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t* label);
void lgref_diag(int64_t n, const int64_t* rowptr, const double* w, double* d);
void lgref_apply_L(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                   const double* x, double* y);

/* ---- low-degree elimination (Section 3.4, Algorithm 2) ---- */
int64_t lgref_elim_select(int64_t n, const int64_t* rowptr, const int32_t* col,
                          int32_t max_degree, uint64_t seed, uint8_t* is_f);
lgref_csr* lgref_schur(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                       const uint8_t* is_f, int32_t* cmap);

/* ---- strength of connection (Section 3.5) ---- */
void lgref_strength_vectors(uint64_t seed, int32_t level, int64_t n, int32_t m, double* y);
void lgref_jacobi(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                  int32_t m, int32_t sweeps, double omega, double* x);
void lgref_affinity(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t m,
                    const double* x, double* S);
void lgref_strength(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                    uint64_t seed, int32_t level, int32_t m, int32_t sweeps, double omega, double* S);

/* ---- aggregation (Section 3.5, Algorithm 3) ---- */
int64_t lgref_aggregate(int64_t n, const int64_t* rowptr, const int32_t* col, const double* S,
                        int32_t iters, int32_t threshold, int32_t* agg, int8_t* state, int32_t* votes);
lgref_csr* lgref_galerkin(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                          const int32_t* agg, int64_t nc);

/* ---- smoothing (Section 3.6) ---- */
double lgref_tridiag_max(int32_t m, const double* alpha, const double* beta);
double lgref_lanczos(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                     uint64_t seed, int32_t level, int32_t iters);
void lgref_cheb_pre(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                    double lambda, double lo, double hi, int32_t degree,
                    const double* f, double* x, double* r);
void lgref_cheb_post(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                     double lambda, double lo, double hi, int32_t degree,
                     const double* f, double* x);

/* ---- coarsest level: dense pseudo-inverse ---- */
int lgref_pinv(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w, double* out);
int lgref_dense_solve(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                      const double* b, double* x);

/* ---- hierarchy, cycle and PCG ---- */
lgref_hier* lgref_setup(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                        const lgref_opts* o, int* status);
void lgref_hier_free(lgref_hier* h);
int32_t lgref_hier_nlevels(const lgref_hier* h);
void lgref_hier_level_info(const lgref_hier* h, int32_t l, int32_t* kind, int64_t* n, int64_t* nnz,
                           int64_t* nc, double* lambda);
void lgref_hier_level_csr(const lgref_hier* h, int32_t l, int64_t* rowptr, int32_t* col, double* w);
void lgref_hier_level_map(const lgref_hier* h, int32_t l, int32_t* map);
void lgref_hier_coarsest_pinv(const lgref_hier* h, double* out);
void lgref_vcycle(const lgref_hier* h, const double* f, double* x);
/* The cycle at level l from x = 0 (what the level above applies to its
 * restricted residual). body_only = 1 leaves out the level's own K-cycle
 * acceleration (its coarser levels keep theirs). */
void lgref_level_cycle(const lgref_hier* h, int32_t l, const double* f, double* x, int32_t body_only);
int lgref_pcg(const lgref_hier* h, const double* b, double* x, double tol, int32_t maxit,
              int32_t* iters, double* relres);

/* ---- CSR results ---- */
int64_t lgref_csr_n(const lgref_csr* a);
int64_t lgref_csr_nnz(const lgref_csr* a);
void lgref_csr_copy(const lgref_csr* a, int64_t* rowptr, int32_t* col, double* w);
void lgref_csr_free(lgref_csr* a);

#ifdef __cplusplus
}
#endif
#endif
