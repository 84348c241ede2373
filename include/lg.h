/*
 * lg.h -- C ABI of the GB300 (sm_103a) multigrid solver for graph Laplacians.
 *
 * The method is the unsmoothed-aggregation multigrid with low-degree
 * elimination of Konolige & Brown, "A Parallel Solver for Graph Laplacians"
 * (PASC'18): the setup builds a hierarchy by low-degree elimination
 * (Section 3.4, Algorithm 2), affinity strength of connection and voting
 * aggregation (Section 3.5, Algorithm 3), and Galerkin products R L P; the
 * solve is conjugate gradients preconditioned by one V-cycle (Section 2.3,
 * Algorithm 1) or K-cycle (Section 3.7) with degree-2 Chebyshev smoothing
 * (Sections 3.6 and 4).
 *
 * Problem statement (Section 2.1): solve L x = b for the Laplacian L = D - A
 * of a weighted, undirected, connected graph with positive weights. L is
 * singular with null space span(1); b has its mean removed inside the
 * library and the returned x has mean zero.
 *
 * Conventions for every entry point:
 *  - Graphs are CSR adjacency: rowptr int64[n+1], col int32[nnz], w double[nnz],
 *    both directions of each edge stored with equal weight, columns strictly
 *    ascending within a row, no self-loops, 0 < w < inf. The diagonal of L is
 *    never passed: it is the row sum of w.
 *  - Pointers may be host or device memory unless the entry point says
 *    otherwise; the library finds out which with cudaPointerGetAttributes.
 *    Host arrays may be pageable or pinned.
 *  - The caller owns every array it passes. The library copies or reads
 *    inputs during the call and keeps no pointer to them after it returns.
 *  - Every call returns an lg status code (LG_OK = 0) and never aborts the
 *    process. On an error the output arrays hold unspecified values unless
 *    stated otherwise.
 *  - Work runs on the stream given in lg_options (a cudaStream_t), or on a
 *    stream the handle owns when that is NULL. Calls that return results to
 *    the host synchronise that stream before returning.
 *  - A handle is not thread-safe: one host thread at a time per handle. The
 *    server (lg_serve_*) is thread-safe.
 */
#ifndef LG_H
#define LG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
enum {
  LG_OK = 0,
  LG_ERR_INVALID = 1,        /* malformed CSR, asymmetric, w <= 0, n < 1, bad argument */
  LG_ERR_DISCONNECTED = 2,   /* graph has more than one connected component */
  LG_ERR_SETUP = 3,          /* coarsening stalled with a coarsest level above max_coarse_n */
  LG_ERR_NOMEM = 4,          /* device allocation or HBM budget exhausted */
  LG_ERR_NOT_CONVERGED = 5,  /* max_iter reached; x holds the last iterate, info->relres its residual */
  LG_ERR_BREAKDOWN = 6,      /* PCG scalar non-finite or r^T z <= 0 */
  LG_ERR_TIMEOUT = 7,        /* a bounded device-side retry loop or host wait gave up */
  LG_ERR_CUDA = 8,           /* a CUDA runtime call failed */
  LG_ERR_BUSY = 9            /* the server has no free slot or budget; retry later */
};

enum { LG_FP64 = 0, LG_FP32_HIER = 1 };             /* precision of the V-cycle */
enum { LG_AUTO = -1, LG_HOST = 0, LG_DEVICE = 1 };  /* memory space of caller pointers */
enum { LG_LEVEL_AGG = 1, LG_LEVEL_ELIM = 2, LG_LEVEL_COARSEST = 3 };
enum { LG_DECIDED = 0, LG_UNDECIDED = 1, LG_SEED = 2 }; /* aggregation states, Section 3.5 */

typedef struct lg_hier* lg_handle;
typedef struct lg_server* lg_server_t;

/* Solver options. lg_options_default fills the paper's constants. */
typedef struct {
  double coarse_nnz;        /* 1000: a level with nnz(L) (diagonal included) <= this is the
                               coarsest (Section 4) */
  double elim_min_frac;     /* 0.05: eliminate only if more than this share goes (Section 3.4) */
  double jacobi_omega;      /* 2/3: damping of the strength test-vector Jacobi sweeps */
  double cheb_lo, cheb_hi;  /* 0.3, 1.1: Chebyshev interval in units of lambda_max (Section 3.6) */
  double stagnation_frac;   /* 0.95: an aggregation keeping more than this share of the
                               vertices ends coarsening */
  uint64_t seed;            /* random streams: elimination hash, test vectors, Lanczos start */
  void* stream;             /* cudaStream_t to run on, or NULL for a stream owned by the handle */
  int32_t precision;        /* LG_FP64 or LG_FP32_HIER: V-cycle precision used by lg_solve */
  int32_t max_levels;       /* 64 */
  int32_t max_iter;         /* 500 PCG iterations */
  int32_t elim_enable;      /* 1 */
  int32_t elim_max_degree;  /* 4 (Section 3.4) */
  int32_t agg_iters;        /* 10 voting iterations (Section 3.5) */
  int32_t vote_threshold;   /* 8 votes make a seed (Section 3.5) */
  int32_t strength_vecs;    /* 4 test vectors, at most 7 (Section 3.5) */
  int32_t strength_sweeps;  /* 3 Jacobi sweeps (Section 3.5) */
  int32_t cheb_degree;      /* 2 (Section 4); 1..8 */
  int32_t eig_iters;        /* 10 Lanczos steps (Section 3.6) */
  int32_t max_coarse_n;     /* 4096: largest coarsest level for the dense pseudo-inverse */
  int32_t residual_replace; /* 50: PCG recomputes r = b - L x every this many iterations */
  int32_t memory_space;     /* LG_AUTO: detect; LG_HOST / LG_DEVICE force the interpretation */
  int32_t use_graphs;       /* 1: replay the preconditioned iteration as a captured CUDA graph */
  int32_t autotune;         /* 1: time the row-binning choices of each large level at setup and keep
                               the fastest (cached per level shape for the life of the process);
                               0: a fixed rule */
  int32_t reorder;          /* 1: renumber the vertices by descending degree before the setup (ties
                               by id), so the gathered values of high-degree vertices share cache
                               lines, and the row classes are contiguous; 2: a random ordering
                               (Section 3.3, which uses it to balance a 2D distribution; a hash of
                               the seed and the vertex id); 0: keep the caller's numbering. Solves
                               take and return vectors in the caller's numbering either way. */
  int32_t kcycle;           /* 0: V-cycle (Section 4's default). 1: K-cycle (Section 3.7): every
                               aggregation level below the first solves its system by two FCG
                               iterations preconditioned by its own cycle (the first is accelerated
                               by the outer iteration; elimination levels are exact). The outer
                               iteration's Polak-Ribiere beta makes it flexible CG. Multi-column
                               solves then run their columns one at a time. */
  int32_t elim_rounds;      /* 1 (Section 3.4 finds one round enough): up to this many elimination
                               levels in a row before each aggregation, each while more than
                               elim_min_frac of the vertices go; more rounds serve chain-like graphs */
  int32_t lp_residual;      /* 1: each aggregation level of at least 4096 vertices also stores
                               W = L P off the own aggregate
                               (n x n_c, row i: sum of w_ij over the neighbours j in aggregate a),
                               and lg_solve's cycle starts post-smoothing (Section 3.6) from
                               r_0 = r_pre - L P x_c, r_pre the pre-smoothing residual, which
                               equals f - L (x + P x_c) and gathers from the short coarse vector;
                               the prolongation x += P x_c joins that pass. 0: r_0 = f - L x. */
  int32_t fp32_only;        /* 0. 1 (with precision LG_FP32_HIER at setup): once the hierarchy is
                               built, release what an FP32-hierarchy solve never reads: the FP64
                               weights, row sums and W = L P weights of every level but the finest
                               operator (the outer FP64 PCG applies L_0 in FP64), the FP64
                               elimination coefficients, and the kept vertices' rows of elimination
                               levels below the finest. The handle then serves FP32-hierarchy solves
                               only: lg_set_precision(LG_FP64), FP64 lg_vcycle / lg_vcycle_batch /
                               lg_level_apply, lg_level_copy of a released level, lg_save, and
                               registration with an FP64 server return LG_ERR_INVALID. */
  int32_t const_weights;    /* 1: when every weight of the finest operator is the same value (an
                               unweighted graph), keep its pattern only and apply the value as a
                               constant: each pass over L_0 streams the 4-byte column ids alone
                               (not 8 + 4 bytes per entry in FP64). Solves give bitwise the same
                               results either way. 0: always store the weights. */
  int32_t row_sorts;        /* 1: the setup's sparse products whose entries are produced row by row
                               (the vertex renumbering, the Schur complement, W = L P) sort each
                               row's entries on its own instead of sorting all entries by (row,
                               column) with a global radix sort; the order, and so every sum and
                               the hierarchy, is the same bit for bit. 0: global sorts. */
} lg_options;

/* Logging: with the environment variable LG_LOG naming a file, lg_setup and
 * every right-hand side solved by lg_solve, lg_solve_batch or lg_solve_many
 * append one JSON line to it (the figures of lg_info, and WDA). */

/* Result of a setup or a solve. */
typedef struct {
  double relres;         /* ||b - L x||_2 / ||b||_2 of the returned x, recomputed in FP64 */
  double op_complexity;  /* sum_l nnz(L_l) / nnz(L_0), diagonals included */
  double setup_ms;       /* device time of lg_setup */
  double solve_ms;       /* device time of this solve (or batch) */
  double work_units;     /* solve work in finest-residual units (Section 2.3.1: WDA = work_units /
                            -log10(relres)), counted from operator nonzeros: per iteration one
                            level-0 operator application plus the cycle (2 deg (nnz_l + n_l) + 2 n_l
                            per aggregation-body visit, 2 nnz_F + n_c + n_l per elimination visit,
                            n_c^2 for the coarsest solve; a K-cycle level is two bodies plus two
                            operator applications), in units of nnz(L_0) + n_0 */
  int64_t nnz;           /* nnz(L_0) = stored off-diagonal entries + n */
  int32_t status;        /* lg status of this result */
  int32_t iterations;    /* PCG iterations */
  int32_t levels;        /* hierarchy levels, coarsest included */
  int32_t reserved;
} lg_info;

/* Fill *o with the defaults above. */
int lg_options_default(lg_options* o);

/* Static string for a status code. */
const char* lg_error_string(int status);

/* Detail of the last error raised on the calling host thread (never NULL). */
const char* lg_last_error_detail(void);

/*
 * Build the multigrid hierarchy of the Laplacian of the graph (rowptr, col, w)
 * with n vertices (Sections 3.4-3.6, 4). Validates the graph (LG_ERR_INVALID,
 * LG_ERR_DISCONNECTED), then alternates [low-degree elimination when more
 * than elim_min_frac of the vertices go] and [aggregation + Galerkin
 * product] until nnz(L) <= coarse_nnz, estimates lambda_max(D^-1 L) on each
 * aggregation level with eig_iters Lanczos steps, and forms the coarsest
 * level's dense FP64 pseudo-inverse. Both an FP64 and an FP32 copy of the
 * level operators are kept. On success *out owns all device memory of the
 * hierarchy until lg_destroy. The graph arrays are only read during the call.
 */
int lg_setup(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
             const lg_options* opts, lg_handle* out);

/* Release a hierarchy and everything it owns. NULL is accepted. */
void lg_destroy(lg_handle h);

/*
 * Solve L x = b (b and x: n doubles each, host or device) with CG
 * preconditioned by one V-cycle per iteration (Sections 2.3 and 4) to
 * ||b - L x|| / ||b|| <= tol in FP64. The cycle runs in the handle's
 * precision; outer dot products, residuals, the mean projection and the
 * coarsest solve are FP64. The constant is projected out of b first; x is
 * returned with mean zero. info (may be NULL) receives iterations, the true
 * relative residual and timings. Returns LG_ERR_NOT_CONVERGED after max_iter
 * iterations with the last iterate in x.
 */
int lg_solve(lg_handle h, const double* b, double* x, double tol, lg_info* info);

/*
 * Solve k systems L X[:, c] = B[:, c] at once (1 <= k <= 32). B and X are
 * column-major n x k blocks with leading dimensions ldb, ldx >= n. The V-cycle
 * runs on all k columns together as a multi-right-hand-side sweep; each column
 * has its own CG scalars and stops on its own tolerance (converged columns
 * are frozen). infos (may be NULL) receives k entries; the return value is
 * LG_OK only if every column converged.
 */
int lg_solve_batch(lg_handle h, int32_t k, const double* B, int64_t ldb, double* X, int64_t ldx,
                   double tol, lg_info* infos);

/*
 * Save and load a hierarchy. lg_save writes h's hierarchy to the file `path`
 * (created or truncated): every level's arrays, the row-binning choices, the
 * Chebyshev constants, the vertex order and the setup options, in host byte
 * order, so that a hierarchy can leave the device and come back without its
 * setup. lg_load builds a new handle from such a file; solves on it return
 * the same results, bit for bit, as on the saved handle. opts (may be NULL)
 * gives the new handle's stream and memory_space; every other option comes
 * from the file.
 * Errors: LG_ERR_INVALID for a NULL argument, a file that cannot be opened,
 * written or read, or one that is not a complete hierarchy file of this
 * format (a wrong header is found before any device work); LG_ERR_NOMEM and
 * LG_ERR_CUDA as for lg_setup.
 */
int lg_save(lg_handle h, const char* path);
int lg_load(const char* path, const lg_options* opts, lg_handle* out);

/* Stored entries of level l's W = L P operator (see lp_residual); 0 when the
 * level has none (elimination and coarsest levels, or lp_residual = 0). */
int lg_level_lp_nnz(lg_handle h, int32_t l, int64_t* nnz);

/* Set the V-cycle precision (LG_FP64 or LG_FP32_HIER) used by later solves. */
int lg_set_precision(lg_handle h, int32_t precision);

/*
 * Many independent solves in one kernel launch: for g = 0 .. count-1, solve
 * L_g x[g] = b[g] on hierarchy hs[g] exactly as lg_solve would (Section 4's
 * PCG, each handle's own precision, cycle and max_iter), but with the whole
 * solve of one graph run by one thread block, so that graphs of a few
 * thousand vertices, which leave lg_solve bound by kernel-launch latency,
 * share one launch. Results agree with lg_solve's to rounding (the order of
 * additions in the reductions differs).
 *   hs:    count distinct handles, all on the current device, each with
 *          nnz(L_0) <= 2^22 and at most 64 levels; x[g] and b[g] hold that
 *          handle's n doubles (host or device, per its memory_space) and
 *          must not overlap other graphs' vectors.
 *   infos: NULL or count entries (solve_ms: the whole launch).
 * Uses each handle's default workspace: no other call may use these handles
 * meanwhile. Host vectors pass through one pinned staging buffer of the
 * process (grown on demand, kept until exit), so concurrent calls from
 * several threads run one after another. Returns LG_OK if every solve
 * converged, else the first failing
 * status in argument order. LG_ERR_INVALID for count < 1, a NULL or repeated
 * handle or vector, tol <= 0, or a graph over the limits above.
 */
int lg_solve_many(int32_t count, const lg_handle* hs, const double* const* b, double* const* x, double tol,
                  lg_info* infos);

/* Hierarchy summary: levels, op_complexity, setup_ms, nnz. */
int lg_hier_info(lg_handle h, lg_info* info);

/* Device bytes held by the hierarchy (level operators, transfer maps, the
 * coarsest pseudo-inverse) and by its solve workspace. */
int lg_hier_bytes(lg_handle h, int64_t* hierarchy_bytes, int64_t* workspace_bytes);

/*
 * Describe level l (0 = finest): kind (LG_LEVEL_*), vertices n, stored
 * off-diagonal entries nnz, size nc of level l+1 (0 for the coarsest) and the
 * Chebyshev eigenvalue estimate lambda (aggregation levels, else 0).
 */
int lg_level_info(lg_handle h, int32_t l, int32_t* kind, int64_t* n, int64_t* nnz, int64_t* nc,
                  double* lambda);

/*
 * Copy level l's FP64 operator to HOST arrays rowptr[n+1], col[nnz], w[nnz]
 * (any may be NULL) and its transfer map to map[n] (may be NULL):
 * aggregation levels give the aggregate of each vertex; elimination levels
 * give the coarse id of each kept vertex and -1 for each eliminated one.
 */
int lg_level_copy(lg_handle h, int32_t l, int64_t* rowptr, int32_t* col, double* w, int32_t* map);

/* Vertex numbering of level 0: perm[i] = the caller's id of level-0 vertex i
 * (the identity unless the options asked for reordering). HOST array of n. */
int lg_permutation(lg_handle h, int32_t* perm);

/* Copy the coarsest level's dense FP64 pseudo-inverse (n_c x n_c, row-major) to host memory. */
int lg_coarsest_pinv(lg_handle h, double* out);

/*
 * Apply one V-cycle of the hierarchy to f (n doubles, host or device) in the
 * given precision, starting from x = 0: x = M f (Algorithm 1,
 * gamma = 1). No mean projection.
 */
int lg_vcycle(lg_handle h, const double* f, double* x, int32_t precision);

/*
 * y = L_l x for level l (0 = finest; not the coarsest) of the hierarchy, in the
 * level's own vertex numbering (lg_level_copy gives its CSR), with the row
 * plan the cycle uses: the operator pass of Section 3.6's smoother on its
 * own, for measuring or profiling one level. precision LG_FP64: x, y are
 * DEVICE doubles (standard form d_i x_i - sum_j w_ij x_j); LG_FP32_HIER:
 * DEVICE floats (difference form sum_j w_ij (x_i - x_j)), n_l values each.
 * Uses the handle's default workspace (no concurrent lg_solve on the handle)
 * and synchronises the handle's stream. LG_ERR_INVALID for a bad level or a
 * precision whose weights the handle does not hold.
 */
int lg_level_apply(lg_handle h, int32_t level, int32_t precision, const void* x, void* y);

/* ---- instrumentation ---- */

/* Kernels the library has launched in this process so far. */
uint64_t lg_kernel_launches(void);

/* Per-kernel timing of the operator passes: the row passes that apply a
 * level's Laplacian (the PCG product and true residual on level 0, the
 * Chebyshev steps of every aggregation level) and, counted apart, the passes
 * over W = L P that start post-smoothing (see lp_residual). When enabled on a
 * handle, each such launch of lg_solve is bracketed by CUDA events on the
 * handle's stream. lg_profile_read returns, for the Laplacian passes of one
 * level l (level = l), the W passes of level l (level = nlevels + l), or all
 * of them (level = -1), the launches, their summed device time and their
 * summed algorithmic bytes (compulsory traffic: the CSR arrays once, the
 * gathered vector once, each epilogue vector stream once). lg_profile also
 * clears the counters. */
typedef struct {
  double total_ms;         /* summed event-measured device time of those launches */
  double bytes;            /* summed algorithmic bytes */
  int64_t launches;
  int64_t reserved;
} lg_kernel_profile;

int lg_profile(lg_handle h, int32_t enable);

/* Launch plan of level l's operator passes: out[0] = entries per lane E of
 * the row binning (a row of class c, E 2^(c-1) < deg <= E 2^c, is served by
 * 2^c lanes), out[1] = rows served by groups of 1..16 lanes, out[2] = rows
 * served by a whole warp, out[3] = long rows (above 2048 entries), out[4] =
 * their chunks, out[5] = blocks of one pass served by chunks, out[6] = tiles
 * of the column-segmented long-row pass (0: the long rows go by chunks; else
 * they go column-segmented, with the gathered vector staged in shared memory,
 * in passes that reduce nothing across the grid), out[7] = 1 when the level's
 * weights are one constant kept in place of its weight arrays (option
 * const_weights), else 0. */
int lg_level_plan(lg_handle h, int32_t l, int64_t out[8]);
/* Multi-column schedule of level l (the SpMM passes of lg_solve_batch and the
 * server), as the autotuner chose it: out[0] = entries per stretch of a long
 * row in the operator passes (64, 256 or 1024, timed per level shape; 0 when
 * the level has no multi-column operator pass), out[1] = their virtual rows,
 * out[2] and out[3] the same for the W = L P pass. LG_ERR_INVALID until the
 * first multi-column solve (or server registration) has built the plans.
 * The paper has no counterpart (its solver applies one right-hand side). */
int lg_batch_plan(lg_handle h, int32_t l, int64_t out[4]);
int lg_profile_read(lg_handle h, int32_t level, lg_kernel_profile* out);

/* One multi-column V-cycle on k right-hand sides at once (1 <= k <= 32): X =
 * M F with F, X column-major n x k blocks (leading dimensions ldf, ldx >= n,
 * host or device), the same preconditioner as lg_vcycle applied to every
 * column, run as SpMM passes. */
int lg_vcycle_batch(lg_handle h, int32_t k, const double* F, int64_t ldf, double* X, int64_t ldx,
                    int32_t precision);

/* ---- single steps on caller data (DEVICE pointers only, on `stream`) ----
 * These run one stage of the setup on an arbitrary graph so that each stage
 * can be checked on its own. The graph must satisfy the conventions above
 * (not re-validated). They synchronise `stream` before returning. */

/* y = L x (Section 2.1) in FP64, in the standard form the FP64 passes of the
 * solve use: y_i = d_i x_i - sum_j w_ij x_j with d_i = sum_j w_ij computed
 * from w first. (The FP32 passes of an FP32-hierarchy solve use the
 * difference form sum_j w_ij (x_i - x_j) instead; both equal (L x)_i in
 * exact arithmetic.) */
int lg_laplacian_apply(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                       const double* x, double* y, void* stream);

/*
 * Low-degree elimination candidates (Section 3.4, Algorithm 2): is_f[i] = 1
 * iff deg(i) <= max_degree and hash(i) is the smallest hash among the candidates of i's closed neighbourhood.
 * hash(i) = SplitMix64 output number i for `seed`. *nf (host) receives |F|.
 */
int lg_elim_select(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t max_degree,
                   uint64_t seed, uint8_t* is_f, int64_t* nf, void* stream);

/*
 * Affinity strength of connection (Section 3.5): m test vectors drawn from
 * the SplitMix64 streams 1..m of (seed, level), smoothed by `sweeps` damped
 * Jacobi sweeps on L y = 0, then C_ij = (x_i . x_j)^2 / (|x_i|^2 |x_j|^2) and
 * S_ij = C_ij / max(max_s C_is, max_s C_sj). S[nnz] is on the graph's pattern.
 */
int lg_strength(int64_t n, const int64_t* rowptr, const int32_t* col, const double* w,
                uint64_t seed, int32_t level, int32_t m, int32_t sweeps, double omega, double* S,
                void* stream);

/*
 * Voting aggregation (Section 3.5, Algorithm 3) on strength values S[nnz]:
 * agg[n] receives the aggregate of each vertex, numbered from 0 in ascending order of the root
 * vertex; *nc (host) the number of aggregates; state[n] (LG_SEED /
 * LG_UNDECIDED / LG_DECIDED) and votes[n] the final status and vote counts
 * (state and votes may be NULL).
 */
int lg_aggregate(int64_t n, const int64_t* rowptr, const int32_t* col, const double* S,
                 int32_t iters, int32_t threshold, int32_t* agg, int64_t* nc, int8_t* state,
                 int32_t* votes, void* stream);

/*
 * lg_elim_select without allocation. Same inputs, outputs and results as
 * lg_elim_select (is_f bit for bit, *nf on the host), for callers that may
 * not allocate device memory during the call: code confined to a memory pool
 * that must not grow, host callbacks or threads of an embedding runtime that
 * forbid cudaMalloc, or loops that cannot afford an allocation's stall. It
 * calls no cudaMalloc / cudaFree and no allocating library routine; its
 * scratch (one 64-bit hash per vertex and a counter) lives in a fixed device
 * array of the library, sized for at most 1048576 vertices (8 MiB held on
 * every device that uses the library, until the process exits). Larger n
 * returns LG_ERR_INVALID with a message in lg_last_error_detail().
 *  - The call reads the count back and synchronises `stream` before it
 *    returns, so it cannot be captured into a CUDA graph.
 *  - The first call on a device looks up the array's device address on that
 *    device. `stream` must belong to the current device (a stream of another
 *    device returns LG_ERR_INVALID).
 *  - Every call shares the array: calls whose work overlaps on the GPU (two
 *    host threads, or two streams) race and give wrong results. Serialise
 *    them, e.g. on one stream.
 *  - The paper has no counterpart; this is an interface variant of
 *    lg_elim_select (Section 3.4).
 */
int lg_elim_select_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t max_degree,
                           uint64_t seed, uint8_t* is_f, int64_t* nf, void* stream);

/* ---- serving: continuous batching of solves over resident hierarchies ---- */
typedef struct {
  double hbm_budget_bytes;  /* admission budget for resident hierarchies + in-flight workspaces */
  int32_t slots;            /* concurrent solves on the device (one stream each), 1..64 */
  int32_t max_queue;        /* pending requests before lg_serve_submit returns LG_ERR_BUSY */
  int32_t precision;        /* V-cycle precision of served solves */
  int32_t policy;           /* which queued request leads the next group: LG_SERVE_ARRIVAL (default)
                               or LG_SERVE_LEAST_WORK (see lg_serve_submit) */
} lg_serve_options;

enum { LG_SERVE_ARRIVAL = 0, LG_SERVE_LEAST_WORK = 1 };

typedef struct {
  double p50_ms, p99_ms;    /* request latency, submit to completion */
  double mean_ms, max_ms;
  double solves_per_s;      /* completed right-hand sides per second since creation */
  double resident_bytes;    /* device bytes of registered hierarchies */
  int64_t completed, failed, pending, running;
  int64_t groups;           /* solves started: multi-column batches and packed launches */
  int64_t packed_groups;    /* of which packed launches of small graphs */
  int64_t workspaces_made;  /* solve workspaces created (the pool had none to reuse) */
  double workspace_ms;      /* host time spent creating them */
  double copy_ms;           /* host time in the groups' host<->device copies of B and X */
  double solve_ms;          /* host time in the groups' solves (multi-column and packed) */
} lg_serve_stats_t;

int lg_serve_options_default(lg_serve_options* o);
int lg_serve_create(const lg_serve_options* o, lg_server_t* out);

/* Make a hierarchy resident and servable. The server does not take ownership:
 * keep h alive until lg_serve_destroy. LG_ERR_NOMEM when the budget is full. */
int lg_serve_register(lg_server_t s, lg_handle h);

/*
 * Queue k right-hand sides (column-major n x k in HOST memory, B and X) for
 * hierarchy h. Returns at once with a ticket. B and X must stay valid until
 * lg_serve_poll reports done. Requests are admitted as slots and budget free
 * up. Policy LG_SERVE_ARRIVAL: in arrival order, except that a request that
 * fits may pass a head request that does not (at most 16 times per head
 * request). Policy LG_SERVE_LEAST_WORK: the admissible request with the least
 * work (k times the entries of all its hierarchy's operators) leads, but a
 * request passed over 16 times leads as soon as it is admissible (the oldest
 * first). A free slot takes the lead request together with the queued
 * requests on the same hierarchy and tolerance (up to 8 columns in all; a
 * wider request runs alone) and solves them as one multi-column batch; a
 * single-column request on a graph of at most
 * 16384 vertices (and 2^22 nonzeros, no K-cycle) instead joins the other such
 * queued requests (one per hierarchy, same tolerance) in one packed launch,
 * which uses the hierarchy's default workspace: do not call lg_solve on a
 * registered handle while the server runs. Each column is computed the same
 * way whatever it is grouped with, so a request's result is bitwise the same
 * alone and in any mix. Groups run concurrently on the slots' streams.
 */
int lg_serve_submit(lg_server_t s, lg_handle h, int32_t k, const double* B, double* X, double tol,
                    uint64_t* ticket);

/* Non-blocking: *done = 1 once the request finished; info (may be NULL) then
 * receives its result (status, iterations, worst column relres, latency in
 * solve_ms). A ticket can be polled done once; later polls return LG_ERR_INVALID. */
int lg_serve_poll(lg_server_t s, uint64_t ticket, int32_t* done, lg_info* info);

/* Device bytes the server reserves from its budget while a request of k
 * right-hand sides on h runs (its solve workspace, k rounded up to a power of
 * two, and staging). A request is admitted only when the registered
 * hierarchies plus the requests already running plus this figure fit the
 * budget. Finished requests leave their workspaces in a pool for reuse by
 * later requests on the same hierarchy; pooled workspaces count against the
 * budget and are released, least recently used first, when a new request
 * needs the room. */
int lg_serve_request_bytes(lg_handle h, int32_t k, double* bytes);

/* Latency and throughput statistics over completed requests. */
int lg_serve_stats(lg_server_t s, lg_serve_stats_t* st);

/* Start the statistics afresh (latencies, counts, phase times, the clock of
 * solves_per_s): successive measurements on one server. */
int lg_serve_reset_stats(lg_server_t s);
/* Switch the policy (LG_SERVE_ARRIVAL or LG_SERVE_LEAST_WORK) of a running
 * server; it applies from the next group a slot takes. Serving has no
 * counterpart in the paper. */
int lg_serve_set_policy(lg_server_t s, int32_t policy);

/* Wait for every queued request, then release the server's threads and streams. */
void lg_serve_destroy(lg_server_t s);

#ifdef __cplusplus
}
#endif
#endif
