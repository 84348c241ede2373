// Many independent small solves in one launch (Section 4's PCG with the
// V-cycle of Algorithm 1, or the K-cycle of Section 3.7).
//
// A graph of a few thousand vertices leaves the multi-kernel solve of
// lg_cycle.cu launch-bound: every level of every cycle costs several kernel
// launches of a few microseconds each, whatever the level's size. Here one
// thread block runs the whole solve of one graph: every row pass, vector
// update and dot product of the PCG and of the cycle is a loop over the
// block's threads, separated by block barriers, so a solve costs one block
// for its duration and no launch at all. The launch takes one block per graph
// (largest graphs first), so thousands of graphs share one launch and the
// hardware schedules blocks onto the 152 SMs as earlier ones finish.
//
// Each graph uses its own hierarchy and the vectors of its handle's default
// workspace. The arithmetic is that of lg_cycle.cu step for step (the
// post-smoothing pass over W = L P included, where the level has it); only the
// order of additions inside a row sum and a dot product differs (the group
// and block reductions here versus the grid-wide ones there), so a result
// agrees with lg_solve's to rounding and takes the same number of iterations
// but for a residual within rounding of the tolerance.
//
// Vectors written inside the launch are read back with plain loads after a
// block barrier (which makes one thread's global stores visible to the
// block); only the hierarchy's arrays, constant for the whole launch, go
// through the read-only path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "lg_hier.h"

namespace lg {

// Threads of the block that solves one graph. A solve is a chain of
// dependent passes, so a graph's time falls with the threads that share each
// pass; 512 threads at 64 registers (two blocks per SM) measured fastest
// against 256 and 1024.
constexpr int kMT = 512;

template <typename T>
struct MVecs {
  T *f, *x, *r, *a, *b, *kc1, *kv1, *kv2;  // a, b: the two Chebyshev direction buffers
};

// One CSR structure with its rows grouped by length (the plan's class
// lists): rows off[c] .. off[c+1] of `rows` have at most E 2^c entries
// (class 5: at most kChunk), rows off[kClasses] .. n are longer.
struct MRows {
  int64_t n = 0;
  const int64_t* ptr = nullptr;
  const int32_t* idx = nullptr;
  const int32_t* rows = nullptr;
  int64_t off[kClasses + 1] = {};
};

struct MLevel {
  int kind = 0;
  int64_t n = 0, nc = 0;
  MRows op, mem, pt, lp;  // lp: W = L P (lp.n = 0 when the level has none)
  const double *lp_w = nullptr, *lp_d = nullptr;
  const float* lp_w32 = nullptr;
  const double *w = nullptr, *d = nullptr, *dinv = nullptr;
  const float *w32 = nullptr, *dinv32 = nullptr;
  double wc = 0.0;  // every weight of the operator when w and w32 are null
  const int32_t *agg = nullptr, *cmap = nullptr, *cfine = nullptr;
  const double* pt_coef = nullptr;
  const float* pt_coef32 = nullptr;
  const double* pinv = nullptr;
  double inv_theta = 0.0, c1[8] = {0}, c2[8] = {0};
  MVecs<double> v64{};
  MVecs<float> v32{};
  double* ks = nullptr;  // K-cycle scalars of the level (kKScal)
};

struct MGraph {
  const MLevel* lv;
  int nlevels, first_agg, kcycle, deg, fp32, maxit, every;
  double tol;
  const int32_t* perm;  // level-0 vertex i is the caller's vertex perm[i]
  const double* b;      // caller's numbering
  double* out;          // caller's numbering, mean removed
  double *bm, *x, *r, *ro, *p, *q;
  double* res;          // iterations, status, relative residual
};

// Device views of a hierarchy's levels, built once per handle.
struct ManyDesc {
  DBuf<MLevel> levels;
};

// ---------------------------------------------------------------------------
// Block primitives.
// ---------------------------------------------------------------------------
struct MShared {
  double red[8 * (kMT / 32) + 8];
  int ph[kManyMaxLevels];  // cycle phase per level (see m_cycle)
};

// Sum of K values over the block, returned to every thread.
template <int K>
__device__ __forceinline__ void m_sum(double (&v)[K], MShared& sm) {
  block_sum<kMT, K>(v, sm.red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sm.red[8 * (kMT / 32) + k] = v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = sm.red[8 * (kMT / 32) + k];
  __syncthreads();
}

#define LG_BLOCK_LOOP(i, n) for (int64_t i = threadIdx.x; i < (n); i += kMT)

// Rows of class c, one aligned group of G lanes per row: s = the row's sum of
// term.acc over its entries, then epi(row, term.fin(row, rv, s)). A group
// takes two rows per step, their loads interleaved, so that each lane has
// two independent chains of gathers in flight.
template <typename A, int G, class Term, class Epi>
__device__ __forceinline__ void m_class(const MRows& R, int c, const Term& term, const Epi& epi) {
  const int64_t lo = R.off[c], cnt = R.off[c + 1] - lo;
  const int grp = threadIdx.x / G, gl = threadIdx.x & (G - 1);
  const unsigned mask = group_mask<G>();
  constexpr int kStep = kMT / G;
  for (int64_t base = 0; base < cnt; base += 2 * kStep) {
    const int64_t q0 = base + grp, q1 = q0 + kStep;
    A s0 = A(0), s1 = A(0), rv0 = A(0), rv1 = A(0);
    int64_t row0 = 0, row1 = 0, b0 = 0, e0 = 0, b1 = 0, e1 = 0;
    if (q0 < cnt) row0 = __ldg(&R.rows[lo + q0]);
    if (q1 < cnt) row1 = __ldg(&R.rows[lo + q1]);
    if (q0 < cnt) { b0 = __ldg(&R.ptr[row0]) + gl; e0 = __ldg(&R.ptr[row0 + 1]); rv0 = term.row(row0); }
    if (q1 < cnt) { b1 = __ldg(&R.ptr[row1]) + gl; e1 = __ldg(&R.ptr[row1 + 1]); rv1 = term.row(row1); }
    for (;;) {
      const bool v0 = b0 < e0, v1 = b1 < e1;
      if (!v0 && !v1) break;
      const int32_t j0 = v0 ? __ldg(&R.idx[b0]) : 0, j1 = v1 ? __ldg(&R.idx[b1]) : 0;
      if (v0) s0 = term.acc(s0, b0, j0, rv0);
      if (v1) s1 = term.acc(s1, b1, j1, rv1);
      b0 += G;
      b1 += G;
    }
    if constexpr (G > 1) {
      s0 = group_sum<G>(s0, mask);
      s1 = group_sum<G>(s1, mask);
    }
    if (gl == 0 && q0 < cnt) epi(row0, term.fin(row0, rv0, s0));
    if (gl == 0 && q1 < cnt) epi(row1, term.fin(row1, rv1, s1));
  }
}

// A row pass over every row of R, then a barrier. Rows longer than kChunk
// entries take the whole block each. Not inlined: a call per pass costs
// nothing next to the pass, and the kernel compiles in a fraction of the time.
template <typename A, class Term, class Epi>
__device__ __noinline__ void m_pass(const MRows& R, const Term& term, const Epi& epi, MShared& sm) {
  m_class<A, 1>(R, 0, term, epi);
  m_class<A, 2>(R, 1, term, epi);
  m_class<A, 4>(R, 2, term, epi);
  m_class<A, 8>(R, 3, term, epi);
  m_class<A, 16>(R, 4, term, epi);
  m_class<A, 32>(R, 5, term, epi);
  for (int64_t q = R.off[kClasses]; q < R.n; ++q) {
    const int64_t row = __ldg(&R.rows[q]);
    const A rv = term.row(row);
    A s = A(0);
    const int64_t e = __ldg(&R.ptr[row + 1]);
    for (int64_t k = __ldg(&R.ptr[row]) + threadIdx.x; k < e; k += kMT) s = term.acc(s, k, __ldg(&R.idx[k]), rv);
    double v[1] = {(double)s};
    m_sum<1>(v, sm);
    if (threadIdx.x == 0) epi(row, term.fin(row, rv, (A)v[0]));
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Row terms (the forms of lg_rows.cuh, with plain loads of the vector).
// ---------------------------------------------------------------------------
template <typename T>
struct MLap;

template <>
struct MLap<float> {  // difference form: sum_j w_ij (x_i - x_j); null w: every weight wc
  const float* w;
  const float* x;
  float wc;
  __device__ __forceinline__ float row(int64_t i) const { return x[i]; }
  __device__ __forceinline__ float acc(float s, int64_t k, int32_t j, float xi) const {
    return fmaf(w ? __ldg(&w[k]) : wc, xi - x[j], s);
  }
  __device__ __forceinline__ float fin(int64_t, float, float s) const { return s; }
};

template <>
struct MLap<double> {  // d_i x_i - sum_j w_ij x_j; null w: every weight wc
  const double* w;
  const double* x;
  const double* d;
  double wc;
  __device__ __forceinline__ double row(int64_t) const { return 0.0; }
  __device__ __forceinline__ double acc(double s, int64_t k, int32_t j, double) const {
    return fma(w ? __ldg(&w[k]) : wc, x[j], s);
  }
  __device__ __forceinline__ double fin(int64_t i, double, double s) const { return fma(__ldg(&d[i]), x[i], -s); }
};

template <typename T>
__device__ __forceinline__ MLap<T> m_lap(const MLevel& L, const T* x);
template <>
__device__ __forceinline__ MLap<float> m_lap<float>(const MLevel& L, const float* x) {
  return MLap<float>{L.w32, x, (float)L.wc};
}
template <>
__device__ __forceinline__ MLap<double> m_lap<double>(const MLevel& L, const double* x) {
  return MLap<double>{L.w, x, L.d, L.wc};
}

// (L P x_c)_i over W = L P off the own aggregate (the forms of LpTerm).
template <typename T>
struct MLpT;

template <>
struct MLpT<float> {
  const float* w;
  const float* xc;
  const int32_t* agg;
  __device__ __forceinline__ float row(int64_t i) const { return xc[__ldg(&agg[i])]; }
  __device__ __forceinline__ float acc(float s, int64_t k, int32_t a, float xa) const {
    return fmaf(__ldg(&w[k]), xa - xc[a], s);
  }
  __device__ __forceinline__ float fin(int64_t, float, float s) const { return s; }
};

template <>
struct MLpT<double> {
  const double* w;
  const double* xc;
  const int32_t* agg;
  const double* d;
  __device__ __forceinline__ double row(int64_t) const { return 0.0; }
  __device__ __forceinline__ double acc(double s, int64_t k, int32_t a, double) const {
    return fma(__ldg(&w[k]), xc[a], s);
  }
  __device__ __forceinline__ double fin(int64_t i, double, double s) const {
    return fma(__ldg(&d[i]), xc[__ldg(&agg[i])], -s);
  }
};

template <typename T>
__device__ __forceinline__ MLpT<T> m_lpt(const MLevel& L, const T* xc);
template <>
__device__ __forceinline__ MLpT<float> m_lpt<float>(const MLevel& L, const float* xc) {
  return MLpT<float>{L.lp_w32, xc, L.agg};
}
template <>
__device__ __forceinline__ MLpT<double> m_lpt<double>(const MLevel& L, const double* xc) {
  return MLpT<double>{L.lp_w, xc, L.agg, L.lp_d};
}

template <typename T>
struct MGather {  // sum_k v[idx_k]
  const T* v;
  __device__ __forceinline__ T row(int64_t) const { return T(0); }
  __device__ __forceinline__ T acc(T s, int64_t, int32_t j, T) const { return s + v[j]; }
  __device__ __forceinline__ T fin(int64_t, T, T s) const { return s; }
};

template <typename T>
struct MWGather {  // sum_k c_k v[idx_k]
  const T* c;
  const T* v;
  __device__ __forceinline__ T row(int64_t) const { return T(0); }
  __device__ __forceinline__ T acc(T s, int64_t k, int32_t j, T) const { return fma(__ldg(&c[k]), v[j], s); }
  __device__ __forceinline__ T fin(int64_t, T, T s) const { return s; }
};

template <typename T> __device__ __forceinline__ const MVecs<T>& m_vecs(const MLevel& L);
template <> __device__ __forceinline__ const MVecs<double>& m_vecs<double>(const MLevel& L) { return L.v64; }
template <> __device__ __forceinline__ const MVecs<float>& m_vecs<float>(const MLevel& L) { return L.v32; }
template <typename T> __device__ __forceinline__ const T* m_dinv(const MLevel& L);
template <> __device__ __forceinline__ const double* m_dinv<double>(const MLevel& L) { return L.dinv; }
template <> __device__ __forceinline__ const float* m_dinv<float>(const MLevel& L) { return L.dinv32; }
template <typename T> __device__ __forceinline__ const T* m_wop(const MLevel& L);
template <> __device__ __forceinline__ const double* m_wop<double>(const MLevel& L) { return L.w; }
template <> __device__ __forceinline__ const float* m_wop<float>(const MLevel& L) { return L.w32; }
template <typename T> __device__ __forceinline__ const T* m_ptc(const MLevel& L);
template <> __device__ __forceinline__ const double* m_ptc<double>(const MLevel& L) { return L.pt_coef; }
template <> __device__ __forceinline__ const float* m_ptc<float>(const MLevel& L) { return L.pt_coef32; }

// ---------------------------------------------------------------------------
// Cycle steps of one level (the kernels of lg_cycle.cu as block loops).
// ---------------------------------------------------------------------------

// One Chebyshev step on D^-1 L (Section 3.6) over gathered g = d_{s-1}:
// r_s = rin - L g, d_s = c1 g + c2 D^-1 r_s (when gn), x = [x +] g [+ d_s]
// (when upd: mode 1 sets, mode 2 adds).
template <typename T>
__device__ __noinline__ void m_cheb(const MLevel& L, const T* g, const T* rin, T* rout, T* gn, T* x, int upd,
                                    int mode, int add_d, T c1, T c2, MShared& sm) {
  const T* dinv = m_dinv<T>(L);
  m_pass<T>(L.op, m_lap<T>(L, g), [=](int64_t i, T s) {
    const T r = rin[i] - s;
    rout[i] = r;
    T d = T(0);
    if (gn) {
      d = c1 * g[i] + c2 * __ldg(&dinv[i]) * r;
      gn[i] = d;
    }
    if (upd) x[i] = (mode == 2 ? x[i] : T(0)) + g[i] + (add_d ? d : T(0));
  }, sm);
}

// The next level's first Chebyshev direction target, when that level smooths.
template <typename T>
__device__ __forceinline__ void m_next_dir(const MGraph& G, int l, T** d0, const T** dinv, T* it) {
  const MLevel& N = G.lv[l + 1];
  if (N.kind == LG_LEVEL_AGG) {
    *d0 = m_vecs<T>(N).a;
    *dinv = m_dinv<T>(N);
    *it = (T)N.inv_theta;
  } else {
    *d0 = nullptr;
    *dinv = nullptr;
    *it = T(0);
  }
}

// Elimination restriction (P^T f)_c = f_c + sum_f (w_fc / d_f) f_f, and the
// next level's d_0 when it smooths.
template <typename T>
__device__ __noinline__ void m_restrict_elim(const MLevel& L, const T* f, T* fc, T* d0n, const T* dinvn, T itn,
                                             MShared& sm) {
  const int32_t* cfine = L.cfine;
  m_pass<T>(L.pt, MWGather<T>{m_ptc<T>(L), f}, [=](int64_t c, T s) {
    const T v = f[__ldg(&cfine[c])] + s;
    fc[c] = v;
    if (d0n) d0n[c] = v * __ldg(&dinvn[c]) * itn;
  }, sm);
}

// Aggregation restriction r_c = R r, and the next level's d_0 when it smooths.
template <typename T>
__device__ __noinline__ void m_restrict_agg(const MLevel& L, const T* r, T* fc, T* d0n, const T* dinvn, T itn,
                                            MShared& sm) {
  m_pass<T>(L.mem, MGather<T>{r}, [=](int64_t I, T s) {
    fc[I] = s;
    if (d0n) d0n[I] = s * __ldg(&dinvn[I]) * itn;
  }, sm);
}

// Going down through level l: pre-smoothing and restriction (aggregation
// level), restriction (elimination level). Leaves the coarse input in l+1.
template <typename T>
__device__ void m_down(const MGraph& G, int l, MShared& sm) {
  const MLevel& L = G.lv[l];
  const MVecs<T>& V = m_vecs<T>(L);
  const MVecs<T>& C = m_vecs<T>(G.lv[l + 1]);
  T* d0n;
  const T* dinvn;
  T itn;
  m_next_dir<T>(G, l, &d0n, &dinvn, &itn);
  if (L.kind == LG_LEVEL_ELIM) {
    m_restrict_elim<T>(L, V.f, C.f, d0n, dinvn, itn, sm);
    return;
  }
  const int deg = G.deg;
  T* g = V.a;
  T* gn = V.b;
  const T* rin = V.f;
  for (int st = 1; st < deg; ++st) {  // pre-smoothing from x = 0
    m_cheb<T>(L, g, rin, V.r, gn, V.x, 1, st == 1 ? 1 : 2, st == deg - 1, (T)L.c1[st], (T)L.c2[st], sm);
    rin = V.r;
    T* t = g;
    g = gn;
    gn = t;
  }
  // residual of the pre-smoothed x (for degree 1 also x = d_0)
  m_cheb<T>(L, g, rin, V.r, nullptr, V.x, deg == 1, 1, 0, T(0), T(0), sm);
  m_restrict_agg<T>(L, V.r, C.f, d0n, dinvn, itn, sm);
}

// Start of post-smoothing over W (see EpiPost in lg_cycle.cu): x += P x_c,
// r_0 = r_pre - (L P x_c), d_0 = D^-1 r_0 / theta, in one pass.
template <typename T>
__device__ __noinline__ void m_post_w(const MLevel& L, T* x, T* r, T* d0, const T* xc, MShared& sm) {
  const T* dinv = m_dinv<T>(L);
  const int32_t* agg = L.agg;
  const T it = (T)L.inv_theta;
  m_pass<T>(L.lp, m_lpt<T>(L, xc), [=](int64_t i, T s) {
    const T r0 = r[i] - s;
    r[i] = r0;
    d0[i] = it * __ldg(&dinv[i]) * r0;
    x[i] = x[i] + xc[__ldg(&agg[i])];
  }, sm);
}

// Coming back up through level l: prolongation and post-smoothing.
template <typename T>
__device__ void m_up(const MGraph& G, int l, MShared& sm) {
  const MLevel& L = G.lv[l];
  const MVecs<T>& V = m_vecs<T>(L);
  const T* xc = m_vecs<T>(G.lv[l + 1]).x;
  if (L.kind == LG_LEVEL_ELIM) {
    // kept vertices take their coarse value; eliminated f: (f_f + sum_c w_fc x_c) / d_f
    const T* w = m_wop<T>(L);
    const T* dinv = m_dinv<T>(L);
    LG_BLOCK_LOOP(i, L.n) {
      const int32_t c = __ldg(&L.cmap[i]);
      T v;
      if (c >= 0) {
        v = xc[c];
      } else {
        T s = V.f[i];
        const int64_t e = __ldg(&L.op.ptr[i + 1]);
        for (int64_t k = __ldg(&L.op.ptr[i]); k < e; ++k)
          s += (w ? __ldg(&w[k]) : (T)L.wc) * xc[__ldg(&L.cmap[__ldg(&L.op.idx[k])])];
        v = s * __ldg(&dinv[i]);
      }
      V.x[i] = v;
    }
    __syncthreads();
    return;
  }
  const int deg = G.deg;
  if (L.lp.n > 0) {  // x += P x_c, r_0 = r_pre - L P x_c, d_0 over W
    m_post_w<T>(L, V.x, V.r, V.a, xc, sm);
  } else {
    LG_BLOCK_LOOP(i, L.n) V.x[i] += xc[__ldg(&L.agg[i])];  // x += P x_c
    __syncthreads();
    // r_0 = f - L x, d_0 = D^-1 r_0 / theta
    m_cheb<T>(L, V.x, V.f, V.r, V.a, nullptr, 0, 0, 0, T(0), (T)L.inv_theta, sm);
  }
  T* g = V.a;
  T* gn = V.b;
  for (int st = 1; st < deg; ++st) {
    m_cheb<T>(L, g, V.r, V.r, gn, V.x, 1, 2, st == deg - 1, (T)L.c1[st], (T)L.c2[st], sm);
    T* t = g;
    g = gn;
    gn = t;
  }
  if (deg == 1) {
    LG_BLOCK_LOOP(i, L.n) V.x[i] += V.a[i];
    __syncthreads();
  }
}

// Coarsest level: x = L_c^+ f with the FP64 pseudo-inverse, a warp per row.
template <typename T>
__device__ void m_coarse(const MLevel& L) {
  const MVecs<T>& V = m_vecs<T>(L);
  const int lane = threadIdx.x & 31;
  const int64_t n = L.n;
  for (int64_t i = threadIdx.x >> 5; i < n; i += kMT / 32) {
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s += __ldg(&L.pinv[i * n + j]) * (double)V.f[j];
    s = group_sum<32>(s, 0xffffffffu);
    if (lane == 0) V.x[i] = (T)s;
  }
  __syncthreads();
}

// v = L x (the K-cycle's products, and q = L p of the PCG).
template <typename T>
__device__ __noinline__ void m_apply(const MLevel& L, const T* x, T* v, MShared& sm) {
  m_pass<T>(L.op, m_lap<T>(L, x), [=](int64_t i, T s) { v[i] = s; }, sm);
}

// K-cycle, after the first body: c1 = x, v1 = L c1, t1 = c1.f / c1.v1,
// r1 = f - t1 v1 in place of f, and its direction d_0 = D^-1 r1 / theta.
template <typename T>
__device__ void m_kfirst(const MLevel& L, MShared& sm) {
  const MVecs<T>& V = m_vecs<T>(L);
  m_apply<T>(L, V.x, V.kv1, sm);
  double acc[2] = {0.0, 0.0};
  LG_BLOCK_LOOP(i, L.n) {
    const T xi = V.x[i];
    V.kc1[i] = xi;
    acc[0] += (double)xi * (double)V.kv1[i];
    acc[1] += (double)xi * (double)V.f[i];
  }
  m_sum<2>(acc, sm);
  const bool ok = acc[0] > 0.0 && isfinite(acc[0]);
  const double t1 = ok ? acc[1] / acc[0] : 0.0;
  if (threadIdx.x == 0) {
    L.ks[kRho1] = acc[0];
    L.ks[kOk1] = ok ? 1.0 : 0.0;
    L.ks[kT1] = t1;
  }
  const T tt = (T)t1, it = (T)L.inv_theta;
  const T* dinv = m_dinv<T>(L);
  LG_BLOCK_LOOP(i, L.n) {
    const T r = V.f[i] - tt * V.kv1[i];
    V.f[i] = r;
    V.a[i] = r * __ldg(&dinv[i]) * it;
  }
  __syncthreads();
}

// K-cycle, after the second body: x = u1 c1 + u2 c2 with c2 = x (see k_ksecond).
template <typename T>
__device__ void m_ksecond(const MLevel& L, MShared& sm) {
  const MVecs<T>& V = m_vecs<T>(L);
  m_apply<T>(L, V.x, V.kv2, sm);
  double acc[3] = {0.0, 0.0, 0.0};
  LG_BLOCK_LOOP(i, L.n) {
    const double xi = (double)V.x[i];
    acc[0] += xi * (double)V.kv1[i];
    acc[1] += xi * (double)V.kv2[i];
    acc[2] += xi * (double)V.f[i];
  }
  m_sum<3>(acc, sm);
  double u1 = 1.0, u2 = 0.0;
  if (L.ks[kOk1] != 0.0) {
    const double rho1 = L.ks[kRho1], t1 = L.ks[kT1], g = acc[0], a2 = acc[2];
    const double rho2 = acc[1] - g * g / rho1;
    if (rho2 > 0.0 && isfinite(rho2)) {
      u1 = t1 - g * a2 / (rho1 * rho2);
      u2 = a2 / rho2;
    } else {
      u1 = t1;
    }
  }
  LG_BLOCK_LOOP(i, L.n) V.x[i] = (T)(u1 * (double)V.kc1[i] + u2 * (double)V.x[i]);
  __syncthreads();
}

// The cycle from level 0 (input in level 0's f, and its d_0 when level 0
// smooths; result in level 0's x), as a loop over levels with a phase per
// level instead of recursion: phase 0 enters the level (going down), phase 1
// returns to it from the coarser level after the first (or only) coarse
// visit, phase 2 after a K-cycle level's second.
template <typename T>
__device__ void m_cycle(const MGraph& G, MShared& sm) {
  int l = 0;
  if (threadIdx.x == 0) sm.ph[0] = 0;
  __syncthreads();
  while (l >= 0) {
    const MLevel& L = G.lv[l];
    if (L.kind == LG_LEVEL_COARSEST) {
      m_coarse<T>(L);
      --l;
      continue;
    }
    const bool K = G.kcycle && L.kind == LG_LEVEL_AGG && l != G.first_agg;
    const int ph = sm.ph[l];
    __syncthreads();  // every thread has read the phase before it changes
    if (ph == 0) {
      m_down<T>(G, l, sm);
    } else {
      m_up<T>(G, l, sm);
      if (ph == 1 && K) {
        m_kfirst<T>(L, sm);
        m_down<T>(G, l, sm);
      } else {
        if (K) m_ksecond<T>(L, sm);
        --l;
        continue;
      }
    }
    if (threadIdx.x == 0) {
      sm.ph[l] = ph + 1;
      sm.ph[l + 1] = 0;
    }
    __syncthreads();
    ++l;
  }
}

// r = b_m - L x and ||r||^2.
__device__ __noinline__ double m_true_res(const MLevel& L0, const double* bm, const double* x, double* r,
                                          MShared& sm) {
  m_pass<double>(L0.op, MLap<double>{L0.w, x, L0.d, L0.wc}, [=](int64_t i, double s) { r[i] = bm[i] - s; }, sm);
  double acc[1] = {0.0};
  LG_BLOCK_LOOP(i, L0.n) acc[0] += r[i] * r[i];
  m_sum<1>(acc, sm);
  return acc[0];
}

// The PCG of one graph (FP64, Polak-Ribiere beta, true residual every
// `every` iterations and to confirm convergence), as pcg_solve runs it.
template <typename T>
__device__ void m_pcg(const MGraph& G, MShared& sm) {
  const MLevel& L0 = G.lv[0];
  const int64_t n = L0.n;
  double acc[1] = {0.0};
  LG_BLOCK_LOOP(i, n) acc[0] += G.b[i];
  m_sum<1>(acc, sm);
  const double mean = acc[0] / (double)n;
  acc[0] = 0.0;
  LG_BLOCK_LOOP(i, n) {
    const double v = G.b[__ldg(&G.perm[i])] - mean;
    G.bm[i] = v;
    G.r[i] = v;
    G.x[i] = 0.0;
    G.p[i] = 0.0;
    acc[0] += v * v;
  }
  m_sum<1>(acc, sm);
  const double bb = acc[0], tol2bb = G.tol * G.tol * bb;
  double rr = bb, rz = 0.0;
  int it = 0, done = 0, brk = 0;
  const MVecs<T>& V0 = m_vecs<T>(L0);
  const T* dinv0 = m_dinv<T>(L0);
  const bool smooth0 = L0.kind == LG_LEVEL_AGG;
  const T it0 = (T)L0.inv_theta;
  if (bb > 0.0) {
    while (it < G.maxit) {
      // z = M r
      LG_BLOCK_LOOP(i, n) {
        const T v = (T)G.r[i];
        V0.f[i] = v;
        if (smooth0) V0.a[i] = v * __ldg(&dinv0[i]) * it0;
      }
      __syncthreads();
      m_cycle<T>(G, sm);
      // sums over z (mean not removed), beta, r^T z
      const int first = it == 0;
      double zs[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      LG_BLOCK_LOOP(i, n) {
        const double zi = (double)V0.x[i], ri = G.r[i], roi = first ? 0.0 : G.ro[i];
        zs[0] += zi;
        zs[1] += zi * ri;
        zs[2] += zi * roi;
        zs[3] += ri;
        zs[4] += roi;
      }
      m_sum<5>(zs, sm);
      const double m = zs[0] / (double)n;
      const double zr = zs[1] - m * zs[3], zro = zs[2] - m * zs[4];
      const double beta = first ? 0.0 : (zr - zro) / rz;
      if (!(zr > 0.0) || !isfinite(zr)) brk = 1;
      rz = zr;
      LG_BLOCK_LOOP(i, n) G.p[i] = ((double)V0.x[i] - m) + beta * G.p[i];
      __syncthreads();
      // q = L p, alpha
      m_apply<double>(L0, G.p, G.q, sm);
      acc[0] = 0.0;
      LG_BLOCK_LOOP(i, n) acc[0] += G.p[i] * G.q[i];
      m_sum<1>(acc, sm);
      const double pq = acc[0];
      double alpha = 0.0;
      if (!(pq > 0.0) || !isfinite(pq) || brk) brk = 1;
      else alpha = rz / pq;
      // x, r
      acc[0] = 0.0;
      LG_BLOCK_LOOP(i, n) {
        const double ri = G.r[i];
        G.ro[i] = ri;
        G.x[i] += alpha * G.p[i];
        const double rn = ri - alpha * G.q[i];
        G.r[i] = rn;
        acc[0] += rn * rn;
      }
      m_sum<1>(acc, sm);
      rr = acc[0];
      ++it;
      if (it % G.every == 0 || rr <= tol2bb) {
        rr = m_true_res(L0, G.bm, G.x, G.r, sm);
        if (rr <= tol2bb) done = 1;
      }
      if (done || brk) break;
    }
  }
  int status = LG_OK;
  double rel = 0.0;
  if (bb > 0.0) {
    status = done ? LG_OK : brk ? LG_ERR_BREAKDOWN : LG_ERR_NOT_CONVERGED;
    if (status != LG_OK) rr = m_true_res(L0, G.bm, G.x, G.r, sm);
    rel = sqrt(rr / bb);
  }
  // x with its mean removed, in the caller's numbering
  acc[0] = 0.0;
  LG_BLOCK_LOOP(i, n) acc[0] += G.x[i];
  m_sum<1>(acc, sm);
  const double mx = acc[0] / (double)n;
  LG_BLOCK_LOOP(i, n) G.out[__ldg(&G.perm[i])] = G.x[i] - mx;
  if (threadIdx.x == 0) {
    G.res[0] = (double)it;
    G.res[1] = (double)status;
    G.res[2] = rel;
  }
}

__global__ void __launch_bounds__(kMT, 2) k_solve_many(const MGraph* __restrict__ graphs) {
  __shared__ MShared sm;
  const MGraph G = graphs[blockIdx.x];
  if (G.fp32) m_pcg<float>(G, sm);
  else m_pcg<double>(G, sm);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static MRows rows_of(int64_t n, const int64_t* ptr, const int32_t* idx, const RowPlan& p) {
  MRows r;
  r.n = n;
  r.ptr = ptr;
  r.idx = idx;
  r.rows = p.rows_by_class;
  for (int c = 0; c <= kClasses; ++c) r.off[c] = p.cls_off[c];
  return r;
}

// On the handle's own stream: the views live (and are freed) with the handle.
static const MLevel* many_levels(Hier& h) {
  if (h.many) return static_cast<ManyDesc*>(h.many.get())->levels.get();
  cudaStream_t s = h.stream;
  const size_t nl = h.levels.size();
  std::vector<MLevel> hv(nl);
  Workspace& ws = *h.ws;
  for (size_t l = 0; l < nl; ++l) {
    const Level& L = *h.levels[l];
    MLevel& m = hv[l];
    m.kind = L.kind;
    m.n = L.n;
    m.nc = L.nc;
    m.op = rows_of(L.n, L.rowptr.get(), L.col.get(), L.plan.plan);
    m.w = L.w.get();
    m.d = L.d.get();
    m.dinv = L.dinv.get();
    m.w32 = L.w32.get();
    m.dinv32 = L.dinv32.get();
    m.wc = L.wconst_on ? L.wconst : 0.0;
    if (L.kind == LG_LEVEL_AGG) {
      m.mem = rows_of(L.nc, L.mem_ptr.get(), L.mem.get(), L.mem_plan.plan);
      m.agg = L.agg.get();
      if (L.lp_nnz > 0) {
        m.lp = rows_of(L.n, L.lp_ptr.get(), L.lp_col.get(), L.lp_plan.plan);
        m.lp_w = L.lp_w.get();
        m.lp_d = L.lp_d.get();
        m.lp_w32 = L.lp_w32.get();
      }
      const Cheb& c = h.cheb[l];
      m.inv_theta = c.inv_theta;
      for (int q = 0; q < 8; ++q) {
        m.c1[q] = c.c1[q];
        m.c2[q] = c.c2[q];
      }
    }
    if (L.kind == LG_LEVEL_ELIM) {
      m.pt = rows_of(L.nc, L.pt_ptr.get(), L.pt_f.get(), L.pt_plan.plan);
      m.cmap = L.cmap.get();
      m.cfine = L.cfine.get();
      m.pt_coef = L.pt_coef.get();
      m.pt_coef32 = L.pt_coef32.get();
    }
    if (L.kind == LG_LEVEL_COARSEST) m.pinv = L.pinv.get();
    const LevelVecs<double>& a = ws.v64[l];
    const LevelVecs<float>& b = ws.v32[l];
    m.v64 = MVecs<double>{a.f.get(), a.x.get(), a.r.get(), a.dA.get(), a.dB.get(),
                          a.kc1.get(), a.kv1.get(), a.kv2.get()};
    m.v32 = MVecs<float>{b.f.get(), b.x.get(), b.r.get(), b.dA.get(), b.dB.get(),
                         b.kc1.get(), b.kv1.get(), b.kv2.get()};
    m.ks = ws.kscal.get() + (size_t)kKScal * l;
  }
  auto d = std::make_shared<ManyDesc>();
  d->levels.alloc(nl, s, &h.bytes);
  LG_CUDA(cudaMemcpyAsync(d->levels.get(), hv.data(), sizeof(MLevel) * nl, cudaMemcpyHostToDevice, s));
  LG_CUDA(cudaStreamSynchronize(s));  // hv goes out of scope
  h.many = d;
  return d->levels.get();
}

// Pinned host staging of a call (descriptors, results and the host-memory
// vectors), so that a call makes one copy each way however many graphs it
// holds. Grown on demand and kept until the process exits (freeing pinned
// memory from a static destructor could run after the CUDA runtime has shut
// down); calls take it one at a time.
struct PinnedStage {
  std::mutex m;
  unsigned char* p = nullptr;
  size_t cap = 0;
};
static PinnedStage g_pin;

void prepare_many(Hier& h) {
  std::lock_guard<std::mutex> lock(g_pin.m);  // solve_many builds the views under the same lock
  many_levels(h);
}

int solve_many(int count, Hier* const* hs, const double* const* b, double* const* x, const bool* b_dev,
               const bool* x_dev, double tol, lg_info* infos, int precision) {
  cudaStream_t s = hs[0]->stream;
  // every event of the call is destroyed on every exit, error paths included
  struct Events {
    std::vector<cudaEvent_t> v;
    cudaEvent_t make(unsigned flags) {
      cudaEvent_t e = nullptr;
      LG_CUDA(cudaEventCreateWithFlags(&e, flags));
      v.push_back(e);
      return e;
    }
    ~Events() {
      for (auto e : v) cudaEventDestroy(e);
    }
  } events;
  // run after whatever the other handles' streams hold
  for (int g = 1; g < count; ++g) {
    if (hs[g]->stream == s) continue;
    cudaEvent_t e = events.make(cudaEventDisableTiming);
    LG_CUDA(cudaEventRecord(e, hs[g]->stream));
    LG_CUDA(cudaStreamWaitEvent(s, e, 0));
  }
  // staging layout: count descriptors, 3 results per graph, then one
  // stretch of n doubles per graph with a host b or x (the kernel reads b
  // there at the start and writes x there at the end)
  std::vector<int64_t> off(count, -1);
  size_t nvec = 0;
  for (int g = 0; g < count; ++g) {
    if (b_dev[g] && x_dev[g]) continue;
    off[g] = (int64_t)nvec;
    nvec += (size_t)hs[g]->levels[0]->n;
  }
  const size_t desc_bytes = sizeof(MGraph) * count, res_bytes = sizeof(double) * 3 * count;
  const size_t total = desc_bytes + res_bytes + sizeof(double) * nvec;
  std::lock_guard<std::mutex> lock(g_pin.m);
  // on every exit, error paths included, the copies that read or write the
  // pinned buffer finish before the next call may take it
  struct SyncOnExit {
    cudaStream_t s;
    ~SyncOnExit() {
      if (cudaStreamSynchronize(s) != cudaSuccess) cudaGetLastError();
    }
  } sync_on_exit{s};
  if (g_pin.cap < total) {
    if (g_pin.p) cudaFreeHost(g_pin.p);  // every earlier call has finished with it
    g_pin.p = nullptr;
    g_pin.cap = 0;
    LG_CUDA(cudaMallocHost(&g_pin.p, total + total / 4));
    g_pin.cap = total + total / 4;
  }
  DBuf<unsigned char> dst(total, s);
  MGraph* hg = reinterpret_cast<MGraph*>(g_pin.p);
  double* hres = reinterpret_cast<double*>(g_pin.p + desc_bytes);
  double* hvec = reinterpret_cast<double*>(g_pin.p + desc_bytes + res_bytes);
  double* dres = reinterpret_cast<double*>(dst.get() + desc_bytes);
  double* dvec = reinterpret_cast<double*>(dst.get() + desc_bytes + res_bytes);
  // largest graphs first, so that the launch does not end on a long tail
  std::vector<int> order(count);
  for (int g = 0; g < count; ++g) order[g] = g;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int c) { return hs[a]->nnz0 > hs[c]->nnz0; });
  for (int q = 0; q < count; ++q) {
    const int g = order[q];
    Hier& h = *hs[g];
    Workspace& ws = *h.ws;
    const int64_t n = h.levels[0]->n;
    MGraph G;
    G.lv = many_levels(h);
    G.nlevels = (int)h.levels.size();
    G.first_agg = h.first_agg;
    G.kcycle = h.opts.kcycle;
    G.deg = h.opts.cheb_degree;
    G.fp32 = (precision < 0 ? h.opts.precision : precision) == LG_FP32_HIER;
    G.maxit = h.opts.max_iter;
    G.every = h.opts.residual_replace > 0 ? h.opts.residual_replace : 1 << 30;
    G.tol = tol;
    G.perm = h.perm.get();
    if (b_dev[g]) {
      G.b = b[g];
    } else {
      std::memcpy(hvec + off[g], b[g], sizeof(double) * n);
      G.b = dvec + off[g];
    }
    G.out = x_dev[g] ? x[g] : dvec + off[g];
    G.bm = ws.bm.get();
    G.x = ws.x.get();
    G.r = ws.r.get();
    G.ro = ws.ro.get();
    G.p = ws.p.get();
    G.q = ws.q.get();
    G.res = dres + (size_t)3 * g;
    hg[q] = G;
  }
  LG_CUDA(cudaMemcpyAsync(dst.get(), g_pin.p, total, cudaMemcpyHostToDevice, s));
  cudaEvent_t e0 = events.make(cudaEventDefault), e1 = events.make(cudaEventDefault);
  LG_CUDA(cudaEventRecord(e0, s));
  k_solve_many<<<count, kMT, 0, s>>>(reinterpret_cast<const MGraph*>(dst.get()));
  LG_LAUNCH_CHECK();
  LG_CUDA(cudaEventRecord(e1, s));
  LG_CUDA(cudaMemcpyAsync(hres, dres, total - desc_bytes, cudaMemcpyDeviceToHost, s));
  LG_CUDA(cudaStreamSynchronize(s));
  for (int g = 0; g < count; ++g)
    if (!x_dev[g]) std::memcpy(x[g], hvec + off[g], sizeof(double) * hs[g]->levels[0]->n);
  float ms = 0.f;
  LG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  int first_bad = LG_OK;
  for (int g = 0; g < count; ++g) {
    const Hier& h = *hs[g];
    const int it = (int)hres[3 * g], st = (int)hres[3 * g + 1];
    if (st != LG_OK && first_bad == LG_OK) first_bad = st;
    if (!infos) continue;
    lg_info& inf = infos[g];
    inf = lg_info{};
    inf.status = st;
    inf.iterations = it;
    inf.relres = hres[3 * g + 2];
    inf.solve_ms = ms;
    inf.work_units = it * iteration_work(h);
    inf.levels = (int)h.levels.size();
    inf.setup_ms = h.setup_ms;
    inf.nnz = h.nnz0;
    double oc = 0.0;
    for (auto& L : h.levels) oc += (double)(L->nnz + L->n);
    inf.op_complexity = oc / (double)h.nnz0;
  }
  return first_bad;
}

}  // namespace lg
