// kf_problems.cuh -- the three scans of arXiv 2511.10363 written as policies
// for the generic scan kernels, in SCAN ORDER: position p = 0, 1, ... is the
// order in which the scan accumulates.  combine(x, y) receives x earlier in
// scan order; apply(c, e) extends a carry by the next element in scan order.
//
//   FilterFwd : Alg. pkf   -- forward scan of a_1..a_T under Lemma 1,
//               carry (b, C), extraction xbar_{k|k} = b_k^+, P_{k|k} = C_k^+,
//               plus the innovation log-likelihood.
//   TfRev     : Alg. ptf   -- reversed scan of (a_2, ..., a_T, e) under
//               Lemma 1, carry (eta, J), extraction eta_{k|k+1:T}, J_{k|k+1:T},
//               fused with the two-filter merge.
//   RtsRev    : Alg. prts  -- reversed scan of (E, g, L) under Lemma 2,
//               carry (g, L), extraction xbar_{k|T} = g_k^+, P_{k|T} = L_k^+.
//
// Sequences: a call scans one sequence or a concatenation of independent
// sequences ("segments").  No segment flags are needed: the operator resets
// by itself at a boundary.  A forward prefix that reaches a segment's a_1
// has A = 0 there, so its (b, C) no longer depends on anything before; a
// reversed RTS suffix that reaches a segment's last element has E = 0; and
// the two-filter scan ends each segment with e = (0, 0, 0, 0, 0), the
// terminal element printed in Alg. ptf, whose (eta, J) = (0, 0) cuts the
// (eta, J) half off from everything after it.
#pragma once

#include <type_traits>

#include "kf_math.cuh"

namespace kfs {

// Where the model constants of a position come from.
template <int N, typename R>
struct OneSeq {
    static constexpr bool ONE = true;
    FiltParams<N, R> prm;
    int64_t T;
};

template <int N, typename R>
struct ManySeq {
    static constexpr bool ONE = false;
    const FiltParams<N, R> *prm;   // [nmodels]
    const int *model_of;           // [nseg] model of each sequence
    const int64_t *offsets;        // [nseg + 1], offsets[0] = 0, non-decreasing
    int nseg;
    int64_t total;
};

// Tracks the segment of the current position while a thread walks
// consecutive positions.
struct SegCursor {
    int s;
    int64_t b, e;   // [b, e) global index range of segment s
};

template <int N, typename R>
KF_D const FiltParams<N, R> &seg_params(const OneSeq<N, R> &q, const SegCursor &) { return q.prm; }
template <int N, typename R>
KF_D const FiltParams<N, R> &seg_params(const ManySeq<N, R> &q, const SegCursor &c) { return q.prm[__ldg(q.model_of + c.s)]; }

template <int N, typename R>
KF_HD int64_t seq_total(const OneSeq<N, R> &q) { return q.T; }
template <int N, typename R>
KF_HD int64_t seq_total(const ManySeq<N, R> &q) { return q.total; }

template <int N, typename R>
KF_D SegCursor seg_find(const OneSeq<N, R> &q, int64_t) { return SegCursor{0, 0, q.T}; }
template <int N, typename R>
KF_D SegCursor seg_find(const ManySeq<N, R> &q, int64_t g) {
    int lo = 0, hi = q.nseg - 1;   // last segment with offsets[s] <= g
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(q.offsets + mid) <= g) lo = mid; else hi = mid - 1;
    }
    return SegCursor{lo, __ldg(q.offsets + lo), __ldg(q.offsets + lo + 1)};
}

template <int N, typename R>
KF_D void seg_move(const OneSeq<N, R> &, SegCursor &, int64_t) {}
template <int N, typename R>
KF_D void seg_move(const ManySeq<N, R> &q, SegCursor &c, int64_t g) {
    while (g >= c.e) { ++c.s; c.b = c.e; c.e = __ldg(q.offsets + c.s + 1); }
    while (g < c.b) { --c.s; c.e = c.b; c.b = __ldg(q.offsets + c.s); }
}

// Filter record: the forward pass hands (xbar_{k|k}, P_{k|k}) to the smoother
// passes as one 16-byte aligned record [m (N), packed P (S), padding].
template <int N, typename R>
struct FRec {
    static constexpr int S = N * (N + 1) / 2, Q = 16 / int(sizeof(R));
    static constexpr int SIZE = ((N + S + Q - 1) / Q) * Q;
};

// Output / intermediate buffers shared by the three problems.
template <typename R>
struct KfBufs {
    const R *y;        // [total][ny]
    R *frec;           // filter records [total][FRec::SIZE] (workspace; null for a plain filter call)
    R *mf_user;        // optional filter means [total][N]
    R *Pf_user;        // optional full filter covariances [total][N][N]
    R *ms;             // smoothed means [total][N]
    R *Ps;             // smoothed full covs [total][N][N]
};

template <int N, typename R>
KF_D void store_full(R *dst, const R *packed) {
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) dst[r * N + c] = packed[si(N, r, c)];
}

// ---------------------------------------------------------------- call policy
// nx <= 4: operators are inlined (everything stays in registers).  nx = 8:
// one element no longer fits in the register file, so each operator is one
// out-of-line function shared by every call site, which keeps code size and
// compile time bounded.
template <int N, typename R, int MODE>
__device__ __noinline__ void lemma1_ool(const FElem<N, R> &a, const FElem<N, R> &b, FElem<N, R> &o) {
    lemma1<N, R, MODE>(a, b, o);
}
template <int N, typename R, int MODE>
KF_D void op_lemma1(const FElem<N, R> &a, const FElem<N, R> &b, FElem<N, R> &o) {
    if constexpr (N >= 8) lemma1_ool<N, R, MODE>(a, b, o); else lemma1<N, R, MODE>(a, b, o);
}
template <int N, typename R, int MODE, bool LL>
__device__ __noinline__ void apply_fwd_ool(FwdCarry<N, R> &c, const FElem<N, R> &e, double *ld, R *q) {
    apply_fwd<N, R, MODE, LL>(c, e, ld, q);
}
template <int N, typename R, int MODE, bool LL>
KF_D void op_apply_fwd(FwdCarry<N, R> &c, const FElem<N, R> &e, double *ld, R *q) {
    if constexpr (N >= 8) apply_fwd_ool<N, R, MODE, LL>(c, e, ld, q); else apply_fwd<N, R, MODE, LL>(c, e, ld, q);
}
template <int N, int M, typename R, int MODE>
__device__ __noinline__ void lemma1_lr_ool(const FElem<N, R> &a, const FElem<N, R> &b, const R *U, FElem<N, R> &o) {
    lemma1_lr<N, M, R, MODE>(a, b, U, o);
}
template <int N, int M, typename R, int MODE>
KF_D void op_lemma1_lr(const FElem<N, R> &a, const FElem<N, R> &b, const R *U, FElem<N, R> &o) {
    if constexpr (N >= 8) lemma1_lr_ool<N, M, R, MODE>(a, b, U, o); else lemma1_lr<N, M, R, MODE>(a, b, U, o);
}
template <int N, int M, typename R, int MODE, bool LL>
__device__ __noinline__ void apply_fwd_lr_ool(FwdCarry<N, R> &c, const FElem<N, R> &e, const R *U, const R *yt, R *q,
                                              R *ld) {
    apply_fwd_lr<N, M, R, MODE, LL>(c, e, U, yt, q, ld);
}
template <int N, int M, typename R, int MODE, bool LL>
KF_D void op_apply_fwd_lr(FwdCarry<N, R> &c, const FElem<N, R> &e, const R *U, const R *yt, R *q, R *ld) {
    if constexpr (N >= 8) apply_fwd_lr_ool<N, M, R, MODE, LL>(c, e, U, yt, q, ld);
    else apply_fwd_lr<N, M, R, MODE, LL>(c, e, U, yt, q, ld);
}
template <int N, typename R, int MODE>
__device__ __noinline__ void apply_rev_ool(RevCarry<N, R> &c, const FElem<N, R> &e) { apply_rev<N, R, MODE>(c, e); }
template <int N, typename R, int MODE>
KF_D void op_apply_rev(RevCarry<N, R> &c, const FElem<N, R> &e) {
    if constexpr (N >= 8) apply_rev_ool<N, R, MODE>(c, e); else apply_rev<N, R, MODE>(c, e);
}
template <int N, typename R>
__device__ __noinline__ void lemma2_ool(const RElem<N, R> &a, const RElem<N, R> &b, RElem<N, R> &o) { lemma2<N, R>(a, b, o); }
template <int N, typename R>
KF_D void op_lemma2(const RElem<N, R> &a, const RElem<N, R> &b, RElem<N, R> &o) {
    if constexpr (N >= 8) lemma2_ool<N, R>(a, b, o); else lemma2<N, R>(a, b, o);
}
template <int N, typename R>
__device__ __noinline__ void apply_rts_ool(RCarry<N, R> &c, const RElem<N, R> &e) { apply_rts<N, R>(c, e); }
template <int N, typename R>
KF_D void op_apply_rts(RCarry<N, R> &c, const RElem<N, R> &e) {
    if constexpr (N >= 8) apply_rts_ool<N, R>(c, e); else apply_rts<N, R>(c, e);
}
template <int N, typename R>
__device__ __noinline__ void build_rts_ool(const FiltParams<N, R> &P, bool last, const R *x, const R *Pk, RElem<N, R> &e) {
    build_rts_elem<N, R>(P, last, x, Pk, e);
}
template <int N, typename R>
KF_D void op_build_rts(const FiltParams<N, R> &P, bool last, const R *x, const R *Pk, RElem<N, R> &e) {
    if constexpr (N >= 8) build_rts_ool<N, R>(P, last, x, Pk, e); else build_rts_elem<N, R>(P, last, x, Pk, e);
}
template <int N, typename R, int MODE>
__device__ __noinline__ void tf_merge_ool(const R *x, const R *Pk, const RevCarry<N, R> &c, R *ms, R *Ps) {
    tf_merge<N, R, MODE>(x, Pk, c, ms, Ps);
}
template <int N, typename R, int MODE>
KF_D void op_tf_merge(const R *x, const R *Pk, const RevCarry<N, R> &c, R *ms, R *Ps) {
    if constexpr (N >= 8) tf_merge_ool<N, R, MODE>(x, Pk, c, ms, Ps); else tf_merge<N, R, MODE>(x, Pk, c, ms, Ps);
}

// ---------------------------------------------------------------- problems
//
// Interface used by the scan kernels.  Positions p are in scan order; the
// global index of p is g = p (forward) or g = total - 1 - p (reverse).  Each
// problem reads at most one per-position input record array (IN_REC
// elements, 0 = none) and writes up to three output record arrays (O1, O2,
// O3 elements per record, 0 = none).  build() and step() receive record
// pointers, which point either into a warp's shared-memory staging buffer or
// straight into device memory.

// ---------------------------------------------------------------- fold table
//
// For a time-invariant model every fresh element a_k (k >= 2) has the same
// (A, C, J), with b_k = K y_k and eta_k = G y_k.  When a thread folds c fresh
// elements from the left, the (A, C, J) half of its running aggregate is
// therefore a function of c alone, and Lemma 1 with the fresh element on the
// right reduces to two affine updates of (b, eta):
//   b   <- T1_c b + T4_c y_k,                  T1_c  = A (I + C_c J)^{-1},
//                                              T4_c  = T1_c C_c G + K,
//   eta <- eta + T3U_c (L^{-1} y_k - U b),     T3U_c = A_c^T (I + J C_c)^{-1} U^T,
// using G = U^T L^{-1} and J = U^T U (U = L^{-1} H F, S = L L^T).  (A_c, C_c)
// is the aggregate of c fresh elements.  The host computes the rows for
// c = 1 .. K-1 and the (A, C, J) of the K-element aggregate in FP64 for the
// launch's K (positions per thread); the kernel copies the rows into shared
// memory and every thread whose K positions are all fresh elements of one
// sequence folds with them.
//
// The run that starts at a_1 (A_1 = 0) has its own rows: its aggregate keeps
// A = 0 and (eta, J) = (eta_1, J_1) = (G y_1, J) (Lemma 1 with A_i = 0), and
// its C_c is the filtering covariance P_{c|c}, so only
// T1'_c = A (I + P_{c|c} J)^{-1} and T4'_c = T1'_c P_{c|c} G + K are needed.
template <int N, int M, typename R>
struct FoldTab {
    static constexpr int S = N * (N + 1) / 2;
    static constexpr int E = N * N + 2 * N * M;                       // row: T1 | T4 | T3U
    static constexpr int E1 = N * N + N * M;                          // first-run row: T1' | T4'
    // rows: up to 16 KB (FP32) / 12 KB (FP64) of T1 | T4 | T3U, at most 128;
    // with the first-run rows and the model constants the kernel parameters
    // stay within their 32 KB
    static constexpr int KT0 = (sizeof(R) == 4 ? 16384 : 12288) / (E * int(sizeof(R)));
    static constexpr int KT = KT0 < 128 ? KT0 : 128;
    int K;                                                            // 0: no table
    R A[N * N], C[S], J[S];                                           // aggregate of K fresh elements
    R C1K[S];                                                         // P_{K|K}: C of the first run
    alignas(16) R t[KT * E];
    alignas(16) R t1[KT * E1];
};
struct NoTab {
    int K;
};

// Tile-scan table.  In a tile where every thread folded K fresh elements
// (the table fold above), every thread aggregate has the same (A, C, J), the
// K-element aggregate; so has every run of c consecutive thread aggregates,
// its c-th power under Lemma 1.  The warp scan (Kogge-Stone, offsets
// s = 1..16) and the scan of the warp aggregates (offsets s = 1..4, spans of
// 32 threads) then combine a left span of p with a right span of s thread
// aggregates, and Lemma 1 reduces to
//   b   <- M1 b_x + M2 eta_y + b_y,      M1 = A_s X,  M2 = A_s X C_p,
//   eta <- eta_x + M3 eta_y - M4 b_x,    M3 = A_p^T X^T,  M4 = M3 J_s,
// X = (I + C_p J_s)^{-1} (x the left, y the right operand).  The host
// computes, in FP64: W(s, p) for the warp scan, V(s, p) for the warp
// aggregates, and the (A, C, J) of spans 1..32 and 32 w (w <= 8 warps),
// which complete the exclusive prefixes and the tile aggregate into
// elements.
template <int N, typename R>
struct ScanTab {
    static constexpr int NN = N * N, S = N * (N + 1) / 2;
    static constexpr int WE = 4 * NN;        // M1 | M2 | M3 | M4, row-major
    static constexpr int PE = NN + 2 * S;    // A | C | J (packed)
    static constexpr int NWARPS = 8, NWE = 31, NVE = 7, NPW = 32 + NWARPS - 1;
    static constexpr int SIZE = (NWE + NVE) * WE + NPW * PE;
    static KF_HD int w_off(int s, int p) { return (s + p - 2) * WE; }
    static KF_HD int v_off(int s, int p) { return (NWE + s + p - 2) * WE; }
    static KF_HD int pw_off(int c) { return (NWE + NVE) * WE + (c <= 32 ? c - 1 : 32 + c / 32 - 2) * PE; }
};

// One table-driven combine of (b, eta) halves: (bx, ex) the left operand,
// (b, e) the right one and the result.
template <int N, typename R>
KF_D void tsc_combine(const R *w, const R *bx, const R *ex, R *b, R *e) {
    constexpr int NN = N * N;
    R nb[N], ne[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R sb = b[r], se = ex[r];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            sb += __ldg(w + r * N + k) * bx[k] + __ldg(w + NN + r * N + k) * e[k];
            se += __ldg(w + 2 * NN + r * N + k) * e[k] - __ldg(w + 3 * NN + r * N + k) * bx[k];
        }
        nb[r] = sb;
        ne[r] = se;
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        b[r] = nb[r];
        e[r] = ne[r];
    }
}

// The element of a span of c thread aggregates with halves (b, eta).
template <int N, typename R>
KF_D void tsc_elem(const R *tab, int c, const R *b, const R *eta, FElem<N, R> &el) {
    using T = ScanTab<N, R>;
    using E = FElem<N, R>;
    const R *pw = tab + T::pw_off(c);
#pragma unroll
    for (int i = 0; i < T::NN; ++i) el.v[E::oA + i] = __ldg(pw + i);
#pragma unroll
    for (int i = 0; i < T::S; ++i) {
        el.v[E::oC + i] = __ldg(pw + T::NN + i);
        el.v[E::oJ + i] = __ldg(pw + T::NN + T::S + i);
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        el.v[E::ob + i] = b[i];
        el.v[E::oe + i] = eta[i];
    }
}

// LR > 0: every fresh element's J is U^T U of rank LR = ny, and the thread
// fold and the carry pass use the low-rank forms (kf_math.cuh).
template <int N, typename Rt, int MODE, class Src, int LR = 0>
struct FilterFwd {
    static constexpr int KIND = 0, NX = N;
    static constexpr bool REV = false;
    using R = Rt;
    using Elem = FElem<N, R>;
    using Carry = FwdCarry<N, R>;
    static constexpr int S = N * (N + 1) / 2;
    // the low-rank path knows ny = LR at compile time and stages y as its input record
    static constexpr int IN_REC = LR, O1 = FRec<N, R>::SIZE, O2 = N, O3 = N * N;
    // table-driven thread fold: low-rank path, one sequence, nx <= 4
    static constexpr bool TABLE = LR > 0 && N <= 4 && Src::ONE;
    using Tab = typename std::conditional<TABLE, FoldTab<N, (LR > 0 ? LR : 1), R>, NoTab>::type;
    struct Args {
        Src src;
        KfBufs<R> buf;
        int want_ll;
        Tab tab;
    };
    struct TabFold {
        R b[N], eta[N];
        int c;
        bool first;   // the run starts at a_1
    };
    static KF_HD int64_t total(const Args &a) { return seq_total(a.src); }
    static KF_HD const R *in_arr(const Args &a) { return LR > 0 ? a.buf.y : nullptr; }
    // rows of the fold table in bytes (0: none)
    static constexpr int tab_bytes() {
        if constexpr (TABLE) return Tab::KT * Tab::E * int(sizeof(R)); else return 0;
    }
    // Copy the table rows into shared memory (all threads of the CTA).
    static KF_D void tab_load(const Args &a, R *dst) {
        if constexpr (TABLE) {
            const int n4 = (a.tab.K > 1 ? (a.tab.K - 1) * Tab::E : 0) * int(sizeof(R)) / 16;
            const float4 *src = reinterpret_cast<const float4 *>(a.tab.t);
            float4 *d = reinterpret_cast<float4 *>(dst);
            for (int i = threadIdx.x; i < n4; i += blockDim.x) d[i] = src[i];
        }
    }
    // Does this thread's run [start, end) fold with the table?  It must hold
    // K positions (the sequence starts at position 0).
    static KF_D bool tab_fast(const Args &a, int64_t start, int64_t end, int K) {
        if constexpr (TABLE) return a.tab.K == K && K >= 2 && end - start == K;
        else return false;
    }
    static KF_D void tab_step(const Args &a, int64_t p, const R *in, const R *tab, TabFold &f) {
        if constexpr (TABLE) {
            const FiltParams<N, R> &P = a.src.prm;
            R y[LR];
            load_rec<LR>(y, y_of(a, p, in, LR));
            if (f.c == 0) {
                f.first = (p == 0);
                if (f.first) {   // a_1: b_1 = c1 + K1 y_1, eta_1 = G y_1
                    Elem e;
                    build_filter_elem<N, R>(P, 1, y, e);
#pragma unroll
                    for (int i = 0; i < N; ++i) {
                        f.b[i] = e.v[Elem::ob + i];
                        f.eta[i] = e.v[Elem::oe + i];
                    }
                } else {
                    fresh_b_eta<N, LR, R>(P, y, f.b, f.eta);
                }
            } else if (f.first) {
                constexpr int E1 = Tab::E1;
                const R *row = a.tab.t1 + (f.c - 1) * E1;   // read in place (one thread)
                const R *T1 = row, *T4 = row + N * N;
                R nb[N];
#pragma unroll
                for (int r = 0; r < N; ++r) {
                    R s = 0;
#pragma unroll
                    for (int j = 0; j < LR; ++j) s += T4[r * LR + j] * y[j];
#pragma unroll
                    for (int k = 0; k < N; ++k) s += T1[r * N + k] * f.b[k];
                    nb[r] = s;
                }
#pragma unroll
                for (int r = 0; r < N; ++r) f.b[r] = nb[r];
            } else {
                constexpr int E = Tab::E;
                R row[E];
                load_rec<E>(row, tab + (f.c - 1) * E);
                const R *T1 = row, *T4 = row + N * N, *T3U = row + N * N + N * LR;
                R v[LR];   // whitened innovation L^{-1} y - U b
#pragma unroll
                for (int i = 0; i < LR; ++i) {
                    R s = 0;
#pragma unroll
                    for (int k = 0; k <= i; ++k) s += P.Linv[i * MAXNY + k] * y[k];
#pragma unroll
                    for (int k = 0; k < N; ++k) s -= P.U[i * N + k] * f.b[k];
                    v[i] = s;
                }
                R nb[N];
#pragma unroll
                for (int r = 0; r < N; ++r) {
                    R s = 0;
#pragma unroll
                    for (int j = 0; j < LR; ++j) s += T4[r * LR + j] * y[j];
#pragma unroll
                    for (int k = 0; k < N; ++k) s += T1[r * N + k] * f.b[k];
                    nb[r] = s;
                }
#pragma unroll
                for (int r = 0; r < N; ++r) {
                    R s = f.eta[r];
#pragma unroll
                    for (int i = 0; i < LR; ++i) s += T3U[r * LR + i] * v[i];
                    f.eta[r] = s;
                }
#pragma unroll
                for (int r = 0; r < N; ++r) f.b[r] = nb[r];
            }
            ++f.c;
        }
    }
    static KF_D void tab_finish(const Args &a, const TabFold &f, Elem &agg) {
        if constexpr (TABLE) {
            if (f.first) {   // A = 0, C = P_{K|K}, (eta, J) = (eta_1, J_1)
                const FiltParams<N, R> &P = a.src.prm;
#pragma unroll
                for (int i = 0; i < N * N; ++i) agg.v[Elem::oA + i] = R(0);
#pragma unroll
                for (int i = 0; i < S; ++i) {
                    agg.v[Elem::oC + i] = a.tab.C1K[i];
                    agg.v[Elem::oJ + i] = P.J[i];
                }
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    agg.v[Elem::ob + i] = f.b[i];
                    agg.v[Elem::oe + i] = f.eta[i];
                }
                return;
            }
#pragma unroll
            for (int i = 0; i < N * N; ++i) agg.v[Elem::oA + i] = a.tab.A[i];
#pragma unroll
            for (int i = 0; i < S; ++i) {
                agg.v[Elem::oC + i] = a.tab.C[i];
                agg.v[Elem::oJ + i] = a.tab.J[i];
            }
#pragma unroll
            for (int i = 0; i < N; ++i) {
                agg.v[Elem::ob + i] = f.b[i];
                agg.v[Elem::oe + i] = f.eta[i];
            }
        }
    }
    static KF_HD R *out_arr(const Args &a, int i) { return i == 0 ? a.buf.frec : i == 1 ? a.buf.mf_user : a.buf.Pf_user; }
    static KF_D SegCursor cursor(const Args &a, int64_t p) { return seg_find(a.src, p); }
    static KF_D void build(const Args &a, int64_t p, SegCursor &cur, const R *in, Elem &e) {
        seg_move(a.src, cur, p);
        const FiltParams<N, R> &P = seg_params(a.src, cur);
        build_filter_elem<N, R>(P, p - cur.b + 1, y_of(a, p, in, P.ny), e);
    }
    static KF_D void combine(const Elem &x, const Elem &y, Elem &o) { op_lemma1<N, R, MODE>(x, y, o); }
    // x (x) y where y is the element of position p (fresh)
    static KF_D void fold(const Args &a, const SegCursor &cur, const Elem &x, const Elem &y, Elem &o) {
        if constexpr (LR > 0) op_lemma1_lr<N, LR, R, MODE>(x, y, seg_params(a.src, cur).U, o);
        else op_lemma1<N, R, MODE>(x, y, o);
    }
    static KF_D void apply(Carry &c, const Elem &e) { op_apply_fwd<N, R, MODE, false>(c, e, nullptr, nullptr); }
    static KF_D void apply_fresh(const Args &a, const SegCursor &cur, Carry &c, const Elem &e) {
        if constexpr (LR > 0)
            op_apply_fwd_lr<N, LR, R, MODE, false>(c, e, seg_params(a.src, cur).U, nullptr, nullptr, nullptr);
        else
            op_apply_fwd<N, R, MODE, false>(c, e, nullptr, nullptr);
    }
    static KF_D void carry_of(const Elem &e, Carry &c) {
#pragma unroll
        for (int i = 0; i < N; ++i) c.v[Carry::ob + i] = e.v[Elem::ob + i];
#pragma unroll
        for (int i = 0; i < S; ++i) c.v[Carry::oC + i] = e.v[Elem::oC + i];
    }
    // A exactly zero: the element's (b, C) is what it makes of any carry
    static KF_D bool zero_transition(const Elem &e) {
        bool z = true;
#pragma unroll
        for (int i = 0; i < N * N; ++i) z = z && e.v[Elem::oA + i] == R(0);
        return z;
    }
    // outputs of the position p (global index p) whose prefix carry is c
    static KF_D void emit(const Args &, int64_t, SegCursor &, const Carry &c, const R *, R *o1, R *o2, R *o3) {
        const R *b = c.v + Carry::ob, *C = c.v + Carry::oC;
        if (o1) {
            R rec[O1];
#pragma unroll
            for (int i = 0; i < N; ++i) rec[i] = b[i];
#pragma unroll
            for (int i = 0; i < S; ++i) rec[N + i] = C[i];
#pragma unroll
            for (int i = N + S; i < O1; ++i) rec[i] = 0;
            store_rec<O1>(o1, rec);
        }
        if (o2) store_rec<N>(o2, b);
        if (o3) {
            R full[N * N];
            store_full<N>(full, C);
            store_rec<N * N>(o3, full);
        }
    }
    // measurement of position p: staged record (low-rank path) or device memory
    static KF_D const R *y_of(const Args &a, int64_t p, const R *in, int ny) {
        return (LR > 0 && in) ? in : a.buf.y + p * ny;
    }
    // agg <- agg (x) a_p
    static KF_D void fold_at(const Args &a, int64_t p, SegCursor &cur, const R *in, Elem &agg) {
        if constexpr (LR > 0) {
            seg_move(a.src, cur, p);
            const FiltParams<N, R> &P = seg_params(a.src, cur);
            if (p != cur.b) {
                R yv[LR], b[N], eta[N];
                load_rec<LR>(yv, y_of(a, p, in, LR));
                fresh_b_eta<N, LR, R>(P, yv, b, eta);
                Elem t;
                if constexpr (N >= 8) {
                    Elem e;
                    build_filter_elem<N, R>(P, 2, yv, e);
                    op_lemma1_lr<N, LR, R, MODE>(agg, e, P.U, t);
                } else {
                    lemma1_lr_parts<N, LR, R, MODE>(agg, P.A, b, P.C, eta, P.U, t);
                }
                agg = t;
                return;
            }
        }
        Elem e, t;
        build(a, p, cur, in, e);
        fold(a, cur, agg, e, t);
        agg = t;
    }
    // log p(y_k | y_{1:k-1}) from the prefix carry c = s_{k-1} before a_k is
    // applied.  k = 1: v = y_1 - H xbar_{1|0}, S_1 precomputed.  k >= 2:
    // S_k = S + HF C F^T H^T, so det S_k = det S det(I + C J) and, with
    // w = eta_k - J b = F^T H^T S^{-1} v, v^T S_k^{-1} v = v^T S^{-1} v - w^T D w,
    // D = (I + C J)^{-1} C (matrix determinant lemma and Woodbury identity).
    // c <- c (x) a_p, outputs of p, log-likelihood term of p
    static KF_D R step_at(const Args &a, int64_t p, SegCursor &cur, Carry &c, const R *in, R *o1, R *o2, R *o3) {
        if constexpr (LR > 0) {
            seg_move(a.src, cur, p);
            const FiltParams<N, R> &P = seg_params(a.src, cur);
            if (p != cur.b) {
                R yv[LR], b[N], eta[N];
                load_rec<LR>(yv, y_of(a, p, in, LR));
                fresh_b_eta<N, LR, R>(P, yv, b, eta);
                R ll = 0;
                if (a.want_ll) {
                    R yt[LR];
#pragma unroll
                    for (int i = 0; i < LR; ++i) {
                        R s = 0;
#pragma unroll
                        for (int k = 0; k <= i; ++k) s += P.Linv[i * MAXNY + k] * yv[k];
                        yt[i] = s;
                    }
                    R q, ld;
                    if constexpr (N >= 8) {
                        Elem e;
                        build_filter_elem<N, R>(P, 2, yv, e);
                        op_apply_fwd_lr<N, LR, R, MODE, true>(c, e, P.U, yt, &q, &ld);
                    } else {
                        apply_fwd_lr_parts<N, LR, R, MODE, true>(c, P.A, b, P.C, eta, P.U, yt, &q, &ld);
                    }
                    // the per-step term in the working precision; FP64 only accumulates
                    ll = R(-0.5) * (q + ld + P.llc_r);
                } else {
                    if constexpr (N >= 8) {
                        Elem e;
                        build_filter_elem<N, R>(P, 2, yv, e);
                        op_apply_fwd_lr<N, LR, R, MODE, false>(c, e, P.U, nullptr, nullptr, nullptr);
                    } else {
                        apply_fwd_lr_parts<N, LR, R, MODE, false>(c, P.A, b, P.C, eta, P.U, nullptr, nullptr, nullptr);
                    }
                }
                emit(a, p, cur, c, in, o1, o2, o3);
                return ll;
            }
        }
        Elem e;
        build(a, p, cur, in, e);
        return R(step(a, p, cur, c, e, in, o1, o2, o3));
    }
    static KF_D double step(const Args &a, int64_t p, SegCursor &cur, Carry &c, const Elem &e, const R *in, R *o1,
                            R *o2, R *o3) {
        if (!a.want_ll) {
            apply_fresh(a, cur, c, e);
            emit(a, p, cur, c, in, o1, o2, o3);
            return 0.0;
        }
        const FiltParams<N, R> &P = seg_params(a.src, cur);
        const int ny = P.ny;
        const R *yk = y_of(a, p, in, ny);
        double ll;
        if (p == cur.b) {
            R v[MAXNY];
#pragma unroll
            for (int j = 0; j < MAXNY; ++j) v[j] = (j < ny) ? yk[j] - P.Hx1[j] : R(0);
            R q = 0;
#pragma unroll
            for (int i = 0; i < MAXNY; ++i)
#pragma unroll
                for (int j = 0; j < MAXNY; ++j)
                    if (i < ny && j < ny) q += v[i] * P.S1inv[i * MAXNY + j] * v[j];
            ll = -0.5 * (double(q) + P.llc1);
            apply_fresh(a, cur, c, e);
        } else if constexpr (LR > 0) {
            R yt[LR];
#pragma unroll
            for (int i = 0; i < LR; ++i) {
                R s = 0;
#pragma unroll
                for (int k = 0; k <= i; ++k) s += P.Linv[i * MAXNY + k] * yk[k];
                yt[i] = s;
            }
            R q, ld;
            op_apply_fwd_lr<N, LR, R, MODE, true>(c, e, P.U, yt, &q, &ld);
            ll = double(R(-0.5) * (q + ld + P.llc_r));
        } else {
            const R *b = c.v + Carry::ob;
            R v[MAXNY];
#pragma unroll
            for (int j = 0; j < MAXNY; ++j) {
                R s = (j < ny) ? yk[j] : R(0);
#pragma unroll
                for (int k = 0; k < N; ++k) s -= (j < ny) ? P.HF[j * N + k] * b[k] : R(0);
                v[j] = s;
            }
            R q = 0;
#pragma unroll
            for (int i = 0; i < MAXNY; ++i)
#pragma unroll
                for (int j = 0; j < MAXNY; ++j)
                    if (i < ny && j < ny) q += v[i] * P.Sinv[i * MAXNY + j] * v[j];
            double ld;
            R wDw;
            op_apply_fwd<N, R, MODE, true>(c, e, &ld, &wDw);
            ll = -0.5 * (double(q) - double(wDw) + P.llc + ld);
        }
        emit(a, p, cur, c, in, o1, o2, o3);
        return ll;
    }
};

// ---------------------------------------------------------------- two-filter (reverse)

template <int N, typename Rt, int MODE, class Src>
struct TfRev {
    static constexpr int KIND = 2;
    static constexpr bool REV = true;
    using R = Rt;
    using Elem = FElem<N, R>;
    using Carry = RevCarry<N, R>;
    static constexpr int S = N * (N + 1) / 2;
    static constexpr int IN_REC = FRec<N, R>::SIZE, O1 = N, O2 = N * N, O3 = 0;
    struct Args {
        Src src;
        KfBufs<R> buf;
        int want_ll;
    };
    static constexpr bool TABLE = false;
    struct TabFold {};
    static constexpr int tab_bytes() { return 0; }
    static KF_D void tab_load(const Args &, R *) {}
    static KF_D bool tab_fast(const Args &, int64_t, int64_t, int) { return false; }
    static KF_D void tab_step(const Args &, int64_t, const R *, const R *, TabFold &) {}
    static KF_D void tab_finish(const Args &, const TabFold &, Elem &) {}
    static KF_HD int64_t total(const Args &a) { return seq_total(a.src); }
    static KF_HD const R *in_arr(const Args &a) { return a.buf.frec; }
    static KF_HD R *out_arr(const Args &a, int i) { return i == 0 ? a.buf.ms : i == 1 ? a.buf.Ps : nullptr; }
    static KF_D SegCursor cursor(const Args &a, int64_t p) { return seg_find(a.src, seq_total(a.src) - 1 - p); }
    // position p holds b_k = a_{k+1} (k < T_s) or e = 0 (k = T_s), where
    // g = total-1-p is the global index of time k.
    static KF_D void build(const Args &a, int64_t p, SegCursor &cur, const R *, Elem &e) {
        const int64_t g = seq_total(a.src) - 1 - p;
        seg_move(a.src, cur, g);
        if (g == cur.e - 1) {
            set_zero(e);
            return;
        }
        const FiltParams<N, R> &P = seg_params(a.src, cur);
        build_filter_elem<N, R>(P, g - cur.b + 2, a.buf.y + (g + 1) * P.ny, e);
    }
    static KF_D void combine(const Elem &x, const Elem &y, Elem &o) { op_lemma1<N, R, MODE>(y, x, o); }
    static KF_D void fold(const Args &, const SegCursor &, const Elem &x, const Elem &y, Elem &o) { combine(x, y, o); }
    static KF_D void apply(Carry &c, const Elem &e) { op_apply_rev<N, R, MODE>(c, e); }
    static KF_D void carry_of(const Elem &e, Carry &c) {
#pragma unroll
        for (int i = 0; i < N; ++i) c.v[Carry::oe + i] = e.v[Elem::oe + i];
#pragma unroll
        for (int i = 0; i < S; ++i) c.v[Carry::oJ + i] = e.v[Elem::oJ + i];
    }
    // A exactly zero: the element's (eta, J) is what it makes of any carry
    static KF_D bool zero_transition(const Elem &e) {
        bool z = true;
#pragma unroll
        for (int i = 0; i < N * N; ++i) z = z && e.v[Elem::oA + i] == R(0);
        return z;
    }
    // merge with the filter record (Eqs. mean_tf_combination / cov_tf_combination)
    static KF_D void emit(const Args &, int64_t, SegCursor &, const Carry &c, const R *in, R *o1, R *o2, R *) {
        R rec[IN_REC], ms[N], Ps[S], full[N * N];
        load_rec<IN_REC>(rec, in);
        op_tf_merge<N, R, MODE>(rec, rec + N, c, ms, Ps);
        store_rec<N>(o1, ms);
        store_full<N>(full, Ps);
        store_rec<N * N>(o2, full);
    }
    static KF_D void fold_at(const Args &a, int64_t p, SegCursor &cur, const R *in, Elem &agg) {
        Elem e, t;
        build(a, p, cur, in, e);
        combine(agg, e, t);
        agg = t;
    }
    static KF_D R step_at(const Args &a, int64_t p, SegCursor &cur, Carry &c, const R *in, R *o1, R *o2, R *o3) {
        Elem e;
        build(a, p, cur, in, e);
        return step(a, p, cur, c, e, in, o1, o2, o3);
    }
    static KF_D double step(const Args &a, int64_t p, SegCursor &cur, Carry &c, const Elem &e, const R *in, R *o1,
                            R *o2, R *o3) {
        apply(c, e);
        emit(a, p, cur, c, in, o1, o2, o3);
        return 0.0;
    }
};

// ---------------------------------------------------------------- RTS (reverse)

template <int N, typename Rt, class Src>
struct RtsRev {
    static constexpr int KIND = 1;
    static constexpr bool REV = true;
    using R = Rt;
    using Elem = RElem<N, R>;
    using Carry = RCarry<N, R>;
    static constexpr int S = N * (N + 1) / 2;
    static constexpr int IN_REC = FRec<N, R>::SIZE, O1 = N, O2 = N * N, O3 = 0;
    struct Args {
        Src src;
        KfBufs<R> buf;
        int want_ll;
    };
    static constexpr bool TABLE = false;
    struct TabFold {};
    static constexpr int tab_bytes() { return 0; }
    static KF_D void tab_load(const Args &, R *) {}
    static KF_D bool tab_fast(const Args &, int64_t, int64_t, int) { return false; }
    static KF_D void tab_step(const Args &, int64_t, const R *, const R *, TabFold &) {}
    static KF_D void tab_finish(const Args &, const TabFold &, Elem &) {}
    static KF_HD int64_t total(const Args &a) { return seq_total(a.src); }
    static KF_HD const R *in_arr(const Args &a) { return a.buf.frec; }
    static KF_HD R *out_arr(const Args &a, int i) { return i == 0 ? a.buf.ms : i == 1 ? a.buf.Ps : nullptr; }
    static KF_D SegCursor cursor(const Args &a, int64_t p) { return seg_find(a.src, seq_total(a.src) - 1 - p); }
    static KF_D void build(const Args &a, int64_t p, SegCursor &cur, const R *in, Elem &e) {
        const int64_t g = seq_total(a.src) - 1 - p;
        seg_move(a.src, cur, g);
        R rec[IN_REC];
        load_rec<IN_REC>(rec, in);
        op_build_rts<N, R>(seg_params(a.src, cur), g == cur.e - 1, rec, rec + N, e);
    }
    static KF_D void fold_at(const Args &a, int64_t p, SegCursor &cur, const R *in, Elem &agg) {
        Elem e, t;
        build(a, p, cur, in, e);
        combine(agg, e, t);
        agg = t;
    }
    static KF_D R step_at(const Args &a, int64_t p, SegCursor &cur, Carry &c, const R *in, R *o1, R *o2, R *o3) {
        Elem e;
        build(a, p, cur, in, e);
        return step(a, p, cur, c, e, in, o1, o2, o3);
    }
    static KF_D void combine(const Elem &x, const Elem &y, Elem &o) { op_lemma2<N, R>(y, x, o); }
    static KF_D void fold(const Args &, const SegCursor &, const Elem &x, const Elem &y, Elem &o) { combine(x, y, o); }
    static KF_D void apply(Carry &c, const Elem &e) { op_apply_rts<N, R>(c, e); }
    static KF_D void carry_of(const Elem &e, Carry &c) {
#pragma unroll
        for (int i = 0; i < N; ++i) c.v[Carry::og + i] = e.v[Elem::og + i];
#pragma unroll
        for (int i = 0; i < S; ++i) c.v[Carry::oL + i] = e.v[Elem::oL + i];
    }
    // E exactly zero: the element's (g, L) is what it makes of any carry
    static KF_D bool zero_transition(const Elem &e) {
        bool z = true;
#pragma unroll
        for (int i = 0; i < N * N; ++i) z = z && e.v[Elem::oE + i] == R(0);
        return z;
    }
    static KF_D void emit(const Args &, int64_t, SegCursor &, const Carry &c, const R *, R *o1, R *o2, R *) {
        R full[N * N];
        store_rec<N>(o1, c.v + Carry::og);
        store_full<N>(full, c.v + Carry::oL);
        store_rec<N * N>(o2, full);
    }
    static KF_D double step(const Args &a, int64_t p, SegCursor &cur, Carry &c, const Elem &e, const R *in, R *o1,
                            R *o2, R *o3) {
        apply(c, e);
        emit(a, p, cur, c, in, o1, o2, o3);
        return 0.0;
    }
};

// Direct (unstaged) record pointers of position p, for the level kernels.
template <class P>
KF_D int64_t global_index(const typename P::Args &a, int64_t p) {
    return P::REV ? P::total(a) - 1 - p : p;
}
template <class P>
KF_D const typename P::R *in_rec_direct(const typename P::Args &a, int64_t g) {
    const typename P::R *b = P::in_arr(a);
    return (P::IN_REC && b) ? b + g * P::IN_REC : nullptr;
}
template <class P>
KF_D typename P::R *out_rec_direct(const typename P::Args &a, int i, int64_t g) {
    constexpr int sz[3] = {P::O1, P::O2, P::O3};
    typename P::R *b = P::out_arr(a, i);
    return (sz[i] && b) ? b + g * sz[i] : nullptr;
}

}  // namespace kfs
