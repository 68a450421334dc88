// kf_tv.cuh -- the three scans of arXiv 2511.10363 on a time-varying model:
// the general linear-Gaussian model of Sec. III-A with per-step F_{k-1},
// Q_{k-1}, u_{k-1}, H_k, R_k, d_k.  Every element is built from its own
// step's matrices inside the scan pass (the "initialization" loops of
// Algs. pkf, prts and ptf), so nothing k-invariant is precomputed; the scan
// kernel, the operators of Lemmas 1 and 2 and the two-filter merge are the
// ones of the time-invariant path.
//
// Per-step arrays (device, working precision), record t = 0 .. T-1 of time
// k = t + 1: F[t] = F_{k-1}, Q[t] = Q_{k-1}, u[t] = u_{k-1} (or none),
// H[t] = H_k, R[t] = R_k, d[t] = d_k (or none), y[t] = y_k.  Only the upper
// triangles of Q[t] and R[t] are read.  ny <= nx.  One sequence per call.
#pragma once

#include <type_traits>

#include "kf_launch.cuh"
#include "kf_tv_host.h"

namespace kfs {

template <int N, typename R>
struct TvSeq {
    const R *F, *Q, *u, *H, *Rm, *d;
    int ny;
    int64_t T;
    double m0[N], P0[N * N];   // prior xbar_{0|0}, P_{0|0}
};

// Lower Cholesky factor L of a packed upper-triangular SPD matrix S (M x M),
// rows packed (row i holds columns 0..i), and the reciprocals of its
// diagonal; the return value is log det S.
template <int M, typename T>
KF_D T tv_chol(const T *S, T *L, T *dinv) {
    T ld = 0;
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            T s = S[su(M, j, i)];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[i * (i + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
            if (i == j) {
                const T dg = ksqrt(s);
                L[i * (i + 1) / 2 + i] = dg;
                dinv[i] = recip(dg);
                ld += klog(s);
            } else {
                L[i * (i + 1) / 2 + j] = s * dinv[j];
            }
        }
    return ld;
}

// X <- L^{-1} X for NC right-hand sides stored by rows (X[i * NC + c]).
template <int M, int NC, typename T>
KF_D void tv_forward_subst(const T *L, const T *dinv, T *X) {
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            T s = X[i * NC + c];
#pragma unroll
            for (int k = 0; k < i; ++k) s -= L[i * (i + 1) / 2 + k] * X[k * NC + c];
            X[i * NC + c] = s * dinv[i];
        }
}

// The measurement model of record g padded to M = N rows: H (rows l >= ny
// zero), the residual r = y - H z - d against a state z, and the packed
// covariance S = H P H^T + R for a packed state covariance P (unit diagonal
// on the padding rows, which then drop out of every product).
template <int N, typename R, typename T>
KF_D void tv_meas(const TvSeq<N, R> &s, int64_t g, const R *yk, const T *z, const T *P, T *Hm, T *HP, T *r, T *Sm) {
    constexpr int M = N;
    const int ny = s.ny;
    const R *Hp = s.H + g * int64_t(ny) * N, *Rp = s.Rm + g * int64_t(ny) * ny;
#pragma unroll
    for (int l = 0; l < M; ++l) {
        const bool on = l < ny;
        T acc = on ? T(yk[l]) - (s.d ? T(__ldg(s.d + g * ny + l)) : T(0)) : T(0);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const T h = on ? T(__ldg(Hp + l * N + k)) : T(0);
            Hm[l * N + k] = h;
            acc -= h * z[k];
        }
        r[l] = acc;
    }
#pragma unroll
    for (int l = 0; l < M; ++l)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            T acc = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) acc += Hm[l * N + k] * P[si(N, k, c)];
            HP[l * N + c] = acc;
        }
#pragma unroll
    for (int l = 0; l < M; ++l)
#pragma unroll
        for (int m = l; m < M; ++m) {
            T acc = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) acc += HP[l * N + k] * Hm[m * N + k];
            const bool on = (l < ny) && (m < ny);
            Sm[su(M, l, m)] = on ? acc + T(__ldg(Rp + l * ny + m)) : (l == m ? T(1) : T(0));
        }
}

// Prediction through record g from (x, P packed): xp = F x + u,
// Pp = F P F^T + Q (packed); F is returned for further use.
template <int N, typename R, typename T, typename X>
KF_D void tv_predict(const TvSeq<N, R> &s, int64_t g, const X *x, const X *P, bool P_full, T *F, T *xp, T *Pp) {
    constexpr int NN = N * N;
    const R *Fp = s.F + g * NN, *Qp = s.Q + g * NN;
#pragma unroll
    for (int i = 0; i < NN; ++i) F[i] = T(__ldg(Fp + i));
    T FP[NN];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            T acc = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) acc += F[r * N + k] * T(P_full ? P[k * N + c] : P[si(N, k, c)]);
            FP[r * N + c] = acc;
        }
#pragma unroll
    for (int r = 0; r < N; ++r) {
#pragma unroll
        for (int c = r; c < N; ++c) {
            T acc = T(__ldg(Qp + r * N + c));
#pragma unroll
            for (int k = 0; k < N; ++k) acc += FP[r * N + k] * F[c * N + k];
            Pp[su(N, r, c)] = acc;
        }
        T acc = s.u ? T(__ldg(s.u + g * N + r)) : T(0);
#pragma unroll
        for (int k = 0; k < N; ++k) acc += F[r * N + k] * T(x[k]);
        xp[r] = acc;
    }
}

// Element a_k of record g (time k = g + 1): Eq. pkf_init1 (k >= 2),
// Eq. pkf_init2 (k = 1) and Eq. pkf_init3, computed in type T.  With
// (Qe, ue) = (Q_{k-1}, u_{k-1}) for k >= 2 and (P_{1|0}, xbar_{1|0}) for
// k = 1, S = H Qe H^T + R = L L^T, W1 = L^{-1} H Qe, W2 = L^{-1} H F and
// w = L^{-1} (y - H ue - d):
//   A = F - W1^T W2 (A_1 = 0),  b = ue + W1^T w,  C = Qe - W1^T W1,
//   eta = W2^T w,  J = W2^T W2,
// since K = Qe H^T S^{-1} = W1^T L^{-1}.  For k = 1, eta_1 and J_1 come out
// with S_1; they never reach an output because A_1 = 0.
template <int N, typename R, typename T>
KF_D void tv_filter_elem(const TvSeq<N, R> &s, int64_t g, const R *yk, FElem<N, R> &e) {
    using E = FElem<N, R>;
    constexpr int NN = N * N, S = N * (N + 1) / 2, M = N;
    T F[NN], Qe[S], ue[N];
    if (g == 0) {
        tv_predict<N, R, T, double>(s, 0, s.m0, s.P0, true, F, ue, Qe);
    } else {
        const R *Fp = s.F + g * NN, *Qp = s.Q + g * NN;
#pragma unroll
        for (int i = 0; i < NN; ++i) F[i] = T(__ldg(Fp + i));
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = i; j < N; ++j) Qe[su(N, i, j)] = T(__ldg(Qp + i * N + j));
#pragma unroll
        for (int i = 0; i < N; ++i) ue[i] = s.u ? T(__ldg(s.u + g * N + i)) : T(0);
    }
    T Hm[M * N], W1[M * N], w[M], Sm[M * (M + 1) / 2];
    tv_meas<N, R, T>(s, g, yk, ue, Qe, Hm, W1, w, Sm);
    T W2[M * N];
#pragma unroll
    for (int l = 0; l < M; ++l)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            T acc = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) acc += Hm[l * N + k] * F[k * N + c];
            W2[l * N + c] = acc;
        }
    T L[M * (M + 1) / 2], dinv[M];
    tv_chol<M, T>(Sm, L, dinv);
    tv_forward_subst<M, N, T>(L, dinv, W1);
    tv_forward_subst<M, N, T>(L, dinv, W2);
    tv_forward_subst<M, 1, T>(L, dinv, w);
    const bool first = (g == 0);
#pragma unroll
    for (int r = 0; r < N; ++r) {
        T sb = ue[r], se = 0;
#pragma unroll
        for (int l = 0; l < M; ++l) {
            sb += W1[l * N + r] * w[l];
            se += W2[l * N + r] * w[l];
        }
        e.v[E::ob + r] = R(sb);
        e.v[E::oe + r] = R(se);
#pragma unroll
        for (int c = 0; c < N; ++c) {
            T acc = F[r * N + c];
#pragma unroll
            for (int l = 0; l < M; ++l) acc -= W1[l * N + r] * W2[l * N + c];
            e.v[E::oA + r * N + c] = first ? R(0) : R(acc);
        }
#pragma unroll
        for (int c = r; c < N; ++c) {
            T ac = Qe[su(N, r, c)], aj = 0;
#pragma unroll
            for (int l = 0; l < M; ++l) {
                ac -= W1[l * N + r] * W1[l * N + c];
                aj += W2[l * N + r] * W2[l * N + c];
            }
            e.v[E::oC + su(N, r, c)] = R(ac);
            e.v[E::oJ + su(N, r, c)] = R(aj);
        }
    }
}

// log p(y_k | y_{1:k-1}) of record g from the filtering result of time k-1
// (x, P packed), or from the prior (m0, P0) at g = 0, in innovation form:
// -1/2 (v^T S_k^{-1} v + log det S_k + ny log 2 pi), v = y_k - H_k xbar_{k|k-1} - d_k,
// S_k = H_k P_{k|k-1} H_k^T + R_k.  The quadratic form and log-determinant
// are computed in type T.
template <int N, typename R, typename T>
KF_D double tv_ll_term(const TvSeq<N, R> &s, int64_t g, const R *yk, const R *x, const R *P) {
    constexpr int NN = N * N, S = N * (N + 1) / 2, M = N;
    T F[NN], xp[N], Pp[S];
    if (g == 0) tv_predict<N, R, T, double>(s, 0, s.m0, s.P0, true, F, xp, Pp);
    else tv_predict<N, R, T, R>(s, g, x, P, false, F, xp, Pp);
    T Hm[M * N], HP[M * N], v[M], Sm[M * (M + 1) / 2], L[M * (M + 1) / 2], dinv[M];
    tv_meas<N, R, T>(s, g, yk, xp, Pp, Hm, HP, v, Sm);
    const T ld = tv_chol<M, T>(Sm, L, dinv);
    tv_forward_subst<M, 1, T>(L, dinv, v);
    T q = 0;
#pragma unroll
    for (int l = 0; l < M; ++l) q += v[l] * v[l];
    return -0.5 * double(q + ld) - 0.5 * s.ny * 1.8378770664093454835606594728112;
}

// RTS element of record g (time k = g + 1) from xbar_{k|k}, P_{k|k} (packed):
// Eq. prts_init1 with the step k -> k+1 of record g + 1 (k < T), or
// Eq. prts_init2 (k = T).  With U = F_k P, Pp = U F_k^T + Q_k = L L^T:
//   E = (Pp^{-1} U)^T,  g = x - E (F_k x + u_k),  L_k = P - E U.
template <int N, typename R>
KF_D void tv_rts_elem(const TvSeq<N, R> &s, int64_t g, const R *x, const R *Pk, RElem<N, R> &e) {
    using E = RElem<N, R>;
    constexpr int NN = N * N;
    if (g == s.T - 1) {
#pragma unroll
        for (int i = 0; i < NN; ++i) e.v[E::oE + i] = 0;
#pragma unroll
        for (int i = 0; i < N; ++i) e.v[E::og + i] = x[i];
#pragma unroll
        for (int i = 0; i < E::S; ++i) e.v[E::oL + i] = Pk[i];
        return;
    }
    const int64_t t = g + 1;
    const R *Fp = s.F + t * NN, *Qp = s.Q + t * NN;
    R F[NN], U[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i) F[i] = __ldg(Fp + i);
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R acc = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) acc += F[r * N + k] * Pk[si(N, k, c)];
            U[r * N + c] = acc;
        }
    R Pp[N * (N + 1) / 2];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            R acc = __ldg(Qp + r * N + c);
#pragma unroll
            for (int k = 0; k < N; ++k) acc += U[r * N + k] * F[c * N + k];
            Pp[su(N, r, c)] = acc;
        }
    R L[N * (N + 1) / 2], dinv[N];
    tv_chol<N, R>(Pp, L, dinv);
    // Et = Pp^{-1} U: forward then backward substitution
    R Et[NN];
#pragma unroll
    for (int i = 0; i < NN; ++i) Et[i] = U[i];
    tv_forward_subst<N, N, R>(L, dinv, Et);
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
            R acc = Et[i * N + c];
#pragma unroll
            for (int k = i + 1; k < N; ++k) acc -= L[k * (k + 1) / 2 + i] * Et[k * N + c];
            Et[i * N + c] = acc * dinv[i];
        }
    R Fx[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R acc = s.u ? __ldg(s.u + t * N + r) : R(0);
#pragma unroll
        for (int k = 0; k < N; ++k) acc += F[r * N + k] * x[k];
        Fx[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
#pragma unroll
        for (int c = 0; c < N; ++c) e.v[E::oE + r * N + c] = Et[c * N + r];
        R acc = x[r];
#pragma unroll
        for (int k = 0; k < N; ++k) acc -= Et[k * N + r] * Fx[k];
        e.v[E::og + r] = acc;
#pragma unroll
        for (int c = r; c < N; ++c) {
            R a2 = Pk[su(N, r, c)];
#pragma unroll
            for (int k = 0; k < N; ++k) a2 -= Et[k * N + r] * U[k * N + c];
            e.v[E::oL + su(N, r, c)] = a2;
        }
    }
}

// nx = 8: the builders are out of line, like the operators (kf_problems.cuh).
template <int N, typename R, typename T>
__device__ __noinline__ void tv_filter_elem_ool(const TvSeq<N, R> &s, int64_t g, const R *yk, FElem<N, R> &e) {
    tv_filter_elem<N, R, T>(s, g, yk, e);
}
template <int N, typename R, typename T>
KF_D void op_tv_filter_elem(const TvSeq<N, R> &s, int64_t g, const R *yk, FElem<N, R> &e) {
    if constexpr (N >= 8) tv_filter_elem_ool<N, R, T>(s, g, yk, e); else tv_filter_elem<N, R, T>(s, g, yk, e);
}
template <int N, typename R, typename T>
__device__ __noinline__ double tv_ll_term_ool(const TvSeq<N, R> &s, int64_t g, const R *yk, const R *x, const R *P) {
    return tv_ll_term<N, R, T>(s, g, yk, x, P);
}
template <int N, typename R, typename T>
KF_D double op_tv_ll_term(const TvSeq<N, R> &s, int64_t g, const R *yk, const R *x, const R *P) {
    if constexpr (N >= 8) return tv_ll_term_ool<N, R, T>(s, g, yk, x, P); else return tv_ll_term<N, R, T>(s, g, yk, x, P);
}
template <int N, typename R>
__device__ __noinline__ void tv_rts_elem_ool(const TvSeq<N, R> &s, int64_t g, const R *x, const R *Pk, RElem<N, R> &e) {
    tv_rts_elem<N, R>(s, g, x, Pk, e);
}
template <int N, typename R>
KF_D void op_tv_rts_elem(const TvSeq<N, R> &s, int64_t g, const R *x, const R *Pk, RElem<N, R> &e) {
    if constexpr (N >= 8) tv_rts_elem_ool<N, R>(s, g, x, Pk, e); else tv_rts_elem<N, R>(s, g, x, Pk, e);
}

// Stubs of the fold-table interface (no table for time-varying models).
#define KF_TV_NO_TABLE                                                                   \
    static constexpr bool TABLE = false;                                                 \
    struct TabFold {};                                                                   \
    static constexpr int tab_bytes() { return 0; }                                       \
    static KF_D void tab_load(const Args &, R *) {}                                      \
    static KF_D bool tab_fast(const Args &, int64_t, int64_t, int) { return false; }     \
    static KF_D void tab_step(const Args &, int64_t, const R *, const R *, TabFold &) {} \
    static KF_D void tab_finish(const Args &, const TabFold &, Elem &) {}

// ---------------------------------------------------------------- filter (forward)

// Alg. pkf: forward scan of a_1..a_T, carry (b, C), extraction
// xbar_{k|k} = b_k^+, P_{k|k} = C_k^+, and the log-likelihood.  MODE 1 builds
// the elements and the log-likelihood terms in FP64.
template <int N, typename Rt, int MODE>
struct FilterTv {
    static constexpr int KIND = 0, NX = N;
    static constexpr bool REV = false;
    using R = Rt;
    using T = typename std::conditional<MODE == 1, double, R>::type;
    using Elem = FElem<N, R>;
    using Carry = FwdCarry<N, R>;
    static constexpr int S = N * (N + 1) / 2;
    static constexpr int IN_REC = 0, O1 = FRec<N, R>::SIZE, O2 = N, O3 = N * N;
    struct Args {
        TvSeq<N, R> src;
        KfBufs<R> buf;
        int want_ll;
        NoTab tab;
    };
    KF_TV_NO_TABLE
    static KF_HD int64_t total(const Args &a) { return a.src.T; }
    static KF_HD const R *in_arr(const Args &) { return nullptr; }
    static KF_HD R *out_arr(const Args &a, int i) { return i == 0 ? a.buf.frec : i == 1 ? a.buf.mf_user : a.buf.Pf_user; }
    static KF_D SegCursor cursor(const Args &a, int64_t) { return SegCursor{0, 0, a.src.T}; }
    static KF_D void build(const Args &a, int64_t p, SegCursor &, const R *, Elem &e) {
        op_tv_filter_elem<N, R, T>(a.src, p, a.buf.y + p * a.src.ny, e);
    }
    static KF_D void combine(const Elem &x, const Elem &y, Elem &o) { op_lemma1<N, R, MODE>(x, y, o); }
    static KF_D void fold(const Args &, const SegCursor &, const Elem &x, const Elem &y, Elem &o) { combine(x, y, o); }
    static KF_D void apply(Carry &c, const Elem &e) { op_apply_fwd<N, R, MODE, false>(c, e, nullptr, nullptr); }
    // the transition block exactly zero: the element's half is what it makes of any carry
    static KF_D bool zero_transition(const Elem &e) {
        bool z = true;
#pragma unroll
        for (int i = 0; i < N * N; ++i) z = z && e.v[Elem::oA + i] == R(0);
        return z;
    }
    static KF_D void carry_of(const Elem &e, Carry &c) {
#pragma unroll
        for (int i = 0; i < N; ++i) c.v[Carry::ob + i] = e.v[Elem::ob + i];
#pragma unroll
        for (int i = 0; i < S; ++i) c.v[Carry::oC + i] = e.v[Elem::oC + i];
    }
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
    static KF_D void fold_at(const Args &a, int64_t p, SegCursor &cur, const R *in, Elem &agg) {
        Elem e, t;
        build(a, p, cur, in, e);
        combine(agg, e, t);
        agg = t;
    }
    static KF_D R step_at(const Args &a, int64_t p, SegCursor &cur, Carry &c, const R *in, R *o1, R *o2, R *o3) {
        Elem e;
        build(a, p, cur, in, e);
        return R(step(a, p, cur, c, e, in, o1, o2, o3));
    }
    // c is the prefix carry s_{k-1} before a_k is applied
    static KF_D double step(const Args &a, int64_t p, SegCursor &cur, Carry &c, const Elem &e, const R *in, R *o1,
                            R *o2, R *o3) {
        double ll = 0.0;
        if (a.want_ll)
            ll = op_tv_ll_term<N, R, T>(a.src, p, a.buf.y + p * a.src.ny, c.v + Carry::ob, c.v + Carry::oC);
        apply(c, e);
        emit(a, p, cur, c, in, o1, o2, o3);
        return ll;
    }
};

// ---------------------------------------------------------------- two-filter (reverse)

// Alg. ptf: reversed scan of (a_2, ..., a_T, e) under Lemma 1, carry
// (eta, J), fused with the two-filter merge (Eqs. mean_tf_combination /
// cov_tf_combination).  Position p holds a_{k+1} of record g + 1 for the
// time k = g + 1 of global index g = T - 1 - p, or e at k = T.
template <int N, typename Rt, int MODE>
struct TfTv {
    static constexpr int KIND = 2, NX = N;
    static constexpr bool REV = true;
    using R = Rt;
    using T = typename std::conditional<MODE == 1, double, R>::type;
    using Elem = FElem<N, R>;
    using Carry = RevCarry<N, R>;
    static constexpr int S = N * (N + 1) / 2;
    static constexpr int IN_REC = FRec<N, R>::SIZE, O1 = N, O2 = N * N, O3 = 0;
    struct Args {
        TvSeq<N, R> src;
        KfBufs<R> buf;
        int want_ll;
        NoTab tab;
    };
    KF_TV_NO_TABLE
    static KF_HD int64_t total(const Args &a) { return a.src.T; }
    static KF_HD const R *in_arr(const Args &a) { return a.buf.frec; }
    static KF_HD R *out_arr(const Args &a, int i) { return i == 0 ? a.buf.ms : i == 1 ? a.buf.Ps : nullptr; }
    static KF_D SegCursor cursor(const Args &a, int64_t) { return SegCursor{0, 0, a.src.T}; }
    static KF_D void build(const Args &a, int64_t p, SegCursor &, const R *, Elem &e) {
        const int64_t g = a.src.T - 1 - p;
        if (g == a.src.T - 1) {
            set_zero(e);
            return;
        }
        op_tv_filter_elem<N, R, T>(a.src, g + 1, a.buf.y + (g + 1) * a.src.ny, e);
    }
    static KF_D void combine(const Elem &x, const Elem &y, Elem &o) { op_lemma1<N, R, MODE>(y, x, o); }
    static KF_D void fold(const Args &, const SegCursor &, const Elem &x, const Elem &y, Elem &o) { combine(x, y, o); }
    static KF_D void apply(Carry &c, const Elem &e) { op_apply_rev<N, R, MODE>(c, e); }
    // the transition block exactly zero: the element's half is what it makes of any carry
    static KF_D bool zero_transition(const Elem &e) {
        bool z = true;
#pragma unroll
        for (int i = 0; i < N * N; ++i) z = z && e.v[Elem::oA + i] == R(0);
        return z;
    }
    static KF_D void carry_of(const Elem &e, Carry &c) {
#pragma unroll
        for (int i = 0; i < N; ++i) c.v[Carry::oe + i] = e.v[Elem::oe + i];
#pragma unroll
        for (int i = 0; i < S; ++i) c.v[Carry::oJ + i] = e.v[Elem::oJ + i];
    }
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
        return R(step(a, p, cur, c, e, in, o1, o2, o3));
    }
    static KF_D double step(const Args &a, int64_t p, SegCursor &cur, Carry &c, const Elem &e, const R *in, R *o1,
                            R *o2, R *o3) {
        apply(c, e);
        emit(a, p, cur, c, in, o1, o2, o3);
        return 0.0;
    }
};

// ---------------------------------------------------------------- RTS (reverse)

// Alg. prts: reversed scan of (E, g, L) under Lemma 2, carry (g, L),
// extraction xbar_{k|T} = g_k^+, P_{k|T} = L_k^+.
template <int N, typename Rt>
struct RtsTv {
    static constexpr int KIND = 1, NX = N;
    static constexpr bool REV = true;
    using R = Rt;
    using Elem = RElem<N, R>;
    using Carry = RCarry<N, R>;
    static constexpr int S = N * (N + 1) / 2;
    static constexpr int IN_REC = FRec<N, R>::SIZE, O1 = N, O2 = N * N, O3 = 0;
    struct Args {
        TvSeq<N, R> src;
        KfBufs<R> buf;
        int want_ll;
        NoTab tab;
    };
    KF_TV_NO_TABLE
    static KF_HD int64_t total(const Args &a) { return a.src.T; }
    static KF_HD const R *in_arr(const Args &a) { return a.buf.frec; }
    static KF_HD R *out_arr(const Args &a, int i) { return i == 0 ? a.buf.ms : i == 1 ? a.buf.Ps : nullptr; }
    static KF_D SegCursor cursor(const Args &a, int64_t) { return SegCursor{0, 0, a.src.T}; }
    static KF_D void build(const Args &a, int64_t p, SegCursor &, const R *in, Elem &e) {
        const int64_t g = a.src.T - 1 - p;
        R rec[IN_REC];
        load_rec<IN_REC>(rec, in);
        op_tv_rts_elem<N, R>(a.src, g, rec, rec + N, e);
    }
    static KF_D void combine(const Elem &x, const Elem &y, Elem &o) { op_lemma2<N, R>(y, x, o); }
    static KF_D void fold(const Args &, const SegCursor &, const Elem &x, const Elem &y, Elem &o) { combine(x, y, o); }
    static KF_D void apply(Carry &c, const Elem &e) { op_apply_rts<N, R>(c, e); }
    // the transition block exactly zero: the element's half is what it makes of any carry
    static KF_D bool zero_transition(const Elem &e) {
        bool z = true;
#pragma unroll
        for (int i = 0; i < N * N; ++i) z = z && e.v[Elem::oE + i] == R(0);
        return z;
    }
    static KF_D void carry_of(const Elem &e, Carry &c) {
#pragma unroll
        for (int i = 0; i < N; ++i) c.v[Carry::og + i] = e.v[Elem::og + i];
#pragma unroll
        for (int i = 0; i < S; ++i) c.v[Carry::oL + i] = e.v[Elem::oL + i];
    }
    static KF_D void emit(const Args &, int64_t, SegCursor &, const Carry &c, const R *, R *o1, R *o2, R *) {
        R full[N * N];
        store_rec<N>(o1, c.v + Carry::og);
        store_full<N>(full, c.v + Carry::oL);
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
        return R(step(a, p, cur, c, e, in, o1, o2, o3));
    }
    static KF_D double step(const Args &a, int64_t p, SegCursor &cur, Carry &c, const Elem &e, const R *in, R *o1,
                            R *o2, R *o3) {
        apply(c, e);
        emit(a, p, cur, c, in, o1, o2, o3);
        return 0.0;
    }
};

#undef KF_TV_NO_TABLE

// ---------------------------------------------------------------- launch

// Filter pass, then the RTS or two-filter pass, each one decoupled look-back
// scan kernel.
template <int N, typename R, int MODE, int THREADS>
static cudaError_t launch_tv_typed(const TvLaunch &t) {
    constexpr int V = (1024 + THREADS - 1) / THREADS;
    const LaunchReq &q = t.q;
    const WsLayout L = ws_layout<N, R>(q.op, KF_SCAN_DLB_I, q.T);
    char *ws = static_cast<char *>(q.ws);
    KfBufs<R> buf;
    buf.y = static_cast<const R *>(q.y);
    buf.ms = static_cast<R *>(q.ms);
    buf.Ps = static_cast<R *>(q.Ps);
    buf.frec = (q.op == KF_OP_FILTER_I) ? nullptr : reinterpret_cast<R *>(ws + L.frec);
    buf.mf_user = static_cast<R *>(q.mf_user);
    buf.Pf_user = static_cast<R *>(q.Pf_user);
    TvSeq<N, R> src;
    src.F = static_cast<const R *>(t.F);
    src.Q = static_cast<const R *>(t.Q);
    src.u = static_cast<const R *>(t.u);
    src.H = static_cast<const R *>(t.H);
    src.Rm = static_cast<const R *>(t.R);
    src.d = static_cast<const R *>(t.d);
    src.ny = t.ny;
    src.T = q.T;
    for (int i = 0; i < N; ++i) src.m0[i] = t.m0[i];
    for (int i = 0; i < N * N; ++i) src.P0[i] = t.P0[i];
    LaunchReq qz = q;
    qz.scan = KF_SCAN_DLB_I;
    if (q.op != KF_OP_FILTER_I) {   // one memset clears both passes' look-back counters
        const cudaError_t ez = cudaMemsetAsync(ws + L.ctl_f, 0, L.agg - L.ctl_f, q.stream);
        if (ez != cudaSuccess) return ez;
        qz.counters_zeroed = 1;
    }
    using PF = FilterTv<N, R, MODE>;
    typename PF::Args fa;
    fa.src = src;
    fa.buf = buf;
    fa.want_ll = q.loglik != nullptr;
    fa.tab.K = 0;
    cudaError_t e = run_dlb<PF, THREADS, V>(fa, ws, L.ctl_f, L, qz, q.loglik);
    if (e != cudaSuccess || q.op == KF_OP_FILTER_I) return e;
    if (q.op == KF_OP_RTS_I) {
        using PR = RtsTv<N, R>;
        typename PR::Args ra;
        ra.src = src;
        ra.buf = buf;
        ra.want_ll = 0;
        ra.tab.K = 0;
        return run_dlb<PR, THREADS, V>(ra, ws, L.ctl_r, L, qz, nullptr);
    }
    using PT = TfTv<N, R, MODE>;
    typename PT::Args ta;
    ta.src = src;
    ta.buf = buf;
    ta.want_ll = 0;
    ta.tab.K = 0;
    return run_dlb<PT, THREADS, V>(ta, ws, L.ctl_r, L, qz, nullptr);
}

template <int N>
static cudaError_t launch_tv_n(const TvLaunch &t) {
    switch (t.q.prec) {
        case KF_FP64_I: return launch_tv_typed<N, double, 0, 128>(t);
        case KF_FP32_I: return launch_tv_typed<N, float, 0, 128>(t);
        case KF_FP32_FP64SOLVE_I: return launch_tv_typed<N, float, 1, 128>(t);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace kfs
