// kf_steps.cuh -- the per-time-step arithmetic of the one-sequence kernels
// (ti_filter.cuh, rts_scan.cuh), as functions of the working type R.  The
// kernels call these; flop_count.cpp instantiates the same functions on the
// host with a counting type, so the flops per step reported for the
// roofline are counted from this code (an FMA counts 2, a reciprocal,
// square root or log 1).
#pragma once

#include "kf_math.cuh"

namespace kfs {

// ---------------------------------------------------------------- forward filter (Alg. pkf)

// One step of the table-driven thread fold of a time-invariant model (the
// c-th fresh element, c >= 1, of a run), Lemma 1 with the fresh element on
// the right reduced to the affine updates of the fold table row
// (T1 | T4 | T3U):
//   v = L^{-1} y - U b,  b <- T1 b + T4 y,  eta <- eta + T3U v.
template <int N, int M, typename R>
KF_D void ti_fold_step(const FiltParams<N, R> &P, const R *row, const R *y, R *b, R *e) {
    const R *T1 = row, *T4 = row + N * N, *T3U = row + N * N + N * M;
    R v[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        R s = 0;
#pragma unroll
        for (int k = 0; k <= i; ++k) s += P.Linv[i * MAXNY + k] * y[k];
#pragma unroll
        for (int k = 0; k < N; ++k) s -= P.U[i * N + k] * b[k];
        v[i] = s;
    }
    R nb[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = 0;
#pragma unroll
        for (int j = 0; j < M; ++j) s += T4[r * M + j] * y[j];
#pragma unroll
        for (int k = 0; k < N; ++k) s += T1[r * N + k] * b[k];
        nb[r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = e[r];
#pragma unroll
        for (int i = 0; i < M; ++i) s += T3U[r * M + i] * v[i];
        e[r] = s;
        b[r] = nb[r];
    }
}

// One step of the carry pass: the carry (b, C) = (xbar_{k-1|k-1},
// P_{k-1|k-1}) extended by the fresh element a_k (b_k = K y_k, eta_k = G y_k)
// with the rank-ny form of Lemma 1.  With LL, returns the innovation term
// -1/2 (v^T S_k^{-1} v + log det S_k + ny log 2 pi) of log p(y_k | y_{1:k-1}).
template <int N, int M, typename R, bool LL>
KF_D R ti_carry_step(const FiltParams<N, R> &P, const R *y, FwdCarry<N, R> &c) {
    R bk[N], ek[N];
    fresh_b_eta<N, M, R>(P, y, bk, ek);
    if constexpr (LL) {
        R yt[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            R s = 0;
#pragma unroll
            for (int k = 0; k <= i; ++k) s += P.Linv[i * MAXNY + k] * y[k];
            yt[i] = s;
        }
        R q, ld;
        apply_fwd_lr_parts<N, M, R, 0, true>(c, P.A, bk, P.C, ek, P.U, yt, &q, &ld);
        return R(-0.5) * (q + ld + P.llc_r);
    } else {
        apply_fwd_lr_parts<N, M, R, 0, false>(c, P.A, bk, P.C, ek, P.U, nullptr, nullptr, nullptr);
        return R(0);
    }
}

// ---------------------------------------------------------------- RTS smoother (Alg. prts)

// Pieces of the RTS element of time k (Eq. prts_init1) from the filter
// record (xbar, packed P): E = P F^T P_{k+1|k}^{-1}, F xbar and
// P_{k+1|k} = F P F^T + Q (packed).  last (k = T, Eq. prts_init2): E = 0.
template <int N, typename R>
KF_D void rs_build(const R *F, const R *Q, bool last, const R *x, const R *P, R *E, R *Fx, R *Pp) {
    if (last) {
#pragma unroll
        for (int i = 0; i < N * N; ++i) E[i] = 0;
#pragma unroll
        for (int i = 0; i < N; ++i) Fx[i] = 0;
#pragma unroll
        for (int i = 0; i < N * (N + 1) / 2; ++i) Pp[i] = 0;
        return;
    }
    R U[N * N];   // F P
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += F[r * N + k] * P[si(N, k, c)];
            U[r * N + c] = s;
        }
    R Lc[N * (N + 1) / 2], dinv[N];   // P_{k+1|k} = U F^T + Q, its Cholesky factor
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            R s = Q[su(N, j, i)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += U[i * N + k] * F[j * N + k];
            Pp[su(N, j, i)] = s;
#pragma unroll
            for (int k = 0; k < j; ++k) s -= Lc[i * (i + 1) / 2 + k] * Lc[j * (j + 1) / 2 + k];
            if (i == j) {
                const R d = ksqrt(s);
                Lc[i * (i + 1) / 2 + i] = d;
                dinv[i] = recip(d);
            } else {
                Lc[i * (i + 1) / 2 + j] = s * dinv[j];
            }
        }
    // E^T = P_{k+1|k}^{-1} U, column by column (forward, then backward substitution)
#pragma unroll
    for (int c = 0; c < N; ++c) {
        R z[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            R s = U[i * N + c];
#pragma unroll
            for (int k = 0; k < i; ++k) s -= Lc[i * (i + 1) / 2 + k] * z[k];
            z[i] = s * dinv[i];
        }
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
            R s = z[i];
#pragma unroll
            for (int k = i + 1; k < N; ++k) s -= Lc[k * (k + 1) / 2 + i] * E[c * N + k];
            E[c * N + i] = s * dinv[i];   // E[c][i] = (E^T)[i][c]
        }
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) s += F[r * N + k] * x[k];
        Fx[r] = s;
    }
}

// Lemma 2 with the element of time k on the left of the later part (g, L),
// in direct form: (g, L) <- (xbar + E (g - F xbar), P + E (L - P_{k+1|k}) E^T),
// which equals (g_k + E g, L_k + E L E^T) without forming g_k, L_k.
template <int N, typename R>
KF_D void rs_direct(const R *E, const R *Fx, const R *Pp, const R *x, const R *P, R *g, R *L) {
    constexpr int S = N * (N + 1) / 2;
    R d[N], D[S];
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = g[i] - Fx[i];
#pragma unroll
    for (int i = 0; i < S; ++i) D[i] = L[i] - Pp[i];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = x[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += E[r * N + k] * d[k];
        g[r] = s;
    }
    R ED[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += E[r * N + k] * D[si(N, k, c)];
            ED[r * N + c] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            R s = P[su(N, r, c)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += ED[r * N + k] * E[c * N + k];
            L[su(N, r, c)] = s;
        }
}

// One step of the RTS thread fold: the aggregate (Ea, g, L) of the later
// elements of the run extended by the element of time k on its left:
// Ea <- E_k Ea, then (g, L) in the direct form.
template <int N, typename R>
KF_D void rs_fold_step(const R *F, const R *Q, bool last, const R *rec, R *Ea, R *g, R *L) {
    R E[N * N], Fx[N], Pp[N * (N + 1) / 2];
    rs_build<N, R>(F, Q, last, rec, rec + N, E, Fx, Pp);
    R nE[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += E[r * N + k] * Ea[k * N + c];
            nE[r * N + c] = s;
        }
    rs_direct<N, R>(E, Fx, Pp, rec, rec + N, g, L);
#pragma unroll
    for (int i = 0; i < N * N; ++i) Ea[i] = nE[i];
}

// One step of the RTS carry pass: the smoothed moments of time k from those
// of time k + 1 (the carry) and the filter record of time k.
template <int N, typename R>
KF_D void rs_carry_step(const R *F, const R *Q, bool last, const R *rec, R *g, R *L) {
    R E[N * N], Fx[N], Pp[N * (N + 1) / 2];
    rs_build<N, R>(F, Q, last, rec, rec + N, E, Fx, Pp);
    rs_direct<N, R>(E, Fx, Pp, rec, rec + N, g, L);
}

}  // namespace kfs
