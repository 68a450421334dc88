/*
 * kf_oracle.c -- plain, sequential, FP64 reference implementation of the
 * Kalman filter, the Rauch-Tung-Striebel smoother, the two-filter smoother
 * and the parallel-form elements / associative operators of
 * Sarkka & Garcia-Fernandez, "On the Performance of Prefix-Sum Parallel
 * Kalman Filters and Smoothers on GPUs" (arXiv 2511.10363).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the GPU library is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header, table or helper with the
 * CUDA path, and it is written for obviousness, not speed: every loop is the
 * textbook definition, every solve a partially pivoted LU (or a Cholesky for
 * a symmetric positive-definite matrix), no blocking, no fusion.
 *
 * Model (Sec. III-A, Eqs. transition/measurement densities), time-invariant,
 * with u = d = 0:
 *     x_k = F x_{k-1} + q_{k-1},   q ~ N(0, Q)
 *     y_k = H x_k + r_k,           r ~ N(0, R)
 *     x_0 ~ N(m0, P0)              (m0 = xbar_{0|0}, P0 = P_{0|0})
 * All matrices are row-major doubles; nx = n, ny = m; y is [T][m].
 * Outputs are for k = 1..T, stored at index k-1.
 *
 * Parity status: every function here is pinned by the CPU test-suite against
 * closed forms, a dense joint-Gaussian brute force, special cases and
 * algebraic identities (see tests/test_oracle_pins.py); none is unpinned.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 16

/* ------------------------------------------------------------------ */
/* tiny dense linear algebra (row-major, n x n unless stated)          */
/* ------------------------------------------------------------------ */

/* C[r x c] = A[r x k] * B[k x c] */
static void mm(int r, int k, int c, const double *A, const double *B, double *C) {
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) {
            double s = 0.0;
            for (int t = 0; t < k; ++t) s += A[i * k + t] * B[t * c + j];
            C[i * c + j] = s;
        }
}

/* B[c x r] = A[r x c]^T */
static void tr(int r, int c, const double *A, double *B) {
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) B[j * r + i] = A[i * c + j];
}

static void add(int len, const double *A, const double *B, double *C) {
    for (int i = 0; i < len; ++i) C[i] = A[i] + B[i];
}

static void sub(int len, const double *A, const double *B, double *C) {
    for (int i = 0; i < len; ++i) C[i] = A[i] - B[i];
}

static void eye(int n, double *A) {
    memset(A, 0, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i) A[i * n + i] = 1.0;
}

/* Solve A X = B for X (A: n x n, B: n x c) by Gaussian elimination with
 * partial pivoting.  A and B are not modified.  Returns 0 on success, -1 if
 * a pivot is exactly zero. */
static int lu_solve(int n, int c, const double *A, const double *B, double *X) {
    double a[ORC_MAXN * ORC_MAXN], b[ORC_MAXN * ORC_MAXN * 2];
    memcpy(a, A, sizeof(double) * n * n);
    memcpy(b, B, sizeof(double) * n * c);
    for (int col = 0; col < n; ++col) {
        int p = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r * n + col]) > fabs(a[p * n + col])) p = r;
        if (a[p * n + col] == 0.0) return -1;
        if (p != col) {
            for (int j = 0; j < n; ++j) { double t = a[col * n + j]; a[col * n + j] = a[p * n + j]; a[p * n + j] = t; }
            for (int j = 0; j < c; ++j) { double t = b[col * c + j]; b[col * c + j] = b[p * c + j]; b[p * c + j] = t; }
        }
        for (int r = col + 1; r < n; ++r) {
            double f = a[r * n + col] / a[col * n + col];
            for (int j = col; j < n; ++j) a[r * n + j] -= f * a[col * n + j];
            for (int j = 0; j < c; ++j) b[r * c + j] -= f * b[col * c + j];
        }
    }
    for (int r = n - 1; r >= 0; --r)
        for (int j = 0; j < c; ++j) {
            double s = b[r * c + j];
            for (int t = r + 1; t < n; ++t) s -= a[r * n + t] * X[t * c + j];
            X[r * c + j] = s / a[r * n + r];
        }
    return 0;
}

/* Inverse via lu_solve with the identity as right-hand side. */
static int inv(int n, const double *A, double *Ai) {
    double I[ORC_MAXN * ORC_MAXN];
    eye(n, I);
    return lu_solve(n, n, A, I, Ai);
}

/* Cholesky A = L L^T of a symmetric positive-definite matrix; returns -1 if
 * A is not positive definite. */
static int chol(int n, const double *A, double *L) {
    memset(L, 0, sizeof(double) * n * n);
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int t = 0; t < j; ++t) s -= L[j * n + t] * L[j * n + t];
        if (!(s > 0.0)) return -1;
        L[j * n + j] = sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double u = A[i * n + j];
            for (int t = 0; t < j; ++t) u -= L[i * n + t] * L[j * n + t];
            L[i * n + j] = u / L[j * n + j];
        }
    }
    return 0;
}

/* Solve A X = B with A symmetric positive definite through its Cholesky
 * factor; also returns log det A. */
static int chol_solve(int n, int c, const double *A, const double *B, double *X, double *logdet) {
    double L[ORC_MAXN * ORC_MAXN], Z[ORC_MAXN * ORC_MAXN * 2];
    if (chol(n, A, L)) return -1;
    for (int j = 0; j < c; ++j) {
        for (int i = 0; i < n; ++i) {            /* L z = b */
            double s = B[i * c + j];
            for (int t = 0; t < i; ++t) s -= L[i * n + t] * Z[t * c + j];
            Z[i * c + j] = s / L[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {       /* L^T x = z */
            double s = Z[i * c + j];
            for (int t = i + 1; t < n; ++t) s -= L[t * n + i] * X[t * c + j];
            X[i * c + j] = s / L[i * n + i];
        }
    }
    if (logdet) {
        double ld = 0.0;
        for (int i = 0; i < n; ++i) ld += 2.0 * log(L[i * n + i]);
        *logdet = ld;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sequential Kalman filter, Sec. III-A (Eqs. KF_mean_pred .. KF_cov_upd) */
/* ------------------------------------------------------------------ */
/* m_out: [T][n], P_out: [T][n][n] (filtering xbar_{k|k}, P_{k|k});
 * mp_out, Pp_out (nullable): predicted xbar_{k|k-1}, P_{k|k-1};
 * loglik (nullable): log p(y_{1:T}) in innovation form,
 *   sum_k -1/2 (v_k^T S_k^{-1} v_k + log det S_k + m log 2 pi),
 *   v_k = y_k - H xbar_{k|k-1}.
 * Returns 0, or -1 if some S_k is not positive definite. */
int orc_kf(int n, int m, const double *F, const double *Q, const double *H, const double *R,
           const double *m0, const double *P0, long T, const double *y,
           double *m_out, double *P_out, double *mp_out, double *Pp_out, double *loglik) {
    double x[ORC_MAXN], P[ORC_MAXN * ORC_MAXN];
    double xp[ORC_MAXN], Pp[ORC_MAXN * ORC_MAXN], t1[ORC_MAXN * ORC_MAXN], t2[ORC_MAXN * ORC_MAXN];
    double Ft[ORC_MAXN * ORC_MAXN], Ht[ORC_MAXN * ORC_MAXN], S[ORC_MAXN * ORC_MAXN];
    double PHt[ORC_MAXN * ORC_MAXN], KT[ORC_MAXN * ORC_MAXN], v[ORC_MAXN], Siv[ORC_MAXN];
    double ll = 0.0;
    const double LOG2PI = 1.8378770664093454835606594728112;
    memcpy(x, m0, sizeof(double) * n);
    memcpy(P, P0, sizeof(double) * n * n);
    tr(n, n, F, Ft);
    tr(m, n, H, Ht);
    for (long k = 0; k < T; ++k) {
        /* prediction: xbar_{k|k-1} = F xbar, P_{k|k-1} = F P F^T + Q */
        mm(n, n, 1, F, x, xp);
        mm(n, n, n, F, P, t1);
        mm(n, n, n, t1, Ft, t2);
        add(n * n, t2, Q, Pp);
        if (mp_out) memcpy(mp_out + k * n, xp, sizeof(double) * n);
        if (Pp_out) memcpy(Pp_out + k * n * n, Pp, sizeof(double) * n * n);
        /* update: S = H P_{k|k-1} H^T + R */
        mm(n, n, m, Pp, Ht, PHt);            /* P_{k|k-1} H^T : n x m */
        mm(m, n, m, H, PHt, t1);
        add(m * m, t1, R, S);
        /* innovation v = y_k - H xbar_{k|k-1} */
        mm(m, n, 1, H, xp, t1);
        sub(m, y + k * m, t1, v);
        /* K^T = S^{-1} (P_{k|k-1} H^T)^T  (S symmetric) */
        tr(n, m, PHt, t1);                   /* m x n */
        double logdetS;
        if (chol_solve(m, n, S, t1, KT, &logdetS)) return -1;
        /* xbar_{k|k} = xbar_{k|k-1} + P H^T S^{-1} v */
        if (chol_solve(m, 1, S, v, Siv, NULL)) return -1;
        mm(n, m, 1, PHt, Siv, t2);
        add(n, xp, t2, x);
        /* P_{k|k} = P_{k|k-1} - P H^T S^{-1} H P */
        mm(n, m, n, PHt, KT, t2);
        sub(n * n, Pp, t2, P);
        memcpy(m_out + k * n, x, sizeof(double) * n);
        memcpy(P_out + k * n * n, P, sizeof(double) * n * n);
        double q = 0.0;
        for (int i = 0; i < m; ++i) q += v[i] * Siv[i];
        ll += -0.5 * (q + logdetS + m * LOG2PI);
    }
    if (loglik) *loglik = ll;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sequential RTS smoother, Sec. III-B (forward-backward smoother)     */
/* ------------------------------------------------------------------ */
/* Input: filtering results mf [T][n], Pf [T][n][n].  Output: ms, Ps.
 * G_k = P_{k|k} F^T P_{k+1|k}^{-1};
 * xbar_{k|T} = xbar_{k|k} + G_k (xbar_{k+1|T} - xbar_{k+1|k});
 * P_{k|T} = P_{k|k} + G_k (P_{k+1|T} - P_{k+1|k}) G_k^T. */
int orc_rts(int n, const double *F, const double *Q, long T, const double *mf, const double *Pf,
            double *ms, double *Ps) {
    double Ft[ORC_MAXN * ORC_MAXN], Pp[ORC_MAXN * ORC_MAXN], xp[ORC_MAXN];
    double t1[ORC_MAXN * ORC_MAXN], t2[ORC_MAXN * ORC_MAXN], G[ORC_MAXN * ORC_MAXN], Gt[ORC_MAXN * ORC_MAXN];
    double dx[ORC_MAXN], dP[ORC_MAXN * ORC_MAXN];
    tr(n, n, F, Ft);
    memcpy(ms + (T - 1) * n, mf + (T - 1) * n, sizeof(double) * n);
    memcpy(Ps + (T - 1) * n * n, Pf + (T - 1) * n * n, sizeof(double) * n * n);
    for (long k = T - 2; k >= 0; --k) {
        const double *x = mf + k * n, *P = Pf + k * n * n;
        mm(n, n, 1, F, x, xp);                       /* xbar_{k+1|k} */
        mm(n, n, n, F, P, t1);
        mm(n, n, n, t1, Ft, t2);
        add(n * n, t2, Q, Pp);                       /* P_{k+1|k} */
        /* G^T = P_{k+1|k}^{-1} (P F^T)^T = P_{k+1|k}^{-1} F P */
        mm(n, n, n, F, P, t1);
        if (lu_solve(n, n, Pp, t1, Gt)) return -1;
        tr(n, n, Gt, G);
        sub(n, ms + (k + 1) * n, xp, dx);
        mm(n, n, 1, G, dx, t1);
        add(n, x, t1, ms + k * n);
        sub(n * n, Ps + (k + 1) * n * n, Pp, dP);
        mm(n, n, n, G, dP, t1);
        mm(n, n, n, t1, Gt, t2);
        add(n * n, P, t2, Ps + k * n * n);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sequential two-filter smoother, Sec. III-B (Eqs. tf_vector_pred ..  */
/* tf_matrix_upd for the backward information filter, Eqs.            */
/* mean_tf_combination / cov_tf_combination for the merge)            */
/* ------------------------------------------------------------------ */
/* eta_out [T][n], J_out [T][n][n] (nullable) receive eta_{k|k+1:T}, J_{k|k+1:T};
 * at k = T both are zero (no future measurements). */
int orc_tf(int n, int m, const double *F, const double *Q, const double *H, const double *R, long T,
           const double *y, const double *mf, const double *Pf, double *ms, double *Ps,
           double *eta_out, double *J_out) {
    double Ft[ORC_MAXN * ORC_MAXN], Ht[ORC_MAXN * ORC_MAXN], Ri[ORC_MAXN * ORC_MAXN];
    double HtRi[ORC_MAXN * ORC_MAXN], HtRiH[ORC_MAXN * ORC_MAXN];
    double eta[ORC_MAXN], J[ORC_MAXN * ORC_MAXN], t1[ORC_MAXN * ORC_MAXN], t2[ORC_MAXN * ORC_MAXN];
    double Mx[ORC_MAXN * ORC_MAXN], I[ORC_MAXN * ORC_MAXN], rhs[ORC_MAXN * (ORC_MAXN + 1)];
    double sol[ORC_MAXN * (ORC_MAXN + 1)];
    tr(n, n, F, Ft);
    tr(m, n, H, Ht);
    if (inv(m, R, Ri)) return -1;
    mm(n, m, m, Ht, Ri, HtRi);
    mm(n, m, n, HtRi, H, HtRiH);
    eye(n, I);
    memset(eta, 0, sizeof(double) * n);          /* eta_{T|T+1:T} = 0 */
    memset(J, 0, sizeof(double) * n * n);        /* J_{T|T+1:T}   = 0 */
    for (long k = T - 1; k >= 0; --k) {          /* k is time step k+1 */
        const double *x = mf + k * n, *P = Pf + k * n * n;
        if (eta_out) memcpy(eta_out + k * n, eta, sizeof(double) * n);
        if (J_out) memcpy(J_out + k * n * n, J, sizeof(double) * n * n);
        /* merge: xbar_{k|T} = (I + P J)^{-1}(xbar + P eta), P_{k|T} = (I + P J)^{-1} P */
        mm(n, n, n, P, J, t1);
        add(n * n, I, t1, Mx);
        mm(n, n, 1, P, eta, t2);
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) rhs[i * (n + 1) + j] = P[i * n + j];
            rhs[i * (n + 1) + n] = x[i] + t2[i];
        }
        if (lu_solve(n, n + 1, Mx, rhs, sol)) return -1;
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) Ps[k * n * n + i * n + j] = sol[i * (n + 1) + j];
            ms[k * n + i] = sol[i * (n + 1) + n];
        }
        if (k == 0) break;
        /* update with y_{k}: eta += H^T R^{-1} y, J += H^T R^{-1} H */
        mm(n, m, 1, HtRi, y + k * m, t1);
        add(n, eta, t1, eta);
        add(n * n, J, HtRiH, J);
        /* backward prediction: eta <- F^T (I + J Q)^{-1} eta,
         *                      J   <- F^T (I + J Q)^{-1} J F */
        mm(n, n, n, J, Q, t1);
        add(n * n, I, t1, Mx);
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) rhs[i * (n + 1) + j] = J[i * n + j];
            rhs[i * (n + 1) + n] = eta[i];
        }
        if (lu_solve(n, n + 1, Mx, rhs, sol)) return -1;
        double JF[ORC_MAXN * ORC_MAXN], v[ORC_MAXN], MiJ[ORC_MAXN * ORC_MAXN];
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) MiJ[i * n + j] = sol[i * (n + 1) + j];
            v[i] = sol[i * (n + 1) + n];
        }
        mm(n, n, 1, Ft, v, eta);
        mm(n, n, n, MiJ, F, JF);
        mm(n, n, n, Ft, JF, J);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Parallel-form elements and operators (Sec. IV-C, IV-D)             */
/* ------------------------------------------------------------------ */
/* Filtering element layout used by the oracle: [A (n*n), b (n), C (n*n),
 * eta (n), J (n*n)], total 3n^2 + 2n doubles. */
int orc_filter_elem_size(int n) { return 3 * n * n + 2 * n; }

/* Element a_k of Eqs. pkf_init1 (k > 1), pkf_init2 (k = 1) and pkf_init3.
 * k is 1-based.  For eta_1, J_1 Eq. pkf_init3 is applied with the S_k of
 * Eq. pkf_init1 (S = H Q H^T + R) for every k, including k = 1; eta_1, J_1
 * never reach an output because A_1 = 0. */
int orc_filter_element(int n, int m, const double *F, const double *Q, const double *H, const double *R,
                       const double *m0, const double *P0, long k, const double *yk, double *e) {
    double *A = e, *b = e + n * n, *C = e + n * n + n, *eta = e + 2 * n * n + n, *J = e + 2 * n * n + 2 * n;
    double Ht[ORC_MAXN * ORC_MAXN], Ft[ORC_MAXN * ORC_MAXN], t1[ORC_MAXN * ORC_MAXN], t2[ORC_MAXN * ORC_MAXN];
    double S[ORC_MAXN * ORC_MAXN], KT[ORC_MAXN * ORC_MAXN], K[ORC_MAXN * ORC_MAXN], IKH[ORC_MAXN * ORC_MAXN];
    double v[ORC_MAXN];
    tr(m, n, H, Ht);
    tr(n, n, F, Ft);
    if (k == 1) {
        double xp[ORC_MAXN], Pp[ORC_MAXN * ORC_MAXN], PHt[ORC_MAXN * ORC_MAXN];
        mm(n, n, 1, F, m0, xp);                  /* xbar_{1|0} = F xbar_{0|0} */
        mm(n, n, n, F, P0, t1);
        mm(n, n, n, t1, Ft, t2);
        add(n * n, t2, Q, Pp);                   /* P_{1|0} = F P_{0|0} F^T + Q */
        mm(n, n, m, Pp, Ht, PHt);
        mm(m, n, m, H, PHt, t1);
        add(m * m, t1, R, S);                    /* S_1 = H P_{1|0} H^T + R */
        tr(n, m, PHt, t1);
        if (chol_solve(m, n, S, t1, KT, NULL)) return -1;
        tr(m, n, KT, K);                         /* K_1 = P_{1|0} H^T S_1^{-1} */
        memset(A, 0, sizeof(double) * n * n);    /* A_1 = 0 */
        mm(m, n, 1, H, xp, t1);
        sub(m, yk, t1, v);
        mm(n, m, 1, K, v, t1);
        add(n, xp, t1, b);                       /* b_1 = xbar_{1|0} + K_1 (y_1 - H xbar_{1|0}) */
        double KS[ORC_MAXN * ORC_MAXN];
        mm(n, m, m, K, S, KS);
        mm(n, m, n, KS, KT, t1);
        sub(n * n, Pp, t1, C);                   /* C_1 = P_{1|0} - K_1 S_1 K_1^T */
    } else {
        double QHt[ORC_MAXN * ORC_MAXN];
        mm(n, n, m, Q, Ht, QHt);
        mm(m, n, m, H, QHt, t1);
        add(m * m, t1, R, S);                    /* S_k = H Q H^T + R */
        tr(n, m, QHt, t1);
        if (chol_solve(m, n, S, t1, KT, NULL)) return -1;
        tr(m, n, KT, K);                         /* K_k = Q H^T S_k^{-1} */
        mm(n, m, n, K, H, t1);
        eye(n, t2);
        sub(n * n, t2, t1, IKH);                 /* I - K_k H */
        mm(n, n, n, IKH, F, A);                  /* A_k = (I - K H) F */
        mm(n, m, 1, K, yk, b);                   /* b_k = K_k y_k */
        mm(n, n, n, IKH, Q, C);                  /* C_k = (I - K H) Q */
    }
    /* Eq. pkf_init3 with S = H Q H^T + R:
     * eta_k = F^T H^T S^{-1} y_k,  J_k = F^T H^T S^{-1} H F */
    {
        double QHt[ORC_MAXN * ORC_MAXN], Sx[ORC_MAXN * ORC_MAXN], SiH[ORC_MAXN * ORC_MAXN], Siy[ORC_MAXN];
        double HF[ORC_MAXN * ORC_MAXN], FtHt[ORC_MAXN * ORC_MAXN];
        mm(n, n, m, Q, Ht, QHt);
        mm(m, n, m, H, QHt, t1);
        add(m * m, t1, R, Sx);
        if (chol_solve(m, 1, Sx, yk, Siy, NULL)) return -1;
        mm(m, n, n, H, F, HF);
        if (chol_solve(m, n, Sx, HF, SiH, NULL)) return -1;   /* S^{-1} H F */
        tr(m, n, HF, FtHt);                                    /* F^T H^T */
        mm(n, m, 1, FtHt, Siy, eta);
        mm(n, m, n, FtHt, SiH, J);
    }
    return 0;
}

/* Lemma 1: (A_i,b_i,C_i,eta_i,J_i) (x) (A_j,b_j,C_j,eta_j,J_j). */
int orc_filter_combine(int n, const double *ei, const double *ej, double *out) {
    const double *Ai = ei, *bi = ei + n * n, *Ci = ei + n * n + n, *etai = ei + 2 * n * n + n, *Ji = ei + 2 * n * n + 2 * n;
    const double *Aj = ej, *bj = ej + n * n, *Cj = ej + n * n + n, *etaj = ej + 2 * n * n + n, *Jj = ej + 2 * n * n + 2 * n;
    double *A = out, *b = out + n * n, *C = out + n * n + n, *eta = out + 2 * n * n + n, *J = out + 2 * n * n + 2 * n;
    double I[ORC_MAXN * ORC_MAXN], t1[ORC_MAXN * ORC_MAXN], t2[ORC_MAXN * ORC_MAXN], t3[ORC_MAXN * ORC_MAXN];
    double M1[ORC_MAXN * ORC_MAXN], M1i[ORC_MAXN * ORC_MAXN], M2[ORC_MAXN * ORC_MAXN], M2i[ORC_MAXN * ORC_MAXN];
    double AjM1i[ORC_MAXN * ORC_MAXN], AiT[ORC_MAXN * ORC_MAXN], AjT[ORC_MAXN * ORC_MAXN], AiTM2i[ORC_MAXN * ORC_MAXN];
    double v[ORC_MAXN], w[ORC_MAXN];
    double rA[ORC_MAXN * ORC_MAXN], rb[ORC_MAXN], rC[ORC_MAXN * ORC_MAXN], reta[ORC_MAXN], rJ[ORC_MAXN * ORC_MAXN];
    eye(n, I);
    tr(n, n, Ai, AiT);
    tr(n, n, Aj, AjT);
    /* (I + C_i J_j)^{-1} */
    mm(n, n, n, Ci, Jj, t1);
    add(n * n, I, t1, M1);
    if (inv(n, M1, M1i)) return -1;
    /* (I + J_j C_i)^{-1} */
    mm(n, n, n, Jj, Ci, t1);
    add(n * n, I, t1, M2);
    if (inv(n, M2, M2i)) return -1;
    mm(n, n, n, Aj, M1i, AjM1i);
    mm(n, n, n, AiT, M2i, AiTM2i);
    /* A_ij = A_j (I + C_i J_j)^{-1} A_i */
    mm(n, n, n, AjM1i, Ai, rA);
    /* b_ij = A_j (I + C_i J_j)^{-1} (b_i + C_i eta_j) + b_j */
    mm(n, n, 1, Ci, etaj, v);
    add(n, bi, v, v);
    mm(n, n, 1, AjM1i, v, w);
    add(n, w, bj, rb);
    /* C_ij = A_j (I + C_i J_j)^{-1} C_i A_j^T + C_j */
    mm(n, n, n, AjM1i, Ci, t2);
    mm(n, n, n, t2, AjT, t3);
    add(n * n, t3, Cj, rC);
    /* eta_ij = A_i^T (I + J_j C_i)^{-1} (eta_j - J_j b_i) + eta_i */
    mm(n, n, 1, Jj, bi, v);
    sub(n, etaj, v, v);
    mm(n, n, 1, AiTM2i, v, w);
    add(n, w, etai, reta);
    /* J_ij = A_i^T (I + J_j C_i)^{-1} J_j A_i + J_i */
    mm(n, n, n, AiTM2i, Jj, t2);
    mm(n, n, n, t2, Ai, t3);
    add(n * n, t3, Ji, rJ);
    memcpy(A, rA, sizeof(double) * n * n);
    memcpy(b, rb, sizeof(double) * n);
    memcpy(C, rC, sizeof(double) * n * n);
    memcpy(eta, reta, sizeof(double) * n);
    memcpy(J, rJ, sizeof(double) * n * n);
    return 0;
}

/* RTS element layout used by the oracle: [E (n*n), g (n), L (n*n)]. */
int orc_rts_elem_size(int n) { return 2 * n * n + n; }

/* Element of Eqs. prts_init1 (k < T) / prts_init2 (k = T) from the
 * filtering mean xk = xbar_{k|k} and covariance Pk = P_{k|k}. */
int orc_rts_element(int n, const double *F, const double *Q, int last, const double *xk, const double *Pk,
                    double *e) {
    double *E = e, *g = e + n * n, *L = e + n * n + n;
    if (last) {
        memset(E, 0, sizeof(double) * n * n);
        memcpy(g, xk, sizeof(double) * n);
        memcpy(L, Pk, sizeof(double) * n * n);
        return 0;
    }
    double Ft[ORC_MAXN * ORC_MAXN], t1[ORC_MAXN * ORC_MAXN], t2[ORC_MAXN * ORC_MAXN], Pp[ORC_MAXN * ORC_MAXN];
    double Et[ORC_MAXN * ORC_MAXN], v[ORC_MAXN], w[ORC_MAXN], rE[ORC_MAXN * ORC_MAXN];
    tr(n, n, F, Ft);
    mm(n, n, n, F, Pk, t1);
    mm(n, n, n, t1, Ft, t2);
    add(n * n, t2, Q, Pp);                         /* F P F^T + Q */
    /* E^T = (F P F^T + Q)^{-1} (P F^T)^T = (F P F^T + Q)^{-1} F P */
    if (lu_solve(n, n, Pp, t1, Et)) return -1;
    tr(n, n, Et, rE);                               /* E_k = P F^T (F P F^T + Q)^{-1} */
    mm(n, n, 1, F, xk, v);
    mm(n, n, 1, rE, v, w);
    sub(n, xk, w, g);                               /* g_k = xbar - E_k F xbar */
    mm(n, n, n, rE, t1, t2);                        /* E_k F P */
    sub(n * n, Pk, t2, L);                          /* L_k = P - E_k F P */
    memcpy(E, rE, sizeof(double) * n * n);
    return 0;
}

/* Lemma 2: (E_i,g_i,L_i) (x) (E_j,g_j,L_j) = (E_i E_j, E_i g_j + g_i, E_i L_j E_i^T + L_i). */
void orc_rts_combine(int n, const double *ei, const double *ej, double *out) {
    const double *Ei = ei, *gi = ei + n * n, *Li = ei + n * n + n;
    const double *Ej = ej, *gj = ej + n * n, *Lj = ej + n * n + n;
    double rE[ORC_MAXN * ORC_MAXN], rg[ORC_MAXN], rL[ORC_MAXN * ORC_MAXN], t1[ORC_MAXN * ORC_MAXN];
    double t2[ORC_MAXN * ORC_MAXN], EiT[ORC_MAXN * ORC_MAXN];
    tr(n, n, Ei, EiT);
    mm(n, n, n, Ei, Ej, rE);
    mm(n, n, 1, Ei, gj, rg);
    add(n, rg, gi, rg);
    mm(n, n, n, Ei, Lj, t1);
    mm(n, n, n, t1, EiT, t2);
    add(n * n, t2, Li, rL);
    memcpy(out, rE, sizeof(double) * n * n);
    memcpy(out + n * n, rg, sizeof(double) * n);
    memcpy(out + n * n + n, rL, sizeof(double) * n * n);
}

/* ------------------------------------------------------------------ */
/* Time-varying model (Sec. III-A, the transition and measurement      */
/* densities with per-step F_{k-1}, Q_{k-1}, u_{k-1}, H_k, R_k, d_k)    */
/* ------------------------------------------------------------------ */
/* Step record t = 0 .. T-1 belongs to time k = t + 1 and holds
 *     F[t] = F_{k-1}, Q[t] = Q_{k-1}, u[t] = u_{k-1}   (n x n, n x n, n)
 *     H[t] = H_k,     R[t] = R_k,     d[t] = d_k       (m x n, m x m, m)
 * and y[t] = y_k.  u and d may be NULL (zero).  The smoothers use
 * F_k, Q_k, u_k of the step into time k + 1, i.e. record k. */

static void vec_or_zero(int len, const double *base, long t, double *out) {
    if (base) memcpy(out, base + t * len, sizeof(double) * len);
    else memset(out, 0, sizeof(double) * len);
}

/* Sequential Kalman filter, Eqs. KF_mean_pred .. KF_cov_upd, with the
 * innovation log-likelihood sum_k -1/2 (v^T S_k^{-1} v + log det S_k + m log 2 pi),
 * v = y_k - H_k xbar_{k|k-1} - d_k. */
int orc_tv_kf(int n, int m, const double *F, const double *Q, const double *u, const double *H, const double *R,
              const double *d, const double *m0, const double *P0, long T, const double *y,
              double *m_out, double *P_out, double *loglik) {
    double x[ORC_MAXN], P[ORC_MAXN * ORC_MAXN], xp[ORC_MAXN], Pp[ORC_MAXN * ORC_MAXN];
    double t1[ORC_MAXN * ORC_MAXN], t2[ORC_MAXN * ORC_MAXN], Ft[ORC_MAXN * ORC_MAXN], Ht[ORC_MAXN * ORC_MAXN];
    double S[ORC_MAXN * ORC_MAXN], PHt[ORC_MAXN * ORC_MAXN], KT[ORC_MAXN * ORC_MAXN];
    double v[ORC_MAXN], Siv[ORC_MAXN], uk[ORC_MAXN], dk[ORC_MAXN];
    double ll = 0.0;
    const double LOG2PI = 1.8378770664093454835606594728112;
    memcpy(x, m0, sizeof(double) * n);
    memcpy(P, P0, sizeof(double) * n * n);
    for (long t = 0; t < T; ++t) {
        const double *Fk = F + t * n * n, *Qk = Q + t * n * n, *Hk = H + t * m * n, *Rk = R + t * m * m;
        vec_or_zero(n, u, t, uk);
        vec_or_zero(m, d, t, dk);
        /* prediction: xbar_{k|k-1} = F_{k-1} xbar + u_{k-1}, P_{k|k-1} = F P F^T + Q_{k-1} */
        tr(n, n, Fk, Ft);
        mm(n, n, 1, Fk, x, xp);
        add(n, xp, uk, xp);
        mm(n, n, n, Fk, P, t1);
        mm(n, n, n, t1, Ft, t2);
        add(n * n, t2, Qk, Pp);
        /* update: S_k = H_k P_{k|k-1} H_k^T + R_k */
        tr(m, n, Hk, Ht);
        mm(n, n, m, Pp, Ht, PHt);
        mm(m, n, m, Hk, PHt, t1);
        add(m * m, t1, Rk, S);
        /* v = y_k - H_k xbar_{k|k-1} - d_k */
        mm(m, n, 1, Hk, xp, t1);
        sub(m, y + t * m, t1, v);
        sub(m, v, dk, v);
        tr(n, m, PHt, t1);
        double logdetS;
        if (chol_solve(m, n, S, t1, KT, &logdetS)) return -1;
        if (chol_solve(m, 1, S, v, Siv, NULL)) return -1;
        mm(n, m, 1, PHt, Siv, t2);
        add(n, xp, t2, x);                           /* xbar_{k|k} */
        mm(n, m, n, PHt, KT, t2);
        sub(n * n, Pp, t2, P);                       /* P_{k|k} */
        memcpy(m_out + t * n, x, sizeof(double) * n);
        memcpy(P_out + t * n * n, P, sizeof(double) * n * n);
        double q = 0.0;
        for (int i = 0; i < m; ++i) q += v[i] * Siv[i];
        ll += -0.5 * (q + logdetS + m * LOG2PI);
    }
    if (loglik) *loglik = ll;
    return 0;
}

/* Sequential RTS smoother for k = T-1 .. 1 with the step k -> k+1:
 * xbar_{k+1|k} = F_k xbar_{k|k} + u_k, P_{k+1|k} = F_k P_{k|k} F_k^T + Q_k,
 * G_k = P_{k|k} F_k^T P_{k+1|k}^{-1}, then the Sec. III-B recursion. */
int orc_tv_rts(int n, const double *F, const double *Q, const double *u, long T, const double *mf, const double *Pf,
               double *ms, double *Ps) {
    double Ft[ORC_MAXN * ORC_MAXN], Pp[ORC_MAXN * ORC_MAXN], xp[ORC_MAXN], uk[ORC_MAXN];
    double t1[ORC_MAXN * ORC_MAXN], t2[ORC_MAXN * ORC_MAXN], G[ORC_MAXN * ORC_MAXN], Gt[ORC_MAXN * ORC_MAXN];
    double dx[ORC_MAXN], dP[ORC_MAXN * ORC_MAXN];
    memcpy(ms + (T - 1) * n, mf + (T - 1) * n, sizeof(double) * n);
    memcpy(Ps + (T - 1) * n * n, Pf + (T - 1) * n * n, sizeof(double) * n * n);
    for (long t = T - 2; t >= 0; --t) {             /* time k = t + 1, step record k = t + 1 */
        const double *x = mf + t * n, *P = Pf + t * n * n;
        const double *Fk = F + (t + 1) * n * n, *Qk = Q + (t + 1) * n * n;
        vec_or_zero(n, u, t + 1, uk);
        tr(n, n, Fk, Ft);
        mm(n, n, 1, Fk, x, xp);
        add(n, xp, uk, xp);                          /* xbar_{k+1|k} */
        mm(n, n, n, Fk, P, t1);
        mm(n, n, n, t1, Ft, t2);
        add(n * n, t2, Qk, Pp);                      /* P_{k+1|k} */
        if (lu_solve(n, n, Pp, t1, Gt)) return -1;   /* G^T = P_{k+1|k}^{-1} F_k P */
        tr(n, n, Gt, G);
        sub(n, ms + (t + 1) * n, xp, dx);
        mm(n, n, 1, G, dx, t1);
        add(n, x, t1, ms + t * n);
        sub(n * n, Ps + (t + 1) * n * n, Pp, dP);
        mm(n, n, n, G, dP, t1);
        mm(n, n, n, t1, Gt, t2);
        add(n * n, P, t2, Ps + t * n * n);
    }
    return 0;
}

/* Sequential two-filter smoother: the backward information filter of
 * Eqs. tf_vector_pred .. tf_matrix_upd with u and d, merged with the filter
 * by Eqs. mean_tf_combination / cov_tf_combination.  eta_out, J_out
 * (nullable) receive eta_{k|k+1:T}, J_{k|k+1:T} (zero at k = T). */
int orc_tv_tf(int n, int m, const double *F, const double *Q, const double *u, const double *H, const double *R,
              const double *d, long T, const double *y, const double *mf, const double *Pf, double *ms, double *Ps,
              double *eta_out, double *J_out) {
    double Ft[ORC_MAXN * ORC_MAXN], Ht[ORC_MAXN * ORC_MAXN], Ri[ORC_MAXN * ORC_MAXN], HtRi[ORC_MAXN * ORC_MAXN];
    double eta[ORC_MAXN], J[ORC_MAXN * ORC_MAXN], t1[ORC_MAXN * ORC_MAXN], t2[ORC_MAXN * ORC_MAXN];
    double Mx[ORC_MAXN * ORC_MAXN], I[ORC_MAXN * ORC_MAXN], rhs[ORC_MAXN * (ORC_MAXN + 1)];
    double sol[ORC_MAXN * (ORC_MAXN + 1)], uk[ORC_MAXN], dk[ORC_MAXN], yd[ORC_MAXN];
    eye(n, I);
    memset(eta, 0, sizeof(double) * n);          /* eta_{T|T+1:T} = 0 */
    memset(J, 0, sizeof(double) * n * n);        /* J_{T|T+1:T}   = 0 */
    for (long t = T - 1; t >= 0; --t) {          /* time k = t + 1 */
        const double *x = mf + t * n, *P = Pf + t * n * n;
        if (eta_out) memcpy(eta_out + t * n, eta, sizeof(double) * n);
        if (J_out) memcpy(J_out + t * n * n, J, sizeof(double) * n * n);
        /* merge: xbar_{k|T} = (I + P J)^{-1}(xbar + P eta), P_{k|T} = (I + P J)^{-1} P */
        mm(n, n, n, P, J, t1);
        add(n * n, I, t1, Mx);
        mm(n, n, 1, P, eta, t2);
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) rhs[i * (n + 1) + j] = P[i * n + j];
            rhs[i * (n + 1) + n] = x[i] + t2[i];
        }
        if (lu_solve(n, n + 1, Mx, rhs, sol)) return -1;
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) Ps[t * n * n + i * n + j] = sol[i * (n + 1) + j];
            ms[t * n + i] = sol[i * (n + 1) + n];
        }
        if (t == 0) break;
        /* update with y_k: eta += H_k^T R_k^{-1} (y_k - d_k), J += H_k^T R_k^{-1} H_k */
        const double *Hk = H + t * m * n, *Rk = R + t * m * m;
        vec_or_zero(m, d, t, dk);
        tr(m, n, Hk, Ht);
        if (inv(m, Rk, Ri)) return -1;
        mm(n, m, m, Ht, Ri, HtRi);
        sub(m, y + t * m, dk, yd);
        mm(n, m, 1, HtRi, yd, t1);
        add(n, eta, t1, eta);
        mm(n, m, n, HtRi, Hk, t1);
        add(n * n, J, t1, J);
        /* backward prediction to time k - 1 with F_{k-1}, Q_{k-1}, u_{k-1} (record t):
         * eta <- F^T (I + J Q)^{-1} (eta - J u),  J <- F^T (I + J Q)^{-1} J F */
        const double *Fk = F + t * n * n, *Qk = Q + t * n * n;
        vec_or_zero(n, u, t, uk);
        tr(n, n, Fk, Ft);
        mm(n, n, n, J, Qk, t1);
        add(n * n, I, t1, Mx);
        mm(n, n, 1, J, uk, t2);
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) rhs[i * (n + 1) + j] = J[i * n + j];
            rhs[i * (n + 1) + n] = eta[i] - t2[i];
        }
        if (lu_solve(n, n + 1, Mx, rhs, sol)) return -1;
        double JF[ORC_MAXN * ORC_MAXN], v[ORC_MAXN], MiJ[ORC_MAXN * ORC_MAXN];
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < n; ++j) MiJ[i * n + j] = sol[i * (n + 1) + j];
            v[i] = sol[i * (n + 1) + n];
        }
        mm(n, n, 1, Ft, v, eta);
        mm(n, n, n, MiJ, Fk, JF);
        mm(n, n, n, Ft, JF, J);
    }
    return 0;
}

/* Element a_k of Eqs. pkf_init1 (first = 0) / pkf_init2 (first = 1) and
 * pkf_init3 for one step, given that step's F_{k-1}, Q_{k-1}, u_{k-1}, H_k,
 * R_k, d_k (u, d nullable) and y_k.  As for the time-invariant element,
 * eta_k and J_k use S_k = H_k Q_{k-1} H_k^T + R_k for every k (eta_1, J_1
 * never reach an output because A_1 = 0). */
int orc_tv_filter_element(int n, int m, const double *F, const double *Q, const double *u, const double *H,
                          const double *R, const double *d, const double *m0, const double *P0, int first,
                          const double *yk, double *e) {
    double *A = e, *b = e + n * n, *C = e + n * n + n, *eta = e + 2 * n * n + n, *J = e + 2 * n * n + 2 * n;
    double Ht[ORC_MAXN * ORC_MAXN], Ft[ORC_MAXN * ORC_MAXN], t1[ORC_MAXN * ORC_MAXN], t2[ORC_MAXN * ORC_MAXN];
    double S[ORC_MAXN * ORC_MAXN], KT[ORC_MAXN * ORC_MAXN], K[ORC_MAXN * ORC_MAXN], IKH[ORC_MAXN * ORC_MAXN];
    double uk[ORC_MAXN], dk[ORC_MAXN], v[ORC_MAXN], QHt[ORC_MAXN * ORC_MAXN];
    vec_or_zero(n, u, 0, uk);
    vec_or_zero(m, d, 0, dk);
    tr(m, n, H, Ht);
    tr(n, n, F, Ft);
    if (first) {
        double xp[ORC_MAXN], Pp[ORC_MAXN * ORC_MAXN], PHt[ORC_MAXN * ORC_MAXN], KS[ORC_MAXN * ORC_MAXN];
        mm(n, n, 1, F, m0, xp);
        add(n, xp, uk, xp);                      /* xbar_{1|0} = F_0 xbar_{0|0} + u_0 */
        mm(n, n, n, F, P0, t1);
        mm(n, n, n, t1, Ft, t2);
        add(n * n, t2, Q, Pp);                   /* P_{1|0} = F_0 P_{0|0} F_0^T + Q_0 */
        mm(n, n, m, Pp, Ht, PHt);
        mm(m, n, m, H, PHt, t1);
        add(m * m, t1, R, S);                    /* S_1 = H_1 P_{1|0} H_1^T + R_1 */
        tr(n, m, PHt, t1);
        if (chol_solve(m, n, S, t1, KT, NULL)) return -1;
        tr(m, n, KT, K);                         /* K_1 = P_{1|0} H_1^T S_1^{-1} */
        memset(A, 0, sizeof(double) * n * n);    /* A_1 = 0 */
        mm(m, n, 1, H, xp, t1);
        sub(m, yk, t1, v);
        sub(m, v, dk, v);
        mm(n, m, 1, K, v, t1);
        add(n, xp, t1, b);                       /* b_1 = xbar_{1|0} + K_1 (y_1 - H_1 xbar_{1|0} - d_1) */
        mm(n, m, m, K, S, KS);
        mm(n, m, n, KS, KT, t1);
        sub(n * n, Pp, t1, C);                   /* C_1 = P_{1|0} - K_1 S_1 K_1^T */
    } else {
        mm(n, n, m, Q, Ht, QHt);
        mm(m, n, m, H, QHt, t1);
        add(m * m, t1, R, S);                    /* S_k = H_k Q_{k-1} H_k^T + R_k */
        tr(n, m, QHt, t1);
        if (chol_solve(m, n, S, t1, KT, NULL)) return -1;
        tr(m, n, KT, K);                         /* K_k = Q_{k-1} H_k^T S_k^{-1} */
        mm(n, m, n, K, H, t1);
        eye(n, t2);
        sub(n * n, t2, t1, IKH);
        mm(n, n, n, IKH, F, A);                  /* A_k = (I - K_k H_k) F_{k-1} */
        mm(m, n, 1, H, uk, t1);
        sub(m, yk, t1, v);
        sub(m, v, dk, v);
        mm(n, m, 1, K, v, t1);
        add(n, uk, t1, b);                       /* b_k = u_{k-1} + K_k (y_k - H_k u_{k-1} - d_k) */
        mm(n, n, n, IKH, Q, C);                  /* C_k = (I - K_k H_k) Q_{k-1} */
    }
    {   /* Eq. pkf_init3: eta_k = F^T H^T S^{-1} (y_k - H_k u_{k-1} - d_k), J_k = F^T H^T S^{-1} H F */
        double Sx[ORC_MAXN * ORC_MAXN], SiH[ORC_MAXN * ORC_MAXN], Siy[ORC_MAXN], HF[ORC_MAXN * ORC_MAXN];
        double FtHt[ORC_MAXN * ORC_MAXN];
        mm(n, n, m, Q, Ht, QHt);
        mm(m, n, m, H, QHt, t1);
        add(m * m, t1, R, Sx);
        mm(m, n, 1, H, uk, t1);
        sub(m, yk, t1, v);
        sub(m, v, dk, v);
        if (chol_solve(m, 1, Sx, v, Siy, NULL)) return -1;
        mm(m, n, n, H, F, HF);
        if (chol_solve(m, n, Sx, HF, SiH, NULL)) return -1;
        tr(m, n, HF, FtHt);
        mm(n, m, 1, FtHt, Siy, eta);
        mm(n, m, n, FtHt, SiH, J);
    }
    return 0;
}

/* Element of Eqs. prts_init1 (last = 0, with the step's F_k, Q_k, u_k;
 * u nullable) / prts_init2 (last = 1) from xbar_{k|k}, P_{k|k}. */
int orc_tv_rts_element(int n, const double *F, const double *Q, const double *u, int last, const double *xk,
                       const double *Pk, double *e) {
    double *E = e, *g = e + n * n, *L = e + n * n + n;
    if (last) {
        memset(E, 0, sizeof(double) * n * n);
        memcpy(g, xk, sizeof(double) * n);
        memcpy(L, Pk, sizeof(double) * n * n);
        return 0;
    }
    double Ft[ORC_MAXN * ORC_MAXN], t1[ORC_MAXN * ORC_MAXN], t2[ORC_MAXN * ORC_MAXN], Pp[ORC_MAXN * ORC_MAXN];
    double Et[ORC_MAXN * ORC_MAXN], v[ORC_MAXN], w[ORC_MAXN], rE[ORC_MAXN * ORC_MAXN], uk[ORC_MAXN];
    vec_or_zero(n, u, 0, uk);
    tr(n, n, F, Ft);
    mm(n, n, n, F, Pk, t1);
    mm(n, n, n, t1, Ft, t2);
    add(n * n, t2, Q, Pp);                         /* F_k P F_k^T + Q_k */
    if (lu_solve(n, n, Pp, t1, Et)) return -1;
    tr(n, n, Et, rE);                               /* E_k = P F_k^T (F_k P F_k^T + Q_k)^{-1} */
    mm(n, n, 1, F, xk, v);
    add(n, v, uk, v);
    mm(n, n, 1, rE, v, w);
    sub(n, xk, w, g);                               /* g_k = xbar - E_k (F_k xbar + u_k) */
    mm(n, n, n, rE, t1, t2);
    sub(n * n, Pk, t2, L);                          /* L_k = P - E_k F_k P */
    memcpy(E, rE, sizeof(double) * n * n);
    return 0;
}
