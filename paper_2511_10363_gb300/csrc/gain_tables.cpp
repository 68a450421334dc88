// gain_tables.cpp -- host FP64 evaluation of the data-independent halves of
// the filtering and RTS elements of a time-invariant model (gain_tables.h).
#include "gain_tables.h"

#include <math.h>
#include <string.h>

namespace kfs {

namespace {

constexpr int MX = 8;
constexpr int KMAX = 1 << 16;        // steps the covariance recursion may take to settle
constexpr double SETTLE = 1.4210854715202004e-14;   // 2^-46
constexpr int SETTLE_RUN = 4;

// C = A B with A r x k, B k x c (row-major)
void mm(int r, int k, int c, const double *A, const double *B, double *C) {
    double t[MX * MX];
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) {
            double s = 0;
            for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * c + j];
            t[i * c + j] = s;
        }
    memcpy(C, t, sizeof(double) * r * c);
}
// C = A B^T with A r x k, B c x k
void mmt(int r, int k, int c, const double *A, const double *B, double *C) {
    double t[MX * MX];
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) {
            double s = 0;
            for (int l = 0; l < k; ++l) s += A[i * k + l] * B[j * k + l];
            t[i * c + j] = s;
        }
    memcpy(C, t, sizeof(double) * r * c);
}
void symm(int n, double *A) {
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) A[i * n + j] = A[j * n + i] = 0.5 * (A[i * n + j] + A[j * n + i]);
}
// lower Cholesky factor L of SPD A (n x n); false if not positive definite
bool chol(int n, const double *A, double *L) {
    memset(L, 0, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(s > 0)) return false;
                L[i * n + i] = sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    return true;
}
// inverse of a lower-triangular L (n x n)
void tri_inv(int n, const double *L, double *Li) {
    memset(Li, 0, sizeof(double) * n * n);
    for (int c = 0; c < n; ++c) {
        Li[c * n + c] = 1.0 / L[c * n + c];
        for (int i = c + 1; i < n; ++i) {
            double s = 0;
            for (int k = c; k < i; ++k) s -= L[i * n + k] * Li[k * n + c];
            Li[i * n + c] = s / L[i * n + i];
        }
    }
}
// X = A^{-1} B for SPD A (n x n), B n x c
bool spd_solve(int n, int c, const double *A, const double *B, double *X) {
    double L[MX * MX], Li[MX * MX], t[MX * MX];
    if (!chol(n, A, L)) return false;
    tri_inv(n, L, Li);
    mm(n, n, c, Li, B, t);
    // A^{-1} = Li^T Li
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < c; ++j) {
            double s = 0;
            for (int k = 0; k < n; ++k) s += Li[k * n + i] * t[k * c + j];
            X[i * c + j] = s;
        }
    return true;
}
double rel_change(int len, const double *a, const double *b) {
    double d = 0, s = 0;
    for (int i = 0; i < len; ++i) {
        d = fmax(d, fabs(a[i] - b[i]));
        s = fmax(s, fabs(b[i]));
    }
    return s > 0 ? d / s : d;
}

// One step of the filtering covariance recursion (Sec. III-A) from P_{k-1|k-1}:
// M_k, K_k, W_k, log det S_k, P_{k|k}.
bool filt_step(int n, int m, const double *F, const double *Q, const double *H, const double *R,
               const double *Pprev, double *Mk, double *Kk, double *Wk, double *ldk, double *Pk) {
    double Pp[MX * MX], S[MX * MX], PHt[MX * MX], KT[MX * MX], L[MX * MX], t[MX * MX];
    mm(n, n, n, F, Pprev, t);
    mmt(n, n, n, t, F, Pp);
    for (int i = 0; i < n * n; ++i) Pp[i] += Q[i];
    symm(n, Pp);
    mmt(n, n, m, Pp, H, PHt);                 // P_{k|k-1} H^T
    mm(m, n, m, H, PHt, S);
    for (int i = 0; i < m * m; ++i) S[i] += R[i];
    symm(m, S);
    if (!chol(m, S, L)) return false;
    double ld = 0;
    for (int i = 0; i < m; ++i) ld += 2.0 * log(L[i * m + i]);
    *ldk = ld;
    tri_inv(m, L, Wk);
    // K^T = S^{-1} (P H^T)^T
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) t[i * n + j] = PHt[j * m + i];
    if (!spd_solve(m, n, S, t, KT)) return false;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) Kk[i * m + j] = KT[j * n + i];
    // P_{k|k} = P_{k|k-1} - P H^T S^{-1} H P
    mm(n, m, n, PHt, KT, t);
    for (int i = 0; i < n * n; ++i) Pk[i] = Pp[i] - t[i];
    symm(n, Pk);
    // M_k = (I - K H) F
    double IKH[MX * MX];
    mm(n, m, n, Kk, H, IKH);
    for (int i = 0; i < n * n; ++i) IKH[i] = -IKH[i];
    for (int i = 0; i < n; ++i) IKH[i * n + i] += 1.0;
    mm(n, n, n, IKH, F, Mk);
    return true;
}

// RTS coefficients of time k from P_{k|k} (Eq. prts_init1): E_k, G_k and
// the predicted covariance P_{k+1|k}.
bool rts_coef(int n, const double *F, const double *Q, const double *Pk, double *Ek, double *Gk, double *Pp) {
    double t[MX * MX], ET[MX * MX];
    mm(n, n, n, F, Pk, t);                    // F P
    mmt(n, n, n, t, F, Pp);
    for (int i = 0; i < n * n; ++i) Pp[i] += Q[i];
    symm(n, Pp);
    // E^T = P_{k+1|k}^{-1} F P
    if (!spd_solve(n, n, Pp, t, ET)) return false;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ek[i * n + j] = ET[j * n + i];
    mm(n, n, n, Ek, F, t);
    for (int i = 0; i < n * n; ++i) Gk[i] = -t[i];
    for (int i = 0; i < n; ++i) Gk[i * n + i] += 1.0;
    return true;
}

// P_{k|T} = P_{k|k} + E_k (P_{k+1|T} - P_{k+1|k}) E_k^T
void smooth_cov(int n, const double *Pk, const double *Ek, const double *Pnext, const double *Pp, double *out) {
    double D[MX * MX], t[MX * MX];
    for (int i = 0; i < n * n; ++i) D[i] = Pnext[i] - Pp[i];
    mm(n, n, n, Ek, D, t);
    mmt(n, n, n, t, Ek, D);
    for (int i = 0; i < n * n; ++i) out[i] = Pk[i] + D[i];
    symm(n, out);
}

}  // namespace

void gain_mat_mul(int n, const double *A, const double *B, double *C) { mm(n, n, n, A, B, C); }

void gain_mat_pow(int n, const double *A, int64_t e, double *out) {
    double r[MX * MX], b[MX * MX];
    memset(r, 0, sizeof(r));
    for (int i = 0; i < n; ++i) r[i * n + i] = 1.0;
    memcpy(b, A, sizeof(double) * n * n);
    while (e > 0) {
        if (e & 1) mm(n, n, n, r, b, r);
        e >>= 1;
        if (e) mm(n, n, n, b, b, b);
    }
    memcpy(out, r, sizeof(double) * n * n);
}

int gain_model_build(int n, int m, const double *F, const double *Q, const double *H, const double *R,
                     const double *m0, const double *P0, GainModel *g) {
    if (n < 1 || n > MX || m < 1 || m > MX) return -1;
    const int nn = n * n, nm = n * m, mmn = m * m;
    g->n = n;
    g->m = m;
    g->M.clear(); g->K.clear(); g->W.clear(); g->P.clear(); g->ld.clear();
    g->E.clear(); g->G.clear(); g->Psf.clear(); g->Pst.clear();
    memcpy(g->F, F, sizeof(double) * nn);
    memcpy(g->m0, m0, sizeof(double) * n);
    mm(m, n, n, H, F, g->HF);
    // ---- filtering covariances, forward until they settle
    double Pprev[MX * MX];
    memcpy(Pprev, P0, sizeof(double) * nn);
    int run = 0, k = 0;
    while (true) {
        if (k >= KMAX) return 1;
        double Mk[MX * MX], Kk[MX * MX], Wk[MX * MX], Pk[MX * MX], ldk;
        if (!filt_step(n, m, F, Q, H, R, Pprev, Mk, Kk, Wk, &ldk, Pk)) return -1;
        ++k;
        g->M.insert(g->M.end(), Mk, Mk + nn);
        g->K.insert(g->K.end(), Kk, Kk + nm);
        g->W.insert(g->W.end(), Wk, Wk + mmn);
        g->P.insert(g->P.end(), Pk, Pk + nn);
        g->ld.push_back(ldk);
        run = (k > 1 && rel_change(nn, Pk, Pprev) <= SETTLE) ? run + 1 : 0;
        memcpy(Pprev, Pk, sizeof(double) * nn);
        if (run >= SETTLE_RUN) break;
    }
    g->k0 = k;
    memcpy(g->Pi, Pprev, sizeof(double) * nn);
    {   // the coefficients of every later step: those of a step from P_inf
        double Ptmp[MX * MX];
        if (!filt_step(n, m, F, Q, H, R, g->Pi, g->Mi, g->Ki, g->Wi, &g->ldi, Ptmp)) return -1;
    }
    // ---- RTS coefficients of times 1..k0 and the settled ones
    g->E.resize(size_t(k) * nn);
    g->G.resize(size_t(k) * nn);
    std::vector<double> Pp(size_t(k) * nn);   // P_{k+1|k}
    for (int t = 0; t < k; ++t)
        if (!rts_coef(n, F, Q, &g->P[size_t(t) * nn], &g->E[size_t(t) * nn], &g->G[size_t(t) * nn],
                      &Pp[size_t(t) * nn]))
            return -1;
    double Ppi[MX * MX];
    if (!rts_coef(n, F, Q, g->Pi, g->Ei, g->Gi, Ppi)) return -1;
    // ---- smoothed covariances near T (times with settled P_{k|k}), until they settle
    {
        double Ps[MX * MX], Pn[MX * MX];
        memcpy(Ps, g->Pi, sizeof(double) * nn);   // P_{T|T}
        g->Pst.insert(g->Pst.end(), Ps, Ps + nn);
        run = 0;
        int d = 0;
        while (true) {
            if (d >= KMAX) return 1;
            smooth_cov(n, g->Pi, g->Ei, Ps, Ppi, Pn);
            ++d;
            run = rel_change(nn, Pn, Ps) <= SETTLE ? run + 1 : 0;
            memcpy(Ps, Pn, sizeof(double) * nn);
            g->Pst.insert(g->Pst.end(), Pn, Pn + nn);
            if (run >= SETTLE_RUN) break;
        }
        g->kb = d + 1;
        memcpy(g->Psi, Ps, sizeof(double) * nn);
    }
    // ---- smoothed covariances of times k0..1 from the settled value at k0 + 1
    {
        g->Psf.resize(size_t(k) * nn);
        double Pn[MX * MX];
        memcpy(Pn, g->Psi, sizeof(double) * nn);
        for (int t = k - 1; t >= 0; --t) {
            smooth_cov(n, &g->P[size_t(t) * nn], &g->E[size_t(t) * nn], Pn, &Pp[size_t(t) * nn],
                       &g->Psf[size_t(t) * nn]);
            memcpy(Pn, &g->Psf[size_t(t) * nn], sizeof(double) * nn);
        }
    }
    // ---- the shorter transients for FP32 work
    {
        const double thr = 9.3132257461547852e-10;   // 2^-30
        auto far = [&](int len, const double *a, const double *b) { return rel_change(len, a, b) > thr; };
        g->k0_32 = 0;
        for (int t = 0; t < k; ++t) {
            const bool d = far(nn, &g->M[size_t(t) * nn], g->Mi) || far(nm, &g->K[size_t(t) * nm], g->Ki) ||
                           far(mmn, &g->W[size_t(t) * mmn], g->Wi) || far(nn, &g->P[size_t(t) * nn], g->Pi) ||
                           far(nn, &g->E[size_t(t) * nn], g->Ei) || far(nn, &g->G[size_t(t) * nn], g->Gi) ||
                           far(nn, &g->Psf[size_t(t) * nn], g->Psi) || fabs(g->ld[size_t(t)] - g->ldi) > thr;
            if (d) g->k0_32 = t + 1;
        }
        g->kb_32 = 1;
        for (int d = 0; d < g->kb; ++d)
            if (far(nn, &g->Pst[size_t(d) * nn], g->Psi)) g->kb_32 = d + 1;
    }
    return 0;
}

}  // namespace kfs
