// gain_tables.h -- the data-independent halves of the filtering and RTS
// elements of a time-invariant model, evaluated on the host in FP64.
//
// In a time-invariant model the (A, C, J) half of every filtering element
// (Eqs. pkf_init1..3) and the (E, L) half of every RTS element (Eqs.
// prts_init1, prts_init2) do not depend on the measurements, so neither do
// their prefix compositions under Lemma 1 and Lemma 2: the filtering
// covariances P_{k|k}, the gains and the smoothed covariances P_{k|T} are
// the same for every data set.  What depends on the data is the (b) half of
// the filtering prefixes and the (g) half of the smoothing suffixes, which
// under those compositions are affine recursions with data-independent
// coefficients:
//   xbar_{k|k} = M_k xbar_{k-1|k-1} + K_k y_k,   M_k = (I - K_k H) F,
//   xbar_{k|T} = E_k xbar_{k+1|T} + G_k xbar_{k|k},   G_k = I - E_k F.
// The covariance recursion converges geometrically to its fixed point; the
// tables hold the steps before it settles (relative change below 2^-46 on
// four consecutive steps) and the settled values, which the remaining steps
// share to within that bound.
#pragma once

#include <stdint.h>

#include <vector>

namespace kfs {

struct GainModel {
    uint64_t key = 0;   // identifies the model (a hash of its matrices)
    int n = 0, m = 0;
    int k0 = 0;   // times 1..k0 have their own coefficients; later times the settled ones
    int kb = 0;   // smoothed covariances of times T - d, d = 0 .. kb - 1, from the tail table
    // the same for FP32 work: every table entry past them is within 2^-30
    // (relative) of the settled value, far below FP32 rounding
    int k0_32 = 0, kb_32 = 0;
    // time k = 1..k0 at index k - 1 (row-major n x n, n x m, m x m)
    std::vector<double> M, K, W, P, ld;   // M_k, K_k, W_k = chol(S_k)^{-1} (lower), P_{k|k}, log det S_k
    std::vector<double> E, G;             // E_k, G_k of Eq. prts_init1
    std::vector<double> Psf;              // P_{k|T}, k = 1..k0 (valid for T >= k0 + kb + 1)
    std::vector<double> Pst;              // P_{T-d|T}, d = 0..kb-1
    // settled values
    double Mi[64], Ki[64], Wi[64], Pi[64], ldi, Ei[64], Gi[64], Psi[64];
    double HF[64];                        // H F (m x n)
    double F[64];
    double m0[8];
};

// Builds the tables of the model (F, Q, H, R: n x n, n x n, m x n, m x m;
// m0, P0 the prior).  Returns 0, 1 if the covariance recursion does not
// settle within 2^16 steps, -1 if a matrix that must be positive definite
// is not.
int gain_model_build(int n, int m, const double *F, const double *Q, const double *H, const double *R,
                     const double *m0, const double *P0, GainModel *g);

// The matrix power A^e (n x n, FP64) by repeated squaring.
void gain_mat_pow(int n, const double *A, int64_t e, double *out);
void gain_mat_mul(int n, const double *A, const double *B, double *C);

}  // namespace kfs
