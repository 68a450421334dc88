// kf_math.cuh -- register-resident small-matrix blocks and the associative
// operators of arXiv 2511.10363 (Sec. IV-C Lemma 1, Sec. IV-D Lemma 2), the
// element constructions (Eqs. pkf_init1/2/3, prts_init1/2) and the
// two-filter merge (Eqs. mean_tf_combination / cov_tf_combination).
//
// Every block is a fixed-size array indexed only with compile-time indices
// after unrolling, so it lives in registers.  Symmetric matrices (C, J, L,
// covariances) are stored as their packed upper triangle, which makes every
// produced covariance exactly symmetric.
//
// One-sided forms.  In Lemma 1 the outputs b_ij and C_ij depend on the left
// operand only through (b_i, C_i), and eta_ij, J_ij depend on the right
// operand only through (eta_j, J_j).  In Lemma 2, g_ij and L_ij depend on the
// right operand only through (g_j, L_j).  A scan carry therefore holds only
// the half it is extracted from, and applying an element to it evaluates
// only that half of the operator ("apply_*" below).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define KF_HD __host__ __device__ __forceinline__
#define KF_D __device__ __forceinline__

namespace kfs {

// Index checks of the bounds-checked build (compiled with KF_BOUNDS_CHECK):
// a failed check records KF_ERR_BOUNDS (10) in the status word, unless it
// already holds an error, and the access it guards is skipped.  In the
// normal build every check is the constant true.
#if defined(KF_BOUNDS_CHECK) && defined(__CUDACC__)
KF_D bool kf_in(bool ok, int *status) {
    if (!ok) atomicCAS(status, 0, 10);
    return ok;
}
#define KF_IN(cond, status) ::kfs::kf_in((cond), (status))
#else
#define KF_IN(cond, status) true
#endif

constexpr int MAXNY = 8;

// packed upper-triangular index, row-major over i <= j
KF_HD constexpr int su(int N, int i, int j) { return i * N - (i * (i - 1)) / 2 + (j - i); }
KF_HD constexpr int si(int N, int i, int j) { return i <= j ? su(N, i, j) : su(N, j, i); }

// ---------------------------------------------------------------- elements

// Filtering element (A, b, C, eta, J) of Sec. IV-C; C and J packed symmetric.
template <int N, typename R>
struct FElem {
    static constexpr int NN = N * N, S = N * (N + 1) / 2;
    static constexpr int oA = 0, ob = NN, oC = NN + N, oe = NN + N + S, oJ = NN + 2 * N + S;
    static constexpr int SIZE = NN + 2 * N + 2 * S;
    R v[SIZE];
};

// Forward filtering carry: (b, C) of a prefix a_1 (x) ... (x) a_k.
template <int N, typename R>
struct FwdCarry {
    static constexpr int S = N * (N + 1) / 2, ob = 0, oC = N, SIZE = N + S;
    R v[SIZE];
};

// Backward information carry: (eta, J) of a suffix a_{k+1} (x) ... (x) e.
template <int N, typename R>
struct RevCarry {
    static constexpr int S = N * (N + 1) / 2, oe = 0, oJ = N, SIZE = N + S;
    R v[SIZE];
};

// RTS element (E, g, L) of Sec. IV-D; L packed symmetric.
template <int N, typename R>
struct RElem {
    static constexpr int NN = N * N, S = N * (N + 1) / 2;
    static constexpr int oE = 0, og = NN, oL = NN + N, SIZE = NN + N + S;
    R v[SIZE];
};

// RTS carry: (g, L) of a suffix a_k (x) ... (x) a_T.
template <int N, typename R>
struct RCarry {
    static constexpr int S = N * (N + 1) / 2, og = 0, oL = N, SIZE = N + S;
    R v[SIZE];
};

template <class X>
KF_HD void set_zero(X &x) {
#pragma unroll
    for (int i = 0; i < X::SIZE; ++i) x.v[i] = 0;
}

// (I, 0, 0, 0, 0): the neutral element of Lemma 1.
template <int N, typename R>
KF_HD void set_identity(FElem<N, R> &e) {
    set_zero(e);
#pragma unroll
    for (int i = 0; i < N; ++i) e.v[FElem<N, R>::oA + i * N + i] = R(1);
}

// (I, 0, 0): the neutral element of Lemma 2.
template <int N, typename R>
KF_HD void set_identity(RElem<N, R> &e) {
    set_zero(e);
#pragma unroll
    for (int i = 0; i < N; ++i) e.v[RElem<N, R>::oE + i * N + i] = R(1);
}

// ---------------------------------------------------------------- record copies

// Copy REC consecutive values between a record (shared or device memory,
// aligned to its size class) and registers with the widest vector accesses
// the record allows (16-, 8- or 4-byte), so that a warp reading its lanes'
// records from a staging buffer with an odd 16-byte stride is conflict-free.
template <int REC, typename R>
KF_D void load_rec(R *dst, const R *src) {
    constexpr int B = REC * int(sizeof(R));
    if constexpr (B % 16 == 0 && sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < REC / 4; ++i) {
            const float4 v = reinterpret_cast<const float4 *>(src)[i];
            dst[4 * i] = v.x; dst[4 * i + 1] = v.y; dst[4 * i + 2] = v.z; dst[4 * i + 3] = v.w;
        }
    } else if constexpr (B % 16 == 0 && sizeof(R) == 8) {
#pragma unroll
        for (int i = 0; i < REC / 2; ++i) {
            const double2 v = reinterpret_cast<const double2 *>(src)[i];
            dst[2 * i] = v.x; dst[2 * i + 1] = v.y;
        }
    } else if constexpr (B % 8 == 0 && sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < REC / 2; ++i) {
            const float2 v = reinterpret_cast<const float2 *>(src)[i];
            dst[2 * i] = v.x; dst[2 * i + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < REC; ++i) dst[i] = src[i];
    }
}
template <int REC, typename R>
KF_D void store_rec(R *dst, const R *src) {
    constexpr int B = REC * int(sizeof(R));
    if constexpr (B % 16 == 0 && sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < REC / 4; ++i)
            reinterpret_cast<float4 *>(dst)[i] = make_float4(src[4 * i], src[4 * i + 1], src[4 * i + 2], src[4 * i + 3]);
    } else if constexpr (B % 16 == 0 && sizeof(R) == 8) {
#pragma unroll
        for (int i = 0; i < REC / 2; ++i) reinterpret_cast<double2 *>(dst)[i] = make_double2(src[2 * i], src[2 * i + 1]);
    } else if constexpr (B % 8 == 0 && sizeof(R) == 4) {
#pragma unroll
        for (int i = 0; i < REC / 2; ++i) reinterpret_cast<float2 *>(dst)[i] = make_float2(src[2 * i], src[2 * i + 1]);
    } else {
#pragma unroll
        for (int i = 0; i < REC; ++i) dst[i] = src[i];
    }
}

// ---------------------------------------------------------------- model constants

// k-invariant quantities, computed on the host in FP64 and rounded once to
// the working precision R.
template <int N, typename R>
struct FiltParams {
    static constexpr int NN = N * N, S = N * (N + 1) / 2;
    R A[NN], C[S], J[S];          // a_k, k >= 2: Eq. pkf_init1 and Eq. pkf_init3
    R K[N * MAXNY];               // b_k = K y_k              (K = Q H^T S^{-1})
    R G[N * MAXNY];               // eta_k = G y_k            (G = F^T H^T S^{-1})
    R K1[N * MAXNY], c1[N], C1[S];// a_1, Eq. pkf_init2: b_1 = c1 + K1 y_1
    R HF[MAXNY * N];              // log-likelihood: v_k = y_k - H F xbar_{k-1|k-1}
    R Sinv[MAXNY * MAXNY];        //   S^{-1}, S = H Q H^T + R
    R S1inv[MAXNY * MAXNY];       //   S_1^{-1}, S_1 = H P_{1|0} H^T + R
    R Hx1[MAXNY];                 //   H xbar_{1|0}
    double llc, llc1;             //   log det S + m log 2 pi,  log det S_1 + m log 2 pi
    R llc_r;                      //   llc in the working precision
    R F[NN], Q[S];                // RTS elements, Eq. prts_init1
    R U[MAXNY * N];               // J = U^T U, U = L^{-1} H F with S = L L^T (low-rank path)
    R Linv[MAXNY * MAXNY];        //   L^{-1} (lower triangular)
    int ny;
};

// ---------------------------------------------------------------- small solves

// Reciprocal, square root and natural log of the small solves.  FP32: the
// hardware approximations (PTX rcp.approx / sqrt.approx, MUFU log2; relative
// error about 2^-23, a few ulp for the log), far below the FP32 tolerance of
// the outputs and cheaper than the correctly rounded sequences.  FP64:
// correctly rounded.  (A host build of these headers, the flop counter of
// flop_count.cpp, supplies its own overloads for its counting type.)
#if defined(__CUDACC__)
KF_D float recip(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
KF_D double recip(double x) { return __drcp_rn(x); }
KF_D float ksqrt(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
KF_D double ksqrt(double x) { return sqrt(x); }
KF_D float klog(float x) { return __logf(x); }
KF_D double klog(double x) { return log(x); }
#endif

// X = (I + C J)^{-1} for packed symmetric C, J, by Gauss-Jordan elimination
// with partial pivoting in precision T.  Returns sum log|pivot| = log det(I + C J)
// in `logdet` when LD (det(I + C J) >= 1 for positive semi-definite C, J).
template <int N, typename T, bool LD, typename RC, typename RJ>
KF_D void inv_I_plus_CJ_T(const RC *C, const RJ *J, T X[N * N], T &logdet) {
    T a[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            T s = (r == c) ? T(1) : T(0);
#pragma unroll
            for (int k = 0; k < N; ++k) s += T(C[si(N, r, k)]) * T(J[si(N, k, c)]);
            a[r * N + c] = s;
            X[r * N + c] = (r == c) ? T(1) : T(0);
        }
#pragma unroll
    for (int c = 0; c < N; ++c) {
        int p = c;
        T best = fabs(a[c * N + c]);
#pragma unroll
        for (int r = c + 1; r < N; ++r) {
            T v = fabs(a[r * N + c]);
            if (v > best) { best = v; p = r; }
        }
#pragma unroll
        for (int r = c + 1; r < N; ++r) {
            const bool s = (p == r);
#pragma unroll
            for (int j = c; j < N; ++j) {
                T u = a[c * N + j], w = a[r * N + j];
                a[c * N + j] = s ? w : u;
                a[r * N + j] = s ? u : w;
            }
#pragma unroll
            for (int j = 0; j < N; ++j) {
                T u = X[c * N + j], w = X[r * N + j];
                X[c * N + j] = s ? w : u;
                X[r * N + j] = s ? u : w;
            }
        }
        const T piv = a[c * N + c];
        if (LD) logdet += klog(fabs(piv));
        const T d = recip(piv);
#pragma unroll
        for (int j = c + 1; j < N; ++j) a[c * N + j] *= d;
#pragma unroll
        for (int j = 0; j < N; ++j) X[c * N + j] *= d;
#pragma unroll
        for (int r = 0; r < N; ++r) {
            if (r == c) continue;
            const T f = a[r * N + c];
#pragma unroll
            for (int j = c + 1; j < N; ++j) a[r * N + j] -= f * a[c * N + j];
#pragma unroll
            for (int j = 0; j < N; ++j) X[r * N + j] -= f * X[c * N + j];
        }
    }
}

// Solve-precision policy.  MODE 0: everything in R.  MODE 1 (R = float):
// Gauss-Jordan in FP32, then one step of iterative refinement with the
// residual E = I - M X formed in FP64 from M = I + C J built in FP64, and
// the correction X <- X + X E applied in FP32; log det in FP64.
template <int N, typename R, int MODE, bool LD>
KF_D void inv_I_plus_CJ(const R *C, const R *J, R X[N * N], double &logdet) {
    if constexpr (MODE == 0) {
        R ld = 0;
        inv_I_plus_CJ_T<N, R, LD>(C, J, X, ld);
        if (LD) logdet += double(ld);
    } else {
        static_assert(sizeof(R) == 4, "the refined solve is for FP32 elements");
        R ld = 0;
        inv_I_plus_CJ_T<N, R, false>(C, J, X, ld);
        double Md[N * N];
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c < N; ++c) {
                double s = (r == c) ? 1.0 : 0.0;
#pragma unroll
                for (int k = 0; k < N; ++k) s += double(C[si(N, r, k)]) * double(J[si(N, k, c)]);
                Md[r * N + c] = s;
            }
        R E[N * N];
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c < N; ++c) {
                double s = (r == c) ? 1.0 : 0.0;
#pragma unroll
                for (int k = 0; k < N; ++k) s -= Md[r * N + k] * double(X[k * N + c]);
                E[r * N + c] = R(s);
            }
        R Xn[N * N];
#pragma unroll
        for (int r = 0; r < N; ++r)
#pragma unroll
            for (int c = 0; c < N; ++c) {
                R s = X[r * N + c];
#pragma unroll
                for (int k = 0; k < N; ++k) s += X[r * N + k] * E[k * N + c];
                Xn[r * N + c] = s;
            }
#pragma unroll
        for (int i = 0; i < N * N; ++i) X[i] = Xn[i];
        if constexpr (LD) {
            // log det M by an FP64 LU of M without refinement: M is only N x N
            double a[N * N];
#pragma unroll
            for (int i = 0; i < N * N; ++i) a[i] = Md[i];
            double l = 0;
#pragma unroll
            for (int c = 0; c < N; ++c) {
                int p = c;
                double best = fabs(a[c * N + c]);
#pragma unroll
                for (int r = c + 1; r < N; ++r) {
                    double v = fabs(a[r * N + c]);
                    if (v > best) { best = v; p = r; }
                }
#pragma unroll
                for (int r = c + 1; r < N; ++r) {
                    const bool s = (p == r);
#pragma unroll
                    for (int j = c; j < N; ++j) {
                        double u = a[c * N + j], w = a[r * N + j];
                        a[c * N + j] = s ? w : u;
                        a[r * N + j] = s ? u : w;
                    }
                }
                const double piv = a[c * N + c];
                l += log(fabs(piv));
                const double d = 1.0 / piv;
#pragma unroll
                for (int r = c + 1; r < N; ++r) {
                    const double f = a[r * N + c] * d;
#pragma unroll
                    for (int j = c + 1; j < N; ++j) a[r * N + j] -= f * a[c * N + j];
                }
            }
            logdet += l;
        }
    }
}

// ---------------------------------------------------------------- Lemma 1

// Full operator of Lemma 1: o = ei (x) ej (ei earlier in time).
//   X = (I + C_i J_j)^{-1},  Z = X A_i
//   A_ij = A_j Z
//   b_ij = A_j X (b_i + C_i eta_j) + b_j
//   C_ij = A_j D A_j^T + C_j,  D = X C_i (symmetric)
//   eta_ij = Z^T (eta_j - J_j b_i) + eta_i         [A_i^T (I + J_j C_i)^{-1} = Z^T]
//   J_ij = Z^T (J_j A_i) + J_i
template <int N, typename R, int MODE>
KF_D void lemma1(const FElem<N, R> &ei, const FElem<N, R> &ej, FElem<N, R> &o) {
    using E = FElem<N, R>;
    const R *Ai = ei.v + E::oA, *bi = ei.v + E::ob, *Ci = ei.v + E::oC, *ei_ = ei.v + E::oe, *Ji = ei.v + E::oJ;
    const R *Aj = ej.v + E::oA, *bj = ej.v + E::ob, *Cj = ej.v + E::oC, *ej_ = ej.v + E::oe, *Jj = ej.v + E::oJ;
    R X[N * N];
    double ld = 0;
    inv_I_plus_CJ<N, R, MODE, false>(Ci, Jj, X, ld);
    R Z[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += X[r * N + k] * Ai[k * N + c];
            Z[r * N + c] = s;
        }
    // b
    R t[N], u[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = bi[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += Ci[si(N, r, k)] * ej_[k];
        t[r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) s += X[r * N + k] * t[k];
        u[r] = s;
    }
    // D = X C_i (upper), AD = A_j D
    R D[N * (N + 1) / 2];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += X[r * N + k] * Ci[si(N, k, c)];
            D[su(N, r, c)] = s;
        }
    R AD[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += Aj[r * N + k] * D[si(N, k, c)];
            AD[r * N + c] = s;
        }
    // eta: w = eta_j - J_j b_i
    R w[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = ej_[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s -= Jj[si(N, r, k)] * bi[k];
        w[r] = s;
    }
    // W = J_j A_i
    R W[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += Jj[si(N, r, k)] * Ai[k * N + c];
            W[r * N + c] = s;
        }
    // outputs
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += Aj[r * N + k] * Z[k * N + c];
            o.v[E::oA + r * N + c] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = bj[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += Aj[r * N + k] * u[k];
        o.v[E::ob + r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            R s = Cj[su(N, r, c)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += AD[r * N + k] * Aj[c * N + k];
            o.v[E::oC + su(N, r, c)] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = ei_[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += Z[k * N + r] * w[k];
        o.v[E::oe + r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            R s = Ji[su(N, r, c)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += Z[k * N + r] * W[k * N + c];
            o.v[E::oJ + su(N, r, c)] = s;
        }
}

// (b, C) half of Lemma 1 with the carry on the left: c <- c (x) ej.
// When LL, also returns the pieces of the innovation log-likelihood:
// logdet(I + C J_j) and w^T D w with w = eta_j - J_j b, D = (I + C J_j)^{-1} C.
template <int N, typename R, int MODE, bool LL>
KF_D void apply_fwd(FwdCarry<N, R> &c, const FElem<N, R> &ej, double *ll_logdet, R *ll_wDw) {
    using E = FElem<N, R>;
    using CT = FwdCarry<N, R>;
    const R *b = c.v + CT::ob, *C = c.v + CT::oC;
    const R *Aj = ej.v + E::oA, *bj = ej.v + E::ob, *Cj = ej.v + E::oC, *ej_ = ej.v + E::oe, *Jj = ej.v + E::oJ;
    R X[N * N];
    double ld = 0;
    inv_I_plus_CJ<N, R, MODE, LL>(C, Jj, X, ld);
    R D[N * (N + 1) / 2];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = r; q < N; ++q) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += X[r * N + k] * C[si(N, k, q)];
            D[su(N, r, q)] = s;
        }
    // u = X (b + C eta_j) = X b + D eta_j
    R u[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) s += X[r * N + k] * b[k] + D[si(N, r, k)] * ej_[k];
        u[r] = s;
    }
    if (LL) {
        R w[N];
#pragma unroll
        for (int r = 0; r < N; ++r) {
            R s = ej_[r];
#pragma unroll
            for (int k = 0; k < N; ++k) s -= Jj[si(N, r, k)] * b[k];
            w[r] = s;
        }
        R q = 0;
#pragma unroll
        for (int r = 0; r < N; ++r) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += D[si(N, r, k)] * w[k];
            q += w[r] * s;
        }
        *ll_wDw = q;
        *ll_logdet = ld;
    }
    R AD[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = 0; q < N; ++q) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += Aj[r * N + k] * D[si(N, k, q)];
            AD[r * N + q] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = bj[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += Aj[r * N + k] * u[k];
        c.v[CT::ob + r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = r; q < N; ++q) {
            R s = Cj[su(N, r, q)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += AD[r * N + k] * Aj[q * N + k];
            c.v[CT::oC + su(N, r, q)] = s;
        }
}

// (eta, J) half of Lemma 1 with the carry on the right: c <- ei (x) c.
template <int N, typename R, int MODE>
KF_D void apply_rev(RevCarry<N, R> &c, const FElem<N, R> &ei) {
    using E = FElem<N, R>;
    using CT = RevCarry<N, R>;
    const R *eta = c.v + CT::oe, *J = c.v + CT::oJ;
    const R *Ai = ei.v + E::oA, *bi = ei.v + E::ob, *Ci = ei.v + E::oC, *ei_ = ei.v + E::oe, *Ji = ei.v + E::oJ;
    R X[N * N];
    double ld = 0;
    inv_I_plus_CJ<N, R, MODE, false>(Ci, J, X, ld);
    R Z[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = 0; q < N; ++q) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += X[r * N + k] * Ai[k * N + q];
            Z[r * N + q] = s;
        }
    R w[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = eta[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s -= J[si(N, r, k)] * bi[k];
        w[r] = s;
    }
    R W[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = 0; q < N; ++q) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += J[si(N, r, k)] * Ai[k * N + q];
            W[r * N + q] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = ei_[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += Z[k * N + r] * w[k];
        c.v[CT::oe + r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = r; q < N; ++q) {
            R s = Ji[su(N, r, q)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += Z[k * N + r] * W[k * N + q];
            c.v[CT::oJ + su(N, r, q)] = s;
        }
}


// ---------------------------------------------------------------- low-rank path
//
// For a fresh filtering element a_k the information matrix has rank m:
// J_k = F^T H^T S^{-1} H F = U^T U with U = L^{-1} H F (m x n), S = L L^T.
// By the Woodbury identity
//     (I + C U^T U)^{-1} = I - C U^T W U,   W = (I_m + U C U^T)^{-1},
// where I_m + U C U^T is m x m symmetric positive definite with eigenvalues
// >= 1, so W needs no pivoting; with G = U C (so C U^T = G^T):
//     X C   = C - G^T W G               (symmetric)
//     X A   = A - G^T W (U A)
//     X v   = v - G^T W (U v)
// and, by Sylvester's determinant identity, det(I + C J_k) = det(I_m + U C U^T).

// Inverse and log-determinant of a small SPD matrix given by its packed
// upper triangle (M = 1, 2 closed forms; larger M by Cholesky).
template <int M, typename T>
KF_D void spd_inverse(const T *Pp, T *W, T &logdet) {
    if constexpr (M == 1) {
        W[0] = recip(Pp[0]);
        logdet = klog(Pp[0]);
    } else if constexpr (M == 2) {
        const T det = Pp[0] * Pp[2] - Pp[1] * Pp[1];
        const T r = recip(det);
        W[0] = Pp[2] * r;
        W[1] = -Pp[1] * r;
        W[2] = Pp[0] * r;
        logdet = klog(det);
    } else {
        T L[M * (M + 1) / 2], dinv[M];
        T ld = 0;
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) {
                T s = Pp[su(M, j, i)];
#pragma unroll
                for (int k = 0; k < j; ++k) s -= L[i * (i + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
                if (i == j) {
                    const T d = ksqrt(s);
                    L[i * (i + 1) / 2 + i] = d;
                    dinv[i] = recip(d);
                    ld += klog(s);
                } else {
                    L[i * (i + 1) / 2 + j] = s * dinv[j];
                }
            }
        // Linv (lower), then W = Linv^T Linv
        T Li[M * M];
#pragma unroll
        for (int c = 0; c < M; ++c)
#pragma unroll
            for (int i = 0; i < M; ++i) {
                if (i < c) {
                    Li[i * M + c] = 0;
                    continue;
                }
                T s = (i == c) ? T(1) : T(0);
#pragma unroll
                for (int k = 0; k < i; ++k)
                    if (k >= c) s -= L[i * (i + 1) / 2 + k] * Li[k * M + c];
                Li[i * M + c] = s * dinv[i];
            }
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = i; j < M; ++j) {
                T s = 0;
#pragma unroll
                for (int k = 0; k < M; ++k) s += Li[k * M + i] * Li[k * M + j];
                W[su(M, i, j)] = s;
            }
        logdet = ld;
    }
}

// G = U C (M x N), W = (I_M + G U^T)^{-1} (packed M x M) and log det of it.
// MODE 1 forms I + G U^T and inverts it in FP64, then applies one step of
// iterative refinement W <- W + W (I - P W) in FP64.
template <int N, int M, typename R, int MODE, typename LD>
KF_D void lowrank_core(const R *C, const R *U, R G[M * N], R Wp[M * (M + 1) / 2], LD &logdet) {
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += U[i * N + k] * C[si(N, k, c)];
            G[i * N + c] = s;
        }
    if constexpr (MODE == 0) {
        R Pp[M * (M + 1) / 2];
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = i; j < M; ++j) {
                R s = (i == j) ? R(1) : R(0);
#pragma unroll
                for (int k = 0; k < N; ++k) s += G[i * N + k] * U[j * N + k];
                Pp[su(M, i, j)] = s;
            }
        R ld;
        spd_inverse<M, R>(Pp, Wp, ld);
        logdet = LD(ld);
    } else {
        double Pp[M * (M + 1) / 2], Wd[M * (M + 1) / 2];
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = i; j < M; ++j) {
                double s = (i == j) ? 1.0 : 0.0;
#pragma unroll
                for (int k = 0; k < N; ++k) s += double(G[i * N + k]) * double(U[j * N + k]);
                Pp[su(M, i, j)] = s;
            }
        double ld;
        spd_inverse<M, double>(Pp, Wd, ld);
        // refinement: E = I - P W, W <- W + W E (symmetric result)
        double E[M * M];
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = 0; j < M; ++j) {
                double t = (i == j) ? 1.0 : 0.0;
#pragma unroll
                for (int k = 0; k < M; ++k) t -= Pp[si(M, i, k)] * Wd[si(M, k, j)];
                E[i * M + j] = t;
            }
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int j = i; j < M; ++j) {
                double t = Wd[su(M, i, j)];
#pragma unroll
                for (int k = 0; k < M; ++k) t += Wd[si(M, i, k)] * E[k * M + j];
                Wp[su(M, i, j)] = R(t);
            }
        logdet = LD(ld);
    }
}

// Lemma 1, ei (x) ej, for a fresh right operand ej whose J is U^T U.
// Fresh right operand given by its parts: A_j, C_j (packed), U from the model
// constants, b_j and eta_j from registers.
template <int N, int M, typename R, int MODE>
KF_D void lemma1_lr_parts(const FElem<N, R> &ei, const R *Aj, const R *bj, const R *Cj, const R *etaj, const R *U,
                          FElem<N, R> &o) {
    using E = FElem<N, R>;
    constexpr int SM = M * (M + 1) / 2;
    const R *Ai = ei.v + E::oA, *bi = ei.v + E::ob, *Ci = ei.v + E::oC, *etai = ei.v + E::oe, *Ji = ei.v + E::oJ;
    R G[M * N], W[SM];
    R ld;
    lowrank_core<N, M, R, MODE, R>(Ci, U, G, W, ld);
    // WG = W G; D = C_i - G^T W G
    R WG[M * N];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < M; ++k) s += W[si(M, i, k)] * G[k * N + c];
            WG[i * N + c] = s;
        }
    R D[N * (N + 1) / 2];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            R s = Ci[su(N, r, c)];
#pragma unroll
            for (int k = 0; k < M; ++k) s -= G[k * N + r] * WG[k * N + c];
            D[su(N, r, c)] = s;
        }
    // UA = U A_i, WUA = W UA, Z = A_i - G^T WUA  (= X A_i)
    R UA[M * N], WUA[M * N];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += U[i * N + k] * Ai[k * N + c];
            UA[i * N + c] = s;
        }
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < M; ++k) s += W[si(M, i, k)] * UA[k * N + c];
            WUA[i * N + c] = s;
        }
    R Z[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = Ai[r * N + c];
#pragma unroll
            for (int k = 0; k < M; ++k) s -= G[k * N + r] * WUA[k * N + c];
            Z[r * N + c] = s;
        }
    // Ub = U b_i; u = b_i - G^T W Ub + D eta_j  (= X (b_i + C_i eta_j))
    R Ub[M], WUb[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) s += U[i * N + k] * bi[k];
        Ub[i] = s;
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < M; ++k) s += W[si(M, i, k)] * Ub[k];
        WUb[i] = s;
    }
    R u[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = bi[r];
#pragma unroll
        for (int k = 0; k < M; ++k) s -= G[k * N + r] * WUb[k];
#pragma unroll
        for (int k = 0; k < N; ++k) s += D[si(N, r, k)] * etaj[k];
        u[r] = s;
    }
    // w = eta_j - U^T Ub  (= eta_j - J_j b_i);  Wj = U^T UA  (= J_j A_i)
    R w[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = etaj[r];
#pragma unroll
        for (int k = 0; k < M; ++k) s -= U[k * N + r] * Ub[k];
        w[r] = s;
    }
    R AD[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += Aj[r * N + k] * D[si(N, k, c)];
            AD[r * N + c] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += Aj[r * N + k] * Z[k * N + c];
            o.v[E::oA + r * N + c] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = bj[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += Aj[r * N + k] * u[k];
        o.v[E::ob + r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            R s = Cj[su(N, r, c)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += AD[r * N + k] * Aj[c * N + k];
            o.v[E::oC + su(N, r, c)] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = etai[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += Z[k * N + r] * w[k];
        o.v[E::oe + r] = s;
    }
    R Wj[N * N];
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int q = 0; q < M; ++q) s += U[q * N + k] * UA[q * N + c];
            Wj[k * N + c] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            R s = Ji[su(N, r, c)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += Z[k * N + r] * Wj[k * N + c];
            o.v[E::oJ + su(N, r, c)] = s;
        }
}

template <int N, int M, typename R, int MODE>
KF_D void lemma1_lr(const FElem<N, R> &ei, const FElem<N, R> &ej, const R *U, FElem<N, R> &o) {
    using E = FElem<N, R>;
    lemma1_lr_parts<N, M, R, MODE>(ei, ej.v + E::oA, ej.v + E::ob, ej.v + E::oC, ej.v + E::oe, U, o);
}

// (b, C) half of Lemma 1 for a fresh right operand: c <- c (x) ej.  With LL
// it also returns, for ytil = L^{-1} y_k, the whitened innovation
// vt = ytil - U b (before the update) and vt^T W vt and log det(I_m + U C U^T),
// which give log N(y_k; H F b, S_k) since S_k = L (I_m + U C U^T) L^T.
template <int N, int M, typename R, int MODE, bool LL>
KF_D void apply_fwd_lr_parts(FwdCarry<N, R> &c, const R *Aj, const R *bj, const R *Cj, const R *etaj, const R *U,
                             const R *ytil, R *quad, R *logdet) {
    using CT = FwdCarry<N, R>;
    const R *b = c.v + CT::ob, *C = c.v + CT::oC;
    R G[M * N], W[M * (M + 1) / 2];
    R ld;
    lowrank_core<N, M, R, MODE, R>(C, U, G, W, ld);
    R WG[M * N];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int q = 0; q < N; ++q) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < M; ++k) s += W[si(M, i, k)] * G[k * N + q];
            WG[i * N + q] = s;
        }
    R D[N * (N + 1) / 2];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = r; q < N; ++q) {
            R s = C[su(N, r, q)];
#pragma unroll
            for (int k = 0; k < M; ++k) s -= G[k * N + r] * WG[k * N + q];
            D[su(N, r, q)] = s;
        }
    R Ub[M], WUb[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) s += U[i * N + k] * b[k];
        Ub[i] = s;
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < M; ++k) s += W[si(M, i, k)] * Ub[k];
        WUb[i] = s;
    }
    if constexpr (LL) {
        R vt[M], q = 0;
#pragma unroll
        for (int i = 0; i < M; ++i) vt[i] = ytil[i] - Ub[i];
#pragma unroll
        for (int i = 0; i < M; ++i)
#pragma unroll
            for (int k = 0; k < M; ++k) q += vt[i] * W[si(M, i, k)] * vt[k];
        *quad = q;
        *logdet = ld;
    }
    R u[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = b[r];
#pragma unroll
        for (int k = 0; k < M; ++k) s -= G[k * N + r] * WUb[k];
#pragma unroll
        for (int k = 0; k < N; ++k) s += D[si(N, r, k)] * etaj[k];
        u[r] = s;
    }
    R AD[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = 0; q < N; ++q) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += Aj[r * N + k] * D[si(N, k, q)];
            AD[r * N + q] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = bj[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += Aj[r * N + k] * u[k];
        c.v[CT::ob + r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = r; q < N; ++q) {
            R s = Cj[su(N, r, q)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += AD[r * N + k] * Aj[q * N + k];
            c.v[CT::oC + su(N, r, q)] = s;
        }
}

template <int N, int M, typename R, int MODE, bool LL>
KF_D void apply_fwd_lr(FwdCarry<N, R> &c, const FElem<N, R> &ej, const R *U, const R *ytil, R *quad, R *logdet) {
    using E = FElem<N, R>;
    apply_fwd_lr_parts<N, M, R, MODE, LL>(c, ej.v + E::oA, ej.v + E::ob, ej.v + E::oC, ej.v + E::oe, U, ytil, quad,
                                          logdet);
}

// ---------------------------------------------------------------- Lemma 2

// o = ei (x) ej = (E_i E_j, E_i g_j + g_i, E_i L_j E_i^T + L_i).
template <int N, typename R>
KF_D void lemma2(const RElem<N, R> &ei, const RElem<N, R> &ej, RElem<N, R> &o) {
    using E = RElem<N, R>;
    const R *Ei = ei.v + E::oE, *gi = ei.v + E::og, *Li = ei.v + E::oL;
    const R *Ej = ej.v + E::oE, *gj = ej.v + E::og, *Lj = ej.v + E::oL;
    R EL[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += Ei[r * N + k] * Lj[si(N, k, c)];
            EL[r * N + c] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += Ei[r * N + k] * Ej[k * N + c];
            o.v[E::oE + r * N + c] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = gi[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += Ei[r * N + k] * gj[k];
        o.v[E::og + r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            R s = Li[su(N, r, c)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += EL[r * N + k] * Ei[c * N + k];
            o.v[E::oL + su(N, r, c)] = s;
        }
}

// (g, L) half of Lemma 2 with the carry on the right: c <- ei (x) c.
template <int N, typename R>
KF_D void apply_rts(RCarry<N, R> &c, const RElem<N, R> &ei) {
    using E = RElem<N, R>;
    using CT = RCarry<N, R>;
    const R *g = c.v + CT::og, *L = c.v + CT::oL;
    const R *Ei = ei.v + E::oE, *gi = ei.v + E::og, *Li = ei.v + E::oL;
    R EL[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = 0; q < N; ++q) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += Ei[r * N + k] * L[si(N, k, q)];
            EL[r * N + q] = s;
        }
    R gn[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = gi[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += Ei[r * N + k] * g[k];
        gn[r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = r; q < N; ++q) {
            R s = Li[su(N, r, q)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += EL[r * N + k] * Ei[q * N + k];
            c.v[CT::oL + su(N, r, q)] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r) c.v[CT::og + r] = gn[r];
}

// ---------------------------------------------------------------- element construction

// Filtering element a_k from y_k (k 1-based).  k = 1: Eq. pkf_init2
// (A_1 = 0); k >= 2: Eq. pkf_init1.  eta_k, J_k: Eq. pkf_init3.
template <int N, typename R>
KF_D void build_filter_elem(const FiltParams<N, R> &P, int64_t k, const R *yk, FElem<N, R> &e) {
    using E = FElem<N, R>;
    const int ny = P.ny;
    R y[MAXNY];
#pragma unroll
    for (int j = 0; j < MAXNY; ++j) y[j] = 0;
#pragma unroll
    for (int j = 0; j < MAXNY; ++j)
        if (j < ny) y[j] = yk[j];
    const bool first = (k == 1);
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R sb = first ? P.c1[r] : R(0), se = 0;
#pragma unroll
        for (int j = 0; j < MAXNY; ++j) {
            if (j < ny) {
                sb += (first ? P.K1[r * MAXNY + j] : P.K[r * MAXNY + j]) * y[j];
                se += P.G[r * MAXNY + j] * y[j];
            }
        }
        e.v[E::ob + r] = sb;
        e.v[E::oe + r] = se;
    }
#pragma unroll
    for (int i = 0; i < N * N; ++i) e.v[E::oA + i] = first ? R(0) : P.A[i];
#pragma unroll
    for (int i = 0; i < E::S; ++i) {
        e.v[E::oC + i] = first ? P.C1[i] : P.C[i];
        e.v[E::oJ + i] = P.J[i];
    }
}

// (b_k, eta_k) of a fresh element a_k, k >= 2 (Eq. pkf_init1, Eq. pkf_init3),
// for a compile-time number of measurements M: b_k = K y_k, eta_k = G y_k.
template <int N, int M, typename R>
KF_D void fresh_b_eta(const FiltParams<N, R> &P, const R *yk, R *b, R *eta) {
    R y[M];
#pragma unroll
    for (int j = 0; j < M; ++j) y[j] = yk[j];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R sb = 0, se = 0;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            sb += P.K[r * MAXNY + j] * y[j];
            se += P.G[r * MAXNY + j] * y[j];
        }
        b[r] = sb;
        eta[r] = se;
    }
}

// RTS element from the filtering mean x = xbar_{k|k} and packed covariance
// Pk = P_{k|k}: Eq. prts_init1 (last = false) or Eq. prts_init2 (last).
//   U = F P,  Pp = U F^T + Q = L L^T (Cholesky),  E = P F^T Pp^{-1} = (Pp^{-1} U)^T,
//   g = x - E F x,  L_k = P - E U.
template <int N, typename R>
KF_D void build_rts_elem(const FiltParams<N, R> &P, bool last, const R *x, const R *Pk, RElem<N, R> &e) {
    using E = RElem<N, R>;
    if (last) {
#pragma unroll
        for (int i = 0; i < N * N; ++i) e.v[E::oE + i] = 0;
#pragma unroll
        for (int i = 0; i < N; ++i) e.v[E::og + i] = x[i];
#pragma unroll
        for (int i = 0; i < E::S; ++i) e.v[E::oL + i] = Pk[i];
        return;
    }
    R U[N * N];
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += P.F[r * N + k] * Pk[si(N, k, c)];
            U[r * N + c] = s;
        }
    // lower Cholesky factor of Pp, packed by rows (row i holds columns 0..i)
    R L[N * (N + 1) / 2];
    R dinv[N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            R s = P.Q[su(N, j, i)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += U[i * N + k] * P.F[j * N + k];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[i * (i + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
            if (i == j) {
                const R d = ksqrt(s);
                L[i * (i + 1) / 2 + i] = d;
                dinv[i] = recip(d);
            } else {
                L[i * (i + 1) / 2 + j] = s * dinv[j];
            }
        }
    // Et = Pp^{-1} U: forward then backward substitution, column by column
    R Et[N * N];
#pragma unroll
    for (int c = 0; c < N; ++c) {
        R z[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            R s = U[i * N + c];
#pragma unroll
            for (int k = 0; k < i; ++k) s -= L[i * (i + 1) / 2 + k] * z[k];
            z[i] = s * dinv[i];
        }
#pragma unroll
        for (int i = N - 1; i >= 0; --i) {
            R s = z[i];
#pragma unroll
            for (int k = i + 1; k < N; ++k) s -= L[k * (k + 1) / 2 + i] * Et[k * N + c];
            Et[i * N + c] = s * dinv[i];
        }
    }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) e.v[E::oE + r * N + c] = Et[c * N + r];
    R Fx[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) s += P.F[r * N + k] * x[k];
        Fx[r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = x[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s -= Et[k * N + r] * Fx[k];
        e.v[E::og + r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            R s = Pk[su(N, r, c)];
#pragma unroll
            for (int k = 0; k < N; ++k) s -= Et[k * N + r] * U[k * N + c];
            e.v[E::oL + su(N, r, c)] = s;
        }
}

// Two-filter merge, Eqs. mean_tf_combination / cov_tf_combination:
//   Xm = (I + P J)^{-1},  ms = Xm (x + P eta),  Ps = Xm P (symmetric).
template <int N, typename R, int MODE>
KF_D void tf_merge(const R *x, const R *Pk, const RevCarry<N, R> &c, R *ms, R *Ps_packed) {
    using CT = RevCarry<N, R>;
    const R *eta = c.v + CT::oe, *J = c.v + CT::oJ;
    R X[N * N];
    double ld = 0;
    inv_I_plus_CJ<N, R, MODE, false>(Pk, J, X, ld);
    R t[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = x[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += Pk[si(N, r, k)] * eta[k];
        t[r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) s += X[r * N + k] * t[k];
        ms[r] = s;
    }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int q = r; q < N; ++q) {
            R s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += X[r * N + k] * Pk[si(N, k, q)];
            Ps_packed[su(N, r, q)] = s;
        }
}

}  // namespace kfs
