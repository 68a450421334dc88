// flop_count.cpp -- flops per time step of the one-sequence kernels, counted
// from their own step code: the functions of kf_steps.cuh instantiated on the
// host with a number type that counts its operations.  Each binary +, -, x
// counts one flop (so a multiply-add counts two), each reciprocal, square
// root and log one; a sign change counts none.  Compiled by the host
// compiler (no device code) and linked into the library.
#include <mutex>

#include "kf_math.cuh"
#include "kfscan.h"

namespace {

struct Counts {
    long long add, mul, rcp, sqr, lg;
};
Counts g_c;
std::mutex g_mu;

struct Cnt {
    double v;
    Cnt(double x = 0.0) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_c.add; return a.v + b.v; }
inline Cnt operator-(Cnt a, Cnt b) { ++g_c.add; return a.v - b.v; }
inline Cnt operator*(Cnt a, Cnt b) { ++g_c.mul; return a.v * b.v; }
inline Cnt operator-(Cnt a) { return -a.v; }
inline Cnt &operator+=(Cnt &a, Cnt b) { ++g_c.add; a.v += b.v; return a; }
inline Cnt &operator-=(Cnt &a, Cnt b) { ++g_c.add; a.v -= b.v; return a; }
inline Cnt &operator*=(Cnt &a, Cnt b) { ++g_c.mul; a.v *= b.v; return a; }
inline bool operator>(Cnt a, Cnt b) { return a.v > b.v; }
inline bool operator==(Cnt a, Cnt b) { return a.v == b.v; }
// found by argument-dependent lookup from the step templates
inline Cnt recip(Cnt a) { ++g_c.rcp; return 1.0 / a.v; }
inline Cnt ksqrt(Cnt a) { ++g_c.sqr; return a.v > 0 ? __builtin_sqrt(a.v) : 0.0; }
inline Cnt klog(Cnt a) { ++g_c.lg; return a.v > 0 ? __builtin_log(a.v) : 0.0; }

}  // namespace

#include "kf_steps.cuh"

namespace {

// A positive definite test point for the arithmetic (the values only keep
// the square roots and logs finite; the counts do not depend on them).
template <int N>
void fill(kfs::FiltParams<N, Cnt> &P, Cnt *row, Cnt *rec, Cnt *y) {
    constexpr int S = N * (N + 1) / 2;
    for (int i = 0; i < N * N; ++i) {
        P.A[i] = P.F[i] = (i % (N + 1) == 0) ? 1.0 : 0.01;
    }
    for (int r = 0; r < N; ++r)
        for (int c = r; c < N; ++c) {
            const double d = r == c ? 1.0 : 0.0;
            P.C[kfs::su(N, r, c)] = P.Q[kfs::su(N, r, c)] = P.J[kfs::su(N, r, c)] = d;
            rec[N + kfs::su(N, r, c)] = d;
        }
    for (int i = 0; i < kfs::MAXNY * N; ++i) P.K[i] = P.G[i] = P.U[i] = 0.1;
    for (int i = 0; i < kfs::MAXNY * kfs::MAXNY; ++i) P.Linv[i] = (i % (kfs::MAXNY + 1) == 0) ? 1.0 : 0.0;
    P.llc_r = 1.0;
    for (int i = 0; i < N * N + N * N; ++i) row[i] = 0.01;
    for (int i = 0; i < N; ++i) rec[i] = y[i] = 1.0;
    (void)S;
}

template <int N>
bool count_step(int what, Counts &out) {
    constexpr int M = N / 2;
    kfs::FiltParams<N, Cnt> P;
    Cnt row[2 * N * N], rec[N + N * (N + 1) / 2], y[N];
    fill<N>(P, row, rec, y);
    Cnt b[N], e[N], g[N], L[N * (N + 1) / 2], Ea[N * N];
    for (int i = 0; i < N; ++i) b[i] = e[i] = g[i] = 0.5;
    for (int i = 0; i < N * (N + 1) / 2; ++i) L[i] = rec[N + i];
    for (int i = 0; i < N * N; ++i) Ea[i] = P.F[i];
    kfs::FwdCarry<N, Cnt> c;
    for (int i = 0; i < N; ++i) c.v[i] = 0.5;
    for (int i = 0; i < N * (N + 1) / 2; ++i) c.v[N + i] = rec[N + i];
    g_c = Counts{0, 0, 0, 0, 0};
    switch (what) {
        case 0: kfs::ti_fold_step<N, M, Cnt>(P, row, y, b, e); break;
        case 1: kfs::ti_carry_step<N, M, Cnt, false>(P, y, c); break;
        case 2: kfs::ti_carry_step<N, M, Cnt, true>(P, y, c); break;
        case 3: kfs::rs_fold_step<N, Cnt>(P.F, P.Q, false, rec, Ea, g, L); break;
        case 4: kfs::rs_carry_step<N, Cnt>(P.F, P.Q, false, rec, g, L); break;
        default: return false;
    }
    out = g_c;
    return true;
}

}  // namespace

extern "C" kf_status_t kf_count_step_flops(int nx, int step, int64_t *counts) {
    if (!counts || (nx != 2 && nx != 4)) return KF_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    Counts c;
    const bool ok = nx == 2 ? count_step<2>(step, c) : count_step<4>(step, c);
    if (!ok) return KF_ERR_ARG;
    counts[0] = c.add + c.mul + c.rcp + c.sqr + c.lg;
    counts[1] = c.add;
    counts[2] = c.mul;
    counts[3] = c.rcp;
    counts[4] = c.sqr;
    counts[5] = c.lg;
    return KF_OK;
}
