// ti_filter.cuh -- the forward filter scan of Alg. pkf for a time-invariant
// model whose measurement has ny = nx / 2 components, on one sequence: a
// single-pass decoupled look-back scan in which every quantity that does not
// depend on the data comes from tables the host computes in FP64.
//
// Structure (Sec. IV-C, Lemma 1).  Every fresh element a_k, k >= 2, has the
// same (A, C, J) (Eqs. pkf_init1, pkf_init3), so the (A, C, J) half of any
// run of fresh elements depends on the run's length only, and Lemma 1 acts
// on the (b, eta) half of such runs through coefficient matrices of the run
// lengths.  The element a_1 (A_1 = 0, Eq. pkf_init2) is taken as the initial
// carry s_1 = (xbar_{1|1}, P_{1|1}); the scan runs over a_2 .. a_T, scan
// position p being time k = p + 2 (record p + 1).  A CTA scans a tile of
// THREADS x K positions:
//   1. tile ticket (atomic counter): a CTA waits only for tiles already
//      claimed by running CTAs;
//   2. thread fold: each thread folds its K elements through the fold table,
//      b <- T1_c b + T4_c y_k, eta <- eta + T3U_c (L^{-1} y_k - U b);
//   3. warp scan and warp-aggregate scan of the (b, eta) halves: a left run
//      of p and a right run of s thread aggregates combine as
//      b <- M1 b_x + M2 eta_y + b_y, eta <- eta_x + M3 eta_y - M4 b_x with
//      M1 = A_s X, M2 = A_s X C_p, M3 = A_p^T X^T, M4 = M3 J_s,
//      X = (I + C_p J_s)^{-1};
//   4. with the carry covariance at the tile's start known to the host, the
//      tile acts on the carry mean as an affine map, b_i = X_i b_{i-1} + u_i,
//      u_i = Y_i eta_agg + b_agg (X_i = A_T (I + C_{i-1} J_T)^{-1},
//      Y_i = X_i C_{i-1}); the tile publishes u_i (tile 0: with X_0 b_1);
//   5. look-back: the maps of all preceding tiles, composed in order by a
//      tree, give the tile's carry mean -- no chain of inclusive prefixes;
//   6. every thread applies its warp's and its own exclusive run to the tile
//      carry (one-sided Lemma 1 in the Cholesky form of apply_run_chol), then
//      walks its K elements with the rank-ny carry update (apply_fwd_lr_parts),
//      and adds its log-likelihood terms; each warp writes the filter records
//      of its 32 runs chunk by chunk through shared memory, as coalesced
//      16-byte stores (per run, the records of a chunk are contiguous).
// Every wait is bounded by a wall-clock limit; on time-out the CTA records
// the time-out in the status word and returns.
#pragma once

#include "kf_problems.cuh"
#include "kf_steps.cuh"
#include "stage.cuh"

namespace kfs {

// Layout of the device tables (values of type R; each region starts on a
// 16-byte boundary).
template <int N, typename R>
struct TiTab {
    static constexpr int M = N / 2, NN = N * N, S = N * (N + 1) / 2;
    static constexpr int E = NN + 2 * N * M;    // fold row: T1 | T4 | T3U
    static constexpr int WE = 4 * NN;           // coefficient set: M1 | M2 | M3 | M4
    static constexpr int Q = 16 / int(sizeof(R));
    static constexpr int WES = WE + Q;          // its stride in shared memory: an odd number of
                                                // 16-byte units, so 16-byte loads of distinct sets
                                                // by the lanes of a quarter warp hit distinct banks
    static constexpr int NSETS = 31 + 7;        // warp level (s, p), then warp-aggregate level
    static constexpr int PE = NN + 2 * S;       // run of c thread aggregates: A | C | J (packed)
    static constexpr int NSPAN = 40;            // c = 0 .. 32, then 32 w for w = 2 .. 8
    static constexpr int TE = 2 * S + 2 * NN;   // tile: C_{i-1} | chol(C_{i-1}) | X_i | Y_i
    static constexpr int TES = (TE + Q - 1) / Q * Q;
    static constexpr int UP = (N + Q - 1) / Q * Q;   // published u_i, padded to 16 bytes
    static KF_HD int wset(int s, int p) { return s + p - 2; }
    static KF_HD int vset(int s, int p) { return 31 + s + p - 2; }
    static KF_HD int span(int c) { return c <= 32 ? c : 31 + c / 32; }
    static KF_HD int al(int x) { return (x + Q - 1) / Q * Q; }
};

template <int N, typename R>
struct TiArgs {
    FiltParams<N, R> prm;
    int64_t T;            // time steps (records)
    const R *y;           // [T][ny]
    R *frec;              // filter records [T][FRec] or null
    R *mf, *Pf;           // optional [T][N], [T][N][N]
    const R *tab;         // device tables (TiTab layout)
    int off_rows, off_sets, off_spans, off_tiles;
    int K, ntiles, lbw, want_ll;
    int *counters;        // [0] tile ticket, [1] finished tiles
    int *flags;           // [ntiles] 1 = u_i published
    R *ubuf;              // [ntiles][UP]
    double *ll_part;      // [ntiles]
    double *ll_out;
    int *status;
    int64_t timeout_ns;
    int inject_skip_tile;
    uint64_t *trace;
    int trace_cap;
};

// ---------------------------------------------------------------- flags

KF_D int ti_ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
KF_D void ti_st_release(int *p, int v) { asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory"); }
KF_D uint64_t ti_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- small dense helpers

// packed lower-triangular index (row i, column j <= i)
KF_HD constexpr int lo(int i, int j) { return i * (i + 1) / 2 + j; }

// Cholesky factor (packed lower) of a packed symmetric positive definite
// matrix, and the reciprocals of its diagonal.  A pivot that rounding made
// non-positive is replaced by the smallest normal number, so the factor
// stays finite.
template <int N, typename R>
KF_D void chol_lo(const R *Ap, R *L, R *dinv) {
    const R tiny = sizeof(R) == 4 ? R(1.17549435e-38f) : R(2.2250738585072014e-308);
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            R s = Ap[su(N, j, i)];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[lo(i, k)] * L[lo(j, k)];
            if (i == j) {
                const R d = ksqrt(s > tiny ? s : tiny);
                L[lo(i, i)] = d;
                dinv[i] = recip(d);
            } else {
                L[lo(i, j)] = s * dinv[j];
            }
        }
}

// One-sided Lemma 1: the carry (b, C) extended by a run with (A, bs, Cs, es,
// J), where the carry covariance is given by its Cholesky factor C = L L^T.
// With Z = I + L^T J L = L2 L2^T (eigenvalues >= 1, so the factorisation
// needs no pivoting), (I + C J)^{-1} = L Z^{-1} L^{-1} and
//   C' = A (I + C J)^{-1} C A^T + Cs = G G^T + Cs,             G = A L L2^{-T},
//   b' = A (I + C J)^{-1} (b + C es) + bs = G L2^{-1} (L^{-1} b + L^T es) + bs.
template <int N, typename R>
KF_D void apply_run_chol(const R *L, const R *Ldinv, const R *b, const R *A, const R *bs, const R *Cs, const R *es,
                         const R *J, R *bo, R *Co) {
    constexpr int S = N * (N + 1) / 2;
    R JL[N * N];   // J L
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = c; k < N; ++k) s += J[si(N, r, k)] * L[lo(k, c)];
            JL[r * N + c] = s;
        }
    R Z[S];        // I + L^T J L
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            R s = (r == c) ? R(1) : R(0);
#pragma unroll
            for (int k = r; k < N; ++k) s += L[lo(k, r)] * JL[k * N + c];
            Z[su(N, r, c)] = s;
        }
    R L2[S], d2[N];
    chol_lo<N, R>(Z, L2, d2);
    R G[N * N];    // A L, then solved against L2^T in place
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = 0; c < N; ++c) {
            R s = 0;
#pragma unroll
            for (int k = c; k < N; ++k) s += A[r * N + k] * L[lo(k, c)];
            G[r * N + c] = s;
        }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            R s = G[r * N + j];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= G[r * N + k] * L2[lo(j, k)];
            G[r * N + j] = s * d2[j];
        }
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int c = r; c < N; ++c) {
            R s = Cs[su(N, r, c)];
#pragma unroll
            for (int k = 0; k < N; ++k) s += G[r * N + k] * G[c * N + k];
            Co[su(N, r, c)] = s;
        }
    R z[N];        // L^{-1} b + L^T es, then L2^{-1} of it
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R s = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= L[lo(i, k)] * z[k];
        z[i] = s * Ldinv[i];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R s = z[i];
#pragma unroll
        for (int k = i; k < N; ++k) s += L[lo(k, i)] * es[k];
        z[i] = s;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        R s = z[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= L2[lo(i, k)] * z[k];
        z[i] = s * d2[i];
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R s = bs[r];
#pragma unroll
        for (int k = 0; k < N; ++k) s += G[r * N + k] * z[k];
        bo[r] = s;
    }
}

// (b, eta) <- (bx, ex) (x) (b, eta) with the coefficient set w (shared
// memory, 16-byte aligned), read row by row as vectors.
template <int N, typename R>
KF_D void ti_combine(const R *w, const R *bx, const R *ex, R *b, R *e) {
    constexpr int NN = N * N;
    R nb[N], ne[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R m1[N], m2[N], m3[N], m4[N];
        load_rec<N>(m1, w + r * N);
        load_rec<N>(m2, w + NN + r * N);
        load_rec<N>(m3, w + 2 * NN + r * N);
        load_rec<N>(m4, w + 3 * NN + r * N);
        R sb = b[r], se = ex[r];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            sb += m1[k] * bx[k] + m2[k] * e[k];
            se += m3[k] * e[k] - m4[k] * bx[k];
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

// y_k (M values) of record g, with the widest aligned read-only load.
template <int M, typename R>
KF_D void ti_load_y(const R *y, int64_t g, R *out) {
    const R *p = y + g * M;
    if constexpr (M * sizeof(R) == 16 && sizeof(R) == 8) {
        const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        out[0] = v.x; out[1] = v.y;
    } else if constexpr (M * sizeof(R) == 8 && sizeof(R) == 4) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        out[0] = v.x; out[1] = v.y;
    } else {
#pragma unroll
        for (int i = 0; i < M; ++i) out[i] = __ldg(p + i);
    }
}

// The (b, C) record of one step: filter record [m | packed P | 0], and the
// optional full outputs.
template <int N, typename R>
KF_D void ti_emit(const TiArgs<N, R> &a, int64_t g, const R *b, const R *C, R *srec) {
    constexpr int S = N * (N + 1) / 2, FR = FRec<N, R>::SIZE;
    if (srec) {
        R rec[FR];
#pragma unroll
        for (int i = 0; i < N; ++i) rec[i] = b[i];
#pragma unroll
        for (int i = 0; i < S; ++i) rec[N + i] = C[i];
#pragma unroll
        for (int i = N + S; i < FR; ++i) rec[i] = 0;
        store_rec<FR>(srec, rec);
    }
    if (!KF_IN(g >= 0 && g < a.T, a.status)) return;
    if (a.mf) store_rec<N>(a.mf + g * N, b);
    if (a.Pf) {
        R full[N * N];
        store_full<N>(full, C);
        store_rec<N * N>(a.Pf + g * N * N, full);
    }
}

// Per-warp shared memory of the staging: a ring of NST input buffers of the
// warp's 32 runs of y (cp.async, chunks of CF steps in the fold, CH steps in
// the carry pass: the two rings share the region), and in the carry pass the
// next CH filter records of the 32 runs, each run's chunk at an odd number of
// 16-byte units so that the lanes' record stores hit distinct banks.
KF_HD constexpr int ti_al16(int x) { return (x + 15) / 16 * 16; }
template <int N, typename R, int THREADS, int CH>
struct TiStage {
    static constexpr int M = N / 2, NST = 4, CF = 4;
    static constexpr int FB = FRec<N, R>::SIZE * int(sizeof(R));
    static constexpr int YF = ti_al16(WarpStage<CF, M, R>::BYTES);    // one fold input buffer
    static constexpr int YC = ti_al16(WarpStage<CH, M, R>::BYTES);    // one carry-pass input buffer
    static constexpr int OUT = 32 * (((CH * FB / 16) | 1) * 16);  // the record buffer
    static constexpr int warp_bytes(bool staged) {
        return NST * YF > NST * YC + (staged ? OUT : 0) ? NST * YF : NST * YC + (staged ? OUT : 0);
    }
    static constexpr int bytes(bool staged) { return (THREADS / 32) * warp_bytes(staged); }
};

// Threads per CTA THREADS, records per staged chunk CH, MINB resident CTAs
// per SM.
template <int N, typename R, int THREADS, int CH, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) ti_filter_kernel(const __grid_constant__ TiArgs<N, R> a) {
    using TT = TiTab<N, R>;
    constexpr int M = N / 2, NN = N * N, S = N * (N + 1) / 2, NW = THREADS / 32, E = TT::E;
    constexpr int FR = FRec<N, R>::SIZE;
    static_assert(NW <= 8, "at most 8 warps");
    __shared__ R s_wb[NW][N], s_we[NW][N];   // warp aggregates, then warp-exclusive (b, eta)
    __shared__ R s_lx[NW][NN + N];           // look-back: one composed map per warp
    __shared__ R s_tb[N];                    // the tile's carry mean
    __shared__ double s_ll[NW];
    __shared__ int s_tile, s_abort, s_last;
    __shared__ unsigned long long s_twait;   // phase trace: the last look-back wait to end

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ __align__(16) unsigned char dsm[];
    R *const rows = reinterpret_cast<R *>(dsm);
    R *const sets = rows + TT::al((a.K > 1 ? a.K - 1 : 0) * E);
    unsigned char *const stage = reinterpret_cast<unsigned char *>(sets + TT::al(TT::NSETS * TT::WES));
    using ST = TiStage<N, R, THREADS, CH>;
    constexpr int NST = ST::NST, CF = ST::CF;
    constexpr int RU = FR * int(sizeof(R)) / 16;              // 16-byte units of a record,
    constexpr int SEGU = CH * RU, STRU = SEGU | 1;            // of a run's chunk, and its odd stride
    unsigned char *const wbase = stage + warp * ST::warp_bytes(a.frec != nullptr);
    float4 *const wstage = a.frec ? reinterpret_cast<float4 *>(wbase + NST * ST::YC) : nullptr;

    if (tid == 0) {
        s_tile = atomicAdd(a.counters, 1);
        s_abort = 0;
        s_twait = 0;
    }
    // tables into shared memory
    {
        const R *src = a.tab + a.off_rows;
        const int nr = (a.K > 1 ? a.K - 1 : 0) * E;
        for (int i = tid; i < nr; i += THREADS) rows[i] = __ldg(src + i);
        const R *ss = a.tab + a.off_sets;
        for (int i = tid; i < TT::NSETS * TT::WE; i += THREADS) sets[(i / TT::WE) * TT::WES + i % TT::WE] = __ldg(ss + i);
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= a.ntiles || tile == a.inject_skip_tile) return;
    uint64_t *const trace = (a.trace && tile < a.trace_cap && tid == 0) ? a.trace + 16 * tile : nullptr;
    if (trace) trace[0] = ti_ns();
    const FiltParams<N, R> &P = a.prm;
    const int64_t treg = a.T - 1;                                  // scan positions
    const int64_t r0 = (int64_t(tile) * THREADS + tid) * a.K;       // this thread's first position
    const int64_t r1 = r0 + a.K < treg ? r0 + a.K : treg;          // one past its last

    // ---- 2. thread fold (y of the warp's 32 runs staged through a cp.async ring)
    const int64_t wr0 = (int64_t(tile) * THREADS + warp * 32) * a.K;   // lane 0's first position
    R b[N], e[N];
#pragma unroll
    for (int i = 0; i < N; ++i) b[i] = e[i] = 0;
    {
        auto fbuf = [&](int ch) { return wbase + (ch % NST) * ST::YF; };
        const int nch = (a.K + CF - 1) / CF;   // the same for every lane
#pragma unroll
        for (int k = 0; k < NST - 1; ++k) {
            if (k < nch) stage_load<CF, M, R>(a.y, wr0 + 1 + int64_t(k) * CF, a.K, a.T, fbuf(k), lane);
            cp_async_commit();
        }
#pragma unroll 1
        for (int ch = 0; ch < nch; ++ch) {
            const int ahead = ch + NST - 1;   // its buffer was last read in chunk ch - 1
            if (ahead < nch) stage_load<CF, M, R>(a.y, wr0 + 1 + int64_t(ahead) * CF, a.K, a.T, fbuf(ahead), lane);
            cp_async_commit();
            cp_async_wait<NST - 1>();
            __syncwarp();
#pragma unroll
            for (int cc = 0; cc < CF; ++cc) {
                const int c = ch * CF + cc;
                if (r0 + c >= r1) break;
                R y[M];
                load_rec<M>(y, stage_rec<CF, M, R>(fbuf(ch), lane, cc));
                if (c == 0) {
                    fresh_b_eta<N, M, R>(P, y, b, e);
                    continue;
                }
                ti_fold_step<N, M, R>(P, rows + (c - 1) * E, y, b, e);
            }
            __syncwarp();
        }
        cp_async_wait<0>();
        __syncwarp();
    }
    if (trace) trace[1] = ti_ns();

    // ---- 3. warp scan and warp-aggregate scan of the (b, eta) halves
#pragma unroll 1
    for (int s = 1; s < 32; s <<= 1) {
        R bx[N], ex[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            bx[i] = __shfl_up_sync(0xffffffffu, b[i], s);
            ex[i] = __shfl_up_sync(0xffffffffu, e[i], s);
        }
        if (lane >= s) {
            const int p = (lane - s + 1) < s ? (lane - s + 1) : s;
            ti_combine<N, R>(sets + TT::wset(s, p) * TT::WES, bx, ex, b, e);
        }
    }
    R blx[N], elx[N];   // lane-exclusive (b, eta): a run of `lane` thread aggregates
#pragma unroll
    for (int i = 0; i < N; ++i) {
        blx[i] = __shfl_up_sync(0xffffffffu, b[i], 1);
        elx[i] = __shfl_up_sync(0xffffffffu, e[i], 1);
    }
    if (lane == 31) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            s_wb[warp][i] = b[i];
            s_we[warp][i] = e[i];
        }
    }
    __syncthreads();
    if (warp == 0) {
        R wb[N], we[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            wb[i] = lane < NW ? s_wb[lane][i] : R(0);
            we[i] = lane < NW ? s_we[lane][i] : R(0);
        }
#pragma unroll 1
        for (int s = 1; s < NW; s <<= 1) {
            R bx[N], ex[N];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                bx[i] = __shfl_up_sync(0xffffffffu, wb[i], s);
                ex[i] = __shfl_up_sync(0xffffffffu, we[i], s);
            }
            if (lane >= s && lane < NW) {
                const int p = (lane - s + 1) < s ? (lane - s + 1) : s;
                ti_combine<N, R>(sets + TT::vset(s, p) * TT::WES, bx, ex, wb, we);
            }
        }
        R xb[N], xe[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            xb[i] = __shfl_up_sync(0xffffffffu, wb[i], 1);
            xe[i] = __shfl_up_sync(0xffffffffu, we[i], 1);
        }
        __syncwarp();
        if (lane < NW) {
#pragma unroll
            for (int i = 0; i < N; ++i) {
                s_wb[lane][i] = lane ? xb[i] : R(0);
                s_we[lane][i] = lane ? xe[i] : R(0);
            }
        }
        // ---- 4. publish u_i = Y_i eta_agg + b_agg (+ X_0 b_1 on tile 0)
        if (lane == NW - 1) {
            const R *te = a.tab + a.off_tiles + int64_t(tile) * TT::TES;
            const R *X = te + 2 * S, *Y = te + 2 * S + NN;
            R u[TT::UP];
#pragma unroll
            for (int r = 0; r < N; ++r) {
                R s = wb[r];
#pragma unroll
                for (int k = 0; k < N; ++k) s += __ldg(Y + r * N + k) * we[k];
                u[r] = s;
            }
            if (tile == 0) {
                R y1[M], b1[N];
                ti_load_y<M, R>(a.y, 0, y1);
#pragma unroll
                for (int r = 0; r < N; ++r) {
                    R s = P.c1[r];
#pragma unroll
                    for (int j = 0; j < M; ++j) s += P.K1[r * MAXNY + j] * y1[j];
                    b1[r] = s;
                }
#pragma unroll
                for (int r = 0; r < N; ++r)
#pragma unroll
                    for (int k = 0; k < N; ++k) u[r] += __ldg(X + r * N + k) * b1[k];
            }
#pragma unroll
            for (int i = N; i < TT::UP; ++i) u[i] = 0;
            if (tile + 1 < a.ntiles) {
                store_rec<TT::UP>(a.ubuf + int64_t(tile) * TT::UP, u);
                ti_st_release(a.flags + tile, 1);
            }
        }
    }
    if (trace) trace[2] = ti_ns();

    // ---- 5. look-back: b_{i-1} = the maps of tiles 0 .. i-1 composed in order
    if (tile > 0) {
        // one warp (the last, idle while warp 0 publishes) waits until every
        // preceding tile has published: its lanes read the flags together and
        // back off exponentially between rounds, so that the waiting tiles
        // keep the L2 free for the tiles still working; the rest of the CTA
        // waits at the barrier
        // X_{i-1} exactly zero (the map of a long tile underflows): b_{i-1} =
        // u_{i-1} + X_{i-1} (...) is u_{i-1} exactly, so only tile i-1 is needed
        bool xz = true;
        {
            const R *Xp = a.tab + a.off_tiles + int64_t(tile - 1) * TT::TES + 2 * S;
#pragma unroll
            for (int i = 0; i < NN; ++i) xz = xz && __ldg(Xp + i) == R(0);
        }
        if (warp == NW - 1) {
            bool ok = true;
            for (int q0 = xz ? tile - 1 : 0; q0 < tile && ok; q0 += 32) {
                const int q = q0 + lane;
                bool seen = q >= tile || !KF_IN(q >= 0, a.status) || ti_ld_relaxed(a.flags + q) != 0;
                unsigned ns = 32;
                const uint64_t t0 = ti_ns();
                while (!__all_sync(0xffffffffu, seen)) {
                    __nanosleep(ns);
                    ns = ns < 1024 ? 2 * ns : 1024;
                    if (!seen) seen = ti_ld_relaxed(a.flags + q) != 0;
                    const bool fail = ti_ld_relaxed(a.status) != 0 || int64_t(ti_ns() - t0) > a.timeout_ns;
                    if (__any_sync(0xffffffffu, fail)) {
                        if (lane == 0) atomicCAS(a.status, 0, 5);   // KF_ERR_TIMEOUT (kept if already set)
                        ok = false;
                        break;
                    }
                }
            }
            if (!ok && lane == 0) s_abort = 1;
        }
        __syncthreads();
        if (s_abort) return;
        const int lbt = 32 * a.lbw;
        const int vv = (tile + lbt - 1) / lbt;
        if (xz) {
            if (tid == 0) {
                asm volatile("fence.acq_rel.gpu;" ::: "memory");
                const R *up = a.ubuf + int64_t(tile - 1) * TT::UP;
#pragma unroll
                for (int i = 0; i < N; ++i) s_tb[i] = __ldcg(up + i);
            }
        } else if (tid < lbt) {
            R F[NN], v[N];
            bool have = false;
#pragma unroll
            for (int i = 0; i < NN; ++i) F[i] = (i % (N + 1) == 0) ? R(1) : R(0);
#pragma unroll
            for (int i = 0; i < N; ++i) v[i] = 0;
            // the flags were seen by another thread of the CTA: the barrier and
            // an acquire fence order them before the loads of the published maps
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            const int q0 = tid * vv, q1 = (q0 + vv < tile) ? q0 + vv : tile;
#pragma unroll 1
            for (int q = q0; q < q1; ++q) {
                const R *X = a.tab + a.off_tiles + int64_t(q) * TT::TES + 2 * S;
                R Xq[NN], uq[TT::UP];
#pragma unroll
                for (int i = 0; i < NN; ++i) Xq[i] = __ldg(X + i);
                {
                    const R *up = a.ubuf + int64_t(q) * TT::UP;
#pragma unroll
                    for (int i = 0; i < TT::UP; ++i) uq[i] = __ldcg(up + i);
                }
                if (!have) {
#pragma unroll
                    for (int i = 0; i < NN; ++i) F[i] = Xq[i];
#pragma unroll
                    for (int i = 0; i < N; ++i) v[i] = uq[i];
                    have = true;
                } else {   // (X_q, u_q) o (F, v) = (X_q F, X_q v + u_q)
                    R nF[NN], nv[N];
#pragma unroll
                    for (int r = 0; r < N; ++r) {
                        R s = uq[r];
#pragma unroll
                        for (int k = 0; k < N; ++k) s += Xq[r * N + k] * v[k];
                        nv[r] = s;
#pragma unroll
                        for (int c = 0; c < N; ++c) {
                            R t = 0;
#pragma unroll
                            for (int k = 0; k < N; ++k) t += Xq[r * N + k] * F[k * N + c];
                            nF[r * N + c] = t;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < NN; ++i) F[i] = nF[i];
#pragma unroll
                    for (int i = 0; i < N; ++i) v[i] = nv[i];
                }
            }
            if (a.trace) atomicMax(&s_twait, (unsigned long long)ti_ns());
            // lanes hold consecutive blocks of tiles, earliest first: compose
            // the later block over the earlier one, down to lane 0
#pragma unroll 1
            for (int s = 1; s < 32; s <<= 1) {
                R oF[NN], ov[N];
#pragma unroll
                for (int i = 0; i < NN; ++i) oF[i] = __shfl_down_sync(0xffffffffu, F[i], s);
#pragma unroll
                for (int i = 0; i < N; ++i) ov[i] = __shfl_down_sync(0xffffffffu, v[i], s);
                if (lane + s < 32) {
                    R nF[NN], nv[N];
#pragma unroll
                    for (int r = 0; r < N; ++r) {
                        R t = ov[r];
#pragma unroll
                        for (int k = 0; k < N; ++k) t += oF[r * N + k] * v[k];
                        nv[r] = t;
#pragma unroll
                        for (int c = 0; c < N; ++c) {
                            R w = 0;
#pragma unroll
                            for (int k = 0; k < N; ++k) w += oF[r * N + k] * F[k * N + c];
                            nF[r * N + c] = w;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < NN; ++i) F[i] = nF[i];
#pragma unroll
                    for (int i = 0; i < N; ++i) v[i] = nv[i];
                }
            }
            if (lane == 0 && a.trace && tile < a.trace_cap && warp < 6)
                a.trace[16 * tile + 8 + warp] = ti_ns();   // phase trace: warp w's tree done
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < NN; ++i) s_lx[warp][i] = F[i];
#pragma unroll
                for (int i = 0; i < N; ++i) s_lx[warp][NN + i] = v[i];
            }
        }
        if (trace) trace[7] = ti_ns();
        __syncthreads();
        if (trace) trace[6] = s_twait;
        if (trace) trace[14] = ti_ns();
        if (tid == 0 && !xz) {   // warps in order: only the mean of the composition is needed
            R v[N];
#pragma unroll
            for (int i = 0; i < N; ++i) v[i] = s_lx[0][NN + i];
            for (int w = 1; w < a.lbw; ++w) {
                R nv[N];
#pragma unroll
                for (int r = 0; r < N; ++r) {
                    R t = s_lx[w][NN + r];
#pragma unroll
                    for (int k = 0; k < N; ++k) t += s_lx[w][r * N + k] * v[k];
                    nv[r] = t;
                }
#pragma unroll
                for (int i = 0; i < N; ++i) v[i] = nv[i];
            }
#pragma unroll
            for (int i = 0; i < N; ++i) s_tb[i] = v[i];
            if (trace) trace[15] = ti_ns();
        }
    } else if (tid == 0) {   // tile 0: the carry is s_1 = (b_1, P_{1|1})
        R y1[M];
        ti_load_y<M, R>(a.y, 0, y1);
#pragma unroll
        for (int r = 0; r < N; ++r) {
            R s = P.c1[r];
#pragma unroll
            for (int j = 0; j < M; ++j) s += P.K1[r * MAXNY + j] * y1[j];
            s_tb[r] = s;
        }
    }
    __syncthreads();
    if (trace) trace[3] = ti_ns();

    // ---- 6a. this thread's exclusive carry: tile carry (x) warp run (x) lane run
    FwdCarry<N, R> c;
    {
        const R *te = a.tab + a.off_tiles + int64_t(tile) * TT::TES;
        R bw[N], Cw[S], Lw[S], dw[N];
#pragma unroll
        for (int i = 0; i < N; ++i) bw[i] = s_tb[i];
#pragma unroll
        for (int i = 0; i < S; ++i) {
            Cw[i] = __ldg(te + i);
            Lw[i] = __ldg(te + S + i);
        }
        if (warp > 0) {   // the run of 32 w thread aggregates before this warp
            const R *sp = a.tab + a.off_spans + TT::span(32 * warp) * TT::PE;
            R A[NN], Cs[S], J[S], bs[N], es[N], bo[N];
#pragma unroll
            for (int i = 0; i < NN; ++i) A[i] = __ldg(sp + i);
#pragma unroll
            for (int i = 0; i < S; ++i) {
                Cs[i] = __ldg(sp + NN + i);
                J[i] = __ldg(sp + NN + S + i);
            }
#pragma unroll
            for (int i = 0; i < N; ++i) {
                bs[i] = s_wb[warp][i];
                es[i] = s_we[warp][i];
                dw[i] = recip(Lw[lo(i, i)]);
            }
            apply_run_chol<N, R>(Lw, dw, bw, A, bs, Cs, es, J, bo, Cw);
#pragma unroll
            for (int i = 0; i < N; ++i) bw[i] = bo[i];
            chol_lo<N, R>(Cw, Lw, dw);
        } else {
#pragma unroll
            for (int i = 0; i < N; ++i) dw[i] = recip(Lw[lo(i, i)]);
        }
        if (lane > 0) {   // the run of `lane` thread aggregates before this thread
            const R *sp = a.tab + a.off_spans + TT::span(lane) * TT::PE;
            R A[NN], Cs[S], J[S];
#pragma unroll
            for (int i = 0; i < NN; ++i) A[i] = __ldg(sp + i);
#pragma unroll
            for (int i = 0; i < S; ++i) {
                Cs[i] = __ldg(sp + NN + i);
                J[i] = __ldg(sp + NN + S + i);
            }
            apply_run_chol<N, R>(Lw, dw, bw, A, blx, Cs, elx, J, c.v + FwdCarry<N, R>::ob, c.v + FwdCarry<N, R>::oC);
        } else {
#pragma unroll
            for (int i = 0; i < N; ++i) c.v[FwdCarry<N, R>::ob + i] = bw[i];
#pragma unroll
            for (int i = 0; i < S; ++i) c.v[FwdCarry<N, R>::oC + i] = Cw[i];
        }
    }
    if (trace) trace[4] = ti_ns();

    // ---- 6b. carry pass: extend by each element, emit, log-likelihood terms
    double ll = 0.0;
    if (tile == 0 && tid == 0) {   // time k = 1: record 0 is s_1 itself
        R y1[M];
        ti_load_y<M, R>(a.y, 0, y1);
        R b1[N];
#pragma unroll
        for (int i = 0; i < N; ++i) b1[i] = s_tb[i];
        ti_emit<N, R>(a, 0, b1, P.C1, a.frec);   // record 0 in place (16-byte aligned)
        if (a.want_ll) {
            R v[M];
#pragma unroll
            for (int j = 0; j < M; ++j) v[j] = y1[j] - P.Hx1[j];
            double q = 0;
#pragma unroll
            for (int i = 0; i < M; ++i)
#pragma unroll
                for (int j = 0; j < M; ++j) q += double(v[i] * P.S1inv[i * MAXNY + j] * v[j]);
            ll = -0.5 * (q + P.llc1);
        }
    }
    {
        // chunks of CH steps, the same count for every lane of the warp (the
        // lanes share each chunk's y ring buffer and record store)
        const int nch = (a.K + CH - 1) / CH;
        auto cbuf = [&](int ch) { return wbase + (ch % NST) * ST::YC; };
#pragma unroll
        for (int k = 0; k < NST - 1; ++k) {
            if (k < nch) stage_load<CH, M, R>(a.y, wr0 + 1 + int64_t(k) * CH, a.K, a.T, cbuf(k), lane);
            cp_async_commit();
        }
#pragma unroll 1
        for (int ch = 0; ch < nch; ++ch) {
            const int ahead = ch + NST - 1;
            if (ahead < nch) stage_load<CH, M, R>(a.y, wr0 + 1 + int64_t(ahead) * CH, a.K, a.T, cbuf(ahead), lane);
            cp_async_commit();
            cp_async_wait<NST - 1>();
            __syncwarp();
            R *buf = wstage ? reinterpret_cast<R *>(wstage + lane * STRU) : nullptr;
            const int64_t p0 = r0 + int64_t(ch) * CH;
            const int cnt = int(r1 - p0 < CH ? (r1 - p0 > 0 ? r1 - p0 : 0) : CH);
            R llc = 0;
#pragma unroll
            for (int cc = 0; cc < CH; ++cc) {
                if (cc >= cnt) break;
                const int64_t g = p0 + cc + 1;   // record of time k = g + 1
                R y[M];
                load_rec<M>(y, stage_rec<CH, M, R>(cbuf(ch), lane, cc));
                if (a.want_ll) llc += ti_carry_step<N, M, R, true>(P, y, c);
                else ti_carry_step<N, M, R, false>(P, y, c);
                ti_emit<N, R>(a, g, c.v + FwdCarry<N, R>::ob, c.v + FwdCarry<N, R>::oC, buf ? buf + cc * FR : nullptr);
            }
            ll += double(llc);
            __syncwarp();   // every lane is done with this chunk's y buffer and records
            if (wstage) {   // the warp's 32 chunks, each run's records contiguous in memory
                // a lane moves the same unit o of every run it visits (SEGU, a
                // power of two, divides 32 when it is at most 32)
                float4 *g = reinterpret_cast<float4 *>(a.frec);
                if constexpr (SEGU <= 32 && (32 % SEGU) == 0) {
                    constexpr int STEP = 32 / SEGU;
                    const int o = lane % SEGU, rc = o / RU, ru = o % RU;
#pragma unroll
                    for (int run = lane / SEGU; run < 32; run += STEP) {
                        const int64_t rs = wr0 + int64_t(run) * a.K;               // the run's first position
                        const int64_t re = rs + a.K < treg ? rs + a.K : treg;      // one past its last
                        const int64_t pos = rs + int64_t(ch) * CH + rc;
                        if (pos < re) g[(pos + 1) * RU + ru] = wstage[run * STRU + o];
                    }
                } else {
#pragma unroll 2
                    for (int idx = lane; idx < 32 * SEGU; idx += 32) {
                        const int run = idx / SEGU, o = idx - run * SEGU;
                        const int64_t rs = wr0 + int64_t(run) * a.K;
                        const int64_t re = rs + a.K < treg ? rs + a.K : treg;
                        const int64_t pos = rs + int64_t(ch) * CH + o / RU;
                        if (pos < re) g[(pos + 1) * RU + o % RU] = wstage[run * STRU + o];
                    }
                }
                __syncwarp();
            }
        }
        cp_async_wait<0>();
    }
    if (trace) trace[5] = ti_ns();

    // ---- log-likelihood: fixed-order sums per tile, then over tiles
    if (a.ll_out) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) ll += __shfl_down_sync(0xffffffffu, ll, s);
        if (lane == 0) s_ll[warp] = ll;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NW; ++w) t += s_ll[w];
            a.ll_part[tile] = t;
            __threadfence();
            s_last = (atomicAdd(a.counters + 1, 1) == a.ntiles - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double t = 0.0;
            for (int i = tid; i < a.ntiles; i += THREADS) t += __ldcg(a.ll_part + i);
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) t += __shfl_down_sync(0xffffffffu, t, s);
            if (lane == 0) s_ll[warp] = t;
            __syncthreads();
            if (tid == 0) {
                double u = 0.0;
                for (int w = 0; w < NW; ++w) u += s_ll[w];
                *a.ll_out = u;
            }
        }
    }
}

}  // namespace kfs
