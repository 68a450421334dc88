// rts_scan.cuh -- the RTS smoother pass of Alg. prts on one sequence: a
// single-pass decoupled look-back scan in reverse time over the elements
// (E_k, g_k, L_k) of Eqs. prts_init1/2 under Lemma 2 (Sec. IV-D).
//
// The elements are built where they are consumed, from the filter records
// (xbar_{k|k}, P_{k|k}) and the model's F, Q:
//   P_{k+1|k} = F P F^T + Q = L L^T,  E_k = P F^T P_{k+1|k}^{-1},
// and both passes over a thread's run use them in the direct form of
// Lemma 2 with the later part (g, L) on the right:
//   g' = xbar + E_k (g - F xbar),   L' = P + E_k (L - P_{k+1|k}) E_k^T,
// which equals (g_k + E_k g, L_k + E_k L E_k^T) with g_k = xbar - E_k F xbar,
// L_k = P - E_k P_{k+1|k} E_k^T, without forming g_k and L_k.  The last
// element (k = T) has E_T = 0: its g' and L' are xbar_T and P_T.
//
// A CTA scans a tile of THREADS x K scan positions (position p is time
// index T - 1 - p): thread fold of its K elements (aggregate E = E_k E,
// g, L as above), warp and warp-aggregate scans under Lemma 2 (the lane- and
// warp-exclusive suffixes kept in shared memory), look-back as in the
// forward scans (one warp waits for the predecessors' flags with back-off;
// the aggregates after the nearest inclusive carry are reduced by a tree),
// then every thread walks its K elements again from its carry and writes the
// smoothed means and covariances through shared memory, warp-coalesced.
#pragma once

#include "kf_problems.cuh"
#include "kf_steps.cuh"
#include "stage.cuh"

namespace kfs {

template <int N, typename R>
struct RsArgs {
    R F[N * N], Q[N * (N + 1) / 2];   // model (Q packed)
    int64_t T;
    const R *frec;                     // filter records [T][FRec]
    R *ms, *Ps;                        // smoothed means [T][N], covariances [T][N][N]
    int K, ntiles, lbw;
    int *counters;                     // [0] tile ticket
    int *flags;                        // [ntiles] 1 aggregate, 2 inclusive carry
    R *agg;                            // [ntiles][RElem padded to 16 bytes]
    R *incl;                           // [ntiles][RCarry]
    int *status;
    int64_t timeout_ns;
    int inject_skip_tile;
    uint64_t *trace;
    int trace_cap;
};

KF_D int rs_ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
KF_D void rs_st_release(int *p, int v) { asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory"); }
KF_D uint64_t rs_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// x <- x (x) y with y later in time (Lemma 2); the scan runs in reverse time,
// so y is the operand earlier in scan order.
template <int N, typename R>
KF_D void rs_combine_later(RElem<N, R> &x, const RElem<N, R> &y) {
    RElem<N, R> t;
    lemma2<N, R>(x, y, t);
    x = t;
}

template <class X>
KF_D void rs_shfl_up(const X &in, X &out, int d) {
#pragma unroll
    for (int i = 0; i < X::SIZE; ++i) out.v[i] = __shfl_up_sync(0xffffffffu, in.v[i], d);
}
template <class X>
KF_D void rs_shfl_down(const X &in, X &out, int d) {
#pragma unroll
    for (int i = 0; i < X::SIZE; ++i) out.v[i] = __shfl_down_sync(0xffffffffu, in.v[i], d);
}

// Shared-memory bytes of one CTA: the lane-exclusive suffixes (odd stride),
// then per warp the staging buffers of CH smoothed means and covariances.
template <int N, typename R, int THREADS, int CH>
struct RsSmem {
    static constexpr int ES = RElem<N, R>::SIZE, LXS = ES | 1;
    static constexpr int LX = ((THREADS * LXS * int(sizeof(R))) + 15) / 16 * 16;
    static constexpr int MB = (WarpStage<CH, N, R>::BYTES + 15) / 16 * 16;
    static constexpr int PB = (WarpStage<CH, N * N, R>::BYTES + 15) / 16 * 16;
    static constexpr int WARP = MB + PB;
    static constexpr int BYTES = LX + (THREADS / 32) * WARP;
};

// Store the staged chunk (CH records of REC values per run, slot c of run r
// holding the record of global index gs0 - r K + c) of the warp's 32 runs,
// coalesced: a lane always moves the same unit o of a run's chunk, runs
// lane / SEGU, lane / SEGU + 32 / SEGU, ... (SEGU, a power of two <= 32,
// divides 32).  Records outside the run's own range [lo_r, hi_r) are skipped.
template <int CH, int REC, typename R>
KF_D void rs_store_chunk(R *gbase, int64_t gs0, int64_t K, int64_t hi0, int64_t T, const void *buf, int lane) {
    using W = WarpStage<CH, REC, R>;
    using UT = typename UnitT<W::U>::T;
    static_assert((32 % W::SEGU) == 0, "chunk units must divide the warp");
    constexpr int STEP = 32 / W::SEGU;
    const int o = lane % W::SEGU, run0 = lane / W::SEGU;
    const int rc = o / W::RU, ru = o % W::RU;
    UT *g = reinterpret_cast<UT *>(gbase);
    const UT *sb = static_cast<const UT *>(buf);
#pragma unroll
    for (int run = run0; run < 32; run += STEP) {
        const int64_t hi = hi0 - int64_t(run) * K;             // one past the run's last record
        const int64_t lo = hi - K > 0 ? hi - K : 0;
        const int64_t rec = gs0 - int64_t(run) * K + rc;
        if (rec >= lo && rec < hi && rec < T) g[rec * W::RU + ru] = sb[run * W::STRIDE + o];
    }
}

template <int N, typename R, int THREADS, int CH, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) rts_kernel(const __grid_constant__ RsArgs<N, R> a) {
    using El = RElem<N, R>;
    using Ca = RCarry<N, R>;
    using SM = RsSmem<N, R, THREADS, CH>;
    constexpr int NN = N * N, S = N * (N + 1) / 2, NW = THREADS / 32, ES = El::SIZE, CS = Ca::SIZE;
    constexpr int FR = FRec<N, R>::SIZE, Q = 16 / int(sizeof(R));
    constexpr int ESP = (ES + Q - 1) / Q * Q;   // published aggregates: 16-byte stride (carries: CS)
    __shared__ R s_wx[NW][ES];     // warp aggregates, then warp-exclusive suffixes
    __shared__ R s_red[NW][ES];    // tile aggregate, then the look-back reduction
    __shared__ R s_carry[CS];      // the tile's carry
    __shared__ int s_tile, s_qstar, s_abort;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ __align__(16) unsigned char dsm[];
    R *const s_lx = reinterpret_cast<R *>(dsm);
    unsigned char *const wstage = dsm + SM::LX + warp * SM::WARP;
    if (tid == 0) {
        s_tile = atomicAdd(a.counters, 1);
        s_qstar = -1;
        s_abort = 0;
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= a.ntiles || tile == a.inject_skip_tile) return;
    uint64_t *const trace = (a.trace && tile < a.trace_cap && tid == 0) ? a.trace + 16 * tile : nullptr;
    if (trace) trace[0] = rs_ns();
    const int64_t T = a.T;
    const int64_t r0 = (int64_t(tile) * THREADS + tid) * a.K;   // this thread's first scan position
    const int64_t r1 = KF_IN(r0 >= 0, a.status) ? (r0 + a.K < T ? r0 + a.K : T) : r0;   // one past its last
    const int64_t start0 = (int64_t(tile) * THREADS + warp * 32) * a.K;   // lane 0's first position

    // ---- fold: the aggregate of this thread's K elements (scan order is
    // decreasing time: each new element is earlier than the aggregate)
    El agg;
    set_identity(agg);
    {
        R rec[FR], nxt[FR];
        if (r0 < r1) load_rec<FR>(rec, a.frec + (T - 1 - r0) * FR);
#pragma unroll 1
        for (int64_t p = r0; p < r1; ++p) {
            if (p + 1 < r1) load_rec<FR>(nxt, a.frec + (T - 2 - p) * FR);   // the next record, in flight
            rs_fold_step<N, R>(a.F, a.Q, p == 0, rec, agg.v + El::oE, agg.v + El::og, agg.v + El::oL);
#pragma unroll
            for (int i = 0; i < FR; ++i) rec[i] = nxt[i];
        }
    }
    if (trace) trace[1] = rs_ns();

    // ---- warp scan and warp-aggregate scan: suffixes in time
#pragma unroll 1
    for (int s = 1; s < 32; s <<= 1) {
        El o;
        rs_shfl_up(agg, o, s);
        if (lane >= s) rs_combine_later(agg, o);
    }
    {
        El lx;   // the lanes before this one in scan order: later in time
        rs_shfl_up(agg, lx, 1);
        if (lane == 0) set_identity(lx);
        R *d = s_lx + tid * SM::LXS;
#pragma unroll
        for (int i = 0; i < ES; ++i) d[i] = lx.v[i];
    }
    if (lane == 31) {
#pragma unroll
        for (int i = 0; i < ES; ++i) s_wx[warp][i] = agg.v[i];
    }
    __syncthreads();
    if (warp == 0) {
        El w;
        if (lane < NW) {
#pragma unroll
            for (int i = 0; i < ES; ++i) w.v[i] = s_wx[lane][i];
        } else {
            set_identity(w);
        }
#pragma unroll 1
        for (int s = 1; s < NW; s <<= 1) {
            El o;
            rs_shfl_up(w, o, s);
            if (lane >= s && lane < NW) rs_combine_later(w, o);
        }
        El wx;
        rs_shfl_up(w, wx, 1);
        if (lane == 0) set_identity(wx);
        __syncwarp();
        if (lane < NW) {
#pragma unroll
            for (int i = 0; i < ES; ++i) s_wx[lane][i] = wx.v[i];
        }
        if (lane == NW - 1) {
#pragma unroll
            for (int i = 0; i < ES; ++i) s_red[0][i] = w.v[i];
        }
    }
    __syncthreads();
    El tagg;
#pragma unroll
    for (int i = 0; i < ES; ++i) tagg.v[i] = s_red[0][i];
    // publish the tile's aggregate (tile 0 publishes its carry directly).  An
    // aggregate whose E is exactly zero (the product of many E_k underflows)
    // makes the carry from the later tiles irrelevant: tagg (x) c = (g, L) of
    // tagg exactly, so it is published at once as the inclusive carry and the
    // earlier tiles' look-backs stop at it.
    bool ezero = true;
#pragma unroll
    for (int i = 0; i < NN; ++i) ezero = ezero && tagg.v[El::oE + i] == R(0);
    if (tile > 0 && tid == 0 && tile + 1 < a.ntiles) {
        if (ezero) {
            R *dst = a.incl + int64_t(tile) * CS;
#pragma unroll
            for (int i = 0; i < N; ++i) dst[Ca::og + i] = tagg.v[El::og + i];
#pragma unroll
            for (int i = 0; i < S; ++i) dst[Ca::oL + i] = tagg.v[El::oL + i];
            rs_st_release(a.flags + tile, 2);
        } else {
            R *dst = a.agg + int64_t(tile) * ESP;
#pragma unroll
            for (int i = 0; i < ES; ++i) dst[i] = tagg.v[i];
            rs_st_release(a.flags + tile, 1);
        }
    }
    __syncthreads();
    if (trace) trace[2] = rs_ns();

    // ---- look-back: the carry from the later tiles
    Ca tc;
    set_zero(tc);
    if (tile > 0) {
        // one warp waits until the predecessors after the nearest one with an
        // inclusive carry have published, with back-off; the rest wait at the
        // barrier
        if (warp == NW - 1) {
            bool ok = true;
            int qloc = -1;
            for (int q0 = tile - 1; q0 >= 0 && ok; q0 -= 32) {
                const int q = q0 - lane;
                int f = q >= 0 && KF_IN(q < a.ntiles, a.status) ? rs_ld_relaxed(a.flags + q) : 1;
                unsigned ns = 32;
                const uint64_t t0 = rs_ns();
                while (!__all_sync(0xffffffffu, f != 0)) {
                    __nanosleep(ns);
                    ns = ns < 1024 ? 2 * ns : 1024;
                    if (f == 0) f = rs_ld_relaxed(a.flags + q);
                    const bool fail = rs_ld_relaxed(a.status) != 0 || int64_t(rs_ns() - t0) > a.timeout_ns;
                    if (__any_sync(0xffffffffu, fail)) {
                        if (lane == 0) atomicCAS(a.status, 0, 5);   // KF_ERR_TIMEOUT
                        ok = false;
                        break;
                    }
                }
                if (q >= 0 && f == 2 && q > qloc) qloc = q;
                if (__any_sync(0xffffffffu, q >= 0 && f == 2)) break;
            }
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                const int o = __shfl_down_sync(0xffffffffu, qloc, s);
                qloc = o > qloc ? o : qloc;
            }
            if (lane == 0) {
                s_qstar = qloc;
                if (!ok) s_abort = 1;
            }
        }
        __syncthreads();
        if (s_abort) return;
        const int lbt = 32 * a.lbw;
        const int vv = (a.ntiles + lbt - 1) / lbt;
        const int qstar = s_qstar;
        if (tid < lbt) {
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            // thread tid takes q = tile-1-(tid*vv + v): the nearest predecessors
            // (the earliest in time) on thread 0; each thread folds its own
            // ones from the latest in time (the smallest q) onwards
            El x;
            bool have = false;
#pragma unroll 1
            for (int v = vv - 1; v >= 0; --v) {
                const int q = tile - 1 - (tid * vv + v);
                if (q > qstar) {
                    El y;
                    const R *src = a.agg + int64_t(q) * ESP;
#pragma unroll
                    for (int i = 0; i < ES; ++i) y.v[i] = __ldcg(src + i);
                    if (!have) {
                        x = y;
                        have = true;
                    } else {   // y is earlier in time than x
                        El t;
                        lemma2<N, R>(y, x, t);
                        x = t;
                    }
                }
            }
            if (!have) set_identity(x);
            // lane l holds earlier tiles in time than lane l+1: reduce to lane 0
#pragma unroll 1
            for (int s = 1; s < 32; s <<= 1) {
                El o;
                rs_shfl_down(x, o, s);
                if (lane + s < 32) rs_combine_later(x, o);
            }
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < ES; ++i) s_red[warp][i] = x.v[i];
            }
        }
        __syncthreads();
        if (trace) trace[5] = rs_ns();
        if (tid == 0) {
            El y;
#pragma unroll
            for (int i = 0; i < ES; ++i) y.v[i] = s_red[0][i];
            for (int w = 1; w < a.lbw; ++w) {
                El o;
#pragma unroll
                for (int i = 0; i < ES; ++i) o.v[i] = s_red[w][i];
                rs_combine_later(y, o);
            }
            if (qstar >= 0) {
                const R *src = a.incl + int64_t(qstar) * CS;
#pragma unroll
                for (int i = 0; i < CS; ++i) tc.v[i] = __ldcg(src + i);
            }
            apply_rts<N, R>(tc, y);
        }
    }
    // ---- publish this tile's inclusive carry
    if (tid == 0) {
        Ca inc = tc;
        apply_rts<N, R>(inc, tagg);
#pragma unroll
        for (int i = 0; i < CS; ++i) s_carry[i] = tc.v[i];
        if (tile + 1 < a.ntiles && !(tile > 0 && ezero)) {
            R *dst = a.incl + int64_t(tile) * CS;
#pragma unroll
            for (int i = 0; i < CS; ++i) dst[i] = inc.v[i];
            rs_st_release(a.flags + tile, 2);
        }
    }
    __syncthreads();
    if (trace) trace[3] = rs_ns();

    // ---- this thread's carry: the tile carry, then the warps and lanes after it
    Ca c;
#pragma unroll
    for (int i = 0; i < CS; ++i) c.v[i] = s_carry[i];
    if (warp > 0) {
        El wx;
#pragma unroll
        for (int i = 0; i < ES; ++i) wx.v[i] = s_wx[warp][i];
        apply_rts<N, R>(c, wx);
    }
    if (lane > 0) {
        El lx;
        const R *d = s_lx + tid * SM::LXS;
#pragma unroll
        for (int i = 0; i < ES; ++i) lx.v[i] = d[i];
        apply_rts<N, R>(c, lx);
    }

    // ---- carry pass: smoothed moments of every element, staged per warp
    {
        unsigned char *const mbuf = wstage, *const pbuf = wstage + SM::MB;
        const int nch = (a.K + CH - 1) / CH;   // the same for every lane of the warp
        R rec[FR], nxt[FR];
        if (r0 < r1) load_rec<FR>(rec, a.frec + (T - 1 - r0) * FR);
#pragma unroll 1
        for (int ch = 0; ch < nch; ++ch) {
#pragma unroll
            for (int cc = 0; cc < CH; ++cc) {
                const int64_t p = r0 + int64_t(ch) * CH + cc;
                if (p >= r1) break;
                if (p + 1 < r1) load_rec<FR>(nxt, a.frec + (T - 2 - p) * FR);
                rs_carry_step<N, R>(a.F, a.Q, p == 0, rec, c.v + Ca::og, c.v + Ca::oL);
                const int slot = CH - 1 - cc;   // records ascend in time within a chunk
                store_rec<N>(stage_rec<CH, N, R>(mbuf, lane, slot), c.v + Ca::og);
                R full[NN];
                store_full<N>(full, c.v + Ca::oL);
                store_rec<NN>(stage_rec<CH, NN, R>(pbuf, lane, slot), full);
#pragma unroll
                for (int i = 0; i < FR; ++i) rec[i] = nxt[i];
            }
            __syncwarp();
            const int64_t gs0 = T - (start0 + int64_t(ch) * CH) - CH;   // first record of lane 0's chunk
            const int64_t hi0 = T - start0;                               // one past lane 0's last record
            rs_store_chunk<CH, N, R>(a.ms, gs0, a.K, hi0, T, mbuf, lane);
            rs_store_chunk<CH, NN, R>(a.Ps, gs0, a.K, hi0, T, pbuf, lane);
            __syncwarp();
        }
    }
    if (trace) trace[4] = rs_ns();
}

}  // namespace kfs
