// scan_dlb.cuh -- single-pass scan with decoupled look-back, generic over a
// problem policy (kf_problems.cuh).
//
// One CTA scans one tile of THREADS * K consecutive scan positions:
//   1. take a tile ticket (atomic counter), so every tile that a CTA waits
//      for was claimed by a CTA that is already running;
//   2. each thread builds its K elements and folds them (full operator, or
//      the problem's fold table when it has one and the run qualifies);
//   3. a warp Kogge-Stone scan (shuffles) and a scan of the warp aggregates
//      give every thread its exclusive prefix inside the tile and the tile
//      aggregate, which is published (flag 1);
//   4. look-back: one warp waits (bounded, with back-off) until the
//      predecessors after the nearest one that already published its
//      inclusive prefix (flag 2) have published their aggregates; the
//      aggregates after it are reduced in order by the look-back warps
//      (thread folds, warp shuffle tree, warp-0 tree) and applied to that
//      inclusive carry;
//   5. the tile's inclusive carry is published (flag 2);
//   6. each thread walks its K elements again, extending the carry one
//      element at a time with the one-sided operator, and emits its outputs
//      (extraction fused into the scan).
// The launcher keeps the number of tiles <= THREADS * V, so one look-back
// window (ceil(ntiles / THREADS) predecessors per thread) always covers every
// predecessor.
//
// Every wait is bounded by a wall-clock limit (%globaltimer); on time-out the
// CTA records KF_ERR_TIMEOUT in the status word and returns; other CTAs see
// the status word and stop waiting too.
#pragma once

#include "kf_problems.cuh"
#include "stage.cuh"

namespace kfs {

struct DlbCtl {
    int *counters;         // [0] tile ticket, [1] finished-tile count
    int *flags;            // [ntiles] 0 empty, 1 aggregate, 2 inclusive
    void *agg;             // [ntiles][Elem::SIZE padded to 16 bytes]
    void *incl;            // [ntiles][Carry::SIZE]
    double *ll_part;       // [ntiles] per-tile log-likelihood partial sums
    double *ll_out;        // final log-likelihood (nullable)
    double *ll_step;       // per-step log-likelihood terms [total] (nullable; batched calls)
    int *status;           // device status word
    int64_t timeout_ns;    // bound of every wait
    int ntiles;
    int K;                 // positions per thread
    int inject_skip_tile;  // test hook: this tile never publishes (-1: none)
    // per-warp dynamic shared memory: byte offsets of the staging buffers
    // (the first of stage_nst input buffers and their stride, three outputs;
    // -1 = not staged: the records are read or written in place) and the
    // warp stride
    int sm_in0, sm_in_stride, sm_out[3], sm_warp;
    int sm_tab;            // byte offset of the fold-table rows (-1: none)
    const void *tsc;       // tile-scan table (ScanTab) in device memory, or null
    int lbw;               // warps that take part in the look-back (1 .. THREADS/32)
    uint64_t *trace;       // optional [ntiles][8] %globaltimer stamps at phase boundaries
    int trace_cap;         // tiles the trace buffer holds
};

constexpr int KF_STATUS_TIMEOUT = 5;

KF_D void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
KF_D int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
KF_D uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <class X>
KF_D void shfl_up_x(const X &in, X &out, int d) {
#pragma unroll
    for (int i = 0; i < X::SIZE; ++i) out.v[i] = __shfl_up_sync(0xffffffffu, in.v[i], d);
}
template <class X>
KF_D void shfl_down_x(const X &in, X &out, int d) {
#pragma unroll
    for (int i = 0; i < X::SIZE; ++i) out.v[i] = __shfl_down_sync(0xffffffffu, in.v[i], d);
}
template <class X, typename R>
KF_D void load_cg(X &x, const R *src) {
#pragma unroll
    for (int i = 0; i < X::SIZE; ++i) x.v[i] = __ldcg(src + i);
}

// Elements published for the look-back sit at a stride padded to 16 bytes
// and move as 16-byte vectors (L2 only: other SMs wrote them).
template <class X, typename R>
constexpr int padded_size() {
    return ((X::SIZE * int(sizeof(R)) + 15) / 16) * 16 / int(sizeof(R));
}
template <class X, typename R>
KF_D void load_cg_vec(X &x, const R *src) {
    constexpr int P = padded_size<X, R>(), W = 16 / int(sizeof(R));
    R t[P];
#pragma unroll
    for (int i = 0; i < P / W; ++i) {
        if constexpr (sizeof(R) == 4) {
            const float4 v = __ldcg(reinterpret_cast<const float4 *>(src) + i);
            t[4 * i] = v.x; t[4 * i + 1] = v.y; t[4 * i + 2] = v.z; t[4 * i + 3] = v.w;
        } else {
            const double2 v = __ldcg(reinterpret_cast<const double2 *>(src) + i);
            t[2 * i] = v.x; t[2 * i + 1] = v.y;
        }
    }
#pragma unroll
    for (int i = 0; i < X::SIZE; ++i) x.v[i] = t[i];
}
template <class X, typename R>
KF_D void store_vec(R *dst, const X &x) {
    constexpr int P = padded_size<X, R>(), W = 16 / int(sizeof(R));
    R t[P];
#pragma unroll
    for (int i = 0; i < P; ++i) t[i] = i < X::SIZE ? x.v[i] : R(0);
#pragma unroll
    for (int i = 0; i < P / W; ++i) {
        if constexpr (sizeof(R) == 4)
            reinterpret_cast<float4 *>(dst)[i] = make_float4(t[4 * i], t[4 * i + 1], t[4 * i + 2], t[4 * i + 3]);
        else
            reinterpret_cast<double2 *>(dst)[i] = make_double2(t[2 * i], t[2 * i + 1]);
    }
}

// Global record index of scan position p, and the first record of the
// C-record segment that holds positions [p0, p0 + C) (record order is the
// global order, so a reverse scan walks its segment backwards).
template <class P>
KF_D int64_t gidx(int64_t total, int64_t p) { return P::REV ? total - 1 - p : p; }
template <class P, int C>
KF_D int64_t seg_first(int64_t total, int64_t p0) { return P::REV ? total - p0 - C : p0; }
template <class P, int C>
KF_D int seg_slot(int c) { return P::REV ? C - 1 - c : c; }

// Resident CTAs per SM that the register allocation of a 128-thread scan
// CTA must allow, per scan kind (filter, RTS, two-filter).
#ifndef KF_DLB_MINB_FILTER
#define KF_DLB_MINB_FILTER 1
#endif
#ifndef KF_DLB_MINB_RTS
#define KF_DLB_MINB_RTS 1
#endif
#ifndef KF_DLB_MINB_TF
#define KF_DLB_MINB_TF 1
#endif
#ifndef KF_DLB_MINB_RTS256
#define KF_DLB_MINB_RTS256 1
#endif
template <class P, int THREADS>
constexpr int dlb_min_blocks() {
    if (THREADS == 256) return P::KIND == 1 ? KF_DLB_MINB_RTS256 : 1;
    if (THREADS != 128) return 1;
    return P::KIND == 0 ? KF_DLB_MINB_FILTER : P::KIND == 1 ? KF_DLB_MINB_RTS : KF_DLB_MINB_TF;
}

template <class P, int THREADS, int V, int C>
__global__ void __launch_bounds__(THREADS, (dlb_min_blocks<P, THREADS>())) dlb_scan_kernel(const __grid_constant__ typename P::Args args,
                                                           const DlbCtl ctl) {
    using R = typename P::R;
    using Elem = typename P::Elem;
    using Carry = typename P::Carry;
    constexpr int NW = THREADS / 32, ES = Elem::SIZE, CS = Carry::SIZE;
    __shared__ R s_wx[NW][ES];     // warp-exclusive prefixes inside the tile
    __shared__ R s_red[NW][ES];    // tile aggregate / look-back reduction
    __shared__ R s_carry[CS];      // tile-exclusive carry
    __shared__ double s_ll[NW];
    __shared__ int s_tile, s_qstar, s_abort, s_last;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ __align__(16) unsigned char dsm[];
    R *const tab = (P::TABLE && ctl.sm_tab >= 0) ? reinterpret_cast<R *>(dsm + ctl.sm_tab) : nullptr;
    if constexpr (P::TABLE) {
        if (tab) P::tab_load(args, tab);
    }
    if (tid == 0) {
        s_tile = atomicAdd(ctl.counters, 1);
        s_qstar = -1;
        s_abort = 0;
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= ctl.ntiles || tile == ctl.inject_skip_tile) return;
    uint64_t *const trace = (ctl.trace && tile < ctl.trace_cap && threadIdx.x == 0) ? ctl.trace + 16 * tile : nullptr;
    if (trace) trace[0] = global_ns();
    const int64_t total = P::total(args);
    const int64_t start = (int64_t(tile) * THREADS + tid) * ctl.K;
    const int64_t start0 = (int64_t(tile) * THREADS + warp * 32) * ctl.K;   // lane 0's run
    const int64_t dK = P::REV ? -int64_t(ctl.K) : int64_t(ctl.K);
    const int64_t end = start + ctl.K < total ? start + ctl.K : total;

    unsigned char *wsm = dsm + warp * ctl.sm_warp;
    // staged input ring (null: the records are read in place)
    constexpr int NST = stage_nst<P>();
    constexpr int IRC = P::IN_REC > 0 ? P::IN_REC : 1;
    unsigned char *const in0 = (P::IN_REC && ctl.sm_in0 >= 0) ? wsm + ctl.sm_in0 : nullptr;
    auto inbuf = [&](int ch) { return in0 + (ch % NST) * ctl.sm_in_stride; };
    const int nchunks = (ctl.K + C - 1) / C;
    const R *in_arr = P::in_arr(args);

    // ---- 2. thread fold (input records staged through shared memory)
    Elem agg;
    {
        bool have = false;
        const bool fast = tab && P::tab_fast(args, start, end, ctl.K);
        typename P::TabFold tf;
        if constexpr (P::TABLE) tf.c = 0;
        SegCursor cur = P::cursor(args, start < total ? start : total - 1);
        if (P::IN_REC > 0 && in0) {
#pragma unroll
            for (int k = 0; k < NST - 1; ++k) {
                if (k < nchunks)
                    stage_load<C, IRC>(in_arr, seg_first<P, C>(total, start0 + k * C), dK, total, inbuf(k), lane);
                cp_async_commit();
            }
        }
        for (int ch = 0; ch < nchunks; ++ch) {
            if (P::IN_REC > 0 && in0) {
                const int ahead = ch + NST - 1;   // its buffer was last read by chunk ch - 1
                if (ahead < nchunks)
                    stage_load<C, IRC>(in_arr, seg_first<P, C>(total, start0 + ahead * C), dK, total, inbuf(ahead), lane);
                cp_async_commit();
                cp_async_wait<NST - 1>();   // chunk ch has arrived
                __syncwarp();
            }
#pragma unroll 1
            for (int c = 0; c < C; ++c) {
                const int64_t p = start + ch * C + c;
                if (p >= end) break;
                const R *in = !P::IN_REC ? nullptr
                              : in0 ? stage_rec<C, P::IN_REC, R>(inbuf(ch), lane, seg_slot<P, C>(c))
                                    : in_arr + gidx<P>(total, p) * P::IN_REC;
                if constexpr (P::TABLE) {
                    if (fast) {
                        P::tab_step(args, p, in, tab, tf);
                        continue;
                    }
                }
                if (!have) {
                    P::build(args, p, cur, in, agg);
                    have = true;
                } else {
                    P::fold_at(args, p, cur, in, agg);
                }
            }
            __syncwarp();
        }
        if constexpr (P::TABLE) {
            if (fast) {
                P::tab_finish(args, tf, agg);
                have = true;
            }
        }
        if (!have) set_identity(agg);
    }

    // ---- 3. warp scan, warp-aggregate scan (cold: kept rolled for code size)
    // FP64: a tile whose threads all folded K fresh elements scans only the
    // (b, eta) halves, with the tile-scan table (ScanTab), which replaces
    // Lemma 1 on the slow FP64 pipe by four matrix-vector products.  (In FP32
    // the table's loads cost as much as the combines they save.)
    bool tscan = false;
    if constexpr (P::TABLE) {
        tscan = sizeof(R) == 8 && ctl.tsc && tab && args.tab.K == ctl.K && tile > 0 && NW <= 8 &&
                (int64_t(tile) + 1) * THREADS * ctl.K <= total;
    }
    Elem lex;
    if constexpr (P::TABLE) {
        if (tscan) {
            constexpr int N = P::NX;
            using ST = ScanTab<N, R>;
            const R *tsc = static_cast<const R *>(ctl.tsc);
            R b[N], e[N];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                b[i] = agg.v[Elem::ob + i];
                e[i] = agg.v[Elem::oe + i];
            }
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
                    tsc_combine<N, R>(tsc + ST::w_off(s, p), bx, ex, b, e);
                }
            }
            R lb[N], le[N];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                lb[i] = __shfl_up_sync(0xffffffffu, b[i], 1);
                le[i] = __shfl_up_sync(0xffffffffu, e[i], 1);
            }
            if (lane > 0) tsc_elem<N, R>(tsc, lane, lb, le, lex);
            else set_identity(lex);
            if (lane == 31) {
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    s_wx[warp][Elem::ob + i] = b[i];
                    s_wx[warp][Elem::oe + i] = e[i];
                }
            }
            __syncthreads();
            if (trace) trace[1] = global_ns();
            if (warp == 0) {
                R wb[N], we[N];
#pragma unroll
                for (int i = 0; i < N; ++i) {
                    wb[i] = lane < NW ? s_wx[lane][Elem::ob + i] : R(0);
                    we[i] = lane < NW ? s_wx[lane][Elem::oe + i] : R(0);
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
                        tsc_combine<N, R>(tsc + ST::v_off(s, p), bx, ex, wb, we);
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
                    Elem wx;
                    if (lane == 0) set_identity(wx);
                    else tsc_elem<N, R>(tsc, 32 * lane, xb, xe, wx);
#pragma unroll
                    for (int i = 0; i < ES; ++i) s_wx[lane][i] = wx.v[i];
                }
                if (lane == NW - 1) {
                    Elem w;
                    tsc_elem<N, R>(tsc, 32 * NW, wb, we, w);
#pragma unroll
                    for (int i = 0; i < ES; ++i) s_red[0][i] = w.v[i];
                }
            }
            __syncthreads();
        }
    }
    if (!tscan) {
#pragma unroll 1
        for (int s = 1; s < 32; s <<= 1) {
            Elem o, t;
            shfl_up_x(agg, o, s);
            if (lane >= s) {
                P::combine(o, agg, t);
                agg = t;
            }
        }
        shfl_up_x(agg, lex, 1);
        if (lane == 31) {
#pragma unroll
            for (int i = 0; i < ES; ++i) s_wx[warp][i] = agg.v[i];
        }
        __syncthreads();
        if (trace) trace[1] = global_ns();
        if (warp == 0) {
            Elem w;
            if (lane < NW) {
#pragma unroll
                for (int i = 0; i < ES; ++i) w.v[i] = s_wx[lane][i];
            } else {
                set_identity(w);
            }
#pragma unroll 1
            for (int s = 1; s < NW; s <<= 1) {
                Elem o, t;
                shfl_up_x(w, o, s);
                if (lane >= s) {
                    P::combine(o, w, t);
                    w = t;
                }
            }
            Elem wx;
            shfl_up_x(w, wx, 1);
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
    }
    Elem tagg;
#pragma unroll
    for (int i = 0; i < ES; ++i) tagg.v[i] = s_red[0][i];

    // publish the tile aggregate (tile 0 publishes its inclusive prefix
    // directly); the release store orders the data stores before the flag.
    // An aggregate whose transition block (A, or E for Lemma 2) is exactly
    // zero -- a product of many steps that underflowed, or a segment start --
    // makes its inclusive carry independent of the tiles before it: it is
    // published at once (flag 2), so later look-backs stop there.
    constexpr int ESP = padded_size<Elem, R>();
    const bool zt = tile > 0 && P::zero_transition(tagg);
    if (tile > 0 && tid == 0 && KF_IN(tile < ctl.ntiles, ctl.status)) {
        if (zt) {
            Carry inc;
            P::carry_of(tagg, inc);
            R *dst = static_cast<R *>(ctl.incl) + int64_t(tile) * CS;
#pragma unroll
            for (int i = 0; i < CS; ++i) dst[i] = inc.v[i];
            st_release(ctl.flags + tile, 2);
        } else {
            store_vec(static_cast<R *>(ctl.agg) + int64_t(tile) * ESP, tagg);
            st_release(ctl.flags + tile, 1);
        }
    }
    __syncthreads();
    if (trace) trace[2] = global_ns();

    // ---- 4. look-back
    Carry tc;
    set_zero(tc);
    if (tile > 0) {
        // the first lbw warps take the predecessors: thread tid < 32*lbw takes
        // q = tile-1-(tid*vv + v), v < vv, with vv*32*lbw >= ntiles
        const int lbt = 32 * ctl.lbw;
        const int vv = (ctl.ntiles + lbt - 1) / lbt;
        const bool lbthread = tid < lbt;
        // One warp (the last) waits until every predecessor has published:
        // its lanes read the flags together, back off exponentially between
        // rounds (so the waiting tiles leave the L2 to the tiles still
        // working) and find the nearest predecessor with an inclusive prefix;
        // the rest of the CTA waits at the barrier.
        if (warp == NW - 1) {
            bool ok = true;
            int qloc = -1;
            for (int q0 = tile - 1; q0 >= 0 && ok; q0 -= 32) {
                const int q = q0 - lane;
                int f = q >= 0 && KF_IN(q < ctl.ntiles, ctl.status) ? ld_relaxed(ctl.flags + q) : 1;
                unsigned ns = 32;
                const uint64_t t0 = global_ns();
                while (!__all_sync(0xffffffffu, f != 0)) {
                    __nanosleep(ns);
                    ns = ns < 1024 ? 2 * ns : 1024;
                    if (f == 0) f = ld_relaxed(ctl.flags + q);
                    const bool fail = ld_relaxed(ctl.status) != 0 || int64_t(global_ns() - t0) > ctl.timeout_ns;
                    if (__any_sync(0xffffffffu, fail)) {
                        if (lane == 0) atomicCAS(ctl.status, 0, KF_STATUS_TIMEOUT);
                        ok = false;
                        break;
                    }
                }
                if (q >= 0 && f == 2 && q > qloc) qloc = q;
                // the nearest inclusive prefix ends the search
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
        // the flags were read by another warp: the barrier and an acquire
        // fence order them before the loads of the published aggregates
        if (lbthread) asm volatile("fence.acq_rel.gpu;" ::: "memory");
        if (trace) trace[5] = global_ns();
        const int qstar = s_qstar;
        if (lbthread) {
            // fold the aggregates of my predecessors after qstar, earliest first
            Elem x;
            bool have = false;
#pragma unroll 1
            for (int v = vv - 1; v >= 0; --v) {
                const int q = tile - 1 - (tid * vv + v);
                if (q > qstar) {
                    Elem a;
                    load_cg_vec(a, static_cast<const R *>(ctl.agg) + int64_t(q) * ESP);
                    if (!have) {
                        x = a;
                        have = true;
                    } else {
                        Elem t;
                        P::combine(x, a, t);
                        x = t;
                    }
                }
            }
            if (!have) set_identity(x);
            if (trace) trace[6] = global_ns();
            // lane l covers later tiles than lane l+1: suffix reduction to lane 0
#pragma unroll 1
            for (int s = 1; s < 32; s <<= 1) {
                Elem o, t;
                shfl_down_x(x, o, s);
                if (lane + s < 32) {
                    P::combine(o, x, t);
                    x = t;
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int i = 0; i < ES; ++i) s_red[warp][i] = x.v[i];
            }
        }
        __syncthreads();
        if (trace) trace[7] = global_ns();
        if (warp == 0) {
            Elem y;
            if (lane < ctl.lbw) {
#pragma unroll
                for (int i = 0; i < ES; ++i) y.v[i] = s_red[lane][i];
            } else {
                set_identity(y);
            }
#pragma unroll 1
            for (int s = 1; s < ctl.lbw; s <<= 1) {
                Elem o, t;
                shfl_down_x(y, o, s);
                if (lane + s < ctl.lbw) {
                    P::combine(o, y, t);
                    y = t;
                }
            }
            if (trace) trace[8] = global_ns();
            if (qstar >= 0) load_cg(tc, static_cast<const R *>(ctl.incl) + int64_t(qstar) * CS);
            if (trace) trace[9] = global_ns();
            P::apply(tc, y);
            if (trace) trace[10] = global_ns();
        }
    }
    // ---- 5. publish the inclusive carry
    if (warp == 0) {
        Carry inc = tc;
        P::apply(inc, tagg);
        if (trace) trace[11] = global_ns();
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < CS; ++i) s_carry[i] = tc.v[i];
            if (!zt && KF_IN(tile < ctl.ntiles, ctl.status)) {   // (already published when the transition is zero)
                R *dst = static_cast<R *>(ctl.incl) + int64_t(tile) * CS;
#pragma unroll
                for (int i = 0; i < CS; ++i) dst[i] = inc.v[i];
                __threadfence();
                st_release(ctl.flags + tile, 2);
            }
            if (trace) trace[12] = global_ns();
        }
    }
    __syncthreads();
    if (trace) trace[3] = global_ns();

    // ---- 6. carries and the fused extraction pass
    Carry c;
#pragma unroll
    for (int i = 0; i < CS; ++i) c.v[i] = s_carry[i];
    if (warp > 0) {
        Elem wx;
#pragma unroll
        for (int i = 0; i < ES; ++i) wx.v[i] = s_wx[warp][i];
        P::apply(c, wx);
    }
    if (lane > 0) P::apply(c, lex);
    double ll = 0.0;
    {
        SegCursor cur = P::cursor(args, start < total ? start : total - 1);
        R *oarr[3] = {P::out_arr(args, 0), P::out_arr(args, 1), P::out_arr(args, 2)};
        void *obuf[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) obuf[i] = (ctl.sm_out[i] >= 0 && oarr[i]) ? wsm + ctl.sm_out[i] : nullptr;
        if (P::IN_REC > 0 && in0) {
#pragma unroll
            for (int k = 0; k < NST - 1; ++k) {
                if (k < nchunks)
                    stage_load<C, IRC>(in_arr, seg_first<P, C>(total, start0 + k * C), dK, total, inbuf(k), lane);
                cp_async_commit();
            }
        }
        for (int ch = 0; ch < nchunks; ++ch) {
            if (P::IN_REC > 0 && in0) {
                const int ahead = ch + NST - 1;
                if (ahead < nchunks)
                    stage_load<C, IRC>(in_arr, seg_first<P, C>(total, start0 + ahead * C), dK, total, inbuf(ahead), lane);
                cp_async_commit();
                cp_async_wait<NST - 1>();
                __syncwarp();
            }
            R llc = 0;   // log-likelihood terms of this chunk, summed in the working precision
#pragma unroll 1
            for (int cc = 0; cc < C; ++cc) {
                const int64_t p = start + ch * C + cc;
                if (p >= end) break;
                const int slot = seg_slot<P, C>(cc);
                const int64_t g = gidx<P>(total, p);
                const R *in = !P::IN_REC ? nullptr
                              : in0 ? stage_rec<C, P::IN_REC, R>(inbuf(ch), lane, slot)
                                    : in_arr + g * P::IN_REC;
                R *o1 = obuf[0] ? stage_rec<C, (P::O1 ? P::O1 : 1), R>(obuf[0], lane, slot)
                                : (P::O1 && oarr[0]) ? oarr[0] + g * P::O1 : nullptr;
                R *o2 = obuf[1] ? stage_rec<C, (P::O2 ? P::O2 : 1), R>(obuf[1], lane, slot)
                                : (P::O2 && oarr[1]) ? oarr[1] + g * P::O2 : nullptr;
                R *o3 = obuf[2] ? stage_rec<C, (P::O3 ? P::O3 : 1), R>(obuf[2], lane, slot)
                                : (P::O3 && oarr[2]) ? oarr[2] + g * P::O3 : nullptr;
                if (!KF_IN(g >= 0 && g < total, ctl.status)) continue;
                const R l = P::step_at(args, p, cur, c, in, o1, o2, o3);
                llc += l;
                if (ctl.ll_step) ctl.ll_step[g] = double(l);
            }
            ll += double(llc);   // FP64 accumulation, once per chunk of at most C steps
            __syncwarp();
            const int64_t gs0 = seg_first<P, C>(total, start0 + ch * C);
            if constexpr (P::O1 > 0)
                if (obuf[0]) stage_store<C, P::O1, P::REV>(oarr[0], gs0, start0, ctl.K, total, obuf[0], lane);
            if constexpr (P::O2 > 0)
                if (obuf[1]) stage_store<C, P::O2, P::REV>(oarr[1], gs0, start0, ctl.K, total, obuf[1], lane);
            if constexpr (P::O3 > 0)
                if (obuf[2]) stage_store<C, P::O3, P::REV>(oarr[2], gs0, start0, ctl.K, total, obuf[2], lane);
            __syncwarp();
        }
    }

    if (trace) trace[4] = global_ns();

    // ---- log-likelihood: fixed-order reduction per tile, then over tiles
    if (ctl.ll_out) {
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) ll += __shfl_down_sync(0xffffffffu, ll, s);
        if (lane == 0) s_ll[warp] = ll;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NW; ++w) t += s_ll[w];
            if (KF_IN(tile < ctl.ntiles, ctl.status)) ctl.ll_part[tile] = t;
            __threadfence();
            s_last = (atomicAdd(ctl.counters + 1, 1) == ctl.ntiles - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double t = 0.0;
            for (int i = tid; i < ctl.ntiles; i += THREADS) t += __ldcg(ctl.ll_part + i);
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) t += __shfl_down_sync(0xffffffffu, t, s);
            if (lane == 0) s_ll[warp] = t;
            __syncthreads();
            if (tid == 0) {
                double u = 0.0;
                for (int w = 0; w < NW; ++w) u += s_ll[w];
                *ctl.ll_out = u;
            }
        }
    }
}

}  // namespace kfs

namespace kfs {

// Per-sequence log-likelihood of a batch: one warp per sequence sums its
// per-step terms in a fixed order (lane-strided partial sums, then a fixed
// shuffle tree), so the result does not depend on scheduling.
static __global__ void segmented_ll_kernel(const double *ll_step, const int64_t *offsets, int nseg, double *ll_out) {
    const int warp = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (warp >= nseg) return;
    const int64_t b = offsets[warp], e = offsets[warp + 1];
    double s = 0.0;
    for (int64_t i = b + lane; i < e; i += 32) s += ll_step[i];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if (lane == 0) ll_out[warp] = s;
}

}  // namespace kfs
