// gain_scan.cuh -- the data-dependent half of the filter and RTS scans of a
// time-invariant model, on one sequence, as a single-pass decoupled
// look-back scan of affine maps over warp-sized tiles.
//
// With the (A, C, J) halves of the filtering elements and the (E, L) halves
// of the RTS elements evaluated on the host (gain_tables.h), the prefixes of
// Lemma 1 and the suffixes of Lemma 2 reduce, on the means, to
//   s_j = A_j s_{j-1} + B_j u_j,   j = 1 .. n,
// forward (filter): s_j = xbar_{j|j}, A_j = M_j, B_j = K_j, u_j = y_j,
//   s_0 = m0, n = T;
// reverse (RTS): scan position j is time k = T - j, s_j = xbar_{k|T},
//   A_j = E_k, B_j = G_k, u_j = xbar_{k|k}, s_0 = xbar_{T|T}, n = T - 1.
// Coefficients differ from step to step only at times 1..k0 (the
// "transient"); every other step has the settled (A, B).
//
// The unit of the scan is a warp: a warp-tile of 32 runs of K positions.
//   - bulk warp-tiles hold 32 K settled positions: each lane folds its K
//     positions into phi (its run maps s to A^K s + phi), the warp scans the
//     phi with the matrix powers A^{K s} from the tables, and publishes its
//     aggregate (A^{32K}, phi_w) -- only phi_w, A^{32K} being common to all
//     bulk warp-tiles;
//   - the one transient warp-tile (forward: the first, reverse: the last,
//     each also taking the positions that do not fill a bulk warp-tile)
//     scans explicit (Phi, phi) pairs, the per-lane maps Phi coming from the
//     tables;
//   - warp-tile 0 knows its carry (s_0) and publishes its inclusive value;
//     every other warp-tile composes the aggregates of at most H
//     predecessors (H: the smallest power of A^{32K} below eps^2 of the
//     working precision, beyond which earlier warp-tiles contribute less
//     than rounding) onto the nearest inclusive value it finds, publishes
//     its own inclusive value, and replays its positions from the exact
//     carry, writing the means (staged through shared memory as coalesced
//     stores) and, forward, the log-likelihood terms
//     -1/2 |W_k (y_k - H F xbar_{k-1|k-1})|^2 (the log det S_k terms are a
//     constant the host adds).
// CTA b takes the WPC warp-tiles from WPC b on; after the constant tables
// are in shared memory its warps run independently (no CTA barrier).  A
// warp-tile waits only for lower-indexed ones, held by CTAs the launch
// dispatches earlier (the order single-pass scans rely on); the waits are
// bounded all the same.
// The data-independent covariance output is written by an extra store warp
// per CTA over a fixed slice of the records (bulk copies of the settled
// record from shared memory, table reads near the ends).
// Published vectors are 64-bit words that each carry 32 bits of the value
// and a nonzero tag, so a reader needs no separate flag (one round trip per
// look-back); the words are cleared before every launch.  Every wait is
// bounded by a wall-clock limit; on time-out the warp records
// KF_ERR_TIMEOUT in the status word and returns.
#pragma once

#include "kf_math.cuh"
#include "stage.cuh"

namespace kfs {

// index checks of the bounds-checked build, against this kernel's status word
#define GS_IN(cond) KF_IN(cond, a.status)

// Offsets (in values of type R) into the device tables of one direction.
// The constant block [0, nconst) is copied to shared memory by every CTA.
struct GsOff {
    int nconst;
    int A, B, HF, W;   // settled: A (N x N), B (N x MI), forward H F (M x N), W (M x M, lower)
    int wl, lx, pt;    // powers of the settled A: A^{K 2^i} (5), A^{K l} (32), A^{32 K} (1)
    int cov_i;         // settled covariance out (N x N)
    // outside the constant block (read through the read-only path)
    int tA, tB, tW;    // times 1..k0: [k0][N N], [k0][N MI], forward [k0][M M]
    int gwin;          // transient warp-tile, scan level i, lane l: the map of lanes l - 2^i + 1 .. l [5][32][N N]
    int gexc;          // transient warp-tile: the map of the lanes before lane l [32][N N]
    int gexc0;         // forward: that map applied to m0 [32][N]; and the whole warp-tile's map applied to m0 [N]
    int cov_t, cov_d;  // covariances out: times 1..k0 [k0][N N], reverse: times T - d [kb][N N]
};

template <int N, typename R>
struct GsArgs {
    int64_t T;            // time steps
    int64_t npos;         // scan positions (forward T, reverse T - 1)
    int64_t n0;           // positions of the transient warp-tile (min(k0, npos))
    int K, Kt;            // positions per lane in bulk warp-tiles, in the transient warp-tile
    int nbw, nwt, ncta;   // bulk warp-tiles, warp-tiles, CTAs
    int H;                // look-back depth in warp-tiles (<= 32)
    int k0, kb;
    const R *u;           // forward y [T][M]; reverse filter means [T][N]
    R *out1, *out2;       // means out [T][N] (out2 may be null)
    R *Pout;              // covariances out [T][N][N] or null
    int64_t cov_slice;    // records of the covariance output per CTA (store warp)
    int covbuf;           // bytes of the shared buffer of repeated settled records
    const R *tab;
    GsOff off;
    int *counters;        // [1] finished warp-tiles (zero at launch)
    uint64_t *words;      // warp-tile v: aggregate at words + v * wstride, inclusive NWD words later
    int wstride;
    double *ll_part;      // [nwt]
    double *ll_out;
    double ll_const;
    int want_ll;
    int *status;
    int64_t timeout_ns;
    int inject_skip_tile; // test hook: this warp-tile never publishes
    uint64_t *trace;      // phase trace (kf_trace_phases, one row per warp-tile) or null
    int trace_cap;
    int pdl_wait;         // launched as a programmatic dependent of the kernel that writes u
    int64_t tab_len;      // values of the table from tab on (index checks of a bounds-checked build)
    int64_t wcap;         // warp-tiles the words and ll_part hold
    R s0[N];              // forward: m0
};

KF_D uint64_t gs_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
KF_D int gs_ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bulk copies shared -> global by the tensor memory accelerator (16-byte
// aligned addresses, sizes multiple of 16), marked evict-first in L2 so that
// the streamed output does not displace data the next kernel reads.
KF_D uint64_t gs_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
KF_D void gs_bulk_store(void *gdst, const void *ssrc, uint32_t bytes, uint64_t pol) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, %3;" ::"l"(gdst),
                 "r"(smem_addr(ssrc)), "r"(bytes), "l"(pol)
                 : "memory");
}
KF_D void gs_bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
KF_D void gs_bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
KF_D void gs_fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// A published vector: 32 bits of the value per 64-bit word, the high half a
// nonzero tag; a word is read whole, so a tagged word is a written word.
template <int N, typename R>
struct GsWords {
    static constexpr int NWD = N * int(sizeof(R)) / 4;
};
template <int N, typename R>
KF_D void gs_put(uint64_t *w, const R *v) {
    constexpr int NWD = GsWords<N, R>::NWD;
    uint32_t bits[NWD];
    memcpy(bits, v, sizeof(bits));
#pragma unroll
    for (int i = 0; i < NWD; ++i) {
        const uint64_t word = (uint64_t(1) << 32) | bits[i];
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(w + i), "l"(word) : "memory");
    }
}
template <int N, typename R>
KF_D bool gs_get(const uint64_t *w, R *v) {
    constexpr int NWD = GsWords<N, R>::NWD;
    uint32_t bits[NWD];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < NWD; ++i) {
        uint64_t word;
        asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(word) : "l"(w + i) : "memory");
        ok = ok && (word >> 32) != 0;
        bits[i] = uint32_t(word);
    }
    memcpy(v, bits, sizeof(bits));
    return ok;
}

// out = A s + B u (A N x N, B N x MI; any address space); out may alias s
template <int N, int MI, typename R>
KF_D void gs_affine(const R *A, const R *B, const R *s, const R *u, R *out) {
    R t[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R acc = 0;
#pragma unroll
        for (int j = 0; j < MI; ++j) acc += B[r * MI + j] * u[j];
#pragma unroll
        for (int k = 0; k < N; ++k) acc += A[r * N + k] * s[k];
        t[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < N; ++r) out[r] = t[r];
}

// v <- X v + w, X in registers
template <int N, typename R>
KF_D void gs_mva(const R *X, R *v, const R *w) {
    R t[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R acc = w[r];
#pragma unroll
        for (int k = 0; k < N; ++k) acc += X[r * N + k] * v[k];
        t[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < N; ++r) v[r] = t[r];
}
// v <- X v + w, X an N x N matrix in shared memory on a 16-byte boundary
// (read row by row with vector loads)
template <int N, typename R>
KF_D void gs_mva_s(const R *X, R *v, const R *w) {
    R t[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
        R row[N];
        load_rec<N>(row, X + r * N);
        R acc = w[r];
#pragma unroll
        for (int k = 0; k < N; ++k) acc += row[k] * v[k];
        t[r] = acc;
    }
#pragma unroll
    for (int r = 0; r < N; ++r) v[r] = t[r];
}

// Per-warp dynamic shared memory: a ring of NST input buffers and (when the
// input records are not the size of the outputs) one output buffer of the
// means, each of 32 runs x C records.  A run of at most NST x C positions
// stays staged from the fold to the replay.
template <int N, int MI, typename R>
struct GsStage {
    static constexpr int C = (MI * int(sizeof(R)) <= 16 && N * int(sizeof(R)) <= 16) ? 4 : 2;
    static constexpr int NST = 4;
    static constexpr int KS = NST * C;   // positions per lane that stay staged
    using WI = WarpStage<C, MI, R>;
    using WO = WarpStage<C, N, R>;
    static constexpr int IB = (WI::BYTES + 15) / 16 * 16;
    // outputs are staged in their input's slot when both are N values
    static constexpr bool INPLACE = MI == N;
    static constexpr int OB = INPLACE ? 0 : (WO::BYTES + 15) / 16 * 16;
    static constexpr int WARP = NST * IB + OB;
};

// Issue the asynchronous loads of one chunk (C records) of the 32 runs of a
// warp: run r's chunk starts at record base + r * dK (its records ascending
// from there); records outside [0, T) are skipped.  A lane moves the same
// unit o of runs lane / SEGU, + 32 / SEGU, ... (SEGU, the units of a run's
// chunk, divides 32).
template <int C, int REC, typename R>
KF_D void gs_stage_load(const R *u, int64_t base, int dK, int64_t T, void *buf, int lane) {
    using W = WarpStage<C, REC, R>;
    using UT = typename UnitT<W::U>::T;
    constexpr int SEGU = W::SEGU, PER = 32 / SEGU;
    static_assert(32 % SEGU == 0, "units of a run's chunk divide 32");
    const int o = lane % SEGU, run0 = lane / SEGU;
    const int64_t rec0 = base + int64_t(run0) * dK + o / W::RU;
    const UT *g = reinterpret_cast<const UT *>(u) + rec0 * W::RU + o % W::RU;
    UT *sp = static_cast<UT *>(buf) + run0 * W::STRIDE + o;
    const int64_t step = int64_t(PER) * dK;
#pragma unroll
    for (int j = 0; j < SEGU; ++j) {
        const int64_t rec = rec0 + j * step;
        if (rec >= 0 && rec < T) cp_async_unit<W::U>(sp + j * PER * W::STRIDE, g + j * step * W::RU);
    }
}

// The covariance of record r (time r + 1) from the tables.
template <int N, typename R, bool REV>
KF_D const R *gs_cov_src(const GsArgs<N, R> &a, int64_t r) {
    const int64_t k = r + 1;
    if (k <= a.k0) return a.tab + a.off.cov_t + (k - 1) * N * N;
    if (REV && a.T - k < a.kb) return a.tab + a.off.cov_d + (a.T - k) * N * N;
    return a.tab + a.off.cov_i;
}

// Records [r0, r1) of the covariance output from the tables, by the 32
// lanes of a warp as consecutive 16-byte units.
template <int N, typename R, bool REV>
KF_D void gs_store_cov(const GsArgs<N, R> &a, int64_t r0, int64_t r1, int lane) {
    constexpr int UPR = N * N * int(sizeof(R)) / 16;   // 16-byte units per record: 1 .. 32, divides 32
    static_assert(UPR >= 1 && 32 % UPR == 0, "covariance record of 16 .. 512 bytes");
    float4 *g = reinterpret_cast<float4 *>(a.Pout);
    const int part = lane % UPR;
    for (int64_t i = lane; i < (r1 - r0) * UPR; i += 32) {
        const int64_t r = r0 + i / UPR;
        const R *src = gs_cov_src<N, R, REV>(a, r);
        if (!GS_IN(r >= 0 && r < a.T && src >= a.tab && src + N * N <= a.tab + a.tab_len)) continue;
        const float4 v = __ldg(reinterpret_cast<const float4 *>(src) + part);
        __stcs(g + r0 * UPR + i, v);
    }
}

// The store warp of a CTA: the covariance output of records
// [b slice, (b + 1) slice), the settled run by bulk copies of the repeated
// settled record, the records near the ends from the tables.
template <int N, typename R, bool REV>
KF_D void gs_store_warp(const GsArgs<N, R> &a, unsigned char *cbuf, int lane) {
    constexpr int NN = N * N, UPR = NN * int(sizeof(R)) / 16;
    const int64_t r0 = int64_t(blockIdx.x) * a.cov_slice;
    const int64_t r1 = r0 + a.cov_slice < a.T ? r0 + a.cov_slice : a.T;
    if (r1 <= r0) return;
    int64_t sa = r0 > a.k0 ? r0 : a.k0, sb = r1;   // settled: time > k0 and, reverse, T - time >= kb
    if (REV && sb > a.T - a.kb) sb = a.T - a.kb;
    if (sb < sa) sb = sa;
    {
        float4 *dst = reinterpret_cast<float4 *>(cbuf);
        const float4 *src = reinterpret_cast<const float4 *>(a.tab + a.off.cov_i);
        for (int i = lane; i < a.covbuf / 16; i += 32) dst[i] = __ldg(src + i % UPR);
        gs_fence_async_shared();
        __syncwarp();
    }
    if (lane == 0 && sb > sa && GS_IN(sa >= 0 && sb <= a.T)) {
        constexpr int64_t REC = NN * int64_t(sizeof(R));
        const uint64_t pol = gs_evict_first_policy();
        char *g = reinterpret_cast<char *>(a.Pout) + sa * REC;
        for (int64_t left = (sb - sa) * REC; left > 0;) {
            const uint32_t b = uint32_t(left < a.covbuf ? left : a.covbuf);
            gs_bulk_store(g, cbuf, b, pol);
            g += b;
            left -= b;
        }
        gs_bulk_commit();
    }
    const int64_t e1 = sa < r1 ? sa : r1;   // [r0, e1) before the settled run, [b2, r1) after it
    if (e1 > r0) gs_store_cov<N, R, REV>(a, r0, e1, lane);
    const int64_t b2 = sb > e1 ? sb : e1;
    if (r1 > b2) gs_store_cov<N, R, REV>(a, b2, r1, lane);
    if (lane == 0) gs_bulk_wait_read();   // the shared buffer outlives its bulk copies
}

// WPC compute warps per CTA (WPC consecutive warp-tiles per ticket); with
// STOREW one more warp writes the covariance output.
template <int N, int MI, typename R, bool REV, int WPC, int MINB, bool STOREW>
__global__ void __launch_bounds__(32 * WPC + (STOREW ? 32 : 0), MINB)
    gs_kernel(const __grid_constant__ GsArgs<N, R> a) {
    constexpr int NN = N * N, M = N / 2, NWD = GsWords<N, R>::NWD;
    using GS = GsStage<N, MI, R>;
    using WO = typename GS::WO;
    constexpr int C = GS::C, NST = GS::NST;
    constexpr bool REG = N <= 4;   // settled coefficients held in registers

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ __align__(16) unsigned char dsm[];
    const R *const sc = reinterpret_cast<const R *>(dsm);   // the constant block
    const int cunits = (a.off.nconst * int(sizeof(R)) + 15) / 16;
    unsigned char *const cbuf = dsm + 16 * cunits;          // repeated settled covariance record
    unsigned char *const wbase = cbuf + (STOREW ? a.covbuf : 0) + warp * GS::WARP;
    unsigned char *const obuf = wbase + NST * GS::IB;
    const R *const sA = sc + a.off.A, *const sB = sc + a.off.B;
    const R *const sHF = sc + a.off.HF, *const sW = sc + a.off.W, *const sPT = sc + a.off.pt;

    // a dependent kernel (the RTS pass after the filter) may be scheduled
    // as this grid's CTAs retire; it waits for this grid before reading it
    if (tid == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (warp < WPC && GS_IN(int64_t(cunits) * 16 <= a.tab_len * int64_t(sizeof(R)))) {
        for (int i = tid; i < cunits; i += 32 * WPC)
            cp_async_unit<16>(dsm + 16 * i, reinterpret_cast<const unsigned char *>(a.tab) + 16 * i);
    }
    cp_async_commit();

    // ---- geometry of warp-tile v: positions [t_lo, t_hi], lane runs of Kc
    const int64_t Lw = int64_t(32) * a.K;
    bool gen = false;
    int Kc = 0, cnt = 0, nch = 0;
    int64_t t_lo = 0, t_hi = 0, pme = 0;   // (the last settled warp-tile may be short)
    const int64_t ns = a.npos - a.n0;   // settled positions
    auto geom = [&](int v) {
        gen = REV ? (v == a.nbw) : (v == 0);
        Kc = gen ? a.Kt : a.K;
        if constexpr (!REV) {   // the transient first, then the settled positions
            t_lo = gen ? 1 : a.n0 + int64_t(v - 1) * Lw + 1;
            t_hi = gen ? a.n0 : (t_lo + Lw - 1 < a.npos ? t_lo + Lw - 1 : a.npos);
        } else {                // the settled positions, then the transient
            t_lo = gen ? ns + 1 : int64_t(v) * Lw + 1;
            t_hi = gen ? a.npos : (t_lo + Lw - 1 < ns ? t_lo + Lw - 1 : ns);
        }
        pme = t_lo + int64_t(lane) * Kc;
        cnt = int(t_hi + 1 - pme < 0 ? 0 : (t_hi + 1 - pme > Kc ? Kc : t_hi + 1 - pme));
        nch = (Kc + C - 1) / C;   // the same for every lane of the warp-tile
    };
    auto ibuf = [&](int ch) { return wbase + (ch % NST) * GS::IB; };
    auto load_chunk = [&](int ch) {
        if constexpr (!REV) gs_stage_load<C, MI, R>(a.u, t_lo - 1 + int64_t(ch) * C, Kc, a.T, ibuf(ch), lane);
        else gs_stage_load<C, MI, R>(a.u, a.T - t_lo - int64_t(ch + 1) * C, -Kc, a.T, ibuf(ch), lane);
    };
    auto slot = [&](int cc) { return REV ? C - 1 - cc : cc; };
    auto load_first = [&](bool on) {   // NST - 1 commit groups in every case
#pragma unroll
        for (int k = 0; k < NST - 1; ++k) {
            if (on && k < nch) load_chunk(k);
            cp_async_commit();
        }
    };
    if constexpr (STOREW) {
        if (warp == WPC) {   // the store warp (its output does not depend on a preceding kernel)
            cp_async_wait<0>();
            gs_store_warp<N, R, REV>(a, cbuf, lane);
            return;
        }
    }
    // launched as a dependent of the filter kernel (programmatic dependent
    // launch): wait for it to complete before reading its means; a no-op
    // otherwise
    if (a.pdl_wait) asm volatile("griddepcontrol.wait;" ::: "memory");
    const int v = int(blockIdx.x) * WPC + warp;
    const bool active = v < a.nwt;
    if (active) geom(v);
    load_first(active);
    cp_async_wait<NST - 1>();   // this thread's part of the constant block
    asm volatile("bar.sync 1, %0;" ::"n"(32 * WPC) : "memory");   // every compute warp's
    if (!active || v == a.inject_skip_tile) {
        cp_async_wait<0>();
        return;
    }
    // phase trace (one row per warp-tile): 0 start, 2 fold done, 3 scanned and
    // published, 4 carry known, 5 replay done, 6 end
    uint64_t *const trace = (a.trace && v < a.trace_cap && lane == 0) ? a.trace + 16 * int64_t(v) : nullptr;
    if (trace) trace[0] = gs_ns();
    const bool restage = nch > NST;   // the replay reloads its inputs
    // a short last settled warp-tile: its lanes past the end are empty, so the
    // uniform powers do not give its aggregate; in the reverse scan (where
    // the transient warp-tile reads it) it publishes its inclusive value from
    // the replay instead
    const bool ragged = !gen && t_hi - t_lo + 1 < Lw;

    // settled coefficients: registers (nx <= 4) or shared memory
    R rA[REG ? NN : 1], rB[REG ? N * MI : 1];
    if constexpr (REG) {
        load_rec<NN>(rA, sA);
#pragma unroll
        for (int i = 0; i < N * MI; ++i) rB[i] = sB[i];
    }
    // coefficients of position j of the transient warp-tile: those of its
    // time when it lies in 1..k0, else the settled ones
    auto coef = [&](int64_t j, const R *&A, const R *&B, const R *&Wk) {
        const int64_t tk = REV ? a.T - j : j;
        if (tk <= a.k0 && GS_IN(tk >= 1 && a.off.tB + tk * N * MI <= a.tab_len && a.off.tA + tk * NN <= a.tab_len)) {
            A = a.tab + a.off.tA + (tk - 1) * NN;
            B = a.tab + a.off.tB + (tk - 1) * N * MI;
            Wk = REV ? sW : a.tab + a.off.tW + (tk - 1) * M * M;
        } else {
            A = sA;
            B = sB;
            Wk = sW;
        }
    };

    // ---- 1. fold of each lane's run
    R phi[N];
#pragma unroll
    for (int i = 0; i < N; ++i) phi[i] = 0;
#pragma unroll 1
    for (int ch = 0; ch < nch; ++ch) {
        if (ch + NST - 1 < nch) load_chunk(ch + NST - 1);
        cp_async_commit();
        cp_async_wait<NST - 1>();
        __syncwarp();
#pragma unroll
        for (int cc = 0; cc < C; ++cc) {
            const int c = ch * C + cc;
            if (c >= cnt) break;
            R u[MI];
            load_rec<MI>(u, stage_rec<C, MI, R>(ibuf(ch), lane, slot(cc)));
            if (gen) {
                const R *A, *B, *Wk;
                coef(pme + c, A, B, Wk);
                gs_affine<N, MI, R>(A, B, phi, u, phi);
            } else if constexpr (REG) {
                gs_affine<N, MI, R>(rA, rB, phi, u, phi);
            } else {
                gs_affine<N, MI, R>(sA, sB, phi, u, phi);
            }
        }
        __syncwarp();
    }
    cp_async_wait<0>();
    __syncwarp();
    if (trace) trace[2] = gs_ns();

    // ---- 2. warp scan: psi = this lane's exclusive vector, wp = the warp-tile's aggregate
    R psi[N], wp[N];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int s = 1 << i;
        R x[N];
#pragma unroll
        for (int k = 0; k < N; ++k) x[k] = __shfl_up_sync(0xffffffffu, phi[k], s);
        if (lane >= s) {   // phi <- (map of this lane's window) x + phi
            if (gen) {
                R Wm[NN];
                const R *g = a.tab + a.off.gwin + (i * 32 + lane) * NN;
                if (!GS_IN(a.off.gwin + (i * 32 + lane + 1) * int64_t(NN) <= a.tab_len)) g = a.tab;
#pragma unroll
                for (int k = 0; k < NN; ++k) Wm[k] = __ldg(g + k);
                gs_mva<N, R>(Wm, x, phi);
            } else {
                gs_mva_s<N, R>(sc + a.off.wl + i * NN, x, phi);   // A^{K s}
            }
#pragma unroll
            for (int k = 0; k < N; ++k) phi[k] = x[k];
        }
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        wp[i] = __shfl_sync(0xffffffffu, phi[i], 31);
        const R e = __shfl_up_sync(0xffffffffu, phi[i], 1);
        psi[i] = lane ? e : R(0);
    }

    // ---- 3. publish: warp-tile 0 its inclusive value (its carry s_0 is
    // known), a bulk warp-tile its aggregate; 4. the carry c
    R c[N];
    uint64_t *const myw = a.words + int64_t(v) * a.wstride;
    if (!GS_IN(v < a.wcap)) return;
    if (v == 0) {
        if constexpr (!REV) {
#pragma unroll
            for (int k = 0; k < N; ++k) c[k] = a.s0[k];
        } else {
            load_rec<N>(c, a.u + (a.T - 1) * N);   // xbar_{T|T}
        }
        if (a.nwt > 1) {
            R t[N];
            if (gen) {   // forward: (the warp-tile's map) m0 from the tables, + wp
                const R *g = a.tab + a.off.gexc0 + 32 * N;
#pragma unroll
                for (int k = 0; k < N; ++k) t[k] = __ldg(g + k) + wp[k];
            } else {
#pragma unroll
                for (int k = 0; k < N; ++k) t[k] = c[k];
                gs_mva_s<N, R>(sPT, t, wp);
            }
            if (lane == 0) gs_put<N, R>(myw + NWD, t);
        }
        if (trace) trace[3] = trace[4] = gs_ns();
    } else {
        if (!gen && !ragged && lane == 0) gs_put<N, R>(myw, wp);
        if (trace) trace[3] = gs_ns();
        // look-back: lane l reads warp-tile v - 1 - l, l < n; the nearest
        // published inclusive value and the aggregates after it
        const int n = v < a.H ? v : a.H;
        const uint64_t *qw = a.words + (int64_t(v) - 1 - lane) * a.wstride;
        R vi[N], va[N];
        bool hi = false, ha = false, ok = true;
        int qlane = -1;
        unsigned ns = 32;
        const uint64_t t0 = gs_ns();
        const unsigned all = n >= 32 ? 0xffffffffu : (1u << n) - 1u;
        for (;;) {
            if (lane < n && !hi && GS_IN(int64_t(v) - 1 - lane >= 0)) {
                hi = gs_get<N, R>(qw + NWD, vi);
                if (!hi && !ha) ha = gs_get<N, R>(qw, va);
            }
            const unsigned im = __ballot_sync(0xffffffffu, lane < n && hi);
            const unsigned rm = __ballot_sync(0xffffffffu, lane < n && (hi || ha));
            const unsigned need = im ? (1u << (__ffs(im) - 1)) - 1u : all;
            if ((rm & need) == need) {
                qlane = im ? __ffs(im) - 1 : -1;
                break;
            }
            __nanosleep(ns);
            ns = ns < 1024 ? 2 * ns : 1024;
            const bool fail = gs_ld_relaxed(a.status) != 0 || int64_t(gs_ns() - t0) > a.timeout_ns;
            if (__any_sync(0xffffffffu, fail)) {
                if (lane == 0) atomicCAS(a.status, 0, 5);   // KF_ERR_TIMEOUT (kept if already set)
                ok = false;
                break;
            }
        }
        if (!ok) return;
        // c = incl_{q*} (or 0 past the depth H), then c <- A^{32K} c + agg_q for the later warp-tiles
#pragma unroll
        for (int k = 0; k < N; ++k) c[k] = qlane >= 0 ? __shfl_sync(0xffffffffu, vi[k], qlane) : R(0);
        for (int l = (qlane >= 0 ? qlane : n) - 1; l >= 0; --l) {
            R w[N];
#pragma unroll
            for (int k = 0; k < N; ++k) w[k] = __shfl_sync(0xffffffffu, va[k], l);
            gs_mva_s<N, R>(sPT, c, w);
        }
        if (!gen && !ragged && v + 1 < a.nwt) {   // this warp-tile's inclusive value
            R t[N];
#pragma unroll
            for (int k = 0; k < N; ++k) t[k] = c[k];
            gs_mva_s<N, R>(sPT, t, wp);
            if (lane == 0) gs_put<N, R>(myw + NWD, t);
        }
        if (trace) trace[4] = gs_ns();
    }
    if (REV && v == 0 && lane == 0) {   // time T: xbar_{T|T}
        store_rec<N>(a.out1 + (a.T - 1) * N, c);
        if (a.out2) store_rec<N>(a.out2 + (a.T - 1) * N, c);
    }

    // ---- 5. this lane's start: the warp-tile's carry through the lanes before it
    R s[N];
    if (gen && !REV) {   // forward: (the lanes' map) m0 from the tables, + psi
        const R *g = a.tab + a.off.gexc0 + lane * N;
#pragma unroll
        for (int k = 0; k < N; ++k) s[k] = __ldg(g + k) + psi[k];
    } else if (gen) {
        R Em[NN];
        const R *g = a.tab + a.off.gexc + lane * NN;
#pragma unroll
        for (int k = 0; k < NN; ++k) Em[k] = __ldg(g + k);
#pragma unroll
        for (int k = 0; k < N; ++k) s[k] = c[k];
        gs_mva<N, R>(Em, s, psi);
    } else {
#pragma unroll
        for (int k = 0; k < N; ++k) s[k] = c[k];
        gs_mva_s<N, R>(sc + a.off.lx + lane * NN, s, psi);   // s <- A^{K l} c + psi_l
    }

    // ---- 6. replay the positions from the exact carry, emit
    double ll = 0.0;
    {
        if (restage) load_first(true);
        R *const ob = reinterpret_cast<R *>(obuf) + lane * WO::RSTRIDE;
        using UT = typename UnitT<WO::U>::T;
        // the warp's records relative to rbase: run r's record of slot o at
        // rbase + r dR + ch C + slot (forward dR = Kc; reverse dR = -Kc, rbase
        // already at the chunk's lowest record)
        const int64_t rbase = REV ? a.T - t_lo - C : t_lo - 1;
        const int dR = REV ? -Kc : Kc;
        UT *const g1 = reinterpret_cast<UT *>(a.out1) + rbase * WO::RU;
        UT *const g2 = a.out2 ? reinterpret_cast<UT *>(a.out2) + rbase * WO::RU : nullptr;
        const int rem0 = int(t_hi + 1 - t_lo);   // positions of the warp-tile
        // the store of each chunk: this lane moves unit o of runs run0 + j 32 / SEGU
        static_assert(32 % WO::SEGU == 0, "units of a run's chunk divide 32");
        const int st_o = lane % WO::SEGU, st_run0 = lane / WO::SEGU, st_sl = st_o / WO::RU;
        const int st_off = REV ? C - 1 - st_sl : st_sl;
        const int st_rel = (st_run0 * dR + st_sl) * WO::RU + st_o % WO::RU;
        const int st_soff = st_run0 * WO::STRIDE + st_o;
        int st_rc[WO::SEGU];   // positions of each of those runs
#pragma unroll
        for (int j = 0; j < WO::SEGU; ++j) {
            const int rc = rem0 - (st_run0 + j * (32 / WO::SEGU)) * Kc;
            st_rc[j] = rc < 0 ? 0 : (rc > Kc ? Kc : rc);
        }
#pragma unroll 1
        for (int ch = 0; ch < nch; ++ch) {
            if (restage) {
                if (ch + NST - 1 < nch) load_chunk(ch + NST - 1);
                cp_async_commit();
                cp_async_wait<NST - 1>();
                __syncwarp();
            }
            R llc = 0;
#pragma unroll
            for (int cc = 0; cc < C; ++cc) {
                const int cpos = ch * C + cc;
                if (cpos >= cnt) break;
                R u[MI];
                load_rec<MI>(u, stage_rec<C, MI, R>(ibuf(ch), lane, slot(cc)));
                // log-likelihood term: v = y_k - H F xbar_{k-1|k-1}, |W_k v|^2
                auto llterm = [&](const R *Wk) {
                    if constexpr (!REV) {
                        R e[M];
#pragma unroll
                        for (int i = 0; i < M; ++i) {
                            R acc = u[i];
#pragma unroll
                            for (int k = 0; k < N; ++k) acc -= sHF[i * N + k] * s[k];
                            e[i] = acc;
                        }
#pragma unroll
                        for (int i = 0; i < M; ++i) {
                            R acc = 0;
#pragma unroll
                            for (int k = 0; k <= i; ++k) acc += Wk[i * M + k] * e[k];
                            llc += acc * acc;
                        }
                    }
                };
                if (gen) {
                    const R *A, *B, *Wk;
                    coef(pme + cpos, A, B, Wk);
                    if (!REV && a.want_ll) llterm(Wk);
                    gs_affine<N, MI, R>(A, B, s, u, s);
                } else {
                    if (!REV && a.want_ll) llterm(sW);
                    if constexpr (REG) gs_affine<N, MI, R>(rA, rB, s, u, s);
                    else gs_affine<N, MI, R>(sA, sB, s, u, s);
                }
                if constexpr (GS::INPLACE) store_rec<N>(stage_rec<C, MI, R>(ibuf(ch), lane, slot(cc)), s);
                else store_rec<N>(ob + slot(cc) * N, s);
            }
            ll += double(llc);
            __syncwarp();
            // the chunk of every run of the warp, coalesced (the same unit o
            // of runs run0, run0 + 32 / SEGU, ... for this lane)
            const UT *sb = reinterpret_cast<const UT *>(GS::INPLACE ? ibuf(ch) : obuf) + st_soff;
            UT *const gc = g1 + st_rel + (REV ? -ch * C : ch * C) * WO::RU;
            UT *const gc2 = g2 ? g2 + st_rel + (REV ? -ch * C : ch * C) * WO::RU : nullptr;
            const int offc = ch * C + st_off;   // this unit's record offset in its run
#pragma unroll
            for (int j = 0; j < WO::SEGU; ++j) {
                const int d = j * (32 / WO::SEGU) * dR * WO::RU;
                // (the record stored: rbase + (run0 + j 32 / SEGU) dR + slot +- ch C)
                if (offc < st_rc[j] &&
                    GS_IN(rbase + (st_run0 + j * (32 / WO::SEGU)) * dR + st_sl + (REV ? -ch * C : ch * C) >= 0 &&
                          rbase + (st_run0 + j * (32 / WO::SEGU)) * dR + st_sl + (REV ? -ch * C : ch * C) < a.T)) {
                    const UT val = sb[j * (32 / WO::SEGU) * WO::STRIDE];
                    if constexpr (REV) __stcs(gc + d, val);   // the smoothed means: streamed out
                    else gc[d] = val;                          // the filter means: read next by the RTS pass
                    if (gc2) gc2[d] = val;
                }
            }
            __syncwarp();
        }
        if (restage) cp_async_wait<0>();
        // a short reverse warp-tile: the lane with its last position publishes
        // the inclusive value
        if (REV && ragged && v + 1 < a.nwt && cnt > 0 && pme + cnt - 1 == t_hi) gs_put<N, R>(myw + NWD, s);
    }
    if (trace) trace[5] = gs_ns();

    // ---- log-likelihood: fixed-order sums per warp-tile, then over warp-tiles
    if constexpr (!REV) {
        if (a.ll_out) {
#pragma unroll
            for (int s2 = 16; s2 > 0; s2 >>= 1) ll += __shfl_down_sync(0xffffffffu, ll, s2);
            int last = 0;
            if (lane == 0 && GS_IN(v < a.wcap)) {
                a.ll_part[v] = ll;
                __threadfence();
                last = atomicAdd(a.counters + 1, 1) == a.nwt - 1;
            }
            if (__shfl_sync(0xffffffffu, last, 0)) {
                __threadfence();
                double t = 0.0;
                for (int i = lane; i < a.nwt; i += 32) t += __ldcg(a.ll_part + i);
#pragma unroll
                for (int s2 = 16; s2 > 0; s2 >>= 1) t += __shfl_down_sync(0xffffffffu, t, s2);
                if (lane == 0) *a.ll_out = -0.5 * t + a.ll_const;
            }
        }
    }
    if (trace) trace[6] = gs_ns();
}

}  // namespace kfs
