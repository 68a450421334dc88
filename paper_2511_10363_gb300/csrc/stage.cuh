// stage.cuh -- warp-cooperative staging of per-thread record runs through
// shared memory.
//
// In the scans every thread owns a run of consecutive time steps, so the 32
// lanes of a warp touch 32 runs that are far apart in memory: a direct
// per-thread access would make each warp-wide load or store touch 32
// different lines.  Here a warp moves the next C records of all 32 runs at
// once: the records of one run are contiguous in device memory, so
// consecutive lanes move consecutive U-byte units of one run (coalesced),
// loads go through cp.async (L2 -> shared, no register round trip) so that
// the next chunk can be in flight while the current one is computed, and
// stores are plain vector stores from shared memory.
//
// Shared layout of one warp's buffer: run s (the run of lane s) starts at
// unit s * STRIDE, record r of it at unit s * STRIDE + r * RU; STRIDE is odd
// so that the 32 lanes reading "their" record c hit distinct banks.
#pragma once

#include "kf_math.cuh"

namespace kfs {

template <int REC, typename R>
struct RecGeom {
    static constexpr int BYTES = REC * int(sizeof(R));
    static constexpr int U = (BYTES % 16 == 0) ? 16 : (BYTES % 8 == 0) ? 8 : 4;   // unit bytes
    static constexpr int RU = BYTES / U;                                          // units per record
};

// Depth of the input pipeline: a warp keeps NST - 1 chunks of input records
// in flight while it computes on one.  Measured on GB300 (T = 2^20, 2^22):
// the forward pass (small y records, chunks of up to 4 steps) is fastest
// with 4 stages, the reverse passes (64-byte filter records, one step per
// chunk) with 5.
#ifndef KF_STAGE_NST
#define KF_STAGE_NST(kind) ((kind) == 0 ? 4 : 5)
#endif
template <class P>
constexpr int stage_nst() { return KF_STAGE_NST(P::KIND); }

template <int C, int REC, typename R>
struct WarpStage {
    using G = RecGeom<REC, R>;
    static constexpr int U = G::U, RU = G::RU;
    static constexpr int SEGU = C * RU;                          // units per run
    static constexpr int STRIDE = SEGU | 1;                      // odd stride (units)
    static constexpr int BYTES = 32 * STRIDE * U;                // one buffer
    static constexpr int RSTRIDE = STRIDE * U / int(sizeof(R));  // per-run stride in R elements
};

KF_D uint32_t smem_addr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

template <int U>
KF_D void cp_async_unit(void *dst_smem, const void *src) {
    if constexpr (U == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src) : "memory");
    else if constexpr (U == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst_smem)), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst_smem)), "l"(src) : "memory");
}
KF_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
KF_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int U>
struct UnitT;
template <>
struct UnitT<16> { using T = float4; };
template <>
struct UnitT<8> { using T = float2; };
template <>
struct UnitT<4> { using T = float; };

// The runs of a warp: lane r's run starts at scan position start0 + r K, and
// its segment of the current chunk begins at global record gs0 + r dK
// (dK = K for a forward scan, -K for a reverse one).  Computing these per
// unit replaces a shuffle of the owner lane's values.

// Issue the asynchronous load of the C records of every lane's run segment;
// records outside [0, total) are skipped.  `buf` is this warp's buffer.
template <int C, int REC, typename R>
KF_D void stage_load(const R *gbase, int64_t gs0, int64_t dK, int64_t total, void *buf, int lane) {
    using W = WarpStage<C, REC, R>;
    using UT = typename UnitT<W::U>::T;
    const UT *g = reinterpret_cast<const UT *>(gbase);
    UT *s = static_cast<UT *>(buf);
#pragma unroll 4
    for (int idx = lane; idx < 32 * W::SEGU; idx += 32) {
        const int run = idx / W::SEGU, o = idx - run * W::SEGU;
        const int64_t rec = gs0 + run * dK + o / W::RU;
        if (rec >= 0 && rec < total) cp_async_unit<W::U>(s + run * W::STRIDE + o, g + rec * W::RU + o % W::RU);
    }
}

// Store the staged records of every lane's run segment that lie in that
// lane's own global record range (the records of positions
// [start, min(start + K, total)) of its run), coalesced.
template <int C, int REC, bool REV, typename R>
KF_D void stage_store(R *gbase, int64_t gs0, int64_t start0, int64_t K, int64_t total, const void *buf, int lane) {
    using W = WarpStage<C, REC, R>;
    using UT = typename UnitT<W::U>::T;
    UT *g = reinterpret_cast<UT *>(gbase);
    const UT *s = static_cast<const UT *>(buf);
#pragma unroll 4
    for (int idx = lane; idx < 32 * W::SEGU; idx += 32) {
        const int run = idx / W::SEGU, o = idx - run * W::SEGU;
        const int64_t st = start0 + run * K;
        int64_t lo, hi;
        if constexpr (REV) {
            hi = total - st;
            lo = hi - K > 0 ? hi - K : 0;
        } else {
            lo = st;
            hi = st + K < total ? st + K : total;
        }
        const int64_t rec = gs0 + (REV ? -run * K : run * K) + o / W::RU;
        if (rec >= lo && rec < hi) g[rec * W::RU + o % W::RU] = s[run * W::STRIDE + o];
    }
}

// This lane's record r inside a warp buffer.
template <int C, int REC, typename R>
KF_D R *stage_rec(void *buf, int lane, int r) {
    using W = WarpStage<C, REC, R>;
    return static_cast<R *>(buf) + lane * W::RSTRIDE + r * REC;
}

}  // namespace kfs
