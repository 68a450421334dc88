// rts_launch.cuh -- host side of the RTS smoother pass kernel (rts_scan.cuh):
// the tile plan and the launch.  Included by the per-(nx, precision) units
// ti_n<N>_<p>.cu.
#pragma once

#include "kf_launch.cuh"
#include "rts_scan.cuh"

namespace kfs {

template <int N, typename R, int THREADS>
struct RsCfg {
    static constexpr int CH = 2;                                   // steps per staged output chunk
    static constexpr int MINB = THREADS == 256 ? 2 : (sizeof(R) == 4 ? 4 : 3);
    static constexpr int SMEM = RsSmem<N, R, THREADS, CH>::BYTES;
};

// Resident CTAs on the device (occupancy query, cached per device).
template <int N, typename R, int THREADS>
static int rs_resident(int dev) {
    using CF = RsCfg<N, R, THREADS>;
    static std::mutex mu;
    static int val[64];
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return 0;
    if (val[dev] == 0) {
        auto kern = rts_kernel<N, R, THREADS, CF::CH, CF::MINB>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::SMEM) != cudaSuccess)
            return 0;
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, THREADS, CF::SMEM) != cudaSuccess || per < 1)
            return 0;
        val[dev] = sms * per;
    }
    return val[dev];
}

// Launches the RTS pass over the filter records in the workspace.  Returns
// false, with nothing enqueued, when the call does not qualify (then the
// generic kernel runs it); *err carries the launch status otherwise.
template <int N, typename R, int THREADS>
static bool rts_run(const FiltParams<N, R> &prm, const LaunchReq &q, const KfBufs<R> &buf, char *ws,
                    const WsLayout &L, cudaError_t *err) {
    using CF = RsCfg<N, R, THREADS>;
    constexpr int S = N * (N + 1) / 2;
    *err = cudaSuccess;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const int resident = rs_resident<N, R, THREADS>(dev);
    if (resident < 1) return false;
    const int64_t T = q.T;
    // one wave of resident CTAs (never more tiles than the flag array holds)
    int64_t K = q.k_override > 0 ? q.k_override
                                 : (T + int64_t(resident) * THREADS - 1) / (int64_t(resident) * THREADS);
    if (K < 1) K = 1;
    int64_t nt = (T + THREADS * K - 1) / (THREADS * K);
    if (nt > KF_MAX_TILES) {
        K = (T + int64_t(KF_MAX_TILES) * THREADS - 1) / (int64_t(KF_MAX_TILES) * THREADS);
        nt = (T + THREADS * K - 1) / (THREADS * K);
    }
    if (K > (int64_t(1) << 30)) return false;
    const int ntiles = int(nt < 1 ? 1 : nt);

    RsArgs<N, R> a;
    for (int i = 0; i < N * N; ++i) a.F[i] = prm.F[i];
    for (int i = 0; i < S; ++i) a.Q[i] = prm.Q[i];
    a.T = T;
    a.frec = buf.frec;
    a.ms = buf.ms;
    a.Ps = buf.Ps;
    a.K = int(K);
    a.ntiles = ntiles;
    a.lbw = (q.lookback_warps > 0 && q.lookback_warps <= THREADS / 32) ? q.lookback_warps : THREADS / 32;
    a.counters = reinterpret_cast<int *>(ws + L.ctl_r);
    a.flags = a.counters + 2;
    a.agg = reinterpret_cast<R *>(ws + L.agg);
    a.incl = reinterpret_cast<R *>(ws + L.incl);
    a.status = q.status;
    a.timeout_ns = q.timeout_ns;
    a.inject_skip_tile = q.inject_skip_tile;
    a.trace = nullptr;
    a.trace_cap = 0;
    trace_target(1, &a.trace, &a.trace_cap);
    cudaError_t e = q.counters_zeroed ? cudaSuccess
                                      : cudaMemsetAsync(a.counters, 0, sizeof(int) * (2 + ntiles), q.stream);
    if (e != cudaSuccess) {
        *err = e;
        return true;
    }
    if (debug_on())
        fprintf(stderr, "[kfscan] rts: T=%lld tiles=%d K=%lld threads=%d smem=%d\n", (long long)T, ntiles,
                (long long)K, THREADS, CF::SMEM);
    cudaEvent_t t0 = nullptr;
    if (timing_on()) timing_record(1, q.stream, &t0);
    rts_kernel<N, R, THREADS, CF::CH, CF::MINB><<<ntiles, THREADS, CF::SMEM, q.stream>>>(a);
    e = cudaGetLastError();
    count_launches(1, 1);
    if (t0) timing_commit(1, q.stream, t0);
    *err = e;
    return true;
}

// The unit's entry: 256-thread CTAs for FP32 when asked (KF_OPT_THREADS), else 128.
template <int N, typename R>
static bool rts_launch_impl(const FiltParams<N, R> &prm, const LaunchReq &q, const KfBufs<R> &buf, char *ws,
                            const WsLayout &L, cudaError_t *err) {
    if (q.threads == 256 && sizeof(R) == 4) return rts_run<N, R, 256>(prm, q, buf, ws, L, err);
    return rts_run<N, R, 128>(prm, q, buf, ws, L, err);
}

}  // namespace kfs
