// ti_launch.cuh -- host side of the time-invariant forward filter kernel
// (ti_filter.cuh): FP64 tables, their device cache, the tile plan and the
// launch.  Included by the per-(nx, precision) units ti_n<N>_<p>.cu.
#pragma once

#include <vector>

#include "kf_launch.cuh"
#include "ti_filter.cuh"

namespace kfs {

// packed lower Cholesky factor of a full FP64 SPD matrix (n x n)
static inline bool host_chol_lo(const double *A, int n, double *Lp) {
    double L[KF_MAXN * KF_MAXN] = {};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i * n + i] = sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) Lp[lo(i, j)] = L[i * n + j];
    return true;
}

// Offsets (in values of R) of the table regions, and the whole size.
struct TiOffsets {
    int rows, sets, spans, tiles, total;
};

template <int N, typename R>
static TiOffsets ti_offsets(int K, int ntiles) {
    using TT = TiTab<N, R>;
    TiOffsets o;
    o.rows = 0;
    o.sets = TT::al((K > 1 ? K - 1 : 0) * TT::E);
    o.spans = o.sets + TT::al(TT::NSETS * TT::WE);
    o.tiles = o.spans + TT::al(TT::NSPAN * TT::PE);
    o.total = o.tiles + ntiles * TT::TES;
    return o;
}

// The tables of one launch, in FP64 rounded once to R:
//   rows    the fold table T1 | T4 | T3U for c = 1 .. K-1 (FoldTab);
//   sets    the coefficients (M1 | M2 | M3 | M4) of a left run of p and a
//           right run of s thread aggregates, warp level (s = 1 .. 16) and
//           warp-aggregate level (s = 1 .. NW/2, runs of 32 p and 32 s);
//   spans   (A, C, J) of runs of c = 0 .. 32 and 32 w thread aggregates
//           (c = 0: the neutral element);
//   tiles   for tile i: the carry covariance at its start C_{i-1} (C_{-1} =
//           P_{1|1}), its Cholesky factor, X_i = A_T (I + C_{i-1} J_T)^{-1}
//           and Y_i = X_i C_{i-1}, with (A_T, C_T, J_T) the tile's run of
//           THREADS thread aggregates; C_i = X_i C_{i-1} A_T^T + C_T.
template <int N, typename R>
static bool ti_build_tables(const HostModel &h, int K, int threads, int ntiles, std::vector<R> &out) {
    using TT = TiTab<N, R>;
    constexpr int M = N / 2, NN = N * N, S = TT::S;
    const int nw = threads / 32;
    const TiOffsets off = ti_offsets<N, R>(K, ntiles);
    out.assign(size_t(off.total), R(0));
    // rows and the K-element aggregate
    double agg[3 * NN];
    if (K >= 2) {
        FoldTab<N, M, R> *ft = new (std::nothrow) FoldTab<N, M, R>;
        if (!ft) return false;
        build_fold_table<N, M, R>(h, K, *ft, agg);
        const bool ok = ft->K == K;
        if (ok)
            for (int i = 0; i < (K - 1) * TT::E; ++i) out[size_t(off.rows + i)] = ft->t[i];
        delete ft;
        if (!ok) return false;
    } else {
        for (int i = 0; i < NN; ++i) {
            agg[i] = h.A[i];
            agg[NN + i] = h.C[i];
            agg[2 * NN + i] = h.J[i];
        }
    }
    // runs of c thread aggregates
    static thread_local double sp[TT::NSPAN][3 * NN];
    for (int i = 0; i < 3 * NN; ++i) sp[0][i] = 0.0;
    for (int i = 0; i < N; ++i) sp[0][i * N + i] = 1.0;
    for (int i = 0; i < 3 * NN; ++i) sp[1][i] = agg[i];
    for (int c = 1; c < 32; ++c)
        if (!host_acj_combine<N>(sp[TT::span(c)], sp[1], sp[TT::span(c + 1)])) return false;
    for (int w = 2; w <= nw; ++w)
        if (!host_acj_combine<N>(sp[TT::span(32 * (w - 1))], sp[TT::span(32)], sp[TT::span(32 * w)])) return false;
    for (int s = 1; s <= 16; s <<= 1)
        for (int p = 1; p <= s; ++p)
            if (!host_scan_coeffs<N, R>(sp[TT::span(p)], sp[TT::span(s)], &out[size_t(off.sets + TT::wset(s, p) * TT::WE)]))
                return false;
    for (int s = 1; s < nw; s <<= 1)
        for (int p = 1; p <= s; ++p)
            if (!host_scan_coeffs<N, R>(sp[TT::span(32 * p)], sp[TT::span(32 * s)],
                                        &out[size_t(off.sets + TT::vset(s, p) * TT::WE)]))
                return false;
    for (int c = 0; c < TT::NSPAN; ++c) {
        if (c > 32 && c - 31 > nw) continue;   // runs of 32 w for w beyond the CTA's warps are not built
        const double *x = sp[c];
        R *o = &out[size_t(off.spans + c * TT::PE)];
        for (int i = 0; i < NN; ++i) o[i] = R(x[i]);
        for (int r = 0; r < N; ++r)
            for (int q = r; q < N; ++q) {
                o[NN + su(N, r, q)] = R(x[NN + r * N + q]);
                o[NN + S + su(N, r, q)] = R(x[2 * NN + r * N + q]);
            }
    }
    // tiles
    const double *tA = sp[TT::span(32 * nw)], *tC = tA + NN, *tJ = tA + 2 * NN;
    double C[NN], X0[NN], X[NN], Y[NN], W[NN], AT[NN], Lp[S];
    for (int i = 0; i < NN; ++i) C[i] = h.C1[i];
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) AT[r * N + c] = tA[c * N + r];
    for (int t = 0; t < ntiles; ++t) {
        if (!host_chol_lo(C, N, Lp)) return false;
        if (!host_inv_I_plus(C, tJ, N, X0)) return false;
        host_mm(tA, X0, N, N, N, X);    // X = A_T (I + C J_T)^{-1}
        host_mm(X, C, N, N, N, Y);      // Y = X C
        R *o = &out[size_t(off.tiles + t * TT::TES)];
        for (int r = 0; r < N; ++r)
            for (int q = r; q < N; ++q) o[su(N, r, q)] = R(0.5 * (C[r * N + q] + C[q * N + r]));
        for (int i = 0; i < S; ++i) o[S + i] = R(Lp[i]);
        for (int i = 0; i < NN; ++i) {
            o[2 * S + i] = R(X[i]);
            o[2 * S + NN + i] = R(Y[i]);
        }
        host_mm(Y, AT, N, N, N, W);     // C <- X C A_T^T + C_T, symmetrised
        for (int r = 0; r < N; ++r)
            for (int q = 0; q < N; ++q) C[r * N + q] = 0.5 * (W[r * N + q] + W[q * N + r]) + tC[r * N + q];
    }
    return true;
}

template <int N, typename R, int THREADS>
struct TiCfg {
    // records per staged chunk (two chunks per thread in flight) and the
    // resident CTAs per SM the register allocation must allow
    static constexpr int CH = (sizeof(R) == 8 && THREADS == 256) ? 1 : 2;
    static constexpr int MINB = THREADS == 256 ? 2 : 4;
    static constexpr int KT = FoldTab<N, N / 2, R>::KT;   // fold rows at most
    // dynamic shared memory of a launch with K positions per thread: fold
    // rows (K - 1 of them), coefficient sets, staging
    static int smem(bool staged, int K) {
        using TT = TiTab<N, R>;
        return int(sizeof(R)) * (TT::al((K > 1 ? K - 1 : 0) * TT::E) + TT::al(TT::NSETS * TT::WES)) +
               TiStage<N, R, THREADS, CH>::bytes(staged);
    }
};

// Resident CTAs on the device for a launch with `smem` bytes of dynamic
// shared memory (occupancy query, cached per device and size).
template <int N, typename R, int THREADS>
static int ti_resident(int dev, int smem) {
    using CF = TiCfg<N, R, THREADS>;
    static std::mutex mu;
    static bool attr[64];
    static int key_dev[32], key_smem[32], val[32], n = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return 0;
    for (int i = 0; i < n; ++i)
        if (key_dev[i] == dev && key_smem[i] == smem) return val[i];
    auto kern = ti_filter_kernel<N, R, THREADS, CF::CH, CF::MINB>;
    if (!attr[dev]) {   // allow the largest launch once per device
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, CF::smem(true, CF::KT + 1)) !=
            cudaSuccess)
            return 0;
        attr[dev] = true;
    }
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, THREADS, smem) != cudaSuccess || per < 1) return 0;
    if (n < 32) {
        key_dev[n] = dev;
        key_smem[n] = smem;
        val[n] = sms * per;
        ++n;
    }
    return sms * per;
}

// Launches the forward filter scan on the table kernel.  Returns false, with
// nothing enqueued, when the call does not qualify (then the generic kernel
// runs it); *err carries the launch status otherwise.
template <int N, typename R, int THREADS>
static bool ti_filter_run(const FiltParams<N, R> &prm, const LaunchReq &q, const KfBufs<R> &buf, char *ws,
                          const WsLayout &L, double *ll_out, cudaError_t *err) {
    using TT = TiTab<N, R>;
    using CF = TiCfg<N, R, THREADS>;
    *err = cudaSuccess;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const bool staged = buf.frec != nullptr;
    const int64_t treg = q.T - 1;
    // one wave of resident CTAs; the fold rows in shared memory depend on K,
    // so the plan is refined once with the shared memory of the chosen K
    auto plan_k = [&](int resident) -> int64_t {
        int64_t K = (treg + int64_t(resident) * THREADS - 1) / (int64_t(resident) * THREADS);
        if (K < 1) K = 1;
        return K > CF::KT + 1 ? CF::KT + 1 : K;
    };
    int64_t K;
    if (q.k_override > 0) {
        K = q.k_override;
        if (K > CF::KT + 1) return false;
        if (ti_resident<N, R, THREADS>(dev, CF::smem(staged, int(K))) < 1) return false;
    } else {
        int resident = ti_resident<N, R, THREADS>(dev, CF::smem(staged, 1));
        if (resident < 1) return false;
        K = plan_k(resident);
        const int r2 = ti_resident<N, R, THREADS>(dev, CF::smem(staged, int(K)));
        if (r2 < 1) return false;
        if (r2 < resident) K = plan_k(r2);
    }
    int64_t nt = (treg + THREADS * K - 1) / (THREADS * K);
    if (nt < 1) nt = 1;
    if (nt > KF_MAX_TILES) return false;
    const int ntiles = int(nt);

    // tables: device cache keyed by the model constants they read and the plan
    const HostModel &h = *q.hm;
    constexpr int NNd = N * N, NM = N * (N / 2);
    const int id[4] = {int(K), THREADS, ntiles, int(sizeof(R))};
    uint64_t key = fnv1a(id, sizeof(id), 0x7469u);
    key = fnv1a(h.A, sizeof(double) * NNd, key);
    key = fnv1a(h.C, sizeof(double) * NNd, key);
    key = fnv1a(h.J, sizeof(double) * NNd, key);
    key = fnv1a(h.C1, sizeof(double) * NNd, key);
    key = fnv1a(h.K, sizeof(double) * NM, key);
    key = fnv1a(h.G, sizeof(double) * NM, key);
    key = fnv1a(h.U, sizeof(double) * NM, key);
    int slot = -1;
    const void *tab = blob_lookup(key, &slot);
    if (!tab) {
        std::vector<R> host;
        if (!ti_build_tables<N, R>(h, int(K), THREADS, ntiles, host)) return false;
        tab = blob_insert(key, host.data(), host.size() * sizeof(R), q.stream, &slot);
        if (!tab) return false;
    }
    const TiOffsets off = ti_offsets<N, R>(int(K), ntiles);

    TiArgs<N, R> a;
    a.prm = prm;
    a.T = q.T;
    a.y = buf.y;
    a.frec = buf.frec;
    a.mf = buf.mf_user;
    a.Pf = buf.Pf_user;
    a.tab = static_cast<const R *>(tab);
    a.off_rows = off.rows;
    a.off_sets = off.sets;
    a.off_spans = off.spans;
    a.off_tiles = off.tiles;
    a.K = int(K);
    a.ntiles = ntiles;
    a.lbw = (q.lookback_warps > 0 && q.lookback_warps <= THREADS / 32) ? q.lookback_warps : THREADS / 32;
    a.want_ll = ll_out != nullptr;
    a.counters = reinterpret_cast<int *>(ws + L.ctl_f);
    a.flags = a.counters + 2;
    a.ubuf = reinterpret_cast<R *>(ws + L.agg);
    a.ll_part = reinterpret_cast<double *>(ws + L.llpart);
    a.ll_out = ll_out;
    a.status = q.status;
    a.timeout_ns = q.timeout_ns;
    a.inject_skip_tile = q.inject_skip_tile;
    a.trace = nullptr;
    a.trace_cap = 0;
    trace_target(0, &a.trace, &a.trace_cap);
    cudaError_t e = q.counters_zeroed ? cudaSuccess
                                      : cudaMemsetAsync(a.counters, 0, sizeof(int) * (2 + ntiles), q.stream);
    if (e != cudaSuccess) {
        *err = e;
        return true;
    }
    const int smem = CF::smem(staged, int(K));
    if (debug_on())
        fprintf(stderr, "[kfscan] ti filter: T=%lld tiles=%d K=%lld threads=%d smem=%d\n", (long long)q.T, ntiles,
                (long long)K, THREADS, smem);
    cudaEvent_t t0 = nullptr;
    if (timing_on()) timing_record(0, q.stream, &t0);
    ti_filter_kernel<N, R, THREADS, CF::CH, CF::MINB><<<ntiles, THREADS, smem, q.stream>>>(a);
    e = cudaGetLastError();
    blob_used(slot, q.stream);
    count_launches(0, 1);
    if (t0) timing_commit(0, q.stream, t0);
    *err = e;
    return true;
}

// The unit's entry: CTA size from the request (256, else 128).
template <int N, typename R>
static bool ti_filter_launch_impl(const FiltParams<N, R> &prm, const LaunchReq &q, const KfBufs<R> &buf, char *ws,
                                  const WsLayout &L, double *ll_out, cudaError_t *err) {
    if (q.threads == 256) return ti_filter_run<N, R, 256>(prm, q, buf, ws, L, ll_out, err);
    return ti_filter_run<N, R, 128>(prm, q, buf, ws, L, ll_out, err);
}

}  // namespace kfs
