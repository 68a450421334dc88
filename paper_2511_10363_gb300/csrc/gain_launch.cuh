// gain_launch.cuh -- host side of the covariance-table path (gain_scan.cuh):
// the device tables of each scan direction, the warp-tile plan, the
// workspace regions, and the launches of the filter scan and the RTS scan of
// one sequence.
#pragma once

#include <math.h>
#include <stdio.h>

#include <mutex>
#include <vector>

#include "gain_scan.cuh"
#include "gain_tables.h"
#include "kf_launch.cuh"

namespace kfs {

// Bytes of the shared buffer of repeated settled covariance records that
// the bulk copies read (a multiple of every record size, 16 .. 512 bytes).
constexpr int GS_COVBUF = 8192;

template <int N, typename R, bool REV>
struct GsCfg {
    static constexpr int M = N / 2, MI = REV ? N : M, WPC = 4;
    // resident CTAs per SM the register budget is sized for (4 compute
    // warps; with the store warp, 5); measured on GB300 at T = 2^20
    static constexpr int MINB = (N <= 4) ? (sizeof(R) == 4 ? 5 : 3) : (sizeof(R) == 4 ? 2 : 1);
    static constexpr int MINB_SW = (N <= 4) ? (sizeof(R) == 4 ? 4 : 2) : (sizeof(R) == 4 ? 2 : 1);
    static constexpr int KS = GsStage<N, MI, R>::KS;
    static constexpr int smem_stage() { return WPC * GsStage<N, MI, R>::WARP; }
};

// Warp-tile plan of one direction.
struct GsPlan {
    int64_t npos, n0;
    int K, Kt, nbw, nwt, ncta, H;
};

// The constant block of the largest table (the 32 + 5 + 1 powers and the
// settled coefficients), for the shared-memory attribute.
template <int N, typename R>
constexpr int gs_const_bytes_max() {
    return int(sizeof(R)) * (N * N * (32 + 5 + 1 + 1 + 1) + 4 * N * N + 64) + 256;
}

template <int N, typename R, bool REV, bool STOREW>
static int gs_resident(int dev, int smem) {
    using CF = GsCfg<N, R, REV>;
    constexpr int MB = STOREW ? CF::MINB_SW : CF::MINB;
    static std::mutex mu;
    static bool attr[64];
    static int key_dev[16], key_smem[16], val[16], n = 0;
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return 0;
    for (int i = 0; i < n; ++i)
        if (key_dev[i] == dev && key_smem[i] == smem) return val[i];
    auto kern = gs_kernel<N, CF::MI, R, REV, CF::WPC, MB, STOREW>;
    if (!attr[dev]) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 CF::smem_stage() + gs_const_bytes_max<N, R>() + GS_COVBUF) != cudaSuccess)
            return 0;
        attr[dev] = true;
    }
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * CF::WPC + (STOREW ? 32 : 0), smem) !=
            cudaSuccess ||
        per < 1)
        return 0;
    if (n < 16) {
        key_dev[n] = dev;
        key_smem[n] = smem;
        val[n] = sms * per;
        ++n;
    }
    return sms * per;
}

// Positions per lane: by default one wave of resident warps, at most KS (the
// positions whose inputs stay staged) unless the warp-tile count would
// exceed `cap`; the request's override wins.
static bool gs_plan(int64_t npos, int k0, int wpc, int resident_ctas, int ks, int k_override, int64_t cap,
                    GsPlan *p) {
    const int64_t lanes = int64_t(resident_ctas) * wpc * 32;
    int64_t K = k_override > 0 ? k_override : (npos + lanes - 1) / lanes;
    if (K < 1) K = 1;
    if (k_override <= 0 && K > ks) K = ks;
    // the transient warp-tile takes the first (forward) or last (reverse)
    // min(k0, npos) positions, the settled ones fill warp-tiles of 32 K, the
    // last one possibly short
    const int64_t n0 = npos < k0 ? npos : k0, ns = npos - n0;
    for (;;) {
        const int64_t Lw = 32 * K;
        const int64_t nbw = (ns + Lw - 1) / Lw;
        if (nbw + 1 <= cap) {
            p->npos = npos;
            p->K = int(K);
            p->nbw = int(nbw);
            p->nwt = int(nbw) + 1;
            p->ncta = (p->nwt + wpc - 1) / wpc;
            p->n0 = n0;
            p->Kt = int((n0 + 31) / 32);
            if (p->Kt < 1) p->Kt = 1;
            return K < (int64_t(1) << 24);
        }
        ++K;
    }
}

static inline void gs_ident(int n, double *A) {
    for (int i = 0; i < n * n; ++i) A[i] = (i % (n + 1) == 0) ? 1.0 : 0.0;
}

// The device tables of one direction, appended to `tab` from a 16-byte
// boundary (values of type R, each region 16-byte aligned); offsets are
// relative to the direction's start, the constant block first.
template <int N, typename R, bool REV>
static GsOff gs_build(const GainModel &g, int k0, int kb, int64_t T, const GsPlan &p, std::vector<R> &tab) {
    constexpr int NN = N * N, M = N / 2, MI = REV ? N : M, Q = 16 / int(sizeof(R));
    GsOff o;
    memset(&o, 0, sizeof(o));
    while (tab.size() % Q) tab.push_back(R(0));
    const size_t base = tab.size();
    auto put = [&](const double *src, size_t n) {
        while (tab.size() % Q) tab.push_back(R(0));
        const int at = int(tab.size() - base);
        for (size_t i = 0; i < n; ++i) tab.push_back(R(src[i]));
        return at;
    };
    const double *Ai = REV ? g.Ei : g.Mi;
    // ---- the constant block
    o.A = put(Ai, NN);
    o.B = put(REV ? g.Gi : g.Ki, size_t(N) * MI);
    o.HF = put(g.HF, size_t(M) * N);
    o.W = put(g.Wi, size_t(M) * M);
    {
        double AK[64], P[64];
        std::vector<double> wl, lx;
        for (int i = 0; i < 5; ++i) {   // A^{K 2^i}
            gain_mat_pow(N, Ai, int64_t(p.K) << i, P);
            wl.insert(wl.end(), P, P + NN);
        }
        gain_mat_pow(N, Ai, p.K, AK);
        gs_ident(N, P);
        for (int l = 0; l < 32; ++l) {   // A^{K l}
            lx.insert(lx.end(), P, P + NN);
            gain_mat_mul(N, AK, P, P);
        }
        o.wl = put(wl.data(), wl.size());
        o.lx = put(lx.data(), lx.size());
        gain_mat_pow(N, Ai, int64_t(32) * p.K, P);   // A^{32 K}
        o.pt = put(P, NN);
    }
    o.cov_i = put(REV ? g.Psi : g.Pi, NN);
    while (tab.size() % Q) tab.push_back(R(0));
    o.nconst = int(tab.size() - base);
    // ---- the rest (read through the read-only path)
    o.tA = put(REV ? g.E.data() : g.M.data(), size_t(k0) * NN);
    o.tB = put(REV ? g.G.data() : g.K.data(), size_t(k0) * N * MI);
    o.tW = put(g.W.data(), size_t(k0) * M * M);
    {   // the transient warp-tile: the map of each lane's run (later steps on the left),
        // its scan's window maps, the lanes' exclusive maps, and forward those applied to m0
        const int64_t g_lo = REV ? p.npos - p.n0 + 1 : 1;
        const int64_t g_hi = REV ? p.npos : p.n0;
        std::vector<double> lanes(size_t(32) * NN);
        double X[64], P[64];
        for (int t = 0; t < 32; ++t) {
            const int64_t p1 = g_lo + int64_t(t) * p.Kt;
            const int64_t p2 = (p1 + p.Kt - 1 < g_hi) ? p1 + p.Kt - 1 : g_hi;
            gs_ident(N, X);
            int64_t j = p1;
            while (j <= p2) {
                const int64_t tk = REV ? T - j : j;   // the time of position j
                if (tk <= k0) {                       // its own A
                    gain_mat_mul(N, REV ? &g.E[size_t(tk - 1) * NN] : &g.M[size_t(tk - 1) * NN], X, X);
                    ++j;
                } else {                              // a run of settled positions
                    int64_t e = p2;
                    if (REV && T - k0 - 1 < e) e = T - k0 - 1;   // reverse: settled down to time k0 + 1
                    gain_mat_pow(N, Ai, e - j + 1, P);
                    gain_mat_mul(N, P, X, X);
                    j = e + 1;
                }
            }
            memcpy(&lanes[size_t(t) * NN], X, sizeof(double) * NN);
        }
        std::vector<double> win(size_t(5) * 32 * NN), exc(size_t(32) * NN), exc0(size_t(33) * N);
        for (int i = 0; i < 5; ++i)
            for (int l = 0; l < 32; ++l) {   // lanes max(0, l - 2^i + 1) .. l, the latest on the left
                gs_ident(N, X);
                for (int t = (l - (1 << i) + 1 > 0 ? l - (1 << i) + 1 : 0); t <= l; ++t)
                    gain_mat_mul(N, &lanes[size_t(t) * NN], X, X);
                memcpy(&win[(size_t(i) * 32 + l) * NN], X, sizeof(double) * NN);
            }
        gs_ident(N, X);
        for (int l = 0; l <= 32; ++l) {
            if (l < 32) memcpy(&exc[size_t(l) * NN], X, sizeof(double) * NN);
            for (int r = 0; r < N; ++r) {   // (map of lanes < l) m0; l = 32: the whole warp-tile's
                double acc = 0;
                for (int k = 0; k < N; ++k) acc += X[r * N + k] * g.m0[k];
                exc0[size_t(l) * N + r] = acc;
            }
            if (l < 32) gain_mat_mul(N, &lanes[size_t(l) * NN], X, X);
        }
        o.gwin = put(win.data(), win.size());
        o.gexc = put(exc.data(), exc.size());
        o.gexc0 = put(exc0.data(), exc0.size());
    }
    o.cov_t = put(REV ? g.Psf.data() : g.P.data(), size_t(k0) * NN);
    o.cov_d = REV ? put(g.Pst.data(), size_t(kb) * NN) : o.cov_i;
    while (tab.size() % Q) tab.push_back(R(0));
    return o;
}

// Look-back depth: the smallest H with max |(A^L)^H| below eps^2 of R (the
// aggregates of warp-tiles farther back then contribute below rounding), at
// most the number of warp-tiles; 33 when it would exceed 32.
template <int N, typename R>
static int gs_depth(const double *Ai, int64_t L, int ntiles) {
    const double eps = sizeof(R) == 4 ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
    double PT[64], P[64];
    gain_mat_pow(N, Ai, L, PT);
    memcpy(P, PT, sizeof(P));
    int H = 1;
    while (H < ntiles) {
        double mx = 0;
        for (int i = 0; i < N * N; ++i) mx = fmax(mx, fabs(P[i]));
        if (mx <= eps * eps) break;
        gain_mat_mul(N, PT, P, P);
        ++H;
        if (H > 32) break;
    }
    return H;
}

template <int N, typename R, bool REV>
static void gs_fill_args(GsArgs<N, R> &a, const GainModel &g, int k0, int kb, const LaunchReq &q, const GsPlan &p,
                         const R *tab, const GsOff &off, char *gw, int64_t gwt) {
    using GL = GwLayout<N, R>;
    a.T = q.T;
    a.npos = p.npos;
    a.n0 = p.n0;
    a.K = p.K;
    a.Kt = p.Kt;
    a.nbw = p.nbw;
    a.nwt = p.nwt;
    a.ncta = p.ncta;
    a.H = p.H;
    a.k0 = k0;
    a.kb = kb;
    a.cov_slice = 0;
    a.covbuf = 0;
    a.tab = tab;
    a.off = off;
    a.counters = reinterpret_cast<int *>(gw) + (REV ? 4 : 0);
    uint64_t *words = reinterpret_cast<uint64_t *>(gw + 256);
    a.words = words + (REV ? 2 * GL::NWD : 0);
    a.wstride = GL::STRIDE;
    a.ll_part = reinterpret_cast<double *>(words + size_t(GL::STRIDE) * gwt);
    a.ll_out = nullptr;
    a.ll_const = 0;
    a.want_ll = 0;
    a.status = q.status;
    a.timeout_ns = q.timeout_ns;
    a.inject_skip_tile = q.inject_skip_tile;
    a.trace = nullptr;
    a.trace_cap = 0;
    trace_target(REV ? 1 : 0, &a.trace, &a.trace_cap);
    a.pdl_wait = 0;
    a.tab_len = 0;
    a.wcap = gwt;
    for (int i = 0; i < N; ++i) a.s0[i] = R(g.m0[i]);
}

// With pdl, the kernel is launched as a programmatic dependent of the
// preceding kernel in the stream (it may start while that one drains, and
// waits for it before reading its output); a plain launch otherwise, or when
// the dependent launch is refused.
template <int N, int MI, typename R, bool REV, int WPC, int MINB, bool STOREW>
static cudaError_t gs_launch(GsArgs<N, R> &a, int smem, cudaStream_t st, bool pdl = false) {
    auto kern = gs_kernel<N, MI, R, REV, WPC, MINB, STOREW>;
    if (pdl) {
        a.pdl_wait = 1;
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cfg.gridDim = dim3(a.ncta);
        cfg.blockDim = dim3(32 * WPC + (STOREW ? 32 : 0));
        cfg.dynamicSmemBytes = size_t(smem);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, kern, a) == cudaSuccess) return cudaSuccess;
        cudaGetLastError();   // refused: a plain launch
    }
    a.pdl_wait = 0;
    kern<<<a.ncta, 32 * WPC + (STOREW ? 32 : 0), smem, st>>>(a);
    return cudaGetLastError();
}

// ---- call graphs
// A call whose launches repeat an earlier call's byte for byte (the same
// buffers, length, model tables, options and device: the key is the
// launches' argument bytes) replays a CUDA graph of its memset and both
// kernels, with the programmatic dependency between them, as one launch.
// The graph is captured on a private stream at the second such call (the
// first only records the key), and launched on the caller's stream; a
// capture that fails is not tried again for that key.  Calls on a stream
// that is itself under capture launch directly.
struct GsGraphEntry {
    std::vector<unsigned char> key;
    uint64_t h = 0, stamp = 0;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;   // after the last launch of exec (waited on before it is destroyed)
    bool failed = false;
};

template <int N, typename R>
struct GsGraphs {
    std::mutex mu;
    GsGraphEntry e[8];
    uint64_t clock = 0;
    cudaStream_t cap[64] = {};
};

template <int N, typename R>
static GsGraphs<N, R> &gs_graphs() {
    static GsGraphs<N, R> g;
    return g;
}

static inline void gs_graph_release(GsGraphEntry &x) {
    if (x.exec) {
        if (x.done) cudaEventSynchronize(x.done);
        cudaGraphExecDestroy(x.exec);
        x.exec = nullptr;
    }
}

// The graph of this key, captured now if the key was seen before; false
// when the call is to launch directly (first sighting, failed capture,
// stream under capture).
template <int N, typename R, class Enq>
static bool gs_graph_get(int dev, cudaStream_t st, const std::vector<unsigned char> &key, Enq &enqueue,
                         cudaGraphExec_t *exec, cudaEvent_t *done) {
    if (dev < 0 || dev >= 64) return false;
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cst) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (cst != cudaStreamCaptureStatusNone) return false;
    GsGraphs<N, R> &G = gs_graphs<N, R>();
    std::lock_guard<std::mutex> lk(G.mu);
    const uint64_t h = fnv1a(key.data(), key.size(), 0x9e37u);
    GsGraphEntry *x = nullptr;
    for (auto &c : G.e)
        if (c.h == h && c.key == key) x = &c;
    if (!x) {   // first sighting: remember the key (replacing the least recently used)
        x = &G.e[0];
        for (auto &c : G.e)
            if (c.stamp < x->stamp) x = &c;
        gs_graph_release(*x);
        x->key = key;
        x->h = h;
        x->failed = false;
        x->stamp = ++G.clock;
        return false;
    }
    x->stamp = ++G.clock;
    if (x->failed) return false;
    if (!x->exec) {
        bool ok = false;
        cudaStream_t cs = G.cap[dev];
        if (!cs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) == cudaSuccess) G.cap[dev] = cs;
        if (cs && (x->done || cudaEventCreateWithFlags(&x->done, cudaEventDisableTiming) == cudaSuccess) &&
            cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const cudaError_t eq = enqueue(cs, false);
            cudaGraph_t gr = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(cs, &gr);
            if (eq == cudaSuccess && ec == cudaSuccess && gr && cudaGraphInstantiate(&x->exec, gr, 0) == cudaSuccess) {
                ok = true;
                count_graph(0);
            }
            if (gr) cudaGraphDestroy(gr);
        }
        if (!ok) {
            cudaGetLastError();
            x->exec = nullptr;
            x->failed = true;
            return false;
        }
    }
    *exec = x->exec;
    *done = x->done;
    return true;
}

// A graph that did not launch: launch this key directly from now on.
template <int N, typename R>
static void gs_graph_fail(const std::vector<unsigned char> &key) {
    GsGraphs<N, R> &G = gs_graphs<N, R>();
    std::lock_guard<std::mutex> lk(G.mu);
    for (auto &c : G.e)
        if (c.key == key) {
            gs_graph_release(c);
            c.failed = true;
        }
}

static inline bool gs_al16(const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Runs the filter (and, for the RTS smoother, the RTS pass) on the
// covariance tables.  Returns false, with nothing enqueued, when the call
// does not qualify; *err carries the launch status otherwise.
template <int N, typename R>
static bool gain_run(const GainModel &g, const LaunchReq &q, const KfBufs<R> &buf, char *ws, const WsLayout &L,
                     double *ll_out, cudaError_t *err) {
    using CFF = GsCfg<N, R, false>;
    using CFR = GsCfg<N, R, true>;
    using GL = GwLayout<N, R>;
    *err = cudaSuccess;
    const bool rts = q.op == KF_OP_RTS_I;
    if (q.op != KF_OP_FILTER_I && !rts) return false;
    if (g.n != N || g.m != N / 2) return false;
    // the transients of the working precision
    const int k0 = sizeof(R) == 4 ? g.k0_32 : g.k0, kb = sizeof(R) == 4 ? g.kb_32 : g.kb;
    if (rts && q.T < int64_t(g.k0) + g.kb + 1) return false;
    R *xrec = rts ? buf.frec : buf.mf_user;   // the filter means the RTS pass reads
    if (!xrec) return false;
    if (!gs_al16(buf.y) || !gs_al16(buf.mf_user) || !gs_al16(buf.Pf_user) || !gs_al16(buf.ms) ||
        !gs_al16(buf.Ps) || !gs_al16(xrec))
        return false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const int64_t cap = L.gw_tiles;
    // the plans (sized for the largest constant block)
    const int cbytes = gs_const_bytes_max<N, R>();
    const bool pf_out = buf.Pf_user != nullptr;
    const int resf = pf_out ? gs_resident<N, R, false, true>(dev, CFF::smem_stage() + cbytes + GS_COVBUF)
                            : gs_resident<N, R, false, false>(dev, CFF::smem_stage() + cbytes);
    const int resr = rts ? gs_resident<N, R, true, true>(dev, CFR::smem_stage() + cbytes + GS_COVBUF) : 1;
    if (resf < 1 || resr < 1) return false;
    GsPlan pf, pr;
    if (!gs_plan(q.T, k0, CFF::WPC, resf, CFF::KS, q.k_override, cap, &pf)) return false;
    pf.H = gs_depth<N, R>(g.Mi, int64_t(32) * pf.K, pf.nwt);
    if (pf.H > 32) return false;
    if (rts) {
        if (!gs_plan(q.T - 1, k0, CFR::WPC, resr, CFR::KS, q.k_override, cap, &pr)) return false;
        pr.H = gs_depth<N, R>(g.Ei, int64_t(32) * pr.K, pr.nwt);
        if (pr.H > 32) return false;
    }

    // device tables: cache keyed by the model, the length and the plans
    const int id[8] = {int(q.op), int(sizeof(R)), N, pf.K, rts ? pr.K : 0, 32, k0, kb};
    uint64_t key = fnv1a(id, sizeof(id), 0x6777u);
    key = fnv1a(&q.T, sizeof(q.T), key);
    key = fnv1a(&g.key, sizeof(g.key), key);
    GsOff of, orr;
    memset(&orr, 0, sizeof(orr));
    size_t rbase = 0, tlen = 0;   // the reverse tables' start, the tables' length (values)
    int slot = -1;
    const void *tab = blob_lookup(key, &slot);
    // the offsets of a cached table (a table is built only on a miss)
    static std::mutex omu;
    static uint64_t okey[16];
    static GsOff ooff[16][2];
    static size_t obase[16], olen[16];
    static int onext = 0;
    bool have = false;
    if (tab) {
        std::lock_guard<std::mutex> lk(omu);
        for (int i = 0; i < 16 && !have; ++i)
            if (okey[i] == key) {
                of = ooff[i][0];
                orr = ooff[i][1];
                rbase = obase[i];
                tlen = olen[i];
                have = true;
            }
    }
    if (!have) {
        std::vector<R> host;
        of = gs_build<N, R, false>(g, k0, kb, q.T, pf, host);
        if (rts) {
            while (host.size() % (16 / sizeof(R))) host.push_back(R(0));
            rbase = host.size();
            orr = gs_build<N, R, true>(g, k0, kb, q.T, pr, host);
        }
        tlen = host.size();
        if (!tab) {
            tab = blob_insert(key, host.data(), host.size() * sizeof(R), q.stream, &slot);
            if (!tab) return false;
        }
        std::lock_guard<std::mutex> lk(omu);
        okey[onext] = key;
        ooff[onext][0] = of;
        ooff[onext][1] = orr;
        obase[onext] = rbase;
        olen[onext] = tlen;
        onext = (onext + 1) % 16;
    }
    if (int(sizeof(R)) * of.nconst > cbytes || (rts && int(sizeof(R)) * orr.nconst > cbytes)) return false;
    const R *dtab = static_cast<const R *>(tab);

    // counters and published words of both directions: one memset
    char *gw = ws + L.gw;
    const int ntmax = rts && pr.nwt > pf.nwt ? pr.nwt : pf.nwt;
    const size_t gw_bytes = 256 + size_t(ntmax) * GL::STRIDE * 8;

    // forward: filter means (the RTS pass's input record, and the user's copy)
    GsArgs<N, R> af;
    memset(&af, 0, sizeof(af));   // (padding too: the arguments' bytes key the call graphs)
    gs_fill_args<N, R, false>(af, g, k0, kb, q, pf, dtab, of, gw, cap);
    af.tab_len = int64_t(rts ? rbase : tlen);
    af.u = buf.y;
    af.out1 = xrec;
    af.out2 = (rts && buf.mf_user) ? buf.mf_user : nullptr;
    af.Pout = buf.Pf_user;
    af.covbuf = pf_out ? GS_COVBUF : 0;
    af.cov_slice = (q.T + pf.ncta - 1) / pf.ncta;
    af.ll_out = ll_out;
    af.want_ll = ll_out != nullptr;
    if (ll_out) {
        const int kk = q.T < k0 ? int(q.T) : k0;
        double s = 0;
        for (int k = 0; k < kk; ++k) s += g.ld[size_t(k)];
        s += double(q.T - kk) * g.ldi + double(q.T) * (N / 2) * 1.8378770664093454835606594728112;
        af.ll_const = -0.5 * s;
    }
    const int smf = CFF::smem_stage() + (int(sizeof(R)) * of.nconst + 15) / 16 * 16 + af.covbuf;
    if (debug_on())
        fprintf(stderr,
                "[kfscan] gain filter: T=%lld k0=%d kb=%d warp-tiles=%d ctas=%d K=%d Kt=%d n0=%lld H=%d smem=%d\n",
                (long long)q.T, k0, kb, pf.nwt, pf.ncta, pf.K, pf.Kt, (long long)pf.n0, pf.H, smf);

    // reverse: smoothed means and covariances
    GsArgs<N, R> ar;
    memset(&ar, 0, sizeof(ar));
    int smr = 0;
    if (rts) {
        gs_fill_args<N, R, true>(ar, g, k0, kb, q, pr, dtab + rbase, orr, gw, cap);
        ar.tab_len = int64_t(tlen - rbase);
        ar.u = xrec;
        ar.out1 = buf.ms;
        ar.out2 = nullptr;
        ar.Pout = buf.Ps;
        ar.covbuf = GS_COVBUF;
        ar.cov_slice = (q.T + pr.ncta - 1) / pr.ncta;
        smr = CFR::smem_stage() + (int(sizeof(R)) * orr.nconst + 15) / 16 * 16 + GS_COVBUF;
        if (debug_on())
            fprintf(stderr, "[kfscan] gain rts: warp-tiles=%d ctas=%d K=%d Kt=%d n0=%lld H=%d smem=%d\n", pr.nwt,
                    pr.ncta, pr.K, pr.Kt, (long long)pr.n0, pr.H, smr);
    }

    // the memset and the launches of this call on stream st; with timing,
    // library events around each kernel (the reverse launch is then not a
    // programmatic dependent: the events stand between the kernels)
    auto enqueue = [&](cudaStream_t st, bool timing) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(gw, 0, gw_bytes, st);
        if (e != cudaSuccess) return e;
        GsArgs<N, R> a1 = af;
        cudaEvent_t t0 = nullptr;
        if (timing) timing_record(0, st, &t0);
        e = pf_out ? gs_launch<N, CFF::MI, R, false, CFF::WPC, CFF::MINB_SW, true>(a1, smf, st)
                   : gs_launch<N, CFF::MI, R, false, CFF::WPC, CFF::MINB, false>(a1, smf, st);
        if (t0) timing_commit(0, st, t0);
        if (e != cudaSuccess || !rts) return e;
        GsArgs<N, R> a2 = ar;
        t0 = nullptr;
        if (timing) timing_record(1, st, &t0);
        e = gs_launch<N, CFR::MI, R, true, CFR::WPC, CFR::MINB_SW, true>(a2, smr, st, t0 == nullptr);
        if (t0) timing_commit(1, st, t0);
        return e;
    };

    // a repeated call: replay its graph
    if (q.call_graphs && !timing_on() && !af.trace && !ar.trace && q.inject_skip_tile < 0) {
        std::vector<unsigned char> key;
        auto put = [&key](const void *p, size_t n) {
            key.insert(key.end(), static_cast<const unsigned char *>(p), static_cast<const unsigned char *>(p) + n);
        };
        const int flags = (rts ? 1 : 0) | (pf_out ? 2 : 0);
        put(&dev, sizeof(dev));
        put(&flags, sizeof(flags));
        put(&gw, sizeof(gw));
        put(&gw_bytes, sizeof(gw_bytes));
        put(&smf, sizeof(smf));
        put(&smr, sizeof(smr));
        put(&af, sizeof(af));
        put(&ar, sizeof(ar));
        cudaGraphExec_t exec = nullptr;
        cudaEvent_t done = nullptr;
        if (gs_graph_get<N, R>(dev, q.stream, key, enqueue, &exec, &done)) {
            const cudaError_t e = cudaGraphLaunch(exec, q.stream);
            if (e == cudaSuccess) {
                cudaEventRecord(done, q.stream);
                count_launches(0, 1);
                if (rts) count_launches(1, 1);
                count_graph(1);
                blob_used(slot, q.stream);
                return true;
            }
            cudaGetLastError();   // not launched: launch directly
            gs_graph_fail<N, R>(key);
        }
    }

    const cudaError_t e = enqueue(q.stream, timing_on());
    count_launches(0, 1);
    if (rts && e == cudaSuccess) count_launches(1, 1);
    blob_used(slot, q.stream);
    *err = e;
    return true;
}

}  // namespace kfs
