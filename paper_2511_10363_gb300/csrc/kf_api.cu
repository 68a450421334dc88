// kf_api.cu -- the C ABI declared in include/kfscan.h: argument checks,
// the k-invariant FP64 precomputation of Eqs. pkf_init1/2/3 on the host,
// the per-device workspace cache and status word, and dispatch to the
// per-state-dimension launch units (time-invariant: kf_n<N>_<precision>.cu;
// time-varying models, kf_tv_*: kf_tv_n<N>.cu).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <new>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "../../include/kfscan.h"
#include "gain_tables.h"
#include "kf_host.h"
#include "kf_tv_host.h"

namespace kfs {

#define KF_PREC_SWITCH(N, prec, F, ...)                          \
    switch (prec) {                                              \
        case KF_FP64_I: return F##_n##N##_f64(__VA_ARGS__);      \
        case KF_FP32_I: return F##_n##N##_f32(__VA_ARGS__);      \
        default: return F##_n##N##_mix(__VA_ARGS__);             \
    }

size_t ws_bytes_dispatch(int nx, int op, int prec, int scan, int64_t T) {
    switch (nx) {
        case 2: KF_PREC_SWITCH(2, prec, ws_bytes, op, scan, T)
        case 4: KF_PREC_SWITCH(4, prec, ws_bytes, op, scan, T)
        case 8: KF_PREC_SWITCH(8, prec, ws_bytes, op, scan, T)
    }
    return 0;
}

cudaError_t launch_dispatch(const LaunchReq &q) {
    switch (q.hm->n) {
        case 2: KF_PREC_SWITCH(2, q.prec, launch, q)
        case 4: KF_PREC_SWITCH(4, q.prec, launch, q)
        case 8: KF_PREC_SWITCH(8, q.prec, launch, q)
    }
    return cudaErrorInvalidValue;
}

size_t batch_ws_bytes_dispatch(int nx, int op, int prec, int64_t T, int nseq, int nmodels, int loglik) {
    switch (nx) {
        case 2: KF_PREC_SWITCH(2, prec, batch_ws_bytes, op, T, nseq, nmodels, loglik)
        case 4: KF_PREC_SWITCH(4, prec, batch_ws_bytes, op, T, nseq, nmodels, loglik)
        case 8: KF_PREC_SWITCH(8, prec, batch_ws_bytes, op, T, nseq, nmodels, loglik)
    }
    return 0;
}

cudaError_t launch_batch_dispatch(const LaunchReq &q, const BatchReq &b) {
    switch (q.hm->n) {
        case 2: KF_PREC_SWITCH(2, q.prec, launch_batch, q, b)
        case 4: KF_PREC_SWITCH(4, q.prec, launch_batch, q, b)
        case 8: KF_PREC_SWITCH(8, q.prec, launch_batch, q, b)
    }
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- small FP64 host algebra

static void mm(int r, int k, int c, const double *A, const double *B, double *C) {
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) {
            double s = 0;
            for (int t = 0; t < k; ++t) s += A[i * k + t] * B[t * c + j];
            C[i * c + j] = s;
        }
}
static void tr(int r, int c, const double *A, double *B) {
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) B[j * r + i] = A[i * c + j];
}
// Cholesky of a symmetric matrix; false if not positive definite.
static bool chol(int n, const double *A, double *L) {
    for (int i = 0; i < n * n; ++i) L[i] = 0;
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0) || !isfinite(s)) return false;
        L[j * n + j] = sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double u = A[i * n + j];
            for (int k = 0; k < j; ++k) u -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = u / L[j * n + j];
        }
    }
    return true;
}
// inverse and log-determinant of a symmetric positive-definite matrix
static bool spd_inv(int n, const double *A, double *Ai, double *logdet) {
    double L[KF_MAXM * KF_MAXM > KF_MAXN * KF_MAXN ? KF_MAXM * KF_MAXM : KF_MAXN * KF_MAXN];
    if (!chol(n, A, L)) return false;
    double ld = 0;
    for (int i = 0; i < n; ++i) ld += 2 * log(L[i * n + i]);
    if (logdet) *logdet = ld;
    for (int c = 0; c < n; ++c) {
        double z[KF_MAXN > KF_MAXM ? KF_MAXN : KF_MAXM], x[KF_MAXN > KF_MAXM ? KF_MAXN : KF_MAXM];
        for (int i = 0; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i * n + k] * z[k];
            z[i] = s / L[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = z[i];
            for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
            x[i] = s / L[i * n + i];
        }
        for (int i = 0; i < n; ++i) Ai[i * n + c] = x[i];
    }
    return true;
}
static bool is_symmetric(int n, const double *A) {
    double mx = 0;
    for (int i = 0; i < n * n; ++i) {
        if (!isfinite(A[i])) return false;
        mx = fmax(mx, fabs(A[i]));
    }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j)
            if (fabs(A[i * n + j] - A[j * n + i]) > 1e-12 * mx) return false;
    return true;
}
// symmetric positive semi-definite: Cholesky of A + delta I with a tiny delta
static bool is_spsd(int n, const double *A) {
    if (!is_symmetric(n, A)) return false;
    double mx = 0, B[KF_MAXN * KF_MAXN], L[KF_MAXN * KF_MAXN];
    for (int i = 0; i < n * n; ++i) mx = fmax(mx, fabs(A[i]));
    const double delta = 1e-10 * (mx > 0 ? mx : 1.0);
    for (int i = 0; i < n * n; ++i) B[i] = A[i];
    for (int i = 0; i < n; ++i) B[i * n + i] += delta;
    return chol(n, B, L);
}
static void symmetrize(int n, double *A) {
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const double s = 0.5 * (A[i * n + j] + A[j * n + i]);
            A[i * n + j] = A[j * n + i] = s;
        }
}

// Eqs. pkf_init1/2/3 (and the constants of the innovation log-likelihood)
// evaluated once in FP64.
static kf_status_t precompute(const kf_model_t *md, HostModel *h) {
    const int n = md->nx, m = md->ny;
    const double *F = md->F, *Q = md->Q, *H = md->H, *R = md->R, *m0 = md->m0, *P0 = md->P0;
    memset(h, 0, sizeof(*h));
    h->n = n;
    h->m = m;
    double Ht[KF_MAXN * KF_MAXM], Ft[KF_MAXN * KF_MAXN], t1[KF_MAXN * KF_MAXN], t2[KF_MAXN * KF_MAXN];
    double S[KF_MAXM * KF_MAXM], QHt[KF_MAXN * KF_MAXM], I[KF_MAXN * KF_MAXN];
    tr(m, n, H, Ht);
    tr(n, n, F, Ft);
    for (int i = 0; i < n * n; ++i) I[i] = (i / n == i % n) ? 1.0 : 0.0;
    // S = H Q H^T + R, K = Q H^T S^{-1}
    mm(n, n, m, Q, Ht, QHt);
    mm(m, n, m, H, QHt, t1);
    for (int i = 0; i < m * m; ++i) S[i] = t1[i] + R[i];
    symmetrize(m, S);
    double logdetS;
    if (!spd_inv(m, S, h->Sinv, &logdetS)) return KF_ERR_NOT_PD;
    {   // S = L L^T, Linv = L^{-1}, U = Linv H F  (so that J = U^T U)
        double Ls[KF_MAXM * KF_MAXM], HFt[KF_MAXM * KF_MAXN];
        if (!chol(m, S, Ls)) return KF_ERR_NOT_PD;
        for (int c = 0; c < m; ++c)
            for (int i = 0; i < m; ++i) {
                double s = (i == c) ? 1.0 : 0.0;
                for (int k = c; k < i; ++k) s -= Ls[i * m + k] * h->Linv[k * m + c];
                h->Linv[i * m + c] = (i < c) ? 0.0 : s / Ls[i * m + i];
            }
        mm(m, n, n, H, F, HFt);
        mm(m, m, n, h->Linv, HFt, h->U);
    }
    mm(n, m, m, QHt, h->Sinv, h->K);
    // A = (I - K H) F, C = (I - K H) Q
    double IKH[KF_MAXN * KF_MAXN];
    mm(n, m, n, h->K, H, t1);
    for (int i = 0; i < n * n; ++i) IKH[i] = I[i] - t1[i];
    mm(n, n, n, IKH, F, h->A);
    mm(n, n, n, IKH, Q, h->C);
    symmetrize(n, h->C);
    // G = F^T H^T S^{-1}, J = G H F
    double FtHt[KF_MAXN * KF_MAXM];
    mm(n, n, m, Ft, Ht, FtHt);
    mm(n, m, m, FtHt, h->Sinv, h->G);
    mm(m, n, n, H, F, h->HF);
    mm(n, m, n, h->G, h->HF, h->J);
    symmetrize(n, h->J);
    // k = 1: xbar_{1|0} = F m0, P_{1|0} = F P0 F^T + Q, S_1, K_1, b_1 = c1 + K_1 y_1, C_1
    double x1[KF_MAXN], P1[KF_MAXN * KF_MAXN], S1[KF_MAXM * KF_MAXM], P1Ht[KF_MAXN * KF_MAXM];
    mm(n, n, 1, F, m0, x1);
    mm(n, n, n, F, P0, t1);
    mm(n, n, n, t1, Ft, t2);
    for (int i = 0; i < n * n; ++i) P1[i] = t2[i] + Q[i];
    symmetrize(n, P1);
    mm(n, n, m, P1, Ht, P1Ht);
    mm(m, n, m, H, P1Ht, t1);
    for (int i = 0; i < m * m; ++i) S1[i] = t1[i] + R[i];
    symmetrize(m, S1);
    double logdetS1;
    if (!spd_inv(m, S1, h->S1inv, &logdetS1)) return KF_ERR_NOT_PD;
    mm(n, m, m, P1Ht, h->S1inv, h->K1);
    mm(m, n, 1, H, x1, h->Hx1);
    double KHx[KF_MAXN];
    mm(n, m, 1, h->K1, h->Hx1, KHx);
    for (int i = 0; i < n; ++i) h->c1[i] = x1[i] - KHx[i];
    // C_1 = P_{1|0} - K_1 S_1 K_1^T = P_{1|0} - K_1 H P_{1|0}
    double KH[KF_MAXN * KF_MAXN];
    mm(n, m, n, h->K1, H, KH);
    mm(n, n, n, KH, P1, t1);
    for (int i = 0; i < n * n; ++i) h->C1[i] = P1[i] - t1[i];
    symmetrize(n, h->C1);
    const double LOG2PI = 1.8378770664093454835606594728112;
    h->llc = logdetS + m * LOG2PI;
    h->llc1 = logdetS1 + m * LOG2PI;
    for (int i = 0; i < n * n; ++i) {
        h->F[i] = F[i];
        h->Q[i] = Q[i];
    }
    symmetrize(n, h->Q);
    return KF_OK;
}

// ---------------------------------------------------------------- process state

static std::mutex g_mu;
static void *g_ws[64];
static size_t g_ws_bytes[64];
static int *g_status[64];
static std::atomic<int64_t> g_opt[11] = {1000000000LL, -1, 0, 0, 0, 0, 1, 0, 0, 0, 1};   // KF_OPT_* by index

// KFSCAN_DEBUG=1 in the environment logs each stage of a call to stderr.
bool debug_on() {
    static int on = -1;
    if (on < 0) {
        const char *v = getenv("KFSCAN_DEBUG");
        on = (v && v[0] && v[0] != '0') ? 1 : 0;
    }
    return on == 1;
}
#define KF_DBG(...)                                  \
    do {                                             \
        if (debug_on()) {                            \
            fprintf(stderr, "[kfscan] " __VA_ARGS__); \
            fflush(stderr);                          \
        }                                            \
    } while (0)

// ---------------------------------------------------------------- kernel accounting

static std::atomic<int64_t> g_launches[KF_KERNEL_KINDS];
static std::atomic<int> g_timing{0};
struct TimingEntry {
    int kind;
    cudaEvent_t a, b;
};
static std::mutex g_tmu;
static TimingEntry *g_tent = nullptr;
static size_t g_tn = 0, g_tcap = 0;
static double g_tms[KF_KERNEL_KINDS];
static int64_t g_tlaunch0[KF_KERNEL_KINDS];

void count_launches(int kind, int n) { g_launches[kind] += n; }

static uint64_t *g_trace[KF_KERNEL_KINDS];
static int g_trace_cap[KF_KERNEL_KINDS];
void trace_target(int kind, uint64_t **buf, int *cap) {
    std::lock_guard<std::mutex> lk(g_tmu);
    *buf = g_trace[kind];
    *cap = g_trace_cap[kind];
}
bool timing_on() { return g_timing.load() != 0; }
void timing_record(int, cudaStream_t s, cudaEvent_t *ev) {
    if (cudaEventCreate(ev) != cudaSuccess) { *ev = nullptr; return; }
    cudaEventRecord(*ev, s);
}
void timing_commit(int kind, cudaStream_t s, cudaEvent_t start) {
    cudaEvent_t stop;
    if (cudaEventCreate(&stop) != cudaSuccess) return;
    cudaEventRecord(stop, s);
    std::lock_guard<std::mutex> lk(g_tmu);
    if (g_tn == g_tcap) {
        size_t cap = g_tcap ? 2 * g_tcap : 256;
        TimingEntry *n = static_cast<TimingEntry *>(realloc(g_tent, cap * sizeof(TimingEntry)));
        if (!n) return;
        g_tent = n;
        g_tcap = cap;
    }
    g_tent[g_tn++] = TimingEntry{kind, start, stop};
}
static void timing_drain() {   // caller holds g_tmu
    for (size_t i = 0; i < g_tn; ++i) {
        float ms = 0;
        if (cudaEventSynchronize(g_tent[i].b) == cudaSuccess &&
            cudaEventElapsedTime(&ms, g_tent[i].a, g_tent[i].b) == cudaSuccess)
            g_tms[g_tent[i].kind] += ms;
        cudaEventDestroy(g_tent[i].a);
        cudaEventDestroy(g_tent[i].b);
    }
    g_tn = 0;
}

static kf_status_t from_cuda(cudaError_t e) {
    if (e != cudaSuccess) KF_DBG("CUDA error %d: %s\n", int(e), cudaGetErrorString(e));
    if (e == cudaSuccess) return KF_OK;
    if (e == cudaErrorMemoryAllocation) return KF_ERR_OOM;
    return KF_ERR_CUDA;
}

static kf_status_t device_status_word(int **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return from_cuda(e);
    if (dev < 0 || dev >= 64) return KF_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status[dev]) {
        int *p = nullptr;
        e = cudaMalloc(&p, sizeof(int));
        if (e != cudaSuccess) return from_cuda(e);
        e = cudaMemset(p, 0, sizeof(int));
        if (e != cudaSuccess) return from_cuda(e);
        g_status[dev] = p;
    }
    *out = g_status[dev];
    return KF_OK;
}

static kf_status_t library_workspace(size_t bytes, void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return from_cuda(e);
    if (dev < 0 || dev >= 64) return KF_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_ws_bytes[dev] < bytes) {
        if (g_ws[dev]) {
            cudaDeviceSynchronize();   // the old buffer may still be in use
            cudaFree(g_ws[dev]);
            g_ws[dev] = nullptr;
            g_ws_bytes[dev] = 0;
        }
        size_t want = bytes + bytes / 4;
        e = cudaMalloc(&g_ws[dev], want);
        if (e != cudaSuccess) {
            g_ws[dev] = nullptr;
            return from_cuda(e);
        }
        g_ws_bytes[dev] = want;
    }
    *out = g_ws[dev];
    return KF_OK;
}

// ---------------------------------------------------------------- tile-scan table cache

// 32 slots of 32 KB per device, allocated on first use, least recently
// used slot replaced; an event per slot marks the last launch that reads it.
namespace {
constexpr int TSC_SLOTS = 32;
constexpr size_t TSC_SLOT_BYTES = 32 << 10;
struct TscSlot {
    uint64_t key;
    uint64_t stamp;
    bool valid;
    cudaEvent_t last_use;
};
struct TscDev {
    char *base = nullptr;
    bool failed = false;
    TscSlot slot[TSC_SLOTS];
};
std::mutex g_tsc_mu;
TscDev g_tsc[64];
uint64_t g_tsc_clock = 0;

TscDev *tsc_dev(int *dev_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    TscDev &d = g_tsc[dev];
    if (d.failed) return nullptr;
    if (!d.base) {
        if (cudaMalloc(&d.base, TSC_SLOTS * TSC_SLOT_BYTES) != cudaSuccess) {
            d.base = nullptr;
            d.failed = true;
            return nullptr;
        }
        for (int i = 0; i < TSC_SLOTS; ++i) {
            d.slot[i].valid = false;
            d.slot[i].stamp = 0;
            if (cudaEventCreateWithFlags(&d.slot[i].last_use, cudaEventDisableTiming) != cudaSuccess) d.failed = true;
        }
        if (d.failed) return nullptr;
    }
    *dev_out = dev;
    return &d;
}
}  // namespace

const void *scan_table_lookup(uint64_t key, int *slot) {
    std::lock_guard<std::mutex> lk(g_tsc_mu);
    int dev = 0;
    TscDev *d = tsc_dev(&dev);
    if (!d) return nullptr;
    for (int i = 0; i < TSC_SLOTS; ++i)
        if (d->slot[i].valid && d->slot[i].key == key) {
            d->slot[i].stamp = ++g_tsc_clock;
            *slot = dev * TSC_SLOTS + i;
            return d->base + size_t(i) * TSC_SLOT_BYTES;
        }
    return nullptr;
}

const void *scan_table_insert(uint64_t key, const void *host, size_t bytes, cudaStream_t st, int *slot) {
    if (bytes > TSC_SLOT_BYTES) return nullptr;
    std::lock_guard<std::mutex> lk(g_tsc_mu);
    int dev = 0;
    TscDev *d = tsc_dev(&dev);
    if (!d) return nullptr;
    int v = 0;
    for (int i = 1; i < TSC_SLOTS; ++i)
        if (!d->slot[i].valid || (d->slot[v].valid && d->slot[i].stamp < d->slot[v].stamp)) v = i;
    if (d->slot[v].valid && cudaEventSynchronize(d->slot[v].last_use) != cudaSuccess) return nullptr;
    char *dst = d->base + size_t(v) * TSC_SLOT_BYTES;
    // pageable source: the copy has been staged when the call returns
    if (cudaMemcpyAsync(dst, host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return nullptr;
    d->slot[v].key = key;
    d->slot[v].valid = true;
    d->slot[v].stamp = ++g_tsc_clock;
    *slot = dev * TSC_SLOTS + v;
    return dst;
}

// ---- device cache of larger tables (time-invariant filter kernel)
namespace {
constexpr int BLOB_SLOTS = 8;
struct BlobSlot {
    uint64_t key, stamp;
    size_t bytes;
    char *ptr;
    cudaEvent_t last_use;
};
struct BlobDev {
    bool init = false, failed = false;
    BlobSlot slot[BLOB_SLOTS];
};
std::mutex g_blob_mu;
BlobDev g_blob[64];
uint64_t g_blob_clock = 0;

BlobDev *blob_dev(int *dev_out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    BlobDev &d = g_blob[dev];
    if (d.failed) return nullptr;
    if (!d.init) {
        for (int i = 0; i < BLOB_SLOTS; ++i) {
            d.slot[i].key = d.slot[i].stamp = 0;
            d.slot[i].bytes = 0;
            d.slot[i].ptr = nullptr;
            if (cudaEventCreateWithFlags(&d.slot[i].last_use, cudaEventDisableTiming) != cudaSuccess) {
                d.failed = true;
                return nullptr;
            }
        }
        d.init = true;
    }
    *dev_out = dev;
    return &d;
}
}  // namespace

const void *blob_lookup(uint64_t key, int *slot) {
    std::lock_guard<std::mutex> lk(g_blob_mu);
    int dev = 0;
    BlobDev *d = blob_dev(&dev);
    if (!d) return nullptr;
    for (int i = 0; i < BLOB_SLOTS; ++i)
        if (d->slot[i].ptr && d->slot[i].key == key) {
            d->slot[i].stamp = ++g_blob_clock;
            *slot = dev * BLOB_SLOTS + i;
            return d->slot[i].ptr;
        }
    return nullptr;
}

const void *blob_insert(uint64_t key, const void *host, size_t bytes, cudaStream_t st, int *slot) {
    std::lock_guard<std::mutex> lk(g_blob_mu);
    int dev = 0;
    BlobDev *d = blob_dev(&dev);
    if (!d) return nullptr;
    int v = 0;   // an empty slot, else the least recently used one
    for (int i = 1; i < BLOB_SLOTS; ++i)
        if (!d->slot[i].ptr || (d->slot[v].ptr && d->slot[i].stamp < d->slot[v].stamp)) v = i;
    BlobSlot &b = d->slot[v];
    if (b.ptr && b.bytes < bytes) {
        if (cudaEventSynchronize(b.last_use) != cudaSuccess) return nullptr;
        cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
    } else if (b.ptr && cudaEventSynchronize(b.last_use) != cudaSuccess) {
        return nullptr;
    }
    if (!b.ptr) {
        if (cudaMalloc(&b.ptr, bytes) != cudaSuccess) {
            b.ptr = nullptr;
            cudaGetLastError();
            return nullptr;
        }
        b.bytes = bytes;
    }
    // pageable source: the copy has been staged when the call returns
    if (cudaMemcpyAsync(b.ptr, host, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return nullptr;
    b.key = key;
    b.stamp = ++g_blob_clock;
    *slot = dev * BLOB_SLOTS + v;
    return b.ptr;
}

void blob_used(int slot, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_blob_mu);
    const int dev = slot / BLOB_SLOTS, i = slot % BLOB_SLOTS;
    if (dev < 0 || dev >= 64 || !g_blob[dev].init) return;
    cudaEventRecord(g_blob[dev].slot[i].last_use, st);
}

void scan_table_used(int slot, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_tsc_mu);
    const int dev = slot / TSC_SLOTS, i = slot % TSC_SLOTS;
    if (dev < 0 || dev >= 64 || !g_tsc[dev].base) return;
    cudaEventRecord(g_tsc[dev].slot[i].last_use, st);
}

static bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Rows of `len` values of w bytes move as the widest of 16-, 8- and 4-byte
// vectors that divides the row: a buffer must be aligned to that width.
static size_t row_align(int len, size_t w) {
    const size_t b = size_t(len) * w;
    return (b % 16 == 0) ? 16 : (b % 8 == 0) ? 8 : 4;
}
static bool rows_aligned(const void *p, int len, size_t w) { return !p || aligned(p, row_align(len, w)); }

static kf_status_t check_model(const kf_model_t *md) {
    if (!md) return KF_ERR_ARG;
    if (md->nx != 2 && md->nx != 4 && md->nx != 8) return KF_ERR_ARG;
    if (md->ny < 1 || md->ny > KF_MAXM) return KF_ERR_ARG;
    if (!md->F || !md->Q || !md->H || !md->R || !md->m0 || !md->P0) return KF_ERR_ARG;
    const int n = md->nx, m = md->ny;
    for (int i = 0; i < n * n; ++i)
        if (!isfinite(md->F[i])) return KF_ERR_ARG;
    for (int i = 0; i < m * n; ++i)
        if (!isfinite(md->H[i])) return KF_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (!isfinite(md->m0[i])) return KF_ERR_ARG;
    double L[KF_MAXM * KF_MAXM];
    if (!is_symmetric(m, md->R) || !chol(m, md->R, L)) return KF_ERR_NOT_PD;
    if (!is_spsd(n, md->Q) || !is_spsd(n, md->P0)) return KF_ERR_NOT_PD;
    return KF_OK;
}

// ---------------------------------------------------------------- tuning table

// Best launch configuration found by kf_autotune, keyed by operation, sizes,
// precision and floor(log2 T); applied to calls that ask for KF_SCAN_AUTO
// while the corresponding process-wide options are at their defaults.
struct TuneKey {
    int op, nx, ny, prec, logT;
    bool operator<(const TuneKey &o) const {
        if (op != o.op) return op < o.op;
        if (nx != o.nx) return nx < o.nx;
        if (ny != o.ny) return ny < o.ny;
        if (prec != o.prec) return prec < o.prec;
        return logT < o.logT;
    }
};
struct TuneCfg {
    int scan, threads, lookback_warps, k;
    double ms;
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneCfg> g_tune;

// Batched launches (kf_batch_smooth, the server's batches) keep their entries
// under op + KF_TUNE_BATCH, keyed by the batch's total number of steps.
constexpr int KF_TUNE_BATCH = 8;

static int floor_log2(int64_t T) {
    int l = 0;
    while ((int64_t(2) << l) <= T) ++l;
    return l;
}

// The launch request of this thread's last call, after the options and the
// tuning table were applied (0 = the library's own choice); see
// kf_last_launch_config.
static thread_local int t_last_cfg[4] = {0, 0, 0, 0};

static void note_launch(int scan, int threads, int lbw, int k) {
    t_last_cfg[0] = scan;
    t_last_cfg[1] = threads;
    t_last_cfg[2] = lbw;
    t_last_cfg[3] = k;
}

static bool tuned(int op, int nx, int ny, int prec, int64_t T, TuneCfg *c) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(TuneKey{op, nx, ny, prec, floor_log2(T)});
    if (it == g_tune.end()) return false;
    *c = it->second;
    return true;
}

// Covariance tables of the models seen last (gain_tables.h), built once per
// model; null for a model whose tables do not apply.
static std::shared_ptr<const GainModel> gain_model_for(const kf_model_t *md) {
    static std::mutex mu;
    static std::vector<std::pair<uint64_t, std::shared_ptr<const GainModel>>> cache;   // most recent last
    const int n = md->nx, m = md->ny;
    uint64_t key = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t bytes) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < bytes; ++i) key = (key ^ c[i]) * 1099511628211ull;
    };
    mix(&n, sizeof(n));
    mix(&m, sizeof(m));
    mix(md->F, sizeof(double) * n * n);
    mix(md->Q, sizeof(double) * n * n);
    mix(md->H, sizeof(double) * m * n);
    mix(md->R, sizeof(double) * m * m);
    mix(md->m0, sizeof(double) * n);
    mix(md->P0, sizeof(double) * n * n);
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &e : cache)
            if (e.first == key) return e.second;
    }
    std::shared_ptr<const GainModel> g;
    {
        auto b = std::make_shared<GainModel>();
        if (gain_model_build(n, m, md->F, md->Q, md->H, md->R, md->m0, md->P0, b.get()) == 0) {
            b->key = key;
            g = b;
        }
    }
    std::lock_guard<std::mutex> lk(mu);
    cache.emplace_back(key, g);
    if (cache.size() > 16) cache.erase(cache.begin());
    return g;
}

static kf_status_t run(int op, const kf_model_t *md, int64_t T, const void *y, kf_precision_t prec,
                       kf_scan_t scan, void *m1, void *P1, void *m2, void *P2, double *loglik, void *workspace,
                       void *stream) {
    kf_status_t s = check_model(md);
    if (s != KF_OK) return s;
    if (T < 1 || T > (int64_t(1) << 40) || !y) return KF_ERR_ARG;
    if (prec != KF_FP64 && prec != KF_FP32 && prec != KF_FP32_FP64SOLVE) return KF_ERR_ARG;
    if (scan < KF_SCAN_AUTO || scan > KF_SCAN_SENGUPTA) return KF_ERR_ARG;
    const size_t w = (prec == KF_FP64) ? 8 : 4;
    LaunchReq q;
    memset(&q, 0, sizeof(q));
    q.op = op;
    q.prec = int(prec);
    q.scan = (scan == KF_SCAN_AUTO) ? KF_SCAN_DLB_I : int(scan);
    q.T = T;
    q.y = y;
    if (op == KF_OP_FILTER_I) {
        if (!m1) return KF_ERR_ARG;
        q.mf_user = m1;
        q.Pf_user = P1;
    } else {
        if (!m1 || !P1) return KF_ERR_ARG;
        q.ms = m1;
        q.Ps = P1;
        q.mf_user = m2;
        q.Pf_user = P2;
    }
    const int nx = md->nx, ny = md->ny;
    if (!rows_aligned(y, ny, w) || !rows_aligned(m1, nx, w) || !rows_aligned(P1, nx * nx, w) ||
        !rows_aligned(m2, nx, w) || !rows_aligned(P2, nx * nx, w))
        return KF_ERR_ARG;
    if (loglik && !aligned(loglik, 8)) return KF_ERR_ARG;
    if (workspace && !aligned(workspace, 256)) return KF_ERR_ARG;
    HostModel hm;
    s = precompute(md, &hm);
    KF_DBG("op=%d nx=%d ny=%d T=%lld prec=%d scan=%d precompute=%d\n", op, md->nx, md->ny, (long long)T, int(prec),
           q.scan, int(s));
    if (s != KF_OK) return s;
    q.hm = &hm;
    q.loglik = loglik;
    q.stream = static_cast<cudaStream_t>(stream);
    q.timeout_ns = g_opt[KF_OPT_WAIT_TIMEOUT_NS].load();
    q.inject_skip_tile = int(g_opt[KF_OPT_TEST_SKIP_TILE].load());
    q.k_override = int(g_opt[KF_OPT_POSITIONS_PER_THREAD].load());
    q.threads = int(g_opt[KF_OPT_THREADS].load());
    q.no_lowrank = int(g_opt[KF_OPT_GENERAL_SOLVE].load());
    q.lookback_warps = int(g_opt[KF_OPT_LOOKBACK_WARPS].load());
    q.sg_n = g_opt[KF_OPT_SENGUPTA_N].load();
    q.filter_kernel = int(g_opt[KF_OPT_FILTER_KERNEL].load());
    q.rts_kernel = int(g_opt[KF_OPT_RTS_KERNEL].load());
    q.call_graphs = int(g_opt[KF_OPT_CALL_GRAPHS].load());
    // covariance tables of a time-invariant model (the per-step kernels when
    // the tables do not apply)
    std::shared_ptr<const GainModel> gm;
    if ((op == KF_OP_FILTER_I || op == KF_OP_RTS_I) && g_opt[KF_OPT_COVARIANCE_TABLES].load() == 0 &&
        q.filter_kernel == 0 && q.rts_kernel == 0 && md->ny * 2 == md->nx &&
        (md->nx == 2 || md->nx == 4 || md->nx == 8)) {
        gm = gain_model_for(md);
        q.gain = gm.get();
    }
    TuneCfg tc;   // (calls on the covariance tables plan their own tiles)
    if (scan == KF_SCAN_AUTO && !q.gain && tuned(op, md->nx, md->ny, q.prec, T, &tc)) {
        q.scan = tc.scan;
        if (q.threads == 0) q.threads = tc.threads;
        if (q.lookback_warps == 0) q.lookback_warps = tc.lookback_warps;
        if (q.k_override == 0) q.k_override = tc.k;
    }
    note_launch(q.scan, q.threads, q.lookback_warps, q.k_override);
    s = device_status_word(&q.status);
    KF_DBG("status word %p (%d)\n", (void *)q.status, int(s));
    if (s != KF_OK) return s;
    const size_t need = ws_bytes_dispatch(md->nx, op, q.prec, q.scan, T);
    if (workspace) {
        q.ws = workspace;
    } else {
        s = library_workspace(need, &q.ws);
        if (s != KF_OK) return s;
    }
    KF_DBG("workspace %p (%zu bytes needed)\n", q.ws, need);
    const cudaError_t e = launch_dispatch(q);
    KF_DBG("launched: %d\n", int(e));
    return from_cuda(e);
}

// Independent FMA chains: 8 per thread, so each warp keeps the FMA pipe busy
// without depending on neighbours; the result is stored only when it equals
// an impossible value, which keeps the chains live.
template <typename T>
__global__ void fma_peak_kernel(T a, T b, int iters, T *sink) {
    T x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = T(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == T(-1.2345e30)) *sink = s;
}

template <typename T>
static kf_status_t fma_peak(double *out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return KF_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    T *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) return KF_ERR_OOM;
    const int threads = 256, blocks = sms * 8;
    const int iters = sizeof(T) == 4 ? 1 << 16 : 1 << 11;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 0;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0);
        fma_peak_kernel<T><<<blocks, threads>>>(T(0.999999), T(1e-7), iters, sink);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        const double flops = 2.0 * 8.0 * double(iters) * blocks * threads;
        if (rep > 0 && ms > 0) best = fmax(best, flops / (ms * 1e-3));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (cudaGetLastError() != cudaSuccess || best == 0) return KF_ERR_CUDA;
    *out = best;
    return KF_OK;
}


// ---------------------------------------------------------------- batches

static kf_status_t run_batch(kf_op_t op, const kf_model_t *models, int nmodels, const int32_t *model_of, int nseq,
                             const int64_t *offsets, const void *y, kf_precision_t prec, void *m1, void *P1,
                             double *loglik, void *workspace, void *stream, int params_resident = 0) {
    if (op < KF_OP_FILTER || op > KF_OP_TWO_FILTER) return KF_ERR_ARG;
    if (!models || nmodels < 1 || nseq < 1 || !offsets || !y || !m1) return KF_ERR_ARG;
    if (op != KF_OP_FILTER && !P1) return KF_ERR_ARG;
    if (prec != KF_FP64 && prec != KF_FP32 && prec != KF_FP32_FP64SOLVE) return KF_ERR_ARG;
    if (offsets[0] != 0) return KF_ERR_ARG;
    for (int s = 0; s < nseq; ++s)
        if (offsets[s + 1] < offsets[s]) return KF_ERR_ARG;
    const int64_t total = offsets[nseq];
    if (total < 1 || total > (int64_t(1) << 40)) return KF_ERR_ARG;
    const int nx = models[0].nx, ny = models[0].ny;
    for (int i = 0; i < nmodels; ++i) {
        if (models[i].nx != nx || models[i].ny != ny) return KF_ERR_ARG;
        const kf_status_t s = check_model(&models[i]);
        if (s != KF_OK) return s;
    }
    int *mof = static_cast<int *>(malloc(sizeof(int) * size_t(nseq)));
    HostModel *hms = static_cast<HostModel *>(malloc(sizeof(HostModel) * size_t(nmodels)));
    kf_status_t s = (mof && hms) ? KF_OK : KF_ERR_OOM;
    for (int i = 0; s == KF_OK && i < nseq; ++i) {
        mof[i] = model_of ? model_of[i] : 0;
        if (mof[i] < 0 || mof[i] >= nmodels) s = KF_ERR_ARG;
    }
    for (int i = 0; s == KF_OK && i < nmodels; ++i) s = precompute(&models[i], &hms[i]);
    const size_t w = (prec == KF_FP64) ? 8 : 4;
    if (s == KF_OK &&
        (!rows_aligned(y, models[0].ny, w) || !rows_aligned(m1, models[0].nx, w) ||
         !rows_aligned(P1, models[0].nx * models[0].nx, w) || (loglik && !aligned(loglik, 8)) ||
         (workspace && !aligned(workspace, 256))))
        s = KF_ERR_ARG;
    LaunchReq q;
    memset(&q, 0, sizeof(q));
    if (s == KF_OK) {
        q.op = int(op);
        q.prec = int(prec);
        q.scan = KF_SCAN_DLB_I;
        q.T = total;
        q.hm = &hms[0];
        q.y = y;
        if (op == KF_OP_FILTER) {
            q.mf_user = m1;
            q.Pf_user = P1;
        } else {
            q.ms = m1;
            q.Ps = P1;
        }
        q.loglik = loglik;
        q.stream = static_cast<cudaStream_t>(stream);
        q.timeout_ns = g_opt[KF_OPT_WAIT_TIMEOUT_NS].load();
        q.inject_skip_tile = int(g_opt[KF_OPT_TEST_SKIP_TILE].load());
        q.k_override = int(g_opt[KF_OPT_POSITIONS_PER_THREAD].load());
        q.threads = int(g_opt[KF_OPT_THREADS].load());
        q.no_lowrank = int(g_opt[KF_OPT_GENERAL_SOLVE].load());
        q.lookback_warps = int(g_opt[KF_OPT_LOOKBACK_WARPS].load());
        // the autotuner's entry for batches of this class and size, when the
        // launch options are at their defaults
        TuneCfg tc;
        if (q.threads == 0 && q.lookback_warps == 0 && q.k_override == 0 &&
            tuned(KF_TUNE_BATCH + int(op), nx, ny, int(prec), total, &tc)) {
            q.lookback_warps = tc.lookback_warps;
            q.k_override = tc.k;
        }
        note_launch(KF_SCAN_DLB_I, 128, q.lookback_warps, q.k_override);
        s = device_status_word(&q.status);
    }
    if (s == KF_OK) {
        const size_t need = batch_ws_bytes_dispatch(nx, int(op), int(prec), total, nseq, nmodels, loglik != nullptr);
        if (workspace) q.ws = workspace;
        else s = library_workspace(need, &q.ws);
    }
    if (s == KF_OK) {
        BatchReq b;
        b.nseq = nseq;
        b.nmodels = nmodels;
        b.offsets = offsets;
        b.model_of = mof;
        b.hms = hms;
        b.all_ny_half = (ny == nx / 2);
        b.params_resident = params_resident;
        s = from_cuda(launch_batch_dispatch(q, b));
    }
    free(mof);
    free(hms);
    return s;
}

// ---------------------------------------------------------------- no-allocation entry point
//
// Scratch of kf_rts_smooth_noalloc: [0, 256) its status word, then the
// workspace of one RTS call.  Declared at file scope, so every GPU that
// loads the library holds it until exit.  In host code the name is only a
// stand-in; the kernels get its device address, looked up once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[KF_NOALLOC_SCRATCH_BYTES];
static unsigned char *g_noalloc_base[64];
static std::mutex g_noalloc_mu;

static kf_status_t noalloc_base(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return KF_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return from_cuda(e);
        if (!p) return KF_ERR_CUDA;
        g_noalloc_base[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_base[dev];
    return KF_OK;
}

static kf_status_t rts_noalloc(const kf_model_t *md, int64_t T, const void *y, kf_precision_t prec, void *ms,
                               void *Ps, double *loglik, int *status_out, void *stream) {
    kf_status_t s = check_model(md);
    if (s != KF_OK) return s;
    if (T < 1 || !y || !ms || !Ps) return KF_ERR_ARG;
    if (prec != KF_FP64 && prec != KF_FP32 && prec != KF_FP32_FP64SOLVE) return KF_ERR_ARG;
    const size_t w = (prec == KF_FP64) ? 8 : 4;
    if (!rows_aligned(y, md->ny, w) || !rows_aligned(ms, md->nx, w) || !rows_aligned(Ps, md->nx * md->nx, w))
        return KF_ERR_ARG;
    if ((loglik && !aligned(loglik, 8)) || (status_out && !aligned(status_out, 4))) return KF_ERR_ARG;
    if (timing_on()) return KF_ERR_ARG;   // kernel timing would create CUDA events
    const size_t need = 256 + ws_bytes_dispatch(md->nx, KF_OP_RTS_I, int(prec), KF_SCAN_DLB_I, T);
    if (need > KF_NOALLOC_SCRATCH_BYTES) return KF_ERR_CAPACITY;
    HostModel hm;
    s = precompute(md, &hm);
    if (s != KF_OK) return s;
    unsigned char *base = nullptr;
    s = noalloc_base(&base);
    if (s != KF_OK) return s;
    LaunchReq q;
    memset(&q, 0, sizeof(q));
    q.op = KF_OP_RTS_I;
    q.prec = int(prec);
    q.scan = KF_SCAN_DLB_I;
    q.T = T;
    q.hm = &hm;
    q.y = y;
    q.ms = ms;
    q.Ps = Ps;
    q.loglik = loglik;
    q.ws = base + 256;
    q.stream = static_cast<cudaStream_t>(stream);
    q.status = status_out ? status_out : reinterpret_cast<int *>(base);
    q.timeout_ns = g_opt[KF_OPT_WAIT_TIMEOUT_NS].load();
    q.inject_skip_tile = int(g_opt[KF_OPT_TEST_SKIP_TILE].load());
    q.k_override = int(g_opt[KF_OPT_POSITIONS_PER_THREAD].load());
    q.threads = int(g_opt[KF_OPT_THREADS].load());
    q.no_lowrank = int(g_opt[KF_OPT_GENERAL_SOLVE].load());
    q.lookback_warps = int(g_opt[KF_OPT_LOOKBACK_WARPS].load());
    q.no_alloc = 1;
    q.filter_kernel = 1;   // the table kernel keeps its tables in a device cache
    q.rts_kernel = 1;      // the kernels of this entry point stay as they were when it was added
    // A caller's status word starts at zero for this call.  Without one, the
    // scratch word is sticky like the library's own status word: it is
    // cleared only by kf_sync_status, which reads it too, so a time-out is
    // never lost (the array is zero when the module loads).
    if (status_out) {
        cudaError_t e = cudaMemsetAsync(q.status, 0, sizeof(int), q.stream);
        if (e != cudaSuccess) return from_cuda(e);
    }
    return from_cuda(launch_dispatch(q));
}

// The status word of kf_rts_smooth_noalloc calls made without status_out on
// the current device (null before the first such lookup).
static int *noalloc_status_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    return reinterpret_cast<int *>(g_noalloc_base[dev]);
}
}  // namespace kfs

using namespace kfs;

static std::atomic<int64_t> g_graph_count[2];

void kfs::count_graph(int what) {
    if (what == 0 || what == 1) g_graph_count[what].fetch_add(1);
}

extern "C" {

kf_status_t kf_call_graph_stats(int64_t *captured, int64_t *replayed) {
    if (captured) *captured = g_graph_count[0].load();
    if (replayed) *replayed = g_graph_count[1].load();
    return KF_OK;
}

int kf_bounds_checked(void) {
#ifdef KF_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

const char *kf_status_string(kf_status_t s) {
    switch (s) {
        case KF_OK: return "ok";
        case KF_ERR_ARG: return "invalid argument";
        case KF_ERR_NOT_PD: return "covariance not positive (semi-)definite";
        case KF_ERR_CUDA: return "CUDA error";
        case KF_ERR_OOM: return "out of device memory";
        case KF_ERR_TIMEOUT: return "bounded wait timed out in a kernel";
        case KF_ERR_BUDGET: return "job exceeds the device memory budget";
        case KF_ERR_BUSY: return "queue full or unknown job";
        case KF_ERR_CAPACITY: return "request exceeds a fixed scratch capacity";
        case KF_ERR_CANCELLED: return "job cancelled before it started";
        case KF_ERR_BOUNDS: return "an index check failed in a kernel (bounds-checked build)";
    }
    return "unknown status";
}

const char *kf_version(void) { return "kfscan 0.1 (sm_103a)"; }

size_t kf_workspace_size(kf_op_t op, int nx, int ny, int64_t total_steps, kf_precision_t prec, kf_scan_t scan) {
    if ((nx != 2 && nx != 4 && nx != 8) || ny < 1 || ny > KF_MAXM || total_steps < 1) return 0;
    if (op < KF_OP_FILTER || op > KF_OP_TWO_FILTER) return 0;
    if (prec != KF_FP64 && prec != KF_FP32 && prec != KF_FP32_FP64SOLVE) return 0;
    if (scan < KF_SCAN_AUTO || scan > KF_SCAN_SENGUPTA) return 0;
    if (scan == KF_SCAN_AUTO) {   // room for whichever algorithm the tuning table may pick
        const size_t a = ws_bytes_dispatch(nx, int(op), int(prec), KF_SCAN_DLB_I, total_steps);
        const size_t b = ws_bytes_dispatch(nx, int(op), int(prec), KF_SCAN_LAFI_I, total_steps);
        return a > b ? a : b;
    }
    return ws_bytes_dispatch(nx, int(op), int(prec), int(scan), total_steps);
}

kf_status_t kf_filter(const kf_model_t *model, int64_t T, const void *y, kf_precision_t prec, kf_scan_t scan,
                      void *m_out, void *P_out, double *loglik, void *workspace, void *stream) {
    return run(KF_OP_FILTER_I, model, T, y, prec, scan, m_out, P_out, nullptr, nullptr, loglik, workspace, stream);
}

kf_status_t kf_rts_smooth(const kf_model_t *model, int64_t T, const void *y, kf_precision_t prec, kf_scan_t scan,
                          void *ms_out, void *Ps_out, void *mf_out, void *Pf_out, double *loglik, void *workspace,
                          void *stream) {
    return run(KF_OP_RTS_I, model, T, y, prec, scan, ms_out, Ps_out, mf_out, Pf_out, loglik, workspace, stream);
}

kf_status_t kf_two_filter_smooth(const kf_model_t *model, int64_t T, const void *y, kf_precision_t prec,
                                 kf_scan_t scan, void *ms_out, void *Ps_out, void *mf_out, void *Pf_out,
                                 double *loglik, void *workspace, void *stream) {
    return run(KF_OP_TF_I, model, T, y, prec, scan, ms_out, Ps_out, mf_out, Pf_out, loglik, workspace, stream);
}

// ---------------------------------------------------------------- time-varying models

// One call on a time-varying model: host checks of the sizes, pointers,
// alignment and prior, then the filter pass and the smoother pass of the
// decoupled look-back scan (kf_tv.cuh).  The per-step device arrays are the
// caller's and are not read on the host.
static kf_status_t run_tv(int op, const kf_tv_model_t *md, int64_t T, const void *y, kf_precision_t prec,
                          kf_scan_t scan, void *m1, void *P1, void *m2, void *P2, double *loglik, void *workspace,
                          void *stream) {
    if (!md || (md->nx != 2 && md->nx != 4 && md->nx != 8) || md->ny < 1 || md->ny > md->nx) return KF_ERR_ARG;
    if (!md->F || !md->Q || !md->H || !md->R || !md->m0 || !md->P0) return KF_ERR_ARG;
    if (T < 1 || T > (int64_t(1) << 40) || !y) return KF_ERR_ARG;
    if (prec != KF_FP64 && prec != KF_FP32 && prec != KF_FP32_FP64SOLVE) return KF_ERR_ARG;
    if (scan != KF_SCAN_AUTO && scan != KF_SCAN_DECOUPLED_LOOKBACK) return KF_ERR_ARG;
    const int n = md->nx, m = md->ny;
    for (int i = 0; i < n; ++i)
        if (!isfinite(md->m0[i])) return KF_ERR_ARG;
    if (!is_spsd(n, md->P0)) return KF_ERR_NOT_PD;
    const size_t w = (prec == KF_FP64) ? 8 : 4;
    const void *arrs[6] = {md->F, md->Q, md->u, md->H, md->R, md->d};
    for (const void *a : arrs)
        if (a && !aligned(a, w)) return KF_ERR_ARG;
    TvLaunch t;
    memset(&t, 0, sizeof(t));
    LaunchReq &q = t.q;
    q.op = op;
    q.prec = int(prec);
    q.scan = KF_SCAN_DLB_I;
    q.T = T;
    q.y = y;
    if (op == KF_OP_FILTER_I) {
        if (!m1) return KF_ERR_ARG;
        q.mf_user = m1;
        q.Pf_user = P1;
    } else {
        if (!m1 || !P1) return KF_ERR_ARG;
        q.ms = m1;
        q.Ps = P1;
        q.mf_user = m2;
        q.Pf_user = P2;
    }
    if (!rows_aligned(y, m, w) || !rows_aligned(m1, n, w) || !rows_aligned(P1, n * n, w) ||
        !rows_aligned(m2, n, w) || !rows_aligned(P2, n * n, w))
        return KF_ERR_ARG;
    if (loglik && !aligned(loglik, 8)) return KF_ERR_ARG;
    if (workspace && !aligned(workspace, 256)) return KF_ERR_ARG;
    t.ny = m;
    t.F = md->F;
    t.Q = md->Q;
    t.u = md->u;
    t.H = md->H;
    t.R = md->R;
    t.d = md->d;
    for (int i = 0; i < n; ++i) t.m0[i] = md->m0[i];
    for (int i = 0; i < n * n; ++i) t.P0[i] = md->P0[i];
    symmetrize(n, t.P0);
    q.loglik = loglik;
    q.stream = static_cast<cudaStream_t>(stream);
    q.timeout_ns = g_opt[KF_OPT_WAIT_TIMEOUT_NS].load();
    q.inject_skip_tile = int(g_opt[KF_OPT_TEST_SKIP_TILE].load());
    q.k_override = int(g_opt[KF_OPT_POSITIONS_PER_THREAD].load());
    q.lookback_warps = int(g_opt[KF_OPT_LOOKBACK_WARPS].load());
    kf_status_t s = device_status_word(&q.status);
    if (s != KF_OK) return s;
    const size_t need = ws_bytes_dispatch(n, op, q.prec, KF_SCAN_DLB_I, T);
    if (workspace) {
        q.ws = workspace;
    } else {
        s = library_workspace(need, &q.ws);
        if (s != KF_OK) return s;
    }
    cudaError_t e;
    switch (n) {
        case 2: e = launch_tv_n2(t); break;
        case 4: e = launch_tv_n4(t); break;
        default: e = launch_tv_n8(t); break;
    }
    return from_cuda(e);
}

kf_status_t kf_tv_filter(const kf_tv_model_t *model, int64_t T, const void *y, kf_precision_t prec, kf_scan_t scan,
                         void *m_out, void *P_out, double *loglik, void *workspace, void *stream) {
    return run_tv(KF_OP_FILTER_I, model, T, y, prec, scan, m_out, P_out, nullptr, nullptr, loglik, workspace, stream);
}

kf_status_t kf_tv_rts_smooth(const kf_tv_model_t *model, int64_t T, const void *y, kf_precision_t prec,
                             kf_scan_t scan, void *ms_out, void *Ps_out, void *mf_out, void *Pf_out, double *loglik,
                             void *workspace, void *stream) {
    return run_tv(KF_OP_RTS_I, model, T, y, prec, scan, ms_out, Ps_out, mf_out, Pf_out, loglik, workspace, stream);
}

kf_status_t kf_tv_two_filter_smooth(const kf_tv_model_t *model, int64_t T, const void *y, kf_precision_t prec,
                                    kf_scan_t scan, void *ms_out, void *Ps_out, void *mf_out, void *Pf_out,
                                    double *loglik, void *workspace, void *stream) {
    return run_tv(KF_OP_TF_I, model, T, y, prec, scan, ms_out, Ps_out, mf_out, Pf_out, loglik, workspace, stream);
}

size_t kf_batch_workspace_size(kf_op_t op, int nx, int ny, int64_t total_steps, int nseq, int nmodels,
                               kf_precision_t prec, int with_loglik) {
    if ((nx != 2 && nx != 4 && nx != 8) || ny < 1 || ny > KF_MAXM || total_steps < 1 || nseq < 1 || nmodels < 1)
        return 0;
    if (op < KF_OP_FILTER || op > KF_OP_TWO_FILTER) return 0;
    if (prec != KF_FP64 && prec != KF_FP32 && prec != KF_FP32_FP64SOLVE) return 0;
    return batch_ws_bytes_dispatch(nx, int(op), int(prec), total_steps, nseq, nmodels, with_loglik ? 1 : 0);
}

kf_status_t kf_batch_smooth(kf_op_t op, const kf_model_t *models, int nmodels, const int32_t *model_of_seq, int nseq,
                            const int64_t *offsets, const void *y, kf_precision_t prec, void *m_out, void *P_out,
                            double *loglik, void *workspace, void *stream) {
    return run_batch(op, models, nmodels, model_of_seq, nseq, offsets, y, prec, m_out, P_out, loglik, workspace,
                     stream);
}

kf_status_t kf_batch_rts_smooth(const kf_model_t *models, int nmodels, const int32_t *model_of_seq, int nseq,
                                const int64_t *offsets, const void *y, kf_precision_t prec, void *ms_out,
                                void *Ps_out, double *loglik, void *workspace, void *stream) {
    return run_batch(KF_OP_RTS, models, nmodels, model_of_seq, nseq, offsets, y, prec, ms_out, Ps_out, loglik,
                     workspace, stream);
}

// ---------------------------------------------------------------- batch graphs

struct kf_batch_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    void *ws;
    int64_t kernels[KF_KERNEL_KINDS];   // kernel launches one replay makes, per kind
};

kf_status_t kf_batch_graph_create(kf_op_t op, const kf_model_t *models, int nmodels, const int32_t *model_of_seq,
                                  int nseq, const int64_t *offsets, const void *y, kf_precision_t prec, void *m_out,
                                  void *P_out, double *loglik, kf_batch_graph_t **graph) {
    if (!graph) return KF_ERR_ARG;
    *graph = nullptr;
    if (timing_on()) return KF_ERR_ARG;
    if (!models || nmodels < 1 || nseq < 1 || !offsets || offsets[0] != 0) return KF_ERR_ARG;
    for (int s = 0; s < nseq; ++s)
        if (offsets[s + 1] < offsets[s]) return KF_ERR_ARG;
    const size_t need = kf_batch_workspace_size(op, models[0].nx, models[0].ny, offsets[nseq], nseq, nmodels, prec,
                                                loglik != nullptr);
    if (need == 0) return KF_ERR_ARG;
    kf_batch_graph *g = new (std::nothrow) kf_batch_graph();
    if (!g) return KF_ERR_OOM;
    g->graph = nullptr;
    g->exec = nullptr;
    g->ws = nullptr;
    for (int k = 0; k < KF_KERNEL_KINDS; ++k) g->kernels[k] = 0;
    cudaStream_t st = nullptr;
    kf_status_t s = from_cuda(cudaMalloc(&g->ws, need));
    if (s == KF_OK) s = from_cuda(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    // a plain run stages the tables into the graph's workspace and loads the kernels
    if (s == KF_OK)
        s = run_batch(op, models, nmodels, model_of_seq, nseq, offsets, y, prec, m_out, P_out, loglik, g->ws, st, 0);
    if (s == KF_OK) s = from_cuda(cudaStreamSynchronize(st));
    if (s == KF_OK && kf_sync_status(st) != KF_OK) s = KF_ERR_TIMEOUT;
    if (s == KF_OK) {
        s = from_cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        if (s == KF_OK) {
            int64_t before[KF_KERNEL_KINDS];
            for (int k = 0; k < KF_KERNEL_KINDS; ++k) before[k] = g_launches[k].load();
            const kf_status_t sr = run_batch(op, models, nmodels, model_of_seq, nseq, offsets, y, prec, m_out, P_out,
                                             loglik, g->ws, st, 1);
            const kf_status_t se = from_cuda(cudaStreamEndCapture(st, &g->graph));
            s = (sr != KF_OK) ? sr : se;
            // the captured kernels did not run: count them at each replay instead
            for (int k = 0; k < KF_KERNEL_KINDS; ++k) {
                g->kernels[k] = g_launches[k].load() - before[k];
                count_launches(k, int(-g->kernels[k]));
            }
        }
    }
    if (s == KF_OK) s = from_cuda(cudaGraphInstantiate(&g->exec, g->graph, 0));
    if (st) cudaStreamDestroy(st);
    if (s != KF_OK) {
        kf_batch_graph_destroy(g);
        return s;
    }
    *graph = g;
    return KF_OK;
}

kf_status_t kf_batch_graph_launch(kf_batch_graph_t *graph, void *stream) {
    if (!graph || !graph->exec) return KF_ERR_ARG;
    const kf_status_t s = from_cuda(cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)));
    if (s == KF_OK)
        for (int k = 0; k < KF_KERNEL_KINDS; ++k) count_launches(k, int(graph->kernels[k]));
    return s;
}

kf_status_t kf_batch_graph_destroy(kf_batch_graph_t *graph) {
    if (!graph) return KF_OK;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    if (graph->ws) cudaFree(graph->ws);
    delete graph;
    return KF_OK;
}

kf_status_t kf_rts_smooth_noalloc(const kf_model_t *model, int64_t T, const void *y, kf_precision_t prec,
                                  void *ms_out, void *Ps_out, double *loglik, int *status_out, void *stream) {
    return rts_noalloc(model, T, y, prec, ms_out, Ps_out, loglik, status_out, stream);
}


// ---------------------------------------------------------------- autotuner

kf_status_t kf_autotune(kf_op_t op, const kf_model_t *model, int64_t T, const void *y, kf_precision_t prec,
                        void *m_out, void *P_out, int reps, void *workspace, void *stream) {
    if (!model || !y || !m_out || reps < 1 || reps > 1000) return KF_ERR_ARG;
    if (op != KF_OP_FILTER && !P_out) return KF_ERR_ARG;
    if (timing_on()) return KF_ERR_ARG;
    const int nx = model->nx;
    std::vector<TuneCfg> cands;
    // level algorithms: in-place Ladner-Fischer (the best of Algs. 1-3 on this hardware)
    cands.push_back(TuneCfg{KF_SCAN_LAFI_I, 0, 0, 0, 0});
    const int threads_opts[2] = {128, 256};
    for (int th : threads_opts) {
        if (th == 256 && !(nx == 4 && prec == KF_FP32)) continue;
        for (int lb = 1; lb <= th / 32; lb *= 2)
            for (int kscale = 0; kscale < 3; ++kscale) {
                // k = 0: one wave of resident tiles; otherwise a fixed number of steps per thread
                int k = 0;
                if (kscale > 0) {
                    int64_t per = (T + int64_t(152) * th - 1) / (int64_t(152) * th);
                    k = int(kscale == 1 ? (per + 1) / 2 : per * 2);
                    if (k < 1) k = 1;
                }
                cands.push_back(TuneCfg{KF_SCAN_DLB_I, th, lb, k, 0});
            }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return KF_ERR_CUDA;
    const int64_t saved[4] = {g_opt[KF_OPT_THREADS].load(), g_opt[KF_OPT_LOOKBACK_WARPS].load(),
                              g_opt[KF_OPT_POSITIONS_PER_THREAD].load(), 0};
    TuneCfg best{KF_SCAN_DLB_I, 0, 0, 0, 1e30};
    kf_status_t s = KF_OK;
    for (TuneCfg c : cands) {
        g_opt[KF_OPT_THREADS].store(c.threads);
        g_opt[KF_OPT_LOOKBACK_WARPS].store(c.lookback_warps);
        g_opt[KF_OPT_POSITIONS_PER_THREAD].store(c.k);
        const kf_scan_t sc = kf_scan_t(c.scan);
        auto call = [&]() -> kf_status_t {
            if (op == KF_OP_FILTER) return kf_filter(model, T, y, prec, sc, m_out, P_out, nullptr, workspace, stream);
            if (op == KF_OP_RTS)
                return kf_rts_smooth(model, T, y, prec, sc, m_out, P_out, nullptr, nullptr, nullptr, workspace, stream);
            return kf_two_filter_smooth(model, T, y, prec, sc, m_out, P_out, nullptr, nullptr, nullptr, workspace,
                                        stream);
        };
        s = call();   // warm-up (also loads the kernels)
        if (s != KF_OK) break;
        std::vector<float> ts;
        for (int r = 0; r < reps && s == KF_OK; ++r) {
            cudaEventRecord(e0, st);
            s = call();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) s = KF_ERR_CUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ts.push_back(ms);
        }
        if (s != KF_OK) break;
        std::sort(ts.begin(), ts.end());
        c.ms = ts[ts.size() / 2];
        if (c.ms < best.ms) best = c;
    }
    g_opt[KF_OPT_THREADS].store(saved[0]);
    g_opt[KF_OPT_LOOKBACK_WARPS].store(saved[1]);
    g_opt[KF_OPT_POSITIONS_PER_THREAD].store(saved[2]);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != KF_OK) return s;
    if (kf_sync_status(stream) != KF_OK) return KF_ERR_TIMEOUT;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[TuneKey{int(op), model->nx, model->ny, int(prec), floor_log2(T)}] = best;
    return KF_OK;
}

kf_status_t kf_autotune_batch(kf_op_t op, const kf_model_t *models, int nmodels, const int32_t *model_of_seq, int nseq,
                              const int64_t *offsets, const void *y, kf_precision_t prec, void *m_out, void *P_out,
                              int reps, void *workspace, void *stream) {
    if (!models || nmodels < 1 || nseq < 1 || !offsets || !y || !m_out || reps < 1 || reps > 1000)
        return KF_ERR_ARG;
    if (op != KF_OP_FILTER && !P_out) return KF_ERR_ARG;
    if (op != KF_OP_FILTER && op != KF_OP_RTS && op != KF_OP_TWO_FILTER) return KF_ERR_ARG;
    if (timing_on()) return KF_ERR_ARG;
    const int64_t total = offsets[nseq];
    if (total < 1) return KF_ERR_ARG;
    // candidates: look-back warps of the 128-thread CTA, and the steps per
    // thread (one wave of resident tiles, half and double that)
    std::vector<TuneCfg> cands;
    for (int lb = 1; lb <= 4; lb *= 2)
        for (int kscale = 0; kscale < 3; ++kscale) {
            int k = 0;
            if (kscale > 0) {
                const int64_t per = (total + int64_t(152) * 128 - 1) / (int64_t(152) * 128);
                k = int(kscale == 1 ? (per + 1) / 2 : per * 2);
                if (k < 1) k = 1;
            }
            cands.push_back(TuneCfg{KF_SCAN_DLB_I, 128, lb, k, 0});
        }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return KF_ERR_CUDA;
    const int64_t saved[3] = {g_opt[KF_OPT_THREADS].load(), g_opt[KF_OPT_LOOKBACK_WARPS].load(),
                              g_opt[KF_OPT_POSITIONS_PER_THREAD].load()};
    TuneCfg best{KF_SCAN_DLB_I, 128, 0, 0, 1e30};
    kf_status_t s = KF_OK;
    for (TuneCfg c : cands) {
        g_opt[KF_OPT_THREADS].store(0);
        g_opt[KF_OPT_LOOKBACK_WARPS].store(c.lookback_warps);
        g_opt[KF_OPT_POSITIONS_PER_THREAD].store(c.k);
        auto call = [&]() {
            return kf_batch_smooth(op, models, nmodels, model_of_seq, nseq, offsets, y, prec, m_out, P_out, nullptr,
                                   workspace, stream);
        };
        s = call();   // warm-up
        if (s != KF_OK) break;
        std::vector<float> ts;
        for (int r = 0; r < reps && s == KF_OK; ++r) {
            cudaEventRecord(e0, st);
            s = call();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) s = KF_ERR_CUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ts.push_back(ms);
        }
        if (s != KF_OK) break;
        std::sort(ts.begin(), ts.end());
        c.ms = ts[ts.size() / 2];
        if (c.ms < best.ms) best = c;
    }
    g_opt[KF_OPT_THREADS].store(saved[0]);
    g_opt[KF_OPT_LOOKBACK_WARPS].store(saved[1]);
    g_opt[KF_OPT_POSITIONS_PER_THREAD].store(saved[2]);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != KF_OK) return s;
    if (kf_sync_status(stream) != KF_OK) return KF_ERR_TIMEOUT;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[TuneKey{KF_TUNE_BATCH + int(op), models[0].nx, models[0].ny, int(prec), floor_log2(total)}] = best;
    return KF_OK;
}

kf_status_t kf_batch_tuning_get(kf_op_t op, int nx, int ny, kf_precision_t prec, int64_t total_steps,
                                int *lookback_warps, int *steps_per_thread, double *ms) {
    TuneCfg c;
    if (!tuned(KF_TUNE_BATCH + int(op), nx, ny, int(prec), total_steps, &c)) return KF_ERR_ARG;
    if (lookback_warps) *lookback_warps = c.lookback_warps;
    if (steps_per_thread) *steps_per_thread = c.k;
    if (ms) *ms = c.ms;
    return KF_OK;
}

kf_status_t kf_covariance_tables(const kf_model_t *model, int *k0, int *kb, double *P_inf, double *K_inf,
                                 double *E_inf, double *Ps_inf) {
    kf_status_t s = check_model(model);
    if (s != KF_OK) return s;
    const int n = model->nx, m = model->ny;
    if (m * 2 != n || (n != 2 && n != 4 && n != 8)) return KF_ERR_ARG;
    std::shared_ptr<const GainModel> g = gain_model_for(model);
    if (!g) return KF_ERR_ARG;
    if (k0) *k0 = g->k0;
    if (kb) *kb = g->kb;
    if (P_inf) memcpy(P_inf, g->Pi, sizeof(double) * n * n);
    if (K_inf) memcpy(K_inf, g->Ki, sizeof(double) * n * m);
    if (E_inf) memcpy(E_inf, g->Ei, sizeof(double) * n * n);
    if (Ps_inf) memcpy(Ps_inf, g->Psi, sizeof(double) * n * n);
    return KF_OK;
}

kf_status_t kf_last_launch_config(int *scan, int *threads, int *lookback_warps, int *steps_per_thread) {
    if (scan) *scan = t_last_cfg[0];
    if (threads) *threads = t_last_cfg[1];
    if (lookback_warps) *lookback_warps = t_last_cfg[2];
    if (steps_per_thread) *steps_per_thread = t_last_cfg[3];
    return KF_OK;
}

kf_status_t kf_tuning_get(kf_op_t op, int nx, int ny, kf_precision_t prec, int64_t T, int *scan, int *threads,
                          int *lookback_warps, int *steps_per_thread, double *ms) {
    TuneCfg c;
    if (!tuned(int(op), nx, ny, int(prec), T, &c)) return KF_ERR_ARG;
    if (scan) *scan = c.scan;
    if (threads) *threads = c.threads;
    if (lookback_warps) *lookback_warps = c.lookback_warps;
    if (steps_per_thread) *steps_per_thread = c.k;
    if (ms) *ms = c.ms;
    return KF_OK;
}

kf_status_t kf_tuning_save(const char *path) {
    if (!path) return KF_ERR_ARG;
    FILE *f = fopen(path, "w");
    if (!f) return KF_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    fprintf(f, "# kfscan tuning: op nx ny prec log2T scan threads lookback_warps steps_per_thread ms\n");
    for (auto &kv : g_tune)
        fprintf(f, "%d %d %d %d %d %d %d %d %d %.17g\n", kv.first.op, kv.first.nx, kv.first.ny, kv.first.prec,
                kv.first.logT, kv.second.scan, kv.second.threads, kv.second.lookback_warps, kv.second.k, kv.second.ms);
    fclose(f);
    return KF_OK;
}

kf_status_t kf_tuning_load(const char *path) {
    if (!path) return KF_ERR_ARG;
    FILE *f = fopen(path, "r");
    if (!f) return KF_ERR_ARG;
    char line[256];
    std::map<TuneKey, TuneCfg> t;
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#') continue;
        TuneKey k;
        TuneCfg c;
        if (sscanf(line, "%d %d %d %d %d %d %d %d %d %lf", &k.op, &k.nx, &k.ny, &k.prec, &k.logT, &c.scan, &c.threads,
                   &c.lookback_warps, &c.k, &c.ms) == 10) {
            if (c.scan < KF_SCAN_DLB_I || c.scan > KF_SCAN_LAFI_I || (c.threads != 0 && c.threads != 128 &&
                                                                     c.threads != 256))
                continue;
            t[k] = c;
        }
    }
    fclose(f);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto &kv : t) g_tune[kv.first] = kv.second;
    return KF_OK;
}

kf_status_t kf_tuning_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    return KF_OK;
}

kf_status_t kf_sync_status(void *stream) {
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return KF_ERR_CUDA;
    int *p = nullptr;
    kf_status_t s = device_status_word(&p);
    if (s != KF_OK) return s;
    // the library's word, then the no-allocation entry point's scratch word
    int *words[2] = {p, noalloc_status_word()};
    int first = 0;
    for (int i = 0; i < 2; ++i) {
        if (!words[i]) continue;
        int v = 0;
        e = cudaMemcpy(&v, words[i], sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return KF_ERR_CUDA;
        if (v != 0) {
            e = cudaMemset(words[i], 0, sizeof(int));
            if (e != cudaSuccess) return KF_ERR_CUDA;
            if (!first) first = v;
        }
    }
    return kf_status_t(first);
}

kf_status_t kf_stream_status(void *stream) { return kf_sync_status(stream); }

kf_status_t kf_trace_phases(kf_kernel_t kind, void *device_buffer, int capacity_tiles) {
    if (kind < 0 || kind > KF_KERNEL_TF_SCAN || capacity_tiles < 0) return KF_ERR_ARG;
    if (device_buffer && (reinterpret_cast<uintptr_t>(device_buffer) % 8)) return KF_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_tmu);
    g_trace[kind] = static_cast<uint64_t *>(device_buffer);
    g_trace_cap[kind] = device_buffer ? capacity_tiles : 0;
    return KF_OK;
}

kf_status_t kf_timing_enable(int on) {
    g_timing.store(on ? 1 : 0);
    return KF_OK;
}

kf_status_t kf_timing_reset(void) {
    std::lock_guard<std::mutex> lk(g_tmu);
    timing_drain();
    for (int k = 0; k < KF_KERNEL_KINDS; ++k) {
        g_tms[k] = 0;
        g_tlaunch0[k] = g_launches[k].load();
    }
    return KF_OK;
}

kf_status_t kf_timing_read(kf_kernel_t kind, int64_t *launches, double *total_ms) {
    if (kind < 0 || kind >= KF_KERNEL_KINDS) return KF_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_tmu);
    timing_drain();
    if (launches) *launches = g_launches[kind].load() - g_tlaunch0[kind];
    if (total_ms) *total_ms = g_tms[kind];
    return KF_OK;
}

kf_status_t kf_measure_fma_peak(int fp64, double *flops_per_second) {
    if (!flops_per_second) return KF_ERR_ARG;
    return fp64 ? fma_peak<double>(flops_per_second) : fma_peak<float>(flops_per_second);
}

kf_status_t kf_set_option(kf_option_t opt, int64_t value) {
    if (opt < KF_OPT_WAIT_TIMEOUT_NS || opt > KF_OPT_CALL_GRAPHS) return KF_ERR_ARG;
    if (opt == KF_OPT_GENERAL_SOLVE && value != 0 && value != 1) return KF_ERR_ARG;
    if ((opt == KF_OPT_FILTER_KERNEL || opt == KF_OPT_RTS_KERNEL || opt == KF_OPT_COVARIANCE_TABLES ||
         opt == KF_OPT_CALL_GRAPHS) && value != 0 &&
        value != 1)
        return KF_ERR_ARG;
    if (opt == KF_OPT_SENGUPTA_N && (value < 1 || value > (int64_t(1) << 30) || (value & (value - 1)) != 0))
        return KF_ERR_ARG;
    if (opt == KF_OPT_LOOKBACK_WARPS && (value < 0 || value > 32)) return KF_ERR_ARG;
    if (opt == KF_OPT_WAIT_TIMEOUT_NS && (value < 1000000 || value > 60000000000LL)) return KF_ERR_ARG;
    if (opt == KF_OPT_POSITIONS_PER_THREAD && (value < 0 || value > (1 << 24))) return KF_ERR_ARG;
    if (opt == KF_OPT_THREADS && value != 0 && value != 128 && value != 256) return KF_ERR_ARG;
    g_opt[opt].store(value);
    return KF_OK;
}

int64_t kf_get_option(kf_option_t opt) {
    if (opt < KF_OPT_WAIT_TIMEOUT_NS || opt > KF_OPT_CALL_GRAPHS) return -1;
    return g_opt[opt].load();
}

}  // extern "C"
