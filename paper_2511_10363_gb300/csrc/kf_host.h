// kf_host.h -- declarations shared by the C-ABI layer (kf_api.cu) and the
// per-state-dimension launch units (kf_n2.cu, kf_n4.cu, kf_n8.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define KF_MAXN 8
#define KF_MAXM 8
#define KF_MAX_TILES 1024

// integer mirrors of the public enums (kfscan.h)
#define KF_OP_FILTER_I 0
#define KF_OP_RTS_I 1
#define KF_OP_TF_I 2
#define KF_SCAN_DLB_I 1
#define KF_SCAN_HS_I 2
#define KF_SCAN_BLELLOCH_I 3
#define KF_SCAN_LAFI_I 4
#define KF_SCAN_SG_I 5
#define KF_FP64_I 0
#define KF_FP32_I 1
#define KF_FP32_FP64SOLVE_I 2

namespace kfs {

// k-invariant model quantities in FP64, n x n / n x m / m x m row-major with
// the runtime sizes n, m (see FiltParams in kf_math.cuh for their meaning).
struct HostModel {
    int n, m;
    double A[KF_MAXN * KF_MAXN], C[KF_MAXN * KF_MAXN], J[KF_MAXN * KF_MAXN];
    double K[KF_MAXN * KF_MAXM], G[KF_MAXN * KF_MAXM];
    double K1[KF_MAXN * KF_MAXM], c1[KF_MAXN], C1[KF_MAXN * KF_MAXN];
    double HF[KF_MAXM * KF_MAXN], Sinv[KF_MAXM * KF_MAXM], S1inv[KF_MAXM * KF_MAXM], Hx1[KF_MAXM];
    double llc, llc1;
    double F[KF_MAXN * KF_MAXN], Q[KF_MAXN * KF_MAXN];
    double U[KF_MAXM * KF_MAXN], Linv[KF_MAXM * KF_MAXM];   // J = U^T U, U = L^{-1} H F, S = L L^T
};

struct LaunchReq {
    int op, prec, scan;
    int64_t T;
    const HostModel *hm;
    const void *y;
    void *mf_user, *Pf_user, *ms, *Ps;
    double *loglik;
    void *ws;
    cudaStream_t stream;
    int *status;
    int64_t timeout_ns;
    int inject_skip_tile;
    int k_override;      // positions per thread (0: planner's choice)
    int threads;         // CTA size of the decoupled look-back scan (0: default)
    int no_lowrank;      // 1: use the general Lemma 1 solve even when ny = nx / 2
    int lookback_warps;  // warps of a CTA that take part in the look-back (0: all)
    double *ll_step;     // per-step log-likelihood terms (batched calls; set by the batch launcher)
    int no_alloc;        // the call may not allocate: no device table cache
    int64_t sg_n;        // Sengupta threshold N (power of two)
    int counters_zeroed; // the look-back counters of this pass were cleared already
    int filter_kernel;   // 0: the time-invariant table kernel where it applies, 1: the generic scan kernel
    int rts_kernel;      // 0: the dedicated one-sequence RTS kernel where it applies, 1: the generic scan kernel
    const void *gain;    // covariance tables of a time-invariant model (GainModel), or null
    int call_graphs;     // 1: repeated covariance-table calls replay a captured CUDA graph
};

// Device cache of tile-scan tables (kf_api.cu): a table is found by its key,
// or inserted (copied from host memory on `st`); scan_table_used records that
// a launch on `st` reads slot `slot`, so that the slot is not overwritten
// before that launch has finished.  Both return null when unavailable.
const void *scan_table_lookup(uint64_t key, int *slot);
const void *scan_table_insert(uint64_t key, const void *host, size_t bytes, cudaStream_t st, int *slot);
void scan_table_used(int slot, cudaStream_t st);

// Device cache of larger tables of any size (kf_api.cu), one allocation per
// entry and a few entries per device, with the same find / insert / used
// protocol.  Both return null when unavailable.
const void *blob_lookup(uint64_t key, int *slot);
const void *blob_insert(uint64_t key, const void *host, size_t bytes, cudaStream_t st, int *slot);
void blob_used(int slot, cudaStream_t st);

// A batch of sequences concatenated in y: sequence s covers
// [offsets[s], offsets[s+1]) and uses model hms[model_of[s]].
struct BatchReq {
    int nseq, nmodels;
    const int64_t *offsets;     // host [nseq + 1]
    const int *model_of;        // host [nseq]
    const HostModel *hms;       // host [nmodels]
    int all_ny_half;            // every model has ny = nx / 2
    int params_resident;        // the tables are already in the workspace (graph capture)
};

bool debug_on();   // KFSCAN_DEBUG set in the environment

// kernel accounting (kf_timing_* in kfscan.h)
void count_launches(int kind, int n);
void count_graph(int what);   // call graphs: 0 one captured, 1 one replayed
bool timing_on();
void timing_record(int kind, cudaStream_t s, cudaEvent_t *ev);          // start event
void timing_commit(int kind, cudaStream_t s, cudaEvent_t start);        // stop event
void trace_target(int kind, uint64_t **buf, int *cap);                  // phase trace buffer of a scan kind
size_t ws_bytes_dispatch(int nx, int op, int prec, int scan, int64_t T);
cudaError_t launch_dispatch(const LaunchReq &q);
size_t batch_ws_bytes_dispatch(int nx, int op, int prec, int64_t T, int nseq, int nmodels, int loglik);
cudaError_t launch_batch_dispatch(const LaunchReq &q, const BatchReq &b);

// per-(N, precision) entry points, one translation unit each (kf_n<N>_<p>.cu)
#define KF_DECL_UNIT(N, P) \
    size_t ws_bytes_n##N##_##P(int op, int scan, int64_t T); \
    cudaError_t launch_n##N##_##P(const LaunchReq &q); \
    size_t batch_ws_bytes_n##N##_##P(int op, int64_t T, int nseq, int nmodels, int loglik); \
    cudaError_t launch_batch_n##N##_##P(const LaunchReq &q, const BatchReq &b);
KF_DECL_UNIT(2, f64) KF_DECL_UNIT(2, f32) KF_DECL_UNIT(2, mix)
KF_DECL_UNIT(4, f64) KF_DECL_UNIT(4, f32) KF_DECL_UNIT(4, mix)
KF_DECL_UNIT(8, f64) KF_DECL_UNIT(8, f32) KF_DECL_UNIT(8, mix)
#undef KF_DECL_UNIT

}  // namespace kfs
