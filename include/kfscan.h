/*
 * kfscan.h -- C ABI of the temporally parallel Kalman filter / smoother
 * library for NVIDIA GB300 (sm_103a).
 *
 * Method: Sarkka & Garcia-Fernandez, "On the Performance of Prefix-Sum
 * Parallel Kalman Filters and Smoothers on GPUs" (arXiv 2511.10363).
 * Filtering is the all-prefix-sum of the elements (A,b,C,eta,J) of
 * Sec. IV-C under the operator of Lemma 1 (Alg. pkf); RTS smoothing is the
 * reversed all-prefix-sum of the elements (E,g,L) of Sec. IV-D under
 * Lemma 2 (Alg. prts); two-filter smoothing combines the forward filter with
 * a reversed all-prefix-sum of (a_2,...,a_T,e) under Lemma 1 and the merge
 * of Eqs. mean_tf_combination / cov_tf_combination (Alg. ptf).
 *
 * Model (Sec. III-A, time-invariant, u = d = 0):
 *     x_k = F x_{k-1} + q_{k-1}, q ~ N(0,Q);  y_k = H x_k + r_k, r ~ N(0,R);
 *     x_0 ~ N(m0, P0), i.e. m0 = xbar_{0|0}, P0 = P_{0|0}.
 * The kf_tv_* entry points take the general model with per-step matrices
 * and inputs u, d instead (section "time-varying models" below).
 *
 * Conventions shared by every entry point
 *   - nx in {2, 4, 8}; 1 <= ny <= 8.  Other sizes return KF_ERR_ARG.
 *   - Model matrices (kf_model_t; kf_tv_model_t holds per-step DEVICE arrays
 *     instead) are HOST pointers to row-major FP64 arrays owned by the
 *     caller and copied during the call: F [nx][nx], Q [nx][nx] symmetric
 *     positive semi-definite, H [ny][nx], R [ny][ny] symmetric positive
 *     definite, m0 [nx], P0 [nx][nx] symmetric positive semi-definite.
 *     R not positive definite, or Q / P0 not symmetric positive
 *     semi-definite, returns KF_ERR_NOT_PD.
 *   - Data and result buffers are DEVICE pointers owned by the caller, in
 *     the working precision: double for KF_FP64, float for KF_FP32 and
 *     KF_FP32_FP64SOLVE.  y is [T][ny] (y[k-1] is y_k, k = 1..T); means are
 *     [T][nx]; covariances are full, row-major [T][nx][nx].  Outputs are for
 *     k = 1..T.  Buffers must not overlap.  Each buffer must be aligned to
 *     the largest of 16, 8 and 4 bytes that divides the byte size of one of
 *     its rows (y: ny values; means: nx; covariances: nx * nx), e.g. 16
 *     bytes for nx = 4 means in float, 8 bytes for ny = 2 in float
 *     (KF_ERR_ARG otherwise): rows move as 16-, 8- or 4-byte vectors.
 *   - loglik, when not NULL, is a DEVICE pointer to one double that receives
 *     log p(y_{1:T}), accumulated in FP64 in a fixed order.
 *   - workspace: a DEVICE buffer of at least kf_workspace_size(...) bytes,
 *     256-byte aligned, owned by the caller, used only by this call until it
 *     completes on the stream.  Passing NULL makes the library use (and grow
 *     with cudaMalloc) a per-device workspace of its own; calls that use the
 *     library's workspace must then not run concurrently on different
 *     streams.
 *   - stream: a cudaStream_t (NULL = legacy default stream).  Every call is
 *     asynchronous with respect to the host: it validates its arguments,
 *     does the k-invariant FP64 precomputation on the host, and enqueues its
 *     kernels.  Errors detected on the host are returned; errors detected by
 *     the kernels (a bounded wait that ran out) are recorded in a per-device
 *     status word read by kf_sync_status().
 *   - Nothing throws across this boundary.
 */
#ifndef KFSCAN_H
#define KFSCAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Scan algorithm.  DECOUPLED_LOOKBACK is the single-pass scan (one kernel
 * per scan direction, element construction and extraction fused in);
 * HILLIS_STEELE, BLELLOCH and LADNER_FISCHER are Algs. 1, 2 and 3 of Sec. II
 * and SENGUPTA is Alg. sengupta (reduce into half-length levels, Hillis-Steele
 * on the level of length KF_OPT_SENGUPTA_N, down-sweep), run level by level
 * over element buffers in device memory (T padded to a power of two with
 * neutral elements).  AUTO takes the autotuner's choice when it has one for
 * the call, else the decoupled look-back. */
typedef enum {
    KF_SCAN_AUTO = 0,
    KF_SCAN_DECOUPLED_LOOKBACK = 1,
    KF_SCAN_HILLIS_STEELE = 2,
    KF_SCAN_BLELLOCH = 3,
    KF_SCAN_LADNER_FISCHER = 4,
    KF_SCAN_SENGUPTA = 5
} kf_scan_t;

/* Working precision.  KF_FP32_FP64SOLVE keeps elements, combines and outputs
 * in FP32 but forms and inverts every (I + C_i J_j) of Lemma 1 (and the
 * (I + P J) of the two-filter merge) in FP64 with one step of iterative
 * refinement. */
typedef enum { KF_FP64 = 0, KF_FP32 = 1, KF_FP32_FP64SOLVE = 2 } kf_precision_t;

typedef enum {
    KF_OK = 0,
    KF_ERR_ARG = 1,      /* bad size, NULL pointer, bad enum, misalignment   */
    KF_ERR_NOT_PD = 2,   /* R not PD, or Q / P0 not symmetric PSD            */
    KF_ERR_CUDA = 3,     /* a CUDA runtime call failed                       */
    KF_ERR_OOM = 4,      /* device allocation failed                         */
    KF_ERR_TIMEOUT = 5,  /* a bounded inter-block wait in a kernel ran out   */
    KF_ERR_BUDGET = 6,   /* serving: job larger than the device budget       */
    KF_ERR_BUSY = 7,     /* serving: queue full / unknown job id             */
    KF_ERR_CAPACITY = 8, /* request larger than a fixed scratch capacity     */
    KF_ERR_CANCELLED = 9, /* server job cancelled before it started         */
    KF_ERR_BOUNDS = 10    /* bounds-checked build: an index check failed in a
                             kernel (the access was skipped)                  */
} kf_status_t;

typedef struct {
    int nx, ny;
    const double *F, *Q, *H, *R, *m0, *P0;   /* host, row-major FP64 */
} kf_model_t;

/* Human-readable name of a status code (static string). */
const char *kf_status_string(kf_status_t s);

/* Library version string (static). */
const char *kf_version(void);

/* Which operation a workspace is sized for. */
typedef enum { KF_OP_FILTER = 0, KF_OP_RTS = 1, KF_OP_TWO_FILTER = 2 } kf_op_t;

/* Bytes of device workspace needed by one call of the given operation on
 * total_steps time steps (the sum of the lengths for a batched call).
 * For KF_SCAN_AUTO it is the larger of the look-back and level-scan needs,
 * so it covers whichever algorithm a tuning-table entry selects. */
size_t kf_workspace_size(kf_op_t op, int nx, int ny, int64_t total_steps, kf_precision_t prec,
                         kf_scan_t scan);

/* Parallel Kalman filter, Alg. pkf (Sec. IV-C): filtering means m_out
 * [T][nx] = xbar_{k|k} and covariances P_out [T][nx][nx] = P_{k|k}.
 * P_out may be NULL (means only).  T >= 1. */
kf_status_t kf_filter(const kf_model_t *model, int64_t T, const void *y, kf_precision_t prec,
                      kf_scan_t scan, void *m_out, void *P_out, double *loglik, void *workspace,
                      void *stream);

/* Parallel RTS smoother, Alg. prts (Sec. IV-D), including its filter pass:
 * smoothed ms_out [T][nx] = xbar_{k|T}, Ps_out [T][nx][nx] = P_{k|T}.
 * mf_out / Pf_out, when not NULL, also receive the filtering results. */
kf_status_t kf_rts_smooth(const kf_model_t *model, int64_t T, const void *y, kf_precision_t prec,
                          kf_scan_t scan, void *ms_out, void *Ps_out, void *mf_out, void *Pf_out,
                          double *loglik, void *workspace, void *stream);

/* Parallel two-filter smoother, Alg. ptf (Secs. IV-E, IV-F), including its
 * filter pass: same outputs as kf_rts_smooth. */
kf_status_t kf_two_filter_smooth(const kf_model_t *model, int64_t T, const void *y,
                                 kf_precision_t prec, kf_scan_t scan, void *ms_out, void *Ps_out,
                                 void *mf_out, void *Pf_out, double *loglik, void *workspace,
                                 void *stream);

/* ---------------------------------------------------------------- time-varying models
 *
 * The general linear-Gaussian model of Sec. III-A (the transition and
 * measurement densities) with per-step matrices and inputs:
 *     x_k = F_{k-1} x_{k-1} + u_{k-1} + q_{k-1},   q_{k-1} ~ N(0, Q_{k-1})
 *     y_k = H_k x_k + d_k + r_k,                   r_k ~ N(0, R_k)
 * Every element is built from its own step (Eqs. pkf_init1..3 with u and d,
 * Eqs. prts_init1/2 with u) inside the scan pass.
 *
 * The per-step arrays are DEVICE buffers in the working precision (FP64 for
 * KF_FP64, FP32 otherwise), row-major, record t = 0 .. T-1 for time k = t + 1:
 *     F [T][nx][nx]  F[t] = F_{k-1}       Q [T][nx][nx]  Q[t] = Q_{k-1}
 *     u [T][nx]      u[t] = u_{k-1}, or NULL (no input)
 *     H [T][ny][nx]  H[t] = H_k           R [T][ny][ny]  R[t] = R_k
 *     d [T][ny]      d[t] = d_k, or NULL (no offset)
 * Each must be aligned to its element size.  Only the upper triangles of
 * Q[t] and R[t] are read.  m0, P0: host FP64 prior xbar_{0|0}, P_{0|0},
 * copied at the call (finite; P0 symmetric positive semi-definite, else
 * KF_ERR_NOT_PD).  nx in {2, 4, 8}, 1 <= ny <= nx.  The device arrays are
 * caller-owned, are not checked, and are read by the call's kernels on
 * `stream`: R[t] must be symmetric positive definite and Q[t] symmetric
 * positive semi-definite (and F_k P_{k|k} F_k^T + Q_k positive definite for
 * the RTS smoother); otherwise the outputs are not finite.
 * scan: KF_SCAN_AUTO or KF_SCAN_DECOUPLED_LOOKBACK (others: KF_ERR_ARG).
 * The CTA size is fixed (128 threads) and the tuning table is not
 * consulted; KF_OPT_WAIT_TIMEOUT_NS, KF_OPT_POSITIONS_PER_THREAD and
 * KF_OPT_LOOKBACK_WARPS apply.
 * Workspace: kf_workspace_size(op, nx, ny, T, prec,
 * KF_SCAN_DECOUPLED_LOOKBACK) bytes, or NULL for the library's cache.
 * y, the outputs, loglik (innovation form with v_k = y_k - H_k xbar_{k|k-1}
 * - d_k), stream and the error behaviour are those of kf_filter and
 * kf_rts_smooth. */
typedef struct {
    int nx, ny;
    const void *F, *Q, *u, *H, *R, *d;
    const double *m0, *P0;
} kf_tv_model_t;

/* Alg. pkf on a time-varying model: m_out [T][nx], P_out [T][nx][nx] (may be NULL). */
kf_status_t kf_tv_filter(const kf_tv_model_t *model, int64_t T, const void *y, kf_precision_t prec,
                         kf_scan_t scan, void *m_out, void *P_out, double *loglik, void *workspace,
                         void *stream);

/* Alg. prts on a time-varying model (RTS elements with F_k, Q_k, u_k of the
 * step k -> k+1); outputs as kf_rts_smooth. */
kf_status_t kf_tv_rts_smooth(const kf_tv_model_t *model, int64_t T, const void *y,
                             kf_precision_t prec, kf_scan_t scan, void *ms_out, void *Ps_out,
                             void *mf_out, void *Pf_out, double *loglik, void *workspace,
                             void *stream);

/* Alg. ptf on a time-varying model; outputs as kf_rts_smooth. */
kf_status_t kf_tv_two_filter_smooth(const kf_tv_model_t *model, int64_t T, const void *y,
                                    kf_precision_t prec, kf_scan_t scan, void *ms_out,
                                    void *Ps_out, void *mf_out, void *Pf_out, double *loglik,
                                    void *workspace, void *stream);

/* Batch of independent sequences (the segmented scan): sequence s is
 * y[offsets[s] .. offsets[s+1]) of the concatenated device buffer y
 * [total][ny], total = offsets[nseq], and uses model
 * models[model_of_seq[s]] (model_of_seq NULL: every sequence uses
 * models[0]).  All models share nx and ny; each carries its own F, Q, H, R
 * and prior m0, P0.  op selects Alg. pkf (m_out/P_out = filtering means and
 * covariances, P_out may be NULL), Alg. prts or Alg. ptf (smoothed means
 * and covariances).  Outputs are concatenated like y.  loglik, when not
 * NULL, is a DEVICE array [nseq] receiving log p(y_{1:T_s}) per sequence,
 * each summed in FP64 in a fixed order.  offsets and model_of_seq are HOST
 * arrays copied during the call; offsets[0] = 0, non-decreasing (empty
 * sequences allowed, total >= 1).  The scan is the decoupled look-back scan
 * over the concatenation, one kernel per pass: no segment flags are needed
 * because the operators reset at a sequence start (A_1 = 0), at a
 * sequence end (E_T = 0) and at the two-filter terminal element
 * e = (0, 0, 0, 0, 0).  Workspace as for the single-sequence calls, sized by
 * kf_batch_workspace_size. */
size_t kf_batch_workspace_size(kf_op_t op, int nx, int ny, int64_t total_steps, int nseq, int nmodels,
                               kf_precision_t prec, int with_loglik);
kf_status_t kf_batch_smooth(kf_op_t op, const kf_model_t *models, int nmodels, const int32_t *model_of_seq,
                            int nseq, const int64_t *offsets, const void *y, kf_precision_t prec, void *m_out,
                            void *P_out, double *loglik, void *workspace, void *stream);

/* kf_batch_smooth with op = KF_OP_RTS (Alg. prts on every sequence of the
 * batch): smoothed means ms_out [total][nx] and covariances Ps_out
 * [total][nx][nx]. */
kf_status_t kf_batch_rts_smooth(const kf_model_t *models, int nmodels, const int32_t *model_of_seq, int nseq,
                                const int64_t *offsets, const void *y, kf_precision_t prec, void *ms_out,
                                void *Ps_out, double *loglik, void *workspace, void *stream);

/* The batched call captured in a CUDA graph.  kf_batch_graph_create runs
 * kf_batch_smooth once with these arguments (writing the outputs) on a
 * private stream, with a workspace that the graph owns (cudaMalloc'd here),
 * then captures the same call -- the look-back counter resets and the
 * kernels of both passes and of the log-likelihood reduction, with the
 * model constants, offsets and model indices left resident in the graph's
 * workspace -- and instantiates it.  kf_batch_graph_launch replays the
 * call on `stream` on the current contents of y (same device buffers, same
 * shapes, models and offsets; new measurements may be written into y
 * between launches).  Launches of one graph must not overlap on the GPU
 * (they share its workspace): launch them on one stream.  Launch
 * configuration options (KF_OPT_*) are taken at creation; kf_timing_enable
 * must be off.  kf_batch_graph_destroy frees the graph and its workspace. */
typedef struct kf_batch_graph kf_batch_graph_t;
kf_status_t kf_batch_graph_create(kf_op_t op, const kf_model_t *models, int nmodels, const int32_t *model_of_seq,
                                  int nseq, const int64_t *offsets, const void *y, kf_precision_t prec, void *m_out,
                                  void *P_out, double *loglik, kf_batch_graph_t **graph);
kf_status_t kf_batch_graph_launch(kf_batch_graph_t *graph, void *stream);
kf_status_t kf_batch_graph_destroy(kf_batch_graph_t *graph);

/* Continuous-batching server.  A scheduler thread owns one device arena of
 * budget_bytes (allocated once, here) and max_inflight CUDA streams on the
 * device current at creation.  Submitted jobs wait in a FIFO queue; whenever
 * a stream is free, the oldest job and the following queued jobs of the
 * same class (op, nx, ny, precision) that fit in the free arena space form
 * one batch of at most max_batch_steps time steps, run as one segmented
 * scan (kf_batch_smooth).  Jobs that arrive while batches run are admitted
 * as streams and memory free up, so their work overlaps on the device.
 *   - kf_server_submit: host buffers y [T][ny], and outputs m_host
 *     [T][nx], P_host [T][nx][nx], loglik_host (1 double), each may be NULL
 *     except y, in the working precision; they must stay valid until the job
 *     is done.  Page-locked buffers let copies overlap the kernels; pageable
 *     ones are correct but serialise the scheduler.  The model is copied.
 *     A job larger than the whole budget returns KF_ERR_BUDGET.
 *   - kf_server_poll: *done = 1 once the results are in the host buffers;
 *     info, when not NULL, receives {submit time, batch start time, done
 *     time (s, steady clock), batch index}.  Returns the job's status once
 *     done, KF_ERR_BUSY for an unknown id.
 *   - kf_server_wait: blocks until the job is done (KF_ERR_TIMEOUT after
 *     timeout_s seconds).  kf_server_release forgets a done job.
 *   - kf_server_cancel: takes a job that is still queued out of the queue;
 *     it is then done with status KF_ERR_CANCELLED (poll and wait report
 *     it) and its output buffers are not touched.  A job already in a batch
 *     on the GPU, or done, returns KF_ERR_BUSY and runs to its end; an
 *     unknown id returns KF_ERR_BUSY too.
 *   - kf_server_destroy: finishes the queued and running jobs, then frees
 *     the arena and streams. */
typedef struct kf_server kf_server_t;
kf_status_t kf_server_create(size_t budget_bytes, int max_inflight, int64_t max_batch_steps, kf_server_t **out);
kf_status_t kf_server_submit(kf_server_t *srv, kf_op_t op, const kf_model_t *model, int64_t T, const void *y_host,
                             kf_precision_t prec, void *m_host, void *P_host, double *loglik_host, int64_t *job_id);
kf_status_t kf_server_poll(kf_server_t *srv, int64_t job_id, int *done, double *info);
kf_status_t kf_server_wait(kf_server_t *srv, int64_t job_id, double timeout_s);
kf_status_t kf_server_release(kf_server_t *srv, int64_t job_id);
kf_status_t kf_server_cancel(kf_server_t *srv, int64_t job_id);
kf_status_t kf_server_destroy(kf_server_t *srv);

/* RTS smoother that allocates no device memory.
 *
 * The paper has no counterpart: this is a deployment variant of
 * kf_rts_smooth for callers that may not allocate device memory at call
 * time -- for example code whose device memory is all owned and accounted
 * for by another allocator (a framework's memory pool or a fixed budget),
 * or a latency-critical loop that cannot afford cudaMalloc's implicit
 * device-wide synchronisation or the risk of an out-of-memory failure in
 * the middle of its work.
 *
 * It computes exactly what kf_rts_smooth computes with the decoupled
 * look-back scan, but its scratch (look-back descriptors, the filter records
 * handed from the forward to the backward pass, and its status word) lives
 * in one statically sized device array of KF_NOALLOC_SCRATCH_BYTES that the
 * library declares at file scope; every GPU that loads the library holds
 * that array until the process exits.  The call makes no cudaMalloc or
 * cudaFree and no other allocating call, not even on its first use.
 *   - The caller still passes y, ms_out [T][nx] and Ps_out [T][nx][nx]
 *     (device, working precision), and may pass loglik (device double) and
 *     status_out (device int, may be NULL).  status_out is set to 0 at the
 *     start of the call and receives KF_ERR_TIMEOUT if a bounded wait in a
 *     kernel runs out.  Without status_out the time-out goes to a status
 *     word inside the array, which stays set until kf_sync_status (which
 *     reads it beside the library's own word) reports and clears it; while
 *     it is set, later calls without status_out give up their waits at once.
 *   - Its first call on a device looks up the device address of the array
 *     (cudaGetSymbolAddress); make that first call before capturing the
 *     stream into a graph.  The array is reserved when the library's device
 *     code is loaded on that device -- under lazy module loading, at that
 *     first call -- and a failure to reserve it there is returned as
 *     KF_ERR_CUDA or KF_ERR_OOM.
 *   - Requests whose scratch would exceed the array (kf_workspace_size of an
 *     RTS call plus 256 bytes, i.e. T <= 258,164 steps at nx = 4 in FP32)
 *     return KF_ERR_CAPACITY and enqueue nothing; kf_timing_enable must be
 *     off (KF_ERR_ARG otherwise).
 *   - All calls share the one array, which keeps the last call's contents;
 *     the call clears what must start at zero.  Calls whose work overlaps on
 *     the GPU (different streams, or different host threads) race on the
 *     array and must be serialised by the caller. */
#define KF_NOALLOC_SCRATCH_BYTES (16u << 20)
kf_status_t kf_rts_smooth_noalloc(const kf_model_t *model, int64_t T, const void *y, kf_precision_t prec,
                                  void *ms_out, void *Ps_out, double *loglik, int *status_out, void *stream);

/* Waits for `stream`, then returns and clears the device status word of the
 * current device: KF_OK, or KF_ERR_TIMEOUT if some kernel's bounded wait ran
 * out since the last call (its outputs are then undefined), or KF_ERR_CUDA
 * if the stream reported an error. */
kf_status_t kf_sync_status(void *stream);

/* The same as kf_sync_status(stream): the status of the kernels enqueued so
 * far, read after `stream` has finished. */
kf_status_t kf_stream_status(void *stream);

/* Process-wide options read at the start of every later call.
 *   KF_OPT_WAIT_TIMEOUT_NS      bound of every inter-CTA wait in the
 *                               decoupled look-back scan (default 1e9 ns;
 *                               1e6 .. 6e10 accepted).
 *   KF_OPT_TEST_SKIP_TILE       test hook: the CTA that takes this tile
 *                               ticket returns without publishing, so the
 *                               later tiles' waits run out and the call
 *                               reports KF_ERR_TIMEOUT (default -1: off).
 *   KF_OPT_POSITIONS_PER_THREAD time steps folded serially by one thread in
 *                               the decoupled look-back scan (0 = planner's
 *                               choice: one wave of resident CTAs).
 *   KF_OPT_THREADS              CTA size of that scan: 0 (default, 128) or 128;
 *                               256 is also built for nx = 4 in FP32.
 *   KF_OPT_GENERAL_SOLVE        1: always invert (I + C_i J_j) of Lemma 1 by
 *                               pivoted Gauss-Jordan; 0 (default): when
 *                               ny = nx / 2, the filter scan's thread fold and
 *                               carry pass use the rank-ny form of a fresh
 *                               element's J (Woodbury identity).
 *   KF_OPT_LOOKBACK_WARPS       warps of a CTA that reduce the predecessor
 *                               aggregates in the look-back: 0 (default: the
 *                               library's choice) or 1 .. 32 (capped at the
 *                               CTA's warp count).
 *   KF_OPT_SENGUPTA_N           threshold N of KF_SCAN_SENGUPTA: the length
 *                               of the level scanned by Hillis-Steele, a power
 *                               of two in 1 .. 2^30 (default 1, the paper's
 *                               "Sengupta A"; larger N, "Sengupta B", is
 *                               capped at the padded length).
 *   KF_OPT_FILTER_KERNEL        0 (default): the forward filter scan of a
 *                               time-invariant model with ny = nx / 2
 *                               (nx 2 or 4, FP32 or FP64, one sequence, the
 *                               decoupled look-back scan) runs the table
 *                               kernel, whose data-independent coefficients
 *                               (fold rows, run coefficients, the carry
 *                               covariance at each tile's start) the host
 *                               computes in FP64 and keeps in a device cache;
 *                               1: the generic look-back kernel.
 *   KF_OPT_RTS_KERNEL           0 (default): the RTS smoother pass of one
 *                               sequence (nx 2 or 4, the decoupled look-back
 *                               scan) runs its dedicated kernel; 1: the
 *                               generic look-back kernel.
 *   KF_OPT_COVARIANCE_TABLES    0 (default): kf_filter and kf_rts_smooth on
 *                               a time-invariant model with ny = nx / 2
 *                               (nx 2, 4 or 8, any precision, the decoupled
 *                               look-back scan, KF_OPT_FILTER_KERNEL and
 *                               KF_OPT_RTS_KERNEL at 0) take the
 *                               data-independent halves of the elements --
 *                               filtering covariances, gains, smoothed
 *                               covariances -- from FP64 tables the host
 *                               computes once per model (the covariance
 *                               recursion to its fixed point, relative change
 *                               below 2^-46), and scan only the means on the
 *                               device; the smoother needs T >= k0 + kb + 1
 *                               (the lengths of the two transients, a few
 *                               hundred steps for a well-damped model).
 *                               1: the per-step kernels above.
 *   KF_OPT_CALL_GRAPHS          1 (default): a covariance-table call whose
 *                               launches repeat an earlier call's exactly
 *                               (same buffers, length, model, options and
 *                               device) is replayed from a CUDA graph of its
 *                               memset and both kernels, captured on a
 *                               private stream at the second such call (8
 *                               graphs per state size and precision, least
 *                               recently used replaced); calls on a stream
 *                               under capture, with kernel timing or phase
 *                               tracing launch directly.  0: always direct.
 * Returns KF_ERR_ARG for an unknown option or a value out of range. */
typedef enum {
    KF_OPT_WAIT_TIMEOUT_NS = 0,
    KF_OPT_TEST_SKIP_TILE = 1,
    KF_OPT_POSITIONS_PER_THREAD = 2,
    KF_OPT_THREADS = 3,
    KF_OPT_GENERAL_SOLVE = 4,
    KF_OPT_LOOKBACK_WARPS = 5,
    KF_OPT_SENGUPTA_N = 6,
    KF_OPT_FILTER_KERNEL = 7,
    KF_OPT_RTS_KERNEL = 8,
    KF_OPT_COVARIANCE_TABLES = 9,
    KF_OPT_CALL_GRAPHS = 10
} kf_option_t;
kf_status_t kf_set_option(kf_option_t opt, int64_t value);
int64_t kf_get_option(kf_option_t opt); /* -1 for an unknown option */

/* Flops per time step of the one-sequence kernels, counted from their own
 * step code (the step functions run on the host with a counting number
 * type): step 0 = one step of the table-driven thread fold of the filter
 * scan, 1 = one step of its carry pass, 2 = the same with the log-likelihood
 * term, 3 = one step of the RTS pass's thread fold, 4 = one step of its carry
 * pass.  nx = 2 or 4 (ny = nx / 2).  counts[6] receives the total (an
 * add, subtract or multiply counts 1, so a multiply-add 2; a reciprocal,
 * square root or log 1), then adds, multiplies, reciprocals, square roots,
 * logs.  Host only.  KF_ERR_ARG for another nx or step. */
kf_status_t kf_count_step_flops(int nx, int step, int64_t *counts);

/* Kernel accounting (diagnostics for benchmarks).  The library counts every
 * kernel it launches, by kind.  While timing is enabled it also brackets each
 * scan (one kernel for the decoupled look-back scan; the whole level-by-level
 * launch sequence otherwise) with two CUDA events on the call's stream.
 * kf_timing_read waits for the recorded events of that kind and returns the
 * number of kernels launched and the milliseconds accumulated since the last
 * kf_timing_reset. */
typedef enum {
    KF_KERNEL_FILTER_SCAN = 0,   /* forward scan, Lemma 1 (Alg. pkf)              */
    KF_KERNEL_RTS_SCAN = 1,      /* reversed scan, Lemma 2 (Alg. prts)            */
    KF_KERNEL_TF_SCAN = 2,       /* reversed scan of (a_2..a_T, e) + merge (ptf)  */
    KF_KERNEL_FILTER_LEVELS = 3, /* the same three, run by a level algorithm      */
    KF_KERNEL_RTS_LEVELS = 4,
    KF_KERNEL_TF_LEVELS = 5,
    KF_KERNEL_KINDS = 6
} kf_kernel_t;
kf_status_t kf_timing_enable(int on);
kf_status_t kf_timing_reset(void);
kf_status_t kf_timing_read(kf_kernel_t kind, int64_t *launches, double *total_ms);

/* Phase trace (diagnostics).  While a buffer is set for a decoupled
 * look-back scan kind (FILTER/RTS/TF_SCAN), every later launch of that scan
 * writes, for each tile t < capacity_tiles, %globaltimer stamps (ns) to
 * device_buffer[16 t + i]: i = 0 CTA start, 1 end of the thread fold + warp
 * scan, 2 aggregate published, 3 look-back done, 4 end of the extraction
 * pass; for tiles > 0 also 5 predecessor flags seen, 6 predecessor folds
 * done, 7 warp trees done, 8 warp-0 tree done, 9 inclusive carry loaded,
 * 10 exclusive carry applied, 11 inclusive carry computed, 12 published.
 * device_buffer is a caller-owned DEVICE buffer of 16 * capacity_tiles
 * uint64; NULL switches the trace off. */
kf_status_t kf_trace_phases(kf_kernel_t kind, void *device_buffer, int capacity_tiles);

/* Autotuner.  kf_autotune times the candidate launch configurations of one
 * call -- the decoupled look-back scan with 128 (and, for nx = 4 in FP32,
 * 256) threads per CTA, 1, 2, 4 or all warps in the look-back and three
 * tile sizes, and the in-place Ladner-Fischer level scan -- on the caller's
 * model, data and output buffers (median of reps runs each, after one
 * warm-up; outputs are overwritten), and records the fastest for
 * (op, nx, ny, precision, floor(log2 T)).  Later calls with KF_SCAN_AUTO and
 * that key use the recorded configuration, unless KF_OPT_THREADS,
 * KF_OPT_LOOKBACK_WARPS or KF_OPT_POSITIONS_PER_THREAD is set.  Synchronous;
 * kf_timing_enable must be off; workspace is null or at least
 * kf_workspace_size(op, ..., KF_SCAN_AUTO) bytes.  kf_tuning_get reads an entry;
 * kf_tuning_save / kf_tuning_load write / merge a text file of entries;
 * kf_tuning_clear empties the table. */
kf_status_t kf_autotune(kf_op_t op, const kf_model_t *model, int64_t T, const void *y, kf_precision_t prec,
                        void *m_out, void *P_out, int reps, void *workspace, void *stream);
kf_status_t kf_tuning_get(kf_op_t op, int nx, int ny, kf_precision_t prec, int64_t T, int *scan, int *threads,
                          int *lookback_warps, int *steps_per_thread, double *ms);
/* Batch autotuner.  kf_autotune_batch times kf_batch_smooth on the caller's
 * batch (same arguments as kf_batch_smooth, no log-likelihoods; outputs are
 * overwritten) for 1, 2 or 4 look-back warps of the 128-thread CTA and
 * three steps-per-thread settings (the library's choice, about half and
 * about twice one wave of resident tiles), median of reps runs each after
 * one warm-up, and records the fastest for (op, nx, ny, precision,
 * floor(log2 total steps)) with nx, ny those of models[0].  Later
 * kf_batch_smooth calls (and the server's batches) whose batch has that key
 * use it, unless KF_OPT_LOOKBACK_WARPS or KF_OPT_POSITIONS_PER_THREAD is set.
 * Synchronous; kf_timing_enable must be off.  The entries share the table
 * (and the file of kf_tuning_save) with the one-sequence entries, under op
 * code op + 8.  kf_batch_tuning_get reads an entry (KF_ERR_ARG if none). */
kf_status_t kf_autotune_batch(kf_op_t op, const kf_model_t *models, int nmodels, const int32_t *model_of_seq, int nseq,
                              const int64_t *offsets, const void *y, kf_precision_t prec, void *m_out, void *P_out,
                              int reps, void *workspace, void *stream);
kf_status_t kf_batch_tuning_get(kf_op_t op, int nx, int ny, kf_precision_t prec, int64_t total_steps,
                                int *lookback_warps, int *steps_per_thread, double *ms);
/* The covariance tables of a time-invariant model with ny = nx / 2 (nx 2,
 * 4 or 8; see KF_OPT_COVARIANCE_TABLES): k0 (the times 1..k0 whose
 * filtering covariance has not yet settled), kb (the times T - kb + 1 .. T
 * whose smoothed covariance has not), and the settled filtering covariance
 * P_inf (nx x nx), gain K_inf (nx x ny), RTS gain E_inf (nx x nx) and
 * smoothed covariance Ps_inf (nx x nx), row-major into host buffers (any
 * may be NULL).  Host only; KF_ERR_ARG when the tables do not apply (the
 * recursion does not settle within 2^16 steps, or a covariance is not
 * positive definite). */
kf_status_t kf_covariance_tables(const kf_model_t *model, int *k0, int *kb, double *P_inf, double *K_inf,
                                 double *E_inf, double *Ps_inf);

/* The launch request of the calling thread's last one-sequence or batched
 * call, after the KF_OPT_* options and the tuning table were applied: the
 * scan (kf_scan_t), threads per CTA, look-back warps and steps per thread,
 * each 0 where the library chooses.  All zero before the first call. */
kf_status_t kf_last_launch_config(int *scan, int *threads, int *lookback_warps, int *steps_per_thread);

/* 1 in the bounds-checked build of the library (compiled with
 * KF_BOUNDS_CHECK: the kernels check their indexes into the inputs, outputs,
 * tables and workspace, record KF_ERR_BOUNDS in the status word on a failed
 * check and skip that access), else 0.  A debugging build: slower, same
 * results. */
int kf_bounds_checked(void);

/* Call graphs (KF_OPT_CALL_GRAPHS) captured and replayed since the library
 * was loaded, over all threads and devices (either pointer may be NULL). */
kf_status_t kf_call_graph_stats(int64_t *captured, int64_t *replayed);
kf_status_t kf_tuning_save(const char *path);
kf_status_t kf_tuning_load(const char *path);
kf_status_t kf_tuning_clear(void);

/* Measures the FP32 (fp64 = 0) or FP64 (fp64 = 1) fused multiply-add
 * throughput of the current device with a kernel of independent FMA chains
 * on every SM, and returns it in FLOP/s (an FMA counts as 2).  Synchronous. */
kf_status_t kf_measure_fma_peak(int fp64, double *flops_per_second);

#ifdef __cplusplus
}
#endif

#endif /* KFSCAN_H */
