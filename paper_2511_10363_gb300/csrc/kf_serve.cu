// kf_serve.cu -- continuous-batching server for filter / smoother jobs
// (kf_server_* in include/kfscan.h).
//
// A scheduler thread owns one device arena of the memory budget (allocated
// once at creation) and a few CUDA streams.  Jobs wait in a FIFO queue.
// Whenever a stream is free, the scheduler takes the oldest queued job,
// gathers the following queued jobs of the same class (operation, nx, ny,
// precision) while they fit in the free arena space and the batch limits,
// copies their measurements in, runs one segmented scan over the batch
// (kf_batch_smooth with a workspace carved from the arena), copies each
// job's results out and records an event.  Jobs that arrive while batches
// are on the GPU are admitted as soon as a stream and enough memory are
// free, so their work overlaps the running batches.  A finished batch
// returns its memory to the arena.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/kfscan.h"
#include "kf_host.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device arena; blocks are 256-byte aligned.
class Arena {
  public:
    void init(size_t bytes) {
        size_ = bytes;
        free_.clear();
        free_[0] = bytes;
    }
    // returns the offset, or SIZE_MAX if no free block is large enough
    size_t alloc(size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_ += bytes;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~size_t(255);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t largest_free() const {
        size_t m = 0;
        for (auto &f : free_) m = std::max(m, f.second);
        return m;
    }
    size_t size() const { return size_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

struct Job {
    int64_t id;
    kf_op_t op;
    kf_precision_t prec;
    int nx, ny;
    int64_t T;
    double mat[6][64];          // deep copy of F, Q, H, R, m0, P0
    kf_model_t model;
    const void *y_host;
    void *m_host, *P_host;
    double *ll_host;
    double t_submit = 0, t_start = 0, t_done = 0;
    int64_t batch = -1;
    int status = KF_OK;
    bool done = false;
};

struct Batch {
    int64_t index;
    std::vector<Job *> jobs;
    int stream_idx;
    size_t off, bytes;
    cudaEvent_t ev;
    int status = KF_OK;
};

size_t elt(kf_precision_t p) { return p == KF_FP64 ? 8 : 4; }

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// device bytes of a batch: y, means, covariances, log-likelihoods, workspace
size_t batch_bytes(kf_op_t op, int nx, int ny, kf_precision_t prec, int64_t total, int nseq) {
    const size_t w = elt(prec);
    size_t b = al256(size_t(total) * ny * w) + al256(size_t(total) * nx * w) + al256(size_t(total) * nx * nx * w) +
               al256(sizeof(double) * size_t(nseq));
    b += al256(kf_batch_workspace_size(op, nx, ny, total, nseq, nseq, prec, 1));
    return b;
}

}  // namespace

struct kf_server {
    int device;
    size_t budget;
    int max_inflight;
    int64_t max_batch_steps;
    int max_batch_jobs;
    char *arena_base = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    std::deque<Job *> queue;
    std::vector<Batch *> inflight;
    std::map<int64_t, Job *> jobs;
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::thread worker;
    bool stop = false;
    int64_t next_id = 1, next_batch = 0;
    int sticky_error = KF_OK;

    void launch(Batch *b);
    void complete(Batch *b);
    void loop();
};

void kf_server::launch(Batch *b) {
    Job *j0 = b->jobs[0];
    const int nx = j0->nx, ny = j0->ny, nseq = int(b->jobs.size());
    const size_t w = elt(j0->prec);
    std::vector<int64_t> offs(nseq + 1, 0);
    std::vector<int32_t> mof(nseq);
    std::vector<kf_model_t> models(nseq);
    for (int s = 0; s < nseq; ++s) {
        offs[s + 1] = offs[s] + b->jobs[s]->T;
        mof[s] = s;
        models[s] = b->jobs[s]->model;
    }
    const int64_t total = offs[nseq];
    char *base = arena_base + b->off;
    char *y = base;
    char *m = y + al256(size_t(total) * ny * w);
    char *P = m + al256(size_t(total) * nx * w);
    double *ll = reinterpret_cast<double *>(P + al256(size_t(total) * nx * nx * w));
    char *ws = reinterpret_cast<char *>(ll) + al256(sizeof(double) * size_t(nseq));
    cudaStream_t st = streams[b->stream_idx];
    int status = KF_OK;
    for (int s = 0; s < nseq && status == KF_OK; ++s) {
        if (cudaMemcpyAsync(y + size_t(offs[s]) * ny * w, b->jobs[s]->y_host, size_t(b->jobs[s]->T) * ny * w,
                            cudaMemcpyHostToDevice, st) != cudaSuccess)
            status = KF_ERR_CUDA;
    }
    if (status == KF_OK)
        status = kf_batch_smooth(j0->op, models.data(), nseq, mof.data(), nseq, offs.data(), y, j0->prec, m, P, ll, ws,
                                 st);
    for (int s = 0; s < nseq && status == KF_OK; ++s) {
        Job *j = b->jobs[s];
        const size_t T = size_t(j->T);
        if (j->m_host && cudaMemcpyAsync(j->m_host, m + size_t(offs[s]) * nx * w, T * nx * w, cudaMemcpyDeviceToHost,
                                          st) != cudaSuccess)
            status = KF_ERR_CUDA;
        if (j->P_host && cudaMemcpyAsync(j->P_host, P + size_t(offs[s]) * nx * nx * w, T * nx * nx * w,
                                          cudaMemcpyDeviceToHost, st) != cudaSuccess)
            status = KF_ERR_CUDA;
        if (j->ll_host && cudaMemcpyAsync(j->ll_host, ll + s, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            status = KF_ERR_CUDA;
    }
    cudaEventRecord(b->ev, st);
    b->status = status;
}

void kf_server::complete(Batch *b) {
    const double t = now_s();
    for (Job *j : b->jobs) {
        j->t_done = t;
        j->status = b->status;
        j->done = true;
    }
    arena.release(b->off, b->bytes);
    stream_busy[b->stream_idx] = false;
    cudaEventDestroy(b->ev);
    delete b;
}

void kf_server::loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        // retire finished batches
        bool progressed = false;
        for (size_t i = 0; i < inflight.size();) {
            if (cudaEventQuery(inflight[i]->ev) == cudaSuccess) {
                complete(inflight[i]);
                inflight.erase(inflight.begin() + i);
                progressed = true;
            } else {
                ++i;
            }
        }
        if (progressed) cv_done.notify_all();
        if (stop && queue.empty() && inflight.empty()) break;
        // admit: form batches while a stream is free
        while (!queue.empty()) {
            int si = -1;
            for (int i = 0; i < max_inflight; ++i)
                if (!stream_busy[i]) {
                    si = i;
                    break;
                }
            if (si < 0) break;
            Job *h = queue.front();
            std::vector<Job *> sel{h};
            int64_t total = h->T;
            size_t need = batch_bytes(h->op, h->nx, h->ny, h->prec, total, 1);
            const size_t avail = arena.largest_free();
            if (need > avail) break;   // wait for memory to free up (FIFO head first)
            for (size_t k = 1; k < queue.size() && int(sel.size()) < max_batch_jobs; ++k) {
                Job *j = queue[k];
                if (j->op != h->op || j->nx != h->nx || j->ny != h->ny || j->prec != h->prec) continue;
                if (total + j->T > max_batch_steps) continue;
                const size_t n2 = batch_bytes(h->op, h->nx, h->ny, h->prec, total + j->T, int(sel.size()) + 1);
                if (n2 > avail) continue;
                sel.push_back(j);
                total += j->T;
                need = n2;
            }
            const size_t off = arena.alloc(need);
            if (off == SIZE_MAX) break;
            for (Job *j : sel) queue.erase(std::find(queue.begin(), queue.end(), j));
            Batch *b = new Batch;
            b->index = next_batch++;
            const double t = now_s();
            for (Job *j : sel) {
                j->t_start = t;
                j->batch = b->index;
            }
            b->jobs = sel;
            b->stream_idx = si;
            b->off = off;
            b->bytes = need;
            cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming);
            stream_busy[si] = true;
            inflight.push_back(b);
            lk.unlock();
            launch(b);   // enqueue copies and kernels without holding the lock
            lk.lock();
        }
        cv_work.wait_for(lk, std::chrono::microseconds(inflight.empty() ? 2000 : 20));
    }
}

extern "C" {

kf_status_t kf_server_create(size_t budget_bytes, int max_inflight, int64_t max_batch_steps, kf_server_t **out) {
    if (!out || budget_bytes < (1u << 20) || max_inflight < 1 || max_inflight > 16 || max_batch_steps < 1)
        return KF_ERR_ARG;
    kf_server *s = new kf_server;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return KF_ERR_CUDA;
    }
    s->budget = budget_bytes;
    s->max_inflight = max_inflight;
    s->max_batch_steps = max_batch_steps;
    s->max_batch_jobs = 4096;
    if (cudaMalloc(&s->arena_base, budget_bytes) != cudaSuccess) {
        delete s;
        return KF_ERR_OOM;
    }
    s->arena.init(budget_bytes);
    s->streams.resize(max_inflight);
    s->stream_busy.assign(max_inflight, false);
    for (auto &st : s->streams) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    s->worker = std::thread([s] { s->loop(); });
    *out = s;
    return KF_OK;
}

kf_status_t kf_server_submit(kf_server_t *srv, kf_op_t op, const kf_model_t *model, int64_t T, const void *y_host,
                             kf_precision_t prec, void *m_host, void *P_host, double *loglik_host, int64_t *job_id) {
    if (!srv || !model || !y_host || T < 1 || !job_id) return KF_ERR_ARG;
    if (op < KF_OP_FILTER || op > KF_OP_TWO_FILTER) return KF_ERR_ARG;
    if (prec != KF_FP64 && prec != KF_FP32 && prec != KF_FP32_FP64SOLVE) return KF_ERR_ARG;
    const int nx = model->nx, ny = model->ny;
    if ((nx != 2 && nx != 4 && nx != 8) || ny < 1 || ny > 8) return KF_ERR_ARG;
    if (!model->F || !model->Q || !model->H || !model->R || !model->m0 || !model->P0) return KF_ERR_ARG;
    if (batch_bytes(op, nx, ny, prec, T, 1) > srv->budget) return KF_ERR_BUDGET;
    Job *j = new Job;
    j->op = op;
    j->prec = prec;
    j->nx = nx;
    j->ny = ny;
    j->T = T;
    const double *src[6] = {model->F, model->Q, model->H, model->R, model->m0, model->P0};
    const int len[6] = {nx * nx, nx * nx, ny * nx, ny * ny, nx, nx * nx};
    for (int i = 0; i < 6; ++i) memcpy(j->mat[i], src[i], sizeof(double) * len[i]);
    j->model = kf_model_t{nx, ny, j->mat[0], j->mat[1], j->mat[2], j->mat[3], j->mat[4], j->mat[5]};
    j->y_host = y_host;
    j->m_host = m_host;
    j->P_host = P_host;
    j->ll_host = loglik_host;
    j->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->stop) {
            delete j;
            return KF_ERR_BUSY;
        }
        j->id = srv->next_id++;
        srv->jobs[j->id] = j;
        srv->queue.push_back(j);
        *job_id = j->id;
    }
    srv->cv_work.notify_one();
    return KF_OK;
}

kf_status_t kf_server_poll(kf_server_t *srv, int64_t job_id, int *done, double *info) {
    if (!srv || !done) return KF_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return KF_ERR_BUSY;
    Job *j = it->second;
    *done = j->done ? 1 : 0;
    if (info) {
        info[0] = j->t_submit;
        info[1] = j->t_start;
        info[2] = j->t_done;
        info[3] = double(j->batch);
    }
    return j->done ? kf_status_t(j->status) : KF_OK;
}

kf_status_t kf_server_wait(kf_server_t *srv, int64_t job_id, double timeout_s) {
    if (!srv) return KF_ERR_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end()) return KF_ERR_BUSY;
    Job *j = it->second;
    const bool ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [j] { return j->done; });
    if (!ok) return KF_ERR_TIMEOUT;
    return kf_status_t(j->status);
}

kf_status_t kf_server_release(kf_server_t *srv, int64_t job_id) {
    if (!srv) return KF_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(job_id);
    if (it == srv->jobs.end() || !it->second->done) return KF_ERR_BUSY;
    delete it->second;
    srv->jobs.erase(it);
    return KF_OK;
}

kf_status_t kf_server_cancel(kf_server_t *srv, int64_t job_id) {
    if (!srv) return KF_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->jobs.find(job_id);
        if (it == srv->jobs.end()) return KF_ERR_BUSY;
        Job *j = it->second;
        auto q = std::find(srv->queue.begin(), srv->queue.end(), j);
        if (j->done || q == srv->queue.end()) return KF_ERR_BUSY;   // running or finished
        srv->queue.erase(q);
        j->status = KF_ERR_CANCELLED;
        j->t_done = now_s();
        j->done = true;
    }
    srv->cv_done.notify_all();
    srv->cv_work.notify_one();
    return KF_OK;
}

kf_status_t kf_server_destroy(kf_server_t *srv) {
    if (!srv) return KF_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    srv->worker.join();
    for (auto &st : srv->streams) cudaStreamDestroy(st);
    cudaFree(srv->arena_base);
    for (auto &kv : srv->jobs) delete kv.second;
    delete srv;
    return KF_OK;
}

}  // extern "C"
