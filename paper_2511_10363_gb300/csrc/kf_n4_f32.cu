// kf_n4_f32.cu -- scans for state dimension nx = 4, precision f32.
#include "kf_launch.cuh"

namespace kfs {

size_t ws_bytes_n4_f32(int op, int scan, int64_t T) { return ws_layout<4, float>(op, scan, T).total; }

// 256-thread CTAs: separate translation unit (kf_n4_f32_t256.cu), compiled in parallel
cudaError_t launch_n4_f32_t256(const LaunchReq &q);

cudaError_t launch_n4_f32(const LaunchReq &q) {
    if (q.threads == 256) return launch_n4_f32_t256(q);
    return launch_typed<4, float, 0, 128>(q);
}

size_t batch_ws_bytes_n4_f32(int op, int64_t T, int nseq, int nmodels, int loglik) {
    return batch_layout<4, float>(op, T, nseq, nmodels, loglik != 0).total;
}

cudaError_t launch_batch_n4_f32(const LaunchReq &q, const BatchReq &b) { return launch_batch_typed<4, float, 0, 128>(q, b); }

}  // namespace kfs
