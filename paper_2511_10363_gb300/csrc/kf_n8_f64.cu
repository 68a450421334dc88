// kf_n8_f64.cu -- scans for state dimension nx = 8, precision f64.
#include "kf_launch.cuh"

namespace kfs {

size_t ws_bytes_n8_f64(int op, int scan, int64_t T) { return ws_layout<8, double>(op, scan, T).total; }

cudaError_t launch_n8_f64(const LaunchReq &q) { return launch_typed<8, double, 0, 128>(q); }

size_t batch_ws_bytes_n8_f64(int op, int64_t T, int nseq, int nmodels, int loglik) {
    return batch_layout<8, double>(op, T, nseq, nmodels, loglik != 0).total;
}


}  // namespace kfs
