// kf_n8_mix.cu -- scans for state dimension nx = 8, precision mix.
#include "kf_launch.cuh"

namespace kfs {

size_t ws_bytes_n8_mix(int op, int scan, int64_t T) { return ws_layout<8, float>(op, scan, T).total; }

cudaError_t launch_n8_mix(const LaunchReq &q) { return launch_typed<8, float, 1, 128>(q); }

size_t batch_ws_bytes_n8_mix(int op, int64_t T, int nseq, int nmodels, int loglik) {
    return batch_layout<8, float>(op, T, nseq, nmodels, loglik != 0).total;
}


}  // namespace kfs
