// kf_n4_mix.cu -- scans for state dimension nx = 4, precision mix.
#include "kf_launch.cuh"

namespace kfs {

size_t ws_bytes_n4_mix(int op, int scan, int64_t T) { return ws_layout<4, float>(op, scan, T).total; }

cudaError_t launch_n4_mix(const LaunchReq &q) { return launch_typed<4, float, 1, 128>(q); }

}  // namespace kfs
