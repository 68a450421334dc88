// kf_n4_f32_t256.cu -- scans for state dimension nx = 4, precision f32, with
// 256-thread CTAs.
#include "kf_launch.cuh"

namespace kfs {

cudaError_t launch_n4_f32_t256(const LaunchReq &q) { return launch_typed<4, float, 0, 256>(q); }

}  // namespace kfs
