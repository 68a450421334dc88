// kf_n8_f64_batch.cu -- batched (segmented) scans for state dimension
// nx = 8, precision f64: a translation unit of its own, compiled in parallel
// with the single-sequence unit.
#include "kf_launch.cuh"

namespace kfs {
cudaError_t launch_batch_n8_f64(const LaunchReq &q, const BatchReq &b) { return launch_batch_typed<8, double, 0, 128>(q, b); }
}  // namespace kfs
