// kf_n4_mix_batch.cu -- batched (segmented) scans for state dimension
// nx = 4, precision mix: a translation unit of its own, compiled in parallel
// with the single-sequence unit.
#include "kf_launch.cuh"

namespace kfs {
cudaError_t launch_batch_n4_mix(const LaunchReq &q, const BatchReq &b) { return launch_batch_typed<4, float, 1, 128>(q, b); }
}  // namespace kfs
