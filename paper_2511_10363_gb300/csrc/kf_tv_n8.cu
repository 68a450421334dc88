// kf_tv_n8.cu -- scans of time-varying models for state dimension nx = 8.
#include "kf_tv.cuh"

namespace kfs {

cudaError_t launch_tv_n8(const TvLaunch &t) { return launch_tv_n<8>(t); }

}  // namespace kfs
