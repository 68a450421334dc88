// kf_tv_n4.cu -- scans of time-varying models for state dimension nx = 4.
#include "kf_tv.cuh"

namespace kfs {

cudaError_t launch_tv_n4(const TvLaunch &t) { return launch_tv_n<4>(t); }

}  // namespace kfs
