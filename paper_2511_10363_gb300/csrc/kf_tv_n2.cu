// kf_tv_n2.cu -- scans of time-varying models for state dimension nx = 2.
#include "kf_tv.cuh"

namespace kfs {

cudaError_t launch_tv_n2(const TvLaunch &t) { return launch_tv_n<2>(t); }

}  // namespace kfs
