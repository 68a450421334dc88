// kf_tv_host.h -- declarations shared by the C-ABI layer (kf_api.cu) and the
// launch units of time-varying models (kf_tv_n2.cu, kf_tv_n4.cu, kf_tv_n8.cu).
#pragma once

#include "kf_host.h"

namespace kfs {

// One call on a time-varying model: per-step arrays in device memory in the
// working precision, record t = 0 .. T-1 belonging to time k = t + 1:
//   F[t] = F_{k-1} [N][N], Q[t] = Q_{k-1} [N][N], u[t] = u_{k-1} [N] (or null),
//   H[t] = H_k [ny][N],   R[t] = R_k [ny][ny],    d[t] = d_k [ny] (or null).
struct TvLaunch {
    LaunchReq q;   // op, prec, T, y, outputs, loglik, workspace, stream, status word, options
    int ny;
    const void *F, *Q, *u, *H, *R, *d;
    double m0[KF_MAXN], P0[KF_MAXN * KF_MAXN];   // prior xbar_{0|0}, P_{0|0} (host FP64)
};

cudaError_t launch_tv_n2(const TvLaunch &t);
cudaError_t launch_tv_n4(const TvLaunch &t);
cudaError_t launch_tv_n8(const TvLaunch &t);

}  // namespace kfs
