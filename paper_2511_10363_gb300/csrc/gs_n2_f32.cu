// The covariance-table path (gain_launch.cuh) for nx = 2 in float.
#include "gain_launch.cuh"

namespace kfs {

bool gain_launch(NTag<2>, const GainModel &g, const LaunchReq &q, const KfBufs<float> &buf, char *ws,
                 const WsLayout &L, double *ll, cudaError_t *err) {
    return gain_run<2, float>(g, q, buf, ws, L, ll, err);
}

}  // namespace kfs
