// The covariance-table path (gain_launch.cuh) for nx = 4 in double.
#include "gain_launch.cuh"

namespace kfs {

bool gain_launch(NTag<4>, const GainModel &g, const LaunchReq &q, const KfBufs<double> &buf, char *ws,
                 const WsLayout &L, double *ll, cudaError_t *err) {
    return gain_run<4, double>(g, q, buf, ws, L, ll, err);
}

}  // namespace kfs
