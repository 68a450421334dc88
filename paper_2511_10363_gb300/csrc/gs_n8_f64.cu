// The covariance-table path (gain_launch.cuh) for nx = 8 in double.
#include "gain_launch.cuh"

namespace kfs {

bool gain_launch(NTag<8>, const GainModel &g, const LaunchReq &q, const KfBufs<double> &buf, char *ws,
                 const WsLayout &L, double *ll, cudaError_t *err) {
    return gain_run<8, double>(g, q, buf, ws, L, ll, err);
}

}  // namespace kfs
