// ti_n4_f64.cu -- the time-invariant forward filter table kernel, nx = 4, FP64.
#include "ti_launch.cuh"

namespace kfs {

bool ti_filter_launch(const FiltParams<4, double> &prm, const LaunchReq &q, const KfBufs<double> &buf, char *ws,
                      const WsLayout &L, double *ll, cudaError_t *err) {
    return ti_filter_launch_impl<4, double>(prm, q, buf, ws, L, ll, err);
}

}  // namespace kfs
