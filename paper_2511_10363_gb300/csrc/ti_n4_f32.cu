// ti_n4_f32.cu -- the time-invariant forward filter table kernel, nx = 4, FP32.
#include "ti_launch.cuh"

namespace kfs {

bool ti_filter_launch(const FiltParams<4, float> &prm, const LaunchReq &q, const KfBufs<float> &buf, char *ws,
                      const WsLayout &L, double *ll, cudaError_t *err) {
    return ti_filter_launch_impl<4, float>(prm, q, buf, ws, L, ll, err);
}

}  // namespace kfs
