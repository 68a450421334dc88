// ti_n4_f32.cu -- the time-invariant forward filter table kernel and the
// one-sequence RTS pass kernel, nx = 4, FP32.
#include "rts_launch.cuh"
#include "ti_launch.cuh"

namespace kfs {

bool ti_filter_launch(const FiltParams<4, float> &prm, const LaunchReq &q, const KfBufs<float> &buf, char *ws,
                      const WsLayout &L, double *ll, cudaError_t *err) {
    return ti_filter_launch_impl<4, float>(prm, q, buf, ws, L, ll, err);
}

bool rts_pass_launch(const FiltParams<4, float> &prm, const LaunchReq &q, const KfBufs<float> &buf, char *ws,
                     const WsLayout &L, cudaError_t *err) {
    return rts_launch_impl<4, float>(prm, q, buf, ws, L, err);
}

}  // namespace kfs
