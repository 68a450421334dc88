"""Failure detection on the GPU without a GPU fault: the tile that takes a
chosen ticket returns without publishing, so every later tile's bounded
wait runs out (a short limit is set for the test).  The kernels record
KF_ERR_TIMEOUT in the status word and return; the context stays usable and
the next call is correct."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import gpu_run, oracle_run, mean_err, cov_err

pytestmark = pytest.mark.gpu


def test_lookback_wait_times_out_and_recovers():
    import torch
    import paper_2511_10363_gb300 as kf
    from paper_2511_10363_gb300 import build
    build.build()
    model = W.cv_model()
    T = 20000
    y = W.simulate(model, T, seed=9)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    kf.kf_set_option("wait_timeout_ns", 50_000_000)
    kf.kf_set_option("positions_per_thread", 2)
    kf.kf_set_option("test_skip_tile", 3)
    try:
        kf.kf_rts_smooth(model, yt, "fp32", "dlb")
        assert kf.kf_sync_status() == 5          # KF_ERR_TIMEOUT
    finally:
        kf.kf_set_option("test_skip_tile", -1)
        kf.kf_set_option("positions_per_thread", 0)
        kf.kf_set_option("wait_timeout_ns", 10 ** 9)
    assert kf.kf_sync_status() == 0              # status was cleared
    out = gpu_run("rts", model, y, "fp64", "dlb")
    ref = oracle_run(model, y)
    assert mean_err(out["ms"], ref["ms_rts"], ref["Ps_rts"]) < 1e-9
    assert cov_err(out["Ps"], ref["Ps_rts"]) < 1e-9
