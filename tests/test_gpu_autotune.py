"""The autotuner records a configuration, KF_SCAN_AUTO applies it, results
stay correct, and the table round-trips through its text file."""
import os

import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import TOL, mean_err, cov_err

pytestmark = pytest.mark.gpu


def test_autotune_applies_and_persists(tmp_path):
    import torch
    import paper_2511_10363_gb300 as kf
    from paper_2511_10363_gb300 import build
    build.build()
    kf.kf_tuning_clear()
    model = W.cv_model()
    T = 50000
    y = W.simulate(model, T, seed=3).astype(np.float32).astype(np.float64)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    entry = kf.kf_autotune("rts", model, yt, "fp32", reps=3)
    assert entry is not None and entry["scan"] in ("dlb", "ladner_fischer") and entry["ms"] > 0
    ms, Ps, _ = kf.kf_rts_smooth(model, yt, "fp32", "auto")
    assert kf.kf_sync_status() == 0
    mf, Pf, _ = oracle.kf(model, y)
    rm, rP = oracle.rts(model, mf, Pf)
    assert mean_err(ms.double().cpu().numpy(), rm, rP) <= TOL["fp32"]
    assert cov_err(Ps.double().cpu().numpy(), rP) <= TOL["fp32"]
    path = os.path.join(str(tmp_path), "tune.txt")
    kf.kf_tuning_save(path)
    kf.kf_tuning_clear()
    assert kf.kf_tuning_get("rts", 4, 2, "fp32", T) is None
    kf.kf_tuning_load(path)
    assert kf.kf_tuning_get("rts", 4, 2, "fp32", T) == entry
    # the same key covers the length bucket [2^15, 2^16)
    assert kf.kf_tuning_get("rts", 4, 2, "fp32", 40000) == entry
    kf.kf_tuning_clear()
