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


@pytest.mark.parametrize("op", ["filter", "rts"])
def test_batch_autotune_applies_and_matches_oracle(op, tmp_path):
    """kf_autotune_batch records an entry for the batch's class and size;
    the next kf_batch_smooth call of that key launches with it (its launch
    request is the entry), and every sequence still matches the oracle."""
    import torch
    import paper_2511_10363_gb300 as kf
    from paper_2511_10363_gb300 import build
    build.build()
    kf.kf_tuning_clear()
    model = W.cv_model()
    rng = np.random.default_rng(17)
    lengths = np.concatenate([[1, 3], rng.integers(100, 6000, size=60)])
    y, _ = W.ragged_batch(model, lengths, seed=23)
    y = y.astype(np.float32).astype(np.float64)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    entry = kf.kf_autotune_batch(op, [model], offs, yt, "fp32", reps=3)
    assert entry is not None and entry["lookback_warps"] in (1, 2, 4) and entry["ms"] > 0
    try:
        m, P, _ = kf.kf_batch_smooth(op, [model], offs, yt, "fp32")
        assert kf.kf_sync_status() == 0
        got = kf.kf_last_launch_config()
        assert got["lookback_warps"] == entry["lookback_warps"]
        assert got["steps_per_thread"] == entry["steps_per_thread"]
        m, P = m.double().cpu().numpy(), P.double().cpu().numpy()
        for s in range(len(lengths)):
            a, b = offs[s], offs[s + 1]
            mf, Pf, _ = oracle.kf(model, y[a:b])
            rm, rP = (mf, Pf) if op == "filter" else oracle.rts(model, mf, Pf)
            assert mean_err(m[a:b], rm, rP) <= TOL["fp32"], s
            assert cov_err(P[a:b], rP) <= TOL["fp32"], s
        # an explicit option overrides the table
        kf.kf_set_option("lookback_warps", 3)
        kf.kf_batch_smooth(op, [model], offs, yt, "fp32")
        assert kf.kf_last_launch_config()["lookback_warps"] == 3
        kf.kf_set_option("lookback_warps", 0)
        # the entry round-trips through the table file
        path = os.path.join(str(tmp_path), "tune.txt")
        kf.kf_tuning_save(path)
        kf.kf_tuning_clear()
        assert kf.kf_batch_tuning_get(op, 4, 2, "fp32", int(offs[-1])) is None
        kf.kf_tuning_load(path)
        assert kf.kf_batch_tuning_get(op, 4, 2, "fp32", int(offs[-1])) == entry
    finally:
        kf.kf_set_option("lookback_warps", 0)
        kf.kf_tuning_clear()
