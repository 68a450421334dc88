"""GPU parity of the covariance-table path (KF_OPT_COVARIANCE_TABLES = 0):
kf_filter and kf_rts_smooth on a time-invariant model with ny = nx / 2 take
the filtering covariances, gains and smoothed covariances from host FP64
tables and scan only the means on the device, as affine maps with
data-independent coefficients (Lemma 1 and Lemma 2 restricted to their
data-dependent halves).

The cases cover the transient tile alone (T below k0, the steps before the
covariance settles), T just above the smoother's minimum k0 + kb + 1, one
and many bulk tiles with the transient tile taking the remainder, forced
steps per thread down to 1 (hundreds of tiles, look-back depth above 1 in
FP64), every precision and state size, the filter outputs of the smoother,
the log-likelihood, agreement with the per-step kernels, and a look-back
that times out."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import TOL, gpu_run, oracle_inputs, oracle_run, mean_err, cov_err, check_psd

pytestmark = pytest.mark.gpu

PRECS = ["fp64", "fp32", "fp32_fp64solve"]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2511_10363_gb300 import build
    build.build()
    import paper_2511_10363_gb300 as kf
    yield
    for k in ("positions_per_thread", "covariance_tables"):
        kf.kf_set_option(k, 0)


def model_for(nx):
    return W.model_for_nx(nx, seed=nx)


def tables_of(model):
    import paper_2511_10363_gb300 as kf
    t = kf.kf_covariance_tables(model)
    assert t is not None
    return t


def check(op, model, y, precision, K=0, loglik=None):
    """loglik (default): in FP64 always, in FP32 up to T = 30001 -- beyond
    that the tracking positions grow until the FP32 spacing exceeds the
    innovation's standard deviation, and no FP32 evaluation of the innovation
    term is accurate (the same limit as for the per-step kernels)."""
    import paper_2511_10363_gb300 as kf
    if loglik is None:
        loglik = precision == "fp64" or y.shape[0] <= 30001
    yo = oracle_inputs(y, precision)
    ref = oracle_run(model, yo)
    kf.kf_set_option("positions_per_thread", K)
    try:
        out = gpu_run(op, model, yo, precision, "dlb", loglik=loglik, want_filter=(op != "filter"))
    finally:
        kf.kf_set_option("positions_per_thread", 0)
    tol = TOL[precision]
    errs = {"mf": mean_err(out["mf"], ref["mf"], ref["Pf"]), "Pf": cov_err(out["Pf"], ref["Pf"])}
    check_psd(out["Pf"])
    if op == "rts":
        errs["ms"] = mean_err(out["ms"], ref["ms_rts"], ref["Ps_rts"])
        errs["Ps"] = cov_err(out["Ps"], ref["Ps_rts"])
        check_psd(out["Ps"])
    for k, v in errs.items():
        assert v <= tol, (op, precision, k, v)
    if loglik:
        ll_tol = 1e-9 if precision == "fp64" else 1e-3
        assert abs(out["ll"] - ref["ll"]) <= ll_tol * max(1.0, abs(ref["ll"])), (out["ll"], ref["ll"])
    return out


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("nx", [2, 4, 8])
@pytest.mark.parametrize("T", [1, 2, 50, "k0", "k0+1", 1000, 4097, 100000])
def test_filter_against_oracle(precision, nx, T):
    model = model_for(nx)
    k0 = tables_of(model)["k0"]
    T = {"k0": k0, "k0+1": k0 + 1}.get(T, T)
    y = W.simulate(model, T, seed=T % 97 + nx)
    check("filter", model, y, precision)


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("nx", [2, 4, 8])
@pytest.mark.parametrize("T", ["min", "min+1", 1000, 4097, 30001, 100000])
def test_rts_against_oracle(precision, nx, T):
    model = model_for(nx)
    t = tables_of(model)
    lo = t["k0"] + t["kb"] + 1
    T = {"min": lo, "min+1": lo + 1}.get(T, T)
    y = W.simulate(model, T, seed=T % 89 + nx)
    check("rts", model, y, precision)


@pytest.mark.parametrize("K", [1, 2, 5])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_many_tiles(K, precision):
    """Forced steps per thread: T = 60000 spans up to 469 tiles, and in FP64
    the look-back composes several predecessors before its depth limit."""
    model = W.cv_model()
    y = W.simulate(model, 60000, seed=70 + K)
    check("filter", model, y, precision, K=K)
    check("rts", model, y, precision, K=K)


@pytest.mark.parametrize("op", ["filter", "rts"])
@pytest.mark.parametrize("nx", [2, 4, 8])
def test_agrees_with_per_step_kernels(op, nx):
    """FP64: the table path and the per-step kernels give the same moments
    to rounding (the tables settle at a relative change of 2^-46)."""
    import paper_2511_10363_gb300 as kf
    model = model_for(nx)
    y = W.simulate(model, 20000, seed=nx)
    a = gpu_run(op, model, y, "fp64", "dlb", loglik=True, want_filter=(op != "filter"))
    kf.kf_set_option("covariance_tables", 1)
    try:
        b = gpu_run(op, model, y, "fp64", "dlb", loglik=True, want_filter=(op != "filter"))
    finally:
        kf.kf_set_option("covariance_tables", 0)
    keys = [("mf", "Pf")] + ([("ms", "Ps")] if op == "rts" else [])
    for km, kP in keys:
        assert mean_err(a[km], b[km], b[kP]) < 1e-11, km
        assert cov_err(a[kP], b[kP]) < 1e-11, kP
    assert abs(a["ll"] - b["ll"]) <= 1e-11 * abs(b["ll"])


def test_bench_length_fp32_sampled():
    """The benchmark's workload (T = 2^20, FP32, smoother with the
    log-likelihood), every output against the oracle."""
    model = W.cv_model()
    y = W.simulate(model, 1 << 20, seed=1)
    check("rts", model, y, "fp32")


def test_lookback_times_out_and_recovers():
    """A bulk tile that never publishes (test hook): the tiles after it time
    out, KF_ERR_TIMEOUT is reported, and the next call is correct."""
    import torch
    import paper_2511_10363_gb300 as kf
    model = W.cv_model()
    T = 50000
    y = W.simulate(model, T, seed=19)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    kf.kf_set_option("wait_timeout_ns", 50_000_000)
    kf.kf_set_option("positions_per_thread", 2)
    kf.kf_set_option("test_skip_tile", 5)
    try:
        kf.kf_rts_smooth(model, yt, "fp32", "dlb")
        assert kf.kf_sync_status() == 5          # KF_ERR_TIMEOUT
    finally:
        kf.kf_set_option("test_skip_tile", -1)
        kf.kf_set_option("positions_per_thread", 0)
        kf.kf_set_option("wait_timeout_ns", 10 ** 9)
    assert kf.kf_sync_status() == 0
    check("rts", model, y, "fp32")


def test_smoother_below_minimum_length_uses_per_step_kernels():
    """T < k0 + kb + 1: the smoother's tables do not cover the length, and the
    call runs the per-step kernels (same results as the oracle)."""
    model = W.cv_model()
    t = tables_of(model)
    T = t["k0"] + t["kb"]
    y = W.simulate(model, T, seed=5)
    check("rts", model, y, "fp32")
    check("rts", model, y, "fp64")


def test_repeated_calls_replay_a_call_graph():
    """KF_OPT_CALL_GRAPHS (default 1): the second call with the same buffers,
    length and model captures a graph of the memset and both kernels, later
    ones replay it.  The replays read the buffers' current contents (the
    measurements alternate between two sequences), every output matches the
    oracle, and the same calls with the option at 0 launch directly."""
    import torch
    import paper_2511_10363_gb300 as kf
    model = W.cv_model()
    T = 30000
    ys = [oracle_inputs(W.simulate(model, T, seed=s), "fp32") for s in (31, 32)]
    refs = [oracle_run(model, yo) for yo in ys]
    yt = torch.empty((T, 2), dtype=torch.float32, device="cuda")
    ms = torch.empty((T, 4), dtype=torch.float32, device="cuda")
    Ps = torch.empty((T, 4, 4), dtype=torch.float32, device="cuda")
    ll = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(kf.kf_workspace_size("rts", 4, 2, T, "fp32", "auto"), dtype=torch.uint8, device="cuda")
    for graphs in (1, 0):
        kf.kf_set_option("call_graphs", graphs)
        try:
            s0 = kf.kf_call_graph_stats()
            for rep in range(3):
                for yo, ref in zip(ys, refs):
                    yt.copy_(torch.tensor(yo, dtype=torch.float32))
                    kf.kf_rts_smooth(model, yt, "fp32", "auto", ms_out=ms, Ps_out=Ps, loglik=ll, workspace=ws)
                    assert kf.kf_sync_status() == 0
                    Ps_h = Ps.double().cpu().numpy()
                    assert mean_err(ms.double().cpu().numpy(), ref["ms_rts"], ref["Ps_rts"]) <= TOL["fp32"]
                    assert cov_err(Ps_h, ref["Ps_rts"]) <= TOL["fp32"]
                    assert abs(ll.item() - ref["ll"]) <= 1e-3 * abs(ref["ll"])
            s1 = kf.kf_call_graph_stats()
        finally:
            kf.kf_set_option("call_graphs", 1)
        if graphs:   # (captured at the second call, unless an earlier test left this key's graph)
            assert s1["captured"] - s0["captured"] <= 1, (s0, s1)
            assert s1["replayed"] - s0["replayed"] >= 5, (s0, s1)
        else:
            assert s1 == s0
