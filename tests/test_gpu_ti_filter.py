"""GPU parity of the time-invariant table kernel of the forward filter scan
(KF_OPT_FILTER_KERNEL = 0, the default for a time-invariant model with
ny = nx / 2 on one sequence) against the FP64 oracle, and against the
generic look-back kernel (KF_OPT_FILTER_KERNEL = 1), through the C ABI.

The table kernel takes a_1 as the initial carry and scans a_2 .. a_T in
tiles of THREADS x K positions, so the cases cover T = 1 (no scan position),
T = 2 and 3, one partial tile, exactly full tiles, many tiles with a ragged
last one, more tiles than one thread of the look-back holds (forced K = 1
at T = 100000: up to 781 tiles), both CTA sizes, and the log-likelihood."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import TOL, gpu_run, oracle_inputs, oracle_run, mean_err, cov_err, check_psd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2511_10363_gb300 import build
    build.build()
    import paper_2511_10363_gb300 as kf
    kf.kf_set_option("covariance_tables", 1)   # the per-step kernels
    yield
    kf.kf_set_option("covariance_tables", 0)
    for k in ("positions_per_thread", "threads", "filter_kernel"):
        kf.kf_set_option(k, 0)


def model_for(nx, seed):
    return W.cv_model() if nx == 4 else W.random_model(2, 1, seed=seed)


def run_case(op, nx, T, precision, threads, K, seed, kernel=0, loglik=True):
    import paper_2511_10363_gb300 as kf
    model = model_for(nx, seed)
    y = oracle_inputs(W.simulate(model, T, seed=seed), precision)
    kf.kf_set_option("threads", threads)
    kf.kf_set_option("positions_per_thread", K)
    kf.kf_set_option("filter_kernel", kernel)
    try:
        out = gpu_run(op, model, y, precision, "dlb", loglik=loglik, want_filter=(op != "filter"))
    finally:
        kf.kf_set_option("positions_per_thread", 0)
        kf.kf_set_option("threads", 0)
        kf.kf_set_option("filter_kernel", 0)
    return model, y, out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nx", [2, 4])
@pytest.mark.parametrize("threads", [128, 256])
@pytest.mark.parametrize("T,K", [(1, 0), (2, 0), (3, 0), (257, 0), (257, 1), (5000, 0), (5000, 3), (20481, 5),
                                 (100000, 1), (100000, 0)])
def test_table_kernel_against_oracle(precision, nx, threads, T, K):
    model, y, out = run_case("filter", nx, T, precision, threads, K, seed=T % 97 + nx)
    ref = oracle_run(model, y)
    tol = TOL[precision]
    e_m, e_P = mean_err(out["mf"], ref["mf"], ref["Pf"]), cov_err(out["Pf"], ref["Pf"])
    assert e_m <= tol and e_P <= tol, (e_m, e_P)
    check_psd(out["Pf"])
    # the FP32 log-likelihood is compared while the FP32 positions resolve
    # the innovation (the long tracking sequences drift to ~1e5 and beyond)
    if precision == "fp64" or T <= 5000:
        ll_tol = 1e-9 if precision == "fp64" else 1e-3
        assert abs(out["ll"] - ref["ll"]) <= ll_tol * max(1.0, abs(ref["ll"])), (out["ll"], ref["ll"])


@pytest.mark.parametrize("op", ["rts", "tf"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_table_kernel_feeds_the_smoothers(op, precision):
    """The filter records the table kernel writes (staged per warp in shared
    memory, coalesced stores) are what the smoother passes read."""
    model, y, out = run_case(op, 4, 30001, precision, 256, 0, seed=5, loglik=(precision == "fp64"))
    ref = oracle_run(model, y)
    key = "rts" if op == "rts" else "tf"
    tol = TOL[precision]
    assert mean_err(out["ms"], ref["ms_" + key], ref["Ps_" + key]) <= tol
    assert cov_err(out["Ps"], ref["Ps_" + key]) <= tol
    assert mean_err(out["mf"], ref["mf"], ref["Pf"]) <= tol and cov_err(out["Pf"], ref["Pf"]) <= tol


@pytest.mark.parametrize("nx", [2, 4])
@pytest.mark.parametrize("T,K", [(4097, 0), (60000, 2)])
def test_table_and_generic_kernels_agree(nx, T, K):
    """FP64: the two forward kernels compute the same prefixes (exact algebra
    of Lemma 1 in different orders) to rounding."""
    _, _, a = run_case("filter", nx, T, "fp64", 128, K, seed=7, kernel=0)
    _, _, b = run_case("filter", nx, T, "fp64", 128, K, seed=7, kernel=1)
    assert mean_err(a["mf"], b["mf"], b["Pf"]) < 1e-11 and cov_err(a["Pf"], b["Pf"]) < 1e-11
    assert abs(a["ll"] - b["ll"]) < 1e-11 * abs(b["ll"])


def test_table_kernel_wait_times_out_and_recovers():
    """A tile that never publishes (test hook): the later tiles' bounded
    waits run out, the status word reports KF_ERR_TIMEOUT, the next call is
    correct."""
    import torch
    import paper_2511_10363_gb300 as kf
    model = W.cv_model()
    T = 20000
    y = W.simulate(model, T, seed=9)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    kf.kf_set_option("wait_timeout_ns", 50_000_000)
    kf.kf_set_option("positions_per_thread", 2)
    kf.kf_set_option("test_skip_tile", 3)
    try:
        kf.kf_filter(model, yt, "fp32", "dlb")
        assert kf.kf_sync_status() == 5          # KF_ERR_TIMEOUT
    finally:
        kf.kf_set_option("test_skip_tile", -1)
        kf.kf_set_option("positions_per_thread", 0)
        kf.kf_set_option("wait_timeout_ns", 10 ** 9)
    assert kf.kf_sync_status() == 0
    out = gpu_run("filter", model, y, "fp64", "dlb", loglik=True)
    ref = oracle_run(model, y)
    assert mean_err(out["mf"], ref["mf"], ref["Pf"]) < 1e-9 and cov_err(out["Pf"], ref["Pf"]) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("threads", [128, 256])
def test_plain_and_smoother_launches_interleave(precision, threads):
    """A plain filter call (no record staging, less shared memory) between
    smoother calls (records staged) of the same kernel configuration: every
    launch must be allowed its shared memory, whichever ran first."""
    for op in ("rts", "filter", "rts", "filter"):
        model, y, out = run_case(op, 4, 3000, precision, threads, 0, seed=31, loglik=False)
        ref = oracle_run(model, y)
        tol = TOL[precision]
        assert mean_err(out["mf"], ref["mf"], ref["Pf"]) <= tol and cov_err(out["Pf"], ref["Pf"]) <= tol
