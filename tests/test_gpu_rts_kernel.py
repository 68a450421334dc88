"""GPU parity of the dedicated RTS pass kernel of one sequence
(KF_OPT_RTS_KERNEL = 0, the default for nx 2 and 4 with the decoupled
look-back scan) against the FP64 oracle, and against the generic look-back
kernel (KF_OPT_RTS_KERNEL = 1), through the C ABI.

The kernel builds each element from its filter record in the direct form of
Lemma 2 and takes the last element (E_T = 0) in place; the cases cover
T = 1, 2 and 3, one partial tile, many tiles with a ragged first one (the
reverse scan's last tile holds the earliest times), more tiles than one
thread of the look-back holds, both CTA sizes, and every precision."""
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
    for k in ("positions_per_thread", "threads", "rts_kernel"):
        kf.kf_set_option(k, 0)


def model_for(nx, seed):
    return W.cv_model() if nx == 4 else W.random_model(2, 1, seed=seed)


def run_case(nx, T, precision, threads, K, seed, kernel=0):
    import paper_2511_10363_gb300 as kf
    model = model_for(nx, seed)
    y = oracle_inputs(W.simulate(model, T, seed=seed), precision)
    kf.kf_set_option("threads", threads)
    kf.kf_set_option("positions_per_thread", K)
    kf.kf_set_option("rts_kernel", kernel)
    try:
        out = gpu_run("rts", model, y, precision, "dlb", loglik=False, want_filter=True)
    finally:
        kf.kf_set_option("positions_per_thread", 0)
        kf.kf_set_option("threads", 0)
        kf.kf_set_option("rts_kernel", 0)
    return model, y, out


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_fp64solve"])
@pytest.mark.parametrize("nx", [2, 4])
@pytest.mark.parametrize("threads", [128, 256])
@pytest.mark.parametrize("T,K", [(1, 0), (2, 0), (3, 0), (257, 0), (257, 1), (5000, 3), (30001, 0), (100000, 1)])
def test_rts_kernel_against_oracle(precision, nx, threads, T, K):
    model, y, out = run_case(nx, T, precision, threads, K, seed=T % 89 + nx)
    ref = oracle_run(model, y)
    tol = TOL[precision]
    e_m, e_P = mean_err(out["ms"], ref["ms_rts"], ref["Ps_rts"]), cov_err(out["Ps"], ref["Ps_rts"])
    assert e_m <= tol and e_P <= tol, (e_m, e_P)
    check_psd(out["Ps"])


@pytest.mark.parametrize("nx", [2, 4])
@pytest.mark.parametrize("T,K", [(4097, 0), (60000, 2)])
def test_rts_kernels_agree(nx, T, K):
    """FP64: the dedicated and the generic RTS kernels give the same smoothed
    moments (Lemma 2 in different association orders) to rounding."""
    _, _, a = run_case(nx, T, "fp64", 128, K, seed=11, kernel=0)
    _, _, b = run_case(nx, T, "fp64", 128, K, seed=11, kernel=1)
    assert mean_err(a["ms"], b["ms"], b["Ps"]) < 1e-11 and cov_err(a["Ps"], b["Ps"]) < 1e-11


def test_rts_kernel_wait_times_out_and_recovers():
    """A tile of the RTS pass that never publishes (test hook; the forward
    pass's tile of the same ticket times out first and the status word stops
    the rest): KF_ERR_TIMEOUT is reported and the next call is correct."""
    import torch
    import paper_2511_10363_gb300 as kf
    model = W.cv_model()
    T = 20000
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
    _, yo, out = run_case(4, T, "fp32", 256, 0, seed=19)
    ref = oracle_run(W.cv_model(), yo)
    assert mean_err(out["ms"], ref["ms_rts"], ref["Ps_rts"]) <= 1e-4
    assert cov_err(out["Ps"], ref["Ps_rts"]) <= 1e-4
