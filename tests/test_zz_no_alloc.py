"""The no-allocation RTS smoother (kf_rts_smooth_noalloc) against the
ordinary entry point and the FP64 oracle, and its wait time-out report.

Some callers cannot allocate device memory during a call (their memory is
owned by another allocator, or they cannot afford cudaMalloc's implicit
synchronisation); kf_rts_smooth_noalloc serves them from a fixed scratch
array inside the library.  This file is named so that pytest collects it
last.  Each test makes two calls in a row through the C ABI and compares
both with kf_rts_smooth on the same inputs, with the tolerances of the
other parity tests, and must pass alone in a fresh process as well as after
every other test."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import TOL, mean_err, cov_err, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,nx,T", [("fp64", 4, 5000), ("fp32", 4, 100000), ("fp32", 8, 3000),
                                            ("fp32_fp64solve", 2, 777)])
def test_noalloc_matches_rts_smooth_twice(precision, nx, T):
    import torch
    import paper_2511_10363_gb300 as kf
    from paper_2511_10363_gb300 import build
    build.build()
    model = W.cv_model() if nx == 4 else (W.random_stable_model(8, 4, seed=3) if nx == 8 else W.cv1d_model())
    dt = kf.dtype_of(precision)
    y = torch.tensor(W.simulate(model, T, seed=T), dtype=dt, device="cuda")
    # the reference runs the same per-step kernels as the no-allocation entry
    # point (which has no device table cache for the covariance tables)
    kf.kf_set_option("covariance_tables", 1)
    try:
        ref_m, ref_P, ref_ll = kf.kf_rts_smooth(model, y, precision, "dlb", loglik=True)
    finally:
        kf.kf_set_option("covariance_tables", 0)
    assert kf.kf_sync_status() == 0
    ref_m, ref_P, ref_ll = ref_m.double().cpu().numpy(), ref_P.double().cpu().numpy(), float(ref_ll.item())
    for _ in range(2):
        ms = torch.full((T, nx), float("nan"), dtype=dt, device="cuda")
        Ps = torch.full((T, nx, nx), float("nan"), dtype=dt, device="cuda")
        ll = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.full((1,), 77, dtype=torch.int32, device="cuda")
        kf.kf_rts_smooth_noalloc(model, y, precision, ms, Ps, loglik=ll, status_out=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        m, P = ms.double().cpu().numpy(), Ps.double().cpu().numpy()
        assert mean_err(m, ref_m, ref_P) <= TOL[precision]
        assert cov_err(P, ref_P) <= TOL[precision]
        tol_ll = 1e-9 if precision == "fp64" else 1e-3
        assert abs(float(ll.item()) - ref_ll) <= tol_ll * max(1.0, abs(ref_ll))


def test_noalloc_rejects_requests_beyond_its_scratch():
    import torch
    import paper_2511_10363_gb300 as kf
    model = W.cv_model()
    T = 1 << 20                      # needs ~64 MB of filter records: beyond the 16 MB array
    y = torch.zeros((T, 2), dtype=torch.float32, device="cuda")
    ms = torch.empty((T, 4), device="cuda")
    Ps = torch.empty((T, 4, 4), device="cuda")
    with pytest.raises(kf.KfError) as e:
        kf.kf_rts_smooth_noalloc(model, y, "fp32", ms, Ps)
    assert e.value.status == 8       # KF_ERR_CAPACITY
    assert kf.kf_workspace_size("rts", 4, 2, T, "fp32", "dlb") + 256 > kf.NOALLOC_SCRATCH_BYTES


def test_noalloc_matches_the_oracle():
    """Against the FP64 oracle directly (not only against kf_rts_smooth), so a
    mistake shared by both entry points cannot pass."""
    import torch
    import paper_2511_10363_gb300 as kf
    model = W.cv_model()
    T = 4097
    y = W.simulate(model, T, seed=21)
    ref = oracle_run(model, y)
    yt = torch.tensor(y, dtype=torch.float64, device="cuda")
    for _ in range(2):
        ms = torch.full((T, 4), float("nan"), dtype=torch.float64, device="cuda")
        Ps = torch.full((T, 4, 4), float("nan"), dtype=torch.float64, device="cuda")
        ll = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = torch.full((1,), 77, dtype=torch.int32, device="cuda")
        kf.kf_rts_smooth_noalloc(model, yt, "fp64", ms, Ps, loglik=ll, status_out=st)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert mean_err(ms.cpu().numpy(), ref["ms_rts"], ref["Ps_rts"]) <= 1e-9
        assert cov_err(Ps.cpu().numpy(), ref["Ps_rts"]) <= 1e-9
        assert abs(float(ll.item()) - ref["ll"]) <= 1e-9 * abs(ref["ll"])


@pytest.mark.parametrize("with_status_out", [True, False])
def test_noalloc_reports_a_wait_time_out(with_status_out):
    """A tile that never publishes (test hook) makes the later tiles' bounded
    waits run out.  The time-out reaches the caller's status word, or,
    without one, kf_sync_status; the next call is correct."""
    import torch
    import paper_2511_10363_gb300 as kf
    model = W.cv_model()
    T = 20000
    y = W.simulate(model, T, seed=9)
    yt = torch.tensor(y, dtype=torch.float32, device="cuda")
    ms = torch.empty((T, 4), dtype=torch.float32, device="cuda")
    Ps = torch.empty((T, 4, 4), dtype=torch.float32, device="cuda")
    st = torch.full((1,), 77, dtype=torch.int32, device="cuda") if with_status_out else None
    assert kf.kf_sync_status() == 0
    kf.kf_set_option("wait_timeout_ns", 50_000_000)
    kf.kf_set_option("positions_per_thread", 2)
    kf.kf_set_option("test_skip_tile", 3)
    try:
        kf.kf_rts_smooth_noalloc(model, yt, "fp32", ms, Ps, status_out=st)
        torch.cuda.synchronize()
    finally:
        kf.kf_set_option("test_skip_tile", -1)
        kf.kf_set_option("positions_per_thread", 0)
        kf.kf_set_option("wait_timeout_ns", 10 ** 9)
    if with_status_out:
        assert int(st.item()) == 5               # KF_ERR_TIMEOUT
        assert kf.kf_sync_status() == 0         # the library's word was not touched
    else:
        assert kf.kf_sync_status() == 5
        assert kf.kf_sync_status() == 0         # read and cleared
    ref = oracle_run(model, np.asarray(y, np.float32).astype(np.float64))
    st2 = torch.full((1,), 77, dtype=torch.int32, device="cuda")
    kf.kf_rts_smooth_noalloc(model, yt, "fp32", ms, Ps, status_out=st2)
    torch.cuda.synchronize()
    assert int(st2.item()) == 0
    assert mean_err(ms.double().cpu().numpy(), ref["ms_rts"], ref["Ps_rts"]) <= TOL["fp32"]
    assert cov_err(Ps.double().cpu().numpy(), ref["Ps_rts"]) <= TOL["fp32"]
