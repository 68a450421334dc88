"""Full-size parity: the benchmark's workload (2D constant-velocity tracking,
T = 2^20) in the launch configuration bench.py times (explicit workspace,
default tile plan, decoupled look-back scan), compared with the FP64 oracle
on every output of every step; also T = 2^22, the largest length of the
sweep.  The sequential C oracle handles these lengths in seconds."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import TOL, mean_err, cov_err, oracle_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,T,tables", [("fp32", 1 << 20, 0), ("fp64", 1 << 20, 0), ("fp32", 1 << 22, 0),
                                                ("fp32", 1 << 20, 1), ("fp64", 1 << 20, 1)])
def test_bench_workload_full_size(precision, T, tables):
    """tables = 0: the default path (covariance tables for the RTS smoother,
    per-step kernels for the two-filter smoother); 1: per-step kernels only."""
    import torch
    import paper_2511_10363_gb300 as kf
    from paper_2511_10363_gb300 import build
    build.build()
    kf.kf_set_option("covariance_tables", tables)
    try:
        _full_size(kf, torch, precision, T)
    finally:
        kf.kf_set_option("covariance_tables", 0)


def _full_size(kf, torch, precision, T):
    model = W.cv_model()
    y = oracle_inputs(W.simulate(model, T, seed=1), precision)
    mf, Pf, ll = oracle.kf(model, y)
    ms, Ps = oracle.rts(model, mf, Pf)
    ms2, Ps2 = oracle.tf(model, y, mf, Pf)
    dt = kf.dtype_of(precision)
    yt = torch.tensor(y, dtype=dt, device="cuda")
    mdl = kf.Model(model)
    for op, rm, rP in (("rts", ms, Ps), ("tf", ms2, Ps2)):
        ws = torch.empty(kf.kf_workspace_size(op, 4, 2, T, precision, "dlb"), dtype=torch.uint8, device="cuda")
        m_out = torch.empty((T, 4), dtype=dt, device="cuda")
        P_out = torch.empty((T, 4, 4), dtype=dt, device="cuda")
        mf_out = torch.empty((T, 4), dtype=dt, device="cuda")
        Pf_out = torch.empty((T, 4, 4), dtype=dt, device="cuda")
        fn = kf.kf_rts_smooth if op == "rts" else kf.kf_two_filter_smooth
        _, _, gll = fn(mdl, yt, precision, "dlb", ms_out=m_out, Ps_out=P_out, mf_out=mf_out, Pf_out=Pf_out,
                       loglik=True, workspace=ws)
        assert kf.kf_sync_status() == 0
        gm, gP = m_out.double().cpu().numpy(), P_out.double().cpu().numpy()
        gmf, gPf = mf_out.double().cpu().numpy(), Pf_out.double().cpu().numpy()
        tol = TOL[precision]
        assert mean_err(gmf, mf, Pf) <= tol and cov_err(gPf, Pf) <= tol
        assert mean_err(gm, rm, rP) <= tol and cov_err(gP, rP) <= tol
        # covariance invariants over every step: symmetric, positive definite
        assert np.array_equal(gP, np.swapaxes(gP, 1, 2))
        assert np.all(np.linalg.eigvalsh(gP) > 0)
        if precision == "fp64":
            assert abs(gll.item() - ll) <= 1e-9 * abs(ll)
        del ws
