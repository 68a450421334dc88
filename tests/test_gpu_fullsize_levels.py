"""Full-size parity of the level-by-level scans (Algs. 1-3 and Alg. sengupta)
and of the mixed-precision mode, against the FP64 oracle on every step.

The level algorithms run one launch per level with grid-stride loops over
the level's operator applications on a power-of-two padded length; at
T = 2^20 every level launch covers the whole device many times over, and
the padding to the next power of two is exercised by T = 2^20 + 333.  The
precision case is the random stable model of the precision benchmark
(nx = 8, ny = 4, T = 2^18) in FP32 with FP64 (I + C J) solves.

Means are gated normwise per step, |dm_k| / max(|m_k|, sqrt tr P_k); the
error in posterior standard deviations, |dm_k| / sqrt tr P_k, is reported
beside it in the assertion messages and gated where the working precision
can represent the means to a fraction of a standard deviation."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import TOL, gpu_run, oracle_inputs, mean_err, cov_err, check_psd

pytestmark = pytest.mark.gpu

_REF = {}


def model_for(nx):
    if nx == 4:
        return W.cv_model()
    if nx == 2:
        return W.random_model(2, 1, seed=12)
    return W.random_stable_model(8, 4, seed=3)


def std_err(m, mref, Pref):
    """max_k |dm_k| / sqrt(tr P_k): the mean error in posterior standard deviations."""
    return float(np.max(np.linalg.norm(m - mref, axis=1) / np.sqrt(np.trace(Pref, axis1=1, axis2=2))))


def reference(nx, T, precision, seed):
    key = (nx, T, precision != "fp64", seed)
    if key not in _REF:
        model = model_for(nx)
        y = oracle_inputs(W.simulate(model, T, seed=seed), precision)
        mf, Pf, ll = oracle.kf(model, y)
        ms, Ps = oracle.rts(model, mf, Pf)
        ms2, Ps2 = oracle.tf(model, y, mf, Pf)
        _REF.clear()   # one reference at a time: these are hundreds of MB
        _REF[key] = dict(model=model, y=y, mf=mf, Pf=Pf, ll=ll, ms_rts=ms, Ps_rts=Ps, ms_tf=ms2, Ps_tf=Ps2)
    return _REF[key]


def check(op, nx, T, precision, scan, seed=1, loglik=None):
    ref = reference(nx, T, precision, seed)
    if loglik is None:
        loglik = precision == "fp64"
    out = gpu_run(op, ref["model"], ref["y"], precision, scan, loglik=loglik, want_filter=(op != "filter"))
    tol = TOL[precision]
    key = "rts" if op == "rts" else "tf"
    pairs = [("mf", "Pf", ref["mf"], ref["Pf"])]
    if op != "filter":
        pairs.append(("ms", "Ps", ref["ms_" + key], ref["Ps_" + key]))
    for mk, Pk, mref, Pref in pairs:
        e_m, e_s, e_P = mean_err(out[mk], mref, Pref), std_err(out[mk], mref, Pref), cov_err(out[Pk], Pref)
        msg = "%s %s %s nx=%d T=%d %s: normwise %.3g, posterior-std units %.3g, cov %.3g" % (
            op, scan, precision, nx, T, mk, e_m, e_s, e_P)
        assert e_m <= tol and e_P <= tol, msg
        if precision == "fp64":
            assert e_s <= 1e-6, msg
        check_psd(out[Pk])
    if loglik:
        ll_tol = 1e-9 if precision == "fp64" else 1e-4
        assert abs(out["ll"] - ref["ll"]) <= ll_tol * abs(ref["ll"]), (out["ll"], ref["ll"])


LEVEL_SCANS = ["hillis_steele", "blelloch", "ladner_fischer", "sengupta"]


@pytest.mark.parametrize("scan", LEVEL_SCANS)
@pytest.mark.parametrize("precision,nx", [("fp32", 2), ("fp32", 4), ("fp32", 8),
                                          ("fp64", 2), ("fp64", 4), ("fp64", 8), ("fp32_fp64solve", 4)])
def test_level_scans_full_size(scan, precision, nx):
    """T = 2^20, RTS smoother (forward filter scan + reverse RTS scan)."""
    from paper_2511_10363_gb300 import build
    build.build()
    check("rts", nx, 1 << 20, precision, scan)


@pytest.mark.parametrize("scan", LEVEL_SCANS)
def test_level_scans_full_size_two_filter_ragged(scan):
    """T = 2^20 + 333 (padded to 2^21): two-filter smoother in FP64, FP32."""
    check("tf", 4, (1 << 20) + 333, "fp64", scan, seed=2)
    check("tf", 4, (1 << 20) + 333, "fp32", scan, seed=2)


def test_sengupta_b_full_size():
    """Alg. sengupta with the Hillis-Steele top level of N = 16384 ("Sengupta
    B", the sweep's configuration) at T = 2^20."""
    import paper_2511_10363_gb300 as kf
    kf.kf_set_option("sengupta_n", 16384)
    try:
        check("rts", 4, 1 << 20, "fp32", "sengupta")
        check("rts", 4, 1 << 20, "fp64", "sengupta")
    finally:
        kf.kf_set_option("sengupta_n", 1)


@pytest.mark.parametrize("op", ["filter", "rts", "tf"])
def test_mixed_precision_config_against_oracle(op):
    """The precision workload: random stable model nx = 8, ny = 4, T = 2^18,
    FP32 element build and combines with the (I + C J) solves in FP64 and one
    refinement step (Lemma 1), every output and the log-likelihood against
    the FP64 oracle on the same FP32-rounded inputs, within 1e-4."""
    check(op, 8, 1 << 18, "fp32_fp64solve", "dlb", loglik=True)
