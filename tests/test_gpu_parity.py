"""GPU parity: every scan variant x precision x state size x length against
the FP64 oracle on the same seeded inputs, through the C ABI.

Lengths cover T = 1, a single partial tile, several tiles with a ragged
tail, and powers of two (the level algorithms pad to the next power of
two).  For the decoupled look-back scan the number of time steps per thread
is also forced to small values so that small T spans many tiles."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import TOL, gpu_run, oracle_inputs, oracle_run, mean_err, cov_err, check_psd

pytestmark = pytest.mark.gpu

SCANS = ["dlb", "hillis_steele", "blelloch", "ladner_fischer", "sengupta"]
PRECS = ["fp64", "fp32", "fp32_fp64solve"]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2511_10363_gb300 import build
    build.build()
    import paper_2511_10363_gb300 as kf
    kf.kf_set_option("positions_per_thread", 0)
    yield
    kf.kf_set_option("positions_per_thread", 0)


def model_for(nx, seed):
    if nx == 4:
        return W.cv_model()
    if nx == 2:
        return W.random_model(2, 1, seed=seed)
    return W.random_stable_model(8, 4, seed=seed)


def compare(op, model, y, precision, scan, loglik=True):
    yo = oracle_inputs(y, precision)
    ref = oracle_run(model, yo)
    out = gpu_run(op, model, yo, precision, scan, loglik=loglik, want_filter=(op != "filter"))
    tol = TOL[precision]
    errs = {"mf": mean_err(out["mf"], ref["mf"], ref["Pf"]), "Pf": cov_err(out["Pf"], ref["Pf"])}
    if op != "filter":
        key = "rts" if op == "rts" else "tf"
        errs["ms"] = mean_err(out["ms"], ref["ms_" + key], ref["Ps_" + key])
        errs["Ps"] = cov_err(out["Ps"], ref["Ps_" + key])
        check_psd(out["Ps"])
    check_psd(out["Pf"])
    for k, v in errs.items():
        assert v <= tol, "%s %s %s: %s error %.3g > %.3g" % (op, precision, scan, k, v, tol)
    if loglik:
        ll_tol = 1e-9 if precision == "fp64" else 1e-3
        assert abs(out["ll"] - ref["ll"]) <= ll_tol * max(1.0, abs(ref["ll"])), (out["ll"], ref["ll"])
    return errs


@pytest.mark.parametrize("tables", [0, 1])
@pytest.mark.parametrize("op", ["filter", "rts", "tf"])
@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("nx", [2, 4, 8])
@pytest.mark.parametrize("T", [1, 2, 3, 100, 1000, 4097])
def test_dlb_parity(op, precision, nx, T, tables):
    """tables = 0: the covariance-table path where it applies (the filter at
    any T, the RTS smoother from T = k0 + kb + 1 on); 1: the per-step kernels."""
    import paper_2511_10363_gb300 as kf
    model = model_for(nx, seed=nx * 7 + T % 5)
    y = W.simulate(model, T, seed=1000 + T)
    kf.kf_set_option("covariance_tables", tables)
    try:
        compare(op, model, y, precision, "dlb")
    finally:
        kf.kf_set_option("covariance_tables", 0)


@pytest.mark.parametrize("op", ["filter", "rts", "tf"])
@pytest.mark.parametrize("scan", SCANS[1:])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("T", [1, 2, 5, 64, 333])
def test_level_scan_parity(op, scan, precision, T):
    model = W.cv_model()
    y = W.simulate(model, T, seed=2000 + T)
    compare(op, model, y, precision, scan)


@pytest.mark.parametrize("N", [2, 16, 1 << 20])
@pytest.mark.parametrize("T", [5, 64, 333])
def test_sengupta_threshold(N, T):
    """Alg. sengupta with a Hillis-Steele top level of length N ("Sengupta
    B"; N beyond the padded length makes it Hillis-Steele outright)."""
    import paper_2511_10363_gb300 as kf
    model = W.cv_model()
    y = W.simulate(model, T, seed=900 + T)
    kf.kf_set_option("sengupta_n", N)
    try:
        for op in ("filter", "rts", "tf"):
            compare(op, model, y, "fp64", "sengupta")
        compare("rts", model, y, "fp32", "sengupta")
    finally:
        kf.kf_set_option("sengupta_n", 1)


@pytest.mark.parametrize("tables", [0, 1])
@pytest.mark.parametrize("K", [1, 2, 3, 7])
@pytest.mark.parametrize("op", ["filter", "rts", "tf"])
def test_dlb_many_tiles(K, op, tables):
    """Force K time steps per thread so that T = 5000 spans many tiles, and
    the look-back combines many predecessor aggregates."""
    import paper_2511_10363_gb300 as kf
    model = W.cv_model()
    y = W.simulate(model, 5000, seed=3000 + K)
    kf.kf_set_option("positions_per_thread", K)
    kf.kf_set_option("covariance_tables", tables)
    try:
        compare(op, model, y, "fp64", "dlb")
        compare(op, model, y, "fp32", "dlb")
    finally:
        kf.kf_set_option("positions_per_thread", 0)
        kf.kf_set_option("covariance_tables", 0)


@pytest.mark.parametrize("nx,ny", [(2, 2), (4, 1), (4, 3), (8, 2), (8, 8), (2, 5)])
def test_measurement_sizes(nx, ny):
    model = W.random_model(nx, ny, seed=nx * 10 + ny)
    y = W.simulate(model, 777, seed=nx + ny)
    for op in ("filter", "rts", "tf"):
        compare(op, model, y, "fp64", "dlb")


def test_rts_equals_two_filter_on_gpu():
    model = W.cv_model()
    y = W.simulate(model, 3000, seed=5)
    a = gpu_run("rts", model, y, "fp64", "dlb")
    b = gpu_run("tf", model, y, "fp64", "dlb")
    assert mean_err(a["ms"], b["ms"], b["Ps"]) < 1e-10 and cov_err(a["Ps"], b["Ps"]) < 1e-10


def test_deterministic_loglik():
    model = W.cv_model()
    y = W.simulate(model, 50000, seed=6)
    l1 = gpu_run("filter", model, y, "fp64", "dlb", loglik=True)["ll"]
    l2 = gpu_run("filter", model, y, "fp64", "dlb", loglik=True)["ll"]
    assert l1 == l2


@pytest.mark.parametrize("general", [0, 1])
@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("nx", [2, 4, 8])
def test_filter_solve_forms(general, precision, nx):
    """With ny = nx / 2 the filter scan uses the rank-ny (Woodbury) form of a
    fresh element's J unless the general pivoted inverse is forced; both
    must match the oracle, the log-likelihood included."""
    import paper_2511_10363_gb300 as kf
    model = model_for(nx, seed=41 + nx)
    y = W.simulate(model, 3000, seed=42 + nx)
    kf.kf_set_option("general_solve", general)
    try:
        for op in ("filter", "rts", "tf"):
            compare(op, model, y, precision, "dlb")
    finally:
        kf.kf_set_option("general_solve", 0)


@pytest.mark.parametrize("threads", [128, 256])
@pytest.mark.parametrize("K", [2, 3, 16, 49, 50, 129, 130, 200])
@pytest.mark.parametrize("model_kind", ["cv", "random4", "random2"])
def test_fold_table(K, model_kind, threads):
    """With ny = nx / 2 and one sequence, the thread fold of the filter scan
    reads the (A, C, J) half of its aggregate from a table built per launch
    for K positions per thread (K up to 129 in FP32 for nx = 4, 49 in FP64;
    beyond that the per-step solve is used); the tiles whose threads all use the
    fold table also run their tile scan on (b, eta) with the tile-scan
    table.  Forced K across the table limits, a ragged last thread, many
    tiles, 128- and 256-thread CTAs (256 exists for nx = 4 in FP32)."""
    import paper_2511_10363_gb300 as kf
    model = {"cv": W.cv_model(), "random4": W.random_stable_model(4, 2, seed=K),
             "random2": W.random_model(2, 1, seed=K)}[model_kind]
    T = K * threads * 5 + 77
    y = W.simulate(model, T, seed=500 + K)
    kf.kf_set_option("positions_per_thread", K)
    kf.kf_set_option("threads", threads)
    kf.kf_set_option("covariance_tables", 1)   # the per-step kernels
    try:
        # the log-likelihood in FP64 only: in the working precision FP32 the
        # innovation of a long tracking sequence (positions ~1e7) cancels
        for precision in PRECS:
            compare("filter", model, y, precision, "dlb", loglik=(precision == "fp64"))
        compare("rts", model, y, "fp32", "dlb", loglik=False)
    finally:
        kf.kf_set_option("positions_per_thread", 0)
        kf.kf_set_option("threads", 0)
        kf.kf_set_option("covariance_tables", 0)
