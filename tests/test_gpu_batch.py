"""GPU parity of the segmented (batched) scan: many independent sequences of
uneven length concatenated in one buffer and scanned by one kernel per
pass.  Each sequence is checked against the oracle run on that sequence
alone, and against the single-sequence entry point ("alone and in the
mix")."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import TOL, mean_err, cov_err, oracle_inputs, check_psd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2511_10363_gb300 import build
    build.build()


def run_batch(op, models, model_of, lengths, y, precision):
    import torch
    import paper_2511_10363_gb300 as kf
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    yt = torch.tensor(y, dtype=kf.dtype_of(precision), device="cuda")
    m, P, ll = kf.kf_batch_smooth(op, models, offs, yt, precision, model_of=model_of, loglik=True)
    assert kf.kf_sync_status() == 0
    return offs, m.double().cpu().numpy(), P.double().cpu().numpy(), ll.cpu().numpy()


def check_against_oracle(op, models, model_of, lengths, y, precision):
    yo = oracle_inputs(y, precision)
    offs, m, P, ll = run_batch(op, models, model_of, lengths, yo, precision)
    tol = TOL[precision]
    for s in range(len(lengths)):
        a, b = offs[s], offs[s + 1]
        if b == a:
            assert ll[s] == 0.0
            continue
        mdl = models[model_of[s]] if model_of is not None else models[0]
        mf, Pf, lref = oracle.kf(mdl, yo[a:b])
        if op == "filter":
            rm, rP = mf, Pf
        elif op == "rts":
            rm, rP = oracle.rts(mdl, mf, Pf)
        else:
            rm, rP = oracle.tf(mdl, yo[a:b], mf, Pf)
        assert mean_err(m[a:b], rm, rP) <= tol, (op, precision, s)
        assert cov_err(P[a:b], rP) <= tol, (op, precision, s)
        check_psd(P[a:b])
        ll_tol = 1e-9 if precision == "fp64" else 1e-3
        assert abs(ll[s] - lref) <= ll_tol * max(1.0, abs(lref)), (s, ll[s], lref)


@pytest.mark.parametrize("op", ["filter", "rts", "tf"])
@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_fp64solve"])
def test_ragged_batch_one_model(op, precision):
    rng = np.random.default_rng(5)
    lengths = np.concatenate([[1, 2, 0, 3, 1], rng.integers(1, 3000, size=40), [0]])
    model = W.cv_model()
    y, _ = W.ragged_batch(model, lengths, seed=7)
    check_against_oracle(op, [model], None, lengths, y, precision)


@pytest.mark.parametrize("op", ["filter", "rts", "tf"])
@pytest.mark.parametrize("nx", [2, 4, 8])
def test_batch_many_models(op, nx):
    ny = max(1, nx // 2)
    models = [W.random_model(nx, ny, seed=100 + i) for i in range(5)]
    rng = np.random.default_rng(nx)
    lengths = rng.integers(1, 800, size=23)
    model_of = rng.integers(0, len(models), size=len(lengths)).astype(np.int32)
    ys = [W.simulate(models[model_of[s]], int(lengths[s]), seed=1000 + s) for s in range(len(lengths))]
    y = np.concatenate(ys)
    check_against_oracle(op, models, model_of, lengths, y, "fp64")


@pytest.mark.parametrize("K", [1, 3])
def test_batch_many_tiles(K):
    import paper_2511_10363_gb300 as kf
    rng = np.random.default_rng(11)
    lengths = rng.integers(1, 400, size=60)
    model = W.cv_model()
    y, _ = W.ragged_batch(model, lengths, seed=12)
    kf.kf_set_option("positions_per_thread", K)
    try:
        for op in ("filter", "rts", "tf"):
            check_against_oracle(op, [model], None, lengths, y, "fp64")
    finally:
        kf.kf_set_option("positions_per_thread", 0)


@pytest.mark.parametrize("op", ["rts", "tf"])
def test_alone_and_in_the_mix(op):
    """Each sequence's result is the same alone (single-sequence call) and
    inside a batch, within the FP32 tolerance."""
    import torch
    import paper_2511_10363_gb300 as kf
    rng = np.random.default_rng(21)
    lengths = rng.integers(100, 5000, size=12)
    model = W.cv_model()
    y, offs = W.ragged_batch(model, lengths, seed=22)
    y = y.astype(np.float32).astype(np.float64)
    _, m, P, ll = run_batch(op, [model], None, lengths, y, "fp32")
    fn = kf.kf_rts_smooth if op == "rts" else kf.kf_two_filter_smooth
    for s in range(len(lengths)):
        a, b = offs[s], offs[s + 1]
        yt = torch.tensor(y[a:b], dtype=torch.float32, device="cuda")
        sm, sP, sll = fn(model, yt, "fp32", "dlb", loglik=True)
        sm, sP = sm.double().cpu().numpy(), sP.double().cpu().numpy()
        assert mean_err(m[a:b], sm, sP) <= TOL["fp32"]
        assert cov_err(P[a:b], sP) <= TOL["fp32"]
        assert abs(ll[s] - sll.item()) <= 1e-3 * max(1.0, abs(sll.item()))


def test_batch_argument_errors():
    import torch
    import paper_2511_10363_gb300 as kf
    model = W.cv_model()
    y = torch.zeros((10, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(kf.KfError):
        kf.kf_batch_smooth("rts", model, [0, 5, 3, 10], y, "fp32")       # decreasing offsets
    with pytest.raises(kf.KfError):
        kf.kf_batch_smooth("rts", model, [1, 10], y, "fp32")             # offsets[0] != 0
    with pytest.raises(kf.KfError):
        kf.kf_batch_smooth("rts", model, [0, 4, 10], y, "fp32", model_of=[0, 3])   # bad model index


@pytest.mark.parametrize("op", ["filter", "rts", "tf"])
def test_batch_graph(op):
    """The batched call captured in a CUDA graph gives the same results as
    kf_batch_smooth, also after new measurements are written into y."""
    import torch
    import paper_2511_10363_gb300 as kf
    rng = np.random.default_rng(31)
    lengths = np.concatenate([[5, 0, 1], rng.integers(50, 3000, size=20)])
    model = W.cv_model()
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    y1, _ = W.ragged_batch(model, lengths, seed=32)
    y2, _ = W.ragged_batch(model, lengths, seed=33)
    yt = torch.tensor(y1, dtype=torch.float32, device="cuda")
    g = kf.BatchGraph(op, model, offs, yt, "fp32", loglik=True)
    try:
        for ynew in (y1, y2, y1):
            yt.copy_(torch.tensor(ynew, dtype=torch.float32))
            m, P, ll = g.launch()
            torch.cuda.synchronize()
            assert kf.kf_sync_status() == 0
            rm, rP, rll = kf.kf_batch_smooth(op, model, offs, yt, "fp32", loglik=True)
            torch.cuda.synchronize()
            # the look-back may combine in a different order from run to run
            # (whichever predecessor has published first): equal up to FP32 rounding
            rm_, rP_ = rm.double().cpu().numpy(), rP.double().cpu().numpy()
            assert mean_err(m.double().cpu().numpy(), rm_, rP_) <= TOL["fp32"]
            assert cov_err(P.double().cpu().numpy(), rP_) <= TOL["fp32"]
            assert np.allclose(ll.cpu().numpy(), rll.cpu().numpy(), rtol=1e-5, atol=1e-3)
        # and against the oracle on the last data
        check_against_oracle(op, [model], None, lengths, y1, "fp32")
    finally:
        g.close()
