"""Pins of the time-varying FP64 oracle (the general model of Sec. III-A
with per-step F_{k-1}, Q_{k-1}, u_{k-1}, H_k, R_k, d_k) against facts
that do not come from the oracle:

* a dense joint-Gaussian brute force of the whole posterior, with every
  matrix and both input sequences different at every step, so that a
  record read one step early or late, or an input with the wrong sign,
  changes the answer;
* constant per-step arrays without inputs reduce to the time-invariant
  oracle (itself pinned by test_oracle_pins.py);
* a measurement offset d_k is the same as subtracting it from y_k;
* the elements of Eqs. pkf_init1..3 and prts_init1/2 with inputs: their
  sequential Lemma 1 / Lemma 2 folds give the sequential recursions, and
  the reverse fold of (a_2, ..., a_T, e) gives the backward information
  filter (Alg. ptf).
A stored fixture (tests/golden/oracle_tv_T48.npz, written by
tests/golden/make_golden.py from the oracle alone) catches accidental
changes.
"""
import numpy as np
import pytest

import oracle
from oracle import scans
from tests import bruteforce
import workloads as W


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def random_tv_model(nx, ny, T, seed, inputs=True):
    """Every per-step matrix random (F from a scaled QR factor, Q and R as
    X X^T plus a floor), random m0, P0 and inputs."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((T, nx, nx))
    Qf, Rf = np.linalg.qr(X)
    F = 0.97 * Qf * np.sign(np.diagonal(Rf, axis1=1, axis2=2))[:, None, :]
    Xq = rng.standard_normal((T, nx, nx)) / np.sqrt(nx)
    Xr = rng.standard_normal((T, ny, ny)) / np.sqrt(ny)
    Q = Xq @ np.transpose(Xq, (0, 2, 1)) + 0.05 * np.eye(nx)
    R = Xr @ np.transpose(Xr, (0, 2, 1)) + 0.05 * np.eye(ny)
    H = rng.standard_normal((T, ny, nx))
    Xp = rng.standard_normal((nx, nx)) / np.sqrt(nx)
    return dict(F=F, Q=Q, H=H, R=R,
                u=rng.standard_normal((T, nx)) if inputs else None,
                d=rng.standard_normal((T, ny)) if inputs else None,
                m0=rng.standard_normal(nx), P0=Xp @ Xp.T + 0.05 * np.eye(nx))


@pytest.mark.parametrize("nx,ny,T,seed,inputs", [(2, 1, 15, 1, True), (4, 2, 30, 2, True), (4, 2, 20, 3, False),
                                                 (8, 4, 16, 4, True), (3, 5, 10, 5, True)])
def test_tv_oracle_vs_dense_joint_gaussian(nx, ny, T, seed, inputs):
    model = random_tv_model(nx, ny, T, seed, inputs)
    y = W.simulate_tv(model, seed=100 + seed)
    mf, Pf, ll = oracle.tv_kf(model, y)
    bm, bP = bruteforce.tv_filtering(model, y)
    assert rel(mf, bm) < 1e-9 and rel(Pf, bP) < 1e-9
    sm, sP, bll = bruteforce.tv_posterior(model, y)
    assert abs(ll - bll) < 1e-9 * max(1.0, abs(bll))
    ms, Ps = oracle.tv_rts(model, mf, Pf)
    assert rel(ms, sm) < 1e-9 and rel(Ps, sP) < 1e-9
    ms2, Ps2 = oracle.tv_tf(model, y, mf, Pf)
    assert rel(ms2, sm) < 1e-9 and rel(Ps2, sP) < 1e-9


def test_tv_dense_cv_tracking_workload():
    """The seeded time-varying tracking model of the GPU tests (nx = 4)."""
    model = W.tv_model(4, 40, seed=9)
    y = W.simulate_tv(model, seed=10)
    mf, Pf, ll = oracle.tv_kf(model, y)
    bm, bP = bruteforce.tv_filtering(model, y)
    assert rel(mf, bm) < 1e-9 and rel(Pf, bP) < 1e-9
    sm, sP, bll = bruteforce.tv_posterior(model, y)
    ms, Ps = oracle.tv_rts(model, mf, Pf)
    assert rel(ms, sm) < 1e-9 and rel(Ps, sP) < 1e-9
    assert abs(ll - bll) < 1e-9 * abs(bll)


@pytest.mark.parametrize("nx,ny", [(2, 1), (4, 2), (8, 4)])
def test_tv_constant_model_is_time_invariant(nx, ny):
    base = W.random_model(nx, ny, seed=20 + nx)
    T = 200
    tv = dict(F=np.broadcast_to(base["F"], (T, nx, nx)), Q=np.broadcast_to(base["Q"], (T, nx, nx)),
              H=np.broadcast_to(base["H"], (T, ny, nx)), R=np.broadcast_to(base["R"], (T, ny, ny)),
              u=None, d=None, m0=base["m0"], P0=base["P0"])
    y = W.simulate(base, T, seed=7)
    mf, Pf, ll = oracle.kf(base, y)
    tmf, tPf, tll = oracle.tv_kf(tv, y)
    assert rel(tmf, mf) < 1e-13 and rel(tPf, Pf) < 1e-13 and abs(tll - ll) < 1e-12 * abs(ll)
    ms, Ps = oracle.rts(base, mf, Pf)
    tms, tPs = oracle.tv_rts(tv, tmf, tPf)
    assert rel(tms, ms) < 1e-13 and rel(tPs, Ps) < 1e-13
    ms2, Ps2 = oracle.tf(base, y, mf, Pf)
    tms2, tPs2 = oracle.tv_tf(tv, y, tmf, tPf)
    assert rel(tms2, ms2) < 1e-13 and rel(tPs2, Ps2) < 1e-13


def test_tv_measurement_offset_is_a_data_shift():
    model = random_tv_model(4, 2, 50, seed=31)
    y = W.simulate_tv(model, seed=32)
    plain = dict(model, d=None)
    for kind in ("rts", "tf"):
        a = oracle.tv_smooth(model, y, kind)
        b = oracle.tv_smooth(plain, y - model["d"], kind)
        for x, z in zip(a[:4], b[:4]):
            assert rel(x, z) < 1e-12
        assert abs(a[4] - b[4]) < 1e-10 * abs(b[4])


def tv_elements(model, y):
    return [oracle.tv_filter_element(model, k + 1, y[k]) for k in range(len(y))]


@pytest.mark.parametrize("nx,ny,seed", [(2, 1, 41), (4, 2, 42), (8, 4, 43)])
def test_tv_filter_fold_equals_kalman_filter(nx, ny, seed):
    """Alg. pkf with the elements of Eqs. pkf_init1..3 including u and d."""
    T = 40
    model = random_tv_model(nx, ny, T, seed)
    y = W.simulate_tv(model, seed=seed)
    mf, Pf, _ = oracle.tv_kf(model, y)
    pref, _ = scans.sequential(tv_elements(model, y), oracle.filter_combine)
    for k in range(T):
        assert rel(pref[k].b, mf[k]) < 1e-10 and rel(pref[k].C, Pf[k]) < 1e-10


@pytest.mark.parametrize("nx,ny,seed", [(2, 1, 51), (4, 2, 52), (8, 4, 53)])
def test_tv_rts_reverse_fold_equals_rts(nx, ny, seed):
    """Alg. prts with the elements of Eqs. prts_init1/2 including u."""
    T = 40
    model = random_tv_model(nx, ny, T, seed)
    y = W.simulate_tv(model, seed=seed)
    mf, Pf, _ = oracle.tv_kf(model, y)
    ms, Ps = oracle.tv_rts(model, mf, Pf)
    els = [oracle.tv_rts_element(model, k + 1, T, mf[k], Pf[k]) for k in range(T)]
    suf, _ = scans.reverse_sequential(els, oracle.rts_combine)
    for k in range(T):
        assert rel(suf[k].g, ms[k]) < 1e-10 and rel(suf[k].L, Ps[k]) < 1e-10


def test_tv_two_filter_reverse_fold_gives_backward_filter():
    """Alg. ptf: the reverse fold of (a_2, ..., a_T, e) of the time-varying
    elements gives eta_{k|k+1:T}, J_{k|k+1:T} of the backward filter."""
    T = 30
    model = random_tv_model(4, 2, T, seed=61)
    y = W.simulate_tv(model, seed=62)
    mf, Pf, _ = oracle.tv_kf(model, y)
    _, _, eta, J = oracle.tv_tf(model, y, mf, Pf, want_info=True)
    seq = tv_elements(model, y)[1:] + [oracle.FilterElem.identity(4)]
    suf, _ = scans.reverse_sequential(seq, oracle.filter_combine)
    for k in range(T - 1):
        assert rel(suf[k].eta, eta[k]) < 1e-10 and rel(suf[k].J, J[k]) < 1e-10
    assert np.all(suf[T - 1].eta == 0) and np.all(suf[T - 1].J == 0)


def test_tv_oracle_regression_fixture():
    """The stored outputs of tests/golden/make_golden.py for a time-varying
    model (written by calling only the oracle) still match."""
    import os
    g = np.load(os.path.join(os.path.dirname(__file__), "golden", "oracle_tv_T48.npz"))
    model = {k: g[k] for k in ("F", "Q", "u", "H", "R", "d", "m0", "P0")}
    ms, Ps, mf, Pf, ll = oracle.tv_smooth(model, g["y"], "rts")
    ms2, Ps2 = oracle.tv_tf(model, g["y"], mf, Pf)
    for a, b in ((mf, g["mf"]), (Pf, g["Pf"]), (ms, g["ms"]), (Ps, g["Ps"]), (ms2, g["ms_tf"]), (Ps2, g["Ps_tf"])):
        assert rel(a, b) < 1e-13
    assert abs(ll - float(g["loglik"])) < 1e-12 * abs(ll)
