"""Pins of the FP64 oracle against facts fixed by the paper and by the
mathematics, never against the oracle itself:

* closed-form steady state of the scalar random walk (local-level model);
* a dense joint-Gaussian brute force of the whole posterior (T <= 64);
* special cases (H = 0, static parameter Q = 0 / F = I, T = 1);
* agreement of the RTS and two-filter smoothers (Sec. III-B);
* the elements of Sec. IV-C/IV-D against direct Gaussian conditioning;
* Lemmas 1 and 2: associativity, the neutral element, folds equal the
  sequential recursions, the split identity s_T = s_{k-1} (x) sbar_k (Sec. II-B);
* the scan algorithms of Sec. II on a non-commutative operator, with their
  work counts.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import scans
from tests import bruteforce
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rw_model(q, r):
    return dict(F=np.eye(1), Q=np.array([[q]]), H=np.eye(1), R=np.array([[r]]),
                m0=np.zeros(1), P0=np.eye(1))


# ---------------------------------------------------------------- closed forms

def test_random_walk_steady_state_closed_form():
    """Local-level model: the Riccati fixed point P^- = P^- - P^-^2/(P^- + r) + q
    gives P^-_inf = (q + sqrt(q^2 + 4qr))/2, P_inf = (-q + sqrt(q^2 + 4qr))/2,
    gain K = P^-/(P^- + r); the RTS fixed point P_s = P + G^2 (P_s - P^-),
    G = P/P^-, gives P_s = q r / sqrt(q^2 + 4 q r)."""
    with open(os.path.join(GOLDEN, "random_walk_steady_state.json")) as f:
        g = json.load(f)
    q, r, T = g["q"], g["r"], g["T"]
    s = math.sqrt(q * q + 4 * q * r)
    Pm, Pf, Ps = (q + s) / 2, (-q + s) / 2, q * r / s
    assert abs(Pm - g["P_pred_inf"]) < 1e-15 and abs(Pf - g["P_filt_inf"]) < 1e-15
    assert abs(Ps - g["P_smooth_inf"]) < 1e-15
    model = rw_model(q, r)
    y = W.simulate(model, T, seed=11)
    mf, Pfk, ll, mp, Ppk = oracle.kf(model, y, want_pred=True)
    k = T // 2
    assert abs(Ppk[k, 0, 0] - Pm) < 1e-12
    assert abs(Pfk[k, 0, 0] - Pf) < 1e-12
    K = Pm / (Pm + r)
    # steady-state mean update is exponential smoothing with gain K
    assert abs(mf[k, 0] - (mf[k - 1, 0] + K * (y[k, 0] - mf[k - 1, 0]))) < 1e-10 * (1 + abs(mf[k, 0]))
    ms, Psk = oracle.rts(model, mf, Pfk)
    assert abs(Psk[k, 0, 0] - Ps) < 1e-12
    G = Pf / Pm
    assert abs(ms[k, 0] - (mf[k, 0] + G * (ms[k + 1, 0] - mf[k, 0]))) < 1e-10 * (1 + abs(ms[k, 0]))
    ms2, Ps2 = oracle.tf(model, y, mf, Pfk)
    assert abs(Ps2[k, 0, 0] - Ps) < 1e-12
    # the last step is a filtering step in every smoother
    assert abs(Psk[-1, 0, 0] - Pf) < 1e-12 and abs(Ps2[-1, 0, 0] - Pf) < 1e-12


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("nx,ny,T,seed", [(2, 1, 17, 1), (4, 2, 40, 2), (8, 4, 24, 3), (3, 5, 12, 4)])
def test_oracle_vs_dense_joint_gaussian(nx, ny, T, seed):
    model = W.random_model(nx, ny, seed=seed)
    y = W.simulate(model, T, seed=100 + seed)
    mf, Pf, ll = oracle.kf(model, y)
    bm, bP = bruteforce.filtering(model, y)
    assert rel(mf, bm) < 1e-9
    assert rel(Pf, bP) < 1e-9
    sm, sP, bll = bruteforce.posterior(model, y)
    assert abs(ll - bll) < 1e-9 * max(1.0, abs(bll))
    ms, Ps = oracle.rts(model, mf, Pf)
    assert rel(ms, sm) < 1e-9
    assert rel(Ps, sP) < 1e-9
    ms2, Ps2 = oracle.tf(model, y, mf, Pf)
    assert rel(ms2, sm) < 1e-9
    assert rel(Ps2, sP) < 1e-9


def test_oracle_vs_dense_cv_tracking():
    model = W.cv_model()
    y = W.simulate(model, 48, seed=5)
    mf, Pf, ll = oracle.kf(model, y)
    bm, bP = bruteforce.filtering(model, y)
    assert rel(mf, bm) < 1e-9 and rel(Pf, bP) < 1e-9
    sm, sP, bll = bruteforce.posterior(model, y)
    ms, Ps = oracle.rts(model, mf, Pf)
    assert rel(ms, sm) < 1e-9 and rel(Ps, sP) < 1e-9
    assert abs(ll - bll) < 1e-9 * abs(bll)


# ---------------------------------------------------------------- special cases

def test_no_measurement_information():
    """H = 0: the filter is pure prediction and the log-likelihood is that of
    i.i.d. N(0, R) noise."""
    model = W.random_model(4, 2, seed=7)
    model["H"] = np.zeros((2, 4))
    T = 30
    y = W.simulate(model, T, seed=8)
    mf, Pf, ll = oracle.kf(model, y)
    F, Q, R = model["F"], model["Q"], model["R"]
    x, P = model["m0"], model["P0"]
    for k in range(T):
        x, P = F @ x, F @ P @ F.T + Q
        assert rel(mf[k], x) < 1e-12 and rel(Pf[k], P) < 1e-12
    Ri = np.linalg.inv(R)
    ref = sum(-0.5 * (yk @ Ri @ yk + np.linalg.slogdet(R)[1] + 2 * np.log(2 * np.pi)) for yk in y)
    assert abs(ll - ref) < 1e-10 * abs(ref)
    ms, Ps = oracle.rts(model, mf, Pf)
    assert rel(Ps, Pf) < 1e-10 and rel(ms, mf) < 1e-10


def test_static_parameter():
    """Q = 0, F = I: P_{k|k} = (P0^{-1} + k H^T R^{-1} H)^{-1} and the
    smoother is constant in k, equal to the final filtering estimate."""
    rng = np.random.default_rng(3)
    n, m, T = 3, 2, 25
    H = rng.standard_normal((m, n))
    R = np.diag([0.5, 2.0])
    P0 = np.diag([1.0, 2.0, 3.0])
    model = dict(F=np.eye(n), Q=np.zeros((n, n)), H=H, R=R, m0=np.ones(n), P0=P0)
    y = rng.standard_normal((T, m))
    mf, Pf, _ = oracle.kf(model, y)
    Ri = np.linalg.inv(R)
    for k in range(1, T + 1):
        assert rel(Pf[k - 1], np.linalg.inv(np.linalg.inv(P0) + k * H.T @ Ri @ H)) < 1e-11
    ms, Ps = oracle.rts(model, mf, Pf)
    ms2, Ps2 = oracle.tf(model, y, mf, Pf)
    for k in range(T):
        assert rel(Ps[k], Pf[-1]) < 1e-10 and rel(ms[k], mf[-1]) < 1e-10
        assert rel(Ps2[k], Pf[-1]) < 1e-10 and rel(ms2[k], mf[-1]) < 1e-10


def test_single_step_smoother_is_filter():
    model = W.random_model(4, 2, seed=9)
    y = W.simulate(model, 1, seed=10)
    mf, Pf, _ = oracle.kf(model, y)
    ms, Ps = oracle.rts(model, mf, Pf)
    ms2, Ps2 = oracle.tf(model, y, mf, Pf)
    assert np.array_equal(ms, mf) and np.array_equal(Ps, Pf)
    assert rel(ms2, mf) < 1e-15 and rel(Ps2, Pf) < 1e-15


@pytest.mark.parametrize("nx,ny,seed", [(2, 1, 21), (4, 2, 22), (8, 4, 23)])
def test_rts_equals_two_filter(nx, ny, seed):
    model = W.random_stable_model(nx, ny, seed=seed) if nx == 8 else W.random_model(nx, ny, seed=seed)
    y = W.simulate(model, 3000, seed=seed + 1)
    mf, Pf, _ = oracle.kf(model, y)
    ms, Ps = oracle.rts(model, mf, Pf)
    ms2, Ps2 = oracle.tf(model, y, mf, Pf)
    scale = np.maximum(np.linalg.norm(ms, axis=1), np.sqrt(np.trace(Ps, axis1=1, axis2=2)))
    assert np.max(np.linalg.norm(ms - ms2, axis=1) / scale) < 1e-10
    assert np.max(np.linalg.norm(Ps - Ps2, axis=(1, 2)) / np.linalg.norm(Ps, axis=(1, 2))) < 1e-10


# ---------------------------------------------------------------- elements

def test_filter_element_is_conditional_density():
    """a_k (k > 1) encodes p(x_k | y_k, x_{k-1}) = N(A x_{k-1} + b, C) and
    p(y_k | x_{k-1}) proportional to N_I(x_{k-1}; eta, J) (Sec. IV-C).  Both are
    checked against plain Gaussian conditioning at random x_{k-1}."""
    model = W.random_model(4, 3, seed=31)
    F, Q, H, R = (model[k] for k in ("F", "Q", "H", "R"))
    rng = np.random.default_rng(0)
    yk = rng.standard_normal(3)
    e = oracle.filter_element(model, 5, yk)
    S = H @ Q @ H.T + R
    for _ in range(3):
        xprev = rng.standard_normal(4)
        mu = F @ xprev
        G = Q @ H.T @ np.linalg.inv(S)
        cond_mean = mu + G @ (yk - H @ mu)
        cond_cov = Q - G @ H @ Q
        assert rel(e.A @ xprev + e.b, cond_mean) < 1e-12
        assert rel(e.C, cond_cov) < 1e-12
    # log p(y_k | x) = -1/2 (y - H F x)^T S^{-1} (y - H F x) + c = -1/2 x^T J x + eta^T x + c'
    def logp(x):
        v = yk - H @ F @ x
        return -0.5 * v @ np.linalg.solve(S, v)
    x0 = np.zeros(4)
    for i in range(4):
        ei = np.eye(4)[i]
        grad = (logp(x0 + ei) - logp(x0 - ei)) / 2
        assert abs(grad - e.eta[i]) < 1e-10 * (1 + abs(e.eta[i]))
        for j in range(4):
            ej = np.eye(4)[j]
            hess = (logp(ei + ej) - logp(ei - ej) - logp(-ei + ej) + logp(-ei - ej)) / 4
            assert abs(-hess - e.J[i, j]) < 1e-9 * (1 + abs(e.J[i, j]))


def test_first_filter_element_is_first_posterior():
    """a_1 has A_1 = 0 and (b_1, C_1) the filtering posterior at k = 1."""
    model = W.random_model(3, 2, seed=32)
    y = W.simulate(model, 1, seed=33)
    e = oracle.filter_element(model, 1, y[0])
    bm, bP = bruteforce.filtering(model, y)
    assert np.all(e.A == 0)
    assert rel(e.b, bm[0]) < 1e-12 and rel(e.C, bP[0]) < 1e-12


def test_rts_element_is_backward_conditional():
    """(E_k, g_k, L_k) encodes p(x_k | y_{1:k}, x_{k+1}) = N(E x_{k+1} + g, L)
    (Sec. IV-D), checked by conditioning the joint Gaussian of (x_k, x_{k+1})."""
    model = W.random_model(4, 2, seed=34)
    F, Q = model["F"], model["Q"]
    rng = np.random.default_rng(1)
    X = rng.standard_normal((4, 4))
    P = X @ X.T + 0.1 * np.eye(4)
    x = rng.standard_normal(4)
    e = oracle.rts_element(model, False, x, P)
    Sxx1 = P @ F.T
    S11 = F @ P @ F.T + Q
    for _ in range(3):
        x1 = rng.standard_normal(4)
        mean = x + Sxx1 @ np.linalg.solve(S11, x1 - F @ x)
        assert rel(e.E @ x1 + e.g, mean) < 1e-12
    assert rel(e.L, P - Sxx1 @ np.linalg.solve(S11, Sxx1.T)) < 1e-12
    last = oracle.rts_element(model, True, x, P)
    assert np.all(last.E == 0) and np.array_equal(last.g, x) and np.array_equal(last.L, P)


# ---------------------------------------------------------------- operators

def rand_filter_elem(rng, n):
    def psd():
        X = rng.standard_normal((n, n))
        return X @ X.T / n
    return oracle.FilterElem(rng.standard_normal((n, n)) * 0.7, rng.standard_normal(n), psd(),
                             rng.standard_normal(n), psd())


def felem_rel(x, y):
    return max(rel(x.A, y.A), rel(x.b, y.b), rel(x.C, y.C), rel(x.eta, y.eta), rel(x.J, y.J))


@pytest.mark.parametrize("n", [2, 4, 8])
def test_lemma1_associative_and_neutral(n):
    rng = np.random.default_rng(n)
    a, b, c = (rand_filter_elem(rng, n) for _ in range(3))
    op = oracle.filter_combine
    assert felem_rel(op(op(a, b), c), op(a, op(b, c))) < 1e-11
    e = oracle.FilterElem.identity(n)
    assert felem_rel(op(e, a), a) < 1e-15 and felem_rel(op(a, e), a) < 1e-15


@pytest.mark.parametrize("n", [2, 4, 8])
def test_lemma2_associative_and_neutral(n):
    rng = np.random.default_rng(10 + n)

    def r():
        X = rng.standard_normal((n, n))
        return oracle.RtsElem(rng.standard_normal((n, n)) * 0.6, rng.standard_normal(n), X @ X.T)
    a, b, c = r(), r(), r()
    op = oracle.rts_combine
    x, y = op(op(a, b), c), op(a, op(b, c))
    assert max(rel(x.E, y.E), rel(x.g, y.g), rel(x.L, y.L)) < 1e-12
    e = oracle.RtsElem.identity(n)
    for z in (op(e, a), op(a, e)):
        assert np.array_equal(z.E, a.E) and np.array_equal(z.g, a.g) and np.array_equal(z.L, a.L)


def filter_elements(model, y):
    return [oracle.filter_element(model, k + 1, y[k]) for k in range(len(y))]


@pytest.mark.parametrize("nx,ny,seed", [(2, 1, 41), (4, 2, 42), (8, 4, 43)])
def test_filter_fold_equals_kalman_filter(nx, ny, seed):
    """Eq. filtering_prefix_sums / Alg. pkf: the prefix a_1 (x) ... (x) a_k has
    b_k^+ = xbar_{k|k}, C_k^+ = P_{k|k}, whatever eta_1, J_1 are."""
    model = W.random_model(nx, ny, seed=seed)
    T = 60
    y = W.simulate(model, T, seed=seed)
    mf, Pf, _ = oracle.kf(model, y)
    els = filter_elements(model, y)
    pref, _ = scans.sequential(els, oracle.filter_combine)
    for k in range(T):
        assert rel(pref[k].b, mf[k]) < 1e-10 and rel(pref[k].C, Pf[k]) < 1e-10
        assert np.all(pref[k].A == 0)
    # eta_1, J_1 never reach (b, C): perturb them and refold
    els[0] = oracle.FilterElem(els[0].A, els[0].b, els[0].C, els[0].eta + 3.0, els[0].J * 2.0)
    pref2, _ = scans.sequential(els, oracle.filter_combine)
    for k in range(T):
        assert np.array_equal(pref2[k].b, pref[k].b) and np.array_equal(pref2[k].C, pref[k].C)


@pytest.mark.parametrize("nx,ny,seed", [(2, 1, 51), (4, 2, 52), (8, 4, 53)])
def test_rts_reverse_fold_equals_rts(nx, ny, seed):
    """Alg. prts: sbar_k = a_k (x) ... (x) a_T gives g_k^+ = xbar_{k|T}, L_k^+ = P_{k|T}."""
    model = W.random_model(nx, ny, seed=seed)
    T = 50
    y = W.simulate(model, T, seed=seed)
    mf, Pf, _ = oracle.kf(model, y)
    ms, Ps = oracle.rts(model, mf, Pf)
    els = [oracle.rts_element(model, k == T - 1, mf[k], Pf[k]) for k in range(T)]
    suf, _ = scans.reverse_sequential(els, oracle.rts_combine)
    for k in range(T):
        assert rel(suf[k].g, ms[k]) < 1e-10 and rel(suf[k].L, Ps[k]) < 1e-10


@pytest.mark.parametrize("terminal", ["identity", "zero"])
def test_two_filter_reverse_fold_gives_backward_filter(terminal):
    """Alg. ptf: the reverse scan of (a_2, ..., a_T, e) has eta_k^- = eta_{k|k+1:T},
    J_k^- = J_{k|k+1:T}; the neutral element (I,0,0,0,0) and the printed
    e = (0,0,0,0,0) give identical (eta, J)."""
    model = W.random_model(4, 2, seed=61)
    T = 40
    y = W.simulate(model, T, seed=62)
    mf, Pf, _ = oracle.kf(model, y)
    _, _, eta, J = oracle.tf(model, y, mf, Pf, want_info=True)
    els = filter_elements(model, y)
    e = oracle.FilterElem.identity(4) if terminal == "identity" else oracle.FilterElem.zero(4)
    seq = els[1:] + [e]
    suf, _ = scans.reverse_sequential(seq, oracle.filter_combine)
    for k in range(T - 1):
        assert rel(suf[k].eta, eta[k]) < 1e-10 and rel(suf[k].J, J[k]) < 1e-10
    assert np.all(suf[T - 1].eta == 0) and np.all(suf[T - 1].J == 0)


def test_split_identity():
    """s_T = s_{k-1} (x) sbar_k for every k (Sec. II-B)."""
    model = W.random_model(4, 2, seed=71)
    T = 24
    y = W.simulate(model, T, seed=72)
    els = filter_elements(model, y)
    pref, _ = scans.sequential(els, oracle.filter_combine)
    suf, _ = scans.reverse_sequential(els, oracle.filter_combine)
    for k in range(1, T):
        z = oracle.filter_combine(pref[k - 1], suf[k])
        assert rel(z.b, pref[-1].b) < 1e-10 and rel(z.C, pref[-1].C) < 1e-10
        assert rel(z.eta, pref[-1].eta) < 1e-10 and rel(z.J, pref[-1].J) < 1e-10


# ---------------------------------------------------------------- scan algorithms

def concat(x, y):
    return x + y


@pytest.mark.parametrize("T", [1, 2, 4, 8, 16, 64, 256])
def test_scans_on_noncommutative_operator(T):
    a = ["<%d>" % k for k in range(1, T + 1)]
    want = ["".join(a[:k]) for k in range(1, T + 1)]
    L = T.bit_length() - 1
    hs, n_hs = scans.hillis_steele(a, concat)
    bl, n_bl = scans.blelloch(a, concat, "")
    lf, n_lf = scans.ladner_fischer(a, concat)
    assert hs == want and bl == want and lf == want
    assert n_hs == T * L - T + 1          # Hillis-Steele work
    assert n_bl == 3 * T - 2              # Blelloch: (T-1) + (T-1) + T
    assert n_lf == max(2 * T - 2 - L, 0)  # in-place Ladner-Fischer
    rwant = ["".join(a[k:]) for k in range(T)]
    for scan, extra in ((scans.hillis_steele, ()), (scans.blelloch, ("",)), (scans.ladner_fischer, ())):
        r, _ = scans.reverse(scan, a, concat, *extra)
        assert r == rwant


@pytest.mark.parametrize("T", [1, 2, 4, 8, 16, 64, 256])
@pytest.mark.parametrize("N", [1, 2, 4, 16, 1024])
def test_sengupta_on_noncommutative_operator(T, N):
    """Alg. sengupta: exact prefixes of a non-commutative operator, forward
    and reversed, and its work: 2(T - N) - d* reduce and down-sweep
    combines plus Hillis-Steele's N log2 N - N + 1 on the top level (so
    N = 1 does the in-place Ladner-Fischer work 2T - 2 - log2 T)."""
    a = ["<%d>" % k for k in range(1, T + 1)]
    want = ["".join(a[:k]) for k in range(1, T + 1)]
    r, n = scans.sengupta(a, concat, N)
    assert r == want
    L = T.bit_length() - 1
    Ne = min(N, T)
    Ln = Ne.bit_length() - 1
    assert n == 2 * (T - Ne) - (L - Ln) + Ne * Ln - Ne + 1
    if N == 1:
        assert n == max(2 * T - 2 - L, 0)
    r, _ = scans.reverse(scans.sengupta, a, concat, N)
    assert r == ["".join(a[k:]) for k in range(T)]


def test_scans_on_kalman_elements():
    model = W.cv_model()
    T = 32
    y = W.simulate(model, T, seed=81)
    els = filter_elements(model, y)
    ref, _ = scans.sequential(els, oracle.filter_combine)
    for res, _ in (scans.hillis_steele(els, oracle.filter_combine),
                   scans.blelloch(els, oracle.filter_combine, oracle.FilterElem.identity(4)),
                   scans.ladner_fischer(els, oracle.filter_combine),
                   scans.sengupta(els, oracle.filter_combine, 1),
                   scans.sengupta(els, oracle.filter_combine, 8)):
        for k in range(T):
            assert rel(res[k].b, ref[k].b) < 1e-10 and rel(res[k].C, ref[k].C) < 1e-10


def test_oracle_regression_fixture():
    """The stored outputs of tests/golden/make_golden.py (written by calling
    only the oracle) still match, so an accidental change shows up."""
    g = np.load(os.path.join(GOLDEN, "oracle_cv_T64.npz"))
    model = W.cv_model()
    ms, Ps, mf, Pf, ll = oracle.smooth(model, g["y"], "rts")
    ms2, Ps2 = oracle.tf(model, g["y"], mf, Pf)
    for a, b in ((mf, g["mf"]), (Pf, g["Pf"]), (ms, g["ms"]), (Ps, g["Ps"]), (ms2, g["ms_tf"]), (Ps2, g["Ps_tf"])):
        assert rel(a, b) < 1e-13
    assert abs(ll - float(g["loglik"])) < 1e-12 * abs(ll)
