"""The host FP64 covariance tables of the covariance-table path
(kf_covariance_tables), pinned to library routines and to the oracle:

- the settled filtering covariance solves the discrete algebraic Riccati
  equation (scipy.linalg.solve_discrete_are, on the predicted covariance),
  and the settled gain and RTS gain are its closed forms;
- the settled smoothed covariance solves the discrete Lyapunov equation
  Ps = E Ps E^T + (P - E Pp E^T) (scipy.linalg.solve_discrete_lyapunov),
  the fixed point of the RTS covariance recursion;
- the sequential oracle's filtering covariance has settled by time k0, and
  its smoothed covariance equals the settled value between k0 and T - kb.
Host only: no GPU needed."""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
import workloads as W


@pytest.fixture(scope="module")
def kf():
    from paper_2511_10363_gb300 import build
    build.build()
    import paper_2511_10363_gb300 as kf
    return kf


def models():
    return [("cv1d", W.model_for_nx(2)), ("cv2d", W.model_for_nx(4)), ("random8", W.model_for_nx(8, seed=8)),
            ("random4", W.random_stable_model(4, 2, seed=3))]


@pytest.mark.parametrize("name,model", models())
def test_settled_values_solve_riccati_and_lyapunov(kf, name, model):
    t = kf.kf_covariance_tables(model)
    assert t is not None
    F, Q, H, R = [np.asarray(model[k], dtype=np.float64) for k in ("F", "Q", "H", "R")]
    Pp = sl.solve_discrete_are(F.T, H.T, Q, R)           # predicted covariance at the fixed point
    S = H @ Pp @ H.T + R
    K = Pp @ H.T @ np.linalg.inv(S)
    P = Pp - K @ S @ K.T
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(t["P_inf"], P) < 1e-12
    assert rel(t["K_inf"], K) < 1e-12
    Pp2 = F @ P @ F.T + Q
    E = P @ F.T @ np.linalg.inv(Pp2)
    assert rel(t["E_inf"], E) < 1e-12
    Ps = sl.solve_discrete_lyapunov(E, P - E @ Pp2 @ E.T)
    assert rel(t["Ps_inf"], Ps) < 1e-11
    assert np.array_equal(t["Ps_inf"], t["Ps_inf"].T) and np.all(np.linalg.eigvalsh(t["Ps_inf"]) > 0)


@pytest.mark.parametrize("name,model", models())
def test_oracle_settles_where_the_tables_say(kf, name, model):
    t = kf.kf_covariance_tables(model)
    k0, kb = t["k0"], t["kb"]
    T = k0 + kb + 200
    y = W.simulate(model, T, seed=2)
    mf, Pf, _ = oracle.kf(model, y)
    ms, Ps = oracle.rts(model, mf, Pf)
    scale = np.abs(t["P_inf"]).max()
    # filtering covariance: settled from k0 on (time k at index k - 1)
    assert np.abs(Pf[k0 - 1:] - t["P_inf"]).max() <= 1e-12 * scale
    # smoothed covariance: settled between the transients
    mid = Ps[k0 + 1: T - kb]
    assert mid.shape[0] > 0
    assert np.abs(mid - t["Ps_inf"]).max() <= 1e-12 * np.abs(t["Ps_inf"]).max()
    # and not yet settled just after the start (the transient is real)
    assert np.abs(Pf[0] - t["P_inf"]).max() > 1e-6 * scale


def test_unsettled_model_is_declined(kf):
    """A model whose covariance recursion does not settle within 2^16 steps
    (an undamped random walk observed with huge noise) gets no tables."""
    model = {"F": np.eye(2), "Q": np.eye(2) * 1e-12, "H": np.array([[1.0, 0.0]]), "R": np.array([[1e12]]),
             "m0": np.zeros(2), "P0": np.eye(2)}
    assert kf.kf_covariance_tables(model) is None
