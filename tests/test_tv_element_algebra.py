"""CPU check of the algebra behind the time-varying element build: with
S = L L^T (Cholesky), W1 = L^{-1} H Qe, W2 = L^{-1} H F, w = L^{-1} r,

    A = F - W1^T W2,  b = ue + W1^T w,  C = Qe - W1^T W1,
    eta = W2^T w,     J = W2^T W2

equal the elements of Eqs. pkf_init1..3 as the oracle writes them
(K = Qe H^T S^{-1}, A = (I - K H) F, b = u + K (y - H u - d), ...), for
(Qe, ue) = (Q_{k-1}, u_{k-1}) at k >= 2 and (P_{1|0}, xbar_{1|0}) at k = 1.
At k = 1 only (A, b, C) are compared: eta_1 and J_1 never reach an output
(A_1 = 0) and the two sides evaluate them with different S.

This pins the algebra (a NumPy restatement of the formulas the device
builders use), not the device code itself: tv_filter_elem and tv_rts_elem
run only on the GPU, where tests/test_gpu_tv.py compares every filtered and
smoothed moment with the time-varying oracle, including ny < nx (nx = 2, 4, 8
with ny = 1, 2, 4, measurement rows padded to nx on the device) and non-zero
inputs u and d, at FP64 within 1e-9."""
import numpy as np
import pytest

import oracle
from tests.test_oracle_tv_pins import random_tv_model


def whitened(F, Qe, ue, H, R, d, y, first):
    S = H @ Qe @ H.T + R
    L = np.linalg.cholesky(S)
    W1 = np.linalg.solve(L, H @ Qe)
    W2 = np.linalg.solve(L, H @ F)
    w = np.linalg.solve(L, y - H @ ue - d)
    A = np.zeros_like(F) if first else F - W1.T @ W2
    return A, ue + W1.T @ w, Qe - W1.T @ W1, W2.T @ w, W2.T @ W2


@pytest.mark.parametrize("nx,ny,seed", [(2, 1, 1), (4, 2, 2), (4, 4, 3), (8, 4, 4), (8, 8, 5)])
def test_whitened_element_equals_paper_element(nx, ny, seed):
    T = 6
    model = random_tv_model(nx, ny, T, seed)
    rng = np.random.default_rng(seed)
    y = rng.standard_normal((T, ny))
    m0, P0 = model["m0"], model["P0"]
    for t in range(T):
        F, Q, u, H, R, d = (model[k][t] for k in ("F", "Q", "u", "H", "R", "d"))
        if t == 0:
            Qe, ue = F @ P0 @ F.T + Q, F @ m0 + u
        else:
            Qe, ue = Q, u
        A, b, C, eta, J = whitened(F, Qe, ue, H, R, d, y[t], t == 0)
        ref = oracle.tv_filter_element(model, t + 1, y[t])
        scale = max(1.0, np.abs(ref.C).max(), np.abs(ref.b).max())
        assert np.abs(A - ref.A).max() < 1e-12 * max(1.0, np.abs(ref.A).max())
        assert np.abs(b - ref.b).max() < 1e-12 * scale
        assert np.abs(C - ref.C).max() < 1e-12 * scale
        if t > 0:
            assert np.abs(eta - ref.eta).max() < 1e-12 * max(1.0, np.abs(ref.eta).max())
            assert np.abs(J - ref.J).max() < 1e-12 * max(1.0, np.abs(ref.J).max())


@pytest.mark.parametrize("nx,seed", [(2, 11), (4, 12), (8, 13)])
def test_cholesky_rts_element_equals_paper_element(nx, seed):
    """The RTS build: with U = F_k P and F_k P F_k^T + Q_k = L L^T,
    E = (L^{-T} L^{-1} U)^T, g = x - E (F_k x + u_k), L_k = P - E U equal
    Eq. prts_init1 as the oracle writes it."""
    T = 5
    model = random_tv_model(nx, max(1, nx // 2), T, seed)
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((nx, nx))
    P = X @ X.T / nx + 0.1 * np.eye(nx)
    x = rng.standard_normal(nx)
    for k in range(1, T):           # time k uses record k: F_k, Q_k, u_k
        F, Q, u = model["F"][k], model["Q"][k], model["u"][k]
        U = F @ P
        L = np.linalg.cholesky(U @ F.T + Q)
        Et = np.linalg.solve(L.T, np.linalg.solve(L, U))
        E = Et.T
        g = x - E @ (F @ x + u)
        Lk = P - E @ U
        ref = oracle.tv_rts_element(model, k, T, x, P)
        assert np.abs(E - ref.E).max() < 1e-12 * max(1.0, np.abs(ref.E).max())
        assert np.abs(g - ref.g).max() < 1e-12 * max(1.0, np.abs(ref.g).max())
        assert np.abs(Lk - ref.L).max() < 1e-12 * max(1.0, np.abs(ref.L).max())
