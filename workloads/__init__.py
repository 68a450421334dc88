"""Seeded synthetic inputs: model matrices and data simulated from the
linear-Gaussian state-space model of Sec. III-A of arXiv 2511.10363.

This module holds NO filtering or smoothing arithmetic: it only draws
random numbers and simulates x_k = F x_{k-1} + q_{k-1}, y_k = H x_k + r_k.
It is shared by the tests, the benchmark and the oracle comparisons, and it
imports neither the oracle nor the CUDA library.

Models:
  * ``cv_model``: 2D constant-velocity tracking, state [p_x, p_y, v_x, v_y],
    white-noise-acceleration Q, position measurements (nx=4, ny=2); the
    tracking workload of the paper's experiments (Sec. VI-A uses nx=4,
    ny=2).  ``cv1d_model`` is its 1D version (nx=2, ny=1).
  * ``random_stable_model``: F = 0.99 * (Q factor of a Gaussian matrix) with
    the sign fixed so that diag(R) > 0 (as in Sec. VI-A), Q = q I,
    H ~ N(0, 1), R = r I.
  * ``random_model``: every matrix random as in Sec. VI-A (F from a QR
    factor, Q and R as Xi Xi^T plus a floor), m0, P0 random.
  * ``tv_model``: a time-varying model (per-step F_{k-1}, Q_{k-1}, u_{k-1},
    H_k, R_k, d_k of the general model of Sec. III-A) as per-step arrays;
    ``simulate_tv`` draws data from it.
"""
from __future__ import annotations

import numpy as np


def _rng(seed):
    return np.random.default_rng(np.random.PCG64(int(seed)))


def cv_model(dt=0.1, q=1.0, r=0.25):
    I2 = np.eye(2)
    Z2 = np.zeros((2, 2))
    F = np.block([[I2, dt * I2], [Z2, I2]])
    Q = q * np.block([[dt ** 3 / 3 * I2, dt ** 2 / 2 * I2], [dt ** 2 / 2 * I2, dt * I2]])
    H = np.hstack([I2, Z2])
    R = r * I2
    return dict(F=F, Q=Q, H=H, R=R, m0=np.zeros(4), P0=np.eye(4))


def cv1d_model(dt=0.1, q=1.0, r=0.25):
    F = np.array([[1.0, dt], [0.0, 1.0]])
    Q = q * np.array([[dt ** 3 / 3, dt ** 2 / 2], [dt ** 2 / 2, dt]])
    H = np.array([[1.0, 0.0]])
    R = np.array([[r]])
    return dict(F=F, Q=Q, H=H, R=R, m0=np.zeros(2), P0=np.eye(2))


def _orth(rng, n):
    X = rng.standard_normal((n, n))
    Qf, Rf = np.linalg.qr(X)
    return Qf * np.sign(np.diag(Rf))[None, :]


def random_stable_model(nx=8, ny=4, seed=0, q=0.1, r=0.5):
    rng = _rng(seed)
    F = 0.99 * _orth(rng, nx)
    H = rng.standard_normal((ny, nx))
    return dict(F=F, Q=q * np.eye(nx), H=H, R=r * np.eye(ny), m0=np.zeros(nx), P0=np.eye(nx))


def random_model(nx, ny, seed=0, floor=0.05):
    rng = _rng(seed)
    F = 0.99 * _orth(rng, nx)
    Xq = rng.standard_normal((nx, nx)) / np.sqrt(nx)
    Xr = rng.standard_normal((ny, ny)) / np.sqrt(ny)
    Xp = rng.standard_normal((nx, nx)) / np.sqrt(nx)
    Q = Xq @ Xq.T + floor * np.eye(nx)
    R = Xr @ Xr.T + floor * np.eye(ny)
    H = rng.standard_normal((ny, nx))
    m0 = rng.standard_normal(nx)
    P0 = Xp @ Xp.T + floor * np.eye(nx)
    return dict(F=F, Q=Q, H=H, R=R, m0=m0, P0=P0)


def model_for_nx(nx, seed=0):
    """The per-size models used by the mixed workloads: nx=2 the 1D
    constant-velocity model, nx=4 the 2D one, nx=8 a random stable model."""
    if nx == 2:
        return cv1d_model()
    if nx == 4:
        return cv_model()
    return random_stable_model(nx, nx // 2, seed=seed)


def simulate(model, T, seed, nseq=None):
    """Draw x_0 ~ N(m0, P0) and simulate T steps.  Returns y of shape
    [T, ny] (or [nseq, T, ny] when nseq is given), FP64."""
    rng = _rng(seed)
    F, Q, H, R = (np.asarray(model[k], dtype=np.float64) for k in ("F", "Q", "H", "R"))
    m0, P0 = np.asarray(model["m0"], np.float64), np.asarray(model["P0"], np.float64)
    nx, ny = F.shape[0], H.shape[0]
    S = 1 if nseq is None else int(nseq)
    Lq = np.linalg.cholesky(Q + 1e-300 * np.eye(nx)) if np.any(Q) else np.zeros((nx, nx))
    Lr = np.linalg.cholesky(R)
    Lp = np.linalg.cholesky(P0) if np.any(P0) else np.zeros((nx, nx))
    x = m0[None, :] + rng.standard_normal((S, nx)) @ Lp.T
    y = np.empty((S, T, ny))
    FT, HT, LqT, LrT = F.T, H.T, Lq.T, Lr.T
    chunk = 4096
    for t0 in range(0, T, chunk):
        t1 = min(T, t0 + chunk)
        qn = rng.standard_normal((t1 - t0, S, nx)) @ LqT
        rn = rng.standard_normal((t1 - t0, S, ny)) @ LrT
        for t in range(t0, t1):
            x = x @ FT + qn[t - t0]
            y[:, t, :] = x @ HT + rn[t - t0]
    return y[0] if nseq is None else y


def loguniform_lengths(nseq, lo, hi, seed):
    """Sequence lengths T_i = floor(exp(U(ln lo, ln hi)))."""
    rng = _rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=nseq))).astype(np.int64)


def ragged_batch(model, lengths, seed):
    """Concatenated data of independent sequences with the given lengths
    (each with its own x_0).  Returns (y [sum T_i, ny], offsets [nseq+1])."""
    lengths = np.asarray(lengths, dtype=np.int64)
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    ny = np.asarray(model["H"]).shape[0]
    y = np.empty((int(offsets[-1]), ny))
    if len(lengths) == 0:
        return y, offsets
    # simulate in groups of similar length so memory stays bounded
    order = np.argsort(lengths, kind="stable")
    group = 256
    for g0 in range(0, len(order), group):
        idx = order[g0:g0 + group]
        Tg = int(lengths[idx].max())
        ys = simulate(model, Tg, seed * 100003 + g0, nseq=len(idx))
        for r, i in enumerate(idx):
            y[offsets[i]:offsets[i + 1]] = ys[r, :lengths[i]]
    return y, offsets


def tv_model(nx, T, seed=0, inputs=True):
    """Seeded time-varying model with per-step arrays, record t = 0 .. T-1
    belonging to time k = t + 1: F[t] = F_{k-1}, Q[t] = Q_{k-1},
    u[t] = u_{k-1}, H[t] = H_k, R[t] = R_k, d[t] = d_k (u = d = None when
    ``inputs`` is false).
      nx = 2: 1D constant velocity with a random step dt_t ~ U(0.05, 0.15),
              noise intensity q_t ~ U(0.5, 1.5), H_t = [h_t, 0] with
              h_t ~ U(0.8, 1.2), R_t ~ U(0.1, 0.4) (ny = 1).
      nx = 4: 2D constant velocity, same dt_t and q_t, H_t = [Rot(theta_t) 0]
              with a slowly turning sensor angle theta_t, R_t = Rot diag Rot^T
              with variances U(0.1, 0.4) (ny = 2).
      nx = 8: F_t = 0.99 x a random orthogonal matrix per step, Q_t = q_t I
              with q_t ~ U(0.05, 0.15), H_t ~ N(0, 1)^{4 x 8},
              R_t = 0.5 I + X X^T / 4 (ny = 4).
    Inputs: u_t is a random acceleration a_t ~ N(0, 0.5^2) entering like the
    noise (nx = 2, 4) or N(0, 0.1^2) per component (nx = 8); d_t ~ N(0, 0.1^2).
    m0 = 0, P0 = I."""
    rng = _rng(seed)
    T = int(T)
    if nx in (2, 4):
        dt = rng.uniform(0.05, 0.15, T)
        q = rng.uniform(0.5, 1.5, T)
        g = 1 if nx == 2 else 2
        Ig = np.eye(g)
        F = np.zeros((T, nx, nx))
        Q = np.zeros((T, nx, nx))
        F[:, :g, :g] = Ig
        F[:, g:, g:] = Ig
        F[:, :g, g:] = dt[:, None, None] * Ig
        Q[:, :g, :g] = (q * dt ** 3 / 3)[:, None, None] * Ig
        Q[:, :g, g:] = (q * dt ** 2 / 2)[:, None, None] * Ig
        Q[:, g:, :g] = (q * dt ** 2 / 2)[:, None, None] * Ig
        Q[:, g:, g:] = (q * dt)[:, None, None] * Ig
        a = 0.5 * rng.standard_normal((T, g))
        u = np.concatenate([(dt ** 2 / 2)[:, None] * a, dt[:, None] * a], axis=1)
        if nx == 2:
            H = np.zeros((T, 1, 2))
            H[:, 0, 0] = rng.uniform(0.8, 1.2, T)
            R = rng.uniform(0.1, 0.4, T)[:, None, None]
        else:
            th = 0.3 * np.sin(2 * np.pi * np.arange(T) / 97.0) + 0.05 * rng.standard_normal(T)
            c, s_ = np.cos(th), np.sin(th)
            Rot = np.stack([np.stack([c, -s_], -1), np.stack([s_, c], -1)], -2)
            H = np.concatenate([Rot, np.zeros((T, 2, 2))], axis=2)
            var = rng.uniform(0.1, 0.4, (T, 2))
            R = Rot @ (var[:, :, None] * np.eye(2)) @ np.transpose(Rot, (0, 2, 1))
    elif nx == 8:
        ny = 4
        X = rng.standard_normal((T, nx, nx))
        Qf, Rf = np.linalg.qr(X)
        F = 0.99 * Qf * np.sign(np.diagonal(Rf, axis1=1, axis2=2))[:, None, :]
        Q = rng.uniform(0.05, 0.15, T)[:, None, None] * np.eye(nx)
        H = rng.standard_normal((T, ny, nx))
        Xr = rng.standard_normal((T, ny, ny))
        R = 0.5 * np.eye(ny) + Xr @ np.transpose(Xr, (0, 2, 1)) / ny
        u = 0.1 * rng.standard_normal((T, nx))
    else:
        raise ValueError("nx must be 2, 4 or 8")
    ny = H.shape[1]
    d = 0.1 * rng.standard_normal((T, ny))
    R = 0.5 * (R + np.transpose(R, (0, 2, 1)))
    Q = 0.5 * (Q + np.transpose(Q, (0, 2, 1)))
    return dict(F=F, Q=Q, u=u if inputs else None, H=H, R=R, d=d if inputs else None,
                m0=np.zeros(nx), P0=np.eye(nx))


def simulate_tv(model, seed):
    """Draw x_0 ~ N(m0, P0) and simulate x_k = F_{k-1} x_{k-1} + u_{k-1} + q,
    y_k = H_k x_k + d_k + r from a ``tv_model``.  Returns y [T, ny], FP64."""
    rng = _rng(seed)
    F, Q, H, R = (np.asarray(model[k], dtype=np.float64) for k in ("F", "Q", "H", "R"))
    T, nx = F.shape[0], F.shape[1]
    ny = H.shape[1]
    u = np.zeros((T, nx)) if model.get("u") is None else np.asarray(model["u"], np.float64)
    d = np.zeros((T, ny)) if model.get("d") is None else np.asarray(model["d"], np.float64)
    Lq = np.linalg.cholesky(Q + 1e-12 * np.eye(nx))
    Lr = np.linalg.cholesky(R)
    qn = np.einsum("tij,tj->ti", Lq, rng.standard_normal((T, nx)))
    rn = np.einsum("tij,tj->ti", Lr, rng.standard_normal((T, ny)))
    x = np.asarray(model["m0"], np.float64) + np.linalg.cholesky(np.asarray(model["P0"], np.float64)) @ \
        rng.standard_normal(nx)
    xs = np.empty((T, nx))
    for t in range(T):
        x = F[t] @ x + u[t] + qn[t]
        xs[t] = x
    return np.einsum("tij,tj->ti", H, xs) + d + rn
