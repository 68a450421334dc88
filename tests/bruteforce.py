"""Dense joint-Gaussian brute force for small T (test helper, CPU only).

Independent of the oracle: it never runs a Kalman recursion.  It writes the
prior of the stacked state x_{1:T} in closed form (x_1 ~ N(F m0, F P0 F^T + Q),
x_k = F x_{k-1} + q), stacks the measurements y = H_blk x + r, and conditions
the joint Gaussian with a dense solve.  Filtering marginals at k condition on
y_{1:k} only; the log-likelihood is log N(y_{1:T}; H mu, H Sigma H^T + R_blk).
"""
import numpy as np


def prior(model, T):
    F, Q, m0, P0 = (np.asarray(model[k], float) for k in ("F", "Q", "m0", "P0"))
    n = F.shape[0]
    mu = np.zeros((T, n))
    Pk = np.zeros((T, n, n))
    x, P = m0, P0
    for k in range(T):
        x = F @ x
        P = F @ P @ F.T + Q
        mu[k], Pk[k] = x, P
    Sig = np.zeros((T * n, T * n))
    for k in range(T):
        Sig[k * n:(k + 1) * n, k * n:(k + 1) * n] = Pk[k]
        G = np.eye(n)
        for j in range(k + 1, T):
            G = F @ G
            blk = G @ Pk[k]              # Cov(x_j, x_k) = F^{j-k} P_k
            Sig[j * n:(j + 1) * n, k * n:(k + 1) * n] = blk
            Sig[k * n:(k + 1) * n, j * n:(j + 1) * n] = blk.T
    return mu.reshape(-1), Sig


def posterior(model, y, upto=None):
    """Condition the stacked prior on y_{1:upto}; returns (mean [T,n],
    cov blocks [T,n,n], loglik of the used measurements)."""
    H, R = np.asarray(model["H"], float), np.asarray(model["R"], float)
    y = np.asarray(y, float)
    T, m = y.shape
    n = H.shape[1]
    K = T if upto is None else upto
    mu, Sig = prior(model, T)
    Hb = np.zeros((K * m, T * n))
    for k in range(K):
        Hb[k * m:(k + 1) * m, k * n:(k + 1) * n] = H
    Rb = np.kron(np.eye(K), R)
    S = Hb @ Sig @ Hb.T + Rb
    v = y[:K].reshape(-1) - Hb @ mu
    Sv = np.linalg.solve(S, v)
    Gain = np.linalg.solve(S, Hb @ Sig).T
    mpost = mu + Gain @ v
    Spost = Sig - Gain @ Hb @ Sig
    sign, logdet = np.linalg.slogdet(S)
    assert sign > 0
    ll = -0.5 * (v @ Sv + logdet + K * m * np.log(2 * np.pi))
    means = mpost.reshape(T, n)
    covs = np.stack([Spost[k * n:(k + 1) * n, k * n:(k + 1) * n] for k in range(T)])
    return means, covs, ll


def filtering(model, y):
    T = y.shape[0]
    ms, Ps = [], []
    for k in range(1, T + 1):
        mk, Pk, _ = posterior(model, y[:k], upto=k)
        ms.append(mk[k - 1])
        Ps.append(Pk[k - 1])
    return np.array(ms), np.array(Ps)


# ---- time-varying model (per-step F, Q, u, H, R, d; record t is time t+1) ----

def tv_prior(model):
    """Stacked prior of x_{1:T}: x_k = F_{k-1} x_{k-1} + u_{k-1} + q_{k-1} with
    x_0 ~ N(m0, P0), written out with the state-transition products."""
    F, Q = np.asarray(model["F"], float), np.asarray(model["Q"], float)
    T, n = F.shape[0], F.shape[1]
    u = np.zeros((T, n)) if model.get("u") is None else np.asarray(model["u"], float)
    x, P = np.asarray(model["m0"], float), np.asarray(model["P0"], float)
    mu = np.zeros((T, n))
    Pk = np.zeros((T, n, n))
    for k in range(T):
        x = F[k] @ x + u[k]
        P = F[k] @ P @ F[k].T + Q[k]
        mu[k], Pk[k] = x, P
    Sig = np.zeros((T * n, T * n))
    for k in range(T):
        Sig[k * n:(k + 1) * n, k * n:(k + 1) * n] = Pk[k]
        G = np.eye(n)
        for j in range(k + 1, T):
            G = F[j] @ G                  # F_{j} ... F_{k+1} in record indexing
            blk = G @ Pk[k]
            Sig[j * n:(j + 1) * n, k * n:(k + 1) * n] = blk
            Sig[k * n:(k + 1) * n, j * n:(j + 1) * n] = blk.T
    return mu.reshape(-1), Sig


def tv_posterior(model, y, upto=None):
    """Condition the stacked time-varying prior on y_{1:upto}
    (y_k = H_k x_k + d_k + r_k); returns (means [T,n], cov blocks, loglik)."""
    H, R = np.asarray(model["H"], float), np.asarray(model["R"], float)
    y = np.asarray(y, float)
    T, m = y.shape
    n = H.shape[2]
    d = np.zeros((T, m)) if model.get("d") is None else np.asarray(model["d"], float)
    K = T if upto is None else upto
    mu, Sig = tv_prior(model)
    Hb = np.zeros((K * m, T * n))
    Rb = np.zeros((K * m, K * m))
    for k in range(K):
        Hb[k * m:(k + 1) * m, k * n:(k + 1) * n] = H[k]
        Rb[k * m:(k + 1) * m, k * m:(k + 1) * m] = R[k]
    S = Hb @ Sig @ Hb.T + Rb
    v = (y[:K] - d[:K]).reshape(-1) - Hb @ mu
    Sv = np.linalg.solve(S, v)
    Gain = np.linalg.solve(S, Hb @ Sig).T
    mpost = mu + Gain @ v
    Spost = Sig - Gain @ Hb @ Sig
    sign, logdet = np.linalg.slogdet(S)
    assert sign > 0
    ll = -0.5 * (v @ Sv + logdet + K * m * np.log(2 * np.pi))
    means = mpost.reshape(T, n)
    covs = np.stack([Spost[k * n:(k + 1) * n, k * n:(k + 1) * n] for k in range(T)])
    return means, covs, ll


def tv_filtering(model, y):
    T = y.shape[0]
    ms, Ps = [], []
    for k in range(1, T + 1):
        mk, Pk, _ = tv_posterior(model, y, upto=k)
        ms.append(mk[k - 1])
        Ps.append(Pk[k - 1])
    return np.array(ms), np.array(Ps)
