"""Helpers for the GPU parity tests: run the CUDA library through its C ABI
and the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np

import oracle

# Tolerances on per-step normwise relative errors:
#   means:       |dm_k| / max(|m_k|, sqrt(tr P_k))
#   covariances: |dP_k|_F / |P_k|_F
# Elementwise relative error is ill-posed for entries near zero (cross
# covariances, velocities near zero), so the gate is normwise per step.
TOL = {"fp64": 1e-9, "fp32": 1e-4, "fp32_fp64solve": 1e-4}


def gpu_run(op, model, y, precision, scan, loglik=False, want_filter=False):
    import torch
    import paper_2511_10363_gb300 as kf
    dt = torch.float64 if precision == "fp64" else torch.float32
    yt = torch.as_tensor(np.ascontiguousarray(y)).to(device="cuda", dtype=dt)
    out = {}
    if op == "filter":
        m, P, ll = kf.kf_filter(model, yt, precision, scan, loglik=loglik)
        out["mf"], out["Pf"] = m, P
    else:
        T, nx = y.shape[0], np.asarray(model["F"]).shape[0]
        mf = torch.empty((T, nx), dtype=dt, device="cuda") if want_filter else None
        Pf = torch.empty((T, nx, nx), dtype=dt, device="cuda") if want_filter else None
        fn = kf.kf_rts_smooth if op == "rts" else kf.kf_two_filter_smooth
        ms, Ps, ll = fn(model, yt, precision, scan, mf_out=mf, Pf_out=Pf, loglik=loglik)
        out["ms"], out["Ps"] = ms, Ps
        if want_filter:
            out["mf"], out["Pf"] = mf, Pf
    st = kf.kf_sync_status()
    assert st == 0, "device status %d" % st
    res = {k: v.double().cpu().numpy() for k, v in out.items()}
    if loglik:
        res["ll"] = float(ll.item())
    return res


def oracle_inputs(y, precision):
    """The oracle sees exactly the values the GPU sees (y rounded to the
    working precision, then widened to FP64)."""
    return np.asarray(y, np.float32).astype(np.float64) if precision != "fp64" else np.asarray(y, np.float64)


def oracle_run(model, y):
    mf, Pf, ll = oracle.kf(model, y)
    ms, Ps = oracle.rts(model, mf, Pf)
    ms2, Ps2 = oracle.tf(model, y, mf, Pf)
    return dict(mf=mf, Pf=Pf, ll=ll, ms_rts=ms, Ps_rts=Ps, ms_tf=ms2, Ps_tf=Ps2)


def mean_err(m, mref, Pref):
    scale = np.maximum(np.linalg.norm(mref, axis=1), np.sqrt(np.abs(np.trace(Pref, axis1=1, axis2=2))))
    return float(np.max(np.linalg.norm(m - mref, axis=1) / scale))


def cov_err(P, Pref):
    return float(np.max(np.linalg.norm(P - Pref, axis=(1, 2)) / np.linalg.norm(Pref, axis=(1, 2))))


def check_psd(P):
    """Covariance invariants: exactly symmetric and positive definite."""
    assert np.array_equal(P, np.swapaxes(P, 1, 2)), "covariance not symmetric"
    ev = np.linalg.eigvalsh(P)
    assert np.all(ev > 0), "covariance not positive definite (min eig %g)" % ev.min()
