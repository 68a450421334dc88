"""Writes the fixtures of tests/golden/.

* random_walk_steady_state.json: the worked example of the local-level model
  (F = H = 1, Q = q, R = r) whose Riccati fixed points have closed forms:
  P^-_inf = (q + sqrt(q^2 + 4qr))/2, P_inf = (-q + sqrt(q^2 + 4qr))/2 and the
  smoothed interior variance q r / sqrt(q^2 + 4qr).  Computed from those
  formulas here, not by any filter.
* oracle_cv_T64.npz: the oracle's own outputs on the 2D constant-velocity
  model (nx=4, ny=2, dt=0.1, q=1, R=0.25 I) at T=64, seed 1, a regression
  fixture that calls only oracle/.
* oracle_tv_T48.npz: the same for a time-varying model (the seeded
  ``tv_model(4, 48, seed=12)`` with inputs u, d, its arrays stored in the
  fixture) at T = 48: filter, RTS, two-filter and the log-likelihood.
"""
import json
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads as W  # noqa: E402


def main():
    q, r = 1.0, 0.25
    s = math.sqrt(q * q + 4 * q * r)
    with open(os.path.join(HERE, "random_walk_steady_state.json"), "w") as f:
        json.dump(dict(q=q, r=r, T=1024, P_pred_inf=(q + s) / 2, P_filt_inf=(-q + s) / 2,
                       P_smooth_inf=q * r / s,
                       source="local-level Riccati fixed points derived from the KF and RTS "
                              "recursions of Sec. III-A/III-B"), f, indent=1)
    model = W.cv_model()
    y = W.simulate(model, 64, seed=1)
    ms, Ps, mf, Pf, ll = oracle.smooth(model, y, "rts")
    ms2, Ps2 = oracle.tf(model, y, mf, Pf)
    np.savez(os.path.join(HERE, "oracle_cv_T64.npz"), y=y, mf=mf, Pf=Pf, ms=ms, Ps=Ps, ms_tf=ms2,
             Ps_tf=Ps2, loglik=ll)
    tv_fixture()


def tv_fixture():
    tv = W.tv_model(4, 48, seed=12)
    y = W.simulate_tv(tv, seed=13)
    ms, Ps, mf, Pf, ll = oracle.tv_smooth(tv, y, "rts")
    ms2, Ps2 = oracle.tv_tf(tv, y, mf, Pf)
    np.savez(os.path.join(HERE, "oracle_tv_T48.npz"), F=tv["F"], Q=tv["Q"], u=tv["u"], H=tv["H"], R=tv["R"],
             d=tv["d"], m0=tv["m0"], P0=tv["P0"], y=y, mf=mf, Pf=Pf, ms=ms, Ps=Ps, ms_tf=ms2, Ps_tf=Ps2, loglik=ll)


if __name__ == "__main__":
    main()
