"""Streaming (resumable) filtering: the filter's last carry is the checkpoint.
Filtering a sequence chunk by chunk, each chunk started from the previous
chunk's last filtered mean and covariance as its prior (m0, P0 =
xbar_{0|0}, P_{0|0} of Sec. III-A), gives the same filtering moments as one
call over the whole sequence, and the chunks' log-likelihoods add up to the
whole sequence's (the chain rule p(y_{1:T}) = prod_k p(y_k | y_{1:k-1}))."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import TOL, mean_err, cov_err, oracle_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("chunks", [[5000], [1, 999, 4000], [1000] * 5, [37, 2048, 1, 2914]])
def test_chunked_filter_equals_whole(precision, chunks):
    import torch
    import paper_2511_10363_gb300 as kf
    from paper_2511_10363_gb300 import build
    build.build()
    model = W.cv_model()
    T = sum(chunks)
    y = oracle_inputs(W.simulate(model, T, seed=77), precision)
    dt = kf.dtype_of(precision)
    mf, Pf, ll = oracle.kf(model, y)
    m_parts, P_parts, lls = [], [], 0.0
    prior = dict(model)
    a = 0
    for n in chunks:
        yt = torch.tensor(y[a:a + n], dtype=dt, device="cuda")
        m, P, l = kf.kf_filter(prior, yt, precision, "dlb", loglik=True)
        assert kf.kf_sync_status() == 0
        m_parts.append(m.double().cpu().numpy())
        P_parts.append(P.double().cpu().numpy())
        lls += float(l.item())
        prior = dict(model, m0=m_parts[-1][-1], P0=P_parts[-1][-1])   # the checkpoint
        a += n
    m_all, P_all = np.concatenate(m_parts), np.concatenate(P_parts)
    tol = TOL[precision]
    assert mean_err(m_all, mf, Pf) <= tol and cov_err(P_all, Pf) <= tol
    if precision == "fp64":
        assert abs(lls - ll) <= 1e-9 * abs(ll)
