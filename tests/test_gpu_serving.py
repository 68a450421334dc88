"""The continuous-batching server: jobs of mixed operation, state size and
length submitted while others run; each result is checked against the
oracle and against the same job run alone through the single-sequence
entry points (within the FP32 tolerance)."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests.gpu_util import TOL, mean_err, cov_err

pytestmark = pytest.mark.gpu


def test_mixed_jobs_alone_and_in_the_mix():
    import torch
    import paper_2511_10363_gb300 as kf
    from paper_2511_10363_gb300 import build
    build.build()
    rng = np.random.default_rng(3)
    models = {nx: W.model_for_nx(nx, seed=nx) for nx in (2, 4, 8)}
    srv = kf.Server(budget_bytes=512 << 20, max_inflight=3, max_batch_steps=1 << 20)
    jobs = []
    try:
        pending = []
        for i in range(60):
            nx = int(rng.choice([2, 4, 8]))
            op = ["filter", "rts", "tf"][int(rng.integers(3))]
            T = int(np.exp(rng.uniform(np.log(50), np.log(20000))))
            model = models[nx]
            y = W.simulate(model, T, seed=500 + i).astype(np.float32)
            yh = torch.tensor(y).pin_memory()
            mh = torch.empty((T, nx), dtype=torch.float32).pin_memory()
            Ph = torch.empty((T, nx, nx), dtype=torch.float32).pin_memory()
            lh = torch.empty(1, dtype=torch.float64).pin_memory()
            pending.append((op, nx, model, yh, mh, Ph, lh))
        # submit in a burst, so that jobs arrive while others run
        for op, nx, model, yh, mh, Ph, lh in pending:
            jid = srv.submit(op, model, yh, "fp32", mh, Ph, lh)
            jobs.append((jid, op, nx, model, yh, mh, Ph, lh))
        batches = set()
        for jid, op, nx, model, yh, mh, Ph, lh in jobs:
            srv.wait(jid, timeout_s=120)
            done, info = srv.poll(jid)
            assert done and info[2] >= info[1] >= info[0]
            batches.add(int(info[3]))
            yo = yh.double().numpy()
            mf, Pf, ll = oracle.kf(model, yo)
            if op == "filter":
                rm, rP = mf, Pf
            elif op == "rts":
                rm, rP = oracle.rts(model, mf, Pf)
            else:
                rm, rP = oracle.tf(model, yo, mf, Pf)
            m, P = mh.double().numpy(), Ph.double().numpy()
            assert mean_err(m, rm, rP) <= TOL["fp32"] and cov_err(P, rP) <= TOL["fp32"]
            assert abs(lh.item() - ll) <= 1e-3 * max(1.0, abs(ll))
            # alone
            yt = yh.cuda()
            if op == "filter":
                am, aP, al = kf.kf_filter(model, yt, "fp32", "dlb", loglik=True)
            elif op == "rts":
                am, aP, al = kf.kf_rts_smooth(model, yt, "fp32", "dlb", loglik=True)
            else:
                am, aP, al = kf.kf_two_filter_smooth(model, yt, "fp32", "dlb", loglik=True)
            am, aP = am.double().cpu().numpy(), aP.double().cpu().numpy()
            assert mean_err(m, am, aP) <= TOL["fp32"] and cov_err(P, aP) <= TOL["fp32"]
            assert abs(lh.item() - al.item()) <= 1e-3 * max(1.0, abs(al.item()))
            srv.release(jid)
        assert len(batches) < len(jobs)      # some jobs were batched together
    finally:
        srv.close()


def test_budget_rejection():
    import torch
    import paper_2511_10363_gb300 as kf
    srv = kf.Server(budget_bytes=4 << 20, max_inflight=1)
    try:
        T = 1 << 18
        y = torch.zeros((T, 2), dtype=torch.float32).pin_memory()
        with pytest.raises(kf.KfError) as e:
            srv.submit("rts", W.cv_model(), y, "fp32")
        assert e.value.status == 6          # KF_ERR_BUDGET
    finally:
        srv.close()


def test_cancel_a_queued_job():
    """A job still waiting in the queue (the server's only stream is busy with
    a long job of another class) is cancelled: it is done with
    KF_ERR_CANCELLED and its outputs are untouched; the running job is not
    affected; cancelling a finished or unknown job reports that it cannot."""
    import time
    import torch
    import paper_2511_10363_gb300 as kf
    big = W.cv_model()
    Tb = 1 << 21
    yb = torch.tensor(W.simulate(big, Tb, seed=77)).pin_memory()
    mb = torch.empty((Tb, 4), dtype=torch.float64).pin_memory()
    Pb = torch.empty((Tb, 4, 4), dtype=torch.float64).pin_memory()
    small = W.model_for_nx(2, seed=2)
    Ts = 500
    ys = torch.tensor(W.simulate(small, Ts, seed=78).astype(np.float32)).pin_memory()
    ms = torch.full((Ts, 2), float("nan"), dtype=torch.float32).pin_memory()
    srv = kf.Server(budget_bytes=2 << 30, max_inflight=1, max_batch_steps=1 << 23)
    try:
        j1 = srv.submit("rts", big, yb, "fp64", mb, Pb, None)
        t0 = time.time()
        while srv.poll(j1)[1][1] == 0.0 and not srv.poll(j1)[0]:   # until its batch has started
            assert time.time() - t0 < 60
            time.sleep(0.0005)
        j2 = srv.submit("filter", small, ys, "fp32", ms, None, None)
        assert srv.cancel(j2)
        with pytest.raises(kf.KfError) as e:
            srv.poll(j2)
        assert e.value.status == 9                 # KF_ERR_CANCELLED
        with pytest.raises(kf.KfError):
            srv.wait(j2, 10)
        srv.wait(j1, 120)
        assert not srv.cancel(j1)                  # finished
        assert not srv.cancel(123456789)           # unknown
        assert torch.isnan(ms).all()               # never written
        mf, Pf, _ = oracle.kf(big, yb.numpy())
        msr, Psr = oracle.rts(big, mf, Pf)
        assert mean_err(mb.numpy(), msr, Psr) < 1e-9 and cov_err(Pb.numpy(), Psr) < 1e-9
    finally:
        srv.close()
