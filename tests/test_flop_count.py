"""The flops per step that bench.py's roofline uses (closed forms counted
loop by loop) against the library's count of the kernels' own step code
(kf_count_step_flops: the step functions run on the host with a counting
number type).  CPU only."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def bench_module():
    spec = importlib.util.spec_from_file_location("bench_work_model", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("nx", [2, 4])
def test_bench_flops_are_the_counted_flops(nx):
    import paper_2511_10363_gb300 as kf
    b = bench_module()
    m = nx // 2
    assert kf.kf_count_step_flops(nx, "filter_fold")["total"] == b.table_fold_flops(nx, m)
    assert kf.kf_count_step_flops(nx, "filter_carry")["total"] == b.filter_carry_flops(nx, m, False)
    assert kf.kf_count_step_flops(nx, "filter_carry_loglik")["total"] == b.filter_carry_flops(nx, m, True)
    assert kf.kf_count_step_flops(nx, "rts_fold")["total"] == b.rts_fold_flops(nx)
    assert kf.kf_count_step_flops(nx, "rts_carry")["total"] == b.rts_carry_flops(nx)
    assert b.filter_step_flops(nx, m, False) == b.table_fold_flops(nx, m) + b.filter_carry_flops(nx, m, False)
    assert b.rts_step_flops(nx) == b.rts_fold_flops(nx) + b.rts_carry_flops(nx)


def test_counter_counts_square_roots_and_reciprocals():
    """The RTS element's Cholesky factor of P_{k+1|k}: nx square roots and
    nx reciprocals per build; the filter's m x m inverse: one reciprocal."""
    import paper_2511_10363_gb300 as kf
    for nx in (2, 4):
        c = kf.kf_count_step_flops(nx, "rts_carry")
        assert c["sqrt"] == nx and c["rcp"] == nx
        assert kf.kf_count_step_flops(nx, "filter_carry")["rcp"] == 1


def test_counter_rejects_other_sizes():
    import paper_2511_10363_gb300 as kf
    with pytest.raises(kf.KfError):
        kf.kf_count_step_flops(8, "rts_fold")
    with pytest.raises(kf.KfError):
        kf.kf_count_step_flops(4, 9)
