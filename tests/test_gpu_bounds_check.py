"""The bounds-checked build (KF_BOUNDS_CHECK) over the small parity cases.

In that build every index the kernels form into the inputs, outputs, tables
and workspace is checked; a failed check records KF_ERR_BOUNDS in the
status word and the access is skipped.  The parity tests read the status
word after every call (it must be 0) and compare every output with the
oracle, so a run of them against the checked library shows that no index of
those launches leaves its buffer.  It runs in a child process, which loads
the checked library through KFSCAN_LIB."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# small-T parity cases: every operation, scan, precision and state size of the
# per-step kernels, the time-invariant filter, the RTS kernel, the
# time-varying path and the covariance-table path (lengths up to 30001)
CASES = [
    ("tests/test_gpu_parity.py", None),
    ("tests/test_gpu_covariance_tables.py",
     "not 100000 and not bench_length and not times_out and not many_tiles"),
    ("tests/test_gpu_rts_kernel.py", "not 100000 and not full_size and not time"),
    ("tests/test_gpu_ti_filter.py", "not 100000 and not full_size and not time"),
    ("tests/test_gpu_tv.py", "not 100000 and not full_size and not time"),
]


@pytest.fixture(scope="module")
def checked_lib():
    from paper_2511_10363_gb300 import build
    return build.build(check=True)


def child_env(lib):
    env = dict(os.environ)
    env["KFSCAN_LIB"] = lib
    return env


def test_checked_library_loads(checked_lib):
    code = ("import paper_2511_10363_gb300 as kf; assert kf.LIB_PATH == %r; "
            "assert kf.kf_bounds_checked(); print('checked')" % checked_lib)
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=child_env(checked_lib),
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "checked" in r.stdout, r.stdout + r.stderr


@pytest.mark.parametrize("path,sel", CASES, ids=[c[0].split("/")[-1][:-3] for c in CASES])
def test_small_parity_cases_pass_the_index_checks(checked_lib, path, sel):
    cmd = [sys.executable, "-m", "pytest", path, "-m", "gpu", "-x", "-q", "-p", "no:cacheprovider"]
    if sel:
        cmd += ["-k", sel]
    r = subprocess.run(cmd, cwd=ROOT, env=child_env(checked_lib), capture_output=True, text=True,
                       timeout=3000)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout, tail
