"""CPU-only checks of the C-ABI library: it loads, exports every function
declared in include/*.h, and its host-side argument checks and workspace
sizing work without a GPU (no compute call is made)."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

import paper_2511_10363_gb300 as kf
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(kf_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2511_10363_gb300 import build
    build.build()
    return kf.lib()


def test_header_declares_the_abi():
    names = declared_functions()
    for required in ("kf_filter", "kf_rts_smooth", "kf_two_filter_smooth", "kf_workspace_size",
                     "kf_sync_status", "kf_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(lib):
    for s in range(8):
        assert kf.kf_status_string(s)
    assert "sm_103a" in kf.kf_version()


FAKE = ctypes.c_void_p(1 << 20)   # never dereferenced: every call below fails its host checks


def call_filter(model, T=16, y=FAKE, prec=1, scan=1, m=FAKE):
    mm = kf.Model(model)
    return kf.lib().kf_filter(ctypes.byref(mm.c), T, y, prec, scan, m, None, None, None, None)


def test_argument_errors(lib):
    good = W.cv_model()
    assert call_filter(good, T=0) == 1                       # T >= 1
    assert call_filter(good, y=None) == 1                    # y required
    assert call_filter(good, m=None) == 1                    # output required
    assert call_filter(good, prec=7) == 1                    # bad enum
    assert call_filter(good, scan=9) == 1
    assert call_filter(good, y=ctypes.c_void_p((1 << 20) + 2)) == 1   # misaligned
    # rows move as vectors: ny = 2 floats need 8-byte, nx = 4 float means 16-byte alignment
    assert call_filter(good, y=ctypes.c_void_p((1 << 20) + 4)) == 1
    assert call_filter(good, m=ctypes.c_void_p((1 << 20) + 8)) == 1
    bad = dict(good)
    bad["F"] = np.eye(3)
    bad["H"] = np.zeros((2, 3))
    bad["Q"] = np.eye(3)
    bad["P0"] = np.eye(3)
    bad["m0"] = np.zeros(3)
    assert call_filter(bad) == 1                             # nx = 3 unsupported
    r = dict(good)
    r["R"] = -np.eye(2)
    assert call_filter(r) == 2                               # R not PD
    q = dict(good)
    q["Q"] = good["Q"] - 0.5 * np.eye(4)
    assert call_filter(q) == 2                               # Q not PSD
    a = dict(good)
    a["P0"] = np.array([[1, 2, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1.0]])
    assert call_filter(a) == 2                               # P0 not symmetric


def test_workspace_size(lib):
    s1 = kf.kf_workspace_size("filter", 4, 2, 1 << 20, "fp32", "dlb")
    s2 = kf.kf_workspace_size("rts", 4, 2, 1 << 20, "fp32", "dlb")
    s3 = kf.kf_workspace_size("rts", 4, 2, 1 << 20, "fp64", "dlb")
    s4 = kf.kf_workspace_size("rts", 4, 2, 1 << 20, "fp32", "blelloch")
    assert 0 < s1 < s2 < s3 and s2 < s4
    # the smoothers keep the filter means and packed covariances: (4 + 10) words per step
    assert s2 - s1 >= (1 << 20) * 14 * 4
    assert kf.kf_workspace_size("rts", 3, 2, 100) == 0
    assert kf.kf_workspace_size("rts", 4, 9, 100) == 0


def test_sengupta_option(lib):
    assert kf.kf_get_option("sengupta_n") == 1
    for bad in (0, 3, 12, 1 << 31):
        with pytest.raises(kf.KfError):
            kf.kf_set_option("sengupta_n", bad)
    kf.kf_set_option("sengupta_n", 16384)
    assert kf.kf_get_option("sengupta_n") == 16384
    kf.kf_set_option("sengupta_n", 1)
    # levels and Hillis-Steele scratch fit in the second level buffer
    assert kf.kf_workspace_size("rts", 4, 2, 1000, "fp32", "sengupta") == \
        kf.kf_workspace_size("rts", 4, 2, 1000, "fp32", "blelloch")


def test_options(lib):
    assert kf.kf_get_option("wait_timeout_ns") == 10 ** 9
    with pytest.raises(kf.KfError):
        kf.kf_set_option("wait_timeout_ns", 10)
    kf.kf_set_option("wait_timeout_ns", 5 * 10 ** 8)
    assert kf.kf_get_option("wait_timeout_ns") == 5 * 10 ** 8
    kf.kf_set_option("wait_timeout_ns", 10 ** 9)


def test_tuning_table_file(lib, tmp_path):
    """The tuning table is host state: load, query, save and clear need no GPU.
    Malformed or out-of-range lines are skipped."""
    kf.kf_tuning_clear()
    src = tmp_path / "in.txt"
    src.write_text("# comment\n"
                   "1 4 2 1 20 1 256 2 0 0.25\n"      # rts, nx 4, ny 2, fp32, T in [2^20, 2^21)
                   "0 8 4 0 12 4 0 0 0 1.5\n"         # filter, nx 8, fp64, level scan
                   "1 4 2 1 19 9 128 1 0 0.1\n"       # unknown scan: skipped
                   "1 4 2 1 18 1 100 1 0 0.1\n"       # bad thread count: skipped
                   "garbage\n")
    kf.kf_tuning_load(src)
    e = kf.kf_tuning_get("rts", 4, 2, "fp32", (1 << 20) + 5)
    assert e == {"scan": "dlb", "threads": 256, "lookback_warps": 2, "steps_per_thread": 0, "ms": 0.25}
    assert kf.kf_tuning_get("rts", 4, 2, "fp32", (1 << 20) - 1) is None
    assert kf.kf_tuning_get("filter", 8, 4, "fp64", 5000)["scan"] == "ladner_fischer"
    assert kf.kf_tuning_get("rts", 4, 2, "fp32", 1 << 19) is None
    assert kf.kf_tuning_get("rts", 4, 2, "fp32", 1 << 18) is None
    out = tmp_path / "out.txt"
    kf.kf_tuning_save(out)
    kf.kf_tuning_clear()
    assert kf.kf_tuning_get("rts", 4, 2, "fp32", 1 << 20) is None
    kf.kf_tuning_load(out)
    assert kf.kf_tuning_get("rts", 4, 2, "fp32", 1 << 20) == e
    with pytest.raises(kf.KfError):
        kf.kf_tuning_load(tmp_path / "missing.txt")
    kf.kf_tuning_clear()
    # the AUTO workspace covers the look-back and the level scans
    auto = kf.kf_workspace_size("rts", 4, 2, 1 << 16, "fp32", "auto")
    assert auto >= kf.kf_workspace_size("rts", 4, 2, 1 << 16, "fp32", "dlb")
    assert auto >= kf.kf_workspace_size("rts", 4, 2, 1 << 16, "fp32", "ladner_fischer")


def call_tv(nx=4, ny=2, T=16, y=FAKE, prec=1, scan=1, m=FAKE, arrays=None, m0=None, P0=None, op="filter"):
    """A kf_tv_* call with fake device arrays; host FP64 prior."""
    D = ctypes.POINTER(ctypes.c_double)
    a = dict(F=FAKE, Q=FAKE, u=None, H=FAKE, R=FAKE, d=None)
    a.update(arrays or {})
    m0 = np.zeros(nx) if m0 is None else np.ascontiguousarray(m0, dtype=np.float64)
    P0 = np.eye(nx) if P0 is None else np.ascontiguousarray(P0, dtype=np.float64)
    c = kf._TvModel(nx, ny, *[a[k] for k in ("F", "Q", "u", "H", "R", "d")], m0.ctypes.data_as(D),
                    P0.ctypes.data_as(D))
    L = kf.lib()
    if op == "filter":
        return L.kf_tv_filter(ctypes.byref(c), T, y, prec, scan, m, None, None, None, None)
    fn = L.kf_tv_rts_smooth if op == "rts" else L.kf_tv_two_filter_smooth
    return fn(ctypes.byref(c), T, y, prec, scan, m, FAKE, None, None, None, None, None)


def test_tv_argument_errors(lib):
    for op in ("filter", "rts", "tf"):
        assert call_tv(T=0, op=op) == 1                      # T >= 1
        assert call_tv(y=None, op=op) == 1
        assert call_tv(m=None, op=op) == 1
        assert call_tv(nx=3, op=op) == 1                     # nx in {2, 4, 8}
        assert call_tv(ny=5, op=op) == 1                     # ny <= nx
        assert call_tv(ny=0, op=op) == 1
        assert call_tv(prec=7, op=op) == 1
        for scan in (2, 3, 4, 5, 9):                         # look-back scan only
            assert call_tv(scan=scan, op=op) == 1
        for k in ("F", "Q", "H", "R"):                       # required arrays
            assert call_tv(arrays={k: None}, op=op) == 1
        # arrays aligned to the element size (FP32: 4 bytes, FP64: 8 bytes)
        assert call_tv(arrays={"u": ctypes.c_void_p((1 << 20) + 2)}, op=op) == 1
        assert call_tv(prec=0, arrays={"F": ctypes.c_void_p((1 << 20) + 4)}, op=op) == 1
        assert call_tv(y=ctypes.c_void_p((1 << 20) + 4), op=op) == 1   # ny = 2 FP32 rows: 8-byte
        assert call_tv(m0=[0, np.nan, 0, 0], op=op) == 1
        assert call_tv(P0=-np.eye(4), op=op) == 2            # prior not PSD
        assert call_tv(P0=np.triu(np.ones((4, 4))), op=op) == 2   # not symmetric


def test_batch_rts_smooth_argument_errors(lib):
    mm = kf.Model(W.cv_model())
    offs = np.array([0, 8, 16], dtype=np.int64)
    L = kf.lib()

    def call(nseq=2, offsets=offs, y=FAKE, m=FAKE, prec=1):
        return L.kf_batch_rts_smooth(ctypes.byref(mm.c), 1, None, nseq, offsets.ctypes.data_as(ctypes.c_void_p), y,
                                     prec, m, FAKE, None, None, None)
    assert call(nseq=0) == 1
    assert call(y=None) == 1
    assert call(m=None) == 1
    assert call(prec=7) == 1
    assert call(offsets=np.array([0, 8, 4], dtype=np.int64)) == 1   # decreasing offsets
