"""The C ABI library builds, loads and exports every symbol include/popcorn.h declares.

CPU-only: argument validation returns before any CUDA call, so it is checked
here too; nothing in this file runs a kernel.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "popcorn.h")


@pytest.fixture(scope="module")
def pc():
    import __graft_entry__ as ge
    b = ge._build_module()
    if not os.path.exists(b.LIB):
        b.build()
    import paper_2501_05587_gb300 as mod
    return mod


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"POPCORN_API\s+[\w\s\*]+?\b(popcorn_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("popcorn_kernel_matrix", "popcorn_fit", "popcorn_assign_step",
                     "popcorn_status_string", "popcorn_last_error_message", "popcorn_version"):
        assert required in names


def test_library_exports_every_declared_symbol(pc):
    lib = ctypes.CDLL(pc.LIBRARY_PATH)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(pc.EXPORTED_SYMBOLS) == set(_declared())


def test_status_strings_and_version(pc):
    lib = ctypes.CDLL(pc.LIBRARY_PATH)
    lib.popcorn_status_string.restype = ctypes.c_char_p
    assert lib.popcorn_status_string(0) == b"POPCORN_OK"
    assert lib.popcorn_status_string(1) == b"POPCORN_ERR_INVALID"
    assert lib.popcorn_status_string(4) == b"POPCORN_ERR_TIMEOUT"
    assert lib.popcorn_status_string(99) == b"POPCORN_ERR_UNKNOWN"
    assert pc.popcorn_version() >= 100
    # the allocation counter answers without a device (no call here allocates)
    a = pc._lib.popcorn_allocation_count()
    assert a >= 0 and pc._lib.popcorn_allocation_count() == a


def test_invalid_arguments_rejected_before_any_cuda_call(pc):
    lib = pc._lib
    kern = pc._Kernel(2, 1, 1.0, 0.0, 1.0)
    # null pointers
    st = lib.popcorn_fit(None, 10, 2, 2, 2, kern, None, 5, 0.0, None, None, None, None, None, None)
    assert st == 1
    assert b"null" in lib.popcorn_last_error_message()
    P = np.zeros((10, 2), np.float32)
    lab = np.zeros(10, np.int32)
    out = np.zeros(10, np.int32)
    obj = ctypes.c_double()
    its = ctypes.c_int32()

    def fit(n=10, d=2, ldp=2, k=2, kern=kern, max_iter=5, tol=0.0, opt=None):
        return lib.popcorn_fit(P.ctypes.data, n, d, ldp, k, kern, lab.ctypes.data, max_iter, tol, opt,
                               out.ctypes.data, ctypes.byref(obj), ctypes.byref(its), None, None)

    assert fit(k=10) == 1            # k must be < n
    assert fit(k=0) == 1
    assert fit(k=300, n=1000) == 1   # k > 256
    assert fit(d=0) == 1
    assert fit(ldp=1) == 1
    assert fit(max_iter=-1) == 1
    assert fit(tol=-1.0) == 1
    assert fit(kern=pc._Kernel(2, 1, 1.0, 0.0, 0.0)) == 1        # sigma = 0
    assert fit(kern=pc._Kernel(1, 0, 1.0, 1.0, 1.0)) == 1        # degree 0
    assert fit(kern=pc._Kernel(7, 1, 1.0, 1.0, 1.0)) == 1        # unknown kind
    bad = pc._Options(0, 1, 1, 0, 0, 0, 0, 0, (ctypes.c_int64 * 4)(1, 0, 0, 0))
    assert fit(opt=ctypes.byref(bad)) == 1                       # reserved must be zero
    bad32 = pc._Options(0, 1, 1, 0, 0, 3, 0, 0, (ctypes.c_int64 * 4)())
    assert fit(opt=ctypes.byref(bad32)) == 1                     # autotune must be 0 or 1
    badks = pc._Options(0, 1, 1, 0, 7, 0, 0, 0, (ctypes.c_int64 * 4)())
    assert fit(opt=ctypes.byref(badks)) == 1                     # unknown K storage type
    rec = pc._Options(0, 0, 1, 0, 0, 0, 0, 0, (ctypes.c_int64 * 4)())
    assert fit(opt=ctypes.byref(rec)) == 5                       # recompute path needs BF16 or FP8
    fp8k = pc._Options(3, 1, 1, 0, 0, 0, 0, 0, (ctypes.c_int64 * 4)())
    assert fit(opt=ctypes.byref(fp8k)) == 5                      # FP8 only without a stored K
    badk = pc._Options(0, 2, 1, 0, 0, 0, 0, 0, (ctypes.c_int64 * 4)())
    assert fit(opt=ctypes.byref(badk)) == 1                      # store_k must be 0 or 1
    badp = pc._Options(0, 1, 1, 0, 0, 0, 3, 0, (ctypes.c_int64 * 4)())
    assert fit(opt=ctypes.byref(badp)) == 1                      # k_pass must be 0 (auto), 1 or 2
    badpad = pc._Options(0, 1, 1, 0, 0, 0, 0, 9, (ctypes.c_int64 * 4)())
    assert fit(opt=ctypes.byref(badpad)) == 1                    # sym_tile must be in [0, 8]
    # batched mode: its options are checked before any CUDA call too
    inst = (pc._Instance * 1)()
    inst[0] = pc._Instance(P.ctypes.data, 10, 2, 2, 2, kern, lab.ctypes.data, out.ctypes.data)
    objs = (ctypes.c_double * 1)()
    itsb = (ctypes.c_int32 * 1)()

    def batched(opt, count=1, max_iter=5):
        return lib.popcorn_fit_batched(count, inst, max_iter, 0.0, opt, objs, itsb, None, None)

    assert batched(ctypes.byref(badks)) == 1                     # unknown K storage type
    assert batched(ctypes.byref(bad)) == 1                       # reserved must be zero
    assert batched(ctypes.byref(rec)) == 5                       # batched mode stores K
    assert batched(ctypes.byref(fp8k)) == 5                      # FP8 is the recompute path's only
    assert batched(None, count=0) == 1
    assert batched(None, max_iter=-1) == 1
    # kernel matrix: ldk must be a multiple of 4 and >= n
    st = lib.popcorn_kernel_matrix(P.ctypes.data, 10, 2, 2, kern, 0, out.ctypes.data, 10, out.ctypes.data, None)
    assert st == 1
    st = lib.popcorn_assign_step(P.ctypes.data, 16, P.ctypes.data, 10, 0, lab.ctypes.data, lab.ctypes.data,
                                 None, None, None, None, None, None)
    assert st == 1


def test_autotune_cache_entries_and_clear(pc):
    """The tuned-schedule cache is host state: counting and clearing it touch no GPU."""
    pc.popcorn_autotune_clear()
    assert pc.popcorn_autotune_entries() == 0


def test_autotune_cache_file_is_read_by_a_new_process(pc, tmp_path):
    """Entries persisted in POPCORN_TUNE_CACHE are loaded by the next process (no GPU
    needed: reading the cache is host work); malformed lines are ignored and a later
    line with the same key replaces an earlier one."""
    import subprocess
    import sys
    path = tmp_path / "tune.txt"
    path.write_text("1 0 256 64 130 52 0 152 : 4096 8 2 0 3.500000\n"
                    "this line is not an entry\n"
                    "2 3 70 128 100 2 0 152 : 2 16 0 0 9.250000\n"
                    "1 0 256 64 130 52 0 152 : 8192 16 1 0 3.000000\n")
    code = ("import paper_2501_05587_gb300 as pc; print(pc.popcorn_autotune_entries()); "
            "pc.popcorn_autotune_clear(); print(pc.popcorn_autotune_entries())")
    env = dict(os.environ, POPCORN_TUNE_CACHE=str(path))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == ["2", "0"]
    assert path.read_text().count("\n") == 4        # clearing leaves the file alone


def test_kmeanspp_arguments_rejected_before_any_cuda_call(pc):
    lib = pc._lib
    kern = pc._Kernel(2, 1, 1.0, 0.0, 1.0)
    P = np.zeros((10, 2), dtype=np.float32)
    u = np.array([0.1, 0.2, 0.3])
    lab = np.zeros(10, dtype=np.int32)

    def seed(n=10, d=2, ldp=2, k=3, kern=kern, u=u, P=P, lab=lab):
        return lib.popcorn_kmeanspp(None if P is None else P.ctypes.data, n, d, ldp, k, kern,
                                    None if u is None else u.ctypes.data,
                                    None if lab is None else lab.ctypes.data, None, None)

    assert seed(P=None) == 1 and seed(u=None) == 1 and seed(lab=None) == 1
    assert seed(k=0) == 1 and seed(k=11) == 1          # 1 <= k <= n
    assert seed(n=0) == 1 and seed(d=0) == 1 and seed(ldp=1) == 1
    assert seed(u=np.array([0.1, 1.0, 0.3])) == 1      # a draw outside [0, 1)
    assert b"u[1]" in lib.popcorn_last_error_message()
    assert seed(kern=pc._Kernel(2, 1, 1.0, 0.0, 0.0)) == 1   # sigma = 0
