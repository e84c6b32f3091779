"""The C-ABI library builds, loads and exports every declared symbol; host-side
validation paths that need no GPU return the documented status codes."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1204_0556_gb300 import build as B
from paper_1204_0556_gb300 import inputs as I
from paper_1204_0556_gb300 import lpdec as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"LPDEC_API[^;(]*?\b(lpdec_\w+)\s*\(", txt))
    return names


def test_header_constants_match_the_binding():
    """Every integer #define LPDEC_* of the header has the binding's value
    (status codes, per-frame statuses, state types, schedules)."""
    txt = open(os.path.join(ROOT, "include", "lpdec.h")).read()
    defs = dict(re.findall(r"^#define (LPDEC_\w+)\s+\(?(-?\d+)\)?", txt, re.M))
    assert len(defs) >= 15
    for name, val in defs.items():
        if hasattr(L, name):
            py = getattr(L, name)
        else:  # LPDEC_STATE_F32 -> STATE_F32, LPDEC_SCHED_AUTO -> SCHED_AUTO
            py = getattr(L, name[len("LPDEC_"):])
        assert py == int(val), name


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_symbols()
    assert len(declared) >= 9
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lpdec_\w+)", out))
    assert declared <= exported, declared - exported
    assert declared == set(L.EXPORTED) | (declared - set(L.EXPORTED))
    assert set(L.EXPORTED) <= declared
    for name in declared:
        assert hasattr(lib, name)
    # nothing but the C-ABI is exported
    assert all(s.startswith("lpdec_") for s in exported)


def test_params_default(lib):
    p = L.lpdec_params_default()
    assert (p.mu, p.rho, p.eps, p.max_iter, p.state_dtype, p.cert_tol, p.schedule, p.iters_per_launch) == \
        (3.0, 1.9, 1e-5, 1000, 0, 1e-2, 0, 1)
    assert ctypes.sizeof(L.lpdec_params) == 72
    assert "sm_103a" in L.lpdec_version()


def _code_arrays(c):
    return [np.ascontiguousarray(a, dtype=np.int32) for a in (c.row_ptr, c.col_idx, c.col_ptr, c.row_idx, c.edge_perm)]


def _create(lib, n, m, arrs):
    out = ctypes.c_void_p()
    ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) for a in arrs]
    return lib.lpdec_code_create(n, m, *ptrs, ctypes.byref(out))


def test_code_create_rejects_bad_graphs(lib):
    c = I.benchmark_code("C96", 0)
    good = _code_arrays(c)
    # unsorted columns in a row
    bad = [a.copy() for a in good]
    bad[1][0], bad[1][1] = bad[1][1], bad[1][0]
    assert _create(lib, c.n, c.m, bad) == L.LPDEC_EINVAL
    assert "ascending" in L.lpdec_last_error()
    # CSC disagreeing with CSR
    bad = [a.copy() for a in good]
    bad[4][0], bad[4][1] = bad[4][1], bad[4][0]
    assert _create(lib, c.n, c.m, bad) == L.LPDEC_EINVAL
    # a variable with no checks: x_i undefined (division by |N_v(i)|, Section 3.2)
    rows = [r for r in c.rows()]
    cc = I.code_from_rows(c.n + 1, rows)
    assert _create(lib, cc.n, cc.m, _code_arrays(cc)) == L.LPDEC_EINVAL
    assert "degree 0" in L.lpdec_last_error()
    # check degree above 32
    big = I.code_from_rows(33, [list(range(33))])
    assert _create(lib, big.n, big.m, _code_arrays(big)) == L.LPDEC_EINVAL
    # n, m not positive
    assert _create(lib, 0, c.m, good) == L.LPDEC_EINVAL


def test_decode_and_project_reject_bad_arguments(lib):
    p = L.lpdec_params_default()
    assert lib.lpdec_decode(None, 1, None, ctypes.byref(p), None, None, None, None, None) == L.LPDEC_EINVAL
    assert lib.lpdec_project(0, 10, None, None, None) == L.LPDEC_EINVAL
    assert lib.lpdec_project(33, 10, None, None, None) == L.LPDEC_EINVAL
    assert lib.lpdec_project(6, -1, None, None, None) == L.LPDEC_EINVAL
    assert lib.lpdec_project(6, 0, None, None, None) == L.LPDEC_OK


def test_tile_calls_reject_bad_arguments(lib):
    """Host-side checks of the tile setters and getter (no code object, no GPU)."""
    gt, g, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    assert lib.lpdec_set_streamed_tile(None, 0, 64, 2, 3) == L.LPDEC_EINVAL
    assert lib.lpdec_get_tile(None, 0, L.SCHED_STREAMED, ctypes.byref(gt), ctypes.byref(g), ctypes.byref(r)) == L.LPDEC_EINVAL
    assert lib.lpdec_set_tile(None, 0, 64, 2) == L.LPDEC_EINVAL


def test_release_memory_without_pools(lib):
    """With no decode run yet in this process there is no pool to trim."""
    assert lib.lpdec_release_memory() == L.LPDEC_OK


def test_python_binding_fails_loudly_without_library(tmp_path):
    saved = L._lib
    try:
        L._lib = None
        with pytest.raises(RuntimeError, match="not found"):
            L.load(str(tmp_path / "missing.so"))
    finally:
        L._lib = saved


def test_server_entry_points_reject_null_arguments(lib):
    rid = ctypes.c_uint64()
    p = L.lpdec_params_default()
    assert lib.lpdec_server_create(1 << 20, None, None) == L.LPDEC_EINVAL
    assert lib.lpdec_server_add_code(None, None, None) == L.LPDEC_EINVAL
    assert lib.lpdec_server_submit(None, 0, 1, None, ctypes.byref(p), ctypes.byref(rid)) == L.LPDEC_EINVAL
    assert lib.lpdec_server_poll(None, 1, 0, None, None, None, None) == L.LPDEC_EINVAL
    assert lib.lpdec_server_stats(None, None, None, None, None) == L.LPDEC_EINVAL
    assert lib.lpdec_server_destroy(None) == L.LPDEC_EINVAL
    assert lib.lpdec_decode_mixed(None, 0, 0, None, None, ctypes.byref(p), None, None, None, None, None) \
        == L.LPDEC_EINVAL
