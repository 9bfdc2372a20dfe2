"""The C-ABI library builds, loads and exports every entry point declared in
include/sem.h; argument checks reject bad input before any CUDA call.  CPU only."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1601_08179_gb300 import build, sem
    build.build()
    return sem.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "sem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sem_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_expected_entry_points():
    names = _declared()
    for must in ("sem_setup", "sem_apply_condensed", "sem_solve", "sem_recover_interior"):
        assert must in names


def test_library_exports_every_declared_symbol(L):
    from paper_1601_08179_gb300 import sem
    for name in _declared():
        assert hasattr(L, name), name
    assert set(sem.exported_symbols()) <= set(_declared())


def test_argument_checks_without_gpu(L):
    from paper_1601_08179_gb300 import sem
    D = sem._D
    h = ctypes.c_void_p()
    ok = np.ones(2)
    bad = np.array([1.0, -1.0])
    nan = np.array([1.0, np.nan])
    cases = [
        (1, ok, ok, ok, 1.0), (33, ok, ok, ok, 1.0), (4, bad, ok, ok, 1.0),
        (4, ok, nan, ok, 1.0), (4, ok, ok, ok, -1.0), (4, ok, ok, ok, float("inf")),
    ]
    for p, hx, hy, hz, lam in cases:
        st = L.sem_setup(ctypes.byref(h), p, 2, 2, 2, hx.ctypes.data_as(D), hy.ctypes.data_as(D),
                         hz.ctypes.data_as(D), lam, None)
        assert st == sem.SEM_EINVAL, (p, lam)
        assert L.sem_last_error().decode()
    st = L.sem_setup(ctypes.byref(h), 4, 0, 2, 2, ok.ctypes.data_as(D), ok.ctypes.data_as(D),
                     ok.ctypes.data_as(D), 1.0, None)
    assert st == sem.SEM_EINVAL
    for o in (sem.default_opts(rtol=2.0), sem.default_opts(deterministic=2), sem.default_opts(onepass_step=-1)):
        st = L.sem_setup(ctypes.byref(h), 4, 2, 2, 2, ok.ctypes.data_as(D), ok.ctypes.data_as(D),
                         ok.ctypes.data_as(D), 1.0, ctypes.byref(o))
        assert st == sem.SEM_EINVAL
        assert L.sem_last_error().decode()
    assert L.sem_debug_cg_step_timeout(None, None, None) == sem.SEM_EINVAL
    # null context
    assert L.sem_apply_condensed(None, None, None, 0, None) == sem.SEM_EINVAL
    assert L.sem_check_vector(None, None, 8) == sem.SEM_EINVAL
    # the bounds record exists in debug builds only (no CUDA call in a release build)
    st, n, first = sem.sem_debug_oob()
    assert (st, n, first) == (sem.SEM_ENOTSUP, 0, -1)
    assert L.sem_debug_limit_skeleton(None, 0) == sem.SEM_EINVAL
    assert L.sem_status_string(sem.SEM_ENOCONV) == b"not converged"
    L.sem_destroy(None)


def test_setup_rejects_a_skeleton_past_int32(L):
    """Entity offsets inside the kernels are 32-bit: a mesh whose packed
    skeleton reaches 2^31 entries (p = 32 on 92^3 elements, N_B ~ 2.3e9) is
    refused with SEM_ENOTSUP before any device work, with the reason."""
    from paper_1601_08179_gb300 import sem
    D = sem._D
    h = ctypes.c_void_p()
    m = 92
    hx = np.full(m, 1.0 / m)
    st = L.sem_setup(ctypes.byref(h), 32, m, m, m, hx.ctypes.data_as(D), hx.ctypes.data_as(D),
                     hx.ctypes.data_as(D), 1.0, None)
    assert st == sem.SEM_ENOTSUP
    assert "2^31" in L.sem_last_error().decode()


def test_default_opts(L):
    from paper_1601_08179_gb300 import sem
    o = sem.default_opts()
    assert o.rtol == 1e-10 and o.precision == sem.PREC_FP64 and o.check_every > 0
    assert o.reliable_delta == 0.0   # automatic, by degree
    assert o.deterministic == 1      # fixed-order edge and vertex sums in the FP64 operator


def test_opts_struct_matches_the_header():
    """The binding's sem_opts mirrors include/sem.h field for field (a
    mismatch would shift every later field)."""
    import os
    import re
    from paper_1601_08179_gb300 import sem
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "sem.h")).read()
    body = hdr[hdr.index("/* Solver options."):hdr.index("} sem_opts;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(double|int)\s+(\w+);", body)
    assert [(n, t) for t, n in fields] == [(n, {ctypes.c_double: "double", ctypes.c_int: "int"}[t])
                                           for n, t in sem.sem_opts._fields_]


def test_debug_build_compiles_and_exports_the_same_entry_points():
    """The SEM_DEBUG build (bounds record) compiles for sm_103a and exports
    every declared entry point; its debug calls check their arguments before
    any CUDA call."""
    from paper_1601_08179_gb300 import build
    D = ctypes.CDLL(build.build(debug=True))
    for name in _declared():
        assert hasattr(D, name), name
    D.sem_debug_oob.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    D.sem_debug_limit_skeleton.argtypes = [ctypes.c_void_p, ctypes.c_longlong]
    SEM_EINVAL = 1
    assert D.sem_debug_oob(None, None) == SEM_EINVAL
    assert D.sem_debug_limit_skeleton(None, 0) == SEM_EINVAL
