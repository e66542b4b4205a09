"""The C-ABI library builds, loads and exports every entry point of include/gsk.h.

Also covers the host-side validation paths, which return before any CUDA call
and therefore run without a GPU.
"""

import ctypes as C
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libgsk():
    from paper_1609_08377_gb300 import build
    build.build()
    from paper_1609_08377_gb300 import gsk
    return gsk


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsk_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(libgsk):
    lib = libgsk.lib()
    headers = [h for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h")]
    names = [n for h in headers for n in _declared(h)]
    assert "gsk_solve" in names and "gsk_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_and_defaults(libgsk):
    assert libgsk.strerror(0) == "ok"
    assert "invalid" in libgsk.strerror(-1)
    o = libgsk.default_options()
    assert o.precision == 0 and o.tol == 1e-8 and o.use_graph == 1 and o.refine == 1


def _pencil(M=8, spd=True):
    rng = np.random.default_rng(0)
    A = rng.uniform(-1, 1, (M, M))
    A = (A + A.T) / 2
    B = np.eye(M) + 0.05 * (A - np.diag(np.diag(A)))
    if not spd:
        B[0, 0] = -1.0
    return sp.csr_matrix(A), sp.csr_matrix(B)


def _create(libgsk, A, B, off, cnt):
    from paper_1609_08377_gb300.gsk import _Csr, _Orbmap, _lib

    keep = []

    def csr(X):
        rp = np.ascontiguousarray(X.indptr, dtype=np.int64)
        ci = np.ascontiguousarray(X.indices, dtype=np.int32)
        v = np.ascontiguousarray(X.data, dtype=np.float64)
        keep.extend([rp, ci, v])
        return _Csr(X.shape[0], rp.ctypes.data, ci.ctypes.data, v.ctypes.data)

    off = np.ascontiguousarray(off, dtype=np.int32)
    cnt = np.ascontiguousarray(cnt, dtype=np.int8)
    om = _Orbmap(off.size, off.ctypes.data, cnt.ctypes.data, None)
    h = C.c_void_p()
    rc = _lib.gsk_create(C.byref(csr(A)), C.byref(csr(B)), C.byref(om), C.byref(h))
    if rc == 0:
        _lib.gsk_destroy(h)
    return rc


def test_create_rejects_bad_inputs_on_host(libgsk):
    A, B = _pencil()
    off, cnt = [0, 4], [4, 4]
    # orbital map that does not tile the rows
    assert _create(libgsk, A, B, [0, 3], [4, 4]) == libgsk.GSK_EINVAL
    # orbital count other than 1 or 4
    assert _create(libgsk, A, B, [0, 2], [2, 6]) == libgsk.GSK_EINVAL
    # non-symmetric A
    An = A.tolil()
    An[0, 1] += 0.5
    assert _create(libgsk, An.tocsr(), B, off, cnt) == libgsk.GSK_EINVAL
    # non-finite value
    Ab = A.copy()
    Ab.data[3] = np.nan
    assert _create(libgsk, Ab, B, off, cnt) == libgsk.GSK_EINVAL
    # B not positive / not diagonally dominant
    A2, B2 = _pencil(spd=False)
    assert _create(libgsk, A2, B2, off, cnt) == libgsk.GSK_ENOTSPD
    # different patterns
    Bd = sp.csr_matrix(np.eye(8))
    assert _create(libgsk, A, Bd, off, cnt) == libgsk.GSK_EINVAL


def _prototypes(header):
    """name -> number of parameters of every function prototype in a header."""
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    out = {}
    for m in re.finditer(r"\b(gsk_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_header(libgsk):
    """Every function the Python binding declares has the parameter count of
    its prototype in include/gsk.h (a mismatch would pass garbage through
    ctypes without any error)."""
    from paper_1609_08377_gb300 import gsk as g

    protos = _prototypes("gsk.h")
    lib = g.lib()
    checked = 0
    for name, proto_n in protos.items():
        f = getattr(lib, name)
        if f.argtypes is None:
            continue
        assert len(f.argtypes) == proto_n, (name, len(f.argtypes), proto_n)
        checked += 1
    assert checked >= 25


def test_per_column_values_are_marshalled_to_n_entries(libgsk):
    """Per-column damping passed to gsk_solve / gsk_autotune / gsk_features
    reaches the C side as exactly n_cols doubles: a scalar is repeated, an
    array of another length is refused on the host (the C side reads n_cols
    entries from the pointer)."""
    g = libgsk
    a = g._per_column(0.2, 3)
    assert a.dtype == np.float64 and a.shape == (3,) and (a == 0.2).all() and a.flags.c_contiguous
    b = g._per_column(np.array([0.05, 0.1, 0.2], dtype=np.float32), 3)
    assert b.dtype == np.float64 and np.allclose(b, [0.05, 0.1, 0.2])
    with pytest.raises(ValueError):
        g._per_column(np.array([0.1, 0.2]), 3)
    with pytest.raises(ValueError):
        g._per_column(np.zeros((3, 1)), 3)


def test_bounds_checked_build_links_and_exports(libgsk):
    """The -DGSK_DEBUG build (libgsk_debug.so) compiles for sm_103a and
    exports the same entry points; the normal build answers the self-test
    with GSK_ENOTSUP before touching the GPU."""
    from paper_1609_08377_gb300 import build

    path = build.build(debug=True)
    assert path.endswith("libgsk_debug.so") and os.path.exists(path)
    dbg = C.CDLL(path)
    for name in _declared("gsk.h"):
        assert hasattr(dbg, name), name
    dbg.gsk_strerror.restype = C.c_char_p
    assert b"index check" in dbg.gsk_strerror(libgsk.GSK_EBOUNDS)
    assert libgsk.debug_selftest() == (libgsk.GSK_ENOTSUP, 0, 0)
