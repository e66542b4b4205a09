"""Thin Python binding of libgsk (argument marshalling only).

Every computation happens in the CUDA library behind the C ABI declared in
include/gsk.h; this module converts Python/NumPy/PyTorch arguments to plain
pointers and sizes. Importing it loads libgsk.so and fails loudly when the
library has not been built (there is no fallback path).
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# GSK_DEBUG=1 in the environment loads the bounds-checked build (build.build(debug=True))
DEBUG_BUILD = os.environ.get("GSK_DEBUG", "0") == "1"
LIB_PATH = os.path.join(_PKG, "libgsk_debug.so" if DEBUG_BUILD else "libgsk.so")

GSK_OK, GSK_EINVAL, GSK_ENOTSPD, GSK_ENOMEM, GSK_ECUDA, GSK_ETIMEOUT, GSK_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
GSK_EBOUNDS = -7
GSK_CONVERGED, GSK_NOT_CONVERGED, GSK_BREAKDOWN, GSK_TIMEOUT = 0, 1, 2, 3
GSK_FP64, GSK_MIXED, GSK_MIXED_DF = 0, 1, 2
GSK_SCHED_FIFO, GSK_SCHED_LEARNED = 0, 1
GSK_SPMM_AUTO, GSK_SPMM_GATHER, GSK_SPMM_STAGED = 0, 1, 2


class GskError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {code} ({strerror(code)})")
        self.code = code


class Stats(C.Structure):
    _fields_ = [("outer_steps", C.c_int64), ("cg_iterations", C.c_int64), ("kernel_launches", C.c_int64),
                ("batch_w", C.c_int32), ("used_graph", C.c_int32), ("spmm_kernel", C.c_int32),
                ("debug_code", C.c_int32), ("debug_index", C.c_int64)]


class _Csr(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p)]


class _Orbmap(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("orb_offset", C.c_void_p), ("orb_count", C.c_void_p), ("pos", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("batch_w", C.c_int32), ("refine", C.c_int32), ("sched", C.c_int32),
                ("inner_tol", C.c_double), ("max_inner", C.c_int32), ("use_graph", C.c_int32),
                ("stream", C.c_void_p), ("spmm_kernel", C.c_int32)]


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        how = "build.build(debug=True)" if DEBUG_BUILD else "__graft_entry__.build()"
        raise ImportError(f"{os.path.basename(LIB_PATH)} not built ({LIB_PATH}); run {how}")
    lib = C.CDLL(LIB_PATH)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "gsk_default_options": (None, [P]),
        "gsk_create": (C.c_int, [P, P, P, P]),
        "gsk_destroy": (C.c_int, [P]),
        "gsk_dims": (C.c_int, [P, P, P]),
        "gsk_pattern_offsets": (C.c_int, [P, I32, P, P]),
        "gsk_solve": (C.c_int, [P, I32, P, P, I32, P, P, P, P, P, P]),
        "gsk_density": (C.c_int, [P, I64, I32, P, P, D, D, P, P, P]),
        "gsk_trace": (C.c_int, [P, I32, P, P, I32, P]),
        "gsk_strerror": (C.c_char_p, [C.c_int]),
        "gsk_last_stats": (C.c_int, [P, P]),
        "gsk_row_order": (C.c_int, [P, P]),
        "gsk_spmm": (C.c_int, [P, I32, I32, I32, P, P, I32, P]),
        "gsk_density_noalloc": (C.c_int, [I64, I32, P, P, D, D, P, P, P]),
        "gsk_alu_peak": (C.c_int, [I32, I32, P, P]),
        "gsk_autotune_result": (C.c_int, [P, I32, P, P, P, P, P, P, P]),
        "gsk_features": (C.c_int, [P, I32, P, P, P, P]),
        "gsk_mlp_forward": (C.c_int, [I32, P, P, P, P, P]),
        "gsk_mlp_workspace_bytes": (C.c_size_t, [I32]),
        "gsk_mlp_train_step": (C.c_int, [I32, P, P, P, P, P, P, I32, C.c_float, P, P, P, P]),
        "gsk_set_sched_model": (C.c_int, [P, P, P]),
        "gsk_autotune": (C.c_int, [P, I32, P, P, I32, P, P, P]),
        "gsk_shift_trace": (C.c_int, [P, I32, P, I32, P, I32, P]),
        "gsk_find_mu": (C.c_int, [P, I32, P, I32, P, P, P, D, D, D, D, P, P]),
        "gsk_atom_pattern": (C.c_int, [P, P, P]),
        "gsk_icohp": (C.c_int, [P, I32, P, P, P, P]),
        "gsk_marnoldi": (C.c_int, [P, I32, P, I32, D, D, P, I32, P, P, P, P, P, P]),
        "gsk_mu_from_traces": (C.c_int, [P, I32, P, P, P, D, D, D, D, P, P]),
        "gsk_marnoldi_projected": (C.c_int, [P, P, I32, I32, P, I32, D, D, P, P, P, P, P, P]),
        "gsk_debug_selftest": (C.c_int, [P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def lib() -> C.CDLL:
    return _lib


def debug_selftest() -> tuple[int, int, int]:
    """gsk_debug_selftest: (status, code, index); GSK_ENOTSUP outside the bounds-checked build."""
    code = C.c_int32()
    idx = C.c_int64()
    rc = _lib.gsk_debug_selftest(C.byref(code), C.byref(idx))
    return int(rc), int(code.value), int(idx.value)


def strerror(code: int) -> str:
    return _lib.gsk_strerror(int(code)).decode()


def _check(code: int, where: str) -> None:
    if code != GSK_OK:
        raise GskError(code, where)


def _ptr(a) -> int:
    """Raw address of a NumPy array or a PyTorch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _per_column(v, n: int) -> np.ndarray:
    """A per-column FP64 array of n entries (a scalar is repeated; another length is refused)."""
    a = np.asarray(v, dtype=np.float64)
    if a.ndim == 0:
        a = np.full(n, float(a))
    if a.shape != (n,):
        raise ValueError(f"expected {n} per-column values, got shape {a.shape}")
    return np.ascontiguousarray(a)


def default_options(**kw) -> Options:
    o = Options()
    _lib.gsk_default_options(C.byref(o))
    names = {"precision": {"fp64": GSK_FP64, "mixed": GSK_MIXED, "mixed_df": GSK_MIXED_DF},
             "sched": {"fifo": GSK_SCHED_FIFO, "learned": GSK_SCHED_LEARNED},
             "spmm_kernel": {"auto": GSK_SPMM_AUTO, "gather": GSK_SPMM_GATHER, "staged": GSK_SPMM_STAGED}}
    for k, v in kw.items():
        if v is None:
            continue
        if k in names and isinstance(v, str):
            v = names[k][v]
        if k == "stream":
            v = getattr(v, "cuda_stream", v)
        setattr(o, k, v)
    return o


class Solver:
    """One libgsk handle: the pencil (A, B) and its orbital-block map."""

    def __init__(self, A, B, orb_offset, orb_count, pos=None):
        self._keep = []
        A = A.tocsr()
        B = B.tocsr()
        self._A = self._csr(A)
        self._B = self._csr(B)
        off = np.ascontiguousarray(orb_offset, dtype=np.int32)
        cnt = np.ascontiguousarray(orb_count, dtype=np.int8)
        ps = None if pos is None else np.ascontiguousarray(pos, dtype=np.float64)
        self._keep += [off, cnt, ps]
        om = _Orbmap(off.size, _ptr(off), _ptr(cnt), _ptr(ps))
        h = C.c_void_p()
        _check(_lib.gsk_create(C.byref(self._A), C.byref(self._B), C.byref(om), C.byref(h)), "gsk_create")
        self._h = h
        self._keep = []
        m = C.c_int32()
        nnz = C.c_int64()
        _check(_lib.gsk_dims(self._h, C.byref(m), C.byref(nnz)), "gsk_dims")
        self.M, self.nnz = int(m.value), int(nnz.value)
        self.n_atoms = int(off.size)

    def _csr(self, X) -> _Csr:
        rp = np.ascontiguousarray(X.indptr, dtype=np.int64)
        ci = np.ascontiguousarray(X.indices, dtype=np.int32)
        v = np.ascontiguousarray(X.data, dtype=np.float64)
        self._keep += [rp, ci, v]
        return _Csr(X.shape[0], _ptr(rp), _ptr(ci), _ptr(v))

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.gsk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_stats(self) -> dict:
        st = Stats()
        _check(_lib.gsk_last_stats(self._h, C.byref(st)), "gsk_last_stats")
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def features(self, cols, eta, feat) -> None:
        """Scheduler features of the columns into feat (device tensor, n x 16 float32)."""
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        eta = _per_column(eta, cols.size)
        _check(_lib.gsk_features(self._h, cols.size, _ptr(cols), _ptr(eta), _ptr(feat), None), "gsk_features")

    def set_sched_model(self, params, norm) -> None:
        p = np.ascontiguousarray(params, dtype=np.float32)
        nm = np.ascontiguousarray(norm, dtype=np.float32)
        _check(_lib.gsk_set_sched_model(self._h, _ptr(p), _ptr(nm)), "gsk_set_sched_model")

    def row_order(self) -> np.ndarray:
        out = np.empty(self.M, dtype=np.int32)
        _check(_lib.gsk_row_order(self._h, _ptr(out)), "gsk_row_order")
        return out

    def spmm(self, which: int, precision: int, W: int, X, Y, n_rep: int = 1, stream=None) -> None:
        s = getattr(stream, "cuda_stream", stream)
        _check(_lib.gsk_spmm(self._h, int(which), int(precision), int(W), _ptr(X), _ptr(Y), int(n_rep), s),
               "gsk_spmm")

    def pattern_offsets(self, cols) -> np.ndarray:
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        out = np.empty(cols.size + 1, dtype=np.int64)
        _check(_lib.gsk_pattern_offsets(self._h, cols.size, _ptr(cols), _ptr(out)), "gsk_pattern_offsets")
        return out

    def solve(self, z, cols, G, eta=None, options: Options | None = None, **kw):
        """Run gsk_solve. G: device tensor or host array of offsets[-1]*S complex128.

        Returns (iters, status, resid) as NumPy arrays.
        """
        z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
        zz = np.ascontiguousarray(np.stack([z.real, z.imag], axis=1).ravel())
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        e = None if eta is None else _per_column(eta, cols.size)
        opt = options if options is not None else default_options(**kw)
        n = cols.size
        iters = np.empty(n, dtype=np.int32)
        status = np.empty(n, dtype=np.int32)
        resid = np.empty(n, dtype=np.float64)
        rc = _lib.gsk_solve(self._h, z.size, _ptr(zz), _ptr(e), n, _ptr(cols), C.byref(opt), _ptr(G),
                            _ptr(iters), _ptr(status), _ptr(resid))
        _check(rc, "gsk_solve")
        return iters, status, resid

    def autotune(self, z, cols, eta=None, **kw) -> int:
        """gsk_autotune: pick and cache the lane width for this precision."""
        z = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
        zz = np.ascontiguousarray(np.stack([z.real, z.imag], axis=1).ravel())
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        e = None if eta is None else _per_column(eta, cols.size)
        opt = default_options(**kw)
        w = C.c_int32()
        _check(_lib.gsk_autotune(self._h, z.size, _ptr(zz), _ptr(e), cols.size, _ptr(cols), C.byref(opt),
                                 C.byref(w)), "gsk_autotune")
        return int(w.value)

    def autotune_result(self, precision) -> dict:
        """gsk_autotune_result: the last autotuner pick and its candidates."""
        if isinstance(precision, str):
            precision = {"fp64": GSK_FP64, "mixed": GSK_MIXED, "mixed_df": GSK_MIXED_DF}[precision]
        w, k, fc, n = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        cw = np.zeros(8, dtype=np.int32)
        ck = np.zeros(8, dtype=np.int32)
        cm = np.zeros(8, dtype=np.float64)
        _check(_lib.gsk_autotune_result(self._h, int(precision), C.byref(w), C.byref(k), C.byref(fc), C.byref(n),
                                        _ptr(cw), _ptr(ck), _ptr(cm)), "gsk_autotune_result")
        names = {GSK_SPMM_GATHER: "gather", GSK_SPMM_STAGED: "staged"}
        return {"W": int(w.value), "kernel": names.get(int(k.value), int(k.value)), "from_cache": bool(fc.value),
                "candidates": [{"W": int(cw[i]), "kernel": names.get(int(ck[i]), int(ck[i])),
                                "ms_per_step": float(cm[i])} for i in range(int(n.value))]}

    def density(self, G, eps, w, mu: float, kT: float, rho, n_elem: int, stream=None) -> None:
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        s = getattr(stream, "cuda_stream", stream)
        _check(_lib.gsk_density(self._h, int(n_elem), eps.size, _ptr(eps), _ptr(w), float(mu), float(kT),
                                _ptr(G), _ptr(rho), s), "gsk_density")

    def trace(self, cols, rho, which: int) -> float:
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        out = C.c_double()
        _check(_lib.gsk_trace(self._h, cols.size, _ptr(cols), _ptr(rho), int(which), C.byref(out)), "gsk_trace")
        return float(out.value)

    def shift_trace(self, cols, n_shifts: int, G, which: int) -> np.ndarray:
        """gsk_shift_trace: s_k = sum over the columns' patterns of Im G(z_k) X."""
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        s = np.zeros(int(n_shifts))
        _check(_lib.gsk_shift_trace(self._h, cols.size, _ptr(cols), int(n_shifts), _ptr(G), int(which),
                                    _ptr(s)), "gsk_shift_trace")
        return s

    def find_mu(self, cols, eps, w, G, kT: float, n_elec: float, mu_lo: float, mu_hi: float):
        """gsk_find_mu: (mu, N(mu)) with N(mu) = n_elec on [mu_lo, mu_hi]."""
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        mu, cnt = C.c_double(), C.c_double()
        _check(_lib.gsk_find_mu(self._h, cols.size, _ptr(cols), eps.size, _ptr(eps), _ptr(w), _ptr(G),
                                float(kT), float(n_elec), float(mu_lo), float(mu_hi), C.byref(mu),
                                C.byref(cnt)), "gsk_find_mu")
        return float(mu.value), float(cnt.value)

    def mu_from_traces(self, eps, w, s, kT: float, n_elec: float, mu_lo: float, mu_hi: float):
        """gsk_mu_from_traces: (mu, N(mu)) from per-shift traces s (host)."""
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        s = np.ascontiguousarray(s, dtype=np.float64)
        mu, cnt = C.c_double(), C.c_double()
        _check(_lib.gsk_mu_from_traces(self._h, eps.size, _ptr(eps), _ptr(w), _ptr(s), float(kT), float(n_elec),
                                       float(mu_lo), float(mu_hi), C.byref(mu), C.byref(cnt)), "gsk_mu_from_traces")
        return float(mu.value), float(cnt.value)

    def atom_pattern(self):
        """gsk_atom_pattern: (aptr, aidx) of the atom-pair pattern of A."""
        aptr = np.zeros(self.n_atoms + 1, dtype=np.int64)
        _check(_lib.gsk_atom_pattern(self._h, _ptr(aptr), None), "gsk_atom_pattern")
        aidx = np.zeros(max(int(aptr[-1]), 1), dtype=np.int32)
        _check(_lib.gsk_atom_pattern(self._h, _ptr(aptr), _ptr(aidx)), "gsk_atom_pattern")
        return aptr, aidx[:int(aptr[-1])]

    def marnoldi(self, cols, nu: int, mu: float, kT: float, rho, z=None, G=None):
        """gsk_marnoldi: multiple Arnoldi rho (and G at shifts z) on the columns'
        patterns; returns (ritz, weight, charge, rank) as host arrays."""
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        n = cols.size
        ritz = np.zeros(max(n * nu, 1))
        weight = np.zeros(max(n * nu, 1))
        charge = np.zeros(max(n * nu, 1))
        rank = np.zeros(max(n, 1), dtype=np.int32)
        if z is None:
            zz, S = None, 0
        else:
            zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128).view(np.float64))
            S = zz.size // 2
        _check(_lib.gsk_marnoldi(self._h, n, _ptr(cols), int(nu), float(mu), float(kT), _ptr(rho), S, _ptr(zz),
                                 _ptr(G), _ptr(ritz), _ptr(weight), _ptr(charge), _ptr(rank)), "gsk_marnoldi")
        sh = (n, nu)
        return ritz[:n * nu].reshape(sh), weight[:n * nu].reshape(sh), charge[:n * nu].reshape(sh), rank[:n]

    def marnoldi_projected(self, cols, kappa: int, nu: int, mu: float, kT: float, rho, box=None):
        """gsk_marnoldi_projected: multiple Arnoldi on each column's kappa-atom
        region; returns (ritz, weight, charge, rank, m_local) as host arrays."""
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        n = cols.size
        ritz = np.zeros(max(n * nu, 1))
        weight = np.zeros(max(n * nu, 1))
        charge = np.zeros(max(n * nu, 1))
        rank = np.zeros(max(n, 1), dtype=np.int32)
        m_local = np.zeros(max(n, 1), dtype=np.int32)
        bx = None if box is None else np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
        _check(_lib.gsk_marnoldi_projected(self._h, _ptr(bx), int(kappa), n, _ptr(cols), int(nu), float(mu),
                                           float(kT), _ptr(rho), _ptr(ritz), _ptr(weight), _ptr(charge),
                                           _ptr(rank), _ptr(m_local)), "gsk_marnoldi_projected")
        sh = (n, nu)
        return (ritz[:n * nu].reshape(sh), weight[:n * nu].reshape(sh), charge[:n * nu].reshape(sh), rank[:n],
                m_local[:n])

    def icohp(self, cols, rho, C_out, stream=None) -> None:
        """gsk_icohp: C_IJ on the atom pattern (device output C_out)."""
        cols = np.ascontiguousarray(cols, dtype=np.int32)
        s = getattr(stream, "cuda_stream", stream)
        _check(_lib.gsk_icohp(self._h, cols.size, _ptr(cols), _ptr(rho), _ptr(C_out), s), "gsk_icohp")


def density_noalloc(G, eps, w, mu: float, kT: float, rho, n_elem: int, stream=None) -> None:
    """gsk_density_noalloc: the density matrix without a handle or any device allocation."""
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    s = getattr(stream, "cuda_stream", stream)
    _check(_lib.gsk_density_noalloc(int(n_elem), eps.size, _ptr(eps), _ptr(w), float(mu), float(kT),
                                    _ptr(G), _ptr(rho), s), "gsk_density_noalloc")


MLP_IN, MLP_HIDDEN, MLP_NPARAM = 16, 64, 5313


def alu_peak(precision: int, n_rep: int = 5, stream=None) -> float:
    """Measured FMA throughput (TFLOP/s) of the current device: gsk_alu_peak."""
    out = C.c_double(0.0)
    s = getattr(stream, "cuda_stream", stream)
    _check(_lib.gsk_alu_peak(int(precision), int(n_rep), C.byref(out), s), "gsk_alu_peak")
    return float(out.value)


def mlp_forward(n: int, feat, norm, params, y, stream=None) -> None:
    s = getattr(stream, "cuda_stream", stream)
    _check(_lib.gsk_mlp_forward(int(n), _ptr(feat), _ptr(norm), _ptr(params), _ptr(y), s), "gsk_mlp_forward")


def mlp_workspace_bytes(n: int) -> int:
    return int(_lib.gsk_mlp_workspace_bytes(int(n)))


def mlp_train_step(n: int, feat, norm, target, params, m, v, t: int, lr: float, work, grad=None, loss=None,
                   stream=None) -> None:
    s = getattr(stream, "cuda_stream", stream)
    _check(_lib.gsk_mlp_train_step(int(n), _ptr(feat), _ptr(norm), _ptr(target), _ptr(params), _ptr(m), _ptr(v),
                                   int(t), float(lr), _ptr(grad), _ptr(loss), _ptr(work), s), "gsk_mlp_train_step")


def from_system(sys_, pos=True) -> Solver:
    """Solver for a synthetic System (see synthetic.make_system)."""
    return Solver(sys_.A, sys_.B, sys_.orb_offset, sys_.orb_count, sys_.pos if pos else None)
