"""ctypes binding of ``liblieclosure.so`` (argument marshalling only).

Every function here forwards to the C ABI of ``include/lieclosure.h`` /
``include/lieclosure_kernels.h`` under the same name; all computation runs in
the library's CUDA kernels.  The library is loaded on first use; if it is
missing (not built) the call raises ``LibraryNotBuilt`` -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblieclosure.so")

LC_OK = 0
LC_ERR_ARG = -1
LC_ERR_NOT_ANTIHERMITIAN = -2
LC_ERR_NONFINITE = -3
LC_ERR_CAPACITY = -4
LC_ERR_CUDA = -5
LC_ERR_OOM = -6
LC_ERR_TIMEOUT = -7
LC_ERR_TOO_LARGE = -8

LC_PREC_FP64 = 0
LC_PREC_MIXED_BF16X3 = 1
PRECISIONS = {"fp64": LC_PREC_FP64, "mixed": LC_PREC_MIXED_BF16X3}

LC_TOL_RELATIVE = 0
LC_TOL_ABSOLUTE = 1
TOL_MODES = {"relative": LC_TOL_RELATIVE, "absolute": LC_TOL_ABSOLUTE}

# every symbol the public headers declare
EXPORTED = ["lc_default_options", "lc_status_string", "lc_version", "lie_closure", "lie_closure_dev",
            "lie_closure_batched", "lie_closure_batched_dev", "lie_closure_alg2", "lie_closure_alg2_dev", "lie_closure_alg3",
            "lie_closure_alg3_dev", "lie_closure_resume",
            "lie_closure_resume_dev", "lie_closure_pauli", "lie_closure_pauli_dev", "lc_split_gemm_f32",
            "lc_split_gemm_f32_noalloc", "lc_gemm_f64_tc"]


class LibraryNotBuilt(RuntimeError):
    pass


class LieClosureError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lie_closure failed: {msg} (status {status})")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("eta_abs", ctypes.c_double), ("tau_screen", ctypes.c_double),
                ("block_k", ctypes.c_int), ("block_k_growth", ctypes.c_int), ("saturation_exit", ctypes.c_int), ("spin_cap", ctypes.c_longlong),
                ("max_candidates", ctypes.c_longlong), ("verbose", ctypes.c_int), ("profile", ctypes.c_int),
                ("fault_inject", ctypes.c_int), ("tol_mode", ctypes.c_int), ("autotune", ctypes.c_int),
                ("ortho_check", ctypes.c_int), ("screen_kappa", ctypes.c_double),
                ("accept_kernel", ctypes.c_int), ("fp64_first_pass", ctypes.c_int),
                ("accept_gemm", ctypes.c_int)]


class Report(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_longlong), ("brackets_checked", ctypes.c_longlong),
                ("generators_checked", ctypes.c_longlong), ("n_nonzero", ctypes.c_longlong),
                ("n_flagged", ctypes.c_longlong), ("n_blocks", ctypes.c_longlong),
                ("cursor_l", ctypes.c_longlong), ("cursor_m", ctypes.c_longlong),
                ("t_total_s", ctypes.c_double), ("t_last_accept_s", ctypes.c_double),
                ("min_acc_rel_res", ctypes.c_double), ("max_rej_rel_res", ctypes.c_double),
                ("tau_screen", ctypes.c_double), ("max_screen_rej_rel_res", ctypes.c_double),
                ("kernel_launches", ctypes.c_longlong), ("gemm_launches", ctypes.c_longlong),
                ("gemm_flops", ctypes.c_double), ("t_phase_s", ctypes.c_double * 6),
                ("precision", ctypes.c_int), ("status", ctypes.c_int),
                ("n_gray", ctypes.c_longlong), ("eps_screen", ctypes.c_double),
                ("min_acc_screen_rel_res", ctypes.c_double), ("ortho_defect", ctypes.c_double),
                ("ortho_rows", ctypes.c_longlong), ("block_k_used", ctypes.c_int),
                ("block_k_growth_used", ctypes.c_int), ("gemm_tile_n", ctypes.c_int), ("gemm_tile_k", ctypes.c_int),
                ("autotuned", ctypes.c_int), ("autotune_trials", ctypes.c_int),
                ("accept_wide_launches", ctypes.c_longlong), ("screen_pass1_blocks", ctypes.c_longlong),
                ("accept_tc_gemms", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if name == "t_phase_s" else v
        return out


_lib = None


def lib():
    """The loaded library (raises LibraryNotBuilt when it is absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LibraryNotBuilt(f"{LIB_PATH} is missing: run paper_2506_01120_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        c_p = ctypes.c_void_p
        L.lc_default_options.argtypes = [ctypes.POINTER(Options)]
        L.lc_default_options.restype = None
        L.lc_status_string.argtypes = [ctypes.c_int]
        L.lc_status_string.restype = ctypes.c_char_p
        L.lc_version.argtypes = []
        L.lc_version.restype = ctypes.c_char_p
        L.lie_closure.argtypes = [c_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, c_p,
                                  ctypes.POINTER(ctypes.c_longlong), ctypes.c_longlong,
                                  ctypes.POINTER(Options), ctypes.POINTER(Report)]
        L.lie_closure.restype = ctypes.c_int
        L.lie_closure_dev.argtypes = L.lie_closure.argtypes + [c_p]
        L.lie_closure_dev.restype = ctypes.c_int
        L.lie_closure_batched.argtypes = [ctypes.c_int, ctypes.POINTER(c_p), ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.POINTER(c_p),
                                          ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Options),
                                          ctypes.POINTER(Report)]
        L.lie_closure_batched.restype = ctypes.c_int
        L.lie_closure_batched_dev.argtypes = L.lie_closure_batched.argtypes + [c_p]
        L.lie_closure_batched_dev.restype = ctypes.c_int
        L.lie_closure_alg2.argtypes = L.lie_closure.argtypes
        L.lie_closure_alg2.restype = ctypes.c_int
        L.lie_closure_alg2_dev.argtypes = L.lie_closure_dev.argtypes
        L.lie_closure_alg2_dev.restype = ctypes.c_int
        L.lie_closure_alg3.argtypes = [c_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, c_p, c_p,
                                       ctypes.POINTER(ctypes.c_longlong), ctypes.c_longlong,
                                       ctypes.POINTER(Options), ctypes.POINTER(Report)]
        L.lie_closure_alg3.restype = ctypes.c_int
        L.lie_closure_alg3_dev.argtypes = L.lie_closure_alg3.argtypes + [c_p]
        L.lie_closure_alg3_dev.restype = ctypes.c_int
        L.lie_closure_resume.argtypes = [c_p, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_longlong, ctypes.c_int,
                                         ctypes.c_double, c_p, ctypes.POINTER(ctypes.c_longlong), ctypes.c_longlong,
                                         ctypes.POINTER(Options), ctypes.POINTER(Report)]
        L.lie_closure_resume.restype = ctypes.c_int
        L.lie_closure_resume_dev.argtypes = L.lie_closure_resume.argtypes + [c_p]
        L.lie_closure_resume_dev.restype = ctypes.c_int
        L.lie_closure_pauli.argtypes = [c_p, c_p, c_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, c_p, c_p, c_p,
                                        ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong), ctypes.c_longlong,
                                        ctypes.POINTER(Options), ctypes.POINTER(Report)]
        L.lie_closure_pauli.restype = ctypes.c_int
        L.lie_closure_pauli_dev.argtypes = L.lie_closure_pauli.argtypes + [c_p]
        L.lie_closure_pauli_dev.restype = ctypes.c_int
        L.lc_split_gemm_f32.argtypes = [c_p, c_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_p, c_p]
        L.lc_split_gemm_f32.restype = ctypes.c_int
        L.lc_split_gemm_f32_noalloc.argtypes = L.lc_split_gemm_f32.argtypes
        L.lc_gemm_f64_tc.argtypes = L.lc_split_gemm_f32.argtypes
        L.lc_gemm_f64_tc.restype = ctypes.c_int
        L.lc_split_gemm_f32_noalloc.restype = ctypes.c_int
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().lc_status_string(int(status)).decode()


def version() -> str:
    return lib().lc_version().decode()


def make_options(precision="mixed", **kw) -> Options:
    o = Options()
    lib().lc_default_options(ctypes.byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    if isinstance(kw.get("tol_mode"), str):
        kw["tol_mode"] = TOL_MODES[kw["tol_mode"]]
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


@dataclass
class ClosureResult:
    dim: int
    basis: np.ndarray | None
    status: int
    report: dict


def _check(status: int, check: bool):
    if check and status != LC_OK:
        raise LieClosureError(status, status_string(status))


def lie_closure(generators, tol: float, max_dim: int | None = None, return_basis: bool = True,
                check: bool = True, precision="mixed", **opts) -> ClosureResult:
    """Algorithm 4 on host arrays: ``generators`` is (k, d, d) complex128."""
    g = np.ascontiguousarray(generators, dtype=np.complex128)
    if g.ndim != 3 or g.shape[1] != g.shape[2]:
        raise ValueError("generators must have shape (k, d, d)")
    k, d, _ = g.shape
    cap = int(max_dim) if max_dim is not None else d * d
    basis = np.zeros((cap, d, d), dtype=np.complex128) if return_basis else None
    dim = ctypes.c_longlong(0)
    rep = Report()
    o = make_options(precision, **opts)
    st = lib().lie_closure(g.ctypes.data, k, d, float(tol), basis.ctypes.data if basis is not None else None,
                           ctypes.byref(dim), cap, ctypes.byref(o), ctypes.byref(rep))
    _check(st, check)
    n = int(dim.value)
    return ClosureResult(n, basis[:n] if basis is not None else None, st, rep.as_dict())


def lie_closure_alg2(generators, tol: float, max_dim: int | None = None, check: bool = True,
                     **opts) -> ClosureResult:
    """Algorithm 2 (matrix-inversion method) on host arrays; basis = unit-norm B."""
    g = np.ascontiguousarray(generators, dtype=np.complex128)
    if g.ndim != 3 or g.shape[1] != g.shape[2]:
        raise ValueError("generators must have shape (k, d, d)")
    k, d, _ = g.shape
    cap = int(max_dim) if max_dim is not None else d * d
    basis = np.zeros((cap, d, d), dtype=np.complex128)
    dim = ctypes.c_longlong(0)
    rep = Report()
    o = make_options("fp64", **opts)
    st = lib().lie_closure_alg2(g.ctypes.data, k, d, float(tol), basis.ctypes.data, ctypes.byref(dim), cap,
                                ctypes.byref(o), ctypes.byref(rep))
    _check(st, check)
    n = int(dim.value)
    return ClosureResult(n, basis[:n], st, rep.as_dict())


def lie_closure_resume(basis, cursor, tol: float, max_dim: int | None = None, check: bool = True,
                       precision="mixed", **opts) -> ClosureResult:
    """Continue Algorithm 4 from (basis, (l, m)) returned by an earlier call."""
    b = np.ascontiguousarray(basis, dtype=np.complex128)
    n, d, _ = b.shape
    cap = int(max_dim) if max_dim is not None else d * d
    out = np.zeros((cap, d, d), dtype=np.complex128)
    dim = ctypes.c_longlong(0)
    rep = Report()
    o = make_options(precision, **opts)
    st = lib().lie_closure_resume(b.ctypes.data, n, int(cursor[0]), int(cursor[1]), d, float(tol), out.ctypes.data,
                                  ctypes.byref(dim), cap, ctypes.byref(o), ctypes.byref(rep))
    _check(st, check)
    k = int(dim.value)
    return ClosureResult(k, out[:k], st, rep.as_dict())


def lie_closure_alg3(generators, tol: float, max_dim: int | None = None, check: bool = True,
                     precision="mixed", **opts):
    """Algorithm 3 on host arrays: returns (B, V, status, report) with B the kept
    generators and nested brackets and V the orthonormal basis."""
    g = np.ascontiguousarray(generators, dtype=np.complex128)
    if g.ndim != 3 or g.shape[1] != g.shape[2]:
        raise ValueError("generators must have shape (k, d, d)")
    k, d, _ = g.shape
    cap = int(max_dim) if max_dim is not None else d * d
    B = np.zeros((cap, d, d), dtype=np.complex128)
    V = np.zeros((cap, d, d), dtype=np.complex128)
    dim = ctypes.c_longlong(0)
    rep = Report()
    o = make_options(precision, **opts)
    st = lib().lie_closure_alg3(g.ctypes.data, k, d, float(tol), B.ctypes.data, V.ctypes.data, ctypes.byref(dim),
                                cap, ctypes.byref(o), ctypes.byref(rep))
    _check(st, check)
    n = int(dim.value)
    return B[:n], V[:n], st, rep.as_dict()


def lie_closure_dev(generators, tol: float, max_dim: int | None = None, basis_out=None, stream=None,
                    check: bool = True, precision="mixed", **opts) -> ClosureResult:
    """Algorithm 4 on device tensors (torch complex128 on the current CUDA device).

    ``basis_out`` (optional) is a (max_dim, d, d) complex128 device tensor that
    receives the basis; ``stream`` a torch.cuda.Stream (default: current)."""
    import torch
    g = generators
    if not (g.is_cuda and g.dtype == torch.complex128 and g.is_contiguous() and g.dim() == 3):
        raise ValueError("generators must be a contiguous (k, d, d) complex128 CUDA tensor")
    k, d, _ = g.shape
    cap = int(max_dim) if max_dim is not None else d * d
    if basis_out is not None:
        if not (basis_out.is_cuda and basis_out.dtype == torch.complex128 and basis_out.is_contiguous()
                and basis_out.shape[0] >= cap and tuple(basis_out.shape[1:]) == (d, d)):
            raise ValueError("basis_out must be a contiguous (max_dim, d, d) complex128 CUDA tensor")
    s = stream if stream is not None else torch.cuda.current_stream()
    dim = ctypes.c_longlong(0)
    rep = Report()
    o = make_options(precision, **opts)
    st = lib().lie_closure_dev(g.data_ptr(), k, d, float(tol),
                               basis_out.data_ptr() if basis_out is not None else None, ctypes.byref(dim), cap,
                               ctypes.byref(o), ctypes.byref(rep), ctypes.c_void_p(s.cuda_stream))
    _check(st, check)
    return ClosureResult(int(dim.value), None, st, rep.as_dict())


def lie_closure_resume_dev(basis, n_in: int, cursor, tol: float, max_dim: int | None = None, basis_out=None,
                           stream=None, check: bool = True, precision="mixed", **opts) -> ClosureResult:
    """``lie_closure_resume`` on device tensors: ``basis`` is a contiguous
    (>= n_in, d, d) complex128 CUDA tensor whose first n_in elements are the
    saved basis; ``basis_out`` (optional) a (max_dim, d, d) device tensor."""
    import torch
    b = basis
    if not (b.is_cuda and b.dtype == torch.complex128 and b.is_contiguous() and b.dim() == 3 and b.shape[0] >= n_in):
        raise ValueError("basis must be a contiguous (>= n_in, d, d) complex128 CUDA tensor")
    d = b.shape[1]
    cap = int(max_dim) if max_dim is not None else d * d
    if basis_out is not None:
        if not (basis_out.is_cuda and basis_out.dtype == torch.complex128 and basis_out.is_contiguous()
                and basis_out.shape[0] >= cap and tuple(basis_out.shape[1:]) == (d, d)):
            raise ValueError("basis_out must be a contiguous (max_dim, d, d) complex128 CUDA tensor")
    s = stream if stream is not None else torch.cuda.current_stream()
    dim = ctypes.c_longlong(0)
    rep = Report()
    o = make_options(precision, **opts)
    st = lib().lie_closure_resume_dev(b.data_ptr(), int(n_in), int(cursor[0]), int(cursor[1]), d, float(tol),
                                      basis_out.data_ptr() if basis_out is not None else None, ctypes.byref(dim),
                                      cap, ctypes.byref(o), ctypes.byref(rep), ctypes.c_void_p(s.cuda_stream))
    _check(st, check)
    return ClosureResult(int(dim.value), None, st, rep.as_dict())


def lie_closure_batched(generator_sets, tol: float, max_dims=None, return_basis: bool = False,
                        precision="mixed", **opts):
    """Algorithm 4 on many independent sets; returns (dims, statuses, bases, reports)."""
    sets = [np.ascontiguousarray(g, dtype=np.complex128) for g in generator_sets]
    n = len(sets)
    ks = (ctypes.c_int * n)(*[g.shape[0] for g in sets])
    ds = (ctypes.c_int * n)(*[g.shape[1] for g in sets])
    caps = [int(max_dims[i]) if max_dims is not None else sets[i].shape[1] ** 2 for i in range(n)]
    cap_arr = (ctypes.c_longlong * n)(*caps)
    gptr = (ctypes.c_void_p * n)(*[g.ctypes.data for g in sets])
    bases = [np.zeros((caps[i], sets[i].shape[1], sets[i].shape[1]), dtype=np.complex128) for i in range(n)] \
        if return_basis else None
    bptr = (ctypes.c_void_p * n)(*[b.ctypes.data for b in bases]) if bases is not None else None
    dims = (ctypes.c_longlong * n)()
    stat = (ctypes.c_int * n)()
    reps = (Report * n)()
    o = make_options(precision, **opts)
    lib().lie_closure_batched(n, gptr, ks, ds, float(tol), bptr, cap_arr, dims, stat, ctypes.byref(o), reps)
    dims_l = [int(x) for x in dims]
    out_b = [bases[i][:dims_l[i]] for i in range(n)] if bases is not None else None
    return dims_l, [int(x) for x in stat], out_b, [r.as_dict() for r in reps]


def lie_closure_batched_dev(generator_sets, tol: float, max_dims=None, bases=None, stream=None,
                            precision="mixed", **opts):
    """Algorithm 4 on many independent sets held on the device: each element of
    ``generator_sets`` is a contiguous (k, d, d) complex128 CUDA tensor;
    ``bases`` (optional) a list of (max_dim, d, d) complex128 CUDA tensors (or
    None entries).  Returns (dims, statuses, reports)."""
    import torch
    n = len(generator_sets)
    for g in generator_sets:
        if not (g.is_cuda and g.dtype == torch.complex128 and g.is_contiguous() and g.dim() == 3):
            raise ValueError("every generator set must be a contiguous (k, d, d) complex128 CUDA tensor")
    ks = (ctypes.c_int * n)(*[g.shape[0] for g in generator_sets])
    ds = (ctypes.c_int * n)(*[g.shape[1] for g in generator_sets])
    caps = [int(max_dims[i]) if max_dims is not None else generator_sets[i].shape[1] ** 2 for i in range(n)]
    cap_arr = (ctypes.c_longlong * n)(*caps)
    gptr = (ctypes.c_void_p * n)(*[g.data_ptr() for g in generator_sets])
    bptr = None
    if bases is not None:
        for i, b in enumerate(bases):
            if b is not None and not (b.is_cuda and b.dtype == torch.complex128 and b.is_contiguous()
                                      and b.shape[0] >= caps[i] and tuple(b.shape[1:]) == tuple(generator_sets[i].shape[1:])):
                raise ValueError("bases[i] must be a contiguous (max_dim, d, d) complex128 CUDA tensor")
        bptr = (ctypes.c_void_p * n)(*[b.data_ptr() if b is not None else None for b in bases])
    dims = (ctypes.c_longlong * n)()
    stat = (ctypes.c_int * n)()
    reps = (Report * n)()
    o = make_options(precision, **opts)
    s = stream if stream is not None else torch.cuda.current_stream()
    lib().lie_closure_batched_dev(n, gptr, ks, ds, float(tol), bptr, cap_arr, dims, stat, ctypes.byref(o), reps,
                                  ctypes.c_void_p(s.cuda_stream))
    return [int(x) for x in dims], [int(x) for x in stat], [r.as_dict() for r in reps]


@dataclass
class PauliClosureResult:
    """Basis of a Pauli-sum closure: element i is i * sum_t coefs[t] P(strings[t])
    over t in [offsets[i], offsets[i+1]); strings packed as x | (z << 32)."""
    dim: int
    strings: np.ndarray
    coefs: np.ndarray
    offsets: np.ndarray
    status: int
    report: dict

    def element(self, i: int) -> list[tuple[int, float]]:
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        return list(zip(self.strings[a:b].tolist(), self.coefs[a:b].tolist()))


def lie_closure_pauli(strings, coefs, offsets, n_qubits: int, tol: float, max_dim: int | None = None,
                      term_capacity: int | None = None, check: bool = True, **opts) -> PauliClosureResult:
    """Algorithm 4 on sparse Pauli-sum generators (host arrays): generator j is
    i * sum_t coefs[t] P(strings[t]) over t in [offsets[j], offsets[j+1])."""
    st_ = np.ascontiguousarray(strings, dtype=np.uint64)
    cf = np.ascontiguousarray(coefs, dtype=np.float64)
    of = np.ascontiguousarray(offsets, dtype=np.int64)
    if st_.shape != cf.shape or of.ndim != 1 or of.size < 2 or int(of[-1]) != st_.size:
        raise ValueError("strings/coefs must be equal-length 1-d arrays and offsets their k+1 bounds")
    k = of.size - 1
    cap = int(max_dim) if max_dim is not None else min(4 ** n_qubits, 1 << 16)
    tcap = int(term_capacity) if term_capacity is not None else max(min(cap * 4 ** n_qubits, 1 << 22), 1024)
    out_s = np.zeros(tcap, dtype=np.uint64)
    out_c = np.zeros(tcap, dtype=np.float64)
    out_o = np.zeros(cap + 1, dtype=np.int64)
    dim = ctypes.c_longlong(0)
    rep = Report()
    o = make_options("fp64", **opts)
    stt = lib().lie_closure_pauli(st_.ctypes.data, cf.ctypes.data, of.ctypes.data, k, int(n_qubits), float(tol),
                                  out_s.ctypes.data, out_c.ctypes.data, out_o.ctypes.data, tcap, ctypes.byref(dim),
                                  cap, ctypes.byref(o), ctypes.byref(rep))
    _check(stt, check)
    n = int(dim.value)
    nt = int(out_o[n]) if n > 0 else 0
    return PauliClosureResult(n, out_s[:nt], out_c[:nt], out_o[:n + 1], stt, rep.as_dict())


def lie_closure_pauli_dev(strings, coefs, offsets, n_qubits: int, tol: float, max_dim: int,
                          term_capacity: int, basis_strings=None, basis_coefs=None, basis_offsets=None,
                          stream=None, check: bool = True, **opts) -> ClosureResult:
    """As ``lie_closure_pauli`` on torch CUDA tensors (int64 strings, float64
    coefs, int64 offsets); the optional outputs are device tensors of
    term_capacity / term_capacity / max_dim + 1 entries."""
    import torch
    for t in (strings, coefs, offsets):
        if not (t.is_cuda and t.is_contiguous()):
            raise ValueError("inputs must be contiguous CUDA tensors")
    k = offsets.numel() - 1
    s = stream if stream is not None else torch.cuda.current_stream()
    dim = ctypes.c_longlong(0)
    rep = Report()
    o = make_options("fp64", **opts)
    ptr = lambda t: t.data_ptr() if t is not None else None
    st = lib().lie_closure_pauli_dev(strings.data_ptr(), coefs.data_ptr(), offsets.data_ptr(), k, int(n_qubits),
                                     float(tol), ptr(basis_strings), ptr(basis_coefs), ptr(basis_offsets),
                                     int(term_capacity), ctypes.byref(dim), int(max_dim), ctypes.byref(o),
                                     ctypes.byref(rep), ctypes.c_void_p(s.cuda_stream))
    _check(st, check)
    return ClosureResult(int(dim.value), None, st, rep.as_dict())


def pauli_label(string: int, n_qubits: int) -> str:
    """Letters of a packed string (qubit 1 first)."""
    x, z = int(string) & 0xFFFFFFFF, int(string) >> 32
    return "".join("IXZY"[((x >> q) & 1) + 2 * ((z >> q) & 1)] for q in range(n_qubits))


def lc_split_gemm_f32(A, B, stream=None):
    """D = A B^T (torch FP32 CUDA tensors) through the split-BF16 tcgen05 GEMM."""
    import torch
    if not (A.is_cuda and B.is_cuda and A.dtype == torch.float32 and B.dtype == torch.float32):
        raise ValueError("A and B must be float32 CUDA tensors")
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N, K2 = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    st = lib().lc_split_gemm_f32(A.data_ptr(), B.data_ptr(), M, N, K, D.data_ptr(), ctypes.c_void_p(s.cuda_stream))
    _check(st, True)
    return D


def lc_gemm_f64_tc(A, B, stream=None):
    """C = A B^T (torch FP64 CUDA tensors) to FP64 accuracy through the sliced
    BF16 tensor-core GEMM."""
    import torch
    if not (A.is_cuda and B.is_cuda and A.dtype == torch.float64 and B.dtype == torch.float64):
        raise ValueError("A and B must be float64 CUDA tensors")
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N, K2 = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    C = torch.empty((M, N), dtype=torch.float64, device=A.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    st = lib().lc_gemm_f64_tc(A.data_ptr(), B.data_ptr(), M, N, K, C.data_ptr(), ctypes.c_void_p(s.cuda_stream))
    _check(st, True)
    return C


def lc_split_gemm_f32_noalloc(A, B, stream=None, check: bool = True):
    """D = A B^T like ``lc_split_gemm_f32``, with the library's fixed device
    scratch array instead of a per-call allocation (for callers that cannot let
    the library allocate).  Returns (D, status); D is allocated here by torch,
    the library itself allocates nothing."""
    import torch
    if not (A.is_cuda and B.is_cuda and A.dtype == torch.float32 and B.dtype == torch.float32):
        raise ValueError("A and B must be float32 CUDA tensors")
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N, K2 = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    s = stream if stream is not None else torch.cuda.current_stream()
    st = lib().lc_split_gemm_f32_noalloc(A.data_ptr(), B.data_ptr(), M, N, K, D.data_ptr(),
                                         ctypes.c_void_p(s.cuda_stream))
    _check(st, check)
    return D, st
