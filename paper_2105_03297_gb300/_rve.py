"""ctypes binding of ``librve.so`` (the C ABI declared in include/rve.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Loading fails loudly when the library is missing; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librve.so")

RVE_OK = 0
RVE_ERR_ARG = -1
RVE_ERR_UNSUPPORTED_SIZE = -2
RVE_ERR_CUDA = -3
RVE_ERR_OOM = -4
RVE_ERR_NOT_CONVERGED = -5
RVE_ERR_NONFINITE = -6
RVE_ERR_TIMEOUT = -7
RVE_ERR_SCRATCH_LIMIT = -8
RVE_FP64, RVE_MIXED = 0, 1
RVE_F32, RVE_F64 = 0, 1
RVE_PTR_HOST, RVE_PTR_DEVICE = 0, 1


class rve_info(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("refine_steps", C.c_int32), ("status", C.c_int32),
                ("reserved", C.c_int32), ("rel_residual", C.c_double), ("cg_rel_residual", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


# name -> (restype, argtypes), one entry per function of include/rve.h
SIGNATURES = {
    "rve_error_string": (C.c_char_p, [C.c_int]),
    "rve_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                             C.c_int, C.c_void_p]),
    "rve_destroy": (C.c_int, [C.c_void_p]),
    "rve_set_material": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int]),
    "rve_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_double, C.c_int,
                            C.POINTER(rve_info)]),
    "rve_mean_stress": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "rve_effective_tangent": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "rve_energy_tangent": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "rve_adjoint": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_double, C.c_int, C.c_void_p, C.c_int]),
    "rve_get_strain": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "rve_apply_operator": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "rve_schedule": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_float)]),
    "rve_set_schedule": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "rve_test_stall_copies": (C.c_int, [C.c_void_p, C.c_int]),
    "rve_set_operator_form": (C.c_int, [C.c_void_p, C.c_int]),
    "rve_set_derivative": (C.c_int, [C.c_void_p, C.c_int]),
    "rve_set_kinematics": (C.c_int, [C.c_void_p, C.c_int]),
    "rve_solve_finite": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_double, C.c_int, C.c_int,
                                   C.POINTER(rve_info)]),
    "rve_mean_piola": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "rve_get_deformation": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "rve_derivative": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "rve_operator_form": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
    "rve_timing_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "rve_timing_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "rve_apply_operator_2d_static": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_void_p,
                                               C.c_double, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "rve_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.POINTER(C.c_int64), C.c_int,
                                   C.c_double]),
    "rve_batch_destroy": (C.c_int, [C.c_void_p]),
    "rve_batch_set_material": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int]),
    "rve_batch_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_double, C.c_int,
                                  C.POINTER(rve_info)]),
    "rve_batch_mean_stress": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "rve_batch_effective_tangent": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "rve_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int),
                            C.POINTER(C.c_int)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load librve.so and declare its prototypes (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class RveError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = load().rve_error_string(code).decode()
        super().__init__(f"{where}: {msg} ({code})")


def _check(code, where, allow=()):
    if code != RVE_OK and code not in allow:
        raise RveError(code, where)
    return code


def _buffer(arr, dtype, count, name):
    """(pointer, flag, keepalive) of a buffer of which the library reads or
    writes ``count`` elements of ``dtype``: a C-contiguous numpy array (host)
    or a contiguous torch tensor (device or host).  A wrong element type, size
    or layout raises here, before the library touches the memory."""
    dtype = np.dtype(dtype)
    if isinstance(arr, np.ndarray):
        if arr.dtype != dtype:
            raise TypeError(f"{name}: dtype {arr.dtype}, expected {dtype}")
        if not arr.flags.c_contiguous:
            raise ValueError(f"{name}: array must be C-contiguous")
        if arr.size != count:
            raise ValueError(f"{name}: {arr.size} elements, expected {count}")
        return arr.ctypes.data_as(C.c_void_p), RVE_PTR_HOST, arr
    import torch
    if isinstance(arr, torch.Tensor):
        want = {np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64}[dtype]
        if arr.dtype != want:
            raise TypeError(f"{name}: dtype {arr.dtype}, expected {want}")
        if not arr.is_contiguous():
            raise ValueError(f"{name}: tensor must be contiguous")
        if arr.numel() != count:
            raise ValueError(f"{name}: {arr.numel()} elements, expected {count}")
        flag = RVE_PTR_DEVICE if arr.is_cuda else RVE_PTR_HOST
        return C.c_void_p(arr.data_ptr()), flag, arr
    raise TypeError(f"{name}: expected a numpy array or a torch tensor, got {type(arr).__name__}")


class RVE:
    """A periodic RVE solver handle (one grid, one precision)."""

    def __init__(self, n, precision="fp64", length=None, stream=None):
        lib = load()
        self.n = tuple(int(v) for v in n)
        self.dim = len(self.n)
        self.precision = precision
        nn = (C.c_int64 * self.dim)(*self.n)
        ln = (C.c_double * self.dim)(*length) if length is not None else None
        h = C.c_void_p()
        prec = RVE_MIXED if precision == "mixed" else RVE_FP64
        st = C.c_void_p(stream) if stream is not None else None
        _check(lib.rve_create(C.byref(h), self.dim, nn, ln, prec, st), "rve_create")
        self.h = h
        N = C.c_int64(); m = C.c_int(); ns = C.c_int(); d = C.c_int()
        _check(lib.rve_sizes(h, C.byref(N), C.byref(m), C.byref(ns), C.byref(d)), "rve_sizes")
        self.N, self.m, self.ns = N.value, m.value, ns.value
        self.inner_dtype = np.float32 if precision == "mixed" else np.float64
        self.L = 0

    def close(self):
        if getattr(self, "h", None):
            load().rve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_material(self, E, nu):
        """Per-voxel Young's moduli E (N values, x fastest: numpy array or torch
        tensor, float32 or float64) and the Poisson ratio nu."""
        if isinstance(E, np.ndarray):
            E = np.ascontiguousarray(E)
            if E.dtype not in (np.float32, np.float64):
                E = E.astype(np.float64)
            dtype = E.dtype
        else:
            import torch
            if not isinstance(E, torch.Tensor) or E.dtype not in (torch.float32, torch.float64):
                raise TypeError("E: expected a float32 or float64 numpy array or torch tensor")
            dtype = np.float32 if E.dtype == torch.float32 else np.float64
        p, flag, _keep = _buffer(E, dtype, self.N, "E")
        dt = RVE_F32 if np.dtype(dtype) == np.float32 else RVE_F64
        _check(load().rve_set_material(self.h, p, dt, float(nu), flag), "rve_set_material")

    def solve(self, E_macro, rel_tol=1e-10, max_iter=5000):
        Em = np.ascontiguousarray(np.atleast_2d(np.asarray(E_macro, dtype=np.float64)))
        if Em.ndim != 2 or Em.shape[1] != self.ns:
            raise ValueError(f"E_macro: shape {Em.shape}, expected (L, {self.ns})")
        L = Em.shape[0]
        info = (rve_info * L)()
        code = load().rve_solve(self.h, Em.ctypes.data_as(C.POINTER(C.c_double)), L, float(rel_tol),
                                int(max_iter), info)
        _check(code, "rve_solve", allow=(RVE_ERR_NOT_CONVERGED,))
        self.L = L
        return code, [i.as_dict() for i in info]

    def mean_stress(self):
        S = np.zeros((self.L, self.ns))
        _check(load().rve_mean_stress(self.h, S.ctypes.data_as(C.POINTER(C.c_double))), "rve_mean_stress")
        return S

    def effective_tangent(self):
        Cm = np.zeros((self.ns, self.ns))
        _check(load().rve_effective_tangent(self.h, Cm.ctypes.data_as(C.POINTER(C.c_double))),
               "rve_effective_tangent")
        return Cm

    def energy_tangent(self):
        """Energy form (E_a + eps~_a) : C : (E_b + eps~_b), averaged, for the solved load cases."""
        Ce = np.zeros((self.L, self.L))
        _check(load().rve_energy_tangent(self.h, Ce.ctypes.data_as(C.POINTER(C.c_double))), "rve_energy_tangent")
        return Ce

    def adjoint(self, W, rel_tol=1e-10, max_iter=5000, out=None):
        W = np.ascontiguousarray(np.asarray(W, dtype=np.float64))
        if W.shape != (self.ns, self.ns):
            raise ValueError(f"W: shape {W.shape}, expected ({self.ns}, {self.ns})")
        if out is None:
            out = np.zeros(self.N)
        p, flag, _keep = _buffer(out, np.float64, self.N, "out")
        code = load().rve_adjoint(self.h, W.ctypes.data_as(C.POINTER(C.c_double)), float(rel_tol),
                                  int(max_iter), p, flag)
        _check(code, "rve_adjoint", allow=(RVE_ERR_NOT_CONVERGED,))
        return out

    def get_strain(self, load_case, out=None):
        if out is None:
            out = np.zeros((self.m, self.N))
        p, flag, _keep = _buffer(out, np.float64, self.m * self.N, "out")
        _check(load().rve_get_strain(self.h, int(load_case), p, flag), "rve_get_strain")
        return out

    SCHED_PASSES, SCHED_VARIANTS = 4, 7

    def schedule(self):
        """(variants [pass A, pass E, split of pass C's axis, split of the y axis],
        candidate times [4][7] in ms)."""
        v = (C.c_int * self.SCHED_PASSES)()
        t = (C.c_float * (self.SCHED_PASSES * self.SCHED_VARIANTS))()
        _check(load().rve_schedule(self.h, v, t), "rve_schedule")
        W = self.SCHED_VARIANTS
        return list(v), [list(t[w * W:(w + 1) * W]) for w in range(self.SCHED_PASSES)]

    def set_schedule(self, var_a, var_e, var_c=0, var_y=0):
        """Force the schedule (-1 = autotune that entry at the next solve)."""
        v = (C.c_int * self.SCHED_PASSES)(int(var_a), int(var_e), int(var_c), int(var_y))
        _check(load().rve_set_schedule(self.h, v), "rve_set_schedule")

    def test_stall_copies(self, on):
        """Test hook: make the pipelined passes' bounded waits run out (see include/rve.h)."""
        _check(load().rve_test_stall_copies(self.h, 1 if on else 0), "rve_test_stall_copies")

    FORMS = {"stress": 0, "factored": 1, "nodal": 2}

    def set_operator_form(self, form):
        """'stress' (default: FFT of every stress component), 'factored'
        (real-space nodal forces, FFT of the D nodal components only) or
        'nodal' (the factored chain with the CG vectors kept as nodal fields)."""
        _check(load().rve_set_operator_form(self.h, self.FORMS[form]), "rve_set_operator_form")

    def operator_form(self):
        f = C.c_int()
        _check(load().rve_operator_form(self.h, C.byref(f)), "rve_operator_form")
        return {v: k for k, v in self.FORMS.items()}[f.value]

    DERIVATIVES = {"fe": 0, "fourier": 1, "central": 2, "forward": 3, "lsq": 4, "fourier2": 5}

    def set_derivative(self, derivative):
        """Discrete derivative of the projection: 'fe' (default), 'fourier',
        'central', 'forward', 'lsq' or 'fourier2' (see include/rve.h).  The
        non-FE ones need an 'fp64' handle in the 'stress' form."""
        lib = load()
        _check(lib.rve_set_derivative(self.h, self.DERIVATIVES[derivative]), "rve_set_derivative")
        N, m, ns, d = C.c_int64(), C.c_int(), C.c_int(), C.c_int()
        _check(lib.rve_sizes(self.h, C.byref(N), C.byref(m), C.byref(ns), C.byref(d)), "rve_sizes")
        self.m = m.value

    def derivative(self):
        d, nq = C.c_int(), C.c_int()
        _check(load().rve_derivative(self.h, C.byref(d), C.byref(nq)), "rve_derivative")
        return {v: k for k, v in self.DERIVATIVES.items()}[d.value]

    def set_kinematics(self, kinematics):
        """'small' (default) or 'finite' (St. Venant-Kirchhoff deformation
        gradients; needs an 'fp64' handle, stress form, FE derivative)."""
        lib = load()
        _check(lib.rve_set_kinematics(self.h, {"small": 0, "finite": 1}[kinematics]), "rve_set_kinematics")
        N, m, ns, d = C.c_int64(), C.c_int(), C.c_int(), C.c_int()
        _check(lib.rve_sizes(self.h, C.byref(N), C.byref(m), C.byref(ns), C.byref(d)), "rve_sizes")
        self.m = m.value

    def solve_finite(self, F_macro, rel_tol=1e-10, max_newton=30, max_iter=20000):
        """Newton-projected-CG for F_macro[L][D][D]; returns (code, info list)."""
        D = self.dim
        Fm = np.ascontiguousarray(np.asarray(F_macro, dtype=np.float64).reshape(-1, D, D))
        L = Fm.shape[0]
        self._L = L
        info = (rve_info * L)()
        code = load().rve_solve_finite(self.h, Fm.ctypes.data_as(C.POINTER(C.c_double)), L, float(rel_tol),
                                       int(max_newton), int(max_iter), info)
        _check(code, "rve_solve_finite", allow=(RVE_ERR_NOT_CONVERGED, RVE_ERR_NONFINITE))
        return code, [i.as_dict() for i in info]

    def mean_piola(self):
        P = np.zeros((self._L, self.dim, self.dim))
        _check(load().rve_mean_piola(self.h, P.ctypes.data_as(C.POINTER(C.c_double))), "rve_mean_piola")
        return P

    def get_deformation(self, load_case):
        nq = 2 if self.dim == 2 else 6
        out = np.zeros((nq, self.dim, self.dim, self.N))
        p, flag, _k = _buffer(out, np.float64, out.size, "out")
        _check(load().rve_get_deformation(self.h, int(load_case), p, flag), "rve_get_deformation")
        return out

    # kind 7: real-space material kernel of the factored / nodal forms and of
    # finite strain; kind 8: real-space update kernel of the factored / nodal forms
    KINDS = ("pass_a", "pass_b", "pass_c", "pass_d", "pass_e", "residual", "other", "force_stencil",
             "strain_update")

    def timing(self, enable):
        _check(load().rve_timing_enable(self.h, 1 if enable else 0), "rve_timing_enable")

    def timing_read(self):
        ms = (C.c_double * len(self.KINDS))()
        cnt = (C.c_int64 * len(self.KINDS))()
        _check(load().rve_timing_read(self.h, ms, cnt), "rve_timing_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.KINDS)}

    def apply_operator(self, p, material=True, out=None):
        """q = G C p (material=False: q = G p) for p[m][N] in the handle's inner
        precision (numpy array or torch tensor; out of the same kind and place)."""
        if isinstance(p, np.ndarray):
            p = np.ascontiguousarray(p, dtype=self.inner_dtype)
        if out is None:
            out = np.zeros_like(p) if isinstance(p, np.ndarray) else p.new_empty(p.shape)
        count = self.m * self.N
        pp, flag, _k1 = _buffer(p, self.inner_dtype, count, "p")
        qp, flag2, _k2 = _buffer(out, self.inner_dtype, count, "out")
        if flag != flag2:
            raise ValueError("p and out must both be host or both be device buffers")
        _check(load().rve_apply_operator(self.h, pp, qp, 1 if material else 0, flag), "rve_apply_operator")
        return out


class RVEBatch:
    """A batch of RVEs of uneven grid size (one dimension, precision and nu)."""

    def __init__(self, sizes, precision="mixed", nu=0.3):
        lib = load()
        sizes = [tuple(int(v) for v in n) for n in sizes]
        self.dim = len(sizes[0])
        self.count = len(sizes)
        self.sizes = sizes
        self.ns = 3 if self.dim == 2 else 6
        flat = (C.c_int64 * (self.count * self.dim))(*[v for n in sizes for v in n])
        h = C.c_void_p()
        prec = RVE_MIXED if precision == "mixed" else RVE_FP64
        _check(lib.rve_batch_create(C.byref(h), self.dim, self.count, flat, prec, float(nu)), "rve_batch_create")
        self.h = h
        self.L = 0

    def close(self):
        if getattr(self, "h", None):
            load().rve_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_material(self, index, E):
        if not 0 <= int(index) < self.count:
            raise IndexError(f"index {index} outside 0..{self.count - 1}")
        E = np.ascontiguousarray(E, dtype=np.float64)
        want = int(np.prod(self.sizes[int(index)]))
        if E.size != want:
            raise ValueError(f"E: {E.size} elements, expected {want} for RVE {index}")
        _check(load().rve_batch_set_material(self.h, int(index), E.ctypes.data_as(C.c_void_p), RVE_F64,
                                             RVE_PTR_HOST), "rve_batch_set_material")

    def solve(self, E_macro, rel_tol=1e-10, max_iter=5000):
        Em = np.ascontiguousarray(np.atleast_2d(np.asarray(E_macro, dtype=np.float64)))
        if Em.ndim != 2 or Em.shape[1] != self.ns:
            raise ValueError(f"E_macro: shape {Em.shape}, expected (L, {self.ns})")
        L = Em.shape[0]
        info = (rve_info * (self.count * L))()
        code = load().rve_batch_solve(self.h, Em.ctypes.data_as(C.POINTER(C.c_double)), L, float(rel_tol),
                                      int(max_iter), info)
        _check(code, "rve_batch_solve", allow=(RVE_ERR_NOT_CONVERGED,))
        self.L = L
        return code, [[info[i * L + l].as_dict() for l in range(L)] for i in range(self.count)]

    def mean_stress(self, index):
        S = np.zeros((self.L, self.ns))
        _check(load().rve_batch_mean_stress(self.h, int(index), S.ctypes.data_as(C.POINTER(C.c_double))),
               "rve_batch_mean_stress")
        return S

    def effective_tangent(self, index):
        Cm = np.zeros((self.ns, self.ns))
        _check(load().rve_batch_effective_tangent(self.h, int(index), Cm.ctypes.data_as(C.POINTER(C.c_double))),
               "rve_batch_effective_tangent")
        return Cm
