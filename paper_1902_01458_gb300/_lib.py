"""ctypes binding of librr's C ABI (include/rr.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts Python
and torch arguments to pointers and sizes, and raises RRError on a non-zero
status.  Device buffers are torch tensors (complex128 / float64, contiguous,
on the operator's device); block vectors have shape [F, N, k].
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librr.so")

RR_OK = 0
STATUS = {0: "RR_OK", 1: "RR_ERR_ARG", 2: "RR_ERR_NOMEM", 3: "RR_ERR_SINGULAR",
          4: "RR_ERR_NOCONV", 5: "RR_ERR_RANK", 6: "RR_ERR_TIMEOUT",
          7: "RR_ERR_CUDA", 8: "RR_ERR_UNSUPPORTED"}
PRECISION = {"fp64": 0, "fp32": 1, "fp32_simt": 2, "fp32_bf16x3": 3, "fp32_bf16x6": 4}
ADVDIFF, NS2D, NS2D_KZ = 1, 3, 4


class RRError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


class rr_grid(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("periodic_y", ctypes.c_int), ("x0", ctypes.c_double),
                ("x1", ctypes.c_double), ("y0", ctypes.c_double),
                ("y1", ctypes.c_double), ("re", ctypes.c_double),
                ("mach", ctypes.c_double), ("sponge_max", ctypes.c_double),
                ("sponge_frac", ctypes.c_double), ("neumann", ctypes.c_int * 4),
                ("kz", ctypes.c_double)]


class rr_baseflow(ctypes.Structure):
    _fields_ = [("rho", ctypes.POINTER(ctypes.c_double)),
                ("u", ctypes.POINTER(ctypes.c_double)),
                ("v", ctypes.POINTER(ctypes.c_double))]


class rr_sketch_opts(ctypes.Structure):
    _fields_ = [("omega_kind", ctypes.c_int), ("density", ctypes.c_double),
                ("power_iters", ctypes.c_int)]


OMEGA_KINDS = {"gaussian": 0, "rademacher": 1, "sparse_rademacher": 2, "orthonormal": 3}


class rr_info(ctypes.Structure):
    _fields_ = [("refine_iters", ctypes.c_int), ("refine_residual", ctypes.c_double),
                ("cqr_cond", ctypes.c_double), ("cqr_shifted", ctypes.c_int),
                ("refine_stagnated", ctypes.c_int), ("first_residual", ctypes.c_double),
                ("problem_solves", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class rr_problem(ctypes.Structure):
    _fields_ = [("op", ctypes.c_void_p), ("s_re", ctypes.c_double), ("s_im", ctypes.c_double),
                ("k", ctypes.c_int), ("seed", ctypes.c_uint64), ("V", ctypes.c_void_p),
                ("U", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("sigma_halko", ctypes.c_void_p)]


class rr_batch_opts(ctypes.Structure):
    _fields_ = [("use_phi", ctypes.c_int), ("refine_tol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("tune", ctypes.c_int), ("lanes", ctypes.c_int)]


class rr_batch_desc(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_int), ("views", ctypes.c_int), ("lanes", ctypes.c_int),
                ("graph_nodes", ctypes.c_int), ("kernel_nodes", ctypes.c_int),
                ("cuda_core_updates", ctypes.c_int), ("plan_ms", ctypes.c_double),
                ("calib_ms", ctypes.c_double), ("tune_ms", ctypes.c_double),
                ("capture_ms", ctypes.c_double), ("tuned_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


# exported symbol -> (restype, argtypes)
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "rr_last_error": (ctypes.c_char_p, []),
    "rr_status_string": (ctypes.c_char_p, [_I]),
    "rr_create_operator": (_I, [ctypes.POINTER(rr_grid), ctypes.POINTER(rr_baseflow),
                                ctypes.POINTER(ctypes.c_double), _I,
                                ctypes.POINTER(_P)]),
    "rr_destroy_operator": (_I, [_P]),
    "rr_operator_dims": (_I, [_P] + [ctypes.POINTER(_I)] * 5),
    "rr_apply": (_I, [_P, _I, ctypes.POINTER(ctypes.c_double), _I, _I, _P, _P, _P]),
    "rr_apply_static": (_I, [_P, _I, ctypes.POINTER(ctypes.c_double), _I, _I, _P, _P, _P]),
    "rr_phi": (_I, [_P, _P, _P]),
    "rr_factor": (_I, [_P, _I, ctypes.POINTER(ctypes.c_double), _I, _P,
                       ctypes.POINTER(_P)]),
    "rr_destroy_factors": (_I, [_P]),
    "rr_factors_dims": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "rr_solve": (_I, [_P, _I, _I, _P, _P, _D, _I, ctypes.POINTER(rr_info)]),
    "rr_sketch": (_I, [_P, _I, ctypes.POINTER(ctypes.c_uint64), _P, _D, _I, _P, _P,
                       ctypes.POINTER(rr_info)]),
    "rr_sketch_ex": (_I, [_P, _I, ctypes.POINTER(ctypes.c_uint64), _P,
                          ctypes.POINTER(rr_sketch_opts), _D, _I, _P, _P,
                          ctypes.POINTER(rr_info)]),
    "rr_test_matrix": (_I, [_I, _I, _I, ctypes.POINTER(ctypes.c_uint64), _P, _I, _D, _P, _P]),
    "rr_modes": (_I, [_P, _I, _P, _P, _P, _I, _D, _I, ctypes.POINTER(rr_info)]),
    "rr_gaussian": (_I, [_I, _I, _I, ctypes.POINTER(ctypes.c_uint64), _P, _P, _P]),
    "rr_refactor": (_I, [_P, ctypes.POINTER(ctypes.c_double)]),
    "rr_gain_grad": (_I, [_P, _I, _I, _P, _P, _P, _D, _I, _P, ctypes.POINTER(rr_info)]),
    "rr_batch_create": (_I, [_I, ctypes.POINTER(rr_problem), _I,
                             ctypes.POINTER(rr_batch_opts), ctypes.POINTER(_P)]),
    "rr_batch_run": (_I, [_P, _P, ctypes.POINTER(rr_info)]),
    "rr_batch_set_shifts": (_I, [_P, ctypes.POINTER(ctypes.c_double)]),
    "rr_batch_describe": (_I, [_P, ctypes.POINTER(rr_batch_desc)]),
    "rr_batch_destroy": (_I, [_P]),
    "rr_debug_waits": (_I, [ctypes.c_uint, _I]),
    "rr_measure_peak": (_I, [_I, _I, ctypes.POINTER(ctypes.c_double)]),
    "rr_launch_count": (ctypes.c_longlong, []),
    "rr_profile_start": (_I, [ctypes.c_uint]),
    "rr_profile_read": (_I, [_I, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_longlong)]),
}

PROFILE_CLASSES = {"schur": 0, "panel": 1, "rowblock": 2, "update": 3, "finalize": 4,
                   "sweep": 5, "residual": 6, "gram": 7, "rightmul": 8, "small": 9, "inner": 10}

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librr.so (built by build.build()); no fallback if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"librr.so not found at {path}: build it with "
            "paper_1902_01458_gb300.build.build() (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != RR_OK:
        msg = load().rr_last_error().decode(errors="replace")
        raise RRError(status, msg)


def _dptr(t) -> int:
    """Device pointer of a contiguous torch tensor."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _check_meta(name, t, dtype, shape):
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")


def _check_place(name, t, device=None):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous CUDA tensor")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name}: on cuda:{t.device.index}, expected cuda:{device}")


def _check_tensor(name, t, dtype, shape, device=None):
    """Raise ValueError unless t is a contiguous CUDA tensor of the given
    dtype and shape (on the given device ordinal when not None).  The C
    library trusts the sizes it is given, so a short or mistyped buffer must
    be caught here, before a kernel reads or writes past its end."""
    _check_meta(name, t, dtype, shape)
    _check_place(name, t, device)


def _check_block_pair(x, y, F, n, device=None):
    """x, y: distinct complex128 block vectors [F, n, k]; returns k."""
    import torch
    if not isinstance(x, torch.Tensor) or x.dim() != 3:
        raise ValueError("x: expected a [F, N, k] tensor")
    k = int(x.shape[2])
    _check_meta("x", x, torch.complex128, (F, n, k))
    _check_meta("y", y, torch.complex128, (F, n, k))
    _check_place("x", x, device)
    _check_place("y", y, device)
    if x.data_ptr() == y.data_ptr():
        raise ValueError("x and y must be distinct buffers")
    return k


def _operator_device(h) -> int:
    """Device ordinal recorded with an operator handle by Operator (None for
    a bare handle)."""
    return _OP_DEVICE.get(int(h.value if hasattr(h, "value") else h))


_OP_DEVICE: dict = {}


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream)


def _shift_array(shifts) -> ctypes.Array:
    s = np.asarray(shifts, dtype=np.complex128).ravel()
    flat = np.empty(2 * s.size, dtype=np.float64)
    flat[0::2] = s.real
    flat[1::2] = s.imag
    return (ctypes.c_double * flat.size)(*flat.tolist())


# ------------------------------------------------------------ the C calls
def rr_create_operator(grid, rho, u, v, weights=None, device: int = 0):
    lib = load()
    g = rr_grid(int(grid.kind), int(grid.nx), int(grid.ny), int(bool(grid.periodic_y)),
                float(grid.x0), float(grid.x1), float(grid.y0), float(grid.y1),
                float(grid.re), float(getattr(grid, "mach", 0.0)),
                float(getattr(grid, "sponge_max", 0.0)),
                float(getattr(grid, "sponge_frac", 0.1)),
                (ctypes.c_int * 4)(*[int(m) for m in getattr(grid, "neumann", (0, 0, 0, 0))]),
                float(getattr(grid, "kz", 0.0)))
    keep = []

    def arr(a):
        if a is None:
            return None
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).ravel())
        keep.append(a)
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    fl = rr_baseflow(arr(rho), arr(u), arr(v))
    w = arr(weights)
    h = ctypes.c_void_p()
    _check(lib.rr_create_operator(ctypes.byref(g), ctypes.byref(fl), w, int(device),
                                  ctypes.byref(h)))
    _OP_DEVICE[int(h.value)] = int(device)
    return h


def rr_destroy_operator(h):
    if h:
        _OP_DEVICE.pop(int(h.value if hasattr(h, "value") else h), None)
        _check(load().rr_destroy_operator(h))


def rr_operator_dims(h):
    vals = [ctypes.c_int() for _ in range(5)]
    _check(load().rr_operator_dims(h, *[ctypes.byref(v) for v in vals]))
    return tuple(v.value for v in vals)


def _apply_args(h, shifts, x, y):
    s = np.asarray(shifts, dtype=np.complex128).ravel()
    n = rr_operator_dims(h)[0]
    F = s.size
    if F < 1:
        raise ValueError("at least one shift")
    k = _check_block_pair(x, y, F, n, _operator_device(h))
    return s, F, k


def rr_apply(h, shifts, x, y, adjoint=False, stream=None):
    s, F, k = _apply_args(h, shifts, x, y)
    _check(load().rr_apply(h, F, _shift_array(s), k, int(adjoint), _dptr(x),
                           _dptr(y), _stream_ptr(stream)))


def rr_apply_static(h, shifts, x, y, adjoint=False, stream=None):
    """rr_apply without any device allocation (shifts staged in a fixed array)."""
    s, F, k = _apply_args(h, shifts, x, y)
    _check(load().rr_apply_static(h, F, _shift_array(s), k, int(adjoint), _dptr(x),
                                  _dptr(y), _stream_ptr(stream)))


def rr_phi(h, phi, stream=None):
    import torch
    _check_tensor("phi", phi, torch.float64, (rr_operator_dims(h)[0],), _operator_device(h))
    _check(load().rr_phi(h, _dptr(phi), _stream_ptr(stream)))


def rr_factor(h, shifts, precision="fp64", stream=None):
    s = np.asarray(shifts, dtype=np.complex128).ravel()
    out = ctypes.c_void_p()
    st = load().rr_factor(h, s.size, _shift_array(s), PRECISION[precision],
                          _stream_ptr(stream), ctypes.byref(out))
    if st != RR_OK and out:
        load().rr_destroy_factors(out)
    _check(st)
    n, _, _, nx, ny = rr_operator_dims(h)
    _FA_DIMS[int(out.value)] = (s.size, n, _operator_device(h), nx * ny)
    return out


def rr_destroy_factors(h):
    if h:
        _FA_DIMS.pop(int(h.value if hasattr(h, "value") else h), None)
        _check(load().rr_destroy_factors(h))


# factors handle -> (F, N, device ordinal) recorded by rr_factor
_FA_DIMS: dict = {}


def _fa_dims(h):
    d = _FA_DIMS.get(int(h.value if hasattr(h, "value") else h))
    if d is None:
        raise ValueError("unknown factors handle (not created by rr_factor)")
    return d[:3]


def _check_blocks(h, k, **tensors):
    """Every named tensor is a complex128 block vector [F, N, k] of the
    factors h (or, for names starting with 'sigma', float64 [F, k])."""
    import torch
    F, n, dev = _fa_dims(h)
    for name, t in tensors.items():
        if t is None:
            continue
        if name.startswith("sigma"):
            _check_meta(name, t, torch.float64, (F, k))
        else:
            _check_meta(name, t, torch.complex128, (F, n, k))
    for name, t in tensors.items():
        if t is not None:
            _check_place(name, t, dev)
    return F, n


def rr_solve(h, b, x, adjoint=False, refine_tol=1e-10, max_refine=10):
    info = rr_info()
    if b.dim() != 3:
        raise ValueError("b: expected a [F, N, k] tensor")
    k = int(b.shape[2])
    _check_blocks(h, k, b=b, x=x)
    if b.data_ptr() == x.data_ptr():
        raise ValueError("b and x must be distinct buffers")
    st = load().rr_solve(h, k, int(adjoint), _dptr(b), _dptr(x), float(refine_tol),
                         int(max_refine), ctypes.byref(info))
    return st, info


def rr_sketch(h, k, seeds, phi, V, sigma_halko, refine_tol=1e-10, max_refine=10,
              omega_kind="gaussian", density=1.0 / 3.0, power_iters=0):
    import torch
    info = rr_info()
    F, n, dev = _fa_dims(h)
    sd = np.asarray(seeds, dtype=np.uint64).ravel()
    if sd.size != F:
        raise ValueError(f"seeds: {sd.size} values, expected one per shift ({F})")
    if phi is not None:
        _check_meta("phi", phi, torch.float64, (n,))
    _check_blocks(h, int(k), V=V, sigma_halko=sigma_halko)
    if phi is not None:
        _check_place("phi", phi, dev)
    arr = (ctypes.c_uint64 * sd.size)(*[int(x) for x in sd])
    phip = None if phi is None else _dptr(phi)
    if omega_kind == "gaussian" and power_iters == 0:
        st = load().rr_sketch(h, int(k), arr, phip, float(refine_tol), int(max_refine),
                              _dptr(V), _dptr(sigma_halko), ctypes.byref(info))
    else:
        kind = OMEGA_KINDS[omega_kind] if isinstance(omega_kind, str) else int(omega_kind)
        opts = rr_sketch_opts(kind, float(density), int(power_iters))
        st = load().rr_sketch_ex(h, int(k), arr, phip, ctypes.byref(opts), float(refine_tol),
                                 int(max_refine), _dptr(V), _dptr(sigma_halko),
                                 ctypes.byref(info))
    return st, info


def rr_modes(h, k, V, U, sigma, orthogonalize=False, refine_tol=1e-10, max_refine=10):
    info = rr_info()
    _check_blocks(h, int(k), V=V, U=U, sigma=sigma)
    if V.data_ptr() == U.data_ptr():
        raise ValueError("V and U must be distinct buffers")
    st = load().rr_modes(h, int(k), _dptr(V), _dptr(U), _dptr(sigma), int(orthogonalize),
                         float(refine_tol), int(max_refine), ctypes.byref(info))
    return st, info


def rr_gain_grad(h, J, U, V, sigma, grad, refine_tol=1e-10, max_refine=10):
    import torch
    info = rr_info()
    if U.dim() != 3:
        raise ValueError("U: expected a [F, N, k] tensor")
    k = int(U.shape[2])
    _fa_dims(h)
    npts = _FA_DIMS[int(h.value if hasattr(h, "value") else h)][3]
    _check_meta("grad", grad.reshape(-1), torch.float64, (3 * npts,))
    _check_blocks(h, k, U=U, V=V, sigma=sigma)
    _check_place("grad", grad, _fa_dims(h)[2])
    st = load().rr_gain_grad(h, int(k), int(J), _dptr(U), _dptr(V), _dptr(sigma),
                             float(refine_tol), int(max_refine), _dptr(grad),
                             ctypes.byref(info))
    return st, info


def rr_refactor(h, shifts):
    s = np.asarray(shifts, dtype=np.complex128).ravel()
    if s.size != _fa_dims(h)[0]:
        raise ValueError("rr_refactor needs one shift per problem of the factors")
    _check(load().rr_refactor(h, _shift_array(s)))


def rr_debug_waits(tries: int = 0, stall_launches: int = 0):
    """Bounded-wait diagnostics (tests of RR_ERR_TIMEOUT): polls per wait
    (0 = default) and the number of next tensor-core sweep launches whose
    first CTA stalls on purpose."""
    _check(load().rr_debug_waits(int(tries), int(stall_launches)))


PEAK_KINDS = {"tf32": 0, "bf16": 1, "fp64": 2, "fp32": 3}


def rr_measure_peak(kind: str, device: int = 0) -> float:
    """Measured TFLOP/s of one arithmetic unit (tcgen05 TF32 / BF16 MMA, FP64 /
    FP32 FMA) on the device, from an on-chip microbenchmark."""
    v = ctypes.c_double()
    _check(load().rr_measure_peak(PEAK_KINDS[kind], int(device), ctypes.byref(v)))
    return v.value


def rr_launch_count() -> int:
    return int(load().rr_launch_count())


def rr_profile_start(classes=()):
    mask = 0
    for c in classes:
        mask |= 1 << PROFILE_CLASSES[c]
    _check(load().rr_profile_start(mask))


def rr_profile_read(cls):
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(load().rr_profile_read(PROFILE_CLASSES[cls], ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def _check_omega(sd, n, k, phi, omega):
    import torch
    _check_meta("omega", omega, torch.complex128, (sd.size, int(n), int(k)))
    if phi is not None:
        _check_meta("phi", phi, torch.float64, (int(n),))
    _check_place("omega", omega)
    if phi is not None:
        _check_place("phi", phi, omega.device.index)


def rr_gaussian(seeds, n, k, phi, omega, stream=None):
    sd = np.asarray(seeds, dtype=np.uint64).ravel()
    _check_omega(sd, n, k, phi, omega)
    arr = (ctypes.c_uint64 * sd.size)(*[int(x) for x in sd])
    _check(load().rr_gaussian(sd.size, int(n), int(k), arr,
                              None if phi is None else _dptr(phi), _dptr(omega),
                              _stream_ptr(stream)))


def rr_test_matrix(seeds, n, k, phi, omega, kind="gaussian", density=1.0 / 3.0, stream=None):
    sd = np.asarray(seeds, dtype=np.uint64).ravel()
    _check_omega(sd, n, k, phi, omega)
    arr = (ctypes.c_uint64 * sd.size)(*[int(x) for x in sd])
    kind = OMEGA_KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(load().rr_test_matrix(sd.size, int(n), int(k), arr,
                                 None if phi is None else _dptr(phi), kind, float(density),
                                 _dptr(omega), _stream_ptr(stream)))


# ---------------------------------------------------------- thin wrappers
@dataclass
class ResolventResult:
    sigma: "object"          # [F, k] float64 (device)
    sigma_halko: "object"    # [F, k]
    U: "object"              # [F, N, k] complex128
    V: "object"              # [F, N, k]
    info: dict


class Operator:
    """Owns an rr_operator handle (device copy of the stencil of L)."""

    def __init__(self, grid, flow, weights=None, device: int = 0):
        rho = getattr(flow, "rho", None)
        self.device = device
        self.handle = rr_create_operator(grid, rho, flow.u, flow.v, weights, device)
        self.n, self.b, self.q, self.nx, self.ny = rr_operator_dims(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            rr_destroy_operator(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, shifts, x, adjoint=False):
        import torch
        y = torch.empty_like(x)
        rr_apply(self.handle, shifts, x, y, adjoint)
        return y

    def phi(self):
        import torch
        p = torch.empty(self.n, dtype=torch.float64, device=f"cuda:{self.device}")
        rr_phi(self.handle, p)
        torch.cuda.synchronize(self.device)
        return p

    def factor(self, shifts, precision="fp64", stream=None) -> "Factors":
        return Factors(self, shifts, precision, stream)


class Factors:
    """Owns an rr_factors handle: the block factors of F shifts."""

    def __init__(self, op: Operator, shifts, precision="fp64", stream=None):
        self.op = op
        self.shifts = np.asarray(shifts, dtype=np.complex128).ravel()
        self.F = self.shifts.size
        self.precision = precision
        self.handle = rr_factor(op.handle, self.shifts, precision, stream)

    def close(self):
        if getattr(self, "handle", None):
            rr_destroy_factors(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self):
        return f"cuda:{self.op.device}"

    def refactor(self, shifts):
        s = np.asarray(shifts, dtype=np.complex128).ravel()
        if s.size != self.F:
            raise ValueError("refactor needs as many shifts as the factors object holds")
        rr_refactor(self.handle, s)
        self.shifts = s

    def solve(self, b, adjoint=False, refine_tol=1e-10, max_refine=10, check=True):
        import torch
        x = torch.empty_like(b)
        st, info = rr_solve(self.handle, b, x, adjoint, refine_tol, max_refine)
        if check:
            _check(st)
        return x, info.as_dict()

    def sketch(self, k, seeds, phi=None, refine_tol=1e-10, max_refine=10,
               omega_kind="gaussian", density=1.0 / 3.0, power_iters=0):
        import torch
        V = torch.empty(self.F, self.op.n, k, dtype=torch.complex128, device=self._dev())
        sh = torch.empty(self.F, k, dtype=torch.float64, device=self._dev())
        st, info = rr_sketch(self.handle, k, seeds, phi, V, sh, refine_tol, max_refine,
                             omega_kind, density, power_iters)
        _check(st)
        return V, sh, info.as_dict()

    def modes(self, V, orthogonalize=False, refine_tol=1e-10, max_refine=10):
        import torch
        k = V.shape[2]
        U = torch.empty_like(V)
        sig = torch.empty(self.F, k, dtype=torch.float64, device=self._dev())
        st, info = rr_modes(self.handle, k, V, U, sig, orthogonalize, refine_tol,
                            max_refine)
        _check(st)
        return U, sig, info.as_dict()

    def gain_grad(self, J, U, V, sigma, grad=None, refine_tol=1e-10, max_refine=10):
        """grad += d(sum over shifts of sum_{j<J} sigma_j^2)/d(rho, U, V), shape
        [3, nx, ny] float64 on the device (allocated zeroed when None)."""
        import torch
        if grad is None:
            grad = torch.zeros(3, self.op.nx, self.op.ny, dtype=torch.float64,
                               device=self._dev())
        st, info = rr_gain_grad(self.handle, J, U, V, sigma, grad, refine_tol, max_refine)
        _check(st)
        return grad, info.as_dict()

    def randomized_resolvent(self, k, seeds, phi=None, orthogonalize=False,
                             refine_tol=1e-10, max_refine=10, omega_kind="gaussian",
                             density=1.0 / 3.0, power_iters=0) -> ResolventResult:
        """Algorithm 1 for every shift of the batch."""
        V, sh, i1 = self.sketch(k, seeds, phi, refine_tol, max_refine, omega_kind, density,
                                power_iters)
        U, sig, i2 = self.modes(V, orthogonalize, refine_tol, max_refine)
        info = {key: max(i1[key], i2[key]) for key in i1}
        return ResolventResult(sig, sh, U, V, info)


class Batch:
    """Owns an rr_batch plan: problems of uneven size (operators, shifts, k)
    run as one captured CUDA graph.  Outputs are allocated here per problem
    (V, U [N, k] complex128; sigma, sigma_halko [k] float64, on the device) and
    rewritten by every run()."""

    def __init__(self, problems, precision="fp32", use_phi=True, refine_tol=1e-10,
                 max_refine=10, tune=False, lanes=0):
        import torch
        self.problems = list(problems)
        if not self.problems:
            raise ValueError("a batch needs at least one problem")
        self.outputs = []
        arr = (rr_problem * len(self.problems))()
        for i, p in enumerate(self.problems):
            op, shift, k, seed = p["op"], complex(p["shift"]), int(p["k"]), int(p["seed"])
            dev = f"cuda:{op.device}"
            out = {"V": torch.empty(op.n, k, dtype=torch.complex128, device=dev),
                   "U": torch.empty(op.n, k, dtype=torch.complex128, device=dev),
                   "sigma": torch.empty(k, dtype=torch.float64, device=dev),
                   "sigma_halko": torch.empty(k, dtype=torch.float64, device=dev)}
            self.outputs.append(out)
            arr[i] = rr_problem(op.handle.value if hasattr(op.handle, "value") else op.handle,
                                shift.real, shift.imag, k, seed, _dptr(out["V"]),
                                _dptr(out["U"]), _dptr(out["sigma"]),
                                _dptr(out["sigma_halko"]))
        opts = rr_batch_opts(int(bool(use_phi)), float(refine_tol), int(max_refine),
                             int(bool(tune)), int(lanes))
        h = ctypes.c_void_p()
        _check(load().rr_batch_create(len(self.problems), arr, PRECISION[precision],
                                      ctypes.byref(opts), ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None, check=True):
        info = rr_info()
        st = load().rr_batch_run(self.handle, _stream_ptr(stream), ctypes.byref(info))
        if check:
            _check(st)
        return st, info.as_dict()

    def set_shifts(self, shifts):
        s = np.asarray(shifts, dtype=np.complex128).ravel()
        if s.size != len(self.problems):
            raise ValueError("one shift per problem")
        _check(load().rr_batch_set_shifts(self.handle, _shift_array(s)))

    def describe(self) -> dict:
        d = rr_batch_desc()
        _check(load().rr_batch_describe(self.handle, ctypes.byref(d)))
        return d.as_dict()

    def close(self):
        if getattr(self, "handle", None):
            _check(load().rr_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
