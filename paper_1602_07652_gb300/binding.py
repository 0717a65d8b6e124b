"""Thin ctypes binding over libls.so (the C ABI in include/ls.h).

Argument marshalling only: every function forwards torch tensor device pointers
(or host pointers for `solve_host`) to the C entry point of the same name and
raises `LSError` on a non-zero status.  No computation happens here, and there
is no fallback: if libls.so is missing or no CUDA device is present, `load()`
raises.
"""
from __future__ import annotations

import ctypes
import weakref
import os

import torch

_LIB = None
_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libls.so")

LS_FP64, LS_MIXED = 0, 1
LS_MAX_BATCH, LS_MAX_BD_BATCH = 64, 32
LS_PC_BD, LS_PC_GS = 0, 1


class LSError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _LIB.ls_strerror(code).decode() if _LIB is not None else str(code)
        super().__init__("%s failed: %s (%d)" % (where, msg, code))
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nz", ctypes.c_int), ("layers", ctypes.c_int),
                ("ext", ctypes.c_int), ("precision", ctypes.c_int)]


class Opts(ctypes.Structure):
    _fields_ = [("inner_tol", ctypes.c_double), ("inner_restart", ctypes.c_int),
                ("inner_maxit", ctypes.c_int), ("outer_restart", ctypes.c_int),
                ("outer_maxit", ctypes.c_int), ("shift", ctypes.c_double),
                ("refine_maxit", ctypes.c_int), ("refine_inner_tol", ctypes.c_double),
                ("use_graphs", ctypes.c_int), ("inner_precond", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters_total", ctypes.c_int),
                ("inner_calls", ctypes.c_int), ("refine_steps", ctypes.c_int),
                ("true_rel_residual", ctypes.c_double), ("t_solve_s", ctypes.c_double),
                ("t_apply_ms", ctypes.c_double), ("n_apply", ctypes.c_int),
                ("t_apply64_ms", ctypes.c_double), ("n_apply64", ctypes.c_int),
                ("t_sweep_ms", ctypes.c_double), ("n_sweep", ctypes.c_int),
                ("kernel_launches", ctypes.c_longlong), ("learned_steps", ctypes.c_int),
                ("t_stencil_ms", ctypes.c_double), ("n_stencil", ctypes.c_int),
                ("t_orth_ms", ctypes.c_double), ("n_orth", ctypes.c_int),
                ("sweep_fields", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("fft_variant", ctypes.c_int), ("bd_chunk", ctypes.c_int),
                ("fft_ms", ctypes.c_double * 9), ("bd_ms", ctypes.c_double * 4),
                ("bd_ms_nosplit", ctypes.c_double * 4), ("cr_split", ctypes.c_int),
                ("bd_ms_tc", ctypes.c_double * 4), ("tensor_steps", ctypes.c_int)]

    def as_dict(self):
        return {"fft_variant": self.fft_variant, "bd_chunk": self.bd_chunk,
                "fft_ms": list(self.fft_ms), "bd_ms_per_rhs": list(self.bd_ms),
                "bd_ms_per_rhs_nosplit": list(self.bd_ms_nosplit), "cr_split": self.cr_split,
                "bd_ms_per_rhs_tc": list(self.bd_ms_tc), "tensor_steps": self.tensor_steps}


_P = ctypes.c_void_p
_SIGS = {
    "ls_default_opts": (None, [ctypes.POINTER(Opts)]),
    "ls_setup": (ctypes.c_int, [ctypes.POINTER(Grid), ctypes.c_double, ctypes.c_double, _P,
                                ctypes.POINTER(Opts), _P, ctypes.POINTER(_P)]),
    "ls_factor": (ctypes.c_int, [_P]),
    "ls_apply": (ctypes.c_int, [_P, _P, _P]),
    "ls_axpby": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, _P, ctypes.c_double, ctypes.c_double, _P]),
    "ls_apply_f32": (ctypes.c_int, [_P, _P, _P]),
    "ls_apply_mixed": (ctypes.c_int, [_P, _P, _P]),
    "ls_apply_double_float": (ctypes.c_int, [_P, _P, _P]),
    "ls_incident_rhs": (ctypes.c_int, [_P, ctypes.c_double, _P]),
    "ls_solve": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, ctypes.c_int, ctypes.POINTER(Stats)]),
    "ls_solve_batch": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_double, _P, ctypes.c_int,
                                      ctypes.POINTER(Stats)]),
    "ls_solve_batch_host": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_double, _P, ctypes.POINTER(Stats)]),
    "ls_solve_group": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.c_double,
                                      ctypes.POINTER(_P), ctypes.POINTER(Stats), ctypes.POINTER(ctypes.c_int)]),
    "ls_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Tuning)]),
    "ls_set_shapes": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "ls_set_reduction": (ctypes.c_int, [_P, ctypes.c_int]),
    "ls_set_tensor_steps": (ctypes.c_int, [_P, ctypes.c_int]),
    "ls_set_reduced_inverse": (ctypes.c_int, [_P, ctypes.c_int]),
    "ls_set_double_float": (ctypes.c_int, [_P, ctypes.c_int]),
    "ls_set_pack_members": (ctypes.c_int, [_P, ctypes.c_int]),
    "ls_get_sweep_histogram": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "ls_host_alloc": (ctypes.c_int, [ctypes.c_size_t, ctypes.POINTER(_P)]),
    "ls_host_free": (ctypes.c_int, [_P]),
    "ls_check_conversions": (ctypes.c_int, [_P, _P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_ulonglong)]),
    "ls_device_timeouts": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint)]),
    "ls_test_tma_shortfall": (ctypes.c_int, [ctypes.c_uint]),
    "ls_solve_host": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, ctypes.POINTER(Stats)]),
    "ls_solve_plane_wave": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, _P, ctypes.POINTER(Stats)]),
    "ls_apply_A": (ctypes.c_int, [_P, _P, _P]),
    "ls_apply_C": (ctypes.c_int, [_P, _P, _P]),
    "ls_sweep": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "ls_precond_bd": (ctypes.c_int, [_P, _P, _P]),
    "ls_precond_bd_batch": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "ls_inner_solve": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, ctypes.POINTER(ctypes.c_int)]),
    "ls_local_solve": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P]),
    "ls_get_stencils": (ctypes.c_int, [_P, _P, _P]),
    "ls_get_spectrum": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int)]),
    "ls_get_diag_weight": (ctypes.c_int, [_P, _P]),
    "ls_get_layout": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "ls_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "ls_kernel_count": (ctypes.c_longlong, [_P]),
    "ls_destroy": (None, [_P]),
    "ls_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "ls_apply_f32_noalloc": (ctypes.c_int, [ctypes.c_int, _P, _P, _P, _P, _P]),
    "ls_net_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_ulonglong, _P, ctypes.POINTER(_P)]),
    "ls_net_param_count": (ctypes.c_size_t, [_P]),
    "ls_net_get_params": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "ls_net_set_params": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "ls_net_forward": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "ls_net_train_step": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P, ctypes.c_float,
                                         ctypes.POINTER(ctypes.c_double)]),
    "ls_net_get_grads": (ctypes.c_int, [_P, _P, ctypes.c_size_t]),
    "ls_net_kernel_count": (ctypes.c_longlong, [_P]),
    "ls_net_destroy": (None, [_P]),
    "ls_set_learned": (ctypes.c_int, [_P, _P]),
    "ls_net_set_tensor_cores": (ctypes.c_int, [_P, ctypes.c_int]),
}

EXPORTED = tuple(_SIGS)


def load_library(path: str = LIB_PATH):
    """dlopen libls.so and declare the prototypes (no GPU needed)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(path):
            raise RuntimeError("libls.so not built (run __graft_entry__.build()): %s" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = lib
    return _LIB


def load():
    """Load the library for GPU use; raises when no CUDA device is available."""
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the Lippmann-Schwinger solver runs only on the GPU")
    return load_library()


def _ck(code: int, where: str):
    if code != 0:
        raise LSError(code, where)


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _c128(t: torch.Tensor, n: int, where: str):
    if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
        raise ValueError("%s: expected a contiguous CUDA complex128 tensor with %d elements" % (where, n))
    return _ptr(t)


def solve_group(solvers, fs, tol, us=None):
    """ls_solve_group over independent problems: solvers[i] (distinct Solver objects,
    factored), fs[i] its right-hand side.  Returns (us, per-problem stats, statuses)."""
    lib = load()
    k = len(solvers)
    us = [torch.empty_like(f) for f in fs] if us is None else us
    hs = (_P * k)(*[s._h for s in solvers])
    fp = (_P * k)(*[_c128(f, s.N, "ls_solve_group").value for s, f in zip(solvers, fs)])
    up = (_P * k)(*[_c128(u, s.N, "ls_solve_group").value for s, u in zip(solvers, us)])
    st = (Stats * k)()
    status = (ctypes.c_int * k)()
    rc = lib.ls_solve_group(k, hs, fp, float(tol), up, st, status)
    if rc != 0 and rc != -5:
        _ck(rc, "ls_solve_group")
    return us, [x.as_dict() for x in st], list(status)


class Net:
    """The learned preconditioner step (ls_net_*): a BF16 U-Net on the GPU."""

    def __init__(self, levels=4, c0=32, max_batch=1, H=128, W=128, train=True, seed=0,
                 stream: torch.cuda.Stream | None = None):
        lib = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _ck(lib.ls_net_create(int(levels), int(c0), int(max_batch), int(H), int(W), 1 if train else 0, int(seed),
                              ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "ls_net_create")
        self._h, self._lib, self.levels, self.c0 = h, lib, levels, c0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ls_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tensor_cores(self, on):
        """Forward / backward-data convolutions on tcgen05 (1, default) or WMMA (0)."""
        _ck(self._lib.ls_net_set_tensor_cores(self._h, int(on)), "ls_net_set_tensor_cores")

    def param_count(self):
        return int(self._lib.ls_net_param_count(self._h))

    def get_params(self):
        out = torch.empty(self.param_count(), dtype=torch.float32)
        _ck(self._lib.ls_net_get_params(self._h, _ptr(out), out.numel()), "ls_net_get_params")
        return out

    def set_params(self, flat):
        flat = flat.to(torch.float32).contiguous().cpu()
        _ck(self._lib.ls_net_set_params(self._h, _ptr(flat), flat.numel()), "ls_net_set_params")

    def get_grads(self):
        out = torch.empty(self.param_count(), dtype=torch.float32)
        _ck(self._lib.ls_net_get_grads(self._h, _ptr(out), out.numel()), "ls_net_get_grads")
        return out

    @staticmethod
    def _check(r, m, e=None):
        nb, H, W = r.shape
        for t, dt in ((r, torch.complex128), (m, torch.float64)) + (((e, torch.complex128),) if e is not None else ()):
            if t.dtype != dt or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != (nb, H, W):
                raise ValueError("ls_net: expected contiguous CUDA tensors of shape (nb, H, W)")
        return nb, H, W

    def forward(self, r, m, z=None):
        nb, H, W = self._check(r, m)
        z = torch.empty_like(r) if z is None else z
        _ck(self._lib.ls_net_forward(self._h, nb, H, W, _ptr(r), _ptr(m), _ptr(z)), "ls_net_forward")
        return z

    def train_step(self, r, m, e, lr):
        nb, H, W = self._check(r, m, e)
        loss = ctypes.c_double()
        _ck(self._lib.ls_net_train_step(self._h, nb, H, W, _ptr(r), _ptr(m), _ptr(e), float(lr), ctypes.byref(loss)),
            "ls_net_train_step")
        return loss.value


def host_empty(shape, dtype=torch.complex128) -> torch.Tensor:
    """A CPU tensor in page-locked memory the library allocates (ls_host_alloc), for the
    host-array entry points; the block is released when the last view of it is gone."""
    lib = load_library()
    nbytes = int(torch.Size(shape).numel()) * torch.empty((), dtype=dtype).element_size()
    p = _P()
    _ck(lib.ls_host_alloc(ctypes.c_size_t(nbytes), ctypes.byref(p)), "ls_host_alloc")
    arr = (ctypes.c_byte * nbytes).from_address(p.value)
    weakref.finalize(arr, lib.ls_host_free, _P(p.value))
    return torch.frombuffer(arr, dtype=dtype).view(shape)


def device_timeouts() -> int:
    """Column tiles whose TMA data did not arrive in time (0 in a healthy run)."""
    c = ctypes.c_uint(0)
    _ck(load().ls_device_timeouts(ctypes.byref(c)), "ls_device_timeouts")
    return int(c.value)


def test_tma_shortfall(nbytes: int) -> None:
    """Test hook: make the TMA column pass's waits run out (0 restores)."""
    _ck(load().ls_test_tma_shortfall(int(nbytes)), "ls_test_tma_shortfall")


def default_opts() -> Opts:
    o = Opts()
    load_library().ls_default_opts(ctypes.byref(o))
    return o


def check_conversions(d: torch.Tensor, f: torch.Tensor) -> int:
    """Mismatches of the library's FP64 <-> FP32 conversions against the hardware's
    (d: CUDA float64, f: CUDA float32, same number of elements)."""
    lib = load()
    if d.dtype != torch.float64 or f.dtype != torch.float32 or not d.is_cuda or not f.is_cuda \
            or not d.is_contiguous() or not f.is_contiguous() or d.numel() != f.numel():
        raise ValueError("check_conversions: contiguous CUDA float64 and float32 tensors of one size")
    out = ctypes.c_ulonglong(0)
    _ck(lib.ls_check_conversions(_ptr(d), _ptr(f), d.numel(), ctypes.byref(out)), "ls_check_conversions")
    return int(out.value)


def ls_apply_f32_noalloc(n: int, m32: torch.Tensor, ghat32: torch.Tensor, u: torch.Tensor,
                         y: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None,
                         check: bool = True):
    """FP32 LS-apply that allocates nothing in the library (fixed device scratch).

    m32: CUDA float32 (n, n); ghat32: CUDA complex64 spectral quadrant; u, y: CUDA
    complex64 (n, n).  Returns (y, status); raises on a non-zero status if check.
    """
    lib = load()
    y = torch.empty_like(u) if y is None else y
    dev = torch.cuda.current_device()
    for t in (m32, ghat32, u, y):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("ls_apply_f32_noalloc takes contiguous CUDA tensors")
        if t.device.index != dev:
            raise ValueError("ls_apply_f32_noalloc: every tensor must be on the current device (cuda:%d)" % dev)
    if m32.dtype != torch.float32 or u.dtype != torch.complex64 or y.dtype != torch.complex64 \
            or ghat32.dtype != torch.complex64:
        raise ValueError("ls_apply_f32_noalloc: m float32, ghat/u/y complex64")
    # the library takes n from the caller and trusts the buffers to hold n*n and
    # (P/2+1)^2 elements: check that here, P as the library computes it
    n = int(n)
    if n >= 8:
        P = 1
        while P < 2 * n - 1:
            P *= 2
        if not (m32.numel() == u.numel() == y.numel() == n * n):
            raise ValueError("ls_apply_f32_noalloc: m, u and y must hold n*n = %d elements" % (n * n))
        if ghat32.numel() < (P // 2 + 1) ** 2:
            raise ValueError("ls_apply_f32_noalloc: ghat must hold (P/2+1)^2 = %d elements" % ((P // 2 + 1) ** 2))
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = lib.ls_apply_f32_noalloc(int(n), _ptr(m32), _ptr(ghat32), _ptr(u), _ptr(y), ctypes.c_void_p(st.cuda_stream))
    if check:
        _ck(rc, "ls_apply_f32_noalloc")
    return y, rc


class Solver:
    """A handle of the C library: setup -> factor -> apply / solve."""

    def __init__(self, m: torch.Tensor, omega: float, layers: int, ext: int = 10,
                 precision: int = LS_FP64, h: float | None = None, opts: Opts | None = None,
                 stream: torch.cuda.Stream | None = None):
        lib = load()
        if m.dim() != 2 or m.shape[0] != m.shape[1]:
            raise ValueError("m must be a square (n_z, n_x) array")
        self.n = int(m.shape[0])
        self.N = self.n * self.n
        md = m.to(device="cuda", dtype=torch.float64).contiguous()
        self.omega = float(omega)
        self.h = 1.0 / self.n if h is None else float(h)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = Grid(self.n, self.n, int(layers), int(ext), int(precision))
        handle = ctypes.c_void_p()
        o = ctypes.byref(opts) if opts is not None else None
        _ck(lib.ls_setup(ctypes.byref(g), self.h, self.omega, _ptr(md), o,
                         ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(handle)), "ls_setup")
        self._h = handle
        self._lib = lib
        self.precision = precision
        t, q = ctypes.c_int(), ctypes.c_int()
        _ck(lib.ls_get_layout(self._h, ctypes.byref(t), ctypes.byref(q)), "ls_get_layout")
        self.t, self.q = t.value, q.value
        self.layers = int(layers)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ls_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- entry points (same names as the C ABI) ----
    def ls_factor(self):
        _ck(self._lib.ls_factor(self._h), "ls_factor")

    def ls_apply(self, u, y=None):
        y = torch.empty_like(u) if y is None else y
        _ck(self._lib.ls_apply(self._h, _c128(u, self.N, "ls_apply"), _c128(y, self.N, "ls_apply")), "ls_apply")
        return y

    def ls_axpby(self, a, x, b, y):
        """y = a x + b y in the library (a, b complex scalars); returns y."""
        a, b = complex(a), complex(b)
        _ck(self._lib.ls_axpby(self._h, a.real, a.imag, _c128(x, self.N, "ls_axpby"), b.real, b.imag,
                               _c128(y, self.N, "ls_axpby")), "ls_axpby")
        return y

    def ls_apply_mixed(self, u, y=None):
        y = torch.empty_like(u) if y is None else y
        _ck(self._lib.ls_apply_mixed(self._h, _c128(u, self.N, "ls_apply_mixed"), _c128(y, self.N, "ls_apply_mixed")),
            "ls_apply_mixed")
        return y

    def ls_apply_double_float(self, u, y=None):
        y = torch.empty_like(u) if y is None else y
        _ck(self._lib.ls_apply_double_float(self._h, _c128(u, self.N, "ls_apply_double_float"),
                                            _c128(y, self.N, "ls_apply_double_float")), "ls_apply_double_float")
        return y

    def ls_apply_f32(self, u, y=None):
        y = torch.empty_like(u) if y is None else y
        if u.dtype != torch.complex64 or y.dtype != torch.complex64:
            raise ValueError("ls_apply_f32 takes complex64 tensors")
        _ck(self._lib.ls_apply_f32(self._h, _ptr(u), _ptr(y)), "ls_apply_f32")
        return y

    def ls_incident_rhs(self, theta, f=None):
        f = torch.empty((self.n, self.n), dtype=torch.complex128, device="cuda") if f is None else f
        _ck(self._lib.ls_incident_rhs(self._h, float(theta), _c128(f, self.N, "ls_incident_rhs")), "ls_incident_rhs")
        return f

    def ls_solve(self, f, tol, u=None, x0=False, check=True):
        u = torch.empty_like(f) if u is None else u
        st = Stats()
        rc = self._lib.ls_solve(self._h, _c128(f, self.N, "ls_solve"), float(tol), _c128(u, self.N, "ls_solve"),
                                1 if x0 else 0, ctypes.byref(st))
        if check:
            _ck(rc, "ls_solve")
        return u, st.as_dict(), rc

    def ls_solve_batch(self, f, tol, u=None, x0=False, check=True):
        """f: CUDA complex128 tensor of nrhs fields (nrhs, n, n), back to back."""
        u = torch.empty_like(f) if u is None else u
        nrhs = f.numel() // self.N
        st = Stats()
        rc = self._lib.ls_solve_batch(self._h, nrhs, _c128(f, nrhs * self.N, "ls_solve_batch"), float(tol),
                                      _c128(u, nrhs * self.N, "ls_solve_batch"), 1 if x0 else 0, ctypes.byref(st))
        if check:
            _ck(rc, "ls_solve_batch")
        return u, st.as_dict(), rc

    def ls_set_learned(self, net):
        _ck(self._lib.ls_set_learned(self._h, net._h if net is not None else None), "ls_set_learned")

    def ls_set_shapes(self, fft_variant, bd_chunk=0):
        _ck(self._lib.ls_set_shapes(self._h, int(fft_variant), int(bd_chunk)), "ls_set_shapes")

    def ls_set_reduction(self, cr_split):
        _ck(self._lib.ls_set_reduction(self._h, int(cr_split)), "ls_set_reduction")

    def ls_set_tensor_steps(self, on):
        _ck(self._lib.ls_set_tensor_steps(self._h, int(on)), "ls_set_tensor_steps")

    def ls_set_reduced_inverse(self, on):
        _ck(self._lib.ls_set_reduced_inverse(self._h, int(on)), "ls_set_reduced_inverse")

    def ls_get_sweep_histogram(self):
        """{batch size: Algorithm 2 applications} of the last solve."""
        counts = (ctypes.c_int * 65)()
        _ck(self._lib.ls_get_sweep_histogram(self._h, counts, 65), "ls_get_sweep_histogram")
        return {k: counts[k] for k in range(65) if counts[k]}

    def ls_set_pack_members(self, on):
        _ck(self._lib.ls_set_pack_members(self._h, int(on)), "ls_set_pack_members")

    def ls_set_double_float(self, on):
        _ck(self._lib.ls_set_double_float(self._h, int(on)), "ls_set_double_float")

    def ls_autotune(self, nrhs=1, reps=3):
        t = Tuning()
        _ck(self._lib.ls_autotune(self._h, int(nrhs), int(reps), ctypes.byref(t)), "ls_autotune")
        return t.as_dict()

    def ls_solve_host(self, f_host, tol, u_host):
        """f_host, u_host: CPU complex128 tensors (pinned or pageable)."""
        for t in (f_host, u_host):
            if t.is_cuda or t.dtype != torch.complex128 or not t.is_contiguous() or t.numel() != self.N:
                raise ValueError("ls_solve_host takes contiguous CPU complex128 tensors")
        st = Stats()
        rc = self._lib.ls_solve_host(self._h, _ptr(f_host), float(tol), _ptr(u_host), ctypes.byref(st))
        _ck(rc, "ls_solve_host")
        return st.as_dict()

    def ls_solve_batch_host(self, f_host, tol, u_host):
        """f_host, u_host: CPU complex128 tensors of nrhs fields (pinned or pageable)."""
        nrhs = f_host.numel() // self.N
        for t in (f_host, u_host):
            if t.is_cuda or t.dtype != torch.complex128 or not t.is_contiguous() or t.numel() != nrhs * self.N:
                raise ValueError("ls_solve_batch_host takes contiguous CPU complex128 tensors of whole fields")
        st = Stats()
        rc = self._lib.ls_solve_batch_host(self._h, nrhs, _ptr(f_host), float(tol), _ptr(u_host), ctypes.byref(st))
        _ck(rc, "ls_solve_batch_host")
        return st.as_dict()

    def ls_solve_plane_wave(self, theta, tol, u=None):
        u = torch.empty((self.n, self.n), dtype=torch.complex128, device="cuda") if u is None else u
        st = Stats()
        _ck(self._lib.ls_solve_plane_wave(self._h, float(theta), float(tol), _c128(u, self.N, "ls_solve_plane_wave"),
                                          ctypes.byref(st)), "ls_solve_plane_wave")
        return u, st.as_dict()

    def ls_apply_A(self, r, y=None):
        y = torch.empty_like(r) if y is None else y
        _ck(self._lib.ls_apply_A(self._h, _c128(r, self.N, "ls_apply_A"), _c128(y, self.N, "ls_apply_A")), "ls_apply_A")
        return y

    def ls_apply_C(self, v, y=None):
        y = torch.empty_like(v) if y is None else y
        _ck(self._lib.ls_apply_C(self._h, _c128(v, self.N, "ls_apply_C"), _c128(y, self.N, "ls_apply_C")), "ls_apply_C")
        return y

    def ls_sweep(self, direction, g, v=None):
        v = torch.empty_like(g) if v is None else v
        _ck(self._lib.ls_sweep(self._h, int(direction), _c128(g, self.N, "ls_sweep"), _c128(v, self.N, "ls_sweep")),
            "ls_sweep")
        return v

    def ls_precond_bd(self, g, v=None):
        v = torch.empty_like(g) if v is None else v
        _ck(self._lib.ls_precond_bd(self._h, _c128(g, self.N, "ls_precond_bd"), _c128(v, self.N, "ls_precond_bd")),
            "ls_precond_bd")
        return v

    def ls_precond_bd_batch(self, g, v=None):
        """g: CUDA complex128 tensor of nrhs fields (nrhs, n, n), back to back."""
        v = torch.empty_like(g) if v is None else v
        nrhs = g.numel() // self.N
        _ck(self._lib.ls_precond_bd_batch(self._h, nrhs, _c128(g, nrhs * self.N, "ls_precond_bd_batch"),
                                          _c128(v, nrhs * self.N, "ls_precond_bd_batch")), "ls_precond_bd_batch")
        return v

    def ls_inner_solve(self, g, tol, v=None, check=True):
        """Returns (v, iterations); with check=False, (v, iterations, status)."""
        v = torch.empty_like(g) if v is None else v
        it = ctypes.c_int()
        rc = self._lib.ls_inner_solve(self._h, _c128(g, self.N, "ls_inner_solve"), float(tol),
                                      _c128(v, self.N, "ls_inner_solve"), ctypes.byref(it))
        if not check:
            return v, it.value, rc
        _ck(rc, "ls_inner_solve")
        return v, it.value

    def ls_local_solve(self, direction, layer, b, x=None):
        x = torch.empty_like(b) if x is None else x
        cnt = self.q * self.n
        _ck(self._lib.ls_local_solve(self._h, int(direction), int(layer), _c128(b, cnt, "ls_local_solve"),
                                     _c128(x, cnt, "ls_local_solve")), "ls_local_solve")
        return x

    def ls_get_stencils(self):
        a = (ctypes.c_double * 162)()
        b = (ctypes.c_double * 162)()
        _ck(self._lib.ls_get_stencils(self._h, a, b), "ls_get_stencils")
        import numpy as np
        A = np.frombuffer(a, dtype=np.complex128).copy().reshape(9, 9)
        B = np.frombuffer(b, dtype=np.complex128).copy().reshape(9, 9)
        return A, B

    def ls_get_spectrum(self):
        P = ctypes.c_int()
        _ck(self._lib.ls_get_spectrum(self._h, None, ctypes.byref(P)), "ls_get_spectrum")
        q1 = P.value // 2 + 1
        g = torch.empty((q1, q1), dtype=torch.complex128, device="cuda")
        _ck(self._lib.ls_get_spectrum(self._h, _ptr(g), ctypes.byref(P)), "ls_get_spectrum")
        torch.cuda.synchronize()
        return g, P.value

    def ls_get_diag_weight(self):
        w = (ctypes.c_double * 2)()
        _ck(self._lib.ls_get_diag_weight(self._h, w), "ls_get_diag_weight")
        return complex(w[0], w[1])

    def ls_set_timing(self, on: bool):
        _ck(self._lib.ls_set_timing(self._h, 1 if on else 0), "ls_set_timing")

    def ls_kernel_count(self) -> int:
        return int(self._lib.ls_kernel_count(self._h))
