"""ctypes binding of the chx C ABI (``include/chx.h``): argument marshalling only.

Every computation runs in ``libchx.so``; this module checks tensor shapes,
dtypes and devices, passes raw device pointers and the current CUDA stream,
and turns status codes into exceptions.  There is no CPU fallback: if the
library is missing the import of the first entry point fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchx.so")

F64, F32 = 0, 1
COEF_UNIFORM, COEF_SHARED, COEF_PER_SYSTEM = 0, 1, 2
PREMAP_NONE, PREMAP_CUBIC_MINUS_C = 0, 1
PREC_F64, PREC_F32_REFINE = 0, 1

STATUS = {0: "CHX_OK", -1: "CHX_EINVAL", -2: "CHX_ESINGULAR", -3: "CHX_ENONFINITE", -4: "CHX_ENOMEM",
          -5: "CHX_ECUDA", -6: "CHX_ETIMEOUT", -7: "CHX_EUNSUPPORTED"}

# every symbol include/chx.h declares
EXPORTS = ("chx_status_string", "chx_last_error", "chx_version", "stencil_apply_2d", "penta_cyclic_factor",
           "penta_cyclic_refactor", "penta_cyclic_solve_batched", "tri_cyclic_factor", "tri_cyclic_refactor",
           "tri_cyclic_solve_batched", "ch_plan_create", "ch_work_bytes", "ch_step", "ch_step_host", "ch_diagnostics",
           "ch_diagnostics_noalloc", "ch1d_plan_create", "ch1d_step", "cn1d_plan_create", "cn1d_step", "ch_noise_normals", "ch_step_noise", "ch_cook_run", "ch_observables", "ens_group_observables", "chx_coarsening_rate", "ch_profile", "ch_profile_read", "ch_profile_slot_name", "ens_create",
           "ens_group_create", "ens_group_destroy", "ens_group_set_active", "ens_group_set_cook", "ens_slot_load", "ens_slot_read",
           "ens_slot_move", "ens_step", "ens_group_step", "ens_autotune", "ens_info", "ens_tune_schedule",
           "ens_schedule_info", "ens_bytes_used",
           "chx_fp64_fma_rate", "chx_sync_status", "chx_plan_destroy")


class ChxError(RuntimeError):
    def __init__(self, status: int, detail: str):
        super().__init__(f"{STATUS.get(status, status)}: {detail}")
        self.status = status


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def lib():
    """Load libchx.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run `python -c 'import __graft_entry__ as g; g.build()'` first")
    L = ctypes.CDLL(LIB_PATH)
    i, d, sz = ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "chx_status_string": (ctypes.c_char_p, [i]),
        "chx_last_error": (ctypes.c_char_p, []),
        "chx_version": (i, []),
        "stencil_apply_2d": (i, [_P, _P, i, i, i, _D, i, i, i, i, i, i, i, _P]),
        "penta_cyclic_factor": (i, [ctypes.POINTER(_P), i, i, _P, _P, _P, _P, _P, i, i, _P]),
        "penta_cyclic_refactor": (i, [_P, _P, _P, _P, _P, _P, _P]),
        "penta_cyclic_solve_batched": (i, [_P, _P, i, i, _P]),
        "tri_cyclic_factor": (i, [ctypes.POINTER(_P), i, i, _P, _P, _P, i, i, _P]),
        "tri_cyclic_refactor": (i, [_P, _P, _P, _P, _P]),
        "tri_cyclic_solve_batched": (i, [_P, _P, i, _P]),
        "ch_plan_create": (i, [ctypes.POINTER(_P), i, i, d, d, d, d, i]),
        "ch_work_bytes": (sz, [_P]),
        "ch_step": (i, [_P, _P, _P, _P, i, _P]),
        "ch_step_host": (i, [_P, _P, _P, _P, _P, _P, _P, i, _P]),
        "ch_diagnostics": (i, [_P, _P, _P, _P, _P]),
        "ch_diagnostics_noalloc": (i, [_P, i, i, d, d, d, _P, _P, _P]),
        "ch1d_plan_create": (i, [ctypes.POINTER(_P), i, i, d, d, d]),
        "ch1d_step": (i, [_P, _P, i, _P]),
        "cn1d_plan_create": (i, [ctypes.POINTER(_P), i, i, i, d, d, d, i]),
        "cn1d_step": (i, [_P, _P, i, _P]),
        "ch_observables": (i, [_P, _P, _P, _P]),
        "ens_group_observables": (i, [_P, i, i, _P, _P]),
        "chx_coarsening_rate": (i, [ctypes.POINTER(d), ctypes.POINTER(d), i, ctypes.POINTER(d)]),
        "ch_noise_normals": (i, [_P, i, i, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _P]),
        "ch_step_noise": (i, [_P, _P, _P, _P, _P, d, _P]),
        "ch_cook_run": (i, [_P, _P, _P, _P, _P, i, d, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, _P]),
        "ch_profile": (i, [_P, i]),
        "ch_profile_read": (i, [_P, _D, ctypes.POINTER(ctypes.c_longlong), i, i]),
        "ch_profile_slot_name": (ctypes.c_char_p, [i]),
        "ens_create": (i, [ctypes.POINTER(_P), i, d, sz]),
        "ens_group_create": (i, [_P, i, d, d, i, ctypes.POINTER(i)]),
        "ens_group_destroy": (i, [_P, i]),
        "ens_group_set_active": (i, [_P, i, i]),
        "ens_group_set_cook": (i, [_P, i, d, ctypes.c_uint64, ctypes.c_uint64]),
        "ens_slot_load": (i, [_P, i, i, _P, _P, d, _P]),
        "ens_slot_read": (i, [_P, i, i, _P, _P, _P]),
        "ens_slot_move": (i, [_P, i, i, i, _P]),
        "ens_step": (i, [_P, i, _P]),
        "ens_group_step": (i, [_P, i, i, _P]),
        "ens_autotune": (i, [_P, i, i, ctypes.POINTER(i), ctypes.POINTER(i), _P]),
        "ens_tune_schedule": (i, [_P, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), _P]),
        "ens_schedule_info": (i, [_P, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]),
        "ens_info": (i, [_P, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i),
                         ctypes.POINTER(i), ctypes.POINTER(sz)]),
        "ens_bytes_used": (sz, [_P]),
        "chx_fp64_fma_rate": (i, [_D, _P]),
        "chx_sync_status": (i, [_P]),
        "chx_plan_destroy": (None, [_P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        raise ChxError(rc, lib().chx_last_error().decode())


def _stream(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev(t, dtype=None, numel=None, name="tensor"):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def _dtype_code(t):
    import torch

    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def status_string(code: int) -> str:
    return lib().chx_status_string(code).decode()


def version() -> int:
    return lib().chx_version()


def stencil_apply_2d(inp, out, weights, left, right, top, bottom, premap=False, periodic=True, stream=None):
    """cuSten-style weighted box stencil on a (ny, nx) field; see include/chx.h."""
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64))
    if w.shape != (top + bottom + 1, left + right + 1):
        raise ValueError("weights must have shape (top+bottom+1, left+right+1)")
    if inp.dim() != 2 or out.shape != inp.shape or out.dtype != inp.dtype:
        raise ValueError("inp and out must be 2D tensors of the same shape and dtype")
    ny, nx = inp.shape
    _check(lib().stencil_apply_2d(_dev(inp, name="inp"), _dev(out, name="out"), nx, ny, nx,
                                  w.ctypes.data_as(_D), left, right, top, bottom,
                                  PREMAP_CUBIC_MINUS_C if premap else PREMAP_NONE, int(bool(periodic)),
                                  _dtype_code(inp), _stream(stream)))
    return out


class _Plan:
    _handle = None

    def sync_status(self):
        _check(lib().chx_sync_status(self._handle))

    def close(self):
        if self._handle:
            lib().chx_plan_destroy(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _coef_ptrs(coefs, mode, n, batch):
    """Host numpy arrays for UNIFORM/SHARED (kept alive by the caller), device tensors for PER_SYSTEM."""
    import torch

    if mode == COEF_PER_SYSTEM:
        return [_dev(c, torch.float64, n * batch, "coefficient") for c in coefs], coefs
    want = 1 if mode == COEF_UNIFORM else n
    arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(c, dtype=np.float64).ravel(), (want,))) for c in coefs]
    return [ctypes.c_void_p(a.ctypes.data) for a in arrs], arrs


class PentaPlan(_Plan):
    """Factorised batched cyclic pentadiagonal operator (penta_cyclic_factor)."""

    def __init__(self, n, coefs, batch, mode=COEF_SHARED, dtype=F64, stream=None):
        ptrs, keep = _coef_ptrs(coefs, mode, n, batch)
        h = ctypes.c_void_p()
        _check(lib().penta_cyclic_factor(ctypes.byref(h), n, mode, *ptrs, batch, dtype, _stream(stream)))
        self._handle, self.n, self.batch, self.mode, self.dtype = h, n, batch, mode, dtype
        del keep

    def refactor(self, coefs, stream=None):
        ptrs, keep = _coef_ptrs(coefs, COEF_PER_SYSTEM, self.n, self.batch)
        _check(lib().penta_cyclic_refactor(self._handle, *ptrs, _stream(stream)))

    def solve(self, rhs, refine=False, stream=None):
        """In-place solve of an interleaved (n * batch) right-hand side."""
        batch = rhs.numel() // self.n
        if batch * self.n != rhs.numel():
            raise ValueError("rhs size must be a multiple of n")
        if _dtype_code(rhs) != self.dtype:
            raise TypeError("rhs dtype does not match the plan")
        _check(lib().penta_cyclic_solve_batched(self._handle, _dev(rhs, name="rhs"), batch, int(bool(refine)),
                                                _stream(stream)))
        return rhs


class TriPlan(_Plan):
    """Factorised batched cyclic tridiagonal operator (tri_cyclic_factor)."""

    def __init__(self, n, coefs, batch, mode=COEF_SHARED, dtype=F64, stream=None):
        ptrs, keep = _coef_ptrs(coefs, mode, n, batch)
        h = ctypes.c_void_p()
        _check(lib().tri_cyclic_factor(ctypes.byref(h), n, mode, *ptrs, batch, dtype, _stream(stream)))
        self._handle, self.n, self.batch, self.mode, self.dtype = h, n, batch, mode, dtype
        del keep

    def refactor(self, coefs, stream=None):
        ptrs, keep = _coef_ptrs(coefs, COEF_PER_SYSTEM, self.n, self.batch)
        _check(lib().tri_cyclic_refactor(self._handle, *ptrs, _stream(stream)))

    def solve(self, rhs, stream=None):
        batch = rhs.numel() // self.n
        if batch * self.n != rhs.numel():
            raise ValueError("rhs size must be a multiple of n")
        if _dtype_code(rhs) != self.dtype:
            raise TypeError("rhs dtype does not match the plan")
        _check(lib().tri_cyclic_solve_batched(self._handle, _dev(rhs, name="rhs"), batch, _stream(stream)))
        return rhs


class ChPlan(_Plan):
    """Plan for the ADI Cahn-Hilliard step (ch_plan_create / ch_step / ch_diagnostics)."""

    def __init__(self, nx, ny, lx, ly, gamma, dt, precision=PREC_F64):
        h = ctypes.c_void_p()
        _check(lib().ch_plan_create(ctypes.byref(h), nx, ny, float(lx), float(ly), float(gamma), float(dt),
                                    precision))
        self._handle = h
        self.nx, self.ny, self.lx, self.ly, self.gamma, self.dt, self.precision = nx, ny, lx, ly, gamma, dt, precision

    @property
    def work_bytes(self) -> int:
        return lib().ch_work_bytes(self._handle)

    def alloc_work(self, device="cuda"):
        import torch

        # torch allocations are at least 512-byte aligned
        return torch.empty(max(self.work_bytes, 1), dtype=torch.uint8, device=device)

    def step(self, c_now, c_prev, work, nsteps=1, stream=None):
        import torch

        n = self.nx * self.ny
        _check(lib().ch_step(self._handle, _dev(c_now, torch.float64, n, "c_now"),
                             _dev(c_prev, torch.float64, n, "c_prev"), _dev(work, None, None, "work"), int(nsteps),
                             _stream(stream)))

    def step_host(self, h_now, h_prev, h_out, d_now, d_prev, work, nsteps=1, stream=None):
        """ch_step_host: host fields in (pinned CPU tensors), nsteps steps on the device fields,
        the new C^n copied back into h_out; asynchronous on `stream`."""
        import torch

        n = self.nx * self.ny
        for t, name in ((h_now, "h_now"), (h_prev, "h_prev"), (h_out, "h_out")):
            if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() \
                    or t.numel() != n:
                raise ValueError(f"{name} must be a contiguous float64 CPU tensor of {n} elements")
        _check(lib().ch_step_host(self._handle, ctypes.c_void_p(h_now.data_ptr()), ctypes.c_void_p(h_prev.data_ptr()),
                                  ctypes.c_void_p(h_out.data_ptr()), _dev(d_now, torch.float64, n, "d_now"),
                                  _dev(d_prev, torch.float64, n, "d_prev"), _dev(work, None, None, "work"),
                                  int(nsteps), _stream(stream)))

    def step_noise(self, c_now, c_prev, work, rho, sigma, stream=None):
        """One Cahn-Hilliard-Cook step with given deviates rho (2*nx*ny float64, device)."""
        import torch

        n = self.nx * self.ny
        _check(lib().ch_step_noise(self._handle, _dev(c_now, torch.float64, n, "c_now"),
                                   _dev(c_prev, torch.float64, n, "c_prev"), _dev(work, None, None, "work"),
                                   _dev(rho, torch.float64, 2 * n, "rho"), float(sigma), _stream(stream)))

    def cook_run(self, c_now, c_prev, work, rho, nsteps, sigma, seed, sim=0, step0=0, stream=None):
        """nsteps Cahn-Hilliard-Cook steps drawing deviates into the scratch rho (2*nx*ny float64)."""
        import torch

        n = self.nx * self.ny
        _check(lib().ch_cook_run(self._handle, _dev(c_now, torch.float64, n, "c_now"),
                                 _dev(c_prev, torch.float64, n, "c_prev"), _dev(work, None, None, "work"),
                                 _dev(rho, torch.float64, 2 * n, "rho"), int(nsteps), float(sigma), int(seed),
                                 int(sim), int(step0), _stream(stream)))

    def observables(self, c, out, stream=None):
        """[mass, F_h, s, k1] of field c into the 4-element float64 device tensor ``out``."""
        import torch

        _check(lib().ch_observables(self._handle, _dev(c, torch.float64, self.nx * self.ny, "c"),
                                    _dev(out, torch.float64, 4, "out"), _stream(stream)))
        return out

    def profile(self, enable: bool = True):
        """Bracket every kernel of later steps with CUDA events (ch_profile)."""
        _check(lib().ch_profile(self._handle, int(bool(enable))))

    def profile_read(self, reset: bool = True) -> dict:
        """{kernel name: (total ms, launches)} accumulated since the last reset."""
        ms = (ctypes.c_double * 16)()
        n = (ctypes.c_longlong * 16)()
        k = lib().ch_profile_read(self._handle, ms, n, 16, int(bool(reset)))
        if k < 0:
            _check(k)
        return {lib().ch_profile_slot_name(i).decode(): (ms[i], n[i]) for i in range(k) if n[i] > 0}

    def diagnostics(self, c, out, stream=None):
        """Writes (mass, energy) into the 2-element float64 device tensor ``out``."""
        import torch

        _dev(out, torch.float64, 2, "out")
        base = out.data_ptr()
        _check(lib().ch_diagnostics(self._handle, _dev(c, torch.float64, self.nx * self.ny, "c"),
                                    ctypes.c_void_p(base), ctypes.c_void_p(base + 8), _stream(stream)))
        return out


def noise_normals(rho, nx, ny, seed, sim, step, stream=None):
    """Cahn-Hilliard-Cook deviates (ch_noise_normals) into rho (2*nx*ny float64, device)."""
    import torch

    _check(lib().ch_noise_normals(_dev(rho, torch.float64, 2 * nx * ny, "rho"), int(nx), int(ny), int(seed), int(sim),
                                  int(step), _stream(stream)))
    return rho


def coarsening_rate(t, F):
    """beta = -(t/F) dF/dt along a sampled series (chx_coarsening_rate, host arrays)."""
    import numpy as np

    t = np.ascontiguousarray(t, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.float64)
    if t.shape != F.shape:
        raise ValueError("t and F must have the same length")
    beta = np.empty_like(t)
    P = ctypes.POINTER(ctypes.c_double)
    _check(lib().chx_coarsening_rate(t.ctypes.data_as(P), F.ctypes.data_as(P), int(t.size), beta.ctypes.data_as(P)))
    return beta


def fp64_fma_rate(stream=None) -> float:
    """The device's FP64 fused multiply-add rate in 1e9 per second (chx_fp64_fma_rate)."""
    v = ctypes.c_double(0.0)
    _check(lib().chx_fp64_fma_rate(ctypes.byref(v), _stream(stream)))
    return v.value


def ch_diagnostics_noalloc(c, lx, ly, gamma, out, stream=None):
    """(mass, energy) of a (ny, nx) float64 CUDA field into the 2-element device tensor ``out``,
    through the allocation-free entry point (no plan, static device scratch)."""
    import torch

    if c.dim() != 2:
        raise ValueError("c must be a 2D (ny, nx) tensor")
    ny, nx = c.shape
    _dev(out, torch.float64, 2, "out")
    base = out.data_ptr()
    _check(lib().ch_diagnostics_noalloc(_dev(c, torch.float64, None, "c"), nx, ny, float(lx), float(ly), float(gamma),
                                        ctypes.c_void_p(base), ctypes.c_void_p(base + 8), _stream(stream)))
    return out


def _any_ptr(t, numel, name):
    """Contiguous float64 tensor on the GPU or in (preferably pinned) host memory."""
    import torch

    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be a contiguous float64 tensor of {numel} elements")
    return ctypes.c_void_p(t.data_ptr())


class Ch1DPlan(_Plan):
    """Batched 1D Cahn-Hilliard (ch1d_plan_create / ch1d_step), interleaved c[i*batch + s]."""

    def __init__(self, n, batch, l, gamma, dt):
        h = ctypes.c_void_p()
        _check(lib().ch1d_plan_create(ctypes.byref(h), n, batch, float(l), float(gamma), float(dt)))
        self._handle, self.n, self.batch = h, n, batch

    def step(self, c, nsteps=1, stream=None):
        import torch

        _check(lib().ch1d_step(self._handle, _dev(c, torch.float64, self.n * self.batch, "c"), int(nsteps),
                               _stream(stream)))
        return c


class CN1DPlan(_Plan):
    """Batched Crank-Nicolson hyperdiffusion (order 4) or diffusion (order 2) steps
    (cn1d_plan_create / cn1d_step), interleaved c[i*batch + s]; rewrite=True resets
    and refactorises every system's matrix each step."""

    def __init__(self, order, n, batch, l, kappa, dt, rewrite=False):
        h = ctypes.c_void_p()
        _check(lib().cn1d_plan_create(ctypes.byref(h), int(order), n, batch, float(l), float(kappa), float(dt),
                                      1 if rewrite else 0))
        self._handle, self.order, self.n, self.batch, self.rewrite = h, order, n, batch, bool(rewrite)

    def step(self, c, nsteps=1, stream=None):
        import torch

        _check(lib().cn1d_step(self._handle, _dev(c, torch.float64, self.n * self.batch, "c"), int(nsteps),
                               _stream(stream)))
        return c


class Ensemble(_Plan):
    """Ensemble runtime (ens_*): groups of same-(n, L) simulations with per-slot gamma,
    device-resident state, graph-captured batched steps."""

    def __init__(self, dt, precision=PREC_F64, hbm_budget=0):
        h = ctypes.c_void_p()
        _check(lib().ens_create(ctypes.byref(h), precision, float(dt), int(hbm_budget)))
        self._handle, self.dt, self.precision = h, dt, precision
        self.groups = {}

    def group_create(self, n, l, gamma, capacity):
        gid = ctypes.c_int()
        _check(lib().ens_group_create(self._handle, n, float(l), float(gamma), capacity, ctypes.byref(gid)))
        self.groups[gid.value] = (n, l, capacity)
        return gid.value

    def group_destroy(self, gid):
        _check(lib().ens_group_destroy(self._handle, gid))
        self.groups.pop(gid, None)

    def set_active(self, gid, active):
        _check(lib().ens_group_set_active(self._handle, gid, active))

    def set_cook(self, gid, sigma, seed=0, step0=0):
        """Cahn-Hilliard-Cook forcing for every slot of group gid (slot s draws with simulation id s)."""
        _check(lib().ens_group_set_cook(self._handle, int(gid), float(sigma), int(seed), int(step0)))

    def load(self, gid, slot, c0, cm1=None, gamma=-1.0, stream=None):
        n = self.groups[gid][0]
        p1 = _any_ptr(c0, n * n, "c0")
        p2 = _any_ptr(cm1, n * n, "cm1") if cm1 is not None else None
        _check(lib().ens_slot_load(self._handle, gid, slot, p1, p2, float(gamma), _stream(stream)))

    def read(self, gid, slot, c_now, c_prev=None, stream=None):
        n = self.groups[gid][0]
        p1 = _any_ptr(c_now, n * n, "c_now")
        p2 = _any_ptr(c_prev, n * n, "c_prev") if c_prev is not None else None
        _check(lib().ens_slot_read(self._handle, gid, slot, p1, p2, _stream(stream)))

    def move(self, gid, src, dst, stream=None):
        _check(lib().ens_slot_move(self._handle, gid, src, dst, _stream(stream)))

    def observables(self, gid, out, with_k1=False, stream=None):
        """[mass, F_h, s, k1] of every active slot of group gid into the float64 device tensor
        ``out`` (4 * active values, slot-major); k1 is NaN unless with_k1."""
        import torch

        _check(lib().ens_group_observables(self._handle, int(gid), 1 if with_k1 else 0,
                                           _dev(out, torch.float64, None, "out"), _stream(stream)))
        return out

    def step(self, nsteps=1, stream=None):
        _check(lib().ens_step(self._handle, int(nsteps), _stream(stream)))

    def group_step(self, gid, nsteps=1, stream=None):
        _check(lib().ens_group_step(self._handle, gid, int(nsteps), _stream(stream)))

    def autotune(self, gid, trial=3, stream=None):
        px, py = ctypes.c_int(), ctypes.c_int()
        _check(lib().ens_autotune(self._handle, gid, int(trial), ctypes.byref(px), ctypes.byref(py), _stream(stream)))
        return px.value, py.value

    def tune_schedule(self, trial=3, stream=None):
        """Pick the packed FP32 schedule (group order, points per work item, y blocks per SM) by timing."""
        order, target = ctypes.c_int(), ctypes.c_int()
        blocks = (ctypes.c_int * 3)()
        _check(lib().ens_tune_schedule(self._handle, int(trial), ctypes.byref(order), ctypes.byref(target), blocks,
                                       _stream(stream)))
        return {"order": order.value, "points_per_item": target.value, "blocks": list(blocks)}

    def schedule_info(self):
        """Work items and blocks of the packed FP32 step's three phases, points per item and group order."""
        items, blocks = (ctypes.c_int * 3)(), (ctypes.c_int * 3)()
        target, order = ctypes.c_int(), ctypes.c_int()
        _check(lib().ens_schedule_info(self._handle, items, blocks, ctypes.byref(target), ctypes.byref(order)))
        return {"items": list(items), "blocks": list(blocks), "points_per_item": target.value, "order": order.value}

    def info(self, gid):
        v = [ctypes.c_int() for _ in range(5)]
        b = ctypes.c_size_t()
        _check(lib().ens_info(self._handle, gid, *[ctypes.byref(x) for x in v], ctypes.byref(b)))
        return {"n": v[0].value, "capacity": v[1].value, "active": v[2].value, "px": v[3].value, "py": v[4].value,
                "bytes": b.value}

    @property
    def bytes_used(self):
        return lib().ens_bytes_used(self._handle)
