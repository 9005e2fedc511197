"""ctypes binding of the C ABI in include/lbm_ewod.h (same entry-point names).

Marshalling only: every step of the method runs in the CUDA library. The
binding fails loudly (``LbmUnavailable``) when the compiled library is
missing; there is no CPU fallback. PyTorch is used for device memory (the
workspace tensor) and for the CUDA stream the context enqueues on.

Low level: ``lbm_workspace_bytes``, ``lbm_create``, ``lbm_set_geometry``,
``lbm_set_field``, ``lbm_set_density_f32``, ``lbm_get_field``, ``lbm_step``, ``lbm_observables``,
``lbm_obs_latest``, ``lbm_obs_latest_async``, ``lbm_time``, ``lbm_last_error``, ``lbm_status_string``,
``lbm_destroy``; each raises ``LbmError`` on a non-zero status.
High level: ``Lattice`` owns a workspace tensor and a context.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENAN, LBM_ETIMEOUT, LBM_ESTATE, LBM_ENOTCONV = range(8)
LBM_GREEN_MC, LBM_GREEN_PRINTED = 0, 1
LBM_FP32, LBM_FP32_DEV, LBM_FP16_DEV, LBM_BF16_DEV = 0, 1, 2, 3
LBM_RHO_U, LBM_POPS, LBM_RHO_U_PHYS, LBM_UX_PROFILE, LBM_RHO = 0, 1, 2, 3, 4
LBM_NORMAL_FACES, LBM_NORMAL_UNIT = 0, 1
LBM_LAYOUT_AUTO, LBM_LAYOUT_PAIRS, LBM_LAYOUT_SINGLE = 0, 1, 2


class LbmUnavailable(RuntimeError):
    """The compiled CUDA library is not present or cannot be loaded."""


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_name(status)}: {message}")
        self.status = status


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("tau", ctypes.c_double), ("G", ctypes.c_double), ("G_wall", ctypes.c_double),
        ("rho0", ctypes.c_double), ("rho_c", ctypes.c_double), ("f_elec", ctypes.c_double),
        ("body_fx", ctypes.c_double), ("body_fy", ctypes.c_double),
        ("green", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("obs_every", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
        ("normal", ctypes.c_int32), ("layout", ctypes.c_int32),
    ]


class lbm_obs(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("mass", ctypes.c_double), ("flux_Q", ctypes.c_double),
        ("mom_x", ctypes.c_double), ("mom_y", ctypes.c_double), ("max_u", ctypes.c_double),
        ("min_rho", ctypes.c_double), ("nonfinite", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def load():
    """Load the compiled library (never builds it; see ``build.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise LbmUnavailable(f"CUDA library {path} is not built; run __graft_entry__.build()")
        try:
            lib = ctypes.CDLL(path)
        except OSError as e:
            raise LbmUnavailable(f"cannot load {path}: {e}") from e
        vp, P, O = ctypes.c_void_p, ctypes.POINTER(lbm_params), ctypes.POINTER(lbm_obs)
        sig = {
            "lbm_workspace_bytes": (ctypes.c_size_t, [P]),
            "lbm_create": (ctypes.c_int, [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]),
            "lbm_set_geometry": (ctypes.c_int, [vp, vp, ctypes.c_int]),
            "lbm_set_field": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int]),
            "lbm_set_density_f32": (ctypes.c_int, [vp, vp, ctypes.c_int]),
            "lbm_get_field": (ctypes.c_int, [vp, ctypes.c_int, vp, ctypes.c_int]),
            "lbm_step": (ctypes.c_int, [vp, ctypes.c_int64]),
            "lbm_observables": (ctypes.c_int, [vp, O]),
            "lbm_obs_latest": (ctypes.c_int, [vp, O]),
            "lbm_obs_latest_async": (ctypes.c_int, [vp, vp]),
            "lbm_run_to_steady": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int64, ctypes.c_int64, O]),
            "lbm_time": (ctypes.c_int64, [vp]),
            "lbm_selftest_timeout": (ctypes.c_int, [vp]),
            "lbm_last_error": (ctypes.c_char_p, [vp]),
            "lbm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "lbm_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        _lib = lib
        return lib


def status_name(status: int) -> str:
    names = ["LBM_OK", "LBM_EINVAL", "LBM_ENOMEM", "LBM_ECUDA", "LBM_ENAN", "LBM_ETIMEOUT", "LBM_ESTATE",
             "LBM_ENOTCONV"]
    return names[status] if 0 <= status < len(names) else f"status {status}"


def _check(ctx, status: int):
    if status != LBM_OK:
        msg = lbm_last_error(ctx) if ctx else ""
        raise LbmError(status, msg)


def make_params(nx, ny, tau=1.0, G=-0.52, G_wall=-0.14, rho0=1.0, rho_c=1.0, f_elec=0.0,
                body_fx=0.0, body_fy=0.0, green=LBM_GREEN_MC, storage=LBM_FP32, obs_every=0,
                tile_rows=0, normal=0, layout=0) -> lbm_params:
    return lbm_params(int(nx), int(ny), float(tau), float(G), float(G_wall), float(rho0),
                      float(rho_c), float(f_elec), float(body_fx), float(body_fy), int(green),
                      int(storage), int(obs_every), int(tile_rows), int(normal), int(layout))


# ---------------------------------------------------------------- low level

def lbm_workspace_bytes(params: lbm_params) -> int:
    return int(load().lbm_workspace_bytes(ctypes.byref(params)))


def lbm_create(params: lbm_params, d_workspace: int, nbytes: int, cuda_stream: int):
    ctx = ctypes.c_void_p()
    _check(None, load().lbm_create(ctypes.byref(params), ctypes.c_void_p(d_workspace), nbytes,
                                   ctypes.c_void_p(cuda_stream), ctypes.byref(ctx)))
    return ctx


def lbm_set_geometry(ctx, solid_ptr: int, on_device: bool):
    _check(ctx, load().lbm_set_geometry(ctx, ctypes.c_void_p(solid_ptr), int(on_device)))


def lbm_set_field(ctx, which: int, data_ptr: int, on_device: bool):
    _check(ctx, load().lbm_set_field(ctx, which, ctypes.c_void_p(data_ptr), int(on_device)))


def lbm_set_density_f32(ctx, rho_ptr: int, on_device: bool):
    _check(ctx, load().lbm_set_density_f32(ctx, ctypes.c_void_p(rho_ptr), int(on_device)))


def lbm_get_field(ctx, which: int, out_ptr: int, on_device: bool):
    _check(ctx, load().lbm_get_field(ctx, which, ctypes.c_void_p(out_ptr), int(on_device)))


def lbm_step(ctx, nsteps: int):
    _check(ctx, load().lbm_step(ctx, int(nsteps)))


def lbm_selftest_timeout(ctx) -> int:
    """Status of the timeout self-test (LBM_ETIMEOUT when the path works)."""
    return int(load().lbm_selftest_timeout(ctx))


def lbm_observables(ctx, check_finite: bool = True) -> dict:
    o = lbm_obs()
    st = load().lbm_observables(ctx, ctypes.byref(o))
    if st != LBM_ENAN or check_finite:
        _check(ctx, st)
    return o.as_dict()


def lbm_obs_latest(ctx, check_finite: bool = True) -> dict:
    o = lbm_obs()
    st = load().lbm_obs_latest(ctx, ctypes.byref(o))
    if st != LBM_ENAN or check_finite:
        _check(ctx, st)
    return o.as_dict()


def lbm_obs_latest_async(ctx, out_ptr: int) -> None:
    """Enqueue the copy of the latest fused record into host memory at
    ``out_ptr`` (an ``lbm_obs``, preferably page-locked); no synchronisation.
    Read it with ``obs_from_buffer`` once the stream has passed this point."""
    _check(ctx, load().lbm_obs_latest_async(ctx, ctypes.c_void_p(out_ptr)))


def obs_from_buffer(ptr: int) -> dict:
    """The ``lbm_obs`` record at host address ``ptr`` as a dict."""
    return lbm_obs.from_address(ptr).as_dict()


def lbm_run_to_steady(ctx, rel_tol: float, check_every: int, max_steps: int) -> tuple[dict, bool]:
    """Step until the flux is steady; returns (observables, converged)."""
    o = lbm_obs()
    st = load().lbm_run_to_steady(ctx, float(rel_tol), int(check_every), int(max_steps), ctypes.byref(o))
    if st not in (LBM_OK, LBM_ENOTCONV):
        _check(ctx, st)
    return o.as_dict(), st == LBM_OK


def lbm_time(ctx) -> int:
    return int(load().lbm_time(ctx))


def lbm_last_error(ctx) -> str:
    s = load().lbm_last_error(ctx)
    return s.decode() if s else ""


def lbm_status_string(status: int) -> str:
    return load().lbm_status_string(int(status)).decode()


def lbm_destroy(ctx):
    if ctx:
        load().lbm_destroy(ctx)


# ---------------------------------------------------------------- high level

def _host_ptr(a: np.ndarray, dtype) -> tuple[np.ndarray, int]:
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


class Lattice:
    """One simulation domain on the current CUDA device.

    The workspace is a torch uint8 tensor sized by ``lbm_workspace_bytes``;
    all work goes to ``stream`` (default: torch's current stream). Host
    arrays are numpy; device arrays may be torch CUDA tensors."""

    def __init__(self, nx: int, ny: int, stream=None, _ctx=None, _owner=None, **params):
        import torch

        self.nx, self.ny = int(nx), int(ny)
        if _ctx is not None:
            # a view on a context owned by a Batch
            self.params = make_params(nx, ny, **params)
            self.stream = stream
            self.workspace = None
            self.ctx = _ctx
            self._owner = _owner
            return
        self._owner = None
        self.params = make_params(nx, ny, **params)
        nbytes = lbm_workspace_bytes(self.params)
        if nbytes == 0:
            raise LbmError(LBM_EINVAL, f"invalid parameters {params}")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.stream.device)
        self.ctx = lbm_create(self.params, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)

    # -- inputs
    def set_geometry(self, solid):
        if hasattr(solid, "is_cuda") and solid.is_cuda:
            t = solid.to(dtype=__import__("torch").uint8).contiguous()
            lbm_set_geometry(self.ctx, t.data_ptr(), True)
            self._keep = t
        else:
            a, p = _host_ptr(solid, np.uint8)
            if a.shape != (self.ny, self.nx):
                raise ValueError(f"mask shape {a.shape} != {(self.ny, self.nx)}")
            lbm_set_geometry(self.ctx, p, False)
            self.stream.synchronize()  # page-locked input is read asynchronously

    def _set(self, which, data, comps):
        if hasattr(data, "is_cuda") and data.is_cuda:
            t = data.to(dtype=__import__("torch").float64).contiguous()
            if tuple(t.shape) != (comps, self.ny, self.nx):
                raise ValueError("bad field shape")
            lbm_set_field(self.ctx, which, t.data_ptr(), True)
            self.stream.synchronize()
        else:
            a, p = _host_ptr(data, np.float64)
            if a.shape != (comps, self.ny, self.nx):
                raise ValueError(f"field shape {a.shape} != {(comps, self.ny, self.nx)}")
            lbm_set_field(self.ctx, which, p, False)
            self.stream.synchronize()

    def set_rho_u(self, rho, ux=0.0, uy=0.0, physical=False):
        """State f = f_eq(rho, u). With physical=True, u is the physical
        velocity that fields() reports and the equilibrium takes u - F/(2 rho)
        (LBM_RHO_U_PHYS), so a (rho, u) snapshot restarts without a kick."""
        if hasattr(rho, "is_cuda") and rho.is_cuda:
            import torch
            data = torch.stack([torch.broadcast_to(torch.as_tensor(v, dtype=torch.float64, device=rho.device),
                                                   (self.ny, self.nx)) for v in (rho, ux, uy)])
        else:
            data = np.stack([np.broadcast_to(np.asarray(v, np.float64), (self.ny, self.nx))
                             for v in (rho, ux, uy)])
        self._set(LBM_RHO_U_PHYS if physical else LBM_RHO_U, data, 3)

    def set_rho(self, rho):
        """A fluid at rest: f = f_eq(rho, 0), from the density alone (LBM_RHO)."""
        if hasattr(rho, "is_cuda") and rho.is_cuda:
            self._set(LBM_RHO, rho.reshape(1, self.ny, self.nx), 1)
        else:
            self._set(LBM_RHO, np.asarray(rho, np.float64).reshape(1, self.ny, self.nx), 1)

    def set_density_f32(self, rho):
        """A fluid at rest from an FP32 density [ny, nx] (numpy array or CUDA
        tensor): the LBM_RHO state with FP32 set-up arithmetic
        (lbm_set_density_f32)."""
        if hasattr(rho, "is_cuda") and rho.is_cuda:
            t = rho.to(dtype=__import__("torch").float32).contiguous()
            if tuple(t.shape) != (self.ny, self.nx):
                raise ValueError("bad density shape")
            lbm_set_density_f32(self.ctx, t.data_ptr(), True)
            self.stream.synchronize()
        else:
            a, p = _host_ptr(rho, np.float32)
            if a.shape != (self.ny, self.nx):
                raise ValueError(f"density shape {a.shape} != {(self.ny, self.nx)}")
            lbm_set_density_f32(self.ctx, p, False)
            self.stream.synchronize()

    def set_rho_u_field(self, data, physical=False):
        """(rho, u_x, u_y) as one [3, ny, nx] array or device tensor (FP64)."""
        self._set(LBM_RHO_U_PHYS if physical else LBM_RHO_U, data, 3)

    def set_populations(self, f):
        self._set(LBM_POPS, f, 9)

    # -- outputs
    def populations(self) -> np.ndarray:
        out = np.empty((9, self.ny, self.nx))
        lbm_get_field(self.ctx, LBM_POPS, out.ctypes.data, False)
        return out

    def fields(self):
        out = np.empty((3, self.ny, self.nx))
        lbm_get_field(self.ctx, LBM_RHO_U, out.ctypes.data, False)
        return out[0], out[1], out[2]

    def populations_device(self):
        import torch
        out = torch.empty((9, self.ny, self.nx), dtype=torch.float64, device=self.stream.device)
        lbm_get_field(self.ctx, LBM_POPS, out.data_ptr(), True)
        return out

    def ux_profile(self) -> np.ndarray:
        """Mean velocity profile across the channel, (1/nx) sum_x u_x(x, y)."""
        out = np.empty(self.ny)
        lbm_get_field(self.ctx, LBM_UX_PROFILE, out.ctypes.data, False)
        return out

    def fields_device(self):
        """(rho, u_x, u_y) as one FP64 device tensor [3, ny, nx]."""
        import torch
        out = torch.empty((3, self.ny, self.nx), dtype=torch.float64, device=self.stream.device)
        lbm_get_field(self.ctx, LBM_RHO_U, out.data_ptr(), True)
        return out

    # -- time stepping
    def step(self, n: int = 1):
        lbm_step(self.ctx, n)

    def observables(self, check_finite: bool = True) -> dict:
        return lbm_observables(self.ctx, check_finite)

    def obs_latest(self, check_finite: bool = True) -> dict:
        return lbm_obs_latest(self.ctx, check_finite)

    def run_to_steady(self, rel_tol: float = 1e-7, check_every: int = 1000, max_steps: int = 10 ** 6):
        return lbm_run_to_steady(self.ctx, rel_tol, check_every, max_steps)

    @property
    def time(self) -> int:
        return lbm_time(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) and getattr(self, "_owner", None) is None:
            lbm_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------- allocation-free call

def lbm_observables_noalloc(params: lbm_params, d_pops: int, d_solid: int, step: int,
                            cuda_stream: int, check_finite: bool = True) -> dict:
    """Observables of device-resident post-streaming populations (double
    [9][ny][nx]) and mask (uint8 [ny][nx]) without a context and without any
    device allocation: for callers that cannot allocate when they need the
    numbers (a process whose device memory budget is spent, monitoring or
    checkpoint tools that must not touch the application's allocator). The
    library keeps the scratch in a fixed 64 KB static device array shared by
    all calls, so calls that overlap on the GPU race; domains above
    16,777,216 nodes are rejected. The first call in a device's context looks
    up the array's address and should come before any stream capture on that
    device. Synchronises cuda_stream."""
    lib = load()
    fn = lib.lbm_observables_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(lbm_params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                   ctypes.c_void_p, ctypes.POINTER(lbm_obs)]
    lib.lbm_noalloc_last_error.restype = ctypes.c_char_p
    lib.lbm_noalloc_last_error.argtypes = []
    o = lbm_obs()
    st = fn(ctypes.byref(params), ctypes.c_void_p(d_pops), ctypes.c_void_p(d_solid), int(step),
            ctypes.c_void_p(cuda_stream), ctypes.byref(o))
    if st != LBM_OK and not (st == LBM_ENAN and not check_finite):
        raise LbmError(st, lib.lbm_noalloc_last_error().decode())
    return o.as_dict()



# ------------------------------------------------------------------- batches

def _batch_lib():
    lib = load()
    if not getattr(lib, "_batch_sigs", False):
        vp, P, O = ctypes.c_void_p, ctypes.POINTER(lbm_params), ctypes.POINTER(lbm_obs)
        sig = {
            "lbm_batch_workspace_bytes": (ctypes.c_size_t, [P, ctypes.c_int32]),
            "lbm_batch_create": (ctypes.c_int, [P, ctypes.c_int32, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]),
            "lbm_batch_domain": (vp, [vp, ctypes.c_int32]),
            "lbm_batch_step": (ctypes.c_int, [vp, ctypes.c_int64]),
            "lbm_batch_observables": (ctypes.c_int, [vp, O]),
            "lbm_batch_set_active": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_uint8)]),
            "lbm_batch_set_tile_rows": (ctypes.c_int, [vp, ctypes.c_int32]),
            "lbm_batch_tile_rows": (ctypes.c_int32, [vp]),
            "lbm_batch_autotune": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                                  ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                                  ctypes.POINTER(ctypes.c_double)]),
            "lbm_batch_run_to_steady": (ctypes.c_int, [vp, ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                                       ctypes.POINTER(ctypes.c_int64), O]),
            "lbm_batch_set_ctas_per_sm": (ctypes.c_int, [vp, ctypes.c_int32]),
            "lbm_batch_ctas_per_sm": (ctypes.c_int32, [vp]),
            "lbm_batch_autotune_grid": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                                       ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                                       ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                                       ctypes.POINTER(ctypes.c_int32),
                                                       ctypes.POINTER(ctypes.c_double)]),
            "lbm_batch_last_error": (ctypes.c_char_p, [vp]),
            "lbm_batch_destroy": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype, fn.argtypes = res, args
        lib._batch_sigs = True
    return lib


class Batch:
    """Many domains advanced together (one persistent launch per step).

    ``specs`` is a list of dicts of ``make_params`` arguments (nx, ny and the
    model parameters of each domain; one storage form for all). ``domains``
    holds a ``Lattice`` view per domain for set-up, read-back and per-domain
    observables."""

    def __init__(self, specs, stream=None):
        import torch
        lib = _batch_lib()
        self.count = len(specs)
        arr = (lbm_params * self.count)(*[make_params(**sp) for sp in specs])
        self._params = arr
        nbytes = int(lib.lbm_batch_workspace_bytes(arr, self.count))
        if nbytes == 0:
            raise LbmError(LBM_EINVAL, "invalid batch parameters")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.stream.device)
        h = ctypes.c_void_p()
        st = lib.lbm_batch_create(arr, self.count, ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if st != LBM_OK:
            raise LbmError(st, "lbm_batch_create failed")
        self.handle = h
        self.domains = []
        for i, sp in enumerate(specs):
            ctx = ctypes.c_void_p(lib.lbm_batch_domain(h, i))
            sp = dict(sp)
            nx, ny = sp.pop("nx"), sp.pop("ny")
            self.domains.append(Lattice(nx, ny, stream=self.stream, _ctx=ctx, _owner=self, **sp))

    def _check(self, st):
        if st != LBM_OK:
            raise LbmError(st, _batch_lib().lbm_batch_last_error(self.handle).decode())

    def step(self, n: int = 1):
        self._check(_batch_lib().lbm_batch_step(self.handle, int(n)))

    def observables(self, check_finite: bool = True) -> list:
        """Per-domain observables; a non-finite domain raises unless
        check_finite is False (its ``nonfinite`` count then tells)."""
        out = (lbm_obs * self.count)()
        st = _batch_lib().lbm_batch_observables(self.handle, out)
        if not (st == LBM_ENAN and not check_finite):
            self._check(st)
        return [o.as_dict() for o in out]

    def set_active(self, flags):
        a = (ctypes.c_uint8 * self.count)(*[1 if f else 0 for f in flags])
        self._check(_batch_lib().lbm_batch_set_active(self.handle, a))

    def set_tile_rows(self, rows: int):
        self._check(_batch_lib().lbm_batch_set_tile_rows(self.handle, int(rows)))

    @property
    def tile_rows(self) -> int:
        return int(_batch_lib().lbm_batch_tile_rows(self.handle))

    def autotune(self, candidates=(8, 16, 32, 64), steps: int = 10):
        c = (ctypes.c_int32 * len(candidates))(*candidates)
        ms = (ctypes.c_double * len(candidates))()
        chosen = ctypes.c_int32()
        self._check(_batch_lib().lbm_batch_autotune(self.handle, c, len(candidates), int(steps),
                                                    ctypes.byref(chosen), ms))
        return int(chosen.value), list(ms)

    def set_ctas_per_sm(self, ctas: int):
        self._check(_batch_lib().lbm_batch_set_ctas_per_sm(self.handle, int(ctas)))

    @property
    def ctas_per_sm(self) -> int:
        return int(_batch_lib().lbm_batch_ctas_per_sm(self.handle))

    def autotune_grid(self, rows=(16, 32, 64, 128), ctas=(2, 3), steps: int = 10):
        """Tile height x CTAs per SM; returns (rows, ctas, {(rows, ctas): ms per step})."""
        r = (ctypes.c_int32 * len(rows))(*rows)
        c = (ctypes.c_int32 * len(ctas))(*ctas)
        ms = (ctypes.c_double * (len(rows) * len(ctas)))()
        cr, cc = ctypes.c_int32(), ctypes.c_int32()
        self._check(_batch_lib().lbm_batch_autotune_grid(self.handle, r, len(rows), c, len(ctas), int(steps),
                                                         ctypes.byref(cr), ctypes.byref(cc), ms))
        table = {(rows[i], ctas[j]): ms[j * len(rows) + i] for j in range(len(ctas)) for i in range(len(rows))}
        return int(cr.value), int(cc.value), table

    def run_to_steady(self, rel_tol=1e-7, check_every=1000, max_steps=10 ** 6):
        steps = (ctypes.c_int64 * self.count)()
        out = (lbm_obs * self.count)()
        st = _batch_lib().lbm_batch_run_to_steady(self.handle, float(rel_tol), int(check_every),
                                                  int(max_steps), steps, out)
        if st not in (LBM_OK, LBM_ENOTCONV, LBM_ENAN):
            self._check(st)
        # steps: -1 not steady within max_steps, -2 became non-finite
        return list(steps), [o.as_dict() for o in out], st == LBM_OK

    def close(self):
        if getattr(self, "handle", None):
            for d in self.domains:
                d.ctx = None
            _batch_lib().lbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
