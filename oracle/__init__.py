"""FP64 CPU oracle for the D2Q9 Shan-Chen electrowetting update.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers. The CUDA library never
imports, links or runs anything here, and this package imports nothing from
the CUDA library.

The arithmetic lives in ``lbm_oracle.c`` (one lattice-wide loop per phase of
the paper's update, double precision); this module compiles it with gcc and
marshals numpy arrays through ctypes. Arrays use the paper's direction order
(D2Q9 paragraph): populations ``f[a, y, x]`` with shape ``(9, ny, nx)``,
masks ``solid[y, x]`` (uint8, 1 = solid).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblbm_oracle.so")

GREEN_MC = 0        # Martys-Chen magnitudes: G on axis links, G/2 on diagonals
GREEN_PRINTED = 1   # weights as printed with Eq. 4: 2G on axis links, G on diagonals
NORMAL_FACES = 0    # electric force f per solid axis face (a corner gets both faces)
NORMAL_UNIT = 1     # electric force f along the unit sum of the face directions

# D2Q9 velocity set in the paper's order.
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])
WEIGHTS = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


@dataclasses.dataclass
class Params:
    """Model parameters (names follow the paper; defaults are its droplet run
    except tau, which the benchmark configurations fix at 1.0)."""
    nx: int
    ny: int
    tau: float = 1.0
    G: float = -0.52
    G_wall: float = -0.14
    rho0: float = 1.0
    rho_c: float = 1.0
    f_elec: float = 0.0
    body_fx: float = 0.0
    body_fy: float = 0.0
    green: int = GREEN_MC
    normal: int = NORMAL_FACES


class _CParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("tau", ctypes.c_double), ("G", ctypes.c_double), ("G_wall", ctypes.c_double),
        ("rho0", ctypes.c_double), ("rho_c", ctypes.c_double), ("f_elec", ctypes.c_double),
        ("body_fx", ctypes.c_double), ("body_fy", ctypes.c_double),
        ("green", ctypes.c_int32), ("normal", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into a shared library (gcc -O3, OpenMP).

    ISO C mode and -ffp-contract=off keep every operation a separately
    rounded IEEE double operation (no fused multiply-adds), so the results
    are the same on x86-64 and AArch64 hosts; no -march=native for the same
    reason."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-Wall",
                    "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None
_lock = threading.Lock()


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_CParams)
            d = ctypes.POINTER(ctypes.c_double)
            u8 = ctypes.POINTER(ctypes.c_uint8)
            lib.orc_equilibrium.argtypes = [P, u8, d, d, d, d]
            lib.orc_step.argtypes = [P, u8, d, ctypes.c_int64]
            lib.orc_fields.argtypes = [P, u8, d, d, d, d]
            lib.orc_forces.argtypes = [P, u8, d, d, d, d, d]
            lib.orc_observables.argtypes = [P, u8, d, d]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            for fn in (lib.orc_equilibrium, lib.orc_step, lib.orc_fields, lib.orc_forces,
                       lib.orc_observables, lib.orc_set_threads):
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _cp(p: Params) -> _CParams:
    return _CParams(p.nx, p.ny, p.tau, p.G, p.G_wall, p.rho0, p.rho_c, p.f_elec,
                    p.body_fx, p.body_fy, p.green, p.normal)


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _mask(p: Params, solid) -> np.ndarray:
    s = np.ascontiguousarray(solid, dtype=np.uint8)
    if s.shape != (p.ny, p.nx):
        raise ValueError(f"mask shape {s.shape} != {(p.ny, p.nx)}")
    return s


def _u8ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops (timing only); returns the count in effect."""
    return int(_load().orc_set_threads(int(n)))


def equilibrium(p: Params, solid, rho, ux, uy) -> np.ndarray:
    """Eq. 3 at every node; returns f of shape (9, ny, nx), zero on solids."""
    s = _mask(p, solid)
    r, x, y = (np.ascontiguousarray(np.broadcast_to(v, (p.ny, p.nx)), dtype=np.float64)
               for v in (rho, ux, uy))
    f = np.zeros((9, p.ny, p.nx))
    _check(_load().orc_equilibrium(ctypes.byref(_cp(p)), _u8ptr(s), _dptr(r), _dptr(x),
                                   _dptr(y), _dptr(f)), "equilibrium")
    return f


def step(p: Params, solid, f: np.ndarray, nsteps: int) -> np.ndarray:
    """Return f advanced by ``nsteps`` time steps (input left untouched)."""
    s = _mask(p, solid)
    out = np.array(f, dtype=np.float64, order="C", copy=True)
    if out.shape != (9, p.ny, p.nx):
        raise ValueError("f must have shape (9, ny, nx)")
    _check(_load().orc_step(ctypes.byref(_cp(p)), _u8ptr(s), _dptr(out), int(nsteps)), "step")
    return out


def fields(p: Params, solid, f: np.ndarray):
    """Density and physical velocity (j + F/2)/rho of the current state."""
    s = _mask(p, solid)
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho, ux, uy = (np.zeros((p.ny, p.nx)) for _ in range(3))
    _check(_load().orc_fields(ctypes.byref(_cp(p)), _u8ptr(s), _dptr(f), _dptr(rho),
                              _dptr(ux), _dptr(uy)), "fields")
    return rho, ux, uy


def forces(p: Params, solid, f: np.ndarray):
    """Moments and the four force terms of the current state.

    Returns (rho, jx, jy, terms) with terms of shape (8, ny, nx) ordered
    F_sigma (x, y), F_w (x, y), electric f_e (x, y), body F_b (x, y)."""
    s = _mask(p, solid)
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho, jx, jy = (np.zeros((p.ny, p.nx)) for _ in range(3))
    terms = np.zeros((8, p.ny, p.nx))
    _check(_load().orc_forces(ctypes.byref(_cp(p)), _u8ptr(s), _dptr(f), _dptr(rho),
                              _dptr(jx), _dptr(jy), _dptr(terms)), "forces")
    return rho, jx, jy, terms


def equilibrium_physical(p: Params, solid, rho, ux, uy) -> np.ndarray:
    """State whose density is rho and whose physical velocity (j + F/2)/rho
    (the velocity of Eq. 11's flux) is u: Eq. 3 evaluated at
    u - F/(2 rho), F the total force that the density field rho exerts
    (Eq. 5, Eq. 6, the electric force, the body force). The force depends on
    the density and the mask only, so it is read off the state f_eq(rho, 0)."""
    s = _mask(p, solid)
    r = np.ascontiguousarray(np.broadcast_to(rho, (p.ny, p.nx)), dtype=np.float64)
    _, _, _, t = forces(p, s, equilibrium(p, s, r, 0.0, 0.0))
    fx = t[0] + t[2] + t[4] + t[6]
    fy = t[1] + t[3] + t[5] + t[7]
    safe = np.where(s == 0, r, 1.0)
    return equilibrium(p, s, r, ux - 0.5 * fx / safe, uy - 0.5 * fy / safe)


def observables(p: Params, solid, f: np.ndarray) -> dict:
    """mass, flux Q (Eq. 11), momentum, max |u|, min rho, non-finite count."""
    s = _mask(p, solid)
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros(7)
    _check(_load().orc_observables(ctypes.byref(_cp(p)), _u8ptr(s), _dptr(f), _dptr(out)),
           "observables")
    return dict(mass=out[0], flux_Q=out[1], mom_x=out[2], mom_y=out[3], max_u=out[4],
                min_rho=out[5], nonfinite=int(out[6]))
