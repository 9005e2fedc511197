"""Precision study: the error of every observable, for every population
storage form, against the FP64 oracle on a 1024 x 256 crop of the benchmark
workload (bottom rows of the droplet-row channel: rough wall, sessile
droplets, a top wall closing the crop, electric-force level 10, body force
1e-6), after 1000 steps.

Errors: relative L2 of the populations; relative mass; flux Q and momentum
x/y scaled by their sums of magnitudes (|dQ| / (sum |u_x| / nx), |dP| /
sum rho |u|); relative max |u| and min rho. Each storage form is held to the
stated bound of every quantity (about twice the value measured on a GB300);
the table is printed (pytest -s).
"""
import numpy as np
import pytest

import oracle
from paper_0708_4182_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

STEPS = 1000
QUANTITIES = ("pop_l2", "mass", "flux_Q", "mom_x", "mom_y", "max_u", "min_rho")
# stated bounds after 1000 steps, per storage form (measured on a GB300:
# fp32     7.5e-7 1.4e-7 7.3e-5 2.3e-5 9.3e-7 5.8e-7 4.2e-7
# fp32dev  5.2e-7 4.8e-8 1.7e-7 1.2e-7 7.7e-7 5.7e-7 4.6e-8
# fp16dev  2.9e-4 6.6e-8 1.9e-4 2.4e-4 1.5e-4 2.0e-4 6.3e-6
# bf16dev  1.6e-3 1.1e-7 2.0e-3 3.9e-4 1.1e-3 8.5e-2 5.0e-4)
BOUNDS = {
    "fp32": (2e-6, 5e-7, 2e-4, 5e-5, 2e-6, 2e-6, 1e-6),
    "fp32dev": (2e-6, 2e-7, 5e-7, 5e-7, 2e-6, 2e-6, 2e-7),
    "fp16dev": (6e-4, 2e-7, 5e-4, 5e-4, 3e-4, 5e-4, 2e-5),
    "bf16dev": (4e-3, 3e-7, 5e-3, 1e-3, 3e-3, 2e-1, 1e-3),
}


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0708_4182_gb300 import lbm as L
    L.load()
    return L


def crop_workload():
    full = wl.droplet_row_channel(nx=1024, ny=512, f_elec=wl.f_level(10))
    cy = 256
    mask = np.ascontiguousarray(full.mask[:cy])
    mask[-1, :] = 1
    rho = np.where(mask == 1, 0.0, full.rho[:cy])
    return mask, rho, full.params


def errors(lat, p, mask, f_ref):
    from tests.test_gpu_parity import pop_err
    _, _, l2 = pop_err(lat.populations(), f_ref, mask)
    o = lat.observables()
    r = oracle.observables(p, mask, f_ref)
    rho, ux, uy = oracle.fields(p, mask, f_ref)
    fl = mask == 0
    q_scale = np.abs(ux[fl]).sum() / p.nx
    px_scale = (rho[fl] * np.abs(ux[fl])).sum()
    py_scale = (rho[fl] * np.abs(uy[fl])).sum()
    return dict(pop_l2=l2, mass=abs(o["mass"] / r["mass"] - 1),
                flux_Q=abs(o["flux_Q"] - r["flux_Q"]) / q_scale,
                mom_x=abs(o["mom_x"] - r["mom_x"]) / px_scale,
                mom_y=abs(o["mom_y"] - r["mom_y"]) / py_scale,
                max_u=abs(o["max_u"] / r["max_u"] - 1), min_rho=abs(o["min_rho"] / r["min_rho"] - 1))


def test_precision_study_every_observable_every_storage(lbm):
    mask, rho, params = crop_workload()
    ny, nx = mask.shape
    p = oracle.Params(nx, ny, **params)
    f_ref = oracle.step(p, mask, oracle.equilibrium(p, mask, rho, 0, 0), STEPS)
    forms = {"fp32": lbm.LBM_FP32, "fp32dev": lbm.LBM_FP32_DEV, "fp16dev": lbm.LBM_FP16_DEV,
             "bf16dev": lbm.LBM_BF16_DEV}
    rows = {}
    for name, st in forms.items():
        lat = lbm.Lattice(nx, ny, storage=st, **params)
        lat.set_geometry(mask)
        lat.set_rho_u(rho)
        lat.step(STEPS)
        rows[name] = errors(lat, p, mask, f_ref)
    print("\nstorage  " + " ".join(f"{q:>9s}" for q in QUANTITIES))
    for name, e in rows.items():
        print(f"{name:8s} " + " ".join(f"{e[q]:9.2e}" for q in QUANTITIES))
    for name, e in rows.items():
        for q, bound in zip(QUANTITIES, BOUNDS[name]):
            assert e[q] <= bound, (name, q, e[q], bound)
