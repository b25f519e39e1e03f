"""Shared helpers of the GPU-vs-oracle parity tests.

Relative error of a field (the reading of "max relative error" used
throughout): ||x_gpu - x_oracle||_inf / ||x_oracle||_inf, per field;
pointwise relative error is meaningless where the field crosses zero.
"""
from __future__ import annotations

import numpy as np

from oracle.lattice import get as get_lattice
from oracle.sim import Simulation

# Tolerances.  FP32 storage: the field and coefficient bounds of the method's
# FP32 target (fields 1e-5 after 1000 steps, C_L / C_T 1e-4).  FP64: both
# sides compute in FP64; the GPU's iterative IB solve stops at a relative
# field residual of 1e-10, so fields agree to ~1e-9 after many steps.
TOL_FIELD_FP32 = 1e-5
TOL_COEF_FP32 = 1e-4
TOL_FIELD_FP64 = 1e-9
TOL_FIELD_FP64_LBM = 1e-12


def rel_err(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / (den if den > 0 else 1.0))


def oracle_from_workload(cfg: dict, u_field=None) -> Simulation:
    sim = Simulation(cfg["lattice"], cfg["grid"], cfg["tau"])
    lat = get_lattice(cfg["lattice"])
    if u_field is not None:
        sim.init_fluid(u=np.asarray(u_field)[:lat.d])
    elif "u_field" in cfg:
        sim.init_fluid(u=np.asarray(cfg["u_field"])[:lat.d])
    else:
        sim.init_fluid(u=np.asarray(cfg.get("u0", (0.0, 0.0, 0.0)))[:lat.d])
    for b in cfg.get("bodies", []):
        sim.add_body(b)
    if "reference" in cfg:
        r = cfg["reference"]
        sim.set_reference(r["U_ref"], r["L"], r.get("rho_ref", 1.0))
    return sim


def gpu_to_oracle_order(ibl, q: int):
    """perm with f_oracle[i] = f_gpu[perm[i]] (directions matched by velocity vector)."""
    c_gpu, _ = ibl.lattice_velocities(q)
    lat = get_lattice(q)
    idx = {tuple(v): i for i, v in enumerate(c_gpu.tolist())}
    return np.array([idx[tuple(v)] for v in lat.c.tolist()])


def compare_fields(ctx, sim, ibl, tol_u, tol_rho=None):
    rho_g = ctx.ibl_get_field(ibl.IBL_FIELD_RHO)
    u_g = ctx.ibl_get_field(ibl.IBL_FIELD_U)
    rho_o, u_o = sim.fields()
    eu = rel_err(u_g, u_o)
    er = rel_err(rho_g, rho_o)
    assert np.isfinite(u_g).all()
    assert eu < tol_u, f"u rel err {eu:.3e} >= {tol_u:.1e}"
    assert er < (tol_rho if tol_rho is not None else tol_u), f"rho rel err {er:.3e}"
    return eu, er
