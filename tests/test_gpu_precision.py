"""Reduced-precision storage (f - w in FP16 or BF16, collision in FP32)
against the FP64 oracle (GPU).

Field bounds are the measured errors with a margin of 3-5x.  Coefficient
errors use the per-step scale of tests/parity.py (each step against its own
force scale, floored at the largest one after the start-up); FP16 is held
to 5e-4 (measured 1.2e-4) and BF16 to 1e-3, the C_L target of the
reduced-precision form.  FP16 rounds each stored
deviation to 2^-11 relative, BF16 to 2^-8, so field errors of ~1e-4..1e-3
(FP16) and ~1e-3..1e-2 (BF16) after hundreds of steps are the arithmetic's
own floor, not a defect."""
import numpy as np
import pytest

import workloads as W
from tests.parity import coef_err, oracle_from_workload, rel_err

pytestmark = pytest.mark.gpu

WINGS = dict(nx=48, ny=40, nz=40, chord=6.0, Re=5.0, J=0.1, period=1200.0)
BOUNDS_WINGS = {"fp16dev": (1e-3, 5e-4), "bf16dev": (6e-3, 1e-3)}
BOUNDS_TGV = {"fp16dev": 3e-3, "bf16dev": 3e-2}


@pytest.fixture(scope="module")
def wings_oracle():
    sim = oracle_from_workload(W.clap_fling_3d(**WINGS))
    sim.step(600)
    return sim


@pytest.mark.parametrize("prec", ["fp16dev", "bf16dev"])
def test_wings_reduced_precision(ibl, wings_oracle, prec):
    sim = wings_oracle
    ctx = ibl.from_workload(W.clap_fling_3d(precision=prec, **WINGS))
    ctx.ibl_step(600)
    u = ctx.ibl_get_field(ibl.IBL_FIELD_U, allow=(ibl.IBL_ENOTCONV,))
    eu = rel_err(u, sim.fields()[1])
    worst = 0.0
    for b in range(2):
        h = ctx.ibl_force_history(b, 600)
        ref = np.array(sim.history[b])
        worst = max(worst, *coef_err(h[:, :2], ref[:, :2]))
    print(f"{prec} wings 600 steps: u {eu:.2e}, C_L/C_T {worst:.2e}")
    tol_u, tol_c = BOUNDS_WINGS[prec]
    assert eu < tol_u and worst < tol_c


@pytest.mark.parametrize("n", [(40, 36, 34), (41, 36, 34)])   # even nx: two cells per thread
@pytest.mark.parametrize("prec", ["fp16dev", "bf16dev"])
def test_tgv_reduced_precision(ibl, prec, n):
    base = {"lattice": 19, "tau": 0.6, "bodies": [], "u_field": W.tgv3d_velocity(*n, 0.05)}
    sim = oracle_from_workload(dict(base, grid=W.grid(*n, [W.PERIODIC] * 6)))
    sim.step(600)
    ctx = ibl.from_workload(dict(base, grid=W.grid(*n, [W.PERIODIC] * 6, precision=prec)))
    ctx.ibl_step(600)
    eu = rel_err(ctx.ibl_get_field(ibl.IBL_FIELD_U), sim.fields()[1])
    print(f"{prec} TGV 600 steps: u {eu:.2e}")
    assert eu < BOUNDS_TGV[prec]
