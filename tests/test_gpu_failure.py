"""Failure detection on the GPU, with every failure made on the host (no
device fault, trap or hang): a NaN written into the populations, mass drift
under FP16 storage against a deliberately tight bound, and the FP64 mass
check on conserving runs, with its totals against the oracle's sum of rho."""
import numpy as np
import pytest

import workloads as W
from tests.parity import oracle_from_workload

pytestmark = pytest.mark.gpu

N = (24, 20, 18)


def _tgv(prec):
    return {"lattice": 19, "tau": 0.6, "grid": W.grid(*N, [W.PERIODIC] * 6, precision=prec), "bodies": [],
            "u_field": W.tgv3d_velocity(*N, 0.05)}


def test_nan_in_the_populations_is_a_sticky_divergence(ibl):
    ctx = ibl.from_workload(_tgv("fp32"))
    ctx.ibl_step(3)
    f = ctx.ibl_get_populations()
    f[5, 7, 11, 13] = np.nan                  # one population of one cell
    ctx.ibl_set_populations(f)
    ctx.ibl_step(1)                           # asynchronous: the error surfaces at the next sync
    with pytest.raises(ibl.IblError) as e:
        ctx.ibl_sync()
    assert e.value.status == ibl.IBL_EDIVERGED
    for call in (lambda: ctx.ibl_step(1), ctx.ibl_sync, lambda: ctx.ibl_get_field(ibl.IBL_FIELD_U)):
        with pytest.raises(ibl.IblError) as e:
            call()
        assert e.value.status == ibl.IBL_EDIVERGED


def test_mass_check_flags_drift_beyond_its_bound(ibl):
    """FP16 deviation storage rounds every stored population, so the total
    mass drifts by ~1e-8 relative per step: with a 1e-13 bound the first
    check flags it, with the default 1e-2 bound nothing is flagged."""
    ctx = ibl.from_workload(_tgv("fp16dev"))
    ctx.ibl_set_mass_check(5, 1e-13)
    ctx.ibl_step(5)
    with pytest.raises(ibl.IblError) as e:
        ctx.ibl_sync()
    assert e.value.status == ibl.IBL_EDIVERGED
    m0, m1, n = ctx.ibl_mass_check_read(allow=(ibl.IBL_EDIVERGED,))
    assert n == 1 and abs(m1 - m0) > 1e-13 * m0
    ok = ibl.from_workload(_tgv("fp16dev"))
    ok.ibl_set_mass_check(5, 0.0)
    ok.ibl_step(200)
    ok.ibl_sync()
    m0, m1, n = ok.ibl_mass_check_read()
    assert n == 40 and abs(m1 - m0) < 1e-2 * m0


def test_mass_check_totals_match_the_oracle(ibl):
    """FP64 storage conserves mass to rounding: 40 checks pass at the default
    1e-9 bound, and the check's totals and ibl_mass equal the oracle's sum of
    rho, initially and after 200 steps."""
    cfg = _tgv("fp64")
    ctx = ibl.from_workload(cfg)
    sim = oracle_from_workload(cfg)
    m_init = float(sim.fields()[0].sum())
    ctx.ibl_set_mass_check(5, 0.0)
    ctx.ibl_step(200)
    sim.step(200)
    ctx.ibl_sync()
    m0, m1, n = ctx.ibl_mass_check_read()
    m_end = float(sim.fields()[0].sum())
    assert n == 40
    assert abs(m0 - m_init) < 1e-13 * m_init
    assert abs(m1 - m_end) < 1e-13 * m_end
    assert abs(ctx.ibl_mass() - m_end) < 1e-13 * m_end
    assert abs(m1 - m0) < 1e-12 * m0
