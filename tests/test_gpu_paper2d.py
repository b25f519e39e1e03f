"""GPU parity on the paper's own 2D cases, through the C ABI.

* Clap and fling (Sec. 3.3): two elliptic foils of chord/thickness 5 hinged
  at their trailing edges, gap c/2, opening per reading R8, in a 50c x 25c
  box with a Zou-He velocity inlet and pressure outlet (chord 16 here).
* Figure-eight hovering (Sec. 3.2, Eqs. 20-22): one foil of chord/thickness
  7.5 pitching about its centre while sweeping along a stroke plane at 60
  degrees, fluid at rest in a periodic 50c x 25c box.
* Stationary cylinder (Sec. 3.1): D = 8 in a 50D x 50D box, Zou-He velocity
  inlet and pressure outlet, Re = 20.

The oracle runs each case once (D2Q9 FP64, dense direct solve); the GPU runs
it in FP64 and in FP32 storage.
"""
import numpy as np
import pytest

import workloads as W
from tests.parity import (TOL_COEF_FP32, TOL_FIELD_FP32, TOL_FIELD_FP64, coef_err, compare_fields,
                          oracle_from_workload)

pytestmark = pytest.mark.gpu

STEPS = 120


def _cases():
    return {
        "clap_fling": lambda prec: W.clap_fling_2d(chord=16.0, Re=50.0, J=1.67e-3, period=800.0,
                                                   precision=prec),
        "figure_eight": lambda prec: W.figure_eight_2d(chord=16.0, Re=75.0, period=2000.0, precision=prec),
        "cylinder_50d": lambda prec: W.cylinder_50d(diameter=8.0, Re=20.0, u_in=0.05, precision=prec),
    }


@pytest.fixture(scope="module")
def oracle_runs():
    runs = {}
    for name, make in _cases().items():
        sim = oracle_from_workload(make("fp64"))
        sim.step(STEPS)
        runs[name] = sim
    return runs


def _coef_err(ctx, sim, body):
    hist = ctx.ibl_force_history(body, STEPS)
    ref = np.array(sim.history[body][-len(hist):])
    return coef_err(hist[:, :2], ref[:, :2])


@pytest.mark.parametrize("name", ["clap_fling", "figure_eight", "cylinder_50d"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_paper_2d_case(ibl, oracle_runs, name, prec):
    cfg = _cases()[name](prec)
    sim = oracle_runs[name]
    ctx = ibl.from_workload(cfg)
    ctx.ibl_step(STEPS)
    tol_f, tol_c = (TOL_FIELD_FP64, 1e-7) if prec == "fp64" else (TOL_FIELD_FP32, TOL_COEF_FP32)
    eu, er = compare_fields(ctx, sim, ibl, tol_f)
    worst = 0.0
    for b in range(len(cfg["bodies"])):
        worst = max(worst, *_coef_err(ctx, sim, b))
    print(f"{name} {prec} {STEPS} steps: u {eu:.2e} rho {er:.2e} coef {worst:.2e}")
    assert worst < tol_c
    if name == "clap_fling":
        # mirror symmetry about the mid-plane: equal and opposite lateral lifts
        hist = np.array(ctx.ibl_force_history(0, STEPS)), np.array(ctx.ibl_force_history(1, STEPS))
        scale = np.abs(hist[0][:, 0]).max()
        assert np.abs(hist[0][:, 0] - hist[1][:, 0]).max() < (1e-9 if prec == "fp64" else 1e-4) * scale


PERIOD = 800


@pytest.fixture(scope="module")
def clap_fling_period_oracle():
    sim = oracle_from_workload(_cases()["clap_fling"]("fp64"))
    sim.step(PERIOD)
    return sim


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_clap_fling_full_period(ibl, clap_fling_period_oracle, prec):
    """One whole flapping period of the paper's 2D clap and fling (Sec. 3.3,
    the span of its force histories): two claps and two flings, 800 steps.
    C_L / C_T of both foils at every step and the final fields against the
    oracle; the foils' lifts stay mirror images of each other."""
    sim = clap_fling_period_oracle
    cfg = _cases()["clap_fling"](prec)
    ctx = ibl.from_workload(cfg)
    ctx.ibl_step(PERIOD)
    tol_f, tol_c = (TOL_FIELD_FP64, 1e-7) if prec == "fp64" else (TOL_FIELD_FP32, TOL_COEF_FP32)
    eu, er = compare_fields(ctx, sim, ibl, tol_f)
    hist = []
    worst = 0.0
    for b in range(2):
        h = np.array(ctx.ibl_force_history(b, PERIOD))
        ref = np.array(sim.history[b][-PERIOD:])
        worst = max(worst, *coef_err(h[:, :2], ref[:, :2]))
        hist.append(h)
    print(f"clap_fling {prec} one period ({PERIOD} steps): u {eu:.2e} rho {er:.2e} coef {worst:.2e}; "
          f"mean C_T {hist[0][:, 1].mean():.4f}, max C_L {hist[0][:, 0].max():.4f}")
    assert worst < tol_c
    scale = np.abs(hist[0][:, 0]).max()
    assert np.abs(hist[0][:, 0] - hist[1][:, 0]).max() < (1e-9 if prec == "fp64" else 1e-4) * scale
