"""The one-kernel collide's launch shape is a tuning knob, not a numerical
one: every thread-block shape, one or two cells per thread (the two-cell
kernels run both collisions as packed FP32 pairs), one or eight z-planes
per thread, and pulls from global memory or from planes staged in shared
memory by bulk asynchronous copies, give bitwise the same populations and
forces.  The TGV box (48 x 34 x 30)
is narrower than a staged block's 144-cell rows and not a multiple of its
4 rows or 16 planes, so the staging wraps rows several times and runs
partial blocks.  Covers D3Q19 without markers (periodic and
bounce-back / Zou-He faces), the small wing pair with the IB band, and D2Q9
with walls and a cylinder."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

SHAPES = [(64, 4, 1), (64, 4, 2), (64, 4, 3), (32, 4, 3), (32, 8, 1), (128, 2, 1), (256, 1, 1), (64, 4, 0), (32, 1, 0), (128, 2, 0)]


def _run(ibl, cfg, shape, steps, bodies=0):
    ctx = ibl.from_workload(cfg)
    ctx.ibl_set_overlap(0)
    ctx.ibl_set_collide_shape(*shape)
    ctx.ibl_step(steps)
    out = [ctx.ibl_get_populations()] + [ctx.ibl_force_history(b, steps) for b in range(bodies)]
    ctx.close()
    return out


def _same(a, b):
    for x, y in zip(a, b):
        assert x.shape == y.shape
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", ["fp16dev", "bf16dev", "fp32", "fp64"])
def test_tgv_every_shape_bitwise(ibl, prec):
    cfg = {"lattice": 19, "tau": 0.6, "grid": W.grid(48, 34, 30, [W.PERIODIC] * 6, precision=prec),
           "bodies": [], "u_field": W.tgv3d_velocity(48, 34, 30, 0.05)}
    ref = _run(ibl, cfg, SHAPES[0], 30)
    for shape in SHAPES[1:]:
        _same(ref, _run(ibl, cfg, shape, 30))


FACES = {"zou_he_x": ([W.VEL_INLET, W.PRESS_OUTLET] + [W.PERIODIC] * 4, (0.03, 0.0, 0.0)),
         "walls_y": ([W.PERIODIC, W.PERIODIC, W.BOUNCEBACK, W.BOUNCEBACK, W.PERIODIC, W.PERIODIC], (0.0, 0.0, 0.0))}


@pytest.mark.parametrize("faces", sorted(FACES))
@pytest.mark.parametrize("prec", ["fp16dev", "bf16dev"])
def test_faces_pairs_vs_single_bitwise(ibl, prec, faces):
    """Zou-He inlet / outlet in x, or bounce-back walls in y: the pairs that
    touch a face run the one-cell gather, the others the packed collision."""
    bc, u_in = FACES[faces]
    force = (1e-5, 0.0, 0.0) if faces == "walls_y" else (0.0, 0.0, 0.0)   # channel flow between the walls
    g = W.grid(40, 26, 22, bc, u_in=u_in, body_force=force, precision=prec)
    cfg = {"lattice": 19, "tau": 0.7, "grid": g, "bodies": [], "u0": u_in}
    ref = _run(ibl, cfg, (64, 4, 2), 60)
    for shape in [(64, 2, 3), (64, 4, 1), (64, 4, 0)]:
        _same(ref, _run(ibl, cfg, shape, 60))


@pytest.mark.parametrize("prec", ["fp16dev", "bf16dev"])
def test_wings_pairs_vs_single_bitwise(ibl, prec):
    """The IB band's velocity correction and force write-back on both lanes."""
    cfg = W.clap_fling_3d(nx=48, ny=40, nz=40, chord=6.0, Re=5.0, J=0.1, period=1200.0, precision=prec)
    ref = _run(ibl, cfg, (64, 4, 2), 80, bodies=2)
    for shape in [(64, 2, 3), (64, 4, 1), (32, 4, 0)]:
        _same(ref, _run(ibl, cfg, shape, 80, bodies=2))


@pytest.mark.parametrize("prec", ["fp16dev", "bf16dev"])
def test_d2q9_cylinder_pairs_vs_single_bitwise(ibl, prec):
    cfg = W.cylinder_channel(nx=96, ny=50, diameter=10.0, center=(30.0, 25.0), m=31, precision=prec)
    ref = _run(ibl, cfg, (64, 4, 1), 80, bodies=1)
    for shape in [(64, 2, 3), (128, 1, 0)]:
        _same(ref, _run(ibl, cfg, shape, 80, bodies=1))


def test_bad_shapes_are_refused(ibl):
    ctx = ibl.from_workload({"lattice": 19, "tau": 0.6, "grid": W.grid(16, 16, 16, [W.PERIODIC] * 6),
                             "bodies": []})
    for shape in [(48, 4, 1), (64, 8, 1), (64, 0, 1), (32, 4, 4), (512, 1, 0), (64, 4, -1)]:
        with pytest.raises(ibl.IblError) as e:
            ctx.ibl_set_collide_shape(*shape)
        assert e.value.status == ibl.IBL_EINVAL
