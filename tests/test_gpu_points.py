"""GPU parity of the stand-alone IB transfers on point clouds (Eqs. 15, 17).

Interpolation of rho and u* (Eq. 11 with the uniform body force) from the
current populations, and spreading of point values onto the grid, compared
with the oracle's sparse delta products on seeded random clouds that
straddle periodic faces and come close to walls; at 256^3 with 1e5 points
on sampled points and cells and by the partition-of-unity sum.  Every call
goes through the C ABI.
"""
import numpy as np
import pytest

import workloads as W
from oracle import ib as oib
from oracle import lbm as olbm
from oracle.lattice import get as get_lattice
from tests.parity import gpu_to_oracle_order, oracle_from_workload, rel_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FIX_QUANTUM = 2.0 ** -46       # resolution of the spreading's fixed-point sums


def _pair(ibl, q, prec, shape, bc, steps, seed=5):
    """GPU context and oracle simulation from the same random populations."""
    rng = np.random.default_rng(seed)
    lat = get_lattice(q)
    grid = W.grid(shape[2], shape[1], shape[0], bc, body_force=(2e-5, -1e-5, 5e-6), precision=prec)
    cfg = {"lattice": q, "tau": 0.7, "grid": grid, "bodies": []}
    f_ora = lat.w[:, None, None, None] * (1 + 0.05 * rng.uniform(-1, 1, size=(q,) + shape))
    ctx = ibl.from_workload(cfg, init=False)
    perm = gpu_to_oracle_order(ibl, q)
    f_gpu = np.empty_like(f_ora)
    f_gpu[perm] = f_ora
    ctx.ibl_set_populations(f_gpu)
    sim = oracle_from_workload(cfg)
    sim.set_populations(f_ora)
    if steps:
        ctx.ibl_step(steps)
        ctx.ibl_sync()
        sim.step(steps)
    return ctx, sim


def _cloud(m, shape, periodic, seed=9):
    """Points over periodic axes (including just outside [0, n)) and inside walls."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    n = [nx, ny, nz]
    X = np.zeros((m, 3))
    for a in range(3 if nz > 1 else 2):
        if periodic[a]:
            X[:, a] = rng.uniform(-1.0, n[a] + 1.0, size=m)
        else:
            X[:, a] = rng.uniform(1.0, n[a] - 2.0, size=m)
    return X


def _oracle_moments(sim):
    rho = olbm.density(sim.f)
    ustar = (olbm.momentum(sim.lat, sim.f) + 0.5 * sim.G[:, None, None, None]) / rho
    return rho, ustar


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


CASES = [
    (19, "fp64", (13, 11, 21), [W.PERIODIC, W.PERIODIC, W.BOUNCEBACK, W.BOUNCEBACK, W.PERIODIC, W.PERIODIC]),
    (19, "fp32", (13, 11, 21), [W.PERIODIC] * 6),
    (9, "fp64", (1, 23, 37), [W.PERIODIC, W.PERIODIC, W.BOUNCEBACK, W.BOUNCEBACK, 0, 0]),
    (19, "fp64", (12, 10, 20), [W.VEL_INLET, W.PRESS_OUTLET, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC]),
]


@pytest.mark.parametrize("q,prec,shape,bc", CASES)
@pytest.mark.parametrize("steps", [0, 2])
def test_interpolate_points_matches_oracle(ibl, q, prec, shape, bc, steps):
    ctx, sim = _pair(ibl, q, prec, shape, bc, steps)
    d = sim.lat.d
    periodic = [bc[2 * a] == W.PERIODIC for a in range(3)]
    if bc[0] == W.VEL_INLET:       # keep stencils off the inlet/outlet faces
        periodic[0] = False
    X = _cloud(300, shape, periodic)
    U, rho = ctx.ibl_interpolate_points(_dev(X))
    rho_o, ustar = _oracle_moments(sim)
    Dm = oib.spread_matrix(X[:, :d], shape, sim.periodic)
    u_o = oib.interpolate(Dm, ustar)
    r_o = oib.interpolate(Dm, rho_o[None])[:, 0]
    tol = 1e-13 if prec == "fp64" else 1e-5
    assert rel_err(U.cpu().numpy(), u_o) < tol
    assert np.abs(rho.cpu().numpy() - r_o).max() < tol


@pytest.mark.parametrize("q,prec,shape,bc", CASES)
@pytest.mark.parametrize("steps", [0, 2])
def test_interpolate_cached_moments_bitwise(ibl, q, prec, shape, bc, steps):
    """A cloud with as many stencil nodes as cells takes the moments-first
    path (every cell's rho, u* formed once); small clouds pull at every
    node.  Both give bitwise the same values: 300 points at once against
    the same points 20 at a time."""
    ctx, _ = _pair(ibl, q, prec, shape, bc, steps)
    periodic = [bc[2 * a] == W.PERIODIC for a in range(3)]
    if bc[0] == W.VEL_INLET:
        periodic[0] = False
    X = _cloud(300, shape, periodic, seed=21)
    nodes = 64 if q == 19 else 16
    n_cells = shape[0] * shape[1] * shape[2]
    assert 300 * nodes >= n_cells > 20 * nodes
    U, rho = ctx.ibl_interpolate_points(_dev(X))
    parts = [ctx.ibl_interpolate_points(_dev(X[k:k + 20])) for k in range(0, 300, 20)]
    assert torch.equal(U, torch.cat([p[0] for p in parts]))
    assert torch.equal(rho, torch.cat([p[1] for p in parts]))


@pytest.mark.parametrize("q,prec,shape,bc", CASES[:3])
def test_spread_points_matches_oracle(ibl, q, prec, shape, bc):
    ctx, sim = _pair(ibl, q, prec, shape, bc, 0)
    d = sim.lat.d
    periodic = [bc[2 * a] == W.PERIODIC for a in range(3)]
    X = _cloud(400, shape, periodic, seed=13)
    rng = np.random.default_rng(17)
    V = rng.uniform(-0.05, 0.05, size=(400, d))
    ds = rng.uniform(0.5, 1.5, size=400)
    out = ctx.ibl_spread_points(_dev(X), _dev(V), _dev(ds))
    Dm = oib.spread_matrix(X[:, :d], shape, sim.periodic)
    ref = oib.spread(Dm, V, ds, shape)
    assert out.shape == ref.shape
    assert rel_err(out.cpu().numpy(), ref) < 1e-10
    again = ctx.ibl_spread_points(_dev(X), _dev(V), _dev(ds))
    assert torch.equal(out, again), "fixed-point spreading must be bitwise reproducible"


def test_point_operators_reject_stencils_through_walls(ibl):
    shape = (1, 23, 37)
    bc = [W.PERIODIC, W.PERIODIC, W.BOUNCEBACK, W.BOUNCEBACK, 0, 0]
    ctx, _ = _pair(ibl, 9, "fp64", shape, bc, 1)
    good = np.array([[5.0, 10.0, 0.0]])
    for bad in ([5.0, 0.5, 0.0], [5.0, 21.5, 0.0], [np.nan, 10.0, 0.0]):
        X = _dev(np.array([bad]))
        with pytest.raises(ibl.IblError) as e:
            ctx.ibl_interpolate_points(X)
        assert e.value.status == ibl.IBL_EINVAL
        with pytest.raises(ibl.IblError) as e:
            ctx.ibl_spread_points(X, _dev(np.ones((1, 2))), _dev(np.ones(1)))
        assert e.value.status == ibl.IBL_EINVAL
    # the context stays usable and the flag is cleared
    U, rho = ctx.ibl_interpolate_points(_dev(good))
    assert np.isfinite(U.cpu().numpy()).all()
    ctx.ibl_step(1)
    ctx.ibl_sync()
    empty = ctx.ibl_interpolate_points(_dev(np.zeros((0, 3))))
    assert empty[0].shape == (0, 2)


def test_points_full_size_sampled(ibl):
    """256^3 periodic D3Q19 FP32 at rest state of a Taylor-Green field, 1e5 points.

    Right after initialisation u* is the initial field at every node, so the
    interpolated values of sampled points follow from the oracle's stencil
    weights applied to that field; spreading is checked on sampled cells by
    brute force over all points and by the exact total sum_l V_l ds_l.
    """
    n, m = 256, 100_000
    u0 = W.tgv3d_velocity(n, n, n, 0.05)
    grid = W.grid(n, n, n, [W.PERIODIC] * 6, precision="fp32")
    cfg = {"lattice": 19, "tau": 0.6, "grid": grid, "bodies": [], "u_field": u0}
    ctx = ibl.from_workload(cfg)
    X, V = W.random_markers(m, n, 2.0, n - 2.0, 0.05)
    ds = np.ones(m)
    U, rho = ctx.ibl_interpolate_points(_dev(X))
    U = U.cpu().numpy()
    rho = rho.cpu().numpy()
    rng = np.random.default_rng(21)
    pick = rng.choice(m, 256, replace=False)
    per = [True, True, True]
    nodes, wts = zip(*[oib.stencil_1d(X[pick, a], n, per[a]) for a in range(3)])
    ref = np.zeros((len(pick), 3))
    for i in range(4):
        for j in range(4):
            for k in range(4):
                w = wts[0][:, i] * wts[1][:, j] * wts[2][:, k]
                ref += w[:, None] * u0[:, nodes[2][:, k], nodes[1][:, j], nodes[0][:, i]].T
    assert rel_err(U[pick], ref) < 1e-5
    assert np.abs(rho - 1.0).max() < 1e-6
    del U

    Vt = _dev(V)
    out = ctx.ibl_spread_points(_dev(X), Vt, _dev(ds))
    tot = out.sum(dim=(1, 2, 3)).cpu().numpy()
    assert np.abs(tot - V.sum(axis=0)).max() < 64 * m * FIX_QUANTUM
    cells = np.stack([np.floor(X[pick[:64], a]).astype(int) for a in range(3)], axis=1)
    got = out[:, cells[:, 2], cells[:, 1], cells[:, 0]].cpu().numpy().T
    want = np.zeros_like(got)
    for c, (cx, cy, cz) in enumerate(cells):
        r = [cx - X[:, 0], cy - X[:, 1], cz - X[:, 2]]
        r = [v - n * np.round(v / n) for v in r]
        w = oib.phi(r[0]) * oib.phi(r[1]) * oib.phi(r[2])
        want[c] = (w[:, None] * V).sum(axis=0)
    assert np.abs(got - want).max() < 1e-11
