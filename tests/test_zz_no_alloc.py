"""The allocation-free mass entry point against ibl_mass (GPU).

ibl_mass_noalloc serves callers that may not allocate device memory after
start-up (real-time loops, where a cudaMalloc can block; device memory fully
claimed by another allocator, where it fails): it takes its partial sums from
a static device array instead of cudaMalloc.
This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _ctx(ibl):
    n = (29, 22, 17)
    cfg = {"lattice": 19, "tau": 0.7, "grid": W.grid(*n, [W.PERIODIC] * 6, precision="fp64"),
           "bodies": [], "u_field": W.tgv3d_velocity(*n, 0.03)}
    return ibl.from_workload(cfg)


def test_noalloc_mass_matches_ibl_mass_twice(ibl):
    ctx = _ctx(ibl)
    ctx.ibl_step(7)
    for _ in range(2):                      # two calls in a row share the static array
        ref = ctx.ibl_mass()
        same = ctx.ibl_mass_noalloc(1024)   # same chunking as ibl_mass: bitwise equal
        assert same == ref
        other = ctx.ibl_mass_noalloc(37)    # other chunking: equal to FP64 rounding
        assert abs(other - ref) <= 1e-12 * abs(ref)
        ctx.ibl_step(3)


def test_noalloc_mass_rejects_oversized_scratch(ibl):
    ctx = _ctx(ibl)
    with pytest.raises(ibl.IblError) as e:
        ctx.ibl_mass_noalloc(4097)
    assert e.value.status == ibl.IBL_EINVAL
    assert np.isfinite(ctx.ibl_mass_noalloc(4096))
