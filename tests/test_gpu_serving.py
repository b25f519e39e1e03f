"""Serving form: continuous batching of clap-and-fling runs (GPU).

A run's result must not depend on what else is running: the same request
alone and inside a mix of concurrent, later-arriving runs gives bitwise the
same force statistics.  The server's runs also match a direct run of the
same wing pair through the plain C ABI."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

REQ = dict(nx=64, ny=48, nz=48, chord=6.0, Re=20.0, period=600.0, J=1e-2, precision="fp32", steps=150)
OTHERS = [dict(nx=72, ny=48, nz=48, chord=6.0, Re=10.0, period=400.0, J=0.1, precision="fp16dev", steps=120),
          dict(nx=64, ny=56, nz=48, chord=7.0, Re=30.0, period=800.0, J=1e-3, precision="fp32", steps=200),
          dict(nx=48, ny=48, nz=40, chord=6.0, Re=15.0, period=500.0, J=2e-2, precision="bf16dev", steps=100)]


def _keys(r):
    return (tuple(r["CL_max"]), tuple(r["CL_mean"]), tuple(r["CT_max"]), tuple(r["CT_mean"]),
            tuple(r["CL_last"]), tuple(r["CT_last"]))


def test_result_is_the_same_alone_and_in_the_mix(ibl):
    alone = ibl.Server(hbm_budget_bytes=8 << 30, max_active=4, chunk_steps=25)
    rid = alone.ibl_server_submit(**REQ)
    alone.ibl_server_wait_all(600)
    ra = alone.ibl_server_poll(rid)
    alone.close()
    assert ra["done"] and ra["status"] == ibl.IBL_OK

    mix = ibl.Server(hbm_budget_bytes=8 << 30, max_active=3, chunk_steps=25)
    ids = [mix.ibl_server_submit(**OTHERS[0])]
    time.sleep(0.05)
    rid = mix.ibl_server_submit(**REQ)                  # arrives while another run is active
    for o in OTHERS[1:]:
        time.sleep(0.02)
        ids.append(mix.ibl_server_submit(**o))         # arrive later, queue behind max_active
    mix.ibl_server_wait_all(600)
    rm = mix.ibl_server_poll(rid)
    others = [mix.ibl_server_poll(i) for i in ids]
    stats = mix.ibl_server_stats()
    mix.close()
    assert rm["done"] and rm["status"] == ibl.IBL_OK
    assert _keys(ra) == _keys(rm)
    assert all(o["done"] for o in others) and stats["finished"] == 4 and stats["hbm_in_use"] == 0


def test_server_run_matches_a_direct_run(ibl):
    srv = ibl.Server(hbm_budget_bytes=8 << 30, max_active=2, chunk_steps=40)
    rid = srv.ibl_server_submit(**REQ)
    srv.ibl_server_wait_all(600)
    r = srv.ibl_server_poll(rid)
    srv.close()
    cfg = W.clap_fling_3d(nx=REQ["nx"], ny=REQ["ny"], nz=REQ["nz"], chord=REQ["chord"], Re=REQ["Re"],
                          J=REQ["J"], period=REQ["period"], faces="periodic")
    ctx = ibl.from_workload(cfg)
    ctx.ibl_solver_blocks(r["solve_blocks"])       # the tuner's block count (it fixes the reduction order)
    ctx.ibl_step(REQ["steps"])
    for w in range(2):
        h = ctx.ibl_force_history(w, REQ["steps"])
        assert np.isclose(h[:, 0].max(), r["CL_max"][w], rtol=1e-12, atol=0)
        assert np.isclose(h[:, 1].mean(), r["CT_mean"][w], rtol=1e-10, atol=1e-14)


def test_budget_and_validation(ibl):
    srv = ibl.Server(hbm_budget_bytes=1 << 20, max_active=2, chunk_steps=10)
    with pytest.raises(ibl.IblError) as e:
        srv.ibl_server_submit(**REQ)              # larger than the whole budget
    assert e.value.status == ibl.IBL_ENOMEM
    with pytest.raises(ibl.IblError) as e:
        srv.ibl_server_submit(**dict(REQ, nz=20))  # the span does not fit
    assert e.value.status == ibl.IBL_EINVAL
    srv.close()


UNSTABLE = dict(nx=48, ny=40, nz=40, chord=6.0, Re=29.0, period=1200.0, J=0.1, precision="fp32", steps=400,
                faces=1)   # tau 0.513 with Zou-He faces: diverges within ~150 steps (the oracle too)


def test_a_diverging_run_fails_alone(ibl):
    """A request that passes the stability screen but diverges (Zou-He
    inlet/outlet at tau 0.513) is stopped at the chunk where its divergence
    shows, with IBL_EDIVERGED; the run beside it gives bitwise its result
    alone."""
    alone = ibl.Server(hbm_budget_bytes=8 << 30, max_active=2, chunk_steps=25)
    rid = alone.ibl_server_submit(**REQ)
    alone.ibl_server_wait_all(600)
    ra = alone.ibl_server_poll(rid)
    alone.close()
    mix = ibl.Server(hbm_budget_bytes=8 << 30, max_active=2, chunk_steps=25)
    bad = mix.ibl_server_submit(**UNSTABLE)
    rid = mix.ibl_server_submit(**REQ)
    mix.ibl_server_wait_all(600)
    rb, rm = mix.ibl_server_poll(bad), mix.ibl_server_poll(rid)
    stats = mix.ibl_server_stats()
    mix.close()
    assert rb["done"] and rb["status"] == ibl.IBL_EDIVERGED and rb["steps_done"] < UNSTABLE["steps"]
    assert rm["status"] == ibl.IBL_OK and _keys(rm) == _keys(ra)
    assert stats["hbm_in_use"] == 0 and stats["finished"] == 2


def test_unstable_requests_are_refused_at_submission(ibl):
    srv = ibl.Server(hbm_budget_bytes=8 << 30, max_active=2, chunk_steps=25)
    for bad in (dict(REQ, Re=2000.0),                  # tau = 0.5013
                dict(REQ, J=5.0),                      # free stream 5 U_tip = 0.21 lattice units
                dict(REQ, period=240.0, Re=40.0)):     # U_tip 0.105 with U_tip / nu = 6.7
        with pytest.raises(ibl.IblError) as e:
            srv.ibl_server_submit(**bad)
        assert e.value.status == ibl.IBL_EUNSTABLE
    ok = srv.ibl_server_submit(**dict(REQ, period=240.0, Re=20.0))   # U_tip 0.105, U_tip / nu = 3.3
    srv.ibl_server_cancel(ok)
    srv.close()


def test_cancel_queued_and_running(ibl):
    srv = ibl.Server(hbm_budget_bytes=8 << 30, max_active=1, chunk_steps=10)
    running = srv.ibl_server_submit(**dict(REQ, steps=20000))
    queued = srv.ibl_server_submit(**REQ)
    t0 = time.time()
    while srv.ibl_server_poll(running)["steps_done"] == 0 and time.time() - t0 < 60:
        time.sleep(0.01)
    srv.ibl_server_cancel(queued)
    srv.ibl_server_cancel(running)
    srv.ibl_server_wait_all(600)
    rr, rq = srv.ibl_server_poll(running), srv.ibl_server_poll(queued)
    stats = srv.ibl_server_stats()
    srv.close()
    assert rr["status"] == ibl.IBL_ECANCELED and 0 < rr["steps_done"] < 20000
    assert rq["status"] == ibl.IBL_ECANCELED and rq["steps_done"] == 0 and rq["start_s"] == 0.0
    assert stats["hbm_in_use"] == 0 and stats["active"] == 0 and stats["finished"] == 2


def _sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_tuning_is_per_request_and_cached_per_shape(ibl):
    """The solve block count follows from the marker count (one block per 64
    markers, 4 .. half the SMs); the overlap mode and collide shape come from
    the first run's timed tuning chunk and are reused by a later run of the
    same shape, which then gives bitwise the same result."""
    srv = ibl.Server(hbm_budget_bytes=8 << 30, max_active=2, chunk_steps=30)
    ra_id = srv.ibl_server_submit(**REQ)
    srv.ibl_server_wait_all(600)
    rb_id = srv.ibl_server_submit(**REQ)
    srv.ibl_server_wait_all(600)
    ra, rb = srv.ibl_server_poll(ra_id), srv.ibl_server_poll(rb_id)
    load = srv.ibl_server_load()
    srv.close()
    _, ds = W.elliptic_planform_markers(REQ["chord"], 5 * REQ["chord"], 1.0)
    want = min(max(4, _sms() // 2), max(4, -(-2 * len(ds) // 64)))
    for r in (ra, rb):
        assert r["status"] == ibl.IBL_OK and r["tuned"] and r["solve_blocks"] == want
    assert (ra["overlap"], ra["collide_shape"], ra["collide_pairs"]) == \
        (rb["overlap"], rb["collide_shape"], rb["collide_pairs"])
    assert ra["overlap"] in (0, 1) and ra["collide_shape"] in [(64, 2), (128, 1), (64, 4)]
    assert _keys(ra) == _keys(rb)
    assert 0 < load["busy_s"] <= load["wall_s"]
    assert load["enqueue_s"] + load["build_s"] + load["retire_s"] <= load["busy_s"] * 1.01 + 1e-3
    print(f"tuned: {want} solve blocks, overlap {ra['overlap']}, collide {ra['collide_shape']}; load {load}")


def test_untuned_server_keeps_library_defaults(ibl):
    srv = ibl.Server(hbm_budget_bytes=8 << 30, max_active=2, chunk_steps=30, tune=0)
    rid = srv.ibl_server_submit(**REQ)
    srv.ibl_server_wait_all(600)
    r = srv.ibl_server_poll(rid)
    srv.close()
    assert r["status"] == ibl.IBL_OK and not r["tuned"] and r["solve_blocks"] == 0 and r["overlap"] == -1
    cfg = W.clap_fling_3d(nx=REQ["nx"], ny=REQ["ny"], nz=REQ["nz"], chord=REQ["chord"], Re=REQ["Re"],
                          J=REQ["J"], period=REQ["period"], faces="periodic")
    ctx = ibl.from_workload(cfg)
    ctx.ibl_step(REQ["steps"])
    h = ctx.ibl_force_history(0, REQ["steps"])
    assert h[:, 0].max() == r["CL_max"][0]


def test_many_concurrent_runs_pass_the_mass_check(ibl):
    """Twelve runs at once, past the FP64 mass check at step 500: each
    context's fills and copies are ordered on its own stream, so the mass
    reference taken at initialisation is never overwritten by a late fill
    while the GPU is loaded with the other runs' kernels."""
    srv = ibl.Server(hbm_budget_bytes=40 << 30, max_active=12, chunk_steps=50)
    ids = []
    for k in range(12):
        prec = ("fp32", "fp16dev", "bf16dev")[k % 3]
        ids.append(srv.ibl_server_submit(nx=64 + 8 * (k % 4), ny=48, nz=48, chord=6.0, Re=20.0 + k, period=600.0,
                                         J=1e-2, precision=prec, steps=520))
    srv.ibl_server_wait_all(900)
    res = [srv.ibl_server_poll(i) for i in ids]
    srv.close()
    assert [ibl.STATUS_NAMES[r["status"]] for r in res] == ["IBL_OK"] * 12
    assert all(r["steps_done"] == 520 for r in res)
