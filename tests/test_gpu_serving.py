"""The continuous-batching server: a job's result does not depend on when it
arrives or who shares its batches (views are keyed by the job's own seed and
iteration; the batched launches keep jobs apart), admission waits for the HBM
budget, a job whose loss turns non-finite is quarantined while the others
finish with unchanged results, and cancelled requests (waiting or live) free
their memory without changing the others' results."""

import math

import numpy as np
import pytest
import torch

from cases import rel_l2, sphere_scene

pytestmark = pytest.mark.gpu

# (candidate freq, texture, seed, tessellation levels), reference freq, views, resolution, iterations
SPECS = [
    ((4, 64, 1, 0), 12, 2, 96, 6),
    ((6, 128, 2, 0), 16, 3, 64, 4),
    ((3, 32, 3, 1), 10, 1, 80, 5),
]
# Adam turns a 1e-6 relative change of a gradient (the order of float atomics
# differs between the single-job and the batched launches) into a change of
# the same relative size in the update; a few steps stay far below this
SERVE_TOL = 1e-5


def _requests():
    from paper_2104_03989_gb300.serving import Request
    out = []
    for rid, ((freq, tex, seed, tess), ref_freq, nv, res, iters) in enumerate(SPECS):
        out.append(Request(rid=rid, cand=sphere_scene(freq, tex, seed, tess), ref=sphere_scene(ref_freq, tex, 50 + seed),
                           n_views=nv, res=res, iterations=iters, seed=100 + rid))
    return out


@pytest.fixture(scope="module")
def alone(gpu_lib):
    from paper_2104_03989_gb300.serving import SimplificationServer
    res = {}
    for req in _requests():
        srv = SimplificationServer()
        rep = srv.run([req])
        assert rep["done"] == 1 and rep["iterations"] == req.iterations
        res[req.rid] = srv.results[req.rid]
        srv.close()
    return res


def _same(a, b):
    assert set(a) == set(b)
    for k in a:
        x, y = a[k].double().cpu().numpy(), b[k].double().cpu().numpy()
        assert np.isfinite(x).all(), k
        assert rel_l2(x, y) < SERVE_TOL, (k, rel_l2(x, y))


def test_staggered_arrivals_give_the_results_of_jobs_served_alone(alone):
    from paper_2104_03989_gb300.serving import SimplificationServer
    reqs = _requests()
    srv = SimplificationServer()
    srv.start()
    srv.submit(reqs[0])
    srv.admit()
    srv.iterate()
    srv.iterate()                       # job 0 alone: the single-job launches
    srv.submit(reqs[1])
    srv.admit()
    srv.iterate()                       # jobs 0, 1: batched launches
    srv.submit(reqs[2])
    srv.admit()
    while srv.live:
        srv.iterate()
    rep = srv.report()
    assert rep["done"] == 3 and rep["max_live"] == 3
    assert rep["p99_iteration_ms"] >= rep["p50_iteration_ms"] > 0
    for r in srv.done:
        assert r.status == "done" and r.it == r.req.iterations
        assert all(math.isfinite(x) for x in r.losses)
        _same(srv.results[r.req.rid], alone[r.req.rid])
    srv.close()


def test_admission_waits_for_the_hbm_budget(gpu_lib):
    from paper_2104_03989_gb300.serving import SimplificationServer
    reqs = _requests()
    a, b = reqs[0], reqs[0].__class__(**{**reqs[0].__dict__, "rid": 7})
    probe = SimplificationServer()
    probe.start()
    probe.submit(a)
    probe.admit()
    need = probe.ctx.bytes_in_use()
    headroom = probe._headroom(probe.live)
    probe.close()
    assert need > 0
    budget = need + need // 2 + headroom      # one job fits, two do not
    srv = SimplificationServer(hbm_budget_bytes=budget)
    peak = []
    srv.start()
    srv.submit(a)
    srv.submit(b)
    while srv.queue or srv.live:
        srv.admit()
        peak.append(srv.ctx.bytes_in_use())
        srv.iterate()
    rep = srv.report()
    assert rep["done"] == 2 and rep["max_live"] == 1 and rep["rejected"] == 0
    assert max(peak) <= budget
    first, second = sorted(srv.done, key=lambda r: r.admitted)
    assert second.admitted >= first.finished
    srv.close()

    # a request that can never fit is rejected, not left waiting
    srv = SimplificationServer(hbm_budget_bytes=need // 2)
    rep = srv.run([a])
    assert rep["rejected"] == 1 and rep["done"] == 0
    srv.close()


def test_non_finite_job_is_quarantined_and_the_others_are_unchanged(alone):
    from paper_2104_03989_gb300 import binding as B
    from paper_2104_03989_gb300.serving import SimplificationServer

    def poison(server, rec):
        if rec.req.rid == 1:
            server.ctx.params(rec.cand)["kd"].fill_(float("nan"))
            B.adms_job_invalidate(server.ctx.ctx, rec.cand)

    srv = SimplificationServer(on_admit=poison)
    rep = srv.run(_requests())
    assert rep["done"] == 2 and rep["quarantined"] == 1
    status = {r.req.rid: r for r in srv.done}
    assert status[1].status == "quarantined" and status[1].it == 1 and not math.isfinite(status[1].losses[0])
    assert status[1].status_code == B.ADMS_ERR_NONFINITE   # latched on the device
    for rid in (0, 2):
        assert status[rid].status == "done"
        _same(srv.results[rid], alone[rid])
    srv.close()


def test_cancelled_requests_free_their_memory_and_the_others_are_unchanged(alone):
    from paper_2104_03989_gb300.serving import SimplificationServer
    reqs = _requests()
    srv = SimplificationServer()
    srv.start()
    for r in reqs:
        srv.submit(r)
    srv.admit()
    assert len(srv.live) == 3
    srv.iterate()
    before = srv.ctx.bytes_in_use()
    assert srv.cancel(1)                      # a live job, between iterations
    assert srv.ctx.bytes_in_use() < before
    assert not srv.cancel(1)
    waiting = reqs[0].__class__(**{**reqs[0].__dict__, "rid": 9})
    srv.submit(waiting)
    assert srv.cancel(9)                      # a request still in the queue
    while srv.queue or srv.live:
        srv.admit()
        srv.iterate()
    rep = srv.report()
    assert rep["done"] == 2 and rep["cancelled"] == 2 and rep["quarantined"] == 0
    status = {r.req.rid: r for r in srv.done}
    assert status[1].status == "cancelled" and status[1].it == 1
    assert status[9].status == "cancelled" and status[9].it == 0
    for rid in (0, 2):
        _same(srv.results[rid], alone[rid])
    srv.close()
