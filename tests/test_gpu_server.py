"""Serving through the C ABI: continuous batching of jobs with different tile
sizes, admission by device-memory budget, and results that are the same alone
and in a mix."""
import time

import numpy as np
import pytest

import synth
from tests._jobs import Job, rel_l2

pytestmark = pytest.mark.gpu

O9 = synth.Optics(led_side=9)
MIX = [
    synth.Workload("s64", sensor=256, tile=64, tiles=4, overlap=16, iters=2, epry=True, optics=O9,
                   defocus_um=(-20.0, 20.0), seed_offset=5000),
    synth.Workload("s128", sensor=384, tile=128, tiles=3, overlap=16, iters=2, epry=True, optics=O9,
                   defocus_um=(-20.0, 20.0), seed_offset=6000),
    synth.Workload("s192", sensor=384, tile=192, tiles=2, overlap=16, iters=2, epry=True, optics=O9,
                   defocus_um=(-20.0, 20.0), seed_offset=7000),
    synth.Workload("s256", sensor=512, tile=256, tiles=2, overlap=16, iters=2, epry=True, optics=O9,
                   defocus_um=(-20.0, 20.0), seed_offset=8000),
]
_JOBS = {}


def job(w):
    if w.name not in _JOBS:
        _JOBS[w.name] = Job(w)
    return _JOBS[w.name]


def wait_done(server, ids, timeout=120.0):
    t0 = time.time()
    states = {}
    while time.time() - t0 < timeout:
        states = {i: server.poll(i) for i in ids}
        if all(s[0] in ("done", "failed") for s in states.values()):
            return states
        time.sleep(0.005)
    raise TimeoutError(states)


def results(plan, w):
    return [plan.spectrum(t) for t in range(w.n_tiles)], [plan.pupil(t) for t in range(w.n_tiles)]


def test_results_are_the_same_alone_and_in_the_mix():
    from paper_2203_02507_b300 import Server
    alone = {}
    for w in MIX:
        j = job(w)
        srv = Server(8 << 30)
        p = j.plan()
        jid = srv.submit(p, w.iters, stack=j.stack, counts_per_unit=j.counts_per_unit)
        st = wait_done(srv, [jid])
        assert st[jid][0] == "done"
        alone[w.name] = results(p, w)
        srv.close()
        p.close()
    # all four together, the last two arriving while the first two run
    srv = Server(8 << 30)
    plans, ids = [], []
    for k, w in enumerate(MIX):
        j = job(w)
        p = j.plan()
        plans.append(p)
        ids.append(srv.submit(p, w.iters, stack=j.stack, counts_per_unit=j.counts_per_unit))
        if k == 1:
            time.sleep(0.02)
    st = wait_done(srv, ids)
    for w, p, jid in zip(MIX, plans, ids):
        assert st[jid][0] == "done"
        spec, pup = results(p, w)
        for a, b in zip(spec + pup, alone[w.name][0] + alone[w.name][1]):
            assert rel_l2(a, b) <= 1e-5
            assert np.array_equal(a, b)           # the per-tile work is deterministic
        p.close()
    srv.close()
    # and what fpm_reconstruct computes for the same job
    for w in MIX:
        j = job(w)
        p = j.plan()
        p.load_tiles(j.stack, j.counts_per_unit)
        p.reconstruct(w.iters, mode="waves")
        spec, pup = results(p, w)
        for a, b in zip(spec + pup, alone[w.name][0] + alone[w.name][1]):
            assert np.array_equal(a, b)
        p.close()


def test_admission_by_budget_and_overlap():
    from paper_2203_02507_b300 import FpmError, Server
    from paper_2203_02507_b300._fpm import EBUDGET
    w_small, w_big = MIX[0], MIX[3]
    js, jb = job(w_small), job(w_big)
    pb = jb.plan()
    # state + tile images (uint16) + the host stack's device staging while it loads
    need_big = pb.info["device_bytes"] + 2 * pb.info["image_elems"] + jb.stack.nbytes
    # a budget that holds the big job but not two of them
    srv = Server(int(need_big * 1.5))
    pb2 = jb.plan()
    a = srv.submit(pb, w_big.iters, stack=jb.stack, counts_per_unit=jb.counts_per_unit)
    b = srv.submit(pb2, w_big.iters, stack=jb.stack, counts_per_unit=jb.counts_per_unit)
    st = wait_done(srv, [a, b])
    (sa, wa, la), (sb, wb, lb) = st[a], st[b]
    assert sa == sb == "done"
    assert wb >= la - 0.05               # b (submitted right after a) was admitted only once a finished
    srv.close()
    # a job larger than the whole budget is refused at submission
    srv = Server(need_big // 4)
    with pytest.raises(FpmError) as e:
        srv.submit(jb.plan(), w_big.iters, stack=jb.stack, counts_per_unit=jb.counts_per_unit)
    assert e.value.code == EBUDGET
    srv.close()
    # with room for both, a job that arrives while another runs is admitted at once and overlaps it
    srv = Server(8 << 30)
    p1, p2 = jb.plan(iters=2), js.plan(iters=2)
    a = srv.submit(p1, 2, stack=jb.stack, counts_per_unit=jb.counts_per_unit)
    for _ in range(2000):
        if srv.poll(a)[0] == "running":
            break
        time.sleep(0.001)
    b = srv.submit(p2, 2, stack=js.stack, counts_per_unit=js.counts_per_unit)
    st = wait_done(srv, [a, b])
    assert st[a][0] == st[b][0] == "done"
    assert st[b][1] < 0.05                # admitted without waiting for the running job
    srv.close()
    for p in (pb, pb2, p1, p2):
        p.close()


@pytest.mark.parametrize("mode,graph", [("persistent", False), ("persistent", True), ("waves", False),
                                        ("waves", True)])
def test_uneven_batch_runs_as_one(mode, graph, monkeypatch):
    """Four jobs with tiles of 64, 128, 192 and 256 run together (one persistent launch, or
    every plan an independent graph branch split into 2 tile branches) end exactly as run
    one by one."""
    from paper_2203_02507_b300 import reconstruct_batch
    monkeypatch.setenv("FPM_WAVE_BRANCHES", "2")
    plans = []
    for w in MIX:
        j = job(w)
        p = j.plan()
        p.load_tiles(j.stack, j.counts_per_unit)
        plans.append(p)
    reconstruct_batch(plans, [w.iters for w in MIX], graph=graph, mode=mode)
    for w, p in zip(MIX, plans):
        assert p.stats()["device_error"] == 0
        j = job(w)
        q = j.plan()
        q.load_tiles(j.stack, j.counts_per_unit)
        q.reconstruct(w.iters, mode="waves")
        for t in range(w.n_tiles):
            assert np.array_equal(p.spectrum(t), q.spectrum(t))
            assert np.array_equal(p.pupil(t), q.pupil(t))
        q.close()
    for p in plans:
        p.close()
