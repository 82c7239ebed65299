"""Online ingestion (Sec. 3.4, Fig. 7(a)): images pushed one at a time give exactly
the state of loading the whole stack and reconstructing wave by wave, whatever
the push order, and the first loop's work starts before the last image."""
import numpy as np
import pytest

import synth
from tests._jobs import Job

pytestmark = pytest.mark.gpu

O9 = synth.Optics(led_side=9)
JOBS = [
    synth.Workload("on64", sensor=160, tile=64, tiles=2, overlap=16, iters=2, epry=True, optics=O9,
                   defocus_um=(-20.0, 20.0), seed_offset=9300),
    synth.Workload("on128", sensor=256, tile=128, tiles=2, overlap=16, iters=2, epry=True, optics=O9,
                   defocus_um=(-20.0, 20.0), seed_offset=9400),
]
_CACHE = {}


def job(w):
    if w.name not in _CACHE:
        _CACHE[w.name] = Job(w)
    return _CACHE[w.name]


def state(p, w):
    return [p.spectrum(t) for t in range(w.n_tiles)] + [p.pupil(t) for t in range(w.n_tiles)]


def offline(j, w):
    p = j.plan()
    p.load_tiles(j.stack, j.counts_per_unit)
    p.reconstruct(w.iters, mode="waves")
    out = state(p, w)
    p.close()
    return out


@pytest.mark.parametrize("w", JOBS, ids=[w.name for w in JOBS])
@pytest.mark.parametrize("how", ["in_order", "shuffled", "device", "branches"])
def test_online_equals_offline(w, how, monkeypatch):
    import torch
    j = job(w)
    ref = offline(j, w)
    if how == "branches":                      # ready steps launched as two tile branches
        monkeypatch.setenv("FPM_WAVE_BRANCHES", "2")
    p = j.plan()
    order = p.schedule()["order"]
    seq = list(order)
    if how == "shuffled":
        seq = list(np.random.default_rng(5).permutation(w.n_leds))
    p.online_begin(w.iters, dtype="u16", counts_per_unit=j.counts_per_unit)
    for led in seq:
        img = j.stack[led]
        if how == "device":
            img = torch.from_numpy(img.view(np.int16)).cuda()
        p.online_push(int(led), img)
    p.online_finish()
    for a, b in zip(state(p, w), ref):
        assert np.array_equal(a, b)
    p.close()


def test_first_loop_runs_while_images_arrive():
    w = JOBS[0]
    j = job(w)
    p = j.plan()
    order = p.schedule()["order"]
    p.online_begin(w.iters, dtype="u16", counts_per_unit=j.counts_per_unit)
    for led in order[:-1]:
        p.online_push(int(led), j.stack[led])
    st = p.stats()
    assert 0 < st["online_launched"] < st["online_steps"]     # started before the last image
    p.online_push(int(order[-1]), j.stack[order[-1]])
    p.online_finish()
    st = p.stats()
    assert st["online_launched"] == st["online_steps"]
    p.close()


def test_online_misuse_is_refused():
    from paper_2203_02507_b300 import FpmError
    from paper_2203_02507_b300._fpm import EINVAL, ESTATE
    w = JOBS[0]
    j = job(w)
    p = j.plan()
    with pytest.raises(FpmError) as e:
        p.online_push(0, j.stack[0])                           # before online_begin
    assert e.value.code == ESTATE
    p.online_begin(w.iters, dtype="u16", counts_per_unit=j.counts_per_unit)
    p.online_push(0, j.stack[0])
    with pytest.raises(FpmError) as e:
        p.online_push(0, j.stack[0])                           # twice
    assert e.value.code == EINVAL
    with pytest.raises(FpmError) as e:
        p.online_push(w.n_leds, j.stack[0])                    # out of range
    assert e.value.code == EINVAL
    with pytest.raises(FpmError) as e:
        p.online_finish()                                      # images missing
    assert e.value.code == ESTATE
    with pytest.raises(FpmError) as e:
        p.spectrum(0)                                          # state not readable mid-ingestion
    assert e.value.code == ESTATE
    p.close()


def test_strided_device_pushes_equal_offline():
    """Device images whose rows are an odd number of pixels apart are gathered
    pixel by pixel; the offline load of the same images moves 16-byte words.
    Both give the same state bit for bit."""
    import torch
    w = JOBS[1]
    j = job(w)
    ref = offline(j, w)
    p = j.plan()
    p.online_begin(w.iters, dtype="u16", counts_per_unit=j.counts_per_unit)
    h, wd = j.stack.shape[1:]
    for led in p.schedule()["order"]:
        big = torch.zeros((h, wd + 3), dtype=torch.int16, device="cuda")
        big[:, :wd] = torch.from_numpy(j.stack[led].view(np.int16)).cuda()
        p.online_push(int(led), big[:, :wd])
    p.online_finish()
    for a, b in zip(state(p, w), ref):
        assert np.array_equal(a, b)
    p.close()


@pytest.mark.parametrize("w", JOBS, ids=[w.name for w in JOBS])
@pytest.mark.parametrize("how", ["in_order", "shuffled"])
def test_online_matches_oracle(w, how):
    """Online ingestion against the FP64 oracle itself (not only against the
    library's offline path): every tile's spectrum and pupil after the job's loops,
    images pushed in LED order or shuffled, within the parity bounds of the
    offline tests (spectrum max(1e-5, 4 x float32 floor), pupil max(1e-4, 4 x
    floor))."""
    from oracle import fpm_oracle as orc
    from tests import _fp32
    from tests._jobs import rel_l2
    j = job(w)
    p = j.plan()
    seq = list(p.schedule()["order"])
    if how == "shuffled":
        seq = list(np.random.default_rng(11).permutation(w.n_leds))
    p.online_begin(w.iters, dtype="u16", counts_per_unit=j.counts_per_unit)
    for led in seq:
        p.online_push(int(led), j.stack[led])
    p.online_finish()
    bad = []
    for t in range(w.n_tiles):
        imgs = j.tile_images(t)
        spec, pup = orc.reconstruct_tile(imgs, j.g.shifts[t], j.g.order, j.g.support, j.g.pupils[t], j.g.n,
                                         w.iters, True)
        fs, fp = _fp32.floor(imgs, j.g.shifts[t], j.g.order, j.g.support, j.g.pupils[t], j.g.n, w.iters, True,
                             spec, pup)
        es, ep = rel_l2(p.spectrum(t), spec), rel_l2(p.pupil(t), pup)
        if es >= max(1e-5, 4.0 * fs) or ep >= max(1e-4, 4.0 * fp):
            bad.append((t, es, fs, ep, fp))
    p.close()
    assert not bad, bad
