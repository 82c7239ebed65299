"""Host-only checks of the C ABI: the library loads, exports every declared
symbol, and its FP64 planning (geometry, order, waves, pupils) matches the
oracle bit for bit.  No GPU and no compute call is needed."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import fpm_oracle as orc

fpm = pytest.importorskip("paper_2203_02507_b300._fpm")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "fpm.h")).read()
    declared = set(re.findall(r"FPM_API\s+(?:int|const char \*)\s*(fpm_\w+)\s*\(", hdr))
    assert declared, "no declarations found"
    assert declared == set(fpm.EXPORTED)
    import ctypes
    lib = ctypes.CDLL(fpm.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name


def _oracle_geometry(w, defocus):
    o = w.optics
    return orc.geometry(w.sensor, w.sensor, w.tile, w.overlap, w.tiles, w.tiles, w.upsample, o.wavelength_um,
                        o.na, o.pixel_um, synth.led_grid(o.led_side, o.led_pitch_um), o.led_height_um, defocus)


@pytest.mark.parametrize("name", ["tile64_plain", "fov2048_m256", "batch_m128", "batch_m192"])
def test_geometry_and_order_match_oracle_exactly(name):
    w = synth.WORKLOADS[name]
    dz = synth.tile_defocus(w.n_tiles, *w.defocus_um, w.seed_offset)
    p = fpm.plan_for(w, defocus_um=dz, iters=1)
    s = p.schedule()
    g = _oracle_geometry(w, dz)
    assert np.array_equal(s["origins"], g.origins)
    assert np.array_equal(s["shifts"], g.shifts)
    assert np.array_equal(s["order"], g.order)
    assert p.info["support_px"] == int(g.support.sum())
    for t in (0, w.n_tiles - 1):
        np.testing.assert_allclose(p.initial_pupil(t), g.pupils[t], rtol=0, atol=2e-7)
        assert np.array_equal(p.initial_pupil(t) != 0, g.support)


@pytest.mark.parametrize("name,iters,tiles", [("tile64_plain", 10, [0]), ("fov2048_m256", 2, [0, 27, 63]),
                                              ("batch_m128", 3, [0, 9]), ("batch_m192", 2, [5])])
def test_waves_match_oracle_exactly(name, iters, tiles):
    w = synth.WORKLOADS[name]
    dz = synth.tile_defocus(w.n_tiles, *w.defocus_um, w.seed_offset)
    p = fpm.plan_for(w, defocus_um=dz, iters=iters)
    s = p.schedule()
    g = _oracle_geometry(w, dz)
    seq = orc.sequence(g.order, iters)
    for t in tiles:
        ref = orc.waves(g.n, g.support, g.shifts[t], seq)
        assert np.array_equal(s["waves"][t], ref), f"tile {t}"


def test_wave_prefix_property():
    """The schedule of k loops is the first k*L entries of the schedule of more loops."""
    w = synth.WORKLOADS["fov2048_m256"]
    a = fpm.plan_for(w, iters=3).schedule()["waves"]
    b = fpm.plan_for(w, iters=1).schedule()["waves"]
    assert np.array_equal(a[:, :b.shape[1]], b)


def _desc(**kw):
    base = dict(sensor=256, tile=64, overlap=0, tiles=1, upsample=4, wavelength_um=0.532, na=0.1,
                pixel_um=1.625, led_xy_um=synth.led_grid(5, 4000.0), led_height_um=90000.0, iters=1)
    base.update(kw)
    return base


@pytest.mark.parametrize("bad", [dict(tile=100), dict(upsample=1), dict(overlap=64), dict(tiles=5),
                                 dict(na=0.0), dict(na=1.5), dict(iters=0), dict(led_height_um=-1.0),
                                 dict(upsample=2, led_xy_um=synth.led_grid(15, 4000.0) * 3)])
def test_invalid_descriptions_are_rejected(bad):
    with pytest.raises(fpm.FpmError) as e:
        fpm.Plan(**_desc(**bad))
    assert e.value.code == fpm.EINVAL
    assert str(e.value)


def test_device_calls_before_load_fail_cleanly():
    p = fpm.Plan(**_desc())
    with pytest.raises(fpm.FpmError) as e:
        p.reconstruct(1)
    assert e.value.code == fpm.ESTATE
    with pytest.raises(fpm.FpmError):
        p.spectrum(0)
    p.close()


def test_sequential_flag_gives_one_update_per_wave():
    w = synth.WORKLOADS["tile64_plain"]
    p = fpm.plan_for(w, iters=2, sequential=True)
    s = p.schedule()
    for t in range(w.n_tiles):
        assert list(s["waves"][t]) == list(range(2 * w.n_leds))
    assert p.info["max_wave_width"] == 1 and p.info["max_waves"] == 2 * w.n_leds
    p.close()


@pytest.mark.parametrize("sel,tile,want", [
    (None, 256, (256, 4)), (None, 192, (192, 2)), (None, 128, (256, 2)), (None, 64, (128, 1)),
    ("448", 256, (448, 2)), ("448x2", 256, (448, 2)), ("256x2", 256, (256, 2)), ("192x4", 256, (192, 4)),
    ("128x4", 64, (128, 4)), ("999", 256, (256, 4)),
])
def test_update_variant_selection(sel, tile, want, monkeypatch):
    """The update-kernel variant a plan starts with (before any tuning): the first
    of its tile side, or the one FPM_UPDATE_THREADS names by threads per CTA, or
    threads x CTAs per cluster; a name that matches none falls back to the first."""
    if sel is None:
        monkeypatch.delenv("FPM_UPDATE_THREADS", raising=False)
    else:
        monkeypatch.setenv("FPM_UPDATE_THREADS", sel)
    w = {64: synth.WORKLOADS["tile64_plain"], 128: synth.WORKLOADS["batch_m128"],
         192: synth.WORKLOADS["batch_m192"], 256: synth.WORKLOADS["fov2048_m256"]}[tile]
    p = fpm.plan_for(w, iters=1)
    assert (p.info["threads"], p.info["cluster"]) == want
    p.close()


def test_tune_entry_limit_matches_the_header():
    hdr = open(os.path.join(ROOT, "include", "fpm.h")).read()
    assert int(re.search(r"#define FPM_TUNE_MAX_ENTRIES (\d+)", hdr).group(1)) == fpm.TUNE_MAX_ENTRIES


@pytest.mark.parametrize("name,iters,tiles", [("tile64_plain", 2, [0]), ("fov2048_m256", 1, [0, 63]),
                                              ("batch_m128", 2, [9])])
def test_unmasked_epry_plan_covers_the_box(name, iters, tiles):
    """FPM_EPRY_UNMASKED: the update region, hence the wave footprints, is the
    whole m x m box (bit-exact against the oracle's waves with an all-true
    support); the initial pupil keeps the circular support."""
    w = synth.WORKLOADS[name].replace(epry=True)
    dz = synth.tile_defocus(w.n_tiles, *w.defocus_um, w.seed_offset)
    p = fpm.plan_for(w, defocus_um=dz, iters=iters, unmasked=True)
    m = w.tile
    assert p.info["support_px"] == m * m and p.info["support_rows"] == m
    g = _oracle_geometry(w, dz)
    s = p.schedule()
    seq = orc.sequence(g.order, iters)
    box = np.ones((m, m), bool)
    for t in tiles:
        assert np.array_equal(s["waves"][t], orc.waves(g.n, box, g.shifts[t], seq)), f"tile {t}"
        p0 = p.initial_pupil(t)
        assert np.array_equal(p0 != 0, g.support)
    masked = fpm.plan_for(w, defocus_um=dz, iters=iters)
    assert p.info["max_waves"] > masked.info["max_waves"]          # larger footprints, more waves
    p.close()
    masked.close()


@pytest.mark.parametrize("name", ["tile64_plain", "fov2048_m256", "batch_m128", "batch_m192", "fov5120_m128"])
def test_band_pruning_flag_follows_the_support(name):
    """The update runs band-pruned radix-16 passes exactly when the tile side's
    first pass is radix 16 (m = 128, 256) and the support (the oracle's pupil
    support: its rows and its columns) lies in box positions [3 m/16, 13 m/16);
    never for the unmasked update, whose support is the whole box."""
    w = synth.WORKLOADS[name]
    dz = synth.tile_defocus(w.n_tiles, *w.defocus_um, w.seed_offset)
    g = _oracle_geometry(w, dz)
    m = w.tile
    rows = np.nonzero(g.support.any(axis=1))[0]
    cols = np.nonzero(g.support.any(axis=0))[0]
    lo, hi = 3 * m // 16, 13 * m // 16 - 1
    want = m in (128, 256) and rows.min() >= lo and rows.max() <= hi and cols.min() >= lo and cols.max() <= hi
    p = fpm.plan_for(w, defocus_um=dz, iters=1)
    assert p.info["band"] == int(want)
    p.close()
    if w.epry:
        q = fpm.plan_for(w, defocus_um=dz, iters=1, unmasked=True)
        assert q.info["band"] == 0
        q.close()


def test_unmasked_flag_needs_epry():
    with pytest.raises(fpm.FpmError) as e:
        fpm.Plan(**_desc(unmasked=True))
    assert e.value.code == fpm.EINVAL


def test_static_update_wrapper_rejects_wrong_tensors_before_the_call():
    """The allocation-free update cannot see tensor sizes through the C ABI, so its
    binding refuses a wrong type, shape or device before calling the library."""
    torch = pytest.importorskip("torch")
    m, n = 64, 256
    spec = torch.zeros((n, n), dtype=torch.complex64)
    pup = torch.zeros((m, m), dtype=torch.complex64)
    img = torch.zeros((m, m), dtype=torch.float32)
    bad = [
        (pup.to(torch.float32), "pupil"),                                       # wrong dtype
        (torch.zeros((n, n // 2), dtype=torch.complex64), "spectrum"),        # not square
        (torch.zeros((m, m), dtype=torch.float64), "image"),                  # wrong dtype
        (torch.zeros((m, m), dtype=torch.uint8), "image"),
        (torch.zeros((m // 2, m // 2), dtype=torch.float32), "image"),        # not the pupil's size
        (np.zeros((m, m), np.float32), "image"),                               # not a tensor
    ]
    for arg, which in bad:
        args = {"spectrum": spec, "pupil": pup, "image": img}
        args[which] = arg
        with pytest.raises(ValueError):
            fpm.update_tile_static(args["spectrum"], args["pupil"], args["image"], (0, 0), 0.532, 0.1, 1.625, True)
    with pytest.raises(ValueError, match="CUDA"):                              # host tensors
        fpm.update_tile_static(spec, pup, img, (0, 0), 0.532, 0.1, 1.625, True)


def test_static_update_refuses_host_pointers():
    """Through the C ABI itself: host memory is not device memory of the current
    device, so the call returns FPM_EINVAL and launches nothing."""
    m, n = 64, 256
    spec = np.zeros((n, n), np.complex64)
    pup = np.zeros((m, m), np.complex64)
    img = np.zeros((m, m), np.float32)
    rc = fpm._lib.fpm_update_tile_static(spec.ctypes.data, n, pup.ctypes.data, m, img.ctypes.data, 0, 0, 0.532,
                                         0.1, 1.625, 1, None)
    assert rc == fpm.EINVAL
    assert "device memory" in fpm._lib.fpm_last_error().decode()
