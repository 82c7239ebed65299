"""The allocation-free single-LED update checked against the plan path.

fpm_update_tile_static is for callers that cannot allocate device memory: a
host whose GPU memory is owned by its own pool, a plug-in that may not
allocate after start-up, or a real-time acquisition loop that an allocation
would stall.  Its temporaries live in a fixed static device array.  It runs the
same update kernel with the same arithmetic as the plan path, so two calls in a
row must give the plan path's state bit for bit.  This file is collected last
so that, should it fail, every other test has already run.
"""
import numpy as np
import pytest

import synth
from oracle import fpm_oracle as orc

pytestmark = pytest.mark.gpu

LAM, NA, DX = 0.532, 0.1, 1.625


def _case(m, epry):
    from paper_2203_02507_b300 import Plan
    leds = np.array([[0.0, 0.0], [4000.0, 0.0]])          # neighbouring LEDs: overlapping discs
    n = 4 * m
    g = orc.geometry(m, m, m, 0, 1, 1, 4, LAM, NA, DX, leds, 90000.0, [6.0])
    obj = synth.hr_object(n, 0, seed_offset=11 * m)
    imgs = orc.forward_images(orc.fft2c(obj), g.pupils[0], g.shifts[0], m).astype(np.float32)
    imgs = np.ascontiguousarray(imgs * np.float32(1.3))   # away from the fixed point
    p = Plan(sensor=m, tile=m, overlap=0, tiles=1, upsample=4, wavelength_um=LAM, na=NA, pixel_um=DX,
             led_xy_um=leds, led_height_um=90000.0, defocus_um=[6.0], iters=1, epry=epry)
    sch = p.schedule()
    assert list(sch["waves"][0]) == [0, 1]                 # the plan runs them one after the other
    p.load_tiles(imgs, 1.0)
    spec0, pup0 = p.spectrum(0), p.pupil(0)
    p.reconstruct(1)
    ref_spec, ref_pup = p.spectrum(0), p.pupil(0)
    p.close()
    return imgs, sch, spec0, pup0, ref_spec, ref_pup


@pytest.mark.parametrize("m", [64, 128, 192, 256])
@pytest.mark.parametrize("epry", [True, False])
def test_two_static_updates_match_the_plan_path(m, epry):
    import torch
    from paper_2203_02507_b300 import update_tile_static
    assert torch.cuda.is_available()
    imgs, sch, spec0, pup0, ref_spec, ref_pup = _case(m, epry)
    spec = torch.from_numpy(spec0).cuda()
    pup = torch.from_numpy(pup0).cuda()
    dimgs = torch.from_numpy(imgs).cuda()
    for led in sch["order"]:                               # two calls in a row
        update_tile_static(spec, pup, dimgs[int(led)], sch["shifts"][0, int(led)], LAM, NA, DX, epry)
    torch.cuda.synchronize()
    assert np.array_equal(spec.cpu().numpy(), ref_spec)
    assert np.array_equal(pup.cpu().numpy(), ref_pup)
    assert not np.array_equal(spec0, ref_spec)             # the updates did change the state


def test_static_updates_allocate_no_device_memory():
    """After a first call (which looks up the static array), further calls leave the
    device's free memory unchanged: nothing is allocated, not even by the
    caching allocator, since the entry point never goes through it."""
    import torch
    from paper_2203_02507_b300 import update_tile_static
    m = 256
    imgs, sch, spec0, pup0, _, _ = _case(m, True)
    spec = torch.from_numpy(spec0).cuda()
    pup = torch.from_numpy(pup0).cuda()
    dimgs = torch.from_numpy(imgs).cuda()
    led0 = int(sch["order"][0])
    update_tile_static(spec, pup, dimgs[led0], sch["shifts"][0, led0], LAM, NA, DX, True)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(5):
        for led in sch["order"]:
            update_tile_static(spec, pup, dimgs[int(led)], sch["shifts"][0, int(led)], LAM, NA, DX, True)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    assert np.isfinite(spec.cpu().numpy()).all()


def test_sizes_beyond_the_static_limit_are_rejected():
    import torch
    from paper_2203_02507_b300 import FpmError, update_tile_static
    m = 512
    spec = torch.zeros((4 * m, 4 * m), dtype=torch.complex64, device="cuda")
    pup = torch.zeros((m, m), dtype=torch.complex64, device="cuda")
    img = torch.zeros((m, m), dtype=torch.float32, device="cuda")
    with pytest.raises(FpmError) as e:
        update_tile_static(spec, pup, img, (0, 0), LAM, NA, DX, True)
    assert "static scratch" in str(e.value)
    big = torch.zeros((9 * 256, 9 * 256), dtype=torch.complex64, device="cuda")   # N = 9 m
    with pytest.raises(FpmError):
        update_tile_static(big, pup[:256, :256].contiguous(), img[:256, :256].contiguous(), (0, 0), LAM, NA, DX,
                           True)
