"""Host checks of bench.py's roofline arithmetic: the support pixel counts agree
with the library's plan and with the closed-form disc counts, and the per-update
FLOP and byte figures the bench divides by are the ones its docstrings state."""
import os
import re

import pytest

import synth

bench = pytest.importorskip("bench")
fpm = pytest.importorskip("paper_2203_02507_b300._fpm")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("name,a", [("tile64_plain", 1201), ("batch_m128", 4809), ("batch_m192", 10797),
                                    ("fov2048_m256", 19213)])
def test_support_pixels_agree_with_the_plan(name, a):
    w = synth.WORKLOADS[name]
    assert bench.support_px(w) == a
    p = fpm.plan_for(w, iters=1)
    assert p.info["support_px"] == a
    p.close()


def test_headline_flops_and_bytes_per_update():
    w = synth.WORKLOADS["fov2048_m256"]
    m, a = 256, 19213
    assert bench.flops_per_update(w) == 2 * 5 * m * m * 16 + 10 * m * m + 36 * a == 11832788
    assert bench.bytes_per_update(w) == 2 * m * m + 16 * a + 16 * a == 745888


def test_traffic_figures_cite_committed_profiles():
    src = open(os.path.join(ROOT, "bench.py")).read()
    block = src[src.index("TRAFFIC_PER_UPDATE = {"):src.index("EXTRA = {")]
    for f in re.findall(r"profiles/([\w.]+\.md)", block):
        assert os.path.exists(os.path.join(ROOT, "profiles", f)), f
    for key in bench.TRAFFIC_PER_UPDATE:
        assert len(key) == 4 and key[0] in ("waves", "persistent")
