"""Host checks of the seeded workloads: every circle is exactly representable (centre and radius
multiples of 1/2, as the geometry requires), every initial drop lies inside its domain and
meets the wall the way its generator states, and the derived quantities (drop placement for a
target angle, tilted gravity) follow their definitions."""
import math

import pytest

from helpers import cap_angle_on_circle
from paper_2202_06516_gb300 import workloads as W


def _half(v):
    return abs(2.0 * v - round(2.0 * v)) < 1e-12


def _check_common(w):
    assert w.nx >= 8 and w.ny >= 8
    if w.circle is not None:
        cx, cy, R = w.circle
        assert _half(cx) and _half(cy) and _half(R) and R > 0
    x, y, r, Wd = w.drop
    assert 0 <= x < w.nx and r > 0 and Wd > 0
    assert y + r < w.ny - 2, w.name          # the drop stays below the top wall


@pytest.mark.parametrize("het", [True, False])
def test_hysteresis_workload(het):
    w = W.hysteresis(het)
    _check_common(w)
    assert (w.nx, w.ny) == (4096, 1024) and w.circle[2] == 800 and w.drop[2] == 120
    assert w.buoyant and w.measure_every == 100 and w.steps == 200000
    # gravity tilted by the 20-degree slope angle, tangential component 5e-7 at the top
    gx, gy = w.g
    assert math.degrees(math.atan2(gx, -gy)) == pytest.approx(20.0)
    assert gx == pytest.approx(5e-7)
    assert (w.stripes is not None) == het
    if het:
        assert w.stripes[0] == 40.0 and w.stripes[1] == W.HYST_MU_REL_60


def test_curvature_sweep_places_drops_at_the_target_angle():
    ws = W.curvature_sweep()
    assert len(ws) == 110
    for w in ws:
        _check_common(w)
        cx, cy, R = w.circle
        x, y, r, _ = w.drop
        assert r <= 0.5 * R
        target = float(w.name.rsplit("theta", 1)[1])
        D = math.hypot(x - cx, y - cy)
        assert cap_angle_on_circle(R + 0.5, r, D, concave=w.concave) == pytest.approx(target)
        if w.concave:
            assert y < cy                   # at the bottom of the cavity
            assert cy - R > 0               # the cavity's lowest wall point is inside the domain


def test_gravity_sweep():
    sw = W.gravity_sweep()
    assert len(sw["instances"]) == 18
    assert sw["g"]["sessile"][1] < 0 < sw["g"]["pendent"][1] and sw["g"]["none"] == (0.0, 0.0)
    for w in sw["instances"]:
        _check_common(w)


def test_batched_instances_fit():
    for w in W.batched(256, seed=0):
        _check_common(w)
        cx, cy, R = w.circle
        assert 2 * R + 16 <= w.nx and R + 2 * w.drop[2] + 8 <= w.ny
