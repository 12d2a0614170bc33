"""Host logic of the warm-start evaluation (CPU): the mass matching of a predicted field, the
time-to-equilibrated-angle criterion and the per-variant summary."""
import numpy as np
import pytest

from paper_2202_06516_gb300 import warmstart as WS


def test_match_mass_hits_the_target_with_one_shift():
    rng = np.random.default_rng(0)
    H = 96
    j, i = np.mgrid[0:H, 0:H]
    phi = 1.0 / (1.0 + np.exp(-(20.0 - np.hypot(i - 48, j - 40)) / 2.0))
    phi = np.clip(phi + rng.normal(0, 0.02, phi.shape), 0, 1)
    mask = j > 6
    rho_g, rho_l = 0.0556, 8.08
    for shift in (-0.3, -0.01, 0.0, 0.05, 0.4):
        target = (rho_g + np.clip(phi + shift, 0, 1) * (rho_l - rho_g))[mask].sum()
        out = WS.match_mass(phi, mask, target, rho_g, rho_l)
        got = (rho_g + out * (rho_l - rho_g))[mask].sum()
        assert got == pytest.approx(target, rel=1e-12)
        # one constant shift, then the clip: nodes strictly inside (0, 1) moved by the same amount
        inner = (out > 0) & (out < 1) & mask
        d = out[inner] - phi[inner]
        assert np.ptp(d) < 1e-12
        assert d.mean() == pytest.approx(shift, abs=1e-9)


def test_reach_index_is_the_first_check_after_which_all_stay_inside():
    final = np.array([90.0, 91.0])
    h = np.array([[80, 80], [89.7, 90.9], [91, 91], [90.2, 91.4], [90.1, 90.8], [90.0, 91.0]])
    # check 2 leaves the window (91 vs 90 by 1.0), so the answer is check 3
    assert WS.reach_index(h, final) == 3
    assert WS.time_to_angle(h, final, 250) == 1000
    h2 = h.copy()
    h2[-1, 1] = np.nan  # a side without contact at the end: never settled
    assert WS.reach_index(h2, final) is None


def _row(cls, plain, cold, warm, gap=0.1):
    return {"class": cls, "plain": plain, "cold": cold, "warm": warm, "plain_identical": True,
            "warm_final_gap": gap, "warm_self": 1000, "cold_self": 2000, "theta_f": [90, 90]}


def test_summary_counts_classes_and_times():
    rows = [_row("ok", (2000, 0.2), (2000, 5.0), (500, 2.0)),
            _row("ok", (4000, 0.4), (4000, 9.0), None, gap=0.9),
            _row("ok", (1000, 0.1), (1000, 3.0), (1500, 4.0)),
            _row("unsettled", None, None, None), _row("no_contact", None, None, None, gap=None)]
    out = WS.summarise(rows, {"prediction_seconds": 1.0})
    assert out["classes"] == {"ok": 3, "unsettled": 1, "no_contact": 1}
    assert out["judged"] == 3
    assert out["plain"]["reached"] == 3 and out["plain"]["all_reached_seconds"] == pytest.approx(0.7)
    assert out["cold"]["all_reached_seconds"] == 9.0  # a batch: the last case to reach
    assert out["warm"]["reached"] == 2 and out["warm"]["reached_fraction"] == pytest.approx(2 / 3)
    assert out["warm"]["median_steps"] == 1000.0
    assert out["warm_faster_fraction"] == 0.5
    assert out["warm_settles_elsewhere"] == 1
    assert out["plain_equals_batched_cold"] is True
    assert out["prediction_seconds"] == 1.0


def test_merge_extra_takes_the_slowest_rank_and_sums_plain():
    parts = [{"prediction_seconds": 1.0, "cold_batch_seconds": 5.0, "warm_batch_seconds": 6.0,
              "plain_seconds": 10.0},
             {"prediction_seconds": 2.0, "cold_batch_seconds": 4.0, "warm_batch_seconds": 7.0,
              "plain_seconds": 11.0}, {}]
    out = WS.merge_extra(parts)
    assert out == {"prediction_seconds": 2.0, "cold_batch_seconds": 5.0,
                   "warm_batch_seconds": 7.0, "plain_seconds": 21.0}
