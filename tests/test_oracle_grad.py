"""Oracle pin: the hand-written parameter gradient dV_mix/dtheta against
central finite differences of the oracle potential (h = 1e-5 relative)."""
import numpy as np
import pytest

import synth


def _sys():
    s = synth.water_box(8, 8.4, 8, 2, seed=3, ion=dict(synth.systems.ION3), electron_P=16)
    s.q = s.q + np.random.default_rng(21).normal(0, 0.08, s.q.shape)
    return s


@pytest.mark.parametrize("ta,tb", [(0, 1), (1, 2), (2, 0)])  # O,H; H,ion; ion,O
def test_grad_theta_matches_central_differences(orc, ta, tb):
    s = _sys()
    th = orc.theta_of(s, ta, tb)
    if th[7] == 0.0:
        # eps_aa = 0 in the system: cross terms stay fixed, V is linear in eps_aa
        th[7] = 0.05
        s = orc.with_theta(s, ta, tb, th)
    g = orc.grad_theta(s, ta, tb)
    for k in range(8):
        h = 1e-5 * abs(th[k])
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        vp = orc.forces(orc.with_theta(s, ta, tb, tp))[1][0]
        vm = orc.forces(orc.with_theta(s, ta, tb, tm))[1][0]
        fd = (vp - vm) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=2e-6, abs=1e-7 * max(1.0, abs(vp))), (orc.THETA_NAMES[k], g[k], fd)


def test_theta_roundtrip_is_identity(orc):
    s = _sys()
    th = orc.theta_of(s, 0, 1)
    s2 = orc.with_theta(s, 0, 1, th)
    assert orc.forces(s2)[1][0] == orc.forces(s)[1][0]
