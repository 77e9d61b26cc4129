"""Differentiation variant on the GPU: V_mix, dV/dq and dV/dtheta through
mixts_potential_grad against the oracle's hand-written gradient, central
differences of the GPU potential, and the autograd.Function wrapper.

Tolerances: V within 1e-11 relative; dV/dq = -F within 1e-11 of RMS(F);
dV/dtheta within 1e-9 relative (+1e-8 * max(1, |V|) absolute, the 2^-40
kcal/mol quantum of the fixed-point sums times the number of warp adds).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_11988_gb300 as P
    return P


def _mixed(seed=3):
    s = synth.water_box(8, 8.4, 8, 2, seed=seed, ion=dict(synth.systems.ION3), electron_P=16)
    s.q = s.q + np.random.default_rng(seed + 18).normal(0, 0.08, s.q.shape)
    return s


def _gtol(V):
    return 1e-8 * max(1.0, abs(V))


@pytest.mark.parametrize("ta,tb,scale", [(0, 1, 1.0), (0, 1, 1.03), (2, 0, 0.97)])
def test_potential_grad_matches_oracle(gpu, ta, tb, scale):
    s = _mixed()
    th0 = oracle.theta_of(s, ta, tb)
    th = th0 * scale
    m = gpu.MixTS(s)
    V, dq, g = m.potential_grad(ta, tb, th, grad_out=1.0)
    so = oracle.with_theta(s, ta, tb, th)
    F_or, parts = oracle.forces(so)
    assert abs(V - parts[0]) <= 1e-11 * abs(parts[0])
    dVdq = dq.cpu().numpy()
    rms = np.sqrt(np.mean(F_or ** 2))
    assert np.abs(dVdq + F_or).max() <= 1e-11 * rms
    g_or = oracle.grad_theta(so, ta, tb)
    for k in range(8):
        assert abs(g[k] - g_or[k]) <= 1e-9 * abs(g_or[k]) + _gtol(V), (gpu.THETA_NAMES[k], g[k], g_or[k])
    # the handle's own parameters are untouched by the theta evaluation
    _, V1 = m.forces()
    assert abs(V1 - oracle.forces(s)[1][0]) <= 1e-11 * abs(V1)
    m.close()


def test_potential_grad_scales_with_grad_out(gpu):
    s = _mixed(seed=5)
    th = oracle.theta_of(s, 0, 1)
    m = gpu.MixTS(s)
    V, dq, g = m.potential_grad(0, 1, th, grad_out=1.0)
    V2, dq2, g2 = m.potential_grad(0, 1, th, grad_out=-2.5)
    assert V2 == V
    assert np.array_equal(g2, -2.5 * g)
    assert np.array_equal(dq2.cpu().numpy(), -2.5 * dq.cpu().numpy())
    m.close()


def test_potential_grad_matches_gpu_central_differences(gpu):
    s = _mixed(seed=7)
    ta, tb = 0, 1
    th = oracle.theta_of(s, ta, tb)
    m = gpu.MixTS(s)
    V, _, g = m.potential_grad(ta, tb, th, want_dvdq=False)
    for k in range(8):
        h = 1e-5 * abs(th[k])
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        vp = m.potential_grad(ta, tb, tp, want_dvdq=False)[0]
        vm = m.potential_grad(ta, tb, tm, want_dvdq=False)[0]
        fd = (vp - vm) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=2e-6, abs=1e-6 * max(1.0, abs(V))), (gpu.THETA_NAMES[k], g[k], fd)
    m.close()


def test_autograd_function(gpu):
    import torch
    s = _mixed(seed=9)
    m = gpu.MixTS(s)
    th = torch.tensor(oracle.theta_of(s, 0, 1), dtype=torch.float64, requires_grad=True)
    q = m.q.clone().requires_grad_(True)
    V = gpu.mixts_potential(th, q, m, 0, 1)
    (3.0 * V).backward()
    so = oracle.with_theta(s, 0, 1, th.detach().numpy())
    F_or, parts = oracle.forces(so)
    assert abs(V.item() - parts[0]) <= 1e-11 * abs(parts[0])
    g_or = oracle.grad_theta(so, 0, 1)
    gt = th.grad.numpy()
    for k in range(8):
        assert abs(gt[k] - 3.0 * g_or[k]) <= 3e-9 * abs(g_or[k]) + 3 * _gtol(V.item())
    rms = np.sqrt(np.mean(F_or ** 2))
    assert np.abs(q.grad.cpu().numpy() + 3.0 * F_or).max() <= 3e-11 * rms
    m.close()


def test_potential_grad_rejects_bad_theta(gpu):
    s = _mixed()
    m = gpu.MixTS(s)
    th = oracle.theta_of(s, 0, 1)
    bad = th.copy()
    bad[0] = -1.0
    with pytest.raises(gpu.MixtsError):
        m.potential_grad(0, 1, bad)
    with pytest.raises(gpu.MixtsError):
        m.potential_grad(0, 0, th)
    with pytest.raises(gpu.MixtsError):
        m.potential_grad(0, 3, th)  # the electron is not a site type
    m.close()


def test_grad_full_size_ion_electron_512(gpu):
    """512 waters + ion + 1024-bead electron (H16/O2): seeded snapshots, GPU
    gradient against the oracle's."""
    base = synth.water_box(512, 24.83, 16, 2, seed=0, ion=dict(synth.systems.ION3), electron_P=1024)
    for k in range(5):
        s = base.copy()
        s.q = base.q + np.random.default_rng(300 + k).normal(0, 0.05, base.q.shape)
        m = gpu.MixTS(s)
        th = oracle.theta_of(s, 0, 1)
        V, dq, g = m.potential_grad(0, 1, th)
        F_or, parts = oracle.forces(s)
        assert abs(V - parts[0]) <= 1e-11 * abs(parts[0])
        rms = np.sqrt(np.mean(F_or ** 2))
        assert np.abs(dq.cpu().numpy() + F_or).max() <= 1e-11 * rms
        g_or = oracle.grad_theta(s, 0, 1)
        for j in range(8):
            assert abs(g[j] - g_or[j]) <= 1e-9 * abs(g_or[j]) + _gtol(V), (gpu.THETA_NAMES[j], g[j], g_or[j])
        m.close()


def test_forward_alone_skips_the_adjoint(gpu):
    """The autograd forward evaluates V only: the adjoint sums over theta run
    in backward, on the pair terms recomputed there (nothing is stored)."""
    torch = pytest.importorskip("torch")
    s = _mixed()
    m = gpu.MixTS(s)
    th = torch.tensor(oracle.theta_of(s, 0, 1), dtype=torch.float64)
    k0 = m.timing()[2]
    V = gpu.mixts_potential(th, m.q, m, 0, 1)
    k1 = m.timing()[2]
    _, _, g = m.potential_grad(0, 1, th.tolist())
    k2 = m.timing()[2]
    assert k1 - k0 < k2 - k1  # the forward launched fewer kernels than a full gradient evaluation
    assert V.item() == m.potential_grad(0, 1, th.tolist(), want_dvdq=False, want_theta=False)[0]
    thg = th.clone().requires_grad_(True)
    V2 = gpu.mixts_potential(thg, m.q, m, 0, 1)
    V2.backward()
    assert np.allclose(thg.grad.numpy(), g, rtol=1e-14, atol=0)
    m.close()
