"""Oracle pins: normal modes, the exact free-ring propagation and the RNG.

* C is orthonormal and diagonalises the ring spring energy of
  Eq. (mts-hamiltonian-b): sum_j N m/(2 beta^2 hbar^2)(q_j - q_{j+1})^2
  = sum_k m omega_k^2 q_k^2 / 2.
* One thermostat-free, force-free step equals the exact flow
  expm(dt * generator) of that quadratic Hamiltonian (scipy.linalg.expm).
* Philox4x32-10 equals triton's independent implementation run in its CPU
  interpreter; the binary32 log and sin/cos stay within a few ulp of libm;
  the Gaussians have the moments and distribution of N(0,1).
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import synth

POW2 = [1, 2, 4, 8, 16, 32, 64, 128, 1024]


@pytest.mark.parametrize("P", POW2)
def test_nm_orthonormal(orc, P):
    Cm = orc.nm_matrix(P)
    assert np.abs(Cm @ Cm.T - np.eye(P)).max() < 1e-12


def _ring_laplacian(P):
    Lm = np.zeros((P, P))
    for j in range(P):
        Lm[j, j] += 2.0
        Lm[j, (j + 1) % P] -= 1.0
        Lm[(j + 1) % P, j] -= 1.0
    if P == 1:
        Lm[:] = 0.0
    return Lm


@pytest.mark.parametrize("P", [2, 4, 8, 32, 1024])
def test_nm_diagonalises_spring_energy(orc, P):
    c = orc.constants()
    bh = c["hbar"] / (c["kB"] * 300.0)
    m = 1.008
    kappa = P * m / bh ** 2
    w = orc.nm_freqs(P, bh)
    Cm = orc.nm_matrix(P)
    rng = np.random.default_rng(P)
    q = rng.normal(0, 0.3, P)
    e_real = 0.5 * kappa * sum((q[j] - q[(j + 1) % P]) ** 2 for j in range(P))
    qk = Cm.T @ q
    e_nm = 0.5 * m * np.sum(w ** 2 * qk ** 2)
    assert e_nm == pytest.approx(e_real, rel=1e-11)
    # the whole Hessian, not only one vector
    D = Cm.T @ (kappa * _ring_laplacian(P)) @ Cm
    assert np.abs(D - np.diag(m * w ** 2)).max() < 1e-9 * kappa


@pytest.mark.parametrize("P", [1, 2, 8])
def test_free_ring_step_is_exact_flow(orc, P):
    c = orc.constants()
    T, dt, m = 300.0, 0.7, 1.008
    bh = c["hbar"] / (c["kB"] * T)
    s = synth.harmonic_tether([P], [], masses=[m], seed=P)
    rng = np.random.default_rng(1)
    s.q = s.q + rng.normal(0, 0.2, s.q.shape)
    prm = orc.make_params(T=T, dt=dt, tau=0.0, lam=0.0, seed=0)
    run = orc.Runner(s, prm)
    q0, p0 = run.q.copy(), run.p.copy()
    run.step(1)
    # exact flow of H = p^2/2m + kappa/2 q^T L q per dimension
    kappa = P * m / bh ** 2
    K = kappa * _ring_laplacian(P)
    G = np.zeros((2 * P, 2 * P))
    G[:P, P:] = np.eye(P) / m      # dq/dt = p/m
    G[P:, :P] = -K                  # dp/dt = -K q
    E = scipy.linalg.expm(dt * G)
    for d in range(3):
        z = E @ np.concatenate([q0[:, d], p0[:, d]])
        assert np.allclose(run.q[:, d], z[:P], rtol=0, atol=1e-11)
        assert np.allclose(run.p[:, d], z[P:], rtol=0, atol=1e-11)


def _free_ring_step(orc, P, dt, m, mf, vv, seed=1):
    """One force-free, thermostat-free step of a P-bead ring; returns (q0, p0, q1, p1, kappa)."""
    c = orc.constants()
    T = 300.0
    bh = c["hbar"] / (c["kB"] * T)
    s = synth.harmonic_tether([P], [], masses=[m], seed=P)
    s.bead_mass_type = np.array([mf])
    rng = np.random.default_rng(seed)
    s.q = s.q + rng.normal(0, 0.2, s.q.shape)
    s.p = rng.normal(0, np.sqrt(mf * c["kB"] * T), s.q.shape)
    run = orc.Runner(s, orc.make_params(T=T, dt=dt, tau=0.0, lam=0.0, seed=0, vv=vv))
    q0, p0 = run.q.copy(), run.p.copy()
    run.step(1)
    return q0, p0, run.q.copy(), run.p.copy(), P * m / bh ** 2


@pytest.mark.parametrize("P,mf_over_m", [(8, 1.0), (8, 0.125), (4, 3.0)])
def test_free_ring_with_bead_mass_is_exact_flow(orc, P, mf_over_m):
    """With a fictitious bead mass m_f the free ring polymer still evolves
    exactly: dq/dt = p/m_f, dp/dt = -K q with the physical-mass springs."""
    m = 1.008
    mf = m * mf_over_m
    q0, p0, q1, p1, kappa = _free_ring_step(orc, P, 0.7, m, mf, 0)
    K = kappa * _ring_laplacian(P)
    G = np.zeros((2 * P, 2 * P))
    G[:P, P:] = np.eye(P) / mf
    G[P:, :P] = -K
    E = scipy.linalg.expm(0.7 * G)
    for d in range(3):
        z = E @ np.concatenate([q0[:, d], p0[:, d]])
        assert np.allclose(q1[:, d], z[:P], rtol=0, atol=1e-11)
        assert np.allclose(p1[:, d], z[P:], rtol=0, atol=1e-10)


@pytest.mark.parametrize("P,mf_over_m", [(8, 1.0), (16, 0.0625)])
def test_velocity_verlet_free_ring_converges_to_exact(orc, P, mf_over_m):
    """Velocity Verlet on the springs (Sec. "Evaluation") is a second-order
    integrator of the same free ring: doubling its sub-steps divides the
    error against the exact evolution by ~4, and it conserves the centroid."""
    m = 1.008
    mf = m * mf_over_m
    dt = 0.25
    qe, pe = _free_ring_step(orc, P, dt, m, mf, 0)[2:4]
    errs = []
    for n in (4, 8, 16, 32):
        q0, p0, q1, p1, _ = _free_ring_step(orc, P, dt, m, mf, n)
        errs.append(np.abs(q1 - qe).max())
        # the springs exert no net force: the centroid drifts freely
        assert np.allclose(q1.mean(0), q0.mean(0) + p0.mean(0) * dt / mf, rtol=0, atol=1e-12)
        assert np.allclose(p1.mean(0), p0.mean(0), rtol=0, atol=1e-12)
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.5 < r < 4.5 for r in ratios), (errs, ratios)
    assert errs[-1] < 1e-3 * np.abs(qe - q0).max()


def test_philox_matches_triton_interpreter(orc):
    pytest.importorskip("triton")
    code = r"""
import os, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl
@triton.jit
def k(out_ptr, c0_ptr, c1_ptr, c2_ptr, c3_ptr, k_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c0_ptr + i).to(tl.uint32, bitcast=True)
    c1 = tl.load(c1_ptr + i).to(tl.uint32, bitcast=True)
    c2 = tl.load(c2_ptr + i).to(tl.uint32, bitcast=True)
    c3 = tl.load(c3_ptr + i).to(tl.uint32, bitcast=True)
    k0 = tl.load(k_ptr + 0 * i).to(tl.uint32, bitcast=True)
    k1 = tl.load(k_ptr + 1 + 0 * i).to(tl.uint32, bitcast=True)
    a, b, c, d = tl.philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(out_ptr + 4 * i, a.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * i + 1, b.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * i + 2, c.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * i + 3, d.to(tl.int32, bitcast=True))
rng = np.random.default_rng(7)
N = 64
ctr = rng.integers(0, 2**32, (4, N), dtype=np.uint64).astype(np.uint32)
ctr[:, 0] = [0, 0, 0, 0]
ctr[:, 1] = [0xFFFFFFFF] * 4
key = np.array([int(sys.argv[1]), int(sys.argv[2])], dtype=np.uint32)
out = torch.zeros(4 * N, dtype=torch.int32)
k[(1,)](out, *[torch.from_numpy(c.view(np.int32).copy()) for c in ctr],
        torch.from_numpy(key.view(np.int32).copy()), N=N)
np.save(sys.argv[3], np.stack([ctr.T, out.numpy().view(np.uint32).reshape(N, 4)]))
"""
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        f = os.path.join(td, "p.npy")
        for key in [(0, 0), (123456789, 987654321), (0xFFFFFFFF, 1)]:
            env = dict(os.environ, TRITON_INTERPRET="1")
            subprocess.check_call([sys.executable, "-c", code, str(key[0]), str(key[1]), f], env=env)
            ctr, ref = np.load(f)
            for i in range(ctr.shape[0]):
                assert np.array_equal(orc.philox(ctr[i], key), ref[i])


def test_log_and_sincos_against_libm(orc):
    rng = np.random.default_rng(3)
    rs = np.concatenate([rng.integers(0, 2**32, 20000, dtype=np.uint64),
                         [0, 1, 511, 512, 2**31, 2**32 - 1]]).astype(np.uint64)
    for r in rs:
        r = int(r)
        u = ((r >> 9) * 2 + 1) * 2.0 ** -24
        lg = orc.log_u24(r)
        ref = math.log(u)
        assert abs(lg - ref) <= 4 * np.spacing(np.float32(abs(ref))) + 1e-7
        quad = r >> 30
        m = (((r >> 7) & 0x7FFFFF) << 1) | 1
        ang = 2 * math.pi * (quad + m * 2.0 ** -24) / 4
        s, c = orc.sincos_2pi(r)
        assert abs(s - math.sin(ang)) < 3e-7
        assert abs(c - math.cos(ang)) < 3e-7


def test_gaussian_distribution(orc):
    z = orc.gaussians(seed=12345, step=7, stage=1, dof0=0, n=400000).astype(np.float64)
    n = len(z)
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(scipy.stats.kurtosis(z, fisher=False) - 3.0) < 0.05
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-4
    # paired lanes are uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 5 / math.sqrt(n / 2)


def test_stream_addressing(orc):
    a = orc.gaussians(1, 5, 0, 1000, 64)
    assert np.array_equal(a, orc.gaussians(1, 5, 0, 1000, 64))
    assert np.array_equal(a[10:20], orc.gaussians(1, 5, 0, 1010, 10))
    for other in [(2, 5, 0), (1, 6, 0), (1, 5, 1)]:
        assert not np.array_equal(a, orc.gaussians(*other, 1000, 64))
