"""Oracle pins on sampled dynamics (statistical, seeded).

* P-bead harmonic oscillator: <x^2>_P = (1/(beta m)) sum_k [w^2 + 4P^2 sin^2(pi k/P)/(beta hbar)^2]^-1,
  exact at finite P for the ring-polymer Hamiltonian Eq. (rpham); the
  primitive and centroid-virial kinetic estimators average to (3/2) m w^2 <x^2>_P,
  whatever the fictitious bead mass and with the velocity-Verlet free ring.
* Two harmonic particles with 8 and 2 beads coupled through the mixTS pair
  map: sampled bead covariance equals (beta K)^-1, K the Hessian of
  H0 + V_mix of Eq. (mts-hamiltonian).
* Free ring polymer: <R_g^2> = (P^2 - 1) beta hbar^2 / (4 P^2 m).
* Thermostat: bead kinetic temperature equals T.
* NVE (thermostat off): H_mix is conserved with fluctuations scaling as dt^2.
* Thermostat bookkeeping: with PILE on, H_mix + heat is conserved to the NVE
  level while H_mix itself swings by the exchanged heat.
"""
import math

import numpy as np
import pytest

import synth
from stats_util import block_mean

T = 300.0


def _consts(orc):
    c = orc.constants()
    kT = c["kB"] * T
    return c, kT, c["hbar"] / kT


def _ho_exact_x2(P, m, w, beta, bh):
    k = np.arange(P)
    return (1.0 / (beta * m)) * np.sum(1.0 / (w ** 2 + 4 * P ** 2 * np.sin(np.pi * k / P) ** 2 / bh ** 2))


@pytest.mark.parametrize("P,mf_over_m,vv", [(1, 1.0, 0), (4, 1.0, 0), (32, 1.0, 0), (8, 0.125, 0), (8, 4.0, 0),
                                         (8, 1.0, 6)])
def test_harmonic_oscillator_closed_form(orc, P, mf_over_m, vv):
    """The closed form holds for any fictitious bead mass m_f (statics do not
    depend on it, Sec. "Theory" after Eq. rpham) and with the velocity-Verlet
    free ring (sampling error of its O(dt^2) shadow Hamiltonian far below the
    statistical error at dt = 1 fs, 6 sub-steps)."""
    c, kT, bh = _consts(orc)
    m = 1.0
    w = 4.0 / bh                      # beta hbar omega = 4
    k_md = m * w ** 2
    k_kcal = k_md / c["kcal"]
    s = synth.harmonic_tether([P, 1], [(0, 1, k_kcal)], masses=[m, 1.0], seed=P)
    s.bead_mass_type = np.array([m * mf_over_m, 1.0])
    prm = orc.make_params(T=T, dt=1.0, tau=20.0, lam=1.0, seed=100 + P, vv=vv)
    run = orc.Runner(s, prm)
    run.step(2000)
    x2, kp, kc, tb = [], [], [], []
    rows_a = s.bead_rows(0)
    row_c = s.bead_rows(1)[0]
    for _ in range(12000):
        run.step(4)
        y = run.q[rows_a] - run.q[row_c]
        x2.append(np.mean(np.sum(y * y, axis=1)) / 3.0)
        e = run.estimators()
        kp.append(e["KE_prim"][0])
        kc.append(e["KE_cv"][0])
        tb.append(e["T_beads"])
    beta = 1.0 / kT
    ex = _ho_exact_x2(P, m, w, beta, bh)
    mean, err = block_mean(x2)
    assert abs(mean - ex) < 4 * err + 1e-3 * ex, (mean, err, ex)
    kin = 1.5 * m * w ** 2 * ex / c["kcal"]   # kcal/mol
    for est in (kp, kc):
        mu, er = block_mean(est)
        assert abs(mu - kin) < 4 * er + 2e-3 * kin, (mu, er, kin)
    mu, er = block_mean(tb)
    assert abs(mu - T) < 4 * er + 0.5


def test_mixts_pair_covariance(orc):
    c, kT, bh = _consts(orc)
    w = 4.0 / bh
    k = 1.0 * w ** 2 / c["kcal"]
    PA, PB = 8, 2
    mA, mB = 1.0, 2.0
    s = synth.harmonic_tether([PA, PB, 1], [(0, 2, k), (1, 2, k), (0, 1, k)],
                              masses=[mA, mB, 1.0], seed=5)
    prm = orc.make_params(T=T, dt=1.0, tau=20.0, lam=1.0, seed=77)
    run = orc.Runner(s, prm)
    run.step(2000)
    ra, rb, rc = s.bead_rows(0), s.bead_rows(1), s.bead_rows(2)[0]
    acc = np.zeros((PA + PB, PA + PB))
    n = 0
    for _ in range(15000):
        run.step(4)
        y = np.concatenate([run.q[ra] - run.q[rc], run.q[rb] - run.q[rc]])  # [10, 3]
        acc += y @ y.T
        n += 3
    cov = acc / n
    # exact: Hessian of H0 + V_mix in the relative coordinates, kcal/mol/A^2
    beta = 1.0 / (kT / c["kcal"])

    def ring(P, m):
        kap = P * m / bh ** 2 / c["kcal"]
        Lm = np.zeros((P, P))
        for j in range(P):
            Lm[j, j] += 2
            Lm[j, (j + 1) % P] -= 1
            Lm[(j + 1) % P, j] -= 1
        return kap * Lm

    K = np.zeros((PA + PB, PA + PB))
    K[:PA, :PA] = ring(PA, mA)
    K[PA:, PA:] = ring(PB, mB)
    for sl in range(PA):                  # A-C, pair map (8,1), weight 1/8
        K[sl, sl] += k / PA
    for b in range(PB):                   # B-C, pair map (2,1), weight 1/2
        K[PA + b, PA + b] += k / PB
    for sl in range(PA):                  # A-B, pair map (8,2), weight 1/8
        b = sl * PB // PA
        K[sl, sl] += k / PA
        K[PA + b, PA + b] += k / PA
        K[sl, PA + b] -= k / PA
        K[PA + b, sl] -= k / PA
    exact = np.linalg.inv(beta * K)
    scale = np.abs(exact).max()
    assert np.abs(cov - exact).max() < 0.08 * scale
    # the coarse particle is mapped onto A's slices: its variance and the A-B
    # covariance carry the structure of the map
    assert np.mean(np.diag(cov)[PA:]) == pytest.approx(np.mean(np.diag(exact)[PA:]), rel=0.08)
    off = [cov[sl, PA + sl * PB // PA] for sl in range(PA)]
    off_ex = [exact[sl, PA + sl * PB // PA] for sl in range(PA)]
    assert np.mean(off) == pytest.approx(np.mean(off_ex), rel=0.1)


def test_free_ring_radius_of_gyration(orc):
    c, kT, bh = _consts(orc)
    P = 64
    m = synth.systems.MASS["e"]
    s = synth.harmonic_tether([P], [], masses=[m], seed=9)
    s.pseudo_type = np.array([1], dtype=np.int32)
    prm = orc.make_params(T=T, dt=2.0, tau=50.0, lam=1.0, seed=3)
    run = orc.Runner(s, prm)
    run.step(500)
    rg = []
    for _ in range(8000):
        run.step(4)
        rg.append(run.estimators()["Rg2"][0])
    ex = (P * P - 1) * (1.0 / kT) * c["hbar"] ** 2 / (4 * P * P * m)
    mu, er = block_mean(rg)
    assert abs(mu - ex) < 4 * er + 5e-3 * ex, (mu, er, ex)


def _nve_fluct(orc, dt, t_total):
    s = synth.water_box(32, 9.865, 8, 2, seed=0)
    prm = orc.make_params(T=T, dt=dt, tau=0.0, lam=0.0, seed=0)
    run = orc.Runner(s, prm)
    h, ke = [], []
    for _ in range(int(round(t_total / dt))):
        run.step(1)
        e = run.estimators()
        h.append(e["H_mix"])
        ke.append(e["KE_beads"])
    return np.array(h), np.array(ke)


def test_nve_conservation_dt2(orc):
    h1, ke1 = _nve_fluct(orc, 0.25, 40.0)
    h2, _ = _nve_fluct(orc, 0.125, 40.0)
    f1 = np.std(h1 - h1[0])
    f2 = np.std(h2 - h2[0])
    # energy is conserved to a small fraction of the kinetic-energy swings
    assert f1 < 0.01 * np.std(ke1)
    assert np.abs(h1 - h1[0]).max() < 0.005 * np.std(ke1)
    # second-order splitting: halving dt divides the fluctuation by ~4
    assert 3.0 < f1 / f2 < 5.5, (f1, f2)


def test_thermostat_heat_conserves_effective_energy(orc):
    """With PILE on, H_mix swings by the heat the thermostat exchanges, while
    H_mix + heat (heat = minus the kinetic energy the two O half steps add)
    is conserved to the integrator's own NVE level (Sec. "System I", PILE)."""
    s = synth.water_box(8, 8.4, 8, 2, seed=3)
    run = orc.Runner(s, orc.make_params(T=T, dt=0.25, tau=20.0, lam=1.0, seed=7))
    h, hc = [], []
    for _ in range(3000):
        run.step(1)
        e = run.estimators()
        h.append(e["H_mix"])
        hc.append(e["H_conserved"])
    h, hc = np.array(h), np.array(hc)
    nve = orc.Runner(s, orc.make_params(T=T, dt=0.25, tau=0.0, lam=0.0, seed=7))
    h0 = []
    for _ in range(3000):
        nve.step(1)
        h0.append(nve.estimators()["H_mix"])
    h0 = np.array(h0)
    assert np.std(h - h[0]) > 1.0                          # the thermostat does exchange heat
    assert np.std(hc - hc[0]) < 2e-3 * np.std(h - h[0])
    assert abs(hc[-1] - hc[0]) < 1e-2 * abs(h[-1] - h[0]) + 0.1
    assert np.std(hc - hc[0]) < 2.0 * np.std(h0 - h0[0])   # no worse than plain NVE


@pytest.mark.parametrize("P", [1, 8])
def test_rpmd_harmonic_centroid_vacf(orc, P):
    """Ring-polymer molecular dynamics in an external harmonic well (bead mass
    m/P, thermostat off): the centroid evolves in the well exactly, so its
    Kubo-transformed velocity autocorrelation is (3 kT / m) cos(w t) at any P
    (Sec. "Output and Analysis": RPMD correlation functions from NVE
    trajectories). Origins are sampled by PILE segments between NVE segments."""
    c, kT, bh = _consts(orc)
    m, M_anchor = 1.0, 1.0e9
    w = 2.0 / bh                               # beta hbar omega = 2
    k_kcal = m * w ** 2 / c["kcal"]
    s = synth.harmonic_tether([P, 1], [(0, 1, k_kcal)], masses=[m, M_anchor], seed=31 + P)
    s.bead_mass_type = orc.rpmd_bead_masses(s)
    run = orc.Runner(s, orc.make_params(T=T, dt=1.0, tau=10.0, lam=1.0, seed=40 + P))
    nve = orc.make_params(T=T, dt=1.0, tau=0.0, lam=0.0, seed=0)
    nvt = run.prm
    run.step(300)
    n_lag, segs = 41, 1500
    acc = np.zeros(n_lag)
    per_seg = []
    for _ in range(segs):
        run.prm = nve
        v0 = orc.centroid_velocities(s, run.p, 0)[0]
        cs = [float(v0 @ v0)]
        for _ in range(n_lag - 1):
            run.step(1)
            cs.append(float(v0 @ orc.centroid_velocities(s, run.p, 0)[0]))
        per_seg.append(cs)
        run.prm = nvt
        run.step(25)
    per_seg = np.array(per_seg)
    mean = per_seg.mean(axis=0)
    err = per_seg.std(axis=0, ddof=1) / np.sqrt(segs)
    t = np.arange(n_lag) * 1.0
    exact = 3.0 * kT / m * np.cos(w * t)
    assert np.all(np.abs(mean - exact) < 4 * err + 0.01 * exact[0]), np.max(np.abs(mean - exact) / err)
    # the accumulator over every origin of one NVE trajectory gives the same
    # lagged products as the direct loop above
    vc = orc.VelocityCorrelation(5)
    run.prm = nve
    frames = []
    for _ in range(12):
        run.step(1)
        v = orc.centroid_velocities(s, run.p, 0)
        frames.append(v)
        vc.add(v)
    for L in range(5):
        direct = sum(float(np.sum(frames[i] * frames[i - L])) for i in range(L, 12))
        assert vc.acc[L] == pytest.approx(direct, rel=1e-13)
        assert vc.cnt[L] == 12 - L
