"""Oracle pins on individual terms, each against something other than the
oracle's own code.

* Bonded energies (Eq. mts-hamiltonian: a bond through the pair map, the
  H-O-H angle through the nested three-body map) against closed forms on one
  molecule and against an independent numpy evaluation in the slice form
  b_x(s) = floor(s P_x / P*), weight 1/P*, in both orientations of the water
  bead counts (H finer than O and O finer than H).
* The virial (sum over terms of r . f) against minus the derivative of V_mix
  under a uniform dilation of every position and the box: each term depends
  on its distances only (or, for the angle, on none of their scale).
* The pseudopotential's small-r series branch against erf(x)/x evaluated in
  30-digit arithmetic, and continuity of value and force across the switch.
* The pseudo-particle site list is complete: every in-cutoff
  (electron bead, site bead, image) term has its entry.
"""
import math

import mpmath
import numpy as np
import pytest

import synth

RC = 9.0


def _small(P_H, P_O, P_e=None, seed=3, spread=0.08, ion=True):
    s = synth.water_box(8, 8.4, P_H, P_O, seed=seed, ion=dict(synth.systems.ION3) if ion else None,
                        electron_P=P_e)
    rng = np.random.default_rng(seed + 100)
    s.q = s.q + rng.normal(0, spread, s.q.shape)
    return s


def test_bonded_closed_form_one_molecule(orc):
    """One classical water: V_bond = k/2 sum (r - r0)^2, V_angle = k/2 (theta - theta0)^2."""
    s = synth.water_box(1, 30.0, 1, 1, seed=0, jitter=0.0)
    w = synth.systems.WATER
    k_b, r0, k_a = w["bond_k"], w["bond_r0"], w["angle_k"]
    th0 = math.radians(w["angle_theta0_deg"])
    o = np.array([15.0, 15.0, 15.0])
    d1, d2, dth = 0.1, -0.05, 0.2
    th = th0 + dth
    u1 = np.array([math.sin(th / 2), 0.0, math.cos(th / 2)])
    u2 = np.array([-math.sin(th / 2), 0.0, math.cos(th / 2)])
    pos = np.array([o, o + (r0 + d1) * u1, o + (r0 + d2) * u2])
    q = np.zeros((s.n_beads, 3))
    for a in range(3):
        q[s.bead_rows(a)] = pos[a]
    F, parts = orc.forces(s, q)
    assert parts[3] == pytest.approx(0.5 * k_b * (d1 ** 2 + d2 ** 2), rel=1e-12)
    assert parts[4] == pytest.approx(0.5 * k_a * dth ** 2, rel=1e-10)
    # at the reference geometry both vanish
    s0 = synth.water_box(1, 30.0, 4, 2, seed=0, jitter=0.0)
    F0, p0 = orc.forces(s0)
    assert abs(p0[3]) < 1e-20 and abs(p0[4]) < 1e-20


def _bonded_slice_form(s):
    """V_bond, V_angle from the slice form of the bead maps (numpy)."""
    Pa = s.P_type[s.type_of_atom]
    vb = 0.0
    for b, (a, c) in enumerate(s.bonds):
        Ps = max(Pa[a], Pa[c])
        sl = np.arange(Ps)
        xa = s.q[s.bead_rows(a)[sl * Pa[a] // Ps]]
        xc = s.q[s.bead_rows(c)[sl * Pa[c] // Ps]]
        r = np.linalg.norm(xc - xa, axis=1)
        vb += np.sum(0.5 * s.bond_k[b] * (r - s.bond_r0[b]) ** 2) / Ps
    va = 0.0
    for g, (a1, o, a2) in enumerate(s.angles):
        Ps = max(Pa[a1], Pa[o], Pa[a2])
        sl = np.arange(Ps)
        x1 = s.q[s.bead_rows(a1)[sl * Pa[a1] // Ps]]
        xo = s.q[s.bead_rows(o)[sl * Pa[o] // Ps]]
        x2 = s.q[s.bead_rows(a2)[sl * Pa[a2] // Ps]]
        u, v = x1 - xo, x2 - xo
        cs = np.sum(u * v, axis=1) / (np.linalg.norm(u, axis=1) * np.linalg.norm(v, axis=1))
        th = np.arccos(np.clip(cs, -1.0, 1.0))
        va += np.sum(0.5 * s.angle_k[g] * (th - s.angle_theta0[g]) ** 2) / Ps
    return vb, va


@pytest.mark.parametrize("P_H,P_O", [(8, 2), (1, 4), (4, 8), (16, 16)])
def test_bonded_against_slice_form(orc, P_H, P_O):
    s = _small(P_H, P_O, spread=0.06)
    F, parts = orc.forces(s)
    vb, va = _bonded_slice_form(s)
    assert parts[3] == pytest.approx(vb, rel=1e-12)
    assert parts[4] == pytest.approx(va, rel=1e-11)


def _dilated(s, lam):
    d = s.copy()
    d.box = s.box * lam
    d.q = s.q * lam
    return d


@pytest.mark.parametrize("P_H,P_O,P_e", [(8, 2, 16), (1, 4, None), (4, 4, 8)])
def test_virial_is_dilation_derivative(orc, P_H, P_O, P_e):
    s = _small(P_H, P_O, P_e, seed=5, spread=0.05)
    F, parts = orc.forces(s)
    h = 1e-6
    vp = orc.forces(_dilated(s, 1 + h))[1][0]
    vm = orc.forces(_dilated(s, 1 - h))[1][0]
    w_fd = -(vp - vm) / (2 * h)
    assert parts[6] == pytest.approx(w_fd, rel=2e-7, abs=1e-6 * abs(parts[0]))


def _electron_site(r_over_sigma, A_eV=0.0, sigma=0.5, charge=0.41, b=0.4):
    s = synth.harmonic_tether([1, 1], [], box=60.0)
    s.pseudo_type = np.array([0, 1], dtype=np.int32)
    s.charge_type = np.array([charge, -1.0])
    s.pp_sigma = np.array([sigma, 1.0])
    s.pp_A_eV = np.array([A_eV, 0.0])
    s.pp_b = np.array([b, 1.0])
    s.mol_of_atom = np.array([0, 1], dtype=np.int32)
    q = np.zeros((2, 3)) + 30.0
    q[1, 2] += r_over_sigma * sigma
    s.q = q
    return s


def _pseudo_ref(orc, r, A_eV=0.0, sigma=0.5, charge=0.41, b=0.4):
    """Shifted-force V(r) and dV/dr(r) - dV/dr(rc) in 30-digit arithmetic."""
    c = orc.constants()
    mpmath.mp.dps = 30
    kq = mpmath.mpf(c["ke"]) * mpmath.mpf(charge)
    A = mpmath.mpf(A_eV) * mpmath.mpf(c["ev_kcal"])
    sig, bb = mpmath.mpf(sigma), mpmath.mpf(b)
    V = lambda x: -kq * mpmath.erf(x / sig) / x + A * mpmath.exp(-x / bb)
    dV = lambda x: mpmath.diff(V, x)
    r, R = mpmath.mpf(r), mpmath.mpf(RC)
    return float(V(r) - V(R) - (r - R) * dV(R)), float(dV(r) - dV(R))


@pytest.mark.parametrize("x", [1e-5, 5e-4, 9.99e-4, 2e-3])
def test_pseudopotential_small_r_series(orc, x):
    s = _electron_site(x)
    F, parts = orc.forces(s)
    r = float(np.linalg.norm(s.q[1] - s.q[0]))
    v_ref, dv_ref = _pseudo_ref(orc, r)
    assert parts[5] == pytest.approx(v_ref, rel=1e-13)
    # the electron sits at +z from the site: the force on the site along +z
    # is dV/dr - dV/dr(rc) (attraction pulls it towards the electron)
    # above the switch the analytic dg/dr = 2 e^{-x^2}/(sqrt(pi) sigma r) - erf(x)/r^2
    # cancels two terms ~1/(sigma r): rounding of order eps/x^2 of dg
    assert F[0, 2] == pytest.approx(dv_ref, rel=1e-12 if x < 1e-3 else 1e-10)


def test_pseudopotential_small_r_slope(orc):
    """Force differences between small-r points cancel the cutoff shift and
    expose the series derivative -(2/sqrt(pi)) (2x/3 - 2x^3/5) / sigma^2."""
    F1 = orc.forces(_electron_site(1e-5))[0][0, 2]
    F2 = orc.forces(_electron_site(5e-4))[0][0, 2]
    r1 = float(np.linalg.norm(_electron_site(1e-5).q[1] - _electron_site(1e-5).q[0]))
    r2 = float(np.linalg.norm(_electron_site(5e-4).q[1] - _electron_site(5e-4).q[0]))
    d1 = _pseudo_ref(orc, r1)[1]
    d2 = _pseudo_ref(orc, r2)[1]
    assert (F1 - F2) == pytest.approx(d1 - d2, rel=1e-7)


def test_pseudopotential_switch_continuity(orc):
    # only the erf part switches branch; the two points are 1e-12 A apart
    lo = orc.forces(_electron_site(1e-3 * (1 - 1e-9)))
    hi = orc.forces(_electron_site(1e-3 * (1 + 1e-9)))
    assert lo[1][5] == pytest.approx(hi[1][5], rel=1e-12)
    assert lo[0][0, 2] == pytest.approx(hi[0][0, 2], rel=1e-9)


def test_pseudo_list_complete(orc):
    s = _small(8, 2, 32, seed=21, spread=0.1)
    tl, th = orc.pseudo_list(s)
    have = set(map(tuple, tl.tolist()))
    L = s.box
    Pt = s.P_type[s.type_of_atom]
    ref = lambda a: s.q[s.bead_rows(a)[0]] - L * np.floor(s.q[s.bead_rows(a)[0]] / L)
    electrons = [a for a in range(s.n_atoms) if s.pseudo_type[s.type_of_atom[a]]]
    sites = [a for a in range(s.n_atoms) if not s.pseudo_type[s.type_of_atom[a]]]
    n_in = 0
    for e in electrons:
        for c in sites:
            for sl in range(Pt[e]):
                xe = s.q[s.bead_rows(e)[sl]]
                xc = s.q[s.bead_rows(c)[sl * Pt[c] // Pt[e]]]
                for nx in range(-3, 4):
                    for ny in range(-3, 4):
                        for nz in range(-3, 4):
                            n = np.array([nx, ny, nz])
                            if np.linalg.norm(xc - xe + n * L) >= RC:
                                continue
                            m = n + np.round(((xc - xe + n * L) - (ref(c) - ref(e))) / L - n).astype(int)
                            key = (e, c, int((m[0] + 2) * 25 + (m[1] + 2) * 5 + m[2] + 2))
                            assert key in have, key
                            n_in += 1
    assert n_in > 0
    # and the count of in-cutoff terms is the oracle's pseudopotential evaluation count
    assert orc.forces(s)[1][8] == n_in
