"""Oracle pins: the mixTS potential and its forces.

* Constants against scipy.constants (CODATA / exact SI).
* Two-body energies against the textbook DSF (Fennell-Gezelter) and LJ forms
  evaluated with scipy's erfc, value and slope vanishing at the cutoff.
* The equal-P limit (standard PIMD) and, more generally, V_mix as the average
  over the P_max slices of the finest grid of classical (P = 1) energies of
  slice configurations; forces likewise.
* All P = 1 (classical MD) against an independent vectorised numpy evaluation.
* Central finite differences, translation invariance, periodicity.
"""
import math

import numpy as np
import pytest
import scipy.constants as sc
from scipy.special import erfc, erf

import synth

RC = 9.0
ALPHA = 0.2


def test_constants(orc):
    c = orc.constants()
    amu = 1e-3 / sc.N_A
    e_md = amu * 1e-20 / 1e-30
    assert c["kB"] == pytest.approx(sc.k / e_md, rel=1e-14)
    assert c["hbar"] == pytest.approx(sc.hbar / (e_md * 1e-15), rel=1e-14)
    assert c["kcal"] == pytest.approx(4184.0 / sc.N_A / e_md, rel=1e-14)
    # epsilon_0 is measured: CODATA 2018 (oracle) and later editions differ by ~1e-9
    assert c["ke"] == pytest.approx(sc.e ** 2 / (4 * math.pi * sc.epsilon_0) * 1e10 * sc.N_A / 4184.0, rel=1e-8)
    assert c["ke"] == pytest.approx(332.0637, rel=1e-6)


def _two_site(r, qa, qb, eps, sig, P=(1, 1)):
    s = synth.harmonic_tether([P[0], P[1]], [], box=60.0)
    s.charge_type = np.array([qa, qb])
    s.lj_eps = np.array([[0.0, eps], [eps, 0.0]])
    s.lj_sig = np.array([[1.0, sig], [sig, 1.0]])
    s.mol_of_atom = np.array([0, 1], dtype=np.int32)
    q = np.zeros((s.n_beads, 3)) + 30.0
    q[s.bead_rows(1), 0] += r
    s.q = q
    return s


def _dsf_ref(r, qq, ke):
    rc, a = RC, ALPHA
    cf = erfc(a * rc) / rc ** 2 + 2 * a / math.sqrt(math.pi) * math.exp(-a * a * rc * rc) / rc
    return ke * qq * (erfc(a * r) / r - erfc(a * rc) / rc + cf * (r - rc))


def _lj_sf_ref(r, eps, sig):
    v = lambda x: 4 * eps * ((sig / x) ** 12 - (sig / x) ** 6)
    dv = lambda x: -24 * eps * (2 * (sig / x) ** 12 - (sig / x) ** 6) / x
    return v(r) - v(RC) - (r - RC) * dv(RC)


@pytest.mark.parametrize("r", [1.7, 2.8, 3.3, 4.9, 7.2, 8.95])
def test_two_body_textbook(orc, r):
    ke = orc.constants()["ke"]
    s = _two_site(r, -0.82, 0.41, 0.1554, 3.1655)
    F, parts = orc.forces(s)
    assert parts[2] == pytest.approx(_dsf_ref(r, -0.82 * 0.41, ke), rel=1e-12)
    assert parts[1] == pytest.approx(_lj_sf_ref(r, 0.1554, 3.1655), rel=1e-12, abs=1e-15)
    # force on the second site = -dV/dr along +x
    h = 1e-5
    vp = _dsf_ref(r + h, -0.82 * 0.41, ke) + _lj_sf_ref(r + h, 0.1554, 3.1655)
    vm = _dsf_ref(r - h, -0.82 * 0.41, ke) + _lj_sf_ref(r - h, 0.1554, 3.1655)
    assert F[1, 0] == pytest.approx(-(vp - vm) / (2 * h), rel=1e-7)
    assert F[0, 0] == pytest.approx(-F[1, 0], rel=1e-14)


def test_cutoff_continuity(orc):
    for r in [RC - 1e-7, RC + 1e-7]:
        s = _two_site(r, 1.0, -1.0, 0.3, 3.0)
        F, parts = orc.forces(s)
        assert abs(parts[0]) < 1e-10
        assert np.abs(F).max() < 1e-6


def _pseudo_pair_system(r, tsite="O"):
    s = synth.water_box(1, 40.0, 1, 1, seed=0, electron_P=1)
    return s


def test_pseudopotential_textbook(orc):
    # one electron bead and one classical site at distance r
    c = orc.constants()
    for r in [0.3, 1.1, 2.5, 6.0]:
        s = synth.harmonic_tether([1, 1], [], box=60.0)
        s.pseudo_type = np.array([0, 1], dtype=np.int32)
        s.charge_type = np.array([0.41, -1.0])
        s.pp_sigma = np.array([0.5, 1.0])
        s.pp_A_eV = np.array([5.0, 0.0])
        s.pp_b = np.array([0.4, 1.0])
        s.mol_of_atom = np.array([0, 1], dtype=np.int32)
        q = np.zeros((2, 3)) + 30.0
        q[1, 1] += r
        s.q = q
        F, parts = orc.forces(s)
        A = 5.0 * c["ev_kcal"]
        v = lambda x: -c["ke"] * 0.41 * erf(x / 0.5) / x + A * math.exp(-x / 0.4)
        h = 1e-6
        dv = lambda x: (v(x + h) - v(x - h)) / (2 * h)
        ref = v(r) - v(RC) - (r - RC) * dv(RC)
        assert parts[5] == pytest.approx(ref, rel=1e-8)
        assert F[1, 1] == pytest.approx(-(dv(r) - dv(RC)), rel=1e-6)


def _small_mixed_system(P_H=8, P_O=2, P_e=16, seed=3):
    s = synth.water_box(8, 8.4, P_H, P_O, seed=seed, ion=dict(synth.systems.ION3), electron_P=P_e)
    rng = np.random.default_rng(seed + 100)
    s.q = s.q + rng.normal(0, 0.08, s.q.shape)
    return s


def _replica(sysm, s_idx, Pmax):
    """Classical (P = 1) copy holding, for every atom, its bead floor(s P_a / Pmax)."""
    r = sysm.copy()
    r.P_type = np.ones_like(sysm.P_type)
    q = np.zeros((sysm.n_atoms, 3))
    for a in range(sysm.n_atoms):
        Pa = sysm.P_type[sysm.type_of_atom[a]]
        q[a] = sysm.q[sysm.bead_rows(a)[s_idx * Pa // Pmax]]
    # P = 1 layout: one row per atom, in type-block order
    rows = np.concatenate([np.where(sysm.type_of_atom == t)[0] for t in range(sysm.n_types)])
    r.q = q[rows]
    return r, rows


@pytest.mark.parametrize("Ps", [(4, 4, 4), (8, 2, 16), (32, 4, 32)])
def test_vmix_is_slice_average(orc, Ps):
    s = _small_mixed_system(*Ps)
    Pmax = int(s.P_type.max())
    F, parts = orc.forces(s)
    V = 0.0
    Fslice = np.zeros_like(F)
    for si in range(Pmax):
        r, rows = _replica(s, si, Pmax)
        Fr, pr = orc.forces(r)
        V += pr[0] / Pmax
        # classical row j is atom rows[j]
        for j, a in enumerate(rows):
            Pa = s.P_type[s.type_of_atom[a]]
            Fslice[s.bead_rows(a)[si * Pa // Pmax]] += Fr[j] / Pmax
    assert parts[0] == pytest.approx(V, rel=1e-12)
    rms = np.sqrt(np.mean(F ** 2))
    assert np.abs(F - Fslice).max() / rms < 1e-12


def _numpy_classical(s, rc=RC, a=ALPHA, ke=None):
    """Independent vectorised classical force-field energy (all P = 1)."""
    x = s.q  # P=1: rows in type-block order
    rows = np.concatenate([np.where(s.type_of_atom == t)[0] for t in range(s.n_types)])
    pos = np.zeros((s.n_atoms, 3))
    pos[rows] = x
    L = s.box
    typ = s.type_of_atom
    ch = s.charge_type[typ]
    nonp = s.pseudo_type[typ] == 0
    e_lj = e_c = e_pp = 0.0
    n = np.arange(-2, 3)
    shifts = np.array(np.meshgrid(n, n, n, indexing="ij")).reshape(3, -1).T * L
    cf = erfc(a * rc) / rc ** 2 + 2 * a / math.sqrt(math.pi) * math.exp(-a * a * rc * rc) / rc
    for i in range(s.n_atoms):
        for j in range(i + 1, s.n_atoms):
            d_unw = pos[j] - pos[i]
            back = L * np.round(d_unw / L)
            dd = (d_unw - back)[None, :] + shifts
            r = np.sqrt((dd ** 2).sum(1))
            if s.mol_of_atom[i] == s.mol_of_atom[j]:
                # the unwrapped (zero-image) partner of the own molecule is excluded
                r = r[np.abs(shifts - back).max(axis=1) > 1e-9]
            r = r[r < rc]
            if nonp[i] and nonp[j]:
                eps = s.lj_eps[typ[i], typ[j]]
                sig = s.lj_sig[typ[i], typ[j]]
                if eps:
                    e_lj += sum(_lj_sf_ref(v, eps, sig) for v in r)
                e_c += sum(_dsf_ref(v, ch[i] * ch[j], ke) for v in r)
    return e_lj, e_c


def test_classical_limit_matches_independent(orc):
    ke = orc.constants()["ke"]
    s = synth.water_box(8, 8.4, 1, 1, seed=5, ion=dict(synth.systems.ION3))
    F, parts = orc.forces(s)
    e_lj, e_c = _numpy_classical(s, ke=ke)
    assert parts[1] == pytest.approx(e_lj, rel=1e-11)
    assert parts[2] == pytest.approx(e_c, rel=1e-11)


def test_finite_difference_forces(orc):
    s = _small_mixed_system(8, 2, 16, seed=7)
    F, parts = orc.forces(s)
    rng = np.random.default_rng(0)
    h = 1e-5
    rows = rng.choice(s.n_beads, 24, replace=False)
    for r in rows:
        for d in range(3):
            qp = s.q.copy(); qp[r, d] += h
            qm = s.q.copy(); qm[r, d] -= h
            vp = orc.forces(s, qp)[1][0]
            vm = orc.forces(s, qm)[1][0]
            fd = -(vp - vm) / (2 * h)
            assert F[r, d] == pytest.approx(fd, rel=2e-6, abs=2e-6)


def test_bead_force_matches_full(orc):
    s = _small_mixed_system(8, 2, 16, seed=9)
    F, _ = orc.forces(s)
    for atom, bead in [(0, 0), (0, 1), (1, 5), (4, 7), (24, 0), (25, 11)]:
        row = s.bead_rows(atom)[bead]
        assert np.allclose(orc.bead_force(s, atom, bead), F[row], rtol=1e-12, atol=1e-12)


def test_translation_and_periodicity(orc):
    s = _small_mixed_system(8, 2, 16, seed=11)
    F, parts = orc.forces(s)
    assert np.abs(F.sum(0)).max() < 1e-9 * np.abs(F).max()
    # rigid translation
    q2 = s.q + np.array([0.37, -1.3, 2.2])
    F2, p2 = orc.forces(s, q2)
    assert p2[0] == pytest.approx(parts[0], rel=1e-12)
    assert np.abs(F2 - F).max() < 1e-10
    # move one whole molecule (all beads of its atoms) by a lattice vector
    q3 = s.q.copy()
    for a in (0, 1, 2):
        q3[s.bead_rows(a)] += np.array([s.box, 0.0, -2 * s.box])
    F3, p3 = orc.forces(s, q3)
    assert p3[0] == pytest.approx(parts[0], rel=1e-12)
    assert np.abs(F3 - F).max() < 1e-10


def _straddling(s, shift):
    """Rigid translation that leaves some molecules across the box faces:
    each atom's bead 0 is wrapped into the box on its own, so atoms of one
    molecule end up in different images of the wrapped frame."""
    t = s.copy()
    t.q = s.q + np.asarray(shift)
    L = s.box
    w = np.array([np.floor(t.q[t.bead_rows(a)[0]] / L) for a in range(t.n_atoms)])
    split = any(len({tuple(w[a]) for a in np.where(t.mol_of_atom == m)[0]}) > 1 for m in set(t.mol_of_atom.tolist()))
    return t, split


@pytest.mark.parametrize("shift", [(0.0, 0.0, 0.0), (1.9, -0.7, 3.3), (-4.2, 2.6, -0.35)])
def test_neighbour_list_complete(orc, shift):
    s, split = _straddling(_small_mixed_system(8, 2, 16, seed=13), shift)
    assert split or not any(shift)
    tl, dmax, R = orc.nlist(s)
    assert R == pytest.approx(RC + 2 * dmax)
    # canonical form: lower atom first, each (pair, image) once
    assert np.all(tl[:, 0] < tl[:, 1])
    assert len(set(map(tuple, tl.tolist()))) == len(tl)
    have = set(map(tuple, tl.tolist()))
    L = s.box
    P = s.P_type[s.type_of_atom]
    nonp = s.pseudo_type[s.type_of_atom] == 0
    ref = lambda a: s.q[s.bead_rows(a)[0]] - L * np.floor(s.q[s.bead_rows(a)[0]] / L)
    for a in range(s.n_atoms):
        for c in range(a + 1, s.n_atoms):
            if not (nonp[a] and nonp[c]):
                continue
            fine, coarse = (a, c) if P[a] >= P[c] else (c, a)
            Pf, Pc = P[fine], P[coarse]
            for bf in range(Pf):
                # displacement from a's bead to c's bead on the pair's fine grid
                xa = s.q[s.bead_rows(a)[bf if a == fine else bf * Pc // Pf]]
                xc = s.q[s.bead_rows(c)[bf if c == fine else bf * Pc // Pf]]
                for nx in range(-3, 4):
                    for ny in range(-3, 4):
                        for nz in range(-3, 4):
                            n = np.array([nx, ny, nz])
                            if s.mol_of_atom[a] == s.mol_of_atom[c] and not n.any():
                                continue
                            if np.linalg.norm(xc - xa + n * L) >= RC:
                                continue
                            # the same image in the wrapped-reference frame
                            m = n + np.round(((xc - xa + n * L) - (ref(c) - ref(a))) / L - n).astype(int)
                            key = (a, c, int((m[0] + 2) * 25 + (m[1] + 2) * 5 + m[2] + 2))
                            assert key in have, key
    # a same-molecule pair is never listed at the zero image of the unwrapped
    # coordinates (its bonded terms act there), whatever frame wrapping put it in
    for a in range(s.n_atoms):
        for c in range(a + 1, s.n_atoms):
            if s.mol_of_atom[a] != s.mol_of_atom[c] or not (nonp[a] and nonp[c]):
                continue
            m = np.round(((s.q[s.bead_rows(c)[0]] - s.q[s.bead_rows(a)[0]]) - (ref(c) - ref(a))) / L).astype(int)
            assert (a, c, int((m[0] + 2) * 25 + (m[1] + 2) * 5 + m[2] + 2)) not in have
