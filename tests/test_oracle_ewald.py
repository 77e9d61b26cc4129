"""Oracle pins for the centroid long-range electrostatics (Ewald split: real
space erfc(alpha r)/r per bead pair, reciprocal space on the ring-polymer
centroids; Sec. "Theory", last paragraph).

* With one bead per atom the scheme is the plain Ewald sum: the rock-salt
  lattice gives the Madelung constant 1.747564594633 (a closed form of the
  textbook lattice sum, not of this code), for two splitting parameters.
* With one bead per atom the total is independent of the splitting parameter
  alpha for a charged (ion + water) system, which pins the self,
  intramolecular and neutralising-background corrections together. With
  beads it is not exactly: the real-space part sees the bead pairs and the
  reciprocal part the centroids, and the mismatch shrinks with the beads'
  spread around their centroids.
* Forces are minus the gradient (central differences), including the
  reciprocal force shared equally by an atom's beads; the virial is minus the
  dilation derivative.
"""
import math

import numpy as np
import pytest

import synth

MADELUNG_NACL = 1.747564594633


def _rock_salt(cells=2, a=5.64):
    """cells^3 conventional cubic cells of edge a: Na+ at fcc sites, Cl- shifted by a/2."""
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    pos, typ = [], []
    for i in range(cells):
        for j in range(cells):
            for k in range(cells):
                o = np.array([i, j, k], dtype=float)
                for f in fcc:
                    pos.append((o + f) * a)
                    typ.append(0)
                    pos.append((o + f + np.array([.5, 0, 0])) * a)
                    typ.append(1)
    n = len(pos)
    s = synth.harmonic_tether([1, 1], [], box=cells * a)
    s.type_of_atom = np.array(typ, dtype=np.int32)
    s.mol_of_atom = np.arange(n, dtype=np.int32)
    s.charge_type = np.array([1.0, -1.0])
    s.lj_eps = np.zeros((2, 2))
    s.bonds = np.zeros((0, 2), dtype=np.int32)
    s.bond_k = np.zeros(0)
    s.bond_r0 = np.zeros(0)
    rows = np.concatenate([np.where(s.type_of_atom == t)[0] for t in range(2)])
    s.q = np.array(pos)[rows] + 0.3  # type-block order; away from the box faces
    s.p = np.zeros_like(s.q)
    s.coulomb = 1
    return s, n


@pytest.mark.parametrize("alpha,kmax", [(0.45, 11), (0.55, 13)])
def test_ewald_rock_salt_madelung(orc, alpha, kmax):
    s, n = _rock_salt()
    s.ewald_kmax = kmax
    F, parts = orc.forces(s, r_cut=9.0, alpha=alpha)
    ke = orc.constants()["ke"]
    r0 = 5.64 / 2
    exact = -MADELUNG_NACL * ke * (n / 2) / r0
    assert parts[2] == pytest.approx(exact, rel=2e-7)
    # a perfect lattice: no net force on any ion
    assert np.abs(F).max() < 1e-6


def _ion_water(P_H=4, P_O=2, seed=2):
    s = synth.water_box(27, 9.3, P_H, P_O, seed=seed, ion=dict(synth.systems.ION3))
    s.q = s.q + np.random.default_rng(seed + 1).normal(0, 0.05, s.q.shape)
    s.coulomb = 1
    return s


def test_ewald_total_independent_of_alpha(orc):
    """Charged classical system (+3 ion in water, one bead per atom): real +
    reciprocal + corrections do not depend on the splitting (r_cut = 9 A with
    alpha >= 0.5 leaves erfc(alpha r_cut) < 3e-10)."""
    s = _ion_water(1, 1)
    vals = []
    for alpha, kmax in [(0.5, 11), (0.6, 13)]:
        s.ewald_kmax = kmax
        vals.append(orc.forces(s, r_cut=9.0, alpha=alpha)[1][2])
    assert vals[0] == pytest.approx(vals[1], rel=1e-8)
    # with beads the centroid approximation of the long-range part depends
    # (weakly) on where the split sits; collapsing every ring polymer onto its
    # centroid restores the classical independence
    sb = _ion_water(8, 2)
    vb = []
    for alpha, kmax in [(0.5, 11), (0.6, 13)]:
        sb.ewald_kmax = kmax
        vb.append(orc.forces(sb, r_cut=9.0, alpha=alpha)[1][2])
    assert 1e-8 < abs(vb[0] - vb[1]) / abs(vb[0]) < 1e-3
    for atom in range(sb.n_atoms):
        rows = sb.bead_rows(atom)
        sb.q[rows] = sb.q[rows].mean(axis=0)
    vc = []
    for alpha, kmax in [(0.5, 11), (0.6, 13)]:
        sb.ewald_kmax = kmax
        vc.append(orc.forces(sb, r_cut=9.0, alpha=alpha)[1][2])
    assert vc[0] == pytest.approx(vc[1], rel=1e-8)


def test_ewald_forces_are_gradient(orc):
    s = _ion_water(8, 2, seed=5)
    s.ewald_kmax = 8
    F, parts = orc.forces(s, alpha=0.35)
    rng = np.random.default_rng(1)
    h = 1e-5
    for r in rng.choice(s.n_beads, 16, replace=False):
        for d in range(3):
            qp = s.q.copy(); qp[r, d] += h
            qm = s.q.copy(); qm[r, d] -= h
            fd = -(orc.forces(s, qp, alpha=0.35)[1][0] - orc.forces(s, qm, alpha=0.35)[1][0]) / (2 * h)
            assert F[r, d] == pytest.approx(fd, rel=2e-6, abs=2e-6)


def test_ewald_virial_is_dilation_derivative(orc):
    s = _ion_water(4, 4, seed=7)
    s.ewald_kmax = 8
    F, parts = orc.forces(s, alpha=0.35)
    h = 1e-6

    def dil(lam):
        d = s.copy()
        d.box = s.box * lam
        d.q = s.q * lam
        return orc.forces(d, alpha=0.35)[1][0]
    w_fd = -(dil(1 + h) - dil(1 - h)) / (2 * h)
    assert parts[6] == pytest.approx(w_fd, rel=2e-7, abs=1e-6 * abs(parts[0]))


def test_ewald_recip_depends_on_centroids_only(orc):
    """The reciprocal part sees only the centroids: collapsing every ring
    polymer onto its centroid leaves it unchanged (the reciprocal part is the
    difference between the full sum and the same sum without wave vectors,
    which keeps the real space and the centroid corrections)."""
    s = _ion_water(8, 2, seed=9)
    s.ewald_kmax = 8
    c = s.copy()
    for atom in range(c.n_atoms):
        rows = c.bead_rows(atom)
        c.q[rows] = c.q[rows].mean(axis=0)
    s0, c0 = s.copy(), c.copy()
    s0.ewald_kmax = c0.ewald_kmax = 0
    rec_s = orc.forces(s, alpha=0.35)[1][2] - orc.forces(s0, alpha=0.35)[1][2]
    rec_c = orc.forces(c, alpha=0.35)[1][2] - orc.forces(c0, alpha=0.35)[1][2]
    assert abs(rec_s) > 1.0
    assert rec_s == pytest.approx(rec_c, rel=1e-12)
