"""Oracle pin: the radial distribution histogram against an independent
numpy brute force that uses the 0-based slice map b_x(s) = floor(s P_x / P*)
(the oracle walks the paper's verbatim pair map), plus the ideal-gas limit
of the normalisation."""
import numpy as np
import pytest

import synth


def _numpy_hist(s, ta, tb, dr, nbins):
    off = s.type_offsets()
    N = s.n_of_type()
    rank = s.rank_in_type()
    h = np.zeros(nbins)
    L = s.box
    for a in range(s.n_atoms):
        if s.type_of_atom[a] != ta:
            continue
        for c in range(s.n_atoms):
            if c == a or s.type_of_atom[c] != tb:
                continue
            Pa, Pc = s.P_type[s.type_of_atom[a]], s.P_type[s.type_of_atom[c]]
            Ps = max(Pa, Pc)
            sl = np.arange(Ps)
            ba, bc = sl * Pa // Ps, sl * Pc // Ps
            ra = off[ta] + ba * N[ta] + rank[a]
            rc = off[tb] + bc * N[tb] + rank[c]
            # finer particle first, as the pair term is written
            if Pc > Pa:
                d0 = s.q[ra] - s.q[rc]
            else:
                d0 = s.q[rc] - s.q[ra]
            n0 = -np.rint(d0 / L)
            same = s.mol_of_atom[a] == s.mol_of_atom[c]
            for ix in range(-2, 3):
                for iy in range(-2, 3):
                    for iz in range(-2, 3):
                        n = n0 + np.array([ix, iy, iz])
                        keep = ~(same & np.all(n == 0, axis=1)) if same else np.ones(Ps, bool)
                        dx = d0[:, 0] + n[:, 0] * L
                        dy = d0[:, 1] + n[:, 1] * L
                        dz = d0[:, 2] + n[:, 2] * L
                        r = np.sqrt(dx * dx + dy * dy + dz * dz)
                        ok = keep & (r < nbins * dr)
                        k = np.floor(r[ok] / dr).astype(int)
                        k = k[k < nbins]
                        np.add.at(h, k, 1.0 / Ps)
    return h


@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_rdf_hist_matches_numpy_brute_force(orc, ta, tb):
    s = synth.water_box(16, synth.density_box_length(16), 8, 2, seed=4)
    s.q = s.q + np.random.default_rng(5).normal(0, 0.1, s.q.shape)
    h = orc.rdf_hist(s, ta, tb, dr=0.05, nbins=140)
    ref = _numpy_hist(s, ta, tb, 0.05, 140)
    assert np.array_equal(h, ref)
    # (a, b) and (b, a) count the same ordered pairs
    if ta != tb:
        assert np.array_equal(h, orc.rdf_hist(s, tb, ta, dr=0.05, nbins=140))


def test_rdf_normalisation_ideal_gas(orc):
    """Uncorrelated positions (atoms placed uniformly, no molecules within
    range that matter at large r) give g(r) -> 1 at large r."""
    s = synth.water_box(64, synth.density_box_length(64), 1, 1, seed=6)
    rng = np.random.default_rng(7)
    N = s.n_of_type()
    frames, acc = 6, np.zeros(150)
    for f in range(frames):
        s.q = rng.uniform(0, s.box, s.q.shape)
        acc += orc.rdf_hist(s, 0, 0, dr=0.05, nbins=150)
    g = orc.rdf_normalise(acc, frames, N[0], N[0], True, s.box, 0.05)
    tail = g[80:150]  # 4-7.5 A
    assert abs(tail.mean() - 1.0) < 0.05
