"""Oracle pins: the bead index maps of Eq. (mts-hamiltonian) and the bead bookkeeping.

* Fig. 1 worked examples (golden file, exact).
* The verbatim 1-based pair/three-body maps equal the 0-based slice form
  b_x(s) = floor(s P_x / P*) for every power-of-two chain up to 1024.
* Bead-count sums of Table I / Table II.
"""
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
POW2 = [1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024]


def _read_fig1():
    rows = []
    for line in open(os.path.join(GOLD, "fig1_maps.txt")):
        if line.startswith("#") or not line.strip():
            continue
        head, pairs = line.split(":")
        n1, n2, w = head.split()
        ps = [tuple(int(v) for v in p.split("-")) for p in pairs.split()]
        rows.append((int(n1), int(n2), float(w), ps))
    return rows


@pytest.mark.parametrize("row", _read_fig1(), ids=lambda r: f"{r[0]}x{r[1]}")
def test_fig1_worked_examples(orc, row):
    n1, n2, w, pairs = row
    bi, bj = orc.pair_map(n1, n2)
    got = sorted(zip((bi + 1).tolist(), (bj + 1).tolist()))
    assert got == sorted(pairs)
    # weight 1/N_i of the finer particle
    assert 1.0 / n1 == pytest.approx(w, abs=0)


def test_pair_map_equals_slice_form(orc):
    for Ni in POW2:
        for Nj in POW2:
            if Nj > Ni:
                continue
            bi, bj = orc.pair_map(Ni, Nj)
            assert len(bi) == Ni
            s = np.arange(Ni)
            ref = sorted(zip(s.tolist(), (s * Nj // Ni).tolist()))
            assert sorted(zip(bi.tolist(), bj.tolist())) == ref
            # every fine bead once, every coarse bead Ni/Nj times
            assert np.array_equal(np.sort(bi), s)
            assert np.all(np.bincount(bj, minlength=Nj) == Ni // Nj)


def test_triple_map_equals_slice_form(orc):
    for Ni in POW2[:9]:
        for Nj in POW2:
            for Nk in POW2:
                if not (Ni >= Nj >= Nk):
                    continue
                b0, b1, b2 = orc.triple_map(Ni, Nj, Nk)
                s = np.arange(Ni)
                ref = sorted(zip(s.tolist(), (s * Nj // Ni).tolist(), (s * Nk // Ni).tolist()))
                assert sorted(zip(b0.tolist(), b1.tolist(), b2.tolist())) == ref


def test_triple_map_reduces_to_pair_map(orc):
    # a three-body term whose third particle is classical maps (i, j) exactly
    # as the pair term does
    for Ni, Nj in [(8, 2), (32, 4), (4, 4), (16, 1)]:
        b0, b1, _ = orc.triple_map(Ni, Nj, 1)
        p0, p1 = orc.pair_map(Ni, Nj)
        assert sorted(zip(b0.tolist(), b1.tolist())) == sorted(zip(p0.tolist(), p1.tolist()))


def test_bead_validation(orc):
    assert orc.validate_beads([1, 2, 4, 1024])
    assert not orc.validate_beads([3, 6])
    assert not orc.validate_beads([0])
    assert not orc.validate_beads([32, 12])


def test_table_bead_counts():
    import synth
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLD, "bead_counts.txt"))
            if l.strip() and not l.startswith("#")]
    for nw, ph, po, nion, pe, total in rows:
        assert synth.bead_counts_table(nw, ph, po, nion, 1, pe) == total
        ion = dict(synth.systems.ION3) if nion else None
        s = synth.water_box(nw, 14.0, ph, po, seed=0, ion=ion, electron_P=pe or None)
        assert s.n_beads == total
