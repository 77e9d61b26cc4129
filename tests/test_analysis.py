"""Host-side summaries of the analysis module (block statistics, RDF peaks),
and one short sampled run and sweep on the GPU."""
import numpy as np
import pytest

import synth


def test_block_stats_and_first_peak():
    from paper_2411_11988_gb300 import analysis
    x = np.arange(16, dtype=float)
    m, e = analysis.block_stats(x, 4)
    blocks = x.reshape(4, 4).mean(axis=1)
    assert m == blocks.mean() and np.isclose(e, blocks.std(ddof=1) / 2)
    v = np.stack([x, 2 * x], axis=1)  # per-type columns
    m2, _ = analysis.block_stats(v, 4)
    assert np.allclose(m2, [x.mean(), 2 * x.mean()])
    g = np.zeros(100)
    g[10], g[40] = 5.0, 3.0  # an intramolecular-like spike below r_min is skipped
    assert analysis.first_peak(g, 0.1, 2.0) == (pytest.approx(4.05), 3.0)
    with pytest.raises(ValueError):
        analysis.block_stats([1.0, 2.0], 8)


@pytest.mark.gpu
def test_sample_and_sweep_on_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2411_11988_gb300 import MixTS, analysis
    s = synth.water_box(32, 9.865, 8, 2, seed=0)
    m = MixTS(s, seed=3)
    res = analysis.sample(m, 50, 160, 10, pairs=[(0, 0), (0, 1)], dr=0.05, nbins=160)
    m.close()
    assert res["frames"] == 16
    ke, ke_err = res["KE_cv"]
    assert ke.shape == (2,) and np.all(ke > 0) and np.all(ke_err >= 0)
    assert set(res["g"]) == {(0, 0), (0, 1)} and res["g"][(0, 0)].shape == (160,)
    sw = analysis.quantisation_sweep(lambda ph, po: synth.water_box(32, 9.865, ph, po, seed=0), [(1, 1), (4, 2)],
                                     n_eq=20, n_samp=80, every=10, pairs=((0, 0),), dr=0.05)
    assert set(sw) == {"H1_O1", "H4_O2"}
    assert set(sw["H4_O2"]["KE_cv_kcal_mol"]) == {"O", "H"}
