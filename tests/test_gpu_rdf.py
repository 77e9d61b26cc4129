"""Radial distribution histograms and long-run statistics, CUDA path vs the
oracle (GPU only).

The histogram is integer work: it must equal the oracle's bin for bin (the
bins come from FP64 distances on both sides; a distance within ~1e-15 A of a
bin edge could in principle fall on the other side, which has never been
seen at these sizes). The long runs compare time averages of the
centroid-virial kinetic energy per type, the bead temperature and g(r)
around the first peaks between a GPU run and an oracle run from the same
start with independent thermostat noise, within 4 combined block standard
errors.
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


def _gpu_hist(m, ta, tb, dr, nbins):
    import torch
    h = torch.zeros(nbins, dtype=torch.int64, device=m.device)
    m.rdf_accumulate(ta, tb, h, dr)
    return h.cpu().numpy().astype(np.float64)


def _unit(s):
    P = [int(p) for p, ps in zip(s.P_type, s.pseudo_type) if not ps]
    return 1.0 / max(P)


@pytest.mark.parametrize("case,precision", [("c1", 0), ("c1", 1), ("mixed", 0)])
def test_rdf_hist_bit_exact(gpu, case, precision):
    if case == "c1":
        s = synth.water_box(32, 9.865, 8, 2, seed=12)
        pairs = [(0, 0), (0, 1), (1, 0), (1, 1)]
    else:
        s = synth.water_box(8, 8.4, 8, 2, seed=3, ion=dict(synth.systems.ION3), electron_P=16)
        pairs = [(2, 0), (0, 2), (2, 1), (0, 0)]
    s.q = s.q + np.random.default_rng(13).normal(0, 0.1, s.q.shape)
    m = gpu.MixTS(s, precision=precision)
    m.forces(energy=False)
    for ta, tb in pairs:
        g = _gpu_hist(m, ta, tb, 0.02, 400) * _unit(s)
        o = oracle.rdf_hist(s, ta, tb, dr=0.02, nbins=400)
        assert np.array_equal(g, o), (ta, tb)
    m.close()


def test_rdf_needs_a_force_evaluation_and_valid_bins(gpu):
    import torch
    s = synth.water_box(32, 9.865, 8, 2, seed=12)
    m = gpu.MixTS(s)
    h = torch.zeros(400, dtype=torch.int64, device=m.device)
    with pytest.raises(gpu.MixtsError):
        m.rdf_accumulate(0, 0, h)  # no list yet
    m.forces(energy=False)
    big = torch.zeros(1000, dtype=torch.int64, device=m.device)
    with pytest.raises(gpu.MixtsError):
        m.rdf_accumulate(0, 0, big, 0.02)  # 20 A > r_cut
    m.close()


def _blocks(x, nb):
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nb * nb
    b = x[:n].reshape(nb, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nb)


def test_long_run_statistics_match_oracle(gpu):
    import torch
    s = synth.water_box(32, 9.865, 8, 2, seed=0)
    dr, nb, NB = 0.05, 160, 8
    every, n_eq, n_samp = 10, 400, 2400
    per_block = n_samp // every // NB
    keys = [(0, 0), (0, 1)]
    windows = {(0, 0): (2.5, 3.3), (0, 1): (1.5, 2.3)}  # first O-O and O-H intermolecular peaks
    N = s.n_of_type()

    def window(g, k):
        lo, hi = windows[k]
        return g[int(lo / dr):int(hi / dr)].mean()

    # GPU run
    m = gpu.MixTS(s, seed=101)
    m.step(n_eq)
    g_ke, g_T, g_w = {0: [], 1: []}, [], {k: [] for k in keys}
    for blk in range(NB):
        hist = {k: torch.zeros(nb, dtype=torch.int64, device=m.device) for k in keys}
        for _ in range(per_block):
            m.step(every)
            e = m.estimators()
            g_ke[0].append(e["KE_cv"][0])
            g_ke[1].append(e["KE_cv"][1])
            g_T.append(e["T_beads"])
            for (a, b), h in hist.items():
                m.rdf_accumulate(a, b, h, dr)
        for k, h in hist.items():
            g_w[k].append(window(m.rdf_normalise(k[0], k[1], h, per_block, dr), k))
    m.close()
    # oracle run, same start, its own noise
    run = oracle.Runner(s, oracle.make_params(T=300.0, dt=0.25, tau=100.0, lam=1.0, seed=202))
    run.step(n_eq)
    o_ke, o_T, o_w = {0: [], 1: []}, [], {k: [] for k in keys}
    for blk in range(NB):
        oh = {k: np.zeros(nb) for k in keys}
        for _ in range(per_block):
            run.step(every)
            e = run.estimators()
            o_ke[0].append(e["KE_cv"][0])
            o_ke[1].append(e["KE_cv"][1])
            o_T.append(e["T_beads"])
            for (a, b) in keys:
                oh[(a, b)] += oracle.rdf_hist(s, a, b, dr=dr, nbins=nb, q=run.q)
        for k, h in oh.items():
            o_w[k].append(window(oracle.rdf_normalise(h, per_block, N[k[0]], N[k[1]], k[0] == k[1], s.box, dr), k))

    def close(x, y, what):
        mx, sx = _blocks(x, NB)
        my, sy = _blocks(y, NB)
        assert abs(mx - my) < 4 * np.hypot(sx, sy) + 1e-12, (what, mx, sx, my, sy)

    close(g_ke[0], o_ke[0], "KE_cv O")
    close(g_ke[1], o_ke[1], "KE_cv H")
    close(g_T, o_T, "T_beads")
    for k in keys:
        close(g_w[k], o_w[k], f"g{k} first-peak window")
