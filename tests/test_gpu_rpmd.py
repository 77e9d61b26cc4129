"""Fictitious bead masses, the velocity-Verlet free ring and ring-polymer
molecular dynamics correlation functions on the GPU, against the oracle.

* One step and twenty steps with bead masses m_f != m (RPMD masses m/P_t, and
  a heavier H) and with the free ring evolved by velocity Verlet on the
  springs (Sec. "Evaluation"), within the FP64 tolerances of the other parity
  tests.
* The centroid velocity autocorrelation accumulated on the device over every
  origin of an NVE trajectory equals the oracle's accumulation over its own
  NVE trajectory from the same start (Sec. "Output and Analysis").
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


def _with_bead_masses(s, bm):
    """Set bead masses and redraw nothing: rescale the Maxwell-Boltzmann bead
    momenta (drawn with the physical masses) to N(0, m_f k_B T)."""
    s.bead_mass_type = np.asarray(bm, dtype=np.float64)
    off = s.type_offsets()
    for t in range(s.n_types):
        s.p[off[t]:off[t + 1]] *= np.sqrt(s.bead_mass_type[t] / s.mass_type[t])
    return s


def _case(name):
    if name in ("c1_rpmd", "c1_vv4"):
        s = synth.water_box(32, 9.865, 8, 2, seed=4)
        if name == "c1_rpmd":
            _with_bead_masses(s, oracle.rpmd_bead_masses(s))
        return s, (0 if name == "c1_rpmd" else 4)
    if name == "mixed_heavyH_vv2":
        s = synth.water_box(8, 8.4, 8, 2, seed=3, ion=dict(synth.systems.ION3), electron_P=64)
        s.q = s.q + np.random.default_rng(103).normal(0, 0.05, s.q.shape)
        bm = np.array(s.mass_type, dtype=np.float64)
        bm[1] *= 2.0
        _with_bead_masses(s, bm)
        return s, 2
    if name == "electron1024_rpmd":
        s = synth.water_box(64, 12.43, 4, 1, seed=5, ion=dict(synth.systems.ION3), electron_P=1024)
        _with_bead_masses(s, oracle.rpmd_bead_masses(s))
        return s, 0
    raise KeyError(name)


@pytest.mark.parametrize("name", ["c1_rpmd", "c1_vv4", "mixed_heavyH_vv2", "electron1024_rpmd"])
def test_bead_mass_and_verlet_steps_match_oracle(gpu, name):
    s, vv = _case(name)
    dt = 0.1 if "electron" in name or "mixed" in name else 0.25
    m = gpu.MixTS(s, dt=dt, tau=100.0, pile_lambda=1.0, seed=21, free_ring_substeps=vv)
    run = oracle.Runner(s, oracle.make_params(T=300.0, dt=dt, tau=100.0, lam=1.0, seed=21, vv=vv))
    for n in (1, 19):
        m.step(n)
        run.step(n)
        q, p, f = (x.cpu().numpy() for x in (m.q, m.p, m.f))
        tol = 1e-11 if n == 1 else 1e-8
        assert np.abs(q - run.q).max() < tol * np.abs(run.q).max(), n
        assert np.abs(p - run.p).max() < 10 * tol * np.sqrt(np.mean(run.p ** 2)), n
        rms = np.sqrt(np.mean(run.F ** 2))
        assert np.abs(f - run.F).max() < 10 * tol * rms, n
        e, eo = m.estimators(), run.estimators()
        for k in ["KE_beads", "E_spring", "H_mix", "heat", "T_beads"]:
            assert abs(e[k] - eo[k]) <= 10 * tol * max(abs(eo[k]), 1.0), (k, n, e[k], eo[k])
        for t in range(len(s.P_type)):
            assert abs(e["KE_cv"][t] - eo["KE_cv"][t]) <= 100 * tol * max(abs(eo["KE_cv"][t]), 1.0)
    m.close()


def test_rpmd_vacf_matches_oracle(gpu):
    from paper_2411_11988_gb300 import analysis
    s = _with_bead_masses(synth.water_box(32, 9.865, 8, 2, seed=6), analysis.rpmd_bead_masses(synth.water_box(32, 9.865, 8, 2, seed=6)))
    m = gpu.MixTS(s, dt=0.25, tau=0.0, pile_lambda=0.0, seed=0)
    run = oracle.Runner(s, oracle.make_params(T=300.0, dt=0.25, tau=0.0, lam=0.0, seed=0))
    n_lag, frames = 10, 40
    N = s.n_of_type()
    gv = [analysis.CentroidVACF(m, t, n_lag, int(N[t])) for t in (0, 1)]
    ov = [oracle.VelocityCorrelation(n_lag) for _ in (0, 1)]
    for _ in range(frames):
        m.step(1)
        run.step(1)
        for t in (0, 1):
            gv[t].add()
            ov[t].add(oracle.centroid_velocities(s, run.p, t))
    for t in (0, 1):
        acc = gv[t].acc.cpu().numpy()
        cnt = gv[t].cnt.cpu().numpy()
        assert np.array_equal(cnt, ov[t].cnt)
        assert np.allclose(acc, ov[t].acc, rtol=1e-8, atol=0), (acc, ov[t].acc)
        c, _ = gv[t].result()
        assert c[0] > 0
    # the lag-0 value is the mean squared centroid velocity, ~3 kT / m per atom
    m.close()


def test_vacf_needs_a_step(gpu):
    from paper_2411_11988_gb300 import analysis
    s = synth.water_box(8, 8.4, 4, 1, seed=1)
    m = gpu.MixTS(s)
    v = analysis.CentroidVACF(m, 0, 4, int(s.n_of_type()[0]))
    with pytest.raises(gpu.MixtsError) as ei:
        v.add()
    assert ei.value.status == 8
    m.close()
