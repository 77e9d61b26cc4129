"""Long-range electrostatics on ring-polymer centroids (coulomb = 1) on the
GPU against the oracle (Sec. "Theory", last paragraph: SPME with the
bead-bead electrostatics approximated by centroid-centroid ones; here a
direct Ewald sum, real space per bead pair).

Tolerances as in the other parity tests: FP64 forces and energies 1e-11 of
RMS force / |V|, one step 1e-11; FP32 pair forces 1e-5.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
ALPHA, KMAX = 0.35, 8


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_11988_gb300 as P
    return P


def _case(name):
    if name == "ion_water_h8o2":
        s = synth.water_box(27, 9.3, 8, 2, seed=2, ion=dict(synth.systems.ION3))
    elif name == "water_h1o4":
        s = synth.water_box(27, 9.3, 1, 4, seed=4)
    elif name == "c1":
        s = synth.water_box(32, 9.865, 8, 2, seed=0)
    elif name == "electron":
        s = synth.water_box(8, 8.4, 8, 2, seed=3, ion=dict(synth.systems.ION3), electron_P=64)
    else:
        raise KeyError(name)
    s.q = s.q + np.random.default_rng(11).normal(0, 0.05, s.q.shape)
    s.coulomb, s.ewald_kmax = 1, KMAX
    return s


def _err(F, F_or):
    return np.abs(F - F_or).max() / np.sqrt(np.mean(F_or ** 2))


@pytest.mark.parametrize("name", ["ion_water_h8o2", "water_h1o4", "c1", "electron"])
def test_ewald_forces_match_oracle(gpu, name):
    s = _case(name)
    m = gpu.MixTS(s, alpha=ALPHA, coulomb=1, ewald_kmax=KMAX)
    f, V = m.forces()
    F_or, parts = oracle.forces(s, alpha=ALPHA)
    assert _err(f.cpu().numpy(), F_or) < 1e-11
    assert abs(V - parts[0]) <= 1e-11 * abs(parts[0])
    e = m.estimators()
    assert abs(e["V_coul"] - parts[2]) <= 1e-11 * abs(parts[0])
    assert abs(e["virial"] - parts[6]) <= 1e-10 * max(abs(parts[6]), 1.0)
    m.close()


def test_ewald_one_step_matches_oracle(gpu):
    s = _case("ion_water_h8o2")
    m = gpu.MixTS(s, dt=0.25, alpha=ALPHA, coulomb=1, ewald_kmax=KMAX, seed=3)
    m.step(1)
    run = oracle.Runner(s, oracle.make_params(T=300.0, dt=0.25, tau=100.0, lam=1.0, seed=3), alpha=ALPHA)
    run.step(1)
    q, p, f = (x.cpu().numpy() for x in (m.q, m.p, m.f))
    assert np.abs(q - run.q).max() < 1e-11 * np.abs(run.q).max()
    assert np.abs(p - run.p).max() < 1e-10 * np.sqrt(np.mean(run.p ** 2))
    assert _err(f, run.F) < 1e-10
    m.close()


def test_ewald_fp32_forces(gpu):
    s = _case("ion_water_h8o2")
    m = gpu.MixTS(s, alpha=ALPHA, coulomb=1, ewald_kmax=KMAX, precision=gpu.FP32_FORCES)
    f, V = m.forces()
    F_or, parts = oracle.forces(s, alpha=ALPHA)
    assert _err(f.cpu().numpy(), F_or) < 1e-5
    assert abs(V - parts[0]) <= 1e-5 * abs(parts[0])
    m.close()


def test_ewald_rejects_bad_arguments(gpu):
    s = _case("c1")
    with pytest.raises(gpu.MixtsError):
        gpu.MixTS(s, alpha=ALPHA, coulomb=1, ewald_kmax=0)
    m = gpu.MixTS(s, alpha=ALPHA, coulomb=1, ewald_kmax=KMAX)
    with pytest.raises(gpu.MixtsError):
        m.potential_grad(0, 1, oracle.theta_of(s, 0, 1))
    m.close()
