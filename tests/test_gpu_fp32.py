"""FP32-forces precision mode against the FP64 oracle (GPU only).

Tolerances (FP32 pair forces, FP64 integration and reductions): forces
max|F_gpu - F_or| / RMS(F_or) <= 1e-5, energies |V_gpu - V_or| / |V_or| <= 1e-5.
The full neighbour list of this mode equals the oracle's canonical list plus
every entry seen from the other atom, bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth
from list_util import both_ways

pytestmark = pytest.mark.gpu
FTOL32 = 1e-5


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
    if name == "c1":
        return synth.water_box(32, 9.865, 8, 2, seed=0)
    if name == "c1_spread":
        s = synth.water_box(32, 9.865, 8, 2, seed=2)
        s.q = s.q + np.random.default_rng(9).normal(0, 0.1, s.q.shape)
        return s
    if name == "mixed":
        s = synth.water_box(8, 8.4, 8, 2, seed=3, ion=dict(synth.systems.ION3), electron_P=128)
        s.q = s.q + np.random.default_rng(103).normal(0, 0.08, s.q.shape)
        return s
    if name in ("h1_o4", "h4_o8"):  # H coarser than O: O owns the O-H terms
        ph, po = (1, 4) if name == "h1_o4" else (4, 8)
        s = synth.water_box(27, 9.3, ph, po, seed=12)
        s.q = s.q + np.random.default_rng(17).normal(0, 0.06, s.q.shape)
        return s
    if name == "c2":
        return synth.water_box(512, 24.83, 32, 4, seed=0)
    if name == "c3":
        return synth.water_box(256, 18.6, 8, 1, seed=0, ion=dict(synth.systems.ION3), electron_P=1024)
    # 768 atoms and more take the window sweep: O-O terms on a grid coarser
    # than the windows (H32/O1), and H coarser than O (H4/O32)
    if name in ("w256_h32_o1", "w256_h4_o32"):
        ph, po = (32, 1) if name == "w256_h32_o1" else (4, 32)
        s = synth.water_box(256, 19.7, ph, po, seed=21)
        s.q = s.q + np.random.default_rng(23).normal(0, 0.05, s.q.shape)
        return s
    raise KeyError(name)


@pytest.mark.parametrize("name", ["c1", "c1_spread", "mixed", "h1_o4", "h4_o8", "c2", "c3", "w256_h32_o1",
                                  "w256_h4_o32"])
def test_fp32_forces(gpu, name):
    s = _case(name)
    m = gpu.MixTS(s, precision=gpu.FP32_FORCES)
    f, V = m.forces()
    F = f.cpu().numpy()
    F_or, parts = oracle.forces(s)
    rms = np.sqrt(np.mean(F_or ** 2))
    err = np.abs(F - F_or).max() / rms
    assert err < FTOL32, err
    assert abs(V - parts[0]) <= FTOL32 * abs(parts[0])
    est = m.estimators()
    assert abs(est["n_evals"] - parts[7]) <= 1e-5 * parts[7] + 2
    m.close()


def test_fp32_full_list_bit_exact(gpu):
    s = _case("c1_spread")
    m = gpu.MixTS(s, precision=gpu.FP32_FORCES)
    m.forces()
    tl, th = m.nlist(0)
    ol, dmax, R = oracle.nlist(s)
    assert th[0] == dmax and th[1] == R
    full = both_ways(ol)
    assert np.array_equal(tl, full)
    m.close()


def test_fp32_cell_list_search(gpu):
    """The FP32 path's full lists through the cell search (r_cut 6 A in the
    24.83 A box: 3 cells per side) equal both orientations of the oracle's
    canonical list, and the forces agree at 1e-5."""
    rc = 6.0
    s = synth.water_box(512, 24.83, 2, 1, seed=21)
    m = gpu.MixTS(s, precision=gpu.FP32_FORCES, r_cut=rc)
    m.forces()
    tl, th = m.nlist(0)
    ol, dmax, R = oracle.nlist(s, r_cut=rc)
    assert th[0] == dmax and th[1] == R
    assert np.array_equal(tl, both_ways(ol))
    F_or = oracle.forces(s, r_cut=rc)[0]
    f = m.f.cpu().numpy()
    assert np.abs(f - F_or).max() / np.sqrt(np.mean(F_or ** 2)) < 1e-5
    m.close()


def test_fp32_step_tracks_fp64(gpu):
    s = _case("c1")
    a = gpu.MixTS(s, precision=gpu.FP32_FORCES, seed=4)
    b = gpu.MixTS(s, precision=gpu.FP64, seed=4)
    a.step(10)
    b.step(10)
    qa, qb = a.q.cpu().numpy(), b.q.cpu().numpy()
    assert np.abs(qa - qb).max() < 1e-6
    ea, eb = a.estimators(), b.estimators()
    for k in ["V", "KE_beads", "E_spring", "H_mix"]:
        assert abs(ea[k] - eb[k]) <= 1e-5 * max(abs(eb[k]), 1.0), k
    a.close()
    b.close()
