"""CUDA path vs the FP64 oracle, through the C ABI (GPU only).

Tolerances (FP64 path): forces max|F_gpu - F_or| / RMS(F_or) <= 1e-11,
energies |V_gpu - V_or| / |V_or| <= 1e-11; neighbour lists and the
thermostat's normals bit for bit; one full step within 1e-11 of RMS.
"""
import numpy as np
import pytest

import oracle
import synth
from list_util import canonical

pytestmark = pytest.mark.gpu

FTOL = 1e-11


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_11988_gb300 as P
    return P


def _c1(seed=0, spread=0.0):
    s = synth.water_box(32, 9.865, 8, 2, seed=seed)
    if spread:
        rng = np.random.default_rng(seed + 7)
        s.q = s.q + rng.normal(0, spread, s.q.shape)
    return s


def _mixed(P_e=16, seed=3, box=8.4, n=8, spread=0.08):
    s = synth.water_box(n, box, 8, 2, seed=seed, ion=dict(synth.systems.ION3), electron_P=P_e)
    rng = np.random.default_rng(seed + 100)
    s.q = s.q + rng.normal(0, spread, s.q.shape)
    return s


def _force_err(F, F_or):
    rms = np.sqrt(np.mean(F_or ** 2))
    return np.abs(F - F_or).max() / rms


def _h_coarser(P_H, P_O, seed=12):
    """Water with the lighter species on the coarser grid: O owns every O-H
    term (Fig. 1's N1 = 4, N2 = 1 and N1 = 4, N2 = 2 maps, read with O as the
    finer particle)."""
    s = synth.water_box(27, 9.3, P_H, P_O, seed=seed)
    s.q = s.q + np.random.default_rng(seed + 5).normal(0, 0.06, s.q.shape)
    return s


@pytest.mark.parametrize("case", ["c1", "c1_spread", "mixed16", "mixed128", "uniform4", "h1_o4", "h4_o8", "h64_o16"])
def test_forces_match_oracle(gpu, case):
    if case == "c1":
        s = _c1()
    elif case == "c1_spread":
        s = _c1(seed=2, spread=0.1)
    elif case == "mixed16":
        s = _mixed(16)
    elif case == "mixed128":
        s = _mixed(128)
    elif case == "h1_o4":
        s = _h_coarser(1, 4)
    elif case == "h4_o8":
        s = _h_coarser(4, 8)
    elif case == "h64_o16":  # two slice blocks per H owner; energies summed from 2^-34 fixed-point lanes
        s = synth.water_box(64, 12.43, 64, 16, seed=15)
        s.q = s.q + np.random.default_rng(16).normal(0, 0.05, s.q.shape)
    else:
        s = synth.water_box(27, 9.3, 4, 4, seed=4)
    m = gpu.MixTS(s)
    f, V = m.forces()
    F = f.cpu().numpy()
    F_or, parts = oracle.forces(s)
    assert _force_err(F, F_or) < FTOL
    assert abs(V - parts[0]) <= FTOL * abs(parts[0])
    est = m.estimators()
    for k, i in [("V_lj", 1), ("V_coul", 2), ("V_bond", 3), ("V_angle", 4), ("V_pseudo", 5)]:
        assert abs(est[k] - parts[i]) <= FTOL * max(abs(parts[0]), 1.0), k
    assert est["n_evals"] == parts[7]
    assert est["n_pseudo_evals"] == parts[8]
    assert abs(est["virial"] - parts[6]) <= 1e-10 * max(abs(parts[6]), 1.0)
    m.close()


@pytest.mark.parametrize("case", ["c1_spread", "mixed16", "mixed128", "h1_o4"])
def test_neighbour_lists_bit_exact(gpu, case):
    if case == "h1_o4":
        s = _h_coarser(1, 4, seed=14)
    else:
        s = _c1(seed=5, spread=0.15) if case == "c1_spread" else _mixed(16 if case == "mixed16" else 128)
    m = gpu.MixTS(s)
    m.forces()
    tl, th = m.nlist(0)
    ol, dmax, R = oracle.nlist(s)
    assert th[0] == dmax and th[1] == R
    # the kernel's rows are owned by the finer atom of each pair
    Pt = s.P_type[s.type_of_atom]
    assert np.all(Pt[tl[:, 0]] >= Pt[tl[:, 1]])
    assert np.array_equal(canonical(tl), ol)
    if s.pseudo_type.any():
        pl, pth = m.nlist(1)
        opl, oth = oracle.pseudo_list(s)
        assert pth[0] == oth[1] and pth[1] == oth[2]
        assert np.array_equal(pl, opl)
    m.close()


@pytest.mark.parametrize("P_e", [128, 256, 512, 1024])
def test_step_path_spread_and_lists(gpu, P_e):
    """After a step, the lists built from the propagation kernel's bead
    spreads (the large-P types' maximum gathered over a thread-block
    cluster) equal the oracle's lists of the same positions, radii included."""
    import copy
    s = _mixed(P_e, seed=3)
    m = gpu.MixTS(s, T=300.0, dt=0.1, tau=100.0, seed=11)
    m.step(1)
    s2 = copy.deepcopy(s)
    s2.q = m.q.cpu().numpy().copy()
    tl, th = m.nlist(0)
    ol, dmax, R = oracle.nlist(s2)
    assert th[0] == dmax and th[1] == R
    assert np.array_equal(canonical(tl), ol)
    pl, pth = m.nlist(1)
    opl, oth = oracle.pseudo_list(s2)
    assert pth[0] == oth[1] and pth[1] == oth[2]
    assert np.array_equal(pl, opl)
    m.close()


@pytest.mark.parametrize("case", ["cells", "cells_fallback"])
def test_cell_list_search(gpu, case):
    """A box at least three list radii wide is searched through its 27
    neighbouring cells (r_cut = 6 A in the 24.83 A box: 3 cells of 8.28 A);
    a step whose list radius r_cut + 2 d_max exceeds the cell side (bead
    spreads above 1.14 A) searches all pairs instead. Either way the lists
    equal the oracle's bit for bit, the forces agree at 1e-11, and one step
    (lists rebuilt from the propagation kernel's spreads) matches."""
    rc = 6.0
    s = synth.water_box(512, 24.83, 2, 1, seed=21)
    if case == "cells_fallback":
        s.q = s.q + np.random.default_rng(22).normal(0, 0.45, s.q.shape)
    m = gpu.MixTS(s, r_cut=rc, T=300.0, dt=0.1, tau=100.0, seed=11)
    m.forces()
    tl, th = m.nlist(0)
    ol, dmax, R = oracle.nlist(s, r_cut=rc)
    assert th[0] == dmax and th[1] == R
    assert (R + 1e-3 <= 24.83 / 3) == (case == "cells")
    assert np.array_equal(canonical(tl), ol)
    F_or = oracle.forces(s, r_cut=rc)[0]
    assert _force_err(m.f.cpu().numpy(), F_or) < FTOL
    m.step(1)
    run = oracle.Runner(s, oracle.make_params(T=300.0, dt=0.1, tau=100.0, lam=1.0, seed=11), r_cut=rc)
    run.step(1)
    q = m.q.cpu().numpy()
    assert np.abs(q - run.q).max() < 1e-11 * np.abs(run.q).max()
    assert _force_err(m.f.cpu().numpy(), run.F) < 1e-10
    m.close()


def test_gaussians_bit_exact(gpu):
    s = _c1()
    m = gpu.MixTS(s, seed=987654321)
    for step, stage, dof0, n in [(0, 0, 0, 4096), (17, 1, 123457, 1001), (2 ** 31 + 5, 0, 2 ** 33 + 3, 513)]:
        g = m.gaussians(step, stage, dof0, n).cpu().numpy()
        o = oracle.gaussians(987654321, step, stage, dof0, n)
        assert np.array_equal(g.view(np.uint32), o.view(np.uint32))
    m.close()


def _run_both(s, nsteps, **kw):
    prm = dict(T=300.0, dt=0.25, tau=100.0, lam=1.0, seed=11)
    prm.update(kw)
    import paper_2411_11988_gb300 as P
    m = P.MixTS(s, T=prm["T"], dt=prm["dt"], tau=prm["tau"], pile_lambda=prm["lam"], seed=prm["seed"])
    m.step(nsteps)
    run = oracle.Runner(s, oracle.make_params(**prm))
    run.step(nsteps)
    return m, run


@pytest.mark.parametrize("case", ["c1", "mixed16", "mixed128", "mixed512", "h64", "h1_o4", "h4_o8", "electron1024",
                                  "h128_o256"])
def test_one_step_matches_oracle(gpu, case):
    if case == "c1":
        s = _c1(seed=1)
    elif case in ("h1_o4", "h4_o8"):
        s = _h_coarser(*((1, 4) if case == "h1_o4" else (4, 8)), seed=13)
    elif case == "h128_o256":
        # many atoms of two FFT-propagated types: 54 H at P = 128 in tiles of
        # ten atoms (even column counts), 27 O at P = 256 in tiles of five
        # (odd column counts, a half-filled last complex column)
        s = _h_coarser(128, 256, seed=17)
    elif case == "electron1024":  # 256 waters H8/O1 + ion + 1024-bead electron, the large-P transforms
        s = synth.water_box(256, 18.6, 8, 1, seed=2, ion=dict(synth.systems.ION3), electron_P=1024)
    elif case == "h64":  # the largest bead count of the fused small-P propagation tile
        s = synth.water_box(8, synth.density_box_length(8), 64, 16, seed=11)
    else:  # mixed512: the four-step split 16 x 32 over a 16-CTA cluster (one frequency row per CTA)
        s = _mixed({"mixed16": 16, "mixed128": 128, "mixed512": 512}[case], seed=9)
    m, run = _run_both(s, 1, dt=0.1 if case in ("mixed16", "mixed128", "mixed512", "electron1024") else 0.25)
    q, p, f = (x.cpu().numpy() for x in (m.q, m.p, m.f))
    assert np.abs(q - run.q).max() < 1e-11 * np.abs(run.q).max()
    assert np.abs(p - run.p).max() < FTOL * 10 * np.sqrt(np.mean(run.p ** 2))
    assert _force_err(f, run.F) < 1e-10
    e, eo = m.estimators(), run.estimators()
    for k in ["V", "KE_beads", "E_spring", "H_mix", "heat", "T_beads"]:
        assert abs(e[k] - eo[k]) <= 1e-10 * max(abs(eo[k]), 1.0), (k, e[k], eo[k])
    for t in range(len(s.P_type)):
        for k in ["KE_prim", "KE_cv", "Rg2", "E_spring_t"]:
            assert abs(e[k][t] - eo[k][t]) <= 1e-9 * max(abs(eo[k][t]), 1.0), (k, t)
    assert e["step"] == 1
    m.close()


def test_twenty_steps_track_oracle(gpu):
    s = _c1(seed=3)
    m, run = _run_both(s, 20)
    q = m.q.cpu().numpy()
    assert np.abs(q - run.q).max() < 1e-8
    e, eo = m.estimators(), run.estimators()
    assert abs(e["H_conserved"] - eo["H_conserved"]) < 1e-7 * abs(eo["H_conserved"])
    m.close()


def test_bitwise_reproducible_and_resumable(gpu):
    s = _c1(seed=6)
    import paper_2411_11988_gb300 as P
    a = P.MixTS(s, seed=5)
    a.step(30)
    qa, pa = a.q.cpu().numpy().copy(), a.p.cpu().numpy().copy()
    b = P.MixTS(s, seed=5)
    b.step(30)
    assert np.array_equal(qa, b.q.cpu().numpy()) and np.array_equal(pa, b.p.cpu().numpy())
    c = P.MixTS(s, seed=5)
    c.step(12)
    blob = c.get_state()
    c.close()
    d = P.MixTS(s, seed=5)
    d.set_state(blob)
    d.step(18)
    assert np.array_equal(qa, d.q.cpu().numpy()) and np.array_equal(pa, d.p.cpu().numpy())
    assert d.estimators()["step"] == 30
    for x in (a, b, d):
        x.close()


def test_c2_full_size_sampled(gpu):
    s = synth.water_box(512, 24.83, 32, 4, seed=0)
    m = gpu.MixTS(s)
    f, V = m.forces()
    F = f.cpu().numpy()
    F_or, parts = oracle.forces(s)
    assert _force_err(F, F_or) < FTOL
    assert abs(V - parts[0]) <= FTOL * abs(parts[0])
    est = m.estimators()
    assert est["n_evals"] == parts[7]
    m.close()


def test_c3_electron_full_size(gpu):
    s = synth.water_box(256, 18.6, 8, 1, seed=0, ion=dict(synth.systems.ION3), electron_P=1024)
    m = gpu.MixTS(s, dt=0.1)
    f, V = m.forces()
    F = f.cpu().numpy()
    F_or, parts = oracle.forces(s)
    assert _force_err(F, F_or) < FTOL
    assert abs(V - parts[0]) <= FTOL * abs(parts[0])
    m.close()


def test_nlist_overflow_reported(gpu):
    s = _c1()
    m = gpu.MixTS(s, nlist_cap=32)
    with pytest.raises(gpu.MixtsError) as ei:
        m.forces()
    assert ei.value.status == 5
    m.close()


@pytest.mark.parametrize("case", ["water", "electron"])
def test_side_stream_steps_equal_serial_order(gpu, case):
    """The default step runs the bonded terms, the pseudopotential sweep, the
    finalisation and the large-P clusters beside the other kernels on a side
    stream; the per-phase timing mode runs everything in order on one
    stream. Fixed-point accumulation makes the two bit-identical."""
    if case == "water":
        s = _c1(seed=9)
    else:
        s = synth.water_box(64, synth.density_box_length(64), 8, 2, seed=4, ion=dict(synth.systems.ION3),
                            electron_P=1024)
    a = gpu.MixTS(s, seed=5, dt=0.1)
    a.step(13)
    b = gpu.MixTS(s, seed=5, dt=0.1)
    b.set_timing(True)
    b.step(13)
    assert np.array_equal(a.q.cpu().numpy(), b.q.cpu().numpy())
    assert np.array_equal(a.p.cpu().numpy(), b.p.cpu().numpy())
    assert np.array_equal(a.f.cpu().numpy(), b.f.cpu().numpy())
    ea, eb = a.estimators(), b.estimators()
    for k in ("V", "KE_beads", "E_spring", "H_conserved", "heat", "virial"):
        assert ea[k] == eb[k], k
    a.close()
    b.close()


def test_graph_steps_equal_plain_launches(gpu):
    """mixts_step by captured-graph replays (10 steps per launch) and by plain
    launches give the same state bit for bit."""
    s = _c1(seed=8)
    a = gpu.MixTS(s, seed=3)
    a.step(27)  # two graph launches + 7 plain steps
    b = gpu.MixTS(s, seed=3)
    b.set_graph(0)
    b.step(27)
    c = gpu.MixTS(s, seed=3)
    c.set_graph(4)
    for n in (9, 1, 17):
        c.step(n)
    for x in (b, c):
        assert np.array_equal(a.q.cpu().numpy(), x.q.cpu().numpy())
        assert np.array_equal(a.p.cpu().numpy(), x.p.cpu().numpy())
        assert x.estimators()["H_conserved"] == a.estimators()["H_conserved"]
    # a graph replay counts the kernels it launches: same count as plain
    # launches in the same call structure (10 + 10 + 7 steps)
    d = gpu.MixTS(s, seed=3)
    d.set_graph(0)
    for n in (10, 10, 7):
        d.step(n)
    assert np.array_equal(a.q.cpu().numpy(), d.q.cpu().numpy())
    assert a.timing()[2] == d.timing()[2]
    for x in (a, b, c, d):
        x.close()


@pytest.mark.parametrize("shift", [(1.9, -0.7, 3.3), (-4.2, 2.6, -0.35), (9.5, 0.2, 0.0)])
@pytest.mark.parametrize("precision", [0, 1])
def test_molecules_across_box_faces(gpu, shift, precision):
    """A rigid translation leaves molecules across the box faces (each atom's
    bead 0 wrapped into the box on its own): forces, energy and the list stay
    those of the oracle, whose image sums work on the unwrapped coordinates."""
    s = _mixed(16, seed=21)
    s.q = s.q + np.asarray(shift)
    L = s.box
    w = np.array([np.floor(s.q[s.bead_rows(a)[0]] / L) for a in range(s.n_atoms)])
    assert any(len({tuple(w[a]) for a in np.where(s.mol_of_atom == m)[0]}) > 1 for m in set(s.mol_of_atom.tolist()))
    m = gpu.MixTS(s, precision=precision)
    f, V = m.forces()
    F_or, parts = oracle.forces(s)
    tol = FTOL if precision == 0 else 1e-5
    assert _force_err(f.cpu().numpy(), F_or) < tol
    assert abs(V - parts[0]) <= tol * abs(parts[0])
    tl, _ = m.nlist(0)
    ol, _, _ = oracle.nlist(s)
    if precision == 0:
        assert np.array_equal(canonical(tl), ol)
    m.close()
