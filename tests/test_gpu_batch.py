"""Batched variant on the GPU: uneven systems behind one handle, stepped by
captured graph launches with autotuned shapes.

Each member must give exactly (bit for bit) what the same system gives
alone, and match the oracle within the single-system tolerances (FP64 1e-11,
FP32 1e-5 of RMS force). FP32 members take the gather sweep; a standalone
handle of 768 atoms or more takes the window sweep, whose sums group the
terms differently, so the bitwise comparisons use smaller systems.
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


def _systems():
    out = []
    for k, (n, ph) in enumerate([(8, 4), (16, 8), (27, 2), (8, 16)]):
        s = synth.water_box(n, synth.density_box_length(n), ph, max(1, ph // 4), seed=40 + k)
        out.append(s)
    return out


def _force_err(F, F_or):
    return np.abs(F - F_or).max() / np.sqrt(np.mean(F_or ** 2))


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 1e-5)])
def test_batch_forces_match_single_and_oracle(gpu, precision, tol):
    systems = _systems()
    b = gpu.MixTSBatch(systems, precision=precision)
    E = b.forces()
    for i, s in enumerate(systems):
        m = gpu.MixTS(s, precision=precision, seed=i)
        f1, e1 = m.forces()
        assert np.array_equal(b.f[i].cpu().numpy(), f1.cpu().numpy())
        assert E[i] == e1
        F_or, parts = oracle.forces(s)
        assert _force_err(b.f[i].cpu().numpy(), F_or) < tol
        assert abs(E[i] - parts[0]) <= tol * abs(parts[0])
        m.close()
    b.close()


def test_batch_graph_steps_equal_single_runs(gpu):
    systems = _systems()
    b = gpu.MixTSBatch(systems)
    _, _, k0 = b.timing()
    b.step(25)  # two graph launches of 10 steps, then 5 eager steps
    _, _, k1 = b.timing()
    assert k1 > k0
    est = b.estimators()
    for i, s in enumerate(systems):
        m = gpu.MixTS(s, seed=i)
        m.step(25)
        assert np.array_equal(b.q[i].cpu().numpy(), m.q.cpu().numpy())
        assert np.array_equal(b.p[i].cpu().numpy(), m.p.cpu().numpy())
        e1 = m.estimators()
        assert est[i]["step"] == e1["step"] == 25
        assert est[i]["H_conserved"] == e1["H_conserved"]
        m.close()
    b.close()


def test_batch_tune_leaves_trajectory_unchanged(gpu):
    systems = _systems()
    a = gpu.MixTSBatch(systems)
    a.step(3)
    t = a.tune(steps_per_launch=5)
    assert t["candidates"] >= 5 and t["ms_per_step"] > 0
    assert t["streams"] >= 1 and t["nl_cpl"] in (2, 4, 8) and t["steps_per_launch"] == 5
    a.step(12)
    b = gpu.MixTSBatch(systems)
    b.step(15)
    for i in range(len(systems)):
        assert np.array_equal(a.q[i].cpu().numpy(), b.q[i].cpu().numpy())
        assert np.array_equal(a.p[i].cpu().numpy(), b.p[i].cpu().numpy())
    assert [e["step"] for e in a.estimators()] == [15] * len(systems)
    a.close()
    b.close()


def test_batch_checkpoint_roundtrip(gpu):
    systems = _systems()
    b = gpu.MixTSBatch(systems)
    b.step(4)
    blob = b.get_state()
    b.step(11)
    q1 = [x.cpu().numpy().copy() for x in b.q]
    b.set_state(blob)
    b.step(11)
    for i in range(len(systems)):
        assert np.array_equal(b.q[i].cpu().numpy(), q1[i])
    b.close()


def test_batch_member_queries(gpu):
    systems = _systems()
    b = gpu.MixTSBatch(systems)
    b.forces()
    m = b.member(2)
    trip, _ = m.nlist()
    single = gpu.MixTS(systems[2], seed=2)
    single.forces()
    trip1, _ = single.nlist()
    assert np.array_equal(trip, trip1)
    # the batched handle itself rejects per-system queries
    view = gpu.MixTS.__new__(gpu.MixTS)
    view.h, view._borrowed, view.n_types = b.h, True, 2
    with pytest.raises(gpu.MixtsError):
        view.nlist()
    single.close()
    b.close()


# members of the 64-system batch workload (water count, P_H, P_O, seed index):
# the largest (512 waters at P_H = 64), the smallest box at P_H = 64, and
# classical-oxygen members at both ends of the size range
C4_MEMBERS = [2, 11, 3, 19, 0, 15]


def test_batch_workload_members_match_oracle(gpu):
    draws = synth.batched_draws(64, 1000)
    systems = [synth.water_box(draws[i][0], synth.density_box_length(draws[i][0]), draws[i][1], draws[i][2], seed=i)
               for i in C4_MEMBERS]
    assert (draws[2][0], draws[2][1]) == (512, 64)
    b = gpu.MixTSBatch(systems, precision=1, seeds=C4_MEMBERS)
    E = b.forces()
    for k, s in enumerate(systems):
        F_or, parts = oracle.forces(s)
        assert _force_err(b.f[k].cpu().numpy(), F_or) < 1e-5, C4_MEMBERS[k]
        assert abs(E[k] - parts[0]) <= 1e-5 * abs(parts[0])
    b.close()


def test_batch_one_launch_per_phase(gpu):
    """Water systems of uneven sizes and bead counts: a batched step launches
    each kernel once for all members (<= 10 kernels per step), and every member
    still matches its own single-system run bit for bit (FP64 and FP32)."""
    systems = _systems()
    for precision in (0, 1):
        b = gpu.MixTSBatch(systems, precision=precision)
        b.step(3)  # below steps_per_launch: plain per-member launches
        _, _, k0 = b.timing()
        b.step(10)  # one graph launch
        _, _, k1 = b.timing()
        assert (k1 - k0) / 10.0 <= 10.0, k1 - k0
        for i, s in enumerate(systems):
            m = gpu.MixTS(s, seed=i, precision=precision)
            m.step(13)
            assert np.array_equal(b.q[i].cpu().numpy(), m.q.cpu().numpy())
            assert np.array_equal(b.p[i].cpu().numpy(), m.p.cpu().numpy())
            m.close()
        b.close()


def test_batch_with_electron_member_falls_back(gpu):
    """A member with a pseudo particle keeps the per-member kernels on
    parallel graph branches; the trajectory is still the single-system one."""
    systems = _systems()[:2] + [synth.water_box(8, 8.4, 8, 2, seed=3, ion=dict(synth.systems.ION3), electron_P=64)]
    b = gpu.MixTSBatch(systems, dt=0.1)
    b.step(12)
    for i, s in enumerate(systems):
        m = gpu.MixTS(s, seed=i, dt=0.1)
        m.step(12)
        assert np.array_equal(b.q[i].cpu().numpy(), m.q.cpu().numpy())
        m.close()
    b.close()
