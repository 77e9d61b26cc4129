"""The allocation-free force entry point against the regular one (GPU only).

mixts_forces_noalloc is for callers that cannot allocate device memory (a
host framework that owns every device byte through its own pool, drivers
that forbid device allocation after start-up): it keeps all scratch in one
static device array. This file is collected last on purpose, so a run that
stops at the first failure has already run every other test; it also passes
on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

FTOL = 1e-11  # the FP64 force tolerance of the other parity tests


@pytest.fixture(scope="module")
def P():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2411_11988_gb300 as pkg
    return pkg


def _noalloc_forces(P, sysm, q, energy=True, with_p=True, nlist_cap=0, expect=0):
    import torch
    L = P.lib()
    qd = torch.from_numpy(np.ascontiguousarray(q)).cuda()
    pd = torch.zeros_like(qd)
    fd = torch.full_like(qd, float("nan"))
    st, keep = P.mixts.pack_system(sysm, qd.data_ptr(), pd.data_ptr() if with_p else 0, fd.data_ptr(), 0)
    prm = P.mixts._Params(300.0, 0.25, 100.0, 1.0, 9.0, 0.2, 0, nlist_cap)
    e = C.c_double(0.0)
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.mixts_forces_noalloc(C.byref(st), C.byref(prm), C.c_void_p(stream), C.byref(e) if energy else None)
    assert rc == expect, P.mixts.STATUS.get(rc, rc)
    return fd.cpu().numpy(), (e.value if energy else None)


@pytest.mark.parametrize("case", ["water32_H8_O2", "ion_electron"])
def test_noalloc_matches_regular_twice(P, case):
    if case == "water32_H8_O2":
        s = synth.water_box(32, 9.865, 8, 2, seed=0)
    else:
        s = synth.water_box(8, 8.4, 8, 2, seed=3, ion=dict(synth.systems.ION3), electron_P=128)
    rng = np.random.default_rng(11)
    qs = [s.q, s.q + rng.normal(0, 0.05, s.q.shape)]
    for q in qs:  # two calls in a row share (and must fully reset) the static scratch
        m = P.MixTS(s, q=q)
        f_ref, v_ref = m.forces()
        f_ref = f_ref.cpu().numpy()
        m.close()
        f, v = _noalloc_forces(P, s, q)
        rms = np.sqrt(np.mean(f_ref ** 2))
        assert np.abs(f - f_ref).max() / rms <= FTOL
        assert abs(v - v_ref) <= FTOL * abs(v_ref)


def test_noalloc_rejects_oversized(P):
    s = synth.water_box(4096, 49.66, 32, 32, seed=0)
    f, _ = None, None
    L = P.lib()
    st, keep = P.mixts.pack_system(s, 1, 1, 1, 0)
    prm = P.mixts._Params(300.0, 0.25, 100.0, 1.0, 9.0, 0.2, 0, 0)
    assert L.mixts_workspace_size(C.byref(st), 1, C.byref(prm)) > (32 << 20)
    rc = L.mixts_forces_noalloc(C.byref(st), C.byref(prm), None, None)
    assert rc == 4


def test_noalloc_without_energy_or_momenta(P):
    """No energy pointer: the call still waits for its work and checks the
    device error word; no momentum array: p = NULL is accepted."""
    s = synth.water_box(32, 9.865, 8, 2, seed=1)
    m = P.MixTS(s)
    f_ref, _ = m.forces()
    f_ref = f_ref.cpu().numpy()
    m.close()
    rms = np.sqrt(np.mean(f_ref ** 2))
    for energy, with_p in [(False, True), (True, False), (False, False)]:
        f, _ = _noalloc_forces(P, s, s.q, energy=energy, with_p=with_p)
        assert np.abs(f - f_ref).max() / rms <= FTOL


def test_noalloc_reports_list_overflow(P):
    """A neighbour-list capacity far below what the system needs is reported
    as MIXTS_ERR_NLIST_OVERFLOW on both the energy and the no-energy path, and
    the next regular call succeeds (the scratch is fully reset)."""
    s = synth.water_box(32, 9.865, 8, 2, seed=0)
    for energy in (True, False):
        _noalloc_forces(P, s, s.q, energy=energy, nlist_cap=32, expect=5)
    f, v = _noalloc_forces(P, s, s.q)
    assert np.isfinite(f).all() and np.isfinite(v)
