"""C ABI: the library loads, exports every symbol include/mixts.h declares,
and rejects bad systems on the host (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_2411_11988_gb300 import build
    build.build()
    import paper_2411_11988_gb300 as pkg
    return pkg


def test_exports_every_declared_symbol(P):
    hdr = open(os.path.join(ROOT, "include", "mixts.h")).read()
    declared = set(re.findall(r"MIXTS_API\s+[\w\s\*]+?\b(mixts_\w+)\s*\(", hdr))
    assert declared, "no declarations found"
    L = P.lib()
    for name in declared:
        assert hasattr(L, name), name
    assert declared == set(P.EXPORTED)


def _sys_struct(P, s, **over):
    st, keep = P.mixts.pack_system(s, 1, 1, 1)
    for k, v in over.items():
        setattr(st, k, v)
    return st, keep


def _params(P, **kw):
    d = dict(T=300.0, dt=0.25, tau_centroid=100.0, pile_lambda=1.0, r_cut=9.0, dsf_alpha=0.2,
             precision=0, nlist_cap=0)
    d.update(kw)
    return P.mixts._Params(**d)


def test_workspace_size_positive(P):
    s = synth.water_box(32, 9.865, 8, 2, seed=0)
    st, keep = _sys_struct(P, s)
    prm = _params(P)
    n = P.lib().mixts_workspace_size(C.byref(st), 1, C.byref(prm))
    assert n > 0


def test_batch_workspace_is_sum_of_members(P):
    prm = _params(P)
    systems = [synth.water_box(32, 9.865, 8, 2, seed=0), synth.water_box(8, 6.21, 4, 1, seed=1),
               synth.water_box(27, 9.3, 16, 4, seed=2)]
    packed = [_sys_struct(P, s) for s in systems]
    arr = (P.mixts._System * 3)(*[x[0] for x in packed])
    singles = [P.lib().mixts_workspace_size(C.byref(x[0]), 1, C.byref(prm)) for x in packed]
    total = P.lib().mixts_workspace_size(arr, 3, C.byref(prm))
    members = sum((n + 255) // 256 * 256 for n in singles) + 256
    # plus the batch's own region (member records and launch prefixes), 256-aligned and small
    assert total >= members and (total - members) % 256 == 0 and total - members < 64 * 1024
    # a batch with one invalid member is rejected as a whole
    bad = synth.water_box(8, 6.21, 4, 3, seed=3)
    bad.P_type = np.array([3, 4], dtype=np.int32)
    bad_st, bad_keep = _sys_struct(P, bad)
    arr2 = (P.mixts._System * 2)(packed[0][0], bad_st)
    assert P.lib().mixts_workspace_size(arr2, 2, C.byref(prm)) == 0
    assert P.lib().mixts_workspace_size(arr, 0, C.byref(prm)) == 0


@pytest.mark.parametrize("bad", [(3, 2), (8, 0), (2048, 2)])
def test_bad_bead_counts_rejected(P, bad):
    s = synth.water_box(8, 8.4, bad[1] if bad[1] else 1, bad[0], seed=0)
    s.P_type = np.array([bad[0], bad[1]], dtype=np.int32)
    st, keep = _sys_struct(P, s)
    prm = _params(P)
    assert P.lib().mixts_workspace_size(C.byref(st), 1, C.byref(prm)) == 0
    h = C.c_void_p()
    rc = P.lib().mixts_init(C.byref(st), 1, C.byref(prm), None, 0, None, C.byref(h))
    assert rc == 2 and not h.value


def test_pseudo_coarser_than_site_rejected(P):
    s = synth.water_box(8, 8.4, 8, 2, seed=0, electron_P=4)
    st, keep = _sys_struct(P, s)
    h = C.c_void_p()
    rc = P.lib().mixts_init(C.byref(st), 1, C.byref(_params(P)), None, 0, None, C.byref(h))
    assert rc == 2


def test_bad_arguments_rejected(P):
    s = synth.water_box(8, 8.4, 8, 2, seed=0)
    st, keep = _sys_struct(P, s)
    h = C.c_void_p()
    L = P.lib()
    assert L.mixts_init(C.byref(st), 1, C.byref(_params(P, dt=0.0)), None, 0, None, C.byref(h)) == 1
    st2, keep2 = _sys_struct(P, s, box=-1.0)
    assert L.mixts_init(C.byref(st2), 1, C.byref(_params(P)), None, 0, None, C.byref(h)) == 1
    # a valid system with no workspace
    assert L.mixts_init(C.byref(st), 1, C.byref(_params(P)), None, 0, None, C.byref(h)) == 4


def test_binding_refuses_without_gpu(P):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    s = synth.water_box(8, 8.4, 8, 2, seed=0)
    with pytest.raises(RuntimeError):
        P.MixTS(s)
