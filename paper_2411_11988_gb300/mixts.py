"""ctypes binding of the C ABI in include/mixts.h (argument marshalling only).

Every step of the hot path runs in the CUDA library ``_build/libmixts.so``;
this module allocates the caller-owned device buffers with torch, packs the
system description into the C struct and forwards calls. There is no CPU
fallback: if the library or a GPU is missing, construction raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmixts.so")
MAX_TYPES = 16

STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_BEADS", 3: "ERR_CUDA", 4: "ERR_WORKSPACE",
          5: "ERR_NLIST_OVERFLOW", 6: "ERR_TIMEOUT", 7: "ERR_NONFINITE", 8: "ERR_STATE", 9: "ERR_BOX"}
FP64, FP32_FORCES = 0, 1

_lib = None


class MixtsError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"mixts {STATUS.get(status, status)}: {msg}")


class _System(C.Structure):
    _fields_ = [
        ("n_atoms", C.c_int), ("n_types", C.c_int),
        ("type_of_atom", C.POINTER(C.c_int)), ("mol_of_atom", C.POINTER(C.c_int)),
        ("P_type", C.POINTER(C.c_int)), ("mass_type", C.POINTER(C.c_double)),
        ("charge_type", C.POINTER(C.c_double)), ("lj_eps", C.POINTER(C.c_double)),
        ("lj_sig", C.POINTER(C.c_double)), ("pseudo_type", C.POINTER(C.c_int)),
        ("pp_sigma", C.POINTER(C.c_double)), ("pp_A_eV", C.POINTER(C.c_double)),
        ("pp_b", C.POINTER(C.c_double)),
        ("n_bonds", C.c_int), ("bonds", C.POINTER(C.c_int)),
        ("bond_k", C.POINTER(C.c_double)), ("bond_r0", C.POINTER(C.c_double)),
        ("n_angles", C.c_int), ("angles", C.POINTER(C.c_int)),
        ("angle_k", C.POINTER(C.c_double)), ("angle_theta0", C.POINTER(C.c_double)),
        ("box", C.c_double),
        ("q", C.c_void_p), ("p", C.c_void_p), ("f", C.c_void_p),
        ("seed", C.c_uint64), ("bead_mass_type", C.POINTER(C.c_double)),
    ]


class _Params(C.Structure):
    _fields_ = [("T", C.c_double), ("dt", C.c_double), ("tau_centroid", C.c_double),
                ("pile_lambda", C.c_double), ("r_cut", C.c_double), ("dsf_alpha", C.c_double),
                ("precision", C.c_int), ("nlist_cap", C.c_int), ("free_ring_substeps", C.c_int),
                ("coulomb", C.c_int), ("ewald_kmax", C.c_int)]


class _Tuning(C.Structure):
    _fields_ = [("grid_scale", C.c_double), ("streams", C.c_int), ("nl_cpl", C.c_int),
                ("steps_per_launch", C.c_int), ("ms_per_step", C.c_double), ("candidates", C.c_int),
                ("persistent", C.c_int), ("item_lg_terms", C.c_int)]


class _Estimates(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "V", "V_lj", "V_coul", "V_bond", "V_angle", "V_pseudo", "KE_beads", "E_spring", "virial",
        "T_beads", "H_mix", "heat", "H_conserved", "n_evals", "n_pseudo_evals", "n_lj_evals")] + [
        ("KE_prim", C.c_double * MAX_TYPES), ("KE_cv", C.c_double * MAX_TYPES),
        ("Rg2", C.c_double * MAX_TYPES), ("E_spring_t", C.c_double * MAX_TYPES),
        ("step", C.c_int64)]


def lib():
    """Load the CUDA library (build it first with ``build.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CUDA library not built: {LIB_PATH} (run paper_2411_11988_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        S, Pp = C.POINTER(_System), C.POINTER(_Params)
        L.mixts_workspace_size.argtypes = [S, C.c_int, Pp]
        L.mixts_workspace_size.restype = C.c_size_t
        L.mixts_init.argtypes = [S, C.c_int, Pp, C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]
        L.mixts_forces.argtypes = [C.c_void_p, C.POINTER(C.c_double)]
        L.mixts_step.argtypes = [C.c_void_p, C.c_int]
        L.mixts_estimators.argtypes = [C.c_void_p, C.POINTER(_Estimates)]
        L.mixts_nlist.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.c_long, C.POINTER(C.c_long),
                                  C.POINTER(C.c_double)]
        L.mixts_state_size.argtypes = [C.c_void_p]
        L.mixts_state_size.restype = C.c_size_t
        L.mixts_get_state.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
        L.mixts_set_state.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
        L.mixts_gaussians.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint64, C.c_long, C.c_void_p]
        L.mixts_reload.argtypes = [C.c_void_p]
        L.mixts_set_timing.argtypes = [C.c_void_p, C.c_int]
        L.mixts_get_timing.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                       C.POINTER(C.c_longlong)]
        L.mixts_forces_noalloc.argtypes = [S, Pp, C.c_void_p, C.POINTER(C.c_double)]
        L.mixts_set_graph.argtypes = [C.c_void_p, C.c_int]
        L.mixts_rdf_accumulate.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int, C.c_void_p]
        L.mixts_rdf_normalise.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int, C.c_longlong,
                                          C.POINTER(C.c_uint64), C.POINTER(C.c_double)]
        L.mixts_batch_member.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]
        L.mixts_batch_tune.argtypes = [C.c_void_p, C.c_int, C.POINTER(_Tuning)]
        L.mixts_potential_grad.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double), C.c_double,
                                           C.POINTER(C.c_double), C.c_void_p, C.POINTER(C.c_double)]
        L.mixts_vacf_accumulate.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.mixts_alu_probe.argtypes = [C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.mixts_destroy.argtypes = [C.c_void_p]
        L.mixts_last_error.argtypes = [C.c_void_p]
        L.mixts_last_error.restype = C.c_char_p
        L.mixts_version.restype = C.c_char_p
        _lib = L
    return _lib


EXPORTED = ["mixts_workspace_size", "mixts_init", "mixts_forces", "mixts_step", "mixts_estimators",
            "mixts_nlist", "mixts_state_size", "mixts_get_state", "mixts_set_state", "mixts_gaussians",
            "mixts_destroy", "mixts_last_error", "mixts_version", "mixts_reload", "mixts_set_timing",
            "mixts_get_timing", "mixts_forces_noalloc", "mixts_potential_grad", "mixts_batch_member",
            "mixts_batch_tune", "mixts_set_graph", "mixts_rdf_accumulate", "mixts_rdf_normalise",
            "mixts_alu_probe", "mixts_vacf_accumulate"]
# force-field parameters of the differentiation variant, in mixts_potential_grad's order
THETA_NAMES = ["sigma_a", "A_a_eV", "b_a", "sigma_b", "A_b_eV", "b_b", "q_a", "eps_aa"]
PHASES = ["nlist", "pair", "bonded", "pseudo", "prop", "final", "other"]


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def pack_system(sysm, q_ptr=0, p_ptr=0, f_ptr=0, seed=0):
    """Pack a system description (attributes as in the synthetic builders) into the C struct.

    Returns (struct, keepalive) -- keep ``keepalive`` until mixts_init returns.
    """
    f64 = lambda x: np.ascontiguousarray(x, dtype=np.float64)
    i32 = lambda x: np.ascontiguousarray(x, dtype=np.int32)
    k = dict(type_of_atom=i32(sysm.type_of_atom), mol_of_atom=i32(sysm.mol_of_atom), P_type=i32(sysm.P_type),
             mass_type=f64(sysm.mass_type), charge_type=f64(sysm.charge_type),
             lj_eps=f64(sysm.lj_eps).ravel(), lj_sig=f64(sysm.lj_sig).ravel(),
             pseudo_type=i32(sysm.pseudo_type), pp_sigma=f64(sysm.pp_sigma), pp_A_eV=f64(sysm.pp_A_eV),
             pp_b=f64(sysm.pp_b), bonds=i32(sysm.bonds).ravel(), bond_k=f64(sysm.bond_k),
             bond_r0=f64(sysm.bond_r0), angles=i32(sysm.angles).ravel(), angle_k=f64(sysm.angle_k),
             angle_theta0=f64(sysm.angle_theta0))
    bm = getattr(sysm, "bead_mass_type", None)
    if bm is not None:
        k["bead_mass_type"] = f64(bm)
    s = _System(len(k["type_of_atom"]), len(k["P_type"]),
                _ptr(k["type_of_atom"], C.c_int), _ptr(k["mol_of_atom"], C.c_int), _ptr(k["P_type"], C.c_int),
                _ptr(k["mass_type"], C.c_double), _ptr(k["charge_type"], C.c_double),
                _ptr(k["lj_eps"], C.c_double), _ptr(k["lj_sig"], C.c_double), _ptr(k["pseudo_type"], C.c_int),
                _ptr(k["pp_sigma"], C.c_double), _ptr(k["pp_A_eV"], C.c_double), _ptr(k["pp_b"], C.c_double),
                int(len(k["bond_k"])), _ptr(k["bonds"], C.c_int), _ptr(k["bond_k"], C.c_double),
                _ptr(k["bond_r0"], C.c_double), int(len(k["angle_k"])), _ptr(k["angles"], C.c_int),
                _ptr(k["angle_k"], C.c_double), _ptr(k["angle_theta0"], C.c_double),
                float(sysm.box), q_ptr, p_ptr, f_ptr, int(seed),
                _ptr(k["bead_mass_type"], C.c_double) if bm is not None else None)
    return s, k


class MixTS:
    """One system on one GPU, driven through the C ABI.

    ``q``, ``p``, ``f`` are float64 torch tensors [n_beads, 3] on the device in
    the library's bead layout; the workspace is a uint8 torch tensor.
    """

    def __init__(self, sysm, T=300.0, dt=0.25, tau=100.0, pile_lambda=1.0, r_cut=9.0, alpha=0.2,
                 precision=FP64, nlist_cap=0, seed=0, device="cuda:0", stream=None, q=None, p=None,
                 free_ring_substeps=0, coulomb=0, ewald_kmax=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("MixTS needs a CUDA device")
        L = lib()
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        q0 = np.asarray(sysm.q if q is None else q, dtype=np.float64)
        p0 = np.asarray(sysm.p if p is None else p, dtype=np.float64)
        self.n_beads = q0.shape[0]
        self.n_types = int(len(sysm.P_type))
        with torch.cuda.device(self.device):
            self.q = torch.from_numpy(q0.copy()).to(self.device)
            self.p = torch.from_numpy(p0.copy()).to(self.device)
            self.f = torch.zeros_like(self.q)
        self.params = _Params(float(T), float(dt), float(tau), float(pile_lambda), float(r_cut), float(alpha),
                              int(precision), int(nlist_cap), int(free_ring_substeps), int(coulomb), int(ewald_kmax))
        s, keep = pack_system(sysm, self.q.data_ptr(), self.p.data_ptr(), self.f.data_ptr(), seed)
        nbytes = L.mixts_workspace_size(C.byref(s), 1, C.byref(self.params))
        if nbytes == 0:
            raise MixtsError(1, "mixts_workspace_size rejected the system")
        self.ws = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        aligned = (base + 255) & ~255
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = L.mixts_init(C.byref(s), 1, C.byref(self.params), C.c_void_p(aligned), int(nbytes),
                              C.c_void_p(self.stream.cuda_stream), C.byref(h))
        del keep
        if st != 0:
            raise MixtsError(st, "mixts_init failed")
        self.h = h

    # -- calls -------------------------------------------------------------
    def _check(self, st):
        if st != 0:
            raise MixtsError(st, lib().mixts_last_error(self.h).decode())

    def forces(self, energy=True):
        e = C.c_double(0.0)
        self._check(lib().mixts_forces(self.h, C.byref(e) if energy else None))
        return self.f, (e.value if energy else None)

    def step(self, n=1):
        self._check(lib().mixts_step(self.h, int(n)))

    def estimators(self) -> dict:
        out = _Estimates()
        self._check(lib().mixts_estimators(self.h, C.byref(out)))
        d = {n: getattr(out, n) for n, _ in _Estimates._fields_[:16]}
        nt = self.n_types
        for n in ("KE_prim", "KE_cv", "Rg2", "E_spring_t"):
            d[n] = list(getattr(out, n))[:nt]
        d["step"] = int(out.step)
        return d

    def nlist(self, kind=0):
        """(triplets [n,3] int32 sorted by (owner, partner, code), thresholds[3])."""
        n = C.c_long(0)
        th = (C.c_double * 3)()
        self._check(lib().mixts_nlist(self.h, kind, None, 0, C.byref(n), th))
        out = np.zeros((max(1, n.value), 3), dtype=np.int32)
        self._check(lib().mixts_nlist(self.h, kind, _ptr(out, C.c_int), n.value, C.byref(n), th))
        t = out[:n.value]
        order = np.lexsort((t[:, 2], t[:, 1], t[:, 0]))
        return t[order], np.array(list(th))

    def get_state(self) -> bytes:
        nb = lib().mixts_state_size(self.h)
        buf = (C.c_ubyte * nb)()
        self._check(lib().mixts_get_state(self.h, buf, nb))
        return bytes(buf)

    def set_state(self, blob: bytes):
        buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
        self._check(lib().mixts_set_state(self.h, buf, len(blob)))

    def gaussians(self, step, stage, dof0, n):
        out = self.torch.empty(int(n), dtype=self.torch.float32, device=self.device)
        self._check(lib().mixts_gaussians(self.h, int(step), int(stage), int(dof0), int(n),
                                          C.c_void_p(out.data_ptr())))
        return out

    def rdf_accumulate(self, type_a, type_b, hist, dr=0.02):
        """Add the current configuration's pair histogram to ``hist`` (int64 device tensor)."""
        self._check(lib().mixts_rdf_accumulate(self.h, int(type_a), int(type_b), float(dr), int(hist.numel()),
                                               C.c_void_p(hist.data_ptr())))

    def rdf_normalise(self, type_a, type_b, hist, n_frames, dr=0.02):
        """g(r) per bin from a histogram summed over n_frames configurations."""
        h = np.ascontiguousarray(hist.cpu().numpy() if hasattr(hist, "cpu") else hist).astype(np.uint64)
        g = np.zeros(h.size)
        self._check(lib().mixts_rdf_normalise(self.h, int(type_a), int(type_b), float(dr), int(h.size),
                                              int(n_frames), _ptr(h, C.c_uint64), _ptr(g, C.c_double)))
        return g

    def vacf_accumulate(self, type_t, ring, acc, cnt):
        """Add the current frame to a centroid velocity autocorrelation
        (float64 device tensors ring [n_lag, N_t, 3], acc [n_lag], int64 cnt
        [n_lag], zeroed before the first call)."""
        self._check(lib().mixts_vacf_accumulate(self.h, int(type_t), int(acc.numel()), C.c_void_p(ring.data_ptr()),
                                                C.c_void_p(acc.data_ptr()), C.c_void_p(cnt.data_ptr())))

    def set_graph(self, steps_per_launch):
        """Steps per captured CUDA graph launch of step() (0: plain launches)."""
        self._check(lib().mixts_set_graph(self.h, int(steps_per_launch)))

    def potential_grad(self, type_a, type_b, theta, grad_out=1.0, want_dvdq=True, want_theta=True):
        """V_mix(q, theta), grad_out * dV/dq (device tensor or None), grad_out * dV/dtheta (8 floats or None).

        theta follows THETA_NAMES; it is applied to this evaluation only.
        Without want_theta the adjoint sums over theta are not run.
        """
        th = (C.c_double * 8)(*[float(x) for x in theta])
        v = C.c_double(0.0)
        g = (C.c_double * 8)()
        dq = self.torch.empty_like(self.q) if want_dvdq else None
        self._check(lib().mixts_potential_grad(self.h, int(type_a), int(type_b), th, float(grad_out), C.byref(v),
                                               C.c_void_p(dq.data_ptr()) if want_dvdq else None,
                                               g if want_theta else None))
        return v.value, dq, (np.array(list(g)) if want_theta else None)

    def reload(self):
        """Declare that q and/or p were rewritten in place (host-resident state)."""
        self._check(lib().mixts_reload(self.h))

    def set_timing(self, on=True):
        self._check(lib().mixts_set_timing(self.h, 1 if on else 0))

    def timing(self):
        """(ms per phase dict, calls per phase dict, kernels launched since init)."""
        ms = (C.c_double * len(PHASES))()
        calls = (C.c_longlong * len(PHASES))()
        k = C.c_longlong(0)
        self._check(lib().mixts_get_timing(self.h, ms, calls, C.byref(k)))
        return dict(zip(PHASES, list(ms))), dict(zip(PHASES, list(calls))), int(k.value)

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "h", None):
            if not getattr(self, "_borrowed", False):
                lib().mixts_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def alu_peak_tflops(fp64, iters=None, stream=None):
    """Measured FMA-chain throughput of this GPU in TFLOP/s (binary64 or binary32)."""
    import torch
    if iters is None:
        iters = 2000 if fp64 else 60000
    st = stream if stream is not None else torch.cuda.current_stream()
    flop, ms = C.c_double(0.0), C.c_double(0.0)
    rc = lib().mixts_alu_probe(1 if fp64 else 0, int(iters), C.c_void_p(st.cuda_stream), C.byref(flop), C.byref(ms))
    if rc != 0:
        raise MixtsError(rc, "mixts_alu_probe failed")
    return flop.value / (ms.value * 1e-3) / 1e12, ms.value


def _potential_fn():
    import torch

    class MixTSPotential(torch.autograd.Function):
        """V_mix as a differentiable function of (theta, q) for one MixTS engine.

        ``theta`` is a float64 CPU tensor of 8 parameters (THETA_NAMES order),
        ``q`` a float64 device tensor [n_beads, 3]. The forward pass evaluates
        V only; the backward pass re-evaluates the pair terms at the saved
        (theta, q) and runs the adjoint sums, scaled by the incoming gradient,
        for the inputs that need one (nothing per pair term is stored).
        """

        @staticmethod
        def forward(ctx, theta, q, engine, type_a, type_b):
            if q.data_ptr() != engine.q.data_ptr():
                engine.q.copy_(q)
            v, _, _ = engine.potential_grad(type_a, type_b, theta.detach().cpu().tolist(), 1.0, want_dvdq=False,
                                            want_theta=False)
            ctx.engine, ctx.types = engine, (type_a, type_b)
            ctx.save_for_backward(theta.detach(), q)
            return torch.tensor(v, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gv):
            theta, q = ctx.saved_tensors
            engine = ctx.engine
            if q.data_ptr() != engine.q.data_ptr():
                engine.q.copy_(q)
            want_th, want_q = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
            _, dq, g = engine.potential_grad(ctx.types[0], ctx.types[1], theta.cpu().tolist(), float(gv),
                                             want_dvdq=want_q, want_theta=want_th)
            gth = torch.from_numpy(g).to(torch.float64) if want_th else None
            return gth, (dq if want_q else None), None, None, None

    return MixTSPotential


_MixTSPotential = None


def mixts_potential(theta, q, engine, type_a, type_b):
    """Differentiable V_mix(theta, q) evaluated by the engine's kernels."""
    global _MixTSPotential
    if _MixTSPotential is None:
        _MixTSPotential = _potential_fn()
    return _MixTSPotential.apply(theta, q, engine, type_a, type_b)


class MixTSBatch:
    """Many independent systems (uneven sizes and bead counts) behind one
    batched handle; a multi-step ``step`` runs as captured CUDA graph launches.

    ``q[i]``, ``p[i]``, ``f[i]`` are the device state tensors of system i.
    """

    def __init__(self, systems, T=300.0, dt=0.25, tau=100.0, pile_lambda=1.0, r_cut=9.0, alpha=0.2,
                 precision=FP64, nlist_cap=0, seeds=None, device="cuda:0", stream=None, free_ring_substeps=0,
                 coulomb=0, ewald_kmax=0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("MixTSBatch needs a CUDA device")
        L = lib()
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        n = len(systems)
        if n < 2:
            raise ValueError("a batch holds at least two systems")
        seeds = list(range(n)) if seeds is None else list(seeds)
        self.q, self.p, self.f, self.n_types = [], [], [], []
        structs, keep = [], []
        with torch.cuda.device(self.device):
            for sysm, seed in zip(systems, seeds):
                q = torch.from_numpy(np.asarray(sysm.q, dtype=np.float64).copy()).to(self.device)
                p = torch.from_numpy(np.asarray(sysm.p, dtype=np.float64).copy()).to(self.device)
                f = torch.zeros_like(q)
                self.q.append(q)
                self.p.append(p)
                self.f.append(f)
                self.n_types.append(int(len(sysm.P_type)))
                st, k = pack_system(sysm, q.data_ptr(), p.data_ptr(), f.data_ptr(), seed)
                structs.append(st)
                keep.append(k)
        arr = (_System * n)(*structs)
        self.n = n
        self.params = _Params(float(T), float(dt), float(tau), float(pile_lambda), float(r_cut), float(alpha),
                              int(precision), int(nlist_cap), int(free_ring_substeps), int(coulomb), int(ewald_kmax))
        nbytes = L.mixts_workspace_size(arr, n, C.byref(self.params))
        if nbytes == 0:
            raise MixtsError(1, "mixts_workspace_size rejected the batch")
        self.ws = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=self.device)
        aligned = (self.ws.data_ptr() + 255) & ~255
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = L.mixts_init(arr, n, C.byref(self.params), C.c_void_p(aligned), int(nbytes),
                              C.c_void_p(self.stream.cuda_stream), C.byref(h))
        del keep
        if st != 0:
            raise MixtsError(st, "mixts_init failed for the batch")
        self.h = h

    def _check(self, st):
        if st != 0:
            raise MixtsError(st, lib().mixts_last_error(self.h).decode())

    def forces(self):
        e = (C.c_double * self.n)()
        self._check(lib().mixts_forces(self.h, e))
        return list(e)

    def step(self, n=1):
        self._check(lib().mixts_step(self.h, int(n)))

    def tune(self, steps_per_launch=10):
        t = _Tuning()
        self._check(lib().mixts_batch_tune(self.h, int(steps_per_launch), C.byref(t)))
        return {n: getattr(t, n) for n, _ in _Tuning._fields_}

    def estimators(self):
        out = (_Estimates * self.n)()
        self._check(lib().mixts_estimators(self.h, out))
        res = []
        for i in range(self.n):
            d = {n: getattr(out[i], n) for n, _ in _Estimates._fields_[:16]}
            for n in ("KE_prim", "KE_cv", "Rg2", "E_spring_t"):
                d[n] = list(getattr(out[i], n))[:self.n_types[i]]
            d["step"] = int(out[i].step)
            res.append(d)
        return res

    def get_state(self) -> bytes:
        nb = lib().mixts_state_size(self.h)
        buf = (C.c_ubyte * nb)()
        self._check(lib().mixts_get_state(self.h, buf, nb))
        return bytes(buf)

    def set_state(self, blob: bytes):
        buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
        self._check(lib().mixts_set_state(self.h, buf, len(blob)))

    def reload(self):
        self._check(lib().mixts_reload(self.h))

    def set_timing(self, on=True):
        self._check(lib().mixts_set_timing(self.h, 1 if on else 0))

    def timing(self):
        ms = (C.c_double * len(PHASES))()
        calls = (C.c_longlong * len(PHASES))()
        k = C.c_longlong(0)
        self._check(lib().mixts_get_timing(self.h, ms, calls, C.byref(k)))
        return dict(zip(PHASES, list(ms))), dict(zip(PHASES, list(calls))), int(k.value)

    def member(self, i):
        """A MixTS view of system i (borrowed handle; per-system queries)."""
        mh = C.c_void_p()
        self._check(lib().mixts_batch_member(self.h, int(i), C.byref(mh)))
        m = MixTS.__new__(MixTS)
        m.torch, m.device, m.stream = self.torch, self.device, self.stream
        m.q, m.p, m.f = self.q[i], self.p[i], self.f[i]
        m.n_beads, m.n_types = self.q[i].shape[0], self.n_types[i]
        m.h, m._borrowed, m._batch = mh, True, self
        return m

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "h", None):
            lib().mixts_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
