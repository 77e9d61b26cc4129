"""ctypes front end of ``mixts_oracle.c`` (see the C header for citations)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mixts_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libmixts_oracle.so")
_lib = None

R_CUT = 9.0
DSF_ALPHA = 0.2


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2 -ffp-contract=off)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    hdr = os.path.join(_HERE, "mixts_oracle.h")
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < max(
            os.path.getmtime(_SRC), os.path.getmtime(hdr)):
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


class OrSystem(C.Structure):
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
        ("box", C.c_double), ("r_cut", C.c_double), ("dsf_alpha", C.c_double),
        ("bead_mass_type", C.POINTER(C.c_double)),
        ("coulomb", C.c_int), ("ewald_kmax", C.c_int),
    ]


class OrParams(C.Structure):
    _fields_ = [("T", C.c_double), ("dt", C.c_double), ("tau_centroid", C.c_double),
                ("pile_lambda", C.c_double), ("seed", C.c_uint64), ("vv_substeps", C.c_int)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def _declare(L):
    S = C.POINTER(OrSystem)
    Pp = C.POINTER(OrParams)
    L.or_constants.argtypes = [_dp]
    L.or_validate_beads.argtypes = [C.c_int, _ip]
    L.or_pair_map.argtypes = [C.c_int, C.c_int, _ip, _ip]
    L.or_triple_map.argtypes = [C.c_int, C.c_int, C.c_int, _ip, _ip, _ip]
    L.or_forces.argtypes = [S, _dp, _dp, _dp]
    L.or_bead_force.argtypes = [S, _dp, C.c_int, C.c_int, _dp]
    L.or_nlist.argtypes = [S, _dp, C.c_long, _ip, _dp]
    L.or_nlist.restype = C.c_long
    L.or_pseudo_list.argtypes = [S, _dp, C.c_long, _ip, _dp]
    L.or_pseudo_list.restype = C.c_long
    L.or_nm_matrix.argtypes = [C.c_int, _dp]
    L.or_nm_freqs.argtypes = [C.c_int, C.c_double, _dp]
    L.or_step.argtypes = [S, Pp, _dp, _dp, _dp, C.c_uint64, _dp, _dp]
    L.or_grad_theta.argtypes = [S, _dp, C.c_int, C.c_int, _dp]
    L.or_rdf.argtypes = [S, _dp, C.c_int, C.c_int, C.c_double, C.c_int, _dp]
    L.or_estimators.argtypes = [S, Pp, _dp, _dp, _dp, _dp, _dp]
    L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]
    L.or_gaussians.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint64, C.c_long,
                               C.POINTER(C.c_float)]
    L.or_log_u24.argtypes = [C.c_uint32]
    L.or_log_u24.restype = C.c_float
    L.or_sincos_2pi.argtypes = [C.c_uint32, C.POINTER(C.c_float), C.POINTER(C.c_float)]


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


class _Bound:
    """Holds the numpy arrays a C struct points into."""

    def __init__(self, sysm, r_cut=R_CUT, alpha=DSF_ALPHA):
        f64 = lambda x: np.ascontiguousarray(x, dtype=np.float64)
        i32 = lambda x: np.ascontiguousarray(x, dtype=np.int32)
        self.keep = dict(
            type_of_atom=i32(sysm.type_of_atom), mol_of_atom=i32(sysm.mol_of_atom),
            P_type=i32(sysm.P_type), mass_type=f64(sysm.mass_type),
            charge_type=f64(sysm.charge_type), lj_eps=f64(sysm.lj_eps).ravel(),
            lj_sig=f64(sysm.lj_sig).ravel(), pseudo_type=i32(sysm.pseudo_type),
            pp_sigma=f64(sysm.pp_sigma), pp_A_eV=f64(sysm.pp_A_eV), pp_b=f64(sysm.pp_b),
            bonds=i32(sysm.bonds).ravel(), bond_k=f64(sysm.bond_k), bond_r0=f64(sysm.bond_r0),
            angles=i32(sysm.angles).ravel(), angle_k=f64(sysm.angle_k),
            angle_theta0=f64(sysm.angle_theta0),
        )
        bm = getattr(sysm, "bead_mass_type", None)
        if bm is not None:
            self.keep["bead_mass_type"] = f64(bm)
        k = self.keep
        self.s = OrSystem(
            sysm.n_atoms, sysm.n_types, _p(k["type_of_atom"], C.c_int), _p(k["mol_of_atom"], C.c_int),
            _p(k["P_type"], C.c_int), _p(k["mass_type"], C.c_double), _p(k["charge_type"], C.c_double),
            _p(k["lj_eps"], C.c_double), _p(k["lj_sig"], C.c_double), _p(k["pseudo_type"], C.c_int),
            _p(k["pp_sigma"], C.c_double), _p(k["pp_A_eV"], C.c_double), _p(k["pp_b"], C.c_double),
            int(sysm.bonds.shape[0]), _p(k["bonds"], C.c_int), _p(k["bond_k"], C.c_double),
            _p(k["bond_r0"], C.c_double), int(sysm.angles.shape[0]), _p(k["angles"], C.c_int),
            _p(k["angle_k"], C.c_double), _p(k["angle_theta0"], C.c_double),
            float(sysm.box), float(r_cut), float(alpha),
            _p(k["bead_mass_type"], C.c_double) if bm is not None else None,
            int(getattr(sysm, "coulomb", 0) or 0), int(getattr(sysm, "ewald_kmax", 0) or 0))
        self.nt = sysm.n_types
        self.nbeads = sysm.n_beads


def constants() -> dict:
    o = np.zeros(6)
    lib().or_constants(_p(o, C.c_double))
    return dict(kB=o[0], hbar=o[1], kcal=o[2], ev=o[3], ke=o[4], ev_kcal=o[5])


def validate_beads(P) -> bool:
    a = np.ascontiguousarray(P, dtype=np.int32)
    return lib().or_validate_beads(len(a), _p(a, C.c_int)) == 0


def pair_map(Ni, Nj):
    bi = np.zeros(Ni, dtype=np.int32)
    bj = np.zeros(Ni, dtype=np.int32)
    n = lib().or_pair_map(Ni, Nj, _p(bi, C.c_int), _p(bj, C.c_int))
    return bi[:n], bj[:n]


def triple_map(Ni, Nj, Nk):
    b = [np.zeros(Ni, dtype=np.int32) for _ in range(3)]
    n = lib().or_triple_map(Ni, Nj, Nk, *[_p(x, C.c_int) for x in b])
    return tuple(x[:n] for x in b)


def forces(sysm, q=None, r_cut=R_CUT, alpha=DSF_ALPHA):
    """Returns (F [n_beads,3] kcal/mol/A, parts[10])."""
    b = _Bound(sysm, r_cut, alpha)
    q = np.ascontiguousarray(sysm.q if q is None else q, dtype=np.float64)
    F = np.zeros_like(q)
    parts = np.zeros(10)
    lib().or_forces(C.byref(b.s), _p(q, C.c_double), _p(F, C.c_double), _p(parts, C.c_double))
    return F, parts


def bead_force(sysm, atom, bead, q=None, r_cut=R_CUT, alpha=DSF_ALPHA):
    b = _Bound(sysm, r_cut, alpha)
    q = np.ascontiguousarray(sysm.q if q is None else q, dtype=np.float64)
    out = np.zeros(3)
    lib().or_bead_force(C.byref(b.s), _p(q, C.c_double), int(atom), int(bead), _p(out, C.c_double))
    return out


def nlist(sysm, q=None, r_cut=R_CUT, cap=None):
    """Returns (triplets [n,3] int32 sorted, d_max, threshold)."""
    b = _Bound(sysm, r_cut)
    q = np.ascontiguousarray(sysm.q if q is None else q, dtype=np.float64)
    cap = cap or 1024
    while True:
        out = np.zeros((cap, 3), dtype=np.int32)
        th = np.zeros(3)
        n = lib().or_nlist(C.byref(b.s), _p(q, C.c_double), cap, _p(out, C.c_int), _p(th, C.c_double))
        if n >= 0:
            break
        cap = -n
    t = out[:n]
    order = np.lexsort((t[:, 2], t[:, 1], t[:, 0]))
    return t[order], th[0], th[1]


def pseudo_list(sysm, q=None, r_cut=R_CUT, cap=None):
    b = _Bound(sysm, r_cut)
    q = np.ascontiguousarray(sysm.q if q is None else q, dtype=np.float64)
    cap = cap or 1024
    while True:
        out = np.zeros((cap, 3), dtype=np.int32)
        th = np.zeros(3)
        n = lib().or_pseudo_list(C.byref(b.s), _p(q, C.c_double), cap, _p(out, C.c_int),
                                 _p(th, C.c_double))
        if n >= 0:
            break
        cap = -n
    t = out[:n]
    order = np.lexsort((t[:, 2], t[:, 1], t[:, 0]))
    return t[order], th


THETA_NAMES = ["sigma_a", "A_a", "b_a", "sigma_b", "A_b", "b_b", "q_a", "eps_aa"]


def theta_of(sysm, ta, tb):
    """Current theta = (sigma_a, A_a [eV], b_a, sigma_b, A_b, b_b, q_a, eps_aa)."""
    return np.array([sysm.pp_sigma[ta], sysm.pp_A_eV[ta], sysm.pp_b[ta], sysm.pp_sigma[tb], sysm.pp_A_eV[tb],
                     sysm.pp_b[tb], sysm.charge_type[ta], sysm.lj_eps[ta, ta]], dtype=np.float64)


def with_theta(sysm, ta, tb, theta):
    """Copy of the system with theta applied; cross LJ of type a rescaled by
    sqrt(eps_aa'/eps_aa) (Lorentz-Berthelot), or left as they are when the
    system's eps_aa is 0."""
    s = sysm.copy()
    s.pp_sigma = sysm.pp_sigma.copy()
    s.pp_A_eV = sysm.pp_A_eV.copy()
    s.pp_b = sysm.pp_b.copy()
    s.charge_type = sysm.charge_type.copy()
    s.lj_eps = sysm.lj_eps.copy()
    s.pp_sigma[ta], s.pp_A_eV[ta], s.pp_b[ta] = theta[0], theta[1], theta[2]
    s.pp_sigma[tb], s.pp_A_eV[tb], s.pp_b[tb] = theta[3], theta[4], theta[5]
    s.charge_type[ta] = theta[6]
    e0 = sysm.lj_eps[ta, ta]
    scale = np.sqrt(theta[7] / e0) if e0 > 0 else 1.0  # cross terms held fixed when eps_aa = 0
    for x in range(s.n_types):
        if x != ta:
            s.lj_eps[ta, x] = sysm.lj_eps[ta, x] * scale
            s.lj_eps[x, ta] = sysm.lj_eps[x, ta] * scale
    s.lj_eps[ta, ta] = theta[7]
    return s


def grad_theta(sysm, ta, tb, q=None, r_cut=R_CUT, alpha=DSF_ALPHA):
    b = _Bound(sysm, r_cut, alpha)
    q = np.ascontiguousarray(sysm.q if q is None else q, dtype=np.float64)
    g = np.zeros(8)
    lib().or_grad_theta(C.byref(b.s), _p(q, C.c_double), int(ta), int(tb), _p(g, C.c_double))
    return g


def rdf_hist(sysm, ta, tb, dr=0.02, nbins=400, q=None):
    """Weighted pair-distance histogram (sum of 1/P* over ordered pairs and slices)."""
    b = _Bound(sysm, R_CUT, DSF_ALPHA)
    q = np.ascontiguousarray(sysm.q if q is None else q, dtype=np.float64)
    h = np.zeros(int(nbins))
    lib().or_rdf(C.byref(b.s), _p(q, C.c_double), int(ta), int(tb), float(dr), int(nbins), _p(h, C.c_double))
    return h


def rdf_normalise(hist, n_frames, N_a, N_b, same, box, dr):
    """g(r) per bin: histogram / (frames * N_a * rho_b * shell volume), rho_b =
    (N_b - [a == b]) / V."""
    k = np.arange(len(hist))
    shell = 4.0 / 3.0 * np.pi * ((k + 1) ** 3 - k ** 3) * dr ** 3
    rho = (N_b - (1 if same else 0)) / box ** 3
    return hist / (n_frames * N_a * rho * shell)


def nm_matrix(P):
    Cm = np.zeros(P * P)
    lib().or_nm_matrix(P, _p(Cm, C.c_double))
    return Cm.reshape(P, P)


def nm_freqs(P, beta_hbar):
    w = np.zeros(P)
    lib().or_nm_freqs(P, float(beta_hbar), _p(w, C.c_double))
    return w


def make_params(T=300.0, dt=0.25, tau=100.0, lam=1.0, seed=0, vv=0):
    """Integrator parameters; vv > 0 evolves the free ring polymer by velocity
    Verlet on the springs with vv sub-steps instead of exactly."""
    return OrParams(float(T), float(dt), float(tau), float(lam), int(seed), int(vv))


class Runner:
    """Holds (q, p, F, step, heat) and advances them with ``or_step``."""

    def __init__(self, sysm, params, q=None, p=None, r_cut=R_CUT, alpha=DSF_ALPHA):
        self.b = _Bound(sysm, r_cut, alpha)
        self.prm = params
        self.q = np.ascontiguousarray((sysm.q if q is None else q).copy(), dtype=np.float64)
        self.p = np.ascontiguousarray((sysm.p if p is None else p).copy(), dtype=np.float64)
        self.F = np.zeros_like(self.q)
        self.parts = np.zeros(10)
        lib().or_forces(C.byref(self.b.s), _p(self.q, C.c_double), _p(self.F, C.c_double),
                        _p(self.parts, C.c_double))
        self.step_index = 0
        self.heat = np.zeros(1)

    def step(self, n=1):
        L = lib()
        for _ in range(n):
            L.or_step(C.byref(self.b.s), C.byref(self.prm), _p(self.q, C.c_double),
                      _p(self.p, C.c_double), _p(self.F, C.c_double), self.step_index,
                      _p(self.heat, C.c_double), _p(self.parts, C.c_double))
            self.step_index += 1

    def estimators(self) -> dict:
        out = np.zeros(16 + 4 * self.b.nt)
        lib().or_estimators(C.byref(self.b.s), C.byref(self.prm), _p(self.q, C.c_double),
                            _p(self.p, C.c_double), _p(self.F, C.c_double),
                            _p(self.parts, C.c_double), _p(out, C.c_double))
        return unpack_estimators(out, self.b.nt, self.heat[0])


def unpack_estimators(out, nt, heat=0.0) -> dict:
    keys = ["V", "V_lj", "V_coul", "V_bond", "V_angle", "V_pseudo", "KE_beads", "E_spring",
            "virial", "T_beads", "H_mix", "n_evals", "n_pseudo_evals"]
    d = {k: float(out[i]) for i, k in enumerate(keys)}
    d["KE_prim"] = [float(out[16 + 4 * t]) for t in range(nt)]
    d["KE_cv"] = [float(out[16 + 4 * t + 1]) for t in range(nt)]
    d["Rg2"] = [float(out[16 + 4 * t + 2]) for t in range(nt)]
    d["E_spring_t"] = [float(out[16 + 4 * t + 3]) for t in range(nt)]
    d["heat"] = float(heat)
    d["H_conserved"] = d["H_mix"] + float(heat)
    return d


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def gaussians(seed, step, stage, dof0, n):
    out = np.zeros(n, dtype=np.float32)
    lib().or_gaussians(int(seed), int(step), int(stage), int(dof0), int(n), _p(out, C.c_float))
    return out


def log_u24(r):
    return lib().or_log_u24(int(r))


def sincos_2pi(r):
    s = C.c_float()
    c = C.c_float()
    lib().or_sincos_2pi(int(r), C.byref(s), C.byref(c))
    return s.value, c.value


def rpmd_bead_masses(sysm):
    """Bead masses m_f = m / P_t per type. In the beta H_mix convention of
    Eq. (mts-hamiltonian) (potential weighted 1/N_i, springs N_i m/(beta hbar)^2)
    Newton's equations with these masses give every centroid the RPMD
    equation of motion m d^2(qbar)/dt^2 = -(1/P) sum_b dV/dq_b."""
    return np.asarray(sysm.mass_type, dtype=np.float64) / np.asarray(sysm.P_type, dtype=np.float64)


def centroid_velocities(sysm, p, type_t):
    """Centroid velocities dq̄/dt = (1/P) sum_b p_b / m_f of the atoms of type t,
    [N_t, 3], from bead momenta p in the flat layout."""
    bm = getattr(sysm, "bead_mass_type", None)
    mf = float(bm[type_t]) if bm is not None else float(sysm.mass_type[type_t])
    off = sysm.type_offsets()
    N = int(sysm.n_of_type()[type_t])
    P = int(sysm.P_type[type_t])
    blk = np.asarray(p[off[type_t]:off[type_t + 1]]).reshape(P, N, 3)
    return blk.mean(axis=0) / mf


class VelocityCorrelation:
    """Time correlation <v(0).v(t)> of centroid velocities, accumulated over
    every time origin of a trajectory (Sec. "Output and Analysis": RPMD
    correlation functions from NVE trajectories). add(v) takes the [N, 3]
    velocities of one frame; acc[L] sums v(now).v(now - L) over atoms and
    origins, cnt[L] counts the origins, for lags L < n_lag frames."""

    def __init__(self, n_lag):
        self.n_lag = int(n_lag)
        self.frames = []
        self.acc = np.zeros(self.n_lag)
        self.cnt = np.zeros(self.n_lag, dtype=np.int64)

    def add(self, v):
        v = np.asarray(v, dtype=np.float64)
        self.frames.append(v)
        n = len(self.frames)
        for L in range(min(self.n_lag, n)):
            self.acc[L] += float(np.sum(v * self.frames[n - 1 - L]))
            self.cnt[L] += 1
        if len(self.frames) > self.n_lag:
            self.frames.pop(0)

    def per_atom(self, n_atoms):
        """C(L) per atom: acc / (cnt * n_atoms)."""
        return self.acc / np.maximum(self.cnt, 1) / n_atoms
