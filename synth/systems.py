"""System builders for the synthetic workloads (inputs only, no method arithmetic)."""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# Exact SI definitions (2019) used only to draw Maxwell-Boltzmann momenta.
_SI_KB = 1.380649e-23
_SI_NA = 6.02214076e23
# k_B in amu A^2 fs^-2 K^-1, with 1 amu = 1e-3/N_A kg.
_KB_MD = _SI_KB * _SI_NA / 1.0e7

MASS = {"O": 15.999, "H": 1.008, "ion": 58.933, "e": 5.48579909e-4}

WATER = dict(
    q_O=-0.82, q_H=0.41, eps_OO=0.1554, sig_OO=3.1655,
    bond_k=1059.2, bond_r0=1.012, angle_k=75.9, angle_theta0_deg=113.24,
)

ION3 = dict(charge=3.0, eps=0.1, sigma=2.0, mass=MASS["ion"], P=1)

# Pseudopotential site parameters of the electron workloads (A in eV).
PSEUDO = dict(
    O=dict(sigma=0.8, A=20.0, b=0.5),
    H=dict(sigma=0.5, A=5.0, b=0.4),
    ion=dict(sigma=0.6, A=30.0, b=0.45),
)


@dataclass
class System:
    """One periodic system in the shared flat bead layout (see package doc)."""

    name: str
    box: float
    type_names: list
    P_type: np.ndarray
    mass_type: np.ndarray
    charge_type: np.ndarray
    lj_eps: np.ndarray
    lj_sig: np.ndarray
    pseudo_type: np.ndarray
    pp_sigma: np.ndarray
    pp_A_eV: np.ndarray
    pp_b: np.ndarray
    type_of_atom: np.ndarray
    mol_of_atom: np.ndarray
    bonds: np.ndarray
    bond_k: np.ndarray
    bond_r0: np.ndarray
    angles: np.ndarray
    angle_k: np.ndarray
    angle_theta0: np.ndarray
    q: np.ndarray = field(default=None)
    p: np.ndarray = field(default=None)
    # fictitious bead mass per type (kinetic term p^2/2m_f); None: the physical mass
    bead_mass_type: np.ndarray = field(default=None)
    # electrostatics: 0 damped shifted force per bead pair; 1 Ewald (real space per
    # bead pair, reciprocal space on centroids with wave vectors |n| <= ewald_kmax)
    coulomb: int = 0
    ewald_kmax: int = 0

    # ---- bookkeeping (layout only) ----
    @property
    def n_atoms(self) -> int:
        return int(self.type_of_atom.shape[0])

    @property
    def n_types(self) -> int:
        return int(self.P_type.shape[0])

    def n_of_type(self) -> np.ndarray:
        return np.bincount(self.type_of_atom, minlength=self.n_types).astype(np.int64)

    def type_offsets(self) -> np.ndarray:
        n = self.n_of_type()
        sizes = n * self.P_type.astype(np.int64)
        return np.concatenate([[0], np.cumsum(sizes)])

    def rank_in_type(self) -> np.ndarray:
        rank = np.zeros(self.n_atoms, dtype=np.int64)
        seen = np.zeros(self.n_types, dtype=np.int64)
        for a, t in enumerate(self.type_of_atom):
            rank[a] = seen[t]
            seen[t] += 1
        return rank

    @property
    def n_beads(self) -> int:
        return int(self.type_offsets()[-1])

    def bead_rows(self, atom: int) -> np.ndarray:
        """Rows of all beads of ``atom`` in bead order."""
        t = int(self.type_of_atom[atom])
        off = self.type_offsets()[t]
        n_t = self.n_of_type()[t]
        k = self.rank_in_type()[atom]
        return off + np.arange(self.P_type[t]) * n_t + k

    def copy(self) -> "System":
        import copy as _c
        s = _c.copy(self)
        s.q = None if self.q is None else self.q.copy()
        s.p = None if self.p is None else self.p.copy()
        return s


def _beads_from_atoms(sysm: System, pos: np.ndarray) -> np.ndarray:
    """Every bead of every atom at the atom's position, in the bead layout."""
    q = np.empty((sysm.n_beads, 3))
    off = sysm.type_offsets()
    n_t = sysm.n_of_type()
    rank = sysm.rank_in_type()
    for t in range(sysm.n_types):
        atoms = np.where(sysm.type_of_atom == t)[0]
        for b in range(int(sysm.P_type[t])):
            q[off[t] + b * n_t[t] + rank[atoms]] = pos[atoms]
    return q


def density_box_length(n_waters: int, density_g_cm3: float = 0.997) -> float:
    """Cubic box edge (A) holding n waters at the given mass density."""
    mol_mass = 18.01528
    vol_cm3 = n_waters * mol_mass / (_SI_NA * density_g_cm3)
    return vol_cm3 ** (1.0 / 3.0) * 1.0e8


def _maxwell_momenta(rng, sysm: System, T: float) -> np.ndarray:
    m_row = np.empty(sysm.n_beads)
    off = sysm.type_offsets()
    for t in range(sysm.n_types):
        m_row[off[t]:off[t + 1]] = sysm.mass_type[t]
    xi = rng.standard_normal((sysm.n_beads, 3))
    return xi * np.sqrt(m_row * _KB_MD * T)[:, None]


def water_box(n_waters: int, box: float, P_H: int, P_O: int, seed: int = 0,
              T: float = 300.0, ion: dict | None = None,
              electron_P: int | None = None, jitter: float = 0.05,
              name: str | None = None) -> System:
    """Flexible-water box, optionally with a classical ion and a quantum electron."""
    rng = np.random.default_rng(seed)
    w = WATER
    names = ["O", "H"]
    P = [P_O, P_H]
    mass = [MASS["O"], MASS["H"]]
    charge = [w["q_O"], w["q_H"]]
    if ion is not None:
        names.append("ion")
        P.append(int(ion.get("P", 1)))
        mass.append(float(ion.get("mass", MASS["ion"])))
        charge.append(float(ion["charge"]))
    if electron_P is not None:
        names.append("e")
        P.append(int(electron_P))
        mass.append(MASS["e"])
        charge.append(-1.0)
    nt = len(names)
    eps = np.zeros((nt, nt))
    sig = np.ones((nt, nt))
    eps[0, 0] = w["eps_OO"]
    sig[0, 0] = w["sig_OO"]
    if ion is not None:
        ti = names.index("ion")
        # Lorentz-Berthelot ion-O pair, no ion-H and no ion-ion LJ.
        e_io = math.sqrt(ion["eps"] * w["eps_OO"])
        s_io = 0.5 * (ion["sigma"] + w["sig_OO"])
        eps[ti, 0] = eps[0, ti] = e_io
        sig[ti, 0] = sig[0, ti] = s_io
    pseudo = np.zeros(nt, dtype=np.int32)
    pp_sigma = np.ones(nt)
    pp_A = np.zeros(nt)
    pp_b = np.ones(nt)
    if electron_P is not None:
        pseudo[names.index("e")] = 1
        for tn in ("O", "H", "ion"):
            if tn in names:
                k = names.index(tn)
                pp_sigma[k] = PSEUDO[tn]["sigma"]
                pp_A[k] = PSEUDO[tn]["A"]
                pp_b[k] = PSEUDO[tn]["b"]

    n_sites = n_waters + (1 if ion is not None else 0)
    m_side = int(math.ceil(n_sites ** (1.0 / 3.0) - 1e-9))
    a = box / m_side
    # even-parity sublattice first (nearest-neighbour spacing sqrt(2) a when
    # at most half the grid is filled), then the odd one; x fastest in each
    sites = []
    for parity in (0, 1):
        for iz in range(m_side):
            for iy in range(m_side):
                for ix in range(m_side):
                    if (ix + iy + iz) % 2 == parity:
                        sites.append(((ix + 0.5) * a, (iy + 0.5) * a, (iz + 0.5) * a))
    sites = np.array(sites)
    if ion is not None:
        c = np.full(3, box / 2)
        d = np.linalg.norm(sites - c, axis=1)
        sites = np.delete(sites, int(np.argmin(d)), axis=0)
    if len(sites) < n_waters:
        raise ValueError("lattice too small for the requested water count")
    sites = sites[:n_waters]

    th = math.radians(w["angle_theta0_deg"]) / 2
    r0 = w["bond_r0"]
    h1 = np.array([math.sin(th), 0.0, math.cos(th)]) * r0
    h2 = np.array([-math.sin(th), 0.0, math.cos(th)]) * r0

    types, mols, pos = [], [], []
    bonds, angles = [], []
    for m, s in enumerate(sites):
        base = len(types)
        types += [0, 1, 1]
        mols += [m, m, m]
        pos += [s, s + h1, s + h2]
        bonds += [(base, base + 1), (base, base + 2)]
        angles += [(base + 1, base, base + 2)]
    pos = np.array(pos) + rng.normal(0.0, jitter, (len(pos), 3))
    pos = list(pos)
    mol_next = n_waters
    if ion is not None:
        types.append(names.index("ion"))
        mols.append(mol_next)
        mol_next += 1
        pos.append(np.full(3, box / 2))
    if electron_P is not None:
        types.append(names.index("e"))
        mols.append(mol_next)
        mol_next += 1
        pos.append(np.full(3, box / 2))

    nb = len(bonds)
    na = len(angles)
    sysm = System(
        name=name or f"water{n_waters}_H{P_H}_O{P_O}",
        box=float(box), type_names=names,
        P_type=np.array(P, dtype=np.int32),
        mass_type=np.array(mass, dtype=np.float64),
        charge_type=np.array(charge, dtype=np.float64),
        lj_eps=eps, lj_sig=sig, pseudo_type=pseudo,
        pp_sigma=pp_sigma, pp_A_eV=pp_A, pp_b=pp_b,
        type_of_atom=np.array(types, dtype=np.int32),
        mol_of_atom=np.array(mols, dtype=np.int32),
        bonds=np.array(bonds, dtype=np.int32).reshape(nb, 2),
        bond_k=np.full(nb, w["bond_k"]), bond_r0=np.full(nb, w["bond_r0"]),
        angles=np.array(angles, dtype=np.int32).reshape(na, 3),
        angle_k=np.full(na, w["angle_k"]),
        angle_theta0=np.full(na, math.radians(w["angle_theta0_deg"])),
    )
    q = _beads_from_atoms(sysm, np.asarray(pos))
    if electron_P is not None:
        e_atom = sysm.n_atoms - 1
        rows = sysm.bead_rows(e_atom)
        q[rows] = np.full(3, box / 2) + rng.normal(0.0, 1.0 / math.sqrt(3.0), (len(rows), 3))
    sysm.q = q
    sysm.p = _maxwell_momenta(rng, sysm, T)
    return sysm


def harmonic_tether(P_list, k_list, masses=None, box: float = 200.0, seed: int = 0,
                    T: float = 300.0, name: str = "tether") -> System:
    """Particles joined by harmonic springs with zero rest length.

    ``P_list`` gives the bead count of each particle (one type per particle);
    ``k_list`` is a list of (a, c, k) springs in kcal/mol/A^2. No charges, no
    LJ; all particles form one molecule, so only the springs act.
    """
    rng = np.random.default_rng(seed)
    n = len(P_list)
    masses = masses if masses is not None else [1.0] * n
    nt = n
    bonds = np.array([(a, c) for a, c, _ in k_list], dtype=np.int32).reshape(-1, 2)
    sysm = System(
        name=name, box=float(box), type_names=[f"T{i}" for i in range(n)],
        P_type=np.array(P_list, dtype=np.int32),
        mass_type=np.array(masses, dtype=np.float64),
        charge_type=np.zeros(nt), lj_eps=np.zeros((nt, nt)), lj_sig=np.ones((nt, nt)),
        pseudo_type=np.zeros(nt, dtype=np.int32), pp_sigma=np.ones(nt),
        pp_A_eV=np.zeros(nt), pp_b=np.ones(nt),
        type_of_atom=np.arange(n, dtype=np.int32), mol_of_atom=np.zeros(n, dtype=np.int32),
        bonds=bonds, bond_k=np.array([k for _, _, k in k_list], dtype=np.float64),
        bond_r0=np.zeros(len(k_list)),
        angles=np.zeros((0, 3), dtype=np.int32), angle_k=np.zeros(0), angle_theta0=np.zeros(0),
    )
    q = np.full((sysm.n_beads, 3), box / 2) + rng.normal(0.0, 0.05, (sysm.n_beads, 3))
    sysm.q = q
    sysm.p = _maxwell_momenta(rng, sysm, T)
    return sysm


def bead_counts_table(n_waters: int, P_H: int, P_O: int, n_ions: int = 0,
                      P_ion: int = 1, electron_P: int = 0) -> int:
    """Total particle count (sum of bead counts) of a water/ion/electron system."""
    return n_waters * (2 * P_H + P_O) + n_ions * P_ion + electron_P


def batched_draws(n_systems: int = 64, seed: int = 1000):
    """Uneven (water count, P_H, P_O) triples for a batch of independent systems."""
    rng = np.random.default_rng(seed)
    waters = rng.choice([32, 64, 128, 256, 512], size=n_systems)
    ph = rng.choice([4, 8, 16, 32, 64], size=n_systems)
    po = np.maximum(1, ph // 4)
    return [(int(w), int(h), int(o)) for w, h, o in zip(waters, ph, po)]
