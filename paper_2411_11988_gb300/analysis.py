"""Sampled observables of mixTS-PIMD runs and the partial-quantisation sweep.

The observables are those of Sec. "Output and Analysis": the centroid-virial
kinetic energy per type, the mean squared bead spread R_g^2 per type, the bead
temperature, radial distribution functions and ring-polymer molecular
dynamics (RPMD) time correlation functions from NVE trajectories, all produced
on the GPU by the library (estimator, RDF histogram and correlation kernels). The partial-quantisation sweep
follows Sec. "System I": the same water box run with the hydrogen and oxygen
bead counts chosen independently, so that the convergence of each observable
can be traced to the quantisation of each species.

This module only schedules runs and summarises what the kernels return
(block means and errors, peak positions); nothing of the path runs here.
"""
from __future__ import annotations

import numpy as np

from .mixts import FP64, MixTS, MixtsError


def block_stats(x, n_blocks=8):
    """Mean and standard error over n_blocks contiguous blocks (axis 0)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // n_blocks * n_blocks
    if n == 0:
        raise ValueError("fewer samples than blocks")
    b = x[:n].reshape(n_blocks, -1, *x.shape[1:]).mean(axis=1)
    return b.mean(axis=0), b.std(axis=0, ddof=1) / np.sqrt(n_blocks)


def first_peak(g, dr, r_min):
    """(position, height) of the largest g(r) value at r >= r_min (bin centres)."""
    k0 = int(round(r_min / dr))
    k = k0 + int(np.argmax(g[k0:]))
    return (k + 0.5) * dr, float(g[k])


def sample(m: MixTS, n_eq, n_samp, every, pairs=(), dr=0.02, nbins=None, n_blocks=8):
    """Equilibrate m for n_eq steps, then take n_samp steps sampling every
    `every`: returns block statistics of KE_cv, Rg2 (per type) and T_beads,
    and g(r) of each type pair in `pairs` over all samples (bins of dr up to
    8 A unless nbins says otherwise)."""
    torch = m.torch
    if nbins is None:
        nbins = int(round(8.0 / dr))
    hist = {k: torch.zeros(nbins, dtype=torch.int64, device=m.device) for k in pairs}
    m.step(n_eq)
    ke, rg, tb = [], [], []
    frames = n_samp // every
    with torch.cuda.stream(m.stream):
        for _ in range(frames):
            m.step(every)
            for (a, b), h in hist.items():
                m.rdf_accumulate(a, b, h, dr)
            e = m.estimators()
            ke.append(e["KE_cv"])
            rg.append(e["Rg2"])
            tb.append(e["T_beads"])
    return {"KE_cv": block_stats(ke, n_blocks), "Rg2": block_stats(rg, n_blocks), "T_beads": block_stats(tb, n_blocks),
            "g": {k: m.rdf_normalise(k[0], k[1], h, frames, dr) for k, h in hist.items()}, "frames": frames}


def rpmd_bead_masses(sysm):
    """Bead masses m_f = m / P_t per type: with them, Newton's equations of the
    beta H_mix convention (potential weighted 1/P_t, springs P_t m/(beta hbar)^2)
    give every centroid the RPMD equation of motion."""
    return np.asarray(sysm.mass_type, dtype=np.float64) / np.asarray(sysm.P_type, dtype=np.float64)


class CentroidVACF:
    """Centroid velocity autocorrelation <v(0).v(t)> of the atoms of one type,
    accumulated on the GPU over every time origin (mixts_vacf_accumulate).
    Call add() after each step of an NVE run (thermostat off, RPMD bead
    masses); result() gives C(L) per atom in (A/fs)^2 for lags of one add()."""

    def __init__(self, m: MixTS, type_t, n_lag, n_atoms):
        torch = m.torch
        self.m, self.t, self.n = m, int(type_t), int(n_atoms)
        self.ring = torch.zeros((int(n_lag), self.n, 3), dtype=torch.float64, device=m.device)
        self.acc = torch.zeros(int(n_lag), dtype=torch.float64, device=m.device)
        self.cnt = torch.zeros(int(n_lag), dtype=torch.int64, device=m.device)

    def add(self):
        self.m.vacf_accumulate(self.t, self.ring, self.acc, self.cnt)

    def result(self):
        acc = self.acc.cpu().numpy()
        cnt = self.cnt.cpu().numpy()
        return acc / np.maximum(cnt, 1) / self.n, cnt


def quantisation_sweep(make_system, combos, dt=0.25, precision=FP64, n_eq=2000, n_samp=2000, every=10,
                       pairs=((0, 0), (0, 1), (1, 1)), dr=0.02, nbins=None, seed=0, device="cuda:0", stream=None,
                       type_names=("O", "H")):
    """Run make_system(P_H, P_O) for every (P_H, P_O) in combos and summarise
    KE_cv per type (mean, error) and the first RDF peak of each pair. The
    neighbour lists get room for a list radius of r_cut + 6 A (bead spreads
    of every bead count); a run that still fails reports its error."""
    out = {}
    for ph, po in combos:
        sysm = make_system(ph, po)
        n_sites = int(sum(1 for t in sysm.type_of_atom if not sysm.pseudo_type[t]))
        cap = int(1.3 * n_sites / sysm.box ** 3 * 4.0 / 3.0 * np.pi * (9.0 + 6.0) ** 3) + 64
        m = MixTS(sysm, T=300.0, dt=dt, tau=100.0, seed=seed, precision=precision, device=device, stream=stream,
                  nlist_cap=cap)
        try:
            res = sample(m, n_eq, n_samp, every, pairs, dr, nbins)
        except MixtsError as err:
            out[f"H{ph}_O{po}"] = {"error": str(err)}
            continue
        finally:
            m.close()
        ke_m, ke_e = res["KE_cv"]
        out[f"H{ph}_O{po}"] = {
            "KE_cv_kcal_mol": {type_names[t]: [float(ke_m[t]), float(ke_e[t])] for t in range(len(type_names))},
            "rdf_first_peak": {f"{type_names[a]}{type_names[b]}": list(first_peak(g, dr, 1.2))
                               for (a, b), g in res["g"].items()},
        }
    return out
