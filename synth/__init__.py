"""Seeded synthetic inputs for the mixTS-PIMD hot path.

This module is shared by the CPU oracle's tests and by the CUDA path's
tests/bench. It builds systems (topology, force-field parameters, initial
bead positions and momenta) and holds none of the method's arithmetic: no
potential, force, bead map, normal mode, thermostat or estimator lives here.

Recipe (one reading per item, all seeded through ``numpy.random.default_rng``):

* Flexible water (SPC/Fw-like parameters as the workloads state them:
  harmonic O-H bonds k=1059.2 kcal/mol/A^2, r0=1.012 A, H-O-H angle
  k=75.9 kcal/mol/rad^2, theta0=113.24 deg, qO=-0.82, qH=+0.41,
  O-O LJ eps=0.1554 kcal/mol, sigma=3.1655 A).
* Molecules sit on a simple-cubic grid of ceil(n^(1/3))^3 sites filled in
  x-fastest order, spacing L/ceil(n^(1/3)), one fixed orientation, every atom
  jittered by an isotropic Gaussian of 0.05 A; all beads of an atom start at
  the atom position.
* With an ion, it sits at the box centre and the grid site nearest the centre
  stays empty.
* An electron's beads are drawn around the ion from N(0, (1 A/sqrt 3)^2) per
  dimension (RMS radius 1 A).
* Bead momenta are Maxwell-Boltzmann per bead degree of freedom,
  N(0, m k_B T) in amu A/fs (the bead kinetic term of the ring-polymer
  Hamiltonian is p^2/2m, sampled at temperature T).

Bead layout shared by every consumer: a flat ``[n_beads, 3]`` float64 array,
blocked by type in type-index order; inside the block of type t (P_t beads,
N_t atoms) bead b of the atom of within-type rank k sits at row
``off_t + b*N_t + k``.
"""
from .systems import (  # noqa: F401
    System,
    water_box,
    harmonic_tether,
    bead_counts_table,
    density_box_length,
    batched_draws,
)
