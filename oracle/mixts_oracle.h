/*
 * mixts_oracle.h -- plain FP64 CPU oracle of the mixTS-PIMD hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library. The product path
 * (the CUDA library) shares no code with it and never calls it.
 *
 * Units: positions A, masses amu, time fs, momenta amu A/fs, potential
 * energies kcal/mol, forces kcal/mol/A, pseudopotential amplitudes eV.
 * Bead layout: flat [n_beads][3] doubles, blocked by type; bead b of the atom
 * of within-type rank k of type t sits at row off_t + b*N_t + k.
 *
 * What each function follows (sections/equations of arXiv 2411.11988):
 *  - or_pair_map / or_triple_map: the bead index maps of Eq. (mts-hamiltonian),
 *    written verbatim with 1-based alpha/gamma/lambda loops.
 *  - or_forces: V_mix of Eq. (mts-hamiltonian) with brute-force lattice
 *    image sums, and its analytic gradient.
 *  - or_step: the split propagator of Sec. "Evaluation" (exact free ring
 *    polymer in normal modes between half kicks), wrapped in PILE
 *    thermostat half steps (Sec. "System I", PILE).
 *  - or_estimators: per-step energies, kinetic estimators and temperature
 *    (Sec. "Output and Analysis").
 *  - or_nlist: the integer neighbour-list definition the GPU path must match.
 *  - Philox4x32-10 is Salmon et al., SC'11; the Gaussian transform is
 *    Box-Muller in binary32 with a series logarithm and series sin/cos.
 */
#ifndef MIXTS_ORACLE_H
#define MIXTS_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int n_atoms, n_types;
  const int* type_of_atom;   /* [n_atoms] */
  const int* mol_of_atom;    /* [n_atoms] */
  const int* P_type;         /* [n_types] bead counts, powers of two */
  const double* mass_type;   /* [n_types] amu */
  const double* charge_type; /* [n_types] e */
  const double* lj_eps;      /* [n_types*n_types] kcal/mol */
  const double* lj_sig;      /* [n_types*n_types] A */
  const int* pseudo_type;    /* [n_types] 1: interacts with sites only via the pseudopotential */
  const double* pp_sigma;    /* [n_types] A, site parameter */
  const double* pp_A_eV;     /* [n_types] eV, site parameter */
  const double* pp_b;        /* [n_types] A, site parameter */
  int n_bonds;
  const int* bonds;          /* [n_bonds*2] */
  const double* bond_k;      /* kcal/mol/A^2, V = k/2 (r-r0)^2 */
  const double* bond_r0;     /* A */
  int n_angles;
  const int* angles;         /* [n_angles*3], vertex in the middle */
  const double* angle_k;     /* kcal/mol/rad^2, V = k/2 (theta-theta0)^2 */
  const double* angle_theta0;/* rad */
  double box, r_cut, dsf_alpha;
  const double* bead_mass_type; /* [n_types] fictitious bead mass m_f (amu) of the kinetic term
                                   p^2/2m_f (Sec. "Theory", Eq. rpham); NULL: m_f = m */
  int coulomb;                  /* 0: damped shifted force (dsf_alpha) on every bead pair;
                                   1: Ewald with splitting dsf_alpha: real space erfc(alpha r)/r on every
                                   bead pair within r_cut, reciprocal space on the ring-polymer centroids
                                   (Sec. "Theory", last paragraph: SPME with centroid electrostatics) */
  int ewald_kmax;               /* reciprocal vectors k = 2 pi n / L with n integer, |n|^2 <= kmax^2 */
} or_system;

typedef struct {
  double T;            /* K */
  double dt;           /* fs */
  double tau_centroid; /* fs; <= 0 switches the centroid friction off */
  double pile_lambda;  /* gamma_k = 2 lambda omega_k for k > 0; 0 switches it off */
  uint64_t seed;
  int vv_substeps;     /* free ring polymer: 0 exact normal-mode evolution; n >= 1 velocity
                          Verlet on the springs with n sub-steps of dt/n (Sec. "Evaluation") */
} or_params;

/* constants in internal units: [0]=kB amu A^2/fs^2/K, [1]=hbar amu A^2/fs,
 * [2]=kcal/mol in amu A^2/fs^2, [3]=eV in amu A^2/fs^2, [4]=Coulomb k_e
 * kcal A/(mol e^2), [5]=eV in kcal/mol */
void or_constants(double* out6);

int or_validate_beads(int n_types, const int* P_type);

/* Eq. (mts-hamiltonian) pair map, i the finer particle (Ni >= Nj). Writes
 * Ni pairs (0-based bead of i, 0-based bead of j) and returns the count. */
int or_pair_map(int Ni, int Nj, int* bead_i, int* bead_j);
/* nested three-body map, Ni >= Nj >= Nk; writes Ni triples */
int or_triple_map(int Ni, int Nj, int Nk, int* bead_i, int* bead_j, int* bead_k);

/* V_mix and F = -dV_mix/dq at q. parts[0..9] = V_total, V_lj, V_coul
 * (with coulomb = 1: real space + reciprocal + intramolecular, self and
 * background corrections),
 * V_bond, V_angle, V_pseudo, virial (sum r.f over interacting bead pairs,
 * kcal/mol), n_evals (algorithmic count of nonbonded in-cutoff bead-pair
 * terms), n_pseudo_evals (same for the pseudopotential), 0. */
void or_forces(const or_system* s, const double* q, double* F, double* parts);
/* force on one bead only (sum over all its terms) */
void or_bead_force(const or_system* s, const double* q, int atom, int bead, double* F3);

/* neighbour list: the canonical set of unordered atom pairs with an image,
 * triplets (i, j, image code of n) with i < j and |r_j - r_i + nL| below the
 * list radius; returns the count (or -needed if cap is too small).
 * out_thresh[0]=d_max, [1]=threshold r_cut + 2 d_max. */
long or_nlist(const or_system* s, const double* q, long cap, int* out3, double* out_thresh);
/* pseudo-particle site list: (pseudo atom, site atom, image code).
 * out_thresh[0]=d_max sites, [1]=d_max pseudo, [2]=threshold */
long or_pseudo_list(const or_system* s, const double* q, long cap, int* out3, double* out_thresh);

/* orthonormal real normal-mode matrix C[j*P+k] and frequencies omega_k (1/fs)
 * of the free ring polymer with bead mass equal to the physical mass; with a
 * bead mass m_f they scale by sqrt(m / m_f) */
void or_nm_matrix(int P, double* C);
void or_nm_freqs(int P, double beta_hbar, double* omega);

/* one O(dt/2) B(dt/2) A(dt) B(dt/2) O(dt/2) step in place; F holds the
 * forces at q on entry and at the new q on exit. heat accumulates minus the
 * kinetic-energy change made by the two thermostat half steps (kcal/mol).
 * Momenta are p = m_f dq/dt with the bead mass m_f. */
void or_step(const or_system* s, const or_params* prm, double* q, double* p, double* F,
             uint64_t step, double* heat, double* parts);

/* estimators; out has 16 + 4*n_types doubles:
 * [0] V_total [1] V_lj [2] V_coul [3] V_bond [4] V_angle [5] V_pseudo
 * [6] KE_beads [7] E_spring [8] virial [9] T_beads (K) [10] H_mix
 * [11] n_evals [12] n_pseudo_evals; then per type t at 16+4t:
 * KE_prim, KE_cv, Rg2 (A^2), E_spring_t (all energies kcal/mol) */
void or_estimators(const or_system* s, const or_params* prm, const double* q, const double* p,
                   const double* F, const double* parts, double* out);

/* dV_mix/dtheta, theta = (sigma_a, A_a [eV], b_a, sigma_b, A_b [eV], b_b,
 * q_a, eps_aa) for site types a = ta, b = tb; the cross Lennard-Jones terms
 * of a scale as eps_ax = eps_ax0 sqrt(eps_aa / eps_aa0) (Lorentz-Berthelot),
 * and are held fixed when eps_aa0 = 0. Units kcal/mol per unit of theta. */
void or_grad_theta(const or_system* s, const double* q, int ta, int tb, double* dVdtheta8);

/* Weighted pair-distance histogram of the radial distribution function of
 * site types ta, tb (ordered pairs; bins of width dr from 0). */
void or_rdf(const or_system* s, const double* q, int ta, int tb, double dr, int nbins, double* hist);

/* Philox4x32-10 */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* standard normals of the thermostat stream for dofs [dof0, dof0+n) */
void or_gaussians(uint64_t seed, uint32_t step, uint32_t stage, uint64_t dof0, long n, float* out);
/* the binary32 building blocks of the transform, exposed for pinning */
float or_log_u24(uint32_t r);
void or_sincos_2pi(uint32_t r, float* s, float* c);

#ifdef __cplusplus
}
#endif
#endif
