/*
 * mixts.h -- C ABI of the GB300 mixTS-PIMD hot path (arXiv 2411.11988, "MixPI").
 *
 * One system = atoms of n_types types; type t carries P_t beads (a power of
 * two, Sec. "Setup"; every pair of counts then has the integer ratio the
 * sequential Trotter splitting needs, Sec. "MixTS Ring Polymer Hamiltonian").
 * The potential is V_mix of Eq. (mts-hamiltonian): every interaction is
 * evaluated on the finer participant's bead grid, bead b of the finer
 * particle i meeting bead floor(b P_j / P_i) of j, with weight 1/P_i.
 * The dynamics is the split propagator of Sec. "Evaluation" (exact normal-mode
 * free ring polymer between half kicks of V_mix) inside PILE thermostat half
 * steps (Sec. "System I"). Estimators follow Sec. "Output and Analysis".
 *
 * Units: A, fs, amu, e; energies kcal/mol, forces kcal/mol/A, momenta
 * amu A/fs, pseudopotential amplitudes eV.
 *
 * Bead layout of every per-bead array (q, p, f): FP64, [n_beads][3], blocked
 * by type in type-index order; inside the block of type t (P_t beads, N_t
 * atoms) bead b of the atom of within-type rank k is row off_t + b*N_t + k.
 *
 * Ownership: the caller owns q, p, f and the workspace (device memory,
 * e.g. torch tensors). The library owns the host handle and, once a handle
 * steps, one side stream and five events of its own; it calls no
 * cudaMalloc. All device work is ordered on the caller's stream: work that
 * runs beside other work goes to the side stream, forked from the caller's
 * stream and joined back into it (with events) before the call returns.
 *
 * Errors: every entry point returns a mixts_status. Conditions detected on
 * the device (neighbour-list overflow, non-finite or out-of-range forces,
 * list radius beyond what [-2,2]^3 images cover) are latched in a device
 * word and reported by the next synchronising call (mixts_forces with an
 * energy pointer, mixts_estimators, mixts_get_state, mixts_nlist).
 * mixts_last_error gives text for the last failure of a handle.
 */
#ifndef MIXTS_H
#define MIXTS_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

#define MIXTS_MAX_TYPES 16

#if defined(__GNUC__)
#define MIXTS_API __attribute__((visibility("default")))
#else
#define MIXTS_API
#endif

typedef struct mixts_ctx* mixts_handle;

typedef enum {
  MIXTS_OK = 0,
  MIXTS_ERR_ARG = 1,            /* bad argument, NULL pointer, size mismatch */
  MIXTS_ERR_BEADS = 2,          /* a bead count is not a power of two, or a pseudo particle is coarser than a site */
  MIXTS_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  MIXTS_ERR_WORKSPACE = 4,      /* workspace too small or misaligned (256 B) */
  MIXTS_ERR_NLIST_OVERFLOW = 5, /* an owner row outgrew nlist_cap; re-create with a larger cap */
  MIXTS_ERR_TIMEOUT = 6,        /* a bounded device wait expired */
  MIXTS_ERR_NONFINITE = 7,      /* non-finite or out-of-range force/energy */
  MIXTS_ERR_STATE = 8,          /* state blob does not match this handle */
  MIXTS_ERR_BOX = 9             /* list radius >= 2 L: the periodic box is too small */
} mixts_status;

typedef enum { MIXTS_FP64 = 0, MIXTS_FP32_FORCES = 1 } mixts_precision;

/* One system. All arrays are HOST pointers read during mixts_init, except
 * q, p, f which are caller-owned DEVICE arrays used for the handle's life. */
typedef struct {
  int n_atoms, n_types;
  const int* type_of_atom;    /* [n_atoms] */
  const int* mol_of_atom;     /* [n_atoms]; same molecule, zero image: no nonbonded term */
  const int* P_type;          /* [n_types] bead counts, powers of two, <= 1024 */
  const double* mass_type;    /* [n_types] amu, physical mass (sets the spring constant N m/(beta hbar)^2) */
  const double* charge_type;  /* [n_types] e */
  const double* lj_eps;       /* [n_types*n_types] kcal/mol, symmetric */
  const double* lj_sig;       /* [n_types*n_types] A */
  const int* pseudo_type;     /* [n_types] 1: particle meets sites only through the pseudopotential */
  const double* pp_sigma;     /* [n_types] site parameters of V(r) = -k_e q erf(r/sigma)/r + A exp(-r/b) */
  const double* pp_A_eV;      /* [n_types] */
  const double* pp_b;         /* [n_types] */
  int n_bonds;
  const int* bonds;           /* [n_bonds*2] atom indices */
  const double* bond_k;       /* [n_bonds] kcal/mol/A^2, V = k/2 (r - r0)^2 */
  const double* bond_r0;      /* [n_bonds] A */
  int n_angles;
  const int* angles;          /* [n_angles*3] atom indices, vertex in the middle */
  const double* angle_k;      /* [n_angles] kcal/mol/rad^2, V = k/2 (theta - theta0)^2 */
  const double* angle_theta0; /* [n_angles] rad */
  double box;                 /* cubic periodic box edge, A */
  double* q;                  /* DEVICE [n_beads][3] positions (unwrapped ring polymers) */
  double* p;                  /* DEVICE [n_beads][3] momenta */
  double* f;                  /* DEVICE [n_beads][3] forces, written by the library */
  uint64_t seed;              /* Philox key of the thermostat noise */
  const double* bead_mass_type; /* [n_types] amu, fictitious bead mass m_f of the kinetic term p^2/2m_f
                                   (Sec. "Theory" after Eq. rpham: statics do not depend on it);
                                   NULL: m_f = m. m_f = m/P_t gives ring-polymer molecular dynamics
                                   in the beta H convention of Eq. (mts-hamiltonian) */
} mixts_system;

typedef struct {
  double T;            /* K */
  double dt;           /* fs */
  double tau_centroid; /* fs, centroid Langevin time; <= 0: off */
  double pile_lambda;  /* internal modes get friction 2*lambda*omega_k; 0: off */
  double r_cut;        /* A, cutoff of every nonbonded and pseudopotential term */
  double dsf_alpha;    /* 1/A, damping of the damped-shifted-force Coulomb (coulomb = 0) or the
                          Ewald splitting parameter (coulomb = 1) */
  int precision;       /* mixts_precision */
  int nlist_cap;       /* entries per owner row of the neighbour list; 0: automatic */
  int free_ring_substeps; /* free ring polymer evolution (Sec. "Evaluation"): 0 exact in normal modes;
                             n >= 1 velocity Verlet on the springs with n sub-steps of dt/n */
  int coulomb;         /* 0: damped-shifted-force Coulomb on every bead pair of the mixTS map;
                          1: Ewald, the paper's treatment (Sec. "Theory", last paragraph: SPME with
                          centroid electrostatics): real space k_e q q erfc(alpha r)/r on every bead
                          pair within r_cut, reciprocal space on the ring-polymer centroids (direct
                          sum over wave vectors 2 pi n / L with |n| <= ewald_kmax, each centroid's force
                          shared equally by its beads), minus the same-molecule erf(alpha r)/r terms
                          of the centroids, the self energy and a neutralising background */
  int ewald_kmax;      /* coulomb = 1: largest |n| of the reciprocal sum, 1..64 */
} mixts_params;

/* Estimates of the state after the last completed step (or of the current
 * state after mixts_forces). Energies kcal/mol, Rg2 A^2. */
typedef struct {
  double V, V_lj, V_coul, V_bond, V_angle, V_pseudo;
  double KE_beads;   /* sum p^2/2m over beads */
  double E_spring;   /* ring-polymer spring energy of Eq. (mts-hamiltonian-b) */
  double virial;     /* sum over bead-pair terms of r . f */
  double T_beads;    /* K, 2 KE_beads / (3 n_beads k_B) */
  double H_mix;      /* KE_beads + E_spring + V */
  double heat;       /* minus the kinetic energy the thermostat added */
  double H_conserved;/* H_mix + heat */
  double n_evals;    /* nonbonded bead-pair terms inside r_cut (algorithmic count) */
  double n_pseudo_evals;
  double n_lj_evals; /* nonbonded terms among them with a Lennard-Jones part */
  double KE_prim[MIXTS_MAX_TYPES]; /* primitive kinetic estimator per type */
  double KE_cv[MIXTS_MAX_TYPES];   /* centroid-virial kinetic estimator per type */
  double Rg2[MIXTS_MAX_TYPES];     /* mean squared bead distance from the centroid */
  double E_spring_t[MIXTS_MAX_TYPES];
  int64_t step;                    /* completed steps */
} mixts_estimates;

/* Launch shapes of a batched handle (n_sys > 1), chosen by mixts_batch_tune. */
typedef struct {
  double grid_scale;    /* persistent force-kernel CTAs of all members together, in SM-filling grids,
                           shared out by each member's share of the force work */
  int streams;          /* parallel branches of the captured step graph (per-member launches only) */
  int nl_cpl;           /* neighbour-list candidates per lane of one list warp */
  int steps_per_launch; /* steps captured in one graph launch */
  double ms_per_step;   /* measured for this shape (whole batch, one step) */
  int candidates;       /* shapes the tuner timed */
  int persistent;       /* 1: every kernel of a step serves all members in one launch (one launch per
                           phase); 0: per-member kernels on parallel graph branches. Systems with a
                           pseudo particle, a type of more than 64 beads or coulomb = 1 always use 0 */
  int item_lg_terms;    /* FP32 pair sweep: log2 of the bead-pair terms of one work item (tile size) */
} mixts_batch_tuning;

/* Bytes of device workspace mixts_init needs for these systems. */
MIXTS_API size_t mixts_workspace_size(const mixts_system* sys, int n_sys, const mixts_params* prm);

/* Validate, build tables, carve the workspace (256-byte aligned, owned by
 * the caller, must outlive the handle). stream is a cudaStream_t (NULL:
 * legacy default stream). The current CUDA device must hold q, p, f and the
 * workspace. n_sys > 1 makes a batched handle over n_sys independent
 * systems (each with its own q, p, f, seed, box, types and bead counts; one
 * mixts_params for all): mixts_forces, mixts_step, mixts_estimators,
 * mixts_get_state/set_state, mixts_reload and the timing calls then act on
 * every member (arrays of n_sys results, state blobs back to back); the
 * per-system queries (mixts_nlist, mixts_gaussians, mixts_potential_grad)
 * take a member handle from mixts_batch_member. A batched mixts_step of at
 * least steps_per_launch steps runs as CUDA graph launches, each advancing
 * every member by steps_per_launch steps. When every member allows it (no
 * pseudo particle, no type of more than 64 beads, coulomb = 0) each kernel of
 * a step is launched once for all members (a block finds its member from a
 * prefix of the members' block counts); otherwise the members' own kernels
 * run on parallel graph branches. Trajectories are bit-identical to stepping
 * each system alone, with two limits for FP32 forces: members take the
 * gather sweep, which a standalone handle takes below 768 non-pseudo atoms
 * only (from 768 atoms it takes the window sweep, which groups the binary32
 * partial sums differently: agreement then within FP32 rounding), and the
 * work-item size must be the single-system default of 2^11 terms (another
 * size regroups the partial sums as well). */
MIXTS_API mixts_status mixts_init(const mixts_system* sys, int n_sys, const mixts_params* prm, void* workspace,
                        size_t ws_bytes, void* stream, mixts_handle* out);

/* Bead forces of the mixTS potential, Eq. (mts-hamiltonian): F <- -dV_mix/dq
 * at the current q, every pair, bond and angle term on its finer
 * participant's bead grid (Fig. 1 and its discussion give the bead maps) with
 * weight 1/N_max, plus the pseudopotential of Sec. "System II". The
 * neighbour list is rebuilt from q. F is written to sys.f ([n_beads][3]
 * FP64, the bead layout above, caller-owned device memory). If energy_host
 * (host, n_sys doubles) is not NULL it receives V_mix per system and the
 * call synchronises and reports device-side errors; otherwise it is
 * asynchronous and such errors surface at the next synchronising call.
 * Reads the caller's q afresh; the next mixts_step restarts from the
 * caller's q and p. */
MIXTS_API mixts_status mixts_forces(mixts_handle h, double* energy_host);

/* Advance n_steps steps of the split propagator of Sec. "Evaluation"
 * (e^{-dt L} = e^{-dt/2 L_mix} e^{-dt L0_RP} e^{-dt/2 L_mix}: half kicks of
 * V_mix around the exact normal-mode evolution of the free ring polymers of
 * Eq. (mts-hamiltonian-b), each type with its own bead count), inside the
 * two PILE thermostat half steps of Sec. "System I" (OBABO). Asynchronous;
 * n_steps >= 0 (MIXTS_ERR_ARG otherwise). On return (in stream order)
 * sys.q, sys.p and sys.f hold the state after the last step. With timing off
 * and n_steps >= the handle's steps per graph launch (default 10, see
 * mixts_set_graph), whole multiples of it run as replays of one captured
 * CUDA graph (captured on first use on a library-owned stream, launched on
 * the handle's stream) and the remainder as plain launches; the results are
 * bit-identical either way. */
MIXTS_API mixts_status mixts_step(mixts_handle h, int n_steps);

/* Steps per captured graph launch of mixts_step (0: never capture; a
 * batched handle needs >= 1). Drops any graph captured so far. */
MIXTS_API mixts_status mixts_set_graph(mixts_handle h, int steps_per_launch);

/* Synchronise and return the estimates of the last completed step (the
 * per-step output of Sec. "Output and Analysis": potential parts, bead
 * kinetic and spring energy of Eq. (mts-hamiltonian-b), temperature, the
 * primitive and centroid-virial kinetic estimators per type, R_g^2, and the
 * conserved H_mix + thermostat heat). out_host: host, n_sys records.
 * Reports latched device-side errors as its status. */
MIXTS_API mixts_status mixts_estimators(mixts_handle h, mixts_estimates* out_host);

/* Synchronise and copy the neighbour list of the last force evaluation:
 * triplets (owner atom, partner atom, image code (nx+2)*25+(ny+2)*5+(nz+2)),
 * unordered. n_out gets the count; thresh_host (3 doubles, may be NULL) gets
 * d_max, the list radius r_cut + 2 d_max, and the pseudo-list radius.
 * kind 0: nonbonded list, 1: pseudo-particle site list. */
MIXTS_API mixts_status mixts_nlist(mixts_handle h, int kind, int* out3_host, long cap, long* n_out, double* thresh_host);

/* Opaque checkpoint of the whole dynamical state (normal-mode coordinates
 * and momenta of the free ring polymers of Eq. (mts-hamiltonian-b), step
 * counter, thermostat heat): size, save (synchronises; blob_host is host
 * memory of at least mixts_state_size bytes; MIXTS_ERR_STATE before the
 * first step), restore (MIXTS_ERR_STATE for a blob of another system). The
 * thermostat noise is counter-based on the step index, so a restore
 * followed by n steps reproduces the saved run bit for bit. */
MIXTS_API size_t mixts_state_size(mixts_handle h);
MIXTS_API mixts_status mixts_get_state(mixts_handle h, void* blob_host, size_t bytes);
MIXTS_API mixts_status mixts_set_state(mixts_handle h, const void* blob_host, size_t bytes);

/* The caller rewrote q and/or p in place: the next mixts_step re-imports
 * them into normal modes and recomputes the forces first. */
MIXTS_API mixts_status mixts_reload(mixts_handle h);

/* Per-phase device timing with CUDA events on the handle's stream.
 * Phases: 0 neighbour lists, 1 nonbonded pair sweep, 2 bonded terms,
 * 3 pseudopotential, 4 propagation (normal modes, thermostat, kicks),
 * 5 step finalisation, 6 other. mixts_set_timing(h, 1) clears and starts
 * collecting, 0 stops. mixts_get_timing synchronises and returns the summed
 * milliseconds and launch counts per phase, plus the total number of kernels
 * the library has launched since mixts_init (counted with timing on or off). */
#define MIXTS_N_PHASES 7
MIXTS_API mixts_status mixts_set_timing(mixts_handle h, int on);
MIXTS_API mixts_status mixts_get_timing(mixts_handle h, double* ms_host, long long* calls_host,
                                        long long* kernels_host);

/* Test hook: standard normals of the thermostat stream (Philox4x32-10 and
 * the binary32 Box-Muller transform) for dofs [dof0, dof0+n), written to a
 * DEVICE float array on the handle's stream. */
MIXTS_API mixts_status mixts_gaussians(mixts_handle h, uint32_t step, uint32_t stage, uint64_t dof0, long n,
                             float* out_dev);

/* Potential and gradients for the differentiation variant (Eq.
 * mts-hamiltonian with force-field parameters theta; damped-shifted-force
 * Coulomb only: MIXTS_ERR_ARG for a handle made with coulomb = 1). theta (8 doubles, host)
 * = (sigma_a, A_a [eV], b_a, sigma_b, A_b [eV], b_b, q_a, eps_aa) for the
 * site types a = type_a and b = type_b: the pseudopotential parameters of
 * both, the charge of a, and the a-a Lennard-Jones epsilon; every other
 * Lennard-Jones epsilon of a is rescaled by sqrt(eps_aa / eps_aa at init)
 * (Lorentz-Berthelot). Evaluated in FP64 at the caller's current q without
 * changing the handle's parameters. V_host (may be NULL) gets V_mix;
 * dVdq_dev (device [n_beads][3], may be NULL) gets grad_out * dV/dq;
 * dVdtheta_host (8, may be NULL) gets grad_out * dV/dtheta in kcal/mol per
 * unit of theta; with it NULL the adjoint sums over theta are skipped (a
 * potential-only or force-only evaluation). Pair terms are recomputed, not
 * stored. Synchronises; the
 * next mixts_step restarts from the caller's q and p. */
MIXTS_API mixts_status mixts_potential_grad(mixts_handle h, int type_a, int type_b, const double* theta,
                                            double grad_out, double* V_host, double* dVdq_dev,
                                            double* dVdtheta_host);

/* Radial distribution function g_ab(r) of site types a, b (Sec. "Output and
 * Analysis"): ordered pairs of a-atoms and b-atoms (the zero image of a
 * same-molecule pair excluded), every slice of the pair's fine grid with
 * weight 1/max(P_a, P_b), bins [k dr, (k+1) dr), n_bins dr <= r_cut.
 * mixts_rdf_accumulate adds the configuration of the last force evaluation
 * (after mixts_step or mixts_forces) to hist_dev (device, n_bins uint64,
 * caller-owned and zeroed by the caller), asynchronously; each unit is
 * 2^-L of a pair, 2^L the largest site bead count. mixts_rdf_normalise (host
 * arithmetic only) turns a histogram summed over n_frames configurations into
 * g_host[k] = hist_k 2^-L / (n_frames N_a rho_b V_shell,k), with
 * rho_b = (N_b - [a == b]) / L^3. */
#define MIXTS_RDF_MAX_BINS 4096
MIXTS_API mixts_status mixts_rdf_accumulate(mixts_handle h, int type_a, int type_b, double dr, int n_bins,
                                            unsigned long long* hist_dev);
MIXTS_API mixts_status mixts_rdf_normalise(mixts_handle h, int type_a, int type_b, double dr, int n_bins,
                                           long long n_frames, const unsigned long long* hist_host,
                                           double* g_host);

/* Centroid velocity autocorrelation of the atoms of one type, for
 * ring-polymer molecular dynamics correlation functions from NVE trajectories
 * (Sec. "Output and Analysis"; run with the thermostat off, tau_centroid = 0
 * and pile_lambda = 0, and bead masses m_f = m/P_t, with which the dynamics of
 * the beta H_mix convention of Eq. (mts-hamiltonian) give every centroid the
 * RPMD equation of motion). Call after each mixts_step of a fixed number of
 * steps (one lag unit). Each call adds sum_k v_k(now) . v_k(now - L) over the
 * type's atoms to acc_dev[L] and 1 to cnt_dev[L] for every lag L < n_lag
 * with a frame L calls back (v = dq̄/dt, A/fs, the centroid velocity from the
 * mode-space momenta of the last step), then stores the current frame in
 * ring_dev. All three are caller-owned DEVICE arrays, zeroed by the caller
 * before the first call and passed unchanged afterwards: ring_dev n_lag * 3
 * N_t doubles, acc_dev n_lag doubles, cnt_dev n_lag uint64 (cnt_dev[0] =
 * frames so far). C(L) per atom = acc_dev[L] / (cnt_dev[L] N_t).
 * Asynchronous on the handle's stream; deterministic (fixed-order sums).
 * MIXTS_ERR_STATE before the first step. */
MIXTS_API mixts_status mixts_vacf_accumulate(mixts_handle h, int type, int n_lag, double* ring_dev,
                                             double* acc_dev, unsigned long long* cnt_dev);

/* Member i of a batched handle (borrowed; valid until the batch is destroyed). */
MIXTS_API mixts_status mixts_batch_member(mixts_handle h, int i, mixts_handle* member);

/* Autotune the launch shapes of a batched handle: time captured graphs of
 * candidate shapes on the live systems (one launch per phase: force-grid
 * scale x FP32 work-item size, then list candidates per warp; per-member
 * launches: branch count x force-grid scale), keep the fastest, capture
 * steps_per_launch steps with it. The trial steps are undone (state saved and restored), so
 * the trajectory is unchanged. Synchronises. out (may be NULL) gets the shape. */
MIXTS_API mixts_status mixts_batch_tune(mixts_handle h, int steps_per_launch, mixts_batch_tuning* out);

/* Allocation-free force evaluation. The paper has no counterpart; this
 * serves callers that cannot allocate device memory: plugins whose host
 * framework owns all device memory through its own pool (a stray
 * cudaMalloc fails or fragments it), and drivers that forbid device
 * allocation after start-up. It computes F <- -dV_mix/dq at sys->q into
 * sys->f (both caller-owned device arrays) and, if energy_host is not NULL,
 * V. sys->p is not used (a force evaluation touches no momenta) and may be
 * NULL. All device scratch (tables, neighbour lists, accumulators) lives in
 * one static device array of MIXTS_NOALLOC_MAX_BYTES that every GPU loading
 * the library holds until exit; systems needing more return
 * MIXTS_ERR_WORKSPACE. It calls no cudaMalloc or cudaFree. The first call on
 * each device looks up that device's address of the array
 * (cudaGetSymbolAddress) and keeps it for the life of the process, so make
 * that first call before any stream capture; a device reset
 * (cudaDeviceReset) invalidates the kept address, so the entry point must
 * not be called in a process after a reset of that device. Every call
 * reuses the same array and clears what must start at zero; calls that
 * overlap on the GPU (other streams, other host threads) race on it and
 * must be serialised by the caller. The call returns after its work on
 * `stream` has finished, with or without energy_host, and reports device-side
 * failures (MIXTS_ERR_NLIST_OVERFLOW with a nlist_cap too small for the
 * system, MIXTS_ERR_NONFINITE, MIXTS_ERR_BOX) as its status, with the reason
 * on stderr. */
#define MIXTS_NOALLOC_MAX_BYTES (32u << 20)
MIXTS_API mixts_status mixts_forces_noalloc(const mixts_system* sys, const mixts_params* prm, void* stream,
                                            double* energy_host);

/* ALU peak probe for roofline denominators (no counterpart in the paper; it
 * measures the pipe the pair sweeps are bound by). Launches one SM-filling
 * grid of independent fused multiply-add chains, binary64 if fp64 != 0 else
 * binary32, `iters` FMAs per chain, once untimed and once timed with CUDA
 * events on `stream` (a cudaStream_t; synchronises it). flop_out (host) gets
 * the timed launch's flop count (2 per FMA), ms_out (host) its device time.
 * Allocates nothing. */
MIXTS_API mixts_status mixts_alu_probe(int fp64, int iters, void* stream, double* flop_out, double* ms_out);

MIXTS_API void mixts_destroy(mixts_handle h);
MIXTS_API const char* mixts_last_error(mixts_handle h);
MIXTS_API const char* mixts_version(void);

#ifdef __cplusplus
}
#endif
#endif
