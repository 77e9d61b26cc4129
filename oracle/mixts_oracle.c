/*
 * mixts_oracle.c -- plain FP64 CPU oracle of the mixTS-PIMD hot path.
 *
 * TEST INFRASTRUCTURE: only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this. It is deliberately slow and literal:
 * no neighbour list in the potential, brute-force lattice image sums, dense
 * normal-mode matrices, one Philox call per random number.
 * Compile with -ffp-contract=off (the neighbour-list decisions and the
 * binary32 Gaussian transform are specified operation by operation).
 *
 * Paper: arXiv 2411.11988 (MixPI). Equations cited by their LaTeX labels.
 */
#include "mixts_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXT 16
#define OR_PI 3.14159265358979323846

typedef struct {
  double kB, hbar, kcal, ev, ke, ev_kcal;
} cst_t;

typedef struct {
  int nt;
  int N[OR_MAXT];
  long off[OR_MAXT + 1];
  int* rank;
} lay_t;

void or_constants(double* o) {
  /* exact SI values (2019 redefinition) and CODATA-2018 epsilon_0 */
  const double h = 6.62607015e-34, e = 1.602176634e-19, kB = 1.380649e-23, NA = 6.02214076e23;
  const double eps0 = 8.8541878128e-12;
  /* 1 amu = 1e-3/N_A kg, so 1 amu A^2 fs^-2 = 1e7/N_A J */
  const double E_md = 1.0e7 / NA;
  o[0] = kB / E_md;
  o[1] = h / (2.0 * OR_PI) / (E_md * 1.0e-15);
  o[2] = (4184.0 / NA) / E_md;
  o[3] = e / E_md;
  o[4] = e * e / (4.0 * OR_PI * eps0) / 1.0e-10 * NA / 4184.0;
  o[5] = e * NA / 4184.0;
}

static cst_t get_cst(void) {
  double o[6];
  or_constants(o);
  cst_t c = {o[0], o[1], o[2], o[3], o[4], o[5]};
  return c;
}

static int is_pow2(int x) { return x >= 1 && (x & (x - 1)) == 0; }

/* Bead counts must be powers of two (Sec. "Setup"), which makes every pair of
 * counts an integer ratio as the sequential Trotter splitting requires. */
int or_validate_beads(int n_types, const int* P) {
  for (int t = 0; t < n_types; ++t)
    if (!is_pow2(P[t])) return 1;
  return 0;
}

static void lay_init(const or_system* s, lay_t* L) {
  L->nt = s->n_types;
  for (int t = 0; t < s->n_types; ++t) L->N[t] = 0;
  L->rank = (int*)malloc(sizeof(int) * (size_t)(s->n_atoms > 0 ? s->n_atoms : 1));
  for (int a = 0; a < s->n_atoms; ++a) L->rank[a] = L->N[s->type_of_atom[a]]++;
  L->off[0] = 0;
  for (int t = 0; t < s->n_types; ++t) L->off[t + 1] = L->off[t] + (long)L->N[t] * s->P_type[t];
}
static void lay_free(lay_t* L) { free(L->rank); }

/* fictitious bead mass of type t (the kinetic term p^2/2m_f of Eq. rpham) */
static double bead_mass(const or_system* s, int t) {
  return s->bead_mass_type ? s->bead_mass_type[t] : s->mass_type[t];
}

static long row_of(const or_system* s, const lay_t* L, int a, int b) {
  int t = s->type_of_atom[a];
  return L->off[t] + (long)b * L->N[t] + L->rank[a];
}

/* ---------------------------------------------------------------------------
 * Bead index maps of Eq. (mts-hamiltonian), verbatim: the pair term of
 * particles i, j with N_i >= N_j is
 *   (1/N_i) sum_{gamma=1}^{N_i/N_j} sum_{alpha=1}^{N_j}
 *           V_ij(q_{i,(alpha-1)N_i/N_j+gamma}, q_{j,alpha})
 * and the three-body term with N_i >= N_j >= N_k is
 *   (1/N_i) sum_{gamma} sum_{alpha=1}^{N_k} sum_{lambda=1}^{N_j/N_k}
 *     V_ijk(q_{i,((alpha-1)N_j/N_k+lambda-1)N_i/N_j+gamma},
 *           q_{j,(alpha-1)N_j/N_k+lambda}, q_{k,alpha}).
 * ------------------------------------------------------------------------- */
int or_pair_map(int Ni, int Nj, int* bi, int* bj) {
  int n = 0, r = Ni / Nj;
  for (int gamma = 1; gamma <= r; ++gamma)
    for (int alpha = 1; alpha <= Nj; ++alpha) {
      bi[n] = (alpha - 1) * r + gamma - 1;
      bj[n] = alpha - 1;
      ++n;
    }
  return n;
}

int or_triple_map(int Ni, int Nj, int Nk, int* bi, int* bj, int* bk) {
  int n = 0, rij = Ni / Nj, rjk = Nj / Nk;
  for (int gamma = 1; gamma <= rij; ++gamma)
    for (int alpha = 1; alpha <= Nk; ++alpha)
      for (int lambda = 1; lambda <= rjk; ++lambda) {
        bi[n] = ((alpha - 1) * rjk + lambda - 1) * rij + gamma - 1;
        bj[n] = (alpha - 1) * rjk + lambda - 1;
        bk[n] = alpha - 1;
        ++n;
      }
  return n;
}

/* ---------------------------------------------------------------------------
 * Pair functions (all truncated at r_cut and shifted so that value and
 * derivative vanish there).
 * ------------------------------------------------------------------------- */
typedef struct {
  double v_lj, v_c, dv; /* value parts and dV/dr */
} pairval_t;

/* Lennard-Jones 4 eps[(s/r)^12-(s/r)^6], shifted force */
static void lj_raw(double eps, double sig, double r, double* v, double* dv) {
  double sr = sig / r;
  double sr6 = sr * sr * sr * sr * sr * sr;
  double sr12 = sr6 * sr6;
  *v = 4.0 * eps * (sr12 - sr6);
  *dv = -24.0 * eps * (2.0 * sr12 - sr6) / r;
}

/* damped shifted-force Coulomb (Fennell & Gezelter 2006) for unit k_e q q */
static void dsf_raw(double alpha, double rc, double r, double* v, double* dv) {
  double erfc_rc = erfc(alpha * rc);
  double g = 2.0 * alpha / sqrt(OR_PI);
  double cf = erfc_rc / (rc * rc) + g * exp(-alpha * alpha * rc * rc) / rc;
  *v = erfc(alpha * r) / r - erfc_rc / rc + cf * (r - rc);
  *dv = -erfc(alpha * r) / (r * r) - g * exp(-alpha * alpha * r * r) / r + cf;
}

static pairval_t nb_pair(const or_system* s, const cst_t* c, int ti, int tj, double r) {
  pairval_t o = {0.0, 0.0, 0.0};
  int nt = s->n_types;
  double eps = s->lj_eps[ti * nt + tj], sig = s->lj_sig[ti * nt + tj];
  double rc = s->r_cut;
  if (eps != 0.0) {
    double v, dv, vc, dvc;
    lj_raw(eps, sig, r, &v, &dv);
    lj_raw(eps, sig, rc, &vc, &dvc);
    o.v_lj = v - vc - (r - rc) * dvc;
    o.dv += dv - dvc;
  }
  double qq = c->ke * s->charge_type[ti] * s->charge_type[tj];
  if (qq != 0.0) {
    double v, dv;
    if (s->coulomb == 1) { /* Ewald real space, truncated at r_cut */
      double a = s->dsf_alpha;
      v = erfc(a * r) / r;
      dv = -erfc(a * r) / (r * r) - 2.0 * a / sqrt(OR_PI) * exp(-a * a * r * r) / r;
    } else {
      dsf_raw(s->dsf_alpha, rc, r, &v, &dv);
    }
    o.v_c = qq * v;
    o.dv += qq * dv;
  }
  return o;
}

/* electron-site pseudopotential V(r) = -k_e q_c erf(r/sigma)/r + A exp(-r/b) */
static void pseudo_raw(const or_system* s, const cst_t* c, int tc, double r, double* v, double* dv) {
  double sig = s->pp_sigma[tc], A = s->pp_A_eV[tc] * c->ev_kcal, b = s->pp_b[tc];
  double kq = c->ke * s->charge_type[tc];
  double x = r / sig;
  double g, dg; /* g = erf(r/sig)/r, dg = dg/dr */
  if (x < 1.0e-3) {
    double x2 = x * x;
    g = (2.0 / sqrt(OR_PI)) / sig * (1.0 - x2 / 3.0 + x2 * x2 / 10.0);
    dg = (2.0 / sqrt(OR_PI)) / (sig * sig) * (-2.0 * x / 3.0 + 0.4 * x2 * x);
  } else {
    g = erf(x) / r;
    dg = (2.0 / sqrt(OR_PI)) * exp(-x * x) / (sig * r) - erf(x) / (r * r);
  }
  *v = -kq * g + A * exp(-r / b);
  *dv = -kq * dg - (A / b) * exp(-r / b);
}

static void pseudo_pair(const or_system* s, const cst_t* c, int tc, double r, double* v, double* dv) {
  double vr, dvr, vc, dvc;
  double rc = s->r_cut;
  pseudo_raw(s, c, tc, r, &vr, &dvr);
  pseudo_raw(s, c, tc, rc, &vc, &dvc);
  *v = vr - vc - (r - rc) * dvc;
  *dv = dvr - dvc;
}

/* ---------------------------------------------------------------------------
 * V_mix and forces.
 * ------------------------------------------------------------------------- */
typedef struct {
  double v_lj, v_c, v_bond, v_angle, v_pseudo, virial;
  double n_nb, n_pp;
} acc_t;

/* sum over lattice images of one bead pair: x (bead of i), y (bead of j).
 * kind 0: nonbonded, kind 1: pseudopotential with site type tc.
 * Adds w*V and the forces on both beads. Images: every n with
 * |y - x + nL| < r_cut; the search window is n0 + [-2,2]^3 around the
 * nearest image n0, complete while r_cut < 1.5 L. */
static void image_sum(const or_system* s, const cst_t* c, int kind, int ti, int tj, int same_mol,
                      const double* x, const double* y, double w, double* Fx, double* Fy, acc_t* acc) {
  double L = s->box, rc = s->r_cut, rc2 = rc * rc;
  double d0[3];
  int n0[3];
  for (int d = 0; d < 3; ++d) {
    d0[d] = y[d] - x[d];
    n0[d] = -(int)nearbyint(d0[d] / L);
  }
  for (int ix = -2; ix <= 2; ++ix) {
    double dx = d0[0] + (n0[0] + ix) * L;
    if (fabs(dx) >= rc) continue;
    for (int iy = -2; iy <= 2; ++iy) {
      double dy = d0[1] + (n0[1] + iy) * L;
      if (fabs(dy) >= rc) continue;
      for (int iz = -2; iz <= 2; ++iz) {
        double dz = d0[2] + (n0[2] + iz) * L;
        if (fabs(dz) >= rc) continue;
        if (same_mol && n0[0] + ix == 0 && n0[1] + iy == 0 && n0[2] + iz == 0) continue;
        double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= rc2) continue;
        double r = sqrt(r2);
        double dv;
        if (kind == 0) {
          pairval_t pv = nb_pair(s, c, ti, tj, r);
          acc->v_lj += w * pv.v_lj;
          acc->v_c += w * pv.v_c;
          dv = pv.dv;
          acc->n_nb += 1.0;
        } else {
          double v;
          pseudo_pair(s, c, tj, r, &v, &dv);
          acc->v_pseudo += w * v;
          acc->n_pp += 1.0;
        }
        /* force on y: -dV/dr * d/r */
        double f = -w * dv / r;
        double fv[3] = {f * dx, f * dy, f * dz};
        for (int d = 0; d < 3; ++d) {
          if (Fy) Fy[d] += fv[d];
          if (Fx) Fx[d] -= fv[d];
        }
        acc->virial += -w * dv * r;
      }
    }
  }
}

/* harmonic bond between two beads (no images: ring polymers are unwrapped) */
static void bond_term(double k, double r0, const double* x, const double* y, double w, double* Fx,
                      double* Fy, acc_t* acc) {
  double d[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
  double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  acc->v_bond += w * 0.5 * k * (r - r0) * (r - r0);
  double f = -w * k * (r - r0) / r;
  for (int a = 0; a < 3; ++a) {
    if (Fy) Fy[a] += f * d[a];
    if (Fx) Fx[a] -= f * d[a];
  }
  acc->virial += f * r * r;
}

/* harmonic angle at vertex o between arms to x1 and x2 */
static void angle_term(double k, double th0, const double* x1, const double* xo, const double* x2,
                       double w, double* F1, double* Fo, double* F2, acc_t* acc) {
  double u[3], v[3];
  for (int d = 0; d < 3; ++d) {
    u[d] = x1[d] - xo[d];
    v[d] = x2[d] - xo[d];
  }
  double uu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  double vv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double cs = (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) / (uu * vv);
  if (cs > 1.0) cs = 1.0;
  if (cs < -1.0) cs = -1.0;
  double th = acos(cs);
  double sn = sqrt(1.0 - cs * cs);
  acc->v_angle += w * 0.5 * k * (th - th0) * (th - th0);
  /* F_1 = -dV/du = k (th-th0)/sin(th) * (v/(|u||v|) - cos(th) u/|u|^2) */
  double pref = w * k * (th - th0) / sn;
  double f1[3], f2[3];
  for (int d = 0; d < 3; ++d) {
    f1[d] = pref * (v[d] / (uu * vv) - cs * u[d] / (uu * uu));
    f2[d] = pref * (u[d] / (uu * vv) - cs * v[d] / (vv * vv));
  }
  for (int d = 0; d < 3; ++d) {
    if (F1) F1[d] += f1[d];
    if (F2) F2[d] += f2[d];
    if (Fo) Fo[d] -= f1[d] + f2[d];
  }
  acc->virial += f1[0] * u[0] + f1[1] * u[1] + f1[2] * u[2] + f2[0] * v[0] + f2[1] * v[1] + f2[2] * v[2];
}

/* evaluate every term of the pair (a, c) through the pair map; if only_row
 * >= 0, forces are accumulated only into that bead row. kind: 0 nonbonded,
 * 1 pseudopotential (a pseudo), 2 bond index `bond` */
static void pair_terms(const or_system* s, const lay_t* L, const cst_t* c, int kind, int a, int cc,
                       int bond, const double* q, double* F, long only_row, acc_t* acc) {
  int ta = s->type_of_atom[a], tc = s->type_of_atom[cc];
  int i = a, j = cc;
  if (s->P_type[tc] > s->P_type[ta]) {
    i = cc;
    j = a;
  }
  int Ni = s->P_type[s->type_of_atom[i]], Nj = s->P_type[s->type_of_atom[j]];
  int* bi = (int*)malloc(sizeof(int) * (size_t)Ni);
  int* bj = (int*)malloc(sizeof(int) * (size_t)Ni);
  int n = or_pair_map(Ni, Nj, bi, bj);
  double w = 1.0 / Ni;
  for (int m = 0; m < n; ++m) {
    long ri = row_of(s, L, i, bi[m]), rj = row_of(s, L, j, bj[m]);
    double* Fi = F ? F + 3 * ri : NULL;
    double* Fj = F ? F + 3 * rj : NULL;
    if (only_row >= 0) {
      if (ri != only_row) Fi = NULL;
      if (rj != only_row) Fj = NULL;
      if (!Fi && !Fj) continue;
    }
    if (kind == 0) {
      int same = s->mol_of_atom[i] == s->mol_of_atom[j];
      image_sum(s, c, 0, s->type_of_atom[i], s->type_of_atom[j], same, q + 3 * ri, q + 3 * rj, w, Fi, Fj, acc);
    } else if (kind == 1) {
      /* pseudo particle is a, site cc; order the image sum as (pseudo, site) */
      long rp = (i == a) ? ri : rj, rs = (i == a) ? rj : ri;
      double* Fp = (i == a) ? Fi : Fj;
      double* Fs = (i == a) ? Fj : Fi;
      image_sum(s, c, 1, ta, tc, 0, q + 3 * rp, q + 3 * rs, w, Fp, Fs, acc);
    } else {
      bond_term(s->bond_k[bond], s->bond_r0[bond], q + 3 * ri, q + 3 * rj, w, Fi, Fj, acc);
    }
  }
  free(bi);
  free(bj);
}

static void angle_terms(const or_system* s, const lay_t* L, int ang, const double* q, double* F,
                        long only_row, acc_t* acc) {
  int role[3] = {s->angles[3 * ang], s->angles[3 * ang + 1], s->angles[3 * ang + 2]};
  /* order the three particles by descending bead count (stable) */
  int ord[3] = {0, 1, 2};
  for (int x = 0; x < 3; ++x)
    for (int y = 0; y < 2 - x; ++y) {
      int Py = s->P_type[s->type_of_atom[role[ord[y]]]];
      int Py1 = s->P_type[s->type_of_atom[role[ord[y + 1]]]];
      if (Py1 > Py) {
        int t = ord[y];
        ord[y] = ord[y + 1];
        ord[y + 1] = t;
      }
    }
  int Ni = s->P_type[s->type_of_atom[role[ord[0]]]];
  int Nj = s->P_type[s->type_of_atom[role[ord[1]]]];
  int Nk = s->P_type[s->type_of_atom[role[ord[2]]]];
  int* b0 = (int*)malloc(sizeof(int) * (size_t)Ni);
  int* b1 = (int*)malloc(sizeof(int) * (size_t)Ni);
  int* b2 = (int*)malloc(sizeof(int) * (size_t)Ni);
  int n = or_triple_map(Ni, Nj, Nk, b0, b1, b2);
  double w = 1.0 / Ni;
  for (int m = 0; m < n; ++m) {
    int bead_of_role[3];
    bead_of_role[ord[0]] = b0[m];
    bead_of_role[ord[1]] = b1[m];
    bead_of_role[ord[2]] = b2[m];
    long r[3];
    double* Fr[3];
    int any = 0;
    for (int x = 0; x < 3; ++x) {
      r[x] = row_of(s, L, role[x], bead_of_role[x]);
      Fr[x] = F ? F + 3 * r[x] : NULL;
      if (only_row >= 0 && r[x] != only_row) Fr[x] = NULL;
      if (Fr[x]) any = 1;
    }
    if (only_row >= 0 && !any) continue;
    angle_term(s->angle_k[ang], s->angle_theta0[ang], q + 3 * r[0], q + 3 * r[1], q + 3 * r[2], w, Fr[0],
               Fr[1], Fr[2], acc);
  }
  free(b0);
  free(b1);
  free(b2);
}

/* ---------------------------------------------------------------------------
 * Long-range electrostatics on centroids (coulomb = 1). The paper treats
 * electrostatics with SPME and approximates the bead-bead interactions by
 * centroid-centroid ones (Sec. "Theory", last paragraph). Here the Ewald
 * split keeps the short-range real-space part erfc(alpha r)/r on every bead
 * pair (the mixTS map, in nb_pair) and evaluates the smooth rest on the
 * centroids qbar_a = (1/P_a) sum_b q_{a,b} of the charged sites:
 *   E_rec = (2 pi k_e / V) sum_{k != 0} exp(-k^2/(4 alpha^2)) / k^2 |S(k)|^2,
 *           S(k) = sum_a q_a exp(i k.qbar_a), k = 2 pi n / L, |n| <= kmax
 *   E_intra = - k_e sum_{a<b same molecule} q_a q_b erf(alpha r_ab) / r_ab
 *             (centroids, zero image: the pairs the real-space part excludes)
 *   E_self = - k_e alpha / sqrt(pi) sum_a q_a^2
 *   E_bg = - k_e pi Q^2 / (2 V alpha^2), Q = sum_a q_a (neutralising background)
 * A centroid force F_a acts as F_a / P_a on each bead of a (dqbar/dq_b =
 * 1/P). The virial is minus the derivative of these terms under a uniform
 * dilation of positions and box. Direct sums, no mesh.
 * ------------------------------------------------------------------------- */
static void ewald_centroid(const or_system* s, const lay_t* L, const cst_t* c, const double* q, double* F,
                           long only_row, int only_atom, acc_t* acc) {
  int na = s->n_atoms;
  double Lb = s->box, V = Lb * Lb * Lb, a = s->dsf_alpha, ke = c->ke;
  double* cen = (double*)calloc(3 * (size_t)(na > 0 ? na : 1), sizeof(double));
  double* fc = (double*)calloc(3 * (size_t)(na > 0 ? na : 1), sizeof(double));
  double Q = 0.0, q2sum = 0.0;
  for (int i = 0; i < na; ++i) {
    int t = s->type_of_atom[i];
    if (s->pseudo_type[t]) continue;
    int P = s->P_type[t];
    for (int b = 0; b < P; ++b) {
      long r = row_of(s, L, i, b);
      for (int d = 0; d < 3; ++d) cen[3 * i + d] += q[3 * r + d];
    }
    for (int d = 0; d < 3; ++d) cen[3 * i + d] /= P;
    Q += s->charge_type[t];
    q2sum += s->charge_type[t] * s->charge_type[t];
  }
  double e = 0.0, w = 0.0;
  int km = s->ewald_kmax;
  for (int nx = -km; nx <= km; ++nx)
    for (int ny = -km; ny <= km; ++ny)
      for (int nz = -km; nz <= km; ++nz) {
        if (nx == 0 && ny == 0 && nz == 0) continue;
        if (nx * nx + ny * ny + nz * nz > km * km) continue;
        double kx = 2.0 * OR_PI * nx / Lb, ky = 2.0 * OR_PI * ny / Lb, kz = 2.0 * OR_PI * nz / Lb;
        double k2 = kx * kx + ky * ky + kz * kz;
        double wk = 2.0 * OR_PI * ke / V * exp(-k2 / (4.0 * a * a)) / k2;
        double sr = 0.0, si = 0.0;
        for (int i = 0; i < na; ++i) {
          int t = s->type_of_atom[i];
          if (s->pseudo_type[t] || s->charge_type[t] == 0.0) continue;
          double ph = kx * cen[3 * i] + ky * cen[3 * i + 1] + kz * cen[3 * i + 2];
          sr += s->charge_type[t] * cos(ph);
          si += s->charge_type[t] * sin(ph);
        }
        double s2 = sr * sr + si * si;
        e += wk * s2;
        w += wk * s2 * (1.0 - k2 / (2.0 * a * a));
        /* F_a = -dE/dqbar_a = 2 wk q_a k (sin(ph) sr - cos(ph) si) */
        for (int i = 0; i < na; ++i) {
          int t = s->type_of_atom[i];
          if (s->pseudo_type[t] || s->charge_type[t] == 0.0) continue;
          double ph = kx * cen[3 * i] + ky * cen[3 * i + 1] + kz * cen[3 * i + 2];
          double g = 2.0 * wk * s->charge_type[t] * (sin(ph) * sr - cos(ph) * si);
          fc[3 * i] += g * kx;
          fc[3 * i + 1] += g * ky;
          fc[3 * i + 2] += g * kz;
        }
      }
  /* intramolecular pairs, on centroids, zero image */
  for (int i = 0; i < na; ++i) {
    int ti = s->type_of_atom[i];
    if (s->pseudo_type[ti] || s->charge_type[ti] == 0.0) continue;
    for (int j = i + 1; j < na; ++j) {
      int tj = s->type_of_atom[j];
      if (s->pseudo_type[tj] || s->charge_type[tj] == 0.0 || s->mol_of_atom[i] != s->mol_of_atom[j]) continue;
      double d[3] = {cen[3 * j] - cen[3 * i], cen[3 * j + 1] - cen[3 * i + 1], cen[3 * j + 2] - cen[3 * i + 2]};
      double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double qq = ke * s->charge_type[ti] * s->charge_type[tj];
      double v = -qq * erf(a * r) / r;
      double dv = -qq * (2.0 * a / sqrt(OR_PI) * exp(-a * a * r * r) / r - erf(a * r) / (r * r));
      e += v;
      w += -dv * r;
      for (int k = 0; k < 3; ++k) {
        fc[3 * j + k] += -dv * d[k] / r;
        fc[3 * i + k] -= -dv * d[k] / r;
      }
    }
  }
  e += -ke * a / sqrt(OR_PI) * q2sum;
  double ebg = -ke * OR_PI * Q * Q / (2.0 * V * a * a);
  e += ebg;
  w += 3.0 * ebg;
  if (only_atom < 0) {
    acc->v_c += e;
    acc->virial += w;
  }
  if (F) {
    for (int i = 0; i < na; ++i) {
      int t = s->type_of_atom[i];
      if (s->pseudo_type[t]) continue;
      if (only_atom >= 0 && i != only_atom) continue;
      int P = s->P_type[t];
      for (int b = 0; b < P; ++b) {
        long r = row_of(s, L, i, b);
        if (only_row >= 0 && r != only_row) continue;
        for (int d = 0; d < 3; ++d) F[3 * r + d] += fc[3 * i + d] / P;
      }
    }
  }
  free(cen);
  free(fc);
}

static void all_terms(const or_system* s, const double* q, double* F, long only_row, int only_atom,
                      double* parts) {
  lay_t L;
  lay_init(s, &L);
  cst_t c = get_cst();
  acc_t acc;
  memset(&acc, 0, sizeof(acc));
  /* nonbonded: every unordered pair of distinct non-pseudo atoms */
  for (int a = 0; a < s->n_atoms; ++a) {
    if (s->pseudo_type[s->type_of_atom[a]]) continue;
    for (int cc = a + 1; cc < s->n_atoms; ++cc) {
      if (s->pseudo_type[s->type_of_atom[cc]]) continue;
      if (only_atom >= 0 && a != only_atom && cc != only_atom) continue;
      pair_terms(s, &L, &c, 0, a, cc, -1, q, F, only_row, &acc);
    }
  }
  /* pseudopotential: every pseudo particle with every site */
  for (int a = 0; a < s->n_atoms; ++a) {
    if (!s->pseudo_type[s->type_of_atom[a]]) continue;
    for (int cc = 0; cc < s->n_atoms; ++cc) {
      if (s->pseudo_type[s->type_of_atom[cc]]) continue;
      if (only_atom >= 0 && a != only_atom && cc != only_atom) continue;
      pair_terms(s, &L, &c, 1, a, cc, -1, q, F, only_row, &acc);
    }
  }
  for (int b = 0; b < s->n_bonds; ++b) {
    int a = s->bonds[2 * b], cc = s->bonds[2 * b + 1];
    if (only_atom >= 0 && a != only_atom && cc != only_atom) continue;
    pair_terms(s, &L, &c, 2, a, cc, b, q, F, only_row, &acc);
  }
  for (int g = 0; g < s->n_angles; ++g) {
    if (only_atom >= 0 && s->angles[3 * g] != only_atom && s->angles[3 * g + 1] != only_atom &&
        s->angles[3 * g + 2] != only_atom)
      continue;
    angle_terms(s, &L, g, q, F, only_row, &acc);
  }
  if (s->coulomb == 1) ewald_centroid(s, &L, &c, q, F, only_row, only_atom, &acc);
  if (parts) {
    parts[1] = acc.v_lj;
    parts[2] = acc.v_c;
    parts[3] = acc.v_bond;
    parts[4] = acc.v_angle;
    parts[5] = acc.v_pseudo;
    parts[0] = acc.v_lj + acc.v_c + acc.v_bond + acc.v_angle + acc.v_pseudo;
    parts[6] = acc.virial;
    parts[7] = acc.n_nb;
    parts[8] = acc.n_pp;
    parts[9] = 0.0;
  }
  lay_free(&L);
}

void or_forces(const or_system* s, const double* q, double* F, double* parts) {
  lay_t L;
  lay_init(s, &L);
  long nb = L.off[s->n_types];
  lay_free(&L);
  if (F) memset(F, 0, sizeof(double) * 3 * (size_t)nb);
  all_terms(s, q, F, -1, -1, parts);
}

void or_bead_force(const or_system* s, const double* q, int atom, int bead, double* F3) {
  lay_t L;
  lay_init(s, &L);
  long nb = L.off[s->n_types];
  long row = row_of(s, &L, atom, bead);
  lay_free(&L);
  double* F = (double*)calloc(3 * (size_t)nb, sizeof(double));
  all_terms(s, q, F, row, atom, NULL);
  F3[0] = F[3 * row];
  F3[1] = F[3 * row + 1];
  F3[2] = F[3 * row + 2];
  free(F);
}

/* ---------------------------------------------------------------------------
 * Neighbour list definition (integer output, matched bit for bit).
 *   r_a = q_{a,0} - L floor(q_{a,0}/L)          wrapped bead-0 reference
 *   d_max = max over non-pseudo beads of |q_{a,b} - q_{a,0}|
 *   R = r_cut + 2 d_max; the list is the set of unordered atom pairs with a
 *   lattice image, written canonically as (i, j, n) with i < j, for which
 *   |(r_j - r_i) + n L|^2 < R^2, n in [-2,2]^3, skipping for a same-molecule
 *   pair the image n = w_j - w_i, w_a = floor(q_{a,0}/L): the zero image of
 *   the unwrapped coordinates, where the intramolecular terms (bonded, not
 *   nonbonded) act. Which atom of a pair a force kernel makes the owner of the entry
 *   is the kernel's business; the set does not depend on it, because every
 *   operation below is odd under swapping i and j with n -> -n.
 * Every product and sum below is one IEEE operation in the order written.
 * ------------------------------------------------------------------------- */
static void wrapped_refs(const or_system* s, const lay_t* L, const double* q, double* ref, int* wrap) {
  double Lb = s->box;
  for (int a = 0; a < s->n_atoms; ++a) {
    long r0 = row_of(s, L, a, 0);
    for (int d = 0; d < 3; ++d) {
      double x = q[3 * r0 + d];
      double fl = floor(x / Lb);
      ref[3 * a + d] = x - Lb * fl;
      if (wrap) wrap[3 * a + d] = (int)fl;
    }
  }
}

static double max_spread(const or_system* s, const lay_t* L, const double* q, int pseudo) {
  double dm = 0.0;
  for (int a = 0; a < s->n_atoms; ++a) {
    int t = s->type_of_atom[a];
    if ((s->pseudo_type[t] != 0) != (pseudo != 0)) continue;
    long r0 = row_of(s, L, a, 0);
    for (int b = 1; b < s->P_type[t]; ++b) {
      long rb = row_of(s, L, a, b);
      double dx = q[3 * rb] - q[3 * r0];
      double dy = q[3 * rb + 1] - q[3 * r0 + 1];
      double dz = q[3 * rb + 2] - q[3 * r0 + 2];
      double d2 = dx * dx;
      d2 = d2 + dy * dy;
      d2 = d2 + dz * dz;
      double dd = sqrt(d2);
      if (dd > dm) dm = dd;
    }
  }
  return dm;
}

static int image_code(int nx, int ny, int nz) { return (nx + 2) * 25 + (ny + 2) * 5 + (nz + 2); }

/* squared length of (r_to - r_from) + n L */
static double disp2(const double* r_to, const double* r_from, int nx, int ny, int nz, double Lb) {
  double dx = (r_to[0] - r_from[0]) + (double)nx * Lb;
  double dy = (r_to[1] - r_from[1]) + (double)ny * Lb;
  double dz = (r_to[2] - r_from[2]) + (double)nz * Lb;
  double d2 = dx * dx;
  d2 = d2 + dy * dy;
  d2 = d2 + dz * dz;
  return d2;
}

long or_nlist(const or_system* s, const double* q, long cap, int* out3, double* out_thresh) {
  lay_t L;
  lay_init(s, &L);
  int na = s->n_atoms;
  double* ref = (double*)malloc(sizeof(double) * 3 * (size_t)na);
  int* wrap = (int*)malloc(sizeof(int) * 3 * (size_t)na);
  wrapped_refs(s, &L, q, ref, wrap);
  double dm = max_spread(s, &L, q, 0);
  double R = s->r_cut + 2.0 * dm;
  double R2 = R * R;
  if (out_thresh) {
    out_thresh[0] = dm;
    out_thresh[1] = R;
  }
  long n = 0;
  for (int i = 0; i < na; ++i) {
    if (s->pseudo_type[s->type_of_atom[i]]) continue;
    for (int j = i + 1; j < na; ++j) {
      if (s->pseudo_type[s->type_of_atom[j]]) continue;
      int same = s->mol_of_atom[i] == s->mol_of_atom[j];
      for (int nx = -2; nx <= 2; ++nx)
        for (int ny = -2; ny <= 2; ++ny)
          for (int nz = -2; nz <= 2; ++nz) {
            if (same && nx == wrap[3 * j] - wrap[3 * i] && ny == wrap[3 * j + 1] - wrap[3 * i + 1] &&
                nz == wrap[3 * j + 2] - wrap[3 * i + 2])
              continue;
            double d2 = disp2(ref + 3 * j, ref + 3 * i, nx, ny, nz, s->box);
            if (d2 < R2) {
              if (n < cap) {
                out3[3 * n] = i;
                out3[3 * n + 1] = j;
                out3[3 * n + 2] = image_code(nx, ny, nz);
              }
              ++n;
            }
          }
    }
  }
  free(ref);
  free(wrap);
  lay_free(&L);
  return n <= cap ? n : -n;
}

long or_pseudo_list(const or_system* s, const double* q, long cap, int* out3, double* out_thresh) {
  lay_t L;
  lay_init(s, &L);
  int na = s->n_atoms;
  double* ref = (double*)malloc(sizeof(double) * 3 * (size_t)na);
  wrapped_refs(s, &L, q, ref, NULL);
  double ds = max_spread(s, &L, q, 0);
  double dp = max_spread(s, &L, q, 1);
  double R = (s->r_cut + ds) + dp;
  double R2 = R * R;
  if (out_thresh) {
    out_thresh[0] = ds;
    out_thresh[1] = dp;
    out_thresh[2] = R;
  }
  long n = 0;
  for (int e = 0; e < na; ++e) {
    if (!s->pseudo_type[s->type_of_atom[e]]) continue;
    for (int c = 0; c < na; ++c) {
      if (s->pseudo_type[s->type_of_atom[c]]) continue;
      for (int nx = -2; nx <= 2; ++nx)
        for (int ny = -2; ny <= 2; ++ny)
          for (int nz = -2; nz <= 2; ++nz) {
            double d2 = disp2(ref + 3 * c, ref + 3 * e, nx, ny, nz, s->box);
            if (d2 < R2) {
              if (n < cap) {
                out3[3 * n] = e;
                out3[3 * n + 1] = c;
                out3[3 * n + 2] = image_code(nx, ny, nz);
              }
              ++n;
            }
          }
    }
  }
  free(ref);
  lay_free(&L);
  return n <= cap ? n : -n;
}

/* ---------------------------------------------------------------------------
 * Normal modes of the free ring polymer H0 of Eq. (mts-hamiltonian-b):
 * spring constant N m/(beta hbar)^2 between neighbouring beads, so mode k has
 * omega_k = 2 sqrt(N)/(beta hbar) sin(pi k/N). C is the orthonormal real
 * transform: column 0 constant, columns 1..N/2-1 cosines, column N/2
 * alternating, columns N/2+1..N-1 sines.  q_nm[k] = sum_j C[j][k] q[j].
 * ------------------------------------------------------------------------- */
void or_nm_matrix(int P, double* C) {
  for (int j = 0; j < P; ++j)
    for (int k = 0; k < P; ++k) {
      double v;
      if (k == 0)
        v = 1.0 / sqrt((double)P);
      else if (2 * k < P)
        v = sqrt(2.0 / P) * cos(2.0 * OR_PI * j * k / P);
      else if (2 * k == P)
        v = ((j % 2) ? -1.0 : 1.0) / sqrt((double)P);
      else
        v = sqrt(2.0 / P) * sin(2.0 * OR_PI * j * k / P);
      C[j * P + k] = v;
    }
}

void or_nm_freqs(int P, double beta_hbar, double* omega) {
  for (int k = 0; k < P; ++k) omega[k] = 2.0 * sqrt((double)P) / beta_hbar * sin(OR_PI * k / P);
}

/* ---------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
 * (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0))
 * with the Weyl key bump between rounds.
 * ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* ln(u) for u = (2 floor(r/2^9) + 1) 2^-24 in binary32: exact split
 * u = f 2^e with f in (sqrt(1/2), sqrt(2)], then the atanh series
 * ln f = 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9), s = (f-1)/(f+1), and
 * e ln 2 added as a two-part (Cody-Waite) constant. */
float or_log_u24(uint32_t r) {
  uint32_t m = ((r >> 9) << 1) | 1u;
  int e = 0;
  while ((m >> (e + 1)) != 0u) ++e;
  uint32_t sbits = (uint32_t)(127 - e) << 23;
  float scale;
  memcpy(&scale, &sbits, 4);
  float f = (float)m * scale;
  if (f > 0x1.6a09e6p+0f) {
    f = f * 0.5f;
    e += 1;
  }
  float s = (f - 1.0f) / (f + 1.0f);
  float s2 = s * s;
  float poly = 0x1.c71c72p-4f;
  poly = fmaf(poly, s2, 0x1.24924ap-3f);
  poly = fmaf(poly, s2, 0x1.99999ap-3f);
  poly = fmaf(poly, s2, 0x1.555556p-2f);
  float s3 = s * s2;
  float lnf = fmaf(s3, poly, s);
  lnf = 2.0f * lnf;
  float k = (float)(e - 24);
  return fmaf(k, 0x1.62e4p-1f, fmaf(k, 0x1.7f7d1cp-20f, lnf));
}

/* sin and cos of 2 pi v, v from the top 25 bits of r: quadrant from the two
 * top bits, the in-quadrant angle folded to (0, pi/4] and Taylor series
 * (through x^9 for sin, x^10 for cos) evaluated by Horner with fma. */
void or_sincos_2pi(uint32_t r, float* sp, float* cp) {
  uint32_t quad = r >> 30;
  uint32_t m = (((r >> 7) & 0x7FFFFFu) << 1) | 1u;
  int comp = m > (1u << 23);
  if (comp) m = (1u << 24) - m;
  float t = (float)m * 0x1p-24f;
  float x = t * 0x1.921fb6p+0f;
  float x2 = x * x;
  float ps = 0x1.71de3ap-19f;
  ps = fmaf(ps, x2, -0x1.a01a02p-13f);
  ps = fmaf(ps, x2, 0x1.111112p-7f);
  ps = fmaf(ps, x2, -0x1.555556p-3f);
  float x3 = x * x2;
  float sn = fmaf(x3, ps, x);
  float pc = -0x1.27e4fcp-22f;
  pc = fmaf(pc, x2, 0x1.a01a02p-16f);
  pc = fmaf(pc, x2, -0x1.6c16c2p-10f);
  pc = fmaf(pc, x2, 0x1.555556p-5f);
  pc = fmaf(pc, x2, -0x1p-1f);
  float cs = fmaf(x2, pc, 1.0f);
  if (comp) {
    float tmp = sn;
    sn = cs;
    cs = tmp;
  }
  switch (quad) {
    case 0: *sp = sn; *cp = cs; break;
    case 1: *sp = cs; *cp = -sn; break;
    case 2: *sp = -sn; *cp = -cs; break;
    default: *sp = -cs; *cp = sn; break;
  }
}

/* standard normal for one degree of freedom of the thermostat stream:
 * key = (seed lo, seed hi), counter = (step, stage, group lo, group hi),
 * group = dof/4; lanes 0,1 use Box-Muller on outputs (0,1), lanes 2,3 on
 * outputs (2,3); even lanes take the cosine, odd lanes the sine. */
static float gauss_one(uint64_t seed, uint32_t step, uint32_t stage, uint64_t dof) {
  uint64_t g = dof >> 2;
  int lane = (int)(dof & 3u);
  uint32_t ctr[4] = {step, stage, (uint32_t)g, (uint32_t)(g >> 32)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  or_philox4x32_10(ctr, key, o);
  int pr = lane >> 1;
  float lg = or_log_u24(o[2 * pr]);
  float rho = sqrtf(-2.0f * lg);
  float sn, cs;
  or_sincos_2pi(o[2 * pr + 1], &sn, &cs);
  return (lane & 1) ? rho * sn : rho * cs;
}

void or_gaussians(uint64_t seed, uint32_t step, uint32_t stage, uint64_t dof0, long n, float* out) {
  for (long i = 0; i < n; ++i) out[i] = gauss_one(seed, step, stage, dof0 + (uint64_t)i);
}

/* ---------------------------------------------------------------------------
 * Integrator: PILE thermostat half steps around the split propagator of
 * Sec. "Evaluation": e^{-dt L} = e^{-dt/2 L_mix} e^{-dt L0_RP} e^{-dt/2 L_mix}.
 * ------------------------------------------------------------------------- */
static void thermostat(const or_system* s, const lay_t* L, const cst_t* c, const or_params* prm,
                       double* p, uint64_t step, uint32_t stage, double* heat) {
  double kT = c->kB * prm->T;
  double bh = c->hbar / kT;
  for (int t = 0; t < s->n_types; ++t) {
    int P = s->P_type[t], N = L->N[t];
    if (N == 0) continue;
    double m = bead_mass(s, t);
    double* C = (double*)malloc(sizeof(double) * (size_t)P * P);
    double* om = (double*)malloc(sizeof(double) * (size_t)P);
    double* v = (double*)malloc(sizeof(double) * (size_t)P);
    double* vn = (double*)malloc(sizeof(double) * (size_t)P);
    or_nm_matrix(P, C);
    or_nm_freqs(P, bh, om);
    /* the modes' frequencies with bead mass m_f: omega_k sqrt(m / m_f) */
    for (int k = 0; k < P; ++k) om[k] *= sqrt(s->mass_type[t] / m);
    for (int k = 0; k < N; ++k)
      for (int d = 0; d < 3; ++d) {
        for (int j = 0; j < P; ++j) v[j] = p[3 * (L->off[t] + (long)j * N + k) + d];
        for (int mm = 0; mm < P; ++mm) {
          double acc = 0.0;
          for (int j = 0; j < P; ++j) acc += C[j * P + mm] * v[j];
          vn[mm] = acc;
        }
        for (int mm = 0; mm < P; ++mm) {
          double gam = (mm == 0) ? (prm->tau_centroid > 0.0 ? 1.0 / prm->tau_centroid : 0.0)
                                 : 2.0 * prm->pile_lambda * om[mm];
          double c1 = exp(-0.5 * prm->dt * gam);
          double c2 = sqrt(1.0 - c1 * c1);
          uint64_t dof = (uint64_t)(3 * (L->off[t] + (long)mm * N + k) + d);
          double xi = (double)gauss_one(prm->seed, (uint32_t)step, stage, dof);
          double pn = c1 * vn[mm] + c2 * sqrt(m * kT) * xi;
          *heat -= (pn * pn - vn[mm] * vn[mm]) / (2.0 * m) / c->kcal;
          vn[mm] = pn;
        }
        for (int j = 0; j < P; ++j) {
          double acc = 0.0;
          for (int mm = 0; mm < P; ++mm) acc += C[j * P + mm] * vn[mm];
          p[3 * (L->off[t] + (long)j * N + k) + d] = acc;
        }
      }
    free(C);
    free(om);
    free(v);
    free(vn);
  }
}

static void kick(const or_system* s, const lay_t* L, const cst_t* c, double h, double* p, const double* F) {
  for (int t = 0; t < s->n_types; ++t)
    for (long r = L->off[t]; r < L->off[t + 1]; ++r)
      for (int d = 0; d < 3; ++d) p[3 * r + d] += h * F[3 * r + d] * c->kcal;
}

/* velocity Verlet on the ring-polymer springs of Eq. (mts-hamiltonian-b),
 * the alternative to the exact normal-mode evolution in Sec. "Evaluation":
 * n sub-steps of h = dt/n, each p += (h/2) f(q), q += h p/m_f,
 * p += (h/2) f(q), with f_b = -kappa (2 q_b - q_{b+1} - q_{b-1}) and
 * kappa = P m/(beta hbar)^2 (ring closure q_P = q_0). One atom, one
 * Cartesian component: P beads in q[], p[]. */
static void free_ring_vv(int P, double kap, double mf, double dt, int n, double* q, double* p, double* f) {
  double h = dt / n;
  for (int j = 0; j < P; ++j) {
    int jp = (j + 1) % P, jm = (j + P - 1) % P;
    f[j] = -kap * (2.0 * q[j] - q[jp] - q[jm]);
  }
  for (int sub = 0; sub < n; ++sub) {
    for (int j = 0; j < P; ++j) p[j] += 0.5 * h * f[j];
    for (int j = 0; j < P; ++j) q[j] += h * p[j] / mf;
    for (int j = 0; j < P; ++j) {
      int jp = (j + 1) % P, jm = (j + P - 1) % P;
      f[j] = -kap * (2.0 * q[j] - q[jp] - q[jm]);
    }
    for (int j = 0; j < P; ++j) p[j] += 0.5 * h * f[j];
  }
}

static void free_ring(const or_system* s, const lay_t* L, const cst_t* c, const or_params* prm, double* q,
                      double* p) {
  double kT = c->kB * prm->T;
  double bh = c->hbar / kT;
  double dt = prm->dt;
  for (int t = 0; t < s->n_types; ++t) {
    int P = s->P_type[t], N = L->N[t];
    if (N == 0) continue;
    double m = bead_mass(s, t);
    double* C = (double*)malloc(sizeof(double) * (size_t)P * P);
    double* om = (double*)malloc(sizeof(double) * (size_t)P);
    double* qv = (double*)malloc(sizeof(double) * (size_t)P);
    double* pv = (double*)malloc(sizeof(double) * (size_t)P);
    double* qn = (double*)malloc(sizeof(double) * (size_t)P);
    double* pn = (double*)malloc(sizeof(double) * (size_t)P);
    or_nm_matrix(P, C);
    or_nm_freqs(P, bh, om);
    for (int k = 0; k < P; ++k) om[k] *= sqrt(s->mass_type[t] / m);
    double kap = P * s->mass_type[t] / (bh * bh);
    for (int k = 0; k < N; ++k)
      for (int d = 0; d < 3; ++d) {
        for (int j = 0; j < P; ++j) {
          qv[j] = q[3 * (L->off[t] + (long)j * N + k) + d];
          pv[j] = p[3 * (L->off[t] + (long)j * N + k) + d];
        }
        if (prm->vv_substeps > 0) {
          free_ring_vv(P, kap, m, dt, prm->vv_substeps, qv, pv, qn);
          for (int j = 0; j < P; ++j) {
            q[3 * (L->off[t] + (long)j * N + k) + d] = qv[j];
            p[3 * (L->off[t] + (long)j * N + k) + d] = pv[j];
          }
          continue;
        }
        for (int mm = 0; mm < P; ++mm) {
          double aq = 0.0, ap = 0.0;
          for (int j = 0; j < P; ++j) {
            aq += C[j * P + mm] * qv[j];
            ap += C[j * P + mm] * pv[j];
          }
          qn[mm] = aq;
          pn[mm] = ap;
        }
        for (int mm = 0; mm < P; ++mm) {
          if (mm == 0) {
            qn[0] += pn[0] * dt / m;
          } else {
            double w = om[mm];
            double cw = cos(w * dt), sw = sin(w * dt);
            double pnew = cw * pn[mm] - m * w * sw * qn[mm];
            double qnew = sw / (m * w) * pn[mm] + cw * qn[mm];
            pn[mm] = pnew;
            qn[mm] = qnew;
          }
        }
        for (int j = 0; j < P; ++j) {
          double aq = 0.0, ap = 0.0;
          for (int mm = 0; mm < P; ++mm) {
            aq += C[j * P + mm] * qn[mm];
            ap += C[j * P + mm] * pn[mm];
          }
          q[3 * (L->off[t] + (long)j * N + k) + d] = aq;
          p[3 * (L->off[t] + (long)j * N + k) + d] = ap;
        }
      }
    free(C);
    free(om);
    free(qv);
    free(pv);
    free(qn);
    free(pn);
  }
}

void or_step(const or_system* s, const or_params* prm, double* q, double* p, double* F, uint64_t step,
             double* heat, double* parts) {
  lay_t L;
  lay_init(s, &L);
  cst_t c = get_cst();
  double h = 0.5 * prm->dt;
  thermostat(s, &L, &c, prm, p, step, 0u, heat);
  kick(s, &L, &c, h, p, F);
  free_ring(s, &L, &c, prm, q, p);
  or_forces(s, q, F, parts);
  kick(s, &L, &c, h, p, F);
  thermostat(s, &L, &c, prm, p, step, 1u, heat);
  lay_free(&L);
}

/* ---------------------------------------------------------------------------
 * Estimators (Sec. "Output and Analysis"): bead kinetic energy, spring
 * energy, temperature, H_mix, and per type the primitive and centroid-virial
 * kinetic energies and the radius of gyration.
 *   KE_prim,t = 3 N_t P_t/(2 beta) - E_spring,t
 *   KE_cv,t   = 3 N_t/(2 beta) - 1/2 sum_a sum_b (q_ab - qbar_a).F_ab
 * ------------------------------------------------------------------------- */
void or_estimators(const or_system* s, const or_params* prm, const double* q, const double* p,
                   const double* F, const double* parts, double* out) {
  lay_t L;
  lay_init(s, &L);
  cst_t c = get_cst();
  double kT = c.kB * prm->T;
  double bh = c.hbar / kT;
  int nt = s->n_types;
  memset(out, 0, sizeof(double) * (size_t)(16 + 4 * nt));
  double ke = 0.0, espr = 0.0;
  long nbeads = L.off[nt];
  for (int t = 0; t < nt; ++t) {
    int P = s->P_type[t], N = L.N[t];
    double m = s->mass_type[t], mf = bead_mass(s, t);
    double kspr = P * m / (bh * bh);
    double et = 0.0, cv = 0.0, rg = 0.0;
    for (long r = L.off[t]; r < L.off[t + 1]; ++r)
      for (int d = 0; d < 3; ++d) ke += p[3 * r + d] * p[3 * r + d] / (2.0 * mf);
    for (int k = 0; k < N; ++k) {
      double cen[3] = {0, 0, 0};
      for (int j = 0; j < P; ++j)
        for (int d = 0; d < 3; ++d) cen[d] += q[3 * (L.off[t] + (long)j * N + k) + d];
      for (int d = 0; d < 3; ++d) cen[d] /= P;
      for (int j = 0; j < P; ++j) {
        long r = L.off[t] + (long)j * N + k;
        long rn = L.off[t] + (long)((j + 1) % P) * N + k;
        for (int d = 0; d < 3; ++d) {
          double dq = q[3 * r + d] - q[3 * rn + d];
          et += 0.5 * kspr * dq * dq;
          double dc = q[3 * r + d] - cen[d];
          cv += dc * F[3 * r + d];
          rg += dc * dc;
        }
      }
    }
    et /= c.kcal;
    espr += et;
    double* o = out + 16 + 4 * t;
    o[0] = 1.5 * N * P * kT / c.kcal - et;
    o[1] = 1.5 * N * kT / c.kcal - 0.5 * cv;
    o[2] = (N > 0) ? rg / ((double)N * P) : 0.0;
    o[3] = et;
  }
  ke /= c.kcal;
  for (int x = 0; x < 6; ++x) out[x] = parts[x];
  out[6] = ke;
  out[7] = espr;
  out[8] = parts[6];
  out[9] = 2.0 * ke * c.kcal / (3.0 * (double)nbeads * c.kB);
  out[10] = ke + espr + parts[0];
  out[11] = parts[7];
  out[12] = parts[8];
  lay_free(&L);
}

/* ---------------------------------------------------------------------------
 * Parameter gradient dV_mix/dtheta, theta = (sigma_a, A_a [eV], b_a,
 * sigma_b, A_b [eV], b_b, q_a, eps_aa) for site types a and b. Charges enter
 * every Coulomb term (DSF, and the pseudopotential's -k_e q erf(r/sigma)/r);
 * eps_aa enters a-a Lennard-Jones directly and every other a-x
 * Lennard-Jones term through eps_ax = sqrt(eps_aa eps_xx) (Lorentz-Berthelot),
 * so d eps_ax / d eps_aa = eps_ax / (2 eps_aa). Each term is differentiated
 * by hand, including the shifted-force corrections at r_cut.
 * ------------------------------------------------------------------------- */
static void dsf_unit(double alpha, double rc, double r, double* v) {
  double dv;
  dsf_raw(alpha, rc, r, v, &dv);
}

/* V, dV/dr of the raw pseudopotential and their derivatives with respect to
 * (sigma, A [kcal/mol], b, q) at distance r */
static void pseudo_param_derivs(double kq_unit, double q, double sig, double A, double b, double r, double dv[4],
                                double ddv[4]) {
  const double sp = sqrt(OR_PI);
  double x = r / sig;
  double ex = exp(-x * x), eb = exp(-r / b);
  double erfx = erf(x);
  /* d/dsigma */
  dv[0] = kq_unit * q * (2.0 / sp) * ex / (sig * sig);
  ddv[0] = -kq_unit * q * (2.0 / sp) * ex * 2.0 * r / (sig * sig * sig * sig);
  /* d/dA */
  dv[1] = eb;
  ddv[1] = -eb / b;
  /* d/db */
  dv[2] = A * eb * r / (b * b);
  ddv[2] = A * eb * (b - r) / (b * b * b);
  /* d/dq */
  dv[3] = -kq_unit * erfx / r;
  ddv[3] = -kq_unit * ((2.0 / (sig * sp)) * ex / r - erfx / (r * r));
}

void or_grad_theta(const or_system* s, const double* q, int ta, int tb, double* g) {
  lay_t L;
  lay_init(s, &L);
  cst_t c = get_cst();
  const double rc = s->r_cut, rc2 = rc * rc, Lb = s->box;
  for (int k = 0; k < 8; ++k) g[k] = 0.0;
  int nt = s->n_types;
  double eaa = s->lj_eps[ta * nt + ta];
  /* nonbonded terms */
  for (int a = 0; a < s->n_atoms; ++a) {
    if (s->pseudo_type[s->type_of_atom[a]]) continue;
    for (int cc = a + 1; cc < s->n_atoms; ++cc) {
      if (s->pseudo_type[s->type_of_atom[cc]]) continue;
      int i = a, j = cc;
      if (s->P_type[s->type_of_atom[cc]] > s->P_type[s->type_of_atom[a]]) {
        i = cc;
        j = a;
      }
      int ti = s->type_of_atom[i], tj = s->type_of_atom[j];
      int Ni = s->P_type[ti], Nj = s->P_type[tj];
      int dq_ij = (ti == ta) + (tj == ta); /* how many charges are q_a */
      double epsij = s->lj_eps[ti * nt + tj];
      /* d eps_ij / d eps_aa: 1 for the a-a pair; eps_ax = eps_ax0 sqrt(eps_aa /
         eps_aa0) for the cross pairs, held fixed when eps_aa0 = 0 */
      double deps = 0.0;
      if (ti == ta && tj == ta) deps = 1.0;
      else if ((ti == ta || tj == ta) && eaa > 0.0) deps = epsij / (2.0 * eaa);
      if (dq_ij == 0 && deps == 0.0) continue;
      int* bi = (int*)malloc(sizeof(int) * (size_t)Ni);
      int* bj = (int*)malloc(sizeof(int) * (size_t)Ni);
      int n = or_pair_map(Ni, Nj, bi, bj);
      double w = 1.0 / Ni;
      int same = s->mol_of_atom[i] == s->mol_of_atom[j];
      for (int m = 0; m < n; ++m) {
        long ri = row_of(s, &L, i, bi[m]), rj = row_of(s, &L, j, bj[m]);
        double d0[3];
        int n0[3];
        for (int d = 0; d < 3; ++d) {
          d0[d] = q[3 * rj + d] - q[3 * ri + d];
          n0[d] = -(int)nearbyint(d0[d] / Lb);
        }
        for (int ix = -2; ix <= 2; ++ix)
          for (int iy = -2; iy <= 2; ++iy)
            for (int iz = -2; iz <= 2; ++iz) {
              if (same && n0[0] + ix == 0 && n0[1] + iy == 0 && n0[2] + iz == 0) continue;
              double dx = d0[0] + (n0[0] + ix) * Lb, dy = d0[1] + (n0[1] + iy) * Lb, dz = d0[2] + (n0[2] + iz) * Lb;
              double r2 = dx * dx + dy * dy + dz * dz;
              if (r2 >= rc2) continue;
              double r = sqrt(r2);
              if (dq_ij) {
                /* d(k_e q_i q_j G)/dq_a, G the unit-charge DSF */
                double G;
                dsf_unit(s->dsf_alpha, rc, r, &G);
                double other = (dq_ij == 2) ? 2.0 * s->charge_type[ta]
                                            : ((ti == ta) ? s->charge_type[tj] : s->charge_type[ti]);
                g[6] += w * c.ke * other * G;
              }
              if (deps != 0.0) {
                double v, dv, vc, dvc;
                /* V_LJ is eps_ij times the unit-epsilon shifted-force term */
                lj_raw(1.0, s->lj_sig[ti * nt + tj], r, &v, &dv);
                lj_raw(1.0, s->lj_sig[ti * nt + tj], rc, &vc, &dvc);
                g[7] += w * (v - vc - (r - rc) * dvc) * deps;
              }
            }
      }
      free(bi);
      free(bj);
    }
  }
  /* pseudopotential terms */
  for (int e = 0; e < s->n_atoms; ++e) {
    if (!s->pseudo_type[s->type_of_atom[e]]) continue;
    for (int cc = 0; cc < s->n_atoms; ++cc) {
      int tc = s->type_of_atom[cc];
      if (s->pseudo_type[tc] || (tc != ta && tc != tb)) continue;
      int Ne = s->P_type[s->type_of_atom[e]], Nc = s->P_type[tc];
      int* bi = (int*)malloc(sizeof(int) * (size_t)Ne);
      int* bj = (int*)malloc(sizeof(int) * (size_t)Ne);
      int n = or_pair_map(Ne, Nc, bi, bj);
      double w = 1.0 / Ne;
      double sig = s->pp_sigma[tc], A = s->pp_A_eV[tc] * c.ev_kcal, b = s->pp_b[tc];
      double dvc[4], ddvc[4];
      pseudo_param_derivs(c.ke, s->charge_type[tc], sig, A, b, rc, dvc, ddvc);
      int off = (tc == ta) ? 0 : 3;
      for (int m = 0; m < n; ++m) {
        long re = row_of(s, &L, e, bi[m]), rs = row_of(s, &L, cc, bj[m]);
        double d0[3];
        int n0[3];
        for (int d = 0; d < 3; ++d) {
          d0[d] = q[3 * rs + d] - q[3 * re + d];
          n0[d] = -(int)nearbyint(d0[d] / Lb);
        }
        for (int ix = -2; ix <= 2; ++ix)
          for (int iy = -2; iy <= 2; ++iy)
            for (int iz = -2; iz <= 2; ++iz) {
              double dx = d0[0] + (n0[0] + ix) * Lb, dy = d0[1] + (n0[1] + iy) * Lb, dz = d0[2] + (n0[2] + iz) * Lb;
              double r2 = dx * dx + dy * dy + dz * dz;
              if (r2 >= rc2) continue;
              double r = sqrt(r2);
              double dv[4], ddv[4];
              pseudo_param_derivs(c.ke, s->charge_type[tc], sig, A, b, r, dv, ddv);
              double t[4];
              for (int k = 0; k < 4; ++k) t[k] = w * (dv[k] - dvc[k] - (r - rc) * ddvc[k]);
              g[off + 0] += t[0];
              g[off + 1] += t[1] * c.ev_kcal; /* per eV */
              g[off + 2] += t[2];
              if (tc == ta) g[6] += t[3];
            }
      }
      free(bi);
      free(bj);
    }
  }
  lay_free(&L);
}

/* ---------------------------------------------------------------------------
 * Radial distribution histogram (Sec. "Output and Analysis"): every ordered
 * pair of atoms (a of type ta, c != a of type tb), every slice of the pair's
 * fine grid through the pair map of Eq. (mts-hamiltonian) with its weight
 * 1/max(P_a, P_c), and every lattice image with
 * r = |q_c - q_a + nL| < nbins dr (the zero image of a same-molecule pair
 * excluded): hist[floor(r / dr)] += weight.
 * ------------------------------------------------------------------------- */
void or_rdf(const or_system* s, const double* q, int ta, int tb, double dr, int nbins, double* hist) {
  lay_t L;
  lay_init(s, &L);
  const double Lb = s->box, rmax = nbins * dr;
  for (int k = 0; k < nbins; ++k) hist[k] = 0.0;
  for (int a = 0; a < s->n_atoms; ++a) {
    if (s->type_of_atom[a] != ta) continue;
    for (int cc = 0; cc < s->n_atoms; ++cc) {
      if (cc == a || s->type_of_atom[cc] != tb) continue;
      int i = a, j = cc; /* i: the finer of the two */
      if (s->P_type[s->type_of_atom[cc]] > s->P_type[s->type_of_atom[a]]) {
        i = cc;
        j = a;
      }
      int Ni = s->P_type[s->type_of_atom[i]], Nj = s->P_type[s->type_of_atom[j]];
      int* bi = (int*)malloc(sizeof(int) * (size_t)Ni);
      int* bj = (int*)malloc(sizeof(int) * (size_t)Ni);
      int n = or_pair_map(Ni, Nj, bi, bj);
      double w = 1.0 / Ni;
      int same = s->mol_of_atom[a] == s->mol_of_atom[cc];
      for (int m = 0; m < n; ++m) {
        long ri = row_of(s, &L, i, bi[m]), rj = row_of(s, &L, j, bj[m]);
        double d0[3];
        int n0[3];
        for (int d = 0; d < 3; ++d) {
          d0[d] = q[3 * rj + d] - q[3 * ri + d];
          n0[d] = -(int)nearbyint(d0[d] / Lb);
        }
        for (int ix = -2; ix <= 2; ++ix)
          for (int iy = -2; iy <= 2; ++iy)
            for (int iz = -2; iz <= 2; ++iz) {
              if (same && n0[0] + ix == 0 && n0[1] + iy == 0 && n0[2] + iz == 0) continue;
              double dx = d0[0] + (n0[0] + ix) * Lb, dy = d0[1] + (n0[1] + iy) * Lb, dz = d0[2] + (n0[2] + iz) * Lb;
              double r = sqrt(dx * dx + dy * dy + dz * dz);
              if (r >= rmax) continue;
              int k = (int)floor(r / dr);
              if (k < nbins) hist[k] += w;
            }
      }
      free(bi);
      free(bj);
    }
  }
  lay_free(&L);
}
