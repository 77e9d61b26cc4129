// mixts_api.cu -- host side of the C ABI declared in include/mixts.h:
// validation, table construction, workspace carving and the per-step launch
// sequence (optionally replayed from a CUDA graph).
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "mixts_internal.cuh"

using namespace mx;

namespace {

constexpr double PI = 3.14159265358979323846;

struct Units {  // internal units: amu, A, fs; potentials kcal/mol
  double kB, hbar, kcal, ev_kcal, ke;
};

// exact SI values of the 2019 redefinition; epsilon_0 from CODATA 2018;
// 1 amu = 1e-3/N_A kg, so one amu A^2 fs^-2 is 1e7/N_A J
Units units() {
  const double h = 6.62607015e-34, e = 1.602176634e-19, kB = 1.380649e-23, NA = 6.02214076e23;
  const double eps0 = 8.8541878128e-12;
  const double E_md = 1.0e7 / NA;
  Units u;
  u.kB = kB / E_md;
  u.hbar = h / (2.0 * PI) / (E_md * 1.0e-15);
  u.kcal = (4184.0 / NA) / E_md;
  u.ev_kcal = e * NA / 4184.0;
  u.ke = e * e / (4.0 * PI * eps0) / 1.0e-10 * NA / 4184.0;
  return u;
}

int ilog2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

struct Arena {
  size_t size = 0;
  size_t add(size_t bytes) {
    size_t o = (size + 255) & ~(size_t)255;
    size = o + bytes;
    return o;
  }
};

// everything mixts_init derives from a system, before touching the device
struct Plan {
  mixts_status st = MIXTS_OK;
  std::string why;
  int nt = 0, na = 0, n_nonp = 0, n_pseudo = 0, n_beads = 0;
  std::vector<int> N, off, atoff, rank, atom_of_tk;
  std::vector<int> pos_atom, pos_mol, pos_of_atom;
  std::vector<AtomInfo> ainfo, ainfo_atom, pinfo;
  std::vector<int> atom_is_pseudo, pseudo_atom;
  std::vector<PairPar> pairpar;
  std::vector<PseudoPar> pspar;
  std::vector<BondItem> bitems;
  std::vector<int> bond_atoms, ang_atoms;
  std::vector<double> bond_par, ang_par;
  std::vector<double> cm;
  std::vector<double> dsf;     // DSF interval table
  std::vector<float> dsf32;    // its binary32 cubic form (FP32 forces)
  std::vector<double> charge, eps, sig, pp_sig, pp_A, pp_b;  // raw force-field parameters (theta variant)
  int dsf_nint = 0, dsf_elo = -2;
  std::vector<double> ps_tab;  // pseudopotential tables (electron systems)
  // centroid Ewald (coulomb == 1)
  std::vector<double> kvec;    // 4 per wave vector
  std::vector<int> kn, qinfo, intra;
  std::vector<double> qcharge;
  int n_kvec = 0, n_qatoms = 0, n_intra = 0;
  double ew_const = 0.0, ew_bg = 0.0;
  size_t o_kvec = 0, o_kn = 0, o_qinfo = 0, o_qcharge = 0, o_intra = 0, o_ewphase = 0, o_ewcen = 0, o_ews = 0,
         o_ewek = 0;
  int ps_nint = 0, ps_elo = -6;
  std::vector<int> cm_off, mc_off;
  std::vector<ModeCoef> mc;
  std::vector<PropTile> tiles;  // small-P tiles, then large-P tiles
  int n_small_tiles = 0, big_cl = 1;
  std::vector<int> slot_type;
  int nl_cap = 0, pl_cap = 0;
  int nc = 0;  // cells per side of the neighbour search (0: all pairs)
  size_t o_cstart = 0, o_catoms = 0, o_cok = 0;
  int n_classes = 0;
  int cls_P[MAX_CLASSES], cls_log2P[MAX_CLASSES], cls_pos0[MAX_CLASSES], cls_n[MAX_CLASSES],
      cls_item0[MAX_CLASSES + 1];
  int n_pitems = 0, n_ppitems = 0;
  // workspace offsets
  Arena ar;
  size_t o_tab = 0, tab_bytes = 0;
  size_t o_ainfo, o_pos_atom, o_pos_mol, o_atom_of_tk, o_ainfo_atom, o_pos_of_atom, o_is_pseudo, o_pseudo_atom, o_pinfo,
      o_pairpar, o_pspar, o_bitems, o_bond_atoms, o_bond_par, o_ang_atoms, o_ang_par, o_cm, o_mc, o_tiles,
      o_slot_type, o_dsf, o_dsf32, o_pstab, o_pairpar_alt, o_pspar_alt, o_pc, o_gacc;
  size_t o_state = 0, state_bytes = 0;
  size_t o_xd = 0, o_xia = 0;
  size_t o_pitems = 0, o_pctr = 0, o_nlb = 0, o_nlseg = 0, o_wrapn = 0;
  size_t o_qnm, o_pnm, o_ffix, o_xw, o_xi, o_xf, o_xl, o_ref, o_refd, o_reff, o_spread, o_nl, o_nlcnt, o_pl, o_plcnt, o_thresh, o_efix,
      o_err, o_step, o_heat, o_est, o_parts;
};

void fail(Plan& p, mixts_status s, const std::string& why) {
  if (p.st == MIXTS_OK) {
    p.st = s;
    p.why = why;
  }
}

void lj_at(double e4, double s2, double r, double* v, double* dv) {
  const double sr2 = s2 / (r * r);
  const double sr6 = sr2 * sr2 * sr2;
  const double sr12 = sr6 * sr6;
  *v = e4 * (sr12 - sr6);
  *dv = -6.0 * e4 * (2.0 * sr12 - sr6) / r;
}

void pseudo_at(const PseudoPar& pp, double r, double* v, double* dv) {
  const double x = r / pp.sig;
  const double ef = erf(x);
  const double gg = ef / r;
  const double dg = 2.0 / sqrt(PI) * exp(-x * x) / (pp.sig * r) - ef / (r * r);
  const double ex = exp(-r / pp.b);
  *v = -pp.kq * gg + pp.A * ex;
  *dv = -pp.kq * dg - (pp.A / pp.b) * ex;
}

// Unit-charge DSF potential G(s) = erfc(a r)/r - erfc(a rc)/rc + cf (r - rc),
// s = r^2, and -2 G'(s), tabulated as quintics in x = s - s0 on 64
// equal sub-intervals of every octave [2^e, 2^(e+1)) of s from 2^elo up past
// rc^2. Each quintic interpolates its function at the six Chebyshev nodes of
// the interval (values in long double). Row layout: c0..c5 of G, then
// c0..c5 of -2 G'.
template <int N>
static void fit_poly(const long double* tn, const long double* val, long double h, double* out) {
  typedef long double LD;
  LD A[N][N + 1];
  for (int i = 0; i < N; ++i) {
    LD tp = 1.0L;
    for (int j = 0; j < N; ++j) {
      A[i][j] = tp;
      tp *= tn[i];
    }
    A[i][N] = val[i];
  }
  for (int c = 0; c < N; ++c) {  // Gauss-Jordan, partial pivoting
    int pv = c;
    for (int r = c + 1; r < N; ++r)
      if (fabsl(A[r][c]) > fabsl(A[pv][c])) pv = r;
    for (int j = 0; j < N + 1; ++j) std::swap(A[c][j], A[pv][j]);
    for (int r = 0; r < N; ++r) {
      if (r == c) continue;
      const LD f = A[r][c] / A[c][c];
      for (int j = c; j < N + 1; ++j) A[r][j] -= f * A[c][j];
    }
  }
  LD hk = 1.0L;
  for (int j = 0; j < N; ++j) {
    out[j] = (double)(A[j][N] / A[j][j] / hk);
    hk *= h;
  }
}

static void fit_quintic(const long double* tn, const long double* val, long double h, double* out) {
  fit_poly<6>(tn, val, h, out);
}

// Interval table of a function of s = r^2 and of a second one (the force
// over r), 64 sub-intervals per octave from 2^elo to past rc^2, a quintic of
// each fitted at Chebyshev nodes in long double.
template <class F1, class F2>
static std::vector<double> interval_table(F1 f, F2 df, double rc, int elo, int* nint_out) {
  typedef long double LD;
  const LD pil = 3.141592653589793238462643383279502884L;
  int ehi = elo;
  while (ldexp(1.0, ehi) <= rc * rc) ++ehi;
  const int nint = (ehi - elo) * 64;
  std::vector<double> tab(12 * (size_t)nint);
  LD tn[6];
  for (int i = 0; i < 6; ++i) tn[i] = (1.0L - cosl((2 * i + 1) * pil / 12.0L)) / 2.0L;
  for (int k = 0; k < nint; ++k) {
    const int oct = k / 64, sub = k % 64;
    const LD s0 = ldexpl(1.0L + sub / 64.0L, elo + oct);
    const LD h = ldexpl(1.0L / 64.0L, elo + oct);
    LD v[6], dv[6];
    for (int i = 0; i < 6; ++i) {
      v[i] = f(s0 + tn[i] * h);
      dv[i] = df(s0 + tn[i] * h);
    }
    fit_quintic(tn, v, h, &tab[12 * (size_t)k]);
    fit_quintic(tn, dv, h, &tab[12 * (size_t)k + 6]);
  }
  *nint_out = nint;
  return tab;
}

// Shifted-force pseudopotential of one site type (Sec. "System II": V(r) =
// -k_e q erf(r/sigma)/r + A exp(-r/b), truncated at r_cut with value and slope
// shifted to zero): the value and -(dV/dr - dV/dr(r_cut)) / r as functions
// of s = r^2.
static std::vector<double> pseudo_table(double kq, double sig, double A, double b, double rc, int elo,
                                        int* nint_out) {
  typedef long double LD;
  const LD pil = 3.141592653589793238462643383279502884L;
  auto V = [&](LD r) { return -(LD)kq * erfl(r / sig) / r + (LD)A * expl(-r / b); };
  auto dV = [&](LD r) {
    const LD x = r / sig;
    return -(LD)kq * (2.0L / sqrtl(pil) * expl(-x * x) / (sig * r) - erfl(x) / (r * r)) - (LD)A / b * expl(-r / b);
  };
  const LD R = rc, vr = V(R), dvr = dV(R);
  return interval_table([&](LD s) { const LD r = sqrtl(s); return V(r) - vr - (r - R) * dvr; },
                        [&](LD s) { const LD r = sqrtl(s); return -(dV(r) - dvr) / r; }, rc, elo, nint_out);
}

// shifted: the damped-shifted-force form; otherwise the Ewald real-space
// kernel erfc(a r)/r (value and slope not shifted at rc). With tab32 also
// the binary32 table of the FP32 pair sweep: per interval the cubics
// (interpolating at four Chebyshev nodes) of the same two functions,
// coefficients c0..c3 of G then c0..c3 of -2 G'.
std::vector<double> dsf_table(double alpha, double rc, int elo, int* nint_out, bool shifted = true,
                              std::vector<float>* tab32 = nullptr) {
  typedef long double LD;
  const LD a = alpha, R = rc;
  const LD pil = 3.141592653589793238462643383279502884L;
  const LD erc = shifted ? erfcl(a * R) : 0.0L;
  const LD gg = 2.0L * a / sqrtl(pil);
  const LD cf = shifted ? erc / (R * R) + gg * expl(-a * a * R * R) / R : 0.0L;
  auto G = [&](LD sv) {
    const LD r = sqrtl(sv);
    return erfcl(a * r) / r - erc / R + cf * (r - R);
  };
  auto dG = [&](LD sv) {  // -2 dG/ds = -(dG/dr) / r, the force over r per unit charge product
    const LD r = sqrtl(sv);
    return -(-erfcl(a * r) / (r * r) - gg * expl(-a * a * sv) / r + cf) / r;
  };
  int ehi = elo;
  while (ldexp(1.0, ehi) <= rc * rc) ++ehi;
  const int nint = (ehi - elo) * 64;
  std::vector<double> tab(12 * (size_t)nint);
  LD tn[6], tc[4];
  for (int i = 0; i < 6; ++i) tn[i] = (1.0L - cosl((2 * i + 1) * pil / 12.0L)) / 2.0L;
  for (int i = 0; i < 4; ++i) tc[i] = (1.0L - cosl((2 * i + 1) * pil / 8.0L)) / 2.0L;
  if (tab32) tab32->assign(8 * (size_t)nint, 0.0f);
  for (int k = 0; k < nint; ++k) {
    const int oct = k / 64, sub = k % 64;
    const LD s0 = ldexpl(1.0L + sub / 64.0L, elo + oct);
    const LD h = ldexpl(1.0L / 64.0L, elo + oct);
    LD v[6], dv[6];
    for (int i = 0; i < 6; ++i) {
      v[i] = G(s0 + tn[i] * h);
      dv[i] = dG(s0 + tn[i] * h);
    }
    fit_quintic(tn, v, h, &tab[12 * (size_t)k]);
    fit_quintic(tn, dv, h, &tab[12 * (size_t)k + 6]);
    if (tab32) {
      double c[8];
      for (int i = 0; i < 4; ++i) {
        v[i] = G(s0 + tc[i] * h);
        dv[i] = dG(s0 + tc[i] * h);
      }
      fit_poly<4>(tc, v, h, c);
      fit_poly<4>(tc, dv, h, c + 4);
      for (int j = 0; j < 8; ++j) (*tab32)[8 * (size_t)k + j] = (float)c[j];
    }
  }
  *nint_out = nint;
  return tab;
}

Plan make_plan(const mixts_system* s, const mixts_params* prm) {
  Plan p;
  const Units u = units();
  if (!s || !prm) {
    fail(p, MIXTS_ERR_ARG, "NULL system or params");
    return p;
  }
  p.nt = s->n_types;
  p.na = s->n_atoms;
  if (p.nt < 1 || p.nt > MT || p.na < 1) {
    fail(p, MIXTS_ERR_ARG, "n_types must be 1..16 and n_atoms >= 1");
    return p;
  }
  if (!s->type_of_atom || !s->mol_of_atom || !s->P_type || !s->mass_type || !s->charge_type || !s->lj_eps ||
      !s->lj_sig || !s->pseudo_type || !s->pp_sigma || !s->pp_A_eV || !s->pp_b) {
    fail(p, MIXTS_ERR_ARG, "NULL per-type or per-atom array");
    return p;
  }
  if (prm->free_ring_substeps < 0) {
    fail(p, MIXTS_ERR_ARG, "free_ring_substeps must be >= 0");
    return p;
  }
  if (prm->precision != MIXTS_FP64 && prm->precision != MIXTS_FP32_FORCES) {
    fail(p, MIXTS_ERR_ARG, "unknown precision");
    return p;
  }
  if (!(s->box > 0.0) || !(prm->r_cut > 0.0) || !(prm->dt > 0.0) || !(prm->T > 0.0)) {
    fail(p, MIXTS_ERR_ARG, "box, r_cut, dt and T must be positive");
    return p;
  }
  for (int t = 0; t < p.nt; ++t) {
    const int P = s->P_type[t];
    if (P < 1 || P > 1024 || (P & (P - 1))) {
      fail(p, MIXTS_ERR_BEADS, "bead counts must be powers of two in 1..1024");
      return p;
    }
    if (!(s->mass_type[t] > 0.0) || (s->bead_mass_type && !(s->bead_mass_type[t] > 0.0))) {
      fail(p, MIXTS_ERR_ARG, "masses must be positive");
      return p;
    }
  }
  p.N.assign(p.nt, 0);
  p.rank.assign(p.na, 0);
  for (int a = 0; a < p.na; ++a) {
    const int t = s->type_of_atom[a];
    if (t < 0 || t >= p.nt) {
      fail(p, MIXTS_ERR_ARG, "type_of_atom out of range");
      return p;
    }
    p.rank[a] = p.N[t]++;
  }
  p.off.assign(p.nt + 1, 0);
  p.atoff.assign(p.nt + 1, 0);
  for (int t = 0; t < p.nt; ++t) {
    p.off[t + 1] = p.off[t] + p.N[t] * s->P_type[t];
    p.atoff[t + 1] = p.atoff[t] + p.N[t];
  }
  p.n_beads = p.off[p.nt];
  p.atom_of_tk.assign(p.na, 0);
  p.ainfo_atom.resize(p.na);
  p.atom_is_pseudo.assign(p.na, 0);
  for (int a = 0; a < p.na; ++a) {
    const int t = s->type_of_atom[a];
    p.atom_of_tk[p.atoff[t] + p.rank[a]] = a;
    p.ainfo_atom[a] = AtomInfo{p.off[t] + p.rank[a], p.N[t], ilog2(s->P_type[t]), t};
    p.atom_is_pseudo[a] = s->pseudo_type[t] ? 1 : 0;
  }
  // sorted positions of non-pseudo atoms: P descending, index ascending
  std::vector<int> order;
  for (int a = 0; a < p.na; ++a)
    if (!p.atom_is_pseudo[a]) order.push_back(a);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return s->P_type[s->type_of_atom[x]] > s->P_type[s->type_of_atom[y]];
  });
  p.n_nonp = (int)order.size();
  p.pos_of_atom.assign(p.na, -1);
  for (int i = 0; i < p.n_nonp; ++i) {
    const int a = order[i];
    p.pos_atom.push_back(a);
    p.pos_mol.push_back(s->mol_of_atom[a]);
    p.ainfo.push_back(p.ainfo_atom[a]);
    p.pos_of_atom[a] = i;
  }
  if ((long long)p.n_nonp >= (1LL << 24) || (long long)p.off[p.nt] >= (1LL << 20)) {
    fail(p, MIXTS_ERR_ARG, "list entries hold bead rows below 2^20 and atom positions below 2^24");
    return p;
  }
  // classes
  p.cls_item0[0] = 0;
  for (int i = 0; i < p.n_nonp;) {
    const int P = 1 << p.ainfo[i].log2P;
    int j = i;
    while (j < p.n_nonp && (1 << p.ainfo[j].log2P) == P) ++j;
    if (p.n_classes >= MAX_CLASSES) {
      fail(p, MIXTS_ERR_BEADS, "too many distinct bead counts");
      return p;
    }
    const int c = p.n_classes++;
    p.cls_P[c] = P;
    p.cls_log2P[c] = ilog2(P);
    p.cls_pos0[c] = i;
    p.cls_n[c] = j - i;
    p.cls_item0[c + 1] = p.cls_item0[c] + P * (j - i);
    i = j;
  }
  p.n_pitems = p.cls_item0[p.n_classes];
  // pseudo particles
  int maxP_site = 1;
  for (int t = 0; t < p.nt; ++t)
    if (!s->pseudo_type[t] && p.N[t] > 0) maxP_site = std::max(maxP_site, s->P_type[t]);
  for (int a = 0; a < p.na; ++a) {
    if (!p.atom_is_pseudo[a]) continue;
    if (s->P_type[s->type_of_atom[a]] < maxP_site) {
      fail(p, MIXTS_ERR_BEADS, "a pseudo particle must have at least as many beads as every site");
      return p;
    }
    p.pseudo_atom.push_back(a);
    p.pinfo.push_back(p.ainfo_atom[a]);
    p.n_ppitems += s->P_type[s->type_of_atom[a]];
  }
  p.n_pseudo = (int)p.pseudo_atom.size();
  // raw parameters, kept for parameter-gradient evaluations
  p.charge.assign(s->charge_type, s->charge_type + p.nt);
  p.eps.assign(s->lj_eps, s->lj_eps + p.nt * p.nt);
  p.sig.assign(s->lj_sig, s->lj_sig + p.nt * p.nt);
  p.pp_sig.assign(s->pp_sigma, s->pp_sigma + p.nt);
  p.pp_A.assign(s->pp_A_eV, s->pp_A_eV + p.nt);
  p.pp_b.assign(s->pp_b, s->pp_b + p.nt);
  // pair parameters
  const double rc = prm->r_cut;
  p.pairpar.assign(MT * MT, PairPar{0, 0, 1, 0, 0});
  for (int a = 0; a < p.nt; ++a)
    for (int b = 0; b < p.nt; ++b) {
      PairPar pp;
      pp.qq = u.ke * s->charge_type[a] * s->charge_type[b];
      const double eps = s->lj_eps[a * p.nt + b], sig = s->lj_sig[a * p.nt + b];
      pp.e4 = 4.0 * eps;
      pp.s2 = sig * sig;
      pp.vrc = 0.0;
      pp.dvrc = 0.0;
      if (eps != 0.0) lj_at(pp.e4, pp.s2, rc, &pp.vrc, &pp.dvrc);
      p.pairpar[a * MT + b] = pp;
    }
  p.pspar.assign(MT, PseudoPar{0, 1, 0, 1, 0, 0});
  for (int t = 0; t < p.nt; ++t) {
    PseudoPar pp;
    pp.kq = u.ke * s->charge_type[t];
    pp.sig = s->pp_sigma[t];
    pp.A = s->pp_A_eV[t] * u.ev_kcal;
    pp.b = s->pp_b[t];
    if (p.n_pseudo > 0 && !s->pseudo_type[t] && p.N[t] > 0 && (!(pp.sig > 0.0) || !(pp.b > 0.0))) {
      fail(p, MIXTS_ERR_ARG, "pseudopotential sigma and b must be positive");
      return p;
    }
    pp.vrc = pp.dvrc = 0.0;
    if (pp.sig > 0.0 && pp.b > 0.0) pseudo_at(pp, rc, &pp.vrc, &pp.dvrc);
    p.pspar[t] = pp;
  }
  // bonded work items: one per (term, slice of the term's finest grid)
  if (s->n_bonds < 0 || s->n_angles < 0 || (s->n_bonds > 0 && (!s->bonds || !s->bond_k || !s->bond_r0)) ||
      (s->n_angles > 0 && (!s->angles || !s->angle_k || !s->angle_theta0))) {
    fail(p, MIXTS_ERR_ARG, "bad bond/angle arrays");
    return p;
  }
  for (int b = 0; b < s->n_bonds; ++b) {
    const int a = s->bonds[2 * b], c = s->bonds[2 * b + 1];
    if (a < 0 || a >= p.na || c < 0 || c >= p.na || a == c) {
      fail(p, MIXTS_ERR_ARG, "bond atom out of range");
      return p;
    }
    p.bond_atoms.push_back(a);
    p.bond_atoms.push_back(c);
    p.bond_par.push_back(s->bond_k[b]);
    p.bond_par.push_back(s->bond_r0[b]);
    const int Ps = std::max(s->P_type[s->type_of_atom[a]], s->P_type[s->type_of_atom[c]]);
    for (int sl = 0; sl < Ps; ++sl) p.bitems.push_back(BondItem{0, b, sl, 0});
  }
  for (int g = 0; g < s->n_angles; ++g) {
    int Ps = 1;
    for (int x = 0; x < 3; ++x) {
      const int a = s->angles[3 * g + x];
      if (a < 0 || a >= p.na) {
        fail(p, MIXTS_ERR_ARG, "angle atom out of range");
        return p;
      }
      p.ang_atoms.push_back(a);
      Ps = std::max(Ps, s->P_type[s->type_of_atom[a]]);
    }
    p.ang_par.push_back(s->angle_k[g]);
    p.ang_par.push_back(s->angle_theta0[g]);
    for (int sl = 0; sl < Ps; ++sl) p.bitems.push_back(BondItem{1, g, sl, 0});
  }
  p.dsf = dsf_table(prm->dsf_alpha, prm->r_cut, p.dsf_elo, &p.dsf_nint, prm->coulomb != 1,
                    prm->precision == MIXTS_FP32_FORCES ? &p.dsf32 : nullptr);
  if (prm->coulomb != 0 && prm->coulomb != 1) {
    fail(p, MIXTS_ERR_ARG, "coulomb must be 0 (damped shifted force) or 1 (Ewald)");
    return p;
  }
  if (prm->coulomb == 1) {  // reciprocal sum on centroids: wave vectors, charged sites, same-molecule pairs
    if (prm->ewald_kmax < 1 || prm->ewald_kmax > 64 || !(prm->dsf_alpha > 0.0)) {
      fail(p, MIXTS_ERR_ARG, "Ewald needs ewald_kmax in 1..64 and a positive splitting parameter");
      return p;
    }
    const double L = s->box, V = L * L * L, a = prm->dsf_alpha;
    const int km = prm->ewald_kmax;
    for (int nx = 0; nx <= km; ++nx)
      for (int ny = -km; ny <= km; ++ny)
        for (int nz = -km; nz <= km; ++nz) {
          if (nx * nx + ny * ny + nz * nz > km * km) continue;
          if (!(nx > 0 || (nx == 0 && (ny > 0 || (ny == 0 && nz > 0))))) continue;  // one of k, -k
          const double kx = 2.0 * PI * nx / L, ky = 2.0 * PI * ny / L, kz = 2.0 * PI * nz / L;
          const double k2 = kx * kx + ky * ky + kz * kz;
          const double W = 2.0 * (2.0 * PI * u.ke / V) * exp(-k2 / (4.0 * a * a)) / k2;
          p.kvec.insert(p.kvec.end(), {kx, ky, kz, W});
          p.kn.insert(p.kn.end(), {nx, ny, nz, 0});
        }
    p.n_kvec = (int)(p.kvec.size() / 4);
    std::vector<int> qidx(p.na, -1);
    double Q = 0.0, q2 = 0.0;
    for (int i = 0; i < p.na; ++i) {
      const int t = s->type_of_atom[i];
      if (s->pseudo_type[t] || s->charge_type[t] == 0.0) continue;
      qidx[i] = p.n_qatoms++;
      p.qinfo.insert(p.qinfo.end(), {p.off[t] + p.rank[i], p.N[t], s->P_type[t], i});
      p.qcharge.push_back(s->charge_type[t]);
      Q += s->charge_type[t];
      q2 += s->charge_type[t] * s->charge_type[t];
    }
    for (int i = 0; i < p.na; ++i)
      for (int j = i + 1; j < p.na; ++j)
        if (qidx[i] >= 0 && qidx[j] >= 0 && s->mol_of_atom[i] == s->mol_of_atom[j])
          p.intra.insert(p.intra.end(), {qidx[i], qidx[j]});
    p.n_intra = (int)(p.intra.size() / 2);
    p.ew_bg = -u.ke * PI * Q * Q / (2.0 * V * a * a);
    p.ew_const = -u.ke * a / sqrt(PI) * q2 + p.ew_bg;
  }
  // normal modes, thermostat, rotation
  const double kT = u.kB * prm->T;
  const double bh = u.hbar / kT;
  p.cm_off.assign(MT, 0);
  p.mc_off.assign(MT, 0);
  for (int t = 0; t < p.nt; ++t) {
    const int P = s->P_type[t];
    const double m = s->mass_type[t];
    const double mf = s->bead_mass_type ? s->bead_mass_type[t] : m;  // fictitious bead mass
    std::vector<double> T(P);
    for (int k = 0; k < P; ++k) T[k] = cos(2.0 * PI * k / P);
    p.cm_off[t] = (int)p.cm.size();
    if (P <= SMALL_P) {
      const double rP = 1.0 / sqrt((double)P), r2P = sqrt(2.0 / P);
      for (int j = 0; j < P; ++j)
        for (int k = 0; k < P; ++k) {
          double v;
          if (k == 0)
            v = rP;
          else if (2 * k < P)
            v = r2P * T[(j * k) & (P - 1)];
          else if (2 * k == P)
            v = (j & 1) ? -rP : rP;
          else
            v = r2P * T[(j * k - P / 4) & (P - 1)];
          p.cm.push_back(v);
        }
    } else {  // FFT twiddles (cos, sin)(2 pi m / P), m < P/2
      for (int k = 0; k < P / 2; ++k) {
        p.cm.push_back(T[k]);
        p.cm.push_back(sin(2.0 * PI * k / P));
      }
    }
    p.mc_off[t] = (int)p.mc.size();
    const int nsub = prm->free_ring_substeps;
    for (int k = 0; k < P; ++k) {
      // mode frequency with bead mass m_f: springs P m/(beta hbar)^2, kinetic p^2/2m_f
      const double w = 2.0 * sqrt((double)P) / bh * sin(PI * k / P) * sqrt(m / mf);
      const double gam = (k == 0) ? (prm->tau_centroid > 0.0 ? 1.0 / prm->tau_centroid : 0.0)
                                  : 2.0 * prm->pile_lambda * w;
      ModeCoef c;
      c.c1 = exp(-0.5 * prm->dt * gam);
      c.c2s = sqrt(1.0 - c.c1 * c.c1) * sqrt(mf * kT);
      c.hmw2 = 0.5 * mf * w * w;
      if (nsub > 0) {
        // velocity Verlet on the springs, which act on mode k as the force
        // -m_f w^2 q_k: one sub-step h maps (p, q) by [[a, -B], [C, a]] with
        // a = 1 - h^2 w^2 / 2, B = m_f w^2 h (1 - h^2 w^2 / 4), C = h / m_f;
        // the step is its n-th power (equal diagonals, determinant 1)
        const double h = prm->dt / nsub, hw2 = h * h * w * w;
        const double a = 1.0 - 0.5 * hw2, B = mf * w * w * h * (1.0 - 0.25 * hw2), Cq = h / mf;
        double M00 = 1.0, M01 = 0.0, M10 = 0.0, M11 = 1.0;  // rows (p, q), columns (p, q)
        for (int j = 0; j < nsub; ++j) {
          const double n00 = a * M00 - B * M10, n01 = a * M01 - B * M11;
          const double n10 = Cq * M00 + a * M10, n11 = Cq * M01 + a * M11;
          M00 = n00;
          M01 = n01;
          M10 = n10;
          M11 = n11;
        }
        c.cw = M00;
        c.mws = -M01;
        c.swm = M10;
      } else if (k == 0) {
        c.cw = 1.0;
        c.mws = 0.0;
        c.swm = prm->dt / mf;
      } else {
        c.cw = cos(w * prm->dt);
        c.mws = mf * w * sin(w * prm->dt);
        c.swm = sin(w * prm->dt) / (mf * w);
      }
      p.mc.push_back(c);
    }
  }
  // propagation tiles and estimator partial slots
  for (int t = 0; t < p.nt; ++t) {
    const int P = s->P_type[t];
    if (P > SMALL_P || p.N[t] == 0) continue;
    const int apt = std::max(1, PROP_TILE_BEADS / P);
    for (int k0 = 0; k0 < p.N[t]; k0 += apt) {
      p.tiles.push_back(PropTile{t, k0, std::min(apt, p.N[t] - k0), (int)p.slot_type.size()});
      p.slot_type.push_back(t);
    }
  }
  // large-P tiles: one cluster of big_cl CTAs each (big_cl <= the shorter
  // four-step factor 2^floor(lg P / 2) of every large-P type), with about
  // two waves of CTAs over the GPU and one estimator slot per CTA
  p.n_small_tiles = (int)p.tiles.size();
  p.big_cl = BIG_CL_MAX;
  for (int t = 0; t < p.nt; ++t)
    if (s->P_type[t] > SMALL_P && p.N[t] > 0) p.big_cl = std::min(p.big_cl, 1 << (ilog2(s->P_type[t]) / 2));
  for (int t = 0; t < p.nt; ++t) {
    const int P = s->P_type[t];
    if (P <= SMALL_P || p.N[t] == 0) continue;
    int apt = std::max(1, std::min(BIG_MAXA, (p.N[t] * p.big_cl + 303) / 304));
    while (apt > 1 && big_prop_smem(P, apt, p.big_cl) > (size_t)BIG_SMEM_TARGET) --apt;
    for (int k0 = 0; k0 < p.N[t]; k0 += apt) {
      p.tiles.push_back(PropTile{t, k0, std::min(apt, p.N[t] - k0), (int)p.slot_type.size()});
      for (int r = 0; r < p.big_cl; ++r) p.slot_type.push_back(t);
    }
  }
  // cell list of the neighbour search: cells at least r_cut + 2 A wide (the
  // list radius is r_cut + 2 d_max; a step whose radius exceeds the cell
  // side searches all pairs instead), used when at least 3 fit per side
  {
    const int nc = (int)floor(s->box / (prm->r_cut + 2.0));
    p.nc = nc >= 3 ? std::min(nc, NC_MAX) : 0;
  }
  // neighbour-list capacities
  const double vol = s->box * s->box * s->box;
  const double rho = p.n_nonp / vol;
  if (prm->nlist_cap > 0) {
    p.nl_cap = prm->nlist_cap;
  } else {
    const double Rest = rc + 2.5;
    const double full = rho * 4.0 / 3.0 * PI * Rest * Rest * Rest;
    p.nl_cap = (int)(1.5 * full) + 96;
    p.nl_cap = (p.nl_cap + 31) & ~31;
  }
  // a pseudo particle's site list holds at most every site in each of the 125
  // images of [-2,2]^3: that bound, so the list cannot overflow however far
  // the ring polymer spreads (one row per pseudo particle)
  p.pl_cap = std::max(64, 125 * std::max(1, p.n_nonp));
  if (p.n_pseudo > 0) {  // pseudopotential tables of the site types
    for (int t = 0; t < p.nt; ++t) {
      const PseudoPar& pp = p.pspar[t];
      std::vector<double> tt;
      int nint = 0;
      if (!s->pseudo_type[t] && pp.sig > 0.0 && pp.b > 0.0) {
        tt = pseudo_table(pp.kq, pp.sig, pp.A, pp.b, prm->r_cut, p.ps_elo, &nint);
      } else {
        int ehi = p.ps_elo;
        while (ldexp(1.0, ehi) <= prm->r_cut * prm->r_cut) ++ehi;
        nint = (ehi - p.ps_elo) * 64;
        tt.assign(12 * (size_t)nint, 0.0);
      }
      p.ps_nint = nint;
      p.ps_tab.insert(p.ps_tab.end(), tt.begin(), tt.end());
    }
  }
  // workspace layout: read-only tables first, then the state
  Arena& A = p.ar;
  p.o_ainfo = A.add(sizeof(AtomInfo) * std::max(1, p.n_nonp));
  p.o_pos_atom = A.add(sizeof(int) * std::max(1, p.n_nonp));
  p.o_pos_mol = A.add(sizeof(int) * std::max(1, p.n_nonp));
  p.o_atom_of_tk = A.add(sizeof(int) * p.na);
  p.o_ainfo_atom = A.add(sizeof(AtomInfo) * p.na);
  p.o_pos_of_atom = A.add(sizeof(int) * p.na);
  p.o_is_pseudo = A.add(sizeof(int) * p.na);
  p.o_pseudo_atom = A.add(sizeof(int) * std::max(1, p.n_pseudo));
  p.o_pinfo = A.add(sizeof(AtomInfo) * std::max(1, p.n_pseudo));
  p.o_pairpar = A.add(sizeof(PairPar) * MT * MT);
  p.o_pspar = A.add(sizeof(PseudoPar) * MT);
  p.o_bitems = A.add(sizeof(BondItem) * std::max<size_t>(1, p.bitems.size()));
  p.o_bond_atoms = A.add(sizeof(int) * std::max<size_t>(1, p.bond_atoms.size()));
  p.o_bond_par = A.add(sizeof(double) * std::max<size_t>(1, p.bond_par.size()));
  p.o_ang_atoms = A.add(sizeof(int) * std::max<size_t>(1, p.ang_atoms.size()));
  p.o_ang_par = A.add(sizeof(double) * std::max<size_t>(1, p.ang_par.size()));
  p.o_cm = A.add(sizeof(double) * p.cm.size());
  p.o_mc = A.add(sizeof(ModeCoef) * p.mc.size());
  p.o_tiles = A.add(sizeof(PropTile) * std::max<size_t>(1, p.tiles.size()));
  p.o_slot_type = A.add(sizeof(int) * std::max<size_t>(1, p.slot_type.size()));
  p.o_dsf = A.add(sizeof(double) * p.dsf.size());
  p.o_dsf32 = A.add(sizeof(float) * std::max<size_t>(8, p.dsf32.size()));
  p.o_pstab = A.add(sizeof(double) * std::max<size_t>(1, p.ps_tab.size()));
  p.o_pairpar_alt = A.add(sizeof(PairPar) * MT * MT);
  p.o_pspar_alt = A.add(sizeof(PseudoPar) * MT);
  p.o_pc = A.add(sizeof(double) * 8 * MT);
  p.o_gacc = A.add(sizeof(unsigned long long) * (2 * MT * MT + 8));
  if (p.n_kvec > 0) {
    p.o_kvec = A.add(sizeof(double) * p.kvec.size());
    p.o_kn = A.add(sizeof(int) * p.kn.size());
    p.o_qinfo = A.add(sizeof(int) * std::max<size_t>(4, p.qinfo.size()));
    p.o_qcharge = A.add(sizeof(double) * std::max<size_t>(1, p.qcharge.size()));
    p.o_intra = A.add(sizeof(int) * std::max<size_t>(2, p.intra.size()));
  }
  p.tab_bytes = A.size;
  const size_t nb3 = (size_t)p.n_beads * 3;
  p.o_qnm = A.add(sizeof(double) * nb3);
  p.o_pnm = A.add(sizeof(double) * nb3);
  p.o_ffix = A.add(sizeof(unsigned long long) * nb3);
  p.o_xw = A.add(sizeof(double4_32a) * p.n_beads);
  p.o_xi = A.add(sizeof(longlong4_32a) * p.n_beads);
  p.o_xf = A.add(sizeof(float4) * p.n_beads);
  p.o_xl = A.add(sizeof(float4) * p.n_beads);
  if (prm->precision == MIXTS_FP32_FORCES) p.o_xd = A.add(sizeof(float4) * p.n_beads);
  // the atom-major fixed-point copy feeds the FP64 sweep, which the
  // parameter-gradient path runs whatever the handle's precision
  p.o_xia = A.add(sizeof(longlong4_32a) * p.n_beads);
  p.o_ref = A.add(sizeof(double) * 3 * p.na);
  p.o_refd = A.add(sizeof(double4_32a) * std::max(1, p.n_nonp));
  p.o_reff = A.add(sizeof(float4) * std::max(1, p.n_nonp));
  p.o_wrapn = A.add(sizeof(int4) * std::max(1, p.n_nonp));
  p.o_spread = A.add(sizeof(double) * (size_t)p.na);
  p.o_nl = A.add(sizeof(int) * (size_t)std::max(1, p.n_nonp) * p.nl_cap);
  p.o_nlcnt = A.add(sizeof(int) * std::max(1, p.n_nonp));
  p.o_cstart = A.add(sizeof(int) * ((size_t)p.nc * p.nc * p.nc + 1));
  p.o_catoms = A.add(sizeof(int) * std::max(1, p.n_nonp));
  p.o_cok = A.add(sizeof(int));
  {  // FP64 pair items: at most every row's slice blocks times 32-entry chunks of a full row
    const int lgM = p.n_classes > 0 ? p.cls_log2P[0] : 0;
    const size_t nsbm = lgM > 5 ? (size_t)1 << (lgM - 5) : 1;
    size_t nitems = (size_t)p.n_nonp * nsbm * ((p.nl_cap + P64_CH - 1) / P64_CH);
    if (prm->precision == MIXTS_FP32_FORCES) {
      // FP32 items: per row and partner type at most ceil(entries / 1) + 1 chunks of >= 1 entry per group...
      // bounded by one item per entry and slice block plus one partial item per type
      nitems = (size_t)p.n_nonp * nsbm * ((size_t)p.nl_cap + p.nt);
      p.o_nlb = A.add(sizeof(float4) * (size_t)std::max(1, p.n_nonp) * p.nl_cap);
      p.o_nlseg = A.add(sizeof(int) * (size_t)std::max(1, p.n_nonp) * (p.nt + 1));
    }
    p.o_pitems = A.add(sizeof(int2) * std::max<size_t>(1, nitems));
    p.o_pctr = A.add(sizeof(int) * (4 + P32W_MAX_NW));
  }
  p.o_pl = A.add(sizeof(int) * (size_t)std::max(1, p.n_pseudo) * p.pl_cap);
  p.o_plcnt = A.add(sizeof(int) * std::max(1, p.n_pseudo));
  p.o_thresh = A.add(sizeof(double) * 12);  // 4 radii, 9 binary32 screen constants, R^2, R_pseudo^2
  p.o_efix = A.add(sizeof(unsigned long long) * E_NSLOTS);
  p.o_err = A.add(sizeof(int) * 4);
  p.o_step = A.add(sizeof(long long));
  p.o_heat = A.add(sizeof(double));
  p.o_est = A.add(sizeof(double) * EST_N);
  p.o_parts = A.add(sizeof(double) * 6 * std::max<size_t>(1, p.slot_type.size()));
  if (p.n_kvec > 0) {
    p.o_ewphase = A.add(sizeof(double2) * (size_t)std::max(1, p.n_qatoms) * 3 * (prm->ewald_kmax + 1));
    p.o_ewcen = A.add(sizeof(double) * 4 * (size_t)std::max(1, p.n_qatoms));
    p.o_ews = A.add(sizeof(double2) * (size_t)p.n_kvec);
    p.o_ewek = A.add(sizeof(double) * 2 * (size_t)p.n_kvec);
  }
  p.state_bytes = A.size - p.tab_bytes;
  return p;
}

template <class T>
void put(std::vector<unsigned char>& img, size_t off, const std::vector<T>& v) {
  if (!v.empty()) memcpy(img.data() + off, v.data(), sizeof(T) * v.size());
}

}  // namespace

struct Timer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<int, size_t>> recs;  // (phase, index of the start event)
  double ms[MIXTS_N_PHASES] = {0};
  long long calls[MIXTS_N_PHASES] = {0};
};

struct mixts_ctx {
  Dev d;
  Timer tm;
  long long kernels = 0;
  Plan plan;
  cudaStream_t stream = nullptr;
  unsigned char* ws = nullptr;
  const int* slot_type = nullptr;
  const AtomInfo* ainfo_atom = nullptr;
  const int* atom_is_pseudo = nullptr;
  bool nm_valid = false;  // mode-space state is authoritative
  bool f_valid = false;   // F_fix holds the forces at the current positions
  long long steps_done = 0;
  std::string err;
  int device = 0;
  int full_grid64 = 0, full_grid32 = 0;  // SM-filling persistent grids
  // batched handle (n_sys > 1): one sub-context per system, advanced by one
  // captured graph whose branches run the systems concurrently
  std::vector<mixts_ctx*> kids;
  std::vector<cudaStream_t> fork;
  std::vector<cudaEvent_t> fev;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int g_steps = 0;
  long long g_kernels = 0;
  mixts_batch_tuning tune{};
  // one launch per phase for all members: member Dev records and per-kernel
  // block prefixes in the batch's own slice of the workspace
  unsigned char* bdev = nullptr;
  int* bpfx = nullptr;
  BatchGeom geom{};
  // single handle: steps per captured graph launch (0: eager launches)
  int graph_steps = 10;
  bool capturing = false;
  bool list_valid = false;  // neighbour lists and position mirrors match the current q
  // bonded and pseudopotential terms beside the pair sweep, large-P
  // propagation beside the small-P tiles
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_list = nullptr, ev_join = nullptr, ev_post = nullptr, ev_fin = nullptr;
  bool fin_pending = false;  // a finalisation on the side stream not yet joined
};

static void timer_fold(mixts_handle h) {
  Timer& T = h->tm;
  if (T.recs.empty()) return;
  cudaStreamSynchronize(h->stream);
  for (auto& r : T.recs) {
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, T.pool[r.second], T.pool[r.second + 1]);
    T.ms[r.first] += ms;
    T.calls[r.first] += 1;
  }
  T.recs.clear();
  T.used = 0;
}

// run one launcher inside a timed phase
template <class F>
static void phase(mixts_handle h, int ph, F&& launch) {
  Timer& T = h->tm;
  if (!T.on) {
    h->kernels += launch();
    return;
  }
  if (T.used + 2 > T.pool.size()) timer_fold(h);
  if (T.pool.size() < 4096) {
    while (T.pool.size() < 4096) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      T.pool.push_back(e);
    }
  }
  const size_t a = T.used;
  cudaEventRecord(T.pool[a], h->stream);
  h->kernels += launch();
  cudaEventRecord(T.pool[a + 1], h->stream);
  T.used += 2;
  T.recs.push_back({ph, a});
}

static mixts_status set_err(mixts_handle h, mixts_status s, const std::string& why) {
  if (h) h->err = why;
  return s;
}

static mixts_status cuda_check(mixts_handle h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MIXTS_OK;
  return set_err(h, MIXTS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// device -> host copy ordered on the handle's stream, then wait for it: the
// caller's stream may be non-blocking, so a legacy-stream cudaMemcpy would not
// be ordered after the kernels that wrote src
static mixts_status d2h(mixts_handle h, void* dst, const void* src, size_t bytes, const char* what) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return cuda_check(h, e, what);
}

static mixts_status device_error(mixts_handle h) {
  int e = 0;
  cudaError_t ce = cudaMemcpyAsync(&e, h->d.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) return cuda_check(h, ce, "synchronise");
  if (e == 0) return MIXTS_OK;
  cudaMemsetAsync(h->d.err, 0, sizeof(int), h->stream);
  if (e & ERR_BOX) return set_err(h, MIXTS_ERR_BOX, "list radius reached twice the box edge");
  if (e & ERR_NLIST)
    return set_err(h, MIXTS_ERR_NLIST_OVERFLOW, "a nonbonded neighbour-list row outgrew nlist_cap");
  if (e & ERR_PLIST)
    return set_err(h, MIXTS_ERR_NLIST_OVERFLOW, "a pseudo-particle site list outgrew its capacity");
  if (e & ERR_NONFINITE) return set_err(h, MIXTS_ERR_NONFINITE, "non-finite or out-of-range force");
  if (e & ERR_TIMEOUT) return set_err(h, MIXTS_ERR_TIMEOUT, "bounded device wait expired");
  return set_err(h, MIXTS_ERR_CUDA, "unknown device error bits");
}

extern "C" {

const char* mixts_version(void) { return "mixts-gb300 0.1 (sm_103a)"; }

static size_t batch_workspace_size(const mixts_system* sys, int n_sys, const mixts_params* prm);
static mixts_status batch_init(const mixts_system* sys, int n_sys, const mixts_params* prm, void* workspace,
                               size_t ws_bytes, void* stream, mixts_handle* out);

size_t mixts_workspace_size(const mixts_system* sys, int n_sys, const mixts_params* prm) {
  if (n_sys > 1 && sys) return batch_workspace_size(sys, n_sys, prm);
  if (n_sys != 1 || !sys) return 0;
  Plan p = make_plan(sys, prm);
  if (p.st != MIXTS_OK) return 0;
  return p.ar.size + 256;
}

mixts_status mixts_init(const mixts_system* sys, int n_sys, const mixts_params* prm, void* workspace,
                        size_t ws_bytes, void* stream, mixts_handle* out) {
  if (!out) return MIXTS_ERR_ARG;
  *out = nullptr;
  if (n_sys > 1 && sys && prm) return batch_init(sys, n_sys, prm, workspace, ws_bytes, stream, out);
  if (n_sys != 1 || !sys || !prm) return MIXTS_ERR_ARG;
  if (!sys->q || !sys->p || !sys->f) return MIXTS_ERR_ARG;
  mixts_handle h = new mixts_ctx();
  h->plan = make_plan(sys, prm);
  Plan& p = h->plan;
  if (p.st != MIXTS_OK) {
    mixts_status st = p.st;
    fprintf(stderr, "mixts_init: %s\n", p.why.c_str());
    delete h;
    return st;
  }
  if (!workspace || ((uintptr_t)workspace & 255) || ws_bytes < p.ar.size) {
    delete h;
    return MIXTS_ERR_WORKSPACE;
  }
  cudaGetDevice(&h->device);
  h->stream = (cudaStream_t)stream;
  h->ws = (unsigned char*)workspace;
  // table image
  std::vector<unsigned char> img(p.tab_bytes, 0);
  put(img, p.o_ainfo, p.ainfo);
  put(img, p.o_pos_atom, p.pos_atom);
  put(img, p.o_pos_mol, p.pos_mol);
  put(img, p.o_atom_of_tk, p.atom_of_tk);
  put(img, p.o_ainfo_atom, p.ainfo_atom);
  put(img, p.o_pos_of_atom, p.pos_of_atom);
  put(img, p.o_is_pseudo, p.atom_is_pseudo);
  put(img, p.o_pseudo_atom, p.pseudo_atom);
  put(img, p.o_pinfo, p.pinfo);
  put(img, p.o_pairpar, p.pairpar);
  put(img, p.o_pspar, p.pspar);
  put(img, p.o_bitems, p.bitems);
  put(img, p.o_bond_atoms, p.bond_atoms);
  put(img, p.o_bond_par, p.bond_par);
  put(img, p.o_ang_atoms, p.ang_atoms);
  put(img, p.o_ang_par, p.ang_par);
  put(img, p.o_cm, p.cm);
  put(img, p.o_mc, p.mc);
  put(img, p.o_tiles, p.tiles);
  put(img, p.o_slot_type, p.slot_type);
  put(img, p.o_dsf, p.dsf);
  if (!p.dsf32.empty()) put(img, p.o_dsf32, p.dsf32);
  if (!p.ps_tab.empty()) put(img, p.o_pstab, p.ps_tab);
  if (p.n_kvec > 0) {
    put(img, p.o_kvec, p.kvec);
    put(img, p.o_kn, p.kn);
    put(img, p.o_qinfo, p.qinfo);
    put(img, p.o_qcharge, p.qcharge);
    put(img, p.o_intra, p.intra);
  }
  // upload on the caller's stream (the kernels that read the tables follow it
  // there); the host image stays alive until the synchronisation below
  mixts_status st =
      cuda_check(h, cudaMemcpyAsync(h->ws, img.data(), p.tab_bytes, cudaMemcpyHostToDevice, h->stream), "upload tables");
  if (st == MIXTS_OK)
    st = cuda_check(h, cudaMemsetAsync(h->ws + p.tab_bytes, 0, p.ar.size - p.tab_bytes, h->stream), "clear state");
  if (st == MIXTS_OK) st = cuda_check(h, cudaStreamSynchronize(h->stream), "init sync");
  if (st != MIXTS_OK) {
    fprintf(stderr, "mixts_init: %s\n", h->err.c_str());
    delete h;
    return st;
  }
  const Units u = units();
  Dev& d = h->d;
  memset(&d, 0, sizeof(d));
  d.n_atoms = p.na;
  d.n_nonp = p.n_nonp;
  d.n_pseudo = p.n_pseudo;
  d.n_types = p.nt;
  d.n_beads = p.n_beads;
  d.n_bitems = (int)p.bitems.size();
  d.n_pitems = p.n_pitems;
  d.n_ppitems = p.n_ppitems;
  d.nl_cap = p.nl_cap;
  d.pl_cap = p.pl_cap;
  d.n_classes = p.n_classes;
  d.n_tiles = p.n_small_tiles;
  d.n_big_tiles = (int)p.tiles.size() - p.n_small_tiles;
  if (d.n_big_tiles > 0) {
    // the cluster size the device co-schedules (the plan's, or smaller: the
    // slots of CTAs that do not exist stay zero)
    std::vector<int> bP, bna;
    for (size_t i = p.n_small_tiles; i < p.tiles.size(); ++i) {
      bP.push_back(sys->P_type[p.tiles[i].type]);
      bna.push_back(p.tiles[i].na);
    }
    d.big_cl = big_cluster_pick(p.big_cl, bP.data(), bna.data(), (int)bP.size(), &d.big_smem);
    if (d.big_cl == 0) {
      fprintf(stderr, "mixts_init: the device runs no thread-block cluster of the large-P propagation\n");
      delete h;
      return MIXTS_ERR_CUDA;
    }
  }
  d.n_part_slots = (int)p.slot_type.size();
  d.precision = prm->precision;
  d.box = sys->box;
  d.rc = prm->r_cut;
  d.rc2 = prm->r_cut * prm->r_cut;
  d.alpha = prm->dsf_alpha;
  d.dsf_g = 2.0 * prm->dsf_alpha / sqrt(PI);
  d.dsf_erfc_rc_over_rc = erfc(prm->dsf_alpha * prm->r_cut) / prm->r_cut;
  d.dsf_cf = erfc(prm->dsf_alpha * prm->r_cut) / (prm->r_cut * prm->r_cut) +
             d.dsf_g * exp(-prm->dsf_alpha * prm->dsf_alpha * prm->r_cut * prm->r_cut) / prm->r_cut;
  d.dsf_tab = (const double*)(h->ws + p.o_dsf);
  d.dsf32 = (const float4*)(h->ws + p.o_dsf32);
  if (prm->coulomb == 1) {  // Ewald real space: erfc(a r)/r, no shift at r_cut
    d.dsf_erfc_rc_over_rc = 0.0;
    d.dsf_cf = 0.0;
  }
  d.coulomb = prm->coulomb;
  d.ew_kmax = prm->ewald_kmax;
  d.n_kvec = p.n_kvec;
  d.n_qatoms = p.n_kvec > 0 ? p.n_qatoms : 0;
  d.n_intra = p.n_intra;
  d.ew_ke = u.ke;
  d.ew_const = p.ew_const;
  d.ew_bg = p.ew_bg;
  d.ew_inv2a2 = prm->coulomb == 1 ? 1.0 / (2.0 * prm->dsf_alpha * prm->dsf_alpha) : 0.0;
  if (p.n_kvec > 0) {
    d.kvec = (const double4_32a*)(h->ws + p.o_kvec);
    d.kn = (const int4*)(h->ws + p.o_kn);
    d.qinfo = (const int4*)(h->ws + p.o_qinfo);
    d.qcharge = (const double*)(h->ws + p.o_qcharge);
    d.intra = (const int2*)(h->ws + p.o_intra);
    d.ew_phase = (double2*)(h->ws + p.o_ewphase);
    d.ew_cen = (double4_32a*)(h->ws + p.o_ewcen);
    d.ew_S = (double2*)(h->ws + p.o_ews);
    d.ew_ek = (double*)(h->ws + p.o_ewek);
  }
  d.full_list = prm->precision == MIXTS_FP32_FORCES ? 1 : 0;
  d.lgPmax_nb = p.n_classes > 0 ? p.cls_log2P[0] : 0;
  d.n_items32 = p.n_nonp << d.lgPmax_nb;
  d.dsf_nint = p.dsf_nint;
  d.dsf_base = (1023 + p.dsf_elo) << 6;
  d.dsf_smin = ldexp(1.0, p.dsf_elo);
  d.ps_tab = p.ps_tab.empty() ? nullptr : (const double*)(h->ws + p.o_pstab);
  d.ps_nint = p.ps_nint;
  d.ps_base = (1023 + p.ps_elo) << 6;
  d.ps_smin = ldexp(1.0, p.ps_elo);
  d.box_hi = (float)(rint(sys->box * 4096.0) / 4096.0);
  d.box_fix = llrint(sys->box * 281474976710656.0);
  d.screen_rc2 = (float)((prm->r_cut + 2e-3) * (prm->r_cut + 2e-3));
  d.dt = prm->dt;
  d.kcal = u.kcal;
  d.kB = u.kB;
  d.kT = u.kB * prm->T;
  d.seed = sys->seed;
  for (int t = 0; t < p.nt; ++t) {
    d.P[t] = sys->P_type[t];
    d.log2P[t] = ilog2(sys->P_type[t]);
    d.N[t] = p.N[t];
    d.off[t] = p.off[t];
    d.atoff[t] = p.atoff[t];
    d.pseudo[t] = sys->pseudo_type[t] ? 1 : 0;
    d.cm_off[t] = p.cm_off[t];
    d.mc_off[t] = p.mc_off[t];
    d.mass[t] = sys->bead_mass_type ? sys->bead_mass_type[t] : sys->mass_type[t];  // kinetic (bead) mass
  }
  for (int c = 0; c < p.n_classes; ++c) {
    d.cls_P[c] = p.cls_P[c];
    d.cls_log2P[c] = p.cls_log2P[c];
    d.cls_pos0[c] = p.cls_pos0[c];
    d.cls_n[c] = p.cls_n[c];
    d.cls_item0[c] = p.cls_item0[c];
  }
  unsigned char* w = h->ws;
  d.ainfo = (const AtomInfo*)(w + p.o_ainfo);
  d.pos_atom = (const int*)(w + p.o_pos_atom);
  d.pos_mol = (const int*)(w + p.o_pos_mol);
  d.atom_of_tk = (const int*)(w + p.o_atom_of_tk);
  h->ainfo_atom = (const AtomInfo*)(w + p.o_ainfo_atom);
  h->atom_is_pseudo = (const int*)(w + p.o_is_pseudo);
  d.pseudo_atom = (const int*)(w + p.o_pseudo_atom);
  d.pinfo = (const AtomInfo*)(w + p.o_pinfo);
  d.pairpar = (const PairPar*)(w + p.o_pairpar);
  d.pspar = (const PseudoPar*)(w + p.o_pspar);
  d.bitems = (const BondItem*)(w + p.o_bitems);
  d.bond_atoms = (const int*)(w + p.o_bond_atoms);
  d.bond_par = (const double*)(w + p.o_bond_par);
  d.ang_atoms = (const int*)(w + p.o_ang_atoms);
  d.ang_par = (const double*)(w + p.o_ang_par);
  d.cm = (const double*)(w + p.o_cm);
  d.mc = (const ModeCoef*)(w + p.o_mc);
  d.tiles = (const PropTile*)(w + p.o_tiles);
  h->slot_type = (const int*)(w + p.o_slot_type);
  d.slot_type = h->slot_type;
  d.ainfo_atom = h->ainfo_atom;
  d.atom_is_pseudo = h->atom_is_pseudo;
  d.q = sys->q;
  d.p = sys->p;
  d.f = sys->f;
  d.q_nm = (double*)(w + p.o_qnm);
  d.p_nm = (double*)(w + p.o_pnm);
  d.F_fix = (unsigned long long*)(w + p.o_ffix);
  d.Xw = (double4_32a*)(w + p.o_xw);
  d.Xi = (longlong4_32a*)(w + p.o_xi);
  d.Xf = (float4*)(w + p.o_xf);
  d.Xl = (float4*)(w + p.o_xl);
  d.Xd = p.o_xd ? (float4*)(w + p.o_xd) : nullptr;
  d.XiA = p.o_xia ? (longlong4_32a*)(w + p.o_xia) : nullptr;
  d.ref = (double*)(w + p.o_ref);
  d.refd = (double4_32a*)(w + p.o_refd);
  d.reff = (float4*)(w + p.o_reff);
  d.wrapn = (int4*)(w + p.o_wrapn);
  d.pos_of_atom = (const int*)(w + p.o_pos_of_atom);
  d.spread = (double*)(w + p.o_spread);
  d.p64_implicit = p.n_nonp <= P64_IMPLICIT_ROWS ? 1 : 0;
  pair_grids(p.nt, pair64_smem(d), p.dsf_nint, &d.pair_grid, &d.pair32_grid);
  h->full_grid64 = d.pair_grid;
  h->full_grid32 = d.pair32_grid;
  d.pseudo_chunks = prm->precision == MIXTS_FP32_FORCES ? 8 : 4;  // site-list slices per pseudo bead (measured)
  d.nl_cpl = 4;
  d.p32_lgt = LG_P32_TERMS;
  pair32w_plan(d);
  d.p64_nch = (p.nl_cap + P64_CH - 1) / P64_CH;  // at most: one lane group, P64_CH entries per item
  d.nl = (int*)(w + p.o_nl);
  d.nl_cnt = (int*)(w + p.o_nlcnt);
  d.nc = p.nc;
  d.cell_inv = p.nc > 0 ? (float)(p.nc / sys->box) : 0.0f;
  d.cell_start = (int*)(w + p.o_cstart);
  d.cell_atoms = (int*)(w + p.o_catoms);
  d.cell_ok = (int*)(w + p.o_cok);
  d.pitems = (int2*)(w + p.o_pitems);
  d.pctr = (int*)(w + p.o_pctr);
  d.nlB = p.o_nlb ? (float4*)(w + p.o_nlb) : nullptr;
  d.nlseg = p.o_nlseg ? (int*)(w + p.o_nlseg) : nullptr;
  d.box_lo = (float)(sys->box - (double)d.box_hi);
  d.pl = (int*)(w + p.o_pl);
  d.pl_cnt = (int*)(w + p.o_plcnt);
  d.thresh = (double*)(w + p.o_thresh);
  d.E_fix = (unsigned long long*)(w + p.o_efix);
  d.err = (int*)(w + p.o_err);
  d.step_ctr = (long long*)(w + p.o_step);
  d.heat = (double*)(w + p.o_heat);
  d.est = (double*)(w + p.o_est);
  d.parts = (double*)(w + p.o_parts);
  *out = h;
  return MIXTS_OK;
}

// Forces at the current positions. With the side stream (steps; not the
// per-phase timing mode) the bonded terms run beside the neighbour search
// and pair sweep, and the pseudopotential sweep beside the pair sweep once
// its list exists: every kernel adds into the fixed-point accumulators with
// integer atomics, so the sums are the same in any order.
static mixts_status eval_forces(mixts_handle h) {
  const Dev& d = h->d;
  cudaStream_t s = h->stream;
  h->list_valid = true;
  const bool par = h->side && !h->tm.on;
  if (par) {
    cudaEventRecord(h->ev_fork, s);
    cudaStreamWaitEvent(h->side, h->ev_fork, 0);
    h->kernels += launch_bonded(d, h->side, h->ainfo_atom);
  }
  phase(h, 0, [&] { return launch_nlist(d, s, h->atom_is_pseudo); });
  if (par) {
    cudaEventRecord(h->ev_list, s);
    cudaStreamWaitEvent(h->side, h->ev_list, 0);
    h->kernels += launch_pseudo(d, h->side);
  }
  if (h->fin_pending) {  // the previous step's finalisation clears the energy accumulators
    cudaStreamWaitEvent(s, h->ev_fin, 0);
    h->fin_pending = false;
  }
  phase(h, 1, [&] { return launch_pair(d, s) + launch_ewald(d, s); });
  if (par) {
    cudaEventRecord(h->ev_join, h->side);
    cudaStreamWaitEvent(s, h->ev_join, 0);
  } else {
    phase(h, 2, [&] { return launch_bonded(d, s, h->ainfo_atom); });
    phase(h, 3, [&] { return launch_pseudo(d, s); });
  }
  return cuda_check(h, cudaGetLastError(), "force launch");
}

// the side stream (with its fork, list and join events) of the force terms
// that run beside the pair sweep and of the large-P clusters, made by the
// step prologue (eager, before any capture; a bare force evaluation never
// makes it); without it everything runs in order on the handle's stream
static void ensure_side(mixts_handle h) {
  if (!h->side) {
    if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_list, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_post, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fin, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (h->side) cudaStreamDestroy(h->side);
      for (cudaEvent_t e : {h->ev_fork, h->ev_list, h->ev_join, h->ev_post})
        if (e) cudaEventDestroy(e);
      h->side = nullptr;
      h->ev_fork = h->ev_list = h->ev_join = h->ev_post = h->ev_fin = nullptr;
    }
  }
}

static void prop(mixts_handle h, int mode) {
  phase(h, 4, [&] { return launch_prop(h->d, h->stream, mode, h->side, h->ev_fork, h->ev_join); });
}

// step finalisation; with the side stream it runs there, beside the next
// step's neighbour search, and the next pair sweep (the first kernel that
// adds to the energy accumulators it clears) or the end of mixts_step waits
// for it
static void fin(mixts_handle h, int mode) {
  if (h->side && !h->tm.on) {
    cudaEventRecord(h->ev_post, h->stream);
    cudaStreamWaitEvent(h->side, h->ev_post, 0);
    h->kernels += launch_final(h->d, h->side, mode, h->slot_type);
    cudaEventRecord(h->ev_fin, h->side);
    h->fin_pending = true;
    return;
  }
  phase(h, 5, [&] { return launch_final(h->d, h->stream, mode, h->slot_type); });
}

static void fin_join(mixts_handle h) {
  if (h->fin_pending) {
    cudaStreamWaitEvent(h->stream, h->ev_fin, 0);
    h->fin_pending = false;
  }
}

mixts_status mixts_forces(mixts_handle h, double* energy_host) {
  if (!h) return MIXTS_ERR_ARG;
  if (!h->kids.empty()) {
    for (size_t i = 0; i < h->kids.size(); ++i) {
      mixts_status st = mixts_forces(h->kids[i], energy_host ? energy_host + i : nullptr);
      if (st != MIXTS_OK) return set_err(h, st, "system " + std::to_string(i) + ": " + h->kids[i]->err);
    }
    return MIXTS_OK;
  }
  // a fresh evaluation from the caller's q: clear the accumulators first
  cudaMemsetAsync(h->d.F_fix, 0, sizeof(unsigned long long) * 3 * (size_t)h->d.n_beads, h->stream);
  cudaMemsetAsync(h->d.E_fix, 0, sizeof(unsigned long long) * E_NSLOTS, h->stream);
  prop(h, PM_MIRROR);
  mixts_status st = eval_forces(h);
  if (st != MIXTS_OK) return st;
  phase(h, 6, [&] { return launch_forces_out(h->d, h->stream); });
  st = cuda_check(h, cudaGetLastError(), "forces out");
  if (st != MIXTS_OK) return st;
  h->nm_valid = false;
  h->f_valid = false;
  if (energy_host) {
    st = device_error(h);
    if (st != MIXTS_OK) return st;
    st = d2h(h, energy_host, h->d.est, sizeof(double), "energy");
  }
  return st;
}

// bring a handle to the steady state of the step loop: modes imported from
// the Cartesian state, forces at the current positions
static mixts_status step_prologue(mixts_handle h) {
  cudaStream_t s = h->stream;
  ensure_side(h);
  if (!h->nm_valid) {
    prop(h, PM_IMPORT);
    h->nm_valid = true;
    h->f_valid = false;
  }
  if (!h->f_valid) {
    cudaMemsetAsync(h->d.F_fix, 0, sizeof(unsigned long long) * 3 * (size_t)h->d.n_beads, s);
    cudaMemsetAsync(h->d.E_fix, 0, sizeof(unsigned long long) * E_NSLOTS, s);
    prop(h, PM_QCART);
    mixts_status st = eval_forces(h);
    if (st != MIXTS_OK) return st;
    h->f_valid = true;
  }
  return MIXTS_OK;
}

static mixts_status batch_step(mixts_handle h, int n_steps);
static mixts_status single_graph_steps(mixts_handle h, int n_steps, int* done);

mixts_status mixts_step(mixts_handle h, int n_steps) {
  if (!h || n_steps < 0) return MIXTS_ERR_ARG;
  if (n_steps == 0) return MIXTS_OK;
  if (!h->kids.empty()) return batch_step(h, n_steps);
  mixts_status st = step_prologue(h);
  if (st != MIXTS_OK) return st;
  if (!h->capturing && !h->tm.on && h->graph_steps > 0 && n_steps >= h->graph_steps) {
    int done = 0;
    if ((st = single_graph_steps(h, n_steps, &done)) != MIXTS_OK) return st;
    n_steps -= done;
    if (n_steps == 0) return MIXTS_OK;
  }
  prop(h, PM_START);
  fin(h, PM_START);
  for (int i = 1; i < n_steps; ++i) {
    eval_forces(h);
    prop(h, PM_END | PM_EST | PM_START);
    fin(h, PM_END | PM_EST | PM_START);
  }
  eval_forces(h);
  prop(h, PM_END | PM_EST | PM_PCART);
  fin(h, PM_END | PM_EST);
  fin_join(h);
  h->steps_done += n_steps;
  return cuda_check(h, cudaGetLastError(), "step launch");
}

mixts_status mixts_estimators(mixts_handle h, mixts_estimates* out) {
  if (!h || !out) return MIXTS_ERR_ARG;
  if (!h->kids.empty()) {
    for (size_t i = 0; i < h->kids.size(); ++i) {
      mixts_status st = mixts_estimators(h->kids[i], out + i);
      if (st != MIXTS_OK) return set_err(h, st, "system " + std::to_string(i) + ": " + h->kids[i]->err);
    }
    return MIXTS_OK;
  }
  mixts_status st = device_error(h);
  if (st != MIXTS_OK) return st;
  double e[EST_N];
  st = d2h(h, e, h->d.est, sizeof(e), "estimates");
  if (st != MIXTS_OK) return st;
  memset(out, 0, sizeof(*out));
  out->V = e[0];
  out->V_lj = e[1];
  out->V_coul = e[2];
  out->V_bond = e[3];
  out->V_angle = e[4];
  out->V_pseudo = e[5];
  out->KE_beads = e[6];
  out->E_spring = e[7];
  out->virial = e[8];
  out->T_beads = e[9];
  out->H_mix = e[10];
  out->heat = e[11];
  out->H_conserved = e[12];
  out->n_evals = e[13];
  out->n_pseudo_evals = e[14];
  out->n_lj_evals = e[16 + 4 * MT];
  out->step = (int64_t)e[15];
  for (int t = 0; t < h->d.n_types; ++t) {
    out->KE_prim[t] = e[16 + 4 * t];
    out->KE_cv[t] = e[16 + 4 * t + 1];
    out->Rg2[t] = e[16 + 4 * t + 2];
    out->E_spring_t[t] = e[16 + 4 * t + 3];
  }
  return MIXTS_OK;
}

mixts_status mixts_nlist(mixts_handle h, int kind, int* out3, long cap, long* n_out, double* thresh) {
  if (!h || !n_out || (kind != 0 && kind != 1)) return MIXTS_ERR_ARG;
  if (!h->kids.empty()) return set_err(h, MIXTS_ERR_ARG, "batched handle: query a member (mixts_batch_member)");
  mixts_status st = device_error(h);
  if (st != MIXTS_OK) return st;
  const Plan& p = h->plan;
  if (thresh) {
    double t4[4];
    if ((st = d2h(h, t4, h->d.thresh, sizeof(t4), "thresholds")) != MIXTS_OK) return st;
    thresh[0] = kind == 0 ? t4[0] : t4[2];
    thresh[1] = kind == 0 ? t4[1] : t4[3];
    thresh[2] = t4[3];
  }
  const int rows = kind == 0 ? p.n_nonp : p.n_pseudo;
  const int rcap = kind == 0 ? p.nl_cap : p.pl_cap;
  std::vector<int> cnt(std::max(1, rows)), ent((size_t)std::max(1, rows) * rcap);
  if (rows > 0) {
    st = d2h(h, cnt.data(), kind == 0 ? h->d.nl_cnt : h->d.pl_cnt, sizeof(int) * rows, "list counts");
    if (st == MIXTS_OK)
      st = d2h(h, ent.data(), kind == 0 ? h->d.nl : h->d.pl, sizeof(int) * (size_t)rows * rcap, "list copy");
    if (st != MIXTS_OK) return st;
  }
  long n = 0;
  for (int r = 0; r < rows; ++r) {
    const int owner = kind == 0 ? p.pos_atom[r] : p.pseudo_atom[r];
    const int c = std::min(cnt[r], rcap);
    for (int k = 0; k < c; ++k) {
      const int e = ent[(size_t)r * rcap + k];
      int partner;
      if (kind == 0) {  // (bead-0 row << 11) | (type << 7) | code
        const int t = (e >> 7) & 15, row0 = e >> 11;
        partner = p.atom_of_tk[p.atoff[t] + (row0 - p.off[t])];
      } else {          // (sorted position << 7) | code
        partner = p.pos_atom[e >> 7];
      }
      if (out3 && n < cap) {
        out3[3 * n] = owner;
        out3[3 * n + 1] = partner;
        out3[3 * n + 2] = e & 127;
      }
      ++n;
    }
  }
  *n_out = n;
  return (out3 && n > cap) ? set_err(h, MIXTS_ERR_ARG, "cap too small") : MIXTS_OK;
}

size_t mixts_state_size(mixts_handle h) {
  if (!h) return 0;
  if (!h->kids.empty()) {
    size_t n = 0;
    for (auto k : h->kids) n += mixts_state_size(k);
    return n;
  }
  return 64 + sizeof(double) * 6 * (size_t)h->d.n_beads;
}

mixts_status mixts_get_state(mixts_handle h, void* blob, size_t bytes) {
  if (!h || !blob || bytes < mixts_state_size(h)) return MIXTS_ERR_ARG;
  if (!h->kids.empty()) {  // members' blobs back to back
    unsigned char* b = (unsigned char*)blob;
    for (auto k : h->kids) {
      const size_t nk = mixts_state_size(k);
      mixts_status st = mixts_get_state(k, b, nk);
      if (st != MIXTS_OK) return set_err(h, st, k->err);
      b += nk;
    }
    return MIXTS_OK;
  }
  mixts_status st = device_error(h);
  if (st != MIXTS_OK) return st;
  if (!h->nm_valid) return set_err(h, MIXTS_ERR_STATE, "no mode-space state yet: call mixts_step first");
  unsigned char* b = (unsigned char*)blob;
  memset(b, 0, 64);
  const uint64_t magic = 0x4d49585453543031ull;  // "MIXTST01"
  const uint64_t nb = (uint64_t)h->d.n_beads;
  memcpy(b, &magic, 8);
  memcpy(b + 8, &nb, 8);
  const size_t n3 = sizeof(double) * 3 * nb;
  cudaMemcpyAsync(b + 16, h->d.step_ctr, 8, cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(b + 24, h->d.heat, 8, cudaMemcpyDeviceToHost, h->stream);
  cudaMemcpyAsync(b + 64, h->d.q_nm, n3, cudaMemcpyDeviceToHost, h->stream);
  return d2h(h, b + 64 + n3, h->d.p_nm, n3, "get state");
}

mixts_status mixts_set_state(mixts_handle h, const void* blob, size_t bytes) {
  if (!h || !blob || bytes < mixts_state_size(h)) return MIXTS_ERR_ARG;
  if (!h->kids.empty()) {
    const unsigned char* b = (const unsigned char*)blob;
    for (auto k : h->kids) {
      const size_t nk = mixts_state_size(k);
      mixts_status st = mixts_set_state(k, b, nk);
      if (st != MIXTS_OK) return set_err(h, st, k->err);
      b += nk;
    }
    return MIXTS_OK;
  }
  const unsigned char* b = (const unsigned char*)blob;
  uint64_t magic, nb;
  memcpy(&magic, b, 8);
  memcpy(&nb, b + 8, 8);
  if (magic != 0x4d49585453543031ull || nb != (uint64_t)h->d.n_beads)
    return set_err(h, MIXTS_ERR_STATE, "state blob does not match this system");
  cudaStream_t s = h->stream;
  const size_t n3 = sizeof(double) * 3 * nb;
  cudaMemcpyAsync(h->d.step_ctr, b + 16, 8, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->d.heat, b + 24, 8, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->d.q_nm, b + 64, n3, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->d.p_nm, b + 64 + n3, n3, cudaMemcpyHostToDevice, s);
  mixts_status st = cuda_check(h, cudaStreamSynchronize(s), "set state");
  if (st != MIXTS_OK) return st;
  h->nm_valid = true;
  h->f_valid = false;
  h->list_valid = false;
  // Cartesian q, p for the caller
  prop(h, PM_QCART | PM_PCART);
  return cuda_check(h, cudaGetLastError(), "set state export");
}

mixts_status mixts_reload(mixts_handle h) {
  if (!h) return MIXTS_ERR_ARG;
  for (auto k : h->kids) mixts_reload(k);
  h->list_valid = false;
  h->nm_valid = false;
  h->f_valid = false;
  return MIXTS_OK;
}

mixts_status mixts_set_timing(mixts_handle h, int on) {
  if (!h) return MIXTS_ERR_ARG;
  for (auto k : h->kids) mixts_set_timing(k, on);
  timer_fold(h);
  if (on) {
    for (int i = 0; i < MIXTS_N_PHASES; ++i) {
      h->tm.ms[i] = 0.0;
      h->tm.calls[i] = 0;
    }
  }
  h->tm.on = on != 0;
  return MIXTS_OK;
}

mixts_status mixts_get_timing(mixts_handle h, double* ms, long long* calls, long long* kernels) {
  if (!h) return MIXTS_ERR_ARG;
  timer_fold(h);
  for (int i = 0; i < MIXTS_N_PHASES; ++i) {
    if (ms) ms[i] = h->tm.ms[i];
    if (calls) calls[i] = h->tm.calls[i];
  }
  if (kernels) *kernels = h->kernels;
  for (auto k : h->kids) {  // members' sums (eager launches) plus the graph launches
    double km[MIXTS_N_PHASES];
    long long kc[MIXTS_N_PHASES], kk = 0;
    mixts_status st = mixts_get_timing(k, km, kc, &kk);
    if (st != MIXTS_OK) return st;
    for (int i = 0; i < MIXTS_N_PHASES; ++i) {
      if (ms) ms[i] += km[i];
      if (calls) calls[i] += kc[i];
    }
    if (kernels) *kernels += kk;
  }
  return cuda_check(h, cudaStreamSynchronize(h->stream), "timing");
}

mixts_status mixts_gaussians(mixts_handle h, uint32_t step, uint32_t stage, uint64_t dof0, long n, float* out) {
  if (!h || !out || n < 0) return MIXTS_ERR_ARG;
  if (!h->kids.empty()) return set_err(h, MIXTS_ERR_ARG, "batched handle: query a member (mixts_batch_member)");
  h->kernels += launch_gauss(h->d, h->stream, step, stage, dof0, n, out);
  return cuda_check(h, cudaGetLastError(), "gaussians");
}

void mixts_destroy(mixts_handle h) {
  if (!h) return;
  if (h->kids.empty() && (h->gexec || h->cap)) {
    cudaStreamSynchronize(h->stream);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->cap) cudaStreamDestroy(h->cap);
    h->gexec = nullptr;
    h->cap = nullptr;
  }
  if (!h->kids.empty()) {
    cudaStreamSynchronize(h->stream);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    for (auto e : h->fev) cudaEventDestroy(e);
    for (auto f : h->fork) cudaStreamDestroy(f);
    if (h->cap) cudaStreamDestroy(h->cap);
    for (auto k : h->kids) mixts_destroy(k);
    h->kids.clear();
  }
  if (!h->tm.pool.empty()) {
    cudaStreamSynchronize(h->stream);
    for (auto e : h->tm.pool) cudaEventDestroy(e);
  }
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_list) cudaEventDestroy(h->ev_list);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_post) cudaEventDestroy(h->ev_post);
  if (h->ev_fin) cudaEventDestroy(h->ev_fin);
  delete h;
}

const char* mixts_last_error(mixts_handle h) { return h ? h->err.c_str() : "NULL handle"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched variant: many independent systems of uneven size advanced together.
// Each system keeps its own sub-context (tables, lists, state) in its slice
// of the workspace; a step of the whole batch is one CUDA graph launch whose
// parallel branches carry the systems' kernel chains (longest first, greedy
// to the least-loaded branch). The shapes of that graph -- branch count,
// persistent force-kernel CTAs per system, list candidates per warp -- come
// from an autotuner that times captured candidates on the live batch.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t BATCH_ALIGN = 256;
size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// estimated force work of a member: pair items times list capacity
double member_work(const mixts_ctx* k) {
  const Dev& d = k->d;
  const double items = d.precision == MIXTS_FP32_FORCES ? (double)d.n_items32 : (double)d.n_pitems;
  return items * (double)d.nl_cap + (double)d.n_ppitems * d.pl_cap + 1.0;
}

// apply a tuning to every member: force grids shared out by work
void apply_tuning(mixts_handle h, const mixts_batch_tuning& t) {
  double W = 0.0;
  for (auto k : h->kids) W += member_work(k);
  for (auto k : h->kids) {
    const double share = member_work(k) / W;
    const int g64 = (int)ceil(t.grid_scale * k->full_grid64 * share);
    const int g32 = (int)ceil(t.grid_scale * k->full_grid32 * share);
    k->d.pair_grid = std::max(1, std::min(k->full_grid64, g64));
    k->d.pair32_grid = std::max(1, std::min(k->full_grid32, g32));
    k->d.nl_cpl = t.nl_cpl;
    k->d.p32_lgt = t.item_lg_terms > 0 ? t.item_lg_terms : LG_P32_TERMS;
  }
  h->tune = t;
}

void drop_graph(mixts_handle h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
  h->g_steps = 0;
  h->g_kernels = 0;
}
}  // namespace

// the batch's own region after the members: Dev records and block prefixes
static size_t batch_region_bytes(int n_sys) {
  return round_up(sizeof(Dev) * (size_t)n_sys, BATCH_ALIGN) + round_up(sizeof(int) * BK_KINDS * (size_t)(n_sys + 1), BATCH_ALIGN);
}

static size_t batch_workspace_size(const mixts_system* sys, int n_sys, const mixts_params* prm) {
  size_t total = 0;
  for (int i = 0; i < n_sys; ++i) {
    const size_t n = mixts_workspace_size(sys + i, 1, prm);
    if (n == 0) return 0;
    total += round_up(n, BATCH_ALIGN);
  }
  return total + batch_region_bytes(n_sys) + BATCH_ALIGN;
}

// every member can run the one-launch-per-phase step: no pseudo particle, no
// type beyond the fused small-P propagation, damped-shifted-force Coulomb
static bool batch_persistent_ok(mixts_handle h) {
  for (auto k : h->kids) {
    const Dev& d = k->d;
    if (d.n_pseudo > 0 || d.coulomb != 0) return false;
    for (int t = 0; t < d.n_types; ++t)
      if (d.P[t] > SMALL_P && d.N[t] > 0) return false;
  }
  return true;
}

// upload the members' Dev records (after the current tuning) and the block
// prefixes of every batched kernel
static mixts_status batch_upload(mixts_handle h) {
  const int nm = (int)h->kids.size();
  std::vector<Dev> devs(nm);
  std::vector<int> pfx((size_t)BK_KINDS * (nm + 1), 0);
  BatchGeom& g = h->geom;
  g = BatchGeom{};
  g.nm = nm;
  g.precision = h->kids[0]->d.precision;
  for (int m = 0; m < nm; ++m) {
    devs[m] = h->kids[m]->d;
    int c[BK_KINDS];
    batch_block_counts(devs[m], c);
    for (int k = 0; k < BK_KINDS; ++k) pfx[(size_t)k * (nm + 1) + m + 1] = pfx[(size_t)k * (nm + 1) + m] + c[k];
    g.prop_smem = std::max(g.prop_smem, batch_prop_smem(devs[m]));
    g.pair_smem = std::max(g.pair_smem, devs[m].precision == MIXTS_FP32_FORCES
                                            ? (size_t)8 * sizeof(float) * (size_t)devs[m].dsf_nint
                                            : pair64_smem(devs[m]));
  }
  for (int k = 0; k < BK_KINDS; ++k) g.blocks[k] = pfx[(size_t)k * (nm + 1) + nm];
  g.devs = (const Dev*)h->bdev;
  g.pfx = h->bpfx;
  cudaError_t e = cudaMemcpyAsync(h->bdev, devs.data(), sizeof(Dev) * nm, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->bpfx, pfx.data(), sizeof(int) * pfx.size(), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // the host copies die here
  return cuda_check(h, e, "batch upload");
}

static mixts_status batch_init(const mixts_system* sys, int n_sys, const mixts_params* prm, void* workspace,
                               size_t ws_bytes, void* stream, mixts_handle* out) {
  *out = nullptr;
  if (!workspace || ((uintptr_t)workspace & 255)) return MIXTS_ERR_WORKSPACE;
  mixts_handle h = new mixts_ctx();
  cudaGetDevice(&h->device);
  h->stream = (cudaStream_t)stream;
  h->ws = (unsigned char*)workspace;
  size_t off = 0;
  for (int i = 0; i < n_sys; ++i) {
    const size_t n = mixts_workspace_size(sys + i, 1, prm);
    if (n == 0 || off + n > ws_bytes) {
      mixts_destroy(h);
      return n == 0 ? MIXTS_ERR_ARG : MIXTS_ERR_WORKSPACE;
    }
    mixts_handle k = nullptr;
    const mixts_status st = mixts_init(sys + i, 1, prm, h->ws + off, ws_bytes - off, stream, &k);
    if (st != MIXTS_OK) {
      fprintf(stderr, "mixts_init: batch member %d rejected\n", i);
      mixts_destroy(h);
      return st;
    }
    k->graph_steps = 0;  // members are captured into the batch graph, never on their own
    // FP32 members take the gather sweep: in one launch for the whole batch
    // the window sweep's 1024-thread CTAs, sized by the largest member's
    // stage, ran slower (2.36 against 1.54 ms per step for 64 members)
    k->d.p32w = 0;
    h->kids.push_back(k);
    off += round_up(n, BATCH_ALIGN);
  }
  if (off + batch_region_bytes(n_sys) > ws_bytes) {
    mixts_destroy(h);
    return MIXTS_ERR_WORKSPACE;
  }
  h->bdev = h->ws + off;
  h->bpfx = (int*)(h->ws + off + round_up(sizeof(Dev) * (size_t)n_sys, BATCH_ALIGN));
  mixts_batch_tuning t{};
  t.grid_scale = 2.0;
  t.streams = std::min(n_sys, 16);
  t.nl_cpl = 4;
  t.steps_per_launch = 10;
  t.persistent = batch_persistent_ok(h) ? 1 : 0;
  t.item_lg_terms = LG_P32_TERMS;
  apply_tuning(h, t);
  *out = h;
  return MIXTS_OK;
}

// one launch per phase for all members: steps_per_launch steps of the
// member step sequence (mixts_step), every kernel serving all members
static mixts_status batch_capture_persistent(mixts_handle h) {
  mixts_status st = batch_upload(h);
  if (st != MIXTS_OK) return st;
  const int K = std::max(1, h->tune.steps_per_launch);
  if (!h->cap) {
    st = cuda_check(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "capture stream");
    if (st != MIXTS_OK) return st;
  }
  ensure_side(h);
  st = cuda_check(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (st != MIXTS_OK) return st;
  const BatchGeom& g = h->geom;
  cudaStream_t s = h->cap;
  long long nk = 0;
  if (h->side) {
    // as a single handle's step: each step's finalisation and the next
    // step's bonded terms run on the side stream beside the neighbour
    // search (and the bonded terms beside the pair sweep); the pair sweep
    // waits for the finalisation (it clears the energy accumulators), the
    // propagation for both
    nk += launch_step_batched(g, s, PM_START, 1);
    int fmode = PM_START;
    for (int i = 0; i < K; ++i) {
      cudaEventRecord(h->ev_post, s);
      cudaStreamWaitEvent(h->side, h->ev_post, 0);
      nk += launch_step_batched(g, h->side, fmode, 2);
      cudaEventRecord(h->ev_fin, h->side);
      nk += launch_forces_batched_part(g, h->side, 2);
      cudaEventRecord(h->ev_join, h->side);
      nk += launch_forces_batched_part(g, s, 0);
      cudaStreamWaitEvent(s, h->ev_fin, 0);
      nk += launch_forces_batched_part(g, s, 1);
      cudaStreamWaitEvent(s, h->ev_join, 0);
      fmode = i + 1 < K ? (PM_END | PM_EST | PM_START) : (PM_END | PM_EST | PM_PCART);
      nk += launch_step_batched(g, s, fmode, 1);
    }
    cudaEventRecord(h->ev_post, s);
    cudaStreamWaitEvent(h->side, h->ev_post, 0);
    nk += launch_step_batched(g, h->side, fmode, 2);
    cudaEventRecord(h->ev_fin, h->side);
    cudaStreamWaitEvent(s, h->ev_fin, 0);
  } else {
    nk += launch_step_batched(g, s, PM_START);
    for (int i = 0; i < K; ++i) {
      nk += launch_forces_batched(g, s);
      nk += launch_step_batched(g, s, i + 1 < K ? (PM_END | PM_EST | PM_START) : (PM_END | PM_EST | PM_PCART));
    }
  }
  cudaGraph_t gr = nullptr;
  st = cuda_check(h, cudaStreamEndCapture(h->cap, &gr), "end capture");
  if (st == MIXTS_OK) st = cuda_check(h, cudaGraphInstantiate(&h->gexec, gr, 0), "graph instantiate");
  if (gr) cudaGraphDestroy(gr);
  if (st != MIXTS_OK) {
    drop_graph(h);
    return st;
  }
  h->g_steps = K;
  h->g_kernels = nk;
  return MIXTS_OK;
}

// capture steps_per_launch steps of every member into one executable graph
static mixts_status batch_capture(mixts_handle h) {
  drop_graph(h);
  if (h->tune.persistent && batch_persistent_ok(h)) return batch_capture_persistent(h);
  const mixts_batch_tuning& t = h->tune;
  const int S = std::max(1, std::min(t.streams, (int)h->kids.size()));
  const int K = std::max(1, t.steps_per_launch);
  if (!h->cap) {
    mixts_status st = cuda_check(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "capture stream");
    if (st != MIXTS_OK) return st;
  }
  while ((int)h->fork.size() < S) {
    cudaStream_t f;
    mixts_status st = cuda_check(h, cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking), "branch stream");
    if (st != MIXTS_OK) return st;
    h->fork.push_back(f);
  }
  while ((int)h->fev.size() < S + 1) {
    cudaEvent_t e;
    mixts_status st = cuda_check(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "branch event");
    if (st != MIXTS_OK) return st;
    h->fev.push_back(e);
  }
  // longest member first onto the least-loaded branch
  std::vector<int> order(h->kids.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return member_work(h->kids[a]) > member_work(h->kids[b]); });
  std::vector<double> load(S, 0.0);
  std::vector<long long> k0(h->kids.size()), s0(h->kids.size());
  for (size_t i = 0; i < h->kids.size(); ++i) {
    k0[i] = h->kids[i]->kernels;
    s0[i] = h->kids[i]->steps_done;
  }
  mixts_status st = cuda_check(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (st != MIXTS_OK) return st;
  cudaEventRecord(h->fev[0], h->cap);
  for (int b = 0; b < S; ++b) cudaStreamWaitEvent(h->fork[b], h->fev[0], 0);
  mixts_status step_st = MIXTS_OK;
  for (int i : order) {
    const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[b] += member_work(h->kids[i]);
    mixts_handle k = h->kids[i];
    cudaStream_t keep = k->stream;
    k->stream = h->fork[b];
    const mixts_status si = mixts_step(k, K);
    k->stream = keep;
    if (si != MIXTS_OK && step_st == MIXTS_OK) step_st = si;
  }
  for (int b = 0; b < S; ++b) {
    cudaEventRecord(h->fev[1 + b], h->fork[b]);
    cudaStreamWaitEvent(h->cap, h->fev[1 + b], 0);
  }
  cudaGraph_t g = nullptr;
  st = cuda_check(h, cudaStreamEndCapture(h->cap, &g), "end capture");
  long long nk = 0;
  for (size_t i = 0; i < h->kids.size(); ++i) {  // capture launched nothing
    nk += h->kids[i]->kernels - k0[i];
    h->kids[i]->kernels = k0[i];
    h->kids[i]->steps_done = s0[i];
  }
  if (st == MIXTS_OK && step_st != MIXTS_OK) st = set_err(h, step_st, "capture of a member step failed");
  if (st == MIXTS_OK) st = cuda_check(h, cudaGraphInstantiate(&h->gexec, g, 0), "graph instantiate");
  if (g) cudaGraphDestroy(g);
  if (st != MIXTS_OK) {
    drop_graph(h);
    return st;
  }
  h->g_steps = K;
  h->g_kernels = nk;
  return MIXTS_OK;
}

// eager batched steps with one launch per phase for all members, each
// phase timed on the batch handle's events (the timing mode of a batch that
// runs its graph that way)
static mixts_status batch_step_eager_persistent(mixts_handle h, int n_steps) {
  mixts_status st;
  for (auto k : h->kids)
    if ((st = step_prologue(k)) != MIXTS_OK) return set_err(h, st, k->err);
  if ((st = batch_upload(h)) != MIXTS_OK) return st;
  const BatchGeom& g = h->geom;
  cudaStream_t s = h->stream;
  phase(h, 4, [&] { return launch_step_batched(g, s, PM_START); });
  for (int i = 0; i < n_steps; ++i) {
    phase(h, 0, [&] { return launch_forces_batched_part(g, s, 0); });
    phase(h, 1, [&] { return launch_forces_batched_part(g, s, 1); });
    phase(h, 2, [&] { return launch_forces_batched_part(g, s, 2); });
    phase(h, 4, [&] {
      return launch_step_batched(g, s, i + 1 < n_steps ? (PM_END | PM_EST | PM_START) : (PM_END | PM_EST | PM_PCART));
    });
  }
  for (auto k : h->kids) k->steps_done += n_steps;
  h->steps_done += n_steps;
  return cuda_check(h, cudaGetLastError(), "batched step launch");
}

static mixts_status batch_step(mixts_handle h, int n_steps) {
  mixts_status st;
  if (h->tm.on && h->tune.persistent && batch_persistent_ok(h)) return batch_step_eager_persistent(h, n_steps);
  bool timing = false;
  for (auto k : h->kids) timing = timing || k->tm.on;
  if (timing || n_steps < h->tune.steps_per_launch) {  // eager, member by member
    for (auto k : h->kids)
      if ((st = mixts_step(k, n_steps)) != MIXTS_OK) return set_err(h, st, k->err);
    return MIXTS_OK;
  }
  for (auto k : h->kids)
    if ((st = step_prologue(k)) != MIXTS_OK) return set_err(h, st, k->err);
  if (!h->gexec && (st = batch_capture(h)) != MIXTS_OK) return st;
  const int reps = n_steps / h->g_steps, rem = n_steps % h->g_steps;
  for (int r = 0; r < reps; ++r) {
    st = cuda_check(h, cudaGraphLaunch(h->gexec, h->stream), "graph launch");
    if (st != MIXTS_OK) return st;
    h->kernels += h->g_kernels;
  }
  for (auto k : h->kids) k->steps_done += (long long)reps * h->g_steps;
  if (rem)
    for (auto k : h->kids)
      if ((st = mixts_step(k, rem)) != MIXTS_OK) return set_err(h, st, k->err);
  h->steps_done += n_steps;
  return MIXTS_OK;
}

// single handle: capture graph_steps steps once, replay it for the whole
// multiples of graph_steps in n_steps; the remainder runs eagerly
static mixts_status single_graph_steps(mixts_handle h, int n_steps, int* done) {
  *done = 0;
  mixts_status st;
  if (!h->gexec) {
    if (!h->cap && (st = cuda_check(h, cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "capture stream")) !=
                       MIXTS_OK)
      return st;
    const long long k0 = h->kernels, s0 = h->steps_done;
    cudaStream_t keep = h->stream;
    if ((st = cuda_check(h, cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture")) !=
        MIXTS_OK)
      return st;
    h->stream = h->cap;
    h->capturing = true;
    const mixts_status si = mixts_step(h, h->graph_steps);
    h->capturing = false;
    h->stream = keep;
    cudaGraph_t g = nullptr;
    st = cuda_check(h, cudaStreamEndCapture(h->cap, &g), "end capture");
    const long long nk = h->kernels - k0;
    h->kernels = k0;
    h->steps_done = s0;
    if (st == MIXTS_OK && si != MIXTS_OK) st = si;
    if (st == MIXTS_OK) st = cuda_check(h, cudaGraphInstantiate(&h->gexec, g, 0), "graph instantiate");
    if (g) cudaGraphDestroy(g);
    if (st != MIXTS_OK) {
      drop_graph(h);
      return st;
    }
    h->g_steps = h->graph_steps;
    h->g_kernels = nk;
  }
  const int reps = n_steps / h->g_steps;
  for (int r = 0; r < reps; ++r) {
    if ((st = cuda_check(h, cudaGraphLaunch(h->gexec, h->stream), "graph launch")) != MIXTS_OK) return st;
    h->kernels += h->g_kernels;
  }
  *done = reps * h->g_steps;
  h->steps_done += *done;
  return MIXTS_OK;
}

extern "C" MIXTS_API mixts_status mixts_set_graph(mixts_handle h, int steps_per_launch) {
  if (!h || steps_per_launch < 0) return MIXTS_ERR_ARG;
  drop_graph(h);
  if (!h->kids.empty()) {
    if (steps_per_launch == 0) return set_err(h, MIXTS_ERR_ARG, "a batched handle always steps by graph");
    h->tune.steps_per_launch = steps_per_launch;
  } else {
    h->graph_steps = steps_per_launch;
  }
  return MIXTS_OK;
}

extern "C" MIXTS_API mixts_status mixts_batch_member(mixts_handle h, int i, mixts_handle* out) {
  if (!h || !out || i < 0 || i >= (int)h->kids.size()) return MIXTS_ERR_ARG;
  *out = h->kids[i];
  return MIXTS_OK;
}

extern "C" MIXTS_API mixts_status mixts_batch_tune(mixts_handle h, int steps_per_launch, mixts_batch_tuning* out) {
  if (!h || h->kids.empty() || steps_per_launch < 1) return MIXTS_ERR_ARG;
  mixts_status st;
  for (auto k : h->kids)
    if (k->tm.on) return set_err(h, MIXTS_ERR_ARG, "switch timing off before tuning");
  for (auto k : h->kids)
    if ((st = step_prologue(k)) != MIXTS_OK) return set_err(h, st, k->err);
  // the trial steps advance the systems: save and restore the state
  std::vector<unsigned char> saved(mixts_state_size(h));
  if ((st = mixts_get_state(h, saved.data(), saved.size())) != MIXTS_OK) return st;
  std::vector<long long> done(h->kids.size());
  for (size_t i = 0; i < h->kids.size(); ++i) done[i] = h->kids[i]->steps_done;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int n = (int)h->kids.size();
  const int trial_steps = std::min(steps_per_launch, 2);
  auto time_shape = [&](mixts_batch_tuning t, double* ms) -> mixts_status {
    t.steps_per_launch = trial_steps;
    apply_tuning(h, t);
    mixts_status s2 = batch_capture(h);
    if (s2 != MIXTS_OK) return s2;
    cudaGraphLaunch(h->gexec, h->stream);  // warm
    cudaEventRecord(e0, h->stream);
    const int reps = 3;
    for (int r = 0; r < reps; ++r) cudaGraphLaunch(h->gexec, h->stream);
    cudaEventRecord(e1, h->stream);
    s2 = cuda_check(h, cudaEventSynchronize(e1), "tuning sync");
    if (s2 != MIXTS_OK) return s2;
    float f = 0.0f;
    cudaEventElapsedTime(&f, e0, e1);
    *ms = f / (reps * trial_steps);
    return MIXTS_OK;
  };
  mixts_batch_tuning best{};
  double best_ms = 1e30;
  int cands = 0;
  const double scales[] = {0.5, 1.0, 2.0, 4.0, 1e9};
  const int branches[] = {4, 8, 16, 32, 64};
  if (batch_persistent_ok(h)) {
    // one launch per phase: force-grid scale x FP32 work-item size (2^lgt terms)
    const bool fp32 = h->kids[0]->d.precision == MIXTS_FP32_FORCES;
    for (double sc : {0.5, 1.0, 2.0, 4.0})
      for (int lgt : {9, 10, 11}) {
        if (!fp32 && lgt != LG_P32_TERMS) continue;
        mixts_batch_tuning t{};
        t.grid_scale = sc;
        t.streams = 1;
        t.nl_cpl = 4;
        t.persistent = 1;
        t.item_lg_terms = lgt;
        double ms = 0.0;
        if ((st = time_shape(t, &ms)) != MIXTS_OK) goto done_tuning;
        ++cands;
        if (ms < best_ms) {
          best_ms = ms;
          best = t;
        }
      }
  } else {
    for (int S : branches) {
      if (S > n && S != branches[0]) continue;
      for (double sc : scales) {
        mixts_batch_tuning t{};
        t.grid_scale = sc;
        t.streams = std::min(S, n);
        t.nl_cpl = 4;
        t.persistent = 0;
        t.item_lg_terms = LG_P32_TERMS;
        double ms = 0.0;
        if ((st = time_shape(t, &ms)) != MIXTS_OK) goto done_tuning;
        ++cands;
        if (ms < best_ms) {
          best_ms = ms;
          best = t;
        }
      }
    }
  }
  for (int cpl : {2, 8}) {
    mixts_batch_tuning t = best;
    t.nl_cpl = cpl;
    double ms = 0.0;
    if ((st = time_shape(t, &ms)) != MIXTS_OK) goto done_tuning;
    ++cands;
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  best.steps_per_launch = steps_per_launch;
  best.ms_per_step = best_ms;
  best.candidates = cands;
  apply_tuning(h, best);
  drop_graph(h);
  st = MIXTS_OK;
done_tuning:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MIXTS_OK) return st;
  if ((st = mixts_set_state(h, saved.data(), saved.size())) != MIXTS_OK) return st;
  for (size_t i = 0; i < h->kids.size(); ++i) h->kids[i]->steps_done = done[i];
  for (auto k : h->kids)
    if ((st = step_prologue(k)) != MIXTS_OK) return set_err(h, st, k->err);
  if ((st = batch_capture(h)) != MIXTS_OK) return st;
  if (out) *out = h->tune;
  return MIXTS_OK;
}

// ---------------------------------------------------------------------------
// Radial distribution function.
// ---------------------------------------------------------------------------
namespace mx {
int launch_rdf(const Dev& d, cudaStream_t s, int ta, int tb, double dr, int nbins, unsigned long long* hist);
}

static mixts_status rdf_args(mixts_handle h, int ta, int tb, double dr, int nbins) {
  if (!h) return MIXTS_ERR_ARG;
  if (!h->kids.empty()) return set_err(h, MIXTS_ERR_ARG, "batched handle: query a member (mixts_batch_member)");
  const int nt = h->d.n_types;
  if (ta < 0 || tb < 0 || ta >= nt || tb >= nt || h->d.pseudo[ta] || h->d.pseudo[tb])
    return set_err(h, MIXTS_ERR_ARG, "rdf types must be site types");
  if (!(dr > 0.0) || nbins < 1 || nbins > MIXTS_RDF_MAX_BINS || nbins * dr > h->d.rc)
    return set_err(h, MIXTS_ERR_ARG, "rdf bins must lie inside r_cut");
  return MIXTS_OK;
}

extern "C" MIXTS_API mixts_status mixts_rdf_accumulate(mixts_handle h, int ta, int tb, double dr, int nbins,
                                                       unsigned long long* hist_dev) {
  mixts_status st = rdf_args(h, ta, tb, dr, nbins);
  if (st != MIXTS_OK) return st;
  if (!hist_dev) return MIXTS_ERR_ARG;
  if (!h->list_valid) return set_err(h, MIXTS_ERR_STATE, "no neighbour list at the current q: step or force first");
  phase(h, 6, [&] { return launch_rdf(h->d, h->stream, ta, tb, dr, nbins, hist_dev); });
  return cuda_check(h, cudaGetLastError(), "rdf launch");
}

extern "C" MIXTS_API mixts_status mixts_rdf_normalise(mixts_handle h, int ta, int tb, double dr, int nbins,
                                                      long long n_frames, const unsigned long long* hist_host,
                                                      double* g_host) {
  mixts_status st = rdf_args(h, ta, tb, dr, nbins);
  if (st != MIXTS_OK) return st;
  if (!hist_host || !g_host || n_frames < 1) return MIXTS_ERR_ARG;
  const double unit = ldexp(1.0, -h->d.lgPmax_nb);
  const double V = h->d.box * h->d.box * h->d.box;
  const double Na = h->d.N[ta], rho = (h->d.N[tb] - (ta == tb ? 1.0 : 0.0)) / V;
  for (int k = 0; k < nbins; ++k) {
    const double shell = 4.0 / 3.0 * PI * ((double)(k + 1) * (k + 1) * (k + 1) - (double)k * k * k) * dr * dr * dr;
    const double ideal = (double)n_frames * Na * rho * shell;
    g_host[k] = ideal > 0.0 ? (double)hist_host[k] * unit / ideal : 0.0;
  }
  return MIXTS_OK;
}

// ---------------------------------------------------------------------------
// Centroid velocity autocorrelation (ring-polymer molecular dynamics).
// ---------------------------------------------------------------------------
namespace mx {
int launch_vacf(const Dev& d, cudaStream_t s, int t, int n_lag, double* ring, double* acc, unsigned long long* cnt);
}

extern "C" MIXTS_API mixts_status mixts_vacf_accumulate(mixts_handle h, int type, int n_lag, double* ring_dev,
                                                        double* acc_dev, unsigned long long* cnt_dev) {
  if (!h || !ring_dev || !acc_dev || !cnt_dev) return MIXTS_ERR_ARG;
  if (!h->kids.empty()) return set_err(h, MIXTS_ERR_ARG, "batched handle: query a member (mixts_batch_member)");
  if (type < 0 || type >= h->d.n_types || h->d.N[type] == 0)
    return set_err(h, MIXTS_ERR_ARG, "type must hold atoms");
  if (n_lag < 1 || n_lag > 65535) return set_err(h, MIXTS_ERR_ARG, "n_lag must be 1..65535");
  if (!h->nm_valid) return set_err(h, MIXTS_ERR_STATE, "no mode-space state yet: call mixts_step first");
  phase(h, 6, [&] { return launch_vacf(h->d, h->stream, type, n_lag, ring_dev, acc_dev, cnt_dev); });
  return cuda_check(h, cudaGetLastError(), "vacf launch");
}

// ---------------------------------------------------------------------------
// Parameter gradient (the differentiation variant).
// ---------------------------------------------------------------------------
namespace {
// parameter derivatives (sigma, A [kcal/mol], b, q) of the raw
// pseudopotential V and of dV/dr at distance r
void pseudo_param_derivs_host(double ke, double q, double sig, double A, double b, double r, double* dv,
                              double* ddv) {
  const double sp = sqrt(PI), x = r / sig, ex = exp(-x * x), eb = exp(-r / b), erfx = erf(x);
  dv[0] = ke * q * (2.0 / sp) * ex / (sig * sig);
  ddv[0] = -ke * q * (2.0 / sp) * ex * 2.0 * r / (sig * sig * sig * sig);
  dv[1] = eb;
  ddv[1] = -eb / b;
  dv[2] = A * eb * r / (b * b);
  ddv[2] = A * eb * (b - r) / (b * b * b);
  dv[3] = -ke * erfx / r;
  ddv[3] = -ke * ((2.0 / (sig * sp)) * ex / r - erfx / (r * r));
}
}  // namespace

namespace mx {
int launch_grad(const Dev& d, cudaStream_t s, int ta, int tb, double ke, const double* pc, unsigned long long* acc,
                double grad_out, double* dvdq, bool want_theta);
}

extern "C" MIXTS_API mixts_status mixts_potential_grad(mixts_handle h, int ta, int tb, const double* theta,
                                                       double grad_out, double* V_host, double* dVdq_dev,
                                                       double* dVdtheta_host) {
  if (!h || !theta) return MIXTS_ERR_ARG;
  if (!h->kids.empty()) return set_err(h, MIXTS_ERR_ARG, "batched handle: query a member (mixts_batch_member)");
  const Plan& p = h->plan;
  const int nt = p.nt;
  if (ta < 0 || ta >= nt || tb < 0 || tb >= nt || ta == tb || h->d.pseudo[ta] || h->d.pseudo[tb])
    return set_err(h, MIXTS_ERR_ARG, "theta types must be two distinct site types");
  if (h->d.coulomb != 0) return set_err(h, MIXTS_ERR_ARG, "parameter gradients need the damped-shifted-force Coulomb");
  const double e0 = p.eps[ta * nt + ta];
  if (!(theta[0] > 0.0) || !(theta[2] > 0.0) || !(theta[3] > 0.0) || !(theta[5] > 0.0) ||
      !(e0 > 0.0 ? theta[7] > 0.0 : theta[7] >= 0.0))
    return set_err(h, MIXTS_ERR_ARG, "sigma and b must be positive, eps_aa positive (non-negative if 0 at init)");
  for (int k = 0; k < 8; ++k)
    if (!std::isfinite(theta[k])) return set_err(h, MIXTS_ERR_ARG, "theta must be finite");
  const Units u = units();
  const double rc = h->d.rc;
  // theta applied to a copy of the raw parameters
  std::vector<double> q = p.charge, eps = p.eps, psig = p.pp_sig, pA = p.pp_A, pb = p.pp_b;
  q[ta] = theta[6];
  // cross terms follow eps_ax = eps_ax0 sqrt(eps_aa / eps_aa0), fixed if eps_aa0 = 0
  const double scale = e0 > 0.0 ? sqrt(theta[7] / e0) : 1.0;
  for (int x = 0; x < nt; ++x)
    if (x != ta) {
      eps[ta * nt + x] = p.eps[ta * nt + x] * scale;
      eps[x * nt + ta] = p.eps[x * nt + ta] * scale;
    }
  eps[ta * nt + ta] = theta[7];
  psig[ta] = theta[0];
  pA[ta] = theta[1];
  pb[ta] = theta[2];
  psig[tb] = theta[3];
  pA[tb] = theta[4];
  pb[tb] = theta[5];
  std::vector<PairPar> pairpar(MT * MT, PairPar{0, 0, 1, 0, 0});
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      PairPar pp;
      pp.qq = u.ke * q[a] * q[b];
      pp.e4 = 4.0 * eps[a * nt + b];
      pp.s2 = p.sig[a * nt + b] * p.sig[a * nt + b];
      pp.vrc = pp.dvrc = 0.0;
      if (pp.e4 != 0.0) lj_at(pp.e4, pp.s2, rc, &pp.vrc, &pp.dvrc);
      pairpar[a * MT + b] = pp;
    }
  std::vector<PseudoPar> pspar(MT, PseudoPar{0, 1, 0, 1, 0, 0});
  std::vector<double> pc(8 * MT, 0.0);
  for (int t = 0; t < nt; ++t) {
    PseudoPar pp;
    pp.kq = u.ke * q[t];
    pp.sig = psig[t];
    pp.A = pA[t] * u.ev_kcal;
    pp.b = pb[t];
    pp.vrc = pp.dvrc = 0.0;
    if (pp.sig > 0.0 && pp.b > 0.0) {
      pseudo_at(pp, rc, &pp.vrc, &pp.dvrc);
      pseudo_param_derivs_host(u.ke, q[t], pp.sig, pp.A, pp.b, rc, &pc[8 * t], &pc[8 * t + 4]);
    }
    pspar[t] = pp;
  }
  cudaStream_t s = h->stream;
  unsigned char* w = h->ws;
  Dev dd = h->d;
  dd.pairpar = (const PairPar*)(w + p.o_pairpar_alt);
  dd.pspar = (const PseudoPar*)(w + p.o_pspar_alt);
  dd.precision = MIXTS_FP64;
  dd.full_list = 0;
  dd.p32w = 0;
  dd.ps_tab = nullptr;  // the tables hold the handle's parameters, not theta's
  unsigned long long* gacc = (unsigned long long*)(w + p.o_gacc);
  cudaMemcpyAsync(w + p.o_pairpar_alt, pairpar.data(), sizeof(PairPar) * MT * MT, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(w + p.o_pspar_alt, pspar.data(), sizeof(PseudoPar) * MT, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(w + p.o_pc, pc.data(), sizeof(double) * 8 * MT, cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(gacc, 0, sizeof(unsigned long long) * (2 * MT * MT + 8), s);
  cudaMemsetAsync(dd.F_fix, 0, sizeof(unsigned long long) * 3 * (size_t)dd.n_beads, s);
  cudaMemsetAsync(dd.E_fix, 0, sizeof(unsigned long long) * E_NSLOTS, s);
  // forward terms recomputed with theta (forces give dV/dq), then the adjoint sums
  phase(h, 4, [&] { return launch_prop(dd, s, PM_MIRROR); });
  phase(h, 0, [&] { return launch_nlist(dd, s, h->atom_is_pseudo); });
  phase(h, 1, [&] { return launch_pair(dd, s); });
  phase(h, 2, [&] { return launch_bonded(dd, s, h->ainfo_atom); });
  phase(h, 3, [&] { return launch_pseudo(dd, s); });
  // the adjoint sums over theta run only when dV/dtheta is asked for
  phase(h, 6, [&] {
    return launch_grad(dd, s, ta, tb, u.ke, (const double*)(w + p.o_pc), gacc, grad_out, dVdq_dev,
                       dVdtheta_host != nullptr);
  });
  phase(h, 6, [&] { return launch_forces_out(dd, s); });
  h->nm_valid = false;
  h->f_valid = false;
  mixts_status st = device_error(h);
  if (st != MIXTS_OK) return st;
  if (V_host && (st = d2h(h, V_host, h->d.est, sizeof(double), "potential")) != MIXTS_OK) return st;
  if (dVdtheta_host) {
    std::vector<long long> g(2 * MT * MT + 8);
    st = d2h(h, g.data(), gacc, sizeof(long long) * g.size(), "grad");
    if (st != MIXTS_OK) return st;
    auto SG = [&](int a, int b) { return (double)g[2 * (a * MT + b)] * EINV; };
    auto SL = [&](int a, int b) { return (double)g[2 * (a * MT + b) + 1] * EINV; };
    const long long* gp = g.data() + 2 * MT * MT;
    double out[8];
    out[0] = (double)gp[0] * EINV;
    out[1] = (double)gp[1] * EINV * u.ev_kcal;
    out[2] = (double)gp[2] * EINV;
    out[3] = (double)gp[4] * EINV;
    out[4] = (double)gp[5] * EINV * u.ev_kcal;
    out[5] = (double)gp[6] * EINV;
    // V_coul = sum over type pairs of k_e q_t q_u G_tu: linear in q_a
    double dq = (double)gp[3] * EINV;
    for (int x = 0; x < nt; ++x) {
      if (x == ta)
        dq += u.ke * 2.0 * q[ta] * SG(ta, ta);
      else
        dq += u.ke * q[x] * (SG(ta, x) + SG(x, ta));
    }
    out[6] = dq;
    // V_LJ = sum over type pairs of eps_tu U_tu, U at unit epsilon
    double de = SL(ta, ta);
    if (e0 > 0.0)
      for (int x = 0; x < nt; ++x)
        if (x != ta) de += eps[ta * nt + x] / (2.0 * theta[7]) * (SL(ta, x) + SL(x, ta));
    out[7] = de;
    for (int k = 0; k < 8; ++k) dVdtheta_host[k] = grad_out * out[k];
  }
  return MIXTS_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free force evaluation.
//
// For callers that cannot allocate device memory: plugins whose host
// framework owns every device byte through its own pool (a stray cudaMalloc
// fails or fragments it), and embedded or real-time drivers that forbid
// device allocation after start-up. mixts_forces_noalloc evaluates the forces with all of its device
// scratch (tables, neighbour lists, accumulators) carved from one file-scope
// static array of MIXTS_NOALLOC_MAX_BYTES. Every GPU that loads this library
// holds that array until the process exits. Host-side bookkeeping still uses
// ordinary host memory. The first call on a device looks up the array's
// address there, so that call belongs before any stream capture.
// ---------------------------------------------------------------------------
namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
// Host code must not use &g_noalloc_scratch as a device address: the symbol
// names a host-side stand-in. Each device's address comes from
// cudaGetSymbolAddress, taken once per device with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[MIXTS_NOALLOC_MAX_BYTES];
void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

mixts_status noalloc_base(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) return MIXTS_ERR_CUDA;
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      fprintf(stderr, "mixts_forces_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
      return MIXTS_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return MIXTS_OK;
}
}  // namespace

extern "C" MIXTS_API mixts_status mixts_forces_noalloc(const mixts_system* sys_in, const mixts_params* prm,
                                                       void* stream, double* energy_host) {
  if (!sys_in || !prm) return MIXTS_ERR_ARG;
  // A force evaluation neither reads nor writes momenta, so a caller without
  // a momentum array may pass p = NULL; the handle then points p at f, which
  // no kernel of this path touches through p.
  mixts_system sys = *sys_in;
  if (!sys.p) sys.p = sys.f;
  const size_t need = mixts_workspace_size(&sys, 1, prm);
  if (need == 0) return MIXTS_ERR_ARG;
  if (need > (size_t)MIXTS_NOALLOC_MAX_BYTES) {
    fprintf(stderr, "mixts_forces_noalloc: system needs %zu bytes of scratch, the static maximum is %zu\n", need,
            (size_t)MIXTS_NOALLOC_MAX_BYTES);
    return MIXTS_ERR_WORKSPACE;
  }
  void* base = nullptr;
  mixts_status st = noalloc_base(&base);
  if (st != MIXTS_OK) return st;
  // mixts_init uploads the tables and clears every accumulator, list counter
  // and flag in the scratch, so nothing carries over from the previous call
  mixts_handle h = nullptr;
  st = mixts_init(&sys, 1, prm, base, (size_t)MIXTS_NOALLOC_MAX_BYTES, stream, &h);
  if (st != MIXTS_OK) return st;
  st = mixts_forces(h, energy_host);
  // without an energy pointer mixts_forces does not synchronise: wait here and
  // read the device error word (list overflow, non-finite forces, box too
  // small) before the handle that locates it goes away
  if (st == MIXTS_OK && !energy_host) st = device_error(h);
  if (st != MIXTS_OK) fprintf(stderr, "mixts_forces_noalloc: %s\n", h->err.c_str());
  mixts_destroy(h);
  return st;
}
