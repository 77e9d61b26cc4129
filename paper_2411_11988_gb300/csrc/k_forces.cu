// k_forces.cu -- neighbour search and the mixTS force sweep.
//
// Pair terms of Eq. (mts-hamiltonian): the pair (i, j) with P_i >= P_j is
// owned by i (the finer ring polymer), and bead b of i meets bead
// floor(b P_j / P_i) = b >> (log2 P_i - log2 P_j) of j with weight 1/P_i.
// Work item = (owner atom i, bead b of i): one warp walks i's list row,
// lanes over entries. Reaction forces on the partner beads go to a 64-bit
// fixed-point accumulator, so the result is independent of atomic order.
#include <math.h>

#include "mixts_internal.cuh"

namespace mx {

// ---------------------------------------------------------------------------
// neighbour list
//
// Definition (integer output, reproduced bit for bit by any IEEE machine):
//   r_a  = q_{a,0} - L floor(q_{a,0} / L)
//   dmax = max over non-pseudo beads of |q_{a,b} - q_{a,0}|
//   R    = r_cut + 2 dmax
//   keep (owner, other, n), n in [-2,2]^3, if
//        ((r_o - r_w) + n L)^2 summed x, y, z left to right  <  R * R
//   except same-molecule n = 0. Owner = finer atom; between equal bead
//   counts the lower sorted position when the positions sum to an even
//   number, the higher one otherwise (balances the rows).
// A binary32 screen with a rigorous error margin settles all but the
// boundary band; the band is decided by the exact binary64 sequence.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double exact_d2(double dlx, double dly, double dlz, int nx, int ny, int nz,
                                           double L) {
  const double dx = __dadd_rn(dlx, __dmul_rn((double)nx, L));
  const double dy = __dadd_rn(dly, __dmul_rn((double)ny, L));
  const double dz = __dadd_rn(dlz, __dmul_rn((double)nz, L));
  double d2 = __dmul_rn(dx, dx);
  d2 = __dadd_rn(d2, __dmul_rn(dy, dy));
  d2 = __dadd_rn(d2, __dmul_rn(dz, dz));
  return d2;
}

// error bound of the binary32 screen (see the derivation beside the list
// definition in the design notes): per-dimension error <= 8 * 2^-24 L.
__device__ __forceinline__ float screen_margin(double L, double R) {
  const double del = 8.0 * 5.9604644775390625e-8 * L;
  const double e2 = 2.0 * 1.7320508075688772 * R * del + 3.0 * del * del + 4.0 * 5.9604644775390625e-8 * R * R;
  return (float)(4.0 * e2 + 1e-9);
}

// max spread over atoms whose pseudo flag equals want
__device__ double reduce_spread_kind(const Dev& d, const int* atom_is_pseudo, int want, double* red) {
  double m = 0.0;
  const int n = d.n_atoms * d.spread_slots;
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    const int atom = a / d.spread_slots;
    if (atom_is_pseudo[atom] == want) m = fmax(m, d.spread[a]);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

constexpr int NL_THREADS = 256;

__global__ void __launch_bounds__(NL_THREADS) k_nlist(Dev d, const int* atom_is_pseudo) {
  __shared__ double red[NL_THREADS / 32];
  __shared__ int cnt[NL_THREADS / 32];
  const double dmax = reduce_spread_kind(d, atom_is_pseudo, 0, red);
  const double L = d.box;
  const double R = __dadd_rn(d.rc, __dmul_rn(2.0, dmax));
  const double R2 = __dmul_rn(R, R);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    d.thresh[0] = dmax;
    d.thresh[1] = R;
  }
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int i = blockIdx.x * (NL_THREADS / 32) + wib;
  if (lane == 0) cnt[wib] = 0;
  __syncwarp();
  if (i >= d.n_nonp) return;
  if (!(R < 2.0 * L)) {
    if (lane == 0) {
      atomicOr(d.err, ERR_BOX);
      d.nl_cnt[i] = 0;
    }
    return;
  }
  const float m2 = screen_margin(L, R);
  const float R2f = (float)R2;
  const float R2lo = R2f - m2, R2hi = R2f + m2;
  const float Lf = (float)L;
  const AtomInfo ai = d.ainfo[i];
  const int Pi = ai.log2P;
  const int ai_atom = d.pos_atom[i];
  const int moli = d.pos_mol[i];
  const double rix = d.ref[3 * ai_atom], riy = d.ref[3 * ai_atom + 1], riz = d.ref[3 * ai_atom + 2];
  const float rfx = (float)rix, rfy = (float)riy, rfz = (float)riz;
  int* row = d.nl + (size_t)i * d.nl_cap;
  for (int c = lane; c < d.n_nonp; c += 32) {
    if (c == i) continue;
    const int Pc = d.ainfo[c].log2P;
    bool own;
    if (Pi != Pc) {
      own = Pi > Pc;
    } else {
      const int lo = i < c ? i : c;
      own = (((i + c) & 1) == 0) ? (i == lo) : (i != lo);
    }
    if (!own) continue;
    const int ca = d.pos_atom[c];
    const double rcx = d.ref[3 * ca], rcy = d.ref[3 * ca + 1], rcz = d.ref[3 * ca + 2];
    const float dfx = (float)rcx - rfx, dfy = (float)rcy - rfy, dfz = (float)rcz - rfz;
    const bool same = d.pos_mol[c] == moli;
    // per-dimension candidate images
    const float Rlin = sqrtf(R2hi);
    for (int nx = -2; nx <= 2; ++nx) {
      const float ex = dfx + (float)nx * Lf;
      if (fabsf(ex) >= Rlin) continue;
      for (int ny = -2; ny <= 2; ++ny) {
        const float ey = dfy + (float)ny * Lf;
        if (fabsf(ey) >= Rlin) continue;
        for (int nz = -2; nz <= 2; ++nz) {
          const float ez = dfz + (float)nz * Lf;
          if (fabsf(ez) >= Rlin) continue;
          if (same && nx == 0 && ny == 0 && nz == 0) continue;
          const float d2f = ex * ex + ey * ey + ez * ez;
          bool keep;
          if (d2f < R2lo) {
            keep = true;
          } else if (d2f > R2hi) {
            keep = false;
          } else {
            const double dlx = __dsub_rn(rcx, rix), dly = __dsub_rn(rcy, riy), dlz = __dsub_rn(rcz, riz);
            keep = exact_d2(dlx, dly, dlz, nx, ny, nz, L) < R2;
          }
          if (keep) {
            const int slot = atomicAdd(&cnt[wib], 1);
            if (slot < d.nl_cap) row[slot] = (c << 7) | ((nx + 2) * 25 + (ny + 2) * 5 + (nz + 2));
          }
        }
      }
    }
  }
  __syncwarp();
  if (lane == 0) {
    const int n = cnt[wib];
    if (n > d.nl_cap) atomicOr(d.err, ERR_NLIST);
    d.nl_cnt[i] = n < d.nl_cap ? n : d.nl_cap;
  }
}

// pseudo-particle site list: one thread per (pseudo atom, site position)
__global__ void k_plist(Dev d, const int* atom_is_pseudo) {
  __shared__ double red[8];
  const double ds = reduce_spread_kind(d, atom_is_pseudo, 0, red);
  const double dp = reduce_spread_kind(d, atom_is_pseudo, 1, red);
  const double L = d.box;
  const double R = __dadd_rn(__dadd_rn(d.rc, ds), dp);
  const double R2 = __dmul_rn(R, R);
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    d.thresh[2] = dp;
    d.thresh[3] = R;
  }
  const int e = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.n_nonp) return;
  if (!(R < 2.0 * L)) {
    atomicOr(d.err, ERR_BOX);
    return;
  }
  const float m2 = screen_margin(L, R);
  const float R2f = (float)R2;
  const float R2lo = R2f - m2, R2hi = R2f + m2;
  const float Lf = (float)L;
  const float Rlin = sqrtf(R2hi);
  const int ea = d.pseudo_atom[e];
  const double rex = d.ref[3 * ea], rey = d.ref[3 * ea + 1], rez = d.ref[3 * ea + 2];
  const int ca = d.pos_atom[c];
  const double rcx = d.ref[3 * ca], rcy = d.ref[3 * ca + 1], rcz = d.ref[3 * ca + 2];
  const float dfx = (float)rcx - (float)rex, dfy = (float)rcy - (float)rey, dfz = (float)rcz - (float)rez;
  for (int nx = -2; nx <= 2; ++nx) {
    const float ex = dfx + (float)nx * Lf;
    if (fabsf(ex) >= Rlin) continue;
    for (int ny = -2; ny <= 2; ++ny) {
      const float ey = dfy + (float)ny * Lf;
      if (fabsf(ey) >= Rlin) continue;
      for (int nz = -2; nz <= 2; ++nz) {
        const float ez = dfz + (float)nz * Lf;
        if (fabsf(ez) >= Rlin) continue;
        const float d2f = ex * ex + ey * ey + ez * ez;
        bool keep;
        if (d2f < R2lo) {
          keep = true;
        } else if (d2f > R2hi) {
          keep = false;
        } else {
          const double dlx = __dsub_rn(rcx, rex), dly = __dsub_rn(rcy, rey), dlz = __dsub_rn(rcz, rez);
          keep = exact_d2(dlx, dly, dlz, nx, ny, nz, L) < R2;
        }
        if (keep) {
          const int slot = atomicAdd(&d.pl_cnt[e], 1);
          if (slot < d.pl_cap)
            d.pl[(size_t)e * d.pl_cap + slot] = (c << 7) | ((nx + 2) * 25 + (ny + 2) * 5 + (nz + 2));
          else
            atomicOr(d.err, ERR_PLIST);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// nonbonded pair sweep, FP64
// ---------------------------------------------------------------------------
constexpr int PAIR_THREADS = 256;

__device__ __forceinline__ void item_of_warp(const Dev& d, int w, int* pos, int* bead) {
  int c = 0;
  while (c + 1 < d.n_classes && w >= d.cls_item0[c + 1]) ++c;
  const int local = w - d.cls_item0[c];
  *bead = local / d.cls_n[c];
  *pos = d.cls_pos0[c] + (local - *bead * d.cls_n[c]);
}

__global__ void __launch_bounds__(PAIR_THREADS) k_pair64(Dev d) {
  __shared__ PairPar tab[MT * MT];
  __shared__ double3 sh[125];
  const int nt = d.n_types;
  for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) tab[e] = d.pairpar[(e / nt) * MT + (e % nt)];
  for (int e = threadIdx.x; e < 125; e += blockDim.x)
    sh[e] = make_double3((e / 25 - 2) * d.box, ((e / 5) % 5 - 2) * d.box, (e % 5 - 2) * d.box);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= d.n_pitems) return;
  int pos, b;
  item_of_warp(d, w, &pos, &b);
  const AtomInfo ai = d.ainfo[pos];
  const int row_i = ai.row0 + b * ai.stride;
  const double4_32a xi = d.Xw[row_i];
  const double wgt = 1.0 / (double)(1 << ai.log2P);
  const int cnt = d.nl_cnt[pos];
  const int* lst = d.nl + (size_t)pos * d.nl_cap;
  const double rc = d.rc, rc2 = d.rc2, al = d.alpha, al2 = d.alpha * d.alpha;
  const double erc = d.dsf_erfc_rc_over_rc, cf = d.dsf_cf, g = d.dsf_g;
  double fix = 0.0, fiy = 0.0, fiz = 0.0, elj = 0.0, ec = 0.0, vir = 0.0;
  int nev = 0;
  for (int e = lane; e < cnt; e += 32) {
    const int ent = lst[e];
    const int j = ent >> 7;
    const AtomInfo aj = d.ainfo[j];
    const int bj = b >> (ai.log2P - aj.log2P);
    const int row_j = aj.row0 + bj * aj.stride;
    const double4_32a xj = d.Xw[row_j];
    const double3 s = sh[ent & 127];
    const double dx = (xj.x - xi.x) + s.x;
    const double dy = (xj.y - xi.y) + s.y;
    const double dz = (xj.z - xi.z) + s.z;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 < rc2) {
      const PairPar pp = tab[ai.type * nt + aj.type];
      const double rinv = rsqrt(r2);
      const double r = r2 * rinv;
      const double rinv2 = rinv * rinv;
      double fr = 0.0;
      if (pp.e4 != 0.0) {
        const double sr2 = pp.s2 * rinv2;
        const double sr6 = sr2 * sr2 * sr2;
        const double sr12 = sr6 * sr6;
        elj += wgt * (pp.e4 * (sr12 - sr6) - pp.vrc - (r - rc) * pp.dvrc);
        fr += (6.0 * pp.e4 * (2.0 * sr12 - sr6) * rinv + pp.dvrc) * rinv;
      }
      if (pp.qq != 0.0) {
        const double erfc_r = erfc(al * r);
        const double ex = exp(-al2 * r2);
        ec += wgt * pp.qq * (erfc_r * rinv - erc + cf * (r - rc));
        fr += pp.qq * ((erfc_r * rinv + g * ex) * rinv2 - cf * rinv);
      }
      fr *= wgt;
      const double fx = fr * dx, fy = fr * dy, fz = fr * dz;  // force on j
      fix -= fx;
      fiy -= fy;
      fiz -= fz;
      vir += fr * r2;
      ++nev;
      fadd3(d.F_fix, row_j, fx, fy, fz, d.err);
    }
  }
  fix = warp_sum(fix);
  fiy = warp_sum(fiy);
  fiz = warp_sum(fiz);
  elj = warp_sum(elj);
  ec = warp_sum(ec);
  vir = warp_sum(vir);
  nev = warp_sumi(nev);
  if (lane == 0) {
    fadd3(d.F_fix, row_i, fix, fiy, fiz, d.err);
    eadd(d.E_fix, E_LJ, elj);
    eadd(d.E_fix, E_COUL, ec);
    eadd(d.E_fix, E_VIRIAL, vir);
    atomicAdd(d.E_fix + E_NEVAL, (unsigned long long)nev);
  }
}

// ---------------------------------------------------------------------------
// bonded terms: one thread per (term, fine slice)
// ---------------------------------------------------------------------------
__global__ void k_bonded(Dev d, const AtomInfo* ainfo_atom) {
  const int it = blockIdx.x * blockDim.x + threadIdx.x;
  double eb = 0.0, ea = 0.0, vir = 0.0;
  if (it < d.n_bitems) {
    const BondItem bi = d.bitems[it];
    const int s = bi.slice;
    if (bi.kind == 0) {
      const int a = d.bond_atoms[2 * bi.term], c = d.bond_atoms[2 * bi.term + 1];
      const AtomInfo A = ainfo_atom[a], Cc = ainfo_atom[c];
      const int lmax = A.log2P > Cc.log2P ? A.log2P : Cc.log2P;
      const double w = 1.0 / (double)(1 << lmax);
      const int ra = A.row0 + (s >> (lmax - A.log2P)) * A.stride;
      const int rcw = Cc.row0 + (s >> (lmax - Cc.log2P)) * Cc.stride;
      const double k = d.bond_par[2 * bi.term], r0 = d.bond_par[2 * bi.term + 1];
      const double dx = d.q[3 * (size_t)rcw] - d.q[3 * (size_t)ra];
      const double dy = d.q[3 * (size_t)rcw + 1] - d.q[3 * (size_t)ra + 1];
      const double dz = d.q[3 * (size_t)rcw + 2] - d.q[3 * (size_t)ra + 2];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      eb = w * 0.5 * k * (r - r0) * (r - r0);
      const double f = -w * k * (r - r0) / r;
      vir = f * r * r;
      fadd3(d.F_fix, rcw, f * dx, f * dy, f * dz, d.err);
      fadd3(d.F_fix, ra, -f * dx, -f * dy, -f * dz, d.err);
    } else {
      const int a1 = d.ang_atoms[3 * bi.term], o = d.ang_atoms[3 * bi.term + 1], a2 = d.ang_atoms[3 * bi.term + 2];
      const AtomInfo A1 = ainfo_atom[a1], O = ainfo_atom[o], A2 = ainfo_atom[a2];
      int lmax = A1.log2P > O.log2P ? A1.log2P : O.log2P;
      lmax = lmax > A2.log2P ? lmax : A2.log2P;
      const double w = 1.0 / (double)(1 << lmax);
      const int r1 = A1.row0 + (s >> (lmax - A1.log2P)) * A1.stride;
      const int ro = O.row0 + (s >> (lmax - O.log2P)) * O.stride;
      const int r2 = A2.row0 + (s >> (lmax - A2.log2P)) * A2.stride;
      const double k = d.ang_par[2 * bi.term], th0 = d.ang_par[2 * bi.term + 1];
      double u[3], v[3];
      for (int x = 0; x < 3; ++x) {
        u[x] = d.q[3 * (size_t)r1 + x] - d.q[3 * (size_t)ro + x];
        v[x] = d.q[3 * (size_t)r2 + x] - d.q[3 * (size_t)ro + x];
      }
      const double uu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      const double vv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      double cs = (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) / (uu * vv);
      cs = fmin(1.0, fmax(-1.0, cs));
      const double th = acos(cs);
      const double sn = sqrt(1.0 - cs * cs);
      ea = w * 0.5 * k * (th - th0) * (th - th0);
      const double pref = w * k * (th - th0) / sn;
      double f1[3], f2[3];
      for (int x = 0; x < 3; ++x) {
        f1[x] = pref * (v[x] / (uu * vv) - cs * u[x] / (uu * uu));
        f2[x] = pref * (u[x] / (uu * vv) - cs * v[x] / (vv * vv));
      }
      vir = f1[0] * u[0] + f1[1] * u[1] + f1[2] * u[2] + f2[0] * v[0] + f2[1] * v[1] + f2[2] * v[2];
      fadd3(d.F_fix, r1, f1[0], f1[1], f1[2], d.err);
      fadd3(d.F_fix, r2, f2[0], f2[1], f2[2], d.err);
      fadd3(d.F_fix, ro, -f1[0] - f2[0], -f1[1] - f2[1], -f1[2] - f2[2], d.err);
    }
  }
  eb = warp_sum(eb);
  ea = warp_sum(ea);
  vir = warp_sum(vir);
  if ((threadIdx.x & 31) == 0) {
    eadd(d.E_fix, E_BOND, eb);
    eadd(d.E_fix, E_ANGLE, ea);
    eadd(d.E_fix, E_VIRIAL, vir);
  }
}

// ---------------------------------------------------------------------------
// pseudopotential: one warp per (pseudo particle, bead); lanes over sites
// V(r) = -k_e q erf(r/sigma)/r + A exp(-r/b), shifted force at r_cut
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pseudo_raw(const PseudoPar& pp, double r, double* v, double* dv) {
  const double x = r / pp.sig;
  double gg, dg;
  if (x < 1.0e-3) {
    const double x2 = x * x;
    const double c = 1.1283791670955126 / pp.sig;  // 2/sqrt(pi)/sigma
    gg = c * (1.0 - x2 / 3.0 + x2 * x2 / 10.0);
    dg = c / pp.sig * (-2.0 * x / 3.0 + 0.4 * x2 * x);
  } else {
    const double ef = erf(x);
    gg = ef / r;
    dg = 1.1283791670955126 * exp(-x * x) / (pp.sig * r) - ef / (r * r);
  }
  const double ex = exp(-r / pp.b);
  *v = -pp.kq * gg + pp.A * ex;
  *dv = -pp.kq * dg - (pp.A / pp.b) * ex;
}

__global__ void __launch_bounds__(PAIR_THREADS) k_pseudo64(Dev d) {
  __shared__ PseudoPar tab[MT];
  __shared__ double3 sh[125];
  for (int e = threadIdx.x; e < d.n_types; e += blockDim.x) tab[e] = d.pspar[e];
  for (int e = threadIdx.x; e < 125; e += blockDim.x)
    sh[e] = make_double3((e / 25 - 2) * d.box, ((e / 5) % 5 - 2) * d.box, (e % 5 - 2) * d.box);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= d.n_ppitems) return;
  // items: pseudo particles in order, all beads of each
  int e = 0, base = 0;
  while (e + 1 < d.n_pseudo && w >= base + (1 << d.pinfo[e].log2P)) {
    base += 1 << d.pinfo[e].log2P;
    ++e;
  }
  const int s = w - base;
  const AtomInfo pe = d.pinfo[e];
  const int row_e = pe.row0 + s * pe.stride;
  const double4_32a xe = d.Xw[row_e];
  const double wgt = 1.0 / (double)(1 << pe.log2P);
  const int cnt = min(d.pl_cnt[e], d.pl_cap);
  const int* lst = d.pl + (size_t)e * d.pl_cap;
  const double rc = d.rc, rc2 = d.rc2;
  double fex = 0.0, fey = 0.0, fez = 0.0, ep = 0.0, vir = 0.0;
  int nev = 0;
  for (int k = lane; k < cnt; k += 32) {
    const int ent = lst[k];
    const int c = ent >> 7;
    const AtomInfo ac = d.ainfo[c];
    const int bc = s >> (pe.log2P - ac.log2P);
    const int row_c = ac.row0 + bc * ac.stride;
    const double4_32a xc = d.Xw[row_c];
    const double3 sv = sh[ent & 127];
    const double dx = (xc.x - xe.x) + sv.x;
    const double dy = (xc.y - xe.y) + sv.y;
    const double dz = (xc.z - xe.z) + sv.z;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 < rc2) {
      const PseudoPar pp = tab[ac.type];
      const double r = sqrt(r2);
      double v, dv;
      pseudo_raw(pp, r, &v, &dv);
      ep += wgt * (v - pp.vrc - (r - rc) * pp.dvrc);
      const double fr = -wgt * (dv - pp.dvrc) / r;  // force on the site along d
      const double fx = fr * dx, fy = fr * dy, fz = fr * dz;
      fex -= fx;
      fey -= fy;
      fez -= fz;
      vir += fr * r2;
      ++nev;
      fadd3(d.F_fix, row_c, fx, fy, fz, d.err);
    }
  }
  fex = warp_sum(fex);
  fey = warp_sum(fey);
  fez = warp_sum(fez);
  ep = warp_sum(ep);
  vir = warp_sum(vir);
  nev = warp_sumi(nev);
  if (lane == 0) {
    fadd3(d.F_fix, row_e, fex, fey, fez, d.err);
    eadd(d.E_fix, E_PSEUDO, ep);
    eadd(d.E_fix, E_VIRIAL, vir);
    atomicAdd(d.E_fix + E_NPEVAL, (unsigned long long)nev);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_nlist(const Dev& d, cudaStream_t s, const int* atom_is_pseudo) {
  if (d.n_nonp > 0) {
    const int wpb = NL_THREADS / 32;
    k_nlist<<<(d.n_nonp + wpb - 1) / wpb, NL_THREADS, 0, s>>>(d, atom_is_pseudo);
  }
  if (d.n_pseudo > 0) {
    cudaMemsetAsync(d.pl_cnt, 0, sizeof(int) * d.n_pseudo, s);
    if (d.n_nonp > 0) {
      dim3 g((d.n_nonp + 127) / 128, d.n_pseudo);
      k_plist<<<g, 128, 0, s>>>(d, atom_is_pseudo);
    }
  }
}

void launch_forces(const Dev& d, cudaStream_t s, const AtomInfo* ainfo_atom) {
  const int wpb = PAIR_THREADS / 32;
  if (d.n_pitems > 0) k_pair64<<<(d.n_pitems + wpb - 1) / wpb, PAIR_THREADS, 0, s>>>(d);
  if (d.n_bitems > 0) k_bonded<<<(d.n_bitems + 255) / 256, 256, 0, s>>>(d, ainfo_atom);
  if (d.n_ppitems > 0 && d.n_nonp > 0)
    k_pseudo64<<<(d.n_ppitems + wpb - 1) / wpb, PAIR_THREADS, 0, s>>>(d);
}

}  // namespace mx
