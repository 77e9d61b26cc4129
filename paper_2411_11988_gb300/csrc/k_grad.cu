// k_grad.cu -- adjoint of the mixTS potential with respect to force-field
// parameters (the differentiation variant). Pair terms are recomputed here
// rather than stored by the forward sweep.
//
// theta = (sigma_a, A_a, b_a, sigma_b, A_b, b_b, q_a, eps_aa). V_mix is linear
// in each charge product and in each Lennard-Jones epsilon, so dV/dq_a and
// dV/deps_aa follow from per-type-pair sums of the unit-charge DSF potential
// and of the Lennard-Jones energy; the pseudopotential parameters (sigma, A,
// b) enter nonlinearly and are differentiated term by term, shifted-force
// corrections at r_cut included.
#include <math.h>

#include "mixts_internal.cuh"

namespace mx {

constexpr int GRAD_THREADS = 256;

// unit-charge DSF G(s) (binary64 table, or direct below its range)
__device__ __forceinline__ double dsf_G(const Dev& d, const double* tab, double s) {
  const int hi = __double2hiint(s);
  if (hi >= __double2hiint(d.dsf_smin)) {
    const double s0 = __hiloint2double((hi >> 14) << 14, 0);
    const double* c = tab + 12 * ((hi >> 14) - d.dsf_base);
    const double x = s - s0;
    double p = fma(c[5], x, c[4]);
    p = fma(p, x, c[3]);
    p = fma(p, x, c[2]);
    p = fma(p, x, c[1]);
    return fma(p, x, c[0]);
  }
  const double r = sqrt(s);
  return erfc(d.alpha * r) / r - d.dsf_erfc_rc_over_rc + d.dsf_cf * (r - d.rc);
}

// Per-type-pair sums over all nonbonded terms in r_cut of (1/P) G and of
// (1/P) U, U the shifted-force Lennard-Jones term at unit epsilon (V_LJ is
// eps_ij U), ordered (owner type, partner type), into
// acc[2*(ti*MT+tj)+{0,1}] (fixed point 2^40).
__global__ void __launch_bounds__(GRAD_THREADS) k_grad_nb(Dev d, unsigned long long* acc) {
  __shared__ double wsum[GRAD_THREADS / 32][MT][2];
  __shared__ double uc[MT * MT][3];  // sigma^2, U(rc), dU/dr(rc)
  __shared__ int tN[MT], tLg[MT];
  const int nt = d.n_types;
  for (int e = threadIdx.x; e < nt; e += blockDim.x) {
    tN[e] = d.N[e];
    tLg[e] = d.log2P[e];
  }
  for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
    const double s2 = d.pairpar[(e / nt) * MT + (e % nt)].s2;
    const double sr2 = s2 / d.rc2, sr6 = sr2 * sr2 * sr2;
    uc[e][0] = s2;
    uc[e][1] = 4.0 * (sr6 * sr6 - sr6);
    uc[e][2] = -24.0 * (2.0 * sr6 * sr6 - sr6) / d.rc;
  }
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int e = lane; e < MT * 2; e += 32) wsum[wib][e / 2][e % 2] = 0.0;
  __syncthreads();
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w < d.n_pitems) {
    int c = 0;
    while (c + 1 < d.n_classes && w >= d.cls_item0[c + 1]) ++c;
    const int local = w - d.cls_item0[c];
    const int b = local / d.cls_n[c];
    const int pos = d.cls_pos0[c] + (local - b * d.cls_n[c]);
    const AtomInfo ai = d.ainfo[pos];
    const int row_i = ai.row0 + b * ai.stride;
    const double4_32a xi = d.Xw[row_i];
    const double wgt = pow2_neg(ai.log2P);
    const int cnt = min(d.nl_cnt[pos], d.nl_cap);
    const int* lst = d.nl + (size_t)pos * d.nl_cap;
    for (int e = lane; e < cnt; e += 32) {
      const int ent = lst[e];
      const int tj = (ent >> 7) & 15;
      const int row_j = (ent >> 11) + (b >> (ai.log2P - tLg[tj])) * tN[tj];
      const double4_32a xj = d.Xw[row_j];
      const int code = ent & 127;
      const double dx = (xj.x - xi.x) + (code / 25 - 2) * d.box;
      const double dy = (xj.y - xi.y) + ((code / 5) % 5 - 2) * d.box;
      const double dz = (xj.z - xi.z) + (code % 5 - 2) * d.box;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (!(r2 < d.rc2)) continue;
      atomicAdd(&wsum[wib][tj][0], wgt * dsf_G(d, d.dsf_tab, r2));
      const double* u = uc[ai.type * nt + tj];
      if (u[0] > 0.0) {
        const double r = sqrt(r2);
        const double sr2 = u[0] / r2, sr6 = sr2 * sr2 * sr2;
        atomicAdd(&wsum[wib][tj][1], wgt * (4.0 * (sr6 * sr6 - sr6) - u[1] - (r - d.rc) * u[2]));
      }
    }
    __syncwarp();
    if (lane < nt) {
      for (int k = 0; k < 2; ++k) {
        const double v = wsum[wib][lane][k];
        if (v != 0.0)
          atomicAdd(acc + 2 * (ai.type * MT + lane) + k, (unsigned long long)__double2ll_rn(v * ESCALE));
      }
    }
  }
}

// d/d(sigma, A, b, q) of the shifted-force pseudopotential term; dvc/ddvc are
// the parameter derivatives of V and dV/dr at r_cut for this site type
__device__ __forceinline__ void pseudo_dtheta(double kq_unit, double q, double sig, double A, double b, double r,
                                              double* dv) {
  const double x = r / sig;
  const double ex = exp(-x * x), eb = exp(-r / b);
  dv[0] = kq_unit * q * 1.1283791670955126 * ex / (sig * sig);
  dv[1] = eb;
  dv[2] = A * eb * r / (b * b);
  dv[3] = -kq_unit * erf(x) / r;
}

// Per (pseudo bead, site) term for site types a and b: out[0..3] =
// d/d(sigma_a, A_a[kcal], b_a, q_a), out[4..6] = d/d(sigma_b, A_b, b_b)
// (fixed point 2^40). pc holds, per site type t, the values at r_cut of the
// four derivatives of V (pc[8t+0..3]) and of dV/dr (pc[8t+4..7]).
__global__ void __launch_bounds__(GRAD_THREADS) k_grad_pseudo(Dev d, int ta, int tb, double ke, const double* pc,
                                                              unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= d.n_ppitems) return;
  int e = 0, base = 0;
  while (e + 1 < d.n_pseudo && w >= base + (1 << d.pinfo[e].log2P)) {
    base += 1 << d.pinfo[e].log2P;
    ++e;
  }
  const int s = w - base;
  const AtomInfo pe = d.pinfo[e];
  const double4_32a xe = d.Xw[pe.row0 + s * pe.stride];
  const double wgt = pow2_neg(pe.log2P);
  const int cnt = min(d.pl_cnt[e], d.pl_cap);
  const int* lst = d.pl + (size_t)e * d.pl_cap;
  double g[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int k = lane; k < cnt; k += 32) {
    const int ent = lst[k];
    const AtomInfo ac = d.ainfo[ent >> 7];
    const int t = ac.type;
    if (t != ta && t != tb) continue;
    const double4_32a xc = d.Xw[ac.row0 + (s >> (pe.log2P - ac.log2P)) * ac.stride];
    const int code = ent & 127;
    const double dx = (xc.x - xe.x) + (code / 25 - 2) * d.box;
    const double dy = (xc.y - xe.y) + ((code / 5) % 5 - 2) * d.box;
    const double dz = (xc.z - xe.z) + (code % 5 - 2) * d.box;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (!(r2 < d.rc2)) continue;
    const double r = sqrt(r2);
    const PseudoPar pp = d.pspar[t];
    double dv[4];
    pseudo_dtheta(ke, pp.kq / ke, pp.sig, pp.A, pp.b, r, dv);
    const double* c = pc + 8 * t;
    double tv[4];
    for (int m = 0; m < 4; ++m) tv[m] = wgt * (dv[m] - c[m] - (r - d.rc) * c[4 + m]);
    if (t == ta) {
      g[0] += tv[0];
      g[1] += tv[1];
      g[2] += tv[2];
      g[3] += tv[3];
    } else {
      g[4] += tv[0];
      g[5] += tv[1];
      g[6] += tv[2];
    }
  }
  for (int m = 0; m < 7; ++m) g[m] = warp_sum(g[m]);
  if (lane == 0)
    for (int m = 0; m < 7; ++m)
      if (g[m] != 0.0) atomicAdd(out + m, (unsigned long long)__double2ll_rn(g[m] * ESCALE));
}

// dV/dq = -F, scaled by grad_out
__global__ void k_grad_q(Dev d, double grad_out, double* dvdq) {
  const size_t n = (size_t)d.n_beads * 3;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    dvdq[e] = -grad_out * fix_to_double(d.F_fix[e], FINV);
}

int launch_grad(const Dev& d, cudaStream_t s, int ta, int tb, double ke, const double* pc, unsigned long long* acc,
                double grad_out, double* dvdq, bool want_theta) {
  int n = 0;
  const int wpb = GRAD_THREADS / 32;
  if (want_theta && d.n_pitems > 0) {
    k_grad_nb<<<(d.n_pitems + wpb - 1) / wpb, GRAD_THREADS, 0, s>>>(d, acc);
    ++n;
  }
  if (want_theta && d.n_ppitems > 0 && d.n_nonp > 0) {
    k_grad_pseudo<<<(d.n_ppitems + wpb - 1) / wpb, GRAD_THREADS, 0, s>>>(d, ta, tb, ke, pc, acc + 2 * MT * MT);
    ++n;
  }
  if (dvdq) {
    k_grad_q<<<296, 256, 0, s>>>(d, grad_out, dvdq);
    ++n;
  }
  return n;
}

}  // namespace mx
