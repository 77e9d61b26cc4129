// k_ewald.cu -- long-range electrostatics on ring-polymer centroids
// (Sec. "Theory", last paragraph: SPME with the bead-bead electrostatics
// approximated by centroid-centroid ones). With coulomb = 1 the pair sweeps
// evaluate the short-range real-space part erfc(alpha r)/r on every bead pair
// of the mixTS map; here the smooth remainder is summed over the centroids
// qbar_a = (1/P_a) sum_b q_{a,b} of the charged sites:
//   E_rec   = sum over half-space wave vectors k = 2 pi n / L, |n| <= kmax, of
//             W_k |S(k)|^2, S(k) = sum_a q_a exp(i k.qbar_a),
//             W_k = 2 (2 pi k_e / V) exp(-k^2 / (4 alpha^2)) / k^2 (k and -k)
//   E_intra = -k_e sum over same-molecule pairs q_a q_b erf(alpha r)/r (zero image)
//   E_self + E_bg = -k_e alpha / sqrt(pi) sum q_a^2 - k_e pi Q^2 / (2 V alpha^2)
// The force on a centroid acts as 1/P_a of it on each bead. Direct sums
// (no mesh): phases exp(i 2 pi n x / L) per centroid and axis by recurrence,
// one warp per wave vector for S(k), one warp per centroid for its force,
// fixed-order reductions and fixed-point accumulation (bitwise reproducible).
#include <math.h>

#include "mixts_internal.cuh"

namespace mx {

constexpr int EW_THREADS = 256;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// exp(i k.qbar_a) for wave vector n from the per-axis phase tables
__device__ __forceinline__ double2 ew_phase_of(const Dev& d, int a, int4 n) {
  const int K = d.ew_kmax + 1;
  const double2* ph = d.ew_phase + (size_t)a * 3 * K;
  const double2 ex = ph[n.x];  // n.x >= 0 in the half space
  double2 ey = ph[K + abs(n.y)];
  double2 ez = ph[2 * K + abs(n.z)];
  if (n.y < 0) ey.y = -ey.y;
  if (n.z < 0) ez.y = -ez.y;
  return cmul(cmul(ex, ey), ez);
}

// centroids of the charged sites (from the caller's unwrapped q, summed over
// beads in order) and their phase tables exp(i 2 pi n x / L), n = 0..kmax
__global__ void k_ew_phase(Dev d) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= d.n_qatoms) return;
  const int4 qi = d.qinfo[a];  // bead-0 row, row stride, P
  double c[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < qi.z; ++b) {
    const size_t r = (size_t)qi.x + (size_t)b * qi.y;
    for (int x = 0; x < 3; ++x) c[x] += d.q[3 * r + x];
  }
  for (int x = 0; x < 3; ++x) c[x] /= (double)qi.z;
  d.ew_cen[a] = make_double4_32a(c[0], c[1], c[2], 0.0);
  const int K = d.ew_kmax + 1;
  double2* ph = d.ew_phase + (size_t)a * 3 * K;
  for (int x = 0; x < 3; ++x) {
    double sn, cs;
    sincos(2.0 * 3.14159265358979323846 * c[x] / d.box, &sn, &cs);
    const double2 e1 = make_double2(cs, sn);
    double2 e = make_double2(1.0, 0.0);
    for (int n = 0; n < K; ++n) {
      ph[x * K + n] = e;
      e = cmul(e, e1);
    }
  }
}

// S(k) per half-space wave vector (one warp each), and W_k |S|^2 and its
// dilation virial W_k |S|^2 (1 - k^2 / (2 alpha^2))
__global__ void __launch_bounds__(EW_THREADS) k_ew_sk(Dev d) {
  const int lane = threadIdx.x & 31;
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= d.n_kvec) return;
  const int4 n = d.kn[k];
  double sr = 0.0, si = 0.0;
  for (int a = lane; a < d.n_qatoms; a += 32) {
    const double2 z = ew_phase_of(d, a, n);
    const double qa = d.qcharge[a];
    sr = fma(qa, z.x, sr);
    si = fma(qa, z.y, si);
  }
  sr = warp_sum(sr);
  si = warp_sum(si);
  if (lane == 0) {
    const double4_32a kv = d.kvec[k];
    const double k2 = kv.x * kv.x + kv.y * kv.y + kv.z * kv.z;
    const double e = kv.w * (sr * sr + si * si);
    d.ew_S[k] = make_double2(sr, si);
    d.ew_ek[2 * k] = e;
    d.ew_ek[2 * k + 1] = e * (1.0 - k2 * d.ew_inv2a2);
  }
}

// force on each charged centroid (one warp each), 1/P of it on every bead
__global__ void __launch_bounds__(EW_THREADS) k_ew_force(Dev d) {
  const int lane = threadIdx.x & 31;
  const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (a >= d.n_qatoms) return;
  const double qa = d.qcharge[a];
  double fx = 0.0, fy = 0.0, fz = 0.0;
  for (int k = lane; k < d.n_kvec; k += 32) {
    const double2 z = ew_phase_of(d, a, d.kn[k]);  // cos and sin of k.qbar_a
    const double2 S = d.ew_S[k];
    const double4_32a kv = d.kvec[k];
    const double g = 2.0 * kv.w * qa * (z.y * S.x - z.x * S.y);
    fx = fma(g, kv.x, fx);
    fy = fma(g, kv.y, fy);
    fz = fma(g, kv.z, fz);
  }
  fx = warp_sum(fx);
  fy = warp_sum(fy);
  fz = warp_sum(fz);
  const int4 qi = d.qinfo[a];
  const double inv = 1.0 / (double)qi.z;
  int bad = 0;
  const long long kx = fix44(fx * inv, 0, &bad), ky = fix44(fy * inv, 0, &bad), kz = fix44(fz * inv, 0, &bad);
  for (int b = lane; b < qi.z; b += 32) {
    unsigned long long* f = d.F_fix + 3 * ((size_t)qi.x + (size_t)b * qi.y);
    atomicAdd(f + 0, (unsigned long long)kx);
    atomicAdd(f + 1, (unsigned long long)ky);
    atomicAdd(f + 2, (unsigned long long)kz);
  }
  if (lane == 0 && bad) atomicOr(d.err, ERR_NONFINITE);
}

// one CTA: the reciprocal energy and virial summed over wave vectors in a
// fixed order, the self and background constants, and the intramolecular
// erf corrections on the centroids (zero image)
__global__ void __launch_bounds__(1024) k_ew_finish(Dev d) {
  __shared__ double red[2][32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  double e = 0.0, v = 0.0;
  for (int k = tid; k < d.n_kvec; k += blockDim.x) {
    e += d.ew_ek[2 * k];
    v += d.ew_ek[2 * k + 1];
  }
  int bad = 0;
  for (int p = tid; p < d.n_intra; p += blockDim.x) {
    const int2 pr = d.intra[p];
    const double4_32a ci = d.ew_cen[pr.x], cj = d.ew_cen[pr.y];
    const double dx = cj.x - ci.x, dy = cj.y - ci.y, dz = cj.z - ci.z;
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double r = sqrt(r2);
    const double qq = d.ew_ke * d.qcharge[pr.x] * d.qcharge[pr.y];
    const double ar = d.alpha * r;
    const double erfr = erf(ar);
    const double vi = -qq * erfr / r;
    // dV/dr of -qq erf(a r)/r
    const double dv = -qq * (1.1283791670955126 * d.alpha * exp(-ar * ar) / r - erfr / r2);
    e += vi;
    v += -dv * r;
    // force on centroid j along d is -dv/dr d/r; on i the opposite; 1/P to each bead
    const double fr = -dv / r;
    const int4 qi = d.qinfo[pr.x], qj = d.qinfo[pr.y];
    const double ui = 1.0 / (double)qi.z, uj = 1.0 / (double)qj.z;
    const long long jx = fix44(fr * dx * uj, 0, &bad), jy = fix44(fr * dy * uj, 0, &bad), jz = fix44(fr * dz * uj, 0, &bad);
    const long long ix = fix44(-fr * dx * ui, 0, &bad), iy = fix44(-fr * dy * ui, 0, &bad), iz = fix44(-fr * dz * ui, 0, &bad);
    for (int b = 0; b < qj.z; ++b) {
      unsigned long long* f = d.F_fix + 3 * ((size_t)qj.x + (size_t)b * qj.y);
      atomicAdd(f + 0, (unsigned long long)jx);
      atomicAdd(f + 1, (unsigned long long)jy);
      atomicAdd(f + 2, (unsigned long long)jz);
    }
    for (int b = 0; b < qi.z; ++b) {
      unsigned long long* f = d.F_fix + 3 * ((size_t)qi.x + (size_t)b * qi.y);
      atomicAdd(f + 0, (unsigned long long)ix);
      atomicAdd(f + 1, (unsigned long long)iy);
      atomicAdd(f + 2, (unsigned long long)iz);
    }
  }
  e = warp_sum(e);
  v = warp_sum(v);
  if (lane == 0) {
    red[0][w] = e;
    red[1][w] = v;
  }
  __syncthreads();
  if (tid == 0) {
    double se = 0.0, sv = 0.0;
    for (int x = 0; x < (int)(blockDim.x >> 5); ++x) {
      se += red[0][x];
      sv += red[1][x];
    }
    se += d.ew_const;
    sv += 3.0 * d.ew_bg;
    atomicAdd(d.E_fix + E_COUL, (unsigned long long)fixs(se, 40, &bad));
    atomicAdd(d.E_fix + E_VIRIAL, (unsigned long long)fixs(sv, 40, &bad));
  }
  bad = __syncthreads_or(bad);
  if (tid == 0 && bad) atomicOr(d.err, ERR_NONFINITE);
}

int launch_ewald(const Dev& d, cudaStream_t s) {
  if (d.coulomb != 1 || d.n_qatoms == 0) return 0;
  const int wpb = EW_THREADS / 32;
  k_ew_phase<<<(d.n_qatoms + 127) / 128, 128, 0, s>>>(d);
  k_ew_sk<<<(d.n_kvec + wpb - 1) / wpb, EW_THREADS, 0, s>>>(d);
  k_ew_force<<<(d.n_qatoms + wpb - 1) / wpb, EW_THREADS, 0, s>>>(d);
  k_ew_finish<<<1, 1024, 0, s>>>(d);
  return 4;
}

}  // namespace mx
