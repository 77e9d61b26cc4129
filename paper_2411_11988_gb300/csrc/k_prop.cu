// k_prop.cu -- ring-polymer propagation: normal-mode transforms, PILE
// thermostat half steps, half kicks and the exact free-ring rotation of the
// split propagator (Sec. "Evaluation"), plus the per-step estimator partials
// (Sec. "Output and Analysis") and the position mirrors the force kernels read.
//
// Types with P <= SMALL_P: one CTA owns all P beads of a few atoms (a P x C
// column tile, C = 3 * atoms) in shared memory and runs transform ->
// elementwise update -> inverse transform in one pass, by the dense (folded)
// mode matrix. Larger P (up to the 1024-bead electron): the same pass by one
// thread-block cluster per tile, with four-step FFTs split over its CTAs.
#include <math.h>

#include <algorithm>

#include "mixts_internal.cuh"

namespace mx {

constexpr int PROP_THREADS = 3 * PROP_TILE_BEADS;  // one thread per element of a P x C tile
constexpr int NPART = 6;  // KE, spring, CV, Rg, heat(end), heat(start)

__device__ __forceinline__ void block_sum6(double* v, double* red) {
  // v[NPART] per thread -> red[0..NPART) on thread 0, fixed order
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NPART; ++i) v[i] = warp_sum(v[i]);
  __syncthreads();
  if (lane == 0)
    for (int i = 0; i < NPART; ++i) red[w * NPART + i] = v[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < NPART; ++i) {
      double s = 0.0;
      for (int x = 0; x < nw; ++x) s += red[x * NPART + i];
      red[i] = s;
    }
  }
  __syncthreads();
}

// writes the force-kernel mirrors of one atom's beads. xc(j, d) is the
// Cartesian coordinate of bead j; rows r(j) = row0 + j * stride.
struct MirrorOut {
  __device__ static void wrap_ref(double x, double L, double* fl_out, double* ref_out) {
    const double fl = floor(__ddiv_rn(x, L));
    *fl_out = fl;
    *ref_out = __dsub_rn(x, __dmul_rn(L, fl));
  }
};

__device__ __forceinline__ void write_mirror(const Dev& d, int row, double x, double y, double z, double mx_,
                                             double my_, double mz_, const double* x0, int arow) {
  const double L = d.box;
  // offset from the atom's bead 0 (unwrapped difference; the shift cancels),
  // atom-major so that one atom's beads are contiguous
  if (d.Xd) d.Xd[arow] = make_float4((float)(x - x0[0]), (float)(y - x0[1]), (float)(z - x0[2]), 0.0f);
  const double wx = fma(-mx_, L, x), wy = fma(-my_, L, y), wz = fma(-mz_, L, z);
  d.Xw[row] = make_double4_32a(wx, wy, wz, 0.0);
  // 2^-48 A fixed point, and the nearest 2^-12 A grid point as binary32
  int bad = 0;
  const long long ix = fixs(wx, 48, &bad), iy = fixs(wy, 48, &bad), iz = fixs(wz, 48, &bad);
  d.Xi[row] = make_longlong4_32a(ix, iy, iz, 0);
  if (d.XiA) d.XiA[arow] = make_longlong4_32a(ix, iy, iz, 0);
  const int gx = (int)((ix + (1LL << 35)) >> 36), gy = (int)((iy + (1LL << 35)) >> 36),
            gz = (int)((iz + (1LL << 35)) >> 36);
  d.Xf[row] = make_float4(small_int_float(gx) * 0x1p-12f, small_int_float(gy) * 0x1p-12f,
                          small_int_float(gz) * 0x1p-12f, 0.0f);
  d.Xl[row] = make_float4((float)(ix - ((long long)gx << 36)) * 0x1p-48f, (float)(iy - ((long long)gy << 36)) * 0x1p-48f,
                          (float)(iz - ((long long)gz << 36)) * 0x1p-48f, 0.0f);
  if (bad) atomicOr(d.err, ERR_NONFINITE);
}

// wrapped bead-0 reference of one atom, by atom index and (for non-pseudo
// atoms) by sorted position for the neighbour search, with the lattice
// vector fl that wrapped it (q_0 = r + fl L), which locates the zero image
// of the caller's unwrapped coordinates for same-molecule pairs
__device__ __forceinline__ void write_ref(const Dev& d, int atom, const double* rf, const double* fl) {
  for (int x = 0; x < 3; ++x) d.ref[3 * atom + x] = rf[x];
  const int pos = d.pos_of_atom[atom];
  if (pos >= 0) {
    d.refd[pos] = make_double4_32a(rf[0], rf[1], rf[2], 0.0);
    d.reff[pos] = make_float4((float)rf[0], (float)rf[1], (float)rf[2], __int_as_float(d.ainfo[pos].log2P));
    d.wrapn[pos] = make_int4((int)fl[0], (int)fl[1], (int)fl[2], 0);
  }
}

__device__ __forceinline__ double bead_d2(double dx, double dy, double dz) {
  double d2 = __dmul_rn(dx, dx);
  d2 = __dadd_rn(d2, __dmul_rn(dy, dy));
  d2 = __dadd_rn(d2, __dmul_rn(dz, dz));
  return d2;
}

__device__ __forceinline__ double bead_dist(double dx, double dy, double dz) { return __dsqrt_rn(bead_d2(dx, dy, dz)); }

// ---------------------------------------------------------------------------
// Folded normal-mode transforms of a P x C tile in shared memory. The real
// orthonormal basis is even or odd under bead j -> P - j: the cosine-like
// modes k <= P/2 (centroid and alternating mode included) have
// C[P-j][k] = C[j][k], the sine-like modes C[P-j][k] = -C[j][k]. With the
// folded beads s_j = x_j + x_{P-j} and d_j = x_j - x_{P-j} (0 < j < P/2) each
// sum runs over half the beads; the inverse computes the even part A_j and
// the odd part B_j for j <= P/2 and writes x_j = A_j + B_j, x_{P-j} = A_j - B_j.
// Half the multiply-adds of the dense products, in another rounding order
// (nm_fold2 below halves them once more for P >= 4).
// ---------------------------------------------------------------------------
// in place: row j <- s_j, row P - j <- d_j (0 < j < P/2)
__device__ __forceinline__ void nm_fold(double* x, int P, int C, int tid, int nt) {
  const int h = P / 2;
  for (int e = tid; e < (h - 1) * C; e += nt) {
    const int j = 1 + e / C, c = e - (e / C) * C;
    const double a = x[j * C + c], b = x[(P - j) * C + c];
    x[j * C + c] = a + b;
    x[(P - j) * C + c] = a - b;
  }
}

// out[k][c] = sum_j C[j][k] x_j from the folded rows f (nm_fold)
__device__ __forceinline__ void nm_forward_folded(const double* Cm, int P, int C, const double* f, double* out,
                                                  int tid, int nt) {
  const int h = P / 2;
  for (int e = tid; e < P * C; e += nt) {
    const int k = e / C, c = e - (e / C) * C;
    double a = 0.0;
    if (k <= h) {
      for (int j = 0; j <= h; ++j) a = fma(Cm[j * P + k], f[j * C + c], a);
    } else {
      for (int j = 1; j < h; ++j) a = fma(Cm[j * P + k], f[(P - j) * C + c], a);
    }
    out[e] = a;
  }
}

// even and odd parts of x_j = sum_k C[j][k] q_k for j <= P/2: A in rows
// 0..P/2 of ev, B in rows 1..P/2-1 of od (two passes' worth of threads)
__device__ __forceinline__ void nm_inverse_parts(const double* Cm, int P, int C, const double* q, double* ev,
                                                 double* od, int tid, int nt) {
  const int h = P / 2;
  const int ne = (h + 1) * C;
  for (int e = tid; e < ne + (h > 1 ? (h - 1) * C : 0); e += nt) {
    if (e < ne) {
      const int j = e / C, c = e - (e / C) * C;
      double a = 0.0;
      for (int k = 0; k <= h; ++k) a = fma(Cm[j * P + k], q[k * C + c], a);
      ev[j * C + c] = a;
    } else {
      const int e2 = e - ne;
      const int j = 1 + e2 / C, c = e2 - (e2 / C) * C;
      double b = 0.0;
      for (int k = h + 1; k < P; ++k) b = fma(Cm[j * P + k], q[k * C + c], b);
      od[j * C + c] = b;
    }
  }
}

// Second fold (P >= 4, h = P/2 even, q = h/2). The cosine-like modes are
// even or odd under j -> h - j as k is even or odd, the sine-like ones odd
// or even; after nm_fold, rows j and h - j of the s part (0 <= j < q) become
// e_j = f_j + f_{h-j} and o_j = f_j - f_{h-j}, and rows P - j and P - h + j of
// the d part (1 <= j < q) become d_j + d_{h-j} and d_j - d_{h-j}; the middle
// rows q and P - q stay. Each mode's sum then runs over a quarter of the beads.
__device__ __forceinline__ void nm_fold2(double* x, int P, int C, int tid, int nt) {
  const int h = P / 2, q = h / 2;
  const int n1 = q * C, n2 = (q - 1) * C;
  for (int e = tid; e < n1 + n2; e += nt) {
    if (e < n1) {
      const int j = e / C, c = e - (e / C) * C;
      const double a = x[j * C + c], b = x[(h - j) * C + c];
      x[j * C + c] = a + b;
      x[(h - j) * C + c] = a - b;
    } else {
      const int e2 = e - n1;
      const int j = 1 + e2 / C, c = e2 - (e2 / C) * C;
      const double a = x[(P - j) * C + c], b = x[(P - h + j) * C + c];
      x[(P - j) * C + c] = a + b;
      x[(P - h + j) * C + c] = a - b;
    }
  }
}

// out[k][c] = sum_j C[j][k] x_j from the twice-folded rows (nm_fold2); the
// middle row enters only where its coefficient (cos or sin of a multiple of
// pi/2) is not zero
__device__ __forceinline__ void nm_forward_folded2(const double* Cm, int P, int C, const double* f, double* out,
                                                   int tid, int nt) {
  const int h = P / 2, q = h / 2;
  for (int e = tid; e < P * C; e += nt) {
    const int k = e / C, c = e - (e / C) * C;
    double a = 0.0;
    if (k <= h) {
      if ((k & 1) == 0) {
        for (int j = 0; j < q; ++j) a = fma(Cm[j * P + k], f[j * C + c], a);
        a = fma(Cm[q * P + k], f[q * C + c], a);
      } else {
        for (int j = 0; j < q; ++j) a = fma(Cm[j * P + k], f[(h - j) * C + c], a);
      }
    } else {
      if ((k & 1) == 0) {
        for (int j = 1; j < q; ++j) a = fma(Cm[j * P + k], f[(P - h + j) * C + c], a);
      } else {
        for (int j = 1; j < q; ++j) a = fma(Cm[j * P + k], f[(P - j) * C + c], a);
        a = fma(Cm[q * P + k], f[(P - q) * C + c], a);
      }
    }
    out[e] = a;
  }
}

// even and odd parts of the inverse from the even- and odd-k halves of each
// sum: A_j, A_{h-j} = Ae_j +/- Ao_j (0 <= j <= q), B_j = Be_j + Bo_j and
// B_{h-j} = Bo_j - Be_j (1 <= j <= q); same rows as nm_inverse_parts
__device__ __forceinline__ void nm_inverse_parts2(const double* Cm, int P, int C, const double* qm, double* ev,
                                                  double* od, int tid, int nt) {
  const int h = P / 2, q = h / 2;
  const int na = (q + 1) * C, nb = q * C;
  for (int e = tid; e < na + nb; e += nt) {
    if (e < na) {
      const int j = e / C, c = e - (e / C) * C;
      double ae = 0.0, ao = 0.0;
      for (int k = 0; k <= h; k += 2) ae = fma(Cm[j * P + k], qm[k * C + c], ae);
      for (int k = 1; k < h; k += 2) ao = fma(Cm[j * P + k], qm[k * C + c], ao);
      ev[j * C + c] = ae + ao;
      if (j != q) ev[(h - j) * C + c] = ae - ao;
    } else {
      const int e2 = e - na;
      const int j = 1 + e2 / C, c = e2 - (e2 / C) * C;
      double be = 0.0, bo = 0.0;
      for (int k = h + 2; k < P; k += 2) be = fma(Cm[j * P + k], qm[k * C + c], be);
      for (int k = h + 1; k < P; k += 2) bo = fma(Cm[j * P + k], qm[k * C + c], bo);
      od[j * C + c] = be + bo;
      if (j != q) od[(h - j) * C + c] = bo - be;
    }
  }
}

// value of bead j from the parts (after nm_inverse_parts and a barrier)
__device__ __forceinline__ double nm_inverse_value(const double* ev, const double* od, int P, int C, int j, int c) {
  const int h = P / 2;
  if (j == 0 || j == h) return ev[j * C + c];
  if (j < h) return ev[j * C + c] + od[j * C + c];
  return ev[(P - j) * C + c] - od[(P - j) * C + c];
}

// ---------------------------------------------------------------------------
// small-P fused tile kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ void b_k_prop_small(const Dev& d, int bx, int mode) {
  extern __shared__ double sm[];
  __shared__ double red[(PROP_THREADS / 32) * NPART];
  __shared__ long long s_step;
  __shared__ long long s_d2[PROP_TILE_BEADS];
  const PropTile tl = d.tiles[bx];
  const int t = tl.type, P = d.P[t], N = d.N[t], k0 = tl.k0, na = tl.na;
  const int C = 3 * na;
  const int PC = P * C;
  double* Cm = sm;
  double* Fb = Cm + P * P;
  double* Fn = Fb + PC;
  double* Qn = Fn + PC;
  double* Pn = Qn + PC;
  double* Xc = Pn + PC;
  const int tid = threadIdx.x, nt = blockDim.x;
  const double m = d.mass[t];
  const double* cmg = d.cm + d.cm_off[t];
  const ModeCoef* mcf = d.mc + d.mc_off[t];
  auto gidx = [&](int j, int c) -> size_t { return (size_t)(d.off[t] + j * N + k0) * 3 + c; };

  if (tid == 0) s_step = *d.step_ctr;
  for (int e = tid; e < P * P; e += nt) Cm[e] = cmg[e];
  const bool need_f = (mode & (PM_END | PM_START)) != 0;
  for (int e = tid; e < PC; e += nt) {
    const int j = e / C, c = e - (e / C) * C;
    const size_t g = gidx(j, c);
    if (mode & PM_IMPORT) {
      Xc[e] = d.q[g];
      Fb[e] = d.p[g];
    } else {
      Qn[e] = d.q_nm[g];
      Pn[e] = d.p_nm[g];
    }
  }
  __syncthreads();
  const bool two_folds = P >= 4;
  if (mode & PM_IMPORT) {
    nm_fold(Xc, P, C, tid, nt);
    nm_fold(Fb, P, C, tid, nt);
    __syncthreads();
    if (two_folds) {
      nm_fold2(Xc, P, C, tid, nt);
      nm_fold2(Fb, P, C, tid, nt);
      __syncthreads();
      nm_forward_folded2(Cm, P, C, Xc, Qn, tid, nt);
      nm_forward_folded2(Cm, P, C, Fb, Pn, tid, nt);
    } else {
      nm_forward_folded(Cm, P, C, Xc, Qn, tid, nt);
      nm_forward_folded(Cm, P, C, Fb, Pn, tid, nt);
    }
    __syncthreads();
  }
  double part[NPART] = {0, 0, 0, 0, 0, 0};
  if (need_f) {
    for (int e = tid; e < PC; e += nt) {
      const int j = e / C, c = e - (e / C) * C;
      const size_t g = gidx(j, c);
      const double f = fix_to_double(d.F_fix[g], FINV);
      Fb[e] = f;
      if (mode & PM_END) d.f[g] = f;
      if (mode & PM_START) d.F_fix[g] = 0ull;
      if ((mode & PM_END) && (mode & PM_EST)) {
        // centroid virial: sum_b (q_b - qbar) . F_b, qbar from the centroid mode
        const double qbar = Qn[c] * rsqrt((double)P);
        part[2] += (d.q[g] - qbar) * f;
      }
    }
    __syncthreads();
    nm_fold(Fb, P, C, tid, nt);
    __syncthreads();
    if (two_folds) {
      nm_fold2(Fb, P, C, tid, nt);
      __syncthreads();
      nm_forward_folded2(Cm, P, C, Fb, Fn, tid, nt);
    } else {
      nm_forward_folded(Cm, P, C, Fb, Fn, tid, nt);
    }
    __syncthreads();
    const double hk = 0.5 * d.dt * d.kcal;  // F in kcal/mol/A -> amu A/fs^2
    const uint32_t s_end = (uint32_t)s_step;
    const uint32_t s_start = (uint32_t)(s_step + ((mode & PM_END) ? 1 : 0));
    const double inv2m = 0.5 / m;
    for (int e = tid; e < PC; e += nt) {
      const int k = e / C, c = e - (e / C) * C;
      const ModeCoef mk = mcf[k];
      const uint64_t dof = (uint64_t)gidx(k, c);
      double p = Pn[e], q = Qn[e];
      const double fk = Fn[e];
      if (mode & PM_END) {
        p = fma(hk, fk, p);
        const double xi = f2d_bits(gauss_dof(d.seed, s_end, 1u, dof));
        const double pn = fma(mk.c1, p, mk.c2s * xi);
        part[4] += (p * p - pn * pn) * inv2m;
        p = pn;
        if (mode & PM_EST) {
          part[0] += p * p * inv2m;
          part[1] += mk.hmw2 * q * q;
          if (k > 0) part[3] += q * q;
        }
      }
      if (mode & PM_START) {
        const double xi = f2d_bits(gauss_dof(d.seed, s_start, 0u, dof));
        const double pn = fma(mk.c1, p, mk.c2s * xi);
        part[5] += (p * p - pn * pn) * inv2m;
        p = fma(hk, fk, pn);
        // exact free ring: [p; q] <- [[cw, -m w sw], [sw/(m w), cw]] [p; q]; k = 0 drifts
        const double pr = fma(mk.cw, p, -mk.mws * q);
        const double qr = fma(mk.swm, p, mk.cw * q);
        p = pr;
        q = qr;
      }
      Pn[e] = p;
      Qn[e] = q;
    }
    __syncthreads();
  }
  // write the mode-space state back
  if (mode & (PM_IMPORT | PM_END | PM_START)) {
    for (int e = tid; e < PC; e += nt) {
      const int j = e / C, c = e - (e / C) * C;
      const size_t g = gidx(j, c);
      d.q_nm[g] = Qn[e];
      d.p_nm[g] = Pn[e];
    }
  }
  // Cartesian positions and mirrors
  if (mode & (PM_START | PM_QCART)) {
    // Fb and Fn are free here: they hold the even and odd parts
    if (two_folds)
      nm_inverse_parts2(Cm, P, C, Qn, Fb, Fn, tid, nt);
    else
      nm_inverse_parts(Cm, P, C, Qn, Fb, Fn, tid, nt);
    __syncthreads();
    for (int e = tid; e < PC; e += nt) {
      const int j = e / C, c = e - (e / C) * C;
      const double a = nm_inverse_value(Fb, Fn, P, C, j, c);
      Xc[e] = a;
      d.q[gidx(j, c)] = a;
    }
    // squared bead-0 distances, max over beads on the bit patterns, one
    // square root per atom: sqrt is monotone, so this equals the max of
    // the rounded distances
    for (int e = tid; e < na; e += nt) s_d2[e] = 0;
    __syncthreads();
    for (int e = tid; e < P * na; e += nt) {
      const int j = e / na, a = e - (e / na) * na;
      const int atom = d.atom_of_tk[d.atoff[t] + k0 + a];
      double fl[3], rf[3];
      for (int x = 0; x < 3; ++x) MirrorOut::wrap_ref(Xc[0 * C + 3 * a + x], d.box, &fl[x], &rf[x]);
      const int row = d.off[t] + j * N + k0 + a;
      write_mirror(d, row, Xc[j * C + 3 * a], Xc[j * C + 3 * a + 1], Xc[j * C + 3 * a + 2], fl[0], fl[1], fl[2],
                   Xc + 3 * a, d.off[t] + (k0 + a) * P + j);
      if (j == 0) {
        write_ref(d, atom, rf, fl);
      } else {
        const double d2 = bead_d2(Xc[j * C + 3 * a] - Xc[3 * a], Xc[j * C + 3 * a + 1] - Xc[3 * a + 1],
                                  Xc[j * C + 3 * a + 2] - Xc[3 * a + 2]);
        atomicMax(&s_d2[a], __double_as_longlong(d2));
      }
    }
    __syncthreads();
    for (int a = tid; a < na; a += nt) {
      const int atom = d.atom_of_tk[d.atoff[t] + k0 + a];
      d.spread[atom] = __dsqrt_rn(__longlong_as_double(s_d2[a]));
    }
  }
  if (mode & PM_PCART) {
    __syncthreads();  // the position pass is done with Fb and Fn
    if (two_folds)
      nm_inverse_parts2(Cm, P, C, Pn, Fb, Fn, tid, nt);
    else
      nm_inverse_parts(Cm, P, C, Pn, Fb, Fn, tid, nt);
    __syncthreads();
    for (int e = tid; e < PC; e += nt) {
      const int j = e / C, c = e - (e / C) * C;
      d.p[gidx(j, c)] = nm_inverse_value(Fb, Fn, P, C, j, c);
    }
  }
  if (mode & (PM_END | PM_START)) {
    block_sum6(part, red);
    if (tid == 0)
      for (int i = 0; i < NPART; ++i) d.parts[(size_t)tl.slot * NPART + i] = red[i];
  }
}

__global__ void __launch_bounds__(PROP_THREADS) k_prop_small(const __grid_constant__ Dev d, int mode) { b_k_prop_small(d, blockIdx.x, mode); }

__global__ void __launch_bounds__(PROP_THREADS) k_prop_small_b(const Dev* __restrict__ devs, const int* __restrict__ pfx, int nm, int mode) {
  MX_BATCH_ENTER();
  b_k_prop_small(d, bx, mode);
}

// ---------------------------------------------------------------------------
// mirrors straight from the caller's Cartesian q (force evaluation without
// touching the mode-space state); one thread per atom
// ---------------------------------------------------------------------------
__global__ void k_mirror_from_q(Dev d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.n_atoms) return;
  int t = 0;
  while (t + 1 < d.n_types && d.atoff[t + 1] <= i) ++t;
  const int k = i - d.atoff[t];
  const int atom = d.atom_of_tk[i];
  const int P = d.P[t], N = d.N[t];
  const int r0 = d.off[t] + k;
  double q0[3], fl[3], rf[3];
  for (int x = 0; x < 3; ++x) {
    q0[x] = d.q[3 * (size_t)r0 + x];
    MirrorOut::wrap_ref(q0[x], d.box, &fl[x], &rf[x]);
  }
  write_ref(d, atom, rf, fl);
  double sp = 0.0;
  for (int j = 0; j < P; ++j) {
    const size_t row = (size_t)r0 + (size_t)j * N;
    const double x = d.q[3 * row], y = d.q[3 * row + 1], z = d.q[3 * row + 2];
    write_mirror(d, (int)row, x, y, z, fl[0], fl[1], fl[2], q0, d.off[t] + k * P + j);
    if (j > 0) {
      const double dd = bead_dist(x - q0[0], y - q0[1], z - q0[2]);
      sp = dd > sp ? dd : sp;
    }
  }
  d.spread[atom] = sp;
}

// ---------------------------------------------------------------------------
// large-P path: one thread-block cluster of CL CTAs owns all P beads of a
// few atoms and computes the orthonormal transforms by a four-step FFT
// (P log P work instead of P^2), split over the cluster's SMs because a
// single SM's FP64 pipe is far too slow for the 1024-bead electron.
//
// Real columns in pairs: two real columns a, b travel as one complex column
// z = a + i b. With Y = DFT(z) (e^{-2 pi i jm/P}, unscaled) the columns'
// real DFTs are (Y_m + conj Y_{P-m})/2 and (Y_m - conj Y_{P-m})/2i, and the
// modes of the basis (1/sqrt P; sqrt(2/P) cos 2 pi jk/P for k < P/2;
// (-1)^j/sqrt P; sqrt(2/P) sin 2 pi jk/P for k > P/2) are their scaled real
// and imaginary parts. The inverse builds both columns' Hermitian spectra,
// packs them the same way and runs the conjugate transform.
//
// Four steps, P = R S, bead j = S j1 + j2, frequency m = m1 + R m2:
//   Y[m1 + R m2] = sum_j2 W_S^{j2 m2} W^{j2 m1} sum_j1 W_R^{j1 m1} x[S j1 + j2].
// CTA r of the cluster owns the bead columns j2 in [r S/CL, (r+1) S/CL)
// (length-R transforms over j1) and the frequencies m1 in [r R/CL, (r+1) R/CL)
// (length-S transforms over m2, the modes k = m1 + R m2); the exchange in
// between reads the other CTAs' shared memory (distributed shared memory).
// ---------------------------------------------------------------------------
constexpr int BIG_THREADS = 256;

__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// barrier over every thread of every CTA of the cluster, with release /
// acquire ordering of shared-memory writes across the cluster
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// generic address of the same shared-memory location in CTA `rank` of the cluster
template <class T>
__device__ __forceinline__ T* dsmem(T* p, unsigned rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"((uint64_t)p), "r"(rank));
  return reinterpret_cast<T*>(out);
}

// w * u with w = (wx, sg wy)
__device__ __forceinline__ double2 cmul(double2 w, double sg, double2 u) {
  const double wi = sg * w.y;
  return make_double2(fma(w.x, u.x, -wi * u.y), fma(w.x, u.y, wi * u.x));
}

// W^k = (cos, sin)(2 pi k / P), k in [0, P), from the half table tw[k < P/2]
__device__ __forceinline__ double2 tw_full(const double2* tw, int k, int lgP) {
  const int h = 1 << (lgP - 1);
  const double2 w = tw[k & (h - 1)];
  return k < h ? w : make_double2(-w.x, -w.y);
}

// In-place decimation-in-time FFTs of nrow rows of length L = 2^lgL (row i at
// B + i L): input in bit-reversed order, output in natural order, exponent
// sign sg (-1 forward, +1 inverse), no scaling; W_L^e = W^{e P/L}. Ends with
// a block barrier.
__device__ void fft_rows(double2* B, int nrow, int lgL, const double2* tw, int lgP, double sg, int tid, int nt) {
  const int hL = 1 << (lgL - 1);
  for (int s = 0; s < lgL; ++s) {
    const int h = 1 << s;
    for (int b = tid; b < nrow * hL; b += nt) {
      const int row = b >> (lgL - 1), bb = b & (hL - 1);
      const int pos = bb & (h - 1);
      const int i0 = ((bb >> s) << (s + 1)) + pos;
      double2* c = B + ((size_t)row << lgL);
      const double2 a = c[i0];
      const double2 t = cmul(tw[(pos << (lgL - 1 - s)) << (lgP - lgL)], sg, c[i0 + h]);
      c[i0] = make_double2(a.x + t.x, a.y + t.y);
      c[i0 + h] = make_double2(a.x - t.x, a.y - t.y);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int brev_n(int v, int lg) { return lg ? (int)(__brev((unsigned)v) >> (32 - lg)) : 0; }

struct BigGeom {   // one CTA's share of a large-P tile
  int P, lgP, R, lgR, S, lgS, CL, JL, ML, C, nz;
  unsigned rank;
  double2* tw;     // [P/2]
  double2* Ab;     // [nz][JL][R]  bead-column rows
  double2* Yb;     // [nz][ML][S]  frequency rows
  double* Qm;      // [ML][S][C]  owned q modes
  double* Pm;      // [ML][S][C]  owned p modes
};

// forward transform of a real array: Ab <- its owned bead columns (loaded by
// the caller, bit-reversed over j1), then Yb <- Y[m1 + R m2] for the owned m1.
// Ends after a cluster barrier, with every CTA's Yb complete.
__device__ void big_forward(const BigGeom& g, int tid, int nt) {
  __syncthreads();
  fft_rows(g.Ab, g.nz * g.JL, g.lgR, g.tw, g.lgP, -1.0, tid, nt);
  for (int e = tid; e < g.nz * g.JL * g.R; e += nt) {  // times e^{-2 pi i j2 m1 / P}
    const int m1 = e & (g.R - 1), jl = (e >> g.lgR) % g.JL;
    const int j2 = (int)g.rank * g.JL + jl;
    g.Ab[e] = cmul(tw_full(g.tw, j2 * m1, g.lgP), -1.0, g.Ab[e]);
  }
  cluster_barrier();
  for (int e = tid; e < g.nz * g.ML * g.S; e += nt) {
    const int j2 = e & (g.S - 1), row = e >> g.lgS;  // row = z ML + ml
    const int z = row / g.ML, ml = row - z * g.ML;
    const int m1 = (int)g.rank * g.ML + ml;
    const double2* src = dsmem(g.Ab, (unsigned)(j2 / g.JL));
    g.Yb[((size_t)row << g.lgS) + brev_n(j2, g.lgS)] = src[((size_t)(z * g.JL + j2 % g.JL) << g.lgR) + m1];
  }
  __syncthreads();
  fft_rows(g.Yb, g.nz * g.ML, g.lgS, g.tw, g.lgP, -1.0, tid, nt);
  cluster_barrier();
}

// mode k = m1 + R m2 (m1 owned: local index ml) of real column c after big_forward
__device__ __forceinline__ double big_mode(const BigGeom& g, int ml, int m2, int c, double rP, double r2P) {
  const int P = g.P;
  const int m1 = (int)g.rank * g.ML + ml, k = m1 + g.R * m2;
  const int z = c >> 1;
  const double2 a = g.Yb[((size_t)(z * g.ML + ml) << g.lgS) + m2];
  const int kk = (P - k) & (P - 1), n1 = kk & (g.R - 1), n2 = kk >> g.lgR;
  const double2* yo = dsmem(g.Yb, (unsigned)(n1 / g.ML));
  const double2 b = yo[((size_t)(z * g.ML + n1 % g.ML) << g.lgS) + n2];
  const bool odd = c & 1;
  if (k == 0 || 2 * k == P) return (odd ? a.y : a.x) * rP;
  if (2 * k < P) return (odd ? a.y + b.y : a.x + b.x) * r2P;
  return odd ? (a.x - b.x) * r2P : (b.y - a.y) * r2P;
}

// inverse transform of the owned modes X (Qm or Pm, every CTA's complete
// and visible): Ab <- the bead values x[S j1 + j2] of the owned columns j2,
// natural order over j1 (pair z: real part column 2z, imaginary part 2z+1).
// Other CTAs may still read this CTA's Yb on return: the caller's next
// cluster barrier orders that before Yb is written again.
__device__ void big_inverse(const BigGeom& g, const double* X, int tid, int nt, double rP, double r2P) {
  const int P = g.P, C = g.C;
  for (int e = tid; e < g.nz * g.ML * g.S; e += nt) {
    const int m2 = e & (g.S - 1), row = e >> g.lgS;
    const int z = row / g.ML, ml = row - z * g.ML;
    const int m = (int)g.rank * g.ML + ml + g.R * m2;
    const int ca = 2 * z, cb = ca + 1;
    const bool hb = cb < C;
    const double* xl = X + ((size_t)ml * g.S + m2) * C;  // local modes at m
    const double am = xl[ca], bm = hb ? xl[cb] : 0.0;
    double2 v;
    if (m == 0 || 2 * m == P) {
      v = make_double2(am * rP, bm * rP);
    } else {
      const int mm = P - m, n1 = mm & (g.R - 1), n2 = mm >> g.lgR;
      const double* xr = dsmem(X, (unsigned)(n1 / g.ML)) + ((size_t)(n1 % g.ML) * g.S + n2) * C;
      const double amm = xr[ca], bmm = hb ? xr[cb] : 0.0;
      v = 2 * m < P ? make_double2((am - bmm) * r2P, (amm + bm) * r2P)
                    : make_double2((amm + bm) * r2P, (bmm - am) * r2P);
    }
    g.Yb[((size_t)row << g.lgS) + brev_n(m2, g.lgS)] = v;
  }
  __syncthreads();
  fft_rows(g.Yb, g.nz * g.ML, g.lgS, g.tw, g.lgP, 1.0, tid, nt);
  for (int e = tid; e < g.nz * g.ML * g.S; e += nt) {  // times e^{+2 pi i j2 m1 / P}
    const int j2 = e & (g.S - 1), ml = (e >> g.lgS) % g.ML;
    const int m1 = (int)g.rank * g.ML + ml;
    g.Yb[e] = cmul(tw_full(g.tw, j2 * m1, g.lgP), 1.0, g.Yb[e]);
  }
  cluster_barrier();
  for (int e = tid; e < g.nz * g.JL * g.R; e += nt) {
    const int m1 = e & (g.R - 1), row = e >> g.lgR;  // row = z JL + jl
    const int z = row / g.JL, jl = row - z * g.JL;
    const int j2 = (int)g.rank * g.JL + jl;
    const double2* src = dsmem(g.Yb, (unsigned)(m1 / g.ML));
    g.Ab[((size_t)row << g.lgR) + brev_n(m1, g.lgR)] = src[((size_t)(z * g.ML + m1 % g.ML) << g.lgS) + j2];
  }
  __syncthreads();
  fft_rows(g.Ab, g.nz * g.JL, g.lgR, g.tw, g.lgP, 1.0, tid, nt);
}

__device__ __forceinline__ void b_k_prop_big(const Dev& d, int mode) {
  extern __shared__ double sm[];
  __shared__ double red[(BIG_THREADS / 32) * NPART];
  __shared__ long long s_step;
  __shared__ long long s_d2[BIG_MAXA];
  __shared__ double qb[3 * BIG_MAXA];
  BigGeom g;
  g.CL = d.big_cl;
  g.rank = cluster_ctarank();
  const PropTile tl = d.tiles[d.n_tiles + blockIdx.x / g.CL];
  const int t = tl.type, N = d.N[t], k0 = tl.k0, na = tl.na;
  g.P = d.P[t];
  g.lgP = __ffs(g.P) - 1;
  g.lgR = g.lgP / 2;
  g.lgS = g.lgP - g.lgR;
  g.R = 1 << g.lgR;
  g.S = 1 << g.lgS;
  g.JL = g.S / g.CL;
  g.ML = g.R / g.CL;
  g.C = 3 * na;
  g.nz = (g.C + 1) >> 1;
  const int P = g.P, C = g.C, R = g.R, S = g.S;
  const int nown = g.ML * S;  // owned modes (and owned beads: JL R of them)
  g.tw = (double2*)sm;
  g.Ab = g.tw + P / 2;
  g.Yb = g.Ab + (size_t)g.nz * g.JL * R;
  g.Qm = (double*)(g.Yb + (size_t)g.nz * g.ML * S);
  g.Pm = g.Qm + (size_t)nown * C;
  double* Abd = (double*)g.Ab;
  const int tid = threadIdx.x, nt = blockDim.x;
  const double rP = rsqrt((double)P), r2P = rsqrt(2.0 * (double)P);
  const double m = d.mass[t];
  const double* cmg = d.cm + d.cm_off[t];
  const ModeCoef* mcf = d.mc + d.mc_off[t];
  const unsigned rank = g.rank;
  auto gidx = [&](int j, int c) -> size_t { return (size_t)(d.off[t] + j * N + k0) * 3 + c; };
  // owned bead (jl, j1) -> bead index; owned mode (ml, m2) -> mode index
  auto bead_of = [&](int jl, int j1) { return S * j1 + (int)rank * g.JL + jl; };
  auto mode_of = [&](int ml, int m2) { return (int)rank * g.ML + ml + R * m2; };
  // loads column values of the owned beads into Ab (bit-reversed over j1)
  auto load_cols = [&](const double* src) {
    if (C & 1)
      for (int e = tid; e < g.JL * R; e += nt) Abd[2 * ((size_t)(g.nz - 1) * g.JL * R + e) + 1] = 0.0;
    for (int e = tid; e < g.JL * R * C; e += nt) {
      const int c = e % C, o = e / C, j1 = o % R, jl = o / R;
      Abd[2 * (((size_t)((c >> 1) * g.JL + jl) << g.lgR) + brev_n(j1, g.lgR)) + (c & 1)] = src[gidx(bead_of(jl, j1), c)];
    }
  };

  if (tid == 0) s_step = *d.step_ctr;
  for (int e = tid; e < P / 2; e += nt) g.tw[e] = make_double2(cmg[2 * e], cmg[2 * e + 1]);
  for (int e = tid; e < na; e += nt) s_d2[e] = 0;
  const bool need_f = (mode & (PM_END | PM_START)) != 0;
  if (mode & PM_IMPORT) {
    for (int pass = 0; pass < 2; ++pass) {
      load_cols(pass == 0 ? d.q : d.p);
      big_forward(g, tid, nt);
      double* dst = pass == 0 ? g.Qm : g.Pm;
      for (int e = tid; e < nown * C; e += nt) {
        const int c = e % C, o = e / C, m2 = o % S, ml = o / S;
        dst[e] = big_mode(g, ml, m2, c, rP, r2P);
      }
    }
  } else {
    for (int e = tid; e < nown * C; e += nt) {
      const int c = e % C, o = e / C, m2 = o % S, ml = o / S;
      const size_t gi = gidx(mode_of(ml, m2), c);
      g.Qm[e] = d.q_nm[gi];
      g.Pm[e] = d.p_nm[gi];
    }
  }
  cluster_barrier();  // every CTA's modes in place (the centroid sits in CTA 0)
  for (int c = tid; c < C; c += nt) qb[c] = dsmem(g.Qm, 0u)[c] * rP;
  __syncthreads();
  double part[NPART] = {0, 0, 0, 0, 0, 0};
  if (need_f) {
    if (C & 1)
      for (int e = tid; e < g.JL * R; e += nt) Abd[2 * ((size_t)(g.nz - 1) * g.JL * R + e) + 1] = 0.0;
    for (int e = tid; e < g.JL * R * C; e += nt) {
      const int c = e % C, o = e / C, j1 = o % R, jl = o / R;
      const size_t gi = gidx(bead_of(jl, j1), c);
      const double f = fix_to_double(d.F_fix[gi], FINV);
      Abd[2 * (((size_t)((c >> 1) * g.JL + jl) << g.lgR) + brev_n(j1, g.lgR)) + (c & 1)] = f;
      if (mode & PM_END) d.f[gi] = f;
      if (mode & PM_START) d.F_fix[gi] = 0ull;
      if ((mode & PM_END) && (mode & PM_EST)) part[2] += (d.q[gi] - qb[c]) * f;
    }
    big_forward(g, tid, nt);
    const double hk = 0.5 * d.dt * d.kcal;  // F in kcal/mol/A -> amu A/fs^2
    const uint32_t s_end = (uint32_t)s_step;
    const uint32_t s_start = (uint32_t)(s_step + ((mode & PM_END) ? 1 : 0));
    const double inv2m = 0.5 / m;
    for (int e = tid; e < nown * C; e += nt) {
      const int c = e % C, o = e / C, m2 = o % S, ml = o / S;
      const int k = mode_of(ml, m2);
      const ModeCoef mk = mcf[k];
      const uint64_t dof = (uint64_t)gidx(k, c);
      double p = g.Pm[e], q = g.Qm[e];
      const double fk = big_mode(g, ml, m2, c, rP, r2P);
      if (mode & PM_END) {
        p = fma(hk, fk, p);
        const double xi = f2d_bits(gauss_dof(d.seed, s_end, 1u, dof));
        const double pn = fma(mk.c1, p, mk.c2s * xi);
        part[4] += (p * p - pn * pn) * inv2m;
        p = pn;
        if (mode & PM_EST) {
          part[0] += p * p * inv2m;
          part[1] += mk.hmw2 * q * q;
          if (k > 0) part[3] += q * q;
        }
      }
      if (mode & PM_START) {
        const double xi = f2d_bits(gauss_dof(d.seed, s_start, 0u, dof));
        const double pn = fma(mk.c1, p, mk.c2s * xi);
        part[5] += (p * p - pn * pn) * inv2m;
        p = fma(hk, fk, pn);
        const double pr = fma(mk.cw, p, -mk.mws * q);
        const double qr = fma(mk.swm, p, mk.cw * q);
        p = pr;
        q = qr;
      }
      g.Pm[e] = p;
      g.Qm[e] = q;
    }
  }
  if (mode & (PM_IMPORT | PM_END | PM_START)) {
    for (int e = tid; e < nown * C; e += nt) {
      const int c = e % C, o = e / C, m2 = o % S, ml = o / S;
      const size_t gi = gidx(mode_of(ml, m2), c);
      d.q_nm[gi] = g.Qm[e];
      d.p_nm[gi] = g.Pm[e];
    }
  }
  cluster_barrier();  // updated modes visible; every read of the forward pass's Yb done
  // Cartesian value of column c at owned bead (jl, j1) after big_inverse
  auto xc = [&](int jl, int j1, int c) -> double {
    return Abd[2 * (((size_t)((c >> 1) * g.JL + jl) << g.lgR) + j1) + (c & 1)];
  };
  if (mode & (PM_START | PM_QCART)) {
    big_inverse(g, g.Qm, tid, nt, rP, r2P);
    for (int e = tid; e < g.JL * R * C; e += nt) {
      const int c = e % C, o = e / C, j1 = o % R, jl = o / R;
      d.q[gidx(bead_of(jl, j1), c)] = xc(jl, j1, c);
    }
    cluster_barrier();  // bead 0 (CTA 0, jl = j1 = 0) visible
    const double* ab0 = (const double*)dsmem(g.Ab, 0u);
    for (int e = tid; e < g.JL * R * na; e += nt) {
      const int a = e % na, o = e / na, j1 = o % R, jl = o / R;
      const int j = bead_of(jl, j1);
      const int atom = d.atom_of_tk[d.atoff[t] + k0 + a];
      double x0[3], fl[3], rf[3];
      for (int x = 0; x < 3; ++x) {
        const int c = 3 * a + x;
        x0[x] = ab0[2 * ((size_t)((c >> 1) * g.JL) << g.lgR) + (c & 1)];
        MirrorOut::wrap_ref(x0[x], d.box, &fl[x], &rf[x]);
      }
      const double bx_ = xc(jl, j1, 3 * a), by_ = xc(jl, j1, 3 * a + 1), bz_ = xc(jl, j1, 3 * a + 2);
      write_mirror(d, d.off[t] + j * N + k0 + a, bx_, by_, bz_, fl[0], fl[1], fl[2], x0, d.off[t] + (k0 + a) * P + j);
      if (j == 0) {
        write_ref(d, atom, rf, fl);
      } else {
        const double d2 = bead_d2(bx_ - x0[0], by_ - x0[1], bz_ - x0[2]);
        atomicMax(&s_d2[a], __double_as_longlong(d2));  // this CTA's beads
      }
    }
    cluster_barrier();  // every CTA's maximum in place; every read of bead 0 done
    if (rank == 0)
      for (int a = tid; a < na; a += nt) {
        long long mx = 0;
        for (int r = 0; r < g.CL; ++r) mx = max(mx, dsmem(s_d2, (unsigned)r)[a]);
        d.spread[d.atom_of_tk[d.atoff[t] + k0 + a]] = __dsqrt_rn(__longlong_as_double(mx));
      }
  }
  if (mode & PM_PCART) {
    cluster_barrier();  // every read of the position pass's Yb and Ab done
    big_inverse(g, g.Pm, tid, nt, rP, r2P);
    for (int e = tid; e < g.JL * R * C; e += nt) {
      const int c = e % C, o = e / C, j1 = o % R, jl = o / R;
      d.p[gidx(bead_of(jl, j1), c)] = xc(jl, j1, c);
    }
  }
  if (mode & (PM_END | PM_START)) {
    block_sum6(part, red);
    if (tid == 0)
      for (int i = 0; i < NPART; ++i) d.parts[(size_t)(tl.slot + (int)rank) * NPART + i] = red[i];
  }
  cluster_barrier();  // no CTA leaves while another may still read its shared memory
}

__global__ void __launch_bounds__(BIG_THREADS) k_prop_big(const __grid_constant__ Dev d, int mode) { b_k_prop_big(d, mode); }

// ---------------------------------------------------------------------------
// step finalisation: reduce estimator partials in a fixed order, advance the
// step counter, clear the energy accumulators
// ---------------------------------------------------------------------------
__device__ __forceinline__ void b_k_final(const Dev& d, int bx, int mode) {
  (void)bx;
  __shared__ double acc[MT * 4 + 2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int nq = d.n_types * 4 + 2;
  const bool have = (mode & (PM_END | PM_START)) != 0;
  if (have) {
    for (int x = warp; x < nq; x += nw) {
      double a = 0.0;
      if (x < d.n_types * 4) {
        const int t = x / 4, qi = x % 4;
        for (int s = lane; s < d.n_part_slots; s += 32)
          if (d.slot_type[s] == t) a += d.parts[(size_t)s * NPART + qi];
      } else {
        const int qi = 4 + (x - d.n_types * 4);
        for (int s = lane; s < d.n_part_slots; s += 32) a += d.parts[(size_t)s * NPART + qi];
      }
      a = warp_sum(a);
      if (lane == 0) acc[x] = a;
    }
  }
  __syncthreads();
  if (tid != 0) return;
  double* est = d.est;
  const double kc = d.kcal;
  double heat = *d.heat;
  if (have) heat += acc[d.n_types * 4] / kc;  // end-of-step thermostat half
  if (mode & PM_END) {
    double v[E_NSLOTS];
    for (int i = 0; i < E_NSLOTS; ++i) v[i] = (double)(long long)d.E_fix[i] * EINV;
    const double V = v[E_LJ] + v[E_COUL] + v[E_BOND] + v[E_ANGLE] + v[E_PSEUDO];
    double ke = 0.0, es = 0.0;
    for (int t = 0; t < d.n_types; ++t) {
      ke += acc[4 * t] / kc;
      es += acc[4 * t + 1] / kc;
    }
    est[0] = V;
    est[1] = v[E_LJ];
    est[2] = v[E_COUL];
    est[3] = v[E_BOND];
    est[4] = v[E_ANGLE];
    est[5] = v[E_PSEUDO];
    est[6] = ke;
    est[7] = es;
    est[8] = v[E_VIRIAL];
    // counters are integers carried in the fixed-point slots
    // full lists (FP32 forces) see every pair term from both atoms
    const double cnt_scale = d.full_list ? 0.5 : 1.0;
    est[13] = cnt_scale * (double)(long long)d.E_fix[E_NEVAL];
    est[14] = (double)(long long)d.E_fix[E_NPEVAL];
    est[16 + 4 * MT] = cnt_scale * (double)(long long)d.E_fix[E_NLJEVAL];
    est[9] = 2.0 * ke * kc / (3.0 * (double)d.n_beads * d.kB);
    est[11] = heat;
    est[10] = ke + es + V;
    est[12] = est[10] + heat;
    const long long st = *d.step_ctr + 1;
    est[15] = (double)st;
    for (int t = 0; t < d.n_types; ++t) {
      const double nP = (double)d.N[t] * d.P[t];
      const double espr = acc[4 * t + 1] / kc;
      const double kT_kcal = d.kT / kc;
      est[16 + 4 * t] = 1.5 * nP * kT_kcal - espr;
      est[16 + 4 * t + 1] = 1.5 * d.N[t] * kT_kcal - 0.5 * acc[4 * t + 2];
      est[16 + 4 * t + 2] = nP > 0 ? acc[4 * t + 3] / nP : 0.0;
      est[16 + 4 * t + 3] = espr;
    }
    *d.step_ctr = st;
  }
  if (have) heat += acc[d.n_types * 4 + 1] / kc;  // start-of-step thermostat half
  *d.heat = heat;
  for (int i = 0; i < E_NSLOTS; ++i) d.E_fix[i] = 0ull;
}

__global__ void k_final(const __grid_constant__ Dev d, int mode) { b_k_final(d, blockIdx.x, mode); }

__global__ void k_final_b(const Dev* __restrict__ devs, const int* __restrict__ pfx, int nm, int mode) {
  MX_BATCH_ENTER();
  b_k_final(d, bx, mode);
}

// caller forces and the energy record after a bare force evaluation
__global__ void k_forces_out(Dev d) {
  const size_t n = (size_t)d.n_beads * 3;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    d.f[e] = fix_to_double(d.F_fix[e], FINV);
    d.F_fix[e] = 0ull;
  }
}

__global__ void k_energy_out(Dev d) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double v[E_NSLOTS];
  for (int i = 0; i < E_NSLOTS; ++i) v[i] = (double)(long long)d.E_fix[i] * EINV;
  d.est[0] = v[E_LJ] + v[E_COUL] + v[E_BOND] + v[E_ANGLE] + v[E_PSEUDO];
  d.est[1] = v[E_LJ];
  d.est[2] = v[E_COUL];
  d.est[3] = v[E_BOND];
  d.est[4] = v[E_ANGLE];
  d.est[5] = v[E_PSEUDO];
  d.est[8] = v[E_VIRIAL];
  const double cnt_scale = d.full_list ? 0.5 : 1.0;
  d.est[13] = cnt_scale * (double)(long long)d.E_fix[E_NEVAL];
  d.est[14] = (double)(long long)d.E_fix[E_NPEVAL];
  d.est[16 + 4 * MT] = cnt_scale * (double)(long long)d.E_fix[E_NLJEVAL];
  for (int i = 0; i < E_NSLOTS; ++i) d.E_fix[i] = 0ull;
}

__global__ void k_gauss(Dev d, uint32_t step, uint32_t stage, uint64_t dof0, long n, float* out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = gauss_dof(d.seed, step, stage, dof0 + (uint64_t)i);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static size_t small_smem(int P) {
  const int C = 3 * (PROP_TILE_BEADS / P);
  return sizeof(double) * ((size_t)P * P + 5 * (size_t)P * C);
}

// dynamic shared memory beyond the 48 KB default needs an opt-in per kernel
static void prop_smem_optin() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_prop_small, cudaFuncAttributeMaxDynamicSharedMemorySize, PROP_SMEM_MAX);
  cudaFuncSetAttribute(k_prop_big, cudaFuncAttributeMaxDynamicSharedMemorySize, PROP_SMEM_MAX);
  cudaFuncSetAttribute(k_prop_big, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  done = true;
}

int launch_prop(const Dev& d, cudaStream_t s, int mode, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join) {
  int n = 0;
  prop_smem_optin();
  if (mode & PM_MIRROR) {
    k_mirror_from_q<<<(d.n_atoms + 127) / 128, 128, 0, s>>>(d);
    return 1;
  }
  // the large-P clusters (few SMs, latency-bound) run beside the small-P
  // tiles when a side stream is given: the two touch disjoint rows, atoms
  // and estimator slots
  const bool split = side && ev_fork && ev_join && d.n_tiles > 0 && d.n_big_tiles > 0;
  cudaStream_t sb = s;
  if (split) {
    cudaEventRecord(ev_fork, s);
    cudaStreamWaitEvent(side, ev_fork, 0);
    sb = side;
  }
  if (d.n_big_tiles > 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)d.big_cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(d.n_big_tiles * d.big_cl));
    cfg.blockDim = dim3(BIG_THREADS);
    cfg.dynamicSmemBytes = (size_t)d.big_smem;
    cfg.stream = sb;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_prop_big, d, mode);
    ++n;
  }
  if (d.n_tiles > 0) {
    size_t smem = 0;
    for (int t = 0; t < d.n_types; ++t)
      if (d.P[t] <= SMALL_P && d.N[t] > 0) smem = small_smem(d.P[t]) > smem ? small_smem(d.P[t]) : smem;
    k_prop_small<<<d.n_tiles, PROP_THREADS, smem, s>>>(d, mode);
    ++n;
  }
  if (split) {
    cudaEventRecord(ev_join, side);
    cudaStreamWaitEvent(s, ev_join, 0);
  }
  return n;
}

int big_cluster_pick(int cl_max, const int* P, const int* na, int n, int* smem) {
  prop_smem_optin();
  for (int cl = cl_max; cl >= 1; cl >>= 1) {
    size_t need = 0;
    for (int i = 0; i < n; ++i) need = std::max(need, big_prop_smem(P[i], na[i], cl));
    if (need > (size_t)PROP_SMEM_MAX) return 0;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)cl);
    cfg.blockDim = dim3(BIG_THREADS);
    cfg.dynamicSmemBytes = need;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, k_prop_big, &cfg) == cudaSuccess && nc > 0) {
      *smem = (int)need;
      return cl;
    }
    cudaGetLastError();  // clear a refused query before trying a smaller cluster
  }
  return 0;
}

size_t batch_prop_smem(const Dev& d) {
  size_t smem = 0;
  for (int t = 0; t < d.n_types; ++t)
    if (d.P[t] <= SMALL_P && d.N[t] > 0) smem = small_smem(d.P[t]) > smem ? small_smem(d.P[t]) : smem;
  return smem;
}

// propagation (types with P <= SMALL_P) and step finalisation of every
// member of a batch, one launch per kernel
int launch_step_batched(const BatchGeom& g, cudaStream_t s, int mode, int parts) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_prop_small_b, cudaFuncAttributeMaxDynamicSharedMemorySize, PROP_SMEM_MAX);
    attr = true;
  }
  const int r = g.nm + 1;
  int n = 0;
  if ((parts & 1) && g.blocks[BK_PROP] > 0) {
    k_prop_small_b<<<g.blocks[BK_PROP], PROP_THREADS, g.prop_smem, s>>>(g.devs, g.pfx + BK_PROP * r, g.nm, mode);
    ++n;
  }
  if (parts & 2) {
    k_final_b<<<g.blocks[BK_FINAL], 1024, 0, s>>>(g.devs, g.pfx + BK_FINAL * r, g.nm, mode);
    ++n;
  }
  return n;
}

int launch_final(const Dev& d, cudaStream_t s, int mode, const int* slot_type) {
  (void)slot_type;  // carried in d
  k_final<<<1, 1024, 0, s>>>(d, mode);
  return 1;
}

int launch_forces_out(const Dev& d, cudaStream_t s) {
  k_forces_out<<<296, 256, 0, s>>>(d);
  k_energy_out<<<1, 32, 0, s>>>(d);
  return 2;
}

int launch_gauss(const Dev& d, cudaStream_t s, uint32_t step, uint32_t stage, uint64_t dof0, long n, float* out) {
  long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_gauss<<<(int)blocks, 256, 0, s>>>(d, step, stage, dof0, n, out);
  return 1;
}

}  // namespace mx
