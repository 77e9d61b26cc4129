// k_prop.cu -- ring-polymer propagation: normal-mode transforms, PILE
// thermostat half steps, half kicks and the exact free-ring rotation of the
// split propagator (Sec. "Evaluation"), plus the per-step estimator partials
// (Sec. "Output and Analysis") and the position mirrors the force kernels read.
//
// Types with P <= SMALL_P: one CTA owns all P beads of a few atoms (a P x C
// column tile, C = 3 * atoms) in shared memory and runs transform ->
// elementwise update -> inverse transform in one pass. Types with larger P
// (the 1024-bead electron) split the transforms over many CTAs by mode/bead
// blocks, with the cosine table in shared memory.
#include <math.h>

#include "mixts_internal.cuh"

namespace mx {

constexpr int PROP_THREADS = 384;  // one thread per element of a P x C tile (P C = 384)
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
// Half the multiply-adds of the dense products, in another rounding order.
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
  __shared__ long long s_d2[128];
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
  if (mode & PM_IMPORT) {
    nm_fold(Xc, P, C, tid, nt);
    nm_fold(Fb, P, C, tid, nt);
    __syncthreads();
    nm_forward_folded(Cm, P, C, Xc, Qn, tid, nt);
    nm_forward_folded(Cm, P, C, Fb, Pn, tid, nt);
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
    nm_forward_folded(Cm, P, C, Fb, Fn, tid, nt);
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
  if (P > SMALL_P) {  // a large-P atom: its block partials must not keep older values
    const int nb = P / BIG_MB;
    for (int s = 0; s < nb; ++s) d.spread_big[d.sb_off[t] + k * nb + s] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// large-P path
// ---------------------------------------------------------------------------
// element (j, k) of the orthonormal normal-mode matrix; T holds
// sqrt(2/P) cos(2 pi m / P), so the cos and sin modes need no multiply
__device__ __forceinline__ double cjk(const double* T, int P, int j, int k, double rP) {
  if (k == 0) return rP;
  if (2 * k < P) return T[(j * k) & (P - 1)];
  if (2 * k == P) return (j & 1) ? -rP : rP;
  return T[(j * k - P / 4) & (P - 1)];  // sin(2 pi jk / P) = cos(2 pi (jk - P/4) / P)
}

constexpr int BIG_CC = 3;  // columns (one atom's x, y, z) per warp of the large-P transforms

// launch shapes of the large-P transforms, and the number of warps that
// share one output group's sum (measured: the forward pass is fastest with 8
// warps and no split, the inverse with 32 warps and a 4-way split)
constexpr int FWD_THREADS = 256, FWD_SPLIT = 1;
constexpr int INV_THREADS = 1024, INV_SPLIT = 4;

// forward transforms (C^T x) of this block's BIG_MB modes and the elementwise
// step on them
__global__ void __launch_bounds__(FWD_THREADS) k_big_fwd(Dev d, int t, int mode) {
  extern __shared__ double sm[];
  const int P = d.P[t], N = d.N[t], C = 3 * N;
  double* T = sm;                       // [P]
  double* Fn = T + P;                   // [BIG_MB*C]
  double* Qi = Fn + BIG_MB * C;         // [BIG_MB*C] imported q modes
  double* Pi = Qi + BIG_MB * C;         // [BIG_MB*C]
  double* qbar = Pi + BIG_MB * C;       // [C]
  __shared__ double red[(FWD_THREADS / 32) * NPART];
  __shared__ long long s_step;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int kb = blockIdx.x * BIG_MB;
  const double rP = rsqrt((double)P);
  const double* cmg = d.cm + d.cm_off[t];
  const ModeCoef* mcf = d.mc + d.mc_off[t];
  const size_t base = (size_t)d.off[t] * 3;  // element (j, c) at base + j*C + c
  if (tid == 0) s_step = *d.step_ctr;
  for (int e = tid; e < P; e += blockDim.x) T[e] = cmg[e];
  __syncthreads();
  const bool need_f = (mode & (PM_END | PM_START)) != 0;
  const int nout = BIG_MB * C;
  // FWD_SPLIT warps per (mode, group of BIG_CC columns), each over a share of
  // the beads: every matrix element is looked up once and feeds BIG_CC
  // independent FMA chains; the shares are added in a fixed order
  __shared__ double pbuf[FWD_THREADS / 32][3 * BIG_CC];
  const int ncg = (C + BIG_CC - 1) / BIG_CC;
  const int items = BIG_MB * ncg, slots = nw / FWD_SPLIT;
  const int qs = warp % FWD_SPLIT, slot = warp / FWD_SPLIT;
  for (int b0 = 0; b0 < items; b0 += slots) {
    const int o = b0 + slot;
    double af[BIG_CC], aq[BIG_CC], ap[BIG_CC];
#pragma unroll
    for (int u = 0; u < BIG_CC; ++u) af[u] = aq[u] = ap[u] = 0.0;
    const int kk = o / ncg, c0 = (o - kk * ncg) * BIG_CC;
    const int k = kb + kk;
    const int ncol = o < items ? min(BIG_CC, C - c0) : 0;
    for (int j = lane + 32 * qs; ncol > 0 && j < P; j += 32 * FWD_SPLIT) {
      const double cj = cjk(T, P, j, k, rP);
      const size_t g = base + (size_t)j * C + c0;
#pragma unroll
      for (int u = 0; u < BIG_CC; ++u) {
        if (u < ncol) {
          if (need_f) af[u] = fma(cj, fix_to_double(d.F_fix[g + u], FINV), af[u]);
          if (mode & PM_IMPORT) {
            aq[u] = fma(cj, d.q[g + u], aq[u]);
            ap[u] = fma(cj, d.p[g + u], ap[u]);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < BIG_CC; ++u) {
      if (need_f) af[u] = warp_sum(af[u]);
      if (mode & PM_IMPORT) {
        aq[u] = warp_sum(aq[u]);
        ap[u] = warp_sum(ap[u]);
      }
      if (lane == 0) {
        pbuf[warp][u] = af[u];
        pbuf[warp][BIG_CC + u] = aq[u];
        pbuf[warp][2 * BIG_CC + u] = ap[u];
      }
    }
    __syncthreads();
    if (tid < slots * 3 * BIG_CC) {
      const int sl = tid / (3 * BIG_CC), v = tid - sl * (3 * BIG_CC);
      const int kind = v / BIG_CC, u = v - kind * BIG_CC;
      const int oo = b0 + sl;
      const int kk2 = oo / ncg, c2 = (oo - kk2 * ncg) * BIG_CC;
      if (oo < items && u < min(BIG_CC, C - c2)) {
        double sum = 0.0;
        for (int w = 0; w < FWD_SPLIT; ++w) sum += pbuf[sl * FWD_SPLIT + w][v];
        double* dst = kind == 0 ? Fn : (kind == 1 ? Qi : Pi);
        dst[kk2 * C + c2 + u] = sum;
      }
    }
    __syncthreads();
  }
  double part[NPART] = {0, 0, 0, 0, 0, 0};
  if ((mode & PM_END) && (mode & PM_EST)) {
    for (int c = warp; c < C; c += nw) {
      double a = 0.0;
      for (int j = lane; j < P; j += 32) a += d.q[base + (size_t)j * C + c];
      a = warp_sum(a);
      if (lane == 0) qbar[c] = a / P;
    }
  }
  __syncthreads();
  if (need_f) {
    // this block's bead range: caller forces and the centroid virial
    for (int e = tid; e < nout; e += blockDim.x) {
      const int j = kb + e / C, c = e - (e / C) * C;
      const size_t g = base + (size_t)j * C + c;
      const double f = fix_to_double(d.F_fix[g], FINV);
      if (mode & PM_END) {
        d.f[g] = f;
        if (mode & PM_EST) part[2] += (d.q[g] - qbar[c]) * f;
      }
    }
  }
  const double m = d.mass[t];
  const double inv2m = 0.5 / m;
  const double hk = 0.5 * d.dt * d.kcal;
  const uint32_t s_end = (uint32_t)s_step;
  const uint32_t s_start = (uint32_t)(s_step + ((mode & PM_END) ? 1 : 0));
  for (int e = tid; e < nout; e += blockDim.x) {
    const int k = kb + e / C, c = e - (e / C) * C;
    const size_t g = base + (size_t)k * C + c;
    double p, q;
    if (mode & PM_IMPORT) {
      p = Pi[e];
      q = Qi[e];
    } else {
      p = d.p_nm[g];
      q = d.q_nm[g];
    }
    if (need_f) {
      const ModeCoef mk = mcf[k];
      const double fk = Fn[e];
      if (mode & PM_END) {
        p = fma(hk, fk, p);
        const double xi = f2d_bits(gauss_dof(d.seed, s_end, 1u, (uint64_t)g));
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
        const double xi = f2d_bits(gauss_dof(d.seed, s_start, 0u, (uint64_t)g));
        const double pn = fma(mk.c1, p, mk.c2s * xi);
        part[5] += (p * p - pn * pn) * inv2m;
        p = fma(hk, fk, pn);
        const double pr = fma(mk.cw, p, -mk.mws * q);
        const double qr = fma(mk.swm, p, mk.cw * q);
        p = pr;
        q = qr;
      }
    }
    if (mode & (PM_IMPORT | PM_END | PM_START)) {
      d.p_nm[g] = p;
      d.q_nm[g] = q;
    }
  }
  if (need_f) {
    block_sum6(part, red);
    if (tid == 0)
      for (int i = 0; i < NPART; ++i) d.parts[(size_t)(d.big_slot0[t] + blockIdx.x) * NPART + i] = red[i];
  }
}

// inverse transforms (C x) of this block's BIG_MB beads, mirrors, spread
__global__ void __launch_bounds__(INV_THREADS) k_big_inv(Dev d, int t, int mode) {
  extern __shared__ double sm[];
  const int P = d.P[t], N = d.N[t], C = 3 * N;
  double* T = sm;
  double* Qc = T + P;                 // [(BIG_MB+1)*C], row 0 = bead 0, rows 1.. = own beads
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int jb = blockIdx.x * BIG_MB;
  const double rP = rsqrt((double)P);
  const double* cmg = d.cm + d.cm_off[t];
  const size_t base = (size_t)d.off[t] * 3;
  for (int e = tid; e < P; e += blockDim.x) T[e] = cmg[e];
  __syncthreads();
  const bool qc = (mode & (PM_START | PM_QCART)) != 0;
  const int nout = (BIG_MB + 1) * C;
  if (qc || (mode & PM_PCART)) {
    // INV_SPLIT warps per (bead, group of BIG_CC columns), as in the forward pass
    __shared__ double pbuf[INV_THREADS / 32][2 * BIG_CC];
    const int ncg = (C + BIG_CC - 1) / BIG_CC;
    const int items = (BIG_MB + 1) * ncg, slots = nw / INV_SPLIT;
    const int qs = warp % INV_SPLIT, slot = warp / INV_SPLIT;
    for (int b0 = 0; b0 < items; b0 += slots) {
      const int o = b0 + slot;
      const int r = o / ncg, c0 = (o - r * ncg) * BIG_CC;
      const int j = r == 0 ? 0 : jb + r - 1;
      const int ncol = o < items ? min(BIG_CC, C - c0) : 0;
      double aq[BIG_CC], ap[BIG_CC];
#pragma unroll
      for (int u = 0; u < BIG_CC; ++u) aq[u] = ap[u] = 0.0;
      for (int k = lane + 32 * qs; ncol > 0 && k < P; k += 32 * INV_SPLIT) {
        const double cj = cjk(T, P, j, k, rP);
        const size_t g = base + (size_t)k * C + c0;
#pragma unroll
        for (int u = 0; u < BIG_CC; ++u) {
          if (u < ncol) {
            if (qc) aq[u] = fma(cj, d.q_nm[g + u], aq[u]);
            if (mode & PM_PCART) ap[u] = fma(cj, d.p_nm[g + u], ap[u]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < BIG_CC; ++u) {
        if (qc) aq[u] = warp_sum(aq[u]);
        if (mode & PM_PCART) ap[u] = warp_sum(ap[u]);
        if (lane == 0) {
          pbuf[warp][u] = aq[u];
          pbuf[warp][BIG_CC + u] = ap[u];
        }
      }
      __syncthreads();
      if (tid < slots * 2 * BIG_CC) {
        const int sl = tid / (2 * BIG_CC), v = tid - sl * (2 * BIG_CC);
        const int kind = v / BIG_CC, u = v - kind * BIG_CC;
        const int oo = b0 + sl;
        const int r2 = oo / ncg, c2 = (oo - r2 * ncg) * BIG_CC;
        const int j2 = r2 == 0 ? 0 : jb + r2 - 1;
        if (oo < items && u < min(BIG_CC, C - c2)) {
          double sum = 0.0;
          for (int w = 0; w < INV_SPLIT; ++w) sum += pbuf[sl * INV_SPLIT + w][v];
          if (kind == 0 && qc) Qc[r2 * C + c2 + u] = sum;
          if (kind == 1 && (mode & PM_PCART) && r2 > 0) d.p[base + (size_t)j2 * C + c2 + u] = sum;
        }
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (qc) {
    for (int e = tid; e < BIG_MB * C; e += blockDim.x) {
      const int j = jb + e / C, c = e - (e / C) * C;
      d.q[base + (size_t)j * C + c] = Qc[C + e];
    }
    for (int e = tid; e < BIG_MB * N; e += blockDim.x) {
      const int jj = e / N, a = e - (e / N) * N;
      const int j = jb + jj;
      const int atom = d.atom_of_tk[d.atoff[t] + a];
      double fl[3], rf[3];
      for (int x = 0; x < 3; ++x) MirrorOut::wrap_ref(Qc[3 * a + x], d.box, &fl[x], &rf[x]);
      const double* xb = Qc + (size_t)(jj + 1) * C + 3 * a;
      write_mirror(d, d.off[t] + j * N + a, xb[0], xb[1], xb[2], fl[0], fl[1], fl[2], Qc + 3 * a, d.off[t] + a * P + j);
      if (jj == 0 && blockIdx.x == 0) write_ref(d, atom, rf, fl);
    }
    // spread partial of this bead block, per atom
    for (int a = warp; a < N; a += nw) {
      double sp = 0.0;
      for (int jj = lane; jj < BIG_MB; jj += 32) {
        const int j = jb + jj;
        if (j == 0) continue;
        const double* xb = Qc + (size_t)(jj + 1) * C + 3 * a;
        const double dd = bead_dist(xb[0] - Qc[3 * a], xb[1] - Qc[3 * a + 1], xb[2] - Qc[3 * a + 2]);
        sp = dd > sp ? dd : sp;
      }
      for (int o = 16; o > 0; o >>= 1) sp = fmax(sp, __shfl_xor_sync(0xffffffffu, sp, o));
      if (lane == 0) {
        const int atom = d.atom_of_tk[d.atoff[t] + a];
        d.spread_big[d.sb_off[t] + a * gridDim.x + blockIdx.x] = sp;
        if (blockIdx.x == 0) d.spread[atom] = 0.0;
      }
    }
  }
  if (mode & PM_START) {
    for (int e = tid; e < BIG_MB * C; e += blockDim.x) {
      const int j = jb + e / C, c = e - (e / C) * C;
      d.F_fix[base + (size_t)j * C + c] = 0ull;
    }
  }
}

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
  const int C = 3 * (128 / P);
  return sizeof(double) * ((size_t)P * P + 5 * (size_t)P * C);
}

// dynamic shared memory beyond the 48 KB default needs an opt-in per kernel
static void prop_smem_optin() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_prop_small, cudaFuncAttributeMaxDynamicSharedMemorySize, PROP_SMEM_MAX);
  cudaFuncSetAttribute(k_big_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, PROP_SMEM_MAX);
  cudaFuncSetAttribute(k_big_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, PROP_SMEM_MAX);
  done = true;
}

int launch_prop(const Dev& d, cudaStream_t s, int mode) {
  int n = 0;
  prop_smem_optin();
  if (mode & PM_MIRROR) {
    k_mirror_from_q<<<(d.n_atoms + 127) / 128, 128, 0, s>>>(d);
    return 1;
  }
  if (d.n_tiles > 0) {
    size_t smem = 0;
    for (int t = 0; t < d.n_types; ++t)
      if (d.P[t] <= SMALL_P && d.N[t] > 0) smem = small_smem(d.P[t]) > smem ? small_smem(d.P[t]) : smem;
    k_prop_small<<<d.n_tiles, PROP_THREADS, smem, s>>>(d, mode);
    ++n;
  }
  for (int t = 0; t < d.n_types; ++t) {
    if (d.P[t] <= SMALL_P || d.N[t] == 0) continue;
    const int C = 3 * d.N[t];
    const int nb = d.P[t] / BIG_MB;
    if (mode & (PM_IMPORT | PM_END | PM_START)) {
      const size_t smem = sizeof(double) * ((size_t)d.P[t] + 3 * (size_t)BIG_MB * C + C);
      k_big_fwd<<<nb, FWD_THREADS, smem, s>>>(d, t, mode);
      ++n;
    }
    if (mode & (PM_START | PM_QCART | PM_PCART)) {
      const size_t smem = sizeof(double) * ((size_t)d.P[t] + (size_t)(BIG_MB + 1) * C);
      k_big_inv<<<nb, INV_THREADS, smem, s>>>(d, t, mode);
      ++n;
    }
  }
  return n;
}

size_t batch_prop_smem(const Dev& d) {
  size_t smem = 0;
  for (int t = 0; t < d.n_types; ++t)
    if (d.P[t] <= SMALL_P && d.N[t] > 0) smem = small_smem(d.P[t]) > smem ? small_smem(d.P[t]) : smem;
  return smem;
}

// propagation (types with P <= SMALL_P) and step finalisation of every
// member of a batch, one launch per kernel
int launch_step_batched(const BatchGeom& g, cudaStream_t s, int mode) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_prop_small_b, cudaFuncAttributeMaxDynamicSharedMemorySize, PROP_SMEM_MAX);
    attr = true;
  }
  const int r = g.nm + 1;
  int n = 0;
  if (g.blocks[BK_PROP] > 0) {
    k_prop_small_b<<<g.blocks[BK_PROP], PROP_THREADS, g.prop_smem, s>>>(g.devs, g.pfx + BK_PROP * r, g.nm, mode);
    ++n;
  }
  k_final_b<<<g.blocks[BK_FINAL], 1024, 0, s>>>(g.devs, g.pfx + BK_FINAL * r, g.nm, mode);
  return n + 1;
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
