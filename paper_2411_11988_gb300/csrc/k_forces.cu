// k_forces.cu -- neighbour search and the mixTS force sweep.
//
// Pair terms of Eq. (mts-hamiltonian): the pair (i, j) with P_i >= P_j is
// owned by i (the finer ring polymer), and bead b of i meets bead
// floor(b P_j / P_i) = b >> (log2 P_i - log2 P_j) of j with weight 1/P_i.
// Work item = (owner atom i, bead b of i): one warp walks i's list row,
// lanes over entries. Reaction forces on the partner beads go to a 64-bit
// fixed-point accumulator, so the result is independent of atomic order.
#include <math.h>

#include <algorithm>

#include "fixmath.cuh"
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
//   except, for a same-molecule pair, the image n = w_other - w_owner with
//   q_0 = r + w L (the zero image of the caller's unwrapped coordinates,
//   where the intramolecular terms live). Owner = finer atom; between equal bead
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

// (float)(k - 2) for 0 <= k < 2^23 without a conversion instruction:
// 2^23 + k has k in its mantissa bits.
__device__ __forceinline__ float img_of(int k) { return __int_as_float(0x4B000000 | k) - 8388610.0f; }

// bit k of the result when |d + (k - 2) L| < Rlin for the one image k
__device__ __forceinline__ unsigned img_bit(float dd, int k, float Lf, float Rlin) {
  return fabsf(dd + img_of(k) * Lf) < Rlin ? 1u << k : 0u;
}

// bit k of the result is set when |d + (k - 2) L| < Rlin, k = 0..4
__device__ __forceinline__ unsigned img_mask(float dd, float Lf, float Rlin) {
  unsigned m = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k) m |= (fabsf(dd + (float)(k - 2) * Lf) < Rlin ? 1u : 0u) << k;
  return m;
}

// max spread over atoms whose pseudo flag equals want; spreads are
// non-negative doubles, whose bit patterns order like the values, so the max
// runs on integer instructions
__device__ double reduce_spread_kind(const Dev& d, const int* atom_is_pseudo, int want, long long* red) {
  long long m = 0;
  for (int a = threadIdx.x; a < d.n_atoms; a += blockDim.x)
    if (atom_is_pseudo[a] == want) m = max(m, __double_as_longlong(d.spread[a]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  long long r = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = max(r, red[w]);
  __syncthreads();
  return __longlong_as_double(r);
}

constexpr int NL_THREADS = 256;

// integer part of 0 <= v < 2^22 without a conversion instruction (those
// share the slow FP64 unit): (v - 1/2) + 2^23 rounds to floor(v) in the
// mantissa bits (a tie at an integer v may give v - 1, harmless for cells)
__device__ __forceinline__ int floor_small(float v) {
  return __float_as_int(__fadd_rn(__fadd_rn(v, -0.5f), 8388608.0f)) - 0x4B000000;
}

// cell of a wrapped bead-0 reference (binary32 position in [0, L)); the
// list-prep sort and the search use this one function
__device__ __forceinline__ int cell_of(float4 r, float inv_side, int nc) {
  const int cx = min(max(floor_small(r.x * inv_side), 0), nc - 1);
  const int cy = min(max(floor_small(r.y * inv_side), 0), nc - 1);
  const int cz = min(max(floor_small(r.z * inv_side), 0), nc - 1);
  return (cx * nc + cy) * nc + cz;
}

// Once per list build: d_max of sites and of pseudo particles, the two list
// radii (binary64, in the order the definition states), and cleared row
// counters. thresh: [0] d_max, [1] R, [2] d_max pseudo, [3] R pseudo. With
// a cell grid, also the atoms sorted by cell (a counting sort in shared
// memory; the order inside a cell is arbitrary) and whether this step's
// radius fits the cell side.
__device__ __forceinline__ void b_k_list_prep(const Dev& d, int bx) {
  (void)bx;
  __shared__ long long red[32];
  __shared__ int ccnt[NC_MAX * NC_MAX * NC_MAX];
  __shared__ int wtot[32];
  const double ds = reduce_spread_kind(d, d.atom_is_pseudo, 0, red);
  const double dp = reduce_spread_kind(d, d.atom_is_pseudo, 1, red);
  if (d.nc > 0) {
    const int nc = d.nc, ncell = nc * nc * nc;
    const float inv_side = d.cell_inv;
    for (int c = threadIdx.x; c < ncell; c += blockDim.x) ccnt[c] = 0;
    __syncthreads();
    for (int a = threadIdx.x; a < d.n_nonp; a += blockDim.x) atomicAdd(&ccnt[cell_of(d.reff[a], inv_side, nc)], 1);
    __syncthreads();
    // exclusive scan over the cells: each thread a contiguous run of cells
    const int per = (ncell + blockDim.x - 1) / blockDim.x;
    const int c0 = threadIdx.x * per, c1 = min(c0 + per, ncell);
    int run = 0;
    for (int c = c0; c < c1; ++c) run += ccnt[c];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = run;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) wtot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int v = lane < (int)(blockDim.x >> 5) ? wtot[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      wtot[lane] = v;
    }
    __syncthreads();
    int start = (wid > 0 ? wtot[wid - 1] : 0) + incl - run;
    for (int c = c0; c < c1; ++c) {
      const int n = ccnt[c];
      d.cell_start[c] = start;
      ccnt[c] = start;  // next free slot of the cell
      start += n;
    }
    if (threadIdx.x == 0) d.cell_start[ncell] = d.n_nonp;
    __syncthreads();
    for (int a = threadIdx.x; a < d.n_nonp; a += blockDim.x)
      d.cell_atoms[atomicAdd(&ccnt[cell_of(d.reff[a], inv_side, nc)], 1)] = a;
  }
  for (int i = threadIdx.x; i < d.n_nonp; i += blockDim.x) d.nl_cnt[i] = 0;
  for (int i = threadIdx.x; i < d.n_pseudo; i += blockDim.x) d.pl_cnt[i] = 0;
  // pair items of the new list and their hand-out counters (one per window
  // of the FP32 window sweep)
  if (threadIdx.x < 2 + (d.p32w ? 1 << d.p32w_lgnw : 0)) d.pctr[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    const double L = d.box;
    const double R = __dadd_rn(d.rc, __dmul_rn(2.0, ds));
    const double Rp = __dadd_rn(__dadd_rn(d.rc, ds), dp);
    d.thresh[0] = ds;
    d.thresh[1] = R;
    d.thresh[2] = dp;
    d.thresh[3] = Rp;
    d.thresh[10] = __dmul_rn(R, R);
    d.thresh[11] = __dmul_rn(Rp, Rp);
    // cells: every pair within R lies in neighbouring cells when R fits the
    // side (with room for the binary32 cell assignment)
    if (d.nc > 0) *d.cell_ok = __dadd_rn(R, 1e-3) <= L / d.nc ? 1 : 0;
    // binary32 screen constants of both lists: R^2 -/+ margin, linear radius
    float* tf = (float*)(d.thresh + 4);
    const double RR[2] = {R, Rp};
    for (int k = 0; k < 2; ++k) {
      const float m2 = screen_margin(L, RR[k]);
      const float R2f = (float)__dmul_rn(RR[k], RR[k]);
      tf[4 * k + 0] = R2f - m2;
      tf[4 * k + 1] = R2f + m2;
      tf[4 * k + 2] = sqrtf(R2f + m2);
      tf[4 * k + 3] = (RR[k] < 2.0 * L) ? 1.0f : 0.0f;
    }
    tf[8] = (float)L;
  }
}

__global__ void k_list_prep(const __grid_constant__ Dev d) { b_k_list_prep(d, blockIdx.x); }

__global__ void k_list_prep_b(const Dev* __restrict__ devs, const int* __restrict__ pfx, int nm) {
  MX_BATCH_ENTER();
  b_k_list_prep(d, bx);
}

constexpr int NL_EBUF = 32 * 8;  // staged entries per warp of the search (one round's worst case)

// appends a warp's staged entries to row i with one reservation
__device__ __forceinline__ void nlist_flush(const Dev& d, int i, int* row, const int* eb, int nb, int lane) {
  if (nb == 0) return;
  int base = 0;
  if (lane == 0) base = atomicAdd(&d.nl_cnt[i], nb);
  base = __shfl_sync(0xffffffffu, base, 0);
  for (int k = lane; k < nb; k += 32) {
    if (base + k < d.nl_cap)
      row[base + k] = eb[k];
    else
      atomicOr(d.err, ERR_NLIST);
  }
  __syncwarp();
}

// parts of one owner row's candidate search: the 27 neighbouring cells with
// a cell grid, otherwise chunks of 32 * nl_cpl candidates
__host__ __device__ __forceinline__ int nlist_parts(const Dev& d) {
  return d.nc > 0 ? 27 : (d.n_nonp + 32 * d.nl_cpl - 1) / (32 * d.nl_cpl);
}

// One warp per (owner row, part of its candidates): a neighbouring cell of
// the row's atom, or (all pairs, or a step whose radius exceeds the cell
// side) a contiguous range of candidates. Entries are appended with a
// per-row counter, so the row order is arbitrary.
__device__ __forceinline__ void b_k_nlist(const Dev& d, int bx) {
  const int lane = threadIdx.x & 31;
  const int w = (bx * blockDim.x + threadIdx.x) >> 5;
  const int nchunk = nlist_parts(d);
  const int i = w / nchunk;
  const int chunk = w - i * nchunk;
  if (i >= d.n_nonp) return;
  const float4 tf = ((const float4*)(d.thresh + 4))[0];
  if (tf.w == 0.0f) {
    if (lane == 0 && chunk == 0) atomicOr(d.err, ERR_BOX);
    return;
  }
  const double L = d.box;
  const double R2 = d.thresh[10];
  const float R2lo = tf.x, R2hi = tf.y, Rlin = tf.z;
  const float Lf = ((const float*)(d.thresh + 4))[8];
  const float4 ri = d.reff[i];
  const int Pi = __float_as_int(ri.w);
  const int moli = d.pos_mol[i];
  int* row = d.nl + (size_t)i * d.nl_cap;
  // this warp's candidates: cand(k) for k < len
  const bool cells = d.nc > 0 && *d.cell_ok;
  int c0, len;
  const int* cand = nullptr;
  int kxc = 0, kyc = 0, kzc = 0;  // cells: the one image code per axis that can lie within R
  if (cells) {
    const int nc = d.nc;
    const int ci = cell_of(ri, d.cell_inv, nc);
    const int cx = ci / (nc * nc), cy = (ci / nc) % nc, cz = ci % nc;
    const int ux = cx + chunk / 9 - 1, uy = cy + (chunk / 3) % 3 - 1, uz = cz + chunk % 3 - 1;
    // a neighbouring cell across a box face holds its atoms' images one L
    // away; with cells at least R wide no other image is within R
    kxc = 2 + (ux < 0 ? -1 : (ux >= nc ? 1 : 0));
    kyc = 2 + (uy < 0 ? -1 : (uy >= nc ? 1 : 0));
    kzc = 2 + (uz < 0 ? -1 : (uz >= nc ? 1 : 0));
    const int nx = (ux + nc) % nc, ny = (uy + nc) % nc, nz = (uz + nc) % nc;
    const int cell = (nx * nc + ny) * nc + nz;
    c0 = d.cell_start[cell];
    len = d.cell_start[cell + 1] - c0;
    cand = d.cell_atoms + c0;
  } else if (d.nc > 0) {  // cell grid, radius too large this step: 27 ranges of all pairs
    const int per = (d.n_nonp + 26) / 27;
    c0 = chunk * per;
    len = max(0, min(per, d.n_nonp - c0));
  } else {
    c0 = chunk * 32 * d.nl_cpl;
    len = max(0, min(32 * d.nl_cpl, d.n_nonp - c0));
  }
  constexpr int MAXE = 8;  // entries one lane keeps per candidate (images)
  __shared__ int ebuf[NL_THREADS / 32][NL_EBUF];
  int* eb = ebuf[(threadIdx.x >> 5) % (NL_THREADS / 32)];
  int nb = 0;  // entries staged (the same on every lane)
#pragma unroll 1
  for (int t = 0; t < len; t += 32) {
    const int k = t + lane;
    const int c = k < len ? (cand ? cand[k] : c0 + k) : -1;
    int ne = 0;
    int ents[MAXE];
    if (c >= 0 && c != i) {
      const float4 rc4 = d.reff[c];
      const int Pc = __float_as_int(rc4.w);
      bool own;
      if (d.full_list) {
        own = true;
      } else if (Pi != Pc) {
        own = Pi > Pc;
      } else {
        const int lo = i < c ? i : c;
        own = (((i + c) & 1) == 0) ? (i == lo) : (i != lo);
      }
      const float dfx = rc4.x - ri.x, dfy = rc4.y - ri.y, dfz = rc4.z - ri.z;
      const unsigned mx = own ? (cells ? img_bit(dfx, kxc, Lf, Rlin) : img_mask(dfx, Lf, Rlin)) : 0u;
      const unsigned my = mx ? (cells ? img_bit(dfy, kyc, Lf, Rlin) : img_mask(dfy, Lf, Rlin)) : 0u;
      const unsigned mz = my ? (cells ? img_bit(dfz, kzc, Lf, Rlin) : img_mask(dfz, Lf, Rlin)) : 0u;
      if (mz) {
        const bool same = d.pos_mol[c] == moli;
        // the image code of the same-molecule zero image in the wrapped frame
        int xcode = -1;
        if (same) {
          const int4 wc = d.wrapn[c], wi = d.wrapn[i];
          const int ex = wc.x - wi.x, ey = wc.y - wi.y, ez = wc.z - wi.z;
          if (abs(ex) <= 2 && abs(ey) <= 2 && abs(ez) <= 2) xcode = (ex + 2) * 25 + (ey + 2) * 5 + (ez + 2);
        }
        const int tag = (d.ainfo[c].row0 << 11) | (d.ainfo[c].type << 7);
        for (unsigned bx = mx; bx; bx &= bx - 1) {
          const int kx = __ffs(bx) - 1;
          const float ex = dfx + img_of(kx) * Lf;
          for (unsigned by = my; by; by &= by - 1) {
            const int ky = __ffs(by) - 1;
            const float ey = dfy + img_of(ky) * Lf;
            for (unsigned bz = mz; bz; bz &= bz - 1) {
              const int kz = __ffs(bz) - 1;
              if (kx * 25 + ky * 5 + kz == xcode) continue;
              const float ez = dfz + img_of(kz) * Lf;
              const float d2f = ex * ex + ey * ey + ez * ez;
              bool keep;
              if (d2f < R2lo) {
                keep = true;
              } else if (d2f > R2hi) {
                keep = false;
              } else {
                const double4_32a a = d.refd[i], bb = d.refd[c];
                keep = exact_d2(__dsub_rn(bb.x, a.x), __dsub_rn(bb.y, a.y), __dsub_rn(bb.z, a.z), kx - 2, ky - 2,
                                kz - 2, L) < R2;
              }
              if (keep) {
                const int en = tag | (kx * 25 + ky * 5 + kz);
                if (ne < MAXE) {
                  ents[ne++] = en;
                } else {  // many images of one partner (small boxes): append alone
                  const int slot = atomicAdd(&d.nl_cnt[i], 1);
                  if (slot < d.nl_cap)
                    row[slot] = en;
                  else
                    atomicOr(d.err, ERR_NLIST);
                }
              }
            }
          }
        }
      }
    }
    // the round's entries go to the warp's staging buffer at the inclusive
    // prefix of the lane counts (flushed first when they would not fit)
    int incl = ne;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (nb + total > NL_EBUF) {
      nlist_flush(d, i, row, eb, nb, lane);
      nb = 0;
    }
    for (int k = 0; k < ne; ++k) eb[nb + incl - ne + k] = ents[k];
    nb += total;
    __syncwarp();
  }
  nlist_flush(d, i, row, eb, nb, lane);
}

__global__ void __launch_bounds__(NL_THREADS) k_nlist(const __grid_constant__ Dev d) { b_k_nlist(d, blockIdx.x); }

__global__ void __launch_bounds__(NL_THREADS) k_nlist_b(const Dev* __restrict__ devs, const int* __restrict__ pfx, int nm) {
  MX_BATCH_ENTER();
  b_k_nlist(d, bx);
}

// pseudo-particle site list: one thread per (pseudo atom, site position)
__global__ void k_plist(Dev d) {
  const double L = d.box;
  const double R2 = d.thresh[11];
  const int e = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.n_nonp) return;
  const float4 tf = ((const float4*)(d.thresh + 4))[1];
  if (tf.w == 0.0f) {
    atomicOr(d.err, ERR_BOX);
    return;
  }
  const float R2lo = tf.x, R2hi = tf.y, Rlin = tf.z;
  const float Lf = (float)L;
  const int ea = d.pseudo_atom[e];
  const double rex = d.ref[3 * ea], rey = d.ref[3 * ea + 1], rez = d.ref[3 * ea + 2];
  const double4_32a rcd = d.refd[c];
  const double rcx = rcd.x, rcy = rcd.y, rcz = rcd.z;
  const float4 rcf = d.reff[c];
  const float dfx = rcf.x - (float)rex, dfy = rcf.y - (float)rey, dfz = rcf.z - (float)rez;
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
// k_pair64 blocks of 14 warps: its ~72 registers then fit two blocks (28
// warps) per SM, each with one copy of the interval table in shared memory
constexpr int PAIR64_THREADS = 448;

// Unit-charge DSF potential G(s), s = r^2, and -2 dG/ds from the interval
// table: each is a quintic in x = s - s0 on each of 64 geometric
// sub-intervals per octave of s; the interval and s0 come straight from the
// exponent and top mantissa bits of s (integer instructions only).
__device__ __forceinline__ void dsf_table(const double* tab, int hi, double s, double* g, double* fg) {
  const double s0 = __hiloint2double((hi >> 14) << 14, 0);
  const double x = s - s0;
  const double* c = tab;
  double p = fma(c[5], x, c[4]);
  double q = fma(c[11], x, c[10]);
  p = fma(p, x, c[3]);
  q = fma(q, x, c[9]);
  p = fma(p, x, c[2]);
  q = fma(q, x, c[8]);
  p = fma(p, x, c[1]);
  q = fma(q, x, c[7]);
  *g = fma(p, x, c[0]);
  *fg = fma(q, x, c[6]);
}

constexpr size_t PAIR64_SMEM_PER_INTERVAL = 6 * sizeof(double) + 8 * sizeof(float);
constexpr size_t PAIR32_SMEM_PER_INTERVAL = 8 * sizeof(float);

// The same two quintics at a given offset x = s - s0 inside the interval,
// split by order: c0 + c1 x + c2 x^2 in binary64 (c = the interval's
// [c0 c1 c2 q0 q1 q2]) and x^3 (c3 + c4 x + c5 x^2) in binary32 (t = [c3 c4 c5
// - q3 q4 q5 -]). With x below 1.1 % of s the cubic tail is below ~1e-6 of
// the value, so its binary32 rounding stays near 1e-13 relative.
__device__ __forceinline__ void dsf_poly_split(const double* c, const float* t, double x, double* g, double* fg) {
  // binary32 x by truncating the binary64 bit fields (x >= 0)
  const unsigned long long xb = (unsigned long long)__double_as_longlong(x);
  const int fe = (int)((xb >> 52) & 0x7FF) - 1023 + 127;
  const float xf = fe > 0 ? __uint_as_float(((unsigned)fe << 23) | (unsigned)((xb >> 29) & 0x7FFFFFull)) : 0.0f;
  const float x3 = xf * xf * xf;
  const float tg = fmaf(fmaf(t[2], xf, t[1]), xf, t[0]) * x3;
  const float tq = fmaf(fmaf(t[6], xf, t[5]), xf, t[4]) * x3;
  const double p = fma(fma(c[2], x, c[1]), x, c[0]);
  const double q = fma(fma(c[5], x, c[4]), x, c[3]);
  *g = p + f2d_bits(tg);
  *fg = q + f2d_bits(tq);
}

// analytic G and -2 dG/ds (r below the table range)
__device__ __forceinline__ void dsf_direct(const Dev& d, double s, double* g, double* fg) {
  const double r = sqrt(s);
  const double rinv = 1.0 / r;
  const double ec = erfc(d.alpha * r);
  const double ex = exp(-d.alpha * d.alpha * s);
  *g = ec * rinv - d.dsf_erfc_rc_over_rc + d.dsf_cf * (r - d.rc);
  // dG/dr = -erfc/r^2 - g exp/r + cf ; -2 dG/ds = -(dG/dr) / r
  *fg = (ec * rinv * rinv + d.dsf_g * ex * rinv - d.dsf_cf) * rinv;
}

// ---------------------------------------------------------------------------
// nonbonded pair sweep, FP64, slice-parallel over the half list.
//
// The owner of a listed pair is its finer atom (P_i >= P_j), so the terms of
// Eq. (mts-hamiltonian) for one entry are exactly the owner's beads b, each
// meeting the partner's bead b >> (lgP_i - lgP_j) with weight 1/P_i. One warp
// takes (owner atom, block of 32 of its beads, chunk of its list); the lanes
// are the owner's beads (groups of min(P_i, 32) lanes take different
// entries), so an entry is decoded once per group and the partner's beads
// are read from the atom-major copy of the fixed-point positions, contiguous
// for the lanes. Per term the arithmetic is that of the sweep above: exact
// 128-bit r^2 and cut-off, table interval and offset from the integer bits,
// binary64 quadratics with binary32 tails, forces rounded once into the fixed
// point; the partner's bead gets the reaction.
// ---------------------------------------------------------------------------
// Work items of the FP64 sweep for the current list: every owner row gets
// (slice blocks) x (chunks of P64_CH entries per lane group) items, only as
// many chunks as its row holds. One CTA per 1024 rows reserves a contiguous
// range of the item array (the counter was cleared with the list) and writes
// its rows' items in row order.
constexpr int ITEM_THREADS = 1024;

// chunks (per slice block) and slice blocks of owner row i's FP64 items
__device__ __forceinline__ void p64_row_items(const Dev& d, int i, int* nch, int* lgsb) {
  const int cnt = min(d.nl_cnt[i], d.nl_cap);
  const int lgP = d.ainfo[i].log2P;
  const int lgPp = lgP < 5 ? lgP : 5;
  const int per = P64_CH << (5 - lgPp);
  *nch = (cnt + per - 1) / per;
  *lgsb = lgP - lgPp;
}

// exclusive prefix over the rows of the FP64 items per row, built by a
// whole CTA in shared memory (rpfx[0..n_nonp]); returns the item count
__device__ int p64_row_prefix(const Dev& d, int* rpfx, int* wtot) {
  const int nr = d.n_nonp, nt = blockDim.x;
  const int per_t = (nr + nt - 1) / nt;
  const int r0 = min((int)threadIdx.x * per_t, nr), r1 = min(r0 + per_t, nr);
  int run = 0;
  for (int i = r0; i < r1; ++i) {
    int nch, lgsb;
    p64_row_items(d, i, &nch, &lgsb);
    rpfx[i] = nch << lgsb;
    run += nch << lgsb;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = nt >> 5;
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wtot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int v = lane < nw ? wtot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < nw) wtot[lane] = v;
  }
  __syncthreads();
  int start = (wid > 0 ? wtot[wid - 1] : 0) + incl - run;
  for (int i = r0; i < r1; ++i) {
    const int n = rpfx[i];
    rpfx[i] = start;
    start += n;
  }
  const int total = wtot[nw - 1];
  if (threadIdx.x == 0) rpfx[nr] = total;
  __syncthreads();
  return total;
}

__device__ __forceinline__ void b_k_pair_items(const Dev& d, int bx) {
  __shared__ int wsum[ITEM_THREADS / 32];
  __shared__ int base;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int i = bx * ITEM_THREADS + tid;
  int n = 0, nch = 0, lgsb = 0;
  if (i < d.n_nonp) {
    p64_row_items(d, i, &nch, &lgsb);
    n = nch << lgsb;
  }
  int incl = n;  // inclusive scan over the block
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int v = lane < ITEM_THREADS / 32 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane < ITEM_THREADS / 32) wsum[lane] = v;
    if (lane == 31) base = atomicAdd(d.pctr, v);
  }
  __syncthreads();
  const int off = base + (wid > 0 ? wsum[wid - 1] : 0) + incl - n;
  for (int k = 0; k < n; ++k) {
    const int sb = k / nch, ch = k - sb * nch;
    d.pitems[off + k] = make_int2(i, (sb << 16) | ch);
  }
}

__global__ void __launch_bounds__(ITEM_THREADS) k_pair_items(const __grid_constant__ Dev d) { b_k_pair_items(d, blockIdx.x); }

__global__ void __launch_bounds__(ITEM_THREADS) k_pair_items_b(const Dev* __restrict__ devs, const int* __restrict__ pfx, int nm) {
  MX_BATCH_ENTER();
  b_k_pair_items(d, bx);
}

__device__ __forceinline__ void b_k_pair64(const Dev& d, int bx) {
  (void)bx;
  extern __shared__ double dtab[];  // DSF interval table: 6 doubles, then 8 floats per interval
  __shared__ PairPar tab[MT * MT];
  __shared__ int flg[MT * MT];      // bit 0: Coulomb, bit 1: Lennard-Jones
  __shared__ longlong4_32a shi[125];
  __shared__ int tN[MT], tLg[MT], tOff[MT];
  const int nt = d.n_types;
  float* ftab = (float*)(dtab + 6 * d.dsf_nint);
  for (int e = threadIdx.x; e < d.dsf_nint; e += blockDim.x) {
    const double* c = d.dsf_tab + 12 * e;
    for (int k = 0; k < 3; ++k) {
      dtab[6 * e + k] = c[k];
      dtab[6 * e + 3 + k] = c[6 + k];
      ftab[8 * e + k] = (float)c[3 + k];
      ftab[8 * e + 4 + k] = (float)c[9 + k];
    }
    ftab[8 * e + 3] = 0.0f;
    ftab[8 * e + 7] = 0.0f;
  }
  for (int e = threadIdx.x; e < nt; e += blockDim.x) {
    tN[e] = d.N[e];
    tLg[e] = d.log2P[e];
    tOff[e] = d.off[e];
  }
  for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
    const PairPar pp = d.pairpar[(e / nt) * MT + (e % nt)];
    tab[e] = pp;
    flg[e] = (pp.qq != 0.0 ? 1 : 0) | (pp.e4 != 0.0 ? 2 : 0);
  }
  for (int e = threadIdx.x; e < 125; e += blockDim.x) {
    const int nx = e / 25 - 2, ny = (e / 5) % 5 - 2, nz = e % 5 - 2;
    shi[e] = make_longlong4_32a(nx * d.box_fix, ny * d.box_fix, nz * d.box_fix, 0);
  }
  // the items: from the item array, or (p64_implicit) from a row prefix this
  // CTA builds after the table in shared memory
  int* rpfx = (int*)(ftab + 8 * d.dsf_nint);
  __shared__ int wtot[32];
  __syncthreads();
  const int n_items = d.p64_implicit ? p64_row_prefix(d, rpfx, wtot) : d.pctr[0];
  const int lane = threadIdx.x & 31;
  const double rc = d.rc;
  // r_cut^2 in the 2^-96 A^2 units of the integer squared distances (exact)
  fm::u128 rc2q;
  {
    const unsigned long long bb = fm::dbl_bits(d.rc2);
    const unsigned long long m = (bb & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const int sh = (int)((bb >> 52) & 0x7FF) - 1075 + 96;
    if (sh >= 64)
      rc2q = fm::u128{m << (sh - 64), 0ull};
    else if (sh > 0)
      rc2q = fm::u128{m >> (64 - sh), m << sh};
    else
      rc2q = fm::u128{0ull, sh > -53 ? m >> (-sh) : 0ull};
  }
  const int base = d.dsf_base;
  // items are handed out one per warp from a counter (the fixed-point sums
  // make the result independent of which warp takes which item)
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(d.pctr + 1, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= n_items) break;
    int pos, sb, ch;
    if (d.p64_implicit) {  // the row holding item w: rpfx[pos] <= w < rpfx[pos + 1]
      int lo = 0, hi = d.n_nonp;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (rpfx[mid] <= w)
          lo = mid;
        else
          hi = mid;
      }
      pos = lo;
      int nch, lgsb;
      p64_row_items(d, pos, &nch, &lgsb);
      const int k = w - rpfx[pos];
      sb = k / nch;
      ch = k - sb * nch;
    } else {
      const int2 it = d.pitems[w];
      pos = it.x;
      sb = it.y >> 16;
      ch = it.y & 0xFFFF;
    }
    const AtomInfo ai = d.ainfo[pos];
    const int lgPi = ai.log2P;
    const int lgPp = lgPi < 5 ? lgPi : 5;  // log2 of the lanes per group
    const int lgG = 5 - lgPp;
    const int cnt = min(d.nl_cnt[pos], d.nl_cap);
    const int e0 = ch * (P64_CH << lgG);
    const int e1 = min(cnt, e0 + (P64_CH << lgG));
    const int sl = lane & ((1 << lgPp) - 1), grp = lane >> lgPp;
    const int b = (sb << lgPp) + sl;  // owner bead of this lane
    const int oi = tOff[ai.type];
    const longlong4_32a xi = d.XiA[oi + ((ai.row0 - oi) << lgPi) + b];
    const int row_i = ai.row0 + b * ai.stride;
    const int wsh = lgPi;  // weight 1/P_i = 2^-wsh
    const int trow = ai.type * nt;
    const int* lst = d.nl + (size_t)pos * d.nl_cap;
    long long fix = 0, fiy = 0, fiz = 0;
    double elj = 0.0, ec = 0.0, vir = 0.0;
    int nev = 0, nlj = 0, bad = 0;
    // every lane runs the same number of rounds (the reaction sums below
    // are warp-collective); a group past the end of the chunk idles
    for (int eb = e0; eb < e1; eb += (1 << lgG)) {
      const int e = eb + grp;
      const bool valid = e < e1;
      const int ent = lst[valid ? e : e0];
      const int tj = (ent >> 7) & 15;
      const int lgPj = tLg[tj];
      const int row0j = ent >> 11, oj = tOff[tj];
      const int bj = b >> (lgPi - lgPj);
      const longlong4_32a xj = d.XiA[oj + ((row0j - oj) << lgPj) + bj];
      const longlong4_32a sv = shi[ent & 127];
      const long long ix = (xj.x - xi.x) + sv.x, iy = (xj.y - xi.y) + sv.y, iz = (xj.z - xi.z) + sv.z;
      const fm::u128 q2 = fm::norm2(ix, iy, iz);
      long long kx = 0, ky = 0, kz = 0;
      if (valid && fm::lt128(q2, rc2q)) {
        const int pq = fm::msb128(q2);
        const double r2 = pq >= 0 ? fm::u128_to_dbl(q2, pq, 96) : 0.0;
        const int fl = flg[trow + tj];
        const PairPar pp = tab[trow + tj];
        double fr = 0.0;
        if (fl & 1) {
          // interval and offset from the binary64 r^2 (exponent and top six
          // mantissa bits; the offset from the interval start is exact)
          double g, fg, x;
          const int key = fm::dsf_key(r2, &x);
          if (key >= base)
            dsf_poly_split(dtab + 6 * (key - base), ftab + 8 * (key - base), x, &g, &fg);
          else
            dsf_direct(d, r2, &g, &fg);
          ec = fma(pp.qq, g, ec);
          fr = pp.qq * fg;
        }
        if (fl & 2) {
          const double rinv = rsqrt(r2);
          const double r = r2 * rinv;
          const double rinv2 = rinv * rinv;
          const double sr2 = pp.s2 * rinv2;
          const double sr6 = sr2 * sr2 * sr2;
          const double sr12 = sr6 * sr6;
          elj += pp.e4 * (sr12 - sr6) - pp.vrc - (r - rc) * pp.dvrc;
          fr += (6.0 * pp.e4 * (2.0 * sr12 - sr6) * rinv + pp.dvrc) * rinv;
          ++nlj;
        }
        kx = fm::mulfix(fr, ix, 4 + wsh, &bad);
        ky = fm::mulfix(fr, iy, 4 + wsh, &bad);
        kz = fm::mulfix(fr, iz, 4 + wsh, &bad);
        fix -= kx;
        fiy -= ky;
        fiz -= kz;
        vir = fma(fr, r2, vir);
        ++nev;
      }
      // A coarser partner's bead is shared by 2^lgR consecutive lanes of the
      // group: sum their reactions exactly in registers first, so one lane
      // issues the atomics instead of 2^lgR lanes on the same address.
      const int lgR = min(lgPi - lgPj, lgPp);
      const int lgRmax = __reduce_max_sync(0xffffffffu, (unsigned)lgR);
      for (int o = 0; o < lgRmax; ++o) {
        const long long vx = __shfl_xor_sync(0xffffffffu, kx, 1 << o);
        const long long vy = __shfl_xor_sync(0xffffffffu, ky, 1 << o);
        const long long vz = __shfl_xor_sync(0xffffffffu, kz, 1 << o);
        if (o < lgR) {
          kx += vx;
          ky += vy;
          kz += vz;
        }
      }
      if ((sl & ((1 << lgR) - 1)) == 0 && (kx | ky | kz) != 0) {
        unsigned long long* fj = d.F_fix + 3 * (size_t)(row0j + bj * tN[tj]);
        atomicAdd(fj + 0, (unsigned long long)kx);
        atomicAdd(fj + 1, (unsigned long long)ky);
        atomicAdd(fj + 2, (unsigned long long)kz);
      }
    }
    // the owner's force: lanes of the same bead (one per group) summed exactly
    for (int o = 1 << lgPp; o < 32; o <<= 1) {
      fix += __shfl_xor_sync(0xffffffffu, fix, o);
      fiy += __shfl_xor_sync(0xffffffffu, fiy, o);
      fiz += __shfl_xor_sync(0xffffffffu, fiz, o);
    }
    if (grp == 0 && (fix | fiy | fiz) != 0) {
      unsigned long long* fi = d.F_fix + 3 * (size_t)row_i;
      atomicAdd(fi + 0, (unsigned long long)fix);
      atomicAdd(fi + 1, (unsigned long long)fiy);
      atomicAdd(fi + 2, (unsigned long long)fiz);
    }
    // energies carry the weight 1/P_i as an exponent offset of the fixed point
    long long kl = fixs(elj, 40 - wsh, &bad), kc = fixs(ec, 40 - wsh, &bad), kv = fixs(vir, 40 - wsh, &bad);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kl += __shfl_xor_sync(0xffffffffu, kl, o);
      kc += __shfl_xor_sync(0xffffffffu, kc, o);
      kv += __shfl_xor_sync(0xffffffffu, kv, o);
    }
    nev = warp_sumi(nev);
    nlj = warp_sumi(nlj);
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      if (kl) atomicAdd(d.E_fix + E_LJ, (unsigned long long)kl);
      if (kc) atomicAdd(d.E_fix + E_COUL, (unsigned long long)kc);
      if (kv) atomicAdd(d.E_fix + E_VIRIAL, (unsigned long long)kv);
      if (nev) atomicAdd(d.E_fix + E_NEVAL, (unsigned long long)nev);
      if (nlj) atomicAdd(d.E_fix + E_NLJEVAL, (unsigned long long)nlj);
      if (bad) atomicOr(d.err, ERR_NONFINITE);
    }
  }
}

__global__ void __launch_bounds__(PAIR64_THREADS) k_pair64(const __grid_constant__ Dev d) { b_k_pair64(d, blockIdx.x); }

__global__ void __launch_bounds__(PAIR64_THREADS) k_pair64_b(const Dev* __restrict__ devs, const int* __restrict__ pfx, int nm) {
  MX_BATCH_ENTER();
  b_k_pair64(d, bx);
}

// ---------------------------------------------------------------------------
// nonbonded pair sweep, FP32 forces (precision MIXTS_FP32_FORCES).
//
// Full neighbour lists (every row lists all partners): only the owner's beads
// are written, so there are no per-term reaction atomics; every term is
// evaluated from both of its atoms and energies and counts carry a factor 1/2.
//
// Before the sweep, k_list_seg32 regroups each row by partner type (a
// counting sort, one warp per row), folds the pair's bead-0 displacement
// (r_j0 + n L) - r_i0 into each entry once, in binary32 from the exact
// 2^-12 A grid parts plus their remainders, and writes the row's work items.
// An item is then (owner atom i,
// partner type t, block of 32 owner beads, chunk of entries) with one fine
// grid P* = max(P_i, P_t), one weight 1/P* and one parameter set: lanes are
// the owner's beads (groups of min(P_i, 32) lanes take different entries) and
// each lane walks the P* / P_i fine slices of its bead, s = b (P*/P_i) + k,
// meeting partner bead s >> log2(P* / P_t). The displacement of a term is
// the entry's bead-0 displacement plus the two beads' binary32 offsets from
// their bead 0, so no large cancellation enters. Items hold ~2^11 terms
// whatever the bead counts and are handed out from a counter.
//
// The damped-shifted-force (or Ewald real-space) Coulomb comes from a
// binary32 interval table of cubics in s = r^2 (the FP64 sweep's table, refit
// as cubics); Lennard-Jones is analytic.
// ---------------------------------------------------------------------------
constexpr int LG_P32_ENTRIES = 7;  // at most 128 entries per item (staged in shared memory)

// log2 of the entries of one FP32 item: 2^lgt terms = entries x
// (owner beads of the block) x (fine slices per owner bead)
// (capped so that the entries plus the staging padding of 4 x 2^(5 - lgPp)
// groups fit P32_STAGE: 128 entries for owners of 4 or more beads, 64 for
// two-bead owners, 32 for classical ones)
__device__ __forceinline__ int p32_lg_entries(int lgPi, int lgPt, int lgt) {
  const int lgPp = lgPi < 5 ? lgPi : 5;
  const int lgS = lgPi > lgPt ? lgPi : lgPt;
  const int lgE = lgt - lgPp - (lgS - lgPi);
  const int cap = lgPp >= 2 ? LG_P32_ENTRIES : LG_P32_ENTRIES - 2 + lgPp;
  return lgE > 0 ? (lgE < cap ? lgE : cap) : 0;
}

// log2 of the entries of one window item (k_pair32w): 2^(lgt - 1) terms =
// entries x pair-grid slices per window (2^lgk, lanes per entry), at most 2^8
// entries (the item's count field); the sweep stages them P32W_BUF at a time.
// Half the gather sweep's item: pair phase 0.0785 -> 0.0769 ms at 512 waters,
// 0.045 -> 0.041 ms at 256 waters + ion (2^(lgt - 2): 0.079 and 0.038 ms)
__device__ __forceinline__ int p32w_lg_entries(int lgS, int lgnw, int lgt) {
  const int lgk = lgS > lgnw ? lgS - lgnw : 0;
  const int lgE = lgt - 1 - lgk;
  return lgE > 0 ? (lgE < 8 ? lgE : 8) : 0;
}

constexpr int SEG32_AHEAD = 4;  // rounds of 32 list entries loaded together by k_list_seg32

__device__ __forceinline__ void b_k_list_seg32(const Dev& d, int bx) {
  const int lane = threadIdx.x & 31;
  const int i = (bx * blockDim.x + threadIdx.x) >> 5;
  if (i >= d.n_nonp) return;
  const int nt = d.n_types;
  const int cnt = min(d.nl_cnt[i], d.nl_cap);
  const int* row = d.nl + (size_t)i * d.nl_cap;
  // lane u counts the entries whose partner is of type u (n_types <= 16);
  // SEG32_AHEAD rounds of 32 entries are loaded before they are used
  int c_mine = 0;
  for (int e0 = 0; e0 < cnt; e0 += 32 * SEG32_AHEAD) {
    int tq[SEG32_AHEAD];
#pragma unroll
    for (int q = 0; q < SEG32_AHEAD; ++q) {
      const int e = e0 + 32 * q + lane;
      tq[q] = e < cnt ? (row[e] >> 7) & 15 : -1;
    }
#pragma unroll
    for (int q = 0; q < SEG32_AHEAD; ++q)
      for (int u = 0; u < nt; ++u) {
        const unsigned m = __ballot_sync(0xffffffffu, tq[q] == u);
        if (lane == u) c_mine += __popc(m);
      }
  }
  int incl = c_mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  int next = incl - c_mine;  // lane u: next slot of type u
  if (lane <= nt) d.nlseg[(size_t)i * (nt + 1) + lane] = lane < nt ? next : cnt;
  // this row's work items, (partner type, slice block, chunk) of ~2^p32_lgt
  // terms each, in a range of the item array reserved with one atomic
  {
    const int lgP = d.ainfo[i].log2P;
    int lgsb, lgE;
    if (d.p32w) {  // window sweep: slice blocks are the windows, one item array for all
      lgsb = 0;
      lgE = lane < nt ? p32w_lg_entries(lgP > d.log2P[lane] ? lgP : d.log2P[lane], d.p32w_lgnw, d.p32_lgt) : 0;
    } else {
      lgsb = lgP > 5 ? lgP - 5 : 0;
      lgE = lane < nt ? p32_lg_entries(lgP, d.log2P[lane], d.p32_lgt) : 0;
    }
    const int nch = lane < nt ? (c_mine + (1 << lgE) - 1) >> lgE : 0;
    const int n = nch << lgsb;
    int ni = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, ni, o);
      if (lane >= o) ni += v;
    }
    const int total = __shfl_sync(0xffffffffu, ni, 31);
    int base = 0;
    if (lane == 0 && total > 0) base = atomicAdd(d.pctr, total);
    base = __shfl_sync(0xffffffffu, base, 0) + ni - n;
    if (d.p32w) {  // window items carry their entries: type << 27 | (count - 1) << 19 | first entry
      for (int k = 0; k < n; ++k) {
        const int e0 = next + (k << lgE), m = min(1 << lgE, c_mine - (k << lgE));
        d.pitems[base + k] = make_int2(i, (lane << 27) | ((m - 1) << 19) | e0);
      }
    } else {
      for (int k = 0; k < n; ++k) {
        const int sb = k / nch, ch = k - sb * nch;
        d.pitems[base + k] = make_int2(i, (lane << 27) | (sb << 20) | ch);
      }
    }
  }
  const int r0i = d.ainfo[i].row0;
  const float4 hi = d.Xf[r0i], lo = d.Xl[r0i];
  const float bh = d.box_hi, bl = d.box_lo;
  float4* out = d.nlB + (size_t)i * d.nl_cap;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int e00 = 0; e00 < cnt; e00 += 32 * SEG32_AHEAD) {
    // the rounds' entries and their partners' bead-0 positions, all loads in
    // flight before the first is used
    int entq[SEG32_AHEAD];
    float4 hq[SEG32_AHEAD], lq[SEG32_AHEAD];
#pragma unroll
    for (int q = 0; q < SEG32_AHEAD; ++q) {
      const int e = e00 + 32 * q + lane;
      entq[q] = e < cnt ? row[e] : -1;
    }
#pragma unroll
    for (int q = 0; q < SEG32_AHEAD; ++q) {
      const int row0j = entq[q] >= 0 ? entq[q] >> 11 : r0i;
      hq[q] = d.Xf[row0j];
      lq[q] = d.Xl[row0j];
    }
#pragma unroll
    for (int q = 0; q < SEG32_AHEAD; ++q) {
      const int ent = entq[q];
      const int t = ent >= 0 ? (ent >> 7) & 15 : -1;
      int dest = 0;
      for (int u = 0; u < nt; ++u) {
        const unsigned m = __ballot_sync(0xffffffffu, t == u);
        const int bse = __shfl_sync(0xffffffffu, next, u);
        if (t == u) dest = bse + __popc(m & lt_mask);
        if (lane == u) next += __popc(m);
      }
      if (ent >= 0) {
        const int row0j = ent >> 11, code = ent & 127;
        const float nx = (float)(code / 25 - 2), ny = (float)((code / 5) % 5 - 2), nz = (float)(code % 5 - 2);
        const float4 hj = hq[q], lj = lq[q];
        const float bx = ((hj.x - hi.x) + nx * bh) + ((lj.x - lo.x) + nx * bl);
        const float by = ((hj.y - hi.y) + ny * bh) + ((lj.y - lo.y) + ny * bl);
        const float bz = ((hj.z - hi.z) + nz * bh) + ((lj.z - lo.z) + nz * bl);
        if (d.p32w) {  // j's first bead in a window stage
          const int sbase = d.p32w_soff[t] + ((row0j - d.off[t]) << d.p32w_lgwt[t]);
          out[dest] = make_float4(bx, by, bz, __int_as_float(sbase));
        } else {  // atom-major bead 0 of j, and j's type
          const int abase = d.off[t] + ((row0j - d.off[t]) << d.log2P[t]);
          out[dest] = make_float4(bx, by, bz, __int_as_float((abase << 4) | t));
        }
      }
    }
  }
}

__global__ void __launch_bounds__(NL_THREADS) k_list_seg32(const __grid_constant__ Dev d) { b_k_list_seg32(d, blockIdx.x); }

__global__ void __launch_bounds__(NL_THREADS) k_list_seg32_b(const Dev* __restrict__ devs, const int* __restrict__ pfx, int nm) {
  MX_BATCH_ENTER();
  b_k_list_seg32(d, bx);
}

// Parameters of one FP32 item (one owner type x partner type pair).
struct P32Par {
  float rc, rc2, smin, qq, e4, s2, vrc, dvrc;
  int kbase;  // key of the table's first interval: (127 + e_lo) << 6
};

// One term of an item, displacement d = x_j - x_i. The Coulomb part per unit
// charge product comes from the binary32 interval table: its value G and its
// force over r F are cubics in x = s - s0 on 64 sub-intervals per octave of
// s = r^2, keyed by the exponent and top six mantissa bits of s. LJ items
// add Lennard-Jones analytically and carry the total force; otherwise the
// force stays per unit charge product (the item scales it once). Skipped as
// a whole when no lane of the warp is inside the cut-off; otherwise
// branch-free and masked at r_cut. nev counts the warp's in-cut-off terms
// (the same on every lane). WSKIP = false (lanes on different entries, so a
// warp is rarely all outside): no skip, and nev counts the lane's own terms.
template <bool LJ, bool WSKIP = true>
__device__ __forceinline__ void pair32_term(const P32Par& c, const float4* tab, float dx, float dy, float dz,
                                            float& fx, float& fy, float& fz, float& ec, float& elj, float& vir,
                                            int& nev) {
  const float s = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  const bool in = s < c.rc2;
  if (WSKIP) {
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (m == 0u) return;
    nev += __popc(m);
  } else {
    nev += in ? 1 : 0;
  }
  const float sc = fminf(fmaxf(s, c.smin), c.rc2);
  const int bits = __float_as_int(sc);
  const int key = (bits >> 17) - c.kbase;
  const float x = sc - __int_as_float(bits & 0xFFFE0000);
  const float4 gq = tab[2 * key], fq = tab[2 * key + 1];
  float g = fmaf(fmaf(fmaf(gq.w, x, gq.z), x, gq.y), x, gq.x);
  float f = fmaf(fmaf(fmaf(fq.w, x, fq.z), x, fq.y), x, fq.x);
  if (LJ) {
    const float rinv = rsqrtf(sc);
    const float r = sc * rinv, rinv2 = rinv * rinv;
    const float sr2 = c.s2 * rinv2, sr6 = sr2 * sr2 * sr2, sr12 = sr6 * sr6;
    const float lt = c.e4 * (sr12 - sr6) - c.vrc - (r - c.rc) * c.dvrc;
    f = fmaf(c.qq, f, (6.0f * c.e4 * (2.0f * sr12 - sr6) * rinv + c.dvrc) * rinv);
    elj += in ? lt : 0.0f;
  }
  g = in ? g : 0.0f;
  f = in ? f : 0.0f;
  ec += g;
  // force on i is minus the force on j along d = x_j - x_i
  fx = fmaf(-f, dx, fx);
  fy = fmaf(-f, dy, fy);
  fz = fmaf(-f, dz, fz);
  vir = fmaf(f, s, vir);
}

// The terms of one lane over its group's entries: local indices grp, grp +
// G, ... below n of the item's entries staged in shared memory (buf, padded
// past n with far entries, so that every group runs the same rounds without
// bounds tests). R1: one fine slice per owner bead (partner not finer), two
// entries per round with the next round's two partner beads loaded ahead.
// Otherwise each entry's 2^lgr slices of the lane's bead.
template <bool LJ, bool R1>
__device__ __forceinline__ void pair32_entries(const float4* buf, int n, int grp, int G, int lgr, int sh_t,
                                               const float4* __restrict__ Xd, int b, float4 di, const P32Par& c,
                                               const float4* tab, float& fx, float& fy, float& fz, float& ec,
                                               float& elj, float& vir, int& nev) {
  const int s0 = b << lgr;  // first fine slice of this lane's owner bead
  const int rounds = (n + G - 1) / G;
  if (R1) {
    const int sj = s0 >> sh_t;
    const int G2 = 2 * G;
    int l = grp;
    float4 Ba = buf[l], Bb = buf[l + G];
    float4 da = __ldg(Xd + (__float_as_int(Ba.w) >> 4) + sj);
    float4 db = __ldg(Xd + (__float_as_int(Bb.w) >> 4) + sj);
    for (int r = 0; r < rounds; r += 2) {
      const int ln = l + G2;
      const float4 Bna = buf[ln], Bnb = buf[ln + G];
      const float4 dna = __ldg(Xd + (__float_as_int(Bna.w) >> 4) + sj);
      const float4 dnb = __ldg(Xd + (__float_as_int(Bnb.w) >> 4) + sj);
      pair32_term<LJ>(c, tab, (Ba.x - di.x) + da.x, (Ba.y - di.y) + da.y, (Ba.z - di.z) + da.z, fx, fy, fz, ec,
                      elj, vir, nev);
      pair32_term<LJ>(c, tab, (Bb.x - di.x) + db.x, (Bb.y - di.y) + db.y, (Bb.z - di.z) + db.z, fx, fy, fz, ec,
                      elj, vir, nev);
      Ba = Bna;
      Bb = Bnb;
      da = dna;
      db = dnb;
      l = ln;
    }
  } else {
    for (int r = 0, l = grp; r < rounds; ++r, l += G) {
      const float4 B = buf[l];
      const int abase = __float_as_int(B.w) >> 4;
      const float bx = B.x - di.x, by = B.y - di.y, bz = B.z - di.z;
#pragma unroll 4
      for (int k = 0; k < (1 << lgr); ++k) {
        const float4 dj = __ldg(Xd + abase + ((s0 + k) >> sh_t));
        pair32_term<LJ>(c, tab, bx + dj.x, by + dj.y, bz + dj.z, fx, fy, fz, ec, elj, vir, nev);
      }
    }
  }
}

// per-warp staging capacity: an item's entries plus the padding that the
// two-ahead loads of the R1 walk reach (< 4 G for G groups); p32_lg_entries
// keeps entries + 4 G within it
constexpr int P32_STAGE = (1 << LG_P32_ENTRIES) + 32;

__device__ __forceinline__ void b_k_pair32(const Dev& d, int bx) {
  (void)bx;
  extern __shared__ float4 tab32[];  // the binary32 DSF table, 2 float4 per interval
  __shared__ float qqt[MT * MT], e4t[MT * MT], s2t[MT * MT], vrct[MT * MT], dvrct[MT * MT];
  __shared__ float4 stage[PAIR_THREADS / 32][P32_STAGE];  // each warp's current item entries
  __shared__ int tLg[MT], tOff[MT];
  const int nt = d.n_types;
  for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
    const PairPar pp = d.pairpar[(e / nt) * MT + (e % nt)];
    qqt[e] = (float)pp.qq;
    e4t[e] = (float)pp.e4;
    s2t[e] = (float)pp.s2;
    vrct[e] = (float)pp.vrc;
    dvrct[e] = (float)pp.dvrc;
  }
  for (int e = threadIdx.x; e < nt; e += blockDim.x) {
    tLg[e] = d.log2P[e];
    tOff[e] = d.off[e];
  }
  for (int e = threadIdx.x; e < 2 * d.dsf_nint; e += blockDim.x) tab32[e] = d.dsf32[e];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int n_items = d.pctr[0];
  const float rc = (float)d.rc, rc2 = (float)d.rc2, smin = (float)d.dsf_smin;
  const int kbase = d.dsf_base - ((1023 - 127) << 6);
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(d.pctr + 1, 1);
    w = __shfl_sync(0xffffffffu, w, 0);
    if (w >= n_items) break;
    const int2 it = d.pitems[w];
    const int i = it.x, t = it.y >> 27, sb = (it.y >> 20) & 127, ch = it.y & 0xFFFFF;
    const AtomInfo ai = d.ainfo[i];
    const int lgPi = ai.log2P, lgPt = tLg[t];
    const int lgPp = lgPi < 5 ? lgPi : 5;  // log2 of the lanes per group
    const int lgG = 5 - lgPp;
    const int lgS = lgPi > lgPt ? lgPi : lgPt;
    const int lgr = lgS - lgPi;  // fine slices per owner bead
    const int sl = lane & ((1 << lgPp) - 1), grp = lane >> lgPp;
    const int b = (sb << lgPp) + sl;  // owner bead of this lane
    const int* seg = d.nlseg + (size_t)i * (nt + 1);
    const int E = 1 << p32_lg_entries(lgPi, lgPt, d.p32_lgt);
    const int e0 = seg[t] + ch * E, e1 = min(seg[t + 1], e0 + E);
    const int oi = tOff[ai.type];
    const float4 di = d.Xd[oi + ((ai.row0 - oi) << lgPi) + b];
    const int k = ai.type * nt + t;
    P32Par c;
    c.rc = rc;
    c.rc2 = rc2;
    c.smin = smin;
    c.kbase = kbase;
    c.qq = qqt[k];
    c.e4 = e4t[k];
    c.s2 = s2t[k];
    c.vrc = vrct[k];
    c.dvrc = dvrct[k];
    const float wgt = __int_as_float((127 - lgS) << 23);  // 1/P*
    float fx = 0.f, fy = 0.f, fz = 0.f, ec = 0.f, elj = 0.f, vir = 0.f;
    int nev = 0;
    const int sh_t = lgS - lgPt;
    const int G = 1 << lgG;
    // stage the item's entries (<= 2^LG_P32_ENTRIES, one coalesced copy),
    // padded with far entries of partner type t whose bead offsets are read
    // from atom-major row 0 (a valid address), then walk them
    float4* buf = stage[threadIdx.x >> 5];
    const float4* lst = d.nlB + (size_t)i * d.nl_cap + e0;
    const int n = e1 - e0;
    const float4 far = make_float4(0.f, 0.f, 1e4f, __int_as_float(t));
    for (int x = lane; x < n + 4 * G; x += 32) buf[x] = x < n ? __ldg(lst + x) : far;
    __syncwarp();
    if (c.e4 != 0.f) {
      if (lgr == 0)
        pair32_entries<true, true>(buf, n, grp, G, 0, sh_t, d.Xd, b, di, c, tab32, fx, fy, fz, ec, elj, vir, nev);
      else
        pair32_entries<true, false>(buf, n, grp, G, lgr, sh_t, d.Xd, b, di, c, tab32, fx, fy, fz, ec, elj, vir, nev);
    } else {
      if (lgr == 0)
        pair32_entries<false, true>(buf, n, grp, G, 0, sh_t, d.Xd, b, di, c, tab32, fx, fy, fz, ec, elj, vir, nev);
      else
        pair32_entries<false, false>(buf, n, grp, G, lgr, sh_t, d.Xd, b, di, c, tab32, fx, fy, fz, ec, elj, vir,
                                     nev);
    }
    __syncwarp();  // the buffer is refilled by the next item
    // LJ items carry the total force; the others the force per unit charge
    // product. Lane partials (times 1/P*) to fixed point by bit assembly,
    // then exact integer sums over the groups, which hold the same owner beads
    const float fs = (c.e4 != 0.f ? 1.0f : c.qq) * wgt;
    int bad = 0;
    long long kx = fm::fixf(fx * fs, 44, &bad), ky = fm::fixf(fy * fs, 44, &bad),
              kz = fm::fixf(fz * fs, 44, &bad);
    for (int o = 1 << lgPp; o < 32; o <<= 1) {
      kx += __shfl_xor_sync(0xffffffffu, kx, o);
      ky += __shfl_xor_sync(0xffffffffu, ky, o);
      kz += __shfl_xor_sync(0xffffffffu, kz, o);
    }
    if (grp == 0 && (kx | ky | kz) != 0) {
      unsigned long long* fi = d.F_fix + 3 * (size_t)(ai.row0 + b * ai.stride);
      atomicAdd(fi + 0, (unsigned long long)kx);
      atomicAdd(fi + 1, (unsigned long long)ky);
      atomicAdd(fi + 2, (unsigned long long)kz);
    }
    // every term is seen from both of its atoms: energies carry a factor 1/2
    long long kl = fm::fixf(elj * wgt, 39, &bad), kc = fm::fixf(ec * (c.qq * wgt), 39, &bad),
              kv = fm::fixf(vir * fs, 39, &bad);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      kl += __shfl_xor_sync(0xffffffffu, kl, o);
      kc += __shfl_xor_sync(0xffffffffu, kc, o);
      kv += __shfl_xor_sync(0xffffffffu, kv, o);
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
      if (kl) atomicAdd(d.E_fix + E_LJ, (unsigned long long)kl);
      if (kc) atomicAdd(d.E_fix + E_COUL, (unsigned long long)kc);
      if (kv) atomicAdd(d.E_fix + E_VIRIAL, (unsigned long long)kv);
      if (nev) {
        atomicAdd(d.E_fix + E_NEVAL, (unsigned long long)nev);
        if (c.e4 != 0.f) atomicAdd(d.E_fix + E_NLJEVAL, (unsigned long long)nev);
      }
      if (bad) atomicOr(d.err, ERR_NONFINITE);
    }
  }
}

__global__ void __launch_bounds__(PAIR_THREADS) k_pair32(const __grid_constant__ Dev d) { b_k_pair32(d, blockIdx.x); }

__global__ void __launch_bounds__(PAIR_THREADS) k_pair32_b(const Dev* __restrict__ devs, const int* __restrict__ pfx, int nm) {
  MX_BATCH_ENTER();
  b_k_pair32(d, bx);
}

// ---------------------------------------------------------------------------
// FP32 pair sweep over imaginary-time windows (the same terms as k_pair32).
//
// A term of the mixTS sum couples bead s >> (log2 P* - log2 P_i) of i with
// bead s >> (log2 P* - log2 P_j) of j on one slice s of their common grid P*
// (Eq. (mts-hamiltonian), the coarse-to-fine map): the beads of one stretch
// of imaginary time interact only with each other. The finest non-pseudo
// bead grid is cut into 2^lgnw windows; every CTA owns one window and copies
// the binary32 bead offsets of all atoms inside it into shared memory once
// (for 512 waters at H32/O4 and four windows: 8 H beads and one O bead per
// atom, 136 KB), so the partner beads of every term come from shared memory
// instead of scattered L2 reads. The CTAs of a window take (owner, partner
// type, entry range) items from that window's counter; lanes are (pair-grid
// slice in the window) x (list entry), 2^lgk x 32 / 2^lgk. Each lane's
// owner-bead partial goes to fixed point, lanes sharing an owner bead are
// summed exactly, and one atomic per bead and component lands in F_fix.
// ---------------------------------------------------------------------------
template <bool LJ>
__device__ __forceinline__ void pair32w_walk(const float4* buf, int nbuf, int grp, int G, const float4* stg, int pj,
                                             float4 di, const P32Par& c, const float4* tab, float& fx, float& fy,
                                             float& fz, float& ec, float& elj, float& vir, int& nev) {
  for (int l = grp; l < nbuf; l += 2 * G) {
    const float4 Ba = buf[l], Bb = buf[l + G];
    const float4 da = stg[__float_as_int(Ba.w) + pj];
    const float4 db = stg[__float_as_int(Bb.w) + pj];
    pair32_term<LJ, false>(c, tab, (Ba.x - di.x) + da.x, (Ba.y - di.y) + da.y, (Ba.z - di.z) + da.z, fx, fy, fz, ec,
                           elj, vir, nev);
    pair32_term<LJ, false>(c, tab, (Bb.x - di.x) + db.x, (Bb.y - di.y) + db.y, (Bb.z - di.z) + db.z, fx, fy, fz, ec,
                           elj, vir, nev);
  }
}

__device__ __forceinline__ void b_k_pair32w(const Dev& d, int bx) {
  extern __shared__ float4 sm32w[];
  __shared__ float qqt[MT * MT], e4t[MT * MT], s2t[MT * MT], vrct[MT * MT], dvrct[MT * MT];
  __shared__ int tLg[MT], tOff[MT], tSoff[MT], tLgw[MT], tB0[MT];
  __shared__ unsigned long long eacc[5];  // the CTA's LJ, Coulomb, virial, term and LJ-term sums
  __shared__ int ebad;
  const int nt = d.n_types;
  const int lgnw = d.p32w_lgnw;
  const int g = bx & ((1 << lgnw) - 1);  // this CTA's window
  float4* tab = sm32w;                   // the binary32 DSF table, 2 float4 per interval
  float4* stg = tab + 2 * d.dsf_nint;    // the window's bead offsets, type blocks atom-major
  float4* ebuf = stg + d.p32w_nstage;    // per-warp staged entries
  for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
    const PairPar pp = d.pairpar[(e / nt) * MT + (e % nt)];
    qqt[e] = (float)pp.qq;
    e4t[e] = (float)pp.e4;
    s2t[e] = (float)pp.s2;
    vrct[e] = (float)pp.vrc;
    dvrct[e] = (float)pp.dvrc;
  }
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const int lg = d.log2P[t];
    tLg[t] = lg;
    tOff[t] = d.off[t];
    tSoff[t] = d.p32w_soff[t];
    tLgw[t] = d.p32w_lgwt[t];
    tB0[t] = lg >= lgnw ? g << (lg - lgnw) : g >> (lgnw - lg);  // first bead of type t in the window
  }
  if (threadIdx.x < 5) eacc[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) ebad = 0;
  for (int e = threadIdx.x; e < 2 * d.dsf_nint; e += blockDim.x) tab[e] = d.dsf32[e];
  for (int t = 0; t < nt; ++t) {
    if (d.pseudo[t]) continue;
    const int lg = d.log2P[t], lgw = d.p32w_lgwt[t];
    const int b0 = lg >= lgnw ? g << (lg - lgnw) : g >> (lgnw - lg);
    const float4* src = d.Xd + d.off[t] + b0;
    float4* dst = stg + d.p32w_soff[t];
    const int cnt = d.N[t] << lgw;
#pragma unroll 4
    for (int x = threadIdx.x; x < cnt; x += blockDim.x)
      dst[x] = __ldg(src + ((x >> lgw) << lg) + (x & ((1 << lgw) - 1)));
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int n_items = d.pctr[0];
  const float rc = (float)d.rc, rc2 = (float)d.rc2, smin = (float)d.dsf_smin;
  const int kbase = d.dsf_base - ((1023 - 127) << 6);
  float4* buf = ebuf + (threadIdx.x >> 5) * P32W_BUF;
  // the warp's energy sums over its items (exact, fixed point)
  long long sl_lj = 0, sl_c = 0, sl_v = 0;
  int s_nev = 0, s_nlj = 0, bad = 0;
  // the next item is pulled and read while the current one is walked
  int w = 0;
  if (lane == 0) w = atomicAdd(d.pctr + 2 + g, 1);
  w = __shfl_sync(0xffffffffu, w, 0);
  int2 it = w < n_items ? d.pitems[w] : make_int2(0, 0);
  while (w < n_items) {
    const int i = it.x, t = it.y >> 27, n = ((it.y >> 19) & 255) + 1, e0 = it.y & 0x7FFFF;
    int wn = 0;
    if (lane == 0) wn = atomicAdd(d.pctr + 2 + g, 1);
    const AtomInfo ai = d.ainfo[i];
    const int ti = ai.type;
    const int lgPi = ai.log2P, lgPt = tLg[t];
    const int lgS = lgPi > lgPt ? lgPi : lgPt;
    // the pair grid's slices in this window: 2^lgk from s0, or for a grid
    // coarser than the windows one slice in every 2^(lgnw - lgS)-th window
    int lgk = 0, s0 = 0;
    bool none = false;
    if (lgS >= lgnw) {
      lgk = lgS - lgnw;
      s0 = g << lgk;
    } else {
      none = (g & ((1 << (lgnw - lgS)) - 1)) != 0;
      s0 = g >> (lgnw - lgS);
    }
    if (!none) {
      const int G = 32 >> lgk;  // entry groups
      const int sl = s0 + (lane & ((1 << lgk) - 1)), grp = lane >> lgk;
      const int bi = sl >> (lgS - lgPi), bj = sl >> (lgS - lgPt);
      const int pj = bj - tB0[t];
      const float4 di = stg[tSoff[ti] + ((ai.row0 - tOff[ti]) << tLgw[ti]) + (bi - tB0[ti])];
      const float4* lst = d.nlB + (size_t)i * d.nl_cap + e0;
      const float4 far = make_float4(0.f, 0.f, 1e4f, __int_as_float(tSoff[t]));
      const int k = ti * nt + t;
      P32Par c;
      c.rc = rc;
      c.rc2 = rc2;
      c.smin = smin;
      c.kbase = kbase;
      c.qq = qqt[k];
      c.e4 = e4t[k];
      c.s2 = s2t[k];
      c.vrc = vrct[k];
      c.dvrc = dvrct[k];
      const float wgt = __int_as_float((127 - lgS) << 23);  // 1/P*
      float fx = 0.f, fy = 0.f, fz = 0.f, ec = 0.f, elj = 0.f, vir = 0.f;
      int nev = 0;
      // the entries P32W_BUF at a time, each part padded to whole double
      // rounds with far entries of type t (their stage reads stay inside type
      // t's first atom)
      for (int c0 = 0; c0 < n; c0 += P32W_BUF) {
        const int m = min(P32W_BUF, n - c0);
        const int nbuf = (m + 2 * G - 1) / (2 * G) * (2 * G);
        const float4 v0 = lane < m ? __ldg(lst + c0 + lane) : far;  // both loads in flight
        const float4 v1 = lane + 32 < m ? __ldg(lst + c0 + 32 + lane) : far;
        if (lane < nbuf) buf[lane] = v0;
        if (lane + 32 < nbuf) buf[lane + 32] = v1;
        __syncwarp();
        if (c.e4 != 0.f)
          pair32w_walk<true>(buf, nbuf, grp, G, stg, pj, di, c, tab, fx, fy, fz, ec, elj, vir, nev);
        else
          pair32w_walk<false>(buf, nbuf, grp, G, stg, pj, di, c, tab, fx, fy, fz, ec, elj, vir, nev);
        __syncwarp();  // the buffer is refilled next
      }
      const float fs = (c.e4 != 0.f ? 1.0f : c.qq) * wgt;
      long long kx = fm::fixf(fx * fs, 44, &bad), ky = fm::fixf(fy * fs, 44, &bad),
                kz = fm::fixf(fz * fs, 44, &bad);
      // exact sums over the lanes of one owner bead: the other entry groups
      // (lane bits >= lgk) and, for an owner coarser than the pair grid, the
      // slices inside its bead (lane bits < lgS - lgPi)
      const int lgc = lgS - lgPi < lgk ? lgS - lgPi : lgk;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        if (o < (1 << lgc) || o >= (1 << lgk)) {
          kx += __shfl_xor_sync(0xffffffffu, kx, o);
          ky += __shfl_xor_sync(0xffffffffu, ky, o);
          kz += __shfl_xor_sync(0xffffffffu, kz, o);
        }
      }
      const int wmask = ((1 << lgc) - 1) | (31 & ~((1 << lgk) - 1));
      if ((lane & wmask) == 0 && (kx | ky | kz) != 0) {
        unsigned long long* fi = d.F_fix + 3 * (size_t)(ai.row0 + bi * ai.stride);
        atomicAdd(fi + 0, (unsigned long long)kx);
        atomicAdd(fi + 1, (unsigned long long)ky);
        atomicAdd(fi + 2, (unsigned long long)kz);
      }
      // every term is seen from both of its atoms: energies carry a factor 1/2
      sl_lj += fm::fixf(elj * wgt, 39, &bad);
      sl_c += fm::fixf(ec * (c.qq * wgt), 39, &bad);
      sl_v += fm::fixf(vir * fs, 39, &bad);
      s_nev += nev;  // this lane's in-cut-off terms
      if (c.e4 != 0.f) s_nlj += nev;
    }
    w = __shfl_sync(0xffffffffu, wn, 0);
    if (w < n_items) it = d.pitems[w];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sl_lj += __shfl_xor_sync(0xffffffffu, sl_lj, o);
    sl_c += __shfl_xor_sync(0xffffffffu, sl_c, o);
    sl_v += __shfl_xor_sync(0xffffffffu, sl_v, o);
    s_nev += __shfl_xor_sync(0xffffffffu, s_nev, o);
    s_nlj += __shfl_xor_sync(0xffffffffu, s_nlj, o);
  }
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    if (sl_lj) atomicAdd(eacc + 0, (unsigned long long)sl_lj);
    if (sl_c) atomicAdd(eacc + 1, (unsigned long long)sl_c);
    if (sl_v) atomicAdd(eacc + 2, (unsigned long long)sl_v);
    if (s_nev) atomicAdd(eacc + 3, (unsigned long long)s_nev);
    if (s_nlj) atomicAdd(eacc + 4, (unsigned long long)s_nlj);
    if (bad) ebad = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int slot[5] = {E_LJ, E_COUL, E_VIRIAL, E_NEVAL, E_NLJEVAL};
    for (int k = 0; k < 5; ++k)
      if (eacc[k]) atomicAdd(d.E_fix + slot[k], eacc[k]);
    if (ebad) atomicOr(d.err, ERR_NONFINITE);
  }
}

__global__ void __launch_bounds__(P32W_THREADS, 1) k_pair32w(const __grid_constant__ Dev d) { b_k_pair32w(d, blockIdx.x); }

// ---------------------------------------------------------------------------
// bonded terms: one thread per (term, fine slice)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fadd3w(unsigned long long* F, int row, double fx, double fy, double fz, int* bad) {
  unsigned long long* r = F + 3 * (size_t)row;
  atomicAdd(r + 0, (unsigned long long)fix44(fx, 0, bad));
  atomicAdd(r + 1, (unsigned long long)fix44(fy, 0, bad));
  atomicAdd(r + 2, (unsigned long long)fix44(fz, 0, bad));
}

__device__ __forceinline__ void b_k_bonded(const Dev& d, int bx) {
  const int it = bx * blockDim.x + threadIdx.x;
  double eb = 0.0, ea = 0.0, vir = 0.0;
  int bad = 0;
  if (it < d.n_bitems) {
    const BondItem bi = d.bitems[it];
    const int s = bi.slice;
    if (bi.kind == 0) {
      const int a = d.bond_atoms[2 * bi.term], c = d.bond_atoms[2 * bi.term + 1];
      const AtomInfo A = d.ainfo_atom[a], Cc = d.ainfo_atom[c];
      const int lmax = A.log2P > Cc.log2P ? A.log2P : Cc.log2P;
      const double w = pow2_neg(lmax);
      const int ra = A.row0 + (s >> (lmax - A.log2P)) * A.stride;
      const int rcw = Cc.row0 + (s >> (lmax - Cc.log2P)) * Cc.stride;
      const double k = d.bond_par[2 * bi.term], r0 = d.bond_par[2 * bi.term + 1];
      const double dx = d.q[3 * (size_t)rcw] - d.q[3 * (size_t)ra];
      const double dy = d.q[3 * (size_t)rcw + 1] - d.q[3 * (size_t)ra + 1];
      const double dz = d.q[3 * (size_t)rcw + 2] - d.q[3 * (size_t)ra + 2];
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double rinv = rsqrt(r2);
      const double r = r2 * rinv;
      const double kd = w * k * (r - r0);
      eb = 0.5 * kd * (r - r0);
      const double f = -kd * rinv;
      vir = f * r2;
      fadd3w(d.F_fix, rcw, f * dx, f * dy, f * dz, &bad);
      fadd3w(d.F_fix, ra, -f * dx, -f * dy, -f * dz, &bad);
    } else {
      const int a1 = d.ang_atoms[3 * bi.term], o = d.ang_atoms[3 * bi.term + 1], a2 = d.ang_atoms[3 * bi.term + 2];
      const AtomInfo A1 = d.ainfo_atom[a1], O = d.ainfo_atom[o], A2 = d.ainfo_atom[a2];
      int lmax = A1.log2P > O.log2P ? A1.log2P : O.log2P;
      lmax = lmax > A2.log2P ? lmax : A2.log2P;
      const double w = pow2_neg(lmax);
      const int r1 = A1.row0 + (s >> (lmax - A1.log2P)) * A1.stride;
      const int ro = O.row0 + (s >> (lmax - O.log2P)) * O.stride;
      const int r2i = A2.row0 + (s >> (lmax - A2.log2P)) * A2.stride;
      const double k = d.ang_par[2 * bi.term], th0 = d.ang_par[2 * bi.term + 1];
      double u[3], v[3];
      for (int x = 0; x < 3; ++x) {
        u[x] = d.q[3 * (size_t)r1 + x] - d.q[3 * (size_t)ro + x];
        v[x] = d.q[3 * (size_t)r2i + x] - d.q[3 * (size_t)ro + x];
      }
      const double iu = rsqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
      const double iv = rsqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      const double iuv = iu * iv;
      double cs = (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]) * iuv;
      cs = fmin(1.0, fmax(-1.0, cs));
      const double th = acos(cs);
      const double isn = rsqrt(1.0 - cs * cs);
      const double dth = th - th0;
      ea = w * 0.5 * k * dth * dth;
      const double pref = w * k * dth * isn;
      const double au = pref * iuv, bu = pref * cs * iu * iu, bv = pref * cs * iv * iv;
      double f1[3], f2[3];
      for (int x = 0; x < 3; ++x) {
        f1[x] = au * v[x] - bu * u[x];
        f2[x] = au * u[x] - bv * v[x];
      }
      vir = f1[0] * u[0] + f1[1] * u[1] + f1[2] * u[2] + f2[0] * v[0] + f2[1] * v[1] + f2[2] * v[2];
      fadd3w(d.F_fix, r1, f1[0], f1[1], f1[2], &bad);
      fadd3w(d.F_fix, r2i, f2[0], f2[1], f2[2], &bad);
      fadd3w(d.F_fix, ro, -f1[0] - f2[0], -f1[1] - f2[1], -f1[2] - f2[2], &bad);
    }
  }
  eb = warp_sum(eb);
  ea = warp_sum(ea);
  vir = warp_sum(vir);
  bad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    if (bad) atomicOr(d.err, ERR_NONFINITE);
    eadd(d.E_fix, E_BOND, eb);
    eadd(d.E_fix, E_ANGLE, ea);
    eadd(d.E_fix, E_VIRIAL, vir);
  }
}

__global__ void __launch_bounds__(64) k_bonded(const __grid_constant__ Dev d) { b_k_bonded(d, blockIdx.x); }

__global__ void __launch_bounds__(64) k_bonded_b(const Dev* __restrict__ devs, const int* __restrict__ pfx, int nm) {
  MX_BATCH_ENTER();
  b_k_bonded(d, bx);
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
  const int wc = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nch = d.pseudo_chunks;
  if (wc >= d.n_ppitems * nch) return;
  const int w = wc / nch, chunk = wc - w * nch;  // (pseudo bead, slice of its site list)
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
  const double wgt = pow2_neg(pe.log2P);
  const int cnt = min(d.pl_cnt[e], d.pl_cap);
  const int* lst = d.pl + (size_t)e * d.pl_cap;
  const double rc = d.rc, rc2 = d.rc2;
  // the electron bead's sums in fixed point per term: the site list's order
  // is set by the parallel list build, and integer sums do not depend on it
  long long kx = 0, ky = 0, kz = 0, ke = 0, kv = 0;
  int nev = 0, bad = 0;
  const int ps_hi_min = __double2hiint(d.ps_smin);
  for (int k = chunk * 32 + lane; k < cnt; k += 32 * nch) {
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
      // shifted-force value and -(dV/dr - dV/dr(rc)) / r: from the site
      // type's interval table, or analytic below its range (and when the
      // parameters differ from the tabulated ones)
      double vsf, fru;
      const int hi = __double2hiint(r2);
      if (d.ps_tab && hi >= ps_hi_min) {
        dsf_table(d.ps_tab + 12 * ((size_t)ac.type * d.ps_nint + ((hi >> 14) - d.ps_base)), hi, r2, &vsf, &fru);
      } else {
        const PseudoPar pp = tab[ac.type];
        const double r = sqrt(r2);
        double v, dv;
        pseudo_raw(pp, r, &v, &dv);
        vsf = v - pp.vrc - (r - rc) * pp.dvrc;
        fru = -(dv - pp.dvrc) / r;
      }
      const double fr = wgt * fru;  // force on the site along d
      const double fx = fr * dx, fy = fr * dy, fz = fr * dz;
      ke += fixs(wgt * vsf, 40, &bad);
      kv += fixs(fr * r2, 40, &bad);
      kx -= fix44(fx, 0, &bad);
      ky -= fix44(fy, 0, &bad);
      kz -= fix44(fz, 0, &bad);
      ++nev;
      fadd3w(d.F_fix, row_c, fx, fy, fz, &bad);
    }
  }
  // exact integer sums over the lanes
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kx += __shfl_xor_sync(0xffffffffu, kx, o);
    ky += __shfl_xor_sync(0xffffffffu, ky, o);
    kz += __shfl_xor_sync(0xffffffffu, kz, o);
    ke += __shfl_xor_sync(0xffffffffu, ke, o);
    kv += __shfl_xor_sync(0xffffffffu, kv, o);
  }
  nev = warp_sumi(nev);
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    unsigned long long* fe = d.F_fix + 3 * (size_t)row_e;
    if (kx | ky | kz) {
      atomicAdd(fe + 0, (unsigned long long)kx);
      atomicAdd(fe + 1, (unsigned long long)ky);
      atomicAdd(fe + 2, (unsigned long long)kz);
    }
    if (ke) atomicAdd(d.E_fix + E_PSEUDO, (unsigned long long)ke);
    if (kv) atomicAdd(d.E_fix + E_VIRIAL, (unsigned long long)kv);
    if (nev) atomicAdd(d.E_fix + E_NPEVAL, (unsigned long long)nev);
    if (bad) atomicOr(d.err, ERR_NONFINITE);
  }
}


// pseudopotential in FP32 (precision MIXTS_FP32_FORCES): one warp per
// (pseudo particle, bead), lanes over sites; site reactions through
// fixed-point atomics assembled from the bit fields
__global__ void __launch_bounds__(PAIR_THREADS) k_pseudo32(Dev d) {
  __shared__ float pk[MT], psg[MT], pA[MT], pb[MT], pvr[MT], pdv[MT];
  __shared__ float4 shh[125], shl[125];
  for (int e = threadIdx.x; e < d.n_types; e += blockDim.x) {
    const PseudoPar pp = d.pspar[e];
    pk[e] = (float)pp.kq;
    psg[e] = (float)pp.sig;
    pA[e] = (float)pp.A;
    pb[e] = (float)pp.b;
    pvr[e] = (float)pp.vrc;
    pdv[e] = (float)pp.dvrc;
  }
  for (int e = threadIdx.x; e < 125; e += blockDim.x) {
    const int nx = e / 25 - 2, ny = (e / 5) % 5 - 2, nz = e % 5 - 2;
    const double lo = d.box - (double)d.box_hi;
    shh[e] = make_float4(nx * d.box_hi, ny * d.box_hi, nz * d.box_hi, 0.0f);
    shl[e] = make_float4((float)(nx * lo), (float)(ny * lo), (float)(nz * lo), 0.0f);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int wc = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nch = d.pseudo_chunks;
  if (wc >= d.n_ppitems * nch) return;
  const int w = wc / nch, chunk = wc - w * nch;  // (pseudo bead, slice of its site list)
  int e = 0, base = 0;
  while (e + 1 < d.n_pseudo && w >= base + (1 << d.pinfo[e].log2P)) {
    base += 1 << d.pinfo[e].log2P;
    ++e;
  }
  const int sb = w - base;
  const AtomInfo pe = d.pinfo[e];
  const int row_e = pe.row0 + sb * pe.stride;
  const float4 eh = d.Xf[row_e], el = d.Xl[row_e];
  const float wgt = __int_as_float((127 - pe.log2P) << 23);
  const int cnt = min(d.pl_cnt[e], d.pl_cap);
  const int* lst = d.pl + (size_t)e * d.pl_cap;
  const float rc = (float)d.rc, rc2 = (float)d.rc2;
  float fex = 0.f, fey = 0.f, fez = 0.f, ep = 0.f, vir = 0.f;
  int nev = 0, bad = 0;
  for (int k = chunk * 32 + lane; k < cnt; k += 32 * nch) {
    const int ent = lst[k];
    const AtomInfo ac = d.ainfo[ent >> 7];
    const int row_c = ac.row0 + (sb >> (pe.log2P - ac.log2P)) * ac.stride;
    const float4 ch = d.Xf[row_c], cl = d.Xl[row_c];
    const float4 sh = shh[ent & 127], sm = shl[ent & 127];
    const float dx = ((ch.x - eh.x) + sh.x) + ((cl.x - el.x) + sm.x);
    const float dy = ((ch.y - eh.y) + sh.y) + ((cl.y - el.y) + sm.y);
    const float dz = ((ch.z - eh.z) + sh.z) + ((cl.z - el.z) + sm.z);
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    if (!(r2 < rc2)) continue;
    const int t = ac.type;
    const float r = sqrtf(r2);
    const float x = r / psg[t];
    float gg, dg;
    if (x < 1.0e-3f) {
      const float x2 = x * x, c = 1.1283791670955126f / psg[t];
      gg = c * (1.0f - x2 / 3.0f + x2 * x2 / 10.0f);
      dg = c / psg[t] * (-2.0f * x / 3.0f + 0.4f * x2 * x);
    } else {
      const float ef = erff(x);
      gg = ef / r;
      dg = 1.1283791670955126f * expf(-x * x) / (psg[t] * r) - ef / r2;
    }
    const float ex = expf(-r / pb[t]);
    const float v = -pk[t] * gg + pA[t] * ex;
    const float dv = -pk[t] * dg - (pA[t] / pb[t]) * ex;
    ep = fmaf(wgt, v - pvr[t] - (r - rc) * pdv[t], ep);
    const float fr = -wgt * (dv - pdv[t]) / r;  // force on the site along d
    const float fx = fr * dx, fy = fr * dy, fz = fr * dz;
    fex -= fx;
    fey -= fy;
    fez -= fz;
    vir = fmaf(fr, r2, vir);
    ++nev;
    unsigned long long* fc = d.F_fix + 3 * (size_t)row_c;
    atomicAdd(fc + 0, (unsigned long long)fm::fixf(fx, 44, &bad));
    atomicAdd(fc + 1, (unsigned long long)fm::fixf(fy, 44, &bad));
    atomicAdd(fc + 2, (unsigned long long)fm::fixf(fz, 44, &bad));
  }
  long long kx = fm::fixf(fex, 44, &bad), ky = fm::fixf(fey, 44, &bad), kz = fm::fixf(fez, 44, &bad);
  long long ke = fm::fixf(ep, 40, &bad), kv = fm::fixf(vir, 40, &bad);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    kx += __shfl_xor_sync(0xffffffffu, kx, o);
    ky += __shfl_xor_sync(0xffffffffu, ky, o);
    kz += __shfl_xor_sync(0xffffffffu, kz, o);
    ke += __shfl_xor_sync(0xffffffffu, ke, o);
    kv += __shfl_xor_sync(0xffffffffu, kv, o);
  }
  nev = warp_sumi(nev);
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    unsigned long long* fe = d.F_fix + 3 * (size_t)row_e;
    atomicAdd(fe + 0, (unsigned long long)kx);
    atomicAdd(fe + 1, (unsigned long long)ky);
    atomicAdd(fe + 2, (unsigned long long)kz);
    atomicAdd(d.E_fix + E_PSEUDO, (unsigned long long)ke);
    atomicAdd(d.E_fix + E_VIRIAL, (unsigned long long)kv);
    atomicAdd(d.E_fix + E_NPEVAL, (unsigned long long)nev);
    if (bad) atomicOr(d.err, ERR_NONFINITE);
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int launch_nlist(const Dev& d, cudaStream_t s, const int* atom_is_pseudo) {
  int n = 1;
  (void)atom_is_pseudo;  // carried in d
  k_list_prep<<<1, 1024, 0, s>>>(d);
  if (d.n_nonp > 0) {
    const long long warps = (long long)d.n_nonp * nlist_parts(d);
    const int wpb = NL_THREADS / 32;
    k_nlist<<<(int)((warps + wpb - 1) / wpb), NL_THREADS, 0, s>>>(d);
    ++n;
  }
  if (d.n_pseudo > 0 && d.n_nonp > 0) {
    dim3 g((d.n_nonp + 127) / 128, d.n_pseudo);
    k_plist<<<g, 128, 0, s>>>(d);
    ++n;
  }
  return n;
}

// persistent grid sizes: resident CTAs per SM times SMs
// dynamic shared memory of k_pair64: the interval table, and the row prefix
// of implicit items
size_t pair64_smem(const Dev& d) {
  return PAIR64_SMEM_PER_INTERVAL * (size_t)d.dsf_nint + (d.p64_implicit ? sizeof(int) * ((size_t)d.n_nonp + 1) : 0);
}

void pair_grids(int nt, size_t smem64, int nint, int* g64, int* g32) {
  int dev = 0, sms = 0, b64 = 0, b32 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  (void)nt;
  cudaFuncSetAttribute(k_pair64, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, k_pair64, PAIR64_THREADS, smem64);
  cudaFuncSetAttribute(k_pair32, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b32, k_pair32, PAIR_THREADS, PAIR32_SMEM_PER_INTERVAL * (size_t)nint);
  *g64 = std::max(1, b64) * std::max(1, sms);
  *g32 = std::max(1, b32) * std::max(1, sms);
}

// FP32 window sweep geometry: the widest window (at most 8 slices of the
// finest non-pseudo bead grid) whose bead stage, DSF table and entry buffers
// fit one CTA's shared memory, and whole multiples of the window count of
// resident CTAs; p32w = 0 (the gather sweep k_pair32) when none fits
void pair32w_plan(Dev& d) {
  d.p32w = 0;
  // small systems give a 1024-thread CTA too few items per window: they keep
  // the gather sweep (as do all members of a batched handle)
  if (d.precision != MIXTS_FP32_FORCES || d.n_nonp < P32W_MIN_ATOMS) return;
  int dev = 0, sms = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_pair32w) != cudaSuccess) return;
  const size_t stat = fa.sharedSizeBytes;
  if (d.nl_cap >= (1 << 19)) return;  // entry offsets of window items have 19 bits
  const int lgPm = d.lgPmax_nb;
  for (int lgw = lgPm < 3 ? lgPm : 3; lgw >= 0; --lgw) {
    const int lgnw = lgPm - lgw;
    if ((1 << lgnw) > P32W_MAX_NW) break;
    long long nst = 0;
    int lgwt[MT] = {0}, soff[MT] = {0};
    for (int t = 0; t < d.n_types; ++t) {
      lgwt[t] = d.log2P[t] > lgnw ? d.log2P[t] - lgnw : 0;
      soff[t] = (int)nst;
      if (!d.pseudo[t]) nst += (long long)d.N[t] << lgwt[t];
    }
    const size_t smem = PAIR32_SMEM_PER_INTERVAL * (size_t)d.dsf_nint +
                        sizeof(float4) * ((size_t)nst + (size_t)(P32W_THREADS / 32) * P32W_BUF);
    if (smem + stat > (size_t)optin) continue;
    // the attribute is the device's limit, so that handles of other sizes
    // never lower it under one another
    if (cudaFuncSetAttribute(k_pair32w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes) != cudaSuccess)
      return;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair32w, P32W_THREADS, smem);
    if (occ < 1) return;
    const int nw = 1 << lgnw;
    d.p32w = 1;
    d.p32w_lgnw = lgnw;
    d.p32w_nstage = (int)nst;
    d.p32w_smem = (int)smem;
    d.p32w_grid = nw * std::max(1, occ * std::max(1, sms) / nw);
    for (int t = 0; t < MT; ++t) {
      d.p32w_lgwt[t] = lgwt[t];
      d.p32w_soff[t] = soff[t];
    }
    return;
  }
}

int launch_pair(const Dev& d, cudaStream_t s) {
  const int wpb = PAIR_THREADS / 32;
  if (d.precision == MIXTS_FP32_FORCES) {
    if (d.n_nonp == 0) return 0;
    static bool attr32 = false;
    if (!attr32) {
      cudaFuncSetAttribute(k_pair32, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
      attr32 = true;
    }
    k_list_seg32<<<(d.n_nonp + wpb - 1) / wpb, NL_THREADS, 0, s>>>(d);
    if (d.p32w)
      k_pair32w<<<d.p32w_grid, P32W_THREADS, d.p32w_smem, s>>>(d);
    else
      k_pair32<<<d.pair32_grid, PAIR_THREADS, PAIR32_SMEM_PER_INTERVAL * (size_t)d.dsf_nint, s>>>(d);
    return 2;
  }
  if (d.n_pitems == 0) return 0;
  const size_t smem = pair64_smem(d);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_pair64, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr = true;
  }
  const int nsbm = d.lgPmax_nb > 5 ? 1 << (d.lgPmax_nb - 5) : 1;
  const long long items = (long long)d.n_nonp * nsbm * d.p64_nch;  // bound on the list's items
  int n = 0;
  if (!d.p64_implicit) {
    k_pair_items<<<(d.n_nonp + ITEM_THREADS - 1) / ITEM_THREADS, ITEM_THREADS, 0, s>>>(d);
    ++n;
  }
  const int wpb64 = PAIR64_THREADS / 32;
  k_pair64<<<(int)std::min<long long>((items + wpb64 - 1) / wpb64, d.pair_grid), PAIR64_THREADS, smem, s>>>(d);
  return n + 1;
}

int launch_bonded(const Dev& d, cudaStream_t s, const AtomInfo* ainfo_atom) {
  if (d.n_bitems == 0) return 0;
  (void)ainfo_atom;  // carried in d
  k_bonded<<<(d.n_bitems + 63) / 64, 64, 0, s>>>(d);
  return 1;
}

// blocks of each batched kernel for one member: the single-system launch shapes
void batch_block_counts(const Dev& d, int* c) {
  for (int k = 0; k < BK_KINDS; ++k) c[k] = 0;
  const int wpb = PAIR_THREADS / 32;
  c[BK_PREP] = 1;
  if (d.n_nonp > 0) {
    c[BK_NLIST] = (int)(((long long)d.n_nonp * nlist_parts(d) + NL_THREADS / 32 - 1) / (NL_THREADS / 32));
    if (d.precision == MIXTS_FP32_FORCES) {  // members take the gather sweep (p32w = 0)
      c[BK_PAIRA] = (d.n_nonp + wpb - 1) / wpb;
      c[BK_PAIRB] = d.pair32_grid;
    } else {
      const int nsbm = d.lgPmax_nb > 5 ? 1 << (d.lgPmax_nb - 5) : 1;
      const long long items = (long long)d.n_nonp * nsbm * d.p64_nch;
      c[BK_PAIRA] = d.p64_implicit ? 0 : (d.n_nonp + ITEM_THREADS - 1) / ITEM_THREADS;
      c[BK_PAIRB] = (int)std::min<long long>((items + PAIR64_THREADS / 32 - 1) / (PAIR64_THREADS / 32), d.pair_grid);
    }
  }
  c[BK_BONDED] = (d.n_bitems + 63) / 64;
  c[BK_PROP] = d.n_tiles;
  c[BK_FINAL] = 1;
}

// one part of the batched force evaluation: 0 neighbour lists, 1 pair sweep,
// 2 bonded terms
int launch_forces_batched_part(const BatchGeom& g, cudaStream_t s, int part) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_pair64_b, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    cudaFuncSetAttribute(k_pair32_b, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr = true;
  }
  const int r = g.nm + 1;
  auto pf = [&](int k) { return g.pfx + k * r; };
  int n = 0;
  if (part == 0) {
    k_list_prep_b<<<g.blocks[BK_PREP], 1024, 0, s>>>(g.devs, pf(BK_PREP), g.nm);
    ++n;
    if (g.blocks[BK_NLIST] > 0) {
      k_nlist_b<<<g.blocks[BK_NLIST], NL_THREADS, 0, s>>>(g.devs, pf(BK_NLIST), g.nm);
      ++n;
    }
  } else if (part == 1) {
    if (g.precision == MIXTS_FP32_FORCES) {
      if (g.blocks[BK_PAIRA] > 0) {
        k_list_seg32_b<<<g.blocks[BK_PAIRA], NL_THREADS, 0, s>>>(g.devs, pf(BK_PAIRA), g.nm);
        k_pair32_b<<<g.blocks[BK_PAIRB], PAIR_THREADS, g.pair_smem, s>>>(g.devs, pf(BK_PAIRB), g.nm);
        n += 2;
      }
    } else {
      // item arrays only for members too large for the in-kernel row prefix
      if (g.blocks[BK_PAIRA] > 0) {
        k_pair_items_b<<<g.blocks[BK_PAIRA], ITEM_THREADS, 0, s>>>(g.devs, pf(BK_PAIRA), g.nm);
        ++n;
      }
      if (g.blocks[BK_PAIRB] > 0) {
        k_pair64_b<<<g.blocks[BK_PAIRB], PAIR64_THREADS, g.pair_smem, s>>>(g.devs, pf(BK_PAIRB), g.nm);
        ++n;
      }
    }
  } else if (g.blocks[BK_BONDED] > 0) {
    k_bonded_b<<<g.blocks[BK_BONDED], 64, 0, s>>>(g.devs, pf(BK_BONDED), g.nm);
    ++n;
  }
  return n;
}

// neighbour lists, pair sweep and bonded terms of every member of a batch,
// one launch per kernel
int launch_forces_batched(const BatchGeom& g, cudaStream_t s) {
  return launch_forces_batched_part(g, s, 0) + launch_forces_batched_part(g, s, 1) +
         launch_forces_batched_part(g, s, 2);
}

int launch_pseudo(const Dev& d, cudaStream_t s) {
  const int wpb = PAIR_THREADS / 32;
  if (d.n_ppitems == 0 || d.n_nonp == 0) return 0;
  const int items = d.n_ppitems * d.pseudo_chunks;
  if (d.precision == MIXTS_FP32_FORCES) {
    k_pseudo32<<<(items + wpb - 1) / wpb, PAIR_THREADS, 0, s>>>(d);
    return 1;
  }
  k_pseudo64<<<(items + wpb - 1) / wpb, PAIR_THREADS, 0, s>>>(d);
  return 1;
}

}  // namespace mx
