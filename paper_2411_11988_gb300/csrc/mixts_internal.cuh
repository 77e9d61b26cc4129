// mixts_internal.cuh -- device-side data view and helpers of the mixTS-PIMD
// hot path for sm_103a. Everything here is used only by the .cu files of
// this library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mixts.h"

namespace mx {

constexpr int MT = MIXTS_MAX_TYPES;
constexpr int MAX_CLASSES = 12;
constexpr int SMALL_P = 64;     // types with P <= SMALL_P propagate in one fused tile kernel
constexpr int PROP_TILE_BEADS = 128;  // beads (P x atoms) of one small-P propagation tile
constexpr int BIG_MAXA = 64;    // atoms per large-P propagation tile at most
constexpr int NC_MAX = 16;      // cells per side of the neighbour search at most (NC_MAX^3 counted in shared memory)
constexpr int BIG_CL_MAX = 16;  // CTAs per large-P tile (one thread-block cluster) at most
constexpr int BIG_SMEM_TARGET = 100 * 1024;  // per-CTA shared memory of a large-P tile at most
constexpr int PROP_SMEM_MAX = 200 * 1024;
constexpr int P64_IMPLICIT_ROWS = 8192;  // FP64 item prefixes in shared memory up to this many rows
constexpr int P64_CH = 16;      // list entries per lane group of one FP64 pair item (8: 0.3 %, 32: 3.5 %, 64: 19 % slower)
constexpr int LG_P32_TERMS = 11; // default log2 of the bead-pair terms of one FP32 pair item (Dev::p32_lgt)
// FP32 pair sweep over imaginary-time windows (k_pair32w): CTA threads,
// staged list entries per warp (a multiple of 64, so that a padded part
// stays within it), and the most windows a system may have
constexpr int P32W_THREADS = 1024;
constexpr int P32W_BUF = 64;
constexpr int P32W_MAX_NW = 64;
constexpr int P32W_MIN_ATOMS = 768;  // fewer non-pseudo atoms: the gather sweep k_pair32
// shared memory of one CTA of a large-P propagation tile of na atoms split
// over a cluster of cl CTAs: the twiddles, the bead-column and frequency
// rows of the packed complex columns, and the owned q and p modes
inline size_t big_prop_smem(int P, int na, int cl) {
  const size_t C = 3 * (size_t)na, nz = (C + 1) / 2, own = (size_t)P / cl;
  return 16 * ((size_t)P / 2) + 16 * 2 * nz * own + 8 * 2 * C * own;
}

// Forces and energies are accumulated in 64-bit fixed point, so that sums
// are exact integers whatever order the atomics land in: the whole step is
// bitwise reproducible.
constexpr double FSCALE = 17592186044416.0;   // 2^44 per kcal/mol/A
constexpr double FINV = 1.0 / 17592186044416.0;
constexpr double ESCALE = 1099511627776.0;    // 2^40 per kcal/mol
constexpr double EINV = 1.0 / 1099511627776.0;
constexpr double FMAX = 262144.0;             // |single contribution| limit, kcal/mol/A

enum : int { ERR_NLIST = 1, ERR_NONFINITE = 2, ERR_BOX = 4, ERR_TIMEOUT = 8, ERR_PLIST = 16 };

// energy accumulator slots (fixed point) and counters
enum : int { E_LJ = 0, E_COUL, E_BOND, E_ANGLE, E_PSEUDO, E_VIRIAL, E_NEVAL, E_NPEVAL, E_NLJEVAL, E_NSLOTS };

// estimator partial slots per propagation block: per type 4 values + heat
constexpr int PART_PER_TYPE = 4;  // KE, spring energy, centroid-virial sum, Rg sum
constexpr int PART_STRIDE = MT * PART_PER_TYPE + 2;

// estimate record (device), see mixts_estimates
constexpr int EST_N = 16 + 4 * MT + 4;  // tail: [16+4MT] LJ eval count

struct AtomInfo {  // one non-pseudo atom, by sorted position
  int row0;        // bead-0 row in the flat layout
  int stride;      // rows between consecutive beads (N_t)
  int log2P;
  int type;
};

struct PairPar {   // nonbonded parameters of a type pair
  double qq;       // k_e q_i q_j
  double e4;       // 4 eps
  double s2;       // sigma^2
  double vrc;      // LJ value at r_cut
  double dvrc;     // LJ slope at r_cut
};

struct PseudoPar { // pseudopotential parameters of a site type
  double kq;       // k_e q_site
  double sig;      // sigma
  double A;        // kcal/mol
  double b;
  double vrc, dvrc;
};

struct ModeCoef {  // per (type, mode): thermostat and exact free-ring rotation
  double c1;       // exp(-gamma dt/2)
  double c2s;      // sqrt(1 - c1^2) sqrt(m kT)
  double cw;       // cos(omega dt)
  double mws;      // m omega sin(omega dt)       (k = 0: 0)
  double swm;      // sin(omega dt)/(m omega)     (k = 0: dt/m)
  double hmw2;     // m omega^2 / 2 (spring energy in mode space)
};

struct PropTile {  // one CTA of the fused propagation
  int type, k0, na, slot;
};

struct BondItem {  // one bonded term evaluated on one fine slice
  int kind;        // 0 bond, 1 angle
  int term;
  int slice;
  int pad;
};

struct Dev {
  // sizes
  int n_atoms, n_nonp, n_pseudo, n_types, n_beads;
  int n_bitems, n_pitems, n_ppitems;
  int nl_cap, pl_cap;
  int n_classes;
  int n_tiles;          // small-P propagation tiles (tiles[0, n_tiles))
  int n_big_tiles;      // large-P propagation tiles (tiles[n_tiles, n_tiles + n_big_tiles))
  int big_smem;         // dynamic shared memory of one CTA of the large-P tile kernel
  int big_cl;           // CTAs per large-P tile (cluster size)
  int n_part_slots;     // estimator partial slots
  int precision;
  double box, rc, rc2, alpha;
  double dsf_erfc_rc_over_rc, dsf_cf, dsf_g;
  // DSF interval table: s in [dsf_smin, 2^e_hi), 64 sub-intervals per octave
  const double* dsf_tab;
  const float4* dsf32;      // binary32 cubics (FP32 forces): [G c0..c3][-2G' c0..c3] per interval
  int dsf_nint, dsf_base;   // interval count; (1023 + e_lo) << 6
  double dsf_smin;          // 2^e_lo
  // pseudopotential interval tables, one per site type (same layout as the
  // DSF table: shifted-force V and -(dV/dr - dV/dr(rc)) / r); null: analytic
  const double* ps_tab;     // [n_types][ps_nint][12]
  int ps_nint, ps_base;     // intervals per type; (1023 + e_lo) << 6
  double ps_smin;           // 2^e_lo
  float box_hi;             // box edge rounded to the 2^-12 A grid
  long long box_fix;        // box edge in 2^-48 A fixed point
  float screen_rc2;         // binary32 screen radius^2 (r_cut + 2e-3)^2
  int full_list;            // 1: every row lists all partners (FP32 force path)
  int lgPmax_nb;            // log2 of the largest bead count among non-pseudo atoms
  int n_items32;            // FP32 pair items: n_nonp * 2^lgPmax_nb
  double dt, kcal, kT, kB;
  uint64_t seed;
  // per type
  int P[MT], log2P[MT], N[MT], off[MT], pseudo[MT], atoff[MT];
  int cm_off[MT];       // offset of C (P <= SMALL_P) or the FFT twiddles (P > SMALL_P)
  int mc_off[MT];       // offset of the ModeCoef rows
  int pair_grid, pair32_grid, pseudo_chunks;  // persistent grid sizes, site-list split
  int nl_cpl;                                 // list candidates per lane of one list warp
  int p32_lgt;                                // log2 of the bead-pair terms of one FP32 pair item (tunable)
  int p64_nch;                                // FP64 slice-parallel items per owner row and slice block (bound)
  int p64_implicit;                           // 1: FP64 items from a row prefix each CTA builds (no item array)
  int2* pitems;                               // FP64 pair items of the current list: (owner pos, sb << 16 | chunk)
  int* pctr;                                  // [0] item count of the current list, [1] next item to hand out,
                                              // [2 + g] next item of window g (k_pair32w)
  // FP32 window sweep: 1 when on; log2 of the windows; window beads and
  // stage offset per type; staged beads of one window; dynamic shared memory
  int p32w, p32w_lgnw, p32w_nstage, p32w_smem, p32w_grid;
  int p32w_lgwt[MT], p32w_soff[MT];
  float4* nlB;                 // FP32 path: list rows regrouped by partner type, (bead-0 displacement, tag)
  int* nlseg;                  // FP32 path: [n_nonp][n_types + 1] first entry of each partner type in nlB
  float box_lo;                // box - box_hi (binary32)
  const int* atom_is_pseudo;   // [n_atoms]
  const AtomInfo* ainfo_atom;  // [n_atoms] by atom index
  const int* slot_type;        // [n_part_slots] type of each estimator partial slot
  // long-range electrostatics on centroids (coulomb == 1, see k_ewald.cu)
  int coulomb, ew_kmax, n_kvec, n_qatoms, n_intra;
  double ew_ke, ew_const, ew_bg, ew_inv2a2;  // k_e; self + background energy; background; 1/(2 alpha^2)
  const double4_32a* kvec;     // [n_kvec] half-space wave vectors (kx, ky, kz, W_k)
  const int4* kn;              // [n_kvec] (nx, ny, nz, 0)
  const int4* qinfo;           // [n_qatoms] charged sites: (bead-0 row, row stride, P, atom)
  const double* qcharge;       // [n_qatoms]
  const int2* intra;           // [n_intra] same-molecule pairs of charged sites (indices into qinfo)
  double2* ew_phase;           // [n_qatoms][3][ew_kmax + 1] exp(i 2 pi n x / L)
  double4_32a* ew_cen;         // [n_qatoms] centroids
  double2* ew_S;               // [n_kvec] structure factors
  double* ew_ek;               // [n_kvec][2] energy and virial per wave vector
  double mass[MT];
  // sorted classes of non-pseudo atoms (P descending)
  int cls_P[MAX_CLASSES], cls_log2P[MAX_CLASSES], cls_pos0[MAX_CLASSES], cls_n[MAX_CLASSES],
      cls_item0[MAX_CLASSES];
  // tables
  const AtomInfo* ainfo;   // [n_nonp]
  const int* pos_atom;     // [n_nonp] atom index of a sorted position
  const int* pos_mol;      // [n_nonp]
  const int* atom_of_tk;   // [n_atoms] atom index of (type, rank), at atoff[t] + k
  const int* pseudo_atom;  // [n_pseudo]
  const AtomInfo* pinfo;   // [n_pseudo]
  const PairPar* pairpar;  // [MT*MT]
  const PseudoPar* pspar;  // [MT]
  const BondItem* bitems;  // [n_bitems]
  const int* bond_atoms;   // [n_bonds*2]
  const double* bond_par;  // [n_bonds*2] k, r0
  const int* ang_atoms;    // [n_angles*3]
  const double* ang_par;   // [n_angles*2] k, theta0
  const double* cm;        // NM matrices / cos tables
  const ModeCoef* mc;      // mode coefficients
  const PropTile* tiles;   // [n_tiles]
  // caller state
  double* q;
  double* p;
  double* f;
  // internal state
  double* q_nm;
  double* p_nm;
  unsigned long long* F_fix;   // [n_beads*3], two's-complement fixed point
  double4_32a* Xw;                 // [n_beads] positions shifted so bead 0 of each atom lies in the box
  longlong4_32a* Xi;               // [n_beads] the same in 2^-48 A fixed point (exact differences)
  float4* Xf;                  // [n_beads] binary32 positions on the 2^-12 A grid (screens)
  float4* Xl;                  // [n_beads] binary32 remainders: Xw = Xf + Xl to ~2^-37 A
  longlong4_32a* XiA;          // [n_beads] Xi atom-major inside each type block (off_t + k P_t + b); FP64 path only
  float4* Xd;                  // [n_beads] binary32 offset of each bead from its atom's bead 0, atom-major
                               // inside each type block (off_t + k P_t + b); FP32 path only, else null
  double* ref;                 // [n_atoms*3] wrapped bead-0 reference positions
  double4_32a* refd;           // [n_nonp] the same by sorted position
  float4* reff;                // [n_nonp] binary32 copy, .w = log2 P (int bits)
  int4* wrapn;                 // [n_nonp] lattice vector that wrapped bead 0 (q_0 = ref + wrapn L)
  const int* pos_of_atom;      // [n_atoms] sorted position, -1 for pseudo particles
  double* spread;              // [n_atoms] max |q_b - q_0|
  int* nl;                     // [n_nonp*nl_cap] (partner position << 7) | image code
  int* nl_cnt;                 // [n_nonp]
  // cell list of the neighbour search (nc >= 3 cells per side; 0: all pairs)
  int nc;                      // cells per side, cell side L / nc
  float cell_inv;              // nc / L
  int* cell_start;             // [nc^3 + 1] first sorted slot of each cell
  int* cell_atoms;             // [n_nonp] atom positions ordered by cell
  int* cell_ok;                // 1 when this step's list radius fits the cell side
  int* pl;                     // [n_pseudo*pl_cap]
  int* pl_cnt;                 // [n_pseudo]
  double* thresh;              // [12] d_max, list radius, d_max pseudo, pseudo radius; 9 binary32
                               // screen constants from byte 32; [10] R^2, [11] R_pseudo^2
  unsigned long long* E_fix;   // [E_NSLOTS]
  int* err;                    // [1]
  long long* step_ctr;         // [1] completed steps
  double* heat;                // [1]
  double* est;                 // [EST_N]
  double* parts;               // [n_part_slots * PART_STRIDE]
};

// ---------------------------------------------------------------------------
// Conversions by integer instructions. On this part the FP64 unit is narrow
// (2 lanes per clock per SM) and int<->float conversions share it, so hot
// loops assemble binary64 values from their bit fields instead.
// ---------------------------------------------------------------------------
// Fixed point without the FP64 pipe: v * 2^scale_log2 rounded to the nearest
// integer (halves away from zero), from the binary64 bit fields (integer
// instructions only). Flags |v 2^scale_log2| >= 2^62 (and inf/NaN) in *bad.
// fix44(v, w) is the force scale 2^44 with a power-of-two weight 2^-w.
__device__ __forceinline__ long long fixs(double v, int scale_log2, int* bad) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF);
  const int sh = e - 1075 + scale_log2;  // v * 2^s = mantissa * 2^(e - 1075 + s)
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  long long r;
  if (e == 0x7FF || sh > 9) {
    *bad = 1;
    r = 0;
  } else if (sh >= 0) {
    r = m << sh;
  } else if (sh >= -53) {
    r = (m + (1LL << (-sh - 1))) >> (-sh);
  } else {
    r = 0;
  }
  return b < 0 ? -r : r;
}

__device__ __forceinline__ long long fix44(double v, int wshift, int* bad) { return fixs(v, 44 - wshift, bad); }

// 2^-l (0 <= l <= 1022) assembled from its bits: the exact value of
// 1.0 / (1 << l) without a division
__device__ __forceinline__ double pow2_neg(int l) { return __hiloint2double((1023 - l) << 20, 0); }

// Binary64 value of v * 2^-scale_log2 by integer instructions (normalise
// with a leading-zero count, assemble exponent and mantissa); exact for
// |v| < 2^53, truncated beyond.
__device__ __forceinline__ double fix_to_dbl(long long v, int scale_log2) {
  if (v == 0) return 0.0;
  const unsigned long long sgn = v < 0 ? 0x8000000000000000ull : 0ull;
  const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int msb = 63 - __clzll((long long)a);
  const unsigned long long m = msb <= 52 ? a << (52 - msb) : a >> (msb - 52);
  const unsigned long long e = (unsigned long long)(msb - scale_log2 + 1023);
  return __longlong_as_double((long long)(sgn | (e << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

__device__ __forceinline__ double fixpos_to_double(long long v) { return fix_to_dbl(v, 48); }

// exact binary32 -> binary64 for zero and normal numbers (bit fields)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int ex = (u >> 23) & 0xFFu;
  if (ex == 0u) return 0.0;
  const unsigned long long sg = (unsigned long long)(u >> 31) << 63;
  const unsigned long long e = (unsigned long long)(ex + 896u) << 52;
  const unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(sg | e | m));
}

// binary32 value of a small integer k, |k| < 2^22, without a conversion
__device__ __forceinline__ float small_int_float(int k) {
  return __int_as_float(0x4B000000 + (k + (1 << 22))) - 12582912.0f;
}

// ---------------------------------------------------------------------------
// fixed-point accumulation
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long to_fix(double v, double scale, int* err) {
  double s = v * scale;
  if (!(fabs(v) < FMAX)) {  // also catches NaN
    atomicOr(err, ERR_NONFINITE);
    s = 0.0;
  }
  return __double2ll_rn(s);
}

__device__ __forceinline__ void fadd3(unsigned long long* F, int row, double fx, double fy, double fz,
                                      int* err) {
  unsigned long long* r = F + 3 * (size_t)row;
  atomicAdd(r + 0, (unsigned long long)to_fix(fx, FSCALE, err));
  atomicAdd(r + 1, (unsigned long long)to_fix(fy, FSCALE, err));
  atomicAdd(r + 2, (unsigned long long)to_fix(fz, FSCALE, err));
}

__device__ __forceinline__ void eadd(unsigned long long* E, int slot, double v) {
  atomicAdd(E + slot, (unsigned long long)__double2ll_rn(v * ESCALE));
}

__device__ __forceinline__ double fix_to_double(unsigned long long v, double inv) {
  (void)inv;
  return fix_to_dbl((long long)v, 44);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sumi(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the thermostat's
// standard normals: a binary32 Box-Muller whose logarithm and sine/cosine are
// fixed sequences of correctly rounded operations (so any IEEE machine
// running the same sequence produces the same bits).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// ln(u), u = (2 floor(r / 2^9) + 1) 2^-24: u = f 2^e exactly with f folded
// into (sqrt(1/2), sqrt(2)], ln f from the odd series of 2 atanh(s),
// s = (f-1)/(f+1), through s^9; e ln 2 added with ln 2 split in two parts.
__device__ __forceinline__ float log_u24(uint32_t r) {
  const uint32_t m = ((r >> 9) << 1) | 1u;
  int e = 31 - __clz((int)m);
  float f = __fmul_rn(__uint2float_rn(m), __int_as_float((127 - e) << 23));
  if (f > 0x1.6a09e6p+0f) {
    f = __fmul_rn(f, 0.5f);
    e += 1;
  }
  const float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
  const float s2 = __fmul_rn(s, s);
  float poly = 0x1.c71c72p-4f;                    // 1/9
  poly = __fmaf_rn(poly, s2, 0x1.24924ap-3f);     // 1/7
  poly = __fmaf_rn(poly, s2, 0x1.99999ap-3f);     // 1/5
  poly = __fmaf_rn(poly, s2, 0x1.555556p-2f);     // 1/3
  const float s3 = __fmul_rn(s, s2);
  float lnf = __fmaf_rn(s3, poly, s);
  lnf = __fmul_rn(2.0f, lnf);
  const float kf = __int2float_rn(e - 24);
  return __fmaf_rn(kf, 0x1.62e4p-1f, __fmaf_rn(kf, 0x1.7f7d1cp-20f, lnf));
}

// sin and cos of 2 pi v, v from the top 25 bits of r: quadrant from the top
// two bits, the in-quadrant angle folded into (0, pi/4], Taylor series of
// sin through x^9 and cos through x^10 by Horner with fma.
__device__ __forceinline__ void sincos_2pi(uint32_t r, float* sp, float* cp) {
  const uint32_t quad = r >> 30;
  uint32_t m = (((r >> 7) & 0x7FFFFFu) << 1) | 1u;
  const bool comp = m > (1u << 23);
  if (comp) m = (1u << 24) - m;
  const float t = __fmul_rn(__uint2float_rn(m), 0x1p-24f);
  const float x = __fmul_rn(t, 0x1.921fb6p+0f);  // pi/2
  const float x2 = __fmul_rn(x, x);
  float ps = 0x1.71de3ap-19f;                      // 1/9!
  ps = __fmaf_rn(ps, x2, -0x1.a01a02p-13f);        // -1/7!
  ps = __fmaf_rn(ps, x2, 0x1.111112p-7f);          // 1/5!
  ps = __fmaf_rn(ps, x2, -0x1.555556p-3f);         // -1/3!
  const float x3 = __fmul_rn(x, x2);
  float sn = __fmaf_rn(x3, ps, x);
  float pc = -0x1.27e4fcp-22f;                     // -1/10!
  pc = __fmaf_rn(pc, x2, 0x1.a01a02p-16f);         // 1/8!
  pc = __fmaf_rn(pc, x2, -0x1.6c16c2p-10f);        // -1/6!
  pc = __fmaf_rn(pc, x2, 0x1.555556p-5f);          // 1/4!
  pc = __fmaf_rn(pc, x2, -0x1p-1f);                // -1/2
  float cs = __fmaf_rn(x2, pc, 1.0f);
  if (comp) {
    const float tmp = sn;
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

// standard normal of degree of freedom `dof`: key (seed lo, seed hi),
// counter (step, stage, dof/4 lo, dof/4 hi); lanes 0,1 from outputs (0,1),
// lanes 2,3 from outputs (2,3); even lanes cosine, odd lanes sine.
__device__ __forceinline__ float gauss_dof(uint64_t seed, uint32_t step, uint32_t stage, uint64_t dof) {
  const uint64_t g = dof >> 2;
  const int lane = (int)(dof & 3u);
  const uint4 o = philox4x32_10(make_uint4(step, stage, (uint32_t)g, (uint32_t)(g >> 32)),
                                make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
  const uint32_t ra = (lane >> 1) ? o.z : o.x;
  const uint32_t rb = (lane >> 1) ? o.w : o.y;
  const float lg = log_u24(ra);
  const float rho = __fsqrt_rn(__fmul_rn(-2.0f, lg));
  float sn, cs;
  sincos_2pi(rb, &sn, &cs);
  return __fmul_rn(rho, (lane & 1) ? sn : cs);
}

// kernel launchers (defined in the .cu files); each returns the number of
// kernels it launched
int launch_nlist(const Dev& d, cudaStream_t s, const int* atom_is_pseudo);
int launch_pair(const Dev& d, cudaStream_t s);
int launch_bonded(const Dev& d, cudaStream_t s, const AtomInfo* ainfo_atom);
int launch_pseudo(const Dev& d, cudaStream_t s);
// side / ev_fork / ev_join (optional): a second stream for the large-P
// clusters, forked from and joined back into s with the two events
int launch_prop(const Dev& d, cudaStream_t s, int mode, cudaStream_t side = nullptr, cudaEvent_t ev_fork = nullptr,
                cudaEvent_t ev_join = nullptr);
int launch_final(const Dev& d, cudaStream_t s, int mode, const int* slot_type);
int launch_forces_out(const Dev& d, cudaStream_t s);
size_t pair64_smem(const Dev& d);  // dynamic shared memory of the FP64 pair sweep
void pair_grids(int nt, size_t smem64, int nint, int* g64, int* g32);
void pair32w_plan(Dev& d);  // FP32 window sweep geometry (sets d.p32w)
int launch_gauss(const Dev& d, cudaStream_t s, uint32_t step, uint32_t stage, uint64_t dof0, long n, float* out);
int launch_ewald(const Dev& d, cudaStream_t s);

// ---------------------------------------------------------------------------
// Batched launches: one kernel launch serves the blocks of many systems. The
// host stores the members' Dev records in device memory and, per kernel, the
// prefix of the members' block counts; a block finds its member by binary
// search, copies that member's Dev into shared memory and runs the same
// kernel body as a single-system launch with its block index inside the
// member's grid.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int batch_member(const int* pfx, int nm, int b) {
  int lo = 0, hi = nm - 1;  // largest m with pfx[m] <= b
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pfx[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

#define MX_BATCH_ENTER()                                                                   \
  __shared__ __align__(16) int bdev_raw_[sizeof(Dev) / sizeof(int)];                       \
  __shared__ int bdev_m_, bdev_bx_;                                                        \
  if (threadIdx.x == 0) {                                                                  \
    const int m_ = batch_member(pfx, nm, (int)blockIdx.x);                                 \
    bdev_m_ = m_;                                                                          \
    bdev_bx_ = (int)blockIdx.x - pfx[m_];                                                  \
  }                                                                                        \
  __syncthreads();                                                                         \
  {                                                                                        \
    const int* src_ = (const int*)(devs + bdev_m_);                                        \
    for (int x_ = threadIdx.x; x_ < (int)(sizeof(Dev) / sizeof(int)); x_ += blockDim.x)    \
      bdev_raw_[x_] = src_[x_];                                                            \
  }                                                                                        \
  __syncthreads();                                                                         \
  const Dev& d = *(const Dev*)bdev_raw_;                                                   \
  const int bx = bdev_bx_

// per-kernel block-count prefixes of a batched launch (rows of nm + 1 ints)
enum : int { BK_PREP = 0, BK_NLIST, BK_PAIRA, BK_PAIRB, BK_BONDED, BK_PROP, BK_FINAL, BK_KINDS };

struct BatchGeom {
  const Dev* devs;   // device [nm]
  const int* pfx;    // device [BK_KINDS][nm + 1]
  int nm;
  int blocks[BK_KINDS];  // total blocks per kind
  size_t prop_smem, pair_smem;
  int precision;
};

// propagation (parts bit 1) and finalisation (bit 2) of every member
int launch_step_batched(const BatchGeom& g, cudaStream_t s, int mode, int parts = 3);
int launch_forces_batched(const BatchGeom& g, cudaStream_t s);           // list, pair sweep, bonded
int launch_forces_batched_part(const BatchGeom& g, cudaStream_t s, int part);  // 0 list, 1 pair, 2 bonded
void batch_block_counts(const Dev& d, int* counts);                       // BK_KINDS blocks of one member
size_t batch_prop_smem(const Dev& d);
// largest cluster size <= cl_max that the device co-schedules for the
// large-P tile kernel (tiles of the n (P, atoms) shapes given), with its
// per-CTA shared memory in *smem; 0 when none does
int big_cluster_pick(int cl_max, const int* P, const int* na, int n, int* smem);

// propagation modes
enum : int {
  PM_END = 1,      // finish a step: B(dt/2), O(dt/2) stage 1
  PM_START = 2,    // begin a step: O(dt/2) stage 0, B(dt/2), A(dt)
  PM_EST = 4,      // estimator partials of the finished step
  PM_PCART = 8,    // write Cartesian momenta to the caller
  PM_QCART = 16,   // write Cartesian positions and force mirrors from q_nm
  PM_IMPORT = 32,  // q_nm, p_nm <- C^T (caller q, p) before anything else
  PM_MIRROR = 64,  // mirrors from the caller's q, mode-space state untouched
};

}  // namespace mx
