// k_rdf.cu -- radial distribution histogram of two site types (Sec. "Output
// and Analysis"): every listed atom pair on its fine slice grid, weight
// 1/max(P_i, P_j), binned by bead distance.
//
// The weights are dyadic, so the histogram is kept in integers: a term of
// grid P* adds 2^(L - log2 P*), L = log2 of the largest site bead count. A
// CTA bins into shared memory and flushes once; integer sums make the result
// independent of the order the atomics land in.
#include <math.h>

#include "mixts_internal.cuh"

namespace mx {

constexpr int RDF_THREADS = 256;

// (owner position, owner bead) of pair item w, items ordered by class
__device__ __forceinline__ void rdf_item(const Dev& d, int w, int* pos, int* bead) {
  int c = 0;
  while (c + 1 < d.n_classes && w >= d.cls_item0[c + 1]) ++c;
  const int local = w - d.cls_item0[c];
  *bead = local / d.cls_n[c];
  *pos = d.cls_pos0[c] + (local - *bead * d.cls_n[c]);
}

__global__ void __launch_bounds__(RDF_THREADS) k_rdf(Dev d, int ta, int tb, double dr, int nbins,
                                                      unsigned long long* hist) {
  extern __shared__ unsigned long long sh[];
  __shared__ int tN[MT], tLg[MT], tOff[MT], tAt[MT];
  for (int e = threadIdx.x; e < nbins; e += blockDim.x) sh[e] = 0ull;
  for (int e = threadIdx.x; e < d.n_types; e += blockDim.x) {
    tN[e] = d.N[e];
    tLg[e] = d.log2P[e];
    tOff[e] = d.off[e];
    tAt[e] = d.atoff[e];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const double rmax = nbins * dr;
  const unsigned long long mult = ta == tb ? 2ull : 1ull;  // ordered pairs
  for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < d.n_pitems; w += nwarps) {
    int pos, b;
    rdf_item(d, w, &pos, &b);
    const AtomInfo ai = d.ainfo[pos];
    const int ti = ai.type;
    if (ti != ta && ti != tb) continue;
    const int want = ti == ta ? tb : ta;
    const double4_32a xi = d.Xw[ai.row0 + b * ai.stride];
    const unsigned long long unit = mult << (d.lgPmax_nb - ai.log2P);
    const int cnt = min(d.nl_cnt[pos], d.nl_cap);
    const int* lst = d.nl + (size_t)pos * d.nl_cap;
    for (int e = lane; e < cnt; e += 32) {
      const int ent = lst[e];
      const int tj = (ent >> 7) & 15;
      if (tj != want) continue;
      const int row0 = ent >> 11;
      if (d.full_list) {  // each unordered pair once: the half-list owner rule
        const int pj = d.pos_of_atom[d.atom_of_tk[tAt[tj] + (row0 - tOff[tj])]];
        bool own;
        if (ai.log2P != tLg[tj]) {
          own = ai.log2P > tLg[tj];
        } else {
          const int lo = pos < pj ? pos : pj;
          own = (((pos + pj) & 1) == 0) ? (pos == lo) : (pos != lo);
        }
        if (!own) continue;
      }
      const double4_32a xj = d.Xw[row0 + (b >> (ai.log2P - tLg[tj])) * tN[tj]];
      const int code = ent & 127;
      const double dx = (xj.x - xi.x) + (code / 25 - 2) * d.box;
      const double dy = (xj.y - xi.y) + ((code / 5) % 5 - 2) * d.box;
      const double dz = (xj.z - xi.z) + (code % 5 - 2) * d.box;
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      if (!(r < rmax)) continue;
      const int k = (int)floor(r / dr);
      if (k < nbins) atomicAdd(&sh[k], unit);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nbins; e += blockDim.x)
    if (sh[e]) atomicAdd(hist + e, sh[e]);
}

int launch_rdf(const Dev& d, cudaStream_t s, int ta, int tb, double dr, int nbins, unsigned long long* hist) {
  if (d.n_pitems == 0) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int wpb = RDF_THREADS / 32;
  const int grid = min((d.n_pitems + wpb - 1) / wpb, 4 * sms);
  k_rdf<<<grid, RDF_THREADS, sizeof(unsigned long long) * (size_t)nbins, s>>>(d, ta, tb, dr, nbins, hist);
  return 1;
}

}  // namespace mx
