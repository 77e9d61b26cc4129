// k_corr.cu -- time correlation functions of ring-polymer molecular dynamics
// (Sec. "Output and Analysis": RPMD correlation functions from NVE
// trajectories): the centroid velocity autocorrelation of one atom type,
// accumulated on the device over every time origin of a trajectory.
//
// The centroid velocity of atom k of type t is dq̄/dt = (1/P) sum_b p_b / m_f
// = p_nm[mode 0] / (sqrt(P) m_f): the centroid mode of the orthonormal
// transform is (1/sqrt P) sum_b. Each call adds, for every lag L with a stored
// frame L calls back, sum_k v_k(now) . v_k(now - L) to acc[L] (one CTA per
// lag, fixed-order block reduction, so the sums are bitwise reproducible) and
// then stores the current velocities in the ring of the last n_lag frames.
#include "mixts_internal.cuh"

namespace mx {

constexpr int CORR_THREADS = 256;

__device__ __forceinline__ double centroid_velocity(const Dev& d, int t, double inv, int e) {
  return d.p_nm[(size_t)(d.off[t] + e / 3) * 3 + (e % 3)] * inv;
}

__global__ void __launch_bounds__(CORR_THREADS) k_vacf_acc(Dev d, int t, int n_lag, const double* ring,
                                                            double* acc, unsigned long long* cnt) {
  __shared__ double red[CORR_THREADS / 32];
  const int L = blockIdx.x;
  const long long n0 = (long long)cnt[0];  // frames added before this call
  if ((long long)L > n0) return;
  const int n3 = 3 * d.N[t];
  const double inv = 1.0 / (sqrt((double)d.P[t]) * d.mass[t]);
  const double* old = ring + (size_t)((n0 - L) % n_lag) * n3;
  double sum = 0.0;
  for (int e = threadIdx.x; e < n3; e += CORR_THREADS) {
    const double v = centroid_velocity(d, t, inv, e);
    sum = fma(v, L == 0 ? v : old[e], sum);
  }
  sum = warp_sum(sum);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < CORR_THREADS / 32; ++w) s += red[w];
    acc[L] += s;
    if (L > 0) cnt[L] += 1ull;
  }
}

// one CTA: store the current frame in ring slot (frames so far) mod n_lag,
// then count the frame
__global__ void __launch_bounds__(1024) k_vacf_push(Dev d, int t, int n_lag, double* ring, unsigned long long* cnt) {
  const long long n0 = (long long)cnt[0];
  const int n3 = 3 * d.N[t];
  const double inv = 1.0 / (sqrt((double)d.P[t]) * d.mass[t]);
  double* dst = ring + (size_t)(n0 % n_lag) * n3;
  for (int e = threadIdx.x; e < n3; e += blockDim.x) dst[e] = centroid_velocity(d, t, inv, e);
  __syncthreads();
  if (threadIdx.x == 0) cnt[0] = (unsigned long long)(n0 + 1);
}

int launch_vacf(const Dev& d, cudaStream_t s, int t, int n_lag, double* ring, double* acc, unsigned long long* cnt) {
  k_vacf_acc<<<n_lag, CORR_THREADS, 0, s>>>(d, t, n_lag, ring, acc, cnt);
  k_vacf_push<<<1, 1024, 0, s>>>(d, t, n_lag, ring, cnt);
  return 2;
}

}  // namespace mx
