// k_probe.cu -- ALU peak probe for the roofline denominators: a grid of
// independent fused multiply-add chains in binary32 or binary64, timed with
// CUDA events. Not part of the method; it measures the pipe the pair sweeps
// are bound by, at the clocks the GPU runs at when the probe runs.
#include <stdio.h>

#include "mixts_internal.cuh"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 16;  // independent chains per thread (hides the FMA latency)

// written only when a chain ends on a value no input can produce, which keeps
// the compiler from dropping the chains; never read by the library
__device__ double g_probe_sink[2];

template <class T>
__global__ void __launch_bounds__(PROBE_THREADS) k_fma_chain(int iters, T a, T b) {
  T x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
  if (s == (T)-1.2345e-30) g_probe_sink[sizeof(T) == 8] = (double)s;
}

}  // namespace

extern "C" MIXTS_API mixts_status mixts_alu_probe(int fp64, int iters, void* stream, double* flop_out,
                                                  double* ms_out) {
  if (iters < 1 || !flop_out || !ms_out) return MIXTS_ERR_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MIXTS_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  if (fp64)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chain<double>, PROBE_THREADS, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chain<float>, PROBE_THREADS, 0);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return MIXTS_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MIXTS_ERR_CUDA;
  }
  // one untimed launch brings the clocks up, then the timed one
  for (int rep = 0; rep < 2; ++rep) {
    if (rep == 1) cudaEventRecord(e0, s);
    if (fp64)
      k_fma_chain<double><<<grid, PROBE_THREADS, 0, s>>>(iters, 0.9999999, 1e-7);
    else
      k_fma_chain<float><<<grid, PROBE_THREADS, 0, s>>>(iters, 0.9999f, 1e-4f);
  }
  cudaEventRecord(e1, s);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess || cudaGetLastError() != cudaSuccess) return MIXTS_ERR_CUDA;
  *flop_out = 2.0 * (double)grid * PROBE_THREADS * PROBE_CHAINS * (double)iters;
  *ms_out = ms;
  return MIXTS_OK;
}
