// Fused multiply-add throughput of the device in FP32 and FP64, the
// denominators of the ALU roofline that the FP64 path (bound by the FP64
// units, not by HBM) is reported against.  Measurement support; the paper has
// no counterpart.
#include "wf_api_internal.h"

// Every thread runs WF_PEAK_CHAINS independent chains x <- x a + b for `iters`
// steps (2 flops each); the chains' sum is stored only if it takes a value it
// cannot take (|x| stays below 2 for a < 1, b small), which keeps the
// arithmetic live without a memory stream.
#define WF_PEAK_CHAINS 8
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(T* sink, int iters, T a, T b) {
  T x[WF_PEAK_CHAINS];
#pragma unroll
  for (int i = 0; i < WF_PEAK_CHAINS; ++i) x[i] = (T)(threadIdx.x & 7) * (T)0.01 + (T)i * (T)0.1;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < WF_PEAK_CHAINS; ++i) x[i] = fma(x[i], a, b);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < WF_PEAK_CHAINS; ++i) s += x[i];
  if (s == (T)1e30) sink[0] = s;
}

template <typename T>
static wf_status alu_peak(double* flops_per_s) {
  int dev = 0, nsm = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fma_peak<T>, 256, 0);
  if (e != cudaSuccess) return wf_cuda_fail(e, "wf_alu_peak: device query");
  const int grid = nsm * (occ > 0 ? occ : 1);
  T* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc((void**)&sink, sizeof(T));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // a short run sizes the timed one to about 40 ms
  int iters = sizeof(T) == 4 ? 4096 : 256;
  float ms = 0.f;
  for (int pass = 0; pass < 3 && e == cudaSuccess; ++pass) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      k_fma_peak<T><<<grid, 256, 0, st>>>(sink, iters, (T)0.999999, (T)1e-7);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && pass < 2) {
      const double scale = 40.0 / (ms > 1e-3 ? ms : 1e-3);
      double next = iters * (scale > 64.0 ? 64.0 : scale);
      if (next > (1 << 26)) next = 1 << 26;
      if (next < 16) next = 16;
      iters = (int)next;
    }
  }
  if (e == cudaSuccess)
    *flops_per_s = 2.0 * WF_PEAK_CHAINS * (double)iters * grid * 256 / (ms * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  return e == cudaSuccess ? WF_OK : wf_cuda_fail(e, "wf_alu_peak");
}

extern "C" wf_status wf_alu_peak(int dtype, double* flops_per_s) {
  if (!flops_per_s) return wf_fail(WF_EINVAL, "wf_alu_peak: null output");
  if (dtype != WF_F32 && dtype != WF_F64) return wf_fail(WF_EINVAL, "wf_alu_peak: bad dtype %d", dtype);
  return dtype == WF_F64 ? alu_peak<double>(flops_per_s) : alu_peak<float>(flops_per_s);
}
