// Allocation-free objective + gradient pass.
//
// Who needs it: a caller whose device memory is owned by someone else (a
// framework's caching allocator or a pool reserved at start-up) or whose
// real-time rules forbid allocation after initialisation cannot call
// cudaMalloc, yet wf_problem_create allocates the prepared inputs and the
// operator's scratch.  wf_eval_noalloc runs the same three operator kernels
// on caller-prepared inputs and keeps its scratch (twiddle tables, sqrt(P)/n,
// partial sums and the intermediate spectra) in the file-scope device array
// below, which every GPU that loads the library holds until the process exits.
//
// Layout of the array: FP64 twiddle tables (176 KiB), FP32 twiddle tables
// (88 KiB), then the sqrt(P)/n table, the partial sums and the intermediate
// spectra, each starting on a 256-byte boundary.
#include <mutex>

#include "wf_api_internal.h"

#define WF_NOALLOC_BYTES (16u << 20)  // 16 MiB per device
#define WF_NOALLOC_TW64 0
#define WF_NOALLOC_TW32 (WF_TWTAB * sizeof(double2))
#define WF_NOALLOC_DATA (WF_NOALLOC_TW32 + WF_TWTAB * sizeof(float2))
#define WF_NOALLOC_MAXDEV 64

static __device__ __align__(256) unsigned char wf_noalloc_scratch[WF_NOALLOC_BYTES];

static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_ptr[WF_NOALLOC_MAXDEV];

// Device address of the array on the current device; the first call on a
// device resolves it, writes the twiddle tables and waits until they have
// landed.  The address and the tables are cached per device for the life of
// the process, so a cudaDeviceReset after that first call is not supported
// (the module's static array would come back zeroed, perhaps elsewhere).
static wf_status noalloc_setup(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev]) {
    *out = g_noalloc_ptr[dev];
    return WF_OK;
  }
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, wf_noalloc_scratch);
  if (e != cudaSuccess) return wf_cuda_fail(e, "wf_eval_noalloc: cudaGetSymbolAddress of the static scratch");
  static double2 tw64[WF_TWTAB];  // host staging (guarded by the mutex)
  static float2 tw32[WF_TWTAB];
  wf_make_twiddles(tw64);
  for (int k = 0; k < WF_TWTAB; ++k) {
    tw32[k].x = (float)tw64[k].x;
    tw32[k].y = (float)tw64[k].y;
  }
  e = cudaMemcpy((unsigned char*)ptr + WF_NOALLOC_TW64, tw64, sizeof tw64, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy((unsigned char*)ptr + WF_NOALLOC_TW32, tw32, sizeof tw32, cudaMemcpyHostToDevice);
  // A pageable host-to-device cudaMemcpy may return before its DMA into device
  // memory has finished, and the kernels run on the caller's stream, which
  // need not be ordered after the legacy default stream (a non-blocking or
  // per-thread stream): wait for the copies before the tables are published.
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
  if (e != cudaSuccess) return wf_cuda_fail(e, "wf_eval_noalloc: writing the twiddle tables");
  g_noalloc_ptr[dev] = (unsigned char*)ptr;
  *out = g_noalloc_ptr[dev];
  return WF_OK;
}

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// sqrt(P)/n in the working type (computed in double, as the prepared path does).
template <typename T>
__global__ void k_noalloc_sqrtp(const T* P, size_t total, int n, T* sp) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const double p = (double)P[i];
    sp[i] = (T)(p > 0.0 ? sqrt(p) / (double)n : 0.0);
  }
}

template <typename T>
static wf_status noalloc_impl(unsigned char* base, const void* s, const void* d, const void* w, const void* P,
                              int n, int C, int count, double* chi2, void* grad, cudaStream_t st) {
  const WfGeo g = wf_make_geo(n, C);
  const size_t elt = sizeof(T);
  const size_t nsp = (size_t)C * n * (n / 2 + 1);
  const size_t off_sp = WF_NOALLOC_DATA;
  const size_t off_part = off_sp + up256(nsp * elt);
  const size_t off_scr = off_part + up256(sizeof(double) * WF_NSLOT * g.maxblk * (size_t)count);
  const size_t need = off_scr + (size_t)count * C * n * n * elt;
  if (need > WF_NOALLOC_BYTES)
    return wf_fail(WF_EINVAL,
                   "wf_eval_noalloc: n = %d, C = %d, count = %d needs %zu bytes of scratch; the static "
                   "scratch holds %u bytes (use wf_problem_create for larger batches)",
                   n, C, count, need, (unsigned)WF_NOALLOC_BYTES);
  T* sp = (T*)(base + off_sp);
  int blocks = (int)((nsp + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  k_noalloc_sqrtp<T><<<blocks, 256, 0, st>>>((const T*)P, nsp, n, sp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return wf_cuda_fail(e, "wf_eval_noalloc: sqrt(P) table");
  WfBufs b;
  b.d = d;
  b.w = w;
  b.sp = sp;
  b.sp_stride = 0;
  b.scratch = base + off_scr;
  b.part = (double*)(base + off_part);
  b.tw = base + (sizeof(T) == 8 ? WF_NOALLOC_TW64 : WF_NOALLOC_TW32);
  b.ticket = nullptr;
  b.B = count;
  e = wf_launch_eval<T>(g, b, WF_ROW_DATA, WF_IN_STD, s, grad, chi2, st);
  return e == cudaSuccess ? WF_OK : wf_cuda_fail(e, "wf_eval_noalloc");
}

extern "C" wf_status wf_eval_noalloc(const void* s, const void* d, const void* w, const void* P, int n, int C,
                                     int count, int precision, double* chi2, void* grad, void* stream) {
  if (!s || !d || !w || !P || !chi2 || !grad) return wf_fail(WF_EINVAL, "wf_eval_noalloc: null argument");
  if (s == grad) return wf_fail(WF_EINVAL, "wf_eval_noalloc: s and grad must not alias");
  if (n < 8 || n > WF_NT || (n & (n - 1)))
    return wf_fail(WF_EINVAL, "wf_eval_noalloc: n = %d is not a power of two in [8, %d]", n, WF_NT);
  if (C != 1 && C != 2) return wf_fail(WF_EINVAL, "wf_eval_noalloc: C = %d (must be 1 or 2)", C);
  if (count < 1) return wf_fail(WF_EINVAL, "wf_eval_noalloc: count = %d", count);
  if (precision != WF_FP64 && precision != WF_MIXED)
    return wf_fail(WF_EINVAL, "wf_eval_noalloc: bad precision %d", precision);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return wf_cuda_fail(e, "wf_eval_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= WF_NOALLOC_MAXDEV) return wf_fail(WF_EINVAL, "wf_eval_noalloc: device %d", dev);
  unsigned char* base = nullptr;
  wf_status rs = noalloc_setup(dev, &base);
  if (rs != WF_OK) return rs;
  cudaStream_t st = (cudaStream_t)stream;
  return precision == WF_FP64 ? noalloc_impl<double>(base, s, d, w, P, n, C, count, chi2, grad, st)
                              : noalloc_impl<float>(base, s, d, w, P, n, C, count, chi2, grad, st);
}

WF_DBG_READER(noalloc)
