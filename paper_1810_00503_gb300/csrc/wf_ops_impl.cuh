// Host-side launchers of the operator kernels, instantiated once per working
// type by wf_ops_f32.cu and wf_ops_f64.cu.
#pragma once
#include "wf_lbfgs.cuh"

namespace wfimpl {

// Shared memory of the in-place stages: the pass tables and the tile (a full
// WF_TILE in the bounds-checked build, where tile indices are checked against
// WF_TILE).
#ifdef WF_DEBUG_BOUNDS
template <typename T> inline size_t col_smem(const WfGeo&) { return (WF_NT + (size_t)WF_TILE) * sizeof(V2<T>); }
template <typename T> inline size_t row_smem(const WfGeo&) { return (2 * WF_NT + (size_t)WF_TILE) * sizeof(V2<T>); }
#else
template <typename T> inline size_t col_smem(const WfGeo& g) {
  return (WF_NT + (size_t)g.C * g.TC * g.n) * sizeof(V2<T>);
}
template <typename T> inline size_t row_smem(const WfGeo& g) {
  return (2 * WF_NT + (size_t)g.RB * g.h) * sizeof(V2<T>);
}
#endif

// Raise the dynamic shared-memory limit of a kernel once per device.
template <typename K> inline cudaError_t ensure_smem(K kernel, size_t bytes, int* done_mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 32 && (*done_mask >> dev) & 1) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wf_pp_smem<double>());
  if (e == cudaSuccess && dev < 32) *done_mask |= 1 << dev;
  (void)bytes;
  return e;
}

// Resident blocks of a persistent kernel: SMs x blocks per SM (cached per device).
template <typename K>
inline cudaError_t persistent_grid(K k, size_t smem, int* occ, int* nsm, int* grid) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int di = dev & 31;
  if (!occ[di]) {
    int o = 0, ns = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, WF_THREADS, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ns, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    occ[di] = o > 0 ? o : 1;
    nsm[di] = ns;
  }
  *grid = occ[di] * nsm[di];
  return cudaSuccess;
}

// Grid of a persistent launch over nitems work items: the resident blocks, at
// most nitems (the items loop inside the kernel, so any grid is correct).
template <typename K>
inline cudaError_t items_grid(K k, size_t smem, int nitems, int* occ, int* nsm, int* grid) {
  cudaError_t e = persistent_grid(k, smem, occ, nsm, grid);
  if (e == cudaSuccess && *grid > nitems) *grid = nitems;
  return e;
}

template <typename T, int C, int IN, int PLAN>
cudaError_t col_inv_r(const WfGeo& g, const WfBufs& b, const void* src, cudaStream_t st) {
  static int done = 0;
  if constexpr (WF_FFT_PP && WF_COLINV_QUEUE) {
    if (b.ticket) {
      static int occq[32] = {0}, nsmq[32] = {0}, doneq = 0;
      auto k = k_col_inv_pp_q<T, C, IN, PLAN>;
      const size_t sm = wf_pp_smem<T>();
      cudaError_t e = ensure_smem(k, sm, &doneq);
      int grid = 0;
      if (e == cudaSuccess) e = items_grid(k, sm, g.ntile * b.B, occq, nsmq, &grid);
      if (e == cudaSuccess) e = cudaMemsetAsync(b.ticket, 0, sizeof(int), st);
      if (e != cudaSuccess) return e;
      k<<<grid, WF_THREADS, sm, st>>>(g, src, (const T*)b.sp, b.sp_stride, b.scratch, b.tw, b.B, b.ticket);
      return cudaGetLastError();
    }
  }
  if constexpr (WF_FFT_PP) {
    static int occ[32] = {0}, nsm[32] = {0};
    auto k = k_col_inv_pp_pers<T, C, IN, PLAN>;
    const size_t sm = wf_pp_smem<T>();
    cudaError_t e = ensure_smem(k, sm, &done);
    int grid = 0;
    if (e == cudaSuccess) e = items_grid(k, sm, g.ntile * b.B, occ, nsm, &grid);
    if (e != cudaSuccess) return e;
    k<<<grid, WF_THREADS, sm, st>>>(g, src, (const T*)b.sp, b.sp_stride, b.scratch, b.tw, b.B);
    return cudaGetLastError();
  } else {
    auto k = k_col_inv<T, C, IN>;
    const size_t sm = col_smem<T>(g);
    cudaError_t e = ensure_smem(k, sm, &done);
    if (e != cudaSuccess) return e;
    k<<<dim3(g.ntile, b.B), WF_THREADS, sm, st>>>(g, src, (const T*)b.sp, b.sp_stride, b.scratch, b.tw);
    return cudaGetLastError();
  }
}

template <typename T, int C, int IN>
cudaError_t col_inv(const WfGeo& g, const WfBufs& b, const void* src, cudaStream_t st) {
  switch (wf_plan_eff(g.lgn, g.col_plan)) {
    case 1: return col_inv_r<T, C, IN, 1>(g, b, src, st);
    case 2: return col_inv_r<T, C, IN, 2>(g, b, src, st);
    default: return col_inv_r<T, C, IN, 0>(g, b, src, st);
  }
}

template <typename T, int C, int IN>
cudaError_t col_fwd(const WfGeo& g, const WfBufs& b, const void* src, void* dst, cudaStream_t st) {
  static int done = 0;
  auto k = k_col_fwd<T, C, IN>;
  const size_t sm = col_smem<T>(g);
  cudaError_t e = ensure_smem(k, sm, &done);
  if (e != cudaSuccess) return e;
  k<<<dim3(g.ntile, b.B), WF_THREADS, sm, st>>>(g, src, (const T*)b.sp, b.sp_stride, b.scratch, dst,
                                                b.part, b.tw);
  return cudaGetLastError();
}

// Deterministic band sums of standard-layout spectra (k_band_reduce, then
// k_band_final); bpart holds B * wf_band_nblk(g) * nb doubles.
template <typename T, int MODE>
cudaError_t band_sums(const WfGeo& g, int B, const void* s, const void* grad, const int16_t* band, int nb,
                      const double* theta, double* bpart, double* out, cudaStream_t st) {
  const int nblk = wf_band_nblk(g);
  const size_t sm = sizeof(double) * (WF_THREADS / 32) * (size_t)nb;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_band_reduce<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_band_reduce<T, MODE><<<dim3(nblk, B), WF_THREADS, sm, st>>>(g, (const V2<T>*)s, (const V2<T>*)grad, band, nb,
                                                                bpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_band_final<<<B, 128, 0, st>>>(bpart, nblk, nb, theta, out);
  return cudaGetLastError();
}

template <typename T, int C>
cudaError_t col_sim(const WfGeo& g, const WfBufs& b, cudaStream_t st) {
  static int done = 0;
  auto k = k_col_sim<T, C>;
  const size_t sm = col_smem<T>(g);
  cudaError_t e = ensure_smem(k, sm, &done);
  if (e != cudaSuccess) return e;
  k<<<dim3(g.ntile, b.B), WF_THREADS, sm, st>>>(g, (const T*)b.sp, b.sp_stride, b.scratch, b.tw);
  return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t row(const WfGeo& g, const WfBufs& b, const void* aux, void* out, cudaStream_t st) {
  static int done = 0;
  if constexpr (WF_FFT_PP && (MODE == WF_ROW_DATA || MODE == WF_ROW_NODATA)) {
    static int done_pp[WF_NPLAN] = {0};
    const int pl = wf_plan_eff(g.lgh, g.row_plan);
    auto k = pl == 1 ? k_row_pp<T, MODE, 1> : pl == 2 ? k_row_pp<T, MODE, 2> : k_row_pp<T, MODE, 0>;
    const size_t sm = wf_pp_smem<T>();
    cudaError_t e = ensure_smem(k, sm, &done_pp[pl]);
    if (e != cudaSuccess) return e;
    k<<<dim3(g.nrb, b.B), WF_THREADS, sm, st>>>(g, b.scratch, b.d, b.w, b.part, b.tw);
    return cudaGetLastError();
  }
  auto k = k_row<T, MODE>;
  const size_t sm = row_smem<T>(g);
  cudaError_t e = ensure_smem(k, sm, &done);
  if (e != cudaSuccess) return e;
  k<<<dim3(g.nrb, b.B), WF_THREADS, sm, st>>>(g, b.scratch, b.d, b.w, aux, out, b.part, b.tw);
  return cudaGetLastError();
}

template <typename T>
cudaError_t row_any(int mode, const WfGeo& g, const WfBufs& b, const void* aux, void* out,
                    cudaStream_t st) {
  switch (mode) {
    case WF_ROW_DATA: return row<T, WF_ROW_DATA>(g, b, aux, out, st);
    case WF_ROW_NODATA: return row<T, WF_ROW_NODATA>(g, b, aux, out, st);
    case WF_ROW_SIGNAL: return row<T, WF_ROW_SIGNAL>(g, b, aux, out, st);
    case WF_ROW_SIM: return row<T, WF_ROW_SIM>(g, b, aux, out, st);
    case WF_ROW_RFFT: return row<T, WF_ROW_RFFT>(g, b, aux, out, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t col_inv_any(const WfGeo& g, const WfBufs& b, int in, const void* src, cudaStream_t st) {
  if (g.C == 1) return in == WF_IN_PK ? col_inv<T, 1, WF_IN_PK>(g, b, src, st) : col_inv<T, 1, WF_IN_STD>(g, b, src, st);
  return in == WF_IN_PK ? col_inv<T, 2, WF_IN_PK>(g, b, src, st) : col_inv<T, 2, WF_IN_STD>(g, b, src, st);
}

template <typename T>
cudaError_t col_fwd_any(const WfGeo& g, const WfBufs& b, int in, const void* src, void* dst,
                        cudaStream_t st) {
  if (g.C == 1)
    return in == WF_IN_PK ? col_fwd<T, 1, WF_IN_PK>(g, b, src, dst, st) : col_fwd<T, 1, WF_IN_STD>(g, b, src, dst, st);
  return in == WF_IN_PK ? col_fwd<T, 2, WF_IN_PK>(g, b, src, dst, st) : col_fwd<T, 2, WF_IN_STD>(g, b, src, dst, st);
}

template <typename K> inline cudaError_t ensure_smem_n(K kernel, size_t bytes, int* done_mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 32 && (*done_mask >> dev) & 1) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess && dev < 32) *done_mask |= 1 << dev;
  return e;
}

// cuTensorMapEncodeTiled, fetched from the driver once (no link to libcuda).
typedef CUresult (*WfEncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
inline WfEncodeTiled wf_encode_fn() {
  static WfEncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (WfEncodeTiled)p;
  }
  return fn;
}

// Persistent TMA-fed inverse column stage (k_lb_colinv_tma).
template <typename T, int C, int PLAN>
cudaError_t lb_colinv_tma(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st) {
  static int done = 0;
  static int occ[32] = {0}, nsm[32] = {0};
  auto k = k_lb_colinv_tma<T, C, PLAN>;
  const size_t sm = wf_colinv_tma_smem<T>();
  cudaError_t e = ensure_smem_n(k, sm, &done);
  if (e != cudaSuccess) return e;
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const int di = dev & 31;
  if (!occ[di]) {
    int o = 0, ns = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, WF_THREADS, sm);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ns, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    occ[di] = o > 0 ? o : 1;
    nsm[di] = ns;
  }
  WfEncodeTiled enc = wf_encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const int rows = C * g.n;
  CUtensorMap tm;
  const cuuint64_t dims[2] = {(cuuint64_t)2 * g.h, (cuuint64_t)2 * lb.m * b.B * rows};
  const cuuint64_t strides[1] = {(cuuint64_t)2 * g.h * sizeof(T)};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * g.TC), (cuuint32_t)(rows < 256 ? rows : 256)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(&tm, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                         lb.ring, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  int grid = nsm[di] * occ[di];
  const int nitems = b.B * g.ntile;
  if (grid > nitems) grid = nitems;
  k<<<grid, WF_THREADS, sm, st>>>(g, (const T*)b.sp, b.sp_stride, b.scratch, b.tw, lb, b.B, tm);
  return cudaGetLastError();
}


template <typename T, int C, int KIND, int PLAN>
cudaError_t lb_colinv_tile(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st) {
  static int done = 0;
  auto k = k_lb_colinv<T, C, KIND, PLAN>;
  const size_t sm = KIND == WF_COLINV_PP_K ? wf_pp_smem<T>() : col_smem<T>(g);
  cudaError_t e = ensure_smem(k, sm, &done);
  if (e != cudaSuccess) return e;
  k<<<dim3(g.ntile, b.B), WF_THREADS, sm, st>>>(g, (const T*)b.sp, b.sp_stride, b.scratch, b.tw, lb);
  return cudaGetLastError();
}

// The variant in g.colinv_kind (the TMA form needs the driver's tensor-map
// encoder; without it the ping-pong form runs).
template <typename T, int C>
cudaError_t lb_colinv(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st) {
  const int pl = wf_plan_eff(g.lgn, g.col_plan);
  if (g.colinv_kind == WF_COLINV_TMA_K && wf_encode_fn())
    return pl == 1 ? lb_colinv_tma<T, C, 1>(g, b, lb, st)
           : pl == 2 ? lb_colinv_tma<T, C, 2>(g, b, lb, st) : lb_colinv_tma<T, C, 0>(g, b, lb, st);
  if (g.colinv_kind == WF_COLINV_INPLACE_K) return lb_colinv_tile<T, C, WF_COLINV_INPLACE_K, 0>(g, b, lb, st);
  return pl == 1 ? lb_colinv_tile<T, C, WF_COLINV_PP_K, 1>(g, b, lb, st)
         : pl == 2 ? lb_colinv_tile<T, C, WF_COLINV_PP_K, 2>(g, b, lb, st)
                   : lb_colinv_tile<T, C, WF_COLINV_PP_K, 0>(g, b, lb, st);
}

template <typename T, int C>
cudaError_t lb_colfwd(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st) {
  static int done = 0;
  auto k = k_lb_colfwd<T, C>;
  const size_t sm = col_smem<T>(g);
  cudaError_t e = ensure_smem(k, sm, &done);
  if (e != cudaSuccess) return e;
  k<<<dim3(g.ntile, b.B), WF_THREADS, sm, st>>>(g, (const T*)b.sp, b.sp_stride, b.scratch, b.tw, lb, b.part);
  return cudaGetLastError();
}

inline int grid1d(size_t total, int cap) {
  size_t blocks = (total + 255) / 256;
  if (blocks > (size_t)cap) blocks = cap;
  return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace wfimpl

// Launcher definitions (explicitly instantiated per working type).
  template <typename T>
  cudaError_t wf_launch_prep(const WfGeo& g, const void* const* dptr,
                                const unsigned char* const* mptr, const void* const* nptr,
                                const void* const* pptr, int in_f64, int B, void* d, void* w,
                                void* sp, int sp_shared, int* flags, cudaStream_t st) {
    WfMapPtrs* hm = (WfMapPtrs*)malloc(sizeof(WfMapPtrs) * (size_t)B);
    if (!hm) return cudaErrorMemoryAllocation;
    for (int i = 0; i < B; ++i) hm[i] = WfMapPtrs{dptr[i], mptr[i], nptr[i], pptr[i]};
    WfMapPtrs* dm = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&dm, sizeof(WfMapPtrs) * (size_t)B, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dm, hm, sizeof(WfMapPtrs) * (size_t)B,
                                              cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
      const size_t npix = (size_t)g.C * g.n * g.nx;
      k_prep<T><<<dim3(wfimpl::grid1d(npix, 1024), B), 256, 0, st>>>(g, dm, in_f64, (T*)d, (T*)w,
                                                                     (T*)sp, sp_shared, flags);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (dm) cudaFreeAsync(dm, st);
    free(hm);
    return e;
  }
  template <typename T>
  cudaError_t wf_launch_set_data(const WfGeo& g, const void* src, int B, void* d,
                                    cudaStream_t st) {
    const size_t total = (size_t)B * g.C * g.n * g.nx;
    k_set_data<T><<<wfimpl::grid1d(total, 4096), 256, 0, st>>>(total, (const T*)src, (T*)d);
    return cudaGetLastError();
  }
  template <typename T>
  cudaError_t wf_launch_eval(const WfGeo& g, const WfBufs& b, int row_mode, int in_layout,
                                const void* src, void* dst, double* chi2, cudaStream_t st) {
    cudaError_t e = wfimpl::col_inv_any<T>(g, b, in_layout, src, st);
    if (e == cudaSuccess) e = wfimpl::row_any<T>(row_mode, g, b, nullptr, nullptr, st);
    if (e == cudaSuccess) e = wfimpl::col_fwd_any<T>(g, b, in_layout, src, dst, st);
    if (e == cudaSuccess && chi2) {
      k_finalize_chi2<<<b.B, WF_THREADS, 0, st>>>(b.part, g.maxblk, g.ntile,
                                                  row_mode == WF_ROW_DATA ? g.nrb : 0, chi2);
      e = cudaGetLastError();
    }
    return e;
  }
  template <typename T>
  cudaError_t wf_launch_signal(const WfGeo& g, const WfBufs& b, int in_layout, const void* src,
                                  void* xout, cudaStream_t st) {
    cudaError_t e = wfimpl::col_inv_any<T>(g, b, in_layout, src, st);
    if (e == cudaSuccess) e = wfimpl::row_any<T>(WF_ROW_SIGNAL, g, b, nullptr, xout, st);
    return e;
  }
  template <typename T>
  cudaError_t wf_launch_simulate(const WfGeo& g, const WfBufs& b, const void* z,
                                    const void* noise, void* dout, cudaStream_t st) {
    cudaError_t e = wfimpl::row_any<T>(WF_ROW_RFFT, g, b, z, nullptr, st);
    if (e == cudaSuccess)
      e = g.C == 1 ? wfimpl::col_sim<T, 1>(g, b, st) : wfimpl::col_sim<T, 2>(g, b, st);
    if (e == cudaSuccess) e = wfimpl::row_any<T>(WF_ROW_SIM, g, b, noise, dout, st);
    return e;
  }
  template <typename T>
  cudaError_t wf_launch_band_energy(const WfGeo& g, int B, const void* s, const int16_t* band,
                                       const double* theta, int n_bands, double* bpart, double* E,
                                       cudaStream_t st) {
    return wfimpl::band_sums<T, 0>(g, B, s, nullptr, band, n_bands, theta, bpart, E, st);
  }
  template <typename T>
  cudaError_t wf_launch_pack(const WfGeo& g, int B, const void* in, void* out,
                                cudaStream_t st) {
    const size_t total = (size_t)B * g.C * g.n * g.h;
    k_pack<T><<<wfimpl::grid1d(total, 4096), 256, 0, st>>>(g, B, (const V2<T>*)in, (V2<T>*)out);
    return cudaGetLastError();
  }
  template <typename T>
  cudaError_t wf_launch_unpack(const WfGeo& g, int B, const void* in, void* out,
                                  cudaStream_t st) {
    const size_t total = (size_t)B * g.C * g.n * g.h;
    k_unpack<T><<<wfimpl::grid1d(total, 4096), 256, 0, st>>>(g, B, (const V2<T>*)in,
                                                             (V2<T>*)out);
    return cudaGetLastError();
  }

template <typename T>
cudaError_t wf_launch_eval_bands(const WfGeo& g, const WfBufs& b, const void* src, void* dst, double* chi2,
                                 const int16_t* band, int n_b, double* bpart, double* dq, cudaStream_t st) {
  cudaError_t e = wf_launch_eval<T>(g, b, WF_ROW_DATA, WF_IN_STD, src, dst, chi2, st);
  if (e == cudaSuccess) e = wfimpl::band_sums<T, 1>(g, b.B, src, dst, band, n_b, nullptr, bpart, dq, st);
  return e;
}
template <typename T>
cudaError_t wf_launch_band_scale(const WfGeo& g, const void* sp0, void* sp, int ntab, const int16_t* band,
                                 const double* q, int n_b, cudaStream_t st) {
  const size_t nsp = (size_t)g.C * g.n * (g.h + 1);
  k_band_scale<T><<<wfimpl::grid1d(nsp * ntab, 4096), 256, 0, st>>>((const T*)sp0, (T*)sp, nsp, ntab, band, q,
                                                                     n_b);
  return cudaGetLastError();
}
template <typename T>
cudaError_t wf_launch_lb_comb(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, int mode, cudaStream_t st) {
  static int done = 0;
  auto k = k_lb_comb<T>;
  const size_t sm = wf_comb_smem<T>(lb.m);
  cudaError_t e = wfimpl::ensure_smem_n(k, wf_comb_smem<T>(WF_MAXM), &done);
  if (e != cudaSuccess) return e;
  k<<<dim3(g.ncomb, b.B), WF_COMB_THREADS, sm, st>>>(g, lb, b.part, mode);
  return cudaGetLastError();
}
template <typename T>
cudaError_t wf_launch_lb_qdots(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st) {
  static int done = 0;
  auto k = k_lb_qdots<T>;
  const size_t sm = wf_comb_smem<T>(lb.m);
  cudaError_t e = wfimpl::ensure_smem_n(k, wf_comb_smem<T>(WF_MAXM), &done);
  if (e != cudaSuccess) return e;
  k<<<dim3(g.ncomb, b.B), WF_COMB_THREADS, sm, st>>>(g, lb, b.part);
  return cudaGetLastError();
}
template <typename T>
cudaError_t wf_launch_lb_colinv(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st) {
  return g.C == 1 ? wfimpl::lb_colinv<T, 1>(g, b, lb, st) : wfimpl::lb_colinv<T, 2>(g, b, lb, st);
}
template <typename T>
cudaError_t wf_launch_lb_colfwd(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st) {
  return g.C == 1 ? wfimpl::lb_colfwd<T, 1>(g, b, lb, st) : wfimpl::lb_colfwd<T, 2>(g, b, lb, st);
}
namespace wfimpl {
template <typename T, int KIND, int PLAN>
cudaError_t lb_row(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st) {
  static int done = 0;
  auto k = k_lb_row<T, KIND, PLAN>;
  const size_t sm = KIND == WF_ROW_PP_K ? wf_pp_smem<T>() : row_smem<T>(g);
  cudaError_t e = ensure_smem(k, sm, &done);
  if (e != cudaSuccess) return e;
  k<<<dim3(g.nrb, b.B), WF_THREADS, sm, st>>>(g, b.scratch, b.w, b.part, b.tw, lb.st);
  return cudaGetLastError();
}
}  // namespace wfimpl
template <typename T>
cudaError_t wf_launch_lb_row(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st) {
  if (g.row_kind == WF_ROW_INPLACE_K) return wfimpl::lb_row<T, WF_ROW_INPLACE_K, 0>(g, b, lb, st);
  const int pl = wf_plan_eff(g.lgh, g.row_plan);
  return pl == 1 ? wfimpl::lb_row<T, WF_ROW_PP_K, 1>(g, b, lb, st)
         : pl == 2 ? wfimpl::lb_row<T, WF_ROW_PP_K, 2>(g, b, lb, st)
                   : wfimpl::lb_row<T, WF_ROW_PP_K, 0>(g, b, lb, st);
}
template <typename T>
cudaError_t wf_launch_eval_pk(const WfGeo& g, const WfBufs& b, const void* src, void* dst, cudaStream_t st) {
  cudaError_t e = wfimpl::col_inv_any<T>(g, b, WF_IN_PK, src, st);
  if (e == cudaSuccess) e = wfimpl::row_any<T>(WF_ROW_DATA, g, b, nullptr, nullptr, st);
  if (e == cudaSuccess) e = wfimpl::col_fwd_any<T>(g, b, WF_IN_PK, src, dst, st);
  return e;
}

// Explicit instantiations, split over translation units that compile in
// parallel: the operator calls, the L-BFGS column stages, the L-BFGS row stage
// and streaming kernels.
#define WF_INSTANTIATE_OPS(T)                                                                      \
  template cudaError_t wf_launch_prep<T>(const WfGeo&, const void* const*,                         \
                                         const unsigned char* const*, const void* const*,          \
                                         const void* const*, int, int, void*, void*, void*, int,   \
                                         int*, cudaStream_t);                                      \
  template cudaError_t wf_launch_set_data<T>(const WfGeo&, const void*, int, void*, cudaStream_t); \
  template cudaError_t wf_launch_eval<T>(const WfGeo&, const WfBufs&, int, int, const void*,       \
                                         void*, double*, cudaStream_t);                            \
  template cudaError_t wf_launch_signal<T>(const WfGeo&, const WfBufs&, int, const void*, void*,   \
                                           cudaStream_t);                                          \
  template cudaError_t wf_launch_simulate<T>(const WfGeo&, const WfBufs&, const void*,             \
                                             const void*, void*, cudaStream_t);                    \
  template cudaError_t wf_launch_band_energy<T>(const WfGeo&, int, const void*, const int16_t*,    \
                                                const double*, int, double*, double*, cudaStream_t); \
  template cudaError_t wf_launch_pack<T>(const WfGeo&, int, const void*, void*, cudaStream_t);     \
  template cudaError_t wf_launch_unpack<T>(const WfGeo&, int, const void*, void*, cudaStream_t);    \
  template cudaError_t wf_launch_eval_pk<T>(const WfGeo&, const WfBufs&, const void*, void*,       \
                                            cudaStream_t);                                         \
  template cudaError_t wf_launch_eval_bands<T>(const WfGeo&, const WfBufs&, const void*, void*,    \
                                               double*, const int16_t*, int, double*, double*,       \
                                               cudaStream_t);                                        \
  template cudaError_t wf_launch_band_scale<T>(const WfGeo&, const void*, void*, int,               \
                                               const int16_t*, const double*, int, cudaStream_t);
#define WF_INSTANTIATE_LBCOL(T)                                                                    \
  template cudaError_t wf_launch_lb_colinv<T>(const WfGeo&, const WfBufs&, const WfLbBufs&,        \
                                              cudaStream_t);                                       \
  template cudaError_t wf_launch_lb_colfwd<T>(const WfGeo&, const WfBufs&, const WfLbBufs&,        \
                                              cudaStream_t);
#define WF_INSTANTIATE_LBROW(T)                                                                    \
  template cudaError_t wf_launch_lb_comb<T>(const WfGeo&, const WfBufs&, const WfLbBufs&, int,      \
                                            cudaStream_t);                                         \
  template cudaError_t wf_launch_lb_qdots<T>(const WfGeo&, const WfBufs&, const WfLbBufs&,         \
                                             cudaStream_t);                                        \
  template cudaError_t wf_launch_lb_row<T>(const WfGeo&, const WfBufs&, const WfLbBufs&,           \
                                           cudaStream_t);
