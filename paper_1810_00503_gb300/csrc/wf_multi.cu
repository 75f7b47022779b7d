// Shared launches of the L-BFGS iteration over several problems (declared in
// wf_internal.h): the streaming kernels, the ping-pong inverse column and row
// stages and the in-place forward column stage, each block locating its
// problem and its coordinates in that problem's own grid.
#include "wf_ops_impl.cuh"

struct WfMultiGrid {
  int np;
  int start[WF_MULTI_MAX + 1];
  int gx[WF_MULTI_MAX];
  int gy[WF_MULTI_MAX];
};

// Problem of this block and its coordinates in the problem's grid.
__device__ __forceinline__ int wf_multi_block(const WfMultiGrid& r, WfBlk& kb) {
  const int bid = blockIdx.x;
  int q = 0;
  while (q + 1 < r.np && bid >= r.start[q + 1]) ++q;
  const int local = bid - r.start[q];
  kb.nx = r.gx[q];
  kb.ny = r.gy[q];
  kb.x = local % kb.nx;
  kb.y = local / kb.nx;
  return q;
}

// Grid of problem q's blocks: gx(q) x (its maps), concatenated over the problems.
template <class F>
static WfMultiGrid wf_multi_grid(const WfMultiArgs& a, F gx) {
  WfMultiGrid r;
  r.np = a.np;
  r.start[0] = 0;
  for (int q = 0; q < a.np; ++q) {
    r.gx[q] = gx(a.g[q]);
    r.gy[q] = a.b[q].B;
    r.start[q + 1] = r.start[q] + r.gx[q] * r.gy[q];
  }
  return r;
}

template <typename T>
__global__ void __launch_bounds__(WF_COMB_THREADS, sizeof(T) == 4 ? WF_COMB_MINB : 2)
k_multi_comb(const __grid_constant__ WfMultiGrid r, const __grid_constant__ WfMultiArgs a, int mode) {
  WfBlk kb;
  const int q = wf_multi_block(r, kb);
  wf_lb_comb<T>(a.g[q], a.lb[q], a.b[q].part, mode, kb);
}

template <typename T>
__global__ void __launch_bounds__(WF_COMB_THREADS, sizeof(T) == 4 ? 4 : 2)
k_multi_qdots(const __grid_constant__ WfMultiGrid r, const __grid_constant__ WfMultiArgs a) {
  WfBlk kb;
  const int q = wf_multi_block(r, kb);
  wf_lb_qdots<T>(a.g[q], a.lb[q], a.b[q].part, kb);
}

template <typename T, int C>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB_PLAN(T, 0))
k_multi_colinv(const __grid_constant__ WfMultiGrid r, const __grid_constant__ WfMultiArgs a) {
  WfBlk kb;
  const int q = wf_multi_block(r, kb);
  const WfBufs& b = a.b[q];
  wf_lb_colinv<T, C, WF_COLINV_PP_K, 0>(a.g[q], (const T*)b.sp, b.sp_stride, b.scratch, b.tw, a.lb[q], kb);
}

template <typename T>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB_PLAN(T, 0))
k_multi_row(const __grid_constant__ WfMultiGrid r, const __grid_constant__ WfMultiArgs a) {
  WfBlk kb;
  const int q = wf_multi_block(r, kb);
  if (!a.lb[q].st[kb.y].active) return;
  const WfBufs& b = a.b[q];
  wf_row_pp<T, WF_ROW_NODATA, 0>(a.g[q], (V2<T>*)b.scratch, nullptr, (const T*)b.w, b.part, b.tw, kb.y, kb.x);
}

template <typename T, int C>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB_LBCOLFWD(T, C))
k_multi_colfwd(const __grid_constant__ WfMultiGrid r, const __grid_constant__ WfMultiArgs a) {
  WfBlk kb;
  const int q = wf_multi_block(r, kb);
  const WfBufs& b = a.b[q];
  wf_lb_colfwd<T, C>(a.g[q], (const T*)b.sp, b.sp_stride, b.scratch, b.tw, a.lb[q], b.part, kb);
}

namespace {
template <typename K>
cudaError_t multi_smem(K k, size_t bytes, int* done) {
  return wfimpl::ensure_smem_n(k, bytes, done);
}
}  // namespace

template <typename T>
cudaError_t wf_launch_multi_comb(const WfMultiArgs& a, int mode, cudaStream_t st) {
  static int done = 0;
  const WfMultiGrid r = wf_multi_grid(a, [](const WfGeo& g) { return g.ncomb; });
  cudaError_t e = multi_smem(k_multi_comb<T>, wf_comb_smem<T>(WF_MAXM), &done);
  if (e != cudaSuccess) return e;
  k_multi_comb<T><<<r.start[a.np], WF_COMB_THREADS, wf_comb_smem<T>(a.lb[0].m), st>>>(r, a, mode);
  return cudaGetLastError();
}

template <typename T>
cudaError_t wf_launch_multi_qdots(const WfMultiArgs& a, cudaStream_t st) {
  static int done = 0;
  const WfMultiGrid r = wf_multi_grid(a, [](const WfGeo& g) { return g.ncomb; });
  cudaError_t e = multi_smem(k_multi_qdots<T>, wf_comb_smem<T>(WF_MAXM), &done);
  if (e != cudaSuccess) return e;
  k_multi_qdots<T><<<r.start[a.np], WF_COMB_THREADS, wf_comb_smem<T>(a.lb[0].m), st>>>(r, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t wf_launch_multi_colinv(const WfMultiArgs& a, cudaStream_t st) {
  static int done[2] = {0, 0};
  const WfMultiGrid r = wf_multi_grid(a, [](const WfGeo& g) { return g.ntile; });
  auto k = a.g[0].C == 1 ? k_multi_colinv<T, 1> : k_multi_colinv<T, 2>;
  cudaError_t e = multi_smem(k, wf_pp_smem<T>(), &done[a.g[0].C - 1]);
  if (e != cudaSuccess) return e;
  k<<<r.start[a.np], WF_THREADS, wf_pp_smem<T>(), st>>>(r, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t wf_launch_multi_row(const WfMultiArgs& a, cudaStream_t st) {
  static int done = 0;
  const WfMultiGrid r = wf_multi_grid(a, [](const WfGeo& g) { return g.nrb; });
  cudaError_t e = multi_smem(k_multi_row<T>, wf_pp_smem<T>(), &done);
  if (e != cudaSuccess) return e;
  k_multi_row<T><<<r.start[a.np], WF_THREADS, wf_pp_smem<T>(), st>>>(r, a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t wf_launch_multi_colfwd(const WfMultiArgs& a, cudaStream_t st) {
  static int done[2] = {0, 0};
  const WfMultiGrid r = wf_multi_grid(a, [](const WfGeo& g) { return g.ntile; });
  size_t sm = 0;
  for (int q = 0; q < a.np; ++q) {
    const size_t s = wfimpl::col_smem<T>(a.g[q]);
    if (s > sm) sm = s;
  }
  auto k = a.g[0].C == 1 ? k_multi_colfwd<T, 1> : k_multi_colfwd<T, 2>;
  cudaError_t e = multi_smem(k, wf_pp_smem<double>(), &done[a.g[0].C - 1]);
  if (e != cudaSuccess) return e;
  k<<<r.start[a.np], WF_THREADS, sm, st>>>(r, a);
  return cudaGetLastError();
}

#define WF_INSTANTIATE_MULTI(T)                                                               \
  template cudaError_t wf_launch_multi_comb<T>(const WfMultiArgs&, int, cudaStream_t);        \
  template cudaError_t wf_launch_multi_colinv<T>(const WfMultiArgs&, cudaStream_t);           \
  template cudaError_t wf_launch_multi_row<T>(const WfMultiArgs&, cudaStream_t);              \
  template cudaError_t wf_launch_multi_colfwd<T>(const WfMultiArgs&, cudaStream_t);           \
  template cudaError_t wf_launch_multi_qdots<T>(const WfMultiArgs&, cudaStream_t);
WF_INSTANTIATE_MULTI(float)
WF_INSTANTIATE_MULTI(double)

WF_DBG_READER(multi)
