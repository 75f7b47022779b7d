// Operator stages on the ping-pong passes of wf_fft_pp.cuh (the same three
// steps as the kernels of wf_ops.cuh; the first FFT pass reads global memory
// with the per-mode operator or the real-FFT pre-step applied on the way in).
//
// Shared memory of every stage: the length-L pass table (WF_NT entries) and
// two tiles A, B of WF_TILE values.
#pragma once
#include "wf_fft_pp.cuh"
#include "wf_ops.cuh"

template <typename T>
__host__ __device__ constexpr size_t wf_pp_smem() {
  return ((size_t)WF_NT + 2 * (size_t)WF_TILE) * sizeof(V2<T>);
}

// Packed value of column tile element (row j, channel c, column kx) after the
// per-mode operator (R(k) sqrt(P)/n, or its adjoint), read through `ld(cc, row)`
// (channel cc's packed value at row `row` of this column).  Column 0 is
// unpacked with row ny - j, the operator applied at kx = 0 and kx = nx/2, and
// packed again.
template <typename T, int C, bool ADJ, class LD>
__device__ __forceinline__ V2<T> wf_mode_packed(LD& ld, int j, int c, int kx, const WfGeo& g, const T* sp) {
  V2<T> v[C];
  if (kx != 0) {
#pragma unroll
    for (int cc = 0; cc < C; ++cc) v[cc] = ld(cc, j);
    wf_mode_op<T, C, ADJ>(v, j, kx, g, sp, (T)1);
    return v[c];
  }
  const int jm = (g.n - j) & (g.n - 1);
  V2<T> X0[C], Xh[C];
#pragma unroll
  for (int cc = 0; cc < C; ++cc) wf_unpack0<T>(ld(cc, j), ld(cc, jm), X0[cc], Xh[cc]);
  wf_mode_op<T, C, ADJ>(X0, j, 0, g, sp, (T)1);
  wf_mode_op<T, C, ADJ>(Xh, j, g.h, g, sp, (T)1);
  return wf_pack0<T>(X0[c], Xh[c]);
}

// Inverse column stage: spectrum (packed [C][n][h], or standard [C][n][h+1])
// -> R sqrt(P)/n -> inverse FFT along y -> scratch (packed), for the column
// tile starting at packed column kx0 (blockIdx.x * TC if negative).  stage:
// copy the pass table to shared memory first (a persistent caller does it
// once).
template <typename T, int C, int IN, int PLAN>
__device__ __forceinline__ void wf_col_inv_pp(const WfGeo& g, const V2<T>* src, const T* sp, V2<T>* scr,
                                              const void* tw_, int kx0 = -1, bool stage = true) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  V2<T>* s_tw = (V2<T>*)wf_smem;
  V2<T>* A = s_tw + WF_NT;
  V2<T>* Bf = A + WF_TILE;
  const int n = g.n, h = g.h, lgn = g.lgn, TC = g.TC, lgTC = __ffs(TC) - 1;
  const int lgCT = lgTC + (C == 2 ? 1 : 0);
  if (kx0 < 0) kx0 = blockIdx.x * TC;
  if (stage) wf_stage_tw<T>(s_tw, (const V2<T>*)tw_, lgn, PLAN);  // first read after the first barrier
  auto ld0 = [&](int t, int row) -> V2<T> {
    const int c = t >> lgTC, kx = kx0 + (t & (TC - 1));
    if constexpr (IN == WF_IN_STD) {
      if (kx == 0) {  // kx = 0 and kx = nx/2 stored separately
        V2<T> X0[C], Xh[C];
#pragma unroll
        for (int cc = 0; cc < C; ++cc) {
          const V2<T>* r = src + WF_CHK(((size_t)cc * n + row) * (h + 1), (size_t)C * n * (h + 1) - h);
          X0[cc] = r[0];
          Xh[cc] = r[h];
        }
        wf_mode_op<T, C, false>(X0, row, 0, g, sp, (T)1);
        wf_mode_op<T, C, false>(Xh, row, h, g, sp, (T)1);
        return wf_pack0<T>(X0[c], Xh[c]);
      }
      auto ldg = [&](int cc, int rr) { return src[WF_CHK(((size_t)cc * n + rr) * (h + 1) + kx, (size_t)C * n * (h + 1))]; };
      return wf_mode_packed<T, C, false>(ldg, row, c, kx, g, sp);
    } else {
      auto ldg = [&](int cc, int rr) { return src[WF_CHK(((size_t)cc * n + rr) * h + kx, (size_t)C * n * h)]; };
      return wf_mode_packed<T, C, false>(ldg, row, c, kx, g, sp);
    }
  };
  auto stl = [&](int t, int row, V2<T> v) {
    scr[WF_CHK(((size_t)(t >> lgTC) * n + row) * h + kx0 + (t & (TC - 1)), (size_t)C * n * h)] = v;
  };
  wf_pp_fft<T, +1, true, PLAN>(lgn, lgCT, 1, C * TC, A, Bf, s_tw, ld0, stl);
}

// Row stage of the objective (MODE DATA: r = d - x) or of the Hessian-vector
// product (MODE NODATA: r = -x): c2r along x, wr = w r, partial sum r.wr, r2c
// of wr along x, back to scratch.  The c2r pre-step pairs X[k] with X[h-k] of
// the same row and is applied as the first pass loads; the r2c post-step runs
// from the last pass's shared output.  src: the RB rows of packed spectra (h
// values each, global or shared memory); sc: where the result rows go
// (global); d, w: the pixel rows (RB nx values from the block's first row);
// roots: exp(-2 pi i k / nx) for k < nx/2, in shared memory.  Returns this
// thread's part of sum r.wr.  after1 runs once the first pass has finished
// reading src.
template <typename T, int MODE, int PLAN, class H = WfNoHook>
__device__ __forceinline__ WfAcc<T> wf_row_pp_core(const WfGeo& g, const V2<T>* src, V2<T>* sc, const T* d,
                                                   const T* w, const V2<T>* roots, const V2<T>* s_pt, V2<T>* A,
                                                   V2<T>* Bf, H after1 = H()) {
  const int h = g.h, lgh = g.lgh, RB = g.RB, lgRB = __ffs(RB) - 1;
  const V2<T>* dv = (const V2<T>*)d;
  const V2<T>* wv = (const V2<T>*)w;
  // c2r pre-step: Z[k] = (X[k] + conj X[h-k]) + i w^k (X[k] - conj X[h-k]), w = exp(+2 pi i / nx);
  // Z[0] from the packed X[0] + i X[h].
  auto ld0 = [&](int t, int k) -> V2<T> {
    const V2<T>* row = src + WF_CHK((size_t)t * h, (size_t)RB * h);
    const V2<T> Xk = row[WF_CHK(k, h)];
    if (k == 0) return mk<T>(Xk.x + Xk.y, Xk.x - Xk.y);
    const V2<T> Xm = row[WF_CHK(h - k, h)];
    const V2<T> w1 = twid<T, +1>(roots, k);
    const V2<T> s1 = mk<T>(Xk.x + Xm.x, Xk.y - Xm.y), d1 = mk<T>(Xk.x - Xm.x, Xk.y + Xm.y);
    return cadd<T>(s1, mul_i<T>(cmul<T>(w1, d1)));
  };
  // pixel step on the c2r output (pixels 2m, 2m+1 of row t): wr = w (d - x)
  V2<T>* O = wf_pp_out<T>(lgh, PLAN, A, Bf);
  WfAcc<T> acc = 0;
  auto stpix = [&](int t, int m, V2<T> x) {
    const size_t e = WF_CHK((size_t)t * h + m, (size_t)RB * h);
    const V2<T> wl = wv[e];
    V2<T> r;
    if constexpr (MODE == WF_ROW_DATA) {
      const V2<T> dl = dv[e];
      r = mk<T>(dl.x - x.x, dl.y - x.y);
    } else {
      r = mk<T>(-x.x, -x.y);
    }
    const V2<T> wr = mk<T>(wl.x * r.x, wl.y * r.y);
    acc += (WfAcc<T>)(r.x * wr.x + r.y * wr.y);
    O[wf_swp<T>(t * h + m)] = wr;
  };
  wf_pp_fft<T, +1, false, PLAN>(lgh, lgRB, h, 1, A, Bf, s_pt, ld0, stpix, after1);
  __syncthreads();
  // r2c of wr: the input is O, so the passes start from the other buffer
  V2<T>* A2 = (O == A) ? Bf : A;
  auto ldO = [&](int t, int e) { return O[wf_swp<T>(t * h + e)]; };
  V2<T>* Z = wf_pp_out<T>(lgh, PLAN, A2, O);
  auto stZ = [&](int t, int e, V2<T> v) { Z[wf_swp<T>(t * h + e)] = v; };
  wf_pp_fft<T, -1, false, PLAN>(lgh, lgRB, h, 1, A2, O, s_pt, ldO, stZ);
  __syncthreads();
  // r2c post-step: X[k] = (Z[k] + conj Z[h-k])/2 - i w^-k (Z[k] - conj Z[h-k])/2, X[0], X[h] packed
  for (int e = threadIdx.x; e < RB * h; e += blockDim.x) {
    const int t = e >> lgh, k = e & (h - 1);
    const V2<T> Zk = Z[wf_swp<T>(t * h + k)];
    V2<T> X;
    if (k == 0) {
      X = mk<T>(Zk.x + Zk.y, Zk.x - Zk.y);
    } else {
      const V2<T> Zm = Z[wf_swp<T>(t * h + h - k)];
      const V2<T> w1 = twid<T, -1>(roots, k);
      const V2<T> s1 = mk<T>(Zk.x + Zm.x, Zk.y - Zm.y), d1 = mk<T>(Zk.x - Zm.x, Zk.y + Zm.y);
      const V2<T> i1 = mul_i<T>(cmul<T>(w1, d1));
      X = mk<T>((T)0.5 * (s1.x - i1.x), (T)0.5 * (s1.y - i1.y));
    }
    sc[WF_CHK(e, RB * h)] = X;
  }
  return acc;
}

// Shared-memory tables of the row stage: the length-h pass table (under
// WF_NT / 2 entries for h <= 512), then the nx-th roots the real-FFT pre- and
// post-steps use.  Read after the caller's next barrier.
template <typename T, int PLAN>
__device__ __forceinline__ void wf_row_pp_tables(const WfGeo& g, V2<T>* s_pt, const void* tw_) {
  const V2<T>* gt = (const V2<T>*)tw_;
  const V2<T>* src = gt + (size_t)WF_TWTAB * PLAN + (size_t)WF_NT * g.lgh;
  const int lgNTn = WF_LOG2_NT - g.lgnx;
  for (int i = threadIdx.x; i < WF_NT / 2; i += blockDim.x) {
    s_pt[i] = src[i];
    if (i < g.h) s_pt[WF_NT / 2 + i] = gt[i << lgNTn];
  }
}

// Row block rb of map b (tables staged), its data partial sum to part.
template <typename T, int MODE, int PLAN>
__device__ __forceinline__ void wf_row_pp_item(const WfGeo& g, V2<T>* scratch, const T* d, const T* w,
                                               double* part, int b, int rb) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  V2<T>* s_pt = (V2<T>*)wf_smem;
  V2<T>* A = s_pt + WF_NT;
  V2<T>* Bf = A + WF_TILE;
  const int n = g.n, nx = g.nx, h = g.h, row0 = rb * g.RB;
  const size_t npix = (size_t)g.C * n * nx;
  V2<T>* sc = scratch + (size_t)b * g.C * n * h + (size_t)row0 * h;
  const size_t poff = (size_t)b * npix + (size_t)row0 * nx;
  const WfAcc<T> acc = wf_row_pp_core<T, MODE, PLAN>(g, sc, sc, MODE == WF_ROW_DATA ? d + poff : nullptr, w + poff,
                                                     s_pt + WF_NT / 2, s_pt, A, Bf);
  const double s = wf_block_sum((double)acc);
  if (threadIdx.x == 0) part[((size_t)b * WF_NSLOT + WF_SLOT_DATA) * g.maxblk + rb] = s;
}

// Start the pixel rows of row block rb of map b towards L2 (the last pass of
// its c2r reads them).
template <typename T, int MODE>
__device__ __forceinline__ void wf_row_pp_prefetch_pix(const WfGeo& g, const T* d, const T* w, int b, int rb) {
  const size_t off = (size_t)b * g.C * g.n * g.nx + (size_t)rb * g.RB * g.nx;
  wf_prefetch_rows(w + off, 1, 0, g.RB * g.nx * (int)sizeof(T));
  if (MODE == WF_ROW_DATA) wf_prefetch_rows(d + off, 1, 0, g.RB * g.nx * (int)sizeof(T));
}

// Row block rb of map b, one block (by default blockIdx.x of map blockIdx.y).
template <typename T, int MODE, int PLAN>
__device__ __forceinline__ void wf_row_pp(const WfGeo& g, V2<T>* scratch, const T* d, const T* w, double* part,
                                          const void* tw_, int b = -1, int rb = -1) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  if (b < 0) {
    b = blockIdx.y;
    rb = blockIdx.x;
  }
  wf_row_pp_prefetch_pix<T, MODE>(g, d, w, b, rb);
  wf_row_pp_tables<T, PLAN>(g, (V2<T>*)wf_smem, tw_);
  __syncthreads();
  wf_row_pp_item<T, MODE, PLAN>(g, scratch, d, w, part, b, rb);
}

// Kernels of the objective + gradient pass on the ping-pong stages.
// The inverse column stage as a persistent kernel: the resident blocks take
// the (map, column tile) items in turn, and while a block transforms one tile
// it asks L2 for the rows of the tile it takes next, so that the first pass of
// that tile, which reads global memory directly, finds them there (0.51 ms
// against 0.59 ms one block per tile on 120 x 1024^2).  The objective pass
// runs its work-queue form below when the problem has a counter for it.  The row stage runs one
// block per row block (as k_row): its persistent form measured 0.59 against
// 0.55 ms.
template <typename T, int C, int IN, int PLAN>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB_PLAN(T, PLAN))
k_col_inv_pp_pers(WfGeo g, const void* src_, const T* sp_, long long sp_stride, void* scratch_, const void* tw_,
                  int B) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  const int n = g.n, h = g.h, pitch = IN == WF_IN_PK ? h : h + 1;
  const size_t sstride = (size_t)C * n * pitch;
  const int nitems = B * g.ntile;
  wf_stage_tw<T>((V2<T>*)wf_smem, (const V2<T>*)tw_, g.lgn, PLAN);
  auto prefetch = [&](int nt) {
    if (nt < nitems) {
      const int nb = nt / g.ntile, nk = (nt - nb * g.ntile) * g.TC;
      wf_prefetch_rows((const V2<T>*)src_ + (size_t)nb * sstride + nk, C * n, (size_t)pitch * sizeof(V2<T>),
                       g.TC * (int)sizeof(V2<T>));
    }
  };
  // the tiles WF_COLINV_AHEAD items ahead are asked for (all of them at the start)
  for (int a = 1; a < WF_COLINV_AHEAD; ++a) prefetch(blockIdx.x + a * gridDim.x);
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int b = it / g.ntile, kx0 = (it - b * g.ntile) * g.TC;
    prefetch(it + WF_COLINV_AHEAD * gridDim.x);
    wf_col_inv_pp<T, C, IN, PLAN>(g, (const V2<T>*)src_ + (size_t)b * sstride, sp_ + (size_t)b * sp_stride,
                                  (V2<T>*)scratch_ + (size_t)b * C * n * h, tw_, kx0, false);
    __syncthreads();  // the next item's first pass rewrites the tiles this one's last pass read
  }
}

// The same stage on a work queue: items from the counter *ticket (zero at
// launch), so the items in flight follow one another as under the hardware's
// in-order block dispatch; a block claims its next item before transforming
// the current one and asks L2 for that item's rows.
template <typename T, int C, int IN, int PLAN>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB_PLAN(T, PLAN))
k_col_inv_pp_q(WfGeo g, const void* src_, const T* sp_, long long sp_stride, void* scratch_, const void* tw_,
               int B, int* ticket) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  __shared__ int s_item[2];
  const int n = g.n, h = g.h, pitch = IN == WF_IN_PK ? h : h + 1;
  const size_t sstride = (size_t)C * n * pitch;
  const int nitems = B * g.ntile;
  wf_stage_tw<T>((V2<T>*)wf_smem, (const V2<T>*)tw_, g.lgn, PLAN);
  if (threadIdx.x == 0) s_item[0] = atomicAdd(ticket, 1);
  __syncthreads();
  int it = s_item[0], cur = 0;
  while (it < nitems) {
    if (threadIdx.x == 0) s_item[cur ^ 1] = atomicAdd(ticket, 1);
    __syncthreads();
    const int nt = s_item[cur ^ 1];
    if (nt < nitems) {
      const int nb = nt / g.ntile, nk = (nt - nb * g.ntile) * g.TC;
      wf_prefetch_rows((const V2<T>*)src_ + (size_t)nb * sstride + nk, C * n, (size_t)pitch * sizeof(V2<T>),
                       g.TC * (int)sizeof(V2<T>));
    }
    const int b = it / g.ntile, kx0 = (it - b * g.ntile) * g.TC;
    wf_col_inv_pp<T, C, IN, PLAN>(g, (const V2<T>*)src_ + (size_t)b * sstride, sp_ + (size_t)b * sp_stride,
                                  (V2<T>*)scratch_ + (size_t)b * C * n * h, tw_, kx0, false);
    __syncthreads();  // the next item's first pass rewrites the tiles this one's last pass read
    it = nt;
    cur ^= 1;
  }
}

template <typename T, int MODE, int PLAN>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB_PLAN(T, PLAN))
k_row_pp(WfGeo g, void* scratch_, const void* d_, const void* w_, double* part, const void* tw_) {
  wf_row_pp<T, MODE, PLAN>(g, (V2<T>*)scratch_, (const T*)d_, (const T*)w_, part, tw_);
}
