// Column kernels of one device L-BFGS iteration (Sec. 2.2: L-BFGS on chi^2).
//
// Per iteration and map:
//   k_lb1  applies the pending update s += a P, g += a Q of the previous step,
//          forms the new direction p = dg g + sum_i (dP_i P_i + dQ_i Q_i) from
//          the coefficients the scalar two-loop produced, stores p into the
//          ring, accumulates the exact dot products of g with every stored
//          vector, then runs the inverse-transform column stage on p;
//   (row stage without data: the Hessian-vector product needs no d)
//   k_lb3  finishes q = H p = 2 (p + A^T W A p) (forward column stage and the
//          adjoint), stores q into the ring and accumulates <q, Q_i>, <q, q>,
//          <p, q>, <g, q>, <g, p>, <p, p>.
// Dot products use the half-plane weights of the packed layout (1 on the
// packed column 0, 2 elsewhere), which equal the full-plane real inner product.
#pragma once
#include "wf_ops.cuh"

// Stage per-warp partial dot products: red[slot * NW + warp].
__device__ __forceinline__ void wf_warp_stash(double v, double* red, int slot) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[slot * (WF_THREADS / 32) + (threadIdx.x >> 5)] = v;
}

// Sum the staged warp partials of slots [0, nslot) into part[slot_id(i)].
__device__ __forceinline__ void wf_flush_slots(const double* red, int nslot, const int* ids, double* part_b,
                                               int maxblk) {
  for (int i = threadIdx.x; i < nslot; i += blockDim.x) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < WF_THREADS / 32; ++w) acc += red[i * (WF_THREADS / 32) + w];
    part_b[(size_t)ids[i] * maxblk + blockIdx.x] = acc;
  }
}

template <typename T>
__device__ __forceinline__ double wf_wdot(V2<T> a, V2<T> b, int kx) {
  const T d = a.x * b.x + a.y * b.y;
  return kx == 0 ? (double)d : 2.0 * (double)d;
}

template <typename T>
__device__ __forceinline__ V2<T> wf_axpy(V2<T> y, double a, V2<T> x) {
  const T s = (T)a;
  return mk<T>(y.x + s * x.x, y.y + s * x.y);
}

// Element e of a column tile: vector offset, shared-memory index, column kx.
struct WfTileIdx {
  int off, sidx, kx;
};
__device__ __forceinline__ WfTileIdx wf_tile_idx(int e, int n, int h, int lgn, int lgTC, int C, int kx0) {
  const int TC = 1 << lgTC;
  const int t = e & (TC - 1), r = e >> lgTC, j = r & (n - 1), c = r >> lgn;
  WfTileIdx x;
  x.kx = kx0 + t;
  x.off = (c * n + j) * h + kx0 + t;
  x.sidx = j * C * TC + c * TC + t;
  return x;
}

template <typename T, int C>
__global__ void __launch_bounds__(WF_THREADS)
k_lb1(WfGeo g, const T* sp_, long long sp_stride, void* scratch_, const void* tw_, WfLbBufs lb,
      double* part, int mode) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  const int b = blockIdx.y;
  const WfLbMap* M = lb.st + b;
  const int active = M->active;
  const double pa = M->pend_alpha;
  if (mode == WF_LB1_FULL && !active && pa == 0.0) return;
  if (mode == WF_LB1_MATERIALIZE && pa == 0.0) return;
  V2<T>* s_tw = (V2<T>*)wf_smem;
  V2<T>* buf = s_tw + WF_NT;
  V2<T>* gb = buf + WF_TILE;
  double* red = (double*)(gb + WF_TILE);
  int* ids = (int*)(red + (2 * WF_MAXM + 1) * (WF_THREADS / 32));
  const int n = g.n, h = g.h, lgn = g.lgn, TC = g.TC, lgTC = __ffs(TC) - 1;
  const int kx0 = blockIdx.x * TC, tot = C * n * TC;
  const size_t vsz = (size_t)C * n * h;
  const int B = gridDim.y, m = lb.m;
  V2<T>* sv = (V2<T>*)lb.s + (size_t)b * vsz;
  V2<T>* gv = (V2<T>*)lb.g + (size_t)b * vsz;
  V2<T>* ring = (V2<T>*)lb.ring;
  auto Pv = [&](int i) { return ring + ((size_t)i * B + b) * vsz; };
  auto Qv = [&](int i) { return ring + ((size_t)(m + i) * B + b) * vsz; };

  // 1. state update of the previous step (or plain load of g)
  if (pa != 0.0 && mode != WF_LB1_DOTS) {
    const V2<T>* Pp = Pv(M->pend_slot);
    const V2<T>* Qp = Qv(M->pend_slot);
#pragma unroll
    for (int i = 0; i < WF_EMAX; ++i) {
      const int e = threadIdx.x + i * WF_THREADS;
      if (e < tot) {
        const WfTileIdx x = wf_tile_idx(e, n, h, lgn, lgTC, C, kx0);
        const V2<T> s1 = wf_axpy<T>(sv[x.off], pa, Pp[x.off]);
        const V2<T> g1 = wf_axpy<T>(gv[x.off], pa, Qp[x.off]);
        sv[x.off] = s1;
        gv[x.off] = g1;
        gb[x.sidx] = g1;
      }
    }
  } else if (mode != WF_LB1_MATERIALIZE) {
#pragma unroll
    for (int i = 0; i < WF_EMAX; ++i) {
      const int e = threadIdx.x + i * WF_THREADS;
      if (e < tot) {
        const WfTileIdx x = wf_tile_idx(e, n, h, lgn, lgTC, C, kx0);
        gb[x.sidx] = gv[x.off];
      }
    }
  }
  if (mode == WF_LB1_MATERIALIZE) return;
  if (mode == WF_LB1_FULL && !active) return;
  const bool full = (mode == WF_LB1_FULL);

  // 2. direction and dot products of g with the stored vectors
  const int np = M->npairs, head = M->head;
  const double dg = M->dg;
  double acc = 0.0;
#pragma unroll
  for (int i = 0; i < WF_EMAX; ++i) {
    const int e = threadIdx.x + i * WF_THREADS;
    if (e < tot) {
      const WfTileIdx x = wf_tile_idx(e, n, h, lgn, lgTC, C, kx0);
      const V2<T> gg = gb[x.sidx];
      acc += wf_wdot<T>(gg, gg, x.kx);
      if (full) buf[x.sidx] = mk<T>((T)dg * gg.x, (T)dg * gg.y);
    }
  }
  wf_warp_stash(acc, red, 0);
  if (threadIdx.x == 0) ids[0] = WF_SLOT_GG;
  for (int q = 0; q < np; ++q) {
    const int sl = (head - q + m) % m;
    for (int half = 0; half < 2; ++half) {
      const V2<T>* vp = half == 0 ? Pv(sl) : Qv(sl);
      const double coef = half == 0 ? M->dP[sl] : M->dQ[sl];
      V2<T> v[WF_EMAX];
#pragma unroll
      for (int i = 0; i < WF_EMAX; ++i) {
        const int e = threadIdx.x + i * WF_THREADS;
        if (e < tot) v[i] = vp[wf_tile_idx(e, n, h, lgn, lgTC, C, kx0).off];
      }
      double a2 = 0.0;
#pragma unroll
      for (int i = 0; i < WF_EMAX; ++i) {
        const int e = threadIdx.x + i * WF_THREADS;
        if (e < tot) {
          const WfTileIdx x = wf_tile_idx(e, n, h, lgn, lgTC, C, kx0);
          a2 += wf_wdot<T>(gb[x.sidx], v[i], x.kx);
          if (full) buf[x.sidx] = wf_axpy<T>(buf[x.sidx], coef, v[i]);
        }
      }
      const int k = 1 + 2 * q + half;
      wf_warp_stash(a2, red, k);
      if (threadIdx.x == 0) ids[k] = (half == 0 ? WF_SLOT_GP : WF_SLOT_GQ) + sl;
    }
  }
  __syncthreads();
  wf_flush_slots(red, 1 + 2 * np, ids, part + (size_t)b * WF_NSLOT * g.maxblk, g.maxblk);
  if (!full) return;

  // 3. store p into its ring slot, then the inverse-transform column stage
  V2<T>* Pn = Pv(M->next);
#pragma unroll
  for (int i = 0; i < WF_EMAX; ++i) {
    const int e = threadIdx.x + i * WF_THREADS;
    if (e < tot) {
      const WfTileIdx x = wf_tile_idx(e, n, h, lgn, lgTC, C, kx0);
      Pn[x.off] = buf[x.sidx];
    }
  }
  wf_stage_tw<T>(s_tw, (const V2<T>*)tw_);
  __syncthreads();
  wf_col_scale<T, C, false>(buf, n, lgTC, kx0, sp_ + (size_t)b * sp_stride, (T)1);
  __syncthreads();
  fft_smem<T, +1, WF_EMAX>(buf, lgn, C * TC, 1, C * TC, s_tw);
  wf_tile_store_pk<T, C>((V2<T>*)scratch_ + (size_t)b * vsz, buf, n, lgTC, kx0);
}

template <typename T, int C>
__global__ void __launch_bounds__(WF_THREADS)
k_lb3(WfGeo g, const T* sp_, long long sp_stride, const void* scratch_, const void* tw_, WfLbBufs lb,
      double* part) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  const int b = blockIdx.y;
  const WfLbMap* M = lb.st + b;
  if (!M->active) return;
  V2<T>* s_tw = (V2<T>*)wf_smem;
  V2<T>* buf = s_tw + WF_NT;
  double* red = (double*)(buf + WF_TILE);
  int* ids = (int*)(red + (WF_MAXM + 5) * (WF_THREADS / 32));
  const int n = g.n, h = g.h, lgn = g.lgn, TC = g.TC, lgTC = __ffs(TC) - 1, CT = C * TC;
  const int kx0 = blockIdx.x * TC, tot = C * n * TC;
  const size_t vsz = (size_t)C * n * h;
  const int B = gridDim.y, m = lb.m;
  V2<T>* ring = (V2<T>*)lb.ring;
  auto Pv = [&](int i) { return ring + ((size_t)i * B + b) * vsz; };
  auto Qv = [&](int i) { return ring + ((size_t)(m + i) * B + b) * vsz; };
  wf_stage_tw<T>(s_tw, (const V2<T>*)tw_);
  const V2<T>* sc = (const V2<T>*)scratch_ + (size_t)b * vsz;
#pragma unroll
  for (int i = 0; i < WF_EMAX; ++i) {
    const int e = threadIdx.x + i * WF_THREADS;
    if (e < tot) {
      const WfTileIdx x = wf_tile_idx(e, n, h, lgn, lgTC, C, kx0);
      buf[x.sidx] = sc[x.off];
    }
  }
  __syncthreads();
  fft_smem<T, -1, WF_EMAX>(buf, lgn, CT, 1, CT, s_tw);
  wf_col_scale<T, C, true>(buf, n, lgTC, kx0, sp_ + (size_t)b * sp_stride, (T)1);
  __syncthreads();
  const int nx = M->next;
  const V2<T>* Pn = Pv(nx);
  V2<T>* Qn = Qv(nx);
  const V2<T>* gv = (const V2<T>*)lb.g + (size_t)b * vsz;
  double qq = 0, pq = 0, pp = 0, gq = 0, gp = 0;
  V2<T> qr[WF_EMAX];
#pragma unroll
  for (int i = 0; i < WF_EMAX; ++i) {
    const int e = threadIdx.x + i * WF_THREADS;
    if (e < tot) {
      const WfTileIdx x = wf_tile_idx(e, n, h, lgn, lgTC, C, kx0);
      const V2<T> p = Pn[x.off], a = buf[x.sidx], gg = gv[x.off];
      const V2<T> q = mk<T>((T)2 * (p.x - a.x), (T)2 * (p.y - a.y));
      Qn[x.off] = q;
      qr[i] = q;
      qq += wf_wdot<T>(q, q, x.kx);
      pq += wf_wdot<T>(p, q, x.kx);
      pp += wf_wdot<T>(p, p, x.kx);
      gq += wf_wdot<T>(gg, q, x.kx);
      gp += wf_wdot<T>(gg, p, x.kx);
    }
  }
  wf_warp_stash(qq, red, 0);
  wf_warp_stash(pq, red, 1);
  wf_warp_stash(pp, red, 2);
  wf_warp_stash(gq, red, 3);
  wf_warp_stash(gp, red, 4);
  if (threadIdx.x == 0) {
    ids[0] = WF_SLOT_QQ; ids[1] = WF_SLOT_PQ; ids[2] = WF_SLOT_PP; ids[3] = WF_SLOT_GQN; ids[4] = WF_SLOT_GPN;
  }
  const int np = M->npairs, head = M->head;
  int k = 5;
  for (int q = 0; q < np; ++q) {
    const int sl = (head - q + m) % m;
    if (sl == nx) continue;
    const V2<T>* vq = Qv(sl);
    double a2 = 0.0;
#pragma unroll
    for (int i = 0; i < WF_EMAX; ++i) {
      const int e = threadIdx.x + i * WF_THREADS;
      if (e < tot) {
        const WfTileIdx x = wf_tile_idx(e, n, h, lgn, lgTC, C, kx0);
        a2 += wf_wdot<T>(qr[i], vq[x.off], x.kx);
      }
    }
    wf_warp_stash(a2, red, k);
    if (threadIdx.x == 0) ids[k] = WF_SLOT_QQI + sl;
    ++k;
  }
  __syncthreads();
  wf_flush_slots(red, k, ids, part + (size_t)b * WF_NSLOT * g.maxblk, g.maxblk);
}

// Row stage of the Hessian-vector product for the maps still iterating.
template <typename T>
__global__ void __launch_bounds__(WF_THREADS)
k_lb_row(WfGeo g, void* scratch_, const void* w_, double* part, const void* tw_, const WfLbMap* st) {
  if (!st[blockIdx.y].active) return;
  k_row_body<T, WF_ROW_NODATA>(g, scratch_, nullptr, w_, nullptr, nullptr, part, tw_);
}
