// Kernels of one device L-BFGS iteration (Sec. 2.2: L-BFGS on chi^2).
//
// Per iteration and map (all maps of a batch in each launch):
//   k_lb_comb   streaming: applies the pending update g += a Q of the previous
//               step (s += a P follows for the steps gathered, once every
//               m - 1 iterations and whenever s is needed), forms the new direction
//               p = dg g + sum_i (dP_i P_i + dQ_i Q_i) from the coefficients of
//               the scalar two-loop, stores p into the ring, and accumulates the
//               dot products of g with every stored vector;
//   k_lb_colinv inverse-transform column stage on p (A1, first half of A2);
//   k_lb_row    row stage of the Hessian-vector product (no data term);
//   k_lb_colfwd forward column stage and adjoint, q = H p = 2 (p + A^T W A p),
//               stores q into the ring, <q,q>, <p,q>, <g,q>, <g,p>, <p,p>;
//   k_lb_qdots  streaming: <q, Q_i> for the stored Q_i.
// The streaming kernels run at high occupancy with 16-byte loads; the column
// kernels keep only the transform work.  Dot products use the weights of the
// packed half plane (1 on the packed column 0, 2 elsewhere), which equal the
// full-plane real inner product.
#pragma once
#include "wf_ops.cuh"
#include "wf_stage_pp.cuh"
#include "wf_tma.cuh"


// Coordinates of a block in its problem's own launch grid: tile or chunk
// group x of map y, in a grid of nx by ny (the map count).  A single-problem
// launch takes them from blockIdx / gridDim; a launch shared by several
// problems (wf_multi.cuh) from its table of problems.
struct WfBlk {
  int x, y, nx, ny;
};
__device__ __forceinline__ WfBlk wf_blk() { return WfBlk{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x, (int)gridDim.y}; }

// Stage per-warp partial dot products: red[slot * NW + warp] (NW = warps of the block).
__device__ __forceinline__ void wf_warp_stash(double v, double* red, int slot, int nw) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[slot * nw + (threadIdx.x >> 5)] = v;
}

// Sum the staged warp partials of slots [0, nslot) into part_b[ids[i] * maxblk + bx].
__device__ __forceinline__ void wf_flush_slots(const double* red, int nslot, int nw, const int* ids,
                                               double* part_b, int maxblk, int bx) {
  for (int i = threadIdx.x; i < nslot; i += blockDim.x) {
    double acc = 0.0;
    for (int w = 0; w < nw; ++w) acc += red[i * nw + w];
    part_b[(size_t)ids[i] * maxblk + bx] = acc;
  }
}

template <typename T>
__device__ __forceinline__ double wf_wdot(V2<T> a, V2<T> b, int kx) {
  const T d = a.x * b.x + a.y * b.y;
  return kx == 0 ? (double)d : 2.0 * (double)d;
}

// A thread's share of a streaming chunk: WF_COMB_EPT complex values as
// NV = WF_COMB_EPT / VW vector loads of VW complex values each (16 bytes).
template <typename T> struct WfVec;
template <> struct WfVec<float> {
  typedef float4 type;
  static constexpr int VW = 2;
};
template <> struct WfVec<double> {
  typedef double2 type;
  static constexpr int VW = 1;
};

template <typename T>
__device__ __forceinline__ typename WfVec<T>::type wf_vaxpy(typename WfVec<T>::type y, T a,
                                                            typename WfVec<T>::type x) {
  typename WfVec<T>::type r;
  if constexpr (sizeof(T) == 4) {
    r.x = y.x + a * x.x; r.y = y.y + a * x.y; r.z = y.z + a * x.z; r.w = y.w + a * x.w;
  } else {
    r.x = y.x + a * x.x; r.y = y.y + a * x.y;
  }
  return r;
}
template <typename T>
__device__ __forceinline__ typename WfVec<T>::type wf_vscale(typename WfVec<T>::type x, T a) {
  typename WfVec<T>::type r;
  if constexpr (sizeof(T) == 4) {
    r.x = a * x.x; r.y = a * x.y; r.z = a * x.z; r.w = a * x.w;
  } else {
    r.x = a * x.x; r.y = a * x.y;
  }
  return r;
}
// Weighted dot of two vector loads starting at complex index `off` of a map
// vector whose rows hold h packed columns (weight 1 on column 0, 2 elsewhere).
template <typename T>
__device__ __forceinline__ float wf_vdotf(typename WfVec<T>::type a, typename WfVec<T>::type b, int kx) {
  if constexpr (sizeof(T) == 4) {
    const float d0 = a.x * b.x + a.y * b.y, d1 = a.z * b.z + a.w * b.w;
    return (kx == 0 ? d0 : 2.f * d0) + 2.f * d1;  // kx even, so kx + 1 >= 1
  } else {
    return 0.f;
  }
}
template <typename T>
__device__ __forceinline__ double wf_vdotd(typename WfVec<T>::type a, typename WfVec<T>::type b, int kx) {
  if constexpr (sizeof(T) == 8) {
    const double d0 = a.x * b.x + a.y * b.y;
    return kx == 0 ? d0 : 2.0 * d0;
  } else {
    return (double)wf_vdotf<T>(a, b, kx);
  }
}

// Block sums of per-thread partial dot products pdot[slot][thread], one warp
// per slot, accumulated in FP64 in a fixed order.
__device__ __forceinline__ void wf_reduce_pdots(const float* pdot, int nslot, const int* ids, double* part_b,
                                                int maxblk, int bx) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = wid; k < nslot; k += nw) {
    double v = 0.0;
    for (int i = lane; i < (int)blockDim.x; i += 32) v += (double)pdot[k * blockDim.x + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) part_b[(size_t)ids[k] * maxblk + bx] = v;
  }
}

// Shared memory of the streaming kernels: per-thread partial dot products,
// [2m + 1][threads] floats.
template <typename T>
constexpr size_t wf_comb_smem(int m) {
  return (size_t)(2 * m + 1) * WF_COMB_THREADS * sizeof(float);
}

// ---------------------------------------------------------------------------
// k_lb_comb: grid (ncomb, B).  A block walks g.sgroup consecutive
// chunks of WF_COMB_CHUNK complex values of the map's packed vectors (fewer for
// small maps), summing its partial dot products once at the end.  Each thread owns
// WF_COMB_EPT complex values of the chunk; the stored vectors are read with
// plain 16-byte loads, one pair (Q, P) per trip, newest first, at the
// occupancy needed to keep HBM busy.  The pending update always belongs to the
// newest pair, whose slot is `head`.
// ---------------------------------------------------------------------------
#ifndef WF_COMB_MINB
#define WF_COMB_MINB 4
#endif
template <typename T>
__device__ __forceinline__ void wf_lb_comb(const WfGeo& g, const WfLbBufs& lb, double* part, int mode,
                                           const WfBlk kb) {
  typedef typename WfVec<T>::type VT;
  constexpr int VW = WfVec<T>::VW, NV = WF_COMB_EPT / VW;
  extern __shared__ __align__(16) unsigned char wf_smem[];
  float* pdot = (float*)wf_smem;  // [2m + 1][threads], this thread's column only until the final sums
  __shared__ int ids[2 * WF_MAXM + 1];
  const int b = kb.y, tid = threadIdx.x;
  const WfLbMap* M = lb.st + b;
  const int active = M->active;
  const double pa = M->pend_alpha;
  const int m = lb.m;
  // steps taken but not in s yet: k - s_k of them, the newest in slot head
  const int unfolded = M->k - M->s_k;
  if (mode == WF_LB1_FULL && !active && pa == 0.0 && unfolded == 0) return;
  if (mode == WF_LB1_MATERIALIZE && pa == 0.0 && unfolded == 0) return;
  if (mode == WF_LB1_FULL && !active) mode = WF_LB1_MATERIALIZE;  // deactivated: finish its state only
  const bool gup = (pa != 0.0 && mode != WF_LB1_DOTS);  // the pending step, into g
  const int nfold = (mode == WF_LB1_DOTS) ? 0
                    : (mode == WF_LB1_MATERIALIZE || unfolded >= wf_sfold(m)) ? unfolded : 0;  // into s now
  const bool full = (mode == WF_LB1_FULL);
  const size_t vsz = (size_t)g.C * g.n * g.h;  // complex values per map vector
  const int h = g.h, B = kb.ny;
  const V2<T>* ring = (const V2<T>*)lb.ring;
  const int head = M->head;
  const int np = (mode == WF_LB1_MATERIALIZE) ? 0 : M->npairs;  // pairs of the direction and dots
  const int nq = np > nfold ? np : nfold;  // slots streamed (newest first)
  const int nslot = 1 + 2 * np;
  if (mode != WF_LB1_MATERIALIZE) {
    for (int k = 0; k < nslot; ++k) pdot[k * WF_COMB_THREADS + tid] = 0.f;
    if (tid == 0) {
      ids[0] = WF_SLOT_GG;
      for (int q = 0; q < np; ++q) {
        const int sl = (head - q + m) % m;
        ids[1 + 2 * q] = WF_SLOT_GQ + sl;
        ids[2 + 2 * q] = WF_SLOT_GP + sl;
      }
    }
  }
  const T dg = (T)M->dg;
  for (int cg = 0; cg < g.sgroup; ++cg) {
    const size_t c0 = ((size_t)kb.x * g.sgroup + cg) * WF_COMB_CHUNK;
    if (c0 >= vsz) break;
    const int clen = (int)((vsz - c0) < (size_t)WF_COMB_CHUNK ? (vsz - c0) : (size_t)WF_COMB_CHUNK);
    VT* sv = (VT*)((V2<T>*)lb.s + (size_t)b * vsz + c0);
    VT* gv = (VT*)((V2<T>*)lb.g + (size_t)b * vsz + c0);
    int u[NV];
    bool ok[NV], col0[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int c = (tid + i * WF_COMB_THREADS) * VW;
      ok[i] = c < clen;
      u[i] = (int)(WF_CHK_IF(ok[i], c0 + c, vsz) - c0) / VW;  // the map vector's element c0 + c
      col0[i] = ((c0 + c) % h) == 0;
    }
    auto wdot = [&](VT a, VT c, int i) -> float {
      if constexpr (sizeof(T) == 4) {
        const float d0 = a.x * c.x + a.y * c.y, d1 = a.z * c.z + a.w * c.w;
        return (col0[i] ? d0 : 2.f * d0) + 2.f * d1;
      } else {
        const double d0 = a.x * c.x + a.y * c.y;
        return (float)(col0[i] ? d0 : 2.0 * d0);
      }
    };
    VT gr[NV], sr[NV], pr[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (ok[i]) {
        if (mode != WF_LB1_MATERIALIZE || gup) gr[i] = gv[u[i]];
        if (nfold) sr[i] = sv[u[i]];
        if (full) pr[i] = wf_vscale<T>(gr[i], (T)0);
      }
    for (int q = 0; q < nq; ++q) {
      const int sl = (head - q + m) % m;
      const VT* Pq = (const VT*)(ring + ((size_t)sl * B + b) * vsz + c0);
      const VT* Qq = (const VT*)(ring + ((size_t)(m + sl) * B + b) * vsz + c0);
      const bool useq = q < np || (gup && q == 0);
      VT xp[NV], xq[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (ok[i]) {
          if (useq) xq[i] = Qq[u[i]];
          xp[i] = Pq[u[i]];
        }
      if (gup && q == 0) {  // the newest pair carries the pending update of g
#pragma unroll
        for (int i = 0; i < NV; ++i)
          if (ok[i]) {
            gr[i] = wf_vaxpy<T>(gr[i], (T)pa, xq[i]);
            gv[u[i]] = gr[i];
          }
      }
      if (q < nfold) {  // step of this pair into s
        const T as = (T)M->alpha[sl];
#pragma unroll
        for (int i = 0; i < NV; ++i)
          if (ok[i]) sr[i] = wf_vaxpy<T>(sr[i], as, xp[i]);
      }
      if (q >= np) continue;
      const T cq = (T)M->dQ[sl], cp = (T)M->dP[sl];
      float aq = 0.f, ap = 0.f;
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (ok[i]) {
          aq += wdot(gr[i], xq[i], i);
          ap += wdot(gr[i], xp[i], i);
          if (full) pr[i] = wf_vaxpy<T>(wf_vaxpy<T>(pr[i], cq, xq[i]), cp, xp[i]);
        }
      pdot[(1 + 2 * q) * WF_COMB_THREADS + tid] += aq;
      pdot[(2 + 2 * q) * WF_COMB_THREADS + tid] += ap;
    }
    if (nfold) {
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (ok[i]) sv[u[i]] = sr[i];
    }
    if (mode == WF_LB1_MATERIALIZE) continue;
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (ok[i]) {
        acc += wdot(gr[i], gr[i], i);
        if (full) pr[i] = wf_vaxpy<T>(pr[i], dg, gr[i]);
      }
    pdot[tid] += acc;
    if (full) {
      VT* Pn = (VT*)((V2<T>*)ring + ((size_t)M->next * B + b) * vsz + c0);
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (ok[i]) Pn[u[i]] = pr[i];
    }
  }
  if (mode == WF_LB1_MATERIALIZE) return;
  __syncthreads();
  wf_reduce_pdots(pdot, nslot, ids, part + (size_t)b * WF_NSLOT * g.maxblk, g.maxblk, kb.x);
}
template <typename T>
__global__ void __launch_bounds__(WF_COMB_THREADS, sizeof(T) == 4 ? WF_COMB_MINB : 2)
k_lb_comb(WfGeo g, WfLbBufs lb, double* part, int mode) {
  wf_lb_comb<T>(g, lb, part, mode, wf_blk());
}

// ---------------------------------------------------------------------------
// k_lb_qdots: grid (ncomb, B).  <q, Q_i> for the stored Q_i other than q, four
// stored vectors per trip, over the same chunk groups as k_lb_comb.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void wf_lb_qdots(const WfGeo& g, const WfLbBufs& lb, double* part, const WfBlk kb) {
  typedef typename WfVec<T>::type VT;
  constexpr int VW = WfVec<T>::VW, NV = WF_COMB_EPT / VW;
  extern __shared__ __align__(16) unsigned char wf_smem[];
  float* pdot = (float*)wf_smem;
  __shared__ int ids[WF_MAXM];
  const int b = kb.y, tid = threadIdx.x;
  const WfLbMap* M = lb.st + b;
  if (!M->active) return;
  const size_t vsz = (size_t)g.C * g.n * g.h;
  const int h = g.h, B = kb.ny, m = lb.m;
  const V2<T>* ring = (const V2<T>*)lb.ring;
  const int nx = M->next, np = M->npairs, head = M->head;
  __shared__ const VT* qv[WF_MAXM];  // the stored Q other than q, newest first
  const int nvec = np - ((head - nx + m) % m < np ? 1 : 0);
  if (tid == 0) {
    int v = 0;
    for (int q = 0; q < np; ++q) {
      const int sl = (head - q + m) % m;
      if (sl == nx) continue;
      qv[v] = (const VT*)(ring + ((size_t)(m + sl) * B + b) * vsz);
      ids[v++] = WF_SLOT_QQI + sl;
    }
  }
  for (int v = 0; v < nvec; ++v) pdot[v * WF_COMB_THREADS + tid] = 0.f;
  __syncthreads();
  for (int cg = 0; cg < g.sgroup; ++cg) {
    const size_t c0 = ((size_t)kb.x * g.sgroup + cg) * WF_COMB_CHUNK;
    if (c0 >= vsz) break;
    const int clen = (int)((vsz - c0) < (size_t)WF_COMB_CHUNK ? (vsz - c0) : (size_t)WF_COMB_CHUNK);
    int u[NV];
    bool ok[NV], col0[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int c = (tid + i * WF_COMB_THREADS) * VW;
      ok[i] = c < clen;
      u[i] = (int)(WF_CHK_IF(ok[i], c0 + c, vsz) - c0) / VW;  // the map vector's element c0 + c
      col0[i] = ((c0 + c) % h) == 0;
    }
    auto wdot = [&](VT a, VT c, int i) -> float {
      if constexpr (sizeof(T) == 4) {
        const float d0 = a.x * c.x + a.y * c.y, d1 = a.z * c.z + a.w * c.w;
        return (col0[i] ? d0 : 2.f * d0) + 2.f * d1;
      } else {
        const double d0 = a.x * c.x + a.y * c.y;
        return (float)(col0[i] ? d0 : 2.0 * d0);
      }
    };
    const VT* Qn = (const VT*)(ring + ((size_t)(m + nx) * B + b) * vsz + c0);
    VT qr[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (ok[i]) qr[i] = Qn[u[i]];
    constexpr int U = 4;  // stored vectors per trip
    for (int w = 0; w < nvec; w += U) {
      VT x[U][NV];
#pragma unroll
      for (int v = 0; v < U; ++v) {
        const VT* Qv = qv[w + v < nvec ? w + v : w] + c0 / VW;
#pragma unroll
        for (int i = 0; i < NV; ++i)
          if (ok[i] && w + v < nvec) x[v][i] = Qv[u[i]];
      }
#pragma unroll
      for (int v = 0; v < U; ++v) {
        if (w + v >= nvec) break;
        float a = 0.f;
#pragma unroll
        for (int i = 0; i < NV; ++i)
          if (ok[i]) a += wdot(qr[i], x[v][i], i);
        pdot[(w + v) * WF_COMB_THREADS + tid] += a;
      }
    }
  }
  __syncthreads();
  wf_reduce_pdots(pdot, nvec, ids, part + (size_t)b * WF_NSLOT * g.maxblk, g.maxblk, kb.x);
}
template <typename T>
__global__ void __launch_bounds__(WF_COMB_THREADS, sizeof(T) == 4 ? 4 : 2)
k_lb_qdots(WfGeo g, WfLbBufs lb, double* part) {
  wf_lb_qdots<T>(g, lb, part, wf_blk());
}

// ---------------------------------------------------------------------------
// Column stages of the Hessian-vector product on p = P[next] of each map.
// ---------------------------------------------------------------------------
// One block per column tile; KIND WF_COLINV_PP_K (ping-pong passes) or
// WF_COLINV_INPLACE_K (in-place passes).
template <typename T, int C, int KIND, int PLAN>
__device__ __forceinline__ void wf_lb_colinv(const WfGeo& g, const T* sp_, long long sp_stride, void* scratch_,
                                             const void* tw_, const WfLbBufs& lb, const WfBlk kb) {
  const int b = kb.y;
  const WfLbMap* M = lb.st + b;
  if (!M->active) return;
  const size_t vsz = (size_t)C * g.n * g.h;
  const V2<T>* p = (const V2<T>*)lb.ring + ((size_t)M->next * kb.ny + b) * vsz;
  if constexpr (KIND == WF_COLINV_PP_K)
    wf_col_inv_pp<T, C, WF_IN_PK, PLAN>(g, p, sp_ + (size_t)b * sp_stride, (V2<T>*)scratch_ + (size_t)b * vsz, tw_,
                                        kb.x * g.TC);
  else
    wf_col_inv_body<T, C, WF_IN_PK>(g, p, sp_ + (size_t)b * sp_stride, (V2<T>*)scratch_ + (size_t)b * vsz, tw_,
                                    kb.x * g.TC);
}
template <typename T, int C, int KIND, int PLAN>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB_PLAN(T, PLAN))
k_lb_colinv(WfGeo g, const T* sp_, long long sp_stride, void* scratch_, const void* tw_, WfLbBufs lb) {
  wf_lb_colinv<T, C, KIND, PLAN>(g, sp_, sp_stride, scratch_, tw_, lb, wf_blk());
}

// Persistent inverse column stage with the next tile prefetched by TMA.
// Shared memory: the TMA tile Ct ([C n][TC] packed values), the ping-pong
// tiles A and B, the pass table.  Work items (map, column tile) are taken
// round-robin by the resident blocks; while a block runs the second and third
// FFT passes of one tile, the copy engine brings in the next tile, whose first
// pass then reads shared memory (the per-mode operator R sqrt(P)/n applied on
// the way in, as in wf_col_inv_pp).  tm: 2-D view of the whole history ring,
// rows of h = nx/2 packed values; the map's direction P[next] is rows
// ((next B + b) C ny + r).
template <typename T>
__host__ __device__ constexpr size_t wf_colinv_tma_smem() {
  return (3 * (size_t)WF_TILE + WF_NT) * sizeof(V2<T>) + 128;  // + room to align the TMA tile to 128 B
}
template <typename T, int C, int PLAN>
__global__ void __launch_bounds__(WF_THREADS, sizeof(T) == 4 ? 2 : 1)
k_lb_colinv_tma(WfGeo g, const T* sp_, long long sp_stride, void* scratch_, const void* tw_, WfLbBufs lb, int B,
                const __grid_constant__ CUtensorMap tm) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  V2<T>* Ct = (V2<T>*)(wf_smem + ((128u - (wf_smem_u32(wf_smem) & 127u)) & 127u));  // TMA destination, 128 B aligned
  V2<T>* A = Ct + WF_TILE;
  V2<T>* Bf = A + WF_TILE;
  V2<T>* s_tw = Bf + WF_TILE;
  __shared__ uint64_t full;
  const int tid = threadIdx.x;
  const int n = g.n, h = g.h, lgn = g.lgn, TC = g.TC, lgTC = __ffs(TC) - 1;
  const int CT = C * TC, lgCT = lgTC + (C == 2 ? 1 : 0);
  const int nitems = B * g.ntile;
  const int rows = C * n, boxr = rows < 256 ? rows : 256;
  const uint32_t tile_bytes = (uint32_t)(rows * TC * sizeof(V2<T>));
  const size_t vsz = (size_t)C * n * h;
  wf_stage_tw<T>(s_tw, (const V2<T>*)tw_, lgn, PLAN);
  if (tid == 0) {
    wf_mbar_init(&full, 1);
    wf_mbar_fence_init();
  }
  __syncthreads();
  auto next_active = [&](int it) {
    while (it < nitems && !lb.st[it / g.ntile].active) it += gridDim.x;
    return it;
  };
  // thread 0: the tile of work item `it` into Ct.  Returns whether a copy was
  // issued (never for the map a diagnostic run names in inject_map).
  auto issue = [&](int it) -> bool {
    const int b = it / g.ntile, tile = it - b * g.ntile;
    if (b == lb.inject_map) return false;
    const int row0 = (lb.st[b].next * B + b) * rows;
    wf_mbar_expect_tx(&full, tile_bytes);
    for (int r = 0; r < rows; r += boxr) wf_tma_load_2d(Ct + (size_t)r * TC, &tm, 2 * tile * TC, row0 + r, &full);
    return true;
  };
  int it = next_active(blockIdx.x);
  uint32_t parity = 0;
  bool pending = false;  // a copy into Ct is in flight (thread 0's view)
  if (tid == 0 && it < nitems) pending = issue(it);
  while (it < nitems) {
    const int b = it / g.ntile, tile = it - b * g.ntile, kx0 = tile * TC;
    const T* sp = sp_ + (size_t)b * sp_stride;
    V2<T>* scr = (V2<T>*)scratch_ + (size_t)b * vsz;
    // A block-wide decision: every thread waits (bounded); if any gave up, the
    // tile never arrived and the block stops.  Its current and remaining maps
    // are marked WF_ETIMEOUT (none of them computes on missing data), and it
    // returns after letting a copy it issued land.  That drain wait is bounded
    // too, by at least the default limit (about 2 s), however short the
    // caller's limit: a 2-D tile copy that was issued lands within
    // microseconds, so a block leaves with a copy still writing into its
    // shared memory only on a device that no longer makes progress at all.
    const bool late = !wf_mbar_wait(&full, parity, lb.spin_limit);
    if (__syncthreads_or(late)) {
      if (tid == 0) {
        for (int r = it; r < nitems; r = next_active(r + gridDim.x)) lb.st[r / g.ntile].status = WF_ETIMEOUT;
        if (pending)
          wf_mbar_wait(&full, parity, lb.spin_limit > WF_WAIT_CYCLES_DEFAULT ? lb.spin_limit : WF_WAIT_CYCLES_DEFAULT);
      }
      return;
    }
    parity ^= 1u;
    auto ld0 = [&](int t, int row) -> V2<T> {
      const int c = t >> lgTC, col = t & (TC - 1);
      auto lds = [&](int cc, int rr) { return Ct[WF_CHK((size_t)(cc * n + rr) * TC + col, WF_TILE)]; };
      return wf_mode_packed<T, C, false>(lds, row, c, kx0 + col, g, sp);
    };
    auto stl = [&](int t, int row, V2<T> v) {
      scr[WF_CHK(((size_t)(t >> lgTC) * n + row) * h + kx0 + (t & (TC - 1)), vsz)] = v;
    };
    const int itn = next_active(it + gridDim.x);
    auto after1 = [&]() {  // every thread is done with Ct: bring in the next tile
      if (tid == 0) pending = itn < nitems ? issue(itn) : false;
    };
    wf_pp_fft<T, +1, true, PLAN>(lgn, lgCT, 1, CT, A, Bf, s_tw, ld0, stl, after1);
    it = itn;
  }
}

template <typename T, int C>
__device__ __forceinline__ void wf_lb_colfwd(const WfGeo& g, const T* sp_, long long sp_stride, const void* scratch_,
                                             const void* tw_, const WfLbBufs& lb, double* part, const WfBlk kb) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  const int b = kb.y;
  const WfLbMap* M = lb.st + b;
  if (!M->active) return;
  V2<T>* s_tw = (V2<T>*)wf_smem;
  V2<T>* buf = s_tw + WF_NT;
  const int n = g.n, h = g.h, lgn = g.lgn, TC = g.TC, lgTC = __ffs(TC) - 1, CT = C * TC;
  const int kx0 = kb.x * TC, tot = C * n * TC;
  const size_t vsz = (size_t)C * n * h;
  const int B = kb.ny, m = lb.m, nx = M->next;
  const V2<T>* Pn = (const V2<T>*)lb.ring + ((size_t)nx * B + b) * vsz;
  V2<T>* Qn = (V2<T>*)lb.ring + ((size_t)(m + nx) * B + b) * vsz;
  const V2<T>* gv = (const V2<T>*)lb.g + (size_t)b * vsz;
  typedef WfAcc<T> A;
  A qq = 0, pq = 0, pp = 0, gq = 0, gp = 0;
  wf_col_fwd_front<T, C>(g, (const V2<T>*)scratch_ + (size_t)b * vsz, sp_ + (size_t)b * sp_stride, buf, s_tw,
                         tw_, kx0);
  constexpr int EB = WF_EMAX;
  // element ii of this thread: packed row r = r0 + ii * rstep (rows c n + j of
  // the C channels), column kx0 + t, fixed for the thread (blockDim is a
  // multiple of TC); offsets fit 32 bits (C n h <= 2^20)
  const int t = threadIdx.x & (TC - 1), r0 = threadIdx.x >> lgTC, rstep = WF_THREADS >> lgTC;
  const int kx = kx0 + t;
  const A wk = kx == 0 ? (A)1 : (A)2;
  const V2<T>* Pb = Pn + kx;
  const V2<T>* gb = gv + kx;
  V2<T>* Qb = Qn + kx;
  const int rows = C * n;
  // the thread's EB rows in WF_LBCF_SPLIT groups: the loads of a group are
  // issued together, and fewer values are live at once the more groups
  constexpr int EG = EB / WF_LBCF_SPLIT;
#pragma unroll
  for (int g0 = 0; g0 < EB; g0 += EG) {
    V2<T> pl[EG], gl[EG];
#pragma unroll
    for (int i = 0; i < EG; ++i) {
      const int r = r0 + (g0 + i) * rstep;
      if (r < rows) {
        pl[i] = Pb[WF_CHK((size_t)r * h + kx, vsz) - kx];
        gl[i] = gb[WF_CHK((size_t)r * h + kx, vsz) - kx];
      }
    }
#pragma unroll
    for (int i = 0; i < EG; ++i) {
      const int ii = i;
      const int r = r0 + (g0 + i) * rstep;
      if (r < rows) {
        const int j = r & (n - 1), c = r >> lgn;
        const V2<T> a = buf[wf_sw<T>(j * CT + c * TC + t)];
        const V2<T> p = pl[ii], gg = gl[ii];
        const V2<T> q = mk<T>((T)2 * (p.x - a.x), (T)2 * (p.y - a.y));
        Qb[WF_CHK((size_t)r * h + kx, vsz) - kx] = q;
        qq += wk * (A)(q.x * q.x + q.y * q.y);
        pq += wk * (A)(p.x * q.x + p.y * q.y);
        pp += wk * (A)(p.x * p.x + p.y * p.y);
        gq += wk * (A)(gg.x * q.x + gg.y * q.y);
        gp += wk * (A)(gg.x * p.x + gg.y * p.y);
      }
    }
  }
  __shared__ double red[5 * (WF_THREADS / 32)];
  __shared__ int ids[5];
  wf_warp_stash((double)qq, red, 0, WF_THREADS / 32);
  wf_warp_stash((double)pq, red, 1, WF_THREADS / 32);
  wf_warp_stash((double)pp, red, 2, WF_THREADS / 32);
  wf_warp_stash((double)gq, red, 3, WF_THREADS / 32);
  wf_warp_stash((double)gp, red, 4, WF_THREADS / 32);
  if (threadIdx.x == 0) {
    ids[0] = WF_SLOT_QQ; ids[1] = WF_SLOT_PQ; ids[2] = WF_SLOT_PP; ids[3] = WF_SLOT_GQN; ids[4] = WF_SLOT_GPN;
  }
  __syncthreads();
  wf_flush_slots(red, 5, WF_THREADS / 32, ids, part + (size_t)b * WF_NSLOT * g.maxblk, g.maxblk, kb.x);
}
template <typename T, int C>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB_LBCOLFWD(T, C))
k_lb_colfwd(WfGeo g, const T* sp_, long long sp_stride, const void* scratch_, const void* tw_, WfLbBufs lb,
            double* part) {
  wf_lb_colfwd<T, C>(g, sp_, sp_stride, scratch_, tw_, lb, part, wf_blk());
}

// Row stage of the Hessian-vector product for the maps still iterating.
// KIND WF_ROW_PP_K (ping-pong passes) or WF_ROW_INPLACE_K (in-place passes).
template <typename T, int KIND, int PLAN>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB_PLAN(T, PLAN))
k_lb_row(WfGeo g, void* scratch_, const void* w_, double* part, const void* tw_, const WfLbMap* st) {
  if (!st[blockIdx.y].active) return;
  if constexpr (KIND == WF_ROW_PP_K)
    wf_row_pp<T, WF_ROW_NODATA, PLAN>(g, (V2<T>*)scratch_, nullptr, (const T*)w_, part, tw_);
  else
    k_row_body<T, WF_ROW_NODATA>(g, scratch_, nullptr, w_, nullptr, nullptr, part, tw_);
}
