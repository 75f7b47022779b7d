// Operator kernels of the Wiener-filter objective (Sec. 2.2, eq_chi / eq_cost).
//
// One objective+gradient pass over a batch of ny x nx maps (n = ny rows of
// nx pixels, h = nx/2 packed columns) is three stages:
//   inverse column stage: load a tile of packed spectrum columns, multiply by
//     R(k) sqrt(P)/n (step A1), inverse FFT along y (first half of A2), store
//     the tile to scratch (k_col_inv; the ping-pong form k_col_inv_pp_pers in
//     wf_stage_pp.cuh);
//   row stage: c2r along x (rest of A2), pixel residual r = d - x, wr = w r
//     and the data term sum r w r (A3), r2c of wr along x (first half of A4),
//     store back to scratch (k_row; k_row_pp in wf_stage_pp.cuh);
//   forward column stage: forward FFT along y (rest of A4), sqrt(P) R(k)^T / n
//     (adjoint, A5), g = 2 (s - .), prior term sum |s|^2, store g
//     (k_col_fwd).
// Spectra are held in a packed half-plane layout [ny][nx/2] in which column 0
// carries the two self-conjugate columns kx = 0 and kx = nx/2 as X0 + i Xh;
// the column FFT of that packed column is then an ordinary complex FFT whose
// real and imaginary parts are the two real row-DC / row-Nyquist signals.
// Only per-mode operations unpack it, pairing ky with ny - ky.  The scale
// written sqrt(P)/n below is sqrt(P / (ny nx)), the unitary normalisation.
#pragma once
#include "wf_fft.cuh"
#include "wf_internal.h"

template <typename T> __device__ __forceinline__ bool wf_isfinite(T x) { return isfinite(x); }

// Sum over the block of one double per thread; valid in thread 0.
__device__ __forceinline__ double wf_block_sum(double v) {
  __shared__ double red[WF_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < WF_THREADS / 32; ++i) r += red[i];
  }
  return r;
}

// Ask L2 to fetch `rows` segments of `seg` bytes, `stride` bytes apart, from
// `base` (one request per 128-byte line, spread over the block's threads), so
// that loads issued later in the kernel find them there.
__device__ __forceinline__ void wf_prefetch_rows(const void* base, int rows, size_t stride, int seg) {
  const int lpr = (seg + 127) >> 7, tot = rows * lpr;
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int r = i / lpr, l = i - r * lpr;
    const char* a = (const char*)base + (size_t)r * stride + ((size_t)l << 7);
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
  }
}

// Stage the roots of unity (lgL = 0) or the pass table of length 2^lgL of
// radix plan `plan`.
template <typename T>
__device__ __forceinline__ void wf_stage_tw(V2<T>* s_tw, const V2<T>* g_tw, int lgL = 0, int plan = 0) {
  const V2<T>* src = g_tw + (size_t)WF_TWTAB * plan + (size_t)WF_NT * lgL;
  for (int i = threadIdx.x; i < WF_NT; i += blockDim.x) s_tw[i] = src[i];
}

// Kaiser-Squires cosine / sine of half-plane mode (row j, column kx), kx in
// [0, nx/2]: c = (qx^2 - qy^2)/q^2, s = 2 qx qy / q^2 for the wavevector
// q = (ksx kx, ksy my) of the mode, my the signed row frequency (row ny/2
// taken as -ny/2; on square maps q is the pair of mode numbers); s = 0 on the
// Nyquist row and column, and R = identity at k = 0 (App. C operator divided
// by -k^2).
template <typename T>
__device__ __forceinline__ void wf_ks(int kx, int j, const WfGeo& g, T& c, T& s) {
  const int hy = g.n >> 1;
  const int ky = j < hy ? j : j - g.n;
  const int qx = kx * g.ksx, qy = ky * g.ksy;
  const int k2 = qx * qx + qy * qy;
  if (k2 == 0) { c = (T)1; s = (T)0; return; }
  const T inv = (T)1 / (T)k2;
  c = (T)(qx * qx - qy * qy) * inv;
  s = (kx == g.h || ky == -hy) ? (T)0 : (T)(2 * qx * qy) * inv;
}

// Per-mode operator on the C channel values of one mode.
//   forward (ADJ = false): v <- R(k) diag(sp) v * extra        (step A1)
//   adjoint (ADJ = true):  v <- diag(sp) R(k)^T v * extra      (step A5)
// wf_mode_op_pre takes a0, a1 = the two channels' sqrt(P)/n times extra (a1
// unused for C = 1); wf_mode_op reads them from sp, this map's [C][ny][nx/2+1]
// table of sqrt(P)/n.
template <typename T, int C, bool ADJ>
__device__ __forceinline__ void wf_mode_op_pre(V2<T>* v, int j, int kx, const WfGeo& g, T a0, T a1) {
  if constexpr (C == 1) {
    v[0] = cscale<T>(v[0], a0);
  } else {
    T c, s;
    wf_ks<T>(kx, j, g, c, s);
    if constexpr (!ADJ) {
      const V2<T> e = cscale<T>(v[0], a0), b = cscale<T>(v[1], a1);
      v[0] = mk<T>(c * e.x - s * b.x, c * e.y - s * b.y);
      v[1] = mk<T>(s * e.x + c * b.x, s * e.y + c * b.y);
    } else {
      const V2<T> e = v[0], b = v[1];
      v[0] = cscale<T>(mk<T>(c * e.x + s * b.x, c * e.y + s * b.y), a0);
      v[1] = cscale<T>(mk<T>(-s * e.x + c * b.x, -s * e.y + c * b.y), a1);
    }
  }
}

template <typename T, int C, bool ADJ>
__device__ __forceinline__ void wf_mode_op(V2<T>* v, int j, int kx, const WfGeo& g, const T* sp, T extra) {
  const int pitch = g.h + 1;
  const T a0 = sp[j * pitch + kx] * extra;
  const T a1 = C == 2 ? sp[(size_t)g.n * pitch + j * pitch + kx] * extra : (T)0;
  wf_mode_op_pre<T, C, ADJ>(v, j, kx, g, a0, a1);
}

// Unpack the packed column value pair (Y[j], Y[ny-j]) into the kx = 0 and
// kx = nx/2 values at row j: X0 = (Y + conj Ym)/2, Xh = -i (Y - conj Ym)/2.
template <typename T>
__device__ __forceinline__ void wf_unpack0(V2<T> Y, V2<T> Ym, V2<T>& X0, V2<T>& Xh) {
  X0 = mk<T>((T)0.5 * (Y.x + Ym.x), (T)0.5 * (Y.y - Ym.y));
  const V2<T> dlt = mk<T>(Y.x - Ym.x, Y.y + Ym.y);  // Y - conj(Ym)
  Xh = mk<T>((T)0.5 * dlt.y, (T)-0.5 * dlt.x);
}
// Y = X0 + i Xh
template <typename T>
__device__ __forceinline__ V2<T> wf_pack0(V2<T> X0, V2<T> Xh) { return mk<T>(X0.x - Xh.y, X0.y + Xh.x); }

// Apply the per-mode operator to a column tile held as [ny][C*TC] in shared
// memory (element (row j, channel c, column t) at j*C*TC + c*TC + t), tile
// starting at packed column kx0.  The packed column 0 is unpacked in pairs.
template <typename T, bool SWP>
__device__ __forceinline__ int wf_swz(int x) {
  if constexpr (SWP) return wf_swp<T>(x);
  else return wf_sw<T>(x);
}
template <typename T, int C, bool ADJ, bool SWP = false>
__device__ __forceinline__ void wf_col_scale(V2<T>* buf, const WfGeo& g, int lgTC, int kx0, const T* sp, T extra) {
  const int n = g.n, TC = 1 << lgTC, CT = C * TC, h = g.h, pitch = h + 1;
  // U elements per trip, their sqrt(P) values loaded before any is used.  A
  // thread's column t is fixed (blockDim is a multiple of TC); the packed
  // column kx = 0 is not written here (its threads' stores are predicated
  // off) and is done in pairs below.
  constexpr int U = 8;
  const int t = threadIdx.x & (TC - 1), kx = kx0 + t, jstep = blockDim.x >> lgTC;
  const bool keep = kx == 0;
  auto trip = [&](int j0, auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
    T a0[U], a1[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * jstep;
      if (FULL || j < n) {
        a0[u] = sp[j * pitch + kx];
        if constexpr (C == 2) a1[u] = sp[(size_t)n * pitch + j * pitch + kx];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int j = j0 + u * jstep;
      if (FULL || j < n) {
        V2<T> v[C];
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] = buf[wf_swz<T, SWP>(j * CT + c * TC + t)];
        wf_mode_op_pre<T, C, ADJ>(v, j, kx, g, a0[u] * extra, C == 2 ? a1[u] * extra : (T)0);
        if (!keep) {
#pragma unroll
          for (int c = 0; c < C; ++c) buf[wf_swz<T, SWP>(j * CT + c * TC + t)] = v[c];
        }
      }
    }
  };
  const int full_trips = n / (U * jstep);
  int j0 = threadIdx.x >> lgTC;
  for (int i = 0; i < full_trips; ++i, j0 += U * jstep) trip(j0, std::true_type());
  if (j0 < n) trip(j0, std::false_type());
  if (kx0 == 0) {
    for (int j = threadIdx.x; j <= (n >> 1); j += blockDim.x) {
      const int jm = (n - j) & (n - 1);
      V2<T> X0[C], Xh[C], X0m[C], Xhm[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const V2<T> Y = buf[wf_swz<T, SWP>(j * CT + c * TC)], Ym = buf[wf_swz<T, SWP>(jm * CT + c * TC)];
        wf_unpack0<T>(Y, Ym, X0[c], Xh[c]);
        wf_unpack0<T>(Ym, Y, X0m[c], Xhm[c]);
      }
      wf_mode_op<T, C, ADJ>(X0, j, 0, g, sp, extra);
      wf_mode_op<T, C, ADJ>(Xh, j, h, g, sp, extra);
      wf_mode_op<T, C, ADJ>(X0m, jm, 0, g, sp, extra);
      wf_mode_op<T, C, ADJ>(Xhm, jm, h, g, sp, extra);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        buf[wf_swz<T, SWP>(j * CT + c * TC)] = wf_pack0<T>(X0[c], Xh[c]);
        buf[wf_swz<T, SWP>(jm * CT + c * TC)] = wf_pack0<T>(X0m[c], Xhm[c]);
      }
    }
  }
}

// Load a column tile of a spectrum given either packed ([C][n][h]) or in the
// standard rfft2 layout ([C][n][h+1]); the tile is stored packed.
template <typename T, int C, int IN>
__device__ __forceinline__ V2<T> wf_load_spec(const V2<T>* src, int c, int j, int kx, int n, int h) {
  if constexpr (IN == WF_IN_PK) {
    return src[WF_CHK(((size_t)c * n + j) * h + kx, (size_t)C * n * h)];
  } else {
    const V2<T>* row = src + WF_CHK(((size_t)c * n + j) * (h + 1), (size_t)C * n * (h + 1) - h);
    if (kx == 0) return wf_pack0<T>(row[0], row[h]);
    return row[WF_CHK(kx, h + 1)];
  }
}

// Position of element e of a column tile: pairs (FP32, 16-byte loads) or
// single complex values.  Tile element (row j, channel c, column t) lives at
// buf[j*C*TC + c*TC + t]; in the packed vector at ((c*n + j)*h + kx0 + t).
template <typename T, int C, int IN>
__device__ __forceinline__ void wf_tile_load(V2<T>* buf, const V2<T>* src, int n, int h, int lgTC, int kx0) {
  const int TC = 1 << lgTC, CT = C * TC, lgn = __ffs(n) - 1, tot = C * n * TC;
  if constexpr (IN == WF_IN_PK && sizeof(T) == 4) {
    if (TC >= 2) {
      // a thread's column pair t is fixed (blockDim is a multiple of TC / 2);
      // its rows r = r0 + i rstep (rows c n + j of the channels), packed
      // offset r h + kx0 + t in 32 bits
      const int lgP = lgTC - 1, rows = C * n;
      const int t = (threadIdx.x & ((1 << lgP) - 1)) << 1, r0 = threadIdx.x >> lgP, rstep = WF_THREADS >> lgP;
      const V2<T>* sb = src + kx0 + t;
      float4 v[WF_EMAX / 2];
#pragma unroll
      for (int i = 0; i < WF_EMAX / 2; ++i) {
        const int r = r0 + i * rstep;
        if (r < rows) v[i] = *(const float4*)(sb + WF_CHK((size_t)r * h + kx0 + t, (size_t)rows * h - 1) - kx0 - t);
      }
#pragma unroll
      for (int i = 0; i < WF_EMAX / 2; ++i) {
        const int r = r0 + i * rstep;
        if (r < rows) {
          const int x = (r & (n - 1)) * CT + (r >> lgn) * TC + t;
          buf[wf_sw<T>(x)] = mk<T>(v[i].x, v[i].y);
          buf[wf_sw<T>(x + 1)] = mk<T>(v[i].z, v[i].w);
        }
      }
      return;
    }
  }
  V2<T> v[WF_EMAX];
#pragma unroll
  for (int i = 0; i < WF_EMAX; ++i) {
    const int e = threadIdx.x + i * WF_THREADS;
    if (e < tot) {
      const int t = e & (TC - 1), r = e >> lgTC, j = r & (n - 1), c = r >> lgn;
      v[i] = wf_load_spec<T, C, IN>(src, c, j, kx0 + t, n, h);
    }
  }
#pragma unroll
  for (int i = 0; i < WF_EMAX; ++i) {
    const int e = threadIdx.x + i * WF_THREADS;
    if (e < tot) {
      const int t = e & (TC - 1), r = e >> lgTC, j = r & (n - 1), c = r >> lgn;
      buf[wf_sw<T>(j * CT + c * TC + t)] = v[i];
    }
  }
}

template <typename T, int C>
__device__ __forceinline__ void wf_tile_store_pk(V2<T>* dst, const V2<T>* buf, int n, int h, int lgTC, int kx0) {
  const int TC = 1 << lgTC, CT = C * TC, lgn = __ffs(n) - 1, tot = C * n * TC;
  if constexpr (sizeof(T) == 4) {
    if (TC >= 2) {
      // as in wf_tile_load: fixed column pair t, rows r0 + i rstep
      const int lgP = lgTC - 1, rows = C * n;
      const int t = (threadIdx.x & ((1 << lgP) - 1)) << 1, r0 = threadIdx.x >> lgP, rstep = WF_THREADS >> lgP;
      V2<T>* db = dst + kx0 + t;
#pragma unroll
      for (int i = 0; i < WF_EMAX / 2; ++i) {
        const int r = r0 + i * rstep;
        if (r < rows) {
          const int x = (r & (n - 1)) * CT + (r >> lgn) * TC + t;
          const V2<T> q0 = buf[wf_sw<T>(x)], q1 = buf[wf_sw<T>(x + 1)];
          *(float4*)(db + r * h) = make_float4(q0.x, q0.y, q1.x, q1.y);
        }
      }
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < WF_EMAX; ++i) {
    const int e = threadIdx.x + i * WF_THREADS;
    if (e < tot) {
      const int t = e & (TC - 1), r = e >> lgTC, j = r & (n - 1), c = r >> lgn;
      dst[((size_t)c * n + j) * h + kx0 + t] = buf[wf_sw<T>(j * CT + c * TC + t)];
    }
  }
}

// Contiguous copies of up to WF_TILE complex values between global and shared
// memory, every load of a thread issued before its stores (16-byte accesses).
template <typename T>
__device__ __forceinline__ void wf_g2s(V2<T>* dst, const V2<T>* src, int tot) {
  if constexpr (sizeof(T) == 4) {
    const float4* s4 = (const float4*)src;
    const int t2 = tot >> 1;
    float4 v[WF_EMAX / 2];
#pragma unroll
    for (int i = 0; i < WF_EMAX / 2; ++i) {
      const int e = threadIdx.x + i * WF_THREADS;
      if (e < t2) v[i] = s4[e];
    }
#pragma unroll
    for (int i = 0; i < WF_EMAX / 2; ++i) {
      const int e = threadIdx.x + i * WF_THREADS;
      if (e < t2) {
        dst[wf_sw<T>(2 * e)] = mk<T>(v[i].x, v[i].y);
        dst[wf_sw<T>(2 * e + 1)] = mk<T>(v[i].z, v[i].w);
      }
    }
  } else {
    V2<T> v[WF_EMAX];
#pragma unroll
    for (int i = 0; i < WF_EMAX; ++i) {
      const int e = threadIdx.x + i * WF_THREADS;
      if (e < tot) v[i] = src[e];
    }
#pragma unroll
    for (int i = 0; i < WF_EMAX; ++i) {
      const int e = threadIdx.x + i * WF_THREADS;
      if (e < tot) dst[wf_sw<T>(e)] = v[i];
    }
  }
}

template <typename T>
__device__ __forceinline__ void wf_s2g(V2<T>* dst, const V2<T>* src, int tot) {
  if constexpr (sizeof(T) == 4) {
    float4* d4 = (float4*)dst;
#pragma unroll
    for (int i = 0; i < WF_EMAX / 2; ++i) {
      const int e = threadIdx.x + i * WF_THREADS;
      if (e < (tot >> 1)) {
        const V2<T> a = src[wf_sw<T>(2 * e)], b = src[wf_sw<T>(2 * e + 1)];
        d4[e] = make_float4(a.x, a.y, b.x, b.y);
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < WF_EMAX; ++i) {
      const int e = threadIdx.x + i * WF_THREADS;
      if (e < tot) dst[e] = src[wf_sw<T>(e)];
    }
  }
}

// ---------------------------------------------------------------------------
// k_col_inv: spectrum tile -> R sqrt(P)/n -> inverse FFT along y -> scratch
// ---------------------------------------------------------------------------
template <typename T, int C, int IN>
__device__ __forceinline__ void wf_col_inv_body(const WfGeo& g, const V2<T>* src, const T* sp, V2<T>* scr,
                                                const void* tw_, int kx0 = -1) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  V2<T>* s_tw = (V2<T>*)wf_smem;
  V2<T>* buf = s_tw + WF_NT;
  const int n = g.n, lgTC = __ffs(g.TC) - 1;
  if (kx0 < 0) kx0 = blockIdx.x * g.TC;
  wf_stage_tw<T>(s_tw, (const V2<T>*)tw_, g.lgn);
  wf_tile_load<T, C, IN>(buf, src, n, g.h, lgTC, kx0);
  __syncthreads();
  wf_col_scale<T, C, false>(buf, g, lgTC, kx0, sp, (T)1);
  __syncthreads();
  fft_smem<T, +1, WF_EMAX>(buf, g.lgn, C * g.TC, 1, C * g.TC, s_tw);
  wf_tile_store_pk<T, C>(scr, buf, n, g.h, lgTC, kx0);
}

template <typename T, int C, int IN>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB(T))
k_col_inv(WfGeo g, const void* src_, const T* sp_, long long sp_stride, void* scratch_, const void* tw_) {
  const int b = blockIdx.y, n = g.n, h = g.h;
  const size_t sstride = (size_t)C * n * (IN == WF_IN_PK ? h : h + 1);
  wf_col_inv_body<T, C, IN>(g, (const V2<T>*)src_ + (size_t)b * sstride, sp_ + (size_t)b * sp_stride,
                            (V2<T>*)scratch_ + (size_t)b * C * n * h, tw_);
}

// Forward column stage shared by the gradient and Hessian-vector epilogues:
// scratch tile at packed column kx0 -> forward FFT along y -> sqrt(P) R^T / n,
// left in buf.
template <typename T, int C>
__device__ __forceinline__ void wf_col_fwd_front(const WfGeo& g, const V2<T>* scr, const T* sp, V2<T>* buf,
                                                 V2<T>* s_tw, const void* tw_, int kx0) {
  const int n = g.n, lgTC = __ffs(g.TC) - 1, CT = C * g.TC;
  wf_stage_tw<T>(s_tw, (const V2<T>*)tw_, g.lgn);
  wf_tile_load<T, C, WF_IN_PK>(buf, scr, n, g.h, lgTC, kx0);
  __syncthreads();
  fft_smem<T, -1, WF_EMAX>(buf, g.lgn, CT, 1, CT, s_tw);
  wf_col_scale<T, C, true>(buf, g, lgTC, kx0, sp, (T)1);
  __syncthreads();
}

// Epilogue of the forward column stage on a transformed, scaled tile `buf`
// ([n][C TC], swizzled as the passes that produced it: SWP for the ping-pong
// passes): out = 2 (src - a) for the tile's columns of src, dst (packed or
// standard layout); the prior partial sum |src|^2 and |out|^2 with the
// half-plane weights go to slot `slot_ix` of the map's partial sums part_b.
template <typename T, int C, int IN, bool SWP>
__device__ __forceinline__ void wf_col_fwd_out(const WfGeo& g, V2<T>* buf, const V2<T>* src, V2<T>* dst, int kx0,
                                               double* part_b, int slot_ix) {
  const int n = g.n, h = g.h, lgn = g.lgn, TC = g.TC, lgTC = __ffs(TC) - 1, CT = C * TC;
  WfAcc<T> acc = 0, acc2 = 0;  // per-thread partials; FP64 from the block sum on
  for (int e = threadIdx.x; e < C * n * TC; e += blockDim.x) {
    const int t = e & (TC - 1), r = e >> lgTC, j = r & (n - 1), c = r >> lgn;
    const int kx = kx0 + t;
    const V2<T> sv = wf_load_spec<T, C, IN>(src, c, j, kx, n, h);
    const V2<T> a = buf[wf_swz<T, SWP>(j * CT + c * TC + t)];
    const V2<T> o = mk<T>((T)2 * (sv.x - a.x), (T)2 * (sv.y - a.y));
    const T m2 = sv.x * sv.x + sv.y * sv.y;
    const T o2 = o.x * o.x + o.y * o.y;
    acc += (kx == 0) ? m2 : (T)2 * m2;
    acc2 += (kx == 0) ? o2 : (T)2 * o2;
    if constexpr (IN == WF_IN_PK) {
      dst[WF_CHK(((size_t)c * n + j) * h + kx, (size_t)C * n * h)] = o;
    } else {
      if (kx == 0) buf[wf_swz<T, SWP>(j * CT + c * TC + t)] = o;
      else dst[WF_CHK(((size_t)c * n + j) * (h + 1) + kx, (size_t)C * n * (h + 1))] = o;
    }
  }
  if constexpr (IN == WF_IN_STD) {
    if (kx0 == 0) {
      __syncthreads();
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int jm = (n - j) & (n - 1);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          V2<T> X0, Xh;
          wf_unpack0<T>(buf[wf_swz<T, SWP>(j * CT + c * TC)], buf[wf_swz<T, SWP>(jm * CT + c * TC)], X0, Xh);
          V2<T>* row = dst + WF_CHK(((size_t)c * n + j) * (h + 1), (size_t)C * n * (h + 1) - h);
          row[0] = X0;
          row[h] = Xh;
        }
      }
    }
  }
  const double tot = wf_block_sum((double)acc);
  if (threadIdx.x == 0) part_b[(size_t)WF_SLOT_PRIOR * g.maxblk + slot_ix] = tot;
  const double tot2 = wf_block_sum((double)acc2);
  if (threadIdx.x == 0) part_b[(size_t)WF_SLOT_OUT2 * g.maxblk + slot_ix] = tot2;
}

// ---------------------------------------------------------------------------
// k_col_fwd: scratch tile -> forward FFT along y -> sqrt(P) R^T / n = a ->
// out = 2 (src - a) (the gradient, or the Hessian-vector product when the row
// stage ran without data); prior partial sum |src|^2 with half-plane weights.
// One block per column tile.  (Persistent forms, the next tile's rows
// prefetched, measured slower on 120 x 1024^2: items taken round-robin 1.01 ms
// against 0.69 ms; items taken in order from an atomic counter, 2.00 ms for
// the whole objective pass against 1.69 ms.)
// ---------------------------------------------------------------------------
template <typename T, int C, int IN>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB_COLFWD(T, C))
k_col_fwd(WfGeo g, const void* src_, const T* sp_, long long sp_stride, const void* scratch_,
          void* dst_, double* part, const void* tw_) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  V2<T>* s_tw = (V2<T>*)wf_smem;
  V2<T>* buf = s_tw + WF_NT;
  const int b = blockIdx.y, n = g.n, h = g.h, lgn = g.lgn;
  const int TC = g.TC, lgTC = __ffs(TC) - 1, CT = C * TC, kx0 = blockIdx.x * TC;
  const int pitch = IN == WF_IN_PK ? h : h + 1;
  const size_t sstride = (size_t)C * n * pitch;
  // the epilogue reads this tile's rows of src after the transform: start them towards L2
  wf_prefetch_rows((const V2<T>*)src_ + (size_t)b * sstride + kx0, C * n, (size_t)pitch * sizeof(V2<T>),
                   TC * (int)sizeof(V2<T>));
  wf_stage_tw<T>(s_tw, (const V2<T>*)tw_, lgn);
  wf_tile_load<T, C, WF_IN_PK>(buf, (const V2<T>*)scratch_ + (size_t)b * C * n * h, n, h, lgTC, kx0);
  __syncthreads();
  fft_smem<T, -1, WF_EMAX>(buf, lgn, CT, 1, CT, s_tw);
  wf_col_scale<T, C, true>(buf, g, lgTC, kx0, sp_ + (size_t)b * sp_stride, (T)1);
  __syncthreads();
  wf_col_fwd_out<T, C, IN, false>(g, buf, (const V2<T>*)src_ + (size_t)b * sstride,
                                  (V2<T>*)dst_ + (size_t)b * sstride, kx0, part + (size_t)b * WF_NSLOT * g.maxblk,
                                  blockIdx.x);
}

// Scale the sqrt(P)/n table by sqrt(q_l) on the modes of band l (others 1):
// sp = sp0 * sqrt(q[band]); q has n_b entries shared by all maps.
template <typename T>
__global__ void k_band_scale(const T* sp0, T* sp, size_t nsp, int ntab, const int16_t* band, const double* q,
                             int n_b) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t tot = nsp * (size_t)ntab;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += stride) {
    const int l = band[i % nsp];
    const double f = (l >= 0 && l < n_b) ? sqrt(q[l]) : 1.0;
    sp[i] = (T)((double)sp0[i] * f);
  }
}

// ---------------------------------------------------------------------------
// k_col_sim: scratch tile holding the row r2c of a white field z -> forward
// FFT along y -> scale by 1/sqrt(ny nx) (unitary U z) -> R sqrt(P)/n -> inverse FFT
// along y -> scratch.  Used to synthesise A z for simulations.
// ---------------------------------------------------------------------------
template <typename T, int C>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB(T))
k_col_sim(WfGeo g, const T* sp_, long long sp_stride, void* scratch_, const void* tw_) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  V2<T>* s_tw = (V2<T>*)wf_smem;
  V2<T>* buf = s_tw + WF_NT;
  const int b = blockIdx.y, n = g.n, h = g.h, lgn = g.lgn;
  const int TC = g.TC, lgTC = __ffs(TC) - 1, CT = C * TC, kx0 = blockIdx.x * TC;
  wf_stage_tw<T>(s_tw, (const V2<T>*)tw_, lgn);
  V2<T>* sc = (V2<T>*)scratch_ + (size_t)b * C * n * h;
  wf_tile_load<T, C, WF_IN_PK>(buf, sc, n, h, lgTC, kx0);
  __syncthreads();
  fft_smem<T, -1, WF_EMAX>(buf, lgn, CT, 1, CT, s_tw);
  const T unit = (T)(1.0 / sqrt((double)n * (double)g.nx));
  wf_col_scale<T, C, false>(buf, g, lgTC, kx0, sp_ + (size_t)b * sp_stride, unit);
  __syncthreads();
  fft_smem<T, +1, WF_EMAX>(buf, lgn, CT, 1, CT, s_tw);
  wf_tile_store_pk<T, C>(sc, buf, n, h, lgTC, kx0);
}

// ---------------------------------------------------------------------------
// k_row: row stage over RB of the C*ny rows of each map (rows of nx pixels).
//   MODE DATA / NODATA: c2r, r = d - x (or -x), wr = w r, data partial sum
//     r.wr, r2c of wr, store packed rows back to scratch.
//   MODE SIGNAL: c2r, write x to out (pixel layout).
//   MODE SIM: c2r, out = (w > 0) ? x + aux : 0 (aux = noise).
//   MODE RFFT: r2c of the pixel rows of aux (a white field), store to scratch.
// ---------------------------------------------------------------------------
template <typename T, int MODE>
__device__ __forceinline__ void k_row_body(WfGeo g, void* scratch_, const void* d_, const void* w_,
                                           const void* aux_, void* out_, double* part, const void* tw_) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  V2<T>* s_tw = (V2<T>*)wf_smem;   // roots of unity (real-FFT pre/post twiddles)
  V2<T>* s_pt = s_tw + WF_NT;       // pass table of length nx/2
  V2<T>* buf = s_pt + WF_NT;
  const int b = blockIdx.y, n = g.n, nx = g.nx, h = g.h, lgh = g.lgh, RB = g.RB;
  const int row0 = blockIdx.x * RB;
  const size_t npix = (size_t)g.C * n * nx;
  wf_stage_tw<T>(s_tw, (const V2<T>*)tw_);
  wf_stage_tw<T>(s_pt, (const V2<T>*)tw_, lgh);
  V2<T>* sc = (V2<T>*)scratch_ + (size_t)b * g.C * n * h + (size_t)row0 * h;
  const int tot = RB * h;
  const int lgNTn = WF_LOG2_NT - g.lgnx;  // table stride of the nx-th roots
  double acc = 0.0;

  if constexpr (MODE == WF_ROW_RFFT) {
    const V2<T>* z = (const V2<T>*)((const T*)aux_ + (size_t)b * npix + (size_t)row0 * nx);
    wf_g2s<T>(buf, z, tot);
    __syncthreads();
  } else {
    wf_g2s<T>(buf, sc, tot);
    __syncthreads();
    // c2r pre-processing: Z[k] = (X[k] + conj X[h-k]) + i w^k (X[k] - conj X[h-k]),
    // w = exp(+2 pi i / nx), X[0], X[h] the real parts packed in Y[0].
    for (int e = threadIdx.x; e < RB * (h / 2 + 1); e += blockDim.x) {
      const int t = e / (h / 2 + 1), k = e - t * (h / 2 + 1);
      const int r0 = t * h;
      if (k == 0) {
        const V2<T> Y = buf[wf_sw<T>(r0)];
        buf[wf_sw<T>(r0)] = mk<T>(Y.x + Y.y, Y.x - Y.y);
      } else {
        const int km = h - k;
        const V2<T> Xk = buf[wf_sw<T>(r0 + k)], Xm = buf[wf_sw<T>(r0 + km)];
        const V2<T> w1 = twid<T, +1>(s_tw, k << lgNTn), w2 = twid<T, +1>(s_tw, km << lgNTn);
        const V2<T> s1 = mk<T>(Xk.x + Xm.x, Xk.y - Xm.y), d1 = mk<T>(Xk.x - Xm.x, Xk.y + Xm.y);
        const V2<T> s2 = mk<T>(Xm.x + Xk.x, Xm.y - Xk.y), d2 = mk<T>(Xm.x - Xk.x, Xm.y + Xk.y);
        buf[wf_sw<T>(r0 + k)] = cadd<T>(s1, mul_i<T>(cmul<T>(w1, d1)));
        buf[wf_sw<T>(r0 + km)] = cadd<T>(s2, mul_i<T>(cmul<T>(w2, d2)));
      }
    }
    __syncthreads();
    fft_smem<T, +1, WF_EMAX>(buf, lgh, RB, h, 1, s_pt);
    // pixel stage: buf[t][m] holds pixels (2m, 2m+1) of row row0 + t
    const V2<T>* dv = (const V2<T>*)((const T*)d_ + (size_t)b * npix + (size_t)row0 * nx);
    const V2<T>* wv = (const V2<T>*)((const T*)w_ + (size_t)b * npix + (size_t)row0 * nx);
    if constexpr (MODE == WF_ROW_SIGNAL) {
      V2<T>* ov = (V2<T>*)((T*)out_ + (size_t)b * npix + (size_t)row0 * nx);
      wf_s2g<T>(ov, buf, tot);
      return;
    } else if constexpr (MODE == WF_ROW_SIM) {
      V2<T>* ov = (V2<T>*)((T*)out_ + (size_t)b * npix + (size_t)row0 * nx);
      const V2<T>* nz = (const V2<T>*)((const T*)aux_ + (size_t)b * npix + (size_t)row0 * nx);
      for (int e = threadIdx.x; e < tot; e += blockDim.x) {
        const V2<T> x = buf[wf_sw<T>(e)], w = wv[e], q = nz[e];
        ov[e] = mk<T>(w.x > (T)0 ? x.x + q.x : (T)0, w.y > (T)0 ? x.y + q.y : (T)0);
      }
      return;
    } else {
      float accf = 0.f;
      V2<T> wl[WF_EMAX], dl[WF_EMAX];
#pragma unroll
      for (int i = 0; i < WF_EMAX; ++i) {
        const int e = threadIdx.x + i * WF_THREADS;
        if (e < tot) {
          wl[i] = wv[e];
          if constexpr (MODE == WF_ROW_DATA) dl[i] = dv[e];
        }
      }
#pragma unroll
      for (int i = 0; i < WF_EMAX; ++i) {
        const int e = threadIdx.x + i * WF_THREADS;
        if (e < tot) {
          const V2<T> x = buf[wf_sw<T>(e)], w = wl[i];
          V2<T> r;
          if constexpr (MODE == WF_ROW_DATA) r = mk<T>(dl[i].x - x.x, dl[i].y - x.y);
          else r = mk<T>(-x.x, -x.y);
          const V2<T> wr = mk<T>(w.x * r.x, w.y * r.y);
          if constexpr (sizeof(T) == 4) accf += r.x * wr.x + r.y * wr.y;
          else acc += (double)(r.x * wr.x) + (double)(r.y * wr.y);
          buf[wf_sw<T>(e)] = wr;
        }
      }
      acc += (double)accf;
      __syncthreads();
    }
  }
  // r2c: forward FFT of the packed pairs, then
  // X[k] = (Z[k] + conj Z[h-k])/2 - i w^-k (Z[k] - conj Z[h-k])/2, X[0], X[h] packed.
  fft_smem<T, -1, WF_EMAX>(buf, lgh, RB, h, 1, s_pt);
  for (int e = threadIdx.x; e < RB * (h / 2 + 1); e += blockDim.x) {
    const int t = e / (h / 2 + 1), k = e - t * (h / 2 + 1);
    const int r0 = t * h;
    if (k == 0) {
      const V2<T> Z = buf[wf_sw<T>(r0)];
      buf[wf_sw<T>(r0)] = mk<T>(Z.x + Z.y, Z.x - Z.y);
    } else {
      const int km = h - k;
      const V2<T> Zk = buf[wf_sw<T>(r0 + k)], Zm = buf[wf_sw<T>(r0 + km)];
      const V2<T> w1 = twid<T, -1>(s_tw, k << lgNTn), w2 = twid<T, -1>(s_tw, km << lgNTn);
      const V2<T> s1 = mk<T>(Zk.x + Zm.x, Zk.y - Zm.y), d1 = mk<T>(Zk.x - Zm.x, Zk.y + Zm.y);
      const V2<T> s2 = mk<T>(Zm.x + Zk.x, Zm.y - Zk.y), d2 = mk<T>(Zm.x - Zk.x, Zm.y + Zk.y);
      const V2<T> i1 = mul_i<T>(cmul<T>(w1, d1)), i2 = mul_i<T>(cmul<T>(w2, d2));
      buf[wf_sw<T>(r0 + k)] = mk<T>((T)0.5 * (s1.x - i1.x), (T)0.5 * (s1.y - i1.y));
      buf[wf_sw<T>(r0 + km)] = mk<T>((T)0.5 * (s2.x - i2.x), (T)0.5 * (s2.y - i2.y));
    }
  }
  __syncthreads();
  wf_s2g<T>(sc, buf, tot);
  if constexpr (MODE == WF_ROW_DATA || MODE == WF_ROW_NODATA) {
    const double s = wf_block_sum(acc);
    if (threadIdx.x == 0) part[((size_t)b * WF_NSLOT + WF_SLOT_DATA) * g.maxblk + blockIdx.x] = s;
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(WF_THREADS, WF_MINB(T))
k_row(WfGeo g, void* scratch_, const void* d_, const void* w_, const void* aux_, void* out_,
      double* part, const void* tw_) {
  k_row_body<T, MODE>(g, scratch_, d_, w_, aux_, out_, part, tw_);
}

// chi2[b] = sum of the prior and data partial sums, in a fixed order.
static __global__ void __launch_bounds__(WF_THREADS)
k_finalize_chi2(const double* part, int maxblk, int nprior, int ndata, double* chi2) {
  const int b = blockIdx.x;
  double acc = 0.0;
  const double* pp = part + (size_t)b * WF_NSLOT * maxblk;
  for (int i = threadIdx.x; i < nprior; i += blockDim.x) acc += pp[WF_SLOT_PRIOR * maxblk + i];
  for (int i = threadIdx.x; i < ndata; i += blockDim.x) acc += pp[WF_SLOT_DATA * maxblk + i];
  const double s = wf_block_sum(acc);
  if (threadIdx.x == 0) chi2[b] = s;
}

// ---------------------------------------------------------------------------
// Input preparation: working-type copies of d, W = mask * Ninv, sqrt(P/(ny nx)),
// with checks recorded in flags[0] as a wf_status bit set (1 << status).
// ---------------------------------------------------------------------------
struct WfMapPtrs { const void* d; const unsigned char* mask; const void* Ninv; const void* P; };

template <typename S>
__device__ __forceinline__ double wf_rd(const void* p, size_t i) { return (double)((const S*)p)[i]; }

template <typename T>
__global__ void k_prep(WfGeo g, const WfMapPtrs* maps, int in_f64, T* d, T* w, T* sp, int sp_shared,
                       int* flags) {
  const int b = blockIdx.y, n = g.n, C = g.C;
  const size_t npix = (size_t)C * n * g.nx, nsp = (size_t)C * n * (g.h + 1);
  const WfMapPtrs m = maps[b];
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride) {
    const size_t pix = i % ((size_t)n * g.nx);
    const double ni = in_f64 ? wf_rd<double>(m.Ninv, i) : wf_rd<float>(m.Ninv, i);
    const double dv = m.d ? (in_f64 ? wf_rd<double>(m.d, i) : wf_rd<float>(m.d, i)) : 0.0;
    const bool obs = m.mask[pix] != 0;
    if (!isfinite(ni)) atomicOr(flags, 1 << WF_ENONFINITE);
    else if (ni < 0.0) atomicOr(flags, 1 << WF_EINVAL);
    if (obs && !isfinite(dv)) atomicOr(flags, 1 << WF_ENONFINITE);
    const double wv = obs && isfinite(ni) && ni > 0.0 ? ni : 0.0;
    w[(size_t)b * npix + i] = (T)wv;
    d[(size_t)b * npix + i] = (T)(obs && isfinite(dv) ? dv : 0.0);
  }
  if (sp_shared && b > 0) return;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nsp; i += stride) {
    const double pv = in_f64 ? wf_rd<double>(m.P, i) : wf_rd<float>(m.P, i);
    if (!isfinite(pv)) atomicOr(flags, 1 << WF_ENONFINITE);
    else if (pv < 0.0) atomicOr(flags, 1 << WF_EINVAL);
    const double s = !(isfinite(pv) && pv > 0.0) ? 0.0
                     : (g.nx == n ? sqrt(pv) / (double)n : sqrt(pv / ((double)n * (double)g.nx)));
    sp[(size_t)b * nsp + i] = (T)s;
  }
}

template <typename T>
__global__ void k_set_data(size_t total, const T* src, T* d) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) d[i] = src[i];
}

// Standard [C][ny][h+1] <-> packed [C][ny][h] spectra.
template <typename T>
__global__ void k_pack(WfGeo g, int B, const V2<T>* in, V2<T>* out) {
  const int n = g.n, h = g.h;
  const size_t rows = (size_t)B * g.C * n;
  const size_t total = rows * h, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const size_t r = i / h;
    const int kx = (int)(i - r * h);
    const V2<T>* row = in + r * (h + 1);
    out[i] = kx == 0 ? wf_pack0<T>(row[0], row[h]) : row[kx];
  }
}

template <typename T>
__global__ void k_unpack(WfGeo g, int B, const V2<T>* in, V2<T>* out) {
  const int n = g.n, h = g.h;
  const size_t rows = (size_t)B * g.C * n;
  const size_t total = rows * h, stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const size_t r = i / h;
    const int kx = (int)(i - r * h);
    V2<T>* orow = out + r * (h + 1);
    if (kx == 0) {
      const int j = (int)(r % n);
      const size_t r0 = r - j, rm = r0 + ((n - j) & (n - 1));
      V2<T> X0, Xh;
      wf_unpack0<T>(in[r * h], in[rm * h], X0, Xh);
      orow[0] = X0;
      orow[h] = Xh;
    } else {
      orow[kx] = in[i];
    }
  }
}

// Per-block band sums over the half-plane modes of standard-layout spectra,
// with the full-plane multiplicity (1 on kx = 0 and nx/2, else 2):
//   MODE 0 (band energy, eq. el):      |s_k|^2
//   MODE 1 (d chi2 / d log q, eq. pilin): -Re(conj(a_k) s_k), a = s - grad / 2
//          (grad = 2 (s - a) from the objective + gradient pass)
// Grid (nblk, B); block x of map b covers a fixed contiguous range of modes
// and writes part[(b nblk + x) nb + l].  Per-warp bins in shared memory
// ([warps][nb]), summed over the warps in a fixed order.
template <typename T, int MODE>
__global__ void __launch_bounds__(WF_THREADS)
k_band_reduce(WfGeo g, const V2<T>* s, const V2<T>* gr, const int16_t* band, int nb, double* part) {
  extern __shared__ double s_bins[];  // [WF_THREADS / 32][nb]
  const int b = blockIdx.y, h = g.h, nw = WF_THREADS / 32, w = threadIdx.x >> 5;
  const size_t nsp = (size_t)g.C * g.n * (h + 1);
  for (int i = threadIdx.x; i < nw * nb; i += blockDim.x) s_bins[i] = 0.0;
  __syncthreads();
  const size_t per = (nsp + gridDim.x - 1) / gridDim.x;
  const size_t lo = (size_t)blockIdx.x * per, hi = lo + per < nsp ? lo + per : nsp;
  const V2<T>* sb = s + (size_t)b * nsp;
  const V2<T>* gb = MODE == 1 ? gr + (size_t)b * nsp : nullptr;
  double* bins = s_bins + (size_t)w * nb;
  for (size_t i0 = lo; i0 < hi; i0 += blockDim.x) {  // uniform trip count across the block
    const size_t i = i0 + threadIdx.x;
    int l = -1;
    double v = 0.0;
    if (i < hi) {
      l = band[i];
      if (l >= nb) l = -1;
      if (l >= 0) {
        const int kx = (int)(i % (h + 1));
        const double mult = (kx == 0 || kx == h) ? 1.0 : 2.0;
        const V2<T> x = sb[i];
        if constexpr (MODE == 0) {
          v = mult * ((double)x.x * x.x + (double)x.y * x.y);
        } else {
          const V2<T> gv = gb[i];
          const T ax = x.x - (T)0.5 * gv.x, ay = x.y - (T)0.5 * gv.y;
          v = -mult * (double)(ax * x.x + ay * x.y);
        }
      }
    }
    wf_warp_bin_add(bins, l, v);
  }
  __syncthreads();
  for (int l = threadIdx.x; l < nb; l += blockDim.x) {
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += s_bins[(size_t)q * nb + l];
    part[((size_t)b * gridDim.x + blockIdx.x) * nb + l] = t;
  }
}

// out[b][l] = scale_l * sum over the nblk block partials of map b, in order:
// scale 1/(2 theta_l) for the band energy (theta given), 1 otherwise.
static __global__ void k_band_final(const double* part, int nblk, int nb, const double* theta, double* out) {
  const int b = blockIdx.x;
  for (int l = threadIdx.x; l < nb; l += blockDim.x) {
    double t = 0.0;
    for (int q = 0; q < nblk; ++q) t += part[((size_t)b * nblk + q) * nb + l];
    out[(size_t)b * nb + l] = theta ? 0.5 * t / theta[l] : t;
  }
}

