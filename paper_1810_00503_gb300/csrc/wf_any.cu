// Objective, gradient and Hessian-vector product of Sec. 2.2 (eq_chi,
// eq_cost) on grids of any side lengths whose prime factors are 2, 3, 5 and 7
// (up to 1024 pixels a side), for callers whose maps are not powers of two.
//
//   chi^2(s) = |s|^2 + (d - x)^T W (d - x),  x = U^-1 R(k) sqrt(P) s,
//   grad     = 2 (s - sqrt(P) R(k)^T U W (d - x)),
//
// with s the half-plane unitary spectrum [C][ny][nx/2+1] of a real field, U
// the unitary 2-D DFT ((ny nx)^-1/2), W = mask * Ninv per pixel and, for the
// joint E/B pair (C = 2), R(k) the Kaiser-Squires rotation of App. C at the
// wavevector (mx / nx, my / ny) with s = 0 on the Nyquist lines.  With d
// omitted the data term sees d = 0, so grad = 2 (I + A^T W A) s: the
// Hessian-vector product.
//
// Three kernels, as in the power-of-two path but unfused and plain:
//   k_any_colinv  per column tile: R sqrt(P) s, inverse DFT along y -> scratch;
//   k_any_row     per row: c2r along x (Hermitian extension), r = d - x,
//                 W r, sum r W r, r2c along x -> scratch;
//   k_any_colfwd  per column tile: forward DFT along y, sqrt(P) R^T / sqrt N,
//                 grad, sum of |s|^2 with the half-plane weights;
// then k_any_final adds the partial sums of each map in a fixed order.
// The DFTs are Stockham autosort transforms in shared memory with radix 4, 2,
// 3, 5 and 7 passes (pass with radix R, span Ns: butterfly j reads j + r L/R,
// multiplies by exp(+-2 pi i r (j mod Ns) / (Ns R)), does a length-R DFT and
// writes (j - j mod Ns) R + j mod Ns + r Ns); the twiddles come from sincospi.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "wf_api_internal.h"
#include "wf_fft.cuh"

#define WF_ANY_THREADS 256
#define WF_ANY_BUF 2048   // complex values per shared buffer: C * (columns of a tile) * ny, or C * nx
#define WF_ANY_MAXP 12    // passes of one transform at most (1024 = 4^5; 7-smooth lengths <= 1024 need <= 10)
#define WF_ANY_MAXN 1024

struct WfAnyGeo {
  int B, C, ny, nx, h1;  // h1 = nx / 2 + 1 half-plane columns
  int cb;                // columns per block of the column kernels
  int gx;                // column tiles: ceil(h1 / cb)
  int npy, npx;          // passes along y and x
  int ry[WF_ANY_MAXP], rx[WF_ANY_MAXP];
  double inv_sqrt_n;     // (ny nx)^-1/2
};

template <typename T> __device__ __forceinline__ void wf_sincospi(T a, T* s, T* c);
template <> __device__ __forceinline__ void wf_sincospi<float>(float a, float* s, float* c) { sincospif(a, s, c); }
template <> __device__ __forceinline__ void wf_sincospi<double>(double a, double* s, double* c) { sincospi(a, s, c); }

// One pass of radix R over cnt sequences of length L (sequence t at in + t L),
// from `in` to `out`; Ns = product of the radices of the earlier passes.
template <typename T, int R, int DIR>
__device__ __forceinline__ void wf_any_pass(const V2<T>* in, V2<T>* out, int L, int cnt, int Ns) {
  T cr[R], sr[R];  // exp(DIR 2 pi i t / R) = cr[t] + i sr[t]
#pragma unroll
  for (int t = 0; t < R; ++t) {
    wf_sincospi<T>((T)(2 * t) / (T)R, &sr[t], &cr[t]);
    sr[t] *= (T)DIR;
  }
  const int LR = L / R, nbf = cnt * LR, span = Ns * R;
  [[maybe_unused]] const int lim = cnt * L;
  for (int bf = threadIdx.x; bf < nbf; bf += blockDim.x) {
    const int t = bf / LR, j = bf - t * LR, k = j % Ns;
    V2<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[WF_CHK(t * L + j + r * LR, lim)];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        T sw, cw;
        wf_sincospi<T>((T)(2 * r * k) / (T)span, &sw, &cw);  // r k < span
        v[r] = cmul<T>(v[r], mk<T>(cw, (T)DIR * sw));
      }
    }
    const int o = t * L + (j - k) * R + k;
#pragma unroll
    for (int q = 0; q < R; ++q) {
      V2<T> acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const int e = (r * q) % R;
        acc.x += v[r].x * cr[e] - v[r].y * sr[e];
        acc.y += v[r].x * sr[e] + v[r].y * cr[e];
      }
      out[WF_CHK(o + q * Ns, lim)] = acc;
    }
  }
}

// Unnormalised DFT (DIR -1 forward, +1 inverse) of cnt sequences of length L
// held in a; b is the other buffer.  Returns the buffer holding the result.
// Called by the whole block; ends with a barrier.
template <typename T, int DIR>
__device__ V2<T>* wf_any_fft(V2<T>* a, V2<T>* b, int L, int cnt, int np, const int* rad) {
  int Ns = 1;
  V2<T>* in = a;
  V2<T>* out = b;
  for (int p = 0; p < np; ++p) {
    const int R = rad[p];
    switch (R) {
      case 2: wf_any_pass<T, 2, DIR>(in, out, L, cnt, Ns); break;
      case 3: wf_any_pass<T, 3, DIR>(in, out, L, cnt, Ns); break;
      case 4: wf_any_pass<T, 4, DIR>(in, out, L, cnt, Ns); break;
      case 5: wf_any_pass<T, 5, DIR>(in, out, L, cnt, Ns); break;
      default: wf_any_pass<T, 7, DIR>(in, out, L, cnt, Ns); break;
    }
    __syncthreads();
    Ns *= R;
    V2<T>* t = in;
    in = out;
    out = t;
  }
  return in;
}

// Kaiser-Squires cosine and sine at half-plane mode (ky, kx): wavevector
// (mx / nx, my / ny) scaled by nx ny to the integers (mx ny, my nx); signed
// mode numbers, R = I at k = 0, sine 0 on the Nyquist line of an even side.
__device__ __forceinline__ void wf_any_ks(const WfAnyGeo& G, int ky, int kx, double* c, double* s) {
  const int my = ky <= (G.ny - 1) / 2 ? ky : ky - G.ny;
  const double qx = (double)kx * G.ny, qy = (double)my * G.nx;
  const double k2 = qx * qx + qy * qy;
  if (k2 == 0.0) {
    *c = 1.0;
    *s = 0.0;
    return;
  }
  *c = (qx * qx - qy * qy) / k2;
  const bool nyq = ((G.nx % 2) == 0 && 2 * kx == G.nx) || ((G.ny % 2) == 0 && 2 * ky == G.ny);
  *s = nyq ? 0.0 : 2.0 * qx * qy / k2;
}

// Fixed-order block sum of one double per thread; the result in thread 0.
__device__ __forceinline__ double wf_any_block_sum(double v) {
  __shared__ double red[WF_ANY_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// Inverse column stage: tile of cb half-plane columns of map blockIdx.y, all
// channels; the per-mode operator R(k) sqrt(P) on the way in, then the inverse
// DFT along y into scratch [B][C][ny][h1].
template <typename T>
__global__ void __launch_bounds__(WF_ANY_THREADS)
k_any_colinv(const __grid_constant__ WfAnyGeo G, const V2<T>* s, const T* P, V2<T>* scr) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  V2<T>* A = (V2<T>*)wf_smem;
  V2<T>* Bf = A + WF_ANY_BUF;
  const int b = blockIdx.y, kx0 = blockIdx.x * G.cb, C = G.C, ny = G.ny, h1 = G.h1;
  const int ncol = min(G.cb, h1 - kx0);
  const size_t vsz = (size_t)C * ny * h1;
  const V2<T>* sb = s + (size_t)b * vsz;
  for (int i = threadIdx.x; i < ncol * ny; i += blockDim.x) {
    const int col = i % ncol, ky = i / ncol, kx = kx0 + col;
    const size_t m0 = (size_t)ky * h1 + kx;  // mode offset within a channel
    const V2<T> s0 = sb[WF_CHK(m0, vsz)];
    const T p0 = sqrt(P[WF_CHK(m0, (size_t)C * ny * h1)]);
    V2<T> a0 = cscale<T>(s0, p0);
    if (C == 2) {
      const size_t m1 = (size_t)ny * h1 + m0;
      const V2<T> s1 = sb[WF_CHK(m1, vsz)];
      const V2<T> a1 = cscale<T>(s1, (T)sqrt(P[WF_CHK(m1, (size_t)C * ny * h1)]));
      double cd, sd;
      wf_any_ks(G, ky, kx, &cd, &sd);
      const T c = (T)cd, sn = (T)sd;
      A[WF_CHK((size_t)(0 * ncol + col) * ny + ky, WF_ANY_BUF)] = mk<T>(c * a0.x - sn * a1.x, c * a0.y - sn * a1.y);
      A[WF_CHK((size_t)(1 * ncol + col) * ny + ky, WF_ANY_BUF)] = mk<T>(sn * a0.x + c * a1.x, sn * a0.y + c * a1.y);
    } else {
      A[WF_CHK((size_t)col * ny + ky, WF_ANY_BUF)] = a0;
    }
  }
  __syncthreads();
  const V2<T>* res = wf_any_fft<T, +1>(A, Bf, ny, C * ncol, G.npy, G.ry);
  V2<T>* out = scr + (size_t)b * vsz;
  for (int i = threadIdx.x; i < C * ncol * ny; i += blockDim.x) {
    const int col = i % ncol, rest = i / ncol, ky = rest % ny, c = rest / ny;
    out[WF_CHK(((size_t)c * ny + ky) * h1 + kx0 + col, vsz)] = res[WF_CHK((size_t)(c * ncol + col) * ny + ky, WF_ANY_BUF)];
  }
}

// Row stage: row blockIdx.x of map blockIdx.y, all channels.  c2r along x by
// the Hermitian extension X[nx - kx] = conj X[kx] (the real part of the
// inverse DFT), the pixel step r = d - x, W r and sum r W r, then r2c along x
// back into the row of scratch.  dpart[b ny + y] = the row's sum r W r.
template <typename T>
__global__ void __launch_bounds__(WF_ANY_THREADS)
k_any_row(const __grid_constant__ WfAnyGeo G, const T* d, const uint8_t* mask, const T* Ninv, V2<T>* scr,
          double* dpart) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  V2<T>* A = (V2<T>*)wf_smem;
  V2<T>* Bf = A + WF_ANY_BUF;
  const int b = blockIdx.y, y = blockIdx.x, C = G.C, ny = G.ny, nx = G.nx, h1 = G.h1;
  const size_t vsz = (size_t)C * ny * h1, psz = (size_t)C * ny * nx;
  V2<T>* row = scr + (size_t)b * vsz;
  for (int i = threadIdx.x; i < C * nx; i += blockDim.x) {
    const int c = i / nx, kx = i - c * nx;
    const size_t base = ((size_t)c * ny + y) * h1;
    A[WF_CHK(i, WF_ANY_BUF)] = kx < h1 ? row[WF_CHK(base + kx, vsz)] : conj_<T>(row[WF_CHK(base + nx - kx, vsz)]);
  }
  __syncthreads();
  V2<T>* res = wf_any_fft<T, +1>(A, Bf, nx, C, G.npx, G.rx);
  V2<T>* oth = res == A ? Bf : A;
  const T sc = (T)G.inv_sqrt_n;
  double acc = 0.0;
  for (int i = threadIdx.x; i < C * nx; i += blockDim.x) {
    const int c = i / nx, x = i - c * nx;
    const size_t pix = (size_t)b * psz + ((size_t)c * ny + y) * nx + x;
    const T xv = res[WF_CHK(i, WF_ANY_BUF)].x * sc;
    const T dv = d ? d[WF_CHK(pix, (size_t)G.B * psz)] : (T)0;
    const T wv = mask[WF_CHK(((size_t)b * ny + y) * nx + x, (size_t)G.B * ny * nx)] ? Ninv[WF_CHK(pix, (size_t)G.B * psz)]
                                                                                     : (T)0;
    const T r = dv - xv, wr = wv * r;
    acc += (double)r * (double)wr;
    oth[WF_CHK(i, WF_ANY_BUF)] = mk<T>(wr, (T)0);
  }
  __syncthreads();
  const double tot = wf_any_block_sum(acc);
  if (threadIdx.x == 0) dpart[(size_t)b * ny + y] = tot;
  const V2<T>* fw = wf_any_fft<T, -1>(oth, res, nx, C, G.npx, G.rx);
  for (int i = threadIdx.x; i < C * h1; i += blockDim.x) {
    const int c = i / h1, kx = i - c * h1;
    row[WF_CHK(((size_t)c * ny + y) * h1 + kx, vsz)] = fw[WF_CHK((size_t)c * nx + kx, WF_ANY_BUF)];
  }
}

// Forward column stage: the forward DFT along y of a tile of the row stage's
// output, then per mode g = 2 (s - sqrt(P) R(k)^T G / sqrt(N)) and the prior
// sum of |s|^2 with the half-plane weights (1 on column 0 and on the Nyquist
// column of an even nx, 2 elsewhere).  ppart[b gx + tile] = the tile's sum.
template <typename T>
__global__ void __launch_bounds__(WF_ANY_THREADS)
k_any_colfwd(const __grid_constant__ WfAnyGeo G, const V2<T>* s, const T* P, const V2<T>* scr, V2<T>* grad,
             double* ppart) {
  extern __shared__ __align__(16) unsigned char wf_smem[];
  V2<T>* A = (V2<T>*)wf_smem;
  V2<T>* Bf = A + WF_ANY_BUF;
  const int b = blockIdx.y, kx0 = blockIdx.x * G.cb, C = G.C, ny = G.ny, nx = G.nx, h1 = G.h1;
  const int ncol = min(G.cb, h1 - kx0);
  const size_t vsz = (size_t)C * ny * h1;
  const V2<T>* in = scr + (size_t)b * vsz;
  for (int i = threadIdx.x; i < C * ncol * ny; i += blockDim.x) {
    const int col = i % ncol, rest = i / ncol, ky = rest % ny, c = rest / ny;
    A[WF_CHK((size_t)(c * ncol + col) * ny + ky, WF_ANY_BUF)] = in[WF_CHK(((size_t)c * ny + ky) * h1 + kx0 + col, vsz)];
  }
  __syncthreads();
  const V2<T>* res = wf_any_fft<T, -1>(A, Bf, ny, C * ncol, G.npy, G.ry);
  const T sc = (T)G.inv_sqrt_n;
  const V2<T>* sb = s + (size_t)b * vsz;
  V2<T>* gb = grad + (size_t)b * vsz;
  double acc = 0.0;
  for (int i = threadIdx.x; i < ncol * ny; i += blockDim.x) {
    const int col = i % ncol, ky = i / ncol, kx = kx0 + col;
    const double wm = (kx == 0 || ((nx % 2) == 0 && 2 * kx == nx)) ? 1.0 : 2.0;
    V2<T> gd0 = cscale<T>(res[WF_CHK((size_t)col * ny + ky, WF_ANY_BUF)], sc);
    V2<T> gd1 = mk<T>((T)0, (T)0);
    if (C == 2) {
      const V2<T> g1 = cscale<T>(res[WF_CHK((size_t)(ncol + col) * ny + ky, WF_ANY_BUF)], sc);
      double cd, sd;
      wf_any_ks(G, ky, kx, &cd, &sd);
      const T c = (T)cd, sn = (T)sd;
      const V2<T> g0 = gd0;
      gd0 = mk<T>(c * g0.x + sn * g1.x, c * g0.y + sn * g1.y);   // R^T: first row (c, s)
      gd1 = mk<T>(-sn * g0.x + c * g1.x, -sn * g0.y + c * g1.y);  // second row (-s, c)
    }
    for (int c = 0; c < C; ++c) {
      const size_t m = ((size_t)c * ny + ky) * h1 + kx;
      const V2<T> sv = sb[WF_CHK(m, vsz)];
      const T sp = sqrt(P[WF_CHK(m, vsz)]);
      const V2<T> a = c == 0 ? gd0 : gd1;
      gb[WF_CHK(m, vsz)] = mk<T>((T)2 * (sv.x - sp * a.x), (T)2 * (sv.y - sp * a.y));
      acc += wm * ((double)sv.x * sv.x + (double)sv.y * sv.y);
    }
  }
  const double tot = wf_any_block_sum(acc);
  if (threadIdx.x == 0) ppart[(size_t)b * G.gx + blockIdx.x] = tot;
}

// chi2[b] = prior sums of the column tiles + data sums of the rows, each in
// index order.
__global__ void k_any_final(const __grid_constant__ WfAnyGeo G, const double* ppart, const double* dpart,
                            double* chi2) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= G.B) return;
  double prior = 0.0, data = 0.0;
  for (int i = 0; i < G.gx; ++i) prior += ppart[(size_t)b * G.gx + i];
  for (int y = 0; y < G.ny; ++y) data += dpart[(size_t)b * G.ny + y];
  chi2[b] = prior + data;
}

// Radices of a transform of length L (4s first, then 2, 3, 5, 7); false if L
// has another prime factor.
static bool wf_any_plan(int L, int* rad, int* np) {
  *np = 0;
  while (L % 4 == 0 && *np < WF_ANY_MAXP) { rad[(*np)++] = 4; L /= 4; }
  const int pr[4] = {2, 3, 5, 7};
  for (int i = 0; i < 4; ++i)
    while (L % pr[i] == 0 && *np < WF_ANY_MAXP) { rad[(*np)++] = pr[i]; L /= pr[i]; }
  return L == 1;
}

template <typename T>
static cudaError_t wf_any_launch(const WfAnyGeo& G, const void* d, const uint8_t* mask, const void* Ninv,
                                 const void* P, const void* s, void* grad, double* chi2, void* scr, double* dpart,
                                 double* ppart, cudaStream_t st) {
  const size_t smem = 2 * (size_t)WF_ANY_BUF * sizeof(V2<T>);
  cudaError_t e = cudaFuncSetAttribute(k_any_colinv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_any_row<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_any_colfwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_any_colinv<T><<<dim3(G.gx, G.B), WF_ANY_THREADS, smem, st>>>(G, (const V2<T>*)s, (const T*)P, (V2<T>*)scr);
  k_any_row<T><<<dim3(G.ny, G.B), WF_ANY_THREADS, smem, st>>>(G, (const T*)d, mask, (const T*)Ninv, (V2<T>*)scr,
                                                                dpart);
  k_any_colfwd<T><<<dim3(G.gx, G.B), WF_ANY_THREADS, smem, st>>>(G, (const V2<T>*)s, (const T*)P,
                                                                   (const V2<T>*)scr, (V2<T>*)grad, ppart);
  k_any_final<<<(G.B + 127) / 128, 128, 0, st>>>(G, ppart, dpart, chi2);
  return cudaGetLastError();
}

extern "C" wf_status wf_eval_any(wf_handle* h, int B, int C, int ny, int nx, int precision, const void* d,
                                 const uint8_t* mask, const void* Ninv, const void* P, const void* s, void* grad,
                                 double* chi2, void* stream) {
  if (!h || !mask || !Ninv || !P || !s || !grad || !chi2) return wf_fail(WF_EINVAL, "wf_eval_any: null argument");
  if (s == grad) return wf_fail(WF_EINVAL, "wf_eval_any: s and grad must not alias");
  if (B < 1 || (C != 1 && C != 2)) return wf_fail(WF_EINVAL, "wf_eval_any: need count >= 1 and C = 1 or 2");
  if (precision != WF_FP64 && precision != WF_MIXED) return wf_fail(WF_EINVAL, "wf_eval_any: unknown precision");
  WfAnyGeo G = {};
  if (ny < 2 || nx < 2 || ny > WF_ANY_MAXN || nx > WF_ANY_MAXN || !wf_any_plan(ny, G.ry, &G.npy) ||
      !wf_any_plan(nx, G.rx, &G.npx))
    return wf_fail(WF_EINVAL, "wf_eval_any: ny = %d, nx = %d: each side must be in [2, %d] with no prime factor "
                   "above 7", ny, nx, WF_ANY_MAXN);
  G.B = B;
  G.C = C;
  G.ny = ny;
  G.nx = nx;
  G.h1 = nx / 2 + 1;
  G.cb = WF_ANY_BUF / (C * ny);
  if (G.cb < 1) G.cb = 1;
  if (G.cb > G.h1) G.cb = G.h1;
  G.gx = (G.h1 + G.cb - 1) / G.cb;
  G.inv_sqrt_n = 1.0 / sqrt((double)ny * (double)nx);
  const bool f64 = precision == WF_FP64;
  const size_t vsz = (size_t)C * ny * G.h1;
  void* scr = nullptr;
  double *dpart = nullptr, *ppart = nullptr;
  wf_status rs = wf_alloc(h, &scr, (size_t)B * vsz * (f64 ? sizeof(double2) : sizeof(float2)), "wf_eval_any scratch");
  if (rs == WF_OK) rs = wf_alloc(h, (void**)&dpart, sizeof(double) * (size_t)B * ny, "wf_eval_any row sums");
  if (rs == WF_OK) rs = wf_alloc(h, (void**)&ppart, sizeof(double) * (size_t)B * G.gx, "wf_eval_any tile sums");
  if (rs == WF_OK) {
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = f64 ? wf_any_launch<double>(G, d, mask, Ninv, P, s, grad, chi2, scr, dpart, ppart, st)
                        : wf_any_launch<float>(G, d, mask, Ninv, P, s, grad, chi2, scr, dpart, ppart, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rs = wf_cuda_fail(e, "wf_eval_any");
  }
  wf_free(h, ppart);
  wf_free(h, dpart);
  wf_free(h, scr);
  return rs;
}

WF_DBG_READER(any)
