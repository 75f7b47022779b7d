// Shared-memory FFT building blocks for the Wiener-filter operator kernels.
//
// Transforms are power-of-two lengths L <= WF_NT held in shared memory as a
// set of `cnt` independent sequences: sample j of sequence t sits at
// buf[t * ts + j * js].  Each transform is a Stockham autosort FFT: a chain of
// radix-R passes (R in {2, 4, 8, 16}), each pass reading R samples strided by
// L/R, applying twiddles, doing a length-R DFT in registers and writing the R
// results strided by the running span Ns.  Every thread stages all of its
// butterflies in registers between two barriers, so a pass is in place.
//
// Sign convention: DIR = -1 is the forward transform sum_j x_j e^{-2 pi i jk/L},
// DIR = +1 the unnormalised inverse.  Twiddles come from tables computed on the
// host in long double (see wf_make_twiddles): the WF_NT-th roots of unity
// tw[k] = exp(-2 pi i k / WF_NT) and, for each length L, a pass table ordered so
// that consecutive butterflies read consecutive entries.  Kernels stage the
// tables they use in shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "wf_internal.h"


// A hook that does nothing (default of the optional callbacks of the stages).
struct WfNoHook {
  __device__ __forceinline__ void operator()() const {}
};

template <typename T> struct V2t;
template <> struct V2t<float>  { typedef float2  type; };
template <> struct V2t<double> { typedef double2 type; };

template <typename T> using V2 = typename V2t<T>::type;

// Per-thread accumulator of a dot product over a thread's few elements: FP32
// in the mixed path (each partial then continues in FP64 across the block),
// FP64 in the FP64 path.
template <typename T> using WfAcc = typename std::conditional<sizeof(T) == 4, float, double>::type;

template <typename T> __device__ __forceinline__ V2<T> mk(T x, T y) { V2<T> r; r.x = x; r.y = y; return r; }
template <typename T> __device__ __forceinline__ V2<T> cadd(V2<T> a, V2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ V2<T> csub(V2<T> a, V2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ V2<T> cmul(V2<T> a, V2<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ V2<T> conj_(V2<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ V2<T> cscale(V2<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
// multiply by i
template <typename T> __device__ __forceinline__ V2<T> mul_i(V2<T> a) { return mk<T>(-a.y, a.x); }

// Thirty-second roots of unity: cos and sin of pi/16, pi/8, 3 pi/16 and
// pi/4, to the precision of the mathematics; the other angles below pi follow
// by symmetry.
#define WF_C16 0.9807852804032304491261822  // cos(pi/16)
#define WF_S16 0.1950903220161282678482849  // sin(pi/16)
#define WF_C1 0.9238795325112867561281832   // cos(pi/8)
#define WF_S1 0.3826834323650897717284600   // sin(pi/8)
#define WF_C3 0.8314696123025452370787884   // cos(3 pi/16)
#define WF_S3 0.5555702330196022247428308   // sin(3 pi/16)
#define WF_R2 0.7071067811865475244008444   // cos(pi/4)

// Multiply v by exp(DIR * 2 pi i q / 32) with q known at compile time.
template <typename T, int DIR, int Q>
__device__ __forceinline__ V2<T> rot32(V2<T> v) {
  static_assert(Q >= 0 && Q < 16, "root index");
  constexpr T s = (T)DIR;  // sign of the angle
  if constexpr (Q == 0) {
    return v;
  } else if constexpr (Q == 8) {  // exp(DIR i pi/2) = DIR * i
    return (DIR > 0) ? mul_i<T>(v) : mk<T>(v.y, -v.x);
  } else {
    constexpr double cs[16] = {1.0,   WF_C16,  WF_C1,  WF_C3,  WF_R2,  WF_S3,  WF_S1,  WF_S16,
                               0.0,  -WF_S16, -WF_S1, -WF_S3, -WF_R2, -WF_C3, -WF_C1, -WF_C16};
    constexpr double sn[16] = {0.0,  WF_S16, WF_S1, WF_S3, WF_R2, WF_C3, WF_C1, WF_C16,
                               1.0,  WF_C16, WF_C1, WF_C3, WF_R2, WF_S3, WF_S1, WF_S16};
    const T c = (T)cs[Q], sv = s * (T)sn[Q];
    return mk<T>(v.x * c - v.y * sv, v.x * sv + v.y * c);
  }
}

template <int R> struct Log2R;
template <> struct Log2R<1> { static constexpr int v = 0; };
template <> struct Log2R<2> { static constexpr int v = 1; };
template <> struct Log2R<4> { static constexpr int v = 2; };
template <> struct Log2R<8> { static constexpr int v = 3; };
template <> struct Log2R<16> { static constexpr int v = 4; };
template <> struct Log2R<32> { static constexpr int v = 5; };

__host__ __device__ constexpr int bitrev_c(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}

// Butterfly stage of an in-register radix-2 DIT network: span LEN, applied to
// every group of LEN consecutive (bit-reversed) registers.
template <typename T, int R, int DIR, int LEN, int Q>
__device__ __forceinline__ void dit_q(V2<T>* v) {
  if constexpr (Q < LEN / 2) {
#pragma unroll
    for (int s = 0; s < R; s += LEN) {
      V2<T> a = v[s + Q];
      V2<T> b = rot32<T, DIR, Q * (32 / LEN)>(v[s + Q + LEN / 2]);
      v[s + Q] = cadd<T>(a, b);
      v[s + Q + LEN / 2] = csub<T>(a, b);
    }
    dit_q<T, R, DIR, LEN, Q + 1>(v);
  }
}

template <typename T, int R, int DIR, int LEN>
__device__ __forceinline__ void dit_stages(V2<T>* v) {
  if constexpr (LEN <= R) {
    dit_q<T, R, DIR, LEN, 0>(v);
    dit_stages<T, R, DIR, LEN * 2>(v);
  }
}

// Length-R DFT in registers, natural order in and out: v_q <- sum_r v_r w^{DIR r q}.
template <typename T, int R, int DIR>
__device__ __forceinline__ void dft_reg(V2<T>* v) {
  constexpr int B = Log2R<R>::v;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int j = bitrev_c(i, B);
    if (i < j) { V2<T> t = v[i]; v[i] = v[j]; v[j] = t; }
  }
  dit_stages<T, R, DIR, 2>(v);
}

// Shared-memory position of flat tile index x.  The low bits are XORed with
// higher bits so that the strided accesses of the Stockham passes (stride R
// in the first pass, stride C*TC in column tiles) spread over all banks:
// 8-byte values fill 16 bank pairs, 16-byte values 8 bank quads.  A bijection
// within each aligned block of 16 (8) values.  This form serves the in-place
// passes, whose lanes walk the rows of one column of a column tile.
template <typename T>
__device__ __forceinline__ int wf_sw(int x) {
  x = (int)WF_CHK(x, WF_TILE);
  if constexpr (sizeof(T) == 4) return x ^ (((x >> 4) ^ (x >> 8)) & 15);
  else return x ^ (((x >> 3) ^ (x >> 6)) & 7);
}
// The same for the ping-pong passes (wf_fft_pp.cuh), whose lanes walk the
// columns of a tile first: there one shifted copy of the index (a shift and
// one three-input logic operation) is conflict-free for 8-byte values on
// every pass of the plans used; 16-byte values keep two.
template <typename T>
__device__ __forceinline__ int wf_swp(int x) {
  x = (int)WF_CHK(x, WF_TILE);
  if constexpr (sizeof(T) == 4) return x ^ ((x >> 4) & 15);
  else return x ^ (((x >> 3) ^ (x >> 6)) & 7);
}

// Twiddle exp(DIR * 2 pi i * k / WF_NT) from the shared table (k < WF_NT).
template <typename T, int DIR>
__device__ __forceinline__ V2<T> twid(const V2<T>* tw, int k) {
  V2<T> w = tw[k];
  if (DIR > 0) w.y = -w.y;
  return w;
}

// One Stockham pass.  EMAX = most samples a thread holds (compile time).
// ptab is the length-L pass table: the twiddles of the pass with span Ns sit at
// ptab[(Ns - R1) + (r - 1) Ns + k] = exp(-2 pi i k r / (Ns R)) (R1 = radix of the
// first pass), so butterflies with consecutive k read consecutive entries.
template <typename T, int R, int DIR, int EMAX>
__device__ __forceinline__ void fft_pass(V2<T>* buf, int L, int lgL, int cnt, int ts, int js,
                                         int Ns, int lgNs, const V2<T>* ptab, int R1) {
  constexpr int NB = (EMAX / R) > 0 ? (EMAX / R) : 1;
  constexpr int lgR = Log2R<R>::v;
  const int lgLR = lgL - lgR;
  const int LR = 1 << lgLR;
  const int nbf = cnt << lgLR;
  // FULL: every thread has NB butterflies (a full tile), so no bounds tests
  auto body = [&](auto full_tag) {
    constexpr bool FULL = decltype(full_tag)::value;
    V2<T> v[NB][R];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int b = threadIdx.x + i * blockDim.x;
      if (FULL || b < nbf) {
        const int t = b >> lgLR, j = b & (LR - 1);
        const int x0 = t * ts + j * js, dx = LR * js;
#pragma unroll
        for (int r = 0; r < R; ++r) v[i][r] = buf[wf_sw<T>(x0 + r * dx)];
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NB; ++i) {
      const int b = threadIdx.x + i * blockDim.x;
      if (FULL || b < nbf) {
        const int t = b >> lgLR, j = b & (LR - 1);
        const int k = j & (Ns - 1);
        if (Ns > 1) {
          const V2<T>* pt = ptab + (Ns - R1) + k;
#pragma unroll
          for (int r = 1; r < R; ++r) v[i][r] = cmul<T>(v[i][r], twid<T, DIR>(pt, (r - 1) * Ns));
        }
        dft_reg<T, R, DIR>(v[i]);
        const int o = ((j - k) << lgR) + k;
        const int x0 = t * ts + o * js, dx = Ns * js;
#pragma unroll
        for (int r = 0; r < R; ++r) buf[wf_sw<T>(x0 + r * dx)] = v[i][r];
      }
    }
    __syncthreads();
  };
  if (nbf == NB * (int)blockDim.x) body(std::true_type());
  else body(std::false_type());
}

// Full transform of `cnt` sequences of length L = 2^lgL (1 <= lgL <= 10).
// Radix plan: ceil(lgL / 4) passes with the bits spread as evenly as possible,
// larger radices first.  Requires cnt * L <= EMAX * blockDim.x.
// ptab: the length-L pass table (see fft_pass), staged in shared memory.
template <typename T, int DIR, int EMAX>
__device__ __forceinline__ void fft_smem(V2<T>* buf, int lgL, int cnt, int ts, int js, const V2<T>* ptab) {
  const int L = 1 << lgL;
  // the passes of plan 0 written out per length (bits (1..4), (3,2) (3,3)
  // (4,3) (4,4), (3,3,3) (4,3,3)), so that each pass is compiled on its own
  if (lgL <= 4) {
    switch (lgL) {
      case 1: fft_pass<T, 2, DIR, EMAX>(buf, L, lgL, cnt, ts, js, 1, 0, ptab, 2); break;
      case 2: fft_pass<T, 4, DIR, EMAX>(buf, L, lgL, cnt, ts, js, 1, 0, ptab, 4); break;
      case 3: fft_pass<T, 8, DIR, EMAX>(buf, L, lgL, cnt, ts, js, 1, 0, ptab, 8); break;
      default: fft_pass<T, 16, DIR, EMAX>(buf, L, lgL, cnt, ts, js, 1, 0, ptab, 16); break;
    }
  } else if (lgL <= 8) {
    const int b1 = (lgL + 1) >> 1, b2 = lgL - b1, R1 = 1 << b1;
    if (b1 == 3) fft_pass<T, 8, DIR, EMAX>(buf, L, lgL, cnt, ts, js, 1, 0, ptab, R1);
    else fft_pass<T, 16, DIR, EMAX>(buf, L, lgL, cnt, ts, js, 1, 0, ptab, R1);
    if (b2 == 2) fft_pass<T, 4, DIR, EMAX>(buf, L, lgL, cnt, ts, js, R1, b1, ptab, R1);
    else if (b2 == 3) fft_pass<T, 8, DIR, EMAX>(buf, L, lgL, cnt, ts, js, R1, b1, ptab, R1);
    else fft_pass<T, 16, DIR, EMAX>(buf, L, lgL, cnt, ts, js, R1, b1, ptab, R1);
  } else {
    const int b1 = lgL - 6, R1 = 1 << b1;
    if (b1 == 3) fft_pass<T, 8, DIR, EMAX>(buf, L, lgL, cnt, ts, js, 1, 0, ptab, R1);
    else fft_pass<T, 16, DIR, EMAX>(buf, L, lgL, cnt, ts, js, 1, 0, ptab, R1);
    fft_pass<T, 8, DIR, EMAX>(buf, L, lgL, cnt, ts, js, R1, b1, ptab, R1);
    fft_pass<T, 8, DIR, EMAX>(buf, L, lgL, cnt, ts, js, R1 << 3, b1 + 3, ptab, R1);
  }
}
