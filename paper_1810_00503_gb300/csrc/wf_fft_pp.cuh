// Ping-pong Stockham passes with direct global input and output.
//
// A pass takes every butterfly of `cnt` interleaved or stacked sequences of
// length L = 2^lgL, one butterfly per thread at a time: R loads through `ld`,
// the pass twiddles, an in-register radix-R DFT, R stores through `st`.  Input
// and output live in different places (global -> A, A -> B, B -> global or
// shared), so a pass needs no barrier between its loads and stores and keeps
// only R values live.  The first pass reads global memory directly (with any
// per-element operator applied in `ld`), and the last pass hands its outputs
// to `st`, which writes global memory or a shared buffer for an epilogue.
// The radices follow one of the plans of wf_internal.h (chosen per shape by the
// autotuner), with that plan's pass tables.
#pragma once
#include "wf_fft.cuh"

// SEQF: consecutive threads take consecutive sequences (column tiles, whose
// sequences are interleaved in memory) rather than consecutive butterflies of
// one sequence (rows, stored one after another).
template <typename T, int R, int DIR, bool SEQF, class LD, class ST>
__device__ __forceinline__ void wf_pp_pass(int lgL, int lgcnt, int lgNs, const V2<T>* ptab, int R1, LD& ld,
                                           ST& st) {
  constexpr int lgR = Log2R<R>::v;
  const int lgLR = lgL - lgR, nbf = 1 << (lgcnt + lgLR), Ns = 1 << lgNs;
  for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
    int t, j;
    if constexpr (SEQF) {
      t = b & ((1 << lgcnt) - 1);
      j = b >> lgcnt;
    } else {
      t = b >> lgLR;
      j = b & ((1 << lgLR) - 1);
    }
    V2<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld(t, j + (r << lgLR));
    const int k = j & (Ns - 1);
    if (Ns > 1) {
      const V2<T>* pt = ptab + (Ns - R1) + k;
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul<T>(v[r], twid<T, DIR>(pt, (r - 1) * Ns));
    }
    dft_reg<T, R, DIR>(v);
    const int o = ((j - k) << lgR) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) st(t, o + r * Ns, v[r]);
  }
}

// The shared buffer the last pass does not read: where `stl` may write.
template <typename T>
__device__ __forceinline__ V2<T>* wf_pp_out(int lgL, int plan, V2<T>* A, V2<T>* B) {
  return wf_plan_np(lgL, plan) == 2 ? B : A;
}

// Full transform under radix plan PLAN (wf_internal.h; ptab is that plan's
// length-L pass table).  Element e of sequence t sits at t * ts + e * js in
// the shared buffers A and B (swizzled).  ld0 feeds the first pass, stl takes
// the last pass's outputs; a barrier separates consecutive passes.  after1
// runs once every thread has finished the first pass (after a barrier), when
// whatever ld0 read may be overwritten.  The caller synchronises before
// anything reads what stl wrote to shared memory.  Each plan compiles only the
// radices it uses.
template <typename T, int DIR, bool SEQF, int PLAN, class LD0, class STL, class H = WfNoHook>
__device__ __forceinline__ void wf_pp_fft(int lgL, int lgcnt, int ts, int js, V2<T>* A, V2<T>* B,
                                          const V2<T>* ptab, LD0& ld0, STL& stl, H after1 = H()) {
  auto ldA = [&](int t, int e) { return A[wf_swp<T>(t * ts + e * js)]; };
  auto ldB = [&](int t, int e) { return B[wf_swp<T>(t * ts + e * js)]; };
  auto stA = [&](int t, int e, V2<T> v) { A[wf_swp<T>(t * ts + e * js)] = v; };
  auto stB = [&](int t, int e, V2<T> v) { B[wf_swp<T>(t * ts + e * js)] = v; };
  const int np = wf_plan_np(lgL, PLAN);
  if (np == 1) {
    switch (lgL) {
      case 1: wf_pp_pass<T, 2, DIR, SEQF>(lgL, lgcnt, 0, ptab, 2, ld0, stl); break;
      case 2: wf_pp_pass<T, 4, DIR, SEQF>(lgL, lgcnt, 0, ptab, 4, ld0, stl); break;
      case 3: wf_pp_pass<T, 8, DIR, SEQF>(lgL, lgcnt, 0, ptab, 8, ld0, stl); break;
      default: wf_pp_pass<T, 16, DIR, SEQF>(lgL, lgcnt, 0, ptab, 16, ld0, stl); break;
    }
    __syncthreads();
    after1();
  } else if (PLAN == 2 && lgL >= 9) {  // 32 x 16, 32 x 32
    if constexpr (PLAN == 2) {
      wf_pp_pass<T, 32, DIR, SEQF>(lgL, lgcnt, 0, ptab, 32, ld0, stA);
      __syncthreads();
      after1();
      if (lgL == 9) wf_pp_pass<T, 16, DIR, SEQF>(lgL, lgcnt, 5, ptab, 32, ldA, stl);
      else wf_pp_pass<T, 32, DIR, SEQF>(lgL, lgcnt, 5, ptab, 32, ldA, stl);
    }
  } else if (np == 2) {  // lgL 5..8: bits (3,2) (3,3) (4,3) (4,4), ascending in plan 1
    const int hi = (lgL + 1) >> 1, lo = lgL - hi;
    const int b1 = PLAN == 1 ? lo : hi, b2 = lgL - b1, R1 = 1 << b1;
    if (b1 == 2) wf_pp_pass<T, 4, DIR, SEQF>(lgL, lgcnt, 0, ptab, R1, ld0, stA);
    else if (b1 == 3) wf_pp_pass<T, 8, DIR, SEQF>(lgL, lgcnt, 0, ptab, R1, ld0, stA);
    else wf_pp_pass<T, 16, DIR, SEQF>(lgL, lgcnt, 0, ptab, R1, ld0, stA);
    __syncthreads();
    after1();
    if (b2 == 2) wf_pp_pass<T, 4, DIR, SEQF>(lgL, lgcnt, b1, ptab, R1, ldA, stl);
    else if (b2 == 3) wf_pp_pass<T, 8, DIR, SEQF>(lgL, lgcnt, b1, ptab, R1, ldA, stl);
    else wf_pp_pass<T, 16, DIR, SEQF>(lgL, lgcnt, b1, ptab, R1, ldA, stl);
  } else if (PLAN == 1) {  // lgL 9, 10: bits (3,3,3) (3,3,4)
    wf_pp_pass<T, 8, DIR, SEQF>(lgL, lgcnt, 0, ptab, 8, ld0, stA);
    __syncthreads();
    after1();
    wf_pp_pass<T, 8, DIR, SEQF>(lgL, lgcnt, 3, ptab, 8, ldA, stB);
    __syncthreads();
    if (lgL == 9) wf_pp_pass<T, 8, DIR, SEQF>(lgL, lgcnt, 6, ptab, 8, ldB, stl);
    else wf_pp_pass<T, 16, DIR, SEQF>(lgL, lgcnt, 6, ptab, 8, ldB, stl);
  } else {  // lgL 9, 10: bits (3,3,3) (4,3,3)
    const int b1 = lgL - 6, R1 = 1 << b1;
    if (b1 == 3) wf_pp_pass<T, 8, DIR, SEQF>(lgL, lgcnt, 0, ptab, R1, ld0, stA);
    else wf_pp_pass<T, 16, DIR, SEQF>(lgL, lgcnt, 0, ptab, R1, ld0, stA);
    __syncthreads();
    after1();
    wf_pp_pass<T, 8, DIR, SEQF>(lgL, lgcnt, b1, ptab, R1, ldA, stB);
    __syncthreads();
    wf_pp_pass<T, 8, DIR, SEQF>(lgL, lgcnt, b1 + 3, ptab, R1, ldB, stl);
  }
}
