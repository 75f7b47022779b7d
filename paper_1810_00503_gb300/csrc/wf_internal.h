// Internal declarations shared by the host API and the kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/wf.h"

// Bounds-checked debug build (compiled with -DWF_DEBUG_BOUNDS into a separate
// library): WF_CHK(i, lim) checks an index against the size of the buffer it
// addresses; a bad one is counted in this translation unit's record (the
// first kept: source line, index, limit) and replaced by 0, an element that
// exists, so that no access leaves its buffer and nothing traps.  Every
// shared-memory tile index passes through the swizzles, which check it;
// global accesses of the FFT stages and the streaming kernels check theirs at
// the call.  In the normal build WF_CHK(i, lim) is i.
#ifdef WF_DEBUG_BOUNDS
static __device__ unsigned long long wf_dbg_rec[4];  // count, line, index, limit
__device__ __noinline__ inline long long wf_dbg_bad(long long i, long long lim, int line) {
  if (atomicAdd(&wf_dbg_rec[0], 1ull) == 0ull) {
    wf_dbg_rec[1] = (unsigned long long)line;
    wf_dbg_rec[2] = (unsigned long long)i;
    wf_dbg_rec[3] = (unsigned long long)lim;
  }
  return 0;
}
__device__ __forceinline__ long long wf_chk(long long i, long long lim, int line) {
  return (i >= 0 && i < lim) ? i : wf_dbg_bad(i, lim, line);
}
#define WF_CHK(i, lim) wf_chk((long long)(i), (long long)(lim), __LINE__)
// the same for an index that is used only when `cond` holds
#define WF_CHK_IF(cond, i, lim) ((cond) ? WF_CHK(i, lim) : (long long)(i))
// Host reader of this translation unit's record (out: count, line, index,
// limit; reset clears it), one per kernel translation unit.
#define WF_DBG_READER(name)                                                              \
  cudaError_t wf_dbg_read_##name(unsigned long long* out, int reset) {                   \
    cudaError_t e = cudaMemcpyFromSymbol(out, wf_dbg_rec, sizeof(unsigned long long) * 4); \
    if (e == cudaSuccess && reset) {                                                     \
      const unsigned long long z[4] = {0, 0, 0, 0};                                      \
      e = cudaMemcpyToSymbol(wf_dbg_rec, z, sizeof z);                                   \
    }                                                                                    \
    return e;                                                                            \
  }
#else
#define WF_CHK(i, lim) (i)
#define WF_CHK_IF(cond, i, lim) (i)
#define WF_DBG_READER(name)                                                    \
  cudaError_t wf_dbg_read_##name(unsigned long long* out, int reset) {         \
    (void)reset;                                                               \
    out[0] = out[1] = out[2] = out[3] = 0;                                     \
    return cudaSuccess;                                                        \
  }
#endif
#define WF_DBG_TUS(X) X(ops_f32) X(ops_f64) X(lbcol_f32) X(lbcol_f64) X(lbrow_f32) X(lbrow_f64) X(solve) X(noalloc) X(bandpower) X(multi) X(any)
#define WF_DBG_DECL(name) cudaError_t wf_dbg_read_##name(unsigned long long* out, int reset);
WF_DBG_TUS(WF_DBG_DECL)

#define WF_NT 1024          // largest transform length and twiddle-table size
#define WF_LOG2_NT 10
// Twiddle buffer: [0, WF_NT) roots of unity exp(-2 pi i k / WF_NT); then for
// lgL = 1..10 the pass table of length 2^lgL at WF_NT * lgL (2^lgL - 1 entries)
// of radix plan 0.  A handle's buffer holds WF_NPLAN such blocks, plan p's
// tables at WF_TWTAB * p + WF_NT * lgL (the roots only in block 0).
#define WF_TWTAB ((WF_LOG2_NT + 1) * WF_NT)
#define WF_NPLAN 3
#define WF_TWTAB_ALL (WF_NPLAN * WF_TWTAB)

// Radix plans of the ping-pong FFT passes (the in-place passes use plan 0):
//   0: ceil(lgL / 4) passes, the bits spread evenly, larger radices first
//      (1024 = 16 x 8 x 8, 512 = 8 x 8 x 8, 256 = 16 x 16, 128 = 16 x 8);
//   1: the same radices in ascending order (1024 = 8 x 8 x 16, 128 = 8 x 16);
//   2: for lgL >= 9 two passes, radix 32 first (1024 = 32 x 32, 512 = 32 x 16);
//      otherwise plan 0.
// wf_plan_np: passes; wf_plan_bits: log2 of the radix of pass p.
__host__ __device__ inline int wf_plan_np(int lgL, int plan) {
  return (plan == 2 && lgL >= 9) ? 2 : (lgL + 3) >> 2;
}
// Kernels are instantiated per plan; those with radix-32 passes (plan 2) are
// compiled for two blocks per SM (FP32) to hold the 32 values.
#define WF_MINB_PLAN(T, PLAN) ((PLAN) == 2 ? (sizeof(T) == 4 ? 2 : 1) : WF_MINB(T))
__host__ __device__ inline int wf_plan_bits(int lgL, int plan, int p) {
  if (plan == 2 && lgL >= 9) return p == 0 ? 5 : lgL - 5;
  const int np = (lgL + 3) >> 2;
  if (plan == 1) p = np - 1 - p;
  int rem = lgL;
  for (int q = 0; q < p; ++q) {
    const int left = np - q;
    rem -= (rem + left - 1) / left;
  }
  const int left = np - p;
  return (rem + left - 1) / left;
}

// Threads per block of every operator kernel and the most samples one thread
// stages in registers during an FFT pass; a tile holds at most their product.
#define WF_THREADS 256
#define WF_EMAX 16
#define WF_TILE (WF_THREADS * WF_EMAX)
// Streaming L-BFGS kernels: threads per block, complex values per thread per
// vector, and the resulting chunk of each map vector a block owns.
#define WF_COMB_THREADS 256
#define WF_COMB_EPT 4
#define WF_COMB_CHUNK (WF_COMB_THREADS * WF_COMB_EPT)
// Chunks a streaming block walks in turn (at most; one partial-sum entry per
// group), and the fewest blocks a streaming launch should have: a small batch
// takes fewer chunks per block, down to one, so that its launch still fills
// the GPU (WfGeo.sgroup).
#ifndef WF_STREAM_GROUP
#define WF_STREAM_GROUP 8
#endif
#define WF_STREAM_MIN_BLOCKS 2048
// FFT stages of the L-BFGS iteration on ping-pong passes with direct global
// input/output (1) or on in-place shared-memory passes (0).
#ifndef WF_FFT_PP
#define WF_FFT_PP 1
#endif
// Inverse column stage of the iteration as a persistent kernel fed by TMA (1)
// or one block per tile (0, also used when the driver lacks the tensor-map
// encoder).  The row and forward column stages stay one block per tile: their
// persistent TMA-fed forms measured slower (0.66 vs 0.59 ms, 0.93 vs 0.80 ms
// on the 120 x 1024^2 batch).
#ifndef WF_COLINV_TMA
#define WF_COLINV_TMA 1
#endif

// Work queue for the objective pass's inverse column stage: the resident
// blocks take (map, tile) items from an atomic counter, in order, each claiming
// its next item before it transforms the current one and asking L2 for that
// item's rows (1.63 ms per 120 x 1024^2 pass against 1.69 with the items taken
// round-robin).
#ifndef WF_COLINV_QUEUE
#define WF_COLINV_QUEUE 1
#endif

// Items ahead whose rows the objective pass's persistent inverse column stage
// asks L2 for (one: 1.70 ms per 120 x 1024^2 pass; two: 1.75; three: 1.77).
#ifndef WF_COLINV_AHEAD
#define WF_COLINV_AHEAD 1
#endif

// Resident blocks per SM requested from the compiler for the FFT-stage kernels.
// FP32: three blocks of 256 threads (85 registers a thread; the radix-16 passes
// spill a few hundred bytes to L1-resident local memory, and the extra resident
// warps still win over two blocks by 8-17% per stage).  FP64: one block.
#ifndef WF_MINB32
#define WF_MINB32 3
#endif
#define WF_MINB(T) (sizeof(T) == 4 ? WF_MINB32 : 1)
// The same for the objective pass's forward column stage (k_col_fwd): its tile
// and tables take 40 KB of shared memory, so four blocks fit, and at 64
// registers it does not spill (1.67 against 1.73 ms for the 120 x 1024^2 pass;
// five blocks, 48 registers: 1.76 ms).  Two channels keep three blocks (at 64
// registers they spill).  The iteration's forward stage has its own setting
// below.
#ifndef WF_MINB_COLFWD32
#define WF_MINB_COLFWD32 4
#endif
#define WF_MINB_COLFWD(T, C) (sizeof(T) == 4 ? ((C) == 1 ? WF_MINB_COLFWD32 : WF_MINB32) : 1)
// The iteration's forward column stage (k_lb_colfwd): blocks per SM, and the
// groups its epilogue takes its rows of p and g in.  Four groups fit 64
// registers without spills at four blocks per SM: 0.668 against 0.683 ms (one
// group, 80 registers, three blocks) on 120 x 1024^2.  Two channels (E/B) keep
// three blocks, where 64 registers would spill.
#ifndef WF_MINB_LBCOLFWD32
#define WF_MINB_LBCOLFWD32 4
#endif
#define WF_MINB_LBCOLFWD(T, C) (sizeof(T) == 4 ? ((C) == 1 ? WF_MINB_LBCOLFWD32 : WF_MINB32) : 1)
#ifndef WF_LBCF_SPLIT
#define WF_LBCF_SPLIT 4
#endif

// Partial-sum slots per map (one FP64 value per block and slot).
#define WF_MAXM 32
#define WF_SLOT_PRIOR 0                         // sum |s|^2 (half-plane weights)
#define WF_SLOT_DATA 1                          // sum r W r
#define WF_SLOT_OUT2 2                          // sum |out|^2 of the column-forward output
#define WF_SLOT_GP 3                            // <g, P_i>, i < WF_MAXM
#define WF_SLOT_GQ (WF_SLOT_GP + WF_MAXM)       // <g, Q_i>
#define WF_SLOT_GG (WF_SLOT_GQ + WF_MAXM)       // <g, g>
#define WF_SLOT_QQI (WF_SLOT_GG + 1)            // <q, Q_i>
#define WF_SLOT_QQ (WF_SLOT_QQI + WF_MAXM)      // <q, q>
#define WF_SLOT_PQ (WF_SLOT_QQ + 1)             // <p, q>
#define WF_SLOT_GQN (WF_SLOT_PQ + 1)            // <g, q>
#define WF_SLOT_GPN (WF_SLOT_GQN + 1)           // <g, p>
#define WF_SLOT_PP (WF_SLOT_GPN + 1)            // <p, p>
#define WF_NSLOT (WF_SLOT_PP + 1)

// Per-map L-BFGS state, FP64, resident on the device.  The history holds m
// pairs as unscaled directions P_i and their Hessian products Q_i = H P_i;
// the curvature pair is (s_i, y_i) = (alpha_i P_i, alpha_i Q_i).  Dot products
// among the stored vectors are kept as Gram matrices so that the two-loop
// recursion runs on scalars.
struct WfLbMap {
  int k;            // iterations completed
  int npairs;       // valid pairs in the ring (<= m)
  int head;         // slot of the newest pair (-1: none)
  int next;         // slot receiving the next direction
  int active;       // 1 while iterating
  int status;       // wf_status of this map
  int evals;        // operator applications
  int pend_slot;    // slot of the pending update
  int s_k;          // steps folded into s: s = s0 + sum over steps i < s_k of alpha_i P_(i mod m)
  int pad_;
  double pend_alpha;  // pending update g += a Q[pend_slot] (s follows when the steps are folded)
  double chi2, chi2_prev, gg, gg0;
  double dg;                    // direction p = dg g + sum dP_i P_i + dQ_i Q_i
  double dP[WF_MAXM], dQ[WF_MAXM];
  double alpha[WF_MAXM];        // step of pair i
  double gP[WF_MAXM], gQ[WF_MAXM];
  double PP[WF_MAXM * WF_MAXM], PQ[WF_MAXM * WF_MAXM], QQ[WF_MAXM * WF_MAXM];
};

// The lowest plan with the same passes as `plan` at length 2^lgL (the kernel
// instantiation that runs it).
__host__ __device__ inline int wf_plan_eff(int lgL, int plan) {
  for (int q = 0; q < plan; ++q) {
    bool same = wf_plan_np(lgL, q) == wf_plan_np(lgL, plan);
    for (int i = 0; same && i < wf_plan_np(lgL, plan); ++i) same = wf_plan_bits(lgL, q, i) == wf_plan_bits(lgL, plan, i);
    if (same) return q;
  }
  return plan;
}

// Band sums that do not depend on scheduling.  Every lane of a warp offers
// one (band l, value v) pair (l < 0: none); lanes with the same band are
// summed in lane order and the lowest of them adds the sum to bins[l], a row
// of per-warp bins that only this warp writes, so the result is the same on
// every run.  All 32 lanes must call it.
__device__ __forceinline__ void wf_warp_bin_add(double* bins, int l, double v) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int l0 = __shfl_sync(full, l, 0);
  if (__all_sync(full, l == l0)) {  // one band across the warp (the common case)
    double t = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(full, t, o);
    if (lane == 0 && l0 >= 0) bins[l0] += t;
    return;
  }
  double t = 0.0;
  bool lead = l >= 0;
  for (int src = 0; src < 32; ++src) {
    const int ls = __shfl_sync(full, l, src);
    const double vs = __shfl_sync(full, v, src);
    if (ls == l) {
      t += vs;
      if (src < lane) lead = false;
    }
  }
  if (lead) bins[l] += t;
}

// Launch geometry of one (ny, nx, C) shape: C channels of ny rows by nx
// pixels, both powers of two.  The column stages run length-ny transforms over
// the packed half plane of ny rows by h = nx/2 columns; the row stages run the
// length-nx real transforms.
// Kernel variants of the L-BFGS FFT stages, chosen per shape by the autotuner
// (wf_solve.cu) or forced through wf_opts.fft_variant.
enum { WF_COLINV_TMA_K = 1, WF_COLINV_PP_K = 2, WF_COLINV_INPLACE_K = 3 };
enum { WF_ROW_PP_K = 1, WF_ROW_INPLACE_K = 2 };
#define WF_TUNE_MAXDIV 4  // tiles may be 1, 2 or 4 times narrower than the widest

struct WfGeo {
  int n, h, lgn, lgh, C;  // n = ny rows (column-transform length), h = nx / 2
  int nx, lgnx;           // pixels per row
  int ksx, ksy;           // wavevector of mode (my, mx) along (ksx mx, ksy my): square pixels
  int TC, ntile;   // packed columns per column tile, tiles per map
  int RB, nrb;     // rows per row block (over the C*n rows), row blocks per map
  int ncomb;       // partial sums per map and slot of the streaming L-BFGS kernels
  int sgroup;      // chunks a streaming block walks (WF_STREAM_GROUP, fewer for small batches)
  int maxblk;      // stride of the partial-sum slots: covers every tile choice
  int colinv_kind, row_kind;  // WF_COLINV_*_K, WF_ROW_*_K
  int tc_div, rb_div;         // TC and RB are the widest tile divided by these (1, 2, 4)
  int col_plan, row_plan;     // radix plans of the ping-pong column and row passes (0..WF_NPLAN-1)
};

// Widest tiles and the default kernel variants.
// B: maps per launch, which sets the streaming kernels' chunk groups (0: many).
WfGeo wf_make_geo(int ny, int nx, int C, int B = 0);
inline WfGeo wf_make_geo(int n, int C) { return wf_make_geo(n, n, C); }
// Blocks per map of the band reductions: about 4096 modes each, at most 64.
inline int wf_band_nblk(const WfGeo& g) {
  const long long nsp = (long long)g.C * g.n * (g.h + 1);
  const long long k = (nsp + 4095) / 4096;
  return (int)(k < 1 ? 1 : (k > 64 ? 64 : k));
}
// Tiles tc_div / rb_div times narrower (TC >= 2, RB >= 1), the same stride.
WfGeo wf_geo_variant(const WfGeo& base, int colinv_kind, int row_kind, int tc_div, int rb_div, int col_plan = 0,
                     int row_plan = 0);

// Device pointers of one problem, in the working type T (float or double).
struct WfBufs {
  const void* d;      // [B][C][ny][nx]
  const void* w;      // [B][C][ny][nx]   mask * Ninv
  const void* sp;     // [B or 1][C][ny][h+1]   sqrt(P / (ny nx))
  long long sp_stride;  // elements between maps' sqrt(P) tables (0 if shared)
  void* scratch;      // [B][C][ny][h] complex: between the column and row stages
  double* part;       // [B][WF_NSLOT][maxblk]
  const void* tw;     // twiddle table, WF_NT complex of type T
  int* ticket;        // device counter of the objective pass's inverse column stage
                      // work queue (nullptr: that stage runs its round-robin form)
  int B;
};

// Row-stage variants.
enum { WF_ROW_DATA = 0, WF_ROW_NODATA = 1, WF_ROW_SIGNAL = 2, WF_ROW_SIM = 3, WF_ROW_RFFT = 4 };
// Column-stage input layouts.
enum { WF_IN_PK = 0, WF_IN_STD = 1 };

// Kernel launchers (defined in wf_ops_f32.cu / wf_ops_f64.cu).
template <typename T>
cudaError_t wf_launch_prep(const WfGeo& g, const void* const* dptr, const unsigned char* const* mptr,
                           const void* const* nptr, const void* const* pptr, int in_f64, int B,
                           void* d, void* w, void* sp, int sp_shared, int* flags, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_set_data(const WfGeo& g, const void* src, int B, void* d, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_eval(const WfGeo& g, const WfBufs& b, int row_mode, int in_layout,
                           const void* src, void* dst, double* chi2, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_signal(const WfGeo& g, const WfBufs& b, int in_layout, const void* src,
                             void* xout, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_simulate(const WfGeo& g, const WfBufs& b, const void* z, const void* noise,
                               void* dout, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_band_energy(const WfGeo& g, int B, const void* s, const int16_t* band,
                                  const double* theta, int n_bands, double* bpart, double* E, cudaStream_t st);
// L-BFGS kernels.  Streaming-kernel modes: full iteration, materialise only, dots only.
enum { WF_LB1_FULL = 0, WF_LB1_MATERIALIZE = 1, WF_LB1_DOTS = 2 };
// The steps taken but not yet added to s are folded in one pass once this
// many have gathered (their P slots are still in the ring: at most m - 1 of
// them), or whenever s itself is needed.
__host__ __device__ inline int wf_sfold(int m) { return m > 1 ? m - 1 : 1; }
// Default bound of a device-side wait, SM clock cycles (about 2 s at 2.07 GHz).
#define WF_WAIT_CYCLES_DEFAULT 4000000000ll
struct WfLbBufs {
  WfLbMap* st;      // [B]
  void* s;          // packed state [B][C][ny][h]
  void* g;          // packed gradient
  void* ring;       // [2m][B][C][ny][h]: P slots then Q slots
  int m;
  int inject_map;   // map whose tile copies are never issued (-1: none), see wf_opts
  long long spin_limit;  // bound of device waits, SM cycles
};
// Launches shared by several problems (wf_map_solve_many: one problem per map
// shape of a heterogeneous batch).  Every problem keeps its own geometry,
// buffers and L-BFGS state; a shared launch covers the blocks of every
// problem's own grid, problem q's at blocks start[q] .. start[q+1] - 1, and
// each block runs the single-problem kernel body at its coordinates in its
// problem's grid, so that every map computes what it computes alone with the
// same FFT-stage variant.  The problems share the working type and C.
#define WF_MULTI_MAX 8
struct WfMultiArgs {
  int np;
  WfGeo g[WF_MULTI_MAX];
  WfBufs b[WF_MULTI_MAX];
  WfLbBufs lb[WF_MULTI_MAX];
};
// FFT-stage variant the shared launches run (ping-pong inverse column and row
// stages, radix plan 0; the widest tiles here, the tile widths tuned per
// problem when the solve autotunes).
#define WF_MULTI_VARIANT 2111
template <typename T>
cudaError_t wf_launch_multi_comb(const WfMultiArgs& a, int mode, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_multi_colinv(const WfMultiArgs& a, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_multi_row(const WfMultiArgs& a, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_multi_colfwd(const WfMultiArgs& a, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_multi_qdots(const WfMultiArgs& a, cudaStream_t st);

template <typename T>
cudaError_t wf_launch_lb_comb(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, int mode, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_lb_colinv(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_lb_row(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_lb_colfwd(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_lb_qdots(const WfGeo& g, const WfBufs& b, const WfLbBufs& lb, cudaStream_t st);
// Full objective+gradient pass on packed vectors (src -> dst), all maps.
template <typename T>
cudaError_t wf_launch_eval_pk(const WfGeo& g, const WfBufs& b, const void* src, void* dst, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_eval_bands(const WfGeo& g, const WfBufs& b, const void* src, void* dst, double* chi2,
                                 const int16_t* band, int n_b, double* bpart, double* dq, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_band_scale(const WfGeo& g, const void* sp0, void* sp, int ntab, const int16_t* band,
                                 const double* q, int n_b, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_pack(const WfGeo& g, int B, const void* std_in, void* pk_out, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_unpack(const WfGeo& g, int B, const void* pk_in, void* std_out, cudaStream_t st);
