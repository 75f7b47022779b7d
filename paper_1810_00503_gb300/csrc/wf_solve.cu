// Device-resident L-BFGS MAP driver (Sec. 2.2: the MAP field minimises chi^2;
// L-BFGS builds a low-rank model of the curvature D, eq_curv, never forming it).
//
// One iteration for every map still active:
//   k_lb_comb   s, g += a (P, Q) of the previous step; p = direction; <g, .>
//   k_lb_colinv, k_lb_row, k_lb_colfwd   q = H p and <q,q>, <p,q>, <g,q>, <g,p>
//   k_lb_qdots  <q, Q_i>
//   k_lb_scalar (one warp per map) exact step a = -g.p / p.Hp along p (the
//             objective is quadratic, so this is the point a Wolfe line search
//             converges to), chi^2 update, Gram-matrix update of the new pair
//             (s, y) = (a p, a q), convergence test, and the two-loop recursion
//             (Nocedal & Wright, Numerical Optimization, Alg. 7.4) evaluated on
//             the Gram matrices to give the next direction's coefficients.
// Iterations are captured in CUDA graphs, `check_every` per graph; the host
// reads one counter of active maps per graph launch.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "wf_api_internal.h"

struct WfScalarArgs {
  double gtol2, dchi2, c1, c2;
  int max_iter, m, ntile, nrb, ncomb, maxblk, phase, init, ls;
  int hcap;      // convergence records kept per map (0: none)
  double* hist;  // [B][hcap][5] ring of (k, chi2, |g|/|g0|, alpha, evals)
};
// Legacy and per-thread default stream handles cannot be captured; the solver
// then runs on its own stream, ordered after the caller's with events.
static inline bool wf_capturable(cudaStream_t s) {
  return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
}

struct WfSolver {
  int m;
  int B;
  int shared_tune;    // the next start tunes only what the shared launches can run

  void* s;
  void* g;
  void* ring;
  WfLbMap* st;
  int* nact;          // device counter of active maps
  int* nact_host;     // pinned
  double* stats_dev;  // [B][4]: k, evals, status, chi2 ... see k_lb_final
  double* stats_host; // pinned
  cudaStream_t stream;
  cudaEvent_t ev_in, ev_out;
  cudaGraphExec_t exec;
  int g_chunk, g_maxit, g_m, g_ls, g_inject, g_variant;
  double g_gtol2, g_dchi2, g_c1, g_c2;
  long long g_spin;
  int started;
  int graph_pending;  // capture the iteration graph after the next plain iteration (a resumed solve)
  cudaStream_t work, g_stream;  // stream in use; stream the graph was captured on
  long long iters;     // iterations launched since the last start
  wf_opts o;
  WfScalarArgs A;
  double* hist;        // convergence ring, hist_cap records per map (allocated on demand)
  int hist_cap;
  double* g_hist;      // ring the graph was captured with
  int g_hcap;
  // FP64 state of the refined solve (wf_map_solve_refined), allocated on its
  // first use: outer state and gradient (packed, FP64), and for a MIXED problem
  // FP64 copies of d, W and sqrt(P)/n with the FP64 operator's scratch.
  void* r_s64;
  void* r_g64;
  void* r_d64;
  void* r_w64;
  void* r_sp64;
  void* r_scr64;
  double* r_res;       // [B][WF_RES] per-map outer results (device)
  double* r_res_host;  // pinned copy
};

// Per-map record of the refined solve: chi^2, |g|^2 and |s|^2 at the FP64
// state, the certificate |g| / (2 |s|), inner iterations and evaluations so
// far, the worst inner status, and |g|^2 at the first outer evaluation.
enum { WF_RES_CHI2 = 0, WF_RES_GG, WF_RES_SS, WF_RES_CERT, WF_RES_ITERS, WF_RES_EVALS, WF_RES_STATUS, WF_RES_GG0,
       WF_RES };

enum { WF_PH_ITER = 0, WF_PH_REFRESH = 1 };

#define WF_SW 1                        // warps (maps) per block of the scalar kernel
#define WF_SCAL_SLOTS (6 + 3 * WF_MAXM)  // partial-sum slots one scalar step reads at most

// Sum over the nb block partials of one slot (every lane gets the total).
__device__ __forceinline__ double wf_warp_slot(const double* pb, int slot, int nb, int maxblk) {
  const int lane = threadIdx.x & 31;
  double v = 0.0;
  for (int i = lane; i < nb; i += 32) v += pb[(size_t)slot * maxblk + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double wf_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block partials of ns slots: out[k] = sum_i pb[slots[k] * maxblk + i], i < cnt[k].
// Every lane first sums its stride-32 share of every slot (independent loads),
// then lane k adds the 32 shares of slot k in lane order: a fixed order, so
// the result is deterministic.
__device__ void wf_gather_slots(const double* pb, int maxblk, const int* slots, const int* cnt, int ns,
                                double (*red)[33], double* out) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < ns; ++k) {
    const double* src = pb + (size_t)slots[k] * maxblk;
    double v = 0.0;
    for (int i = lane; i < cnt[k]; i += 32) v += src[i];
    red[k][lane] = v;
  }
  __syncwarp();
  for (int k = lane; k < ns; k += 32) {
    double v = 0.0;
    for (int l = 0; l < 32; ++l) v += red[k][l];
    out[k] = v;
  }
  __syncwarp();
}

// Two-loop recursion on coefficients (Nocedal & Wright, Alg. 7.4): r = H_k g
// expressed over the basis {g, P_i, Q_i}; the direction is p = -r.  Lane l
// holds the coefficients of history slot l (m <= 32); each step of the two
// loops is one warp sum over the stored pairs.  Called by all 32 lanes.
__device__ void wf_two_loop(WfLbMap& M, int m, int lane) {
  const int np = M.npairs, head = M.head;
  const bool act = np > 0 && lane < m && (head - lane + m) % m < np;  // slot `lane` holds a stored pair
  double cP = 0.0, cQ = 0.0, aa = 0.0, cg = 1.0;
  for (int q = 0; q < np; ++q) {  // newest to oldest
    const int i = (head - q + m) % m;
    const double t = act ? cP * M.PP[i * WF_MAXM + lane] + cQ * M.PQ[i * WF_MAXM + lane] : 0.0;
    const double d = cg * M.gP[i] + wf_warp_sum(t);
    const double ai = M.alpha[i];
    const double rho = 1.0 / (ai * ai * M.PQ[i * WF_MAXM + i]);
    const double a = rho * ai * d;
    if (lane == i) {
      aa = a;
      cQ -= a * ai;
    }
  }
  double gamma = 1.0;
  if (np > 0) gamma = M.PQ[head * WF_MAXM + head] / M.QQ[head * WF_MAXM + head];
  cg *= gamma;
  cP *= gamma;
  cQ *= gamma;
  for (int q = np - 1; q >= 0; --q) {  // oldest to newest
    const int i = (head - q + m) % m;
    const double t = act ? cP * M.PQ[lane * WF_MAXM + i] + cQ * M.QQ[i * WF_MAXM + lane] : 0.0;
    const double d = cg * M.gQ[i] + wf_warp_sum(t);
    const double ai = M.alpha[i];
    const double rho = 1.0 / (ai * ai * M.PQ[i * WF_MAXM + i]);
    const double beta = rho * ai * d;
    if (lane == i) cP += ai * (aa - beta);
  }
  __syncwarp();  // every lane has read the old coefficients' Gram entries
  if (lane == 0) {
    M.dg = -cg;
    M.next = (head + 1) % m;
  }
  if (lane < m) {
    M.dP[lane] = -cP;
    M.dQ[lane] = -cQ;
  }
  __syncwarp();
}

// Strong Wolfe step along p (Nocedal & Wright, Alg. 3.5, zoom Alg. 3.6) on the
// exact quadratic model of chi^2: f(a) = phi(a) - phi(0) = a d0 + a^2 c / 2 and
// phi'(a) = d0 + a c, with d0 = g.p < 0 and c = p.Hp > 0.  Trial a = 1, then
// doubling up to 1e6; zoom by quadratic interpolation of f(lo), phi'(lo), f(hi),
// kept inside the middle 80% of the bracket (else bisection).
__device__ double wf_wolfe_zoom(double lo, double f_lo, double d_lo, double hi, double f_hi, double d0, double c,
                                double c1, double c2) {
  for (int it = 0; it < 60; ++it) {
    const double da = hi - lo, den = 2.0 * (f_hi - f_lo - d_lo * da);
    double a = den > 0.0 ? lo - d_lo * da * da / den : 0.5 * (lo + hi);
    const double bl = fmin(lo, hi), bh = fmax(lo, hi);
    if (!(a >= bl + 0.1 * (bh - bl) && a <= bh - 0.1 * (bh - bl))) a = 0.5 * (lo + hi);
    const double f = a * d0 + 0.5 * a * a * c, d = d0 + a * c;
    if (f > c1 * a * d0 || f >= f_lo) {
      hi = a;
      f_hi = f;
    } else {
      if (fabs(d) <= -c2 * d0) return a;
      if (d * (hi - lo) >= 0.0) {
        hi = lo;
        f_hi = f_lo;
      }
      lo = a;
      f_lo = f;
      d_lo = d;
    }
  }
  return lo;
}
__device__ double wf_wolfe_step(double d0, double c, double c1, double c2) {
  double a_prev = 0.0, f_prev = 0.0, d_prev = d0, a = 1.0;
  for (int i = 0; i < 40; ++i) {
    const double f = a * d0 + 0.5 * a * a * c, d = d0 + a * c;
    if (f > c1 * a * d0 || (i > 0 && f >= f_prev)) return wf_wolfe_zoom(a_prev, f_prev, d_prev, a, f, d0, c, c1, c2);
    if (fabs(d) <= -c2 * d0) return a;
    if (d >= 0.0) return wf_wolfe_zoom(a, f, d, a_prev, f_prev, d0, c, c1, c2);
    a_prev = a;
    f_prev = f;
    d_prev = d;
    a = fmin(2.0 * a, 1e6);
  }
  return a;
}

// One warp per map.  ITER: exact or Wolfe step along p, chi^2 and Gram-matrix
// update of the new pair, convergence test, two-loop for the next direction.
// REFRESH: true chi^2 and gradient dots after a full evaluation.
__device__ __forceinline__ void wf_lb_scalar(WfLbMap* st, const double* part, const WfScalarArgs& A, int b,
                                             int* nact) {
  __shared__ double red[WF_SCAL_SLOTS][33];
  __shared__ double S[WF_SCAL_SLOTS];
  __shared__ int slots[WF_SCAL_SLOTS], cnt[WF_SCAL_SLOTS];
  const int lane = threadIdx.x & 31;
  WfLbMap& M = st[b];
  const double* pb = part + (size_t)b * WF_NSLOT * A.maxblk;
  const int m = A.m;
  // Steps the streaming pass just folded into s (the rule of k_lb_comb): all of
  // them before a refresh and for a map that had stopped, otherwise all once
  // wf_sfold(m) have gathered.
  if (lane == 0 && (A.phase != WF_PH_ITER || !M.active || M.k - M.s_k >= wf_sfold(m))) M.s_k = M.k;
  __syncwarp();
  if (M.status == WF_ETIMEOUT) {  // a bounded device wait gave up on this map's data
    if (lane == 0) {
      M.active = 0;
      M.pend_alpha = 0.0;
    }
    return;
  }
  if (A.phase == WF_PH_ITER) {
    if (!M.active) {
      if (lane == 0) M.pend_alpha = 0.0;
      return;
    }
    const int np = M.npairs, head = M.head, nx = M.next;
    // slot list: 0 GG, 1 QQ, 2 PQ, 3 GQN, 4 GPN, 5 PP, then per stored pair q:
    // 6 + 3q GP, 7 + 3q GQ, 8 + 3q QQI (of slot (head - q) mod m)
    if (lane == 0) {
      const int fixed[6] = {WF_SLOT_GG, WF_SLOT_QQ, WF_SLOT_PQ, WF_SLOT_GQN, WF_SLOT_GPN, WF_SLOT_PP};
      for (int k = 0; k < 6; ++k) {
        slots[k] = fixed[k];
        cnt[k] = k == 0 ? A.ncomb : A.ntile;
      }
      for (int q = 0; q < np; ++q) {
        const int sl = (head - q + m) % m;
        slots[6 + 3 * q] = WF_SLOT_GP + sl;
        slots[7 + 3 * q] = WF_SLOT_GQ + sl;
        slots[8 + 3 * q] = WF_SLOT_QQI + sl;
        cnt[6 + 3 * q] = cnt[7 + 3 * q] = cnt[8 + 3 * q] = A.ncomb;
      }
    }
    __syncwarp();
    wf_gather_slots(pb, A.maxblk, slots, cnt, 6 + 3 * np, red, S);
    const double ggk = S[0], qq = S[1], pq = S[2], gq = S[3], gp = S[4], pp = S[5];
    // position of slot `lane` among the stored pairs (newest first), if stored
    const int ql = (head - lane + m) % m;
    const bool act = np > 0 && lane < m && ql < np;
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(gp) || !isfinite(ggk) ||
        !(pq > 1e-12 * sqrt(pp * qq))) {
      // no decrease along p, a non-finite value, or A8's curvature test
      // s.y > 1e-12 |s| |y| failing (on this positive definite objective only
      // when rounding has taken over): the map stops
      if (lane == 0) {
        M.evals += 1;
        M.status = (isfinite(pq) && isfinite(gp) && isfinite(ggk)) ? WF_ELINESEARCH : WF_ENONFINITE;
        M.active = 0;
        M.pend_alpha = 0.0;
      }
      return;
    }
    const double alpha = A.ls == WF_LS_WOLFE ? wf_wolfe_step(gp, pq, A.c1, A.c2) : -gp / pq;
    // Gram row of the new direction p = dg g + sum (dP_l P_l + dQ_l Q_l), from the old
    // entries: lane i computes <p, P_i> and <p, Q_i> = <P_i, H p> for its stored slot i
    double rowPP = 0.0, rowPQ = 0.0, gPk = 0.0, gQk = 0.0;
    if (act) {
      gPk = S[6 + 3 * ql];
      gQk = S[7 + 3 * ql];
    }
    if (act && lane != nx) {
      const int i = lane;
      double a = M.dg * gPk, c = M.dg * gQk;
      for (int u = 0; u < np; ++u) {
        const int l = (head - u + m) % m;
        a += M.dP[l] * M.PP[l * WF_MAXM + i] + M.dQ[l] * M.PQ[i * WF_MAXM + l];
        c += M.dP[l] * M.PQ[l * WF_MAXM + i] + M.dQ[l] * M.QQ[l * WF_MAXM + i];
      }
      rowPP = a;
      rowPQ = c;
    }
    __syncwarp();  // all reads of the old Gram entries are done
    if (act && lane != nx) {
      const int i = lane;
      M.PP[nx * WF_MAXM + i] = M.PP[i * WF_MAXM + nx] = rowPP;
      M.PQ[nx * WF_MAXM + i] = rowPQ;  // <p, Q_i>
      M.PQ[i * WF_MAXM + nx] = rowPQ;  // <P_i, H p> = <H P_i, p>
      const double qqi = S[8 + 3 * ql];
      M.QQ[nx * WF_MAXM + i] = M.QQ[i * WF_MAXM + nx] = qqi;
      // dot products of g_{k+1} = g_k + alpha q with the stored vectors
      M.gP[i] = gPk + alpha * rowPQ;
      M.gQ[i] = gQk + alpha * qqi;
    }
    bool done = false;
    if (lane == 0) {
      M.evals += 1;
      M.chi2_prev = M.chi2;
      M.chi2 = M.chi2 + alpha * gp + 0.5 * alpha * alpha * pq;
      M.PP[nx * WF_MAXM + nx] = pp;
      M.PQ[nx * WF_MAXM + nx] = pq;
      M.QQ[nx * WF_MAXM + nx] = qq;
      M.gP[nx] = gp + alpha * pq;
      M.gQ[nx] = gq + alpha * qq;
      double gg = ggk + 2.0 * alpha * gq + alpha * alpha * qq;
      if (gg < 0.0) gg = 0.0;
      M.gg = gg;
      M.alpha[nx] = alpha;
      M.pend_alpha = alpha;
      M.pend_slot = nx;
      M.head = nx;
      M.npairs = np + 1 < m ? np + 1 : m;
      M.next = (nx + 1) % m;
      M.k += 1;
      if (A.hcap > 0) {  // convergence record of iteration k
        double* rec = A.hist + ((size_t)b * A.hcap + (M.k - 1) % A.hcap) * 5;
        rec[0] = M.k;
        rec[1] = M.chi2;
        rec[2] = M.gg0 > 0.0 ? sqrt(gg / M.gg0) : 0.0;
        rec[3] = alpha;
        rec[4] = M.evals;
      }
      if (!isfinite(M.chi2) || !isfinite(gg)) { done = true; M.status = WF_ENONFINITE; }
      else if (gg <= A.gtol2 * M.gg0) { done = true; }
      else if (A.dchi2 > 0.0 && fabs(M.chi2 - M.chi2_prev) < A.dchi2) { done = true; }
      else if (M.k >= A.max_iter) { done = true; M.status = WF_ENOTCONVERGED; }
      if (done) M.active = 0;
    }
    done = __shfl_sync(0xffffffffu, done, 0);
    __syncwarp();
    if (!done) {
      wf_two_loop(M, m, lane);
      if (lane == 0) atomicAdd(nact, 1);
    }
    return;
  }
  // WF_PH_REFRESH: true chi^2 and gradient at the current state, exact dots.
  const int np = A.init ? 0 : M.npairs, head = M.head;
  if (lane == 0) {
    slots[0] = WF_SLOT_PRIOR;
    cnt[0] = A.ntile;
    slots[1] = WF_SLOT_DATA;
    cnt[1] = A.nrb;
    slots[2] = WF_SLOT_GG;
    cnt[2] = A.ncomb;
    for (int q = 0; q < np; ++q) {
      const int sl = (head - q + m) % m;
      slots[3 + 2 * q] = WF_SLOT_GP + sl;
      slots[4 + 2 * q] = WF_SLOT_GQ + sl;
      cnt[3 + 2 * q] = cnt[4 + 2 * q] = A.ncomb;
    }
  }
  __syncwarp();
  wf_gather_slots(pb, A.maxblk, slots, cnt, 3 + 2 * np, red, S);
  const double prior = S[0], data = S[1], gg = S[2];
  bool go = false;
  if (lane == 0) {
    if (A.init) {
      M.k = 0;
      M.npairs = 0;
      M.head = -1;
      M.next = 0;
      M.status = WF_OK;
      M.evals = 1;
      M.gg0 = gg;
      M.active = 1;
      M.chi2_prev = prior + data;
    } else {
      M.evals += 1;
    }
    M.chi2 = prior + data;
    M.gg = gg;
    M.pend_alpha = 0.0;
    if (M.active) {
      for (int q = 0; q < np; ++q) {
        const int sl = (head - q + m) % m;
        M.gP[sl] = S[3 + 2 * q];
        M.gQ[sl] = S[4 + 2 * q];
      }
      bool done = false;
      if (!isfinite(M.chi2) || !isfinite(gg)) { done = true; M.status = WF_ENONFINITE; }
      else if (gg <= A.gtol2 * M.gg0) { done = true; M.status = WF_OK; }
      else if (M.k >= A.max_iter) { done = true; M.status = WF_ENOTCONVERGED; }
      if (done) M.active = 0;
      go = !done;
    }
  }
  go = __shfl_sync(0xffffffffu, go, 0);
  __syncwarp();
  if (go) {
    wf_two_loop(M, m, lane);
    if (lane == 0) atomicAdd(nact, 1);
  }
}

__global__ void __launch_bounds__(32 * WF_SW)
k_lb_scalar(WfLbMap* st, const double* part, WfScalarArgs A, int B, int* nact) {
  if ((int)blockIdx.x < B) wf_lb_scalar(st, part, A, blockIdx.x, nact);
}

// The scalar step of several problems in one launch (wf_map_solve_many): one
// block (warp) per map of every problem, problem q's maps at blocks
// start[q] .. start[q+1] - 1; and the zeroing of their active counters.
struct WfMultiScalar {
  int np;
  int start[WF_MULTI_MAX + 1];
  WfLbMap* st[WF_MULTI_MAX];
  const double* part[WF_MULTI_MAX];
  int* nact[WF_MULTI_MAX];
  WfScalarArgs A[WF_MULTI_MAX];
};
__global__ void __launch_bounds__(32 * WF_SW) k_multi_scalar(const __grid_constant__ WfMultiScalar ms) {
  const int bid = blockIdx.x;
  int q = 0;
  while (q + 1 < ms.np && bid >= ms.start[q + 1]) ++q;
  wf_lb_scalar(ms.st[q], ms.part[q], ms.A[q], bid - ms.start[q], ms.nact[q]);
}
__global__ void k_multi_zero(const __grid_constant__ WfMultiScalar ms) {
  if ((int)threadIdx.x < ms.np) *ms.nact[threadIdx.x] = 0;
}

// Final statistics from the closing true evaluation: [k, evals, status, chi2, gnorm_rel].
__global__ void k_lb_final(const WfLbMap* st, const double* part, int ntile, int nrb, int maxblk, int B,
                           double* out) {
  const int w = threadIdx.x >> 5;
  const int b = blockIdx.x * WF_SW + w;
  if (b >= B) return;
  const double* pb = part + (size_t)b * WF_NSLOT * maxblk;
  const double prior = wf_warp_slot(pb, WF_SLOT_PRIOR, ntile, maxblk);
  const double data = wf_warp_slot(pb, WF_SLOT_DATA, nrb, maxblk);
  const double g2 = wf_warp_slot(pb, WF_SLOT_OUT2, ntile, maxblk);
  if ((threadIdx.x & 31) != 0) return;
  const WfLbMap& M = st[b];
  out[b * 5 + 0] = M.k;
  out[b * 5 + 1] = M.evals + 1;
  out[b * 5 + 2] = M.status;
  out[b * 5 + 3] = prior + data;
  out[b * 5 + 4] = M.gg0 > 0.0 ? sqrt(g2 / M.gg0) : 0.0;
}

// ---------------------------------------------------------------------------
// Kernels of the refined solve.  Spectra are handled as flat arrays of reals
// (the packed complex layout interleaves re and im), `per` reals per map.
// ---------------------------------------------------------------------------
// Blocks of 256 threads for a grid-stride loop over `total` elements.
static inline int wf_grid(size_t total) {
  size_t b = (total + 255) / 256;
  return (int)(b > 2048 ? 2048 : (b < 1 ? 1 : b));
}

template <typename S, typename D>
__global__ void k_convert(const S* in, D* out, size_t total) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) out[i] = (D)in[i];
}

// s64 += delta (the correction of one round, in the working type).
template <typename T>
__global__ void k_refine_accum(const T* delta, double* s64, size_t total) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride)
    s64[i] += (double)delta[i];
}

// After an outer FP64 evaluation: chi^2, |g|^2, |s|^2 and the certificate
// |g| / (2 |s|) of each map (the prior partial sums are |s|^2, the output
// sums |g|^2, both with the half-plane weights).  One warp per map.
__global__ void k_refine_round(const double* part, int ntile, int nrb, int maxblk, int B, int first,
                               double* res) {
  const int b = blockIdx.x;
  if (b >= B) return;
  const double* pb = part + (size_t)b * WF_NSLOT * maxblk;
  const double prior = wf_warp_slot(pb, WF_SLOT_PRIOR, ntile, maxblk);
  const double data = wf_warp_slot(pb, WF_SLOT_DATA, nrb, maxblk);
  const double gg = wf_warp_slot(pb, WF_SLOT_OUT2, ntile, maxblk);
  if ((threadIdx.x & 31) != 0) return;
  double* r = res + (size_t)b * WF_RES;
  r[WF_RES_CHI2] = prior + data;
  r[WF_RES_GG] = gg;
  r[WF_RES_SS] = prior;
  r[WF_RES_CERT] = gg == 0.0 ? 0.0 : (prior > 0.0 ? 0.5 * sqrt(gg / prior) : INFINITY);
  r[WF_RES_EVALS] += 1.0;
  if (first) r[WF_RES_GG0] = gg;
}

// Start of an inner round: the correction problem's gradient at delta = 0 is
// the FP64 gradient g64 (0 for the maps already certified, which then stop at
// once), and its chi^2 is the outer one, seeded as the prior partial sum.
template <typename T>
__global__ void k_refine_seed(const double* g64, const double* res, double tol, size_t per, T* g, double* part,
                              int ntile, int nrb, int maxblk) {
  const int b = blockIdx.y;
  const double* r = res + (size_t)b * WF_RES;
  const bool done = !(r[WF_RES_CERT] > tol) || r[WF_RES_STATUS] != 0.0;  // certified, or stopped
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < per; i += stride)
    g[(size_t)b * per + i] = done ? (T)0 : (T)g64[(size_t)b * per + i];
  if (blockIdx.x == 0) {
    double* pb = part + (size_t)b * WF_NSLOT * maxblk;
    for (int i = threadIdx.x; i < ntile; i += blockDim.x) pb[(size_t)WF_SLOT_PRIOR * maxblk + i] = i == 0 ? r[WF_RES_CHI2] : 0.0;
    for (int i = threadIdx.x; i < nrb; i += blockDim.x) pb[(size_t)WF_SLOT_DATA * maxblk + i] = 0.0;
  }
}

// After an inner round: its iterations and evaluations, and a fatal status.
__global__ void k_refine_tally(const WfLbMap* st, int B, double* res) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double* r = res + (size_t)b * WF_RES;
  r[WF_RES_ITERS] += st[b].k;
  r[WF_RES_EVALS] += st[b].evals;
  const int s = st[b].status;
  if (s == WF_ENONFINITE || s == WF_ETIMEOUT) r[WF_RES_STATUS] = s;
}

void wf_solver_free(wf_problem* p) {
  WfSolver* S = p->solver;
  if (!S) return;
  if (S->exec) cudaGraphExecDestroy(S->exec);
  void* ptrs[] = {S->s, S->g, S->ring, S->st, S->nact, S->stats_dev, S->hist, S->r_s64, S->r_g64, S->r_d64,
                  S->r_w64, S->r_sp64, S->r_scr64, S->r_res};
  for (void* q : ptrs) wf_free(p->h, q);
  if (S->r_res_host) cudaFreeHost(S->r_res_host);
  if (S->nact_host) cudaFreeHost(S->nact_host);
  if (S->stats_host) cudaFreeHost(S->stats_host);
  if (S->stream) cudaStreamDestroy(S->stream);
  if (S->ev_in) cudaEventDestroy(S->ev_in);
  if (S->ev_out) cudaEventDestroy(S->ev_out);
  free(S);
  p->solver = nullptr;
}

static wf_status ensure_solver(wf_problem* p, int m) {
  if (p->solver && p->solver->m >= m) return WF_OK;
  wf_solver_free(p);
  WfSolver* S = (WfSolver*)calloc(1, sizeof(WfSolver));
  if (!S) return wf_fail(WF_ENOMEM, "wf_map_solve: host allocation failed");
  p->solver = S;
  S->m = m;
  S->B = p->count;
  const size_t vbytes = (size_t)p->count * p->C * p->n * p->nx * p->elt;  // packed complex = ny nx reals
  wf_status s = wf_alloc(p->h, &S->s, vbytes, "L-BFGS state");
  if (s == WF_OK) s = wf_alloc(p->h, &S->g, vbytes, "L-BFGS gradient");
  if (s == WF_OK) s = wf_alloc(p->h, &S->ring, vbytes * 2 * m, "L-BFGS history");
  if (s == WF_OK) s = wf_alloc(p->h, (void**)&S->st, sizeof(WfLbMap) * p->count, "L-BFGS scalars");
  if (s == WF_OK) s = wf_alloc(p->h, (void**)&S->nact, sizeof(int), "active counter");
  if (s == WF_OK) s = wf_alloc(p->h, (void**)&S->stats_dev, sizeof(double) * 5 * p->count, "statistics");
  cudaError_t e = cudaSuccess;
  if (s == WF_OK) e = cudaMallocHost((void**)&S->nact_host, sizeof(int));
  if (s == WF_OK && e == cudaSuccess) e = cudaMallocHost((void**)&S->stats_host, sizeof(double) * 5 * p->count);
  if (s == WF_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
  if (s == WF_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_in, cudaEventDisableTiming);
  if (s == WF_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_out, cudaEventDisableTiming);
  if (s == WF_OK && e != cudaSuccess) s = wf_cuda_fail(e, "wf_map_solve: solver set-up");
  if (s != WF_OK) wf_solver_free(p);
  return s;
}

#define WF_TRY(expr)                                    \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return wf_cuda_fail(e_, #expr); \
  } while (0)

template <typename T>
static cudaError_t iteration(const wf_problem* p, const WfBufs& b, const WfLbBufs& lb, const WfScalarArgs& A,
                             WfSolver* S, cudaStream_t st) {
  cudaError_t e = wf_launch_lb_comb<T>(p->g, b, lb, WF_LB1_FULL, st);
  if (e == cudaSuccess) e = wf_launch_lb_colinv<T>(p->g, b, lb, st);
  if (e == cudaSuccess) e = wf_launch_lb_row<T>(p->g, b, lb, st);
  if (e == cudaSuccess) e = wf_launch_lb_colfwd<T>(p->g, b, lb, st);
  if (e == cudaSuccess) e = wf_launch_lb_qdots<T>(p->g, b, lb, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(S->nact, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    k_lb_scalar<<<(p->count + WF_SW - 1) / WF_SW, 32 * WF_SW, 0, st>>>(lb.st, b.part, A, p->count, S->nact);
    e = cudaGetLastError();
  }
  return e;
}

template <typename T>
static cudaError_t refresh(const wf_problem* p, const WfBufs& b, const WfLbBufs& lb, WfScalarArgs A, int init,
                           WfSolver* S, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (!init) e = wf_launch_lb_comb<T>(p->g, b, lb, WF_LB1_MATERIALIZE, st);
  if (e == cudaSuccess) e = wf_launch_eval_pk<T>(p->g, b, lb.s, lb.g, st);
  if (e == cudaSuccess) e = wf_launch_lb_comb<T>(p->g, b, lb, WF_LB1_DOTS, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(S->nact, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    A.phase = WF_PH_REFRESH;
    A.init = init;
    k_lb_scalar<<<(p->count + WF_SW - 1) / WF_SW, 32 * WF_SW, 0, st>>>(lb.st, b.part, A, p->count, S->nact);
    e = cudaGetLastError();
  }
  return e;
}

template <typename T>
static WfLbBufs lb_bufs(WfSolver* S) {
  WfLbBufs lb;
  lb.st = S->st;
  lb.s = S->s;
  lb.g = S->g;
  lb.ring = S->ring;
  lb.m = S->o.lbfgs_m;
  lb.inject_map = S->o.inject_timeout_map - 1;
  lb.spin_limit = S->o.spin_limit > 0 ? S->o.spin_limit : WF_WAIT_CYCLES_DEFAULT;
  return lb;
}

// FFT-stage variants (wf_opts.fft_variant encoding:
// 100000 f + 10000 e + 1000 a + 100 b + 10 c + d, f / e the column / row radix plans).
static int variant_code(const WfGeo& g) {
  return 100000 * g.col_plan + 10000 * g.row_plan + 1000 * g.colinv_kind + 100 * g.row_kind + 10 * g.tc_div +
         g.rb_div;
}
static bool variant_valid(int v) {
  const int f = v / 100000, e = (v / 10000) % 10, a = (v / 1000) % 10, b = (v / 100) % 10, c = (v / 10) % 10,
            d = v % 10;
  auto div_ok = [](int x) { return x == 1 || x == 2 || x == 4; };
  return v >= 1000 && f < WF_NPLAN && e < WF_NPLAN && a >= WF_COLINV_TMA_K && a <= WF_COLINV_INPLACE_K &&
         b >= WF_ROW_PP_K && b <= WF_ROW_INPLACE_K && div_ok(c) && div_ok(d);
}
static WfGeo variant_geo(const WfGeo& base, int v) {
  return wf_geo_variant(base, (v / 1000) % 10, (v / 100) % 10, (v / 10) % 10, v % 10, v / 100000,
                        (v / 10000) % 10);
}
// Radix plans q and p give the same passes for length 2^lgL.
static bool plan_same(int lgL, int p, int q) {
  if (wf_plan_np(lgL, p) != wf_plan_np(lgL, q)) return false;
  for (int i = 0; i < wf_plan_np(lgL, p); ++i)
    if (wf_plan_bits(lgL, p, i) != wf_plan_bits(lgL, q, i)) return false;
  return true;
}
static bool plan_new(int lgL, int p) {  // p differs from every lower plan
  for (int q = 0; q < p; ++q)
    if (plan_same(lgL, p, q)) return false;
  return true;
}

// Timing state for the autotuner: every map active with a full history ring
// (npairs = m, newest pair in slot m - 1, next = 0), so that the candidates
// stream what a steady-state iteration streams.
__global__ void k_tune_state(WfLbMap* st, int B, int m) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  st[b].active = 1;
  st[b].npairs = m;
  st[b].head = m - 1;
  st[b].next = 0;
}

// Autotuner: times the FFT-stage variants of the Hessian-vector pass on the
// problem's own buffers, before the solve's first refresh (whose outputs and
// the first iteration's rewrite what the timing runs write), and keeps the
// fastest.  Column choices (inverse column stage variant, radix plan and
// column tile width) are timed with the forward column stage, then the row
// choices (row stage variant, radix plan and row block height) with those
// fixed.  Results are cached in the handle per (ny, nx, C, precision,
// history length, maps).  For a problem of a batch in shared launches
// (S->shared_tune) only the stage kinds and radix plan of those launches are
// candidates (WF_MULTI_VARIANT), so only the tile widths are tuned; that
// choice is cached apart.
template <typename T>
static wf_status choose_variant(wf_problem* p, WfSolver* S, cudaStream_t st) {
  const wf_opts* o = &S->o;
  const bool shared = S->shared_tune != 0;
  const WfGeo base = shared ? variant_geo(wf_make_geo(p->n, p->nx, p->C, p->count), WF_MULTI_VARIANT)
                            : wf_make_geo(p->n, p->nx, p->C, p->count);
  if (o->fft_variant) {
    p->g = variant_geo(base, o->fft_variant);
    return WF_OK;
  }
  if (!o->autotune || o->inject_timeout_map > 0) {  // the injected wait lives in the TMA-fed stage
    p->g = base;
    return WF_OK;
  }
  const int m = S->o.lbfgs_m;
  const long long key =
      ((((((long long)p->n * 2048 + p->nx) * 4 + p->C) * 2 + p->precision) * 64 + m) * 1000000LL + p->count) * 2 +
      (shared ? 1 : 0);
  {
    std::lock_guard<std::mutex> lock(p->h->mu);
    auto it = p->h->tuned.find(key);
    if (it != p->h->tuned.end()) {
      p->g = variant_geo(base, it->second);
      return WF_OK;
    }
  }
  const WfBufs b = wf_bufs(p);
  WfLbBufs lb = lb_bufs<T>(S);
  // Candidates run against map states set to a full history ring, with the
  // start state as the direction P[0].  The first refresh and iteration
  // rewrite P[0], Q[0], the scratch and the partial sums they write.
  WfLbMap* tst = nullptr;
  if (wf_alloc(p->h, (void**)&tst, sizeof(WfLbMap) * p->count, "autotune state") != WF_OK) {
    p->g = base;  // no room to time the candidates: the defaults, not cached
    return WF_OK;
  }
  cudaError_t ce = cudaMemcpyAsync(S->ring, S->s, (size_t)p->count * p->C * p->n * p->nx * p->elt,
                                   cudaMemcpyDeviceToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(tst, 0, sizeof(WfLbMap) * p->count, st);
  if (ce == cudaSuccess) {
    k_tune_state<<<(p->count + 127) / 128, 128, 0, st>>>(tst, p->count, m);
    ce = cudaGetLastError();
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaStreamSynchronize(st);
    wf_free(p->h, tst);
    return wf_cuda_fail(ce, "autotune: set-up");
  }
  lb.st = tst;
  lb.inject_map = -1;
  auto timed = [&](auto&& run) -> float {  // ms of 3 runs after 2 warm-up runs; inf on failure
    for (int i = 0; i < 2; ++i)
      if (run() != cudaSuccess) return INFINITY;
    if (cudaEventRecord(e0, st) != cudaSuccess) return INFINITY;
    for (int i = 0; i < 3; ++i)
      if (run() != cudaSuccess) return INFINITY;
    float ms = INFINITY;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      return INFINITY;
    return ms;
  };
  // column choices (inverse and forward column stage together), then the row
  // choices with the column choice fixed; radix plans only for the ping-pong
  // passes, and only those that differ at this length
  WfGeo best = base;
  float best_ms = INFINITY;
  const int divs[3] = {1, 2, 4};
  for (int ck = WF_COLINV_TMA_K; ck <= WF_COLINV_INPLACE_K; ++ck)
    for (int cp = 0; cp < (ck == WF_COLINV_INPLACE_K ? 1 : WF_NPLAN); ++cp) {
      if (!plan_new(p->g.lgn, cp)) continue;
      if (shared && (ck != base.colinv_kind || cp != base.col_plan)) continue;
      int last_tc = -1;
      for (int di : divs) {
        const WfGeo g = wf_geo_variant(base, ck, base.row_kind, di, 1, cp, 0);
        if (g.TC == last_tc) continue;  // no narrower tile possible
        last_tc = g.TC;
        const float ms = timed([&]() {
          cudaError_t e = wf_launch_lb_colinv<T>(g, b, lb, st);
          if (e == cudaSuccess) e = wf_launch_lb_colfwd<T>(g, b, lb, st);
          return e;
        });
        if (ms < best_ms) { best_ms = ms; best = g; }
      }
    }
  best_ms = INFINITY;
  WfGeo bestr = best;
  for (int rk = WF_ROW_PP_K; rk <= WF_ROW_INPLACE_K; ++rk)
    for (int rp = 0; rp < (rk == WF_ROW_INPLACE_K ? 1 : WF_NPLAN); ++rp) {
      if (!plan_new(p->g.lgh, rp)) continue;
      if (shared && (rk != base.row_kind || rp != base.row_plan)) continue;
      int last_rb = -1;
      for (int di : divs) {
        const WfGeo g = wf_geo_variant(base, best.colinv_kind, rk, best.tc_div, di, best.col_plan, rp);
        if (g.RB == last_rb) continue;
        last_rb = g.RB;
        const float ms = timed([&]() { return wf_launch_lb_row<T>(g, b, lb, st); });
        if (ms < best_ms) { best_ms = ms; bestr = g; }
      }
    }
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  wf_free(p->h, tst);
  cudaGetLastError();
  p->g = bestr;
  std::lock_guard<std::mutex> lock(p->h->mu);
  p->h->tuned[key] = variant_code(bestr);
  return WF_OK;
}

// Scalar-step arguments and the convergence ring of a solve with options o.
static wf_status setup_args(wf_problem* p, WfSolver* S, const wf_opts* o) {
  const int m = o->lbfgs_m;
  WfScalarArgs& A = S->A;
  A.gtol2 = o->gtol_rel * o->gtol_rel;
  A.dchi2 = o->dchi2_abs;
  A.max_iter = o->max_iter;
  A.m = m;
  A.ls = o->line_search;
  A.c1 = o->c1;
  A.c2 = o->c2;
  A.ntile = p->g.ntile;
  A.nrb = p->g.nrb;
  A.ncomb = p->g.ncomb;
  A.maxblk = p->g.maxblk;
  A.phase = WF_PH_ITER;
  A.init = 0;
  A.hcap = 0;
  A.hist = nullptr;
  if (o->history > 0) {  // the convergence ring, kept (and grown) across solves
    if (S->hist_cap < o->history) {
      wf_free(p->h, S->hist);
      S->hist = nullptr;
      S->hist_cap = 0;
      const wf_status rs =
          wf_alloc(p->h, (void**)&S->hist, sizeof(double) * 5 * (size_t)o->history * p->count, "history ring");
      if (rs != WF_OK) return rs;
      S->hist_cap = o->history;
    }
    A.hcap = o->history;
    A.hist = S->hist;
  }
  return WF_OK;
}

// Capture `chunk` iterations in a CUDA graph on st (unless the graph in hand
// was captured with the same settings).  Every kernel's attributes must have
// been set outside capture: one plain iteration has run before.
// Whether the graph in hand was captured with the solve's current settings.
static bool graph_current(const wf_problem* p, const WfSolver* S, cudaStream_t st) {
  const wf_opts* o = &S->o;
  const WfScalarArgs& A = S->A;
  const int chunk = o->check_every > 0 ? o->check_every : 16;
  return S->exec && S->g_chunk == chunk && S->g_maxit == o->max_iter && S->g_gtol2 == A.gtol2 &&
         S->g_dchi2 == A.dchi2 && S->g_m == o->lbfgs_m && S->g_ls == A.ls && S->g_c1 == A.c1 && S->g_c2 == A.c2 &&
         S->g_inject == o->inject_timeout_map && S->g_spin == o->spin_limit && S->g_variant == variant_code(p->g) &&
         S->g_hist == A.hist && S->g_hcap == A.hcap && S->g_stream == st;
}

template <typename T>
static wf_status build_graph(wf_problem* p, WfSolver* S, cudaStream_t st) {
  const wf_opts* o = &S->o;
  const WfScalarArgs& A = S->A;
  const WfBufs b = wf_bufs(p);
  const WfLbBufs lb = lb_bufs<T>(S);
  const int m = o->lbfgs_m;
  const int chunk = o->check_every > 0 ? o->check_every : 16;
  if (graph_current(p, S, st)) return WF_OK;
  if (S->exec) { cudaGraphExecDestroy(S->exec); S->exec = nullptr; }
  cudaGraph_t graph;
  WF_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  cudaError_t ce = cudaSuccess;
  for (int i = 0; i < chunk && ce == cudaSuccess; ++i) ce = iteration<T>(p, b, lb, A, S, st);
  cudaError_t ee = cudaStreamEndCapture(st, &graph);
  if (ce != cudaSuccess) return wf_cuda_fail(ce, "wf_solver: graph capture");
  if (ee != cudaSuccess) return wf_cuda_fail(ee, "wf_solver: end capture");
  ce = cudaGraphInstantiate(&S->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) { S->exec = nullptr; return wf_cuda_fail(ce, "wf_solver: graph instantiate"); }
  S->g_chunk = chunk;
  S->g_maxit = o->max_iter;
  S->g_gtol2 = A.gtol2;
  S->g_dchi2 = A.dchi2;
  S->g_m = m;
  S->g_ls = A.ls;
  S->g_c1 = A.c1;
  S->g_c2 = A.c2;
  S->g_inject = o->inject_timeout_map;
  S->g_variant = variant_code(p->g);
  S->g_spin = o->spin_limit;
  S->g_hist = A.hist;
  S->g_hcap = A.hcap;
  S->g_stream = st;
  return WF_OK;
}

// Start of an inner round of the refined solve: the correction starts at 0
// with the FP64 gradient g64 of the outer state (see k_refine_seed).
struct WfSeed {
  const double* g64;
  const double* res;
  double tol;
};

// Set up the state at s0 (or 0): true gradient, chi^2, first direction.  With
// a seed, the state is the correction delta = 0 of a refined solve's round and
// its gradient and chi^2 come from the seed instead of an evaluation.
template <typename T>
static wf_status start_impl(wf_problem* p, const wf_opts* o, const void* s0, const WfSeed* seed = nullptr) {
  const int m = o->lbfgs_m;
  wf_status rs = ensure_solver(p, m);
  if (rs != WF_OK) return rs;
  WfSolver* S = p->solver;
  S->o = *o;
  S->iters = 0;
  cudaStream_t us = (cudaStream_t)o->stream;
  cudaStream_t st = wf_capturable(us) ? us : S->stream;
  if (S->exec && S->g_stream != st) { cudaGraphExecDestroy(S->exec); S->exec = nullptr; }
  S->work = st;
  WfBufs b = wf_bufs(p);
  WfLbBufs lb = lb_bufs<T>(S);
  rs = setup_args(p, S, o);
  if (rs != WF_OK) return rs;
  WfScalarArgs& A = S->A;
  WF_TRY(cudaEventRecord(S->ev_in, us));
  WF_TRY(cudaStreamWaitEvent(st, S->ev_in, 0));
  if (s0 && !seed) WF_TRY(wf_launch_pack<T>(p->g, p->count, s0, S->s, st));
  else WF_TRY(cudaMemsetAsync(S->s, 0, (size_t)p->count * p->C * p->n * p->nx * p->elt, st));
  WF_TRY(cudaMemsetAsync(S->st, 0, sizeof(WfLbMap) * p->count, st));
  rs = choose_variant<T>(p, S, st);  // before the first refresh: one variant for the whole solve
  if (rs != WF_OK) return rs;
  A.ntile = p->g.ntile;
  A.nrb = p->g.nrb;
  if (seed) {
    const size_t per = (size_t)p->C * p->n * p->nx;  // reals per packed map vector
    k_refine_seed<T><<<dim3(wf_grid(per), p->count), 256, 0, st>>>(seed->g64, seed->res, seed->tol, per,
                                                                     (T*)S->g, p->part, A.ntile, A.nrb, A.maxblk);
    WF_TRY(cudaGetLastError());
    WF_TRY(wf_launch_lb_comb<T>(p->g, b, lb, WF_LB1_DOTS, st));  // <g, g> (no stored pairs yet)
    WF_TRY(cudaMemsetAsync(S->nact, 0, sizeof(int), st));
    WfScalarArgs Ai = A;
    Ai.phase = WF_PH_REFRESH;
    Ai.init = 1;
    k_lb_scalar<<<(p->count + WF_SW - 1) / WF_SW, 32 * WF_SW, 0, st>>>(lb.st, b.part, Ai, p->count, S->nact);
    WF_TRY(cudaGetLastError());
  } else {
    WF_TRY(refresh<T>(p, b, lb, A, 1, S, st));
  }
  if (o->use_graphs && !graph_current(p, S, st)) {
    // Set every kernel's attributes outside capture: one iteration (a genuine
    // iteration of the solve), then the graph.
    WF_TRY(iteration<T>(p, b, lb, A, S, st));
    S->iters += 1;
    rs = build_graph<T>(p, S, st);
    if (rs != WF_OK) return rs;
  }
  S->graph_pending = 0;
  S->started = 1;
  return WF_OK;
}

// Run n iterations (graph chunks plus plain launches for the remainder);
// optionally read the number of maps still active (one synchronisation).
template <typename T>
static wf_status step_impl(wf_problem* p, int n_iter, int* n_active) {
  WfSolver* S = p->solver;
  const wf_opts* o = &S->o;
  cudaStream_t st = S->work;
  WfBufs b = wf_bufs(p);
  WfLbBufs lb = lb_bufs<T>(S);
  // iterations per graph launch: the graph's own count (a resumed solve
  // captures its graph below, so this is read again after the capture)
  int chunk = S->g_chunk > 0 ? S->g_chunk : (o->check_every > 0 ? o->check_every : 16);
  int done = 0;
  while (done < n_iter) {
    if (o->refresh_every > 0 && S->iters > 0 && S->iters % o->refresh_every == 0)
      WF_TRY(refresh<T>(p, b, lb, S->A, 0, S, st));
    int left = n_iter - done;
    if (o->refresh_every > 0) {
      const int to_refresh = o->refresh_every - (int)(S->iters % o->refresh_every);
      if (to_refresh < left) left = to_refresh;
    }
    if (o->use_graphs && S->graph_pending && left > chunk) {  // a resumed solve: one plain iteration, then capture
      WF_TRY(iteration<T>(p, b, lb, S->A, S, st));
      done += 1;
      S->iters += 1;
      const wf_status rs = build_graph<T>(p, S, st);
      if (rs != WF_OK) return rs;
      S->graph_pending = 0;
      chunk = S->g_chunk;
      continue;
    }
    if (o->use_graphs && S->exec && !S->graph_pending && left >= chunk) {
      WF_TRY(cudaGraphLaunch(S->exec, st));
      done += chunk;
      S->iters += chunk;
    } else {
      WF_TRY(iteration<T>(p, b, lb, S->A, S, st));
      done += 1;
      S->iters += 1;
    }
  }
  if (n_active) {
    WF_TRY(cudaMemcpyAsync(S->nact_host, S->nact, sizeof(int), cudaMemcpyDeviceToHost, st));
    WF_TRY(cudaStreamSynchronize(st));
    *n_active = *S->nact_host;
  }
  return WF_OK;
}

// Apply the last step, evaluate the true chi^2 and gradient, write outputs.
template <typename T>
static wf_status finish_impl(wf_problem* p, void* s_out, void* x_out, wf_solve_stats* stats) {
  WfSolver* S = p->solver;
  cudaStream_t us = (cudaStream_t)S->o.stream, st = S->work;
  WfBufs b = wf_bufs(p);
  WfLbBufs lb = lb_bufs<T>(S);
  WF_TRY(wf_launch_lb_comb<T>(p->g, b, lb, WF_LB1_MATERIALIZE, st));
  WF_TRY(wf_launch_eval_pk<T>(p->g, b, lb.s, lb.g, st));
  k_lb_final<<<(p->count + WF_SW - 1) / WF_SW, 32 * WF_SW, 0, st>>>(lb.st, b.part, p->g.ntile, p->g.nrb,
                                                                    p->g.maxblk, p->count, S->stats_dev);
  WF_TRY(cudaGetLastError());
  if (s_out) WF_TRY(wf_launch_unpack<T>(p->g, p->count, S->s, s_out, st));
  if (x_out) WF_TRY(wf_launch_signal<T>(p->g, b, WF_IN_PK, S->s, x_out, st));
  WF_TRY(cudaMemcpyAsync(S->stats_host, S->stats_dev, sizeof(double) * 5 * p->count, cudaMemcpyDeviceToHost, st));
  WF_TRY(cudaEventRecord(S->ev_out, st));
  WF_TRY(cudaStreamWaitEvent(us, S->ev_out, 0));
  WF_TRY(cudaStreamSynchronize(st));
  S->started = 0;
  int worst = WF_OK;
  auto rank = [](int s) {
    return s == WF_ETIMEOUT ? 4 : s == WF_ENONFINITE ? 3 : s == WF_ELINESEARCH ? 2 : s == WF_ENOTCONVERGED ? 1 : 0;
  };
  for (int i = 0; i < p->count; ++i) {
    const double* r = S->stats_host + 5 * i;
    const int status = (int)r[2];
    if (stats) {
      stats[i].iters = (int)r[0];
      stats[i].evals = (int)r[1];
      stats[i].status = status;
      stats[i].fft_variant = variant_code(p->g);
      stats[i].chi2 = r[3];
      stats[i].gnorm_rel = r[4];
    }
    if (rank(status) > rank(worst)) worst = status;
  }
  if (worst != WF_OK) {
    if (worst == WF_ENOTCONVERGED) wf_fail((wf_status)worst, "wf_map_solve: iteration limit reached");
    else wf_fail((wf_status)worst, "wf_map_solve: a map stopped with status %d", worst);
  }
  return (wf_status)worst;
}

// MAP solve with FP64 iterative refinement and an error certificate (Sec. 2.2
// for the objective; the certificate follows from the whitened half-Hessian
// I + A^T W A having every eigenvalue >= 1, so |s - s*| <= |grad chi2(s)| / 2).
// Rounds: evaluate the true gradient g at the FP64 state s in FP64; stop the
// maps with |g| <= 2 tol |s|; otherwise minimise the quadratic model of
// chi^2(s + delta) from delta = 0 with the device L-BFGS in the problem's
// working precision (its gradient starts at g; Hessian-vector passes only),
// then s += delta in FP64.  The correction is small, so the working type's
// rounding stays relative to it, not to s: the state converges to the FP64
// answer although every operator pass of the inner solves runs in FP32.
template <typename T>
static wf_status refined_impl(wf_problem* p, const wf_opts* o, double tol, int max_rounds, const void* s0,
                              void* s_out, double* cert, wf_solve_stats* stats) {
  wf_status rs = ensure_solver(p, o->lbfgs_m);
  if (rs != WF_OK) return rs;
  WfSolver* S = p->solver;
  const int B = p->count;
  const size_t per = (size_t)p->C * p->n * p->nx;  // reals per packed map vector, pixels per map
  const size_t nsp = (size_t)p->C * p->n * (p->nx / 2 + 1) * (p->sp_shared ? 1 : B);
  const bool mixed = p->precision == WF_MIXED;
  auto need = [&](void** q, size_t bytes, const char* what) {
    if (rs == WF_OK && !*q) rs = wf_alloc(p->h, q, bytes, what);
  };
  need(&S->r_s64, sizeof(double) * per * B, "refined state");
  need(&S->r_g64, sizeof(double) * per * B, "refined gradient");
  need((void**)&S->r_res, sizeof(double) * WF_RES * B, "refined records");
  if (mixed) {
    need(&S->r_d64, sizeof(double) * per * B, "FP64 data maps");
    need(&S->r_w64, sizeof(double) * per * B, "FP64 weights");
    need(&S->r_sp64, sizeof(double) * nsp, "FP64 sqrt(P) tables");
    need(&S->r_scr64, sizeof(double) * per * B, "FP64 scratch");
  }
  if (rs != WF_OK) return rs;
  if (!S->r_res_host) {
    cudaError_t e = cudaMallocHost((void**)&S->r_res_host, sizeof(double) * WF_RES * B);
    if (e != cudaSuccess) { S->r_res_host = nullptr; return wf_cuda_fail(e, "wf_map_solve_refined: host records"); }
  }
  cudaStream_t us = (cudaStream_t)o->stream;
  cudaStream_t st = wf_capturable(us) ? us : S->stream;
  WF_TRY(cudaEventRecord(S->ev_in, us));
  WF_TRY(cudaStreamWaitEvent(st, S->ev_in, 0));
  // The FP64 operator of the outer evaluations: for a MIXED problem on exact
  // FP64 copies of the working-precision inputs (the problem the inner solves
  // see), always on the default tiles.
  const WfGeo go = wf_make_geo(p->n, p->nx, p->C, p->count);
  WfBufs bo = wf_bufs(p);
  if (mixed) {
    k_convert<float, double><<<wf_grid(per * B), 256, 0, st>>>((const float*)p->d, (double*)S->r_d64, per * B);
    k_convert<float, double><<<wf_grid(per * B), 256, 0, st>>>((const float*)p->w, (double*)S->r_w64, per * B);
    k_convert<float, double><<<wf_grid(nsp), 256, 0, st>>>((const float*)p->sp, (double*)S->r_sp64, nsp);
    WF_TRY(cudaGetLastError());
    bo.d = S->r_d64;
    bo.w = S->r_w64;
    bo.sp = S->r_sp64;
    bo.scratch = S->r_scr64;
    bo.tw = p->h->tw64;
  }
  double* s64 = (double*)S->r_s64;
  double* res = S->r_res;
  if (s0) {
    WF_TRY(wf_launch_pack<T>(p->g, B, s0, S->s, st));
    k_convert<T, double><<<wf_grid(per * B), 256, 0, st>>>((const T*)S->s, s64, per * B);
    WF_TRY(cudaGetLastError());
  } else {
    WF_TRY(cudaMemsetAsync(s64, 0, sizeof(double) * per * B, st));
  }
  WF_TRY(cudaMemsetAsync(res, 0, sizeof(double) * WF_RES * B, st));
  double* rh = S->r_res_host;
  for (int round = 0;; ++round) {
    WF_TRY(wf_launch_eval_pk<double>(go, bo, s64, S->r_g64, st));
    k_refine_round<<<B, 32, 0, st>>>(p->part, go.ntile, go.nrb, go.maxblk, B, round == 0, res);
    WF_TRY(cudaGetLastError());
    WF_TRY(cudaMemcpyAsync(rh, res, sizeof(double) * WF_RES * B, cudaMemcpyDeviceToHost, st));
    WF_TRY(cudaStreamSynchronize(st));
    int left = 0;
    double ratio = 0.5;  // the largest reduction a round is asked for: at least 2x
    for (int b = 0; b < B; ++b) {
      const double* r = rh + (size_t)b * WF_RES;
      if (r[WF_RES_STATUS] != 0.0 || !(r[WF_RES_CERT] > tol)) continue;
      ++left;
      if (r[WF_RES_SS] > 0.0 && r[WF_RES_GG] > 0.0) {
        const double need_b = 0.5 * 2.0 * tol * sqrt(r[WF_RES_SS] / r[WF_RES_GG]);  // half the reduction needed
        if (need_b < ratio) ratio = need_b;
      }
    }
    if (left == 0 || round >= max_rounds) break;
    // Inner round: the first from the caller's tolerance, later ones only as
    // far as the least advanced map needs (with a factor 2 to spare).
    wf_opts oi = *o;
    oi.refresh_every = 0;  // the outer FP64 evaluations are this solve's refreshes
    if (round > 0 && ratio > oi.gtol_rel) oi.gtol_rel = ratio;
    const WfSeed sd{(const double*)S->r_g64, res, tol};
    rs = start_impl<T>(p, &oi, nullptr, &sd);
    if (rs != WF_OK) return rs;
    const int chunk = oi.check_every > 0 ? oi.check_every : 16;
    const long long max_chunks = (long long)oi.max_iter / chunk + 2;
    for (long long c = 0; c < max_chunks; ++c) {
      int nact = 0;
      rs = step_impl<T>(p, chunk, &nact);
      if (rs != WF_OK) return rs;
      if (nact == 0) break;
    }
    const WfBufs bw = wf_bufs(p);
    WF_TRY(wf_launch_lb_comb<T>(p->g, bw, lb_bufs<T>(S), WF_LB1_MATERIALIZE, st));  // delta into S->s
    k_refine_tally<<<(B + 127) / 128, 128, 0, st>>>(S->st, B, res);
    k_refine_accum<T><<<wf_grid(per * B), 256, 0, st>>>((const T*)S->s, s64, per * B);
    WF_TRY(cudaGetLastError());
    S->started = 0;
  }
  WF_TRY(wf_launch_unpack<double>(go, B, s64, s_out, st));
  WF_TRY(cudaEventRecord(S->ev_out, st));
  WF_TRY(cudaStreamWaitEvent(us, S->ev_out, 0));
  WF_TRY(cudaStreamSynchronize(st));
  int worst = WF_OK;
  auto rank = [](int s) {
    return s == WF_ETIMEOUT ? 4 : s == WF_ENONFINITE ? 3 : s == WF_ELINESEARCH ? 2 : s == WF_ENOTCONVERGED ? 1 : 0;
  };
  for (int b = 0; b < B; ++b) {
    const double* r = rh + (size_t)b * WF_RES;
    int status = (int)r[WF_RES_STATUS];
    if (status == WF_OK && !(r[WF_RES_CERT] <= tol))
      status = isfinite(r[WF_RES_CERT]) ? WF_ENOTCONVERGED : WF_ENONFINITE;
    if (cert) cert[b] = r[WF_RES_CERT];
    if (stats) {
      stats[b].iters = (int)r[WF_RES_ITERS];
      stats[b].evals = (int)r[WF_RES_EVALS];
      stats[b].status = status;
      stats[b].fft_variant = variant_code(p->g);
      stats[b].chi2 = r[WF_RES_CHI2];
      stats[b].gnorm_rel = r[WF_RES_GG0] > 0.0 ? sqrt(r[WF_RES_GG] / r[WF_RES_GG0]) : 0.0;
    }
    if (rank(status) > rank(worst)) worst = status;
  }
  if (worst != WF_OK)
    wf_fail((wf_status)worst, worst == WF_ENOTCONVERGED ? "wf_map_solve_refined: certificate not reached"
                                                        : "wf_map_solve_refined: a map stopped with an error");
  return (wf_status)worst;
}

// Run n iterations with plain launches and CUDA events around each kernel on
// the working stream; ms[0..5] = average duration of k_lb_comb, k_lb_colinv,
// the row stage, k_lb_colfwd, k_lb_qdots and the scalar step.
template <typename T>
static wf_status profile_impl(wf_problem* p, int n_iter, float* ms) {
  WfSolver* S = p->solver;
  cudaStream_t st = S->work;
  WfBufs b = wf_bufs(p);
  WfLbBufs lb = lb_bufs<T>(S);
  cudaEvent_t ev[7];
  for (int i = 0; i < 7; ++i) WF_TRY(cudaEventCreate(&ev[i]));
  double acc[6] = {0, 0, 0, 0, 0, 0};
  wf_status rs = WF_OK;
  for (int it = 0; it < n_iter && rs == WF_OK; ++it) {
    cudaError_t e = cudaEventRecord(ev[0], st);
    if (e == cudaSuccess) e = wf_launch_lb_comb<T>(p->g, b, lb, WF_LB1_FULL, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
    if (e == cudaSuccess) e = wf_launch_lb_colinv<T>(p->g, b, lb, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], st);
    if (e == cudaSuccess) e = wf_launch_lb_row<T>(p->g, b, lb, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], st);
    if (e == cudaSuccess) e = wf_launch_lb_colfwd<T>(p->g, b, lb, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[4], st);
    if (e == cudaSuccess) e = wf_launch_lb_qdots<T>(p->g, b, lb, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[5], st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->nact, 0, sizeof(int), st);
    if (e == cudaSuccess) {
      k_lb_scalar<<<(p->count + WF_SW - 1) / WF_SW, 32 * WF_SW, 0, st>>>(lb.st, b.part, S->A, p->count, S->nact);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[6], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[6]);
    for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      acc[k] += t;
    }
    if (e != cudaSuccess) rs = wf_cuda_fail(e, "wf_solver_profile");
    S->iters += 1;
  }
  for (int i = 0; i < 7; ++i) cudaEventDestroy(ev[i]);
  for (int k = 0; k < 6; ++k) ms[k] = n_iter > 0 ? (float)(acc[k] / n_iter) : 0.f;
  return rs;
}

static wf_status check_opts(const wf_problem* p, const wf_opts* o) {
  if (o->lbfgs_m < 1 || o->lbfgs_m > WF_MAXM)
    return wf_fail(WF_EINVAL, "lbfgs_m = %d outside [1, %d]", o->lbfgs_m, WF_MAXM);
  if (o->max_iter < 1) return wf_fail(WF_EINVAL, "max_iter must be >= 1");
  if (!(o->gtol_rel >= 0.0) || !(o->dchi2_abs >= 0.0)) return wf_fail(WF_EINVAL, "tolerances must be >= 0");
  if (o->check_every < 0 || o->check_every > 4096) return wf_fail(WF_EINVAL, "bad check_every");
  if (o->refresh_every < 0) return wf_fail(WF_EINVAL, "bad refresh_every");
  if (o->spin_limit < 0) return wf_fail(WF_EINVAL, "spin_limit must be >= 0");
  if (o->history < 0 || o->history > (1 << 20)) return wf_fail(WF_EINVAL, "history = %d outside [0, 2^20]", o->history);
  if (o->fft_variant != 0 && !variant_valid(o->fft_variant))
    return wf_fail(WF_EINVAL, "fft_variant = %d is not a valid variant code", o->fft_variant);
  if (o->inject_timeout_map > 0 && o->fft_variant != 0 && (o->fft_variant / 1000) % 10 != WF_COLINV_TMA_K)
    return wf_fail(WF_EINVAL, "inject_timeout_map needs the TMA-fed inverse column stage (fft_variant %d)",
                   o->fft_variant);
  if (o->inject_timeout_map < 0 || o->inject_timeout_map > p->count)
    return wf_fail(WF_EINVAL, "inject_timeout_map = %d outside [0, %d]", o->inject_timeout_map, p->count);
  if (o->inject_timeout_map > 0 && wf_make_geo(p->n, p->nx, p->C).colinv_kind != WF_COLINV_TMA_K)
    return wf_fail(WF_EINVAL, "inject_timeout_map: %d x %d maps have no TMA-fed inverse column stage", p->n,
                   p->nx);
  if (o->line_search != WF_LS_EXACT && o->line_search != WF_LS_WOLFE)
    return wf_fail(WF_EINVAL, "line_search = %d is not WF_LS_EXACT or WF_LS_WOLFE", o->line_search);
  if (o->line_search == WF_LS_WOLFE && !(0.0 < o->c1 && o->c1 < o->c2 && o->c2 < 1.0))
    return wf_fail(WF_EINVAL, "Wolfe constants need 0 < c1 < c2 < 1 (c1 = %g, c2 = %g)", o->c1, o->c2);
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != p->h->device) return wf_fail(WF_EINVAL, "current device differs from the problem's");
  return WF_OK;
}

extern "C" wf_status wf_solver_start(wf_problem* p, const wf_opts* opts, const void* s0) {
  if (!p) return wf_fail(WF_EINVAL, "wf_solver_start: null problem");
  wf_opts o;
  if (opts) o = *opts;
  else wf_opts_default(&o);
  wf_status s = check_opts(p, &o);
  if (s != WF_OK) return s;
  return p->precision == WF_FP64 ? start_impl<double>(p, &o, s0) : start_impl<float>(p, &o, s0);
}

extern "C" wf_status wf_solver_step(wf_problem* p, int n_iter, int* n_active) {
  if (!p || !p->solver || !p->solver->started) return wf_fail(WF_EINVAL, "wf_solver_step: no solve started");
  if (n_iter < 0) return wf_fail(WF_EINVAL, "wf_solver_step: n_iter < 0");
  return p->precision == WF_FP64 ? step_impl<double>(p, n_iter, n_active) : step_impl<float>(p, n_iter, n_active);
}

extern "C" wf_status wf_solver_profile(wf_problem* p, int n_iter, float* ms) {
  if (!p || !p->solver || !p->solver->started || !ms)
    return wf_fail(WF_EINVAL, "wf_solver_profile: no solve started or null output");
  if (n_iter < 1) return wf_fail(WF_EINVAL, "wf_solver_profile: n_iter < 1");
  return p->precision == WF_FP64 ? profile_impl<double>(p, n_iter, ms) : profile_impl<float>(p, n_iter, ms);
}

extern "C" wf_status wf_solver_finish(wf_problem* p, void* s_out, void* x_out, wf_solve_stats* stats) {
  if (!p || !p->solver || !p->solver->started) return wf_fail(WF_EINVAL, "wf_solver_finish: no solve started");
  return p->precision == WF_FP64 ? finish_impl<double>(p, s_out, x_out, stats)
                                 : finish_impl<float>(p, s_out, x_out, stats);
}

extern "C" wf_status wf_map_solve(wf_problem* p, const wf_opts* opts, const void* s0, void* s_out,
                                  void* x_out, wf_solve_stats* stats) {
  if (!p || !s_out) return wf_fail(WF_EINVAL, "wf_map_solve: null problem or output");
  wf_opts o;
  if (opts) o = *opts;
  else wf_opts_default(&o);
  wf_status s = wf_solver_start(p, &o, s0);
  if (s != WF_OK) return s;
  const int chunk = o.check_every > 0 ? o.check_every : 16;
  const long long max_chunks = (long long)o.max_iter / chunk + 2;
  for (long long c = 0; c < max_chunks; ++c) {
    int nact = 0;
    s = wf_solver_step(p, chunk, &nact);
    if (s != WF_OK) return s;
    if (nact == 0) break;
  }
  return wf_solver_finish(p, s_out, x_out, stats);
}

extern "C" wf_status wf_map_solve_refined(wf_problem* p, const wf_opts* opts, double cert_tol, int max_rounds,
                                          const void* s0, void* s_out, double* cert, wf_solve_stats* stats) {
  if (!p || !s_out) return wf_fail(WF_EINVAL, "wf_map_solve_refined: null problem or output");
  if (!(cert_tol > 0.0) || !isfinite(cert_tol))
    return wf_fail(WF_EINVAL, "wf_map_solve_refined: cert_tol must be finite and > 0");
  if (max_rounds < 1 || max_rounds > 1000)
    return wf_fail(WF_EINVAL, "wf_map_solve_refined: max_rounds = %d outside [1, 1000]", max_rounds);
  wf_opts o;
  if (opts) o = *opts;
  else wf_opts_default(&o);
  wf_status s = check_opts(p, &o);
  if (s != WF_OK) return s;
  if (o.inject_timeout_map > 0) return wf_fail(WF_EINVAL, "wf_map_solve_refined: no timeout injection");
  return p->precision == WF_FP64 ? refined_impl<double>(p, &o, cert_tol, max_rounds, s0, s_out, cert, stats)
                                 : refined_impl<float>(p, &o, cert_tol, max_rounds, s0, s_out, cert, stats);
}

// Helpers of the batched multi-problem solve: one iteration or one refresh of
// a started problem, in its working precision.
template <typename T>
static cudaError_t iteration_of(wf_problem* p, cudaStream_t st) {
  WfSolver* S = p->solver;
  return iteration<T>(p, wf_bufs(p), lb_bufs<T>(S), S->A, S, st);
}
static cudaError_t any_iteration(wf_problem* p, cudaStream_t st) {
  return p->precision == WF_FP64 ? iteration_of<double>(p, st) : iteration_of<float>(p, st);
}
static cudaError_t any_refresh(wf_problem* p, cudaStream_t st) {
  WfSolver* S = p->solver;
  return p->precision == WF_FP64 ? refresh<double>(p, wf_bufs(p), lb_bufs<double>(S), S->A, 0, S, st)
                                 : refresh<float>(p, wf_bufs(p), lb_bufs<float>(S), S->A, 0, S, st);
}

// One L-BFGS iteration of several problems in shared launches (see
// WfMultiArgs): the five kernels of iteration() plus the active counters'
// reset and the scalar step, seven launches whatever the number of problems.
static_assert(WF_SW == 1, "the shared scalar launch takes one block per map");
template <typename T>
static cudaError_t multi_iteration(const WfMultiArgs& a, const WfMultiScalar& ms, cudaStream_t st) {
  cudaError_t e = wf_launch_multi_comb<T>(a, WF_LB1_FULL, st);
  if (e == cudaSuccess) e = wf_launch_multi_colinv<T>(a, st);
  if (e == cudaSuccess) e = wf_launch_multi_row<T>(a, st);
  if (e == cudaSuccess) e = wf_launch_multi_colfwd<T>(a, st);
  if (e == cudaSuccess) e = wf_launch_multi_qdots<T>(a, st);
  if (e == cudaSuccess) {
    k_multi_zero<<<1, 32, 0, st>>>(ms);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_multi_scalar<<<ms.start[ms.np], 32 * WF_SW, 0, st>>>(ms);
    e = cudaGetLastError();
  }
  return e;
}

// Several problems (typically one per map shape of a heterogeneous batch)
// solved as one batch.  Every problem is started on its own stream (first
// gradient).  When the problems share the working type and C (and no FFT-stage
// variant is forced), each iteration of the whole batch is seven shared
// launches (multi_iteration), every problem on the ping-pong stages of
// WF_MULTI_VARIANT with its own tuned tile widths; otherwise each problem is
// tuned freely and runs its own kernels, as a parallel branch per problem.  check_every iterations are
// captured in one CUDA graph, so that each round is one graph launch for the
// whole batch; the maps of every shape advance together and a problem whose
// maps have all stopped costs only its blocks' early exits.  The host reads
// the active counts once per round.
extern "C" wf_status wf_map_solve_many(wf_problem* const* ps, int np, const wf_opts* opts, void* const* s_out,
                                       wf_solve_stats* const* stats) {
  if (!ps || np < 1 || !s_out) return wf_fail(WF_EINVAL, "wf_map_solve_many: null or empty arguments");
  for (int i = 0; i < np; ++i)
    if (!ps[i] || !s_out[i]) return wf_fail(WF_EINVAL, "wf_map_solve_many: problem %d or its output is null", i);
  for (int i = 0; i < np; ++i)
    for (int k = 0; k < i; ++k)
      if (ps[i] == ps[k]) return wf_fail(WF_EINVAL, "wf_map_solve_many: problem %d is listed twice", i);
  wf_opts o;
  if (opts) o = *opts;
  else wf_opts_default(&o);
  const int chunk = o.check_every > 0 ? o.check_every : 16;
  cudaStream_t us = (cudaStream_t)o.stream;
  std::vector<cudaEvent_t> ev((size_t)np + 1, nullptr);
  cudaStream_t bs = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    if (bs) cudaStreamDestroy(bs);
  };
  cudaError_t e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
  for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev[np], us);
  if (e != cudaSuccess) { cleanup(); return wf_cuda_fail(e, "wf_map_solve_many: set-up"); }
  wf_opts oi = o;
  oi.stream = nullptr;  // every problem starts on its own internal stream
  oi.use_graphs = 0;    // the batch graph replaces the per-problem ones
  oi.inject_timeout_map = 0;
  bool shared = np >= 2 && np <= WF_MULTI_MAX && o.fft_variant == 0;
  for (int i = 1; i < np && shared; ++i) shared = ps[i]->precision == ps[0]->precision && ps[i]->C == ps[0]->C;
  const bool f64 = ps[0]->precision == WF_FP64;
  WfMultiArgs ma;
  WfMultiScalar ms;
  memset(&ma, 0, sizeof ma);
  memset(&ms, 0, sizeof ms);
  wf_status rs = WF_OK;
  for (int i = 0; i < np && rs == WF_OK; ++i) {
    rs = check_opts(ps[i], &oi);
    if (rs == WF_OK) rs = ensure_solver(ps[i], oi.lbfgs_m);
    if (rs != WF_OK) break;
    e = cudaStreamWaitEvent(ps[i]->solver->stream, ev[np], 0);
    if (e != cudaSuccess) { rs = wf_cuda_fail(e, "wf_map_solve_many: ordering"); break; }
    ps[i]->solver->shared_tune = shared ? 1 : 0;
    rs = ps[i]->precision == WF_FP64 ? start_impl<double>(ps[i], &oi, nullptr) : start_impl<float>(ps[i], &oi, nullptr);
    ps[i]->solver->shared_tune = 0;
  }
  if (shared && rs == WF_OK) {
    ma.np = ms.np = np;
    ms.start[0] = 0;
    for (int i = 0; i < np; ++i) {
      WfSolver* S = ps[i]->solver;
      ma.g[i] = ps[i]->g;
      ma.b[i] = wf_bufs(ps[i]);
      ma.lb[i] = lb_bufs<float>(S);
      ms.st[i] = S->st;
      ms.part[i] = ps[i]->part;
      ms.nact[i] = S->nact;
      ms.A[i] = S->A;
      ms.start[i + 1] = ms.start[i] + ps[i]->count;
    }
  }
  auto batch_iteration = [&](cudaStream_t s) -> cudaError_t {
    return f64 ? multi_iteration<double>(ma, ms, s) : multi_iteration<float>(ma, ms, s);
  };
  // one plain iteration of every problem (every kernel's attributes set outside
  // capture), then the batch stream waits for all of them
  for (int i = 0; i < np && rs == WF_OK; ++i) {
    WfSolver* S = ps[i]->solver;
    e = shared ? cudaSuccess : any_iteration(ps[i], S->work);
    if (e == cudaSuccess) e = cudaEventRecord(ev[i], S->work);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(bs, ev[i], 0);
    if (e != cudaSuccess) rs = wf_cuda_fail(e, "wf_map_solve_many: first iteration");
    S->iters += 1;
  }
  if (shared && rs == WF_OK) {
    e = batch_iteration(bs);
    if (e != cudaSuccess) rs = wf_cuda_fail(e, "wf_map_solve_many: first iteration");
  }
  if (rs == WF_OK && o.use_graphs) {
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(bs, cudaStreamCaptureModeRelaxed);
    if (shared) {
      for (int k = 0; k < chunk && e == cudaSuccess; ++k) e = batch_iteration(bs);
    } else {
      if (e == cudaSuccess) e = cudaEventRecord(ev[np], bs);
      for (int i = 0; i < np && e == cudaSuccess; ++i) {  // a branch per problem, forked from and joined to bs
        cudaStream_t si = ps[i]->solver->work;
        e = cudaStreamWaitEvent(si, ev[np], 0);
        for (int k = 0; k < chunk && e == cudaSuccess; ++k) e = any_iteration(ps[i], si);
        if (e == cudaSuccess) e = cudaEventRecord(ev[i], si);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(bs, ev[i], 0);
      }
    }
    const cudaError_t ee = cudaStreamEndCapture(bs, &graph);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      exec = nullptr;
      rs = wf_cuda_fail(e, "wf_map_solve_many: batch graph");
    }
  }
  std::vector<int> live((size_t)np, 1);
  std::vector<long long> last_refresh((size_t)np, 0);
  const long long max_rounds = (long long)o.max_iter / chunk + 2;
  for (long long r = 0; r < max_rounds && rs == WF_OK; ++r) {
    for (int i = 0; i < np && rs == WF_OK; ++i) {  // refreshes that are due, on the batch stream
      WfSolver* S = ps[i]->solver;
      if (o.refresh_every > 0 && live[i] && S->iters / o.refresh_every > last_refresh[i]) {
        last_refresh[i] = S->iters / o.refresh_every;
        e = any_refresh(ps[i], bs);
        if (e != cudaSuccess) rs = wf_cuda_fail(e, "wf_map_solve_many: refresh");
      }
    }
    if (rs != WF_OK) break;
    if (exec) {
      e = cudaGraphLaunch(exec, bs);
    } else if (shared) {
      for (int k = 0; k < chunk && e == cudaSuccess; ++k) e = batch_iteration(bs);
    } else {
      for (int i = 0; i < np && e == cudaSuccess; ++i)
        for (int k = 0; k < chunk && e == cudaSuccess; ++k) e = any_iteration(ps[i], bs);
    }
    for (int i = 0; i < np && e == cudaSuccess; ++i) {
      ps[i]->solver->iters += chunk;
      e = cudaMemcpyAsync(ps[i]->solver->nact_host, ps[i]->solver->nact, sizeof(int), cudaMemcpyDeviceToHost, bs);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(bs);
    if (e != cudaSuccess) { rs = wf_cuda_fail(e, "wf_map_solve_many: iterations"); break; }
    int any = 0;
    for (int i = 0; i < np; ++i) {
      live[i] = *ps[i]->solver->nact_host > 0;
      any |= live[i];
    }
    if (!any) break;
  }
  if (rs == WF_OK) {  // the problems' own streams continue after the batch stream
    e = cudaEventRecord(ev[np], bs);
    for (int i = 0; i < np && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(ps[i]->solver->work, ev[np], 0);
    if (e != cudaSuccess) rs = wf_cuda_fail(e, "wf_map_solve_many: ordering");
  }
  wf_status worst = rs;
  for (int i = 0; i < np && rs == WF_OK; ++i) {
    const wf_status si = wf_solver_finish(ps[i], s_out[i], nullptr, stats ? stats[i] : nullptr);
    if (si != WF_OK && (worst == WF_OK || worst == WF_ENOTCONVERGED)) worst = si;
  }
  cudaStreamSynchronize(bs);
  cleanup();
  if (us) cudaStreamSynchronize(us);
  return worst;
}

// Checkpoint of a started solve: header, the per-map scalar state, then the
// state s, the gradient g and the 2m stored vectors of the ring (packed, the
// working type), each starting on a 256-byte boundary.
struct WfStateHeader {
  char magic[8];
  int n, nx, C, precision, count, lbfgs_m, variant;
  long long iters;
  size_t vbytes;  // bytes of one packed vector set (all maps)
  wf_opts o;      // the solve's options (stream not kept)
};
static const char kWfStateMagic[8] = {'W', 'F', 'S', 'T', 'A', 'T', 'E', '2'};
static size_t up256s(size_t x) { return (x + 255) & ~(size_t)255; }
static size_t state_bytes(const wf_problem* p, int m, size_t* off_st, size_t* off_vec) {
  const size_t vbytes = (size_t)p->count * p->C * p->n * p->nx * p->elt;
  *off_st = up256s(sizeof(WfStateHeader));
  *off_vec = *off_st + up256s(sizeof(WfLbMap) * p->count);
  return *off_vec + (2 + 2 * (size_t)m) * up256s(vbytes);
}

extern "C" wf_status wf_solver_state_size(const wf_problem* p, size_t* bytes) {
  if (!p || !bytes) return wf_fail(WF_EINVAL, "wf_solver_state_size: null argument");
  if (!p->solver || !p->solver->started) return wf_fail(WF_EINVAL, "wf_solver_state_size: no solve started");
  size_t a, b;
  *bytes = state_bytes(p, p->solver->o.lbfgs_m, &a, &b);
  return WF_OK;
}

extern "C" wf_status wf_solver_export(wf_problem* p, void* dst, size_t bytes) {
  if (!p || !dst) return wf_fail(WF_EINVAL, "wf_solver_export: null argument");
  WfSolver* S = p->solver;
  if (!S || !S->started) return wf_fail(WF_EINVAL, "wf_solver_export: no solve started");
  const int m = S->o.lbfgs_m;
  size_t off_st, off_vec;
  const size_t need = state_bytes(p, m, &off_st, &off_vec);
  if (bytes < need) return wf_fail(WF_EINVAL, "wf_solver_export: %zu bytes given, %zu needed", bytes, need);
  WfStateHeader hd;
  memset(&hd, 0, sizeof hd);
  memcpy(hd.magic, kWfStateMagic, 8);
  hd.n = p->n;
  hd.nx = p->nx;
  hd.C = p->C;
  hd.precision = p->precision;
  hd.count = p->count;
  hd.lbfgs_m = m;
  hd.variant = variant_code(p->g);
  hd.iters = S->iters;
  hd.vbytes = (size_t)p->count * p->C * p->n * p->nx * p->elt;
  hd.o = S->o;
  hd.o.stream = nullptr;
  // Every copy is ordered on the solver's stream and finished before the call
  // returns: a device-to-device cudaMemcpy on the legacy stream would neither
  // block the host nor order the solver's (non-blocking) stream, so the next
  // step could overwrite the state while it is being copied.
  cudaStream_t st = S->work;
  char* out = (char*)dst;
  WF_TRY(cudaMemcpyAsync(out, &hd, sizeof hd, cudaMemcpyDefault, st));
  WF_TRY(cudaMemcpyAsync(out + off_st, S->st, sizeof(WfLbMap) * p->count, cudaMemcpyDefault, st));
  const void* vecs[2] = {S->s, S->g};
  const size_t vs = up256s(hd.vbytes);
  for (int i = 0; i < 2; ++i)
    WF_TRY(cudaMemcpyAsync(out + off_vec + i * vs, vecs[i], hd.vbytes, cudaMemcpyDefault, st));
  for (int i = 0; i < 2 * m; ++i)
    WF_TRY(cudaMemcpyAsync(out + off_vec + (2 + (size_t)i) * vs, (const char*)S->ring + (size_t)i * hd.vbytes,
                           hd.vbytes, cudaMemcpyDefault, st));
  WF_TRY(cudaStreamSynchronize(st));
  return WF_OK;
}

template <typename T>
static wf_status import_impl(wf_problem* p, const WfStateHeader& hd, const char* in, void* stream) {
  const int m = hd.lbfgs_m;
  wf_status rs = ensure_solver(p, m);
  if (rs != WF_OK) return rs;
  WfSolver* S = p->solver;
  S->o = hd.o;
  S->o.stream = stream;
  S->iters = hd.iters;
  cudaStream_t us = (cudaStream_t)stream;
  cudaStream_t st = wf_capturable(us) ? us : S->stream;
  if (S->exec) { cudaGraphExecDestroy(S->exec); S->exec = nullptr; }
  S->work = st;
  p->g = variant_geo(wf_make_geo(p->n, p->nx, p->C, p->count), hd.variant);
  rs = setup_args(p, S, &S->o);
  if (rs != WF_OK) return rs;
  size_t off_st, off_vec;
  state_bytes(p, m, &off_st, &off_vec);
  const size_t vs = up256s(hd.vbytes);
  WF_TRY(cudaEventRecord(S->ev_in, us));
  WF_TRY(cudaStreamWaitEvent(st, S->ev_in, 0));
  WF_TRY(cudaMemcpyAsync(S->st, in + off_st, sizeof(WfLbMap) * p->count, cudaMemcpyDefault, st));
  void* vecs[2] = {S->s, S->g};
  for (int i = 0; i < 2; ++i) WF_TRY(cudaMemcpyAsync(vecs[i], in + off_vec + i * vs, hd.vbytes, cudaMemcpyDefault, st));
  for (int i = 0; i < 2 * m; ++i)
    WF_TRY(cudaMemcpyAsync((char*)S->ring + (size_t)i * hd.vbytes, in + off_vec + (2 + (size_t)i) * vs, hd.vbytes,
                           cudaMemcpyDefault, st));
  WF_TRY(cudaStreamSynchronize(st));  // the source may be pageable host memory the caller frees next
  S->graph_pending = S->o.use_graphs ? 1 : 0;
  S->started = 1;
  return WF_OK;
}

extern "C" wf_status wf_solver_import(wf_problem* p, const void* src, size_t bytes, void* stream) {
  if (!p || !src) return wf_fail(WF_EINVAL, "wf_solver_import: null argument");
  if (bytes < sizeof(WfStateHeader)) return wf_fail(WF_EINVAL, "wf_solver_import: %zu bytes is no checkpoint", bytes);
  WfStateHeader hd;
  WF_TRY(cudaMemcpy(&hd, src, sizeof hd, cudaMemcpyDefault));
  if (memcmp(hd.magic, kWfStateMagic, 8) != 0) return wf_fail(WF_EINVAL, "wf_solver_import: not a solver checkpoint");
  if (hd.n != p->n || hd.nx != p->nx || hd.C != p->C || hd.precision != p->precision || hd.count != p->count)
    return wf_fail(WF_EINVAL,
                   "wf_solver_import: checkpoint of %d x %d maps, C = %d, precision %d, %d maps; problem has %d x %d, "
                   "%d, %d, %d",
                   hd.n, hd.nx, hd.C, hd.precision, hd.count, p->n, p->nx, p->C, p->precision, p->count);
  if (!variant_valid(hd.variant) || hd.lbfgs_m < 1 || hd.lbfgs_m > WF_MAXM ||
      hd.vbytes != (size_t)p->count * p->C * p->n * p->nx * p->elt)
    return wf_fail(WF_EINVAL, "wf_solver_import: corrupt checkpoint header");
  size_t off_st, off_vec;
  const size_t need = state_bytes(p, hd.lbfgs_m, &off_st, &off_vec);
  if (bytes < need) return wf_fail(WF_EINVAL, "wf_solver_import: %zu bytes given, %zu needed", bytes, need);
  wf_opts o = hd.o;
  o.stream = stream;
  o.fft_variant = 0;
  o.inject_timeout_map = 0;
  wf_status rs = check_opts(p, &o);
  if (rs != WF_OK) return rs;
  if (hd.o.inject_timeout_map != 0) return wf_fail(WF_EINVAL, "wf_solver_import: checkpoint of a diagnostic run");
  return p->precision == WF_FP64 ? import_impl<double>(p, hd, (const char*)src, stream)
                                 : import_impl<float>(p, hd, (const char*)src, stream);
}

extern "C" wf_status wf_problem_variant(const wf_problem* p, int* variant) {
  if (!p || !variant) return wf_fail(WF_EINVAL, "wf_problem_variant: null argument");
  *variant = variant_code(p->g);
  return WF_OK;
}

extern "C" wf_status wf_solver_history(const wf_problem* p, double* out, int* counts) {
  if (!p || !out || !counts) return wf_fail(WF_EINVAL, "wf_solver_history: null argument");
  const WfSolver* S = p->solver;
  if (!S || !S->hist || S->A.hcap <= 0)
    return wf_fail(WF_EINVAL, "wf_solver_history: no solve with a history was started");
  const int cap = S->A.hcap, B = p->count;
  std::vector<double> ring((size_t)B * cap * 5);
  std::vector<WfLbMap> st(B);
  cudaError_t e = cudaStreamSynchronize(S->work);
  if (e == cudaSuccess) e = cudaMemcpy(ring.data(), S->hist, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(st.data(), S->st, sizeof(WfLbMap) * B, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return wf_cuda_fail(e, "wf_solver_history");
  for (int b = 0; b < B; ++b) {
    const int k = st[b].k, nrec = k < cap ? k : cap;
    counts[b] = nrec;
    double* ob = out + (size_t)b * cap * 5;
    for (int i = 0; i < cap * 5; ++i) ob[i] = NAN;
    for (int i = 0; i < nrec; ++i) {  // iterations k - nrec + 1 .. k, oldest first
      const int it = k - nrec + 1 + i;
      const double* r = ring.data() + ((size_t)b * cap + (it - 1) % cap) * 5;
      for (int c = 0; c < 5; ++c) ob[(size_t)i * 5 + c] = r[c];
    }
  }
  return WF_OK;
}

// Self-test of the bounds checks: one index five past the end of a tile.
__global__ void k_dbg_selftest(int* sink) {
  const long long i = WF_CHK((long long)WF_TILE + 5, WF_TILE);
  if (sink) *sink = (int)i;
}
cudaError_t wf_dbg_selftest() {
  k_dbg_selftest<<<1, 1>>>(nullptr);
  return cudaGetLastError();
}

WF_DBG_READER(solve)
