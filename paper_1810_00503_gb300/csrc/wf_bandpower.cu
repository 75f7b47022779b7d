// Band powers from simulations (Sec. 2.4-2.5 of the paper):
//   E_l  = 1/2 sum_{k in l} |s_hat_k|^2 / Theta_fid,l           (eq. el, whitened)
//   b_l  = mean over simulations j of E_l(MAP(d_j)),
//          d_j = M (A z_j + n_j)                               (eq. blmv)
//   F_ll' Delta Theta_l' = mean_j [E_l(MAP(d_j + delta_l'j)) - E_l(MAP(d_j))],
//          delta_l'j = M A_l' u_l'j, Delta Theta_l' = Theta_fid,l' (eq. fisher)
//   Theta_hat = Theta_fid + F^-1 (E - b),  cov = F^-1         (eq. eq:wfmv, eq:var)
// Theta_fid,l is the mean of P over the band's full-plane modes.  The data,
// noise-bias and Fisher maps are solved together in one batched L-BFGS run.
// Random fields are inputs, or drawn here from a counter-based generator with
// a caller-given seed, so a run is reproducible and testable.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <cmath>
#include <utility>
#include <vector>

#include "wf_api_internal.h"

// Theta_fid,l: full-plane mean of P over band l (half-plane multiplicity 1 on
// the kx = 0 and kx = nx/2 columns, 2 elsewhere; P is [C][ny][nx/2+1]).  One block; per-warp bins
// ([warps][2 nb]: sums, then counts) summed in a fixed order, so the result is
// the same on every run.
template <typename S>
__global__ void k_theta_fid(const S* P, const int16_t* band, int ny, int nx, int C, int nb, double* theta) {
  extern __shared__ double sh[];
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < 2 * nb * nw; i += blockDim.x) sh[i] = 0.0;
  __syncthreads();
  const int h = nx / 2;
  const size_t tot = (size_t)C * ny * (h + 1);
  double* bins = sh + (size_t)w * 2 * nb;
  for (size_t i0 = 0; i0 < tot; i0 += blockDim.x) {  // uniform trip count across the block
    const size_t i = i0 + threadIdx.x;
    int l = -1;
    double wt = 0.0, pv = 0.0;
    if (i < tot) {
      l = band[i];
      if (l >= nb) l = -1;
      if (l >= 0) {
        const int kx = (int)(i % (h + 1));
        wt = (kx == 0 || kx == h) ? 1.0 : 2.0;
        pv = wt * (double)P[i];
      }
    }
    wf_warp_bin_add(bins, l, pv);
    wf_warp_bin_add(bins + nb, l, wt);
  }
  __syncthreads();
  for (int l = threadIdx.x; l < nb; l += blockDim.x) {
    double sum = 0.0, cnt = 0.0;
    for (int q = 0; q < nw; ++q) {
      sum += sh[(size_t)q * 2 * nb + l];
      cnt += sh[(size_t)q * 2 * nb + nb + l];
    }
    theta[l] = cnt > 0.0 ? sum / cnt : 0.0;
  }
}

// P restricted to each band: out[l][i] = band[i] == l ? P[i] : 0; with lo > 0
// one more table, P on the bands lo and above (the B bands of the
// leakage-bias form): out[nb][i] = band[i] >= lo ? P[i] : 0.
template <typename S>
__global__ void k_band_P(const S* P, const int16_t* band, size_t tot, int nb, int lo, S* out) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += stride) {
    const int l = band[i];
    const S p = P[i];
    for (int k = 0; k < nb; ++k) out[(size_t)k * tot + i] = (l == k) ? p : (S)0;
    if (lo > 0) out[(size_t)nb * tot + i] = (l >= lo) ? p : (S)0;
  }
}

// Rows of wf_bandpower_in.u: the bands with per-band Fisher maps (every band,
// the listed ones, or the E bands of the leakage-bias form), then with
// leak_split the one row of joint B maps.
static int bp_fisher_rows(const wf_bandpower_in* in) {
  const int nE = in->leak_split > 0 ? in->leak_split : in->n_bands;
  return (in->fd_bands ? in->n_fd_bands : nE) + (in->leak_split > 0 ? 1 : 0);
}

// Fisher-map bookkeeping shared by the estimator and the combination of
// partial sums: fdb[k] is the band of Fisher row k (k < nbF), fdk[l] the row
// band l's column comes from (-1: interpolated), with leak_split every B band
// pointing at the last row, the joint B maps.  Checks fd_bands.
static wf_status bp_rows(const wf_bandpower_in* in, const char* who, int* fdb, int* fdk, int* nbF_out) {
  const int nb = in->n_bands, L = in->leak_split;
  const int nE = L > 0 ? L : nb;
  int nbF = 0;
  for (int l = 0; l < nb; ++l) fdk[l] = -1;
  if (in->fd_bands) {
    if (in->n_fd_bands < 1 || in->n_fd_bands > nE) return wf_fail(WF_EINVAL, "%s: n_fd_bands = %d", who, in->n_fd_bands);
    for (int k = 0; k < in->n_fd_bands; ++k) {
      const int l = in->fd_bands[k];
      if (l < 0 || l >= nE || (k > 0 && l <= fdb[k - 1]))
        return wf_fail(WF_EINVAL, "%s: fd_bands must be ascending band ids in [0, %s)", who,
                       L > 0 ? "leak_split" : "n_bands");
      fdb[nbF] = l;
      fdk[l] = nbF++;
    }
  } else {
    for (int l = 0; l < nE; ++l) fdb[nbF] = l, fdk[l] = nbF++;
  }
  for (int l = nE; l < nb; ++l) fdk[l] = nbF;
  *nbF_out = nbF;
  return WF_OK;
}

// Partial sums of the estimator over a set of simulations, from the band
// energies of its solved maps (rows: 0 = data, 1..J = noise-bias simulations,
// 1+J+k*nfd+j = Fisher map of row k reusing simulation j):
//   [J, J_fd, sum_j E_j (nb), sum_j E_j E_j^T (nb x nb),
//    sum_{j < J_fd} (E(Fisher map k, j) - E_j) (nR x nb, [k][l])]
// Sums over several GPUs' simulations add entry by entry.  Entry i, in a
// fixed summation order (the device kernel and the host call share it).
static __host__ __device__ inline size_t bp_sums_len(int nb, int nR) {
  return 2 + (size_t)nb + (size_t)nb * nb + (size_t)nR * nb;
}
static __host__ __device__ double bp_sum_entry(const double* E, int nb, int J, int nfd, size_t i) {
  if (i == 0) return (double)J;
  if (i == 1) return (double)nfd;
  i -= 2;
  double s = 0.0;
  if (i < (size_t)nb) {
    for (int j = 0; j < J; ++j) s += E[(size_t)(1 + j) * nb + i];
    return s;
  }
  i -= nb;
  if (i < (size_t)nb * nb) {
    const size_t l = i / nb, lp = i % nb;
    for (int j = 0; j < J; ++j) s += E[(size_t)(1 + j) * nb + l] * E[(size_t)(1 + j) * nb + lp];
    return s;
  }
  i -= (size_t)nb * nb;
  const size_t k = i / nb, l = i % nb;
  for (int j = 0; j < nfd; ++j) s += E[(size_t)(1 + J + k * nfd + j) * nb + l] - E[(size_t)(1 + j) * nb + l];
  return s;
}
__global__ void k_bp_sums(const double* E, int nb, int J, int nfd, size_t len, double* sums) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x)
    sums[i] = bp_sum_entry(E, nb, J, nfd, i);
}

// The estimator from the partial sums (eq. blmv, eq. fisher, eq:wfmv), FP64 on
// the host for any number of contributing GPUs:
//   b = S1 / J;  cov_E = (S2 - J b b^T) / (J - 1);
//   F[l][l'] = D[fdk[l']][l] / J_fd / Theta_fid,l' for a band with Fisher maps.
// A column without them is interpolated from the sampled ones (Sec. 3.1: the
// Fisher matrix is smooth and nearly translation invariant): between sampled
// s0 < l' < s1, F[l'+o][l'] = (1-t) F[s0+o][s0] + t F[s1+o][s1],
// t = (l'-s0)/(s1-s0), a term whose row leaves the matrix dropped and the other
// weighted alone; beyond the first or last sampled column the nearest one is
// shifted.  Then F[l][l'] = 0 for l, l' < trunc_n with |l - l'| > trunc_w
// (App. C: far off-diagonal EE terms).  leak > 0 (the leakage-bias form of
// App. C, B bands leak..nb-1): a B band keeps only its diagonal term, the E-B
// cross terms are zero, and the interpolation of an E column stays inside the
// E block.  F^-1 by Gauss-Jordan elimination with partial pivoting;
// Theta_hat = Theta_fid + F^-1 (E - b).  out = [theta | E | b | F | Finv |
// theta_hat | covE] (sizes nb, nb, nb, nb^2, nb^2, nb, nb^2).  J_fd = 0 leaves
// F, F^-1 and Theta_hat NaN.  Returns true if F is singular.
static bool bp_final(const double* sums, const double* E_data, const double* theta, int nb, const int* fdk,
                     int trunc_n, int trunc_w, int leak, double* out) {
  const double J = sums[0], Jfd = sums[1];
  const double* S1 = sums + 2;
  const double* S2 = S1 + nb;
  const double* D = S2 + (size_t)nb * nb;
  double* o_theta = out;
  double* o_E = out + nb;
  double* o_b = out + 2 * nb;
  double* o_F = out + 3 * nb;
  double* o_Fi = o_F + (size_t)nb * nb;
  double* o_th = o_Fi + (size_t)nb * nb;
  double* o_cE = o_th + nb;
  for (int l = 0; l < nb; ++l) {
    o_theta[l] = theta[l];
    o_E[l] = E_data[l];
    o_b[l] = S1[l] / J;
  }
  for (int l = 0; l < nb; ++l)
    for (int lp = 0; lp < nb; ++lp) {
      const int k = fdk[lp];
      o_F[l * nb + lp] = (Jfd > 0.0 && k >= 0) ? D[(size_t)k * nb + l] / Jfd / theta[lp] : 0.0;
      o_cE[l * nb + lp] = J > 1.0 ? (S2[l * nb + lp] - J * o_b[l] * o_b[lp]) / (J - 1.0) : NAN;
    }
  const int lim = leak > 0 ? leak : nb;  // bands an interpolated column draws on (its block)
  std::vector<double> F0(o_F, o_F + (size_t)nb * nb);  // the sampled columns, read by the interpolation
  for (int lp = 0; lp < nb && Jfd > 0.0; ++lp) {
    if (fdk[lp] >= 0) continue;
    int s0 = -1, s1 = -1;
    for (int q = lp - 1; q >= 0 && s0 < 0; --q)
      if (fdk[q] >= 0) s0 = q;
    for (int q = lp + 1; q < lim && s1 < 0; ++q)
      if (fdk[q] >= 0) s1 = q;
    double w0 = 0.0, w1 = 0.0;
    if (s0 >= 0 && s1 >= 0) {
      w1 = (double)(lp - s0) / (double)(s1 - s0);
      w0 = 1.0 - w1;
    } else if (s0 >= 0) {
      w0 = 1.0;
    } else {
      w1 = 1.0;
    }
    for (int l = 0; l < nb; ++l) {
      if (l >= lim) {
        o_F[l * nb + lp] = 0.0;
        continue;
      }
      const int o = l - lp;
      double acc = 0.0, ws = 0.0;
      if (s0 >= 0 && w0 > 0.0 && s0 + o >= 0 && s0 + o < lim) {
        acc += w0 * F0[(size_t)(s0 + o) * nb + s0];
        ws += w0;
      }
      if (s1 >= 0 && w1 > 0.0 && s1 + o >= 0 && s1 + o < lim) {
        acc += w1 * F0[(size_t)(s1 + o) * nb + s1];
        ws += w1;
      }
      o_F[l * nb + lp] = ws > 0.0 ? acc / ws : 0.0;
    }
  }
  for (int l = 0; l < nb; ++l)
    for (int lp = 0; lp < nb; ++lp) {
      if (l < trunc_n && lp < trunc_n && abs(l - lp) > trunc_w) o_F[l * nb + lp] = 0.0;
      if (leak > 0 && (l >= leak || lp >= leak) && l != lp) o_F[l * nb + lp] = 0.0;  // cross blocks, BB off-diagonal
    }
  if (!(Jfd > 0.0)) {  // no Fisher maps: F, F^-1 and Theta_hat are undefined
    for (size_t i = 0; i < (size_t)nb * nb; ++i) o_F[i] = o_Fi[i] = NAN;
    for (int l = 0; l < nb; ++l) o_th[l] = NAN;
    return false;
  }
  // Gauss-Jordan elimination with partial pivoting on [F | I]
  const int w2 = 2 * nb;
  std::vector<double> M((size_t)nb * w2);
  for (int r = 0; r < nb; ++r)
    for (int c = 0; c < w2; ++c) M[(size_t)r * w2 + c] = c < nb ? o_F[r * nb + c] : (c - nb == r ? 1.0 : 0.0);
  bool singular = false;
  for (int col = 0; col < nb; ++col) {
    int best = col;
    double bv = fabs(M[(size_t)col * w2 + col]);
    for (int r = col + 1; r < nb; ++r)
      if (fabs(M[(size_t)r * w2 + col]) > bv) { bv = fabs(M[(size_t)r * w2 + col]); best = r; }
    if (!(bv > 0.0) || !std::isfinite(bv)) singular = true;
    if (best != col)
      for (int c = 0; c < w2; ++c) std::swap(M[(size_t)col * w2 + c], M[(size_t)best * w2 + c]);
    const double pv = M[(size_t)col * w2 + col];
    for (int c = 0; c < w2; ++c) M[(size_t)col * w2 + c] /= pv;
    for (int r = 0; r < nb; ++r) {
      if (r == col) continue;
      const double f = M[(size_t)r * w2 + col];
      for (int c = 0; c < w2; ++c)
        if (c != col) M[(size_t)r * w2 + c] -= f * M[(size_t)col * w2 + c];
      M[(size_t)r * w2 + col] = 0.0;
    }
  }
  for (int l = 0; l < nb; ++l)
    for (int lp = 0; lp < nb; ++lp) o_Fi[l * nb + lp] = M[(size_t)l * w2 + nb + lp];
  for (int l = 0; l < nb; ++l) {
    double s = 0.0;
    for (int k = 0; k < nb; ++k) s += o_Fi[l * nb + k] * (o_E[k] - o_b[k]);
    o_th[l] = o_theta[l] + s;
  }
  return singular;
}

// Writes the estimator's host results (layout of bp_final) to the caller's
// output arrays, host or device.
static wf_status bp_write_out(const double* hout, int nb, int on_device, wf_bandpower_out* out, const char* who) {
  const size_t nb2 = (size_t)nb * nb;
  double* dst[7] = {out->theta_fid, out->E, out->bias, out->fisher, out->cov, out->theta_hat, out->cov_E};
  const size_t off[7] = {0, (size_t)nb, 2 * (size_t)nb, 3 * (size_t)nb, 3 * nb + nb2, 3 * nb + 2 * nb2,
                         4 * nb + 2 * nb2};
  const size_t len[7] = {(size_t)nb, (size_t)nb, (size_t)nb, nb2, nb2, (size_t)nb, nb2};
  for (int i = 0; i < 7; ++i) {
    if (on_device) {
      const cudaError_t e = cudaMemcpy(dst[i], hout + off[i], sizeof(double) * len[i], cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return wf_cuda_fail(e, who);
    } else {
      memcpy(dst[i], hout + off[i], sizeof(double) * len[i]);
    }
  }
  return WF_OK;
}

namespace {
struct Scope {  // frees what the estimator allocates, on every return path
  wf_handle* h;
  void* ptrs[16] = {};
  int n = 0;
  wf_problem* probs[4] = {};
  int np = 0;
  explicit Scope(wf_handle* hh) : h(hh) {}
  void* add(void* p) { ptrs[n++] = p; return p; }
  void addp(wf_problem* p) { probs[np++] = p; }
  ~Scope() {
    for (int i = 0; i < np; ++i) wf_problem_destroy(probs[i]);
    for (int i = 0; i < n; ++i) wf_free(h, ptrs[i]);
  }
};
}  // namespace

#define BP_TRY(expr)                                                      \
  do {                                                                    \
    cudaError_t e_ = (expr);                                              \
    if (e_ != cudaSuccess) return wf_cuda_fail(e_, "bandpower_estimate: " #expr); \
  } while (0)
#define BP_OK(expr)                        \
  do {                                     \
    wf_status s_ = (expr);                 \
    if (s_ != WF_OK) return s_;            \
  } while (0)

extern "C" wf_status bandpower_estimate_rect(wf_handle* h, const wf_map* data, int ny, int nx, int C, int dtype,
                                             int precision, const wf_bandpower_in* in, const wf_opts* opts,
                                             wf_bandpower_out* out, wf_solve_stats* stats) {
  if (!h || !data || !in || !out) return wf_fail(WF_EINVAL, "bandpower_estimate: null argument");
  if (!data->d || !data->mask || !data->Ninv || !data->P)
    return wf_fail(WF_EINVAL, "bandpower_estimate: the data map needs d, mask, Ninv and P");
  if (ny < 8 || ny > WF_NT || (ny & (ny - 1)) || nx < 8 || nx > WF_NT || (nx & (nx - 1)) || (C != 1 && C != 2))
    return wf_fail(WF_EINVAL,
                   "bandpower_estimate: %d x %d maps, C = %d (each side a power of two in [8, %d], C 1 or 2)", ny, nx, C,
                   WF_NT);
  const int nb = in->n_bands, J = in->n_sim, nfd = in->n_fd;
  if (nb < 1 || nb > 64) return wf_fail(WF_EINVAL, "bandpower_estimate: n_bands = %d outside [1, 64]", nb);
  if (J < 1) return wf_fail(WF_EINVAL, "bandpower_estimate: n_sim = %d (need >= 1)", J);
  if (nfd < 0 || nfd > J) return wf_fail(WF_EINVAL, "bandpower_estimate: n_fd = %d outside [0, n_sim]", nfd);
  if (!in->band) return wf_fail(WF_EINVAL, "bandpower_estimate: null band table");
  const bool draw = !in->z && !in->noise && !in->u;  // fields drawn here from opts->seed
  if (!draw && (!in->z || !in->noise || (nfd > 0 && !in->u)))
    return wf_fail(WF_EINVAL, "bandpower_estimate: supply all random fields (z, noise, u) or none");
  if (in->trunc_bands < 0 || in->trunc_bands > nb || in->trunc_width < 0)
    return wf_fail(WF_EINVAL, "bandpower_estimate: trunc_bands = %d, trunc_width = %d", in->trunc_bands,
                   in->trunc_width);
  const int L = in->leak_split;  // > 0: leakage-bias form, B bands L..nb-1
  if (L < 0 || L >= nb || (L > 0 && C != 2))
    return wf_fail(WF_EINVAL, "bandpower_estimate: leak_split = %d (need 0, or 1..n_bands-1 with C = 2)", L);
  if (L > 0 && in->trunc_bands > L)
    return wf_fail(WF_EINVAL, "bandpower_estimate: trunc_bands = %d beyond the E bands (leak_split = %d)",
                   in->trunc_bands, L);
  const int nE = L > 0 ? L : nb;  // bands that may get per-band Fisher maps
  if (in->fd_bands && (in->n_fd_bands < 1 || in->n_fd_bands > nE))
    return wf_fail(WF_EINVAL, "bandpower_estimate: n_fd_bands = %d", in->n_fd_bands);
  if (in->sim_index) {
    const unsigned long long lim = (1ull << 62) / ((unsigned long long)C * ny * nx * (nb + 1));
    for (int j = 0; j < J; ++j)
      if (in->sim_index[j] < 0 || (unsigned long long)in->sim_index[j] >= lim)
        return wf_fail(WF_EINVAL, "bandpower_estimate: sim_index[%d] = %lld out of range", j, in->sim_index[j]);
  }
  if (!out->theta_fid || !out->E || !out->bias || !out->fisher || !out->cov || !out->theta_hat || !out->cov_E)
    return wf_fail(WF_EINVAL, "bandpower_estimate: null output array");
  if (in->out_on_device != 0 && in->out_on_device != 1)
    return wf_fail(WF_EINVAL, "bandpower_estimate: out_on_device = %d is not 0 or 1", in->out_on_device);
  if (dtype != WF_F32 && dtype != WF_F64) return wf_fail(WF_EINVAL, "bandpower_estimate: bad dtype");
  wf_opts o;
  if (opts) o = *opts;
  else wf_opts_default(&o);
  cudaStream_t st = (cudaStream_t)o.stream;
  const size_t delt = dtype == WF_F64 ? 8 : 4;
  const size_t welt = precision == WF_FP64 ? 8 : 4;
  const size_t npix = (size_t)C * ny * nx, nsp = (size_t)C * ny * (nx / 2 + 1);
  int fdb[64], fdk[64], nbF = 0;
  BP_OK(bp_rows(in, "bandpower_estimate", fdb, fdk, &nbF));
  const int nR = bp_fisher_rows(in);  // nbF, plus the joint B row
  const int nF = nR * nfd, Btot = 1 + J + nF;
  Scope sc(h);
  // Theta_fid and the band-restricted power tables
  double* theta = nullptr;
  BP_OK(wf_alloc(h, (void**)&theta, sizeof(double) * nb, "theta_fid"));
  sc.add(theta);
  if (dtype == WF_F64)
    k_theta_fid<double><<<1, 1024, 64 * nb * sizeof(double), st>>>((const double*)data->P, in->band, ny, nx, C, nb, theta);
  else
    k_theta_fid<float><<<1, 1024, 64 * nb * sizeof(double), st>>>((const float*)data->P, in->band, ny, nx, C, nb, theta);
  BP_TRY(cudaGetLastError());
  void* Pl = nullptr;
  BP_OK(wf_alloc(h, &Pl, nsp * (nb + (L > 0)) * delt, "band-restricted power"));
  sc.add(Pl);
  const int gblk = (int)((nsp + 255) / 256 < 4096 ? (nsp + 255) / 256 : 4096);
  if (dtype == WF_F64)
    k_band_P<double><<<gblk, 256, 0, st>>>((const double*)data->P, in->band, nsp, nb, L, (double*)Pl);
  else
    k_band_P<float><<<gblk, 256, 0, st>>>((const float*)data->P, in->band, nsp, nb, L, (float*)Pl);
  BP_TRY(cudaGetLastError());

  // noise-bias simulations d_j = M (A z_j + n_j)
  wf_map* maps = (wf_map*)calloc((size_t)Btot, sizeof(wf_map));
  if (!maps) return wf_fail(WF_ENOMEM, "bandpower_estimate: host allocation");
  for (int i = 0; i < Btot; ++i) {
    maps[i].d = nullptr;
    maps[i].mask = data->mask;
    maps[i].Ninv = data->Ninv;
    maps[i].P = data->P;
  }
  wf_problem* psim = nullptr;
  wf_status rs = wf_problem_create_rect(h, maps, J, ny, nx, C, dtype, precision, 1, (void*)st, &psim);
  if (rs != WF_OK) { free(maps); return rs; }
  sc.addp(psim);
  const void* zin = in->z;
  const void* nzin = in->noise;
  const void* uin = in->u;
  if (draw) {  // streams 0, 1, 2 of opts->seed; noise scaled by the simulations' W = M Ninv
    void *zb = nullptr, *nb_ = nullptr, *ub = nullptr;
    rs = wf_alloc(h, &zb, npix * J * welt, "drawn signal fields");
    if (rs == WF_OK) { sc.add(zb); rs = wf_alloc(h, &nb_, npix * J * welt, "drawn noise"); }
    if (rs == WF_OK) { sc.add(nb_); if (nF > 0) rs = wf_alloc(h, &ub, npix * nF * welt, "drawn Fisher fields"); }
    if (rs == WF_OK && ub) sc.add(ub);
    const int f64 = precision == WF_FP64;
    for (int j = 0; j < J && rs == WF_OK; ++j) {  // simulation j: global index g, deviates g npix ..
      const unsigned long long g = in->sim_index ? (unsigned long long)in->sim_index[j] : (unsigned long long)j;
      rs = wf_draw_normal(o.seed, 0, g * npix, npix, f64, (char*)zb + j * npix * welt, nullptr, st);
      if (rs == WF_OK)
        rs = wf_draw_normal(o.seed, 1, g * npix, npix, f64, (char*)nb_ + j * npix * welt,
                            (const char*)psim->w + j * npix * welt, st);
      for (int k = 0; k < nR && j < nfd && rs == WF_OK; ++k)  // Fisher map (row k, j) reuses simulation j;
        rs = wf_draw_normal(o.seed, 2, (g * nb + (k < nbF ? fdb[k] : L)) * npix, npix, f64,  // joint B: band L's
                            (char*)ub + ((size_t)k * nfd + j) * npix * welt, nullptr, st);
    }
    if (rs != WF_OK) { free(maps); return rs; }
    zin = zb;
    nzin = nb_;
    uin = ub;
  }
  void* dsim = nullptr;
  rs = wf_alloc(h, &dsim, npix * J * welt, "simulated data");
  if (rs != WF_OK) { free(maps); return rs; }
  sc.add(dsim);
  rs = wf_simulate_data(psim, zin, nzin, dsim, st);
  if (rs != WF_OK) { free(maps); return rs; }

  // Fisher maps: d_j + M A_l u_lj, synthesised with the band-restricted power as
  // signal and the simulation's data as "noise" (M d_j = d_j); the joint B maps
  // with the power of every B band
  for (int k = 0; k < nR; ++k)
    for (int j = 0; j < nfd; ++j)
      maps[k * nfd + j].P = (const char*)Pl + (size_t)(k < nbF ? fdb[k] : nb) * nsp * delt;
  void* dfd = nullptr;
  if (nF > 0) {
    wf_problem* pfd = nullptr;
    rs = wf_problem_create_rect(h, maps, nF, ny, nx, C, dtype, precision, 1, (void*)st, &pfd);
    if (rs != WF_OK) { free(maps); return rs; }
    sc.addp(pfd);
    void* nfd_in = nullptr;
    rs = wf_alloc(h, &nfd_in, npix * nF * welt, "Fisher base data");
    if (rs == WF_OK) { sc.add(nfd_in); rs = wf_alloc(h, &dfd, npix * nF * welt, "Fisher data"); }
    if (rs != WF_OK) { free(maps); return rs; }
    sc.add(dfd);
    for (int k = 0; k < nR; ++k)
      for (int j = 0; j < nfd; ++j) {
        cudaError_t e = cudaMemcpyAsync((char*)nfd_in + (size_t)(k * nfd + j) * npix * welt,
                                        (const char*)dsim + (size_t)j * npix * welt, npix * welt,
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) { free(maps); return wf_cuda_fail(e, "bandpower_estimate: Fisher base copy"); }
      }
    rs = wf_simulate_data(pfd, uin, nfd_in, dfd, st);
    if (rs != WF_OK) { free(maps); return rs; }
  }

  // one batched MAP solve: data, simulations, Fisher maps
  for (int i = 0; i < Btot; ++i) maps[i].P = data->P;
  maps[0].d = data->d;
  wf_problem* ps = nullptr;
  rs = wf_problem_create_rect(h, maps, Btot, ny, nx, C, dtype, precision, o.lbfgs_m, (void*)st, &ps);
  free(maps);
  if (rs != WF_OK) return rs;
  sc.addp(ps);
  BP_TRY(cudaMemcpyAsync((char*)ps->d + npix * welt, dsim, npix * J * welt, cudaMemcpyDeviceToDevice, st));
  if (nF > 0)
    BP_TRY(cudaMemcpyAsync((char*)ps->d + (size_t)(1 + J) * npix * welt, dfd, npix * nF * welt,
                           cudaMemcpyDeviceToDevice, st));
  void* sall = nullptr;
  BP_OK(wf_alloc(h, &sall, nsp * Btot * 2 * welt, "MAP spectra"));
  sc.add(sall);
  wf_solve_stats* hst = (wf_solve_stats*)calloc((size_t)Btot, sizeof(wf_solve_stats));
  if (!hst) return wf_fail(WF_ENOMEM, "bandpower_estimate: host allocation");
  rs = wf_map_solve(ps, &o, nullptr, sall, nullptr, hst);
  if (stats) memcpy(stats, hst, sizeof(wf_solve_stats) * Btot);
  free(hst);
  if (rs != WF_OK && rs != WF_ENOTCONVERGED) return rs;
  const wf_status solve_status = rs;
  double* Eall = nullptr;
  BP_OK(wf_alloc(h, (void**)&Eall, sizeof(double) * Btot * nb, "band energies"));
  sc.add(Eall);
  BP_OK(wf_band_energy(ps, sall, in->band, theta, nb, Eall, st));
  const size_t slen = bp_sums_len(nb, nR);
  double* dsums = nullptr;
  BP_OK(wf_alloc(h, (void**)&dsums, sizeof(double) * slen, "partial sums"));
  sc.add(dsums);
  k_bp_sums<<<(int)((slen + 127) / 128), 128, 0, st>>>(Eall, nb, J, nfd, slen, dsums);
  BP_TRY(cudaGetLastError());
  std::vector<double> hsums(slen), hhead(2 * (size_t)nb);  // sums; theta_fid and the data map's E
  BP_TRY(cudaMemcpyAsync(hsums.data(), dsums, sizeof(double) * slen, cudaMemcpyDeviceToHost, st));
  BP_TRY(cudaMemcpyAsync(hhead.data(), theta, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
  BP_TRY(cudaMemcpyAsync(hhead.data() + nb, Eall, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
  BP_TRY(cudaStreamSynchronize(st));
  std::vector<double> hout(4 * (size_t)nb + 3 * (size_t)nb * nb);
  const bool singular = bp_final(hsums.data(), hhead.data() + nb, hhead.data(), nb, fdk, in->trunc_bands,
                                 in->trunc_width, L, hout.data());
  BP_OK(bp_write_out(hout.data(), nb, in->out_on_device, out, "bandpower_estimate: writing results"));
  if (out->E_maps) {
    const cudaError_t e = cudaMemcpy(out->E_maps, Eall, sizeof(double) * (size_t)Btot * nb,
                                     in->out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return wf_cuda_fail(e, "bandpower_estimate: reading E_maps");
  }
  if (nfd > 0 && singular) return wf_fail(WF_ENONFINITE, "bandpower_estimate: the Fisher matrix is singular");
  return solve_status;
}

extern "C" wf_status bandpower_estimate(wf_handle* h, const wf_map* data, int n, int C, int dtype, int precision,
                                        const wf_bandpower_in* in, const wf_opts* opts, wf_bandpower_out* out,
                                        wf_solve_stats* stats) {
  return bandpower_estimate_rect(h, data, n, n, C, dtype, precision, in, opts, out, stats);
}

extern "C" size_t bandpower_sums_len(int n_bands, int n_rows) {
  if (n_bands < 1 || n_rows < 0) return 0;
  return bp_sums_len(n_bands, n_rows);
}

extern "C" wf_status bandpower_sums(const double* E_maps, int n_bands, int n_sim, int n_fd, int n_rows,
                                    double* sums) {
  if (!E_maps || !sums) return wf_fail(WF_EINVAL, "bandpower_sums: null argument");
  if (n_bands < 1 || n_bands > 64 || n_sim < 1 || n_fd < 0 || n_fd > n_sim || n_rows < 0 || (n_fd > 0 && n_rows < 1))
    return wf_fail(WF_EINVAL, "bandpower_sums: n_bands = %d, n_sim = %d, n_fd = %d, n_rows = %d", n_bands, n_sim,
                   n_fd, n_rows);
  const size_t len = bp_sums_len(n_bands, n_rows);
  for (size_t i = 0; i < len; ++i) sums[i] = bp_sum_entry(E_maps, n_bands, n_sim, n_fd, i);
  return WF_OK;
}

extern "C" wf_status bandpower_combine(const double* sums, const double* E_data, const double* theta_fid,
                                       const wf_bandpower_in* rules, wf_bandpower_out* out) {
  if (!sums || !E_data || !theta_fid || !rules || !out) return wf_fail(WF_EINVAL, "bandpower_combine: null argument");
  const int nb = rules->n_bands, L = rules->leak_split;
  if (nb < 1 || nb > 64) return wf_fail(WF_EINVAL, "bandpower_combine: n_bands = %d outside [1, 64]", nb);
  if (L < 0 || L >= nb) return wf_fail(WF_EINVAL, "bandpower_combine: leak_split = %d", L);
  if (rules->trunc_bands < 0 || rules->trunc_bands > (L > 0 ? L : nb) || rules->trunc_width < 0)
    return wf_fail(WF_EINVAL, "bandpower_combine: trunc_bands = %d, trunc_width = %d", rules->trunc_bands,
                   rules->trunc_width);
  if (rules->out_on_device != 0 && rules->out_on_device != 1)
    return wf_fail(WF_EINVAL, "bandpower_combine: out_on_device = %d is not 0 or 1", rules->out_on_device);
  if (!out->theta_fid || !out->E || !out->bias || !out->fisher || !out->cov || !out->theta_hat || !out->cov_E)
    return wf_fail(WF_EINVAL, "bandpower_combine: null output array");
  const double J = sums[0], Jfd = sums[1];
  if (!(J >= 1.0) || !(Jfd >= 0.0) || Jfd > J || J != floor(J) || Jfd != floor(Jfd))
    return wf_fail(WF_EINVAL, "bandpower_combine: the sums hold J = %g simulations, J_fd = %g Fisher ones", J, Jfd);
  for (int l = 0; l < nb; ++l)
    if (!(theta_fid[l] > 0.0)) return wf_fail(WF_EINVAL, "bandpower_combine: theta_fid[%d] = %g", l, theta_fid[l]);
  int fdb[64], fdk[64], nbF = 0;
  wf_status rs = bp_rows(rules, "bandpower_combine", fdb, fdk, &nbF);
  if (rs != WF_OK) return rs;
  std::vector<double> hout(4 * (size_t)nb + 3 * (size_t)nb * nb);
  const bool singular = bp_final(sums, E_data, theta_fid, nb, fdk, rules->trunc_bands, rules->trunc_width, L,
                                 hout.data());
  rs = bp_write_out(hout.data(), nb, rules->out_on_device, out, "bandpower_combine: writing results");
  if (rs != WF_OK) return rs;
  if (Jfd > 0.0 && singular) return wf_fail(WF_ENONFINITE, "bandpower_combine: the Fisher matrix is singular");
  return WF_OK;
}

// P <- P * q[l] on the modes of band l (others unchanged), in the input dtype.
template <typename S>
__global__ void k_scale_bands(S* P, const int16_t* band, size_t tot, const double* q, int nb) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += stride) {
    const int l = band[i];
    if (l >= 0 && l < nb) P[i] = (S)((double)P[i] * q[l]);
  }
}

extern "C" wf_status bandpower_iterate_rect(wf_handle* h, const wf_map* data, int ny, int nx, int C, int dtype,
                                            int precision, const wf_bandpower_in* in, const wf_opts* opts,
                                            int n_iter, double q_min, double q_max, void* P_out,
                                            double* theta_hat_hist, wf_bandpower_out* out, wf_solve_stats* stats) {
  if (!h || !data || !in || !out) return wf_fail(WF_EINVAL, "bandpower_iterate: null argument");
  if (n_iter < 1 || n_iter > 100) return wf_fail(WF_EINVAL, "bandpower_iterate: n_iter = %d outside [1, 100]", n_iter);
  if (!(q_min > 0.0 && q_min <= 1.0 && q_max >= 1.0 && isfinite(q_max)))
    return wf_fail(WF_EINVAL, "bandpower_iterate: need 0 < q_min <= 1 <= q_max (got %g, %g)", q_min, q_max);
  if (in->n_fd < 1) return wf_fail(WF_EINVAL, "bandpower_iterate: needs n_fd >= 1 (the Fisher matrix)");
  if (!data->P || !in->band) return wf_fail(WF_EINVAL, "bandpower_iterate: null P or band table");
  if (ny < 8 || ny > WF_NT || (ny & (ny - 1)) || nx < 8 || nx > WF_NT || (nx & (nx - 1)) || (C != 1 && C != 2))
    return wf_fail(WF_EINVAL,
                   "bandpower_iterate: %d x %d maps, C = %d (each side a power of two in [8, %d], C 1 or 2)", ny,
                   nx, C, WF_NT);
  if (dtype != WF_F32 && dtype != WF_F64) return wf_fail(WF_EINVAL, "bandpower_iterate: bad dtype");
  wf_opts o;
  if (opts) o = *opts;
  else wf_opts_default(&o);
  cudaStream_t st = (cudaStream_t)o.stream;
  const int nb = in->n_bands;
  const size_t delt = dtype == WF_F64 ? 8 : 4;
  const size_t nsp = (size_t)C * ny * (nx / 2 + 1);
  Scope sc(h);
  void* Pc = nullptr;
  double* qd = nullptr;
  BP_OK(wf_alloc(h, &Pc, nsp * delt, "iterated fiducial power"));
  sc.add(Pc);
  BP_OK(wf_alloc(h, (void**)&qd, sizeof(double) * (nb > 0 ? nb : 1), "band factors"));
  sc.add(qd);
  BP_TRY(cudaMemcpyAsync(Pc, data->P, nsp * delt, cudaMemcpyDeviceToDevice, st));
  wf_map m = *data;
  m.P = Pc;
  wf_status worst = WF_OK;
  double q[64];
  // device outputs: the estimates go to host arrays (the fiducial moves on the
  // host between them) and the last one is copied out at the end
  const bool dev = in->out_on_device != 0;
  wf_bandpower_in inh = *in;
  inh.out_on_device = 0;
  const size_t nb2 = (size_t)nb * nb;
  const size_t nEm = (size_t)(1 + in->n_sim + (size_t)bp_fisher_rows(in) * in->n_fd) * nb;
  std::vector<double> hbuf(dev ? 4 * (size_t)nb + 3 * nb2 + (out->E_maps ? nEm : 0) : 0);
  wf_bandpower_out hs = *out;
  if (dev) {
    double* p = hbuf.data();
    hs.theta_fid = p; p += nb;
    hs.E = p; p += nb;
    hs.bias = p; p += nb;
    hs.fisher = p; p += nb2;
    hs.cov = p; p += nb2;
    hs.theta_hat = p; p += nb;
    hs.cov_E = p; p += nb2;
    hs.E_maps = out->E_maps ? p : nullptr;
  }
  wf_bandpower_out* ob = dev ? &hs : out;
  for (int it = 0; it < n_iter; ++it) {
    const wf_status rs = bandpower_estimate_rect(h, &m, ny, nx, C, dtype, precision, &inh, &o, ob, stats);
    if (rs != WF_OK && rs != WF_ENOTCONVERGED) return rs;
    if (rs != WF_OK) worst = rs;
    if (theta_hat_hist) memcpy(theta_hat_hist + (size_t)it * nb, ob->theta_hat, sizeof(double) * nb);
    if (it + 1 == n_iter) break;
    for (int l = 0; l < nb; ++l) {  // regularised move of each band: ratio kept in [q_min, q_max]
      const double r = ob->theta_hat[l] / ob->theta_fid[l];
      q[l] = isfinite(r) ? fmin(fmax(r, q_min), q_max) : 1.0;
    }
    BP_TRY(cudaMemcpyAsync(qd, q, sizeof(double) * nb, cudaMemcpyHostToDevice, st));
    const int gblk = (int)((nsp + 255) / 256 < 4096 ? (nsp + 255) / 256 : 4096);
    if (dtype == WF_F64) k_scale_bands<double><<<gblk, 256, 0, st>>>((double*)Pc, in->band, nsp, qd, nb);
    else k_scale_bands<float><<<gblk, 256, 0, st>>>((float*)Pc, in->band, nsp, qd, nb);
    BP_TRY(cudaGetLastError());
  }
  if (P_out) BP_TRY(cudaMemcpyAsync(P_out, Pc, nsp * delt, cudaMemcpyDeviceToDevice, st));
  BP_TRY(cudaStreamSynchronize(st));
  if (dev) {
    double* dst[8] = {out->theta_fid, out->E, out->bias, out->fisher, out->cov, out->theta_hat, out->cov_E, out->E_maps};
    const double* src[8] = {hs.theta_fid, hs.E, hs.bias, hs.fisher, hs.cov, hs.theta_hat, hs.cov_E, hs.E_maps};
    const size_t len[8] = {(size_t)nb, (size_t)nb, (size_t)nb, nb2, nb2, (size_t)nb, nb2, nEm};
    for (int i = 0; i < 8; ++i)
      if (dst[i]) BP_TRY(cudaMemcpy(dst[i], src[i], sizeof(double) * len[i], cudaMemcpyHostToDevice));
  }
  if (worst != WF_OK) wf_fail(worst, "bandpower_iterate: a solve hit its iteration limit");
  return worst;
}

extern "C" wf_status bandpower_iterate(wf_handle* h, const wf_map* data, int n, int C, int dtype, int precision,
                                       const wf_bandpower_in* in, const wf_opts* opts, int n_iter, double q_min,
                                       double q_max, void* P_out, double* theta_hat_hist, wf_bandpower_out* out,
                                       wf_solve_stats* stats) {
  return bandpower_iterate_rect(h, data, n, n, C, dtype, precision, in, opts, n_iter, q_min, q_max, P_out,
                                theta_hat_hist, out, stats);
}

WF_DBG_READER(bandpower)
