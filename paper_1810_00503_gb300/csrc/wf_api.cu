// C ABI of the Wiener-filter library: handle, prepared problems and the
// single-pass operator calls.  The L-BFGS driver lives in wf_solve.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "wf_api_internal.h"

static thread_local char g_errbuf[1024];

wf_status wf_fail(wf_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_errbuf, sizeof g_errbuf, fmt, ap);
  va_end(ap);
  return s;
}

wf_status wf_cuda_fail(cudaError_t e, const char* what) {
  return wf_fail(e == cudaErrorMemoryAllocation ? WF_ENOMEM : WF_ECUDA, "%s: %s (%s)", what,
                 cudaGetErrorString(e), cudaGetErrorName(e));
}

extern "C" const char* wf_last_error(void) { return g_errbuf; }

extern "C" void wf_opts_default(wf_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->lbfgs_m = 10;
  o->max_iter = 10000;
  o->gtol_rel = 1e-6;
  o->dchi2_abs = 0.0;
  o->refresh_every = 0;
  o->check_every = 16;
  o->use_graphs = 1;
  o->stream = nullptr;
  o->line_search = WF_LS_EXACT;
  o->c1 = 1e-4;
  o->c2 = 0.9;
  o->seed = 0;
  o->spin_limit = 0;
  o->inject_timeout_map = 0;
  o->autotune = 1;
  o->fft_variant = 0;
}

static void wf_geo_tiles(WfGeo& g, int tc_div, int rb_div) {
  int tc = WF_TILE / (g.C * g.n);
  if (tc > g.h) tc = g.h;
  if (tc > WF_THREADS) tc = WF_THREADS;  // a thread keeps one column: the block spans a tile row
  tc /= tc_div;
  if (tc < 2) tc = g.h < 2 ? g.h : 2;
  g.TC = tc;
  g.ntile = g.h / tc;
  int rb = WF_TILE / g.h;
  if (rb > g.C * g.n) rb = g.C * g.n;
  rb /= rb_div;
  if (rb < 1) rb = 1;
  g.RB = rb;
  g.nrb = g.C * g.n / rb;
  g.tc_div = tc_div;
  g.rb_div = rb_div;
}

// A TMA box spans at most 256 elements per dimension: a column tile wider
// than 128 complex values (a map of few rows and many columns) cannot be one
// box row, so such shapes run the inverse column stage on ping-pong passes.
static void wf_geo_fix_kind(WfGeo& g) {
  if (g.colinv_kind == WF_COLINV_TMA_K && 2 * g.TC > 256) g.colinv_kind = WF_COLINV_PP_K;
}

WfGeo wf_make_geo(int ny, int nx, int C, int B) {
  WfGeo g;
  g.n = ny;
  g.nx = nx;
  g.h = nx / 2;
  g.C = C;
  g.lgn = 0;
  while ((1 << g.lgn) < ny) ++g.lgn;
  g.lgnx = 0;
  while ((1 << g.lgnx) < nx) ++g.lgnx;
  g.lgh = g.lgnx - 1;
  // mode (my, mx) has wavevector 2 pi (mx / nx, my / ny) / pixel: scaled by
  // max(ny, nx) both components are integers
  g.ksx = nx < ny ? ny / nx : 1;
  g.ksy = ny < nx ? nx / ny : 1;
  const long long vsz = (long long)C * ny * (nx / 2);
  const int nchunk = (int)((vsz + WF_COMB_CHUNK - 1) / WF_COMB_CHUNK);
  g.sgroup = WF_STREAM_GROUP;
  if (B > 0)
    while (g.sgroup > 1 && (long long)B * ((nchunk + g.sgroup - 1) / g.sgroup) < WF_STREAM_MIN_BLOCKS) g.sgroup /= 2;
  g.ncomb = (nchunk + g.sgroup - 1) / g.sgroup;
  wf_geo_tiles(g, WF_TUNE_MAXDIV, WF_TUNE_MAXDIV);  // the narrowest tiles set the stride
  g.maxblk = g.ntile > g.nrb ? g.ntile : g.nrb;
  if (g.ncomb > g.maxblk) g.maxblk = g.ncomb;
  wf_geo_tiles(g, 1, 1);
  g.colinv_kind = WF_COLINV_TMA ? WF_COLINV_TMA_K : WF_COLINV_PP_K;
  g.row_kind = WF_ROW_PP_K;
  g.col_plan = g.row_plan = 0;
  wf_geo_fix_kind(g);
  return g;
}

WfGeo wf_geo_variant(const WfGeo& base, int colinv_kind, int row_kind, int tc_div, int rb_div, int col_plan,
                     int row_plan) {
  WfGeo g = base;
  wf_geo_tiles(g, tc_div, rb_div);
  g.colinv_kind = colinv_kind;
  g.row_kind = row_kind;
  g.col_plan = col_plan;
  g.row_plan = row_plan;
  wf_geo_fix_kind(g);
  return g;
}

// Pass tables of radix plan `plan` (layout in wf_internal.h) from the roots
// of unity in roots[0, WF_NT): the pass with span Ns and radix R of the length
// 2^lgL transform holds exp(-2 pi i k r / (Ns R)) at (Ns - R1) + (r - 1) Ns + k,
// R1 the radix of the first pass, so consecutive butterflies read consecutive
// entries.
static void wf_plan_tables(const double2* roots, int plan, double2* block) {
  for (int lgL = 1; lgL <= WF_LOG2_NT; ++lgL) {
    double2* tab = block + (size_t)WF_NT * lgL;
    for (int i = 0; i < WF_NT; ++i) { tab[i].x = 0.0; tab[i].y = 0.0; }
    const int np = wf_plan_np(lgL, plan);
    int lgNs = 0, R1 = 1;
    for (int p = 0; p < np; ++p) {
      const int bits = wf_plan_bits(lgL, plan, p), R = 1 << bits, Ns = 1 << lgNs;
      if (p == 0) R1 = R;
      if (Ns > 1) {
        const int sh = WF_LOG2_NT - lgNs - bits;
        for (int r = 1; r < R; ++r)
          for (int k = 0; k < Ns; ++k) tab[(Ns - R1) + (r - 1) * Ns + k] = roots[(k * r) << sh];
      }
      lgNs += bits;
    }
  }
}

// Twiddle buffer of WF_TWTAB entries (plan 0; layout in wf_internal.h).  Roots
// of unity exp(-2 pi i k / WF_NT) are computed in long double, with the values
// at multiples of pi/2 set exactly.
void wf_make_twiddles(double2* out) {
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int k = 0; k < WF_NT; ++k) {
    long double a = -two_pi * (long double)k / (long double)WF_NT;
    double c = (double)cosl(a), s = (double)sinl(a);
    if (k % (WF_NT / 4) == 0) {
      const int q = k / (WF_NT / 4);
      c = (q == 0) ? 1.0 : (q == 2 ? -1.0 : 0.0);
      s = (q == 1) ? -1.0 : (q == 3 ? 1.0 : 0.0);
    }
    out[k].x = c;
    out[k].y = s;
  }
  wf_plan_tables(out, 0, out);
}

// All WF_NPLAN blocks (WF_TWTAB_ALL entries).
static void wf_make_twiddles_all(double2* out) {
  wf_make_twiddles(out);
  for (int plan = 1; plan < WF_NPLAN; ++plan) {
    double2* block = out + (size_t)WF_TWTAB * plan;
    for (int k = 0; k < WF_NT; ++k) block[k] = out[k];
    wf_plan_tables(out, plan, block);
  }
}

extern "C" wf_status wf_create(wf_handle** out, size_t workspace_limit) {
  if (!out) return wf_fail(WF_EINVAL, "wf_create: null output pointer");
  *out = nullptr;
  wf_handle* h = new (std::nothrow) wf_handle();
  if (!h) return wf_fail(WF_ENOMEM, "wf_create: host allocation failed");
  h->limit = workspace_limit;
  h->used = 0;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) { delete h; return wf_cuda_fail(e, "wf_create: cudaGetDevice"); }
  double2* tw64 = (double2*)malloc(sizeof(double2) * WF_TWTAB_ALL);
  float2* tw32 = (float2*)malloc(sizeof(float2) * WF_TWTAB_ALL);
  if (!tw64 || !tw32) {
    free(tw64);
    free(tw32);
    delete h;
    return wf_fail(WF_ENOMEM, "wf_create: host allocation failed");
  }
  wf_make_twiddles_all(tw64);
  for (int k = 0; k < WF_TWTAB_ALL; ++k) { tw32[k].x = (float)tw64[k].x; tw32[k].y = (float)tw64[k].y; }
  wf_status s = wf_alloc(h, &h->tw64, sizeof(double2) * WF_TWTAB_ALL, "twiddle tables");
  if (s == WF_OK) s = wf_alloc(h, &h->tw32, sizeof(float2) * WF_TWTAB_ALL, "twiddle tables");
  e = cudaSuccess;
  if (s == WF_OK) e = cudaMemcpy(h->tw64, tw64, sizeof(double2) * WF_TWTAB_ALL, cudaMemcpyHostToDevice);
  if (s == WF_OK && e == cudaSuccess)
    e = cudaMemcpy(h->tw32, tw32, sizeof(float2) * WF_TWTAB_ALL, cudaMemcpyHostToDevice);
  // A pageable host-to-device cudaMemcpy may return before the DMA into device
  // memory ends; the handle's kernels may run on non-blocking streams that are
  // not ordered after the legacy stream, so wait for the tables here.
  if (s == WF_OK && e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
  free(tw64);
  free(tw32);
  if (s != WF_OK || e != cudaSuccess) {
    wf_free(h, h->tw64);
    wf_free(h, h->tw32);
    delete h;
    return s != WF_OK ? s : wf_cuda_fail(e, "wf_create: twiddle tables");
  }
  *out = h;
  return WF_OK;
}

extern "C" wf_status wf_destroy(wf_handle* h) {
  if (!h) return WF_OK;
  wf_free(h, h->tw64);
  wf_free(h, h->tw32);
  delete h;
  return WF_OK;
}

extern "C" wf_status wf_workspace_used(const wf_handle* h, size_t* bytes) {
  if (!h || !bytes) return wf_fail(WF_EINVAL, "wf_workspace_used: null argument");
  std::lock_guard<std::mutex> lock(const_cast<wf_handle*>(h)->mu);
  *bytes = h->used;
  return WF_OK;
}

static void free_problem(wf_problem* p) {
  if (!p) return;
  void* ptrs[] = {p->d, p->w, p->sp, p->sp0, p->scratch, p->part, p->flags, p->bpart};
  for (void* q : ptrs) wf_free(p->h, q);
  wf_solver_free(p);
  free(p);
}

wf_status wf_alloc(wf_handle* h, void** ptr, size_t bytes, const char* what) {
  *ptr = nullptr;
  {
    std::lock_guard<std::mutex> lock(h->mu);
    if (h->limit && h->used + bytes > h->limit)
      return wf_fail(WF_ENOMEM, "%s: %zu more bytes would exceed the workspace limit (%zu of %zu in use)", what,
                     bytes, h->used, h->limit);
    h->used += bytes;  // reserved before the allocation, so concurrent callers cannot overshoot
  }
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    std::lock_guard<std::mutex> lock(h->mu);
    h->used -= bytes;
    return wf_fail(e == cudaErrorMemoryAllocation ? WF_ENOMEM : WF_ECUDA,
                   "device allocation of %zu bytes for %s failed: %s", bytes, what,
                   cudaGetErrorString(e));
  }
  std::lock_guard<std::mutex> lock(h->mu);
  h->live[*ptr] = bytes;
  return WF_OK;
}

void wf_free(wf_handle* h, void* ptr) {
  if (!ptr) return;
  cudaFree(ptr);
  std::lock_guard<std::mutex> lock(h->mu);
  auto it = h->live.find(ptr);
  if (it != h->live.end()) {
    h->used -= it->second;
    h->live.erase(it);
  }
}

extern "C" wf_status wf_problem_create_rect(wf_handle* h, const wf_map* maps, int count, int ny, int nx, int C,
                                            int dtype, int precision, int lbfgs_m, void* stream,
                                            wf_problem** out) {
  if (!out) return wf_fail(WF_EINVAL, "wf_problem_create: null output pointer");
  *out = nullptr;
  if (!h) return wf_fail(WF_EINVAL, "wf_problem_create: null handle");
  if (!maps || count < 1) return wf_fail(WF_EINVAL, "wf_problem_create: need count >= 1 maps");
  if (ny < 8 || ny > WF_NT || (ny & (ny - 1)))
    return wf_fail(WF_EINVAL, "wf_problem_create: ny = %d is not a power of two in [8, %d]", ny, WF_NT);
  if (nx < 8 || nx > WF_NT || (nx & (nx - 1)))
    return wf_fail(WF_EINVAL, "wf_problem_create: nx = %d is not a power of two in [8, %d]", nx, WF_NT);
  if (C != 1 && C != 2) return wf_fail(WF_EINVAL, "wf_problem_create: C = %d (must be 1 or 2)", C);
  if (dtype != WF_F32 && dtype != WF_F64) return wf_fail(WF_EINVAL, "wf_problem_create: bad dtype %d", dtype);
  if (precision != WF_FP64 && precision != WF_MIXED)
    return wf_fail(WF_EINVAL, "wf_problem_create: bad precision %d", precision);
  if (lbfgs_m < 1 || lbfgs_m > WF_MAXM)
    return wf_fail(WF_EINVAL, "wf_problem_create: lbfgs_m = %d outside [1, %d]", lbfgs_m, WF_MAXM);
  for (int i = 0; i < count; ++i)
    if (!maps[i].mask || !maps[i].Ninv || !maps[i].P)
      return wf_fail(WF_EINVAL, "wf_problem_create: map %d has a null mask, Ninv or P pointer", i);
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != h->device)
    return wf_fail(WF_EINVAL, "wf_problem_create: current device %d differs from the handle's %d", dev,
                   h->device);

  wf_problem* p = (wf_problem*)calloc(1, sizeof(wf_problem));
  if (!p) return wf_fail(WF_ENOMEM, "wf_problem_create: host allocation failed");
  p->h = h;
  p->count = count;
  p->n = ny;
  p->nx = nx;
  p->C = C;
  p->dtype = dtype;
  p->precision = precision;
  p->m = lbfgs_m;
  p->g = wf_make_geo(ny, nx, C, count);
  p->elt = precision == WF_FP64 ? sizeof(double) : sizeof(float);
  int shared = 1;
  for (int i = 1; i < count; ++i) shared &= maps[i].P == maps[0].P;
  p->sp_shared = shared;
  const size_t npix = (size_t)C * ny * nx, nsp = (size_t)C * ny * (nx / 2 + 1);
  p->sp_stride = shared ? 0 : (long long)nsp;
  wf_status s = WF_OK;
  if (s == WF_OK) s = wf_alloc(h, &p->d, npix * count * p->elt, "data maps");
  if (s == WF_OK) s = wf_alloc(h, &p->w, npix * count * p->elt, "weights");
  if (s == WF_OK) s = wf_alloc(h, &p->sp, nsp * (shared ? 1 : count) * p->elt, "sqrt(P) tables");
  if (s == WF_OK) s = wf_alloc(h, &p->scratch, npix * count * p->elt, "scratch");
  if (s == WF_OK) s = wf_alloc(h, (void**)&p->part, sizeof(double) * WF_NSLOT * p->g.maxblk * count, "partial sums");
  if (s == WF_OK) s = wf_alloc(h, (void**)&p->flags, sizeof(int) * 4, "flags");
  if (s != WF_OK) { free_problem(p); return s; }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(p->flags, 0, sizeof(int) * 4, st);
  const void** dp = (const void**)malloc(sizeof(void*) * 4 * (size_t)count);
  if (!dp) { free_problem(p); return wf_fail(WF_ENOMEM, "wf_problem_create: host allocation failed"); }
  const unsigned char** mp = (const unsigned char**)(dp + count);
  const void** np = dp + 2 * count;
  const void** pp = dp + 3 * count;
  for (int i = 0; i < count; ++i) {
    dp[i] = maps[i].d;
    mp[i] = maps[i].mask;
    np[i] = maps[i].Ninv;
    pp[i] = maps[i].P;
  }
  if (e == cudaSuccess) {
    if (precision == WF_FP64)
      e = wf_launch_prep<double>(p->g, dp, mp, np, pp, dtype == WF_F64, count, p->d, p->w, p->sp,
                                 shared, p->flags, st);
    else
      e = wf_launch_prep<float>(p->g, dp, mp, np, pp, dtype == WF_F64, count, p->d, p->w, p->sp,
                                shared, p->flags, st);
  }
  free(dp);
  if (e != cudaSuccess) { free_problem(p); return wf_cuda_fail(e, "wf_problem_create: input preparation"); }
  int flags = 0;
  e = cudaMemcpy(&flags, p->flags, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) { free_problem(p); return wf_cuda_fail(e, "wf_problem_create: reading checks"); }
  if (flags & (1 << WF_ENONFINITE)) {
    free_problem(p);
    return wf_fail(WF_ENONFINITE, "wf_problem_create: non-finite value in d, Ninv or P");
  }
  if (flags & (1 << WF_EINVAL)) {
    free_problem(p);
    return wf_fail(WF_EINVAL, "wf_problem_create: negative value in Ninv or P");
  }
  *out = p;
  return WF_OK;
}

extern "C" wf_status wf_problem_create(wf_handle* h, const wf_map* maps, int count, int n, int C, int dtype,
                                       int precision, int lbfgs_m, void* stream, wf_problem** out) {
  return wf_problem_create_rect(h, maps, count, n, n, C, dtype, precision, lbfgs_m, stream, out);
}

extern "C" wf_status wf_problem_destroy(wf_problem* p) {
  if (p) {
    cudaDeviceSynchronize();
    free_problem(p);
  }
  return WF_OK;
}

WfBufs wf_bufs(const wf_problem* p) {
  WfBufs b;
  b.d = p->d;
  b.w = p->w;
  b.sp = p->sp;
  b.sp_stride = p->sp_stride;
  b.scratch = p->scratch;
  b.part = p->part;
  b.tw = p->precision == WF_FP64 ? p->h->tw64 : p->h->tw32;
  b.ticket = p->flags + 2;  // flags[0] holds the input checks
  b.B = p->count;
  return b;
}

#define WF_DISPATCH(p, call)                                                    \
  ((p)->precision == WF_FP64 ? call<double> : call<float>)

extern "C" wf_status wf_problem_set_data(wf_problem* p, const void* d, void* stream) {
  if (!p || !d) return wf_fail(WF_EINVAL, "wf_problem_set_data: null argument");
  cudaError_t e = WF_DISPATCH(p, wf_launch_set_data)(p->g, d, p->count, p->d, (cudaStream_t)stream);
  return e == cudaSuccess ? WF_OK : wf_cuda_fail(e, "wf_problem_set_data");
}

extern "C" wf_status wf_eval(wf_problem* p, const void* s, void* grad, double* chi2, void* stream) {
  if (!p || !s || !grad) return wf_fail(WF_EINVAL, "wf_eval: null argument");
  if (s == grad) return wf_fail(WF_EINVAL, "wf_eval: s and grad must not alias");
  WfBufs b = wf_bufs(p);
  cudaError_t e = WF_DISPATCH(p, wf_launch_eval)(p->g, b, WF_ROW_DATA, WF_IN_STD, s, grad, chi2,
                                                 (cudaStream_t)stream);
  return e == cudaSuccess ? WF_OK : wf_cuda_fail(e, "wf_eval");
}

extern "C" wf_status wf_hess_vec(wf_problem* p, const void* v, void* hv, void* stream) {
  if (!p || !v || !hv) return wf_fail(WF_EINVAL, "wf_hess_vec: null argument");
  if (v == hv) return wf_fail(WF_EINVAL, "wf_hess_vec: v and hv must not alias");
  WfBufs b = wf_bufs(p);
  cudaError_t e = WF_DISPATCH(p, wf_launch_eval)(p->g, b, WF_ROW_NODATA, WF_IN_STD, v, hv, nullptr,
                                                 (cudaStream_t)stream);
  return e == cudaSuccess ? WF_OK : wf_cuda_fail(e, "wf_hess_vec");
}

extern "C" wf_status wf_signal_map(wf_problem* p, const void* s, void* x, void* stream) {
  if (!p || !s || !x) return wf_fail(WF_EINVAL, "wf_signal_map: null argument");
  WfBufs b = wf_bufs(p);
  cudaError_t e = WF_DISPATCH(p, wf_launch_signal)(p->g, b, WF_IN_STD, s, x, (cudaStream_t)stream);
  return e == cudaSuccess ? WF_OK : wf_cuda_fail(e, "wf_signal_map");
}

extern "C" wf_status wf_simulate_data(wf_problem* p, const void* z, const void* noise, void* d_out,
                                      void* stream) {
  if (!p || !z || !noise || !d_out) return wf_fail(WF_EINVAL, "wf_simulate_data: null argument");
  WfBufs b = wf_bufs(p);
  cudaError_t e = WF_DISPATCH(p, wf_launch_simulate)(p->g, b, z, noise, d_out, (cudaStream_t)stream);
  return e == cudaSuccess ? WF_OK : wf_cuda_fail(e, "wf_simulate_data");
}

// Band-sum partials of nb bands for every map, kept by the problem and grown
// on demand (the allocation orders itself after earlier work on the device).
static wf_status band_partials(wf_problem* p, int nb) {
  const size_t need = (size_t)p->count * wf_band_nblk(p->g) * nb;
  if (p->bpart && p->bpart_n >= need) return WF_OK;
  if (p->bpart) {
    cudaDeviceSynchronize();  // a pending band sum may still read the old buffer
    wf_free(p->h, p->bpart);
    p->bpart = nullptr;
    p->bpart_n = 0;
  }
  wf_status s = wf_alloc(p->h, (void**)&p->bpart, sizeof(double) * need, "band-sum partials");
  if (s == WF_OK) p->bpart_n = need;
  return s;
}

extern "C" wf_status wf_band_energy(wf_problem* p, const void* s, const int16_t* band,
                                    const double* theta, int n_bands, double* E, void* stream) {
  if (!p || !s || !band || !theta || !E) return wf_fail(WF_EINVAL, "wf_band_energy: null argument");
  if (n_bands < 1 || n_bands > 4096) return wf_fail(WF_EINVAL, "wf_band_energy: n_bands = %d", n_bands);
  wf_status rs = band_partials(p, n_bands);
  if (rs != WF_OK) return rs;
  cudaError_t e = WF_DISPATCH(p, wf_launch_band_energy)(p->g, p->count, s, band, theta, n_bands, p->bpart, E,
                                                        (cudaStream_t)stream);
  return e == cudaSuccess ? WF_OK : wf_cuda_fail(e, "wf_band_energy");
}

extern "C" wf_status wf_problem_set_band_scale(wf_problem* p, const int16_t* band, const double* q, int n_b,
                                               void* stream) {
  if (!p || !band || !q) return wf_fail(WF_EINVAL, "wf_problem_set_band_scale: null argument");
  if (n_b < 1 || n_b > 1024) return wf_fail(WF_EINVAL, "wf_problem_set_band_scale: n_b = %d", n_b);
  const size_t nsp = (size_t)p->C * p->n * (p->nx / 2 + 1);
  const int ntab = p->sp_shared ? 1 : p->count;
  cudaStream_t st = (cudaStream_t)stream;
  if (!p->sp0) {
    wf_status s = wf_alloc(p->h, &p->sp0, nsp * ntab * p->elt, "unscaled sqrt(P) table");
    if (s != WF_OK) return s;
    cudaError_t e = cudaMemcpyAsync(p->sp0, p->sp, nsp * ntab * p->elt, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return wf_cuda_fail(e, "wf_problem_set_band_scale: copy");
  }
  cudaError_t e = WF_DISPATCH(p, wf_launch_band_scale)(p->g, p->sp0, p->sp, ntab, band, q, n_b, st);
  return e == cudaSuccess ? WF_OK : wf_cuda_fail(e, "wf_problem_set_band_scale");
}

extern "C" wf_status wf_eval_bands(wf_problem* p, const void* s, void* grad, double* chi2, const int16_t* band,
                                   int n_b, double* dlogq, void* stream) {
  if (!p || !s || !grad || !chi2 || !band || !dlogq) return wf_fail(WF_EINVAL, "wf_eval_bands: null argument");
  if (s == grad) return wf_fail(WF_EINVAL, "wf_eval_bands: s and grad must not alias");
  if (n_b < 1 || n_b > 1024) return wf_fail(WF_EINVAL, "wf_eval_bands: n_b = %d outside [1, 1024]", n_b);
  wf_status rs = band_partials(p, n_b);
  if (rs != WF_OK) return rs;
  WfBufs b = wf_bufs(p);
  cudaError_t e = WF_DISPATCH(p, wf_launch_eval_bands)(p->g, b, s, grad, chi2, band, n_b, p->bpart, dlogq,
                                                       (cudaStream_t)stream);
  return e == cudaSuccess ? WF_OK : wf_cuda_fail(e, "wf_eval_bands");
}

extern "C" wf_status wf_band_table_rect(int ny, int nx, int C, const double* edges, int n_bands, double kscale,
                                        int16_t* out) {
  if (!edges || !out) return wf_fail(WF_EINVAL, "wf_band_table: null argument");
  if (ny < 2 || (ny & 1) || nx < 2 || (nx & 1) || (C != 1 && C != 2))
    return wf_fail(WF_EINVAL, "wf_band_table: %d x %d, C = %d", ny, nx, C);
  if (n_bands < 1 || n_bands > 32767) return wf_fail(WF_EINVAL, "wf_band_table: n_bands = %d", n_bands);
  if (!(kscale > 0.0)) return wf_fail(WF_EINVAL, "wf_band_table: kscale must be > 0");
  for (int l = 0; l < n_bands; ++l)
    if (!(edges[l] < edges[l + 1])) return wf_fail(WF_EINVAL, "wf_band_table: edges must increase");
  const int h = nx / 2, N = ny > nx ? ny : nx;
  const double fx = (double)N / nx, fy = (double)N / ny;  // 1 when square
  for (int j = 0; j < ny; ++j) {
    const int ky = j < ny / 2 ? j : j - ny;
    for (int kx = 0; kx <= h; ++kx) {
      const double qx = fx * kx, qy = fy * ky;
      const double k = kscale * sqrt(qx * qx + qy * qy);
      int band = -1;
      if (k >= edges[0] && k < edges[n_bands]) {
        int lo = 0, hi = n_bands;  // edges[lo] <= k < edges[hi]
        while (hi - lo > 1) {
          const int mid = (lo + hi) / 2;
          if (k >= edges[mid]) lo = mid;
          else hi = mid;
        }
        band = lo;
      }
      for (int c = 0; c < C; ++c) out[((size_t)c * ny + j) * (h + 1) + kx] = (int16_t)band;
    }
  }
  return WF_OK;
}

extern "C" wf_status wf_band_table(int n, int C, const double* edges, int n_bands, double kscale, int16_t* out) {
  return wf_band_table_rect(n, n, C, edges, n_bands, kscale, out);
}

cudaError_t wf_dbg_selftest();

extern "C" wf_status wf_debug_bounds(unsigned long long* count, long long* first, int mode) {
  if (!count) return wf_fail(WF_EINVAL, "wf_debug_bounds: null count");
  *count = 0;
  if (mode < 0 || mode > 2) return wf_fail(WF_EINVAL, "wf_debug_bounds: mode = %d (0 read, 1 read and clear, 2 self-test)", mode);
#ifndef WF_DEBUG_BOUNDS
  (void)first;
  return wf_fail(WF_EINVAL, "wf_debug_bounds: this library was not built with bounds checks (WF_DEBUG_BOUNDS)");
#else
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && mode == 2) e = wf_dbg_selftest();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return wf_cuda_fail(e, "wf_debug_bounds");
  typedef cudaError_t (*Reader)(unsigned long long*, int);
#define WF_DBG_ENTRY(name) wf_dbg_read_##name,
  const Reader readers[] = {WF_DBG_TUS(WF_DBG_ENTRY)};
#undef WF_DBG_ENTRY
  bool have_first = false;
  for (int u = 0; u < (int)(sizeof readers / sizeof readers[0]); ++u) {
    unsigned long long rec[4];
    e = readers[u](rec, mode == 1);
    if (e != cudaSuccess) return wf_cuda_fail(e, "wf_debug_bounds: reading a record");
    *count += rec[0];
    if (rec[0] && !have_first && first) {
      first[0] = u;
      first[1] = (long long)rec[1];
      first[2] = (long long)rec[2];
      first[3] = (long long)rec[3];
      have_first = true;
    }
  }
  return WF_OK;
#endif
}
