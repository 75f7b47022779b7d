// Host-side structures of the C ABI (handle, prepared problem, solver state).
#pragma once
#include <mutex>
#include <unordered_map>
#include "wf_internal.h"

struct wf_handle {
  int device;
  void* tw64;   // WF_TWTAB_ALL double2 twiddles (roots of unity, pass tables of every plan)
  void* tw32;   // WF_TWTAB_ALL float2 twiddles
  size_t limit;  // workspace limit in bytes (0 = none)
  size_t used;   // device bytes held by this handle's allocations
  std::mutex mu;
  std::unordered_map<void*, size_t> live;  // allocation -> bytes
  std::unordered_map<long long, int> tuned;  // (ny, nx, C, precision, maps) -> FFT-stage variant
};

struct WfSolver;  // L-BFGS state, allocated on the first solve (wf_solve.cu)

struct wf_problem {
  wf_handle* h;
  int count, n, nx, C, dtype, precision, m;  // n = ny rows of nx pixels
  WfGeo g;
  size_t elt;            // bytes of the working type
  int sp_shared;         // one sqrt(P) table serves every map
  long long sp_stride;   // elements between maps' sqrt(P) tables
  void* d;               // [count][C][ny][nx] working type
  void* w;               // [count][C][ny][nx] mask * Ninv
  void* sp;              // [1 or count][C][ny][nx/2+1] sqrt(P/(ny nx)) (band-scaled if set)
  void* sp0;             // unscaled copy, kept once a band scale has been set
  void* scratch;         // [count][C][ny][nx/2] complex
  double* part;          // [count][WF_NSLOT][maxblk]
  int* flags;            // device status words
  double* bpart;         // band-sum partials [count][blocks][bands] (grown on demand)
  size_t bpart_n;        // doubles held by bpart
  WfSolver* solver;
};

wf_status wf_fail(wf_status s, const char* fmt, ...);
wf_status wf_cuda_fail(cudaError_t e, const char* what);
// Device allocation charged to the handle's workspace (WF_ENOMEM beyond its
// limit), and its release; wf_free(h, nullptr) does nothing.
wf_status wf_alloc(wf_handle* h, void** ptr, size_t bytes, const char* what);
void wf_free(wf_handle* h, void* ptr);
WfBufs wf_bufs(const wf_problem* p);
void wf_solver_free(wf_problem* p);
void wf_make_twiddles(double2* out);  // WF_TWTAB entries: roots of unity and pass tables
// Normal deviates offset .. offset + count - 1 of (seed, stream_id) into out
// (working type); scaled by w^-1/2 where w > 0 and zeroed elsewhere if w given.
wf_status wf_draw_normal(unsigned long long seed, unsigned stream_id, unsigned long long offset, size_t count,
                         int working_f64, void* out, const void* w, cudaStream_t st);
