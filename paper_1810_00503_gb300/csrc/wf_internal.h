// Internal declarations shared by the host API and the kernel translation units.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/wf.h"

#define WF_NT 1024          // largest transform length and twiddle-table size
#define WF_LOG2_NT 10

// Threads per block of every operator kernel and the most samples one thread
// stages in registers during an FFT pass; a tile holds at most their product.
#define WF_THREADS 256
#define WF_EMAX 16
#define WF_TILE (WF_THREADS * WF_EMAX)

// Partial-sum slots per map (one FP64 value per block and slot).
#define WF_SLOT_PRIOR 0
#define WF_SLOT_DATA 1
#define WF_SLOT_DOT0 2   // first of the L-BFGS dot-product slots
#define WF_MAXM 32
#define WF_NSLOT (WF_SLOT_DOT0 + 2 * WF_MAXM + 4)

// Launch geometry of one (n, C) shape.
struct WfGeo {
  int n, h, lgn, lgh, C;
  int TC, ntile;   // packed columns per column tile, tiles per map
  int RB, nrb;     // rows per row block (over the C*n rows), row blocks per map
  int maxblk;      // max(ntile, nrb): stride of the partial-sum slots
};

WfGeo wf_make_geo(int n, int C);

// Device pointers of one problem, in the working type T (float or double).
struct WfBufs {
  const void* d;      // [B][C][n][n]
  const void* w;      // [B][C][n][n]   mask * Ninv
  const void* sp;     // [B or 1][C][n][h+1]   sqrt(P) / n
  long long sp_stride;  // elements between maps' sqrt(P) tables (0 if shared)
  void* scratch;      // [B][C][n][h] complex: between the column and row stages
  double* part;       // [B][WF_NSLOT][maxblk]
  const void* tw;     // twiddle table, WF_NT complex of type T
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
                                  const double* theta, int n_bands, double* E, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_pack(const WfGeo& g, int B, const void* std_in, void* pk_out, cudaStream_t st);
template <typename T>
cudaError_t wf_launch_unpack(const WfGeo& g, int B, const void* pk_in, void* std_out, cudaStream_t st);
