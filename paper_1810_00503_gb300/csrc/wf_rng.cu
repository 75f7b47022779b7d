// Normal deviates drawn on the device for the band-power simulations
// (Sec. 2.5: white signal fields z_j, noise n_j with covariance N, white fields
// of the Fisher signals).
//
// Generator: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
// (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with the key bumped by (0x9E3779B9, 0xBB67AE85) between rounds.  Deviate i of
// (seed, stream) comes from block j = i / 2: counter (j mod 2^32, j div 2^32,
// stream, 0), key (seed mod 2^32, seed div 2^32); the four words give two 53-bit
// uniforms u1, u2 in (0, 1) and the Box-Muller pair r (cos, sin)(2 pi u2),
// r = sqrt(-2 ln u1), deviate 2j the cosine and 2j + 1 the sine.
#include <math.h>

#include "wf_api_internal.h"

__device__ __forceinline__ void wf_philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, uint32_t k0,
                                                 uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
}

// out[k] = deviate (offset + k) of (seed, stream), k < count; with w given,
// scaled by w[k]^-1/2 where w[k] > 0 and set to 0 elsewhere (noise of
// variance 1/Ninv on observed pixels).
template <typename T>
__global__ void k_normal(unsigned long long seed, uint32_t stream, unsigned long long offset, unsigned long long count,
                         T* out, const T* w) {
  const unsigned long long j0 = offset >> 1, j1 = (offset + count - 1) >> 1;
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long j = j0 + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j <= j1; j += step) {
    uint32_t c0 = (uint32_t)j, c1 = (uint32_t)(j >> 32), c2 = stream, c3 = 0u;
    wf_philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u1 = ((double)(c0 >> 5) * 67108864.0 + (double)(c1 >> 6) + 0.5) * 0x1p-53;
    const double u2 = ((double)(c2 >> 5) * 67108864.0 + (double)(c3 >> 6) + 0.5) * 0x1p-53;
    const double r = sqrt(-2.0 * log(u1)), th = 2.0 * M_PI * u2;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const unsigned long long i = 2 * j + q;
      if (i < offset || i >= offset + count) continue;
      const unsigned long long k = i - offset;
      double z = q == 0 ? r * cos(th) : r * sin(th);
      if (w) {
        const double wv = (double)w[k];
        z = wv > 0.0 ? z / sqrt(wv) : 0.0;
      }
      out[k] = (T)z;
    }
  }
}

wf_status wf_draw_normal(unsigned long long seed, unsigned stream_id, unsigned long long offset, size_t count,
                         int working_f64, void* out, const void* w, cudaStream_t st) {
  if (count == 0) return WF_OK;
  const unsigned long long blocks_needed = ((offset + count - 1) >> 1) - (offset >> 1) + 1;
  unsigned long long grid = (blocks_needed + 255) / 256;
  if (grid > 8192) grid = 8192;
  if (working_f64)
    k_normal<double><<<(unsigned)grid, 256, 0, st>>>(seed, stream_id, offset, count, (double*)out, (const double*)w);
  else
    k_normal<float><<<(unsigned)grid, 256, 0, st>>>(seed, stream_id, offset, count, (float*)out, (const float*)w);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WF_OK : wf_cuda_fail(e, "normal deviates");
}

extern "C" wf_status wf_normal_draw(unsigned long long seed, unsigned int stream_id, unsigned long long offset,
                                    size_t count, int dtype, void* out, void* stream) {
  if (!out && count > 0) return wf_fail(WF_EINVAL, "wf_normal_draw: null output");
  if (dtype != WF_F32 && dtype != WF_F64) return wf_fail(WF_EINVAL, "wf_normal_draw: bad dtype %d", dtype);
  if (offset + count < offset) return wf_fail(WF_EINVAL, "wf_normal_draw: offset + count overflows");
  return wf_draw_normal(seed, stream_id, offset, count, dtype == WF_F64, out, nullptr, (cudaStream_t)stream);
}
