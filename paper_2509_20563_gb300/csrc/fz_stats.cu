// fz_stats.cu -- reconstruction-quality statistics of a decompressed field
// against its original, for the rate-distortion evaluation of FZModules §4.2
// (bit rate = stream bits per value, PSNR from the value range and the mean
// squared error).  Two kernels: every CTA reduces a contiguous slice into one
// partial record (grid-stride over 16-byte loads, double accumulation), then
// one CTA adds the partials in index order, so the result does not depend on
// scheduling.  Non-finite originals count as mismatches unless the
// reconstruction carries the same bits (the method stores them verbatim).
#include <math.h>
#include <string.h>

#include "fz_host.h"

namespace fz {
namespace {

constexpr int kStThreads = 256;

struct Partial {
  double sse, max_err;
  uint32_t lo_key, hi_key;  // ordered keys of the finite minimum (inverted) and maximum
  unsigned long long n_finite, n_bad;
};

__device__ __forceinline__ void acc_one(float x, float y, double &sse, double &mx, uint32_t &lo, uint32_t &hi,
                                        unsigned long long &nf, unsigned long long &nb) {
  if (isfinite(x)) {
    const double d = (double)y - (double)x;
    sse += d * d;
    const double a = fabs(d);
    mx = a > mx || a != a ? a : mx;  // a NaN reconstruction of a finite value is an infinite error
    const uint32_t k = fkey(x);
    lo = max(lo, ~k);
    hi = max(hi, k);
    ++nf;
  } else if (__float_as_uint(x) != __float_as_uint(y)) {
    ++nb;
  }
}

__global__ void __launch_bounds__(kStThreads) k_stats_partial(const float *__restrict__ x,
                                                              const float *__restrict__ y, uint64_t n,
                                                              Partial *part) {
  double sse = 0.0, mx = 0.0;
  uint32_t lo = 0, hi = 0;
  unsigned long long nf = 0, nb = 0;
  const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint64_t b0 = (uint64_t)blockIdx.x * per, b1 = b0 + per < n ? b0 + per : n;
  // 16-byte loads where both pointers allow them, scalar head and tail
  const bool vec = (((uintptr_t)(x + b0) | (uintptr_t)(y + b0)) & 15u) == 0;
  uint64_t i = b0;
  if (vec) {
    const uint64_t nv = (b1 - b0) / 4;
    const float4 *x4 = reinterpret_cast<const float4 *>(x + b0);
    const float4 *y4 = reinterpret_cast<const float4 *>(y + b0);
    for (uint64_t v = threadIdx.x; v < nv; v += kStThreads) {
      const float4 a = __ldcs(x4 + v), b = __ldcs(y4 + v);
      acc_one(a.x, b.x, sse, mx, lo, hi, nf, nb);
      acc_one(a.y, b.y, sse, mx, lo, hi, nf, nb);
      acc_one(a.z, b.z, sse, mx, lo, hi, nf, nb);
      acc_one(a.w, b.w, sse, mx, lo, hi, nf, nb);
    }
    i = b0 + 4 * nv;
  }
  for (uint64_t k = i + threadIdx.x; k < b1; k += kStThreads) acc_one(x[k], y[k], sse, mx, lo, hi, nf, nb);
  // CTA reduction in a fixed order: warp shuffles, then warp 0 over the warps
  __shared__ Partial s[kStThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    sse += __shfl_down_sync(0xffffffffu, sse, off);
    const double m2 = __shfl_down_sync(0xffffffffu, mx, off);
    mx = m2 > mx || m2 != m2 ? m2 : mx;
    lo = max(lo, __shfl_down_sync(0xffffffffu, lo, off));
    hi = max(hi, __shfl_down_sync(0xffffffffu, hi, off));
    nf += __shfl_down_sync(0xffffffffu, nf, off);
    nb += __shfl_down_sync(0xffffffffu, nb, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s[warp] = Partial{sse, mx, lo, hi, nf, nb};
  __syncthreads();
  if (threadIdx.x == 0) {
    Partial r = s[0];
    for (int w = 1; w < kStThreads / 32; ++w) {
      r.sse += s[w].sse;
      r.max_err = s[w].max_err > r.max_err || s[w].max_err != s[w].max_err ? s[w].max_err : r.max_err;
      r.lo_key = max(r.lo_key, s[w].lo_key);
      r.hi_key = max(r.hi_key, s[w].hi_key);
      r.n_finite += s[w].n_finite;
      r.n_bad += s[w].n_bad;
    }
    part[blockIdx.x] = r;
  }
}

// One thread adds the partials in index order.
__global__ void k_stats_final(const Partial *part, uint32_t n_part, fz_error_report *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Partial r = part[0];
  for (uint32_t i = 1; i < n_part; ++i) {
    r.sse += part[i].sse;
    r.max_err = part[i].max_err > r.max_err || part[i].max_err != part[i].max_err ? part[i].max_err : r.max_err;
    r.lo_key = max(r.lo_key, part[i].lo_key);
    r.hi_key = max(r.hi_key, part[i].hi_key);
    r.n_finite += part[i].n_finite;
    r.n_bad += part[i].n_bad;
  }
  out->max_abs_err = r.max_err;
  out->sse = r.sse;
  out->x_min = r.n_finite ? (double)fkey_inv(~r.lo_key) : 0.0;
  out->x_max = r.n_finite ? (double)fkey_inv(r.hi_key) : 0.0;
  out->n_finite = r.n_finite;
  out->n_nonfinite_mismatch = r.n_bad;
}

}  // namespace
}  // namespace fz

using namespace fz;

extern "C" fz_status fz_error_stats(fz_ctx *ctx, const float *d_x, const float *d_y, uint64_t n,
                                    fz_error_report *out, void *stream) {
  if (!ctx || !d_x || !d_y || !out || n == 0) return FZ_EINVAL;
  if (((uintptr_t)d_x & 3u) || ((uintptr_t)d_y & 3u)) return FZ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
  uint64_t grid = (n + 4095) / 4096;
  const uint64_t cap = (uint64_t)ctx->sm_count * 4;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  // the context workspace holds the partials and the report
  const size_t need = up(sizeof(Partial) * grid) + up(sizeof(fz_error_report));
  if (ctx->ws_bytes < need) {
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
    if (cudaMalloc(&ctx->ws, need) != cudaSuccess) {
      cudaGetLastError();
      return FZ_ENOMEM;
    }
    ctx->ws_bytes = need;
  }
  Partial *part = reinterpret_cast<Partial *>(ctx->ws);
  fz_error_report *dev_out = reinterpret_cast<fz_error_report *>(reinterpret_cast<char *>(ctx->ws) +
                                                                 up(sizeof(Partial) * grid));
  k_stats_partial<<<(unsigned)grid, kStThreads, 0, s>>>(d_x, d_y, n, part);
  k_stats_final<<<1, 32, 0, s>>>(part, (uint32_t)grid, dev_out);
  ctx->launches += 2;
  fz_error_report r;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&r, dev_out, sizeof(r), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  // PSNR over the finite values: 20 log10(value range) - 10 log10(MSE)
  const double mse = r.n_finite ? r.sse / (double)r.n_finite : 0.0;
  const double range = r.x_max - r.x_min;
  r.psnr_db = (mse > 0.0 && range > 0.0) ? 20.0 * log10(range) - 10.0 * log10(mse) : INFINITY;
  *out = r;
  return FZ_OK;
}
