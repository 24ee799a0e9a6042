// fz_hist.cu -- the histogram module of FZModules §3.2 as a stage of its
// own: counts of every code of a quantization-code array, by one of two
// methods that give the same (exact) counts.
//
//   FZ_HIST_PRIVATE -- every warp of a CTA owns a shared-memory copy of the
//     histogram and counts each code with one shared atomic; the copies are
//     added up per CTA and flushed to the global counts.
//   FZ_HIST_TOPK -- the top-k variant (§3.2: better when the codes repeat a
//     few values, as after a good predictor).  A one-CTA pass counts a
//     sample (64 windows of 1024 codes spread over the array) and keeps its
//     k = 16 most frequent codes; in the main
//     pass each thread counts those 16 codes in two 64-bit registers of
//     eight 8-bit counters (an add of 1 << 8 slot), folded into shared
//     memory every 255 codes, and only the other codes take a shared
//     atomic.  Which codes are chosen only moves work between the two
//     paths: the counts are exact either way.
//
// Both read the codes with 16-byte loads over a grid of a few CTAs per SM.
#include <string.h>

#include "fz_host.h"

namespace fz {
namespace {

constexpr int kHiThreads = 256;
constexpr int kHiWarps = kHiThreads / 32;
constexpr int kTopK = 16;
constexpr uint32_t kSampleWindows = 64, kSampleWindow = 1024;  // 64K codes in 64 evenly spread windows

// Warp-private shared histograms; n a multiple of 8 codes is read as uint4.
__global__ void __launch_bounds__(kHiThreads) k_hist_private(const uint16_t *__restrict__ codes, uint64_t n,
                                                             uint32_t nsym, unsigned long long *hist) {
  extern __shared__ uint32_t hs[];  // kHiWarps x nsym
  for (uint32_t i = threadIdx.x; i < kHiWarps * nsym; i += kHiThreads) hs[i] = 0;
  __syncthreads();
  uint32_t *mine = hs + (threadIdx.x >> 5) * nsym;
  const uint64_t nv = n / 8;
  const uint4 *c4 = reinterpret_cast<const uint4 *>(codes);
  bool bad = false;
  for (uint64_t v = (uint64_t)blockIdx.x * kHiThreads + threadIdx.x; v < nv; v += (uint64_t)gridDim.x * kHiThreads) {
    const uint4 w = __ldcs(c4 + v);
    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t a = ww[k] & 0xffffu, b = ww[k] >> 16;
      bad |= a >= nsym || b >= nsym;
      if (a < nsym) atomicAdd(mine + a, 1u);
      if (b < nsym) atomicAdd(mine + b, 1u);
    }
  }
  for (uint64_t i = nv * 8 + (uint64_t)blockIdx.x * kHiThreads + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * kHiThreads) {
    const uint32_t a = codes[i];
    bad |= a >= nsym;
    if (a < nsym) atomicAdd(mine + a, 1u);
  }
  __syncthreads();
  for (uint32_t s = threadIdx.x; s < nsym; s += kHiThreads) {
    unsigned long long t = 0;
    for (int w = 0; w < kHiWarps; ++w) t += hs[w * nsym + s];
    if (t) atomicAdd(hist + s, t);
  }
  if (bad) atomicAdd(hist + nsym, 1ull);  // codes outside the alphabet: counted apart
}

// One CTA: counts a sample of at most 64K codes (64 windows of 1024
// consecutive codes spread evenly over the array, read coalesced) and
// writes the 16 most frequent codes (ties to the lower code) into slot[] as
// a code -> slot table (0xff: none).
__global__ void __launch_bounds__(kHiThreads) k_hist_sample(const uint16_t *__restrict__ codes, uint64_t n,
                                                            uint32_t nsym, uint8_t *slot) {
  extern __shared__ uint32_t hs[];  // nsym
  for (uint32_t i = threadIdx.x; i < nsym; i += kHiThreads) hs[i] = 0;
  __syncthreads();
  // window starts at multiples of 8 codes (16-byte aligned: the array is),
  // each thread's 32 loads of 8 codes issued before any is counted
  const uint64_t span = n > kSampleWindow ? ((n - kSampleWindow) / (kSampleWindows - 1)) & ~7ull : 0;
  constexpr int kPer = kSampleWindows * kSampleWindow / 8 / kHiThreads;  // uint4 loads per thread
  const uint4 *c4 = reinterpret_cast<const uint4 *>(codes);
  uint4 v[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const uint32_t i = threadIdx.x + k * kHiThreads;  // uint4 index within the sample
    const uint64_t pos = (uint64_t)(i / (kSampleWindow / 8)) * span + 8ull * (i % (kSampleWindow / 8));
    v[k] = pos + 8 <= n ? __ldg(c4 + pos / 8) : make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
  }
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const uint32_t ww[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const uint32_t a = (ww[h >> 1] >> (16 * (h & 1))) & 0xffffu;
      if (a < nsym) atomicAdd(hs + a, 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // one warp picks the top 16 by repeated arg-max
    const int lane = threadIdx.x;
    for (uint32_t s = lane; s < nsym; s += 32) slot[s] = 0xff;
    __syncwarp();
    for (int k = 0; k < kTopK; ++k) {
      uint32_t best = 0, arg = 0xffffffffu;
      for (uint32_t s = lane; s < nsym; s += 32) {
        const uint32_t c = hs[s];
        if (slot[s] == 0xff && (c > best || (c == best && c > 0 && s < arg))) { best = c; arg = s; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const uint32_t b2 = __shfl_down_sync(0xffffffffu, best, off), a2 = __shfl_down_sync(0xffffffffu, arg, off);
        if (b2 > best || (b2 == best && a2 < arg)) { best = b2; arg = a2; }
      }
      arg = __shfl_sync(0xffffffffu, arg, 0);
      best = __shfl_sync(0xffffffffu, best, 0);
      if (best == 0 || arg == 0xffffffffu) break;  // fewer than 16 codes seen
      if (lane == 0) slot[arg] = (uint8_t)k;
      __syncwarp();
    }
  }
}

// Adds the 16 packed byte counters of every thread of the CTA into the
// shared counts of their codes (warp reductions, one lane adds).
__device__ __forceinline__ void fold_topk(unsigned long long &lo, unsigned long long &hi, const uint16_t *topsym,
                                          uint32_t *hs) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < kTopK; ++k) {
    const uint32_t c = (uint32_t)(((k < 8 ? lo : hi) >> (8 * (k & 7))) & 0xffu);
    const uint32_t t = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0 && t) atomicAdd(hs + topsym[k], t);
  }
  lo = 0;
  hi = 0;
}

__global__ void __launch_bounds__(kHiThreads) k_hist_topk(const uint16_t *__restrict__ codes, uint64_t n,
                                                          uint32_t nsym, const uint8_t *__restrict__ slot_g,
                                                          unsigned long long *hist) {
  extern __shared__ uint32_t hs[];            // nsym counts
  uint8_t *slot = reinterpret_cast<uint8_t *>(hs + nsym);  // nsym code -> slot
  __shared__ uint16_t topsym[kTopK];
  for (uint32_t i = threadIdx.x; i < nsym; i += kHiThreads) {
    hs[i] = 0;
    const uint8_t sl = slot_g[i];
    slot[i] = sl;
    if (sl < kTopK) topsym[sl] = (uint16_t)i;
  }
  if (threadIdx.x < kTopK) {
    // slots the sample left empty point at code 0, whose counter stays 0
    bool used = false;
    for (uint32_t i = 0; i < nsym; ++i) used |= slot_g[i] == threadIdx.x;
    if (!used) topsym[threadIdx.x] = 0;
  }
  __syncthreads();
  unsigned long long lo = 0, hi = 0;
  bool bad = false;
  const uint64_t nv = n / 8;
  const uint4 *c4 = reinterpret_cast<const uint4 *>(codes);
  // every thread runs the same number of iterations so that the warp-wide
  // folds line up; iterations past the end count nothing
  const uint64_t stride = (uint64_t)gridDim.x * kHiThreads;
  const uint64_t iters = (nv + stride - 1) / stride;
  uint32_t since = 0;
  for (uint64_t it = 0; it < iters; ++it) {
    const uint64_t v = it * stride + (uint64_t)blockIdx.x * kHiThreads + threadIdx.x;
    if (v < nv) {
      const uint4 w = __ldcs(c4 + v);
      const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const uint32_t a = (ww[k >> 1] >> (16 * (k & 1))) & 0xffffu;
        if (a >= nsym) { bad = true; continue; }
        const uint32_t sl = slot[a];
        if (sl < 8) lo += 1ull << (8 * sl);
        else if (sl < kTopK) hi += 1ull << (8 * (sl - 8));
        else atomicAdd(hs + a, 1u);
      }
    }
    since += 8;
    if (since > 255 - 8) {  // before any 8-bit counter can overflow
      fold_topk(lo, hi, topsym, hs);
      since = 0;
    }
  }
  fold_topk(lo, hi, topsym, hs);
  for (uint64_t i = nv * 8 + (uint64_t)blockIdx.x * kHiThreads + threadIdx.x; i < n; i += stride) {
    const uint32_t a = codes[i];
    if (a < nsym) atomicAdd(hs + a, 1u);
    else bad = true;
  }
  __syncthreads();
  for (uint32_t s = threadIdx.x; s < nsym; s += kHiThreads)
    if (hs[s]) atomicAdd(hist + s, (unsigned long long)hs[s]);
  if (bad) atomicAdd(hist + nsym, 1ull);
}

}  // namespace
}  // namespace fz

using namespace fz;

extern "C" fz_status fz_histogram(fz_ctx *ctx, const uint16_t *d_codes, uint64_t n, uint32_t nsym, uint32_t method,
                                  uint64_t *d_hist, void *stream) {
  if (!ctx || !d_codes || !d_hist || n == 0 || nsym == 0 || nsym > (uint32_t)kMaxSym) return FZ_EINVAL;
  if (method != FZ_HIST_PRIVATE && method != FZ_HIST_TOPK) return FZ_EINVAL;
  if ((uintptr_t)d_codes & 15u) return FZ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
  // workspace: the counts (nsym + 1 words, the last one flags codes >= nsym)
  // and the code -> slot table of the top-k method
  const size_t need = up(8 * (nsym + 1)) + up(nsym);
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
  if (!ctx->h_pinned && cudaMallocHost(&ctx->h_pinned, sizeof(Result) + 64) != cudaSuccess) {
    cudaGetLastError();
    ctx->h_pinned = nullptr;
    return FZ_ENOMEM;
  }
  unsigned long long *counts = reinterpret_cast<unsigned long long *>(ctx->ws);
  uint8_t *slot = reinterpret_cast<uint8_t *>(ctx->ws) + up(8 * (nsym + 1));
  uint64_t grid = (n / 8 + kHiThreads - 1) / kHiThreads;
  const uint64_t cap = (uint64_t)ctx->sm_count * 4;
  if (grid > cap) grid = cap;
  if (grid < 1) grid = 1;
  cudaError_t e = cudaMemsetAsync(counts, 0, 8 * (nsym + 1), s);
  if (method == FZ_HIST_PRIVATE) {
    const int smem = (int)(sizeof(uint32_t) * kHiWarps * nsym);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_hist_private, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) {
      k_hist_private<<<(unsigned)grid, kHiThreads, smem, s>>>(d_codes, n, nsym, counts);
      e = cudaGetLastError();
    }
    ctx->launches += 1;
  } else {
    if (e == cudaSuccess) {
      k_hist_sample<<<1, kHiThreads, sizeof(uint32_t) * nsym, s>>>(d_codes, n, nsym, slot);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_hist_topk<<<(unsigned)grid, kHiThreads, sizeof(uint32_t) * nsym + nsym, s>>>(d_codes, n, nsym, slot, counts);
      e = cudaGetLastError();
    }
    ctx->launches += 2;
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_hist, counts, 8 * (size_t)nsym, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_pinned, counts + nsym, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  uint64_t out_of_range = 0;
  memcpy(&out_of_range, ctx->h_pinned, 8);
  return out_of_range ? FZ_EINVAL : FZ_OK;
}
