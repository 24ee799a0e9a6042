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
//     k = 4 most frequent codes; in the main pass every 32-bit word (two
//     codes) is compared with each of the 4 codes at once (a packed 16-bit
//     equality), the matches are counted in four 32-bit registers per
//     thread, and only the other codes take a shared atomic -- so codes that
//     repeat do not serialize on one shared address.  Which codes are chosen
//     only moves work between the two paths: the counts are exact either
//     way.
//
// Both read the codes with 16-byte loads over a grid of a few CTAs per SM.
#include <string.h>

#include "fz_host.h"

namespace fz {
namespace {

constexpr int kHiThreads = 256;
constexpr int kHiWarps = kHiThreads / 32;
constexpr int kTopK = 4;
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
// consecutive codes spread evenly over the array) and writes its kTopK most
// frequent codes (ties to the lower code) to top[0..kTopK), 0xffff for a
// slot that the sample leaves empty.
__global__ void __launch_bounds__(kHiThreads) k_hist_sample(const uint16_t *__restrict__ codes, uint64_t n,
                                                            uint32_t nsym, uint16_t *top) {
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
  if (threadIdx.x < 32) {  // one warp picks the top codes by repeated arg-max
    const int lane = threadIdx.x;
    if (lane < kTopK) top[lane] = 0xffffu;
    __syncwarp();
    for (int k = 0; k < kTopK; ++k) {
      uint32_t best = 0, arg = 0xffffffffu;
      for (uint32_t s = lane; s < nsym; s += 32) {
        const uint32_t c = hs[s];
        if (c > best || (c == best && c > 0 && s < arg)) { best = c; arg = s; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const uint32_t b2 = __shfl_down_sync(0xffffffffu, best, off), a2 = __shfl_down_sync(0xffffffffu, arg, off);
        if (b2 > best || (b2 == best && a2 < arg)) { best = b2; arg = a2; }
      }
      arg = __shfl_sync(0xffffffffu, arg, 0);
      best = __shfl_sync(0xffffffffu, best, 0);
      if (best == 0 || arg == 0xffffffffu) break;  // fewer than kTopK codes seen
      if (lane == 0) {
        top[k] = (uint16_t)arg;
        hs[arg] = 0;  // not picked again
      }
      __syncwarp();
    }
  }
}

// The main pass: per 32-bit word (two codes), one packed 16-bit equality
// with each chosen code pair (c | c << 16) gives 0xffff per matching half;
// popcount / 16 over a thread's words is its count of that code.  Halves
// that match none take one shared atomic.  Chosen slots left empty (0xffff)
// are masked off.
__global__ void __launch_bounds__(kHiThreads) k_hist_topk(const uint16_t *__restrict__ codes, uint64_t n,
                                                          uint32_t nsym, const uint16_t *__restrict__ top_g,
                                                          unsigned long long *hist) {
  extern __shared__ uint32_t hs[];  // nsym counts
  for (uint32_t i = threadIdx.x; i < nsym; i += kHiThreads) hs[i] = 0;
  uint32_t pair[kTopK], en[kTopK], cnt[kTopK];
#pragma unroll
  for (int k = 0; k < kTopK; ++k) {
    const uint32_t c = __ldg(top_g + k);
    en[k] = c < nsym ? 0xffffffffu : 0u;
    pair[k] = c | (c << 16);
    cnt[k] = 0;
  }
  __syncthreads();
  bool bad = false;
  const uint64_t nv = n / 8;
  const uint4 *c4 = reinterpret_cast<const uint4 *>(codes);
  const uint64_t stride = (uint64_t)gridDim.x * kHiThreads;
  for (uint64_t v = (uint64_t)blockIdx.x * kHiThreads + threadIdx.x; v < nv; v += stride) {
    const uint4 w = __ldcs(c4 + v);
    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t hit = 0;
#pragma unroll
      for (int k = 0; k < kTopK; ++k) {
        const uint32_t m = __vcmpeq2(ww[q], pair[k]) & en[k];
        cnt[k] += __popc(m);
        hit |= m;
      }
      if (hit != 0xffffffffu) {  // a code that is none of the chosen ones
        const uint32_t a = ww[q] & 0xffffu, b2 = ww[q] >> 16;
        if (!(hit & 0xffffu)) {
          if (a < nsym) atomicAdd(hs + a, 1u); else bad = true;
        }
        if (!(hit >> 16)) {
          if (b2 < nsym) atomicAdd(hs + b2, 1u); else bad = true;
        }
      }
    }
  }
  for (uint64_t i = nv * 8 + (uint64_t)blockIdx.x * kHiThreads + threadIdx.x; i < n; i += stride) {
    const uint32_t a = codes[i];
    if (a < nsym) atomicAdd(hs + a, 1u);
    else bad = true;
  }
  // the chosen codes' counts: a warp sum per code, one shared atomic per warp
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < kTopK; ++k) {
    const uint32_t t = __reduce_add_sync(0xffffffffu, cnt[k] >> 4);
    if (lane == 0 && t) atomicAdd(hs + (pair[k] & 0xffffu), t);
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
  // and the chosen codes of the top-k method
  const size_t need = up(8 * (nsym + 1)) + up(2 * kTopK);
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
  uint16_t *top = reinterpret_cast<uint16_t *>(reinterpret_cast<uint8_t *>(ctx->ws) + up(8 * (nsym + 1)));
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
      k_hist_sample<<<1, kHiThreads, sizeof(uint32_t) * nsym, s>>>(d_codes, n, nsym, top);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_hist_topk<<<(unsigned)grid, kHiThreads, sizeof(uint32_t) * nsym, s>>>(d_codes, n, nsym, top, counts);
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
