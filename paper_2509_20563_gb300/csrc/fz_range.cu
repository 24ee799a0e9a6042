// fz_range.cu -- value-range preprocessing (FZModules §3.2): the minimum and
// maximum over the finite values of the field, reduced in one HBM pass, and a
// one-thread tail (last CTA to finish) that turns the bound into the float32
// constants of the quantizer.  ABS mode runs only the tail.
#include "fz_internal.cuh"

namespace fz {

namespace {

constexpr int kRangeThreads = 512;

struct Acc {
  uint32_t lo_nkey, hi_key, bits_nmin, bits_max, any;
  __device__ void init() { lo_nkey = hi_key = bits_nmin = bits_max = any = 0; }
  __device__ void add(float v) {
    uint32_t b = __float_as_uint(v);
    bits_nmin = max(bits_nmin, ~b);
    bits_max = max(bits_max, b);
    if (isfinite(v)) {
      uint32_t k = fkey(v);
      lo_nkey = max(lo_nkey, ~k);
      hi_key = max(hi_key, k);
      any = 1;
    }
  }
  __device__ void merge(const Acc &o) {
    lo_nkey = max(lo_nkey, o.lo_nkey);
    hi_key = max(hi_key, o.hi_key);
    bits_nmin = max(bits_nmin, o.bits_nmin);
    bits_max = max(bits_max, o.bits_max);
    any |= o.any;
  }
  __device__ void shfl_merge(int off) {
    Acc o;
    o.lo_nkey = __shfl_down_sync(0xffffffffu, lo_nkey, off);
    o.hi_key = __shfl_down_sync(0xffffffffu, hi_key, off);
    o.bits_nmin = __shfl_down_sync(0xffffffffu, bits_nmin, off);
    o.bits_max = __shfl_down_sync(0xffffffffu, bits_max, off);
    o.any = __shfl_down_sync(0xffffffffu, any, off);
    merge(o);
  }
};

// Decide the stream mode from the range and derive the constants.
__device__ void range_tail(Ctl *ctl, uint32_t eb_mode, double eb) {
  if (eb_mode == FZ_EB_REL) {
    uint32_t any = ctl->any_finite;
    float lo = fkey_inv(~ctl->lo_nkey), hi = fkey_inv(ctl->hi_key);
    if (!any || hi == lo) {
      uint32_t bmin = ~ctl->bits_nmin, bmax = ctl->bits_max;
      ctl->mode = (bmin == bmax) ? kModeConst : kModeRaw;
      ctl->const_bits = bmax;
      ctl->eb_abs = 0.0;
      return;
    }
    double range = __dsub_rn((double)hi, (double)lo);
    ctl->eb_abs = __dmul_rn(eb, range);
  } else {
    ctl->eb_abs = eb;
  }
  float a, b, c;
  device_constants(ctl->eb_abs, a, b, c);
  ctl->ebx2 = a;
  ctl->inv2eb = b;
  ctl->eb_chk = c;
  ctl->mode = kModeNormal;
}

__global__ void __launch_bounds__(kRangeThreads) k_range(const float *__restrict__ x, uint64_t n, Ctl *ctl,
                                                          uint32_t eb_mode, double eb) {
  dep_trigger();  // the quantizer's first loads (of the input) may start
  Acc a;
  a.init();
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  if (((uintptr_t)x & 15u) == 0) {
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const uint64_t n4 = n / 4;
    uint64_t i = tid;
    // four independent 16-byte loads in flight per thread
    for (; i + 3 * nth < n4; i += 4 * nth) {
      float4 v0 = __ldcs(x4 + i), v1 = __ldcs(x4 + i + nth), v2 = __ldcs(x4 + i + 2 * nth),
             v3 = __ldcs(x4 + i + 3 * nth);
      a.add(v0.x); a.add(v0.y); a.add(v0.z); a.add(v0.w);
      a.add(v1.x); a.add(v1.y); a.add(v1.z); a.add(v1.w);
      a.add(v2.x); a.add(v2.y); a.add(v2.z); a.add(v2.w);
      a.add(v3.x); a.add(v3.y); a.add(v3.z); a.add(v3.w);
    }
    for (; i < n4; i += nth) {
      float4 v = __ldcs(x4 + i);
      a.add(v.x); a.add(v.y); a.add(v.z); a.add(v.w);
    }
    for (uint64_t j = n4 * 4 + tid; j < n; j += nth) a.add(x[j]);
  } else {
    for (uint64_t j = tid; j < n; j += nth) a.add(x[j]);
  }
  for (int off = 16; off > 0; off >>= 1) a.shfl_merge(off);
  __shared__ Acc sh[kRangeThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = a;
  __syncthreads();
  if (warp == 0) {
    a.init();
    if (lane < kRangeThreads / 32) a = sh[lane];
    for (int off = 16; off > 0; off >>= 1) a.shfl_merge(off);
    if (lane == 0) {
      atomicMax(&ctl->lo_nkey, a.lo_nkey);
      atomicMax(&ctl->hi_key, a.hi_key);
      atomicMax(&ctl->bits_nmin, a.bits_nmin);
      atomicMax(&ctl->bits_max, a.bits_max);
      if (a.any) atomicOr(&ctl->any_finite, 1u);
      __threadfence();
      unsigned int done = atomicAdd(&ctl->range_done, 1u);
      if (done == gridDim.x - 1) {
        __threadfence();
        range_tail(ctl, eb_mode, eb);
      }
    }
  }
}

__global__ void k_constants_abs(Ctl *ctl, double eb) { range_tail(ctl, FZ_EB_ABS, eb); }

// Batched variant: every REL field is cut into segments of 2^seg_log2
// values (an ABS field is one empty segment), and the segments of all
// fields form one queue.  The CTA that finishes a field's last segment runs
// that field's tail.
__global__ void __launch_bounds__(kRangeThreads) k_range_batch(const BatchJob *__restrict__ jobs, uint32_t n,
                                                                uint64_t total_segs, int seg_log2) {
  __shared__ Acc sh[kRangeThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t sgi = blockIdx.x; sgi < total_segs; sgi += gridDim.x) {
    uint32_t a = 0, b = n;  // the field whose segments contain sgi
    while (a < b) {
      const uint32_t m = (a + b) >> 1;
      if (jobs[m].range_base + jobs[m].range_segs <= sgi) a = m + 1; else b = m;
    }
    const BatchJob &J = jobs[a];
    Acc acc;
    acc.init();
    if (J.eb_mode == FZ_EB_REL) {
      const uint64_t lo = (sgi - J.range_base) << seg_log2;
      uint64_t hi = lo + (1ull << seg_log2);
      if (hi > J.g.n) hi = J.g.n;
      const float *x = J.x;
      if (((uintptr_t)x & 15u) == 0) {
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        const uint64_t a4 = lo / 4, b4 = hi / 4;  // lo is a multiple of 4
        for (uint64_t i = a4 + threadIdx.x; i < b4; i += kRangeThreads) {
          const float4 v = __ldcs(x4 + i);
          acc.add(v.x); acc.add(v.y); acc.add(v.z); acc.add(v.w);
        }
        for (uint64_t j = b4 * 4 + threadIdx.x; j < hi; j += kRangeThreads) acc.add(x[j]);
      } else {
        for (uint64_t j = lo + threadIdx.x; j < hi; j += kRangeThreads) acc.add(x[j]);
      }
    }
    for (int off = 16; off > 0; off >>= 1) acc.shfl_merge(off);
    if (lane == 0) sh[warp] = acc;
    __syncthreads();
    if (warp == 0) {
      acc.init();
      if (lane < kRangeThreads / 32) acc = sh[lane];
      for (int off = 16; off > 0; off >>= 1) acc.shfl_merge(off);
      if (lane == 0) {
        Ctl *ctl = J.ws.ctl;
        atomicMax(&ctl->lo_nkey, acc.lo_nkey);
        atomicMax(&ctl->hi_key, acc.hi_key);
        atomicMax(&ctl->bits_nmin, acc.bits_nmin);
        atomicMax(&ctl->bits_max, acc.bits_max);
        if (acc.any) atomicOr(&ctl->any_finite, 1u);
        __threadfence();
        const unsigned int done = atomicAdd(&ctl->range_done, 1u);
        if (done == J.range_segs - 1) {
          __threadfence();
          range_tail(ctl, J.eb_mode, J.eb);
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_range_batch(const BatchJob *jobs, uint32_t n, uint64_t total_segs, int seg_log2, cudaStream_t s,
                               int sm_count) {
  uint64_t grid = (uint64_t)sm_count * 4;
  if (grid > total_segs) grid = total_segs;
  if (grid < 1) grid = 1;
  k_range_batch<<<(unsigned)grid, kRangeThreads, 0, s>>>(jobs, n, total_segs, seg_log2);
  return cudaGetLastError();
}

cudaError_t launch_range(const float *x, const Geom &g, uint32_t eb_mode, double eb, Ctl *ctl, cudaStream_t s) {
  if (eb_mode == FZ_EB_ABS) {
    k_constants_abs<<<1, 1, 0, s>>>(ctl, eb);
    return cudaGetLastError();
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t want = (g.n / 4 + kRangeThreads * 4 - 1) / (kRangeThreads * 4);
  uint64_t grid = (uint64_t)sms * 4;
  if (want < grid) grid = want > 0 ? want : 1;
  k_range<<<(unsigned)grid, kRangeThreads, 0, s>>>(x, g.n, ctl, eb_mode, eb);
  return cudaGetLastError();
}

}  // namespace fz
