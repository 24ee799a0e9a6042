// fz_decode_common.cuh -- pieces shared by the decoders: the decode table
// format, the asynchronous per-thread bit reader and small helpers.
#pragma once

#include "fz_internal.cuh"

namespace fz {

constexpr int kLutSize = 1 << kLutBits;
// decode-table entry: bit 15 valid, bits 10..13 length-1, bits 0..9 symbol
constexpr uint16_t kLutValid = 0x8000u;

__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void cp_async4(uint32_t *dst_smem, const uint32_t *src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
  const int n = valid ? 4 : 0;  // zero-fill past the end of the bitstream
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait3() { asm volatile("cp.async.wait_group 3;\n" ::: "memory"); }

constexpr int kRing = 4;  // stream words in flight per thread

// MSB-first bit reader over one chunk, all 32-bit: a window of two stream
// words (a, b) and a bit offset into a; the next 32 bits are one funnel shift
// away.  When the offset passes 32 the window slides by a word.  The words
// ahead of the window wait in a per-thread ring in shared memory, filled by
// asynchronous copies issued four slides early, so a slide never waits on
// memory and no register is ever read while its load is in flight.  Words
// past the end of the bitstream read as zero.
struct BitReader {
  const uint32_t *W;   // the chunk's first word
  uint32_t nw;         // words from W to the end of the bitstream
  uint32_t wi;         // next word to fetch into the ring, relative to W
  uint32_t *ring;      // this thread's ring: ring[k * kDecThreads]
  uint32_t rd;         // next ring slot to read
  uint32_t a, b;
  uint32_t off;        // bits of a already consumed (0..31)
  uint32_t vall;       // AND of all table entries used (valid bit check)
  __device__ __forceinline__ uint32_t ld(uint32_t i) const { return i < nw ? __ldg(W + i) : 0u; }
  __device__ __forceinline__ void init(const uint32_t *words, uint64_t n_words, uint64_t bitpos, uint32_t bits,
                                       uint32_t *ring_col) {
    const uint64_t sw = bitpos >> 5;
    W = words + sw;
    nw = (uint32_t)(n_words > sw ? (n_words - sw < 0xffffffffull ? n_words - sw : 0xffffffffull) : 0);
    off = (uint32_t)(bitpos & 31u);
    ring = ring_col;
    a = ld(0);
    b = ld(1);
#pragma unroll
    for (int k = 0; k < kRing; ++k) cp_async4(ring + k * kDecThreads, W + (2 + k < nw ? 2 + k : 0), 2 + k < nw);
    wi = 2 + kRing;
    rd = 0;
    vall = 0xffffffffu;
    // the whole chunk (a few 128-byte lines) is pulled into L2 up front
    const uint32_t cw = (off + bits + 31) / 32 + 2;
    for (uint32_t i = 32; i < cw && i < nw; i += 32) prefetch_l2(W + i);
  }
  __device__ __forceinline__ uint32_t next(const uint16_t *slut) {
    const uint32_t win = __funnelshift_l(b, a, off);
    const uint32_t e = slut[win >> (32 - kLutBits)];
    vall &= e;
    off += ((e >> 10) & 15u) + 1u;
    if (off >= 32) {
      off -= 32;
      cp_async_wait3();
      a = b;
      b = ring[rd * kDecThreads];
      cp_async4(ring + rd * kDecThreads, W + (wi < nw ? wi : 0), wi < nw);
      rd = (rd + 1) & (kRing - 1);
      ++wi;
    }
    return e & 1023u;
  }
  // bits consumed since init, given the starting offset
  __device__ __forceinline__ uint32_t consumed(uint32_t start_off) const {
    return (wi - 2 - kRing) * 32 + off - start_off;
  }
};

__device__ __forceinline__ uint64_t lower_bound_u32(const uint32_t *a, uint64_t n, uint32_t key) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}


}  // namespace fz
