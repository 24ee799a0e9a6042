// fz_decode_common.cuh -- pieces shared by the decoders: the decode table
// format, the asynchronous per-thread bit reader and small helpers.
#pragma once

#include "fz_internal.cuh"

namespace fz {

constexpr int kLutSize = 1 << kLutBits;
// Decode-table entry, read as a signed 16-bit value e: e >> 4 (arithmetic)
// is the decoded value v = symbol - offset, e & 15 the codeword length
// (1..14).  The residual decoders build their table with offset R, so v is
// the Lorenzo residual and code 0 (an outlier) reads as -R; the code
// decoder uses offset 0 (v is the code).  A window that starts no codeword
// (only in a corrupt stream) holds code 0 with length 0: the reader stops
// advancing there and the chunk's bit count check fails.
__host__ __device__ constexpr uint16_t lut_entry(int32_t v, uint32_t len) {
  return (uint16_t)(((uint32_t)v << 4) | len);
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void cp_async4(uint32_t *dst_smem, const uint32_t *src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
  const int n = valid ? 4 : 0;  // zero-fill past the end of the bitstream
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

constexpr int kRing = 4;  // stream words in flight per thread (a power of two)

// MSB-first bit reader over one chunk, all 32-bit: a window of three stream
// words (a, b, c) and a bit offset (< 32) into a.  Codewords are decoded
// four at a time, all within the window, after which the window slides by
// up to two words.  The slide is predicated, not branched, so a warp whose lanes slide at different times
// never diverges: the next word comes from a per-thread ring in shared
// memory that asynchronous copies fill kRing slides ahead, so a slide never
// waits on memory and no register is read while its load is in flight.
// Words past the end of the bitstream read as zero.
template <int T>  // threads of the CTA: the stride of the per-thread ring columns
struct BitReader {
  const uint32_t *W;   // the chunk's first word
  uint32_t nw;         // words from W to the end of the bitstream
  uint32_t wi;         // next word to fetch into the ring, relative to W
  uint32_t ring_s;     // shared-memory address of this thread's ring column
  uint32_t rd;         // next ring slot to read
  uint32_t a, b, c;
  uint32_t off;        // bits of a already consumed (0..31)
  __device__ __forceinline__ uint32_t ld(uint32_t i) const { return i < nw ? __ldg(W + i) : 0u; }
  __device__ __forceinline__ void init(const uint32_t *words, uint64_t n_words, uint64_t bitpos, uint32_t bits,
                                       uint32_t *ring_col) {
    const uint64_t sw = bitpos >> 5;
    W = words + sw;
    nw = (uint32_t)(n_words > sw ? (n_words - sw < 0xffffffffull ? n_words - sw : 0xffffffffull) : 0);
    off = (uint32_t)(bitpos & 31u);
    ring_s = (uint32_t)__cvta_generic_to_shared(ring_col);
    a = ld(0);
    b = ld(1);
    c = ld(2);
#pragma unroll
    for (int k = 0; k < kRing; ++k) cp_async4(ring_col + k * T, W + (3 + k < nw ? 3 + k : 0), 3 + k < nw);
    wi = 3 + kRing;
    rd = 0;
    // the whole chunk (a few 128-byte lines) is pulled into L2 up front
    const uint32_t cw = (off + bits + 31) / 32 + 2;
    for (uint32_t i = 32; i < cw && i < nw; i += 32) prefetch_l2(W + i);
  }
  // Four symbols.  They all lie in the window: from an offset below 32,
  // four codewords of at most 14 bits end by bit 87 < 96, and the fourth
  // starts by bit 73, so its 14-bit lookup window needs no fourth word.  The
  // window then slides by 0, 1 or 2 words, predicated rather than branched.
  __device__ __forceinline__ void next4(const uint16_t *slut, int32_t (&s)[4]) {
    uint32_t o = off;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      uint32_t w;
      if (k == 0) w = __funnelshift_l(b, a, o);                                   // o < 32
      else if (k < 3) w = o < 32 ? __funnelshift_l(b, a, o) : __funnelshift_l(c, b, o);  // o < 60
      else w = o < 32 ? __funnelshift_l(b, a, o) : (o < 64 ? __funnelshift_l(c, b, o) : c << (o & 31u));
      const int32_t e = (int16_t)slut[w >> (32 - kLutBits)];
      s[k] = e >> 4;
      o += (uint32_t)e & 15u;
    }
    const uint32_t adv = o >> 5;  // 0, 1 or 2
    off = o & 31u;
    // the oldest one or two ring slots become the window's new words and are
    // refilled with the words kRing slides ahead; waiting for all but the
    // newest kRing - 2 copies covers both slots
    const uint32_t slot0 = ring_s + rd * (uint32_t)(T * 4);
    const uint32_t slot1 = ring_s + ((rd + 1) & (kRing - 1)) * (uint32_t)(T * 4);
    const bool more0 = wi < nw, more1 = wi + 1 < nw;
    const uint32_t *src0 = W + (more0 ? wi : 0u);
    const uint32_t *src1 = W + (more1 ? wi + 1 : 0u);
    uint32_t r0 = 0, r1 = 0;
    asm volatile(
        "{\n"
        " .reg .pred p1, p2;\n"
        " setp.ne.u32 p1, %2, 0;\n"
        " setp.gt.u32 p2, %2, 1;\n"
        " @p1 cp.async.wait_group %9;\n"
        " @p1 ld.shared.u32 %0, [%3];\n"
        " @p2 ld.shared.u32 %1, [%4];\n"
        " @p1 cp.async.ca.shared.global [%3], [%5], 4, %7;\n"
        " @p1 cp.async.commit_group;\n"
        " @p2 cp.async.ca.shared.global [%4], [%6], 4, %8;\n"
        " @p2 cp.async.commit_group;\n"
        "}\n"
        : "+r"(r0), "+r"(r1)
        : "r"(adv), "r"(slot0), "r"(slot1), "l"(src0), "l"(src1), "r"(more0 ? 4 : 0), "r"(more1 ? 4 : 0),
          "n"(kRing - 2));
    const uint32_t na = adv == 0 ? a : (adv == 1 ? b : c);
    const uint32_t nb = adv == 0 ? b : (adv == 1 ? c : r0);
    const uint32_t nc = adv == 0 ? c : (adv == 1 ? r0 : r1);
    a = na;
    b = nb;
    c = nc;
    rd = (rd + adv) & (kRing - 1);
    wi += adv;
  }
  // Eight residuals from a table built with offset R; returns whether any
  // is -R (code 0: an outlier, whose residual is looked up afterwards).
  __device__ __forceinline__ bool group8(const uint16_t *slut, int32_t R, int32_t (&d)[8]) {
    bool zero = false;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      int32_t s[4];
      next4(slut, s);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        zero = zero || s[u] == -R;
        d[4 * k + u] = s[u];
      }
    }
    return zero;
  }
  // bits consumed since init, given the starting offset
  __device__ __forceinline__ uint32_t consumed(uint32_t start_off) const {
    return (wi - 3 - kRing) * 32 + off - start_off;
  }
};

// Start bit of each lane's chunk in work unit u (lane = chunk within the
// unit); also returns the chunk's bit count.  All lanes call it.
__device__ __forceinline__ uint64_t unit_start(const uint32_t *chunk_bits, const uint64_t *uoff, uint64_t n_chunks,
                                               uint64_t u, uint32_t &cb) {
  const int lane = threadIdx.x & 31;
  const uint64_t j = u * kDecUnit + lane;
  cb = j < n_chunks ? __ldg(chunk_bits + j) : 0u;
  uint32_t incl = cb;  // a unit holds at most 32 x 1024 x 14 bits
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  return uoff[u] + (incl - cb);
}

// Next work unit for this warp from a counter shared by all CTAs.
__device__ __forceinline__ uint32_t claim_unit(uint32_t *counter) {
  uint32_t u = 0;
  if ((threadIdx.x & 31) == 0) u = atomicAdd(counter, 1u);
  return __shfl_sync(0xffffffffu, u, 0);
}

__device__ __forceinline__ uint64_t lower_bound_u32(const uint32_t *a, uint64_t n, uint32_t key) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}


}  // namespace fz
