// fz_decode.cu -- the inverse path (FZModules §3.3.1): chunked Huffman
// decode, outlier scatter, anchor restore, inverse Lorenzo and
// dequantization fused in one kernel.  The paper overlaps a CPU Huffman
// decode with a GPU outlier scatter; here both happen in the same GPU
// thread, which decodes one chunk (= one block) straight into registers:
// the inverse Lorenzo is an inclusive prefix sum along x (a running sum),
// then along y (per-column sums), then along z (per-(x,y) plane sums), so
// a thread never needs the decoded codes in memory.  Every output row is
// written as soon as it is complete: a warp covers 32 consecutive blocks
// along x, so its rows form long contiguous runs in HBM.
//
// Kernels:
//   k_dec_gsum  -- per group of 128 chunks, the sum of their bit lengths
//   k_dec_prep  -- one CTA: canonical codes from the length table, the
//                  first-level decode table (12 bits), long-code tables,
//                  and the exclusive scan of the group sums
//   k_decode    -- one thread per chunk
#include <string.h>

#include "fz_internal.cuh"

namespace fz {

namespace {

constexpr int kPrepThreads = 1024;
constexpr int kLtFirst = 0, kLtCount = 25, kLtBase = 50, kLtSorted = 75, kLtWords = 75 + kMaxSym;

__device__ __forceinline__ void dec_err(uint32_t *err, uint32_t code) { atomicCAS(err, 0u, code); }

__global__ void k_dec_gsum(const uint32_t *__restrict__ chunk_bits, uint64_t n_chunks, uint64_t n_groups,
                           uint64_t *gsum) {
  const uint64_t gidx = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gidx >= n_groups) return;
  const uint64_t c0 = gidx * kDecThreads + 4 * lane;
  unsigned long long s = 0;
  if (c0 + 3 < n_chunks) {
    uint4 v = *reinterpret_cast<const uint4 *>(chunk_bits + c0);
    s = (unsigned long long)v.x + v.y + v.z + v.w;
  } else {
    for (uint64_t c = c0; c < n_chunks && c < c0 + 4; ++c) s += chunk_bits[c];
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) gsum[gidx] = s;
}

__global__ void __launch_bounds__(kPrepThreads) k_dec_prep(const uint8_t *__restrict__ lens_in, uint32_t nsym,
                                                            uint64_t *gsum, uint64_t n_groups,
                                                            uint64_t total_bits, uint32_t *lut, uint32_t *ltab,
                                                            uint32_t *err) {
  __shared__ uint32_t bl[kLmax + 1], first[kLmax + 1], basel[kLmax + 1];
  __shared__ uint32_t wcnt[32][kLmax + 1];
  __shared__ unsigned long long kraft;
  __shared__ unsigned long long wsum[32];
  __shared__ int bad;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t <= kLmax) bl[t] = 0;
  if (t == 0) { kraft = 0; bad = 0; }
  if (t < 32 * (kLmax + 1)) (&wcnt[0][0])[t] = 0;
  for (int i = t; i < (1 << kLutBits); i += kPrepThreads) lut[i] = 0;
  __syncthreads();
  int L = t < (int)nsym ? lens_in[t] : 0;
  if (L > kLmax) { bad = 1; L = 0; }
  if (L) {
    atomicAdd(&bl[L], 1u);
    atomicAdd(&kraft, 1ull << (kLmax - L));
  }
  __syncthreads();
  if (bad || kraft == 0 || kraft > (1ull << kLmax)) {
    if (t == 0) dec_err(err, FZ_ECORRUPT);
    return;
  }
  uint32_t rank = 0;
#pragma unroll 1
  for (int l = 1; l <= kLmax; ++l) {
    uint32_t b = __ballot_sync(0xffffffffu, L == l);
    if (L == l) rank = __popc(b & ((1u << lane) - 1));
    if (lane == 0) wcnt[warp][l] = __popc(b);
  }
  __syncthreads();
  if (t >= 1 && t <= kLmax) {
    uint32_t acc = 0;
    for (int w = 0; w < 32; ++w) { uint32_t v = wcnt[w][t]; wcnt[w][t] = acc; acc += v; }
  }
  if (t == 0) {
    uint32_t c = 0, b = 0;
    for (int l = 1; l <= kLmax; ++l) {
      c = (c + (l > 1 ? bl[l - 1] : 0u)) << 1;
      first[l] = c;
      basel[l] = b;
      b += bl[l];
      ltab[kLtFirst + l] = c;
      ltab[kLtCount + l] = bl[l];
      ltab[kLtBase + l] = basel[l];
    }
    ltab[kLtFirst] = ltab[kLtCount] = ltab[kLtBase] = 0;
  }
  __syncthreads();
  if (L) {
    const uint32_t r = wcnt[warp][L] + rank;
    const uint32_t code = first[L] + r;
    ltab[kLtSorted + basel[L] + r] = (uint32_t)t;
    if (L <= kLutBits) {
      const uint32_t e = ((uint32_t)L << 16) | (uint32_t)t;
      const uint32_t lo = code << (kLutBits - L), cnt = 1u << (kLutBits - L);
      for (uint32_t i = 0; i < cnt; ++i) lut[lo + i] = e;
    }
  }
  // exclusive scan of the group bit sums (in place)
  const uint64_t per = (n_groups + kPrepThreads - 1) / kPrepThreads;
  const uint64_t g0 = (uint64_t)t * per;
  unsigned long long loc = 0;
  for (uint64_t i = g0; i < g0 + per && i < n_groups; ++i) loc += gsum[i];
  unsigned long long incl = loc;
  for (int off = 1; off < 32; off <<= 1) {
    unsigned long long v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long v = wsum[lane], iv = v;
    for (int off = 1; off < 32; off <<= 1) {
      unsigned long long u = __shfl_up_sync(0xffffffffu, iv, off);
      if (lane >= off) iv += u;
    }
    wsum[lane] = iv - v;
    if (lane == 31 && iv != total_bits) dec_err(err, FZ_ECORRUPT);
  }
  __syncthreads();
  unsigned long long run = wsum[warp] + incl - loc;
  for (uint64_t i = g0; i < g0 + per && i < n_groups; ++i) {
    unsigned long long v = gsum[i];
    gsum[i] = run;
    run += v;
  }
}

struct DecParams {
  const uint32_t *words;
  uint64_t n_words;
  const uint32_t *chunk_bits;
  const int32_t *anchors;
  const uint32_t *out_idx;
  const int32_t *out_val;
  const uint32_t *exc_idx;
  const uint32_t *exc_val;
  uint64_t n_out, n_exc, n_chunks;
  const uint64_t *goff;
  const uint32_t *lut;
  const uint32_t *ltab;
  uint32_t *err;
  float *out;
  float ebx2;
  int32_t R;
};

struct BitReader {
  const uint32_t *W;
  uint64_t nw, wi;
  unsigned long long buf;
  int nb;
  uint32_t used;
  __device__ __forceinline__ uint32_t ld(uint64_t i) const { return i < nw ? __ldg(W + i) : 0u; }
  __device__ __forceinline__ void init(const uint32_t *w, uint64_t n, uint64_t bitpos) {
    W = w; nw = n; wi = bitpos >> 5;
    const int sk = (int)(bitpos & 31u);
    buf = (((unsigned long long)ld(wi) << 32) | ld(wi + 1)) << sk;
    nb = 64 - sk;
    wi += 2;
    used = 0;
  }
};

__device__ __noinline__ uint32_t decode_long(unsigned long long buf, const uint32_t *slt, const uint16_t *ssorted,
                                             uint32_t &L) {
  for (int l = kLutBits + 1; l <= kLmax; ++l) {
    const uint32_t v = (uint32_t)(buf >> (64 - l));
    const uint32_t d = v - slt[kLtFirst + l];
    if (d < slt[kLtCount + l]) { L = (uint32_t)l; return ssorted[slt[kLtBase + l] + d]; }
  }
  L = 0;
  return 0xffffffffu;
}

__device__ __forceinline__ uint32_t next_sym(BitReader &br, const uint32_t *slut, const uint32_t *slt,
                                             const uint16_t *ssorted, bool &bad) {
  if (br.nb < 32) {
    br.buf |= (unsigned long long)br.ld(br.wi) << (32 - br.nb);
    ++br.wi;
    br.nb += 32;
  }
  const uint32_t e = slut[br.buf >> (64 - kLutBits)];
  uint32_t L = e >> 16, sym = e & 0xffffu;
  if (L == 0) {
    sym = decode_long(br.buf, slt, ssorted, L);
    if (L == 0) { bad = true; L = 1; sym = 0xffffffffu; }
  }
  br.buf <<= L;
  br.nb -= (int)L;
  br.used += L;
  return sym;
}

__device__ __forceinline__ uint64_t lower_bound_u32(const uint32_t *a, uint64_t n, uint32_t key) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Per-thread state for outliers and exceptions of one block.
struct Side {
  uint64_t oc, ec;
  uint32_t next_e;
  __device__ __forceinline__ int32_t outlier(const DecParams &p, uint32_t pos0, uint32_t pos, bool &bad) {
    if (oc == ~0ull) oc = lower_bound_u32(p.out_idx, p.n_out, pos0);
    if (oc < p.n_out && __ldg(p.out_idx + oc) == pos) return __ldg(p.out_val + oc++);
    bad = true;
    return 0;
  }
  __device__ __forceinline__ void init_exc(const DecParams &p, uint32_t pos0) {
    oc = ~0ull;
    next_e = 0xffffffffu;
    ec = 0;
    if (p.n_exc) {
      ec = lower_bound_u32(p.exc_idx, p.n_exc, pos0);
      if (ec < p.n_exc) next_e = __ldg(p.exc_idx + ec);
    }
  }
  __device__ __forceinline__ float exc(const DecParams &p, uint32_t pos, float v) {
    if (pos != next_e) return v;
    float r = __uint_as_float(__ldg(p.exc_val + ec));
    ++ec;
    next_e = ec < p.n_exc ? __ldg(p.exc_idx + ec) : 0xffffffffu;
    return r;
  }
};

// Residual of the next symbol: code - R, the outlier value for code 0.
__device__ __forceinline__ int32_t next_delta(BitReader &br, const uint32_t *slut, const uint32_t *slt,
                                              const uint16_t *ssorted, const DecParams &p, Side &sd,
                                              uint32_t pos0, uint32_t pos, bool &bad) {
  const uint32_t sym = next_sym(br, slut, slt, ssorted, bad);
  if (sym == 0) return sd.outlier(p, pos0, pos, bad);
  return (int32_t)sym - p.R;
}

__device__ __forceinline__ void store4(float *out, uint64_t f, bool vec, const float *o) {
  if (vec) {
    *reinterpret_cast<float4 *>(out + f) = make_float4(o[0], o[1], o[2], o[3]);
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) out[f + u] = o[u];
  }
}

template <int NDIM, int K>
__global__ void __launch_bounds__(kDecThreads) k_decode(DecParams p, Geom g) {
  __shared__ uint32_t slut[1 << kLutBits];
  __shared__ uint32_t slt[kLtSorted];
  __shared__ uint16_t ssorted[kMaxSym];
  __shared__ unsigned long long swarp[kDecThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int i = t; i < (1 << kLutBits); i += kDecThreads) slut[i] = __ldg(p.lut + i);
  for (int i = t; i < kLtSorted; i += kDecThreads) slt[i] = __ldg(p.ltab + i);
  for (int i = t; i < kMaxSym; i += kDecThreads) ssorted[i] = (uint16_t)__ldg(p.ltab + kLtSorted + i);
  const uint64_t j = (uint64_t)blockIdx.x * kDecThreads + t;
  const bool valid = j < p.n_chunks;
  const uint32_t cb = valid ? __ldg(p.chunk_bits + j) : 0u;
  unsigned long long incl = cb;
  for (int off = 1; off < 32; off <<= 1) {
    unsigned long long v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) swarp[warp] = incl;
  __syncthreads();
  unsigned long long start = p.goff[blockIdx.x] + incl - cb;
  for (int w = 0; w < warp; ++w) start += swarp[w];
  if (!valid) return;

  bool bad = false;
  BitReader br;
  br.init(p.words, p.n_words, start);
  const uint32_t pos0 = (uint32_t)(j * g.bsize);
  Side sd;
  sd.init_exc(p, pos0);
  const int32_t anchor = __ldg(p.anchors + j);
  const float ebx2 = p.ebx2;
  const uint32_t bxi = (uint32_t)(j % g.nbx);
  const uint64_t jr = j / g.nbx;
  const uint32_t byi = (uint32_t)(jr % g.nby), bzi = (uint32_t)(jr / g.nby);
  const uint32_t X0 = bxi * g.bx, Y0 = byi * g.by, Z0 = bzi * g.bz;
  const bool vecbase = ((g.nx & 3u) == 0) && (((uintptr_t)p.out & 15u) == 0);

  if (NDIM == 3) {
    int32_t P1[64], P2[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) { P1[i] = 0; P2[i] = 0; }
    const bool xfull = X0 + 8 <= g.nx;
#pragma unroll 1
    for (int z = 0; z < 8; ++z) {
      int32_t Y1[8], Y2[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) { Y1[i] = 0; Y2[i] = 0; }
      const bool zin = Z0 + z < g.nz;
#pragma unroll
      for (int y = 0; y < 8; ++y) {
        int32_t r1 = 0, r2 = 0;
        float o[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          const uint32_t pos = pos0 + (uint32_t)(z * 64 + y * 8 + x);
          int32_t d = next_delta(br, slut, slt, ssorted, p, sd, pos0, pos, bad);
          if (y == 0 && x == 0) d += (z == 0) ? anchor : 0;
          int32_t q;
          if (K == 1) {
            r1 += d; Y1[x] += r1; P1[y * 8 + x] += Y1[x]; q = P1[y * 8 + x];
          } else {
            r1 += d; r2 += r1; Y1[x] += r2; Y2[x] += Y1[x];
            P1[y * 8 + x] += Y2[x]; P2[y * 8 + x] += P1[y * 8 + x]; q = P2[y * 8 + x];
          }
          o[x] = sd.exc(p, pos, __fmul_rn(__int2float_rn(q), ebx2));
        }
        if (zin && Y0 + y < g.ny) {
          const uint64_t f = ((uint64_t)(Z0 + z) * g.ny + (Y0 + y)) * g.nx + X0;
          if (xfull) {
            store4(p.out, f, vecbase, o);
            store4(p.out, f + 4, vecbase, o + 4);
          } else {
#pragma unroll
            for (int x = 0; x < 8; ++x)
              if (X0 + x < g.nx) p.out[f + x] = o[x];
          }
        }
      }
    }
  } else if (NDIM == 2) {
    int32_t Y1[32], Y2[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) { Y1[i] = 0; Y2[i] = 0; }
    const bool xfull = X0 + 32 <= g.nx;
#pragma unroll 1
    for (int y = 0; y < 32; ++y) {
      int32_t r1 = 0, r2 = 0;
      const bool yin = Y0 + y < g.ny;
      const uint64_t f = ((uint64_t)(Y0 + y)) * g.nx + X0;
#pragma unroll
      for (int x4 = 0; x4 < 8; ++x4) {
        float o[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int x = 4 * x4 + u;
          const uint32_t pos = pos0 + (uint32_t)(y * 32 + x);
          int32_t d = next_delta(br, slut, slt, ssorted, p, sd, pos0, pos, bad);
          if (x == 0) d += (y == 0) ? anchor : 0;
          int32_t q;
          if (K == 1) { r1 += d; Y1[x] += r1; q = Y1[x]; }
          else { r1 += d; r2 += r1; Y1[x] += r2; Y2[x] += Y1[x]; q = Y2[x]; }
          o[u] = sd.exc(p, pos, __fmul_rn(__int2float_rn(q), ebx2));
        }
        if (yin) {
          if (xfull) store4(p.out, f + 4 * x4, vecbase, o);
          else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (X0 + 4 * x4 + u < g.nx) p.out[f + 4 * x4 + u] = o[u];
          }
        }
      }
    }
  } else {
    int32_t r1 = anchor, r2 = 0;
    const uint64_t f0 = (uint64_t)X0;
    const bool full = X0 + 1024 <= g.nx;
#pragma unroll 2
    for (int x4 = 0; x4 < 256; ++x4) {
      float o[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t pos = pos0 + (uint32_t)(4 * x4 + u);
        int32_t d = next_delta(br, slut, slt, ssorted, p, sd, pos0, pos, bad);
        int32_t q;
        if (K == 1) { r1 += d; q = r1; }
        else {
          // anchor enters the first running sum once, as the origin residual
          r1 += d; r2 += r1; q = r2;
        }
        o[u] = sd.exc(p, pos, __fmul_rn(__int2float_rn(q), ebx2));
      }
      if (full) store4(p.out, f0 + 4 * x4, vecbase, o);
      else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (X0 + 4 * x4 + u < g.nx) p.out[f0 + 4 * x4 + u] = o[u];
      }
    }
  }
  if (br.used != cb || bad) dec_err(p.err, FZ_ECORRUPT);
}

template <int NDIM, int K>
void launch_dec_t(const DecParams &p, const Geom &g, uint64_t n_groups, cudaStream_t s) {
  k_decode<NDIM, K><<<(unsigned)n_groups, kDecThreads, 0, s>>>(p, g);
}

}  // namespace

cudaError_t launch_decode_prep(const uint8_t *d_in, const fz_header &h, const DecodeWs &ws, cudaStream_t s) {
  const uint64_t n_chunks = h.n_chunks;
  const uint64_t n_groups = (n_chunks + kDecThreads - 1) / kDecThreads;
  const uint32_t *cbits = reinterpret_cast<const uint32_t *>(d_in + h.off_chunk_bits);
  {
    const uint64_t threads = n_groups * 32;
    k_dec_gsum<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(cbits, n_chunks, n_groups, ws.gsum);
  }
  k_dec_prep<<<1, kPrepThreads, 0, s>>>(d_in + h.off_lens, 2 * h.radius, ws.gsum, n_groups, h.total_bits, ws.lut,
                                        ws.ltab, ws.err);
  return cudaGetLastError();
}

cudaError_t launch_decode_main(const uint8_t *d_in, const fz_header &h, float *d_out, const DecodeWs &ws,
                               cudaStream_t s) {
  Geom g;
  make_geom(h.ndim, h.dims, g);
  const uint64_t n_chunks = h.n_chunks;
  const uint64_t n_groups = (n_chunks + kDecThreads - 1) / kDecThreads;
  const uint32_t *cbits = reinterpret_cast<const uint32_t *>(d_in + h.off_chunk_bits);
  DecParams p;
  p.words = reinterpret_cast<const uint32_t *>(d_in + h.off_bits);
  p.n_words = (h.total_bits + 31) / 32;
  p.chunk_bits = cbits;
  p.anchors = reinterpret_cast<const int32_t *>(d_in + h.off_anchors);
  p.out_idx = reinterpret_cast<const uint32_t *>(d_in + h.off_out_idx);
  p.out_val = reinterpret_cast<const int32_t *>(d_in + h.off_out_val);
  p.exc_idx = reinterpret_cast<const uint32_t *>(d_in + h.off_exc_idx);
  p.exc_val = reinterpret_cast<const uint32_t *>(d_in + h.off_exc_val);
  p.n_out = h.n_out;
  p.n_exc = h.n_exc;
  p.n_chunks = n_chunks;
  p.goff = ws.gsum;
  p.lut = ws.lut;
  p.ltab = ws.ltab;
  p.err = ws.err;
  p.out = d_out;
  memcpy(&p.ebx2, &h.ebx2_bits, 4);
  p.R = (int32_t)h.radius;
  const bool k2 = h.predictor == FZ_PRED_LORENZO2;
  switch (g.ndim) {
    case 1: k2 ? launch_dec_t<1, 2>(p, g, n_groups, s) : launch_dec_t<1, 1>(p, g, n_groups, s); break;
    case 2: k2 ? launch_dec_t<2, 2>(p, g, n_groups, s) : launch_dec_t<2, 1>(p, g, n_groups, s); break;
    default: k2 ? launch_dec_t<3, 2>(p, g, n_groups, s) : launch_dec_t<3, 1>(p, g, n_groups, s); break;
  }
  return cudaGetLastError();
}

}  // namespace fz

namespace fz {
namespace {
__global__ void k_fill(float *out, uint64_t n, uint32_t bits) {
  const float v = __uint_as_float(bits);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = v;
}
}  // namespace

// CONST streams: every value is the stored one.
cudaError_t launch_fill(float *out, uint64_t n, uint32_t bits, cudaStream_t s, int sm_count) {
  uint64_t grid = (n + 255) / 256;
  if (grid > (uint64_t)sm_count * 8) grid = (uint64_t)sm_count * 8;
  if (grid < 1) grid = 1;
  k_fill<<<(unsigned)grid, 256, 0, s>>>(out, n, bits);
  return cudaGetLastError();
}
}  // namespace fz
