// fz_decode.cu -- the inverse path (FZModules §3.3.1): chunked Huffman
// decode, outlier scatter, anchor restore, inverse Lorenzo and
// dequantization fused in one kernel.  The paper overlaps a CPU Huffman
// decode with a GPU outlier scatter; here both happen in the same GPU
// thread, which decodes one chunk (= one block) symbol by symbol and never
// stores the codes: the inverse Lorenzo is an inclusive prefix sum along x (a
// running sum in a register), then along y (per-column sums), then along z
// (per-(x,y) plane sums, kept in a per-thread column of shared memory), and
// every output row is written as soon as it is complete.  A warp covers 32
// consecutive blocks along x, so its rows form long contiguous runs in HBM.
// The loop body is one row of symbols, small enough for the instruction
// cache.
//
// The code-length limit of the format (14 bits) equals the width of the
// shared-memory decode table, so every codeword resolves with one lookup
// and the decode loop has no data-dependent branch.
//
// Kernels:
//   k_dec_gsum  -- per group of 256 chunks, the sum of their bit lengths
//   k_dec_prep  -- one CTA: canonical codes from the length table, the
//                  16384-entry decode table, and the exclusive scan of the
//                  group sums
//   k_decode    -- persistent; one thread per chunk of the current group
#include <string.h>

#include "fz_decode_common.cuh"

namespace fz {

namespace {

constexpr int kPrepThreads = 1024;

__device__ __forceinline__ void dec_err(uint32_t *err, uint32_t code) { atomicCAS(err, 0u, code); }

__global__ void k_dec_gsum(const uint32_t *__restrict__ chunk_bits, uint64_t n_chunks, uint64_t n_groups,
                           uint64_t *gsum) {
  const uint64_t gidx = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gidx >= n_groups) return;
  constexpr int kPerLane = kDecThreads / 32;  // 8
  const uint64_t c0 = gidx * kDecThreads + kPerLane * lane;
  unsigned long long s = 0;
  if (c0 + kPerLane - 1 < n_chunks) {
    const uint4 v = *reinterpret_cast<const uint4 *>(chunk_bits + c0);
    const uint4 w = *reinterpret_cast<const uint4 *>(chunk_bits + c0 + 4);
    s = (unsigned long long)v.x + v.y + v.z + v.w + w.x + w.y + w.z + w.w;
  } else {
    for (uint64_t c = c0; c < n_chunks && c < c0 + kPerLane; ++c) s += chunk_bits[c];
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) gsum[gidx] = s;
}

__global__ void __launch_bounds__(kPrepThreads) k_dec_prep(const uint8_t *__restrict__ lens_in, uint32_t nsym,
                                                            uint64_t *gsum, uint64_t n_groups,
                                                            uint64_t total_bits, uint16_t *lut, uint32_t *err) {
  __shared__ uint32_t first[kLmax + 1], cnt[kLmax + 1], basel[kLmax + 1];
  __shared__ uint32_t wcnt[32][kLmax + 1];
  __shared__ uint32_t wk[32];
  __shared__ uint16_t sorted[kMaxSym];
  __shared__ unsigned long long wsum[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int L = t < (int)nsym ? lens_in[t] : 0;
  const bool badlen = L > kLmax;
  if (badlen) L = 0;
  // Kraft sum in units of 2^-14 (fits 32 bits for 1024 symbols)
  uint32_t k = L ? (1u << (kLmax - L)) : 0u;
  k = __reduce_add_sync(0xffffffffu, k);
  const bool wbad = __any_sync(0xffffffffu, badlen);
  uint32_t rank = 0;
#pragma unroll 1
  for (int l = 1; l <= kLmax; ++l) {
    uint32_t b = __ballot_sync(0xffffffffu, L == l);
    if (L == l) rank = __popc(b & ((1u << lane) - 1));
    if (lane == 0) wcnt[warp][l] = __popc(b);
  }
  if (lane == 0) wk[warp] = wbad ? 0xffffffffu : k;
  __syncthreads();
  if (t >= 1 && t <= kLmax) {  // per-length counts and warp prefixes
    uint32_t acc = 0;
    for (int w = 0; w < 32; ++w) { uint32_t v = wcnt[w][t]; wcnt[w][t] = acc; acc += v; }
    cnt[t] = acc;
  }
  if (t == 32) {
    unsigned long long kraft = 0;
    bool bad = false;
    for (int w = 0; w < 32; ++w) {
      if (wk[w] == 0xffffffffu) bad = true;
      else kraft += wk[w];
    }
    first[0] = (bad || kraft == 0 || kraft > (1ull << kLmax)) ? 1u : 0u;  // status flag
  }
  __syncthreads();
  if (first[0]) {
    if (t == 0) dec_err(err, FZ_ECORRUPT);
    return;
  }
  __syncthreads();
  if (t == 0) {
    uint32_t c = 0, b = 0;
    cnt[0] = 0;
    first[0] = 0;
    for (int l = 1; l <= kLmax; ++l) {
      c = (c + cnt[l - 1]) << 1;
      first[l] = c;
      basel[l] = b;
      b += cnt[l];
    }
  }
  __syncthreads();
  if (L) sorted[basel[L] + wcnt[warp][L] + rank] = (uint16_t)t;
  __syncthreads();
  // every table entry: the codeword whose left-aligned range contains it
  for (int e = t; e < kLutSize; e += kPrepThreads) {
    uint16_t v = 0;
#pragma unroll
    for (int l = 1; l <= kLmax; ++l) {
      const uint32_t c = (uint32_t)e >> (kLmax - l);
      if (cnt[l] && c >= first[l] && c - first[l] < cnt[l])
        v = (uint16_t)(kLutValid | ((l - 1) << 10) | sorted[basel[l] + c - first[l]]);
    }
    lut[e] = v;
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
  uint64_t n_words;       // bitstream words
  const uint32_t *chunk_bits;
  const int32_t *anchors;
  const uint32_t *out_idx;
  const int32_t *out_val;
  const uint32_t *exc_idx;
  const uint32_t *exc_val;
  uint64_t n_out, n_exc, n_chunks, n_groups;
  const uint64_t *goff;
  const uint16_t *lut;
  uint32_t *err;
  float *out;
  float ebx2;
  int32_t R;
};

// Outliers and exceptions of one block (both lists ascend by code-stream
// position).  The rare paths are out of line to keep the decode loop small;
// they take and return their state by value so that nothing in the loop has
// its address taken (which would move it to local memory).
struct Side {
  uint64_t oc, ec;
  uint32_t next_e;
};

struct OutlierHit {
  int32_t value;
  uint32_t ok;
  uint64_t oc;
};

__device__ __noinline__ OutlierHit fetch_outlier(const uint32_t *out_idx, const int32_t *out_val, uint64_t n_out,
                                                 uint64_t oc, uint32_t pos0, uint32_t pos) {
  OutlierHit r;
  if (oc == ~0ull) oc = lower_bound_u32(out_idx, n_out, pos0);
  if (oc < n_out && __ldg(out_idx + oc) == pos) {
    r.value = __ldg(out_val + oc);
    r.ok = 1;
    r.oc = oc + 1;
  } else {
    r.value = 0;
    r.ok = 0;
    r.oc = oc;
  }
  return r;
}

struct ExceptionHit {
  uint32_t bits, next_e;
  uint64_t ec;
};

__device__ __noinline__ ExceptionHit fetch_exception(const uint32_t *exc_idx, const uint32_t *exc_val,
                                                     uint64_t n_exc, uint64_t ec) {
  ExceptionHit r;
  r.bits = __ldg(exc_val + ec);
  r.ec = ec + 1;
  r.next_e = r.ec < n_exc ? __ldg(exc_idx + r.ec) : 0xffffffffu;
  return r;
}

__device__ __forceinline__ void init_side(const DecParams &p, Side &sd, uint32_t pos0) {
  sd.oc = ~0ull;
  sd.ec = 0;
  sd.next_e = 0xffffffffu;
  if (p.n_exc) {
    sd.ec = lower_bound_u32(p.exc_idx, p.n_exc, pos0);
    if (sd.ec < p.n_exc) sd.next_e = __ldg(p.exc_idx + sd.ec);
  }
}

// Residual of the next symbol: code - R, or the stored outlier for code 0.
__device__ __forceinline__ int32_t next_delta(BitReader &br, const uint16_t *slut, const DecParams &p, Side &sd,
                                              uint32_t pos0, uint32_t pos, bool &bad) {
  const uint32_t sym = br.next(slut);
  if (sym == 0) {
    const OutlierHit h = fetch_outlier(p.out_idx, p.out_val, p.n_out, sd.oc, pos0, pos);
    sd.oc = h.oc;
    bad |= !h.ok;
    return h.value;
  }
  return (int32_t)sym - p.R;
}

template <bool EXC>
__device__ __forceinline__ float value(const DecParams &p, Side &sd, uint32_t pos, int32_t q) {
  float v = __fmul_rn(__int2float_rn(q), p.ebx2);
  if (EXC && pos == sd.next_e) {
    const ExceptionHit h = fetch_exception(p.exc_idx, p.exc_val, p.n_exc, sd.ec);
    sd.ec = h.ec;
    sd.next_e = h.next_e;
    v = __uint_as_float(h.bits);
  }
  return v;
}

__device__ __forceinline__ void store4(float *out, uint64_t f, bool vec, const float *o) {
  if (vec) {
    *reinterpret_cast<float4 *>(out + f) = make_float4(o[0], o[1], o[2], o[3]);
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) out[f + u] = o[u];
  }
}

// Per-thread prefix state that does not fit registers lives in shared
// memory, one column per thread ([i][thread] layout, conflict-free):
// 3D: the plane sums P (64 per order), 2D: the column sums Y (32 per order).
template <int NDIM, int K>
struct DecState {
  static constexpr int kWords = NDIM == 3 ? 64 * K : (NDIM == 2 ? 32 * K : 0);
};

template <int NDIM, int K>
constexpr size_t dec_smem_bytes() {
  return sizeof(uint16_t) * kLutSize +
         sizeof(int32_t) * (size_t)(DecState<NDIM, K>::kWords + kRing) * kDecThreads;
}

template <int NDIM, int K, bool EXC>
__device__ __forceinline__ void decode_chunk(const DecParams &p, const Geom &g, const uint16_t *slut,
                                             int32_t *st, uint32_t *ring, uint64_t j, uint64_t start, bool vecbase) {
  constexpr int T = kDecThreads;
  bool bad = false;
  BitReader br;
  const uint32_t cbits = __ldg(p.chunk_bits + j);
  br.init(p.words, p.n_words, start, cbits, ring);
  const uint32_t start_off = br.off;
  const uint32_t pos0 = (uint32_t)(j * g.bsize);
  Side sd;
  init_side(p, sd, pos0);
  const int32_t anchor = __ldg(p.anchors + j);
  const uint32_t bxi = (uint32_t)(j % g.nbx);
  const uint64_t jr = j / g.nbx;
  const uint32_t byi = (uint32_t)(jr % g.nby), bzi = (uint32_t)(jr / g.nby);
  const uint32_t X0 = bxi * g.bx, Y0 = byi * g.by, Z0 = bzi * g.bz;
  for (int i = 0; i < DecState<NDIM, K>::kWords; ++i) st[i * T] = 0;

  if (NDIM == 3) {
    // st[(y*8+x)*T]: plane sums of order 1; st[(64+y*8+x)*T]: order 2
    const bool xfull = X0 + 8 <= g.nx;
#pragma unroll 1
    for (int z = 0; z < 8; ++z) {
      int32_t Y1[8], Y2[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) { Y1[i] = 0; Y2[i] = 0; }
      const bool zin = Z0 + z < g.nz;
#pragma unroll 1
      for (int y = 0; y < 8; ++y) {
        int32_t r1 = 0, r2 = 0;
        float o[8];
        int32_t *row = st + (y * 8) * T;
#pragma unroll
        for (int x = 0; x < 8; ++x) {
          const uint32_t pos = pos0 + (uint32_t)(z * 64 + y * 8 + x);
          int32_t d = next_delta(br, slut, p, sd, pos0, pos, bad);
          if (x == 0) d += (y == 0 && z == 0) ? anchor : 0;
          int32_t q;
          if (K == 1) {
            r1 += d; Y1[x] += r1;
            q = row[x * T] + Y1[x];
            row[x * T] = q;
          } else {
            r1 += d; r2 += r1; Y1[x] += r2; Y2[x] += Y1[x];
            const int32_t p1 = row[x * T] + Y2[x];
            row[x * T] = p1;
            q = row[(64 + x) * T] + p1;
            row[(64 + x) * T] = q;
          }
          o[x] = value<EXC>(p, sd, pos, q);
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
    // st[x*T]: column sums of order 1; st[(32+x)*T]: order 2
    const bool xfull = X0 + 32 <= g.nx;
#pragma unroll 1
    for (int y = 0; y < 32; ++y) {
      int32_t r1 = 0, r2 = 0;
      const bool yin = Y0 + y < g.ny;
      const uint64_t f = ((uint64_t)(Y0 + y)) * g.nx + X0;
#pragma unroll 1
      for (int x8 = 0; x8 < 4; ++x8) {
        float o[8];
        int32_t *col = st + (x8 * 8) * T;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const uint32_t pos = pos0 + (uint32_t)(y * 32 + x8 * 8 + u);
          int32_t d = next_delta(br, slut, p, sd, pos0, pos, bad);
          if (u == 0) d += (x8 == 0 && y == 0) ? anchor : 0;
          int32_t q;
          if (K == 1) {
            r1 += d;
            q = col[u * T] + r1;
            col[u * T] = q;
          } else {
            r1 += d; r2 += r1;
            const int32_t y1 = col[u * T] + r2;
            col[u * T] = y1;
            q = col[(32 + u) * T] + y1;
            col[(32 + u) * T] = q;
          }
          o[u] = value<EXC>(p, sd, pos, q);
        }
        if (yin) {
          const uint64_t fx = f + 8 * x8;
          if (xfull) {
            store4(p.out, fx, vecbase, o);
            store4(p.out, fx + 4, vecbase, o + 4);
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u)
              if (X0 + 8 * x8 + u < g.nx) p.out[fx + u] = o[u];
          }
        }
      }
    }
  } else {
    // the anchor enters the first running sum once, as the origin residual
    int32_t r1 = anchor, r2 = 0;
    const uint64_t f0 = (uint64_t)X0;
    const bool full = X0 + 1024 <= g.nx;
#pragma unroll 1
    for (int x8 = 0; x8 < 128; ++x8) {
      float o[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint32_t pos = pos0 + (uint32_t)(8 * x8 + u);
        int32_t d = next_delta(br, slut, p, sd, pos0, pos, bad);
        int32_t q;
        if (K == 1) { r1 += d; q = r1; }
        else { r1 += d; r2 += r1; q = r2; }
        o[u] = value<EXC>(p, sd, pos, q);
      }
      if (full) {
        store4(p.out, f0 + 8 * x8, vecbase, o);
        store4(p.out, f0 + 8 * x8 + 4, vecbase, o + 4);
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (X0 + 8 * x8 + u < g.nx) p.out[f0 + 8 * x8 + u] = o[u];
      }
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");  // the ring is reused by the next chunk
  if (br.consumed(start_off) != cbits || bad || !(br.vall & kLutValid))
    dec_err(p.err, FZ_ECORRUPT);
}

template <int NDIM, int K>
__global__ void __launch_bounds__(kDecThreads) k_decode(DecParams p, Geom g) {
  extern __shared__ __align__(16) unsigned char d_smem[];
  uint16_t *slut = reinterpret_cast<uint16_t *>(d_smem);
  int32_t *sstate = reinterpret_cast<int32_t *>(d_smem + sizeof(uint16_t) * kLutSize);
  uint32_t *sring = reinterpret_cast<uint32_t *>(sstate + DecState<NDIM, K>::kWords * kDecThreads);
  __shared__ unsigned long long swarp[kDecThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(p.lut);
    uint4 *dst = reinterpret_cast<uint4 *>(slut);
    for (int i = t; i < kLutSize / 8; i += kDecThreads) dst[i] = __ldg(src + i);
  }
  const bool vecbase = ((g.nx & 3u) == 0) && (((uintptr_t)p.out & 15u) == 0);
  for (uint64_t grp = blockIdx.x; grp < p.n_groups; grp += gridDim.x) {
    const uint64_t j = grp * kDecThreads + t;
    const bool valid = j < p.n_chunks;
    const uint32_t cb = valid ? __ldg(p.chunk_bits + j) : 0u;
    unsigned long long incl = cb;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    __syncthreads();  // the table is in place and swarp is free again
    if (lane == 31) swarp[warp] = incl;
    __syncthreads();
    unsigned long long start = p.goff[grp] + incl - cb;
    for (int w = 0; w < warp; ++w) start += swarp[w];
    if (valid) {
      if (p.n_exc) decode_chunk<NDIM, K, true>(p, g, slut, sstate + t, sring + t, j, start, vecbase);
      else decode_chunk<NDIM, K, false>(p, g, slut, sstate + t, sring + t, j, start, vecbase);
    }
  }
}

template <int NDIM, int K>
cudaError_t launch_dec_t(const DecParams &p, const Geom &g, int sm_count, cudaStream_t s) {
  const int smem = (int)dec_smem_bytes<NDIM, K>();
  cudaError_t e = cudaFuncSetAttribute(k_decode<NDIM, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_decode<NDIM, K>, kDecThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t grid = (uint64_t)sm_count * per_sm;
  if (grid > p.n_groups) grid = p.n_groups;
  k_decode<NDIM, K><<<(unsigned)grid, kDecThreads, smem, s>>>(p, g);
  return cudaGetLastError();
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
                                        ws.err);
  return cudaGetLastError();
}

cudaError_t launch_decode_main(const uint8_t *d_in, const fz_header &h, float *d_out, const DecodeWs &ws,
                               cudaStream_t s, int sm_count) {
  Geom g;
  make_geom(h.ndim, h.dims, g);
  DecParams p;
  p.words = reinterpret_cast<const uint32_t *>(d_in + h.off_bits);
  p.n_words = (h.total_bits + 31) / 32;
  p.chunk_bits = reinterpret_cast<const uint32_t *>(d_in + h.off_chunk_bits);
  p.anchors = reinterpret_cast<const int32_t *>(d_in + h.off_anchors);
  p.out_idx = reinterpret_cast<const uint32_t *>(d_in + h.off_out_idx);
  p.out_val = reinterpret_cast<const int32_t *>(d_in + h.off_out_val);
  p.exc_idx = reinterpret_cast<const uint32_t *>(d_in + h.off_exc_idx);
  p.exc_val = reinterpret_cast<const uint32_t *>(d_in + h.off_exc_val);
  p.n_out = h.n_out;
  p.n_exc = h.n_exc;
  p.n_chunks = h.n_chunks;
  p.n_groups = (h.n_chunks + kDecThreads - 1) / kDecThreads;
  p.goff = ws.gsum;
  p.lut = ws.lut;
  p.err = ws.err;
  p.out = d_out;
  memcpy(&p.ebx2, &h.ebx2_bits, 4);
  p.R = (int32_t)h.radius;
  const bool k2 = h.predictor == FZ_PRED_LORENZO2;
  switch (g.ndim) {
    case 1: return k2 ? launch_dec_t<1, 2>(p, g, sm_count, s) : launch_dec_t<1, 1>(p, g, sm_count, s);
    case 2: return k2 ? launch_dec_t<2, 2>(p, g, sm_count, s) : launch_dec_t<2, 1>(p, g, sm_count, s);
    default: return k2 ? launch_dec_t<3, 2>(p, g, sm_count, s) : launch_dec_t<3, 1>(p, g, sm_count, s);
  }
}

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
