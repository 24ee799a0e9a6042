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

__device__ __forceinline__ void k_dec_prep_body(const uint8_t *__restrict__ lens_in, uint32_t nsym, uint64_t *gsum,
                                                uint64_t n_groups, uint64_t total_bits, uint16_t *lut, uint32_t *err) {
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

__global__ void __launch_bounds__(kPrepThreads) k_dec_prep(const uint8_t *__restrict__ lens_in, uint32_t nsym,
                                                            uint64_t *gsum, uint64_t n_groups,
                                                            uint64_t total_bits, uint16_t *lut, uint32_t *err) {
  k_dec_prep_body(lens_in, nsym, gsum, n_groups, total_bits, lut, err);
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

// Decode groups grp, grp + step, ... below g_end of one field whose table
// is in slut; all threads of the CTA call it together.
template <int NDIM, int K>
__device__ __forceinline__ void decode_groups(const DecParams &p, const Geom &g, const uint16_t *slut,
                                              int32_t *sstate, uint32_t *sring, unsigned long long *swarp,
                                              uint64_t grp, uint64_t g_end, uint64_t step) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool vecbase = ((g.nx & 3u) == 0) && (((uintptr_t)p.out & 15u) == 0);
  for (; grp < g_end; grp += step) {
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

__device__ __forceinline__ void load_lut(uint16_t *slut, const uint16_t *lut) {
  const uint4 *src = reinterpret_cast<const uint4 *>(lut);
  uint4 *dst = reinterpret_cast<uint4 *>(slut);
  for (int i = threadIdx.x; i < kLutSize / 8; i += kDecThreads) dst[i] = __ldg(src + i);
}

template <int NDIM, int K>
__global__ void __launch_bounds__(kDecThreads) k_decode(DecParams p, Geom g) {
  extern __shared__ __align__(16) unsigned char d_smem[];
  uint16_t *slut = reinterpret_cast<uint16_t *>(d_smem);
  int32_t *sstate = reinterpret_cast<int32_t *>(d_smem + sizeof(uint16_t) * kLutSize);
  uint32_t *sring = reinterpret_cast<uint32_t *>(sstate + DecState<NDIM, K>::kWords * kDecThreads);
  __shared__ unsigned long long swarp[kDecThreads / 32];
  load_lut(slut, p.lut);
  decode_groups<NDIM, K>(p, g, slut, sstate, sring, swarp, blockIdx.x, p.n_groups, gridDim.x);
}

// ---------------------------------------------------------------- batched decode
// One field of a batched decompress (Huffman streams only).
struct DecJob {
  DecParams p;
  Geom g;
  const uint8_t *lens;
  uint32_t nsym, pad;
  uint64_t total_bits;
  uint64_t group_base;  // first decode group in the job's class queue
};

// Group bit sums of every field: blockIdx.y = field.
__global__ void k_dec_gsum_batch(const DecJob *__restrict__ jobs) {
  const DecJob &J = jobs[blockIdx.y];
  const uint64_t gidx = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gidx >= J.p.n_groups) return;
  const uint64_t c0 = gidx * kDecThreads + 8 * lane;
  unsigned long long s = 0;
  for (uint64_t c = c0; c < J.p.n_chunks && c < c0 + 8; ++c) s += J.p.chunk_bits[c];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) const_cast<uint64_t *>(J.p.goff)[gidx] = s;
}

// Decode tables and group offsets: one CTA per field.
__global__ void __launch_bounds__(kPrepThreads) k_dec_prep_batch(const DecJob *__restrict__ jobs) {
  const DecJob &J = jobs[blockIdx.x];
  k_dec_prep_body(J.lens, J.nsym, const_cast<uint64_t *>(J.p.goff), J.p.n_groups, J.total_bits,
                  const_cast<uint16_t *>(J.p.lut), J.p.err);
}

// The decode groups of every field of one class (dimensionality, Lorenzo
// order) form one queue cut into equal contiguous ranges, one per CTA; the
// decode table is reloaded when the CTA moves to another field.
template <int NDIM, int K>
__global__ void __launch_bounds__(kDecThreads) k_decode_batch(const DecJob *__restrict__ jobs,
                                                               const uint32_t *__restrict__ members,
                                                               uint32_t n_members, uint64_t total_groups) {
  extern __shared__ __align__(16) unsigned char d_smem[];
  uint16_t *slut = reinterpret_cast<uint16_t *>(d_smem);
  int32_t *sstate = reinterpret_cast<int32_t *>(d_smem + sizeof(uint16_t) * kLutSize);
  uint32_t *sring = reinterpret_cast<uint32_t *>(sstate + DecState<NDIM, K>::kWords * kDecThreads);
  __shared__ unsigned long long swarp[kDecThreads / 32];
  __shared__ DecParams sp;
  __shared__ Geom sg;
  const uint64_t lo = total_groups * blockIdx.x / gridDim.x, hi = total_groups * (blockIdx.x + 1) / gridDim.x;
  uint32_t a = 0, b = n_members;
  while (a < b) {
    const uint32_t m = (a + b) >> 1;
    const DecJob &J = jobs[members[m]];
    if (J.group_base + J.p.n_groups <= lo) a = m + 1; else b = m;
  }
  for (uint64_t t = lo; t < hi && a < n_members; ++a) {
    const DecJob &J = jobs[members[a]];
    const uint64_t jb = J.group_base, je = jb + J.p.n_groups;
    const uint64_t t0 = t > jb ? t : jb, t1 = hi < je ? hi : je;
    __syncthreads();  // the previous field is done with the table and the staged parameters
    if (threadIdx.x == 0) { sp = J.p; sg = J.g; }
    load_lut(slut, J.p.lut);
    __syncthreads();
    if (t0 < t1) decode_groups<NDIM, K>(sp, sg, slut, sstate, sring, swarp, t0 - jb, t1 - jb, 1);
    t = t1;
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

// ---------------------------------------------------------------- batched decode: host side
namespace {
// RAW and CONST fields of a batched decompress.
struct PlainJob {
  const uint8_t *src;  // the stream
  float *out;
  uint64_t n;
  uint32_t is_const, pad;
};

__global__ void k_plain_batch(const PlainJob *__restrict__ jobs, uint32_t n) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (uint64_t)gridDim.x * blockDim.x;
  for (uint32_t j = 0; j < n; ++j) {
    const PlainJob &J = jobs[j];
    const uint8_t *src = J.src + FZ_HEADER_BYTES;
    if (J.is_const) {
      const float v = *reinterpret_cast<const float *>(src);
      for (uint64_t i = tid; i < J.n; i += nth) J.out[i] = v;
    } else {
      const float *f = reinterpret_cast<const float *>(src);
      for (uint64_t i = tid; i < J.n; i += nth) J.out[i] = f[i];
    }
  }
}

template <int NDIM, int K>
cudaError_t launch_dec_batch_t(const DecJob *jobs, const uint32_t *members, uint32_t n_members,
                               uint64_t total_groups, int per_sm, cudaStream_t s, int sms) {
  const int smem = (int)dec_smem_bytes<NDIM, K>();
  cudaError_t e = cudaFuncSetAttribute(k_decode_batch<NDIM, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_decode_batch<NDIM, K>, kDecThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  if (per_sm < 1 || per_sm > occ) per_sm = occ;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > total_groups) grid = total_groups;
  if (grid < 1) grid = 1;
  k_decode_batch<NDIM, K><<<(unsigned)grid, kDecThreads, smem, s>>>(jobs, members, n_members, total_groups);
  return cudaGetLastError();
}
}  // namespace

size_t dec_job_bytes() { return sizeof(DecJob); }
size_t plain_job_bytes() { return sizeof(PlainJob); }
uint64_t dec_groups(const fz_header &h) { return (h.n_chunks + kDecThreads - 1) / kDecThreads; }

void fill_dec_job(void *dst, const uint8_t *d_in, const fz_header &h, float *d_out, uint16_t *lut, uint64_t *gsum,
                  uint32_t *err, uint64_t group_base) {
  DecJob J;
  memset(&J, 0, sizeof(J));
  make_geom(h.ndim, h.dims, J.g);
  DecParams &p = J.p;
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
  p.n_groups = dec_groups(h);
  p.goff = gsum;
  p.lut = lut;
  p.err = err;
  p.out = d_out;
  memcpy(&p.ebx2, &h.ebx2_bits, 4);
  p.R = (int32_t)h.radius;
  J.lens = d_in + h.off_lens;
  J.nsym = 2 * h.radius;
  J.total_bits = h.total_bits;
  J.group_base = group_base;
  memcpy(dst, &J, sizeof(J));
}

void fill_plain_job(void *dst, const uint8_t *d_in, uint64_t n, bool is_const, float *d_out) {
  PlainJob J;
  memset(&J, 0, sizeof(J));
  J.src = d_in;
  J.out = d_out;
  J.n = n;
  J.is_const = is_const ? 1u : 0u;
  memcpy(dst, &J, sizeof(J));
}

cudaError_t launch_decode_batch_prep(const void *jobs, uint32_t n, uint64_t max_groups, cudaStream_t s) {
  const DecJob *J = reinterpret_cast<const DecJob *>(jobs);
  const uint64_t gx = (max_groups * 32 + 255) / 256;
  k_dec_gsum_batch<<<dim3((unsigned)gx, n), 256, 0, s>>>(J);
  k_dec_prep_batch<<<n, kPrepThreads, 0, s>>>(J);
  return cudaGetLastError();
}

cudaError_t launch_decode_batch_main(int ndim, int k, const void *jobs, const uint32_t *members, uint32_t n_members,
                                     uint64_t total_groups, int per_sm, cudaStream_t s, int sms) {
  const DecJob *J = reinterpret_cast<const DecJob *>(jobs);
  const bool k2 = k == 2;
  switch (ndim) {
    case 1:
      return k2 ? launch_dec_batch_t<1, 2>(J, members, n_members, total_groups, per_sm, s, sms)
                : launch_dec_batch_t<1, 1>(J, members, n_members, total_groups, per_sm, s, sms);
    case 2:
      return k2 ? launch_dec_batch_t<2, 2>(J, members, n_members, total_groups, per_sm, s, sms)
                : launch_dec_batch_t<2, 1>(J, members, n_members, total_groups, per_sm, s, sms);
    default:
      return k2 ? launch_dec_batch_t<3, 2>(J, members, n_members, total_groups, per_sm, s, sms)
                : launch_dec_batch_t<3, 1>(J, members, n_members, total_groups, per_sm, s, sms);
  }
}

cudaError_t launch_plain_batch(const void *jobs, uint32_t n, uint64_t max_n, cudaStream_t s, int sms) {
  uint64_t grid = (max_n + 255) / 256;
  if (grid > (uint64_t)sms * 8) grid = (uint64_t)sms * 8;
  if (grid < 1) grid = 1;
  k_plain_batch<<<(unsigned)grid, 256, 0, s>>>(reinterpret_cast<const PlainJob *>(jobs), n);
  return cudaGetLastError();
}

// CONST streams: every value is the stored one.
cudaError_t launch_fill(float *out, uint64_t n, uint32_t bits, cudaStream_t s, int sm_count) {
  uint64_t grid = (n + 255) / 256;
  if (grid > (uint64_t)sm_count * 8) grid = (uint64_t)sm_count * 8;
  if (grid < 1) grid = 1;
  k_fill<<<(unsigned)grid, 256, 0, s>>>(out, n, bits);
  return cudaGetLastError();
}

}  // namespace fz
