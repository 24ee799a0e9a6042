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
//   k_dec_offsets    -- first bit of every work unit (32 chunks): a CTA scan
//                       of the chunk bit lengths and a decoupled look-back
//                       across CTAs; checks the total against the header
//   k_outlier_starts -- per block, its first outlier (streams with many)
//   k_decode         -- persistent, one CTA per SM: each CTA builds the
//                       decode table from the length table, each warp
//                       claims work units and each lane decodes one chunk
//   k_dec_gsum, k_dec_prep (per-block predictor streams and batches): unit
//                       sums, one-CTA scan and decode table
//   k_*_batch        -- the same for every field of a batch
#include <string.h>

#include "fz_decode_common.cuh"

namespace fz {

namespace {

constexpr int kPrepThreads = 1024;

__device__ __forceinline__ void dec_err(uint32_t *err, uint32_t code) { atomicCAS(err, 0u, code); }

// Bit length of every work unit (kDecUnit chunks): one warp per unit.
__global__ void k_dec_gsum(const uint32_t *__restrict__ chunk_bits, uint64_t n_chunks, uint64_t n_units,
                           uint64_t *usum) {
  const uint64_t u = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= n_units) return;
  const uint64_t j = u * kDecUnit + lane;
  uint32_t v = j < n_chunks ? __ldg(chunk_bits + j) : 0u;
  v = __reduce_add_sync(0xffffffffu, v);
  if (lane == 0) usum[u] = v;
}

__device__ __forceinline__ void dec_scan_body(uint64_t *gsum, uint64_t n_units, uint64_t total_bits, uint32_t *err);

__device__ __forceinline__ void k_dec_prep_body(const uint8_t *__restrict__ lens_in, uint32_t nsym, int32_t off,
                                                uint64_t *gsum, uint64_t n_units, uint64_t total_bits, uint16_t *lut,
                                                uint32_t *err) {
  __shared__ uint32_t first[kLmax + 1], cnt[kLmax + 1], basel[kLmax + 1];
  __shared__ uint32_t wcnt[32][kLmax + 1];
  __shared__ uint32_t wk[32];
  __shared__ uint16_t sorted[kMaxSym];
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
    uint16_t v = lut_entry(-off, 0);
#pragma unroll
    for (int l = 1; l <= kLmax; ++l) {
      const uint32_t c = (uint32_t)e >> (kLmax - l);
      if (cnt[l] && c >= first[l] && c - first[l] < cnt[l])
        v = lut_entry((int32_t)sorted[basel[l] + c - first[l]] - off, (uint32_t)l);
    }
    lut[e] = v;
  }
  dec_scan_body(gsum, n_units, total_bits, err);
}

// Exclusive scan, in place, of the work units' bit sums by one CTA of
// kPrepThreads threads; the grand total must equal the header's bit count.
__device__ __forceinline__ void dec_scan_body(uint64_t *gsum, uint64_t n_units, uint64_t total_bits, uint32_t *err) {
  __shared__ unsigned long long wsum[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint64_t per = (n_units + kPrepThreads - 1) / kPrepThreads;
  const uint64_t g0 = (uint64_t)t * per;
  unsigned long long loc = 0;
  for (uint64_t i = g0; i < g0 + per && i < n_units; ++i) loc += gsum[i];
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
  for (uint64_t i = g0; i < g0 + per && i < n_units; ++i) {
    unsigned long long v = gsum[i];
    gsum[i] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(kPrepThreads) k_dec_prep(const uint8_t *__restrict__ lens_in, uint32_t nsym,
                                                            uint64_t *gsum, uint64_t n_units,
                                                            uint64_t total_bits, uint16_t *lut, uint32_t *err) {
  k_dec_prep_body(lens_in, nsym, 0, gsum, n_units, total_bits, lut, err);  // codes, for the code decoder
}

// Shared memory of the in-kernel decode-table build.
struct LutBuild {
  uint32_t wcnt[32][kLmax + 1];  // per group of 32 symbols and length: count, then exclusive prefix
  uint32_t gk[32];               // per group: Kraft sum in units of 2^-14, or ~0 for a length above 14
  uint32_t cnt[kLmax + 1], first[kLmax + 1], basel[kLmax + 1], limit[kLmax + 1];
  uint32_t ok;
  uint16_t sorted[kMaxSym];
};

// The canonical decode table of the length table lens[0..nsym) built by the
// T threads of a CTA into slut: codes of length l occupy the contiguous
// range [first[l], first[l] + cnt[l]) << (14 - l) of the 14-bit window, the
// ranges follow each other in length order, and entry e holds l and the
// symbol of rank (e >> (14 - l)) - first[l] among the symbols of its length
// l, minus off.  Windows past the last range (an incomplete code) hold code
// 0 with length 0.  Returns false (in every thread) for a length above 14 or
// a Kraft sum outside (0, 1].
template <int T>
__device__ bool build_lut(const uint8_t *__restrict__ lens, uint32_t nsym, int32_t off, uint16_t *slut, LutBuild &b) {
  constexpr int W = T / 32;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (int grp = warp; grp < 32; grp += W) {
    const int sym = grp * 32 + lane;
    int L = sym < (int)nsym ? lens[sym] : 0;
    const bool badlen = L > kLmax;
    if (badlen) L = 0;
    const uint32_t k = __reduce_add_sync(0xffffffffu, L ? (1u << (kLmax - L)) : 0u);
    const bool wbad = __any_sync(0xffffffffu, badlen);
#pragma unroll 1
    for (int l = 1; l <= kLmax; ++l) {
      const uint32_t bl = __ballot_sync(0xffffffffu, L == l);
      if (lane == l) b.wcnt[grp][l] = __popc(bl);
    }
    if (lane == 0) b.gk[grp] = wbad ? 0xffffffffu : k;
  }
  __syncthreads();
  if (t >= 1 && t <= kLmax) {  // per-length counts and group prefixes
    uint32_t acc = 0;
    for (int grp = 0; grp < 32; ++grp) { const uint32_t v = b.wcnt[grp][t]; b.wcnt[grp][t] = acc; acc += v; }
    b.cnt[t] = acc;
  }
  if (t == 32) {
    unsigned long long kraft = 0;
    bool bad = false;
    for (int grp = 0; grp < 32; ++grp) {
      if (b.gk[grp] == 0xffffffffu) bad = true;
      else kraft += b.gk[grp];
    }
    b.ok = (!bad && kraft > 0 && kraft <= (1ull << kLmax)) ? 1u : 0u;
  }
  __syncthreads();
  if (!b.ok) return false;
  if (t == 0) {
    uint32_t c = 0, base = 0;
    b.cnt[0] = 0;
    for (int l = 1; l <= kLmax; ++l) {
      c = (c + b.cnt[l - 1]) << 1;
      b.first[l] = c;
      b.basel[l] = base;
      base += b.cnt[l];
      b.limit[l] = (c + b.cnt[l]) << (kLmax - l);
    }
  }
  __syncthreads();
  for (int grp = warp; grp < 32; grp += W) {
    const int sym = grp * 32 + lane;
    const int L = sym < (int)nsym ? lens[sym] : 0;
    uint32_t rank = 0;
#pragma unroll 1
    for (int l = 1; l <= kLmax; ++l) {
      const uint32_t bl = __ballot_sync(0xffffffffu, L == l);
      if (L == l) rank = __popc(bl & ((1u << lane) - 1));
    }
    if (L) b.sorted[b.basel[L] + b.wcnt[grp][L] + rank] = (uint16_t)sym;
  }
  __syncthreads();
  uint32_t lim[kLmax + 1];
#pragma unroll
  for (int l = 1; l <= kLmax; ++l) lim[l] = b.limit[l];
  for (int e = t; e < kLutSize; e += T) {
    int l = 1;
#pragma unroll
    for (int k = 1; k < kLmax; ++k) l += (uint32_t)e >= lim[k] ? 1 : 0;
    uint16_t v = lut_entry(-off, 0);
    if ((uint32_t)e < lim[kLmax])
      v = lut_entry((int32_t)b.sorted[b.basel[l] + ((uint32_t)e >> (kLmax - l)) - b.first[l]] - off, (uint32_t)l);
    slut[e] = v;
  }
  return true;
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
  uint64_t n_out, n_exc, n_chunks, n_units;
  const uint64_t *goff;   // per work unit: first bit
  const uint16_t *lut;    // decode table (batched decode)
  const uint8_t *lens;    // code-length table (single-field decode builds its table from it)
  const uint32_t *ofirst; // per block with outliers: index of its first outlier (or null: search)
  uint32_t nsym;
  uint64_t total_bits;
  uint32_t *err;          // err[0] error word, err[1] work-unit counter, err[2] CTAs done
  uint32_t *h_err;        // host-mapped copy of err[0], written by the last CTA (or null)
  float *out;
  float ebx2;
  int32_t R;
  uint32_t gate = 0;      // 0 decode; 1 only if err[4] is clear; 2 only if err[4] is set
};

// Outliers and exceptions of one block (both lists ascend by code-stream
// position).  The rare paths are out of line to keep the decode loop small;
// they take and return their state by value so that nothing in the loop has
// its address taken (which would move it to local memory).
struct Side {
  uint64_t oc, ec;   // next outlier / exception of the block in the lists (oc ~0: not located yet)
  uint32_t next_o;   // position of outlier oc (prefetched; ~0 past the end)
  int32_t next_v;    // its residual
  uint32_t next_e;
};

// Position and residual of outlier oc, loaded ahead of their use.
__device__ __forceinline__ void load_outlier(const DecParams &p, Side &sd) {
  const bool in = sd.oc < p.n_out;
  sd.next_o = in ? __ldg(p.out_idx + sd.oc) : 0xffffffffu;
  sd.next_v = in ? __ldg(p.out_val + sd.oc) : 0;
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
  sd.next_o = 0xffffffffu;
  sd.next_v = 0;
  sd.ec = 0;
  sd.next_e = 0xffffffffu;
  if (p.n_exc) {
    sd.ec = lower_bound_u32(p.exc_idx, p.n_exc, pos0);
    if (sd.ec < p.n_exc) sd.next_e = __ldg(p.exc_idx + sd.ec);
  }
}

// Dequantized values of eight reconstructed integers q, exceptions replaced
// by their stored bits.
template <bool EXC>
__device__ __forceinline__ void values8(const DecParams &p, Side &sd, uint32_t pos, const int32_t (&q)[8],
                                        float (&o)[8]) {
#pragma unroll
  for (int x = 0; x < 8; ++x) o[x] = __fmul_rn(__int2float_rn(q[x]), p.ebx2);
  if (EXC) {
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      if (pos + x == sd.next_e) {
        const ExceptionHit h = fetch_exception(p.exc_idx, p.exc_val, p.n_exc, sd.ec);
        sd.ec = h.ec;
        sd.next_e = h.next_e;
        o[x] = __uint_as_float(h.bits);
      }
    }
  }
}

__device__ __forceinline__ void store4(float *out, uint64_t f, bool vec, const float *o) {
  if (vec) {
    *reinterpret_cast<float4 *>(out + f) = make_float4(o[0], o[1], o[2], o[3]);
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) out[f + u] = o[u];
  }
}

// Eight consecutive outputs of a block row starting at field index f, of
// which those below x_end (field x) exist.
__device__ __forceinline__ void store8(float *out, uint64_t f, bool full, bool vec, uint32_t x0, uint32_t nx,
                                       const float (&o)[8]) {
  if (full) {
    store4(out, f, vec, o);
    store4(out, f + 4, vec, o + 4);
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (x0 + u < nx) out[f + u] = o[u];
  }
}

// Per-thread prefix state that does not fit registers lives in shared
// memory, one column per thread ([i][thread] layout, conflict-free):
// 3D: the plane sums P (64 per order), 2D: the column sums Y (32 per order).
// Words of per-thread prefix state.  NS (narrow state, 3D order 1): the
// previous plane's values relative to the block's anchor as 16-bit integers,
// 32 words instead of 64 (see narrow_state_candidate).
template <int NDIM, int K, bool NS = false>
struct DecState {
  static constexpr int kWords = NS ? 32 : (NDIM == 3 ? 64 * K : (NDIM == 2 ? 32 * K : 0));
};

// Threads per decode CTA (one CTA per SM).  The decode table is shared by
// all of them, and the rest of the SM's 256 KB of shared memory + L1 is
// split between the per-thread state and L1, which must keep about one
// 128-byte line of every thread's bitstream resident: the asynchronous word
// copies then hit L1 instead of going to L2 one sector per word.
#ifndef FZ_DEC_T3
#define FZ_DEC_T3 448
#endif
#ifndef FZ_DEC_T2
#define FZ_DEC_T2 256  // 2D order 1: 384 to 768 measured slower on a 1800 x 3600 field
#endif
#ifndef FZ_DEC_T1
#define FZ_DEC_T1 1024  // 1D: 768 and 896 measured slower on a 281M-value field
#endif
#ifndef FZ_DEC_NARROW
#define FZ_DEC_NARROW 1
#endif
#ifndef FZ_DEC_T3N
// narrow state: 576 and 640 threads measured alike, 704 slower (L1 then too
// small for the bitstream lines)
#define FZ_DEC_T3N 576
#endif
template <int NDIM, int K, bool NS = false>
struct DecCta {
  static constexpr int T = NS ? FZ_DEC_T3N
                              : (NDIM == 3 ? (K == 1 ? FZ_DEC_T3 : 288) : (NDIM == 2 ? (K == 1 ? FZ_DEC_T2 : 448) : FZ_DEC_T1));
};

template <int NDIM, int K, bool NS = false>
constexpr size_t dec_smem_bytes() {
  return sizeof(uint16_t) * kLutSize +
         sizeof(int32_t) * (size_t)(DecState<NDIM, K, NS>::kWords + kRing) * DecCta<NDIM, K, NS>::T;
}

// The stored residuals of the outliers among eight codes (code 0 decodes
// to -R, which no in-range code gives).  Rare: out of the decode loop's
// straight-line code.
__device__ __forceinline__ void fix_outliers(const DecParams &p, Side &sd, uint64_t j, uint32_t pos0, uint32_t pos,
                                             int32_t (&d)[8], bool &bad) {
  if (sd.oc == ~0ull) {  // the block's first outlier: from the per-block table, else by search
    sd.oc = p.ofirst ? __ldg(p.ofirst + j) : lower_bound_u32(p.out_idx, p.n_out, pos0);
    load_outlier(p, sd);
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    if (d[u] == -p.R) {
      const bool hit = sd.next_o == pos + u;
      bad |= !hit;
      d[u] = hit ? sd.next_v : 0;
      if (hit) {
        ++sd.oc;
        load_outlier(p, sd);  // consumed at the next outlier, so its latency hides behind the decode
      }
    }
  }
}

// A thread's per-block prefix state in shared memory, in 16-byte slots:
// words 4k..4k+3 of thread t at slot k * T + t, so the eight words of a row
// move with two 16-byte accesses (four shared-memory instructions per row
// instead of sixteen).
template <int T>
__device__ __forceinline__ void st_load8(const int32_t *st, int w0, int32_t (&v)[8]) {
  const int4 *p = reinterpret_cast<const int4 *>(st) + (w0 >> 2) * T;
  const int4 a = p[0], b = p[T];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
template <int T>
__device__ __forceinline__ void st_store8(int32_t *st, int w0, const int32_t (&v)[8]) {
  int4 *p = reinterpret_cast<int4 *>(st) + (w0 >> 2) * T;
  p[0] = make_int4(v[0], v[1], v[2], v[3]);
  p[T] = make_int4(v[4], v[5], v[6], v[7]);
}
// the state pointer of thread t
__device__ __forceinline__ int32_t *st_thread(int32_t *sstate, int t) { return sstate + 4 * t; }

// Prefix-sum state of the inverse Lorenzo for one chunk.
struct Prefix {
  int32_t r1, r2;          // running sums along x (orders 1, 2)
  int32_t Y1[8], Y2[8];    // 3D: per-column sums along y within the plane
};

// Inverse Lorenzo, dequantization and store of group gi (eight codes) of a
// chunk: 3D group = one x-row (z = gi / 8, y = gi % 8); 2D group = a quarter
// row (y = gi / 4); 1D group = eight consecutive values.
template <int NDIM, int K, bool EXC, int T, bool NS = false>
__device__ __forceinline__ void consume(const DecParams &p, const Geom &g, Side &sd, Prefix &s, int32_t *st,
                                        int gi, const int32_t (&d)[8], uint32_t pos0, uint32_t X0, uint32_t Y0,
                                        uint32_t Z0, bool vecbase, int32_t anchor) {
  float o[8];
  const uint32_t pos = pos0 + (uint32_t)gi * 8;
  if (NDIM == 3) {
    const int y = gi & 7, z = gi >> 3;
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      s.Y1[x] = y ? s.Y1[x] : 0;
      if (K == 2) s.Y2[x] = y ? s.Y2[x] : 0;
    }
    int32_t r1 = 0, r2 = 0, q[8], z1[8], z2[8];
    int4 *nrow = reinterpret_cast<int4 *>(st) + y * T;  // NS: row y's eight 16-bit values
    if (NS) {
      const int4 w = *nrow;
      const uint32_t wv[4] = {(uint32_t)w.x, (uint32_t)w.y, (uint32_t)w.z, (uint32_t)w.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        z1[2 * i] = (int32_t)(wv[i] << 16) >> 16;
        z1[2 * i + 1] = (int32_t)wv[i] >> 16;
      }
    } else {
      st_load8<T>(st, y * 8, z1);
    }
    if (K == 2) st_load8<T>(st, 64 + y * 8, z2);
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      if (K == 1) {
        r1 += d[x];
        s.Y1[x] += r1;
        q[x] = z1[x] + s.Y1[x];
      } else {
        r1 += d[x];
        r2 += r1;
        s.Y1[x] += r2;
        s.Y2[x] += s.Y1[x];
        z1[x] += s.Y2[x];
        q[x] = z2[x] + z1[x];
      }
    }
    if (K == 2) st_store8<T>(st, y * 8, z1);
    if (NS) {
      *nrow = make_int4((int32_t)__byte_perm(q[0], q[1], 0x5410), (int32_t)__byte_perm(q[2], q[3], 0x5410),
                        (int32_t)__byte_perm(q[4], q[5], 0x5410), (int32_t)__byte_perm(q[6], q[7], 0x5410));
#pragma unroll
      for (int x = 0; x < 8; ++x) q[x] += anchor;
    } else {
      st_store8<T>(st, K == 1 ? y * 8 : 64 + y * 8, q);
    }
    values8<EXC>(p, sd, pos, q, o);
    if (Z0 + z < g.nz && Y0 + y < g.ny)
      store8(p.out, ((uint64_t)(Z0 + z) * g.ny + (Y0 + y)) * g.nx + X0, X0 + 8 <= g.nx, vecbase, X0, g.nx, o);
  } else if (NDIM == 2) {
    const int y = gi >> 2, x8 = gi & 3;
    s.r1 = x8 ? s.r1 : 0;
    if (K == 2) s.r2 = x8 ? s.r2 : 0;
    int32_t q[8], c1[8], c2[8];
    st_load8<T>(st, x8 * 8, c1);
    if (K == 2) st_load8<T>(st, 32 + x8 * 8, c2);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (K == 1) {
        s.r1 += d[u];
        q[u] = c1[u] + s.r1;
      } else {
        s.r1 += d[u];
        s.r2 += s.r1;
        c1[u] += s.r2;
        q[u] = c2[u] + c1[u];
      }
    }
    if (K == 2) st_store8<T>(st, x8 * 8, c1);
    st_store8<T>(st, K == 1 ? x8 * 8 : 32 + x8 * 8, q);
    values8<EXC>(p, sd, pos, q, o);
    if (Y0 + y < g.ny)
      store8(p.out, (uint64_t)(Y0 + y) * g.nx + X0 + 8 * x8, X0 + 8 * x8 + 8 <= g.nx, vecbase, X0 + 8 * x8, g.nx,
             o);
  } else {
    int32_t q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      s.r1 += d[u];
      if (K == 2) s.r2 += s.r1;
      q[u] = K == 1 ? s.r1 : s.r2;
    }
    values8<EXC>(p, sd, pos, q, o);
    const uint32_t x0 = X0 + 8 * (uint32_t)gi;
    store8(p.out, x0, x0 + 8 <= g.nx, vecbase, x0, g.nx, o);
  }
}

// One chunk: nblk consecutive blocks from jb on (the chunk is one block, or
// a power-of-two number of blocks), read by one bit reader.  The codes are
// decoded eight at a time, one
// group ahead of the reconstruction: the decode of group gi+1 (a serial
// chain through the bit reader) and the reconstruction of group gi
// (independent arithmetic and stores) sit in the same straight-line code,
// so they overlap.  Outliers are looked up per group, off that path.
template <int NDIM, int K, bool EXC, int T, bool NS = false>
__device__ __forceinline__ void decode_chunk(const DecParams &p, const Geom &g, const uint16_t *slut,
                                             int32_t *st, uint32_t *ring, uint64_t jb, uint32_t nblk,
                                             uint64_t start, uint32_t cbits, bool vecbase) {
  constexpr int NG = (NDIM == 3 ? 512 : 1024) / 8;
  bool bad = false;
  BitReader<T> br;
  br.init(p.words, p.n_words, start, cbits, ring);
  const uint32_t start_off = br.off;
#pragma unroll 1
  for (uint32_t bi = 0; bi < nblk; ++bi) {
    const uint64_t j = jb + bi;
    const uint32_t pos0 = (uint32_t)(j * g.bsize);
    Side sd;
    init_side(p, sd, pos0);
    const int32_t anchor = __ldg(p.anchors + j);
    const uint32_t j32 = (uint32_t)j;  // blocks number at most nx*ny*nz < 2^32
    const uint32_t bxi = j32 % g.nbx, jr = j32 / g.nbx;
    const uint32_t byi = jr % g.nby, bzi = jr / g.nby;
    const uint32_t X0 = bxi * g.bx, Y0 = byi * g.by, Z0 = bzi * g.bz;
    for (int i = 0; i < DecState<NDIM, K, NS>::kWords / 4; ++i)
      reinterpret_cast<int4 *>(st)[i * T] = make_int4(0, 0, 0, 0);
    Prefix s;
    s.r1 = 0;
    s.r2 = 0;
#pragma unroll
    for (int x = 0; x < 8; ++x) { s.Y1[x] = 0; s.Y2[x] = 0; }

    int32_t cur[8];
    if (br.group8(slut, p.R, cur)) fix_outliers(p, sd, j, pos0, pos0, cur, bad);
    if (!NS) cur[0] += anchor;  // the block origin's residual is its anchor (NS: added at the output)
#pragma unroll 1
    for (int gi = 0; gi < NG - 1; ++gi) {
      int32_t nxt[8];
      const bool zero = br.group8(slut, p.R, nxt);
      consume<NDIM, K, EXC, T, NS>(p, g, sd, s, st, gi, cur, pos0, X0, Y0, Z0, vecbase, anchor);
      if (zero) fix_outliers(p, sd, j, pos0, pos0 + (uint32_t)(gi + 1) * 8, nxt, bad);
#pragma unroll
      for (int u = 0; u < 8; ++u) cur[u] = nxt[u];
    }
    consume<NDIM, K, EXC, T, NS>(p, g, sd, s, st, NG - 1, cur, pos0, X0, Y0, Z0, vecbase, anchor);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");  // the ring is reused by the next chunk
  if (br.consumed(start_off) != cbits || bad) dec_err(p.err, FZ_ECORRUPT);
}

// Work units of one field whose table is in slut, claimed by this warp from
// the field's counter until none is left.
template <int NDIM, int K, bool NS>
__device__ __forceinline__ void decode_units(const DecParams &p, const Geom &g, const uint16_t *slut,
                                             int32_t *sstate, uint32_t *sring) {
  constexpr int T = DecCta<NDIM, K, NS>::T;
  const int t = threadIdx.x;
  // 16-byte stores of 4 consecutive x: aligned whenever rows start on a
  // 4-value boundary (1D: always; 2D/3D: nx a multiple of 4)
  const bool vecbase = (NDIM == 1 || (g.nx & 3u) == 0) && (((uintptr_t)p.out & 15u) == 0);
  const int lane = t & 31;
  for (;;) {
    const uint32_t u = claim_unit(p.err + 1);
    if (u >= p.n_units) break;
    uint32_t cb;
    const uint64_t start = unit_start(p.chunk_bits, p.goff, p.n_chunks, u, cb);
    const uint64_t j = (uint64_t)u * kDecUnit + lane;
    if (j < p.n_chunks) {
      // a chunk of k >= 1 whole blocks (the last one may hold fewer)
      const uint32_t k = g.chunk / g.bsize;
      const uint64_t jb = j * k;
      const uint32_t nblk = (uint32_t)(g.n_blocks - jb < k ? g.n_blocks - jb : k);
      int32_t *st = st_thread(sstate, t);
      if (p.n_exc) decode_chunk<NDIM, K, true, T, NS>(p, g, slut, st, sring + t, jb, nblk, start, cb, vecbase);
      else decode_chunk<NDIM, K, false, T, NS>(p, g, slut, st, sring + t, jb, nblk, start, cb, vecbase);
    }
  }
}

// ---------------------------------------------------------------- 2D chunks below the block
// A 2D first-order Lorenzo stream whose chunks are 4, 8 or 16 rows of a
// 32x32 block (C = 128, 256 or 512): lane l of work unit u decodes chunk
// 32u + l, rows RPC s .. RPC s + RPC - 1 (RPC = C / 32) of its block, s the
// chunk's index within the block.  The state a chunk starts from (the
// values of the row above it, per column) depends on the chunks above it,
// which neighbouring lanes of the same warp decode.  So every lane decodes
// its chunk into a shared-memory buffer of residuals (16-bit) while it sums
// its column totals; each lane then adds up the totals of the chunks above
// its own (read from their lanes' state columns) into its starting state;
// and reconstructs its rows from the buffer.  Every lane takes part in the
// warp-wide steps, with or without a chunk.  The CTA holds 384 x 128 / C
// threads, so the buffers take 96 KB at every C.
constexpr int kSub2dWords = 32;  // column state per thread (first order)

template <int C>
struct Sub2d {
  static constexpr int T = 384 * 128 / C;  // 384, 192 or 96 threads
  static constexpr int kSlots = C / 8;     // 16-byte buffer slots (eight residuals) per thread
  static constexpr size_t kSmem =
      sizeof(uint16_t) * kLutSize + sizeof(int32_t) * (size_t)(kSub2dWords + kRing) * T + 16 * (size_t)kSlots * T;
};

template <int C, bool EXC>
__device__ __forceinline__ void decode_sub2d_chunk(const DecParams &p, const Geom &g, const uint16_t *slut,
                                                   int32_t *sstate, uint32_t *ring, int4 *buf, uint64_t j,
                                                   uint64_t start, uint32_t cbits, bool live, bool vecbase) {
  constexpr int T = Sub2d<C>::T;
  constexpr uint32_t kCpb = 1024 / C;  // chunks per block
  constexpr uint32_t kNg = C / 8;      // groups of eight codes per chunk
  const int t = threadIdx.x;
  const uint64_t jb = j / kCpb;
  const uint32_t sub = (uint32_t)(j % kCpb);
  const uint32_t pos0 = (uint32_t)(jb * 1024);  // the block's first position
  const uint32_t cpos = pos0 + sub * C;         // the chunk's first position
  int32_t *st = st_thread(sstate, t);
  const uint32_t j32 = (uint32_t)jb;
  const uint32_t X0 = (j32 % g.nbx) * g.bx, Y0 = (j32 / g.nbx) * g.by;
  const int32_t anchor = live ? __ldg(p.anchors + jb) : 0;
  bool bad = false;
  // ---- pass 1: decode into the buffer, sum the column totals (row prefix
  // sums added per column)
  for (int i = 0; i < kSub2dWords / 4; ++i) reinterpret_cast<int4 *>(st)[i * T] = make_int4(0, 0, 0, 0);
  if (live) {
    BitReader<T> br;
    br.init(p.words, p.n_words, start, cbits, ring);
    const uint32_t start_off = br.off;
    Side sd;
    init_side(p, sd, cpos);
    int32_t r1 = 0;
#pragma unroll 1
    for (uint32_t gi = 0; gi < kNg; ++gi) {
      int32_t d[8];
      const bool zero = br.group8(slut, p.R, d);
      buf[gi * T] = make_int4((int32_t)__byte_perm(d[0], d[1], 0x5410), (int32_t)__byte_perm(d[2], d[3], 0x5410),
                              (int32_t)__byte_perm(d[4], d[5], 0x5410), (int32_t)__byte_perm(d[6], d[7], 0x5410));
      if (zero) fix_outliers(p, sd, j, cpos, cpos + gi * 8, d, bad);
      if (gi == 0 && sub == 0) d[0] += anchor;  // the block origin's residual is its anchor
      const uint32_t x8 = gi & 3u;
      r1 = x8 ? r1 : 0;
      int32_t c[8];
      st_load8<T>(st, (int)x8 * 8, c);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        r1 += d[u];
        c[u] += r1;
      }
      st_store8<T>(st, (int)x8 * 8, c);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (br.consumed(start_off) != cbits) bad = true;
  }
  __syncwarp();
  // ---- starting state: the totals of the chunks above this one in the block
  // (lanes t - sub .. t - 1 of this warp), gathered before any lane writes
  int32_t a[kSub2dWords];
#pragma unroll
  for (int x = 0; x < kSub2dWords; ++x) a[x] = 0;
  for (uint32_t k = 1; k <= sub; ++k) {
    const int32_t *o = st_thread(sstate, t - (int)k);
#pragma unroll
    for (int w0 = 0; w0 < kSub2dWords; w0 += 8) {
      int32_t c[8];
      st_load8<T>(o, w0, c);
#pragma unroll
      for (int u = 0; u < 8; ++u) a[w0 + u] += c[u];
    }
  }
  __syncwarp();
#pragma unroll
  for (int w0 = 0; w0 < kSub2dWords; w0 += 8) {
    int32_t c[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) c[u] = a[w0 + u];
    st_store8<T>(st, w0, c);
  }
  // ---- pass 2: reconstruct the chunk's rows from the buffered residuals
  if (live) {
    Side sd;
    init_side(p, sd, cpos);
    Prefix pf;
    pf.r1 = 0;
    pf.r2 = 0;
#pragma unroll 1
    for (uint32_t gi = 0; gi < kNg; ++gi) {
      const int4 w = buf[gi * T];
      const uint32_t wv[4] = {(uint32_t)w.x, (uint32_t)w.y, (uint32_t)w.z, (uint32_t)w.w};
      int32_t d[8];
      bool zero = false;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        d[2 * i] = (int32_t)(wv[i] << 16) >> 16;
        d[2 * i + 1] = (int32_t)wv[i] >> 16;
        zero = zero || d[2 * i] == -p.R || d[2 * i + 1] == -p.R;
      }
      if (zero) fix_outliers(p, sd, j, cpos, cpos + gi * 8, d, bad);
      if (gi == 0 && sub == 0) d[0] += anchor;
      consume<2, 1, EXC, T>(p, g, sd, pf, st, (int)(sub * kNg + gi), d, pos0, X0, Y0, 0, vecbase, anchor);
    }
  }
  if (bad) dec_err(p.err, FZ_ECORRUPT);
}

template <int C>
__global__ void __launch_bounds__(Sub2d<C>::T) k_decode_sub2d(DecParams p, Geom g) {
  constexpr int T = Sub2d<C>::T;
  extern __shared__ __align__(16) unsigned char d_smem[];
  uint16_t *slut = reinterpret_cast<uint16_t *>(d_smem);
  int32_t *sstate = reinterpret_cast<int32_t *>(d_smem + sizeof(uint16_t) * kLutSize);
  uint32_t *sring = reinterpret_cast<uint32_t *>(sstate + kSub2dWords * T);
  int4 *sbuf = reinterpret_cast<int4 *>(sring + kRing * T);
  __shared__ LutBuild lb;
  const bool ok = build_lut<T>(p.lens, p.nsym, p.R, slut, lb);
  dep_wait();  // the unit offsets
  if (ok) {
    __syncthreads();
    const int t = threadIdx.x, lane = t & 31;
    const bool vecbase = (g.nx & 3u) == 0 && (((uintptr_t)p.out & 15u) == 0);
    for (;;) {
      const uint32_t u = claim_unit(p.err + 1);
      if (u >= p.n_units) break;
      uint32_t cb;
      const uint64_t start = unit_start(p.chunk_bits, p.goff, p.n_chunks, u, cb);
      const uint64_t j = (uint64_t)u * kDecUnit + lane;
      const bool live = j < p.n_chunks;
      if (p.n_exc) decode_sub2d_chunk<C, true>(p, g, slut, sstate, sring + t, sbuf + t, j, start, cb, live, vecbase);
      else decode_sub2d_chunk<C, false>(p, g, slut, sstate, sring + t, sbuf + t, j, start, cb, live, vecbase);
    }
  } else if (threadIdx.x == 0) {
    dec_err(p.err, FZ_ECORRUPT);
  }
  __syncthreads();
  if (p.h_err && threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(p.err + 2, 1u) == gridDim.x - 1) {
      __threadfence();
      *reinterpret_cast<volatile uint32_t *>(p.h_err) = atomicAdd(p.err, 0u);
      __threadfence_system();
    }
  }
}

template <int C>
cudaError_t launch_sub2d_t(const DecParams &p, const Geom &g, int sm_count, cudaStream_t s) {
  constexpr int T = Sub2d<C>::T;
  const int smem = (int)Sub2d<C>::kSmem;
  static LaunchCache cache;
  int per_sm = 0;
  const cudaError_t e = cached_per_sm(k_decode_sub2d<C>, T, smem, cache, per_sm);
  if (e != cudaSuccess) return e;
  uint64_t grid = (uint64_t)sm_count * per_sm;
  const uint64_t need = (p.n_units + T / 32 - 1) / (T / 32);  // CTAs whose warps all have a unit
  if (grid > need) grid = need;
  return launch_dep(k_decode_sub2d<C>, (unsigned)grid, (unsigned)T, (size_t)smem, s, p, g);
}

cudaError_t launch_sub2d(const DecParams &p, const Geom &g, int sm_count, cudaStream_t s) {
  if (g.chunk == 128) return launch_sub2d_t<128>(p, g, sm_count, s);
  if (g.chunk == 256) return launch_sub2d_t<256>(p, g, sm_count, s);
  return launch_sub2d_t<512>(p, g, sm_count, s);
}

// ---------------------------------------------------------------- 64-symbol chunks (3D)
// A stream whose Huffman chunk is one 8x8 plane of a block (64 symbols) is
// decoded plane-parallel: a work unit of 32 chunks is 4 blocks x 8 planes,
// lane l of the warp decodes plane l & 7 of block 4u + (l >> 3).  Per row
// y, each lane forms the x and y prefix sums of its plane's row (the first
// two of the three inverse-Lorenzo sums); an 8x8 transpose through a small
// per-warp shared tile then gives lane (group, x) the eight planes' values
// at column x, whose prefix sum along z completes the inverse in
// registers.  So no lane keeps a plane of prefix state (the one-block-per-
// lane decoder needs 256 bytes of it per thread), and the eight stores of a
// row (one per z) each cover 4 blocks x 8 floats of one field row.
// Exceptions are written by k_exc_scatter afterwards.
#ifndef FZ_DEC_TP
#define FZ_DEC_TP 768
#endif
constexpr int kPlaneT = FZ_DEC_TP;
constexpr int kPlaneTile = 4 * 72;  // per warp: 4 blocks x (8 planes x 8 values + 8 words of padding)

template <int K, int T>
__device__ __forceinline__ void decode_plane_unit(const DecParams &p, const Geom &g, const uint16_t *slut,
                                                  uint32_t *ring, int32_t *tile, uint64_t u) {
  const int lane = threadIdx.x & 31, zpl = lane & 7, grp = lane >> 3;
  uint32_t cb;
  const uint64_t start = unit_start(p.chunk_bits, p.goff, p.n_chunks, u, cb);
  const uint64_t j = u * kDecUnit + (uint64_t)lane;
  const bool valid = j < p.n_chunks;  // n_chunks is 8 n_blocks: a block's 8 lanes agree
  const uint64_t blk = valid ? j >> 3 : 0;
  bool bad = false;
  BitReader<T> br;
  br.init(p.words, p.n_words, valid ? start : 0, valid ? cb : 0, ring);
  const uint32_t start_off = br.off;
  const uint32_t pos0 = (uint32_t)(blk * 512u) + (uint32_t)zpl * 64u;  // this lane's plane
  Side sd;
  sd.oc = ~0ull;
  sd.next_o = 0xffffffffu;
  sd.next_v = 0;
  const uint32_t b32 = (uint32_t)blk;
  const uint32_t bxi = b32 % g.nbx, br_ = b32 / g.nbx;
  const uint32_t byi = br_ % g.nby, bzi = br_ / g.nby;
  const uint32_t X0 = bxi * 8u, Y0 = byi * 8u, Z0 = bzi * 8u;
  // after the transpose this lane writes column x = zpl of the block
  const bool xin = valid && X0 + (uint32_t)zpl < g.nx;
  const uint32_t nz_in = g.nz - Z0 < 8u ? g.nz - Z0 : 8u;
  const uint64_t plane = (uint64_t)g.ny * g.nx;
  int32_t Y1[8], Y2[8];
#pragma unroll
  for (int x = 0; x < 8; ++x) { Y1[x] = 0; Y2[x] = 0; }
  int32_t *trow = tile + grp * 72;
  int32_t cur[8];
  if (br.group8(slut, p.R, cur)) fix_outliers(p, sd, blk, pos0, pos0, cur, bad);
  if (zpl == 0 && valid) cur[0] += __ldg(p.anchors + blk);  // the block origin's residual is its anchor
#pragma unroll 1
  for (int y = 0; y < 8; ++y) {
    int32_t nxt[8];
    bool zn = false;
    if (y < 7) zn = br.group8(slut, p.R, nxt);
    // x and y prefix sums of this plane's row y
    int32_t v[8], r1 = 0, r2 = 0;
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      r1 += cur[x];
      if (K == 1) {
        Y1[x] += r1;
        v[x] = Y1[x];
      } else {
        r2 += r1;
        Y1[x] += r2;
        Y2[x] += Y1[x];
        v[x] = Y2[x];
      }
    }
    // transpose within the block's 8 lanes: lane (grp, x) gets w[z]
    __syncwarp();
    reinterpret_cast<int4 *>(trow + zpl * 8)[0] = make_int4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<int4 *>(trow + zpl * 8)[1] = make_int4(v[4], v[5], v[6], v[7]);
    __syncwarp();
    int32_t w[8];
#pragma unroll
    for (int z = 0; z < 8; ++z) w[z] = trow[z * 8 + zpl];
    // z prefix sum(s), dequantization and the row's eight stores
#pragma unroll
    for (int z = 1; z < 8; ++z) w[z] += w[z - 1];
    if (K == 2) {
#pragma unroll
      for (int z = 1; z < 8; ++z) w[z] += w[z - 1];
    }
    if (xin && Y0 + (uint32_t)y < g.ny) {
      uint64_t f = ((uint64_t)Z0 * g.ny + Y0 + (uint32_t)y) * g.nx + X0 + (uint32_t)zpl;
#pragma unroll
      for (int z = 0; z < 8; ++z) {
        if ((uint32_t)z < nz_in) p.out[f] = __fmul_rn(__int2float_rn(w[z]), p.ebx2);
        f += plane;
      }
    }
    if (y < 7) {
      if (zn) fix_outliers(p, sd, blk, pos0, pos0 + (uint32_t)(y + 1) * 8u, nxt, bad);
#pragma unroll
      for (int x = 0; x < 8; ++x) cur[x] = nxt[x];
    }
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");  // the ring is reused by the next unit
  if (valid && (br.consumed(start_off) != cb || bad)) dec_err(p.err, FZ_ECORRUPT);
}

// One CTA per SM, as k_decode: every CTA builds the decode table, every warp
// claims work units from the counter.
template <int K>
__global__ void __launch_bounds__(kPlaneT, 1) k_decode_planes(DecParams p, Geom g) {
  constexpr int T = kPlaneT;
  extern __shared__ __align__(16) unsigned char d_smem[];
  uint16_t *slut = reinterpret_cast<uint16_t *>(d_smem);
  uint32_t *sring = reinterpret_cast<uint32_t *>(d_smem + sizeof(uint16_t) * kLutSize);
  int32_t *stile = reinterpret_cast<int32_t *>(sring + kRing * T);
  __shared__ LutBuild lb;
  const int t = threadIdx.x;
  if (build_lut<T>(p.lens, p.nsym, p.R, slut, lb)) {
    __syncthreads();
    int32_t *tile = stile + (t >> 5) * kPlaneTile;
    for (;;) {
      const uint32_t u = claim_unit(p.err + 1);
      if (u >= p.n_units) break;
      decode_plane_unit<K, T>(p, g, slut, sring + t, tile, u);
    }
  } else if (t == 0) {
    dec_err(p.err, FZ_ECORRUPT);
  }
  __syncthreads();
  if (p.h_err && t == 0) {
    __threadfence();
    if (atomicAdd(p.err + 2, 1u) == gridDim.x - 1) {
      __threadfence();
      *reinterpret_cast<volatile uint32_t *>(p.h_err) = atomicAdd(p.err, 0u);
      __threadfence_system();
    }
  }
}

constexpr size_t plane_smem_bytes() {
  return sizeof(uint16_t) * kLutSize + sizeof(uint32_t) * kRing * kPlaneT +
         sizeof(int32_t) * kPlaneTile * (kPlaneT / 32);
}

// Exceptions of a stream decoded plane-parallel: each stored value
// overwrites its position (code-stream index in 8x8x8 blocks -> field
// index).  The list must ascend strictly and name in-domain points.  The
// last CTA hands the error word to the host when asked.
__global__ void k_exc_scatter(const uint32_t *__restrict__ exc_idx, const uint32_t *__restrict__ exc_val,
                              uint64_t n_exc, Geom g, float *out, uint32_t *err, uint32_t *h_err) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_exc;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t pos = __ldg(exc_idx + i);
    const uint32_t b = pos >> 9, w = pos & 511u;
    const uint32_t x = (b % g.nbx) * 8u + (w & 7u), r = b / g.nbx;
    const uint32_t y = (r % g.nby) * 8u + ((w >> 3) & 7u), z = (r / g.nby) * 8u + (w >> 6);
    const bool ok = (uint64_t)b < g.n_blocks && x < g.nx && y < g.ny && z < g.nz &&
                    (i == 0 || __ldg(exc_idx + i - 1) < pos);
    if (ok) out[((uint64_t)z * g.ny + y) * g.nx + x] = __uint_as_float(__ldg(exc_val + i));
    else dec_err(err, FZ_ECORRUPT);
  }
  __syncthreads();
  if (h_err && threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(err + 2, 1u) == gridDim.x - 1) {
      __threadfence();
      *reinterpret_cast<volatile uint32_t *>(h_err) = atomicAdd(err, 0u);
      __threadfence_system();
    }
  }
}

template <int K>
cudaError_t launch_planes_t(const DecParams &p, const Geom &g, int sm_count, cudaStream_t s) {
  const int smem = (int)plane_smem_bytes();
  static LaunchCache cache;
  int per_sm = 0;
  const cudaError_t e = cached_per_sm(k_decode_planes<K>, kPlaneT, smem, cache, per_sm);
  if (e != cudaSuccess) return e;
  uint64_t grid = (uint64_t)sm_count * per_sm;
  if (grid > p.n_units) grid = p.n_units;
  DecParams q = p;
  if (p.n_exc) q.h_err = nullptr;  // the exception pass reports instead
  k_decode_planes<K><<<(unsigned)grid, kPlaneT, smem, s>>>(q, g);
  cudaError_t e2 = cudaGetLastError();
  if (e2 != cudaSuccess || !p.n_exc) return e2;
  uint64_t eg = (p.n_exc + 255) / 256;
  if (eg > (uint64_t)sm_count * 4) eg = (uint64_t)sm_count * 4;
  k_exc_scatter<<<(unsigned)eg, 256, 0, s>>>(p.exc_idx, p.exc_val, p.n_exc, g, p.out, p.err, p.h_err);
  return cudaGetLastError();
}

template <int T>
__device__ __forceinline__ void load_lut(uint16_t *slut, const uint16_t *lut) {
  const uint4 *src = reinterpret_cast<const uint4 *>(lut);
  uint4 *dst = reinterpret_cast<uint4 *>(slut);
  for (int i = threadIdx.x; i < kLutSize / 8; i += T) dst[i] = __ldg(src + i);
}

// One CTA per SM; every warp takes work units (32 chunks, one per lane)
// from a counter, so uneven chunks and small fields still spread over all
// SMs.
template <int NDIM, int K, bool NS>
__global__ void __launch_bounds__(DecCta<NDIM, K, NS>::T, 1) k_decode(DecParams p, Geom g) {
  constexpr int T = DecCta<NDIM, K, NS>::T;
  extern __shared__ __align__(16) unsigned char d_smem[];
  uint16_t *slut = reinterpret_cast<uint16_t *>(d_smem);
  int32_t *sstate = reinterpret_cast<int32_t *>(d_smem + sizeof(uint16_t) * kLutSize);
  uint32_t *sring = reinterpret_cast<uint32_t *>(sstate + DecState<NDIM, K, NS>::kWords * T);
  __shared__ LutBuild lb;
  // A gated pair (the 16-bit-state decoder, then the 32-bit one) decodes a
  // stream whose exceptions the offset pass checked: exactly one of the two
  // runs.  The second is launched once every CTA of the first has ended, so
  // the offset pass's verdict (err[4]) is final when it starts.
  const volatile uint32_t *verdict = p.err + 4;
  if (p.gate == 2 && *verdict == 0) return;
  // every CTA builds the decode table from the 1 KB length table itself (an
  // input of the call: it overlaps the offset pass, launched before)
  const bool ok = build_lut<T>(p.lens, p.nsym, p.R, slut, lb);
  dep_wait();  // the unit offsets
  if (p.gate == 1 && *verdict != 0) return;
  if (ok) {
    __syncthreads();
    decode_units<NDIM, K, NS>(p, g, slut, sstate, sring);
  } else if (threadIdx.x == 0) {
    dec_err(p.err, FZ_ECORRUPT);
  }
  // the last CTA to finish hands the error word to the host directly
  __syncthreads();
  if (p.h_err && threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(p.err + 2, 1u) == gridDim.x - 1) {
      __threadfence();
      *reinterpret_cast<volatile uint32_t *>(p.h_err) = atomicAdd(p.err, 0u);
      __threadfence_system();
    }
  }
}

// ---------------------------------------------------------------- batched decode
// One field of a batched decompress (Huffman streams only).
struct DecJob {
  DecParams p;
  Geom g;
  const uint8_t *lens;
  uint32_t nsym, pad;
  uint64_t total_bits;
  uint64_t unit_base;   // first work unit in the job's class queue
};

// Work-unit bit sums of every field: blockIdx.y = field.
__global__ void k_dec_gsum_batch(const DecJob *__restrict__ jobs) {
  const DecJob &J = jobs[blockIdx.y];
  const uint64_t u = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= J.p.n_units) return;
  const uint64_t j = u * kDecUnit + lane;
  uint32_t v = j < J.p.n_chunks ? __ldg(J.p.chunk_bits + j) : 0u;
  v = __reduce_add_sync(0xffffffffu, v);
  if (lane == 0) const_cast<uint64_t *>(J.p.goff)[u] = v;
}

// Decode tables and unit offsets: one CTA per field.
__global__ void __launch_bounds__(kPrepThreads) k_dec_prep_batch(const DecJob *__restrict__ jobs) {
  const DecJob &J = jobs[blockIdx.x];
  k_dec_prep_body(J.lens, J.nsym, J.p.R, const_cast<uint64_t *>(J.p.goff), J.p.n_units, J.total_bits,
                  const_cast<uint16_t *>(J.p.lut), J.p.err);
}

// The work units of every field of one class (dimensionality, Lorenzo
// order) form one queue cut into equal contiguous ranges, one per CTA; the
// CTA's warps share the units of each field in its range, and the decode
// table is reloaded when the CTA moves to another field.
template <int NDIM, int K>
__global__ void __launch_bounds__(DecCta<NDIM, K>::T, 1) k_decode_batch(const DecJob *__restrict__ jobs,
                                                                         const uint32_t *__restrict__ members,
                                                                         uint32_t n_members, uint64_t total_units) {
  constexpr int T = DecCta<NDIM, K>::T;
  constexpr int kWarps = T / 32;
  extern __shared__ __align__(16) unsigned char d_smem[];
  uint16_t *slut = reinterpret_cast<uint16_t *>(d_smem);
  int32_t *sstate = reinterpret_cast<int32_t *>(d_smem + sizeof(uint16_t) * kLutSize);
  uint32_t *sring = reinterpret_cast<uint32_t *>(sstate + DecState<NDIM, K>::kWords * T);
  __shared__ DecParams sp;
  __shared__ Geom sg;
  const int t = threadIdx.x, warp = t >> 5;
  const uint64_t lo = total_units * blockIdx.x / gridDim.x, hi = total_units * (blockIdx.x + 1) / gridDim.x;
  uint32_t a = 0, b = n_members;
  while (a < b) {
    const uint32_t m = (a + b) >> 1;
    const DecJob &J = jobs[members[m]];
    if (J.unit_base + J.p.n_units <= lo) a = m + 1; else b = m;
  }
  for (uint64_t r = lo; r < hi && a < n_members; ++a) {
    const DecJob &J = jobs[members[a]];
    const uint64_t jb = J.unit_base, je = jb + J.p.n_units;
    const uint64_t t0 = r > jb ? r : jb, t1 = hi < je ? hi : je;
    __syncthreads();  // the previous field is done with the table and the staged parameters
    if (t == 0) { sp = J.p; sg = J.g; }
    load_lut<T>(slut, J.p.lut);
    __syncthreads();
    const bool vecbase = (NDIM == 1 || (sg.nx & 3u) == 0) && (((uintptr_t)sp.out & 15u) == 0);
    for (uint64_t u = t0 - jb + warp; u < t1 - jb; u += kWarps) {
      uint32_t cb;
      const uint64_t start = unit_start(sp.chunk_bits, sp.goff, sp.n_chunks, u, cb);
      const uint64_t j = u * kDecUnit + (t & 31);
      if (j < sp.n_chunks) {
        const uint32_t k = sg.chunk / sg.bsize;  // blocks per chunk
        const uint64_t jb = j * k;
        const uint32_t nblk = (uint32_t)(sg.n_blocks - jb < k ? sg.n_blocks - jb : k);
        int32_t *st = st_thread(sstate, t);
        if (sp.n_exc) decode_chunk<NDIM, K, true, T>(sp, sg, slut, st, sring + t, jb, nblk, start, cb, vecbase);
        else decode_chunk<NDIM, K, false, T>(sp, sg, slut, st, sring + t, jb, nblk, start, cb, vecbase);
      }
    }
    r = t1;
  }
}

template <int NDIM, int K, bool NS = false>
cudaError_t launch_dec_t(const DecParams &p, const Geom &g, int sm_count, cudaStream_t s) {
  constexpr int T = DecCta<NDIM, K, NS>::T;
  const int smem = (int)dec_smem_bytes<NDIM, K, NS>();
  static LaunchCache cache;
  int per_sm = 0;
  const cudaError_t e = cached_per_sm(k_decode<NDIM, K, NS>, T, smem, cache, per_sm);
  if (e != cudaSuccess) return e;
  // at most one CTA per unit: the units of a small field spread over SMs
  uint64_t grid = (uint64_t)sm_count * per_sm;
  if (grid > p.n_units) grid = p.n_units;
  return launch_dep(k_decode<NDIM, K, NS>, (unsigned)grid, (unsigned)T, (size_t)smem, s, p, g);
}

}  // namespace

// Whether the 16-bit relative plane state may decode the stream (3D,
// first-order Lorenzo, chunks of whole blocks, REL bound eb >= 2^-15): every
// quantized value q then lies within range * inv2eb + 2 <= 1 / (2 eb) + 2 <=
// 16386 of its block's anchor -- both are prequantized finite values in [lo,
// hi] (|x * inv2eb| < 2^23, so each product and each rounding to an integer
// is off by at most 1/2), and inv2eb = 1 / (2 eb (hi - lo)) up to float
// rounding.  Exceptions whose value was quantized (a rounding check that
// failed) keep that bound; one that was not (non-finite, or |x * inv2eb| of
// 2^23 or more) has q = 0, which may lie anywhere relative to its anchor, so
// a stream with exceptions needs the offset pass's check of their values.
constexpr uint64_t kNarrowPairUnits = 4096;  // work units from which a stream with exceptions tries the 16-bit state
static bool narrow_state_candidate(const fz_header &h) {
#if FZ_DEC_NARROW
  return h.ndim == 3 && h.predictor == FZ_PRED_LORENZO1 && h.flags == 0 && h.chunk >= 512 &&
         h.eb_mode == FZ_EB_REL && h.eb >= 1.0 / 32768.0;
#else
  (void)h;
  return false;
#endif
}

cudaError_t launch_decode_prep(const uint8_t *d_in, const fz_header &h, const DecodeWs &ws, cudaStream_t s) {
  const uint64_t n_chunks = h.n_chunks;
  const uint64_t n_units = dec_units_of(n_chunks);
  const uint32_t *cbits = reinterpret_cast<const uint32_t *>(d_in + h.off_chunk_bits);
  k_dec_gsum<<<(unsigned)((n_units * 32 + 255) / 256), 256, 0, s>>>(cbits, n_chunks, n_units, ws.gsum);
  k_dec_prep<<<1, kPrepThreads, 0, s>>>(d_in + h.off_lens, 2 * h.radius, ws.gsum, n_units, h.total_bits, ws.lut,
                                        ws.err);
  return cudaGetLastError();
}

namespace {
// First outlier of every block that has outliers (the list ascends by
// position).  Blocks without outliers keep the ~0 the caller filled in; a
// decoder that meets an outlier code there finds no outlier at that index
// and reports a corrupt stream.
__global__ void k_outlier_starts(const uint32_t *__restrict__ out_idx, uint64_t n_out, uint32_t bsize,
                                 uint64_t n_blocks, uint32_t *ofirst) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_out;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = __ldg(out_idx + i) / bsize;
    if (c < n_blocks && (i == 0 || __ldg(out_idx + i - 1) / bsize != c)) ofirst[c] = (uint32_t)i;
  }
}
}  // namespace

cudaError_t launch_exc_scatter(const uint8_t *d_in, const fz_header &h, float *d_out, uint32_t *err, uint32_t *h_err,
                               cudaStream_t s, int sm_count) {
  Geom g;
  make_geom(h.ndim, h.dims, g);
  uint64_t eg = (h.n_exc + 255) / 256;
  if (eg > (uint64_t)sm_count * 4) eg = (uint64_t)sm_count * 4;
  if (eg == 0) eg = 1;
  k_exc_scatter<<<(unsigned)eg, 256, 0, s>>>(reinterpret_cast<const uint32_t *>(d_in + h.off_exc_idx),
                                             reinterpret_cast<const uint32_t *>(d_in + h.off_exc_val), h.n_exc, g,
                                             d_out, err, h_err);
  return cudaGetLastError();
}

cudaError_t launch_outlier_starts(const uint8_t *d_in, const fz_header &h, const DecodeWs &ws, cudaStream_t s,
                                  int sm_count) {
  Geom g;
  make_geom(h.ndim, h.dims, g);
  uint64_t grid = (h.n_out + 255) / 256;
  if (grid > (uint64_t)sm_count * 8) grid = (uint64_t)sm_count * 8;
  if (grid < 1) grid = 1;
  k_outlier_starts<<<(unsigned)grid, 256, 0, s>>>(reinterpret_cast<const uint32_t *>(d_in + h.off_out_idx), h.n_out,
                                                  g.bsize, h.n_blocks, ws.ofirst);
  return cudaGetLastError();
}

namespace {
constexpr int kOffThreads = 256;  // work units per CTA of k_dec_offsets (one per thread)

// First bit of every work unit in one pass: thread = unit, the unit's bit
// total from its 32 chunk lengths (128 contiguous bytes), a CTA scan, and a
// bounded decoupled look-back over the CTAs for the CTA's base.  A CTA's
// range of units is the ticket it draws from a counter (err[3]) when it
// starts, not its blockIdx: every predecessor in ticket order has started
// and will publish, whatever order the hardware dispatches the CTAs in.  The
// control words are err[0] error word, err[1] work-unit counter, err[2] CTA
// counter, err[3] ticket, err[4] set when an exception is out of the
// quantizer's range (see below), err[5..7] unused; the status words follow;
// everything starts at zero.  With n_scan > 0 the pass also checks the
// stream's n_scan exception values: one that was not quantized (non-finite,
// or |x * inv2eb| not below 2^23, exactly the quantizer's test) sets err[4]
// -- its q of 0 may lie far from its block's anchor, which rules out the
// decoder's 16-bit plane state.
__global__ void __launch_bounds__(kOffThreads) k_dec_offsets(const uint32_t *__restrict__ chunk_bits,
                                                             uint64_t n_chunks, uint64_t n_units,
                                                             uint64_t total_bits, uint64_t *uoff, uint32_t *err,
                                                             long long spin, const uint32_t *__restrict__ exc_val,
                                                             uint64_t n_scan, float inv2eb) {
  dep_trigger();  // the decoder builds its table meanwhile
  __shared__ unsigned long long wsum[kOffThreads / 32];
  __shared__ unsigned long long s_base;
  __shared__ uint32_t s_tile;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  uint64_t *status = reinterpret_cast<uint64_t *>(err + kDecCtlWords);
  if (n_scan) {
    bool out = false;
    for (uint64_t i = (uint64_t)blockIdx.x * kOffThreads + t; i < n_scan; i += (uint64_t)gridDim.x * kOffThreads)
      out |= !(fabsf(__fmul_rn(__uint_as_float(__ldg(exc_val + i)), inv2eb)) < 8388608.0f);
    if (__any_sync(0xffffffffu, out) && lane == 0) atomicOr(err + 4, 1u);
  }
  if (t == 0) s_tile = atomicAdd(err + 3, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t u = (uint64_t)tile * kOffThreads + t;
  unsigned long long v = 0;
  if (u < n_units) {
    const uint64_t c0 = u * kDecUnit;
    if (c0 + kDecUnit <= n_chunks && ((uintptr_t)(chunk_bits + c0) & 15u) == 0) {
      const uint4 *p = reinterpret_cast<const uint4 *>(chunk_bits + c0);
#pragma unroll
      for (int k = 0; k < kDecUnit / 4; ++k) {
        const uint4 w = __ldg(p + k);
        v += (unsigned long long)w.x + w.y + w.z + w.w;
      }
    } else {
      for (uint64_t c = c0; c < n_chunks && c < c0 + kDecUnit; ++c) v += __ldg(chunk_bits + c);
    }
  }
  unsigned long long incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long x = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += x;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  unsigned long long wpre = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kOffThreads / 32; ++w) {
    wpre += w < warp ? wsum[w] : 0ull;
    tot += wsum[w];
  }
  if (warp == 0) {
    if (lane == 0) lookback_publish(status, tile, tot);
    const unsigned long long base = lookback_resolve_warp(status, tile, tot, err, spin);
    if (lane == 0) {
      s_base = base;
      if (tile == gridDim.x - 1 && base + tot != total_bits) dec_err(err, FZ_ECORRUPT);
    }
  }
  __syncthreads();
  if (u < n_units) uoff[u] = s_base + wpre + incl - v;
}
}  // namespace

namespace {
// A look-back whose one predecessor never publishes: the bounded wait must
// give up after `spin` cycles and record FZ_ETIMEOUT in err[0].
__global__ void k_lookback_selftest(uint64_t *status, uint32_t *err, long long spin) {
  lookback_resolve_warp(status, 1, 1, err, spin);
}
}  // namespace

cudaError_t launch_lookback_selftest(uint32_t *scratch, long long spin, cudaStream_t s) {
  k_lookback_selftest<<<1, 32, 0, s>>>(reinterpret_cast<uint64_t *>(scratch + 4), scratch, spin);
  return cudaGetLastError();
}

uint64_t dec_offset_zero_bytes(const fz_header &h) {
  return 4 * kDecCtlWords + 8 * ((dec_units_of(h.n_chunks) + kOffThreads - 1) / kOffThreads);
}

cudaError_t launch_decode_offsets(const uint8_t *d_in, const fz_header &h, const DecodeWs &ws, cudaStream_t s) {
  const uint64_t n_chunks = h.n_chunks;
  const uint64_t n_units = dec_units_of(n_chunks);
  const uint32_t *cbits = reinterpret_cast<const uint32_t *>(d_in + h.off_chunk_bits);
  const uint64_t grid = (n_units + kOffThreads - 1) / kOffThreads;
  // the exception values are checked for the 16-bit-state decoder's choice
  const uint64_t n_scan =
      (narrow_state_candidate(h) && h.flags == 0 && n_units >= kNarrowPairUnits) ? h.n_exc : 0;
  float inv2eb;
  memcpy(&inv2eb, &h.inv2eb_bits, 4);
  k_dec_offsets<<<(unsigned)grid, kOffThreads, 0, s>>>(cbits, n_chunks, n_units, h.total_bits, ws.gsum, ws.err,
                                                       ws.spin,
                                                       reinterpret_cast<const uint32_t *>(d_in + h.off_exc_val),
                                                       n_scan, inv2eb);
  return cudaGetLastError();
}

cudaError_t launch_decode_main(const uint8_t *d_in, const fz_header &h, float *d_out, const DecodeWs &ws,
                               cudaStream_t s, int sm_count) {
  Geom g;
  make_geom(h.ndim, h.dims, g);
  set_chunk(g, h.chunk);
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
  p.n_units = dec_units_of(h.n_chunks);
  p.goff = ws.gsum;
  p.lens = d_in + h.off_lens;
  p.ofirst = ws.ofirst;
  p.nsym = 2 * h.radius;
  p.total_bits = h.total_bits;
  p.lut = ws.lut;
  p.err = ws.err;
  p.h_err = ws.h_err;
  p.out = d_out;
  memcpy(&p.ebx2, &h.ebx2_bits, 4);
  p.R = (int32_t)h.radius;
  const bool k2 = h.predictor == FZ_PRED_LORENZO2;
  if (h.flags == FZ_FLAG_SHUF) return launch_shuf_decode(d_in, h, d_out, ws, s, sm_count);
  if (g.ndim == 2 && g.chunk < g.bsize) {
    p.ofirst = nullptr;  // outliers are located per chunk by search
    return launch_sub2d(p, g, sm_count, s);
  }
  if (g.ndim == 3 && g.chunk == 64) {
    p.ofirst = nullptr;  // outliers are located per plane by search
    return k2 ? launch_planes_t<2>(p, g, sm_count, s) : launch_planes_t<1>(p, g, sm_count, s);
  }
  switch (g.ndim) {
    case 1: return k2 ? launch_dec_t<1, 2>(p, g, sm_count, s) : launch_dec_t<1, 1>(p, g, sm_count, s);
    case 2: return k2 ? launch_dec_t<2, 2>(p, g, sm_count, s) : launch_dec_t<2, 1>(p, g, sm_count, s);
    default: {
      if (k2) return launch_dec_t<3, 2>(p, g, sm_count, s);
      if (!narrow_state_candidate(h)) return launch_dec_t<3, 1>(p, g, sm_count, s);
      if (h.n_exc == 0) return launch_dec_t<3, 1, true>(p, g, sm_count, s);
      // exceptions: the offset pass has checked their values; the 16-bit
      // decoder runs if all were quantized, else the 32-bit one.  The pair's
      // second launch only pays on large streams (256^3 field, 1024 units:
      // 112 against 100 us for the 32-bit decoder alone; 640^3: 525 against
      // 587 us)
      if (p.n_units < kNarrowPairUnits) return launch_dec_t<3, 1>(p, g, sm_count, s);
      p.gate = 1;
      const cudaError_t e = launch_dec_t<3, 1, true>(p, g, sm_count, s);
      if (e != cudaSuccess) return e;
      p.gate = 2;
      return launch_dec_t<3, 1>(p, g, sm_count, s);
    }
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
                               uint64_t total_units, int per_sm, cudaStream_t s, int sms) {
  constexpr int T = DecCta<NDIM, K>::T;
  const int smem = (int)dec_smem_bytes<NDIM, K>();
  cudaError_t e = cudaFuncSetAttribute(k_decode_batch<NDIM, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_decode_batch<NDIM, K>, T, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  if (per_sm < 1 || per_sm > occ) per_sm = occ;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > total_units) grid = total_units;
  if (grid < 1) grid = 1;
  k_decode_batch<NDIM, K><<<(unsigned)grid, T, smem, s>>>(jobs, members, n_members, total_units);
  return cudaGetLastError();
}
}  // namespace

size_t dec_job_bytes() { return sizeof(DecJob); }
size_t plain_job_bytes() { return sizeof(PlainJob); }
uint64_t dec_units(const fz_header &h) { return dec_units_of(h.n_chunks); }

void fill_dec_job(void *dst, const uint8_t *d_in, const fz_header &h, float *d_out, uint16_t *lut, uint64_t *gsum,
                  uint32_t *err, uint64_t unit_base) {
  DecJob J;
  memset(&J, 0, sizeof(J));
  make_geom(h.ndim, h.dims, J.g);
  set_chunk(J.g, h.chunk);
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
  p.n_units = dec_units(h);
  p.goff = gsum;
  p.lut = lut;
  p.err = err;
  p.out = d_out;
  memcpy(&p.ebx2, &h.ebx2_bits, 4);
  p.R = (int32_t)h.radius;
  J.lens = d_in + h.off_lens;
  J.nsym = 2 * h.radius;
  p.lens = d_in + h.off_lens;
  p.ofirst = nullptr;
  J.total_bits = h.total_bits;
  J.unit_base = unit_base;
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

cudaError_t launch_decode_batch_prep(const void *jobs, uint32_t n, uint64_t max_units, cudaStream_t s) {
  const DecJob *J = reinterpret_cast<const DecJob *>(jobs);
  const uint64_t gx = (max_units * 32 + 255) / 256;
  k_dec_gsum_batch<<<dim3((unsigned)gx, n), 256, 0, s>>>(J);
  k_dec_prep_batch<<<n, kPrepThreads, 0, s>>>(J);
  return cudaGetLastError();
}

cudaError_t launch_decode_batch_main(int ndim, int k, const void *jobs, const uint32_t *members, uint32_t n_members,
                                     uint64_t total_units, int per_sm, cudaStream_t s, int sms) {
  const DecJob *J = reinterpret_cast<const DecJob *>(jobs);
  const bool k2 = k == 2;
  switch (ndim) {
    case 1:
      return k2 ? launch_dec_batch_t<1, 2>(J, members, n_members, total_units, per_sm, s, sms)
                : launch_dec_batch_t<1, 1>(J, members, n_members, total_units, per_sm, s, sms);
    case 2:
      return k2 ? launch_dec_batch_t<2, 2>(J, members, n_members, total_units, per_sm, s, sms)
                : launch_dec_batch_t<2, 1>(J, members, n_members, total_units, per_sm, s, sms);
    default:
      return k2 ? launch_dec_batch_t<3, 2>(J, members, n_members, total_units, per_sm, s, sms)
                : launch_dec_batch_t<3, 1>(J, members, n_members, total_units, per_sm, s, sms);
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
