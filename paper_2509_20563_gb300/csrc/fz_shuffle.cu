// fz_shuffle.cu -- the bit-shuffle + zero-word encoder of FZMod-Speed
// (FZModules §3.2-§3.3: the encoder FZ-GPU uses, in place of Huffman coding),
// on the same quantization codes as the Huffman path.
//
// Format (flag FZ_FLAG_SHUF): the residual d = code - R of every code (code
// 0 = outlier, d = -R) becomes the zig-zag value v = 2d or -2d - 1 (v < 2R).
// Each run of 64 codes is a 32x32 bit matrix, row r = v[2r] | v[2r+1] << 16,
// whose transpose gives 32 column words; a 32-bit map per run (the section
// where Huffman streams keep their code lengths) flags the nonzero words, and
// only those are stored, in column order, in the bitstream section.  A tile
// of 1024 codes is one chunk; its stored length is 32 bits per word.
//
// GPU mapping: a warp holds one run as one 32-bit row per lane, and the
// transpose is five exchange stages of shuffle, funnel shift and logic op --
// the same instructions decode (the transpose is its own inverse).  There is
// no serial decode chain: every run decodes independently.
//   k_shuf_layout -- header and section offsets once the code counts are known
//   k_shuf_encode -- warps take 4096-code units from a ticket counter, stage
//                    their words in shared memory, place them after a bounded
//                    decoupled look-back, and the last unit completes the
//                    header (or turns the stream into a RAW one)
//   k_shuf_decode -- warps take groups of four chunks; per chunk the runs'
//                    words are gathered and transposed back, outliers patched
//                    in, and the inverse Lorenzo (x and y across lanes, z in
//                    registers for 3D) and dequantization done in registers
#include <string.h>

#include "fz_decode_common.cuh"

namespace fz {
namespace {

// Transpose of the 32x32 bit matrix whose row l is lane l's word: afterwards
// lane c holds column c (bit r = bit c of row r).  Stage j swaps the
// off-diagonal j x j blocks of every 2j x 2j block: the lanes whose bit j is
// clear keep their low blocks and take their partner's low blocks shifted
// up, the others keep their high blocks and take the partner's high blocks
// shifted down.
__device__ __forceinline__ uint32_t transpose32(uint32_t x) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const uint32_t j = 16u >> s, m = masks[s];
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, (int)j);
    const bool low = (lane & j) == 0;
    const uint32_t t = low ? (y << j) : (y >> j);
    const uint32_t keep = low ? m : ~m;
    x = (x & keep) | (t & ~keep);
  }
  return x;
}

__device__ __forceinline__ uint32_t zigzag(int32_t d) { return ((uint32_t)d << 1) ^ (uint32_t)(d >> 31); }
__device__ __forceinline__ int32_t unzigzag(uint32_t v) { return (int32_t)(v >> 1) ^ -(int32_t)(v & 1u); }

constexpr int kShThreads = 256;
constexpr int kShUnitRuns = 64;                  // 4096 codes per encode unit
constexpr int kShStage = kShUnitRuns * 20;       // v < 1024: at most 20 nonzero columns per run

__device__ __forceinline__ void sh_err(Ctl *ctl, uint32_t code) { atomicCAS(&ctl->res.err, 0u, code); }

// Header of a shuffle stream once the quantizer's counts are known; the
// total size is set by the encoder's last unit.
__global__ void k_shuf_layout(Geom g, uint32_t R, uint32_t pred, uint32_t eb_mode, double eb, CompressWs ws) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Ctl *ctl = ws.ctl;
  fz_header &h = ctl->res.hdr;
  uint32_t mode = ctl->mode;
  if (mode == kModeNormal && ctl->n_out + ctl->n_exc > ws.cap_list) mode = kModeRaw;
  const uint64_t N = g.n;
  if (mode == kModeNormal) {
    const uint64_t nb = g.n_blocks, n_out = ctl->n_out, n_exc = ctl->n_exc;
    const uint64_t n_runs = g.npad / 64, nch = (g.npad + 1023) / 1024;
    const uint64_t off_maps = FZ_HEADER_BYTES;
    const uint64_t off_anch = align16(off_maps + 4 * n_runs);
    const uint64_t off_cb = align16(off_anch + 4 * nb);
    const uint64_t off_oidx = align16(off_cb + 4 * nch);
    const uint64_t off_oval = align16(off_oidx + 4 * n_out);
    const uint64_t off_eidx = align16(off_oval + 4 * n_out);
    const uint64_t off_eval = align16(off_eidx + 4 * n_exc);
    const uint64_t off_bits = align16(off_eval + 4 * n_exc);
    write_min_header(h, FZ_FLAG_SHUF, g, eb_mode, eb, 0);
    h.eb_abs = ctl->eb_abs;
    h.ebx2_bits = __float_as_uint(ctl->ebx2);
    h.inv2eb_bits = __float_as_uint(ctl->inv2eb);
    h.ebchk_bits = __float_as_uint(ctl->eb_chk);
    h.radius = R;
    h.block[0] = g.bx; h.block[1] = g.by; h.block[2] = g.bz;
    h.predictor = pred;
    h.chunk = 1024;
    h.n_blocks = nb; h.n_chunks = nch; h.n_out = n_out; h.n_exc = n_exc; h.total_bits = 0;
    h.off_lens = off_maps; h.off_ids = 0; h.off_anchors = off_anch; h.off_chunk_bits = off_cb;
    h.off_out_idx = off_oidx; h.off_out_val = off_oval; h.off_exc_idx = off_eidx; h.off_exc_val = off_eval;
    h.off_bits = off_bits;
  }
  if (mode == kModeRaw) write_min_header(h, FZ_FLAG_RAW, g, eb_mode, eb, FZ_HEADER_BYTES + 4 * N);
  if (mode == kModeConst) write_min_header(h, FZ_FLAG_CONST, g, eb_mode, eb, FZ_HEADER_BYTES + 16);
  ctl->mode = mode;
  ctl->res.mode = mode;
  ctl->res.total_bytes = h.total_bytes;
  ctl->res.n_out = ctl->n_out;
  ctl->res.n_exc = ctl->n_exc;
}

__global__ void __launch_bounds__(kShThreads) k_shuf_encode(Geom g, CompressWs ws, uint8_t *d_out) {
  __shared__ uint32_t stage[kShThreads / 32][kShStage];
  Ctl *ctl = ws.ctl;
  if (ctl->mode != kModeNormal) return;
  fz_header &h = ctl->res.hdr;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *maps = reinterpret_cast<uint32_t *>(d_out + h.off_lens);
  uint32_t *chunk_bits = reinterpret_cast<uint32_t *>(d_out + h.off_chunk_bits);
  uint32_t *words = reinterpret_cast<uint32_t *>(d_out + h.off_bits);
  const uint32_t *rows = reinterpret_cast<const uint32_t *>(ws.codes);  // two codes per 32-bit row
  const uint64_t n_runs = g.npad / 64, n_chunks = h.n_chunks;
  const uint64_t n_units = (n_runs + kShUnitRuns - 1) / kShUnitRuns;
  const uint64_t raw_end = FZ_HEADER_BYTES + 4 * g.n;  // a longer stream is replaced by the RAW one
  const uint64_t wlimit = h.off_bits < raw_end ? (raw_end - h.off_bits) / 4 : 0;
  const int32_t R = (int32_t)h.radius;
  uint32_t *st = stage[warp];
  for (;;) {
    uint32_t u = 0;
    if (lane == 0) u = atomicAdd(&ctl->encode_ticket, 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= n_units) break;
    const uint64_t k0 = (uint64_t)u * kShUnitRuns;
    const int nr = (int)(n_runs - k0 < (uint64_t)kShUnitRuns ? n_runs - k0 : kShUnitRuns);
    uint32_t cnt = 0, cstart = 0, cwords = 0, mapk = 0;
    uint32_t w_next = __ldcs(rows + k0 * 32 + lane);
#pragma unroll 1
    for (int kk = 0; kk < nr; ++kk) {
      const uint32_t w = w_next;
      if (kk + 1 < nr) w_next = __ldcs(rows + (k0 + kk + 1) * 32 + lane);  // one run ahead
      const uint32_t v0 = zigzag((int32_t)(w & 0xffffu) - R), v1 = zigzag((int32_t)(w >> 16) - R);
      const uint32_t col = transpose32(v0 | (v1 << 16));
      const uint32_t nz = __ballot_sync(0xffffffffu, col != 0u);
      const uint32_t si = cnt + __popc(nz & ((1u << lane) - 1u));
      if (col && si < (uint32_t)kShStage) st[si] = col;
      if (col && si >= (uint32_t)kShStage) sh_err(ctl, FZ_ECORRUPT);  // a code outside 0..2R-1
      cnt += __popc(nz);
      if (lane == (kk & 31)) mapk = nz;
      if ((kk & 31) == 31 || kk + 1 == nr) {  // the maps of up to 32 runs in one store
        const uint64_t kb = k0 + (uint64_t)(kk & ~31);
        if (lane <= (kk & 31)) maps[kb + lane] = mapk;
      }
      if ((kk & 15) == 15 || kk + 1 == nr) {  // end of a 1024-code chunk
        if (lane == (kk >> 4)) cwords = cnt - cstart;
        cstart = cnt;
      }
    }
    const uint64_t c = (uint64_t)u * 4 + (uint64_t)lane;
    if (lane < 4 && lane * 16 < nr && c < n_chunks) chunk_bits[c] = 32u * cwords;
    if (lane == 0) lookback_publish(ws.estatus, u, cnt);
    const uint64_t base = lookback_resolve_warp(ws.estatus, u, cnt, &ctl->res.err, ws.spin);
    const uint32_t staged = cnt < (uint32_t)kShStage ? cnt : (uint32_t)kShStage;
    for (uint32_t i = lane; i < staged; i += 32)
      if (base + i < wlimit) words[base + i] = st[i];
    if (u == n_units - 1 && lane == 0) {
      // the total is known: complete the header, or fall back to RAW when
      // the encoded stream would not be shorter than the raw floats
      const uint64_t total_words = base + cnt;
      const uint64_t total = align16(h.off_bits + 4 * total_words);
      if (total > raw_end) {
        const uint32_t em = h.eb_mode;
        const double eb = h.eb;
        write_min_header(h, FZ_FLAG_RAW, g, em, eb, raw_end);
        ctl->mode = kModeRaw;
        ctl->res.mode = kModeRaw;
        ctl->res.total_bytes = raw_end;
      } else {
        h.total_bits = 32 * total_words;
        h.total_bytes = total;
        ctl->total_bits = 32 * total_words;
        ctl->res.total_bytes = total;
      }
    }
    __syncwarp();  // the stage is reused by the next unit
  }
}

// ---------------------------------------------------------------- decode
struct ShDec {
  const uint32_t *maps, *chunk_bits, *words;
  const uint64_t *goff;      // per work unit of 32 chunks: first bit
  const int32_t *anchors;
  const uint32_t *out_idx;
  const int32_t *out_val;
  const uint32_t *exc_idx, *exc_val;
  uint64_t n_words, n_chunks, n_runs, n_out, n_exc;
  float *out;
  float ebx2;
  int32_t R;
  uint32_t *err;             // err[0] error word, err[1] chunk-group counter, err[2] CTAs done
  uint32_t *h_err;
};

__device__ __forceinline__ void sh_dec_err(uint32_t *err, uint32_t code) { atomicCAS(err, 0u, code); }

// Inclusive scan of v over the lanes of each aligned group of W lanes.
template <int W>
__device__ __forceinline__ int32_t group_scan(int32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 1; off < W; off <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, v, off);
    if ((lane & (W - 1)) >= off) v += t;
  }
  return v;
}

// Inclusive scan of v over lanes l, l + S, l + 2S, ... (stride S).
template <int S>
__device__ __forceinline__ int32_t stride_scan(int32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = S; off < 32; off <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += t;
  }
  return v;
}

// One 1024-code chunk j (or the 512 codes of a last 3D half chunk) starting
// at word w0 of the bitstream.
template <int NDIM, int K>
__device__ __forceinline__ void decode_shuf_chunk(const ShDec &p, const Geom &g, uint64_t j, uint64_t w0,
                                                  uint32_t cbits, bool &bad) {
  const int lane = threadIdx.x & 31;
  const uint64_t r0 = j * 16;
  const int nr = (int)(p.n_runs - r0 < 16 ? p.n_runs - r0 : 16);
  const uint32_t mymap = lane < nr ? __ldg(p.maps + r0 + lane) : 0u;
  int32_t d[16][2];
  uint64_t w = w0;
  uint32_t zeros = 0;
  // every word of the chunk is requested before the first transpose, so
  // the loads' latencies overlap (their addresses depend on the maps only)
  uint32_t cols[16];
#pragma unroll
  for (int kk = 0; kk < 16; ++kk) {
    cols[kk] = 0;
    if (kk < nr) {
      const uint32_t map = __shfl_sync(0xffffffffu, mymap, kk);
      const uint64_t wi = w + __popc(map & ((1u << lane) - 1u));
      if ((map >> lane) & 1u) {
        if (wi < p.n_words) cols[kk] = __ldg(p.words + wi);
        else bad = true;
      }
      w += __popc(map);
    }
  }
#pragma unroll
  for (int kk = 0; kk < 16; ++kk) {
    d[kk][0] = 0;
    d[kk][1] = 0;
    if (kk < nr) {
      const uint32_t row = transpose32(cols[kk]);
      const uint32_t v0 = row & 0xffffu, v1 = row >> 16;
      bad |= v0 >= 2u * (uint32_t)p.R || v1 >= 2u * (uint32_t)p.R;
      d[kk][0] = unzigzag(v0);
      d[kk][1] = unzigzag(v1);
      zeros += __popc(__ballot_sync(0xffffffffu, d[kk][0] == -p.R)) +
               __popc(__ballot_sync(0xffffffffu, d[kk][1] == -p.R));
    }
  }
  if (32ull * (w - w0) != cbits) bad = true;
  const uint32_t pos0 = (uint32_t)(j * 1024);
  // outliers: the chunk holds exactly `zeros` of them, each on a code-0 place
  if (zeros) {
    uint64_t ob = 0;
    if (lane == 0) ob = lower_bound_u32(p.out_idx, p.n_out, pos0);
    ob = __shfl_sync(0xffffffffu, ob, 0);
    if (ob + zeros > p.n_out) bad = true;
    for (uint32_t i = 0; i < zeros && ob + i < p.n_out; ++i) {
      const uint32_t pos = __ldg(p.out_idx + ob + i);
      const int32_t val = __ldg(p.out_val + ob + i);
      const uint32_t rel = pos - pos0;
      if (rel >= (uint32_t)nr * 64u) { bad = true; break; }
      const int kt = (int)(rel >> 6), rt = (int)((rel >> 1) & 31u), et = (int)(rel & 1u);
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        if (kk == kt && lane == rt) {
          int32_t &slot = et ? d[kk][1] : d[kk][0];
          if (slot != -p.R) bad = true;
          slot = val;
        }
      }
    }
    if (ob + zeros < p.n_out && __ldg(p.out_idx + ob + zeros) < pos0 + (uint32_t)nr * 64u) bad = true;
  }
  // anchors (the block origins) and the inverse Lorenzo, K sums per axis
  if (NDIM == 3) {
    // runs 8b..8b+7 are block 2j + b: z = run & 7, y = lane >> 2, x = 2 (lane & 3) + e
    if (lane == 0) {
      d[0][0] += __ldg(p.anchors + 2 * j);
      if (nr > 8) d[8][0] += __ldg(p.anchors + 2 * j + 1);
    }
#pragma unroll
    for (int rep = 0; rep < K; ++rep) {
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        const int32_t a = d[kk][0], b = d[kk][1] + a;      // x within the lane's pair
        const int32_t s = group_scan<4>(b);                 // x across the row's 4 lanes
        d[kk][0] = a + s - b;
        d[kk][1] = s;
        d[kk][0] = stride_scan<4>(d[kk][0]);                // y across the 8 rows
        d[kk][1] = stride_scan<4>(d[kk][1]);
      }
#pragma unroll
      for (int kk = 1; kk < 16; ++kk) {                     // z within each block
        if ((kk & 7) != 0) {
          d[kk][0] += d[kk - 1][0];
          d[kk][1] += d[kk - 1][1];
        }
      }
    }
  } else if (NDIM == 1) {
    // one block of 1024: position 64 run + 2 lane + e
    if (lane == 0) d[0][0] += __ldg(p.anchors + j);
#pragma unroll
    for (int rep = 0; rep < K; ++rep) {
      int32_t carry = 0;
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        const int32_t a = d[kk][0], b = d[kk][1] + a;
        const int32_t s = group_scan<32>(b);
        d[kk][0] = carry + a + s - b;
        d[kk][1] = carry + s;
        carry += __shfl_sync(0xffffffffu, s, 31);
      }
    }
  } else {
    // one 32 x 32 block: y = 2 run + (lane >> 4), x = 2 (lane & 15) + e
    if (lane == 0) d[0][0] += __ldg(p.anchors + j);
    const int xc = lane & 15, hf = lane >> 4;
#pragma unroll
    for (int rep = 0; rep < K; ++rep) {
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        const int32_t a = d[kk][0], b = d[kk][1] + a;
        const int32_t s = group_scan<16>(b);
        d[kk][0] = a + s - b;
        d[kk][1] = s;
      }
      int32_t col0 = 0, col1 = 0;  // column sums of the rows above
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        const int32_t e0 = __shfl_sync(0xffffffffu, d[kk][0], xc), f0 = __shfl_sync(0xffffffffu, d[kk][0], 16 + xc);
        const int32_t e1 = __shfl_sync(0xffffffffu, d[kk][1], xc), f1 = __shfl_sync(0xffffffffu, d[kk][1], 16 + xc);
        d[kk][0] = col0 + e0 + (hf ? f0 : 0);
        d[kk][1] = col1 + e1 + (hf ? f1 : 0);
        col0 += e0 + f0;
        col1 += e1 + f1;
      }
    }
  }
  // exceptions of the chunk (rare): their values replace the dequantized ones
  uint64_t eb0 = 0, ee0 = 0;
  if (p.n_exc) {
    if (lane == 0) {
      eb0 = lower_bound_u32(p.exc_idx, p.n_exc, pos0);
      ee0 = lower_bound_u32(p.exc_idx, p.n_exc, pos0 + (uint32_t)nr * 64u);
    }
    eb0 = __shfl_sync(0xffffffffu, eb0, 0);
    ee0 = __shfl_sync(0xffffffffu, ee0, 0);
  }
  // dequantize and store; block coordinates once per chunk
  uint32_t bx0 = 0, by0 = 0, bz0 = 0, bx1 = 0, by1 = 0, bz1 = 0;
  {
    const uint32_t b0 = NDIM == 3 ? (uint32_t)(2 * j) : (uint32_t)j;
    bx0 = b0 % g.nbx;
    const uint32_t r_0 = b0 / g.nbx;
    by0 = r_0 % g.nby;
    bz0 = r_0 / g.nby;
    if (NDIM == 3) {
      const uint32_t b1 = b0 + 1;
      bx1 = b1 % g.nbx;
      const uint32_t r_1 = b1 / g.nbx;
      by1 = r_1 % g.nby;
      bz1 = r_1 / g.nby;
    }
  }
  // field coordinates of code (run kk, lane ln, half e) of the chunk; field
  // indices fit 32 bits (fewer than 2^32 values)
  auto coords = [&](int kk, int ln, uint32_t e, uint32_t &x, uint32_t &y, uint32_t &z) {
    if (NDIM == 3) {
      const bool second = kk >= 8;
      x = (second ? bx1 : bx0) * 8u + 2u * (uint32_t)(ln & 3) + e;
      y = (second ? by1 : by0) * 8u + (uint32_t)(ln >> 2);
      z = (second ? bz1 : bz0) * 8u + (uint32_t)(kk & 7);
    } else if (NDIM == 2) {
      x = bx0 * 32u + 2u * (uint32_t)(ln & 15) + e;
      y = by0 * 32u + 2u * (uint32_t)kk + (uint32_t)(ln >> 4);
      z = 0;
    } else {
      x = (uint32_t)j * 1024u + 64u * (uint32_t)kk + 2u * (uint32_t)ln + e;
      y = 0;
      z = 0;
    }
  };
  const bool vec = (((uintptr_t)p.out) & 7u) == 0;
#pragma unroll
  for (int kk = 0; kk < 16; ++kk) {
    if (kk >= nr) continue;
    const float o0 = __fmul_rn(__int2float_rn(d[kk][0]), p.ebx2), o1 = __fmul_rn(__int2float_rn(d[kk][1]), p.ebx2);
    uint32_t x, y, z;
    coords(kk, lane, 0u, x, y, z);
    const uint32_t f = (z * g.ny + y) * g.nx + x;
    if (y < g.ny && z < g.nz) {
      if (x + 1 < g.nx && (f & 1) == 0 && vec) {
        *reinterpret_cast<float2 *>(p.out + f) = make_float2(o0, o1);
      } else {
        if (x < g.nx) p.out[f] = o0;
        if (x + 1 < g.nx) p.out[f + 1] = o1;
      }
    }
  }
  // exceptions of the chunk (rare): their stored bits replace the values the
  // warp has just written (the warp's stores are ordered before these)
  if (eb0 < ee0) {
    __syncwarp();
    for (uint64_t i = eb0 + (uint64_t)lane; i < ee0; i += 32) {
      const uint32_t rel = __ldg(p.exc_idx + i) - pos0;  // < nr * 64: the chunk's range
      uint32_t x, y, z;
      coords((int)(rel >> 6), (int)((rel >> 1) & 31u), rel & 1u, x, y, z);
      if (x < g.nx && y < g.ny && z < g.nz) p.out[(z * g.ny + y) * g.nx + x] = __uint_as_float(__ldg(p.exc_val + i));
      else bad = true;
    }
  }
}

template <int NDIM, int K>
__global__ void __launch_bounds__(kShThreads) k_shuf_decode(ShDec p, Geom g) {
  const int lane = threadIdx.x & 31;
  bool bad = false;
  const uint64_t n_groups = (p.n_chunks + 3) / 4;
  for (;;) {
    uint32_t q = 0;
    if (lane == 0) q = atomicAdd(p.err + 1, 1u);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= n_groups) break;
    // bit offsets of the group's chunks: the unit's first bit plus the
    // lengths of the unit's earlier chunks (the 4 chunks share one unit)
    const uint64_t u = ((uint64_t)q * 4) / kDecUnit;
    const uint64_t jl = u * kDecUnit + lane;
    const uint32_t cb = jl < p.n_chunks ? __ldg(p.chunk_bits + jl) : 0u;
    uint32_t incl = cb;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    const uint64_t ubase = __ldg(p.goff + u);
    for (int c = 0; c < 4; ++c) {
      const uint64_t j = (uint64_t)q * 4 + c;
      if (j >= p.n_chunks) break;
      const int src = (int)(j - u * kDecUnit);
      const uint32_t ex = __shfl_sync(0xffffffffu, incl - cb, src);
      const uint32_t cbj = __shfl_sync(0xffffffffu, cb, src);
      const uint64_t start = ubase + ex;
      if (start & 31u) bad = true;
      decode_shuf_chunk<NDIM, K>(p, g, j, start >> 5, cbj, bad);
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) sh_dec_err(p.err, FZ_ECORRUPT);
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

template <int NDIM, int K>
cudaError_t launch_shuf_dec_t(const ShDec &p, const Geom &g, int sm_count, cudaStream_t s) {
  static LaunchCache cache;
  int per_sm = 0;
  const cudaError_t e = cached_per_sm(k_shuf_decode<NDIM, K>, kShThreads, 0, cache, per_sm);
  if (e != cudaSuccess) return e;
  const uint64_t n_groups = (p.n_chunks + 3) / 4;
  uint64_t grid = (uint64_t)sm_count * per_sm;
  const uint64_t need = (n_groups + kShThreads / 32 - 1) / (kShThreads / 32);
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  k_shuf_decode<NDIM, K><<<(unsigned)grid, kShThreads, 0, s>>>(p, g);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_shuf_layout(const Geom &g, uint32_t R, uint32_t pred, uint32_t eb_mode, double eb,
                               const CompressWs &ws, cudaStream_t s) {
  k_shuf_layout<<<1, 32, 0, s>>>(g, R, pred, eb_mode, eb, ws);
  return cudaGetLastError();
}

cudaError_t launch_shuf_encode(const Geom &g, const CompressWs &ws, uint8_t *d_out, cudaStream_t s, int sm_count) {
  static LaunchCache cache;
  int per_sm = 0;
  const cudaError_t e = cached_per_sm(k_shuf_encode, kShThreads, 0, cache, per_sm);
  if (e != cudaSuccess) return e;
  const uint64_t n_units = (g.npad / 64 + kShUnitRuns - 1) / kShUnitRuns;
  uint64_t grid = (uint64_t)sm_count * per_sm;
  const uint64_t need = (n_units + kShThreads / 32 - 1) / (kShThreads / 32);
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  k_shuf_encode<<<(unsigned)grid, kShThreads, 0, s>>>(g, ws, d_out);
  return cudaGetLastError();
}

cudaError_t launch_shuf_decode(const uint8_t *d_in, const fz_header &h, float *d_out, const DecodeWs &ws,
                               cudaStream_t s, int sm_count) {
  Geom g;
  make_geom(h.ndim, h.dims, g);
  ShDec p;
  p.maps = reinterpret_cast<const uint32_t *>(d_in + h.off_lens);
  p.chunk_bits = reinterpret_cast<const uint32_t *>(d_in + h.off_chunk_bits);
  p.words = reinterpret_cast<const uint32_t *>(d_in + h.off_bits);
  p.goff = ws.gsum;
  p.anchors = reinterpret_cast<const int32_t *>(d_in + h.off_anchors);
  p.out_idx = reinterpret_cast<const uint32_t *>(d_in + h.off_out_idx);
  p.out_val = reinterpret_cast<const int32_t *>(d_in + h.off_out_val);
  p.exc_idx = reinterpret_cast<const uint32_t *>(d_in + h.off_exc_idx);
  p.exc_val = reinterpret_cast<const uint32_t *>(d_in + h.off_exc_val);
  p.n_words = h.total_bits / 32;
  p.n_chunks = h.n_chunks;
  p.n_runs = g.npad / 64;
  p.n_out = h.n_out;
  p.n_exc = h.n_exc;
  p.out = d_out;
  memcpy(&p.ebx2, &h.ebx2_bits, 4);
  p.R = (int32_t)h.radius;
  p.err = ws.err;
  p.h_err = ws.h_err;
  const bool k2 = h.predictor == FZ_PRED_LORENZO2;
  switch (g.ndim) {
    case 1: return k2 ? launch_shuf_dec_t<1, 2>(p, g, sm_count, s) : launch_shuf_dec_t<1, 1>(p, g, sm_count, s);
    case 2: return k2 ? launch_shuf_dec_t<2, 2>(p, g, sm_count, s) : launch_shuf_dec_t<2, 1>(p, g, sm_count, s);
    default: return k2 ? launch_shuf_dec_t<3, 2>(p, g, sm_count, s) : launch_shuf_dec_t<3, 1>(p, g, sm_count, s);
  }
}

}  // namespace fz
