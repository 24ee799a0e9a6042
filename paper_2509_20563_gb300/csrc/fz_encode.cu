// fz_encode.cu -- chunked canonical Huffman encoder (FZModules §3.1: cuSZ's
// GPU Huffman encoder; FZMod-Default runs it on the CPU, §3.3).
//
// Persistent CTAs take tiles of 8 consecutive chunks (chunk = one block of
// codes) from a ticket counter, one warp per chunk.  Each lane owns a
// contiguous run of codes: it sums their codeword lengths, the warp scans
// the lane totals (the chunk's bit length, stored in the stream) and the CTA
// sums the chunk totals.  The tile publishes its bit total for a bounded
// decoupled look-back right away, then packs its codewords (two at a time)
// MSB-first into a shared-memory image of the tile aligned to bit 0 and
// appends the first 32 bits of the next tile (encoded from that tile's first
// codes).  A single field's CTAs keep two tiles in flight (k_encode_pipe):
// the tile packed in one step resolves its global bit offset and is stored
// in the next, so its predecessors have had a whole step to publish; the
// codes of a CTA's next tile are loaded into registers during the step
// before (its ticket is taken a step ahead).  The
// image is written out with a funnel shift by the offset's low 5 bits; the
// CTA stores exactly the words whose first bit lies in its tile, so every
// word is written once, by plain coalesced stores, and the output needs no
// zeroing.  Batches (k_encode_batch) run one tile per step through
// encode_tile, which lets a CTA switch fields between tiles.
// HBM traffic: 2 bytes read per code plus the bitstream.
#include "fz_internal.cuh"

namespace fz {

namespace {

constexpr int kEncThreads = kEncWarps * 32;

#ifndef FZ_ENC_MINB
#define FZ_ENC_MINB 6  // CTAs per SM, 512-code chunks (3D)
#endif
#ifndef FZ_ENC_MINB1024
#define FZ_ENC_MINB1024 3  // CTAs per SM, 1024-code chunks (1D, 2D)
#endif

template <int CH>
struct EncSmem {
  static constexpr int kMaxWords = (CH * kEncWarps * kLmax + 32) / 32 + 3;  // tile image + next-tile head
  uint32_t senc[kMaxSym];
  __align__(16) uint32_t lw[kMaxWords];
  uint32_t wtot[kEncWarps], woff[kEncWarps];
  uint32_t tile, tbits, job;
  unsigned long long base;
};

// Stored chunk lengths below one block: with chunks of C symbols and PER
// codes per lane (3D: C = 64, PER = 16; 2D: C = 128, 256, 512, PER = 32) the
// lanes LPC s .. LPC s + LPC - 1 (LPC = C / PER) hold sub-chunk s, and the
// last of them stores the difference of the inclusive scan.  Every lane of
// the warp calls it; chunks of a block or more store nothing here.
template <int PER>
__device__ __forceinline__ void store_sub_chunks(uint32_t *chunk_bits, uint64_t block, uint32_t incl, int lane,
                                                 uint32_t chunk, bool valid) {
  if (chunk >= 32u * PER || chunk < 2u * PER) return;
  const uint32_t lpc = chunk / PER;  // a power of two: 2 to 16 lanes
  const uint32_t prev = __shfl_up_sync(0xffffffffu, incl, lpc);
  if (valid && ((uint32_t)lane & (lpc - 1)) == lpc - 1)
    chunk_bits[block * (32 / lpc) + (uint32_t)lane / lpc] = (uint32_t)lane >= lpc ? incl - prev : incl;
}

// Stored chunk lengths above one block (chunk = k blocks, k = 2, 4, 8 divides
// the tile's 8 blocks): the first 8 / k threads each add up the bit totals
// of k consecutive blocks of the tile.
__device__ __forceinline__ void store_multi_chunks(uint32_t *chunk_bits, const uint32_t *wtot, uint64_t tile,
                                                   uint32_t k, uint64_t n_chunks, int tid) {
  if (k <= 1 || tid >= (int)(kEncWarps / k)) return;
  uint32_t sum = 0;
  for (uint32_t w = (uint32_t)tid * k; w < (uint32_t)(tid + 1) * k; ++w) sum += wtot[w];
  const uint64_t c = tile * (kEncWarps / k) + (uint64_t)tid;
  if (c < n_chunks) chunk_bits[c] = sum;
}

// Codeword table entries (Ctl::enc): the codeword left-aligned in the high
// L bits, L (at most 14) in the low 5 bits.  One lane's PER codewords are
// packed MSB-first into the tile image lw from tile-local bit rb, two at a
// time (at most 28 bits: the pair is one left-aligned word, so at most one
// image word fills per step); the funnel shift gives the pair's bits that
// spill past the current word.
template <int PER>
__device__ __forceinline__ void pack_lane(const uint32_t (&cw)[PER], uint32_t rb, uint32_t *lw) {
  uint32_t wi = rb >> 5;
  uint32_t cnt = rb & 31u;  // bits of word wi in front of this lane's next codeword
  uint32_t cur = 0;         // this lane's bits of word wi
#pragma unroll
  for (int k = 0; k < PER; k += 2) {
    const uint32_t L0 = cw[k] & 31u;
    const uint32_t v = (cw[k] & ~31u) | ((cw[k + 1] & ~31u) >> L0);
    cur |= v >> cnt;
    const uint32_t spill = __funnelshift_r(0u, v, cnt);
    cnt += L0 + (cw[k + 1] & 31u);
    if (cnt >= 32) {
      atomicOr(&lw[wi], cur);
      ++wi;
      cur = spill;
      cnt -= 32;
    }
  }
  if (cnt > 0) atomicOr(&lw[wi], cur);
}

// The first 32 bits of the codewords of a tile's first 32 codes, one code
// per lane (entry e of the lane's code): every lane of the warp calls it.
__device__ __forceinline__ uint32_t head_bits(uint32_t e, int lane) {
  const uint32_t L = e & 31u;
  uint32_t p = L;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, p, off);
    if (lane >= off) p += v;
  }
  p -= L;
  return __reduce_or_sync(0xffffffffu, p < 32 ? (e & ~31u) >> p : 0u);
}

// One encode tile (kEncWarps chunks) of one field whose codeword table is
// in sm.senc; all threads of the CTA call it together.
template <int CH>
__device__ __forceinline__ void encode_tile(const CompressWs &ws, uint8_t *d_out, uint64_t n_blk, uint64_t tile,
                                            EncSmem<CH> &sm) {
  constexpr int PER = CH / 32;  // codes per lane (16 or 32)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Ctl *ctl = ws.ctl;
  const fz_header &h = ctl->res.hdr;
  uint32_t *chunk_bits = reinterpret_cast<uint32_t *>(d_out + h.off_chunk_bits);
  uint32_t *words = reinterpret_cast<uint32_t *>(d_out + h.off_bits);
  const uint64_t n_tiles = (n_blk + kEncWarps - 1) / kEncWarps;
  const uint64_t wlimit = (ctl->total_bits + 31) / 32;
  uint32_t *senc = sm.senc, *lw = sm.lw;

  // ---- lane codes and bit counts
  const uint64_t blk = tile * kEncWarps + warp;
  const bool valid = blk < n_blk;
  uint32_t cw[PER];
  uint32_t lbits = 0;
  if (valid) {
    const uint4 *src = reinterpret_cast<const uint4 *>(ws.codes + blk * CH + lane * PER);
#pragma unroll
    for (int v = 0; v < PER / 8; ++v) {
      const uint4 u = __ldcs(src + v);
      const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        cw[8 * v + 2 * k] = senc[w4[k] & 0xffffu];
        cw[8 * v + 2 * k + 1] = senc[w4[k] >> 16];
      }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) lbits += cw[k] & 31u;
  } else {
#pragma unroll
    for (int k = 0; k < PER; ++k) cw[k] = 0;
  }
  uint32_t incl = lbits;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  const uint32_t lane_off = incl - lbits;
  if (lane == 31) {
    sm.wtot[warp] = incl;
    if (valid && h.chunk == CH) chunk_bits[blk] = incl;
  }
  store_sub_chunks<PER>(chunk_bits, blk, incl, lane, h.chunk, valid);
  __syncthreads();
  store_multi_chunks(chunk_bits, sm.wtot, tile, h.chunk / CH, h.n_chunks, tid);
  if (tid == 0) {
    uint32_t acc = 0;
    for (int w = 0; w < kEncWarps; ++w) { sm.woff[w] = acc; acc += sm.wtot[w]; }
    sm.tbits = acc;
    lookback_publish(ws.estatus, tile, acc);
  }
  __syncthreads();
  const uint32_t tbits = sm.tbits;
  const uint32_t nl = (tbits + 32 + 31) / 32 + 1;
  for (uint32_t w = tid; w < nl; w += kEncThreads) lw[w] = 0;
  __syncthreads();

  // ---- pack this lane's codewords MSB-first at its tile-local bit offset
  if (valid) pack_lane<PER>(cw, sm.woff[warp] + lane_off, lw);
  __syncthreads();

  if (warp == 0) {
    // first 32 bits of the next tile, placed right after this tile's bits
    if (tile + 1 < n_tiles) {
      const uint32_t head = head_bits(senc[ws.codes[(tile + 1) * kEncWarps * (uint64_t)CH + lane]], lane);
      if (lane == 0) {
        const uint32_t r = tbits & 31u, w0 = tbits >> 5;
        lw[w0] |= head >> r;
        if (r) lw[w0 + 1] |= head << (32 - r);
      }
    }
    const unsigned long long base = lookback_resolve_warp(ws.estatus, tile, tbits, &ctl->res.err, ws.spin);
    if (lane == 0) {
      sm.base = base;
      if (tile == n_tiles - 1 && base + tbits != ctl->total_bits) set_err(ctl, FZ_ECORRUPT);
    }
  }
  __syncthreads();

  // ---- write every word whose first bit lies in this tile (funnel shift
  // by the offset's low bits; never past the bitstream section)
  const unsigned long long base = sm.base;
  const uint32_t r = (uint32_t)(base & 31u);
  const uint64_t gw0 = base >> 5;
  const uint32_t jmax = (uint32_t)(((base + tbits - 1) >> 5) - gw0);
  if (tid == 0 && gw0 + jmax >= wlimit) set_err(ctl, FZ_ECORRUPT);
  for (uint32_t j = (r ? 1u : 0u) + tid; j <= jmax; j += kEncThreads) {
    const uint32_t v = r ? ((lw[j - 1] << (32 - r)) | (lw[j] >> r)) : lw[j];
    if (gw0 + j < wlimit) words[gw0 + j] = v;
  }
}

// Batched variant: the encode tiles of every field of one chunk-size class
// form one ticket queue, in field order, so a field's tiles are claimed in
// order and its look-back always ends.  The codeword table is reloaded when
// a CTA moves to another field; fields without a Huffman section, or
// without room in the packed output, are skipped.
template <int CH>
__global__ void __launch_bounds__(kEncThreads) k_encode_batch(const BatchJob *__restrict__ jobs,
                                                               const uint32_t *__restrict__ members,
                                                               uint32_t n_members, uint64_t total_tiles,
                                                               uint32_t *ticket, uint8_t *d_out) {
  __shared__ EncSmem<CH> sm;
  const int tid = threadIdx.x;
  uint32_t cur = 0xffffffffu;
  for (;;) {
    if (tid == 0) {
      const uint32_t tk = atomicAdd(ticket, 1u);
      sm.tile = tk;
      if (tk < total_tiles) {
        uint32_t a = 0, b = n_members;  // the member whose tiles contain tk
        while (a < b) {
          const uint32_t m = (a + b) >> 1;
          const BatchJob &J = jobs[members[m]];
          if (J.etile_base + (J.g.n_blocks + kEncWarps - 1) / kEncWarps <= tk) a = m + 1; else b = m;
        }
        sm.job = members[a];
      }
    }
    __syncthreads();
    const uint64_t tk = sm.tile;
    if (tk >= total_tiles) break;
    const uint32_t j = sm.job;
    const BatchJob &J = jobs[j];
    if (J.ws.ctl->mode != kModeNormal || J.out_off == kNoOutput) {
      __syncthreads();
      continue;
    }
    if (j != cur) {
      for (int s = tid; s < kMaxSym; s += kEncThreads) sm.senc[s] = J.ws.ctl->enc[s];
      cur = j;
      __syncthreads();
    }
    encode_tile<CH>(J.ws, d_out + J.out_off, J.g.n_blocks, tk - J.etile_base, sm);
    __syncthreads();
  }
}

// Single field, two tiles in flight per CTA: in each step the CTA counts,
// publishes and packs its newest tile, then resolves the look-back and
// stores the tile packed one step earlier, whose predecessors have had a
// whole step to publish their prefixes.  Two images alternate.
// D tile images in a ring: the tile packed in one step is stored D - 1
// steps later, so its look-back predecessors have had D - 1 steps to
// publish (D = 2 by default; FZ_ENC_DEPTH selects another depth).
#ifndef FZ_ENC_DEPTH
#define FZ_ENC_DEPTH 2
#endif
// FZ_ENC_ZB: one image more than the depth, and the image stored in one step
// is cleared in the next (the barrier at the end of a step orders the
// clearing after its reads and before its next use), which saves the
// barrier between storing an image and clearing it (512^3 field: 196.6 µs
// against 204.8; equal on 1D fields and 1024-code chunks)
#ifndef FZ_ENC_ZB
#define FZ_ENC_ZB 1
#endif
// FZ_ENC_NOEND (with FZ_ENC_ZB): no barrier at the end of a step -- the
// per-warp bit totals alternate between two arrays by step parity, and the
// image stored in one step is cleared after the next step's first barrier
// (which every thread reaches only after its part of the previous step);
// the ticket slots alternate already, and the look-back base is written
// only after that barrier (512^3 field: 192.5 µs against 196.6)
#ifndef FZ_ENC_NOEND
#define FZ_ENC_NOEND 1
#endif
template <int CH, int D>
struct PipeSmem {
  static constexpr int kMaxWords = EncSmem<CH>::kMaxWords;
  static constexpr int kImages = D + (FZ_ENC_ZB ? 1 : 0);
  uint32_t senc[kMaxSym];
  __align__(16) uint32_t lw[kImages][kMaxWords];
  uint32_t wtot[2][kEncWarps];  // per-warp bit totals of the step (by parity when the steps overlap)
  uint32_t tk[2];  // tickets: the current tile and the next one
  unsigned long long base;
};

// The codes of one lane of one chunk (PER consecutive codes, 16-byte loads).
template <int PER>
__device__ __forceinline__ void load_lane_codes(const uint16_t *codes, uint64_t chunk, int CH, int lane,
                                                uint4 (&raw)[PER / 8]) {
  const uint4 *src = reinterpret_cast<const uint4 *>(codes + chunk * CH + lane * PER);
#pragma unroll
  for (int v = 0; v < PER / 8; ++v) raw[v] = __ldcs(src + v);
}

// CM: how chunk lengths are stored -- 0 one chunk per block, 1 64-symbol
// chunks (3D), 2 chunks of several blocks; a template parameter so that the
// default case carries none of the others' code.
template <int CH, int CM>
__global__ void __launch_bounds__(kEncThreads, CH == 512 ? FZ_ENC_MINB : FZ_ENC_MINB1024) k_encode_pipe(Geom g, CompressWs ws, uint8_t *d_out) {
  constexpr int PER = CH / 32;
  constexpr int D = FZ_ENC_DEPTH;
  __shared__ PipeSmem<CH, D> sm;
  Ctl *ctl = ws.ctl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t n_blk = g.n_blocks;
  const uint64_t n_tiles = (n_blk + kEncWarps - 1) / kEncWarps;
  constexpr int NI = PipeSmem<CH, D>::kImages;
  // Before the wait for the codebook: the first ticket, the images cleared
  // and the first tile's codes loaded (the quantizer, which wrote them, has
  // finished once the codebook runs; the ticket counter was zeroed before it)
  for (int i = tid; i < NI * PipeSmem<CH, D>::kMaxWords; i += kEncThreads) (&sm.lw[0][0])[i] = 0;
  if (tid == 0) sm.tk[0] = atomicAdd(&ctl->encode_ticket, 1u);
  __syncthreads();
  uint64_t tile = sm.tk[0];
  // the codes of the tile in hand are loaded one step ahead of their use
  uint4 raw[PER / 8];
  if (tile < n_tiles && tile * kEncWarps + warp < n_blk) load_lane_codes<PER>(ws.codes, tile * kEncWarps + warp, CH, lane, raw);
  dep_wait();  // the codebook: table, header, mode, total bits
  dep_trigger();
  if (ctl->mode != kModeNormal) return;
  const fz_header &h = ctl->res.hdr;
  uint32_t *chunk_bits = reinterpret_cast<uint32_t *>(d_out + h.off_chunk_bits);
  uint32_t *words = reinterpret_cast<uint32_t *>(d_out + h.off_bits);
  const uint64_t wlimit = (ctl->total_bits + 31) / 32;
  for (int i = tid; i < kMaxSym; i += kEncThreads) sm.senc[i] = ctl->enc[i];
  uint32_t stored_bits = 0;  // bits of the tile stored in the previous step (FZ_ENC_ZB)
  int par = 0;               // step parity (FZ_ENC_NOEND)
  __syncthreads();  // the codeword table is in place
  // tiles packed but not yet stored, oldest first, and their bit totals
  uint64_t pend[D - 1];
  uint32_t pend_bits[D - 1];
#pragma unroll
  for (int i = 0; i < D - 1; ++i) { pend[i] = ~0ull; pend_bits[i] = 0; }
  int cb = 0;  // image of the current tile; the oldest pending tile's is (cb + NI - (D - 1)) % NI
  int tb = 0;  // ticket slot of the current tile
  for (;;) {
    const bool have = tile < n_tiles;
    uint32_t tbits = 0;
    uint32_t *lw = sm.lw[cb];
    uint32_t *wt = sm.wtot[FZ_ENC_NOEND ? par : 0];
    if (FZ_ENC_ZB && !FZ_ENC_NOEND) {
      // the image stored in the previous step is the next step's packing image
      uint32_t *z = sm.lw[(cb + 1) % NI];
      const uint32_t nz = stored_bits ? (stored_bits + 32 + 31) / 32 + 1 : 0u;
      for (uint32_t w = tid; w < nz; w += kEncThreads) z[w] = 0;
    }
    const uint64_t blk = tile * kEncWarps + warp;
    const bool valid = have && blk < n_blk;
    if (tid == 0 && have) sm.tk[tb ^ 1] = atomicAdd(&ctl->encode_ticket, 1u);
    // the next tile's first 32 codes (its head), read ahead of their use
    uint32_t hcode = 0;
    if (have && warp == kEncWarps - 1 && tile + 1 < n_tiles)
      hcode = ws.codes[(tile + 1) * kEncWarps * (uint64_t)CH + lane];
    // ---- count and publish
    uint32_t cw[PER];
    uint32_t lbits = 0;
    if (valid) {
#pragma unroll
      for (int v = 0; v < PER / 8; ++v) {
        const uint32_t w4[4] = {raw[v].x, raw[v].y, raw[v].z, raw[v].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          cw[8 * v + 2 * k] = sm.senc[w4[k] & 0xffffu];
          cw[8 * v + 2 * k + 1] = sm.senc[w4[k] >> 16];
        }
      }
#pragma unroll
      for (int k = 0; k < PER; ++k) lbits += cw[k] & 31u;
    } else {
#pragma unroll
      for (int k = 0; k < PER; ++k) cw[k] = 0;
    }
    uint32_t incl = lbits;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += v;
    }
    if (lane == 31) {
      wt[warp] = incl;
      if (CM == 0 && valid) chunk_bits[blk] = incl;
    }
    if (CM == 1) store_sub_chunks<PER>(chunk_bits, blk, incl, lane, g.chunk, valid);
    __syncthreads();
    if (FZ_ENC_ZB && FZ_ENC_NOEND) {
      // every thread has finished the previous step (its store included)
      uint32_t *z = sm.lw[(cb + 1) % NI];
      const uint32_t nz = stored_bits ? (stored_bits + 32 + 31) / 32 + 1 : 0u;
      for (uint32_t w = tid; w < nz; w += kEncThreads) z[w] = 0;
    }
    if (CM == 2 && have) store_multi_chunks(chunk_bits, wt, tile, g.chunk / CH, g.n_chunks, tid);
    // ---- the next tile's codes go out now and land during this step
    const uint64_t next = have ? (uint64_t)sm.tk[tb ^ 1] : n_tiles;
    if (next < n_tiles && next * kEncWarps + warp < n_blk)
      load_lane_codes<PER>(ws.codes, next * kEncWarps + warp, CH, lane, raw);
    if (have) {
      uint32_t woff = 0;
#pragma unroll
      for (int w = 0; w < kEncWarps; ++w) {
        const uint32_t t = wt[w];
        woff += w < warp ? t : 0u;
        tbits += t;
      }
      if (tid == 0) lookback_publish(ws.estatus, tile, tbits);
      // ---- pack MSB-first at the tile-local bit offset, codewords in pairs
      if (valid) pack_lane<PER>(cw, woff + incl - lbits, lw);
      // ---- first 32 bits of the next tile, right after this tile's bits
      if (warp == kEncWarps - 1 && tile + 1 < n_tiles) {
        const uint32_t head = head_bits(sm.senc[hcode], lane);
        if (lane == 0) {
          const uint32_t r = tbits & 31u, w0 = tbits >> 5;
          atomicOr(&lw[w0], head >> r);
          if (r) atomicOr(&lw[w0 + 1], head << (32 - r));
        }
      }
    }
    // ---- the oldest pending tile: its base by look-back, then its words
    const uint64_t prev = pend[0];
    const uint32_t prev_bits = pend_bits[0];
    const int pcb = (cb + NI - (D - 1)) % NI;
    if (prev != ~0ull && warp == 0) {
      const unsigned long long base = lookback_resolve_warp(ws.estatus, prev, prev_bits, &ctl->res.err, ws.spin);
      if (lane == 0) {
        sm.base = base;
        if (prev == n_tiles - 1 && base + prev_bits != ctl->total_bits) set_err(ctl, FZ_ECORRUPT);
      }
    }
    __syncthreads();  // packing, head and base are visible
    if (prev != ~0ull) {
      const uint32_t *plw = sm.lw[pcb];
      const unsigned long long base = sm.base;
      const uint32_t r = (uint32_t)(base & 31u);
      const uint64_t gw0 = base >> 5;
      const uint32_t jmax = (uint32_t)(((base + prev_bits - 1) >> 5) - gw0);
      if (tid == 0 && gw0 + jmax >= wlimit) set_err(ctl, FZ_ECORRUPT);
      for (uint32_t j = (r ? 1u : 0u) + tid; j <= jmax; j += kEncThreads) {
        const uint32_t v = r ? ((plw[j - 1] << (32 - r)) | (plw[j] >> r)) : plw[j];
        if (gw0 + j < wlimit) words[gw0 + j] = v;
      }
      if (!FZ_ENC_ZB) {
        __syncthreads();  // every word of the previous image has been read
        uint32_t *z = sm.lw[pcb];
        const uint32_t nz = (prev_bits + 32 + 31) / 32 + 1;
        for (uint32_t w = tid; w < nz; w += kEncThreads) z[w] = 0;
      }
    }
    stored_bits = prev != ~0ull ? prev_bits : 0u;
    // shift the pending queue; after the last tile, drain what is left
#pragma unroll
    for (int i = 0; i < D - 2; ++i) { pend[i] = pend[i + 1]; pend_bits[i] = pend_bits[i + 1]; }
    pend[D - 2] = have ? tile : ~0ull;
    pend_bits[D - 2] = have ? tbits : 0u;
    bool left = false;
#pragma unroll
    for (int i = 0; i < D - 1; ++i) left = left || pend[i] != ~0ull;
    if (!have && !left) break;
    if (have) {
      tile = next;
      tb ^= 1;
    }
    cb = (cb + 1) % NI;
    par ^= 1;
    if (!FZ_ENC_NOEND) __syncthreads();  // the cleared image is ready for the next tile
  }
}

template <int CH, int CM>
cudaError_t launch_t(const Geom &g, const CompressWs &ws, uint8_t *d_out, cudaStream_t s, int sms) {
  static LaunchCache cache;
  int per_sm = 0;
  const cudaError_t e = cached_per_sm(k_encode_pipe<CH, CM>, kEncThreads, 0, cache, per_sm);
  if (e != cudaSuccess) return e;
  const uint64_t n_tiles = (g.n_blocks + kEncWarps - 1) / kEncWarps;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > n_tiles) grid = n_tiles;
  return launch_dep(k_encode_pipe<CH, CM>, (unsigned)grid, (unsigned)kEncThreads, 0, s, g, ws, d_out);
}

template <int CH>
cudaError_t launch_batch_t(const BatchJob *jobs, const uint32_t *members, uint32_t n_members, uint64_t total_tiles,
                           uint32_t *ticket, uint8_t *d_out, int per_sm, cudaStream_t s, int sms) {
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_encode_batch<CH>, kEncThreads, 0);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  if (per_sm < 1 || per_sm > occ) per_sm = occ;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > total_tiles) grid = total_tiles;
  if (grid < 1) grid = 1;
  k_encode_batch<CH><<<(unsigned)grid, kEncThreads, 0, s>>>(jobs, members, n_members, total_tiles, ticket, d_out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_encode_batch(int chunk, const BatchJob *jobs, const uint32_t *members, uint32_t n_members,
                                uint64_t total_tiles, uint32_t *ticket, uint8_t *d_out, int per_sm, cudaStream_t s,
                                int sm_count) {
  if (chunk == 512) return launch_batch_t<512>(jobs, members, n_members, total_tiles, ticket, d_out, per_sm, s, sm_count);
  return launch_batch_t<1024>(jobs, members, n_members, total_tiles, ticket, d_out, per_sm, s, sm_count);
}

cudaError_t launch_encode(const Geom &g, const CompressWs &ws, uint8_t *d_out, cudaStream_t s, int sm_count) {
  const int cm = g.chunk == g.bsize ? 0 : (g.chunk < g.bsize ? 1 : 2);
  if (g.bsize == 512) {
    if (cm == 0) return launch_t<512, 0>(g, ws, d_out, s, sm_count);
    if (cm == 1) return launch_t<512, 1>(g, ws, d_out, s, sm_count);
    return launch_t<512, 2>(g, ws, d_out, s, sm_count);
  }
  if (cm == 0) return launch_t<1024, 0>(g, ws, d_out, s, sm_count);
  if (cm == 1) return launch_t<1024, 1>(g, ws, d_out, s, sm_count);
  return launch_t<1024, 2>(g, ws, d_out, s, sm_count);
}

}  // namespace fz
