// fz_encode.cu -- chunked canonical Huffman encoder (FZModules §3.1: cuSZ's
// GPU Huffman encoder; FZMod-Default runs it on the CPU, §3.3).
//
// A tile is 8 consecutive chunks (chunk = one block of codes), one warp per
// chunk.  Each lane owns a contiguous run of codes: it sums their codeword
// lengths, the warp scans the lane totals (chunk bit length, stored in the
// stream), the CTA scans the chunk totals and a bounded decoupled look-back
// over tiles (ordered by a ticket) yields the tile's global bit offset.  The
// lanes then pack their codewords MSB-first into a shared-memory copy of the
// tile's words, and the CTA writes every word whose first bit lies inside the
// tile with plain coalesced stores.  The last, partial word also needs the
// first bits of the next tile: the CTA computes them itself by encoding the
// next tile's first 32 codes, so no word is written twice and the output
// needs no zeroing.  HBM traffic: 2 bytes read per code plus the bitstream.
#include "fz_internal.cuh"

namespace fz {

namespace {

template <int CH>
__global__ void __launch_bounds__(kEncWarps * 32) k_encode(Geom g, CompressWs ws, uint8_t *d_out) {
  constexpr int PER = CH / 32;                       // codes per lane (16 or 32)
  constexpr int kMaxWords = CH * kEncWarps * kLmax / 32 + 2;
  __shared__ uint32_t senc[kMaxSym];
  __shared__ __align__(16) uint32_t sw[kMaxWords];
  __shared__ uint32_t s_wtot[kEncWarps], s_woff[kEncWarps];
  __shared__ uint32_t s_tile;
  __shared__ unsigned long long s_base;
  __shared__ uint32_t s_tbits;

  Ctl *ctl = ws.ctl;
  if (ctl->mode != kModeNormal) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const fz_header &h = ctl->res.hdr;
  uint32_t *chunk_bits = reinterpret_cast<uint32_t *>(d_out + h.off_chunk_bits);
  uint32_t *words = reinterpret_cast<uint32_t *>(d_out + h.off_bits);
  const uint64_t n_chunks = g.n_blocks;
  const uint64_t n_tiles = (n_chunks + kEncWarps - 1) / kEncWarps;

  for (int s = tid; s < kMaxSym; s += kEncWarps * 32) senc[s] = ctl->enc[s];
  if (tid == 0) s_tile = atomicAdd(&ctl->encode_ticket, 1u);
  __syncthreads();
  const uint64_t tile = s_tile;
  if (tile >= n_tiles) return;

  // ---- lane codes and bit counts
  const uint64_t chunk = tile * kEncWarps + warp;
  const bool valid = chunk < n_chunks;
  uint32_t cw[PER];
  uint32_t lbits = 0;
  if (valid) {
    const uint4 *src = reinterpret_cast<const uint4 *>(ws.codes + chunk * CH + lane * PER);
#pragma unroll
    for (int v = 0; v < PER / 8; ++v) {
      uint4 u = src[v];
      uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        cw[8 * v + 2 * k] = senc[w4[k] & 0xffffu];
        cw[8 * v + 2 * k + 1] = senc[w4[k] >> 16];
      }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) lbits += cw[k] >> 24;
  }
  uint32_t incl = lbits;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  const uint32_t lane_off = incl - lbits;
  if (lane == 31) {
    s_wtot[warp] = incl;
    if (valid) chunk_bits[chunk] = incl;
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t acc = 0;
    for (int w = 0; w < kEncWarps; ++w) { s_woff[w] = acc; acc += s_wtot[w]; }
    s_tbits = acc;
    s_base = lookback<false>(ws.estatus, tile, acc, ctl);
    if (tile == n_tiles - 1 && s_base + acc != ctl->total_bits) set_err(ctl, FZ_ECORRUPT);
  }
  __syncthreads();
  const uint64_t base = s_base;
  const uint32_t tbits = s_tbits;
  const uint32_t rb0 = (uint32_t)(base & 31u);
  const uint32_t nwords = (rb0 + tbits + 31) / 32;
  for (uint32_t w = tid; w < nwords; w += kEncWarps * 32) sw[w] = 0;
  __syncthreads();

  // ---- pack this lane's codewords MSB-first into the shared word buffer
  if (valid) {
    uint32_t rb = rb0 + s_woff[warp] + lane_off;
    uint32_t wi = rb >> 5;
    int cnt = (int)(rb & 31u);
    unsigned long long buf = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const uint32_t L = cw[k] >> 24, c = cw[k] & 0xffffffu;
      buf |= (unsigned long long)c << (64 - cnt - (int)L);
      cnt += (int)L;
      if (cnt >= 32) {
        atomicOr(&sw[wi], (uint32_t)(buf >> 32));
        ++wi;
        buf <<= 32;
        cnt -= 32;
      }
    }
    if (cnt > 0) atomicOr(&sw[wi], (uint32_t)(buf >> 32));
  }
  __syncthreads();

  // ---- head bits of the next tile for our last, partial word
  const uint32_t r_end = (rb0 + tbits) & 31u;
  if (warp == 0 && r_end != 0 && tile + 1 < n_tiles) {
    const uint32_t need = 32 - r_end;
    const uint32_t e = senc[ws.codes[(tile + 1) * kEncWarps * (uint64_t)CH + lane]];
    const uint32_t L = e >> 24, c = e & 0xffffffu;
    uint32_t p = L;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      uint32_t v = __shfl_up_sync(0xffffffffu, p, off);
      if (lane >= off) p += v;
    }
    p -= L;  // exclusive: first bit of this codeword within the next tile
    uint32_t contrib = 0;
    if (p < need) contrib = (uint32_t)(((unsigned long long)c << (64 - p - L)) >> 32);
    uint32_t head = __reduce_or_sync(0xffffffffu, contrib);
    if (lane == 0) sw[nwords - 1] |= head >> r_end;
  }
  __syncthreads();

  // ---- store every word whose first bit lies in this tile (never past the
  // bitstream section: an inconsistent total is reported, not written)
  const uint64_t gw0 = base >> 5;
  const uint64_t wlimit = (ctl->total_bits + 31) / 32;
  if (gw0 + nwords > wlimit && tid == 0) set_err(ctl, FZ_ECORRUPT);
  for (uint32_t w = (rb0 ? 1u : 0u) + tid; w < nwords; w += kEncWarps * 32)
    if (gw0 + w < wlimit) words[gw0 + w] = sw[w];
}

}  // namespace

cudaError_t launch_encode(const Geom &g, const CompressWs &ws, uint8_t *d_out, cudaStream_t s) {
  const uint64_t n_tiles = (g.n_blocks + kEncWarps - 1) / kEncWarps;
  if (g.bsize == 512) k_encode<512><<<(unsigned)n_tiles, kEncWarps * 32, 0, s>>>(g, ws, d_out);
  else k_encode<1024><<<(unsigned)n_tiles, kEncWarps * 32, 0, s>>>(g, ws, d_out);
  return cudaGetLastError();
}

}  // namespace fz
