// fz_assemble.cu -- stream assembly: the header, the code-length table and
// the anchors are copied into their 16-byte aligned sections, the outliers
// and exceptions are gathered from the quantizer's per-warp scratch slots
// into code-stream order (slot offsets per tile and the list of tiles that
// hold any in k_assemble; the copies in k_gather, a warp per (tile, block)
// of those tiles in 3D, else per tile), and the alignment gaps are zeroed
// (the chunk bit lengths and the bitstream were written in place by the
// encoder).  For a RAW stream the input floats are copied; for a CONST
// stream the single value is written.  k_gather, the last kernel of a
// single-field compress, also copies the call's result to the host.
#include "fz_internal.cuh"

namespace fz {

namespace {

constexpr int kAsmThreads = 256;
constexpr int kTilesPerThread = kTileGroup / kAsmThreads;

// Grid-stride byte copy using the widest access both pointers allow.
__device__ void copy_bytes(uint8_t *dst, const uint8_t *src, uint64_t n, uint64_t tid, uint64_t nth) {
  if ((((uintptr_t)dst | (uintptr_t)src) & 15u) == 0) {
    const uint64_t n16 = n / 16;
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    for (uint64_t i = tid; i < n16; i += nth) d[i] = __ldcs(s + i);
    for (uint64_t i = n16 * 16 + tid; i < n; i += nth) dst[i] = src[i];
  } else if ((((uintptr_t)dst | (uintptr_t)src) & 3u) == 0) {
    const uint64_t n4 = n / 4;
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    for (uint64_t i = tid; i < n4; i += nth) d[i] = s[i];
    for (uint64_t i = n4 * 4 + tid; i < n; i += nth) dst[i] = src[i];
  } else {
    for (uint64_t i = tid; i < n; i += nth) dst[i] = src[i];
  }
}

__device__ void zero_gap(uint8_t *out, uint64_t from, uint64_t to) {
  for (uint64_t i = from; i < to; ++i) out[i] = 0;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ uint2 block_exscan2(uint2 v, uint2 &excl, uint2 *sw) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint2 inc = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t a = __shfl_up_sync(0xffffffffu, inc.x, off), b = __shfl_up_sync(0xffffffffu, inc.y, off);
    if (lane >= off) { inc.x += a; inc.y += b; }
  }
  if (lane == 31) sw[warp] = inc;
  __syncthreads();
  uint2 wpre = make_uint2(0, 0), tot = make_uint2(0, 0);
  for (int w = 0; w < kAsmThreads / 32; ++w) {
    if (w < warp) { wpre.x += sw[w].x; wpre.y += sw[w].y; }
    tot.x += sw[w].x;
    tot.y += sw[w].y;
  }
  excl = make_uint2(wpre.x + inc.x - v.x, wpre.y + inc.y - v.y);
  __syncthreads();
  return tot;
}

struct AsmSmem {
  uint2 sw[kAsmThreads / 32];
  unsigned long long ob, eb;
};

// Assembly of one field's stream by CTAs bid = 0..nblk-1 (all threads of
// each CTA call it together).
// pad16: also zero the bytes from the stream's end to the next 16-byte
// boundary (batched calls pack the streams at 16-byte offsets; a RAW stream of
// N floats ends unaligned when N is not a multiple of 4).
__device__ __forceinline__ void assemble_body(const float *__restrict__ x, const Geom &g, uint32_t R,
                                              const CompressWs &ws, uint8_t *d_out, uint32_t bid, uint32_t nblk,
                                              AsmSmem &sm, bool pad16 = false) {
  uint2 *sw = sm.sw;
  unsigned long long &s_ob = sm.ob, &s_eb = sm.eb;
  const Ctl *ctl = ws.ctl;
  const uint32_t mode = ctl->mode;
  const fz_header &h = ctl->res.hdr;
  const uint64_t tid = (uint64_t)bid * blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)nblk * blockDim.x;
  const uint8_t *hb = reinterpret_cast<const uint8_t *>(&h);
  if (tid < FZ_HEADER_BYTES) d_out[tid] = hb[tid];
  if (pad16 && tid < 16) {
    const uint64_t t = h.total_bytes;
    if (t + tid < align16(t)) d_out[t + tid] = 0;
  }
  if (mode == kModeRaw) {
    copy_bytes(d_out + FZ_HEADER_BYTES, reinterpret_cast<const uint8_t *>(x), 4 * g.n, tid, nth);
    return;
  }
  if (mode == kModeConst) {
    if (tid < 16) d_out[FZ_HEADER_BYTES + tid] = tid < 4 ? (uint8_t)(ctl->const_bits >> (8 * tid)) : 0;
    return;
  }
  const uint32_t nsym = 2 * R;
  const uint64_t nb = h.n_blocks, n_out = h.n_out, n_exc = h.n_exc;
  uint64_t lens_end = h.off_lens + nsym;
  if (h.flags & FZ_FLAG_SHUF) lens_end = h.off_lens + 4 * (g.npad / 64);  // the encoder wrote the word maps
  else copy_bytes(d_out + h.off_lens, ctl->lens, nsym, tid, nth);
  copy_bytes(d_out + h.off_anchors, reinterpret_cast<const uint8_t *>(ws.anchors), 4 * nb, tid, nth);
  if (h.flags & FZ_FLAG_IDS) {
    // 2-bit predictor ids, four blocks per byte, first block in the low bits
    const uint64_t nbytes = (nb + 3) / 4;
    for (uint64_t i = tid; i < nbytes; i += nth) {
      uint8_t v = 0;
      for (int k = 0; k < 4; ++k)
        if (4 * i + k < nb) v |= (uint8_t)((ws.ids[4 * i + k] & 3u) << (2 * k));
      d_out[h.off_ids + i] = v;
    }
    if (tid == 0) zero_gap(d_out, lens_end, h.off_ids);
    lens_end = h.off_ids + nbytes;
  }
  if (tid == 0) {
    zero_gap(d_out, lens_end, h.off_anchors);
    zero_gap(d_out, h.off_anchors + 4 * nb, h.off_chunk_bits);
    zero_gap(d_out, h.off_chunk_bits + 4 * h.n_chunks, h.off_out_idx);
    zero_gap(d_out, h.off_out_idx + 4 * n_out, h.off_out_val);
    zero_gap(d_out, h.off_out_val + 4 * n_out, h.off_exc_idx);
    zero_gap(d_out, h.off_exc_idx + 4 * n_exc, h.off_exc_val);
    zero_gap(d_out, h.off_exc_val + 4 * n_exc, h.off_bits);
    zero_gap(d_out, h.off_bits + 4 * ((h.total_bits + 31) / 32), h.total_bytes);
  }
  if ((n_out | n_exc) == 0) return;
  // ---- every tile's first outlier and exception slot in the stream (tile
  // order = code-stream order): one CTA per group of kTileGroup tiles; the
  // copies follow in gather_body
  const uint64_t n_tg = (g.n_qtiles + kTileGroup - 1) / kTileGroup;
  for (uint64_t grp = bid; grp < n_tg; grp += nblk) {
    // totals of the earlier groups
    unsigned long long po = 0, pe = 0;
    for (uint64_t q = threadIdx.x; q < grp; q += kAsmThreads) { po += ws.tgroup[q].x; pe += ws.tgroup[q].y; }
    for (int off = 16; off > 0; off >>= 1) {
      po += __shfl_down_sync(0xffffffffu, po, off);
      pe += __shfl_down_sync(0xffffffffu, pe, off);
    }
    if (threadIdx.x == 0) { s_ob = 0; s_eb = 0; }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { atomicAdd(&s_ob, po); atomicAdd(&s_eb, pe); }
    __syncthreads();
    const unsigned long long ob = s_ob, eb = s_eb;
    // this thread's tiles
    const uint64_t t0 = grp * kTileGroup + (uint64_t)threadIdx.x * kTilesPerThread;
    uint2 cnt[kTilesPerThread];
    uint2 mine = make_uint2(0, 0);
#pragma unroll
    for (int k = 0; k < kTilesPerThread; ++k) {
      const uint4 ti = (t0 + k < g.n_qtiles) ? ws.tinfo[t0 + k] : make_uint4(0, 0, 0, 0);
      cnt[k] = make_uint2(ti.x, ti.y);
      mine.x += ti.x;
      mine.y += ti.y;
    }
    uint2 excl;
    block_exscan2(mine, excl, sw);
    unsigned long long o = ob + excl.x, e = eb + excl.y;
#pragma unroll
    for (int k = 0; k < kTilesPerThread; ++k) {
      if (t0 + k < g.n_qtiles) {
        ws.tdst[t0 + k] = make_uint2((uint32_t)o, (uint32_t)e);
        if (cnt[k].x | cnt[k].y)  // list the tile for the gather
          ws.otiles[atomicAdd(&const_cast<Ctl *>(ctl)->n_otiles, 1u)] = (uint32_t)(t0 + k);
      }
      o += cnt[k].x;
      e += cnt[k].y;
    }
    __syncthreads();
  }
}

// The ordered gather of the outliers and exceptions: each tile's entries
// are contiguous in the scratch lists and go to the stream slots computed
// by assemble_body.  A warp takes one item (a tile, or in 3D Lorenzo one
// block of a tile) whose entries sit in 8 slices of the scratch lists (one
// per quantizer warp): lane k < 8 holds slice k's count n and start slot,
// and the warp copies the item's entries as one range -- entry i lies in
// the last slice whose prefix offset is <= i -- with four entries in flight
// per lane.
__device__ __forceinline__ void gather_range(uint32_t n, uint32_t slot, uint64_t dst, uint64_t limit, uint64_t cap,
                                             const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ sval,
                                             uint32_t *didx, uint32_t *dval) {
  const int lane = threadIdx.x & 31;
  uint32_t incl = n;  // inclusive prefix of the 8 counts (lanes 8..31 hold 0)
#pragma unroll
  for (int off = 1; off < 8; off <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
    if ((lane & 7) >= off) incl += v;
  }
  const uint32_t total = __shfl_sync(0xffffffffu, incl, 7);
  if (total == 0) return;
  uint32_t ex[8], base[8];  // slice k: prefix offset, start slot - prefix offset (mod 2^32)
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    ex[k] = __shfl_sync(0xffffffffu, incl - n, k);
    base[k] = __shfl_sync(0xffffffffu, slot, k) - ex[k];
  }
  for (uint32_t i0 = 0; i0 < total; i0 += 128) {
    uint32_t vi[4], vv[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t i = i0 + 32 * u + lane;
      uint32_t b = base[0];
#pragma unroll
      for (int k = 1; k < 8; ++k) b = i >= ex[k] ? base[k] : b;
      const uint64_t src = (uint32_t)(b + i);
      ok[u] = i < total && src < cap && dst + i < limit;
      vi[u] = ok[u] ? __ldg(sidx + src) : 0u;
      vv[u] = ok[u] ? __ldg(sval + src) : 0u;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t i = i0 + 32 * u + lane;
      if (ok[u]) {
        didx[dst + i] = vi[u];
        dval[dst + i] = vv[u];
      }
    }
  }
}

__device__ __forceinline__ void gather_body(const Geom &g, const CompressWs &ws, uint8_t *d_out, uint64_t w,
                                            uint64_t nw) {
  const Ctl *ctl = ws.ctl;
  if (ctl->mode != kModeNormal) return;
  const fz_header &h = ctl->res.hdr;
  const uint64_t n_out = h.n_out, n_exc = h.n_exc;
  if ((n_out | n_exc) == 0) return;
  uint32_t *oidx = reinterpret_cast<uint32_t *>(d_out + h.off_out_idx);
  uint32_t *oval = reinterpret_cast<uint32_t *>(d_out + h.off_out_val);
  uint32_t *eidx = reinterpret_cast<uint32_t *>(d_out + h.off_exc_idx);
  uint32_t *eval = reinterpret_cast<uint32_t *>(d_out + h.off_exc_val);
  const uint32_t *s_oval = reinterpret_cast<const uint32_t *>(ws.out_val);
  const int lane = threadIdx.x & 31;
  // the 3D Lorenzo quantizer files 8 slices per warp (one per block, by
  // block then warp); the other quantizers one slice per warp
  const bool by_block = g.ndim == 3 && h.predictor <= FZ_PRED_LORENZO2;
  const uint64_t n_list = ctl->n_otiles;
  const uint64_t n_items = by_block ? n_list * 8 : n_list;
  auto bytesum = [](unsigned long long v) -> uint32_t {
    return (uint32_t)__dp4a((uint32_t)v, 0x01010101u, 0u) + (uint32_t)__dp4a((uint32_t)(v >> 32), 0x01010101u, 0u);
  };
  for (uint64_t item = w; item < n_items; item += nw) {
    const uint64_t tile = ws.otiles[by_block ? item >> 3 : item];
    const uint2 dst = ws.tdst[tile];
    uint32_t no = 0, ne = 0, so = 0, se = 0;
    uint64_t o = dst.x, e = dst.y;
    if (by_block) {
      // a (tile, block) item: the block's slices follow the earlier blocks'
      // entries of each quantizer warp's slice
      const int b = (int)(item & 7);
      const unsigned long long below = b ? (1ull << (8 * b)) - 1 : 0ull;
      uint32_t po = 0, pe = 0;
      if (lane < 8) {
        const WarpSlots wsl = ws.winfo[tile * 8 + lane];
        no = (uint32_t)(wsl.ocnt >> (8 * b)) & 255u;
        ne = (uint32_t)(wsl.ecnt >> (8 * b)) & 255u;
        po = bytesum(wsl.ocnt & below);
        pe = bytesum(wsl.ecnt & below);
        so = wsl.oslot + po;
        se = wsl.eslot + pe;
      }
      o += __reduce_add_sync(0xffffffffu, po);
      e += __reduce_add_sync(0xffffffffu, pe);
    } else if (lane < 8) {
      const WarpSlots wsl = ws.winfo[tile * 8 + lane];
      no = (uint32_t)(wsl.ocnt & 0xffffu);
      ne = (uint32_t)(wsl.ecnt & 0xffffu);
      so = wsl.oslot;
      se = wsl.eslot;
    }
    gather_range(no, so, o, n_out, ws.cap_list, ws.out_idx, s_oval, oidx, oval);
    gather_range(ne, se, e, n_exc, ws.cap_list, ws.exc_idx, ws.exc_val, eidx, eval);
  }
}

__global__ void __launch_bounds__(kAsmThreads) k_assemble(const float *__restrict__ x, Geom g, uint32_t R,
                                                           CompressWs ws, uint8_t *d_out) {
  __shared__ AsmSmem sm;
  dep_wait();
  dep_trigger();
  assemble_body(x, g, R, ws, d_out, blockIdx.x, gridDim.x, sm);
}

__global__ void __launch_bounds__(kAsmThreads) k_gather(Geom g, CompressWs ws, uint8_t *d_out) {
  dep_wait();
  // the call's result, final once the encoder has run, goes straight to the
  // host's pinned buffer (no device-to-host copy after the kernels)
  if (blockIdx.x == 0 && threadIdx.x < 32 && ws.h_res) {
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(&ws.ctl->res);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(ws.h_res);
    for (int i = threadIdx.x; i < (int)(sizeof(Result) / 8); i += 32) dst[i] = src[i];
    __threadfence_system();
  }
  const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  gather_body(g, ws, d_out, w, (uint64_t)gridDim.x * (blockDim.x >> 5));
}

// Batched variant: the whole grid assembles the fields one after another.
__global__ void __launch_bounds__(kAsmThreads) k_assemble_batch(const BatchJob *__restrict__ jobs, uint32_t n,
                                                                 uint8_t *d_out) {
  __shared__ AsmSmem sm;
  for (uint32_t j = 0; j < n; ++j) {
    const BatchJob &J = jobs[j];
    if (J.out_off == kNoOutput) continue;
    assemble_body(J.x, J.g, J.R, J.ws, d_out + J.out_off, blockIdx.x, gridDim.x, sm, true);
  }
}

__global__ void __launch_bounds__(kAsmThreads) k_gather_batch(const BatchJob *__restrict__ jobs, uint32_t n,
                                                               uint8_t *d_out) {
  const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint32_t j = 0; j < n; ++j) {
    const BatchJob &J = jobs[j];
    if (J.out_off == kNoOutput) continue;
    gather_body(J.g, J.ws, d_out + J.out_off, w, nw);
  }
}

}  // namespace

cudaError_t launch_assemble_batch(const BatchJob *jobs, uint32_t n, uint8_t *d_out, uint64_t max_n, cudaStream_t s,
                                  int sm_count) {
  uint64_t grid = (uint64_t)sm_count * 4;
  const uint64_t want = (4 * max_n / 16 + kAsmThreads - 1) / kAsmThreads;
  if (want < grid) grid = want;
  if (grid < 2) grid = 2;
  k_assemble_batch<<<(unsigned)grid, kAsmThreads, 0, s>>>(jobs, n, d_out);
  k_gather_batch<<<(unsigned)(sm_count * 8), kAsmThreads, 0, s>>>(jobs, n, d_out);
  return cudaGetLastError();
}

cudaError_t launch_assemble(const float *x, const Geom &g, uint32_t R, const CompressWs &ws, uint8_t *d_out,
                            cudaStream_t s, int sm_count) {
  // the grid covers the raw-copy worst case and the tile groups; idle threads exit quickly
  uint64_t want = (4 * g.n / 16 + kAsmThreads - 1) / kAsmThreads;
  uint64_t grid = (uint64_t)sm_count * 8;
  if (want < grid) grid = want;
  const uint64_t n_tg = (g.n_qtiles + kTileGroup - 1) / kTileGroup;
  if (grid < n_tg) grid = n_tg < (uint64_t)sm_count * 8 ? n_tg : (uint64_t)sm_count * 8;
  if (grid < 2) grid = 2;
  cudaError_t e = launch_dep(k_assemble, (unsigned)grid, (unsigned)kAsmThreads, 0, s, x, g, R, ws, d_out);
  if (e != cudaSuccess) return e;
  uint64_t ggrid = (8 * g.n_qtiles + kAsmThreads / 32 - 1) / (kAsmThreads / 32);
  if (ggrid > (uint64_t)sm_count * 8) ggrid = (uint64_t)sm_count * 8;
  return launch_dep(k_gather, (unsigned)ggrid, (unsigned)kAsmThreads, 0, s, g, ws, d_out);
}

}  // namespace fz
