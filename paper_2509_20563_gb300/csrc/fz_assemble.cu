// fz_assemble.cu -- stream assembly: copies the header, the code-length
// table, anchors, outliers and exceptions from the workspace into their
// 16-byte aligned sections of the output and zeroes the alignment gaps (the
// chunk bit lengths and the bitstream were written in place by the encoder).
// For a RAW stream it copies the input floats; for a CONST stream it writes
// the single value.
#include "fz_internal.cuh"

namespace fz {

namespace {

constexpr int kAsmThreads = 256;

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

__global__ void __launch_bounds__(kAsmThreads) k_assemble(const float *__restrict__ x, Geom g, uint32_t R,
                                                           CompressWs ws, uint8_t *d_out) {
  const Ctl *ctl = ws.ctl;
  const uint32_t mode = ctl->mode;
  const fz_header &h = ctl->res.hdr;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  const uint8_t *hb = reinterpret_cast<const uint8_t *>(&h);
  if (tid < FZ_HEADER_BYTES) d_out[tid] = hb[tid];
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
  copy_bytes(d_out + h.off_lens, ctl->lens, nsym, tid, nth);
  copy_bytes(d_out + h.off_anchors, reinterpret_cast<const uint8_t *>(ws.anchors), 4 * nb, tid, nth);
  copy_bytes(d_out + h.off_out_idx, reinterpret_cast<const uint8_t *>(ws.out_idx), 4 * n_out, tid, nth);
  copy_bytes(d_out + h.off_out_val, reinterpret_cast<const uint8_t *>(ws.out_val), 4 * n_out, tid, nth);
  copy_bytes(d_out + h.off_exc_idx, reinterpret_cast<const uint8_t *>(ws.exc_idx), 4 * n_exc, tid, nth);
  copy_bytes(d_out + h.off_exc_val, reinterpret_cast<const uint8_t *>(ws.exc_val), 4 * n_exc, tid, nth);
  if (tid == 0) {
    zero_gap(d_out, h.off_lens + nsym, h.off_anchors);
    zero_gap(d_out, h.off_anchors + 4 * nb, h.off_chunk_bits);
    zero_gap(d_out, h.off_chunk_bits + 4 * h.n_chunks, h.off_out_idx);
    zero_gap(d_out, h.off_out_idx + 4 * n_out, h.off_out_val);
    zero_gap(d_out, h.off_out_val + 4 * n_out, h.off_exc_idx);
    zero_gap(d_out, h.off_exc_idx + 4 * n_exc, h.off_exc_val);
    zero_gap(d_out, h.off_exc_val + 4 * n_exc, h.off_bits);
    zero_gap(d_out, h.off_bits + 4 * ((h.total_bits + 31) / 32), h.total_bytes);
  }
}

}  // namespace

cudaError_t launch_assemble(const float *x, const Geom &g, uint32_t R, const CompressWs &ws, uint8_t *d_out,
                            cudaStream_t s, int sm_count) {
  // the grid covers the raw-copy worst case; idle threads exit quickly
  uint64_t want = (4 * g.n / 16 + kAsmThreads - 1) / kAsmThreads;
  uint64_t grid = (uint64_t)sm_count * 8;
  if (want < grid) grid = want;
  if (grid < 2) grid = 2;
  k_assemble<<<(unsigned)grid, kAsmThreads, 0, s>>>(x, g, R, ws, d_out);
  return cudaGetLastError();
}

}  // namespace fz
