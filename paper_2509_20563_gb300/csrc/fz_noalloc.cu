// fz_noalloc.cu -- decompression that allocates nothing.
//
// fz_decompress keeps its scratch (error word, per-unit bit offsets) in a
// context workspace that it grows with cudaMalloc, and reads the
// error word back through pinned host memory.  Some callers cannot allow
// either: code that runs while another component owns the device's memory
// budget (a framework's caching allocator holding the whole pool), code in
// latency-critical paths where the implicit device synchronization of
// cudaMalloc/cudaFree is not acceptable, or code that must not leave a
// library-owned allocation behind.  fz_decompress_noalloc serves them: its
// scratch is the fixed array below, in the library's own device image, and
// the call makes no allocation of any kind -- no cudaMalloc, cudaFree,
// cudaMallocHost or allocating library routine, and no context.
//
// The array holds the error word and work-unit counter (cleared at the start
// of every call) and one bit offset per work unit of 32 chunks (the decoder
// builds its decode table in shared memory), so it bounds the stream: at
// most FZ_NOALLOC_MAX_CHUNKS chunks (Huffman blocks).  Larger streams are
// rejected with FZ_EBUFFER before any device work.  Every call on a device
// shares the one array: calls whose device work overlaps (on different
// streams, or from different host threads) race on it and must be ordered by
// the caller.  Every call looks the array's address up with
// cudaGetSymbolAddress on the current device, so the calls stay valid after
// the device's context is recreated.
#include <string.h>

#include "fz_host.h"

namespace fz {
namespace {

constexpr size_t kNaErrBytes = 256;  // decoder control words, look-back words of the offset pass (<= 28 CTAs)
constexpr size_t kNaUnitBytes = 8 * (FZ_NOALLOC_MAX_CHUNKS / kDecUnit);  // per-unit bit offsets
constexpr size_t kNaScratchBytes = kNaErrBytes + kNaUnitBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

// Device address of the scratch array in the current device's context.
// Looked up on every call (a cheap query that allocates nothing): a cached
// address would go stale if the context were torn down and recreated, for
// example after cudaDeviceReset, which loads the module at a new address.
fz_status scratch_ptr(void **out) {
  void *p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return FZ_ECUDA;
  }
  *out = p;
  return FZ_OK;
}

}  // namespace
}  // namespace fz

using namespace fz;

extern "C" {

fz_status fz_decompress_noalloc(const void *d_in, uint64_t in_bytes, const void *h_header, float *d_out,
                                uint64_t out_cap_values, void *stream) {
  if (!d_in || !d_out || in_bytes < FZ_HEADER_BYTES) return FZ_EINVAL;
  if (((uintptr_t)d_in & 15u) || ((uintptr_t)d_out & 3u)) return FZ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return FZ_ECUDA; }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FZ_ECUDA;
  fz_header h;
  cudaError_t e = cudaSuccess;
  if (h_header) {
    memcpy(&h, h_header, sizeof(h));
  } else {
    // pageable destination: a plain staged copy, no allocation
    e = cudaMemcpyAsync(&h, d_in, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
  }
  Geom g;
  fz_status st = check_header(h, in_bytes, g);
  if (st) return st;
  if (out_cap_values < g.n) return FZ_EBUFFER;
  if (overlaps(d_in, in_bytes, d_out, 4 * g.n)) return FZ_EINVAL;
  const uint8_t *in = reinterpret_cast<const uint8_t *>(d_in);
  if (h.flags == FZ_FLAG_RAW) {
    e = cudaMemcpyAsync(d_out, in + FZ_HEADER_BYTES, 4 * g.n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return from_cuda(e);
  }
  if (h.flags == FZ_FLAG_CONST) {
    uint32_t bits = 0;
    e = cudaMemcpyAsync(&bits, in + FZ_HEADER_BYTES, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = launch_fill(d_out, g.n, bits, s, sms);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return from_cuda(e);
  }
  // the per-block predictor streams need a code buffer of the field's size
  if (h.predictor > FZ_PRED_LORENZO2) return FZ_EUNSUPPORTED;
  if (h.n_chunks > FZ_NOALLOC_MAX_CHUNKS) return FZ_EBUFFER;
  void *base = nullptr;
  if ((st = scratch_ptr(&base))) return st;
  char *b = reinterpret_cast<char *>(base);
  DecodeWs ws;
  ws.err = reinterpret_cast<uint32_t *>(b);
  ws.lut = nullptr;
  ws.gsum = reinterpret_cast<uint64_t *>(b + kNaErrBytes);
  // error word, work-unit counter and the offset pass's look-back words start at zero
  e = cudaMemsetAsync(ws.err, 0, dec_offset_zero_bytes(h), s);
  if (e == cudaSuccess) e = launch_decode_offsets(in, h, ws, s);
  if (e == cudaSuccess) e = launch_decode_main(in, h, d_out, ws, s, sms);
  uint32_t err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, ws.err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  return (fz_status)err;
}

}  // extern "C"
