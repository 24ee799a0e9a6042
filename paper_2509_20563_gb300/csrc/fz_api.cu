// fz_api.cu -- the C ABI of libfz.so: argument validation, workspace sizing,
// launch order of the stage kernels and the final status read-back.  No
// stage of the compression path runs on the host.
#include <stddef.h>
#include <string.h>

#include <new>

#include "fz_host.h"

namespace {
// Records stage boundaries of one call when profiling is on.
struct StageClock {
  fz_ctx *ctx;
  cudaStream_t s;
  bool dec;
  uint32_t n = 0;
  StageClock(fz_ctx *c, cudaStream_t st, bool decompress) : ctx(c), s(st), dec(decompress) {
    if (ctx->profiling) cudaEventRecord(dec ? ctx->dev_[0] : ctx->cev[0], s);
    (dec ? ctx->nd : ctx->nc) = 0;
  }
  void mark(const char *name, int kernels) {
    ctx->launches += (uint64_t)kernels;
    if (!ctx->profiling || n >= FZ_MAX_STAGES) return;
    cudaEventRecord(dec ? ctx->dev_[n + 1] : ctx->cev[n + 1], s);
    (dec ? ctx->dname : ctx->cname)[n] = name;
    ++n;
    (dec ? ctx->nd : ctx->nc) = n;
  }
};
}  // namespace

namespace fz {
namespace {




fz_status ensure_ws(fz_ctx *ctx, size_t bytes) {
  if (ctx->ws_bytes >= bytes) return FZ_OK;
  if (ctx->ws) {
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  size_t want = bytes + bytes / 8;  // headroom so similar sizes do not reallocate
  cudaError_t e = cudaMalloc(&ctx->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&ctx->ws, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ctx->ws = nullptr;
      return FZ_ENOMEM;
    }
    want = bytes;
  }
  ctx->ws_bytes = want;
  return FZ_OK;
}

fz_status ensure_pinned(fz_ctx *ctx) {
  if (ctx->h_pinned) return FZ_OK;
  cudaError_t e = cudaMallocHost(&ctx->h_pinned, sizeof(Result) + 64);
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->h_pinned = nullptr;
    return FZ_ENOMEM;
  }
  return FZ_OK;
}

}  // namespace

// Carve the compress workspace out of two regions: the part zeroed at the
// start of every call (control block, per-tile counts, look-back status) at
// zbase, and the rest at rbase.  Returns the zeroed part's size and stores
// the rest's in *rest_bytes.  Null bases only compute the sizes.
size_t layout_compress_split(const Geom &g, char *zbase, char *rbase, CompressWs &ws, size_t *rest_bytes) {
  size_t zo = 0, ro = 0;
  auto ztake = [&](size_t bytes) {
    char *p = zbase ? zbase + zo : nullptr;
    zo += up(bytes);
    return p;
  };
  auto rtake = [&](size_t bytes) {
    char *p = rbase ? rbase + ro : nullptr;
    ro += up(bytes);
    return p;
  };
  // look-back words: one per Huffman encode tile (8 blocks) or per
  // bit-shuffle unit (4096 codes), whichever are more
  uint64_t n_etiles = (g.n_blocks + kEncWarps - 1) / kEncWarps;
  const uint64_t n_sunits = (g.npad + 4095) / 4096;
  if (n_sunits > n_etiles) n_etiles = n_sunits;
  ws.ctl = reinterpret_cast<Ctl *>(ztake(sizeof(Ctl)));
  ws.tinfo = reinterpret_cast<uint4 *>(ztake(16 * g.n_qtiles));
  ws.tgroup = reinterpret_cast<uint2 *>(ztake(8 * ((g.n_qtiles + kTileGroup - 1) / kTileGroup)));
  ws.estatus = reinterpret_cast<uint64_t *>(ztake(8 * n_etiles));
  ws.zero_bytes = zo;
  ws.cap_list = g.n / 8;
  const uint64_t cap = ws.cap_list + 1;
  ws.codes = reinterpret_cast<uint16_t *>(rtake(2 * g.npad));
  ws.anchors = reinterpret_cast<int32_t *>(rtake(4 * g.n_blocks));
  ws.out_idx = reinterpret_cast<uint32_t *>(rtake(4 * cap));
  ws.out_val = reinterpret_cast<int32_t *>(rtake(4 * cap));
  ws.exc_idx = reinterpret_cast<uint32_t *>(rtake(4 * cap));
  ws.exc_val = reinterpret_cast<uint32_t *>(rtake(4 * cap));
  ws.ids = reinterpret_cast<uint8_t *>(rtake(g.n_blocks));
  ws.tdst = reinterpret_cast<uint2 *>(rtake(8 * g.n_qtiles));
  ws.winfo = reinterpret_cast<WarpSlots *>(rtake(sizeof(WarpSlots) * 8 * g.n_qtiles));
  ws.otiles = reinterpret_cast<uint32_t *>(rtake(4 * g.n_qtiles));
  ws.h_res = nullptr;  // set by the single-field compress only
  if (rest_bytes) *rest_bytes = ro;
  return zo;
}

namespace {

// Single-field layout: the zeroed part first, the rest right after it.
size_t layout_compress(const Geom &g, char *base, CompressWs &ws) {
  size_t rest = 0;
  const size_t z = layout_compress_split(g, nullptr, nullptr, ws, &rest);
  if (base) layout_compress_split(g, base, base + z, ws, nullptr);
  return z + rest;
}

struct Req {
  uint32_t pred, R;
  uint32_t chunk;    // 0: the block size
  uint32_t encoder;  // FZ_ENC_*
  const uint16_t *weights;
};

fz_status parse_pipe(const fz_pipeline *pipe, uint32_t ndim, Req &r) {
  r.pred = FZ_PRED_LORENZO1;
  r.R = 512;
  r.chunk = 0;
  r.encoder = FZ_ENC_HUFFMAN;
  r.weights = nullptr;
  if (pipe) {
    if (pipe->struct_size < sizeof(uint32_t) * 3) return FZ_EINVAL;
    r.pred = pipe->predictor;
    if (pipe->radius) r.R = pipe->radius;
    if (pipe->struct_size >= offsetof(fz_pipeline, encoder)) {
      const uint64_t d1[3] = {1, 1, 1};
      Geom g;
      make_geom(ndim, d1, g);
      const uint32_t want[3] = {g.bx, g.by, g.bz};
      const bool dflt = !pipe->block[0] && !pipe->block[1] && !pipe->block[2];
      for (uint32_t a = 0; a < 3 && !dflt; ++a) {
        const uint32_t b = pipe->block[a];
        if (a >= ndim ? b > 1 : b == 0) return FZ_EINVAL;
        if (a < ndim && b != want[a]) return FZ_EUNSUPPORTED;
      }
      r.chunk = pipe->chunk;
    }
    if (pipe->struct_size >= sizeof(fz_pipeline)) {
      r.encoder = pipe->encoder;
      r.weights = reinterpret_cast<const uint16_t *>(pipe->selector_weights);
    }
    if (r.encoder > FZ_ENC_SHUFFLE) return FZ_EINVAL;
    if (r.encoder == FZ_ENC_SHUFFLE) {
      // the shuffle format fixes its chunk at 1024 codes
      if (pipe->predictor > FZ_PRED_LORENZO2 || (r.chunk && r.chunk != 1024)) return FZ_EUNSUPPORTED;
      r.chunk = 0;
    } else if (r.chunk) {
      const uint64_t d1[3] = {1, 1, 1};
      Geom g;
      make_geom(ndim, d1, g);
      if (!chunk_supported(ndim, g.bsize, r.chunk, pipe->predictor)) return FZ_EUNSUPPORTED;
      if (r.chunk != g.bsize && pipe->predictor > FZ_PRED_LORENZO2) return FZ_EUNSUPPORTED;
    }
  }
  if (r.R < 2 || r.R > 512) return FZ_EINVAL;
  switch (r.pred) {
    case FZ_PRED_LORENZO1:
    case FZ_PRED_LORENZO2: return FZ_OK;
    case FZ_PRED_INTERP_LIN:
    case FZ_PRED_INTERP_CUBIC:
    case FZ_PRED_GINTERP:
    case FZ_SEL_EXHAUSTIVE: return ndim == 3 ? FZ_OK : FZ_EUNSUPPORTED;
    case FZ_SEL_MLP:
      if (ndim != 3) return FZ_EUNSUPPORTED;
      return r.weights ? FZ_OK : FZ_EINVAL;
    default: return FZ_EINVAL;
  }
}

// Run range + quantization into `ws` (shared by compress and the stage call).
fz_status run_front(fz_ctx *ctx, const float *d_in, const Geom &g, uint32_t eb_mode, double eb, const Req &r,
                    const CompressWs &ws, cudaStream_t st, StageClock &clk) {
  cudaError_t e = cudaMemsetAsync(ws.ctl, 0, ws.zero_bytes, st);
  if (e != cudaSuccess) return from_cuda(e);
  clk.mark("memset", 0);
  e = launch_range(d_in, g, eb_mode, eb, ws.ctl, st);
  if (e != cudaSuccess) return from_cuda(e);
  clk.mark("range", 1);
  if (r.pred <= FZ_PRED_LORENZO2) e = launch_quant(d_in, g, r.R, r.pred, ws, st, ctx->sm_count);
  else e = launch_selquant(d_in, g, r.R, r.pred, ws, r.weights, st, ctx->sm_count);
  clk.mark("quant", 1);
  return from_cuda(e);
}


}  // namespace

// Host-side validation of a stream header against the stream length.
fz_status check_header(const fz_header &h, uint64_t in_bytes, Geom &g) {
  if (h.magic != FZ_MAGIC || h.version != 1) return FZ_ECORRUPT;
  uint64_t n;
  if (!valid_dims(h.ndim, h.dims, &n)) return FZ_ECORRUPT;
  for (uint32_t a = h.ndim; a < 3; ++a)
    if (h.dims[a] != 1) return FZ_ECORRUPT;
  if (h.total_bytes > in_bytes || h.total_bytes < FZ_HEADER_BYTES) return FZ_ECORRUPT;
  make_geom(h.ndim, h.dims, g);
  if (h.flags != FZ_FLAG_RAW && h.flags != FZ_FLAG_CONST && !positions_fit(g)) return FZ_ECORRUPT;
  if (h.flags == FZ_FLAG_RAW) return h.total_bytes == FZ_HEADER_BYTES + 4 * n ? FZ_OK : FZ_ECORRUPT;
  if (h.flags == FZ_FLAG_CONST) return h.total_bytes == FZ_HEADER_BYTES + 16 ? FZ_OK : FZ_ECORRUPT;
  if (h.flags != 0 && h.flags != FZ_FLAG_IDS && h.flags != FZ_FLAG_SHUF) return FZ_EUNSUPPORTED;
  const bool shuf = h.flags == FZ_FLAG_SHUF;
  if (h.radius < 2 || h.radius > 512) return FZ_ECORRUPT;
  const bool sel = h.predictor == FZ_SEL_MLP || h.predictor == FZ_SEL_EXHAUSTIVE;
  if (!(h.predictor <= FZ_PRED_GINTERP || sel)) return FZ_ECORRUPT;
  if (sel != (h.flags == FZ_FLAG_IDS)) return FZ_ECORRUPT;
  if (h.predictor > FZ_PRED_LORENZO2 && h.ndim != 3) return FZ_ECORRUPT;
  // every bound below is written so that no sum can wrap around 2^64: an
  // offset is first checked against the stream length, a length against
  // what is left of the stream after its offset
  auto fits = [&](uint64_t off, uint64_t len) { return off <= in_bytes && len <= in_bytes - off; };
  if (sel && (h.off_ids < FZ_HEADER_BYTES + 2ull * h.radius || (h.off_ids & 15u) ||
              !fits(h.off_ids, (h.n_blocks + 3) / 4) || h.off_ids + (h.n_blocks + 3) / 4 > h.off_anchors))
    return FZ_ECORRUPT;
  if (h.block[0] != g.bx || h.block[1] != g.by || h.block[2] != g.bz) return FZ_ECORRUPT;
  if (shuf ? (h.chunk != 1024 || h.predictor > FZ_PRED_LORENZO2) : !chunk_supported(h.ndim, g.bsize, h.chunk, h.predictor))
    return FZ_ECORRUPT;
  if (h.chunk != g.bsize && h.predictor > FZ_PRED_LORENZO2) return FZ_EUNSUPPORTED;
  if (shuf && (h.total_bits & 31u)) return FZ_ECORRUPT;
  set_chunk(g, h.chunk);
  if (h.n_blocks != g.n_blocks || h.n_chunks != g.n_chunks) return FZ_ECORRUPT;
  if (h.n_out > n || h.n_exc > n || h.total_bits > (uint64_t)kLmax * g.npad) return FZ_ECORRUPT;
  const uint64_t secs[9][2] = {{h.off_lens, sel ? h.off_ids - h.off_lens : (shuf ? 4 * (g.npad / 64) : 2ull * h.radius)},
                               {h.off_anchors, 4 * h.n_blocks},
                               {h.off_chunk_bits, 4 * h.n_chunks},   {h.off_out_idx, 4 * h.n_out},
                               {h.off_out_val, 4 * h.n_out},         {h.off_exc_idx, 4 * h.n_exc},
                               {h.off_exc_val, 4 * h.n_exc},         {h.off_bits, 4 * ((h.total_bits + 31) / 32)},
                               {h.total_bytes, 0}};
  if (h.off_lens != FZ_HEADER_BYTES) return FZ_ECORRUPT;
  for (int i = 0; i < 8; ++i) {
    if (secs[i][0] & 15u) return FZ_ECORRUPT;
    if (!fits(secs[i][0], secs[i][1])) return FZ_ECORRUPT;
    if (secs[i][0] + secs[i][1] > secs[i + 1][0]) return FZ_ECORRUPT;
  }
  return FZ_OK;
}

}  // namespace fz

using namespace fz;

extern "C" {

const char *fz_status_str(fz_status s) {
  switch (s) {
    case FZ_OK: return "ok";
    case FZ_EINVAL: return "invalid argument";
    case FZ_ENOMEM: return "out of device memory";
    case FZ_ECUDA: return "CUDA error";
    case FZ_EBUFFER: return "output buffer too small";
    case FZ_ECORRUPT: return "corrupt stream";
    case FZ_ETIMEOUT: return "device wait timed out";
    case FZ_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

fz_status fz_ctx_create(int device, fz_ctx **out) {
  if (!out) return FZ_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) { cudaGetLastError(); return FZ_ECUDA; }
  if (device < 0 || device >= n) return FZ_EINVAL;
  fz_ctx *c = new (std::nothrow) fz_ctx();
  if (!c) return FZ_ENOMEM;
  c->device = device;
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    return FZ_ECUDA;
  }
  *out = c;
  return FZ_OK;
}

fz_status fz_ctx_set_profiling(fz_ctx *ctx, int enable) {
  if (!ctx) return FZ_EINVAL;
  if (enable && !ctx->cev[0]) {
    if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
    for (int i = 0; i <= FZ_MAX_STAGES; ++i) {
      if (cudaEventCreate(&ctx->cev[i]) != cudaSuccess || cudaEventCreate(&ctx->dev_[i]) != cudaSuccess)
        return FZ_ECUDA;
    }
  }
  ctx->profiling = enable != 0;
  return FZ_OK;
}

fz_status fz_ctx_get_profile(fz_ctx *ctx, fz_profile *out) {
  if (!ctx || !out) return FZ_EINVAL;
  memset(out, 0, sizeof(*out));
  out->launches = ctx->launches;
  out->batch_plans = (uint32_t)ctx->plans.size();
  out->batch_graphs = 0;
  for (const BatchPlan *p : ctx->plans) out->batch_graphs += p->exec ? 1u : 0u;
  if (!ctx->plans.empty()) {
    const BatchTune &t = ctx->plans.back()->tune;
    out->batch_tune[0] = t.range_seg_log2;
    out->batch_tune[1] = t.quant_per_sm;
    out->batch_tune[2] = t.encode_per_sm;
    out->batch_tune[3] = t.decode_per_sm;
  }
  for (auto it = ctx->plans.rbegin(); it != ctx->plans.rend(); ++it) {
    if ((*it)->decompress) continue;
    for (int c = 0; c < 2; ++c) out->batch_chunk[c] = (*it)->chunk[c];
    break;
  }
  if (!ctx->profiling) return FZ_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
  for (int kind = 0; kind < 2; ++kind) {
    const uint32_t n = kind ? ctx->nd : ctx->nc;
    cudaEvent_t *ev = kind ? ctx->dev_ : ctx->cev;
    if (n == 0) continue;
    if (cudaEventSynchronize(ev[n]) != cudaSuccess) return FZ_ECUDA;
    for (uint32_t i = 0; i < n; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) != cudaSuccess) return FZ_ECUDA;
      const char *nm = kind ? ctx->dname[i] : ctx->cname[i];
      char *dst = kind ? out->decompress_names[i] : out->compress_names[i];
      strncpy(dst, nm ? nm : "", 15);
      (kind ? out->decompress_ms : out->compress_ms)[i] = ms;
    }
    (kind ? out->n_decompress : out->n_compress) = n;
  }
  return FZ_OK;
}

fz_status fz_ctx_destroy(fz_ctx *ctx) {
  if (!ctx) return FZ_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  for (int i = 0; i <= FZ_MAX_STAGES; ++i) {
    if (ctx->cev[i]) cudaEventDestroy(ctx->cev[i]);
    if (ctx->dev_[i]) cudaEventDestroy(ctx->dev_[i]);
  }
  destroy_batch_plans(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (int k = 0; k < 2; ++k) {
    if (ctx->bws[k]) cudaFree(ctx->bws[k]);
    if (ctx->h_batch[k]) cudaFreeHost(ctx->h_batch[k]);
  }
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  cudaSetDevice(prev);
  delete ctx;
  return FZ_OK;
}

uint64_t fz_compress_bound(uint32_t ndim, const uint64_t dims[3]) {
  uint64_t n;
  if (!valid_dims(ndim, dims, &n)) return 0;
  return align16(FZ_HEADER_BYTES + 4 * n);
}

fz_status fz_stream_info(const void *h_header, uint64_t header_bytes, uint32_t *ndim, uint64_t dims[3],
                         double *eb_abs, uint32_t *flags) {
  if (!h_header || header_bytes < FZ_HEADER_BYTES) return FZ_EINVAL;
  fz_header h;
  memcpy(&h, h_header, sizeof(h));
  uint64_t n;
  if (h.magic != FZ_MAGIC || h.version != 1 || !valid_dims(h.ndim, h.dims, &n)) return FZ_ECORRUPT;
  if (ndim) *ndim = h.ndim;
  if (dims) for (int a = 0; a < 3; ++a) dims[a] = h.dims[a];
  if (eb_abs) *eb_abs = h.eb_abs;
  if (flags) *flags = h.flags;
  return FZ_OK;
}

fz_status fz_stream_check(const void *h_header, uint64_t stream_bytes) {
  if (!h_header || stream_bytes < FZ_HEADER_BYTES) return FZ_EINVAL;
  fz_header h;
  memcpy(&h, h_header, sizeof(h));
  Geom g;
  return check_header(h, stream_bytes, g);
}

fz_status fz_compress(fz_ctx *ctx, const float *d_in, uint32_t ndim, const uint64_t dims[3], uint32_t eb_mode,
                      double eb, const fz_pipeline *pipe, void *d_out, uint64_t out_cap, uint64_t *out_bytes,
                      void *h_header, void *stream) {
  if (!ctx || !d_in || !d_out || !out_bytes) return FZ_EINVAL;
  uint64_t n;
  if (!valid_dims(ndim, dims, &n)) return FZ_EINVAL;
  if (eb_mode > FZ_EB_REL || !(eb > 0.0) || !(eb < __builtin_inf())) return FZ_EINVAL;
  if (((uintptr_t)d_out & 15u) || ((uintptr_t)d_in & 3u)) return FZ_EINVAL;
  Req r;
  fz_status st = parse_pipe(pipe, ndim, r);
  if (st) return st;
  if (out_cap < FZ_HEADER_BYTES + 4 * n) return FZ_EBUFFER;
  if (overlaps(d_in, 4 * n, d_out, out_cap)) return FZ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
  uint64_t d3[3] = {dims[0], ndim >= 2 ? dims[1] : 1, ndim >= 3 ? dims[2] : 1};
  Geom g;
  make_geom(ndim, d3, g);
  if (!positions_fit(g)) return FZ_EUNSUPPORTED;
  if (r.chunk) set_chunk(g, r.chunk);
  CompressWs ws;
  size_t need = layout_compress(g, nullptr, ws);
  if ((st = ensure_ws(ctx, need)) || (st = ensure_pinned(ctx))) return st;
  layout_compress(g, reinterpret_cast<char *>(ctx->ws), ws);
  ws.spin = ctx->spin_cycles;
  StageClock clk(ctx, s, false);
  if ((st = run_front(ctx, d_in, g, eb_mode, eb, r, ws, s, clk))) return st;
  uint8_t *out = reinterpret_cast<uint8_t *>(d_out);
  cudaError_t e;
  if (r.encoder == FZ_ENC_SHUFFLE) {
    e = launch_shuf_layout(g, r.R, r.pred, eb_mode, eb, ws, s);
    clk.mark("layout", 1);
    if (e == cudaSuccess) { e = launch_shuf_encode(g, ws, out, s, ctx->sm_count); clk.mark("encode", 1); }
  } else {
    e = launch_codebook(g, r.R, r.pred, eb_mode, eb, ws, s);
    clk.mark("codebook", 1);
    if (e == cudaSuccess) { e = launch_encode(g, ws, out, s, ctx->sm_count); clk.mark("encode", 1); }
  }
  ws.h_res = reinterpret_cast<Result *>(ctx->h_pinned);  // pinned, mapped: written by the last kernel
  if (e == cudaSuccess) { e = launch_assemble(d_in, g, r.R, ws, out, s, ctx->sm_count); clk.mark("assemble", 2); }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  const Result *res = reinterpret_cast<const Result *>(ctx->h_pinned);
  if (res->err) return (fz_status)res->err;
  *out_bytes = res->total_bytes;
  if (h_header) memcpy(h_header, &res->hdr, FZ_HEADER_BYTES);
  return FZ_OK;
}

fz_status fz_decompress(fz_ctx *ctx, const void *d_in, uint64_t in_bytes, const void *h_header, float *d_out,
                        uint64_t out_cap_values, void *stream) {
  if (!ctx || !d_in || !d_out || in_bytes < FZ_HEADER_BYTES) return FZ_EINVAL;
  if (((uintptr_t)d_in & 15u) || ((uintptr_t)d_out & 3u)) return FZ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
  fz_status st = ensure_pinned(ctx);
  if (st) return st;
  fz_header h;
  if (h_header) {
    memcpy(&h, h_header, sizeof(h));
  } else {
    cudaError_t e = cudaMemcpyAsync(ctx->h_pinned, d_in, FZ_HEADER_BYTES, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    memcpy(&h, ctx->h_pinned, sizeof(h));
  }
  Geom g;
  if ((st = check_header(h, in_bytes, g))) return st;
  if (out_cap_values < g.n) return FZ_EBUFFER;
  if (overlaps(d_in, in_bytes, d_out, 4 * g.n)) return FZ_EINVAL;
  const uint8_t *in = reinterpret_cast<const uint8_t *>(d_in);
  cudaError_t e = cudaSuccess;
  if (h.flags == FZ_FLAG_RAW) {
    e = cudaMemcpyAsync(d_out, in + FZ_HEADER_BYTES, 4 * g.n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return from_cuda(e);
  }
  if (h.flags == FZ_FLAG_CONST) {
    uint32_t bits = 0;
    e = cudaMemcpyAsync(ctx->h_pinned, in + FZ_HEADER_BYTES, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return from_cuda(e);
    memcpy(&bits, ctx->h_pinned, 4);
    e = launch_fill(d_out, g.n, bits, s, ctx->sm_count);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return from_cuda(e);
  }
  const uint64_t n_units = dec_units_of(h.n_chunks);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += up(bytes); return o; };
  const bool selpath = h.predictor > FZ_PRED_LORENZO2;
  // The per-block first-outlier table: the full-field interpolation decoder
  // always takes it (its code decoder matches every outlier code to the list
  // through it), the per-block predictor decoder whenever there are
  // outliers; for Lorenzo streams it pays off when most blocks hold outliers
  // (streams with chunks below the block and bit-shuffle streams locate
  // outliers per plane or chunk instead).
  const bool gipath = h.predictor == FZ_PRED_GINTERP;
  const bool ofirst = gipath || (selpath && h.n_out) || (!selpath && h.n_out > h.n_blocks / 8 &&
                                             h.chunk >= g.bsize && h.flags != FZ_FLAG_SHUF);
  const size_t o_err = take(dec_offset_zero_bytes(h)), o_gsum = take(8 * n_units), o_lut = take(2u << kLutBits),
               o_codes = selpath ? take(2 * g.npad) : 0, o_ofirst = ofirst ? take(4 * h.n_blocks) : 0,
               o_q4 = gipath ? take(4 * ginterp_level_values(h, 4)) : 0,
               o_q2 = gipath ? take(4 * ginterp_level_values(h, 2)) : 0,
               o_ovals = gipath ? take(4 * g.npad) : 0;
  if ((st = ensure_ws(ctx, off))) return st;
  char *base = reinterpret_cast<char *>(ctx->ws);
  DecodeWs ws;
  ws.err = reinterpret_cast<uint32_t *>(base + o_err);
  ws.lut = reinterpret_cast<uint16_t *>(base + o_lut);
  ws.gsum = reinterpret_cast<uint64_t *>(base + o_gsum);
  ws.ofirst = ofirst ? reinterpret_cast<uint32_t *>(base + o_ofirst) : nullptr;
  ws.spin = ctx->spin_cycles;
  StageClock clk(ctx, s, true);
  if (selpath) {
    e = cudaMemsetAsync(ws.err, 0, 16, s);
    if (e == cudaSuccess) { e = launch_decode_prep(in, h, ws, s); clk.mark("dec_prep", 2); }
    if (e == cudaSuccess && ofirst) e = cudaMemsetAsync(ws.ofirst, 0xff, 4 * h.n_blocks, s);
    if (e == cudaSuccess && ofirst) { e = launch_outlier_starts(in, h, ws, s, ctx->sm_count); clk.mark("outliers", 1); }
    if (e == cudaSuccess && gipath) {
      e = launch_gi_decode(in, h, d_out, ws, reinterpret_cast<uint16_t *>(base + o_codes),
                           reinterpret_cast<int32_t *>(base + o_ovals),
                           reinterpret_cast<int32_t *>(base + o_q4), reinterpret_cast<int32_t *>(base + o_q2), s,
                           ctx->sm_count);
      clk.mark("decode", 5 + (h.n_exc ? 1 : 0));
    } else if (e == cudaSuccess) {
      e = launch_sel_decode(in, h, d_out, ws, reinterpret_cast<uint16_t *>(base + o_codes), s, ctx->sm_count);
      clk.mark("decode", 2);
    }
  } else {
    // unit offsets, then the decoder (which builds its decode table itself)
    e = cudaMemsetAsync(ws.err, 0, dec_offset_zero_bytes(h), s);
    if (e == cudaSuccess) { e = launch_decode_offsets(in, h, ws, s); clk.mark("dec_offsets", 1); }
    // blocks without outliers keep ~0 in the table: a corrupt chunk that
    // decodes an outlier code there is then always reported
    if (e == cudaSuccess && ofirst) e = cudaMemsetAsync(ws.ofirst, 0xff, 4 * h.n_blocks, s);
    if (e == cudaSuccess && ofirst) { e = launch_outlier_starts(in, h, ws, s, ctx->sm_count); clk.mark("outliers", 1); }
    // the decoder's last CTA writes the error word into the pinned buffer
    ws.h_err = reinterpret_cast<uint32_t *>(ctx->h_pinned);
    *reinterpret_cast<volatile uint32_t *>(ws.h_err) = 0;
    if (e == cudaSuccess) { e = launch_decode_main(in, h, d_out, ws, s, ctx->sm_count); clk.mark("decode", 1); }
  }
  if (e == cudaSuccess && selpath) e = cudaMemcpyAsync(ctx->h_pinned, ws.err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  const uint32_t err = *reinterpret_cast<volatile const uint32_t *>(ctx->h_pinned);
  return (fz_status)err;
}

fz_status fz_lorenzo_quantize(fz_ctx *ctx, const float *d_in, uint32_t ndim, const uint64_t dims[3],
                              uint32_t eb_mode, double eb, const fz_pipeline *pipe, uint16_t *d_codes,
                              int32_t *d_anchors, uint64_t *d_hist, uint64_t *n_out, uint64_t *n_exc,
                              double *eb_abs, void *stream) {
  if (!ctx || !d_in || !d_codes || !d_anchors || !d_hist || !n_out || !n_exc || !eb_abs) return FZ_EINVAL;
  uint64_t n;
  if (!valid_dims(ndim, dims, &n)) return FZ_EINVAL;
  if (eb_mode > FZ_EB_REL || !(eb > 0.0) || !(eb < __builtin_inf())) return FZ_EINVAL;
  if (((uintptr_t)d_codes & 15u) || ((uintptr_t)d_in & 3u) || ((uintptr_t)d_anchors & 3u)) return FZ_EINVAL;
  Req r;
  fz_status st = parse_pipe(pipe, ndim, r);
  if (st) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
  uint64_t d3[3] = {dims[0], ndim >= 2 ? dims[1] : 1, ndim >= 3 ? dims[2] : 1};
  Geom g;
  make_geom(ndim, d3, g);
  if (!positions_fit(g)) return FZ_EUNSUPPORTED;
  CompressWs ws;
  size_t need = layout_compress(g, nullptr, ws);
  if ((st = ensure_ws(ctx, need)) || (st = ensure_pinned(ctx))) return st;
  layout_compress(g, reinterpret_cast<char *>(ctx->ws), ws);
  ws.codes = d_codes;
  ws.anchors = d_anchors;
  StageClock clk(ctx, s, false);
  if ((st = run_front(ctx, d_in, g, eb_mode, eb, r, ws, s, clk))) return st;
  cudaError_t e = cudaMemcpyAsync(d_hist, ws.ctl->hist, 8ull * 2 * r.R, cudaMemcpyDeviceToDevice, s);
  // gather the scalar results: counts, bound and error word
  struct Small { unsigned long long n_out, n_exc; double eb_abs; uint32_t err, mode; };
  Small *hs = reinterpret_cast<Small *>(ctx->h_pinned);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs->n_out, &ws.ctl->n_out, 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs->eb_abs, &ws.ctl->eb_abs, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs->err, &ws.ctl->res.err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  if (hs->err) return (fz_status)hs->err;
  *n_out = hs->n_out;
  *n_exc = hs->n_exc;
  *eb_abs = hs->eb_abs;
  return FZ_OK;
}

fz_status fz_huffman_codebook(fz_ctx *ctx, const uint64_t *d_hist, uint32_t nsym, uint8_t *d_lens,
                              uint32_t *d_codes, void *stream) {
  if (!ctx || !d_hist || !d_lens || !d_codes || nsym == 0 || nsym > (uint32_t)kMaxSym) return FZ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
  fz_status st = ensure_ws(ctx, up(sizeof(Ctl)));
  if (st) return st;
  Ctl *ctl = reinterpret_cast<Ctl *>(ctx->ws);
  if ((st = ensure_pinned(ctx))) return st;
  cudaError_t e = cudaMemsetAsync(&ctl->res.err, 0, 4, s);
  if (e == cudaSuccess) { e = launch_codebook_only(d_hist, nsym, d_lens, d_codes, ctl, s); ctx->launches += 1; }
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_pinned, &ctl->res.err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  uint32_t err;
  memcpy(&err, ctx->h_pinned, 4);
  return (fz_status)err;
}

fz_status fz_block_report(fz_ctx *ctx, const float *d_in, const uint64_t dims[3], uint32_t eb_mode, double eb,
                          uint32_t radius, uint8_t *d_labels, uint32_t *d_costs, uint16_t *d_features,
                          void *stream) {
  if (!ctx || !d_in || !d_labels) return FZ_EINVAL;
  uint64_t n;
  if (!valid_dims(3, dims, &n)) return FZ_EINVAL;
  if (eb_mode > FZ_EB_REL || !(eb > 0.0) || !(eb < __builtin_inf())) return FZ_EINVAL;
  const uint32_t R = radius ? radius : 512;
  if (R < 2 || R > 512 || ((uintptr_t)d_in & 3u)) return FZ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
  Geom g;
  make_geom(3, dims, g);
  CompressWs ws;
  size_t need = layout_compress(g, nullptr, ws);
  fz_status st;
  if ((st = ensure_ws(ctx, need)) || (st = ensure_pinned(ctx))) return st;
  layout_compress(g, reinterpret_cast<char *>(ctx->ws), ws);
  cudaError_t e = cudaMemsetAsync(ws.ctl, 0, ws.zero_bytes, s);
  if (e == cudaSuccess) e = launch_range(d_in, g, eb_mode, eb, ws.ctl, s);
  if (e == cudaSuccess) e = launch_select_report(d_in, g, R, ws, d_labels, d_costs, d_features, s, ctx->sm_count);
  ctx->launches += 2;
  struct Small { uint32_t err, mode; };
  Small *hs = reinterpret_cast<Small *>(ctx->h_pinned);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs->err, &ws.ctl->res.err, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs->mode, &ws.ctl->mode, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  if (hs->err) return (fz_status)hs->err;
  return hs->mode == kModeNormal ? FZ_OK : FZ_EUNSUPPORTED;
}

fz_status fz_mlp_grad(fz_ctx *ctx, const float *d_weights, const uint16_t *d_features, const uint8_t *d_labels,
                      uint32_t n, float *d_grad, float *h_loss, void *stream) {
  if (!ctx || !d_weights || !d_features || !d_labels || !d_grad || n == 0) return FZ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
  const size_t part = up(sizeof(float) * mlp_partial_floats(n));
  fz_status st;
  if ((st = ensure_ws(ctx, part + up(16))) || (st = ensure_pinned(ctx))) return st;
  float *partial = reinterpret_cast<float *>(ctx->ws);
  float *dloss = reinterpret_cast<float *>(reinterpret_cast<char *>(ctx->ws) + part);
  cudaError_t e = launch_mlp_grad(d_weights, d_features, d_labels, n, partial, d_grad, dloss, s);
  ctx->launches += 2;
  if (h_loss) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_pinned, dloss, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) memcpy(h_loss, ctx->h_pinned, 4);
  }
  return from_cuda(e);
}

fz_status fz_ctx_set_spin_limit(fz_ctx *ctx, long long cycles) {
  if (!ctx || cycles < 0) return FZ_EINVAL;
  ctx->spin_cycles = cycles;
  return FZ_OK;
}

fz_status fz_selftest_bounded_wait(fz_ctx *ctx, void *stream) {
  if (!ctx) return FZ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
  fz_status st;
  if ((st = ensure_ws(ctx, 256)) || (st = ensure_pinned(ctx))) return st;
  uint32_t *scratch = reinterpret_cast<uint32_t *>(ctx->ws);
  cudaError_t e = cudaMemsetAsync(scratch, 0, 32, s);
  if (e == cudaSuccess) { e = launch_lookback_selftest(scratch, ctx->spin_cycles, s); ctx->launches += 1; }
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_pinned, scratch, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  uint32_t err = 0;
  memcpy(&err, ctx->h_pinned, 4);
  return (fz_status)err;
}

fz_status fz_mlp_adam(fz_ctx *ctx, float *d_weights, const float *d_grad, float *d_m, float *d_v, uint32_t step,
                      float lr, float beta1, float beta2, float eps, uint16_t *d_weights_bf16, void *stream) {
  if (!ctx || !d_weights || !d_grad || !d_m || !d_v || step == 0) return FZ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
  ctx->launches += 1;
  return from_cuda(launch_adam(d_weights, d_grad, d_m, d_v, d_weights_bf16, step, lr, beta1, beta2, eps, s));
}

}  // extern "C"
