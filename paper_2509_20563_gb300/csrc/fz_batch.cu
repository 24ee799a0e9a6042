// fz_batch.cu -- batched compression and decompression of many fields of
// uneven size.
//
// Every stage of the path runs once for the whole batch, as one persistent
// kernel over a batch-wide work queue: the range over segments of every
// field, the quantizer over the tiles of every field of a class (same
// dimensionality and Lorenzo order), one codebook CTA per field, the packed
// placement of the streams, the encoder over the encode tiles of a
// chunk-size class, the assembler over the fields in turn.  The decoder
// likewise runs over the decode groups of every field of a class.  The
// fields' parameters travel in a device table, so nothing in the sequence
// depends on the host between the first launch and the final copy of the
// results: the sequence is captured once per batch shape as a CUDA graph and
// replayed by later calls with the same shape (new data pointers and error
// bounds only rewrite the table, which the graph's first node uploads).
//
// Launch shapes do not change the bytes produced (every stage is the same
// code as in the single-field path; only the scheduling differs), so they
// are left to a small autotuner: on the first call with a new batch shape it
// times candidate shapes -- the range segment size, the quantizer's and
// encoder's CTAs per SM, the decoder's CTAs per SM -- by coordinate descent
// with CUDA events, keeps the fastest, then captures the graph.  The chunk
// of the Huffman code is the block (a format parameter recorded in the
// header), so every field's stream is byte-identical to the one
// fz_compress produces for it alone.
//
// FZModules composes its pipelines from modules launched one field at a time
// (§3.3); batching many fields into one graph is this library's addition.
#include <stddef.h>
#include <string.h>

#include <new>

#include "fz_host.h"

namespace fz {

void destroy_batch_plans(fz_ctx *ctx, int kind) {
  std::vector<BatchPlan *> keep;
  for (BatchPlan *p : ctx->plans) {
    if (kind >= 0 && (int)p->decompress != kind) {
      keep.push_back(p);
      continue;
    }
    if (p->exec) cudaGraphExecDestroy(p->exec);
    delete p;
  }
  ctx->plans.swap(keep);
}

namespace {

constexpr uint32_t kMaxBatch = 65535;
constexpr int kQClasses = 6;  // (ndim 1..3) x (Lorenzo order 1..2)

inline int qclass(uint32_t ndim, uint32_t k) { return (int)(ndim - 1) * 2 + (int)(k - 1); }

// Device and pinned host memory of batched calls of one kind (0 compress,
// 1 decompress), grown with 25% headroom.  Growing either invalidates that
// kind's cached graphs (they hold the old addresses).
fz_status ensure_batch_mem(fz_ctx *ctx, int kind, size_t dev_bytes, size_t host_bytes) {
  if (ctx->bws_bytes[kind] < dev_bytes) {
    destroy_batch_plans(ctx, kind);
    if (ctx->bws[kind]) cudaFree(ctx->bws[kind]);
    ctx->bws[kind] = nullptr;
    ctx->bws_bytes[kind] = 0;
    size_t want = dev_bytes + dev_bytes / 4;
    if (cudaMalloc(&ctx->bws[kind], want) != cudaSuccess) {
      cudaGetLastError();
      want = dev_bytes;
      if (cudaMalloc(&ctx->bws[kind], want) != cudaSuccess) {
        cudaGetLastError();
        ctx->bws[kind] = nullptr;
        return FZ_ENOMEM;
      }
    }
    ctx->bws_bytes[kind] = want;
  }
  if (ctx->h_batch_bytes[kind] < host_bytes) {
    destroy_batch_plans(ctx, kind);
    if (ctx->h_batch[kind]) cudaFreeHost(ctx->h_batch[kind]);
    ctx->h_batch[kind] = nullptr;
    ctx->h_batch_bytes[kind] = 0;
    const size_t want = host_bytes + host_bytes / 4;
    if (cudaMallocHost(&ctx->h_batch[kind], want) != cudaSuccess) {
      cudaGetLastError();
      ctx->h_batch[kind] = nullptr;
      return FZ_ENOMEM;
    }
    ctx->h_batch_bytes[kind] = want;
  }
  if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return FZ_ECUDA;
  }
  return FZ_OK;
}

BatchPlan *find_plan(fz_ctx *ctx, const std::vector<uint64_t> &key) {
  for (BatchPlan *p : ctx->plans)
    if (p->key == key) return p;
  return nullptr;
}

BatchPlan *add_plan(fz_ctx *ctx, const std::vector<uint64_t> &key, bool decompress) {
  constexpr size_t kMaxPlans = 16;
  if (ctx->plans.size() >= kMaxPlans) {  // drop the oldest
    BatchPlan *old = ctx->plans.front();
    if (old->exec) cudaGraphExecDestroy(old->exec);
    delete old;
    ctx->plans.erase(ctx->plans.begin());
  }
  BatchPlan *p = new (std::nothrow) BatchPlan();
  if (!p) return nullptr;
  p->key = key;
  p->decompress = decompress;
  ctx->plans.push_back(p);
  return p;
}

// Runs `enqueue` on `s` and returns its duration in ms (negative on error).
template <class F>
float time_run(cudaStream_t s, F &&enqueue) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return -1.f; }
  float ms = -1.f;
  if (cudaEventRecord(a, s) == cudaSuccess && enqueue(s) == cudaSuccess && cudaEventRecord(b, s) == cudaSuccess &&
      cudaEventSynchronize(b) == cudaSuccess)
    cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

// Captures `enqueue` into a graph on the context's capture stream.  Returns
// null when the sequence cannot be captured (the plan then runs eagerly).
template <class F>
cudaGraphExec_t capture(fz_ctx *ctx, F &&enqueue) {
  cudaStream_t cs = ctx->cap_stream;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  const cudaError_t e = enqueue(cs);
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess && ee == cudaSuccess && graph) {
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  return exec;
}

// Coordinate descent over the candidate values of each tuned parameter;
// `run(t)` times one eager run with launch shape t (negative on error).  A
// candidate's time is the best of two runs, and it must beat the incumbent
// by 3% to replace it, so that timing noise does not pick a worse shape.
template <class R>
fz_status autotune(BatchTune &best, const std::vector<std::pair<int BatchTune::*, std::vector<int>>> &space,
                   R &&run) {
  auto best_of_two = [&](const BatchTune &t) {
    const float a = run(t), b = run(t);
    return (a < 0 || b < 0) ? -1.f : (a < b ? a : b);
  };
  if (run(best) < 0) return FZ_ECUDA;  // warm-up run (first touch of the workspace)
  float best_ms = best_of_two(best);
  if (best_ms < 0) return FZ_ECUDA;
  for (const auto &dim : space) {
    const int keep = best.*(dim.first);
    int arg = keep;
    for (int v : dim.second) {
      if (v == keep) continue;
      BatchTune t = best;
      t.*(dim.first) = v;
      const float ms = best_of_two(t);
      if (ms < 0) return FZ_ECUDA;
      if (ms < 0.97f * best_ms) { best_ms = ms; arg = v; }
    }
    best.*(dim.first) = arg;
  }
  return FZ_OK;
}

// Chunk tuning of a batched compress: for each encode class (3D; 1D and 2D)
// that has fields, the chunk multipliers 4, 2, 1 (largest first: the
// shortest stream) are tried in turn; each trial compresses the batch with
// `compress(t)` (timed, results in `offs`) and decompresses it into
// temporary device memory with fz_decompress_batch (timed, untuned, eager).
// A smaller chunk replaces the incumbent only if its round trip is at least
// 3% faster.  Every trial's round trip must succeed.
template <class C>
fz_status tune_chunks(fz_ctx *ctx, BatchTune &best, uint32_t n, const std::vector<uint32_t> *emem,
                      void *d_out, const float *const *d_in, const std::vector<Geom> &geo, cudaStream_t s,
                      C &&compress, const uint64_t *offs) {
  if (emem[0].empty() && emem[1].empty()) return FZ_OK;
  uint64_t total = 0;
  std::vector<uint64_t> at(n);
  for (uint32_t j = 0; j < n; ++j) { at[j] = total; total += up(4 * geo[j].n); }
  void *scratch = nullptr;
  if (cudaMalloc(&scratch, total) != cudaSuccess) {
    cudaGetLastError();
    return FZ_OK;  // no room to tune: keep the incumbent
  }
  std::vector<float *> outs(n);
  for (uint32_t j = 0; j < n; ++j) outs[j] = reinterpret_cast<float *>(reinterpret_cast<char *>(scratch) + at[j]);
  const bool tuning = ctx->batch_tuning, graphs = ctx->batch_graphs;
  ctx->batch_tuning = false;
  ctx->batch_graphs = false;
  std::vector<uint64_t> h(n + 1);
  fz_status st = FZ_OK;
  bool give_up = false;  // the batch itself fails (output too small, ...): the real call reports it
  auto round_trip = [&](const BatchTune &t) -> float {
    const float c = compress(t);
    if (c < 0) return -1.f;
    if (offs[n + 1]) { give_up = true; return -1.f; }
    for (uint32_t j = 0; j <= n; ++j) h[j] = offs[j];
    fz_status ds = FZ_OK;
    const float d = time_run(s, [&](cudaStream_t q) {
      ds = fz_decompress_batch(ctx, n, d_out, h.data(), outs.data(), nullptr, q);
      return ds == FZ_OK ? cudaSuccess : cudaErrorUnknown;
    });
    return (d < 0 || ds != FZ_OK) ? -1.f : c + d;
  };
  for (int c = 0; c < 2 && st == FZ_OK; ++c) {
    if (emem[c].empty()) continue;
    BatchTune t = best;
    t.chunk_log2[c] = 2;
    round_trip(t);  // warm-up of this class's chunk
    float inc = round_trip(t);
    if (give_up) break;
    if (inc < 0) { st = FZ_ECUDA; break; }
    int arg = 2;
    for (int v = 1; v >= 0; --v) {
      BatchTune u = best;
      u.chunk_log2[c] = v;
      const float a = round_trip(u), b = round_trip(u);
      if (give_up) { arg = 0; break; }
      if (a < 0 || b < 0) { st = FZ_ECUDA; break; }
      const float ms = a < b ? a : b;
      if (ms < 0.97f * inc) { inc = ms; arg = v; }
    }
    if (give_up) break;
    best.chunk_log2[c] = arg;
  }
  if (give_up) best.chunk_log2[0] = best.chunk_log2[1] = 0;
  ctx->batch_tuning = tuning;
  ctx->batch_graphs = graphs;
  destroy_batch_plans(ctx, 1);  // the untuned decompress plans of the trials
  cudaFree(scratch);
  (void)d_in;
  return st;
}

// ----------------------------------------------------------------- compress
struct CPlan {
  uint32_t n = 0;
  size_t jobs_bytes = 0, table_bytes = 0, zero_bytes = 0, res_bytes = 0;
  size_t o_jobs = 0, o_members = 0, o_res = 0, o_offs = 0, dev_bytes = 0;
  std::vector<uint32_t> qmem[kQClasses], emem[2];
  uint64_t qtiles[kQClasses] = {}, etiles[2] = {};
  uint32_t qoff[kQClasses] = {}, eoff[2] = {};
  uint64_t max_n = 0;
};

}  // namespace
}  // namespace fz

using namespace fz;

extern "C" {

uint64_t fz_compress_batch_bound(uint32_t n, const uint32_t *ndim, const uint64_t *dims) {
  if (!n || !ndim || !dims) return 0;
  uint64_t tot = 0;
  for (uint32_t j = 0; j < n; ++j) {
    uint64_t nv;
    if (!valid_dims(ndim[j], dims + 3 * j, &nv)) return 0;
    tot += align16(FZ_HEADER_BYTES + 4 * nv);
  }
  return tot;
}

fz_status fz_ctx_set_batch_options(fz_ctx *ctx, int autotune, int graphs) {
  if (!ctx) return FZ_EINVAL;
  ctx->batch_tuning = autotune != 0;
  ctx->batch_graphs = graphs != 0;
  destroy_batch_plans(ctx);
  return FZ_OK;
}

fz_status fz_compress_batch(fz_ctx *ctx, uint32_t n, const float *const *d_in, const uint32_t *ndim,
                            const uint64_t *dims, uint32_t eb_mode, const double *eb, const fz_pipeline *pipe,
                            void *d_out, uint64_t out_cap, uint64_t *h_offsets, void *stream) {
  if (!ctx || !d_in || !ndim || !dims || !eb || !d_out || !h_offsets || n == 0 || n > kMaxBatch) return FZ_EINVAL;
  if (eb_mode > FZ_EB_REL || ((uintptr_t)d_out & 15u)) return FZ_EINVAL;
  uint32_t pred = FZ_PRED_LORENZO1, R = 512, chunk = 0;
  if (pipe) {
    if (pipe->struct_size < sizeof(uint32_t) * 3) return FZ_EINVAL;
    pred = pipe->predictor;
    if (pipe->radius) R = pipe->radius;
    if (pipe->struct_size >= offsetof(fz_pipeline, encoder)) chunk = pipe->chunk;
  }
  if (R < 2 || R > 512) return FZ_EINVAL;
  if (pred > FZ_PRED_LORENZO2) return pred <= FZ_SEL_EXHAUSTIVE ? FZ_EUNSUPPORTED : FZ_EINVAL;
  const uint32_t K = pred == FZ_PRED_LORENZO2 ? 2 : 1;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;

  // ---- per-field geometry, classes and workspace sizes
  CPlan P;
  P.n = n;
  std::vector<Geom> geo(n);
  std::vector<size_t> zsz(n), rsz(n);
  size_t ztot = up(sizeof(BatchCtl)), rtot = 0;
  std::vector<uint64_t> key;
  key.reserve(8 + 4 * (size_t)n);
  key.push_back(0);
  key.push_back(n);
  key.push_back(eb_mode);
  key.push_back(R);
  key.push_back(pred);
  key.push_back(chunk);
  key.push_back((uint64_t)(uintptr_t)d_out);
  key.push_back(out_cap);
  for (uint32_t j = 0; j < n; ++j) {
    uint64_t nv;
    const uint64_t *dj = dims + 3 * j;
    if (!d_in[j] || ((uintptr_t)d_in[j] & 3u) || !valid_dims(ndim[j], dj, &nv)) return FZ_EINVAL;
    if (!(eb[j] > 0.0) || !(eb[j] < __builtin_inf())) return FZ_EINVAL;
    if (overlaps(d_in[j], 4 * nv, d_out, out_cap)) return FZ_EINVAL;
    const uint64_t d3[3] = {dj[0], ndim[j] >= 2 ? dj[1] : 1, ndim[j] >= 3 ? dj[2] : 1};
    make_geom(ndim[j], d3, geo[j]);
    if (!positions_fit(geo[j])) return FZ_EUNSUPPORTED;
    if (chunk && (chunk < geo[j].bsize || !chunk_supported(ndim[j], geo[j].bsize, chunk, pred))) return FZ_EUNSUPPORTED;
    CompressWs tmp;
    zsz[j] = layout_compress_split(geo[j], nullptr, nullptr, tmp, &rsz[j]);
    ztot += zsz[j];
    rtot += rsz[j];
    const int qc = qclass(ndim[j], K);
    P.qtiles[qc] += geo[j].n_qtiles;
    P.qmem[qc].push_back(j);
    const int ec = geo[j].bsize == 512 ? 0 : 1;
    P.etiles[ec] += (geo[j].n_blocks + kEncWarps - 1) / kEncWarps;
    P.emem[ec].push_back(j);
    if (geo[j].n > P.max_n) P.max_n = geo[j].n;
    key.push_back(ndim[j]);
    key.push_back(d3[0]);
    key.push_back(d3[1]);
    key.push_back(d3[2]);
  }
  P.zero_bytes = ztot;
  P.jobs_bytes = sizeof(BatchJob) * (size_t)n;
  P.table_bytes = P.jobs_bytes + sizeof(uint32_t) * 2 * (size_t)n;
  P.o_jobs = ztot;
  P.o_members = P.o_jobs + P.jobs_bytes;
  P.o_res = P.o_jobs + up(P.table_bytes);
  P.o_offs = P.o_res + sizeof(Result) * (size_t)n;
  P.res_bytes = sizeof(Result) * (size_t)n + sizeof(uint64_t) * ((size_t)n + 2);
  const size_t o_rest = P.o_res + up(P.res_bytes);
  P.dev_bytes = o_rest + rtot;
  const size_t host_bytes = up(P.table_bytes) + up(P.res_bytes);
  fz_status st = ensure_batch_mem(ctx, 0, P.dev_bytes, host_bytes);
  if (st) return st;

  // ---- the device table (host image in pinned memory)
  char *dbase = reinterpret_cast<char *>(ctx->bws[0]);
  char *hbase = reinterpret_cast<char *>(ctx->h_batch[0]);
  BatchJob *hjobs = reinterpret_cast<BatchJob *>(hbase);
  uint32_t *hmem = reinterpret_cast<uint32_t *>(hbase + P.jobs_bytes);
  char *hres = hbase + up(P.table_bytes);
  BatchJob *djobs = reinterpret_cast<BatchJob *>(dbase + P.o_jobs);
  const uint32_t *dmem = reinterpret_cast<const uint32_t *>(dbase + P.o_members);
  BatchCtl *bctl = reinterpret_cast<BatchCtl *>(dbase);
  {
    uint32_t m = 0;
    for (int c = 0; c < kQClasses; ++c) {
      P.qoff[c] = m;
      for (uint32_t j : P.qmem[c]) hmem[m++] = j;
    }
    for (int c = 0; c < 2; ++c) {
      P.eoff[c] = m;
      for (uint32_t j : P.emem[c]) hmem[m++] = j;
    }
  }
  auto fill = [&](const BatchTune &t) {
    size_t zo = up(sizeof(BatchCtl)), ro = o_rest;
    uint64_t qb[kQClasses] = {}, eb2[2] = {}, rseg = 0;
    for (uint32_t j = 0; j < n; ++j) {
      BatchJob &J = hjobs[j];
      memset(&J, 0, sizeof(J));
      J.x = d_in[j];
      J.g = geo[j];
      // the Huffman chunk of the field's encode class (explicit or tuned)
      set_chunk(J.g, chunk ? chunk : geo[j].bsize << t.chunk_log2[geo[j].bsize == 512 ? 0 : 1]);
      layout_compress_split(geo[j], dbase + zo, dbase + ro, J.ws, nullptr);
      J.ws.spin = ctx->spin_cycles;
      zo += zsz[j];
      ro += rsz[j];
      J.eb = eb[j];
      J.eb_mode = eb_mode;
      J.R = R;
      J.pred = pred;
      J.range_base = rseg;
      J.range_segs = eb_mode == FZ_EB_REL ? (geo[j].n + (1ull << t.range_seg_log2) - 1) >> t.range_seg_log2 : 1;
      rseg += J.range_segs;
      const int qc = qclass(geo[j].ndim, K);
      J.qtile_base = qb[qc];
      qb[qc] += geo[j].n_qtiles;
      const int ec = geo[j].bsize == 512 ? 0 : 1;
      J.etile_base = eb2[ec];
      eb2[ec] += (geo[j].n_blocks + kEncWarps - 1) / kEncWarps;
      J.out_off = 0;
    }
    return rseg;
  };
  uint8_t *out = reinterpret_cast<uint8_t *>(d_out);
  int nlaunch = 6;  // range, codebook, offsets, assemble (two kernels), results
  for (int c = 0; c < kQClasses; ++c) nlaunch += P.qmem[c].empty() ? 0 : 1;
  for (int c = 0; c < 2; ++c) nlaunch += P.emem[c].empty() ? 0 : 1;
  auto enqueue = [&](const BatchTune &t, uint64_t total_segs, cudaStream_t q) -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(dbase, 0, P.zero_bytes, q);
    if (e == cudaSuccess) e = cudaMemcpyAsync(djobs, hjobs, P.table_bytes, cudaMemcpyHostToDevice, q);
    if (e == cudaSuccess) e = launch_range_batch(djobs, n, total_segs, t.range_seg_log2, q, ctx->sm_count);
    for (int c = 0; c < kQClasses && e == cudaSuccess; ++c) {
      if (P.qmem[c].empty()) continue;
      e = launch_quant_batch(c / 2 + 1, c % 2 + 1, djobs, dmem + P.qoff[c], (uint32_t)P.qmem[c].size(), P.qtiles[c],
                             t.quant_per_sm, q, ctx->sm_count);
    }
    if (e == cudaSuccess) e = launch_codebook_batch(djobs, n, q);
    if (e == cudaSuccess) e = launch_batch_offsets(djobs, n, out_cap, bctl, q);
    for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
      if (P.emem[c].empty()) continue;
      e = launch_encode_batch(c == 0 ? 512 : 1024, djobs, dmem + P.eoff[c], (uint32_t)P.emem[c].size(), P.etiles[c],
                              &bctl->ticket[c], out, t.encode_per_sm, q, ctx->sm_count);
    }
    if (e == cudaSuccess) e = launch_assemble_batch(djobs, n, out, P.max_n, q, ctx->sm_count);
    if (e == cudaSuccess)
      e = launch_batch_results(djobs, n, bctl, reinterpret_cast<Result *>(dbase + P.o_res),
                               reinterpret_cast<uint64_t *>(dbase + P.o_offs), q);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hres, dbase + P.o_res, P.res_bytes, cudaMemcpyDeviceToHost, q);
    return e;
  };

  // ---- plan: tuned launch shape and captured graph, cached per batch shape
  BatchPlan *plan = find_plan(ctx, key);
  cudaError_t e = cudaSuccess;
  if (!plan) {
    BatchTune t{18, 0, 0, 0, {0, 0}};  // 0 = the occupancy limit
    if (ctx->batch_tuning) {
      auto run = [&](const BatchTune &c) {
        const uint64_t segs = fill(c);
        return time_run(s, [&](cudaStream_t q) { return enqueue(c, segs, q); });
      };
      std::vector<std::pair<int BatchTune::*, std::vector<int>>> space = {
          {&BatchTune::range_seg_log2, {16, 18, 20}},
          {&BatchTune::quant_per_sm, {1, 2, 0}},
          {&BatchTune::encode_per_sm, {2, 4, 0}},
      };
      if ((st = autotune(t, space, run))) return st;
      if (!chunk && (st = tune_chunks(ctx, t, n, P.emem, d_out, d_in, geo, s, [&](const BatchTune &c) {
            const uint64_t segs = fill(c);
            return time_run(s, [&](cudaStream_t q) { return enqueue(c, segs, q); });
          }, reinterpret_cast<const uint64_t *>(hres + sizeof(Result) * (size_t)n))))
        return st;
    }
    plan = add_plan(ctx, key, false);
    if (!plan) return FZ_ENOMEM;
    plan->tune = t;
    for (int c = 0; c < 2; ++c)
      plan->chunk[c] = P.emem[c].empty() ? 0u : (chunk ? chunk : (c == 0 ? 512u : 1024u) << t.chunk_log2[c]);
    if (ctx->batch_graphs) {
      const uint64_t segs = fill(t);
      plan->exec = capture(ctx, [&](cudaStream_t q) { return enqueue(t, segs, q); });
    }
  }
  const uint64_t segs = fill(plan->tune);
  e = plan->exec ? cudaGraphLaunch(plan->exec, s) : enqueue(plan->tune, segs, s);
  ctx->launches += (uint64_t)nlaunch;  // the graph holds the same kernels as the eager sequence
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  const Result *res = reinterpret_cast<const Result *>(hres);
  const uint64_t *offs = reinterpret_cast<const uint64_t *>(hres + sizeof(Result) * (size_t)n);
  if (offs[n + 1]) return (fz_status)offs[n + 1];
  for (uint32_t j = 0; j < n; ++j)
    if (res[j].err) return (fz_status)res[j].err;
  for (uint32_t j = 0; j <= n; ++j) h_offsets[j] = offs[j];
  return FZ_OK;
}

fz_status fz_decompress_batch(fz_ctx *ctx, uint32_t n, const void *d_in, const uint64_t *h_offsets,
                              float *const *d_out, const uint64_t *out_cap_values, void *stream) {
  if (!ctx || !d_in || !h_offsets || !d_out || n == 0 || n > kMaxBatch) return FZ_EINVAL;
  if ((uintptr_t)d_in & 15u) return FZ_EINVAL;
  for (uint32_t j = 0; j < n; ++j)
    if ((h_offsets[j] & 15u) || h_offsets[j + 1] < h_offsets[j] + FZ_HEADER_BYTES || !d_out[j] ||
        ((uintptr_t)d_out[j] & 3u))
      return FZ_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaSetDevice(ctx->device) != cudaSuccess) return FZ_ECUDA;
  const uint8_t *in = reinterpret_cast<const uint8_t *>(d_in);
  const uint64_t in_total = h_offsets[n];

  // ---- headers to the host (the geometry of every field)
  const size_t hdr_bytes = (size_t)FZ_HEADER_BYTES * n;
  const size_t djb = dec_job_bytes(), pjb = plain_job_bytes();
  const size_t tbl_max = djb * n + pjb * n + sizeof(uint32_t) * n;
  fz_status st = ensure_batch_mem(ctx, 1, up(16) + up(tbl_max), up(hdr_bytes) + up(tbl_max) + up(16));
  if (st) return st;
  char *hbase = reinterpret_cast<char *>(ctx->h_batch[1]);
  cudaError_t e = cudaSuccess;
  for (uint32_t j = 0; j < n && e == cudaSuccess; ++j)
    e = cudaMemcpyAsync(hbase + (size_t)FZ_HEADER_BYTES * j, in + h_offsets[j], FZ_HEADER_BYTES,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  std::vector<fz_header> hs(n);
  std::vector<Geom> geo(n);
  std::vector<uint32_t> dec, plain;
  std::vector<uint32_t> mem[kQClasses];
  uint64_t units[kQClasses] = {}, max_units = 0, max_plain = 0;
  std::vector<uint64_t> key;
  key.push_back(1);
  key.push_back(n);
  for (uint32_t j = 0; j < n; ++j) {
    memcpy(&hs[j], hbase + (size_t)FZ_HEADER_BYTES * j, sizeof(fz_header));
    const fz_header &h = hs[j];
    if ((st = check_header(h, h_offsets[j + 1] - h_offsets[j], geo[j]))) return st;
    if (out_cap_values && out_cap_values[j] < geo[j].n) return FZ_EBUFFER;
    if (overlaps(d_in, in_total, d_out[j], 4 * geo[j].n)) return FZ_EINVAL;
    if (h.flags == FZ_FLAG_RAW || h.flags == FZ_FLAG_CONST) {
      plain.push_back(j);
      if (geo[j].n > max_plain) max_plain = geo[j].n;
    } else {
      if (h.predictor > FZ_PRED_LORENZO2) return FZ_EUNSUPPORTED;
      if (h.chunk < geo[j].bsize) return FZ_EUNSUPPORTED;  // batched decode: chunks of whole blocks
      const int c = qclass(h.ndim, h.predictor == FZ_PRED_LORENZO2 ? 2 : 1);
      mem[c].push_back((uint32_t)dec.size());
      units[c] += dec_units(h);
      if (dec_units(h) > max_units) max_units = dec_units(h);
      dec.push_back(j);
    }
    key.push_back(h.flags);
    key.push_back(h.predictor);
    key.push_back(h.chunk);
    key.push_back(h.ndim);
    for (int a = 0; a < 3; ++a) key.push_back(h.dims[a]);
  }
  const uint32_t nd = (uint32_t)dec.size(), np = (uint32_t)plain.size();

  // ---- device layout: error word, tables, then per field the decode table and group sums
  const size_t tbl = djb * nd + pjb * np + sizeof(uint32_t) * nd;
  const size_t o_tbl = up(16), o_fields = o_tbl + up(tbl);
  size_t dev = o_fields;
  std::vector<size_t> o_lut(nd), o_gsum(nd);
  for (uint32_t i = 0; i < nd; ++i) {
    o_lut[i] = dev;
    dev += up(2u << kLutBits);
    o_gsum[i] = dev;
    dev += up(8 * dec_units(hs[dec[i]]));
  }
  if ((st = ensure_batch_mem(ctx, 1, dev, up(hdr_bytes) + up(tbl) + up(16)))) return st;
  char *dbase = reinterpret_cast<char *>(ctx->bws[1]);
  hbase = reinterpret_cast<char *>(ctx->h_batch[1]);
  char *htbl = hbase + up(hdr_bytes);
  uint32_t *herr = reinterpret_cast<uint32_t *>(htbl + up(tbl));
  uint32_t *derr = reinterpret_cast<uint32_t *>(dbase);
  char *ddec = dbase + o_tbl, *dplain = ddec + djb * nd;
  uint32_t *dmem = reinterpret_cast<uint32_t *>(dplain + pjb * np);
  {
    uint64_t gb[kQClasses] = {};
    for (uint32_t i = 0; i < nd; ++i) {
      const uint32_t j = dec[i];
      const fz_header &h = hs[j];
      const int c = qclass(h.ndim, h.predictor == FZ_PRED_LORENZO2 ? 2 : 1);
      fill_dec_job(htbl + djb * i, in + h_offsets[j], h, d_out[j], reinterpret_cast<uint16_t *>(dbase + o_lut[i]),
                   reinterpret_cast<uint64_t *>(dbase + o_gsum[i]), derr, gb[c]);
      gb[c] += dec_units(h);
    }
    for (uint32_t i = 0; i < np; ++i) {
      const uint32_t j = plain[i];
      fill_plain_job(htbl + djb * nd + pjb * i, in + h_offsets[j], geo[j].n, hs[j].flags == FZ_FLAG_CONST, d_out[j]);
    }
    uint32_t *hm = reinterpret_cast<uint32_t *>(htbl + djb * nd + pjb * np);
    uint32_t m = 0;
    for (int c = 0; c < kQClasses; ++c)
      for (uint32_t i : mem[c]) hm[m++] = i;
  }
  uint32_t moff[kQClasses];
  {
    uint32_t m = 0;
    for (int c = 0; c < kQClasses; ++c) { moff[c] = m; m += (uint32_t)mem[c].size(); }
  }
  int nlaunch = (nd ? 2 : 0) + (np ? 1 : 0);
  for (int c = 0; c < kQClasses; ++c) nlaunch += mem[c].empty() ? 0 : 1;
  auto enqueue = [&](const BatchTune &t, cudaStream_t q) -> cudaError_t {
    cudaError_t e2 = cudaMemsetAsync(derr, 0, 16, q);
    if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(ddec, htbl, tbl, cudaMemcpyHostToDevice, q);
    if (e2 == cudaSuccess && nd) e2 = launch_decode_batch_prep(ddec, nd, max_units, q);
    for (int c = 0; c < kQClasses && e2 == cudaSuccess; ++c) {
      if (mem[c].empty()) continue;
      e2 = launch_decode_batch_main(c / 2 + 1, c % 2 + 1, ddec, dmem + moff[c], (uint32_t)mem[c].size(), units[c],
                                    t.decode_per_sm, q, ctx->sm_count);
    }
    if (e2 == cudaSuccess && np) e2 = launch_plain_batch(dplain, np, max_plain, q, ctx->sm_count);
    if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(herr, derr, 4, cudaMemcpyDeviceToHost, q);
    return e2;
  };
  BatchPlan *plan = find_plan(ctx, key);
  if (!plan) {
    BatchTune t{18, 0, 0, 0, {0, 0}};
    if (ctx->batch_tuning && nd) {
      auto run = [&](const BatchTune &c) { return time_run(s, [&](cudaStream_t q) { return enqueue(c, q); }); };
      std::vector<std::pair<int BatchTune::*, std::vector<int>>> space = {{&BatchTune::decode_per_sm, {1, 0}}};
      if ((st = autotune(t, space, run))) return st;
    }
    plan = add_plan(ctx, key, true);
    if (!plan) return FZ_ENOMEM;
    plan->tune = t;
    if (ctx->batch_graphs) plan->exec = capture(ctx, [&](cudaStream_t q) { return enqueue(t, q); });
  }
  e = plan->exec ? cudaGraphLaunch(plan->exec, s) : enqueue(plan->tune, s);
  ctx->launches += (uint64_t)nlaunch;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  return (fz_status)*herr;
}

}  // extern "C"
