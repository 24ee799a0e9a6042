/*
 * fz.h -- C ABI of the GB300 error-bounded compression library (libfz.so).
 *
 * The library implements the data-parallel hot path of the FZMod-Default
 * pipeline of FZModules (§3.3): value-range preprocessing (§3.2), Lorenzo
 * dual-quant prediction with a fixed code radius and outliers (§3.1), a
 * histogram of the quantization codes (§3.2), a canonical Huffman codebook and
 * a chunked Huffman encoder (§3.1-§3.2), and the inverse path (decode, outlier
 * scatter, inverse Lorenzo, dequantization; §3.3.1).  Every stage runs as a
 * CUDA kernel for sm_103a; the host code only validates arguments, sizes the
 * workspace and launches.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers on the context's device; h_* are
 *     host pointers.  The caller owns all buffers it passes.  The context owns
 *     its workspace (device scratch), which grows on demand, and a small
 *     pinned host block into which the last kernel of a compress or
 *     decompress writes the call's result or error word.
 *   - Fields are float32, C order with x fastest: dims[0] = nx (fastest),
 *     dims[1] = ny, dims[2] = nz.  Unused trailing dims must be 1 or are
 *     ignored beyond ndim.  1 <= ndim <= 3, every dim >= 1, N = prod(dims) <
 *     2^32.
 *   - Every call returns an fz_status and never throws.  Argument errors are
 *     detected before any launch.  On an error the contents of the output
 *     buffer are unspecified.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that return sizes or device-detected errors
 *     synchronize that stream before returning.
 *   - A context may be used by one host thread at a time; distinct contexts
 *     are independent.
 */
#ifndef FZ_H
#define FZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FZ_OK = 0,
  FZ_EINVAL = 1,        /* bad argument (null pointer, bad dims, eb <= 0 or not finite, ...) */
  FZ_ENOMEM = 2,        /* device workspace could not be allocated */
  FZ_ECUDA = 3,         /* a CUDA runtime call failed */
  FZ_EBUFFER = 4,       /* output buffer too small */
  FZ_ECORRUPT = 5,      /* compressed stream failed validation */
  FZ_ETIMEOUT = 6,      /* a bounded device-side wait expired */
  FZ_EUNSUPPORTED = 7   /* valid request this build does not implement */
} fz_status;

typedef enum {
  FZ_EB_ABS = 0,        /* eb is the absolute bound */
  FZ_EB_REL = 1         /* eb is relative to the value range (max - min over finite values), §3.2, §4.2 */
} fz_eb_mode;

typedef enum {
  FZ_PRED_LORENZO1 = 0, /* first-order Lorenzo, 1D/2D/3D (cuSZ, §3.1) */
  FZ_PRED_LORENZO2 = 1, /* second-order Lorenzo, 1D/2D/3D */
  FZ_PRED_INTERP_LIN = 2,   /* block-local interpolation (3D), the selector's candidates */
  FZ_PRED_INTERP_CUBIC = 3,
  FZ_PRED_GINTERP = 4,      /* full-field multilevel interpolation, FZMod-Quality's G-Interp predictor (§3.3,
                               from cuSZ-i via §3.1-§3.2), 3D only: anchors at the points whose coordinates
                               are all multiples of 8; levels 4, 2, 1, passes along x, y, z; cubic from
                               p +- s, p +- 3s where all four lie in the domain, else linear, else p - s;
                               Huffman encoder with the default chunk only */
  FZ_SEL_MLP = 16,      /* per-block predictor picked by the learned selector */
  FZ_SEL_EXHAUSTIVE = 17/* per-block predictor picked by exhaustive trial */
} fz_predictor;

/* Pipeline description: the modules of one pipeline (§3.2-§3.3: predictor,
 * quantization radius, block shape of the predictor, Huffman chunk size).
 * Zero-initialise and set struct_size = sizeof(fz_pipeline).  A NULL
 * pipeline pointer means: first-order Lorenzo, radius 512, default block,
 * default chunk. */
typedef struct {
  uint32_t struct_size;
  uint32_t predictor;          /* fz_predictor */
  uint32_t radius;             /* code radius R, 2..512; 0 selects 512 */
  uint32_t block[3];           /* predictor block extents x, y, z; all 0 = the default for ndim (1D 1024,
                                  2D 32x32, 3D 8x8x8), which is also the only shape this build accepts
                                  (others: FZ_EUNSUPPORTED); axes beyond ndim must be 0 or 1 */
  uint32_t chunk;              /* symbols per Huffman chunk (§3.2 chunked encoder; chunk j holds code-stream
                                  symbols [jC, (j+1)C)); 0 = the block size.  Also: a power-of-two multiple
                                  of the block up to 4096; 3D: 64 (one 8x8 plane of a block); 2D first-order
                                  Lorenzo: 128, 256 or 512 (4, 8 or 16 rows of a 32x32 block, decoded by
                                  neighbouring lanes that pass each other the column state); Lorenzo
                                  predictors only for chunks other than the block; else FZ_EUNSUPPORTED */
  uint32_t encoder;            /* FZ_ENC_HUFFMAN (0) or FZ_ENC_SHUFFLE (1, the bit-shuffle + zero-word encoder of
                                  FZMod-Speed, §3.3; Lorenzo predictors only, chunk 0 or 1024) */
  const void *selector_weights;/* device pointer to a selector weight blob (FZ_SEL_MLP only) */
} fz_pipeline;

/* The 256-byte little-endian stream header.  Sections follow at 16-byte
 * aligned offsets: lens u8[2R], [predictor ids], anchors i32[n_blocks],
 * chunk_bits u32[n_chunks], outlier index u32[n_out], outlier residual
 * i32[n_out], exception index u32[n_exc], exception bits u32[n_exc], then the
 * MSB-first bitstream in u32 words.  A RAW stream is the header followed by
 * the N input floats; a CONST stream is the header followed by one float
 * (padded to 16 bytes).  For RAW and CONST streams only magic, version,
 * flags, ndim, eb_mode, dims, eb and total_bytes are set; the rest is 0. */
typedef struct {
  uint32_t magic;              /* 'F','Z','G','B' */
  uint16_t version;            /* 1 */
  uint16_t flags;              /* FZ_FLAG_* */
  uint32_t ndim;
  uint32_t eb_mode;
  uint64_t dims[3];
  double eb;                   /* as requested */
  double eb_abs;               /* absolute bound used */
  uint32_t ebx2_bits;          /* float32 quantization bin width */
  uint32_t inv2eb_bits;        /* float32 reciprocal of the bin width */
  uint32_t ebchk_bits;         /* float32 per-value check bound */
  uint32_t radius;
  uint32_t block[3];
  uint32_t predictor;          /* fz_predictor used for every block, or FZ_SEL_* when ids are stored */
  uint32_t chunk;              /* symbols per Huffman chunk (see fz_pipeline.chunk) */
  uint32_t reserved0;
  uint64_t n_blocks, n_chunks, n_out, n_exc, total_bits;
  uint64_t off_lens, off_ids, off_anchors, off_chunk_bits, off_out_idx, off_out_val,
      off_exc_idx, off_exc_val, off_bits, total_bytes;
  uint8_t pad[40];
} fz_header;

#define FZ_MAGIC 0x42475A46u
#define FZ_HEADER_BYTES 256u
#define FZ_FLAG_RAW 1u
#define FZ_FLAG_CONST 2u
#define FZ_FLAG_IDS 4u
#define FZ_FLAG_SHUF 8u  /* bit-shuffle stream: the lens section holds one u32 map of nonzero column words per 64
                            codes, the chunk (1024 codes) lengths count 32 bits per stored word, the bitstream
                            section holds the words (see fz_pipeline.encoder) */
#define FZ_ENC_HUFFMAN 0u
#define FZ_ENC_SHUFFLE 1u

typedef struct fz_ctx fz_ctx;

/* Create a context bound to CUDA device `device` (its workspace is allocated
 * lazily by the first call that needs it).  *out receives the handle. */
fz_status fz_ctx_create(int device, fz_ctx **out);

/* Free the context and its workspace.  Safe on NULL. */
fz_status fz_ctx_destroy(fz_ctx *ctx);

/* Bytes of output space fz_compress may need: 256 + 4N rounded up to 16.
 * Returns 0 for invalid dims. */
uint64_t fz_compress_bound(uint32_t ndim, const uint64_t dims[3]);

/* Compress the float32 field d_in into the stream d_out (FZMod-Default,
 * §3.3): REL range (§3.2) -> prequantization and Lorenzo prediction with
 * radius-R codes, anchors and outliers (§3.1) -> code histogram (§3.2) ->
 * canonical Huffman codebook -> chunked encode.  d_out must be 16-byte
 * aligned, must not overlap d_in, and out_cap must be >= 256 + 4N.  On
 * success *out_bytes (host) receives the stream length; if h_header is not
 * NULL the 256-byte header is also copied to it (host).  The call
 * synchronizes `stream`.  Errors: FZ_EINVAL, FZ_EBUFFER, FZ_EUNSUPPORTED,
 * FZ_ENOMEM, FZ_ECUDA, FZ_ETIMEOUT. */
fz_status fz_compress(fz_ctx *ctx, const float *d_in, uint32_t ndim, const uint64_t dims[3],
                      uint32_t eb_mode, double eb, const fz_pipeline *pipe, void *d_out,
                      uint64_t out_cap, uint64_t *out_bytes, void *h_header, void *stream);

/* Reconstruct the field from the stream d_in (in_bytes long, 16-byte
 * aligned) into d_out (out_cap_values floats, >= N): Huffman decode per
 * chunk, outlier scatter, anchor restore, inverse Lorenzo prefix sums,
 * dequantization, exception overwrite, all in one fused kernel (§3.3.1).
 * h_header may point to a host copy of the stream's first 256 bytes (saves
 * one device-to-host copy); NULL makes the call read it from d_in.  The call
 * synchronizes `stream`.  Errors: FZ_EINVAL, FZ_EBUFFER, FZ_ECORRUPT,
 * FZ_EUNSUPPORTED, FZ_ENOMEM, FZ_ECUDA. */
fz_status fz_decompress(fz_ctx *ctx, const void *d_in, uint64_t in_bytes, const void *h_header,
                        float *d_out, uint64_t out_cap_values, void *stream);

/* Parse a host copy of a stream header: dimensionality, dims, absolute
 * bound and flags.  Any output pointer may be NULL.  FZ_ECORRUPT on a bad
 * header. */
fz_status fz_stream_info(const void *h_header, uint64_t header_bytes, uint32_t *ndim, uint64_t dims[3],
                         double *eb_abs, uint32_t *flags);

/* Validate a host copy of a stream header (at least 256 bytes) against a
 * stream of stream_bytes bytes without touching the device: magic, version,
 * dims, flags, radius, predictor, block shape and chunk size, and that
 * every section lies 16-byte aligned, in order and entirely inside the
 * stream (no offset or length may reach past stream_bytes, whatever its
 * value).  fz_decompress, fz_decompress_noalloc and fz_decompress_batch run
 * the same check before any launch.  The paper defines no stream format;
 * this is the library's own.  Returns FZ_OK, FZ_ECORRUPT,
 * FZ_EUNSUPPORTED (flags of a later format) or FZ_EINVAL (null pointer or
 * stream_bytes < 256). */
fz_status fz_stream_check(const void *h_header, uint64_t stream_bytes);

/* Stage entry point (prediction + quantization module, §3.1-§3.2): runs the
 * REL range and constants, prequantization, Lorenzo prediction and code
 * histogram on d_in and writes the block-major code stream d_codes
 * (u16[n_blocks*block_size]), the anchors d_anchors (i32[n_blocks]) and the
 * histogram d_hist (u64[2R]); *n_out and *n_exc (host) receive the outlier
 * and exception counts and *eb_abs the absolute bound.  Synchronizes
 * `stream`. */
fz_status fz_lorenzo_quantize(fz_ctx *ctx, const float *d_in, uint32_t ndim, const uint64_t dims[3],
                              uint32_t eb_mode, double eb, const fz_pipeline *pipe, uint16_t *d_codes,
                              int32_t *d_anchors, uint64_t *d_hist, uint64_t *n_out, uint64_t *n_exc,
                              double *eb_abs, void *stream);

/* Stage entry point (Huffman codebook module, §3.2): from the histogram
 * d_hist (u64[nsym], nsym <= 1024, at least one nonzero count) compute the
 * code lengths d_lens (u8[nsym]: the optimal prefix code with lengths <= 14
 * found by package-merge, leaves ordered by (count, symbol), a leaf before a
 * package of equal weight; a single used symbol gets length 1) and the
 * canonical codewords d_codes (u32[nsym], RFC 1951 order).  Synchronizes
 * `stream`; FZ_EINVAL if no count is nonzero. */
fz_status fz_huffman_codebook(fz_ctx *ctx, const uint64_t *d_hist, uint32_t nsym, uint8_t *d_lens,
                              uint32_t *d_codes, void *stream);

/* ---- per-block predictor selection (3D): FZ_PRED_INTERP_*, FZ_SEL_* ----
 * The auto-selection of modules named as future work in FZModules §5 and the
 * dynamic module selection of §3.3.1.  Four predictors per 8x8x8 block:
 * 0 Lorenzo-1, 1 Lorenzo-2, 2 interpolation linear, 3 interpolation cubic
 * (levels 4, 2, 1 over the block with the corner anchors o + {0,8}^3).
 * FZ_SEL_EXHAUSTIVE picks per block the predictor with the smallest trial
 * cost (sum over the block of 1 + 2 floor(log2(|d|+1)) bits for codes, 96
 * for outliers); FZ_SEL_MLP picks the argmax of a 32 -> 64 (ReLU) -> 4
 * network over 32 block statistics (log2fix, bfloat16), with bfloat16
 * weights given as fz_pipeline.selector_weights: a device array of
 * FZ_SELECTOR_WEIGHTS uint16 bfloat16 values in the order W1[64][32], b1[64],
 * W2[4][64], b2[4].  Streams then carry a 2-bit id per block. */
#define FZ_SELECTOR_WEIGHTS 2372
#define FZ_SELECTOR_FEATURES 32

/* Stage entry point (label generation for the selector): for every block
 * of the 3D field d_in, the exhaustive-trial label d_labels (u8[n_blocks]),
 * optionally the four trial costs d_costs (u32[n_blocks][4]) and the 32
 * bfloat16 features d_features (u16[n_blocks][32]).  eb_mode/eb/radius as
 * for fz_compress.  Synchronizes `stream`; FZ_EUNSUPPORTED for a constant
 * field. */
fz_status fz_block_report(fz_ctx *ctx, const float *d_in, const uint64_t dims[3], uint32_t eb_mode, double eb,
                          uint32_t radius, uint8_t *d_labels, uint32_t *d_costs, uint16_t *d_features,
                          void *stream);

/* Selector training, gradient: mean softmax cross-entropy of n samples
 * (features u16[n][32] bfloat16, labels u8[n]) under the bfloat16 rounding
 * of the float32 master weights d_weights (FZ_SELECTOR_WEIGHTS values);
 * writes the gradient with respect to the master weights to d_grad
 * (float32, same layout) and, if h_loss is not NULL, the loss (host; the
 * call then synchronizes `stream`).  Deterministic (fixed reduction order). */
fz_status fz_mlp_grad(fz_ctx *ctx, const float *d_weights, const uint16_t *d_features, const uint8_t *d_labels,
                      uint32_t n, float *d_grad, float *h_loss, void *stream);

/* Selector training, Adam step number `step` (from 1) on the float32 master
 * weights with moment buffers d_m, d_v; also writes their bfloat16 copy to
 * d_weights_bf16 when it is not NULL.  Does not synchronize. */
fz_status fz_mlp_adam(fz_ctx *ctx, float *d_weights, const float *d_grad, float *d_m, float *d_v, uint32_t step,
                      float lr, float beta1, float beta2, float eps, uint16_t *d_weights_bf16, void *stream);

/* Per-stage timing of the last fz_compress and fz_decompress on a context.
 * When profiling is enabled, each call records a CUDA event on its stream
 * before the first and after every stage launch; a stage time is the
 * elapsed time between consecutive events.  `launches` counts the kernel
 * launches the context has issued since it was created (always counted);
 * `batch_plans` and `batch_graphs` count the cached batch plans and those of
 * them that run as an instantiated CUDA graph. */
#define FZ_MAX_STAGES 12
typedef struct {
  uint32_t n_compress, n_decompress;      /* stages recorded for the last call of each kind */
  char compress_names[FZ_MAX_STAGES][16];
  float compress_ms[FZ_MAX_STAGES];
  char decompress_names[FZ_MAX_STAGES][16];
  float decompress_ms[FZ_MAX_STAGES];
  uint64_t launches;
  uint32_t batch_plans, batch_graphs;
  int32_t batch_tune[4];                  /* launch shape of the newest batch plan: range segment log2,
                                             quantizer / encoder / decoder CTAs per SM (0 = occupancy limit) */
  uint32_t batch_chunk[2];                /* Huffman chunk of the newest batch compress plan: 3D fields,
                                             1D and 2D fields (0 = no field of that kind) */
} fz_profile;

/* Turn stage timing on (enable != 0) or off.  Host-only bookkeeping; the
 * events are created on the context's device. */
fz_status fz_ctx_set_profiling(fz_ctx *ctx, int enable);

/* Copy the stage times of the last calls into *out (synchronizes on the
 * recorded events). */
fz_status fz_ctx_get_profile(fz_ctx *ctx, fz_profile *out);

/* Bound of every device-side wait of the context's calls (the decoupled
 * look-back of the encoder and of the decoder's offset pass), in SM clock
 * cycles; 0 restores the default of 4e9 (about two seconds).  A wait that
 * runs out records FZ_ETIMEOUT, which the call returns, and the kernel
 * finishes normally, so the context stays usable.  The look-backs resolve
 * tiles in the order of a ticket counter, so their waits end by
 * construction; the bound guards against a corrupted device state.  The
 * paper describes no device-side waits; this is a library setting.
 * FZ_EINVAL for a negative value. */
fz_status fz_ctx_set_spin_limit(fz_ctx *ctx, long long cycles);

/* Self-test of the bounded wait: one warp runs the library's look-back on a
 * predecessor status word that nothing ever writes, under the context's
 * spin limit.  Returns FZ_ETIMEOUT when the wait gave up as designed and
 * the device is still usable; FZ_OK would mean the wait ended without its
 * predecessor (a defect).  Synchronizes `stream`.  No counterpart in the
 * paper. */
fz_status fz_selftest_bounded_wait(fz_ctx *ctx, void *stream);

/* ---- histogram module (§3.2) as a stage of its own ----
 * Counts of the n codes d_codes (u16, 16-byte aligned, every code < nsym,
 * nsym <= 1024) into d_hist (u64[nsym], device), by one of two methods that
 * give the same exact counts: FZ_HIST_PRIVATE (warp-private shared-memory
 * histograms) or FZ_HIST_TOPK, the top-k variant §3.2 describes as the better
 * one when the codes repeat a few values: the 4 most frequent codes of a
 * sample (64 windows of 1024 codes spread over the array) are counted by
 * packed 16-bit comparisons into per-thread registers and only the others
 * take shared-memory atomics.  (The compression path counts its codes
 * inside the quantizer; this entry point serves a code array on its own, such
 * as the output of fz_lorenzo_quantize.)  Uses the context workspace;
 * synchronizes `stream`.  FZ_EINVAL for bad arguments or a code >= nsym. */
#define FZ_HIST_PRIVATE 0u
#define FZ_HIST_TOPK 1u
fz_status fz_histogram(fz_ctx *ctx, const uint16_t *d_codes, uint64_t n, uint32_t nsym, uint32_t method,
                       uint64_t *d_hist, void *stream);

/* ---- reconstruction quality (rate-distortion evaluation, §4.2) ----
 * Statistics of a reconstruction d_y against its original d_x (n float32
 * values each, device): over the finite originals the largest |y - x| and the
 * sum of squared errors (double accumulation, deterministic order), the
 * value range, their count, and the number of non-finite originals whose
 * reconstruction does not carry the same bits; psnr_db = 20 log10(range) -
 * 10 log10(sse / n_finite) (infinite for an exact reconstruction).  The
 * paper's rate-distortion figure plots this PSNR against the bit rate
 * (stream bits per value).  Uses the context workspace; synchronizes
 * `stream`.  FZ_EINVAL for n = 0 or unaligned pointers. */
typedef struct {
  double max_abs_err, sse, x_min, x_max, psnr_db;
  uint64_t n_finite, n_nonfinite_mismatch;
} fz_error_report;
fz_status fz_error_stats(fz_ctx *ctx, const float *d_x, const float *d_y, uint64_t n, fz_error_report *out,
                         void *stream);

/* Human-readable name of a status code (static string). */
const char *fz_status_str(fz_status s);

/* ---- batched calls: many fields of uneven size in one pass ----
 * The paper composes its pipelines from modules launched one field at a
 * time (§3.3); these two calls are this library's batching of the same path.
 * Each stage runs as one persistent kernel over a work queue spanning every
 * field of the batch; the whole sequence is captured as a CUDA graph the
 * first time a batch shape (count, dims, mode, radius, predictor, output
 * buffer) is seen -- after an autotuner has timed candidate launch shapes --
 * and replayed by later calls of the same shape.  Launch shapes never change
 * the bytes: stream j is byte-identical to fz_compress of field j alone.
 * Only Lorenzo predictors (FZ_PRED_LORENZO1/2) are batched; others give
 * FZ_EUNSUPPORTED. */

/* Worst-case packed output of a batch: the sum over fields of
 * fz_compress_bound rounded up to 16 bytes.  dims holds 3 values per field
 * (unused trailing dims ignored).  0 on invalid dims. */
uint64_t fz_compress_batch_bound(uint32_t n, const uint32_t *ndim, const uint64_t *dims);

/* Compress n fields (1 <= n <= 65535).  d_in: host array of n device
 * pointers (float32, 4-byte aligned); ndim: n values; dims: 3n values; eb:
 * n error bounds (all in mode eb_mode).  pipe->chunk: 0 lets the autotuner
 * pick the Huffman chunk of each kind of field (3D; 1D and 2D) among the
 * block size and its double and quadruple -- the round trip (compress then
 * decompress) of the batch is timed for each, starting from the largest
 * chunk (the shortest stream), and a smaller chunk is kept only when it is
 * at least 3% faster; the tuning pass decompresses into temporary device
 * memory the size of the batch's input, freed before the call returns.
 * Without tuning (fz_ctx_set_batch_options) chunk 0 means the block size.
 * A nonzero chunk applies to every field and must be a supported chunk of
 * at least the block size (64-symbol chunks are not batched).  The streams are packed into d_out
 * (device, 16-byte aligned, out_cap bytes), stream j starting at
 * h_offsets[j] (a multiple of 16) and its length in its header
 * (total_bytes); h_offsets[n] is the packed size (host array of n+1
 * values).  FZ_EBUFFER if the packed streams do not fit out_cap (contents
 * then unspecified).  Synchronizes `stream`.  The first call with a new
 * batch shape runs the autotuner (a few extra passes over the batch). */
fz_status fz_compress_batch(fz_ctx *ctx, uint32_t n, const float *const *d_in, const uint32_t *ndim,
                            const uint64_t *dims, uint32_t eb_mode, const double *eb, const fz_pipeline *pipe,
                            void *d_out, uint64_t out_cap, uint64_t *h_offsets, void *stream);

/* Reconstruct n streams packed in d_in (device, 16-byte aligned) at the
 * host offsets h_offsets[0..n] (stream j occupies [h_offsets[j],
 * h_offsets[j+1]), as fz_compress_batch lays them out) into the n device
 * arrays d_out[j] (host array of device pointers); out_cap_values (host, n
 * values, may be NULL) bounds each output.  Reads the n headers to the host
 * first.  Synchronizes `stream`. */
fz_status fz_decompress_batch(fz_ctx *ctx, uint32_t n, const void *d_in, const uint64_t *h_offsets,
                              float *const *d_out, const uint64_t *out_cap_values, void *stream);

/* ---- decompression that allocates nothing ----
 * The paper has no counterpart; this is a library convenience.  For callers
 * that must not allocate: code running while another component owns the
 * device's memory budget, or latency-critical paths where the implicit
 * synchronization of cudaMalloc/cudaFree is not acceptable.  Same result as
 * fz_decompress, bit for bit, but without a context: the scratch (error
 * word, work-unit counter, per-unit bit offsets) is one fixed array in the
 * library's device image, shared by every call on a device,
 * and the call makes no cudaMalloc, cudaFree, cudaMallocHost or other
 * allocating call.  Limits: Lorenzo streams of at most FZ_NOALLOC_MAX_CHUNKS
 * chunks (FZ_EBUFFER beyond; 3D blocks of 8^3 = 33.5M values, 1D/2D blocks
 * of 1024 = 67M values), plus RAW and CONST streams of any size;
 * per-block-selection streams give FZ_EUNSUPPORTED.  Runs on the calling
 * thread's current device.  Calls whose device work overlaps (different
 * streams or host threads) race on the shared array and must be ordered by
 * the caller.  Every call looks up the array's address on the current
 * device (cudaGetSymbolAddress, which allocates nothing), so calls remain
 * valid after the device's context is recreated.  Synchronizes `stream`. */
#define FZ_NOALLOC_MAX_CHUNKS 65536
fz_status fz_decompress_noalloc(const void *d_in, uint64_t in_bytes, const void *h_header, float *d_out,
                                uint64_t out_cap_values, void *stream);

/* Batched-call options: autotune (default 1) times candidate launch shapes
 * on the first call with a new batch shape; graphs (default 1) captures and
 * replays the batch sequence as a CUDA graph (0 runs it eagerly every call).
 * Clears the cached plans. */
fz_status fz_ctx_set_batch_options(fz_ctx *ctx, int autotune, int graphs);

#ifdef __cplusplus
}
#endif

#endif /* FZ_H */
