// fz_internal.cuh -- device-side data structures shared by the kernels of
// libfz.so: the per-call control block, the workspace layout, block/tile
// geometry, bounded decoupled look-back and small device helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/fz.h"

namespace fz {

constexpr int kMaxSym = 1024;      // 2R <= 1024 (R <= 512)
constexpr int kLmax = 14;          // longest Huffman codeword (length limit of the format)
constexpr int kLutBits = 14;       // decode table width: every codeword resolves in one lookup
constexpr int kTileElems = 4096;   // elements per quantization tile
constexpr int kQuantThreads = 256; // 8 warps per quantization tile
constexpr int kEncWarps = 8;       // chunks per encode tile (one warp per chunk)
constexpr int kDecUnit = 32;       // chunks per decode work unit (one warp, one chunk per lane)
constexpr int kDecCtlWords = 8;    // decoder control words ahead of the unit-offset pass's look-back words
constexpr int kTileGroup = 1024;   // quantization tiles per outlier-offset group

enum Mode : uint32_t { kModeNormal = 0, kModeConst = 1, kModeRaw = 2 };

// Block geometry: block shape per dimensionality (1D 1024, 2D 32x32,
// 3D 8x8x8) and the field extents, x fastest.
struct Geom {
  uint32_t ndim;
  uint32_t nx, ny, nz;     // extents (unused axes 1)
  uint32_t bx, by, bz;     // block extents
  uint32_t nbx, nby, nbz;  // blocks per axis
  uint32_t bsize;          // elements per block
  uint64_t n;              // nx*ny*nz
  uint64_t n_blocks;
  uint64_t npad;           // n_blocks * bsize
  // quantization tiles: NB consecutive blocks along x
  uint32_t tile_nb;        // blocks per tile along x
  uint32_t tiles_x;        // tiles per block-row
  uint64_t n_qtiles;
  // Huffman chunks: chunk j covers code-stream symbols [j chunk, (j+1) chunk)
  uint32_t chunk;          // symbols per chunk (default: bsize)
  uint64_t n_chunks;       // ceil(npad / chunk)
};

// ---- programmatic dependent launch between the stages of one call
// A stage launched with launch_dep may start while the previous kernel of the
// stream runs; before it reads anything an earlier stage wrote it calls
// dep_wait(), which returns once the previous kernel has completed and its
// writes are visible (an earlier kernel of the stream completed before that
// one passed its own wait).  Work before dep_wait() touches only the call's
// inputs.  dep_trigger(), called after the kernel's own wait, lets the next
// stage start.  Both are no-ops in kernels launched the ordinary way.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void dep_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Code-stream positions (block-major, padding included) are 32-bit in the
// stream format (outlier and exception indices) and in the kernels.
inline __host__ __device__ bool positions_fit(const Geom &g) { return g.npad <= 0xffffffffull; }

inline __host__ __device__ void make_geom(uint32_t ndim, const uint64_t dims[3], Geom &g) {
  g.ndim = ndim;
  g.nx = (uint32_t)dims[0];
  g.ny = ndim >= 2 ? (uint32_t)dims[1] : 1u;
  g.nz = ndim >= 3 ? (uint32_t)dims[2] : 1u;
  if (ndim == 1) { g.bx = 1024; g.by = 1; g.bz = 1; g.tile_nb = 4; }
  else if (ndim == 2) { g.bx = 32; g.by = 32; g.bz = 1; g.tile_nb = 4; }
  else { g.bx = 8; g.by = 8; g.bz = 8; g.tile_nb = 8; }
  g.nbx = (g.nx + g.bx - 1) / g.bx;
  g.nby = (g.ny + g.by - 1) / g.by;
  g.nbz = (g.nz + g.bz - 1) / g.bz;
  g.bsize = g.bx * g.by * g.bz;
  g.n = (uint64_t)g.nx * g.ny * g.nz;
  g.n_blocks = (uint64_t)g.nbx * g.nby * g.nbz;
  g.npad = g.n_blocks * g.bsize;
  g.tiles_x = (g.nbx + g.tile_nb - 1) / g.tile_nb;
  g.n_qtiles = (uint64_t)g.tiles_x * g.nby * g.nbz;
  g.chunk = g.bsize;
  g.n_chunks = g.n_blocks;
}

// Huffman chunk sizes of the format: the block size, a power-of-two
// multiple of it up to 4096, for 3D blocks 64 (one 8x8 plane), or, for 2D
// first-order Lorenzo streams, 128, 256 or 512 (4, 8 or 16 rows of a 32x32
// block).  Only first- and second-order Lorenzo streams use a chunk other
// than the block.
inline __host__ __device__ bool chunk_supported(uint32_t ndim, uint32_t bsize, uint32_t C, uint32_t pred) {
  if (C == bsize) return true;
  if (ndim == 3 && C == 64) return true;
  if (ndim == 2 && pred == FZ_PRED_LORENZO1 && (C == 128 || C == 256 || C == 512)) return true;
  return C > bsize && C <= 4096 && C % bsize == 0 && (C & (C - 1)) == 0;
}

inline __host__ __device__ void set_chunk(Geom &g, uint32_t C) {
  g.chunk = C;
  g.n_chunks = (g.npad + C - 1) / C;
}

// Launch shape of one kernel, computed on its first launch on each device:
// the kernel's dynamic shared memory limit raised to the launch's size and
// its resident CTAs per SM, so that later launches make no attribute or
// occupancy query.
constexpr int kMaxLaunchDevices = 64;
struct LaunchCache {
  std::atomic<int> per_sm[kMaxLaunchDevices];
};
template <typename Kernel>
cudaError_t cached_per_sm(Kernel kernel, int threads, int smem, LaunchCache &c, int &per_sm) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cacheable = dev >= 0 && dev < kMaxLaunchDevices;
  if (cacheable) {
    const int v = c.per_sm[dev].load(std::memory_order_relaxed);
    if (v > 0) {
      per_sm = v;
      return cudaSuccess;
    }
  }
  if (smem > 0) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  int v = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  if (v < 1) v = 1;
  if (cacheable) c.per_sm[dev].store(v, std::memory_order_relaxed);
  per_sm = v;
  return cudaSuccess;
}

// Per-call control block.  Zeroed by one memset at the start of each
// compress; every field is designed so that zero is the right initial value.
struct Result {
  uint64_t total_bytes;
  uint32_t err;            // first fz_status reported by a kernel (0 = none)
  uint32_t mode;
  uint64_t n_out, n_exc;
  fz_header hdr;           // the stream header as written
};

struct Ctl {
  unsigned long long hist[kMaxSym];
  // REL range: max of inverted ordered keys for the minimum, max of ordered
  // keys for the maximum, and the same on raw bit patterns.
  unsigned int lo_nkey, hi_key, bits_nmin, bits_max, any_finite, range_done;
  unsigned int encode_ticket, n_otiles;  // encoder tickets; quantization tiles holding outliers/exceptions
  unsigned long long n_out, n_exc;   // totals; also the append cursors of the scratch lists
  // constants (written by the range tail or the ABS constants kernel)
  double eb_abs;
  float ebx2, inv2eb, eb_chk;
  uint32_t mode;           // Mode after the range stage
  uint32_t const_bits;
  uint32_t pad0;
  // codebook results
  uint32_t enc[kMaxSym];   // codeword left-aligned in the high len bits, len in the low 5 (0: unused)
  uint8_t lens[kMaxSym];
  uint64_t total_bits;
  Result res;
};

// The header of a RAW or CONST stream (and the start of every header): only
// magic, version, flags, ndim, eb_mode, dims, eb and total_bytes are set.
__device__ __forceinline__ void write_min_header(fz_header &h, uint16_t flags, const Geom &g, uint32_t eb_mode,
                                                 double eb, uint64_t total) {
  uint8_t *p = reinterpret_cast<uint8_t *>(&h);
  for (int i = 0; i < (int)sizeof(fz_header); ++i) p[i] = 0;
  h.magic = FZ_MAGIC;
  h.version = 1;
  h.flags = flags;
  h.ndim = g.ndim;
  h.eb_mode = eb_mode;
  h.dims[0] = g.nx; h.dims[1] = g.ny; h.dims[2] = g.nz;
  h.eb = eb;
  h.total_bytes = total;
}

// ---------------------------------------------------------------- errors
__device__ __forceinline__ void set_err(Ctl *ctl, uint32_t code) { atomicCAS(&ctl->res.err, 0u, code); }

// ---------------------------------------------------------------- ordered float keys
// Monotone map from float bit patterns to unsigned keys (for atomic min/max).
__device__ __forceinline__ uint32_t fkey(float f) {
  uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(u);
}

// ---------------------------------------------------------------- constants
// eb_abs -> bin width ebx2 (rounded down), its reciprocal (nearest), and the
// per-value check bound (rounded down); each step one IEEE operation.
__device__ __forceinline__ void device_constants(double eb_abs, float &ebx2, float &inv2eb, float &eb_chk) {
  double w = __dmul_rn(2.0, eb_abs);
  w = __dmul_rn(w, 1.0 - 0x1p-12);
  ebx2 = __double2float_rd(w);
  double inv = __ddiv_rn(1.0, (double)ebx2);
  inv2eb = __double2float_rn(inv);
  double c = __dmul_rn(eb_abs, 1.0 - 0x1p-23);
  eb_chk = __double2float_rd(c);
}

// ---------------------------------------------------------------- bounded decoupled look-back
// Status word per tile: bits 63..62 = 1 (aggregate) or 2 (inclusive prefix),
// low 62 bits = value.  Tiles are numbered in the order they are claimed from
// a ticket counter, so every predecessor is resident or finished and the wait
// always ends; the clock bound (kSpinCycles unless the context sets another)
// only guards against a corrupted state, and turns it into FZ_ETIMEOUT.
constexpr uint64_t kLbFlagAgg = 1ull << 62;
constexpr uint64_t kLbFlagInc = 2ull << 62;
constexpr uint64_t kLbMask = (1ull << 62) - 1;
constexpr long long kSpinCycles = 4000000000ll;  // about two seconds at 2 GHz

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t *p) {
  return *(const volatile uint64_t *)p;
}
__device__ __forceinline__ void st_status(uint64_t *p, uint64_t v) {
  atomicExch((unsigned long long *)p, (unsigned long long)v);
}

// Combine two packed values.  `packed2` packs two 31-bit saturating counters.
template <bool kPacked2>
__device__ __forceinline__ uint64_t lb_add(uint64_t a, uint64_t b) {
  if (!kPacked2) return (a + b) & kLbMask;
  const uint64_t m = (1ull << 31) - 1;
  uint64_t lo = (a & m) + (b & m), hi = ((a >> 31) & m) + ((b >> 31) & m);
  lo = lo > m ? m : lo;
  hi = hi > m ? m : hi;
  return lo | (hi << 31);
}

// Publishes the tile's aggregate (tile 0 publishes its inclusive prefix).
__device__ __forceinline__ void lookback_publish(uint64_t *status, uint64_t tile, uint64_t agg) {
  st_status(&status[tile], (tile == 0 ? kLbFlagInc : kLbFlagAgg) | agg);
}

// After lookback_publish: walks back to the nearest inclusive prefix, then
// publishes this tile's inclusive prefix.  Called by one thread of the tile;
// returns the exclusive prefix.
template <bool kPacked2>
__device__ uint64_t lookback_resolve(uint64_t *status, uint64_t tile, uint64_t agg, Ctl *ctl) {
  if (tile == 0) return 0;
  uint64_t excl = 0;
  int64_t j = (int64_t)tile - 1;
  long long t0 = clock64();
  while (j >= 0) {
    uint64_t v = ld_volatile_u64(&status[j]);
    if ((v >> 62) == 0) {
      if (clock64() - t0 > kSpinCycles) {
        set_err(ctl, FZ_ETIMEOUT);
        break;
      }
      __nanosleep(32);
      continue;
    }
    excl = lb_add<kPacked2>(excl, v & kLbMask);
    if ((v >> 62) == 2) break;
    j--;
  }
  st_status(&status[tile], kLbFlagInc | lb_add<kPacked2>(excl, agg));
  return excl;
}

// Warp-cooperative variant of lookback_resolve (non-packed values): the 32
// lanes read 32 predecessors at once, so the walk back costs one round of
// loads per 32 tiles.  All lanes of the warp must call it; returns the
// exclusive prefix in every lane.
__device__ __forceinline__ uint64_t lookback_resolve_warp(uint64_t *status, uint64_t tile, uint64_t agg,
                                                          uint32_t *err, long long spin = 0) {
  const int lane = threadIdx.x & 31;
  if (spin <= 0) spin = kSpinCycles;
  if (tile == 0) return 0;
  uint64_t excl = 0;
  int64_t hi = (int64_t)tile - 1;  // highest predecessor not yet summed
  long long t0 = clock64();
  bool timed_out = false;
  while (hi >= 0) {
    const int64_t j = hi - lane;
    uint64_t v = j >= 0 ? ld_volatile_u64(&status[j]) : (kLbFlagInc | 0ull);
    uint32_t flag = (uint32_t)(v >> 62);
    // the nearest inclusive prefix in the window (lowest lane index with flag 2)
    const uint32_t inc_mask = __ballot_sync(0xffffffffu, flag == 2);
    const int stop = inc_mask ? __ffs(inc_mask) - 1 : 31;
    const uint32_t missing = __ballot_sync(0xffffffffu, flag == 0 && lane <= stop);
    if (missing) {
      if (clock64() - t0 > spin) { timed_out = true; break; }
      __nanosleep(32);
      continue;
    }
    uint64_t part = lane <= stop ? (v & kLbMask) : 0ull;
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    part = __shfl_sync(0xffffffffu, part, 0);
    excl = (excl + part) & kLbMask;
    if (inc_mask) break;
    hi -= 32;
  }
  if (timed_out && lane == 0) atomicCAS(err, 0u, (uint32_t)FZ_ETIMEOUT);
  if (lane == 0) st_status(&status[tile], kLbFlagInc | ((excl + agg) & kLbMask));
  return excl;
}

template <bool kPacked2>
__device__ __forceinline__ uint64_t lookback(uint64_t *status, uint64_t tile, uint64_t agg, Ctl *ctl) {
  lookback_publish(status, tile, agg);
  return lookback_resolve<kPacked2>(status, tile, agg, ctl);
}

inline __host__ __device__ uint64_t align16(uint64_t v) { return (v + 15u) & ~(uint64_t)15u; }

// q = rint(x * inv2eb) (binary32, half to even); an exception when |t| is
// not below 2^23 (this also catches NaN and infinities, q forced to 0) or
// when q * ebx2 misses x by more than eb_chk (q kept).
__device__ __forceinline__ int32_t prequant(float x, float inv2eb, float ebx2, float eb_chk, bool &exc) {
  const float t = __fmul_rn(x, inv2eb);
  const bool ok = fabsf(t) < 8388608.0f;
  const int32_t q = ok ? __float2int_rn(t) : 0;
  const float r = __fmul_rn(__int2float_rn(q), ebx2);
  const float d = fabsf(__fsub_rn(x, r));
  exc = !ok || d > eb_chk;
  return q;
}

// prequant() without the float<->int conversion instructions, for
// |x * inv2eb| < 2^22: t + 1.5*2^23 then lies in [2^23, 2^24), where the
// floats are exactly the integers, so the rounded sum is rint(t) (ties to
// even, like cvt.rni) and its mantissa holds rint(t) + 2^22.  Sets slow
// (and returns garbage) outside that range, NaN included; the caller then
// takes prequant().  Same q and exception flag as prequant() otherwise.
__device__ __forceinline__ int32_t prequant_fast(float x, float inv2eb, float ebx2, float eb_chk, bool &exc,
                                                 bool &slow) {
  constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23, bit pattern 0x4B400000
  const float t = __fmul_rn(x, inv2eb);
  slow = !(fabsf(t) < 4194304.0f);
  const float s = __fadd_rn(t, kMagic);
  const float r = __fmul_rn(__fsub_rn(s, kMagic), ebx2);
  exc = fabsf(__fsub_rn(x, r)) > eb_chk;
  return __float_as_int(s) - 0x4B400000;
}

// Selector network shape: 32 block features -> 64 hidden (ReLU) -> 4
// predictor logits.  Parameter order in every weight array: W1[64][32],
// b1[64], W2[4][64], b2[4].
constexpr int kNFeat = 32, kNHid = 64, kNPred = 4;
constexpr int kOffW1 = 0, kOffB1 = kNHid * kNFeat, kOffW2 = kOffB1 + kNHid, kOffB2 = kOffW2 + kNPred * kNHid;
constexpr int kNWeights = kOffB2 + kNPred;  // 2372

__device__ __forceinline__ uint16_t f32_to_bf16_rne(float f) {
  uint32_t u = __float_as_uint(f);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
__device__ __forceinline__ float bf16_to_f32(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// Outliers and exceptions one warp of a quantization tile appended to the
// scratch lists: the first slots and the counts per slice.  The 3D Lorenzo
// quantizer's warp holds one z-plane of the tile's 8 blocks: 8 slices (one
// per block, a count per byte).  Otherwise the warp's positions form one
// slice (count in the low 16 bits).  Slices go to the stream in code order:
// 3D Lorenzo by block then warp, otherwise by warp.
struct WarpSlots {
  uint32_t oslot, eslot;
  unsigned long long ocnt, ecnt;
};

// ---------------------------------------------------------------- workspace layout
// Device scratch owned by the context for one compress call.
struct CompressWs {
  Ctl *ctl;
  uint4 *tinfo;            // per quantization tile: n_out, n_exc, first outlier slot, first exception slot
  uint2 *tgroup;           // per group of kTileGroup tiles: outlier and exception counts
  uint2 *tdst;             // per quantization tile: its first outlier and exception slot in the stream
  struct WarpSlots *winfo; // per quantization tile and warp: where its outliers/exceptions went (8 per tile)
  uint32_t *otiles;        // the tiles that hold outliers or exceptions (Ctl::n_otiles of them), any order
  uint64_t *estatus;       // look-back status per encode tile
  size_t zero_bytes;       // bytes from ctl to the end of estatus (memset per call)
  uint16_t *codes;         // npad block-major codes
  int32_t *anchors;        // n_blocks
  uint32_t *out_idx;       // cap_list entries, grouped by tile (tile order given by tinfo)
  int32_t *out_val;
  uint32_t *exc_idx;
  uint32_t *exc_val;
  uint64_t cap_list;       // floor(N/8)
  uint8_t *ids;            // per block: predictor id (per-block selection only)
  Result *h_res;           // host-mapped copy of ctl->res written by the last compress kernel (or null)
  long long spin = 0;      // look-back wait bound in clock cycles (0: kSpinCycles)
};

// ---------------------------------------------------------------- batched calls
// One field of a batched compress.  The host fills everything except
// out_off, which k_batch_offsets writes once every stream size is known.
struct BatchJob {
  const float *x;
  Geom g;
  CompressWs ws;
  double eb;
  uint32_t eb_mode, R, pred, pad;
  uint64_t range_base, range_segs;  // the field's range segments in the batch-wide segment queue
  uint64_t qtile_base;              // first quantization tile in its quantizer class queue
  uint64_t etile_base;              // first encode tile in its chunk-size class queue
  uint64_t out_off;                 // byte offset of the field's stream in the packed output
};

// Batch-wide control words (zeroed with the fields' control blocks).
struct BatchCtl {
  uint32_t ticket[2];               // encode tickets of the two chunk-size classes (512, 1024)
  uint32_t err;
  uint32_t pad;
  uint64_t total_bytes;             // packed output bytes
};

constexpr uint64_t kNoOutput = ~0ull;  // out_off of every field when the packed output does not fit

// Launch shape of the batched kernels, chosen by the autotuner.
struct BatchTune {
  int range_seg_log2;   // elements per range segment = 2^range_seg_log2
  int quant_per_sm;     // quantizer CTAs per SM
  int encode_per_sm;    // encoder CTAs per SM
  int decode_per_sm;    // decoder CTAs per SM
  int chunk_log2[2];    // Huffman chunk = block size << chunk_log2, per encode class (3D; 1D and 2D)
};

}  // namespace fz

// Host-side launchers (defined in the .cu files).
namespace fz {
cudaError_t launch_range(const float *x, const Geom &g, uint32_t eb_mode, double eb, Ctl *ctl, cudaStream_t s);
cudaError_t launch_quant(const float *x, const Geom &g, uint32_t R, uint32_t pred, const CompressWs &ws,
                         cudaStream_t s, int sm_count);
cudaError_t launch_codebook(const Geom &g, uint32_t R, uint32_t pred, uint32_t eb_mode, double eb,
                            const CompressWs &ws, cudaStream_t s);
cudaError_t launch_encode(const Geom &g, const CompressWs &ws, uint8_t *d_out, cudaStream_t s, int sm_count);
cudaError_t launch_assemble(const float *x, const Geom &g, uint32_t R, const CompressWs &ws, uint8_t *d_out,
                            cudaStream_t s, int sm_count);
cudaError_t launch_codebook_only(const uint64_t *hist, uint32_t nsym, uint8_t *lens, uint32_t *codes,
                                 Ctl *ctl, cudaStream_t s);
// bit-shuffle + zero-word encoder (FZMod-Speed)
cudaError_t launch_shuf_layout(const Geom &g, uint32_t R, uint32_t pred, uint32_t eb_mode, double eb,
                               const CompressWs &ws, cudaStream_t s);
cudaError_t launch_shuf_encode(const Geom &g, const CompressWs &ws, uint8_t *d_out, cudaStream_t s, int sm_count);

struct DecodeWs {
  uint16_t *lut;           // 1 << kLutBits entries: codeword length, symbol
  uint64_t *gsum;          // per work unit of kDecUnit chunks: sum of chunk bits, then exclusive offset
  uint32_t *err;           // device error word; err[1] is the work-unit counter (both zeroed per call)
  uint32_t *ofirst = nullptr;  // per block: index of its first outlier (filled when outliers are many)
  uint32_t *h_err = nullptr;   // host-mapped word that receives the final error word (or null)
  long long spin = 0;          // look-back wait bound in clock cycles (0: kSpinCycles)
};

inline __host__ __device__ uint64_t dec_units_of(uint64_t n_chunks) { return (n_chunks + kDecUnit - 1) / kDecUnit; }
cudaError_t launch_decode_prep(const uint8_t *d_in, const fz_header &h, const DecodeWs &ws, cudaStream_t s);
cudaError_t launch_outlier_starts(const uint8_t *d_in, const fz_header &h, const DecodeWs &ws, cudaStream_t s,
                                  int sm_count);
// bytes from the error word that launch_decode_offsets needs zeroed (error
// word, work-unit counter, its look-back status words)
uint64_t dec_offset_zero_bytes(const fz_header &h);
// work-unit bit offsets only (the Lorenzo decoder builds its decode table itself)
cudaError_t launch_decode_offsets(const uint8_t *d_in, const fz_header &h, const DecodeWs &ws, cudaStream_t s);
cudaError_t launch_decode_main(const uint8_t *d_in, const fz_header &h, float *d_out, const DecodeWs &ws,
                               cudaStream_t s, int sm_count);
cudaError_t launch_fill(float *out, uint64_t n, uint32_t bits, cudaStream_t s, int sm_count);
cudaError_t launch_shuf_decode(const uint8_t *d_in, const fz_header &h, float *d_out, const DecodeWs &ws,
                               cudaStream_t s, int sm_count);
// one warp waits on a look-back predecessor that never publishes (scratch:
// err word at [0], status words from [4], 32 bytes zeroed by the caller)
cudaError_t launch_lookback_selftest(uint32_t *scratch, long long spin, cudaStream_t s);
cudaError_t launch_selquant(const float *x, const Geom &g, uint32_t R, uint32_t pred, const CompressWs &ws,
                            const uint16_t *weights, cudaStream_t s, int sm_count);
cudaError_t launch_select_report(const float *x, const Geom &g, uint32_t R, const CompressWs &ws, uint8_t *labels,
                                 uint32_t *costs, uint16_t *feat, cudaStream_t s, int sm_count);
cudaError_t launch_sel_decode(const uint8_t *d_in, const fz_header &h, float *d_out, const DecodeWs &ws,
                              uint16_t *codes, cudaStream_t s, int sm_count);
// the code stream of a stream with one chunk per block into `codes` (npad symbols); with `ovals`
// (npad entries) and ws.ofirst also every outlier's residual at its position, the list checked
cudaError_t launch_dec_codes(const uint8_t *d_in, const fz_header &h, const DecodeWs &ws, uint16_t *codes,
                             int32_t *ovals, cudaStream_t s, int sm_count);
// the exceptions of a stream over the reconstructed field (list checked: ascending, in the domain)
cudaError_t launch_exc_scatter(const uint8_t *d_in, const fz_header &h, float *d_out, uint32_t *err, uint32_t *h_err,
                               cudaStream_t s, int sm_count);
// full-field interpolation streams: values of the level-s grid (ceil(dims / s) points)
uint64_t ginterp_level_values(const fz_header &h, uint32_t s);
// codes, the level-4 grid into q4, the level-2 grid into q2, the field into d_out
cudaError_t launch_gi_decode(const uint8_t *d_in, const fz_header &h, float *d_out, const DecodeWs &ws,
                             uint16_t *codes, int32_t *ovals, int32_t *q4, int32_t *q2, cudaStream_t s, int sm_count);
cudaError_t launch_mlp_grad(const float *w, const uint16_t *feat, const uint8_t *labels, uint32_t n,
                            float *partial, float *grad, float *loss, cudaStream_t s);
cudaError_t launch_adam(float *w, const float *grad, float *m, float *v, uint16_t *w_bf16, uint32_t step, float lr,
                        float beta1, float beta2, float eps, cudaStream_t s);
size_t mlp_partial_floats(uint32_t n);

// batched compress stages (fields of one call described by a device table)
cudaError_t launch_range_batch(const BatchJob *jobs, uint32_t n, uint64_t total_segs, int seg_log2,
                               cudaStream_t s, int sm_count);
cudaError_t launch_quant_batch(int ndim, int k, const BatchJob *jobs, const uint32_t *members, uint32_t n_members,
                               uint64_t total_tiles, int per_sm, cudaStream_t s, int sm_count);
cudaError_t launch_codebook_batch(const BatchJob *jobs, uint32_t n, cudaStream_t s);
cudaError_t launch_batch_offsets(BatchJob *jobs, uint32_t n, uint64_t out_cap, BatchCtl *bctl, cudaStream_t s);
cudaError_t launch_encode_batch(int chunk, const BatchJob *jobs, const uint32_t *members, uint32_t n_members,
                                uint64_t total_tiles, uint32_t *ticket, uint8_t *d_out, int per_sm, cudaStream_t s,
                                int sm_count);
cudaError_t launch_assemble_batch(const BatchJob *jobs, uint32_t n, uint8_t *d_out, uint64_t max_n, cudaStream_t s,
                                  int sm_count);
// batched decompress (the job tables are opaque to the API layer)
size_t dec_job_bytes();
size_t plain_job_bytes();
uint64_t dec_units(const fz_header &h);
void fill_dec_job(void *dst, const uint8_t *d_in, const fz_header &h, float *d_out, uint16_t *lut, uint64_t *gsum,
                  uint32_t *err, uint64_t unit_base);
void fill_plain_job(void *dst, const uint8_t *d_in, uint64_t n, bool is_const, float *d_out);
cudaError_t launch_decode_batch_prep(const void *jobs, uint32_t n, uint64_t max_units, cudaStream_t s);
cudaError_t launch_decode_batch_main(int ndim, int k, const void *jobs, const uint32_t *members, uint32_t n_members,
                                     uint64_t total_units, int per_sm, cudaStream_t s, int sms);
cudaError_t launch_plain_batch(const void *jobs, uint32_t n, uint64_t max_n, cudaStream_t s, int sms);
cudaError_t launch_batch_results(const BatchJob *jobs, uint32_t n, const BatchCtl *bctl, Result *res,
                                 uint64_t *offsets, cudaStream_t s);
}  // namespace fz
