// fz_codebook.cu -- Huffman codebook module (FZModules §3.2: the Huffman
// encoder is fed by the histogram of quantization codes) and the stream
// layout decision.  One CTA of 1024 threads:
//   1. bitonic sort of (count, symbol) keys of the used symbols;
//   2. package-merge for the optimal code with lengths <= 14 (a Huffman code
//      whenever the unlimited one fits): 13 levels, each a parallel merge of
//      the sorted leaves with the packages of the level below;
//   3. selection of 2m-2 items and code lengths from the per-level counts;
//   4. canonical codewords in RFC 1951 order via warp ballots;
//   5. total bit count, section offsets, raw-fallback rule and the header.
#include "fz_internal.cuh"

namespace fz {

namespace {

constexpr int kCbThreads = 1024;

struct CbSmem {
  unsigned long long key[kMaxSym];
  unsigned long long cnt[kMaxSym];
  unsigned long long lw[kMaxSym];          // sorted leaf weights
  unsigned long long S[2][2 * kMaxSym];    // items of the current / next level
  unsigned long long pk[kMaxSym];          // packages of the current level
  uint8_t leaf[kLmax + 1][2 * kMaxSym];      // per level and merged item: 1 for a leaf, 0 for a package
  uint32_t a[kLmax + 1];                   // selected leaves per level
  uint16_t lsym[kMaxSym];                  // sorted leaf symbols
  uint8_t len[kMaxSym];
  uint32_t wcnt[32][kLmax + 1];
  uint32_t next_code[kLmax + 2];
  unsigned long long total_bits;
};

// Number of elements of the sorted array a[0..n) that are < v (strict) or
// <= v (!strict).
__device__ __forceinline__ uint32_t rank_of(const unsigned long long *a, uint32_t n, unsigned long long v,
                                            bool strict) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const bool before = strict ? (a[mid] < v) : (a[mid] <= v);
    if (before) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Code lengths (into s.len) and canonical codewords (into code[]) for the
// counts in s.cnt[0..nsym): the optimal prefix code with lengths <= 14
// (package-merge), leaves in (count, symbol) order, a leaf before a package
// of equal weight.  Each level's merge is parallel: every leaf and every
// package finds its merged position by binary search in the other list.
// Returns false if no symbol is used.
__device__ bool build_codebook(CbSmem &s, uint32_t nsym, uint32_t *code_out, uint32_t &my_code) {
  const int t = threadIdx.x, lane = t & 31;
  // ---- 1. sort keys (count << 10 | symbol); unused symbols sort last.
  // Bitonic network, one key per thread: partners closer than 32 are in the
  // same warp (shuffles); farther ones meet in shared memory, alternating
  // between two arrays so that each step needs one barrier.
  unsigned long long v = (t < (int)nsym && s.cnt[t]) ? ((s.cnt[t] << 10) | (unsigned long long)t) : ~0ull;
  s.len[t] = 0;
  int buf = 0;
  for (int k = 2; k <= kMaxSym; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      unsigned long long o;
      if (j >= 32) {
        s.S[buf][t] = v;
        __syncthreads();
        o = s.S[buf][t ^ j];
        buf ^= 1;
      } else {
        o = __shfl_xor_sync(0xffffffffu, v, j);
      }
      const bool keep_min = ((t & j) == 0) == ((t & k) == 0);
      v = keep_min ? (v < o ? v : o) : (v < o ? o : v);
    }
  }
  s.key[t] = v;
  __syncthreads();
  const uint32_t m = (uint32_t)__syncthreads_count(s.key[t] != ~0ull);
  if (m == 0) return false;
  if ((uint32_t)t < m) {
    s.lsym[t] = (uint16_t)(s.key[t] & 1023u);
    s.lw[t] = s.key[t] >> 10;
  }
  __syncthreads();
  if (m == 1) {
    if (t == 0) s.len[s.lsym[0]] = 1;
    __syncthreads();
  } else {
    // ---- 2. package-merge, level kLmax (leaves only) down to level 1
    // (the flags are plain byte stores: every merged position of a level is
    // written once, by its leaf or its package)
    for (int i = t; i < (kLmax + 1) * (2 * kMaxSym) / 4; i += kCbThreads)
      reinterpret_cast<uint32_t *>(&s.leaf[0][0])[i] = 0u;
    if ((uint32_t)t < m) s.S[0][t] = s.lw[t];
    __syncthreads();
    if ((uint32_t)t < m) s.leaf[kLmax][t] = 1;
    uint32_t n_cur = m;
    int cb = 0;
    for (int l = kLmax - 1; l >= 1; --l) {
      const uint32_t np = n_cur >> 1;
      if ((uint32_t)t < np) s.pk[t] = s.S[cb][2 * t] + s.S[cb][2 * t + 1];
      __syncthreads();
      if ((uint32_t)t < m) {
        const uint32_t pos = (uint32_t)t + rank_of(s.pk, np, s.lw[t], true);
        s.S[cb ^ 1][pos] = s.lw[t];
        s.leaf[l][pos] = 1;
      }
      if ((uint32_t)t < np) {
        const uint32_t pos = (uint32_t)t + rank_of(s.lw, m, s.pk[t], false);
        s.S[cb ^ 1][pos] = s.pk[t];
      }
      __syncthreads();
      n_cur = m + np;
      cb ^= 1;
    }
    // ---- 3. selection: 2m-2 items at level 1; a_l leaves per level, counted
    // by the whole CTA (thread t: items 2t and 2t + 1 of the level)
    {
      uint32_t sel = 2 * m - 2;
      for (int l = 1; l <= kLmax; ++l) {
        const uint32_t i0 = 2u * (uint32_t)t;
        const uint32_t c = (uint32_t)__syncthreads_count(i0 < sel && s.leaf[l][i0]) +
                           (uint32_t)__syncthreads_count(i0 + 1 < sel && s.leaf[l][i0 + 1]);
        if (t == 0) s.a[l] = c;
        sel = 2 * (sel - c);
      }
    }
    __syncthreads();
    if ((uint32_t)t < m) {
      uint32_t L = 0;
#pragma unroll
      for (int l = 1; l <= kLmax; ++l) L += (uint32_t)t < s.a[l];
      s.len[s.lsym[t]] = (uint8_t)L;
    }
    __syncthreads();
  }
  // ---- 4. canonical codewords (RFC 1951 order)
  const int warp = t >> 5;
  const int L = (t < (int)nsym) ? s.len[t] : 0;
  if (t < 32 * (kLmax + 1)) (&s.wcnt[0][0])[t] = 0;
  __syncthreads();
  uint32_t rank = 0;
#pragma unroll 1
  for (int l = 1; l <= kLmax; ++l) {
    uint32_t b = __ballot_sync(0xffffffffu, L == l);
    if (L == l) rank = __popc(b & ((1u << lane) - 1));
    if (lane == 0) s.wcnt[warp][l] = __popc(b);
  }
  __syncthreads();
  if (t >= 1 && t <= kLmax) {  // exclusive prefix over warps for length t
    uint32_t acc = 0;
    for (int w = 0; w < 32; ++w) { uint32_t v = s.wcnt[w][t]; s.wcnt[w][t] = acc; acc += v; }
    s.wcnt[0][0] = 0;
    // total per length stored in next_code temporarily via a second pass below
    s.next_code[t] = acc;
  }
  __syncthreads();
  if (t == 0) {
    uint32_t bl[kLmax + 1];
    bl[0] = 0;
    for (int l = 1; l <= kLmax; ++l) bl[l] = s.next_code[l];
    uint32_t c = 0;
    for (int l = 1; l <= kLmax; ++l) {
      c = (c + bl[l - 1]) << 1;
      s.next_code[l] = c;
    }
  }
  __syncthreads();
  my_code = L ? (s.next_code[L] + s.wcnt[warp][L] + rank) : 0u;
  if (code_out && t < (int)nsym) code_out[t] = my_code;
  return true;
}

// The codebook, the layout decision and the header of one field; all
// threads of the CTA call it together.
__device__ __forceinline__ void codebook_body(const Geom &g, uint32_t R, uint32_t pred, uint32_t eb_mode, double eb,
                                              const CompressWs &ws, CbSmem &s, uint32_t &s_mode) {
  Ctl *ctl = ws.ctl;
  const int t = threadIdx.x;
  const uint32_t nsym = 2 * R;
  if (t == 0) {
    uint32_t mode = ctl->mode;
    if (mode == kModeNormal && ctl->n_out + ctl->n_exc > ws.cap_list) mode = kModeRaw;
    s_mode = mode;
    s.total_bits = 0;
  }
  __syncthreads();
  uint32_t mode = s_mode;
  if (mode == kModeNormal) {
    s.cnt[t] = t < (int)nsym ? ctl->hist[t] : 0ull;
    __syncthreads();
    uint32_t code = 0;
    bool ok = build_codebook(s, nsym, nullptr, code);
    __syncthreads();
    if (!ok) {
      if (t == 0) set_err(ctl, FZ_ECORRUPT);
      return;
    }
    unsigned long long b = 0;
    if (t < (int)nsym) {
      uint32_t L = s.len[t];
      ctl->lens[t] = (uint8_t)L;
      ctl->enc[t] = L ? (code << (32u - L)) | L : 0u;  // L <= 14
      b = s.cnt[t] * (unsigned long long)L;
    }
    for (int off = 16; off > 0; off >>= 1) b += __shfl_down_sync(0xffffffffu, b, off);
    if ((t & 31) == 0) s.key[t >> 5] = b;  // the sort keys are no longer needed
    __syncthreads();
    if (t < 32) {
      unsigned long long v = s.key[t];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (t == 0) s.total_bits = v;
    }
    __syncthreads();
  }
  if (t != 0) return;
  fz_header &h = ctl->res.hdr;
  const uint64_t N = g.n;
  if (mode == kModeNormal) {
    const uint64_t nb = g.n_blocks, nch = g.n_chunks;
    const uint64_t n_out = ctl->n_out, n_exc = ctl->n_exc, tb = s.total_bits;
    const bool sel = pred == FZ_SEL_MLP || pred == FZ_SEL_EXHAUSTIVE;
    const uint64_t off_lens = FZ_HEADER_BYTES;
    const uint64_t off_ids = align16(off_lens + nsym);
    const uint64_t off_anch = align16(off_ids + (sel ? (nb + 3) / 4 : 0));
    const uint64_t off_cb = align16(off_anch + 4 * nb);
    const uint64_t off_oidx = align16(off_cb + 4 * nch);
    const uint64_t off_oval = align16(off_oidx + 4 * n_out);
    const uint64_t off_eidx = align16(off_oval + 4 * n_out);
    const uint64_t off_eval = align16(off_eidx + 4 * n_exc);
    const uint64_t off_bits = align16(off_eval + 4 * n_exc);
    const uint64_t total = align16(off_bits + 4 * ((tb + 31) / 32));
    if (total > FZ_HEADER_BYTES + 4 * N) {
      mode = kModeRaw;
    } else {
      write_min_header(h, sel ? FZ_FLAG_IDS : 0, g, eb_mode, eb, total);
      h.eb_abs = ctl->eb_abs;
      h.ebx2_bits = __float_as_uint(ctl->ebx2);
      h.inv2eb_bits = __float_as_uint(ctl->inv2eb);
      h.ebchk_bits = __float_as_uint(ctl->eb_chk);
      h.radius = R;
      h.block[0] = g.bx; h.block[1] = g.by; h.block[2] = g.bz;
      h.predictor = pred;
      h.chunk = g.chunk;
      h.n_blocks = nb; h.n_chunks = nch; h.n_out = n_out; h.n_exc = n_exc; h.total_bits = tb;
      h.off_lens = off_lens; h.off_ids = sel ? off_ids : 0; h.off_anchors = off_anch; h.off_chunk_bits = off_cb;
      h.off_out_idx = off_oidx; h.off_out_val = off_oval; h.off_exc_idx = off_eidx; h.off_exc_val = off_eval;
      h.off_bits = off_bits;
      ctl->total_bits = tb;
    }
  }
  if (mode == kModeRaw) write_min_header(h, FZ_FLAG_RAW, g, eb_mode, eb, FZ_HEADER_BYTES + 4 * N);
  if (mode == kModeConst) write_min_header(h, FZ_FLAG_CONST, g, eb_mode, eb, FZ_HEADER_BYTES + 16);
  ctl->mode = mode;
  ctl->res.mode = mode;
  ctl->res.total_bytes = h.total_bytes;
  ctl->res.n_out = ctl->n_out;
  ctl->res.n_exc = ctl->n_exc;
}

__global__ void __launch_bounds__(kCbThreads) k_codebook(Geom g, uint32_t R, uint32_t pred, uint32_t eb_mode,
                                                          double eb, CompressWs ws) {
  extern __shared__ __align__(16) unsigned char cb_smem[];
  __shared__ uint32_t s_mode;
  dep_wait();
  dep_trigger();
  codebook_body(g, R, pred, eb_mode, eb, ws, *reinterpret_cast<CbSmem *>(cb_smem), s_mode);
}

// Batched variant: one CTA per field.
__global__ void __launch_bounds__(kCbThreads) k_codebook_batch(const BatchJob *__restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char cb_smem[];
  __shared__ uint32_t s_mode;
  const BatchJob &J = jobs[blockIdx.x];
  codebook_body(J.g, J.R, J.pred, J.eb_mode, J.eb, J.ws, *reinterpret_cast<CbSmem *>(cb_smem), s_mode);
}

// Packed placement of the batch's streams: each field's stream starts at a
// 16-byte boundary, in field order.  One CTA; also decides whether the
// packed output fits.
__global__ void __launch_bounds__(kCbThreads) k_batch_offsets(BatchJob *jobs, uint32_t n, uint64_t out_cap,
                                                               BatchCtl *bctl) {
  __shared__ unsigned long long wsum[kCbThreads / 32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const uint32_t per = (n + kCbThreads - 1) / kCbThreads;
  const uint32_t j0 = t * per;
  unsigned long long loc = 0;
  for (uint32_t j = j0; j < j0 + per && j < n; ++j) loc += align16(jobs[j].ws.ctl->res.total_bytes);
  unsigned long long incl = loc;
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  unsigned long long total = 0, run = incl - loc;
  for (int w = 0; w < kCbThreads / 32; ++w) {
    if (w < warp) run += wsum[w];
    total += wsum[w];
  }
  const bool fits = total <= out_cap;
  for (uint32_t j = j0; j < j0 + per && j < n; ++j) {
    jobs[j].out_off = fits ? run : kNoOutput;
    run += align16(jobs[j].ws.ctl->res.total_bytes);
  }
  if (t == 0) {
    bctl->total_bytes = total;
    if (!fits) atomicCAS(&bctl->err, 0u, (uint32_t)FZ_EBUFFER);
  }
}

// Per-field results and packed offsets, gathered for one copy to the host:
// offsets[0..n) the stream starts, offsets[n] the packed size, offsets[n+1]
// the batch-wide error word.
__global__ void k_batch_results(const BatchJob *__restrict__ jobs, uint32_t n, const BatchCtl *bctl, Result *res,
                                uint64_t *offsets) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n + 2; j += gridDim.x * blockDim.x) {
    if (j < n) {
      res[j] = jobs[j].ws.ctl->res;
      offsets[j] = jobs[j].out_off;
    } else if (j == n) {
      offsets[n] = bctl->total_bytes;
    } else {
      offsets[n + 1] = bctl->err;
    }
  }
}

__global__ void __launch_bounds__(kCbThreads) k_codebook_only(const uint64_t *hist, uint32_t nsym, uint8_t *lens,
                                                               uint32_t *codes, Ctl *ctl) {
  extern __shared__ __align__(16) unsigned char cb_smem[];
  CbSmem &s = *reinterpret_cast<CbSmem *>(cb_smem);
  const int t = threadIdx.x;
  s.cnt[t] = t < (int)nsym ? hist[t] : 0ull;
  __syncthreads();
  uint32_t code = 0;
  bool ok = build_codebook(s, nsym, codes, code);
  __syncthreads();
  if (!ok) {
    if (t == 0) set_err(ctl, FZ_EINVAL);
    return;
  }
  if (t < (int)nsym) lens[t] = s.len[t];
}

}  // namespace

cudaError_t launch_codebook(const Geom &g, uint32_t R, uint32_t pred, uint32_t eb_mode, double eb,
                            const CompressWs &ws, cudaStream_t st) {
  static LaunchCache cache;
  int per_sm = 0;
  // (sets the kernel's shared-memory limit once)
  const cudaError_t e = cached_per_sm(k_codebook, kCbThreads, (int)sizeof(CbSmem), cache, per_sm);
  if (e != cudaSuccess) return e;
  return launch_dep(k_codebook, 1u, (unsigned)kCbThreads, sizeof(CbSmem), st, g, R, pred, eb_mode, eb, ws);
}

cudaError_t launch_codebook_batch(const BatchJob *jobs, uint32_t n, cudaStream_t st) {
  cudaError_t e =
      cudaFuncSetAttribute(k_codebook_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CbSmem));
  if (e != cudaSuccess) return e;
  k_codebook_batch<<<n, kCbThreads, sizeof(CbSmem), st>>>(jobs);
  return cudaGetLastError();
}

cudaError_t launch_batch_offsets(BatchJob *jobs, uint32_t n, uint64_t out_cap, BatchCtl *bctl, cudaStream_t st) {
  k_batch_offsets<<<1, kCbThreads, 0, st>>>(jobs, n, out_cap, bctl);
  return cudaGetLastError();
}

cudaError_t launch_batch_results(const BatchJob *jobs, uint32_t n, const BatchCtl *bctl, Result *res,
                                 uint64_t *offsets, cudaStream_t st) {
  k_batch_results<<<(n + 2 + 255) / 256, 256, 0, st>>>(jobs, n, bctl, res, offsets);
  return cudaGetLastError();
}

cudaError_t launch_codebook_only(const uint64_t *hist, uint32_t nsym, uint8_t *lens, uint32_t *codes, Ctl *ctl,
                                 cudaStream_t st) {
  cudaError_t e =
      cudaFuncSetAttribute(k_codebook_only, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CbSmem));
  if (e != cudaSuccess) return e;
  k_codebook_only<<<1, kCbThreads, sizeof(CbSmem), st>>>(hist, nsym, lens, codes, ctl);
  return cudaGetLastError();
}

}  // namespace fz
