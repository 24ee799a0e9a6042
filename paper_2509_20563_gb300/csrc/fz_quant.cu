// fz_quant.cu -- prediction + quantization module (FZModules §3.1-§3.2).
//
// One persistent kernel does, per tile of 4096 values (a run of consecutive
// blocks along x): coalesced 16-byte loads of the field into shared memory
// with FP32 prequantization (q = rint(x * inv2eb), per-value bound check ->
// exceptions), the block-local Lorenzo residual read back from shared memory,
// radius-R codes written in block-major order, anchors at block origins, the
// code histogram in shared memory, and ordered compaction of outliers and
// exceptions whose global offsets come from a bounded decoupled look-back
// over tiles.  HBM traffic: 4 bytes read and 2 bytes written per value.
#include "fz_internal.cuh"

namespace fz {

namespace {

template <int NDIM>
struct TileShape;
template <>
struct TileShape<1> {
  static constexpr int BX = 1024, BY = 1, BZ = 1, NB = 4, TX = 4096, ROWS = 1, WPB = 2;
};
template <>
struct TileShape<2> {
  static constexpr int BX = 32, BY = 32, BZ = 1, NB = 4, TX = 128, ROWS = 32, WPB = 2;
};
template <>
struct TileShape<3> {
  static constexpr int BX = 8, BY = 8, BZ = 8, NB = 8, TX = 64, ROWS = 64, WPB = 1;
};

__device__ __forceinline__ int32_t prequant(float x, float inv2eb, float ebx2, float eb_chk, bool &exc) {
  if (!isfinite(x)) { exc = true; return 0; }
  float t = __fmul_rn(x, inv2eb);
  if (!(fabsf(t) < 8388608.0f)) { exc = true; return 0; }
  int32_t q = __float2int_rn(t);
  float r = __fmul_rn(__int2float_rn(q), ebx2);
  float d = fabsf(__fsub_rn(x, r));
  exc = d > eb_chk;
  return q;
}

template <int K>
__device__ __forceinline__ int lz_coef(int o) {
  if (K == 1) return o == 0 ? 1 : -1;
  return o == 1 ? -2 : 1;
}

// Lorenzo-K residual of the point at (row, col) of the shared tile; terms that
// fall before the block origin along any axis are zero.
template <int NDIM, int K, int TXP>
__device__ __forceinline__ int32_t lorenzo_residual(const int32_t *sq, int row, int col, int px, int py, int pz) {
  using S = TileShape<NDIM>;
  int32_t s = 0;
#pragma unroll
  for (int oz = 0; oz <= (NDIM >= 3 ? K : 0); ++oz)
#pragma unroll
    for (int oy = 0; oy <= (NDIM >= 2 ? K : 0); ++oy)
#pragma unroll
      for (int ox = 0; ox <= K; ++ox) {
        int c = lz_coef<K>(ox);
        if (NDIM >= 2) c *= lz_coef<K>(oy);
        if (NDIM >= 3) c *= lz_coef<K>(oz);
        bool ok = px >= ox && py >= oy && pz >= oz;
        int32_t v = ok ? sq[(row - oy - S::BY * oz) * TXP + col - ox] : 0;
        s += c * v;
      }
  return s;
}

template <int NDIM, int K>
__global__ void __launch_bounds__(kQuantThreads) k_quant(const float *__restrict__ x, Geom g, uint32_t R,
                                                          CompressWs ws) {
  using S = TileShape<NDIM>;
  constexpr int TXP = S::TX + 8;
  constexpr int kPerWarp = S::BX * S::BY * S::BZ / S::WPB;  // 512 positions
  constexpr int kIter = kPerWarp / 32;                      // 16
  static_assert(S::TX * S::ROWS == kTileElems, "tile size");
  static_assert(S::NB * S::WPB == kQuantThreads / 32, "warps per tile");

  __shared__ __align__(16) int32_t sq[S::ROWS * TXP];
  __shared__ __align__(16) uint8_t sexc[kTileElems];
  __shared__ uint32_t shist[kMaxSym];
  __shared__ uint32_t s_wout[8], s_wexc[8], s_wout_off[8], s_wexc_off[8];
  __shared__ uint32_t s_tile;

  Ctl *ctl = ws.ctl;
  if (ctl->mode != kModeNormal) return;
  const float inv2eb = ctl->inv2eb, ebx2 = ctl->ebx2, eb_chk = ctl->eb_chk;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t nsym = 2 * R;
  for (int s = tid; s < kMaxSym; s += kQuantThreads) shist[s] = 0;
  const bool vec_ok = ((g.nx & 3u) == 0) && (((uintptr_t)x & 15u) == 0);

  for (;;) {
    if (tid == 0) s_tile = atomicAdd(&ctl->quant_ticket, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= g.n_qtiles) break;
    const uint32_t tx = (uint32_t)(tile % g.tiles_x);
    const uint64_t rest = tile / g.tiles_x;
    const uint32_t by = (uint32_t)(rest % g.nby), bz = (uint32_t)(rest / g.nby);
    const uint32_t x0 = tx * S::NB * S::BX;
    const uint32_t y0 = by * S::BY, z0 = bz * S::BZ;

    // ---- phase 1: load + prequantize into shared memory (row-major tile)
#pragma unroll
    for (int j = 0; j < kTileElems / 4 / kQuantThreads; ++j) {
      const int e = 4 * (tid + kQuantThreads * j);
      const int row = e / S::TX, col = e % S::TX;
      const uint32_t X = x0 + col;
      const uint32_t Y = y0 + (row % S::BY), Z = z0 + row / S::BY;
      float v[4];
      bool inrow = Y < g.ny && Z < g.nz;
      uint64_t fi = ((uint64_t)Z * g.ny + Y) * g.nx + X;
      if (inrow && vec_ok && X < g.nx) {
        float4 f = __ldcs(reinterpret_cast<const float4 *>(x + fi));
        v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = (inrow && X + u < g.nx) ? x[fi + u] : 0.0f;
      }
      int4 q4;
      uint32_t ex = 0;
      int32_t qq[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        bool in = inrow && X + u < g.nx;
        bool ee = false;
        qq[u] = in ? prequant(v[u], inv2eb, ebx2, eb_chk, ee) : 0;
        ex |= (uint32_t)(in && ee) << (8 * u);
      }
      q4.x = qq[0]; q4.y = qq[1]; q4.z = qq[2]; q4.w = qq[3];
      *reinterpret_cast<int4 *>(&sq[row * TXP + col]) = q4;
      *reinterpret_cast<uint32_t *>(&sexc[e]) = ex;
    }
    __syncthreads();

    // ---- phase 2: residuals, codes, histogram, counts (warp = block segment)
    const int wb = warp / S::WPB, seg = warp % S::WPB;
    const uint32_t bxi = tx * S::NB + wb;
    const bool wvalid = bxi < g.nbx;
    const uint64_t blk = (uint64_t)bxi + (uint64_t)g.nbx * (by + (uint64_t)g.nby * bz);
    uint32_t nout = 0, nexc = 0;
    if (wvalid) {
      uint16_t *cdst = ws.codes + blk * g.bsize + seg * kPerWarp;
#pragma unroll 4
      for (int i = 0; i < kIter; ++i) {
        const int p = seg * kPerWarp + 32 * i + lane;
        const int px = p % S::BX, py = (p / S::BX) % S::BY, pz = p / (S::BX * S::BY);
        const int row = py + S::BY * pz, col = wb * S::BX + px;
        const bool in = (x0 + col < g.nx) && (y0 + py < g.ny) && (z0 + pz < g.nz);
        const int32_t d = lorenzo_residual<NDIM, K, TXP>(sq, row, col, px, py, pz);
        uint32_t code;
        bool outl = false;
        if (!in) code = R;
        else if (p == 0) { code = R; ws.anchors[blk] = d; }
        else if (d > -(int32_t)R && d < (int32_t)R) code = (uint32_t)(d + (int32_t)R);
        else { code = 0; outl = true; }
        cdst[32 * i + lane] = (uint16_t)code;
        const uint32_t c0 = __shfl_sync(0xffffffffu, code, 0);
        if (__all_sync(0xffffffffu, code == c0)) {
          if (lane == 0) atomicAdd(&shist[c0], 32u);
        } else {
          atomicAdd(&shist[code], 1u);
        }
        nout += __popc(__ballot_sync(0xffffffffu, outl));
        nexc += __popc(__ballot_sync(0xffffffffu, in && sexc[row * S::TX + col]));
      }
    }
    if (lane == 0) { s_wout[warp] = nout; s_wexc[warp] = nexc; }
    __syncthreads();

    // ---- phase 3: tile totals and their global offsets (look-back)
    if (tid == 0) {
      uint32_t to = 0, te = 0;
      for (int w = 0; w < 8; ++w) {
        s_wout_off[w] = to; to += s_wout[w];
        s_wexc_off[w] = te; te += s_wexc[w];
      }
      uint64_t agg = (uint64_t)to | ((uint64_t)te << 31);
      uint64_t ex = lookback<true>(ws.qstatus, tile, agg, ctl);
      uint32_t eo = (uint32_t)(ex & ((1ull << 31) - 1)), ee = (uint32_t)(ex >> 31);
      for (int w = 0; w < 8; ++w) { s_wout_off[w] += eo; s_wexc_off[w] += ee; }
      if (to) atomicAdd(&ctl->n_out, (unsigned long long)to);
      if (te) atomicAdd(&ctl->n_exc, (unsigned long long)te);
    }
    __syncthreads();

    // ---- phase 4: ordered write of this warp's outliers and exceptions
    if (wvalid && (nout | nexc)) {
      uint32_t oo = s_wout_off[warp], eo = s_wexc_off[warp];
      for (int i = 0; i < kIter; ++i) {
        const int p = seg * kPerWarp + 32 * i + lane;
        const int px = p % S::BX, py = (p / S::BX) % S::BY, pz = p / (S::BX * S::BY);
        const int row = py + S::BY * pz, col = wb * S::BX + px;
        const bool in = (x0 + col < g.nx) && (y0 + py < g.ny) && (z0 + pz < g.nz);
        const uint32_t pos = (uint32_t)(blk * g.bsize + p);
        if (nout) {
          const int32_t d = lorenzo_residual<NDIM, K, TXP>(sq, row, col, px, py, pz);
          const bool outl = in && p != 0 && !(d > -(int32_t)R && d < (int32_t)R);
          const uint32_t m = __ballot_sync(0xffffffffu, outl);
          if (outl) {
            uint64_t o = (uint64_t)oo + __popc(m & ((1u << lane) - 1));
            if (o < ws.cap_list) { ws.out_idx[o] = pos; ws.out_val[o] = d; }
          }
          oo += __popc(m);
        }
        if (nexc) {
          const bool e = in && sexc[row * S::TX + col];
          const uint32_t m = __ballot_sync(0xffffffffu, e);
          if (e) {
            uint64_t o = (uint64_t)eo + __popc(m & ((1u << lane) - 1));
            uint64_t fi = ((uint64_t)(z0 + pz) * g.ny + (y0 + py)) * g.nx + (x0 + col);
            if (o < ws.cap_list) { ws.exc_idx[o] = pos; ws.exc_val[o] = __float_as_uint(x[fi]); }
          }
          eo += __popc(m);
        }
      }
    }
    __syncthreads();
  }
  // flush the CTA histogram
  for (int s = tid; s < (int)nsym; s += kQuantThreads)
    if (shist[s]) atomicAdd(&ctl->hist[s], (unsigned long long)shist[s]);
}

template <int NDIM, int K>
cudaError_t launch_t(const float *x, const Geom &g, uint32_t R, const CompressWs &ws, cudaStream_t s, int sms) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_quant<NDIM, K>, kQuantThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > g.n_qtiles) grid = g.n_qtiles;
  k_quant<NDIM, K><<<(unsigned)grid, kQuantThreads, 0, s>>>(x, g, R, ws);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_quant(const float *x, const Geom &g, uint32_t R, uint32_t pred, const CompressWs &ws,
                         cudaStream_t s, int sm_count) {
  const bool k2 = pred == FZ_PRED_LORENZO2;
  switch (g.ndim) {
    case 1: return k2 ? launch_t<1, 2>(x, g, R, ws, s, sm_count) : launch_t<1, 1>(x, g, R, ws, s, sm_count);
    case 2: return k2 ? launch_t<2, 2>(x, g, R, ws, s, sm_count) : launch_t<2, 1>(x, g, R, ws, s, sm_count);
    default: return k2 ? launch_t<3, 2>(x, g, R, ws, s, sm_count) : launch_t<3, 1>(x, g, R, ws, s, sm_count);
  }
}

}  // namespace fz
