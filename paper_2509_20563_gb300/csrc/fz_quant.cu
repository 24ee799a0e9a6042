// fz_quant.cu -- prediction + quantization module (FZModules §3.1-§3.2).
//
// One persistent kernel walks the tiles of 4096 values (runs of consecutive
// blocks along x) in a static schedule; the loads of the next tile are in
// flight while the current one is processed, and the tile after that is
// being pulled into L2.  Per tile:
//   * FP32 prequantization q = rint(x * inv2eb) with the per-value bound
//     check (exceptions), straight from registers;
//   * the block-local Lorenzo residual, written as successive differences
//     (1 - S_x)^k, (1 - S_y)^k, (1 - S_z)^k with zero padding at the block
//     origin.  In 3D each warp owns one z-plane of the tile, each thread a
//     4x4 patch, so the x and y differences stay in registers (warp
//     shuffles for the patch borders) and only the z difference goes
//     through shared memory.  1D and 2D tiles difference in shared memory;
//   * radius-R codes in block-major order, anchors at block origins, the
//     code histogram in shared memory;
//   * outliers and exceptions, compacted by each warp in code-stream order
//     into a scratch list at slots taken with one atomic per warp and tile;
//     the assembler later lays the tiles out in order.
// HBM traffic: 4 bytes read and 2 bytes written per value.
#include "fz_internal.cuh"

#ifndef FZ_QUANT_MINB
#define FZ_QUANT_MINB 4
#endif
#ifndef FZ_QUANT_PREFETCH
#define FZ_QUANT_PREFETCH 1
#endif

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

template <int K>
__device__ __forceinline__ int lz_coef(int o) {
  if (K == 1) return o == 0 ? 1 : -1;
  return o == 1 ? -2 : 1;
}

struct QuantConst {
  float inv2eb, ebx2, eb_chk;
  int32_t R;
};

// Code of residual d at a position; marks outliers.  Out-of-domain
// positions and block origins get R.
__device__ __forceinline__ uint32_t make_code(int32_t d, int32_t R, bool in, bool origin, bool &outl) {
  const uint32_t c = (uint32_t)(d + R);
  const bool o = (c - 1u) >= (uint32_t)(2 * R - 1);
  const bool keep = in && !origin;
  outl = keep && o;
  return keep ? (o ? 0u : c) : (uint32_t)R;
}

// Tile coordinates.
struct TileXY {
  uint32_t tx, by, bz, x0, y0, z0;
};
template <int NDIM>
__device__ __forceinline__ TileXY tile_xy(const Geom &g, uint64_t tile) {
  using S = TileShape<NDIM>;
  TileXY t;
  const uint32_t t32 = (uint32_t)tile;  // tiles number at most nx*ny*nz < 2^32
  t.tx = t32 % g.tiles_x;
  const uint32_t rest = t32 / g.tiles_x;
  t.by = rest % g.nby;
  t.bz = rest / g.nby;
  t.x0 = t.tx * S::NB * S::BX;
  t.y0 = t.by * S::BY;
  t.z0 = t.bz * S::BZ;
  return t;
}

// A tile step split like a tile index (x, y, z tile counts), so that the
// coordinates of tile + step follow from those of tile by adds and carries.
struct TileStep {
  uint32_t sx, sy, sz;
};
__device__ __forceinline__ TileStep tile_step(const Geom &g, uint64_t step) {
  const uint32_t s32 = (uint32_t)step, r = s32 / g.tiles_x;
  return TileStep{s32 % g.tiles_x, r % g.nby, r / g.nby};
}
template <int NDIM>
__device__ __forceinline__ TileXY tile_advance(const Geom &g, TileXY t, const TileStep &s) {
  using S = TileShape<NDIM>;
  t.tx += s.sx;
  const uint32_t cx = t.tx >= g.tiles_x ? 1u : 0u;
  t.tx -= cx ? g.tiles_x : 0u;
  t.by += s.sy + cx;
  const uint32_t cy = t.by >= g.nby ? 1u : 0u;
  t.by -= cy ? g.nby : 0u;
  t.bz += s.sz + cy;
  t.x0 = t.tx * S::NB * S::BX;
  t.y0 = t.by * S::BY;
  t.z0 = t.bz * S::BZ;
  return t;
}

// Per-thread element mapping of a tile for the loads: 4 float4 per thread.
// 3D: warp = z-plane, lanes 0-15 rows 0-3, lanes 16-31 rows 4-7, 4 columns
// each.  1D/2D: float4 index tid + 256 j in row-major tile order.
template <int NDIM>
__device__ __forceinline__ void elem_rc(int tid, int j, int &row, int &col) {
  using S = TileShape<NDIM>;
  if (NDIM == 3) {
    const int warp = tid >> 5, lane = tid & 31;
    row = warp * 8 + (lane >> 4) * 4 + j;
    col = (lane & 15) * 4;
  } else {
    const int e = 4 * (tid + kQuantThreads * j);
    row = e / S::TX;
    col = e % S::TX;
  }
}

template <int NDIM>
__device__ __forceinline__ void load_tile(const float *__restrict__ x, const Geom &g, const TileXY &t, int tid,
                                          bool vec_ok, float4 (&v)[4]) {
  using S = TileShape<NDIM>;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int row, col;
    elem_rc<NDIM>(tid, j, row, col);
    const uint32_t X = t.x0 + col, Y = t.y0 + (row % S::BY), Z = t.z0 + row / S::BY;
    const bool inrow = Y < g.ny && Z < g.nz;
    const uint64_t fi = ((uint64_t)Z * g.ny + Y) * g.nx + X;
    if (inrow && vec_ok && X + 4 <= g.nx) {
      v[j] = __ldcs(reinterpret_cast<const float4 *>(x + fi));
    } else {
      float a[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = (inrow && X + u < g.nx) ? x[fi + u] : 0.0f;
      v[j] = make_float4(a[0], a[1], a[2], a[3]);
    }
  }
}

// L2 prefetch of a tile's input, one 128-byte line per thread for the first
// 128 threads (a tile is 16 KB: 3D 64 rows of 256 B, 2D 32 rows of 512 B,
// 1D one run of 16 KB); lines outside the field are skipped.
template <int NDIM>
__device__ __forceinline__ void prefetch_tile(const float *x, const Geom &g, const TileXY &t, int tid) {
  if (tid >= 128) return;
  uint32_t X, Y, Z;
  if (NDIM == 3) {
    const int row = tid >> 1;
    X = t.x0 + (tid & 1) * 32;
    Y = t.y0 + (row & 7);
    Z = t.z0 + (row >> 3);
  } else if (NDIM == 2) {
    X = t.x0 + (tid & 3) * 32;
    Y = t.y0 + (tid >> 2);
    Z = 0;
  } else {
    X = t.x0 + tid * 32;
    Y = 0;
    Z = 0;
  }
  if (X < g.nx && Y < g.ny && Z < g.nz) {
    const float *p = x + ((uint64_t)Z * g.ny + Y) * g.nx + X;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
  }
}

// Shared memory of one CTA.
template <int NDIM>
struct QuantSmem {
  static constexpr int TXP = TileShape<NDIM>::TX + 8;
  int32_t sq[2][TileShape<NDIM>::ROWS * TXP];  // double-buffered q (1D/2D) or x/y-differenced q (3D)
  uint8_t sexc[2][NDIM == 3 ? 16 : kTileElems];  // exception flags, tile row-major (1D/2D)
  uint32_t shist[kMaxSym];
};

// Residual at (row, col) of the shared tile for the ordered-compaction pass
// and for 1D/2D codes.  3D tiles hold x/y-differenced values: only the z
// difference remains.  1D/2D tiles hold q: the full difference is taken.
template <int NDIM, int K>
__device__ __forceinline__ int32_t smem_residual(const int32_t *sq, int row, int col, int px, int py, int pz) {
  using S = TileShape<NDIM>;
  constexpr int TXP = S::TX + 8;
  int32_t s = 0;
  if constexpr (NDIM == 3) {
#pragma unroll
    for (int oz = 0; oz <= K; ++oz)
      if (pz >= oz) s += lz_coef<K>(oz) * sq[(row - 8 * oz) * TXP + col];
  } else {
#pragma unroll
    for (int oy = 0; oy <= (NDIM >= 2 ? K : 0); ++oy)
#pragma unroll
      for (int ox = 0; ox <= K; ++ox) {
        int c = lz_coef<K>(ox);
        if (NDIM >= 2) c *= lz_coef<K>(oy);
        const bool ok = px >= ox && py >= oy;
        s += ok ? c * sq[(row - oy) * TXP + col - ox] : 0;
      }
  }
  return s;
}

// Phase A of a tile: prequantize this thread's 16 values, difference them
// along x and y in registers (3D), and store them to the shared tile.  The
// thread's exceptions: 1D/2D flag them in the shared tile (their codes are
// produced by other threads), 3D only counts them (the same thread codes
// them; the rare compaction pass finds them again from the input).
template <int NDIM, int K, bool INTERIOR>
__device__ __forceinline__ void tile_front(const Geom &g, const TileXY &t, const float4 (&v)[4],
                                           const QuantConst &qc, int32_t *sq, uint8_t *sexc, int32_t (&q)[4][4],
                                           uint32_t &nexc) {
  using S = TileShape<NDIM>;
  constexpr int TXP = S::TX + 8;
  constexpr bool kCountOnly = NDIM == 3 && INTERIOR;
  const int tid = threadIdx.x, lane = tid & 31;
  // prequantization by the float adder; values of magnitude 2^22 steps and
  // above (and NaN/Inf) send the thread's 16 values through prequant()
  bool slow_any = false;
  uint32_t exf[4];
  nexc = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float a[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
    exf[j] = 0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      bool ee, sl;
      q[j][u] = prequant_fast(a[u], qc.inv2eb, qc.ebx2, qc.eb_chk, ee, sl);
      slow_any |= sl;
      if (kCountOnly) nexc += ee ? 1u : 0u;
      else exf[j] |= (uint32_t)ee << (8 * u);
    }
  }
  if (slow_any) {
    nexc = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float a[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
      exf[j] = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        bool ee;
        q[j][u] = prequant(a[u], qc.inv2eb, qc.ebx2, qc.eb_chk, ee);
        if (kCountOnly) nexc += ee ? 1u : 0u;
        else exf[j] |= (uint32_t)ee << (8 * u);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int row, col;
    elem_rc<NDIM>(tid, j, row, col);
    const uint32_t X = t.x0 + col, Y = t.y0 + (row % S::BY), Z = t.z0 + row / S::BY;
    const bool inrow = INTERIOR || (Y < g.ny && Z < g.nz);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool in = INTERIOR || (inrow && X + u < g.nx);
      q[j][u] = in ? q[j][u] : 0;
      exf[j] &= in ? 0xffffffffu : ~(0xffu << (8 * u));
    }
    if (NDIM == 3) {
      if (!kCountOnly) nexc += __popc(exf[j]);
    } else {
      *reinterpret_cast<uint32_t *>(&sexc[row * S::TX + col]) = exf[j];
    }
  }
  if (NDIM == 3) {
    // (1 - S_x)^K within the thread's 4 columns; the left neighbour column
    // comes from lane - 1 unless the patch starts a block (px = 0).
    const bool blk_start = ((lane & 15) & 1) == 0;
#pragma unroll
    for (int rep = 0; rep < K; ++rep) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int32_t left = __shfl_up_sync(0xffffffffu, q[j][3], 1);
        q[j][3] -= q[j][2];
        q[j][2] -= q[j][1];
        q[j][1] -= q[j][0];
        q[j][0] -= blk_start ? 0 : left;
      }
    }
    // (1 - S_y)^K within rows 0-3 / 4-7; row 4 takes row 3 from lane - 16.
    const bool upper = (lane >> 4) != 0;
#pragma unroll
    for (int rep = 0; rep < K; ++rep) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int32_t above = __shfl_up_sync(0xffffffffu, q[3][u], 16);
        q[3][u] -= q[2][u];
        q[2][u] -= q[1][u];
        q[1][u] -= q[0][u];
        q[0][u] -= upper ? above : 0;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int row, col;
    elem_rc<NDIM>(tid, j, row, col);
    *reinterpret_cast<int4 *>(&sq[row * TXP + col]) = make_int4(q[j][0], q[j][1], q[j][2], q[j][3]);
  }
}

// Phase B of a 3D tile: the z difference, codes, anchors, histogram; the
// thread keeps its 4x4 patch of one z-plane.
template <int K, bool INTERIOR>
__device__ __forceinline__ void tile_codes3(const Geom &g, const TileXY &t, const QuantConst &qc,
                                            const CompressWs &ws, const int32_t *sq, uint32_t *shist,
                                            const int32_t (&q)[4][4], uint32_t &nout, uint32_t &nexc) {
  using S = TileShape<3>;
  constexpr int TXP = S::TX + 8;
  const int tid = threadIdx.x, lane = tid & 31, pz = tid >> 5;
  const int h = lane >> 4, c = (lane & 15) * 4;
  const int wb = c >> 3, px0 = c & 7;
  const uint32_t bxi = t.tx * S::NB + wb;
  const bool bvalid = INTERIOR || bxi < g.nbx;
  const uint64_t blk = (uint64_t)bxi + (uint64_t)g.nbx * (t.by + (uint64_t)g.nby * t.bz);
  uint32_t codes[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int py = 4 * h + j, row = pz * 8 + py;
    int32_t d[4] = {q[j][0], q[j][1], q[j][2], q[j][3]};
#pragma unroll
    for (int oz = 1; oz <= K; ++oz) {
      if (pz >= oz) {
        const int4 b = *reinterpret_cast<const int4 *>(&sq[(row - 8 * oz) * TXP + c]);
        const int cf = lz_coef<K>(oz);
        d[0] += cf * b.x; d[1] += cf * b.y; d[2] += cf * b.z; d[3] += cf * b.w;
      }
    }
    const bool yzin = INTERIOR || ((t.y0 + py < g.ny) && (t.z0 + pz < g.nz));
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool in = INTERIOR || (yzin && (t.x0 + c + u < g.nx));
      const bool origin = (j == 0 && u == 0) && (h == 0 && pz == 0 && px0 == 0);
      bool outl;
      codes[j][u] = make_code(d[u], qc.R, in, origin, outl);
      if (origin && bvalid) ws.anchors[blk] = d[u];
      nout += outl;
    }
    if (bvalid) {
      const uint64_t p0 = blk * 512 + pz * 64 + py * 8 + px0;
      *reinterpret_cast<uint2 *>(ws.codes + p0) =
          make_uint2(codes[j][0] | (codes[j][1] << 16), codes[j][2] | (codes[j][3] << 16));
    }
  }
  if (bvalid) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int u = 0; u < 4; ++u) atomicAdd(&shist[codes[j][u]], 1u);
  } else {
    nout = 0;
    nexc = 0;
  }
}

// Phase B of a 1D/2D tile: warp = half a block, 16 steps of 32 positions.
template <int NDIM, int K, bool INTERIOR>
__device__ __forceinline__ void tile_codes12(const Geom &g, const TileXY &t, const QuantConst &qc,
                                             const CompressWs &ws, const int32_t *sq, const uint8_t *sexc,
                                             uint32_t *shist, uint32_t &nout, uint32_t &nexc) {
  using S = TileShape<NDIM>;
  constexpr int kPerWarp = S::BX * S::BY / S::WPB;
  constexpr int kIter = kPerWarp / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wb = warp / S::WPB, seg = warp % S::WPB;
  const uint32_t bxi = t.tx * S::NB + wb;
  if (!INTERIOR && bxi >= g.nbx) return;
  const uint64_t blk = (uint64_t)bxi + (uint64_t)g.nbx * (t.by + (uint64_t)g.nby * t.bz);
  uint16_t *cdst = ws.codes + blk * g.bsize + seg * kPerWarp;
#pragma unroll 4
  for (int i = 0; i < kIter; ++i) {
    const int p = seg * kPerWarp + 32 * i + lane;
    const int px = p % S::BX, py = p / S::BX;
    const int row = py, col = wb * S::BX + px;
    const bool in = INTERIOR || ((t.x0 + col < g.nx) && (t.y0 + py < g.ny));
    const int32_t d = smem_residual<NDIM, K>(sq, row, col, px, py, 0);
    bool outl;
    const uint32_t code = make_code(d, qc.R, in, p == 0, outl);
    if (p == 0) ws.anchors[blk] = d;
    cdst[32 * i + lane] = (uint16_t)code;
    atomicAdd(&shist[code], 1u);
    nout += outl;
    nexc += (in && sexc[row * S::TX + col]) ? 1u : 0u;
  }
}

// The tiles tile, tile + step, ... below t_end of one field, then the
// field's histogram flush.  All threads of the CTA call it together.  DEP:
// launched behind the range pass (launch_dep): the first tile's loads of the
// input go out before the wait for the pass's constants.
template <int NDIM, int K, bool DEP = false>
__device__ __forceinline__ void quant_tiles(const float *__restrict__ x, const Geom &g, uint32_t R,
                                            const CompressWs &ws, uint64_t tile, uint64_t t_end, uint64_t t_step,
                                            QuantSmem<NDIM> &sm) {
  using S = TileShape<NDIM>;
  constexpr int kPerWarp = S::BX * S::BY * S::BZ / S::WPB;  // 512 positions
  constexpr int kIter = kPerWarp / 32;                      // 16
  static_assert(S::TX * S::ROWS == kTileElems, "tile size");
  static_assert(S::NB * S::WPB == kQuantThreads / 32, "warps per tile");

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t nsym = 2 * R;
  for (int s = tid; s < kMaxSym; s += kQuantThreads) sm.shist[s] = 0;
  // 16-byte loads of 4 consecutive x: aligned whenever rows start on a
  // 4-value boundary (1D: always; 2D/3D: nx a multiple of 4)
  const bool vec_ok = (NDIM == 1 || (g.nx & 3u) == 0) && (((uintptr_t)x & 15u) == 0);

  float4 v[4];
  const TileStep tstep = tile_step(g, t_step);
  TileXY tn = tile_xy<NDIM>(g, tile);  // coordinates of the tile whose loads are in flight
  if (tile < t_end) load_tile<NDIM>(x, g, tn, tid, vec_ok, v);
  if (DEP) {
    dep_wait();
    dep_trigger();
  }
  Ctl *ctl = ws.ctl;
  if (ctl->mode != kModeNormal) return;
  QuantConst qc;
  qc.inv2eb = ctl->inv2eb;
  qc.ebx2 = ctl->ebx2;
  qc.eb_chk = ctl->eb_chk;
  qc.R = (int32_t)R;
  for (int buf = 0; tile < t_end; tile += t_step, buf ^= 1) {
    const TileXY t = tn;
    // a tile that lies wholly inside the domain skips every bounds test
    const bool interior = vec_ok && t.x0 + S::TX <= g.nx && t.y0 + S::BY <= g.ny && t.z0 + S::BZ <= g.nz;
    int32_t *sq = sm.sq[buf];
    uint8_t *sexc = sm.sexc[buf];
    uint32_t nout = 0, nexc = 0;
    int32_t q[4][4];
    if (interior) tile_front<NDIM, K, true>(g, t, v, qc, sq, sexc, q, nexc);
    else tile_front<NDIM, K, false>(g, t, v, qc, sq, sexc, q, nexc);
    __syncthreads();
    // ---- next tile's loads go out now and land while this tile is coded
    {
      const uint64_t nt = tile + t_step;
      tn = tile_advance<NDIM>(g, t, tstep);
      if (nt < t_end) load_tile<NDIM>(x, g, tn, tid, vec_ok, v);
#if FZ_QUANT_PREFETCH
      // and the tile after it is pulled into L2
      if (nt + t_step < t_end) prefetch_tile<NDIM>(x, g, tile_advance<NDIM>(g, tn, tstep), tid);
#endif
    }
    if (NDIM == 3) {
      if (interior) tile_codes3<K, true>(g, t, qc, ws, sq, sm.shist, q, nout, nexc);
      else tile_codes3<K, false>(g, t, qc, ws, sq, sm.shist, q, nout, nexc);
    } else {
      nexc = 0;  // counted by the coding threads from the shared flags
      if (interior) tile_codes12<NDIM, K, true>(g, t, qc, ws, sq, sexc, sm.shist, nout, nexc);
      else tile_codes12<NDIM, K, false>(g, t, qc, ws, sq, sexc, sm.shist, nout, nexc);
    }

    // ---- outliers / exceptions (rare): each warp compacts its own positions
    // in code order, without waiting for the other warps -- 3D: its z-plane of
    // each of the tile's blocks, 1D/2D: its half block.  The shared tiles are
    // double-buffered, so the values read here stay put until the next-but-one
    // tile, which starts after the next tile's barrier.
    nout = __reduce_add_sync(0xffffffffu, nout);
    nexc = __reduce_add_sync(0xffffffffu, nexc);
    WarpSlots wsl;
    wsl.oslot = 0;
    wsl.eslot = 0;
    wsl.ocnt = 0;
    wsl.ecnt = 0;
    if ((nout | nexc) != 0) {
      if (lane == 0) {
        wsl.oslot = nout ? (uint32_t)atomicAdd(&ctl->n_out, (unsigned long long)nout) : 0u;
        wsl.eslot = nexc ? (uint32_t)atomicAdd(&ctl->n_exc, (unsigned long long)nexc) : 0u;
        if (nout) atomicAdd(&ws.tinfo[tile].x, nout);
        if (nexc) atomicAdd(&ws.tinfo[tile].y, nexc);
        const uint64_t grp = tile / kTileGroup;
        if (nout) atomicAdd(&ws.tgroup[grp].x, nout);
        if (nexc) atomicAdd(&ws.tgroup[grp].y, nexc);
      }
      wsl.oslot = __shfl_sync(0xffffffffu, wsl.oslot, 0);
      wsl.eslot = __shfl_sync(0xffffffffu, wsl.eslot, 0);
      uint32_t oo = wsl.oslot, eo = wsl.eslot;
      // append the outliers and exceptions of `n` positions (code order = lane order per step)
      auto emit = [&](bool outl, int32_t d, bool e, uint32_t pos, uint64_t fi, uint32_t &co, uint32_t &ce) {
        uint32_t m = __ballot_sync(0xffffffffu, outl);
        if (outl) {
          const uint64_t o = (uint64_t)oo + __popc(m & ((1u << lane) - 1));
          if (o < ws.cap_list) { ws.out_idx[o] = pos; ws.out_val[o] = d; }
        }
        oo += __popc(m);
        co += __popc(m);
        m = __ballot_sync(0xffffffffu, e);
        if (e) {
          const uint64_t o = (uint64_t)eo + __popc(m & ((1u << lane) - 1));
          if (o < ws.cap_list) { ws.exc_idx[o] = pos; ws.exc_val[o] = __float_as_uint(x[fi]); }
        }
        eo += __popc(m);
        ce += __popc(m);
      };
      if (NDIM == 3) {
        const int pz = warp;
        for (int b = 0; b < S::NB; ++b) {
          const uint32_t bxi = t.tx * S::NB + b;
          if (bxi >= g.nbx) break;
          const uint64_t blk = (uint64_t)bxi + (uint64_t)g.nbx * (t.by + (uint64_t)g.nby * t.bz);
          uint32_t co = 0, ce = 0;
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const int idx = 32 * half + lane, px = idx & 7, py = idx >> 3;
            const int row = py + 8 * pz, col = 8 * b + px;
            const bool in = (t.x0 + col < g.nx) && (t.y0 + py < g.ny) && (t.z0 + pz < g.nz);
            const int32_t d = smem_residual<3, K>(sq, row, col, px, py, pz);
            bool outl;
            make_code(d, qc.R, in, idx == 0 && pz == 0, outl);
            const uint64_t fi = ((uint64_t)(t.z0 + pz) * g.ny + (t.y0 + py)) * g.nx + (t.x0 + col);
            // this warp's exceptions, found again from the input (nexc > 0 only)
            bool ex = false;
            if (nexc != 0 && in) prequant(x[fi], qc.inv2eb, qc.ebx2, qc.eb_chk, ex);
            emit(outl, d, ex, (uint32_t)(blk * 512 + 64 * pz + idx), fi, co, ce);
          }
          wsl.ocnt |= (unsigned long long)co << (8 * b);
          wsl.ecnt |= (unsigned long long)ce << (8 * b);
        }
      } else {
        const int wb = warp / S::WPB, seg = warp % S::WPB;
        const uint32_t bxi = t.tx * S::NB + wb;
        const uint64_t blk = (uint64_t)bxi + (uint64_t)g.nbx * (t.by + (uint64_t)g.nby * t.bz);
        uint32_t co = 0, ce = 0;
        if (bxi < g.nbx) {
          for (int i = 0; i < kIter; ++i) {
            const int p = seg * kPerWarp + 32 * i + lane;
            const int px = p % S::BX, py = (p / S::BX) % S::BY;
            const int row = py, col = wb * S::BX + px;
            const bool in = (t.x0 + col < g.nx) && (t.y0 + py < g.ny);
            const int32_t d = smem_residual<NDIM, K>(sq, row, col, px, py, 0);
            bool outl;
            make_code(d, qc.R, in, p == 0, outl);
            const uint64_t fi = (uint64_t)(t.y0 + py) * g.nx + (t.x0 + col);
            emit(outl, d, in && sexc[row * S::TX + col], (uint32_t)(blk * g.bsize + p), fi, co, ce);
          }
        }
        wsl.ocnt = co;
        wsl.ecnt = ce;
      }
    }
    if (lane == 0) ws.winfo[tile * 8 + warp] = wsl;
  }
  __syncthreads();
  for (int s = tid; s < (int)nsym; s += kQuantThreads)
    if (sm.shist[s]) atomicAdd(&ctl->hist[s], (unsigned long long)sm.shist[s]);
}

template <int NDIM, int K>
__global__ void __launch_bounds__(kQuantThreads, FZ_QUANT_MINB) k_quant(const float *__restrict__ x, Geom g, uint32_t R,
                                                             CompressWs ws) {
  extern __shared__ __align__(16) unsigned char q_smem[];
  QuantSmem<NDIM> &sm = *reinterpret_cast<QuantSmem<NDIM> *>(q_smem);
  quant_tiles<NDIM, K, true>(x, g, R, ws, blockIdx.x, g.n_qtiles, gridDim.x, sm);
}

// Batched variant: the quantization tiles of every field of one class
// (dimensionality, Lorenzo order) form one queue, cut into equal contiguous
// ranges, one per CTA; a CTA runs the fields its range overlaps in turn
// (field parameters staged in shared memory, the histogram flushed per
// field).
template <int NDIM, int K>
__global__ void __launch_bounds__(kQuantThreads, 3) k_quant_batch(const BatchJob *__restrict__ jobs,
                                                                   const uint32_t *__restrict__ members,
                                                                   uint32_t n_members, uint64_t total_tiles) {
  extern __shared__ __align__(16) unsigned char q_smem[];
  QuantSmem<NDIM> &sm = *reinterpret_cast<QuantSmem<NDIM> *>(q_smem);
  __shared__ Geom sg;
  __shared__ CompressWs sws;
  __shared__ const float *sx;
  __shared__ uint32_t sR;
  const uint64_t lo = total_tiles * blockIdx.x / gridDim.x, hi = total_tiles * (blockIdx.x + 1) / gridDim.x;
  // first member whose tiles reach past lo
  uint32_t a = 0, b = n_members;
  while (a < b) {
    const uint32_t m = (a + b) >> 1;
    const BatchJob &J = jobs[members[m]];
    if (J.qtile_base + J.g.n_qtiles <= lo) a = m + 1; else b = m;
  }
  for (uint64_t t = lo; t < hi && a < n_members; ++a) {
    const BatchJob &J = jobs[members[a]];
    const uint64_t jb = J.qtile_base, je = jb + J.g.n_qtiles;
    const uint64_t t0 = t > jb ? t : jb, t1 = hi < je ? hi : je;
    __syncthreads();  // the previous field's flush is done with the staged parameters
    if (threadIdx.x == 0) { sg = J.g; sws = J.ws; sx = J.x; sR = J.R; }
    __syncthreads();
    if (t0 < t1) quant_tiles<NDIM, K>(sx, sg, sR, sws, t0 - jb, t1 - jb, 1, sm);
    t = t1;
  }
}

template <int NDIM, int K>
cudaError_t launch_t(const float *x, const Geom &g, uint32_t R, const CompressWs &ws, cudaStream_t s, int sms) {
  const int smem = (int)sizeof(QuantSmem<NDIM>);
  static LaunchCache cache;
  int per_sm = 0;
  const cudaError_t e = cached_per_sm(k_quant<NDIM, K>, kQuantThreads, smem, cache, per_sm);
  if (e != cudaSuccess) return e;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > g.n_qtiles) grid = g.n_qtiles;
  return launch_dep(k_quant<NDIM, K>, (unsigned)grid, kQuantThreads, (size_t)smem, s, x, g, R, ws);
}

template <int NDIM, int K>
cudaError_t launch_batch_t(const BatchJob *jobs, const uint32_t *members, uint32_t n_members, uint64_t total_tiles,
                           int per_sm, cudaStream_t s, int sms) {
  const int smem = (int)sizeof(QuantSmem<NDIM>);
  cudaError_t e = cudaFuncSetAttribute(k_quant_batch<NDIM, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_quant_batch<NDIM, K>, kQuantThreads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  if (per_sm < 1 || per_sm > occ) per_sm = occ;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > total_tiles) grid = total_tiles;
  if (grid < 1) grid = 1;
  k_quant_batch<NDIM, K><<<(unsigned)grid, kQuantThreads, smem, s>>>(jobs, members, n_members, total_tiles);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_quant_batch(int ndim, int k, const BatchJob *jobs, const uint32_t *members, uint32_t n_members,
                               uint64_t total_tiles, int per_sm, cudaStream_t s, int sm_count) {
  const bool k2 = k == 2;
  switch (ndim) {
    case 1:
      return k2 ? launch_batch_t<1, 2>(jobs, members, n_members, total_tiles, per_sm, s, sm_count)
                : launch_batch_t<1, 1>(jobs, members, n_members, total_tiles, per_sm, s, sm_count);
    case 2:
      return k2 ? launch_batch_t<2, 2>(jobs, members, n_members, total_tiles, per_sm, s, sm_count)
                : launch_batch_t<2, 1>(jobs, members, n_members, total_tiles, per_sm, s, sm_count);
    default:
      return k2 ? launch_batch_t<3, 2>(jobs, members, n_members, total_tiles, per_sm, s, sm_count)
                : launch_batch_t<3, 1>(jobs, members, n_members, total_tiles, per_sm, s, sm_count);
  }
}

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
