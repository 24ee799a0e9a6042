// fz_select.cu -- per-block predictor selection for 3D fields (the
// auto-selection of modules that FZModules names as future work in §5, and
// the dynamic module selection of §3.3.1), built on the prediction +
// quantization module of §3.1.
//
// Each 8x8x8 block is predicted by one of four predictors: Lorenzo order 1
// or 2, or in-block interpolation (linear or cubic; levels 4, 2, 1 with the
// corner anchors o + {0,8}^3).  The choice comes from an exhaustive trial
// (the predictor with the smallest trial cost) or from a small network
// (32 block statistics -> 64 hidden -> 4 logits, bfloat16 weights, binary32
// fmaf accumulation in a fixed order).  The 2-bit choice of every block goes
// into the stream.
//
// Kernels:
//   k_selquant   -- one warp per block of a 4096-value tile: prequantize,
//                   gather the corner anchors, choose the predictor (or only
//                   report labels, trial costs and features), then codes,
//                   anchors, histogram and ordered outliers/exceptions like
//                   the plain quantizer
//   k_dec_codes  -- one thread per chunk: Huffman decode into a code buffer
//   k_sel_recon  -- one warp per block: outlier scatter, anchor, inverse of
//                   the block's predictor, dequantization, exceptions
#include <string.h>

#include "fz_decode_common.cuh"

#ifndef FZ_SEL_MINB
#define FZ_SEL_MINB 3
#endif

namespace fz {

namespace {

constexpr int kTX = 64, kTXP = 72, kRows = 64;  // tile: 8 blocks along x, rows (y, z)
constexpr int kSelThreads = 256;

enum SelMode : int { kSelFixed = 0, kSelExhaustive = 1, kSelNet = 2, kSelReport = 3, kSelGinterp = 4 };

// Per-warp view of one block inside the shared tile.
struct BlockView {
  const int32_t *sq;   // tile q, row (py + 8 pz), column (8 wb + px)
  const int32_t *cq;   // q at the 8 corners o + 8 (cx, cy, cz), index cx + 2 cy + 4 cz
  uint32_t cin;        // corner availability bits
  int wb;              // block within the tile
  uint32_t xlim, ylim, zlim;  // in-domain extent of the block (1..8 per axis)
  const uint4 *itab;   // full-block interpolation stencils (InterpTab entries), quantizer only
  __device__ __forceinline__ bool in(int px, int py, int pz) const {
    return (uint32_t)px < xlim && (uint32_t)py < ylim && (uint32_t)pz < zlim;
  }
  __device__ __forceinline__ int32_t at(int px, int py, int pz) const {
    return sq[(py + 8 * pz) * kTXP + 8 * wb + px];
  }
  // value and availability of a neighbourhood point during interpolation
  __device__ __forceinline__ bool get(int x, int y, int z, int64_t &v) const {
    if (x >= 0 && y >= 0 && z >= 0 && x < 8 && y < 8 && z < 8) {
      if (!in(x, y, z)) return false;
      v = at(x, y, z);
      return true;
    }
    if ((x != 0 && x != 8) || (y != 0 && y != 8) || (z != 0 && z != 8)) return false;
    const int c = (x >> 3) + 2 * (y >> 3) + 4 * (z >> 3);
    if (!((cin >> c) & 1u)) return false;
    v = cq[c];
    return true;
  }
};

template <int K>
__device__ __forceinline__ int lzc(int o) {
  if (K == 1) return o == 0 ? 1 : -1;
  return o == 1 ? -2 : 1;
}

// Lorenzo-K residual (zero outside the block; the lower neighbours of an
// in-domain point are in the domain).
template <int K>
__device__ __forceinline__ int32_t res_lorenzo(const BlockView &b, int px, int py, int pz) {
  int32_t s = 0;
#pragma unroll
  for (int oz = 0; oz <= K; ++oz)
#pragma unroll
    for (int oy = 0; oy <= K; ++oy)
#pragma unroll
      for (int ox = 0; ox <= K; ++ox)
        if (px >= ox && py >= oy && pz >= oz) s += lzc<K>(ox) * lzc<K>(oy) * lzc<K>(oz) * b.at(px - ox, py - oy, pz - oz);
  return s;
}

// Level and pass axis of a non-origin block point.
__device__ __forceinline__ void level_axis(int px, int py, int pz, int &s, int &a) {
  const int v = px | py | pz;
  s = (v & 1) ? 1 : ((v & 2) ? 2 : 4);
  a = ((pz / s) & 1) ? 2 : (((py / s) & 1) ? 1 : 0);
}

// Interpolation prediction of a non-origin point from the values `b`
// exposes (q during compression, reconstructed q during decompression).
__device__ __forceinline__ int64_t interp_pred(const BlockView &b, bool cubic, int px, int py, int pz) {
  int s, a;
  level_axis(px, py, pz, s, a);
  const int dx = a == 0 ? s : 0, dy = a == 1 ? s : 0, dz = a == 2 ? s : 0;
  int64_t vm1 = 0, vp1 = 0, vm3 = 0, vp3 = 0;
  const bool am1 = b.get(px - dx, py - dy, pz - dz, vm1);
  const bool ap1 = b.get(px + dx, py + dy, pz + dz, vp1);
  if (cubic) {
    const bool am3 = b.get(px - 3 * dx, py - 3 * dy, pz - 3 * dz, vm3);
    const bool ap3 = b.get(px + 3 * dx, py + 3 * dy, pz + 3 * dz, vp3);
    if (am3 && am1 && ap1 && ap3) return (-vm3 + 9 * vm1 + 9 * vp1 - vp3 + 8) >> 4;
  }
  if (am1 && ap1) return (vm1 + vp1 + 1) >> 1;
  return vm1;
}

// Residual of predictor pid at an in-domain point (the origin keeps q).
__device__ __forceinline__ int32_t residual(const BlockView &b, int pid, int px, int py, int pz) {
  if ((px | py | pz) == 0) return b.at(0, 0, 0);
  switch (pid) {
    case 0: return res_lorenzo<1>(b, px, py, pz);
    case 1: return res_lorenzo<2>(b, px, py, pz);
    default: return (int32_t)((int64_t)b.at(px, py, pz) - interp_pred(b, pid == 3, px, py, pz));
  }
}

// ---------------------------------------------------------------- full-field interpolation
// Residual of the full-field multilevel interpolation (FZMod-Quality's
// G-Interp, §3.3) at a non-origin point of a block: the level s and pass axis
// come from the point's coordinates in its block (block origins are
// multiples of 8, so these are its field coordinates mod 8), and the
// neighbours p +- s, p +- 3s along the axis are available anywhere in the
// domain.  Their q comes from the shared tile when they lie in it, else from
// the input, prequantized here (the same q the tile would hold).
struct GiTile {
  const float *x;
  const int32_t *sq;       // the tile's q, row (y + 8 z), column x (kTXP per row)
  uint32_t x0, y0, z0;     // tile origin in the field
  uint32_t nx, ny, nz;
  float inv2eb, ebx2, eb_chk;
  __device__ __forceinline__ int32_t q(uint32_t X, uint32_t Y, uint32_t Z) const {
    const uint32_t tx = X - x0, ty = Y - y0, tz = Z - z0;  // below the tile wraps to large
    if (tx < (uint32_t)kTX && ty < 8u && tz < 8u) return sq[(ty + 8 * tz) * kTXP + tx];
    bool e;
    return prequant(__ldg(x + ((uint64_t)Z * ny + Y) * nx + X), inv2eb, ebx2, eb_chk, e);
  }
};

__device__ __forceinline__ int32_t gi_residual(const GiTile &t, int px, int py, int pz, uint32_t X, uint32_t Y,
                                               uint32_t Z) {
  int s, a;
  level_axis(px, py, pz, s, a);
  const uint32_t c = a == 0 ? X : (a == 1 ? Y : Z), m = a == 0 ? t.nx : (a == 1 ? t.ny : t.nz);
  const int sx = a == 0 ? s : 0, sy = a == 1 ? s : 0, sz = a == 2 ? s : 0;
  auto at = [&](int k) { return (int64_t)t.q(X + k * sx, Y + k * sy, Z + k * sz); };
  const int64_t qm1 = at(-1);
  int64_t pred;
  if (c >= 3u * s && c + 3u * s < m) pred = (-at(-3) + 9 * qm1 + 9 * at(1) - at(3) + 8) >> 4;
  else if (c + (uint32_t)s < m) pred = (qm1 + at(1) + 1) >> 1;
  else pred = qm1;
  return (int32_t)(at(0) - pred);
}

__device__ __forceinline__ uint32_t trial_bits(int32_t d, uint32_t R) {
  const uint32_t a = (uint32_t)(d < 0 ? -d : d);
  if (a >= R) return 96u;
  return 1u + 2u * (31u - (uint32_t)__clz((int)(a + 1)));
}

// ---------------------------------------------------------------- full blocks
// A block wholly inside the domain whose far corners o + 8 {0,1}^3 are all in
// the domain (every block except those on the field's upper faces).  Lane l
// holds the 16 points p = 32 i + l: px = l & 7, py = (l >> 3) + 4 (i & 1),
// pz = i >> 1.  The Lorenzo residuals come from registers by successive
// differences with zero padding -- (1 - S_x)(1 - S_y)(1 - S_z), applied once
// for order 1 and twice for order 2 -- instead of 8 or 27 shared-memory
// reads per point.

__device__ __forceinline__ bool full_block(const BlockView &b) {
  return b.xlim == 8 && b.ylim == 8 && b.zlim == 8 && (b.cin & 0xffu) == 0xffu;
}

__device__ __forceinline__ void fb_load(const BlockView &b, int32_t (&a)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = b.at(lane & 7, (lane >> 3) + 4 * (i & 1), i >> 1);
}

// One application of (1 - S_x)(1 - S_y)(1 - S_z), zero padding, in place.
__device__ __forceinline__ void fb_lorenzo(int32_t (&a)[16]) {
  const int lane = threadIdx.x & 31;
  const bool xin = (lane & 7) != 0, yin = lane >= 8;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int32_t l = __shfl_up_sync(0xffffffffu, a[i], 1);
    a[i] -= xin ? l : 0;
  }
  // the row below: lane - 8, or for row 4 (odd i, lanes 0-7) row 3 of the same
  // plane (lane + 24, i - 1); descending i reads every row before its own step
#pragma unroll
  for (int i = 15; i >= 0; --i) {
    const int32_t up = __shfl_up_sync(0xffffffffu, a[i], 8);
    const int32_t wrap = (i & 1) ? __shfl_down_sync(0xffffffffu, a[i - 1], 24) : 0;
    a[i] -= yin ? up : wrap;
  }
#pragma unroll
  for (int i = 15; i >= 2; --i) a[i] -= a[i - 2];  // the plane below, before its own z step
}

// The interpolation stencil of every non-origin point p of a full block
// (every in-block point is available, and a neighbour at coordinate 8 on the
// pass axis is the corner anchor o + 8 e_a when the other two coordinates
// are 0), one 16-byte entry per p, built once per CTA:
//   x, y: the shared-tile offsets (relative to p, int16 pairs) of p - s, p + s
//         and of p - 3s, p + 3s along the pass axis;
//   z:    bits 0-1 the form with the cubic predictor (0: q[-s], 1: linear,
//         2: cubic; the linear predictor takes at most 1), bit 8 / bit 9:
//         p + s / p + 3s is the corner anchor, bits 16+: its index 1 << a.
__device__ void build_interp_table(uint4 *tab) {
  for (int p = threadIdx.x; p < 512; p += blockDim.x) {
    const int px = p & 7, py = (p >> 3) & 7, pz = p >> 6;
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    if (p != 0) {
      int s, a;
      level_axis(px, py, pz, s, a);
      const int c = a == 0 ? px : (a == 1 ? py : pz);
      const bool on_axis = (a == 0 ? (py | pz) : (a == 1 ? (px | pz) : (px | py))) == 0;
      const int d = a == 0 ? 1 : (a == 1 ? kTXP : 8 * kTXP);
      const bool ap1 = c + s < 8 || on_axis;  // c + s <= 8 at every level
      const bool am3 = c - 3 * s >= 0, ap3 = c + 3 * s < 8 || (c + 3 * s == 8 && on_axis);
      const uint32_t form = (am3 && ap1 && ap3) ? 2u : (ap1 ? 1u : 0u);
      auto pk = [](int lo, int hi) { return (uint32_t)(uint16_t)(int16_t)lo | ((uint32_t)(uint16_t)(int16_t)hi << 16); };
      e.x = pk(-s * d, s * d);
      e.y = pk(-3 * s * d, 3 * s * d);
      e.z = form | (c + s == 8 ? 0x100u : 0u) | (c + 3 * s == 8 ? 0x200u : 0u) | ((uint32_t)(1 << a) << 16);
    }
    tab[p] = e;
  }
}

// Interpolation residual at a non-origin point of a full block, from its
// stencil entry.
__device__ __forceinline__ int32_t fb_interp(const BlockView &b, bool cubic, int px, int py, int pz) {
  const uint4 e = b.itab[px + 8 * py + 64 * pz];
  const int idx = (py + 8 * pz) * kTXP + 8 * b.wb + px;
  const int32_t q = b.sq[idx];
  const uint32_t form = e.z & 3u;
  const int32_t vm1 = b.sq[idx + (int16_t)(e.x & 0xffffu)];  // c - s >= 0 at every level
  if (form == 0) return q - vm1;
  const int32_t vp1 = (e.z & 0x100u) ? b.cq[e.z >> 16] : b.sq[idx + (int16_t)(e.x >> 16)];
  if (cubic && form == 2) {
    const int32_t vm3 = b.sq[idx + (int16_t)(e.y & 0xffffu)];
    const int32_t vp3 = (e.z & 0x200u) ? b.cq[e.z >> 16] : b.sq[idx + (int16_t)(e.y >> 16)];
    return q - ((-vm3 + 9 * vm1 + 9 * vp1 - vp3 + 8) >> 4);
  }
  return q - ((vm1 + vp1 + 1) >> 1);
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ unsigned long long warp_max64(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  return v;
}
__device__ __forceinline__ long long warp_min_s64(long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o < v ? o : v;
  }
  return v;
}
__device__ __forceinline__ long long warp_max_s64(long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const long long o = __shfl_xor_sync(0xffffffffu, v, off);
    v = o > v ? o : v;
  }
  return v;
}
__device__ __forceinline__ unsigned long long uabs64(long long v) {
  return (unsigned long long)(v < 0 ? -v : v);
}

// Trial costs of the four predictors (every lane gets all four).
__device__ void block_costs(const BlockView &b, uint32_t R, uint32_t cost[kNPred]) {
  const int lane = threadIdx.x & 31;
  if (full_block(b)) {
    int32_t a[16];
    fb_load(b, a);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      fb_lorenzo(a);  // order 1, then order 2
      uint32_t c = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) c += (i == 0 && lane == 0) ? 0u : trial_bits(a[i], R);
      cost[k] = (uint32_t)warp_sum64(c);
    }
#pragma unroll
    for (int k = 2; k < kNPred; ++k) {
      uint32_t c = 0;
      for (int i = 0; i < 16; ++i) {
        const int p = 32 * i + lane;
        if (p == 0) continue;
        c += trial_bits(fb_interp(b, k == 3, p & 7, (p >> 3) & 7, p >> 6), R);
      }
      cost[k] = (uint32_t)warp_sum64(c);
    }
    return;
  }
#pragma unroll
  for (int k = 0; k < kNPred; ++k) {
    uint32_t c = 0;
    for (int i = 0; i < 16; ++i) {
      const int p = 32 * i + lane;
      const int px = p & 7, py = (p >> 3) & 7, pz = p >> 6;
      if (p == 0 || !b.in(px, py, pz)) continue;
      c += trial_bits(residual(b, k, px, py, pz), R);
    }
    cost[k] = (uint32_t)warp_sum64(c);
  }
}

__device__ __forceinline__ float log2fix(unsigned long long s) {
  const unsigned long long v = s + 1;
  const int e = 63 - __clzll((long long)v);
  const unsigned long long m = e >= 4 ? (v >> (e - 4)) & 15ull : (v << (4 - e)) & 15ull;
  return __fadd_rn((float)e, (float)m * 0.0625f);
}

__device__ __forceinline__ uint32_t uabs32(int32_t v) { return (uint32_t)(v < 0 ? -v : v); }

// Sum over the warp of 32 per-lane values at once: lane f ends with the sum
// of everyone's v[f].  Five exchange steps; in each a lane keeps half of
// its values, sends the other half to its partner and adds what it gets.
__device__ __forceinline__ unsigned long long warp_transpose_sum(const uint32_t (&v)[32]) {
  const int lane = threadIdx.x & 31;
  unsigned long long w[16];
  {
    const bool up = (lane & 16) != 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const uint32_t send = up ? v[k] : v[k + 16], keep = up ? v[k + 16] : v[k];
      w[k] = (unsigned long long)keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
#pragma unroll
  for (int half = 8; half >= 1; half >>= 1) {
    const bool up = (lane & half) != 0;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const unsigned long long send = up ? w[k] : w[k + half], keep = up ? w[k + half] : w[k];
      w[k] = keep + __shfl_xor_sync(0xffffffffu, send, half);
    }
  }
  return w[0];
}

// The 32 statistics of a full block (every point in the domain, every
// corner available), the same integers as the general path below: the block
// is held in registers in the full-block layout (lane: x = lane & 7, rows
// y0 = lane >> 3 and y0 + 4; register i: y = y0 + 4 (i & 1), z = i >> 1),
// neighbours along x come by shuffles within the row's 8 lanes, along y by
// shuffles from the lanes 8, 16, 24 apart (or, for the upper rows, from the
// register of the lower row), along z from the registers two, four and six
// back.  Per-lane sums stay in 32 bits (|q| < 2^23: 16 third differences stay
// below 2^30); the warp sums are exact 64-bit sums.
__device__ uint16_t fb_features(const BlockView &b, uint32_t R) {
  const int lane = threadIdx.x & 31;
  const int px = lane & 7, y0 = lane >> 3;
  int32_t a[16];
  fb_load(b, a);
  uint32_t v[32];
#pragma unroll
  for (int f = 0; f < 32; ++f) v[f] = 0;
  uint32_t mx[4] = {0, 0, 0, 0};
  // predictor residuals on the all-odd points (two per lane)
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int o = lane + 32 * h;
    const int ox = 2 * (o & 3) + 1, oy = 2 * ((o >> 2) & 3) + 1, oz = 2 * (o >> 4) + 1;
    const uint32_t r[4] = {uabs32(res_lorenzo<1>(b, ox, oy, oz)), uabs32(res_lorenzo<2>(b, ox, oy, oz)),
                           uabs32(fb_interp(b, false, ox, oy, oz)), uabs32(fb_interp(b, true, ox, oy, oz))};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[2 * k] += r[k];
      mx[k] = r[k] > mx[k] ? r[k] : mx[k];
    }
    v[25] += r[0] >= R ? 1u : 0u;
  }
  int32_t qmin = a[0], qmax = a[0], qsum = 0;  // 16 values below 2^23: the sum fits
  int32_t qx1[16], qy1[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int py = y0 + 4 * (i & 1), pz = i >> 1;
    const int32_t q = a[i];
    qsum += q;
    qmin = q < qmin ? q : qmin;
    qmax = q > qmax ? q : qmax;
    // neighbours along x (lanes 1, 2, 3 back in the same row)
    const int32_t x1 = __shfl_up_sync(0xffffffffu, q, 1), x2 = __shfl_up_sync(0xffffffffu, q, 2),
                  x3 = __shfl_up_sync(0xffffffffu, q, 3);
    // along y: rows y - 1, y - 2, y - 3
    const int32_t u8 = __shfl_up_sync(0xffffffffu, q, 8), u16 = __shfl_up_sync(0xffffffffu, q, 16),
                  u24 = __shfl_up_sync(0xffffffffu, q, 24);
    int32_t y1 = u8, y2 = u16, y3 = u24;
    if (i & 1) {  // upper row: rows below 4 are the lower row's register of the lanes 24, 16, 8 ahead
      const int32_t d24 = __shfl_down_sync(0xffffffffu, a[i - 1], 24), d16 = __shfl_down_sync(0xffffffffu, a[i - 1], 16),
                    d8 = __shfl_down_sync(0xffffffffu, a[i - 1], 8);
      y1 = y0 >= 1 ? u8 : d24;
      y2 = y0 >= 2 ? u16 : d16;
      y3 = y0 >= 3 ? u24 : d8;
    }
    qx1[i] = x1;
    qy1[i] = y1;
    const int32_t z1 = i >= 2 ? a[i - 2] : 0, z2 = i >= 4 ? a[i - 4] : 0, z3 = i >= 6 ? a[i - 6] : 0;
    const int32_t n1[3] = {x1, y1, z1}, n2[3] = {x2, y2, z2}, n3[3] = {x3, y3, z3};
    const int c[3] = {px, py, pz};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      if (c[ax] >= 1) {
        const int32_t d1 = q - n1[ax];
        v[8 + ax] += uabs32(d1);
        if (c[ax] >= 2) {
          const int32_t d1p = n1[ax] - n2[ax];
          v[11 + ax] += uabs32(d1 - d1p);
          v[20 + ax] += ((d1 > 0 && d1p < 0) || (d1 < 0 && d1p > 0)) ? 1u : 0u;
          if (c[ax] >= 3) v[14 + ax] += uabs32(d1 - 2 * d1p + (n2[ax] - n3[ax]));
        }
      }
    }
    // mixed differences: (x, y) with the x-neighbour's y-neighbour, (x, z)
    // and (y, z) with the plane below's neighbours
    const int32_t xy = __shfl_up_sync(0xffffffffu, y1, 1);
    if (px >= 1 && py >= 1) v[17] += uabs32(q - x1 - y1 + xy);
    if (px >= 1 && pz >= 1) v[18] += uabs32(q - x1 - z1 + qx1[i >= 2 ? i - 2 : 0]);
    if (py >= 1 && pz >= 1) v[19] += uabs32(q - y1 - z1 + qy1[i >= 2 ? i - 2 : 0]);
    if (px >= 2) v[31] += uabs32(q - x2);
  }
  // the block sum needs 64 bits: 32 lane sums below 2^27 each
  long long tsum = (long long)qsum;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, off);
  const long long mean = tsum >> 9;  // floor(sum / 512)
#pragma unroll
  for (int i = 0; i < 16; ++i) v[23] += (uint32_t)((long long)a[i] >= mean ? (long long)a[i] - mean : mean - (long long)a[i]);
  unsigned long long st = warp_transpose_sum(v);
  // maxima, spread and the constant statistics of a full block
  const uint32_t m0 = __reduce_max_sync(0xffffffffu, mx[0]), m1 = __reduce_max_sync(0xffffffffu, mx[1]),
                 m2 = __reduce_max_sync(0xffffffffu, mx[2]), m3 = __reduce_max_sync(0xffffffffu, mx[3]);
  const int32_t gmax = __reduce_max_sync(0xffffffffu, qmax), gmin = __reduce_min_sync(0xffffffffu, qmin);
  if (lane == 1) st = m0;
  if (lane == 3) st = m1;
  if (lane == 5) st = m2;
  if (lane == 7) st = m3;
  if (lane == 24) st = (unsigned long long)((long long)gmax - (long long)gmin);
  if (lane >= 26 && lane <= 28) st = 1;  // the +x, +y, +z corners
  if (lane == 29) st = 512;
  if (lane == 30) st = uabs32(b.at(0, 0, 0));
  return f32_to_bf16_rne(log2fix(st));
}

// The 32 block statistics (see the selector's definition: sums and maxima
// of predictor residuals on the 64 all-odd points, difference sums, sign
// changes, spread, corner availability, size, anchor) -> bfloat16 features.
// Returns this lane's feature (lane f holds feature f).
__device__ uint16_t block_feature(const BlockView &b, uint32_t R) {
  if (full_block(b)) return fb_features(b, R);
  const int lane = threadIdx.x & 31;
  unsigned long long st[kNFeat];
#pragma unroll
  for (int f = 0; f < kNFeat; ++f) st[f] = 0;
  // predictor residuals on the odd sub-lattice: points lane and lane + 32
#pragma unroll
  for (int k = 0; k < kNPred; ++k) {
    unsigned long long sum = 0, mx = 0, outl = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int o = lane + 32 * h;
      const int px = 2 * (o & 3) + 1, py = 2 * ((o >> 2) & 3) + 1, pz = 2 * (o >> 4) + 1;
      if (!b.in(px, py, pz)) continue;
      const unsigned long long a = uabs64(residual(b, k, px, py, pz));
      sum += a;
      mx = a > mx ? a : mx;
      outl += a >= R ? 1 : 0;
    }
    st[2 * k] = warp_sum64(sum);
    st[2 * k + 1] = warp_max64(mx);
    if (k == 0) st[25] = warp_sum64(outl);
  }
  long long qsum = 0, qmn = 0x7fffffffffffffffll, qmx = -0x7fffffffffffffffll - 1;
  unsigned long long n = 0;
  unsigned long long d1[3] = {0, 0, 0}, d2[3] = {0, 0, 0}, d3[3] = {0, 0, 0}, mix[3] = {0, 0, 0}, sc[3] = {0, 0, 0};
  unsigned long long x2 = 0;
  for (int i = 0; i < 16; ++i) {
    const int p = 32 * i + lane;
    const int c[3] = {p & 7, (p >> 3) & 7, p >> 6};
    if (!b.in(c[0], c[1], c[2])) continue;
    const long long q = b.at(c[0], c[1], c[2]);
    qsum += q;
    qmn = q < qmn ? q : qmn;
    qmx = q > qmx ? q : qmx;
    ++n;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int e[3] = {0, 0, 0};
      e[a] = 1;
      if (c[a] >= 1) {
        const long long q1 = b.at(c[0] - e[0], c[1] - e[1], c[2] - e[2]);
        const long long dd1 = q - q1;
        d1[a] += uabs64(dd1);
        if (c[a] >= 2) {
          const long long q2 = b.at(c[0] - 2 * e[0], c[1] - 2 * e[1], c[2] - 2 * e[2]);
          const long long dd1p = q1 - q2;
          d2[a] += uabs64(dd1 - dd1p);
          sc[a] += ((dd1 > 0 && dd1p < 0) || (dd1 < 0 && dd1p > 0)) ? 1 : 0;
          if (c[a] >= 3) {
            const long long q3 = b.at(c[0] - 3 * e[0], c[1] - 3 * e[1], c[2] - 3 * e[2]);
            d3[a] += uabs64(dd1 - 2 * dd1p + (q2 - q3));
          }
        }
      }
    }
    const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
#pragma unroll
    for (int pr = 0; pr < 3; ++pr) {
      const int a = pa[pr], bb = pb[pr];
      if (c[a] >= 1 && c[bb] >= 1) {
        int ea[3] = {0, 0, 0}, eb[3] = {0, 0, 0};
        ea[a] = 1;
        eb[bb] = 1;
        const long long m = q - b.at(c[0] - ea[0], c[1] - ea[1], c[2] - ea[2]) -
                            b.at(c[0] - eb[0], c[1] - eb[1], c[2] - eb[2]) +
                            b.at(c[0] - ea[0] - eb[0], c[1] - ea[1] - eb[1], c[2] - ea[2] - eb[2]);
        mix[pr] += uabs64(m);
      }
    }
    if (c[0] >= 2) x2 += uabs64(q - b.at(c[0] - 2, c[1], c[2]));
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    st[8 + a] = warp_sum64(d1[a]);
    st[11 + a] = warp_sum64(d2[a]);
    st[14 + a] = warp_sum64(d3[a]);
    st[17 + a] = warp_sum64(mix[a]);
    st[20 + a] = warp_sum64(sc[a]);
  }
  st[31] = warp_sum64(x2);
  const long long total = (long long)warp_sum64((unsigned long long)qsum);
  const long long nn = (long long)warp_sum64(n);
  long long mean = total / nn;
  if ((total % nn) != 0 && total < 0) mean -= 1;
  unsigned long long dev = 0;
  for (int i = 0; i < 16; ++i) {
    const int p = 32 * i + lane;
    const int px = p & 7, py = (p >> 3) & 7, pz = p >> 6;
    if (b.in(px, py, pz)) dev += uabs64((long long)b.at(px, py, pz) - mean);
  }
  st[23] = warp_sum64(dev);
  st[24] = (unsigned long long)(warp_max_s64(qmx) - warp_min_s64(qmn));
  st[26] = (b.cin >> 1) & 1u;
  st[27] = (b.cin >> 2) & 1u;
  st[28] = (b.cin >> 4) & 1u;
  st[29] = (unsigned long long)nn;
  st[30] = uabs64(b.at(0, 0, 0));
  unsigned long long mine = 0;
#pragma unroll
  for (int f = 0; f < kNFeat; ++f) mine = (lane == f) ? st[f] : mine;
  return f32_to_bf16_rne(log2fix(mine));
}

// The network's weights as the CTA keeps them in shared memory (binary32):
// the stream order, except W1 and W2 transposed (W1t[k][j], W2t[j][i]) so
// that the lanes of a warp, one per hidden unit or logit, read consecutive
// words (the stored order puts them a row apart: one shared-memory bank).
__device__ __forceinline__ int smem_weight_index(int i) {
  if (i < kOffB1) return kOffW1 + (i % kNFeat) * kNHid + i / kNFeat;              // W1[j][k] -> W1t[k][j]
  if (i >= kOffW2 && i < kOffB2) return kOffW2 + ((i - kOffW2) % kNHid) * kNPred + (i - kOffW2) / kNHid;
  return i;
}

// Exact network inference: lane l computes hidden units l and l + 32,
// lanes 0..3 the logits, each with fmaf in index order.  Returns the
// argmax (ties to the lowest id) in every lane.
__device__ int mlp_choose(const float *w, uint16_t feat_lane) {
  const int lane = threadIdx.x & 31;
  const float f = bf16_to_f32(feat_lane);
  float h[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int j = lane + 32 * u;
    float acc = w[kOffB1 + j];
#pragma unroll 8
    for (int k = 0; k < kNFeat; ++k) acc = __fmaf_rn(w[kOffW1 + k * kNHid + j], __shfl_sync(0xffffffffu, f, k), acc);
    acc = acc > 0.0f ? acc : 0.0f;
    h[u] = bf16_to_f32(f32_to_bf16_rne(acc));
  }
  float lg = 0.0f;
  {
    const int i = lane < kNPred ? lane : 0;
    float acc = w[kOffB2 + i];
    for (int j = 0; j < kNHid; ++j) {
      const float hj = __shfl_sync(0xffffffffu, h[j >> 5], j & 31);
      acc = __fmaf_rn(w[kOffW2 + j * kNPred + i], hj, acc);
    }
    lg = acc;
  }
  int best = 0;
  float bv = __shfl_sync(0xffffffffu, lg, 0);
#pragma unroll
  for (int i = 1; i < kNPred; ++i) {
    const float v = __shfl_sync(0xffffffffu, lg, i);
    if (v > bv) { bv = v; best = i; }
  }
  return best;
}

struct SelOut {
  uint8_t *labels;            // report mode: exhaustive label per block
  uint32_t *costs;            // report mode: 4 trial costs per block (may be null)
  uint16_t *feat;             // report mode: 32 bfloat16 features per block (may be null)
  const uint16_t *weights;    // network mode: bfloat16 weights
};

struct SelSmem {
  float4 stage[4][kSelThreads];  // the next tile's input, thread t's four 4-vectors (asynchronous copies)
  int32_t sq[kRows * kTXP];
  uint8_t sexc[kTileElems];
  uint32_t shist[kMaxSym];
  int32_t cq[8][8];
  uint32_t cin[8];
  float w[kNWeights];
  uint32_t wout[8], wexc[8];
  uint32_t oslot, eslot;
  int pid[8];
  uint4 itab[512];
};

// 16-byte asynchronous copy global -> shared; an invalid copy zero-fills
// and reads nothing.
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

// Issue the copies of tile tl's input that thread tid will prequantize: its
// four 4-vectors (row-major tile order, 4 values per thread per step), those
// wholly inside the domain; the others are loaded when they are used.
__device__ __forceinline__ void sel_issue_tile(const float *x, const Geom &g, uint64_t tl, bool vec_ok, int tid,
                                               float4 (&stage)[4][kSelThreads]) {
  if (!vec_ok || tl >= g.n_qtiles) return;
  const uint32_t t32 = (uint32_t)tl;
  const uint32_t tx = t32 % g.tiles_x, rest = t32 / g.tiles_x;
  const uint32_t x0 = tx * kTX, y0 = (rest % g.nby) * 8, z0 = (rest / g.nby) * 8;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int e = 4 * (tid + kSelThreads * j);
    const int row = e / kTX, col = e % kTX;
    const uint32_t X = x0 + col, Y = y0 + (row & 7), Z = z0 + (row >> 3);
    const bool ok = Y < g.ny && Z < g.nz && X + 4 <= g.nx;
    const uint64_t fi = ((uint64_t)Z * g.ny + Y) * g.nx + X;
    cp_async16(&stage[j][tid], ok ? x + fi : x, ok);
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

template <int MODE>
__global__ void __launch_bounds__(kSelThreads, (MODE == kSelNet || MODE == kSelReport) ? 2 : FZ_SEL_MINB) k_selquant(const float *__restrict__ x, Geom g, uint32_t R,
                                                           uint32_t fixed_pid, CompressWs ws, SelOut so) {
  extern __shared__ __align__(16) unsigned char sel_smem[];
  SelSmem &sm = *reinterpret_cast<SelSmem *>(sel_smem);
  Ctl *ctl = ws.ctl;
  if (ctl->mode != kModeNormal) return;
  const float inv2eb = ctl->inv2eb, ebx2 = ctl->ebx2, eb_chk = ctl->eb_chk;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool vec_ok = ((g.nx & 3u) == 0) && (((uintptr_t)x & 15u) == 0);
  for (int s = tid; s < kMaxSym; s += kSelThreads) sm.shist[s] = 0;
  build_interp_table(sm.itab);
  if (MODE == kSelNet)
    for (int i = tid; i < kNWeights; i += kSelThreads) sm.w[smem_weight_index(i)] = bf16_to_f32(so.weights[i]);
  __syncthreads();

  sel_issue_tile(x, g, blockIdx.x, vec_ok, tid, sm.stage);
  for (uint64_t tile = blockIdx.x; tile < g.n_qtiles; tile += gridDim.x) {
    const uint32_t t32 = (uint32_t)tile;
    const uint32_t tx = t32 % g.tiles_x, rest = t32 / g.tiles_x;
    const uint32_t by = rest % g.nby, bz = rest / g.nby;
    const uint32_t x0 = tx * kTX, y0 = by * 8, z0 = bz * 8;
    // ---- prequantize the tile (row-major, 4 values per thread per step) from
    // the copies issued a tile ahead; then the next tile's copies go out
    asm volatile("cp.async.wait_all;\n" ::: "memory");
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int e = 4 * (tid + kSelThreads * j);
      const int row = e / kTX, col = e % kTX;
      const uint32_t X = x0 + col, Y = y0 + (row & 7), Z = z0 + (row >> 3);
      const bool inrow = Y < g.ny && Z < g.nz;
      const uint64_t fi = ((uint64_t)Z * g.ny + Y) * g.nx + X;
      float xv[4];
      if (inrow && vec_ok && X + 4 <= g.nx) {
        const float4 f4 = sm.stage[j][tid];
        xv[0] = f4.x; xv[1] = f4.y; xv[2] = f4.z; xv[3] = f4.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) xv[u] = (inrow && X + u < g.nx) ? x[fi + u] : 0.0f;
      }
      uint32_t ex = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool in = inrow && X + u < g.nx;
        bool ee = false;
        const int32_t q = in ? prequant(xv[u], inv2eb, ebx2, eb_chk, ee) : 0;
        sm.sq[row * kTXP + col + u] = q;
        ex |= (uint32_t)(in && ee) << (8 * u);
      }
      *reinterpret_cast<uint32_t *>(&sm.sexc[e]) = ex;
    }
    sel_issue_tile(x, g, tile + gridDim.x, vec_ok, tid, sm.stage);
    // ---- corner anchors of every block: q at o + 8 (cx, cy, cz)
    {
      const int wb = warp, c = lane;
      if (c < 8) {
        const uint64_t X = (uint64_t)x0 + 8 * wb + 8 * (c & 1), Y = y0 + 8 * ((c >> 1) & 1), Z = z0 + 8 * (c >> 2);
        const bool in = X < g.nx && Y < g.ny && Z < g.nz;
        bool ee;
        sm.cq[wb][c] = in ? prequant(x[(Z * g.ny + Y) * g.nx + X], inv2eb, ebx2, eb_chk, ee) : 0;
        const uint32_t bits = __ballot_sync(0x000000ffu, in);
        if (c == 0) sm.cin[wb] = bits & 0xffu;
      }
    }
    __syncthreads();

    // ---- one warp per block: choose, then codes
    const int wb = warp;
    const uint32_t bxi = tx * 8 + wb;
    const bool bvalid = bxi < g.nbx;
    const uint64_t blk = (uint64_t)bxi + (uint64_t)g.nbx * (by + (uint64_t)g.nby * bz);
    BlockView b;
    b.sq = sm.sq;
    b.cq = sm.cq[wb];
    b.cin = sm.cin[wb];
    b.wb = wb;
    b.xlim = g.nx - x0 - 8 * wb < 8 ? g.nx - x0 - 8 * wb : 8;
    b.ylim = g.ny - y0 < 8 ? g.ny - y0 : 8;
    b.zlim = g.nz - z0 < 8 ? g.nz - z0 : 8;
    b.itab = sm.itab;
    GiTile gt;
    if (MODE == kSelGinterp) {
      gt.x = x;
      gt.sq = sm.sq;
      gt.x0 = x0;
      gt.y0 = y0;
      gt.z0 = z0;
      gt.nx = g.nx;
      gt.ny = g.ny;
      gt.nz = g.nz;
      gt.inv2eb = inv2eb;
      gt.ebx2 = ebx2;
      gt.eb_chk = eb_chk;
    }
    uint32_t nout = 0, nexc = 0;
    if (bvalid) {
      int pid = (int)fixed_pid;
      if (MODE == kSelExhaustive || MODE == kSelReport) {
        uint32_t cost[kNPred];
        block_costs(b, R, cost);
        pid = 0;
#pragma unroll
        for (int k = 1; k < kNPred; ++k)
          if (cost[k] < cost[pid]) pid = k;
        if (MODE == kSelReport) {
          if (lane == 0) so.labels[blk] = (uint8_t)pid;
          if (so.costs && lane < kNPred) so.costs[blk * kNPred + lane] = cost[lane];
        }
      }
      if (MODE == kSelNet || (MODE == kSelReport && so.feat)) {
        const uint16_t f = block_feature(b, R);
        if (MODE == kSelReport) so.feat[blk * kNFeat + lane] = f;
        else pid = mlp_choose(sm.w, f);
      }
      if (MODE != kSelReport) {
        if (lane == 0) { ws.ids[blk] = (uint8_t)pid; sm.pid[wb] = pid; }
        uint16_t *cdst = ws.codes + blk * 512;
        // full blocks: Lorenzo residuals from registers, interpolation without availability tests
        const bool full = full_block(b);
        const bool fl = pid <= 1 && full;
        int32_t ra[16];
        if (fl) {
          fb_load(b, ra);
          fb_lorenzo(ra);
          if (pid == 1) fb_lorenzo(ra);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int p = 32 * i + lane;
          const int px = p & 7, py = (p >> 3) & 7, pz = p >> 6;
          const bool in = b.in(px, py, pz);
          uint32_t code = R;
          if (!fl) ra[i] = 0;
          if (in) {
            int32_t d;
            if (MODE == kSelGinterp)
              d = p == 0 ? b.at(0, 0, 0) : gi_residual(gt, px, py, pz, gt.x0 + 8 * wb + px, y0 + py, z0 + pz);
            else
              d = fl ? ra[i] : (full && p != 0 ? fb_interp(b, pid == 3, px, py, pz) : residual(b, pid, px, py, pz));
            ra[i] = d;
            if (p == 0) ws.anchors[blk] = d;
            else {
              const uint32_t c = (uint32_t)(d + (int32_t)R);
              const bool o = (c - 1u) >= 2u * R - 1u;
              code = o ? 0u : c;
              nout += o;
            }
            nexc += sm.sexc[(py + 8 * pz) * kTX + 8 * wb + px] ? 1u : 0u;
          }
          cdst[p] = (uint16_t)code;
          atomicAdd(&sm.shist[code], 1u);
        }
        // the block's residuals replace its q in the shared tile (only this warp
        // reads them), for the outlier compaction below; the full-field
        // interpolation reads the q of neighbouring blocks in the tile, so it
        // keeps q and the compaction recomputes its residuals
        if (MODE != kSelGinterp) {
          __syncwarp();
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int p = 32 * i + lane;
            sm.sq[(((p >> 3) & 7) + 8 * (p >> 6)) * kTXP + 8 * wb + (p & 7)] = ra[i];
          }
        }
      }
    }
    if (MODE == kSelReport) {
      __syncthreads();
      continue;
    }
    // ---- ordered outliers / exceptions (warp = block, position order)
    nout = __reduce_add_sync(0xffffffffu, nout);
    nexc = __reduce_add_sync(0xffffffffu, nexc);
    if (lane == 0) { sm.wout[warp] = nout; sm.wexc[warp] = nexc; }
    if (__syncthreads_or((nout | nexc) != 0)) {
      if (tid == 0) {
        uint32_t to = 0, te = 0;
        for (int w = 0; w < 8; ++w) { to += sm.wout[w]; te += sm.wexc[w]; }
        const unsigned long long os = to ? atomicAdd(&ctl->n_out, (unsigned long long)to) : 0ull;
        const unsigned long long es = te ? atomicAdd(&ctl->n_exc, (unsigned long long)te) : 0ull;
        ws.tinfo[tile] = make_uint4(to, te, (uint32_t)os, (uint32_t)es);
        const uint64_t grp = tile / kTileGroup;
        if (to) atomicAdd(&ws.tgroup[grp].x, to);
        if (te) atomicAdd(&ws.tgroup[grp].y, te);
        sm.oslot = (uint32_t)os;
        sm.eslot = (uint32_t)es;
      }
      __syncthreads();
      uint32_t oo = sm.oslot, eo = sm.eslot;
      for (int w = 0; w < warp; ++w) { oo += sm.wout[w]; eo += sm.wexc[w]; }
      if (lane == 0) {  // one slice per warp (= block), in warp order
        WarpSlots wsl;
        wsl.oslot = oo;
        wsl.eslot = eo;
        wsl.ocnt = sm.wout[warp];
        wsl.ecnt = sm.wexc[warp];
        ws.winfo[tile * 8 + warp] = wsl;
      }
      if (bvalid && (nout | nexc)) {
        for (int i = 0; i < 16; ++i) {
          const int p = 32 * i + lane;
          const int px = p & 7, py = (p >> 3) & 7, pz = p >> 6;
          const bool in = b.in(px, py, pz);
          const uint32_t pos = (uint32_t)(blk * 512 + p);
          int32_t d = 0;
          bool outl = false;
          if (in && p != 0) {
            if (MODE == kSelGinterp) d = gi_residual(gt, px, py, pz, gt.x0 + 8 * wb + px, y0 + py, z0 + pz);
            else d = b.at(px, py, pz);  // the residual, stored by the code pass
            const uint32_t c = (uint32_t)(d + (int32_t)R);
            outl = (c - 1u) >= 2u * R - 1u;
          }
          uint32_t m = __ballot_sync(0xffffffffu, outl);
          if (outl) {
            const uint64_t o = (uint64_t)oo + __popc(m & ((1u << lane) - 1));
            if (o < ws.cap_list) { ws.out_idx[o] = pos; ws.out_val[o] = d; }
          }
          oo += __popc(m);
          const bool e = in && sm.sexc[(py + 8 * pz) * kTX + 8 * wb + px];
          m = __ballot_sync(0xffffffffu, e);
          if (e) {
            const uint64_t o = (uint64_t)eo + __popc(m & ((1u << lane) - 1));
            const uint64_t fi = ((uint64_t)(z0 + pz) * g.ny + (y0 + py)) * g.nx + (x0 + 8 * wb + px);
            if (o < ws.cap_list) { ws.exc_idx[o] = pos; ws.exc_val[o] = __float_as_uint(x[fi]); }
          }
          eo += __popc(m);
        }
      }
    }
    __syncthreads();
  }
  for (int s = tid; s < (int)(2 * R); s += kSelThreads)
    if (sm.shist[s]) atomicAdd(&ctl->hist[s], (unsigned long long)sm.shist[s]);
}

template <int MODE>
cudaError_t launch_sel_t(const float *x, const Geom &g, uint32_t R, uint32_t pid, const CompressWs &ws,
                         const SelOut &so, cudaStream_t s, int sms) {
  const int smem = (int)sizeof(SelSmem);
  static LaunchCache cache;
  int per_sm = 0;
  const cudaError_t e = cached_per_sm(k_selquant<MODE>, kSelThreads, smem, cache, per_sm);
  if (e != cudaSuccess) return e;
  uint64_t grid = (uint64_t)sms * per_sm;
  if (grid > g.n_qtiles) grid = g.n_qtiles;
  k_selquant<MODE><<<(unsigned)grid, kSelThreads, smem, s>>>(x, g, R, pid, ws, so);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- decoding
struct SelDecParams {
  const uint32_t *words;
  uint64_t n_words;
  const uint32_t *chunk_bits;
  const uint64_t *goff;     // per work unit: first bit
  uint64_t n_chunks, n_units;
  const uint16_t *lut;
  uint16_t *codes;
  uint32_t *err;            // err[0] error word, err[1] work-unit counter
  // optional (OV): the residual of every outlier written at its position
  const uint32_t *ofirst;   // per block with outliers: index of its first outlier (others ~0)
  const uint32_t *out_idx;
  const int32_t *out_val;
  uint64_t n_out;
  int32_t *ovals;
};

__device__ __forceinline__ void sel_err(uint32_t *err, uint32_t code) { atomicCAS(err, 0u, code); }

// threads of the code decoder's CTA (one per SM): 864 and 576 give the 512^3
// field's 8192 work units a whole number of rounds per warp (2 and 3);
// measured 872 / 875 / 904 us for 864 / 576 / 768 on its interpolation decode
#ifndef FZ_SELDEC_T
#define FZ_SELDEC_T 864
#endif
constexpr int kSelDecThreads = FZ_SELDEC_T;

// Phase 1: one thread per chunk (= block), codes written row by row; warps
// take work units of 32 chunks from a counter.
// With OV, the r-th outlier code (0) of a block takes entry r of the
// block's run of the outlier list (from the block's first entry on) and
// its residual goes to ovals at the code's position; the outlier codes are
// counted in err[3].  The list is checked elsewhere to ascend strictly and
// to name only outlier codes; with as many entries as outlier codes, it is
// then exactly the outlier codes in order, and every match made here is
// right.
template <bool OV>
__global__ void __launch_bounds__(kSelDecThreads, 1) k_dec_codes(SelDecParams p) {
  constexpr int T = kSelDecThreads;
  extern __shared__ __align__(16) unsigned char dc_smem[];
  uint16_t *slut = reinterpret_cast<uint16_t *>(dc_smem);
  uint32_t *sring = reinterpret_cast<uint32_t *>(dc_smem + sizeof(uint16_t) * kLutSize);
  const int t = threadIdx.x;
  {
    const uint4 *src = reinterpret_cast<const uint4 *>(p.lut);
    uint4 *dst = reinterpret_cast<uint4 *>(slut);
    for (int i = t; i < kLutSize / 8; i += T) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  for (;;) {
    const uint32_t u = claim_unit(p.err + 1);
    if (u >= p.n_units) break;
    uint32_t cb;
    const uint64_t start = unit_start(p.chunk_bits, p.goff, p.n_chunks, u, cb);
    const uint64_t j = (uint64_t)u * kDecUnit + (t & 31);
    if (j >= p.n_chunks) continue;
    BitReader<T> br;
    br.init(p.words, p.n_words, start, cb, sring + t);
    const uint32_t start_off = br.off;
    uint4 *dst = reinterpret_cast<uint4 *>(p.codes + j * 512);
    uint64_t oc = ~0ull;  // next outlier entry of this block (located at its first outlier)
    uint32_t nzero = 0;
    bool bad = false;
    // sixteen codes (two rows) per step, four codewords per window read; the
    // lane's 32 bytes are stored back to back (one whole sector)
#pragma unroll 1
    for (int r = 0; r < 64; r += 2) {
      uint32_t c[16];
#pragma unroll
      for (int u4 = 0; u4 < 4; ++u4) {
        int32_t s4[4];
        br.next4(slut, s4);  // a table of offset 0: the codes themselves
#pragma unroll
        for (int k = 0; k < 4; ++k) c[4 * u4 + k] = (uint32_t)s4[k];
      }
      dst[r] = make_uint4(c[0] | (c[1] << 16), c[2] | (c[3] << 16), c[4] | (c[5] << 16), c[6] | (c[7] << 16));
      dst[r + 1] =
          make_uint4(c[8] | (c[9] << 16), c[10] | (c[11] << 16), c[12] | (c[13] << 16), c[14] | (c[15] << 16));
      if (OV) {
        bool z = false;
#pragma unroll
        for (int k = 0; k < 16; ++k) z = z || c[k] == 0;
        if (z) {
          if (oc == ~0ull) oc = __ldg(p.ofirst + j);  // ~0 for a block without outliers: out of the list
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            if (c[k] != 0) continue;
            if (oc < p.n_out) p.ovals[j * 512u + (uint64_t)(8 * r + k)] = __ldg(p.out_val + oc);
            else bad = true;
            ++oc;
            ++nzero;
          }
        }
      }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (OV && nzero) atomicAdd(p.err + 3, nzero);
    if (br.consumed(start_off) != cb || bad) sel_err(p.err, FZ_ECORRUPT);
  }
}

struct ReconParams {
  const uint16_t *codes;
  const int32_t *anchors;
  const uint8_t *ids;       // packed 2-bit ids, or null for a fixed predictor
  uint32_t fixed_pid;
  const uint32_t *out_idx;
  const int32_t *out_val;
  const uint32_t *exc_idx;
  const uint32_t *exc_val;
  uint64_t n_out, n_exc;
  const uint32_t *ofirst;     // per block with outliers: index of its first outlier (others ~0); n_out > 0
  float *out;
  float ebx2;
  int32_t R;
  uint32_t *err;
};

__device__ __forceinline__ uint64_t lb_u32(const uint32_t *a, uint64_t n, uint32_t key) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (__ldg(a + mid) < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

constexpr int kReconWarps = 8;

// Phase 2: one warp per block.  The block's q is rebuilt in shared memory.
// First point of each interpolation pass (levels 4, 2, 1; axes x, y, z) in
// the pass-ordered point list: a pass of level s along axis a holds
// (8 / 2s) (8 / s)^a (8 / 2s)^(2 - a) points.
__constant__ uint16_t kPassStart[10] = {0, 1, 3, 7, 15, 31, 63, 127, 255, 511};

// The pass-ordered point list of an 8x8x8 block (each pass's points in
// raster order: slot = the pass's start + the point's rank on the pass's
// lattice) and every non-origin point's stencil in the block layout (the
// entry format of build_interp_table, offsets with strides 1, 8, 64).
__device__ void build_recon_tables(uint16_t *list, uint4 *tab) {
  for (int p = threadIdx.x; p < 512; p += blockDim.x) {
    const int c[3] = {p & 7, (p >> 3) & 7, p >> 6};
    uint4 e = make_uint4(0u, 0u, 0u, 0u);
    if (p != 0) {
      int s, a;
      level_axis(c[0], c[1], c[2], s, a);
      const bool on_axis = (a == 0 ? (c[1] | c[2]) : (a == 1 ? (c[0] | c[2]) : (c[0] | c[1]))) == 0;
      const int d = a == 0 ? 1 : (a == 1 ? 8 : 64);
      const int ca = c[a];
      const bool ap1 = ca + s < 8 || on_axis;
      const bool am3 = ca - 3 * s >= 0, ap3 = ca + 3 * s < 8 || (ca + 3 * s == 8 && on_axis);
      const uint32_t form = (am3 && ap1 && ap3) ? 2u : (ap1 ? 1u : 0u);
      auto pk = [](int lo, int hi) { return (uint32_t)(uint16_t)(int16_t)lo | ((uint32_t)(uint16_t)(int16_t)hi << 16); };
      e.x = pk(-s * d, s * d);
      e.y = pk(-3 * s * d, 3 * s * d);
      e.z = form | (ca + s == 8 ? 0x100u : 0u) | (ca + 3 * s == 8 ? 0x200u : 0u) | ((uint32_t)(1 << a) << 16);
      // rank on the pass's lattice: per axis the coordinate's index and count
      int rank = 0;
      for (int b = 2; b >= 0; --b) {
        const int step = b == a ? 2 * s : (b < a ? s : 2 * s), first = b == a ? s : 0;
        rank = rank * (8 / step) + (c[b] - first) / step;
      }
      const int li = s == 4 ? 0 : (s == 2 ? 1 : 2);
      list[kPassStart[3 * li + a] + rank] = (uint16_t)p;
    }
    tab[p] = e;
  }
}

__global__ void __launch_bounds__(kReconWarps * 32, 4) k_sel_recon(ReconParams rp, Geom g) {
  __shared__ __align__(16) int32_t sq[kReconWarps][512];
  __shared__ int32_t scq[kReconWarps][8];
  __shared__ uint32_t sov[kReconWarps][512];
  __shared__ uint32_t smask[kReconWarps][16];
  __shared__ uint16_t rlist[512];
  __shared__ uint4 rtab[512];
  build_recon_tables(rlist, rtab);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t nwarps = (uint64_t)gridDim.x * kReconWarps;
  for (uint64_t blk = (uint64_t)blockIdx.x * kReconWarps + w; blk < g.n_blocks; blk += nwarps) {
    const uint32_t bxi = (uint32_t)(blk % g.nbx);
    const uint64_t br_ = blk / g.nbx;
    const uint32_t byi = (uint32_t)(br_ % g.nby), bzi = (uint32_t)(br_ / g.nby);
    const uint32_t X0 = 8 * bxi, Y0 = 8 * byi, Z0 = 8 * bzi;
    const uint32_t xl = g.nx - X0 < 8 ? g.nx - X0 : 8, yl = g.ny - Y0 < 8 ? g.ny - Y0 : 8,
                   zl = g.nz - Z0 < 8 ? g.nz - Z0 : 8;
    const uint32_t pos0 = (uint32_t)(blk * 512);
    const int pid = rp.ids ? (rp.ids[blk >> 2] >> (2 * (blk & 3))) & 3 : (int)rp.fixed_pid;
    // corner anchors (origins of the neighbouring blocks)
    uint32_t cin = 0;
    if (lane < 8) {
      const uint64_t cx = bxi + (lane & 1), cy = byi + ((lane >> 1) & 1), cz = bzi + (lane >> 2);
      const bool in = cx < g.nbx && cy < g.nby && cz < g.nbz;
      scq[w][lane] = in ? __ldg(rp.anchors + (cz * g.nby + cy) * g.nbx + cx) : 0;
    }
    {
      const uint64_t cx = bxi + (lane & 1), cy = byi + ((lane >> 1) & 1), cz = bzi + ((lane >> 2) & 1);
      cin = __ballot_sync(0xffffffffu, lane < 8 && cx < g.nbx && cy < g.nby && cz < g.nbz) & 0xffu;
    }
    // residuals, with outliers scattered in position order
    // the block's first outlier from the per-block table (~0: none, so an
    // outlier code there finds no entry and is reported)
    uint64_t obase = 0;
    if (rp.n_out) obase = __ldg(rp.ofirst + blk);
    bool bad = false;
    {
      // lane l: the block's codes 16 l .. 16 l + 15, two 16-byte loads (the
      // code buffer holds whole blocks at 1 KB boundaries)
      const uint4 *cp = reinterpret_cast<const uint4 *>(rp.codes + pos0) + 2 * lane;
      const uint4 c0 = __ldg(cp), c1 = __ldg(cp + 1);
      const uint32_t cw[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
      int32_t dv[16];
      uint32_t nz = 0;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const uint32_t code = (cw[k >> 1] >> (16 * (k & 1))) & 0xffffu;
        dv[k] = (int32_t)code - rp.R;
        nz += code == 0 ? 1u : 0u;
      }
      if (__any_sync(0xffffffffu, nz != 0)) {
        // outliers in position order: the lanes' zero counts scanned
        uint32_t incl = nz;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
          if (lane >= off) incl += v;
        }
        uint64_t k = obase + (incl - nz);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          if (((cw[kk >> 1] >> (16 * (kk & 1))) & 0xffffu) == 0) {
            const uint32_t pos = pos0 + 16u * (uint32_t)lane + (uint32_t)kk;
            int32_t d = 0;
            if (k < rp.n_out && __ldg(rp.out_idx + k) == pos) d = __ldg(rp.out_val + k);
            else bad = true;
            dv[kk] = d;
            ++k;
          }
        }
      }
      if (lane == 0) dv[0] += __ldg(rp.anchors + blk);
      int4 *dst = reinterpret_cast<int4 *>(&sq[w][16 * lane]);
#pragma unroll
      for (int u = 0; u < 4; ++u) dst[u] = make_int4(dv[4 * u], dv[4 * u + 1], dv[4 * u + 2], dv[4 * u + 3]);
    }
    if (lane < 16) smask[w][lane] = 0;  // no exception yet (the override values are read only where set)
    __syncwarp();
    BlockView b;
    b.sq = nullptr;
    b.itab = nullptr;
    b.cq = scq[w];
    b.cin = cin;
    b.wb = 0;
    b.xlim = xl;
    b.ylim = yl;
    b.zlim = zl;
    if (pid < 2) {
      // K inclusive prefix sums along x, y, z (lanes own two lines each)
      for (int rep = 0; rep <= pid; ++rep) {
        for (int axis = 0; axis < 3; ++axis) {
          const int stride = axis == 0 ? 1 : (axis == 1 ? 8 : 64);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int line = lane + 32 * h;  // 64 lines of 8 along the axis
            int base;
            if (axis == 0) base = line * 8;
            else if (axis == 1) base = (line & 7) + 64 * (line >> 3);
            else base = line;
            int32_t acc = 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              acc += sq[w][base + k * stride];
              sq[w][base + k * stride] = acc;
            }
          }
          __syncwarp();
        }
      }
    } else if (xl == 8 && yl == 8 && zl == 8 && cin == 0xffu) {
      // interpolation of a full block: the passes' points from the list,
      // each from its stencil entry (every in-block point is available)
      const bool cubic = pid == 3;
      for (int pass = 0; pass < 9; ++pass) {
        for (int k = kPassStart[pass] + lane; k < kPassStart[pass + 1]; k += 32) {
          const int p = rlist[k];
          const uint4 e = rtab[p];
          const uint32_t form = e.z & 3u;
          const int32_t vm1 = sq[w][p + (int16_t)(e.x & 0xffffu)];
          int32_t pred = vm1;
          if (form != 0) {
            const int32_t vp1 = (e.z & 0x100u) ? scq[w][e.z >> 16] : sq[w][p + (int16_t)(e.x >> 16)];
            // 32-bit wrapping arithmetic: exact for every stream the
            // compressor writes (|q| < 2^23), harmless for a damaged one
            if (cubic && form == 2) {
              const int32_t vm3 = sq[w][p + (int16_t)(e.y & 0xffffu)];
              const int32_t vp3 = (e.z & 0x200u) ? scq[w][e.z >> 16] : sq[w][p + (int16_t)(e.y >> 16)];
              pred = (int32_t)(9u * ((uint32_t)vm1 + (uint32_t)vp1) - (uint32_t)vm3 - (uint32_t)vp3 + 8u) >> 4;
            } else {
              pred = (int32_t)((uint32_t)vm1 + (uint32_t)vp1 + 1u) >> 1;
            }
          }
          sq[w][p] = (int32_t)((uint32_t)sq[w][p] + (uint32_t)pred);
        }
        __syncwarp();
      }
    } else {
      // interpolation: passes in order, each pass's points are independent
      const bool cubic = pid == 3;
      for (int s = 4; s >= 1; s >>= 1)
        for (int a = 0; a < 3; ++a) {
          for (int i = 0; i < 16; ++i) {
            const int p = 32 * i + lane;
            const int c[3] = {p & 7, (p >> 3) & 7, p >> 6};
            bool ok = p != 0 && (c[a] % (2 * s)) == s;
#pragma unroll
            for (int bb = 0; bb < 3; ++bb) {
              if (bb < a && c[bb] % s != 0) ok = false;
              if (bb > a && c[bb] % (2 * s) != 0) ok = false;
            }
            if (!ok || !b.in(c[0], c[1], c[2])) continue;
            // predict from the reconstructed values of earlier passes
            int sl, al;
            level_axis(c[0], c[1], c[2], sl, al);
            const int dx = al == 0 ? sl : 0, dy = al == 1 ? sl : 0, dz = al == 2 ? sl : 0;
            auto get = [&](int xx, int yy, int zz, int64_t &val) -> bool {
              if (xx >= 0 && yy >= 0 && zz >= 0 && xx < 8 && yy < 8 && zz < 8) {
                if (!b.in(xx, yy, zz)) return false;
                val = sq[w][(zz * 8 + yy) * 8 + xx];
                return true;
              }
              if ((xx != 0 && xx != 8) || (yy != 0 && yy != 8) || (zz != 0 && zz != 8)) return false;
              const int cc = (xx >> 3) + 2 * (yy >> 3) + 4 * (zz >> 3);
              if (!((cin >> cc) & 1u)) return false;
              val = scq[w][cc];
              return true;
            };
            int64_t vm1 = 0, vp1 = 0, vm3 = 0, vp3 = 0, pred;
            const bool am1 = get(c[0] - dx, c[1] - dy, c[2] - dz, vm1);
            const bool ap1 = get(c[0] + dx, c[1] + dy, c[2] + dz, vp1);
            const bool am3 = cubic && get(c[0] - 3 * dx, c[1] - 3 * dy, c[2] - 3 * dz, vm3);
            const bool ap3 = cubic && get(c[0] + 3 * dx, c[1] + 3 * dy, c[2] + 3 * dz, vp3);
            if (cubic && am3 && am1 && ap1 && ap3) pred = (-vm3 + 9 * vm1 + 9 * vp1 - vp3 + 8) >> 4;
            else if (am1 && ap1) pred = (vm1 + vp1 + 1) >> 1;
            else pred = vm1;
            sq[w][p] = (int32_t)(sq[w][p] + pred);
          }
          __syncwarp();
        }
    }
    // exceptions of this block into a per-warp override table
    if (rp.n_exc) {
      uint64_t e0 = 0, e1 = 0;
      if (lane == 0) {
        e0 = lb_u32(rp.exc_idx, rp.n_exc, pos0);
        e1 = lb_u32(rp.exc_idx, rp.n_exc, pos0 + 512);
      }
      e0 = __shfl_sync(0xffffffffu, e0, 0);
      e1 = __shfl_sync(0xffffffffu, e1, 0);
      for (uint64_t k = e0 + lane; k < e1; k += 32) {
        const uint32_t p = __ldg(rp.exc_idx + k) - pos0;
        sov[w][p] = __ldg(rp.exc_val + k);
        atomicOr(&smask[w][p >> 5], 1u << (p & 31));
      }
      __syncwarp();
    }
    // dequantize and store (lane i of step k: point 32 k + i)
    for (int i = 0; i < 16; ++i) {
      const int p = 32 * i + lane;
      const int px = p & 7, py = (p >> 3) & 7, pz = p >> 6;
      if (!b.in(px, py, pz)) continue;
      float v = __fmul_rn(__int2float_rn(sq[w][p]), rp.ebx2);
      if ((smask[w][p >> 5] >> (p & 31)) & 1u) v = __uint_as_float(sov[w][p]);
      rp.out[((uint64_t)(Z0 + pz) * g.ny + (Y0 + py)) * g.nx + (X0 + px)] = v;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) sel_err(rp.err, FZ_ECORRUPT);
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_selquant(const float *x, const Geom &g, uint32_t R, uint32_t pred, const CompressWs &ws,
                            const uint16_t *weights, cudaStream_t s, int sm_count) {
  SelOut so = {};
  so.weights = weights;
  switch (pred) {
    case FZ_SEL_MLP: return launch_sel_t<kSelNet>(x, g, R, 0, ws, so, s, sm_count);
    case FZ_SEL_EXHAUSTIVE: return launch_sel_t<kSelExhaustive>(x, g, R, 0, ws, so, s, sm_count);
    case FZ_PRED_GINTERP: return launch_sel_t<kSelGinterp>(x, g, R, pred, ws, so, s, sm_count);
    default: return launch_sel_t<kSelFixed>(x, g, R, pred, ws, so, s, sm_count);
  }
}

cudaError_t launch_select_report(const float *x, const Geom &g, uint32_t R, const CompressWs &ws, uint8_t *labels,
                                 uint32_t *costs, uint16_t *feat, cudaStream_t s, int sm_count) {
  SelOut so = {};
  so.labels = labels;
  so.costs = costs;
  so.feat = feat;
  return launch_sel_t<kSelReport>(x, g, R, 0, ws, so, s, sm_count);
}

cudaError_t launch_dec_codes(const uint8_t *d_in, const fz_header &h, const DecodeWs &ws, uint16_t *codes,
                             int32_t *ovals, cudaStream_t s, int sm_count) {
  SelDecParams p;
  p.ofirst = ws.ofirst;
  p.out_idx = reinterpret_cast<const uint32_t *>(d_in + h.off_out_idx);
  p.out_val = reinterpret_cast<const int32_t *>(d_in + h.off_out_val);
  p.n_out = h.n_out;
  p.ovals = ovals;
  p.words = reinterpret_cast<const uint32_t *>(d_in + h.off_bits);
  p.n_words = (h.total_bits + 31) / 32;
  p.chunk_bits = reinterpret_cast<const uint32_t *>(d_in + h.off_chunk_bits);
  p.goff = ws.gsum;
  p.n_chunks = h.n_chunks;
  p.n_units = dec_units_of(h.n_chunks);
  p.lut = ws.lut;
  p.codes = codes;
  p.err = ws.err;
  const int smem = (int)(sizeof(uint16_t) * kLutSize + sizeof(uint32_t) * kRing * kSelDecThreads);
  const bool ov = ovals != nullptr;
  cudaError_t e = cudaFuncSetAttribute(ov ? k_dec_codes<true> : k_dec_codes<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  uint64_t grid = (uint64_t)sm_count;
  if (grid > p.n_units) grid = p.n_units;
  if (ov) k_dec_codes<true><<<(unsigned)grid, kSelDecThreads, smem, s>>>(p);
  else k_dec_codes<false><<<(unsigned)grid, kSelDecThreads, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_sel_decode(const uint8_t *d_in, const fz_header &h, float *d_out, const DecodeWs &ws,
                              uint16_t *codes, cudaStream_t s, int sm_count) {
  Geom g;
  make_geom(h.ndim, h.dims, g);
  cudaError_t e = launch_dec_codes(d_in, h, ws, codes, nullptr, s, sm_count);
  if (e != cudaSuccess) return e;
  ReconParams rp;
  rp.codes = codes;
  rp.anchors = reinterpret_cast<const int32_t *>(d_in + h.off_anchors);
  rp.ids = (h.flags & FZ_FLAG_IDS) ? d_in + h.off_ids : nullptr;
  rp.fixed_pid = h.predictor;
  rp.out_idx = reinterpret_cast<const uint32_t *>(d_in + h.off_out_idx);
  rp.out_val = reinterpret_cast<const int32_t *>(d_in + h.off_out_val);
  rp.exc_idx = reinterpret_cast<const uint32_t *>(d_in + h.off_exc_idx);
  rp.exc_val = reinterpret_cast<const uint32_t *>(d_in + h.off_exc_val);
  rp.n_out = h.n_out;
  rp.n_exc = h.n_exc;
  rp.ofirst = ws.ofirst;
  rp.out = d_out;
  memcpy(&rp.ebx2, &h.ebx2_bits, 4);
  rp.R = (int32_t)h.radius;
  rp.err = ws.err;
  uint64_t rgrid = (g.n_blocks + kReconWarps - 1) / kReconWarps;
  if (rgrid > (uint64_t)sm_count * 16) rgrid = (uint64_t)sm_count * 16;
  k_sel_recon<<<(unsigned)rgrid, kReconWarps * 32, 0, s>>>(rp, g);
  return cudaGetLastError();
}

}  // namespace fz
