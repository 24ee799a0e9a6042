// fz_ginterp.cu -- decompression of full-field multilevel interpolation
// streams (the G-Interp spline predictor of FZMod-Quality, §3.3, taken from
// cuSZ-i via §3.1-§3.2), 3D fields with 8x8x8 blocks.
//
// The predictor works on the prequantized integer field q.  The anchors are
// the points whose coordinates are all multiples of 8 (the block origins);
// every other point is predicted once, at level s = 4, 2 or 1, along the x,
// y or z pass of that level, from its neighbours p +- s and p +- 3s along the
// pass axis (cubic form when all four lie in the domain, linear when p + s
// does, else p - s).  Neighbours are taken anywhere in the domain, so a
// point's reconstruction depends on the neighbouring blocks: the inverse
// runs level by level over the whole field.
//
// The points of level s with all coordinates multiples of s form a grid of
// extents m = ceil(n / s), whose even sub-grid (extents ceil(m / 2)) is the
// grid of level 2s.  One refine pass rebuilds a level's grid from its even
// sub-grid and the residuals: in grid coordinates its x pass fills the
// points (odd, even, even), its y pass (any, odd, even) and its z pass
// (any, any, odd), each from grid neighbours at +-1 and +-3 along its axis.
// Three passes -- anchors -> level 4, level 4 -> level 2, level 2 -> the
// field -- rebuild q; the last one also dequantizes.
//
// Kernels:
//   k_gi_refine   -- one CTA per (64 x 16 columns, run of planes) task:
//                    even planes in order (their x and y passes, from the
//                    even sub-grid, with a 2-row halo of the x pass for the
//                    y pass), kept in a ring of four; each odd plane from the
//                    four even planes around it (z pass); outputs q of the
//                    level's grid, or the dequantized field on the last pass
//   k_gi_outliers -- the outlier list: strictly ascending, each entry at a
//                    zero code (together with the refine pass finding every
//                    zero code in the list, the list is exactly the zero
//                    codes in order)
// The code stream itself comes from the selector path's chunk decoder
// (one thread per 512-symbol chunk into a code buffer), the exceptions from
// the shared exception scatter.
#include "fz_decode_common.cuh"

namespace fz {

namespace {

constexpr int kGiTX = 64, kGiTY = 16, kGiThreads = 256;
constexpr int kGiEX = kGiTX / 2 + 3;  // even sub-grid columns of a tile: X = X0 - 2 + 2 c
constexpr int kGiEXP = kGiEX + 1;
constexpr int kGiER = kGiTY / 2 + 3;  // even rows of a tile with the y halo: Y = Y0 - 2 + 2 r

struct GiParams {
  const uint16_t *codes;    // block-major code stream
  const int32_t *ein;       // the level's even sub-grid (natural order, extents ex, ey, ez)
  int32_t *qout;            // the level's grid (natural order, extents mx, my, mz); null on the last pass
  float *out;               // the field (last pass)
  const int32_t *ovals;     // the outliers' residuals at their positions (written by the code decoder)
  uint32_t *err;
  uint32_t mx, my, mz, ex, ey, ez;
  uint32_t s;               // grid point (X, Y, Z) is field point s (X, Y, Z)
  uint32_t tiles_x, tiles_y, zseg, n_tasks;
  int32_t R;
  float ebx2;
};

__device__ __forceinline__ void gi_err(uint32_t *err, uint32_t code) { atomicCAS(err, 0u, code); }

// Residual of grid point (X, Y, Z): code - R, or for code 0 the outlier's
// residual, which the code decoder stored at its position (after matching
// it to the outlier list).
__device__ __forceinline__ int32_t gi_delta(const GiParams &p, const Geom &g, uint32_t X, uint32_t Y, uint32_t Z) {
  // code-stream positions fit 32 bits (the format's outlier indices are u32)
  const uint32_t gx = X * p.s, gy = Y * p.s, gz = Z * p.s;
  const uint32_t blk = ((gz >> 3) * g.nby + (gy >> 3)) * g.nbx + (gx >> 3);
  const uint32_t pos = blk * 512u + (((gz & 7u) * 8u + (gy & 7u)) * 8u + (gx & 7u));
  const uint32_t c = __ldg(p.codes + pos);
  return c != 0 ? (int32_t)c - p.R : __ldg(p.ovals + pos);
}

// Prediction along one axis from the values at -3, -1, +1, +3 (grid steps)
// and their availability: c is the point's grid coordinate, m the extent.
// 32-bit arithmetic: every q of a stream the compressor writes lies below
// 2^23 in magnitude, so the cubic numerator stays below 2^28 (a damaged
// stream may wrap, harmlessly); the shifts are arithmetic (floor).
__device__ __forceinline__ int32_t gi_pred(uint32_t c, uint32_t m, int32_t vm3, int32_t vm1, int32_t vp1,
                                           int32_t vp3) {
  if (c >= 3 && c + 3 < m) {
    const uint32_t num = 9u * ((uint32_t)vm1 + (uint32_t)vp1) - (uint32_t)vm3 - (uint32_t)vp3 + 8u;
    return (int32_t)num >> 4;
  }
  if (c + 1 < m) return (int32_t)((uint32_t)vm1 + (uint32_t)vp1 + 1u) >> 1;
  return vm1;
}

template <bool LAST>
__device__ __forceinline__ void gi_store(const GiParams &p, const Geom &g, uint32_t X, uint32_t Y, uint32_t Z,
                                         int32_t q) {
  // field indices fit 32 bits (fewer values than 2^32 code positions)
  if (LAST) p.out[(Z * g.ny + Y) * g.nx + X] = __fmul_rn(__int2float_rn(q), p.ebx2);
  else p.qout[(Z * p.my + Y) * p.mx + X] = q;
}

#ifndef FZ_GI_MINB
#define FZ_GI_MINB 8  // CTAs per SM (4 and 6 measured slower on 512^3 fields)
#endif
template <bool LAST>
__global__ void __launch_bounds__(kGiThreads, FZ_GI_MINB) k_gi_refine(GiParams p, Geom g) {
  __shared__ int32_t sE[kGiER][kGiEXP];        // even sub-grid values of the current even plane
  __shared__ int32_t sP[kGiER][kGiTX];         // the even rows of the current even plane (x pass done)
  __shared__ int32_t sRing[4][kGiTY][kGiTX];   // finished even planes, slot (Z / 2) & 3
  const int t = threadIdx.x;
  for (uint32_t task = blockIdx.x; task < p.n_tasks; task += gridDim.x) {
    const uint32_t tx = task % p.tiles_x, r_ = task / p.tiles_x;
    const uint32_t ty = r_ % p.tiles_y, seg = r_ / p.tiles_y;
    const uint32_t X0 = tx * kGiTX, Y0 = ty * kGiTY, Z0 = seg * p.zseg;
    const uint32_t Z1 = Z0 + p.zseg < p.mz ? Z0 + p.zseg : p.mz;
    const uint32_t zs = Z0 >= 2 ? Z0 - 2 : 0;
    // even planes zs, zs + 2, ..., Z1 + 2; after even plane Ze, odd plane Ze - 3
    for (uint32_t Ze = zs; Ze <= Z1 + 2; Ze += 2) {
      const bool have_e = Ze < p.mz;
      if (have_e) {
        // 1. the even sub-grid rows of this plane around the tile
        const uint32_t ez = Ze >> 1;
        for (int i = t; i < kGiER * kGiEX; i += kGiThreads) {
          const int r = i / kGiEX, c = i % kGiEX;
          const uint32_t ex = (X0 >> 1) + (uint32_t)c - 1u, ey = (Y0 >> 1) + (uint32_t)r - 1u;  // may wrap: out
          sE[r][c] = (ex < p.ex && ey < p.ey) ? __ldg(p.ein + ((uint64_t)ez * p.ey + ey) * p.ex + ex) : 0;
        }
        __syncthreads();
        // 2. even rows (tile rows and the 2-row halo): a thread takes the
        // column pair (2 c2, 2 c2 + 1), the even column copied, the odd one
        // by the x pass
        {
          const int c2 = t & 31;
          const uint32_t Xe = X0 + 2u * (uint32_t)c2, Xo = Xe + 1u;
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int r = (t >> 5) + 8 * k;
            if (r < kGiER) {
              const uint32_t Y = Y0 + 2u * (uint32_t)r - 2u;  // may wrap: out
              const bool yin = Y < p.my;
              sP[r][2 * c2] = (yin && Xe < p.mx) ? sE[r][c2 + 1] : 0;
              int32_t v = 0;
              if (yin && Xo < p.mx)
                v = gi_delta(p, g, Xo, Y, Ze) + gi_pred(Xo, p.mx, sE[r][c2], sE[r][c2 + 1], sE[r][c2 + 2], sE[r][c2 + 3]);
              sP[r][2 * c2 + 1] = v;
            }
          }
        }
        __syncthreads();
        // 3. tile rows: a thread takes column xl and the rows yq + 4k (all of
        // one parity): even ones from above, odd ones by the y pass
        int32_t(*ring)[kGiTX] = sRing[(Ze >> 1) & 3];
        const bool emit = Ze >= Z0 && Ze < Z1;
        {
          const int xl = t & (kGiTX - 1), yq = t >> 6;
          const uint32_t X = X0 + (uint32_t)xl;
          const bool xin = X < p.mx;
          if (yq & 1) {
            int32_t d[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint32_t Y = Y0 + (uint32_t)(yq + 4 * k);
              d[k] = (xin && Y < p.my) ? gi_delta(p, g, X, Y, Ze) : 0;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int yl = yq + 4 * k, r = (yl - 1) >> 1;  // row of Y - 3
              const uint32_t Y = Y0 + (uint32_t)yl;
              int32_t v = 0;
              if (xin && Y < p.my) {
                v = d[k] + gi_pred(Y, p.my, sP[r][xl], sP[r + 1][xl], sP[r + 2][xl], sP[r + 3][xl]);
                if (emit) gi_store<LAST>(p, g, X, Y, Ze, v);
              }
              ring[yl][xl] = v;
            }
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int yl = yq + 4 * k;
              const uint32_t Y = Y0 + (uint32_t)yl;
              const int32_t v = sP[(yl >> 1) + 1][xl];  // 0 outside the domain
              if (emit && xin && Y < p.my) gi_store<LAST>(p, g, X, Y, Ze, v);
              ring[yl][xl] = v;
            }
          }
        }
        __syncthreads();
      }
      // 4. the odd plane between the four even planes Ze - 6 .. Ze
      if (Ze >= 3) {
        const uint32_t Zo = Ze - 3;
        if (Zo >= Z0 && Zo < Z1) {
          const int sm3 = (int)(((Zo - 3) >> 1) & 3), sm1 = (int)(((Zo - 1) >> 1) & 3);
          const int sp1 = (int)(((Zo + 1) >> 1) & 3), sp3 = (int)(((Zo + 3) >> 1) & 3);
          const int xl = t & (kGiTX - 1), yq = t >> 6;
          const uint32_t X = X0 + (uint32_t)xl;
          const bool xin = X < p.mx;
          int32_t d[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t Y = Y0 + (uint32_t)(yq + 4 * k);
            d[k] = (xin && Y < p.my) ? gi_delta(p, g, X, Y, Zo) : 0;
          }
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int yl = yq + 4 * k;
            const uint32_t Y = Y0 + (uint32_t)yl;
            if (xin && Y < p.my) {
              // slots of planes outside the domain are read only when unused
              const int32_t v = d[k] + gi_pred(Zo, p.mz, sRing[sm3][yl][xl], sRing[sm1][yl][xl], sRing[sp1][yl][xl],
                                               sRing[sp3][yl][xl]);
              gi_store<LAST>(p, g, X, Y, Zo, v);
            }
          }
        }
      }
      // the next even plane overwrites the slot of Ze - 6 and the sE / sP rows
      __syncthreads();
    }
  }
}

// err[3] holds the number of outlier codes the code decoder met.
__global__ void k_gi_outliers(const uint32_t *__restrict__ out_idx, uint64_t n_out, const uint16_t *__restrict__ codes,
                              uint64_t npad, uint32_t *err) {
  if (blockIdx.x == 0 && threadIdx.x == 0 && (uint64_t)err[3] != n_out) gi_err(err, FZ_ECORRUPT);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_out;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t pos = __ldg(out_idx + i);
    const bool ok = pos < npad && __ldg(codes + pos) == 0 && (i == 0 || __ldg(out_idx + i - 1) < pos);
    if (!ok) gi_err(err, FZ_ECORRUPT);
  }
}

template <bool LAST>
cudaError_t refine(GiParams p, const Geom &g, int sm_count, cudaStream_t s) {
  p.ex = (p.mx + 1) / 2;
  p.ey = (p.my + 1) / 2;
  p.ez = (p.mz + 1) / 2;
  p.tiles_x = (p.mx + kGiTX - 1) / kGiTX;
  p.tiles_y = (p.my + kGiTY - 1) / kGiTY;
  // plane runs: a task of zseg planes costs about zseg + 3 plane steps (its
  // even planes, three halo planes, its odd planes); take the run length
  // whose number of waves over the resident CTAs costs least
  static LaunchCache cache;
  int per_sm = 0;
  const cudaError_t e = cached_per_sm(k_gi_refine<LAST>, kGiThreads, 0, cache, per_sm);
  if (e != cudaSuccess) return e;
  const uint64_t cols = (uint64_t)p.tiles_x * p.tiles_y, slots = (uint64_t)sm_count * (uint64_t)per_sm;
  uint64_t best = ~0ull;
  for (uint32_t zs = 8; zs <= 64; zs *= 2) {
    const uint64_t tasks = cols * ((p.mz + zs - 1) / zs);
    const uint64_t cost = (tasks + slots - 1) / slots * (zs + 3);
    if (cost < best) { best = cost; p.zseg = zs; }
  }
  const uint64_t tasks = cols * ((p.mz + p.zseg - 1) / p.zseg);
  p.n_tasks = (uint32_t)tasks;
  uint64_t grid = tasks < slots ? tasks : slots;
  k_gi_refine<LAST><<<(unsigned)grid, kGiThreads, 0, s>>>(p, g);
  return cudaGetLastError();
}

}  // namespace

uint64_t ginterp_level_values(const fz_header &h, uint32_t s) {
  const uint64_t mx = (h.dims[0] + s - 1) / s, my = (h.dims[1] + s - 1) / s, mz = (h.dims[2] + s - 1) / s;
  return mx * my * mz;
}

cudaError_t launch_gi_decode(const uint8_t *d_in, const fz_header &h, float *d_out, const DecodeWs &ws,
                             uint16_t *codes, int32_t *ovals, int32_t *q4, int32_t *q2, cudaStream_t s, int sm_count) {
  Geom g;
  make_geom(h.ndim, h.dims, g);
  cudaError_t e = launch_dec_codes(d_in, h, ws, codes, ovals, s, sm_count);
  if (e != cudaSuccess) return e;
  GiParams p = {};
  p.codes = codes;
  p.ovals = ovals;
  p.err = ws.err;
  p.R = (int32_t)h.radius;
  memcpy(&p.ebx2, &h.ebx2_bits, 4);
  p.out = d_out;
  const int32_t *anchors = reinterpret_cast<const int32_t *>(d_in + h.off_anchors);
  const int32_t *ein[3] = {anchors, q4, q2};
  int32_t *qo[3] = {q4, q2, nullptr};
  for (int lv = 0; lv < 3 && e == cudaSuccess; ++lv) {
    p.s = 4u >> lv;
    p.mx = (g.nx + p.s - 1) / p.s;
    p.my = (g.ny + p.s - 1) / p.s;
    p.mz = (g.nz + p.s - 1) / p.s;
    p.ein = ein[lv];
    p.qout = qo[lv];
    e = lv < 2 ? refine<false>(p, g, sm_count, s) : refine<true>(p, g, sm_count, s);
  }
  if (e == cudaSuccess) {  // also when the list is empty: the count of outlier codes must be 0
    uint64_t og = (h.n_out + 255) / 256;
    if (og == 0) og = 1;
    if (og > (uint64_t)sm_count * 4) og = (uint64_t)sm_count * 4;
    k_gi_outliers<<<(unsigned)og, 256, 0, s>>>(reinterpret_cast<const uint32_t *>(d_in + h.off_out_idx), h.n_out,
                                               codes, g.npad, ws.err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && h.n_exc) e = launch_exc_scatter(d_in, h, d_out, ws.err, nullptr, s, sm_count);
  return e;
}

}  // namespace fz
