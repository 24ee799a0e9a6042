/*
 * fz_oracle.c -- plain, sequential CPU oracle of the error-bounded compression
 * path (FZMod-Default: value-range preprocessing, Lorenzo dual-quant with
 * outliers, code histogram, Huffman; FZModules §3.1-§3.3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  It shares no code, header,
 * table or constant generator with the CUDA library: the stream layout below is
 * written out here by byte offset, from the format definition.
 *
 * The paper defers the arithmetic of every stage to the cuSZ papers (§3.1), so
 * the method's exact steps are the readings fixed for this project (rounding,
 * block-local prediction, Huffman tie-break, bit order, stream layout).  Each
 * function below states the step it implements; nothing is blocked, fused or
 * reordered beyond that statement.  Build with -O2 -ffp-contract=off and no
 * fast-math so that every float operation is a single IEEE-754 binary32 op.
 *
 * Parity status: every function here is pinned by the CPU tests
 * (invariants, closed forms, brute force, independent Huffman) except the
 * compression ratio values of the paper's Table 3, which need datasets that
 * are not available ("parity unpinned" for those numbers only).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_EBUFFER 4
#define ORC_ECORRUPT 5
#define ORC_EUNSUPPORTED 7

#define ORC_LMAX 14
#define ORC_MAXSYM 1024

/* ------------------------------------------------------------------------ */
/* little-endian byte access (the stream is defined byte by byte)            */
/* ------------------------------------------------------------------------ */
static void put_u16(uint8_t *p, uint16_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void put_u32(uint8_t *p, uint32_t v) {
  for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static void put_u64(uint8_t *p, uint64_t v) {
  for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static uint16_t get_u16(const uint8_t *p) { return (uint16_t)(p[0] | (p[1] << 8)); }
static uint32_t get_u32(const uint8_t *p) {
  uint32_t v = 0;
  for (int i = 3; i >= 0; i--) v = (v << 8) | p[i];
  return v;
}
static uint64_t get_u64(const uint8_t *p) {
  uint64_t v = 0;
  for (int i = 7; i >= 0; i--) v = (v << 8) | p[i];
  return v;
}
static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint64_t d2u(double d) { uint64_t u; memcpy(&u, &d, 8); return u; }
static double u2d(uint64_t u) { double d; memcpy(&d, &u, 8); return d; }
static uint64_t align16(uint64_t v) { return (v + 15u) & ~(uint64_t)15u; }

/* ------------------------------------------------------------------------ */
/* Step 1-2: error bound and the FP32 constants (§3.2 preprocessing)         */
/* ------------------------------------------------------------------------ */

/* Largest binary32 value <= d, for finite d >= 0 (directed rounding down). */
static float round_down_f32(double d) {
  float f = (float)d;
  if ((double)f > d) f = nextafterf(f, 0.0f);
  return f;
}

/* REL range: minimum and maximum over the finite values of x.  Returns 1 if
 * x holds a finite value, else 0.  Also reports whether every value of x has
 * the same bit pattern (needed for the constant-field stream). */
int orc_range(const float *x, uint64_t n, float *lo, float *hi, int *all_same_bits) {
  uint64_t nf = 0;
  float mn = 0.0f, mx = 0.0f;
  int same = 1;
  uint32_t b0 = n ? f2u(x[0]) : 0;
  for (uint64_t i = 0; i < n; i++) {
    if (f2u(x[i]) != b0) same = 0;
    if (!isfinite(x[i])) continue;
    if (nf == 0) { mn = x[i]; mx = x[i]; }
    else {
      if (x[i] < mn) mn = x[i];
      if (x[i] > mx) mx = x[i];
    }
    nf++;
  }
  *lo = mn; *hi = mx; *all_same_bits = same;
  return (int)(nf > 0);
}

/* eb_abs -> (ebx2, inv2eb, eb_chk):
 *   ebx2   = round-down-to-f32( 2*eb_abs*(1 - 2^-12) )   quantization bin width
 *   inv2eb = round-to-nearest-f32( 1 / (double)ebx2 )
 *   eb_chk = round-down-to-f32( eb_abs*(1 - 2^-23) )     per-value check bound */
void orc_constants(double eb_abs, float *ebx2, float *inv2eb, float *eb_chk) {
  double w = 2.0 * eb_abs;
  w = w * (1.0 - 0x1p-12);
  float e2 = round_down_f32(w);
  double inv = 1.0 / (double)e2;
  *ebx2 = e2;
  *inv2eb = (float)inv;
  double c = eb_abs * (1.0 - 0x1p-23);
  *eb_chk = round_down_f32(c);
}

/* ------------------------------------------------------------------------ */
/* Step 3: prequantization (dual-quant step one, cuSZ via §3.1)              */
/* ------------------------------------------------------------------------ */

/* One value: q = rint(x * inv2eb) in binary32, half to even.  The value is an
 * exception (stored verbatim) when it is not finite, when |t| is not below
 * 2^23 (q forced to 0), or when the reconstruction q*ebx2 misses x by more than
 * eb_chk (q kept).  Returns 1 for an exception. */
int orc_prequant_one(float x, float inv2eb, float ebx2, float eb_chk, int32_t *q) {
  if (!isfinite(x)) { *q = 0; return 1; }
  float t = x * inv2eb;
  if (!(fabsf(t) < 0x1p23f)) { *q = 0; return 1; }
  float r0 = rintf(t);
  int32_t qi = (int32_t)r0;
  *q = qi;
  float r = (float)qi * ebx2;
  float d = fabsf(x - r);
  return d > eb_chk;
}

void orc_prequant(const float *x, uint64_t n, float inv2eb, float ebx2, float eb_chk,
                  int32_t *q, uint8_t *exc) {
  for (uint64_t i = 0; i < n; i++) exc[i] = (uint8_t)orc_prequant_one(x[i], inv2eb, ebx2, eb_chk, &q[i]);
}

/* ------------------------------------------------------------------------ */
/* Step 4: block decomposition                                               */
/* ------------------------------------------------------------------------ */

/* Default block shape per dimensionality: 1D 1024, 2D 32x32, 3D 8x8x8. */
void orc_block_shape(uint32_t ndim, uint32_t blk[3]) {
  blk[0] = blk[1] = blk[2] = 1;
  if (ndim == 1) blk[0] = 1024;
  else if (ndim == 2) { blk[0] = 32; blk[1] = 32; }
  else { blk[0] = 8; blk[1] = 8; blk[2] = 8; }
}

typedef struct {
  uint64_t d[3];   /* field extents, x fastest (unused axes are 1) */
  uint32_t b[3];   /* block extents */
  uint64_t nb[3];  /* blocks per axis */
  uint64_t n_blocks, bsize, npad;
} grid_t;

static void make_grid(uint32_t ndim, const uint64_t dims[3], grid_t *g) {
  for (int a = 0; a < 3; a++) g->d[a] = (a < (int)ndim) ? dims[a] : 1;
  orc_block_shape(ndim, g->b);
  g->n_blocks = 1;
  g->bsize = 1;
  for (int a = 0; a < 3; a++) {
    g->nb[a] = (g->d[a] + g->b[a] - 1) / g->b[a];
    g->n_blocks *= g->nb[a];
    g->bsize *= g->b[a];
  }
  g->npad = g->n_blocks * g->bsize;
}

/* ------------------------------------------------------------------------ */
/* Step 5: predictors on block-local q (zero outside the block and domain)   */
/* ------------------------------------------------------------------------ */

/* Signed binomial coefficient of (1 - S)^k at shift o. */
static int64_t lz_coef(int k, int o) {
  if (k == 1) return o == 0 ? 1 : -1;
  /* k == 2: 1, -2, 1 */
  return o == 1 ? -2 : 1;
}

/* Lorenzo-k residual of one block: delta = prod_a (1 - S_a)^k q, written out
 * as the direct sum over all shift vectors o in {0..k}^ndim of
 * prod_a c_k(o_a) * q(p - o), with q taken as 0 where p - o leaves the block
 * or the domain.  qb holds the block's q in block order (x fastest);
 * inb[i] says whether position i lies in the domain. */
void orc_lorenzo_block(int k, uint32_t ndim, const uint32_t b[3], const int32_t *qb,
                       const uint8_t *inb, int64_t *delta) {
  uint32_t bx = b[0], by = b[1], bz = b[2];
  int ox_max = k, oy_max = ndim >= 2 ? k : 0, oz_max = ndim >= 3 ? k : 0;
  for (uint32_t z = 0; z < bz; z++)
    for (uint32_t y = 0; y < by; y++)
      for (uint32_t x = 0; x < bx; x++) {
        uint64_t i = ((uint64_t)z * by + y) * bx + x;
        int64_t s = 0;
        for (int oz = 0; oz <= oz_max; oz++)
          for (int oy = 0; oy <= oy_max; oy++)
            for (int ox = 0; ox <= ox_max; ox++) {
              int64_t xx = (int64_t)x - ox, yy = (int64_t)y - oy, zz = (int64_t)z - oz;
              if (xx < 0 || yy < 0 || zz < 0) continue;
              uint64_t j = ((uint64_t)zz * by + (uint64_t)yy) * bx + (uint64_t)xx;
              if (!inb[j]) continue;
              int64_t c = lz_coef(k, ox);
              if (ndim >= 2) c *= lz_coef(k, oy);
              if (ndim >= 3) c *= lz_coef(k, oz);
              s += c * qb[j];
            }
        delta[i] = s;
      }
}

/* Inverse of Lorenzo-k on one block: k inclusive prefix sums along each axis
 * (exact integer arithmetic, so the axis order does not matter). */
void orc_lorenzo_block_inverse(int k, uint32_t ndim, const uint32_t b[3], int64_t *v) {
  uint32_t bx = b[0], by = b[1], bz = b[2];
  for (int rep = 0; rep < k; rep++) {
    for (uint32_t z = 0; z < bz; z++)
      for (uint32_t y = 0; y < by; y++)
        for (uint32_t x = 1; x < bx; x++) {
          uint64_t i = ((uint64_t)z * by + y) * bx + x;
          v[i] += v[i - 1];
        }
    if (ndim >= 2)
      for (uint32_t z = 0; z < bz; z++)
        for (uint32_t y = 1; y < by; y++)
          for (uint32_t x = 0; x < bx; x++) {
            uint64_t i = ((uint64_t)z * by + y) * bx + x;
            v[i] += v[i - bx];
          }
    if (ndim >= 3)
      for (uint32_t z = 1; z < bz; z++)
        for (uint32_t y = 0; y < by; y++)
          for (uint32_t x = 0; x < bx; x++) {
            uint64_t i = ((uint64_t)z * by + y) * bx + x;
            v[i] += v[i - (uint64_t)bx * by];
          }
  }
}

/* Gather one block of a field-order array into block order; positions outside
 * the domain get 0 and inb = 0. */
static void gather_block(const grid_t *g, uint64_t blk, const int32_t *q, int32_t *qb, uint8_t *inb,
                         uint64_t *fidx) {
  uint64_t bxi = blk % g->nb[0], byi = (blk / g->nb[0]) % g->nb[1], bzi = blk / (g->nb[0] * g->nb[1]);
  uint64_t i = 0;
  for (uint32_t z = 0; z < g->b[2]; z++)
    for (uint32_t y = 0; y < g->b[1]; y++)
      for (uint32_t x = 0; x < g->b[0]; x++, i++) {
        uint64_t X = bxi * g->b[0] + x, Y = byi * g->b[1] + y, Z = bzi * g->b[2] + z;
        int in = X < g->d[0] && Y < g->d[1] && Z < g->d[2];
        inb[i] = (uint8_t)in;
        uint64_t f = in ? (Z * g->d[1] + Y) * g->d[0] + X : 0;
        fidx[i] = f;
        qb[i] = in && q ? q[f] : 0;
      }
}

/* ------------------------------------------------------------------------ */
/* Steps 8-9: Huffman code lengths and canonical codes (§3.2)                */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t w; uint32_t s; } leaf_t;

static int leaf_cmp(const void *a, const void *b) {
  const leaf_t *x = (const leaf_t *)a, *y = (const leaf_t *)b;
  if (x->w != y->w) return x->w < y->w ? -1 : 1;
  return x->s < y->s ? -1 : (x->s > y->s);
}

/* Code lengths of the Huffman code of the histogram, limited to ORC_LMAX
 * bits: the optimal prefix code among those whose lengths are all <= 14,
 * computed by the package-merge algorithm of Larmore and Hirschberg (when the
 * plain Huffman code already fits in 14 bits this is a Huffman code).
 *   Leaves: the used symbols sorted by (count, symbol).
 *   Level L = 14 holds the leaves.  Level l < L holds the leaves merged with
 *   the packages of level l+1 (sums of its consecutive item pairs; an odd
 *   last item is dropped), ordered by weight, a leaf before a package of
 *   equal weight.
 *   The first 2m-2 items of level 1 are selected.  At each level, of the
 *   selected items a_l are leaves and the others packages, which select the
 *   first 2(m_l - a_l) items of the next level.
 *   The length of the i-th leaf is the number of levels where i < a_l.
 * A single used symbol gets length 1. */
int orc_huffman_lengths(const uint64_t *counts_in, uint32_t nsym, uint8_t *len) {
  if (nsym == 0 || nsym > ORC_MAXSYM) return ORC_EINVAL;
  leaf_t leaf[ORC_MAXSYM];
  memset(len, 0, nsym);
  uint32_t m = 0;
  for (uint32_t s = 0; s < nsym; s++)
    if (counts_in[s]) { leaf[m].w = counts_in[s]; leaf[m].s = s; m++; }
  if (m == 0) return ORC_EINVAL;
  if (m == 1) { len[leaf[0].s] = 1; return ORC_OK; }
  qsort(leaf, m, sizeof(leaf_t), leaf_cmp);
  static uint64_t cur[2 * ORC_MAXSYM], nxt[2 * ORC_MAXSYM], pk[ORC_MAXSYM];
  static uint8_t isleaf[ORC_LMAX + 1][2 * ORC_MAXSYM];
  uint32_t n_cur = m;
  for (uint32_t i = 0; i < m; i++) { cur[i] = leaf[i].w; isleaf[ORC_LMAX][i] = 1; }
  for (int l = ORC_LMAX - 1; l >= 1; l--) {
    uint32_t np = n_cur / 2;
    for (uint32_t j = 0; j < np; j++) pk[j] = cur[2 * j] + cur[2 * j + 1];
    uint32_t i = 0, j = 0, k = 0;
    while (i < m || j < np) {
      if (j >= np || (i < m && leaf[i].w <= pk[j])) { nxt[k] = leaf[i].w; isleaf[l][k] = 1; i++; }
      else { nxt[k] = pk[j]; isleaf[l][k] = 0; j++; }
      k++;
    }
    n_cur = k;
    memcpy(cur, nxt, n_cur * sizeof(uint64_t));
  }
  uint32_t sel = 2 * m - 2;
  for (int l = 1; l <= ORC_LMAX && sel > 0; l++) {
    uint32_t a = 0;
    for (uint32_t k = 0; k < sel; k++) a += isleaf[l][k];
    for (uint32_t i = 0; i < a; i++) len[leaf[i].s]++;
    sel = 2 * (sel - a);
  }
  return ORC_OK;
}

/* Canonical codes from lengths, in the order of RFC 1951 §3.2.2: count codes
 * per length, first code of each length, then numerically consecutive codes
 * within a length in symbol order.  Returns ORC_ECORRUPT when the lengths
 * over-subscribe the code space (Kraft sum > 1) or exceed 14 bits. */
int orc_canonical_codes(const uint8_t *len, uint32_t nsym, uint32_t *code) {
  uint32_t bl_count[ORC_LMAX + 1] = {0}, next_code[ORC_LMAX + 2] = {0};
  for (uint32_t s = 0; s < nsym; s++) {
    if (len[s] > ORC_LMAX) return ORC_ECORRUPT;
    if (len[s]) bl_count[len[s]]++;
  }
  uint64_t kraft = 0; /* in units of 2^-ORC_LMAX */
  for (int l = 1; l <= ORC_LMAX; l++) kraft += (uint64_t)bl_count[l] << (ORC_LMAX - l);
  if (kraft > ((uint64_t)1 << ORC_LMAX)) return ORC_ECORRUPT;
  uint32_t c = 0;
  for (int bits = 1; bits <= ORC_LMAX; bits++) {
    c = (c + bl_count[bits - 1]) << 1;
    next_code[bits] = c;
  }
  for (uint32_t s = 0; s < nsym; s++) {
    code[s] = 0;
    if (len[s]) code[s] = next_code[len[s]]++;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Step 10: bit writer / reader, MSB first into 32-bit words                 */
/* ------------------------------------------------------------------------ */

/* Write the low `l` bits of `c`, most significant first, at global bit p:
 * bit p goes to word p>>5, bit position 31-(p&31). */
static void put_bits(uint32_t *w, uint64_t p, uint32_t c, uint32_t l) {
  for (uint32_t i = 0; i < l; i++) {
    uint32_t bit = (c >> (l - 1 - i)) & 1u;
    uint64_t q = p + i;
    if (bit) w[q >> 5] |= 1u << (31 - (q & 31));
  }
}

static uint32_t get_bit(const uint32_t *w, uint64_t p) { return (w[p >> 5] >> (31 - (p & 31))) & 1u; }

/* ------------------------------------------------------------------------ */
/* Stream header layout (byte offsets)                                       */
/* ------------------------------------------------------------------------ */
#define H_MAGIC 0
#define H_VERSION 4
#define H_FLAGS 6
#define H_NDIM 8
#define H_EBMODE 12
#define H_DIMS 16
#define H_EB 40
#define H_EBABS 48
#define H_EBX2 56
#define H_INV2EB 60
#define H_EBCHK 64
#define H_RADIUS 68
#define H_BLOCK 72
#define H_PRED 84
#define H_CHUNK 88
#define H_NBLOCKS 96
#define H_NCHUNKS 104
#define H_NOUT 112
#define H_NEXC 120
#define H_TBITS 128
#define H_OFF_LENS 136
#define H_OFF_IDS 144
#define H_OFF_ANCH 152
#define H_OFF_CBITS 160
#define H_OFF_OIDX 168
#define H_OFF_OVAL 176
#define H_OFF_EIDX 184
#define H_OFF_EVAL 192
#define H_OFF_BITS 200
#define H_TOTAL 208
#define HDR 256u
#define MAGIC 0x42475A46u /* bytes 'F' 'Z' 'G' 'B' */
#define F_RAW 1u
#define F_CONST 2u
#define F_IDS 4u
#define F_SHUF 8u /* bit-shuffle + zero-word encoding instead of Huffman */

static void put_min_header(uint8_t *h, uint16_t flags, uint32_t ndim, uint32_t ebmode,
                           const uint64_t dims[3], double eb, uint64_t total) {
  memset(h, 0, HDR);
  put_u32(h + H_MAGIC, MAGIC);
  put_u16(h + H_VERSION, 1);
  put_u16(h + H_FLAGS, flags);
  put_u32(h + H_NDIM, ndim);
  put_u32(h + H_EBMODE, ebmode);
  for (int a = 0; a < 3; a++) put_u64(h + H_DIMS + 8 * a, a < (int)ndim ? dims[a] : 1);
  put_u64(h + H_EB, d2u(eb));
  put_u64(h + H_TOTAL, total);
}

/* ------------------------------------------------------------------------ */
/* Per-block predictor selection (3D, 8x8x8 blocks): interpolation           */
/* predictors, exhaustive trial, block features and the selector MLP         */
/* (the auto-selection of modules named as future work in §5; the dynamic   */
/* module selection of §3.3.1)                                               */
/* ------------------------------------------------------------------------ */

static int check_args(uint32_t ndim, const uint64_t dims[3], uint64_t *n);

#define ORC_NPRED 4
#define ORC_NFEAT 32
#define ORC_HID 64

/* Corner c = cx + 2 cy + 4 cz of a block: the point o + 8 (cx, cy, cz). */
static int corner_of(int x, int y, int z) {
  if ((x != 0 && x != 8) || (y != 0 && y != 8) || (z != 0 && z != 8)) return -1;
  return (x >> 3) + 2 * (y >> 3) + 4 * (z >> 3);
}

/* Value and availability of a point of the block's neighbourhood during the
 * interpolation: in-block points (in the domain) and in-domain corners. */
static int interp_get(const int64_t *vb, const uint8_t *inb, const int32_t cq[8], const uint8_t cin[8], int x, int y,
                      int z, int64_t *v) {
  if (x >= 0 && y >= 0 && z >= 0 && x < 8 && y < 8 && z < 8) {
    int i = (z * 8 + y) * 8 + x;
    if (!inb[i]) return 0;
    *v = vb[i];
    return 1;
  }
  int c = corner_of(x, y, z);
  if (c < 0 || !cin[c]) return 0;
  *v = cq[c];
  return 1;
}

/* Interpolation predictor of one 8x8x8 block on the integer field q, open
 * loop.  Known first: the block origin (its anchor) and the in-domain
 * corners o + {0,8}^3.  Levels s = 4, 2, 1; within a level, passes along x,
 * then y, then z; the pass along axis a predicts the points whose a
 * coordinate is s mod 2s, whose earlier coordinates are 0 mod s and whose
 * later coordinates are 0 mod 2s.  With neighbours p +- s and p +- 3s along
 * a: the cubic form (-q[-3] + 9 q[-1] + 9 q[+1] - q[+3] + 8) >> 4 when
 * `cubic` and all four are available, else the linear form
 * (q[-1] + q[+1] + 1) >> 1 when both near neighbours are, else q[-1].  The
 * residual is q - prediction (at the origin: q itself, the anchor).  When
 * `inverse` is set, v holds residuals on entry and q on exit. */
void orc_interp_block(int cubic, int inverse, const uint8_t *inb, const int32_t cq[8], const uint8_t cin[8],
                      int64_t *v) {
  /* w: q values.  Forward: all of q (the traversal only ever reads points
   * of earlier levels or passes).  Inverse: filled in traversal order,
   * starting from the origin, whose residual is q itself. */
  int64_t *w = (int64_t *)malloc(512 * sizeof(int64_t));
  if (!w) return;
  for (int i = 0; i < 512; i++) w[i] = inverse ? 0 : v[i];
  if (inverse) w[0] = v[0];
  for (int s = 4; s >= 1; s >>= 1)
    for (int a = 0; a < 3; a++)
      for (int z = 0; z < 8; z++)
        for (int y = 0; y < 8; y++)
          for (int x = 0; x < 8; x++) {
            int c[3] = {x, y, z};
            int ok = (c[a] % (2 * s)) == s;
            for (int b = 0; b < 3 && ok; b++) {
              if (b < a && c[b] % s != 0) ok = 0;
              if (b > a && c[b] % (2 * s) != 0) ok = 0;
            }
            if (!ok) continue;
            int i = (z * 8 + y) * 8 + x;
            if (!inb[i]) continue;
            int64_t vm1, vp1, vm3, vp3;
            int d[3] = {0, 0, 0};
            d[a] = s;
            int am1 = interp_get(w, inb, cq, cin, x - d[0], y - d[1], z - d[2], &vm1);
            int ap1 = interp_get(w, inb, cq, cin, x + d[0], y + d[1], z + d[2], &vp1);
            int am3 = interp_get(w, inb, cq, cin, x - 3 * d[0], y - 3 * d[1], z - 3 * d[2], &vm3);
            int ap3 = interp_get(w, inb, cq, cin, x + 3 * d[0], y + 3 * d[1], z + 3 * d[2], &vp3);
            int64_t pred;
            if (cubic && am3 && am1 && ap1 && ap3) pred = (-vm3 + 9 * vm1 + 9 * vp1 - vp3 + 8) >> 4;
            else if (am1 && ap1) pred = (vm1 + vp1 + 1) >> 1;
            else pred = vm1; /* p - s is in the block and the domain whenever p is */
            if (inverse) w[i] = v[i] + pred;  /* reconstruct q */
            else v[i] = w[i] - pred;          /* residual; w keeps q */
          }
  if (inverse) for (int i = 0; i < 512; i++) v[i] = inb[i] ? w[i] : 0;
  free(w);
}

/* ------------------------------------------------------------------------ */
/* Full-field multilevel interpolation (FZMod-Quality, §3.3: the G-Interp    */
/* spline predictor of cuSZ-i in place of Lorenzo, §3.1-§3.2)                */
/* ------------------------------------------------------------------------ */

/* Open loop on the integer field q of a 3D field (field order, x fastest),
 * with the anchor grid of the 8x8x8 blocks: the points whose three
 * coordinates are all multiples of 8 keep q.  Every other point is predicted
 * exactly once.  Levels s = 4, 2, 1; within a level the passes along x, then
 * y, then z; the pass (s, a) covers the points whose a coordinate is s mod 2s,
 * whose earlier coordinates are 0 mod s and whose later coordinates are 0 mod
 * 2s.  Its neighbours p +- s and p +- 3s along a were predicted in an earlier
 * pass or are anchors; a neighbour is available when it lies in the domain,
 * anywhere in the field (not only in p's block).  Prediction: the cubic form
 * (-q[-3] + 9 q[-1] + 9 q[+1] - q[+3] + 8) >> 4 when all four are available,
 * else (q[-1] + q[+1] + 1) >> 1 when both near ones are, else q[-1] (p - s is
 * always in the domain).  Forward (inverse = 0): v holds q on entry and the
 * residuals q - prediction on exit (anchors keep q).  Inverse: v holds the
 * residuals on entry (anchors: q) and q on exit. */
int orc_ginterp_field(int inverse, const uint64_t d[3], int64_t *v) {
  const uint64_t n = d[0] * d[1] * d[2];
  int64_t *w = (int64_t *)malloc((n ? n : 1) * sizeof(int64_t));
  if (!w) return ORC_ENOMEM;
  /* w: q.  Forward: all of q.  Inverse: the anchors now, the other points
   * as their pass reconstructs them. */
  for (uint64_t i = 0; i < n; i++) w[i] = v[i];
  for (uint64_t s = 4; s >= 1; s >>= 1)
    for (int a = 0; a < 3; a++) {
      uint64_t start[3], step[3];
      for (int b = 0; b < 3; b++) {
        start[b] = b == a ? s : 0;
        step[b] = b == a ? 2 * s : (b < a ? s : 2 * s);
      }
      const uint64_t stride = a == 0 ? 1 : (a == 1 ? d[0] : d[0] * d[1]);
      for (uint64_t z = start[2]; z < d[2]; z += step[2])
        for (uint64_t y = start[1]; y < d[1]; y += step[1])
          for (uint64_t x = start[0]; x < d[0]; x += step[0]) {
            const uint64_t c = a == 0 ? x : (a == 1 ? y : z);
            const uint64_t i = (z * d[1] + y) * d[0] + x;
            const int am3 = c >= 3 * s, ap1 = c + s < d[a], ap3 = c + 3 * s < d[a];
            const int64_t qm1 = w[i - s * stride];
            int64_t pred;
            if (am3 && ap3) {
              const int64_t qm3 = w[i - 3 * s * stride], qp1 = w[i + s * stride], qp3 = w[i + 3 * s * stride];
              pred = (-qm3 + 9 * qm1 + 9 * qp1 - qp3 + 8) >> 4;
            } else if (ap1) {
              pred = (qm1 + w[i + s * stride] + 1) >> 1;
            } else {
              pred = qm1;
            }
            if (inverse) w[i] = v[i] + pred;
            else v[i] = w[i] - pred;
          }
    }
  if (inverse)
    for (uint64_t i = 0; i < n; i++) v[i] = w[i];
  free(w);
  return ORC_OK;
}

/* Residuals of predictor pid (0 Lorenzo-1, 1 Lorenzo-2, 2 interpolation
 * linear, 3 interpolation cubic) for one block; qb in block order. */
static void block_residual(int pid, uint32_t ndim, const uint32_t b[3], const int32_t *qb, const uint8_t *inb,
                           const int32_t cq[8], const uint8_t cin[8], int64_t *delta) {
  if (pid < 2) {
    orc_lorenzo_block(pid + 1, ndim, b, qb, inb, delta);
    return;
  }
  for (int i = 0; i < 512; i++) delta[i] = inb[i] ? qb[i] : 0;
  orc_interp_block(pid == 3, 0, inb, cq, cin, delta);
}

/* q values at the 8 corners o + {0,8}^3 of block blk and whether each lies
 * in the domain. */
static void block_corners(const grid_t *g, uint64_t blk, const int32_t *q, int32_t cq[8], uint8_t cin[8]) {
  uint64_t bxi = blk % g->nb[0], byi = (blk / g->nb[0]) % g->nb[1], bzi = blk / (g->nb[0] * g->nb[1]);
  for (int c = 0; c < 8; c++) {
    uint64_t X = (bxi + (c & 1)) * 8, Y = (byi + ((c >> 1) & 1)) * 8, Z = (bzi + (c >> 2)) * 8;
    cin[c] = (uint8_t)(X < g->d[0] && Y < g->d[1] && Z < g->d[2]);
    cq[c] = cin[c] ? q[(Z * g->d[1] + Y) * g->d[0] + X] : 0;
  }
}

/* Trial cost of a residual: 1 + 2 floor(log2(|d| + 1)) bits inside the code
 * range (an Elias-gamma-like size), 96 bits for an outlier. */
static uint64_t trial_bits(int64_t d, uint32_t R) {
  uint64_t a = (uint64_t)(d < 0 ? -d : d);
  if (a >= R) return 96;
  uint64_t v = a + 1, e = 0;
  while (v >>= 1) e++;
  return 1 + 2 * e;
}

/* Exhaustive trial: cost of every predictor over the block's in-domain
 * points except the origin; returns the argmin (ties: lowest id). */
int orc_block_costs(const int32_t *qb, const uint8_t *inb, const int32_t cq[8], const uint8_t cin[8], uint32_t R,
                    uint64_t cost[ORC_NPRED]) {
  static const uint32_t b3[3] = {8, 8, 8};
  int64_t delta[512];
  int best = 0;
  for (int k = 0; k < ORC_NPRED; k++) {
    block_residual(k, 3, b3, qb, inb, cq, cin, delta);
    uint64_t c = 0;
    for (int i = 1; i < 512; i++)
      if (inb[i]) c += trial_bits(delta[i], R);
    cost[k] = c;
    if (c < cost[best]) best = k;
  }
  return best;
}

/* log2fix(s) = e + m/16 with e = floor(log2(s+1)) and m the 4 bits of s+1
 * below its leading one (zero-filled when s+1 has fewer bits); exact in
 * binary32. */
float orc_log2fix(uint64_t s) {
  uint64_t v = s + 1;
  int e = 63;
  while (!((v >> e) & 1)) e--;
  uint64_t m = e >= 4 ? (v >> (e - 4)) & 15u : (v << (4 - e)) & 15u;
  return (float)e + (float)m / 16.0f;
}

/* binary32 -> bfloat16 bits, round to nearest, ties to even (finite input). */
uint16_t orc_f32_to_bf16(float f) {
  uint32_t u = f2u(f);
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}
float orc_bf16_to_f32(uint16_t h) { return u2f((uint32_t)h << 16); }

static uint64_t uabs64(int64_t v) { return (uint64_t)(v < 0 ? -v : v); }

/* The 32 block statistics (all integers >= 0) behind the selector's inputs:
 *  0-7   sum and max of |residual| of predictors 0..3 on the 64 points with
 *        all-odd in-block coordinates
 *  8-10  sum |q(p) - q(p - e_a)|               (first differences, a = x,y,z)
 *  11-13 sum |second differences|, 14-16 sum |third differences| per axis
 *  17-19 sum |mixed differences| for (x,y), (x,z), (y,z)
 *  20-22 sign changes between consecutive first differences per axis
 *  23    sum |q - mean| (mean = floor(sum q / n))
 *  24    max q - min q
 *  25    outliers of Lorenzo-1 on the odd sub-lattice
 *  26-28 availability of the +x, +y, +z corner anchors
 *  29    in-domain points, 30 |anchor|, 31 sum |q(p) - q(p - 2 e_x)|
 * A difference is taken where all the points it uses lie in the block and
 * the domain.  Then feature = bf16(log2fix(statistic)). */
void orc_block_features(const int32_t *qb, const uint8_t *inb, const int32_t cq[8], const uint8_t cin[8], uint32_t R,
                        uint64_t stat[ORC_NFEAT], uint16_t feat[ORC_NFEAT]) {
  static const uint32_t b3[3] = {8, 8, 8};
  int64_t delta[512];
  memset(stat, 0, ORC_NFEAT * sizeof(uint64_t));
  for (int k = 0; k < ORC_NPRED; k++) {
    block_residual(k, 3, b3, qb, inb, cq, cin, delta);
    for (int z = 1; z < 8; z += 2)
      for (int y = 1; y < 8; y += 2)
        for (int x = 1; x < 8; x += 2) {
          int i = (z * 8 + y) * 8 + x;
          if (!inb[i]) continue;
          uint64_t a = uabs64(delta[i]);
          stat[2 * k] += a;
          if (a > stat[2 * k + 1]) stat[2 * k + 1] = a;
          if (k == 0 && a >= R) stat[25]++;
        }
  }
  int64_t sum = 0, mn = 0, mx = 0;
  uint64_t n = 0;
  for (int i = 0; i < 512; i++)
    if (inb[i]) {
      if (n == 0) { mn = qb[i]; mx = qb[i]; }
      if (qb[i] < mn) mn = qb[i];
      if (qb[i] > mx) mx = qb[i];
      sum += qb[i];
      n++;
    }
  for (int z = 0; z < 8; z++)
    for (int y = 0; y < 8; y++)
      for (int x = 0; x < 8; x++) {
        int c[3] = {x, y, z};
        int i = (z * 8 + y) * 8 + x;
        if (!inb[i]) continue;
        int st[3] = {1, 8, 64};
        for (int a = 0; a < 3; a++) {
          if (c[a] >= 1 && inb[i - st[a]]) {
            int64_t d1 = (int64_t)qb[i] - qb[i - st[a]];
            stat[8 + a] += uabs64(d1);
            if (c[a] >= 2 && inb[i - 2 * st[a]]) {
              int64_t d1p = (int64_t)qb[i - st[a]] - qb[i - 2 * st[a]];
              stat[11 + a] += uabs64(d1 - d1p);
              if ((d1 > 0 && d1p < 0) || (d1 < 0 && d1p > 0)) stat[20 + a]++;
              if (c[a] >= 3 && inb[i - 3 * st[a]]) {
                int64_t d1pp = (int64_t)qb[i - 2 * st[a]] - qb[i - 3 * st[a]];
                stat[14 + a] += uabs64(d1 - 2 * d1p + d1pp);
              }
            }
          }
        }
        int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        for (int pr = 0; pr < 3; pr++) {
          int a = pairs[pr][0], bb = pairs[pr][1];
          if (c[a] >= 1 && c[bb] >= 1 && inb[i - st[a]] && inb[i - st[bb]] && inb[i - st[a] - st[bb]]) {
            int64_t m = (int64_t)qb[i] - qb[i - st[a]] - qb[i - st[bb]] + qb[i - st[a] - st[bb]];
            stat[17 + pr] += uabs64(m);
          }
        }
        if (x >= 2 && inb[i - 2]) stat[31] += uabs64((int64_t)qb[i] - qb[i - 2]);
      }
  int64_t mean = sum / (int64_t)n;
  if ((sum % (int64_t)n) != 0 && sum < 0) mean -= 1; /* floor */
  for (int i = 0; i < 512; i++)
    if (inb[i]) stat[23] += uabs64((int64_t)qb[i] - mean);
  stat[24] = (uint64_t)(mx - mn);
  stat[26] = cin[1];
  stat[27] = cin[2];
  stat[28] = cin[4];
  stat[29] = n;
  stat[30] = uabs64(qb[0]);
  for (int f = 0; f < ORC_NFEAT; f++) feat[f] = orc_f32_to_bf16(orc_log2fix(stat[f]));
}

/* Selector network weights, all bfloat16 bits: W1[64][32], b1[64],
 * W2[4][64], b2[4] (2372 values). */
#define ORC_W1 0
#define ORC_B1 (ORC_W1 + ORC_HID * ORC_NFEAT)
#define ORC_W2 (ORC_B1 + ORC_HID)
#define ORC_B2 (ORC_W2 + ORC_NPRED * ORC_HID)
#define ORC_NW (ORC_B2 + ORC_NPRED)

/* Inference: h_j = bf16(max(0, fma chain over k of W1[j][k] f[k] starting
 * from b1[j])), logits_i = fma chain over j of W2[i][j] h_j starting from
 * b2[i]; binary32 fmaf in index order; argmax with ties to the lowest id. */
int orc_mlp_infer(const uint16_t *w, const uint16_t feat[ORC_NFEAT], float logits[ORC_NPRED]) {
  float h[ORC_HID];
  for (int j = 0; j < ORC_HID; j++) {
    float acc = orc_bf16_to_f32(w[ORC_B1 + j]);
    for (int k = 0; k < ORC_NFEAT; k++)
      acc = fmaf(orc_bf16_to_f32(w[ORC_W1 + j * ORC_NFEAT + k]), orc_bf16_to_f32(feat[k]), acc);
    if (!(acc > 0.0f)) acc = 0.0f;
    h[j] = orc_bf16_to_f32(orc_f32_to_bf16(acc));
  }
  int best = 0;
  for (int i = 0; i < ORC_NPRED; i++) {
    float acc = orc_bf16_to_f32(w[ORC_B2 + i]);
    for (int j = 0; j < ORC_HID; j++) acc = fmaf(orc_bf16_to_f32(w[ORC_W2 + i * ORC_HID + j]), h[j], acc);
    logits[i] = acc;
    if (acc > logits[best]) best = i;
  }
  return best;
}

/* Training objective in double: z = b1 + W1 f, h = max(0, z),
 * logits = b2 + W2 h, loss = mean over the minibatch of -log softmax(logits)
 * at the label; analytic gradients with respect to all parameters (the
 * weights are the bfloat16 values, as doubles).  grad has ORC_NW entries. */
double orc_mlp_loss_grad(const uint16_t *w, const uint16_t *feat, const uint8_t *label, uint64_t nb, double *grad) {
  double W[ORC_NW];
  for (int i = 0; i < ORC_NW; i++) W[i] = (double)orc_bf16_to_f32(w[i]);
  if (grad) memset(grad, 0, ORC_NW * sizeof(double));
  double loss = 0.0;
  for (uint64_t s = 0; s < nb; s++) {
    const uint16_t *f16 = feat + s * ORC_NFEAT;
    double f[ORC_NFEAT], z[ORC_HID], h[ORC_HID], lg[ORC_NPRED], p[ORC_NPRED];
    for (int k = 0; k < ORC_NFEAT; k++) f[k] = (double)orc_bf16_to_f32(f16[k]);
    for (int j = 0; j < ORC_HID; j++) {
      double acc = W[ORC_B1 + j];
      for (int k = 0; k < ORC_NFEAT; k++) acc += W[ORC_W1 + j * ORC_NFEAT + k] * f[k];
      z[j] = acc;
      h[j] = acc > 0.0 ? acc : 0.0;
    }
    double mxl = -1e300;
    for (int i = 0; i < ORC_NPRED; i++) {
      double acc = W[ORC_B2 + i];
      for (int j = 0; j < ORC_HID; j++) acc += W[ORC_W2 + i * ORC_HID + j] * h[j];
      lg[i] = acc;
      if (acc > mxl) mxl = acc;
    }
    double den = 0.0;
    for (int i = 0; i < ORC_NPRED; i++) { p[i] = exp(lg[i] - mxl); den += p[i]; }
    for (int i = 0; i < ORC_NPRED; i++) p[i] /= den;
    loss += -log(p[label[s]]);
    if (!grad) continue;
    double dl[ORC_NPRED], dh[ORC_HID];
    for (int i = 0; i < ORC_NPRED; i++) dl[i] = (p[i] - (i == label[s] ? 1.0 : 0.0)) / (double)nb;
    for (int i = 0; i < ORC_NPRED; i++) {
      grad[ORC_B2 + i] += dl[i];
      for (int j = 0; j < ORC_HID; j++) grad[ORC_W2 + i * ORC_HID + j] += dl[i] * h[j];
    }
    for (int j = 0; j < ORC_HID; j++) {
      double a = 0.0;
      for (int i = 0; i < ORC_NPRED; i++) a += W[ORC_W2 + i * ORC_HID + j] * dl[i];
      dh[j] = z[j] > 0.0 ? a : 0.0;
      grad[ORC_B1 + j] += dh[j];
      for (int k = 0; k < ORC_NFEAT; k++) grad[ORC_W1 + j * ORC_NFEAT + k] += dh[j] * f[k];
    }
  }
  return loss / (double)nb;
}

/* One step of Adam (Kingma and Ba, "Adam: A method for stochastic
 * optimization", ICLR 2015, Algorithm 1), step number t >= 1, in double, on
 * n parameters:
 *   m <- b1 m + (1 - b1) g
 *   v <- b2 v + (1 - b2) g^2
 *   mhat = m / (1 - b1^t),  vhat = v / (1 - b2^t)
 *   w <- w - lr mhat / (sqrt(vhat) + eps)
 * (the selector's optimizer on its float32 master weights). */
void orc_adam_step(double *w, const double *g, double *m, double *v, uint64_t n, uint32_t t, double lr, double b1,
                   double b2, double eps) {
  const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
  for (uint64_t i = 0; i < n; i++) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    const double mhat = m[i] / c1, vhat = v[i] / c2;
    w[i] = w[i] - lr * mhat / (sqrt(vhat) + eps);
  }
}

/* The same loss with the weights given as doubles (for finite differences). */
double orc_mlp_loss_double(const double *W, const uint16_t *feat, const uint8_t *label, uint64_t nb) {
  double loss = 0.0;
  for (uint64_t s = 0; s < nb; s++) {
    const uint16_t *f16 = feat + s * ORC_NFEAT;
    double f[ORC_NFEAT], h[ORC_HID], lg[ORC_NPRED];
    for (int k = 0; k < ORC_NFEAT; k++) f[k] = (double)orc_bf16_to_f32(f16[k]);
    for (int j = 0; j < ORC_HID; j++) {
      double acc = W[ORC_B1 + j];
      for (int k = 0; k < ORC_NFEAT; k++) acc += W[ORC_W1 + j * ORC_NFEAT + k] * f[k];
      h[j] = acc > 0.0 ? acc : 0.0;
    }
    double mxl = -1e300, den = 0.0;
    for (int i = 0; i < ORC_NPRED; i++) {
      double acc = W[ORC_B2 + i];
      for (int j = 0; j < ORC_HID; j++) acc += W[ORC_W2 + i * ORC_HID + j] * h[j];
      lg[i] = acc;
      if (acc > mxl) mxl = acc;
    }
    for (int i = 0; i < ORC_NPRED; i++) den += exp(lg[i] - mxl);
    loss += -(lg[label[s]] - mxl - log(den));
  }
  return loss / (double)nb;
}

/* Labels and features of every block of a 3D field (for training and for
 * the stage tests): exhaustive-trial label, the 4 trial costs and the 32
 * bfloat16 features. */
int orc_field_blocks(const float *x, const uint64_t dims[3], uint32_t eb_mode, double eb, uint32_t R, uint8_t *label,
                     uint64_t *costs, uint16_t *feat) {
  uint64_t n;
  int st = check_args(3, dims, &n);
  if (st) return st;
  double eb_abs = eb;
  if (eb_mode == 1) {
    float lo, hi;
    int same;
    if (!orc_range(x, n, &lo, &hi, &same) || hi == lo) return ORC_EUNSUPPORTED;
    eb_abs = eb * ((double)hi - (double)lo);
  }
  float ebx2, inv2eb, eb_chk;
  orc_constants(eb_abs, &ebx2, &inv2eb, &eb_chk);
  int32_t *q = (int32_t *)malloc(n * 4);
  uint8_t *exc = (uint8_t *)malloc(n);
  if (!q || !exc) { free(q); free(exc); return ORC_ENOMEM; }
  orc_prequant(x, n, inv2eb, ebx2, eb_chk, q, exc);
  grid_t g;
  make_grid(3, dims, &g);
  int32_t qb[512], cq[8];
  uint8_t inb[512], cin[8];
  uint64_t fidx[512], stat[ORC_NFEAT];
  for (uint64_t blk = 0; blk < g.n_blocks; blk++) {
    gather_block(&g, blk, q, qb, inb, fidx);
    block_corners(&g, blk, q, cq, cin);
    uint64_t c[ORC_NPRED];
    int best = orc_block_costs(qb, inb, cq, cin, R, c);
    if (label) label[blk] = (uint8_t)best;
    if (costs) memcpy(costs + blk * ORC_NPRED, c, sizeof(c));
    if (feat) orc_block_features(qb, inb, cq, cin, R, stat, feat + blk * ORC_NFEAT);
  }
  free(q);
  free(exc);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Whole pipeline: compress                                                  */
/* ------------------------------------------------------------------------ */

uint64_t orc_compress_bound(uint32_t ndim, const uint64_t dims[3]) {
  uint64_t n = 1;
  for (uint32_t a = 0; a < ndim; a++) n *= dims[a];
  return align16(HDR + 4 * n);
}

static int check_args(uint32_t ndim, const uint64_t dims[3], uint64_t *n) {
  if (ndim < 1 || ndim > 3) return ORC_EINVAL;
  uint64_t v = 1;
  for (uint32_t a = 0; a < ndim; a++) {
    if (dims[a] == 0 || dims[a] >= ((uint64_t)1 << 32)) return ORC_EINVAL;
    v *= dims[a];
    if (v >= ((uint64_t)1 << 32)) return ORC_EINVAL;
  }
  *n = v;
  return ORC_OK;
}

static int write_raw(const float *x, uint64_t n, uint32_t ndim, uint32_t ebmode, const uint64_t dims[3],
                     double eb, uint8_t *out, uint64_t cap, uint64_t *out_bytes) {
  uint64_t total = HDR + 4 * n;
  if (cap < total) return ORC_EBUFFER;
  put_min_header(out, F_RAW, ndim, ebmode, dims, eb, total);
  memcpy(out + HDR, x, 4 * n);
  *out_bytes = total;
  return ORC_OK;
}

/* Compress x (field order, x fastest) with predictor `pred` (0 Lorenzo-1,
 * 1 Lorenzo-2 in any dimension; 2 interpolation linear, 3 interpolation
 * cubic, 16 per-block choice by the selector network with bfloat16 weights
 * `w`, 17 per-block choice by exhaustive trial, 3D only) and radius R.
 * eb_mode 0 = ABS, 1 = REL (value range over finite values).  Output is the
 * complete stream; with a per-block choice it carries the 2-bit predictor id
 * of every block. */
/* ------------------------------------------------------------------------ */
/* Bit-shuffle + zero-word encoder (FZMod-Speed, §3.2-§3.3: the encoder of  */
/* FZ-GPU, in place of the Huffman coder)                                   */
/* ------------------------------------------------------------------------ */
/* The codes (0..2R-1, code 0 = outlier) become residuals d = code - R and
 * then zig-zag values v = 2d (d >= 0) or -2d - 1 (d < 0), so that small
 * residuals have few nonzero bits (v < 2R).  Each run of 64 codes is read as
 * 32 rows of 32 bits, row r = v[2r] | v[2r+1] << 16, and the 32x32 bit
 * matrix is transposed: column word b has bit r = bit b of row r.  A 32-bit
 * map per run flags the nonzero column words; only those are stored, in
 * column order.  A tile of 1024 codes (16 runs) is one chunk: its stored
 * length is 32 bits per word it stores. */
#define SHUF_RUN 64u
#define SHUF_TILE 1024u

static uint32_t zigzag(int32_t d) { return d >= 0 ? (uint32_t)d << 1 : ((uint32_t)(-(d + 1)) << 1) | 1u; }
static int32_t unzigzag(uint32_t v) { return (v & 1u) ? -(int32_t)(v >> 1) - 1 : (int32_t)(v >> 1); }

/* Encodes npad codes: maps[npad/64], words (capacity cap_words), per-tile
 * lengths in bits; returns the number of words, or ~0 if cap_words is too
 * small. */
static uint64_t shuf_encode(const uint16_t *codes, uint64_t npad, uint32_t R, uint32_t *maps, uint32_t *words,
                            uint64_t cap_words, uint32_t *tile_bits) {
  uint64_t nw = 0;
  const uint64_t n_runs = npad / SHUF_RUN, n_tiles = (npad + SHUF_TILE - 1) / SHUF_TILE;
  for (uint64_t t = 0; t < n_tiles; t++) tile_bits[t] = 0;
  for (uint64_t k = 0; k < n_runs; k++) {
    uint32_t row[32];
    for (int r = 0; r < 32; r++) {
      uint32_t v0 = zigzag((int32_t)codes[k * SHUF_RUN + 2 * r] - (int32_t)R);
      uint32_t v1 = zigzag((int32_t)codes[k * SHUF_RUN + 2 * r + 1] - (int32_t)R);
      row[r] = v0 | (v1 << 16);
    }
    uint32_t map = 0;
    for (int b = 0; b < 32; b++) {
      uint32_t w = 0;
      for (int r = 0; r < 32; r++) w |= ((row[r] >> b) & 1u) << r;
      if (w) {
        map |= 1u << b;
        if (nw >= cap_words) return ~0ull;
        words[nw++] = w;
        tile_bits[k * SHUF_RUN / SHUF_TILE] += 32;
      }
    }
    maps[k] = map;
  }
  return nw;
}

/* Inverse of shuf_encode for one tile: reads the tile's runs from maps and
 * words[*pw ..], checks that the tile uses exactly tile_bits bits and that
 * every value is below 2R; writes the codes. */
static int shuf_decode_tile(const uint8_t *maps_b, const uint8_t *words_b, uint64_t n_words, uint64_t *pw,
                            uint64_t t, uint64_t npad, uint32_t R, uint32_t tile_bits, uint16_t *codes) {
  if (tile_bits % 32) return ORC_ECORRUPT;
  const uint64_t w_end = *pw + tile_bits / 32;
  if (w_end > n_words) return ORC_ECORRUPT;
  for (uint64_t k = t * (SHUF_TILE / SHUF_RUN); k < (t + 1) * (SHUF_TILE / SHUF_RUN) && k * SHUF_RUN < npad; k++) {
    uint32_t map = get_u32(maps_b + 4 * k), row[32];
    memset(row, 0, sizeof(row));
    for (int b = 0; b < 32; b++) {
      if (!((map >> b) & 1u)) continue;
      if (*pw >= w_end) return ORC_ECORRUPT;
      uint32_t w = get_u32(words_b + 4 * *pw);
      (*pw)++;
      for (int r = 0; r < 32; r++) row[r] |= ((w >> r) & 1u) << b;
    }
    for (int r = 0; r < 32; r++) {
      uint32_t v0 = row[r] & 0xffffu, v1 = row[r] >> 16;
      if (v0 >= 2 * R || v1 >= 2 * R) return ORC_ECORRUPT;
      codes[k * SHUF_RUN + 2 * r] = (uint16_t)(unzigzag(v0) + (int32_t)R);
      codes[k * SHUF_RUN + 2 * r + 1] = (uint16_t)(unzigzag(v1) + (int32_t)R);
    }
  }
  return *pw == w_end ? ORC_OK : ORC_ECORRUPT;
}

/* Huffman chunk sizes of the format (symbols per chunk; chunk j covers
 * code-stream symbols [jC, min((j+1)C, Npad))): the block size, a power-of-
 * two multiple of it up to 4096, for 3D 64 (one 8x8 plane of a block), or,
 * for 2D with the first-order Lorenzo predictor (pred 0), 128, 256 or 512
 * (4, 8 or 16 rows of a 32x32 block).  The chunking only decides where
 * chunk_bits cuts the bitstream: the bitstream itself does not depend on C. */
static int chunk_valid(uint32_t ndim, uint64_t bsize, uint64_t C, uint32_t pred) {
  if (C == bsize) return 1;
  if (ndim == 3 && C == 64) return 1;
  if (ndim == 2 && pred == 0 && (C == 128 || C == 256 || C == 512)) return 1;
  return C > bsize && C <= 4096 && (C % bsize) == 0 && (C & (C - 1)) == 0;
}

int orc_compress_full(const float *x, uint32_t ndim, const uint64_t dims[3], uint32_t eb_mode, double eb,
                      uint32_t pred, uint32_t R, const uint16_t *w, uint32_t chunk, uint32_t encoder, uint8_t *out,
                      uint64_t cap, uint64_t *out_bytes);

int orc_compress_chunk(const float *x, uint32_t ndim, const uint64_t dims[3], uint32_t eb_mode, double eb,
                       uint32_t pred, uint32_t R, const uint16_t *w, uint32_t chunk, uint8_t *out, uint64_t cap,
                       uint64_t *out_bytes) {
  return orc_compress_full(x, ndim, dims, eb_mode, eb, pred, R, w, chunk, 0, out, cap, out_bytes);
}

int orc_compress_pred(const float *x, uint32_t ndim, const uint64_t dims[3], uint32_t eb_mode, double eb,
                      uint32_t pred, uint32_t R, const uint16_t *w, uint8_t *out, uint64_t cap,
                      uint64_t *out_bytes) {
  return orc_compress_chunk(x, ndim, dims, eb_mode, eb, pred, R, w, 0, out, cap, out_bytes);
}

/* The whole compression path.  encoder 0: Huffman with chunks of `chunk`
 * symbols (0: the block size); encoder 1: the bit-shuffle + zero-word
 * encoder (Lorenzo predictors only, chunk 0 or 1024). */
int orc_compress_full(const float *x, uint32_t ndim, const uint64_t dims[3], uint32_t eb_mode, double eb,
                      uint32_t pred, uint32_t R, const uint16_t *w, uint32_t chunk, uint32_t encoder, uint8_t *out,
                      uint64_t cap, uint64_t *out_bytes) {
  uint64_t n;
  int st = check_args(ndim, dims, &n);
  if (st) return st;
  if (!(eb > 0.0) || !isfinite(eb) || eb_mode > 1) return ORC_EINVAL;
  if (!(pred <= 4 || pred == 16 || pred == 17)) return ORC_EINVAL;
  if (pred >= 2 && ndim != 3) return ORC_EUNSUPPORTED;
  if (pred == 16 && !w) return ORC_EINVAL;
  if (R < 2 || R > 512) return ORC_EINVAL;
  if (encoder > 1) return ORC_EINVAL;
  if (encoder == 1) {
    if (pred > 1 || (chunk && chunk != SHUF_TILE)) return ORC_EUNSUPPORTED;
    chunk = SHUF_TILE;
  } else {
    uint32_t b[3];
    orc_block_shape(ndim, b);
    if (chunk && !chunk_valid(ndim, (uint64_t)b[0] * b[1] * b[2], chunk, pred)) return ORC_EUNSUPPORTED;
  }
  const int sel = pred >= 16;
  uint64_t dd[3] = {1, 1, 1};
  for (uint32_t a = 0; a < ndim; a++) dd[a] = dims[a];

  /* step 1: error bound */
  double eb_abs = eb;
  if (eb_mode == 1) {
    float lo, hi;
    int same;
    int anyf = orc_range(x, n, &lo, &hi, &same);
    if (!anyf || hi == lo) {
      if (same) {
        uint64_t total = HDR + 16;
        if (cap < total) return ORC_EBUFFER;
        put_min_header(out, F_CONST, ndim, eb_mode, dd, eb, total);
        memset(out + HDR, 0, 16);
        put_u32(out + HDR, f2u(x[0]));
        *out_bytes = total;
        return ORC_OK;
      }
      return write_raw(x, n, ndim, eb_mode, dd, eb, out, cap, out_bytes);
    }
    eb_abs = eb * ((double)hi - (double)lo);
  }
  /* step 2: constants */
  float ebx2, inv2eb, eb_chk;
  orc_constants(eb_abs, &ebx2, &inv2eb, &eb_chk);

  /* step 3: prequant, field order */
  int32_t *q = (int32_t *)malloc(n * sizeof(int32_t));
  uint8_t *exc = (uint8_t *)malloc(n);
  if (!q || !exc) { free(q); free(exc); return ORC_ENOMEM; }
  orc_prequant(x, n, inv2eb, ebx2, eb_chk, q, exc);

  /* steps 4-7: blocks, residuals, codes, outliers, exceptions, histogram;
   * code-stream positions are 32-bit in the format (outlier and exception
   * indices) */
  grid_t g;
  make_grid(ndim, dd, &g);
  if (g.npad > 0xffffffffull) { free(q); free(exc); return ORC_EUNSUPPORTED; }
  uint16_t *codes = (uint16_t *)malloc(g.npad * sizeof(uint16_t));
  int32_t *anchors = (int32_t *)malloc(g.n_blocks * sizeof(int32_t));
  uint64_t cap_list = n / 8;
  uint32_t *oidx = (uint32_t *)malloc((cap_list + 1) * 4);
  int32_t *oval = (int32_t *)malloc((cap_list + 1) * 4);
  uint32_t *eidx = (uint32_t *)malloc((cap_list + 1) * 4);
  uint32_t *eval = (uint32_t *)malloc((cap_list + 1) * 4);
  int32_t *qb = (int32_t *)malloc(g.bsize * 4);
  uint8_t *inb = (uint8_t *)malloc(g.bsize);
  uint64_t *fidx = (uint64_t *)malloc(g.bsize * 8);
  int64_t *delta = (int64_t *)malloc(g.bsize * 8);
  uint8_t *ids = (uint8_t *)calloc(g.n_blocks / 4 + 1, 1);
  uint64_t hist[ORC_MAXSYM];
  memset(hist, 0, sizeof(hist));
  uint64_t n_out = 0, n_exc = 0;
  int overflow = 0;
  /* full-field interpolation: the residuals of the whole field first */
  int64_t *gres = pred == 4 ? (int64_t *)malloc(n * sizeof(int64_t)) : NULL;
  if (!codes || !anchors || !oidx || !oval || !eidx || !eval || !qb || !inb || !fidx || !delta || !ids ||
      (pred == 4 && !gres)) {
    st = ORC_ENOMEM;
    goto done;
  }
  if (pred == 4) {
    for (uint64_t i = 0; i < n; i++) gres[i] = q[i];
    st = orc_ginterp_field(0, dd, gres);
    if (st) goto done;
  }
  for (uint64_t blk = 0; blk < g.n_blocks; blk++) {
    gather_block(&g, blk, q, qb, inb, fidx);
    int32_t cq[8];
    uint8_t cin[8];
    int pid = (int)pred;
    if (ndim == 3) block_corners(&g, blk, q, cq, cin);
    if (pred == 17) {
      uint64_t c[ORC_NPRED];
      pid = orc_block_costs(qb, inb, cq, cin, R, c);
    } else if (pred == 16) {
      uint64_t stat[ORC_NFEAT];
      uint16_t feat[ORC_NFEAT];
      float lg[ORC_NPRED];
      orc_block_features(qb, inb, cq, cin, R, stat, feat);
      pid = orc_mlp_infer(w, feat, lg);
    }
    if (sel) ids[blk >> 2] |= (uint8_t)(pid << (2 * (blk & 3)));
    if (pid == 4)
      for (uint64_t i = 0; i < g.bsize; i++) delta[i] = inb[i] ? gres[fidx[i]] : 0;
    else
      block_residual(pid, ndim, g.b, qb, inb, cq, cin, delta);
    for (uint64_t i = 0; i < g.bsize; i++) {
      uint64_t pos = blk * g.bsize + i;
      uint16_t c;
      if (!inb[i]) c = (uint16_t)R;
      else if (i == 0) { anchors[blk] = (int32_t)delta[0]; c = (uint16_t)R; }
      else if (delta[i] > -(int64_t)R && delta[i] < (int64_t)R) c = (uint16_t)(delta[i] + R);
      else {
        c = 0;
        if (n_out < cap_list) { oidx[n_out] = (uint32_t)pos; oval[n_out] = (int32_t)delta[i]; }
        else overflow = 1;
        n_out++;
      }
      if (inb[i] && exc[fidx[i]]) {
        if (n_exc < cap_list) { eidx[n_exc] = (uint32_t)pos; eval[n_exc] = f2u(x[fidx[i]]); }
        else overflow = 1;
        n_exc++;
      }
      codes[pos] = c;
      hist[c]++;
    }
  }
  if (overflow || n_out + n_exc > cap_list) {
    st = write_raw(x, n, ndim, eb_mode, dd, eb, out, cap, out_bytes);
    goto done;
  }
  /* steps 8-9: codebook */
  uint32_t nsym = 2 * R;
  uint8_t len[ORC_MAXSYM];
  uint32_t code[ORC_MAXSYM];
  uint64_t total_bits = 0;
  const uint64_t npad = g.n_blocks * g.bsize;
  uint32_t *smaps = NULL, *swords = NULL, *stile = NULL;
  if (encoder == 0) {
    st = orc_huffman_lengths(hist, nsym, len);
    if (st) goto done;
    st = orc_canonical_codes(len, nsym, code);
    if (st) goto done;
    for (uint32_t s = 0; s < nsym; s++) total_bits += hist[s] * len[s];
  } else {
    /* step 10 (shuffle): the whole encoding first; its size decides the layout */
    const uint64_t cap_words = (npad / SHUF_RUN) * 32;
    smaps = (uint32_t *)malloc((npad / SHUF_RUN) * 4 + 4);
    swords = (uint32_t *)malloc(cap_words * 4 + 4);
    stile = (uint32_t *)malloc(((npad + SHUF_TILE - 1) / SHUF_TILE) * 4 + 4);
    if (!smaps || !swords || !stile) { st = ORC_ENOMEM; free(smaps); free(swords); free(stile); goto done; }
    total_bits = 32 * shuf_encode(codes, npad, R, smaps, swords, cap_words, stile);
  }

  /* layout */
  uint64_t C = chunk ? chunk : g.bsize;
  uint64_t n_chunks = (npad + C - 1) / C;
  uint64_t off_lens = HDR;
  /* Huffman: the code lengths; shuffle: the 32-bit word maps, one per 64 codes */
  uint64_t off_ids = align16(off_lens + (encoder ? 4 * (npad / SHUF_RUN) : nsym));
  uint64_t ids_bytes = sel ? (g.n_blocks + 3) / 4 : 0;
  uint64_t off_anch = align16(off_ids + ids_bytes);
  uint64_t off_cb = align16(off_anch + 4 * g.n_blocks);
  uint64_t off_oidx = align16(off_cb + 4 * n_chunks);
  uint64_t off_oval = align16(off_oidx + 4 * n_out);
  uint64_t off_eidx = align16(off_oval + 4 * n_out);
  uint64_t off_eval = align16(off_eidx + 4 * n_exc);
  uint64_t off_bits = align16(off_eval + 4 * n_exc);
  uint64_t n_words = (total_bits + 31) / 32;
  uint64_t total = align16(off_bits + 4 * n_words);
  if (total > HDR + 4 * n) {
    st = write_raw(x, n, ndim, eb_mode, dd, eb, out, cap, out_bytes);
    free(smaps); free(swords); free(stile);
    goto done;
  }
  if (cap < total) { st = ORC_EBUFFER; free(smaps); free(swords); free(stile); goto done; }
  memset(out, 0, total);
  uint8_t *h = out;
  put_u32(h + H_MAGIC, MAGIC);
  put_u16(h + H_VERSION, 1);
  put_u16(h + H_FLAGS, sel ? F_IDS : (encoder ? F_SHUF : 0));
  put_u32(h + H_NDIM, ndim);
  put_u32(h + H_EBMODE, eb_mode);
  for (int a = 0; a < 3; a++) put_u64(h + H_DIMS + 8 * a, dd[a]);
  put_u64(h + H_EB, d2u(eb));
  put_u64(h + H_EBABS, d2u(eb_abs));
  put_u32(h + H_EBX2, f2u(ebx2));
  put_u32(h + H_INV2EB, f2u(inv2eb));
  put_u32(h + H_EBCHK, f2u(eb_chk));
  put_u32(h + H_RADIUS, R);
  for (int a = 0; a < 3; a++) put_u32(h + H_BLOCK + 4 * a, g.b[a]);
  put_u32(h + H_PRED, pred);
  put_u32(h + H_CHUNK, (uint32_t)C);
  put_u64(h + H_NBLOCKS, g.n_blocks);
  put_u64(h + H_NCHUNKS, n_chunks);
  put_u64(h + H_NOUT, n_out);
  put_u64(h + H_NEXC, n_exc);
  put_u64(h + H_TBITS, total_bits);
  put_u64(h + H_OFF_LENS, off_lens);
  put_u64(h + H_OFF_IDS, sel ? off_ids : 0);
  put_u64(h + H_OFF_ANCH, off_anch);
  put_u64(h + H_OFF_CBITS, off_cb);
  put_u64(h + H_OFF_OIDX, off_oidx);
  put_u64(h + H_OFF_OVAL, off_oval);
  put_u64(h + H_OFF_EIDX, off_eidx);
  put_u64(h + H_OFF_EVAL, off_eval);
  put_u64(h + H_OFF_BITS, off_bits);
  put_u64(h + H_TOTAL, total);
  if (encoder == 0) memcpy(out + off_lens, len, nsym);
  else for (uint64_t k = 0; k < npad / SHUF_RUN; k++) put_u32(out + off_lens + 4 * k, smaps[k]);
  if (sel) memcpy(out + off_ids, ids, ids_bytes);
  for (uint64_t b = 0; b < g.n_blocks; b++) put_u32(out + off_anch + 4 * b, (uint32_t)anchors[b]);
  for (uint64_t i = 0; i < n_out; i++) {
    put_u32(out + off_oidx + 4 * i, oidx[i]);
    put_u32(out + off_oval + 4 * i, (uint32_t)oval[i]);
  }
  for (uint64_t i = 0; i < n_exc; i++) {
    put_u32(out + off_eidx + 4 * i, eidx[i]);
    put_u32(out + off_eval + 4 * i, eval[i]);
  }
  if (encoder == 1) {
    for (uint64_t j = 0; j < n_chunks; j++) put_u32(out + off_cb + 4 * j, stile[j]);
    for (uint64_t k = 0; k < n_words; k++) put_u32(out + off_bits + 4 * k, swords[k]);
    free(smaps); free(swords); free(stile);
    *out_bytes = total;
    st = ORC_OK;
    goto done;
  }
  /* step 10: chunked encode; chunk j = code-stream symbols [jC, (j+1)C) */
  uint32_t *words = (uint32_t *)calloc(n_words + 1, 4);
  if (!words) { st = ORC_ENOMEM; goto done; }
  uint64_t p = 0;
  for (uint64_t j = 0; j < n_chunks; j++) {
    uint64_t cb = 0;
    for (uint64_t i = j * C; i < (j + 1) * C && i < npad; i++) {
      put_bits(words, p, code[codes[i]], len[codes[i]]);
      p += len[codes[i]];
      cb += len[codes[i]];
    }
    put_u32(out + off_cb + 4 * j, (uint32_t)cb);
  }
  for (uint64_t w = 0; w < n_words; w++) put_u32(out + off_bits + 4 * w, words[w]);
  free(words);
  *out_bytes = total;
  st = ORC_OK;
done:
  free(q); free(exc); free(codes); free(anchors); free(oidx); free(oval); free(eidx); free(eval);
  free(qb); free(inb); free(fidx); free(delta); free(ids); free(gres);
  return st;
}

/* Lorenzo order k (1 or 2) for every block. */
int orc_compress(const float *x, uint32_t ndim, const uint64_t dims[3], uint32_t eb_mode, double eb,
                 uint32_t lorenzo_k, uint32_t R, uint8_t *out, uint64_t cap, uint64_t *out_bytes) {
  if (lorenzo_k < 1 || lorenzo_k > 2) return ORC_EUNSUPPORTED;
  return orc_compress_pred(x, ndim, dims, eb_mode, eb, lorenzo_k - 1, R, NULL, out, cap, out_bytes);
}

/* ------------------------------------------------------------------------ */
/* Step 11: decompress                                                       */
/* ------------------------------------------------------------------------ */

/* Decode one canonical codeword starting at bit p by walking lengths 1..14:
 * the first length l whose l-bit prefix v satisfies first[l] <= v < first[l] +
 * count[l] identifies symbol sorted[base[l] + v - first[l]]. */
static int decode_one(const uint32_t *w, uint64_t nbits_total, uint64_t *p, const uint32_t *first,
                      const uint32_t *count, const uint32_t *base, const uint16_t *sorted, uint32_t *sym) {
  uint32_t v = 0;
  for (int l = 1; l <= ORC_LMAX; l++) {
    if (*p + (uint64_t)l > nbits_total) return ORC_ECORRUPT;
    v = (v << 1) | get_bit(w, *p + l - 1);
    if (count[l] && v >= first[l] && v - first[l] < count[l]) {
      *sym = sorted[base[l] + (v - first[l])];
      *p += (uint64_t)l;
      return ORC_OK;
    }
  }
  return ORC_ECORRUPT;
}

int orc_stream_info(const uint8_t *in, uint64_t in_bytes, uint32_t *ndim, uint64_t dims[3], uint64_t *n) {
  if (in_bytes < HDR || get_u32(in + H_MAGIC) != MAGIC || get_u16(in + H_VERSION) != 1) return ORC_ECORRUPT;
  *ndim = get_u32(in + H_NDIM);
  for (int a = 0; a < 3; a++) dims[a] = get_u64(in + H_DIMS + 8 * a);
  return check_args(*ndim, dims, n) ? ORC_ECORRUPT : ORC_OK;
}

int orc_decompress(const uint8_t *in, uint64_t in_bytes, float *out, uint64_t out_cap_values) {
  uint32_t ndim;
  uint64_t dims[3], n;
  int st = orc_stream_info(in, in_bytes, &ndim, dims, &n);
  if (st) return st;
  if (out_cap_values < n) return ORC_EBUFFER;
  uint16_t flags = get_u16(in + H_FLAGS);
  uint64_t total = get_u64(in + H_TOTAL);
  if (total > in_bytes) return ORC_ECORRUPT;
  if (flags & F_RAW) {
    if (total != HDR + 4 * n) return ORC_ECORRUPT;
    memcpy(out, in + HDR, 4 * n);
    return ORC_OK;
  }
  if (flags & F_CONST) {
    if (total != HDR + 16) return ORC_ECORRUPT;
    float v = u2f(get_u32(in + HDR));
    for (uint64_t i = 0; i < n; i++) out[i] = v;
    return ORC_OK;
  }
  if (flags != 0 && flags != F_IDS && flags != F_SHUF) return ORC_EUNSUPPORTED;
  const int shuf = flags == F_SHUF;
  grid_t g;
  make_grid(ndim, dims, &g);
  uint32_t R = get_u32(in + H_RADIUS), nsym = 2 * R;
  uint32_t pred = get_u32(in + H_PRED);
  const int sel = flags == F_IDS;
  if (R < 2 || R > 512) return ORC_ECORRUPT;
  if (sel != (pred == 16 || pred == 17) || !(pred <= 4 || pred == 16 || pred == 17)) return ORC_ECORRUPT;
  if (pred >= 2 && ndim != 3) return ORC_ECORRUPT;
  if (shuf && pred > 1) return ORC_ECORRUPT;
  uint64_t o_ids = get_u64(in + H_OFF_IDS);
  for (int a = 0; a < 3; a++)
    if (get_u32(in + H_BLOCK + 4 * a) != g.b[a]) return ORC_ECORRUPT;
  float ebx2 = u2f(get_u32(in + H_EBX2));
  uint64_t nb = get_u64(in + H_NBLOCKS), nch = get_u64(in + H_NCHUNKS);
  uint64_t n_out = get_u64(in + H_NOUT), n_exc = get_u64(in + H_NEXC), tbits = get_u64(in + H_TBITS);
  uint64_t C = get_u32(in + H_CHUNK);
  const uint64_t npad = g.n_blocks * g.bsize;
  if (nb != g.n_blocks || !(shuf ? C == SHUF_TILE : chunk_valid(ndim, g.bsize, C, pred)) ||
      nch != (npad + C - 1) / C)
    return ORC_ECORRUPT;
  const uint64_t lens_bytes = shuf ? 4 * (npad / SHUF_RUN) : nsym;
  if (n_out > n || n_exc > n) return ORC_ECORRUPT;
  uint64_t o_len = get_u64(in + H_OFF_LENS), o_anch = get_u64(in + H_OFF_ANCH), o_cb = get_u64(in + H_OFF_CBITS);
  uint64_t o_oi = get_u64(in + H_OFF_OIDX), o_ov = get_u64(in + H_OFF_OVAL), o_ei = get_u64(in + H_OFF_EIDX);
  uint64_t o_ev = get_u64(in + H_OFF_EVAL), o_bits = get_u64(in + H_OFF_BITS);
  uint64_t n_words = (tbits + 31) / 32;
  if (sel && o_ids + (nb + 3) / 4 > total) return ORC_ECORRUPT;
  if (o_len + lens_bytes > total || o_anch + 4 * nb > total || o_cb + 4 * nch > total || o_oi + 4 * n_out > total ||
      o_ov + 4 * n_out > total || o_ei + 4 * n_exc > total || o_ev + 4 * n_exc > total ||
      o_bits + 4 * n_words > total)
    return ORC_ECORRUPT;
  uint8_t len[ORC_MAXSYM];
  uint32_t code[ORC_MAXSYM];
  /* canonical decode tables: per length the first code, count and the start
   * of its symbols in the (length, symbol)-sorted list */
  uint32_t first[ORC_LMAX + 1] = {0}, count[ORC_LMAX + 1] = {0}, base[ORC_LMAX + 1] = {0};
  uint16_t sorted[ORC_MAXSYM];
  if (!shuf) {
    memcpy(len, in + o_len, nsym);
    if (orc_canonical_codes(len, nsym, code)) return ORC_ECORRUPT;
    uint32_t ns = 0;
    for (int l = 1; l <= ORC_LMAX; l++) {
      base[l] = ns;
      for (uint32_t s = 0; s < nsym; s++)
        if (len[s] == l) {
          if (count[l] == 0) first[l] = code[s];
          count[l]++;
          sorted[ns++] = (uint16_t)s;
        }
    }
    if (ns == 0) return ORC_ECORRUPT;
  }
  uint32_t *words = (uint32_t *)malloc((n_words + 1) * 4);
  uint16_t *codes = (uint16_t *)malloc(npad * 2);
  int64_t *v = (int64_t *)malloc(g.bsize * 8);
  int32_t *qb = (int32_t *)malloc(g.bsize * 4);
  uint8_t *inb = (uint8_t *)malloc(g.bsize);
  uint64_t *fidx = (uint64_t *)malloc(g.bsize * 8);
  /* full-field interpolation: the residual field, inverted as a whole */
  int64_t *gres = pred == 4 ? (int64_t *)malloc(n * sizeof(int64_t)) : NULL;
  if (!words || !codes || !v || !qb || !inb || !fidx || (pred == 4 && !gres)) { st = ORC_ENOMEM; goto ddone; }
  for (uint64_t w = 0; w < n_words; w++) words[w] = get_u32(in + o_bits + 4 * w);
  /* step 11a: the code stream, chunk by chunk; each chunk must use exactly
   * its stored bit count */
  uint64_t p = 0, oc = 0, ec = 0;
  if (shuf) {
    uint64_t pw = 0;
    for (uint64_t j = 0; j < nch; j++) {
      st = shuf_decode_tile(in + o_len, in + o_bits, n_words, &pw, j, npad, R, get_u32(in + o_cb + 4 * j), codes);
      if (st) goto ddone;
    }
    if (pw != n_words || tbits != 32 * n_words) { st = ORC_ECORRUPT; goto ddone; }
    p = tbits;
  }
  for (uint64_t j = 0; j < nch && !shuf; j++) {
    uint64_t cb = get_u32(in + o_cb + 4 * j), p_end = p + cb;
    if (p_end > tbits) { st = ORC_ECORRUPT; goto ddone; }
    for (uint64_t i = j * C; i < (j + 1) * C && i < npad; i++) {
      uint32_t sym;
      if (decode_one(words, p_end, &p, first, count, base, sorted, &sym)) { st = ORC_ECORRUPT; goto ddone; }
      codes[i] = (uint16_t)sym;
    }
    if (p != p_end) { st = ORC_ECORRUPT; goto ddone; }
  }
  /* step 11b: per block, residuals (outliers from their list), anchors,
   * inverse prediction, dequantization and exceptions */
  for (uint64_t blk = 0; blk < nb; blk++) {
    gather_block(&g, blk, NULL, qb, inb, fidx);
    for (uint64_t i = 0; i < g.bsize; i++) {
      uint64_t pos = blk * g.bsize + i;
      const uint32_t sym = codes[pos];
      if (sym == 0) {
        if (oc >= n_out || get_u32(in + o_oi + 4 * oc) != pos) { st = ORC_ECORRUPT; goto ddone; }
        v[i] = (int32_t)get_u32(in + o_ov + 4 * oc);
        oc++;
      } else {
        v[i] = (int64_t)sym - (int64_t)R;
      }
    }
    v[0] += (int32_t)get_u32(in + o_anch + 4 * blk);
    int pid = sel ? (in[o_ids + (blk >> 2)] >> (2 * (blk & 3))) & 3 : (int)pred;
    if (pid == 4) {
      for (uint64_t i = 0; i < g.bsize; i++)
        if (inb[i]) gres[fidx[i]] = v[i];
      continue;
    }
    if (pid < 2) {
      orc_lorenzo_block_inverse(pid + 1, ndim, g.b, v);
    } else {
      /* corner anchors: origins of the neighbouring blocks */
      int32_t cq[8];
      uint8_t cin[8];
      uint64_t bxi = blk % g.nb[0], byi = (blk / g.nb[0]) % g.nb[1], bzi = blk / (g.nb[0] * g.nb[1]);
      for (int c = 0; c < 8; c++) {
        uint64_t X = bxi + (c & 1), Y = byi + ((c >> 1) & 1), Z = bzi + (c >> 2);
        cin[c] = (uint8_t)(X < g.nb[0] && Y < g.nb[1] && Z < g.nb[2]);
        cq[c] = cin[c] ? (int32_t)get_u32(in + o_anch + 4 * ((Z * g.nb[1] + Y) * g.nb[0] + X)) : 0;
      }
      orc_interp_block(pid == 3, 1, inb, cq, cin, v);
    }
    for (uint64_t i = 0; i < g.bsize; i++) {
      if (!inb[i]) continue;
      uint64_t pos = blk * g.bsize + i;
      float r = (float)(int32_t)v[i] * ebx2;
      if (ec < n_exc && get_u32(in + o_ei + 4 * ec) == pos) {
        r = u2f(get_u32(in + o_ev + 4 * ec));
        ec++;
      }
      out[fidx[i]] = r;
    }
  }
  if (pred == 4) {
    /* step 11c: inverse interpolation of the whole field, then
     * dequantization and exceptions in code-stream order */
    st = orc_ginterp_field(1, g.d, gres);
    if (st) goto ddone;
    for (uint64_t blk = 0; blk < nb; blk++) {
      gather_block(&g, blk, NULL, qb, inb, fidx);
      for (uint64_t i = 0; i < g.bsize; i++) {
        if (!inb[i]) continue;
        uint64_t pos = blk * g.bsize + i;
        float r = (float)(int32_t)gres[fidx[i]] * ebx2;
        if (ec < n_exc && get_u32(in + o_ei + 4 * ec) == pos) {
          r = u2f(get_u32(in + o_ev + 4 * ec));
          ec++;
        }
        out[fidx[i]] = r;
      }
    }
  }
  if (oc != n_out || ec != n_exc || p != tbits) st = ORC_ECORRUPT;
ddone:
  free(words); free(codes); free(v); free(qb); free(inb); free(fidx); free(gres);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Stage access for the tests: codes, histogram and lists of one field       */
/* ------------------------------------------------------------------------ */

/* Runs steps 1-7 and returns the block-major code stream (npad values), the
 * anchors, the histogram and the counts of outliers and exceptions. */
int orc_quantize_stage(const float *x, uint32_t ndim, const uint64_t dims[3], float inv2eb, float ebx2,
                       float eb_chk, uint32_t lorenzo_k, uint32_t R, uint16_t *codes, int32_t *anchors,
                       uint64_t *hist, uint64_t *n_out, uint64_t *n_exc) {
  uint64_t n;
  int st = check_args(ndim, dims, &n);
  if (st) return st;
  uint64_t dd[3] = {1, 1, 1};
  for (uint32_t a = 0; a < ndim; a++) dd[a] = dims[a];
  grid_t g;
  make_grid(ndim, dd, &g);
  int32_t *q = (int32_t *)malloc(n * 4);
  uint8_t *exc = (uint8_t *)malloc(n);
  int32_t *qb = (int32_t *)malloc(g.bsize * 4);
  uint8_t *inb = (uint8_t *)malloc(g.bsize);
  uint64_t *fidx = (uint64_t *)malloc(g.bsize * 8);
  int64_t *delta = (int64_t *)malloc(g.bsize * 8);
  if (!q || !exc || !qb || !inb || !fidx || !delta) st = ORC_ENOMEM;
  else {
    orc_prequant(x, n, inv2eb, ebx2, eb_chk, q, exc);
    memset(hist, 0, 2 * R * sizeof(uint64_t));
    *n_out = *n_exc = 0;
    for (uint64_t blk = 0; blk < g.n_blocks; blk++) {
      gather_block(&g, blk, q, qb, inb, fidx);
      orc_lorenzo_block((int)lorenzo_k, ndim, g.b, qb, inb, delta);
      for (uint64_t i = 0; i < g.bsize; i++) {
        uint16_t c;
        if (!inb[i]) c = (uint16_t)R;
        else if (i == 0) { anchors[blk] = (int32_t)delta[0]; c = (uint16_t)R; }
        else if (delta[i] > -(int64_t)R && delta[i] < (int64_t)R) c = (uint16_t)(delta[i] + R);
        else { c = 0; (*n_out)++; }
        if (inb[i] && exc[fidx[i]]) (*n_exc)++;
        codes[blk * g.bsize + i] = c;
        hist[c]++;
      }
    }
  }
  free(q); free(exc); free(qb); free(inb); free(fidx); free(delta);
  return st;
}

/* Encode a code stream with a given set of lengths (chunk = C symbols). */
int orc_encode(const uint16_t *codes, uint64_t n, uint64_t C, const uint8_t *len, uint32_t nsym,
               uint32_t *words, uint64_t n_words_cap, uint32_t *chunk_bits, uint64_t *total_bits) {
  uint32_t code[ORC_MAXSYM];
  if (orc_canonical_codes(len, nsym, code)) return ORC_ECORRUPT;
  uint64_t tb = 0;
  for (uint64_t i = 0; i < n; i++) {
    if (codes[i] >= nsym || !len[codes[i]]) return ORC_EINVAL;
    tb += len[codes[i]];
  }
  if ((tb + 31) / 32 > n_words_cap) return ORC_EBUFFER;
  memset(words, 0, ((tb + 31) / 32) * 4);
  uint64_t p = 0;
  for (uint64_t j = 0; j * C < n; j++) {
    uint64_t cb = 0;
    for (uint64_t i = j * C; i < n && i < (j + 1) * C; i++) {
      put_bits(words, p, code[codes[i]], len[codes[i]]);
      p += len[codes[i]];
      cb += len[codes[i]];
    }
    chunk_bits[j] = (uint32_t)cb;
  }
  *total_bits = tb;
  return ORC_OK;
}

/* Decode n symbols from a bit string with a given set of lengths. */
int orc_decode(const uint32_t *words, uint64_t total_bits, const uint8_t *len, uint32_t nsym, uint64_t n,
               uint16_t *codes) {
  uint32_t code[ORC_MAXSYM];
  if (orc_canonical_codes(len, nsym, code)) return ORC_ECORRUPT;
  uint32_t first[ORC_LMAX + 1] = {0}, count[ORC_LMAX + 1] = {0}, base[ORC_LMAX + 1] = {0};
  uint16_t sorted[ORC_MAXSYM];
  uint32_t ns = 0;
  for (int l = 1; l <= ORC_LMAX; l++) {
    base[l] = ns;
    for (uint32_t s = 0; s < nsym; s++)
      if (len[s] == l) {
        if (count[l] == 0) first[l] = code[s];
        count[l]++;
        sorted[ns++] = (uint16_t)s;
      }
  }
  uint64_t p = 0;
  for (uint64_t i = 0; i < n; i++) {
    uint32_t s;
    if (decode_one(words, total_bits, &p, first, count, base, sorted, &s)) return ORC_ECORRUPT;
    codes[i] = (uint16_t)s;
  }
  return p == total_bits ? ORC_OK : ORC_ECORRUPT;
}
