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

/* REL range: minimum and maximum over the finite values of x.  Returns the
 * number of finite values.  Also reports whether every value of x has the same
 * bit pattern (needed for the constant-field stream). */
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

/* Compress x (field order, x fastest) with Lorenzo order `lorenzo_k` (1 or 2)
 * and radius R.  eb_mode 0 = ABS, 1 = REL (value range over finite values).
 * Output is the complete stream. */
int orc_compress(const float *x, uint32_t ndim, const uint64_t dims[3], uint32_t eb_mode, double eb,
                 uint32_t lorenzo_k, uint32_t R, uint8_t *out, uint64_t cap, uint64_t *out_bytes) {
  uint64_t n;
  int st = check_args(ndim, dims, &n);
  if (st) return st;
  if (!(eb > 0.0) || !isfinite(eb) || eb_mode > 1) return ORC_EINVAL;
  if (lorenzo_k < 1 || lorenzo_k > 2) return ORC_EUNSUPPORTED;
  if (R < 2 || R > 512) return ORC_EINVAL;
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

  /* steps 4-7: blocks, residuals, codes, outliers, exceptions, histogram */
  grid_t g;
  make_grid(ndim, dd, &g);
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
  uint64_t hist[ORC_MAXSYM];
  memset(hist, 0, sizeof(hist));
  uint64_t n_out = 0, n_exc = 0;
  int overflow = 0;
  if (!codes || !anchors || !oidx || !oval || !eidx || !eval || !qb || !inb || !fidx || !delta) {
    st = ORC_ENOMEM;
    goto done;
  }
  for (uint64_t blk = 0; blk < g.n_blocks; blk++) {
    gather_block(&g, blk, q, qb, inb, fidx);
    orc_lorenzo_block((int)lorenzo_k, ndim, g.b, qb, inb, delta);
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
  st = orc_huffman_lengths(hist, nsym, len);
  if (st) goto done;
  st = orc_canonical_codes(len, nsym, code);
  if (st) goto done;
  uint64_t total_bits = 0;
  for (uint32_t s = 0; s < nsym; s++) total_bits += hist[s] * len[s];

  /* layout */
  uint64_t n_chunks = g.n_blocks, C = g.bsize;
  uint64_t off_lens = HDR;
  uint64_t off_ids = align16(off_lens + nsym);
  uint64_t off_anch = off_ids;
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
    goto done;
  }
  if (cap < total) { st = ORC_EBUFFER; goto done; }
  memset(out, 0, total);
  uint8_t *h = out;
  put_u32(h + H_MAGIC, MAGIC);
  put_u16(h + H_VERSION, 1);
  put_u16(h + H_FLAGS, 0);
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
  put_u32(h + H_PRED, lorenzo_k - 1);
  put_u32(h + H_CHUNK, (uint32_t)C);
  put_u64(h + H_NBLOCKS, g.n_blocks);
  put_u64(h + H_NCHUNKS, n_chunks);
  put_u64(h + H_NOUT, n_out);
  put_u64(h + H_NEXC, n_exc);
  put_u64(h + H_TBITS, total_bits);
  put_u64(h + H_OFF_LENS, off_lens);
  put_u64(h + H_OFF_IDS, 0);
  put_u64(h + H_OFF_ANCH, off_anch);
  put_u64(h + H_OFF_CBITS, off_cb);
  put_u64(h + H_OFF_OIDX, off_oidx);
  put_u64(h + H_OFF_OVAL, off_oval);
  put_u64(h + H_OFF_EIDX, off_eidx);
  put_u64(h + H_OFF_EVAL, off_eval);
  put_u64(h + H_OFF_BITS, off_bits);
  put_u64(h + H_TOTAL, total);
  memcpy(out + off_lens, len, nsym);
  for (uint64_t b = 0; b < g.n_blocks; b++) put_u32(out + off_anch + 4 * b, (uint32_t)anchors[b]);
  for (uint64_t i = 0; i < n_out; i++) {
    put_u32(out + off_oidx + 4 * i, oidx[i]);
    put_u32(out + off_oval + 4 * i, (uint32_t)oval[i]);
  }
  for (uint64_t i = 0; i < n_exc; i++) {
    put_u32(out + off_eidx + 4 * i, eidx[i]);
    put_u32(out + off_eval + 4 * i, eval[i]);
  }
  /* step 10: chunked encode; chunk j = code-stream symbols [jC, (j+1)C) */
  uint32_t *words = (uint32_t *)calloc(n_words + 1, 4);
  if (!words) { st = ORC_ENOMEM; goto done; }
  uint64_t p = 0;
  for (uint64_t j = 0; j < n_chunks; j++) {
    uint64_t cb = 0;
    for (uint64_t i = j * C; i < (j + 1) * C; i++) {
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
  free(qb); free(inb); free(fidx); free(delta);
  return st;
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
  if (flags != 0) return ORC_EUNSUPPORTED;
  grid_t g;
  make_grid(ndim, dims, &g);
  uint32_t R = get_u32(in + H_RADIUS), nsym = 2 * R;
  uint32_t pred = get_u32(in + H_PRED);
  if (R < 2 || R > 512 || pred > 1) return ORC_ECORRUPT;
  for (int a = 0; a < 3; a++)
    if (get_u32(in + H_BLOCK + 4 * a) != g.b[a]) return ORC_ECORRUPT;
  float ebx2 = u2f(get_u32(in + H_EBX2));
  uint64_t nb = get_u64(in + H_NBLOCKS), nch = get_u64(in + H_NCHUNKS);
  uint64_t n_out = get_u64(in + H_NOUT), n_exc = get_u64(in + H_NEXC), tbits = get_u64(in + H_TBITS);
  uint64_t C = get_u32(in + H_CHUNK);
  if (nb != g.n_blocks || nch != g.n_blocks || C != g.bsize) return ORC_ECORRUPT;
  if (n_out > n || n_exc > n) return ORC_ECORRUPT;
  uint64_t o_len = get_u64(in + H_OFF_LENS), o_anch = get_u64(in + H_OFF_ANCH), o_cb = get_u64(in + H_OFF_CBITS);
  uint64_t o_oi = get_u64(in + H_OFF_OIDX), o_ov = get_u64(in + H_OFF_OVAL), o_ei = get_u64(in + H_OFF_EIDX);
  uint64_t o_ev = get_u64(in + H_OFF_EVAL), o_bits = get_u64(in + H_OFF_BITS);
  uint64_t n_words = (tbits + 31) / 32;
  if (o_len + nsym > total || o_anch + 4 * nb > total || o_cb + 4 * nch > total || o_oi + 4 * n_out > total ||
      o_ov + 4 * n_out > total || o_ei + 4 * n_exc > total || o_ev + 4 * n_exc > total ||
      o_bits + 4 * n_words > total)
    return ORC_ECORRUPT;
  uint8_t len[ORC_MAXSYM];
  uint32_t code[ORC_MAXSYM];
  memcpy(len, in + o_len, nsym);
  if (orc_canonical_codes(len, nsym, code)) return ORC_ECORRUPT;
  /* canonical decode tables: per length the first code, count and the start
   * of its symbols in the (length, symbol)-sorted list */
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
  if (ns == 0) return ORC_ECORRUPT;
  uint32_t *words = (uint32_t *)malloc((n_words + 1) * 4);
  int64_t *v = (int64_t *)malloc(g.bsize * 8);
  int32_t *qb = (int32_t *)malloc(g.bsize * 4);
  uint8_t *inb = (uint8_t *)malloc(g.bsize);
  uint64_t *fidx = (uint64_t *)malloc(g.bsize * 8);
  if (!words || !v || !qb || !inb || !fidx) { st = ORC_ENOMEM; goto ddone; }
  for (uint64_t w = 0; w < n_words; w++) words[w] = get_u32(in + o_bits + 4 * w);
  uint64_t p = 0, oc = 0, ec = 0;
  for (uint64_t blk = 0; blk < nb; blk++) {
    uint64_t cb = get_u32(in + o_cb + 4 * blk), p_end = p + cb;
    if (p_end > tbits) { st = ORC_ECORRUPT; goto ddone; }
    gather_block(&g, blk, NULL, qb, inb, fidx);
    for (uint64_t i = 0; i < g.bsize; i++) {
      uint32_t sym;
      if (decode_one(words, p_end, &p, first, count, base, sorted, &sym)) { st = ORC_ECORRUPT; goto ddone; }
      uint64_t pos = blk * g.bsize + i;
      if (sym == 0) {
        if (oc >= n_out || get_u32(in + o_oi + 4 * oc) != pos) { st = ORC_ECORRUPT; goto ddone; }
        v[i] = (int32_t)get_u32(in + o_ov + 4 * oc);
        oc++;
      } else {
        v[i] = (int64_t)sym - (int64_t)R;
      }
    }
    if (p != p_end) { st = ORC_ECORRUPT; goto ddone; }
    v[0] += (int32_t)get_u32(in + o_anch + 4 * blk);
    orc_lorenzo_block_inverse((int)pred + 1, ndim, g.b, v);
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
  if (oc != n_out || ec != n_exc || p != tbits) st = ORC_ECORRUPT;
ddone:
  free(words); free(v); free(qb); free(inb); free(fidx);
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
