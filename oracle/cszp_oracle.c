/*
 * Scalar CPU oracle of the cuSZ+ compressor's data-parallel path
 * (arXiv 2105.12912).  TEST INFRASTRUCTURE ONLY: only tests/,
 * __graft_entry__.smoke() and the CPU-baseline leg of bench.py use it.
 *
 * Plain, sequential, single-threaded C.  Every stage is written from the paper's
 * definition (cited per function) or from a reading of it that is stated inline;
 * nothing is blocked, fused or reordered.  The decompressor rebuilds the field
 * with the sequential Lorenzo recurrence (Sec. II-A, cuSZ's per-chunk scheme),
 * not with prefix sums, so it is an independent check of the GPU's partial-sum
 * reconstruction (Sec. IV-B2).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (no fused multiply-adds anywhere except the explicit fmaf() of the MLP).
 *
 * Archive layout (little-endian; all sections 8-byte aligned)
 *   [0,128)        header (see write_header)
 *   codec[nblk]    u8 per codec block
 *   blk_bytes[nblk] u32 payload bytes per block (each a multiple of 4)
 *   records[n_rec] (u32 key, u32 val): key = slot*2 + kind; kind 0 = outlier
 *                  (val = delta as int32), kind 1 = verbatim patch (val = float bits)
 *   payload        per-block payloads, concatenated in block order
 *   books          code lengths: [1024] quant-code book if any HUFF block;
 *                  [1024] run-value book + [4096] run-length book if any RLE_HUFF block
 */
#include "cszp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NSYM_CODE 1024   /* 2 * radius for the largest radius, 512 */
#define NSYM_LEN 4096    /* run lengths 1..4096 (one codec block) */
#define SLOTS 4096       /* code-stream slots per codec block */
#define HDR 128
#define MAGIC 0x2B5A5343u /* "CSZ+" */
#define VERSION 2
#define MAXLEN 64

/* ------------------------------------------------------------------------------- */
/* geometry                                                                         */
/* ------------------------------------------------------------------------------- */

/*
 * Chunks (Sec. II-A "Step-1"; Sec. IV-B3): prediction restarts from zero at every
 * chunk edge.  1-D chunks are 256 and 2-D chunks 16x16 (Sec. IV-B3); the paper
 * gives no 3-D chunk size, the reading here is 8x8x8.
 * Codec blocks (a reading; the paper encodes chunkwise without fixing a size):
 * 1-D 4096, 2-D 64x64, 3-D 16x16x16, each a whole number of chunks.
 */
typedef struct {
  int ndim;
  uint64_t n[3];   /* extents z, y, x (x fastest) */
  uint64_t blk[3]; /* codec block extents */
  uint64_t chk[3]; /* Lorenzo chunk extents */
  uint64_t g[3];   /* blocks along each axis */
  uint64_t nblk, nelem;
} geom_t;

static int make_geom(int ndim, const uint64_t* dims, geom_t* g) {
  static const uint64_t B[4][3] = {{0, 0, 0}, {1, 1, 4096}, {1, 64, 64}, {16, 16, 16}};
  static const uint64_t C[4][3] = {{0, 0, 0}, {1, 1, 256}, {1, 16, 16}, {8, 8, 8}};
  if (ndim < 1 || ndim > 3 || !dims) return ORC_E_ARG;
  memset(g, 0, sizeof(*g));
  g->ndim = ndim;
  for (int d = 0; d < 3; d++) g->n[d] = 1;
  for (int i = 0; i < ndim; i++) {
    if (dims[i] == 0 || dims[i] >= (1ull << 31)) return ORC_E_ARG;
    g->n[3 - ndim + i] = dims[i];
  }
  g->nblk = 1;
  g->nelem = 1;
  for (int d = 0; d < 3; d++) {
    g->blk[d] = B[ndim][d];
    g->chk[d] = C[ndim][d];
    g->g[d] = (g->n[d] + g->blk[d] - 1) / g->blk[d];
    g->nblk *= g->g[d];
    g->nelem *= g->n[d];
  }
  /* slot indices times two must fit in 32 bits */
  if (g->nblk * SLOTS >= (1ull << 31)) return ORC_E_ARG;
  return ORC_OK;
}

/* Global (unchunked) Lorenzo prediction (the extension the paper's partial-sum proof
   allows, Sec. IV-B "Partial-Sum Lorenzo Reconstruction": the proof holds for a
   whole field): one chunk spans the field, so prediction reads zero only outside the
   field.  Codec blocks are unchanged. */
static void make_global(geom_t* g) {
  for (int d = 0; d < 3; d++) g->chk[d] = g->n[d];
}

/* origin and in-field extents of codec block b (blocks in row-major order) */
static void block_box(const geom_t* g, uint64_t b, uint64_t org[3], uint64_t w[3]) {
  uint64_t bi[3];
  bi[0] = b / (g->g[1] * g->g[2]);
  bi[1] = (b / g->g[2]) % g->g[1];
  bi[2] = b % g->g[2];
  for (int d = 0; d < 3; d++) {
    org[d] = bi[d] * g->blk[d];
    w[d] = g->n[d] - org[d];
    if (w[d] > g->blk[d]) w[d] = g->blk[d];
  }
}

static uint64_t block_count(const geom_t* g, uint64_t b) {
  uint64_t org[3], w[3];
  block_box(g, b, org, w);
  return w[0] * w[1] * w[2];
}

/* code-stream slot of element (z,y,x): 4096*block + row-major index among the
   block's in-field elements */
static uint64_t slot_of(const geom_t* g, uint64_t z, uint64_t y, uint64_t x) {
  uint64_t c[3] = {z, y, x}, bi[3], r[3];
  for (int d = 0; d < 3; d++) {
    bi[d] = c[d] / g->blk[d];
    r[d] = c[d] % g->blk[d];
  }
  uint64_t b = (bi[0] * g->g[1] + bi[1]) * g->g[2] + bi[2];
  uint64_t org[3], w[3];
  block_box(g, b, org, w);
  return b * SLOTS + (r[0] * w[1] + r[1]) * w[2] + r[2];
}

static uint64_t elem_of_slot(const geom_t* g, uint64_t slot) {
  uint64_t b = slot / SLOTS, j = slot % SLOTS, org[3], w[3];
  block_box(g, b, org, w);
  uint64_t z = org[0] + j / (w[1] * w[2]);
  uint64_t y = org[1] + (j / w[2]) % w[1];
  uint64_t x = org[2] + j % w[2];
  return (z * g->n[1] + y) * g->n[2] + x;
}

int orc_geometry(int ndim, const uint64_t* dims, uint64_t* nblk, uint64_t* nelem) {
  geom_t g;
  int st = make_geom(ndim, dims, &g);
  if (st) return st;
  if (nblk) *nblk = g.nblk;
  if (nelem) *nelem = g.nelem;
  return ORC_OK;
}

/* ------------------------------------------------------------------------------- */
/* error bound and prequantization                                                  */
/* ------------------------------------------------------------------------------- */

/* value range for the relative error bound (bounds relative to the value range: Sec. II-B table captions, Sec. V-C) */
int orc_value_range(const float* x, uint64_t n, float* vmin, float* vmax) {
  float lo = INFINITY, hi = -INFINITY;
  for (uint64_t i = 0; i < n; i++) {
    if (!isfinite(x[i])) return ORC_E_NONFINITE;
    if (x[i] < lo) lo = x[i];
    if (x[i] > hi) hi = x[i];
  }
  *vmin = lo;
  *vmax = hi;
  return ORC_OK;
}

/*
 * eb in single precision.  ABS: eb_d = eb.  REL: eb_d = eb * (max - min) in double.
 * eb_f is the largest float not above eb_d (so the bound never loosens),
 * ebx2_f = 2 eb_f (exact) and ebx2_r = fl32(1 / ebx2_f) computed in double.
 * The paper is silent on degenerate bounds; a zero, negative or non-finite bound
 * (e.g. a constant field in REL mode) is rejected as ORC_E_ARG.
 */
int orc_eb_params(int eb_mode, double eb, float vmin, float vmax, double* eb_d, float* eb_f,
                  float* ebx2_f, float* ebx2_r) {
  if (!(eb > 0.0) || !isfinite(eb)) return ORC_E_ARG;
  double d;
  if (eb_mode == ORC_EB_ABS) {
    d = eb;
  } else if (eb_mode == ORC_EB_REL) {
    double range = (double)vmax - (double)vmin;
    d = eb * range;
  } else {
    return ORC_E_ARG;
  }
  float f = (float)d;
  if ((double)f > d) f = nextafterf(f, 0.0f);
  if (!(f > 0.0f)) return ORC_E_ARG;
  float x2 = 2.0f * f;
  if (!isfinite(x2)) return ORC_E_ARG;
  float r = (float)(1.0 / (double)x2);
  if (!(r > 0.0f) || !isfinite(r)) return ORC_E_ARG;
  *eb_d = d;
  *eb_f = f;
  *ebx2_f = x2;
  *ebx2_r = r;
  return ORC_OK;
}

/*
 * |x - y| > eb decided exactly.  Here y = fl32(k * 2eb) for the k the prequantizer
 * considers, so y is 0 or has x's sign and lies within a factor 8 of x; the double
 * difference of two such floats is exact.
 */
static int exceeds(float x, float y, float eb) {
  double d = (double)x - (double)y;
  return fabs(d) > (double)eb;
}

/*
 * Prequantization (Sec. IV-A1, Alg. 1 prequantization step): d° = round(d / 2eb), so that
 * |d - d°*2eb| < eb in exact arithmetic.  In FP32 the product d*(1/2eb) and the
 * reconstruction fl32(d°*2eb) both round, so:
 *   k0 = nearest integer to fl32(x * ebx2_r), ties to even;
 *   if the reconstruction of k0 misses x by more than eb_f, try the neighbour
 *   integer on x's side; if neither meets the bound, keep k0 and mark the value
 *   for a verbatim patch (the SZ family's "unpredictable" fallback).
 * |fl32(x*ebx2_r)| must stay below 2^23 (float integers exact, Lorenzo sums in
 * int32); otherwise ORC_E_RANGE.
 */
int orc_prequant(float x, float eb_f, float ebx2_f, float ebx2_r, int32_t* k, int* patch) {
  if (!isfinite(x)) return ORC_E_NONFINITE;
  float v = x * ebx2_r;
  if (!(fabsf(v) < 8388608.0f)) return ORC_E_RANGE;
  int32_t k0 = (int32_t)rintf(v); /* nearest integer, ties to even (IEEE default mode) */
  float x0 = (float)k0 * ebx2_f;
  *patch = 0;
  if (!exceeds(x, x0, eb_f)) {
    *k = k0;
    return ORC_OK;
  }
  int32_t k1 = k0 + (x > x0 ? 1 : -1);
  float x1 = (float)k1 * ebx2_f;
  if (!exceeds(x, x1, eb_f)) {
    *k = k1;
    return ORC_OK;
  }
  *k = k0;
  *patch = 1;
  return ORC_OK;
}

/* ------------------------------------------------------------------------------- */
/* double-precision input (SZ's double-precision datasets, Sec. II-B and V-A; the    */
/* paper's kernels take FP32).  Everything after prequantization is the FP32 path.  */
/* ------------------------------------------------------------------------------- */

int orc_value_range_f64(const double* x, uint64_t n, double* vmin, double* vmax) {
  double lo = INFINITY, hi = -INFINITY;
  for (uint64_t i = 0; i < n; i++) {
    if (!isfinite(x[i])) return ORC_E_NONFINITE;
    if (x[i] < lo) lo = x[i];
    if (x[i] > hi) hi = x[i];
  }
  *vmin = lo;
  *vmax = hi;
  return ORC_OK;
}

/*
 * Bound and quantization step in double precision (a reading: the paper defines
 * prequantization only as d° = round(d / 2eb)).  ABS: eb_d = eb; REL: eb_d =
 * eb * (max - min).  The step is 2 eb_d shrunk by one part in 2^24,
 * step = fl64(2 eb_d * (1 - 2^-24)), and rstep = fl64(1 / step).  With |k| < 2^27 the
 * rounding of fl64(k * step) moves the reconstruction by at most 2^-53 * 2^28 eb_d
 * = 2^-25 eb_d, less than the 2^-24 eb_d the shrink leaves, so the nearest integer
 * always meets |x - fl64(k * step)| <= eb_d and no value needs a verbatim patch.
 */
int orc_eb_params_f64(int eb_mode, double eb, double vmin, double vmax, double* eb_d, double* step,
                      double* rstep) {
  if (!(eb > 0.0) || !isfinite(eb)) return ORC_E_ARG;
  double d;
  if (eb_mode == ORC_EB_ABS) {
    d = eb;
  } else if (eb_mode == ORC_EB_REL) {
    d = eb * (vmax - vmin);
  } else {
    return ORC_E_ARG;
  }
  if (!(d > 0.0) || !isfinite(d)) return ORC_E_ARG;
  double st = (2.0 * d) * (1.0 - 0x1p-24);
  double r = 1.0 / st;
  if (!(st > 0.0) || !isfinite(st) || !(r > 0.0) || !isfinite(r)) return ORC_E_ARG;
  *eb_d = d;
  *step = st;
  *rstep = r;
  return ORC_OK;
}

/* |x - y| > eb decided exactly for doubles: Knuth's TwoSum gives x - y = s + e
   exactly with s = fl64(x - y); |s| < eb or |s| > eb decides by monotonicity of
   rounding, |s| == eb by the sign of e. */
static int exceeds_f64(double x, double y, double eb) {
  double s = x - y;
  if (fabs(s) < eb) return 0;
  if (fabs(s) > eb) return 1;
  double bv = s - x;
  double e = (x - (s - bv)) + (-y - bv);
  return s > 0.0 ? e > 0.0 : e < 0.0;
}

/* Prequantization of one double (Sec. IV-A1 read for FP64): k0 = nearest integer
   (ties to even) to fl64(x * rstep); if fl64(k0 * step) misses x by more than eb_d,
   the neighbour on x's side (k0 is within one of the exact nearest integer, which
   always meets the bound).  |fl64(x * rstep)| must stay below 2^27 (Lorenzo sums in
   int32: 3-D residuals reach 8 |k|); otherwise ORC_E_RANGE. */
int orc_prequant_f64(double x, double eb_d, double step, double rstep, int32_t* k) {
  if (!isfinite(x)) return ORC_E_NONFINITE;
  double v = x * rstep;
  if (!(fabs(v) < 134217728.0)) return ORC_E_RANGE;
  int32_t k0 = (int32_t)rint(v);
  double x0 = (double)k0 * step;
  if (!exceeds_f64(x, x0, eb_d)) {
    *k = k0;
    return ORC_OK;
  }
  int32_t k1 = k0 + (x > x0 ? 1 : -1);
  if (!exceeds_f64(x, (double)k1 * step, eb_d)) {
    *k = k1;
    return ORC_OK;
  }
  return ORC_E_RANGE; /* unreachable by the step's margin */
}

/* ------------------------------------------------------------------------------- */
/* Lorenzo prediction (Sec. IV-B2 equations), chunk-local: a neighbour outside the  */
/* element's chunk reads as zero ("we initially predict from zeros")                */
/* ------------------------------------------------------------------------------- */

static int64_t kat(const int32_t* K, const geom_t* g, uint64_t z, uint64_t y, uint64_t x, int dz,
                   int dy, int dx) {
  if ((z % g->chk[0]) < (uint64_t)dz) return 0;
  if ((y % g->chk[1]) < (uint64_t)dy) return 0;
  if ((x % g->chk[2]) < (uint64_t)dx) return 0;
  return K[((z - dz) * g->n[1] + (y - dy)) * g->n[2] + (x - dx)];
}

static int64_t lorenzo_predict(const int32_t* K, const geom_t* g, uint64_t z, uint64_t y,
                               uint64_t x) {
  if (g->ndim == 1) {
    /* p_x = d_{x-1} */
    return kat(K, g, z, y, x, 0, 0, 1);
  }
  if (g->ndim == 2) {
    /* p_{y,x} = -d_{y-1,x-1} + d_{y-1,x} + d_{y,x-1} */
    return -kat(K, g, z, y, x, 0, 1, 1) + kat(K, g, z, y, x, 0, 1, 0) + kat(K, g, z, y, x, 0, 0, 1);
  }
  /* p_{z,y,x} = + d_{z-1,y-1,x-1} - d_{z-1,y-1,x} - d_{z,y-1,x-1} + d_{z,y-1,x}
                 - d_{z-1,y,x-1}   + d_{z-1,y,x}   + d_{z,y,x-1} */
  return +kat(K, g, z, y, x, 1, 1, 1) - kat(K, g, z, y, x, 1, 1, 0) - kat(K, g, z, y, x, 0, 1, 1) +
         kat(K, g, z, y, x, 0, 1, 0) - kat(K, g, z, y, x, 1, 0, 1) + kat(K, g, z, y, x, 1, 0, 0) +
         kat(K, g, z, y, x, 0, 0, 1);
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/*
 * Dual-quantization construction (Sec. IV-A1, Alg. 1 compression part, modified
 * scheme of Sec. IV-B1):  k = prequant(x);  delta = k - p(k)  (Alg. 1's residual step
 * prints p - d; the text, "delta = d° - p°", and the reconstruction d = p + q' fix
 * the sign as d - p); in range iff |delta| < radius (Alg. 1's range test omits the
 * absolute value): q = delta +
 * radius; otherwise q = 0 and delta itself is the outlier (the cuSZ+ change).
 * Codes go to the block-major code stream; records are sorted by key.
 */
/* Residuals, codes and records from the prequantized integers K[nelem] (raster
   order); P[e] marks a verbatim patch of the value patch_vals[e] (FP32 only; P may
   be NULL). */
static int construct_k(const int32_t* K, const uint8_t* P, const float* patch_vals, const geom_t* gp,
                       uint32_t radius, uint16_t* codes, uint32_t* rec_key, uint32_t* rec_val,
                       uint64_t rec_cap, uint64_t* n_rec, uint32_t* hist) {
  const geom_t g = *gp;
  uint64_t n = g.nelem;
  uint64_t* recs = (uint64_t*)malloc((2 * n + 1) * sizeof(uint64_t));
  if (!recs) return ORC_E_CAPACITY;
  memset(codes, 0, g.nblk * SLOTS * sizeof(uint16_t));
  memset(hist, 0, NSYM_CODE * sizeof(uint32_t));
  uint64_t nr = 0;
  const int64_t r = (int64_t)radius;
  for (uint64_t z = 0; z < g.n[0]; z++)
    for (uint64_t y = 0; y < g.n[1]; y++)
      for (uint64_t xx = 0; xx < g.n[2]; xx++) {
        uint64_t e = (z * g.n[1] + y) * g.n[2] + xx;
        int64_t delta = (int64_t)K[e] - lorenzo_predict(K, &g, z, y, xx);
        uint64_t slot = slot_of(&g, z, y, xx);
        uint16_t q;
        if (delta > -r && delta < r) {
          q = (uint16_t)(delta + r);
        } else {
          q = 0;
          uint32_t dv = (uint32_t)(int32_t)delta;
          recs[nr++] = ((slot * 2 + 0) << 32) | dv;
        }
        codes[slot] = q;
        hist[q]++;
        if (P && P[e]) {
          uint32_t bits;
          memcpy(&bits, &patch_vals[e], 4);
          recs[nr++] = ((slot * 2 + 1) << 32) | bits;
        }
      }
  qsort(recs, nr, sizeof(uint64_t), cmp_u64);
  *n_rec = nr;
  if (nr > rec_cap) {
    free(recs);
    return ORC_E_CAPACITY;
  }
  for (uint64_t i = 0; i < nr; i++) {
    rec_key[i] = (uint32_t)(recs[i] >> 32);
    rec_val[i] = (uint32_t)(recs[i] & 0xffffffffu);
  }
  free(recs);
  return ORC_OK;
}

int orc_construct(const float* x, int ndim, const uint64_t* dims, float eb_f, float ebx2_f,
                  float ebx2_r, uint32_t radius, uint16_t* codes, uint32_t* rec_key,
                  uint32_t* rec_val, uint64_t rec_cap, uint64_t* n_rec, uint32_t* hist) {
  geom_t g;
  int st = make_geom(ndim, dims, &g);
  if (st) return st;
  if (radius < 1 || radius > 512) return ORC_E_ARG;
  uint64_t n = g.nelem;
  int32_t* K = (int32_t*)malloc(n * sizeof(int32_t));
  uint8_t* P = (uint8_t*)malloc(n);
  if (!K || !P) {
    free(K);
    free(P);
    return ORC_E_CAPACITY;
  }
  for (uint64_t e = 0; e < n && !st; e++) {
    int patch = 0;
    st = orc_prequant(x[e], eb_f, ebx2_f, ebx2_r, &K[e], &patch);
    P[e] = (uint8_t)patch;
  }
  if (!st)
    st = construct_k(K, P, x, &g, radius, codes, rec_key, rec_val, rec_cap, n_rec, hist);
  free(K);
  free(P);
  return st;
}

/* Lorenzo construction of a double-precision field (prequantization above, then the
   FP32 path's residuals; no patches). */
int orc_construct_f64(const double* x, int ndim, const uint64_t* dims, double eb_d, double step,
                      double rstep, uint32_t radius, uint16_t* codes, uint32_t* rec_key,
                      uint32_t* rec_val, uint64_t rec_cap, uint64_t* n_rec, uint32_t* hist) {
  geom_t g;
  int st = make_geom(ndim, dims, &g);
  if (st) return st;
  if (radius < 1 || radius > 512) return ORC_E_ARG;
  int32_t* K = (int32_t*)malloc(g.nelem * sizeof(int32_t));
  if (!K) return ORC_E_CAPACITY;
  for (uint64_t e = 0; e < g.nelem && !st; e++) st = orc_prequant_f64(x[e], eb_d, step, rstep, &K[e]);
  if (!st) st = construct_k(K, NULL, NULL, &g, radius, codes, rec_key, rec_val, rec_cap, n_rec, hist);
  free(K);
  return st;
}

/* ------------------------------------------------------------------------------- */
/* run-length encoding (Sec. III-B): maximal runs of equal codes within one block,  */
/* e.g. "aabcccccaa" -> (a,2)(b,1)(c,5)(a,2)                                        */
/* ------------------------------------------------------------------------------- */

typedef struct {
  uint16_t v;
  uint16_t len;
} run_t;

static uint64_t make_runs(const uint16_t* c, uint64_t m, run_t* out) {
  uint64_t nr = 0, i = 0;
  while (i < m) {
    uint64_t l = 1;
    while (i + l < m && c[i + l] == c[i]) l++;
    out[nr].v = c[i];
    out[nr].len = (uint16_t)l;
    nr++;
    i += l;
  }
  return nr;
}

/*
 * Run eligibility (a reading): a block whose runs average fewer than 4 codes
 * (4 * runs > m) gains nothing from Huffman-coding its runs, so in the adaptive modes
 * it never uses RLE+Huffman and its runs stay out of the run books (plain RLE needs
 * no book and stays available to the exhaustive choice).  Forced RLE and RLE+Huffman
 * make every block eligible.
 */
static int run_eligible(uint64_t nr, uint64_t m, int all_blocks) { return all_blocks || 4 * nr <= m; }

int orc_run_stats(const uint16_t* codes, int ndim, const uint64_t* dims, int all_blocks,
                  uint32_t* val_hist, uint32_t* len_hist, uint32_t* nruns) {
  geom_t g;
  int st = make_geom(ndim, dims, &g);
  if (st) return st;
  run_t* runs = (run_t*)malloc(SLOTS * sizeof(run_t));
  memset(val_hist, 0, NSYM_CODE * sizeof(uint32_t));
  memset(len_hist, 0, NSYM_LEN * sizeof(uint32_t));
  for (uint64_t b = 0; b < g.nblk; b++) {
    uint64_t m = block_count(&g, b);
    uint64_t nr = make_runs(codes + b * SLOTS, m, runs);
    if (run_eligible(nr, m, all_blocks))
      for (uint64_t i = 0; i < nr; i++) {
        val_hist[runs[i].v]++;
        len_hist[runs[i].len - 1]++;
      }
    nruns[b] = (uint32_t)nr;
  }
  free(runs);
  return ORC_OK;
}

/* ------------------------------------------------------------------------------- */
/* canonical Huffman (Sec. II-A Step-6; the paper defers the construction to cuSZ) */
/* ------------------------------------------------------------------------------- */

typedef struct {
  uint32_t f, s;
} leaf_t;

static int cmp_leaf(const void* a, const void* b) {
  const leaf_t* x = (const leaf_t*)a;
  const leaf_t* y = (const leaf_t*)b;
  if (x->f != y->f) return x->f < y->f ? -1 : 1;
  return x->s < y->s ? -1 : (x->s > y->s ? 1 : 0);
}

/*
 * Optimal code lengths by the two-queue Huffman construction.  Deterministic
 * reading: leaves sorted by (frequency, symbol) ascending; each step merges the two
 * lightest nodes, taking from the leaf queue on a weight tie; a single present
 * symbol gets length 1.  Lengths are the leaf depths, no length limit.
 */
int orc_huffman_lengths(const uint32_t* freq, int nsym, uint8_t* len) {
  memset(len, 0, (size_t)nsym);
  leaf_t* lv = (leaf_t*)malloc((size_t)nsym * sizeof(leaf_t));
  int L = 0;
  for (int s = 0; s < nsym; s++)
    if (freq[s]) {
      lv[L].f = freq[s];
      lv[L].s = (uint32_t)s;
      L++;
    }
  if (L == 0) {
    free(lv);
    return ORC_OK;
  }
  if (L == 1) {
    len[lv[0].s] = 1;
    free(lv);
    return ORC_OK;
  }
  qsort(lv, (size_t)L, sizeof(leaf_t), cmp_leaf);
  int nn = 2 * L - 1;
  uint64_t* w = (uint64_t*)malloc((size_t)nn * sizeof(uint64_t));
  int* parent = (int*)malloc((size_t)nn * sizeof(int));
  int* depth = (int*)malloc((size_t)nn * sizeof(int));
  for (int i = 0; i < L; i++) w[i] = lv[i].f;
  int qi = 0, qj = L, next = L;
  while (next < nn) {
    int pick[2];
    for (int t = 0; t < 2; t++) {
      if (qi < L && (qj >= next || w[qi] <= w[qj]))
        pick[t] = qi++;
      else
        pick[t] = qj++;
    }
    w[next] = w[pick[0]] + w[pick[1]];
    parent[pick[0]] = next;
    parent[pick[1]] = next;
    next++;
  }
  depth[nn - 1] = 0;
  for (int v = nn - 2; v >= 0; v--) depth[v] = depth[parent[v]] + 1;
  int st = ORC_OK;
  for (int i = 0; i < L; i++) {
    if (depth[i] > MAXLEN) st = ORC_E_RANGE;
    len[lv[i].s] = (uint8_t)depth[i];
  }
  free(lv);
  free(w);
  free(parent);
  free(depth);
  return st;
}

/* canonical codes: ordered by (length, symbol); each length starts at
   (first code of the previous length + its count) << 1 */
int orc_canonical_codes(const uint8_t* len, int nsym, uint64_t* code) {
  uint64_t cnt[MAXLEN + 1] = {0}, next[MAXLEN + 1] = {0};
  for (int s = 0; s < nsym; s++)
    if (len[s]) {
      if (len[s] > MAXLEN) return ORC_E_CORRUPT;
      cnt[len[s]]++;
    }
  uint64_t c = 0;
  for (int l = 1; l <= MAXLEN; l++) {
    c = (c + cnt[l - 1]) << 1;
    next[l] = c;
  }
  for (int s = 0; s < nsym; s++) code[s] = len[s] ? next[len[s]]++ : 0;
  return ORC_OK;
}

/* Kraft sum <= 1 (prefix code exists for these lengths) */
static int kraft_ok(const uint8_t* len, int nsym) {
  int64_t cnt[MAXLEN + 1] = {0};
  for (int s = 0; s < nsym; s++) {
    if (len[s] > MAXLEN) return 0;
    if (len[s]) cnt[len[s]]++;
  }
  int64_t avail = 1;
  for (int l = 1; l <= MAXLEN; l++) {
    avail = avail * 2 - cnt[l];
    if (avail < 0) return 0;
    if (avail > (1ll << 40)) avail = 1ll << 40;
  }
  return 1;
}

typedef struct {
  uint64_t first[MAXLEN + 1];
  uint64_t count[MAXLEN + 1];
  uint64_t offset[MAXLEN + 1];
  uint16_t sorted[NSYM_LEN];
} dectab_t;

static void build_dectab(const uint8_t* len, int nsym, dectab_t* t) {
  uint64_t code[NSYM_LEN];
  orc_canonical_codes(len, nsym, code);
  memset(t, 0, sizeof(*t));
  for (int s = 0; s < nsym; s++)
    if (len[s]) t->count[len[s]]++;
  uint64_t off = 0;
  for (int l = 1; l <= MAXLEN; l++) {
    t->offset[l] = off;
    off += t->count[l];
  }
  uint64_t fill[MAXLEN + 1];
  memcpy(fill, t->offset, sizeof(fill));
  for (int s = 0; s < nsym; s++)
    if (len[s]) {
      if (fill[len[s]] == t->offset[len[s]]) t->first[len[s]] = code[s];
      t->sorted[fill[len[s]]++] = (uint16_t)s;
    }
}

static uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
static uint64_t align4(uint64_t a) { return (a + 3) & ~3ull; }
static uint64_t align8(uint64_t a) { return (a + 7) & ~7ull; }

/* ------------------------------------------------------------------------------- */
/* Interleaved Huffman stream (the concatenated codes of Sec. II-A Step-7/8, laid   */
/* out for a 32-lane decoder).  Symbol i of a sequence belongs to lane i % 32.  A   */
/* lane's bit string is its symbols' codes, MSB first, zero-padded to a multiple of */
/* 16 and cut into 16-bit units (first bit = MSB of the unit).  Units are stored in */
/* the order a 32-lane decoder reads them: at step t the lanes holding symbols      */
/* 32t..32t+31 top up in rounds -- in each round every lane whose next code is      */
/* longer than the bits it holds takes one unit, lanes in increasing order -- and   */
/* then all of them consume their code.                                             */
/* ------------------------------------------------------------------------------- */
#define LANES 32
#define UNIT 16

typedef struct {
  uint16_t* u;
  uint64_t bits;
} lane_t;

static void lane_put(lane_t* L, uint64_t code, int len) {
  for (int i = len - 1; i >= 0; i--) {
    if ((code >> i) & 1u) L->u[L->bits >> 4] |= (uint16_t)(1u << (15 - (L->bits & 15)));
    L->bits++;
  }
}

/* number of units of the stream; writes them to out unless out is NULL */
static uint64_t ihs_encode(const uint16_t* sym, uint64_t N, int add, const uint8_t* len,
                           const uint64_t* code, uint16_t* out, int* missing) {
  lane_t L[LANES];
  const uint64_t per = ceil_div(N, LANES);
  for (int l = 0; l < LANES; l++) {
    L[l].u = (uint16_t*)calloc(ceil_div(per * MAXLEN, UNIT) + 1, sizeof(uint16_t));
    L[l].bits = 0;
  }
  for (uint64_t i = 0; i < N; i++) {
    const int s = sym[i] + add;
    if (!len[s]) *missing = 1;
    lane_put(&L[i % LANES], code[s], len[s]);
  }
  int nb[LANES] = {0};
  uint64_t next[LANES] = {0}, pos = 0;
  for (uint64_t t = 0; t * LANES < N; t++) {
    for (;;) {
      int any = 0;
      for (uint64_t l = 0; l < LANES && t * LANES + l < N; l++) {
        if (len[sym[t * LANES + l] + add] > nb[l]) {
          if (out) out[pos] = L[l].u[next[l]];
          next[l]++;
          pos++;
          nb[l] += UNIT;
          any = 1;
        }
      }
      if (!any) break;
    }
    for (uint64_t l = 0; l < LANES && t * LANES + l < N; l++) nb[l] -= len[sym[t * LANES + l] + add];
  }
  for (int l = 0; l < LANES; l++) free(L[l].u);
  return pos;
}

/* length of the codeword that is a prefix of the nb valid top bits of buf, 0 if none */
static int match_len(const dectab_t* t, uint64_t buf, int nb) {
  for (int l = 1; l <= nb && l <= MAXLEN; l++) {
    uint64_t c = buf >> (64 - l);
    if (t->count[l] && c >= t->first[l] && c - t->first[l] < t->count[l]) return l;
  }
  return 0;
}

/* decode N symbols from the units in[0..avail); returns the units read, -1 if the
   stream is damaged (a lane needs bits it cannot hold, or the units run out) */
static int64_t ihs_decode(const uint16_t* in, uint64_t avail, uint64_t N, const dectab_t* t,
                          uint16_t* out) {
  uint64_t buf[LANES] = {0}, pos = 0;
  int nb[LANES] = {0};
  for (uint64_t s = 0; s * LANES < N; s++) {
    for (;;) {
      int any = 0;
      for (uint64_t l = 0; l < LANES && s * LANES + l < N; l++) {
        if (match_len(t, buf[l], nb[l]) == 0) {
          if (nb[l] > 64 - UNIT || pos >= avail) return -1;
          buf[l] |= (uint64_t)in[pos++] << (64 - UNIT - nb[l]);
          nb[l] += UNIT;
          any = 1;
        }
      }
      if (!any) break;
    }
    for (uint64_t l = 0; l < LANES && s * LANES + l < N; l++) {
      const int ml = match_len(t, buf[l], nb[l]);
      const uint64_t c = buf[l] >> (64 - ml);
      out[s * LANES + l] = t->sorted[t->offset[ml] + (c - t->first[ml])];
      buf[l] = ml == 64 ? 0 : buf[l] << ml;
      nb[l] -= ml;
    }
  }
  return (int64_t)pos;
}

/* ------------------------------------------------------------------------------- */
/* per-block payloads                                                               */
/*   HUFF      : u16 unit count of stream A, then two interleaved streams: A holds  */
/*               the block's first h codes, B the rest (h = the multiple of 32 at or */
/*               above m/2, at most m), padded to 4 B                                */
/*   RLE       : u16 value[nr], u16 length[nr]                                       */
/*   RLE_HUFF  : u32 nr, u32 value units, value stream, length stream (length-1      */
/*               coded), padded to 4 B                                               */
/* ------------------------------------------------------------------------------- */

/* codes in stream A of a Huffman block of m codes */
static uint64_t huff_split(uint64_t m) {
  const uint64_t h = 32 * ceil_div(m, 64);
  return h < m ? h : m;
}

static uint64_t huff_size(const uint16_t* c, uint64_t m, const uint8_t* len, const uint64_t* code,
                          int* missing) {
  const uint64_t h = huff_split(m);
  const uint64_t na = ihs_encode(c, h, 0, len, code, NULL, missing);
  const uint64_t nb = ihs_encode(c + h, m - h, 0, len, code, NULL, missing);
  return align4(2 * (1 + na + nb));
}

static void run_streams(const run_t* runs, uint64_t nr, uint16_t* v, uint16_t* l) {
  for (uint64_t i = 0; i < nr; i++) {
    v[i] = runs[i].v;
    l[i] = runs[i].len;
  }
}

static uint64_t rlehuff_size(const run_t* runs, uint64_t nr, const uint8_t* vlen, const uint64_t* vcode,
                             const uint8_t* llen, const uint64_t* lcode, int* missing) {
  uint16_t* v = (uint16_t*)malloc((nr + 1) * 2);
  uint16_t* l = (uint16_t*)malloc((nr + 1) * 2);
  run_streams(runs, nr, v, l);
  uint64_t vu = ihs_encode(v, nr, 0, vlen, vcode, NULL, missing);
  uint64_t lu = ihs_encode(l, nr, -1, llen, lcode, NULL, missing);
  free(v);
  free(l);
  return align4(8 + 2 * (vu + lu));
}

static void huff_write(const uint16_t* c, uint64_t m, const uint8_t* len, const uint64_t* code,
                       uint8_t* out) {
  int missing = 0;
  const uint64_t h = huff_split(m);
  const uint64_t na = ihs_encode(c, h, 0, len, code, NULL, &missing);
  const uint64_t nb = ihs_encode(c + h, m - h, 0, len, code, NULL, &missing);
  uint16_t* u = (uint16_t*)calloc(1 + na + nb + 2, sizeof(uint16_t));
  u[0] = (uint16_t)na;
  ihs_encode(c, h, 0, len, code, u + 1, &missing);
  ihs_encode(c + h, m - h, 0, len, code, u + 1 + na, &missing);
  memset(out, 0, align4(2 * (1 + na + nb)));
  memcpy(out, u, 2 * (1 + na + nb));
  free(u);
}

static void rle_write(const run_t* runs, uint64_t nr, uint8_t* out) {
  for (uint64_t i = 0; i < nr; i++) {
    memcpy(out + 2 * i, &runs[i].v, 2);
    memcpy(out + 2 * nr + 2 * i, &runs[i].len, 2);
  }
}

static void rlehuff_write(const run_t* runs, uint64_t nr, const uint8_t* vlen,
                          const uint64_t* vcode, const uint8_t* llen, const uint64_t* lcode,
                          uint8_t* out) {
  int missing = 0;
  uint16_t* v = (uint16_t*)malloc((nr + 1) * 2);
  uint16_t* l = (uint16_t*)malloc((nr + 1) * 2);
  run_streams(runs, nr, v, l);
  uint64_t vu = ihs_encode(v, nr, 0, vlen, vcode, NULL, &missing);
  uint64_t lu = ihs_encode(l, nr, -1, llen, lcode, NULL, &missing);
  uint16_t* u = (uint16_t*)calloc(vu + lu + 2, sizeof(uint16_t));
  ihs_encode(v, nr, 0, vlen, vcode, u, &missing);
  ihs_encode(l, nr, -1, llen, lcode, u + vu, &missing);
  uint32_t h[2] = {(uint32_t)nr, (uint32_t)vu};
  memset(out, 0, align4(8 + 2 * (vu + lu)));
  memcpy(out, h, 8);
  memcpy(out + 8, u, 2 * (vu + lu));
  free(u);
  free(v);
  free(l);
}

int orc_block_sizes(const uint16_t* codes, int ndim, const uint64_t* dims, uint32_t radius,
                    const uint8_t* code_len, const uint8_t* val_len, const uint8_t* len_len,
                    uint32_t lanes, int all_blocks, uint64_t* sizes) {
  geom_t g;
  int st = make_geom(ndim, dims, &g);
  if (st) return st;
  (void)radius;
  if (lanes != LANES) return ORC_E_ARG;
  uint64_t ccode[NSYM_CODE], vcode[NSYM_CODE], lcode[NSYM_LEN];
  orc_canonical_codes(code_len, NSYM_CODE, ccode);
  orc_canonical_codes(val_len, NSYM_CODE, vcode);
  orc_canonical_codes(len_len, NSYM_LEN, lcode);
  run_t* runs = (run_t*)malloc(SLOTS * sizeof(run_t));
  int missing = 0;
  for (uint64_t b = 0; b < g.nblk; b++) {
    uint64_t m = block_count(&g, b);
    const uint16_t* c = codes + b * SLOTS;
    uint64_t nr = make_runs(c, m, runs);
    int miss_h = 0, miss_r = 0;
    sizes[3 * b + ORC_CODEC_HUFF] = huff_size(c, m, code_len, ccode, &miss_h);
    sizes[3 * b + ORC_CODEC_RLE] = 4 * nr;
    if (run_eligible(nr, m, all_blocks))
      sizes[3 * b + ORC_CODEC_RLE_HUFF] = rlehuff_size(runs, nr, val_len, vcode, len_len, lcode, &miss_r);
    else
      sizes[3 * b + ORC_CODEC_RLE_HUFF] = UINT64_MAX;
    missing |= miss_h | miss_r;
  }
  free(runs);
  return missing ? ORC_E_ARG : ORC_OK;
}

/* ------------------------------------------------------------------------------- */
/* selection (Sec. III-B1)                                                          */
/* ------------------------------------------------------------------------------- */

/*
 * Binary logarithm in Q16 fixed point by the bit-by-bit squaring method: write
 * v = 2^e * m with m in [1,2) (Q31), then 16 times square m and emit one fraction
 * bit (1 and halve m when m >= 2).  Integer-only, so the pick it feeds is the same
 * on every machine.
 */
uint32_t orc_log2_q16(uint64_t v) {
  if (v == 0) return 0;
  uint32_t e = 0;
  while ((v >> (e + 1)) != 0) e++;
  uint64_t m = e >= 31 ? (v >> (e - 31)) : (v << (31 - e));
  uint32_t frac = 0;
  for (int i = 0; i < 16; i++) {
    m = (m * m) >> 31;
    frac <<= 1;
    if (m >= (2ull << 31)) {
      m >>= 1;
      frac |= 1;
    }
  }
  return e * 65536u + frac;
}

/*
 * Histogram estimate (Sec. III-B1): H = -sum p log2 p; with p1 the top probability,
 * the Huffman redundancy lower bound R- = 1 - H(p1, 1-p1) when p1 > 0.4 (else 0);
 * <b> is estimated by H + R-, and RLE (here RLE followed by VLE) is chosen when
 * Huffman would likely average no more than 1.09 bits (Sec. III-B2, "1.09").
 * Reading: "likely" uses the lower bound.  All terms are scaled by m*2^16 and
 * compared in integers.
 */
int orc_heuristic_pick(const uint32_t* h, int nsym, uint32_t m) {
  if (m == 0) return ORC_CODEC_HUFF;
  int64_t Lm = orc_log2_q16(m);
  int64_t S = 0;
  uint32_t f1 = 0;
  for (int s = 0; s < nsym; s++)
    if (h[s]) {
      S += (int64_t)h[s] * orc_log2_q16(h[s]);
      if (h[s] > f1) f1 = h[s];
    }
  int64_t NH = (int64_t)m * Lm - S;
  int64_t Rm = 0;
  if (10ll * f1 > 4ll * m) {
    int64_t rest = (int64_t)m - f1;
    Rm = (int64_t)m * 65536 + (int64_t)f1 * orc_log2_q16(f1) +
         (rest > 0 ? rest * (int64_t)orc_log2_q16((uint64_t)rest) : 0) - (int64_t)m * Lm;
    if (Rm < 0) Rm = 0;
  }
  int64_t est = NH + Rm;
  return (100 * est <= 109ll * (int64_t)m * 65536) ? ORC_CODEC_RLE_HUFF : ORC_CODEC_HUFF;
}

/*
 * Selector features of one block (dense codes c[0..m), radius r).  q == 0 marks an
 * outlier; every other code carries delta = q - r.  Each feature is a ratio of two
 * integers, both exact in FP32, formed with one IEEE division:
 *  0 zero-residual fraction        #(q == r) / m
 *  1 code entropy H (bits)         (m log2 m - sum_s h_s log2 h_s) / m, Q16 logarithms
 *  2 top-code probability p1       max_s h_s / m, outliers' code 0 included
 *  3 log2(1 + max |delta|)         over in-range codes (0 if there are none), the Q16
 *                                  logarithm divided by 65536
 *  4 runs per element              #runs / m
 *  5 outlier fraction              #(q == 0) / m
 *  6 mean |delta| / r              sum of |q - r| over in-range codes / (m r): the
 *                                  denominator counts all m codes, so an outlier adds 0
 *                                  (its delta lives in a record, not in the code)
 *  7 RLE roughness                 the madogram with binary variance (Sec. III-B,
 *                                  "Modeling RLE Compressibility") on a systematic
 *                                  sample of pairs: position i is paired with
 *                                  i + d(i), d(i) = 1 + 25 (i mod 8), so the distances
 *                                  1, 26, ..., 176 (every 25th of the paper's uniform
 *                                  d in [1, 200]) each take every 8th position; the
 *                                  feature is the fraction of the pairs inside the
 *                                  block whose codes differ (0 if there are none)
 */
static const uint32_t MADO_D0 = 1, MADO_STEP = 25, MADO_N = 8;

static void features_of(const uint16_t* c, uint64_t m, uint32_t radius, float* f) {
  uint32_t* h = (uint32_t*)calloc(NSYM_CODE, sizeof(uint32_t));
  uint64_t zero = 0, outl = 0, absd = 0, maxd = 0, runs = 0, mism = 0, pairs = 0;
  for (uint64_t i = 0; i < m; i++) {
    h[c[i]]++;
    if (c[i] == 0) {
      outl++;
    } else {
      int64_t d = (int64_t)c[i] - radius;
      if (d < 0) d = -d;
      if (d == 0) zero++;
      if ((uint64_t)d > maxd) maxd = (uint64_t)d;
      absd += (uint64_t)d;
    }
    if (i == 0 || c[i] != c[i - 1]) runs++;
  }
  for (uint64_t i = 0; i < m; i++) {
    const uint64_t d = MADO_D0 + MADO_STEP * (i % MADO_N);
    if (i + d < m) {
      pairs++;
      if (c[i] != c[i + d]) mism++;
    }
  }
  int64_t Lm = orc_log2_q16(m), S = 0;
  uint32_t f1 = 0;
  for (int s = 0; s < NSYM_CODE; s++)
    if (h[s]) {
      S += (int64_t)h[s] * orc_log2_q16(h[s]);
      if (h[s] > f1) f1 = h[s];
    }
  int64_t NH = (int64_t)m * Lm - S;
  float fm = (float)m;
  f[0] = (float)zero / fm;
  f[1] = (float)NH / (float)(m * 65536);
  f[2] = (float)f1 / fm;
  f[3] = (float)orc_log2_q16(1 + maxd) / 65536.0f;
  f[4] = (float)runs / fm;
  f[5] = (float)outl / fm;
  f[6] = (float)absd / (float)(m * radius);
  f[7] = pairs ? (float)mism / (float)pairs : 0.0f;
  free(h);
}

int orc_block_features(const uint16_t* codes, int ndim, const uint64_t* dims, uint32_t radius,
                       float* feat) {
  geom_t g;
  int st = make_geom(ndim, dims, &g);
  if (st) return st;
  for (uint64_t b = 0; b < g.nblk; b++)
    features_of(codes + b * SLOTS, block_count(&g, b), radius, feat + 8 * b);
  return ORC_OK;
}

/* MLP 8 -> 32 -> 32 -> 3 (ReLU), parameters W1[32][8] b1 W2[32][32] b2 W3[3][32] b3;
   every dot product is a chain of fmaf starting from the bias, inputs in order */
void orc_mlp_forward(const float* w, const float* feat, uint64_t nrows, float* out) {
  const float* W1 = w;
  const float* b1 = W1 + ORC_MLP_H * ORC_MLP_IN;
  const float* W2 = b1 + ORC_MLP_H;
  const float* b2 = W2 + ORC_MLP_H * ORC_MLP_H;
  const float* W3 = b2 + ORC_MLP_H;
  const float* b3 = W3 + ORC_MLP_OUT * ORC_MLP_H;
  for (uint64_t r = 0; r < nrows; r++) {
    const float* x = feat + ORC_MLP_IN * r;
    float h1[ORC_MLP_H], h2[ORC_MLP_H];
    for (int i = 0; i < ORC_MLP_H; i++) {
      float a = b1[i];
      for (int j = 0; j < ORC_MLP_IN; j++) a = fmaf(W1[i * ORC_MLP_IN + j], x[j], a);
      h1[i] = a > 0.0f ? a : 0.0f;
    }
    for (int i = 0; i < ORC_MLP_H; i++) {
      float a = b2[i];
      for (int j = 0; j < ORC_MLP_H; j++) a = fmaf(W2[i * ORC_MLP_H + j], h1[j], a);
      h2[i] = a > 0.0f ? a : 0.0f;
    }
    for (int c = 0; c < ORC_MLP_OUT; c++) {
      float a = b3[c];
      for (int j = 0; j < ORC_MLP_H; j++) a = fmaf(W3[c * ORC_MLP_H + j], h2[j], a);
      out[ORC_MLP_OUT * r + c] = a;
    }
  }
}

/* loss = mean over rows and outputs of (y - t)^2, with its gradient, in double */
double orc_mlp_loss_grad_f64(const float* w, const float* feat, const float* target,
                             uint64_t nrows, double* grad) {
  const int nW1 = ORC_MLP_H * ORC_MLP_IN, nW2 = ORC_MLP_H * ORC_MLP_H;
  const float* W1 = w;
  const float* b1 = W1 + nW1;
  const float* W2 = b1 + ORC_MLP_H;
  const float* b2 = W2 + nW2;
  const float* W3 = b2 + ORC_MLP_H;
  const float* b3 = W3 + ORC_MLP_OUT * ORC_MLP_H;
  double* gW1 = grad;
  double* gb1 = gW1 + nW1;
  double* gW2 = gb1 + ORC_MLP_H;
  double* gb2 = gW2 + nW2;
  double* gW3 = gb2 + ORC_MLP_H;
  double* gb3 = gW3 + ORC_MLP_OUT * ORC_MLP_H;
  memset(grad, 0, ORC_MLP_PARAMS * sizeof(double));
  double loss = 0.0, scale = 1.0 / ((double)nrows * ORC_MLP_OUT);
  for (uint64_t r = 0; r < nrows; r++) {
    const float* x = feat + ORC_MLP_IN * r;
    double a1[ORC_MLP_H], h1[ORC_MLP_H], a2[ORC_MLP_H], h2[ORC_MLP_H], y[ORC_MLP_OUT];
    for (int i = 0; i < ORC_MLP_H; i++) {
      double a = b1[i];
      for (int j = 0; j < ORC_MLP_IN; j++) a += (double)W1[i * ORC_MLP_IN + j] * x[j];
      a1[i] = a;
      h1[i] = a > 0 ? a : 0;
    }
    for (int i = 0; i < ORC_MLP_H; i++) {
      double a = b2[i];
      for (int j = 0; j < ORC_MLP_H; j++) a += (double)W2[i * ORC_MLP_H + j] * h1[j];
      a2[i] = a;
      h2[i] = a > 0 ? a : 0;
    }
    double dy[ORC_MLP_OUT], dh2[ORC_MLP_H] = {0}, dh1[ORC_MLP_H] = {0};
    for (int c = 0; c < ORC_MLP_OUT; c++) {
      double a = b3[c];
      for (int j = 0; j < ORC_MLP_H; j++) a += (double)W3[c * ORC_MLP_H + j] * h2[j];
      y[c] = a;
      double e = y[c] - (double)target[ORC_MLP_OUT * r + c];
      loss += e * e * scale;
      dy[c] = 2.0 * e * scale;
    }
    for (int c = 0; c < ORC_MLP_OUT; c++) {
      gb3[c] += dy[c];
      for (int j = 0; j < ORC_MLP_H; j++) {
        gW3[c * ORC_MLP_H + j] += dy[c] * h2[j];
        dh2[j] += dy[c] * W3[c * ORC_MLP_H + j];
      }
    }
    for (int i = 0; i < ORC_MLP_H; i++) {
      double d = a2[i] > 0 ? dh2[i] : 0.0;
      gb2[i] += d;
      for (int j = 0; j < ORC_MLP_H; j++) {
        gW2[i * ORC_MLP_H + j] += d * h1[j];
        dh1[j] += d * W2[i * ORC_MLP_H + j];
      }
    }
    for (int i = 0; i < ORC_MLP_H; i++) {
      double d = a1[i] > 0 ? dh1[i] : 0.0;
      gb1[i] += d;
      for (int j = 0; j < ORC_MLP_IN; j++) gW1[i * ORC_MLP_IN + j] += d * x[j];
    }
  }
  return loss;
}

/* ------------------------------------------------------------------------------- */
/* archive                                                                          */
/* ------------------------------------------------------------------------------- */

typedef struct {
  uint32_t magic;
  uint16_t version;
  uint8_t ndim, eb_mode;
  uint64_t dims[3];
  double eb_user, eb_d;
  float eb_f;
  uint32_t radius, lanes, flags;
  uint64_t nblk, n_rec, n_out, n_patch, payload, total;
  uint32_t select, n_codec[3];
} hdr_t;

static void put32(uint8_t* p, uint32_t v) { memcpy(p, &v, 4); }
static void put64(uint8_t* p, uint64_t v) { memcpy(p, &v, 8); }
static uint32_t get32(const uint8_t* p) {
  uint32_t v;
  memcpy(&v, p, 4);
  return v;
}
static uint64_t get64(const uint8_t* p) {
  uint64_t v;
  memcpy(&v, p, 8);
  return v;
}

static void write_header(uint8_t* o, const hdr_t* h) {
  memset(o, 0, HDR);
  put32(o + 0, h->magic);
  memcpy(o + 4, &h->version, 2);
  o[6] = h->ndim;
  o[7] = h->eb_mode;
  for (int i = 0; i < 3; i++) put64(o + 8 + 8 * i, h->dims[i]);
  memcpy(o + 32, &h->eb_user, 8);
  memcpy(o + 40, &h->eb_d, 8);
  memcpy(o + 48, &h->eb_f, 4);
  put32(o + 52, h->radius);
  put32(o + 56, h->lanes);
  put32(o + 60, h->flags);
  put64(o + 64, h->nblk);
  put64(o + 72, h->n_rec);
  put64(o + 80, h->n_out);
  put64(o + 88, h->n_patch);
  put64(o + 96, h->payload);
  put64(o + 104, h->total);
  put32(o + 112, h->select);
  for (int i = 0; i < 3; i++) put32(o + 116 + 4 * i, h->n_codec[i]);
}

static void read_header(const uint8_t* o, hdr_t* h) {
  h->magic = get32(o);
  memcpy(&h->version, o + 4, 2);
  h->ndim = o[6];
  h->eb_mode = o[7];
  for (int i = 0; i < 3; i++) h->dims[i] = get64(o + 8 + 8 * i);
  memcpy(&h->eb_user, o + 32, 8);
  memcpy(&h->eb_d, o + 40, 8);
  memcpy(&h->eb_f, o + 48, 4);
  h->radius = get32(o + 52);
  h->lanes = get32(o + 56);
  h->flags = get32(o + 60);
  h->nblk = get64(o + 64);
  h->n_rec = get64(o + 72);
  h->n_out = get64(o + 80);
  h->n_patch = get64(o + 88);
  h->payload = get64(o + 96);
  h->total = get64(o + 104);
  h->select = get32(o + 112);
  for (int i = 0; i < 3; i++) h->n_codec[i] = get32(o + 116 + 4 * i);
}

size_t orc_max_archive_bytes(int ndim, const uint64_t* dims) {
  geom_t g;
  if (make_geom(ndim, dims, &g)) return 0;
  uint64_t slots = g.nblk * SLOTS;
  /* records: an outlier and a patch per element at most; payload: 64-bit codes */
  uint64_t payload = 16 * slots + 64 * g.nblk;
  return (size_t)(HDR + align8(g.nblk) + align8(4 * g.nblk) + 16 * g.nelem + payload + 6144);
}

/* smallest exact size; ties prefer HUFF, then RLE_HUFF, then RLE */
static int exhaustive_pick(const uint64_t* s) {
  int c = ORC_CODEC_HUFF;
  if (s[ORC_CODEC_RLE_HUFF] < s[c]) c = ORC_CODEC_RLE_HUFF;
  if (s[ORC_CODEC_RLE] < s[c]) c = ORC_CODEC_RLE;
  return c;
}

/*
 * Learned selection: the codec with the smallest predicted size (first index on
 * ties); when the runner-up is predicted within ORC_MLP_MARGIN of it the network is
 * not trusted and the exact sizes decide, as in exhaustive selection (the exhaustive
 * choice is the selector's fallback).  All comparisons are plain FP32 compares, so a
 * NaN prediction never triggers the fallback and never wins.
 */
int orc_learned_pick(const float* y, const uint64_t* s) {
  int c = 0;
  for (int k = 1; k < 3; k++)
    if (y[k] < y[c]) c = k;
  int r = -1;
  for (int k = 0; k < 3; k++)
    if (k != c && (r < 0 || y[k] < y[r])) r = k;
  const float gap = y[r] - y[c];
  if (gap < ORC_MLP_MARGIN) c = exhaustive_pick(s);
  return c;
}

int orc_selector_targets(const uint64_t* sizes, int ndim, const uint64_t* dims, float* target,
                         uint8_t* valid) {
  geom_t g;
  int st = make_geom(ndim, dims, &g);
  if (st) return st;
  for (uint64_t b = 0; b < g.nblk; b++) {
    const uint64_t m = block_count(&g, b);
    const int64_t lm = orc_log2_q16(m);
    valid[b] = sizes[3 * b + ORC_CODEC_RLE_HUFF] != UINT64_MAX;
    for (int c = 0; c < 3; c++) {
      const uint64_t sz = sizes[3 * b + c];
      target[3 * b + c] =
          sz == UINT64_MAX ? 0.0f : (float)((int64_t)orc_log2_q16(8 * sz) - lm) * (1.0f / 65536.0f);
    }
  }
  return ORC_OK;
}

/* Compression of an FP32 field (x32) or, with the archive flag ORC_FLAG_F64, of a
   double-precision one (x64). */
static int compress_impl(const float* x32, const double* x64, int ndim, const uint64_t* dims, int eb_mode,
                         double eb, uint32_t radius, int select, const float* mlp_w, int global, uint8_t* out,
                         size_t cap, size_t* out_bytes) {
  geom_t g;
  int st = make_geom(ndim, dims, &g);
  if (st) return st;
  if (global) make_global(&g);
  if (radius < 1 || radius > 512) return ORC_E_ARG;
  if (select < ORC_SEL_HUFF || select > ORC_SEL_LEARNED) return ORC_E_ARG;
  if (select == ORC_SEL_LEARNED && !mlp_w) return ORC_E_ARG;
  if (!(eb > 0.0) || !isfinite(eb) || (eb_mode != ORC_EB_ABS && eb_mode != ORC_EB_REL)) return ORC_E_ARG;
  /* a non-finite value is reported before any range error, in either mode */
  double eb_d, step = 0.0, rstep = 0.0;
  float eb_f = 0.0f, ebx2_f = 0.0f, ebx2_r = 0.0f;
  if (x64) {
    double vmin = 0.0, vmax = 0.0;
    st = orc_value_range_f64(x64, g.nelem, &vmin, &vmax);
    if (st) return st;
    st = orc_eb_params_f64(eb_mode, eb, vmin, vmax, &eb_d, &step, &rstep);
    if (st) return st;
    /* informational FP32 copy of the bound: the largest float not above eb_d */
    eb_f = (float)eb_d;
    if ((double)eb_f > eb_d) eb_f = nextafterf(eb_f, 0.0f);
  } else {
    float vmin = 0.0f, vmax = 0.0f;
    st = orc_value_range(x32, g.nelem, &vmin, &vmax);
    if (st) return st;
    st = orc_eb_params(eb_mode, eb, vmin, vmax, &eb_d, &eb_f, &ebx2_f, &ebx2_r);
    if (st) return st;
  }

  uint64_t slots = g.nblk * SLOTS;
  uint16_t* codes = (uint16_t*)malloc(slots * sizeof(uint16_t));
  uint32_t* rk = (uint32_t*)malloc((2 * g.nelem + 1) * 4);
  uint32_t* rv = (uint32_t*)malloc((2 * g.nelem + 1) * 4);
  uint32_t hist[NSYM_CODE], vh[NSYM_CODE], lh[NSYM_LEN];
  uint32_t* nruns = (uint32_t*)malloc(g.nblk * 4);
  uint64_t* sizes = (uint64_t*)malloc(g.nblk * 3 * 8);
  uint8_t* codec = (uint8_t*)malloc(g.nblk);
  run_t* runs = (run_t*)malloc(SLOTS * sizeof(run_t));
  uint64_t nrec = 0;
  {
    /* prequantization, then the residuals under the chunking of g */
    int32_t* K = (int32_t*)malloc(g.nelem * sizeof(int32_t));
    uint8_t* P = x64 ? NULL : (uint8_t*)malloc(g.nelem);
    if (!K || (!x64 && !P)) {
      free(K);
      free(P);
      st = ORC_E_CAPACITY;
      goto done;
    }
    for (uint64_t e = 0; e < g.nelem && !st; e++) {
      if (x64) {
        st = orc_prequant_f64(x64[e], eb_d, step, rstep, &K[e]);
      } else {
        int patch = 0;
        st = orc_prequant(x32[e], eb_f, ebx2_f, ebx2_r, &K[e], &patch);
        P[e] = (uint8_t)patch;
      }
    }
    if (!st) st = construct_k(K, P, x32, &g, radius, codes, rk, rv, 2 * g.nelem + 1, &nrec, hist);
    free(K);
    free(P);
  }
  if (st) goto done;
  const int all_blocks = select == ORC_SEL_RLE_HUFF || select == ORC_SEL_RLE;
  orc_run_stats(codes, ndim, dims, all_blocks, vh, lh, nruns);

  uint8_t clen[NSYM_CODE], vlen[NSYM_CODE], llen[NSYM_LEN];
  uint64_t ccode[NSYM_CODE], vcode[NSYM_CODE], lcode[NSYM_LEN];
  if ((st = orc_huffman_lengths(hist, NSYM_CODE, clen))) goto done;
  if ((st = orc_huffman_lengths(vh, NSYM_CODE, vlen))) goto done;
  if ((st = orc_huffman_lengths(lh, NSYM_LEN, llen))) goto done;
  orc_canonical_codes(clen, NSYM_CODE, ccode);
  orc_canonical_codes(vlen, NSYM_CODE, vcode);
  orc_canonical_codes(llen, NSYM_LEN, lcode);
  st = orc_block_sizes(codes, ndim, dims, radius, clen, vlen, llen, LANES, all_blocks, sizes);
  if (st) goto done;

  /* codec per block */
  uint64_t payload = 0, ncodec[3] = {0, 0, 0};
  for (uint64_t b = 0; b < g.nblk; b++) {
    const uint64_t* s = sizes + 3 * b;
    int c;
    if (select <= ORC_SEL_RLE_HUFF) {
      c = select;
    } else if (select == ORC_SEL_EXHAUSTIVE) {
      c = exhaustive_pick(s);
    } else if (!run_eligible(nruns[b], block_count(&g, b), 0)) {
      c = ORC_CODEC_HUFF; /* heuristic and learned choose between Huffman and RLE+Huffman */
    } else if (select == ORC_SEL_HEURISTIC) {
      uint32_t bh[NSYM_CODE] = {0};
      uint64_t m = block_count(&g, b);
      for (uint64_t i = 0; i < m; i++) bh[codes[b * SLOTS + i]]++;
      c = orc_heuristic_pick(bh, NSYM_CODE, (uint32_t)m);
    } else {
      float f[8], y[3];
      features_of(codes + b * SLOTS, block_count(&g, b), radius, f);
      orc_mlp_forward(mlp_w, f, 1, y);
      c = orc_learned_pick(y, s);
    }
    codec[b] = (uint8_t)c;
    ncodec[c]++;
    payload += s[c];
  }
  uint32_t flags = (ncodec[ORC_CODEC_HUFF] ? 1u : 0u) | (ncodec[ORC_CODEC_RLE_HUFF] ? 2u : 0u) |
                   (x64 ? ORC_FLAG_F64 : 0u) | (global ? ORC_FLAG_GLOBAL : 0u);
  uint64_t off_bb = HDR + align8(g.nblk);
  uint64_t off_rec = off_bb + align8(4 * g.nblk);
  uint64_t off_pay = off_rec + 8 * nrec;
  uint64_t off_books = off_pay + align8(payload);
  uint64_t total = off_books + ((flags & 1) ? NSYM_CODE : 0) + ((flags & 2) ? NSYM_CODE + NSYM_LEN : 0);
  *out_bytes = (size_t)total;
  if (total > cap) {
    st = ORC_E_CAPACITY;
    goto done;
  }
  memset(out, 0, (size_t)total);
  hdr_t h;
  memset(&h, 0, sizeof(h));
  h.magic = MAGIC;
  h.version = VERSION;
  h.ndim = (uint8_t)ndim;
  h.eb_mode = (uint8_t)eb_mode;
  for (int i = 0; i < ndim; i++) h.dims[i] = dims[i];
  h.eb_user = eb;
  h.eb_d = eb_d;
  h.eb_f = eb_f;
  h.radius = radius;
  h.lanes = LANES;
  h.flags = flags;
  h.nblk = g.nblk;
  h.n_rec = nrec;
  for (uint64_t i = 0; i < nrec; i++) {
    if (rk[i] & 1)
      h.n_patch++;
    else
      h.n_out++;
  }
  h.payload = payload;
  h.total = total;
  h.select = (uint32_t)select;
  for (int i = 0; i < 3; i++) h.n_codec[i] = (uint32_t)ncodec[i];
  write_header(out, &h);
  memcpy(out + HDR, codec, g.nblk);
  for (uint64_t b = 0; b < g.nblk; b++) put32(out + off_bb + 4 * b, (uint32_t)sizes[3 * b + codec[b]]);
  for (uint64_t i = 0; i < nrec; i++) {
    put32(out + off_rec + 8 * i, rk[i]);
    put32(out + off_rec + 8 * i + 4, rv[i]);
  }
  uint8_t* p = out + off_pay;
  for (uint64_t b = 0; b < g.nblk; b++) {
    uint64_t m = block_count(&g, b);
    const uint16_t* c = codes + b * SLOTS;
    if (codec[b] == ORC_CODEC_HUFF) {
      huff_write(c, m, clen, ccode, p);
    } else {
      uint64_t nr = make_runs(c, m, runs);
      if (codec[b] == ORC_CODEC_RLE)
        rle_write(runs, nr, p);
      else
        rlehuff_write(runs, nr, vlen, vcode, llen, lcode, p);
    }
    p += sizes[3 * b + codec[b]];
  }
  uint8_t* bk = out + off_books;
  if (flags & 1) {
    memcpy(bk, clen, NSYM_CODE);
    bk += NSYM_CODE;
  }
  if (flags & 2) {
    memcpy(bk, vlen, NSYM_CODE);
    memcpy(bk + NSYM_CODE, llen, NSYM_LEN);
  }
  st = ORC_OK;
done:
  free(codes);
  free(rk);
  free(rv);
  free(nruns);
  free(sizes);
  free(codec);
  free(runs);
  return st;
}

int orc_compress(const float* x, int ndim, const uint64_t* dims, int eb_mode, double eb,
                 uint32_t radius, int select, const float* mlp_w, uint8_t* out, size_t cap,
                 size_t* out_bytes) {
  return compress_impl(x, NULL, ndim, dims, eb_mode, eb, radius, select, mlp_w, 0, out, cap, out_bytes);
}

int orc_compress_f64(const double* x, int ndim, const uint64_t* dims, int eb_mode, double eb,
                     uint32_t radius, int select, const float* mlp_w, uint8_t* out, size_t cap,
                     size_t* out_bytes) {
  return compress_impl(NULL, x, ndim, dims, eb_mode, eb, radius, select, mlp_w, 0, out, cap, out_bytes);
}

int orc_compress_ex(const float* x32, const double* x64, int ndim, const uint64_t* dims, int eb_mode,
                    double eb, uint32_t radius, int select, const float* mlp_w, int global, uint8_t* out,
                    size_t cap, size_t* out_bytes) {
  if ((x32 == NULL) == (x64 == NULL)) return ORC_E_ARG;
  return compress_impl(x32, x64, ndim, dims, eb_mode, eb, radius, select, mlp_w, global, out, cap, out_bytes);
}

/* parse and validate an archive: header, sections, books, per-block decode into codes */
typedef struct {
  hdr_t h;
  geom_t g;
  uint64_t off_bb, off_rec, off_pay, off_books;
  uint8_t clen[NSYM_CODE], vlen[NSYM_CODE], llen[NSYM_LEN];
} parsed_t;

static int parse(const uint8_t* ar, size_t bytes, parsed_t* P) {
  if (!ar || bytes < HDR) return ORC_E_CORRUPT;
  hdr_t* h = &P->h;
  read_header(ar, h);
  if (h->magic != MAGIC || h->version != VERSION) return ORC_E_CORRUPT;
  if (h->ndim < 1 || h->ndim > 3 || h->eb_mode > 1) return ORC_E_CORRUPT;
  if (make_geom(h->ndim, h->dims, &P->g)) return ORC_E_CORRUPT;
  for (int i = h->ndim; i < 3; i++)
    if (h->dims[i]) return ORC_E_CORRUPT;
  if (h->radius < 1 || h->radius > 512 || h->lanes != LANES || h->flags > 15) return ORC_E_CORRUPT;
  if (h->flags & ORC_FLAG_GLOBAL) make_global(&P->g);
  if (h->nblk != P->g.nblk || h->n_rec != h->n_out + h->n_patch) return ORC_E_CORRUPT;
  if (h->flags & ORC_FLAG_F64) {
    /* double fields: the step follows from eb_d; there are no verbatim patches */
    double d = h->eb_d, stp = (2.0 * d) * (1.0 - 0x1p-24);
    if (!(d > 0.0) || !isfinite(d) || !(stp > 0.0) || !isfinite(stp) || h->n_patch) return ORC_E_CORRUPT;
  } else if (!(h->eb_f > 0.0f) || !isfinite(2.0f * h->eb_f)) {
    return ORC_E_CORRUPT;
  }
  if (h->n_rec > 2 * P->g.nelem || h->payload > bytes || (h->payload & 3)) return ORC_E_CORRUPT;
  P->off_bb = HDR + align8(h->nblk);
  P->off_rec = P->off_bb + align8(4 * h->nblk);
  P->off_pay = P->off_rec + 8 * h->n_rec;
  P->off_books = P->off_pay + align8(h->payload);
  uint64_t total = P->off_books + ((h->flags & 1) ? NSYM_CODE : 0) +
                   ((h->flags & 2) ? NSYM_CODE + NSYM_LEN : 0);
  if (h->total != total || total > bytes) return ORC_E_CORRUPT;
  memset(P->clen, 0, sizeof(P->clen));
  memset(P->vlen, 0, sizeof(P->vlen));
  memset(P->llen, 0, sizeof(P->llen));
  const uint8_t* bk = ar + P->off_books;
  if (h->flags & 1) {
    memcpy(P->clen, bk, NSYM_CODE);
    bk += NSYM_CODE;
  }
  if (h->flags & 2) {
    memcpy(P->vlen, bk, NSYM_CODE);
    memcpy(P->llen, bk + NSYM_CODE, NSYM_LEN);
  }
  for (int s = 2 * (int)h->radius; s < NSYM_CODE; s++)
    if (P->clen[s] || P->vlen[s]) return ORC_E_CORRUPT;
  if (!kraft_ok(P->clen, NSYM_CODE) || !kraft_ok(P->vlen, NSYM_CODE) || !kraft_ok(P->llen, NSYM_LEN))
    return ORC_E_CORRUPT;
  uint64_t sum = 0, nc[3] = {0, 0, 0};
  for (uint64_t b = 0; b < h->nblk; b++) {
    uint8_t c = ar[HDR + b];
    if (c > 2) return ORC_E_CORRUPT;
    nc[c]++;
    uint32_t bb = get32(ar + P->off_bb + 4 * b);
    if (bb & 3) return ORC_E_CORRUPT;
    sum += bb;
  }
  if (sum != h->payload) return ORC_E_CORRUPT;
  if ((nc[0] && !(h->flags & 1)) || (nc[2] && !(h->flags & 2))) return ORC_E_CORRUPT;
  return ORC_OK;
}

static int decode_block(const parsed_t* P, const uint8_t* pay, uint64_t bytes, int codec,
                        uint64_t m, const dectab_t* tc, const dectab_t* tv, const dectab_t* tl,
                        uint16_t* c) {
  const uint32_t nsym = 2 * P->h.radius;
  if (codec == ORC_CODEC_HUFF) {
    uint64_t nu = bytes / 2;
    if (nu < 1) return ORC_E_CORRUPT;
    uint16_t* u = (uint16_t*)malloc((nu + 1) * sizeof(uint16_t));
    memcpy(u, pay, 2 * nu);
    const uint64_t h = huff_split(m), na = u[0];
    int64_t ua = -1, ub = -1;
    if (na <= nu - 1) {
      ua = ihs_decode(u + 1, na, h, tc, c);
      if (ua == (int64_t)na) ub = ihs_decode(u + 1 + na, nu - 1 - na, m - h, tc, c + h);
    }
    free(u);
    if (ua != (int64_t)na || ub < 0 || align4(2 * (1 + na + (uint64_t)ub)) != bytes) return ORC_E_CORRUPT;
    for (uint64_t i = 0; i < m; i++)
      if (c[i] >= nsym) return ORC_E_CORRUPT;
    return ORC_OK;
  }
  run_t* runs = (run_t*)malloc((SLOTS + 1) * sizeof(run_t));
  uint64_t nr;
  if (codec == ORC_CODEC_RLE) {
    nr = bytes / 4;
    if (nr > m) {
      free(runs);
      return ORC_E_CORRUPT;
    }
    for (uint64_t i = 0; i < nr; i++) {
      memcpy(&runs[i].v, pay + 2 * i, 2);
      memcpy(&runs[i].len, pay + 2 * nr + 2 * i, 2);
    }
  } else {
    if (bytes < 8) {
      free(runs);
      return ORC_E_CORRUPT;
    }
    nr = get32(pay);
    uint64_t vu = get32(pay + 4);
    if (nr > m || 8 + 2 * vu > bytes) {
      free(runs);
      return ORC_E_CORRUPT;
    }
    uint64_t lavail = (bytes - 8) / 2 - vu;
    uint16_t* u = (uint16_t*)malloc((vu + lavail + 1) * sizeof(uint16_t));
    uint16_t* v = (uint16_t*)malloc((nr + 1) * sizeof(uint16_t));
    uint16_t* l = (uint16_t*)malloc((nr + 1) * sizeof(uint16_t));
    memcpy(u, pay + 8, 2 * (vu + lavail));
    int64_t uv = ihs_decode(u, vu, nr, tv, v);
    int64_t ul = ihs_decode(u + vu, lavail, nr, tl, l);
    int ok = uv >= 0 && (uint64_t)uv == vu && ul >= 0 && align4(8 + 2 * (vu + (uint64_t)ul)) == bytes;
    for (uint64_t i = 0; ok && i < nr; i++) {
      runs[i].v = v[i];
      runs[i].len = (uint16_t)(l[i] + 1);
    }
    free(u);
    free(v);
    free(l);
    if (!ok) {
      free(runs);
      return ORC_E_CORRUPT;
    }
  }
  uint64_t pos = 0;
  for (uint64_t i = 0; i < nr; i++) {
    if (runs[i].v >= nsym || runs[i].len == 0 || pos + runs[i].len > m) {
      free(runs);
      return ORC_E_CORRUPT;
    }
    for (uint64_t t = 0; t < runs[i].len; t++) c[pos++] = runs[i].v;
  }
  free(runs);
  return pos == m ? ORC_OK : ORC_E_CORRUPT;
}

static int decode_all(const uint8_t* ar, size_t bytes, parsed_t* P, uint16_t* codes) {
  dectab_t* tabs = (dectab_t*)malloc(3 * sizeof(dectab_t));
  build_dectab(P->clen, NSYM_CODE, &tabs[0]);
  build_dectab(P->vlen, NSYM_CODE, &tabs[1]);
  build_dectab(P->llen, NSYM_LEN, &tabs[2]);
  (void)bytes;
  memset(codes, 0, P->g.nblk * SLOTS * sizeof(uint16_t));
  uint64_t off = P->off_pay;
  int st = ORC_OK;
  for (uint64_t b = 0; b < P->h.nblk && st == ORC_OK; b++) {
    uint32_t bb = get32(ar + P->off_bb + 4 * b);
    st = decode_block(P, ar + off, bb, ar[HDR + b], block_count(&P->g, b), &tabs[0], &tabs[1],
                      &tabs[2], codes + b * SLOTS);
    off += bb;
  }
  free(tabs);
  return st;
}

int orc_decode_codes(const uint8_t* ar, size_t bytes, uint16_t* codes, uint64_t cap_slots) {
  parsed_t* P = (parsed_t*)malloc(sizeof(parsed_t));
  int st = parse(ar, bytes, P);
  if (st == ORC_OK && cap_slots < P->g.nblk * SLOTS) st = ORC_E_CAPACITY;
  if (st == ORC_OK) st = decode_all(ar, bytes, P, codes);
  free(P);
  return st;
}

/*
 * Decompression (Alg. 1 decompression part, read through the recurrence it replaces):
 * fuse q' = q - r, or delta at an outlier slot (Sec. IV-B1), then rebuild each
 * prequantized integer sequentially, k = p(k) + q', in raster order (every
 * predictor neighbour precedes its element).  K receives the integers; the callers
 * scale them by the quantization step and put back the verbatim patches.
 */
static int rebuild_k(const uint8_t* ar, size_t bytes, parsed_t* P, int32_t* K) {
  const geom_t* g = &P->g;
  uint64_t slots = g->nblk * SLOTS;
  uint16_t* codes = (uint16_t*)malloc(slots * sizeof(uint16_t));
  int32_t* qp = (int32_t*)malloc(slots * sizeof(int32_t));
  int st = decode_all(ar, bytes, P, codes);
  if (st) goto fail;
  const int32_t r = (int32_t)P->h.radius;
  for (uint64_t s = 0; s < slots; s++) qp[s] = (int32_t)codes[s] - r;
  uint64_t prev = 0;
  for (uint64_t i = 0; i < P->h.n_rec; i++) {
    uint32_t key = get32(ar + P->off_rec + 8 * i);
    uint32_t val = get32(ar + P->off_rec + 8 * i + 4);
    uint64_t slot = key >> 1;
    if ((i > 0 && key <= prev) || slot >= slots || slot % SLOTS >= block_count(g, slot / SLOTS)) {
      st = ORC_E_CORRUPT;
      goto fail;
    }
    prev = key;
    if ((key & 1) == 0) qp[slot] = (int32_t)val;
  }
  for (uint64_t z = 0; z < g->n[0]; z++)
    for (uint64_t y = 0; y < g->n[1]; y++)
      for (uint64_t x = 0; x < g->n[2]; x++) {
        uint64_t e = (z * g->n[1] + y) * g->n[2] + x;
        int64_t k = lorenzo_predict(K, g, z, y, x) + qp[slot_of(g, z, y, x)];
        K[e] = (int32_t)(uint32_t)k; /* modular int32: the exact k of a valid archive */
      }
  st = ORC_OK;
fail:
  free(codes);
  free(qp);
  return st;
}

/* FP32 archive: x' = fl32(k * 2 eb_f), then the verbatim patches */
int orc_decompress(const uint8_t* ar, size_t bytes, float* out, uint64_t cap_elems) {
  parsed_t* P = (parsed_t*)malloc(sizeof(parsed_t));
  int st = parse(ar, bytes, P);
  if (st == ORC_OK && (P->h.flags & ORC_FLAG_F64)) st = ORC_E_ARG; /* a double field */
  if (st == ORC_OK && cap_elems < P->g.nelem) st = ORC_E_CAPACITY;
  int32_t* K = st ? NULL : (int32_t*)malloc(P->g.nelem * sizeof(int32_t));
  if (st == ORC_OK) st = rebuild_k(ar, bytes, P, K);
  if (st == ORC_OK) {
    const geom_t* g = &P->g;
    const float ebx2 = 2.0f * P->h.eb_f;
    for (uint64_t e = 0; e < g->nelem; e++) out[e] = (float)K[e] * ebx2;
    for (uint64_t i = 0; i < P->h.n_rec; i++) {
      uint32_t key = get32(ar + P->off_rec + 8 * i);
      if (key & 1) {
        uint32_t val = get32(ar + P->off_rec + 8 * i + 4);
        memcpy(&out[elem_of_slot(g, key >> 1)], &val, 4);
      }
    }
  }
  free(K);
  free(P);
  return st;
}

/* double archive: x' = fl64(k * step), step = fl64(2 eb_d (1 - 2^-24)) */
int orc_decompress_f64(const uint8_t* ar, size_t bytes, double* out, uint64_t cap_elems) {
  parsed_t* P = (parsed_t*)malloc(sizeof(parsed_t));
  int st = parse(ar, bytes, P);
  if (st == ORC_OK && !(P->h.flags & ORC_FLAG_F64)) st = ORC_E_ARG; /* an FP32 field */
  if (st == ORC_OK && cap_elems < P->g.nelem) st = ORC_E_CAPACITY;
  int32_t* K = st ? NULL : (int32_t*)malloc(P->g.nelem * sizeof(int32_t));
  if (st == ORC_OK) st = rebuild_k(ar, bytes, P, K);
  if (st == ORC_OK) {
    const double step = (2.0 * P->h.eb_d) * (1.0 - 0x1p-24);
    for (uint64_t e = 0; e < P->g.nelem; e++) out[e] = (double)K[e] * step;
  }
  free(K);
  free(P);
  return st;
}
