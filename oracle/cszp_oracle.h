/*
 * Scalar CPU oracle of the cuSZ+ error-bounded lossy compressor
 * (Tian et al., "Optimizing Error-Bounded Lossy Compression for Scientific Data
 * on GPUs", arXiv 2105.12912).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  It shares no code, header,
 * table or constant generator with the CUDA library; the archive layout and
 * status numbers are restated here independently because both sides must
 * produce the same bytes.
 *
 * Every function follows a passage of the paper (cited at its definition) or,
 * where the paper is silent, a reading written down next to it.
 */
#ifndef CSZP_ORACLE_H
#define CSZP_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
enum {
  ORC_OK = 0,
  ORC_E_ARG = 1,
  ORC_E_NONFINITE = 2,
  ORC_E_RANGE = 3,
  ORC_E_CORRUPT = 4,
  ORC_E_CAPACITY = 5
};

/* error-bound modes: absolute, or relative to the value range (Sec. II-B table captions, Sec. V-C) */
enum { ORC_EB_ABS = 0, ORC_EB_REL = 1 };

/* selection modes: three forced codecs and three adaptive pickers */
enum {
  ORC_SEL_HUFF = 0,
  ORC_SEL_RLE = 1,
  ORC_SEL_RLE_HUFF = 2,
  ORC_SEL_HEURISTIC = 3,
  ORC_SEL_EXHAUSTIVE = 4,
  ORC_SEL_LEARNED = 5
};

/* per-block codec identifiers stored in the archive */
enum { ORC_CODEC_HUFF = 0, ORC_CODEC_RLE = 1, ORC_CODEC_RLE_HUFF = 2 };

#define ORC_MLP_IN 8
#define ORC_MLP_H 32
#define ORC_MLP_OUT 3
#define ORC_MLP_PARAMS (ORC_MLP_H * ORC_MLP_IN + ORC_MLP_H + ORC_MLP_H * ORC_MLP_H + ORC_MLP_H + \
                        ORC_MLP_OUT * ORC_MLP_H + ORC_MLP_OUT)
/* learned selection falls back to the exact sizes when the runner-up prediction is
   within this many log2 units (about 2%) of the best */
#define ORC_MLP_MARGIN 0.028569152f

/* ---- whole-pipeline entry points ------------------------------------------------ */
size_t orc_max_archive_bytes(int ndim, const uint64_t* dims);

int orc_compress(const float* x, int ndim, const uint64_t* dims, int eb_mode, double eb,
                 uint32_t radius, int select, const float* mlp_w, uint8_t* out, size_t cap,
                 size_t* out_bytes);

int orc_decompress(const uint8_t* ar, size_t bytes, float* out, uint64_t cap_elems);

/* double-precision fields: the same archive with flag ORC_FLAG_F64; prequantization in
   double with the step 2 eb (1 - 2^-24), reconstruction x' = fl64(k * step), and the
   guarantee |x - x'| <= eb_d on every element.  orc_decompress refuses such an
   archive (ORC_E_ARG), orc_decompress_f64 an FP32 one. */
#define ORC_FLAG_F64 4u
/* global (unchunked) Lorenzo: one chunk spans the whole field, so prediction reads
   zero only outside it; the archive carries flag ORC_FLAG_GLOBAL and decompresses
   through the same recurrence */
#define ORC_FLAG_GLOBAL 8u
/* general entry: exactly one of x32 / x64; global selects the unchunked predictor */
int orc_compress_ex(const float* x32, const double* x64, int ndim, const uint64_t* dims, int eb_mode,
                    double eb, uint32_t radius, int select, const float* mlp_w, int global, uint8_t* out,
                    size_t cap, size_t* out_bytes);
int orc_compress_f64(const double* x, int ndim, const uint64_t* dims, int eb_mode, double eb,
                     uint32_t radius, int select, const float* mlp_w, uint8_t* out, size_t cap,
                     size_t* out_bytes);
int orc_decompress_f64(const uint8_t* ar, size_t bytes, double* out, uint64_t cap_elems);
int orc_value_range_f64(const double* x, uint64_t n, double* vmin, double* vmax);
int orc_eb_params_f64(int eb_mode, double eb, double vmin, double vmax, double* eb_d, double* step,
                      double* rstep);
int orc_prequant_f64(double x, double eb_d, double step, double rstep, int32_t* k);
int orc_construct_f64(const double* x, int ndim, const uint64_t* dims, double eb_d, double step,
                      double rstep, uint32_t radius, uint16_t* codes, uint32_t* rec_key,
                      uint32_t* rec_val, uint64_t rec_cap, uint64_t* n_rec, uint32_t* hist);

/* ---- stage-level entry points (parity and pin tests) ------------------------------ */
int orc_value_range(const float* x, uint64_t n, float* vmin, float* vmax);

int orc_eb_params(int eb_mode, double eb, float vmin, float vmax, double* eb_d, float* eb_f,
                  float* ebx2_f, float* ebx2_r);

/* prequantization of one value (Sec. IV-A1); returns ORC_OK/ORC_E_RANGE/ORC_E_NONFINITE */
int orc_prequant(float x, float eb_f, float ebx2_f, float ebx2_r, int32_t* k, int* patch);

/* number of codec blocks and slots (4096 per block) of a shape */
int orc_geometry(int ndim, const uint64_t* dims, uint64_t* nblk, uint64_t* nelem);

/* Lorenzo construction: codes[nblk*4096] (block-major, dense within a block),
   records sorted by key, global histogram hist[1024]. */
int orc_construct(const float* x, int ndim, const uint64_t* dims, float eb_f, float ebx2_f,
                  float ebx2_r, uint32_t radius, uint16_t* codes, uint32_t* rec_key,
                  uint32_t* rec_val, uint64_t rec_cap, uint64_t* n_rec, uint32_t* hist);

/* runs of each block: value histogram [1024], length histogram [4096] (index len-1)
   over run-eligible blocks (every block if all_blocks), runs per block */
int orc_run_stats(const uint16_t* codes, int ndim, const uint64_t* dims, int all_blocks,
                  uint32_t* val_hist, uint32_t* len_hist, uint32_t* nruns);

/* Huffman code lengths (two-queue construction) and canonical codes */
int orc_huffman_lengths(const uint32_t* freq, int nsym, uint8_t* len);
int orc_canonical_codes(const uint8_t* len, int nsym, uint64_t* code);

/* per-block exact encoded sizes [nblk][3] (bytes) for the three codecs (UINT64_MAX for
   RLE+Huffman of a block that is not run-eligible); lanes must be 32 (the interleave
   width of Huffman streams) */
int orc_block_sizes(const uint16_t* codes, int ndim, const uint64_t* dims, uint32_t radius,
                    const uint8_t* code_len, const uint8_t* val_len, const uint8_t* len_len,
                    uint32_t lanes, int all_blocks, uint64_t* sizes);

/* per-block selector features [nblk][8] */
int orc_block_features(const uint16_t* codes, int ndim, const uint64_t* dims, uint32_t radius,
                       float* feat);

/* training rows of the learned selector from exact sizes [nblk][3]: target[b][c] is
   log2 of codec c's bits per element in Q16 steps, ((log2q16(8 size) - log2q16(m)) /
   65536, exact in FP32); valid[b] = 1 where the block is run-eligible, i.e. where
   the learned selector decides (other blocks are Huffman-coded) */
int orc_selector_targets(const uint64_t* sizes, int ndim, const uint64_t* dims, float* target,
                         uint8_t* valid);

/* the learned selector's pick from predictions y[3] and exact sizes s[3] */
int orc_learned_pick(const float* y, const uint64_t* s);

/* the paper's histogram heuristic for one block: returns the codec it picks */
int orc_heuristic_pick(const uint32_t* block_hist, int nsym, uint32_t m);

/* fixed-point binary logarithm used by the heuristic and the features */
uint32_t orc_log2_q16(uint64_t v);

/* MLP selector: forward in FP32 with fused multiply-adds in a fixed order */
void orc_mlp_forward(const float* w, const float* feat, uint64_t nrows, float* out);
/* MSE loss and gradient in double precision over rows (for gradient checks) */
double orc_mlp_loss_grad_f64(const float* w, const float* feat, const float* target,
                             uint64_t nrows, double* grad);

/* decode the code stream of an archive into codes[nblk*4096] (parity of decoding) */
int orc_decode_codes(const uint8_t* ar, size_t bytes, uint16_t* codes, uint64_t cap_slots);

#ifdef __cplusplus
}
#endif
#endif
