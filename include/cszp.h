/*
 * cszp -- GB300 (sm_103a) error-bounded lossy compressor: the data-parallel path of
 * cuSZ+ (Tian et al., "Optimizing Error-Bounded Lossy Compression for Scientific
 * Data on GPUs", arXiv 2105.12912).
 *
 * C ABI: plain pointers and sizes, no CUDA or PyTorch types.  A `stream` argument is
 * a cudaStream_t passed as void* (NULL = the legacy default stream).
 *
 * Ownership: the caller owns every buffer.  Device buffers (field, archive, output,
 * workspace) are caller-allocated device memory; the library allocates nothing
 * during a call.  Host pointers are marked h_.
 *
 * Errors: every call returns a csz_status; nothing throws across the ABI.  On error
 * the contents of output buffers are unspecified, but no write ever leaves the
 * capacity the caller passed.  Device-side failures (non-finite input, range,
 * corrupt archive, capacity, a bounded wait that expired) are reported through the
 * single synchronisation each call performs.
 *
 * Layout: fields are row-major FP32 with dims given slowest-first (dims[ndim-1] is
 * the contiguous axis).  ndim is 1, 2 or 3; every extent is >= 1 and < 2^31, and
 * the shape may hold at most 524287 codec blocks (1-D: 4096 elements, 2-D: 64x64,
 * 3-D: 16^3 per block).
 */
#ifndef CSZP_H
#define CSZP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CSZ_OK = 0,
  CSZ_E_ARG = 1,       /* bad argument, empty shape, zero/negative/non-finite bound */
  CSZ_E_NONFINITE = 2, /* the field holds NaN or Inf */
  CSZ_E_RANGE = 3,     /* |x| / (2 eb) reaches 2^23: eb too small for the data */
  CSZ_E_CORRUPT = 4,   /* archive failed validation */
  CSZ_E_CAPACITY = 5,  /* output or workspace buffer too small */
  CSZ_E_CUDA = 6,      /* a CUDA runtime call failed */
  CSZ_E_TIMEOUT = 7    /* a bounded device-side wait expired */
} csz_status;

/* Error-bound mode (Sec. II-B table captions, Sec. V-C): absolute, or relative to the field's value range
   (eb_abs = eb * (max - min), computed in double). */
typedef enum { CSZ_EB_ABS = 0, CSZ_EB_REL = 1 } csz_eb_mode;

/* Per-block codec selection.  The first three force one codec on every block;
   HEURISTIC is the paper's histogram estimate with the 1.09-bit rule (Sec. III-B);
   EXHAUSTIVE computes all three exact sizes and keeps the smallest; LEARNED runs
   the 8-32-32-3 MLP selector on per-block statistics.  The choice only changes
   the encoding: reconstructions are identical. */
typedef enum {
  CSZ_SEL_HUFF = 0,
  CSZ_SEL_RLE = 1,
  CSZ_SEL_RLE_HUFF = 2,
  CSZ_SEL_HEURISTIC = 3,
  CSZ_SEL_EXHAUSTIVE = 4,
  CSZ_SEL_LEARNED = 5
} csz_select;

typedef struct {
  uint32_t radius;               /* quantization radius r (Alg. 1), 1..512; 0 = 512 */
  uint32_t select;               /* csz_select; default EXHAUSTIVE */
  const float* selector_weights; /* device pointer, CSZ_MLP_PARAMS floats; LEARNED only */
  uint32_t flags;                /* CSZ_FLAG_* bits; 0 = chunked Lorenzo */
  uint32_t reserved[3];          /* must be zero */
} csz_options;

/* Global (unchunked) Lorenzo prediction: one chunk spans the whole field, so the
   predictor reads zero only outside the field, not at every chunk face (the paper's
   partial-sum reconstruction, Sec. IV-B, holds for the whole field).  Smaller
   archives on smooth fields; compression and decompression take more passes.
   Single-field FP32 calls only (csz_compress / csz_compress_with_header with this
   flag; decompression follows the archive's header flag): CSZ_E_ARG for double
   fields and batches. */
#define CSZ_FLAG_GLOBAL_LORENZO 1u

#define CSZ_MLP_PARAMS 1443 /* W1[32][8] b1[32] W2[32][32] b2[32] W3[3][32] b3[3] */

/* Worst-case archive size for a shape (0 if the shape is invalid). */
size_t csz_max_archive_bytes(int ndim, const uint64_t* dims);

/* Device workspace both csz_compress and csz_decompress need for a shape
   (0 if the shape is invalid).  The workspace may be reused across calls on one
   stream; calls that run concurrently need separate workspaces. */
size_t csz_workspace_bytes(int ndim, const uint64_t* dims);

/*
 * Compress a device-resident FP32 field (Sec. IV-A; Alg. 1 compression part):
 * value range (REL), dual-quantization Lorenzo construction with outliers that keep
 * delta, histograms, canonical Huffman books, per-block codec selection and
 * encoding.  Writes the archive to d_archive (capacity archive_cap bytes) and its
 * size to *h_archive_bytes.  Synchronises `stream` once, to read the size and the
 * device status.
 * Guarantee: every reconstructed element x' satisfies |x - x'| <= eb_f, where eb_f
 * is the largest float not above the absolute bound.
 */
csz_status csz_compress(const float* d_field, int ndim, const uint64_t* dims, int eb_mode,
                        double eb, const csz_options* opt, void* d_workspace,
                        size_t workspace_bytes, uint8_t* d_archive, size_t archive_cap,
                        size_t* h_archive_bytes, void* stream);

/*
 * csz_compress that also copies the archive's 128-byte header to h_header (host
 * memory, 128 bytes) within its one synchronisation, for csz_decompress_async.
 * h_header is written only when the call returns CSZ_OK; NULL is CSZ_E_ARG.
 */
csz_status csz_compress_with_header(const float* d_field, int ndim, const uint64_t* dims, int eb_mode,
                                    double eb, const csz_options* opt, void* d_workspace,
                                    size_t workspace_bytes, uint8_t* d_archive, size_t archive_cap,
                                    size_t* h_archive_bytes, uint8_t* h_header, void* stream);

/* Read shape and bound from an archive header held in host memory (first 128
   bytes suffice). */
csz_status csz_archive_info(const uint8_t* h_archive, size_t bytes, int* ndim, uint64_t* dims,
                            double* eb_abs, uint64_t* total_bytes);

/*
 * Decompress a device-resident archive into d_out (out_cap_elems floats): decode
 * each block's codes, fuse outliers, rebuild the prequantized integers as an N-D
 * partial sum per chunk and scale by 2 eb (Alg. 1 decompression part, Sec. IV-B).
 * Copies the 128-byte header to the host, then synchronises `stream` once at the
 * end to read the device status.
 */
csz_status csz_decompress(const uint8_t* d_archive, size_t bytes, float* d_out,
                          uint64_t out_cap_elems, void* d_workspace, size_t workspace_bytes,
                          void* stream);

/*
 * csz_decompress without any host synchronisation.  The caller passes the archive's
 * 128-byte header as a host copy (h_header: e.g. from csz_compress_with_header, or
 * read once and kept), so nothing is read back before the launches; the device
 * compares the archive's own header with that copy and reports a mismatch as
 * CSZ_E_CORRUPT.  The decompression's status (a csz_status value) is written to the
 * device word *d_status when the work completes in stream order.  The call returns
 * CSZ_OK once everything is enqueued, or an error it finds on the host before any
 * launch (a header copy that does not parse against `bytes`: CSZ_E_CORRUPT;
 * capacities: CSZ_E_CAPACITY; NULL pointers: CSZ_E_ARG).  d_out and the workspace
 * must stay untouched until the status is read.
 */
csz_status csz_decompress_async(const uint8_t* d_archive, size_t bytes, const uint8_t* h_header,
                                float* d_out, uint64_t out_cap_elems, void* d_workspace,
                                size_t workspace_bytes, uint32_t* d_status, void* stream);

/*
 * Double-precision fields (SZ's double datasets; the paper's kernels take FP32).  The
 * same method with prequantization in double: the quantization step is
 * step = fl64(2 eb_d (1 - 2^-24)), k = nearest integer to x / step (checked exactly
 * against the bound, moving to the neighbour if the product rounded across a half
 * point), and the reconstruction x' = fl64(k * step).  Guarantee: |x - x'| <= eb_d on
 * every element, with no verbatim patches (the shrink covers the rounding of
 * k * step).  |x / step| must stay below 2^27 (CSZ_E_RANGE otherwise).  The archive is
 * the FP32 layout with header flag 4; csz_decompress refuses it (CSZ_E_ARG) and
 * csz_decompress_f64 refuses an FP32 archive.  Arguments, workspace (the same size),
 * ownership and errors as for csz_compress / csz_decompress; the batch calls take FP32
 * fields only.
 */
csz_status csz_compress_f64(const double* d_field, int ndim, const uint64_t* dims, int eb_mode,
                            double eb, const csz_options* opt, void* d_workspace,
                            size_t workspace_bytes, uint8_t* d_archive, size_t archive_cap,
                            size_t* h_archive_bytes, void* stream);
csz_status csz_decompress_f64(const uint8_t* d_archive, size_t bytes, double* d_out,
                              uint64_t out_cap_elems, void* d_workspace, size_t workspace_bytes,
                              void* stream);

/* Bytes per element of the field an archive holds (4: FP32, 8: double), from its
   header in host memory; 0 if the header is not valid. */
int csz_archive_elem_bytes(const uint8_t* h_archive, size_t bytes);

/*
 * Decompression that allocates nothing and takes no workspace.  Some callers cannot
 * call cudaMalloc: a compression filter plug-in inside an I/O library is handed only
 * the archive and the output buffer, and an application whose device memory is all
 * reserved by its own pool allocator cannot let a library allocate beside it.  This
 * entry point uses a scratch array the library holds on every GPU that loads it
 * (1.25 MiB, kept until the process exits) instead of a workspace.  The paper has no
 * counterpart; it is a convenience of this library.
 *
 * Limit: archives of at most 64 codec blocks (1-D: 262,144 elements; 2-D: 64 blocks
 * of 64x64; 3-D: 64 blocks of 16^3).  Larger archives return CSZ_E_CAPACITY before
 * any device work.  Other arguments, output and errors as for csz_decompress.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture starts.
 * Every call shares the one array, which keeps the previous call's contents (each
 * call clears the status word it needs zeroed): calls that overlap on the GPU, from
 * two streams or two host threads, race and must be serialised by the caller.
 */
csz_status csz_decompress_static(const uint8_t* d_archive, size_t bytes, float* d_out,
                                 uint64_t out_cap_elems, void* stream);

/*
 * Batched compression (the batching pattern the build adds beyond the paper; each
 * field is compressed as csz_compress does it, Alg. 1 and Sec. III).  Many fields of
 * any shape and dimensionality are compressed by one persistent kernel launch: every
 * CTA runs the stages (value range, construction, books and record offsets,
 * encoding) as phases, taking the items of each phase from one ticket over all
 * fields and waiting, bounded, only for the field hand-overs an earlier phase
 * releases.  The staged plan, one launch per stage, is the alternative.
 * csz_batch_create validates the fields, lays out the workspace, uploads the tables,
 * chooses the plan (`autotune` flags: CSZ_BATCH_AUTOTUNE times every allowed
 * candidate -- either plan with 1..4 resident CTAs per SM -- on the batch, running it
 * a few times, and keeps the fastest; CSZ_BATCH_PERSISTENT or CSZ_BATCH_STAGED alone
 * restricts the candidates to one plan; with neither flag and no tuning the plan is
 * the persistent launch on every resident CTA), and captures it into a CUDA graph.
 * Each csz_batch_compress replays the graph on `stream` without synchronising; the
 * archives then hold exactly what csz_compress would write for each field with the
 * same options.  csz_batch_results synchronises and reads every field's archive
 * size and status.
 * The field pointers, archive buffers and workspace are baked into the graph: they
 * must stay valid, and keep their addresses, until csz_batch_destroy.  One batch
 * must not be replayed on two streams at once.  Options (radius, selector, MLP
 * weights) apply to every field.  The handle is host memory owned by the library.
 */
typedef struct {
  const float* d_field; /* device FP32 field, row-major, dims slowest-first */
  int ndim;
  uint64_t dims[3];
  int eb_mode;          /* csz_eb_mode */
  double eb;
  uint8_t* d_archive;   /* device archive buffer of archive_cap bytes */
  size_t archive_cap;
} csz_field;

typedef struct csz_batch csz_batch;

/* csz_batch_create `autotune` flags */
#define CSZ_BATCH_AUTOTUNE 1   /* time the candidate plans on the batch, keep the fastest */
#define CSZ_BATCH_STAGED 2     /* candidates: the staged launches */
#define CSZ_BATCH_PERSISTENT 4 /* candidates: the single persistent launch */

/* Workspace for a batch (0 if any field is invalid); it includes 124 KB per field of
   working memory for the persistent plan's run-length books. */
size_t csz_batch_workspace_bytes(int nfields, const csz_field* fields);
csz_status csz_batch_create(int nfields, const csz_field* fields, const csz_options* opt,
                            void* d_workspace, size_t workspace_bytes, int autotune,
                            void* stream, csz_batch** batch);
csz_status csz_batch_compress(csz_batch* batch, void* stream);
/* h_bytes[nfields] / h_status[nfields] (either may be NULL); returns the first
   failing field's status, or CSZ_OK. */
csz_status csz_batch_results(csz_batch* batch, uint64_t* h_bytes, int* h_status, void* stream);
/* The staged plan's construction grid the autotuner chose and the batch times (ms)
   it measured with 1..4 resident CTAs per SM (0 where not tried). */
csz_status csz_batch_info(const csz_batch* batch, int* construct_grid, double* tuned_ms);
/* The plan the graph holds: *persistent = 1 for the single persistent launch (0 for
   the staged launches), *grid its CTAs (the construction grid when staged), and
   persist_ms[4] the batch times (ms) of the persistent plan with 1..4 resident CTAs
   per SM (0 where not tried).  Any pointer may be NULL. */
csz_status csz_batch_plan(const csz_batch* batch, int* persistent, int* grid, double* persist_ms);
/*
 * Batched decompression, the counterpart of the above: one launch per stage (header
 * checks, set-up, entropy decoding, run expansion, reconstruction) for all fields,
 * captured into a CUDA graph at csz_batch_dec_create and replayed by
 * csz_batch_decompress.  Each field names its archive (archive_bytes readable
 * bytes), its output (out_cap_elems floats) and the shape it must decode to; the
 * headers are read and checked on the device at every replay, so the archives'
 * contents may change between replays as long as each keeps its shape.  A field
 * whose header or data fail validation gets CSZ_E_CORRUPT (CSZ_E_TIMEOUT for an
 * expired wait) in csz_batch_dec_results without disturbing the others.  Buffers
 * and workspace stay bound until csz_batch_dec_destroy.
 */
typedef struct {
  const uint8_t* d_archive;
  size_t archive_bytes;
  float* d_out;
  uint64_t out_cap_elems;
  int ndim;
  uint64_t dims[3];
} csz_dfield;

typedef struct csz_batch_dec csz_batch_dec;

size_t csz_batch_dec_workspace_bytes(int nfields, const csz_dfield* fields);
csz_status csz_batch_dec_create(int nfields, const csz_dfield* fields, void* d_workspace,
                                size_t workspace_bytes, void* stream, csz_batch_dec** batch);
csz_status csz_batch_decompress(csz_batch_dec* batch, void* stream);
/* Autotuner of the batch decoder's CTA shape: times the batch (three replays each)
   with entropy-decoding CTAs of 8, 16 and 32 warps (4, 8 and 16 codec blocks per
   CTA), keeps the fastest and re-captures the graph with it.  The shape never
   changes the output.  Call it once the archive buffers hold archives of the
   planned shapes (a tuning run decompresses them); it synchronises `stream`.
   h_warps (may be NULL) receives the chosen warps per CTA, h_ms[3] (may be NULL)
   the mean milliseconds of each shape. */
csz_status csz_batch_dec_tune(csz_batch_dec* batch, void* stream, int* h_warps, double* h_ms);
csz_status csz_batch_dec_results(csz_batch_dec* batch, int* h_status, void* stream);
void csz_batch_dec_destroy(csz_batch_dec* batch);

/* Where the last failing csz_batch_create / csz_batch_dec_create call stopped and
   the CUDA error it met. */
const char* csz_batch_last_error(void);
void csz_batch_destroy(csz_batch* batch);

/*
 * Learned codec selector (an extension beside the paper's Sec. III-B heuristic; the
 * paper has no learned selector).  The network maps 8 per-block statistics to the
 * predicted log2 bits per element of HUFF, RLE and RLE_HUFF; CSZ_SEL_LEARNED codes
 * each run-eligible block (at most one run per four codes) with the smallest
 * prediction, falling back to the exact sizes when the two best predictions are
 * within log2(1.02); other blocks are Huffman coded.  Parameters: CSZ_MLP_PARAMS
 * FP32 values, W1[32][8] b1[32] W2[32][32] b2[32] W3[3][32] b3[3] (row = output unit).
 *
 * csz_selector_rows: the method's own training data for one field.  Runs the
 * compression pipeline with exhaustive sizing but writes no archive; for every codec
 * block b (block-major order, as in the archive) it writes
 *   d_feat[b][8]    features: zero-residual fraction, code entropy (bits), top-code
 *                   probability, log2(1 + max |delta|) over in-range codes, runs per
 *                   element, outlier fraction, mean |delta|/r (outliers count 0), and
 *                   the RLE roughness of Sec. III-B (binary-variance madogram on the
 *                   pairs (i, i + 1 + 25 (i mod 8))); each a ratio of integers formed
 *                   with one FP32 division
 *   d_target[b][3]  log2 of each codec's bits per element, in 1/65536 steps
 *   d_sizes[b][3]   each codec's exact payload bytes (0xffffffff: not applicable)
 *   d_valid[b]      1 where the learned selector decides the block
 * Each output holds nblk rows.  Workspace, arguments and errors as for
 * csz_compress (radius 0 = 512).  Synchronises.
 */
csz_status csz_selector_rows(const float* d_field, int ndim, const uint64_t* dims, int eb_mode,
                             double eb, uint32_t radius, void* d_workspace, size_t workspace_bytes,
                             float* d_feat, float* d_target, uint32_t* d_sizes, uint8_t* d_valid,
                             void* stream);

/* Network outputs d_out[nrows][3] for d_feat[nrows][8], computed exactly as the
   encoder computes them (fused multiply-add chains from the bias, inputs in order).
   Synchronises. */
csz_status csz_selector_predict(const float* d_weights, const float* d_feat, uint64_t nrows,
                                float* d_out, void* stream);

/* Device workspace of csz_selector_grad / csz_selector_train for nrows rows. */
size_t csz_selector_workspace_bytes(uint64_t nrows);

/* Mean squared error over the rows with d_valid[r] != 0 (d_valid may be NULL: all
   rows) and all 3 outputs, and its gradient d_grad[CSZ_MLP_PARAMS] (FP32, summed in
   a fixed order: reproducible).  *h_loss (may be NULL) receives the loss.
   Synchronises. */
csz_status csz_selector_grad(const float* d_weights, const float* d_feat, const float* d_target,
                             const uint8_t* d_valid, uint64_t nrows, float* d_grad, double* h_loss,
                             void* d_workspace, size_t workspace_bytes, void* stream);

/* `steps` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8) on d_weights in
   place, learning rate decaying linearly from lr to lr/10.  *h_loss receives the
   loss at the weights the last step started from.  Synchronises once, at the end. */
csz_status csz_selector_train(float* d_weights, const float* d_feat, const float* d_target,
                              const uint8_t* d_valid, uint64_t nrows, uint32_t steps, float lr,
                              void* d_workspace, size_t workspace_bytes, double* h_loss,
                              void* stream);

/*
 * Failure-path self-test (a test aid).  Runs one bounded wait that nothing
 * satisfies, with the same code the pipeline uses: which = 0, the decoupled
 * look-back of a tile whose predecessor never publishes; which = 1, an mbarrier
 * phase that no copy or arrival completes; which = 2, a field hand-over of the
 * batched persistent kernel (a counter no earlier phase releases, read with
 * acquire semantics).  The wait gives up after spin_limit
 * tries, the kernel sets the timeout bit and returns, and the call reports
 * CSZ_E_TIMEOUT.  The context stays usable.  d_scratch: device memory, at least
 * 512 bytes, overwritten.  Synchronises `stream`.
 */
csz_status csz_wait_selftest(int which, uint32_t spin_limit, void* d_scratch, size_t scratch_bytes,
                             void* stream);

/* Human-readable name of a status. */
const char* csz_status_string(int status);

/*
 * Kernel tracing (benchmarking aid; process-global, not thread-safe).
 * csz_kernel_count() kernels are numbered 0..count-1 and named by csz_kernel_name().
 * Launch counts are always kept.  While tracing is enabled every launch is bracketed
 * by CUDA events on the caller's stream and the elapsed milliseconds are added to the
 * kernel's total at the call's synchronisation.  While tracing is enabled,
 * csz_batch_compress and csz_batch_decompress launch their kernels one by one instead
 * of replaying the graph, so that each gets its events, and synchronise `stream`
 * before returning.  csz_trace_read fills ms[count] and launches[count] (either may
 * be NULL) and optionally resets both.
 */
int csz_kernel_count(void);
const char* csz_kernel_name(int id);
csz_status csz_trace_enable(int on);
csz_status csz_trace_read(double* ms, uint64_t* launches, int reset);

#ifdef __cplusplus
}
#endif
#endif /* CSZP_H */
