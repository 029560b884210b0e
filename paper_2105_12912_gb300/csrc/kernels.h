// Kernel argument blocks and host-side launchers of the cszp CUDA library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace cszp {

struct ConstructArgs {
  const float* x;
  const double* x64;   // double-precision field (x is null then)
  Geom g;
  DevState* st;
  uint32_t radius;
  uint16_t* codes;     // nblk * 4096, block-major
  uint32_t* hist_code; // [1024]
  uint32_t* hist_val;  // [1024]
  uint32_t* hist_len;  // [4096]
  uint32_t* counts;    // [nblk] (outliers << 16) | patches of each block
  uint32_t* masks;     // [nblk][256] patch bit words [128], then outlier bit words [128]
  int32_t* deltas;     // [nblk * 4096] outlier residuals by slot (written at outliers only)
  uint16_t* block_runs;  // [nblk] runs of equal codes in each block
  uint32_t spin_limit;
  int all_runs;        // every block's runs feed the run books (forced run codecs)
  int global;          // global (unchunked) Lorenzo: halo'd tiles (single-field launches)
};

// Value range / error bound of one field of a batch.
struct RangeTask {
  const float* x;
  uint64_t n;
  DevState* st;
  int mode;  // CSZ_EB_ABS / CSZ_EB_REL
  double eb;
};

// Record placement: the exclusive prefix of the blocks' record counts (one CTA of
// the codebook launch), then each encode CTA writes its block's outlier and patch
// records in slot order at that offset.
struct RecordArgs {
  const float* x;
  const uint32_t* counts;  // [nblk] (outliers << 16) | patches
  const uint32_t* masks;   // [nblk][256] patch words, then outlier words
  const int32_t* deltas;   // [nblk * 4096] outlier residuals by slot
  uint64_t* rec_off;       // [nblk] exclusive prefix of record counts
  uint32_t* rec;           // archive record section (u32 key, u32 val pairs)
  uint64_t rec_cap;        // records that fit before the archive capacity ends
};

// One field of a construction launch: its arguments and, when TMA can describe
// the field, the tensor map the kernel fetches tiles with (the struct is 128-byte
// aligned, as CUtensorMap requires).
struct ConstructTask {
  CUtensorMap tmap;
  ConstructArgs a;
  int use_tma;
};

struct BookArgs {
  const uint32_t* hist_code;
  const uint32_t* hist_val;
  const uint32_t* hist_len;
  uint8_t* lens;    // 1024 + 1024 + 4096
  uint64_t* codes;  // 1024 + 1024 + 4096
  DevState* st;
  int place_records;  // a fourth CTA scans the record counts into rec.rec_off
  uint32_t nblk;
  RecordArgs rec;
};

struct FinalizeArgs {
  DevState* st;
  int f64;     // double-precision field
  int global;  // global (unchunked) Lorenzo
  uint8_t* ar;
  uint64_t cap;
  int ndim, eb_mode;
  uint64_t dims[3];
  double eb_user;
  uint32_t radius;
  int select;
  uint64_t nblk, off_bb, off_rec;
  const uint8_t* lens;
};

struct EncodeArgs {
  Geom g;
  DevState* st;
  uint32_t radius;
  int select;
  const uint16_t* codes;
  const uint16_t* block_runs;  // [nblk] runs per block (from construction)
  const uint8_t* lens;
  const uint64_t* bcodes;
  const float* mlp_w;
  int all_runs;     // every block may use run codecs (forced RLE / RLE+Huffman)
  // analysis mode (selector training rows, no archive): per block the 8 features, the
  // 3 log2-size targets, the 3 exact sizes and whether the learned selector decides it
  int analyze;
  float* feat_out;      // [nblk][8]
  float* tgt_out;       // [nblk][3]
  uint32_t* size_out;   // [nblk][3], 0xffffffff where a codec does not apply
  uint8_t* valid_out;   // [nblk]
  uint8_t* ar;
  uint64_t cap;
  uint64_t off_codec, off_bb, off_rec;
  uint64_t* lb;
  uint32_t spin_limit;
  int place_records;  // write each block's records (compression, not analysis)
  RecordArgs rec;
  FinalizeArgs fin;  // used by the last block to finish
};

// decode tables of one canonical book
struct DecTab {
  unsigned long long first[kMaxLen + 1];
  unsigned long long limit[kMaxLen + 1];  // left-justified end of the codes up to each length
  unsigned long long fullmask;            // bit l: the codes up to length l reach 2^64
  uint32_t count[kMaxLen + 1];
  uint32_t off[kMaxLen + 1];
  uint32_t present;
  uint32_t maxlen;
  uint16_t sorted[kNsymLen];
  alignas(16) LutEntry lut[1 << kLutBits];  // lut_entry(symbol, length), 0 = longer than kLutBits
};

struct DecodeArgs {
  Geom g;
  DevState* st;
  const uint8_t* ar;
  uint64_t bytes;
  uint64_t off_codec, off_bb, off_rec, off_pay, off_books;
  uint64_t n_rec, payload;
  uint32_t flags, radius;
  uint32_t n_codec[3];  // blocks per codec, as the header states (checked against the codec bytes)
  float ebx2_f;
  uint64_t* blk_off;   // [nblk+1]
  uint32_t* rec_start; // [nblk+1]
  DecTab* tabs;        // [3]
  uint16_t* codes;     // nblk * 4096
  uint16_t* runv;      // decoded run values of RLE+Huffman blocks (may alias codes)
  uint16_t* runl;      // nblk * 4096 decoded run lengths
  uint32_t* runblk;    // indices of the RLE / RLE+Huffman blocks, ascending (null: not listed)
  uint32_t* slowblk;   // fused decoding: blocks the entropy decoder does not reconstruct
                       // itself (not Huffman, or not of full block extent), ascending
  int fuse;            // full Huffman blocks are reconstructed by the warps that decode them
  float* out;
  double* out64;       // double-precision archives (f64): the output, and the step
  double step_d;
  int f64;
  uint64_t* prep_lb;   // set-up chunks' look-back states (2 per 1024 blocks), zeroed per call
  int global;          // global (unchunked) Lorenzo archive: reconstruction by per-axis passes
  uint64_t* scan_state;  // their look-back states (one per 4096 elements), zeroed per call
  int dead;            // batches: the header failed validation, do nothing
  int check_hdr;       // the arguments come from a host copy of the header (hdr): the
  uint32_t hdr[32];    // set-up compares the device archive's header with it
};

// ---- per-kernel tracing (CUDA events around each launch; defined in api.cu) -------
enum KernelId : int {
  K_RANGE = 0,
  K_PARAMS,
  K_CONSTRUCT,
  K_CODEBOOK,
  K_ENCODE,
  K_DEC_SETUP,
  K_STREAM_DECODE,
  K_RLE_EXPAND,
  K_RECONSTRUCT,
  K_MLP_PREDICT,
  K_MLP_GRAD,
  K_MLP_UPDATE,
  K_DEC_STATUS,
  K_DEC_HEADER,
  K_BATCH,  // the batched persistent compression kernel
  K_COUNT
};
void trace_begin(int id, cudaStream_t s);
void trace_end(int id, cudaStream_t s);
bool trace_suspend();           // stop event tracing (stream capture); returns the old state
bool trace_on();                // event tracing is enabled
void trace_fold();              // fold the recorded events into the totals (after a synchronisation)
void trace_resume(bool on);
void trace_count_batch(bool persistent);  // one replay of a compression batch graph: count its launches
void trace_count_decode_batch();  // the same for a decompression batch graph

// ---- launchers (return cudaGetLastError of the launch) ---------------------------
cudaError_t launch_abs_params(DevState* st, double eb, cudaStream_t s);
cudaError_t launch_range(const float* x, uint64_t n, DevState* st, int mode, double eb, cudaStream_t s);
// double-precision fields: value range (REL) or the bound alone (ABS), and the step
cudaError_t launch_range_d(const double* x, uint64_t n, DevState* st, int mode, double eb, cudaStream_t s);
void prepare_construct_task(ConstructTask& t);  // tensor map when TMA applies
size_t construct_smem_bytes();
int construct_grid(uint32_t ntiles);  // persistent grid: all resident CTAs, at most ntiles
cudaError_t launch_construct(const ConstructTask& one, uint32_t* ticket, cudaStream_t s);
cudaError_t launch_construct_batch(const ConstructTask* d_tasks, const uint32_t* d_tile0, int nfields,
                                   uint32_t ntiles, uint32_t* ticket, uint32_t spin_limit, int grid, int nd,
                                   cudaStream_t s);  // nd: the fields' common dimensionality, 0 if mixed
cudaError_t launch_codebook(const BookArgs& a, cudaStream_t s);
cudaError_t launch_encode(const EncodeArgs& a, cudaStream_t s);
// batches: per-field tables in device memory
uint32_t range_ctas(uint64_t n);  // CTAs the range pass gives a REL field of n elements
cudaError_t launch_range_batch(const RangeTask* d_tasks, const uint32_t* d_cta0, int nfields, uint32_t nctas,
                               cudaStream_t s);
cudaError_t launch_codebook_batch(const BookArgs* d_tasks, int nfields, cudaStream_t s);
cudaError_t launch_encode_batch(const EncodeArgs* d_tasks, const uint32_t* d_tile0, int nfields, uint32_t ntiles,
                                uint32_t* ticket, cudaStream_t s);

// Batched compression as one persistent kernel: every CTA goes through the same
// four phases in order, taking work items from one ticket per phase -- value-range
// CTAs (cta0 prefix), construction tiles, the four book-phase items of each field,
// encoding blocks -- and waits (bounded) only on the hand-over counters of
// DevState that an earlier phase releases, so the whole batch is one launch.
struct PersistArgs {
  const RangeTask* rtasks;
  const uint32_t* cta0;  // nfields + 1
  uint32_t nrange;
  const ConstructTask* ctasks;
  const uint32_t* tile0;  // nfields + 1
  uint32_t ntiles;
  const BookArgs* btasks;
  unsigned char* len_books;  // nfields x persist_len_book_bytes(): working memory of the run-length books
  const EncodeArgs* etasks;
  int nfields;
  uint32_t* tickets;  // [0] construction, [1] encoding, [2] value range, [3] books
  uint32_t spin_limit;
};
size_t persist_len_book_bytes();
int persist_grid_max();  // resident CTAs of the persistent kernel on this GPU (all SMs)
// grid <= persist_grid_max(); nd: the fields' common dimensionality, 0 if mixed
cudaError_t launch_batch_persistent(const PersistArgs& p, int grid, int nd, cudaStream_t s);

cudaError_t launch_decode(const DecodeArgs& a, cudaStream_t s);
// the decompression's csz_status into a device word (asynchronous decompression)
cudaError_t launch_dec_status(const DevState* st, uint32_t* d_status, cudaStream_t s);
// one bounded wait nothing satisfies (0: look-back, 1: mbarrier): ERR_TIMEOUT in st
cudaError_t launch_wait_selftest(int which, uint32_t spin_limit, uint64_t* lb, DevState* st, cudaStream_t s);

// Batched decompression: a device table of per-field decode arguments (headers are
// read and checked on the device) and CTA prefixes per stage.
struct DecodeBatchLaunch {
  DecodeArgs* tasks;
  int nfields;
  const uint32_t* setup0;  // nfields + 1: set-up CTAs (prep, 3 tables, records)
  uint32_t nsetup;
  const uint32_t* chunk0;  // nfields + 1: stream-decode CTAs (kStreamWarpsPerCta / 2 blocks each)
  uint32_t nchunks;
  const uint32_t* tile0;   // nfields + 1: codec blocks
  uint32_t ntiles;
  int nd;                  // the fields' common dimensionality (fused decoding), 0 if mixed
  int warps;               // stream-decode warps per CTA (8, 16 or 32; 0 = 16)
};
constexpr int kStreamWarpsPerCta = 16;
// batched decoding: a decoding CTA of w warps takes kDecChunkRounds * w / 2 codec
// blocks (its decode tables staged once for them), its warps drawing the blocks'
// streams one at a time
constexpr uint32_t kDecChunkRounds = 4;
cudaError_t launch_decode_batch(const DecodeBatchLaunch& L, cudaStream_t s);

}  // namespace cszp
