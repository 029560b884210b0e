// Host side of the cszp C ABI: argument and archive-header validation, workspace
// layout, kernel sequencing on the caller's stream, one synchronisation per call.
#include <cmath>
#include <cstring>

#include "cszp.h"
#include "host.h"
#include "kernels.h"

using namespace cszp;

namespace {

uint32_t g_spin_limit = kSpinLimit;

// Tracing: CUDA events around every launch while enabled, folded into per-kernel
// totals at the call's synchronisation; launch counts are always kept.
struct TraceState {
  bool on = false;
  bool armed[K_COUNT] = {};
  cudaEvent_t ev[K_COUNT][2] = {};
  double ms[K_COUNT] = {};
  unsigned long long launches[K_COUNT] = {};
} g_trace;

void trace_collect() {
  if (!g_trace.on) return;
  for (int k = 0; k < K_COUNT; k++) {
    if (!g_trace.armed[k]) continue;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, g_trace.ev[k][0], g_trace.ev[k][1]) == cudaSuccess) g_trace.ms[k] += ms;
    g_trace.armed[k] = false;
  }
}

struct Header {
  uint32_t magic;
  uint16_t version;
  uint8_t ndim, eb_mode;
  uint64_t dims[3];
  double eb_user, eb_d;
  float eb_f;
  uint32_t radius, lanes, flags;
  uint64_t nblk, n_rec, n_out, n_patch, payload, total;
  uint32_t n_codec[3];
};

// Header checks that need no device data (magic, shape, bound, section sizes).  With
// whole = false only the header itself is present, so section ends are not compared
// with `bytes`.
csz_status parse_header(const uint8_t* h, size_t bytes, Header& H, Geom& g, bool whole = true) {
  if (bytes < (size_t)kHdr) return CSZ_E_CORRUPT;
  memcpy(&H.magic, h, 4);
  memcpy(&H.version, h + 4, 2);
  H.ndim = h[6];
  H.eb_mode = h[7];
  memcpy(H.dims, h + 8, 24);
  memcpy(&H.eb_user, h + 32, 8);
  memcpy(&H.eb_d, h + 40, 8);
  memcpy(&H.eb_f, h + 48, 4);
  memcpy(&H.radius, h + 52, 4);
  memcpy(&H.lanes, h + 56, 4);
  memcpy(&H.flags, h + 60, 4);
  memcpy(&H.nblk, h + 64, 8);
  memcpy(&H.n_rec, h + 72, 8);
  memcpy(&H.n_out, h + 80, 8);
  memcpy(&H.n_patch, h + 88, 8);
  memcpy(&H.payload, h + 96, 8);
  memcpy(&H.total, h + 104, 8);
  memcpy(H.n_codec, h + 116, 12);
  if (H.magic != kMagic || H.version != kVersion) return CSZ_E_CORRUPT;
  if (H.ndim < 1 || H.ndim > 3 || H.eb_mode > 1) return CSZ_E_CORRUPT;
  if (!make_geom(H.ndim, H.dims, g)) return CSZ_E_CORRUPT;
  for (int i = H.ndim; i < 3; i++)
    if (H.dims[i]) return CSZ_E_CORRUPT;
  if (H.radius < 1 || H.radius > 512 || H.lanes != (uint32_t)kLanes || H.flags > 15) return CSZ_E_CORRUPT;
  if (H.nblk != g.nblk || H.n_rec != H.n_out + H.n_patch) return CSZ_E_CORRUPT;
  if (H.flags & kFlagF64) {
    // double fields: the step follows from eb_d; they have no verbatim patches
    const double stp = (2.0 * H.eb_d) * kStepShrink;
    if (!(H.eb_d > 0.0) || !std::isfinite(H.eb_d) || !(stp > 0.0) || !std::isfinite(stp) || H.n_patch)
      return CSZ_E_CORRUPT;
  } else if (!(H.eb_f > 0.0f) || !std::isfinite(2.0f * H.eb_f)) {
    return CSZ_E_CORRUPT;
  }
  if (H.n_rec > 2 * g.nelem || (whole && H.payload > bytes) || (H.payload & 3)) return CSZ_E_CORRUPT;
  const uint64_t off_bb = kHdr + a8(H.nblk);
  const uint64_t off_rec = off_bb + a8(4 * H.nblk);
  const uint64_t off_books = off_rec + 8 * H.n_rec + a8(H.payload);
  const uint64_t total =
      off_books + ((H.flags & 1) ? kNsymCode : 0) + ((H.flags & 2) ? kNsymCode + kNsymLen : 0);
  if (H.total != total || (whole && total > bytes)) return CSZ_E_CORRUPT;
  return CSZ_OK;
}

}  // namespace

namespace cszp {
void trace_begin(int id, cudaStream_t s) {
  g_trace.launches[id]++;
  if (!g_trace.on) return;
  if (!g_trace.ev[id][0]) {
    cudaEventCreate(&g_trace.ev[id][0]);
    cudaEventCreate(&g_trace.ev[id][1]);
  }
  cudaEventRecord(g_trace.ev[id][0], s);
}
void trace_end(int id, cudaStream_t s) {
  if (!g_trace.on) return;
  cudaEventRecord(g_trace.ev[id][1], s);
  g_trace.armed[id] = true;
}
bool trace_suspend() {
  const bool on = g_trace.on;
  g_trace.on = false;
  return on;
}
void trace_resume(bool on) { g_trace.on = on; }
bool trace_on() { return g_trace.on; }
void trace_fold() { trace_collect(); }
void trace_count_batch(bool persistent) {
  if (persistent) {
    g_trace.launches[K_BATCH]++;
    return;
  }
  for (int k : {K_RANGE, K_CONSTRUCT, K_CODEBOOK, K_ENCODE}) g_trace.launches[k]++;
}
void trace_count_decode_batch() {
  for (int k : {K_DEC_HEADER, K_DEC_SETUP, K_STREAM_DECODE, K_RECONSTRUCT}) g_trace.launches[k]++;
}
}  // namespace cszp

extern "C" {

static const char* const kKernelNames[K_COUNT] = {
    "range", "abs_params", "construct", "codebook", "encode", "dec_setup",
    "stream_decode", "rle_expand", "reconstruct", "mlp_predict", "mlp_grad", "mlp_update", "dec_status",
    "dec_header", "batch_persistent"};

int csz_kernel_count(void) { return K_COUNT; }

const char* csz_kernel_name(int id) { return (id >= 0 && id < K_COUNT) ? kKernelNames[id] : ""; }

csz_status csz_trace_enable(int on) {
  g_trace.on = on != 0;
  return CSZ_OK;
}

csz_status csz_trace_read(double* ms, uint64_t* launches, int reset) {
  // launches whose events are complete but not yet folded (an asynchronous
  // decompression has no synchronisation of its own to fold them at)
  for (int k = 0; k < K_COUNT; k++)
    if (g_trace.armed[k] && cudaEventQuery(g_trace.ev[k][1]) == cudaSuccess) {
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, g_trace.ev[k][0], g_trace.ev[k][1]) == cudaSuccess) g_trace.ms[k] += t;
      g_trace.armed[k] = false;
    }
  for (int k = 0; k < K_COUNT; k++) {
    if (ms) ms[k] = g_trace.ms[k];
    if (launches) launches[k] = g_trace.launches[k];
    if (reset) {
      g_trace.ms[k] = 0.0;
      g_trace.launches[k] = 0;
    }
  }
  return CSZ_OK;
}


csz_status csz_wait_selftest(int which, uint32_t spin_limit, void* d_scratch, size_t scratch_bytes,
                              void* stream) {
  if (!d_scratch || scratch_bytes < 512 || which < 0 || which > 2 || spin_limit == 0) return CSZ_E_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevState* st = static_cast<DevState*>(d_scratch);
  uint64_t* lb = reinterpret_cast<uint64_t*>(static_cast<unsigned char*>(d_scratch) + 256);
  if (cudaMemsetAsync(d_scratch, 0, 512, s) != cudaSuccess) return CSZ_E_CUDA;
  if (launch_wait_selftest(which, spin_limit, lb, st, s) != cudaSuccess) return CSZ_E_CUDA;
  DevState hs;
  if (cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CSZ_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
  return fold(hs.status);
}

const char* csz_status_string(int s) {
  switch (s) {
    case CSZ_OK: return "ok";
    case CSZ_E_ARG: return "invalid argument";
    case CSZ_E_NONFINITE: return "non-finite input value";
    case CSZ_E_RANGE: return "value too large for the error bound";
    case CSZ_E_CORRUPT: return "corrupt archive";
    case CSZ_E_CAPACITY: return "buffer too small";
    case CSZ_E_CUDA: return "CUDA runtime error";
    case CSZ_E_TIMEOUT: return "bounded device wait expired";
    default: return "unknown status";
  }
}

size_t csz_max_archive_bytes(int ndim, const uint64_t* dims) {
  Geom g;
  if (!make_geom(ndim, dims, g)) return 0;
  const uint64_t slots = (uint64_t)g.nblk * kSlots;
  return (size_t)(kHdr + a8(g.nblk) + a8(4ull * g.nblk) + 16 * g.nelem + 16 * slots + 64ull * g.nblk +
                  2 * kNsymCode + kNsymLen);
}

size_t csz_workspace_bytes(int ndim, const uint64_t* dims) {
  Geom g;
  if (!make_geom(ndim, dims, g)) return 0;
  return (size_t)layout(g).total;
}

}  // extern "C"

namespace {

// Outputs of the analysis pass (selector training rows) instead of an archive.
struct Analysis {
  float* feat;
  float* target;
  uint32_t* sizes;
  uint8_t* valid;
};

// The compression pipeline on the caller's stream: value range or bound, Lorenzo
// construction, books, per-block selection and encoding (or, with `an`, the analysis
// of every block), then one synchronisation to read the device status and size.
csz_status run_pipeline(const void* d_field, int ndim, const uint64_t* dims, int eb_mode, double eb,
                        const csz_options* opt, void* d_ws, size_t ws_bytes, uint8_t* d_ar, size_t cap,
                        size_t* h_bytes, const Analysis* an, void* stream, uint8_t* h_header = nullptr,
                        bool f64 = false) {
  Geom g;
  if (!d_field || !d_ws) return CSZ_E_ARG;
  if (!an && (!d_ar || !h_bytes)) return CSZ_E_ARG;
  if (!make_geom(ndim, dims, g)) return CSZ_E_ARG;
  const uint32_t radius = (opt && opt->radius) ? opt->radius : 512u;
  const int select = an ? SEL_EXHAUSTIVE : (opt ? (int)opt->select : SEL_EXHAUSTIVE);
  if (radius > 512 || select < 0 || select > SEL_LEARNED) return CSZ_E_ARG;
  if (select == SEL_LEARNED && !(opt && opt->selector_weights)) return CSZ_E_ARG;
  if (opt)
    for (int i = 0; i < 3; i++)
      if (opt->reserved[i]) return CSZ_E_ARG;
  const uint32_t oflags = opt ? opt->flags : 0u;
  if (oflags & ~CSZ_FLAG_GLOBAL_LORENZO) return CSZ_E_ARG;
  const bool global = (oflags & CSZ_FLAG_GLOBAL_LORENZO) != 0;
  if (global && f64) return CSZ_E_ARG;  // the global reconstruction is FP32 only
  if (!(eb > 0.0) || !std::isfinite(eb) || (eb_mode != CSZ_EB_ABS && eb_mode != CSZ_EB_REL)) return CSZ_E_ARG;
  const Layout L = layout(g);
  if (ws_bytes < L.total) return CSZ_E_CAPACITY;
  const uint64_t off_bb = kHdr + a8(g.nblk);
  const uint64_t off_rec = off_bb + a8(4ull * g.nblk);
  if (!an && cap < off_rec) return CSZ_E_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevState* st = at<DevState>(d_ws, L.st);

  if (cudaMemsetAsync(d_ws, 0, L.zero_end, s) != cudaSuccess) return CSZ_E_CUDA;
  const float* x32 = f64 ? nullptr : static_cast<const float*>(d_field);
  const double* x64 = f64 ? static_cast<const double*>(d_field) : nullptr;
  cudaError_t e = f64 ? launch_range_d(x64, g.nelem, st, eb_mode == CSZ_EB_REL ? 1 : 0, eb, s)
                      : (eb_mode == CSZ_EB_REL ? launch_range(x32, g.nelem, st, 1, eb, s)
                                               : launch_abs_params(st, eb, s));
  if (e != cudaSuccess) return CSZ_E_CUDA;

  ConstructTask task;
  memset(&task, 0, sizeof(task));
  ConstructArgs& ca = task.a;
  ca.x = x32;
  ca.x64 = x64;
  ca.g = g;
  ca.st = st;
  ca.radius = radius;
  ca.codes = at<uint16_t>(d_ws, L.codes);
  ca.hist_code = at<uint32_t>(d_ws, L.hist_code);
  ca.hist_val = at<uint32_t>(d_ws, L.hist_val);
  ca.hist_len = at<uint32_t>(d_ws, L.hist_len);
  ca.counts = at<uint32_t>(d_ws, L.counts);
  ca.masks = at<uint32_t>(d_ws, L.masks);
  ca.deltas = at<int32_t>(d_ws, L.deltas);
  ca.block_runs = at<uint16_t>(d_ws, L.runs);
  ca.spin_limit = g_spin_limit;
  ca.all_runs = (select == SEL_RLE || select == SEL_RLE_HUFF) ? 1 : 0;
  ca.global = global ? 1 : 0;
  prepare_construct_task(task);
  if (launch_construct(task, &st->ticket_construct, s) != cudaSuccess) return CSZ_E_CUDA;

  BookArgs ba;
  memset(&ba, 0, sizeof(ba));
  ba.hist_code = ca.hist_code;
  ba.hist_val = ca.hist_val;
  ba.hist_len = ca.hist_len;
  ba.lens = at<uint8_t>(d_ws, L.lens);
  ba.codes = at<uint64_t>(d_ws, L.bcodes);
  ba.st = st;
  RecordArgs ra;
  memset(&ra, 0, sizeof(ra));
  if (!an) {
    // a fourth CTA beside the book builders scans the record counts; the encode
    // CTAs then write each block's records
    ra.x = x32;  // patch values (FP32 fields only: double fields have no patches)
    ra.counts = ca.counts;
    ra.masks = ca.masks;
    ra.deltas = ca.deltas;
    ra.rec_off = at<uint64_t>(d_ws, L.rec_off);
    ra.rec = reinterpret_cast<uint32_t*>(d_ar + off_rec);
    ra.rec_cap = (cap - off_rec) / 8;
    ba.place_records = 1;
    ba.nblk = g.nblk;
    ba.rec = ra;
  }
  if (launch_codebook(ba, s) != cudaSuccess) return CSZ_E_CUDA;

  EncodeArgs ea;
  memset(&ea, 0, sizeof(ea));
  ea.g = g;
  ea.st = st;
  ea.radius = radius;
  ea.select = select;
  ea.codes = ca.codes;
  ea.block_runs = ca.block_runs;
  ea.lens = ba.lens;
  ea.bcodes = ba.codes;
  ea.mlp_w = opt ? opt->selector_weights : nullptr;
  ea.all_runs = ca.all_runs;
  if (an) {
    ea.analyze = 1;
    ea.feat_out = an->feat;
    ea.tgt_out = an->target;
    ea.size_out = an->sizes;
    ea.valid_out = an->valid;
  }
  ea.ar = d_ar;
  ea.cap = cap;
  ea.off_codec = kHdr;
  ea.off_bb = off_bb;
  ea.off_rec = off_rec;
  ea.lb = at<uint64_t>(d_ws, L.lb_e);
  ea.spin_limit = g_spin_limit;
  ea.place_records = an ? 0 : 1;
  ea.rec = ra;
  FinalizeArgs& fa = ea.fin;
  fa.st = st;
  fa.f64 = f64 ? 1 : 0;
  fa.global = global ? 1 : 0;
  fa.ar = d_ar;
  fa.cap = cap;
  fa.ndim = ndim;
  fa.eb_mode = eb_mode;
  for (int i = 0; i < 3; i++) fa.dims[i] = i < ndim ? dims[i] : 0;
  fa.eb_user = eb;
  fa.radius = radius;
  fa.select = select;
  fa.nblk = g.nblk;
  fa.off_bb = off_bb;
  fa.off_rec = off_rec;
  fa.lens = ba.lens;
  if (launch_encode(ea, s) != cudaSuccess) return CSZ_E_CUDA;

  DevState hs;
  if (cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CSZ_E_CUDA;
  if (h_header && cudaMemcpyAsync(h_header, d_ar, kHdr, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CSZ_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
  trace_collect();
  const csz_status r = fold(hs.status);
  if (r != CSZ_OK) return r;
  if (h_bytes) *h_bytes = an ? 0 : (size_t)hs.total;
  return CSZ_OK;
}

// Decode set-up from a parsed header h (read back from the device, or a host copy
// the caller kept: then check_hdr makes the device compare it with the archive) and
// the decode launches.  *st_out: the decompression's device state.
csz_status enqueue_decode(const uint8_t* d_ar, size_t bytes, const uint8_t* h, bool check_hdr, void* d_out,
                          uint64_t out_cap, void* d_ws, size_t ws_bytes, cudaStream_t s, DevState** st_out,
                          bool f64 = false) {
  Header H;
  Geom g;
  csz_status r = parse_header(h, bytes, H, g);
  if (r != CSZ_OK) return r;
  if (((H.flags & kFlagF64) != 0) != f64) return CSZ_E_ARG;  // the output's type is not the field's
  const bool global = (H.flags & kFlagGlobal) != 0;
  if (global && f64) return CSZ_E_CORRUPT;  // no such archive is written
  if (out_cap < g.nelem) return CSZ_E_CAPACITY;
  const Layout L = layout(g);
  if (ws_bytes < L.dec_total) return CSZ_E_CAPACITY;
  DevState* st = at<DevState>(d_ws, L.st);
  // the device state and the set-up's look-back states (adjacent)
  if (cudaMemsetAsync(st, 0, L.hist_code - L.st, s) != cudaSuccess) return CSZ_E_CUDA;
  DecodeArgs da;
  memset(&da, 0, sizeof(da));
  da.g = g;
  da.st = st;
  da.ar = d_ar;
  da.bytes = bytes;
  da.off_codec = kHdr;
  da.off_bb = kHdr + a8(g.nblk);
  da.off_rec = da.off_bb + a8(4ull * g.nblk);
  da.off_pay = da.off_rec + 8 * H.n_rec;
  da.off_books = da.off_pay + a8(H.payload);
  da.n_rec = H.n_rec;
  da.payload = H.payload;
  da.flags = H.flags;
  for (int i = 0; i < 3; i++) da.n_codec[i] = H.n_codec[i];
  da.radius = H.radius;
  da.ebx2_f = 2.0f * H.eb_f;
  da.blk_off = at<uint64_t>(d_ws, L.blk_off);
  da.rec_start = at<uint32_t>(d_ws, L.rec_start);
  da.tabs = at<DecTab>(d_ws, L.tabs);
  da.codes = at<uint16_t>(d_ws, L.codes);
  da.runv = da.codes;  // run values of an RLE+Huffman block wait in its own code slots
  da.runl = at<uint16_t>(d_ws, L.runl);
  da.runblk = at<uint32_t>(d_ws, L.runblk);
  da.slowblk = at<uint32_t>(d_ws, L.slowblk);
  da.prep_lb = at<uint64_t>(d_ws, L.prep_lb);
  da.fuse = global ? 0 : 1;
  da.f64 = f64 ? 1 : 0;
  if (global) {
    // the x pass's look-back states, one per 4096 elements (at most one per codec block)
    da.global = 1;
    da.scan_state = at<uint64_t>(d_ws, L.lb_e);
    if (cudaMemsetAsync(da.scan_state, 0, 8ull * ((g.nelem + 4095) / 4096), s) != cudaSuccess) return CSZ_E_CUDA;
  }
  if (f64) {
    da.out64 = static_cast<double*>(d_out);
    da.step_d = (2.0 * H.eb_d) * kStepShrink;
  } else {
    da.out = static_cast<float*>(d_out);
  }
  da.check_hdr = check_hdr ? 1 : 0;
  memcpy(da.hdr, h, kHdr);
  if (launch_decode(da, s) != cudaSuccess) return CSZ_E_CUDA;
  *st_out = st;
  return CSZ_OK;
}

}  // namespace

extern "C" {

csz_status csz_compress(const float* d_field, int ndim, const uint64_t* dims, int eb_mode, double eb,
                        const csz_options* opt, void* d_ws, size_t ws_bytes, uint8_t* d_ar, size_t cap,
                        size_t* h_bytes, void* stream) {
  return run_pipeline(d_field, ndim, dims, eb_mode, eb, opt, d_ws, ws_bytes, d_ar, cap, h_bytes, nullptr, stream);
}

csz_status csz_selector_rows(const float* d_field, int ndim, const uint64_t* dims, int eb_mode, double eb,
                             uint32_t radius, void* d_ws, size_t ws_bytes, float* d_feat, float* d_target,
                             uint32_t* d_sizes, uint8_t* d_valid, void* stream) {
  if (!d_feat || !d_target || !d_sizes || !d_valid) return CSZ_E_ARG;
  csz_options opt;
  memset(&opt, 0, sizeof(opt));
  opt.radius = radius;
  opt.select = CSZ_SEL_EXHAUSTIVE;
  const Analysis an{d_feat, d_target, d_sizes, d_valid};
  return run_pipeline(d_field, ndim, dims, eb_mode, eb, &opt, d_ws, ws_bytes, nullptr, 0, nullptr, &an, stream);
}

csz_status csz_archive_info(const uint8_t* h, size_t bytes, int* ndim, uint64_t* dims, double* eb_abs,
                            uint64_t* total_bytes) {
  if (!h) return CSZ_E_ARG;
  Header H;
  Geom g;
  csz_status r = parse_header(h, bytes, H, g, false);
  if (r != CSZ_OK) return r;
  if (ndim) *ndim = H.ndim;
  if (dims)
    for (int i = 0; i < 3; i++) dims[i] = H.dims[i];
  if (eb_abs) *eb_abs = H.eb_d;
  if (total_bytes) *total_bytes = H.total;
  return CSZ_OK;
}

csz_status csz_decompress(const uint8_t* d_ar, size_t bytes, float* d_out, uint64_t out_cap, void* d_ws,
                          size_t ws_bytes, void* stream) {
  if (!d_ar || !d_out || !d_ws) return CSZ_E_ARG;
  if (bytes < (size_t)kHdr) return CSZ_E_CORRUPT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t h[kHdr];
  if (cudaMemcpyAsync(h, d_ar, kHdr, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CSZ_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
  DevState* st = nullptr;
  const csz_status r = enqueue_decode(d_ar, bytes, h, false, d_out, out_cap, d_ws, ws_bytes, s, &st);
  if (r != CSZ_OK) return r;
  DevState hs;
  if (cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CSZ_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
  trace_collect();
  return fold(hs.status);
}

csz_status csz_compress_f64(const double* d_field, int ndim, const uint64_t* dims, int eb_mode, double eb,
                            const csz_options* opt, void* d_ws, size_t ws_bytes, uint8_t* d_ar, size_t cap,
                            size_t* h_bytes, void* stream) {
  return run_pipeline(d_field, ndim, dims, eb_mode, eb, opt, d_ws, ws_bytes, d_ar, cap, h_bytes, nullptr, stream,
                      nullptr, true);
}

csz_status csz_decompress_f64(const uint8_t* d_ar, size_t bytes, double* d_out, uint64_t out_cap, void* d_ws,
                              size_t ws_bytes, void* stream) {
  if (!d_ar || !d_out || !d_ws) return CSZ_E_ARG;
  if (bytes < (size_t)kHdr) return CSZ_E_CORRUPT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t h[kHdr];
  if (cudaMemcpyAsync(h, d_ar, kHdr, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CSZ_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
  DevState* st = nullptr;
  const csz_status r = enqueue_decode(d_ar, bytes, h, false, d_out, out_cap, d_ws, ws_bytes, s, &st, true);
  if (r != CSZ_OK) return r;
  DevState hs;
  if (cudaMemcpyAsync(&hs, st, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CSZ_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
  trace_collect();
  return fold(hs.status);
}

int csz_archive_elem_bytes(const uint8_t* h, size_t bytes) {
  if (!h) return 0;
  Header H;
  Geom g;
  if (parse_header(h, bytes, H, g, false) != CSZ_OK) return 0;
  return (H.flags & kFlagF64) ? 8 : 4;
}

csz_status csz_decompress_async(const uint8_t* d_ar, size_t bytes, const uint8_t* h_header, float* d_out,
                                uint64_t out_cap, void* d_ws, size_t ws_bytes, uint32_t* d_status,
                                void* stream) {
  if (!d_ar || !h_header || !d_out || !d_ws || !d_status) return CSZ_E_ARG;
  if (bytes < (size_t)kHdr) return CSZ_E_CORRUPT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DevState* st = nullptr;
  const csz_status r = enqueue_decode(d_ar, bytes, h_header, true, d_out, out_cap, d_ws, ws_bytes, s, &st);
  if (r != CSZ_OK) return r;
  if (launch_dec_status(st, d_status, s) != cudaSuccess) return CSZ_E_CUDA;
  return CSZ_OK;
}

csz_status csz_compress_with_header(const float* d_field, int ndim, const uint64_t* dims, int eb_mode, double eb,
                                    const csz_options* opt, void* d_ws, size_t ws_bytes, uint8_t* d_ar, size_t cap,
                                    size_t* h_bytes, uint8_t* h_header, void* stream) {
  if (!h_header) return CSZ_E_ARG;
  return run_pipeline(d_field, ndim, dims, eb_mode, eb, opt, d_ws, ws_bytes, d_ar, cap, h_bytes, nullptr, stream,
                      h_header);
}

}  // extern "C"
