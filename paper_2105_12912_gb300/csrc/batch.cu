// Batched compression: many fields of any shape and dimensionality go through one
// persistent launch (batch_persistent_kernel: range, construction, books and record
// offsets, encoding as phases of every CTA, handed over per field) or, as the staged
// plan, one launch per stage, each kernel walking a per-field table in device memory
// (the construction and encoding kernels take codec blocks of all fields from one
// ticket).  The plan is captured once into a CUDA graph and replayed; results stay on
// the device until the caller reads them.  An autotuner picks the plan and its
// persistent grid (resident CTAs per SM) by timing the candidates on the batch.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "cszp.h"
#include "host.h"
#include "kernels.h"

using namespace cszp;

struct csz_batch {
  int nfields = 0;
  std::vector<Geom> geom;
  // device tables and regions (inside the caller's workspace)
  unsigned char* zero_base = nullptr;
  uint64_t zero_bytes = 0;
  uint32_t* tickets = nullptr;  // [0] construction, [1] encoding
  DevState* states = nullptr;   // nfields, kStateStride apart
  ConstructTask* ctasks = nullptr;
  uint32_t* tile0 = nullptr;  // nfields + 1
  RangeTask* rtasks = nullptr;
  uint32_t* cta0 = nullptr;  // nfields + 1
  BookArgs* btasks = nullptr;
  EncodeArgs* etasks = nullptr;
  uint32_t ntiles = 0, nrange = 0;
  int construct_grid = 0;  // 0 = default (all resident CTAs)
  int common_nd = 0;       // the fields' dimensionality when they all share it, else 0
  int tuned_grid = 0;
  double tuned_ms[4] = {0, 0, 0, 0};
  // the one-launch plan: every stage in batch_persistent_kernel
  PersistArgs pargs{};
  int persistent = 0;      // the graph holds the persistent kernel (else the staged launches)
  int persist_grid = 0;
  double persist_ms[4] = {0, 0, 0, 0};
  cudaGraphExec_t exec = nullptr;
};

namespace {

// last CUDA failure inside csz_batch_create (step name and runtime error)
const char* g_fail_step = "";
cudaError_t g_fail_err = cudaSuccess;

bool failed(cudaError_t e, const char* step) {
  if (e == cudaSuccess) return false;
  g_fail_step = step;
  g_fail_err = e;
  return true;
}

constexpr uint64_t kStateStride = 256;
static_assert(sizeof(DevState) <= kStateStride, "DevState stride");
constexpr uint64_t kHistBytes = (kNsymCode + kNsymCode + kNsymLen) * 4;

struct FieldLayout {  // offsets from the start of the per-field part
  uint64_t lens, bcodes, codes, counts, masks, deltas, rec_off, runs, total;
};

FieldLayout field_layout(const Geom& g) {
  FieldLayout L;
  uint64_t o = 0;
  L.lens = o;
  o += a256(2 * kNsymCode + kNsymLen);
  L.bcodes = o;
  o += a256(8ull * (2 * kNsymCode + kNsymLen));
  L.codes = o;
  o += a256(2ull * kSlots * g.nblk);
  L.counts = o;
  o += a256(4ull * g.nblk);
  L.masks = o;
  o += a256(1024ull * g.nblk);
  L.deltas = o;
  o += a256(4ull * kSlots * g.nblk);
  L.rec_off = o;
  o += a256(8ull * g.nblk);
  L.runs = o;
  o += a256(2ull * g.nblk);
  L.total = o;
  return L;
}

// Whole-batch layout: zeroed part (tickets, states, histograms, look-back states),
// tables, then the fields' own regions.
struct BatchLayout {
  uint64_t tickets, states, hists, lb, zero_end;
  uint64_t ctasks, tile0, rtasks, cta0, btasks, etasks, len_books, fields_begin;
  std::vector<uint64_t> lb_at, field_at;
  uint64_t total;
};

BatchLayout batch_layout(const std::vector<Geom>& gs) {
  const uint64_t F = gs.size();
  BatchLayout B;
  uint64_t o = 0;
  B.tickets = o;
  o += 256;
  B.states = o;
  o += kStateStride * F;
  B.hists = o;
  o += a256(kHistBytes) * F;
  B.lb = o;
  B.lb_at.resize(F);
  for (uint64_t f = 0; f < F; f++) {
    B.lb_at[f] = o;
    o += a256(8ull * gs[f].nblk);
  }
  B.zero_end = o;
  B.ctasks = o;
  o += a256(sizeof(ConstructTask) * F);
  B.tile0 = o;
  o += a256(4 * (F + 1));
  B.rtasks = o;
  o += a256(sizeof(RangeTask) * F);
  B.cta0 = o;
  o += a256(4 * (F + 1));
  B.btasks = o;
  o += a256(sizeof(BookArgs) * F);
  B.etasks = o;
  o += a256(sizeof(EncodeArgs) * F);
  B.len_books = o;  // the persistent kernel's run-length book working memory
  o += a256(persist_len_book_bytes() * F);
  B.fields_begin = o;
  B.field_at.resize(F);
  for (uint64_t f = 0; f < F; f++) {
    B.field_at[f] = o;
    o += field_layout(gs[f]).total;
  }
  B.total = o;
  return B;
}

csz_status check_fields(int nfields, const csz_field* fields, std::vector<Geom>& gs) {
  if (nfields <= 0 || !fields) return CSZ_E_ARG;
  gs.resize(nfields);
  uint64_t tiles = 0;
  for (int f = 0; f < nfields; f++) {
    const csz_field& d = fields[f];
    if (!make_geom(d.ndim, d.dims, gs[f])) return CSZ_E_ARG;
    if (!(d.eb > 0.0) || !std::isfinite(d.eb) || (d.eb_mode != CSZ_EB_ABS && d.eb_mode != CSZ_EB_REL))
      return CSZ_E_ARG;
    tiles += gs[f].nblk;
  }
  if (tiles >= (1ull << 32)) return CSZ_E_ARG;
  return CSZ_OK;
}

template <typename T>
cudaError_t upload(T* dst, const std::vector<T>& src, cudaStream_t s) {
  return cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s);
}

// The batch's launch sequence on `s` (also what the graph captures).
cudaError_t enqueue(const csz_batch* b, int construct_grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->zero_base, 0, b->zero_bytes, s);
  if (e != cudaSuccess) return e;
  if ((e = launch_range_batch(b->rtasks, b->cta0, b->nfields, b->nrange, s)) != cudaSuccess) return e;
  if ((e = launch_construct_batch(b->ctasks, b->tile0, b->nfields, b->ntiles, &b->tickets[0], kSpinLimit,
                                  construct_grid, b->common_nd, s)) != cudaSuccess)
    return e;
  if ((e = launch_codebook_batch(b->btasks, b->nfields, s)) != cudaSuccess) return e;
  return launch_encode_batch(b->etasks, b->tile0, b->nfields, b->ntiles, &b->tickets[1], s);
}

// The same batch as one launch of the persistent kernel.
cudaError_t enqueue_persistent(const csz_batch* b, int grid, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->zero_base, 0, b->zero_bytes, s);
  if (e != cudaSuccess) return e;
  return launch_batch_persistent(b->pargs, grid, b->common_nd, s);
}

cudaError_t enqueue_plan(const csz_batch* b, cudaStream_t s) {
  return b->persistent ? enqueue_persistent(b, b->persist_grid, s) : enqueue(b, b->construct_grid, s);
}

}  // namespace

extern "C" {

size_t csz_batch_workspace_bytes(int nfields, const csz_field* fields) {
  std::vector<Geom> gs;
  if (check_fields(nfields, fields, gs) != CSZ_OK) return 0;
  return (size_t)batch_layout(gs).total;
}

csz_status csz_batch_create(int nfields, const csz_field* fields, const csz_options* opt, void* d_ws,
                            size_t ws_bytes, int autotune, void* stream, csz_batch** out) {
  if (!out || !d_ws) return CSZ_E_ARG;
  *out = nullptr;
  std::vector<Geom> gs;
  csz_status r = check_fields(nfields, fields, gs);
  if (r != CSZ_OK) return r;
  const uint32_t radius = (opt && opt->radius) ? opt->radius : 512u;
  const int select = opt ? (int)opt->select : SEL_EXHAUSTIVE;
  if (radius > 512 || select < 0 || select > SEL_LEARNED) return CSZ_E_ARG;
  if (select == SEL_LEARNED && !(opt && opt->selector_weights)) return CSZ_E_ARG;
  if (opt) {
    for (int i = 0; i < 3; i++)
      if (opt->reserved[i]) return CSZ_E_ARG;
    if (opt->flags) return CSZ_E_ARG;  // batches compress with chunked Lorenzo only
  }
  const BatchLayout B = batch_layout(gs);
  if (ws_bytes < B.total) return CSZ_E_CAPACITY;
  for (int f = 0; f < nfields; f++) {
    const uint64_t off_rec = kHdr + a8(gs[f].nblk) + a8(4ull * gs[f].nblk);
    if (!fields[f].d_field || !fields[f].d_archive) return CSZ_E_ARG;
    if (fields[f].archive_cap < off_rec) return CSZ_E_CAPACITY;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(d_ws);

  csz_batch* b = new (std::nothrow) csz_batch();
  if (!b) return CSZ_E_ARG;
  b->nfields = nfields;
  b->geom = gs;
  b->zero_base = ws;
  b->zero_bytes = B.zero_end;
  b->tickets = at<uint32_t>(ws, B.tickets);
  b->states = at<DevState>(ws, B.states);
  b->ctasks = at<ConstructTask>(ws, B.ctasks);
  b->tile0 = at<uint32_t>(ws, B.tile0);
  b->rtasks = at<RangeTask>(ws, B.rtasks);
  b->cta0 = at<uint32_t>(ws, B.cta0);
  b->btasks = at<BookArgs>(ws, B.btasks);
  b->etasks = at<EncodeArgs>(ws, B.etasks);

  std::vector<ConstructTask> ct(nfields);
  std::vector<RangeTask> rt(nfields);
  std::vector<BookArgs> bt(nfields);
  std::vector<EncodeArgs> et(nfields);
  std::vector<uint32_t> tile0(nfields + 1), cta0(nfields + 1);
  uint32_t tiles = 0, ctas = 0;
  for (int f = 0; f < nfields; f++) {
    const csz_field& d = fields[f];
    const Geom& g = gs[f];
    const FieldLayout FL = field_layout(g);
    unsigned char* fw = ws + B.field_at[f];
    DevState* st = reinterpret_cast<DevState*>(ws + B.states + kStateStride * f);
    uint32_t* hists = reinterpret_cast<uint32_t*>(ws + B.hists + a256(kHistBytes) * f);
    const uint64_t off_bb = kHdr + a8(g.nblk);
    const uint64_t off_rec = off_bb + a8(4ull * g.nblk);
    tile0[f] = tiles;
    tiles += g.nblk;
    cta0[f] = ctas;
    ctas += d.eb_mode == CSZ_EB_REL ? range_ctas(g.nelem) : 1u;

    RangeTask& R = rt[f];
    R.x = d.d_field;
    R.n = g.nelem;
    R.st = st;
    R.mode = d.eb_mode;
    R.eb = d.eb;

    memset(&ct[f], 0, sizeof(ConstructTask));
    ConstructArgs& ca = ct[f].a;
    ca.x = d.d_field;
    ca.g = g;
    ca.st = st;
    ca.radius = radius;
    ca.codes = at<uint16_t>(fw, FL.codes);
    ca.hist_code = hists;
    ca.hist_val = hists + kNsymCode;
    ca.hist_len = hists + 2 * kNsymCode;
    ca.counts = at<uint32_t>(fw, FL.counts);
    ca.masks = at<uint32_t>(fw, FL.masks);
    ca.deltas = at<int32_t>(fw, FL.deltas);
    ca.block_runs = at<uint16_t>(fw, FL.runs);
    ca.spin_limit = kSpinLimit;
    ca.all_runs = (select == SEL_RLE || select == SEL_RLE_HUFF) ? 1 : 0;
    prepare_construct_task(ct[f]);

    RecordArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.x = d.d_field;
    ra.counts = ca.counts;
    ra.masks = ca.masks;
    ra.deltas = ca.deltas;
    ra.rec_off = at<uint64_t>(fw, FL.rec_off);
    ra.rec = reinterpret_cast<uint32_t*>(d.d_archive + off_rec);
    ra.rec_cap = (d.archive_cap - off_rec) / 8;

    BookArgs& ba = bt[f];
    memset(&ba, 0, sizeof(ba));
    ba.hist_code = ca.hist_code;
    ba.hist_val = ca.hist_val;
    ba.hist_len = ca.hist_len;
    ba.lens = at<uint8_t>(fw, FL.lens);
    ba.codes = at<uint64_t>(fw, FL.bcodes);
    ba.st = st;
    ba.place_records = 1;
    ba.nblk = g.nblk;
    ba.rec = ra;

    EncodeArgs& ea = et[f];
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
    ea.ar = d.d_archive;
    ea.cap = d.archive_cap;
    ea.off_codec = kHdr;
    ea.off_bb = off_bb;
    ea.off_rec = off_rec;
    ea.lb = at<uint64_t>(ws, B.lb_at[f]);
    ea.spin_limit = kSpinLimit;
    ea.place_records = 1;
    ea.rec = ra;
    FinalizeArgs& fa = ea.fin;
    fa.st = st;
    fa.ar = d.d_archive;
    fa.cap = d.archive_cap;
    fa.ndim = d.ndim;
    fa.eb_mode = d.eb_mode;
    for (int i = 0; i < 3; i++) fa.dims[i] = i < d.ndim ? d.dims[i] : 0;
    fa.eb_user = d.eb;
    fa.radius = radius;
    fa.select = select;
    fa.nblk = g.nblk;
    fa.off_bb = off_bb;
    fa.off_rec = off_rec;
    fa.lens = ba.lens;
  }
  tile0[nfields] = tiles;
  cta0[nfields] = ctas;
  b->ntiles = tiles;
  b->common_nd = fields[0].ndim;
  for (int f = 1; f < nfields; f++)
    if (fields[f].ndim != b->common_nd) b->common_nd = 0;
  b->nrange = ctas;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload(b->ctasks, ct, s);
  if (e == cudaSuccess) e = upload(b->tile0, tile0, s);
  if (e == cudaSuccess) e = upload(b->rtasks, rt, s);
  if (e == cudaSuccess) e = upload(b->cta0, cta0, s);
  if (e == cudaSuccess) e = upload(b->btasks, bt, s);
  if (e == cudaSuccess) e = upload(b->etasks, et, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (failed(e, "table upload")) {
    delete b;
    return CSZ_E_CUDA;
  }

  // the persistent kernel's tables (its argument block, passed by value)
  PersistArgs& P = b->pargs;
  P.rtasks = b->rtasks;
  P.cta0 = b->cta0;
  P.nrange = b->nrange;
  P.ctasks = b->ctasks;
  P.tile0 = b->tile0;
  P.ntiles = tiles;
  P.btasks = b->btasks;
  P.len_books = ws + B.len_books;
  P.etasks = b->etasks;
  P.nfields = nfields;
  P.tickets = b->tickets;
  P.spin_limit = kSpinLimit;

  // The plan: one persistent launch (default) or the staged launches, and its grid.
  // With CSZ_BATCH_AUTOTUNE every allowed candidate is timed on the batch (resident
  // CTAs per SM 1..4 for either plan) and the fastest is kept; the archives do not
  // depend on the choice.
  const bool allow_staged = (autotune & CSZ_BATCH_STAGED) || !(autotune & CSZ_BATCH_PERSISTENT);
  const int pmax = persist_grid_max();
  const bool allow_persist = pmax > 0 && ((autotune & CSZ_BATCH_PERSISTENT) || !(autotune & CSZ_BATCH_STAGED));
  const int full = construct_grid(tiles);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  b->tuned_grid = full;
  b->construct_grid = full;
  b->persist_grid = pmax;
  b->persistent = allow_persist ? 1 : 0;
  if ((autotune & CSZ_BATCH_AUTOTUNE) && sms > 0) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 0.0f;
    auto time_it = [&](bool persist, int grid, float& ms) {
      for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
        cudaEventRecord(e0, s);
        e = persist ? enqueue_persistent(b, grid, s) : enqueue(b, grid, s);
        cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
      }
    };
    for (int k = 1; k <= 4 && allow_staged && e == cudaSuccess; k++) {
      int grid = sms * k;
      if (grid > full) grid = full;
      float ms = 0.0f;
      time_it(false, grid, ms);
      if (e != cudaSuccess) break;
      b->tuned_ms[k - 1] = ms;
      if (best == 0.0f || ms < best) {
        best = ms;
        b->tuned_grid = grid;
        b->construct_grid = grid;
        b->persistent = 0;
      }
      if (grid == full) break;
    }
    for (int k = 1; k <= 4 && allow_persist && e == cudaSuccess; k++) {
      int grid = sms * k;
      if (grid > pmax) grid = pmax;
      float ms = 0.0f;
      time_it(true, grid, ms);
      if (e != cudaSuccess) break;
      b->persist_ms[k - 1] = ms;
      if (best == 0.0f || ms < best) {
        best = ms;
        b->persist_grid = grid;
        b->persistent = 1;
      }
      if (grid == pmax) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (failed(e, "autotune run")) {
      delete b;
      return CSZ_E_CUDA;
    }
  }

  // capture the launch sequence once, on a private stream (the caller's may be the
  // legacy default stream, which cannot be captured); replays go to any stream
  const bool tracing = trace_suspend();
  cudaGraph_t graph = nullptr;
  cudaStream_t cap = nullptr;
  e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  const char* step = "capture stream";
  if (e == cudaSuccess) {
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    step = "begin capture";
  }
  if (e == cudaSuccess) {
    const cudaError_t e2 = enqueue_plan(b, cap);
    e = cudaStreamEndCapture(cap, &graph);
    step = "end capture";
    if (e == cudaSuccess && e2 != cudaSuccess) {
      e = e2;
      step = "captured launches";
    }
  }
  if (e == cudaSuccess) {
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    step = "instantiate";
  }
  if (graph) cudaGraphDestroy(graph);
  if (cap) cudaStreamDestroy(cap);
  trace_resume(tracing);
  if (failed(e, step)) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    delete b;
    return CSZ_E_CUDA;
  }
  *out = b;
  return CSZ_OK;
}

csz_status csz_batch_compress(csz_batch* b, void* stream) {
  if (!b || !b->exec) return CSZ_E_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (trace_on()) {
    // with tracing on, the graph's launches run one by one so that each gets its
    // events, and the call waits for them (tracing is a diagnostic mode)
    if (enqueue_plan(b, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
    trace_fold();
    return CSZ_OK;
  }
  if (cudaGraphLaunch(b->exec, s) != cudaSuccess) return CSZ_E_CUDA;
  trace_count_batch(b->persistent != 0);
  return CSZ_OK;
}

csz_status csz_batch_results(csz_batch* b, uint64_t* h_bytes, int* h_status, void* stream) {
  if (!b) return CSZ_E_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<unsigned char> buf(kStateStride * b->nfields);
  if (cudaMemcpyAsync(buf.data(), b->states, buf.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CSZ_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
  csz_status worst = CSZ_OK;
  for (int f = 0; f < b->nfields; f++) {
    DevState st;
    memcpy(&st, buf.data() + kStateStride * f, sizeof(st));
    const csz_status r = fold(st.status);
    if (h_status) h_status[f] = (int)r;
    if (h_bytes) h_bytes[f] = r == CSZ_OK ? st.total : 0;
    if (r != CSZ_OK && worst == CSZ_OK) worst = r;
  }
  return worst;
}

csz_status csz_batch_info(const csz_batch* b, int* construct_grid, double* tuned_ms) {
  if (!b) return CSZ_E_ARG;
  if (construct_grid) *construct_grid = b->construct_grid;
  if (tuned_ms)
    for (int i = 0; i < 4; i++) tuned_ms[i] = b->tuned_ms[i];
  return CSZ_OK;
}

csz_status csz_batch_plan(const csz_batch* b, int* persistent, int* grid, double* persist_ms) {
  if (!b) return CSZ_E_ARG;
  if (persistent) *persistent = b->persistent;
  if (grid) *grid = b->persistent ? b->persist_grid : b->construct_grid;
  if (persist_ms)
    for (int i = 0; i < 4; i++) persist_ms[i] = b->persist_ms[i];
  return CSZ_OK;
}

// ---------------------------------------------------------------------------------
// batched decompression
// ---------------------------------------------------------------------------------
}  // extern "C"

// Stream-decode CTA shapes the batch's tuner chooses among (warps per CTA; a CTA
// decodes kDecChunkRounds * warps / 2 codec blocks).  None changes the output.
constexpr int kDecShapes[3] = {8, 16, 32};

struct csz_batch_dec {
  int nfields = 0;
  unsigned char* zero_base = nullptr;
  uint64_t zero_bytes = 0;
  DevState* states = nullptr;
  DecodeBatchLaunch launch{};
  DecodeArgs* d_tasks = nullptr;
  cudaGraphExec_t exec = nullptr;
  const uint32_t* chunk0[3] = {nullptr, nullptr, nullptr};  // per shape: stream-decode CTA prefix
  uint32_t nchunks[3] = {0, 0, 0};
};

namespace {

struct DecFieldLayout {
  uint64_t blk_off, rec_start, tabs, codes, runl, total;
};

DecFieldLayout dec_field_layout(const Geom& g) {
  DecFieldLayout L;
  uint64_t o = 0;
  L.blk_off = o;
  o += a256(8ull * (g.nblk + 1));
  L.rec_start = o;
  o += a256(4ull * (g.nblk + 1));
  L.tabs = o;
  o += a256(3 * sizeof(DecTab));
  L.codes = o;
  o += a256(2ull * kSlots * g.nblk);
  L.runl = o;
  o += a256(2ull * kSlots * g.nblk);
  L.total = o;
  return L;
}

struct DecBatchLayout {
  uint64_t states, prep, zero_end, tasks, setup0, chunk0, tile0;
  std::vector<uint64_t> field_at, prep_at;
  uint64_t total;
};

// set-up chunks of a field (one CTA per 1024 codec blocks)
inline uint32_t prep_chunks(const Geom& g) { return (g.nblk + 1023) / 1024; }

DecBatchLayout dec_batch_layout(const std::vector<Geom>& gs) {
  const uint64_t F = gs.size();
  DecBatchLayout B;
  uint64_t o = 0;
  B.states = o;
  o += kStateStride * F;
  // the set-up chunks' look-back states (two per chunk), zeroed with the states
  B.prep = o;
  B.prep_at.resize(F);
  for (uint64_t f = 0; f < F; f++) {
    B.prep_at[f] = o;
    o += 16ull * prep_chunks(gs[f]);
  }
  B.zero_end = o;
  o = a256(o);
  B.tasks = o;
  o += a256(sizeof(DecodeArgs) * F);
  B.setup0 = o;
  o += a256(4 * (F + 1));
  B.chunk0 = o;
  o += 3 * a256(4 * (F + 1));  // one prefix per CTA shape
  B.tile0 = o;
  o += a256(4 * (F + 1));
  B.field_at.resize(F);
  for (uint64_t f = 0; f < F; f++) {
    B.field_at[f] = o;
    o += dec_field_layout(gs[f]).total;
  }
  B.total = o;
  return B;
}

csz_status check_dfields(int n, const csz_dfield* fields, std::vector<Geom>& gs) {
  if (n <= 0 || !fields) return CSZ_E_ARG;
  gs.resize(n);
  uint64_t tiles = 0;
  for (int f = 0; f < n; f++) {
    if (!make_geom(fields[f].ndim, fields[f].dims, gs[f])) return CSZ_E_ARG;
    tiles += gs[f].nblk;
  }
  if (tiles >= (1ull << 32)) return CSZ_E_ARG;
  return CSZ_OK;
}

cudaError_t dec_capture(csz_batch_dec* b);

cudaError_t dec_enqueue(const csz_batch_dec* b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->zero_base, 0, b->zero_bytes, s);
  if (e != cudaSuccess) return e;
  // the header pass rewrites the tables' header-derived fields every run
  return launch_decode_batch(b->launch, s);
}

}  // namespace

extern "C" {

size_t csz_batch_dec_workspace_bytes(int nfields, const csz_dfield* fields) {
  std::vector<Geom> gs;
  if (check_dfields(nfields, fields, gs) != CSZ_OK) return 0;
  return (size_t)dec_batch_layout(gs).total;
}

csz_status csz_batch_dec_create(int nfields, const csz_dfield* fields, void* d_ws, size_t ws_bytes, void* stream,
                                csz_batch_dec** out) {
  if (!out || !d_ws) return CSZ_E_ARG;
  *out = nullptr;
  std::vector<Geom> gs;
  csz_status r = check_dfields(nfields, fields, gs);
  if (r != CSZ_OK) return r;
  for (int f = 0; f < nfields; f++) {
    if (!fields[f].d_archive || !fields[f].d_out) return CSZ_E_ARG;
    if (fields[f].out_cap_elems < gs[f].nelem) return CSZ_E_CAPACITY;
  }
  const DecBatchLayout B = dec_batch_layout(gs);
  if (ws_bytes < B.total) return CSZ_E_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(d_ws);
  csz_batch_dec* b = new (std::nothrow) csz_batch_dec();
  if (!b) return CSZ_E_ARG;
  b->nfields = nfields;
  b->zero_base = ws;
  b->zero_bytes = B.zero_end;
  b->states = at<DevState>(ws, B.states);
  b->d_tasks = at<DecodeArgs>(ws, B.tasks);
  std::vector<DecodeArgs> tasks(nfields);
  std::vector<uint32_t> setup0(nfields + 1), tile0(nfields + 1);
  std::vector<uint32_t> chunk0s[3];
  for (auto& c : chunk0s) c.resize(nfields + 1);
  uint32_t nsetup = 0, ntiles = 0, nchunks_v[3] = {0, 0, 0};
  // fields that share their dimensionality decode with the fused reconstruction
  int common_nd = gs[0].ndim;
  for (int f = 1; f < nfields; f++)
    if (gs[f].ndim != common_nd) common_nd = 0;
  for (int f = 0; f < nfields; f++) {
    const Geom& g = gs[f];
    const DecFieldLayout FL = dec_field_layout(g);
    unsigned char* fw = ws + B.field_at[f];
    DecodeArgs& a = tasks[f];
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.st = reinterpret_cast<DevState*>(ws + B.states + kStateStride * f);
    a.ar = fields[f].d_archive;
    a.bytes = fields[f].archive_bytes;
    a.blk_off = at<uint64_t>(fw, FL.blk_off);
    a.rec_start = at<uint32_t>(fw, FL.rec_start);
    a.tabs = at<DecTab>(fw, FL.tabs);
    a.codes = at<uint16_t>(fw, FL.codes);
    a.runv = a.codes;
    a.runl = at<uint16_t>(fw, FL.runl);
    a.out = fields[f].d_out;
    a.fuse = common_nd != 0 ? 1 : 0;
    a.prep_lb = at<uint64_t>(ws, B.prep_at[f]);
    a.dead = 1;  // until the header pass accepts the field
    setup0[f] = nsetup;
    uint64_t rec_ctas = (g.nelem + 32767) / 32768;
    if (rec_ctas < 1) rec_ctas = 1;
    if (rec_ctas > 256) rec_ctas = 256;
    nsetup += prep_chunks(g) + 3 + (uint32_t)rec_ctas;
    for (int v = 0; v < 3; v++) {
      const uint32_t per = kDecChunkRounds * ((uint32_t)kDecShapes[v] / 2);
      chunk0s[v][f] = nchunks_v[v];
      nchunks_v[v] += (g.nblk + per - 1) / per;
    }
    tile0[f] = ntiles;
    ntiles += g.nblk;
  }
  setup0[nfields] = nsetup;
  for (int v = 0; v < 3; v++) chunk0s[v][nfields] = nchunks_v[v];
  tile0[nfields] = ntiles;
  cudaError_t e = upload(b->d_tasks, tasks, s);
  if (e == cudaSuccess) e = upload(at<uint32_t>(ws, B.setup0), setup0, s);
  for (int v = 0; v < 3; v++) {
    b->chunk0[v] = at<uint32_t>(ws, B.chunk0 + (uint64_t)v * a256(4 * (nfields + 1)));
    b->nchunks[v] = nchunks_v[v];
    if (e == cudaSuccess) e = upload(const_cast<uint32_t*>(b->chunk0[v]), chunk0s[v], s);
  }
  if (e == cudaSuccess) e = upload(at<uint32_t>(ws, B.tile0), tile0, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (failed(e, "decompression table upload")) {
    delete b;
    return CSZ_E_CUDA;
  }
  b->launch = DecodeBatchLaunch{b->d_tasks, nfields, at<uint32_t>(ws, B.setup0), nsetup, b->chunk0[1],
                                b->nchunks[1], at<uint32_t>(ws, B.tile0), ntiles, common_nd, kDecShapes[1]};
  if (dec_capture(b) != cudaSuccess) {
    delete b;
    return CSZ_E_CUDA;
  }
  *out = b;
  return CSZ_OK;
}

}  // extern "C"

namespace {

// (Re)captures the batch's decompression graph with its current launch shape.
cudaError_t dec_capture(csz_batch_dec* b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  cudaError_t e;
  const bool tracing = trace_suspend();
  cudaGraph_t graph = nullptr;
  cudaStream_t cap = nullptr;
  const char* step = "capture stream";
  e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    step = "begin capture";
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  }
  if (e == cudaSuccess) {
    const cudaError_t e2 = dec_enqueue(b, cap);
    e = cudaStreamEndCapture(cap, &graph);
    step = "end capture";
    if (e == cudaSuccess && e2 != cudaSuccess) {
      e = e2;
      step = "captured launches";
    }
  }
  if (e == cudaSuccess) {
    step = "instantiate";
    e = cudaGraphInstantiate(&b->exec, graph, 0);
  }
  if (graph) cudaGraphDestroy(graph);
  if (cap) cudaStreamDestroy(cap);
  trace_resume(tracing);
  if (failed(e, step)) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return e;
}

}  // namespace

extern "C" {

csz_status csz_batch_dec_tune(csz_batch_dec* b, void* stream, int* h_warps, double* h_ms) {
  if (!b || !b->exec) return CSZ_E_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool tracing = trace_suspend();
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  cudaError_t e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  double best = -1.0;
  int pick = 1;
  for (int v = 0; v < 3 && e == cudaSuccess; v++) {
    b->launch.warps = kDecShapes[v];
    b->launch.chunk0 = b->chunk0[v];
    b->launch.nchunks = b->nchunks[v];
    e = dec_enqueue(b, s);  // warm-up
    float ms = 0.0f, tot = 0.0f;
    for (int r = 0; r < 3 && e == cudaSuccess; r++) {
      e = cudaEventRecord(t0, s);
      if (e == cudaSuccess) e = dec_enqueue(b, s);
      if (e == cudaSuccess) e = cudaEventRecord(t1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
      tot += ms;
    }
    if (h_ms) h_ms[v] = tot / 3.0;
    if (e == cudaSuccess && (best < 0.0 || tot < best)) {
      best = tot;
      pick = v;
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  trace_resume(tracing);
  b->launch.warps = kDecShapes[pick];
  b->launch.chunk0 = b->chunk0[pick];
  b->launch.nchunks = b->nchunks[pick];
  if (h_warps) *h_warps = kDecShapes[pick];
  if (e != cudaSuccess) {
    failed(e, "decompression tuning");
    return CSZ_E_CUDA;
  }
  return dec_capture(b) == cudaSuccess ? CSZ_OK : CSZ_E_CUDA;
}

csz_status csz_batch_decompress(csz_batch_dec* b, void* stream) {
  if (!b || !b->exec) return CSZ_E_ARG;
  if (trace_on()) {  // as for compression: launches one by one, each with its events
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (dec_enqueue(b, s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
    trace_fold();
    return CSZ_OK;
  }
  if (cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return CSZ_E_CUDA;
  trace_count_decode_batch();
  return CSZ_OK;
}

csz_status csz_batch_dec_results(csz_batch_dec* b, int* h_status, void* stream) {
  if (!b) return CSZ_E_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<unsigned char> buf(kStateStride * b->nfields);
  if (cudaMemcpyAsync(buf.data(), b->states, buf.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CSZ_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
  csz_status worst = CSZ_OK;
  for (int f = 0; f < b->nfields; f++) {
    DevState st;
    memcpy(&st, buf.data() + kStateStride * f, sizeof(st));
    const csz_status r = fold(st.status);
    if (h_status) h_status[f] = (int)r;
    if (r != CSZ_OK && worst == CSZ_OK) worst = r;
  }
  return worst;
}

void csz_batch_dec_destroy(csz_batch_dec* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  delete b;
}

const char* csz_batch_last_error(void) {
  static char buf[160];
  snprintf(buf, sizeof(buf), "%s: %s", g_fail_step, cudaGetErrorString(g_fail_err));
  return buf;
}

void csz_batch_destroy(csz_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  delete b;
}

}  // extern "C"
