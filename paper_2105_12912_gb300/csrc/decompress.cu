// Decompression kernels of cszp (sm_103a).
//
//   dec_setup_kernel       codec / block-size validation and payload offsets (scan),
//                          decode tables + 14-bit lookup table per book, record
//                          validation and each block's first record
//   stream_decode_kernel   one warp per interleaved 32-lane stream (Huffman code
//                          streams, RLE+Huffman value and length streams)
//   rle_expand_kernel      one CTA per listed RLE / RLE+Huffman block: runs to codes
//   reconstruct_kernel<ND> fuse outliers (q' = q - r, or delta), N-D partial sums
//                          per chunk (Alg. 1, Sec. IV-B2), scale by 2eb, verbatim
//                          patches
//   dec_status_kernel      the status word of an asynchronous decompression
// and their batch forms (per-field tables in device memory, headers read and checked
// on the device by dec_header_batch_kernel).
#include "common.cuh"
#include "host.h"
#include "kernels.h"

namespace cszp {

__device__ __forceinline__ void flag(DevState* st, uint32_t bits) { atomicOr(&st->status, bits); }

// =================================================================================
// archive validation and offsets
// =================================================================================
__device__ void dec_prep_body(const DecodeArgs& a) {
  if (a.dead) return;
  __shared__ uint64_t s_scan[33];
  __shared__ uint32_t s_nc[3];
  const int tid = threadIdx.x;
  if (a.check_hdr && tid < 32) {
    // the launch was set up from a host copy of the header: it must be this archive's
    const uint8_t* h = a.ar + 4 * tid;
    const uint32_t v = (uint32_t)h[0] | ((uint32_t)h[1] << 8) | ((uint32_t)h[2] << 16) | ((uint32_t)h[3] << 24);
    if (__any_sync(~0u, v != a.hdr[tid]) && tid == 0) flag(a.st, ERR_CORRUPT);
  }
  if (tid < 3) s_nc[tid] = 0;
  __syncthreads();
  // payload offsets and, packed above them in the same scan (bits 40-51 and 52-63; a
  // scan step covers at most 1024 blocks), the lists of run blocks and of the blocks
  // the reconstruction kernel takes (those not reconstructed by their decoder warps)
  constexpr uint64_t kLow = (1ull << 40) - 1, kMid = (1ull << 12) - 1;
  uint64_t carry = 0, rcarry = 0, scarry = 0;
  bool bad = false;
  for (uint32_t base = 0; base < a.g.nblk; base += blockDim.x) {
    const uint32_t b = base + tid;
    uint64_t bb = 0;
    bool run = false, slow = false;
    if (b < a.g.nblk) {
      const uint32_t c = a.ar[a.off_codec + b];
      bb = reinterpret_cast<const uint32_t*>(a.ar + a.off_bb)[b];
      if (c > 2 || (bb & 3) || bb >= (1ull << 30)) bad = true;  // a valid block is below 2^17 bytes
      else atomicAdd(&s_nc[c], 1u);
      run = c == CODEC_RLE || c == CODEC_RLE_HUFF;
      slow = !(a.fuse && c == CODEC_HUFF && block_is_full(a.g, b));
    }
    if (bb >= (1ull << 30)) bb = 0;
    uint64_t tot;
    const uint64_t ex =
        block_excl_scan<uint64_t>(bb | ((uint64_t)slow << 40) | ((uint64_t)run << 52), s_scan, &tot);
    if (b < a.g.nblk) a.blk_off[b] = carry + (ex & kLow);
    if (run && a.runblk) a.runblk[rcarry + (ex >> 52)] = b;
    if (slow && a.slowblk) a.slowblk[scarry + ((ex >> 40) & kMid)] = b;
    carry += tot & kLow;
    rcarry += tot >> 52;
    scarry += (tot >> 40) & kMid;
  }
  if (tid == 0) {
    a.st->n_slow = (uint32_t)scarry;
    a.blk_off[a.g.nblk] = carry;
    if (carry != a.payload) bad = true;
    if ((s_nc[CODEC_HUFF] && !(a.flags & 1u)) || (s_nc[CODEC_RLE_HUFF] && !(a.flags & 2u))) bad = true;
    for (int c = 0; c < 3; c++)
      if (s_nc[c] != a.n_codec[c]) bad = true;  // the header's counts decide which kernels run
  }
  if (bad) flag(a.st, ERR_CORRUPT);
}

// Single-field set-up, one CTA per 1024 codec blocks (chunks taken by ticket and
// chained by decoupled look-back, so no CTA scans the whole block list): codec and
// block-size validation, payload offsets, the lists of run blocks and of the blocks
// the reconstruction kernel takes, per-codec counts.  The chunk counted last checks
// the totals against the header.
__device__ void dec_prep_chunk_body(const DecodeArgs& a, uint32_t nchunks) {
  if (a.dead) return;  // (a batch field whose header failed: all its chunks leave)
  __shared__ uint64_t s_scan[33];
  __shared__ uint32_t s_scan32[33];
  __shared__ uint32_t s_nc[3];
  __shared__ uint32_t s_chunk;
  __shared__ unsigned long long s_cp, s_cc;
  __shared__ bool s_last;
  const int tid = threadIdx.x;
  if (tid == 0) s_chunk = atomicAdd(&a.st->ticket_encode, 1u);
  if (tid < 3) s_nc[tid] = 0;
  __syncthreads();
  const uint32_t chunk = s_chunk;
  if (chunk == 0 && a.check_hdr && tid < 32) {
    // the launch was set up from a host copy of the header: it must be this archive's
    const uint8_t* h = a.ar + 4 * tid;
    const uint32_t v = (uint32_t)h[0] | ((uint32_t)h[1] << 8) | ((uint32_t)h[2] << 16) | ((uint32_t)h[3] << 24);
    if (__any_sync(~0u, v != a.hdr[tid]) && tid == 0) flag(a.st, ERR_CORRUPT);
  }
  const uint32_t b = chunk * 1024u + tid;
  uint64_t bb = 0;
  bool run = false, slow = false, bad = false;
  if (b < a.g.nblk) {
    const uint32_t c = a.ar[a.off_codec + b];
    bb = reinterpret_cast<const uint32_t*>(a.ar + a.off_bb)[b];
    if (c > 2 || (bb & 3)) bad = true;
    else atomicAdd(&s_nc[c], 1u);
    run = c == CODEC_RLE || c == CODEC_RLE_HUFF;
    slow = !(a.fuse && c == CODEC_HUFF && block_is_full(a.g, b));
  }
  uint64_t tot_pay;
  const uint64_t ex_pay = block_excl_scan<uint64_t>(bb, s_scan, &tot_pay);
  uint32_t tot_cnt;  // (slow << 16) | run, at most 1024 each in a chunk
  const uint32_t ex_cnt = block_excl_scan<uint32_t>(((uint32_t)slow << 16) | (uint32_t)run, s_scan32, &tot_cnt);
  if (tid < 32) {
    // chunk totals: payload bytes; (slow blocks << 32) | run blocks (each below 2^19)
    const uint64_t cnt = ((uint64_t)(tot_cnt >> 16) << 32) | (tot_cnt & 0xffffu);
    if (tid == 0) {
      lookback_publish(a.prep_lb, chunk, tot_pay);
      lookback_publish(a.prep_lb + nchunks, chunk, cnt);
    }
    const uint64_t cp = lookback_warp(a.prep_lb, chunk, tot_pay, &a.st->status, kSpinLimit);
    const uint64_t cc = lookback_warp(a.prep_lb + nchunks, chunk, cnt, &a.st->status, kSpinLimit);
    if (tid == 0) {
      s_cp = cp;
      s_cc = cc;
    }
  }
  __syncthreads();
  const uint64_t cp = s_cp, cc = s_cc;
  if (b < a.g.nblk) a.blk_off[b] = cp + ex_pay;
  if (run && a.runblk) a.runblk[(uint32_t)cc + (ex_cnt & 0xffffu)] = b;
  if (slow && a.slowblk) a.slowblk[(uint32_t)(cc >> 32) + (ex_cnt >> 16)] = b;
  if (tid == 0) {
    if (chunk == nchunks - 1) {
      a.blk_off[a.g.nblk] = cp + tot_pay;
      a.st->n_slow = (uint32_t)(cc >> 32) + (tot_cnt >> 16);
      if (cp + tot_pay != a.payload) bad = true;
    }
    for (int c = 0; c < 3; c++)
      if (s_nc[c]) atomicAdd(&a.st->ncodec[c], s_nc[c]);
    __threadfence();
    s_last = atomicAdd(&a.st->encode_done, 1u) == nchunks - 1;
  }
  if (bad) flag(a.st, ERR_CORRUPT);
  __syncthreads();
  if (s_last && tid == 0) {
    __threadfence();
    uint32_t nc[3];
    for (int c = 0; c < 3; c++) nc[c] = atomicAdd(&a.st->ncodec[c], 0u);
    bool wrong = (nc[CODEC_HUFF] && !(a.flags & 1u)) || (nc[CODEC_RLE_HUFF] && !(a.flags & 2u));
    for (int c = 0; c < 3; c++)
      if (nc[c] != a.n_codec[c]) wrong = true;  // the header's counts decide which kernels run
    if (wrong) flag(a.st, ERR_CORRUPT);
  }
}

__device__ void dec_records_body(const DecodeArgs& a, uint32_t cta, uint32_t nctas) {
  if (a.dead) return;
  const uint32_t* rec = reinterpret_cast<const uint32_t*>(a.ar + a.off_rec);
  const uint64_t nslots = (uint64_t)a.g.nblk * kSlots;
  const uint64_t n = a.n_rec > (uint64_t)a.g.nblk + 1 ? a.n_rec : (uint64_t)a.g.nblk + 1;
  for (uint64_t i = cta * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)nctas * blockDim.x) {
    if (i < a.n_rec) {
      const uint32_t key = rec[2 * i];
      bool bad = ((i + 1 < a.n_rec) && key >= rec[2 * (i + 1)]) || (a.f64 && (key & 1u));
      const uint64_t slot = key >> 1;
      if (slot >= nslots) {
        bad = true;
      } else {
        uint32_t org[3], w[3];
        block_box(a.g, (uint32_t)(slot / kSlots), org, w);
        if (slot % kSlots >= (uint64_t)w[0] * w[1] * w[2]) bad = true;
      }
      if (bad) flag(a.st, ERR_CORRUPT);
    }
    if (i <= a.g.nblk) {
      const uint64_t target = i * (uint64_t)kSlots * 2;
      uint64_t lo = 0, hi = a.n_rec;
      while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if ((uint64_t)rec[2 * mid] < target) lo = mid + 1;
        else hi = mid;
      }
      a.rec_start[i] = (uint32_t)lo;
    }
  }
}

// One CTA per book: lengths from the archive, Kraft check, canonical tables and a
// 14-bit lookup table (16-bit entries).
__device__ void dec_tables_body(const DecodeArgs& a, int book) {
  if (a.dead) return;
  __shared__ uint8_t s_len[kNsymLen];
  __shared__ uint16_t s_wcnt[(kNsymLen / 32) * (kMaxLen + 1)];
  __shared__ CanonSmem cs;
  __shared__ uint32_t s_cnt[kMaxLen + 2];
  __shared__ uint32_t s_bad;
  const int tid = threadIdx.x;
  const int nsym = book == 2 ? kNsymLen : kNsymCode;
  DecTab* t = &a.tabs[book];
  const bool present = book == 0 ? (a.flags & 1u) : (a.flags & 2u);
  if (!present) {
    if (tid == 0) t->present = 0;
    return;
  }
  uint64_t off = a.off_books;
  if (book >= 1 && (a.flags & 1u)) off += kNsymCode;
  if (book == 2) off += kNsymCode;
  if (tid == 0) s_bad = 0;
  for (int l = tid; l < kMaxLen + 2; l += blockDim.x) s_cnt[l] = 0;
  __syncthreads();
  for (int s = tid; s < nsym; s += blockDim.x) {
    const uint8_t l = a.ar[off + s];
    s_len[s] = l;
    if (l > kMaxLen || (book < 2 && s >= (int)(2 * a.radius) && l)) s_bad = 1;
    else if (l) atomicAdd(&s_cnt[l], 1u);
  }
  __syncthreads();
  if (tid == 0) {
    long long avail = 1;
    for (int l = 1; l <= kMaxLen; l++) {
      avail = avail * 2 - (long long)s_cnt[l];
      if (avail < 0) {
        s_bad = 1;
        break;
      }
      if (avail > (1ll << 40)) avail = 1ll << 40;
    }
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) {
      flag(a.st, ERR_CORRUPT);
      t->present = 0;
    }
    return;
  }
  canonical_build(s_len, nsym, &cs, s_wcnt, nullptr, t->sorted);
  for (int l = tid; l <= kMaxLen; l += blockDim.x) {
    t->first[l] = cs.first[l];
    t->count[l] = cs.cnt[l];
    t->off[l] = cs.off[l];
  }
  if (tid == 0) {
    // canonical codes of length l, left-justified to 64 bits, occupy
    // [first_l << (64-l), (first_l + count_l) << (64-l)); these ends never decrease
    uint32_t mx = 0;
    unsigned long long lim = 0, full = 0;
    for (int l = 1; l <= kMaxLen; l++) {
      if (cs.cnt[l]) {
        mx = l;
        const unsigned long long end = cs.first[l] + cs.cnt[l];
        if (l == 64) {
          lim = end;
        } else if ((end >> l) != 0) {
          full |= ~0ull << l;  // the code space is exhausted from this length on
          lim = 0;
        } else {
          lim = end << (64 - l);
        }
      }
      t->limit[l] = lim;
    }
    t->fullmask = full;
    t->limit[0] = 0;
    t->maxlen = mx;
    t->present = 1;
  }
  // lookup: for each kLutBits-bit prefix, the code of length <= kLutBits it starts with
  for (int v = tid; v < (1 << kLutBits); v += blockDim.x) {
    uint32_t e = 0;
    for (int l = 1; l <= kLutBits; l++) {
      const uint64_t c = (uint64_t)(v >> (kLutBits - l));
      if (cs.cnt[l] && c >= cs.first[l] && c - cs.first[l] < cs.cnt[l]) {
        e = lut_entry(t->sorted[cs.off[l] + (uint32_t)(c - cs.first[l])], (uint32_t)l);
        break;
      }
    }
    t->lut[v] = (LutEntry)e;
  }
}

// One launch for archive set-up: the first `nchunks` CTAs validate codecs and scan
// block sizes (one chunk of 1024 blocks each), the next three build the decode tables
// of the three books, the rest validate records and find each block's first record.
__global__ __launch_bounds__(1024) void dec_setup_kernel(DecodeArgs a, uint32_t nchunks) {
  if (blockIdx.x < nchunks) {
    dec_prep_chunk_body(a, nchunks);
  } else if (blockIdx.x < nchunks + 3) {
    dec_tables_body(a, (int)(blockIdx.x - nchunks));
  } else {
    dec_records_body(a, blockIdx.x - nchunks - 3, gridDim.x - nchunks - 3);
  }
}

// =================================================================================
// interleaved Huffman streams: one warp decodes one stream (see common.cuh)
// =================================================================================
struct BookView {
  const LutEntry* lut;  // 1 << kLutBits entries
  const unsigned long long* first;
  const unsigned long long* limit;
  const uint32_t* count;
  const uint32_t* off;
  const uint16_t* sorted;
  int maxlen;
  unsigned long long fullmask;
};

// Matching the next codeword among the nb valid top bits of bb.  A table code of
// length l <= nb found among the zero-padded top kLutBits bits is the next codeword (no
// codeword is a prefix of another).  A table miss with more than kLutBits bits at hand is
// a longer code: its length is the smallest one whose left-justified codes end above
// bb (a binary search over the canonical limits), the true length whenever it is <= nb
// (zero bits below nb cannot complete a shorter codeword), checked to be a codeword.
// Returns that length (0 if none fits in nb bits) and sets sym.
__device__ __forceinline__ int ihs_match_long(uint64_t bb, int nb, const BookView& bk, int& sym) {
  int lo = kLutBits + 1, hi = bk.maxlen + 1;  // smallest k whose codes end above bb
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (((bk.fullmask >> mid) & 1ull) || bb < bk.limit[mid]) hi = mid;
    else lo = mid + 1;
  }
  if (lo > bk.maxlen || lo > nb) return 0;
  const uint64_t c = bb >> (64 - lo);
  if (c < bk.first[lo] || c - bk.first[lo] >= bk.count[lo]) return 0;  // not a codeword
  sym = (int)bk.sorted[bk.off[lo] + (uint32_t)(c - bk.first[lo])];
  return lo;
}

// A warp's reader of one interleaved stream in[0..avail).  The warp reads the stream
// strictly in order, so the next 96 units are kept in three 32-unit register windows
// (lane i holds unit base+i of each); a top-up takes its unit from a window by
// shuffle and a window is reloaded (one 64-byte load) two windows before it is
// needed, so no load sits on the decode's critical path.
struct IhsReader {
  const uint16_t* __restrict__ in;
  uint32_t avail;
  uint32_t w0, w1, w2;
  uint32_t wbase;  // stream index of w0's lane 0
  uint32_t cur;    // units taken so far by the warp
  uint64_t bb;     // this lane's bits, left-aligned
  int nb;
  bool bad;        // this lane met a damaged stream

  __device__ __forceinline__ uint32_t fetch(uint32_t i) const { return i < avail ? (uint32_t)__ldg(&in[i]) : 0u; }

  __device__ __forceinline__ void init(const uint16_t* p, uint32_t n) {
    const uint32_t lane = threadIdx.x & 31;
    in = p;
    avail = n;
    w0 = fetch(lane);
    w1 = fetch(32 + lane);
    w2 = fetch(64 + lane);
    wbase = 0;
    cur = 0;
    bb = 0;
    nb = 0;
    bad = false;
  }

  // One decoding step of the 32 lanes (every lane calls): each active lane tops up
  // its bits in rounds until a codeword is complete, then consumes it.  Returns the
  // symbol, meaningful where the lane was active and is not bad.  Control flow is
  // warp-uniform: a round's unit goes in by selects, and the search for codes longer
  // than the table runs only when some lane has one.
  __device__ __forceinline__ int step(bool active, const BookView& bk) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const bool live = active && !bad;
    uint32_t e = bk.lut[(uint32_t)(bb >> (64 - kLutBits))];
    int l = lut_len(e);
    int sym = lut_sym(e);
    int ml = (live && (uint32_t)(l - 1) < (uint32_t)nb) ? l : 0;  // a table code within the bits
    bool lng = live && l == 0 && nb > kLutBits;
    if (__any_sync(~0u, lng)) {
      if (lng) ml = ihs_match_long(bb, nb, bk, sym);
    }
    bool need = live && ml == 0;
    uint32_t ballot = __ballot_sync(~0u, need);
    while (ballot != 0u) {
      const uint32_t before = __popc(ballot & lt);
      const uint32_t rel = cur - wbase + before;  // < 64 while cur - wbase < 32
      const uint32_t u0 = __shfl_sync(~0u, w0, rel & 31);
      const uint32_t u1 = __shfl_sync(~0u, w1, rel & 31);
      const bool over = nb > 64 - 16 || cur + before >= avail;
      bad = bad || (need && over);
      const bool take = need && !over;
      const uint64_t unit = (uint64_t)(rel < 32 ? u0 : u1) << ((48 - nb) & 63);
      bb |= take ? unit : 0ull;
      nb += take ? 16 : 0;
      cur += __popc(ballot);
      if (cur - wbase >= 32) {
        w0 = w1;
        w1 = w2;
        wbase += 32;
        w2 = fetch(wbase + 64 + lane);
      }
      // only lanes that took a unit look again
      e = bk.lut[(uint32_t)(bb >> (64 - kLutBits))];
      l = lut_len(e);
      if (take && (uint32_t)(l - 1) < (uint32_t)nb) {
        ml = l;
        sym = lut_sym(e);
      }
      lng = take && l == 0 && nb > kLutBits;
      if (__any_sync(~0u, lng)) {
        if (lng) ml = ihs_match_long(bb, nb, bk, sym);
      }
      need = take && ml == 0;
      ballot = __ballot_sync(~0u, need);
    }
    bb = ml >= 64 ? 0ull : bb << ml;  // ml = 0 where the lane consumes nothing
    nb -= ml;
    return live ? sym : 0;
  }
};

// One warp decodes N symbols (+add) from in[0..avail) into out[].  Returns false
// (warp-uniform) if the stream is damaged; *used gets the units read.
__device__ bool ihs_decode_warp(const uint16_t* __restrict__ in, uint32_t avail, uint32_t N,
                                const BookView& bk, uint16_t* out, int add, uint32_t* used) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t T = (N + 31) / 32;
  IhsReader rd;
  rd.init(in, avail);
  for (uint32_t t = 0; t < T; t++) {
    const bool active = 32 * t + lane < N;
    const int sym = rd.step(active, bk);
    if (active && !rd.bad) out[32 * t + lane] = (uint16_t)(sym + add);
  }
  *used = rd.cur;
  return !__any_sync(~0u, rd.bad);
}

__device__ __forceinline__ float scale(int32_t k, float ebx2) { return __fmul_rn(__int2float_rn(k), ebx2); }

// The reconstruction's output by element type: x' = fl32(k * 2eb_f) for FP32 fields,
// x' = fl64(k * step) for double fields (which have no verbatim patches).
template <typename E>
struct Out;
template <>
struct Out<float> {
  float* __restrict__ p;
  float ebx2;
  __device__ explicit Out(const DecodeArgs& a) : p(a.out), ebx2(a.ebx2_f) {}
  __device__ __forceinline__ float value(int32_t k) const { return scale(k, ebx2); }
  __device__ __forceinline__ void put(uint64_t i, int32_t k) const { __stcs(&p[i], scale(k, ebx2)); }
  __device__ __forceinline__ void put_patch(uint64_t i, int32_t k, bool patch, uint32_t bits) const {
    __stcs(&p[i], patch ? __uint_as_float(bits) : scale(k, ebx2));
  }
  __device__ __forceinline__ void patch(uint64_t i, uint32_t bits) const { p[i] = __uint_as_float(bits); }
};
template <>
struct Out<double> {
  double* __restrict__ p;
  double step;
  __device__ explicit Out(const DecodeArgs& a) : p(a.out64), step(a.step_d) {}
  __device__ __forceinline__ void put(uint64_t i, int32_t k) const { __stcs(&p[i], __dmul_rn((double)k, step)); }
  __device__ __forceinline__ void put_patch(uint64_t i, int32_t k, bool, uint32_t) const { put(i, k); }
  __device__ __forceinline__ void patch(uint64_t, uint32_t) const {}
};

// =================================================================================
// fused decoding and reconstruction of full Huffman blocks (Alg. 1 decompression,
// Sec. IV-B "Partial-Sum Lorenzo Reconstruction")
//
// A full block's stream A holds its first 2048 codes and stream B the rest, and
// 2048 codes end on a Lorenzo-chunk boundary in every dimensionality: 8 chunks of
// 256 (1-D), rows 0-31 / 32-63 (2-D, 16x16 chunks), z 0-7 / 8-15 (3-D, 8^3 chunks).
// So the warp that decodes a stream owns whole chunks, and at step t lane l holds
// code 32t + l, which is already where the partial sums want it:
//   1-D  element 32t + l: the x sum is a warp scan plus a carry within each chunk
//        of 8 steps;
//   2-D  row t/2, column 32(t&1) + l: x sums over 16-lane groups by shuffles, y sums
//        in a register per column half, restarting every 16 rows;
//   3-D  plane t/8, row 2(t%8) + l/16, column l%16: x sums over 8-lane groups, y sums
//        across the lane pair (l, l^16) by one shuffle and a running pair sum that
//        restarts every 4 steps, z sums in a register per step of the plane.
// Each step then scales the exact integers and stores them: the codes never leave
// the registers.  Outliers (code 0) take their delta from the block's records, found
// by binary search (records are sorted by slot); verbatim patches overwrite their
// elements after the warp's own stores.
// =================================================================================

// The block's outlier records, merged into the decode order.  Records are sorted by
// key (slot * 2 + kind), and step t of a stream covers 32 consecutive slots, so the
// warp keeps the key of its next record in a register; only a step that reaches it
// loads the step's records (at most 64: an outlier and a patch per slot) and hands
// each outlier's delta to the lane of its slot through a 32-word per-warp table in
// shared memory (the fused code q' of Alg. 1).  The step's outlier records must match
// its code-0 slots one for one; anything else marks the stream corrupt.  Patches are
// applied after the stream (they only overwrite output values).
struct RecordCursor {
  const uint2* __restrict__ rec;
  uint32_t ptr, end;  // next record, end of the block's records
  uint32_t next;      // key of rec[ptr] (0xffffffff when none is left)

  // Positions the cursor at the first record with key >= key_lo among rec[rs..re).
  __device__ __forceinline__ void init(const uint2* r, uint32_t rs, uint32_t re, uint32_t key_lo) {
    rec = r;
    end = re;
    uint32_t lo = rs, hi = re;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (rec[mid].x < key_lo) lo = mid + 1;
      else hi = mid;
    }
    ptr = lo;
    next = ptr < end ? rec[ptr].x : 0xffffffffu;
  }

  // The step whose first slot has key key0 (the calling lane's slot has key key0 +
  // 2 lane): where sym == 0, q becomes the outlier's delta.  All lanes call
  // (warp-uniform control flow).  s_tab: this warp's 32 words of shared memory.
  __device__ __forceinline__ void step(uint32_t key0, int sym, int32_t& q, bool& bad, uint32_t* s_tab) {
    const uint32_t lane = threadIdx.x & 31;
    if (next >= key0 + 64u) {  // no record in this step (the common case)
      bad |= sym == 0;
      return;
    }
    uint32_t omask = 0;
#pragma unroll
    for (int half = 0; half < 2; half++) {
      const uint32_t i = ptr + lane;  // ptr has moved past the first half's records
      const uint2 kv = i < end ? rec[i] : make_uint2(0xffffffffu, 0u);
      const bool here = kv.x < key0 + 64u;
      const uint32_t l = ((kv.x >> 1) - (key0 >> 1)) & 31u;  // the record's lane
      const bool outlier = here && !(kv.x & 1u);
      if (outlier) s_tab[l] = kv.y;
      omask |= __reduce_or_sync(~0u, outlier ? 1u << l : 0u);
      const uint32_t hb = __ballot_sync(~0u, here);
      ptr += __popc(hb);
      if (hb != ~0u) break;
    }
    __syncwarp();
    if ((omask >> lane) & 1u) q = (int32_t)s_tab[lane];
    bad |= __ballot_sync(~0u, sym == 0) != omask;
    next = ptr < end ? rec[ptr].x : 0xffffffffu;
    __syncwarp();  // the table is free again
  }
};

// Decodes stream `which` (0: A, 1: B) of full Huffman block b from u[0..avail) and
// writes its 2048 reconstructed elements.  The warp decodes 8 steps into a register
// window, then runs their 8 prefix chains together (independent shuffles overlap)
// and stores them.  Returns false (warp-uniform) if the stream is damaged or its records do not
// match its outlier slots; *used gets the units read.  s_tab: this warp's 288 words
// of shared memory (the record table, then the 3-D running sums).
template <int ND, typename E>
__device__ bool fused_decode_reconstruct(const DecodeArgs& a, uint32_t b, uint32_t which, const uint16_t* u,
                                         uint32_t avail, const BookView& bk, uint32_t* used, uint32_t* s_tab) {
  const uint32_t lane = threadIdx.x & 31;
  const int32_t r = (int32_t)a.radius;
  const Out<E> out(a);
  const uint32_t key0 = (b * (uint32_t)kSlots + 2048u * which) * 2u;  // record key of the stream's first slot
  uint32_t org[3], w[3];
  block_box(a.g, b, org, w);
  const uint64_t ny = a.g.n[1], nx = a.g.n[2];
  const uint2* rec = reinterpret_cast<const uint2*>(a.ar + a.off_rec);
  const uint32_t rs = a.rec_start[b], re = a.rec_start[b + 1];
  IhsReader rd;
  rd.init(u, avail);
  RecordCursor rc;
  rc.init(rec, rs, re, key0);
  bool bad = false;
  // 3-D: the running z sum of each of the lane's 8 rows of a plane, in this warp's
  // shared-memory strip (row s of lane l at zs[32 s + l]: no bank conflicts)
  int32_t* zs = reinterpret_cast<int32_t*>(s_tab) + 32;
  int32_t carry = 0, ysum0 = 0, ysum1 = 0;
  if (ND == 3) {
#pragma unroll
    for (int s = 0; s < 8; s++) zs[32 * s + lane] = 0;
  }
#pragma unroll 1
  for (uint32_t t0 = 0; t0 < 64; t0 += 8) {
    // the decoding step runs two copies per iteration (four overflow the instruction
    // cache); each pair of steps' q' shifts into an 8-register window
    int32_t q[8];
#pragma unroll 1
    for (uint32_t s0 = 0; s0 < 8; s0 += 2) {
#pragma unroll
      for (uint32_t u = 0; u < 2; u++) {
        const int sym = rd.step(true, bk);
        int32_t v = sym - r;
        rc.step(key0 + 64u * (t0 + s0 + u), sym, v, bad, s_tab);
        q[6 + u] = v;
      }
      if (s0 + 2 < 8) {
#pragma unroll
        for (int k = 0; k < 6; k++) q[k] = q[k + 2];
      }
    }
    if (ND == 1) {
      // 8 steps = one 256-element chunk: per-step warp scans, then the carries
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int s = 0; s < 8; s++) {
          const int32_t up = __shfl_up_sync(~0u, q[s], o);
          if (lane >= (uint32_t)o) q[s] += up;
        }
      }
      carry = 0;
      const uint64_t base = (uint64_t)org[2] + 2048u * which + 32u * t0 + lane;
#pragma unroll
      for (int s = 0; s < 8; s++) {
        const int32_t v = q[s] + carry;
        carry += __shfl_sync(~0u, q[s], 31);
        out.put(base + 32u * s, v);
      }
    } else if (ND == 2) {
      // rows t/2, columns 32 (t&1) + lane: x sums over 16-lane groups, y sums down
      // each column half, restarting every 16 rows (32 steps)
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) {
#pragma unroll
        for (int s = 0; s < 8; s++) {
          const int32_t up = __shfl_up_sync(~0u, q[s], o);
          if ((lane & 15) >= (uint32_t)o) q[s] += up;
        }
      }
      if ((t0 & 31) == 0) ysum0 = ysum1 = 0;
      const uint64_t base = ((uint64_t)org[1] + 32u * which + (t0 >> 1)) * nx + org[2] + lane;
#pragma unroll
      for (int s = 0; s < 8; s++) {
        int32_t& ys = (s & 1) ? ysum1 : ysum0;
        ys += q[s];
        out.put(base + (uint64_t)(s >> 1) * nx + 32u * (s & 1), ys);
      }
    } else {
      // plane t/8 of the stream's z chunk, rows 2s + lane/16, column lane%16: x sums
      // over 8-lane groups, y sums across the lane pair (l, l^16) within each 8-row
      // chunk, z sums in registers
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
#pragma unroll
        for (int s = 0; s < 8; s++) {
          const int32_t up = __shfl_up_sync(~0u, q[s], o);
          if ((lane & 7) >= (uint32_t)o) q[s] += up;
        }
      }
      const uint32_t p = lane >> 4;
      const uint32_t zp = t0 >> 3;
      const uint64_t base = ((uint64_t)(org[0] + 8u * which + zp) * ny + org[1] + p) * nx + org[2] + (lane & 15);
      int32_t pair = 0;
#pragma unroll
      for (int s = 0; s < 8; s++) {
        const int32_t other = __shfl_xor_sync(~0u, q[s], 16);
        if (s == 4) pair = 0;  // rows 8-15: the second y chunk
        const int32_t k = zs[32 * s + lane] + pair + q[s] + (p ? other : 0);
        zs[32 * s + lane] = k;
        pair += q[s] + other;
        out.put(base + (uint64_t)(2 * s) * nx, k);
      }
    }
  }
  *used = rd.cur;
  const bool ok = !__any_sync(~0u, rd.bad || bad);
  // verbatim patches of this stream's slots overwrite their elements (after the
  // warp's own stores: __syncwarp orders them)
  __syncwarp();
  for (uint32_t i = rs + lane; i < re; i += 32) {
    const uint2 kv = rec[i];
    const uint32_t j = (kv.x >> 1) % kSlots;
    if ((kv.x & 1u) && (j >> 11) == which) {
      uint64_t e;
      if (ND == 1) e = (uint64_t)org[2] + j;
      else if (ND == 2) e = (uint64_t)(org[1] + (j >> 6)) * nx + org[2] + (j & 63);
      else e = ((uint64_t)(org[0] + (j >> 8)) * ny + org[1] + ((j >> 4) & 15)) * nx + org[2] + (j & 15);
      out.patch(e, kv.y);
    }
  }
  return ok;
}

constexpr int kStreamWarps = kStreamWarpsPerCta;
constexpr int kRecTabWords = 288;  // per decoding warp of a fused stream: record table 32 + 3-D sums 256

// Entropy decoding, persistent: each CTA stages the lookup tables of the books the
// archive uses in shared memory once, then its warps take (block, stream) slots from
// a ticket; a warp decodes one stream of a Huffman block, or the value or the length
// stream of an RLE+Huffman block (runs go to the workspace run arrays).  With fusion
// (ND != 0 and a.fuse), a stream of a full Huffman block is reconstructed by the
// warp as it is decoded (fused_decode_reconstruct); other Huffman streams leave
// their codes in the workspace for the reconstruction kernel.
// Streams come from the field's ticket (b_end == 0) or, in batches, from the CTA's
// chunk of blocks [b_begin, b_end): each warp draws the chunk's next stream from a
// shared counter until none is left.
template <int ND, typename E>
__device__ void stream_decode_body(const DecodeArgs& a, uint32_t b_begin, uint32_t b_end) {
  extern __shared__ __align__(16) uint32_t s_dyn[];  // the present books' tables, then record tables
  __shared__ unsigned long long s_first[kMaxLen + 1], s_limit[kMaxLen + 1];
  __shared__ uint32_t s_off[kMaxLen + 1], s_count[kMaxLen + 1];
  __shared__ int s_go;
  if (a.dead) return;
  // the status is read once, by thread 0, and acted on after the staging barrier, so
  // that a corruption flagged by another CTA meanwhile cannot split this CTA
  __shared__ uint32_t s_next;  // batches: the chunk's next stream slot
  if (threadIdx.x == 0) {
    s_go = !(a.st->status & ERR_CORRUPT);
    s_next = 0;
  }
  const bool huff = (a.flags & 1u) != 0, rle = (a.flags & 2u) != 0;
  LutEntry* s_luts = reinterpret_cast<LutEntry*>(s_dyn);
  LutEntry* lut_code = s_luts;
  LutEntry* lut_val = s_luts + (huff ? (1 << kLutBits) : 0);
  LutEntry* lut_len = lut_val + (1 << kLutBits);
  // fused streams: after the tables, per warp a record table (32 words) and the 3-D
  // running sums (256 words); the launch sizes the dynamic shared memory for them
  uint32_t* s_rectab =
      reinterpret_cast<uint32_t*>(s_luts + (huff ? (1 << kLutBits) : 0) + (rle ? 2 * (1 << kLutBits) : 0));
  // a chunk of blocks (batches) copies only the tables its own blocks use
  bool need_code = huff, need_runs = rle;
  if (b_end != 0) {
    const uint32_t b = b_begin + threadIdx.x;
    const int c = (b < b_end) ? a.ar[a.off_codec + b] : -1;
    need_code = __syncthreads_or(huff && c == CODEC_HUFF) != 0;
    need_runs = __syncthreads_or(rle && c == CODEC_RLE_HUFF) != 0;
  }
  constexpr int kLutVec = (1 << kLutBits) * (int)sizeof(LutEntry) / 16;  // 16-byte pieces per table
  for (int i = threadIdx.x; i < kLutVec; i += blockDim.x) {
    if (need_code) reinterpret_cast<uint4*>(lut_code)[i] = reinterpret_cast<const uint4*>(a.tabs[0].lut)[i];
    if (need_runs) {
      reinterpret_cast<uint4*>(lut_val)[i] = reinterpret_cast<const uint4*>(a.tabs[1].lut)[i];
      reinterpret_cast<uint4*>(lut_len)[i] = reinterpret_cast<const uint4*>(a.tabs[2].lut)[i];
    }
  }
  for (int i = threadIdx.x; i <= kMaxLen; i += blockDim.x) {
    s_first[i] = a.tabs[0].first[i];
    s_limit[i] = a.tabs[0].limit[i];
    s_off[i] = a.tabs[0].off[i];
    s_count[i] = a.tabs[0].count[i];
  }
  __syncthreads();
  if (!s_go) return;
  const bool lane0 = (threadIdx.x & 31) == 0;
  const bool ticketed = b_end == 0;
  // work items are (block, stream) slots: a Huffman block's streams A and B, an
  // RLE+Huffman block's value and length streams
  for (;;) {
    uint32_t slot = 0;
    if (ticketed) {
      if (lane0) slot = atomicAdd(&a.st->ticket_decode, 1u);
      slot = __shfl_sync(~0u, slot, 0);
      if (slot >= 2 * a.g.nblk) break;
    } else {
      // the chunk's streams, drawn one at a time by whichever warp is free
      if (lane0) slot = atomicAdd(&s_next, 1u);
      slot = 2 * b_begin + __shfl_sync(~0u, slot, 0);
      if (slot >= 2 * b_end) break;
    }
    const uint32_t b = slot >> 1, which = slot & 1;
    const int codec = a.ar[a.off_codec + b];
    if (codec == CODEC_RLE) continue;
    uint32_t org[3], w[3];
    block_box(a.g, b, org, w);
    const uint32_t m = w[0] * w[1] * w[2];
    const uint64_t bytes = a.blk_off[b + 1] - a.blk_off[b];
    const uint8_t* pay = a.ar + a.off_pay + a.blk_off[b];
    uint32_t used = 0;
    bool ok;
    if (codec == CODEC_HUFF) {
      const DecTab* t = &a.tabs[0];
      const uint16_t* u = reinterpret_cast<const uint16_t*>(pay);
      const uint32_t nu = (uint32_t)(bytes / 2);
      const uint32_t na = nu >= 1 ? u[0] : 0u;
      if (!t->present || nu < 1 || na > nu - 1) {
        if (lane0) flag(a.st, ERR_CORRUPT);
        continue;
      }
      const uint32_t h = huff_split(m);
      const BookView bk{lut_code, s_first, s_limit, s_count, s_off, t->sorted, (int)t->maxlen, t->fullmask};
      if (ND != 0 && a.fuse && m == (uint32_t)kSlots) {
        if (which == 0) {
          ok = fused_decode_reconstruct<ND, E>(a, b, 0, u + 1, na, bk, &used, s_rectab + kRecTabWords * (threadIdx.x >> 5));
          ok = ok && used == na;
        } else {
          ok = fused_decode_reconstruct<ND, E>(a, b, 1, u + 1 + na, nu - 1 - na, bk, &used,
                                            s_rectab + kRecTabWords * (threadIdx.x >> 5));
          ok = ok && ((2ull * (1ull + na + used) + 3) & ~3ull) == bytes;
        }
      } else if (which == 0) {
        ok = ihs_decode_warp(u + 1, na, h, bk, a.codes + (uint64_t)b * kSlots, 0, &used);
        ok = ok && used == na;
      } else {
        ok = ihs_decode_warp(u + 1 + na, nu - 1 - na, m - h, bk, a.codes + (uint64_t)b * kSlots + h, 0, &used);
        ok = ok && ((2ull * (1ull + na + used) + 3) & ~3ull) == bytes;
      }
    } else {
      const DecTab* tv = &a.tabs[1];
      const DecTab* tl = &a.tabs[2];
      if (!tv->present || !tl->present) {
        if (lane0) flag(a.st, ERR_CORRUPT);
        continue;
      }
      const uint32_t* p32 = reinterpret_cast<const uint32_t*>(pay);
      const uint32_t nr = bytes >= 8 ? p32[0] : 0u, vu = bytes >= 8 ? p32[1] : 0u;
      if (bytes < 8 || nr > m || 8ull + 2ull * vu > bytes) {
        if (lane0) flag(a.st, ERR_CORRUPT);
        continue;
      }
      const uint32_t lavail = (uint32_t)((bytes - 8) / 2 - vu);
      const uint16_t* p16 = reinterpret_cast<const uint16_t*>(pay) + 4;
      if (which == 0) {
        const BookView bv{lut_val, tv->first, tv->limit, tv->count, tv->off, tv->sorted, (int)tv->maxlen,
                          tv->fullmask};
        ok = ihs_decode_warp(p16, vu, nr, bv, a.runv + (uint64_t)b * kSlots, 0, &used);
        ok = ok && used == vu;
      } else {
        const BookView bl{lut_len, tl->first, tl->limit, tl->count, tl->off, tl->sorted, (int)tl->maxlen,
                          tl->fullmask};
        ok = ihs_decode_warp(p16 + vu, lavail, nr, bl, a.runl + (uint64_t)b * kSlots, 1, &used);
        ok = ok && ((8ull + 2ull * (vu + used) + 3) & ~3ull) == bytes;
      }
    }
    if (!ok && lane0) flag(a.st, ERR_CORRUPT);
  }
}

template <int ND, typename E>
__global__ __launch_bounds__(32 * kStreamWarps, 2) void stream_decode_kernel(DecodeArgs a) {
  stream_decode_body<ND, E>(a, 0, 0);
}

constexpr int kRleThreads = 256;

// RLE and RLE+Huffman blocks: run starts by a block scan, then every code position
// finds its run by binary search.
// Runs of run block b to its 4096 codes at `out` (global or shared memory, 16-byte
// aligned), with shared scratch s_v, s_l (kSlots each) and s_start (kSlots + 1).
// Returns false (the same in every thread) when the block is not expanded: not a run
// block, corrupt (flagged), or its field already flagged corrupt.
__device__ bool rle_expand_into(const DecodeArgs& a, uint32_t b, uint16_t* out, uint16_t* s_v, uint16_t* s_l,
                                uint32_t* s_start) {
  __shared__ uint32_t s_scan[33];
  __shared__ uint32_t s_bad;
  const int tid = threadIdx.x;
  if (a.dead) return false;
  const int codec = a.ar[a.off_codec + b];
  if (codec != CODEC_RLE && codec != CODEC_RLE_HUFF) return false;
  uint32_t org[3], w[3];
  block_box(a.g, b, org, w);
  const uint32_t m = w[0] * w[1] * w[2];
  const uint64_t bytes = a.blk_off[b + 1] - a.blk_off[b];
  const uint8_t* pay = a.ar + a.off_pay + a.blk_off[b];
  const uint32_t lim = 2 * a.radius;
  uint32_t nr;
  const uint16_t *v, *l;
  if (codec == CODEC_RLE) {
    nr = (uint32_t)(bytes / 4);
    v = reinterpret_cast<const uint16_t*>(pay);
    l = v + nr;
  } else {
    nr = reinterpret_cast<const uint32_t*>(pay)[0];
    v = a.runv + (uint64_t)b * kSlots;
    l = a.runl + (uint64_t)b * kSlots;
  }
  if (nr > m) {
    if (tid == 0) flag(a.st, ERR_CORRUPT);
    return false;
  }
  // the status is read once, by thread 0, and acted on after the barrier, so that a
  // corruption flagged by another CTA meanwhile cannot split this CTA's threads
  if (tid == 0) s_bad = (a.st->status & ERR_CORRUPT) ? 2u : 0u;
  __syncthreads();
  if (s_bad == 2u) return false;
  for (uint32_t i = tid; i < nr; i += blockDim.x) {
    s_v[i] = v[i];
    s_l[i] = l[i];
  }
  __syncthreads();
  const uint32_t per = (nr + blockDim.x - 1) / blockDim.x;
  const uint32_t lo = min(nr, tid * per), hi = min(nr, lo + per);
  uint32_t sum = 0;
  for (uint32_t i = lo; i < hi; i++) {
    if (s_v[i] >= lim || s_l[i] == 0) s_bad = 1;
    sum += s_l[i];
  }
  uint32_t tot;
  uint32_t off = block_excl_scan<uint32_t>(sum, s_scan, &tot);
  for (uint32_t i = lo; i < hi; i++) {
    s_start[i] = off;
    off += s_l[i];
  }
  if (tid == 0) s_start[nr] = tot;
  __syncthreads();
  if (s_bad || tot != m) {
    if (tid == 0) flag(a.st, ERR_CORRUPT);
    return false;
  }
  // run index of every position: mark run starts, then a running maximum
  uint32_t* s_idx = s_start;  // starts are no longer needed once marked below
  uint32_t my_starts[16];
  const uint32_t cnt = hi - lo;
  for (uint32_t i = 0; i < cnt && i < 16; i++) my_starts[i] = s_start[lo + i];
  __syncthreads();
  for (int i = tid; i < kSlots; i += blockDim.x) s_idx[i] = 0;
  __syncthreads();
  if (cnt <= 16) {
    for (uint32_t i = 0; i < cnt; i++)
      if (my_starts[i] < m) s_idx[my_starts[i]] = lo + i;
  }
  __syncthreads();
  // contiguous 16 positions per thread: local running max, then a block scan of maxima
  uint32_t run = 0;
  const uint32_t p0 = 16 * tid;
#pragma unroll
  for (int i = 0; i < 16; i++) run = max(run, s_idx[p0 + i]);
  // exclusive running max over threads (warp scan + per-warp carries)
  uint32_t incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(~0u, incl, o);
    if ((tid & 31) >= o) incl = max(incl, u);
  }
  if ((tid & 31) == 31) s_scan[tid >> 5] = incl;
  __syncthreads();
  uint32_t carry = 0;
  for (int wv = 0; wv < (tid >> 5); wv++) carry = max(carry, s_scan[wv]);
  uint32_t excl = __shfl_up_sync(~0u, incl, 1);
  if ((tid & 31) == 0) excl = 0;
  uint32_t cur = max(carry, excl);
  uint32_t vals[8];
#pragma unroll
  for (int i = 0; i < 16; i++) {
    cur = max(cur, s_idx[p0 + i]);
    const uint16_t v = s_v[cur];
    if (i & 1) vals[i >> 1] |= (uint32_t)v << 16;
    else vals[i >> 1] = v;
  }
  // positions >= m get whatever run they fall in; they are never read
  uint4* o4 = reinterpret_cast<uint4*>(out + p0);
  o4[0] = make_uint4(vals[0], vals[1], vals[2], vals[3]);
  o4[1] = make_uint4(vals[4], vals[5], vals[6], vals[7]);
  return true;
}

// Run block b expanded in place in the code stream (global), with its own scratch.
__device__ void rle_expand_body(const DecodeArgs& a, uint32_t b) {
  __shared__ __align__(16) uint16_t s_v[kSlots];
  __shared__ __align__(16) uint16_t s_l[kSlots];
  __shared__ __align__(16) uint32_t s_start[kSlots + 1];
  rle_expand_into(a, b, a.codes + (uint64_t)b * kSlots, s_v, s_l, s_start);
}

// One CTA per listed run block (the list the set-up wrote; it holds exactly the
// header's count unless the archive is corrupt, which the set-up has flagged and
// the body checks).
__global__ __launch_bounds__(kRleThreads) void rle_expand_kernel(DecodeArgs a) {
  if (a.dead) return;
  const uint32_t b = a.runblk[blockIdx.x];
  if (b >= a.g.nblk) return;
  rle_expand_body(a, b);
}

// =================================================================================
// reconstruction: N-D partial sums per chunk (Sec. IV-B2), scaled by 2eb
// =================================================================================
constexpr int kRecThreads = 256;

// codes: the block's 4096 code slots (global memory, or a shared-memory copy)
template <int ND, typename E>
__device__ void reconstruct_body(const DecodeArgs& a, uint32_t b, int32_t* s_q, const uint16_t* codes) {
  // (the caller has checked the field's status, the same way in every thread)
  const int tid = threadIdx.x;
  uint32_t org[3], w[3];
  block_box(a.g, b, org, w);
  const uint32_t m = w[0] * w[1] * w[2];
  const int32_t r = (int32_t)a.radius;
  const Out<E> out(a);
  const uint32_t rs = a.rec_start[b], re = a.rec_start[b + 1];
  const uint2* rec = reinterpret_cast<const uint2*>(a.ar + a.off_rec);
  // a full 3-D block without records reads its codes directly; otherwise
  // codes -> q' = q - r in s_q, then the outliers' deltas
  const bool direct = ND == 3 && m == (uint32_t)kSlots && rs == re;
  if (!direct) {
    const uint4* src = reinterpret_cast<const uint4*>(codes);
    for (uint32_t i = tid; i < (m + 7) / 8; i += kRecThreads) {
      const uint4 v = src[i];
      const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; k++) {
        s_q[8 * i + 2 * k] = (int32_t)(u[k] & 0xffffu) - r;
        s_q[8 * i + 2 * k + 1] = (int32_t)(u[k] >> 16) - r;
      }
    }
    __syncthreads();
    for (uint32_t i = rs + tid; i < re; i += kRecThreads) {
      const uint2 kv = rec[i];
      if ((kv.x & 1u) == 0) s_q[(kv.x >> 1) % kSlots] = (int32_t)kv.y;
    }
    __syncthreads();
  }
  const uint64_t ny = a.g.n[1], nx = a.g.n[2];
  if (ND == 1) {
    // each warp scans whole 256-chunks, 32 elements per step
    const int lane = tid & 31, wid = tid >> 5;
    for (uint32_t c = wid; c * 256 < m; c += kRecThreads / 32) {
      int32_t carry = 0;
#pragma unroll
      for (int i = 0; i < 8; i++) {
        const uint32_t j = c * 256 + i * 32 + lane;
        const int32_t v = j < m ? s_q[j] : 0;
        const int32_t inc = warp_incl_scan(v) + carry;
        carry = __shfl_sync(~0u, inc, 31);
        if (j < m) out.put((uint64_t)org[2] + j, inc);
      }
    }
  } else if (ND == 2) {
    // thread = (column x, 16-row chunk band): y sums in registers, x sums by shuffles
    const uint32_t x = tid & 63, ry = tid >> 6;
    const bool xin = x < w[2];
    int32_t v[16];
#pragma unroll
    for (int i = 0; i < 16; i++) {
      const uint32_t y = ry * 16 + i;
      v[i] = (xin && y < w[1]) ? s_q[y * w[2] + x] : 0;
    }
#pragma unroll
    for (int i = 1; i < 16; i++) v[i] += v[i - 1];
#pragma unroll
    for (int i = 0; i < 16; i++) {
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) {
        const int32_t u = __shfl_up_sync(~0u, v[i], o);
        if ((x & 15) >= (uint32_t)o) v[i] += u;
      }
    }
    if (xin) {
      const uint64_t base = (uint64_t)org[1] * nx + org[2] + x;
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const uint32_t y = ry * 16 + i;
        if (y < w[1]) out.put(base + (uint64_t)y * nx, v[i]);
      }
    }
  } else if (m == (uint32_t)kSlots) {
    // full 16^3 block: thread (x, y) takes the z column -- z sums in registers, x
    // sums by shuffles -- then, after one exchange through shared memory, thread
    // (x, z) takes the y column, adds along y in registers and stores its row
    // segment (16 consecutive floats per half-warp)
    const uint32_t x = tid & 15, y = tid >> 4;
    int32_t v[16];
#pragma unroll
    for (int i = 0; i < 16; i++)
      v[i] = direct ? (int32_t)codes[(i * 16 + y) * 16 + x] - r : s_q[(i * 16 + y) * 16 + x];
#pragma unroll
    for (int i = 1; i < 16; i++)
      if (i & 7) v[i] += v[i - 1];
#pragma unroll
    for (int i = 0; i < 16; i++) {
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const int32_t u = __shfl_up_sync(~0u, v[i], o);
        if ((x & 7) >= (uint32_t)o) v[i] += u;
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; i++) s_q[(i * 16 + y) * 16 + x] = v[i];
    __syncthreads();
    const uint32_t z = tid >> 4;
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = s_q[(z * 16 + i) * 16 + x];
#pragma unroll
    for (int i = 1; i < 16; i++)
      if (i & 7) v[i] += v[i - 1];
    const uint64_t base = ((uint64_t)(org[0] + z) * ny + org[1]) * nx + org[2] + x;
#pragma unroll
    for (int i = 0; i < 16; i++) out.put(base + (uint64_t)i * nx, v[i]);
  } else {
    // edge block: z sums in registers, x sums by shuffles, y sums through shared
    // memory
    const uint32_t x = tid & 15, y = tid >> 4;
    const bool in_xy = x < w[2] && y < w[1];
    int32_t v[16];
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = (in_xy && (uint32_t)i < w[0]) ? s_q[(i * w[1] + y) * w[2] + x] : 0;
#pragma unroll
    for (int i = 1; i < 16; i++)
      if (i & 7) v[i] += v[i - 1];
#pragma unroll
    for (int i = 0; i < 16; i++) {
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const int32_t u = __shfl_up_sync(~0u, v[i], o);
        if ((x & 7) >= (uint32_t)o) v[i] += u;
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 16; i++)
      if (in_xy && (uint32_t)i < w[0]) s_q[(i * w[1] + y) * w[2] + x] = v[i];
    __syncthreads();
    {
      const uint32_t xx = tid & 15, zz = tid >> 4;
      if (xx < w[2] && zz < w[0]) {
        int32_t acc = 0;
        for (uint32_t yy = 0; yy < w[1]; yy++) {
          const uint32_t j = (zz * w[1] + yy) * w[2] + xx;
          acc = (yy & 7) ? acc + s_q[j] : s_q[j];
          s_q[j] = acc;
        }
      }
    }
    __syncthreads();
    for (uint32_t j = tid; j < m; j += kRecThreads) {
      const uint32_t p = w[1] * w[2];
      const uint32_t zz = j / p, rem = j - zz * p, yy = rem / w[2], xx = rem - yy * w[2];
      out.put(((uint64_t)(org[0] + zz) * ny + (org[1] + yy)) * nx + org[2] + xx, s_q[j]);
    }
  }
  __syncthreads();
  // verbatim patches overwrite their elements (ordered after the block's stores)
  for (uint32_t i = rs + tid; i < re; i += kRecThreads) {
    const uint2 kv = rec[i];
    if (kv.x & 1u) {
      const uint32_t j = (kv.x >> 1) % kSlots;
      const uint32_t p = w[1] * w[2];
      const uint32_t zz = j / p, rem = j - zz * p, yy = rem / w[2], xx = rem - yy * w[2];
      out.patch(((uint64_t)(org[0] + zz) * ny + (org[1] + yy)) * nx + org[2] + xx, kv.y);
    }
  }
}

// Persistent: CTA c takes work items c, c + grid, ...; while it reconstructs one
// block, a bulk copy is already bringing the next block's 8 KB of codes into shared
// memory.  The work items are all blocks, or, when the entropy decoder reconstructs
// full Huffman blocks itself (a.fuse), the listed other blocks.
template <int ND, typename E>
__global__ __launch_bounds__(kRecThreads) void reconstruct_kernel(DecodeArgs a) {
  __shared__ __align__(128) uint16_t s_codes[2][kSlots];
  __shared__ __align__(16) int32_t s_q[kSlots];
  __shared__ unsigned long long s_bar[2];
  __shared__ uint32_t s_fail;
  if (a.dead || (a.st->status & ERR_CORRUPT)) return;
  const int tid = threadIdx.x;
  const uint32_t grid = gridDim.x;
  const uint32_t nwork = a.fuse ? a.st->n_slow : a.g.nblk;
  auto block_of = [&](uint32_t i) -> uint32_t { return a.fuse ? a.slowblk[i] : i; };
  auto issue = [&](uint32_t b, int buf) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&s_bar[buf], kSlots * 2);
    bulk_load(s_codes[buf], a.codes + (uint64_t)b * kSlots, kSlots * 2, &s_bar[buf]);
  };
  if (tid == 0) {
    mbar_init(&s_bar[0]);
    mbar_init(&s_bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    if (blockIdx.x < nwork) issue(block_of(blockIdx.x), 0);
  }
  __syncthreads();
  uint32_t it = 0, i = blockIdx.x;
  bool next_issued = false;
  for (; i < nwork; i += grid, it++) {
    const int cur = it & 1;
    const uint32_t b = block_of(i);
    next_issued = i + grid < nwork;
    if (tid == 0 && next_issued) issue(block_of(i + grid), cur ^ 1);
    if (!mbar_wait(&s_bar[cur], (it >> 1) & 1u, kSpinLimit)) {
      atomicOr(&a.st->status, ERR_TIMEOUT);
      s_fail = 1;
    }
    __syncthreads();
    if (s_fail) break;
    reconstruct_body<ND, E>(a, b, s_q, s_codes[cur]);
    __syncthreads();
  }
  if (s_fail && tid == 0) {
    // wait once more (bounded) for this block's copy and the next one in flight
    mbar_wait(&s_bar[it & 1], (it >> 1) & 1u, kSpinLimit);
    if (next_issued) mbar_wait(&s_bar[(it + 1) & 1], ((it + 1) >> 1) & 1u, kSpinLimit);
  }
}

// =================================================================================
// global (unchunked) Lorenzo reconstruction: the N-D partial sum of q' over the whole
// field (Sec. IV-B "Partial-Sum Lorenzo Reconstruction" holds without chunks), as
// one pass per axis over an int32 copy of q' kept in the output buffer; the last pass
// scales to FP32 in place, then the verbatim patches are written.
// =================================================================================
constexpr uint32_t kScanTile = 4096;  // elements per tile of the x pass (256 threads x 16)

// q' of codec block b (q - r, or the outlier's delta) at its elements' field positions.
__global__ __launch_bounds__(kRecThreads) void gfuse_kernel(DecodeArgs a) {
  if (a.dead || (a.st->status & ERR_CORRUPT)) return;
  const uint32_t b = blockIdx.x;
  uint32_t org[3], w[3];
  block_box(a.g, b, org, w);
  const uint32_t m = w[0] * w[1] * w[2];
  const int32_t r = (int32_t)a.radius;
  int32_t* q = reinterpret_cast<int32_t*>(a.out);
  const uint16_t* codes = a.codes + (uint64_t)b * kSlots;
  const uint64_t ny = a.g.n[1], nx = a.g.n[2];
  auto elem = [&](uint32_t j) -> uint64_t {
    const uint32_t pl = w[1] * w[2], zz = j / pl, rr = j - zz * pl, yy = rr / w[2], xx = rr - yy * w[2];
    return ((uint64_t)(org[0] + zz) * ny + (org[1] + yy)) * nx + org[2] + xx;
  };
  for (uint32_t j = threadIdx.x; j < m; j += kRecThreads) q[elem(j)] = (int32_t)codes[j] - r;
  __syncthreads();  // orders the outliers' writes after the codes' writes
  const uint2* rec = reinterpret_cast<const uint2*>(a.ar + a.off_rec);
  for (uint32_t i = a.rec_start[b] + threadIdx.x; i < a.rec_start[b + 1]; i += kRecThreads) {
    const uint2 kv = rec[i];
    if ((kv.x & 1u) == 0) q[elem((kv.x >> 1) % kSlots)] = (int32_t)kv.y;
  }
}

// Exclusive prefix, for a segmented scan, of the tiles before `tile`: the aggregates
// back to the nearest tile that published an inclusive value (a tile holding a segment
// start), summed modulo 2^62 and read back as a signed value.  One full warp calls;
// the wait is bounded (ERR_TIMEOUT and 0 on expiry).
__device__ int64_t seg_lookback_warp(const uint64_t* state, uint32_t tile, uint32_t* status, uint32_t spin_limit) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) return 0;
  uint64_t excl = 0;
  int64_t base = (int64_t)tile - 1;
  uint32_t spins = 0;
  while (true) {
    const int64_t idx = base - lane;
    const uint64_t v = idx >= 0 ? ld_relaxed(&state[idx]) : LB_INC;
    const uint32_t inc = __ballot_sync(~0u, (v & LB_INC) != 0);
    const uint32_t bad = __ballot_sync(~0u, (v & (LB_INC | LB_AGG)) == 0);
    const int first = inc ? __ffs(inc) : 32;
    const uint32_t upto = first >= 32 ? ~0u : ((1u << first) - 1u);
    if (bad & upto) {
      if (++spins > spin_limit) {
        if (lane == 0) atomicOr(status, ERR_TIMEOUT);
        return 0;
      }
      __nanosleep(64);
      continue;
    }
    const uint64_t add = warp_sum(((1u << lane) & upto) ? (v & LB_VAL) : 0ull);
    excl = (excl + add) & LB_VAL;
    if (inc) break;
    base -= 32;
  }
  return (int64_t)(excl << 2) >> 2;
}

__device__ __forceinline__ void seg_publish(uint64_t* state, uint32_t tile, bool inclusive, int64_t v) {
  st_relaxed(&state[tile], (inclusive ? LB_INC : LB_AGG) | ((uint64_t)v & LB_VAL));
}

// Pass along x: an inclusive scan of the flattened field restarted at every row start
// (a segment of n[2] elements), one tile of 4096 elements per CTA in ticket order;
// tiles chain their carries by decoupled look-back.  `last`: scale to FP32 in place.
__global__ __launch_bounds__(256) void gscan_x_kernel(DecodeArgs a, uint64_t* state, int last) {
  __shared__ uint32_t s_tile;
  __shared__ int s_go;
  __shared__ int s_wf[8];
  __shared__ int32_t s_ws[8];
  __shared__ int32_t s_carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    s_go = !(a.st->status & ERR_CORRUPT);
    s_tile = atomicAdd(&a.st->ticket_construct, 1u);
  }
  __syncthreads();
  if (!s_go) return;  // every CTA leaves: no tile waits on another
  const uint32_t tile = s_tile;
  const uint64_t n = a.g.nelem, seg = a.g.n[2];
  int32_t* q = reinterpret_cast<int32_t*>(a.out);
  const uint64_t base = (uint64_t)tile * kScanTile + 16u * tid;
  int32_t v[16];
  uint32_t heads = 0;
  uint64_t rpos = base % seg;
#pragma unroll
  for (int i = 0; i < 16; i++) {
    const uint64_t idx = base + i;
    v[i] = idx < n ? q[idx] : 0;
    if (idx < n && rpos == 0) heads |= 1u << i;
    rpos = rpos + 1 == seg ? 0 : rpos + 1;
  }
  // the thread's own segmented inclusive scan, and its pair (head seen, sum since it)
  bool f = false;
  int32_t run = 0;
#pragma unroll
  for (int i = 0; i < 16; i++) {
    if ((heads >> i) & 1u) {
      run = v[i];
      f = true;
    } else {
      run += v[i];
    }
    v[i] = run;
  }
  // warp scan of the pairs (combine a then b: (fa | fb, fb ? sb : sa + sb))
  bool F = f;
  int32_t S = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const bool fu = __shfl_up_sync(~0u, (int)F, o) != 0;
    const int32_t su = __shfl_up_sync(~0u, S, o);
    if (lane >= o) {
      if (!F) S += su;
      F = F || fu;
    }
  }
  bool Fe = __shfl_up_sync(~0u, (int)F, 1) != 0;
  int32_t Se = __shfl_up_sync(~0u, S, 1);
  if (lane == 0) {
    Fe = false;
    Se = 0;
  }
  if (lane == 31) {
    s_wf[wid] = F;
    s_ws[wid] = S;
  }
  __syncthreads();
  bool Fw = false;
  int32_t Sw = 0;
  for (int ww = 0; ww < wid; ww++) {
    Sw = s_wf[ww] ? s_ws[ww] : Sw + s_ws[ww];
    Fw = Fw || s_wf[ww];
  }
  const bool Ft = Fw || Fe;               // a segment starts before this thread, in the tile
  const int32_t St = Fe ? Se : Sw + Se;   // and the sum since the latest such start
  if (wid == 0) {
    bool TF = false;
    int32_t TS = 0;
    for (int ww = 0; ww < 8; ww++) {
      TS = s_wf[ww] ? s_ws[ww] : TS + s_ws[ww];
      TF = TF || s_wf[ww];
    }
    if (lane == 0) seg_publish(state, tile, TF, TS);  // a tile with a segment start needs no carry
    int64_t c = 0;
    if ((uint64_t)tile * kScanTile % seg != 0) c = seg_lookback_warp(state, tile, &a.st->status, kSpinLimit);
    if (lane == 0) {
      if (!TF) seg_publish(state, tile, true, c + TS);
      s_carry = (int32_t)c;
    }
  }
  __syncthreads();
  const int32_t pre = Ft ? St : s_carry + St;  // what precedes the thread's first element
  const float ebx2 = a.ebx2_f;
  float* out = a.out;
#pragma unroll
  for (int i = 0; i < 16; i++) {
    const uint64_t idx = base + i;
    // elements before the thread's first head add what precedes the thread
    const bool own = (heads & ((2u << i) - 1u)) != 0;
    const int32_t k = own ? v[i] : pre + v[i];
    if (idx < n) {
      if (last) out[idx] = scale(k, ebx2);
      else q[idx] = k;
    }
  }
}

// Pass along y (or z): thread (outer, x) runs down its column; `last`: scale in place.
__global__ __launch_bounds__(256) void gscan_col_kernel(DecodeArgs a, int axis, int last) {
  if (a.dead || (a.st->status & ERR_CORRUPT)) return;
  const uint64_t nz = a.g.n[0], ny = a.g.n[1], nx = a.g.n[2];
  // axis 1 (y): columns (z, x), stride nx, length ny; axis 0 (z): columns (y, x), stride ny nx, length nz
  const uint64_t ncol = axis == 1 ? nz * nx : ny * nx;
  const uint64_t c = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (c >= ncol) return;
  const uint64_t stride = axis == 1 ? nx : ny * nx, len = axis == 1 ? ny : nz;
  const uint64_t start = axis == 1 ? (c / nx) * ny * nx + c % nx : c;
  int32_t* q = reinterpret_cast<int32_t*>(a.out);
  float* out = a.out;
  const float ebx2 = a.ebx2_f;
  int32_t acc = 0;
  uint64_t i = 0;
  for (; i + 4 <= len; i += 4) {
    int32_t t[4];
#pragma unroll
    for (int u = 0; u < 4; u++) t[u] = q[start + (i + u) * stride];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      acc += t[u];
      if (last) out[start + (i + u) * stride] = scale(acc, ebx2);
      else q[start + (i + u) * stride] = acc;
    }
  }
  for (; i < len; i++) {
    acc += q[start + i * stride];
    if (last) out[start + i * stride] = scale(acc, ebx2);
    else q[start + i * stride] = acc;
  }
}

// Verbatim patches (after the last pass).
__global__ void gpatch_kernel(DecodeArgs a) {
  if (a.dead || (a.st->status & ERR_CORRUPT)) return;
  const uint2* rec = reinterpret_cast<const uint2*>(a.ar + a.off_rec);
  const uint64_t ny = a.g.n[1], nx = a.g.n[2];
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < a.n_rec; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint2 kv = rec[i];
    if ((kv.x & 1u) == 0) continue;
    const uint32_t slot = kv.x >> 1, b = slot / kSlots, j = slot % kSlots;
    uint32_t org[3], w[3];
    block_box(a.g, b, org, w);
    const uint32_t pl = w[1] * w[2], zz = j / pl, rr = j - zz * pl, yy = rr / w[2], xx = rr - yy * w[2];
    a.out[((uint64_t)(org[0] + zz) * ny + (org[1] + yy)) * nx + org[2] + xx] = __uint_as_float(kv.y);
  }
}

// The global reconstruction's launches (after set-up, decoding and run expansion).
cudaError_t launch_global_reconstruct(const DecodeArgs& a, cudaStream_t s) {
  trace_begin(K_RECONSTRUCT, s);
  gfuse_kernel<<<a.g.nblk, kRecThreads, 0, s>>>(a);
  const int nd = a.g.ndim;
  const uint64_t ntiles = (a.g.nelem + kScanTile - 1) / kScanTile;
  gscan_x_kernel<<<(unsigned)ntiles, 256, 0, s>>>(a, a.scan_state, nd == 1 ? 1 : 0);
  if (nd >= 2) {
    const uint64_t cy = (uint64_t)a.g.n[0] * a.g.n[2];
    gscan_col_kernel<<<(unsigned)((cy + 255) / 256), 256, 0, s>>>(a, 1, nd == 2 ? 1 : 0);
  }
  if (nd == 3) {
    const uint64_t cz = (uint64_t)a.g.n[1] * a.g.n[2];
    gscan_col_kernel<<<(unsigned)((cz + 255) / 256), 256, 0, s>>>(a, 0, 1);
  }
  if (a.n_rec) gpatch_kernel<<<(unsigned)((a.n_rec + 255) / 256 < 1024 ? (a.n_rec + 255) / 256 : 1024), 256, 0, s>>>(a);
  trace_end(K_RECONSTRUCT, s);
  return cudaGetLastError();
}

// =================================================================================
// batches: device-side header checks and table-driven launches
// =================================================================================
__device__ __forceinline__ uint64_t dev_a8(uint64_t v) { return (v + 7) & ~7ull; }

// Reads field f's archive header on the device, checks it against the shape the
// batch was planned for (the same checks the single-field entry makes on the host)
// and completes the field's decode arguments; a failing header marks the field
// dead (every later stage skips it) and corrupt.
__global__ void dec_header_batch_kernel(DecodeArgs* tasks, int nfields) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nfields) return;
  DecodeArgs& a = tasks[f];
  const Geom& g = a.g;
  bool ok = a.bytes >= (uint64_t)kHdr;
  uint64_t n_rec = 0, n_out = 0, n_patch = 0, payload = 0, total = 0, nblk = 0, dims[3] = {0, 0, 0};
  uint32_t magic = 0, radius = 0, lanes = 0, flags = 0;
  uint16_t version = 0;
  uint8_t ndim = 0, mode = 0;
  float eb_f = 0.0f;
  if (ok) {
    const uint8_t* h = a.ar;
    memcpy(&magic, h, 4);
    memcpy(&version, h + 4, 2);
    ndim = h[6];
    mode = h[7];
    memcpy(dims, h + 8, 24);
    memcpy(&eb_f, h + 48, 4);
    memcpy(&radius, h + 52, 4);
    memcpy(&lanes, h + 56, 4);
    memcpy(&flags, h + 60, 4);
    memcpy(&nblk, h + 64, 8);
    memcpy(&n_rec, h + 72, 8);
    memcpy(&n_out, h + 80, 8);
    memcpy(&n_patch, h + 88, 8);
    memcpy(&payload, h + 96, 8);
    memcpy(&total, h + 104, 8);
    memcpy(a.n_codec, h + 116, 12);
    ok = magic == kMagic && version == kVersion && ndim == g.ndim && mode <= 1;
    for (int d = 0; d < 3 && ok; d++) {
      const uint64_t want = d < g.ndim ? (uint64_t)g.n[3 - g.ndim + d] : 0ull;
      ok = dims[d] == want;
    }
    ok = ok && radius >= 1 && radius <= 512 && lanes == (uint32_t)kLanes && flags <= 3;
    ok = ok && nblk == g.nblk && n_rec == n_out + n_patch && eb_f > 0.0f && isfinite(2.0f * eb_f);
    ok = ok && n_rec <= 2 * g.nelem && payload <= a.bytes && (payload & 3) == 0;
    const uint64_t off_bb = kHdr + dev_a8(g.nblk);
    const uint64_t off_rec = off_bb + dev_a8(4ull * g.nblk);
    const uint64_t off_books = off_rec + 8 * n_rec + dev_a8(payload);
    const uint64_t want_total = off_books + ((flags & 1) ? kNsymCode : 0) + ((flags & 2) ? kNsymCode + kNsymLen : 0);
    ok = ok && total == want_total && total <= a.bytes;
    if (ok) {
      a.off_codec = kHdr;
      a.off_bb = off_bb;
      a.off_rec = off_rec;
      a.off_pay = off_rec + 8 * n_rec;
      a.off_books = off_books;
      a.n_rec = n_rec;
      a.payload = payload;
      a.flags = flags;
      a.radius = radius;
      a.ebx2_f = 2.0f * eb_f;
    }
  }
  a.dead = ok ? 0 : 1;
  if (!ok) atomicOr(&a.st->status, ERR_CORRUPT);
}

__device__ __forceinline__ int field_of(const uint32_t* prefix, int nfields, uint32_t c) {
  int lo = 0, hi = nfields - 1;  // last field with prefix[f] <= c
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// set-up: per field its prep chunks (one CTA per 1024 blocks, chained by look-back),
// 3 table CTAs, then its record CTAs (setup0 prefix)
__global__ __launch_bounds__(1024) void dec_setup_batch_kernel(const DecodeArgs* __restrict__ tasks,
                                                               const uint32_t* __restrict__ setup0, int nfields) {
  const int f = field_of(setup0, nfields, blockIdx.x);
  const DecodeArgs& a = tasks[f];
  const uint32_t role = blockIdx.x - setup0[f], nroles = setup0[f + 1] - setup0[f];
  const uint32_t nprep = (a.g.nblk + 1023) / 1024;
  if (role < nprep) dec_prep_chunk_body(a, nprep);
  else if (role < nprep + 3) dec_tables_body(a, (int)(role - nprep));
  else dec_records_body(a, role - nprep - 3, nroles - nprep - 3);
}

// entropy decoding: per field ceil(nblk / (W / 2)) CTAs of W warps (W = blockDim.x / 32,
// chosen by the batch's tuner: 8, 16 or 32), one stream per warp; ND != 0 (the
// batch's common dimensionality): full Huffman blocks reconstructed in the decoding
// warps, as for single fields
template <int ND>
__global__ __launch_bounds__(1024) void stream_decode_batch_kernel(const DecodeArgs* __restrict__ tasks,
                                                                   const uint32_t* __restrict__ chunk0, int nfields) {
  const int f = field_of(chunk0, nfields, blockIdx.x);
  const DecodeArgs& a = tasks[f];
  const uint32_t per = kDecChunkRounds * (blockDim.x / 64);  // blocks per CTA: two streams each
  const uint32_t b0 = (blockIdx.x - chunk0[f]) * per;
  const uint32_t b1 = min(a.g.nblk, b0 + per);
  stream_decode_body<ND, float>(a, b0, b1);
}

// Reconstruction of a batch, one CTA per codec block of every field.  A run block's
// runs are expanded here, into shared memory, instead of by a separate launch: the
// expansion's scratch then serves as the reconstruction's (s_q overlays the run
// values and lengths, read no more once the codes are out).
__global__ __launch_bounds__(kRecThreads) void reconstruct_batch_kernel(const DecodeArgs* __restrict__ tasks,
                                                                        const uint32_t* __restrict__ tile0, int nfields) {
  static_assert(kRecThreads == kRleThreads, "run expansion assumes its CTA size");
  __shared__ __align__(16) uint32_t s_scr[kSlots + (kSlots + 1) + 3];  // run values and lengths, then starts
  __shared__ __align__(16) uint16_t s_codes[kSlots];
  __shared__ int s_go;
  int32_t* s_q = reinterpret_cast<int32_t*>(s_scr);
  const int f = field_of(tile0, nfields, blockIdx.x);
  const DecodeArgs& a = tasks[f];
  const uint32_t b = blockIdx.x - tile0[f];
  if (a.dead) return;
  // full Huffman blocks were reconstructed by the decoding warps (fused batches)
  if (a.fuse && a.ar[a.off_codec + b] == CODEC_HUFF && block_is_full(a.g, b)) return;
  // the status is read once, by thread 0 (run expansions in other CTAs may flag
  // corruption meanwhile), so every thread takes the same path
  if (threadIdx.x == 0) s_go = !(a.st->status & ERR_CORRUPT);
  __syncthreads();
  if (!s_go) return;
  const int codec = a.ar[a.off_codec + b];
  const uint16_t* codes = a.codes + (uint64_t)b * kSlots;
  if (codec == CODEC_RLE || codec == CODEC_RLE_HUFF) {
    uint16_t* sv = reinterpret_cast<uint16_t*>(s_scr);
    if (!rle_expand_into(a, b, s_codes, sv, sv + kSlots, s_scr + kSlots)) return;
    __syncthreads();
    codes = s_codes;
  }
  if (a.g.ndim == 1) reconstruct_body<1, float>(a, b, s_q, codes);
  else if (a.g.ndim == 2) reconstruct_body<2, float>(a, b, s_q, codes);
  else reconstruct_body<3, float>(a, b, s_q, codes);
}

cudaError_t launch_decode_batch(const DecodeBatchLaunch& L, cudaStream_t s) {
  cudaError_t e;
  trace_begin(K_DEC_HEADER, s);
  dec_header_batch_kernel<<<(L.nfields + 127) / 128, 128, 0, s>>>(L.tasks, L.nfields);
  trace_end(K_DEC_HEADER, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  trace_begin(K_DEC_SETUP, s);
  dec_setup_batch_kernel<<<L.nsetup, 1024, 0, s>>>(L.tasks, L.setup0, L.nfields);
  trace_end(K_DEC_SETUP, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int warps = L.warps ? L.warps : kStreamWarps;
  const size_t smem = 3 * (1u << kLutBits) * sizeof(LutEntry) + (L.nd ? (size_t)warps * kRecTabWords * 4 : 0);
  auto k = L.nd == 1 ? stream_decode_batch_kernel<1>
                     : (L.nd == 2 ? stream_decode_batch_kernel<2>
                                  : (L.nd == 3 ? stream_decode_batch_kernel<3> : stream_decode_batch_kernel<0>));
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  trace_begin(K_STREAM_DECODE, s);
  k<<<L.nchunks, 32 * warps, smem, s>>>(L.tasks, L.chunk0, L.nfields);
  trace_end(K_STREAM_DECODE, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // (run blocks are expanded inside the reconstruction)
  trace_begin(K_RECONSTRUCT, s);
  reconstruct_batch_kernel<<<L.ntiles, kRecThreads, 0, s>>>(L.tasks, L.tile0, L.nfields);
  trace_end(K_RECONSTRUCT, s);
  return cudaGetLastError();
}

// One bounded wait that nothing satisfies (a test aid for the failure path): which 0,
// the payload look-back of tile 1 behind a tile 0 that never publishes; which 1, an
// mbarrier phase no copy or arrival completes.  Either gives up after `spin_limit`
// tries and leaves ERR_TIMEOUT in the status, and the kernel returns normally.
__global__ void wait_selftest_kernel(int which, uint32_t spin_limit, uint64_t* lb, DevState* st) {
  __shared__ unsigned long long s_bar;
  if (which == 0) {
    if (threadIdx.x < 32) lookback_warp(lb, 1, 5, &st->status, spin_limit);
  } else if (which == 2) {
    // a field hand-over of the batched persistent kernel that no producer releases
    if (threadIdx.x == 0 && !wait_ge_acquire(&st->tiles_flushed, 1u, spin_limit)) atomicOr(&st->status, ERR_TIMEOUT);
  } else if (threadIdx.x == 0) {
    mbar_init(&s_bar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&s_bar, 0, spin_limit)) atomicOr(&st->status, ERR_TIMEOUT);
  }
}

cudaError_t launch_wait_selftest(int which, uint32_t spin_limit, uint64_t* lb, DevState* st, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(which, spin_limit, lb, st);
  return cudaGetLastError();
}

__global__ void dec_status_kernel(const DevState* st, uint32_t* d_status) {
  *d_status = (uint32_t)fold(st->status);
}

cudaError_t launch_dec_status(const DevState* st, uint32_t* d_status, cudaStream_t s) {
  trace_begin(K_DEC_STATUS, s);
  dec_status_kernel<<<1, 1, 0, s>>>(st, d_status);
  trace_end(K_DEC_STATUS, s);
  return cudaGetLastError();
}

// The entropy decoding and reconstruction launches of one field, for element type E.
template <typename E>
cudaError_t launch_decode_stages(const DecodeArgs& a, cudaStream_t s) {
  const int nd = a.g.ndim;
  const int nluts = ((a.flags & 1u) ? 1 : 0) + ((a.flags & 2u) ? 2 : 0);
  if (nluts) {
    const size_t lut_bytes =
        (size_t)nluts * (1u << kLutBits) * sizeof(LutEntry) + (size_t)kStreamWarps * kRecTabWords * 4;
    static int sms = 0, occ[4][4] = {};
    auto k = nd == 1 ? stream_decode_kernel<1, E> : (nd == 2 ? stream_decode_kernel<2, E> : stream_decode_kernel<3, E>);
    if (sms == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      for (auto kk : {stream_decode_kernel<1, E>, stream_decode_kernel<2, E>, stream_decode_kernel<3, E>})
        cudaFuncSetAttribute(kk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(3 * (1u << kLutBits) * sizeof(LutEntry) + kStreamWarps * kRecTabWords * 4));
    }
    if (occ[nd][nluts] == 0) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[nd][nluts], k, 32 * kStreamWarps, lut_bytes);
      if (occ[nd][nluts] <= 0) occ[nd][nluts] = 1;
    }
    const uint64_t want = (2ull * a.g.nblk + kStreamWarps - 1) / kStreamWarps;
    const uint64_t cap = (uint64_t)sms * occ[nd][nluts];
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    trace_begin(K_STREAM_DECODE, s);
    k<<<grid, 32 * kStreamWarps, lut_bytes, s>>>(a);
    trace_end(K_STREAM_DECODE, s);
  }
  if (a.n_codec[CODEC_RLE] + a.n_codec[CODEC_RLE_HUFF]) {  // run blocks present
    trace_begin(K_RLE_EXPAND, s);
    rle_expand_kernel<<<a.n_codec[CODEC_RLE] + a.n_codec[CODEC_RLE_HUFF], kRleThreads, 0, s>>>(a);
    trace_end(K_RLE_EXPAND, s);
  }
  if (a.global) return launch_global_reconstruct(a, s);
  // blocks left to the reconstruction kernel: with fusion at most the edge blocks and
  // the run blocks (the header's counts, which the set-up checks); none, and the launch
  // is skipped
  uint64_t work = a.g.nblk;
  if (a.fuse) {
    uint64_t full = 1;
    for (int d = 0; d < 3; d++) full *= a.g.n[d] / a.g.blk[d];
    work = (a.g.nblk - full) + a.n_codec[CODEC_RLE] + a.n_codec[CODEC_RLE_HUFF];
    if (work > a.g.nblk) work = a.g.nblk;
  }
  if (work) {
    static int sms = 0, occ[4] = {0, 0, 0, 0};
    auto k = nd == 1 ? reconstruct_kernel<1, E> : (nd == 2 ? reconstruct_kernel<2, E> : reconstruct_kernel<3, E>);
    if (sms == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (occ[nd] == 0) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[nd], k, kRecThreads, 0);
      if (occ[nd] <= 0) occ[nd] = 1;
    }
    // persistent only when every CTA gets several blocks to prefetch
    const uint64_t cap = (uint64_t)sms * occ[nd];
    const unsigned grid = (unsigned)(work <= 3 * cap ? work : cap);
    trace_begin(K_RECONSTRUCT, s);
    k<<<grid, kRecThreads, 0, s>>>(a);
    trace_end(K_RECONSTRUCT, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_decode(const DecodeArgs& a, cudaStream_t s) {
  const uint64_t n = (a.n_rec > (uint64_t)a.g.nblk + 1 ? a.n_rec : (uint64_t)a.g.nblk + 1);
  uint64_t rec_ctas = (n + 1023) / 1024;
  if (rec_ctas > 1024) rec_ctas = 1024;
  const uint32_t nchunks = (a.g.nblk + 1023) / 1024;
  trace_begin(K_DEC_SETUP, s);
  dec_setup_kernel<<<(unsigned)(nchunks + 3 + rec_ctas), 1024, 0, s>>>(a, nchunks);
  trace_end(K_DEC_SETUP, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return a.f64 ? launch_decode_stages<double>(a, s) : launch_decode_stages<float>(a, s);
}

}  // namespace cszp
