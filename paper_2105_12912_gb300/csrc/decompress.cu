// Decompression kernels of cszp (sm_103a).
//
//   dec_setup_kernel       codec / block-size validation and payload offsets (scan),
//                          decode tables + 12-bit lookup table per book, record
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
  // payload offsets and, packed above bit 48 of the same scan, the list of run blocks
  constexpr uint64_t kLow = (1ull << 48) - 1;
  uint64_t carry = 0, rcarry = 0;
  bool bad = false;
  for (uint32_t base = 0; base < a.g.nblk; base += blockDim.x) {
    const uint32_t b = base + tid;
    uint64_t bb = 0;
    bool run = false;
    if (b < a.g.nblk) {
      const uint32_t c = a.ar[a.off_codec + b];
      bb = reinterpret_cast<const uint32_t*>(a.ar + a.off_bb)[b];
      if (c > 2 || (bb & 3)) bad = true;
      else atomicAdd(&s_nc[c], 1u);
      run = c == CODEC_RLE || c == CODEC_RLE_HUFF;
    }
    uint64_t tot;
    const uint64_t ex = block_excl_scan<uint64_t>(bb | ((uint64_t)run << 48), s_scan, &tot);
    if (b < a.g.nblk) a.blk_off[b] = carry + (ex & kLow);
    if (run && a.runblk) a.runblk[rcarry + (ex >> 48)] = b;
    carry += tot & kLow;
    rcarry += tot >> 48;
  }
  if (tid == 0) {
    a.blk_off[a.g.nblk] = carry;
    if (carry != a.payload) bad = true;
    if ((s_nc[CODEC_HUFF] && !(a.flags & 1u)) || (s_nc[CODEC_RLE_HUFF] && !(a.flags & 2u))) bad = true;
    for (int c = 0; c < 3; c++)
      if (s_nc[c] != a.n_codec[c]) bad = true;  // the header's counts decide which kernels run
  }
  if (bad) flag(a.st, ERR_CORRUPT);
}

__device__ void dec_records_body(const DecodeArgs& a, uint32_t cta, uint32_t nctas) {
  if (a.dead) return;
  const uint32_t* rec = reinterpret_cast<const uint32_t*>(a.ar + a.off_rec);
  const uint64_t nslots = (uint64_t)a.g.nblk * kSlots;
  const uint64_t n = a.n_rec > (uint64_t)a.g.nblk + 1 ? a.n_rec : (uint64_t)a.g.nblk + 1;
  for (uint64_t i = cta * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)nctas * blockDim.x) {
    if (i < a.n_rec) {
      const uint32_t key = rec[2 * i];
      bool bad = (i + 1 < a.n_rec) && key >= rec[2 * (i + 1)];
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
// 12-bit lookup table.
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
  // lookup: for each 12-bit prefix, the shortest matching code of length <= 12
  for (int v = tid; v < (1 << kLutBits); v += blockDim.x) {
    uint32_t e = 0;
    for (int l = 1; l <= kLutBits; l++) {
      const uint64_t c = (uint64_t)(v >> (kLutBits - l));
      if (cs.cnt[l] && c >= cs.first[l] && c - cs.first[l] < cs.cnt[l]) {
        e = ((uint32_t)t->sorted[cs.off[l] + (uint32_t)(c - cs.first[l])] << 8) | (uint32_t)l;
        break;
      }
    }
    t->lut[v] = e;
  }
}

// One launch for archive set-up: CTA 0 validates codecs and scans block sizes, CTAs
// 1-3 build the decode tables of the three books, the rest validate records and find
// each block's first record.
__global__ __launch_bounds__(1024) void dec_setup_kernel(DecodeArgs a) {
  if (blockIdx.x == 0) {
    dec_prep_body(a);
  } else if (blockIdx.x <= 3) {
    dec_tables_body(a, (int)blockIdx.x - 1);
  } else {
    dec_records_body(a, blockIdx.x - 4, gridDim.x - 4);
  }
}

// =================================================================================
// interleaved Huffman streams: one warp decodes one stream (see common.cuh)
// =================================================================================
struct BookView {
  const uint32_t* lut;  // 1 << kLutBits entries
  const unsigned long long* first;
  const unsigned long long* limit;
  const uint32_t* count;
  const uint32_t* off;
  const uint16_t* sorted;
  int maxlen;
  unsigned long long fullmask;
};

// Length of the codeword that is a prefix of the nb valid top bits of bb (0 if none
// fits in nb bits), and its symbol.  Short codes come from the lookup table; longer
// ones from the smallest length whose left-justified end exceeds bb, which is the
// true length whenever it is <= nb (zero bits below nb cannot complete a shorter
// codeword).
__device__ __forceinline__ int ihs_match(uint64_t bb, int nb, const BookView& bk, int& sym) {
  if (nb <= 0) return 0;
  const uint32_t e = bk.lut[bb >> (64 - kLutBits)];
  const int l = (int)(e & 0xffu);
  if (l) {
    if (l <= nb) {
      sym = (int)(e >> 8);
      return l;
    }
    return 0;
  }
  if (nb <= kLutBits) return 0;
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

// One warp decodes N symbols (+add) from in[0..avail) into out[].  Returns false
// (warp-uniform) if the stream is damaged; *used gets the units read.
// The warp reads the stream strictly in order, so the next 96 units are kept in three
// 32-unit register windows (lane i holds unit base+i of each); a top-up takes its unit
// from a window by shuffle and a window is reloaded (one 64-byte load) two windows
// before it is needed, so no load sits on the decode's critical path.
__device__ bool ihs_decode_warp(const uint16_t* __restrict__ in, uint32_t avail, uint32_t N,
                                const BookView& bk, uint16_t* out, int add, uint32_t* used) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t T = (N + 31) / 32;
  auto fetch = [&](uint32_t i) -> uint32_t { return i < avail ? (uint32_t)__ldg(&in[i]) : 0u; };
  uint32_t w0 = fetch(lane), w1 = fetch(32 + lane), w2 = fetch(64 + lane);
  uint32_t wbase = 0;  // stream index of w0's lane 0
  uint64_t bb = 0;
  int nb = 0;
  uint32_t cur = 0;
  bool bad = false;
  for (uint32_t t = 0; t < T; t++) {
    const bool active = 32 * t + lane < N && !bad;
    int sym = 0, ml = active ? ihs_match(bb, nb, bk, sym) : 0;
    bool need = active && ml == 0;
    uint32_t ballot;
    while ((ballot = __ballot_sync(~0u, need)) != 0u) {
      const uint32_t pos = cur + __popc(ballot & ((1u << lane) - 1u));
      const uint32_t rel = pos - wbase;  // < 64 while cur - wbase < 32
      const uint32_t u0 = __shfl_sync(~0u, w0, rel & 31);
      const uint32_t u1 = __shfl_sync(~0u, w1, rel & 31);
      if (need) {
        if (nb > 64 - 16 || pos >= avail) {
          bad = true;
          need = false;
        } else {
          bb |= (uint64_t)(rel < 32 ? u0 : u1) << (48 - nb);
          nb += 16;
          ml = ihs_match(bb, nb, bk, sym);  // only lanes that took a unit look again
          need = ml == 0;
        }
      }
      cur += __popc(ballot);
      if (cur - wbase >= 32) {
        w0 = w1;
        w1 = w2;
        wbase += 32;
        w2 = fetch(wbase + 64 + lane);
      }
    }
    if (active && !bad) {
      out[32 * t + lane] = (uint16_t)(sym + add);
      bb = ml >= 64 ? 0ull : bb << ml;
      nb -= ml;
    }
  }
  *used = cur;
  return !__any_sync(~0u, bad);
}

constexpr int kStreamWarps = kStreamWarpsPerCta;

// Entropy decoding, persistent: each CTA stages the lookup tables of the books the
// archive uses in shared memory once, then its warps take codec blocks from a ticket;
// a warp decodes a Huffman block's code stream, or an RLE+Huffman block's value
// stream and then its length stream (runs go to the workspace run arrays).
// Blocks come from the field's ticket (b_end == 0) or, in batches, warp i of the
// CTA takes block b_begin + i if below b_end.
__device__ void stream_decode_body(const DecodeArgs& a, uint32_t b_begin, uint32_t b_end) {
  extern __shared__ __align__(16) uint32_t s_luts[];  // the present books' tables
  __shared__ unsigned long long s_first[kMaxLen + 1], s_limit[kMaxLen + 1];
  __shared__ uint32_t s_off[kMaxLen + 1], s_count[kMaxLen + 1];
  __shared__ int s_go;
  if (a.dead) return;
  // the status is read once, by thread 0, and acted on after the staging barrier, so
  // that a corruption flagged by another CTA meanwhile cannot split this CTA
  if (threadIdx.x == 0) s_go = !(a.st->status & ERR_CORRUPT);
  const bool huff = (a.flags & 1u) != 0, rle = (a.flags & 2u) != 0;
  uint32_t* lut_code = s_luts;
  uint32_t* lut_val = s_luts + (huff ? (1 << kLutBits) : 0);
  uint32_t* lut_len = lut_val + (1 << kLutBits);
  // a chunk of blocks (batches) copies only the tables its own blocks use
  bool need_code = huff, need_runs = rle;
  if (b_end != 0) {
    const uint32_t b = b_begin + threadIdx.x;
    const int c = (b < b_end) ? a.ar[a.off_codec + b] : -1;
    need_code = __syncthreads_or(huff && c == CODEC_HUFF) != 0;
    need_runs = __syncthreads_or(rle && c == CODEC_RLE_HUFF) != 0;
  }
  for (int i = threadIdx.x; i < (1 << kLutBits); i += blockDim.x) {
    if (need_code) lut_code[i] = a.tabs[0].lut[i];
    if (need_runs) {
      lut_val[i] = a.tabs[1].lut[i];
      lut_len[i] = a.tabs[2].lut[i];
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
  for (uint32_t round = 0;; round++) {
    uint32_t slot = 0;
    if (ticketed) {
      if (lane0) slot = atomicAdd(&a.st->ticket_decode, 1u);
      slot = __shfl_sync(~0u, slot, 0);
      if (slot >= 2 * a.g.nblk) break;
    } else {
      slot = 2 * b_begin + (threadIdx.x >> 5);
      if (round > 0 || slot >= 2 * b_end) break;
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
      if (which == 0) {
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

__global__ __launch_bounds__(32 * kStreamWarps) void stream_decode_kernel(DecodeArgs a) {
  stream_decode_body(a, 0, 0);
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

__device__ __forceinline__ float scale(int32_t k, float ebx2) { return __fmul_rn(__int2float_rn(k), ebx2); }

// codes: the block's 4096 code slots (global memory, or a shared-memory copy)
template <int ND>
__device__ void reconstruct_body(const DecodeArgs& a, uint32_t b, int32_t* s_q, const uint16_t* codes) {
  // (the caller has checked the field's status, the same way in every thread)
  const int tid = threadIdx.x;
  uint32_t org[3], w[3];
  block_box(a.g, b, org, w);
  const uint32_t m = w[0] * w[1] * w[2];
  const int32_t r = (int32_t)a.radius;
  const float ebx2 = a.ebx2_f;
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
  float* __restrict__ out = a.out;
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
        if (j < m) __stcs(&out[(uint64_t)org[2] + j], scale(inc, ebx2));
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
        if (y < w[1]) __stcs(&out[base + (uint64_t)y * nx], scale(v[i], ebx2));
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
    for (int i = 0; i < 16; i++) __stcs(&out[base + (uint64_t)i * nx], scale(v[i], ebx2));
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
      __stcs(&out[((uint64_t)(org[0] + zz) * ny + (org[1] + yy)) * nx + org[2] + xx], scale(s_q[j], ebx2));
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
      out[((uint64_t)(org[0] + zz) * ny + (org[1] + yy)) * nx + org[2] + xx] = __uint_as_float(kv.y);
    }
  }
}

// Persistent: CTA c takes blocks c, c + grid, ...; while it reconstructs one, a bulk
// copy is already bringing the next block's 8 KB of codes into shared memory.
template <int ND>
__global__ __launch_bounds__(kRecThreads) void reconstruct_kernel(DecodeArgs a) {
  __shared__ __align__(128) uint16_t s_codes[2][kSlots];
  __shared__ __align__(16) int32_t s_q[kSlots];
  __shared__ unsigned long long s_bar[2];
  __shared__ uint32_t s_fail;
  if (a.dead || (a.st->status & ERR_CORRUPT)) return;
  const int tid = threadIdx.x;
  const uint32_t grid = gridDim.x;
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
    if (blockIdx.x < a.g.nblk) issue(blockIdx.x, 0);
  }
  __syncthreads();
  uint32_t it = 0, b = blockIdx.x;
  bool next_issued = false;
  for (; b < a.g.nblk; b += grid, it++) {
    const int cur = it & 1;
    next_issued = b + grid < a.g.nblk;
    if (tid == 0 && next_issued) issue(b + grid, cur ^ 1);
    if (!mbar_wait(&s_bar[cur], (it >> 1) & 1u, kSpinLimit)) {
      atomicOr(&a.st->status, ERR_TIMEOUT);
      s_fail = 1;
    }
    __syncthreads();
    if (s_fail) break;
    reconstruct_body<ND>(a, b, s_q, s_codes[cur]);
    __syncthreads();
  }
  if (s_fail && tid == 0) {
    // wait once more (bounded) for this block's copy and the next one in flight
    mbar_wait(&s_bar[it & 1], (it >> 1) & 1u, kSpinLimit);
    if (next_issued) mbar_wait(&s_bar[(it + 1) & 1], ((it + 1) >> 1) & 1u, kSpinLimit);
  }
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

// set-up: per field 1 prep CTA, 3 table CTAs, then its record CTAs (setup0 prefix)
__global__ __launch_bounds__(1024) void dec_setup_batch_kernel(const DecodeArgs* __restrict__ tasks,
                                                               const uint32_t* __restrict__ setup0, int nfields) {
  const int f = field_of(setup0, nfields, blockIdx.x);
  const DecodeArgs& a = tasks[f];
  const uint32_t role = blockIdx.x - setup0[f], nroles = setup0[f + 1] - setup0[f];
  if (role == 0) dec_prep_body(a);
  else if (role <= 3) dec_tables_body(a, (int)role - 1);
  else dec_records_body(a, role - 4, nroles - 4);
}

// entropy decoding: per field ceil(nblk / (kStreamWarps / 2)) CTAs, one stream per warp
__global__ __launch_bounds__(32 * kStreamWarps) void stream_decode_batch_kernel(const DecodeArgs* __restrict__ tasks,
                                                                                const uint32_t* __restrict__ chunk0,
                                                                                int nfields) {
  const int f = field_of(chunk0, nfields, blockIdx.x);
  const DecodeArgs& a = tasks[f];
  const uint32_t b0 = (blockIdx.x - chunk0[f]) * (kStreamWarps / 2);
  const uint32_t b1 = min(a.g.nblk, b0 + kStreamWarps / 2);
  stream_decode_body(a, b0, b1);
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
  if (a.g.ndim == 1) reconstruct_body<1>(a, b, s_q, codes);
  else if (a.g.ndim == 2) reconstruct_body<2>(a, b, s_q, codes);
  else reconstruct_body<3>(a, b, s_q, codes);
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
  const size_t lut_bytes = 3 * (1u << kLutBits) * sizeof(uint32_t);
  e = cudaFuncSetAttribute(stream_decode_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lut_bytes);
  if (e != cudaSuccess) return e;
  trace_begin(K_STREAM_DECODE, s);
  stream_decode_batch_kernel<<<L.nchunks, 32 * kStreamWarps, lut_bytes, s>>>(L.tasks, L.chunk0, L.nfields);
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

cudaError_t launch_decode(const DecodeArgs& a, cudaStream_t s) {
  const uint64_t n = (a.n_rec > (uint64_t)a.g.nblk + 1 ? a.n_rec : (uint64_t)a.g.nblk + 1);
  uint64_t rec_ctas = (n + 1023) / 1024;
  if (rec_ctas > 1024) rec_ctas = 1024;
  trace_begin(K_DEC_SETUP, s);
  dec_setup_kernel<<<(unsigned)(4 + rec_ctas), 1024, 0, s>>>(a);
  trace_end(K_DEC_SETUP, s);
  const int nluts = ((a.flags & 1u) ? 1 : 0) + ((a.flags & 2u) ? 2 : 0);
  if (nluts) {
    const size_t lut_bytes = (size_t)nluts * (1u << kLutBits) * sizeof(uint32_t);
    static int sms = 0, occ[4] = {0, 0, 0, 0};
    if (sms == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaFuncSetAttribute(stream_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(3 * (1u << kLutBits) * sizeof(uint32_t)));
    }
    if (occ[nluts] == 0) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[nluts], stream_decode_kernel, 32 * kStreamWarps, lut_bytes);
      if (occ[nluts] <= 0) occ[nluts] = 1;
    }
    const uint64_t want = (2ull * a.g.nblk + kStreamWarps - 1) / kStreamWarps;
    const uint64_t cap = (uint64_t)sms * occ[nluts];
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    trace_begin(K_STREAM_DECODE, s);
    stream_decode_kernel<<<grid, 32 * kStreamWarps, lut_bytes, s>>>(a);
    trace_end(K_STREAM_DECODE, s);
  }
  if (a.n_codec[CODEC_RLE] + a.n_codec[CODEC_RLE_HUFF]) {  // run blocks present
    trace_begin(K_RLE_EXPAND, s);
    rle_expand_kernel<<<a.n_codec[CODEC_RLE] + a.n_codec[CODEC_RLE_HUFF], kRleThreads, 0, s>>>(a);
    trace_end(K_RLE_EXPAND, s);
  }
  {
    static int sms = 0, occ[4] = {0, 0, 0, 0};
    auto k = a.g.ndim == 1 ? reconstruct_kernel<1> : (a.g.ndim == 2 ? reconstruct_kernel<2> : reconstruct_kernel<3>);
    if (sms == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    if (occ[a.g.ndim] == 0) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[a.g.ndim], k, kRecThreads, 0);
      if (occ[a.g.ndim] <= 0) occ[a.g.ndim] = 1;
    }
    // persistent only when every CTA gets several blocks to prefetch
    const uint64_t cap = (uint64_t)sms * occ[a.g.ndim];
    const unsigned grid = (unsigned)(a.g.nblk <= 3 * cap ? a.g.nblk : cap);
    trace_begin(K_RECONSTRUCT, s);
    k<<<grid, kRecThreads, 0, s>>>(a);
    trace_end(K_RECONSTRUCT, s);
  }
  return cudaGetLastError();
}

}  // namespace cszp
