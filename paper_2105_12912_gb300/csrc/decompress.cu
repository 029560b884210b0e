// Decompression kernels of cszp (sm_103a).
//
//   dec_prep_kernel        codec / block-size validation, payload offsets (scan)
//   dec_records_kernel     record validation, first record of every block
//   dec_tables_kernel      canonical decode tables + 12-bit lookup table per book
//   huff_decode_kernel     one thread per 1024-symbol Huffman segment
//   rle_decode_kernel      one CTA per RLE / RLE+Huffman block
//   reconstruct_kernel<ND> fuse outliers (q' = q - r, or delta), N-D partial sums
//                          per chunk (Alg. 1 l.9-13, Sec. IV-B2), scale by 2eb,
//                          verbatim patches
#include "common.cuh"
#include "kernels.h"

namespace cszp {

__device__ __forceinline__ void flag(DevState* st, uint32_t bits) { atomicOr(&st->status, bits); }

// =================================================================================
// archive validation and offsets
// =================================================================================
__global__ __launch_bounds__(1024) void dec_prep_kernel(DecodeArgs a) {
  __shared__ uint64_t s_scan[33];
  __shared__ uint32_t s_nc[3];
  const int tid = threadIdx.x;
  if (tid < 3) s_nc[tid] = 0;
  __syncthreads();
  uint64_t carry = 0;
  bool bad = false;
  for (uint32_t base = 0; base < a.g.nblk; base += blockDim.x) {
    const uint32_t b = base + tid;
    uint64_t bb = 0;
    if (b < a.g.nblk) {
      const uint32_t c = a.ar[a.off_codec + b];
      bb = reinterpret_cast<const uint32_t*>(a.ar + a.off_bb)[b];
      if (c > 2 || (bb & 3)) bad = true;
      else atomicAdd(&s_nc[c], 1u);
    }
    uint64_t tot;
    const uint64_t ex = block_excl_scan<uint64_t>(bb, s_scan, &tot);
    if (b < a.g.nblk) a.blk_off[b] = carry + ex;
    carry += tot;
  }
  if (tid == 0) {
    a.blk_off[a.g.nblk] = carry;
    if (carry != a.payload) bad = true;
    if ((s_nc[CODEC_HUFF] && !(a.flags & 1u)) || (s_nc[CODEC_RLE_HUFF] && !(a.flags & 2u))) bad = true;
  }
  if (bad) flag(a.st, ERR_CORRUPT);
}

__global__ void dec_records_kernel(DecodeArgs a) {
  const uint32_t* rec = reinterpret_cast<const uint32_t*>(a.ar + a.off_rec);
  const uint64_t nslots = (uint64_t)a.g.nblk * kSlots;
  const uint64_t n = a.n_rec > (uint64_t)a.g.nblk + 1 ? a.n_rec : (uint64_t)a.g.nblk + 1;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
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
__global__ __launch_bounds__(1024) void dec_tables_kernel(DecodeArgs a) {
  __shared__ uint8_t s_len[kNsymLen];
  __shared__ uint16_t s_wcnt[(kNsymLen / 32) * (kMaxLen + 1)];
  __shared__ CanonSmem cs;
  __shared__ uint32_t s_cnt[kMaxLen + 2];
  __shared__ uint32_t s_bad;
  const int book = blockIdx.x, tid = threadIdx.x;
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
  if (tid == 0) t->present = 1;
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

// =================================================================================
// canonical Huffman decoding
// =================================================================================
struct BitReader {
  const uint32_t* wp;
  uint32_t wleft;
  uint64_t bb;  // MSB-aligned bit buffer
  int nb;       // valid bits in bb
  __device__ __forceinline__ void refill() {
    while (nb <= 32 && wleft) {
      bb |= (uint64_t)(*wp++) << (32 - nb);
      nb += 32;
      wleft--;
    }
  }
};

// Decode one symbol; -1 when the stream ends or no code matches.
__device__ __forceinline__ int decode_one(BitReader& br, const uint32_t* lut, const unsigned long long* first,
                                          const uint32_t* count, const uint32_t* off,
                                          const uint16_t* sorted) {
  br.refill();
  if (br.nb == 0) return -1;
  const uint32_t e = lut[br.bb >> (64 - kLutBits)];
  const int l = (int)(e & 0xffu);
  if (l && l <= br.nb) {
    br.bb <<= l;
    br.nb -= l;
    return (int)(e >> 8);
  }
  uint64_t c = 0;
  for (int k = 1; k <= kMaxLen; k++) {
    if (br.nb == 0) {
      br.refill();
      if (br.nb == 0) return -1;
    }
    c = (c << 1) | (br.bb >> 63);
    br.bb <<= 1;
    br.nb--;
    if (count[k] && c >= first[k] && c - first[k] < count[k]) return (int)sorted[off[k] + (uint32_t)(c - first[k])];
  }
  return -1;
}

constexpr int kHuffDecThreads = 128;

__global__ __launch_bounds__(kHuffDecThreads) void huff_decode_kernel(DecodeArgs a) {
  __shared__ uint32_t s_lut[1 << kLutBits];
  __shared__ unsigned long long s_first[kMaxLen + 1];
  __shared__ uint32_t s_count[kMaxLen + 1], s_off[kMaxLen + 1];
  const DecTab* t = &a.tabs[0];
  if (!(a.flags & 1u) || (a.st->status & ERR_CORRUPT)) return;
  for (int i = threadIdx.x; i < (1 << kLutBits); i += blockDim.x) s_lut[i] = t->lut[i];
  for (int i = threadIdx.x; i <= kMaxLen; i += blockDim.x) {
    s_first[i] = t->first[i];
    s_count[i] = t->count[i];
    s_off[i] = t->off[i];
  }
  __syncthreads();
  if (!t->present) return;
  const uint64_t gid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint32_t b = (uint32_t)(gid >> 2), s = (uint32_t)(gid & 3);
  if (b >= a.g.nblk) return;
  if (a.ar[a.off_codec + b] != CODEC_HUFF) return;
  uint32_t org[3], w[3];
  block_box(a.g, b, org, w);
  const uint32_t m = w[0] * w[1] * w[2];
  const uint32_t S = (m + kHuffSeg - 1) / kHuffSeg;
  if (s >= S) return;
  const uint64_t bytes = a.blk_off[b + 1] - a.blk_off[b];
  const uint8_t* pay = a.ar + a.off_pay + a.blk_off[b];
  const uint32_t hdr = (2 * S + 3) & ~3u;
  if (hdr > bytes) {
    flag(a.st, ERR_CORRUPT);
    return;
  }
  const uint16_t* nw16 = reinterpret_cast<const uint16_t*>(pay);
  uint64_t w0 = hdr / 4, nwtot = hdr / 4;
  for (uint32_t k = 0; k < S; k++) {
    if (k < s) w0 += nw16[k];
    nwtot += nw16[k];
  }
  const uint32_t nw = nw16[s];
  if (4 * nwtot != bytes) {
    if (s == 0) flag(a.st, ERR_CORRUPT);
    return;
  }
  BitReader br{reinterpret_cast<const uint32_t*>(pay) + w0, nw, 0ull, 0};
  const uint32_t cnt = min((uint32_t)kHuffSeg, m - s * kHuffSeg);
  uint16_t* out = a.codes + (uint64_t)b * kSlots + s * kHuffSeg;
  const uint32_t lim = 2 * a.radius;
  uint32_t i = 0;
  for (; i + 8 <= cnt; i += 8) {
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const int sym = decode_one(br, s_lut, s_first, s_count, s_off, t->sorted);
      if (sym < 0 || (uint32_t)sym >= lim) {
        flag(a.st, ERR_CORRUPT);
        return;
      }
      if (k & 1) v[k >> 1] |= (uint32_t)sym << 16;
      else v[k >> 1] = (uint32_t)sym;
    }
    *reinterpret_cast<uint4*>(out + i) = make_uint4(v[0], v[1], v[2], v[3]);
  }
  for (; i < cnt; i++) {
    const int sym = decode_one(br, s_lut, s_first, s_count, s_off, t->sorted);
    if (sym < 0 || (uint32_t)sym >= lim) {
      flag(a.st, ERR_CORRUPT);
      return;
    }
    out[i] = (uint16_t)sym;
  }
}

constexpr int kRleThreads = 256;

__global__ __launch_bounds__(kRleThreads) void rle_decode_kernel(DecodeArgs a) {
  __shared__ uint16_t s_v[kSlots];
  __shared__ uint16_t s_l[kSlots];
  __shared__ uint32_t s_start[kSlots + 1];
  __shared__ uint32_t s_scan[33];
  __shared__ uint32_t s_nr, s_bad;
  const uint32_t b = blockIdx.x;
  const int tid = threadIdx.x;
  const int codec = a.ar[a.off_codec + b];
  if (codec != CODEC_RLE && codec != CODEC_RLE_HUFF) return;
  if (a.st->status & ERR_CORRUPT) return;
  uint32_t org[3], w[3];
  block_box(a.g, b, org, w);
  const uint32_t m = w[0] * w[1] * w[2];
  const uint64_t bytes = a.blk_off[b + 1] - a.blk_off[b];
  const uint8_t* pay = a.ar + a.off_pay + a.blk_off[b];
  const uint32_t lim = 2 * a.radius;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  if (codec == CODEC_RLE) {
    const uint64_t nr = bytes / 4;
    if (nr > m) {
      if (tid == 0) flag(a.st, ERR_CORRUPT);
      return;
    }
    const uint16_t* p16 = reinterpret_cast<const uint16_t*>(pay);
    for (uint32_t i = tid; i < nr; i += blockDim.x) {
      s_v[i] = p16[i];
      s_l[i] = p16[nr + i];
    }
    if (tid == 0) s_nr = (uint32_t)nr;
  } else {
    const uint32_t* p32 = reinterpret_cast<const uint32_t*>(pay);
    uint32_t nr = 0, vw = 0;
    if (bytes >= 8) {
      nr = p32[0];
      vw = p32[1];
    }
    if (bytes < 8 || nr > m || 8ull + 4ull * vw > bytes) {
      if (tid == 0) flag(a.st, ERR_CORRUPT);
      return;
    }
    const uint32_t lw = (uint32_t)((bytes - 8 - 4ull * vw) / 4);
    // values on warp 0 lane 0, lengths on warp 1 lane 0
    if (tid == 0 || tid == 32) {
      const DecTab* t = &a.tabs[tid == 0 ? 1 : 2];
      if (!t->present) {
        s_bad = 1;
      } else {
        BitReader br = tid == 0 ? BitReader{p32 + 2, vw, 0ull, 0} : BitReader{p32 + 2 + vw, lw, 0ull, 0};
        uint16_t* dst = tid == 0 ? s_v : s_l;
        for (uint32_t i = 0; i < nr; i++) {
          const int sym = decode_one(br, t->lut, t->first, t->count, t->off, t->sorted);
          if (sym < 0) {
            s_bad = 1;
            break;
          }
          dst[i] = (uint16_t)(tid == 0 ? sym : sym + 1);
        }
      }
    }
    if (tid == 0) s_nr = nr;
  }
  __syncthreads();
  const uint32_t nr = s_nr;
  // run starts by a block scan over contiguous shares of the runs
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
    return;
  }
  uint16_t* out = a.codes + (uint64_t)b * kSlots;
  for (uint32_t j = tid; j < m; j += blockDim.x) {
    uint32_t l = 0, h = nr;  // last run with start <= j
    while (h - l > 1) {
      const uint32_t mid = (l + h) >> 1;
      if (s_start[mid] <= j) l = mid;
      else h = mid;
    }
    out[j] = s_v[l];
  }
}

// =================================================================================
// reconstruction: N-D partial sums per chunk (Sec. IV-B2), scaled by 2eb
// =================================================================================
constexpr int kRecThreads = 256;

__device__ __forceinline__ float scale(int32_t k, float ebx2) { return __fmul_rn(__int2float_rn(k), ebx2); }

template <int ND>
__global__ __launch_bounds__(kRecThreads) void reconstruct_kernel(DecodeArgs a) {
  __shared__ __align__(16) int32_t s_q[kSlots];
  const uint32_t b = blockIdx.x;
  const int tid = threadIdx.x;
  if (a.st->status & ERR_CORRUPT) return;
  uint32_t org[3], w[3];
  block_box(a.g, b, org, w);
  const uint32_t m = w[0] * w[1] * w[2];
  const int32_t r = (int32_t)a.radius;
  const float ebx2 = a.ebx2_f;
  // codes -> q' = q - r
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.codes + (uint64_t)b * kSlots);
    for (uint32_t i = tid; i < (m + 7) / 8; i += kRecThreads) {
      const uint4 v = __ldcs(&src[i]);
      const uint32_t u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; k++) {
        s_q[8 * i + 2 * k] = (int32_t)(u[k] & 0xffffu) - r;
        s_q[8 * i + 2 * k + 1] = (int32_t)(u[k] >> 16) - r;
      }
    }
  }
  __syncthreads();
  const uint32_t rs = a.rec_start[b], re = a.rec_start[b + 1];
  const uint2* rec = reinterpret_cast<const uint2*>(a.ar + a.off_rec);
  for (uint32_t i = rs + tid; i < re; i += kRecThreads) {
    const uint2 kv = rec[i];
    if ((kv.x & 1u) == 0) s_q[(kv.x >> 1) % kSlots] = (int32_t)kv.y;
  }
  __syncthreads();
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
  } else {
    // z sums in registers, x sums by shuffles, y sums through shared memory
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

cudaError_t launch_decode(const DecodeArgs& a, cudaStream_t s) {
  trace_begin(K_DEC_PREP, s);
  dec_prep_kernel<<<1, 1024, 0, s>>>(a);
  trace_end(K_DEC_PREP, s);
  const uint64_t n = (a.n_rec > (uint64_t)a.g.nblk + 1 ? a.n_rec : (uint64_t)a.g.nblk + 1);
  uint64_t grid = (n + 255) / 256;
  if (grid > 4096) grid = 4096;
  trace_begin(K_DEC_RECORDS, s);
  dec_records_kernel<<<(unsigned)grid, 256, 0, s>>>(a);
  trace_end(K_DEC_RECORDS, s);
  trace_begin(K_DEC_TABLES, s);
  dec_tables_kernel<<<3, 1024, 0, s>>>(a);
  trace_end(K_DEC_TABLES, s);
  const uint64_t nseg = (uint64_t)a.g.nblk * 4;
  trace_begin(K_HUFF_DECODE, s);
  huff_decode_kernel<<<(unsigned)((nseg + kHuffDecThreads - 1) / kHuffDecThreads), kHuffDecThreads, 0, s>>>(a);
  trace_end(K_HUFF_DECODE, s);
  trace_begin(K_RLE_DECODE, s);
  rle_decode_kernel<<<a.g.nblk, kRleThreads, 0, s>>>(a);
  trace_end(K_RLE_DECODE, s);
  trace_begin(K_RECONSTRUCT, s);
  if (a.g.ndim == 1)
    reconstruct_kernel<1><<<a.g.nblk, kRecThreads, 0, s>>>(a);
  else if (a.g.ndim == 2)
    reconstruct_kernel<2><<<a.g.nblk, kRecThreads, 0, s>>>(a);
  else
    reconstruct_kernel<3><<<a.g.nblk, kRecThreads, 0, s>>>(a);
  trace_end(K_RECONSTRUCT, s);
  return cudaGetLastError();
}

}  // namespace cszp
