// Shared device-side definitions of the cszp CUDA library (sm_103a).
//
// Archive layout (little-endian, sections 8-byte aligned):
//   [0,128)          header
//   codec[nblk]      u8 per codec block (0 HUFF, 1 RLE, 2 RLE_HUFF)
//   blk_bytes[nblk]  u32 payload bytes of each block (multiples of 4)
//   records[n_rec]   (u32 key, u32 val), key = slot*2 + kind; kind 0 outlier (val =
//                    delta as int32), kind 1 verbatim patch (val = float bits);
//                    sorted by key
//   payload          per-block payloads in block order
//   books            u8 code lengths: quant-code book [1024] if any HUFF block, then
//                    run-value book [1024] + run-length book [4096] if any RLE_HUFF
//                    block
// A slot is 4096*block + the element's row-major index among the block's in-field
// elements.  Codec blocks: 1-D 4096, 2-D 64x64, 3-D 16^3.  Lorenzo chunks (where
// prediction restarts from zero, Sec. II-A "Step-1" and Sec. IV-B3): 1-D 256,
// 2-D 16x16, 3-D 8^3 (the paper gives no 3-D size).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cszp {

constexpr int kSlots = 4096;
constexpr int kNsymCode = 1024;
constexpr int kNsymLen = 4096;
constexpr int kHdr = 128;
constexpr uint32_t kMagic = 0x2B5A5343u;  // "CSZ+"
constexpr uint32_t kVersion = 2;
constexpr int kLanes = 32;  // interleave width of Huffman streams (header field)
constexpr int kMaxLen = 64;
// decode lookup tables: one 16-bit entry per kLutBits-bit prefix, (symbol << 4) | the
// length of the code it starts with (0: a longer code)
constexpr int kLutBits = 14;
using LutEntry = uint16_t;
__host__ __device__ constexpr uint32_t lut_entry(uint32_t sym, uint32_t len) { return (sym << 4) | len; }
__host__ __device__ constexpr int lut_len(uint32_t e) { return (int)(e & 15u); }
__host__ __device__ constexpr int lut_sym(uint32_t e) { return (int)(e >> 4); }
static_assert(kLutBits <= 15 && kNsymLen <= 4096, "symbol and length fit a 16-bit entry");
constexpr uint32_t kSpinLimit = 1u << 20;

enum : int { CODEC_HUFF = 0, CODEC_RLE = 1, CODEC_RLE_HUFF = 2 };
constexpr uint32_t kFlagF64 = 4u;     // header flag: the field is double precision
constexpr uint32_t kFlagGlobal = 8u;  // header flag: global (unchunked) Lorenzo prediction

// learned selector: MLP 8 -> 32 -> 32 -> 3 with ReLU, parameters packed as
// W1[32][8] b1[32] W2[32][32] b2[32] W3[3][32] b3[3]
constexpr int kMlpIn = 8, kMlpHid = 32, kMlpOut = 3;
constexpr int kMlpW1 = 0, kMlpB1 = kMlpW1 + kMlpHid * kMlpIn, kMlpW2 = kMlpB1 + kMlpHid,
              kMlpB2 = kMlpW2 + kMlpHid * kMlpHid, kMlpW3 = kMlpB2 + kMlpHid,
              kMlpB3 = kMlpW3 + kMlpOut * kMlpHid, kMlpParams = kMlpB3 + kMlpOut;
static_assert(kMlpParams == 1443, "MLP parameter count");
// the runner-up within this many log2 units (about 2%) of the best prediction sends
// the block to exact sizes
constexpr float kMlpMargin = 0.028569152f;
// RLE roughness feature (Sec. III-B madogram with binary variance): position j is
// paired with j + kMadoD0 + kMadoStep * (j mod kMadoN), i.e. the distances 1, 26,
// ..., 176 (every 25th of 1..200), each on every 8th position
constexpr uint32_t kMadoD0 = 1, kMadoStep = 25, kMadoN = 8;
enum : int { SEL_HUFF = 0, SEL_RLE = 1, SEL_RLE_HUFF = 2, SEL_HEURISTIC = 3, SEL_EXHAUSTIVE = 4, SEL_LEARNED = 5 };

// device status bits, folded into a csz_status by the host
enum : uint32_t {
  ERR_ARG = 1u,
  ERR_NONFINITE = 2u,
  ERR_RANGE = 4u,
  ERR_CORRUPT = 8u,
  ERR_CAPACITY = 16u,
  ERR_TIMEOUT = 32u
};

struct Geom {
  int ndim;
  uint32_t n[3];    // extents z, y, x (x contiguous)
  uint32_t blk[3];  // codec block extents
  uint32_t g[3];    // blocks per axis
  uint32_t nblk;
  uint64_t nelem;
};

__host__ __device__ inline uint32_t imin(uint32_t a, uint32_t b) { return a < b ? a : b; }

// origin and in-field extents of codec block b (row-major over the block grid)
__host__ __device__ inline void block_box(const Geom& g, uint32_t b, uint32_t org[3], uint32_t w[3]) {
  uint32_t bi[3];
  bi[0] = b / (g.g[1] * g.g[2]);
  bi[1] = (b / g.g[2]) % g.g[1];
  bi[2] = b % g.g[2];
#pragma unroll
  for (int d = 0; d < 3; d++) {
    org[d] = bi[d] * g.blk[d];
    w[d] = imin(g.blk[d], g.n[d] - org[d]);
  }
}

// codec block b has the full block extent on every axis (not cut by the field's edge)
__host__ __device__ inline bool block_is_full(const Geom& g, uint32_t b) {
  uint32_t org[3], w[3];
  block_box(g, b, org, w);
  return w[0] == g.blk[0] && w[1] == g.blk[1] && w[2] == g.blk[2];
}

// Values the device derives once per compression (error bound, range, counters).
struct DevState {
  double eb_d;
  float eb_f, ebx2_f, ebx2_r;
  uint32_t status;        // ERR_* bits
  uint32_t range_lo_inv;  // max of ~orderkey(x): gives the minimum
  uint32_t range_hi;      // max of orderkey(x)
  uint32_t range_done;    // CTAs finished in the range pass
  uint32_t ticket_construct;
  uint32_t ticket_encode;
  uint32_t ticket_decode;
  uint32_t encode_done;
  uint32_t ncodec[3];
  unsigned long long n_rec;
  unsigned long long n_patch;
  unsigned long long payload;
  unsigned long long total;
  float vmin, vmax;
  uint32_t n_slow;        // decompression: blocks the reconstruction kernel takes (listed)
  // double-precision fields: value range as order keys, quantization step and inverse
  unsigned long long range64_lo_inv, range64_hi;
  double step_d, rstep_d;
  // batched persistent kernel: phase hand-overs of this field (released by the
  // producer, acquired by the consumer)
  uint32_t ready_range;    // 1 once the bound is derived
  uint32_t tiles_flushed;  // tiles whose histograms, counts and codes are in place
  uint32_t books_done;     // book-phase items finished (three books and the record offsets)
};

// ---------------------------------------------------------------------------------
// memory-model helpers for the decoupled look-back
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

constexpr uint64_t LB_AGG = 1ull << 62;
constexpr uint64_t LB_INC = 1ull << 63;
constexpr uint64_t LB_VAL = LB_AGG - 1;

// Publish a tile's own aggregate (any thread).
__device__ __forceinline__ void lookback_publish(uint64_t* state, uint32_t tile, uint64_t agg) {
  st_relaxed(&state[tile], (tile == 0 ? LB_INC : LB_AGG) | agg);
}

// Decoupled look-back (single-pass prefix scan over tiles taken in ticket order):
// called by one full warp after lookback_publish; returns the exclusive prefix and
// publishes the inclusive one.  The wait is bounded; on expiry the status gets
// ERR_TIMEOUT and the tile publishes what it has so successors finish too.
__device__ inline uint64_t lookback_warp(uint64_t* state, uint32_t tile, uint64_t agg,
                                         uint32_t* status, uint32_t spin_limit) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) return 0;
  uint64_t excl = 0;
  int64_t base = (int64_t)tile - 1;
  uint32_t spins = 0;
  while (true) {
    int64_t idx = base - lane;
    uint64_t v = idx >= 0 ? ld_relaxed(&state[idx]) : LB_INC;
    uint32_t inc = __ballot_sync(~0u, (v & LB_INC) != 0);
    uint32_t bad = __ballot_sync(~0u, (v & (LB_INC | LB_AGG)) == 0);
    int first = inc ? __ffs(inc) : 32;  // 1-based lane of the nearest inclusive value
    uint32_t upto = first >= 32 ? ~0u : ((1u << first) - 1u);
    if (bad & upto) {
      if (++spins > spin_limit) {
        if (lane == 0) atomicOr(status, ERR_TIMEOUT);
        break;
      }
      __nanosleep(64);
      continue;
    }
    uint64_t add = ((1u << lane) & upto) ? (v & LB_VAL) : 0ull;
#pragma unroll
    for (int o = 16; o; o >>= 1) add += __shfl_xor_sync(~0u, add, o);
    excl += add;
    if (inc) break;
    base -= 32;
  }
  if (lane == 0) st_relaxed(&state[tile], LB_INC | (excl + agg));
  return excl;
}

// ---------------------------------------------------------------------------------
// block-wide scans and reductions (blockDim.x a multiple of 32, <= 1024)
// ---------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T u = __shfl_up_sync(~0u, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(~0u, v, o);
  return v;
}

// exclusive scan; *total receives the block sum; scratch holds >= 33 T.
// Contains __syncthreads; all threads must call.
template <typename T>
__device__ T block_excl_scan(T v, T* scratch, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) scratch[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T s = lane < nw ? scratch[lane] : T(0);
    T si = warp_incl_scan(s);
    if (lane < nw) scratch[lane] = si - s;
    if (lane == nw - 1) scratch[32] = si;
  }
  __syncthreads();
  T r = scratch[wid] + inc - v;
  if (total) *total = scratch[32];
  __syncthreads();
  return r;
}

template <typename T>
__device__ T block_sum(T v, T* scratch) {
  T t;
  block_excl_scan(v, scratch, &t);
  return t;
}

__device__ inline uint32_t block_max_u32(uint32_t v, uint32_t* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(~0u, v, o));
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < nw ? scratch[lane] : 0u;
#pragma unroll
    for (int o = 16; o; o >>= 1) s = max(s, __shfl_xor_sync(~0u, s, o));
    if (lane == 0) scratch[32] = s;
  }
  __syncthreads();
  uint32_t r = scratch[32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------------
// prequantization arithmetic (Sec. IV-A1), bit-identical to a plain C reading
// ---------------------------------------------------------------------------------

// |x - y| > eb, decided exactly: Knuth's TwoSum gives x - y = s + e exactly, then
// the comparison against the float eb follows from s = RN(x - y).
__device__ __forceinline__ bool exceeds_exact(float x, float y, float eb) {
  const float s = __fsub_rn(x, y);
  // s = RN(x - y) and eb is a float, so |s| < eb implies |x - y| <= eb and |s| > eb
  // implies |x - y| > eb; only |s| == eb needs the rounding error
  if (fabsf(s) < eb) return false;
  if (fabsf(s) > eb) return true;
  const float bb = __fsub_rn(s, x);
  const float e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, bb)), __fsub_rn(-y, bb));
  return s > 0.0f ? e > 0.0f : e < 0.0f;
}

// k0 = nearest integer to fl32(x/2eb), ties to even; if fl32(k0*2eb) misses x by more than eb, try the
// neighbour integer on x's side, else keep k0 and ask for a verbatim patch.
// Returns ERR_* bits (0 on success).
__device__ __forceinline__ uint32_t prequant(float x, float eb_f, float ebx2_f, float ebx2_r,
                                             int32_t& k, bool& patch) {
  patch = false;
  k = 0;
  const float v = __fmul_rn(x, ebx2_r);
  // one compare covers both failures: ebx2_r is finite and positive, so |v| < 2^23
  // holds only for finite x
  if (!(fabsf(v) < 8388608.0f)) return isfinite(x) ? ERR_RANGE : ERR_NONFINITE;
  int32_t k0 = __float2int_rn(v);
  float x0 = __fmul_rn(__int2float_rn(k0), ebx2_f);
  if (!exceeds_exact(x, x0, eb_f)) {
    k = k0;
    return 0;
  }
  int32_t k1 = k0 + (x > x0 ? 1 : -1);
  float x1 = __fmul_rn(__int2float_rn(k1), ebx2_f);
  if (!exceeds_exact(x, x1, eb_f)) {
    k = k1;
    return 0;
  }
  k = k0;
  patch = true;
  return 0;
}

// The common case of prequant with no branches: k0 is final when |x / 2eb| < 2^23
// and fl32(k0 * 2eb) lies strictly within eb of x (the rounded difference then
// decides exactly).  Returns false when prequant must decide instead (non-finite
// or out-of-range input, a tie at exactly eb, a miss needing the neighbour or a
// patch); k then holds no meaningful value.
__device__ __forceinline__ bool prequant_fast(float x, float eb_f, float ebx2_f, float ebx2_r, int32_t& k) {
  const float v = __fmul_rn(x, ebx2_r);
  k = __float2int_rn(v);
  const float s = __fsub_rn(x, __fmul_rn(__int2float_rn(k), ebx2_f));
  return (fabsf(v) < 8388608.0f) & (fabsf(s) < eb_f);
}

// ---------------------------------------------------------------------------------
// double-precision fields: the same prequantization with the step
// step = fl64(2 eb (1 - 2^-24)); |k| < 2^27 keeps the rounding of fl64(k * step)
// (at most 2^-25 eb) inside the margin the shrink leaves, so the nearest integer, or
// its neighbour when the product x * (1 / step) rounds across a half point, always
// meets the bound and no value needs a verbatim patch
// ---------------------------------------------------------------------------------
constexpr double kStepShrink = 1.0 - 0x1p-24;
constexpr double kMaxK64 = 134217728.0;  // 2^27

__device__ __forceinline__ bool exceeds_exact_d(double x, double y, double eb) {
  const double s = __dsub_rn(x, y);
  if (fabs(s) < eb) return false;
  if (fabs(s) > eb) return true;
  const double bb = __dsub_rn(s, x);
  const double e = __dadd_rn(__dsub_rn(x, __dsub_rn(s, bb)), __dsub_rn(-y, bb));
  return s > 0.0 ? e > 0.0 : e < 0.0;
}

// Returns ERR_* bits (0 on success); no patches for doubles.
__device__ __forceinline__ uint32_t prequant_d(double x, double eb_d, double step, double rstep, int32_t& k) {
  k = 0;
  const double v = __dmul_rn(x, rstep);
  if (!(fabs(v) < kMaxK64)) return isfinite(x) ? ERR_RANGE : ERR_NONFINITE;
  const int32_t k0 = __double2int_rn(v);
  const double x0 = __dmul_rn((double)k0, step);
  if (!exceeds_exact_d(x, x0, eb_d)) {
    k = k0;
    return 0;
  }
  const int32_t k1 = k0 + (x > x0 ? 1 : -1);
  if (!exceeds_exact_d(x, __dmul_rn((double)k1, step), eb_d)) {
    k = k1;
    return 0;
  }
  return ERR_RANGE;  // unreachable by the step's margin
}

__device__ __forceinline__ bool prequant_fast_d(double x, double eb_d, double step, double rstep, int32_t& k) {
  const double v = __dmul_rn(x, rstep);
  k = __double2int_rn(v);
  const double s = __dsub_rn(x, __dmul_rn((double)k, step));
  return (fabs(v) < kMaxK64) & (fabs(s) < eb_d);
}

// Binary logarithm in Q16 by bit-by-bit squaring of the mantissa (integer only).
// constexpr so that the same routine also fills the table of small arguments below.
__host__ __device__ constexpr uint32_t log2_q16(uint64_t v) {
  if (v == 0) return 0;
  uint32_t e = 0;
  for (uint32_t s = 32; s; s >>= 1)
    if (v >> (e + s)) e += s;
  uint64_t m = e >= 31 ? (v >> (e - 31)) : (v << (31 - e));
  uint32_t frac = 0;
#pragma unroll 1
  for (int i = 0; i < 16; i++) {
    m = (m * m) >> 31;
    frac <<= 1;
    if (m >= (2ull << 31)) {
      m >>= 1;
      frac |= 1u;
    }
  }
  return e * 65536u + frac;
}

// log2_q16 of 0..4096 (every count a codec block can hold), evaluated at compile
// time: block statistics look their per-bin terms up instead of squaring 16 times.
struct Log2Table {
  uint32_t v[kSlots + 1];
};
constexpr Log2Table make_log2_table() {
  Log2Table t{};
  for (uint32_t i = 0; i <= (uint32_t)kSlots; i++) t.v[i] = log2_q16(i);
  return t;
}
static_assert(make_log2_table().v[1] == 0u && make_log2_table().v[2] == 65536u &&
                  make_log2_table().v[kSlots] == 12u * 65536u,
              "log2 table: exact powers of two");
__device__ const Log2Table kLog2Table = make_log2_table();

__device__ __forceinline__ uint32_t log2_q16_small(uint32_t v) { return __ldg(&kLog2Table.v[v]); }

// ---------------------------------------------------------------------------------
// canonical Huffman codes from lengths (block-wide).  Codes are ordered by
// (length, symbol); the first code of length l is (first(l-1) + count(l-1)) << 1.
// Outputs per symbol its code and its rank in (length, symbol) order; per length
// the first code, the count and the offset of its first symbol in that order.
// smem: cnt[kMaxLen+1] u32, first[kMaxLen+1] u64, off[kMaxLen+1] u32,
//       wcnt[(nsym/32)*(kMaxLen+1)] u16
// Contains __syncthreads; all threads call.
// ---------------------------------------------------------------------------------
struct CanonSmem {
  uint32_t cnt[kMaxLen + 1];
  uint32_t off[kMaxLen + 1];
  unsigned long long first[kMaxLen + 1];
  uint32_t bad;
};

__device__ inline void canonical_build(const uint8_t* len, int nsym, CanonSmem* cs, uint16_t* wcnt,
                                       uint64_t* code_out, uint16_t* sorted_out) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int l = tid; l <= kMaxLen; l += nt) cs->cnt[l] = 0;
  if (tid == 0) cs->bad = 0;
  const int nchunk = nsym / 32;
  for (int i = tid; i < nchunk * (kMaxLen + 1); i += nt) wcnt[i] = 0;
  __syncthreads();
  // per-warp-chunk counts and ranks by length
  for (int base = (tid & ~31); base < nsym; base += nt) {
    const int s = base + (tid & 31);
    const int l = len[s];
    const uint32_t peers = __match_any_sync(~0u, l);
    if (l > kMaxLen) cs->bad = 1;
    if (l && l <= kMaxLen && (peers & ((1u << (tid & 31)) - 1u)) == 0) {
      wcnt[(s >> 5) * (kMaxLen + 1) + l] = (uint16_t)__popc(peers);
      atomicAdd(&cs->cnt[l], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long c = 0;
    uint32_t o = 0;
    cs->first[0] = 0;
    cs->off[0] = 0;
    for (int l = 1; l <= kMaxLen; l++) {
      c = (c + (l > 1 ? cs->cnt[l - 1] : 0u)) << 1;
      cs->first[l] = c;
      cs->off[l] = o;
      o += cs->cnt[l];
    }
  }
  // prefix of per-chunk counts over chunks, per length (in place)
  for (int l = 1 + tid; l <= kMaxLen; l += nt) {
    uint32_t run = 0;
    for (int ch = 0; ch < nchunk; ch++) {
      uint16_t c = wcnt[ch * (kMaxLen + 1) + l];
      wcnt[ch * (kMaxLen + 1) + l] = (uint16_t)run;
      run += c;
    }
  }
  __syncthreads();
  for (int base = (tid & ~31); base < nsym; base += nt) {
    const int s = base + (tid & 31);
    const int l = len[s];
    const uint32_t peers = __match_any_sync(~0u, l);
    if (l && l <= kMaxLen) {
      uint32_t rank = wcnt[(s >> 5) * (kMaxLen + 1) + l] + __popc(peers & ((1u << (tid & 31)) - 1u));
      if (code_out) code_out[s] = cs->first[l] + rank;
      if (sorted_out) sorted_out[cs->off[l] + rank] = (uint16_t)s;
    } else if (code_out) {
      code_out[s] = 0;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------------
// runs of a block's dense codes c[0..m) (m <= 4096), blockDim.x == 256.
// head[w] bit b: position 32w+b starts a run; woff[w]: runs before word w;
// nexthead[w]: first run start at or after word w's first position (m if none).
// ---------------------------------------------------------------------------------
// Run heads of the block's codes c[0..m) as bit words head[j >> 5] (bit j & 31 set
// where a run starts).  Returns, in lane 0 of each warp, the number of heads in the
// words that warp wrote (0 elsewhere).  Reads c only; no barrier.
__device__ inline uint32_t run_head_words(const uint16_t* c, uint32_t m, uint32_t* head) {
  const int tid = threadIdx.x, lane = tid & 31;
  uint32_t n = 0;
#pragma unroll 4
  for (int i = 0; i < kSlots / 256; i++) {
    const uint32_t j = tid + 256 * i;
    const bool h = j < m && (j == 0 || c[j] != c[j - 1]);
    const uint32_t hb = __ballot_sync(~0u, h);
    if (lane == 0) {
      head[j >> 5] = hb;
      n += __popc(hb);
    }
  }
  return n;
}

// Index of the run heads (warp 0, after the head words are complete): woff[w] = runs
// starting before word w (woff[kSlots/32] = total), nexthead[w] = first head at or
// after word w (m if none).
__device__ inline void run_head_index(const uint32_t* head, uint32_t m, uint32_t* woff, uint32_t* nexthead) {
  const int lane = threadIdx.x & 31;
  // lane covers words 4*lane .. 4*lane+3
  uint32_t cnt[4], first[4];
  uint32_t tot = 0;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const uint32_t w = 4 * lane + k, hm = head[w];
    cnt[k] = __popc(hm);
    first[k] = hm ? w * 32 + (__ffs(hm) - 1) : 0xffffffffu;
    tot += cnt[k];
  }
  const uint32_t incl = warp_incl_scan(tot);
  uint32_t run = incl - tot;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    woff[4 * lane + k] = run;
    run += cnt[k];
  }
  // suffix minimum of first-head positions
  uint32_t lf = min(min(first[0], first[1]), min(first[2], first[3]));
  uint32_t suf = lf;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_down_sync(~0u, suf, o);
    if (lane + o < 32) suf = min(suf, v);
  }
  uint32_t after = __shfl_down_sync(~0u, suf, 1);
  if (lane == 31) after = 0xffffffffu;
  uint32_t cur = after;
#pragma unroll
  for (int k = 3; k >= 0; k--) {
    cur = min(cur, first[k]);
    nexthead[4 * lane + k] = cur == 0xffffffffu ? m : cur;
  }
  if (lane == 31) woff[kSlots / 32] = incl;
}

// Both of the above for a whole CTA of 256 threads; returns the number of runs.
__device__ inline uint32_t block_run_heads(const uint16_t* c, uint32_t m, uint32_t* head, uint32_t* woff,
                                           uint32_t* nexthead) {
  run_head_words(c, m, head);
  __syncthreads();
  if (threadIdx.x < 32) run_head_index(head, m, woff, nexthead);
  __syncthreads();
  return woff[kSlots / 32];
}

// position of the run start after position j (a run start), using the head words
__device__ __forceinline__ uint32_t next_head(const uint32_t* head, const uint32_t* nexthead, uint32_t j,
                                              uint32_t m) {
  const uint32_t w = j >> 5, b = j & 31;
  const uint32_t rest = b == 31 ? 0u : (head[w] >> (b + 1)) << (b + 1);
  if (rest) return w * 32 + (__ffs(rest) - 1);
  return w + 1 < (uint32_t)(kSlots / 32) ? nexthead[w + 1] : m;
}

// ---------------------------------------------------------------------------------
// Interleaved Huffman stream (32 lanes, 16-bit units): symbol i belongs to lane i%32;
// a lane's bit string (its codes, MSB first, zero-padded) is cut into 16-bit units
// stored in the order a 32-lane decoder reads them: at step t the lanes holding
// symbols 32t..32t+31 top up in rounds (each lane whose next code is longer than
// the bits it holds takes one unit per round, lanes in increasing order), then all
// consume their code.
// ---------------------------------------------------------------------------------

// One warp encodes sym[0..N) (+add) with a book into out[]; returns the unit count.
__device__ inline uint32_t ihs_encode_warp(const uint16_t* sym, uint32_t N, int add,
                                           const uint8_t* __restrict__ lens,
                                           const uint64_t* __restrict__ codes, uint16_t* out) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t mine = N > lane ? (N - lane + 31) / 32 : 0;
  uint64_t acc = 0;   // produced, not yet emitted bits (MSB-aligned)
  int nacc = 0;
  uint32_t enext = 0;  // next own symbol to produce
  int nb = 0;          // bits the simulated decoder lane holds
  uint32_t base = 0;
  const uint32_t T = (N + 31) / 32;
  for (uint32_t t = 0; t < T; t++) {
    const bool active = t < mine;
    const int len = active ? (int)__ldg(&lens[sym[32 * t + lane] + add]) : 0;
    while (true) {
      const bool need = active && len > nb;
      const uint32_t ballot = __ballot_sync(~0u, need);
      if (!ballot) break;
      if (need) {
        while (nacc < 16 && enext < mine) {
          const int s = sym[32 * enext + lane] + add;
          const int l = __ldg(&lens[s]);
          acc |= (__ldg(&codes[s]) << (64 - l)) >> nacc;
          nacc += l;
          enext++;
        }
        out[base + __popc(ballot & ((1u << lane) - 1u))] = (uint16_t)(acc >> 48);
        acc <<= 16;
        nacc = nacc > 16 ? nacc - 16 : 0;
        nb += 16;
      }
      base += __popc(ballot);
    }
    nb -= len;
  }
  return base;
}

// Block-wide encoder of the same stream (blockDim.x == 256): thread (lane l, warp w)
// owns lane l's steps 16w..16w+15.  A lane holding cum(t) bits of codes after step t
// has taken U(t) = ceil(cum(t)/16) units, so at step t it takes U(t) - U(t-1) units,
// one per round; positions follow from per-step ballots (rounds, then lane order).
// Every unit a lane takes at step t starts inside the code of its symbol t, so the
// owner of step t gathers the unit's 16 bits from that code onwards.  Each unit is
// written exactly once.  Returns the unit count.  scratch: >= 8*32 + 8 u32.
__device__ inline uint32_t ihs_unit_gather(const uint16_t* sym, uint32_t N, int add,
                                           const uint8_t* __restrict__ lens,
                                           const uint64_t* __restrict__ codes, uint32_t lane,
                                           uint32_t t, uint32_t skip) {
  uint32_t unit = 0;
  int have = 0;
  for (uint32_t tt = t; have < 16 && 32 * tt + lane < N; tt++) {
    const int s = sym[32 * tt + lane] + add;
    const int L = __ldg(&lens[s]);
    const uint64_t C = __ldg(&codes[s]);
    const int avail = L - (int)skip;
    const int take = min(avail, 16 - have);
    const uint32_t bits = (uint32_t)((C >> (avail - take)) & ((1ull << take) - 1ull));
    unit |= bits << (16 - have - take);
    have += take;
    skip = 0;
  }
  return unit;
}

__device__ inline uint32_t ihs_encode_block(const uint16_t* sym, uint32_t N, int add,
                                            const uint8_t* __restrict__ lens,
                                            const uint64_t* __restrict__ codes, uint16_t* out16,
                                            uint32_t* scratch) {
  const uint32_t tid = threadIdx.x, l = tid & 31, w = tid >> 5;
  const uint32_t t0 = 16 * w;
  auto len_at = [&](uint32_t t) -> uint32_t {
    const uint32_t j = 32 * t + l;
    return j < N ? (uint32_t)__ldg(&lens[sym[j] + add]) : 0u;
  };
  __syncthreads();
  uint32_t cum = 0;
  for (int i = 0; i < 16; i++) cum += len_at(t0 + i);
  scratch[32 * w + l] = cum;
  __syncthreads();
  uint32_t pre = 0;
  for (uint32_t v = 0; v < w; v++) pre += scratch[32 * v + l];
  // units per step summed over lanes, per warp
  uint32_t c = pre, uprev = (pre + 15) >> 4, wtot = 0;
  for (int i = 0; i < 16; i++) {
    c += len_at(t0 + i);
    const uint32_t u = (c + 15) >> 4;
    wtot += warp_sum(u - uprev);
    uprev = u;
  }
  if (l == 0) scratch[256 + w] = wtot;
  __syncthreads();
  uint32_t base = 0, total = 0;
  for (uint32_t v = 0; v < 8; v++) {
    if (v < w) base += scratch[256 + v];
    total += scratch[256 + v];
  }
  const uint32_t lt = (1u << l) - 1u;
  c = pre;
  uprev = (pre + 15) >> 4;
#pragma unroll 1
  for (int i = 0; i < 16; i++) {
    const uint32_t cn = c + len_at(t0 + i);
    const uint32_t u = (cn + 15) >> 4;
    const uint32_t D = u - uprev;
#pragma unroll 1
    for (uint32_t r = 1; r <= 4; r++) {
      const uint32_t br = __ballot_sync(~0u, D >= r);
      if (!br) break;
      if (D >= r) {
        const uint32_t k = uprev + r - 1;
        out16[base + __popc(br & lt)] = (uint16_t)ihs_unit_gather(sym, N, add, lens, codes, l, t0 + i, 16 * k - c);
      }
      base += __popc(br);
    }
    c = cn;
    uprev = u;
  }
  return total;
}

// A Huffman codec block is a u16 unit count of stream A, then two interleaved
// streams: A codes the block's first huff_split(m) symbols, B the rest.
__host__ __device__ __forceinline__ uint32_t huff_split(uint32_t m) {
  const uint32_t h = 32u * ((m + 63u) / 64u);
  return h < m ? h : m;
}

// Block-wide encoder of one Huffman block's two streams (256 threads).  Pass 1
// (ihs_plan2): thread (lane l, warp w) reads the lengths of lane l's steps
// 16(w&3)..16(w&3)+15 of stream w>>2 once into registers; per-lane totals give both
// streams' sizes.  Pass 2 (ihs_emit2): each thread appends its codes to its lane's
// bit string in shared memory (64 strings of 64 words, word index XOR-swizzled by
// the lane so a warp's 32 lanes hit 32 banks), then every unit is cut straight out
// of its lane's string and stored at its decoder-order position (rounds within
// steps, lanes in order within a round).  Lanes above 2016 bits take the gather
// encoder instead.
struct IhsPlan {
  uint32_t len4[4];    // the thread's 16 code lengths, 8 bits each
  uint32_t pre;        // bits of the lane before the thread's first step
  uint32_t cum;        // bits of the thread's 16 steps
};

constexpr uint32_t kLaneWords = 64;                       // words per lane string
constexpr uint32_t kLaneBitsMax = 32 * (kLaneWords - 1);  // 2016 bits: a string and the word after it fit

__device__ __forceinline__ uint32_t plan_len(const IhsPlan& P, int i) {
  // selects rather than an indexed load, so the plan stays in registers
  const uint32_t wsel = i < 8 ? (i < 4 ? P.len4[0] : P.len4[1]) : (i < 12 ? P.len4[2] : P.len4[3]);
  return (wsel >> (8 * (i & 3))) & 0xffu;
}

struct IhsPlan2Out {
  uint32_t units_a, units_b;  // units of each stream
  uint32_t max_lane_bits;     // over both streams
};

// Fills P; returns the units of both streams and the largest lane total.  scratch:
// >= 256 + 4 u32.  Contains __syncthreads.
__device__ inline IhsPlan2Out ihs_plan2(const uint16_t* sym, uint32_t m, const uint8_t* __restrict__ lens,
                                       uint32_t* scratch, IhsPlan& P) {
  const uint32_t tid = threadIdx.x, l = tid & 31, w = tid >> 5, sidx = w >> 2, wl = w & 3;
  const uint32_t h = huff_split(m);
  const uint32_t N = sidx ? m - h : h;
  const uint16_t* ss = sym + (sidx ? h : 0);
  const uint32_t t0 = 16 * wl;
  uint32_t cum = 0;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    uint32_t pk = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t j = 32 * (t0 + 4 * q + k) + l;
      const uint32_t L = j < N ? (uint32_t)__ldg(&lens[ss[j]]) : 0u;
      pk |= L << (8 * k);
      cum += L;
    }
    P.len4[q] = pk;
  }
  P.cum = cum;
  __syncthreads();
  scratch[32 * w + l] = cum;
  __syncthreads();
  uint32_t pre = 0, tot = 0;
#pragma unroll
  for (uint32_t v = 0; v < 4; v++) {
    const uint32_t c = scratch[32 * (4 * sidx + v) + l];
    if (v < wl) pre += c;
    tot += c;
  }
  P.pre = pre;
  if (wl == 0) {  // warps 0 and 4 total their stream
    const uint32_t units = warp_sum((tot + 15) >> 4);
    uint32_t mx = tot;
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(~0u, mx, o));
    if (l == 0) {
      scratch[256 + sidx] = units;
      scratch[258 + sidx] = mx;
    }
  }
  __syncthreads();
  IhsPlan2Out r;
  r.units_a = scratch[256];
  r.units_b = scratch[257];
  r.max_lane_bits = max(scratch[258], scratch[259]);
  __syncthreads();
  return r;
}

// Pass 2; requires every lane total <= kLaneBitsMax.  out16[0] receives units_a,
// stream A starts at out16[1], stream B at out16[1 + units_a].  lanebuf: 64 *
// kLaneWords u32, all zero if `clean` (cleared before a block barrier the caller
// passed), else cleared here.  scratch: >= 8 u32.  Contains __syncthreads.
__device__ inline void ihs_emit2(const uint16_t* sym, uint32_t m, const uint64_t* __restrict__ codes,
                                 const IhsPlan& P, uint32_t units_a, uint32_t* lanebuf, uint16_t* out16,
                                 uint32_t* scratch, bool clean) {
  const uint32_t tid = threadIdx.x, l = tid & 31, w = tid >> 5, sidx = w >> 2, wl = w & 3;
  const uint32_t h = huff_split(m);
  const uint16_t* ss = sym + (sidx ? h : 0);
  const uint32_t t0 = 16 * wl;
  uint32_t* mine = lanebuf + kLaneWords * (32 * sidx + l);
  // each thread clears the words its bits land in (and the one after them); together
  // the threads of a lane clear every word that is read
  if (!clean) {
    const uint32_t w0 = P.pre >> 5, w1 = min((P.pre + P.cum + 31) >> 5, kLaneWords - 1);
    for (uint32_t wi = w0; wi <= w1; wi++) mine[wi ^ l] = 0;
    __syncthreads();
  }
  // codes gather in a 64-bit window (left-aligned, `fill` bits used, < 32 between
  // codes); each completed word is stored.  Only the thread's first and last words
  // can be shared with the neighbouring steps of the lane: those two are OR-ed in.
  {
    uint32_t wi = P.pre >> 5;
    int fill = (int)(P.pre & 31);
    uint64_t win = 0;
    bool first = true;
    auto flush = [&]() {
      const uint32_t word = (uint32_t)(win >> 32);
      if (first) atomicOr(&mine[wi ^ l], word);
      else mine[wi ^ l] = word;
      first = false;
      win <<= 32;
      fill -= 32;
      wi++;
    };
#pragma unroll 4
    for (int i = 0; i < 16; i++) {
      const int L = (int)plan_len(P, i);
      if (L == 0) continue;
      const uint64_t C = __ldg(&codes[ss[32 * (t0 + i) + l]]);
      if (L <= 32) {
        win |= C << (64 - fill - L);
        fill += L;
        if (fill >= 32) flush();
      } else {  // a code longer than 32 bits: its top L - 32 bits, then the low 32
        const int hl = L - 32;
        win |= (C >> 32) << (64 - fill - hl);
        fill += hl;
        if (fill >= 32) flush();
        win |= (C & 0xffffffffull) << (32 - fill);
        fill += 32;
        flush();
      }
    }
    if (fill > 0) atomicOr(&mine[wi ^ l], (uint32_t)(win >> 32));
  }
  // units each warp's steps take, for the warp's first output position in its stream
  const uint32_t u_begin = (P.pre + 15) >> 4, u_end = (P.pre + P.cum + 15) >> 4;
  const uint32_t wtot = warp_sum(u_end - u_begin);
  if (l == 0) scratch[w] = wtot;
  __syncthreads();
  uint32_t base = 1 + (sidx ? units_a : 0);
  for (uint32_t v = 0; v < wl; v++) base += scratch[4 * sidx + v];
  if (tid == 0) out16[0] = (uint16_t)units_a;
  const uint32_t lt = (1u << l) - 1u;
  // unit k of this lane's string: units are 16-bit aligned, so unit k is the upper
  // (k even) or lower (k odd) half of word k / 2
  auto unit_at = [&](uint32_t k) -> uint16_t { return (uint16_t)(mine[(k >> 1) ^ l] >> ((~k & 1u) << 4)); };
  uint32_t c = P.pre, uprev = u_begin;
  // four steps at a time; a lane takes two or more units in one step only for a code
  // longer than 16 bits, so usually one ballot per step gives every position
#pragma unroll
  for (int i0 = 0; i0 < 16; i0 += 4) {
    uint32_t D[4], up[4];
    bool multi = false;
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t cn = c + plan_len(P, i0 + k);
      const uint32_t u = (cn + 15) >> 4;
      D[k] = u - uprev;
      up[k] = uprev;
      multi |= D[k] >= 2;
      c = cn;
      uprev = u;
    }
    if (!__any_sync(~0u, multi)) {
      uint32_t b1[4];
#pragma unroll
      for (int k = 0; k < 4; k++) b1[k] = __ballot_sync(~0u, D[k] != 0);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        if (D[k]) out16[base + __popc(b1[k] & lt)] = unit_at(up[k]);
        base += __popc(b1[k]);
      }
    } else {
      // rounds, as the decoder takes them
#pragma unroll
      for (int k = 0; k < 4; k++) {
#pragma unroll 1
        for (uint32_t r = 1; r <= 4; r++) {
          const uint32_t br = __ballot_sync(~0u, D[k] >= r);
          if (!br) break;
          if (D[k] >= r) out16[base + __popc(br & lt)] = unit_at(up[k] + r - 1);
          base += __popc(br);
        }
      }
    }
  }
  __syncthreads();
}

// Units lane `lane` of a stream needs: ceil(bits/16), given its bit total.
__device__ __forceinline__ uint32_t ihs_lane_units(uint32_t bits) { return (bits + 15) / 16; }


// One forward pass of the selector MLP by a full warp: lane i owns hidden unit i, and
// every dot product is a chain of fused multiply-adds from the bias over the inputs
// in order (so the FP32 result is reproducible by any implementation that chains the
// same way).  f: the 8 features (same in every lane); y: the 3 outputs, in every lane.
__device__ __forceinline__ void mlp_forward_warp(const float* __restrict__ w, const float* f, float* y) {
  const int lane = threadIdx.x & 31;
  float acc = __ldg(&w[kMlpB1 + lane]);
#pragma unroll
  for (int j = 0; j < kMlpIn; j++) acc = fmaf(__ldg(&w[kMlpW1 + lane * kMlpIn + j]), f[j], acc);
  const float h1 = acc > 0.0f ? acc : 0.0f;
  acc = __ldg(&w[kMlpB2 + lane]);
#pragma unroll
  for (int j = 0; j < kMlpHid; j++)
    acc = fmaf(__ldg(&w[kMlpW2 + lane * kMlpHid + j]), __shfl_sync(~0u, h1, j), acc);
  const float h2 = acc > 0.0f ? acc : 0.0f;
  const int o = lane < kMlpOut ? lane : 0;
  acc = __ldg(&w[kMlpB3 + o]);
#pragma unroll
  for (int j = 0; j < kMlpHid; j++)
    acc = fmaf(__ldg(&w[kMlpW3 + o * kMlpHid + j]), __shfl_sync(~0u, h2, j), acc);
#pragma unroll
  for (int c = 0; c < kMlpOut; c++) y[c] = __shfl_sync(~0u, acc, c);
}

// ---------------------------------------------------------------------------------
// mbarrier helpers for bulk asynchronous copies (TMA)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Ends an mbarrier's life, so that its shared-memory words can hold other data.
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Sets the flag *p to 1 with release semantics at GPU scope: what the calling thread
// wrote before is visible to a thread that reads the 1 with acquire semantics.
__device__ __forceinline__ void release_flag(uint32_t* p) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(1u) : "memory");
}

// Bounded wait (one thread) until the counter *p reaches `target`, read with acquire
// semantics at GPU scope, so that what the producers wrote before their release is
// visible after it; false when `limit` polls (about 64 ns apart) pass first.
__device__ __forceinline__ bool wait_ge_acquire(const uint32_t* p, uint32_t target, uint32_t limit) {
  for (uint32_t i = 0;; i++) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    if (v >= target) return true;
    if (i >= limit) return false;
    __nanosleep(64);
  }
}

// Bounded wait for phase `parity` of an mbarrier: at most `limit` tries, each
// suspending the thread for about a microsecond at most; false when the limit
// expired.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, uint32_t limit) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < limit; i++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from global
// to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace cszp
