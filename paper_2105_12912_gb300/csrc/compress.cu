// Compression kernels of cszp (sm_103a).
//
// Pipeline (one stream, no host round trip until the end):
//   range_kernel / abs_params_kernel  value range (REL) and the FP32 error bound
//   construct_kernel<ND>              prequant + chunk-local Lorenzo + postquant
//                                     (Alg. 1 l.1-8), outlier/patch records placed by
//                                     decoupled look-back, code / run-value /
//                                     run-length histograms
//   codebook_kernel                   three canonical Huffman books
//   encode_kernel                     per block: exact sizes or heuristic / MLP pick,
//                                     payload placement by decoupled look-back, payload
//   finalize_kernel                   header, padding, books
#include "common.cuh"
#include "kernels.h"

namespace cszp {

// =================================================================================
// value range and error bound
// =================================================================================

__device__ __forceinline__ uint32_t order_key(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_to_float(uint32_t k) {
  uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
  return __uint_as_float(b);
}

// ABS: eb_d = eb; REL: eb_d = eb * (max - min) in double.  eb_f = largest float <= eb_d,
// ebx2_f = 2 eb_f, ebx2_r = fl32(1 / (double)ebx2_f).  Degenerate bounds -> ERR_ARG.
__device__ void derive_eb(DevState* st, int mode, double eb, float vmin, float vmax) {
  double d = mode == 0 ? eb : eb * ((double)vmax - (double)vmin);
  float f = __double2float_rd(d);
  float x2 = 2.0f * f;
  float r = __double2float_rn(1.0 / (double)x2);
  st->eb_d = d;
  st->eb_f = f;
  st->ebx2_f = x2;
  st->ebx2_r = r;
  st->vmin = vmin;
  st->vmax = vmax;
  if (!(f > 0.0f) || !isfinite(x2) || !(r > 0.0f) || !isfinite(r)) atomicOr(&st->status, ERR_ARG);
}

__global__ void abs_params_kernel(DevState* st, double eb) {
  if (threadIdx.x == 0 && blockIdx.x == 0) derive_eb(st, 0, eb, 0.0f, 0.0f);
}

// Grid-stride min/max with float4 loads; non-finite values are flagged.  The last CTA
// to finish derives the error bound.
__global__ __launch_bounds__(256) void range_kernel(const float* __restrict__ x, uint64_t n,
                                                    DevState* st, int mode, double eb) {
  __shared__ uint32_t s_red[2][33];
  __shared__ bool s_last;
  uint32_t lo_inv = 0, hi = 0, bad = 0;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  const bool vec = (((uintptr_t)x) & 15) == 0;
  uint64_t nvec = vec ? n / 4 : 0;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  for (uint64_t i = tid; i < nvec; i += nth) {
    float4 v = __ldcs(&x4[i]);
    float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (!isfinite(a[k])) {
        bad = 1;
      } else {
        uint32_t key = order_key(a[k]);
        lo_inv = max(lo_inv, ~key);
        hi = max(hi, key);
      }
    }
  }
  for (uint64_t i = nvec * 4 + tid; i < n; i += nth) {
    float a = x[i];
    if (!isfinite(a)) {
      bad = 1;
    } else {
      uint32_t key = order_key(a);
      lo_inv = max(lo_inv, ~key);
      hi = max(hi, key);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    lo_inv = max(lo_inv, __shfl_xor_sync(~0u, lo_inv, o));
    hi = max(hi, __shfl_xor_sync(~0u, hi, o));
  }
  bad = __any_sync(~0u, bad);
  if (lane == 0) {
    s_red[0][wid] = lo_inv;
    s_red[1][wid] = hi;
  }
  if (bad && lane == 0) atomicOr(&st->status, ERR_NONFINITE);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      a = max(a, s_red[0][w]);
      b = max(b, s_red[1][w]);
    }
    atomicMax(&st->range_lo_inv, a);
    atomicMax(&st->range_hi, b);
    __threadfence();
    s_last = atomicAdd(&st->range_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    uint32_t a = atomicAdd(&st->range_lo_inv, 0u);
    uint32_t b = atomicAdd(&st->range_hi, 0u);
    if (b == 0) {  // nothing finite was seen
      atomicOr(&st->status, ERR_NONFINITE);
      return;
    }
    derive_eb(st, mode, eb, key_to_float(~a), key_to_float(b));
  }
}

// =================================================================================
// Lorenzo construction
// =================================================================================

template <int ND>
struct Chunk;
template <>
struct Chunk<1> {
  static constexpr uint32_t z = 1, y = 1, x = 256;
};
template <>
struct Chunk<2> {
  static constexpr uint32_t z = 1, y = 16, x = 16;
};
template <>
struct Chunk<3> {
  static constexpr uint32_t z = 8, y = 8, x = 8;
};

constexpr int kConstructThreads = 256;
constexpr int kPer = kSlots / kConstructThreads;  // 16 elements per thread

// packed 16-bit counter pairs in a u32 word (per-CTA counts stay below 65536)
__device__ __forceinline__ void add16(uint32_t* words, uint32_t bin, uint32_t v) {
  atomicAdd(&words[bin >> 1], v << ((bin & 1u) * 16u));
}

__device__ __forceinline__ void flush16(const uint32_t* words, int nwords, uint32_t* global) {
  for (int i = threadIdx.x; i < nwords; i += blockDim.x) {
    uint32_t v = words[i];
    if (v & 0xffffu) atomicAdd(&global[2 * i], v & 0xffffu);
    if (v >> 16) atomicAdd(&global[2 * i + 1], v >> 16);
  }
}

// coordinates of dense in-block index j
template <int ND>
__device__ __forceinline__ void dense_coords(uint32_t j, uint32_t wy, uint32_t wx, uint32_t& zz,
                                             uint32_t& yy, uint32_t& xx) {
  if (ND == 1) {
    zz = 0;
    yy = 0;
    xx = j;
  } else if (ND == 2) {
    zz = 0;
    yy = j / wx;
    xx = j - yy * wx;
  } else {
    uint32_t p = wy * wx;
    zz = j / p;
    uint32_t r = j - zz * p;
    yy = r / wx;
    xx = r - yy * wx;
  }
}

template <int ND>
__global__ __launch_bounds__(kConstructThreads) void construct_kernel(ConstructArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  int32_t* s_k = reinterpret_cast<int32_t*>(smem);             // 4096: k, then delta
  uint16_t* s_c = reinterpret_cast<uint16_t*>(s_k + kSlots);  // 4096 codes
  uint32_t* s_hc = reinterpret_cast<uint32_t*>(s_c + kSlots);  // 512 words: code hist
  uint32_t* s_hv = s_hc + kNsymCode / 2;                       // 512 words: run values
  uint32_t* s_hl = s_hv + kNsymCode / 2;                       // 2048 words: run lengths
  uint32_t* s_patch = s_hl + kNsymLen / 2;                     // 128 words
  uint32_t* s_outl = s_patch + kSlots / 32;                    // 128 words
  uint32_t* s_head = s_outl + kSlots / 32;                     // 128 words
  uint64_t* s_scan = reinterpret_cast<uint64_t*>(s_head + kSlots / 32);  // 33
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_prefix;

  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(&a.st->ticket_construct, 1u);
  for (int i = tid; i < (kNsymCode + kNsymCode + kNsymLen) / 2 + 3 * (kSlots / 32); i += blockDim.x)
    s_hc[i] = 0;
  __syncthreads();
  const uint32_t b = s_tile;
  const Geom& g = a.g;
  uint32_t org[3], w[3];
  block_box(g, b, org, w);
  const uint32_t m = w[0] * w[1] * w[2];
  const float eb_f = a.st->eb_f, ebx2_f = a.st->ebx2_f, ebx2_r = a.st->ebx2_r;
  const int32_t r = (int32_t)a.radius;
  uint32_t err = 0;

  // ---- load and prequantize ------------------------------------------------------
  const float* __restrict__ x = a.x;
  const uint64_t ny = g.n[1], nx = g.n[2];
  const bool aligned = ((((uintptr_t)x) & 15) == 0) && (nx % 4 == 0);
  auto put_k = [&](uint32_t j, float v) {
    int32_t k;
    bool p;
    err |= prequant(v, eb_f, ebx2_f, ebx2_r, k, p);
    s_k[j] = k;
    if (p) atomicOr(&s_patch[j >> 5], 1u << (j & 31));
  };
  if (ND == 1) {
    const uint64_t base = org[2];
    if (m == (uint32_t)kSlots && aligned) {
      const float4* x4 = reinterpret_cast<const float4*>(x + base);
#pragma unroll
      for (int i = 0; i < 4; i++) {
        uint32_t f = tid + kConstructThreads * i;
        float4 v = __ldcs(&x4[f]);
        put_k(4 * f + 0, v.x);
        put_k(4 * f + 1, v.y);
        put_k(4 * f + 2, v.z);
        put_k(4 * f + 3, v.w);
      }
    } else {
      for (uint32_t j = tid; j < m; j += kConstructThreads) put_k(j, x[base + j]);
    }
  } else if (ND == 2) {
    const uint64_t base = (uint64_t)org[1] * nx + org[2];
    if (w[2] == 64 && aligned) {
#pragma unroll
      for (int i = 0; i < 4; i++) {
        uint32_t f = tid + kConstructThreads * i;
        uint32_t yy = f >> 4, c4 = f & 15;
        if (yy < w[1]) {
          float4 v = __ldcs(reinterpret_cast<const float4*>(x + base + yy * nx + 4 * c4));
          uint32_t j = yy * 64 + 4 * c4;
          put_k(j + 0, v.x);
          put_k(j + 1, v.y);
          put_k(j + 2, v.z);
          put_k(j + 3, v.w);
        }
      }
    } else {
      for (uint32_t j = tid; j < m; j += kConstructThreads) {
        uint32_t yy = j / w[2], xx = j - yy * w[2];
        put_k(j, x[base + yy * nx + xx]);
      }
    }
  } else {
    const uint64_t base = ((uint64_t)org[0] * ny + org[1]) * nx + org[2];
    if (w[2] == 16 && aligned) {
      const uint32_t rows = w[0] * w[1];
#pragma unroll
      for (int i = 0; i < 4; i++) {
        uint32_t f = tid + kConstructThreads * i;
        uint32_t row = f >> 2, c4 = f & 3;
        if (row < rows) {
          uint32_t zz = row / w[1], yy = row - zz * w[1];
          float4 v = __ldcs(reinterpret_cast<const float4*>(x + base + (zz * ny + yy) * nx + 4 * c4));
          uint32_t j = row * 16 + 4 * c4;
          put_k(j + 0, v.x);
          put_k(j + 1, v.y);
          put_k(j + 2, v.z);
          put_k(j + 3, v.w);
        }
      }
    } else {
      for (uint32_t j = tid; j < m; j += kConstructThreads) {
        uint32_t zz, yy, xx;
        dense_coords<3>(j, w[1], w[2], zz, yy, xx);
        put_k(j, x[base + (zz * ny + yy) * nx + xx]);
      }
    }
  }
  __syncthreads();

  // ---- Lorenzo residual (Sec. IV-B2 predictors, chunk-local) and postquant -------
  int32_t dl[kPer];
  const uint32_t sy = w[2], sz = w[1] * w[2];
#pragma unroll
  for (int i = 0; i < kPer; i++) {
    const uint32_t j = tid + kConstructThreads * i;
    int32_t delta = 0;
    uint16_t q = 0;
    bool in = j < m;
    if (in) {
      uint32_t zz, yy, xx;
      dense_coords<ND>(j, w[1], w[2], zz, yy, xx);
      const bool hx = (xx % Chunk<ND>::x) != 0;
      const bool hy = ND >= 2 && (yy % Chunk<ND>::y) != 0;
      const bool hz = ND >= 3 && (zz % Chunk<ND>::z) != 0;
      int32_t p;
      if (ND == 1) {
        p = hx ? s_k[j - 1] : 0;
      } else if (ND == 2) {
        p = (hx ? s_k[j - 1] : 0) + (hy ? s_k[j - sy] : 0) - ((hx && hy) ? s_k[j - sy - 1] : 0);
      } else {
        p = (hx ? s_k[j - 1] : 0) + (hy ? s_k[j - sy] : 0) + (hz ? s_k[j - sz] : 0) -
            ((hx && hy) ? s_k[j - sy - 1] : 0) - ((hx && hz) ? s_k[j - sz - 1] : 0) -
            ((hy && hz) ? s_k[j - sz - sy] : 0) + ((hx && hy && hz) ? s_k[j - sz - sy - 1] : 0);
      }
      delta = s_k[j] - p;
      q = (delta > -r && delta < r) ? (uint16_t)(delta + r) : (uint16_t)0;
    }
    dl[i] = delta;
    s_c[j] = q;  // zero beyond m
    uint32_t ob = __ballot_sync(~0u, in && q == 0);
    if ((tid & 31) == 0) s_outl[j >> 5] = ob;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kPer; i++) s_k[tid + kConstructThreads * i] = dl[i];

  // ---- record count per thread (contiguous 16 slots) and tile aggregate ----------
  const uint32_t lo = tid * kPer;
  const uint32_t ob = (s_outl[lo >> 5] >> (lo & 31)) & 0xffffu;
  const uint32_t pb = (s_patch[lo >> 5] >> (lo & 31)) & 0xffffu;
  uint64_t tile_total;
  const uint64_t my_off = block_excl_scan<uint64_t>((uint64_t)(__popc(ob) + __popc(pb)), s_scan, &tile_total);
  if (tid == 0) {
    lookback_publish(a.lb, b, tile_total);
    if (tile_total) {
      atomicAdd(&a.st->n_rec, (unsigned long long)tile_total);
      uint32_t np = 0;
      for (int i = 0; i < kSlots / 32; i++) np += __popc(s_patch[i]);
      if (np) atomicAdd(&a.st->n_patch, (unsigned long long)np);
    }
  }

  // ---- codes to the block-major stream (whole 4096-slot block, zero tail) --------
  {
    const uint4* src = reinterpret_cast<const uint4*>(s_c);
    uint4* dst = reinterpret_cast<uint4*>(a.codes + (uint64_t)b * kSlots);
    for (int i = tid; i < kSlots / 8; i += kConstructThreads) __stcg(&dst[i], src[i]);
  }

  // ---- runs: heads, lengths, histograms (code hist = sum of run lengths) ---------
#pragma unroll
  for (int i = 0; i < kPer; i++) {
    const uint32_t j = tid + kConstructThreads * i;
    const bool head = j < m && (j == 0 || s_c[j] != s_c[j - 1]);
    uint32_t hb = __ballot_sync(~0u, head);
    if ((tid & 31) == 0) s_head[j >> 5] = hb;
  }
  __syncthreads();
  if (tid < kSlots / 32) {
    uint32_t mask = s_head[tid];
    while (mask) {
      const int bit = __ffs(mask) - 1;
      mask &= mask - 1;
      const uint32_t j = tid * 32 + bit;
      uint32_t nxt;
      if (mask) {
        nxt = tid * 32 + (__ffs(mask) - 1);
      } else {
        nxt = m;
        for (int wd = tid + 1; wd < kSlots / 32; wd++) {
          uint32_t hm = s_head[wd];
          if (hm) {
            nxt = wd * 32 + (__ffs(hm) - 1);
            break;
          }
        }
      }
      const uint32_t len = nxt - j;
      const uint32_t v = s_c[j];
      add16(s_hc, v, len);
      add16(s_hv, v, 1u);
      add16(s_hl, len - 1, 1u);
    }
  }

  // ---- place records: exclusive prefix over tiles, then ordered writes -----------
  if (tid < 32) {
    uint64_t pre = lookback_warp(a.lb, b, tile_total, &a.st->status, a.spin_limit);
    if (tid == 0) s_prefix = pre;
  }
  __syncthreads();
  if (ob | pb) {
    uint64_t pos = s_prefix + my_off;
    uint32_t zz, yy, xx;
    for (int i = 0; i < kPer; i++) {
      const uint32_t j = lo + i;
      const uint32_t slot2 = (b * (uint32_t)kSlots + j) * 2u;
      if ((ob >> i) & 1u) {
        if (pos < a.rec_cap)
          reinterpret_cast<uint2*>(a.rec)[pos] = make_uint2(slot2, (uint32_t)s_k[j]);
        else
          err |= ERR_CAPACITY;
        pos++;
      }
      if ((pb >> i) & 1u) {
        dense_coords<ND>(j, w[1], w[2], zz, yy, xx);
        const uint64_t e = ((uint64_t)(org[0] + zz) * ny + (org[1] + yy)) * nx + (org[2] + xx);
        if (pos < a.rec_cap)
          reinterpret_cast<uint2*>(a.rec)[pos] = make_uint2(slot2 + 1u, __float_as_uint(x[e]));
        else
          err |= ERR_CAPACITY;
        pos++;
      }
    }
  }
  if (err) atomicOr(&a.st->status, err);
  flush16(s_hc, kNsymCode / 2, a.hist_code);
  flush16(s_hv, kNsymCode / 2, a.hist_val);
  flush16(s_hl, kNsymLen / 2, a.hist_len);
}

static size_t construct_smem_bytes() {
  return kSlots * 4 + kSlots * 2 + (kNsymCode + kNsymCode + kNsymLen) / 2 * 4 + 3 * (kSlots / 32) * 4 +
         33 * 8 + 16;
}

// =================================================================================
// canonical Huffman books (two-queue construction, Sec. II-A Step-6 via cuSZ)
// =================================================================================

constexpr int kBookThreads = 1024;

__device__ void bitonic_sort_u64(uint64_t* k, int P) {
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = threadIdx.x; t < P / 2; t += blockDim.x) {
        int i = 2 * t - (t & (stride - 1));
        int j = i + stride;
        bool up = (i & size) == 0;
        uint64_t a = k[i], c = k[j];
        if ((a > c) == up) {
          k[i] = c;
          k[j] = a;
        }
      }
      __syncthreads();
    }
  }
}

// One CTA per book: 0 quant codes [1024], 1 run values [1024], 2 run lengths [4096].
__global__ __launch_bounds__(kBookThreads) void codebook_kernel(BookArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int book = blockIdx.x;
  const int nsym = book == 2 ? kNsymLen : kNsymCode;
  const uint32_t* hist = book == 0 ? a.hist_code : (book == 1 ? a.hist_val : a.hist_len);
  uint8_t* len_out = a.lens + (book == 0 ? 0 : (book == 1 ? kNsymCode : 2 * kNsymCode));
  uint64_t* code_out = a.codes + (book == 0 ? 0 : (book == 1 ? kNsymCode : 2 * kNsymCode));

  uint8_t* s_len = smem;                                                // 4096
  uint64_t* s_key = reinterpret_cast<uint64_t*>(smem + kNsymLen);       // 4096 u64
  uint32_t* s_w = reinterpret_cast<uint32_t*>(s_key);                   // 8192 u32 (aliases)
  uint16_t* s_sym = reinterpret_cast<uint16_t*>(s_key + kNsymLen);      // 4096
  uint16_t* s_anc = s_sym + kNsymLen;                                   // 8192
  uint16_t* s_dep = s_anc + 2 * kNsymLen;                               // 8192
  __shared__ uint32_t s_L;
  __shared__ CanonSmem cs;
  const int tid = threadIdx.x;

  if (tid == 0) s_L = 0;
  for (int s = tid; s < nsym; s += blockDim.x) s_len[s] = 0;
  __syncthreads();
  for (int s = tid; s < nsym; s += blockDim.x) {
    uint32_t f = hist[s];
    if (f) {
      uint32_t p = atomicAdd(&s_L, 1u);
      s_key[p] = ((uint64_t)f << 12) | (uint64_t)s;
    }
  }
  __syncthreads();
  const int L = (int)s_L;
  if (L == 1) {
    if (tid == 0) s_len[s_key[0] & 0xfff] = 1;
  } else if (L > 1) {
    int P = 1;
    while (P < L) P <<= 1;
    for (int i = L + tid; i < P; i += blockDim.x) s_key[i] = ~0ull;
    __syncthreads();
    bitonic_sort_u64(s_key, P);
    // leaves: weights and symbols in (frequency, symbol) order
    uint64_t kk[4];
    int cntk = 0;
    for (int i = tid; i < L; i += blockDim.x) kk[cntk++] = s_key[i];
    __syncthreads();
    cntk = 0;
    for (int i = tid; i < L; i += blockDim.x) {
      s_w[i] = (uint32_t)(kk[cntk] >> 12);
      s_sym[i] = (uint16_t)(kk[cntk] & 0xfff);
      cntk++;
    }
    __syncthreads();
    const int nn = 2 * L - 1;
    if (tid == 0) {
      // two queues: leaves [qi, L), internal nodes [qj, nxt); a weight tie takes the leaf
      int qi = 0, qj = L, nxt = L;
      uint32_t wi = s_w[0], wj = 0;
      while (nxt < nn) {
        int pk[2];
        uint32_t pw[2];
#pragma unroll
        for (int t = 0; t < 2; t++) {
          if (qi < L && (qj >= nxt || wi <= wj)) {
            pk[t] = qi;
            pw[t] = wi;
            qi++;
            wi = qi < L ? s_w[qi] : 0u;
          } else {
            pk[t] = qj;
            pw[t] = wj;
            qj++;
            wj = qj < nxt ? s_w[qj] : 0u;
          }
        }
        const uint32_t sum = pw[0] + pw[1];
        s_w[nxt] = sum;
        if (qj == nxt) wj = sum;  // the internal queue was empty: new node is its front
        s_anc[pk[0]] = (uint16_t)nxt;
        s_anc[pk[1]] = (uint16_t)nxt;
        nxt++;
      }
      s_anc[nn - 1] = (uint16_t)(nn - 1);
    }
    __syncthreads();
    // depths by pointer jumping
    for (int i = tid; i < nn; i += blockDim.x) s_dep[i] = (i == nn - 1) ? 0 : 1;
    __syncthreads();
    for (int step = 1; step < nn; step <<= 1) {
      uint16_t na[8], nd[8];
      int c = 0;
      for (int i = tid; i < nn; i += blockDim.x) {
        uint16_t an = s_anc[i];
        nd[c] = s_dep[i] + s_dep[an];
        na[c] = s_anc[an];
        c++;
      }
      __syncthreads();
      c = 0;
      for (int i = tid; i < nn; i += blockDim.x) {
        s_dep[i] = nd[c];
        s_anc[i] = na[c];
        c++;
      }
      __syncthreads();
    }
    for (int i = tid; i < L; i += blockDim.x) {
      uint16_t d = s_dep[i];
      if (d > kMaxLen) atomicOr(&a.st->status, ERR_RANGE);
      s_len[s_sym[i]] = (uint8_t)d;
    }
  }
  __syncthreads();
  for (int s = tid; s < nsym; s += blockDim.x) len_out[s] = s_len[s];
  uint16_t* wcnt = reinterpret_cast<uint16_t*>(s_key);  // tree storage is free now
  canonical_build(s_len, nsym, &cs, wcnt, code_out, nullptr);
}

static size_t codebook_smem_bytes() { return kNsymLen + kNsymLen * 8 + kNsymLen * 2 + 2 * kNsymLen * 2 * 2; }

// =================================================================================
// per-block selection and encoding
// =================================================================================

constexpr int kEncThreads = 256;
constexpr int kBufWords = 4096;  // 16 KB payload assembly buffer

// MSB-first bits of `code` (len bits) at bit offset off of a u32 word buffer
__device__ __forceinline__ void put_bits(uint32_t* buf, uint32_t off, uint64_t code, int len) {
  uint32_t wd = off >> 5;
  int sh = off & 31;
  int rem = len;
  while (rem > 0) {
    int take = min(rem, 32 - sh);
    uint32_t chunk = (uint32_t)((code >> (rem - take)) & ((1ull << take) - 1ull));
    atomicOr(&buf[wd], chunk << (32 - sh - take));
    rem -= take;
    wd++;
    sh = 0;
  }
}

// Encode syms[0..cnt) (+sym_add) with a book into buf (zeroed) from bit 0; each thread
// takes a contiguous share; returns total bits.
__device__ uint32_t encode_seq(const uint16_t* syms, int cnt, int sym_add, const uint8_t* __restrict__ lens,
                               const uint64_t* __restrict__ codes, uint32_t* buf, uint32_t* scan) {
  const int per = (cnt + blockDim.x - 1) / blockDim.x;
  const int lo = min(cnt, (int)threadIdx.x * per), hi = min(cnt, lo + per);
  uint32_t bits = 0;
  for (int i = lo; i < hi; i++) bits += __ldg(&lens[syms[i] + sym_add]);
  uint32_t total;
  uint32_t off = block_excl_scan<uint32_t>(bits, scan, &total);
  for (int i = lo; i < hi; i++) {
    const int s = syms[i] + sym_add;
    const int l = __ldg(&lens[s]);
    put_bits(buf, off, __ldg(&codes[s]), l);
    off += l;
  }
  __syncthreads();
  return total;
}

__device__ int mlp_pick_warp(const float* __restrict__ w, const float* f) {
  const int lane = threadIdx.x & 31;
  const float* W1 = w;
  const float* b1 = W1 + 32 * 8;
  const float* W2 = b1 + 32;
  const float* b2 = W2 + 32 * 32;
  const float* W3 = b2 + 32;
  const float* b3 = W3 + 3 * 32;
  float acc = __ldg(&b1[lane]);
#pragma unroll
  for (int j = 0; j < 8; j++) acc = fmaf(__ldg(&W1[lane * 8 + j]), f[j], acc);
  const float h1 = acc > 0.0f ? acc : 0.0f;
  acc = __ldg(&b2[lane]);
#pragma unroll
  for (int j = 0; j < 32; j++) acc = fmaf(__ldg(&W2[lane * 32 + j]), __shfl_sync(~0u, h1, j), acc);
  const float h2 = acc > 0.0f ? acc : 0.0f;
  const int o = lane < 3 ? lane : 0;
  acc = __ldg(&b3[o]);
#pragma unroll
  for (int j = 0; j < 32; j++) acc = fmaf(__ldg(&W3[o * 32 + j]), __shfl_sync(~0u, h2, j), acc);
  const float y0 = __shfl_sync(~0u, acc, 0), y1 = __shfl_sync(~0u, acc, 1), y2 = __shfl_sync(~0u, acc, 2);
  int c = 0;
  float best = y0;
  if (y1 < best) {
    c = 1;
    best = y1;
  }
  if (y2 < best) c = 2;
  return c;
}

__global__ __launch_bounds__(kEncThreads) void encode_kernel(EncodeArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* s_c = reinterpret_cast<uint16_t*>(smem);        // 4096 codes
  uint16_t* s_rv = s_c + kSlots;                            // run values
  uint16_t* s_rl = s_rv + kSlots;                           // run lengths
  uint32_t* s_buf = reinterpret_cast<uint32_t*>(s_rl + kSlots);  // 4096 words
  uint32_t* s_head = s_buf + kBufWords;                     // 128
  uint32_t* s_woff = s_head + kSlots / 32;                  // 128
  uint32_t* s_scan = s_woff + kSlots / 32;                  // 33
  uint64_t* s_scan64 = reinterpret_cast<uint64_t*>(s_scan + 34);  // 33
  __shared__ uint32_t s_tile, s_codec;
  __shared__ uint64_t s_prefix;
  __shared__ float s_feat[8];

  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(&a.st->ticket_encode, 1u);
  __syncthreads();
  const uint32_t b = s_tile;
  uint32_t org[3], w[3];
  block_box(a.g, b, org, w);
  const uint32_t m = w[0] * w[1] * w[2];
  const int sel = a.select;
  const uint32_t r = a.radius;
  const uint8_t* clen = a.lens;
  const uint8_t* vlen = a.lens + kNsymCode;
  const uint8_t* llen = a.lens + 2 * kNsymCode;
  const uint64_t* ccode = a.bcodes;
  const uint64_t* vcode = a.bcodes + kNsymCode;
  const uint64_t* lcode = a.bcodes + 2 * kNsymCode;

  {
    const uint4* src = reinterpret_cast<const uint4*>(a.codes + (uint64_t)b * kSlots);
    uint4* dst = reinterpret_cast<uint4*>(s_c);
    for (int i = tid; i < kSlots / 8; i += kEncThreads) dst[i] = __ldcs(&src[i]);
  }
  __syncthreads();

  // runs (needed by every mode except forced HUFF)
  const bool need_runs = sel != SEL_HUFF;
  uint32_t nr = 0;
  if (need_runs) {
    for (int i = 0; i < kSlots / kEncThreads; i++) {
      const uint32_t j = tid + kEncThreads * i;
      const bool head = j < m && (j == 0 || s_c[j] != s_c[j - 1]);
      const uint32_t hb = __ballot_sync(~0u, head);
      if ((tid & 31) == 0) s_head[j >> 5] = hb;
    }
    __syncthreads();
    uint32_t tot;
    const uint32_t wo = block_excl_scan<uint32_t>(tid < kSlots / 32 ? __popc(s_head[tid]) : 0u, s_scan, &tot);
    nr = tot;
    if (tid < kSlots / 32) {
      uint32_t mask = s_head[tid];
      uint32_t ri = wo;
      while (mask) {
        const int bit = __ffs(mask) - 1;
        mask &= mask - 1;
        const uint32_t j = tid * 32 + bit;
        uint32_t nxt;
        if (mask) {
          nxt = tid * 32 + (__ffs(mask) - 1);
        } else {
          nxt = m;
          for (int wd = tid + 1; wd < kSlots / 32; wd++) {
            uint32_t hm = s_head[wd];
            if (hm) {
              nxt = wd * 32 + (__ffs(hm) - 1);
              break;
            }
          }
        }
        s_rv[ri] = s_c[j];
        s_rl[ri] = (uint16_t)(nxt - j);
        ri++;
      }
    }
    __syncthreads();
  }

  // sizes
  const uint32_t S = (m + kHuffSeg - 1) / kHuffSeg;
  const uint32_t hdr_bytes = (2 * S + 3) & ~3u;
  uint64_t size_h = ~0ull, size_r = ~0ull, size_rh = ~0ull;
  if (sel == SEL_HUFF || sel == SEL_EXHAUSTIVE) {
    uint32_t sb[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < kSlots / kEncThreads; i++) {
      const uint32_t j = tid + kEncThreads * i;
      if (j < m) sb[i >> 2] += __ldg(&clen[s_c[j]]);
    }
    uint64_t sz = hdr_bytes;
    for (int s = 0; s < 4; s++) {
      uint32_t t = block_sum<uint32_t>(sb[s], s_scan);
      sz += 4ull * ((t + 31) / 32);
    }
    size_h = sz;
  }
  if (sel == SEL_RLE || sel == SEL_EXHAUSTIVE) size_r = 4ull * nr;
  uint32_t vbits = 0, lbits = 0;
  if (sel == SEL_RLE_HUFF || sel == SEL_EXHAUSTIVE) {
    uint32_t vb = 0, lb = 0;
    for (uint32_t i = tid; i < nr; i += kEncThreads) {
      vb += __ldg(&vlen[s_rv[i]]);
      lb += __ldg(&llen[s_rl[i] - 1]);
    }
    vbits = block_sum<uint32_t>(vb, s_scan);
    lbits = block_sum<uint32_t>(lb, s_scan);
    size_rh = 8ull + 4ull * ((vbits + 31) / 32) + 4ull * ((lbits + 31) / 32);
  }

  // selection
  if (sel == SEL_HEURISTIC || sel == SEL_LEARNED) {
    // block histogram from the runs, then the statistics of the features
    uint32_t* s_hist = s_buf;  // 1024 words
    for (int i = tid; i < kNsymCode; i += kEncThreads) s_hist[i] = 0;
    __syncthreads();
    for (uint32_t i = tid; i < nr; i += kEncThreads) atomicAdd(&s_hist[s_rv[i]], (uint32_t)s_rl[i]);
    __syncthreads();
    uint64_t S_ = 0, absd = 0;
    uint32_t f1 = 0;
    for (int c = tid; c < kNsymCode; c += kEncThreads) {
      const uint32_t h = s_hist[c];
      if (h) {
        S_ += (uint64_t)h * log2_q16(h);
        f1 = max(f1, h);
        if (c != 0) absd += (uint64_t)h * (uint64_t)abs((int)c - (int)r);
      }
    }
    S_ = block_sum<uint64_t>(S_, s_scan64);
    absd = block_sum<uint64_t>(absd, s_scan64);
    f1 = block_max_u32(f1, s_scan);
    const int64_t Lm = log2_q16(m);
    const int64_t NH = (int64_t)m * Lm - (int64_t)S_;
    if (sel == SEL_HEURISTIC) {
      if (tid == 0) {
        int64_t Rm = 0;
        if (10ll * f1 > 4ll * m) {
          const int64_t rest = (int64_t)m - f1;
          Rm = (int64_t)m * 65536 + (int64_t)f1 * log2_q16(f1) +
               (rest > 0 ? rest * (int64_t)log2_q16((uint64_t)rest) : 0) - (int64_t)m * Lm;
          if (Rm < 0) Rm = 0;
        }
        const int64_t est = NH + Rm;
        s_codec = (100 * est <= 109ll * (int64_t)m * 65536) ? CODEC_RLE_HUFF : CODEC_HUFF;
      }
    } else {
      uint32_t var8 = 0;
      for (uint32_t j = tid; j + 8 < m; j += kEncThreads) var8 += s_c[j] != s_c[j + 8];
      var8 = block_sum<uint32_t>(var8, s_scan);
      if (tid == 0) {
        const uint32_t zero = s_hist[r];
        const uint32_t outl = s_hist[0];
        uint32_t near1 = s_hist[r] + (r + 1 < 2 * r ? s_hist[r + 1] : 0u) + (r - 1 > 0 ? s_hist[r - 1] : 0u);
        const float fm = (float)m;
        s_feat[0] = (float)zero / fm;
        s_feat[1] = (float)NH / (float)((uint64_t)m * 65536ull);
        s_feat[2] = (float)f1 / fm;
        s_feat[3] = (float)near1 / fm;
        s_feat[4] = (float)nr / fm;
        s_feat[5] = (float)outl / fm;
        s_feat[6] = (float)absd / (float)((uint64_t)m * r);
        s_feat[7] = (float)var8 / fm;
      }
      __syncthreads();
      if (tid < 32) {
        const int c = mlp_pick_warp(a.mlp_w, s_feat);
        if (tid == 0) s_codec = (uint32_t)c;
      }
      if (a.feat_out && tid < 8) a.feat_out[(uint64_t)b * 8 + tid] = s_feat[tid];
    }
    __syncthreads();
  } else if (tid == 0) {
    if (sel <= SEL_RLE_HUFF) {
      s_codec = (uint32_t)sel;
    } else {
      int c = CODEC_HUFF;
      uint64_t best = size_h;
      if (size_rh < best) {
        c = CODEC_RLE_HUFF;
        best = size_rh;
      }
      if (size_r < best) c = CODEC_RLE;
      s_codec = (uint32_t)c;
    }
  }
  __syncthreads();
  const int codec = (int)s_codec;
  // exact size of the chosen codec (computed here if the mode skipped it)
  if (codec == CODEC_HUFF && size_h == ~0ull) {
    uint32_t sb[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < kSlots / kEncThreads; i++) {
      const uint32_t j = tid + kEncThreads * i;
      if (j < m) sb[i >> 2] += __ldg(&clen[s_c[j]]);
    }
    uint64_t sz = hdr_bytes;
    for (int s = 0; s < 4; s++) {
      uint32_t t = block_sum<uint32_t>(sb[s], s_scan);
      sz += 4ull * ((t + 31) / 32);
    }
    size_h = sz;
  }
  if (codec == CODEC_RLE_HUFF && size_rh == ~0ull) {
    uint32_t vb = 0, lb = 0;
    for (uint32_t i = tid; i < nr; i += kEncThreads) {
      vb += __ldg(&vlen[s_rv[i]]);
      lb += __ldg(&llen[s_rl[i] - 1]);
    }
    vbits = block_sum<uint32_t>(vb, s_scan);
    lbits = block_sum<uint32_t>(lb, s_scan);
    size_rh = 8ull + 4ull * ((vbits + 31) / 32) + 4ull * ((lbits + 31) / 32);
  }
  const uint64_t size = codec == CODEC_HUFF ? size_h : (codec == CODEC_RLE ? 4ull * nr : size_rh);
  if (tid == 0) {
    lookback_publish(a.lb, b, size);
    atomicAdd(&a.st->ncodec[codec], 1u);
    atomicAdd(&a.st->payload, (unsigned long long)size);
  }
  __syncthreads();

  // payload assembly in shared memory (every chosen size fits 16 KB unless a forced
  // Huffman mode meets codes longer than 32 bits on average; those blocks go direct)
  const bool in_smem = size <= (uint64_t)kBufWords * 4;
  if (in_smem && codec != CODEC_RLE) {
    for (int i = tid; i < kBufWords; i += kEncThreads) s_buf[i] = 0;
    __syncthreads();
    if (codec == CODEC_HUFF) {
      uint32_t wo = hdr_bytes / 4;
      for (uint32_t s = 0; s < S; s++) {
        const int cnt = (int)min((uint32_t)kHuffSeg, m - s * kHuffSeg);
        const uint32_t bits = encode_seq(s_c + s * kHuffSeg, cnt, 0, clen, ccode, s_buf + wo, s_scan);
        const uint32_t nw = (bits + 31) / 32;
        if (tid == 0) reinterpret_cast<uint16_t*>(s_buf)[s] = (uint16_t)nw;
        wo += nw;
      }
    } else {
      const uint32_t vw = (vbits + 31) / 32;
      if (tid == 0) {
        s_buf[0] = nr;
        s_buf[1] = vw;
      }
      encode_seq(s_rv, (int)nr, 0, vlen, vcode, s_buf + 2, s_scan);
      encode_seq(s_rl, (int)nr, -1, llen, lcode, s_buf + 2 + vw, s_scan);
    }
    __syncthreads();
  }

  // placement
  if (tid < 32) {
    const uint64_t pre = lookback_warp(a.lb, b, size, &a.st->status, a.spin_limit);
    if (tid == 0) s_prefix = pre;
  }
  __syncthreads();
  const uint64_t off_pay = a.off_rec + 8ull * a.st->n_rec;
  const uint64_t dst_off = off_pay + s_prefix;
  if (tid == 0) {
    a.ar[a.off_codec + b] = (uint8_t)codec;
    if (a.off_bb + 4ull * b + 4 <= a.cap) reinterpret_cast<uint32_t*>(a.ar + a.off_bb)[b] = (uint32_t)size;
  }
  if (dst_off + size > a.cap) {
    if (tid == 0) atomicOr(&a.st->status, ERR_CAPACITY);
    return;
  }
  uint32_t* dst = reinterpret_cast<uint32_t*>(a.ar + dst_off);
  const uint32_t nwords = (uint32_t)(size / 4);
  if (codec == CODEC_RLE) {
    uint16_t* d16 = reinterpret_cast<uint16_t*>(dst);
    for (uint32_t i = tid; i < nr; i += kEncThreads) {
      d16[i] = s_rv[i];
      d16[nr + i] = s_rl[i];
    }
  } else if (in_smem) {
    for (uint32_t i = tid; i < nwords; i += kEncThreads) dst[i] = s_buf[i];
  } else {
    // direct path: zero the block's own region, then OR the bits in place
    for (uint32_t i = tid; i < nwords; i += kEncThreads) dst[i] = 0u;
    __syncthreads();
    if (codec == CODEC_HUFF) {
      uint32_t wo = hdr_bytes / 4;
      for (uint32_t s = 0; s < S; s++) {
        const int cnt = (int)min((uint32_t)kHuffSeg, m - s * kHuffSeg);
        const uint32_t bits = encode_seq(s_c + s * kHuffSeg, cnt, 0, clen, ccode, dst + wo, s_scan);
        const uint32_t nw = (bits + 31) / 32;
        if (tid == 0) atomicOr(&dst[s >> 1], nw << ((s & 1) * 16));
        wo += nw;
      }
    } else {
      const uint32_t vw = (vbits + 31) / 32;
      if (tid == 0) {
        dst[0] = nr;
        dst[1] = vw;
      }
      encode_seq(s_rv, (int)nr, 0, vlen, vcode, dst + 2, s_scan);
      encode_seq(s_rl, (int)nr, -1, llen, lcode, dst + 2 + vw, s_scan);
    }
  }
}

static size_t encode_smem_bytes() { return kSlots * 2 * 3 + kBufWords * 4 + 2 * (kSlots / 32) * 4 + 34 * 4 + 33 * 8 + 16; }

// =================================================================================
// header, section padding and books
// =================================================================================
__global__ void finalize_kernel(FinalizeArgs a) {
  __shared__ uint32_t s_hdr[kHdr / 4];
  __shared__ uint64_t s_total, s_off_books;
  __shared__ uint32_t s_flags;
  DevState* st = a.st;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const uint64_t n_rec = st->n_rec, payload = st->payload;
    const uint32_t flags = (st->ncodec[CODEC_HUFF] ? 1u : 0u) | (st->ncodec[CODEC_RLE_HUFF] ? 2u : 0u);
    const uint64_t off_pay = a.off_rec + 8 * n_rec;
    const uint64_t off_books = off_pay + ((payload + 7) & ~7ull);
    const uint64_t total = off_books + ((flags & 1) ? kNsymCode : 0) + ((flags & 2) ? kNsymCode + kNsymLen : 0);
    s_total = total;
    s_off_books = off_books;
    s_flags = flags;
    st->total = total;
    if (total > a.cap) atomicOr(&st->status, ERR_CAPACITY);
    for (int i = 0; i < kHdr / 4; i++) s_hdr[i] = 0;
    unsigned char* h = reinterpret_cast<unsigned char*>(s_hdr);
    auto put32 = [&](int off, uint32_t v) { memcpy(h + off, &v, 4); };
    auto put64 = [&](int off, uint64_t v) { memcpy(h + off, &v, 8); };
    put32(0, kMagic);
    h[4] = (unsigned char)(kVersion & 0xff);
    h[5] = (unsigned char)(kVersion >> 8);
    h[6] = (unsigned char)a.ndim;
    h[7] = (unsigned char)a.eb_mode;
    for (int i = 0; i < 3; i++) put64(8 + 8 * i, i < a.ndim ? a.dims[i] : 0ull);
    double eu = a.eb_user, ed = st->eb_d;
    memcpy(h + 32, &eu, 8);
    memcpy(h + 40, &ed, 8);
    float ef = st->eb_f;
    memcpy(h + 48, &ef, 4);
    put32(52, a.radius);
    put32(56, (uint32_t)kHuffSeg);
    put32(60, flags);
    put64(64, a.nblk);
    put64(72, n_rec);
    put64(80, n_rec - st->n_patch);
    put64(88, st->n_patch);
    put64(96, payload);
    put64(104, total);
    put32(112, (uint32_t)a.select);
    for (int i = 0; i < 3; i++) put32(116 + 4 * i, st->ncodec[i]);
  }
  __syncthreads();
  if (s_total > a.cap) return;
  uint8_t* ar = a.ar;
  for (int i = tid; i < kHdr / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(ar)[i] = s_hdr[i];
  // zero padding: codec section, blk_bytes section, payload tail
  for (uint64_t i = kHdr + a.nblk + tid; i < a.off_bb; i += blockDim.x) ar[i] = 0;
  for (uint64_t i = a.off_bb + 4ull * a.nblk + tid; i < a.off_rec; i += blockDim.x) ar[i] = 0;
  const uint64_t pay_end = a.off_rec + 8 * st->n_rec + st->payload;
  for (uint64_t i = pay_end + tid; i < s_off_books; i += blockDim.x) ar[i] = 0;
  uint64_t o = s_off_books;
  if (s_flags & 1) {
    for (int i = tid; i < kNsymCode; i += blockDim.x) ar[o + i] = a.lens[i];
    o += kNsymCode;
  }
  if (s_flags & 2) {
    for (int i = tid; i < kNsymCode + kNsymLen; i += blockDim.x) ar[o + i] = a.lens[kNsymCode + i];
  }
}

// =================================================================================
// launchers
// =================================================================================
cudaError_t launch_abs_params(DevState* st, double eb, cudaStream_t s) {
  trace_begin(K_PARAMS, s);
  abs_params_kernel<<<1, 32, 0, s>>>(st, eb);
  trace_end(K_PARAMS, s);
  return cudaGetLastError();
}

cudaError_t launch_range(const float* x, uint64_t n, DevState* st, int mode, double eb, cudaStream_t s) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t want = (n / 4 + 255) / 256;
  uint64_t grid = want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8;
  if (grid == 0) grid = 1;
  trace_begin(K_RANGE, s);
  range_kernel<<<(unsigned)grid, 256, 0, s>>>(x, n, st, mode, eb);
  trace_end(K_RANGE, s);
  return cudaGetLastError();
}

cudaError_t launch_construct(int ndim, const ConstructArgs& a, cudaStream_t s) {
  const size_t sm = construct_smem_bytes();
  trace_begin(K_CONSTRUCT, s);
  if (ndim == 1) {
    construct_kernel<1><<<a.g.nblk, kConstructThreads, sm, s>>>(a);
  } else if (ndim == 2) {
    construct_kernel<2><<<a.g.nblk, kConstructThreads, sm, s>>>(a);
  } else {
    construct_kernel<3><<<a.g.nblk, kConstructThreads, sm, s>>>(a);
  }
  trace_end(K_CONSTRUCT, s);
  return cudaGetLastError();
}

cudaError_t launch_codebook(const BookArgs& a, cudaStream_t s) {
  const size_t sm = codebook_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(codebook_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  trace_begin(K_CODEBOOK, s);
  codebook_kernel<<<3, kBookThreads, sm, s>>>(a);
  trace_end(K_CODEBOOK, s);
  return cudaGetLastError();
}

cudaError_t launch_encode(const EncodeArgs& a, cudaStream_t s) {
  trace_begin(K_ENCODE, s);
  encode_kernel<<<a.g.nblk, kEncThreads, encode_smem_bytes(), s>>>(a);
  trace_end(K_ENCODE, s);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs& a, cudaStream_t s) {
  trace_begin(K_FINALIZE, s);
  finalize_kernel<<<1, 256, 0, s>>>(a);
  trace_end(K_FINALIZE, s);
  return cudaGetLastError();
}

}  // namespace cszp
