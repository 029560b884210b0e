// Compression kernels of cszp (sm_103a).
//
// Pipeline (one stream, no host round trip until the end):
//   range_kernel / abs_params_kernel  value range (REL) and the FP32 error bound
//   construct_kernel (construct.cu,   prequant + chunk-local Lorenzo + postquant,
//     device code construct_body.cuh) record counts, bit words, residuals, histograms
//   codebook_kernel                   three canonical Huffman books; a fourth CTA
//                                     scans the blocks' record counts
//   encode_kernel                     per block: its records, exact sizes or heuristic /
//                                     MLP pick, payload placement by decoupled
//                                     look-back, payload
//   (the block counted last)          header, padding, books
// Batches run the same bodies either as one launch per stage (the *_batch kernels)
// or as the phases of one persistent kernel (batch_persistent_kernel).
#include "common.cuh"
#include "construct_body.cuh"
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

// Double-precision fields: eb_d as above (from the double range), the quantization
// step fl64(2 eb_d (1 - 2^-24)) and its inverse; eb_f is the largest float <= eb_d
// (informational, in the header).  Degenerate bounds -> ERR_ARG.
__device__ void derive_eb_d(DevState* st, int mode, double eb, double vmin, double vmax) {
  const double d = mode == 0 ? eb : __dmul_rn(eb, __dsub_rn(vmax, vmin));
  const double stp = __dmul_rn(__dmul_rn(2.0, d), kStepShrink);
  const double r = __ddiv_rn(1.0, stp);
  st->eb_d = d;
  st->eb_f = __double2float_rd(d);
  st->step_d = stp;
  st->rstep_d = r;
  if (!(d > 0.0) || !isfinite(d) || !(stp > 0.0) || !isfinite(stp) || !(r > 0.0) || !isfinite(r))
    atomicOr(&st->status, ERR_ARG);
}

__global__ void abs_params_d_kernel(DevState* st, double eb) {
  if (threadIdx.x == 0 && blockIdx.x == 0) derive_eb_d(st, 0, eb, 0.0, 0.0);
}

__device__ __forceinline__ unsigned long long order_key_d(double f) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(f);
  return (b >> 63) ? ~b : (b | (1ull << 63));
}
__device__ __forceinline__ double key_to_double(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & ~(1ull << 63)) : ~k));
}

// Min / max of a double field (grid-stride, 16-byte loads); the last CTA derives the
// bound and the step.
__global__ __launch_bounds__(256) void range_d_kernel(const double* __restrict__ x, uint64_t n, DevState* st,
                                                      int mode, double eb) {
  __shared__ unsigned long long s_red[2][33];
  __shared__ bool s_last;
  unsigned long long lo_inv = 0, hi = 0;
  uint32_t bad = 0;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  const bool vec = (((uintptr_t)x) & 15) == 0;
  const uint64_t nvec = vec ? n / 2 : 0;
  const double2* x2 = reinterpret_cast<const double2*>(x);
  auto take = [&](double a) {
    if (!isfinite(a)) {
      bad = 1;
    } else {
      const unsigned long long key = order_key_d(a);
      lo_inv = max(lo_inv, ~key);
      hi = max(hi, key);
    }
  };
  for (uint64_t i = tid; i < nvec; i += nth) {
    const double2 v = __ldcs(&x2[i]);
    take(v.x);
    take(v.y);
  }
  for (uint64_t i = nvec * 2 + tid; i < n; i += nth) take(x[i]);
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
    unsigned long long a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      a = max(a, s_red[0][w]);
      b = max(b, s_red[1][w]);
    }
    atomicMax(&st->range64_lo_inv, a);
    atomicMax(&st->range64_hi, b);
    __threadfence();
    s_last = atomicAdd(&st->range_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    const unsigned long long a = atomicAdd(&st->range64_lo_inv, 0ull);
    const unsigned long long b = atomicAdd(&st->range64_hi, 0ull);
    if (b == 0) {  // nothing finite was seen
      atomicOr(&st->status, ERR_NONFINITE);
      return;
    }
    derive_eb_d(st, mode, eb, key_to_double(~a), key_to_double(b));
  }
}

// Grid-stride min/max with float4 loads; non-finite values are flagged.  The last CTA
// to finish derives the error bound.
// ready (batched persistent kernel only, else nullptr): released as 1 by the last CTA
// once the bound is derived or found impossible.
__device__ __forceinline__ void range_body(const float* __restrict__ x, uint64_t n, DevState* st, int mode, double eb,
                           uint32_t cta, uint32_t nctas, uint32_t* ready = nullptr) {
  __shared__ uint32_t s_red[2][33];
  __shared__ bool s_last;
  uint32_t lo_inv = 0, hi = 0, bad = 0;
  const uint64_t tid = cta * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)nctas * blockDim.x;
  const bool vec = (((uintptr_t)x) & 15) == 0;
  uint64_t nvec = vec ? n / 4 : 0;
  const float4* x4 = reinterpret_cast<const float4*>(x);
  auto take = [&](float4 v) {
    const float a[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (!isfinite(a[k])) {
        bad = 1;
      } else {
        const uint32_t key = order_key(a[k]);
        lo_inv = max(lo_inv, ~key);
        hi = max(hi, key);
      }
    }
  };
  // four independent 16-byte loads in flight per thread per iteration
  uint64_t i = tid;
  for (; i + 3 * nth < nvec; i += 4 * nth) {
    const float4 v0 = __ldcs(&x4[i]), v1 = __ldcs(&x4[i + nth]), v2 = __ldcs(&x4[i + 2 * nth]),
                 v3 = __ldcs(&x4[i + 3 * nth]);
    take(v0);
    take(v1);
    take(v2);
    take(v3);
  }
  for (; i < nvec; i += nth) take(__ldcs(&x4[i]));
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
    s_last = atomicAdd(&st->range_done, 1u) == nctas - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    uint32_t a = atomicAdd(&st->range_lo_inv, 0u);
    uint32_t b = atomicAdd(&st->range_hi, 0u);
    if (b == 0) {  // nothing finite was seen
      atomicOr(&st->status, ERR_NONFINITE);
    } else {
      derive_eb(st, mode, eb, key_to_float(~a), key_to_float(b));
    }
    if (ready) release_flag(ready);
  }
}

__global__ __launch_bounds__(256) void range_kernel(const float* __restrict__ x, uint64_t n, DevState* st, int mode,
                                                    double eb) {
  range_body(x, n, st, mode, eb, blockIdx.x, gridDim.x);
}

// Batch: cta0[f] .. cta0[f+1]-1 are field f's CTAs; an ABS field has one CTA, which
// only derives the bound.
__global__ __launch_bounds__(256) void range_batch_kernel(const RangeTask* __restrict__ tasks,
                                                          const uint32_t* __restrict__ cta0, int nfields) {
  const uint32_t c = blockIdx.x;
  int lo = 0, hi = nfields - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cta0[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  const RangeTask& t = tasks[lo];
  if (t.mode == 0) {
    if (threadIdx.x == 0) derive_eb(t.st, 0, t.eb, 0.0f, 0.0f);
    return;
  }
  range_body(t.x, t.n, t.st, t.mode, t.eb, c - cta0[lo], cta0[lo + 1] - cta0[lo]);
}


// =================================================================================
// canonical Huffman books (two-queue construction, Sec. II-A Step-6 via cuSZ)
// =================================================================================

constexpr int kBookThreads = 1024;

// Ascending sort of L distinct keys by merging runs: an element's place in the merged
// run is its index in its own run plus the number of smaller keys in the partner run
// (binary search).  a holds the keys on entry and on exit; b is scratch of L keys.
__device__ void rank_merge_sort_u64(uint64_t* a, uint64_t* b, int L) {
  uint64_t* src = a;
  uint64_t* dst = b;
  for (int run = 1; run < L; run <<= 1) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
      const uint64_t k = src[i];
      const int r = i / run;
      const int r0 = r * run;
      const bool left = (r & 1) == 0;
      const int p0 = left ? r0 + run : r0 - run;
      const int pn = left ? max(0, min(run, L - p0)) : run;
      int lo = 0, hi = pn;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (src[p0 + mid] < k) lo = mid + 1;
        else hi = mid;
      }
      dst[(left ? r0 : p0) + (i - r0) + lo] = k;
    }
    __syncthreads();
    uint64_t* t = src;
    src = dst;
    dst = t;
  }
  if (src != a) {
    for (int i = threadIdx.x; i < L; i += blockDim.x) a[i] = src[i];
    __syncthreads();
  }
}

// One CTA per book: 0 quant codes [1024], 1 run values [1024], 2 run lengths [4096].
// Shared memory (bytes): len 4K | sym 8K | weight by node 32K | parent by node 16K |
// region A 32K (sort keys, live node list, canonical scratch) | region B 32K (sort
// scratch, new nodes, depth pass).
// =================================================================================
// record offsets: exclusive prefix of the blocks' record counts (one CTA)
// =================================================================================
__device__ void record_offsets_body(const BookArgs& a) {
  __shared__ uint64_t s_scan[33];
  constexpr int kPerThread = 8;
  const int tid = threadIdx.x;
  const uint32_t nblk = a.nblk;
  uint64_t carry = 0;
  for (uint32_t base = 0; base < nblk; base += blockDim.x * kPerThread) {
    const uint32_t b0 = base + tid * kPerThread;
    uint32_t c[kPerThread];
    uint64_t mine = 0;
#pragma unroll
    for (int i = 0; i < kPerThread; i++) {
      const uint32_t v = b0 + i < nblk ? a.rec.counts[b0 + i] : 0u;
      c[i] = (v >> 16) + (v & 0xffffu);
      mine += c[i];
    }
    uint64_t agg;
    uint64_t off = carry + block_excl_scan<uint64_t>(mine, s_scan, &agg);
#pragma unroll
    for (int i = 0; i < kPerThread; i++) {
      if (b0 + i < nblk) a.rec.rec_off[b0 + i] = off;
      off += c[i];
    }
    carry += agg;
  }
}

// Working memory of one book over nsym symbols: len nsym B | sym 2 nsym | weight by
// node 8 nsym | parent by node 4 nsym | region A 8 nsym (sort keys, live node list,
// canonical scratch) | region B 8 nsym (sort scratch, new nodes, depth pass).
__host__ __device__ constexpr uint32_t book_mem_bytes(int nsym) { return 31u * (uint32_t)nsym; }

// One canonical book (role 0 code, 1 run value, 2 run length) or, role 3, the
// record offsets of a field, by a CTA of NT threads.  mem: book_mem_bytes(nsym) of
// working memory, shared (the book kernels) or global (the batched persistent
// kernel's run-length books).
template <int NT>
__device__ void codebook_core(const BookArgs& a, int role, unsigned char* mem) {
  if (role == 3) {
    record_offsets_body(a);
    return;
  }
  const int book = role;
  const int nsym = book == 2 ? kNsymLen : kNsymCode;
  const uint32_t* hist = book == 0 ? a.hist_code : (book == 1 ? a.hist_val : a.hist_len);
  uint8_t* len_out = a.lens + (book == 0 ? 0 : (book == 1 ? kNsymCode : 2 * kNsymCode));
  uint64_t* code_out = a.codes + (book == 0 ? 0 : (book == 1 ? kNsymCode : 2 * kNsymCode));

  uint8_t* s_len = mem;
  uint16_t* s_sym = reinterpret_cast<uint16_t*>(mem + nsym);
  uint32_t* s_wt = reinterpret_cast<uint32_t*>(mem + 3 * nsym);
  uint16_t* s_par = reinterpret_cast<uint16_t*>(mem + 11 * nsym);
  uint64_t* A = reinterpret_cast<uint64_t*>(mem + 15 * nsym);
  uint64_t* B = reinterpret_cast<uint64_t*>(mem + 23 * nsym);
  __shared__ uint32_t s_L;
  __shared__ int s_n, s_k, s_next;
  __shared__ CanonSmem cs;
  const int tid = threadIdx.x;

  if (tid == 0) s_L = 0;
  for (int s = tid; s < nsym; s += blockDim.x) s_len[s] = 0;
  __syncthreads();
  for (int s = tid; s < nsym; s += blockDim.x) {
    const uint32_t f = hist[s];
    if (f) A[atomicAdd(&s_L, 1u)] = ((uint64_t)f << 12) | (uint64_t)s;
  }
  __syncthreads();
  const int L = (int)s_L;
  if (L == 1) {
    if (tid == 0) s_len[A[0] & 0xfff] = 1;
  } else if (L > 1) {
    // leaves in (frequency, symbol) order
    rank_merge_sort_u64(A, B, L);
    for (int i = tid; i < L; i += blockDim.x) {
      s_wt[i] = (uint32_t)(A[i] >> 12);
      s_sym[i] = (uint16_t)(A[i] & 0xfff);
    }
    __syncthreads();
    const int nn = 2 * L - 1;
    // ---- pairing rounds ----------------------------------------------------------
    // Keys order the live nodes as the sequential two-queue method picks them:
    // (weight, leaves before internal nodes, creation order).  With t the sum of the
    // two lightest, every consecutive pair whose second member weighs <= t precedes
    // the new node of weight t in that order, so all such pairs merge in one round;
    // the new nodes are rank-merged back.  When a round would merge few pairs the
    // rest is finished by the sequential loop, from the same state.
    constexpr uint64_t kClass = 1ull << 13, kIdx = kClass - 1;
    for (int i = tid; i < L; i += blockDim.x) A[i] = ((uint64_t)s_wt[i] << 14) | (uint64_t)i;
    if (tid == 0) {
      s_n = L;
      s_next = L;
    }
    __syncthreads();
    while (true) {
      const int n = s_n;
      if (n <= 1) break;
      if (tid == 0) {
        const uint64_t t = (A[0] >> 14) + (A[1] >> 14);
        int lo = 0, hi = n / 2;  // pairs i with weight(A[2i+1]) <= t
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if ((A[2 * mid + 1] >> 14) <= t) lo = mid + 1;
          else hi = mid;
        }
        s_k = lo;
      }
      __syncthreads();
      const int k = s_k;
      if (k < 16) break;
      const int next = s_next;
      for (int i = tid; i < k; i += blockDim.x) {
        const uint64_t x = A[2 * i], y = A[2 * i + 1];
        const uint64_t wn = (x >> 14) + (y >> 14);
        const uint32_t id = (uint32_t)next + i;
        s_par[x & kIdx] = (uint16_t)id;
        s_par[y & kIdx] = (uint16_t)id;
        s_wt[id] = (uint32_t)wn;
        B[i] = (wn << 14) | kClass | id;
      }
      __syncthreads();
      const int nr = n - 2 * k;
      uint64_t mine[(kNsymLen + NT - 1) / NT];
      int dst[(kNsymLen + NT - 1) / NT], cnt = 0;
      for (int i = tid; i < n - k; i += blockDim.x) {
        const bool from_rest = i < nr;
        const uint64_t x = from_rest ? A[2 * k + i] : B[i - nr];
        const uint64_t* other = from_rest ? B : A + 2 * k;
        int lo = 0, hi = from_rest ? k : nr;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (other[mid] < x) lo = mid + 1;
          else hi = mid;
        }
        mine[cnt] = x;
        dst[cnt] = (from_rest ? i : i - nr) + lo;
        cnt++;
      }
      __syncthreads();
      for (int c = 0; c < cnt; c++) A[dst[c]] = mine[c];
      if (tid == 0) {
        s_n = n - k;
        s_next = next + k;
      }
      __syncthreads();
    }
    if (tid == 0) {
      // sequential finish; consumed leaves and internal nodes are prefixes of their
      // queues, so the live list gives the queue fronts
      const int n = s_n;
      int live_leaves = 0;
      for (int i = 0; i < n; i++) live_leaves += (A[i] & kClass) ? 0 : 1;
      int qi = L - live_leaves, nxt = s_next, qj = nxt - (n - live_leaves);
      constexpr uint32_t INF = 0xffffffffu;
      uint32_t l0 = qi < L ? s_wt[qi] : INF, l1 = qi + 1 < L ? s_wt[qi + 1] : INF,
               l2 = qi + 2 < L ? s_wt[qi + 2] : INF;
      uint32_t i0 = qj < nxt ? s_wt[qj] : INF, i1 = qj + 1 < nxt ? s_wt[qj + 1] : INF;
      while (nxt < nn) {
        int pk[2];
        uint32_t pw[2];
#pragma unroll
        for (int t = 0; t < 2; t++) {
          if (l0 <= i0) {
            pk[t] = qi;
            pw[t] = l0;
            qi++;
            l0 = l1;
            l1 = l2;
            l2 = qi + 2 < L ? s_wt[qi + 2] : INF;
          } else {
            pk[t] = qj;
            pw[t] = i0;
            qj++;
            i0 = i1;
            i1 = qj + 1 < nxt ? s_wt[qj + 1] : INF;
          }
        }
        const uint32_t sum = pw[0] + pw[1];
        s_wt[nxt] = sum;
        s_par[pk[0]] = (uint16_t)nxt;
        s_par[pk[1]] = (uint16_t)nxt;
        if (qj == nxt) {
          i0 = sum;
        } else if (qj + 1 == nxt) {
          i1 = sum;
        }
        nxt++;
      }
      s_par[nn - 1] = (uint16_t)(nn - 1);
    }
    __syncthreads();
    // depths by pointer jumping (region B)
    uint16_t* s_anc = reinterpret_cast<uint16_t*>(B);
    uint16_t* s_dep = s_anc + 2 * nsym;
    for (int i = tid; i < nn; i += blockDim.x) {
      s_anc[i] = s_par[i];
      s_dep[i] = (i == nn - 1) ? 0 : 1;
    }
    __syncthreads();
    // (done once every node's ancestor is the root: the depths no longer change)
    for (int step = 1; step < nn; step <<= 1) {
      uint16_t na[(2 * kNsymLen + NT - 1) / NT], nd[(2 * kNsymLen + NT - 1) / NT];
      int c = 0;
      bool open = false;
      for (int i = tid; i < nn; i += blockDim.x) {
        const uint16_t an = s_anc[i];
        nd[c] = s_dep[i] + s_dep[an];
        na[c] = s_anc[an];
        open |= na[c] != (uint16_t)(nn - 1);
        c++;
      }
      __syncthreads();
      c = 0;
      for (int i = tid; i < nn; i += blockDim.x) {
        s_dep[i] = nd[c];
        s_anc[i] = na[c];
        c++;
      }
      if (!__syncthreads_or(open)) break;
    }
    for (int i = tid; i < L; i += blockDim.x) {
      const uint16_t d = s_dep[i];
      if (d > kMaxLen) atomicOr(&a.st->status, ERR_RANGE);
      s_len[s_sym[i]] = (uint8_t)d;
    }
  }
  __syncthreads();
  for (int s = tid; s < nsym; s += blockDim.x) len_out[s] = s_len[s];
  canonical_build(s_len, nsym, &cs, reinterpret_cast<uint16_t*>(A), code_out, nullptr);
}

__global__ __launch_bounds__(kBookThreads) void codebook_kernel(BookArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  codebook_core<kBookThreads>(a, blockIdx.x, smem);
}

// Batch: four CTAs per field (three books and the record offsets).
__global__ __launch_bounds__(kBookThreads) void codebook_batch_kernel(const BookArgs* __restrict__ tasks) {
  extern __shared__ __align__(16) unsigned char smem[];
  codebook_core<kBookThreads>(tasks[blockIdx.x >> 2], blockIdx.x & 3, smem);
}

static size_t codebook_smem_bytes() { return book_mem_bytes(kNsymLen); }

// =================================================================================
// per-block selection and encoding
// =================================================================================

// =================================================================================
// header, section padding and books
// =================================================================================
__device__ void finalize_body(const FinalizeArgs& a) {
  __shared__ uint32_t s_hdr[kHdr / 4];
  __shared__ uint64_t s_total, s_off_books, s_pay_end;
  __shared__ uint32_t s_flags;
  DevState* st = a.st;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const uint64_t n_rec = st->n_rec, payload = st->payload;
    const uint32_t flags = (st->ncodec[CODEC_HUFF] ? 1u : 0u) | (st->ncodec[CODEC_RLE_HUFF] ? 2u : 0u) |
                           (a.f64 ? kFlagF64 : 0u) | (a.global ? kFlagGlobal : 0u);
    const uint64_t off_pay = a.off_rec + 8 * n_rec;
    const uint64_t off_books = off_pay + ((payload + 7) & ~7ull);
    const uint64_t total = off_books + ((flags & 1) ? kNsymCode : 0) + ((flags & 2) ? kNsymCode + kNsymLen : 0);
    s_total = total;
    s_off_books = off_books;
    s_pay_end = off_pay + payload;
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
    put32(56, (uint32_t)kLanes);
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
  for (uint64_t i = s_pay_end + tid; i < s_off_books; i += blockDim.x) ar[i] = 0;
  uint64_t o = s_off_books;
  if (s_flags & 1) {
    for (int i = tid; i < kNsymCode; i += blockDim.x) ar[o + i] = a.lens[i];
    o += kNsymCode;
  }
  if (s_flags & 2) {
    for (int i = tid; i < kNsymCode + kNsymLen; i += blockDim.x) ar[o + i] = a.lens[kNsymCode + i];
  }
}

constexpr int kEncThreads = 256;
constexpr int kBufBytes = 16384;  // payload assembly buffer

// Learned pick from the network's three predictions (identical in every lane): the
// smallest (first index on ties), and whether the runner-up lies within the margin,
// in which case the caller decides by exact sizes.  Plain FP32 compares only.
__device__ __forceinline__ int learned_pick(const float* y, bool& fallback) {
  int c = 0;
  if (y[1] < y[c]) c = 1;
  if (y[2] < y[c]) c = 2;
  int r = -1;
#pragma unroll
  for (int k = 0; k < 3; k++)
    if (k != c && (r < 0 || y[k] < y[r])) r = k;
  const float gap = y[r] - y[c];
  fallback = gap < kMlpMargin;
  return c;
}

// The network's parameters staged in shared memory for one forward pass per block:
// the weight matrices transposed (the 32 lanes' weights for one input are consecutive
// words) and padded to 33 words per row, so each multiply-add step of the warp reads
// one conflict-free row instead of 32 scattered cache lines of the packed layout.
constexpr int kSwW1 = 0;                     // [8][33]  W1 transposed
constexpr int kSwB1 = kSwW1 + kMlpIn * 33;   // [32]
constexpr int kSwW2 = kSwB1 + kMlpHid;       // [32][33] W2 transposed
constexpr int kSwB2 = kSwW2 + kMlpHid * 33;  // [32]
constexpr int kSwW3 = kSwB2 + kMlpHid;       // [3][33]  W3 rows
constexpr int kSwB3 = kSwW3 + kMlpOut * 33;  // [3]
constexpr int kSwWords = kSwB3 + kMlpOut;

__device__ __forceinline__ void stage_mlp(const float* __restrict__ w, float* sw) {
  for (int i = threadIdx.x; i < kMlpParams; i += kEncThreads) {
    const float v = __ldg(&w[i]);
    int d;
    if (i < kMlpB1) {
      d = kSwW1 + (i % kMlpIn) * 33 + i / kMlpIn;
    } else if (i < kMlpW2) {
      d = kSwB1 + (i - kMlpB1);
    } else if (i < kMlpB2) {
      const int k = i - kMlpW2;
      d = kSwW2 + (k % kMlpHid) * 33 + k / kMlpHid;
    } else if (i < kMlpW3) {
      d = kSwB2 + (i - kMlpB2);
    } else if (i < kMlpB3) {
      const int k = i - kMlpW3;
      d = kSwW3 + (k / kMlpHid) * 33 + k % kMlpHid;
    } else {
      d = kSwB3 + (i - kMlpB3);
    }
    sw[d] = v;
  }
}

// mlp_forward_warp on the staged parameters: the same operands in the same order, so
// the same FP32 results.  f: the 8 features (same in every lane).
__device__ __forceinline__ void mlp_forward_staged(const float* sw, const float (&f)[kMlpIn], float* y) {
  const int lane = threadIdx.x & 31;
  float acc = sw[kSwB1 + lane];
#pragma unroll
  for (int j = 0; j < kMlpIn; j++) acc = fmaf(sw[kSwW1 + 33 * j + lane], f[j], acc);
  const float h1 = acc > 0.0f ? acc : 0.0f;
  acc = sw[kSwB2 + lane];
#pragma unroll
  for (int j = 0; j < kMlpHid; j++) acc = fmaf(sw[kSwW2 + 33 * j + lane], __shfl_sync(~0u, h1, j), acc);
  const float h2 = acc > 0.0f ? acc : 0.0f;
  const int o = lane < kMlpOut ? lane : 0;
  acc = sw[kSwB3 + o];
#pragma unroll
  for (int j = 0; j < kMlpHid; j++) acc = fmaf(sw[kSwW3 + 33 * o + j], __shfl_sync(~0u, h2, j), acc);
#pragma unroll
  for (int c = 0; c < kMlpOut; c++) y[c] = __shfl_sync(~0u, acc, c);
}

// smallest exact size; ties prefer HUFF, then RLE_HUFF, then RLE
__device__ __forceinline__ int exhaustive_pick(uint64_t sh, uint64_t sr, uint64_t srh) {
  int c = CODEC_HUFF;
  uint64_t best = sh;
  if (srh < best) {
    c = CODEC_RLE_HUFF;
    best = srh;
  }
  if (sr < best) c = CODEC_RLE;
  return c;
}

// interleaved-stream units from per-thread bit partials: thread t's symbols all belong
// to lane t % 32 (strided mapping over 256 threads); called by warp 0
__device__ __forceinline__ uint32_t units_from_partials(const uint32_t* part) {
  const int lane = threadIdx.x & 31;
  uint32_t bits = 0;
#pragma unroll
  for (int wv = 0; wv < kEncThreads / 32; wv++) bits += part[32 * wv + lane];
  return warp_sum(ihs_lane_units(bits));
}

static_assert(kEncThreads % kMadoN == 0, "madogram distances by thread");

// Selection and encoding of codec block b of one field (all threads of the CTA).
// smem: encode_smem_bytes() of dynamic shared memory.
__device__ void encode_body(const EncodeArgs& a, uint32_t b, unsigned char* smem) {
  uint16_t* s_c = reinterpret_cast<uint16_t*>(smem);             // 4096 codes
  uint16_t* s_rv = s_c + kSlots;                                 // run values
  uint16_t* s_rl = s_rv + kSlots;                                // run lengths
  uint32_t* s_buf = reinterpret_cast<uint32_t*>(s_rl + kSlots);  // 16 KB
  uint32_t* s_head = s_buf + kBufBytes / 4;                      // 128
  uint32_t* s_woff = s_head + kSlots / 32;                       // 129 (+3)
  uint32_t* s_next = s_woff + kSlots / 32 + 4;                   // 128
  uint32_t* s_part = s_next + kSlots / 32;                       // 2 x 256
  uint32_t* s_scan = s_part + 2 * kEncThreads;                   // 34
  uint64_t* s_scan64 = reinterpret_cast<uint64_t*>(s_scan + 34); // 33
  __shared__ uint32_t s_codec, s_units[3];
  __shared__ uint64_t s_prefix;
  __shared__ float s_feat[8];

  const int tid = threadIdx.x, wid = tid >> 5;
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
    // the Huffman emitter's lane strings (s_rv and s_rl, 16 KB) start cleared; run
    // extraction overwrites them, and the emitter then clears what it uses itself
    uint4* lanes = reinterpret_cast<uint4*>(s_rv);
    for (int i = tid; i < 2 * kSlots * 2 / 16; i += kEncThreads) lanes[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  // the block statistics' code histogram (the first 1024 words of s_buf, which holds
  // no payload until assembly) starts at zero, and the learned selector's parameters
  // sit after it; both are ready at the barrier after the records
  const bool analyze = a.analyze != 0;
  static_assert(kNsymCode == 4 * kEncThreads && 4 * (kNsymCode + kSwWords) <= kBufBytes, "s_buf layout");
  if (analyze || sel == SEL_HEURISTIC || sel == SEL_LEARNED)
    reinterpret_cast<uint4*>(s_buf)[tid] = make_uint4(0u, 0u, 0u, 0u);
  if (sel == SEL_LEARNED && !analyze) stage_mlp(a.mlp_w, reinterpret_cast<float*>(s_buf) + kNsymCode);

  // this block's outlier and patch records, in slot order, at its record offset
  if (a.place_records && a.rec.counts[b] != 0) {
    const RecordArgs& R = a.rec;
    const uint32_t lo = tid * 16;
    const uint32_t* mw = R.masks + (uint64_t)b * 256;
    const uint32_t pb = (mw[lo >> 5] >> (lo & 31)) & 0xffffu;
    const uint32_t ob = (mw[128 + (lo >> 5)] >> (lo & 31)) & 0xffffu;
    uint64_t pos = R.rec_off[b] + block_excl_scan<uint64_t>((uint64_t)(__popc(ob) + __popc(pb)), s_scan64, nullptr);
    if (ob | pb) {
      const int32_t* dl = R.deltas + (uint64_t)b * kSlots;
      const uint64_t ny = a.g.n[1], nx = a.g.n[2];
      uint32_t err = 0;
      for (int i = 0; i < 16; i++) {
        const uint32_t j = lo + i;
        const uint32_t slot2 = (b * (uint32_t)kSlots + j) * 2u;
        if ((ob >> i) & 1u) {
          if (pos < R.rec_cap) reinterpret_cast<uint2*>(R.rec)[pos] = make_uint2(slot2, (uint32_t)dl[j]);
          else err |= ERR_CAPACITY;
          pos++;
        }
        if ((pb >> i) & 1u) {
          uint32_t zz = 0, yy = 0, xx = j;
          if (a.g.ndim == 2) {
            yy = j / w[2];
            xx = j - yy * w[2];
          } else if (a.g.ndim == 3) {
            const uint32_t pl = w[1] * w[2];
            zz = j / pl;
            const uint32_t rr = j - zz * pl;
            yy = rr / w[2];
            xx = rr - yy * w[2];
          }
          const uint64_t e = ((uint64_t)(org[0] + zz) * ny + (org[1] + yy)) * nx + (org[2] + xx);
          if (pos < R.rec_cap) reinterpret_cast<uint2*>(R.rec)[pos] = make_uint2(slot2 + 1u, __float_as_uint(R.x[e]));
          else err |= ERR_CAPACITY;
          pos++;
        }
      }
      if (err) atomicOr(&a.st->status, err);
    }
  }
  __syncthreads();

  // Analysis (selector training data): every size and every feature of every block,
  // no payload.  Otherwise runs are counted in every mode except forced Huffman and
  // extracted (values, lengths) only when a run codec or the statistics need them.
  uint32_t nr = 0;
  bool have_runs = false;
  // the run count comes from construction; the run index is built only when runs
  // are extracted
  if (sel != SEL_HUFF || analyze) nr = a.block_runs[b];
  const bool eligible = a.all_runs || 4 * nr <= m;
  auto extract_runs = [&]() {
    if (have_runs) return;
    block_run_heads(s_c, m, s_head, s_woff, s_next);
#pragma unroll 4
    for (int i = 0; i < kSlots / kEncThreads; i++) {
      const uint32_t j = tid + kEncThreads * i;
      if (j < m) {
        const uint32_t hb = s_head[j >> 5], bit = j & 31;
        if ((hb >> bit) & 1u) {
          const uint32_t ri = s_woff[j >> 5] + __popc(hb & ((1u << bit) - 1u));
          s_rv[ri] = s_c[j];
          s_rl[ri] = (uint16_t)(next_head(s_head, s_next, j, m) - j);
        }
      }
    }
    __syncthreads();
    have_runs = true;
  };
  if (analyze || (sel != SEL_HUFF && eligible && sel != SEL_RLE)) extract_runs();

  // exact sizes: Huffman units from per-lane bit totals; the plan (code lengths in
  // registers, lane offsets) is kept for the payload
  IhsPlan plan;
  IhsPlan2Out plan_out{0u, 0u, ~0u};
  auto huff_units = [&]() {  // u16 count + both streams
    plan_out = ihs_plan2(s_c, m, clen, s_part, plan);
    return 1u + plan_out.units_a + plan_out.units_b;
  };
  auto rlehuff_units = [&]() {
    uint32_t vb = 0, lb = 0;
    for (uint32_t i = tid; i < nr; i += kEncThreads) {
      vb += __ldg(&vlen[s_rv[i]]);
      lb += __ldg(&llen[s_rl[i] - 1]);
    }
    s_part[tid] = vb;
    s_part[kEncThreads + tid] = lb;
    __syncthreads();
    if (tid < 32) {
      const uint32_t vu = units_from_partials(s_part);
      const uint32_t lu = units_from_partials(s_part + kEncThreads);
      if (tid == 0) {
        s_units[1] = vu;
        s_units[2] = lu;
      }
    }
    __syncthreads();
  };
  uint64_t size_h = ~0ull, size_r = ~0ull, size_rh = ~0ull;
  // for_pick: the sizes only decide an exhaustive pick, so the Huffman size is left
  // unknown (~0) when a run codec is already smaller than any Huffman payload can be:
  // every code takes at least one bit, so a Huffman block of m codes holds at least
  // m / 16 units plus its unit count, 2 + m / 8 bytes.  The pick is the same.
  auto exact_sizes = [&](bool h, bool rl, bool rh, bool for_pick) {
    if (rl) size_r = 4ull * nr;
    if (rh && eligible && size_rh == ~0ull) {
      rlehuff_units();
      size_rh = (8ull + 2ull * (s_units[1] + s_units[2]) + 3) & ~3ull;
    }
    const bool beaten = for_pick && min(size_r, size_rh) < 2ull + m / 8;
    if (h && size_h == ~0ull && !beaten) size_h = (2ull * huff_units() + 3) & ~3ull;
  };
  exact_sizes(analyze || sel == SEL_HUFF || sel == SEL_EXHAUSTIVE, analyze || sel == SEL_RLE || sel == SEL_EXHAUSTIVE,
              analyze || sel == SEL_RLE_HUFF || sel == SEL_EXHAUSTIVE, sel == SEL_EXHAUSTIVE && !analyze);

  // selection
  const bool statistics = analyze || ((sel == SEL_HEURISTIC || sel == SEL_LEARNED) && eligible);
  if ((sel == SEL_HEURISTIC || sel == SEL_LEARNED) && !eligible && !analyze) {
    if (tid == 0) s_codec = CODEC_HUFF;  // both pick between Huffman and RLE+Huffman
  } else if (statistics) {
    uint32_t* s_hist = s_buf;  // 1024 words (zeroed above), before the payload is assembled
    for (uint32_t i = tid; i < nr; i += kEncThreads) atomicAdd(&s_hist[s_rv[i]], (uint32_t)s_rl[i]);
    __syncthreads();
    // block statistics in one pass and one reduction: entropy sum, |delta| sum, top
    // count and largest in-range |delta|, and (selector) the madogram's code changes
    // on the pairs (j, j + 1 + 25 (j mod 8))
    uint64_t S_ = 0, absd = 0;
    uint32_t f1 = 0, maxd = 0, mism = 0;
    for (int c = tid; c < kNsymCode; c += kEncThreads) {
      const uint32_t h = s_hist[c];
      if (h) {
        S_ += (uint64_t)h * log2_q16_small(h);
        f1 = max(f1, h);
        if (c != 0) {
          const uint32_t d = (uint32_t)abs((int)c - (int)r);
          absd += (uint64_t)h * d;
          maxd = max(maxd, d);
        }
      }
    }
    const bool want_mado = !(sel == SEL_HEURISTIC && !analyze);
    if (want_mado) {
      // kEncThreads is a multiple of kMadoN, so a thread's distance is fixed
      const uint32_t d = kMadoD0 + kMadoStep * (tid % kMadoN);
      for (uint32_t j = tid; j + d < m; j += kEncThreads) mism += s_c[j] != s_c[j + d];
    }
    S_ = warp_sum(S_);
    absd = warp_sum(absd);
    mism = warp_sum(mism);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      f1 = max(f1, __shfl_xor_sync(~0u, f1, o));
      maxd = max(maxd, __shfl_xor_sync(~0u, maxd, o));
    }
    if ((tid & 31) == 0) {
      s_scan64[4 * wid + 0] = S_;
      s_scan64[4 * wid + 1] = absd;
      s_scan64[4 * wid + 2] = ((uint64_t)f1 << 32) | maxd;
      s_scan64[4 * wid + 3] = mism;
    }
    __syncthreads();
    const int64_t Lm = log2_q16_small(m);
    __shared__ bool s_fallback;
    if (sel == SEL_HEURISTIC && !analyze) {
      if (tid == 0) {
        S_ = 0;
        f1 = 0;
        for (int v = 0; v < kEncThreads / 32; v++) {
          S_ += s_scan64[4 * v + 0];
          f1 = max(f1, (uint32_t)(s_scan64[4 * v + 2] >> 32));
        }
        const int64_t NH = (int64_t)m * Lm - (int64_t)S_;
        int64_t Rm = 0;
        if (10ll * f1 > 4ll * m) {
          const int64_t rest = (int64_t)m - f1;
          Rm = (int64_t)m * 65536 + (int64_t)f1 * log2_q16_small(f1) +
               (rest > 0 ? rest * (int64_t)log2_q16_small((uint32_t)rest) : 0) - (int64_t)m * Lm;
          if (Rm < 0) Rm = 0;
        }
        const int64_t est = NH + Rm;
        s_codec = (100 * est <= 109ll * (int64_t)m * 65536) ? CODEC_RLE_HUFF : CODEC_HUFF;
      }
    } else {
      if (wid == 0) {
        // warp 0: the block totals (lane v < 8 brings warp v's partials), one feature
        // per lane k < 8, then the network on the staged parameters
        const int lane = tid & 31;
        uint64_t tS = 0, tA = 0, tM = 0;
        uint32_t tF = 0, tD = 0;
        if (lane < kEncThreads / 32) {
          tS = s_scan64[4 * lane + 0];
          tA = s_scan64[4 * lane + 1];
          tF = (uint32_t)(s_scan64[4 * lane + 2] >> 32);
          tD = (uint32_t)s_scan64[4 * lane + 2];
          tM = s_scan64[4 * lane + 3];
        }
        tS = warp_sum(tS);
        tA = warp_sum(tA);
        tM = warp_sum(tM);
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          tF = max(tF, __shfl_xor_sync(~0u, tF, o));
          tD = max(tD, __shfl_xor_sync(~0u, tD, o));
        }
        const float fm = (float)m;
        float fk = 0.0f;
        if (lane == 0) {
          fk = (float)s_hist[r] / fm;  // zero residuals
        } else if (lane == 1) {
          const int64_t NH = (int64_t)m * Lm - (int64_t)tS;
          fk = (float)NH / (float)((uint64_t)m * 65536ull);
        } else if (lane == 2) {
          fk = (float)tF / fm;
        } else if (lane == 3) {
          fk = (float)log2_q16_small(1u + tD) / 65536.0f;
        } else if (lane == 4) {
          fk = (float)nr / fm;
        } else if (lane == 5) {
          fk = (float)s_hist[0] / fm;  // outliers
        } else if (lane == 6) {
          fk = (float)tA / (float)((uint64_t)m * r);
        } else if (lane == 7) {
          // pairs inside the block: positions j < m - d for each residue class j mod 8
          uint32_t pairs = 0;
          for (uint32_t k = 0; k < kMadoN; k++) {
            const uint32_t d = kMadoD0 + kMadoStep * k;
            if (m > d + k) pairs += (m - d - k + kMadoN - 1) / kMadoN;
          }
          fk = pairs ? (float)(uint32_t)tM / (float)pairs : 0.0f;
        }
        if (analyze) {
          if (lane < kMlpIn) s_feat[lane] = fk;
        } else {
          float f[kMlpIn], y[kMlpOut];
#pragma unroll
          for (int j = 0; j < kMlpIn; j++) f[j] = __shfl_sync(~0u, fk, j);
          mlp_forward_staged(reinterpret_cast<const float*>(s_buf) + kNsymCode, f, y);
          bool fb;
          const int c = learned_pick(y, fb);
          if (lane == 0) {
            s_codec = (uint32_t)c;
            s_fallback = fb;
          }
        }
      }
      __syncthreads();
      if (analyze) {
        // one training row: features, log2 bits per element of each codec (Q16-exact),
        // exact sizes, and whether the learned selector decides this block
        if (tid < kMlpIn) a.feat_out[(uint64_t)b * kMlpIn + tid] = s_feat[tid];
        if (tid < kMlpOut) {
          const uint64_t sz = tid == CODEC_HUFF ? size_h : (tid == CODEC_RLE ? size_r : size_rh);
          const bool have = sz != ~0ull;
          a.size_out[(uint64_t)b * kMlpOut + tid] = have ? (uint32_t)sz : 0xffffffffu;
          a.tgt_out[(uint64_t)b * kMlpOut + tid] =
              have ? (float)((int64_t)log2_q16(8 * sz) - (int64_t)log2_q16(m)) * (1.0f / 65536.0f) : 0.0f;
          if (tid == 0) a.valid_out[b] = eligible ? 1 : 0;
        }
        return;
      }
      if (s_fallback) {
        // the network is unsure: exact sizes decide
        exact_sizes(true, true, true, true);
        if (tid == 0) s_codec = (uint32_t)exhaustive_pick(size_h, size_r, size_rh);
      }
    }
    __syncthreads();
  } else if (tid == 0) {
    s_codec = sel <= SEL_RLE_HUFF ? (uint32_t)sel : (uint32_t)exhaustive_pick(size_h, size_r, size_rh);
  }
  __syncthreads();
  const int codec = (int)s_codec;
  if (codec == CODEC_RLE || codec == CODEC_RLE_HUFF) extract_runs();
  exact_sizes(codec == CODEC_HUFF, codec == CODEC_RLE, codec == CODEC_RLE_HUFF, false);
  const uint64_t size = codec == CODEC_HUFF ? size_h : (codec == CODEC_RLE ? 4ull * nr : size_rh);
  // The block's codec and size are counted, then the block counts itself done with
  // release semantics: the block that takes the last count (acquire) writes the
  // header from complete totals once its own payload is out.  No other block's
  // payload bytes are needed for that, so the count need not wait for them.
  __shared__ bool s_last;
  uint32_t done = 0;
  if (tid == 0) {
    lookback_publish(a.lb, b, size);
    atomicAdd(&a.st->ncodec[codec], 1u);
    atomicAdd(&a.st->payload, (unsigned long long)size);
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(done) : "l"(&a.st->encode_done) : "memory");
  }

  // payload assembly in shared memory while predecessors publish (every chosen size
  // fits 16 KB unless a forced Huffman mode meets very long codes; those go direct)
  auto assemble = [&](uint16_t* out16) {
    if (codec == CODEC_HUFF) {
      const uint32_t u = 1u + plan_out.units_a + plan_out.units_b;
      if (plan_out.max_lane_bits <= kLaneBitsMax) {
        ihs_emit2(s_c, m, ccode, plan, plan_out.units_a, reinterpret_cast<uint32_t*>(s_rv), out16, s_part,
                  !have_runs);
      } else {
        const uint32_t h = huff_split(m);
        if (tid == 0) out16[0] = (uint16_t)plan_out.units_a;
        ihs_encode_block(s_c, h, 0, clen, ccode, out16 + 1, s_part);
        ihs_encode_block(s_c + h, m - h, 0, clen, ccode, out16 + 1 + plan_out.units_a, s_part);
      }
      if ((u & 1u) && tid == 0) out16[u] = 0;
    } else if (codec == CODEC_RLE_HUFF) {
      const uint32_t vu = s_units[1], lu = s_units[2];
      if (tid == 0) {
        uint32_t* out32 = reinterpret_cast<uint32_t*>(out16);
        out32[0] = nr;
        out32[1] = vu;
        if ((vu + lu) & 1u) out16[4 + vu + lu] = 0;
      }
      ihs_encode_block(s_rv, nr, 0, vlen, vcode, out16 + 4, s_part);
      ihs_encode_block(s_rl, nr, -1, llen, lcode, out16 + 4 + vu, s_part);
    }
  };
  const bool in_smem = size <= (uint64_t)kBufBytes;
  if (in_smem) assemble(reinterpret_cast<uint16_t*>(s_buf));
  if (tid == 0) s_last = done == a.g.nblk - 1;
  __syncthreads();

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
    reinterpret_cast<uint32_t*>(a.ar + a.off_bb)[b] = (uint32_t)size;
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
    assemble(reinterpret_cast<uint16_t*>(dst));
  }
  // the block that counted last writes the header, section padding and books
  if (s_last) finalize_body(a.fin);
}

// Blocks are taken in ticket order, so the payload look-back only ever waits on
// blocks that CTAs already hold.
__global__ __launch_bounds__(kEncThreads, 5) void encode_kernel(EncodeArgs a) {
  __shared__ uint32_t s_tile;
  extern __shared__ __align__(16) unsigned char smem[];
  if (threadIdx.x == 0) s_tile = atomicAdd(&a.st->ticket_encode, 1u);
  __syncthreads();
  encode_body(a, s_tile, smem);
}

// Batch: one CTA per codec block of every field; the ticket runs over the blocks of
// all fields in order (tile0[f] = first block of field f).
__global__ __launch_bounds__(kEncThreads, 5) void encode_batch_kernel(const EncodeArgs* __restrict__ tasks,
                                                                   const uint32_t* __restrict__ tile0, int nfields,
                                                                   uint32_t* ticket) {
  __shared__ uint32_t s_tile;
  __shared__ int s_field;
  if (threadIdx.x == 0) {
    const uint32_t t = atomicAdd(ticket, 1u);
    int lo = 0, hi = nfields - 1;  // last field with tile0[f] <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile0[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    s_field = lo;
    s_tile = t - tile0[lo];
  }
  __syncthreads();
  extern __shared__ __align__(16) unsigned char smem[];
  encode_body(tasks[s_field], s_tile, smem);
}

static size_t encode_smem_bytes() {
  return kSlots * 2 * 3 + kBufBytes + (kSlots / 32) * 4 * 3 + 16 + 2 * kEncThreads * 4 + 34 * 4 + 33 * 8 + 16;
}

// =================================================================================
// batched compression in one persistent launch
// =================================================================================
// Every CTA runs the four phases of the staged batch in order, so the work items of
// each phase are taken (by ticket) only after those of the phases before it were all
// taken: a waiting CTA waits on items that running CTAs hold (only a running CTA takes
// an item), and those wait only on earlier phases, so the launch cannot deadlock even
// when not all of its CTAs are resident at once.  The
// hand-overs are per field (DevState ready_range, tiles_flushed, books_done: a
// release by the producer, an acquire by thread 0 of the consumer, then a CTA
// barrier), so one field's books and encoding start while other fields are still
// being constructed.  Every wait is bounded (ERR_TIMEOUT in the field's status).
// The output is the staged path's, byte for byte: the same bodies run on the same
// items.
constexpr int kPersistThreads = 256;
static_assert(kPersistThreads == kEncThreads, "one CTA shape for every phase");

__device__ __forceinline__ int field_of_prefix(const uint32_t* prefix, int nfields, uint32_t c) {
  int lo = 0, hi = nfields - 1;  // last field with prefix[f] <= c
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= c) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// thread 0 draws the next item of a phase; every thread gets it (two barriers, so the
// word is free for the next draw)
__device__ __forceinline__ uint32_t draw_item(uint32_t* ticket, uint32_t* s_word) {
  if (threadIdx.x == 0) *s_word = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t v = *s_word;
  __syncthreads();
  return v;
}

// thread 0 waits for a field's hand-over counter, then the CTA proceeds together
__device__ __forceinline__ void await_field(const uint32_t* counter, uint32_t target, DevState* st, uint32_t limit) {
  if (threadIdx.x == 0 && !wait_ge_acquire(counter, target, limit)) atomicOr(&st->status, ERR_TIMEOUT);
  __syncthreads();
}

template <int ND>
__global__ __launch_bounds__(kPersistThreads, 4) void batch_persistent_kernel(const __grid_constant__ PersistArgs p) {
  // the construction phase's swizzled TMA tiles want 1024-byte aligned buffers; the
  // alignment is taken here (1 KB of slack in the dynamic size) rather than declared,
  // which would pad the static shared memory of every kernel in this file
  extern __shared__ __align__(16) unsigned char smem_dyn[];
  unsigned char* smem_raw = smem_dyn + ((1024u - (smem_u32(smem_dyn) & 1023u)) & 1023u);
  __shared__ uint32_t s_word;
  const int tid = threadIdx.x;
  // ---- phase 1: value ranges and bounds ---------------------------------------------
  while (true) {
    const uint32_t c = draw_item(&p.tickets[2], &s_word);
    if (c >= p.nrange) break;
    const int f = field_of_prefix(p.cta0, p.nfields, c);
    const RangeTask& t = p.rtasks[f];
    if (t.mode == 0) {
      if (tid == 0) {
        derive_eb(t.st, 0, t.eb, 0.0f, 0.0f);
        release_flag(&t.st->ready_range);
      }
    } else {
      range_body(t.x, t.n, t.st, t.mode, t.eb, c - p.cta0[f], p.cta0[f + 1] - p.cta0[f], &t.st->ready_range);
    }
    __syncthreads();
  }
  // ---- phase 2: construction (waits for each field's bound) ---------------------------
  cons::construct_loop<ND, float, false, true>(p.ctasks[0], p.ctasks, p.tile0, p.nfields, p.ntiles, &p.tickets[0],
                                               p.spin_limit, smem_raw);
  // ---- phase 3: books and record offsets (wait for each field's tiles) ---------------
  while (true) {
    const uint32_t j = draw_item(&p.tickets[3], &s_word);
    if (j >= 4u * (uint32_t)p.nfields) break;
    const int f = (int)(j >> 2), role = (int)(j & 3);
    const BookArgs& ba = p.btasks[f];
    await_field(&ba.st->tiles_flushed, p.tile0[f + 1] - p.tile0[f], ba.st, p.spin_limit);
    unsigned char* mem = role == 2 ? p.len_books + (size_t)f * book_mem_bytes(kNsymLen) : smem_raw;
    codebook_core<kPersistThreads>(ba, role, mem);
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(&ba.st->books_done, 1u);
    }
  }
  // ---- phase 4: encoding (waits for each field's books) -------------------------------
  int ready_field = -1;
  while (true) {
    const uint32_t t = draw_item(&p.tickets[1], &s_word);
    if (t >= p.ntiles) break;
    const int f = field_of_prefix(p.tile0, p.nfields, t);
    const EncodeArgs& ea = p.etasks[f];
    if (f != ready_field) {
      await_field(&ea.st->books_done, 4u, ea.st, p.spin_limit);
      ready_field = f;
    }
    encode_body(ea, t - p.tile0[f], smem_raw);
    __syncthreads();
  }
}

static size_t persist_smem_bytes() {
  size_t b = construct_smem_bytes();
  if (encode_smem_bytes() > b) b = encode_smem_bytes();
  if (book_mem_bytes(kNsymCode) > b) b = book_mem_bytes(kNsymCode);
  return b + 1024;  // alignment slack
}

size_t persist_len_book_bytes() { return book_mem_bytes(kNsymLen); }

template <int ND>
static int persist_occupancy() {
  static int occ = -1;
  if (occ < 0) {
    const int sm = (int)persist_smem_bytes();
    if (cudaFuncSetAttribute(batch_persistent_kernel<ND>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_persistent_kernel<ND>, kPersistThreads, sm) !=
            cudaSuccess)
      occ = 0;
  }
  return occ;
}

int persist_grid_max() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int occ = persist_occupancy<0>();
  for (int o : {persist_occupancy<1>(), persist_occupancy<2>(), persist_occupancy<3>()})
    if (o < occ) occ = o;
  return occ * (sms > 0 ? sms : 0);
}

cudaError_t launch_batch_persistent(const PersistArgs& p, int grid, int nd, cudaStream_t s) {
  auto k = nd == 1 ? batch_persistent_kernel<1>
                   : (nd == 2 ? batch_persistent_kernel<2> : (nd == 3 ? batch_persistent_kernel<3> : batch_persistent_kernel<0>));
  if (grid <= 0 || grid > persist_grid_max()) return cudaErrorInvalidConfiguration;
  trace_begin(K_BATCH, s);
  k<<<grid, kPersistThreads, persist_smem_bytes(), s>>>(p);
  trace_end(K_BATCH, s);
  return cudaGetLastError();
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
  const uint32_t grid = range_ctas(n);
  trace_begin(K_RANGE, s);
  range_kernel<<<grid, 256, 0, s>>>(x, n, st, mode, eb);
  trace_end(K_RANGE, s);
  return cudaGetLastError();
}

cudaError_t launch_range_d(const double* x, uint64_t n, DevState* st, int mode, double eb, cudaStream_t s) {
  trace_begin(K_RANGE, s);
  if (mode == 0) abs_params_d_kernel<<<1, 32, 0, s>>>(st, eb);
  else range_d_kernel<<<range_ctas(2 * n), 256, 0, s>>>(x, n, st, mode, eb);
  trace_end(K_RANGE, s);
  return cudaGetLastError();
}

cudaError_t launch_codebook(const BookArgs& a, cudaStream_t s) {
  const size_t sm = codebook_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(codebook_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int grid = a.place_records ? 4 : 3;
  trace_begin(K_CODEBOOK, s);
  codebook_kernel<<<grid, kBookThreads, sm, s>>>(a);
  trace_end(K_CODEBOOK, s);
  return cudaGetLastError();
}

cudaError_t launch_encode(const EncodeArgs& a, cudaStream_t s) {
  trace_begin(K_ENCODE, s);
  encode_kernel<<<a.g.nblk, kEncThreads, encode_smem_bytes(), s>>>(a);
  trace_end(K_ENCODE, s);
  return cudaGetLastError();
}

uint32_t range_ctas(uint64_t n) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const uint64_t want = (n / 4 + 255) / 256;
  const uint64_t grid = want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8;
  return grid ? (uint32_t)grid : 1u;
}

cudaError_t launch_range_batch(const RangeTask* d_tasks, const uint32_t* d_cta0, int nfields, uint32_t nctas,
                               cudaStream_t s) {
  trace_begin(K_RANGE, s);
  range_batch_kernel<<<nctas, 256, 0, s>>>(d_tasks, d_cta0, nfields);
  trace_end(K_RANGE, s);
  return cudaGetLastError();
}

cudaError_t launch_codebook_batch(const BookArgs* d_tasks, int nfields, cudaStream_t s) {
  const size_t sm = codebook_smem_bytes();
  cudaError_t e =
      cudaFuncSetAttribute(codebook_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  trace_begin(K_CODEBOOK, s);
  codebook_batch_kernel<<<4 * nfields, kBookThreads, sm, s>>>(d_tasks);
  trace_end(K_CODEBOOK, s);
  return cudaGetLastError();
}

cudaError_t launch_encode_batch(const EncodeArgs* d_tasks, const uint32_t* d_tile0, int nfields, uint32_t ntiles,
                                uint32_t* ticket, cudaStream_t s) {
  trace_begin(K_ENCODE, s);
  encode_batch_kernel<<<ntiles, kEncThreads, encode_smem_bytes(), s>>>(d_tasks, d_tile0, nfields, ticket);
  trace_end(K_ENCODE, s);
  return cudaGetLastError();
}


}  // namespace cszp
