// Lorenzo construction (Sec. IV-A, Alg. 1 compression part): prequantization, the
// chunk-local Lorenzo residual, postquantization into uint16 codes with outlier and
// verbatim-patch records, and the code / run histograms the codebooks need.
//
// Persistent kernel: each CTA takes codec blocks (tiles) in ticket order from one
// counter shared by every field of the launch (one field, or a batch), and keeps
// two 16 KB input buffers.  While it works on one tile, the tensor memory
// accelerator (cp.async.bulk.tensor, completion on an mbarrier) is already fetching
// the next one, so the memory system always has the next tile in flight.  Tiles
// arrive as full 16^3 / 64x64 / 4096 boxes with zeros outside the field.  Fields
// whose layout TMA cannot describe (base not 16-byte aligned, row pitch not a
// multiple of 16 bytes) are loaded by the threads instead, without prefetch.
//
// Histograms are accumulated per CTA in shared memory (32-bit counters) over all its
// tiles of one field and added to the field's global histograms when the CTA moves
// to another field or finishes.  Records are not placed here: each tile leaves its
// outlier / patch counts, bit words and outlier residuals; the codebook launch scans
// the counts and the encode CTAs write the records in slot order.
//
// This header holds the device code: construct.cu instantiates it as the
// construction kernels, compress.cu as one phase of the batched persistent kernel.
#pragma once
#include <cuda.h>

#include "common.cuh"
#include "kernels.h"

namespace cszp {
namespace cons {

namespace {

constexpr int kThreads = 256;
constexpr int kPer = kSlots / kThreads;  // 16 elements per thread
constexpr int kHlShared = 256;  // run lengths counted in shared memory; longer runs go to the field's
                                // histogram directly (they are rare: one per long constant stretch)

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

// ---- prequantization by element type (Sec. IV-A1; doubles: step 2eb (1 - 2^-24)) ---
template <typename T>
struct Pq;
// The bound's words are read once per CTA and field (load_pq, thread 0, through L2:
// in the batched persistent kernel another SM derived them during the same launch)
// into the CTA's shared copy w, which every thread reads per tile.
template <>
struct Pq<float> {
  float eb_f, ebx2_f, ebx2_r;
  __device__ explicit Pq(const float* w) : eb_f(w[0]), ebx2_f(w[1]), ebx2_r(w[2]) {}
  __device__ static void load(const DevState* st, float* w) {
    w[0] = __ldcg(&st->eb_f);
    w[1] = __ldcg(&st->ebx2_f);
    w[2] = __ldcg(&st->ebx2_r);
  }
  __device__ __forceinline__ bool fast(float x, int32_t& k) const { return prequant_fast(x, eb_f, ebx2_f, ebx2_r, k); }
  __device__ __forceinline__ uint32_t full(float x, int32_t& k, bool& patch) const {
    return prequant(x, eb_f, ebx2_f, ebx2_r, k, patch);
  }
};
template <>
struct Pq<double> {
  double eb_d, step, rstep;
  __device__ explicit Pq(const double* w) : eb_d(w[0]), step(w[1]), rstep(w[2]) {}
  __device__ static void load(const DevState* st, double* w) {
    w[0] = __ldcg(&st->eb_d);
    w[1] = __ldcg(&st->step_d);
    w[2] = __ldcg(&st->rstep_d);
  }
  __device__ __forceinline__ bool fast(double x, int32_t& k) const { return prequant_fast_d(x, eb_d, step, rstep, k); }
  __device__ __forceinline__ uint32_t full(double x, int32_t& k, bool& patch) const {
    patch = false;
    return prequant_d(x, eb_d, step, rstep, k);
  }
};

// 16 consecutive elements of a shared-memory tile (16-byte loads)
__device__ __forceinline__ void load16(const float* p, float (&f)[16]) {
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const float4 v = reinterpret_cast<const float4*>(p)[i];
    f[4 * i] = v.x;
    f[4 * i + 1] = v.y;
    f[4 * i + 2] = v.z;
    f[4 * i + 3] = v.w;
  }
}
__device__ __forceinline__ void load16(const double* p, double (&f)[16]) {
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const double2 v = reinterpret_cast<const double2*>(p)[i];
    f[2 * i] = v.x;
    f[2 * i + 1] = v.y;
  }
}

// ---- FP32 3-D tiles: 64-byte swizzled rows ------------------------------------------
// A 16^3 FP32 box has 64-byte x rows.  Its TMA copy uses the 64-byte swizzle: the
// 16-byte chunk c of row R lands at chunk c ^ ((R >> 1) & 3) of that row (the buffer
// is 1024-byte aligned), so that eight threads reading one chunk of eight consecutive
// rows touch all 32 banks.  Thread loads and every reader of such a box use the same
// placement: element e of the box sits at swz64(e).
__device__ __forceinline__ uint32_t swz64(uint32_t e) { return e ^ ((e >> 3) & 12u); }
template <typename E>
constexpr bool kRowSwizzled = false;
template <>
constexpr bool kRowSwizzled<float> = true;

__device__ __forceinline__ void ld_row(const float* row, uint32_t key, float (&f)[16]) {
#pragma unroll
  for (int c = 0; c < 4; c++) {
    const float4 v = reinterpret_cast<const float4*>(row)[c ^ key];
    f[4 * c] = v.x;
    f[4 * c + 1] = v.y;
    f[4 * c + 2] = v.z;
    f[4 * c + 3] = v.w;
  }
}
__device__ __forceinline__ void st_row(int32_t* row, uint32_t key, const int32_t (&k)[16]) {
#pragma unroll
  for (int c = 0; c < 4; c++)
    reinterpret_cast<int4*>(row)[c ^ key] = make_int4(k[4 * c], k[4 * c + 1], k[4 * c + 2], k[4 * c + 3]);
}

// ---- shared memory -----------------------------------------------------------------
template <typename T, uint32_t NIN = kSlots>
struct SmemT {
  T in[2][NIN];                 // TMA destinations (box layout); in 3-D the current
                                // one then carries the partly differenced k
  int32_t zrow[16];             // zeros: the neighbour row of a chunk's first row / plane
  uint16_t c[kSlots];           // codes of the current tile (dense order)
  uint32_t hc[kNsymCode];       // code histogram (per CTA, current field)
  uint32_t hv[kNsymCode];       // run-value histogram
  uint32_t hl[kHlShared];       // run-length histogram (length - 1), short runs
  uint32_t patch[kSlots / 32];  // verbatim-patch positions
  uint32_t outl[kSlots / 32];   // outlier positions
  uint32_t head[kSlots / 32];   // run heads
  uint32_t woff[kSlots / 32 + 4];
  uint32_t next[kSlots / 32];
  unsigned long long scan[33];
  unsigned long long bar[2];    // mbarriers of the two buffers
  uint32_t box[2][6];           // origin and extent of each buffer's tile (thread 0 writes)
  T pq[3];                      // the current field's bound (Pq<T>::load)
};

// One TMA tile copy (box at element coordinates c0 (x), c1, c2) into shared memory.
__device__ __forceinline__ void tma_load(int rank, void* dst, const CUtensorMap* map, int32_t c0, int32_t c1,
                                         int32_t c2, unsigned long long* bar) {
  const uint32_t d = smem_u32(dst), b = smem_u32(bar);
  const uint64_t m = reinterpret_cast<uint64_t>(map);
  if (rank == 1) {
    asm volatile(
        "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2}], "
        "[%3];" ::"r"(d),
        "l"(m), "r"(c0), "r"(b)
        : "memory");
  } else if (rank == 2) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(d),
        "l"(m), "r"(c0), "r"(c1), "r"(b)
        : "memory");
  } else {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];" ::"r"(d),
        "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(b)
        : "memory");
  }
}

// Start fetching tile b of task T into buffer `buf` (thread 0 only).  The buffer was
// last touched by ordinary loads and stores, hence the proxy fence.
template <typename E>
__device__ void issue_tile(const ConstructTask* T, const uint32_t* org, E* buf, unsigned long long* bar) {
  const Geom& g = T->a.g;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, (uint32_t)(kSlots * sizeof(E)));
  if (g.ndim == 1) {
    // a 1-D box holds at most 256 elements: 16 copies
    for (int i = 0; i < kSlots / 256; i++)
      tma_load(1, buf + 256 * i, &T->tmap, (int32_t)(org[2] + 256 * i), 0, 0, bar);
  } else if (g.ndim == 2) {
    tma_load(2, buf, &T->tmap, (int32_t)org[2], (int32_t)org[1], 0, bar);
  } else {
    tma_load(3, buf, &T->tmap, (int32_t)org[2], (int32_t)org[1], (int32_t)org[0], bar);
  }
}

template <typename E>
__device__ __forceinline__ const E* field_ptr(const ConstructArgs& A);
template <>
__device__ __forceinline__ const float* field_ptr<float>(const ConstructArgs& A) { return A.x; }
template <>
__device__ __forceinline__ const double* field_ptr<double>(const ConstructArgs& A) { return A.x64; }

// Thread-loaded tile (fields TMA cannot describe): box layout (FP32 3-D boxes
// swizzled like their TMA copies), zeros outside.
template <typename E>
__device__ void load_tile_threads(const ConstructArgs& A, uint32_t b, E* buf) {
  const E* xs = field_ptr<E>(A);
  const Geom& g = A.g;
  uint32_t org[3], w[3];
  block_box(g, b, org, w);
  const uint64_t ny = g.n[1], nx = g.n[2];
  for (uint32_t p = threadIdx.x; p < (uint32_t)kSlots; p += kThreads) {
    uint32_t zz, yy, xx;
    if (g.ndim == 1) {
      zz = 0;
      yy = 0;
      xx = p;
    } else if (g.ndim == 2) {
      zz = 0;
      yy = p >> 6;
      xx = p & 63;
    } else {
      zz = p >> 8;
      yy = (p >> 4) & 15;
      xx = p & 15;
    }
    E v = E(0);
    if (zz < w[0] && yy < w[1] && xx < w[2]) v = xs[((uint64_t)(org[0] + zz) * ny + (org[1] + yy)) * nx + org[2] + xx];
    buf[kRowSwizzled<E> && g.ndim == 3 ? swz64(p) : p] = v;
  }
}

__device__ __forceinline__ void flush_hist(const uint32_t* h, int n, uint32_t* global) {
  for (int i = threadIdx.x; i < n; i += kThreads) {
    const uint32_t v = h[i];
    if (v) atomicAdd(&global[i], v);
  }
}

// ---- edge blocks (not inlined: keeps the full-block paths compact in the
// instruction cache): prequantize into registers in dense order, stage k, residuals
// from the staged neighbours.  Returns error bits.
template <int ND, typename E>
__device__ __noinline__ uint32_t edge_codes(const ConstructArgs& A, uint32_t b, SmemT<E>& S, E* in,
                                            const uint32_t* w, uint32_t m, int32_t* dglob) {
  const int tid = threadIdx.x, lane = tid & 31;
  const Pq<E> pq(S.pq);
  const int32_t r = (int32_t)A.radius;
  int32_t* s_k = reinterpret_cast<int32_t*>(in);
  uint32_t err = 0;
  int32_t kv[kPer];
  uint32_t pm = 0;
#pragma unroll
  for (int i = 0; i < kPer; i++) {
    const uint32_t j = tid + kThreads * i;
    kv[i] = 0;
    if (j < m) {
      uint32_t zz, yy, xx;
      if (ND == 1) {
        zz = 0;
        yy = 0;
        xx = j;
      } else if (ND == 2) {
        zz = 0;
        yy = j / w[2];
        xx = j - yy * w[2];
      } else {
        const uint32_t p = w[1] * w[2];
        zz = j / p;
        const uint32_t rr = j - zz * p;
        yy = rr / w[2];
        xx = rr - yy * w[2];
      }
      uint32_t box = ND == 1 ? xx : (ND == 2 ? yy * 64 + xx : (zz * 16 + yy) * 16 + xx);
      if (ND == 3 && kRowSwizzled<E>) box = swz64(box);
      bool p;
      err |= pq.full(in[box], kv[i], p);
      pm |= (uint32_t)p << i;
    }
  }
  __syncthreads();  // box read: it becomes s_k (dense)
#pragma unroll
  for (int i = 0; i < kPer; i++) {
    const uint32_t j = tid + kThreads * i;
    s_k[j] = kv[i];
    const uint32_t pb = __ballot_sync(~0u, (pm >> i) & 1u);
    if (lane == 0) S.patch[j >> 5] = pb;
  }
  __syncthreads();
  const uint32_t sy = w[2], sz = w[1] * w[2];
#pragma unroll
  for (int i = 0; i < kPer; i++) {
    const uint32_t j = tid + kThreads * i;
    int32_t delta = 0;
    uint16_t q = 0;
    const bool inb = j < m;
    (void)delta;
    if (inb) {
      uint32_t zz = 0, yy = 0, xx = j;
      if (ND == 2) {
        yy = j / w[2];
        xx = j - yy * w[2];
      } else if (ND == 3) {
        zz = j / sz;
        const uint32_t rr = j - zz * sz;
        yy = rr / w[2];
        xx = rr - yy * w[2];
      }
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
      atomicAdd(&S.hc[q], 1u);
    }
    S.c[j] = q;  // zero beyond m
    if (inb && q == 0) dglob[j] = delta;
    const uint32_t ob = __ballot_sync(~0u, inb && q == 0);
    if (lane == 0) S.outl[j >> 5] = ob;
  }
  __syncthreads();
    return err;
}

// ---- the tile's tail: run heads at word boundaries (full tiles), counts from the
// bit words, bulk copies of codes and masks, run histograms of run-eligible blocks
template <typename E, uint32_t NIN>
__device__ void tile_tail(const ConstructArgs& A, uint32_t b, SmemT<E, NIN>& S, uint32_t m, bool full, uint32_t err,
                          uint32_t& n_rec_acc, uint32_t& n_patch_acc) {
  const int tid = threadIdx.x, lane = tid & 31;
  // ---- head bit 0 of every word, then the tile's counts from the bit words -------
  // (outliers << 42 | patches << 21 | runs; each count is at most 4096)
  if (tid < kSlots / 32) {
    uint32_t hw = S.head[tid];
    if (full) {
      const uint32_t j0 = 32u * tid;
      hw |= (uint32_t)(tid == 0 || S.c[j0] != S.c[j0 - 1]);
      S.head[tid] = hw;
    }
    const unsigned long long v = ((unsigned long long)__popc(S.outl[tid]) << 42) |
                                 ((unsigned long long)__popc(S.patch[tid]) << 21) | (unsigned long long)__popc(hw);
    const unsigned long long ws = warp_sum(v);
    if (lane == 0) S.scan[tid >> 5] = ws;
  }
  __syncthreads();
  const unsigned long long tot = S.scan[0] + S.scan[1] + S.scan[2] + S.scan[3];
  constexpr uint64_t kF = (1ull << 21) - 1;
  const uint32_t n_out = (uint32_t)(tot >> 42), n_patch = (uint32_t)((tot >> 21) & kF);
  const uint32_t nruns = (uint32_t)(tot & kF);
  if (tid == 0) {
    A.counts[b] = (n_out << 16) | n_patch;
    A.block_runs[b] = (uint16_t)nruns;
    n_rec_acc += n_out + n_patch;
    n_patch_acc += n_patch;
    // codes to the block-major stream (whole 4096-slot block, zero tail) and the
    // patch / outlier bit words: bulk copies from shared memory, waited for before
    // those buffers are written again
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(A.codes + (uint64_t)b * kSlots),
                 "r"(smem_u32(S.c)), "r"((uint32_t)(kSlots * 2))
                 : "memory");
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(A.masks + (uint64_t)b * 256),
                 "r"(smem_u32(S.patch)), "r"((uint32_t)(2 * (kSlots / 32) * 4))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }

  // ---- run-eligible blocks: run-value and run-length histograms -----------------
  if (A.all_runs || 4 * nruns <= m) {
    if (tid < 32) run_head_index(S.head, m, S.woff, S.next);
    __syncthreads();
    // thread t: the run heads among slots 16t .. 16t + 15 (head bits are clear at and
    // beyond m); a run ends at the next head in these bits, else at the next head after
    // slot 16t + 15.  Single-element runs are counted in a register and added once per
    // warp.
    uint32_t ones = 0;
    const uint32_t j0 = 16u * tid;
    uint32_t hb = (S.head[tid >> 1] >> (16 * (tid & 1))) & 0xffffu;
    while (hb) {
      const uint32_t j = j0 + (uint32_t)(__ffs(hb) - 1);
      hb &= hb - 1;
      const uint32_t end = hb ? j0 + (uint32_t)(__ffs(hb) - 1) : next_head(S.head, S.next, j0 + 15, m);
      const uint32_t len = end - j;
      atomicAdd(&S.hv[S.c[j]], 1u);
      if (len == 1)
        ones++;
      else if (len <= (uint32_t)kHlShared)
        atomicAdd(&S.hl[len - 1], 1u);
      else
        atomicAdd(&A.hist_len[len - 1], 1u);
    }
    ones = warp_sum(ones);
    if (lane == 0 && ones) atomicAdd(&S.hl[0], ones);
  }
  // the next block writes S.c, S.patch and S.outl again (after the caller's barrier)
  if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  if (err) atomicOr(&A.st->status, err);
}

// Postquantization of one thread's 16 consecutive slots j0 .. j0 + 15 (j0 = 16 t) from
// u = delta + r: codes (two 16-byte stores), outlier residuals, the slots' outlier /
// patch / run-head bits (two threads fill one 32-bit word) and the code histogram (one
// add when the 16 codes agree).  Head bit 0 of lane 0 compares with another warp's
// slot: it is left clear here and set after the tile.
template <typename SM>
__device__ __forceinline__ void post16(SM& S, const uint32_t (&u)[16], uint32_t pm, int32_t r, int32_t* dglob) {
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t j0 = 16u * tid;
  uint32_t q[16], om = 0, hm = 0;
#pragma unroll
  for (int i = 0; i < 16; i++) {
    q[i] = u[i] - 1u < (uint32_t)(2 * r - 1) ? u[i] : 0u;  // |delta| < r
    om |= (uint32_t)(q[i] == 0) << i;
    if (i) hm |= (uint32_t)(q[i] != q[i - 1]) << i;
  }
  uint4* cw = reinterpret_cast<uint4*>(S.c + j0);
  cw[0] = make_uint4(q[0] | q[1] << 16, q[2] | q[3] << 16, q[4] | q[5] << 16, q[6] | q[7] << 16);
  cw[1] = make_uint4(q[8] | q[9] << 16, q[10] | q[11] << 16, q[12] | q[13] << 16, q[14] | q[15] << 16);
  if (om) {
#pragma unroll
    for (int i = 0; i < 16; i++)
      if ((om >> i) & 1u) dglob[j0 + i] = (int32_t)(u[i] - (uint32_t)r);
  }
  if ((hm >> 1) == 0) {
    atomicAdd(&S.hc[q[0]], 16u);
  } else {
#pragma unroll
    for (int i = 0; i < 16; i++) atomicAdd(&S.hc[q[i]], 1u);
  }
  const uint32_t qb = __shfl_up_sync(~0u, q[15], 1);
  if (lane != 0 && q[0] != qb) hm |= 1u;
  const uint32_t om2 = __shfl_down_sync(~0u, om, 1), pm2 = __shfl_down_sync(~0u, pm, 1),
                 hm2 = __shfl_down_sync(~0u, hm, 1);
  if ((lane & 1) == 0) {
    S.outl[tid >> 1] = om | (om2 << 16);
    S.patch[tid >> 1] = pm | (pm2 << 16);
    S.head[tid >> 1] = hm | (hm2 << 16);
  }
}

// ---- one tile ------------------------------------------------------------------------
// Codes, records and histogram updates of codec block b (origin box[0..2], extent
// box[3..5]) from the box in `in` (which this call overwrites with k and outlier
// deltas).  Thread 0 adds the tile's record and patch counts to n_rec_acc /
// n_patch_acc.
template <int ND, typename E>
__device__ void process_tile(const ConstructArgs& A, uint32_t b, const uint32_t* box, SmemT<E>& S, E* in,
                             uint32_t& n_rec_acc, uint32_t& n_patch_acc) {
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t w[3] = {box[3], box[4], box[5]};
  const uint32_t m = w[0] * w[1] * w[2];
  const Pq<E> pq(S.pq);
  const int32_t r = (int32_t)A.radius;
  const Geom& g = A.g;
  const bool full = w[0] == g.blk[0] && w[1] == g.blk[1] && w[2] == g.blk[2];
  int32_t* s_k = reinterpret_cast<int32_t*>(in);
  int32_t* dglob = A.deltas + (uint64_t)b * kSlots;  // outlier residuals of this block, by slot
  uint32_t err = 0;

  // Postquantization of one warp step over the 32 consecutive slots of word j >> 5:
  // code, outlier delta, the word's outlier / patch / run-head bits, and the code
  // histogram (one add for the whole step when its 32 codes agree, as in zero
  // regions).  Head bit 0 compares with the previous word, written by another warp:
  // it is left clear here and set after the tile.
  auto post = [&](int32_t delta, uint32_t j, bool patch_step, bool patch_bit) {
    const uint32_t u = (uint32_t)(delta + r);
    const uint32_t q = u - 1u < (uint32_t)(2 * r - 1) ? u : 0u;  // |delta| < r
    S.c[j] = (uint16_t)q;
    if (q == 0) dglob[j] = delta;
    const uint32_t left = __shfl_up_sync(~0u, q, 1);
    const uint32_t hd = __ballot_sync(~0u, lane != 0 && q != left);
    const uint32_t ob = __ballot_sync(~0u, q == 0);
    const uint32_t pb = patch_step ? __ballot_sync(~0u, patch_bit) : 0u;
    if (hd == 0) {
      if (lane == 0) atomicAdd(&S.hc[q], 32u);
    } else {
      atomicAdd(&S.hc[q], 1u);
    }
    if (lane == 0) {
      S.head[j >> 5] = hd;
      S.outl[j >> 5] = ob;
      S.patch[j >> 5] = pb;
    }
  };

  // ---- prequantization, Lorenzo residual (Sec. IV-B2), postquantization ----------
  // The residual is the mixed difference (1 - S_x)(1 - S_y)(1 - S_z) k, each shift
  // reading zero outside the chunk; that expansion is the paper's 1/2/3-D predictor.
  if (full) {
    if (ND == 1) {
      // thread t: 16 consecutive elements (a warp covers two whole 256-chunks)
      int32_t k[16];
      uint32_t pm = 0;
      E f[16];
      load16(in + 16 * tid, f);
      bool ok = true;
#pragma unroll
      for (int i = 0; i < 16; i++) ok = pq.fast(f[i], k[i]) & ok;
      if (!__all_sync(~0u, ok)) {
#pragma unroll
        for (int i = 0; i < 16; i++) {
          int32_t kk;
          if (!pq.fast(f[i], kk)) {
            bool p;
            err |= pq.full(f[i], k[i], p);
            pm |= (uint32_t)p << i;
          }
        }
      }
      const int32_t up = __shfl_up_sync(~0u, k[15], 1);
      const int32_t prev = (tid & 15) ? up : 0;  // a 256-chunk is 16 threads
      uint32_t u[16];
#pragma unroll
      for (int i = 0; i < 16; i++) u[i] = (uint32_t)(k[i] - (i ? k[i - 1] : prev) + r);
      post16(S, u, pm, r, dglob);
    } else if (ND == 2) {
      // thread t: column xx = t & 63 of the 16-row chunk band t >> 6
      const uint32_t xx = tid & 63, ry = tid >> 6;
      int32_t k[16];
      uint32_t pm = 0, slow = 0;
#pragma unroll
      for (int i = 0; i < 16; i++)
        slow |= (uint32_t)!pq.fast(in[(16 * ry + i) * 64 + xx], k[i]) << i;
      if (__any_sync(~0u, slow != 0)) {
#pragma unroll
        for (int i = 0; i < 16; i++) {
          if ((slow >> i) & 1u) {
            bool p;
            err |= pq.full(in[(16 * ry + i) * 64 + xx], k[i], p);
            pm |= (uint32_t)p << i;
          }
        }
      }
      const bool anyp = __any_sync(~0u, pm != 0);
#pragma unroll
      for (int i = 15; i > 0; i--) k[i] -= k[i - 1];  // y difference within the chunk band
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const int32_t left = __shfl_up_sync(~0u, k[i], 1);
        const int32_t delta = (xx & 15) ? k[i] - left : k[i];  // x difference
        const uint32_t j = (16 * ry + i) * 64 + xx;
        post(delta, j, anyp, (pm >> i) & 1u);
      }
    } else if constexpr (kRowSwizzled<E>) {
      // FP32: thread t holds the x row (z, y) = (t >> 4, t & 15), two 8-chunks along x,
      // i.e. the 16 consecutive slots 16t .. 16t + 15.  The x difference runs in
      // registers; the y and z differences read the rows t - 1, t - 16 and t - 17 (the
      // zero row at a chunk's first row or plane), which by then hold their x differences.
      const uint32_t zz = tid >> 4, yy = tid & 15, key = (tid >> 1) & 3;
      float f[16];
      ld_row(in + 16 * tid, key, f);
      int32_t k[16];
      bool ok = true;
#pragma unroll
      for (int i = 0; i < 16; i++) ok = pq.fast(f[i], k[i]) & ok;
      uint32_t pm = 0;
      if (!__all_sync(~0u, ok)) {
#pragma unroll
        for (int i = 0; i < 16; i++) {
          int32_t kk;
          if (!pq.fast(f[i], kk)) {
            bool p;
            err |= pq.full(f[i], k[i], p);
            pm |= (uint32_t)p << i;
          }
        }
      }
#pragma unroll
      for (int i = 15; i > 0; i--)
        if (i & 7) k[i] -= k[i - 1];  // x difference within 8-chunks
      // the box carries the x differences from here: each thread overwrites only its own
      // row, which only it has read, so no barrier comes first; the neighbour rows lie
      // in the same 8-plane chunk, and planes 0-7 (8-15) belong to threads 0-127
      // (128-255), so each half of the CTA waits only for itself (named barriers 1, 2)
      st_row(s_k + 16 * tid, key, k);
      asm volatile("bar.sync %0, %1;" ::"r"(1 + (tid >> 7)), "r"(128) : "memory");
      const bool hy = (yy & 7) != 0, hz = (zz & 7) != 0;
      const int ty = hy ? tid - 1 : 0, tz = hz ? tid - 16 : 0, tyz = hy && hz ? tid - 17 : 0;
      const int4* ry = reinterpret_cast<const int4*>(hy ? s_k + 16 * ty : S.zrow);
      const int4* rz = reinterpret_cast<const int4*>(hz ? s_k + 16 * tz : S.zrow);
      const int4* ryz = reinterpret_cast<const int4*>(hy && hz ? s_k + 16 * tyz : S.zrow);
      // rows t - 16 and t - 17 have the swizzle keys of rows t and t - 1
      const uint32_t ky = ((uint32_t)(tid + 7) >> 1) & 3;  // = ((t - 1) >> 1) & 3 for t >= 1
      uint32_t u[16];
#pragma unroll
      for (int c = 0; c < 4; c++) {
        const int4 a = ry[c ^ ky], bz = rz[c ^ key], d = ryz[c ^ ky];
        u[4 * c] = (uint32_t)(k[4 * c] - a.x - bz.x + d.x + r);
        u[4 * c + 1] = (uint32_t)(k[4 * c + 1] - a.y - bz.y + d.y + r);
        u[4 * c + 2] = (uint32_t)(k[4 * c + 2] - a.z - bz.z + d.z + r);
        u[4 * c + 3] = (uint32_t)(k[4 * c + 3] - a.w - bz.w + d.w + r);
      }
      post16(S, u, pm, r, dglob);
    } else {
      // thread t: z column of (xx, yy) = (t & 15, t >> 4); z and x differences in
      // registers and shuffles, the y difference through shared memory
      const uint32_t xx = tid & 15, yy = tid >> 4;
      int32_t k[16];
      uint32_t pm = 0, slow = 0;
#pragma unroll
      for (int i = 0; i < 16; i++)
        slow |= (uint32_t)!pq.fast(in[(i * 16 + yy) * 16 + xx], k[i]) << i;
      if (__any_sync(~0u, slow != 0)) {
#pragma unroll
        for (int i = 0; i < 16; i++) {
          if ((slow >> i) & 1u) {
            bool p;
            err |= pq.full(in[(i * 16 + yy) * 16 + xx], k[i], p);
            pm |= (uint32_t)p << i;
          }
        }
      }
#pragma unroll
      for (int i = 15; i > 0; i--)
        if (i & 7) k[i] -= k[i - 1];  // z difference within 8-chunks
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const int32_t left = __shfl_up_sync(~0u, k[i], 1);
        if (xx & 7) k[i] -= left;  // x difference
      }
      const bool anyp = __any_sync(~0u, pm != 0);
      // the box carries k from here: each thread overwrites only its own column, which
      // only it has read, so no barrier comes first; the y difference reads the row
      // below in the same 8-row chunk, and rows 0-7 (8-15) belong to warps 0-3 (4-7),
      // so each group of four warps waits only for itself (named barriers 1 and 2)
#pragma unroll
      for (int i = 0; i < 16; i++) s_k[(i * 16 + yy) * 16 + xx] = k[i];
      asm volatile("bar.sync %0, %1;" ::"r"(1 + (tid >> 7)), "r"(128) : "memory");
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const uint32_t j = (i * 16 + yy) * 16 + xx;
        const int32_t below = (yy & 7) ? s_k[(i * 16 + yy - 1) * 16 + xx] : 0;
        post(k[i] - below, j, anyp, (pm >> i) & 1u);
      }
    }
    __syncthreads();
  } else {
    err |= edge_codes<ND, E>(A, b, S, in, w, m, dglob);
    run_head_words(S.c, m, S.head);
    __syncthreads();
  }

  tile_tail(A, b, S, m, full, err, n_rec_acc, n_patch_acc);
}

// ---- global (unchunked) Lorenzo: tiles with a halo -----------------------------------
// The box holds the tile and the elements one step before it on every axis, so the
// predictor of the tile's first row, column and plane reads its real neighbours
// instead of zeros; x is padded to four elements before the tile so that the box
// starts on a 16-byte boundary (the TMA's rule).  Outside the field the box reads
// zero: the predictor's boundary at the field's faces.
template <int ND>
struct Halo;
template <>
struct Halo<1> {
  static constexpr uint32_t X = 17 * 256, Y = 1, Z = 1;  // 17 copies of 256 from x0 - 4
};
template <>
struct Halo<2> {
  static constexpr uint32_t X = 68, Y = 65, Z = 1;
};
template <>
struct Halo<3> {
  static constexpr uint32_t X = 20, Y = 17, Z = 17;
};
constexpr uint32_t kHaloPadX = 4;
// the largest box (3-D, 5780 elements) rounded up to 32 elements, so each buffer
// starts 128-byte aligned like the chunked tiles
constexpr uint32_t kHaloMax = (20 * 17 * 17 + 31) / 32 * 32;
static_assert(Halo<1>::X <= kHaloMax && Halo<2>::X * Halo<2>::Y <= kHaloMax, "halo boxes fit the buffer");

template <typename E>
__device__ void issue_tile_global(const ConstructTask* T, const uint32_t* org, E* buf, unsigned long long* bar) {
  const Geom& g = T->a.g;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const int32_t x0 = (int32_t)org[2] - (int32_t)kHaloPadX;
  if (g.ndim == 1) {
    mbar_expect_tx(bar, (uint32_t)(Halo<1>::X * sizeof(E)));
    for (int i = 0; i < 17; i++) tma_load(1, buf + 256 * i, &T->tmap, x0 + 256 * i, 0, 0, bar);
  } else if (g.ndim == 2) {
    mbar_expect_tx(bar, (uint32_t)(Halo<2>::X * Halo<2>::Y * sizeof(E)));
    tma_load(2, buf, &T->tmap, x0, (int32_t)org[1] - 1, 0, bar);
  } else {
    mbar_expect_tx(bar, (uint32_t)(Halo<3>::X * Halo<3>::Y * Halo<3>::Z * sizeof(E)));
    tma_load(3, buf, &T->tmap, x0, (int32_t)org[1] - 1, (int32_t)org[0] - 1, bar);
  }
}

// Thread-loaded halo box (fields TMA cannot describe), zeros outside the field.
template <int ND, typename E>
__device__ void load_halo_threads(const ConstructArgs& A, const uint32_t* org, E* buf) {
  using H = Halo<ND>;
  constexpr uint32_t NB = H::X * H::Y * H::Z;
  constexpr int hz = ND == 3 ? 1 : 0, hy = ND >= 2 ? 1 : 0;
  const E* xs = field_ptr<E>(A);
  const Geom& g = A.g;
  for (uint32_t p = threadIdx.x; p < NB; p += kThreads) {
    const int64_t x = (int64_t)org[2] + (int64_t)(p % H::X) - (int64_t)kHaloPadX;
    const int64_t y = (int64_t)org[1] + (int64_t)((p / H::X) % H::Y) - hy;
    const int64_t z = (int64_t)org[0] + (int64_t)(p / (H::X * H::Y)) - hz;
    E v = E(0);
    if (x >= 0 && y >= 0 && z >= 0 && x < (int64_t)g.n[2] && y < (int64_t)g.n[1] && z < (int64_t)g.n[0])
      v = xs[((uint64_t)z * g.n[1] + (uint64_t)y) * g.n[2] + (uint64_t)x];
    buf[p] = v;
  }
}

// Codes, records and histograms of codec block b under the global predictor: the
// halo'd box is prequantized in place (each element's k as int32), then every slot's
// residual is the mixed difference (1 - S_x)(1 - S_y)(1 - S_z) k over the box (the
// paper's 1/2/3-D predictor, Sec. IV-B2, with no chunk restarts), then the tail.
template <int ND, typename E>
__device__ void process_tile_global(const ConstructArgs& A, uint32_t b, const uint32_t* box,
                                    SmemT<E, kHaloMax>& S, E* in, uint32_t& n_rec_acc, uint32_t& n_patch_acc) {
  using H = Halo<ND>;
  constexpr uint32_t NB = H::X * H::Y * H::Z;
  constexpr uint32_t PER = (NB + kThreads - 1) / kThreads;
  constexpr int hz = ND == 3 ? 1 : 0, hy = ND >= 2 ? 1 : 0;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t w[3] = {box[3], box[4], box[5]};
  const uint32_t m = w[0] * w[1] * w[2];
  const Pq<E> pq(S.pq);
  const int32_t r = (int32_t)A.radius;
  int32_t* dglob = A.deltas + (uint64_t)b * kSlots;
  uint32_t err = 0;
  if (tid < kSlots / 32) S.patch[tid] = 0;
  __syncthreads();
  // prequantize every box element the predictor reads (x >= -1) into registers
  int32_t kv[PER];
#pragma unroll
  for (uint32_t i = 0; i < PER; i++) {
    const uint32_t p = tid + kThreads * i;
    kv[i] = 0;
    if (p < NB) {
      const int x = (int)(p % H::X) - (int)kHaloPadX;
      const int y = (int)((p / H::X) % H::Y) - hy, z = (int)(p / (H::X * H::Y)) - hz;
      if (x >= -1) {
        bool patch = false;
        if (!pq.fast(in[p], kv[i])) err |= pq.full(in[p], kv[i], patch);
        if (patch && x >= 0 && y >= 0 && z >= 0 && (uint32_t)x < w[2] && (uint32_t)y < w[1] && (uint32_t)z < w[0]) {
          const uint32_t j = ((uint32_t)z * w[1] + (uint32_t)y) * w[2] + (uint32_t)x;
          atomicOr(&S.patch[j >> 5], 1u << (j & 31));
        }
      }
    }
  }
  __syncthreads();  // every element read: the box now carries k (int32, from its start)
  int32_t* K = reinterpret_cast<int32_t*>(in);
#pragma unroll
  for (uint32_t i = 0; i < PER; i++) {
    const uint32_t p = tid + kThreads * i;
    if (p < NB) K[p] = kv[i];
  }
  __syncthreads();
#pragma unroll 4
  for (int i = 0; i < kPer; i++) {
    const uint32_t j = tid + kThreads * i;
    const bool inb = j < m;
    uint32_t q = 0;
    if (inb) {
      uint32_t x = j, y = 0, z = 0;
      if (ND == 2) {
        y = j / w[2];
        x = j - y * w[2];
      } else if (ND == 3) {
        const uint32_t pl = w[1] * w[2];
        z = j / pl;
        const uint32_t rr = j - z * pl;
        y = rr / w[2];
        x = rr - y * w[2];
      }
      const uint32_t p = ((z + hz) * H::Y + (y + hy)) * H::X + (x + kHaloPadX);
      int32_t d = K[p] - K[p - 1];
      if (ND >= 2) d -= K[p - H::X] - K[p - H::X - 1];
      if (ND == 3) {
        constexpr uint32_t PL = H::X * H::Y;
        d -= K[p - PL] - K[p - PL - 1];
        d += K[p - PL - H::X] - K[p - PL - H::X - 1];
      }
      const uint32_t u = (uint32_t)(d + r);
      q = u - 1u < (uint32_t)(2 * r - 1) ? u : 0u;  // |delta| < r
      atomicAdd(&S.hc[q], 1u);
      if (q == 0) dglob[j] = d;
    }
    S.c[j] = (uint16_t)q;  // zero beyond m
    const uint32_t ob = __ballot_sync(~0u, inb && q == 0);
    if (lane == 0) S.outl[j >> 5] = ob;
  }
  __syncthreads();
  run_head_words(S.c, m, S.head);
  __syncthreads();
  tile_tail(A, b, S, m, false, err, n_rec_acc, n_patch_acc);
}

__device__ __forceinline__ int find_field(const uint32_t* tile0, int nfields, uint32_t t, int hint) {
  if (t < tile0[hint + 1]) return hint;
  int lo = hint + 1, hi = nfields - 1;  // tile0[lo] <= t
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile0[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}



// Persistent construction over the tiles of `nfields` fields.  The single-field
// entry passes the task by value (`one`, tasks == nullptr, ntiles = its block
// count); batches pass a device table and tile0[f], the first global tile of field
// f (tile0[nfields] = ntiles).
// ND 1, 2, 3; 0 = any (batches of mixed dimensionality); E the element type; G the
// global (unchunked) predictor with halo'd tiles; P the phase of the batched
// persistent kernel, where nothing orders this phase after the value-range phase or
// the book phase after this one: before a field's first tile the CTA waits for the
// field's bound (DevState::ready_range, set by the range phase), and after it hands
// a field's histograms on it adds the field's tiles to DevState::tiles_flushed (once
// its bulk copies have completed), which the book phase waits for.
// smem_raw: the dynamic shared memory, 1024-byte aligned for the TMA swizzle.
template <int ND, typename E, bool G, bool P>
__device__ __forceinline__ void construct_loop(const ConstructTask& one, const ConstructTask* __restrict__ tasks,
                                               const uint32_t* __restrict__ tile0, int nfields, uint32_t ntiles,
                                               uint32_t* ticket, uint32_t spin_limit, unsigned char* smem_raw) {
  using SM = SmemT<E, G ? kHaloMax : kSlots>;
  SM& S = *reinterpret_cast<SM*>(smem_raw);
  // the swizzled FP32 3-D copies assume 1024-byte aligned buffers: without that
  // alignment every tile is loaded by the threads (same placement, no TMA)
  const bool tma_ok = (smem_u32(smem_raw) & 1023u) == 0;
  __shared__ uint32_t s_t[2];
  __shared__ int s_f[2];
  uint32_t n_rec_acc = 0, n_patch_acc = 0, pending = 0;  // thread 0: the field's counts, the next ticket
  uint32_t ntile_acc = 0;                                 // thread 0 (P): the field's tiles since its last flush
  const int tid = threadIdx.x;
  auto task = [&](int f) -> const ConstructTask* { return tasks ? &tasks[f] : &one; };
  auto base = [&](int f) -> uint32_t { return tasks ? tile0[f] : 0u; };
  // thread 0: ticket t goes to buffer `slot`: its field, its box, and its fetch.
  // Tickets are drawn one tile ahead of the fetches (`pending`), so the counter's
  // round trip overlaps the work on the current tile.  (A fixed stride over the tiles
  // measured slower: tiles differ in cost, and the counter balances them.)
  auto claim = [&](int slot, uint32_t t, int hint) {
    const int f = t < ntiles ? (tasks ? find_field(tile0, nfields, t, hint) : 0) : -1;
    s_t[slot] = t;
    s_f[slot] = f;
    if (f >= 0) {
      uint32_t* bx = S.box[slot];
      block_box(task(f)->a.g, t - base(f), bx, bx + 3);
      if (task(f)->use_tma && tma_ok) {
        if (G) issue_tile_global(task(f), bx, S.in[slot], &S.bar[slot]);
        else issue_tile(task(f), bx, S.in[slot], &S.bar[slot]);
      }
    }
  };

  if (tid == 0) {
    mbar_init(&S.bar[0]);
    mbar_init(&S.bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    claim(0, atomicAdd(ticket, 1u), 0);
    pending = atomicAdd(ticket, 1u);
  }
  for (int i = tid; i < kNsymCode + kNsymCode + kHlShared; i += kThreads) S.hc[i] = 0;  // hc, hv, hl
  if (tid < 16) S.zrow[tid] = 0;
  __syncthreads();

  int cur = 0, field = -1;
  bool failed = false;
  uint32_t phase = 0u;  // bit i: the phase awaited on buffer i
  auto flush_field = [&](int f) {
    const ConstructArgs& P = task(f)->a;
    flush_hist(S.hc, kNsymCode, P.hist_code);
    flush_hist(S.hv, kNsymCode, P.hist_val);
    flush_hist(S.hl, kHlShared, P.hist_len);
    if (tid == 0) {
      if (n_rec_acc) atomicAdd(&P.st->n_rec, (unsigned long long)n_rec_acc);
      if (n_patch_acc) atomicAdd(&P.st->n_patch, (unsigned long long)n_patch_acc);
      n_rec_acc = n_patch_acc = 0;
    }
  };
  // P, thread 0, after the CTA's barrier that follows flush_field: the field's code
  // and mask copies complete, then the release of its tile count
  auto signal_field = [&](int f, uint32_t ntl) {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __threadfence();
    if (ntl) atomicAdd(&task(f)->a.st->tiles_flushed, ntl);
  };
  // P, thread 0: the field's bound must be derived before its first tile
  auto await_bound = [&](int f) {
    if (!wait_ge_acquire(&task(f)->a.st->ready_range, 1u, spin_limit)) atomicOr(&task(f)->a.st->status, ERR_TIMEOUT);
  };
  while (true) {
    const uint32_t t = s_t[cur];
    const int f = s_f[cur];
    if (f < 0) break;
    const ConstructTask* T = task(f);
    // claim the next tile and start its fetch before working on this one
    if (tid == 0) {
      claim(cur ^ 1, pending, f);
      pending = atomicAdd(ticket, 1u);
    }
    if (f != field) {
      // moving to another field: the previous one's histograms and counters go out
      if (field >= 0) {
        flush_field(field);
        __syncthreads();
        if (P && tid == 0) {
          signal_field(field, ntile_acc);
          ntile_acc = 0;
        }
        for (int i = tid; i < kNsymCode + kNsymCode + kHlShared; i += kThreads) S.hc[i] = 0;
        if (tid == 0) {
          if (P) await_bound(f);
          Pq<E>::load(T->a.st, S.pq);
        }
        __syncthreads();
      } else {
        if (tid == 0) {
          if (P) await_bound(f);
          Pq<E>::load(T->a.st, S.pq);
        }
        __syncthreads();
      }
      field = f;
    }
    const ConstructArgs& A = T->a;
    const uint32_t b = t - base(f);
    bool late = false;
    if (T->use_tma && tma_ok) {
      // every thread observes the completion itself (acquire of the TMA writes), so no
      // barrier follows; the phase advances only when the wait succeeded, so that after
      // a timeout the drain below still waits on the phase of the copy that did not
      // complete.  A thread that gave up works on whatever the buffer holds (every index
      // stays in range whatever the data) and the CTA leaves after the tile.
      if (mbar_wait(&S.bar[cur], (phase >> cur) & 1u, spin_limit)) {
        phase ^= 1u << cur;
      } else {
        atomicOr(&A.st->status, ERR_TIMEOUT);
        late = true;
      }
    } else {
      if (G) load_halo_threads<ND == 0 ? 3 : ND, E>(A, S.box[cur], S.in[cur]);
      else load_tile_threads(A, b, S.in[cur]);
      __syncthreads();
    }
    const uint32_t* bx = S.box[cur];
    if constexpr (G) {
      static_assert(ND != 0, "global tiles: one dimensionality per launch");
      process_tile_global<ND == 0 ? 3 : ND, E>(A, b, bx, S, S.in[cur], n_rec_acc, n_patch_acc);
    } else {
      if (ND == 1 || (ND == 0 && A.g.ndim == 1)) process_tile<1, E>(A, b, bx, S, S.in[cur], n_rec_acc, n_patch_acc);
      else if (ND == 2 || (ND == 0 && A.g.ndim == 2))
        process_tile<2, E>(A, b, bx, S, S.in[cur], n_rec_acc, n_patch_acc);
      else process_tile<3, E>(A, b, bx, S, S.in[cur], n_rec_acc, n_patch_acc);
    }
    if (P && tid == 0) ntile_acc++;
    if (__syncthreads_or(late)) {
      failed = true;
      break;
    }
    cur ^= 1;
  }
  if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  if (failed) {
    // a fetch did not complete in time: wait once more (bounded) for both buffers'
    // copies so no transfer outlives the CTA, then leave (bit cur of `phase` still
    // names the phase of the copy that timed out, bit cur ^ 1 that of the one issued
    // after it)
    if (tid == 0) {
      mbar_wait(&S.bar[cur], (phase >> cur) & 1u, spin_limit);
      if (s_f[cur ^ 1] >= 0 && task(s_f[cur ^ 1])->use_tma && tma_ok)
        mbar_wait(&S.bar[cur ^ 1], (phase >> (cur ^ 1)) & 1u, spin_limit);
      if (P) {
        // the later phases still count on every tile: the current field's, the one
        // claimed next and the ticket drawn after it are handed on unprocessed (the
        // status already says that the results are void)
        signal_field(field, ntile_acc);
        auto abandon = [&](int f2) {
          atomicOr(&task(f2)->a.st->status, ERR_TIMEOUT);
          signal_field(f2, 1u);
        };
        if (s_f[cur ^ 1] >= 0) abandon(s_f[cur ^ 1]);
        if (pending < ntiles) abandon(tasks ? find_field(tile0, nfields, pending, 0) : 0);
      }
    }
    if (P) {
      if (tid == 0) {
        mbar_inval(&S.bar[0]);
        mbar_inval(&S.bar[1]);
      }
      __syncthreads();
    }
    return;
  }
  if (field >= 0) flush_field(field);
  if (P) __syncthreads();
  if (tid == 0) {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (P) {
      if (field >= 0) signal_field(field, ntile_acc);
      // the buffers become other phases' shared memory
      mbar_inval(&S.bar[0]);
      mbar_inval(&S.bar[1]);
    }
  }
  if (P) __syncthreads();
}

}  // namespace
}  // namespace cons
}  // namespace cszp
