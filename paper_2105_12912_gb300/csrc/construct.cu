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
#include <cuda.h>

#include "common.cuh"
#include "kernels.h"

namespace cszp {

namespace {

constexpr int kThreads = 256;
constexpr int kPer = kSlots / kThreads;  // 16 elements per thread
constexpr uint32_t kTileBytes = kSlots * 4;
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

// ---- shared memory -----------------------------------------------------------------
struct Smem {
  float in[2][kSlots];          // TMA destinations (box layout); in 3-D the current
                                // one then carries k for the y difference
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
__device__ void issue_tile(const ConstructTask* T, const uint32_t* org, float* buf, unsigned long long* bar) {
  const Geom& g = T->a.g;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_expect_tx(bar, kTileBytes);
  if (g.ndim == 1) {
    // a 1-D box holds at most 256 elements: 16 copies of 1 KB
    for (int i = 0; i < kSlots / 256; i++)
      tma_load(1, buf + 256 * i, &T->tmap, (int32_t)(org[2] + 256 * i), 0, 0, bar);
  } else if (g.ndim == 2) {
    tma_load(2, buf, &T->tmap, (int32_t)org[2], (int32_t)org[1], 0, bar);
  } else {
    tma_load(3, buf, &T->tmap, (int32_t)org[2], (int32_t)org[1], (int32_t)org[0], bar);
  }
}

// Thread-loaded tile (fields TMA cannot describe): box layout, zeros outside.
__device__ void load_tile_threads(const ConstructArgs& A, uint32_t b, float* buf) {
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
    float v = 0.0f;
    if (zz < w[0] && yy < w[1] && xx < w[2])
      v = A.x[((uint64_t)(org[0] + zz) * ny + (org[1] + yy)) * nx + org[2] + xx];
    buf[p] = v;
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
template <int ND>
__device__ __noinline__ uint32_t edge_codes(const ConstructArgs& A, uint32_t b, Smem& S, float* in,
                                            const uint32_t* w, uint32_t m, int32_t* dglob) {
  const int tid = threadIdx.x, lane = tid & 31;
  const float eb_f = A.st->eb_f, ebx2_f = A.st->ebx2_f, ebx2_r = A.st->ebx2_r;
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
      const uint32_t box = ND == 1 ? xx : (ND == 2 ? yy * 64 + xx : (zz * 16 + yy) * 16 + xx);
      bool p;
      err |= prequant(in[box], eb_f, ebx2_f, ebx2_r, kv[i], p);
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

// ---- one tile ------------------------------------------------------------------------
// Codes, records and histogram updates of codec block b (origin box[0..2], extent
// box[3..5]) from the box in `in` (which this call overwrites with k and outlier
// deltas).  Thread 0 adds the tile's record and patch counts to n_rec_acc /
// n_patch_acc.
template <int ND>
__device__ void process_tile(const ConstructArgs& A, uint32_t b, const uint32_t* box, Smem& S, float* in,
                             uint32_t& n_rec_acc, uint32_t& n_patch_acc) {
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t w[3] = {box[3], box[4], box[5]};
  const uint32_t m = w[0] * w[1] * w[2];
  const float eb_f = A.st->eb_f, ebx2_f = A.st->ebx2_f, ebx2_r = A.st->ebx2_r;
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
      uint32_t pm = 0, slow = 0;
      const float4* in4 = reinterpret_cast<const float4*>(in) + 4 * tid;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const float4 v = in4[i];
        const float f[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int c = 0; c < 4; c++)
          slow |= (uint32_t)!prequant_fast(f[c], eb_f, ebx2_f, ebx2_r, k[4 * i + c]) << (4 * i + c);
      }
      if (__any_sync(~0u, slow != 0)) {
#pragma unroll
        for (int i = 0; i < 16; i++) {
          if ((slow >> i) & 1u) {
            bool p;
            err |= prequant(in[16 * tid + i], eb_f, ebx2_f, ebx2_r, k[i], p);
            pm |= (uint32_t)p << i;
          }
        }
      }
      const int32_t prev = __shfl_up_sync(~0u, k[15], 1);
      uint32_t om = 0, hm = 0, qprev = 0, qfirst = 0;
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const uint32_t j = 16 * tid + i;
        const int32_t left = i ? k[i - 1] : prev;
        const int32_t delta = (j & 255) ? k[i] - left : k[i];
        const uint32_t u = (uint32_t)(delta + r);
        const uint32_t q = u - 1u < (uint32_t)(2 * r - 1) ? u : 0u;  // |delta| < r
        S.c[j] = (uint16_t)q;
        if (q == 0) dglob[j] = delta;
        atomicAdd(&S.hc[q], 1u);
        om |= (uint32_t)(q == 0) << i;
        if (i == 0) qfirst = q;
        else hm |= (uint32_t)(q != qprev) << i;
        qprev = q;
      }
      // the first slot's left neighbour is the last slot of the lane below (lane 0:
      // another warp's, set after the tile)
      const uint32_t qbelow = __shfl_up_sync(~0u, qprev, 1);
      if (lane != 0 && qfirst != qbelow) hm |= 1u;
      const uint32_t om2 = __shfl_down_sync(~0u, om, 1), pm2 = __shfl_down_sync(~0u, pm, 1),
                     hm2 = __shfl_down_sync(~0u, hm, 1);
      if ((lane & 1) == 0) {
        S.outl[tid >> 1] = om | (om2 << 16);
        S.patch[tid >> 1] = pm | (pm2 << 16);
        S.head[tid >> 1] = hm | (hm2 << 16);
      }
    } else if (ND == 2) {
      // thread t: column xx = t & 63 of the 16-row chunk band t >> 6
      const uint32_t xx = tid & 63, ry = tid >> 6;
      int32_t k[16];
      uint32_t pm = 0, slow = 0;
#pragma unroll
      for (int i = 0; i < 16; i++)
        slow |= (uint32_t)!prequant_fast(in[(16 * ry + i) * 64 + xx], eb_f, ebx2_f, ebx2_r, k[i]) << i;
      if (__any_sync(~0u, slow != 0)) {
#pragma unroll
        for (int i = 0; i < 16; i++) {
          if ((slow >> i) & 1u) {
            bool p;
            err |= prequant(in[(16 * ry + i) * 64 + xx], eb_f, ebx2_f, ebx2_r, k[i], p);
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
    } else {
      // thread t: z column of (xx, yy) = (t & 15, t >> 4); z and x differences in
      // registers and shuffles, the y difference through shared memory
      const uint32_t xx = tid & 15, yy = tid >> 4;
      int32_t k[16];
      uint32_t pm = 0, slow = 0;
#pragma unroll
      for (int i = 0; i < 16; i++)
        slow |= (uint32_t)!prequant_fast(in[(i * 16 + yy) * 16 + xx], eb_f, ebx2_f, ebx2_r, k[i]) << i;
      if (__any_sync(~0u, slow != 0)) {
#pragma unroll
        for (int i = 0; i < 16; i++) {
          if ((slow >> i) & 1u) {
            bool p;
            err |= prequant(in[(i * 16 + yy) * 16 + xx], eb_f, ebx2_f, ebx2_r, k[i], p);
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
      __syncthreads();  // every thread has read the box: it carries k from here
#pragma unroll
      for (int i = 0; i < 16; i++) s_k[(i * 16 + yy) * 16 + xx] = k[i];
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 16; i++) {
        const uint32_t j = (i * 16 + yy) * 16 + xx;
        const int32_t below = (yy & 7) ? s_k[(i * 16 + yy - 1) * 16 + xx] : 0;
        post(k[i] - below, j, anyp, (pm >> i) & 1u);
      }
    }
    __syncthreads();
  } else {
    err |= edge_codes<ND>(A, b, S, in, w, m, dglob);
    run_head_words(S.c, m, S.head);
    __syncthreads();
  }

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
    // single-element runs are counted in a register and added once per warp
    uint32_t ones = 0;
#pragma unroll 4
    for (int i = 0; i < kPer; i++) {
      const uint32_t j = tid + kThreads * i;
      if (j < m && ((S.head[j >> 5] >> (j & 31)) & 1u)) {
        const uint32_t v = S.c[j];
        const uint32_t len = next_head(S.head, S.next, j, m) - j;
        atomicAdd(&S.hv[v], 1u);
        if (len == 1)
          ones++;
        else if (len <= (uint32_t)kHlShared)
          atomicAdd(&S.hl[len - 1], 1u);
        else
          atomicAdd(&A.hist_len[len - 1], 1u);
      }
    }
    ones = warp_sum(ones);
    if (lane == 0 && ones) atomicAdd(&S.hl[0], ones);
  }
  // the next block writes S.c, S.patch and S.outl again (after the caller's barrier)
  if (tid == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  if (err) atomicOr(&A.st->status, err);
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

}  // namespace

// Persistent construction over the tiles of `nfields` fields.  The single-field
// entry passes the task by value (`one`, tasks == nullptr, ntiles = its block
// count); batches pass a device table and tile0[f], the first global tile of field
// f (tile0[nfields] = ntiles).
template <int ND>  // 1, 2, 3; 0 = any (batches of mixed dimensionality)
__global__ __launch_bounds__(kThreads, 4) void construct_kernel(const __grid_constant__ ConstructTask one,
                                                             const ConstructTask* __restrict__ tasks,
                                                             const uint32_t* __restrict__ tile0, int nfields,
                                                             uint32_t ntiles, uint32_t* ticket,
                                                             uint32_t spin_limit) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Smem& S = *reinterpret_cast<Smem*>(smem_raw);
  __shared__ uint32_t s_t[2];
  __shared__ int s_f[2];
  __shared__ uint32_t s_fail;
  const int tid = threadIdx.x;
  auto task = [&](int f) -> const ConstructTask* { return tasks ? &tasks[f] : &one; };
  auto base = [&](int f) -> uint32_t { return tasks ? tile0[f] : 0u; };
  // thread 0: ticket t goes to buffer `slot`: its field, its box, and its fetch.
  // Tickets are drawn one tile ahead of the fetches (`pending`), so the counter's
  // round trip overlaps the work on the current tile.
  auto claim = [&](int slot, uint32_t t, int hint) {
    const int f = t < ntiles ? (tasks ? find_field(tile0, nfields, t, hint) : 0) : -1;
    s_t[slot] = t;
    s_f[slot] = f;
    if (f >= 0) {
      uint32_t* bx = S.box[slot];
      block_box(task(f)->a.g, t - base(f), bx, bx + 3);
      if (task(f)->use_tma) issue_tile(task(f), bx, S.in[slot], &S.bar[slot]);
    }
  };
  uint32_t pending = 0;

  if (tid == 0) {
    mbar_init(&S.bar[0]);
    mbar_init(&S.bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
    claim(0, atomicAdd(ticket, 1u), 0);
    pending = atomicAdd(ticket, 1u);
  }
  for (int i = tid; i < kNsymCode + kNsymCode + kHlShared; i += kThreads) S.hc[i] = 0;  // hc, hv, hl
  __syncthreads();

  int cur = 0, field = -1;
  uint32_t phase[2] = {0u, 0u};
  uint32_t n_rec_acc = 0, n_patch_acc = 0;  // thread 0: the current field's counts
  auto flush_field = [&](int f) {
    const ConstructArgs& P = task(f)->a;
    flush_hist(S.hc, kNsymCode, P.hist_code);
    flush_hist(S.hv, kNsymCode, P.hist_val);
    flush_hist(S.hl, kHlShared, P.hist_len);
    if (tid == 0) {
      if (n_rec_acc) atomicAdd(&P.st->n_rec, (unsigned long long)n_rec_acc);
      if (n_patch_acc) atomicAdd(&P.st->n_patch, (unsigned long long)n_patch_acc);
    }
    n_rec_acc = n_patch_acc = 0;
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
        for (int i = tid; i < kNsymCode + kNsymCode + kHlShared; i += kThreads) S.hc[i] = 0;
      }
      field = f;
    }
    const ConstructArgs& A = T->a;
    const uint32_t b = t - base(f);
    if (T->use_tma) {
      // every thread observes the completion itself (acquire of the TMA writes); the
      // phase advances only when the wait succeeded, so that after a timeout the drain
      // below still waits on the phase of the copy that did not complete
      if (mbar_wait(&S.bar[cur], phase[cur], spin_limit)) {
        phase[cur] ^= 1u;
      } else {
        atomicOr(&A.st->status, ERR_TIMEOUT);
        s_fail = 1;
      }
    } else {
      load_tile_threads(A, b, S.in[cur]);
    }
    __syncthreads();
    if (s_fail) break;
    const uint32_t* bx = S.box[cur];
    if (ND == 1 || (ND == 0 && A.g.ndim == 1)) process_tile<1>(A, b, bx, S, S.in[cur], n_rec_acc, n_patch_acc);
    else if (ND == 2 || (ND == 0 && A.g.ndim == 2)) process_tile<2>(A, b, bx, S, S.in[cur], n_rec_acc, n_patch_acc);
    else process_tile<3>(A, b, bx, S, S.in[cur], n_rec_acc, n_patch_acc);
    __syncthreads();
    cur ^= 1;
  }
  if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  if (s_fail) {
    // a fetch did not complete in time: wait once more (bounded) for both buffers'
    // copies so no transfer outlives the CTA, then leave (phase[cur] still names the
    // phase of the copy that timed out; phase[cur ^ 1] that of the one issued after it)
    if (tid == 0) {
      mbar_wait(&S.bar[cur], phase[cur], spin_limit);
      if (s_f[cur ^ 1] >= 0 && task(s_f[cur ^ 1])->use_tma)
        mbar_wait(&S.bar[cur ^ 1], phase[cur ^ 1], spin_limit);
    }
    return;
  }
  if (field >= 0) flush_field(field);
  if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

size_t construct_smem_bytes() { return sizeof(Smem); }

// ---- host side ------------------------------------------------------------------------
namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

int g_sms = 0, g_occ = 0;

}  // namespace

// Fill the tensor map of a task when TMA can describe the field: 16-byte aligned
// base and row pitches that are multiples of 16 bytes.  Otherwise use_tma = 0.
void prepare_construct_task(ConstructTask& T) {
  T.use_tma = 0;
  const Geom& g = T.a.g;
  const uintptr_t base = reinterpret_cast<uintptr_t>(T.a.x);
  if (base & 15) return;
  if (g.ndim >= 2 && (g.n[2] % 4) != 0) return;
  EncodeTiledFn fn = encode_fn();
  if (!fn) return;
  cuuint64_t dim[3], stride[2];
  cuuint32_t box[3], estr[3] = {1, 1, 1};
  const int rank = g.ndim;
  if (rank == 1) {
    dim[0] = g.nelem;
    box[0] = 256;
  } else if (rank == 2) {
    dim[0] = g.n[2];
    dim[1] = g.n[1];
    stride[0] = (cuuint64_t)g.n[2] * 4;
    box[0] = 64;
    box[1] = 64;
  } else {
    dim[0] = g.n[2];
    dim[1] = g.n[1];
    dim[2] = g.n[0];
    stride[0] = (cuuint64_t)g.n[2] * 4;
    stride[1] = (cuuint64_t)g.n[2] * g.n[1] * 4;
    box[0] = box[1] = box[2] = 16;
  }
  if (rank == 1 && g.nelem >= (1ull << 32)) return;
  const CUresult r = fn(&T.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<float*>(T.a.x), dim,
                        stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  T.use_tma = r == CUDA_SUCCESS ? 1 : 0;
}

// Persistent grid size: resident CTAs per SM times SMs, capped by the tile count.
int construct_grid(uint32_t ntiles) {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(construct_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
    cudaFuncSetAttribute(construct_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
    cudaFuncSetAttribute(construct_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
    cudaFuncSetAttribute(construct_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ, construct_kernel<0>, kThreads, sizeof(Smem));
    if (g_sms <= 0) g_sms = 1;
    if (g_occ <= 0) g_occ = 1;
  }
  const uint64_t cap = (uint64_t)g_sms * g_occ;
  return (int)(ntiles < cap ? (ntiles ? ntiles : 1) : cap);
}

cudaError_t launch_construct(const ConstructTask& one, uint32_t* ticket, cudaStream_t s) {
  const int grid = construct_grid(one.a.g.nblk);
  trace_begin(K_CONSTRUCT, s);
  const int nd = one.a.g.ndim;
  auto k = nd == 1 ? construct_kernel<1> : (nd == 2 ? construct_kernel<2> : construct_kernel<3>);
  k<<<grid, kThreads, sizeof(Smem), s>>>(one, nullptr, nullptr, 1, one.a.g.nblk, ticket, one.a.spin_limit);
  trace_end(K_CONSTRUCT, s);
  return cudaGetLastError();
}

cudaError_t launch_construct_batch(const ConstructTask* d_tasks, const uint32_t* d_tile0, int nfields,
                                   uint32_t ntiles, uint32_t* ticket, uint32_t spin_limit, int grid, int nd,
                                   cudaStream_t s) {
  ConstructTask dummy;
  memset(&dummy, 0, sizeof(dummy));
  if (grid <= 0) grid = construct_grid(ntiles);
  // the specialised kernel when every field has the same dimensionality
  auto k = nd == 1 ? construct_kernel<1>
                   : (nd == 2 ? construct_kernel<2> : (nd == 3 ? construct_kernel<3> : construct_kernel<0>));
  trace_begin(K_CONSTRUCT, s);
  k<<<grid, kThreads, sizeof(Smem), s>>>(dummy, d_tasks, d_tile0, nfields, ntiles, ticket, spin_limit);
  trace_end(K_CONSTRUCT, s);
  return cudaGetLastError();
}

}  // namespace cszp
