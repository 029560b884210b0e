// Host-side helpers shared by the single-field and batch entry points: codec-block
// geometry, workspace layout, status folding.
#pragma once

#include <cstring>

#include "cszp.h"
#include "kernels.h"

namespace cszp {

constexpr uint64_t kMaxBlocks = (1ull << 31) / kSlots;  // slots*2 must fit in 32 bits

inline uint64_t a8(uint64_t v) { return (v + 7) & ~7ull; }
inline uint64_t a256(uint64_t v) { return (v + 255) & ~255ull; }

// Codec blocks: 1-D 4096, 2-D 64x64, 3-D 16^3 (x fastest).
inline bool make_geom(int ndim, const uint64_t* dims, Geom& g) {
  static const uint32_t B[4][3] = {{0, 0, 0}, {1, 1, 4096}, {1, 64, 64}, {16, 16, 16}};
  if (ndim < 1 || ndim > 3 || !dims) return false;
  memset(&g, 0, sizeof(g));
  g.ndim = ndim;
  uint64_t n[3] = {1, 1, 1};
  for (int i = 0; i < ndim; i++) {
    if (dims[i] == 0 || dims[i] >= (1ull << 31)) return false;
    n[3 - ndim + i] = dims[i];
  }
  uint64_t nblk = 1, nelem = 1;
  for (int d = 0; d < 3; d++) {
    g.n[d] = (uint32_t)n[d];
    g.blk[d] = B[ndim][d];
    g.g[d] = (uint32_t)((n[d] + B[ndim][d] - 1) / B[ndim][d]);
    nblk *= g.g[d];
    nelem *= n[d];
  }
  if (nblk >= kMaxBlocks) return false;
  g.nblk = (uint32_t)nblk;
  g.nelem = nelem;
  return true;
}

// Workspace: [DevState | set-up look-back states | histograms | look-back states]
// (zeroed per compression; decompression zeroes the first two),
// books, decode tables and offsets, block-major code stream, decoded run lengths,
// the lists of run blocks and of blocks reconstructed apart from their decoding
// (the part decompression needs ends at dec_total), then compression-only scratch:
// per-block record counts, patch / outlier bit masks, outlier residuals and record
// offsets.
struct Layout {
  uint64_t st, prep_lb, hist_code, hist_val, hist_len, lb_e, zero_end;
  uint64_t lens, bcodes, blk_off, rec_start, tabs, codes, runl, runblk, slowblk, dec_total;
  uint64_t counts, masks, deltas, rec_off, runs, total;
};

inline Layout layout(const Geom& g) {
  Layout L;
  uint64_t o = 0;
  L.st = o;
  o += a256(sizeof(DevState));
  L.prep_lb = o;  // decompression set-up: two look-back states per 1024 blocks
  o += a256(16ull * ((g.nblk + 1023) / 1024));
  L.hist_code = o;
  o += kNsymCode * 4;
  L.hist_val = o;
  o += kNsymCode * 4;
  L.hist_len = o;
  o += kNsymLen * 4;
  L.lb_e = o;
  o += 8ull * g.nblk;
  L.zero_end = o;
  o = a256(o);
  L.lens = o;
  o += a256(2 * kNsymCode + kNsymLen);
  L.bcodes = o;
  o += 8ull * (2 * kNsymCode + kNsymLen);
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
  L.runblk = o;
  o += a256(4ull * g.nblk);
  L.slowblk = o;
  o += a256(4ull * g.nblk);
  L.dec_total = o;
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

template <typename T>
inline T* at(void* base, uint64_t off) {
  return reinterpret_cast<T*>(static_cast<unsigned char*>(base) + off);
}

__host__ __device__ inline csz_status fold(uint32_t bits) {
  if (bits & ERR_NONFINITE) return CSZ_E_NONFINITE;
  if (bits & ERR_ARG) return CSZ_E_ARG;
  if (bits & ERR_RANGE) return CSZ_E_RANGE;
  if (bits & ERR_CORRUPT) return CSZ_E_CORRUPT;
  if (bits & ERR_CAPACITY) return CSZ_E_CAPACITY;
  if (bits & ERR_TIMEOUT) return CSZ_E_TIMEOUT;
  return CSZ_OK;
}

}  // namespace cszp
