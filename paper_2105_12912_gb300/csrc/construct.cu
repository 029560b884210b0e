// Lorenzo construction kernels (Sec. IV-A, Alg. 1 compression part) and their
// host-side set-up: tensor maps, persistent grids and launches.  The device code
// is in construct_body.cuh.
#include "construct_body.cuh"

namespace cszp {

using namespace cons;

template <int ND, typename E, bool G = false>
__global__ __launch_bounds__(kThreads, 4) void construct_kernel(const __grid_constant__ ConstructTask one,
                                                             const ConstructTask* __restrict__ tasks,
                                                             const uint32_t* __restrict__ tile0, int nfields,
                                                             uint32_t ntiles, uint32_t* ticket,
                                                             uint32_t spin_limit) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  construct_loop<ND, E, G, false>(one, tasks, tile0, nfields, ntiles, ticket, spin_limit, smem_raw);
}


size_t construct_smem_bytes() { return sizeof(SmemT<float>); }

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

int g_sms = 0;

}  // namespace

// Fill the tensor map of a task when TMA can describe the field: 16-byte aligned
// base and row pitches that are multiples of 16 bytes.  Otherwise use_tma = 0.
void prepare_construct_task(ConstructTask& T) {
  T.use_tma = 0;
  const Geom& g = T.a.g;
  const bool f64 = T.a.x64 != nullptr;
  const uint32_t esz = f64 ? 8u : 4u;
  void* xp = f64 ? const_cast<double*>(T.a.x64) : static_cast<void*>(const_cast<float*>(T.a.x));
  const uintptr_t base = reinterpret_cast<uintptr_t>(xp);
  if (base & 15) return;
  if (g.ndim >= 2 && ((uint64_t)g.n[2] * esz) % 16 != 0) return;
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
    stride[0] = (cuuint64_t)g.n[2] * esz;
    box[0] = T.a.global ? Halo<2>::X : 64;
    box[1] = T.a.global ? Halo<2>::Y : 64;
  } else {
    dim[0] = g.n[2];
    dim[1] = g.n[1];
    dim[2] = g.n[0];
    stride[0] = (cuuint64_t)g.n[2] * esz;
    stride[1] = (cuuint64_t)g.n[2] * g.n[1] * esz;
    box[0] = T.a.global ? Halo<3>::X : 16;
    box[1] = T.a.global ? Halo<3>::Y : 16;
    box[2] = T.a.global ? Halo<3>::Z : 16;
  }
  if (rank == 1 && g.nelem >= (1ull << 32)) return;
  const CUresult r = fn(&T.tmap, f64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        (cuuint32_t)rank, xp, dim, stride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        rank == 3 && !f64 && !T.a.global ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  T.use_tma = r == CUDA_SUCCESS ? 1 : 0;
}

// Persistent grid size: resident CTAs per SM (of the kernel that runs, with its
// shared memory) times SMs, capped by the tile count.
template <int ND, typename E, bool G>
int grid_of(uint32_t ntiles) {
  using SM = SmemT<E, G ? kHaloMax : kSlots>;
  static int occ = 0;
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 1;
  }
  if (occ == 0) {
    cudaFuncSetAttribute(construct_kernel<ND, E, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SM));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, construct_kernel<ND, E, G>, kThreads, sizeof(SM));
    if (occ <= 0) occ = 1;
  }
  const uint64_t cap = (uint64_t)g_sms * occ;
  return (int)(ntiles < cap ? (ntiles ? ntiles : 1) : cap);
}

int construct_grid(uint32_t ntiles) { return grid_of<0, float, false>(ntiles); }

template <int ND, typename E, bool G>
void launch_one(const ConstructTask& one, uint32_t* ticket, cudaStream_t s) {
  using SM = SmemT<E, G ? kHaloMax : kSlots>;
  const int grid = grid_of<ND, E, G>(one.a.g.nblk);
  construct_kernel<ND, E, G><<<grid, kThreads, sizeof(SM), s>>>(one, nullptr, nullptr, 1, one.a.g.nblk, ticket,
                                                                one.a.spin_limit);
}

template <typename E, bool G>
void launch_nd(const ConstructTask& one, uint32_t* ticket, cudaStream_t s) {
  const int nd = one.a.g.ndim;
  if (nd == 1) launch_one<1, E, G>(one, ticket, s);
  else if (nd == 2) launch_one<2, E, G>(one, ticket, s);
  else launch_one<3, E, G>(one, ticket, s);
}

cudaError_t launch_construct(const ConstructTask& one, uint32_t* ticket, cudaStream_t s) {
  const bool f64 = one.a.x64 != nullptr, global = one.a.global != 0;
  trace_begin(K_CONSTRUCT, s);
  if (f64) {
    if (global) launch_nd<double, true>(one, ticket, s);
    else launch_nd<double, false>(one, ticket, s);
  } else {
    if (global) launch_nd<float, true>(one, ticket, s);
    else launch_nd<float, false>(one, ticket, s);
  }
  trace_end(K_CONSTRUCT, s);
  return cudaGetLastError();
}

cudaError_t launch_construct_batch(const ConstructTask* d_tasks, const uint32_t* d_tile0, int nfields,
                                   uint32_t ntiles, uint32_t* ticket, uint32_t spin_limit, int grid, int nd,
                                   cudaStream_t s) {
  ConstructTask dummy;
  memset(&dummy, 0, sizeof(dummy));
  // the specialised kernel when every field has the same dimensionality (grid_of also
  // sets the kernel's shared-memory limit); an explicit grid comes from the autotuner
  const int full = nd == 1 ? grid_of<1, float, false>(ntiles)
                           : (nd == 2 ? grid_of<2, float, false>(ntiles)
                                      : (nd == 3 ? grid_of<3, float, false>(ntiles) : grid_of<0, float, false>(ntiles)));
  if (grid <= 0) grid = full;
  auto k = nd == 1 ? construct_kernel<1, float>
                   : (nd == 2 ? construct_kernel<2, float> : (nd == 3 ? construct_kernel<3, float> : construct_kernel<0, float>));
  trace_begin(K_CONSTRUCT, s);
  k<<<grid, kThreads, sizeof(SmemT<float>), s>>>(dummy, d_tasks, d_tile0, nfields, ntiles, ticket, spin_limit);
  trace_end(K_CONSTRUCT, s);
  return cudaGetLastError();
}

}  // namespace cszp
