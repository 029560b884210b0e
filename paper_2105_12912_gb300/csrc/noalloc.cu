// Decompression without a caller-provided workspace, for callers that cannot
// allocate device memory (see csz_decompress_static in cszp.h).  The scratch lives
// in one file-scope device array; this file only adds the entry point and leaves
// csz_decompress untouched.
#include <mutex>

#include "cszp.h"
#include "host.h"
#include "kernels.h"

namespace {

// Scratch for any archive of at most kStaticMaxBlocks codec blocks: the workspace of
// a 64-block shape is about 1.16 MiB, and the last 256 bytes hold the call's status
// word.  Every GPU that loads the library holds this array until the process exits.
constexpr size_t kStaticScratchBytes = 1280 * 1024;
constexpr size_t kStatusBytes = 256;
constexpr size_t kStaticWorkspaceBytes = kStaticScratchBytes - kStatusBytes;
constexpr uint64_t kStaticMaxBlocks = 64;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device, looked up once (host code must not
// use the symbol itself as a pointer: on the host it names a stand-in, not device
// memory).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" csz_status csz_decompress_static(const uint8_t* d_archive, size_t bytes, float* d_out,
                                            uint64_t out_cap_elems, void* stream) {
  if (!d_archive || !d_out) return CSZ_E_ARG;
  if (bytes < 128) return CSZ_E_CORRUPT;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CSZ_E_CUDA;
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return CSZ_E_CUDA;
      g_scratch_addr[dev] = p;
    }
    scratch = static_cast<unsigned char*>(g_scratch_addr[dev]);
  }
  // the size limit needs the shape, which is in the header; the same host copy then
  // drives the decompression (which checks it against the archive on the device)
  uint8_t h[128];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(h, d_archive, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CSZ_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
  int ndim = 0;
  uint64_t dims[3] = {0, 0, 0};
  csz_status r = csz_archive_info(h, sizeof(h), &ndim, dims, nullptr, nullptr);
  if (r != CSZ_OK) return r;
  cszp::Geom g;
  if (!cszp::make_geom(ndim, dims, g)) return CSZ_E_CORRUPT;
  if (g.nblk > kStaticMaxBlocks) return CSZ_E_CAPACITY;
  // the decompression clears the device status at the start of every call; the rest
  // of the scratch is fully rewritten before it is read
  uint32_t* d_status = reinterpret_cast<uint32_t*>(scratch + kStaticWorkspaceBytes);
  r = csz_decompress_async(d_archive, bytes, h, d_out, out_cap_elems, scratch, kStaticWorkspaceBytes, d_status,
                           stream);
  if (r != CSZ_OK) return r;
  uint32_t hs = 0;
  if (cudaMemcpyAsync(&hs, d_status, sizeof(hs), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CSZ_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CSZ_E_CUDA;
  return static_cast<csz_status>(hs);
}
