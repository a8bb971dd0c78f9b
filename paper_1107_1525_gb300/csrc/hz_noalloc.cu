// hz_noalloc.cu -- hz_compress_noalloc: the compressor for callers that must
// not allocate device memory.  Its scratch (status word, histogram, code
// table and the encoder's per-tile scan records) lives in one file-scope
// __device__ array instead of a context's cudaMalloc'ed buffers.
#include <stddef.h>
#include <string.h>

#include <mutex>

#include "hz_batch.h"
#include "hz_internal.cuh"

using namespace hz;

namespace {

// Largest input the fixed scratch can serve: 256 MiB = 32768 encoder tiles.
constexpr uint64_t kNoallocMaxInput = 256ull << 20;
constexpr uint32_t kNoallocMaxTiles = (uint32_t)(kNoallocMaxInput / kEncTile);
constexpr size_t kStateBytes = (sizeof(DevState) + 255) & ~size_t(255);
constexpr size_t kScratchBytes = kStateBytes + (size_t)kNoallocMaxTiles * sizeof(TileStatus);

// Every GPU that loads the library holds this array (about 1 MiB) until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};  // device address of the array, per device

// Move the status word into the caller's d_status and clear it for the next call.
__global__ void noalloc_finish_kernel(DevState* st, int32_t* d_status) {
  *d_status = -(int32_t)st->error;
  st->error = 0;
  st->error_where = 0;
}

}  // namespace

extern "C" hz_status hz_compress_noalloc(const uint8_t* d_in, uint64_t n, uint32_t block_size,
                                         uint8_t* d_out, uint64_t out_cap, uint64_t* d_out_len,
                                         int32_t* d_status, void* stream) {
  if (!d_out || !d_out_len || !d_status || (n && !d_in)) return HZ_ERR_ARG;
  if (n > kNoallocMaxInput || block_size > kMaxBlock) return HZ_ERR_ARG;
  if (((uintptr_t)d_out & 3) || ((uintptr_t)d_out_len & 7) || ((uintptr_t)d_status & 3))
    return HZ_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HZ_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      // once per device: in host code the array's name is only a stand-in, so
      // fetch its device address and clear it (status, counters, scan records)
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return HZ_ERR_CUDA;
      }
      if (cudaMemset(p, 0, kScratchBytes) != cudaSuccess) {
        cudaGetLastError();
        return HZ_ERR_CUDA;
      }
      g_scratch_ptr[dev] = (unsigned char*)p;
    }
    base = g_scratch_ptr[dev];
  }
  DevState* st = reinterpret_cast<DevState*>(base);
  TileStatus* tiles = reinterpret_cast<TileStatus*>(base + kStateBytes);

  int num_sms = 0;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HZ_ERR_CUDA;
  const uint32_t B = block_size ? block_size : hz_batch_tuned_block_size(n);
  const uint32_t nb = (uint32_t)((n + B - 1) / B);
  const uint32_t ntiles = (uint32_t)((n + kEncTile - 1) / kEncTile);
  // the previous call's status word, counters and histogram are still in the
  // array: clear them (the status word too, in case a launch of the previous
  // call failed before its finish kernel could clear it)
  if (cudaMemsetAsync(st, 0, offsetof(DevState, codes), s) != cudaSuccess)
    return HZ_ERR_CUDA;
  LenParam none;
  memset(&none, 0, sizeof(none));
  if (n > 0 && launch_histogram(d_in, n, st, num_sms, s) != cudaSuccess) return HZ_ERR_CUDA;
  if (launch_build_codes(st, 1, none, n, B, nb, kFlagIndex, 0, d_out, out_cap, d_out_len, s) !=
      cudaSuccess)
    return HZ_ERR_CUDA;
  if (n > 0) {
    EncodeArgs a;
    a.in = d_in;
    a.n = n;
    a.B = B;
    a.nb = nb;
    a.flags = kFlagIndex;
    a.out = d_out;
    a.out_cap = out_cap;
    a.out_len = d_out_len;
    a.st = st;
    a.tiles = tiles;
    a.ntiles = ntiles;
    a.tile_begin = 0;
    a.tile_end = ntiles;
    a.fdB = make_fastdiv(B);
    a.sub_S = 0;
    a.sub_M = 1;
    a.fdS = make_fastdiv(1);
    a.spin_limit = kSpinLimit;
    a.meta = nullptr;  // (no room for it in the fixed scratch)
    if (launch_encode_summary(a, num_sms, s) != cudaSuccess ||
        launch_encode_scan(a, s) != cudaSuccess || launch_encode_pack(a, num_sms, s) != cudaSuccess)
      return HZ_ERR_CUDA;
  }
  noalloc_finish_kernel<<<1, 1, 0, s>>>(st, d_status);
  return cudaGetLastError() == cudaSuccess ? HZ_OK : HZ_ERR_CUDA;
}
