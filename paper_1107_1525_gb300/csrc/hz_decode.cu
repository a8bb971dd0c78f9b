// hz_decode.cu -- block decoder (Sec. 2.1, last paragraph, and Sec. 3.2 of
// Cloud et al.): blocks are located through a table of offsets built from the
// length delimiters and decoded independently.
//
// decode_setup_kernel (one CTA) parses and checks the container header and
// builds the canonical decode tables: per-length first code and count, the
// symbols in (length, byte) order, and a lookup table indexed by the next W
// (or 10) payload bits, in one of two layouts (hz_decode_dev.cuh).  For
// streams without a stored index it rebuilds the offset table by walking the
// delimiters (the paper's own scheme), or leaves that to the chase kernel.
//
// The paper gives each block to one thread; a 64 KiB block is then a chain of
// 65 536 dependent table lookups, far too long for a GPU.  Here a block's
// payload is cut into equal bit ranges, one per thread, and every thread
// starts decoding at the start of its range as if a code began there.
// Huffman codes resynchronise after a few symbols (the observation of Klein
// and Wiseman that the paper cites in Sec. 2.1), so a decode that started at a
// wrong bit soon lands on the true code boundaries.  A fix-up loop re-decodes
// each range from the true boundary handed over by its left neighbour only
// until the two decodes meet, which corrects the range's symbol count; a scan
// of the counts gives every range its output position; a second pass decodes
// and stores the symbols.  Nothing about the stream format changes.
//
// Streams that carry sub-block offsets (flags bit 1) need none of this: the
// offsets give the code boundary of every S-th symbol, so each lane decodes
// one sub-block of S symbols from its stored start straight into the output
// (decode_units_warp*), in a single pass.
//
// decode_fast_kernel does this with one warp per block of at most 64 KiB:
// lane i takes the i-th of 32 equal word ranges of the payload (about 2000
// symbols each, so the resynchronisation costs next to nothing), the fix-up
// and the scan are warp shuffles, every lane reads its range through a
// cp.async ring in shared memory and writes its contiguous run of decoded
// bytes with 16-byte stores.  Larger blocks are decoded by the same launch,
// one CTA per block.
#include "hz_decode_dev.cuh"

namespace hz {

size_t dec_tables_bytes() { return sizeof(DecTables); }

__global__ void __launch_bounds__(256) decode_setup_kernel(DecodeArgs a, DecTables* T) {
  decode_setup_device(a, T);
}

// Blocks longer than kFastMaxB: one CTA of NT threads per block
// (decode_block_generic), its shared state laid over the fast decoder's, so
// that no second launch is needed.
template <int NT>
struct GenAll {
  GenShared sh;
  GenBlockShared<NT> bs;
};

template <int NT>
__device__ __noinline__ void decode_generic_blocks(const DecodeArgs& a, const DecTables* T) {
  GenAll<NT>& g = *reinterpret_cast<GenAll<NT>*>(g_fast_smem);
  const int W = (int)T->lut_bits;
  for (int i = threadIdx.x; i < (1 << W); i += NT) g.sh.lut[i] = T->lut[i];
  load_canon(g.sh.c, T, threadIdx.x, NT);
  __syncthreads();
  const uint32_t k_end = a.k_end < g.sh.c.nb ? a.k_end : g.sh.c.nb;
  for (uint32_t k = a.k_begin + blockIdx.x; k < k_end; k += gridDim.x)
    decode_block_generic<NT>(a, g.sh, g.bs, k);
}

// Streams with sub-block offsets (flags bit 1): a lane per sub-block, in one
// pass, inside decode_fast_kernel (one launch per decompression whatever the
// layout).  The common table mode (mode 0 with the replicated 10-bit table)
// runs inlined, with the registers of the kernel itself; the other modes
// call their separate functions.
//
// A warp takes 32 sub-blocks at a time: first the group of its own index in
// the launch, then, each time it has finished one, the group a ticket
// counter in the device state hands it.  The groups left after the first
// round go to the warps that finish first, wherever they run, where a fixed
// assignment gives them to the launch's first warps (and so to a few SMs).
// A ticket taken when a group starts instead, to hide the atomic's latency,
// assigns them as the fixed order does: on the 2^28-byte field (about one
// group per warp) that was 15 % slower.  The launch's last CTA to finish
// puts the counter back to zero for the next launch on the stream.
template <class Body>
static __device__ __forceinline__ void sub_groups(const DecodeArgs& a, uint32_t u_begin,
                                                  uint32_t u_end, Body body) {
  const uint32_t warps = blockDim.x / 32;
  const uint32_t P = gridDim.x * warps;
  const uint32_t groups = (u_end - u_begin + 31) / 32;
  uint32_t g = blockIdx.x * warps + (threadIdx.x >> 5);
  while (g < groups) {  // uniform per warp
    body(u_begin + 32 * g);
    uint32_t t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(&a.st->dec_ticket, 1u);
    g = P + __shfl_sync(0xFFFFFFFFu, t, 0);
  }
}

static __device__ __forceinline__ void decode_sub_blocks(const DecodeArgs& a, const DecTables* T) {
  const uint32_t warps = blockDim.x / 32;
  const uint32_t nb = T->nb;
  const uint32_t k_end = a.k_end < nb ? a.k_end : nb;
  const uint32_t M = T->sub_M;
  const uint32_t u_begin = a.k_begin * M, u_end = k_end > a.k_begin ? k_end * M : u_begin;
  if (u_begin + 32 * blockIdx.x * warps < u_end) {  // uniform: this CTA has work
    FastShared& sh = fast_sh();
    load_fast_tables<true>(sh, T, threadIdx.x, blockDim.x);
    if (threadIdx.x == 0) sh.args = a;
    __syncthreads();
    const int mode = fast_mode(T, sh.c);
    if (mode == 0 && sh.pair) {
      sub_groups(a, u_begin, u_end, [&](uint32_t u0) { decode_units0_pair_body(u0, u_end); });
    } else if (mode == 0 && sh.fill_k == 3) {
      sub_groups(a, u_begin, u_end, [&](uint32_t u0) { decode_units0_body<3, true>(u0, u_end); });
    } else if (mode == 0 && sh.fill_k == 4) {
      sub_groups(a, u_begin, u_end, [&](uint32_t u0) { decode_units0_body<4, true>(u0, u_end); });
    } else {
      sub_groups(a, u_begin, u_end, [&](uint32_t u0) { decode_units_fast(u0, u_end, mode); });
    }
  }
  // every CTA counts itself done; the last one resets the tickets
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&a.st->dec_done, 1u) == gridDim.x - 1) {
      a.st->dec_ticket = 0;
      a.st->dec_done = 0;
    }
  }
}

// Launched with 128 or 256 threads and decode_smem_bytes(threads) of dynamic
// shared memory.  With at least as many blocks as the launch has warps, warp j
// of CTA i takes block k_begin + i * warps + j (a CTA's warps read adjacent
// records), then every (grid * warps)-th after it; with fewer, it takes
// k_begin + j * grid + i, so that the blocks spread over all CTAs (and so over
// all SMs) instead of filling a few CTAs' warps.
__global__ void __launch_bounds__(kFastThreads, 3) decode_fast_kernel(DecodeArgs a,
                                                                  const DecTables* T) {
  if (!T->ok) return;
  const uint32_t warps = blockDim.x / 32;
  const uint32_t warp = threadIdx.x >> 5;
  const uint32_t nb = T->nb;
  const uint32_t k_end = a.k_end < nb ? a.k_end : nb;
  if (T->sub_M) {  // uniform: sub-block offsets, a lane per sub-block
    decode_sub_blocks(a, T);
    return;
  }
  if (!fast_block_size(T->B)) {  // uniform: every CTA takes whole blocks
    if (blockDim.x == 128) decode_generic_blocks<128>(a, T);
    else decode_generic_blocks<kFastThreads>(a, T);
    return;
  }
  if (a.k_begin + blockIdx.x >= k_end) return;  // uniform: no block for any warp here
  const bool spread = k_end - a.k_begin < gridDim.x * warps;
  const uint32_t k0 = a.k_begin + (spread ? warp * gridDim.x + blockIdx.x : blockIdx.x * warps + warp);
  FastShared& sh = fast_sh();
  load_fast_tables<true>(sh, T, threadIdx.x, blockDim.x);
  __syncthreads();
  const int mode = fast_mode(T, sh.c);
  const uint32_t stride = gridDim.x * warps;
  for (uint32_t k = k0; k < k_end; k += stride) decode_block_fast(a, k, mode);
}

size_t decode_smem_bytes(int threads) {
  const size_t fast = fast_smem_bytes(threads);
  const size_t gen = threads == 128 ? sizeof(GenAll<128>) : sizeof(GenAll<kFastThreads>);
  return fast > gen ? fast : gen;
}

// ================================================================ launchers
static PerDeviceSetup<2> g_decode_setup;

cudaError_t launch_decode_setup(const DecodeArgs& a, DecTables* T, cudaStream_t s) {
  decode_setup_kernel<<<1, 256, 0, s>>>(a, T);
  return cudaGetLastError();
}

cudaError_t launch_decode_blocks(const DecodeArgs& a, const DecTables* T, int threads, int num_sms,
                                 cudaStream_t s) {
  if (threads != 128) threads = kFastThreads;
  const size_t smem = decode_smem_bytes(threads);
  // the raised shared-memory limit and the CTAs resident per SM hold for the
  // device that is current when they are set or queried: kept per device
  int per_sm = 1;
  const cudaError_t e = launch_setup_per_device(
      g_decode_setup, threads == 128 ? 0 : 1, &per_sm, [&](int& out) {
        cudaError_t r = cudaFuncSetAttribute(decode_fast_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)decode_smem_bytes(kFastThreads));
        if (r == cudaSuccess)
          r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out, decode_fast_kernel, threads, smem);
        return r;
      });
  if (e != cudaSuccess) return e;
  uint64_t grid = (uint64_t)num_sms * per_sm;
  // a block range shorter than the resident warps needs fewer CTAs (the
  // block count itself is only known on the device: an unbounded range keeps
  // the full grid)
  if (a.k_end != 0xFFFFFFFFu) {
    const uint64_t need = ((uint64_t)(a.k_end - a.k_begin) + threads / 32 - 1) / (threads / 32);
    if (need < grid) grid = need ? need : 1;
  }
  decode_fast_kernel<<<(unsigned)grid, threads, smem, s>>>(a, T);
  return cudaGetLastError();
}

}  // namespace hz
