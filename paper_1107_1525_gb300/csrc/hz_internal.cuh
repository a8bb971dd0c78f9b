// hz_internal.cuh -- device-side layout, helpers and launcher declarations
// shared by libhz's translation units.  Nothing here is exported.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hz.h"

namespace hz {

// ----------------------------------------------------------------- limits
constexpr uint32_t kHeaderBytes = 280;
constexpr uint32_t kMaxBlock = 1u << 24;
constexpr int kMaxLen = 64;
constexpr uint32_t kFlagIndex = 1;
// Bounded spin waits: a wait that runs out records HZ_ERR_TIMEOUT and the
// kernel gives up the work item instead of hanging the GPU.
constexpr uint32_t kSpinLimit = 1u << 20;

// Encode tiles: NT threads x SPT symbols per thread.
constexpr int kEncThreads = 256;
constexpr int kEncSymPerThread = 32;
constexpr int kEncTile = kEncThreads * kEncSymPerThread;  // 8192 symbols
constexpr int kEncStageWords = 4096 + 64;                 // staging window

// Decode-table width bounds.
constexpr int kLutMinBits = 8;
constexpr int kLutMaxBits = 12;

// ------------------------------------------------------------ device state
// Status word values are -hz_status (so 0 = OK).
struct CodeTable {
  uint8_t len[256];
  uint32_t maxlen;
  uint32_t nsym;            // symbols with nonzero length
  uint64_t code[256];
};

// Encode decoupled look-back record for one tile (32 bytes).  `flag` holds
// (epoch << 2) | state; state 1 = aggregate ready, 2 = inclusive prefix ready.
struct TileStatus {
  uint32_t flag;
  uint32_t has_head;        // bit 31: the tile holds a block start; low 31: head bits
  uint32_t omega;           // words of complete blocks inside the tile
  uint32_t tail;            // bits of the open block at the tile's end
  uint64_t pre_O;           // inclusive prefix: header word of the open block
  uint32_t pre_b;           // inclusive prefix: bits in the open block
  uint32_t pad;
};

struct DevState {
  uint32_t error;           // first error recorded (as -hz_status), 0 = none
  uint32_t error_where;     // kernel-specific detail for debugging
  uint32_t tile_counter;    // dynamic tile ticket of the encode kernel
  uint32_t block_counter;   // dynamic block ticket of the decode kernel
  uint32_t hist[256];
  CodeTable codes;
};

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ void set_error(DevState* st, hz_status s, uint32_t where) {
  if (atomicCAS(&st->error, 0u, (uint32_t)(-s)) == 0u) atomicExch(&st->error_where, where);
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ceil32(uint64_t bits) { return (uint32_t)((bits + 31) >> 5); }

// ------------------------------------------------------------ launchers
// Kernel ids for the profile log.
enum KernelId : int32_t {
  K_HIST = 0,
  K_BUILD = 1,
  K_ENCODE = 2,
  K_DECODE_SETUP = 3,
  K_DECODE = 4,
  K_INDEX_CHASE = 5,
  K_BATCH = 6,
  K_COUNT
};

struct EncodeArgs {
  const uint8_t* in;
  uint64_t n;
  uint32_t B;
  uint32_t nb;
  uint32_t flags;
  uint8_t* out;             // stream base
  uint64_t out_cap;
  uint64_t* out_len;
  DevState* st;
  TileStatus* tiles;
  uint32_t ntiles;
  uint32_t epoch;
};

struct DecodeArgs {
  const uint8_t* in;        // stream base
  uint64_t in_len;
  uint8_t* out;
  uint64_t out_cap;
  uint64_t* out_len;
  DevState* st;
  uint32_t* chase_index;    // scratch index for streams without one (nb words)
  uint32_t chase_cap;       // capacity of chase_index in entries
  int lut_bits;
};

// Each returns the cudaError_t of its launch.
cudaError_t launch_histogram(const uint8_t* in, uint64_t n, DevState* st, int num_sms,
                             cudaStream_t s);
// Code lengths handed to the build kernel by value (no host staging needed).
struct LenParam {
  uint8_t len[256];
};
cudaError_t launch_build_codes(DevState* st, int from_hist, const LenParam& given, uint64_t n,
                               uint32_t B, uint32_t nb, uint32_t flags, uint8_t* out,
                               uint64_t out_cap, uint64_t* out_len, cudaStream_t s);
cudaError_t launch_encode(const EncodeArgs& a, int num_sms, cudaStream_t s);
struct DecTables;
size_t dec_tables_bytes();
cudaError_t launch_decode_setup(const DecodeArgs& a, DecTables* T, cudaStream_t s);
cudaError_t launch_decode_blocks(const DecodeArgs& a, const DecTables* T, int threads, int num_sms,
                                 cudaStream_t s);

}  // namespace hz
