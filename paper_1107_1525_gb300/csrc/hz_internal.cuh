// hz_internal.cuh -- device-side layout, helpers and launcher declarations
// shared by libhz's translation units.  Nothing here is exported.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "hz.h"

namespace hz {

// ----------------------------------------------------------------- limits
constexpr uint32_t kHeaderBytes = 280;
constexpr uint32_t kMaxBlock = 1u << 24;
constexpr int kMaxLen = 64;
constexpr uint32_t kFlagIndex = 1;
// Sub-block offsets (flags bit 1, only with bit 0): after the index, u32 S and
// then, per block, the payload bit offsets of its symbols S, 2S, ..., B - S.
// S is a multiple of 32 dividing B.
constexpr uint32_t kFlagSub = 2;
// Bounded spin waits: a wait that runs out records HZ_ERR_TIMEOUT and the
// kernel gives up the work item instead of hanging the GPU.
constexpr uint32_t kSpinLimit = 1u << 20;

// Encode tiles: NT threads x SPT symbols per thread.
constexpr int kEncThreads = 256;
constexpr int kEncSymPerThread = 32;
constexpr int kEncTile = kEncThreads * kEncSymPerThread;  // 8192 symbols
constexpr int kEncStageWords = kEncTile + 64;             // staging window (words)

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

// Per-tile record of the encoder: the tile's summary (written by the
// length-sum pass) and its exclusive scan state (written by the scan).
struct TileStatus {
  uint32_t has_head;        // bit 31: the tile holds a record start; low 31: head bits
  uint32_t omega;           // words of records that start and end inside the tile
  uint32_t tail;            // bits of the tile's last record
  uint32_t pad0;
  uint64_t pre_O;           // exclusive state: word index of the open record's delimiter
  uint32_t pre_b;           // exclusive state: payload bits already in that record
  uint32_t pad1;
};

// What the length-summing pass records about a tile when every tile lies
// inside one record and no code is longer than 32 bits (the warp-parallel
// path): each thread's payload bits (its 32 symbols), each warp's bits, and
// the last 32 code bits of the odd warps' runs (the bits the next packing
// item's first word continues).  The tile scan sums the warps' bits.
struct TileMeta {
  uint16_t lane_bits[kEncThreads];
  uint32_t warp_bits[kEncThreads / 32];
  uint32_t warp_tail[kEncThreads / 32];
};

// The warp-parallel path's condition, the same in every encoder kernel.
__host__ __device__ __forceinline__ bool warp_path(const TileMeta* meta, uint32_t B,
                                                   uint32_t maxlen) {
  return meta != nullptr && B % (uint32_t)kEncTile == 0 && maxlen <= 32;
}

// The encoder's tile scan runs in CTAs of kScanCtaTiles tiles (one a
// thread); n < 2^32 bounds their number.  The batched scan (one CTA a buffer)
// walks a buffer's tiles in chunks of kScanTilesPerCta.
constexpr int kScanCtaTiles = 1024;
constexpr int kScanTilesPerCta = 4096;
constexpr int kMaxScanCtas = (int)((1ull << 32) / kEncTile / kScanCtaTiles);  // 512

struct DevState {
  uint32_t error;           // first error recorded (as -hz_status), 0 = none
  uint32_t error_where;     // kernel-specific detail for debugging
  // the sub-block decoder's work tickets (groups of 32 sub-blocks handed out
  // after each warp's first) and its count of finished CTAs: zero between
  // launches, the launch's last CTA puts both back to zero
  uint32_t dec_ticket, dec_done;
  // ---- cleared before every compress (one memset from here to `codes`)
  uint32_t tile_counter;    // ticket of the scan CTAs
  uint32_t enc_ok;          // set by the encoder's scan: 1 when the stream fits the output
  uint32_t hist[256];
  // 1 = aggregate published, 2 = inclusive prefix (one spare entry: with the
  // scan-stall injection the tickets run from 1 to the CTA count)
  uint32_t scan_flags[kMaxScanCtas + 1];
  // ---- not cleared
  CodeTable codes;
  TileStatus scan_aux[kMaxScanCtas + 1];  // per scan CTA: aggregate and inclusive prefix
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

// Stream layout: bytes before the first record (header, index, sub-block
// section), and where the sub-block entries start.
__host__ __device__ __forceinline__ uint64_t records_at(uint64_t nb, uint32_t B, uint32_t flags,
                                                        uint32_t S) {
  uint64_t at = kHeaderBytes;
  if (flags & kFlagIndex) at += 4 * nb;
  if (flags & kFlagSub) at += 4 + 4 * nb * (uint64_t)(B / S - 1);
  return at;
}
__host__ __device__ __forceinline__ uint64_t sub_entries_at(uint64_t nb) {
  return kHeaderBytes + 4 * nb + 4;
}
// A sub-block size S suits blocks of B symbols.
__host__ __device__ __forceinline__ bool sub_size_ok(uint32_t B, uint32_t S) {
  return S >= 32 && S % 32 == 0 && B % S == 0;
}

// ------------------------------------------------------------ launchers
// Kernel ids for the profile log.
enum KernelId : int32_t {
  K_HIST = 0,
  K_BUILD = 1,
  K_ENC_SUMMARY = 2,
  K_ENC_SCAN = 3,
  K_ENC_PACK = 4,
  K_DECODE_SETUP = 5,
  K_DECODE = 6,
  K_DECODE_GENERIC = 7,  // not launched any more (decode_fast_kernel takes large blocks); id kept
  K_BATCH = 8,
  K_DECODE_CHASE = 9,
  K_COUNT
};

// Division of 32-bit values by a divisor fixed per launch, with one
// multiply-high and two shifts (Granlund and Montgomery, "Division by
// Invariant Integers using Multiplication", PLDI 1994, Fig. 4.1).
struct FastDiv {
  uint32_t d, m, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while (l < 32 && (1ull << l) < d) ++l;  // l = ceil(log2 d)
  FastDiv f;
  f.d = d;
  f.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

__device__ __forceinline__ uint32_t fast_div(uint32_t x, const FastDiv& f) {
  const uint32_t t = __umulhi(f.m, x);
  return (t + ((x - t) >> f.s1)) >> f.s2;
}

__device__ __forceinline__ uint32_t fast_mod(uint32_t x, const FastDiv& f) {
  return x - fast_div(x, f) * f.d;
}

// Launch set-up that belongs to a device -- a kernel's raised dynamic
// shared-memory limit and the CTAs of it that fit on one SM hold for the
// device that is current when they are set or queried -- done once per device
// and variant, under a lock, and the CTAs-per-SM figure kept.
constexpr int kMaxDevices = 64;
template <int NV>
struct PerDeviceSetup {
  std::mutex mu;
  int per_sm[kMaxDevices][NV] = {};
};

// f(int& per_sm) sets the device's attributes and queries the occupancy;
// *per_sm receives the cached figure (at least 1) on success.
template <int NV, class F>
cudaError_t launch_setup_per_device(PerDeviceSetup<NV>& p, int variant, int* per_sm, F&& f) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) {  // not cached: set up on every launch
    int v = 0;
    e = f(v);
    *per_sm = v > 0 ? v : 1;
    return e;
  }
  std::lock_guard<std::mutex> lock(p.mu);
  int& v = p.per_sm[dev][variant];
  if (v < 1) {
    int got = 0;
    e = f(got);
    if (e != cudaSuccess) return e;
    v = got > 0 ? got : 1;
  }
  *per_sm = v;
  return cudaSuccess;
}

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
  FastDiv fdB;              // division by B
  uint32_t tile_begin, tile_end;  // tiles the single-buffer packing launch packs
  // sub-block offsets (flags bit 1): S symbols per sub-block, M = B / S per block
  uint32_t sub_S, sub_M;
  FastDiv fdS;              // division by S (S = 1 without bit 1)
  uint32_t spin_limit;      // polls of the scan's look-back before it gives up
  // per-tile metadata for the warp-parallel packing path (null: not used);
  // written by the length-summing pass for tiles inside one record when no
  // code is longer than 32 bits
  TileMeta* meta;
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
  uint32_t k_begin, k_end;  // blocks the fast kernel decodes: [k_begin, min(k_end, nb))
  // streams without an index: 1 = leave the offset table to the chase kernel
  uint32_t defer_chase;
  uint32_t* seen_no_index;  // set to 1 when such a stream is seen (may be null)
};

// Each returns the cudaError_t of its launch.
cudaError_t launch_histogram(const uint8_t* in, uint64_t n, DevState* st, int num_sms,
                             cudaStream_t s);
// Code lengths handed to the build kernel by value (no host staging needed).
struct LenParam {
  uint8_t len[256];
};
cudaError_t launch_build_codes(DevState* st, int from_hist, const LenParam& given, uint64_t n,
                               uint32_t B, uint32_t nb, uint32_t flags, uint32_t sub_S,
                               uint8_t* out, uint64_t out_cap, uint64_t* out_len, cudaStream_t s);
// The encoder's three launches: length-sum pass, scan, packing.
cudaError_t launch_encode_summary(const EncodeArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_encode_scan(const EncodeArgs& a, cudaStream_t s);
cudaError_t launch_encode_pack(const EncodeArgs& a, int num_sms, cudaStream_t s);
struct DecTables;
size_t dec_tables_bytes();
cudaError_t launch_decode_setup(const DecodeArgs& a, DecTables* T, cudaStream_t s);
cudaError_t launch_decode_blocks(const DecodeArgs& a, const DecTables* T, int threads, int num_sms,
                                 cudaStream_t s);
}  // namespace hz
