// hz_api.cu -- the exported C ABI of libhz (declared in include/hz.h): the
// context, argument checks, kernel launch sequences, device status, profiling
// and the host-buffer round trips.
#include <stdlib.h>
#include <string.h>

#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include "hz_batch.h"
#include "hz_chase.h"
#include "hz_internal.cuh"

using namespace hz;

struct ProfRec {
  int32_t id;
  cudaEvent_t a, b;
};

// Host-buffer decompression of large streams with an index runs as a
// pipeline of this many block groups (copy in, decode, copy out overlap).
constexpr int kPipeGroups = 12;
constexpr uint64_t kPipeMinBytes = 32ull << 20;
// Streams without an index at least this long get the parallel chase.
constexpr uint64_t kChaseParallelMin = 8ull << 20;

struct hz_ctx {
  int device = 0;
  int num_sms = 0;
  uint64_t mem_budget = 0;
  DevState* d_state = nullptr;
  DecTables* d_dec = nullptr;
  TileStatus* d_tiles = nullptr;
  uint32_t tiles_cap = 0;
  TileMeta* d_meta = nullptr;  // per-tile metadata for the warp-parallel packer (tiles_cap)
  uint32_t* d_chase = nullptr;
  uint32_t chase_cap = 0;
  uint32_t* h_err = nullptr;  // pinned readback of the status words
  hz_codes* h_codes = nullptr;
  // staging for the host-buffer round trips
  uint8_t* d_hin = nullptr;
  uint64_t d_hin_cap = 0;
  uint8_t* d_hout = nullptr;
  uint64_t d_hout_cap = 0;
  uint64_t* d_len = nullptr;
  uint64_t* h_len = nullptr;  // [0]: a stream length; [1..]: the host pipeline's boundaries
  // streams without an index: the setup kernel sets *h_seen (mapped pinned
  // memory) when it meets one; from then on large streams get the parallel
  // chase and its scratch
  uint32_t* h_seen = nullptr;
  uint32_t* d_seen = nullptr;
  uint8_t* d_chase_work = nullptr;
  uint64_t chase_work_cap = 0;
  hz::ChaseScratch cs{};
  // pipelined host-buffer decode: copy-in and copy-out streams, group events
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t e_start = nullptr, e_in[kPipeGroups] = {}, e_dec[kPipeGroups] = {};
  // options
  int opt_index = 1;
  uint32_t opt_sub = 0;  // symbols per sub-block for the sub-block offsets, 0 = none
  uint32_t opt_spin_limit = kSpinLimit;
  bool inject_scan_stall = false;  // one shot: the next scan's tickets start at 1
  int opt_tune_batched = 0;
  int opt_profile = 0;
  int opt_lut_bits = 12;
  int opt_dec_threads = 256;
  int opt_autotune = 1;
  uint32_t tuned_B[4] = {0, 0, 0, 0};  // per size class; 0 = not tuned
  uint64_t launches = 0;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;
  BatchState* batch = nullptr;
};

void hz_tune_load_cache(hz_ctx* c);

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

cudaEvent_t take_event(hz_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Bracket one launch with profile events (when enabled) and count it.
template <class F>
hz_status launch(hz_ctx* c, int32_t id, cudaStream_t s, F&& f) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (c->opt_profile) {
    a = take_event(c);
    b = take_event(c);
    cudaEventRecord(a, s);
  }
  cudaError_t e = f();
  if (c->opt_profile) {
    cudaEventRecord(b, s);
    c->prof.push_back({id, a, b});
  }
  c->launches += 1;
  return e == cudaSuccess ? HZ_OK : HZ_ERR_CUDA;
}

hz_status grow(void** p, uint64_t* cap, uint64_t need) {
  if (need <= *cap) return HZ_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, need) != cudaSuccess) {
    cudaGetLastError();
    return HZ_ERR_NOMEM;
  }
  *cap = need;
  return HZ_OK;
}

int size_class(uint64_t n) {
  return n <= (64u << 10) ? 0 : n <= (1u << 20) ? 1 : n <= (16u << 20) ? 2 : 3;
}

uint32_t autotuned_block(hz_ctx* c, uint64_t n) {
  if (c->opt_autotune && c->tuned_B[size_class(n)]) return c->tuned_B[size_class(n)];
  return hz_batch_tuned_block_size(n);
}

}  // namespace

extern "C" {

hz_status hz_create(hz_ctx** out, int device, uint64_t mem_budget_bytes) {
  if (!out) return HZ_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return HZ_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return HZ_ERR_ARG;
  DeviceGuard g(device);
  hz_ctx* c = new hz_ctx();
  c->device = device;
  c->mem_budget = mem_budget_bytes;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  bool ok = cudaMalloc(&c->d_state, sizeof(DevState)) == cudaSuccess &&
            cudaMalloc(&c->d_dec, dec_tables_bytes()) == cudaSuccess &&
            cudaMalloc(&c->d_len, sizeof(uint64_t)) == cudaSuccess &&
            cudaHostAlloc(&c->h_err, 4 * sizeof(uint32_t), cudaHostAllocDefault) == cudaSuccess &&
            cudaHostAlloc(&c->h_codes, sizeof(hz_codes), cudaHostAllocDefault) == cudaSuccess &&
            cudaHostAlloc(&c->h_len, (kPipeGroups + 1) * sizeof(uint64_t),
                          cudaHostAllocDefault) == cudaSuccess;
  if (ok) ok = cudaMemset(c->d_state, 0, sizeof(DevState)) == cudaSuccess;
  if (ok) {
    // streams without a stored index need a rebuilt offset table
    c->chase_cap = 1u << 20;
    ok = cudaMalloc(&c->d_chase, 4ull * c->chase_cap) == cudaSuccess;
  }
  if (ok) ok = cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    hz_destroy(c);
    return HZ_ERR_NOMEM;
  }
  c->batch = hz_batch_create(c->device, c->num_sms, mem_budget_bytes);
  if (cudaHostAlloc(&c->h_seen, sizeof(uint32_t), cudaHostAllocMapped) == cudaSuccess) {
    *c->h_seen = 0;
    if (cudaHostGetDevicePointer((void**)&c->d_seen, c->h_seen, 0) != cudaSuccess) {
      cudaGetLastError();
      c->d_seen = nullptr;
    }
  } else {
    cudaGetLastError();
    c->h_seen = nullptr;
  }
  cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking);
  cudaStreamCreateWithFlags(&c->s_out, cudaStreamNonBlocking);
  cudaEventCreateWithFlags(&c->e_start, cudaEventDisableTiming);
  for (int g = 0; g < kPipeGroups; ++g) {
    cudaEventCreateWithFlags(&c->e_in[g], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&c->e_dec[g], cudaEventDisableTiming);
  }
  hz_tune_load_cache(c);
  *out = c;
  return HZ_OK;
}

void hz_destroy(hz_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaDeviceSynchronize();
  if (c->batch) hz_batch_destroy(c->batch);
  if (c->s_in) cudaStreamSynchronize(c->s_in);
  if (c->s_out) cudaStreamSynchronize(c->s_out);
  if (c->e_start) cudaEventDestroy(c->e_start);
  for (int g = 0; g < kPipeGroups; ++g) {
    if (c->e_in[g]) cudaEventDestroy(c->e_in[g]);
    if (c->e_dec[g]) cudaEventDestroy(c->e_dec[g]);
  }
  if (c->s_in) cudaStreamDestroy(c->s_in);
  cudaFree(c->d_chase_work);
  if (c->h_seen) cudaFreeHost(c->h_seen);
  if (c->s_out) cudaStreamDestroy(c->s_out);
  for (auto& r : c->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  cudaFree(c->d_state);
  cudaFree(c->d_dec);
  cudaFree(c->d_tiles);
  cudaFree(c->d_meta);
  cudaFree(c->d_chase);
  cudaFree(c->d_hin);
  cudaFree(c->d_hout);
  cudaFree(c->d_len);
  cudaFreeHost(c->h_err);
  cudaFreeHost(c->h_codes);
  cudaFreeHost(c->h_len);
  delete c;
}

uint64_t hz_compress_bound(uint64_t n, uint32_t block_size) {
  if (n > 0xFFFFFFFFull) return 0;
  const uint64_t B = block_size ? block_size : 1;
  const uint64_t nb = (n + B - 1) / B;
  // header + index + per block (delimiter + up to 2 partial words) + at most 8 bits per byte
  return kHeaderBytes + 4 * nb + 12 * nb + 4 * ((n + 3) / 4);
}

constexpr uint32_t kSubAuto = HZ_SUB_BLOCK_AUTO;

// The sub-block size S a compression of n bytes in blocks of B writes (0:
// none).  HZ_OPT_SUB_BLOCK = 1 picks it: the largest of 4096, 2048, 1024 and
// 512 that divides B and leaves at least four sub-blocks for every lane the
// sub-block decoder keeps resident (three CTAs of 256 threads per SM).  A
// lane decodes a sub-block in one chain of dependent steps, so the launch
// takes at least one sub-block's time after the last full round; with four
// or more rounds that tail stays small.  Below that, 512 (the stream grows
// by at most 1 %) while there is at least one sub-block of 512 per lane;
// shorter streams keep the paper's layout, whose decoder splits every block
// over a warp's 32 lanes and so has more parallel work to give them.
static uint32_t resolve_sub(const hz_ctx* c, uint64_t n, uint32_t B) {
  if (!c->opt_index || !c->opt_sub) return 0;
  if (c->opt_sub != kSubAuto) return sub_size_ok(B, c->opt_sub) ? c->opt_sub : 0u;
  const uint64_t lanes = (uint64_t)c->num_sms * 3 * 256;
  for (uint32_t S = 4096; S >= 512; S /= 2)
    if (sub_size_ok(B, S) && n / S >= 4 * lanes) return S;
  return sub_size_ok(B, 512) && n / 512 >= lanes ? 512u : 0u;
}

uint64_t hz_compress_bound_ctx(hz_ctx* c, uint64_t n, uint32_t block_size) {
  if (!c || n > 0xFFFFFFFFull) return 0;
  const uint32_t B = block_size ? block_size : autotuned_block(c, n);
  uint64_t bound = hz_compress_bound(n, B);
  const uint32_t S = resolve_sub(c, n, B);
  if (S) {
    const uint64_t nb = (n + B - 1) / B;
    bound += 4 + 4 * nb * (B / S - 1);
  }
  return bound;
}

hz_status hz_set_option(hz_ctx* c, int key, int64_t v) {
  if (!c) return HZ_ERR_ARG;
  switch (key) {
    case HZ_OPT_INDEX:
      if (v != 0 && v != 1) return HZ_ERR_ARG;
      c->opt_index = (int)v;
      return HZ_OK;
    case HZ_OPT_PROFILE:
      if (v != 0 && v != 1) return HZ_ERR_ARG;
      c->opt_profile = (int)v;
      return HZ_OK;
    case HZ_OPT_SPIN_LIMIT:
      if (v < 1 || v > (1 << 24)) return HZ_ERR_ARG;
      c->opt_spin_limit = (uint32_t)v;
      return HZ_OK;
    case HZ_OPT_INJECT_SCAN_STALL:
      if (v != 0 && v != 1) return HZ_ERR_ARG;
      c->inject_scan_stall = v != 0;
      return HZ_OK;
    case HZ_OPT_TUNE_BATCHED:
      if (v != 0 && v != 1) return HZ_ERR_ARG;
      c->opt_tune_batched = (int)v;
      return HZ_OK;
    case HZ_OPT_SUB_BLOCK:
      if (v != 0 && v != kSubAuto && (v < 32 || v % 32 != 0 || v > (int64_t)kMaxBlock))
        return HZ_ERR_ARG;
      c->opt_sub = (uint32_t)v;
      return HZ_OK;
    case HZ_OPT_DECODE_LUT_BITS:
      if (v < kLutMinBits || v > kLutMaxBits) return HZ_ERR_ARG;
      c->opt_lut_bits = (int)v;
      return HZ_OK;
    case HZ_OPT_DECODE_THREADS:
      if (v != 128 && v != 256) return HZ_ERR_ARG;
      c->opt_dec_threads = (int)v;
      return HZ_OK;
    case HZ_OPT_AUTOTUNE:
      if (v != 0 && v != 1) return HZ_ERR_ARG;
      c->opt_autotune = (int)v;
      return HZ_OK;
    case HZ_OPT_BATCH_PLAIN:
      if (v != 0 && v != 1) return HZ_ERR_ARG;
      hz_batch_set_plain(c->batch, v != 0);
      return HZ_OK;
    case HZ_OPT_BATCH_MAX_REQS:
      if (v < 1 || v > (1 << 20)) return HZ_ERR_ARG;
      return hz_batch_set_max_reqs(c->batch, (uint32_t)v);
    default:
      return HZ_ERR_ARG;
  }
}

int64_t hz_get_option(hz_ctx* c, int key) {
  if (!c) return -1;
  switch (key) {
    case HZ_OPT_INDEX: return c->opt_index;
    case HZ_OPT_PROFILE: return c->opt_profile;
    case HZ_OPT_SUB_BLOCK: return c->opt_sub;
    case HZ_OPT_TUNE_BATCHED: return c->opt_tune_batched;
    case HZ_OPT_SPIN_LIMIT: return c->opt_spin_limit;
    case HZ_OPT_INJECT_SCAN_STALL: return c->inject_scan_stall ? 1 : 0;
    case HZ_OPT_DECODE_LUT_BITS: return c->opt_lut_bits;
    case HZ_OPT_DECODE_THREADS: return c->opt_dec_threads;
    case HZ_OPT_AUTOTUNE: return c->opt_autotune;
    case HZ_OPT_BATCH_PLAIN: return hz_batch_plain(c->batch) ? 1 : 0;
    case HZ_OPT_BATCH_MAX_REQS: return hz_batch_max_reqs(c->batch);
    default: return -1;
  }
}

uint64_t hz_launch_count(hz_ctx* c) { return c ? c->launches : 0; }

uint32_t hz_tuned_block_size(hz_ctx* c, uint64_t n) {
  return c ? autotuned_block(c, n) : hz_batch_tuned_block_size(n);
}

const char* hz_kernel_name(int32_t id) {
  static const char* names[] = {"histogram",   "build_codes",  "encode_summary", "encode_scan",
                                "encode_pack", "decode_setup", "decode",         "decode_generic",
                                "batch",       "decode_chase"};
  if (id < 0 || id >= (int32_t)(sizeof(names) / sizeof(names[0]))) return "?";
  return names[id];
}

int hz_profile_read(hz_ctx* c, int32_t* ids, float* ms, int max) {
  if (!c) return 0;
  DeviceGuard g(c->device);
  int k = 0;
  for (auto& r : c->prof) {
    float t = 0.f;
    cudaEventSynchronize(r.b);
    cudaEventElapsedTime(&t, r.a, r.b);
    if (k < max) {
      if (ids) ids[k] = r.id;
      if (ms) ms[k] = t;
      ++k;
    }
    c->ev_pool.push_back(r.a);
    c->ev_pool.push_back(r.b);
  }
  c->prof.clear();
  return k;
}

hz_status hz_sync(hz_ctx* c, void* stream) {
  if (!c) return HZ_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return HZ_ERR_CUDA;
  }
  if (cudaMemcpy(c->h_err, c->d_state, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HZ_ERR_CUDA;
  const uint32_t e = c->h_err[0];
  if (e) {
    if (cudaMemset(c->d_state, 0, 2 * sizeof(uint32_t)) != cudaSuccess) return HZ_ERR_CUDA;
    return -(hz_status)e;
  }
  return HZ_OK;
}

// Enqueue histogram + code construction (Sec. 2) into the context state.
static hz_status enqueue_codes(hz_ctx* c, const uint8_t* d_in, uint64_t n, const hz_codes* codes,
                               uint32_t B, uint32_t nb, uint32_t flags, uint32_t sub_S,
                               uint8_t* d_out, uint64_t out_cap, uint64_t* d_out_len,
                               cudaStream_t s) {
  // clear the ticket counters and the histogram (the status word is kept)
  if (cudaMemsetAsync(&c->d_state->tile_counter, 0,
                      offsetof(DevState, codes) - offsetof(DevState, tile_counter), s) !=
      cudaSuccess)
    return HZ_ERR_CUDA;
  LenParam given;
  memset(&given, 0, sizeof(given));
  hz_status st = HZ_OK;
  if (codes) {
    memcpy(given.len, codes->len, 256);
  } else if (n > 0) {
    st = launch(c, K_HIST, s, [&] { return launch_histogram(d_in, n, c->d_state, c->num_sms, s); });
    if (st != HZ_OK) return st;
  }
  return launch(c, K_BUILD, s, [&] {
    return launch_build_codes(c->d_state, codes ? 0 : 1, given, n, B, nb, flags, sub_S, d_out,
                              out_cap, d_out_len, s);
  });
}

// Host-side check of a caller's code table: Kraft's inequality and canonical values.
static bool codes_valid(const hz_codes* codes) {
  uint64_t lo = 0, hi = 0;
  for (int s = 0; s < 256; ++s) {
    const int l = codes->len[s];
    if (!l) continue;
    if (l > kMaxLen) return false;
    const uint64_t add = l == 64 ? 1 : (1ull << (64 - l));
    const uint64_t prev = lo;
    lo += add;
    if (lo < prev) hi += 1;
  }
  if (!(hi == 0 || (hi == 1 && lo == 0))) return false;
  uint64_t code = 0;
  int prev_len = 0;
  bool firstc = true;
  for (int l = 1; l <= kMaxLen; ++l)
    for (int s = 0; s < 256; ++s) {
      if (codes->len[s] != l) continue;
      code = firstc ? 0 : (code + 1) << (l - prev_len);
      firstc = false;
      prev_len = l;
      if (codes->code[s] != code) return false;
    }
  return true;
}

hz_status hz_build_codes(hz_ctx* c, const uint8_t* d_in, uint64_t n, hz_codes* codes_out,
                         void* stream) {
  if (!c || !codes_out || n > 0xFFFFFFFFull || (n && !d_in)) return HZ_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  hz_status st = enqueue_codes(c, d_in, n, nullptr, 1, 0, 0, 0, nullptr, 0, nullptr, s);
  if (st != HZ_OK) return st;
  if (cudaMemcpyAsync(c->h_codes->len, c->d_state->codes.len, 256, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaMemcpyAsync(c->h_codes->code, c->d_state->codes.code, 256 * sizeof(uint64_t),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return HZ_ERR_CUDA;
  st = hz_sync(c, stream);
  if (st != HZ_OK) return st;
  memcpy(codes_out, c->h_codes, sizeof(hz_codes));
  return HZ_OK;
}

// The encoder's launch arguments for n bytes in blocks of B, and its per-tile
// scratch (shared by hz_compress and the host-buffer pipeline).
static hz_status encode_setup(hz_ctx* c, const uint8_t* d_in, uint64_t n, uint32_t B,
                              uint8_t* d_out, uint64_t out_cap, uint64_t* d_out_len,
                              EncodeArgs* a) {
  const uint32_t ntiles = (uint32_t)((n + kEncTile - 1) / kEncTile);
  if (ntiles > c->tiles_cap) {
    uint64_t cap = c->tiles_cap ? c->tiles_cap : 1024;
    while (cap < ntiles) cap *= 2;
    cudaFree(c->d_tiles);
    cudaFree(c->d_meta);
    c->d_tiles = nullptr;
    c->d_meta = nullptr;
    c->tiles_cap = 0;
    if (cudaMalloc(&c->d_tiles, cap * sizeof(TileStatus)) != cudaSuccess ||
        cudaMalloc(&c->d_meta, cap * sizeof(TileMeta)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(c->d_tiles);
      c->d_tiles = nullptr;
      return HZ_ERR_NOMEM;
    }
    c->tiles_cap = (uint32_t)cap;
  }
  a->in = d_in;
  a->n = n;
  a->B = B;
  a->nb = (uint32_t)((n + B - 1) / B);
  a->flags = c->opt_index ? kFlagIndex : 0;
  // sub-block offsets when asked for and S suits B (they need the index)
  const uint32_t S = resolve_sub(c, n, B);
  if (S) a->flags |= kFlagSub;
  a->sub_S = S;
  a->sub_M = S ? B / S : 1;
  a->fdS = make_fastdiv(S ? S : 1);
  a->spin_limit = c->opt_spin_limit;
  a->meta = c->d_meta;
  a->out = d_out;
  a->out_cap = out_cap;
  a->out_len = d_out_len;
  a->st = c->d_state;
  a->tiles = c->d_tiles;
  a->ntiles = ntiles;
  a->fdB = make_fastdiv(B);
  a->tile_begin = 0;
  a->tile_end = ntiles;
  return HZ_OK;
}

hz_status hz_compress(hz_ctx* c, const uint8_t* d_in, uint64_t n, uint32_t block_size,
                      const hz_codes* codes, uint8_t* d_out, uint64_t out_cap,
                      uint64_t* d_out_len, void* stream) {
  if (!c || !d_out || !d_out_len || n > 0xFFFFFFFFull || (n && !d_in)) return HZ_ERR_ARG;
  if (((uintptr_t)d_out & 3) || ((uintptr_t)d_out_len & 7)) return HZ_ERR_ARG;
  if (block_size > kMaxBlock) return HZ_ERR_ARG;
  if (codes && !codes_valid(codes)) return HZ_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t B = block_size ? block_size : autotuned_block(c, n);
  EncodeArgs a;
  hz_status st = encode_setup(c, d_in, n, B, d_out, out_cap, d_out_len, &a);
  if (st != HZ_OK) return st;
  st = enqueue_codes(c, d_in, n, codes, B, a.nb, a.flags, a.sub_S, d_out, out_cap, d_out_len, s);
  if (st != HZ_OK || n == 0) return st;
  if (c->inject_scan_stall) {
    // host-side fault injection: no scan CTA gets ticket 0, so the first one
    // looks back for a predecessor that never publishes, until its bounded
    // wait runs out (HZ_ERR_TIMEOUT)
    c->inject_scan_stall = false;
    if (cudaMemsetAsync(&c->d_state->tile_counter, 1, 1, s) != cudaSuccess) return HZ_ERR_CUDA;
  }
  st = launch(c, K_ENC_SUMMARY, s, [&] { return launch_encode_summary(a, c->num_sms, s); });
  if (st == HZ_OK) st = launch(c, K_ENC_SCAN, s, [&] { return launch_encode_scan(a, s); });
  if (st == HZ_OK) st = launch(c, K_ENC_PACK, s, [&] { return launch_encode_pack(a, c->num_sms, s); });
  return st;
}

// Scratch of the parallel chase for a stream of in_len bytes (one allocation
// carved into the ChaseScratch arrays).
static hz_status ensure_chase_scratch(hz_ctx* c, uint64_t in_len) {
  const uint64_t bm = (in_len / 4 + 31) / 32 + 2;
  if (bm > 0xFFFFFFF0ull) return HZ_ERR_ARG;
  const uint64_t ccap = (uint64_t)c->chase_cap + 65536, cta = 4096;
  const uint64_t words = 4 + cta + 2 * bm + 5 * ccap + c->chase_cap;
  if (words * 4 > c->chase_work_cap) {
    cudaFree(c->d_chase_work);
    c->d_chase_work = nullptr;
    c->chase_work_cap = 0;
    if (cudaMalloc(&c->d_chase_work, words * 4) != cudaSuccess) {
      cudaGetLastError();
      return HZ_ERR_NOMEM;
    }
    c->chase_work_cap = words * 4;
  }
  uint32_t* p = reinterpret_cast<uint32_t*>(c->d_chase_work);
  hz::ChaseScratch& cs = c->cs;
  cs.bar = p;
  cs.flag = p + 2;
  p += 4;
  cs.cta_tot = p;
  cs.cta_cap = (uint32_t)cta;
  p += cta;
  cs.bitmap = p;
  p += bm;
  cs.base = p;
  p += bm;
  cs.bm_cap = (uint32_t)bm;
  cs.pos = p;
  cs.s0 = p + ccap;
  cs.s1 = p + 2 * ccap;
  cs.r0 = p + 3 * ccap;
  cs.r1 = p + 4 * ccap;
  cs.c_cap = (uint32_t)ccap;
  p += 5 * ccap;
  cs.hits = p;
  return HZ_OK;
}

hz_status hz_decompress(hz_ctx* c, const uint8_t* d_in, uint64_t in_len, uint8_t* d_out,
                        uint64_t out_cap, uint64_t* d_out_len, void* stream) {
  if (!c || !d_in || !d_out_len || ((uintptr_t)d_in & 3) || ((uintptr_t)d_out_len & 7))
    return HZ_ERR_ARG;
  if (out_cap && !d_out) return HZ_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  DecodeArgs a;
  a.in = d_in;
  a.in_len = in_len;
  a.out = d_out;
  a.out_cap = out_cap;
  a.out_len = d_out_len;
  a.st = c->d_state;
  a.chase_index = c->d_chase;
  a.chase_cap = c->chase_cap;
  a.lut_bits = c->opt_lut_bits;
  a.k_begin = 0;
  a.k_end = 0xFFFFFFFFu;
  a.seen_no_index = c->d_seen;
  a.defer_chase = 0;
  if (c->h_seen && *reinterpret_cast<volatile uint32_t*>(c->h_seen) &&
      in_len >= kChaseParallelMin && ensure_chase_scratch(c, in_len) == HZ_OK)
    a.defer_chase = 1;
  hz_status st = launch(c, K_DECODE_SETUP, s, [&] { return launch_decode_setup(a, c->d_dec, s); });
  if (st != HZ_OK) return st;
  if (a.defer_chase) {
    st = launch(c, K_DECODE_CHASE, s,
                [&] { return launch_decode_chase(a, c->d_dec, c->cs, c->num_sms, s); });
    if (st != HZ_OK) return st;
  }
  // (blocks longer than 64 KiB are decoded by the same launch, a CTA per block)
  return launch(c, K_DECODE, s, [&] {
    return launch_decode_blocks(a, c->d_dec, c->opt_dec_threads, c->num_sms, s);
  });
}

// Decompress a large host-resident stream with an index as a pipeline of
// kPipeGroups groups of consecutive blocks: each group's records are copied
// in on one stream, decoded as soon as they have landed (the decoder needs
// only the header, the index and a block's own record), and its output is
// copied out on a third stream while later groups are still coming in.  The
// host reads the header and the index from the caller's buffer only to cut
// the groups.  Returns HZ_PENDING, having done nothing, when the stream is
// small, has no index, has blocks too large for the fast decoder, or its
// header or index does not describe the buffer (the plain path then reports
// what is wrong).  On a decoding error the output buffer may hold partial
// data; the status says so.
static hz_status decompress_host_pipelined(hz_ctx* c, const uint8_t* h_in, uint64_t in_len,
                                           uint8_t* h_out, uint64_t out_cap, uint64_t* out_len,
                                           cudaStream_t s) {
  if (in_len < kPipeMinBytes || !c->s_in) return HZ_PENDING;
  uint32_t flags, B, nb;
  uint64_t n;
  memcpy(&flags, h_in + 4, 4);
  memcpy(&n, h_in + 8, 8);
  memcpy(&B, h_in + 16, 4);
  memcpy(&nb, h_in + 20, 4);
  if (memcmp(h_in, "HZB1", 4) != 0 || !(flags & kFlagIndex) || (flags & ~(kFlagIndex | kFlagSub)) ||
      B == 0 || nb < (uint32_t)kPipeGroups || (uint64_t)nb != (n + B - 1) / B || n > out_cap)
    return HZ_PENDING;
  uint32_t S = 0;
  if (flags & kFlagSub) {
    if (kHeaderBytes + 4ull * nb + 4 > in_len) return HZ_PENDING;
    memcpy(&S, h_in + kHeaderBytes + 4ull * nb, 4);
    if (!sub_size_ok(B, S)) return HZ_PENDING;
  } else if (B > 65536) {
    return HZ_PENDING;  // blocks for the CTA-per-block decoder: one launch
  }
  const uint64_t blocks_at = records_at(nb, B, flags, S);
  if (blocks_at > in_len) return HZ_PENDING;
  // group g covers blocks [kg[g], kg[g + 1]) and stream bytes [at[g], at[g + 1])
  uint32_t kg[kPipeGroups + 1];
  uint64_t at[kPipeGroups + 1];
  for (int gi = 0; gi <= kPipeGroups; ++gi) {
    kg[gi] = (uint32_t)((uint64_t)nb * gi / kPipeGroups);
    uint32_t O = 0;
    if (kg[gi] < nb) memcpy(&O, h_in + kHeaderBytes + 4ull * kg[gi], 4);
    at[gi] = kg[gi] < nb ? blocks_at + 4ull * O : in_len;
    if (at[gi] > in_len || (gi && at[gi] < at[gi - 1])) return HZ_PENDING;
  }
  at[0] = 0;  // the first group also brings the header and the index
  DecodeArgs a;
  a.in = c->d_hin;
  a.in_len = in_len;
  a.out = c->d_hout;
  a.out_cap = out_cap;
  a.out_len = c->d_len;
  a.st = c->d_state;
  a.chase_index = c->d_chase;
  a.chase_cap = c->chase_cap;
  a.lut_bits = c->opt_lut_bits;
  a.seen_no_index = c->d_seen;
  a.defer_chase = 0;  // the stream has an index
  // the caller's stream may have work on these buffers queued: start after it
  if (cudaEventRecord(c->e_start, s) != cudaSuccess ||
      cudaStreamWaitEvent(c->s_in, c->e_start, 0) != cudaSuccess ||
      cudaStreamWaitEvent(c->s_out, c->e_start, 0) != cudaSuccess)
    return HZ_ERR_CUDA;
  for (int gi = 0; gi < kPipeGroups; ++gi) {
    if (cudaMemcpyAsync(c->d_hin + at[gi], h_in + at[gi], at[gi + 1] - at[gi],
                        cudaMemcpyHostToDevice, c->s_in) != cudaSuccess ||
        cudaEventRecord(c->e_in[gi], c->s_in) != cudaSuccess)
      return HZ_ERR_CUDA;
  }
  hz_status st = HZ_OK;
  for (int gi = 0; gi < kPipeGroups && st == HZ_OK; ++gi) {
    if (cudaStreamWaitEvent(s, c->e_in[gi], 0) != cudaSuccess) st = HZ_ERR_CUDA;
    if (st == HZ_OK && gi == 0)
      st = launch(c, K_DECODE_SETUP, s, [&] { return launch_decode_setup(a, c->d_dec, s); });
    a.k_begin = kg[gi];
    a.k_end = kg[gi + 1];
    if (st == HZ_OK)
      st = launch(c, K_DECODE, s, [&] {
        return launch_decode_blocks(a, c->d_dec, c->opt_dec_threads, c->num_sms, s);
      });
    if (st == HZ_OK && cudaEventRecord(c->e_dec[gi], s) != cudaSuccess) st = HZ_ERR_CUDA;
    if (st == HZ_OK && cudaStreamWaitEvent(c->s_out, c->e_dec[gi], 0) != cudaSuccess)
      st = HZ_ERR_CUDA;
    const uint64_t o0 = (uint64_t)kg[gi] * B;
    const uint64_t o1 = gi + 1 < kPipeGroups ? (uint64_t)kg[gi + 1] * B : n;
    if (st == HZ_OK && o1 > o0 &&
        cudaMemcpyAsync(h_out + o0, c->d_hout + o0, o1 - o0, cudaMemcpyDeviceToHost, c->s_out) !=
            cudaSuccess)
      st = HZ_ERR_CUDA;
  }
  const bool in_done = cudaStreamSynchronize(c->s_in) == cudaSuccess;
  const bool out_done = cudaStreamSynchronize(c->s_out) == cudaSuccess;
  if (st != HZ_OK) {
    cudaStreamSynchronize(s);
    return st;
  }
  if (cudaMemcpyAsync(c->h_len, c->d_len, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return HZ_ERR_CUDA;
  st = hz_sync(c, s);
  if (st == HZ_OK && (!in_done || !out_done)) st = HZ_ERR_CUDA;
  *out_len = *c->h_len;
  return st;
}

// Compress a large host-resident buffer with the copies overlapped:
//   - the input goes in as kPipeGroups chunks on s_in, and each chunk's
//     histogram runs as soon as it has landed;
//   - after code construction, the length-summing pass and the scan, one sync
//     brings back the stream size and the start states of kPipeGroups - 1
//     tile boundaries;
//   - the tiles are then packed in kPipeGroups groups, and after each group
//     the stream words it finished are copied out on s_out: every word before
//     the delimiter of the record that is open where the next group starts
//     (each record's words and delimiter come from its own tiles);
//   - the header and the index (whose entries the packing writes) go last.
// HZ_PENDING: the buffer is too small for the pipeline to pay.
static hz_status compress_host_pipelined(hz_ctx* c, const uint8_t* h_in, uint64_t n,
                                         uint32_t block_size, uint8_t* h_out, uint64_t out_cap,
                                         uint64_t* out_len, cudaStream_t s) {
  if (n < kPipeMinBytes || !c->s_in || !c->s_out) return HZ_PENDING;
  const uint32_t B = block_size ? block_size : autotuned_block(c, n);
  const uint64_t bound = hz_compress_bound_ctx(c, n, B);
  const uint64_t dcap = out_cap < bound ? out_cap : bound;
  hz_status st = grow((void**)&c->d_hin, &c->d_hin_cap, n);
  if (st == HZ_OK) st = grow((void**)&c->d_hout, &c->d_hout_cap, dcap ? dcap : 16);
  EncodeArgs a;
  if (st == HZ_OK) st = encode_setup(c, c->d_hin, n, B, c->d_hout, dcap, c->d_len, &a);
  if (st != HZ_OK) return st;
  if (cudaMemsetAsync(&c->d_state->tile_counter, 0,
                      offsetof(DevState, codes) - offsetof(DevState, tile_counter), s) !=
      cudaSuccess)
    return HZ_ERR_CUDA;
  // input chunks of whole MiB (16-byte aligned for the histogram's loads)
  const uint64_t chunk = ((n + kPipeGroups - 1) / kPipeGroups + (1u << 20) - 1) & ~((1ull << 20) - 1);
  for (int gi = 0; gi < kPipeGroups && st == HZ_OK; ++gi) {
    const uint64_t off = (uint64_t)gi * chunk;
    if (off >= n) break;
    const uint64_t len = n - off < chunk ? n - off : chunk;
    if (cudaMemcpyAsync(c->d_hin + off, h_in + off, len, cudaMemcpyHostToDevice, c->s_in) !=
            cudaSuccess ||
        cudaEventRecord(c->e_in[gi], c->s_in) != cudaSuccess ||
        cudaStreamWaitEvent(s, c->e_in[gi], 0) != cudaSuccess)
      st = HZ_ERR_CUDA;
    if (st == HZ_OK)
      st = launch(c, K_HIST, s,
                  [&] { return launch_histogram(c->d_hin + off, len, c->d_state, c->num_sms, s); });
  }
  LenParam none;
  memset(&none, 0, sizeof(none));
  if (st == HZ_OK)
    st = launch(c, K_BUILD, s, [&] {
      return launch_build_codes(c->d_state, 1, none, n, B, a.nb, a.flags, a.sub_S, c->d_hout,
                                dcap, c->d_len, s);
    });
  if (st == HZ_OK)
    st = launch(c, K_ENC_SUMMARY, s, [&] { return launch_encode_summary(a, c->num_sms, s); });
  if (st == HZ_OK) st = launch(c, K_ENC_SCAN, s, [&] { return launch_encode_scan(a, s); });
  // tile groups, and the start state (open record's delimiter word) of each
  uint32_t tg[kPipeGroups + 1];
  for (int gi = 0; gi <= kPipeGroups; ++gi)
    tg[gi] = (uint32_t)((uint64_t)a.ntiles * gi / kPipeGroups);
  for (int gi = 1; gi < kPipeGroups && st == HZ_OK; ++gi)
    if (cudaMemcpyAsync(c->h_len + gi, &a.tiles[tg[gi]].pre_O, 8, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
      st = HZ_ERR_CUDA;
  if (st == HZ_OK && cudaMemcpyAsync(c->h_len, c->d_len, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    st = HZ_ERR_CUDA;
  if (st != HZ_OK) {
    cudaStreamSynchronize(c->s_in);
    cudaStreamSynchronize(s);
    return st;
  }
  st = hz_sync(c, s);  // size, capacity and code errors are known here
  *out_len = *c->h_len;
  if (st != HZ_OK) return st;
  if (*out_len > out_cap) return HZ_ERR_CAPACITY;
  const uint64_t rec_base = records_at(a.nb, a.B, a.flags, a.sub_S);
  uint64_t wb[kPipeGroups + 1];
  wb[0] = 0;
  for (int gi = 1; gi < kPipeGroups; ++gi) wb[gi] = c->h_len[gi];
  wb[kPipeGroups] = (*out_len - rec_base) / 4;
  for (int gi = 0; gi < kPipeGroups && st == HZ_OK; ++gi) {
    a.tile_begin = tg[gi];
    a.tile_end = tg[gi + 1];
    st = launch(c, K_ENC_PACK, s, [&] { return launch_encode_pack(a, c->num_sms, s); });
    if (st == HZ_OK && (cudaEventRecord(c->e_dec[gi], s) != cudaSuccess ||
                        cudaStreamWaitEvent(c->s_out, c->e_dec[gi], 0) != cudaSuccess))
      st = HZ_ERR_CUDA;
    const uint64_t b0 = rec_base + 4 * wb[gi], b1 = rec_base + 4 * wb[gi + 1];
    if (st == HZ_OK && b1 > b0 &&
        cudaMemcpyAsync(h_out + b0, c->d_hout + b0, b1 - b0, cudaMemcpyDeviceToHost, c->s_out) !=
            cudaSuccess)
      st = HZ_ERR_CUDA;
  }
  if (st == HZ_OK &&
      cudaMemcpyAsync(h_out, c->d_hout, rec_base, cudaMemcpyDeviceToHost, c->s_out) != cudaSuccess)
    st = HZ_ERR_CUDA;
  const bool out_done = cudaStreamSynchronize(c->s_out) == cudaSuccess;
  const hz_status st2 = hz_sync(c, s);  // errors of the packing
  if (st != HZ_OK) return st;
  if (!out_done) return HZ_ERR_CUDA;
  return st2;
}

hz_status hz_compress_host(hz_ctx* c, const uint8_t* h_in, uint64_t n, uint32_t block_size,
                           uint8_t* h_out, uint64_t out_cap, uint64_t* out_len, void* stream) {
  if (!c || !h_out || !out_len || (n && !h_in) || n > 0xFFFFFFFFull) return HZ_ERR_ARG;
  if (block_size > kMaxBlock) return HZ_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  hz_status st = compress_host_pipelined(c, h_in, n, block_size, h_out, out_cap, out_len, s);
  if (st != HZ_PENDING) return st;
  const uint64_t bound = hz_compress_bound_ctx(c, n, block_size);
  const uint64_t dcap = out_cap < bound ? out_cap : bound;
  st = grow((void**)&c->d_hin, &c->d_hin_cap, n ? n : 16);
  if (st == HZ_OK) st = grow((void**)&c->d_hout, &c->d_hout_cap, dcap ? dcap : 16);
  if (st != HZ_OK) return st;
  if (n && cudaMemcpyAsync(c->d_hin, h_in, n, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return HZ_ERR_CUDA;
  st = hz_compress(c, c->d_hin, n, block_size, nullptr, c->d_hout, dcap, c->d_len, stream);
  if (st != HZ_OK) return st;
  if (cudaMemcpyAsync(c->h_len, c->d_len, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return HZ_ERR_CUDA;
  st = hz_sync(c, stream);
  *out_len = *c->h_len;
  if (st != HZ_OK) return st;
  if (*out_len > out_cap) return HZ_ERR_CAPACITY;
  if (cudaMemcpyAsync(h_out, c->d_hout, *out_len, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return HZ_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? HZ_OK : HZ_ERR_CUDA;
}

hz_status hz_decompress_host(hz_ctx* c, const uint8_t* h_in, uint64_t in_len, uint8_t* h_out,
                             uint64_t out_cap, uint64_t* out_len, void* stream) {
  if (!c || !h_in || !out_len || (out_cap && !h_out)) return HZ_ERR_ARG;
  DeviceGuard g(c->device);
  cudaStream_t s = (cudaStream_t)stream;
  hz_status st = grow((void**)&c->d_hin, &c->d_hin_cap, in_len ? in_len : 16);
  if (st == HZ_OK) st = grow((void**)&c->d_hout, &c->d_hout_cap, out_cap ? out_cap : 16);
  if (st != HZ_OK) return st;
  st = decompress_host_pipelined(c, h_in, in_len, h_out, out_cap, out_len, s);
  if (st != HZ_PENDING) return st;  // HZ_PENDING: the stream does not suit the pipeline
  if (cudaMemcpyAsync(c->d_hin, h_in, in_len, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return HZ_ERR_CUDA;
  st = hz_decompress(c, c->d_hin, in_len, c->d_hout, out_cap, c->d_len, stream);
  if (st != HZ_OK) return st;
  if (cudaMemcpyAsync(c->h_len, c->d_len, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return HZ_ERR_CUDA;
  // the decoded size is known from the header once setup has run; copy back
  // only after the status is known
  st = hz_sync(c, stream);
  *out_len = *c->h_len;
  if (st != HZ_OK) return st;
  if (*out_len && cudaMemcpyAsync(h_out, c->d_hout, *out_len, cudaMemcpyDeviceToHost, s) !=
                      cudaSuccess)
    return HZ_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? HZ_OK : HZ_ERR_CUDA;
}

hz_status hz_submit(hz_ctx* c, const hz_request* reqs, uint32_t count, uint64_t* ticket_out,
                    void* stream) {
  if (!c || !ticket_out || (count && !reqs)) return HZ_ERR_ARG;
  DeviceGuard g(c->device);
  return hz_batch_submit(c->batch, c, reqs, count, ticket_out, true, stream);
}

hz_status hz_poll(hz_ctx* c, uint64_t ticket, int64_t timeout_ns, hz_status* per_req,
                  uint64_t* out_lens) {
  if (!c) return HZ_ERR_ARG;
  DeviceGuard g(c->device);
  return hz_batch_poll(c->batch, ticket, timeout_ns, per_req, out_lens);
}

}  // extern "C"

hz::DevState* hz_ctx_state(hz_ctx* c) { return c->d_state; }
uint32_t hz_ctx_block_size(hz_ctx* c, uint64_t n) { return autotuned_block(c, n); }
void hz_ctx_set_tuned(hz_ctx* c, const uint32_t* B, int lut_bits, int dec_threads) {
  for (int k = 0; k < 4; ++k) c->tuned_B[k] = B[k];
  if (lut_bits) c->opt_lut_bits = lut_bits;
  if (dec_threads) c->opt_dec_threads = dec_threads;
}
void hz_ctx_get_tuned(hz_ctx* c, uint32_t* B, int* lut_bits, int* dec_threads) {
  for (int k = 0; k < 4; ++k) B[k] = c->tuned_B[k];
  *lut_bits = c->opt_lut_bits;
  *dec_threads = c->opt_dec_threads;
}
int hz_ctx_device(hz_ctx* c) { return c->device; }
int hz_ctx_lut_bits(hz_ctx* c) { return c->opt_lut_bits; }
BatchState* hz_ctx_batch(hz_ctx* c) { return c->batch; }
