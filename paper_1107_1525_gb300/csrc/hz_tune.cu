// hz_tune.cu -- the autotuner behind hz_autotune (declared in include/hz.h)
// and its JSON cache.
//
// Per input-size class it times compress + decompress round trips of a slice
// of the caller's sample for every candidate block size (or, with
// HZ_OPT_TUNE_BATCHED, batches of such slices through hz_submit), keeps the
// fastest one whose per-block format overhead stays within 1 % (Sec. 2.1:
// each block costs 32-63 bits) -- a candidate must beat the default by 3 % --
// and then times the decoder's table width and its CTA width on the largest
// class the same way.  The result lives in the context; HZ_TUNE_CACHE names a file that
// stores it across processes.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <chrono>

#include "hz_internal.cuh"

uint32_t hz_ctx_block_size(hz_ctx* c, uint64_t n);
void hz_ctx_set_tuned(hz_ctx* c, const uint32_t* B, int lut_bits, int dec_threads);
void hz_ctx_get_tuned(hz_ctx* c, uint32_t* B, int* lut_bits, int* dec_threads);
int hz_ctx_device(hz_ctx* c);
uint32_t hz_batch_tuned_block_size(uint64_t n);

// A candidate replaces the current choice only when it is faster by more than
// this fraction: timing noise alone must not move a choice.
constexpr float kTuneMargin = 0.03f;

namespace {

constexpr uint64_t kClassSize[4] = {64ull << 10, 1ull << 20, 16ull << 20, 256ull << 20};
constexpr uint32_t kCandB[5] = {4096, 8192, 16384, 32768, 65536};
constexpr int kCandW[3] = {10, 11, 12};
constexpr int kCandThreads[2] = {256, 128};

void write_cache(const uint32_t* B, int W, int T) {
  const char* path = getenv("HZ_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "w");
  if (!f) return;
  fprintf(f,
          "{\"version\": 1, \"block_size\": [%u, %u, %u, %u], \"lut_bits\": %d, "
          "\"dec_threads\": %d}\n",
          B[0], B[1], B[2], B[3], W, T);
  fclose(f);
}

}  // namespace

void hz_tune_load_cache(hz_ctx* c) {
  const char* path = getenv("HZ_TUNE_CACHE");
  if (!path || !*path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char buf[512] = {0};
  const size_t got = fread(buf, 1, sizeof(buf) - 1, f);
  fclose(f);
  buf[got] = 0;
  uint32_t B[4];
  int W = 0, T = 0;
  const char* p = strstr(buf, "\"block_size\"");
  const char* q = strstr(buf, "\"lut_bits\"");
  const char* t = strstr(buf, "\"dec_threads\"");  // absent from older files: keep the default
  if (!p || !q) return;
  if (sscanf(p, "\"block_size\": [%u, %u, %u, %u]", &B[0], &B[1], &B[2], &B[3]) != 4) return;
  if (sscanf(q, "\"lut_bits\": %d", &W) != 1) return;
  if (t && (sscanf(t, "\"dec_threads\": %d", &T) != 1 || (T != 128 && T != 256))) return;
  for (int k = 0; k < 4; ++k)
    if (B[k] == 0 || B[k] > hz::kMaxBlock) return;
  if (W < hz::kLutMinBits || W > hz::kLutMaxBits) return;
  hz_ctx_set_tuned(c, B, W, T);
}

extern "C" hz_status hz_autotune(hz_ctx* c, const uint8_t* d_sample, uint64_t n, void* stream) {
  if (!c || !d_sample || n < 4096 || n > 0xFFFFFFFFull) return HZ_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(hz_ctx_device(c));
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t m_max = n < kClassSize[3] ? n : kClassSize[3];
  // room for the largest trial stream (with the context's options, e.g. sub-block offsets)
  uint64_t cap = 0;
  for (uint32_t B : kCandB) {
    const uint64_t b = hz_compress_bound_ctx(c, m_max, B);
    cap = b > cap ? b : cap;
  }
  uint8_t *d_out = nullptr, *d_dec = nullptr;
  uint64_t* d_len = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hz_status result = HZ_OK;
  uint32_t best_B[4];
  int best_W = 12, best_T = 256;
  uint32_t old_B[4];
  int old_W = 12, old_T = 256;
  hz_ctx_get_tuned(c, old_B, &old_W, &old_T);
  if (cudaMalloc(&d_out, cap) != cudaSuccess || cudaMalloc(&d_dec, m_max) != cudaSuccess ||
      cudaMalloc(&d_len, 2 * sizeof(uint64_t)) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    result = HZ_ERR_NOMEM;
  }
  auto round_trip = [&](uint64_t m, uint32_t B, int iters, float* ms, uint64_t* len) -> hz_status {
    hz_status st = HZ_OK;
    cudaEventRecord(e0, s);
    for (int it = 0; it < iters && st == HZ_OK; ++it) {
      st = hz_compress(c, d_sample, m, B, nullptr, d_out, cap, d_len, s);
      uint64_t slen = 0;
      if (st == HZ_OK && it == 0) {
        // the first stream's size, for the decode and the overhead check
        cudaMemcpyAsync(&slen, d_len, 8, cudaMemcpyDeviceToHost, s);
        st = hz_sync(c, s);
        *len = slen;
      }
      if (st == HZ_OK) st = hz_decompress(c, d_out, *len, d_dec, m, d_len + 1, s);
    }
    cudaEventRecord(e1, s);
    if (st == HZ_OK) st = hz_sync(c, s);
    if (st == HZ_OK) cudaEventElapsedTime(ms, e0, e1);
    return st;
  };
  // Batched objective: a class's slices go through hz_submit as one batch of
  // up to kBatchSlices requests (compress, then decompress of the streams).
  const bool batched = hz_get_option(c, HZ_OPT_TUNE_BATCHED) != 0;
  constexpr uint32_t kBatchSlices = 64;
  auto batch_trip = [&](uint64_t m, uint32_t B, int iters, float* ms, uint64_t* len) -> hz_status {
    const uint32_t k = (uint32_t)(n / m < kBatchSlices ? n / m : kBatchSlices);
    const uint64_t scap = hz_compress_bound_ctx(c, m, B);
    if (k == 0 || (uint64_t)k * scap > cap || (uint64_t)k * m > m_max) return HZ_ERR_ARG;
    hz_request rq[kBatchSlices];
    uint64_t lens[kBatchSlices];
    hz_status per[kBatchSlices];
    auto run = [&](int op) -> hz_status {
      for (uint32_t i = 0; i < k; ++i) {
        rq[i].op = op;
        rq[i].block_size = B;
        rq[i].d_src = op == HZ_OP_COMPRESS ? d_sample + i * m : d_out + i * scap;
        rq[i].src_len = op == HZ_OP_COMPRESS ? m : lens[i];
        rq[i].d_dst = op == HZ_OP_COMPRESS ? d_out + i * scap : d_dec + i * m;
        rq[i].dst_cap = op == HZ_OP_COMPRESS ? scap : m;
      }
      uint64_t t = 0;
      hz_status st = hz_submit(c, rq, k, &t, s);
      if (st == HZ_OK) st = hz_poll(c, t, -1, per, op == HZ_OP_COMPRESS ? lens : nullptr);
      for (uint32_t i = 0; st == HZ_OK && i < k; ++i)
        if (per[i] != HZ_OK) st = per[i];
      return st;
    };
    hz_status st = run(HZ_OP_COMPRESS);  // warm-up; also the streams' sizes
    if (st == HZ_OK) st = run(HZ_OP_DECOMPRESS);
    uint64_t total = 0;
    for (uint32_t i = 0; i < k; ++i) total += lens[i];
    *len = total / k;
    const auto t0 = std::chrono::steady_clock::now();
    for (int it = 0; it < iters && st == HZ_OK; ++it) {
      st = run(HZ_OP_COMPRESS);
      if (st == HZ_OK) st = run(HZ_OP_DECOMPRESS);
    }
    *ms = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return st;
  };
  for (int k = 0; k < 4 && result == HZ_OK; ++k) {
    const uint64_t m = n < kClassSize[k] ? n : kClassSize[k];
    const int iters = (int)((256ull << 20) / m) < 1 ? 1 : ((256ull << 20) / m > 64 ? 64 : (int)((256ull << 20) / m));
    const int biters = iters / 16 > 2 ? iters / 16 : 2;
    // the default (the built-in size table) is the choice to beat
    const uint32_t B0 = hz_batch_tuned_block_size(m);
    float best = 1e30f;
    best_B[k] = B0;
    for (int pass = 0; pass < 2; ++pass) {
      for (uint32_t B : kCandB) {
        if ((pass == 0) != (B == B0)) continue;  // the default first
        float ms = 0;
        uint64_t len = 0;
        // warm-up, then the timed round trips
        if (!batched && round_trip(m, B, 1, &ms, &len) != HZ_OK) continue;
        const uint64_t nb = (m + B - 1) / B;
        if (batched ? batch_trip(m, B, biters, &ms, &len) != HZ_OK
                    : (nb * 8 > len / 100 || round_trip(m, B, iters, &ms, &len) != HZ_OK))
          continue;
        if (nb * 8 > len / 100) continue;  // up to 63 bits + delimiter per block: keep within 1 %
        if (ms < best * (pass == 0 ? 1.0f : 1.0f - kTuneMargin)) {
          best = ms;
          best_B[k] = B;
        }
      }
    }
  }
  if (result == HZ_OK) {
    // decoder table width, on the largest class with its chosen block size
    const uint64_t m = m_max;
    float best = 1e30f;
    uint64_t len = 0;
    hz_compress(c, d_sample, m, best_B[3], nullptr, d_out, cap, d_len, s);
    cudaMemcpyAsync(&len, d_len, 8, cudaMemcpyDeviceToHost, s);
    // eight decompressions after a warm-up, in ms (1e30 if one failed)
    auto time_decode = [&]() -> float {
      float ms = 0;
      hz_decompress(c, d_out, len, d_dec, m, d_len + 1, s);
      cudaEventRecord(e0, s);
      for (int it = 0; it < 8; ++it) hz_decompress(c, d_out, len, d_dec, m, d_len + 1, s);
      cudaEventRecord(e1, s);
      if (hz_sync(c, s) != HZ_OK) return 1e30f;
      cudaEventElapsedTime(&ms, e0, e1);
      return ms;
    };
    if (hz_sync(c, s) == HZ_OK) {
      // the defaults (W = 12, 256 threads) are the choices to beat, by the margin
      hz_set_option(c, HZ_OPT_DECODE_THREADS, 256);
      hz_set_option(c, HZ_OPT_DECODE_LUT_BITS, 12);
      best = time_decode();
      best_W = 12;
      for (int W : kCandW) {
        if (W == 12) continue;
        hz_set_option(c, HZ_OPT_DECODE_LUT_BITS, W);
        const float ms = time_decode();
        if (ms < best * (1.0f - kTuneMargin)) {
          best = ms;
          best_W = W;
        }
      }
      hz_set_option(c, HZ_OPT_DECODE_LUT_BITS, best_W);
      best = 1e30f;
      for (int T : kCandThreads) {
        hz_set_option(c, HZ_OPT_DECODE_THREADS, T);
        const float ms = time_decode();
        if (ms < best * (T == 256 ? 1.0f : 1.0f - kTuneMargin)) {
          best = ms;
          best_T = T;
        }
      }
    }
    hz_ctx_set_tuned(c, best_B, best_W, best_T);
    write_cache(best_B, best_W, best_T);
  } else {
    hz_ctx_set_tuned(c, old_B, old_W, old_T);
  }
  cudaFree(d_out);
  cudaFree(d_dec);
  cudaFree(d_len);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (prev >= 0) cudaSetDevice(prev);
  return result;
}
