// hz_hist_dev.cuh -- byte counting helpers shared by the histogram kernels.
#pragma once

#include "hz_internal.cuh"

namespace hz {

constexpr int kHistThreads = 512;
constexpr int kHistCtasPerSm = 4;


static __device__ __forceinline__ void count_word(uint32_t* col, uint32_t w) {
  atomicAdd(col + ((w & 0xFFu) << 5), 1u);
  atomicAdd(col + (((w >> 8) & 0xFFu) << 5), 1u);
  atomicAdd(col + (((w >> 16) & 0xFFu) << 5), 1u);
  atomicAdd(col + ((w >> 24) << 5), 1u);
}

static __device__ __forceinline__ void count_vec(uint32_t* col, uint4 v) {
  count_word(col, v.x);
  count_word(col, v.y);
  count_word(col, v.z);
  count_word(col, v.w);
}

// Count in[0..len) into the per-lane columns h[symbol * 32 + lane] (all
// threads of the CTA take part; 16-byte loads on the aligned body).
static __device__ __forceinline__ void count_range(const uint8_t* __restrict__ in, uint64_t len,
                                            uint32_t* h) {
  uint32_t* col = h + (threadIdx.x & 31);
  uint64_t head = (16 - ((uintptr_t)in & 15)) & 15;
  if (head > len) head = len;
  const uint4* body = reinterpret_cast<const uint4*>(in + head);
  const uint64_t nvec = (len - head) >> 4;
  const uint64_t tail_lo = head + (nvec << 4);
  uint64_t i = threadIdx.x;
  for (; i + 3 * blockDim.x < nvec; i += 4 * blockDim.x) {
    uint4 a = __ldg(body + i);
    uint4 b = __ldg(body + i + blockDim.x);
    uint4 c = __ldg(body + i + 2 * blockDim.x);
    uint4 d = __ldg(body + i + 3 * blockDim.x);
    count_vec(col, a);
    count_vec(col, b);
    count_vec(col, c);
    count_vec(col, d);
  }
  for (; i < nvec; i += blockDim.x) count_vec(col, __ldg(body + i));
  for (uint64_t j = threadIdx.x; j < head; j += blockDim.x) atomicAdd(col + ((uint32_t)in[j] << 5), 1u);
  for (uint64_t j = tail_lo + threadIdx.x; j < len; j += blockDim.x)
    atomicAdd(col + ((uint32_t)in[j] << 5), 1u);
}

// Fold the 32 columns and add them to hist[256]; the lane index is rotated
// so a warp's reads spread over the banks.
static __device__ __forceinline__ void fold_columns(const uint32_t* h, uint32_t* hist) {
  for (int s = threadIdx.x; s < 256; s += blockDim.x) {
    uint32_t sum = 0;
#pragma unroll 8
    for (int l = 0; l < 32; ++l) sum += h[(s << 5) + ((l + s) & 31)];
    if (sum) atomicAdd(&hist[s], sum);
  }
}

}  // namespace hz
