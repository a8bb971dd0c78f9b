// hz_hist.cu -- byte histogram (Sec. 2 of Cloud et al.: "counting the
// appearance of every distinct symbol in the uncompressed data").
//
// Design: a grid of 4 CTAs per SM streams the input with 16-byte loads.  Each
// CTA keeps 32 private copies of the 256 counters in shared memory, laid out
// h[symbol][lane] so that the 32 lanes of a warp always hit 32 different
// banks, whatever bytes they hold -- skewed data (a Zipf head symbol, a
// 16-symbol alphabet) causes no intra-warp serialisation.  Warps of one CTA
// share the copies through shared-memory atomics.  At the end every CTA folds
// its copies and adds its 256 sums to the global counters.
#include "hz_hist_dev.cuh"

namespace hz {

__global__ void __launch_bounds__(kHistThreads) histogram_kernel(const uint8_t* __restrict__ in,
                                                                 uint64_t n, DevState* st) {
  __shared__ uint32_t h[256 * 32];
  for (int i = threadIdx.x; i < 256 * 32; i += blockDim.x) h[i] = 0;
  __syncthreads();
  uint32_t* col = h + (threadIdx.x & 31);

  // unaligned head bytes, the 16-byte aligned body, and the tail bytes
  uint64_t head = (16 - ((uintptr_t)in & 15)) & 15;
  if (head > n) head = n;
  const uint4* body = reinterpret_cast<const uint4*>(in + head);
  uint64_t nvec = (n - head) >> 4;
  uint64_t tail_lo = head + (nvec << 4);

  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < nvec; i += 4 * stride) {
    uint4 a = __ldg(body + i);
    uint4 b = __ldg(body + i + stride);
    uint4 c = __ldg(body + i + 2 * stride);
    uint4 d = __ldg(body + i + 3 * stride);
    count_vec(col, a);
    count_vec(col, b);
    count_vec(col, c);
    count_vec(col, d);
  }
  for (; i < nvec; i += stride) count_vec(col, __ldg(body + i));
  if (blockIdx.x == gridDim.x - 1) {
    for (uint64_t j = threadIdx.x; j < head; j += blockDim.x) atomicAdd(col + ((uint32_t)in[j] << 5), 1u);
    for (uint64_t j = tail_lo + threadIdx.x; j < n; j += blockDim.x)
      atomicAdd(col + ((uint32_t)in[j] << 5), 1u);
  }
  __syncthreads();
  // fold the 32 copies; rotate the lane index so a warp's reads spread over banks
  for (int s = threadIdx.x; s < 256; s += blockDim.x) {
    uint32_t sum = 0;
#pragma unroll 8
    for (int l = 0; l < 32; ++l) sum += h[(s << 5) + ((l + s) & 31)];
    if (sum) atomicAdd(&st->hist[s], sum);
  }
}

cudaError_t launch_histogram(const uint8_t* in, uint64_t n, DevState* st, int num_sms,
                             cudaStream_t s) {
  uint64_t nvec = n >> 4;
  uint64_t want = (nvec + 2 * kHistThreads - 1) / (2 * kHistThreads);
  int grid = (int)(want < 1 ? 1 : (want > (uint64_t)num_sms * kHistCtasPerSm
                                       ? (uint64_t)num_sms * kHistCtasPerSm
                                       : want));
  histogram_kernel<<<grid, kHistThreads, 0, s>>>(in, n, st);
  return cudaGetLastError();
}

}  // namespace hz
