// hz_build.cu -- Huffman code construction (Sec. 2 and Fig. 2 of Cloud et
// al.) and the stream header, in one CTA of 256 threads (one per byte value).
//
//   1. rank the present symbols by (frequency, byte value) -- 256 threads,
//      one comparison sweep each;
//   2. two-queue Huffman merge (leaf queue sorted, merged nodes in creation
//      order; on equal weight the leaf is taken, which is the (weight, id)
//      order with leaf id = byte value and merged id = 256 + t) -- one
//      thread, at most 255 steps;
//   3. depth of every merged node by pointer jumping (8 rounds), leaf length
//      = parent depth + 1;
//   4. canonical codes: per-length counts, first code per length, rank of a
//      symbol among the symbols of its length;
//   5. the 280-byte container header (and the sub-block section's S word),
//      when an output stream is given.
#include "hz_build_dev.cuh"

namespace hz {

__global__ void __launch_bounds__(256) build_codes_kernel(DevState* st, int from_hist,
                                                          const LenParam given, uint64_t n,
                                                          uint32_t B, uint32_t nb, uint32_t flags,
                                                          uint32_t sub_S, uint8_t* out,
                                                          uint64_t out_cap, uint64_t* out_len) {
  build_codes_device(st, from_hist, given, n, B, nb, flags, sub_S, out, out_cap, out_len);
}

cudaError_t launch_build_codes(DevState* st, int from_hist, const LenParam& given, uint64_t n,
                               uint32_t B, uint32_t nb, uint32_t flags, uint32_t sub_S,
                               uint8_t* out, uint64_t out_cap, uint64_t* out_len, cudaStream_t s) {
  build_codes_kernel<<<1, 256, 0, s>>>(st, from_hist, given, n, B, nb, flags, sub_S, out, out_cap,
                                       out_len);
  return cudaGetLastError();
}

}  // namespace hz
