// hz_build_dev.cuh -- Huffman code construction and the stream header (one
// CTA of 256 threads); used by the single-buffer and the batched kernels.
// The steps are described in hz_build.cu.
#pragma once

#include "hz_internal.cuh"

namespace hz {

static __device__ void build_codes_device(DevState* st, int from_hist, const LenParam& given,
                                   uint64_t n, uint32_t B, uint32_t nb, uint32_t flags,
                                   uint32_t sub_S, uint8_t* out, uint64_t out_cap,
                                   uint64_t* out_len) {
  // weights fit 32 bits: every count and every sum of counts is at most n < 2^32
  __shared__ uint32_t s_freq[256];
  __shared__ uint32_t leaf_w[256];
  __shared__ int leaf_sym[256];
  __shared__ int leaf_par[256];
  __shared__ uint32_t int_w[256];
  __shared__ int anc[2][256];
  __shared__ int dep[2][256];
  __shared__ uint32_t s_len[256];
  __shared__ uint32_t cnt[65];
  __shared__ uint64_t first[65];
  __shared__ uint16_t s_wcnt[256 / 32][kMaxLen + 1];  // symbols of each length per warp
  __shared__ int s_ok;
  const int t = threadIdx.x;

  if (from_hist) {
    s_freq[t] = st->hist[t];
    s_len[t] = 0;
    __syncthreads();
    const uint32_t f = s_freq[t];
    const int present = f > 0;
    const int m = __syncthreads_count(present);
    if (present) {
      int r = 0;
      for (int u = 0; u < 256; ++u) {
        const uint32_t g = s_freq[u];
        r += (g > 0) & ((g < f) | ((g == f) & (u < t)));
      }
      leaf_w[r] = f;
      leaf_sym[r] = t;
    }
    __syncthreads();
    if (m == 1) {
      if (t == 0) s_len[leaf_sym[0]] = 1;  // a single distinct symbol: one 1-bit code
    } else if (m >= 2) {
      if (t == 0) {
        // One thread, so every shared-memory latency on the loop's path would
        // be paid in full: the heads of both queues and the element after
        // each are kept in registers, and the loads run one element ahead.
        int li = 0, qh = 0, qt = 0;
        uint32_t lhead = leaf_w[0], lnext = leaf_w[1];  // leaf_w[li], leaf_w[li + 1]
        uint32_t ihead = 0, inext = 0;  // int_w[qh] if qh < qt, int_w[qh + 1] if qh + 1 < qt
        for (int k = 0; k < m - 1; ++k) {
          uint32_t w = 0;
#pragma unroll
          for (int r = 0; r < 2; ++r) {
            const bool take_leaf = li < m && (qh >= qt || lhead <= ihead);
            if (take_leaf) {
              w += lhead;
              leaf_par[li] = k;
              ++li;
              lhead = lnext;
              lnext = li + 1 < m ? leaf_w[li + 1] : 0u;
            } else {
              w += ihead;
              anc[0][qh] = k;
              ++qh;
              ihead = inext;
              inext = qh + 1 < qt ? int_w[qh + 1] : 0u;
            }
          }
          if (qt == qh) ihead = w;           // the queue was empty
          else if (qt == qh + 1) inext = w;  // it held one node
          int_w[qt++] = w;
        }
        anc[0][m - 2] = -1;  // the last merge is the root
      }
      __syncthreads();
      if (t < m - 1) {
        int p = anc[0][t];
        dep[0][t] = p < 0 ? 0 : 1;
        anc[0][t] = p < 0 ? t : p;
      }
      __syncthreads();
      int cur = 0;
      for (int it = 0; it < 8; ++it) {  // 2^8 > 254, the deepest possible merged node
        if (t < m - 1) {
          int p = anc[cur][t];
          dep[cur ^ 1][t] = dep[cur][t] + dep[cur][p];
          anc[cur ^ 1][t] = anc[cur][p];
        }
        __syncthreads();
        cur ^= 1;
      }
      if (t < m) s_len[leaf_sym[t]] = (uint32_t)dep[cur][leaf_par[t]] + 1;
    }
  } else {
    s_len[t] = given.len[t];  // lengths chosen by the caller
  }
  if (t < 65) cnt[t] = 0;
  if (t == 0) s_ok = 1;
  for (int i = t; i < (256 / 32) * (kMaxLen + 1); i += 256) (&s_wcnt[0][0])[i] = 0;
  __syncthreads();
  const uint32_t myl = s_len[t];
  if (myl > (uint32_t)kMaxLen) s_ok = 0;
  else if (myl) atomicAdd(&cnt[myl], 1u);
  __syncthreads();
  if (t == 0) {
    // Kraft's inequality in exact arithmetic: sum cnt[l] * 2^(64-l) <= 2^64
    uint64_t lo = 0, hi = 0, code = 0;
    uint32_t maxl = 0, nsym = 0;
    for (int l = 1; l <= kMaxLen; ++l) {
      uint64_t c = cnt[l];
      uint64_t add_hi = l < 64 ? (c >> l) : 0;
      uint64_t add_lo = l < 64 ? (c << (64 - l)) : c;
      uint64_t prev = lo;
      lo += add_lo;
      hi += add_hi + (lo < prev ? 1 : 0);
      // first canonical code of length l (cnt[0] is 0): codes of each length
      // follow on from the previous length's last code, shifted one bit
      code = (code + cnt[l - 1]) << 1;
      first[l] = code;
      if (c) {
        maxl = l;
        nsym += (uint32_t)c;
      }
    }
    if (!(hi == 0 || (hi == 1 && lo == 0))) s_ok = 0;
    if (n > 0 && nsym == 0) s_ok = 0;
    st->codes.maxlen = maxl;
    st->codes.nsym = nsym;
  }
  // rank of t among the symbols of its length: its warp's lanes below it
  // with that length, plus those of the earlier warps
  const uint32_t lane = t & 31, warp = t >> 5;
  const uint32_t peers = __match_any_sync(0xFFFFFFFFu, myl);
  if (myl <= (uint32_t)kMaxLen && lane == (uint32_t)(__ffs(peers) - 1))
    s_wcnt[warp][myl] = (uint16_t)__popc(peers);
  __syncthreads();
  uint32_t rank = __popc(peers & ((1u << lane) - 1u));
  if (myl <= (uint32_t)kMaxLen)
    for (uint32_t w = 0; w < warp; ++w) rank += s_wcnt[w][myl];
  const uint64_t mycode = (myl && myl <= (uint32_t)kMaxLen) ? first[myl] + rank : 0;
  st->codes.len[t] = (uint8_t)myl;
  st->codes.code[t] = mycode;
  if (!s_ok) {
    if (t == 0) {
      set_error(st, HZ_ERR_ARG, 0x100);
      st->codes.maxlen = 0xFFFFFFFFu;  // marks the table unusable
    }
    return;
  }
  if (out == nullptr) return;
  // an empty input's stream is the header and, with sub-block offsets, their S word
  const uint64_t head = kHeaderBytes + ((flags & kFlagSub) ? 4ull * nb + 4 : 0ull);
  if (out_cap < head) {
    if (t == 0) {
      set_error(st, HZ_ERR_CAPACITY, 0x101);
      if (nb == 0) *out_len = head;
    }
    return;
  }
  if ((flags & kFlagSub) && t == 0)
    *reinterpret_cast<uint32_t*>(out + kHeaderBytes + 4ull * nb) = sub_S;
  out[24 + t] = (uint8_t)myl;
  if (t < 24) {
    uint8_t b;
    if (t < 4) b = (uint8_t)"HZB1"[t];
    else if (t < 8) b = (uint8_t)(flags >> (8 * (t - 4)));
    else if (t < 16) b = (uint8_t)(n >> (8 * (t - 8)));
    else if (t < 20) b = (uint8_t)(B >> (8 * (t - 16)));
    else b = (uint8_t)(nb >> (8 * (t - 20)));
    out[t] = b;
  }
  if (nb == 0 && t == 0) *out_len = head;
}

}  // namespace hz
