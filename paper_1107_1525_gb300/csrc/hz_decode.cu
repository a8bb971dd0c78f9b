// hz_decode.cu -- block decoder (Sec. 2.1, last paragraph, and Sec. 3.2 of
// Cloud et al.): blocks are located through a table of offsets built from the
// length delimiters and decoded independently.
//
// decode_setup_kernel (one CTA) parses and checks the container header,
// builds the canonical decode tables -- per-length first code and count, the
// symbols in (length, byte) order, and a 2^W-entry lookup table that resolves
// every code of at most W bits in one shared-memory read -- and, for streams
// without a stored index, rebuilds the offset table by walking the
// delimiters (the paper's own scheme).
//
// decode_kernel (persistent CTAs) decodes one block per CTA at a time.  The
// paper gives each block to one thread; a 64 KiB block is then a chain of
// 65 536 dependent table lookups, far too long for a GPU.  Here a block's
// payload is cut into NT equal bit ranges, one per thread, and every thread
// starts decoding at the start of its range as if a code began there.
// Huffman codes resynchronise after a few symbols (the observation of Klein
// and Wiseman that the paper cites in Sec. 2.1), so the decode that started
// at a wrong bit soon lands on the true code boundaries.  A fix-up loop
// re-decodes each range from the true boundary handed over by its left
// neighbour only until the two decodes meet, which corrects the range's
// symbol count; a scan of the counts gives every range its output position;
// a second pass decodes and stores the symbols.  Nothing about the stream
// format changes.
#include "hz_internal.cuh"

namespace hz {

struct DecTables {
  uint32_t ok;          // 1 once the header has been checked
  uint32_t flags, B, nb;
  uint64_t n;
  uint64_t blocks_at;   // byte offset of the record area
  uint32_t maxlen, lut_bits;
  uint32_t cnt[kMaxLen + 1];
  uint32_t offs[kMaxLen + 1];   // position in sorted[] of the first code of each length
  uint64_t first[kMaxLen + 1];  // first canonical code of each length
  uint8_t sorted[256];          // symbols in (length, byte) order
  uint16_t lut[1 << kLutMaxBits];  // len << 8 | symbol, 0 = longer than W bits / invalid
};

size_t dec_tables_bytes() { return sizeof(DecTables); }

__device__ __forceinline__ uint32_t ld_u32_bytes(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

__global__ void __launch_bounds__(256) decode_setup_kernel(DecodeArgs a, DecTables* T) {
  __shared__ uint32_t s_len[256];
  __shared__ uint8_t s_sorted[256];
  __shared__ uint32_t cnt[kMaxLen + 1];
  __shared__ uint64_t first[kMaxLen + 1];
  __shared__ uint32_t offs[kMaxLen + 1];
  __shared__ int s_ok;
  __shared__ uint32_t s_maxlen;
  const int t = threadIdx.x;
  if (t == 0) {
    T->ok = 0;
    s_ok = a.in_len >= kHeaderBytes;
  }
  if (t <= kMaxLen) cnt[t] = 0;
  __syncthreads();
  if (!s_ok) {
    if (t == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x300);
    return;  // uniform: every thread leaves here
  }
  const uint8_t* h = a.in;
  const uint32_t flags = ld_u32_bytes(h + 4);
  const uint64_t n = (uint64_t)ld_u32_bytes(h + 8) | ((uint64_t)ld_u32_bytes(h + 12) << 32);
  const uint32_t B = ld_u32_bytes(h + 16);
  const uint32_t nb = ld_u32_bytes(h + 20);
  bool ok = h[0] == 'H' && h[1] == 'Z' && h[2] == 'B' && h[3] == '1';
  ok = ok && (flags & ~kFlagIndex) == 0 && B >= 1 && B <= kMaxBlock && n <= 0xFFFFFFFFull;
  ok = ok && (uint64_t)nb == (n + B - 1) / (B ? B : 1);
  const uint64_t blocks_at = kHeaderBytes + ((flags & kFlagIndex) ? 4ull * nb : 0ull);
  ok = ok && blocks_at <= a.in_len;
  const uint32_t l = h[24 + t];
  s_len[t] = l;
  if (l > (uint32_t)kMaxLen) ok = false;
  if (!ok) s_ok = 0;
  __syncthreads();
  if (s_ok && l) atomicAdd(&cnt[l], 1u);
  __syncthreads();
  if (t == 0 && s_ok) {
    // Kraft's inequality exactly: sum cnt[k] * 2^(64-k) <= 2^64
    uint64_t lo = 0, hi = 0, code = 0;
    uint32_t maxl = 0, nsym = 0, off = 0;
    first[0] = 0;
    offs[0] = 0;
    for (int k = 1; k <= kMaxLen; ++k) {
      const uint64_t c = cnt[k];
      const uint64_t add_hi = k < 64 ? (c >> k) : 0;
      const uint64_t add_lo = k < 64 ? (c << (64 - k)) : c;
      const uint64_t prev = lo;
      lo += add_lo;
      hi += add_hi + (lo < prev ? 1 : 0);
      code = (code + cnt[k - 1]) << 1;
      first[k] = code;
      offs[k] = off;
      off += (uint32_t)c;
      if (c) {
        maxl = k;
        nsym += (uint32_t)c;
      }
    }
    const bool kraft = hi == 0 || (hi == 1 && lo == 0);
    if (!kraft || (n > 0 && nsym == 0)) s_ok = 0;
    s_maxlen = maxl;
  }
  __syncthreads();
  if (!s_ok) {
    if (t == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x301);
    return;  // uniform
  }
  // symbols in (length, byte) order
  if (l) {
    uint32_t rank = 0;
    for (int u = 0; u < t; ++u) rank += s_len[u] == l;
    s_sorted[offs[l] + rank] = (uint8_t)t;
  }
  __syncthreads();
  T->sorted[t] = s_sorted[t];
  if (t <= kMaxLen) {
    T->cnt[t] = cnt[t];
    T->offs[t] = offs[t];
    T->first[t] = first[t];
  }
  // lookup table: entry v resolves the code that is a prefix of the W-bit value v
  const int W = a.lut_bits;
  const uint32_t maxl = s_maxlen;
  for (uint32_t v = t; v < (1u << W); v += blockDim.x) {
    uint16_t e = 0;
    for (int k = 1; k <= W && k <= (int)maxl; ++k) {
      if (!cnt[k]) continue;
      const uint64_t p = v >> (W - k);
      if (p >= first[k] && p - first[k] < cnt[k]) {
        e = (uint16_t)((k << 8) | s_sorted[offs[k] + (uint32_t)(p - first[k])]);
        break;
      }
    }
    T->lut[v] = e;
  }
  const bool cap_ok = n <= a.out_cap;
  if (t == 0) {
    T->flags = flags;
    T->B = B;
    T->nb = nb;
    T->n = n;
    T->blocks_at = blocks_at;
    T->maxlen = maxl;
    T->lut_bits = (uint32_t)W;
    *a.out_len = n;
    if (!cap_ok) set_error(a.st, HZ_ERR_CAPACITY, 0x302);
  }
  if (!cap_ok) return;  // uniform
  __syncthreads();
  if (t == 0) {
    bool chase_ok = true;
    if (!(flags & kFlagIndex)) {
      // no stored index: walk the delimiters (one dependent load per block)
      if (nb > a.chase_cap) {
        set_error(a.st, HZ_ERR_NOMEM, 0x303);
        chase_ok = false;
      }
      uint64_t O = 0;
      for (uint32_t k = 0; chase_ok && k < nb; ++k) {
        const uint64_t at = blocks_at + 4 * O;
        if (at + 4 > a.in_len || O > 0xFFFFFFFFull) {
          set_error(a.st, HZ_ERR_CORRUPT, 0x304);
          chase_ok = false;
          break;
        }
        a.chase_index[k] = (uint32_t)O;
        O += 1 + ceil32(*reinterpret_cast<const uint32_t*>(a.in + at));
      }
    }
    if (chase_ok) {
      __threadfence();
      T->ok = 1;
    }
  }
}

// ------------------------------------------------------------ block decoding
struct BitReader {
  const uint32_t* p;
  uint32_t nw, wi, w0, w1, w2;
  __device__ __forceinline__ uint32_t ld(uint32_t i) const { return i < nw ? __ldg(p + i) : 0u; }
  __device__ __forceinline__ void init(const uint32_t* p_, uint32_t nw_, uint32_t pos) {
    p = p_;
    nw = nw_;
    wi = pos >> 5;
    w0 = ld(wi);
    w1 = ld(wi + 1);
    w2 = ld(wi + 2);
  }
  __device__ __forceinline__ void seek(uint32_t pos) {  // forward only
    while ((pos >> 5) > wi) {
      w0 = w1;
      w1 = w2;
      w2 = ld(wi + 3);
      ++wi;
    }
  }
  __device__ __forceinline__ uint32_t peek32(uint32_t pos) const {
    return __funnelshift_l(w1, w0, pos & 31);
  }
  __device__ __forceinline__ uint64_t peek64(uint32_t pos) const {
    const uint32_t s = pos & 31;
    return ((uint64_t)__funnelshift_l(w1, w0, s) << 32) | __funnelshift_l(w2, w1, s);
  }
};

struct DecShared {
  uint16_t lut[1 << kLutMaxBits];
  uint32_t cnt[kMaxLen + 1];
  uint32_t offs[kMaxLen + 1];
  uint64_t first[kMaxLen + 1];
  uint8_t sorted[256];
  uint32_t maxlen, W, flags, B, nb;
  uint64_t n, blocks_at;
};

// Decode the code starting at bit `pos`: returns its length (0 if no code
// matches, possible only with an incomplete code) and the symbol.
__device__ __forceinline__ uint32_t decode_one(const DecShared& sh, const BitReader& br,
                                               uint32_t pos, uint32_t& sym) {
  const uint32_t v = br.peek32(pos);
  const uint32_t e = sh.lut[v >> (32 - sh.W)];
  if (e >> 8) {
    sym = e & 0xFFu;
    return e >> 8;
  }
  const uint64_t v64 = br.peek64(pos);
  for (uint32_t k = sh.W + 1; k <= sh.maxlen; ++k) {
    const uint32_t c = sh.cnt[k];
    if (!c) continue;
    const uint64_t p = v64 >> (64 - k);
    if (p >= sh.first[k] && p - sh.first[k] < c) {
      sym = sh.sorted[sh.offs[k] + (uint32_t)(p - sh.first[k])];
      return k;
    }
  }
  sym = 0;
  return 0;
}

template <int NT>
struct DecBlockShared {
  uint32_t start[NT], exit[NT], count[NT], offset[NT];
  uint32_t warp_tot[NT / 32];
  uint32_t bits, nw, cnt_k;
  uint64_t rec;
  int ok;
};

template <int NT>
__device__ void decode_block(const DecodeArgs& a, const DecShared& sh, DecBlockShared<NT>& bs,
                             uint32_t k) {
  const int t = threadIdx.x;
  __syncthreads();  // every thread is done with the previous block's shared state
  if (t == 0) {
    bs.ok = 1;
    const uint32_t* idx = (sh.flags & kFlagIndex)
                              ? reinterpret_cast<const uint32_t*>(a.in + kHeaderBytes)
                              : a.chase_index;
    const uint64_t O = idx[k];
    const uint64_t rec = sh.blocks_at + 4 * O;
    uint32_t bits = 0, nw = 0;
    bool ok = rec + 4 <= a.in_len;
    if (ok) {
      bits = *reinterpret_cast<const uint32_t*>(a.in + rec);
      nw = ceil32(bits);
      ok = rec + 4 + 4ull * nw <= a.in_len;
    }
    if (ok) {
      if (k + 1 < sh.nb) ok = (uint64_t)idx[k + 1] == O + 1 + nw;
      else ok = rec + 4 + 4ull * nw == a.in_len;
    }
    const uint64_t lo = (uint64_t)k * sh.B;
    const uint32_t cnt_k = (uint32_t)((lo + sh.B <= sh.n) ? sh.B : sh.n - lo);
    // at least one bit per symbol, at most maxlen bits per symbol
    ok = ok && bits >= cnt_k && (uint64_t)bits <= (uint64_t)cnt_k * sh.maxlen;
    if (ok && (bits & 31)) {
      // padding bits after the last code must be zero
      const uint32_t last = *reinterpret_cast<const uint32_t*>(a.in + rec + 4 + 4ull * (nw - 1));
      ok = (last & ((1u << (32 - (bits & 31))) - 1u)) == 0;
    }
    bs.bits = bits;
    bs.nw = nw;
    bs.cnt_k = cnt_k;
    bs.rec = rec;
    bs.ok = ok;
  }
  __syncthreads();
  if (!bs.ok) {
    if (t == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x310);
    return;
  }
  const uint32_t bits = bs.bits;
  const uint32_t* payload = reinterpret_cast<const uint32_t*>(a.in + bs.rec + 4);
  const uint32_t nw = bs.nw;
  uint32_t L = (bits + NT - 1) / NT;
  L = L < 32 ? 32 : (L + 31) & ~31u;
  const uint32_t nsub = (bits + L - 1) / L;
  const bool active = (uint32_t)t < nsub;
  const uint32_t my_end = active ? ((uint32_t)t + 1) * L < bits ? ((uint32_t)t + 1) * L : bits : 0;

  // ---- pass 1: speculative decode of my range, counting symbols
  if (active) {
    uint32_t pos = (uint32_t)t * L, c = 0, sym;
    BitReader br;
    br.init(payload, nw, pos);
    while (pos < my_end) {
      uint32_t l = decode_one(sh, br, pos, sym);
      pos += l ? l : 1;
      br.seek(pos);
      ++c;
    }
    bs.start[t] = (uint32_t)t * L;
    bs.exit[t] = pos;
    bs.count[t] = c;
  }
  // ---- fix-up: restart each range at its left neighbour's exit until all agree
  for (uint32_t round = 0; round <= (uint32_t)NT; ++round) {
    __syncthreads();
    const uint32_t want = (active && t > 0) ? bs.exit[t - 1] : 0u;
    const bool mismatch = active && t > 0 && want != bs.start[t];
    if (!__syncthreads_or(mismatch)) break;
    if (mismatch) {
      uint32_t pa = want, pb = bs.start[t], ca = 0, cb = 0, sym;
      BitReader ra, rb;
      ra.init(payload, nw, pa);
      rb.init(payload, nw, pb);
      while (pa != pb && (pa < my_end || pb < my_end)) {
        if (pa < pb) {
          uint32_t l = decode_one(sh, ra, pa, sym);
          pa += l ? l : 1;
          ra.seek(pa);
          ++ca;
        } else {
          uint32_t l = decode_one(sh, rb, pb, sym);
          pb += l ? l : 1;
          rb.seek(pb);
          ++cb;
        }
      }
      if (pa == pb) {
        bs.count[t] = bs.count[t] - cb + ca;
      } else {
        bs.exit[t] = pa;
        bs.count[t] = ca;
      }
      bs.start[t] = want;
    }
  }
  __syncthreads();
  // ---- exclusive scan of the counts
  const int lane = t & 31, warp = t >> 5;
  uint32_t v = active ? bs.count[t] : 0u;
  uint32_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) bs.warp_tot[warp] = inc;
  __syncthreads();
  uint32_t wpre = 0;
  for (int w = 0; w < warp; ++w) wpre += bs.warp_tot[w];
  const uint32_t my_off = wpre + inc - v;
  if (t == NT - 1) {
    const uint32_t total = wpre + inc;
    if (total != bs.cnt_k || bs.exit[nsub - 1] != bits) bs.ok = 0;
  }
  __syncthreads();
  if (!bs.ok) {
    if (t == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x311);
    return;
  }
  // ---- pass 2: decode from the true boundary and store the symbols
  if (active && v) {
    uint32_t pos = bs.start[t], sym;
    BitReader br;
    br.init(payload, nw, pos);
    uint8_t* dst = a.out + (uint64_t)k * sh.B + my_off;
    uint32_t fill = (uint32_t)((uintptr_t)dst & 3u);
    uint32_t lo = fill;
    uint32_t* wp = reinterpret_cast<uint32_t*>(dst - fill);
    uint32_t acc = 0;
    bool bad = false;
    for (uint32_t j = 0; j < v; ++j) {
      uint32_t l = decode_one(sh, br, pos, sym);
      bad |= l == 0;
      pos += l ? l : 1;
      br.seek(pos);
      acc |= sym << (8 * fill);
      if (++fill == 4) {
        if (lo == 0) {
          *wp = acc;
        } else {
          uint8_t* b = reinterpret_cast<uint8_t*>(wp);
          for (uint32_t q = lo; q < 4; ++q) b[q] = (uint8_t)(acc >> (8 * q));
          lo = 0;
        }
        ++wp;
        acc = 0;
        fill = 0;
      }
    }
    if (fill) {
      uint8_t* b = reinterpret_cast<uint8_t*>(wp);
      for (uint32_t q = lo; q < fill; ++q) b[q] = (uint8_t)(acc >> (8 * q));
    }
    if (bad || pos != bs.exit[t]) set_error(a.st, HZ_ERR_CORRUPT, 0x312);
  }
  __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT) decode_kernel(DecodeArgs a, const DecTables* T) {
  __shared__ DecShared sh;
  __shared__ DecBlockShared<NT> bs;
  if (!T->ok) return;
  const int W = (int)T->lut_bits;
  for (int i = threadIdx.x; i < (1 << W); i += NT) sh.lut[i] = T->lut[i];
  for (int i = threadIdx.x; i <= kMaxLen; i += NT) {
    sh.cnt[i] = T->cnt[i];
    sh.offs[i] = T->offs[i];
    sh.first[i] = T->first[i];
  }
  for (int i = threadIdx.x; i < 256; i += NT) sh.sorted[i] = T->sorted[i];
  if (threadIdx.x == 0) {
    sh.maxlen = T->maxlen;
    sh.W = T->lut_bits;
    sh.flags = T->flags;
    sh.B = T->B;
    sh.nb = T->nb;
    sh.n = T->n;
    sh.blocks_at = T->blocks_at;
  }
  __syncthreads();
  for (uint32_t k = blockIdx.x; k < sh.nb; k += gridDim.x) decode_block<NT>(a, sh, bs, k);
}

cudaError_t launch_decode_setup(const DecodeArgs& a, DecTables* T, cudaStream_t s) {
  decode_setup_kernel<<<1, 256, 0, s>>>(a, T);
  return cudaGetLastError();
}

template <int NT>
static cudaError_t launch_decode_nt(const DecodeArgs& a, const DecTables* T, int num_sms,
                                    cudaStream_t s) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decode_kernel<NT>, NT, 0);
  if (per_sm < 1) per_sm = 1;
  decode_kernel<NT><<<num_sms * per_sm, NT, 0, s>>>(a, T);
  return cudaGetLastError();
}

cudaError_t launch_decode_blocks(const DecodeArgs& a, const DecTables* T, int threads, int num_sms,
                                 cudaStream_t s) {
  switch (threads) {
    case 128: return launch_decode_nt<128>(a, T, num_sms, s);
    case 512: return launch_decode_nt<512>(a, T, num_sms, s);
    default: return launch_decode_nt<256>(a, T, num_sms, s);
  }
}

}  // namespace hz
