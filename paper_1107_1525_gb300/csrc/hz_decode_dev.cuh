// hz_decode_dev.cuh -- device functions of the block decoder, shared by the
// single-stream kernels (hz_decode.cu) and the batched kernels (hz_batch.cu).
// The design is described in hz_decode.cu.
#pragma once

#include "hz_internal.cuh"

namespace hz {

// Lookup-table entry for the W-bit value v (u32):
//   bits  0..7   first symbol            bits  8..15  second symbol (0 if none)
//   bits 16..17  symbols resolved (0: the first code is longer than W bits,
//                or no code matches), 1 or 2
//   bits 18..22  bits consumed by them   bits 23..26  length of the first code
// When no symbol resolves and the second-level table exists, a value that
// starts codes longer than W bits holds instead, in bits 0..15, the start of
// its part of the second-level table and, in bits 18..22, the e >= 1 extra
// bits that index it; an all-zero entry means no code starts with v.
static __host__ __device__ constexpr uint32_t lut_entry(uint32_t s0, uint32_t s1, uint32_t ns,
                                                 uint32_t nbits, uint32_t l0) {
  return s0 | (s1 << 8) | (ns << 16) | (nbits << 18) | (l0 << 23);
}
static __device__ __forceinline__ uint32_t e_ns(uint32_t e) { return (e >> 16) & 3u; }
static __device__ __forceinline__ uint32_t e_nbits(uint32_t e) { return (e >> 18) & 31u; }
static __device__ __forceinline__ uint32_t e_l0(uint32_t e) { return (e >> 23) & 15u; }

// Decoder mode 0 (complete code, no code longer than W bits, blocks of at most
// kFastMaxB symbols) stores another layout, as two 16-bit halves:
//   low half   bits 0..4  bits taken by every complete code that starts in the
//                         W-bit window and ends within its first cap bits
//              bits 8..15 how many codes that is (at least 1)
//   high half  bits 0..4  length of the first code, bits 8..15 its symbol
// Bits 5..7 are zero in both halves, so a step can shift the bit buffer by the
// half itself (funnel shifts use the amount modulo 32) and subtract the whole
// half from one accumulator whose low byte tracks the buffer's bit count.
static __host__ __device__ constexpr uint32_t lut0_entry(uint32_t nbits, uint32_t ns, uint32_t l0,
                                                  uint32_t s0) {
  return nbits | (ns << 8) | ((l0 | (s0 << 8)) << 16);
}
// When no code is longer than 10 bits (and W >= 10) every entry is fixed by the
// top 10 bits, and shared memory holds 8 interleaved copies of that 1024-entry
// table: entry u of copy c (c = lane mod 8) is word 8u + c, so the lanes that
// share a copy (lane, lane + 8, lane + 16, lane + 24) spread over banks c,
// c+8, c+16, c+24 (about 2 wavefronts per lookup instead of about 3.5).
// Otherwise the mode-0 entry of value v sits at lut0_pos(v): bits 5..9 of v folded into
// the bank bits, since v's low bits are the start of the next code, which
// repeats across lanes (long codes share their leading ones) and would pile
// the lanes' lookups onto a few shared-memory banks.  A bijection on [0, 2^W).
static __host__ __device__ constexpr uint32_t lut0_pos(uint32_t v) { return v ^ ((v >> 5) & 31u); }
constexpr uint32_t kFastMaxB = 65536;  // larger blocks go to the generic kernel

// Second-level table entries: codes longer than W bits whose W-bit prefixes
// have at most this many continuations in all; larger code sets take the
// per-length search.
constexpr uint32_t kL2Entries = 2048;

struct DecTables {
  uint32_t ok;          // 1 once the header has been checked (and the offsets are known)
  uint32_t needs_chase; // 1: no stored index, the chase kernel rebuilds the offsets
  uint32_t minlen;      // shortest code length
  uint32_t flags, B, nb;
  uint64_t n;
  uint64_t blocks_at;   // byte offset of the record area
  uint32_t maxlen, lut_bits;
  uint32_t complete;            // Kraft sum exactly 1: every bit string decodes
  uint32_t fill_k;              // mode 0: lut holds the mode-0 layout; steps per buffer fill
                                // of the output pass (2, 3 or 4); 0: the general layout
  uint32_t lut_rep;             // mode 0, no code longer than 10 bits, W >= 10: lut[0, 1024)
                                // is indexed by the top 10 bits, kept 8 times in shared memory
  uint32_t pair;                // lut_rep, sub-block offsets and no code longer than 5 bits:
                                // every 10-bit window holds two whole codes, and the
                                // sub-block decoder takes two symbols a lookup
  uint32_t cnt[kMaxLen + 1];
  uint32_t offs[kMaxLen + 1];   // position in sorted[] of the first code of each length
  uint64_t first[kMaxLen + 1];  // first canonical code of each length
  uint8_t sorted[256];          // symbols in (length, byte) order
  uint32_t lut[1 << kLutMaxBits];
  uint32_t has_l2;              // the second-level table below is built
  uint16_t l2[kL2Entries];      // symbol | length << 8 of codes longer than W (0: none)
  // sub-block offsets (flags bit 1): S symbols per sub-block, M = B / S per
  // block (0 without them), units = nb * M
  uint32_t sub_S, sub_M, units;
};


static __device__ __forceinline__ uint32_t ld_u32_bytes(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

// ================================================================ setup
// Parse the header and build the tables (one CTA of 256 threads).
// The offsets of a stream without a stored index by walking its delimiters,
// one dependent load per record (the paper's own way, Sec. 2.1): record k
// starts 1 + ceil(bits / 32) words after record k - 1.  One thread; false
// (with the error recorded) when the records do not fit the stream.
static __device__ bool serial_chase(const DecodeArgs& a, uint64_t blocks_at, uint32_t nb) {
  if (nb > a.chase_cap) {
    set_error(a.st, HZ_ERR_NOMEM, 0x303);
    return false;
  }
  uint64_t O = 0;
  for (uint32_t k = 0; k < nb; ++k) {
    const uint64_t at = blocks_at + 4 * O;
    if (at + 4 > a.in_len || O > 0xFFFFFFFFull) {
      set_error(a.st, HZ_ERR_CORRUPT, 0x304);
      return false;
    }
    a.chase_index[k] = (uint32_t)O;
    O += 1 + ceil32(*reinterpret_cast<const uint32_t*>(a.in + at));
  }
  return true;
}

static __device__ void decode_setup_device(const DecodeArgs& a, DecTables* T) {
  __shared__ uint32_t s_len[256];
  __shared__ uint8_t s_sorted[256];
  __shared__ uint32_t cnt[kMaxLen + 1];
  __shared__ uint64_t first[kMaxLen + 1];
  __shared__ uint32_t offs[kMaxLen + 1];
  __shared__ int s_ok;
  __shared__ uint32_t s_maxlen, s_complete;
  const int t = threadIdx.x;
  if (t == 0) {
    T->ok = 0;
    T->needs_chase = 0;
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
  ok = ok && (flags & ~(kFlagIndex | kFlagSub)) == 0 && B >= 1 && B <= kMaxBlock &&
       n <= 0xFFFFFFFFull;
  ok = ok && (uint64_t)nb == (n + B - 1) / (B ? B : 1);
  // sub-block offsets: only with the index; S a multiple of 32 dividing B
  uint32_t S = 0;
  if (ok && (flags & kFlagSub)) {
    ok = (flags & kFlagIndex) && kHeaderBytes + 4ull * nb + 4 <= a.in_len;
    if (ok) S = ld_u32_bytes(h + kHeaderBytes + 4ull * nb);
    ok = ok && sub_size_ok(B, S);
  }
  const uint64_t blocks_at = ok ? records_at(nb, B, flags, S) : 0ull;
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
    T->complete = hi == 1 && lo == 0;
    s_complete = hi == 1 && lo == 0;
  }
  __syncthreads();
  if (!s_ok) {
    if (t == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x301);
    return;  // uniform
  }
  // symbols in (length, byte) order: the rank among the symbols of the same
  // length is the count of lower lanes of the warp with it plus the counts of
  // the earlier warps
  __shared__ uint16_t s_wcnt[256 / 32][kMaxLen + 1];
  {
    const uint32_t lane = t & 31, warp = t >> 5;
    for (int i = t; i < (256 / 32) * (kMaxLen + 1); i += blockDim.x) (&s_wcnt[0][0])[i] = 0;
    __syncthreads();
    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, l);
    if (lane == (uint32_t)(__ffs(peers) - 1)) s_wcnt[warp][l] = (uint16_t)__popc(peers);
    __syncthreads();
    if (l) {
      uint32_t rank = __popc(peers & ((1u << lane) - 1u));
      for (uint32_t w = 0; w < warp; ++w) rank += s_wcnt[w][l];
      s_sorted[offs[l] + rank] = (uint8_t)t;
    }
  }
  __syncthreads();
  T->sorted[t] = s_sorted[t];
  if (t <= kMaxLen) {
    T->cnt[t] = cnt[t];
    T->offs[t] = offs[t];
    T->first[t] = first[t];
  }
  // lookup table: the code that prefixes the W-bit value v, and the next one
  // when it also fits in the W bits
  const int W = a.lut_bits;
  const uint32_t maxl = s_maxlen;
  auto code_at = [&](uint32_t v, int width, uint32_t& sym) -> uint32_t {
    for (int k = 1; k <= width && k <= (int)maxl; ++k) {
      if (!cnt[k]) continue;
      const uint64_t p = v >> (width - k);
      if (p >= first[k] && p - first[k] < cnt[k]) {
        sym = s_sorted[offs[k] + (uint32_t)(p - first[k])];
        return (uint32_t)k;
      }
    }
    return 0;
  };
  // each thread takes a run of consecutive values, so that the second-level
  // parts can be laid out in value order by one scan
  __shared__ uint8_t s_ext[1 << kLutMaxBits];     // extra bits of an escape value, else 0
  __shared__ uint16_t s_base[1 << kLutMaxBits];   // its first second-level entry
  __shared__ uint32_t s_part[256];
  __shared__ uint32_t s_wpart[256 / 32];
  __shared__ uint32_t s_l2_total;
  const uint32_t nv = 1u << W, per = (nv + blockDim.x - 1) / blockDim.x;
  uint32_t my_l2 = 0;
  // single-symbol table first: value v starts the last code (in canonical
  // order, i.e. by left-justified value) whose W-bit left-justified value is
  // at most v, if v lies inside its range
  __shared__ uint32_t s_lj[256];      // left-justified codes of at most W bits, ascending
  __shared__ uint16_t s_t1[1 << kLutMaxBits];  // symbol | length << 8, 0: no code of <= W bits
  uint32_t nshort = 0;
  for (int k = 1; k <= W && k <= (int)maxl; ++k) nshort += cnt[k];
  if ((uint32_t)t < nshort) {
    const uint32_t k = s_len[s_sorted[t]];  // the length of sorted code t
    s_lj[t] = (uint32_t)((first[k] + (t - offs[k])) << (W - k));
  }
  __syncthreads();
  for (uint32_t v = t; v < nv; v += blockDim.x) {
    uint16_t e1 = 0;
    if (nshort) {
      uint32_t lo_i = 0, hi_i = nshort;  // last i with s_lj[i] <= v
      while (hi_i - lo_i > 1) {
        const uint32_t mid = (lo_i + hi_i) >> 1;
        if (s_lj[mid] <= v) lo_i = mid;
        else hi_i = mid;
      }
      if (s_lj[lo_i] <= v) {
        const uint32_t sym = s_sorted[lo_i], k = s_len[sym];
        if (v - s_lj[lo_i] < (1u << (W - k))) e1 = (uint16_t)(sym | (k << 8));
      }
    }
    s_t1[v] = e1;
  }
  __syncthreads();
  // Mode 0: every W-bit value starts a code of at most W bits.  The counting
  // pass's steps then take all the codes that end within cap bits: 10 when no
  // code is longer (so that three steps follow one buffer fill), else W.
  // (blocks over kFastMaxB only with sub-block offsets: their decoder takes
  // mode 0; the CTA-per-block decoder does not)
  const bool mode0 = s_complete && maxl <= (uint32_t)W && (B <= kFastMaxB || (flags & kFlagSub));
  const bool rep = mode0 && maxl <= 10 && W >= 10;
  const uint32_t cap = rep ? 10u : (uint32_t)W;
  for (uint32_t v = t * per; v < (t + 1) * per && v < nv; ++v) {
    const uint32_t e1 = s_t1[v];
    const uint32_t l0 = e1 >> 8, s0 = e1 & 0xFFu;
    uint32_t e = 0, ext = 0;
    if (rep) {
      // the 10-bit table is built below
    } else if (mode0) {
      uint32_t used = l0, ns = 1;
      for (;;) {
        const uint32_t l = s_t1[(v << used) & (nv - 1)] >> 8;  // >= 1: the code is complete
        if (used + l > cap) break;
        used += l;
        ++ns;
      }
      e = lut0_entry(used, ns, l0, s0);
    } else if (l0) {
      // the next code, when it fits in the W - l0 bits that follow
      const uint32_t e2 = l0 < (uint32_t)W ? s_t1[(v << l0) & (nv - 1)] : 0u;
      const uint32_t l1 = e2 >> 8;
      e = (l1 && l1 <= (uint32_t)W - l0) ? lut_entry(s0, e2 & 0xFFu, 2, l0 + l1, l0)
                                          : lut_entry(s0, 0, 1, l0, l0);
    } else {
      // the longest code (of up to 32 bits) that starts with v
      for (uint32_t k = (uint32_t)W + 1; k <= maxl && k <= 32; ++k) {
        if (!cnt[k]) continue;
        const uint64_t lo_p = first[k] >> (k - W), hi_p = (first[k] + cnt[k] - 1) >> (k - W);
        if (v >= lo_p && v <= hi_p) ext = k - (uint32_t)W;
      }
      my_l2 += ext ? (1u << ext) : 0u;
    }
    s_ext[v] = (uint8_t)ext;
    if (!rep) T->lut[mode0 ? lut0_pos(v) : v] = e;
  }
  if (rep) {
    for (uint32_t u = t; u < 1024u; u += blockDim.x) {
      const uint32_t v = u << (W - 10);  // the W-bit value with u on top
      const uint32_t e1 = s_t1[v];
      const uint32_t l0 = e1 >> 8;       // <= 10: fixed by u
      uint32_t used = l0, ns = 1;
      for (;;) {
        const uint32_t l = s_t1[(v << used) & (nv - 1)] >> 8;
        if (used + l > cap) break;
        used += l;
        ++ns;
      }
      T->lut[u] = lut0_entry(used, ns, l0, e1 & 0xFFu);
    }
  }
  {
    // exclusive scan of the threads' second-level sizes (value order)
    const uint32_t lane = t & 31, warp = t >> 5;
    uint32_t inc = my_l2;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
      if (lane >= (uint32_t)d) inc += o;
    }
    if (lane == 31) s_wpart[warp] = inc;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (uint32_t w = 0; w < blockDim.x / 32; ++w) {
      before += w < warp ? s_wpart[w] : 0u;
      total += s_wpart[w];
    }
    s_part[t] = before + inc - my_l2;
    if (t == 0) s_l2_total = total;
  }
  __syncthreads();
  const uint32_t l2_total = s_l2_total;
  const bool l2_ok = maxl <= 32 && l2_total <= kL2Entries;
  {
    uint32_t at = s_part[t];
    for (uint32_t v = t * per; v < (t + 1) * per && v < nv; ++v) {
      const uint32_t ext = s_ext[v];
      s_base[v] = (uint16_t)(l2_ok ? at : 0u);
      if (ext && l2_ok) {
        T->lut[v] = at | (ext << 18);
        at += 1u << ext;
      }
    }
  }
  __syncthreads();
  if (l2_ok) {
    // entry i belongs to the escape value with the last base <= i
    for (uint32_t i = t; i < l2_total; i += blockDim.x) {
      uint32_t lo_v = 0, hi_v = nv;  // last v with s_base[v] <= i
      while (hi_v - lo_v > 1) {
        const uint32_t mid = (lo_v + hi_v) >> 1;
        if (s_base[mid] <= i) lo_v = mid;
        else hi_v = mid;
      }
      while (lo_v > 0 && s_ext[lo_v] == 0) --lo_v;  // values without a part share the next base
      const uint32_t ext = s_ext[lo_v];
      const uint32_t u = (lo_v << ext) | (i - s_base[lo_v]);
      uint32_t sym = 0;
      const uint32_t k = code_at(u, W + (int)ext, sym);
      T->l2[i] = k ? (uint16_t)(sym | (k << 8)) : (uint16_t)0;
    }
  }
  if (t == 0) T->has_l2 = l2_ok && !mode0 ? 1u : 0u;
  const bool cap_ok = n <= a.out_cap;
  if (t == 0) {
    T->flags = flags;
    T->B = B;
    T->nb = nb;
    T->n = n;
    T->blocks_at = blocks_at;
    T->maxlen = maxl;
    T->lut_bits = (uint32_t)W;
    T->fill_k = mode0 ? (rep ? (maxl <= 8 ? 4u : 3u) : 2u) : 0u;
    T->lut_rep = rep ? 1u : 0u;
    T->pair = rep && maxl <= 5 && S ? 1u : 0u;
    T->sub_S = S;
    T->sub_M = S ? B / S : 0u;
    T->units = S ? nb * (B / S) : 0u;
    *a.out_len = n;
    if (!cap_ok) set_error(a.st, HZ_ERR_CAPACITY, 0x302);
  }
  if (!cap_ok) return;  // uniform
  __syncthreads();
  if (t == 0) {
    uint32_t minl = 0;
    for (int k = kMaxLen; k >= 1; --k)
      if (cnt[k]) minl = (uint32_t)k;
    T->minlen = minl;
    bool chase_ok = true;
    if (!(flags & kFlagIndex)) {
      if (a.seen_no_index) *a.seen_no_index = 1u;
      if (a.defer_chase) {
        T->needs_chase = 1;  // the chase kernel rebuilds the offsets and sets ok
        chase_ok = false;
      } else {
        chase_ok = serial_chase(a, blocks_at, nb);
      }
    }
    if (chase_ok) {
      __threadfence();
      T->ok = 1;
    }
  }
}

// ================================================================ shared pieces
struct CanonTables {
  uint32_t cnt[kMaxLen + 1];
  uint32_t offs[kMaxLen + 1];
  uint64_t first[kMaxLen + 1];
  uint8_t sorted[256];
  uint32_t maxlen, W, flags, B, nb;
  uint64_t n, blocks_at;
};

static __device__ __forceinline__ void load_canon(CanonTables& c, const DecTables* T, int tid, int nt) {
  for (int i = tid; i <= kMaxLen; i += nt) {
    c.cnt[i] = T->cnt[i];
    c.offs[i] = T->offs[i];
    c.first[i] = T->first[i];
  }
  for (int i = tid; i < 256; i += nt) c.sorted[i] = T->sorted[i];
  if (tid == 0) {
    c.maxlen = T->maxlen;
    c.W = T->lut_bits;
    c.flags = T->flags;
    c.B = T->B;
    c.nb = T->nb;
    c.n = T->n;
    c.blocks_at = T->blocks_at;
  }
}

// A code longer than W bits at the top of v64 (canonical first-code search):
// returns length << 8 | symbol, 0 when nothing matches.  (Results come back
// packed, never through a reference, so callers keep them in registers.)
static __device__ __noinline__ uint32_t decode_long(const CanonTables& c, uint64_t v64) {
  for (uint32_t k = c.W + 1; k <= c.maxlen; ++k) {
    const uint32_t n = c.cnt[k];
    if (!n) continue;
    const uint64_t p = v64 >> (64 - k);
    if (p >= c.first[k] && p - c.first[k] < n)
      return (k << 8) | c.sorted[c.offs[k] + (uint32_t)(p - c.first[k])];
  }
  return 0;
}

// Record k: check it and return its payload position.  Shared by both kernels.
struct RecInfo {
  uint64_t rec;
  uint32_t bits, nw, cnt_k;
  bool ok;
};

static __device__ __forceinline__ RecInfo read_record(const DecodeArgs& a, const CanonTables& c,
                                               uint32_t k) {
  RecInfo r;
  const uint32_t* idx = (c.flags & kFlagIndex)
                            ? reinterpret_cast<const uint32_t*>(a.in + kHeaderBytes)
                            : a.chase_index;
  const uint64_t O = idx[k];
  r.rec = c.blocks_at + 4 * O;
  r.bits = 0;
  r.nw = 0;
  bool ok = r.rec + 4 <= a.in_len;
  if (ok) {
    r.bits = *reinterpret_cast<const uint32_t*>(a.in + r.rec);
    r.nw = ceil32(r.bits);
    ok = r.rec + 4 + 4ull * r.nw <= a.in_len;
  }
  if (ok) {
    if (k + 1 < c.nb) ok = (uint64_t)idx[k + 1] == O + 1 + r.nw;
    else ok = r.rec + 4 + 4ull * r.nw == a.in_len;
  }
  const uint64_t lo = (uint64_t)k * c.B;
  r.cnt_k = (uint32_t)((lo + c.B <= c.n) ? c.B : c.n - lo);
  // at least one bit per symbol, at most maxlen bits per symbol
  ok = ok && r.bits >= r.cnt_k && (uint64_t)r.bits <= (uint64_t)r.cnt_k * c.maxlen;
  if (ok && (r.bits & 31)) {
    // padding bits after the last code must be zero
    const uint32_t last = *reinterpret_cast<const uint32_t*>(a.in + r.rec + 4 + 4ull * (r.nw - 1));
    ok = (last & ((1u << (32 - (r.bits & 31))) - 1u)) == 0;
  }
  r.ok = ok;
  return r;
}

// ================================================================ fast kernel
// One warp decodes one block.  Lane i takes the i-th of 32 equal word ranges
// of the payload; ranges of ~2000 symbols make the resynchronisation (tens of
// bits) negligible, and every step after the table lookup is warp-local.
constexpr int kFastThreads = 256;

static __host__ __device__ __forceinline__ bool fast_block_size(uint32_t B) { return B <= kFastMaxB; }


// Per lane, a ring of kRingSlots slots of 32 bytes of its payload range in
// shared memory, fed by cp.async.  Refills happen at warp-uniform points,
// every kRefillSteps decode steps: each lane keeps the slots after the one it
// is reading requested, and makes sure the next one has landed.  A step
// advances at most W <= 12 bits, so kRefillSteps steps read at most six words
// and the window fills in between are plain shared-memory reads.
constexpr uint32_t kSlotWords = 8;
constexpr uint32_t kRingSlots = 4;
constexpr uint32_t kRingWords = kSlotWords * kRingSlots;
constexpr uint32_t kRingStride = kRingWords + 4;  // words between lanes' rings (16-byte aligned)
constexpr uint32_t kRefillSteps = 16;

// Table area: the first-level table (words [0, 2^W)) and the second-level one
// (from word 4096), or the 8 copies of the 10-bit mode-0 table.
constexpr uint32_t kFastLutWords = 8192;
static_assert((1u << kLutMaxBits) + kL2Entries / 2 <= kFastLutWords, "table area");

struct FastShared {
  uint32_t lut[kFastLutWords];
  uint32_t has_l2, fill_k, lut_rep, pair;
  uint32_t sub_S, sub_M, units;  // sub-block offsets (sub_M = 0: none)
  CanonTables c;
  // the launch's arguments (the stream being decoded), for the sub-block
  // decoders: read from here they cost a shared-memory load, where a kernel
  // parameter passed by reference to a separate function lives on the stack
  DecodeArgs args;
};

// The fast decoders' shared state, one per CTA of any kernel that uses it, in
// the launch's dynamic shared memory: the tables, then kRingStride words of
// payload ring per thread, so that the size follows the CTA's width (128 or
// 256 threads).  The block decoders below are separate (not inlined)
// functions, so that each gets its own register allocation; they reach the
// state through this symbol, not a parameter, so that their accesses stay
// shared-memory loads.
constexpr size_t kFastRingOffset = (sizeof(FastShared) + 15) & ~(size_t)15;
static __host__ __device__ constexpr size_t fast_smem_bytes(int threads) {
  return kFastRingOffset + (size_t)threads * kRingStride * 4;
}
extern __shared__ __align__(16) uint8_t g_fast_smem[];
static __device__ __forceinline__ FastShared& fast_sh() {
  return *reinterpret_cast<FastShared*>(g_fast_smem);
}
// the dynamic shared memory as words, and this thread's payload ring as a
// word index into it (32-bit shared-memory addressing, no generic pointer)
static __device__ __forceinline__ uint32_t* fast_smem_words() {
  return reinterpret_cast<uint32_t*>(g_fast_smem);
}
static __device__ __forceinline__ uint32_t fast_ring_word() {
  return (uint32_t)(kFastRingOffset / 4) + threadIdx.x * kRingStride;
}

// The lookup tables of T into shared memory (all threads of the CTA).
// kPair: the caller decodes streams in the pair layout two codes a lookup
// (the single-stream kernel); otherwise their tables load as plain mode-0
// tables (the batched kernel, whose other decode functions keep their
// registers without that path).
template <bool kPair>
static __device__ __forceinline__ void load_fast_tables(FastShared& sh, const DecTables* T,
                                                        int tid, int nt) {
  const int W = (int)T->lut_bits;
  const uint32_t lut_rep = T->lut_rep, pair = kPair ? T->pair : 0u;
  if (lut_rep && pair) {
    // the pair layout: entry u (copy c at word 8u + c) holds the two codes
    // that start the 10-bit value u -- the second is fixed by the 10 - l1 >= 5
    // bits after the first, as no code is longer than 5 bits:
    // l1 + l2 | l1 << 8 | s1 << 16 | s2 << 24
    for (int i = tid; i < (int)kFastLutWords; i += nt) {
      const uint32_t u = (uint32_t)i >> 3;
      const uint32_t e1 = T->lut[u] >> 16;  // l1 | s1 << 8
      const uint32_t l1 = e1 & 31u;
      const uint32_t e2 = T->lut[(u << l1) & 1023u] >> 16;
      sh.lut[i] = (l1 + (e2 & 31u)) | (l1 << 8) | ((e1 >> 8) << 16) | ((e2 >> 8) << 24);
    }
  } else if (lut_rep) {
    for (int i = tid; i < (int)kFastLutWords; i += nt) sh.lut[i] = T->lut[i >> 3];
  } else {
    for (int i = tid; i < (1 << W); i += nt) sh.lut[i] = T->lut[i];
  }
  // (the replicated table fills the whole area; mode 0 needs no second level)
  const uint32_t has_l2 = lut_rep ? 0u : T->has_l2;
  if (has_l2) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(T->l2);
    for (int i = tid; i < (int)(kL2Entries / 2); i += nt) sh.lut[(1 << kLutMaxBits) + i] = src[i];
  }
  if (tid == 0) {
    sh.has_l2 = has_l2;
    sh.fill_k = T->fill_k;
    sh.lut_rep = lut_rep;
    sh.pair = pair;
    sh.sub_S = T->sub_S;
    sh.sub_M = T->sub_M;
    sh.units = T->units;
  }
  load_canon(sh.c, T, tid, nt);
}

// (.cg: the payload goes to shared memory through L2 only; allocating it in L1
// as well costs data-pipe wavefronts and L1 room for nothing, since a lane
// reads its slots once per pass)
static __device__ __forceinline__ void cp_async16(uint32_t smem_addr, const void* gptr, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr), "l"(gptr),
               "r"(bytes)
               : "memory");
}
static __device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// 32 bytes (8 words) to a 32-byte aligned global address in one request
static __device__ __forceinline__ void st_global_v8(uint8_t* p, const uint32_t (&q)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(q[0]),
               "r"(q[1]), "r"(q[2]), "r"(q[3]), "r"(q[4]), "r"(q[5]), "r"(q[6]), "r"(q[7])
               : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The lane's bit reader: a 64-bit buffer (bh:bl) holding the next nb payload
// bits left-aligned (bits below them are zero), topped up one word at a time
// from the lane's ring.  Peeking W bits is one shift and consuming l <= 31
// bits is a funnel shift and a shift; fill() adds a word when nb <= 32, so
// after it nb > 32 and two steps of at most 12 bits can follow before the
// next fill.  Words are indexed from the 16-byte-aligned address at or below
// the payload start.
struct RingWin {
  const uint8_t* abase;  // 16-byte aligned base of the payload's slots
  uint32_t full_slots;   // slots [0, full_slots) lie wholly inside the stream buffer
  uint32_t tail_bytes;   // bytes of slot full_slots inside the buffer
  uint32_t ring_w;       // my ring: its first word's index in the dynamic shared memory
  uint32_t ring_s;       // my ring (shared-memory address)
  uint32_t off_w;        // payload word 0 = aligned word off_w
  uint32_t next_slot;    // next slot index (absolute) to request
  uint32_t rw;           // next aligned word to move into the buffer
  uint32_t nxt;          // that word, read from the ring one fill ahead
  uint32_t bh, bl, nb;
  uint32_t nacc;         // mode 0: nb = (32 * rw + nacc) mod 256
  __device__ __forceinline__ void setup(const uint8_t* payload, const uint8_t* gend) {
    abase = reinterpret_cast<const uint8_t*>(((uintptr_t)payload) & ~(uintptr_t)15);
    off_w = (uint32_t)(payload - abase) >> 2;
    const uint64_t span = (uint64_t)(gend - abase);
    full_slots = (uint32_t)(span >> 5);
    tail_bytes = (uint32_t)(span & 31);
    ring_w = fast_ring_word();
    ring_s = (uint32_t)__cvta_generic_to_shared(fast_smem_words() + ring_w);
  }
  // word i (mod the ring) of my ring
  __device__ __forceinline__ uint32_t ring(uint32_t i) const {
    return fast_smem_words()[ring_w + i % kRingWords];
  }
  __device__ __forceinline__ void request(uint32_t h) {
    const uint8_t* src = abase + 32ull * h;
    const uint32_t dst = ring_s + 32 * (h % kRingSlots);
    if (h < full_slots) {  // a slot wholly inside the stream buffer (all but the last)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16), "l"(src + 16)
                   : "memory");
    } else {  // the buffer's last bytes, zero-filled past its end
      const uint32_t bytes = h == full_slots ? tail_bytes : 0u;
      const uint32_t b0 = bytes < 16 ? bytes : 16u, b1 = bytes > 16 ? bytes - 16 : 0u;
      cp_async16(dst, b0 ? src : abase, b0);
      cp_async16(dst + 16, b1 ? src + 16 : abase, b1);
    }
    cp_async_commit();
  }
  // Start at payload bit `pos`.  kLongSteps (steps of up to 32 bits, decoder
  // mode 1): wait for all three slots requested here, else for the first two.
  template <bool kLongSteps>
  __device__ __forceinline__ void init(uint32_t pos) {
    cp_async_wait<0>();
    const uint32_t A = off_w + (pos >> 5);
    const uint32_t h0 = A / kSlotWords;
    request(h0);
    request(h0 + 1);
    request(h0 + 2);
    next_slot = h0 + 3;
    if (kLongSteps) cp_async_wait<0>();
    else cp_async_wait<1>();
    const uint32_t w0 = ring(A), w1 = ring(A + 1);
    const uint32_t r = pos & 31u;
    bh = __funnelshift_l(w1, w0, r);
    bl = w1 << r;
    nb = 64u - r;
    rw = A + 2;
    nxt = ring(rw);
  }
  // Warp-uniform refill point, every kRefillSteps steps; slots up to rw / 8 + 3
  // are kept requested.  Steps of at most 12 bits read at most 6 words before
  // the next refill point (7 with the word read ahead), all in slots rw / 8
  // and the one after: wait for those.  Steps of up to 32 bits (kLongSteps)
  // read up to 17 (18): wait for every requested slot.
  template <bool kLongSteps>
  __device__ __forceinline__ void refill() {
    const uint32_t cur = rw / kSlotWords;
    while (next_slot <= cur + 3) request(next_slot++);
    if (kLongSteps) cp_async_wait<0>();
    else cp_async_wait<2>();
  }
  // Top the buffer up with the word read ahead, and read the next one: its
  // shared-memory latency then overlaps the steps before the next fill.
  __device__ __forceinline__ void fill() {
    if (nb <= 32u) {
      const uint32_t w = nxt;
      const uint32_t s = 32u - nb;
      uint32_t lo;
      asm("shl.b32 %0, %1, %2;" : "=r"(lo) : "r"(w), "r"(s));  // 0 for s = 32
      bh |= __funnelshift_lc(w, 0u, s);
      bl |= lo;
      nb += 32u;
      ++rw;
      nxt = ring(rw);
    }
  }
  __device__ __forceinline__ uint32_t peek(uint32_t W) const { return bh >> (32u - W); }
  // l <= 31 (a step of at most W bits)
  __device__ __forceinline__ void consume(uint32_t l) {
    bh = __funnelshift_l(bl, bh, l);
    bl <<= l;
    nb -= l;
  }
  // the buffer as 64 bits, MSB first (valid for the next nb bits)
  __device__ __forceinline__ uint64_t peek64() const { return ((uint64_t)bh << 32) | bl; }
  // ---- mode 0.  The bit count is implicit: nb = (32 * rw + nacc) mod 256.  A
  // step consumes the low 5 bits of a table half and subtracts the whole half
  // from nacc; what the half holds above bit 7 drops out of the low byte.
  __device__ __forceinline__ void init0(uint32_t pos) {
    init<false>(pos);
    nacc = nb - 32u * rw;
  }
  __device__ __forceinline__ uint32_t nb0() const { return (32u * rw + nacc) & 255u; }
  // the payload bit position of the next unread bit
  __device__ __forceinline__ uint32_t pos0() const { return 32u * (rw - off_w) - nb0(); }
  // a word into the buffer when it holds at most 32 bits (after it, more than 32)
  // Without a branch: the shifts clamp at 32, so for n > 32 the high part
  // adds nothing and the low part is selected away.
  __device__ __forceinline__ void fill0() {
    const uint32_t n = nb0();
    const bool take = n <= 32u;
    bh |= __funnelshift_rc(nxt, 0u, n);                   // nxt >> n (0 for n >= 32)
    const uint32_t lo = __funnelshift_rc(0u, nxt, n);     // nxt << (32 - n)
    bl |= take ? lo : 0u;
    rw += take ? 1u : 0u;
    nxt = ring(rw);
  }
  __device__ __forceinline__ void take0(uint32_t h) {
    bh = __funnelshift_l(bl, bh, h);
    bl = __funnelshift_l(0u, bl, h);
    nacc -= h;
  }
  // l <= 32 <= nb (a code of up to 32 bits, right after a fill)
  __device__ __forceinline__ void consume_long(uint32_t l) {
    uint32_t lo;
    asm("shl.b32 %0, %1, %2;" : "=r"(lo) : "r"(bl), "r"(l));  // 0 for l = 32
    bh = __funnelshift_lc(bl, bh, l);
    bl = lo;
    nb -= l;
  }
};

// How the fast decoder reads codes.  Mode 0 -- the code is complete and no
// code is longer than the table width W, so every table entry resolves at
// least one symbol: decode_block_warp0, with its own table layout.  The
// general layout (lut_entry) serves decode_block_warp: kMode 1 -- codes of up
// to 32 bits: a longer code is decoded from the window itself (filled before
// every step, so it holds more than 32 bits), through the second-level table
// when there is one; kMode 2 -- any length: a longer code is read straight
// from memory and restarts the window.

// 64-bit window over the payload words read straight from global memory
// (through L1), refilled one word at a time: the fix-up's short walks and
// the rare codes longer than W bits use it.
struct GWin {
  const uint32_t* p;
  uint32_t nw, wi, w0, w1;
  __device__ __forceinline__ uint32_t ld(uint32_t i) const { return i < nw ? __ldg(p + i) : 0u; }
  __device__ __forceinline__ void init(uint32_t pos) {
    wi = pos >> 5;
    w0 = ld(wi);
    w1 = ld(wi + 1);
  }
  __device__ __forceinline__ uint32_t peek(uint32_t pos) const { return __funnelshift_l(w1, w0, pos); }
  // after an advance of at most 32 bits
  __device__ __forceinline__ void step(uint32_t pos) {
    if ((pos >> 5) != wi) {
      w0 = w1;
      w1 = ld(wi + 2);
      ++wi;
    }
  }
  __device__ __forceinline__ uint64_t peek64(uint32_t pos) const {
    return ((uint64_t)__funnelshift_l(w1, w0, pos) << 32) | __funnelshift_l(ld(wi + 2), w1, pos);
  }
  // 64 bits at any position, straight from memory (for the rare long codes)
  __device__ __forceinline__ uint64_t peek64_at(uint32_t pos) const {
    const uint32_t i = pos >> 5;
    const uint32_t a0 = ld(i), a1 = ld(i + 1), a2 = ld(i + 2);
    return ((uint64_t)__funnelshift_l(a1, a0, pos) << 32) | __funnelshift_l(a2, a1, pos);
  }
};

// One symbol at pos: length << 8 | symbol (0 when no code matches).
static __device__ __forceinline__ uint32_t one_symbol(const FastShared& sh, const GWin& w, uint32_t pos,
                                               uint32_t W) {
  const uint32_t e = sh.lut[w.peek(pos) >> (32 - W)];
  const uint32_t l0 = e_l0(e);
  if (l0) return (l0 << 8) | (e & 0xFFu);
  return decode_long(sh.c, w.peek64(pos));
}

// Decode one symbol, advance, and report a miss (no code) through `bad`.
static __device__ __forceinline__ uint32_t take_symbol(const FastShared& sh, GWin& w, uint32_t& pos,
                                                uint32_t W, bool& bad) {
  const uint32_t ls = one_symbol(sh, w, pos, W);
  const uint32_t l = ls >> 8;
  bad |= l == 0;
  const uint32_t adv = l ? l : 1u;
  pos += adv;
  if (adv <= 32) w.step(pos);
  else w.init(pos);
  return ls & 0xFFu;
}

// A code longer than W bits (kMode 1) from the window's first 64 bits, given
// its table entry e: length << 8 | symbol, 0 when no code matches.
static __device__ __forceinline__ uint32_t long_code(const FastShared& sh, uint32_t e,
                                                     uint64_t v64, uint32_t W) {
  if (sh.has_l2) {
    const uint32_t ext = e_nbits(e);
    if (!ext) return 0u;  // no code starts with these W bits
    const uint16_t* l2 = reinterpret_cast<const uint16_t*>(sh.lut + (1 << kLutMaxBits));
    return l2[(e & 0xFFFFu) + (uint32_t)((v64 << W) >> (64 - ext))];
  }
  return decode_long(sh.c, v64);
}

// Decode one symbol from the ring window and advance; the window holds at
// least W bits (more than 32 for kMode 1).  In kMode 2 a long code, read
// straight from memory, restarts the window (which waits for the ring and
// leaves it full).
template <int kMode>
__device__ __forceinline__ uint32_t ring_step(const FastShared& sh, RingWin& w, uint32_t& pos,
                                              uint32_t W, const GWin& g, bool& bad) {
  static_assert(kMode == 1 || kMode == 2, "mode 0 has its own decoder");
  const uint32_t e = sh.lut[w.peek(W)];
  const uint32_t l0 = e_l0(e);
  if (l0) {
    pos += l0;
    w.consume(l0);
    return e & 0xFFu;
  }
  if (kMode == 1) {
    const uint32_t ls = long_code(sh, e, w.peek64(), W);
    const uint32_t l = ls >> 8;
    bad |= l == 0;
    const uint32_t adv = l ? l : 1u;
    pos += adv;
    w.consume_long(adv);
    return ls & 0xFFu;
  }
  const uint32_t ls = decode_long(sh.c, g.peek64_at(pos));
  const uint32_t l = ls >> 8;
  bad |= l == 0;
  pos += l ? l : 1u;
  w.template init<false>(pos);  // kMode 2: steps through the window stay within W bits
  return ls & 0xFFu;
}

// The same, filling the window first.
template <int kMode>
__device__ __forceinline__ uint32_t ring_take(const FastShared& sh, RingWin& w, uint32_t& pos,
                                              uint32_t W, const GWin& g, bool& bad) {
  w.fill();
  return ring_step<kMode>(sh, w, pos, W, g, bad);
}

template <int kMode>
__device__ __noinline__ void decode_block_warp(const DecodeArgs& a, uint32_t k) {
  FastShared& sh = fast_sh();
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t W = sh.c.W;
  RecInfo r;
  if (lane == 0) r = read_record(a, sh.c, k);
  r.rec = __shfl_sync(0xFFFFFFFFu, r.rec, 0);
  r.bits = __shfl_sync(0xFFFFFFFFu, r.bits, 0);
  r.nw = __shfl_sync(0xFFFFFFFFu, r.nw, 0);
  r.cnt_k = __shfl_sync(0xFFFFFFFFu, r.cnt_k, 0);
  r.ok = __shfl_sync(0xFFFFFFFFu, (int)r.ok, 0);
  if (!r.ok) {
    if (lane == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x320);
    return;
  }
  const uint32_t bits = r.bits, nw = r.nw;
  const uint8_t* payload = a.in + r.rec + 4;
  GWin g;  // plain reader: long codes and the fix-up
  g.p = reinterpret_cast<const uint32_t*>(payload);
  g.nw = nw;
  RingWin w;
  w.setup(payload, a.in + a.in_len);
  const uint32_t Lw = (nw + 31) / 32;
  const uint32_t L = Lw * 32;
  const uint32_t nsub = (bits + L - 1) / L;
  const bool active = lane < nsub;
  const uint32_t my_start = lane * L;
  const uint32_t my_end = active ? min(my_start + L, bits) : 0u;

  // ---- pass 1: speculative decode of my range, counting symbols
  uint32_t start = my_start, exit_ = my_start, count = 0;
  {
    uint32_t pos = my_start, c = 0;
    if (active) w.template init<kMode == 1>(pos);
    bool dummy = false;
    while (__any_sync(0xFFFFFFFFu, active && pos + W <= my_end)) {
      if (active) w.template refill<kMode == 1>();
#pragma unroll 2
      for (uint32_t s = 0; s < kRefillSteps; s += 2) {
        w.fill();  // two steps of at most W <= 12 bits follow
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          if (kMode == 1 && t == 1) w.fill();  // a long code needs more than 32 bits
          if (active && pos + W <= my_end) {
            const uint32_t e = sh.lut[w.peek(W)];
            const uint32_t ns = e_ns(e);
            if (kMode == 1 && ns == 0) {  // a long code, or no code at all on a wrong path
              const uint32_t l = long_code(sh, e, w.peek64(), W) >> 8;
              const uint32_t adv = l ? l : 1u;
              pos += adv;
              ++c;
              w.consume_long(adv);
            } else if (kMode == 2 && ns == 0) {
              const uint32_t l = decode_long(sh.c, g.peek64_at(pos)) >> 8;
              pos += l ? l : 1u;
              ++c;
              w.template init<kMode == 1>(pos);
            } else {
              const uint32_t nbits = e_nbits(e);
              pos += nbits;
              c += ns;
              w.consume(nbits);
            }
          }
        }
      }
    }
    if (active) {
      w.template refill<kMode == 1>();
      while (pos < my_end) {
        ring_take<kMode>(sh, w, pos, W, g, dummy);
        ++c;
      }
      exit_ = pos;
      count = c;
    }
  }
  // ---- fix-up: restart each range at its left neighbour's exit until all agree
  for (uint32_t round = 0; round <= 32; ++round) {
    const uint32_t want = __shfl_up_sync(0xFFFFFFFFu, exit_, 1);
    const bool mismatch = active && lane > 0 && want != start;
    if (!__any_sync(0xFFFFFFFFu, mismatch)) break;
    if (mismatch) {
      // advance the new (a) and old (b) decodes, the one behind first, until they meet
      uint32_t pa = want, pb = start, ca = 0, cb = 0;
      GWin wa = g, wb = g;
      wa.init(pa);
      wb.init(pb);
      bool dummy = false;
      while (pa != pb && (pa < my_end || pb < my_end)) {
        if (pa < pb) {
          take_symbol(sh, wa, pa, W, dummy);
          ++ca;
        } else {
          take_symbol(sh, wb, pb, W, dummy);
          ++cb;
        }
      }
      if (pa == pb) {
        count = count - cb + ca;
      } else {
        exit_ = pa;
        count = ca;
      }
      start = want;
    }
  }
  // ---- exclusive scan of the counts
  const uint32_t v = active ? count : 0u;
  uint32_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane >= (uint32_t)d) inc += o;
  }
  const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
  const uint32_t last_exit = __shfl_sync(0xFFFFFFFFu, exit_, nsub - 1);
  if (total != r.cnt_k || last_exit != bits) {
    if (lane == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x321);
    cp_async_wait<0>();
    return;  // uniform
  }
  // ---- pass 2: decode from the true boundary and store the symbols
  bool bad = false;
  {
    uint32_t pos = start, rem = active ? v : 0u;
    uint8_t* dst = a.out + (uint64_t)k * sh.c.B + (inc - v);
    if (rem) {
      w.template init<kMode == 1>(pos);
      // bytes up to a 16-byte boundary (at most 15 steps: within the slots init awaited)
      while (rem && (((uintptr_t)dst) & 15)) {
        *dst++ = (uint8_t)ring_take<kMode>(sh, w, pos, W, g, bad);
        --rem;
      }
    }
    // 16 symbols per 16-byte store, one refill point per 16 symbols
    while (__any_sync(0xFFFFFFFFu, rem >= 16)) {
      if (rem >= 16) {
        w.template refill<kMode == 1>();
        uint32_t q[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          uint32_t word = 0;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            w.fill();
            word |= ring_step<kMode>(sh, w, pos, W, g, bad) << (8 * b);
          }
          q[j] = word;
        }
        *reinterpret_cast<uint4*>(dst) = make_uint4(q[0], q[1], q[2], q[3]);
        dst += 16;
        rem -= 16;
      }
    }
    if (rem) {
      w.template refill<kMode == 1>();
      while (rem) {
        *dst++ = (uint8_t)ring_take<kMode>(sh, w, pos, W, g, bad);
        --rem;
      }
    }
    if (active && v) bad |= pos != exit_;
  }
  cp_async_wait<0>();  // nothing of this block may land in the ring after we leave
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x322);
}

// ---------------------------------------------------------------- mode 0
// The same three phases as decode_block_warp, for codes that all fit the
// table (every W-bit value starts one) and the mode-0 table layout.  The
// counting pass takes every code that ends within cap bits in one step (cap:
// 10 (or W if smaller) and K1 = 3 when no code is longer, else W and K1 = 2)
// and fills the buffer every K1 steps; the output
// pass takes one code per step and fills every K2 steps (codes of at most
// 32 / K2 bits).  A fill leaves more than 32 bits in the buffer as long as it
// held at least one, so K steps of at most c bits with K * c <= 32 keep at
// least c bits in it for every step's lookup (an entry depends on its first
// c bits only).  While a lane is more than a refill period's worth of steps
// from the end of its range, its steps run without a bounds check.
// The 16-bit index of the entry's low half for a bit buffer whose top 32 bits
// are `top` (c2: twice the lane's copy, for the replicated table).
template <bool kRep>
static __device__ __forceinline__ uint32_t lut0_at(uint32_t top, uint32_t sW, uint32_t c2) {
  if (kRep) return ((top >> 22) << 4) | c2;  // word 8u + c
  return lut0_pos(top >> sW) << 1;
}
static __device__ __forceinline__ uint32_t lut0_lo(const FastShared& sh, uint32_t i) {
  return reinterpret_cast<const uint16_t*>(sh.lut)[i];
}
static __device__ __forceinline__ uint32_t lut0_hi(const FastShared& sh, uint32_t i) {
  return reinterpret_cast<const uint16_t*>(sh.lut)[i + 1];
}
// one code from the plain reader (the fix-up): advance pos by its length
template <bool kRep>
static __device__ __forceinline__ void skip_symbol0(const FastShared& sh, GWin& g, uint32_t& pos,
                                                    uint32_t sW, uint32_t c2) {
  const uint32_t l = lut0_hi(sh, lut0_at<kRep>(g.peek(pos), sW, c2)) & 31u;
  pos += l ? l : 1u;  // >= 1 in a mode-0 table; never stall on a bad one
  g.step(pos);
}

template <int K1, int K2, bool kRep>
__device__ __noinline__ void decode_block_warp0(const DecodeArgs& a, uint32_t k) {
  FastShared& sh = fast_sh();
  constexpr uint32_t kCap = K1 == 3 ? 10u : (uint32_t)kLutMaxBits;  // bits per counting step
  constexpr uint32_t kG1 = K1 == 3 ? 15u : 16u;                      // counting steps per refill
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t sW = 32u - sh.c.W;
  const uint32_t c2 = (lane & 7u) << 1;
  RecInfo r;
  if (lane == 0) r = read_record(a, sh.c, k);
  r.rec = __shfl_sync(0xFFFFFFFFu, r.rec, 0);
  r.bits = __shfl_sync(0xFFFFFFFFu, r.bits, 0);
  r.nw = __shfl_sync(0xFFFFFFFFu, r.nw, 0);
  r.cnt_k = __shfl_sync(0xFFFFFFFFu, r.cnt_k, 0);
  r.ok = __shfl_sync(0xFFFFFFFFu, (int)r.ok, 0);
  if (!r.ok) {
    if (lane == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x320);
    return;
  }
  const uint32_t bits = r.bits, nw = r.nw;
  const uint8_t* payload = a.in + r.rec + 4;
  GWin g;
  g.p = reinterpret_cast<const uint32_t*>(payload);
  g.nw = nw;
  RingWin w;
  w.setup(payload, a.in + a.in_len);
  const uint32_t Lw = (nw + 31) / 32;
  const uint32_t L = Lw * 32;
  const uint32_t nsub = (bits + L - 1) / L;
  const bool active = lane < nsub;
  const uint32_t my_start = lane * L;
  const uint32_t my_end = active ? min(my_start + L, bits) : 0u;

  // ---- pass 1: speculative count of the codes that start in my range
  uint32_t start = my_start, exit_ = my_start, count = 0;
  bool stalled = false;
  if (active) {
    w.init0(my_start);
    const uint32_t nacc0 = w.nacc;
    // Every step of a mode-0 table takes at least one bit, so a range of L
    // bits needs at most L steps; the budget only guards against a bad table.
    uint32_t budget = my_end - my_start + 2 * kCap;
    // far from the end: kG1 steps of at most kCap bits, unchecked
    while (w.pos0() + kG1 * kCap <= my_end && budget >= kG1) {
      budget -= kG1;
      w.refill<false>();
#pragma unroll
      for (uint32_t s = 0; s < kG1; ++s) {
        if (s % K1 == 0) w.fill0();
        w.take0(lut0_lo(sh, lut0_at<kRep>(w.bh, sW, c2)));
      }
    }
    // near it: steps while all their codes start before the end
    w.refill<false>();
    for (; budget; --budget) {
      w.fill0();
      if (w.pos0() + kCap > my_end) break;
      w.take0(lut0_lo(sh, lut0_at<kRep>(w.bh, sW, c2)));
    }
    // then one code at a time (counted as 256 in nacc, like a step's count)
    uint32_t pos = w.pos0();
    for (; pos < my_end && budget; --budget) {
      w.fill0();
      const uint32_t l = lut0_hi(sh, lut0_at<kRep>(w.bh, sW, c2)) & 31u;
      w.take0(l | 256u);
      pos += l;
    }
    stalled = pos < my_end;
    exit_ = pos;
    count = ((nacc0 - w.nacc) - (pos - my_start)) >> 8;
  }
  if (__any_sync(0xFFFFFFFFu, stalled)) {
    if (lane == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x323);
    cp_async_wait<0>();
    return;  // uniform
  }
  // ---- fix-up: restart each range at its left neighbour's exit until all agree
  for (uint32_t round = 0; round <= 32; ++round) {
    const uint32_t want = __shfl_up_sync(0xFFFFFFFFu, exit_, 1);
    const bool mismatch = active && lane > 0 && want != start;
    if (!__any_sync(0xFFFFFFFFu, mismatch)) break;
    if (mismatch) {
      uint32_t pa = want, pb = start, ca = 0, cb = 0;
      GWin wa = g, wb = g;
      wa.init(pa);
      wb.init(pb);
      while (pa != pb && (pa < my_end || pb < my_end)) {
        if (pa < pb) {
          skip_symbol0<kRep>(sh, wa, pa, sW, c2);
          ++ca;
        } else {
          skip_symbol0<kRep>(sh, wb, pb, sW, c2);
          ++cb;
        }
      }
      if (pa == pb) {
        count = count - cb + ca;
      } else {
        exit_ = pa;
        count = ca;
      }
      start = want;
    }
  }
  // ---- exclusive scan of the counts
  const uint32_t v = active ? count : 0u;
  uint32_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane >= (uint32_t)d) inc += o;
  }
  const uint32_t total = __shfl_sync(0xFFFFFFFFu, inc, 31);
  const uint32_t last_exit = __shfl_sync(0xFFFFFFFFu, exit_, nsub - 1);
  if (total != r.cnt_k || last_exit != bits) {
    if (lane == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x321);
    cp_async_wait<0>();
    return;  // uniform
  }
  // ---- pass 2: decode from the true boundary and store the symbols
  bool bad = false;
  {
    uint32_t rem = active ? v : 0u;
    uint8_t* dst = a.out + (uint64_t)k * sh.c.B + (inc - v);
    auto step = [&]() -> uint32_t {
      const uint32_t h = lut0_hi(sh, lut0_at<kRep>(w.bh, sW, c2));
      w.take0(h);
      return h;
    };
    if (rem) w.init0(start);
    if (sh.c.B >= 65536) {  // uniform: long ranges (2048+ symbols a lane)
      // bytes up to a 32-byte boundary, a refill point every 8 (a step reads at
      // most 12 bits: 8 steps stay within the slots a refill awaits)
      while (rem && (((uintptr_t)dst) & 31)) {
        if ((((uintptr_t)dst) & 7) == 0) w.refill<false>();
        w.fill0();
        *dst++ = (uint8_t)(step() >> 8);
        --rem;
      }
      // 32 symbols per 32-byte store (one whole sector per write request), a
      // refill point every 16 steps, a fill every K2 steps counted over the 32;
      // four symbols into a word with three byte permutes
      while (__any_sync(0xFFFFFFFFu, rem >= 32)) {
        if (rem >= 32) {
          uint32_t q[8];
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            w.refill<false>();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              uint32_t h[4];
#pragma unroll
              for (int b = 0; b < 4; ++b) {
                if ((16 * half + 4 * j + b) % K2 == 0) w.fill0();
                h[b] = step();
              }
              q[4 * half + j] = __byte_perm(__byte_perm(h[0], h[1], 0x0051u),
                                            __byte_perm(h[2], h[3], 0x0051u), 0x5410u);
            }
          }
          st_global_v8(dst, q);
          dst += 32;
          rem -= 32;
        }
      }
    } else {  // short ranges: 16-byte stores, fewer single bytes at the ends
      // bytes up to a 16-byte boundary (at most 15 steps: within the slots init awaited)
      while (rem && (((uintptr_t)dst) & 15)) {
        w.fill0();
        *dst++ = (uint8_t)(step() >> 8);
        --rem;
      }
      // 16 symbols per 16-byte store, one refill point per 16 symbols
      while (__any_sync(0xFFFFFFFFu, rem >= 16)) {
        if (rem >= 16) {
          w.refill<false>();
          uint32_t q[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            uint32_t h[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              if ((4 * j + b) % K2 == 0) w.fill0();
              h[b] = step();
            }
            q[j] = __byte_perm(__byte_perm(h[0], h[1], 0x0051u),
                               __byte_perm(h[2], h[3], 0x0051u), 0x5410u);
          }
          *reinterpret_cast<uint4*>(dst) = make_uint4(q[0], q[1], q[2], q[3]);
          dst += 16;
          rem -= 16;
        }
      }
    }
    for (uint32_t t = 0; rem; ++t) {  // a refill point every 8
      if ((t & 7) == 0) w.refill<false>();
      w.fill0();
      *dst++ = (uint8_t)(step() >> 8);
      --rem;
    }
    if (active && v) bad = w.pos0() != exit_;
  }
  cp_async_wait<0>();  // nothing of this block may land in the ring after we leave
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x322);
}

// The decoder mode for the tables (see RingWin), and one block in that mode.
static __device__ __forceinline__ int fast_mode(const DecTables* T, const CanonTables& c) {
  if (T->fill_k) return 0;  // every code fits the table: no escapes
  return c.maxlen <= 32 ? 1 : 2;
}

static __device__ __forceinline__ void decode_block_fast(const DecodeArgs& a,
                                                         uint32_t k, int mode) {
  if (mode == 0) {
    if (fast_sh().fill_k == 4) decode_block_warp0<3, 4, true>(a, k);
    else if (fast_sh().fill_k == 3) decode_block_warp0<3, 3, true>(a, k);
    else decode_block_warp0<2, 2, false>(a, k);
  } else if (mode == 1) decode_block_warp<1>(a, k);
  else decode_block_warp<2>(a, k);
}

// ================================================================ sub-block decoder
// Streams with sub-block offsets (flags bit 1): the stored offsets give the
// payload bit of the code of every S-th symbol of a block, so a lane decodes
// the S symbols of one sub-block from a known bit straight into their place
// in the output -- one pass over the payload, with no speculative counting,
// no fix-up and no scan.  Unit u = k * M + j is symbols [j*S, min((j+1)*S,
// cnt_k)) of block k (units past the last block's end hold no symbol); a warp
// takes 32 consecutive units, lane l the unit u0 + l.
struct SubRange {
  const uint8_t* payload;  // the unit's record payload
  uint32_t nw;             // the record's payload words
  uint32_t start, end;     // payload bits [start, end) hold the unit's codes
  uint32_t count;          // its symbols
  uint64_t out_at;         // output index of its first symbol
  bool ok;
};

// Unit u's range, checked: the record itself (read_record: index, delimiter,
// padding), offsets in order and inside the record, at least one and at most
// maxlen bits per symbol, the block's last unit ending at bits_k, and the
// entries past the block's last symbol equal to bits_k (each entry is the
// start of exactly one unit, so every entry gets checked).
static __device__ __forceinline__ SubRange sub_range(const DecodeArgs& a, const CanonTables& c,
                                                     uint32_t S, uint32_t M, uint32_t u) {
  SubRange r;
  const uint32_t k = u / M, j = u - k * M;
  const RecInfo rec = read_record(a, c, k);
  const uint32_t* e =
      reinterpret_cast<const uint32_t*>(a.in + sub_entries_at(c.nb)) + (uint64_t)k * (M - 1);
  const uint32_t lo = j * S;
  r.payload = a.in + rec.rec + 4;
  r.nw = rec.nw;
  r.count = lo < rec.cnt_k ? min(S, rec.cnt_k - lo) : 0u;
  r.start = j ? e[j - 1] : 0u;
  r.end = j + 1 < M ? e[j] : rec.bits;
  r.out_at = (uint64_t)k * c.B + lo;
  bool ok = rec.ok && r.start <= r.end && r.end <= rec.bits;
  if (r.count == 0) {
    ok = ok && r.start == rec.bits;
  } else {
    ok = ok && r.end - r.start >= r.count &&
         (uint64_t)(r.end - r.start) <= (uint64_t)r.count * c.maxlen;
    if (lo + r.count == rec.cnt_k) ok = ok && r.end == rec.bits;
  }
  r.ok = ok;
  return r;
}

// Mode 0 (see decode_block_warp0): one code per step from the mode-0 table,
// a buffer fill every K2 steps, 16 symbols per 16-byte store.  Inlined into
// the single-stream kernel (no call: its registers are the kernel's own), a
// separate function in the batched one.
template <int K2, bool kRep>
__device__ __forceinline__ void decode_units0_body(uint32_t u0, uint32_t u_end) {
  FastShared& sh = fast_sh();
  const DecodeArgs& a = sh.args;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t sW = 32u - sh.c.W;
  const uint32_t c2 = (lane & 7u) << 1;
  const uint32_t u = u0 + lane;
  SubRange r;
  r.ok = true;
  r.count = 0;
  r.out_at = 0;
  if (u < u_end) r = sub_range(a, sh.c, sh.sub_S, sh.sub_M, u);
  bool bad = !r.ok;
  uint32_t rem = r.ok ? r.count : 0u;
  uint8_t* dst = a.out + r.out_at;
  RingWin w;
  // one code: its symbol (the high half's byte 1) and the buffer advanced
  auto step = [&]() -> uint32_t {
    const uint32_t h = lut0_hi(sh, lut0_at<kRep>(w.bh, sW, c2));
    w.take0(h);
    return h;
  };
  if (rem) {
    w.setup(r.payload, a.in + a.in_len);
    w.init0(r.start);
    // bytes up to a 32-byte boundary, a refill point every 8 (a step reads at
    // most 12 bits: 8 steps stay within the slots a refill awaits)
    while (rem && (((uintptr_t)dst) & 31)) {
      if ((((uintptr_t)dst) & 7) == 0) w.refill<false>();
      w.fill0();
      *dst++ = (uint8_t)(step() >> 8);
      --rem;
    }
  }
  // 32 symbols per 32-byte store (one whole sector per write request), a
  // refill point every 16 steps, a fill every K2 steps counted over the 32
  // (the last fill of a group is at most K2 - 1 steps before the next
  // group's first)
  while (__any_sync(0xFFFFFFFFu, rem >= 32)) {
    if (rem >= 32) {
      uint32_t q[8];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        w.refill<false>();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          uint32_t h[4];
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            if ((16 * half + 4 * j + b) % K2 == 0) w.fill0();
            h[b] = step();
          }
          // the four symbols (byte 1 of each h) into one word, two at a time
          q[4 * half + j] = __byte_perm(__byte_perm(h[0], h[1], 0x0051u),
                                        __byte_perm(h[2], h[3], 0x0051u), 0x5410u);
        }
      }
      st_global_v8(dst, q);
      dst += 32;
      rem -= 32;
    }
  }
  if (rem) {
    while (rem) {
      if ((rem & 7) == 0) w.refill<false>();
      w.fill0();
      *dst++ = (uint8_t)(step() >> 8);
      --rem;
    }
  }
  if (r.ok && r.count) bad = w.pos0() != r.end;
  cp_async_wait<0>();  // nothing of this warp's units may land in the ring after we leave
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x330);
}

// Mode 0 with the pair layout (no code longer than 5 bits): two codes per
// lookup in the 32-symbol groups -- a step consumes at most 10 bits, so a
// fill every 3 steps, counted over the group's 16 steps; the group's words
// take one byte permute each (bytes 2 and 3 of two entries).  The bytes before
// the first 32-byte boundary and after the last group take one code a step
// (the entry's first code, its length in bits 8-12).
static __device__ __forceinline__ void decode_units0_pair_body(uint32_t u0, uint32_t u_end) {
  FastShared& sh = fast_sh();
  const DecodeArgs& a = sh.args;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t cw = lane & 7u;  // the lane's copy of the table
  const uint32_t u = u0 + lane;
  SubRange r;
  r.ok = true;
  r.count = 0;
  r.out_at = 0;
  if (u < u_end) r = sub_range(a, sh.c, sh.sub_S, sh.sub_M, u);
  bool bad = !r.ok;
  uint32_t rem = r.ok ? r.count : 0u;
  uint8_t* dst = a.out + r.out_at;
  RingWin w;
  auto entry = [&]() -> uint32_t { return sh.lut[((w.bh >> 22) << 3) | cw]; };
  // one code: its symbol, the buffer advanced by its length
  auto step1 = [&]() -> uint8_t {
    const uint32_t h = entry();
    w.take0((h >> 8) & 31u);
    return (uint8_t)(h >> 16);
  };
  // two codes: the entry (symbols in bytes 2 and 3), the buffer advanced by
  // both lengths (bits 8 and up drop out of the bit count's low byte)
  auto step2 = [&]() -> uint32_t {
    const uint32_t h = entry();
    w.take0(h);
    return h;
  };
  if (rem) {
    w.setup(r.payload, a.in + a.in_len);
    w.init0(r.start);
    while (rem && (((uintptr_t)dst) & 31)) {
      if ((((uintptr_t)dst) & 7) == 0) w.refill<false>();
      w.fill0();
      *dst++ = step1();
      --rem;
    }
  }
  while (__any_sync(0xFFFFFFFFu, rem >= 32)) {
    if (rem >= 32) {
      uint32_t q[8];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        w.refill<false>();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int s = 8 * half + 2 * j;  // the group's step
          if (s % 3 == 0) w.fill0();
          const uint32_t ha = step2();
          if ((s + 1) % 3 == 0) w.fill0();
          const uint32_t hb = step2();
          q[4 * half + j] = __byte_perm(ha, hb, 0x7632u);
        }
      }
      st_global_v8(dst, q);
      dst += 32;
      rem -= 32;
    }
  }
  while (rem) {
    if ((rem & 7) == 0) w.refill<false>();
    w.fill0();
    *dst++ = step1();
    --rem;
  }
  if (r.ok && r.count) bad = w.pos0() != r.end;
  cp_async_wait<0>();  // nothing of this warp's units may land in the ring after we leave
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x332);
}

template <int K2, bool kRep>
__device__ __noinline__ void decode_units_warp0(uint32_t u0, uint32_t u_end) {
  decode_units0_body<K2, kRep>(u0, u_end);
}

// Modes 1 and 2 (see decode_block_warp): one code per step from the general
// table; longer codes through the second-level table or from memory.
template <int kMode>
__device__ __noinline__ void decode_units_warp(uint32_t u0, uint32_t u_end) {
  FastShared& sh = fast_sh();
  const DecodeArgs& a = sh.args;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t W = sh.c.W;
  const uint32_t u = u0 + lane;
  SubRange r;
  r.ok = true;
  r.count = 0;
  r.out_at = 0;
  r.payload = a.in;
  r.nw = 0;
  r.start = 0;
  if (u < u_end) r = sub_range(a, sh.c, sh.sub_S, sh.sub_M, u);
  bool bad = !r.ok;
  uint32_t rem = r.ok ? r.count : 0u;
  uint32_t pos = r.start;
  uint8_t* dst = a.out + r.out_at;
  GWin g;  // plain reader for codes longer than the table (mode 2)
  g.p = reinterpret_cast<const uint32_t*>(r.payload);
  g.nw = r.nw;
  RingWin w;
  if (rem) {
    w.setup(r.payload, a.in + a.in_len);
    w.template init<kMode == 1>(pos);
    while (rem && (((uintptr_t)dst) & 15)) {
      *dst++ = (uint8_t)ring_take<kMode>(sh, w, pos, W, g, bad);
      --rem;
    }
  }
  while (__any_sync(0xFFFFFFFFu, rem >= 16)) {
    if (rem >= 16) {
      w.template refill<kMode == 1>();
      uint32_t q[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        uint32_t word = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          w.fill();
          word |= ring_step<kMode>(sh, w, pos, W, g, bad) << (8 * b);
        }
        q[j] = word;
      }
      *reinterpret_cast<uint4*>(dst) = make_uint4(q[0], q[1], q[2], q[3]);
      dst += 16;
      rem -= 16;
    }
  }
  if (rem) {
    w.template refill<kMode == 1>();
    while (rem) {
      *dst++ = (uint8_t)ring_take<kMode>(sh, w, pos, W, g, bad);
      --rem;
    }
  }
  if (r.ok && r.count) bad |= pos != r.end;
  cp_async_wait<0>();
  if (__any_sync(0xFFFFFFFFu, bad) && lane == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x331);
}

// Units [u0, u0 + 32) of the stream whose arguments are in fast_sh().args,
// capped at u_end, in the stream's mode (not the pair layout: the
// single-stream kernel decodes that inline).
static __device__ __forceinline__ void decode_units_fast(uint32_t u0, uint32_t u_end, int mode) {
  if (mode == 0) {
    if (fast_sh().fill_k == 4) decode_units_warp0<4, true>(u0, u_end);
    else if (fast_sh().fill_k == 3) decode_units_warp0<3, true>(u0, u_end);
    else decode_units_warp0<2, false>(u0, u_end);
  } else if (mode == 1) decode_units_warp<1>(u0, u_end);
  else decode_units_warp<2>(u0, u_end);
}

// ================================================================ generic kernel
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

struct GenShared {
  uint32_t lut[1 << kLutMaxBits];
  CanonTables c;
};

static __device__ __forceinline__ uint32_t generic_one(const GenShared& sh, const BitReader& br,
                                                uint32_t pos, uint32_t& sym) {
  const uint32_t e = sh.lut[br.peek32(pos) >> (32 - sh.c.W)];
  const uint32_t l0 = e_l0(e);
  if (l0) {
    sym = e & 0xFFu;
    return l0;
  }
  const uint32_t ls = decode_long(sh.c, br.peek64(pos));
  sym = ls & 0xFFu;
  return ls >> 8;
}

template <int NT>
struct GenBlockShared {
  uint32_t start[NT], exit[NT], count[NT];
  uint32_t warp_tot[NT / 32];
  RecInfo r;
  int ok;
};

template <int NT>
__device__ void decode_block_generic(const DecodeArgs& a, const GenShared& sh,
                                     GenBlockShared<NT>& bs, uint32_t k) {
  const int t = threadIdx.x;
  __syncthreads();  // every thread is done with the previous block's shared state
  if (t == 0) {
    bs.r = read_record(a, sh.c, k);
    bs.ok = bs.r.ok ? 1 : 0;
    if (!bs.r.ok) set_error(a.st, HZ_ERR_CORRUPT, 0x310);
  }
  __syncthreads();
  if (!bs.ok) return;  // uniform
  const uint32_t bits = bs.r.bits;
  const uint32_t* payload = reinterpret_cast<const uint32_t*>(a.in + bs.r.rec + 4);
  const uint32_t nw = bs.r.nw;
  uint32_t L = (bits + NT - 1) / NT;
  L = L < 32 ? 32 : (L + 31) & ~31u;
  const uint32_t nsub = (bits + L - 1) / L;
  const bool active = (uint32_t)t < nsub;
  const uint32_t my_end = active ? min(((uint32_t)t + 1) * L, bits) : 0u;

  if (active) {
    uint32_t pos = (uint32_t)t * L, c = 0, sym;
    BitReader br;
    br.init(payload, nw, pos);
    while (pos < my_end) {
      const uint32_t l = generic_one(sh, br, pos, sym);
      pos += l ? l : 1u;
      br.seek(pos);
      ++c;
    }
    bs.start[t] = (uint32_t)t * L;
    bs.exit[t] = pos;
    bs.count[t] = c;
  }
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
          const uint32_t l = generic_one(sh, ra, pa, sym);
          pa += l ? l : 1u;
          ra.seek(pa);
          ++ca;
        } else {
          const uint32_t l = generic_one(sh, rb, pb, sym);
          pb += l ? l : 1u;
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
  const int lane = t & 31, warp = t >> 5;
  const uint32_t v = active ? bs.count[t] : 0u;
  uint32_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) bs.warp_tot[warp] = inc;
  __syncthreads();
  uint32_t wpre = 0, total = 0;
  for (int w = 0; w < NT / 32; ++w) {
    wpre += w < warp ? bs.warp_tot[w] : 0u;
    total += bs.warp_tot[w];
  }
  const uint32_t my_off = wpre + inc - v;
  const bool bad = (uint32_t)t == nsub - 1 && (total != bs.r.cnt_k || bs.exit[t] != bits);
  if (__syncthreads_or(bad)) {
    if (t == 0) set_error(a.st, HZ_ERR_CORRUPT, 0x311);
    return;  // uniform
  }
  if (active && v) {
    uint32_t pos = bs.start[t], sym;
    BitReader br;
    br.init(payload, nw, pos);
    uint8_t* dst = a.out + (uint64_t)k * sh.c.B + my_off;
    bool bad2 = false;
    for (uint32_t j = 0; j < v; ++j) {
      const uint32_t l = generic_one(sh, br, pos, sym);
      bad2 |= l == 0;
      pos += l ? l : 1u;
      br.seek(pos);
      dst[j] = (uint8_t)sym;
    }
    if (bad2 || pos != bs.exit[t]) set_error(a.st, HZ_ERR_CORRUPT, 0x312);
  }
}

}  // namespace hz
