// hz_encode_dev.cuh -- device functions of the block encoder, shared by the
// single-buffer kernels (hz_encode.cu) and the batched kernels (hz_batch.cu).
// The design is described in hz_encode.cu.
#pragma once

#include "hz_internal.cuh"

namespace hz {

// A run of symbols, seen as a function on the scan state (O, b):
//   has == 0: the run lies inside one record:  (O, b) -> (O, b + head)
//   has == 1: the run starts >= 1 record:      (O, b) -> (O + 1 + ceil((b + head)/32) + omega, tail)
// head = bits before the run's first record start, omega = words of records
// that start and end inside the run, tail = bits of the run's last record.
struct Summary {
  uint32_t has, head, omega, tail;
};

struct ScanState {
  uint64_t O;  // word index (in the record area) of the open record's delimiter
  uint32_t b;  // payload bits already in the open record
};

static __device__ __forceinline__ Summary combine(const Summary& a, const Summary& x) {  // a, then x
  Summary r;
  if (!x.has) {
    r.has = a.has;
    r.head = a.has ? a.head : a.head + x.head;
    r.omega = a.omega;
    r.tail = a.has ? a.tail + x.head : 0;
  } else if (!a.has) {
    r.has = 1;
    r.head = a.head + x.head;
    r.omega = x.omega;
    r.tail = x.tail;
  } else {
    r.has = 1;
    r.head = a.head;
    r.omega = a.omega + 1 + ceil32((uint64_t)a.tail + x.head) + x.omega;
    r.tail = x.tail;
  }
  return r;
}

static __device__ __forceinline__ ScanState apply(const ScanState& s, const Summary& x) {
  ScanState r;
  if (!x.has) {
    r.O = s.O;
    r.b = s.b + x.head;
  } else {
    r.O = s.O + 1 + ceil32((uint64_t)s.b + x.head) + x.omega;
    r.b = x.tail;
  }
  return r;
}

static __device__ __forceinline__ Summary shfl_up_summary(const Summary& v, int d) {
  Summary r;
  r.has = __shfl_up_sync(0xFFFFFFFFu, v.has, d);
  r.head = __shfl_up_sync(0xFFFFFFFFu, v.head, d);
  r.omega = __shfl_up_sync(0xFFFFFFFFu, v.omega, d);
  r.tail = __shfl_up_sync(0xFFFFFFFFu, v.tail, d);
  return r;
}

static __device__ __forceinline__ Summary load_summary(const TileStatus& t) {
  return Summary{t.has_head >> 31, t.has_head & 0x7FFFFFFFu, t.omega, t.tail};
}

static __device__ __forceinline__ void store_summary(TileStatus& t, const Summary& s) {
  t.has_head = (s.has << 31) | s.head;
  t.omega = s.omega;
  t.tail = s.tail;
}

// a virtual empty record before the first one: its "next record" is word 0
static __device__ __forceinline__ ScanState init_state() { return ScanState{~0ull, 0u}; }

static __device__ __forceinline__ uint32_t sym_of(const uint32_t (&x)[kEncSymPerThread / 4], int i) {
  return (x[i >> 2] >> (8 * (i & 3))) & 0xFFu;
}

// The thread's 32 consecutive symbols (fewer at the end of the input).
static __device__ __forceinline__ void load_symbols(const uint8_t* src, int cnt,
                                             uint32_t (&x)[kEncSymPerThread / 4]) {
  if (cnt == kEncSymPerThread && (((uintptr_t)src) & 15) == 0) {
    uint4 v0 = __ldg(reinterpret_cast<const uint4*>(src));
    uint4 v1 = __ldg(reinterpret_cast<const uint4*>(src) + 1);
    x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
    x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
  } else {
    // static indices only, so that x stays in registers
#pragma unroll
    for (int w = 0; w < kEncSymPerThread / 4; ++w) x[w] = 0;
#pragma unroll
    for (int i = 0; i < kEncSymPerThread; ++i)
      if (i < cnt) x[i >> 2] |= (uint32_t)src[i] << (8 * (i & 3));
  }
}

struct TileGeom {
  uint32_t lo, hi, g0;  // n < 2^32, so every symbol index fits 32 bits
  int my_cnt;
  bool starts_record, ends_record, interior_start;
};

static __device__ __forceinline__ TileGeom tile_geom(uint32_t tile, uint32_t n, const FastDiv& fdB) {
  TileGeom g;
  g.lo = tile * (uint32_t)kEncTile;
  g.hi = n - g.lo > (uint32_t)kEncTile ? g.lo + (uint32_t)kEncTile : n;
  g.g0 = g.lo + threadIdx.x * (uint32_t)kEncSymPerThread;
  g.my_cnt = g.g0 >= g.hi ? 0 : (int)min(g.hi - g.g0, (uint32_t)kEncSymPerThread);
  const uint32_t r_lo = fast_mod(g.lo, fdB);
  g.starts_record = r_lo == 0;
  g.ends_record = fast_mod(g.hi, fdB) == 0 || g.hi == n;
  // first record start after lo: lo + (B - r_lo)
  g.interior_start = (uint64_t)g.lo + (fdB.d - r_lo) < g.hi;
  return g;
}

// Segment summary of one thread's symbols; lens() maps a symbol to its length.
template <class LenF>
__device__ __forceinline__ Summary thread_summary(const uint32_t (&x)[kEncSymPerThread / 4],
                                                  int my_cnt, uint32_t g0, const FastDiv& fdB,
                                                  LenF lens, bool& bad) {
  const uint32_t r0 = fast_mod(g0, fdB);
  uint32_t next_start = r0 == 0 ? 0u : fdB.d - r0;
  Summary s{0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < kEncSymPerThread; ++i) {
    if (i < my_cnt) {
      const uint32_t l = lens(sym_of(x, i));
      bad |= l == 0;
      if ((uint32_t)i == next_start) {
        if (s.has) s.omega += 1 + ceil32(s.tail);
        s.has = 1;
        s.tail = 0;
        next_start += fdB.d;
      }
      if (s.has) s.tail += l;
      else s.head += l;
    }
  }
  return s;
}

// =================================================================== pass 1
// Summary of one tile into a.tiles[tile].  s_len: the code lengths (shared),
// s_wsum / s_warp: per-warp scratch (shared).  Ends with a CTA barrier.
// The thread's symbols of `tile` (see load_symbols).
static __device__ __forceinline__ void load_tile_symbols(const EncodeArgs& a, uint32_t tile,
                                                         uint32_t (&x)[kEncSymPerThread / 4]) {
  const TileGeom g = tile_geom(tile, (uint32_t)a.n, a.fdB);
  load_symbols(a.in + g.g0, g.my_cnt, x);
}

// The length-summing pass of the warp-parallel path: every warp of a tile on
// its own, no CTA barrier.  Records the tile's TileMeta: each lane's bits (the
// sum of its 32 code lengths), the warp's bits, and, for the odd runs of a
// tile (the ones a packing item starts after), the warp's last 32 code bits
// -- found in parallel: each lane takes one of the last lane's 32
// symbols, a suffix sum of their lengths places its code, and the codes that
// end within the last 32 bits are ORed together.  s_tab: the lengths once per
// lane, entry s of lane l at byte 256 s + 4 l (in the lane's own bank, so
// that 32 lanes' lookups are one shared-memory wavefront, as the histogram's
// counters are); a 256-byte row makes a lookup's offset one byte permute of
// the symbol byte and the lane's 4 l (bytes 128-255 of a row are not read).
// s_code: right-aligned codes; s_sym: 32 bytes of per-warp scratch.  Warps of
// a CTA take items (1024-symbol runs) in turn, kSumWarpThreads / 32 per CTA.
constexpr uint32_t kLenNoCode = 1u << 16;  // > 32 codes of at most 32 bits
constexpr int kSumWarpThreads = 512;
constexpr int kSumTabBytes = 256 * 256;
static __device__ __forceinline__ void count_warps(const EncodeArgs& a, const uint8_t* s_tab,
                                                   const uint32_t* s_code, uint8_t* s_sym,
                                                   bool& bad) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t lr = lane * 4;  // byte 0 of a lookup's offset; bytes 1-3 zero
  // the length of the symbol that selector sel moves into byte 1, for this lane
  auto len_of = [&](uint32_t v, uint32_t sel) -> uint32_t {
    return *reinterpret_cast<const uint32_t*>(s_tab + __byte_perm(v, lr, sel));
  };
  constexpr uint32_t kWarps = kEncThreads / 32;  // runs per tile
  constexpr uint32_t kCtaWarps = kSumWarpThreads / 32;
  const uint32_t n = (uint32_t)a.n;
  const uint32_t items = a.ntiles * kWarps;
  const uint32_t stride = gridDim.x * kCtaWarps;
  uint8_t* my_sym = s_sym + 32 * warp;
  // item it's symbols for this lane (g0, cnt); false when the warp has none
  auto geometry = [&](uint32_t it, uint32_t& g0, uint32_t& cnt) -> bool {
    const uint32_t lo = (it / kWarps) * (uint32_t)kEncTile;
    const uint32_t hi = n - lo > (uint32_t)kEncTile ? lo + (uint32_t)kEncTile : n;
    const uint32_t wlo = lo + (it % kWarps) * 32 * kEncSymPerThread;
    g0 = wlo + lane * kEncSymPerThread;
    cnt = g0 >= hi ? 0u : min(hi - g0, (uint32_t)kEncSymPerThread);
    return wlo < hi;
  };
  // the next item's symbols are loaded while the current one is summed
  uint32_t it = blockIdx.x * kCtaWarps + warp;
  uint32_t g0 = 0, cnt = 0;
  bool has = it < items && geometry(it, g0, cnt);
  uint32_t x[kEncSymPerThread / 4], xn[kEncSymPerThread / 4];
  if (has) load_symbols(a.in + g0, (int)cnt, x);
  for (; it < items; it += stride) {
    uint32_t ng0 = 0, ncnt = 0;
    const bool nhas = it + stride < items && geometry(it + stride, ng0, ncnt);
    if (nhas) load_symbols(a.in + ng0, (int)ncnt, xn);
    if (!has) {  // uniform
#pragma unroll
      for (int k = 0; k < kEncSymPerThread / 4; ++k) x[k] = xn[k];
      has = nhas;
      g0 = ng0;
      cnt = ncnt;
      continue;
    }
    const uint32_t tile = it / kWarps, w = it % kWarps;
    // (static indices: x stays in registers; a byte without a code counts
    // kLenNoCode, which no sum of real lengths reaches)
    // (selector 0x55b4: byte 0 from lr, byte 1 the symbol byte b, bytes 2-3 zero)
    uint32_t bits = 0;
    if (cnt == kEncSymPerThread) {
#pragma unroll
      for (int i = 0; i < kEncSymPerThread; ++i)
        bits += len_of(x[i >> 2], 0x5504u | ((uint32_t)(i & 3) << 4));
    } else {
#pragma unroll
      for (int i = 0; i < kEncSymPerThread; ++i)
        if ((uint32_t)i < cnt) bits += len_of(x[i >> 2], 0x5504u | ((uint32_t)(i & 3) << 4));
    }
    bad |= bits >= kLenNoCode;
    TileMeta& m = a.meta[tile];
    m.lane_bits[w * 32 + lane] = (uint16_t)bits;
    const uint32_t tot = __reduce_add_sync(0xFFFFFFFFu, bits);
    // the warp's last 32 bits, when its last lane is full and the packer
    // starts a warp item after it (it packs two of these runs per item, so
    // only the odd runs' tails are read)
    const bool full = __shfl_sync(0xFFFFFFFFu, cnt, 31) == kEncSymPerThread;
    if (full && (w & 1u)) {
      if (lane == 31) {
#pragma unroll
        for (int k = 0; k < kEncSymPerThread / 4; ++k)
          reinterpret_cast<uint32_t*>(my_sym)[k] = x[k];
      }
      __syncwarp();
      const uint32_t sym = my_sym[lane];
      __syncwarp();
      const uint32_t l = *reinterpret_cast<const uint32_t*>(s_tab + ((sym << 8) | lr));
      uint32_t suf = l;  // lengths of symbols lane .. 31
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_down_sync(0xFFFFFFFFu, suf, d);
        if (lane + d < 32) suf += o;
      }
      const uint32_t after = suf - l;  // bits after my code
      const uint32_t t = __reduce_or_sync(0xFFFFFFFFu, after < 32 ? s_code[sym] << after : 0u);
      if (lane == 0) m.warp_tail[w] = t;
    }
    if (lane == 0) m.warp_bits[w] = tot;
#pragma unroll
    for (int k = 0; k < kEncSymPerThread / 4; ++k) x[k] = xn[k];
    has = nhas;
    g0 = ng0;
    cnt = ncnt;
  }
}

// A tile's summary from its TileMeta (warp-parallel path: the tile lies
// inside one record).
static __device__ __forceinline__ Summary meta_summary(const EncodeArgs& a, uint32_t tile) {
  const TileMeta& m = a.meta[tile];
  const uint32_t lo = tile * (uint32_t)kEncTile, n = (uint32_t)a.n;
  const uint32_t syms = n - lo > (uint32_t)kEncTile ? (uint32_t)kEncTile : n - lo;
  const uint32_t warps = (syms + 32 * kEncSymPerThread - 1) / (32 * kEncSymPerThread);
  uint32_t total = 0;  // (warps past the input's end hold no symbol and write nothing)
  const uint4 v0 = *reinterpret_cast<const uint4*>(&m.warp_bits[0]);
  const uint4 v1 = *reinterpret_cast<const uint4*>(&m.warp_bits[4]);
  const uint32_t wb[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
  for (uint32_t w = 0; w < kEncThreads / 32; ++w) total += w < warps ? wb[w] : 0u;
  const bool starts = fast_mod(tile * (uint32_t)kEncTile, a.fdB) == 0;
  return starts ? Summary{1, 0, 0, total} : Summary{0, total, 0, 0};
}

// The barrier of the per-tile summary: the first kEncThreads threads of the
// CTA (all of a kEncThreads-thread CTA; the lower half of the warp-parallel
// summing kernel, whose other threads have left when it runs this path).
static __device__ __forceinline__ void tile_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kEncThreads) : "memory");
}

static __device__ __forceinline__ void summary_tile_x(const EncodeArgs& a, uint32_t tile,
                                                      const uint32_t (&x)[kEncSymPerThread / 4],
                                                      const uint8_t* s_len, uint32_t* s_wsum,
                                                      Summary* s_warp, bool& bad) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TileGeom g = tile_geom(tile, (uint32_t)a.n, a.fdB);
  if (!g.interior_start) {
    // the tile lies inside one record (which may start at its first symbol)
    uint32_t bits = 0, minl = 64;
    if (g.my_cnt == kEncSymPerThread) {
#pragma unroll
      for (int i = 0; i < kEncSymPerThread; ++i) {
        const uint32_t l = s_len[sym_of(x, i)];
        minl = min(minl, l);
        bits += l;
      }
    } else {
#pragma unroll
      for (int i = 0; i < kEncSymPerThread; ++i) {
        if (i < g.my_cnt) {
          const uint32_t l = s_len[sym_of(x, i)];
          minl = min(minl, l);
          bits += l;
        }
      }
    }
    bad |= minl == 0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) bits += __shfl_xor_sync(0xFFFFFFFFu, bits, d);
    if (lane == 0) s_wsum[warp] = bits;
    tile_sync();
    if (tid == 0) {
      uint32_t total = 0;
      for (int w = 0; w < kEncThreads / 32; ++w) total += s_wsum[w];
      store_summary(a.tiles[tile], g.starts_record ? Summary{1, 0, 0, total}
                                                   : Summary{0, total, 0, 0});
    }
  } else {
    Summary sm = thread_summary(x, g.my_cnt, g.g0, a.fdB, [&](uint32_t v) { return s_len[v]; },
                                bad);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      Summary o = shfl_up_summary(sm, d);
      if (lane >= d) sm = combine(o, sm);
    }
    if (lane == 31) s_warp[warp] = sm;
    tile_sync();
    if (tid == 0) {
      Summary t{0, 0, 0, 0};
      for (int w = 0; w < kEncThreads / 32; ++w) t = combine(t, s_warp[w]);
      store_summary(a.tiles[tile], t);
    }
  }
  tile_sync();
}

static __device__ __forceinline__ void summary_tile(const EncodeArgs& a, uint32_t tile,
                                             const uint8_t* s_len, uint32_t* s_wsum,
                                             Summary* s_warp, bool& bad) {
  uint32_t x[kEncSymPerThread / 4];
  load_tile_symbols(a, tile, x);
  summary_tile_x(a, tile, x, s_len, s_wsum, s_warp, bad);
}

// The stream size, from the state after the last tile, and the capacity check.
static __device__ __forceinline__ void finish_stream(const EncodeArgs& a, const ScanState& s,
                                              bool aborted) {
  const uint64_t rec_base = records_at(a.nb, a.B, a.flags, a.sub_S);
  const uint64_t words = s.O + 1 + ceil32(s.b);
  const uint64_t size = rec_base + 4 * words;
  *a.out_len = size;
  bool ok = a.st->error == 0 && !aborted;
  if (size > a.out_cap || words > 0xFFFFFFFFull) {
    set_error(a.st, HZ_ERR_CAPACITY, 0x203);
    ok = false;
  }
  a.st->enc_ok = ok ? 1u : 0u;
}

// Scan of all of a buffer's tile summaries by one CTA of kScanThreads threads
// (chunks of kScanTilesPerCta tiles, a running carry between chunks): the
// batched encoder's scan, where one buffer rarely has more than a few chunks.
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = kScanTilesPerCta / kScanThreads;

static __device__ void scan_tiles_cta(const EncodeArgs& a, Summary* s_warp /* [32] */,
                               ScanState* s_carry) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t nt = a.ntiles;
  if (tid == 0) *s_carry = init_state();
  for (uint32_t base = 0; base < nt; base += kScanTilesPerCta) {
    __syncthreads();
    const uint32_t t0 = base + tid * kScanPerThread;
    Summary mine[kScanPerThread];
    Summary agg{0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
      mine[k] = t0 + k < nt ? load_summary(a.tiles[t0 + k]) : Summary{0, 0, 0, 0};
      agg = combine(agg, mine[k]);
    }
    Summary inc = agg;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      Summary o = shfl_up_summary(inc, d);
      if (lane >= d) inc = combine(o, inc);
    }
    Summary ex = shfl_up_summary(inc, 1);
    if (lane == 0) ex = Summary{0, 0, 0, 0};
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    Summary wpre{0, 0, 0, 0}, cta_agg{0, 0, 0, 0};
    for (int w = 0; w < kScanThreads / 32; ++w) {
      if (w < warp) wpre = combine(wpre, s_warp[w]);
      cta_agg = combine(cta_agg, s_warp[w]);
    }
    const ScanState carry = *s_carry;
    ScanState st = apply(carry, combine(wpre, ex));
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
      if (t0 + k < nt) {
        a.tiles[t0 + k].pre_O = st.O;
        a.tiles[t0 + k].pre_b = st.b;
        st = apply(st, mine[k]);
        if (t0 + k == nt - 1) finish_stream(a, st, false);
      }
    }
    __syncthreads();
    if (tid == 0) *s_carry = apply(carry, cta_agg);
  }
}

// =================================================================== pass 3
// Sub-block offsets (flags bit 1).  Every sub-block boundary (symbol j*S of a
// block, j >= 1) is the first symbol of some thread's 32-symbol run, since B
// and S are multiples of 32; that thread knows the payload bit its run starts
// at and writes the entry.
static __device__ __forceinline__ void put_sub_entry(const EncodeArgs& a, uint32_t g,
                                                     uint32_t bit) {
  if (fast_mod(g, a.fdS) != 0) return;  // (S divides B: not a boundary; the common case)
  const uint32_t k = fast_div(g, a.fdB);
  const uint32_t r = g - k * a.B;  // position in the block
  if (r == 0) return;  // a block start: no entry
  uint32_t* e = reinterpret_cast<uint32_t*>(a.out + sub_entries_at(a.nb));
  e[(uint64_t)k * (a.sub_M - 1) + fast_div(r, a.fdS) - 1] = bit;
}
// The last block's entries past its last symbol hold its payload bit count.
static __device__ __forceinline__ void put_sub_tail(const EncodeArgs& a, uint32_t bits) {
  const uint32_t k = a.nb - 1;
  const uint32_t cnt = (uint32_t)(a.n - (uint64_t)k * a.B);
  uint32_t* e = reinterpret_cast<uint32_t*>(a.out + sub_entries_at(a.nb)) +
                (uint64_t)k * (a.sub_M - 1);
  for (uint32_t j = fast_div(cnt + a.sub_S - 1, a.fdS); j < a.sub_M; ++j) e[j - 1] = bits;
}

struct PackShared {
  EncodeArgs a;         // the launch arguments, read by the per-tile functions
  uint32_t entry[256];  // code << 6 | len, valid for codes of up to 26 bits
  uint32_t lent[256];   // code << (32 - len) | len, valid for codes of up to 16 bits
  uint2 cl[256];        // {code << (32 - len), len}, valid for codes of up to 32 bits
  uint32_t len[256];
  uint32_t code_lo[256];
  uint32_t code_hi[256];
  uint32_t wsum[kEncThreads / 32];
  Summary warp_sum[kEncThreads / 32];
  uint32_t prev_bits;
  __align__(16) uint8_t prev32[32];  // the 32 input bytes before the tile (single-record path)
  __align__(16) uint32_t stage[kEncStageWords + 4];
};

template <bool kLong>
__device__ __forceinline__ void lookup(const PackShared& sh, uint32_t sym, uint32_t& l,
                                       uint64_t& c) {
  if (!kLong) {
    const uint32_t e = sh.entry[sym];
    l = e & 63u;
    c = e >> 6;
  } else {
    l = sh.len[sym];
    c = ((uint64_t)sh.code_hi[sym] << 32) | sh.code_lo[sym];
  }
}

// The r (< 32) payload bits just before input position `pos` (all inside the
// record that continues at `pos`), right-aligned.
template <bool kLong>
__device__ uint32_t bits_before(const PackShared& sh, const uint8_t* in, uint32_t pos,
                                uint32_t r) {
  uint64_t v = 0;
  uint32_t got = 0;
  int64_t j = (int64_t)pos - 1;
  while (got < r && j >= 0) {
    uint32_t l;
    uint64_t c;
    lookup<kLong>(sh, in[j], l, c);
    if (got < 64) v |= c << got;
    got += l;
    --j;
  }
  return (uint32_t)(v & ((1u << r) - 1u));
}

// bits_before from the 32 bytes before the tile, staged in shared memory by a
// cp.async that thread 0 issues when the tile starts (so that the input's
// latency overlaps the tile's own loads): at most 31 codes make up r < 32 bits.
template <bool kLong>
__device__ uint32_t bits_before_staged(const PackShared& sh, uint32_t r) {
  uint64_t v = 0;
  uint32_t got = 0;
  for (int j = 31; j >= 0 && got < r; --j) {
    uint32_t l;
    uint64_t c;
    lookup<kLong>(sh, sh.prev32[j], l, c);
    if (got < 64) v |= c << got;
    got += l;
  }
  return (uint32_t)(v & ((1u << r) - 1u));
}
static __device__ __forceinline__ void stage_prev32(PackShared& sh, const uint8_t* src) {
  const uint32_t dst = (uint32_t)__cvta_generic_to_shared(sh.prev32);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16), "l"(src + 16) : "memory");
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Pack one thread's 32 cached entries (code << 6 | len) MSB-first into
// st[wrel...], starting `nacc` bits into word wrel.  A word that may hold an
// earlier thread's bits (the first one, when nacc != 0) or a later thread's
// (the last, partial one) is combined with atomicOr.
template <bool kPair>
__device__ __forceinline__ void pack_entries(const uint32_t (&e)[kEncSymPerThread], uint32_t* st,
                                             uint32_t wrel, uint32_t nacc) {
  bool first_shared = nacc != 0;
  uint64_t acc = 0;
  auto push = [&](uint32_t c, uint32_t l) {
    acc = (acc << l) | c;
    nacc += l;
    if (nacc >= 32) {
      nacc -= 32;
      const uint32_t v = (uint32_t)(acc >> nacc);
      if (first_shared) atomicOr(st + wrel, v);
      else st[wrel] = v;
      first_shared = false;
      ++wrel;
    }
  };
  if (kPair) {
#pragma unroll
    for (int j = 0; j < kEncSymPerThread / 2; ++j) {
      const uint32_t ea = e[2 * j], eb = e[2 * j + 1];
      const uint32_t lb = eb & 63u;
      push(((ea >> 6) << lb) | (eb >> 6), (ea & 63u) + lb);
    }
  } else {
#pragma unroll
    for (int i = 0; i < kEncSymPerThread; ++i) push(e[i] >> 6, e[i] & 63u);
  }
  if (nacc) atomicOr(st + wrel, (uint32_t)(acc << (32 - nacc)));
}

// Write stage[off .. end) to gbase[off .. end) with 16-byte stores where a
// whole aligned chunk is inside the range, skipping index skip_i.
static __device__ __forceinline__ void copy_out(const uint32_t* stage, uint32_t* gbase, uint32_t off,
                                         uint32_t end, uint32_t skip_i) {
  const uint32_t nchunks = (end + 3) >> 2;
  for (uint32_t c = threadIdx.x; c < nchunks; c += kEncThreads) {
    const uint32_t i0 = c << 2;
    if (i0 >= off && i0 + 4 <= end && (skip_i < i0 || skip_i >= i0 + 4)) {
      *reinterpret_cast<uint4*>(gbase + i0) = *reinterpret_cast<const uint4*>(stage + i0);
    } else {
#pragma unroll
      for (uint32_t k = 0; k < 4; ++k) {
        const uint32_t i = i0 + k;
        if (i >= off && i < end && i != skip_i) gbase[i] = stage[i];
      }
    }
  }
}

// pack_entries for codes of up to 32 bits: the symbols in x[], their code
// lengths six bits each, five to a word, in lp[]; the codes are looked up.
__device__ __forceinline__ void pack_entries_wide(const PackShared& sh,
                                                  const uint32_t (&x)[kEncSymPerThread / 4],
                                                  const uint32_t (&lp)[(kEncSymPerThread + 4) / 5],
                                                  uint32_t* st, uint32_t wrel, uint32_t nacc) {
  bool first_shared = nacc != 0;
  uint64_t acc = 0;  // fewer than 32 pending bits before each code of at most 32
#pragma unroll
  for (int i = 0; i < kEncSymPerThread; ++i) {
    const uint32_t l = (lp[i / 5] >> (6 * (i % 5))) & 63u;
    const uint32_t c = l ? sh.code_lo[sym_of(x, i)] : 0u;  // l = 0 past the thread's symbols
    acc = (acc << l) | c;
    nacc += l;
    if (nacc >= 32) {
      nacc -= 32;
      const uint32_t v = (uint32_t)(acc >> nacc);
      if (first_shared) atomicOr(st + wrel, v);
      else st[wrel] = v;
      first_shared = false;
      ++wrel;
    }
  }
  if (nacc) atomicOr(st + wrel, (uint32_t)(acc << (32 - nacc)));
}

// Single-record path: the tile lies inside one record (which may start at its
// first symbol); thread positions come from a plain scan of bit counts.
// kKind 0: codes of at most 16 bits, packed two at a time; 1: at most 26
// bits (code and length in one cached word); 2: at most 32 bits (lengths
// cached, codes looked up again while packing).
template <int kKind>
__device__ __noinline__ void pack_tile_single(PackShared& sh, uint32_t tile, const TileGeom g,
                                                 uint32_t* rec_words) {
  const EncodeArgs& a = sh.a;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const ScanState S{a.tiles[tile].pre_O, a.tiles[tile].pre_b};
  const uint64_t O1 = g.starts_record ? S.O + 1 + ceil32(S.b) : S.O;
  const uint32_t b0 = g.starts_record ? 0u : S.b;
  const uint32_t r_prev = b0 & 31u;  // bits of the previous tile in this tile's first word
  const uint8_t* prev_src = a.in + g.lo - 32;
  const bool staged = r_prev && g.lo >= 32 && (((uintptr_t)prev_src) & 15) == 0;
  if (tid == 0 && staged) stage_prev32(sh, prev_src);

  uint32_t x[kEncSymPerThread / 4];
  load_symbols(a.in + g.g0, g.my_cnt, x);
  uint32_t e[kEncSymPerThread];
  uint32_t lp[(kEncSymPerThread + 4) / 5] = {};
  uint32_t bits = 0;
#pragma unroll
  for (int i = 0; i < kEncSymPerThread; ++i) {
    if (kKind == 2) {  // codes are looked up again while packing
      const uint32_t l = i < g.my_cnt ? sh.len[sym_of(x, i)] : 0u;
      lp[i / 5] |= l << (6 * (i % 5));
      bits += l;
    } else {
      e[i] = i < g.my_cnt ? sh.entry[sym_of(x, i)] : 0u;
      bits += e[i] & 63u;
    }
  }
  uint32_t inc = bits;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) sh.wsum[warp] = inc;
  __syncthreads();
  uint32_t wpre = 0, total = 0;
#pragma unroll
  for (int w = 0; w < kEncThreads / 32; ++w) {
    const uint32_t v = sh.wsum[w];
    wpre += w < warp ? v : 0u;
    total += v;
  }
  const uint32_t ex = wpre + inc - bits;
  const uint32_t bend = b0 + total;
  const uint64_t W0 = O1 + 1 + (b0 >> 5);
  const uint32_t nwords = ((bend - 1) >> 5) - (b0 >> 5) + 1;
  const uint32_t off = (uint32_t)((((uintptr_t)rec_words) >> 2) + W0) & 3u;
  if (total == 0 || off + nwords > (uint32_t)kEncStageWords + 4) {
    if (tid == 0) {
      set_error(a.st, HZ_ERR_ARG, 0x206);
      asm volatile("cp.async.wait_all;\n" ::: "memory");
    }
    return;  // uniform
  }
  for (uint32_t i = tid; i < off + nwords; i += kEncThreads) sh.stage[i] = 0;
  if (tid == 0 && r_prev) {
    // (codes of more than 26 bits: the entry table truncates them, so the
    // length and code tables)
    if (staged) {
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      sh.prev_bits = bits_before_staged<kKind == 2>(sh, r_prev);
    } else {
      sh.prev_bits = bits_before<kKind == 2>(sh, a.in, g.lo, r_prev);
    }
  }
  __syncthreads();
  if (tid == 0 && r_prev) sh.stage[off] = sh.prev_bits << (32 - r_prev);
  __syncthreads();
  if (bits) {
    const uint32_t p = b0 + ex;
    if (kKind == 2) pack_entries_wide(sh, x, lp, sh.stage + off, (p >> 5) - (b0 >> 5), p & 31u);
    else pack_entries<kKind == 0>(e, sh.stage + off, (p >> 5) - (b0 >> 5), p & 31u);
  }
  if ((a.flags & kFlagSub) && g.my_cnt > 0) put_sub_entry(a, g.g0, b0 + ex);
  __syncthreads();
  // the last word belongs to the next tile when the record goes on mid-word
  const bool skip_last = !g.ends_record && (bend & 31u) != 0;
  copy_out(sh.stage, rec_words + (W0 - off), off, off + nwords - (skip_last ? 1u : 0u),
           0xFFFFFFFFu);
  if (tid == 0) {
    if (g.ends_record) rec_words[O1] = bend;  // this tile holds the record's last symbol
    if ((a.flags & kFlagSub) && g.hi == (uint32_t)a.n) put_sub_tail(a, bend);
    if (g.starts_record && (a.flags & kFlagIndex))
      reinterpret_cast<uint32_t*>(a.out + kHeaderBytes)[fast_div(g.lo, a.fdB)] = (uint32_t)O1;
  }
}

// Chunked path: B is a multiple of 32, so records start and end only at the
// boundaries of the threads' 32-symbol chunks, and codes have at most 26
// bits.  Each chunk lies inside one record; a thread's start state comes from
// a CTA scan of chunk summaries.
template <bool kPair>
__device__ __noinline__ void pack_tile_chunked(PackShared& sh, uint32_t tile, const TileGeom g,
                                                  uint32_t* rec_words) {
  const EncodeArgs& a = sh.a;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const ScanState S_s{a.tiles[tile].pre_O, a.tiles[tile].pre_b};

  uint32_t x[kEncSymPerThread / 4];
  load_symbols(a.in + g.g0, g.my_cnt, x);
  uint32_t e[kEncSymPerThread];
  uint32_t bits = 0;
#pragma unroll
  for (int i = 0; i < kEncSymPerThread; ++i) {
    e[i] = i < g.my_cnt ? sh.entry[sym_of(x, i)] : 0u;
    bits += e[i] & 63u;
  }
  const bool starts = g.my_cnt > 0 && fast_mod(g.g0, a.fdB) == 0;
  const uint32_t gend = g.g0 + (uint32_t)g.my_cnt;
  const bool ends = g.my_cnt > 0 && (fast_mod(gend, a.fdB) == 0 || gend == (uint32_t)a.n);
  const Summary mine = starts ? Summary{1, 0, 0, bits} : Summary{0, bits, 0, 0};
  Summary inc = mine;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    Summary o = shfl_up_summary(inc, d);
    if (lane >= d) inc = combine(o, inc);
  }
  Summary ex = shfl_up_summary(inc, 1);
  if (lane == 0) ex = Summary{0, 0, 0, 0};
  if (lane == 31) sh.warp_sum[warp] = inc;
  __syncthreads();
  Summary wpre{0, 0, 0, 0}, agg{0, 0, 0, 0};
#pragma unroll
  for (int w = 0; w < kEncThreads / 32; ++w) {
    const Summary v = sh.warp_sum[w];
    if (w < warp) wpre = combine(wpre, v);
    agg = combine(agg, v);
  }
  const ScanState S_t = apply(S_s, combine(wpre, ex));  // before my chunk
  const uint64_t myO = starts ? S_t.O + 1 + ceil32(S_t.b) : S_t.O;
  const uint32_t myb = starts ? 0u : S_t.b;
  const ScanState S_e = apply(S_s, agg);
  const uint64_t w_first = g.starts_record ? S_s.O + 1 + ceil32(S_s.b) : S_s.O + 1 + (S_s.b >> 5);
  const uint64_t w_last = S_e.O + 1 + ((S_e.b - 1) >> 5);
  const uint32_t off = (uint32_t)((((uintptr_t)rec_words) >> 2) + w_first) & 3u;
  if (S_e.b == 0 || w_last < w_first || w_last - w_first + off >= (uint64_t)kEncStageWords + 4) {
    if (tid == 0) set_error(a.st, HZ_ERR_ARG, 0x207);
    return;  // uniform
  }
  const uint32_t nwords = (uint32_t)(w_last - w_first + 1);
  const bool skip_last = !g.ends_record && (S_e.b & 31u) != 0;
  // the delimiter of a record that starts here but ends in a later tile is
  // written by that later tile
  const uint32_t skip_i = (!g.ends_record && S_e.O >= w_first)
                              ? off + (uint32_t)(S_e.O - w_first) : 0xFFFFFFFFu;
  const uint32_t r_prev = g.starts_record ? 0u : (S_s.b & 31u);
  for (uint32_t i = tid; i < off + nwords; i += kEncThreads) sh.stage[i] = 0;
  if (tid == 0 && r_prev) sh.prev_bits = bits_before<false>(sh, a.in, g.lo, r_prev);
  __syncthreads();
  if (tid == 0 && r_prev) sh.stage[off] = sh.prev_bits << (32 - r_prev);
  __syncthreads();
  uint32_t* st = sh.stage + off;
  if (g.my_cnt > 0) {
    if (bits) pack_entries<kPair>(e, st, (uint32_t)(myO + 1 + (myb >> 5) - w_first), myb & 31u);
    if (ends) {
      // last chunk of a record: its delimiter is now known
      if (myO >= w_first) st[myO - w_first] = myb + bits;
      else rec_words[myO] = myb + bits;
      if ((a.flags & kFlagSub) && gend == (uint32_t)a.n) put_sub_tail(a, myb + bits);
    }
    if (a.flags & kFlagSub) put_sub_entry(a, g.g0, myb);
    if (starts && (a.flags & kFlagIndex))
      reinterpret_cast<uint32_t*>(a.out + kHeaderBytes)[fast_div(g.g0, a.fdB)] = (uint32_t)myO;
  }
  __syncthreads();
  copy_out(sh.stage, rec_words + (w_first - off), off, off + nwords - (skip_last ? 1u : 0u),
           skip_i);
}

// Writer for one thread's words in the general path: words inside the current
// staging window go to shared memory, others are dropped (another window pass
// writes them).
struct Emitter {
  uint32_t* stage;
  uint64_t win_lo, win_hi;
  __device__ __forceinline__ void put(uint64_t w, uint32_t v, bool shared_word) {
    if (w >= win_lo && w < win_hi) {
      uint32_t* p = stage + (w - win_lo);
      if (shared_word) atomicOr(p, v);
      else *p = v;
    }
  }
};

// General path: record starts anywhere in the tile, codes of any length.
template <bool kLong>
__device__ __noinline__ void pack_tile_general(PackShared& sh, uint32_t tile, const TileGeom g,
                                                  uint32_t* rec_words) {
  const EncodeArgs& a = sh.a;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t n = (uint32_t)a.n;
  const uint32_t B = a.fdB.d;
  uint32_t x[kEncSymPerThread / 4];
  load_symbols(a.in + g.g0, g.my_cnt, x);
  bool bad = false;
  const Summary s = thread_summary(
      x, g.my_cnt, g.g0, a.fdB,
      [&](uint32_t v) {
        uint32_t l;
        uint64_t c;
        lookup<kLong>(sh, v, l, c);
        return l;
      },
      bad);
  Summary inc = s;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    Summary o = shfl_up_summary(inc, d);
    if (lane >= d) inc = combine(o, inc);
  }
  Summary ex = shfl_up_summary(inc, 1);
  if (lane == 0) ex = Summary{0, 0, 0, 0};
  if (lane == 31) sh.warp_sum[warp] = inc;
  __syncthreads();
  Summary wpre{0, 0, 0, 0}, agg{0, 0, 0, 0};
  for (int w = 0; w < kEncThreads / 32; ++w) {
    if (w < warp) wpre = combine(wpre, sh.warp_sum[w]);
    agg = combine(agg, sh.warp_sum[w]);
  }
  ex = combine(wpre, ex);

  const ScanState S_s{a.tiles[tile].pre_O, a.tiles[tile].pre_b};
  const ScanState S_e = apply(S_s, agg);
  const uint64_t w_first = g.starts_record ? S_s.O + 1 + ceil32(S_s.b) : S_s.O + 1 + (S_s.b >> 5);
  const uint64_t w_last = S_e.O + 1 + ((S_e.b - 1) >> 5);
  const bool skip_last = !g.ends_record && (S_e.b & 31u) != 0;
  const bool skip_open = !g.ends_record && S_e.O >= w_first && S_e.O <= w_last;
  const uint32_t r_prev = g.starts_record ? 0u : (S_s.b & 31u);
  if (S_e.b == 0 || w_last < w_first || w_last - w_first > 3ull * kEncTile + 64) {
    if (tid == 0) set_error(a.st, HZ_ERR_ARG, 0x204);
    return;  // uniform
  }
  if (tid == 0) sh.prev_bits = r_prev ? bits_before<kLong>(sh, a.in, g.lo, r_prev) : 0u;
  const ScanState S_t = apply(S_s, ex);  // state before my first symbol
  const uint32_t r0 = fast_mod(g.g0, a.fdB);
  const uint32_t first_start = r0 == 0 ? 0u : B - r0;
  // one past the last symbol of my first record
  const uint32_t first_end = (uint32_t)min((uint64_t)g.g0 - r0 + B, (uint64_t)n);

  for (uint64_t wlo = w_first; wlo <= w_last; wlo += kEncStageWords) {
    const uint64_t whi = wlo + kEncStageWords < w_last + 1 ? wlo + kEncStageWords : w_last + 1;
    for (int i = tid; i < kEncStageWords; i += kEncThreads) sh.stage[i] = 0;
    __syncthreads();
    if (tid == 0 && wlo == w_first && r_prev) sh.stage[0] = sh.prev_bits << (32 - r_prev);
    __syncthreads();
    Emitter em{sh.stage, wlo, whi};
    ScanState cur = S_t;
    uint64_t wcur = cur.O + 1 + (cur.b >> 5);
    uint32_t nacc = cur.b & 31u;
    bool first_shared = nacc != 0;
    uint64_t acc = 0;
    uint32_t next_start = first_start;
    uint32_t next_end = first_end;
    // (sub-block offsets need B a multiple of 32: no record starts inside the run)
    if ((a.flags & kFlagSub) && wlo == w_first && g.my_cnt > 0) put_sub_entry(a, g.g0, cur.b);
#pragma unroll
    for (int i = 0; i < kEncSymPerThread; ++i) {
      if (i < g.my_cnt) {
        if ((uint32_t)i == next_start) {
          if (nacc) em.put(wcur, (uint32_t)(acc << (32 - nacc)), true);
          cur.O = cur.O + 1 + ceil32(cur.b);
          cur.b = 0;
          if ((a.flags & kFlagIndex) && wlo == w_first)
            reinterpret_cast<uint32_t*>(a.out + kHeaderBytes)[fast_div(g.g0 + i, a.fdB)] =
                (uint32_t)cur.O;
          wcur = cur.O + 1;
          nacc = 0;
          acc = 0;
          first_shared = false;
          next_start += B;
        }
        uint32_t l;
        uint64_t c;
        lookup<kLong>(sh, sym_of(x, i), l, c);
        if (kLong && l > 32) {
          const uint32_t lh = l - 32;
          acc = (acc << lh) | (c >> 32);
          nacc += lh;
          if (nacc >= 32) {
            nacc -= 32;
            em.put(wcur++, (uint32_t)(acc >> nacc), first_shared);
            first_shared = false;
          }
          acc = (acc << 32) | (c & 0xFFFFFFFFull);
          em.put(wcur++, (uint32_t)(acc >> nacc), first_shared);
          first_shared = false;
        } else {
          acc = (acc << l) | c;
          nacc += l;
          if (nacc >= 32) {
            nacc -= 32;
            em.put(wcur++, (uint32_t)(acc >> nacc), first_shared);
            first_shared = false;
          }
        }
        cur.b += l;
        if (g.g0 + (uint32_t)i + 1 == next_end) {
          // last symbol of a record: its delimiter is now known
          if (cur.O >= wlo && cur.O < whi) sh.stage[cur.O - wlo] = cur.b;
          else if (cur.O < w_first && wlo == w_first) rec_words[cur.O] = cur.b;
          if ((a.flags & kFlagSub) && wlo == w_first && next_end == n) put_sub_tail(a, cur.b);
          next_end = (uint32_t)min((uint64_t)next_end + B, (uint64_t)n);
        }
      }
    }
    if (nacc && g.my_cnt) em.put(wcur, (uint32_t)(acc << (32 - nacc)), true);
    __syncthreads();
    const uint64_t cnt_w = whi - wlo;
    for (uint64_t i = tid; i < cnt_w; i += kEncThreads) {
      const uint64_t w = wlo + i;
      if ((skip_last && w == w_last) || (skip_open && w == S_e.O)) continue;
      rec_words[w] = sh.stage[i];
    }
    __syncthreads();
  }
}

// ------------------------------------------------- warp-parallel packing
// Tiles that lie inside one record (B a multiple of the tile), codes of at
// most 32 bits, with the TileMeta the length-summing pass wrote: a warp packs
// 2048 symbols of a tile (two of the summing pass's 1024-symbol runs) on its
// own, with no CTA barrier.
//   - lane l takes the 64 symbols of the summing pass's 32-symbol runs 2l and
//     2l + 1; their bit counts (from the metadata, one 32-bit load) are
//     scanned with shuffles, the warp's own offset within the tile and the
//     tile's start state come from the metadata and the tile scan;
//   - a lane packs its symbols two codes at a time (a pair is at most 32
//     bits; four at a time when no code is longer than 8 bits) into one
//     32-bit accumulator and writes each word it completes into the warp's
//     staging area in shared memory;
//   - the word a lane shares with the lane before it (its first word, when it
//     starts mid-word) gets that lane's partial last word through one shuffle;
//     a warp's first word gets the previous run's last bits from the
//     metadata's warp tail (the run before in the tile, or the last run of
//     the tile before);
//   - a lane's partial last word belongs to the next lane (or warp), except
//     at the end of the record, where it is written zero-padded;
//   - the item's whole 16-byte chunks leave the staging area by one bulk
//     copy (cp.async.bulk), the ragged words at its ends by lanes' stores.
// No word is written twice and the output needs no clearing.  Taking 64
// symbols a lane halves the per-lane work that does not depend on the symbol
// count (offsets, shuffles, the shared words, the copy-out).
// kWide (codes of 17 to 32 bits): one code per step, from sh.cl.  A warp's
// words may then not fit its staging area (2048 codes of 32 bits are 2048
// words): such an item is written straight to the output instead, each lane
// storing the words it completes and, last, its first word with the bits of
// the lane before.
constexpr uint32_t kPackRuns = 2;                                  // summing-pass runs per lane
constexpr uint32_t kPackSyms = kPackRuns * kEncSymPerThread;       // symbols per lane
constexpr uint32_t kPackItems = kEncThreads / 32 / kPackRuns;      // warp items per tile
constexpr uint32_t kWarpStageWords = kPackSyms * 32 * 16 / 32 + 8;  // codes of <= 16 bits, + alignment
static_assert(kWarpStageWords * (kEncThreads / 32) <= (uint32_t)kEncStageWords + 4, "staging");

// Bulk copies from the staging area to the output (the copy engine reads the
// shared memory while the warp goes on packing).  The staging words are
// written by ordinary stores: each writing thread makes them visible to the
// copy engine (the async proxy) with a proxy fence before the copy is issued.
static __device__ __forceinline__ void bulk_fence_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// bytes (a multiple of 16) from shared s to global g, both 16-byte aligned
static __device__ __forceinline__ void bulk_store(void* g, const void* s, uint32_t bytes) {
  asm volatile(
      "cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n"
      "cp.async.bulk.commit_group;\n" ::"l"((uint64_t)__cvta_generic_to_global(g)),
      "r"((uint32_t)__cvta_generic_to_shared(s)), "r"(bytes)
      : "memory");
}
// this thread's bulk copies have read their sources
static __device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// this thread's bulk copies are complete
static __device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

template <bool kWide, bool kQuad = false>
static __device__ __forceinline__ void pack_warps_fast(PackShared& sh) {
  const EncodeArgs& a = sh.a;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr uint32_t kWarps = kEncThreads / 32;
  const uint32_t n = (uint32_t)a.n;
  uint32_t* rec_words =
      reinterpret_cast<uint32_t*>(a.out + records_at(a.nb, a.B, a.flags, a.sub_S));
  uint32_t* stw = sh.stage + warp * kWarpStageWords;
  const uint32_t items = (a.tile_end - a.tile_begin) * kPackItems;
  for (uint32_t it = blockIdx.x * kWarps + warp; it < items; it += gridDim.x * kWarps) {
    // last tiles first: their input is still in L2 from the length-summing pass
    const uint32_t tile = a.tile_end - 1 - it / kPackItems;
    const uint32_t v0 = (it % kPackItems) * kPackRuns;  // the item's first summing-pass run
    const uint32_t lo = tile * (uint32_t)kEncTile;
    const uint32_t hi = n - lo > (uint32_t)kEncTile ? lo + (uint32_t)kEncTile : n;
    const uint32_t wlo = lo + v0 * 32 * kEncSymPerThread;
    if (wlo >= hi) continue;  // uniform: no symbol for this warp
    const uint32_t g0 = wlo + lane * kPackSyms;
    const uint32_t cnt = g0 >= hi ? 0u : min(hi - g0, kPackSyms);
    const uint32_t cnt0 = min(cnt, (uint32_t)kEncSymPerThread);  // symbols of my first run
    const uint32_t cnt1 = cnt - cnt0;                            // and of my second
    const TileMeta& m = a.meta[tile];
    const bool starts = fast_mod(lo, a.fdB) == 0;
    const bool ends = fast_mod(hi, a.fdB) == 0 || hi == n;  // the tile ends its record
    const uint64_t pre_O = a.tiles[tile].pre_O;
    const uint32_t pre_b = a.tiles[tile].pre_b;
    const uint64_t O1 = starts ? pre_O + 1 + ceil32(pre_b) : pre_O;  // the record's delimiter
    const uint32_t b0 = starts ? 0u : pre_b;
    // my runs' bit counts: lane_bits[32 v + j] of runs j = 2l, 2l + 1 of the
    // item (v = v0 + l / 16), two adjacent u16 (a run without symbols may not
    // have been written)
    const uint32_t bb = cnt ? reinterpret_cast<const uint32_t*>(m.lane_bits)[v0 * 16 + lane] : 0u;
    const uint32_t c0 = cnt0 ? (bb & 0xFFFFu) : 0u;
    const uint32_t c = c0 + (cnt1 ? (bb >> 16) : 0u);
    uint32_t inc = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
      if (lane >= (uint32_t)d) inc += o;
    }
    // bits of the tile's earlier runs: lane v < v0 loads run v's count
    const uint32_t wp = __reduce_add_sync(0xFFFFFFFFu, lane < v0 ? m.warp_bits[lane] : 0u);
    const uint32_t ws = b0 + wp;  // the warp's first payload bit
    const uint32_t we = ws + __shfl_sync(0xFFFFFFFFu, inc, 31);
    const uint32_t p = ws + inc - c;
    const uint32_t r = ws & 31u;
    // the last lane with symbols, and whether the record ends with it
    const uint32_t last_lane = 31u - (__clz(__ballot_sync(0xFFFFFFFFu, cnt > 0)));
    const bool rec_end = ends && hi - wlo <= 32u * kPackSyms;  // the warp holds the tile's end
    // staging: word index i of the payload goes to stw[i - wb + off], so that
    // 16-byte chunks of stw are 16-byte aligned in the output
    const uint32_t wb = ws >> 5;
    uint32_t* pay = rec_words + O1 + 1;
    const uint32_t off = (uint32_t)(((uintptr_t)(pay + wb)) >> 2) & 3u;
    // ---- pack: every completed word goes to the staging area (a shared first
    // word too: the previous lane's bits are ORed into it below)
    uint32_t acc_hi = 0, nacc = p & 31u;
    const uint32_t w_first = (p >> 5) - wb + off;
    uint32_t wi = w_first;
    const bool shared_head = (p & 31u) != 0 && c != 0;
    // ---- copy-out range: payload words [wb, wend); the partial last word
    // only at the record's end
    const uint32_t wend = (we >> 5) + ((rec_end && (we & 31u)) ? 1u : 0u);
    const uint32_t nw = wend - wb;
    uint32_t* gbase = pay + wb - off;  // 16-byte aligned
    // (uniform) the item's words do not fit the staging area: straight out
    const bool direct = kWide && nw + off > kWarpStageWords;
    uint32_t fw = 0;  // direct: my first completed word, stored last
    auto emit = [&](uint32_t v) {
      if (!kWide || !direct) stw[wi] = v;
      else if (wi == w_first) fw = v;
      else gbase[wi] = v;
      ++wi;
    };
    // one code of up to 32 bits, left-aligned in c
    // (what passes the word, cc << (32 - nacc), is non-zero only when the word
    // completes: it becomes the next word's start)
    auto push1 = [&](uint32_t cc, uint32_t l) {
      const uint32_t over = __funnelshift_r(0u, cc, nacc);  // 0 for nacc = 0
      acc_hi |= cc >> nacc;
      nacc += l;
      if (nacc >= 32u) {
        emit(acc_hi);
        acc_hi = over;
        nacc -= 32u;
      }
    };
    // Two codes of at most 16 bits a step.  The shifts take their amounts mod
    // 32, so ea's and nacc's bits above the low five ride along: nacc's low six
    // bits count the accumulator's bits (at most 31 + 32), and the codes' bits
    // that ea + eb adds land above bit 15 (bits 5-15 of an entry are zero).
    // The bits of the pair that pass the word (cw << (32 - nacc)) are non-zero
    // only when the word completes, so they need no second accumulator: they
    // become the next word's start.
    auto push = [&](uint32_t ea, uint32_t eb) {
      const uint32_t cw = (ea & ~31u) | __funnelshift_r(eb & ~31u, 0u, ea);  // eb's code >> la
      const uint32_t over = __funnelshift_r(0u, cw, nacc);  // cw << (32 - nacc), 0 for nacc = 0
      acc_hi |= __funnelshift_r(cw, 0u, nacc);              // cw >> nacc
      nacc += ea + eb;
      if (nacc & 32u) {
        emit(acc_hi);
        acc_hi = over;
        nacc ^= 32u;
      }
    };
    // Four codes of at most 8 bits a step: two pairs joined as above, the
    // second shifted by the first pair's length (ea + eb: its low five bits
    // are la + lb <= 16), then pushed as one code of at most 32 bits.
    auto push4 = [&](uint32_t ea, uint32_t eb, uint32_t ec, uint32_t ed) {
      const uint32_t cab = (ea & ~31u) | __funnelshift_r(eb & ~31u, 0u, ea);
      const uint32_t ccd = (ec & ~31u) | __funnelshift_r(ed & ~31u, 0u, ec);
      const uint32_t eab = ea + eb;
      const uint32_t cw = cab | __funnelshift_r(ccd, 0u, eab);  // ccd >> (la + lb)
      const uint32_t over = __funnelshift_r(0u, cw, nacc);       // cw << (32 - nacc)
      acc_hi |= __funnelshift_r(cw, 0u, nacc);                   // cw >> nacc
      nacc += eab + ec + ed;
      if (nacc & 32u) {
        emit(acc_hi);
        acc_hi = over;
        nacc ^= 32u;
      }
    };
    // one 32-symbol run at g (k symbols of it)
    auto pack_run = [&](uint32_t g, uint32_t k) {
      uint32_t x[kEncSymPerThread / 4];
      load_symbols(a.in + g, (int)k, x);
      if (kWide) {
#pragma unroll
        for (int j = 0; j < kEncSymPerThread; ++j) {
          if (k == (uint32_t)kEncSymPerThread || (uint32_t)j < k) {
            const uint2 e = sh.cl[sym_of(x, j)];
            push1(e.x, e.y);
          }
        }
      } else if (kQuad && k == (uint32_t)kEncSymPerThread) {
#pragma unroll
        for (int j = 0; j < kEncSymPerThread / 4; ++j)
          push4(sh.lent[sym_of(x, 4 * j)], sh.lent[sym_of(x, 4 * j + 1)],
                sh.lent[sym_of(x, 4 * j + 2)], sh.lent[sym_of(x, 4 * j + 3)]);
      } else if (k == (uint32_t)kEncSymPerThread) {
#pragma unroll
        for (int j = 0; j < kEncSymPerThread / 2; ++j)
          push(sh.lent[sym_of(x, 2 * j)], sh.lent[sym_of(x, 2 * j + 1)]);
      } else {
#pragma unroll
        for (int j = 0; j < kEncSymPerThread / 2; ++j)
          push((uint32_t)(2 * j) < k ? sh.lent[sym_of(x, 2 * j)] : 0u,
               (uint32_t)(2 * j + 1) < k ? sh.lent[sym_of(x, 2 * j + 1)] : 0u);
      }
    };
    // the previous item's bulk copy has read the staging area
    if (lane == 0) bulk_wait_read();
    __syncwarp();
    if (cnt0) pack_run(g0, cnt0);
    if (cnt1) pack_run(g0 + kEncSymPerThread, cnt1);
    const bool first = wi == w_first;  // no word completed
    // ---- the words shared with the lane before (or the warp before)
    nacc &= 31u;
    const uint32_t tail = nacc ? acc_hi : 0u;  // my partial last word
    uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, tail, 1);
    if (lane == 0) {
      prev = 0;
      if (r) {
        const uint32_t t = v0 ? m.warp_tail[v0 - 1] : a.meta[tile - 1].warp_tail[kWarps - 1];
        prev = (t & ((1u << r) - 1u)) << (32u - r);
      }
    }
    if (kWide && direct) {
      if (!first) gbase[w_first] = shared_head ? (fw | prev) : fw;
    } else if (shared_head && !first) {
      stw[w_first] |= prev;
    }
    // a lane that completed no word keeps its bits, and the lane before's, in
    // `tail`: only the record's last lane can (a full lane holds >= 32 bits)
    const bool own_tail = lane == last_lane && rec_end;
    if (own_tail && nacc) {
      const uint32_t v = first && shared_head ? (tail | prev) : tail;
      if (kWide && direct) gbase[wi] = v;
      else stw[wi] = v;
    }
    // ---- delimiter, index, sub-block offsets
    if (own_tail) {
      pay[-1] = p + c;  // rec_words[O1]: the record's bit count
      if ((a.flags & kFlagSub) && hi == n) put_sub_tail(a, p + c);
    }
    if (starts && v0 == 0 && lane == 0 && (a.flags & kFlagIndex))
      reinterpret_cast<uint32_t*>(a.out + kHeaderBytes)[fast_div(lo, a.fdB)] = (uint32_t)O1;
    if (a.flags & kFlagSub) {  // each run's first symbol may start a sub-block
      if (cnt0) put_sub_entry(a, g0, p);
      if (cnt1) put_sub_entry(a, g0 + kEncSymPerThread, p + c0);
    }
    __syncwarp();
    if (kWide && direct) continue;  // (uniform) already written
    // ---- copy out: staging words [off, off + nw) to gbase[off ..]; the whole
    // 16-byte chunks [c_lo, c_hi) by one bulk copy, the up to three words
    // before and after them by lanes 0-2 and 4-6 (all of them, at most six,
    // when there is no whole chunk).  The next item waits for the copy to
    // have read the staging area before it writes there.
    const uint32_t e_w = nw + off;
    const uint32_t c_lo = (off + 3u) & ~3u, c_hi = e_w & ~3u;
    if (c_hi > c_lo) {
      bulk_fence_shared();
      __syncwarp();
      if (lane == 0) bulk_store(gbase + c_lo, stw + c_lo, 4u * (c_hi - c_lo));
      if (lane < c_lo - off) gbase[off + lane] = stw[off + lane];
      else if (lane >= 4u && lane - 4u < e_w - c_hi) gbase[c_hi + lane - 4u] = stw[c_hi + lane - 4u];
    } else if (lane < nw) {
      gbase[off + lane] = stw[off + lane];
    }
  }
  if (lane == 0) bulk_wait_all();  // (the staging area outlives no copy)
}

// Load the code table of the buffer `a` describes into the packing tables.
static __device__ __forceinline__ void pack_load_tables(PackShared& sh, const EncodeArgs& a) {
  const CodeTable* ct = &a.st->codes;
  for (int s = threadIdx.x; s < 256; s += kEncThreads) {
    const uint32_t l = ct->len[s];
    const uint64_t c = ct->code[s];
    sh.len[s] = l;
    sh.code_lo[s] = (uint32_t)c;
    sh.code_hi[s] = (uint32_t)(c >> 32);
    sh.entry[s] = (uint32_t)(c << 6) | l;
    sh.lent[s] = (l && l <= 16) ? ((uint32_t)c << (32 - l)) | l : 0u;
    sh.cl[s] = (l && l <= 32) ? make_uint2((uint32_t)(c << (32 - l)), l) : make_uint2(0u, 0u);
  }
  if (threadIdx.x == 0) sh.a = a;
}

// Pack one tile of the buffer whose tables and arguments are in sh.
static __device__ __forceinline__ void pack_one_tile(PackShared& sh, uint32_t tile, uint32_t maxlen) {
  const EncodeArgs& a = sh.a;
  uint32_t* rec_words =
      reinterpret_cast<uint32_t*>(a.out + records_at(a.nb, a.B, a.flags, a.sub_S));
  const TileGeom g = tile_geom(tile, (uint32_t)a.n, a.fdB);
  const bool chunked_ok = a.fdB.d % kEncSymPerThread == 0;
  if (maxlen > 32) pack_tile_general<true>(sh, tile, g, rec_words);
  else if (!g.interior_start && maxlen <= 16) pack_tile_single<0>(sh, tile, g, rec_words);
  else if (!g.interior_start && maxlen <= 26) pack_tile_single<1>(sh, tile, g, rec_words);
  else if (!g.interior_start) pack_tile_single<2>(sh, tile, g, rec_words);
  else if (maxlen > 26) pack_tile_general<true>(sh, tile, g, rec_words);
  else if (chunked_ok && maxlen <= 16) pack_tile_chunked<true>(sh, tile, g, rec_words);
  else if (chunked_ok) pack_tile_chunked<false>(sh, tile, g, rec_words);
  else pack_tile_general<false>(sh, tile, g, rec_words);
}

}  // namespace hz
