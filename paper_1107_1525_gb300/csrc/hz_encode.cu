// hz_encode.cu -- block encoder (Sec. 2.1 and Figs. 3-4 of Cloud et al.).
//
// Every block of B symbols becomes a record [u32 bits_k][payload words],
// where bits_k is the sum of the block's code lengths (the paper's "additional
// pass ... summing the lengths of the code representation") and the payload
// is padded to a 32-bit boundary.  Records are laid out back to back, so the
// position of every record depends on the sizes of all earlier ones.
//
// One kernel does the whole encode in a single read of the input:
//   * persistent CTAs take 8192-symbol tiles from a ticket counter, so a tile
//     only ever waits on tiles that are already running;
//   * each thread holds 32 consecutive symbols in registers and summarises
//     them as a segment (see Summary below) -- this is the length-sum pass,
//     fused with the load;
//   * a CTA scan combines the thread summaries, and a decoupled look-back over
//     earlier tiles (32 predecessors per warp step) yields the tile's exclusive
//     prefix: the word position of the open record and the bits already in it;
//   * each thread then packs its codes, MSB first, into 32-bit words with a
//     64-bit shift accumulator, staging the tile's words in shared memory
//     (shared-memory atomicOr only for words split between two threads), and
//     the CTA writes the staged words out with coalesced stores;
//   * a word split between two tiles is written by the later tile, which
//     re-derives the earlier tile's last (< 32) bits from the input; the
//     delimiter of a record that spans tiles is written by the tile holding
//     the record's last symbol.  No word is ever written twice, and the output
//     buffer needs no clearing.
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

__device__ __forceinline__ Summary combine(const Summary& a, const Summary& x) {  // a, then x
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

__device__ __forceinline__ ScanState apply(const ScanState& s, const Summary& x) {
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

__device__ __forceinline__ Summary shfl_summary(const Summary& v, int src) {
  Summary r;
  r.has = __shfl_sync(0xFFFFFFFFu, v.has, src);
  r.head = __shfl_sync(0xFFFFFFFFu, v.head, src);
  r.omega = __shfl_sync(0xFFFFFFFFu, v.omega, src);
  r.tail = __shfl_sync(0xFFFFFFFFu, v.tail, src);
  return r;
}

__device__ __forceinline__ Summary shfl_up_summary(const Summary& v, int d) {
  Summary r;
  r.has = __shfl_up_sync(0xFFFFFFFFu, v.has, d);
  r.head = __shfl_up_sync(0xFFFFFFFFu, v.head, d);
  r.omega = __shfl_up_sync(0xFFFFFFFFu, v.omega, d);
  r.tail = __shfl_up_sync(0xFFFFFFFFu, v.tail, d);
  return r;
}

struct EncShared {
  uint32_t entry[256];       // code << 6 | len   (codes of up to 26 bits)
  uint32_t len[256];
  uint32_t code_lo[256];
  uint32_t code_hi[256];
  Summary warp_sum[kEncThreads / 32];
  uint32_t stage[kEncStageWords];
  ScanState excl;            // tile exclusive prefix
  Summary agg;               // tile aggregate
  uint32_t tile;
  uint32_t prev_bits;        // bits of the previous tile in this tile's first word
  uint32_t abort;
};

__device__ __forceinline__ uint32_t sym_of(const uint32_t (&x)[kEncSymPerThread / 4], int i) {
  return (x[i >> 2] >> (8 * (i & 3))) & 0xFFu;
}

// Writer for one thread's words: words inside the current staging window go
// to shared memory, others are dropped (a later window pass writes them).
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

template <bool kLong>
__device__ __forceinline__ void lookup(const EncShared& sh, uint32_t sym, uint32_t& l,
                                       uint64_t& c) {
  if (!kLong) {
    uint32_t e = sh.entry[sym];
    l = e & 63u;
    c = e >> 6;
  } else {
    l = sh.len[sym];
    c = ((uint64_t)sh.code_hi[sym] << 32) | sh.code_lo[sym];
  }
}

template <bool kLong>
__device__ void encode_tile(const EncodeArgs& a, EncShared& sh, uint32_t tile,
                            const uint8_t* __restrict__ rec_area) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t n = a.n;
  const uint32_t B = a.B;
  const uint64_t tile_lo = (uint64_t)tile * kEncTile;
  const uint64_t tile_hi = tile_lo + kEncTile < n ? tile_lo + kEncTile : n;
  const uint64_t g0 = tile_lo + (uint64_t)tid * kEncSymPerThread;
  const int my_cnt = g0 >= tile_hi ? 0 : (int)((tile_hi - g0) < (uint64_t)kEncSymPerThread
                                                   ? (tile_hi - g0)
                                                   : kEncSymPerThread);

  // ---- load 32 symbols (two 16-byte loads when possible)
  uint32_t x[kEncSymPerThread / 4];
  const uint8_t* src = a.in + g0;
  if (my_cnt == kEncSymPerThread && (((uintptr_t)src) & 15) == 0) {
    uint4 v0 = __ldg(reinterpret_cast<const uint4*>(src));
    uint4 v1 = __ldg(reinterpret_cast<const uint4*>(src) + 1);
    x[0] = v0.x; x[1] = v0.y; x[2] = v0.z; x[3] = v0.w;
    x[4] = v1.x; x[5] = v1.y; x[6] = v1.z; x[7] = v1.w;
  } else {
#pragma unroll
    for (int w = 0; w < kEncSymPerThread / 4; ++w) x[w] = 0;
    for (int i = 0; i < my_cnt; ++i) x[i >> 2] |= (uint32_t)src[i] << (8 * (i & 3));
  }

  // ---- segment summary of my symbols (Sec. 2.1's length-summing pass)
  const uint32_t r0 = (uint32_t)(g0 % B);
  const uint32_t first_start = r0 == 0 ? 0u : B - r0;  // offset of my first record start
  Summary s{0, 0, 0, 0};
  bool bad = false;
  {
    uint32_t next_start = first_start;
#pragma unroll
    for (int i = 0; i < kEncSymPerThread; ++i) {
      if (i < my_cnt) {
        uint32_t l;
        uint64_t c;
        lookup<kLong>(sh, sym_of(x, i), l, c);
        bad |= l == 0;
        if ((uint32_t)i == next_start) {
          if (s.has) s.omega += 1 + ceil32(s.tail);
          s.has = 1;
          s.tail = 0;
          next_start += B;
        }
        if (s.has) s.tail += l;
        else s.head += l;
      }
    }
  }
  if (bad) {
    set_error(a.st, HZ_ERR_ARG, 0x200);  // a byte without a code (given code table)
    sh.abort = 1;  // seen by all threads after the scan's barrier
  }

  // ---- CTA scan of summaries: warp inclusive scan, then across warps
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
  Summary wpre{0, 0, 0, 0};
  for (int w = 0; w < warp; ++w) wpre = combine(wpre, sh.warp_sum[w]);
  ex = combine(wpre, ex);  // exclusive within the tile
  if (tid == kEncThreads - 1) sh.agg = combine(wpre, inc);
  __syncthreads();

  // ---- decoupled look-back across tiles (warp 0)
  const uint32_t ep = a.epoch << 2;
  if (warp == 0) {
    const Summary agg = sh.agg;
    TileStatus* ts = a.tiles;
    if (tile == 0) {
      if (lane == 0) {
        ScanState init{~0ull, 0};
        ScanState incl = apply(init, agg);
        ts[0].pre_O = incl.O;
        ts[0].pre_b = incl.b;
        ts[0].has_head = (agg.has << 31) | agg.head;
        ts[0].omega = agg.omega;
        ts[0].tail = agg.tail;
        st_release(&ts[0].flag, ep | 2u);
        sh.excl = init;
      }
    } else {
      if (lane == 0) {
        ts[tile].has_head = (agg.has << 31) | agg.head;
        ts[tile].omega = agg.omega;
        ts[tile].tail = agg.tail;
        st_release(&ts[tile].flag, ep | 1u);
      }
      Summary acc{0, 0, 0, 0};
      int64_t j = (int64_t)tile - 1;
      bool timed_out = false;
      ScanState result{~0ull, 0};
      for (;;) {
        const int64_t idx = j - lane;
        uint32_t state = 2;  // index -1 stands for the virtual start state
        Summary mine{0, 0, 0, 0};
        ScanState pre{~0ull, 0};
        if (idx >= 0) {
          uint32_t f = ld_acquire(&ts[idx].flag);
          uint32_t spins = 0;
          while ((f & ~3u) != ep || (f & 3u) == 0) {
            if (++spins > kSpinLimit) { timed_out = true; break; }
            __nanosleep(32);
            f = ld_acquire(&ts[idx].flag);
          }
          state = timed_out ? 2u : (f & 3u);
          if (state == 1) {
            uint32_t hh = ts[idx].has_head;
            mine = Summary{hh >> 31, hh & 0x7FFFFFFFu, ts[idx].omega, ts[idx].tail};
          } else if (!timed_out) {
            pre = ScanState{ts[idx].pre_O, ts[idx].pre_b};
          }
        }
        const uint32_t pmask = __ballot_sync(0xFFFFFFFFu, state == 2);
        const int stop = pmask ? __ffs(pmask) - 1 : 32;
        // combine aggregates of lanes stop-1 .. 0 (oldest first), then what came before
        Summary c{0, 0, 0, 0};
        for (int l = (stop < 32 ? stop : 32) - 1; l >= 0; --l) c = combine(c, shfl_summary(mine, l));
        acc = combine(c, acc);
        if (stop < 32) {
          ScanState p;
          p.O = __shfl_sync(0xFFFFFFFFu, pre.O, stop);
          p.b = __shfl_sync(0xFFFFFFFFu, pre.b, stop);
          result = apply(p, acc);
          break;
        }
        j -= 32;
      }
      if (__any_sync(0xFFFFFFFFu, timed_out)) {
        if (lane == 0) {
          set_error(a.st, HZ_ERR_TIMEOUT, 0x201);
          sh.abort = 1;
        }
      }
      if (lane == 0) {
        ScanState incl = apply(result, agg);
        ts[tile].pre_O = incl.O;
        ts[tile].pre_b = incl.b;
        st_release(&ts[tile].flag, ep | 2u);
        sh.excl = result;
      }
    }
  }
  __syncthreads();

  // the prefix has been published either way, so successors never wait on an aborted tile
  if (sh.abort) return;

  // ---- the tile's word range and the words it must not write
  const ScanState S_s = sh.excl;
  const Summary agg = sh.agg;
  const ScanState S_e = apply(S_s, agg);
  const bool starts_record = (tile_lo % B) == 0;
  const bool ends_record = (tile_hi % B) == 0 || tile_hi == n;
  const uint64_t w_first = starts_record ? S_s.O + 1 + ceil32(S_s.b) : S_s.O + 1 + (S_s.b >> 5);
  const uint64_t w_last = S_e.O + 1 + ((S_e.b - 1) >> 5);
  const bool skip_last = !ends_record && (S_e.b & 31u) != 0;
  const bool skip_open = !ends_record && S_e.O >= w_first && S_e.O <= w_last;
  const uint32_t r_prev = starts_record ? 0u : (S_s.b & 31u);
  // a tile spans at most 3 words per symbol (delimiter + a 64-bit code), plus slack
  if (S_e.b == 0 || w_last < w_first || w_last - w_first > 3ull * kEncTile + 64) {
    if (tid == 0) set_error(a.st, HZ_ERR_ARG, 0x204);
    return;
  }
  if (tid == 0) {
    uint32_t pv = 0;
    if (r_prev) {
      // the last r_prev payload bits before this tile, from the preceding symbols
      uint64_t v = 0;
      uint32_t got = 0;
      int64_t jj = (int64_t)tile_lo - 1;
      while (got < r_prev && jj >= 0) {
        uint32_t l;
        uint64_t c;
        lookup<kLong>(sh, a.in[jj], l, c);
        if (got < 64) v |= c << got;
        got += l;
        --jj;
      }
      pv = (uint32_t)(v & ((1u << r_prev) - 1u));
    }
    sh.prev_bits = pv;
  }

  const uint64_t rec_bytes_base = (uint64_t)(rec_area - a.out);
  const uint64_t nwin = w_last - w_first + 1;
  const ScanState S_t = apply(S_s, ex);  // state before my first symbol

  for (uint64_t wlo = w_first; wlo <= w_last; wlo += kEncStageWords) {
    const uint64_t whi = wlo + kEncStageWords < w_last + 1 ? wlo + kEncStageWords : w_last + 1;
    for (int i = tid; i < kEncStageWords; i += kEncThreads) sh.stage[i] = 0;
    __syncthreads();
    if (tid == 0 && wlo == w_first && r_prev) sh.stage[0] = sh.prev_bits << (32 - r_prev);
    __syncthreads();

    // ---- pack my codes
    Emitter em{sh.stage, wlo, whi};
    ScanState cur = S_t;
    uint64_t wcur = cur.O + 1 + (cur.b >> 5);
    uint32_t nacc = cur.b & 31u;
    bool first_shared = nacc != 0;
    uint64_t acc = 0;
    uint32_t next_start = first_start;
    uint64_t next_end = (g0 / B + 1) * (uint64_t)B;  // one past the last symbol of my first record
    if (next_end > n) next_end = n;
#pragma unroll
    for (int i = 0; i < kEncSymPerThread; ++i) {
      if (i < my_cnt) {
        if ((uint32_t)i == next_start) {
          if (nacc) em.put(wcur, (uint32_t)(acc << (32 - nacc)), true);
          cur.O = cur.O + 1 + ceil32(cur.b);
          cur.b = 0;
          const uint64_t k = (g0 + i) / B;
          if ((a.flags & kFlagIndex) && wlo == w_first) {
            if (cur.O > 0xFFFFFFFFull) set_error(a.st, HZ_ERR_CAPACITY, 0x202);
            else if (kHeaderBytes + 4 * (k + 1) <= a.out_cap)
              reinterpret_cast<uint32_t*>(a.out + kHeaderBytes)[k] = (uint32_t)cur.O;
          }
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
          // emit the high (l - 32) bits, then the low 32
          uint32_t lh = l - 32;
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
        if (g0 + i + 1 == next_end) {
          // last symbol of a record: its delimiter is now known
          if (cur.O >= wlo && cur.O < whi) {
            sh.stage[cur.O - wlo] = cur.b;
          } else if (cur.O < w_first && wlo == w_first) {
            const uint64_t off = rec_bytes_base + 4 * cur.O;
            if (off + 4 <= a.out_cap) *reinterpret_cast<uint32_t*>(a.out + off) = cur.b;
          }
          next_end += B;
          if (next_end > n) next_end = n;
        }
      }
    }
    if (nacc && my_cnt) em.put(wcur, (uint32_t)(acc << (32 - nacc)), true);
    __syncthreads();

    // ---- write the window out (coalesced)
    const uint64_t cnt_w = whi - wlo;
    for (uint64_t i = tid; i < cnt_w; i += kEncThreads) {
      const uint64_t w = wlo + i;
      if ((skip_last && w == w_last) || (skip_open && w == S_e.O)) continue;
      const uint64_t off = rec_bytes_base + 4 * w;
      if (off + 4 <= a.out_cap) *reinterpret_cast<uint32_t*>(a.out + off) = sh.stage[i];
    }
    __syncthreads();
  }
  (void)nwin;

  // ---- the thread holding the last symbol knows the stream size
  if (my_cnt && g0 + my_cnt == n) {
    const uint64_t total = rec_bytes_base + 4 * (S_e.O + 1 + ceil32(S_e.b));
    *a.out_len = total;
    if (total > a.out_cap) set_error(a.st, HZ_ERR_CAPACITY, 0x203);
  }
}

__global__ void __launch_bounds__(kEncThreads, 2) encode_kernel(EncodeArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  EncShared& sh = *reinterpret_cast<EncShared*>(smem_raw);
  const CodeTable* ct = &a.st->codes;
  const uint32_t maxlen = ct->maxlen;
  if (maxlen > (uint32_t)kMaxLen) return;  // code construction failed; already reported
  for (int s = threadIdx.x; s < 256; s += blockDim.x) {
    uint32_t l = ct->len[s];
    uint64_t c = ct->code[s];
    sh.len[s] = l;
    sh.code_lo[s] = (uint32_t)c;
    sh.code_hi[s] = (uint32_t)(c >> 32);
    sh.entry[s] = (uint32_t)(c << 6) | l;
  }
  const uint8_t* rec_area = a.out + kHeaderBytes + ((a.flags & kFlagIndex) ? 4ull * a.nb : 0ull);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      sh.tile = atomicAdd(&a.st->tile_counter, 1u);
      sh.abort = 0;
    }
    __syncthreads();
    const uint32_t tile = sh.tile;
    if (tile >= a.ntiles) break;
    if (maxlen <= 26) encode_tile<false>(a, sh, tile, rec_area);
    else encode_tile<true>(a, sh, tile, rec_area);
  }
}

cudaError_t launch_encode(const EncodeArgs& a, int num_sms, cudaStream_t s) {
  static bool configured = false;
  const int smem = (int)sizeof(EncShared);
  if (!configured) {
    cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    configured = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, encode_kernel, kEncThreads, smem);
  if (per_sm < 1) per_sm = 1;
  uint64_t grid = (uint64_t)num_sms * per_sm;
  if (grid > a.ntiles) grid = a.ntiles;
  if (grid < 1) grid = 1;
  encode_kernel<<<(unsigned)grid, kEncThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace hz
