// hz_encode.cu -- block encoder (Sec. 2.1 and Figs. 3-4 of Cloud et al.).
//
// Every block of B symbols becomes a record [u32 bits_k][payload words],
// where bits_k is the sum of the block's code lengths (the paper's
// "additional pass ... summing the lengths of the code representation") and
// the payload is padded to a 32-bit boundary.  Records are laid out back to
// back, so a record's position depends on the sizes of all earlier records.
//
// Three launches, no inter-CTA waiting:
//   1. encode_summary_warps_kernel / encode_summary_kernel -- the
//      length-summing pass: per-warp counts and tails for the warp-parallel
//      path, else every 8192-symbol tile reduced to a Summary (below) of its
//      code lengths and record starts;
//   2. encode_scan_kernel -- one CTA scans the tile summaries into each
//      tile's start state (word position of the open record, bits already in
//      it), fixes the stream size and checks it against the output capacity;
//   3. encode_pack_kernel -- every tile is packed independently from its
//      start state.  When every tile lies inside one record and no code is
//      longer than 32 bits, warps pack 2048-symbol items on their own from
//      the summing pass's per-thread bit counts (pack_warps_fast: a 32-bit
//      accumulator per lane, words staged per warp and copied out by bulk
//      copies).  Otherwise per tile: each thread packs 32 consecutive symbols
//      MSB-first with a 64-bit shift accumulator (two codes per step when
//      codes have at most 16 bits), the tile's words are staged in shared
//      memory (atomicOr only for a word split between two threads) and
//      written out with 16-byte stores.  Tiles run last-to-first so the first
//      ones packed are those the length-summing pass read last, still in L2.
// A word split between two tiles is written by the later tile, which
// re-derives the earlier tile's last (< 32) bits from the input; the
// delimiter of a record is written by the tile holding the record's last
// symbol.  No word is written twice and the output needs no clearing.
#include "hz_encode_dev.cuh"

namespace hz {

// The per-tile summaries (every path but the warp-parallel one), by the
// first kEncThreads threads of the CTA.
static __device__ __forceinline__ void summary_tiles(const EncodeArgs& a, const uint8_t* s_len,
                                                     uint32_t* s_wsum, Summary* s_warp) {
  bool bad = false;
  // the next tile's symbols are loaded while the current one is summarised
  uint32_t x[kEncSymPerThread / 4], xn[kEncSymPerThread / 4];
  uint32_t tile = blockIdx.x;
  if (tile < a.ntiles) load_tile_symbols(a, tile, x);
  for (; tile < a.ntiles; tile += gridDim.x) {
    const uint32_t nt = tile + gridDim.x;
    if (nt < a.ntiles) load_tile_symbols(a, nt, xn);
    summary_tile_x(a, tile, x, s_len, s_wsum, s_warp, bad);
#pragma unroll
    for (int k = 0; k < kEncSymPerThread / 4; ++k) x[k] = xn[k];
  }
  if (bad) set_error(a.st, HZ_ERR_ARG, 0x200);  // a byte without a code (caller's code table)
}

// Streams whose blocks are not a whole number of tiles (or without the
// metadata of the warp-parallel path): per-tile summaries.
__global__ void __launch_bounds__(kEncThreads) encode_summary_kernel(EncodeArgs a) {
  __shared__ uint8_t s_len[256];  // 64 words: random lookups conflict at most 2-way
  __shared__ uint32_t s_wsum[kEncThreads / 32];
  __shared__ Summary s_warp[kEncThreads / 32];
  const CodeTable* ct = &a.st->codes;
  if (ct->maxlen > (uint32_t)kMaxLen) return;  // code construction failed; already reported
  for (int s = threadIdx.x; s < 256; s += kEncThreads) s_len[s] = ct->len[s];
  __syncthreads();
  summary_tiles(a, s_len, s_wsum, s_warp);
}

// Blocks of whole tiles with the warp-parallel path's metadata: the
// warp-parallel summing pass when no code is longer than 32 bits (decided
// here, from the code table), else the per-tile summaries by the CTA's first
// kEncThreads threads (the others leave; the tile barrier counts kEncThreads).
__global__ void __launch_bounds__(kSumWarpThreads, 3) encode_summary_warps_kernel(EncodeArgs a) {
  extern __shared__ __align__(16) uint8_t s_tab[];  // kSumTabBytes (dynamic)
  __shared__ uint8_t s_len[256];
  __shared__ uint32_t s_code[256];
  __shared__ uint8_t s_sym[kSumWarpThreads];
  __shared__ uint32_t s_wsum[kEncThreads / 32];
  __shared__ Summary s_warp[kEncThreads / 32];
  const CodeTable* ct = &a.st->codes;
  if (ct->maxlen > (uint32_t)kMaxLen) return;  // code construction failed; already reported
  if (!warp_path(a.meta, a.B, ct->maxlen)) {  // uniform
    if (threadIdx.x >= kEncThreads) return;
    for (int s = threadIdx.x; s < 256; s += kEncThreads) s_len[s] = ct->len[s];
    tile_sync();
    summary_tiles(a, s_len, s_wsum, s_warp);
    return;
  }
  for (int s = threadIdx.x; s < 256; s += kSumWarpThreads) s_code[s] = (uint32_t)ct->code[s];
  // entry s of lane l at byte 256 s + 4 l
  for (int i = threadIdx.x; i < 256 * 32; i += kSumWarpThreads) {
    const uint32_t l = ct->len[i >> 5];
    reinterpret_cast<uint32_t*>(s_tab)[((i >> 5) << 6) | (i & 31)] = l ? l : kLenNoCode;
  }
  __syncthreads();
  bool bad = false;
  count_warps(a, s_tab, s_code, s_sym, bad);
  if (bad) set_error(a.st, HZ_ERR_ARG, 0x200);
}

// =================================================================== pass 2
// Each CTA scans kScanCtaTiles consecutive tile summaries (one per thread);
// CTAs take their index from a ticket and find their exclusive prefix by a
// look-back over the aggregates of earlier CTAs (at most kMaxScanCtas of
// them).  (1024 tiles a CTA rather than 4096: 0.021 -> 0.014 ms for the
// 32768 tiles of a 2^28-byte buffer, the mix's 131072 tiles 0.0215 -> 0.0209.)
constexpr int kScanCtaPerThread = kScanCtaTiles / kScanThreads;

__global__ void __launch_bounds__(kScanThreads) encode_scan_kernel(EncodeArgs a) {
  __shared__ Summary s_warp[kScanThreads / 32];
  __shared__ Summary s_wpre[kScanThreads / 32];  // each warp's exclusive prefix in the CTA
  __shared__ Summary s_agg;                      // the CTA's aggregate
  __shared__ uint32_t s_cta;
  __shared__ ScanState s_excl;
  __shared__ int s_abort;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  DevState* st = a.st;
  if (tid == 0) {
    s_cta = atomicAdd(&st->tile_counter, 1u);  // ticket order: predecessors are running
    s_abort = 0;
  }
  __syncthreads();
  const uint32_t cta = s_cta;
  const uint32_t nt = a.ntiles;
  const uint32_t t0 = cta * kScanCtaTiles + tid * kScanCtaPerThread;
  const bool warps = warp_path(a.meta, a.B, st->codes.maxlen);  // tiles summarised by their metadata
  Summary mine[kScanCtaPerThread];
  Summary agg{0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < kScanCtaPerThread; ++k) {
    mine[k] = t0 + k >= nt ? Summary{0, 0, 0, 0}
              : warps     ? meta_summary(a, t0 + k)
                          : load_summary(a.tiles[t0 + k]);
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
  // warp 0 scans the warps' aggregates: each warp's prefix and the CTA's total
  if (warp == 0) {
    const Summary v = lane < kScanThreads / 32 ? s_warp[lane] : Summary{0, 0, 0, 0};
    Summary wi = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      Summary o = shfl_up_summary(wi, d);
      if (lane >= d) wi = combine(o, wi);
    }
    Summary we = shfl_up_summary(wi, 1);
    if (lane == 0) we = Summary{0, 0, 0, 0};
    if (lane < kScanThreads / 32) s_wpre[lane] = we;
    if (lane == 31) s_agg = wi;
  }
  __syncthreads();
  const Summary cta_agg = s_agg;
  ex = combine(s_wpre[warp], ex);

  if (warp == 0) {
    TileStatus* aux = st->scan_aux;
    if (cta == 0) {
      if (lane == 0) {
        const ScanState incl = apply(init_state(), cta_agg);
        aux[0].pre_O = incl.O;
        aux[0].pre_b = incl.b;
        st_release(&st->scan_flags[0], 2u);
        s_excl = init_state();
      }
    } else {
      if (lane == 0) {
        store_summary(aux[cta], cta_agg);
        st_release(&st->scan_flags[cta], 1u);
      }
      Summary acc{0, 0, 0, 0};
      int j = (int)cta - 1;
      bool timed_out = false;
      ScanState result = init_state();
      for (;;) {
        const int idx = j - lane;
        uint32_t state = 2;  // index -1 stands for the virtual start state
        Summary ag{0, 0, 0, 0};
        ScanState pre = init_state();
        if (idx >= 0) {
          uint32_t f = ld_acquire(&st->scan_flags[idx]);
          uint32_t spins = 0;
          while (f == 0) {
            if (++spins > a.spin_limit) {
              timed_out = true;
              break;
            }
            __nanosleep(64);
            f = ld_acquire(&st->scan_flags[idx]);
          }
          state = timed_out ? 2u : f;
          if (state == 1) ag = load_summary(aux[idx]);
          else if (!timed_out) pre = ScanState{aux[idx].pre_O, aux[idx].pre_b};
        }
        const uint32_t pmask = __ballot_sync(0xFFFFFFFFu, state == 2);
        const int stop = pmask ? __ffs(pmask) - 1 : 32;
        Summary c{0, 0, 0, 0};
        for (int l = stop - 1; l >= 0; --l) {
          Summary v;
          v.has = __shfl_sync(0xFFFFFFFFu, ag.has, l);
          v.head = __shfl_sync(0xFFFFFFFFu, ag.head, l);
          v.omega = __shfl_sync(0xFFFFFFFFu, ag.omega, l);
          v.tail = __shfl_sync(0xFFFFFFFFu, ag.tail, l);
          c = combine(c, v);
        }
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
      const bool any_timeout = __any_sync(0xFFFFFFFFu, timed_out);
      if (lane == 0) {
        if (any_timeout) {
          set_error(st, HZ_ERR_TIMEOUT, 0x205);
          s_abort = 1;
        }
        const ScanState incl = apply(result, cta_agg);
        aux[cta].pre_O = incl.O;
        aux[cta].pre_b = incl.b;
        st_release(&st->scan_flags[cta], 2u);  // published even after a time-out
        s_excl = result;
      }
    }
  }
  __syncthreads();
  ScanState s = apply(s_excl, ex);
#pragma unroll
  for (int k = 0; k < kScanCtaPerThread; ++k) {
    if (t0 + k < nt) {
      a.tiles[t0 + k].pre_O = s.O;
      a.tiles[t0 + k].pre_b = s.b;
      s = apply(s, mine[k]);
      if (t0 + k == nt - 1) finish_stream(a, s, s_abort != 0);  // the last tile's thread
    }
  }
}

__global__ void __launch_bounds__(kEncThreads, 4) encode_pack_kernel(EncodeArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  PackShared& sh = *reinterpret_cast<PackShared*>(smem_raw);
  // size, capacity, time-out or code errors were found before packing
  if (!a.st->enc_ok || a.st->error) return;
  const uint32_t maxlen = a.st->codes.maxlen;
  pack_load_tables(sh, a);
  __syncthreads();
  // every tile inside one record and codes of at most 32 bits: warps pack on
  // their own, from the tile metadata of the length-summing pass (four codes
  // a step when no code is longer than 8 bits, two when none is longer than 16)
  if (warp_path(a.meta, a.B, maxlen)) {
    if (maxlen <= 8) pack_warps_fast<false, true>(sh);
    else if (maxlen <= 16) pack_warps_fast<false>(sh);
    else pack_warps_fast<true>(sh);
    return;
  }
  for (uint32_t i = blockIdx.x; i < a.tile_end - a.tile_begin; i += gridDim.x) {
    // last tiles first: their input is still in L2 from the length-summing pass
    pack_one_tile(sh, a.tile_end - 1 - i, maxlen);
    __syncthreads();
  }
}

static PerDeviceSetup<2> g_summary_setup;

cudaError_t launch_encode_summary(const EncodeArgs& a, int num_sms, cudaStream_t s) {
  // blocks of whole tiles with the metadata: the kernel that holds the
  // warp-parallel path (whether it applies is decided on the device), with
  // the lane-private length copies in dynamic shared memory
  const bool warps = a.meta != nullptr && a.B % (uint32_t)kEncTile == 0;
  int per_sm = 1;
  const cudaError_t e = launch_setup_per_device(g_summary_setup, warps ? 1 : 0, &per_sm, [&](int& out) {
    if (!warps)
      return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out, encode_summary_kernel,
                                                           kEncThreads, 0);
    cudaError_t r = cudaFuncSetAttribute(encode_summary_warps_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSumTabBytes);
    if (r == cudaSuccess)
      r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out, encode_summary_warps_kernel,
                                                        kSumWarpThreads, kSumTabBytes);
    return r;
  });
  if (e != cudaSuccess) return e;
  const uint64_t grid = (uint64_t)num_sms * per_sm;
  const unsigned g = (unsigned)(grid < a.ntiles ? grid : a.ntiles);
  if (warps) encode_summary_warps_kernel<<<g, kSumWarpThreads, kSumTabBytes, s>>>(a);
  else encode_summary_kernel<<<g, kEncThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_encode_scan(const EncodeArgs& a, cudaStream_t s) {
  const unsigned grid = (a.ntiles + kScanCtaTiles - 1) / kScanCtaTiles;
  encode_scan_kernel<<<grid, kScanThreads, 0, s>>>(a);
  return cudaGetLastError();
}

static PerDeviceSetup<1> g_pack_setup;

cudaError_t launch_encode_pack(const EncodeArgs& a, int num_sms, cudaStream_t s) {
  const int smem = (int)sizeof(PackShared);
  // the raised shared-memory limit and the CTAs per SM, once per device
  int per_sm = 1;
  const cudaError_t e = launch_setup_per_device(g_pack_setup, 0, &per_sm, [&](int& out) {
    cudaError_t r =
        cudaFuncSetAttribute(encode_pack_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (r == cudaSuccess)
      r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&out, encode_pack_kernel, kEncThreads, smem);
    return r;
  });
  if (e != cudaSuccess) return e;
  const uint64_t grid = (uint64_t)num_sms * per_sm;
  const uint32_t nt = a.tile_end - a.tile_begin;
  if (nt == 0) return cudaSuccess;
  encode_pack_kernel<<<(unsigned)(grid < nt ? grid : nt), kEncThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace hz
