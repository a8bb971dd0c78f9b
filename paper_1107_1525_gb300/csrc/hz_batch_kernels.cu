// hz_batch_kernels.cu -- kernels of the batched path (hz_submit / hz_poll).
//
// A batch holds any mix of compress and decompress requests over independent
// buffers of uneven sizes.  Each phase of the method runs as one persistent
// kernel over the whole batch: CTAs take work units from a ticket counter over
// a flattened (request, unit) index -- 64 KiB histogram chunks, 8192-symbol
// encoder tiles, groups of decoder blocks -- and find the request a unit
// belongs to by binary search over per-request unit prefixes.  Phases that
// need a whole request (code construction, the tile scan, decode set-up) run
// one CTA per request in a grid-stride loop.  Every launch has a fixed grid
// and reads the batch's sizes from device memory, so the host captures the
// sequence once in a CUDA graph and replays it for every batch.
#include <stddef.h>

#include "hz_batch_dev.h"
#include "hz_build_dev.cuh"
#include "hz_decode_dev.cuh"
#include "hz_encode_dev.cuh"
#include "hz_hist_dev.cuh"

namespace hz {

// Index of the request whose [base[i], base[i + 1]) range holds unit u
// (bases ascending, base[0] = 0).
__device__ __forceinline__ uint32_t find_item(const uint32_t* base, uint32_t count, uint32_t u) {
  uint32_t lo = 0, hi = count;  // last i with base[i] <= u
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(base + mid) <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Encoder tiles are handed out in chunks of consecutive tiles, so that a CTA
// mostly stays inside one request and loads its tables once per chunk: up to
// kBatchTileChunk tiles, fewer when the batch has too few tiles to give every
// CTA several chunks.
constexpr uint32_t kBatchTileChunk = 8;

__device__ __forceinline__ uint32_t tile_chunk(uint32_t ntiles) {
  const uint32_t k = ntiles / (gridDim.x * 8u);
  return k < 1 ? 1u : (k > kBatchTileChunk ? kBatchTileChunk : k);
}

// The request that holds a unit, remembered across calls: a unit inside the
// last request's range needs no search.  Works for any order of units.
struct RequestCursor {
  const uint32_t* base;
  uint32_t count, total;
  uint32_t i = 0xFFFFFFFFu, lo = 1, hi = 0;  // [lo, hi): units of request i
  __device__ __forceinline__ uint32_t find(uint32_t u) {
    if (u < lo || u >= hi) {
      i = find_item(base, count, u);
      lo = __ldg(base + i);
      hi = i + 1 < count ? __ldg(base + i + 1) : total;
    }
    return i;
  }
};

__device__ __forceinline__ EncodeArgs comp_args(const BatchComp& c) {
  EncodeArgs a;
  a.in = c.src;
  a.n = c.n;
  a.B = c.B;
  a.nb = c.nb;
  a.flags = c.flags;
  a.out = c.dst;
  a.out_cap = c.cap;
  a.out_len = c.out_len;
  a.st = c.st;
  a.tiles = c.tiles;
  a.ntiles = c.ntiles;
  a.fdB = c.fdB;
  a.tile_begin = 0;
  a.tile_end = c.ntiles;
  a.sub_S = 0;  // batched streams carry no sub-block offsets
  a.sub_M = 1;
  a.fdS = FastDiv{1, 1, 0, 0};
  a.spin_limit = kSpinLimit;  // (the batched scan runs in one CTA: no waits)
  a.meta = nullptr;
  return a;
}

__device__ __forceinline__ DecodeArgs decomp_args(const BatchDecomp& d) {
  DecodeArgs a;
  a.in = d.src;
  a.in_len = d.in_len;
  a.out = d.dst;
  a.out_cap = d.cap;
  a.out_len = d.out_len;
  a.st = d.st;
  a.chase_index = nullptr;  // batched streams must carry the block-offset index
  a.chase_cap = 0;
  a.lut_bits = (int)d.lut_bits;
  a.k_begin = 0;
  a.k_end = 0xFFFFFFFFu;
  a.defer_chase = 0;
  a.seen_no_index = nullptr;
  return a;
}

// A CTA's stream of work units from a global ticket counter.  Thread 0 asks
// for the next ticket as soon as it hands out the current one, so the atomic's
// round trip overlaps the current unit's work instead of stalling the CTA.
// Every thread of the CTA calls first() and next() (they hold barriers).
struct TicketStream {
  uint32_t* counter;
  uint32_t* slot;  // shared: the current ticket
  uint32_t ahead;  // thread 0: the ticket after it
  __device__ __forceinline__ uint32_t first() {
    if (threadIdx.x == 0) {
      *slot = atomicAdd(counter, 1u);
      ahead = atomicAdd(counter, 1u);
    }
    __syncthreads();
    return *slot;
  }
  __device__ __forceinline__ uint32_t next() {
    __syncthreads();  // every thread is done with the current unit
    if (threadIdx.x == 0) {
      *slot = ahead;
      ahead = atomicAdd(counter, 1u);
    }
    __syncthreads();
    return *slot;
  }
};

// ------------------------------------------------------------- histogram
__global__ void __launch_bounds__(kHistThreads) batch_hist_kernel(BatchCtl* ctl,
                                                                   const BatchComp* comps) {
  __shared__ uint32_t h[256 * 32];
  __shared__ uint32_t s_u;
  const uint32_t nunits = ctl->hist_units, ncomp = ctl->ncomp;
  TicketStream ts{&ctl->tickets[kTicketHist], &s_u, 0u};
  for (uint32_t u = ts.first(); u < nunits; u = ts.next()) {
    const uint32_t i = find_item(ctl->hist_base, ncomp, u);
    const BatchComp& c = comps[i];
    const uint64_t lo = (uint64_t)(u - c.hist_base) * kBatchHistChunk;
    const uint64_t len = c.n - lo < kBatchHistChunk ? c.n - lo : kBatchHistChunk;
    for (int k = threadIdx.x; k < 256 * 32; k += blockDim.x) h[k] = 0;
    __syncthreads();
    count_range(c.src + lo, len, h);
    __syncthreads();
    fold_columns(h, c.st->hist);
  }
}

// ------------------------------------------------------------- code build
__global__ void __launch_bounds__(256) batch_build_kernel(BatchCtl* ctl, const BatchComp* comps) {
  const LenParam none{};
  for (uint32_t i = blockIdx.x; i < ctl->ncomp; i += gridDim.x) {
    const BatchComp& c = comps[i];
    build_codes_device(c.st, 1, none, c.n, c.B, c.nb, c.flags, 0, c.dst, c.cap, c.out_len);
    __syncthreads();
  }
}

// ------------------------------------------------------------- tile summaries
__global__ void __launch_bounds__(kEncThreads) batch_summary_kernel(BatchCtl* ctl,
                                                                    const BatchComp* comps) {
  __shared__ uint8_t s_len[256];
  __shared__ uint32_t s_wsum[kEncThreads / 32];
  __shared__ Summary s_warp[kEncThreads / 32];
  __shared__ uint32_t s_u;
  const uint32_t ntiles = ctl->tiles, ncomp = ctl->ncomp;
  RequestCursor rc{ctl->tile_base, ncomp, ntiles};
  uint32_t loaded = 0xFFFFFFFFu;  // the request whose lengths are in s_len
  TicketStream ts{&ctl->tickets[kTicketSummary], &s_u, 0u};
  const uint32_t K = tile_chunk(ntiles);
  for (uint32_t u = ts.first(); u * K < ntiles; u = ts.next()) {
    const uint32_t t_end = min(u * K + K, ntiles);
    for (uint32_t tile = u * K; tile < t_end; ++tile) {
      const uint32_t i = rc.find(tile);
      const BatchComp& c = comps[i];
      if (c.st->codes.maxlen > (uint32_t)kMaxLen) continue;  // code construction failed
      if (i != loaded) {
        __syncthreads();  // nobody still reads the previous request's lengths
        for (int s = threadIdx.x; s < 256; s += kEncThreads) s_len[s] = c.st->codes.len[s];
        loaded = i;
        __syncthreads();
      }
      bool bad = false;
      summary_tile(comp_args(c), tile - c.tile_base, s_len, s_wsum, s_warp, bad);
      if (bad) set_error(c.st, HZ_ERR_ARG, 0x200);
    }
  }
}

// ------------------------------------------------------------- tile scan
__global__ void __launch_bounds__(kScanThreads) batch_scan_kernel(BatchCtl* ctl,
                                                                   const BatchComp* comps) {
  __shared__ Summary s_warp[kScanThreads / 32];
  __shared__ ScanState s_carry;
  for (uint32_t i = blockIdx.x; i < ctl->ncomp; i += gridDim.x) {
    const BatchComp& c = comps[i];
    if (c.ntiles == 0 || c.st->codes.maxlen > (uint32_t)kMaxLen) continue;  // uniform
    scan_tiles_cta(comp_args(c), s_warp, &s_carry);
    __syncthreads();
  }
}

// ------------------------------------------------------------- packing
__global__ void __launch_bounds__(kEncThreads, 3) batch_pack_kernel(BatchCtl* ctl,
                                                                    const BatchComp* comps) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  PackShared& sh = *reinterpret_cast<PackShared*>(smem_raw);
  __shared__ uint32_t s_u;
  const uint32_t ntiles = ctl->tiles, ncomp = ctl->ncomp;
  uint32_t maxlen = 0;
  RequestCursor rc{ctl->tile_base, ncomp, ntiles};
  uint32_t loaded = 0xFFFFFFFFu;  // the request whose tables are in sh
  TicketStream ts{&ctl->tickets[kTicketPack], &s_u, 0u};
  const uint32_t K = tile_chunk(ntiles);
  for (uint32_t u = ts.first(); u * K < ntiles; u = ts.next()) {
    const uint32_t t_end = min(u * K + K, ntiles);
    for (uint32_t tile = u * K; tile < t_end; ++tile) {
      const uint32_t i = rc.find(tile);
      const BatchComp& c = comps[i];
      if (!c.st->enc_ok || c.st->error) continue;  // uniform: nothing to pack for this request
      if (i != loaded) {
        __syncthreads();  // nobody still reads the previous request's tables
        pack_load_tables(sh, comp_args(c));
        maxlen = c.st->codes.maxlen;
        loaded = i;
        __syncthreads();
      }
      pack_one_tile(sh, tile - c.tile_base, maxlen);
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------- decode set-up
__global__ void __launch_bounds__(256) batch_dsetup_kernel(BatchCtl* ctl, BatchDecomp* decomps) {
  for (uint32_t i = blockIdx.x; i < ctl->ndecomp; i += gridDim.x) {
    BatchDecomp& d = decomps[i];
    decode_setup_device(decomp_args(d), d.T);
    __syncthreads();
  }
}

// Decode units per stream: groups of 8 warps x `per_warp` blocks, sized so a
// unit holds at least 256 KiB of output (small blocks share a table load) --
// except in streams of fewer than kDecodeGroupMinBlocks blocks, where every
// warp takes one block so that the stream spreads over more warps.
constexpr uint32_t kDecodeGroupMinBlocks = 2048;
__global__ void __launch_bounds__(1024) batch_dscan_kernel(BatchCtl* ctl, BatchDecomp* decomps) {
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_carry;
  const uint32_t n = ctl->ndecomp;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  for (uint32_t base = 0; base < n; base += blockDim.x) {
    __syncthreads();
    const uint32_t i = base + threadIdx.x;
    uint32_t units = 0;
    if (i < n) {
      BatchDecomp& d = decomps[i];
      const DecTables* T = d.T;
      if (T->ok && T->nb && T->sub_M) {
        // sub-block offsets: a unit is 8 warps of 32 sub-blocks, a lane each
        d.per_warp = 0;
        units = (T->units + 255) / 256;
      } else if (T->ok && T->nb) {
        // a stream with few blocks gives every warp one block (latency); a
        // long one groups small blocks so that a table load serves 256 KiB
        const uint32_t per_warp =
            (T->B >= (32u << 10) || T->nb < kDecodeGroupMinBlocks) ? 1u : (32u << 10) / T->B;
        d.per_warp = per_warp;
        units = (T->nb + 8 * per_warp - 1) / (8 * per_warp);
      }
    }
    uint32_t inc = units;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, dd);
      if (lane >= dd) inc += o;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    uint32_t wpre = 0, tot = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      wpre += w < warp ? s_warp[w] : 0u;
      tot += s_warp[w];
    }
    const uint32_t carry = s_carry;
    if (i < n) {
      decomps[i].unit_base = carry + wpre + inc - units;
      ctl->unit_base[i] = carry + wpre + inc - units;
    }
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + tot;
  }
  __syncthreads();
  if (threadIdx.x == 0) ctl->dec_units = s_carry;
}

// ------------------------------------------------------------- block decoding
__global__ void __launch_bounds__(kFastThreads, 3) batch_decode_kernel(BatchCtl* ctl,
                                                                    const BatchDecomp* decomps) {
  FastShared& sh = fast_sh();
  __shared__ uint32_t s_u;
  const uint32_t nunits = ctl->dec_units, n = ctl->ndecomp;
  uint32_t cur = 0xFFFFFFFFu;
  int mode = 2;
  TicketStream ts{&ctl->tickets[kTicketDecode], &s_u, 0u};
  for (uint32_t u = ts.first(); u < nunits; u = ts.next()) {
    const uint32_t i = find_item(ctl->unit_base, n, u);
    const BatchDecomp& d = decomps[i];
    const DecTables* T = d.T;
    if (i != cur) {
      load_fast_tables<false>(sh, T, threadIdx.x, kFastThreads);
      if (threadIdx.x == 0) sh.args = decomp_args(d);
      cur = i;
      __syncthreads();
      mode = fast_mode(T, sh.c);
    }
    const DecodeArgs a = decomp_args(d);
    const uint32_t warp = threadIdx.x >> 5;
    if (sh.sub_M) {  // uniform: 32 sub-blocks per warp
      const uint32_t u0 = ((u - d.unit_base) * 8 + warp) * 32;
      if (u0 < sh.units) decode_units_fast(u0, sh.units, mode);
      continue;
    }
    const uint32_t k0 = ((u - d.unit_base) * 8 + warp) * d.per_warp;
    for (uint32_t j = 0; j < d.per_warp; ++j) {
      const uint32_t k = k0 + j;
      if (k >= sh.c.nb) break;
      decode_block_fast(a, k, mode);
    }
  }
}

// ------------------------------------------------------------- results
__global__ void batch_finish_kernel(BatchCtl* ctl, const BatchComp* comps,
                                    const BatchDecomp* decomps, BatchResult* results) {
  const uint32_t nc = ctl->ncomp, nd = ctl->ndecomp;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nc + nd;
       i += gridDim.x * blockDim.x) {
    const bool is_c = i < nc;
    DevState* st = is_c ? comps[i].st : decomps[i - nc].st;
    const uint64_t* len = is_c ? comps[i].out_len : decomps[i - nc].out_len;
    BatchResult r;
    r.req = is_c ? comps[i].req : decomps[i - nc].req;
    r.status = -(int32_t)st->error;
    r.out_len = *len;
    results[i] = r;
  }
}

// ------------------------------------------------------------- per-request state
// Clear what must start at zero in every request's state: status words,
// counters, histogram, scan flags (everything before the code table); and
// copy each compress request's first histogram unit and tile into the
// compact arrays the unit search reads.
__global__ void batch_clear_kernel(BatchCtl* ctl, const BatchComp* comps,
                                   const BatchDecomp* decomps) {
  constexpr uint32_t kWords = (uint32_t)(offsetof(DevState, codes) / 4);
  const uint32_t nc = ctl->ncomp, nd = ctl->ndecomp;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    ctl->hist_base[i] = comps[i].hist_base;
    ctl->tile_base[i] = comps[i].tile_base;
  }
  for (uint32_t i = blockIdx.x; i < nc + nd; i += gridDim.x) {
    uint32_t* w = reinterpret_cast<uint32_t*>(i < nc ? comps[i].st : decomps[i - nc].st);
    for (uint32_t k = threadIdx.x; k < kWords; k += blockDim.x) w[k] = 0;
  }
}

// ------------------------------------------------------------- launch sequence
void batch_configure() {
  cudaFuncSetAttribute(batch_pack_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(PackShared));
  cudaFuncSetAttribute(batch_decode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fast_smem_bytes(kFastThreads));
}

void batch_enqueue(const BatchLaunch& L, cudaStream_t s) {
  const int sms = L.num_sms;
  batch_clear_kernel<<<sms * 2, 256, 0, s>>>(L.ctl, L.comps, L.decomps);
  batch_hist_kernel<<<sms * kHistCtasPerSm, kHistThreads, 0, s>>>(L.ctl, L.comps);
  batch_build_kernel<<<sms * 2, 256, 0, s>>>(L.ctl, L.comps);
  batch_summary_kernel<<<sms * 6, kEncThreads, 0, s>>>(L.ctl, L.comps);
  batch_scan_kernel<<<sms * 2, kScanThreads, 0, s>>>(L.ctl, L.comps);
  batch_pack_kernel<<<sms * 3, kEncThreads, (int)sizeof(PackShared), s>>>(L.ctl, L.comps);
  batch_dsetup_kernel<<<sms * 2, 256, 0, s>>>(L.ctl, L.decomps);
  batch_dscan_kernel<<<1, 1024, 0, s>>>(L.ctl, L.decomps);
  batch_decode_kernel<<<sms * 4, kFastThreads, fast_smem_bytes(kFastThreads), s>>>(L.ctl,
                                                                                 L.decomps);
  batch_finish_kernel<<<sms, 256, 0, s>>>(L.ctl, L.comps, L.decomps, L.results);
}

size_t batch_dec_tables_bytes() { return sizeof(DecTables); }

}  // namespace hz
