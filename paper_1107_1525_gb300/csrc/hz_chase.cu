// hz_chase.cu -- the record offsets of a stream without a stored index
// (flags bit 0 clear), found in parallel.
//
// The paper finds block i by following the delimiters of blocks 0..i-1 (Sec.
// 2.1): one dependent load per record.  Here every record-area word that
// could start a record is a candidate:
//   - its value v (the record's payload bits) lies between the fewest and the
//     most bits a block can hold (symbols x shortest / longest code);
//   - the record, 1 + ceil(v / 32) words, fits before the end of the stream;
//   - the padding bits of its last payload word are zero.
// Candidates are numbered through a bitmap and prefix counts.  Each points to
// the candidate where its record would end (or to the end of the stream, or
// nowhere), and pointer jumping gives every candidate the number of records
// from it to the end.  Every true record start is a candidate, and record k
// is nb - k records from the end.  A slot k claimed by one candidate is record
// k.  False chains that run into the true one also claim slots; through such
// a run the true records are followed from the record before it, one
// successor at a time, and the walk must arrive at the record after the run.
// A slot nobody claims means a corrupt stream (or scratch too small): then one
// thread walks the delimiters as the paper does, and the decoder reports the
// error.
//
// One cooperative launch: every CTA is resident, and the phases are separated
// by a grid barrier whose waits are bounded (HZ_ERR_TIMEOUT when one runs out).
#include "hz_chase.h"
#include "hz_decode_dev.cuh"

namespace hz {

namespace {

constexpr int kChaseThreads = 256;
constexpr uint32_t kTerm = 0xFFFFFFFEu;  // "the end of the stream"
constexpr uint32_t kDead = 0xFFFFFFFFu;  // "not a record start"

// All CTAs wait here.  bar[0] counts arrivals, bar[1] is the generation;
// `gen` is the caller's count of barriers passed.  Returns false in every
// thread of a CTA whose wait ran out.
__device__ bool grid_barrier(uint32_t* bar, uint32_t& gen) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      bar[0] = 0;
      __threadfence();
      atomicExch(&bar[1], gen + 1);
    } else {
      uint32_t spins = 0;  // each poll is a round trip to L2: the bound is seconds
      while (ld_acquire(&bar[1]) == gen) {
        if (++spins > (kSpinLimit << 4)) {
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  ++gen;
  __syncthreads();
  return s_ok != 0;
}

// Exclusive prefix sum of v over the CTA; the CTA total in *total.
__device__ uint32_t cta_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t s_warp[kChaseThreads / 32];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane >= (uint32_t)d) inc += o;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  uint32_t pre = 0, tot = 0;
  for (uint32_t w = 0; w < kChaseThreads / 32; ++w) {
    const uint32_t x = s_warp[w];
    pre += w < warp ? x : 0u;
    tot += x;
  }
  __syncthreads();
  *total = tot;
  return pre + inc - v;
}

}  // namespace

__global__ void __launch_bounds__(kChaseThreads) decode_chase_kernel(DecodeArgs a, DecTables* T,
                                                                     ChaseScratch cs) {
  if (!T->needs_chase) return;  // the same answer in every CTA: nobody waits
  const uint32_t nb = T->nb;
  const uint64_t blocks_at = T->blocks_at;
  const uint64_t tw = a.in_len >= blocks_at ? (a.in_len - blocks_at) / 4 : 0;
  const uint32_t* words = reinterpret_cast<const uint32_t*>(a.in + blocks_at);
  const uint64_t nwg = (tw + 31) / 32;  // bitmap words
  const bool parallel = nb >= 1 && nb <= a.chase_cap && tw < 0xFFFFFF00ull &&
                        nwg + 1 <= cs.bm_cap && gridDim.x + 1 <= cs.cta_cap;
  auto serial = [&]() {  // the paper's walk, by one thread
    if (blockIdx.x == 0 && threadIdx.x == 0 && serial_chase(a, blocks_at, nb)) {
      __threadfence();
      T->ok = 1;
    }
  };
  if (!parallel) {
    serial();
    return;
  }
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t gtid = blockIdx.x * kChaseThreads + threadIdx.x;
  const uint32_t nthreads = gridDim.x * kChaseThreads;
  const uint32_t gwarp = gtid >> 5, nwarps = nthreads >> 5;
  uint32_t gen = 0;
  auto timeout = [&]() {
    if (threadIdx.x == 0) set_error(a.st, HZ_ERR_TIMEOUT, 0x330);
  };

  // ---- candidates: one bitmap bit per record-area word
  const uint64_t cnt_last = T->n - (uint64_t)(nb - 1) * T->B;
  const uint64_t lo = (cnt_last < T->B ? cnt_last : (uint64_t)T->B) * T->minlen;
  const uint64_t hi = (uint64_t)T->B * T->maxlen;
  for (uint32_t k = gtid; k < nb; k += nthreads) cs.hits[k] = 0;
  // each warp takes eight groups of 32 words at a time, so that eight loads
  // per lane are in flight
  constexpr uint32_t kGroups = 8;
  for (uint64_t g0 = (uint64_t)gwarp * kGroups; g0 < nwg; g0 += (uint64_t)nwarps * kGroups) {
    uint32_t v[kGroups];
#pragma unroll
    for (uint32_t i = 0; i < kGroups; ++i) {
      const uint64_t w = (g0 + i) * 32 + lane;
      v[i] = w < tw ? words[w] : 0u;
    }
#pragma unroll
    for (uint32_t i = 0; i < kGroups; ++i) {
      const uint64_t w = (g0 + i) * 32 + lane;
      bool cand = false;
      if (w < tw && v[i] >= lo && v[i] <= hi) {
        const uint64_t nw = (v[i] + 31) >> 5;
        if (w + 1 + nw <= tw)
          cand = (v[i] & 31) == 0 || (words[w + nw] & ((1u << (32 - (v[i] & 31))) - 1u)) == 0;
      }
      const uint32_t bm = __ballot_sync(0xFFFFFFFFu, cand);
      if (lane == 0 && g0 + i < nwg) cs.bitmap[g0 + i] = bm;
    }
  }
  if (!grid_barrier(cs.bar, gen)) return timeout();

  // ---- number the candidates: prefix counts over the bitmap, CTA by CTA
  const uint64_t per = (nwg + gridDim.x - 1) / gridDim.x;
  const uint64_t c0 = (uint64_t)blockIdx.x * per, c1 = c0 + per < nwg ? c0 + per : nwg;
  uint32_t carry = 0;
  for (uint64_t g0 = c0; g0 < c1; g0 += kChaseThreads) {
    const uint64_t g = g0 + threadIdx.x;
    const uint32_t v = g < c1 ? __popc(cs.bitmap[g]) : 0u;
    uint32_t tot;
    const uint32_t ex = cta_exclusive_scan(v, &tot);
    if (g < c1) cs.base[g] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) cs.cta_tot[blockIdx.x] = carry;
  if (!grid_barrier(cs.bar, gen)) return timeout();
  if (blockIdx.x == 0) {
    uint32_t run = 0;
    for (uint32_t i0 = 0; i0 < gridDim.x; i0 += kChaseThreads) {
      const uint32_t i = i0 + threadIdx.x;
      const uint32_t v = i < gridDim.x ? cs.cta_tot[i] : 0u;
      uint32_t tot;
      const uint32_t ex = cta_exclusive_scan(v, &tot);
      if (i < gridDim.x) cs.cta_tot[i] = run + ex;
      run += tot;
    }
    if (threadIdx.x == 0) cs.cta_tot[gridDim.x] = run;  // all candidates
  }
  if (!grid_barrier(cs.bar, gen)) return timeout();
  const uint32_t C = cs.cta_tot[gridDim.x];
  {
    const uint32_t add = cs.cta_tot[blockIdx.x];
    for (uint64_t g = c0 + threadIdx.x; g < c1; g += kChaseThreads) cs.base[g] += add;
  }
  if (C > cs.c_cap || C == 0) {
    serial();  // too many candidates for the scratch (or none at all)
    return;
  }
  if (!grid_barrier(cs.bar, gen)) return timeout();

  // ---- each candidate points to the candidate where its record would end
  // (the candidate number of a word, or the end of the stream, or nowhere)
  auto id_of = [&](uint64_t w) -> uint32_t {
    const uint32_t wb = cs.bitmap[w >> 5], wj = (uint32_t)(w & 31);
    return ((wb >> wj) & 1u) ? cs.base[w >> 5] + __popc(wb & ((1u << wj) - 1u)) : kDead;
  };
  auto succ_of_word = [&](uint64_t w) -> uint32_t {
    const uint64_t q = w + 1 + ((words[w] + 31ull) >> 5);
    return q == tw ? kTerm : (q < tw ? id_of(q) : kDead);
  };
  for (uint64_t g = gtid; g < nwg; g += nthreads) {
    uint32_t bits = cs.bitmap[g];
    uint32_t id = cs.base[g];
    while (bits) {
      const uint32_t j = __ffs(bits) - 1;
      bits &= bits - 1;
      const uint64_t w = g * 32 + j;
      const uint32_t succ = succ_of_word(w);
      cs.pos[id] = (uint32_t)w;
      cs.s0[id] = succ;
      cs.r0[id] = 1;
      ++id;
    }
  }
  if (!grid_barrier(cs.bar, gen)) return timeout();

  // ---- pointer jumping: after round j each pointer is 2^j records ahead
  uint32_t *sa = cs.s0, *sb = cs.s1, *ra = cs.r0, *rb = cs.r1;
  for (uint32_t span = 1; span < C; span <<= 1) {
    for (uint32_t id = gtid; id < C; id += nthreads) {
      const uint32_t s = sa[id];
      if (s < kTerm) {
        sb[id] = sa[s];
        rb[id] = ra[id] + ra[s];
      } else {
        sb[id] = s;
        rb[id] = ra[id];
      }
    }
    if (!grid_barrier(cs.bar, gen)) return timeout();
    uint32_t* t = sa;
    sa = sb;
    sb = t;
    t = ra;
    ra = rb;
    rb = t;
  }

  // ---- a candidate r records from the end is record nb - r
  for (uint32_t id = gtid; id < C; id += nthreads) {
    if (sa[id] != kTerm) continue;
    const uint32_t r = ra[id];
    if (r >= 1 && r <= nb) {
      atomicAdd(&cs.hits[nb - r], 1u);
      a.chase_index[nb - r] = cs.pos[id];
    }
  }
  if (!grid_barrier(cs.bar, gen)) return timeout();
  // A record claimed by one candidate is that candidate (the true record start
  // always claims its own slot).  A false chain that runs into the true one
  // claims the slots of the true records before the meeting point as well:
  // through such a run the true records are the successors of the record
  // before it, and the walk through the run must arrive at the record after
  // it (or at the end of the stream).  A record nobody claims means a broken
  // chain: the stream is corrupt, and the walk reports where.
  for (uint32_t k = gtid; k < nb; k += nthreads) {
    const uint32_t h = cs.hits[k];
    if (h == 0) {
      atomicOr(cs.flag, 1u);
      continue;
    }
    if (h == 1) {
      if (k == 0 && a.chase_index[0] != 0u) atomicOr(cs.flag, 1u);
      continue;
    }
    if (k > 0 && cs.hits[k - 1] != 1u) continue;  // inside a run: its first slot walks it
    uint32_t t = k == 0 ? id_of(0) : succ_of_word(a.chase_index[k - 1]);
    uint32_t j = k;
    bool ok = t < kTerm;
    while (ok) {
      a.chase_index[j] = cs.pos[t];
      const uint32_t nx = succ_of_word(cs.pos[t]);
      if (++j == nb) {
        ok = nx == kTerm;
        break;
      }
      const uint32_t hj = cs.hits[j];
      if (hj == 1u) {
        ok = nx == id_of(a.chase_index[j]);
        break;
      }
      ok = hj != 0u && nx < kTerm;
      t = nx;
    }
    if (!ok) atomicOr(cs.flag, 1u);
  }
  if (!grid_barrier(cs.bar, gen)) return timeout();
  if (*cs.flag) {
    serial();  // a broken chain: the walk finds and reports the error
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    __threadfence();
    T->ok = 1;
  }
}

cudaError_t launch_decode_chase(const DecodeArgs& a, DecTables* T, const ChaseScratch& cs,
                                int num_sms, cudaStream_t s) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decode_chase_kernel, kChaseThreads, 0);
  if (per_sm < 1) per_sm = 1;
  uint32_t grid = (uint32_t)(num_sms * per_sm);
  if (grid + 1 > cs.cta_cap) grid = cs.cta_cap - 1;
  if (cudaMemsetAsync(cs.bar, 0, 4 * sizeof(uint32_t), s) != cudaSuccess) return cudaGetLastError();
  DecodeArgs aa = a;
  DecTables* tt = T;
  ChaseScratch cc = cs;
  void* args[] = {&aa, &tt, &cc};
  return cudaLaunchCooperativeKernel((const void*)decode_chase_kernel, dim3(grid),
                                     dim3(kChaseThreads), args, 0, s);
}

}  // namespace hz
