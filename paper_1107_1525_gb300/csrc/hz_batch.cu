// hz_batch.cu -- host side of hz_submit / hz_poll.
//
// Batches are queued in submission order and admitted against the context's
// device-memory budget (request buffers plus the batch's scratch).  An
// admitted batch takes one of kSlots slots; each slot has its own stream,
// device scratch (per-request state, encoder tile records, decode tables),
// pinned descriptor staging and a CUDA graph of the batched kernel sequence
// (hz_batch_kernels.cu), captured once per scratch allocation and replayed for
// every batch.  Batches in different slots run concurrently on the device, so
// requests that arrive while others are on the GPU are admitted as slots and
// memory free up, and their work overlaps.
//
// Plain mode (HZ_OPT_BATCH_PLAIN = 1) runs the same requests one after another
// through hz_compress / hz_decompress -- one launch sequence per buffer -- as
// the baseline the batched path is measured against.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "hz_batch.h"
#include "hz_batch_dev.h"

using namespace hz;

namespace {

constexpr int kSlots = 3;
constexpr uint32_t kPlainRing = 1u << 16;  // plain-mode result records in flight

struct Job {
  uint64_t ticket = 0;
  std::vector<hz_request> reqs;
  uint64_t footprint = 0;
  int slot = -1;
  uint64_t launch_id = 0;  // device batch (or plain launch sequence) that carried it
  bool plain = false;
  bool launched = false;
  bool done = false;
  int64_t done_ns = 0;  // host steady-clock time at which completion was seen
  hz_status launch_status = HZ_OK;
  std::vector<hz_status> status;
  std::vector<uint64_t> lens;
  // plain mode: the job's records in the plain ring, and its completion event
  uint32_t plain_pos = 0;
  cudaEvent_t plain_done = nullptr;
  // recorded at submission on the caller's stream: the launch that carries
  // the job waits for it, so work the caller enqueued before hz_submit (that
  // writes the sources, or reads the destinations) comes first
  cudaEvent_t ready = nullptr;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::vector<Job*> jobs;  // the submissions this slot's current launch carries
  // capacities
  uint32_t req_cap = 0;
  uint64_t tiles_cap = 0;
  // device
  BatchCtl* d_ctl = nullptr;
  BatchComp* d_comps = nullptr;
  BatchDecomp* d_decomps = nullptr;
  BatchResult* d_results = nullptr;
  DevState* d_states = nullptr;
  uint32_t* d_bases = nullptr;  // 3 x req_cap: histogram, tile and decode-unit bases
  DecTables* d_dec = nullptr;
  uint64_t* d_lens = nullptr;
  TileStatus* d_tiles = nullptr;
  // pinned host
  BatchCtl* h_ctl = nullptr;
  BatchComp* h_comps = nullptr;
  BatchDecomp* h_decomps = nullptr;
  BatchResult* h_results = nullptr;
};

__global__ void snapshot_status_kernel(DevState* st, int32_t* dst) {
  dst[0] = -(int32_t)st->error;
  st->error = 0;
  st->error_where = 0;
}

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

struct BatchState {
  int device = 0;
  int num_sms = 0;
  uint64_t budget = 0;
  uint64_t admitted = 0;
  uint64_t next_ticket = 1;
  uint64_t launches = 0;
  uint32_t max_reqs = 4096;  // requests per device batch when several submissions merge
  bool plain = false;
  hz_ctx* ctx = nullptr;
  Slot slots[kSlots];
  std::deque<Job*> queue;  // submitted, not yet finished, in order
  std::map<uint64_t, Job*> jobs;
  bool track_finished = false;     // record completions for hz_batch_drain_finished
  std::vector<uint64_t> finished;  // tickets completed since the last drain
  // plain mode: one stream, per-request status and length records in a ring
  cudaStream_t plain_stream = nullptr;
  int32_t* d_plain_status = nullptr;
  uint64_t* d_plain_lens = nullptr;
  int32_t* h_plain_status = nullptr;
  uint64_t* h_plain_lens = nullptr;
  uint32_t plain_head = 0;      // next free record
  uint32_t plain_inflight = 0;  // records held by unfinished plain jobs
  std::vector<cudaEvent_t> free_events;  // for Job::ready
};

// Make `s` wait for the job's submission event and return the event to the
// pool (a wait takes the event's state when it is enqueued, so the event can
// be recorded again at once).
static bool wait_ready(BatchState* b, Job* j, cudaStream_t s) {
  if (!j->ready) return true;
  const bool ok = cudaStreamWaitEvent(s, j->ready, 0) == cudaSuccess;
  b->free_events.push_back(j->ready);
  j->ready = nullptr;
  return ok;
}

extern "C" hz_status hz_compress(hz_ctx*, const uint8_t*, uint64_t, uint32_t, const hz_codes*,
                                 uint8_t*, uint64_t, uint64_t*, void*);
extern "C" hz_status hz_decompress(hz_ctx*, const uint8_t*, uint64_t, uint8_t*, uint64_t,
                                   uint64_t*, void*);
hz::DevState* hz_ctx_state(hz_ctx* c);
uint32_t hz_ctx_block_size(hz_ctx* c, uint64_t n);
int hz_ctx_lut_bits(hz_ctx* c);

static void free_slot_buffers(Slot& s) {
  if (s.graph) cudaGraphExecDestroy(s.graph);
  s.graph = nullptr;
  cudaFree(s.d_ctl);
  cudaFree(s.d_comps);
  cudaFree(s.d_decomps);
  cudaFree(s.d_results);
  cudaFree(s.d_states);
  cudaFree(s.d_bases);
  cudaFree(s.d_dec);
  cudaFree(s.d_lens);
  cudaFree(s.d_tiles);
  cudaFreeHost(s.h_ctl);
  cudaFreeHost(s.h_comps);
  cudaFreeHost(s.h_decomps);
  cudaFreeHost(s.h_results);
  s.d_ctl = nullptr;
  s.d_comps = nullptr;
  s.d_decomps = nullptr;
  s.d_results = nullptr;
  s.d_states = nullptr;
  s.d_bases = nullptr;
  s.d_dec = nullptr;
  s.d_lens = nullptr;
  s.d_tiles = nullptr;
  s.h_ctl = nullptr;
  s.h_comps = nullptr;
  s.h_decomps = nullptr;
  s.h_results = nullptr;
  s.req_cap = 0;
  s.tiles_cap = 0;
}

// Make the slot hold `reqs` requests and `tiles` encoder tiles; re-captures
// the slot's graph after any reallocation.
static hz_status ensure_slot(BatchState* b, Slot& s, uint32_t reqs, uint64_t tiles) {
  if (reqs <= s.req_cap && tiles <= s.tiles_cap && s.graph) return HZ_OK;
  uint32_t rc = s.req_cap, need_r = reqs ? reqs : 1;
  uint64_t tc = s.tiles_cap, need_t = tiles ? tiles : 1;
  if (need_r > rc) {
    rc = rc ? rc : 64;
    while (rc < need_r) rc *= 2;
  }
  if (need_t > tc) {
    tc = tc ? tc : 4096;
    while (tc < need_t) tc *= 2;
  }
  cudaStreamSynchronize(s.stream);
  free_slot_buffers(s);
  bool ok = cudaMalloc(&s.d_ctl, sizeof(BatchCtl)) == cudaSuccess &&
            cudaMalloc(&s.d_comps, rc * sizeof(BatchComp)) == cudaSuccess &&
            cudaMalloc(&s.d_decomps, rc * sizeof(BatchDecomp)) == cudaSuccess &&
            cudaMalloc(&s.d_results, rc * sizeof(BatchResult)) == cudaSuccess &&
            cudaMalloc(&s.d_states, rc * sizeof(DevState)) == cudaSuccess &&
            cudaMalloc(&s.d_bases, 3ull * rc * sizeof(uint32_t)) == cudaSuccess &&
            cudaMalloc(&s.d_dec, rc * batch_dec_tables_bytes()) == cudaSuccess &&
            cudaMalloc(&s.d_lens, rc * sizeof(uint64_t)) == cudaSuccess &&
            cudaMalloc(&s.d_tiles, tc * sizeof(TileStatus)) == cudaSuccess &&
            cudaHostAlloc(&s.h_ctl, sizeof(BatchCtl), cudaHostAllocDefault) == cudaSuccess &&
            cudaHostAlloc(&s.h_comps, rc * sizeof(BatchComp), cudaHostAllocDefault) == cudaSuccess &&
            cudaHostAlloc(&s.h_decomps, rc * sizeof(BatchDecomp), cudaHostAllocDefault) ==
                cudaSuccess &&
            cudaHostAlloc(&s.h_results, rc * sizeof(BatchResult), cudaHostAllocDefault) ==
                cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    free_slot_buffers(s);
    return HZ_ERR_NOMEM;
  }
  s.req_cap = rc;
  s.tiles_cap = tc;
  // the graph: descriptors in, the kernel sequence, results out
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return HZ_ERR_CUDA;
  cudaMemcpyAsync(s.d_ctl, s.h_ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.d_comps, s.h_comps, rc * sizeof(BatchComp), cudaMemcpyHostToDevice, s.stream);
  cudaMemcpyAsync(s.d_decomps, s.h_decomps, rc * sizeof(BatchDecomp), cudaMemcpyHostToDevice,
                  s.stream);
  BatchLaunch L{s.d_ctl, s.d_comps, s.d_decomps, s.d_results, b->num_sms};
  batch_enqueue(L, s.stream);
  cudaMemcpyAsync(s.h_results, s.d_results, rc * sizeof(BatchResult), cudaMemcpyDeviceToHost,
                  s.stream);
  if (cudaStreamEndCapture(s.stream, &g) != cudaSuccess || !g) {
    cudaGetLastError();
    return HZ_ERR_CUDA;
  }
  const cudaError_t e = cudaGraphInstantiate(&s.graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s.graph = nullptr;
    return HZ_ERR_CUDA;
  }
  return HZ_OK;
}

BatchState* hz_batch_create(int device, int num_sms, uint64_t mem_budget) {
  BatchState* b = new BatchState();
  b->device = device;
  b->num_sms = num_sms;
  b->budget = mem_budget;
  batch_configure();
  cudaStreamCreateWithFlags(&b->plain_stream, cudaStreamNonBlocking);
  for (Slot& s : b->slots) {
    cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
  }
  return b;
}

static void free_job(BatchState* b, Job* j) {
  if (j->plain_done) cudaEventDestroy(j->plain_done);
  if (j->ready) b->free_events.push_back(j->ready);
  delete j;
}

void hz_batch_destroy(BatchState* b) {
  if (!b) return;
  for (Slot& s : b->slots) {
    cudaStreamSynchronize(s.stream);
    free_slot_buffers(s);
    cudaEventDestroy(s.done);
    cudaStreamDestroy(s.stream);
  }
  cudaStreamSynchronize(b->plain_stream);
  cudaStreamDestroy(b->plain_stream);
  cudaFree(b->d_plain_status);
  cudaFree(b->d_plain_lens);
  cudaFreeHost(b->h_plain_status);
  cudaFreeHost(b->h_plain_lens);
  for (auto& kv : b->jobs) free_job(b, kv.second);
  for (cudaEvent_t e : b->free_events) cudaEventDestroy(e);
  delete b;
}

void hz_batch_set_plain(BatchState* b, bool plain) { b->plain = plain; }
bool hz_batch_plain(BatchState* b) { return b->plain; }
hz_status hz_batch_set_max_reqs(BatchState* b, uint32_t m) {
  if (m == 0) return HZ_ERR_ARG;
  b->max_reqs = m;
  return HZ_OK;
}
uint32_t hz_batch_max_reqs(BatchState* b) { return b->max_reqs; }

uint32_t hz_batch_tuned_block_size(uint64_t n) {
  // 16 KiB blocks keep the per-block overhead near 0.05 % (Sec. 2.1: 32-63 bits
  // a block) and decode as fast as 64 KiB ones, while a buffer of a few MiB
  // still spreads over many warps (a lone 7 MB stream in 64 KiB blocks keeps
  // only 107 warps busy); the smallest buffers take 4 KiB blocks, the largest
  // 64 KiB
  if (n <= (64u << 10)) return 4096;
  if (n <= (32u << 20)) return 16384;
  return 65536;
}

// ----------------------------------------------------------- plain baseline
// Each request runs through hz_compress / hz_decompress on the plain stream,
// followed by a one-thread kernel that moves the context's error word into the
// request's status record; the records come back to pinned host memory with
// one copy per job.  Nothing is allocated per job, so the baseline pays only
// for its launches.
static hz_status plain_reserve(BatchState* b, uint32_t n, uint32_t* pos) {
  if (!b->d_plain_status) {
    if (cudaMalloc(&b->d_plain_status, kPlainRing * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&b->d_plain_lens, kPlainRing * sizeof(uint64_t)) != cudaSuccess ||
        cudaHostAlloc(&b->h_plain_status, kPlainRing * sizeof(int32_t), cudaHostAllocDefault) !=
            cudaSuccess ||
        cudaHostAlloc(&b->h_plain_lens, kPlainRing * sizeof(uint64_t), cudaHostAllocDefault) !=
            cudaSuccess) {
      cudaGetLastError();
      return HZ_ERR_NOMEM;
    }
  }
  // jobs finish in launch order, so the records in flight are one contiguous
  // (circular) range ending at plain_head
  if (b->plain_head + n > kPlainRing) {
    if (b->plain_inflight > 0) return HZ_PENDING;  // wait for the wrap
    b->plain_head = 0;
  }
  if (b->plain_inflight + n > kPlainRing) return HZ_PENDING;
  *pos = b->plain_head;
  b->plain_head += n;
  b->plain_inflight += n;
  return HZ_OK;
}

static hz_status launch_plain(BatchState* b, Job* j) {
  const uint32_t n = (uint32_t)j->reqs.size();
  int32_t* d_status = b->d_plain_status + j->plain_pos;
  uint64_t* d_lens = b->d_plain_lens + j->plain_pos;
  if (cudaEventCreateWithFlags(&j->plain_done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return HZ_ERR_CUDA;
  }
  if (!wait_ready(b, j, b->plain_stream)) {
    cudaGetLastError();
    return HZ_ERR_CUDA;
  }
  if (n) {
    cudaMemsetAsync(d_status, 0, n * sizeof(int32_t), b->plain_stream);
    cudaMemsetAsync(d_lens, 0, n * sizeof(uint64_t), b->plain_stream);
  }
  for (uint32_t i = 0; i < n; ++i) {
    const hz_request& r = j->reqs[i];
    hz_status st;
    if (r.op == HZ_OP_COMPRESS)
      st = hz_compress(b->ctx, r.d_src, r.src_len, r.block_size, nullptr, r.d_dst, r.dst_cap,
                       d_lens + i, b->plain_stream);
    else
      st = hz_decompress(b->ctx, r.d_src, r.src_len, r.d_dst, r.dst_cap, d_lens + i,
                         b->plain_stream);
    if (st != HZ_OK) return st;
    snapshot_status_kernel<<<1, 1, 0, b->plain_stream>>>(hz_ctx_state(b->ctx), d_status + i);
  }
  if (n) {
    cudaMemcpyAsync(b->h_plain_status + j->plain_pos, d_status, n * sizeof(int32_t),
                    cudaMemcpyDeviceToHost, b->plain_stream);
    cudaMemcpyAsync(b->h_plain_lens + j->plain_pos, d_lens, n * sizeof(uint64_t),
                    cudaMemcpyDeviceToHost, b->plain_stream);
  }
  return cudaEventRecord(j->plain_done, b->plain_stream) == cudaSuccess ? HZ_OK : HZ_ERR_CUDA;
}

// ----------------------------------------------------------- batched path
static uint64_t scratch_bytes(const std::vector<hz_request>& reqs) {
  uint64_t t = 0;
  for (const hz_request& r : reqs) {
    t += sizeof(DevState) + sizeof(BatchComp) + sizeof(BatchDecomp) + 16;
    if (r.op == HZ_OP_COMPRESS) t += ((r.src_len + kEncTile - 1) / kEncTile) * sizeof(TileStatus);
    else t += batch_dec_tables_bytes();
  }
  return t;
}

// Launch the requests of `group` (one or more submissions, in order) as one
// device batch on slot `slot_index`.
static hz_status launch_batched(BatchState* b, const std::vector<Job*>& group, int slot_index) {
  Slot& s = b->slots[slot_index];
  uint32_t n = 0;
  uint64_t tiles = 0;
  for (const Job* j : group) {
    n += (uint32_t)j->reqs.size();
    for (const hz_request& r : j->reqs)
      if (r.op == HZ_OP_COMPRESS) tiles += (r.src_len + kEncTile - 1) / kEncTile;
  }
  hz_status st = ensure_slot(b, s, n, tiles);
  if (st != HZ_OK) return st;
  BatchCtl ctl;
  memset(&ctl, 0, sizeof(ctl));
  const int W = hz_ctx_lut_bits(b->ctx);
  uint32_t nc = 0, nd = 0, hist_units = 0, tile_base = 0, i = 0;
  for (const Job* j : group) {
    for (const hz_request& r : j->reqs) {
      if (r.op == HZ_OP_COMPRESS) {
        BatchComp& c = s.h_comps[nc];
        memset(&c, 0, sizeof(c));
        const uint32_t B = r.block_size ? r.block_size : hz_ctx_block_size(b->ctx, r.src_len);
        c.src = r.d_src;
        c.n = r.src_len;
        c.dst = r.d_dst;
        c.cap = r.dst_cap;
        c.B = B;
        c.nb = (uint32_t)((r.src_len + B - 1) / B);
        c.ntiles = (uint32_t)((r.src_len + kEncTile - 1) / kEncTile);
        c.flags = kFlagIndex;
        c.fdB = make_fastdiv(B);
        c.st = s.d_states + i;
        c.tiles = s.d_tiles + tile_base;
        c.out_len = s.d_lens + i;
        c.hist_base = hist_units;
        c.tile_base = tile_base;
        c.req = i;
        hist_units += (uint32_t)((r.src_len + kBatchHistChunk - 1) / kBatchHistChunk);
        tile_base += c.ntiles;
        ++nc;
      } else {
        BatchDecomp& d = s.h_decomps[nd];
        memset(&d, 0, sizeof(d));
        d.src = r.d_src;
        d.in_len = r.src_len;
        d.dst = r.d_dst;
        d.cap = r.dst_cap;
        d.st = s.d_states + i;
        d.T = reinterpret_cast<DecTables*>(reinterpret_cast<uint8_t*>(s.d_dec) +
                                           (uint64_t)nd * batch_dec_tables_bytes());
        d.out_len = s.d_lens + i;
        d.lut_bits = (uint32_t)W;
        d.req = i;
        ++nd;
      }
      ++i;
    }
  }
  ctl.ncomp = nc;
  ctl.ndecomp = nd;
  ctl.hist_units = hist_units;
  ctl.tiles = tile_base;
  ctl.hist_base = s.d_bases;
  ctl.tile_base = s.d_bases + s.req_cap;
  ctl.unit_base = s.d_bases + 2ull * s.req_cap;
  *s.h_ctl = ctl;
  bool waited = true;
  for (Job* j : group) waited &= wait_ready(b, j, s.stream);
  if (!waited || cudaGraphLaunch(s.graph, s.stream) != cudaSuccess ||
      cudaEventRecord(s.done, s.stream) != cudaSuccess) {
    cudaGetLastError();
    return HZ_ERR_CUDA;
  }
  s.jobs = group;
  const uint64_t id = ++b->launches;
  for (Job* j : group) {
    j->slot = slot_index;
    j->launch_id = id;
  }
  return HZ_OK;
}

static void mark_done(BatchState* b, Job* j) {
  b->admitted -= j->footprint;
  j->done = true;
  j->done_ns = now_ns();
  if (b->track_finished) b->finished.push_back(j->ticket);
}

// A job whose launch failed: every request gets the launch's status.
static void fail_job(BatchState* b, Job* j) {
  const uint32_t n = (uint32_t)j->reqs.size();
  j->status.assign(n, j->launch_status);
  j->lens.assign(n, 0);
  mark_done(b, j);
}

static void finish_plain(BatchState* b, Job* j) {
  const uint32_t n = (uint32_t)j->reqs.size();
  j->status.assign(n, HZ_OK);
  j->lens.assign(n, 0);
  for (uint32_t i = 0; i < n; ++i) {
    j->status[i] = b->h_plain_status[j->plain_pos + i];
    j->lens[i] = b->h_plain_lens[j->plain_pos + i];
  }
  b->plain_inflight -= n;
  mark_done(b, j);
}

static void finish_slot(BatchState* b, Slot& s) {
  uint32_t base = 0;
  for (Job* j : s.jobs) {
    const uint32_t n = (uint32_t)j->reqs.size();
    j->status.assign(n, HZ_ERR_CUDA);
    j->lens.assign(n, 0);
    base += n;
  }
  // results are in phase order (compress requests, then decompress ones);
  // BatchResult.req is the request's position in the launch
  std::vector<std::pair<Job*, uint32_t>> where;
  where.reserve(base);
  for (Job* j : s.jobs)
    for (uint32_t k = 0; k < (uint32_t)j->reqs.size(); ++k) where.push_back({j, k});
  for (uint32_t i = 0; i < base; ++i) {
    const BatchResult& r = s.h_results[i];
    if (r.req < base) {
      where[r.req].first->status[where[r.req].second] = r.status;
      where[r.req].first->lens[where[r.req].second] = r.out_len;
    }
  }
  for (Job* j : s.jobs) mark_done(b, j);
  s.jobs.clear();
}

// Retire finished launches, then launch queued submissions, in order, while
// slots and the budget allow.  A free slot takes every queued submission that
// fits (up to max_reqs requests, or one larger submission alone): requests
// that arrived while the device was busy go out together in the next batch.
static void progress(BatchState* b) {
  for (Slot& s : b->slots) {
    if (s.jobs.empty()) continue;
    if (cudaEventQuery(s.done) == cudaSuccess) finish_slot(b, s);
    else cudaGetLastError();
  }
  for (Job* j : b->queue) {
    if (!j->plain || !j->launched || j->done) continue;
    if (cudaEventQuery(j->plain_done) != cudaSuccess) {
      cudaGetLastError();
      break;  // plain jobs finish in order
    }
    finish_plain(b, j);
  }
  // finished submissions leave the queue wherever they are: completions come
  // back out of order across slots, and hz_batch_take frees them
  b->queue.erase(std::remove_if(b->queue.begin(), b->queue.end(), [](Job* j) { return j->done; }),
                 b->queue.end());
  size_t q = 0;
  while (q < b->queue.size()) {
    Job* j = b->queue[q];
    if (j->launched) {
      ++q;
      continue;
    }
    if (b->budget && b->admitted + j->footprint > b->budget) break;
    if (j->plain) {
      const hz_status r = plain_reserve(b, (uint32_t)j->reqs.size(), &j->plain_pos);
      if (r == HZ_PENDING) break;
      j->launched = true;
      b->admitted += j->footprint;
      j->launch_status = r == HZ_OK ? launch_plain(b, j) : r;
      j->launch_id = ++b->launches;
      if (j->launch_status != HZ_OK) {
        if (r == HZ_OK) {
          // records stay reserved until the stream has passed them
          cudaStreamSynchronize(b->plain_stream);
          cudaGetLastError();
          b->plain_inflight -= (uint32_t)j->reqs.size();
        }
        fail_job(b, j);
      }
      ++q;
      continue;
    }
    int free_slot = -1;
    for (int k = 0; k < kSlots; ++k)
      if (b->slots[k].jobs.empty()) {
        free_slot = k;
        break;
      }
    if (free_slot < 0) break;
    std::vector<Job*> group{j};
    uint64_t add = j->footprint;
    uint32_t nreq = (uint32_t)j->reqs.size();
    for (size_t r = q + 1; r < b->queue.size(); ++r) {
      Job* k = b->queue[r];
      if (k->launched || k->plain) break;
      if (nreq + k->reqs.size() > b->max_reqs) break;
      if (b->budget && b->admitted + add + k->footprint > b->budget) break;
      group.push_back(k);
      add += k->footprint;
      nreq += (uint32_t)k->reqs.size();
    }
    for (Job* k : group) {
      k->launched = true;
      b->admitted += k->footprint;
    }
    const hz_status st = launch_batched(b, group, free_slot);
    if (st != HZ_OK) {
      for (Job* k : group) {
        k->launch_status = st;
        k->slot = -1;
        fail_job(b, k);
      }
    }
    q += group.size();
  }
}

hz_status hz_batch_submit(BatchState* b, hz_ctx* ctx, const hz_request* reqs, uint32_t count,
                          uint64_t* ticket, bool ordered, void* after) {
  b->ctx = ctx;
  uint64_t fp = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const hz_request& r = reqs[i];
    if ((r.op != HZ_OP_COMPRESS && r.op != HZ_OP_DECOMPRESS) || !r.d_dst || !r.d_src ||
        r.src_len > 0xFFFFFFFFull || r.block_size > kMaxBlock || ((uintptr_t)r.d_dst & 3) ||
        (r.op == HZ_OP_DECOMPRESS && ((uintptr_t)r.d_src & 3)))
      return HZ_ERR_ARG;
    fp += r.src_len + r.dst_cap;
  }
  if (b->plain && count > kPlainRing) return HZ_ERR_BUSY;
  Job* j = new Job();
  j->reqs.assign(reqs, reqs + count);
  j->plain = b->plain;
  j->footprint = fp + (j->plain ? 0 : scratch_bytes(j->reqs));
  if (b->budget && j->footprint > b->budget) {
    delete j;
    return HZ_ERR_BUSY;
  }
  if (ordered) {
    if (!b->free_events.empty()) {
      j->ready = b->free_events.back();
      b->free_events.pop_back();
    } else if (cudaEventCreateWithFlags(&j->ready, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      j->ready = nullptr;
      free_job(b, j);
      return HZ_ERR_CUDA;
    }
    if (cudaEventRecord(j->ready, (cudaStream_t)after) != cudaSuccess) {
      cudaGetLastError();
      free_job(b, j);
      return HZ_ERR_CUDA;
    }
  }
  j->ticket = b->next_ticket++;
  b->queue.push_back(j);
  b->jobs[j->ticket] = j;
  progress(b);
  *ticket = j->ticket;
  return HZ_OK;
}

void hz_batch_progress(BatchState* b) { progress(b); }

void hz_batch_track_finished(BatchState* b, bool on) {
  b->track_finished = on;
  b->finished.clear();
}

void hz_batch_drain_finished(BatchState* b, std::vector<uint64_t>& out) {
  out.swap(b->finished);
  b->finished.clear();
}

hz_status hz_batch_take(BatchState* b, uint64_t ticket, hz_status* per_req, uint64_t* out_lens,
                        uint64_t* launch_id, int64_t* done_ns) {
  auto it = b->jobs.find(ticket);
  if (it == b->jobs.end()) return HZ_ERR_ARG;
  Job* j = it->second;
  if (!j->done) return HZ_PENDING;
  const uint32_t n = (uint32_t)j->reqs.size();
  for (uint32_t i = 0; i < n; ++i) {
    if (per_req) per_req[i] = j->status[i];
    if (out_lens) out_lens[i] = j->lens[i];
  }
  if (launch_id) *launch_id = j->launch_id;
  if (done_ns) *done_ns = j->done_ns;
  b->jobs.erase(it);
  auto q = std::find(b->queue.begin(), b->queue.end(), j);
  if (q != b->queue.end()) b->queue.erase(q);  // failed at launch, not yet swept
  free_job(b, j);
  return HZ_OK;
}

hz_status hz_batch_poll(BatchState* b, uint64_t ticket, int64_t timeout_ns, hz_status* per_req,
                        uint64_t* out_lens) {
  auto it = b->jobs.find(ticket);
  if (it == b->jobs.end()) return HZ_ERR_ARG;
  Job* j = it->second;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    progress(b);
    if (j->done) break;
    if (timeout_ns == 0) return HZ_PENDING;
    if (timeout_ns > 0 && std::chrono::duration_cast<std::chrono::nanoseconds>(
                              std::chrono::steady_clock::now() - t0)
                                  .count() >= timeout_ns)
      return HZ_PENDING;
    std::this_thread::sleep_for(std::chrono::microseconds(10));
  }
  return hz_batch_take(b, ticket, per_req, out_lens, nullptr, nullptr);
}
