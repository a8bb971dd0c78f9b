// hz_serve.cu -- hz_serve_replay (declared in include/hz.h): an open-loop
// request loop over the batcher.
//
// Requests are handed to the batcher at their scheduled arrival times, one
// submission each; the batcher admits them against the device-memory budget
// and, whenever one of its slots frees up, launches every queued request that
// fits as one device batch (continuous batching), so requests that arrive
// while others are on the GPU join the next batch and overlap with the running
// ones.  Results without a caller buffer go to a device ring owned by the
// caller; ring space is taken at submission and returned at completion, and a
// request that finds no room waits (the wait counts toward its latency).
// Latency of a request = completion seen on the host - scheduled arrival.
#include <chrono>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hz.h"
#include "hz_batch.h"
#include "hz_ring.h"

static_assert(sizeof(hz_serve_item) == 48, "hz_serve_item layout");
static_assert(sizeof(hz_serve_record) == 48, "hz_serve_record layout");

BatchState* hz_ctx_batch(hz_ctx* c);
int hz_ctx_device(hz_ctx* c);

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

extern "C" hz_status hz_serve_replay(hz_ctx* ctx, const hz_serve_item* items, uint64_t count,
                                     uint8_t* d_ring, uint64_t ring_bytes,
                                     hz_serve_record* records, double* wall_s) {
  if (!ctx || (count && (!items || !records))) return HZ_ERR_ARG;
  for (uint64_t i = 0; i < count; ++i) {
    if (i && items[i].arrival_s < items[i - 1].arrival_s) return HZ_ERR_ARG;
    if (!items[i].req.d_dst && (!d_ring || items[i].req.dst_cap > ring_bytes ||
                                ((uintptr_t)d_ring & 255)))
      return HZ_ERR_ARG;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(hz_ctx_device(ctx));
  BatchState* b = hz_ctx_batch(ctx);
  // the items' sources may still be written on any stream: the submissions
  // below are not ordered after the caller's work, so wait for all of it
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    if (prev >= 0) cudaSetDevice(prev);
    return HZ_ERR_CUDA;
  }
  hz_batch_track_finished(b, true);

  hz::Ring ring(ring_bytes);
  std::unordered_map<uint64_t, uint64_t> by_ticket;  // ticket -> item
  std::vector<uint64_t> ring_seq(count, ~0ull);
  std::deque<uint64_t> waiting;  // arrived, not yet submitted (no ring room)
  std::vector<uint64_t> finished;
  uint64_t next = 0, done = 0, in_flight = 0;
  const int64_t t0 = now_ns();
  int64_t last_done = t0;

  auto complete = [&](uint64_t i, hz_status st, uint64_t len, uint64_t launch, int64_t t) {
    records[i].done_s = (double)(t - t0) * 1e-9;
    records[i].status = st;
    records[i].out_len = len;
    records[i].launch = launch;
    if (ring_seq[i] != ~0ull) ring.release(ring_seq[i]);
    if (t > last_done) last_done = t;
    ++done;
  };

  for (uint64_t i = 0; i < count; ++i) {
    records[i] = hz_serve_record{};
    records[i].dst_offset = ~0ull;
  }
  while (done < count) {
    const int64_t now = now_ns();
    while (next < count && t0 + (int64_t)(items[next].arrival_s * 1e9) <= now)
      waiting.push_back(next++);
    bool acted = false;
    while (!waiting.empty()) {
      const uint64_t i = waiting.front();
      hz_request r = items[i].req;
      if (!r.d_dst) {
        uint64_t off = 0, seq = 0;
        if (!ring.alloc(r.dst_cap, &off, &seq)) break;  // wait for ring space
        r.d_dst = d_ring + off;
        ring_seq[i] = seq;
        records[i].dst_offset = off;
      }
      waiting.pop_front();
      records[i].submit_s = (double)(now_ns() - t0) * 1e-9;
      uint64_t ticket = 0;
      const hz_status st = hz_batch_submit(b, ctx, &r, 1, &ticket, false, nullptr);
      if (st != HZ_OK) complete(i, st, 0, 0, now_ns());
      else {
        by_ticket[ticket] = i;
        ++in_flight;
      }
      acted = true;
    }
    hz_batch_progress(b);
    hz_batch_drain_finished(b, finished);
    for (uint64_t t : finished) {
      auto it = by_ticket.find(t);
      if (it == by_ticket.end()) continue;  // a submission from outside the replay
      hz_status st = HZ_OK;
      uint64_t len = 0, launch = 0;
      int64_t tdone = 0;
      if (hz_batch_take(b, t, &st, &len, &launch, &tdone) != HZ_OK) continue;
      complete(it->second, st, len, launch, tdone);
      by_ticket.erase(it);
      --in_flight;
      acted = true;
    }
    finished.clear();
    if (acted) continue;
    if (in_flight == 0 && waiting.empty() && next < count) {
      // idle until shortly before the next arrival
      const int64_t wait = t0 + (int64_t)(items[next].arrival_s * 1e9) - now_ns();
      if (wait > 100000) {
        std::this_thread::sleep_for(std::chrono::nanoseconds(wait - 50000));
        continue;
      }
    }
    std::this_thread::yield();
  }
  hz_batch_track_finished(b, false);
  if (wall_s) *wall_s = (double)(last_done - t0) * 1e-9;
  if (prev >= 0) cudaSetDevice(prev);
  return HZ_OK;
}
