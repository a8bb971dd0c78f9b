// hz_batch.cu -- hz_submit / hz_poll: batches are queued in submission order,
// admitted against the context's device-memory budget, and run on the batch
// stream; every request's status and result size land in device arrays that
// hz_poll copies back once the batch's completion event has fired.
#include <chrono>
#include <deque>
#include <map>
#include <thread>
#include <vector>

#include "hz_batch.h"
#include "hz_internal.cuh"

namespace {

struct Job {
  uint64_t ticket = 0;
  std::vector<hz_request> reqs;
  uint64_t footprint = 0;
  int32_t* d_status = nullptr;   // per request
  uint64_t* d_lens = nullptr;    // per request
  cudaEvent_t done = nullptr;
  bool launched = false;
  hz_status launch_status = HZ_OK;
};

// Copy the context's status word into one request's slot and clear it.
__global__ void snapshot_status_kernel(hz::DevState* st, int32_t* dst) {
  dst[0] = -(int32_t)st->error;
  st->error = 0;
  st->error_where = 0;
}

}  // namespace

struct BatchState {
  int device = 0;
  int num_sms = 0;
  uint64_t budget = 0;
  uint64_t admitted = 0;
  uint64_t next_ticket = 1;
  cudaStream_t stream = nullptr;
  std::deque<Job*> queue;          // submitted, in order (launched ones first)
  std::map<uint64_t, Job*> jobs;
  hz_ctx* ctx = nullptr;
};


BatchState* hz_batch_create(int device, int num_sms, uint64_t mem_budget) {
  BatchState* b = new BatchState();
  b->device = device;
  b->num_sms = num_sms;
  b->budget = mem_budget;
  cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
  return b;
}

static void free_job(Job* j) {
  cudaFree(j->d_status);
  cudaFree(j->d_lens);
  if (j->done) cudaEventDestroy(j->done);
  delete j;
}

void hz_batch_destroy(BatchState* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& kv : b->jobs) free_job(kv.second);
  cudaStreamDestroy(b->stream);
  delete b;
}

uint32_t hz_batch_tuned_block_size(uint64_t n) {
  // one record per 64 KiB keeps the per-block overhead below 0.1 % (Sec. 2.1);
  // small inputs take smaller blocks so that they still spread over many CTAs
  if (n <= (64u << 10)) return 4096;
  if (n <= (4u << 20)) return 16384;
  return 65536;
}

extern "C" hz_status hz_compress(hz_ctx*, const uint8_t*, uint64_t, uint32_t, const hz_codes*,
                                 uint8_t*, uint64_t, uint64_t*, void*);
extern "C" hz_status hz_decompress(hz_ctx*, const uint8_t*, uint64_t, uint8_t*, uint64_t,
                                   uint64_t*, void*);
hz::DevState* hz_ctx_state(hz_ctx* c);

static hz_status launch_job(BatchState* b, Job* j) {
  const uint32_t n = (uint32_t)j->reqs.size();
  for (uint32_t i = 0; i < n; ++i) {
    const hz_request& r = j->reqs[i];
    hz_status st;
    if (r.op == HZ_OP_COMPRESS)
      st = hz_compress(b->ctx, r.d_src, r.src_len, r.block_size, nullptr, r.d_dst, r.dst_cap,
                       j->d_lens + i, b->stream);
    else
      st = hz_decompress(b->ctx, r.d_src, r.src_len, r.d_dst, r.dst_cap, j->d_lens + i,
                         b->stream);
    if (st != HZ_OK) return st;
    snapshot_status_kernel<<<1, 1, 0, b->stream>>>(hz_ctx_state(b->ctx), j->d_status + i);
  }
  if (cudaEventRecord(j->done, b->stream) != cudaSuccess) return HZ_ERR_CUDA;
  j->launched = true;
  b->admitted += j->footprint;
  return HZ_OK;
}

// Launch queued batches, in order, while they fit the budget.
static void admit(BatchState* b) {
  for (Job* j : b->queue) {
    if (j->launched) continue;
    if (b->budget && b->admitted + j->footprint > b->budget) break;
    j->launch_status = launch_job(b, j);
    if (j->launch_status != HZ_OK) {
      j->launched = true;
      cudaEventRecord(j->done, b->stream);
    }
  }
}

hz_status hz_batch_submit(BatchState* b, hz_ctx* ctx, const hz_request* reqs, uint32_t count,
                          uint64_t* ticket) {
  b->ctx = ctx;
  uint64_t fp = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const hz_request& r = reqs[i];
    if ((r.op != HZ_OP_COMPRESS && r.op != HZ_OP_DECOMPRESS) || !r.d_dst || !r.d_src ||
        r.src_len > 0xFFFFFFFFull || r.block_size > hz::kMaxBlock)
      return HZ_ERR_ARG;
    fp += r.src_len + r.dst_cap;
  }
  if (b->budget && fp > b->budget) return HZ_ERR_BUSY;
  Job* j = new Job();
  j->ticket = b->next_ticket++;
  j->reqs.assign(reqs, reqs + count);
  j->footprint = fp;
  const uint32_t m = count ? count : 1;
  if (cudaMalloc(&j->d_status, m * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&j->d_lens, m * sizeof(uint64_t)) != cudaSuccess ||
      cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    free_job(j);
    return HZ_ERR_NOMEM;
  }
  cudaMemsetAsync(j->d_status, 0, m * sizeof(int32_t), b->stream);
  cudaMemsetAsync(j->d_lens, 0, m * sizeof(uint64_t), b->stream);
  b->queue.push_back(j);
  b->jobs[j->ticket] = j;
  admit(b);
  *ticket = j->ticket;
  return HZ_OK;
}

hz_status hz_batch_poll(BatchState* b, uint64_t ticket, int64_t timeout_ns, hz_status* per_req,
                        uint64_t* out_lens) {
  auto it = b->jobs.find(ticket);
  if (it == b->jobs.end()) return HZ_ERR_ARG;
  Job* j = it->second;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    // retire finished batches at the head so that waiting ones can be admitted
    while (!b->queue.empty() && b->queue.front()->launched &&
           cudaEventQuery(b->queue.front()->done) == cudaSuccess) {
      Job* h = b->queue.front();
      b->queue.pop_front();
      b->admitted -= h->launch_status == HZ_OK ? h->footprint : 0;
      h->footprint = 0;
    }
    admit(b);
    if (j->launched && cudaEventQuery(j->done) == cudaSuccess) break;
    cudaGetLastError();
    if (timeout_ns == 0) return HZ_PENDING;
    if (timeout_ns > 0 && std::chrono::duration_cast<std::chrono::nanoseconds>(
                              std::chrono::steady_clock::now() - t0)
                                  .count() >= timeout_ns)
      return HZ_PENDING;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  const uint32_t n = (uint32_t)j->reqs.size();
  hz_status rs = j->launch_status;
  if (rs == HZ_OK && n) {
    std::vector<int32_t> s(n);
    std::vector<uint64_t> l(n);
    if (cudaMemcpy(s.data(), j->d_status, n * sizeof(int32_t), cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(l.data(), j->d_lens, n * sizeof(uint64_t), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
      rs = HZ_ERR_CUDA;
    for (uint32_t i = 0; i < n && rs == HZ_OK; ++i) {
      if (per_req) per_req[i] = s[i];
      if (out_lens) out_lens[i] = l[i];
    }
  }
  if (rs != HZ_OK)
    for (uint32_t i = 0; i < n; ++i) {
      if (per_req) per_req[i] = rs;
      if (out_lens) out_lens[i] = 0;
    }
  b->jobs.erase(it);
  free_job(j);
  return HZ_OK;
}
