// hz_batch.h -- batch submission and admission behind hz_submit / hz_poll,
// and the hooks the request-replay loop (hz_serve.cu) drives it through.
#pragma once
#include <stdint.h>

#include <vector>

#include "hz.h"

struct BatchState;

BatchState* hz_batch_create(int device, int num_sms, uint64_t mem_budget);
void hz_batch_destroy(BatchState* b);
// ordered: the launch that carries the submission first waits for the work
// enqueued on the cudaStream_t `after` (NULL = the legacy default stream)
// before this call.
hz_status hz_batch_submit(BatchState* b, hz_ctx* ctx, const hz_request* reqs, uint32_t count,
                          uint64_t* ticket, bool ordered, void* after);
hz_status hz_batch_poll(BatchState* b, uint64_t ticket, int64_t timeout_ns, hz_status* per_req,
                        uint64_t* out_lens);
// Block size used when a caller passes 0 and nothing has been tuned.
uint32_t hz_batch_tuned_block_size(uint64_t n);
// Plain mode: requests run one after another through hz_compress / hz_decompress.
void hz_batch_set_plain(BatchState* b, bool plain);
bool hz_batch_plain(BatchState* b);
// Most requests one device batch takes when queued submissions merge.
hz_status hz_batch_set_max_reqs(BatchState* b, uint32_t m);
uint32_t hz_batch_max_reqs(BatchState* b);

// Retire finished launches and launch what the slots and budget allow.
void hz_batch_progress(BatchState* b);
// While on, every completed ticket is recorded; drain moves them to `out`.
void hz_batch_track_finished(BatchState* b, bool on);
void hz_batch_drain_finished(BatchState* b, std::vector<uint64_t>& out);
// Non-blocking hz_poll that also reports the device batch that carried the
// ticket and the host steady-clock time (ns) at which its completion was seen.
hz_status hz_batch_take(BatchState* b, uint64_t ticket, hz_status* per_req, uint64_t* out_lens,
                        uint64_t* launch_id, int64_t* done_ns);
