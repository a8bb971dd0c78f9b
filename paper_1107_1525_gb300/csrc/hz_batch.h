// hz_batch.h -- batch submission and admission behind hz_submit / hz_poll.
#pragma once
#include <stdint.h>

#include "hz.h"

struct BatchState;

BatchState* hz_batch_create(int device, int num_sms, uint64_t mem_budget);
void hz_batch_destroy(BatchState* b);
hz_status hz_batch_submit(BatchState* b, hz_ctx* ctx, const hz_request* reqs, uint32_t count,
                          uint64_t* ticket);
hz_status hz_batch_poll(BatchState* b, uint64_t ticket, int64_t timeout_ns, hz_status* per_req,
                        uint64_t* out_lens);
// Block size used when a caller passes 0 and nothing has been tuned.
uint32_t hz_batch_tuned_block_size(uint64_t n);
// Plain mode: requests run one after another through hz_compress / hz_decompress.
void hz_batch_set_plain(BatchState* b, bool plain);
bool hz_batch_plain(BatchState* b);
