// hz_chase.h -- scratch and launch of the parallel offset chase (hz_chase.cu).
#pragma once
#include "hz_internal.cuh"

namespace hz {

// Device scratch of the chase, carved by the host out of one allocation.
struct ChaseScratch {
  uint32_t* bar;      // bar[0..1]: grid barrier; bar[2]: the fallback flag (flag == bar + 2)
  uint32_t* flag;
  uint32_t* cta_tot;  // per CTA, plus one: candidate counts
  uint32_t cta_cap;
  uint32_t* bitmap;   // one bit per record-area word
  uint32_t* base;     // candidates before each bitmap word
  uint32_t bm_cap;    // bitmap words available
  uint32_t* pos;      // candidate -> record-area word
  uint32_t *s0, *s1;  // jump pointers
  uint32_t *r0, *r1;  // records to the pointer target
  uint32_t c_cap;     // candidates available
  uint32_t* hits;     // per record: candidates claiming it
};

struct DecTables;
// Queue the chase on s: it does nothing unless the decode set-up left the
// offsets to it (a stream without an index, DecodeArgs::defer_chase set).
cudaError_t launch_decode_chase(const DecodeArgs& a, DecTables* T, const ChaseScratch& cs,
                                int num_sms, cudaStream_t s);

}  // namespace hz
