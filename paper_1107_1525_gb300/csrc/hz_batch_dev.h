// hz_batch_dev.h -- descriptors of a batch, shared by the host engine
// (hz_batch.cu) and the batched kernels (hz_batch_kernels.cu).
#pragma once

#include "hz_internal.cuh"

namespace hz {

constexpr uint64_t kBatchHistChunk = 256ull << 10;  // bytes per histogram work unit

enum : int { kTicketHist = 0, kTicketSummary = 1, kTicketPack = 2, kTicketDecode = 3, kTickets = 4 };

struct BatchCtl {
  uint32_t ncomp, ndecomp;
  uint32_t hist_units;  // sum over compress requests of ceil(n / kBatchHistChunk)
  uint32_t tiles;       // sum over compress requests of their encoder tiles
  uint32_t dec_units;   // decode units, counted on the device
  uint32_t pad[3];
  uint32_t tickets[kTickets];
  // first work unit of each request, as compact arrays (filled on the device)
  // so that finding a unit's request searches a few cache lines
  uint32_t* hist_base;  // [ncomp]
  uint32_t* tile_base;  // [ncomp]
  uint32_t* unit_base;  // [ndecomp]
};

struct BatchComp {
  const uint8_t* src;
  uint64_t n;
  uint8_t* dst;
  uint64_t cap;
  uint32_t B, nb, ntiles, flags;
  FastDiv fdB;
  DevState* st;
  TileStatus* tiles;
  uint64_t* out_len;
  uint32_t hist_base;  // first histogram unit of this request
  uint32_t tile_base;  // first tile (flattened over the batch)
  uint32_t req;        // index in the submitted batch
  uint32_t pad;
};

struct BatchDecomp {
  const uint8_t* src;
  uint64_t in_len;
  uint8_t* dst;
  uint64_t cap;
  DevState* st;
  DecTables* T;
  uint64_t* out_len;
  uint32_t lut_bits;
  uint32_t unit_base;  // written on the device
  uint32_t per_warp;   // blocks per warp in a decode unit, written on the device
  uint32_t req;
};

struct BatchResult {
  uint32_t req;
  int32_t status;
  uint64_t out_len;
};

struct BatchLaunch {
  BatchCtl* ctl;
  BatchComp* comps;
  BatchDecomp* decomps;
  BatchResult* results;
  int num_sms;
};

// Enqueue the batch's kernels on s (captured in a graph by the host).
void batch_enqueue(const BatchLaunch& L, cudaStream_t s);
// One-time kernel attributes; call before any capture.
void batch_configure();
size_t batch_dec_tables_bytes();

}  // namespace hz
