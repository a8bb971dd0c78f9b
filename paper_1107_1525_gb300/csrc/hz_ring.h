// hz_ring.h -- the device-ring allocator of the request replay (hz_serve.cu).
// Plain C++ with no CUDA, so the host tests can build and check it alone.
#pragma once
#include <stdint.h>

#include <deque>

namespace hz {

// First-in first-out allocator over [0, cap): allocations are made in order
// and freed in any order; space comes back when every older one is free.
class Ring {
 public:
  explicit Ring(uint64_t cap) : cap_(cap) {}

  bool alloc(uint64_t size, uint64_t* off, uint64_t* seq) {
    const uint64_t sz = (size + 255) & ~255ull;
    if (sz == 0 || sz > cap_) return false;
    uint64_t at;
    if (live_.empty()) {
      at = 0;
    } else {
      const uint64_t tail = live_.front().off;
      if (head_ > tail) {  // live range [tail, head): room after head, or before tail
        if (head_ + sz <= cap_) at = head_;
        else if (sz <= tail) at = 0;
        else return false;
      } else {  // wrapped: room in [head, tail)
        if (head_ + sz <= tail) at = head_;
        else return false;
      }
    }
    head_ = at + sz;
    live_.push_back({at, false});
    *off = at;
    *seq = first_seq_ + live_.size() - 1;
    return true;
  }

  void release(uint64_t seq) {
    if (seq < first_seq_ || seq - first_seq_ >= live_.size()) return;
    live_[seq - first_seq_].freed = true;
    while (!live_.empty() && live_.front().freed) {
      live_.pop_front();
      ++first_seq_;
    }
    if (live_.empty()) head_ = 0;
  }

 private:
  struct Entry {
    uint64_t off;
    bool freed;
  };
  uint64_t cap_;
  uint64_t head_ = 0;
  uint64_t first_seq_ = 0;
  std::deque<Entry> live_;
};

}  // namespace hz
