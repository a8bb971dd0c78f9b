"""The request replay's device-ring allocator (csrc/hz_ring.h), built alone with
g++ and driven by random alloc / out-of-order free traffic: live ranges must
stay inside the ring, never overlap, be 256-byte aligned, and an empty ring
must take any request up to its capacity."""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1107_1525_gb300", "csrc")

HARNESS = r"""
#include <stdio.h>
#include <stdlib.h>
#include <vector>
#include <algorithm>
#include "hz_ring.h"

struct Live { uint64_t off, size, seq; };

static uint64_t rng_state = 88172645463325252ull;
static uint64_t next_rand() {  // xorshift64
  rng_state ^= rng_state << 13; rng_state ^= rng_state >> 7; rng_state ^= rng_state << 17;
  return rng_state;
}

int main() {
  for (int trial = 0; trial < 40; ++trial) {
    const uint64_t cap = 4096 + (next_rand() % 64) * 256;
    hz::Ring ring(cap);
    std::vector<Live> live;
    uint64_t ok = 0, refused = 0;
    for (int step = 0; step < 20000; ++step) {
      if (live.empty() || next_rand() % 100 < 55) {
        const uint64_t size = 1 + next_rand() % (cap / 3);
        uint64_t off = 0, seq = 0;
        if (ring.alloc(size, &off, &seq)) {
          const uint64_t sz = (size + 255) & ~255ull;
          if (off % 256 || off + sz > cap) { printf("out of range\n"); return 1; }
          for (const Live& l : live)
            if (off < l.off + l.size && l.off < off + sz) { printf("overlap\n"); return 1; }
          live.push_back({off, sz, seq});
          ++ok;
        } else {
          ++refused;
          if (live.empty()) { printf("empty ring refused %llu\n", (unsigned long long)size); return 1; }
        }
      } else {
        const size_t k = next_rand() % live.size();
        ring.release(live[k].seq);
        live.erase(live.begin() + k);
      }
    }
    for (const Live& l : live) ring.release(l.seq);
    uint64_t off = 0, seq = 0;
    if (!ring.alloc(cap, &off, &seq) || off != 0) { printf("not empty at the end\n"); return 1; }
    if (!ok || !refused) { printf("traffic did not exercise both paths\n"); return 1; }
  }
  printf("ok\n");
  return 0;
}
"""


def test_ring_allocator(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "ring_test.cc"
    src.write_text(HARNESS)
    exe = tmp_path / "ring_test"
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout
