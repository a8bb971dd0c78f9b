/*
 * hz_oracle_omp.c -- the oracle's coder spread over host cores with OpenMP,
 * the CPU side of the paper's sequential vs. OpenMP comparison (Sec. 3.1
 * Encoding and Sec. 3.2 Decoding, both of which time an OpenMP coder that
 * works on independent blocks).
 *
 * TEST AND BASELINE INFRASTRUCTURE ONLY, like hz_oracle.c: only the test
 * suite and the benchmark's CPU-baseline leg may load it.  It contains no
 * coding arithmetic of its own: every step is one of the oracle's functions
 * (hz_oracle.h), called for independent blocks (or, for the histogram,
 * independent slices whose counts are added) from an OpenMP loop.  The only
 * sequential steps are the exclusive sum of record sizes that places the
 * records and the delimiter walk that locates them.  Its streams must equal
 * oracle_compress's byte for byte, which the tests check.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

#include "hz_oracle.h"

#define OMP_OK 0
#define OMP_ERR_ARG (-1)
#define OMP_ERR_CAPACITY (-2)
#define OMP_ERR_CORRUPT (-3)
#define OMP_ERR_NOMEM (-4)

static uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

/* Threads the driver uses for `threads` (0 = every core OpenMP offers). */
int oracle_omp_threads(int threads) { return threads > 0 ? threads : omp_get_max_threads(); }

/*
 * oracle_compress with the histogram over slices and the blocks' bit counts
 * and records over blocks in parallel.  Same arguments and results.
 */
int oracle_compress_omp(const uint8_t* x, uint64_t n, uint32_t B, const uint8_t* given_len,
                        uint32_t flags, uint32_t S, uint8_t* out, uint64_t cap,
                        uint64_t* out_len, int threads) {
  *out_len = 0;
  if (B == 0 || B > (1u << 24) || n > 0xFFFFFFFFull || !oracle_layout_ok(flags, B, S))
    return OMP_ERR_ARG;
  int nt = oracle_omp_threads(threads);
  uint8_t len[256];
  uint64_t code[256];
  int st;
  if (given_len) {
    st = oracle_stream_code(x, n, given_len, len, code);
  } else {
    /* the histogram of x as the sum of its slices' histograms */
    uint64_t freq[256];
    memset(freq, 0, sizeof(freq));
    uint64_t slice = ceil_div(n ? n : 1, (uint64_t)nt);
#pragma omp parallel num_threads(nt)
    {
      uint64_t f[256];
      uint64_t lo = (uint64_t)omp_get_thread_num() * slice;
      uint64_t hi = lo + slice < n ? lo + slice : n;
      oracle_histogram(x + (lo < n ? lo : n), lo < hi ? hi - lo : 0, f);
#pragma omp critical
      for (int s = 0; s < 256; ++s) freq[s] += f[s];
    }
    st = oracle_code_lengths(freq, len);
    if (st == OMP_OK) st = oracle_canonical_codes(len, code) == OMP_OK ? OMP_OK : OMP_ERR_ARG;
  }
  if (st != OMP_OK) return st;
  uint64_t nb = ceil_div(n, B);
  uint64_t* words = (uint64_t*)malloc((nb + 1) * sizeof(uint64_t));
  if (!words) return OMP_ERR_NOMEM;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16)
  for (int64_t k = 0; k < (int64_t)nb; ++k) {
    uint64_t lo = (uint64_t)k * B, hi = lo + B < n ? lo + B : n;
    words[k] = 1 + ceil_div(oracle_block_bits(x + lo, hi - lo, len), 32);
  }
  /* records back to back: exclusive sum of their sizes */
  uint64_t total = 0;
  for (uint64_t k = 0; k < nb; ++k) {
    uint64_t w = words[k];
    words[k] = total;
    total += w;
  }
  uint64_t size = oracle_records_at(nb, B, flags, S) + 4 * total;
  *out_len = size;
  if (size > cap) {
    free(words);
    return OMP_ERR_CAPACITY;
  }
  memset(out, 0, size);
  oracle_write_header(out, n, B, (uint32_t)nb, flags, S, len);
  int bad = 0;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16) reduction(| : bad)
  for (int64_t k = 0; k < (int64_t)nb; ++k)
    bad |= oracle_write_block(out, x, n, B, (uint32_t)nb, flags, S, len, code, (uint64_t)k,
                              words[k]) != OMP_OK;
  free(words);
  return bad ? OMP_ERR_NOMEM : OMP_OK;
}

/*
 * oracle_decompress with the blocks decoded in parallel after the sequential
 * delimiter walk.  Same arguments and results (every decoding error is
 * OMP_ERR_CORRUPT, as in the oracle).
 */
int oracle_decompress_omp(const uint8_t* s, uint64_t s_len, uint8_t* out, uint64_t cap,
                          uint64_t* n_out, int threads) {
  uint64_t n;
  uint32_t flags, B, nb, S;
  uint8_t len[256];
  *n_out = 0;
  int st = oracle_parse_header(s, s_len, &n, &flags, &B, &nb, &S, len);
  if (st != OMP_OK) return st;
  *n_out = n;
  if (n > cap) return OMP_ERR_CAPACITY;
  oracle_dec_tables t;
  oracle_decode_tables(len, &t);
  uint64_t* rec_at = (uint64_t*)malloc((nb ? nb : 1) * sizeof(uint64_t));
  if (!rec_at) return OMP_ERR_NOMEM;
  st = oracle_locate_records(s, s_len, flags, B, nb, S, rec_at);
  if (st != OMP_OK) {
    free(rec_at);
    return st;
  }
  uint32_t M = S ? B / S : 1;
  int nt = oracle_omp_threads(threads);
  int bad = 0;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 16) reduction(| : bad)
  for (int64_t k = 0; k < (int64_t)nb; ++k) {
    uint64_t lo = (uint64_t)k * B, hi = lo + B < n ? lo + B : n;
    const uint8_t* sub = oracle_sub_entries(s, nb, B, flags, S, (uint64_t)k);
    bad |= oracle_decode_block(&t, s + rec_at[k], hi - lo, sub, S, M, out + lo) != OMP_OK;
  }
  free(rec_at);
  return bad ? OMP_ERR_CORRUPT : OMP_OK;
}
