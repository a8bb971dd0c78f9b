/*
 * hz_oracle.h -- declarations of the CPU oracle's functions (hz_oracle.c), for
 * its own translation units only (the OpenMP driver in hz_oracle_omp.c).  TEST
 * INFRASTRUCTURE ONLY; nothing of the CUDA library includes it.
 */
#ifndef HZ_ORACLE_H
#define HZ_ORACLE_H

#include <stdint.h>

/* Canonical decoding tables: per length the first code value and the number
 * of codes, and the symbols in (length, symbol) order. */
typedef struct {
  uint64_t first[65];
  uint64_t count[65];
  int start[65];
  int sorted[256];
} oracle_dec_tables;

void oracle_histogram(const uint8_t* x, uint64_t n, uint64_t* freq);
int oracle_code_lengths(const uint64_t* freq, uint8_t* len);
int oracle_canonical_codes(const uint8_t* len, uint64_t* code);
uint64_t oracle_block_bits(const uint8_t* x, uint64_t count, const uint8_t* len);
int oracle_layout_ok(uint32_t flags, uint32_t B, uint32_t S);
const uint8_t* oracle_sub_entries(const uint8_t* s, uint32_t nb, uint32_t B, uint32_t flags,
                                  uint32_t S, uint64_t k);
uint64_t oracle_records_at(uint64_t nb, uint32_t B, uint32_t flags, uint32_t S);
int oracle_stream_code(const uint8_t* x, uint64_t n, const uint8_t* given_len, uint8_t* len,
                       uint64_t* code);
void oracle_write_header(uint8_t* out, uint64_t n, uint32_t B, uint32_t nb, uint32_t flags,
                         uint32_t S, const uint8_t* len);
int oracle_write_block(uint8_t* out, const uint8_t* x, uint64_t n, uint32_t B, uint32_t nb,
                       uint32_t flags, uint32_t S, const uint8_t* len, const uint64_t* code,
                       uint64_t k, uint64_t word_off);
int oracle_compress(const uint8_t* x, uint64_t n, uint32_t B, const uint8_t* given_len,
                    uint32_t flags, uint32_t S, uint8_t* out, uint64_t cap, uint64_t* out_len);
int oracle_parse_header(const uint8_t* s, uint64_t s_len, uint64_t* n, uint32_t* flags,
                        uint32_t* B, uint32_t* nb, uint32_t* S, uint8_t* len);
void oracle_decode_tables(const uint8_t* len, oracle_dec_tables* t);
int oracle_locate_records(const uint8_t* s, uint64_t s_len, uint32_t flags, uint32_t B,
                          uint32_t nb, uint32_t S, uint64_t* rec_at);
int oracle_decode_block(const oracle_dec_tables* t, const uint8_t* rec, uint64_t count,
                        const uint8_t* sub, uint32_t S, uint32_t M, uint8_t* out);
int oracle_decompress(const uint8_t* s, uint64_t s_len, uint8_t* out, uint64_t cap,
                      uint64_t* n_out);

#endif /* HZ_ORACLE_H */
