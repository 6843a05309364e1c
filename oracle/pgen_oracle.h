/*
 * pgen oracle -- TEST INFRASTRUCTURE ONLY (see pgen_oracle.c).
 * Plain C, single-threaded; shares nothing with the CUDA library.
 * Return codes: 0 ok, 1 bad argument, 2 out of host memory, 3 capacity.
 */
#ifndef PGEN_ORACLE_H
#define PGEN_ORACLE_H
#include <stdint.h>

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint64_t or_uniform(uint32_t w0, uint32_t w1, uint64_t R);
uint64_t or_coin_threshold(double f);

int or_ba(uint64_t n, uint32_t m, uint32_t n0, uint64_t seed, uint32_t stream, uint64_t* out);

int or_pba_count(const uint32_t* A, uint64_t len, uint32_t B, uint64_t* counts);
int or_pba_phase1_general(uint32_t p, uint32_t B, const uint32_t* flist, uint32_t s,
                          uint64_t n_entries, double f, uint64_t seed,
                          uint32_t* A, uint64_t* counts, uint64_t* fresh_out);
int or_pba_phase1(uint32_t p, uint32_t B, uint32_t W, uint64_t n_entries, double f,
                  uint64_t seed, uint32_t* A, uint64_t* counts, uint64_t* fresh_out);
int or_pba_endpoints(uint32_t q, uint64_t R_q, uint64_t n_b, uint32_t n0, uint64_t seed,
                     uint64_t len, uint32_t* T);
int or_pba_substitute(const uint32_t* A, uint64_t len, uint32_t B, const uint64_t* start,
                      const uint32_t* const* T, uint32_t* out);
int or_pba_factions(uint64_t n, uint32_t m, uint32_t B, uint32_t n0, const uint32_t* foff,
                    const uint32_t* flist, double f, uint64_t seed, uint64_t* out,
                    uint64_t* counts_out, uint64_t* fresh_out);
int or_pba(uint64_t n, uint32_t m, uint32_t B, uint32_t n0, uint32_t W, double f,
           uint64_t seed, uint64_t* out, uint64_t* counts_out, uint64_t* fresh_out);

int or_kron_thresholds(const double* P, uint32_t n0, uint64_t* T);
uint32_t or_kron_pick(const uint64_t* T, uint32_t n_thr, uint32_t w);
int or_kron(const double* P, uint32_t n0, uint32_t k, uint64_t M, uint64_t seed, uint64_t* out);
int or_kron_det(const double* P, uint32_t n0, uint32_t k, uint64_t* out, uint64_t cap,
                uint64_t* n_out, uint64_t* max_depth_out);

int or_csr(const uint64_t* pairs, uint64_t M, uint64_t N, uint64_t* row_ptr, uint64_t* col);
int or_csr_opts(const uint64_t* pairs, uint64_t M, uint64_t N, uint32_t flags, uint64_t* row_ptr,
                uint64_t* col, uint64_t* M_out);
int or_random_cells(uint64_t N, uint64_t M, uint64_t seed, uint64_t* out);

int or_degrees(const uint64_t* pairs, uint64_t M, uint64_t N, int which, uint64_t* deg);
int or_degree_histogram(const uint64_t* deg, uint64_t N, uint64_t max_deg, uint64_t* hist);
int or_bfs(const uint64_t* row_ptr, const uint64_t* col, uint64_t N, uint64_t source,
           uint32_t* dist, uint32_t* levels, uint64_t* scanned);

#endif
