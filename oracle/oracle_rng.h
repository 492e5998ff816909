/*
 * Random-number pieces shared by the two oracle sources (oracle.c: SISe /
 * SISe3; general.c: the general compartment model).  TEST INFRASTRUCTURE ONLY;
 * never included by the CUDA library.
 */
#ifndef ORACLE_RNG_H
#define ORACLE_RNG_H
#include <stdint.h>

typedef struct {
    uint32_t key[2];
    uint32_t ctr[4];
    uint32_t buf[4];
    uint32_t q;                /* next word index */
} word_stream;

void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_uniform(uint32_t lo, uint32_t hi);
double orc_neglog(uint64_t j);
/* The word stream of scheduled event ev_index (position in the day-stable
 * order) on day `day`: Philox counter (ev_index, day | 2^30, block, replicate). */
void orc_ws_start(word_stream* s, uint64_t seed, int32_t replicate, int64_t ev_index, int32_t day);
/* Uniform integer in [0, bound), bound >= 1, from the stream (Lemire 2019). */
uint32_t orc_ws_lemire(word_stream* s, uint32_t bound);

#endif
