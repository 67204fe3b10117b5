/* Seeded synthetic error / syndrome generator (input side only).
 *
 * Error model: i.i.d. Bernoulli(p_v) flip per column v of H (code-capacity
 * or phenomenological noise on the space-time matrix).  Column v of shot g
 * is in error iff  u < thresh[v],  where thresh[v] = floor(p_v * 2^32) and u
 * is the low 32 bits of the SplitMix64 output at counter (g << 32) | v.
 * The syndrome is s = H e (mod 2).
 *
 * SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the k-th output (k >= 1) of
 * the stream with initial state x is mix(x + k * 0x9E3779B97F4A7C15), which
 * makes it counter-addressable.  Bits pack little-endian: bit j of 64-bit
 * word w is index 64 w + j.
 *
 * This file holds none of the decoder's arithmetic.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t synth_splitmix64_at(uint64_t seed, uint64_t counter) {
    return sm64_mix(seed + (counter + 1ULL) * 0x9E3779B97F4A7C15ULL);
}

typedef struct {
    int m, n;
    const int32_t *col_ptr, *row_idx;
    const uint32_t *thresh;
    uint64_t seed, shot_offset;
    int64_t lo, hi;
    uint64_t *err_out, *syn_out;
} job_t;

static void *run(void *arg) {
    job_t *j = (job_t *)arg;
    const int wn = (j->n + 63) / 64, wm = (j->m + 63) / 64;
    uint64_t *e = (uint64_t *)calloc((size_t)wn, 8);
    uint64_t *s = (uint64_t *)calloc((size_t)wm, 8);
    for (int64_t b = j->lo; b < j->hi; ++b) {
        memset(e, 0, (size_t)wn * 8);
        memset(s, 0, (size_t)wm * 8);
        const uint64_t g = j->shot_offset + (uint64_t)b;
        for (int v = 0; v < j->n; ++v) {
            if (j->thresh[v] == 0) continue;
            uint32_t u = (uint32_t)synth_splitmix64_at(j->seed, (g << 32) | (uint64_t)v);
            if (u < j->thresh[v]) {
                e[v >> 6] |= 1ULL << (v & 63);
                for (int k = j->col_ptr[v]; k < j->col_ptr[v + 1]; ++k) {
                    int c = j->row_idx[k];
                    s[c >> 6] ^= 1ULL << (c & 63);
                }
            }
        }
        if (j->err_out) memcpy(j->err_out + (size_t)b * wn, e, (size_t)wn * 8);
        memcpy(j->syn_out + (size_t)b * wm, s, (size_t)wm * 8);
    }
    free(e);
    free(s);
    return NULL;
}

/* Fill syn_out [num_shots][ceil(m/64)] and, if non-null, err_out
 * [num_shots][ceil(n/64)].  (col_ptr, row_idx) is H in CSC form.
 * Returns 0, or -1 on bad arguments. */
int synth_sample(int m, int n, const int32_t *col_ptr, const int32_t *row_idx,
                 const uint32_t *thresh, uint64_t seed, uint64_t shot_offset,
                 int64_t num_shots, uint64_t *err_out, uint64_t *syn_out,
                 int nthreads) {
    if (m < 0 || n < 0 || num_shots < 0 || !syn_out || !col_ptr || !thresh) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > num_shots) nthreads = num_shots > 0 ? (int)num_shots : 1;
    pthread_t th[256];
    job_t jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        job_t *j = &jobs[t];
        j->m = m; j->n = n; j->col_ptr = col_ptr; j->row_idx = row_idx;
        j->thresh = thresh; j->seed = seed; j->shot_offset = shot_offset;
        j->lo = num_shots * t / nthreads;
        j->hi = num_shots * (t + 1) / nthreads;
        j->err_out = err_out; j->syn_out = syn_out;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, run, &jobs[t]);
    run(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    return 0;
}
