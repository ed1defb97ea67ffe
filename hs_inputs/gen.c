/*
 * Fast C form of the seeded input generators in hs_inputs/__init__.py (same
 * definitions, checked against the numpy forms by tests/test_inputs.py).
 * Holds no sorting arithmetic.  SplitMix64 (Steele, Lea, Flood, OOPSLA 2014)
 * used counter-based: output i of stream `seed` is mix(seed + (i+1)*gamma).
 */
#include <stdint.h>

static inline uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t sm(uint64_t seed, uint64_t i) {
    return mix(seed + (i + 1) * 0x9E3779B97F4A7C15ULL);
}

static inline int32_t clip32(int64_t v) {
    if (v < INT32_MIN) return INT32_MIN;
    if (v > INT32_MAX) return INT32_MAX;
    return (int32_t)v;
}

/* Low 32 bits of outputs start .. start+count-1. */
void hsg_u32(uint64_t seed, uint64_t start, uint64_t count, uint32_t *out) {
    for (uint64_t i = 0; i < count; i++) out[i] = (uint32_t)sm(seed, start + i);
}

/* Ascending keys: running sum of gaps (output i mod max(1, 2^33/n)) - 2^31. */
void hsg_sorted(uint64_t seed, int64_t n, int32_t *out) {
    if (n <= 0) return;
    uint64_t max_gap = (1ULL << 33) / (uint64_t)n;
    if (max_gap < 1) max_gap = 1;
    int64_t acc = 0;
    for (int64_t i = 0; i < n; i++) {
        acc += (int64_t)(sm(seed, (uint64_t)i) % max_gap);
        out[i] = clip32(acc - (1LL << 31));
    }
}

/* Sorted, then floor(n/100) sequential swaps of (draw 2t mod n, draw 2t+1 mod n)
 * from stream seed ^ 0x6E6561726C79. */
void hsg_nearly(uint64_t seed, int64_t n, int32_t *out) {
    hsg_sorted(seed, n, out);
    int64_t k = n / 100;
    uint64_t s2 = seed ^ 0x6E6561726C79ULL;
    for (int64_t t = 0; t < k; t++) {
        int64_t i = (int64_t)(sm(s2, 2 * (uint64_t)t) % (uint64_t)n);
        int64_t j = (int64_t)(sm(s2, 2 * (uint64_t)t + 1) % (uint64_t)n);
        int32_t x = out[i];
        out[i] = out[j];
        out[j] = x;
    }
}

/* Segmented workload (see hs_inputs.segmented): random keys everywhere from
 * stream seed ^ 0x6B657973; sorted / nearly segments (dist 1 / 2) rebuilt as
 * segment-local running sums of gaps from one stream (seed ^ 0x67617073)
 * indexed over their positions in segment order; nearly segments then get
 * floor(size/100) sequential swaps from one stream (seed ^ 0x6E656172). */
void hsg_segmented(uint64_t seed, int64_t nseg, const int64_t *off, const int64_t *dist,
                   int32_t *out) {
    int64_t total = off[nseg];
    hsg_u32(seed ^ 0x6B657973ULL, 0, (uint64_t)total, (uint32_t *)out);
    uint64_t gs = seed ^ 0x67617073ULL, ns = seed ^ 0x6E656172ULL;
    uint64_t gpos = 0, npos = 0;
    for (int64_t s = 0; s < nseg; s++) {
        int64_t b = off[s], size = off[s + 1] - off[s];
        if (dist[s] == 0 || size <= 0) continue;
        uint64_t max_gap = (1ULL << 33) / (uint64_t)size;
        if (max_gap < 1) max_gap = 1;
        int64_t acc = 0;
        for (int64_t i = 0; i < size; i++) {
            acc += (int64_t)(sm(gs, gpos++) % max_gap);
            out[b + i] = clip32(acc - (1LL << 31));
        }
    }
    for (int64_t s = 0; s < nseg; s++) {
        int64_t b = off[s], size = off[s + 1] - off[s];
        if (dist[s] != 2 || size <= 0) continue;
        for (int64_t t = 0; t < size / 100; t++) {
            int64_t i = b + (int64_t)(sm(ns, npos++) % (uint64_t)size);
            int64_t j = b + (int64_t)(sm(ns, npos++) % (uint64_t)size);
            int32_t x = out[i];
            out[i] = out[j];
            out[j] = x;
        }
    }
}
