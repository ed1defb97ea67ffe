/*
 * Plain CPU oracle for hybrid network-leaf merge sort and quick sort
 * (Aly, Jensen, ElAarag, "Improving Merge Sort and Quick Sort Performance by
 * Utilizing AlphaDev's Sorting Networks as Base Cases", ACMSE 2025).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this library: only the tests, the smoke check and the benchmark's CPU
 * baseline use it.  It shares no code, header, table or generator with the
 * CUDA library; its networks come from Batcher's odd-even merge sort (the CUDA
 * side builds Bose-Nelson networks instead).
 *
 * Everything is single-threaded, sequential and written to be read against the
 * paper: Algorithm 1 and Algorithm 2 are followed step by step.  Keys are
 * signed 32-bit integers (the paper does not state the element type).
 *
 * Network sets (Table 3, "Sorting Network Configurations"): bit k of a netset
 * means "a network of size k is available", k in 3..8.  0 is the classical
 * algorithm with no networks.  OR_VARSORT together with exactly one size bit
 * k is VarSortk (Table 3's VarSort3/4/5, "dynamic sorting networks" for any
 * input of up to k elements): every subarray of 2..k elements is a leaf,
 * sorted by the size-k network on a copy padded with +infinity sentinels.
 */
#ifndef HS_ORACLE_H
#define HS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_VARSORT 0x10000u

/* Instrumentation counters, filled by the sorts when non-NULL. */
typedef struct {
    uint64_t merge_calls;     /* calls of Merge (Algorithm 1) */
    uint64_t net_calls[9];    /* net_calls[k]: sortk applications, k in 3..8 */
    uint64_t partition_calls; /* calls of HoarePartition (Algorithm 2) */
    uint64_t max_depth;       /* deepest recursion level reached (root = 0) */
} or_counters;

/* Comparator list of the size-m network (m in 2..8), Batcher's odd-even merge
 * sort pruned to m wires.  Writes up to cap pairs (lo, hi) into pairs[2*i],
 * pairs[2*i+1]; returns the number of comparators, or -1 if m is out of range. */
int or_network(int m, int *pairs, int cap);

/* Applies the size-m network to a[0..m-1] (ApplySortingNetwork, Algorithm 1). */
void or_apply_network(int m, int32_t *a);

/* Merge(array, left, mid, right) of Algorithm 1: stable two-way merge of the
 * sorted runs a[left..mid] and a[mid+1..right] (inclusive bounds) through the
 * caller's scratch tmp (at least right-left+1 elements).  Ties take the left
 * run's element first. */
void or_merge(int32_t *a, int64_t left, int64_t mid, int64_t right, int32_t *tmp);

/* Algorithm 1 on a[0..n-1].  netset: Table 3 bitmask (0 = classical). */
int or_merge_sort(int32_t *a, int64_t n, uint32_t netset, or_counters *c);

/* Algorithm 1 on int64 keys a[0..n-1] (same networks, leaf rule and stable
 * Merge as or_merge_sort). */
int or_merge_sort_i64(int64_t *a, int64_t n, uint32_t netset, or_counters *c);

/* MedianOfThree(array, low, high) of Algorithm 2: orders a[low], a[mid],
 * a[high] in place, mid = low + (high-low)/2, and returns mid. */
int64_t or_median_of_three(int32_t *a, int64_t low, int64_t high);

/* HoarePartition(array, low, high, pivotIndex) of Algorithm 2 (Hoare 1962):
 * partitions a[low..high] around the value a[pivotIndex] and returns j with
 * every element of a[low..j] <= pivot <= every element of a[j+1..high]. */
int64_t or_hoare_partition(int32_t *a, int64_t low, int64_t high, int64_t pivot_index);

/* Algorithm 2 on a[0..n-1]. */
int or_quick_sort(int32_t *a, int64_t n, uint32_t netset, or_counters *c);

/* Stable key/value form of Algorithm 1: networks compare (key, original
 * position); Merge takes the left run on ties.  Values travel with keys. */
int or_merge_sort_pairs(int32_t *keys, int32_t *vals, int64_t n, uint32_t netset,
                        or_counters *c);

/* Sorts each segment a[off[s] .. off[s+1]-1], s < nseg, independently with
 * Algorithm 1 (algo 0) or Algorithm 2 (algo 1). */
int or_segsort(int32_t *a, const int64_t *off, int64_t nseg, int algo, uint32_t netset);

/* Checks used by tests at sizes where a full oracle run is too slow. */
int or_is_sorted(const int32_t *a, int64_t n);
int64_t or_count_less(const int32_t *a, int64_t n, int32_t v);
int64_t or_count_less_equal(const int32_t *a, int64_t n, int32_t v);

#ifdef __cplusplus
}
#endif
#endif
