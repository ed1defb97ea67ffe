/*
 * Plain CPU oracle.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and
 * the benchmark's CPU baseline are its only users; the CUDA library never
 * includes, links or calls it.  See oracle.h for the contract of each function.
 *
 * Citations name the paper's algorithms and tables: Algorithm 1 (Optimized
 * Merge Sort with Sorting Networks), Algorithm 2 (Optimized Quick Sort with
 * Sorting Networks), Table 3 (Sorting Network Configurations).
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Networks.  The paper uses fixed sorting networks for sizes 3..8 (Section 1
 * and Section 3).  Their comparator lists are not printed, so this oracle
 * derives its own: Batcher's odd-even merge sort (Batcher 1968; Knuth, TAOCP
 * vol. 3, Section 5.3.4) on 4 wires for m <= 4 and on 8 wires for m >= 5,
 * pruned to m wires by treating wires >= m as +infinity (a comparator that
 * touches such a wire never moves anything and is deleted).  The result has
 * 3/5/9/12/16/19 comparators for m = 3..8.                                  */

#define OR_MAX_CE 32

typedef struct {
    int n;
    int lo[OR_MAX_CE];
    int hi[OR_MAX_CE];
} or_net;

static or_net g_nets[9];
static int g_nets_ready = 0;

static void oem_push(or_net *net, int i, int j) {
    net->lo[net->n] = i;
    net->hi[net->n] = j;
    net->n++;
}

/* Batcher's merge of the two sorted halves of wires lo..lo+n-1, taking every
 * r-th wire (the odd/even subsequence recursion). */
static void oem_merge(or_net *net, int lo, int n, int r) {
    int step = 2 * r;
    if (step < n) {
        oem_merge(net, lo, n, step);     /* even subsequence */
        oem_merge(net, lo + r, n, step); /* odd subsequence */
        for (int i = lo + r; i + r < lo + n; i += step) oem_push(net, i, i + r);
    } else {
        oem_push(net, lo, lo + r);
    }
}

static void oem_sort(or_net *net, int lo, int n) {
    if (n > 1) {
        int m = n / 2;
        oem_sort(net, lo, m);
        oem_sort(net, lo + m, m);
        oem_merge(net, lo, n, 1);
    }
}

static void build_nets(void) {
    if (g_nets_ready) return;
    or_net full4, full8;
    memset(&full4, 0, sizeof full4);
    memset(&full8, 0, sizeof full8);
    oem_sort(&full4, 0, 4);
    oem_sort(&full8, 0, 8);
    for (int m = 2; m <= 8; m++) {
        or_net *src = (m <= 4) ? &full4 : &full8;
        or_net *dst = &g_nets[m];
        memset(dst, 0, sizeof *dst);
        for (int c = 0; c < src->n; c++)
            if (src->hi[c] < m) oem_push(dst, src->lo[c], src->hi[c]);
    }
    g_nets_ready = 1;
}

int or_network(int m, int *pairs, int cap) {
    if (m < 2 || m > 8) return -1;
    build_nets();
    const or_net *net = &g_nets[m];
    for (int c = 0; c < net->n && c < cap; c++) {
        pairs[2 * c] = net->lo[c];
        pairs[2 * c + 1] = net->hi[c];
    }
    return net->n;
}

/* Compare-exchange: afterwards a[i] <= a[j]. */
void or_apply_network(int m, int32_t *a) {
    build_nets();
    const or_net *net = &g_nets[m];
    for (int c = 0; c < net->n; c++) {
        int i = net->lo[c], j = net->hi[c];
        if (a[j] < a[i]) {
            int32_t t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
}

/* Pair form: orders by (key, original position) so that the network result is
 * the stable order even though networks themselves are not stable. */
static void apply_network_pairs(int m, int32_t *k, int32_t *v, int64_t *p) {
    const or_net *net = &g_nets[m];
    for (int c = 0; c < net->n; c++) {
        int i = net->lo[c], j = net->hi[c];
        if (k[j] < k[i] || (k[j] == k[i] && p[j] < p[i])) {
            int32_t tk = k[i]; k[i] = k[j]; k[j] = tk;
            int32_t tv = v[i]; v[i] = v[j]; v[j] = tv;
            int64_t tp = p[i]; p[i] = p[j]; p[j] = tp;
        }
    }
}

/* The size k of a VarSortk configuration, else 0. */
static int varsort_size(uint32_t netset) {
    if (!(netset & OR_VARSORT)) return 0;
    for (int k = 3; k <= 8; ++k)
        if ((netset & ~OR_VARSORT) == (1u << k)) return k;
    return 0;
}

/* "size matches sorting network size" (Algorithm 1 and 2): for a set of fixed
 * networks, membership of size in the configuration's set (Table 3); for
 * VarSortk, any size from 2 to k.  Returns the network to apply (0: none). */
static int leaf_network(int64_t size, uint32_t netset) {
    const int k = varsort_size(netset);
    if (k) return (size >= 2 && size <= k) ? k : 0;
    return (size >= 3 && size <= 8 && ((netset >> size) & 1u)) ? (int)size : 0;
}

static int netset_valid(uint32_t netset) {
    if (netset & OR_VARSORT) return varsort_size(netset) != 0;
    return (netset & ~0x1F8u) == 0;
}

/* Sorts a[0..size) with the size-m network (m >= size): the keys are copied
 * into m slots, the missing ones set to +infinity, and the first size copied
 * back (for size == m this is the plain network). */
static void apply_leaf(int m, int32_t *a, int64_t size) {
    int32_t t[8];
    for (int i = 0; i < m; ++i) t[i] = i < size ? a[i] : INT32_MAX;
    or_apply_network(m, t);
    for (int64_t i = 0; i < size; ++i) a[i] = t[i];
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1.                                                              */

void or_merge(int32_t *a, int64_t left, int64_t mid, int64_t right, int32_t *tmp) {
    int64_t i = left, j = mid + 1, o = 0;
    while (i <= mid && j <= right) {
        if (a[j] < a[i]) tmp[o++] = a[j++]; /* right wins only when strictly smaller */
        else tmp[o++] = a[i++];
    }
    while (i <= mid) tmp[o++] = a[i++];
    while (j <= right) tmp[o++] = a[j++];
    memcpy(a + left, tmp, (size_t)o * sizeof(int32_t));
}

static void merge_sort_rec(int32_t *a, int64_t left, int64_t right, uint32_t netset,
                           int32_t *tmp, or_counters *c, uint64_t depth) {
    if (c && depth > c->max_depth) c->max_depth = depth;
    int64_t size = right - left + 1;
    const int m = leaf_network(size, netset);
    if (m) {
        apply_leaf(m, a + left, size);
        if (c) c->net_calls[m]++;
        return;
    }
    if (left < right) {
        int64_t mid = left + (right - left) / 2;
        merge_sort_rec(a, left, mid, netset, tmp, c, depth + 1);
        merge_sort_rec(a, mid + 1, right, netset, tmp, c, depth + 1);
        or_merge(a, left, mid, right, tmp);
        if (c) c->merge_calls++;
    }
}

int or_merge_sort(int32_t *a, int64_t n, uint32_t netset, or_counters *c) {
    if (!netset_valid(netset) || n < 0) return -1;
    if (n == 0) return 0;
    build_nets();
    int32_t *tmp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!tmp) return -2;
    merge_sort_rec(a, 0, n - 1, netset, tmp, c, 0);
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 on int64 keys: the same recursion, leaf rule and stable merge. */

static void apply_network_i64(int m, int64_t *a) {
    const or_net *net = &g_nets[m];
    for (int c = 0; c < net->n; c++) {
        int i = net->lo[c], j = net->hi[c];
        if (a[j] < a[i]) {
            int64_t t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
}

static void apply_leaf_i64(int m, int64_t *a, int64_t size) {
    int64_t t[8];
    for (int i = 0; i < m; ++i) t[i] = i < size ? a[i] : INT64_MAX;
    apply_network_i64(m, t);
    for (int64_t i = 0; i < size; ++i) a[i] = t[i];
}

static void merge_i64(int64_t *a, int64_t left, int64_t mid, int64_t right, int64_t *tmp) {
    int64_t i = left, j = mid + 1, o = 0;
    while (i <= mid && j <= right) {
        if (a[j] < a[i]) tmp[o++] = a[j++];
        else tmp[o++] = a[i++];
    }
    while (i <= mid) tmp[o++] = a[i++];
    while (j <= right) tmp[o++] = a[j++];
    memcpy(a + left, tmp, (size_t)o * sizeof(int64_t));
}

static void merge_sort_rec_i64(int64_t *a, int64_t left, int64_t right, uint32_t netset,
                               int64_t *tmp, or_counters *c, uint64_t depth) {
    if (c && depth > c->max_depth) c->max_depth = depth;
    int64_t size = right - left + 1;
    const int m = leaf_network(size, netset);
    if (m) {
        apply_leaf_i64(m, a + left, size);
        if (c) c->net_calls[m]++;
        return;
    }
    if (left < right) {
        int64_t mid = left + (right - left) / 2;
        merge_sort_rec_i64(a, left, mid, netset, tmp, c, depth + 1);
        merge_sort_rec_i64(a, mid + 1, right, netset, tmp, c, depth + 1);
        merge_i64(a, left, mid, right, tmp);
        if (c) c->merge_calls++;
    }
}

int or_merge_sort_i64(int64_t *a, int64_t n, uint32_t netset, or_counters *c) {
    if (!netset_valid(netset) || n < 0) return -1;
    if (n == 0) return 0;
    build_nets();
    int64_t *tmp = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!tmp) return -2;
    merge_sort_rec_i64(a, 0, n - 1, netset, tmp, c, 0);
    free(tmp);
    return 0;
}

/* Pairs: the same recursion; positions ride along only to order equal keys
 * inside networks. */
static void merge_pairs(int32_t *k, int32_t *v, int64_t *p, int64_t left, int64_t mid,
                        int64_t right, int32_t *tk, int32_t *tv, int64_t *tp) {
    int64_t i = left, j = mid + 1, o = 0;
    while (i <= mid && j <= right) {
        if (k[j] < k[i]) { tk[o] = k[j]; tv[o] = v[j]; tp[o] = p[j]; o++; j++; }
        else             { tk[o] = k[i]; tv[o] = v[i]; tp[o] = p[i]; o++; i++; }
    }
    while (i <= mid)   { tk[o] = k[i]; tv[o] = v[i]; tp[o] = p[i]; o++; i++; }
    while (j <= right) { tk[o] = k[j]; tv[o] = v[j]; tp[o] = p[j]; o++; j++; }
    memcpy(k + left, tk, (size_t)o * sizeof(int32_t));
    memcpy(v + left, tv, (size_t)o * sizeof(int32_t));
    memcpy(p + left, tp, (size_t)o * sizeof(int64_t));
}

static void merge_sort_pairs_rec(int32_t *k, int32_t *v, int64_t *p, int64_t left,
                                 int64_t right, uint32_t netset, int32_t *tk, int32_t *tv,
                                 int64_t *tp, or_counters *c, uint64_t depth) {
    if (c && depth > c->max_depth) c->max_depth = depth;
    int64_t size = right - left + 1;
    const int m = leaf_network(size, netset);
    if (m) {
        /* Padded slots carry key +infinity and a position past every real one. */
        int32_t tk8[8], tv8[8];
        int64_t tp8[8];
        for (int i = 0; i < m; ++i) {
            tk8[i] = i < size ? k[left + i] : INT32_MAX;
            tv8[i] = i < size ? v[left + i] : 0;
            tp8[i] = i < size ? p[left + i] : INT64_MAX;
        }
        apply_network_pairs(m, tk8, tv8, tp8);
        for (int64_t i = 0; i < size; ++i) {
            k[left + i] = tk8[i];
            v[left + i] = tv8[i];
            p[left + i] = tp8[i];
        }
        if (c) c->net_calls[m]++;
        return;
    }
    if (left < right) {
        int64_t mid = left + (right - left) / 2;
        merge_sort_pairs_rec(k, v, p, left, mid, netset, tk, tv, tp, c, depth + 1);
        merge_sort_pairs_rec(k, v, p, mid + 1, right, netset, tk, tv, tp, c, depth + 1);
        merge_pairs(k, v, p, left, mid, right, tk, tv, tp);
        if (c) c->merge_calls++;
    }
}

int or_merge_sort_pairs(int32_t *keys, int32_t *vals, int64_t n, uint32_t netset,
                        or_counters *c) {
    if (!netset_valid(netset) || n < 0) return -1;
    if (n == 0) return 0;
    build_nets();
    int64_t *pos = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *tp = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int32_t *tk = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *tv = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int rc = 0;
    if (!pos || !tp || !tk || !tv) {
        rc = -2;
    } else {
        for (int64_t i = 0; i < n; i++) pos[i] = i;
        merge_sort_pairs_rec(keys, vals, pos, 0, n - 1, netset, tk, tv, tp, c, 0);
    }
    free(pos); free(tp); free(tk); free(tv);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2.  MedianOfThree and HoarePartition are named but not printed;
 * this is the textbook reading (median-of-three ordering of the first, middle
 * and last element; Hoare's two-pointer scan with the median as pivot).     */

static void swap32(int32_t *a, int64_t i, int64_t j) {
    int32_t t = a[i];
    a[i] = a[j];
    a[j] = t;
}

int64_t or_median_of_three(int32_t *a, int64_t low, int64_t high) {
    int64_t mid = low + (high - low) / 2;
    if (a[mid] < a[low]) swap32(a, mid, low);
    if (a[high] < a[low]) swap32(a, high, low);
    if (a[high] < a[mid]) swap32(a, high, mid);
    return mid;
}

int64_t or_hoare_partition(int32_t *a, int64_t low, int64_t high, int64_t pivot_index) {
    int32_t pivot = a[pivot_index];
    int64_t i = low - 1, j = high + 1;
    for (;;) {
        do { i++; } while (a[i] < pivot);
        do { j--; } while (a[j] > pivot);
        if (i >= j) return j;
        swap32(a, i, j);
    }
}

static void quick_sort_rec(int32_t *a, int64_t low, int64_t high, uint32_t netset,
                           or_counters *c, uint64_t depth) {
    if (c && depth > c->max_depth) c->max_depth = depth;
    int64_t size = high - low + 1;
    const int m = leaf_network(size, netset);
    if (m) {
        apply_leaf(m, a + low, size);
        if (c) c->net_calls[m]++;
        return;
    }
    if (low < high) {
        int64_t pivot_index = or_median_of_three(a, low, high);
        int64_t p = or_hoare_partition(a, low, high, pivot_index);
        if (c) c->partition_calls++;
        quick_sort_rec(a, low, p, netset, c, depth + 1);
        quick_sort_rec(a, p + 1, high, netset, c, depth + 1);
    }
}

int or_quick_sort(int32_t *a, int64_t n, uint32_t netset, or_counters *c) {
    if (!netset_valid(netset) || n < 0) return -1;
    if (n == 0) return 0;
    build_nets();
    quick_sort_rec(a, 0, n - 1, netset, c, 0);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Segments and checks.                                                      */

int or_segsort(int32_t *a, const int64_t *off, int64_t nseg, int algo, uint32_t netset) {
    for (int64_t s = 0; s < nseg; s++) {
        int64_t b = off[s], e = off[s + 1];
        if (e < b) return -1;
        int rc = (algo == 0) ? or_merge_sort(a + b, e - b, netset, NULL)
                             : or_quick_sort(a + b, e - b, netset, NULL);
        if (rc) return rc;
    }
    return 0;
}

int or_is_sorted(const int32_t *a, int64_t n) {
    for (int64_t i = 1; i < n; i++)
        if (a[i] < a[i - 1]) return 0;
    return 1;
}

int64_t or_count_less(const int32_t *a, int64_t n, int32_t v) {
    int64_t c = 0;
    for (int64_t i = 0; i < n; i++) c += (a[i] < v);
    return c;
}

int64_t or_count_less_equal(const int32_t *a, int64_t n, int32_t v) {
    int64_t c = 0;
    for (int64_t i = 0; i < n; i++) c += (a[i] <= v);
    return c;
}
