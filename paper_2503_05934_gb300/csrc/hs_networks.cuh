// Fixed sorting networks for 2..8 keys held in registers.
//
// The paper sorts base-case subarrays of 3..8 elements with fixed networks
// (Section 1; Algorithm 1 and Algorithm 2, "ApplySortingNetwork") taken from
// AlphaDev's x86 assembly, which is CPU-only.  On the GPU a network is a
// branch-free sequence of min/max compare-exchanges on a thread's register
// array.  The comparator lists are generated at compile time by Bose and
// Nelson's recursive construction (R. C. Bose, R. J. Nelson, "A Sorting
// Problem", J. ACM 9(2), 1962), which is size-optimal for n <= 8:
// 3, 5, 9, 12, 16 and 19 comparators for n = 3..8.
//
// Every index is a template constant, so after inlining the register array
// never touches local memory.  The same templates compile for the host, which
// lets CPU tests check the device networks exhaustively.
#pragma once

#include "hs_common.cuh"

namespace hs {

// Bose-Nelson merge of the sorted wire blocks [I, I+X) and [J, J+Y).
template <int I, int X, int J, int Y>
struct BNMerge {
    template <class Op>
    static HS_HD void run(Op &op) {
        if constexpr (X == 0 || Y == 0) {
        } else if constexpr (X == 1 && Y == 1) {
            op.template ce<I, J>();
        } else if constexpr (X == 1 && Y == 2) {
            op.template ce<I, J + 1>();
            op.template ce<I, J>();
        } else if constexpr (X == 2 && Y == 1) {
            op.template ce<I, J>();
            op.template ce<I + 1, J>();
        } else {
            constexpr int A = X / 2;
            constexpr int B = (X & 1) ? Y / 2 : (Y + 1) / 2;
            BNMerge<I, A, J, B>::run(op);
            BNMerge<I + A, X - A, J + B, Y - B>::run(op);
            BNMerge<I + A, X - A, J, B>::run(op);
        }
    }
};

// Bose-Nelson sort of wires [I, I+N): sort both halves, then merge them.
template <int I, int N>
struct BNSort {
    template <class Op>
    static HS_HD void run(Op &op) {
        if constexpr (N > 1) {
            constexpr int A = N / 2;
            BNSort<I, A>::run(op);
            BNSort<I + A, N - A>::run(op);
            BNMerge<I, A, I + A, N - A>::run(op);
        }
    }
};

// Compare-exchange on keys: afterwards k[i] <= k[j].
struct KeyCE {
    int32_t *k;
    template <int i, int j>
    HS_HD void ce() {
        int32_t a = k[i], b = k[j];
        k[i] = hs_min(a, b);
        k[j] = hs_max(a, b);
    }
};

// Compare-exchange on (key, position) with the value riding along: the
// lexicographic order makes the network's result the stable order.
struct PairCE {
    int32_t *k, *v, *p;
    template <int i, int j>
    HS_HD void ce() {
        int32_t ki = k[i], kj = k[j], vi = v[i], vj = v[j], pi = p[i], pj = p[j];
        bool sw = (kj < ki) || (kj == ki && pj < pi);
        k[i] = sw ? kj : ki;
        k[j] = sw ? ki : kj;
        v[i] = sw ? vj : vi;
        v[j] = sw ? vi : vj;
        p[i] = sw ? pj : pi;
        p[j] = sw ? pi : pj;
    }
};

// Counts comparators and records them (host-side checks only).
struct CountCE {
    int n = 0;
    int *pairs = nullptr;
    int cap = 0;
    template <int i, int j>
    HS_HD void ce() {
        if (pairs && n < cap) {
            pairs[2 * n] = i;
            pairs[2 * n + 1] = j;
        }
        n++;
    }
};

template <int M, class Op>
HS_HD void network(Op &op) {
    BNSort<0, M>::run(op);
}

// Runtime-sized network, used for the ragged leaf at the end of an array.
template <class Op>
HS_HD void network_dyn(int m, Op &op) {
    switch (m) {
        case 2: network<2>(op); break;
        case 3: network<3>(op); break;
        case 4: network<4>(op); break;
        case 5: network<5>(op); break;
        case 6: network<6>(op); break;
        case 7: network<7>(op); break;
        case 8: network<8>(op); break;
        default: break;
    }
}

// Leaf size of a network set (bit k = a size-k network is available, Table 3
// of the paper): the largest available size, or 1 (no network) for the empty
// set, which is the classical algorithm.
HS_HD int leaf_size(uint32_t netset) {
    for (int m = 8; m >= 3; --m)
        if ((netset >> m) & 1u) return m;
    return 1;
}

// Network used for a ragged leaf of r live keys (r < leaf size): the size-r
// network when the set has one, else the smallest available size above r,
// with the missing keys padded by +infinity sentinels.
HS_HD int ragged_net_size(int r, uint32_t netset) {
    if (r <= 1) return 1;
    for (int m = r; m <= 8; ++m)
        if (m >= 3 && ((netset >> m) & 1u)) return m;
    return r <= 1 ? 1 : 2;  // r <= 2 with no larger network: one comparator
}

}  // namespace hs
