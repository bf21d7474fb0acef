// grouped.cuh -- work distribution of the grouped (batched) kernels.
//
// A grouped launch runs one step of the residual for every system of a batch.
// Its table holds one entry per system; entry e owns the work items
// [first(e), first(e + 1)).  Worker w (a warp or a block) of nw takes the
// contiguous range [w per, min(total, (w + 1) per)), per = ceil(total / nw),
// so its items belong to one entry, or to a few neighbouring ones: the entry is
// found once by binary search over the entries' first items and then stepped
// forward, and the entry's descriptor stays in L1 across the worker's items.
// (A grid-stride walk puts a worker's consecutive items in different systems,
// and each item then pays a binary search and its descriptor loads from L2.)
#pragma once
#include <cstdint>

#include "kernels.h"

namespace ccb {

template <typename E> __device__ __forceinline__ int64_t first_item(const E &e) { return e.item0; }
__device__ __forceinline__ int64_t first_item(const GroupedSplit &e) { return e.tile0; }

template <typename E> struct EntryWalk {
    const E *tab;
    int n, cur;
    int64_t next;                      // first item of entry cur + 1
    __device__ __forceinline__ EntryWalk(const E *t, int n_, int64_t it) : tab(t), n(n_) {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first_item(tab[mid]) <= it) lo = mid;
            else hi = mid - 1;
        }
        cur = lo;
        next = cur + 1 < n ? first_item(tab[cur + 1]) : INT64_MAX;
    }
    // the entry of item it; it never decreases from one call to the next
    __device__ __forceinline__ int at(int64_t it) {
        while (it >= next) {
            cur++;
            next = cur + 1 < n ? first_item(tab[cur + 1]) : INT64_MAX;
        }
        return cur;
    }
};

struct WorkRange {
    int64_t begin, end;
};
__device__ __forceinline__ WorkRange work_range(int64_t total, int64_t w, int64_t nw) {
    const int64_t per = (total + nw - 1) / nw;
    const int64_t b = w * per;
    return {b < total ? b : total, b + per < total ? b + per : total};
}

}  // namespace ccb
