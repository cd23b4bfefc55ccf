// bt_sort.cuh -- block-wide bitonic sort of unique 32-bit keys held in
// registers (E keys per thread, NT threads, N = NT*E), used to put a work
// unit's candidate particles in ascending original-index order.
//
// Every comparator is ascending: merge step k first compares element i with
// its mirror i ^ (k-1) inside the k-block, then with i ^ j for j = k/4 .. 1.
// Pairs inside a thread use min/max on registers, pairs inside a warp one
// shuffle, pairs across warps go through shared memory.
#pragma once

#include <stdint.h>

namespace bt {

// Barrier over the NT threads that take part in the sort (threads 0..NT-1 of
// the block): __syncthreads when they are the whole block, else named
// barrier 1.
template <int NT>
__device__ __forceinline__ void sort_barrier()
{
    if (NT == 0) return;
    asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

template <int V>
struct Log2 { static constexpr int value = 1 + Log2<V / 2>::value; };
template <>
struct Log2<1> { static constexpr int value = 0; };

template <int V>
struct HighBit { static constexpr int value = 1 << Log2<V>::value; };

template <int NT, int E, int M>
__device__ __forceinline__ void bsort_stage(uint32_t (&v)[E], uint32_t *buf)
{
    constexpr int LE = Log2<E>::value;
    constexpr int MT = M >> LE;
    constexpr int MR = M & (E - 1);
    if constexpr (MT == 0) {
        constexpr int HB = HighBit<MR>::value;
#pragma unroll
        for (int r = 0; r < E; r++) {
            if ((r & HB) == 0) {
                const int r2 = r ^ MR;
                uint32_t a = v[r], b = v[r2];
                v[r] = min(a, b);
                v[r2] = max(a, b);
            }
        }
    } else {
        constexpr int HBT = HighBit<MT>::value;
        const bool upper = (threadIdx.x & HBT) != 0;
        uint32_t x[E];
        if constexpr (MT < 32) {
#pragma unroll
            for (int r = 0; r < E; r++) x[r] = __shfl_xor_sync(0xffffffffu, v[r ^ MR], MT);
        } else {
            sort_barrier<NT>();
#pragma unroll
            for (int r = 0; r < E; r++) buf[threadIdx.x * E + r] = v[r];
            sort_barrier<NT>();
            const int tp = threadIdx.x ^ MT;
#pragma unroll
            for (int r = 0; r < E; r++) x[r] = buf[tp * E + (r ^ MR)];
        }
#pragma unroll
        for (int r = 0; r < E; r++) v[r] = upper ? max(v[r], x[r]) : min(v[r], x[r]);
    }
}

template <int NT, int E, int J>
__device__ __forceinline__ void bsort_inner(uint32_t (&v)[E], uint32_t *buf)
{
    if constexpr (J >= 1) {
        bsort_stage<NT, E, J>(v, buf);
        bsort_inner<NT, E, J / 2>(v, buf);
    }
}

template <int NT, int E, int K>
__device__ __forceinline__ void bsort_outer(uint32_t (&v)[E], uint32_t *buf)
{
    if constexpr (K <= NT * E) {
        bsort_stage<NT, E, K - 1>(v, buf);   // mirror comparison
        bsort_inner<NT, E, K / 4>(v, buf);
        bsort_outer<NT, E, K * 2>(v, buf);
    }
}

// Sorts buf[0 .. NT*E) ascending in place.  Threads 0..NT-1 of the block
// must call it (others must not); it synchronises only them.
template <int NT, int E>
__device__ __forceinline__ void block_sort(uint32_t *buf)
{
    uint32_t v[E];
#pragma unroll
    for (int r = 0; r < E; r++) v[r] = buf[threadIdx.x * E + r];
    bsort_outer<NT, E, 2>(v, buf);
    sort_barrier<NT>();
#pragma unroll
    for (int r = 0; r < E; r++) buf[threadIdx.x * E + r] = v[r];
    sort_barrier<NT>();
}

}  // namespace bt
