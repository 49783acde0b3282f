// Bounded grid-wide barrier for cooperative launches (all blocks co-resident).
#pragma once

#include "common.cuh"

namespace gs {

// Barrier state in device memory (zeroed before a launch that uses it);
// `error` is set when a wait gives up.
struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    int error;
    int pad;
};

constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  One
// word counts arrivals: block 0 adds 2^31 - (nb - 1) and every other block
// adds 1, so the top bit flips exactly when the last block arrives and the low
// bits return to their value; waiters watch the top bit.  A wait gives up
// after kBarrierTimeoutNs and raises the error flag, which releases the others.
struct GridSync {
    GridBarrier* b;
    unsigned nb;
    unsigned long long limit_ns = kBarrierTimeoutNs;   // how long one wait may last
    __device__ bool sync() const {
        __shared__ int s_ok;
        __syncthreads();
        if (threadIdx.x == 0) {
            int ok = 1;
            const unsigned add = blockIdx.x == 0 ? 0x80000000u - (nb - 1) : 1u;
            volatile unsigned* word = &b->count;
            __threadfence();
            const unsigned old = atomicAdd(&b->count, add);
            if (((old ^ *word) & 0x80000000u) == 0) {
                const unsigned long long t0 = global_ns();
                while (((old ^ *word) & 0x80000000u) == 0) {
                    if (*(volatile int*)&b->error) { ok = 0; break; }
                    if (global_ns() - t0 > limit_ns) {
                        atomicExch(&b->error, 1);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
            s_ok = ok;
        }
        __syncthreads();
        return s_ok != 0;
    }
};

}  // namespace gs
