// Random finite discounted games drawn on the device from a counter-based
// stream: the synthetic workload family of the serving and batch benchmarks
// (games of Sec. 2 with n states, m1 x m2 action pairs and k successors per
// row).  Row rho uses outputs rho*17 .. rho*17+16 of the SplitMix64 stream
// `seed`: outputs 0..k-1 pick k distinct successors uniformly (without
// replacement, by rank adjustment past the earlier picks), outputs 8..8+k-1
// give Exp(1) draws that are normalised to Dirichlet(1) probabilities (the
// last one set to one minus the others), output 16 the reward U(-1, 1).
// Within a row the successors are stored in increasing column order.
#include <cuda_runtime.h>

#include "common.cuh"
#include "games.cuh"

namespace gs {

namespace {

constexpr int kRowDraws = 17;
constexpr int kMaxSucc = 8;

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output i of the stream `seed`,
// and the double in [0, 1) from its top 53 bits.
__device__ __forceinline__ uint64_t sm64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double unit(uint64_t seed, uint64_t i) {
    return (double)(sm64(seed, i) >> 11) * 0x1.0p-53;
}

__global__ void k_random_game(int64_t rows, int64_t n, int k, uint64_t seed, int64_t nnz_base,
                              int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                              double* __restrict__ prob, double* __restrict__ reward) {
    for (int64_t rho = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; rho < rows;
         rho += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t base = (uint64_t)rho * kRowDraws;
        int64_t pick[kMaxSucc], sorted[kMaxSucc];
        double p[kMaxSucc];
        for (int t = 0; t < k; ++t) {
            const double u = unit(seed, base + t);
            int64_t idx = (int64_t)(u * (double)(n - t));
            if (idx > n - t - 1) idx = n - t - 1;
            // the rank among the n - t states not picked yet: step past each
            // earlier pick in ascending order
            for (int s = 0; s < t; ++s) idx += idx >= sorted[s] ? 1 : 0;
            pick[t] = idx;
            int s = t;   // insert into the ascending list
            while (s > 0 && sorted[s - 1] > idx) {
                sorted[s] = sorted[s - 1];
                --s;
            }
            sorted[s] = idx;
        }
        for (int t = 0; t < k; ++t) p[t] = -log1p(-unit(seed, base + 8 + t));
        // the sum of the k draws: pairwise for k = 8, left to right otherwise
        double tot;
        if (k == kMaxSucc) {
            tot = ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
        } else {
            tot = 0.0;
            for (int t = 0; t < k; ++t) tot += p[t];
        }
        for (int t = 0; t < k; ++t) p[t] /= tot;
        if (k > 1) {
            double head = 0.0;
            for (int t = 0; t < k - 1; ++t) head += p[t];
            p[k - 1] = fmax(1.0 - head, 0.0);
        } else {
            p[0] = 1.0;
        }
        reward[rho] = unit(seed, base + 16) * 2.0 - 1.0;
        // columns ascending, each with its probability
        for (int j = 0; j < k; ++j) {
            int t = 0;
            while (pick[t] != sorted[j]) ++t;
            col[rho * k + j] = (int32_t)sorted[j];
            prob[rho * k + j] = p[t];
        }
        row_ptr[rho] = nnz_base + rho * k;
        if (rho == rows - 1) row_ptr[rows] = nnz_base + rows * k;
    }
}

}  // namespace

bool random_game_args_ok(int64_t n, int32_t m1, int32_t m2, int32_t k) {
    return n >= 1 && n < (int64_t)1 << 31 && m1 >= 1 && m1 <= kGameMaxM1 && m2 >= 1 && m2 <= kGameMaxM2 &&
           k >= 1 && k <= kMaxSucc && k <= n;
}

void launch_random_game(int64_t n, int32_t m1, int32_t m2, int32_t k, uint64_t seed, int64_t* row_ptr,
                        int32_t* col, double* prob, double* reward, cudaStream_t st, int64_t nnz_base) {
    const int64_t rows = n * m1 * m2;
    const int threads = 256;
    const int64_t want = (rows + threads - 1) / threads;
    const int blocks = (int)(want < 152 * 64 ? want : 152 * 64);
    k_random_game<<<blocks, threads, 0, st>>>(rows, n, k, seed, nnz_base, row_ptr, col, prob, reward);
    GS_CHECK_LAUNCH();
}

}  // namespace gs
