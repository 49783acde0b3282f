// Two-sided stopping game on a line (Sec. 6.3): device-side argument block.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace gs {

constexpr int kLineThreads = 1024;
constexpr int kLineMaxLevels = 12;
constexpr int kLineMaxStates = 2047;   // the block's shared memory holds the hierarchy

struct LineArgs {
    int n;                                  // interior points, 2^k - 1
    const double *c, *psi1, *psi2;          // per state, device
    double v_left, v_right;                 // end values
    double eps, fmg_c;
    int fmg, max_outer, max_inner, max_cycles, nu1, nu2;
    double* v_out;
    uint8_t* alpha_out;
    uint8_t* beta_out;                      // 2 per state
    int* stats;                             // outer, systems, cycles, converged, grids
    double* res_out;                        // |F(v) - v|_inf at the end
};

size_t line_smem_bytes(int n);
void launch_line_pi(const LineArgs& A, cudaStream_t st);

}  // namespace gs
