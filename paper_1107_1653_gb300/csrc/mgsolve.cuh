// Persistent multigrid solve of one policy-fixed system (Eq. (LSPI)): the
// arguments the host passes to the single cooperative kernel that runs the
// Galerkin set-up, the V-cycles (Algorithm 3) and the float64 stopping test.
#pragma once

#include "gridsync.cuh"

namespace gs {

constexpr int kMaxLevels = 14;
constexpr int kMGThreads = 256;
// Largest shared-memory footprint of the tail levels staged by block 0.
constexpr int kTailSmemMax = 100 * 1024;

// Plain data (no initialisers): copies live in shared memory.
struct LevelArgs {
    int side;            // grid side of the level
    int sc;              // side of the next coarser level, (side - 1) / 2
    size_t n;
    void* u;             // V-cycle unknown (float32 in the mixed path, else float64)
    void* f;             // V-cycle right-hand side
    const void* A;       // V-cycle operator, levels >= 1 (float32/bfloat16 leakage or float64)
    const void* P;       // V-cycle interpolation weights from level + 1
    double* A64;         // Galerkin operator, levels >= 1 (written by the set-up)
    float* A32;          // its rounded leakage copy (mixed path: float32, or bfloat16 in
                         // the first half of the same buffer)
    double* P64;         // interpolation weights (written by the set-up)
    float* P32;          // their rounded copy (float32, or bfloat16 likewise)
    void* u2;            // tiled cycles: u after the post-smoothing (levels >= 1)
};


struct SolveOut {
    unsigned long long rmax[2];   // |b - A v|_inf per residual evaluation (bits), ping-pong
    unsigned long long vmax[2];   // |v|_inf (bits)
    int cycles;
    int reason;                   // 1 tolerance or float64 floor, 2 relative drop, 3 cycle cap
    double res;                   // final |b - A v|_inf
    double vmax_final;            // |v|_inf at the final residual evaluation
};

struct SolveArgs {
    const IsaacsConsts* K;
    const uint8_t* code;
    double* v;
    const double* rhs;
    int nlev;        // levels; nlev - 1 is the coarsest (explicit inverse)
    int tail;        // levels >= tail are relaxed by thread block 0 alone
    int smem_from;   // levels >= smem_from (>= max(tail, 1)) live in block 0's shared memory
    int nu1, nu2, max_cycles;
    int nu1c, nu2c;  // sweeps on the coarse levels (l >= 1)
    int gamma;       // coarse visits per level visit: 1 V-cycle, 2 W-cycle
    int mixed;       // float32 V-cycles on the float64 residual (iterative refinement)
    int wbf16;       // mixed path with bfloat16 storage of the V-cycle operators and weights
    int do_setup;    // build interpolation, Galerkin operators and coarse inverse first
    int max_blocks;  // cap on the grid (0 = whole GPU)
    double lin_tol;
    double rel_tol;  // also stop once the residual fell by this factor (0: floor only)
    int tiled;       // V-cycles with tiled grid-wide levels (k_mg_cycles_tiled)
    int tile_from;   // tiled cycles: coarse levels l >= tile_from are tiled, larger ones
                     // (1 <= l < tile_from) take one grid-wide phase per colour
    int tc[kMaxLevels];   // tile side of level l >= 1, in points of level l + 1
    double* inv;     // inverse of the coarsest operator (n_L x n_L)
    int* inv_status;
    GridBarrier* bar;
    SolveOut* out;
    LevelArgs L[kMaxLevels];
};

// Cooperative launches on `st` (asynchronous): the Galerkin set-up, then the
// V-cycles with the stopping test.  bar and out must be zeroed on the stream
// before the first of them.
void launch_mg_setup(const SolveArgs& a, cudaStream_t st);
void launch_mg_cycles(const SolveArgs& a, cudaStream_t st);

// Shared memory the tail levels >= a.smem_from need.
size_t tail_smem_bytes(const SolveArgs& a);

// Largest dynamic shared memory a tiled cycle launch may take, and what one
// needs (the tail's and the largest tile's, whichever is more).
constexpr int kTiledSmemMax = 110 * 1024;
// Largest coarse level side the tiled kernel tiles: a 1023 x 1023 coarse level
// (the 2047 x 2047 grid's first) measured faster one phase per colour; in
// float64 (tiles of at most 8 x 8 next-level points: shared memory) already a
// 511 x 511 one (1023^2 float64 solve 19.8 -> 17.7 ms).
constexpr int kTiledMaxSide = 511;
constexpr int kTiledMaxSideF64 = 255;
size_t tiled_smem_bytes(const SolveArgs& a);

// Tile sides of a tiled launch for `workers` tile-taking thread blocks.
void set_tile_sides(SolveArgs& a, int workers);

}  // namespace gs
