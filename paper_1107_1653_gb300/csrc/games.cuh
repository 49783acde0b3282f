// Finite games given by CSR transition tables: device-side argument blocks.
#pragma once

#include <cuda_bf16.h>

#include "gridsync.cuh"

namespace gs {

// Concatenated CSR tables of one or more games.  Rows of game g are
// (x * m1 + a) * m2 + b for its states x, numbered after the earlier games'
// rows; columns are state indices within the game.
struct GameTables {
    int m1, m2;
    const int64_t* row_ptr;   // total rows + 1 (global nnz offsets)
    const int32_t* col;
    const double* prob;
    const float* prob32;      // float32 copy (relaxation; null with bfloat16 storage)
    const __nv_bfloat16* prob16;   // bfloat16 copy (relaxation; null unless chosen)
    const double* rew;        // per row
    const double* leak;       // per row: 1 - mu sum_k p_k
    const float* leak32;      // the same rounded to float32 (relaxation)
    int64_t k_uniform;        // > 0: every row has exactly this many entries (row_ptr unused
                              // by the walks); 0: general CSR
};

// Entries [k0, k1) of a row.
__device__ __forceinline__ void row_range(const GameTables& T, int64_t row, int64_t* k0, int64_t* k1) {
    if (T.k_uniform > 0) {
        *k0 = row * T.k_uniform;
        *k1 = *k0 + T.k_uniform;
    } else {
        *k0 = T.row_ptr[row];
        *k1 = T.row_ptr[row + 1];
    }
}

struct BatchOut {
    double* v;        // per state (global numbering): value, also the iterate
    float* v32;       // its float32 rounding, kept beside it (screened improvement)
    uint8_t* alpha;   // per state
    uint8_t* beta;    // per state x m1
    int64_t* sel;     // per state: the selected row of the policy-fixed system
    double* rhs;      // per state: its reward r^{alpha beta}
    int* gstats;      // per game: outer, systems, cycles, converged
    double* gres;     // per game: |F(v) - v|_inf at the end
};

struct BatchOpts {
    int max_outer, max_inner, max_cycles, nu1, nu2, default_alpha;
    double eps, lin_tol, pi_rtol;
};

// The selected rows of a game's policy-fixed system gathered slot-major
// (entry k of state i at [k * n + i], n the game's states) at the start of
// each evaluation, so that the cycles read them coalesced and without the
// selection's indirection.  Only for rows of one length K (col null: not used).
struct Compact {
    int32_t* col;
    float* p32;          // the relaxation's copy (float32, or bfloat16 widened)
    double* p64;
    float* leak32;
    double* leak64;
    int K;
};

struct BatchArgs {
    GameTables T;
    BatchOut out;
    BatchOpts opt;
    int count;              // games
    int max_n;              // largest game (sizes the shared-memory vectors)
    const int64_t* st_off;  // count + 1 state offsets
    const double* mu;       // per game
    int* queue;             // work counter (zeroed before the launch)
    const int* order;       // queue position -> game, `count` entries (one-block kernel)
    Compact cp;             // one-block kernel: slot-major rows of all games, game g's at
                            // state offset st_off[g] (cp.col null: rows read in place)
};

// Work vectors of the grid-wide single-game kernel (global memory).
struct GridWork {
    void *r, *e, *t;     // n elements each (float32 or float64)
    double* part;        // 2 x (blocks) per-block partials
    GridBarrier* bar;    // zeroed before the launch
    Compact cp;          // the selected rows, slot-major (cp.col null: rows read in place)
};

// Action counts: MAX at most kGameMaxM1, MIN at most kGameMaxM2 (policies are
// bytes).  Games with at most kScreenMaxM1 MAX actions take the float32-screened
// improvement, larger ones the float64 decisions directly.
constexpr int kGameMaxM1 = 64;
constexpr int kGameMaxM2 = 255;
constexpr int kScreenMaxM1 = 8;

// Largest game the one-block-per-game kernel takes (its three correction
// vectors live in shared memory).
constexpr int kGameMaxStatesMixed = 16384;
constexpr int kGameMaxStatesFP64 = 8192;

void launch_game_validate(const GameTables& T, int count, const int64_t* st_off, int64_t rows,
                          int* bad, cudaStream_t st);
// Writes the leakage per row and the rounded copy of p (float32 into prob32, or
// bfloat16 into prob16: exactly one of them is non-null).
void launch_game_prepare(const GameTables& T, int count, const int64_t* st_off, int64_t rows,
                         const double* mu, double* leak, float* leak32, float* prob32,
                         __nv_bfloat16* prob16, cudaStream_t st);
size_t games_smem_bytes(int max_n, bool mixed);
// Threads per game of the one-block kernel's instantiations.
constexpr int kBatchShapes[2] = {256, 512};
// Batches of at least this many games autotune the shape on a sample of this many.
constexpr int kAutotuneMinGames = 1024;
constexpr int kAutotuneSample = 608;
void launch_games_pi(const BatchArgs& B, bool mixed, int threads, cudaStream_t st);
// Thread blocks for the grid-wide kernel on a game of n states (cap > 0 limits them).
int game_grid_blocks(int64_t n, int cap);
void launch_game_pi_grid(const BatchArgs& B, const GridWork& W, int blocks, bool mixed,
                         cudaStream_t st);

// One policy improvement of a single game (game 0 of B) over the whole grid:
// mode 0 outer (alpha and beta), 1 inner (beta at alpha), 2 MIN's reply for
// every a; assembles sel/rhs.  scal[0] += changed entries, scal + 2 (bits) =
// max |F(v) - v| (outer); the tie tolerance comes from |v|_inf at scal + 4.
void launch_game_improve_one(const BatchArgs& B, int mode, int64_t n, int* scal, cudaStream_t st);

// Games of at least this many states, set alone, run on the whole grid.
constexpr int64_t kGameGridMinStates = 4096;

// Random games drawn on the device (randgame.cu): n states, m1 x m2 rows per
// state, k <= 8 successors per row; CSR table into device buffers of
// n*m1*m2 + 1, n*m1*m2*k, n*m1*m2*k and n*m1*m2 entries, row_ptr offset by
// nnz_base (a game placed after others in a batch's concatenated table).
bool random_game_args_ok(int64_t n, int32_t m1, int32_t m2, int32_t k);
void launch_random_game(int64_t n, int32_t m1, int32_t m2, int32_t k, uint64_t seed, int64_t* row_ptr,
                        int32_t* col, double* prob, double* reward, cudaStream_t st, int64_t nnz_base = 0);

}  // namespace gs
