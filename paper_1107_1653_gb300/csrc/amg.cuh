// Algebraic multigrid for the policy-fixed systems of a finite game given by
// CSR tables (Sec. 4.3): strength of connection, C/F splitting, direct
// interpolation, Galerkin coarse operators R A P with R = P^T, and V-cycles
// with C/F relaxation, all on the device.  Host side: the hierarchy's memory
// and the order of the set-up kernels.
#pragma once

#include <memory>
#include <vector>

#include "games.cuh"

namespace gs {

constexpr int kAmgMaxLevels = 24;
constexpr int kAmgCoarsest = 128;       // the coarsest level is solved by its inverse
constexpr int kAmgInvSmem = 64;         // inverted in shared memory up to this size
constexpr int kAmgRowCap = 96;          // entries of a coarse row the set-up accumulates
constexpr int kAmgCoarseSweeps = 30;    // Jacobi sweeps on a coarsest level too large to invert
constexpr int kAmgMaxColours = 128;     // colours of the Gauss-Seidel smoother's colouring
constexpr int kAmgTailN = 2048;         // levels this small run in one thread block, with
                                        // block barriers instead of grid barriers

// One level of the hierarchy, rows in ELL form (slot 0 holds the diagonal;
// unused slots have column -1 and value 0).
struct AmgLevelArgs {
    int n;
    int W;                  // ELL width of A
    const int* col;         // [n][W]
    const double* a64;      // [n][W]
    const float* a32;       // [n][W]
    int WP;                 // ELL width of P (interpolation from level + 1)
    const int* pcol;        // [n][WP] columns in level + 1
    const double* p64;
    const float* p32;
    int WR;                 // ELL width of R = P^T (rows of level + 1 over this level's points)
    const int* rcol;        // [n_{l+1}][WR]
    const double* r64;
    const float* r32;
    const int8_t* cf;       // 1 C point, 2 F point (this level's splitting)
    const int* ord;         // the points ordered by class: C points by colour, then F points
    const int* kofs;        // class k (C: colour k, F: ncolour + colour k) is ord[kofs[k], kofs[k+1])
    int ncolour;
    unsigned long long cmaskC[2], cmaskF[2];   // colours that hold C (F) points
    void* u;                // V-cycle unknown (float32 in the mixed path, else float64)
    void* f;                // V-cycle right-hand side
    void* t;                // relaxation's second buffer
};

struct AmgOut {
    unsigned long long rmax[2], vmax[2];
    int cycles, reason;
    double res, vmax_final;
};

struct AmgSolveArgs {
    int nlev;               // levels; nlev - 1 is the coarsest
    int nu1, nu2, max_cycles, mixed;
    double lin_tol, rel_tol;
    const double* rhs;      // fine right-hand side (float64)
    double* v;              // fine iterate (float64)
    const double* inv;      // inverse of the coarsest operator (n_L <= kAmgCoarsest)
    int coarse_sweeps;      // > 0: the coarsest level is relaxed this many times instead
    int tail;               // levels tail .. nlev - 1 are cycled by thread block 0 alone
                            // (nlev: none)
    GridBarrier* bar;
    AmgOut* out;
    AmgLevelArgs L[kAmgMaxLevels];
};

// Device memory of one hierarchy (rebuilt for every policy-fixed system).
struct AmgLevelMem {
    int n = 0, W = 0, WP = 0, WR = 0;
    int* col = nullptr;
    double* a64 = nullptr;
    float* a32 = nullptr;
    int* pcol = nullptr;
    double* p64 = nullptr;
    float* p32 = nullptr;
    int* rcol = nullptr;
    double* r64 = nullptr;
    float* r32 = nullptr;
    int8_t* cf = nullptr;
    int16_t* colour = nullptr;
    int* ord = nullptr;
    int* kofs = nullptr;
    int ncolour = 0;
    unsigned long long cmaskC[2] = {0, 0}, cmaskF[2] = {0, 0};
    void *u = nullptr, *f = nullptr, *t = nullptr;
};

class Arena;

// A hierarchy for one policy-fixed system, built on the device.
struct AmgHierarchy {
    std::unique_ptr<Arena> ar;          // all of its device memory
    std::vector<AmgLevelMem> lv;
    double* inv = nullptr;              // inverse of the coarsest operator
    int coarse_n = 0;
    int coarse_sweeps = 0;              // > 0: coarsest relaxed, not inverted
    AmgHierarchy();
    ~AmgHierarchy();
    // Set-up for the rows sel[0..n) of the tables (W0 >= 1 + the longest row).
    void build(const GameTables& T, const int64_t* sel, double mu, int n, int W0,
               const gs_options& opt, cudaStream_t st);
    // V-cycles on A v = rhs from v until the float64 floor, rel_tol drop or
    // max_cycles; returns the stop reason (1 floor/tolerance, 2 drop, 3 cap).
    int solve(double* v, const double* rhs, const gs_options& opt, double rel_tol,
              GridBarrier* bar_state, AmgOut* dout, AmgOut* hout, int* cycles, double* res,
              double* vmax, cudaStream_t st);
    static AmgLevelArgs args_of(const AmgLevelMem& m);
    template <class Read>
    void colour_level(AmgLevelMem& F, int* flag, int* scal, int* hs, Read&& read_scal, unsigned g,
                      cudaStream_t st);
};

}  // namespace gs
