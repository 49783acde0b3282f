// Host-side solver objects: device memory, multigrid hierarchies and the
// policy-iteration driver.
#pragma once

#include <memory>
#include <vector>

#include "amg.cuh"
#include "kernels.cuh"
#include "mgsolve.cuh"
#include "games.cuh"

namespace gs {

// All device allocations of one problem, counted against the memory budget.
// Allocations are stream-ordered (cudaMallocAsync / cudaFreeAsync on the
// owner's stream), so replacing a problem never synchronises the device.
class Arena {
public:
    Arena(size_t budget, size_t already_held, cudaStream_t st = nullptr)
        : budget_(budget), base_(already_held), st_(st) {}
    ~Arena();
    Arena(const Arena&) = delete;
    Arena& operator=(const Arena&) = delete;
    template <typename T>
    T* alloc(size_t count) {
        return static_cast<T*>(raw(count * sizeof(T)));
    }
    void* raw_bytes(size_t bytes) { return raw(bytes); }
    size_t held() const { return held_; }

private:
    void* raw(size_t bytes);
    size_t budget_, base_, held_ = 0;
    cudaStream_t st_;
    std::vector<void*> ptrs_;
};

// One multigrid level.  Level 0 of an Isaacs hierarchy is the implicit fine
// operator (policy codes); levels >= 1 hold explicit 9-point stencils.
struct Level {
    int side = 0;
    size_t n = 0;
    double* A64 = nullptr;     // [9][n], levels >= 1
    float* A32 = nullptr;      // [9][n]: row sum, then off-diagonals
    double* P64 = nullptr;     // interpolation from level+1: [8][(sc+1)^2]
    float* P32 = nullptr;
    double *u64 = nullptr, *f64 = nullptr, *r64 = nullptr;
    float *u32 = nullptr, *f32 = nullptr, *r32 = nullptr;
};

// An Isaacs grid with its policies, value and multigrid hierarchy.
struct IsaacsGrid {
    int side = 0, variant = 0;
    size_t n = 0;
    IsaacsConsts Kh{};
    IsaacsConsts* Kd = nullptr;
    double *r0 = nullptr, *v = nullptr, *rhs = nullptr, *fv = nullptr;
    uint8_t *alpha = nullptr, *code = nullptr, *beta4 = nullptr;
    uint32_t* beta = nullptr;
    std::vector<Level> lv;
    double* inv = nullptr;     // explicit inverse of the coarsest operator
    int* dstatus = nullptr;
    bool hier_valid = false;   // hierarchy built for (nearly) the current codes
    long long stale_rows = 0;  // rows whose code changed since the hierarchy was built
};

// One or more finite games (CSR tables) on the device.
struct GameProblem {
    int count = 0, m1 = 0, m2 = 0, max_n = 0;
    int64_t n_total = 0, rows = 0, nnz = 0;
    std::vector<int64_t> st_off_h;
    int64_t *st_off = nullptr, *row_ptr = nullptr, *sel = nullptr;
    int32_t* col = nullptr;
    double *prob = nullptr, *rew = nullptr, *leak = nullptr, *mu = nullptr, *v = nullptr,
           *rhs = nullptr, *gres = nullptr;
    float* prob32 = nullptr;   // rounded copy of prob: float32, or bfloat16 in its first half
    float* leak32 = nullptr;   // float32 copy of leak
    float* v32 = nullptr;      // float32 copy of v
    int64_t k_uniform = 0;     // every row has this many entries (0: not uniform)
    bool prob_bf16 = false;
    uint8_t *alpha = nullptr, *beta = nullptr;
    int *gstats = nullptr, *queue = nullptr;
    int* order = nullptr;                  // games largest first (the queue's order)
    int* sample = nullptr;                 // every k-th entry of order (shape autotuning)
    int n_sample = 0;
    int shape = 0;                         // threads per game of the last solve (0: grid)
    bool grid = false;                     // one large game on the whole grid
    double *wr = nullptr, *we = nullptr, *wt = nullptr, *part = nullptr;
    GridBarrier* bar = nullptr;
    Compact cp{};                          // grid: the selected rows slot-major (rows of one length)
    std::vector<int> stats_h;
    std::vector<double> res_h;
    // algebraic multigrid path (options.game_solver = 1): the current
    // hierarchy, small device scalars and the longest row of the tables
    std::unique_ptr<AmgHierarchy> amg;
    int* amg_scal = nullptr;               // [0] changed, [2..3] |F(v)-v| bits, [4..5] |v| bits
    int amg_row_max = 0;
    GameTables tables() const {
        return {m1,   m2, row_ptr, col, prob, prob_bf16 ? nullptr : prob32,
                prob_bf16 ? (const __nv_bfloat16*)prob32 : nullptr, rew, leak, leak32, k_uniform};
    }
};

// The two-sided stopping game on a line (Sec. 6.3) on the device.
struct LineProblem {
    int n = 0;
    double *c = nullptr, *psi1 = nullptr, *psi2 = nullptr;   // per state
    double v_left = 0, v_right = 0;
    double *v = nullptr, *res = nullptr;
    uint8_t *alpha = nullptr, *beta = nullptr;               // beta: 2 per state
    int* stats = nullptr;                                    // outer, systems, cycles, converged, grids
};

struct Problem {
    Problem(size_t budget, size_t held, cudaStream_t st) : arena(budget, held, st) {}
    Arena arena;
    int kind = 0;                                // 1 Isaacs, 2 finite games, 3 line game
    std::unique_ptr<GameProblem> game;
    std::unique_ptr<LineProblem> line;
    std::vector<std::unique_ptr<IsaacsGrid>> grids;   // FAMGpi levels, coarse to fine
    double* xi = nullptr;                        // finest-grid noise (when given)
};

struct Counters {
    int outer = 0, systems = 0, cycles = 0;
    double res_inf = 0, res_l2 = 0;
    bool converged = false;
    bool lin_capped = false;   // a linear solve stopped at max_cycles
    double last_lin_res = 0;
};

// Why a multigrid linear solve stopped (SolveOut::reason).
enum { kLinExact = 1, kLinInexact = 2, kLinCapped = 3 };

}  // namespace gs

namespace gs {
// Device state of one multigrid solve launch (barrier and results).
struct MGState {
    GridBarrier bar;
    SolveOut out;
};

// CUDA-event brackets around the launches of one kernel class.
struct Tracer {
    int cls = 0;
    std::vector<cudaEvent_t> ev;   // pairs: start, stop
    size_t used = 0;               // events recorded since the last harvest
    double ms = 0.0;
    long long launches = 0;
};
}  // namespace gs

struct gs_solver {
    gs_options opt;
    gs::Tracer trace;
    cudaStream_t st = nullptr;
    gs::DevScalars* dsc = nullptr;     // device scalars
    gs::DevScalars* hsc = nullptr;     // pinned host mirror
    gs::MGState* mgd = nullptr;        // multigrid launch state (device)
    gs::MGState* mgh = nullptr;        // pinned host mirror
    std::unique_ptr<gs::Problem> prob;
    bool init_v = false, init_alpha = false, init_beta = false;
    int last_levels = 0;
    std::vector<int> level_stats;      // per FAMGpi level of the last solve: side, outer, systems
};

namespace gs {

IsaacsConsts make_isaacs_consts(int side, int variant, int mu_mode);
std::unique_ptr<Problem> build_isaacs_problem(gs_solver* s, int side, int variant, uint64_t seed,
                                              const double* xi);
void reset_initial(gs_solver* s);
std::unique_ptr<Problem> build_game_problem(gs_solver* s, int count, int m1, int m2,
                                            const int64_t* state_offsets, const int64_t* row_ptr,
                                            const int32_t* col, const double* prob,
                                            const double* reward, const double* mu);
gs_status run_games(gs_solver* s, gs_solve_stats* stats);
gs_status run_game_amg(gs_solver* s, gs_solve_stats* stats);
std::unique_ptr<Problem> build_line_problem(gs_solver* s, int32_t n, const double* c,
                                            const double* psi1, const double* psi2, double v_left,
                                            double v_right);
gs_status run_line(gs_solver* s, gs_solve_stats* stats);
gs_status run_solve(gs_solver* s, gs_solve_stats* stats);
gs_status run_improve(gs_solver* s, const double* v, uint8_t* alpha_out, uint8_t* beta_out,
                      double* fv_out);
gs_status run_fmg_interpolate(int side_c, int variant, const double* v_c, const uint8_t* alpha_c,
                              const uint8_t* beta_c, double* v_f, uint8_t* alpha_f,
                              uint8_t* beta_f, cudaStream_t st);
gs_status run_policy_solve(gs_solver* s, const uint8_t* alpha, const uint8_t* beta,
                           const double* w0, double* w_out, gs_solve_stats* stats);
// Multigrid solve of the assembled policy-fixed system of g to the float64
// floor (fresh hierarchy); g.v holds the initial guess and receives w.
// Returns false when max_cycles was reached before the floor.
bool solve_policy_system(gs_solver* s, IsaacsGrid& g, int* cycles, double* res);
void launch_pack_beta(const uint8_t* src, int m1, size_t n, uint32_t* beta, uint8_t* beta4,
                      cudaStream_t st);
void launch_check_actions(const uint8_t* a, size_t n, int limit, int* bad, cudaStream_t st);
void trace_harvest(gs_solver* s);
unsigned long long launch_count();
void trace_reset(gs_solver* s, int cls);
void pack_beta_upload(gs_solver* s, IsaacsGrid& g, const uint8_t* beta_host);
void unpack_beta_download(gs_solver* s, const IsaacsGrid& g, uint8_t* beta_out);

}  // namespace gs
