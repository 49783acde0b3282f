// Host side of the finite-game path: copying and validating the CSR tables
// (gamesolve_set_game / gamesolve_set_game_batch) and running the batched
// policy iteration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <tuple>

#include "games.cuh"
#include "solver.cuh"

namespace gs {

std::unique_ptr<Problem> build_game_problem(gs_solver* s, int count, int m1, int m2,
                                            const int64_t* state_offsets, const int64_t* row_ptr,
                                            const int32_t* col, const double* prob,
                                            const double* reward, const double* mu) {
    cudaStream_t st = s->st;
    std::vector<int64_t> off(count + 1);
    GS_CUDA(cudaMemcpy(off.data(), state_offsets, sizeof(int64_t) * (count + 1), cudaMemcpyDefault));
    if (off[0] != 0) {
        set_last_error("set_game: state offsets must start at 0");
        throw Error{GS_EINVAL};
    }
    int64_t max_n = 0;
    for (int g = 0; g < count; ++g) {
        const int64_t n = off[g + 1] - off[g];
        if (n < 1) {
            set_last_error("set_game: game %d has %lld states", g, (long long)n);
            throw Error{GS_EINVAL};
        }
        max_n = std::max(max_n, n);
    }
    const bool mixed = s->opt.precision != GS_PREC_FP64;
    const int64_t cap = mixed ? kGameMaxStatesMixed : kGameMaxStatesFP64;
    const bool grid = count == 1 && max_n >= kGameGridMinStates;
    if (!grid && max_n > cap) {
        set_last_error("set_game: a game has %lld states; this build takes at most %lld per game",
                       (long long)max_n, (long long)cap);
        throw Error{GS_EINVAL};
    }
    std::vector<double> mu_h(count);
    GS_CUDA(cudaMemcpy(mu_h.data(), mu, sizeof(double) * count, cudaMemcpyDefault));
    // mu = 1 (undiscounted, as the stopping games of Sec. 6.2-6.3) only for one
    // game on the algebraic multigrid path: the constant-vector correction
    // of the two-level method needs leakage on every row
    const bool undiscounted_ok = count == 1 && s->opt.game_solver == 1;
    for (double m : mu_h)
        if (!(m > 0.0 && (m < 1.0 || (m == 1.0 && undiscounted_ok)))) {
            set_last_error("set_game: mu must lie in (0, 1) (mu = 1 only with options.game_solver = 1)");
            throw Error{GS_EINVAL};
        }
    const int64_t n_total = off[count];
    const int64_t rows = n_total * m1 * m2;
    int64_t nnz_ends[2];
    GS_CUDA(cudaMemcpy(&nnz_ends[0], row_ptr, sizeof(int64_t), cudaMemcpyDefault));
    GS_CUDA(cudaMemcpy(&nnz_ends[1], row_ptr + rows, sizeof(int64_t), cudaMemcpyDefault));
    if (nnz_ends[0] != 0 || nnz_ends[1] < 0) {
        set_last_error("set_game: row_ptr must start at 0 and be non-decreasing");
        throw Error{GS_EINVAL};
    }
    const int64_t nnz = nnz_ends[1];

    size_t held = s->prob ? s->prob->arena.held() : 0;
    auto P = std::make_unique<Problem>(s->opt.mem_budget, held, s->st);
    P->kind = 2;
    auto G = std::make_unique<GameProblem>();
    G->count = count;
    G->m1 = m1;
    G->m2 = m2;
    G->n_total = n_total;
    G->rows = rows;
    G->nnz = nnz;
    G->max_n = (int)max_n;
    G->prob_bf16 = s->opt.precision == GS_PREC_MIXED_BF16;
    G->st_off_h = off;
    Arena& ar = P->arena;
    G->st_off = ar.alloc<int64_t>(count + 1);
    G->row_ptr = ar.alloc<int64_t>(rows + 1);
    G->col = ar.alloc<int32_t>(std::max<int64_t>(nnz, 1));
    G->prob = ar.alloc<double>(std::max<int64_t>(nnz, 1));
    G->prob32 = ar.alloc<float>(std::max<int64_t>(nnz, 1));
    G->rew = ar.alloc<double>(rows);
    G->leak = ar.alloc<double>(rows);
    G->leak32 = ar.alloc<float>(rows);
    G->mu = ar.alloc<double>(count);
    G->v = ar.alloc<double>(n_total);
    G->v32 = ar.alloc<float>(n_total);
    G->alpha = ar.alloc<uint8_t>(n_total);
    G->beta = ar.alloc<uint8_t>(n_total * m1);
    G->sel = ar.alloc<int64_t>(n_total);
    G->rhs = ar.alloc<double>(n_total);
    G->gstats = ar.alloc<int>(4 * (size_t)count);
    G->gres = ar.alloc<double>(count);
    G->queue = ar.alloc<int>(2);
    // largest games first, so that no large game starts as the batch drains;
    // the autotuning sample takes every k-th game of that order (the same mix)
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return off[a + 1] - off[a] > off[b + 1] - off[b];
    });
    const int stride = count >= kAutotuneMinGames ? count / kAutotuneSample : 1;
    std::vector<int> sample;
    for (int q = 0; q < count && (int)sample.size() < kAutotuneSample; q += stride)
        sample.push_back(order[q]);
    G->order = ar.alloc<int>(count);
    G->sample = ar.alloc<int>(sample.size());
    G->n_sample = (int)sample.size();
    if (grid) {
        G->grid = true;
        G->wr = ar.alloc<double>(n_total);
        G->we = ar.alloc<double>(n_total);
        G->wt = ar.alloc<double>(n_total);
        G->part = ar.alloc<double>(2 * 152 * 64);
        G->bar = ar.alloc<GridBarrier>(1);
    }
    GS_CUDA(cudaMemcpyAsync(G->st_off, off.data(), sizeof(int64_t) * (count + 1),
                            cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemcpyAsync(G->row_ptr, row_ptr, sizeof(int64_t) * (rows + 1), cudaMemcpyDefault, st));
    if (nnz) {
        GS_CUDA(cudaMemcpyAsync(G->col, col, sizeof(int32_t) * nnz, cudaMemcpyDefault, st));
        GS_CUDA(cudaMemcpyAsync(G->prob, prob, sizeof(double) * nnz, cudaMemcpyDefault, st));
    }
    GS_CUDA(cudaMemcpyAsync(G->rew, reward, sizeof(double) * rows, cudaMemcpyDefault, st));
    GS_CUDA(cudaMemcpyAsync(G->mu, mu_h.data(), sizeof(double) * count, cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemsetAsync(G->queue, 0, 2 * sizeof(int), st));
    GS_CUDA(cudaMemcpyAsync(G->order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemcpyAsync(G->sample, sample.data(), sizeof(int) * sample.size(),
                            cudaMemcpyHostToDevice, st));
    GameTables T = G->tables();
    launch_game_validate(T, count, G->st_off, rows, G->queue + 1, st);
    int bad = 0;
    GS_CUDA(cudaMemcpyAsync(&bad, G->queue + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    if (bad & 31) {
        set_last_error("set_game: invalid table (%s%s%s%s%s)", bad & 1 ? "row_ptr decreasing " : "",
                       bad & 2 ? "column out of range " : "", bad & 4 ? "probability outside [0,1] " : "",
                       bad & 8 ? "row sum above 1 " : "", bad & 16 ? "reward not finite" : "");
        throw Error{GS_EINVAL};
    }
    // rows of one length let the walks skip row_ptr (the validation flags any other)
    if (!(bad & 32) && rows > 0) {
        int64_t rp1 = 0;
        GS_CUDA(cudaMemcpy(&rp1, row_ptr + 1, sizeof(int64_t), cudaMemcpyDefault));
        G->k_uniform = rp1 > 0 ? rp1 : 0;
        T = G->tables();
        // each evaluation of the two-level path gathers its rows slot-major
        if (G->k_uniform > 0 && G->k_uniform <= 64 && s->opt.game_solver == 0) {
            const size_t m = (size_t)n_total * G->k_uniform;
            G->cp.col = ar.alloc<int32_t>(m);
            G->cp.p32 = ar.alloc<float>(m);
            G->cp.p64 = ar.alloc<double>(m);
            G->cp.leak32 = ar.alloc<float>(n_total);
            G->cp.leak64 = ar.alloc<double>(n_total);
            G->cp.K = (int)G->k_uniform;
        }
    }
    launch_game_prepare(T, count, G->st_off, rows, G->mu, G->leak, G->leak32,
                        G->prob_bf16 ? nullptr : G->prob32,
                        G->prob_bf16 ? (__nv_bfloat16*)G->prob32 : nullptr, st);
    GS_CUDA(cudaStreamSynchronize(st));
    P->game = std::move(G);
    return P;
}

namespace {

// Block-shape autotuner of the one-block batch kernel.  Games are latency
// bound, so the better shape (fewer threads per game and more games in flight,
// or the reverse) depends on the games' sizes, the precision and the shared
// memory each game takes.  The first solve of a large batch times every shape
// on a sample of it (every k-th game, largest first) and keeps the faster; the
// choice is cached per (precision, largest game rounded up to a power of two,
// actions, row length) for the process.
using ShapeKey = std::tuple<int, int, int, int, int64_t>;
std::mutex g_shape_mu;
std::map<ShapeKey, int> g_shapes;

int tuned_shape(gs_solver* s, GameProblem& G, const BatchArgs& B, bool mixed) {
    if (s->opt.game_threads > 0) return s->opt.game_threads;
    if (G.count < kAutotuneMinGames) return 512;
    int pow2 = 1;
    while (pow2 < G.max_n) pow2 <<= 1;
    const ShapeKey key{s->opt.precision, pow2, G.m1, G.m2, G.k_uniform};
    {
        std::lock_guard<std::mutex> lk(g_shape_mu);
        auto it = g_shapes.find(key);
        if (it != g_shapes.end()) return it->second;
    }
    cudaStream_t st = s->st;
    BatchArgs T = B;
    T.count = G.n_sample;
    T.order = G.sample;
    cudaEvent_t e0, e1;
    GS_CUDA(cudaEventCreate(&e0));
    GS_CUDA(cudaEventCreate(&e1));
    int best = 512;
    float best_ms = 0.0f;
    for (int shape : kBatchShapes) {
        GS_CUDA(cudaMemsetAsync(G.queue, 0, sizeof(int), st));
        GS_CUDA(cudaEventRecord(e0, st));
        launch_games_pi(T, mixed, shape, st);
        GS_CUDA(cudaEventRecord(e1, st));
        GS_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        GS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (best_ms == 0.0f || ms < best_ms) {
            best = shape;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(g_shape_mu);
    g_shapes[key] = best;
    return best;
}

}  // namespace

gs_status run_games(gs_solver* s, gs_solve_stats* stats) {
    GameProblem& G = *s->prob->game;
    cudaStream_t st = s->st;
    const bool mixed = s->opt.precision != GS_PREC_FP64;
    BatchArgs B{};
    B.T = G.tables();
    B.out = {G.v, G.v32, G.alpha, G.beta, G.sel, G.rhs, G.gstats, G.gres};
    B.opt.max_outer = s->opt.max_outer;
    B.opt.max_inner = s->opt.max_inner;
    B.opt.max_cycles = s->opt.max_cycles;
    B.opt.nu1 = s->opt.nu1;
    B.opt.nu2 = s->opt.nu2;
    B.opt.default_alpha = 0;
    B.opt.eps = s->opt.eps;
    B.opt.lin_tol = s->opt.lin_tol;
    B.opt.pi_rtol = s->opt.pi_rtol;
    B.count = G.count;
    B.max_n = G.max_n;
    B.st_off = G.st_off;
    B.mu = G.mu;
    B.queue = G.queue;
    B.order = G.order;
    B.cp = G.cp;
    const int shape = G.grid ? 0 : tuned_shape(s, G, B, mixed);
    G.shape = shape;
    cudaEvent_t e0, e1;
    GS_CUDA(cudaEventCreate(&e0));
    GS_CUDA(cudaEventCreate(&e1));
    GS_CUDA(cudaMemsetAsync(G.queue, 0, sizeof(int), st));
    if (G.grid) GS_CUDA(cudaMemsetAsync(G.bar, 0, sizeof(GridBarrier), st));
    GS_CUDA(cudaEventRecord(e0, st));
    if (G.grid) {
        GridWork W{G.wr, G.we, G.wt, G.part, G.bar, G.cp};
        const int blocks = std::min(game_grid_blocks(G.n_total, s->opt.grid_blocks), 152 * 64);
        launch_game_pi_grid(B, W, blocks, mixed, st);
    } else {
        launch_games_pi(B, mixed, shape, st);
    }
    GS_CUDA(cudaEventRecord(e1, st));
    G.stats_h.resize(4 * (size_t)G.count);
    G.res_h.resize(G.count);
    GS_CUDA(cudaMemcpyAsync(G.stats_h.data(), G.gstats, sizeof(int) * 4 * G.count,
                            cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaMemcpyAsync(G.res_h.data(), G.gres, sizeof(double) * G.count,
                            cudaMemcpyDeviceToHost, st));
    GridBarrier hb{};
    if (G.grid) GS_CUDA(cudaMemcpyAsync(&hb, G.bar, sizeof hb, cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    if (hb.error) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        set_last_error("game solve: a grid barrier wait timed out");
        return GS_ETIMEOUT;
    }
    float ms = 0;
    GS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int outer = 0, systems = 0, cycles = 0, conv = 1;
    double res = 0.0;
    for (int g = 0; g < G.count; ++g) {
        outer = std::max(outer, G.stats_h[4 * g]);
        systems += G.stats_h[4 * g + 1];
        cycles += G.stats_h[4 * g + 2];
        conv &= G.stats_h[4 * g + 3];
        res = std::max(res, G.res_h[g]);
    }
    reset_initial(s);
    if (stats) {
        stats->outer = outer;
        stats->systems = systems;
        stats->cycles = cycles;
        stats->levels = 2;
        stats->res_inf = res;
        stats->res_l2 = 0.0;
        stats->seconds = ms * 1e-3;
        stats->converged = conv;
        stats->fmg_levels = 0;
    }
    return conv ? GS_OK : GS_ENOTCONV;
}

}  // namespace gs
