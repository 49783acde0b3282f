// C ABI entry points (include/gamesolve.h): argument checks, error mapping,
// and dispatch to the host orchestrator.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "solver.cuh"

namespace gs {

static thread_local char g_last_error[512] = "";

void set_last_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
}

template <typename F>
static gs_status guarded(F&& f) {
    try {
        return f();
    } catch (const Error& e) {
        return e.st;
    } catch (...) {
        set_last_error("unexpected host exception");
        return GS_ECUDA;
    }
}

// Memory freed back to the device's stream-ordered pool stays there for the
// next problem instead of returning to the driver at every synchronisation.
static void keep_pool_memory(int dev) {
    static std::once_flag once[64];
    if (dev < 0 || dev >= 64) return;
    std::call_once(once[dev], [dev]() {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    });
}

static bool is_pow2m1(int side) {
    return side >= 1 && ((side + 1) & side) == 0;
}

}  // namespace gs

using namespace gs;

extern "C" {

void gamesolve_default_options(gs_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = GS_PREC_FP64;
    o->eps = 0.0;
    o->max_outer = 1000;
    o->max_inner = 1000;
    o->nu1 = 1;
    o->nu2 = 1;
    o->max_cycles = 200;
    o->lin_tol = 1e-15;
    o->coarse_max = 9;
    o->tail_side = 31;
    o->fmg = 0;
    o->fmg_side = 31;
    o->fmg_c = 0.1;
    o->mu_mode = 0;
    o->mem_budget = 0;
    o->stream = nullptr;
    o->pi_rtol = 1e-2;
    o->setup_reuse = 1e-2;
    o->cycle_gamma = 1;
    o->nu1_coarse = -1;
    o->nu2_coarse = -1;
    o->game_threads = 0;
    o->cycle_kernel = 0;
    o->game_solver = 0;
    o->amg_coarsening = 0;
    o->amg_theta = 0.0;
}

gs_status gamesolve_create(gs_solver** out, const gs_options* opt) {
    if (!out) {
        set_last_error("create: out is NULL");
        return GS_EINVAL;
    }
    *out = nullptr;
    gs_options o;
    if (opt) o = *opt;
    else gamesolve_default_options(&o);
    if (o.precision < GS_PREC_FP64 || o.precision > GS_PREC_MIXED_BF16 || o.max_outer < 1 || o.max_inner < 1 || o.nu1 < 0 ||
        o.nu2 < 0 || o.nu1 + o.nu2 < 1 || o.max_cycles < 1 || !(o.lin_tol >= 0) ||
        o.coarse_max < 1 || o.coarse_max > 64 || o.tail_side < 0 || !(o.eps >= 0) || !(o.fmg_c > 0) ||
        (o.fmg && !is_pow2m1(o.fmg_side)) || o.mu_mode < 0 || o.mu_mode > 1 ||
        !(o.pi_rtol >= 0.0 && o.pi_rtol < 1.0) || !(o.setup_reuse >= 0.0 && o.setup_reuse <= 1.0) ||
        o.grid_blocks < 0 || o.cycle_gamma < 0 || o.cycle_gamma > 2 || o.nu1_coarse < -1 ||
        o.nu2_coarse < -1 ||
        (o.game_threads != 0 && o.game_threads != 256 && o.game_threads != 512) ||
        o.cycle_kernel < 0 || o.cycle_kernel > 1 || o.game_solver < 0 || o.game_solver > 1 ||
        o.amg_coarsening < 0 || o.amg_coarsening > 1 || !(o.amg_theta >= 0.0 && o.amg_theta < 1.0) ||
        (o.nu1_coarse < 0 ? o.nu1 : o.nu1_coarse) + (o.nu2_coarse < 0 ? o.nu2 : o.nu2_coarse) < 1) {
        set_last_error("create: invalid option value");
        return GS_EINVAL;
    }
    return guarded([&]() -> gs_status {
        int dev = 0;
        GS_CUDA(cudaGetDevice(&dev));
        keep_pool_memory(dev);
        auto* s = new gs_solver();
        s->opt = o;
        s->st = (cudaStream_t)o.stream;
        cudaError_t e1 = cudaMalloc(&s->dsc, sizeof(DevScalars));
        cudaError_t e2 = cudaMallocHost(&s->hsc, sizeof(DevScalars));
        cudaError_t e3 = cudaMalloc(&s->mgd, sizeof(MGState));
        cudaError_t e4 = cudaMallocHost(&s->mgh, sizeof(MGState));
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess) {
            cudaError_t e = e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3 != cudaSuccess ? e3 : e4;
            set_last_error("create: %s", cudaGetErrorString(e));
            if (s->dsc) cudaFree(s->dsc);
            if (s->hsc) cudaFreeHost(s->hsc);
            if (s->mgd) cudaFree(s->mgd);
            if (s->mgh) cudaFreeHost(s->mgh);
            delete s;
            cudaGetLastError();
            return GS_ECUDA;
        }
        *out = s;
        return GS_OK;
    });
}

gs_status gamesolve_set_game(gs_solver* s, int64_t n, int32_t m1, int32_t m2,
                             const int64_t* row_ptr, const int32_t* col, const double* prob,
                             const double* reward, double mu) {
    if (!s || n < 1 || m1 < 1 || m1 > kGameMaxM1 || m2 < 1 || m2 > kGameMaxM2 || !row_ptr || !col || !prob ||
        !reward || !(mu > 0.0 && (mu < 1.0 || (mu == 1.0 && s->opt.game_solver == 1)))) {
        set_last_error("set_game: invalid argument");
        return GS_EINVAL;
    }
    return guarded([&]() -> gs_status {
        const int64_t off[2] = {0, n};
        auto P = build_game_problem(s, 1, m1, m2, off, row_ptr, col, prob, reward, &mu);
        s->prob = std::move(P);
        reset_initial(s);
        return GS_OK;
    });
}

gs_status gamesolve_set_stopping_line(gs_solver* s, int32_t n, const double* c,
                                      const double* psi1, const double* psi2, double v_left,
                                      double v_right) {
    if (!s) return GS_EINVAL;
    return guarded([&]() -> gs_status {
        auto P = build_line_problem(s, n, c, psi1, psi2, v_left, v_right);
        s->prob = std::move(P);
        reset_initial(s);
        return GS_OK;
    });
}

gs_status gamesolve_set_game_batch(gs_solver* s, int32_t count, int32_t m1, int32_t m2,
                                   const int64_t* state_offsets, const int64_t* row_ptr,
                                   const int32_t* col, const double* prob, const double* reward,
                                   const double* mu) {
    if (!s || count < 1 || m1 < 1 || m1 > kGameMaxM1 || m2 < 1 || m2 > kGameMaxM2 || !state_offsets || !row_ptr ||
        !col || !prob || !reward || !mu) {
        set_last_error("set_game_batch: invalid argument");
        return GS_EINVAL;
    }
    return guarded([&]() -> gs_status {
        auto P = build_game_problem(s, count, m1, m2, state_offsets, row_ptr, col, prob, reward, mu);
        s->prob = std::move(P);
        reset_initial(s);
        return GS_OK;
    });
}

namespace {
// Device memory of the current device, or managed memory.
bool on_device(const void* p) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (at.type != cudaMemoryTypeDevice || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.device == dev;
}
}  // namespace

gs_status gamesolve_random_game(int64_t n, int32_t m1, int32_t m2, int32_t k, uint64_t seed,
                                int64_t* row_ptr, int32_t* col, double* prob, double* reward,
                                void* stream) {
    if (!random_game_args_ok(n, m1, m2, k) || !row_ptr || !col || !prob || !reward) {
        set_last_error("random_game: invalid argument");
        return GS_EINVAL;
    }
    if (!on_device(row_ptr) || !on_device(col) || !on_device(prob) || !on_device(reward)) {
        set_last_error("random_game: the table buffers must be device memory");
        return GS_EINVAL;
    }
    return guarded([&]() -> gs_status {
        launch_random_game(n, m1, m2, k, seed, row_ptr, col, prob, reward, (cudaStream_t)stream);
        return GS_OK;
    });
}

gs_status gamesolve_set_random_game(gs_solver* s, int64_t n, int32_t m1, int32_t m2, int32_t k,
                                    uint64_t seed, double mu) {
    if (!s || !random_game_args_ok(n, m1, m2, k) || !(mu > 0.0 && mu < 1.0)) {
        set_last_error("set_random_game: invalid argument");
        return GS_EINVAL;
    }
    return guarded([&]() -> gs_status {
        // drawn into scratch buffers on the solver's stream, then set as a
        // table given in device memory (copied into the problem)
        const int64_t rows = n * m1 * m2, nnz = rows * k;
        int64_t* rp = nullptr;
        int32_t* col = nullptr;
        double *prob = nullptr, *rew = nullptr;
        auto release = [&]() {
            cudaStreamSynchronize(s->st);
            cudaFree(rp);
            cudaFree(col);
            cudaFree(prob);
            cudaFree(rew);
        };
        try {
            GS_CUDA(cudaMalloc(&rp, sizeof(int64_t) * (rows + 1)));
            GS_CUDA(cudaMalloc(&col, sizeof(int32_t) * nnz));
            GS_CUDA(cudaMalloc(&prob, sizeof(double) * nnz));
            GS_CUDA(cudaMalloc(&rew, sizeof(double) * rows));
            launch_random_game(n, m1, m2, k, seed, rp, col, prob, rew, s->st);
            GS_CUDA(cudaStreamSynchronize(s->st));
            const int64_t off[2] = {0, n};
            auto P = build_game_problem(s, 1, m1, m2, off, rp, col, prob, rew, &mu);
            s->prob = std::move(P);
            reset_initial(s);
        } catch (...) {
            release();
            throw;
        }
        release();
        return GS_OK;
    });
}

gs_status gamesolve_get_batch_stats(const gs_solver* s, int32_t* stats, double* res) {
    if (!s) return GS_EINVAL;
    if (!s->prob || s->prob->kind != 2) {
        set_last_error("get_batch_stats: no game batch set");
        return GS_ESTATE;
    }
    const GameProblem& G = *s->prob->game;
    if (G.stats_h.empty()) {
        set_last_error("get_batch_stats: not solved yet");
        return GS_ESTATE;
    }
    if (stats) std::memcpy(stats, G.stats_h.data(), sizeof(int32_t) * 4 * G.count);
    if (res) std::memcpy(res, G.res_h.data(), sizeof(double) * G.count);
    return GS_OK;
}

gs_status gamesolve_get_batch_shape(const gs_solver* s, int32_t* threads) {
    if (!s || !threads) return GS_EINVAL;
    if (!s->prob || s->prob->kind != 2 || s->prob->game->stats_h.empty()) {
        set_last_error("get_batch_shape: no solved game batch held");
        return GS_ESTATE;
    }
    *threads = s->prob->game->shape;
    return GS_OK;
}

gs_status gamesolve_set_isaacs_grid(gs_solver* s, int32_t side, int32_t variant, uint64_t seed,
                                    const double* xi) {
    if (!s || !is_pow2m1(side) || side > kIsaacsMaxSide || (variant != 0 && variant != 1)) {
        set_last_error("set_isaacs_grid: side must be 2^k - 1 <= 16383 and variant 0 or 1");
        return GS_EINVAL;
    }
    if (s->opt.fmg && side < s->opt.fmg_side) {
        set_last_error("set_isaacs_grid: side below the FAMGpi coarsest side");
        return GS_EINVAL;
    }
    return guarded([&]() -> gs_status {
        auto P = build_isaacs_problem(s, side, variant, seed, xi);
        s->prob = std::move(P);
        reset_initial(s);
        return GS_OK;
    });
}

gs_status gamesolve_set_initial(gs_solver* s, const double* v0, const uint8_t* alpha0,
                                const uint8_t* beta0) {
    if (!s) return GS_EINVAL;
    if (!s->prob) {
        set_last_error("set_initial: no problem set");
        return GS_ESTATE;
    }
    if (s->prob->kind != 1) {
        set_last_error("set_initial: warm starts are for Isaacs grids in this build");
        return GS_EINVAL;
    }
    return guarded([&]() -> gs_status {
        IsaacsGrid& g = *s->prob->grids.back();
        const int m1 = g.variant == 1 ? 5 : 4;
        if (alpha0 || beta0) {
            // validate on the host side copy
            std::vector<uint8_t> a(alpha0 ? g.n : 0), b(beta0 ? g.n * m1 : 0);
            if (alpha0) GS_CUDA(cudaMemcpy(a.data(), alpha0, g.n, cudaMemcpyDefault));
            if (beta0) GS_CUDA(cudaMemcpy(b.data(), beta0, g.n * m1, cudaMemcpyDefault));
            for (uint8_t x : a)
                if (x >= m1) { set_last_error("set_initial: alpha out of range"); return GS_EINVAL; }
            for (uint8_t x : b)
                if (x >= 4) { set_last_error("set_initial: beta out of range"); return GS_EINVAL; }
        }
        if (v0) {
            GS_CUDA(cudaMemcpyAsync(g.v, v0, g.n * sizeof(double), cudaMemcpyDefault, s->st));
            s->init_v = true;
        }
        if (alpha0) {
            GS_CUDA(cudaMemcpyAsync(g.alpha, alpha0, g.n, cudaMemcpyDefault, s->st));
            s->init_alpha = true;
        }
        if (beta0) {
            pack_beta_upload(s, g, beta0);
            s->init_beta = true;
        }
        GS_CUDA(cudaStreamSynchronize(s->st));
        return GS_OK;
    });
}

gs_status gamesolve_solve(gs_solver* s, gs_solve_stats* stats) {
    if (!s) return GS_EINVAL;
    if (!s->prob) {
        set_last_error("solve: no problem set");
        return GS_ESTATE;
    }
    if (s->prob->kind == 2) {
        if (s->opt.game_solver == 1 && s->prob->game->count == 1)
            return guarded([&]() { return run_game_amg(s, stats); });
        return guarded([&]() { return run_games(s, stats); });
    }
    if (s->prob->kind == 3) return guarded([&]() { return run_line(s, stats); });
    return guarded([&]() { return run_solve(s, stats); });
}

gs_status gamesolve_get_value(const gs_solver* s, double* v_out, int64_t n) {
    if (!s || !v_out) return GS_EINVAL;
    if (!s->prob) return GS_ESTATE;
    const int kind = s->prob->kind;
    const size_t total = kind == 2   ? (size_t)s->prob->game->n_total
                         : kind == 3 ? (size_t)s->prob->line->n
                                     : s->prob->grids.back()->n;
    const double* src = kind == 2   ? s->prob->game->v
                        : kind == 3 ? s->prob->line->v
                                    : s->prob->grids.back()->v;
    if (n != (int64_t)total) {
        set_last_error("get_value: n = %lld, problem has %zu states", (long long)n, total);
        return GS_EINVAL;
    }
    return guarded([&]() -> gs_status {
        GS_CUDA(cudaMemcpyAsync(v_out, src, total * sizeof(double), cudaMemcpyDefault, s->st));
        GS_CUDA(cudaStreamSynchronize(s->st));
        return GS_OK;
    });
}

gs_status gamesolve_get_policy(const gs_solver* s, uint8_t* alpha, uint8_t* beta) {
    if (!s) return GS_EINVAL;
    if (!s->prob) return GS_ESTATE;
    gs_solver* sm = const_cast<gs_solver*>(s);
    if (s->prob->kind == 3) {
        const LineProblem& L = *s->prob->line;
        return guarded([&]() -> gs_status {
            if (alpha) GS_CUDA(cudaMemcpyAsync(alpha, L.alpha, L.n, cudaMemcpyDefault, s->st));
            if (beta) GS_CUDA(cudaMemcpyAsync(beta, L.beta, 2 * (size_t)L.n, cudaMemcpyDefault, s->st));
            GS_CUDA(cudaStreamSynchronize(s->st));
            return GS_OK;
        });
    }
    if (s->prob->kind == 2) {
        const GameProblem& G = *s->prob->game;
        return guarded([&]() -> gs_status {
            if (alpha) GS_CUDA(cudaMemcpyAsync(alpha, G.alpha, G.n_total, cudaMemcpyDefault, s->st));
            if (beta)
                GS_CUDA(cudaMemcpyAsync(beta, G.beta, G.n_total * G.m1, cudaMemcpyDefault, s->st));
            GS_CUDA(cudaStreamSynchronize(s->st));
            return GS_OK;
        });
    }
    return guarded([&]() -> gs_status {
        const IsaacsGrid& g = *s->prob->grids.back();
        if (alpha) GS_CUDA(cudaMemcpyAsync(alpha, g.alpha, g.n, cudaMemcpyDefault, s->st));
        if (beta) unpack_beta_download(sm, g, beta);
        GS_CUDA(cudaStreamSynchronize(s->st));
        return GS_OK;
    });
}

gs_status gamesolve_improve(gs_solver* s, const double* v, uint8_t* alpha_out, uint8_t* beta_out,
                            double* fv_out) {
    if (!s || !v) return GS_EINVAL;
    if (!s->prob) return GS_ESTATE;
    if (s->prob->kind != 1) {
        set_last_error("improve: available for Isaacs grids in this build");
        return GS_EINVAL;
    }
    return guarded([&]() { return run_improve(s, v, alpha_out, beta_out, fv_out); });
}

gs_status gamesolve_policy_solve(gs_solver* s, const uint8_t* alpha, const uint8_t* beta,
                                 const double* w0, double* w_out, gs_solve_stats* stats) {
    if (!s || !alpha || !beta || !w_out) return GS_EINVAL;
    if (!s->prob) return GS_ESTATE;
    if (s->prob->kind != 1) {
        set_last_error("policy_solve: available for Isaacs grids in this build");
        return GS_EINVAL;
    }
    return guarded([&]() { return run_policy_solve(s, alpha, beta, w0, w_out, stats); });
}

gs_status gamesolve_fmg_interpolate(int32_t side_c, int32_t variant, const double* v_c,
                                    const uint8_t* alpha_c, const uint8_t* beta_c, double* v_f,
                                    uint8_t* alpha_f, uint8_t* beta_f, void* stream) {
    if (side_c < 1 || side_c > 8191 || (variant != 0 && variant != 1) || !v_c || !alpha_c ||
        !beta_c) {
        set_last_error("fmg_interpolate: invalid argument");
        return GS_EINVAL;
    }
    return guarded([&]() {
        return run_fmg_interpolate(side_c, variant, v_c, alpha_c, beta_c, v_f, alpha_f, beta_f,
                                   (cudaStream_t)stream);
    });
}

gs_status gamesolve_get_level_stats(const gs_solver* s, int32_t* stats, int32_t cap,
                                    int32_t* levels) {
    if (!s || cap < 0 || (cap > 0 && !stats)) return GS_EINVAL;
    if (!s->prob || (s->prob->kind != 1 && s->prob->kind != 2) || s->level_stats.empty()) {
        set_last_error("get_level_stats: no solved Isaacs grid or single game");
        return GS_ESTATE;
    }
    const int nl = (int)s->level_stats.size() / 3;
    if (levels) *levels = nl;
    for (int k = 0; k < nl && k < cap; ++k)
        for (int j = 0; j < 3; ++j) stats[3 * k + j] = s->level_stats[3 * k + j];
    return GS_OK;
}

gs_status gamesolve_trace(gs_solver* s, int32_t kernel_class) {
    if (!s || kernel_class < GS_K_NONE || kernel_class > GS_K_MG_CYCLES) return GS_EINVAL;
    return guarded([&]() -> gs_status {
        trace_reset(s, kernel_class);
        return GS_OK;
    });
}

gs_status gamesolve_trace_read(gs_solver* s, double* total_ms, int64_t* launches) {
    if (!s) return GS_EINVAL;
    return guarded([&]() -> gs_status {
        trace_harvest(s);
        if (total_ms) *total_ms = s->trace.ms;
        if (launches) *launches = s->trace.launches;
        return GS_OK;
    });
}

uint64_t gamesolve_kernel_launches(void) { return launch_count(); }

void gamesolve_destroy(gs_solver* s) {
    if (!s) return;
    for (cudaEvent_t e : s->trace.ev) cudaEventDestroy(e);
    if (s->st) cudaStreamSynchronize(s->st);
    else cudaDeviceSynchronize();
    s->prob.reset();
    if (s->dsc) cudaFree(s->dsc);
    if (s->hsc) cudaFreeHost(s->hsc);
    if (s->mgd) cudaFree(s->mgd);
    if (s->mgh) cudaFreeHost(s->mgh);
    delete s;
}

const char* gamesolve_strerror(gs_status st) {
    switch (st) {
    case GS_OK: return "ok";
    case GS_EINVAL: return "invalid argument";
    case GS_ENOMEM: return "out of device memory or over the memory budget";
    case GS_ENOTCONV: return "iteration caps reached before convergence";
    case GS_ETIMEOUT: return "a bounded device-side wait timed out";
    case GS_ECUDA: return "CUDA error";
    case GS_ESTATE: return "call out of order";
    }
    return "unknown status";
}

const char* gamesolve_last_error(void) { return g_last_error; }

}  // extern "C"
