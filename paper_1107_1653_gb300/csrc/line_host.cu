// Host side of the two-sided stopping game on a line (Sec. 6.3).
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "line.cuh"
#include "solver.cuh"

namespace gs {

std::unique_ptr<Problem> build_line_problem(gs_solver* s, int32_t n, const double* c,
                                            const double* psi1, const double* psi2, double v_left,
                                            double v_right) {
    if (n < 1 || n > kLineMaxStates || ((n + 1) & n) != 0) {
        set_last_error("set_stopping_line: n must be 2^k - 1 and at most %d", kLineMaxStates);
        throw Error{GS_EINVAL};
    }
    if (!c || !psi1 || !psi2 || !(std::fabs(v_left) <= DBL_MAX) || !(std::fabs(v_right) <= DBL_MAX)) {
        set_last_error("set_stopping_line: missing array or end value not finite");
        throw Error{GS_EINVAL};
    }
    std::vector<double> h_c(n), h_p1(n), h_p2(n);
    GS_CUDA(cudaMemcpy(h_c.data(), c, sizeof(double) * n, cudaMemcpyDefault));
    GS_CUDA(cudaMemcpy(h_p1.data(), psi1, sizeof(double) * n, cudaMemcpyDefault));
    GS_CUDA(cudaMemcpy(h_p2.data(), psi2, sizeof(double) * n, cudaMemcpyDefault));
    for (int i = 0; i < n; ++i)
        if (!(std::fabs(h_c[i]) <= DBL_MAX) || !(h_p1[i] <= h_p2[i]) || !(std::fabs(h_p1[i]) <= DBL_MAX) ||
            !(std::fabs(h_p2[i]) <= DBL_MAX)) {
            set_last_error("set_stopping_line: state %d needs finite c and psi1 <= psi2", i);
            throw Error{GS_EINVAL};
        }
    size_t held = s->prob ? s->prob->arena.held() : 0;
    auto P = std::make_unique<Problem>(s->opt.mem_budget, held, s->st);
    P->kind = 3;
    auto L = std::make_unique<LineProblem>();
    Arena& ar = P->arena;
    L->n = n;
    L->c = ar.alloc<double>(n);
    L->psi1 = ar.alloc<double>(n);
    L->psi2 = ar.alloc<double>(n);
    L->v = ar.alloc<double>(n);
    L->res = ar.alloc<double>(1);
    L->alpha = ar.alloc<uint8_t>(n);
    L->beta = ar.alloc<uint8_t>(2 * (size_t)n);
    L->stats = ar.alloc<int>(5);
    L->v_left = v_left;
    L->v_right = v_right;
    GS_CUDA(cudaMemcpyAsync(L->c, h_c.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
    GS_CUDA(cudaMemcpyAsync(L->psi1, h_p1.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
    GS_CUDA(cudaMemcpyAsync(L->psi2, h_p2.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s->st));
    GS_CUDA(cudaStreamSynchronize(s->st));
    P->line = std::move(L);
    return P;
}

gs_status run_line(gs_solver* s, gs_solve_stats* stats) {
    LineProblem& L = *s->prob->line;
    LineArgs A{};
    A.n = L.n;
    A.c = L.c;
    A.psi1 = L.psi1;
    A.psi2 = L.psi2;
    A.v_left = L.v_left;
    A.v_right = L.v_right;
    A.eps = s->opt.eps;
    A.fmg_c = s->opt.fmg_c;
    A.fmg = s->opt.fmg;
    A.max_outer = s->opt.max_outer;
    A.max_inner = s->opt.max_inner;
    A.max_cycles = s->opt.max_cycles;
    A.nu1 = s->opt.nu1;
    A.nu2 = s->opt.nu2;
    A.v_out = L.v;
    A.alpha_out = L.alpha;
    A.beta_out = L.beta;
    A.stats = L.stats;
    A.res_out = L.res;
    cudaEvent_t e0, e1;
    GS_CUDA(cudaEventCreate(&e0));
    GS_CUDA(cudaEventCreate(&e1));
    GS_CUDA(cudaEventRecord(e0, s->st));
    launch_line_pi(A, s->st);
    GS_CUDA(cudaEventRecord(e1, s->st));
    int st[5];
    double res;
    GS_CUDA(cudaMemcpyAsync(st, L.stats, sizeof st, cudaMemcpyDeviceToHost, s->st));
    GS_CUDA(cudaMemcpyAsync(&res, L.res, sizeof res, cudaMemcpyDeviceToHost, s->st));
    GS_CUDA(cudaStreamSynchronize(s->st));
    float ms = 0;
    GS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    GS_CUDA(cudaEventDestroy(e0));
    GS_CUDA(cudaEventDestroy(e1));
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->outer = st[0];
        stats->systems = st[1];
        stats->cycles = st[2];
        stats->converged = st[3];
        stats->fmg_levels = s->opt.fmg ? st[4] : 0;
        stats->levels = 1;
        for (int m = L.n; m > 3; m = (m - 1) / 2) ++stats->levels;
        stats->res_inf = res;
        stats->res_l2 = 0.0;
        stats->seconds = ms * 1e-3;
    }
    return st[3] ? GS_OK : GS_ENOTCONV;
}

}  // namespace gs
