// Policy iteration with algebraic multigrid (AMGpi, Sec. 5.1) and the full
// multilevel scheme FAMGpi (Algorithm 4, Sec. 5.2): host orchestration of the
// kernels on the solver's stream.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

#include "solver.cuh"

namespace gs {

// ------------------------------------------------------------------ memory
Arena::~Arena() {
    for (void* p : ptrs_) cudaFree(p);
}

void* Arena::raw(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (budget_ && base_ + held_ + bytes > budget_) {
        set_last_error("device memory budget exceeded: %zu + %zu > %zu bytes", base_ + held_, bytes,
                       budget_);
        throw Error{GS_ENOMEM};
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_last_error("cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
        throw Error{e == cudaErrorMemoryAllocation ? GS_ENOMEM : GS_ECUDA};
    }
    ptrs_.push_back(p);
    held_ += bytes;
    return p;
}

// ------------------------------------------------------------------ tracing
static std::atomic<unsigned long long> g_launches{0};
void note_launches(int k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(); }

namespace {

// Brackets the launches issued in its scope with events when `cls` is traced.
class KScope {
public:
    KScope(gs_solver* s, int cls) : s_(s), on_(s->trace.cls == cls && cls != 0) {
        if (on_) record();
    }
    ~KScope() {
        if (on_) {
            record();
            ++s_->trace.launches;
        }
    }

private:
    void record() {
        Tracer& t = s_->trace;
        if (t.used == t.ev.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) { on_ = false; return; }
            t.ev.push_back(e);
        }
        cudaEventRecord(t.ev[t.used++], s_->st);
    }
    gs_solver* s_;
    bool on_;
};

}  // namespace

void trace_harvest(gs_solver* s) {
    Tracer& t = s->trace;
    if (!t.used) return;
    GS_CUDA(cudaStreamSynchronize(s->st));
    for (size_t k = 0; k + 1 < t.used; k += 2) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, t.ev[k], t.ev[k + 1]) == cudaSuccess) t.ms += ms;
    }
    t.used = 0;
}

void trace_reset(gs_solver* s, int cls) {
    trace_harvest(s);
    s->trace.cls = cls;
    s->trace.ms = 0;
    s->trace.launches = 0;
}

namespace {

__global__ void k_pack_beta(const uint8_t* __restrict__ src, int m1, size_t n,
                            uint32_t* __restrict__ beta, uint8_t* __restrict__ beta4) {
    size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const uint8_t* s = src + x * m1;
    beta[x] = (uint32_t)s[0] | ((uint32_t)s[1] << 8) | ((uint32_t)s[2] << 16) | ((uint32_t)s[3] << 24);
    if (m1 == 5) beta4[x] = s[4];
}

__global__ void k_unpack_beta(const uint32_t* __restrict__ beta, const uint8_t* __restrict__ beta4,
                              int m1, size_t n, uint8_t* __restrict__ dst) {
    size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    uint32_t b = beta[x];
    uint8_t* d = dst + x * m1;
    d[0] = b & 0xff;
    d[1] = (b >> 8) & 0xff;
    d[2] = (b >> 16) & 0xff;
    d[3] = (b >> 24) & 0xff;
    if (m1 == 5) d[4] = beta4[x];
}

__global__ void k_fill_u8(uint8_t* p, size_t n, uint8_t val) {
    size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) p[x] = val;
}

__global__ void k_check_actions(const uint8_t* a, size_t n, int limit, int* bad) {
    size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n && a[x] >= limit) atomicAdd(bad, 1);
}

void sync(gs_solver* s) { GS_CUDA(cudaStreamSynchronize(s->st)); }

void clear_scalars(gs_solver* s) { GS_CUDA(cudaMemsetAsync(s->dsc, 0, sizeof(DevScalars), s->st)); }

const DevScalars& read_scalars(gs_solver* s) {
    GS_CUDA(cudaMemcpyAsync(s->hsc, s->dsc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s->st));
    sync(s);
    return *s->hsc;
}

}  // namespace

// ------------------------------------------------------------------ set-up
IsaacsConsts make_isaacs_consts(int side, int variant, int mu_mode) {
    IsaacsConsts K{};
    K.side = side;
    K.variant = variant;
    const double h = 1.0 / (side + 1);
    const double c0 = 2.0 + h;
    K.h = h;
    if (mu_mode == 1) {
        K.mu = c0 / (c0 + h * h);
        K.kappa = (h * h) / (c0 + h * h);
    } else {
        K.mu = 1.0 / (1.0 + h * h);
        K.kappa = (h * h) / (1.0 + h * h);
    }
    static const int E[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};   // +x1, -x1, +x2, -x2
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            const double b1 = 0.5 * (E[a][0] - E[b][0]), b2 = 0.5 * (E[a][1] - E[b][1]);
            double* p = K.p[4 * a + b];
            p[0] = (0.5 + h * std::max(b1, 0.0)) / c0;    // +x1 (E)
            p[1] = (0.5 + h * std::max(-b1, 0.0)) / c0;   // -x1 (W)
            p[2] = (0.5 + h * std::max(b2, 0.0)) / c0;    // +x2 (N)
            p[3] = (0.5 + h * std::max(-b2, 0.0)) / c0;   // -x2 (S)
            p[4] = a == b ? h / c0 : 0.0;                 // self
            double* am = K.am[4 * a + b];
            am[0] = 1.0 - K.mu * p[4];
            am[1] = -(K.mu * p[1]);
            am[2] = -(K.mu * p[0]);
            am[3] = -(K.mu * p[3]);
            am[4] = -(K.mu * p[2]);
            K.dr[a][b] = K.kappa * (0.1 * (a - b));
        }
    K.am[kStopCode][0] = 1.0;
    for (int c = 0; c < kCodes; ++c)
        for (int d = 0; d < 5; ++d) K.amf[c][d] = (float)K.am[c][d];
    return K;
}

static void alloc_grid(gs_solver* s, Arena& ar, IsaacsGrid& g) {
    const size_t n = g.n;
    g.Kd = ar.alloc<IsaacsConsts>(1);
    GS_CUDA(cudaMemcpyAsync(g.Kd, &g.Kh, sizeof(IsaacsConsts), cudaMemcpyHostToDevice, s->st));
    g.r0 = ar.alloc<double>(n);
    g.v = ar.alloc<double>(n);
    g.rhs = ar.alloc<double>(n);
    g.fv = ar.alloc<double>(n);
    g.alpha = ar.alloc<uint8_t>(n);
    g.code = ar.alloc<uint8_t>(n);
    g.beta = ar.alloc<uint32_t>(n);
    g.beta4 = ar.alloc<uint8_t>(n);
    g.dstatus = ar.alloc<int>(4);
    // multigrid levels
    const int coarse_max = std::max(1, std::min<int>(s->opt.coarse_max, 64));
    int side = g.side;
    g.lv.clear();
    while (true) {
        Level L;
        L.side = side;
        L.n = (size_t)side * side;
        g.lv.push_back(L);
        if ((int)L.n <= coarse_max || side < 3) break;
        side = (side - 1) / 2;
    }
    for (size_t l = 0; l < g.lv.size(); ++l) {
        Level& L = g.lv[l];
        if (l > 0) {
            L.A64 = ar.alloc<double>(9 * L.n);
            L.A32 = ar.alloc<float>(9 * L.n);
            L.u64 = ar.alloc<double>(L.n);
            L.f64 = ar.alloc<double>(L.n);
        }
        L.r64 = ar.alloc<double>(L.n);
        L.u32 = ar.alloc<float>(L.n);
        L.f32 = ar.alloc<float>(L.n);
        L.r32 = ar.alloc<float>(L.n);
        if (l + 1 < g.lv.size()) {
            const size_t sc = (size_t)(L.side - 1) / 2;
            L.P64 = ar.alloc<double>(8 * (sc + 1) * (sc + 1));
            L.P32 = ar.alloc<float>(8 * (sc + 1) * (sc + 1));
        }
    }
    const int nL = (int)g.lv.back().n;
    g.inv = ar.alloc<double>((size_t)nL * nL);
}

std::unique_ptr<Problem> build_isaacs_problem(gs_solver* s, int side, int variant, uint64_t seed,
                                              const double* xi) {
    size_t held = s->prob ? s->prob->arena.held() : 0;
    auto P = std::make_unique<Problem>(s->opt.mem_budget, held);
    P->kind = 1;
    std::vector<int> sides{side};
    if (s->opt.fmg) {
        while (sides.back() > s->opt.fmg_side) sides.push_back((sides.back() - 1) / 2);
        std::reverse(sides.begin(), sides.end());
    }
    if (xi) {
        P->xi = P->arena.alloc<double>((size_t)side * side);
        GS_CUDA(cudaMemcpyAsync(P->xi, xi, sizeof(double) * side * side, cudaMemcpyDefault, s->st));
    }
    for (int sd : sides) {
        auto g = std::make_unique<IsaacsGrid>();
        g->side = sd;
        g->variant = variant;
        g->n = (size_t)sd * sd;
        g->Kh = make_isaacs_consts(sd, variant, s->opt.mu_mode);
        alloc_grid(s, P->arena, *g);
        NoiseSrc ns{P->xi, seed, side, (side + 1) / (sd + 1)};
        launch_isaacs_r0(g->Kd, sd, g->Kh.kappa, ns, g->r0, s->st);
        P->grids.push_back(std::move(g));
    }
    sync(s);
    return P;
}

void reset_initial(gs_solver* s) { s->init_v = s->init_alpha = s->init_beta = false; }

void pack_beta_upload(gs_solver* s, IsaacsGrid& g, const uint8_t* beta_host) {
    const int m1 = g.variant == 1 ? 5 : 4;
    if (m1 == 4) {
        GS_CUDA(cudaMemcpyAsync(g.beta, beta_host, g.n * 4, cudaMemcpyDefault, s->st));
        return;
    }
    uint8_t* stage = reinterpret_cast<uint8_t*>(g.fv);   // n doubles >= 5 n bytes
    GS_CUDA(cudaMemcpyAsync(stage, beta_host, g.n * m1, cudaMemcpyDefault, s->st));
    k_pack_beta<<<div_up(g.n, 256), 256, 0, s->st>>>(stage, m1, g.n, g.beta, g.beta4);
    GS_CHECK_LAUNCH();
}

void unpack_beta_download(gs_solver* s, const IsaacsGrid& g, uint8_t* beta_out) {
    const int m1 = g.variant == 1 ? 5 : 4;
    if (m1 == 4) {
        GS_CUDA(cudaMemcpyAsync(beta_out, g.beta, g.n * 4, cudaMemcpyDefault, s->st));
        return;
    }
    uint8_t* stage = reinterpret_cast<uint8_t*>(g.fv);
    k_unpack_beta<<<div_up(g.n, 256), 256, 0, s->st>>>(g.beta, g.beta4, m1, g.n, stage);
    GS_CHECK_LAUNCH();
    GS_CUDA(cudaMemcpyAsync(beta_out, stage, g.n * m1, cudaMemcpyDefault, s->st));
}

// ------------------------------------------------------------------ multigrid
namespace {

// Galerkin hierarchy for the current policy codes of grid g: interpolation
// weights and A^{l+1} = P^T A^l P on every level, float32 copies for the mixed
// path, and the explicit inverse of the coarsest operator (float64).
void setup_hierarchy(gs_solver* s, IsaacsGrid& g, bool need32) {
    cudaStream_t st = s->st;
    const int L = (int)g.lv.size() - 1;
    KScope ks(s, GS_K_SETUP);
    if (L == 0) {
        launch_l0_coarse_invert(g.Kd, g.side, g.code, g.inv, g.dstatus, st);
        return;
    }
    launch_l0_interp(g.Kd, g.side, g.code, g.lv[0].P64, g.lv[0].P32, st);
    launch_l0_rap(g.Kd, g.side, g.code, g.lv[0].P64, g.lv[1].A64, st);
    for (int l = 1; l < L; ++l) {
        launch_interp9(g.lv[l].A64, g.lv[l].side, g.lv[l].P64, g.lv[l].P32, st);
        launch_rap9(g.lv[l].A64, g.lv[l].side, g.lv[l].P64, g.lv[l + 1].A64, st);
    }
    if (need32)
        for (int l = 1; l <= L; ++l) launch_stencil_to32(g.lv[l].A64, g.lv[l].n, g.lv[l].A32, st);
    launch_coarse_invert9(g.lv[L].A64, g.lv[L].side, g.inv, g.dstatus, st);
}

template <typename T>
struct Vec {
    T *u, *f, *r;
};

template <typename T>
Vec<T> level_vec(IsaacsGrid& g, int l);
template <>
Vec<double> level_vec<double>(IsaacsGrid& g, int l) {
    if (l == 0) return {g.v, g.rhs, g.lv[0].r64};
    return {g.lv[l].u64, g.lv[l].f64, g.lv[l].r64};
}
template <>
Vec<float> level_vec<float>(IsaacsGrid& g, int l) {
    return {g.lv[l].u32, g.lv[l].f32, g.lv[l].r32};
}

template <typename T>
void smooth(gs_solver* s, IsaacsGrid& g, int l, bool from_zero) {
    Vec<T> V = level_vec<T>(g, l);
    const Level& L = g.lv[l];
    if (l == 0) {
        for (int c = 0; c < 2; ++c) {
            KScope ks(s, GS_K_FINE_RELAX);
            if constexpr (sizeof(T) == 8)
                launch_l0_smooth64(g.Kd, L.side, g.code, V.f, V.u, c, s->st);
            else
                launch_l0_smooth32(g.Kd, L.side, g.code, V.f, V.u, c, from_zero && c == 0, s->st);
        }
    } else {
        const void* A = sizeof(T) == 8 ? (const void*)L.A64 : (const void*)L.A32;
        for (int ph = 0; ph < 4; ++ph) {
            KScope ks(s, GS_K_COARSE);
            launch_smooth9<T>(A, L.side, V.f, V.u, ph, from_zero && ph == 0, s->st);
        }
    }
}

// Algorithm 3 with gamma = 1 (V-cycle): nu1 pre-relaxations, residual
// restriction, recursive coarse correction from zero, prolongation and
// correction, nu2 post-relaxations; exact solve on the coarsest level.
template <typename T>
void vcycle(gs_solver* s, IsaacsGrid& g, int l, bool u_is_zero) {
    const int L = (int)g.lv.size() - 1;
    Vec<T> V = level_vec<T>(g, l);
    const Level& Lv = g.lv[l];
    const int tcls = l == 0 ? GS_K_TRANSFER : GS_K_COARSE;
    if (l == L) {
        KScope ks(s, GS_K_COARSE);
        launch_coarse_apply<T>(g.inv, (int)Lv.n, V.f, V.u, s->st);
        return;
    }
    for (int k = 0; k < s->opt.nu1; ++k) smooth<T>(s, g, l, u_is_zero && k == 0);
    {
        KScope ks(s, l == 0 ? GS_K_FINE_RESIDUAL : GS_K_COARSE);
        if constexpr (sizeof(T) == 8) {
            if (l == 0) launch_l0_residual64(g.Kd, Lv.side, g.code, V.f, V.u, V.r, nullptr, s->st);
            else launch_residual9<double>(Lv.A64, Lv.side, V.f, V.u, V.r, s->st);
        } else {
            if (l == 0) launch_l0_residual32(g.Kd, Lv.side, g.code, V.f, V.u, V.r, s->st);
            else launch_residual9<float>(Lv.A32, Lv.side, V.f, V.u, V.r, s->st);
        }
    }
    Vec<T> C = level_vec<T>(g, l + 1);
    {
        KScope ks(s, tcls);
        launch_restrict<T>(V.r, Lv.P64, Lv.P32, Lv.side, C.f, s->st);
    }
    GS_CUDA(cudaMemsetAsync(C.u, 0, sizeof(T) * g.lv[l + 1].n, s->st));
    vcycle<T>(s, g, l + 1, true);
    {
        KScope ks(s, tcls);
        launch_prolong<T>(C.u, Lv.P64, Lv.P32, Lv.side, V.u, s->st);
    }
    for (int k = 0; k < s->opt.nu2; ++k) smooth<T>(s, g, l, false);
}

double fine_residual(gs_solver* s, IsaacsGrid& g, float* r32) {
    clear_scalars(s);
    {
        KScope ks(s, GS_K_REFINE);
        if (r32)
            launch_l0_residual64_to32(g.Kd, g.side, g.code, g.rhs, g.v, r32, &s->dsc->res, s->st);
        else
            launch_l0_residual64(g.Kd, g.side, g.code, g.rhs, g.v, g.lv[0].r64, &s->dsc->res, s->st);
    }
    launch_absmax(g.v, g.n, &s->dsc->vmax, s->st);
    const DevScalars& h = read_scalars(s);
    return bits_to_double(h.res);
}

// Solves (I - mu M) v = r for the assembled codes/rhs of g, warm-started from
// g.v: float64 V-cycles, or (mixed) float32 V-cycles on the float64 residual
// with float64 correction (iterative refinement).  Returns the cycles used.
int linear_solve(gs_solver* s, IsaacsGrid& g, Counters& cnt) {
    const bool mixed = s->opt.precision != GS_PREC_FP64;
    setup_hierarchy(s, g, mixed);
    float* r32 = mixed ? g.lv[0].f32 : nullptr;
    double res = fine_residual(s, g, r32);
    double vmax = bits_to_double(s->hsc->vmax);
    int cycles = 0, slow = 0;
    double prev = res;
    while (cycles < s->opt.max_cycles) {
        const double tol = s->opt.lin_tol * std::max(vmax, 1e-300);
        if (res <= tol || res == 0.0) break;
        if (mixed) {
            vcycle<float>(s, g, 0, true);
            launch_axpy32(g.v, g.lv[0].u32, g.n, s->st);
        } else {
            vcycle<double>(s, g, 0, false);
        }
        ++cycles;
        res = fine_residual(s, g, r32);
        vmax = bits_to_double(s->hsc->vmax);
        // float64 floor: the residual no longer decreases
        slow = res > 0.5 * prev ? slow + 1 : 0;
        if (slow >= 2 && res < 1e-12 * std::max(vmax, 1e-300)) break;
        prev = std::min(prev, res);
    }
    cnt.cycles += cycles;
    cnt.last_lin_res = res;
    return cycles;
}

void vmax_to_device(gs_solver* s, IsaacsGrid& g) {
    clear_scalars(s);
    launch_absmax(g.v, g.n, &s->dsc->vmax, s->st);
}

// AMGpi (Sec. 5.1): Algorithm 2 with Algorithm 1 inside, every linear system
// solved by multigrid.  Starts from g.v, g.alpha and (if beta_given) g.beta.
bool amgpi(gs_solver* s, IsaacsGrid& g, double eps, bool beta_given, Counters& cnt) {
    cudaStream_t st = s->st;
    if (!beta_given) {
        vmax_to_device(s, g);
        KScope ks(s, GS_K_IMPROVE);
        launch_isaacs_improve(IMP_REPLY, g.Kd, g.side, g.variant, g.v, g.r0, g.alpha, g.beta,
                              g.code, g.rhs, nullptr, s->dsc, st);
    } else {
        launch_isaacs_assemble(g.Kd, g.side, g.alpha, g.beta, g.r0, g.code, g.rhs, st);
    }
    bool converged = false;
    int outer = 0;
    while (true) {
        for (int j = 0; j < s->opt.max_inner; ++j) {
            linear_solve(s, g, cnt);
            ++cnt.systems;
            vmax_to_device(s, g);
            KScope ks(s, GS_K_IMPROVE);
            launch_isaacs_improve(IMP_INNER, g.Kd, g.side, g.variant, g.v, g.r0, g.alpha, g.beta,
                                  g.code, g.rhs, nullptr, s->dsc, st);
            if (read_scalars(s).changed == 0) break;
        }
        ++outer;
        vmax_to_device(s, g);
        {
            KScope ks(s, GS_K_IMPROVE);
            launch_isaacs_improve(IMP_OUTER, g.Kd, g.side, g.variant, g.v, g.r0, g.alpha, g.beta,
                                  g.code, g.rhs, g.fv, s->dsc, st);
        }
        const DevScalars& h = read_scalars(s);
        cnt.res_inf = bits_to_double(h.res);
        cnt.res_l2 = std::sqrt(h.res_sq / (double)g.n);
        if (cnt.res_inf <= eps || h.changed == 0) {
            converged = true;
            break;
        }
        if (outer >= s->opt.max_outer) break;
    }
    cnt.outer += outer;
    return converged;
}

void default_policies(gs_solver* s, IsaacsGrid& g) {
    const uint8_t a0 = g.variant == 1 ? 4 : 0;
    k_fill_u8<<<div_up(g.n, 256), 256, 0, s->st>>>(g.alpha, g.n, a0);
    GS_CHECK_LAUNCH();
    GS_CUDA(cudaMemsetAsync(g.beta, 0, g.n * 4, s->st));
    GS_CUDA(cudaMemsetAsync(g.beta4, 0, g.n, s->st));
}

}  // namespace

gs_status run_solve(gs_solver* s, gs_solve_stats* stats) {
    Problem& P = *s->prob;
    Counters cnt;
    cudaEvent_t e0, e1;
    GS_CUDA(cudaEventCreate(&e0));
    GS_CUDA(cudaEventCreate(&e1));
    GS_CUDA(cudaEventRecord(e0, s->st));
    bool converged;
    int fmg_levels = 0;
    IsaacsGrid& fine = *P.grids.back();
    if (s->opt.fmg && P.grids.size() > 1) {
        IsaacsGrid& g0 = *P.grids.front();
        default_policies(s, g0);
        GS_CUDA(cudaMemsetAsync(g0.v, 0, g0.n * sizeof(double), s->st));
        bool beta_given = false;
        converged = false;
        for (size_t k = 0; k < P.grids.size(); ++k) {
            IsaacsGrid& g = *P.grids[k];
            const bool last = k + 1 == P.grids.size();
            const double h = 1.0 / (g.side + 1);
            converged = amgpi(s, g, last ? s->opt.eps : s->opt.fmg_c * h * h, beta_given, cnt);
            ++fmg_levels;
            if (!last) {
                IsaacsGrid& f = *P.grids[k + 1];
                launch_fmg_interp(g.side, g.v, g.alpha, g.beta, g.beta4, f.v, f.alpha, f.beta,
                                  f.beta4, s->st);
                beta_given = true;
            }
        }
    } else {
        if (!s->init_alpha || !s->init_beta) {
            if (!s->init_alpha) {
                const uint8_t a0 = fine.variant == 1 ? 4 : 0;
                k_fill_u8<<<div_up(fine.n, 256), 256, 0, s->st>>>(fine.alpha, fine.n, a0);
                GS_CHECK_LAUNCH();
            }
            if (!s->init_beta) {
                GS_CUDA(cudaMemsetAsync(fine.beta, 0, fine.n * 4, s->st));
                GS_CUDA(cudaMemsetAsync(fine.beta4, 0, fine.n, s->st));
            }
        }
        if (!s->init_v) GS_CUDA(cudaMemsetAsync(fine.v, 0, fine.n * sizeof(double), s->st));
        converged = amgpi(s, fine, s->opt.eps, s->init_beta, cnt);
    }
    GS_CUDA(cudaEventRecord(e1, s->st));
    sync(s);
    float ms = 0;
    GS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->last_levels = (int)fine.lv.size();
    trace_harvest(s);
    reset_initial(s);
    if (stats) {
        stats->outer = cnt.outer;
        stats->systems = cnt.systems;
        stats->cycles = cnt.cycles;
        stats->levels = (int)fine.lv.size();
        stats->res_inf = cnt.res_inf;
        stats->res_l2 = cnt.res_l2;
        stats->seconds = ms * 1e-3;
        stats->converged = converged ? 1 : 0;
        stats->fmg_levels = fmg_levels;
    }
    return converged ? GS_OK : GS_ENOTCONV;
}

gs_status run_improve(gs_solver* s, const double* v, uint8_t* alpha_out, uint8_t* beta_out,
                      double* fv_out) {
    Problem& P = *s->prob;
    IsaacsGrid& g = *P.grids.back();
    // work on copies so that the solver's state is untouched
    Arena scratch(0, 0);
    double* vd = scratch.alloc<double>(g.n);
    uint8_t* a = scratch.alloc<uint8_t>(g.n);
    uint32_t* b = scratch.alloc<uint32_t>(g.n);
    uint8_t* code = scratch.alloc<uint8_t>(g.n);
    double* rhs = scratch.alloc<double>(g.n);
    double* fv = scratch.alloc<double>(g.n);
    GS_CUDA(cudaMemcpyAsync(vd, v, g.n * sizeof(double), cudaMemcpyDefault, s->st));
    GS_CUDA(cudaMemcpyAsync(a, g.alpha, g.n, cudaMemcpyDeviceToDevice, s->st));
    GS_CUDA(cudaMemcpyAsync(b, g.beta, g.n * 4, cudaMemcpyDeviceToDevice, s->st));
    clear_scalars(s);
    launch_absmax(vd, g.n, &s->dsc->vmax, s->st);
    launch_isaacs_improve(IMP_OUTER, g.Kd, g.side, g.variant, vd, g.r0, a, b, code, rhs, fv, s->dsc,
                          s->st);
    if (alpha_out) GS_CUDA(cudaMemcpyAsync(alpha_out, a, g.n, cudaMemcpyDefault, s->st));
    if (fv_out) GS_CUDA(cudaMemcpyAsync(fv_out, fv, g.n * sizeof(double), cudaMemcpyDefault, s->st));
    if (beta_out) {
        const int m1 = g.variant == 1 ? 5 : 4;
        if (m1 == 4) {
            GS_CUDA(cudaMemcpyAsync(beta_out, b, g.n * 4, cudaMemcpyDefault, s->st));
        } else {
            uint8_t* stage = scratch.alloc<uint8_t>(g.n * m1);
            k_unpack_beta<<<div_up(g.n, 256), 256, 0, s->st>>>(b, g.beta4, m1, g.n, stage);
            GS_CHECK_LAUNCH();
            GS_CUDA(cudaMemcpyAsync(beta_out, stage, g.n * m1, cudaMemcpyDefault, s->st));
        }
    }
    sync(s);
    return GS_OK;
}

gs_status run_policy_solve(gs_solver* s, const uint8_t* alpha, const uint8_t* beta,
                           const double* w0, double* w_out, gs_solve_stats* stats) {
    Problem& P = *s->prob;
    IsaacsGrid& g = *P.grids.back();
    const int m1 = g.variant == 1 ? 5 : 4;
    // validate actions on the device before touching the state
    Arena scratch(0, 0);
    uint8_t* a = scratch.alloc<uint8_t>(g.n);
    uint8_t* bst = scratch.alloc<uint8_t>(g.n * m1);
    int* bad = scratch.alloc<int>(2);
    GS_CUDA(cudaMemcpyAsync(a, alpha, g.n, cudaMemcpyDefault, s->st));
    GS_CUDA(cudaMemcpyAsync(bst, beta, g.n * m1, cudaMemcpyDefault, s->st));
    GS_CUDA(cudaMemsetAsync(bad, 0, 2 * sizeof(int), s->st));
    k_check_actions<<<div_up(g.n, 256), 256, 0, s->st>>>(a, g.n, m1, bad);
    k_check_actions<<<div_up(g.n * m1, 256), 256, 0, s->st>>>(bst, g.n * m1, 4, bad + 1);
    GS_CHECK_LAUNCH_N(2);
    int hbad[2];
    GS_CUDA(cudaMemcpyAsync(hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, s->st));
    sync(s);
    if (hbad[0] || hbad[1]) {
        set_last_error("policy_solve: action out of range");
        return GS_EINVAL;
    }
    GS_CUDA(cudaMemcpyAsync(g.alpha, a, g.n, cudaMemcpyDeviceToDevice, s->st));
    k_pack_beta<<<div_up(g.n, 256), 256, 0, s->st>>>(bst, m1, g.n, g.beta, g.beta4);
    GS_CHECK_LAUNCH();
    if (w0) GS_CUDA(cudaMemcpyAsync(g.v, w0, g.n * sizeof(double), cudaMemcpyDefault, s->st));
    else GS_CUDA(cudaMemsetAsync(g.v, 0, g.n * sizeof(double), s->st));
    launch_isaacs_assemble(g.Kd, g.side, g.alpha, g.beta, g.r0, g.code, g.rhs, s->st);
    Counters cnt;
    linear_solve(s, g, cnt);
    GS_CUDA(cudaMemcpyAsync(w_out, g.v, g.n * sizeof(double), cudaMemcpyDefault, s->st));
    sync(s);
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->cycles = cnt.cycles;
        stats->systems = 1;
        stats->levels = (int)g.lv.size();
        stats->res_inf = cnt.last_lin_res;
    }
    return GS_OK;
}

}  // namespace gs
