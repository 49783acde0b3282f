// Policy iteration with algebraic multigrid (AMGpi, Sec. 5.1) and the full
// multilevel scheme FAMGpi (Algorithm 4, Sec. 5.2): host orchestration of the
// kernels on the solver's stream.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

#include "mgsolve.cuh"
#include "solver.cuh"

namespace gs {

// ------------------------------------------------------------------ memory
Arena::~Arena() {
    for (void* p : ptrs_) cudaFreeAsync(p, st_);
}

void* Arena::raw(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (budget_ && base_ + held_ + bytes > budget_) {
        set_last_error("device memory budget exceeded: %zu + %zu > %zu bytes", base_ + held_, bytes,
                       budget_);
        throw Error{GS_ENOMEM};
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes, st_);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_last_error("cudaMallocAsync(%zu): %s", bytes, cudaGetErrorString(e));
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

void launch_pack_beta(const uint8_t* src, int m1, size_t n, uint32_t* beta, uint8_t* beta4,
                      cudaStream_t st) {
    k_pack_beta<<<div_up(n, 256), 256, 0, st>>>(src, m1, n, beta, beta4);
    GS_CHECK_LAUNCH();
}

void launch_check_actions(const uint8_t* a, size_t n, int limit, int* bad, cudaStream_t st) {
    k_check_actions<<<div_up(n, 256), 256, 0, st>>>(a, n, limit, bad);
    GS_CHECK_LAUNCH();
}

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
    K.kappa_f = (float)K.kappa;
    K.w0mu = K.mu * (0.5 / c0);
    K.gmu = K.mu * (h / (2.0 * c0));
    K.c01 = 0.1 * K.kappa;
    K.w0mu_f = (float)K.w0mu;
    K.gmu_f = (float)K.gmu;
    K.c01_f = (float)K.c01;
    K.h_f = (float)K.h;
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
    auto P = std::make_unique<Problem>(s->opt.mem_budget, held, s->st);
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

// First level whose side is at most the single-block threshold (capped at the
// coarsest): from there on one thread block relaxes, without grid barriers.
int tail_level(const gs_solver* s, const IsaacsGrid& g) {
    const int thr = s->opt.tail_side > 0 ? s->opt.tail_side : 31;
    const int Lc = (int)g.lv.size() - 1;
    for (int l = 0; l < Lc; ++l)
        if (g.lv[l].side <= thr) return l;
    return Lc;
}

// Solves (I - mu M) v = r for the assembled codes/rhs of g, warm-started from
// g.v, in one cooperative launch: Galerkin set-up for the current policies,
// then float64 V-cycles, or float32 V-cycles on the float64 residual with
// float64 correction (iterative refinement), until the float64 stopping test.
// rel_tol > 0 also stops once the residual fell by that factor (an inexact
// policy evaluation); do_setup = false reuses the hierarchy of the previous
// call (valid when the policy codes are unchanged).  Returns why the solve
// stopped: kLinExact (float64 floor or tolerance), kLinInexact (the residual
// fell by rel_tol) or kLinCapped (max_cycles reached short of both).
int linear_solve(gs_solver* s, IsaacsGrid& g, Counters& cnt, double rel_tol, bool do_setup) {
    const bool mixed = s->opt.precision != GS_PREC_FP64;
    SolveArgs a{};
    a.K = g.Kd;
    a.code = g.code;
    a.v = g.v;
    a.rhs = g.rhs;
    a.nlev = (int)g.lv.size();
    a.tail = tail_level(s, g);
    a.nu1 = s->opt.nu1;
    a.nu2 = s->opt.nu2;
    a.nu1c = s->opt.nu1_coarse < 0 ? a.nu1 : s->opt.nu1_coarse;
    a.nu2c = s->opt.nu2_coarse < 0 ? a.nu2 : s->opt.nu2_coarse;
    a.gamma = s->opt.cycle_gamma == 2 ? 2 : 1;
    a.max_cycles = s->opt.max_cycles;
    a.mixed = mixed ? 1 : 0;
    a.wbf16 = s->opt.precision == GS_PREC_MIXED_BF16 ? 1 : 0;
    a.do_setup = do_setup ? 1 : 0;
    a.max_blocks = s->opt.grid_blocks;
    a.lin_tol = s->opt.lin_tol;
    a.rel_tol = rel_tol;
    a.inv = g.inv;
    a.inv_status = g.dstatus;
    a.bar = &s->mgd->bar;
    a.out = &s->mgd->out;
    for (int l = 0; l < a.nlev; ++l) {
        Level& Lv = g.lv[l];
        LevelArgs& L = a.L[l];
        L.side = Lv.side;
        L.sc = (Lv.side - 1) / 2;
        L.n = Lv.n;
        if (l == 0) {
            L.u = mixed ? (void*)Lv.u32 : (void*)g.v;
            L.f = mixed ? (void*)Lv.f32 : (void*)g.rhs;
        } else {
            L.u = mixed ? (void*)Lv.u32 : (void*)Lv.u64;
            L.f = mixed ? (void*)Lv.f32 : (void*)Lv.f64;
            L.A = mixed ? (const void*)Lv.A32 : (const void*)Lv.A64;
        }
        L.P = mixed ? (const void*)Lv.P32 : (const void*)Lv.P64;
        L.A64 = Lv.A64;
        L.A32 = Lv.A32;
        L.P64 = Lv.P64;
        L.P32 = Lv.P32;
        L.u2 = mixed ? (void*)Lv.r32 : (void*)Lv.r64;
    }
    // about two blocks per SM in a tiled launch; tile sides for that many workers
    {
        int dev = 0, sms = 0;
        GS_CUDA(cudaGetDevice(&dev));
        GS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int blocks = 2 * sms;
        if (a.max_blocks > 0) blocks = std::min(blocks, a.max_blocks);
        set_tile_sides(a, std::max(1, blocks - 1));
    }
    a.tile_from = 1;
    const int tile_max = a.mixed ? kTiledMaxSide : kTiledMaxSideF64;
    while (a.tile_from < a.tail && a.L[a.tile_from].side > tile_max) ++a.tile_from;
    // levels from smem_from on are staged in block 0's shared memory, as many as fit
    a.smem_from = std::max(a.tail, 1);
    while (a.smem_from < a.nlev && tail_smem_bytes(a) > (size_t)kTailSmemMax)
        ++a.smem_from;
    // tiled V-cycles where they apply: V-cycles with at least one grid-wide
    // level, shared memory within the launch's limit
    a.tiled = s->opt.cycle_kernel == 0 && a.gamma == 1 && a.tail >= 1 &&
              (a.max_blocks == 0 || a.max_blocks >= 2) &&
              tiled_smem_bytes(a) <= (size_t)kTiledSmemMax;
    GS_CUDA(cudaMemsetAsync(s->mgd, 0, sizeof(MGState), s->st));
    if (do_setup) {
        KScope ks(s, GS_K_MG_SETUP);
        launch_mg_setup(a, s->st);
    }
    {
        KScope ks(s, GS_K_MG_CYCLES);
        launch_mg_cycles(a, s->st);
    }
    GS_CUDA(cudaMemcpyAsync(s->mgh, s->mgd, sizeof(MGState), cudaMemcpyDeviceToHost, s->st));
    sync(s);
    if (s->mgh->bar.error) {
        set_last_error("multigrid solve: a grid barrier wait timed out");
        throw Error{GS_ETIMEOUT};
    }
    if (do_setup) {
        g.hier_valid = true;
        g.stale_rows = 0;
    } else if (rel_tol > 0.0 && s->mgh->out.cycles > 3) {
        // a reused hierarchy that needs more than 3 cycles for an inexact
        // evaluation's drop (a fresh one needs 1-2 at rel_tol 1e-2) has gone
        // stale for the changed rows: rebuild it for the next system
        g.hier_valid = false;
    }
    cnt.cycles += s->mgh->out.cycles;
    cnt.last_lin_res = s->mgh->out.res;
    const int why = s->mgh->out.reason;
    if (why == kLinCapped) cnt.lin_capped = true;
    return why;
}

// The Galerkin hierarchy must be rebuilt unless it was built for (nearly)
// the current policy codes.
bool need_setup(const gs_solver* s, const IsaacsGrid& g) {
    if (!g.hier_valid) return true;
    return (double)g.stale_rows > s->opt.setup_reuse * (double)g.n;
}

// Keep-current tolerance 1e-13 max(1, |v|_inf) with |v|_inf from the last
// multigrid solve's final residual evaluation (v has not changed since).
double tie_tol(const gs_solver* s) { return 1e-13 * std::max(1.0, s->mgh->out.vmax_final); }

void vmax_to_device(gs_solver* s, IsaacsGrid& g) {
    clear_scalars(s);
    launch_absmax(g.v, g.n, &s->dsc->vmax, s->st);
}

// AMGpi (Sec. 5.1): Algorithm 2 with Algorithm 1 inside, every linear system
// solved by multigrid.  Starts from g.v, g.alpha and (if beta_given) g.beta.
bool amgpi(gs_solver* s, IsaacsGrid& g, double eps, bool beta_given, Counters& cnt) {
    cudaStream_t st = s->st;
    g.hier_valid = false;
    if (!beta_given) {
        vmax_to_device(s, g);
        KScope ks(s, GS_K_IMPROVE);
        launch_isaacs_improve(IMP_REPLY, g.Kd, g.side, g.variant, g.v, g.r0, g.alpha, g.beta,
                              g.code, g.rhs, nullptr, s->dsc, -1.0, st);
    } else {
        launch_isaacs_assemble(g.Kd, g.side, g.alpha, g.beta, g.r0, g.code, g.rhs, st);
    }
    bool converged = false;
    int outer = 0;
    while (true) {
        auto inner_improve = [&]() {
            clear_scalars(s);
            KScope ks(s, GS_K_IMPROVE);
            launch_isaacs_improve(IMP_INNER, g.Kd, g.side, g.variant, g.v, g.r0, g.alpha, g.beta,
                                  g.code, g.rhs, nullptr, s->dsc, tie_tol(s), st);
            const DevScalars& h = read_scalars(s);
            g.stale_rows += h.code_changed;
            return h.changed;
        };
        for (int j = 0; j < s->opt.max_inner; ++j) {
            // Algorithm 1 step 1: evaluate MIN's policy (inexactly inside the loop)
            const int why = linear_solve(s, g, cnt, s->opt.pi_rtol, need_setup(s, g));
            ++cnt.systems;
            if (why == kLinCapped) break;   // not evaluated: no decision may rest on it
            if (inner_improve() != 0) continue;
            if (why == kLinInexact) {
                // confirm on the float64-floor solution of the same system before stopping
                if (linear_solve(s, g, cnt, 0.0, need_setup(s, g)) == kLinCapped) break;
                if (inner_improve() != 0) continue;
            }
            break;
        }
        ++outer;
        clear_scalars(s);
        {
            KScope ks(s, GS_K_IMPROVE);
            launch_isaacs_improve(IMP_OUTER, g.Kd, g.side, g.variant, g.v, g.r0, g.alpha, g.beta,
                                  g.code, g.rhs, g.fv, s->dsc, tie_tol(s), st);
        }
        const DevScalars& h = read_scalars(s);
        g.stale_rows += h.code_changed;
        cnt.res_inf = bits_to_double(h.res);
        cnt.res_l2 = std::sqrt(h.res_sq / (double)g.n);
        // a policy evaluation stopped at the cycle cap ends the iteration
        // unconverged: its value is the best iterate, not a fixed point
        if (cnt.lin_capped) break;
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

bool solve_policy_system(gs_solver* s, IsaacsGrid& g, int* cycles, double* res) {
    Counters cnt;
    g.hier_valid = false;
    const int why = linear_solve(s, g, cnt, 0.0, true);
    *cycles = cnt.cycles;
    *res = cnt.last_lin_res;
    return why == kLinExact;
}

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
        s->level_stats.clear();
        for (size_t k = 0; k < P.grids.size(); ++k) {
            IsaacsGrid& g = *P.grids[k];
            const bool last = k + 1 == P.grids.size();
            const double h = 1.0 / (g.side + 1);
            const int outer0 = cnt.outer, systems0 = cnt.systems;
            converged = amgpi(s, g, last ? s->opt.eps : s->opt.fmg_c * h * h, beta_given, cnt);
            ++fmg_levels;
            s->level_stats.insert(s->level_stats.end(),
                                  {g.side, cnt.outer - outer0, cnt.systems - systems0});
            if (cnt.lin_capped) {   // the finer levels are not reached
                converged = false;
                break;
            }
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
        s->level_stats = {fine.side, cnt.outer, cnt.systems};
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
    Arena scratch(0, 0, s->st);
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
                          -1.0, s->st);
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

gs_status run_fmg_interpolate(int side_c, int variant, const double* v_c, const uint8_t* alpha_c,
                              const uint8_t* beta_c, double* v_f, uint8_t* alpha_f,
                              uint8_t* beta_f, cudaStream_t st) {
    const int m1 = variant == 1 ? 5 : 4;
    const size_t nc = (size_t)side_c * side_c;
    const int side_f = 2 * side_c + 1;
    const size_t nf = (size_t)side_f * side_f;
    Arena ar(0, 0, st);
    double* vc = ar.alloc<double>(nc);
    uint8_t* ac = ar.alloc<uint8_t>(nc);
    uint8_t* bstage_c = ar.alloc<uint8_t>(nc * m1);
    uint32_t* bc = ar.alloc<uint32_t>(nc);
    uint8_t* b4c = ar.alloc<uint8_t>(nc);
    double* vf = ar.alloc<double>(nf);
    uint8_t* af = ar.alloc<uint8_t>(nf);
    uint32_t* bf = ar.alloc<uint32_t>(nf);
    uint8_t* b4f = ar.alloc<uint8_t>(nf);
    uint8_t* bstage_f = ar.alloc<uint8_t>(nf * m1);
    int* bad = ar.alloc<int>(2);
    GS_CUDA(cudaMemcpyAsync(vc, v_c, nc * sizeof(double), cudaMemcpyDefault, st));
    GS_CUDA(cudaMemcpyAsync(ac, alpha_c, nc, cudaMemcpyDefault, st));
    GS_CUDA(cudaMemcpyAsync(bstage_c, beta_c, nc * m1, cudaMemcpyDefault, st));
    GS_CUDA(cudaMemsetAsync(bad, 0, 2 * sizeof(int), st));
    GS_CUDA(cudaMemsetAsync(b4c, 0, nc, st));
    k_check_actions<<<div_up(nc, 256), 256, 0, st>>>(ac, nc, m1, bad);
    k_check_actions<<<div_up(nc * m1, 256), 256, 0, st>>>(bstage_c, nc * m1, 4, bad + 1);
    GS_CHECK_LAUNCH_N(2);
    int hbad[2];
    GS_CUDA(cudaMemcpyAsync(hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    if (hbad[0] || hbad[1]) {
        set_last_error("fmg_interpolate: action out of range");
        return GS_EINVAL;
    }
    k_pack_beta<<<div_up(nc, 256), 256, 0, st>>>(bstage_c, m1, nc, bc, b4c);
    GS_CHECK_LAUNCH();
    launch_fmg_interp(side_c, vc, ac, bc, m1 == 5 ? b4c : nullptr, vf, af, bf,
                      m1 == 5 ? b4f : nullptr, st);
    k_unpack_beta<<<div_up(nf, 256), 256, 0, st>>>(bf, b4f, m1, nf, bstage_f);
    GS_CHECK_LAUNCH();
    if (v_f) GS_CUDA(cudaMemcpyAsync(v_f, vf, nf * sizeof(double), cudaMemcpyDefault, st));
    if (alpha_f) GS_CUDA(cudaMemcpyAsync(alpha_f, af, nf, cudaMemcpyDefault, st));
    if (beta_f) GS_CUDA(cudaMemcpyAsync(beta_f, bstage_f, nf * m1, cudaMemcpyDefault, st));
    GS_CUDA(cudaStreamSynchronize(st));
    return GS_OK;
}

gs_status run_policy_solve(gs_solver* s, const uint8_t* alpha, const uint8_t* beta,
                           const double* w0, double* w_out, gs_solve_stats* stats) {
    Problem& P = *s->prob;
    IsaacsGrid& g = *P.grids.back();
    const int m1 = g.variant == 1 ? 5 : 4;
    // validate actions on the device before touching the state
    Arena scratch(0, 0, s->st);
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
    g.hier_valid = false;
    const int why = linear_solve(s, g, cnt, 0.0, true);
    GS_CUDA(cudaMemcpyAsync(w_out, g.v, g.n * sizeof(double), cudaMemcpyDefault, s->st));
    sync(s);
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->cycles = cnt.cycles;
        stats->systems = 1;
        stats->levels = (int)g.lv.size();
        stats->res_inf = cnt.last_lin_res;
        stats->converged = why == kLinExact ? 1 : 0;
    }
    if (why != kLinExact) {
        set_last_error("policy_solve: %d cycles reached before the float64 floor", cnt.cycles);
        return GS_ENOTCONV;
    }
    return GS_OK;
}

}  // namespace gs
