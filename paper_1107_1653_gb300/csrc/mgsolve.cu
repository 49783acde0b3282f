// Two cooperative kernels per policy-fixed linear system: the Galerkin set-up,
// then the V-cycles (Algorithm 3, gamma = 1) with the float64 stopping test.
// The small coarse levels (the "tail") are relaxed by thread block 0 alone,
// out of shared memory.  Every grid-wide wait is bounded in time; a wait that
// gives up sets an error flag and the kernels return.
#include <mutex>

#include "gridsync.cuh"
#include "mgsolve.cuh"
#include "stencil.cuh"

namespace gs {

namespace {

// Optional phase timestamps (diagnostic builds with -DGS_PHASE_PROF): block 0
// records the global timer after every grid-wide barrier.
#ifdef GS_PHASE_PROF
constexpr unsigned kProfCap = 1u << 16;
__device__ unsigned long long g_prof_ts[kProfCap];
__device__ int g_prof_tag[kProfCap];
__device__ unsigned g_prof_n;
__device__ __forceinline__ void prof_mark(int tag) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned k = g_prof_n++;
        if (k < kProfCap) {
            g_prof_ts[k] = global_ns();
            g_prof_tag[k] = tag;
        }
    }
}
#else
__device__ __forceinline__ void prof_mark(int) {}
#endif

__device__ __forceinline__ int colour_ox(int c) { return c == 0 || c == 3 ? 1 : 0; }
__device__ __forceinline__ int colour_oy(int c) { return c == 0 || c == 2 ? 1 : 0; }

// ------------------------------------------------------------------ phases
// One colour of the C/F relaxation.  Level 0 (5-point) is red-black: colour 0
// = the C points and the cell corners (mutually uncoupled), colour 1 = the
// edge F points.  9-point levels: C points, then corners, x-edges, y-edges.
template <typename T>
__device__ void relax_fine(const L0Op<T>& op, const LevelArgs& L, int c, bool zero, size_t start,
                           size_t stride) {
    T* __restrict__ u = (T*)L.u;
    const T* __restrict__ f = (const T*)L.f;
    const int side = L.side, hs = (side + 1) / 2;
    const size_t cnt = (size_t)side * hs;
    size_t t = start;
    // two independent points per step: the colour's updates read only the other colour
    for (; t + stride < cnt; t += 2 * stride) {
        const size_t t2 = t + stride;
        const int j1 = (int)(t / hs), i1 = ((j1 + c) & 1) + 2 * (int)(t % hs);
        const int j2 = (int)(t2 / hs), i2 = ((j2 + c) & 1) + 2 * (int)(t2 % hs);
        T v1 = T(0), v2 = T(0);
        const bool ok1 = i1 < side, ok2 = i2 < side;
        if (ok1) v1 = op.relaxed(f, u, i1, j1, zero);
        if (ok2) v2 = op.relaxed(f, u, i2, j2, zero);
        if (ok1) u[(size_t)j1 * side + i1] = v1;
        if (ok2) u[(size_t)j2 * side + i2] = v2;
    }
    if (t < cnt) {
        const int j = (int)(t / hs), i = ((j + c) & 1) + 2 * (int)(t % hs);
        if (i < side) u[(size_t)j * side + i] = op.relaxed(f, u, i, j, zero);
    }
}

// The last colour of the last fine relaxation fused with the float64 update
// v += e of the mixed path: points of colour c are relaxed (their e is final
// once written), the other colour's e is already final; nothing reads v here.
__device__ void relax_fine_update(const L0Op<float>& op, const LevelArgs& L, double* __restrict__ v,
                                  int c, size_t start, size_t stride) {
    float* __restrict__ u = (float*)L.u;
    const float* __restrict__ f = (const float*)L.f;
    const int side = L.side;
    for (size_t x = start; x < L.n; x += stride) {
        const int i = (int)(x % side), j = (int)(x / side);
        float e;
        if (((i + j) & 1) == c) {
            e = op.relaxed(f, u, i, j, false);
            u[x] = e;
        } else {
            e = u[x];
        }
        v[x] += (double)e;
    }
}

template <typename T, typename W>
__device__ void relax_coarse(const LevelArgs& L, int c, bool zero, size_t start, size_t stride) {
    const L9Op<T, W> op{(const W*)L.A, L.n, L.side};
    T* u = (T*)L.u;
    const T* f = (const T*)L.f;
    const int ox = colour_ox(c), oy = colour_oy(c);
    const int nx = (L.side - ox + 1) / 2, ny = (L.side - oy + 1) / 2;
    const size_t cnt = (size_t)nx * ny;
    for (size_t t = start; t < cnt; t += stride)
        op.relax(f, u, ox + 2 * (int)(t % nx), oy + 2 * (int)(t / nx), zero);
}

// f_{l+1} = R (f_l - A_l u_l) with the fine residuals formed on the fly;
// u_{l+1} = 0.
template <typename T, typename W, class Op>
__device__ void restrict_with(const Op& op, const LevelArgs& L, const LevelArgs& C, size_t start,
                              size_t stride) {
    const int sc = L.sc;
    const T* u = (const T*)L.u;
    const T* f = (const T*)L.f;
    const W* P = (const W*)L.P;
    T* fc = (T*)C.f;
    T* uc = (T*)C.u;
    const size_t nc = (size_t)sc * sc;
    for (size_t t = start; t < nc; t += stride) {
        const int I = (int)(t % sc), J = (int)(t / sc);
        T acc = 0;
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
                acc += (T)restrict_weight(P, sc, I, J, di, dj) * op.resid(f, u, 2 * I + 1 + di, 2 * J + 1 + dj);
            }
        fc[t] = acc;
        uc[t] = T(0);
    }
}

// u_l += P u_{l+1}, one item per coarse cell (its corner, edge and C points).
template <typename T, typename W>
__device__ void prolong_phase(const LevelArgs& L, const LevelArgs& C, size_t start, size_t stride) {
    const int sc = L.sc, sf = L.side, nc1 = sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    const W* Pw = (const W*)L.P;
    auto P = [&](int k, size_t c) -> T { return (T)wval(Pw[k * ncell + c]); };
    const T* uc = (const T*)C.u;
    T* uf = (T*)L.u;
    for (size_t t = start; t < ncell; t += stride) {
        const int I = (int)(t % nc1), J = (int)(t / nc1);
        auto U = [&](int p, int q) -> T {
            return (p < 0 || q < 0 || p >= sc || q >= sc) ? T(0) : uc[(size_t)q * sc + p];
        };
        const T uSW = U(I - 1, J - 1), uSE = U(I, J - 1), uNW = U(I - 1, J), uNE = U(I, J);
        uf[(size_t)(2 * J) * sf + 2 * I] += P(PSW, t) * uSW + P(PSE, t) * uSE + P(PNW, t) * uNW +
                                            P(PNE, t) * uNE;
        if (J < sc) uf[(size_t)(2 * J + 1) * sf + 2 * I] += P(PXW, t) * uNW + P(PXE, t) * uNE;
        if (I < sc) uf[(size_t)(2 * J) * sf + 2 * I + 1] += P(PYS, t) * uSE + P(PYN, t) * uNE;
        if (I < sc && J < sc) uf[(size_t)(2 * J + 1) * sf + 2 * I + 1] += uNE;
    }
}

// Level-generic wrappers (level 0 is the implicit fine operator).
template <typename T, typename W>
__device__ void relax_level(const SolveArgs& a, const LevelArgs& L, int l, int c, bool zero,
                            size_t start, size_t stride) {
    if (l == 0) relax_fine<T>(L0Op<T>{a.K, a.code, L.side}, L, c, zero, start, stride);
    else relax_coarse<T, W>(L, c, zero, start, stride);
}

template <typename T, typename W>
__device__ void restrict_level(const SolveArgs& a, const LevelArgs& L, const LevelArgs& C, int l,
                               size_t start, size_t stride) {
    if (l == 0) restrict_with<T, W>(L0Op<T>{a.K, a.code, L.side}, L, C, start, stride);
    else restrict_with<T, W>(L9Op<T, W>{(const W*)L.A, L.n, L.side}, L, C, start, stride);
}

// Exact solve on the coarsest level by its explicit inverse (one block).
template <typename T>
__device__ void coarse_apply_block(const LevelArgs& L, const double* inv) {
    __shared__ double fs[64];
    const int n = (int)L.n;
    const T* f = (const T*)L.f;
    T* u = (T*)L.u;
    for (int k = threadIdx.x; k < n; k += blockDim.x) fs[k] = (double)f[k];
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += inv[(size_t)r * n + k] * fs[k];
        u[r] = (T)acc;
    }
    __syncthreads();
}

// V-cycle over levels [lbeg, nlev) by thread block 0 alone, on the level
// descriptors `tl` (shared-memory copies of the levels >= a.smem_from).
template <typename T, typename W>
__device__ void block_vcycle(const SolveArgs& a, const LevelArgs* tl, const double* inv, int lbeg,
                             bool first_zero) {
    const size_t s0 = threadIdx.x, st = blockDim.x;
    const int Lc = a.nlev - 1;
    if (lbeg > 0 && lbeg >= a.smem_from) {
        // right-hand side written by the grid restriction: stage it in
        const T* fg = (const T*)a.L[lbeg].f;
        T* fs = (T*)tl[lbeg].f;
        T* us = (T*)tl[lbeg].u;
        for (size_t k = s0; k < tl[lbeg].n; k += st) {
            fs[k] = fg[k];
            us[k] = T(0);
        }
        __syncthreads();
    }
    for (int l = lbeg; l < Lc; ++l) {
        const int ncol = l == 0 ? 2 : 4;
        const bool z = l > lbeg || first_zero;
        for (int k = 0; k < a.nu1; ++k)
            for (int c = 0; c < ncol; ++c) {
                relax_level<T, W>(a, tl[l], l, c, z && k == 0 && c == 0, s0, st);
                __syncthreads();
            }
        restrict_level<T, W>(a, tl[l], tl[l + 1], l, s0, st);
        __syncthreads();
    }
    coarse_apply_block<T>(tl[Lc], inv);
    for (int l = Lc - 1; l >= lbeg; --l) {
        const int ncol = l == 0 ? 2 : 4;
        prolong_phase<T, W>(tl[l], tl[l + 1], s0, st);
        __syncthreads();
        for (int k = 0; k < a.nu2; ++k)
            for (int c = 0; c < ncol; ++c) {
                relax_level<T, W>(a, tl[l], l, c, false, s0, st);
                __syncthreads();
            }
    }
    if (lbeg > 0 && lbeg >= a.smem_from) {
        // correction for the grid prolongation: stage it out
        T* ug = (T*)a.L[lbeg].u;
        const T* us = (const T*)tl[lbeg].u;
        for (size_t k = s0; k < tl[lbeg].n; k += st) ug[k] = us[k];
        __syncthreads();
    }
}

// Algorithm 3 with gamma = 1 over the whole hierarchy.
template <typename T, typename W>
__device__ bool grid_vcycle(const SolveArgs& a, const LevelArgs* tl, const double* inv,
                            const GridSync& G, size_t gt, size_t gs, bool fine_zero) {
    for (int l = 0; l < a.tail; ++l) {
        const int ncol = l == 0 ? 2 : 4;
        const bool z = l > 0 || fine_zero;
        for (int k = 0; k < a.nu1; ++k)
            for (int c = 0; c < ncol; ++c) {
                relax_level<T, W>(a, a.L[l], l, c, z && k == 0 && c == 0, gt, gs);
                if (!G.sync()) return false;
                prof_mark(1000 + 10 * l + c);
            }
        restrict_level<T, W>(a, a.L[l], a.L[l + 1], l, gt, gs);
        if (!G.sync()) return false;
        prof_mark(2000 + 10 * l);
    }
    if (blockIdx.x == 0) block_vcycle<T, W>(a, tl, inv, a.tail, a.tail > 0 ? true : fine_zero);
    if (!G.sync()) return false;
    prof_mark(4000);
    for (int l = a.tail - 1; l >= 0; --l) {
        const int ncol = l == 0 ? 2 : 4;
        prolong_phase<T, W>(a.L[l], a.L[l + 1], gt, gs);
        if (!G.sync()) return false;
        prof_mark(3000 + 10 * l);
        for (int k = 0; k < a.nu2; ++k)
            for (int c = 0; c < ncol; ++c) {
                if constexpr (sizeof(T) == 4) {
                    if (l == 0 && k == a.nu2 - 1 && c == ncol - 1) {
                        relax_fine_update(L0Op<float>{a.K, a.code, a.L[0].side}, a.L[0], a.v, c, gt, gs);
                        if (!G.sync()) return false;
                        prof_mark(1000 + 10 * l + c);
                        continue;
                    }
                }
                relax_level<T, W>(a, a.L[l], l, c, false, gt, gs);
                if (!G.sync()) return false;
                prof_mark(1000 + 10 * l + c);
            }
    }
    return true;
}

// ------------------------------------------------------------------ set-up
// Set-up item kinds of one level: 0 edge weights, 1 corner weights, 2 Galerkin rows.
__device__ void setup_items(const SolveArgs& a, int l, int kind, size_t start, size_t stride) {
    const LevelArgs& L = a.L[l];
    const int sc = L.sc;
    const WOut Pw{a.mixed && !a.wbf16 ? L.P32 : nullptr, a.wbf16 ? (__nv_bfloat16*)L.P32 : nullptr};
    if (kind < 2) {
        const size_t ncell = (size_t)(sc + 1) * (sc + 1);
        for (size_t t = start; t < ncell; t += stride) {
            if (l == 0) {
                const Src5 src{a.K, a.code, L.side};
                if (kind == 0) interp_edges_item(src, sc, t, L.P64, Pw);
                else interp_corners_item(src, sc, t, L.P64, Pw);
            } else {
                const Src9 src{L.A64, L.side, L.n};
                if (kind == 0) interp_edges_item(src, sc, t, L.P64, Pw);
                else interp_corners_item(src, sc, t, L.P64, Pw);
            }
        }
    } else {
        const size_t nc = (size_t)sc * sc;
        const LevelArgs& C = a.L[l + 1];
        const WOut Aw{a.mixed && !a.wbf16 ? C.A32 : nullptr, a.wbf16 ? (__nv_bfloat16*)C.A32 : nullptr};
        for (size_t t = start; t < nc; t += stride) {
            if (l == 0) rap_item(Src5{a.K, a.code, L.side}, sc, t, L.P64, C.A64, Aw);
            else rap_item(Src9{L.A64, L.side, L.n}, sc, t, L.P64, C.A64, Aw);
        }
    }
}

// Interpolation weights and Galerkin operators of every level for the current
// policy codes, then the explicit inverse of the coarsest operator.
__global__ void __launch_bounds__(kMGThreads) k_mg_setup(const __grid_constant__ SolveArgs a) {
    extern __shared__ double smem[];
    const GridSync G{a.bar, gridDim.x};
    const size_t gt = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gs = (size_t)gridDim.x * blockDim.x;
    const int Lc = a.nlev - 1;
    for (int l = 0; l < Lc && l < a.tail; ++l)
        for (int kind = 0; kind < 3; ++kind) {
            setup_items(a, l, kind, gt, gs);
            if (!G.sync()) return;
            prof_mark(7000 + 10 * l + kind);
        }
    if (blockIdx.x == 0) {
        for (int l = a.tail; l < Lc; ++l)
            for (int kind = 0; kind < 3; ++kind) {
                setup_items(a, l, kind, threadIdx.x, blockDim.x);
                __syncthreads();
            }
        const LevelArgs& L = a.L[Lc];
        if (Lc == 0) coarse_invert_block(Src5{a.K, a.code, L.side}, L.side, smem, a.inv, a.inv_status);
        else coarse_invert_block(Src9{L.A64, L.side, L.n}, L.side, smem, a.inv, a.inv_status);
    }
}

// ------------------------------------------------------------------ cycles
__device__ __forceinline__ float warp_maxf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// float64 residual b - A v of the fine system and |v|_inf; in the mixed path
// the residual, rounded to float32, is the next correction's right-hand side.
__device__ void check_phase(const SolveArgs& a, int slot, size_t gt, size_t gs) {
    const LevelArgs& L = a.L[0];
    const L0Op<double> op{a.K, a.code, L.side};
    float* __restrict__ r32 = a.mixed ? (float*)L.f : nullptr;
    float* __restrict__ e32 = (a.mixed && a.nu1 == 0) ? (float*)L.u : nullptr;
    const double* __restrict__ v = a.v;
    // maxima in float32 (a stopping-test scale; float64 compares are slow here)
    float rm = 0.0f, vm = 0.0f;
    const int side = L.side;
    size_t x = gt;
    for (; x + 3 * gs < L.n; x += 4 * gs) {
        double r[4], vx[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const size_t y = x + k * gs;
            r[k] = op.resid(a.rhs, v, (int)(y % side), (int)(y / side));
            vx[k] = v[y];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const size_t y = x + k * gs;
            if (r32) r32[y] = (float)r[k];
            if (e32) e32[y] = 0.0f;
            rm = fmaxf(rm, fabsf((float)r[k]));
            vm = fmaxf(vm, fabsf((float)vx[k]));
        }
    }
    for (; x < L.n; x += gs) {
        const double r = op.resid(a.rhs, v, (int)(x % side), (int)(x / side));
        if (r32) r32[x] = (float)r;
        if (e32) e32[x] = 0.0f;
        rm = fmaxf(rm, fabsf((float)r));
        vm = fmaxf(vm, fabsf((float)v[x]));
    }
    rm = warp_maxf(rm);
    vm = warp_maxf(vm);
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(&a.out->rmax[slot], (double)rm);
        atomic_max_nonneg(&a.out->vmax[slot], (double)vm);
    }
}

__device__ void axpy_phase(const SolveArgs& a, size_t gt, size_t gs) {
    const float* __restrict__ e = (const float*)a.L[0].u;
    double* __restrict__ v = a.v;
    const size_t n = a.L[0].n;
#pragma unroll 4
    for (size_t x = gt; x < n; x += gs) v[x] += (double)e[x];
}

// Copies the tail levels' operators and transfers (fixed during one launch)
// into block 0's shared memory and builds their descriptors.
template <typename T, typename W>
__device__ void stage_tail(const SolveArgs& a, char* smem, LevelArgs* tl, double** inv_out) {
    for (int l = threadIdx.x; l < a.nlev; l += blockDim.x) tl[l] = a.L[l];
    __syncthreads();
    const int Lc = a.nlev - 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = smem + off;
        off += (bytes + 15) & ~size_t(15);
        return p;
    };
    for (int l = a.smem_from; l <= Lc; ++l) {
        const LevelArgs& G = a.L[l];
        W* A = (W*)take(9 * G.n * sizeof(W));
        const size_t ncell = (size_t)(G.sc + 1) * (G.sc + 1);
        W* P = l < Lc ? (W*)take(8 * ncell * sizeof(W)) : nullptr;
        T* u = (T*)take(G.n * sizeof(T));
        T* f = (T*)take(G.n * sizeof(T));
        const W* gA = (const W*)G.A;
        for (size_t k = threadIdx.x; k < 9 * G.n; k += blockDim.x) A[k] = gA[k];
        if (P) {
            const W* gP = (const W*)G.P;
            for (size_t k = threadIdx.x; k < 8 * ncell; k += blockDim.x) P[k] = gP[k];
        }
        if (threadIdx.x == 0) {
            tl[l].A = A;
            tl[l].P = P;
            tl[l].u = u;
            tl[l].f = f;
        }
    }
    double* inv = (double*)take(a.L[Lc].n * a.L[Lc].n * sizeof(double));
    for (size_t k = threadIdx.x; k < a.L[Lc].n * a.L[Lc].n; k += blockDim.x) inv[k] = a.inv[k];
    *inv_out = inv;
    __syncthreads();
}

template <typename T, typename W>
__global__ void __launch_bounds__(kMGThreads) k_mg_cycles(const __grid_constant__ SolveArgs a) {
    extern __shared__ __align__(16) char smem_c[];
    __shared__ LevelArgs tl[kMaxLevels];
    const GridSync G{a.bar, gridDim.x};
    const size_t gt = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gs = (size_t)gridDim.x * blockDim.x;
    if (!G.sync()) return;   // set-up complete (and error state shared)
    prof_mark(8000);
    double* inv = a.inv;
    if (blockIdx.x == 0) stage_tail<T, W>(a, smem_c, tl, &inv);
    int slot = 0;
    check_phase(a, slot, gt, gs);
    if (!G.sync()) return;
    prof_mark(6000);
    double prev = 0.0, res0 = 0.0;
    int slow = 0;
    for (int cycles = 0;; ++cycles) {
        const double res = __longlong_as_double((long long)__ldcg(&a.out->rmax[slot]));
        const double vm = __longlong_as_double((long long)__ldcg(&a.out->vmax[slot]));
        if (cycles == 0) res0 = res;
        int reason = 0;
        if (res <= a.lin_tol * fmax(vm, 1e-300) || res == 0.0) reason = 1;
        if (cycles > 0) {
            // float64 floor: the residual no longer decreases
            slow = res > 0.5 * prev ? slow + 1 : 0;
            if (!reason && slow >= 2 && res < 1e-12 * fmax(vm, 1e-300)) reason = 1;
            if (!reason && res <= a.rel_tol * res0) reason = 2;
            prev = fmin(prev, res);
        } else {
            prev = res;
        }
        if (!reason && cycles >= a.max_cycles) reason = 3;
        if (reason) {
            if (gt == 0) {
                a.out->cycles = cycles;
                a.out->reason = reason;
                a.out->res = res;
                a.out->vmax_final = vm;
            }
            return;
        }
        if (gt == 0) {
            a.out->rmax[slot ^ 1] = 0ull;
            a.out->vmax[slot ^ 1] = 0ull;
        }
        if (!grid_vcycle<T, W>(a, tl, inv, G, gt, gs, a.mixed != 0)) return;
        if (a.mixed && (a.tail == 0 || a.nu2 == 0)) {   // not fused into the fine relaxation
            axpy_phase(a, gt, gs);
            if (!G.sync()) return;
            prof_mark(5000);
        }
        slot ^= 1;
        check_phase(a, slot, gt, gs);
        if (!G.sync()) return;
        prof_mark(6000);
    }
}

// ------------------------------------------------------------------ launch
struct Occupancy {
    int sms = 0;
    int setup_per_sm = 0;
    int cyc_per_sm[3] = {0, 0, 0};   // float32, float64, float32 on bfloat16 weights
};

Occupancy& occupancy() {
    static Occupancy o;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!o.sms) {
        int dev = 0;
        GS_CUDA(cudaGetDevice(&dev));
        GS_CUDA(cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev));
        const int big = kTailSmemMax;
        GS_CUDA(cudaFuncSetAttribute(k_mg_setup, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     64 * 128 * 8));
        GS_CUDA(cudaFuncSetAttribute(k_mg_cycles<float, float>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        GS_CUDA(cudaFuncSetAttribute(k_mg_cycles<double, double>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        GS_CUDA(cudaFuncSetAttribute(k_mg_cycles<float, __nv_bfloat16>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, big));
        GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.setup_per_sm, k_mg_setup, kMGThreads,
                                                              64 * 128 * 8));
        GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.cyc_per_sm[0], k_mg_cycles<float, float>,
                                                              kMGThreads, big));
        GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.cyc_per_sm[1], k_mg_cycles<double, double>,
                                                              kMGThreads, big));
        GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &o.cyc_per_sm[2], k_mg_cycles<float, __nv_bfloat16>, kMGThreads, big));
        o.setup_per_sm = o.setup_per_sm < 1 ? 1 : o.setup_per_sm;
        for (int& c : o.cyc_per_sm) c = c < 1 ? 1 : c;
    }
    return o;
}

int grid_blocks(const SolveArgs& a, int per_sm, int sms) {
    if (a.tail == 0) return 1;
    const size_t want = (a.L[0].n / 2 + kMGThreads - 1) / kMGThreads;
    size_t cap = (size_t)per_sm * sms;
    if (a.max_blocks > 0) cap = std::min(cap, (size_t)a.max_blocks);
    return (int)std::max<size_t>(1, std::min(want, cap));
}

}  // namespace

size_t tail_smem_bytes(const SolveArgs& a) {
    const int elem = a.mixed ? 4 : 8;
    const int welem = a.wbf16 ? 2 : elem;
    const int Lc = a.nlev - 1;
    size_t off = 0;
    auto take = [&](size_t bytes) { off += (bytes + 15) & ~size_t(15); };
    for (int l = a.smem_from; l <= Lc; ++l) {
        const LevelArgs& G = a.L[l];
        take(9 * G.n * welem);
        if (l < Lc) take(8 * (size_t)(G.sc + 1) * (G.sc + 1) * welem);
        take(G.n * elem);
        take(G.n * elem);
    }
    take(a.L[Lc].n * a.L[Lc].n * sizeof(double));
    return off;
}

#ifdef GS_PHASE_PROF
extern "C" int gamesolve_debug_phase_prof(unsigned long long* ts, int* tags, int cap) {
    unsigned n = 0;
    cudaDeviceSynchronize();
    cudaMemcpyFromSymbol(&n, g_prof_n, sizeof n);
    if (n > kProfCap) n = kProfCap;
    if ((int)n > cap) n = cap;
    cudaMemcpyFromSymbol(ts, g_prof_ts, n * sizeof(unsigned long long));
    cudaMemcpyFromSymbol(tags, g_prof_tag, n * sizeof(int));
    const unsigned zero = 0;
    cudaMemcpyToSymbol(g_prof_n, &zero, sizeof zero);
    return (int)n;
}
#endif

void launch_mg_setup(const SolveArgs& a, cudaStream_t st) {
    const Occupancy& o = occupancy();
    const int nL = (int)a.L[a.nlev - 1].n;
    void* args[] = {(void*)&a};
    const size_t smem = (size_t)2 * nL * nL * sizeof(double);
    GS_CUDA(cudaLaunchCooperativeKernel((const void*)k_mg_setup,
                                        dim3(grid_blocks(a, o.setup_per_sm, o.sms)),
                                        dim3(kMGThreads), args, smem, st));
    note_launches(1);
}

void launch_mg_cycles(const SolveArgs& a, cudaStream_t st) {
    const Occupancy& o = occupancy();
    void* args[] = {(void*)&a};
    const size_t smem = tail_smem_bytes(a);
    const int kind = !a.mixed ? 1 : a.wbf16 ? 2 : 0;
    const void* fn = kind == 1   ? (const void*)k_mg_cycles<double, double>
                     : kind == 2 ? (const void*)k_mg_cycles<float, __nv_bfloat16>
                                 : (const void*)k_mg_cycles<float, float>;
    GS_CUDA(cudaLaunchCooperativeKernel(fn, dim3(grid_blocks(a, o.cyc_per_sm[kind], o.sms)),
                                        dim3(kMGThreads), args, smem, st));
    note_launches(1);
}

}  // namespace gs
