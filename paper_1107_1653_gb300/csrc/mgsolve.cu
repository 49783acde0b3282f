// Two cooperative kernels per policy-fixed linear system: the Galerkin set-up,
// then the multigrid cycles (Algorithm 3; V-cycles, or W-cycles with gamma = 2)
// with the float64 stopping test.
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
    const unsigned cnt = (unsigned)side * hs, st = (unsigned)stride;
    const FastDiv dv(hs);
    unsigned t = (unsigned)start;
    // four independent points per step: the colour's updates read only the other colour
    constexpr int K = 4;
    for (; t + (K - 1) * st < cnt; t += K * st) {
        int i[K], j[K];
        T val[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            unsigned r;
            j[k] = (int)dv.divmod(t + k * st, &r);
            i[k] = ((j[k] + c) & 1) + 2 * (int)r;
            val[k] = i[k] < side ? op.relaxed(f, u, i[k], j[k], zero) : T(0);
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (i[k] < side) u[(size_t)j[k] * side + i[k]] = val[k];
    }
    for (; t < cnt; t += st) {
        unsigned r;
        const int j = (int)dv.divmod(t, &r), i = ((j + c) & 1) + 2 * (int)r;
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
    const unsigned n = (unsigned)L.n, st = (unsigned)stride;
    const FastDiv dv(side);
    unsigned x = (unsigned)start;
    constexpr int K = 4;
    for (; x + (K - 1) * st < n; x += K * st) {
        float e[K];
        bool mine[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            unsigned i;
            const int j = (int)dv.divmod(x + k * st, &i);
            mine[k] = (((int)i + j) & 1) == c;
            e[k] = mine[k] ? op.relaxed(f, u, (int)i, j, false) : u[x + k * st];
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (mine[k]) u[x + k * st] = e[k];
            v[x + k * st] += f32_to_f64(e[k]);
        }
    }
    for (; x < n; x += st) {
        unsigned i;
        const int j = (int)dv.divmod(x, &i);
        float e;
        if ((((int)i + j) & 1) == c) {
            e = op.relaxed(f, u, (int)i, j, false);
            u[x] = e;
        } else {
            e = u[x];
        }
        v[x] += f32_to_f64(e);
    }
}

template <typename T, typename W>
__device__ void relax_coarse(const LevelArgs& L, int c, bool zero, size_t start, size_t stride) {
    const L9Op<T, W> op{(const W*)L.A, L.n, L.side};
    T* u = (T*)L.u;
    const T* f = (const T*)L.f;
    const int ox = colour_ox(c), oy = colour_oy(c);
    const int nx = (L.side - ox + 1) / 2, ny = (L.side - oy + 1) / 2;
    const unsigned cnt = (unsigned)nx * ny, st = (unsigned)stride;
    const FastDiv dv(nx);
    unsigned t = (unsigned)start;
    // two independent points per step (a colour's points are mutually uncoupled)
    for (; t + st < cnt; t += 2 * st) {
        unsigned r1, r2;
        const int j1 = oy + 2 * (int)dv.divmod(t, &r1), i1 = ox + 2 * (int)r1;
        const int j2 = oy + 2 * (int)dv.divmod(t + st, &r2), i2 = ox + 2 * (int)r2;
        const T v1 = op.relaxed(f, u, i1, j1, zero);
        const T v2 = op.relaxed(f, u, i2, j2, zero);
        u[(size_t)j1 * L.side + i1] = v1;
        u[(size_t)j2 * L.side + i2] = v2;
    }
    if (t < cnt) {
        unsigned r;
        const int j = oy + 2 * (int)dv.divmod(t, &r), i = ox + 2 * (int)r;
        u[(size_t)j * L.side + i] = op.relaxed(f, u, i, j, zero);
    }
}

// f_{l+1} = R (f_l - A_l u_l) with the fine residuals formed on the fly;
// u_{l+1} = 0.  With `fuse` the coarse level's first relaxation colour (its
// C points, relaxed from the zero start) is done here too: such a point's
// Gauss-Seidel value is f / diag, from data this item already has.
template <typename T, typename W, class Op>
__device__ void restrict_with(const Op& op, const LevelArgs& L, const LevelArgs& C, bool fuse,
                              size_t start, size_t stride) {
    const int sc = L.sc;
    const T* u = (const T*)L.u;
    const T* f = (const T*)L.f;
    const W* P = (const W*)L.P;
    T* fc = (T*)C.f;
    T* uc = (T*)C.u;
    const L9Op<T, W> cop{(const W*)C.A, C.n, C.side};
    const unsigned nc = (unsigned)sc * sc;
    const FastDiv dv(sc);
    for (unsigned t = (unsigned)start; t < nc; t += (unsigned)stride) {
        unsigned Iu;
        const int J = (int)dv.divmod(t, &Iu), I = (int)Iu;
        T acc = 0;
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
                acc += (T)restrict_weight(P, sc, I, J, di, dj) * op.resid(f, u, 2 * I + 1 + di, 2 * J + 1 + dj);
            }
        fc[t] = acc;
        uc[t] = fuse && (I & J & 1) ? acc / cop.diag(I, J) : T(0);
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
    const FastDiv dv(nc1);
    for (unsigned t = (unsigned)start; t < (unsigned)ncell; t += (unsigned)stride) {
        unsigned Iu;
        const int J = (int)dv.divmod(t, &Iu), I = (int)Iu;
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
                               bool fuse, size_t start, size_t stride) {
    if (l == 0) restrict_with<T, W>(L0Op<T>{a.K, a.code, L.side}, L, C, fuse, start, stride);
    else restrict_with<T, W>(L9Op<T, W>{(const W*)L.A, L.n, L.side}, L, C, fuse, start, stride);
}

// Relaxation sweeps on level l before and after its coarse-grid correction
// (Algorithm 3's nu1, nu2): the finest level's counts, or the coarse levels'.
__device__ __forceinline__ int sweeps_pre(const SolveArgs& a, int l) { return l == 0 ? a.nu1 : a.nu1c; }
__device__ __forceinline__ int sweeps_post(const SolveArgs& a, int l) { return l == 0 ? a.nu2 : a.nu2c; }

// Whether the residual check already relaxed the fine level's first colour
// from the zero start (mixed path: the correction starts from zero).
__device__ __forceinline__ bool fine_colour0_in_check(const SolveArgs& a) {
    return a.mixed && a.nu1 > 0;
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
        // first colour from the zero start already done by the restriction into
        // this level, or (fine level) by the residual check
        const bool done0 = z && (l > lbeg || (l == 0 && fine_colour0_in_check(a)));
        for (int k = 0; k < sweeps_pre(a, l); ++k)
            for (int c = 0; c < ncol; ++c) {
                if (done0 && k == 0 && c == 0) continue;
                relax_level<T, W>(a, tl[l], l, c, z && k == 0 && c == 0, s0, st);
                __syncthreads();
            }
        restrict_level<T, W>(a, tl[l], tl[l + 1], l, l + 1 < Lc && sweeps_pre(a, l + 1) > 0, s0, st);
        __syncthreads();
    }
    coarse_apply_block<T>(tl[Lc], inv);
    for (int l = Lc - 1; l >= lbeg; --l) {
        const int ncol = l == 0 ? 2 : 4;
        prolong_phase<T, W>(tl[l], tl[l + 1], s0, st);
        __syncthreads();
        for (int k = 0; k < sweeps_post(a, l); ++k)
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
    const int Lc = a.nlev - 1;
    for (int l = 0; l < a.tail; ++l) {
        const int ncol = l == 0 ? 2 : 4;
        const bool z = l > 0 || fine_zero;
        // first colour from the zero start already done by the restriction into
        // this level, or (fine level) by the residual check
        const bool done0 = z && (l > 0 || fine_colour0_in_check(a));
        for (int k = 0; k < sweeps_pre(a, l); ++k)
            for (int c = 0; c < ncol; ++c) {
                if (done0 && k == 0 && c == 0) continue;
                relax_level<T, W>(a, a.L[l], l, c, z && k == 0 && c == 0, gt, gs);
                if (!G.sync()) return false;
                prof_mark(1000 + 10 * l + c);
            }
        // the block relaxes level a.tail from its own staged copy: no fusion into it
        restrict_level<T, W>(a, a.L[l], a.L[l + 1], l,
                             l + 1 < a.tail && l + 1 < Lc && sweeps_pre(a, l + 1) > 0, gt, gs);
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
        for (int k = 0; k < sweeps_post(a, l); ++k)
            for (int c = 0; c < ncol; ++c) {
                if constexpr (sizeof(T) == 4) {
                    if (l == 0 && k == sweeps_post(a, l) - 1 && c == ncol - 1) {
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

// ------------------------------------------------------------------ W-cycles
// Algorithm 3 with gamma = 2 (a.gamma): each visit of level l visits level
// l + 1 twice before prolongating.  The first visit of a level starts from
// u = 0 (its first colour may then be done by the restriction into it); the
// second continues from the first visit's u with the same right-hand side.
// Written as a loop over an explicit stack of visit counts (all threads of the
// grid, or of block 0 for the tail, follow the same path).
//
// One visit of the levels [lbeg, nlev) by thread block 0 on the levels' copies
// `tl`; `zero`: u of level lbeg is zero at entry (first visit).
template <typename T, typename W>
__device__ void block_wcycle(const SolveArgs& a, const LevelArgs* tl, const double* inv, int lbeg,
                             bool zero) {
    const size_t s0 = threadIdx.x, st = blockDim.x;
    const int Lc = a.nlev - 1;
    const bool staged = lbeg > 0 && lbeg >= a.smem_from;
    if (staged && zero) {
        const T* fg = (const T*)a.L[lbeg].f;
        T* fs = (T*)tl[lbeg].f;
        T* us = (T*)tl[lbeg].u;
        for (size_t k = s0; k < tl[lbeg].n; k += st) {
            fs[k] = fg[k];
            us[k] = T(0);
        }
        __syncthreads();
    }
    int visits[kMaxLevels];
    int l = lbeg;
    bool z = zero;
    while (true) {
        // enter a visit of level l
        if (l == Lc) {
            coarse_apply_block<T>(tl[Lc], inv);
        } else {
            const int ncol = l == 0 ? 2 : 4;
            const bool done0 = z && (l > lbeg || (l == 0 && fine_colour0_in_check(a)));
            for (int k = 0; k < sweeps_pre(a, l); ++k)
                for (int c = 0; c < ncol; ++c) {
                    if (done0 && k == 0 && c == 0) continue;
                    relax_level<T, W>(a, tl[l], l, c, z && k == 0 && c == 0, s0, st);
                    __syncthreads();
                }
            restrict_level<T, W>(a, tl[l], tl[l + 1], l, l + 1 < Lc && sweeps_pre(a, l + 1) > 0, s0, st);
            __syncthreads();
            visits[l] = 0;
            ++l;
            z = true;
            continue;
        }
        // the visit of level l is complete: return to its parent
        while (true) {
            if (l == lbeg) goto out;
            --l;
            if (++visits[l] < a.gamma) {   // visit level l + 1 again, from its current u
                ++l;
                z = false;
                break;
            }
            const int ncol = l == 0 ? 2 : 4;
            prolong_phase<T, W>(tl[l], tl[l + 1], s0, st);
            __syncthreads();
            for (int k = 0; k < sweeps_post(a, l); ++k)
                for (int c = 0; c < ncol; ++c) {
                    relax_level<T, W>(a, tl[l], l, c, false, s0, st);
                    __syncthreads();
                }
        }
    }
out:
    if (staged) {
        T* ug = (T*)a.L[lbeg].u;
        const T* us = (const T*)tl[lbeg].u;
        for (size_t k = s0; k < tl[lbeg].n; k += st) ug[k] = us[k];
        __syncthreads();
    }
}

// One W-cycle over the whole hierarchy: grid-wide levels [0, a.tail), the tail
// by block 0 (each visit of level a.tail is one block_wcycle).
template <typename T, typename W>
__device__ bool grid_wcycle(const SolveArgs& a, const LevelArgs* tl, const double* inv,
                            const GridSync& G, size_t gt, size_t gs, bool fine_zero) {
    const int Lc = a.nlev - 1;
    int visits[kMaxLevels];
    int l = 0;
    bool z = fine_zero;
    while (true) {
        if (l == a.tail) {
            if (blockIdx.x == 0) block_wcycle<T, W>(a, tl, inv, a.tail, l > 0 ? z : fine_zero);
            if (!G.sync()) return false;
        } else {
            const int ncol = l == 0 ? 2 : 4;
            const bool done0 = z && (l > 0 || fine_colour0_in_check(a));
            for (int k = 0; k < sweeps_pre(a, l); ++k)
                for (int c = 0; c < ncol; ++c) {
                    if (done0 && k == 0 && c == 0) continue;
                    relax_level<T, W>(a, a.L[l], l, c, z && k == 0 && c == 0, gt, gs);
                    if (!G.sync()) return false;
                }
            restrict_level<T, W>(a, a.L[l], a.L[l + 1], l,
                                 l + 1 < a.tail && l + 1 < Lc && sweeps_pre(a, l + 1) > 0, gt, gs);
            if (!G.sync()) return false;
            visits[l] = 0;
            ++l;
            z = true;
            continue;
        }
        while (true) {
            if (l == 0) return true;
            --l;
            if (++visits[l] < a.gamma) {
                ++l;
                z = false;
                break;
            }
            const int ncol = l == 0 ? 2 : 4;
            prolong_phase<T, W>(a.L[l], a.L[l + 1], gt, gs);
            if (!G.sync()) return false;
            for (int k = 0; k < sweeps_post(a, l); ++k)
                for (int c = 0; c < ncol; ++c) {
                    if constexpr (sizeof(T) == 4) {
                        if (l == 0 && k == sweeps_post(a, l) - 1 && c == ncol - 1) {
                            relax_fine_update(L0Op<float>{a.K, a.code, a.L[0].side}, a.L[0], a.v, c,
                                              gt, gs);
                            if (!G.sync()) return false;
                            continue;
                        }
                    }
                    relax_level<T, W>(a, a.L[l], l, c, false, gt, gs);
                    if (!G.sync()) return false;
                }
        }
    }
}

// ------------------------------------------------------------------ set-up
// Float32 storage of level l's set-up in the mixed path: the operator the
// next level's set-up reads (leakage form) and the interpolation weights.
// With bfloat16 weights for the V-cycle, the float32 copies live in the
// (otherwise unused) float64 buffers and the bfloat16 ones in the float32 buffers.
__device__ __forceinline__ float* setup_A32(const SolveArgs& a, const LevelArgs& L) {
    return a.wbf16 ? (float*)L.A64 : L.A32;
}
__device__ __forceinline__ float* setup_P32(const SolveArgs& a, const LevelArgs& L) {
    return a.wbf16 ? (float*)L.P64 : L.P32;
}

// Mixed path set-up items (float32, exact leakage); delta(g) lives in the
// level's float32 right-hand side vector, free during the set-up.
__device__ void setup_items_f(const SolveArgs& a, int l, int kind, size_t start, size_t stride) {
    const LevelArgs& L = a.L[l];
    const int sc = L.sc;
    float* P = setup_P32(a, L);
    __nv_bfloat16* P16 = a.wbf16 ? (__nv_bfloat16*)L.P32 : nullptr;
    float* delta = (float*)L.f;
    const Src5f s5{a.K, a.code, L.side};
    const Src9f s9{setup_A32(a, L), L.side, L.n};
    if (kind < 2) {
        const unsigned ncell = (unsigned)(sc + 1) * (sc + 1);
        for (unsigned t = (unsigned)start; t < ncell; t += (unsigned)stride) {
            if (l == 0) {
                if (kind == 0) interp_edges_item_f(s5, sc, t, P, P16, delta);
                else interp_corners_item_f(s5, sc, t, P, P16, delta);
            } else {
                if (kind == 0) interp_edges_item_f(s9, sc, t, P, P16, delta);
                else interp_corners_item_f(s9, sc, t, P, P16, delta);
            }
        }
    } else {
        const LevelArgs& C = a.L[l + 1];
        float* Ac = setup_A32(a, C);
        __nv_bfloat16* A16 = a.wbf16 ? (__nv_bfloat16*)C.A32 : nullptr;
        const unsigned nc = (unsigned)sc * sc;
        for (unsigned t = (unsigned)start; t < nc; t += (unsigned)stride) {
            if (l == 0) rap_item_f(s5, sc, t, P, delta, Ac, A16);
            else rap_item_f(s9, sc, t, P, delta, Ac, A16);
        }
    }
}

// Set-up item kinds of one level: 0 edge weights, 1 corner weights, 2 Galerkin rows.
__device__ void setup_items(const SolveArgs& a, int l, int kind, size_t start, size_t stride) {
    if (a.mixed) {
        setup_items_f(a, l, kind, start, stride);
        return;
    }
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

// Position of this thread in a warp-major order over the grid: warp w of
// every block comes before warp w + 1 of any block, lanes stay consecutive.
// A level with few items then spreads one warp per block over all SMs
// instead of filling the first blocks (the set-up's items are float64-bound,
// so where they run decides how fast they run).
__device__ __forceinline__ size_t warp_spread_index() {
    const size_t w = (size_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    return w * 32 + (threadIdx.x & 31);
}

// Interpolation weights and Galerkin operators of every level for the current
// policy codes, then the explicit inverse of the coarsest operator.
__global__ void __launch_bounds__(kMGThreads, 2) k_mg_setup(const __grid_constant__ SolveArgs a) {
    extern __shared__ double smem[];
    const GridSync G{a.bar, gridDim.x};
    const size_t gt = warp_spread_index();
    const size_t gs = (size_t)gridDim.x * blockDim.x;
    const int Lc = a.nlev - 1;
    for (int l = 0; l < Lc; ++l)
        for (int kind = 0; kind < 3; ++kind) {
            setup_items(a, l, kind, gt, gs);
            if (!G.sync()) return;
            prof_mark(7000 + 10 * l + kind);
        }
    if (blockIdx.x == 0) {
        const LevelArgs& L = a.L[Lc];
        if (Lc == 0) coarse_invert_block(Src5{a.K, a.code, L.side}, L.side, smem, a.inv, a.inv_status);
        else if (a.mixed)
            coarse_invert_block(Src9fd{setup_A32(a, L), L.side, L.n}, L.side, smem, a.inv, a.inv_status);
        else coarse_invert_block(Src9{L.A64, L.side, L.n}, L.side, smem, a.inv, a.inv_status);
    }
}

// ------------------------------------------------------------------ cycles

// float64 residual b - A v of the fine system and |v|_inf; in the mixed path
// the residual, rounded to float32, is the next correction's right-hand side.
// |x| of a float64 as its bit pattern: non-negative doubles order like their
// bits, so maxima can be taken with integer operations (the float64 pipe is
// the scarce one).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return bits_of(x) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// The float64 residual r = rhs - A v of the fine level with |r|_inf and
// |v|_inf (exact, as bit patterns).  Mixed path: r is also the float32
// right-hand side of the correction, and the correction's first relaxation
// colour from the zero start (C points and cell corners: e = r / diag) is
// done here; with no pre-relaxation the correction is zeroed instead.
__device__ void check_phase(const SolveArgs& a, int slot, size_t gt, size_t gs) {
    const LevelArgs& L = a.L[0];
    const L0Op<double> op{a.K, a.code, L.side};
    const L0Op<float> opf{a.K, a.code, L.side};
    float* __restrict__ r32 = a.mixed ? (float*)L.f : nullptr;
    float* __restrict__ e32 = a.mixed ? (float*)L.u : nullptr;
    const bool relax0 = fine_colour0_in_check(a);
    const double* __restrict__ v = a.v;
    unsigned long long rm = 0, vm = 0;
    const int side = L.side;
    const unsigned n = (unsigned)L.n, st = (unsigned)gs;
    const FastDiv dv(side);
    auto finish = [&](unsigned x, int i, int j, double r) {
        if (r32) {
            const float rf = f64_to_f32(r);
            r32[x] = rf;
            if (relax0) {
                if (((i + j) & 1) == 0) e32[x] = rf / opf.diag(i, j);
            } else {
                e32[x] = 0.0f;
            }
        }
        rm = max(rm, abs_bits(r));
    };
    unsigned x = (unsigned)gt;
    constexpr int K = 4;
    for (; x + (K - 1) * st < n; x += K * st) {
        double r[K];
        int i[K], j[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            unsigned iu;
            j[k] = (int)dv.divmod(x + k * st, &iu);
            i[k] = (int)iu;
            r[k] = op.resid(a.rhs, v, i[k], j[k]);
            vm = max(vm, abs_bits(v[x + k * st]));
        }
#pragma unroll
        for (int k = 0; k < K; ++k) finish(x + k * st, i[k], j[k], r[k]);
    }
    for (; x < n; x += st) {
        unsigned iu;
        const int j = (int)dv.divmod(x, &iu);
        finish(x, (int)iu, j, op.resid(a.rhs, v, (int)iu, j));
        vm = max(vm, abs_bits(v[x]));
    }
    rm = warp_max_u64(rm);
    vm = warp_max_u64(vm);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&a.out->rmax[slot], rm);
        atomicMax(&a.out->vmax[slot], vm);
    }
}

__device__ void axpy_phase(const SolveArgs& a, size_t gt, size_t gs) {
    const float* __restrict__ e = (const float*)a.L[0].u;
    double* __restrict__ v = a.v;
    const size_t n = a.L[0].n;
#pragma unroll 4
    for (size_t x = gt; x < n; x += gs) v[x] += f32_to_f64(e[x]);
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
    int slot = 0;
    if (gridDim.x > 1) {
        // block 0 stages the tail while the others take the first residual check
        if (blockIdx.x == 0) stage_tail<T, W>(a, smem_c, tl, &inv);
        else check_phase(a, slot, gt - blockDim.x, gs - blockDim.x);
    } else {
        stage_tail<T, W>(a, smem_c, tl, &inv);
        check_phase(a, slot, gt, gs);
    }
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
        const bool ok = a.gamma == 2 ? grid_wcycle<T, W>(a, tl, inv, G, gt, gs, a.mixed != 0)
                                     : grid_vcycle<T, W>(a, tl, inv, G, gt, gs, a.mixed != 0);
        if (!ok) return;
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
