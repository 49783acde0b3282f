// Two cooperative kernels per policy-fixed linear system: the Galerkin set-up,
// then the multigrid cycles (Algorithm 3; V-cycles, or W-cycles with gamma = 2)
// with the float64 stopping test.
// The small coarse levels (the "tail") are relaxed by thread block 0 alone,
// out of shared memory.  Every grid-wide wait is bounded in time; a wait that
// gives up sets an error flag and the kernels return.
#include <algorithm>
#include <cmath>
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
__device__ __forceinline__ void prof_record(int tag) {
    const unsigned k = atomicAdd(&g_prof_n, 1u);
    if (k < kProfCap) {
        g_prof_ts[k] = global_ns();
        g_prof_tag[k] = tag;
    }
}
__device__ __forceinline__ void prof_mark(int tag) {
    if (blockIdx.x == 0 && threadIdx.x == 0) prof_record(tag);
}
// Blocks 1 and the last one record when their own work in a phase ended
// (tag + 100000, tag + 200000), before they wait at the grid barrier.
__device__ __forceinline__ void prof_done(int tag) {
    if (blockIdx.x == 1 || blockIdx.x == gridDim.x - 1) {
        __syncthreads();
        if (threadIdx.x == 0) prof_record(tag + (blockIdx.x == 1 ? 100000 : 200000));
    }
}
#else
__device__ __forceinline__ void prof_mark(int) {}
__device__ __forceinline__ void prof_done(int) {}
#endif

__device__ __forceinline__ int colour_ox(int c) { return c == 0 || c == 3 ? 1 : 0; }
__device__ __forceinline__ int colour_oy(int c) { return c == 0 || c == 2 ? 1 : 0; }

// ------------------------------------------------------------------ phases
// One colour of the C/F relaxation.  Level 0 (5-point) is red-black: colour 0
// = the C points and the cell corners (mutually uncoupled), colour 1 = the
// edge F points.  9-point levels: C points, then corners, x-edges, y-edges.
// The zero-start flag is a template parameter: a run-time flag guarding the
// neighbour loads kept the compiler from issuing a batch's loads together,
// which doubled a phase's time.
template <typename T, bool zero>
__device__ void relax_fine_z(const L0Op<T>& op, const LevelArgs& L, int c, size_t start, size_t stride) {
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

template <typename T>
__device__ void relax_fine(const L0Op<T>& op, const LevelArgs& L, int c, bool zero, size_t start,
                           size_t stride) {
    if (zero) relax_fine_z<T, true>(op, L, c, start, stride);
    else relax_fine_z<T, false>(op, L, c, start, stride);
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

template <typename T, typename W, bool zero>
__device__ void relax_coarse_z(const LevelArgs& L, int c, size_t start, size_t stride) {
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

template <typename T, typename W>
__device__ void relax_coarse(const LevelArgs& L, int c, bool zero, size_t start, size_t stride) {
    if (zero) relax_coarse_z<T, W, true>(L, c, start, stride);
    else relax_coarse_z<T, W, false>(L, c, start, stride);
}

// f_{l+1} = R (f_l - A_l u_l) with the fine residuals formed on the fly;
// u_{l+1} = 0.  With `fuse` the coarse level's first relaxation colour (its
// C points, relaxed from the zero start) is done here too: such a point's
// Gauss-Seidel value is f / diag, from data this item already has.
// skip1 (the finest level after at least one pre-smoothing sweep): the
// red-black sweep ends with colour 1, whose points' residuals that update has
// just made zero (up to rounding), so only the colour-0 points' residuals
// (the C point and the cell corners of each coarse point's stencil) are
// formed; the edge points' are taken as zero.
template <typename T, typename W, bool skip1, class Op>
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
                if (skip1 && ((di + dj) & 1)) continue;
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
    if (l == 0 && a.nu1 > 0) restrict_with<T, W, true>(L0Op<T>{a.K, a.code, L.side}, L, C, fuse, start, stride);
    else if (l == 0) restrict_with<T, W, false>(L0Op<T>{a.K, a.code, L.side}, L, C, fuse, start, stride);
    else restrict_with<T, W, false>(L9Op<T, W>{(const W*)L.A, L.n, L.side}, L, C, fuse, start, stride);
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

// ------------------------------------------------------------------ tiled V-cycle
// The same V-cycle (Algorithm 3, gamma = 1) with far fewer grid-wide barriers.
// A grid-wide level is cut into tiles, one thread block per tile at a time.
// A tile stages its points plus a halo in shared memory and runs a whole leg
// of the cycle there:
//  - down, coarse level l: the pre-smoothing colours, the residual and the
//    restriction into level l + 1 (with that level's first colour);
//  - up, coarse level l: the prolongation from level l + 1 and every
//    post-smoothing colour;
//  - the finest level, one phase per cycle: prolongation, post-smoothing,
//    the float64 update v += e (mixed path), the float64 residual of the
//    stopping test, then the next cycle's pre-smoothing and restriction
//    (discarded when the test stops the solve).
// Each colour update leaves the values it computed exact on a region one
// point narrower on every side that faces another tile (a point's new value
// needs its neighbours' current ones), so the halo is as deep as the updates
// a leg makes; the tile's own points are exact at the end and only they are
// written back.  Every point is computed by the same arithmetic as in the
// phase-per-colour kernel above; the halo points are recomputed by the
// neighbouring tiles.  One grid-wide barrier per leg remains (about 2 per
// level and cycle instead of 13 at V(1,2)); thread block 0 keeps the tail
// levels in its shared memory and takes no tiles.

// Tile k of a level of side sf whose next coarser level has side sc: the
// coarser points [I0, I1) x [J0, J1) it restricts to, the points of this level
// it owns ([2 I0, 2 I1) per direction, plus the last point 2 sc for the last
// tile) and the staged region: [2 I0 - H, 2 I1 + 1 + H) clipped to the level.
struct Tile {
    int I0, I1, J0, J1;
    int ox0, ox1, oy0, oy1;
    int gx0, gx1, gy0, gy1;
    int w, h;
    __device__ __forceinline__ int loc(int i, int j) const { return (j - gy0) * w + (i - gx0); }
};

__device__ __forceinline__ Tile make_tile(int k, int tc, int sc, int sf, int H) {
    const int ntx = (sc + tc - 1) / tc;
    Tile t;
    const int ty = k / ntx, tx = k - ty * ntx;
    t.I0 = tx * tc;
    t.I1 = min(sc, t.I0 + tc);
    t.J0 = ty * tc;
    t.J1 = min(sc, t.J0 + tc);
    t.ox0 = 2 * t.I0;
    t.ox1 = t.I1 == sc ? sf : 2 * t.I1;
    t.oy0 = 2 * t.J0;
    t.oy1 = t.J1 == sc ? sf : 2 * t.J1;
    t.gx0 = max(0, 2 * t.I0 - H);
    t.gx1 = min(sf, 2 * t.I1 + 1 + H);
    t.gy0 = max(0, 2 * t.J0 - H);
    t.gy1 = min(sf, 2 * t.J1 + 1 + H);
    t.w = t.gx1 - t.gx0;
    t.h = t.gy1 - t.gy0;
    return t;
}

__device__ __forceinline__ int tile_count(int tc, int sc) {
    const int nt = (sc + tc - 1) / tc;
    return nt * nt;
}

// Rectangle on which the staged values are still exact.
struct Valid {
    int x0, x1, y0, y1;
    // One colour update: sides that face another tile lose one point.
    __device__ __forceinline__ void shrink(int side) {
        if (x0 > 0) ++x0;
        if (x1 < side) --x1;
        if (y0 > 0) ++y0;
        if (y1 < side) --y1;
    }
};

// Calls f(i, j) for the points i = px, j = py (mod 2) of the rectangle,
// spread over the block's threads.
template <class F>
__device__ __forceinline__ void for_sublattice(const Valid& r, int px, int py, F&& f) {
    const int i0 = r.x0 + ((r.x0 ^ px) & 1), j0 = r.y0 + ((r.y0 ^ py) & 1);
    const int nx = (r.x1 - i0 + 1) >> 1, ny = (r.y1 - j0 + 1) >> 1;
    if (nx <= 0 || ny <= 0) return;
    const FastDiv dv((unsigned)nx);
    for (unsigned t = threadIdx.x; t < (unsigned)(nx * ny); t += blockDim.x) {
        unsigned rr;
        const int q = (int)dv.divmod(t, &rr);
        f(i0 + 2 * (int)rr, j0 + 2 * q);
    }
}

template <class F>
__device__ __forceinline__ void for_rect(int x0, int x1, int y0, int y1, F&& f) {
    const int nx = x1 - x0, ny = y1 - y0;
    if (nx <= 0 || ny <= 0) return;
    const FastDiv dv((unsigned)nx);
    for (unsigned t = threadIdx.x; t < (unsigned)(nx * ny); t += blockDim.x) {
        unsigned rr;
        const int q = (int)dv.divmod(t, &rr);
        f(x0 + (int)rr, y0 + q);
    }
}

// Like for_rect, with B points per thread in flight: ld(i, j) (global loads)
// runs for all B points before st(i, j, value) (shared-memory stores), so a
// thread has B points' loads outstanding at once.
template <int B, class Load, class Store>
__device__ __forceinline__ void batched_rect(int x0, int x1, int y0, int y1, Load&& ld, Store&& st) {
    const int nx = x1 - x0, ny = y1 - y0;
    if (nx <= 0 || ny <= 0) return;
    const FastDiv dv((unsigned)nx);
    const unsigned cnt = (unsigned)(nx * ny);
    using V = decltype(ld(0, 0));
    for (unsigned base = threadIdx.x; base < cnt; base += B * blockDim.x) {
        V val[B];
        int ii[B], jj[B];
        bool ok[B];
#pragma unroll
        for (int b = 0; b < B; ++b) {
            const unsigned t = base + b * blockDim.x;
            ok[b] = t < cnt;
            unsigned r;
            const int q = (int)dv.divmod(ok[b] ? t : 0u, &r);
            ii[b] = x0 + (int)r;
            jj[b] = y0 + q;
            if (ok[b]) val[b] = ld(ii[b], jj[b]);
        }
#pragma unroll
        for (int b = 0; b < B; ++b)
            if (ok[b]) st(ii[b], jj[b], val[b]);
    }
}

// Shared-memory form of the 9-point level operator (same arithmetic as L9Op).
// 9-point level in shared memory: A[d * wh + k] in the cycle's type (float32
// rows in leakage form: row sum in slot 0).
template <typename T>
struct T9 {
    const T* A;
    int side, w, wh;
    __device__ __forceinline__ T resid(const T* f, const T* u, int k, int i, int j) const {
        const T ux = u[k];
        T Au = A[k] * ux;
#pragma unroll
        for (int d = 1; d < 9; ++d) {
            const int gi = i + dir_di(d), gj = j + dir_dj(d);
            const bool in = gi >= 0 && gj >= 0 && gi < side && gj < side;
            const T ud = in ? u[k + dir_di(d) + dir_dj(d) * w] : T(0);
            if constexpr (sizeof(T) == 8) Au += A[d * wh + k] * ud;
            else Au += A[d * wh + k] * (ud - ux);
        }
        return f[k] - Au;
    }
    __device__ __forceinline__ T relaxed(const T* f, const T* u, int k, int i, int j) const {
        T s = f[k];
        T diag = A[k];
#pragma unroll
        for (int d = 1; d < 9; ++d) {
            const T a = A[d * wh + k];
            if constexpr (sizeof(T) == 4) diag -= a;
            const int gi = i + dir_di(d), gj = j + dir_dj(d);
            if (gi < 0 || gj < 0 || gi >= side || gj >= side) continue;
            s -= a * u[k + dir_di(d) + dir_dj(d) * w];
        }
        return s / diag;
    }
};

// Correction of level l at its point (i, j) from level l + 1 (u_c of side sc,
// weights P of the cells (I, J) in [0, sc]^2): the prolongation P u_c.
template <typename T, typename W>
__device__ __forceinline__ T prolonged(const W* Pw, const T* uc, int sc, int i, int j) {
    const int nc1 = sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    auto P = [&](int k, size_t c) -> T { return (T)wval(Pw[k * ncell + c]); };
    auto U = [&](int p, int q) -> T {
        return (p < 0 || q < 0 || p >= sc || q >= sc) ? T(0) : uc[(size_t)q * sc + p];
    };
    if (!(i & 1)) {
        const int I = i >> 1;
        if (!(j & 1)) {   // cell corner (2I, 2J)
            const int J = j >> 1;
            const size_t t = (size_t)J * nc1 + I;
            return P(PSW, t) * U(I - 1, J - 1) + P(PSE, t) * U(I, J - 1) + P(PNW, t) * U(I - 1, J) +
                   P(PNE, t) * U(I, J);
        }
        const int J = j >> 1;   // x-edge (2I, 2J + 1)
        const size_t t = (size_t)J * nc1 + I;
        return P(PXW, t) * U(I - 1, J) + P(PXE, t) * U(I, J);
    }
    const int I = i >> 1;
    if (!(j & 1)) {   // y-edge (2I + 1, 2J)
        const int J = j >> 1;
        const size_t t = (size_t)J * nc1 + I;
        return P(PYS, t) * U(I, J - 1) + P(PYN, t) * U(I, J);
    }
    return U(I, j >> 1);   // C point (2I + 1, 2J + 1)
}

// Restriction of the staged residuals r (rows of width rw from fine point
// (2 I0, 2 J0)) into the tile's points of level l + 1: f_c = R r.  The next
// level's first colour (f_c / diag at its C points) is formed by whoever
// stages f_c; zero_uc clears u_c instead (level l + 1 is the tail, relaxed by
// block 0 from u_c = 0).
template <typename T, typename W>
__device__ void tile_restrict(const Tile& t, const T* r, int rw, const LevelArgs& L,
                              const LevelArgs& C, bool zero_uc) {
    const W* P = (const W*)L.P;
    const int sc = L.sc;
    T* fc = (T*)C.f;
    T* uc = (T*)C.u;
    for_rect(t.I0, t.I1, t.J0, t.J1, [&](int I, int J) {
        T acc = 0;
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
            for (int di = -1; di <= 1; ++di)
                acc += (T)restrict_weight(P, sc, I, J, di, dj) *
                       r[(2 * (J - t.J0) + 1 + dj) * rw + 2 * (I - t.I0) + 1 + di];
        const size_t x = (size_t)J * sc + I;
        fc[x] = acc;
        if (zero_uc) uc[x] = T(0);
    });
}

// Down leg of a coarse level l (1 <= l < tail): pre-smoothing (the first
// colour was done by the restriction into l), residual, restriction.
template <typename T, typename W>
__device__ __noinline__ void tile_down(const SolveArgs& a, int l, char* smem, int worker, int nworkers) {
    const LevelArgs& L = a.L[l];
    const LevelArgs& C = a.L[l + 1];
    const int sf = L.side, sc = L.sc, nu = a.nu1c;
    const int K1 = nu > 0 ? 4 * nu - 1 : 0;
    const int H = 1 + K1;
    const bool zero_uc = l + 1 == a.tail;
    const int tc = a.tc[l];
    const int ntiles = tile_count(tc, sc);
    const W* gA = (const W*)L.A;
    T* gu = (T*)L.u;
    const T* gf = (const T*)L.f;
    struct Pt { T f, A[9]; };
    for (int k = worker; k < ntiles; k += nworkers) {
        const Tile t = make_tile(k, tc, sc, sf, H);
        const int wh = t.w * t.h;
        T* A = (T*)smem;
        T* u = A + 9 * wh;
        T* f = u + wh;
        T* r = f + wh;   // residuals at fine points [2 I0, 2 I1] x [2 J0, 2 J1]
        batched_rect<2>(
            t.gx0, t.gx1, t.gy0, t.gy1,
            [&](int i, int j) {
                const size_t x = (size_t)j * sf + i;
                Pt p;
                p.f = gf[x];
#pragma unroll
                for (int d = 0; d < 9; ++d) p.A[d] = (T)wval(gA[d * L.n + x]);
                return p;
            },
            [&](int i, int j, const Pt& p) {
                const int q = t.loc(i, j);
                f[q] = p.f;
                T d = p.A[0];
#pragma unroll
                for (int e = 0; e < 9; ++e) A[e * wh + q] = p.A[e];
                if constexpr (sizeof(T) == 4) {
#pragma unroll
                    for (int e = 1; e < 9; ++e) d -= p.A[e];
                }
                // u from the zero start, the first colour (C points) relaxed: f / diag
                u[q] = nu > 0 && (i & j & 1) ? p.f / d : T(0);
            });
        __syncthreads();
        const T9<T> op{A, sf, t.w, wh};
        Valid v{t.gx0, t.gx1, t.gy0, t.gy1};
        for (int s = 0; s < nu; ++s)
            for (int c = 0; c < 4; ++c) {
                if (s == 0 && c == 0) continue;   // done by the restriction into this level
                v.shrink(sf);
                for_sublattice(v, colour_ox(c), colour_oy(c), [&](int i, int j) {
                    const int q = t.loc(i, j);
                    u[q] = op.relaxed(f, u, q, i, j);
                });
                __syncthreads();
            }
        const int rx1 = min(sf, 2 * t.I1 + 1), ry1 = min(sf, 2 * t.J1 + 1);
        const int rw = 2 * (t.I1 - t.I0) + 1;
        for_rect(t.ox0, rx1, t.oy0, ry1, [&](int i, int j) {
            r[(j - t.oy0) * rw + (i - t.ox0)] = op.resid(f, u, t.loc(i, j), i, j);
        });
        __syncthreads();
        tile_restrict<T, W>(t, r, rw, L, C, zero_uc);
        for_rect(t.ox0, t.ox1, t.oy0, t.oy1, [&](int i, int j) { gu[(size_t)j * sf + i] = u[t.loc(i, j)]; });
        __syncthreads();
    }
}

// Up leg of a coarse level l: prolongation from l + 1, post-smoothing.
template <typename T, typename W>
__device__ __noinline__ void tile_up(const SolveArgs& a, int l, char* smem, int worker, int nworkers) {
    const LevelArgs& L = a.L[l];
    const LevelArgs& C = a.L[l + 1];
    const int sf = L.side, sc = L.sc, nu = a.nu2c;
    const int H = 4 * nu;
    const int tc = a.tc[l];
    const int ntiles = tile_count(tc, sc);
    const W* gA = (const W*)L.A;
    const W* gP = (const W*)L.P;
    const T* guc = (const T*)(l + 1 == a.tail ? C.u : C.u2);
    const T* gu = (const T*)L.u;   // after the pre-smoothing
    T* gu2 = (T*)L.u2;             // after the post-smoothing (other tiles still read gu)
    const T* gf = (const T*)L.f;
    struct Pt { T u, f, A[9]; };
    for (int k = worker; k < ntiles; k += nworkers) {
        const Tile t = make_tile(k, tc, sc, sf, H);
        const int wh = t.w * t.h;
        T* A = (T*)smem;
        T* u = A + 9 * wh;
        T* f = u + wh;
        batched_rect<2>(
            t.gx0, t.gx1, t.gy0, t.gy1,
            [&](int i, int j) {
                const size_t x = (size_t)j * sf + i;
                Pt p;
                p.u = gu[x] + prolonged<T, W>(gP, guc, sc, i, j);
                p.f = gf[x];
#pragma unroll
                for (int d = 0; d < 9; ++d) p.A[d] = (T)wval(gA[d * L.n + x]);
                return p;
            },
            [&](int i, int j, const Pt& p) {
                const int q = t.loc(i, j);
                u[q] = p.u;
                f[q] = p.f;
#pragma unroll
                for (int d = 0; d < 9; ++d) A[d * wh + q] = p.A[d];
            });
        __syncthreads();
        const T9<T> op{A, sf, t.w, wh};
        Valid v{t.gx0, t.gx1, t.gy0, t.gy1};
        for (int s = 0; s < nu; ++s)
            for (int c = 0; c < 4; ++c) {
                v.shrink(sf);
                for_sublattice(v, colour_ox(c), colour_oy(c), [&](int i, int j) {
                    const int q = t.loc(i, j);
                    u[q] = op.relaxed(f, u, q, i, j);
                });
                __syncthreads();
            }
        for_rect(t.ox0, t.ox1, t.oy0, t.oy1, [&](int i, int j) { gu2[(size_t)j * sf + i] = u[t.loc(i, j)]; });
        __syncthreads();
    }
}

// First post-smoothing colour of the finest level fused with the
// prolongation: a colour-0 point's Gauss-Seidel value needs only its four
// neighbours (colour 1), taken as u + P u_c on the fly; the colour-0 points'
// own prolonged values would be overwritten unread, and the colour-1 points'
// are not needed by the next colour either (it reads only colour 0).
template <typename T, typename W>
__device__ __noinline__ void relax_fine_prolonged(const SolveArgs& a, const T* uc, size_t start,
                                                  size_t stride) {
    const LevelArgs& L = a.L[0];
    const L0Op<T> op{a.K, a.code, L.side};
    T* __restrict__ u = (T*)L.u;
    const T* __restrict__ f = (const T*)L.f;
    const W* P = (const W*)L.P;
    const int side = L.side, sc = L.sc, hs = (side + 1) / 2;
    const unsigned cnt = (unsigned)side * hs, st = (unsigned)stride;
    const FastDiv dv(hs);
    auto nb = [&](int i, int j) -> T {
        return u[(size_t)j * side + i] + prolonged<T, W>(P, uc, sc, i, j);
    };
    for (unsigned t = (unsigned)start; t < cnt; t += st) {
        unsigned r;
        const int j = (int)dv.divmod(t, &r), i = (j & 1) + 2 * (int)r;
        if (i >= side) continue;
        const T uW = i > 0 ? nb(i - 1, j) : T(0);
        const T uE = i + 1 < side ? nb(i + 1, j) : T(0);
        const T uS = j > 0 ? nb(i, j - 1) : T(0);
        const T uN = j + 1 < side ? nb(i, j + 1) : T(0);
        u[(size_t)j * side + i] = op.relaxed_nb(f, i, j, uW, uE, uS, uN);
    }
}

// u_0 += P u_1 at the finest level's colour-1 points (its edge points) only:
// the colour-0 values are overwritten, unread, by the relaxation that follows.
template <typename T, typename W>
__device__ __noinline__ void prolong_colour1(const SolveArgs& a, const T* uc, size_t start, size_t stride) {
    const LevelArgs& L = a.L[0];
    T* __restrict__ u = (T*)L.u;
    const W* P = (const W*)L.P;
    const int side = L.side, sc = L.sc, hs = (side + 1) / 2;
    const unsigned cnt = (unsigned)side * hs, st = (unsigned)stride;
    const FastDiv dv(hs);
    constexpr int K = 4;
    unsigned t = (unsigned)start;
    for (; t + (K - 1) * st < cnt; t += K * st) {
        int i[K], j[K];
        T val[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            unsigned r;
            j[k] = (int)dv.divmod(t + k * st, &r);
            i[k] = ((j[k] + 1) & 1) + 2 * (int)r;
            val[k] = i[k] < side ? u[(size_t)j[k] * side + i[k]] + prolonged<T, W>(P, uc, sc, i[k], j[k]) : T(0);
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (i[k] < side) u[(size_t)j[k] * side + i[k]] = val[k];
    }
    for (; t < cnt; t += st) {
        unsigned r;
        const int j = (int)dv.divmod(t, &r), i = ((j + 1) & 1) + 2 * (int)r;
        if (i < side) u[(size_t)j * side + i] += prolonged<T, W>(P, uc, sc, i, j);
    }
}

// Where level l's values after its post-smoothing are, in the tiled kernel:
// u2 for a tiled level (its neighbours stage u while it writes), u for the
// tail's top level and for the large coarse levels relaxed one phase per colour.
__device__ __forceinline__ const void* final_u(const SolveArgs& a, int l) {
    return l == a.tail || l < a.tile_from ? a.L[l].u : a.L[l].u2;
}

// The tail's V-cycle and the grid-wide phases of the finest level as calls of
// their own (the tiled kernel's register budget is that of two blocks per SM).
template <typename T, typename W>
__device__ __noinline__ void tail_vcycle(const SolveArgs& a, const LevelArgs* tl, const double* inv) {
    block_vcycle<T, W>(a, tl, inv, a.tail, true);
}
template <typename T, typename W>
__device__ __noinline__ void fine_relax(const SolveArgs& a, int c, bool zero, size_t gt, size_t gs) {
    relax_level<T, W>(a, a.L[0], 0, c, zero, gt, gs);
}
template <typename T, typename W>
__device__ __noinline__ void fine_restrict(const SolveArgs& a, size_t gt, size_t gs) {
    restrict_level<T, W>(a, a.L[0], a.L[1], 0, 1 < a.tail && 1 < a.nlev - 1 && sweeps_pre(a, 1) > 0, gt, gs);
}
// One colour of a large coarse level l (first sweep's first colour excluded:
// the restriction into l did it), its restriction into l + 1, and the
// prolongation into it from l + 1.
template <typename T, typename W>
__device__ __noinline__ void coarse_relax(const SolveArgs& a, int l, int c, size_t gt, size_t gs) {
    relax_level<T, W>(a, a.L[l], l, c, false, gt, gs);
}
template <typename T, typename W>
__device__ __noinline__ void coarse_restrict(const SolveArgs& a, int l, size_t gt, size_t gs) {
    restrict_level<T, W>(a, a.L[l], a.L[l + 1], l,
                         l + 1 < a.tail && l + 1 < a.nlev - 1 && sweeps_pre(a, l + 1) > 0, gt, gs);
}
template <typename T, typename W>
__device__ __noinline__ void coarse_prolong(const SolveArgs& a, int l, size_t gt, size_t gs) {
    LevelArgs C = a.L[l + 1];
    C.u = (void*)final_u(a, l + 1);
    prolong_phase<T, W>(a.L[l], C, gt, gs);
}
__device__ __noinline__ void fine_check(const SolveArgs& a, int slot, size_t gt, size_t gs) {
    check_phase(a, slot, gt, gs);
}
__device__ __noinline__ void fine_update(const SolveArgs& a, int c, size_t gt, size_t gs) {
    relax_fine_update(L0Op<float>{a.K, a.code, a.L[0].side}, a.L[0], a.v, c, gt, gs);
}

// V-cycles with tiled grid-wide levels; block 0 stages and runs the tail.
template <typename T, typename W>
__global__ void __launch_bounds__(kMGThreads, 2) k_mg_cycles_tiled(const __grid_constant__ SolveArgs a) {
    extern __shared__ __align__(16) char smem_t[];
    __shared__ LevelArgs tl[kMaxLevels];
    const GridSync G{a.bar, gridDim.x};
    const int worker = (int)blockIdx.x - 1, nworkers = (int)gridDim.x - 1;
    const size_t gt = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gs = (size_t)gridDim.x * blockDim.x;
    if (!G.sync()) return;   // set-up complete (and error state shared)
    prof_mark(8000);
    double* inv = a.inv;
    int slot = 0;
    // block 0 stages the tail while the others take the first residual check
    if (blockIdx.x == 0) stage_tail<T, W>(a, smem_t, tl, &inv);
    else fine_check(a, slot, gt - blockDim.x, gs - blockDim.x);
    prof_done(6000);
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
            slow = res > 0.5 * prev ? slow + 1 : 0;
            if (!reason && slow >= 2 && res < 1e-12 * fmax(vm, 1e-300)) reason = 1;
            if (!reason && res <= a.rel_tol * res0) reason = 2;
            prev = fmin(prev, res);
        } else {
            prev = res;
        }
        if (!reason && cycles >= a.max_cycles) reason = 3;
        if (reason) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                a.out->cycles = cycles;
                a.out->reason = reason;
                a.out->res = res;
                a.out->vmax_final = vm;
            }
            return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.out->rmax[slot ^ 1] = 0ull;
            a.out->vmax[slot ^ 1] = 0ull;
        }
        {
            // finest level, one phase per colour: pre-smoothing (the first
            // colour from the zero start was done by the residual check in
            // the mixed path), then the restriction
            const bool z = a.mixed != 0;
            const bool done0 = z && fine_colour0_in_check(a);
            for (int k = 0; k < a.nu1; ++k)
                for (int c = 0; c < 2; ++c) {
                    if (done0 && k == 0 && c == 0) continue;
                    fine_relax<T, W>(a, c, z && k == 0 && c == 0, gt, gs);
                    prof_done(1000 + c);
                    if (!G.sync()) return;
                    prof_mark(1000 + c);
                }
            fine_restrict<T, W>(a, gt, gs);
            prof_done(2000);
            if (!G.sync()) return;
            prof_mark(2000);
        }
        for (int l = 1; l < a.tail; ++l) {
            if (l < a.tile_from) {
                // a large coarse level, one phase per colour: its first colour
                // from the zero start came with the restriction into it
                for (int k = 0; k < a.nu1c; ++k)
                    for (int c = 0; c < 4; ++c) {
                        if (k == 0 && c == 0) continue;
                        coarse_relax<T, W>(a, l, c, gt, gs);
                        if (!G.sync()) return;
                        prof_mark(1000 + 10 * l + c);
                    }
                coarse_restrict<T, W>(a, l, gt, gs);
            } else if (worker >= 0) {
                tile_down<T, W>(a, l, smem_t, worker, nworkers);
            }
            prof_done(2000 + 10 * l);
            if (!G.sync()) return;
            prof_mark(2000 + 10 * l);
        }
        if (blockIdx.x == 0) tail_vcycle<T, W>(a, tl, inv);
        prof_done(4000);
        if (!G.sync()) return;
        prof_mark(4000);
        for (int l = a.tail - 1; l >= 1; --l) {
            if (l < a.tile_from) {
                coarse_prolong<T, W>(a, l, gt, gs);
                if (!G.sync()) return;
                prof_mark(3000 + 10 * l);
                for (int k = 0; k < a.nu2c; ++k)
                    for (int c = 0; c < 4; ++c) {
                        coarse_relax<T, W>(a, l, c, gt, gs);
                        if (!G.sync()) return;
                        prof_mark(1500 + 10 * l + c);
                    }
                continue;
            }
            if (worker >= 0) tile_up<T, W>(a, l, smem_t, worker, nworkers);
            prof_done(3000 + 10 * l);
            if (!G.sync()) return;
            prof_mark(3000 + 10 * l);
        }
        slot ^= 1;
        // finest level, one phase per colour: the prolongation folded into
        // the first post-smoothing colour, the float64 update v += e into the
        // last (mixed path), then the residual check
        const T* uc = (const T*)final_u(a, 1);
        if (a.nu2 == 0) {
            LevelArgs C = a.L[1];
            C.u = (void*)uc;
            prolong_phase<T, W>(a.L[0], C, gt, gs);
            if (!G.sync()) return;
            if (a.mixed) {
                axpy_phase(a, gt, gs);
                if (!G.sync()) return;
            }
        }
        for (int k = 0; k < a.nu2; ++k)
            for (int c = 0; c < 2; ++c) {
                if (k == 0 && c == 0 && a.tile_from > 1) {
                    // large grids: the colour-1 points' prolongation in a phase
                    // of its own (each is added once, not once per neighbour),
                    // then a plain colour-0 relaxation
                    prolong_colour1<T, W>(a, uc, gt, gs);
                    if (!G.sync()) return;
                    prof_mark(1090);
                    fine_relax<T, W>(a, 0, false, gt, gs);
                } else if (k == 0 && c == 0) {
                    relax_fine_prolonged<T, W>(a, uc, gt, gs);
                } else {
                    bool done = false;
                    if constexpr (sizeof(T) == 4) {
                        if (k == a.nu2 - 1 && c == 1) {
                            fine_update(a, c, gt, gs);
                            done = true;
                        }
                    }
                    if (!done) fine_relax<T, W>(a, c, false, gt, gs);
                }
                prof_done(1100 + 10 * k + c);
                if (!G.sync()) return;
                prof_mark(1100 + 10 * k + c);
            }
        fine_check(a, slot, gt, gs);
        prof_done(6000);
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

// The tiled cycle kernel of a precision kind (0 float32, 1 float64, 2 bfloat16 weights).
const void* tiled_kernel(int kind) {
    return kind == 1   ? (const void*)k_mg_cycles_tiled<double, double>
           : kind == 2 ? (const void*)k_mg_cycles_tiled<float, __nv_bfloat16>
                       : (const void*)k_mg_cycles_tiled<float, float>;
}

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
        for (int kind = 0; kind < 3; ++kind)
            GS_CUDA(cudaFuncSetAttribute(tiled_kernel(kind), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kTiledSmemMax));
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

// Tiles of the largest tiled phase (the grid needs one more block: block 0 runs the tail).
int tiled_max_tiles(const SolveArgs& a) {
    auto tiles = [](int tc, int sc) {
        const int nt = (sc + tc - 1) / tc;
        return nt * nt;
    };
    int m = 0;
    for (int l = std::max(1, a.tile_from); l < a.tail; ++l) m = std::max(m, tiles(a.tc[l], a.L[l].sc));
    return m;
}

}  // namespace

size_t tiled_smem_bytes(const SolveArgs& a) {
    const size_t T = a.mixed ? 4 : 8;
    auto side = [](int tc, int sc, int sf, int H) {
        return (size_t)std::min(sf, 2 * std::min(tc, sc) + 1 + 2 * H);
    };
    size_t need = tail_smem_bytes(a);
    for (int l = std::max(1, a.tile_from); l < a.tail; ++l) {
        const LevelArgs& L = a.L[l];
        const int K1 = a.nu1c > 0 ? 4 * a.nu1c - 1 : 0;
        const size_t wd = side(a.tc[l], L.sc, L.side, 1 + K1);
        const size_t rw = 2 * (size_t)std::min(a.tc[l], L.sc) + 1;
        need = std::max(need, 11 * T * wd * wd + rw * rw * T);
        const size_t wu = side(a.tc[l], L.sc, L.side, 4 * a.nu2c);
        need = std::max(need, 11 * T * wu * wu);
    }
    return need;
}

void set_tile_sides(SolveArgs& a, int workers) {
    a.tc[0] = 0;   // the finest level is not tiled (one grid-wide phase per colour)
    // coarse levels: about one tile per worker block, at least 2 x 2 points
    // of the next level, at most 16 x 16 (8 x 8 in float64: shared memory)
    int root = 1;
    while ((root + 1) * (root + 1) <= std::max(1, workers)) ++root;
    const int cap = a.mixed ? 16 : 8;
    for (int l = 1; l < kMaxLevels; ++l) {
        const int sc = l < a.nlev ? a.L[l].sc : 1;
        a.tc[l] = std::max(2, std::min(cap, (sc + root - 1) / root));
    }
}

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
    if (a.tiled) {
        const int kind = !a.mixed ? 1 : a.wbf16 ? 2 : 0;
        const size_t smem = tiled_smem_bytes(a);
        int per_sm = 0;
        GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tiled_kernel(kind), kMGThreads,
                                                              smem));
        // one block per tile of the largest tiled level (plus block 0), the
        // whole GPU when a large coarse level runs grid-wide phases
        int nb = std::max(1, per_sm) * o.sms;
        if (a.tile_from <= 1) nb = std::min(nb, 1 + tiled_max_tiles(a));
        if (a.max_blocks > 0) nb = std::min(nb, a.max_blocks);
        nb = std::max(nb, 2);
        GS_CUDA(cudaLaunchCooperativeKernel(tiled_kernel(kind), dim3(nb), dim3(kMGThreads), args, smem,
                                            st));
        note_launches(1);
        return;
    }
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
