// Finite games given by explicit transition tables (Sec. 2): validation and
// set-up of the CSR tables, and a persistent kernel in which each thread block
// takes games from a queue and runs the whole policy iteration on one game
// (Algorithm 2 with Algorithm 1 inside) -- improvement, assembly, multigrid
// policy evaluation, stopping tests -- with the game's vectors in shared memory.
//
// Multigrid for the policy-fixed system (I - mu M) w = r of a general game: the
// smoother is Jacobi relaxation; the coarse space is spanned by the constant
// vector, whose Galerkin operator is 1^T A 1 = sum of A's row sums.  For a
// stochastic M the constant vector is the slow mode of I - mu M (eigenvalue
// 1 - mu), which relaxation cannot remove and the coarse correction removes
// exactly; the other modes contract at the rate of M's second eigenvalue.
#include <algorithm>
#include <cfloat>

#include "games.cuh"
#include "gridsync.cuh"

namespace gs {

namespace {

constexpr int kThreads = 512;

// ------------------------------------------------------------------ validation
__global__ void k_game_validate(GameTables T, int count, const int64_t* __restrict__ st_off,
                                int* __restrict__ bad) {
    const int64_t R = (int64_t)T.m1 * T.m2;
    const int64_t rows = st_off[count] * R;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
         row += (int64_t)gridDim.x * blockDim.x) {
        // game of this row: binary search over the state offsets
        const int64_t x = row / R;
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (st_off[mid] <= x) lo = mid;
            else hi = mid - 1;
        }
        const int64_t n = st_off[lo + 1] - st_off[lo];
        const int64_t k0 = T.row_ptr[row], k1 = T.row_ptr[row + 1];
        int err = 0;
        if (k1 < k0) err |= 1;
        double sum = 0.0;
        for (int64_t k = k0; k < k1 && !(err & 1); ++k) {
            const int32_t c = T.col[k];
            const double p = T.prob[k];
            if (c < 0 || c >= n) err |= 2;
            if (!(p >= 0.0) || !(p <= 1.0)) err |= 4;
            sum += p;
        }
        if (sum > 1.0 + 1e-12) err |= 8;
        if (!(fabs(T.rew[row]) <= DBL_MAX)) err |= 16;
        if (k1 - k0 != T.row_ptr[1] - T.row_ptr[0]) err |= 32;   // rows of unequal length (allowed)
        if (err) atomicOr(bad, err);
    }
}

// Per row: leakage 1 - mu sum_k p_k (float64) and the float32 or bfloat16 copy of p.
__global__ void k_game_prepare(GameTables T, int count, const int64_t* __restrict__ st_off,
                               const double* __restrict__ mu, double* __restrict__ leak,
                               float* __restrict__ leak32, float* __restrict__ prob32,
                               __nv_bfloat16* __restrict__ prob16) {
    const int64_t R = (int64_t)T.m1 * T.m2;
    const int64_t rows = st_off[count] * R;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = row / R;
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (st_off[mid] <= x) lo = mid;
            else hi = mid - 1;
        }
        double sum = 0.0;
        for (int64_t k = T.row_ptr[row]; k < T.row_ptr[row + 1]; ++k) {
            sum += T.prob[k];
            if (prob16) prob16[k] = __double2bfloat16(T.prob[k]);
            else prob32[k] = (float)T.prob[k];
        }
        leak[row] = 1.0 - mu[lo] * sum;
        leak32[row] = (float)leak[row];
    }
}

// ------------------------------------------------------------------ block helpers
__device__ __forceinline__ double warp_maxd(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide reductions; every thread gets the result.  `red` is shared scratch.
__device__ double block_max(double v, double* red) {
    v = warp_maxd(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    return m;
}
template <typename T>
__device__ T block_sum(T v, T* red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    T s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];   // fixed order
    return s;
}

// ------------------------------------------------------------------ one game
// Transition probability k rounded to float32 (the screen's error bound
// assumes float32 rounding: with bfloat16 storage it rounds the float64 value).
__device__ __forceinline__ float prob_at_f(const GameTables& tb, int64_t k) {
    return tb.prob16 ? f64_to_f32(tb.prob[k]) : tb.prob32[k];
}

struct Game {
    GameTables T;
    int64_t x0, n, row0;   // first state, states, first row
    double mu;
    float mu_f;            // mu rounded to float32
    int R;                 // m1 * m2
};

// sum_k p_k v(col_k) over a row, v indexed locally.  Two partial sums: a
// float64 operation's latency is 64 cycles here.
__device__ __forceinline__ double row_sum(const Game& G, int64_t row, const double* v) {
    int64_t k0, k1;
    row_range(G.T, row, &k0, &k1);
    double s0 = 0.0, s1 = 0.0;
    int64_t k = k0;
    for (; k + 1 < k1; k += 2) {
        s0 = fma(G.T.prob[k], v[G.T.col[k]], s0);
        s1 = fma(G.T.prob[k + 1], v[G.T.col[k + 1]], s1);
    }
    if (k < k1) s0 = fma(G.T.prob[k], v[G.T.col[k]], s0);
    return s0 + s1;
}

// F(v; x, a, b) = mu sum_k p_k v(col_k) + r(x, a, b)  (Eq. (ILPI)).
__device__ __forceinline__ double row_value(const Game& G, int64_t row, const double* v) {
    return G.mu * row_sum(G, row, v) + G.T.rew[row];
}

// The same in float32 from the float32 copies (a screen; |error| <= err_of).
__device__ __forceinline__ float row_value_f(const Game& G, int64_t row, const float* v32) {
    int64_t k0, k1;
    row_range(G.T, row, &k0, &k1);
    float s = 0.0f;
    for (int64_t k = k0; k < k1; ++k) s = fmaf(prob_at_f(G.T, k), v32[G.T.col[k]], s);
    return G.mu_f * s + f64_to_f32(G.T.rew[row]);
}

// The exact float64 decisions for one state (near-ties of the float32 screen).
// Not inlined: the compiler must not evaluate these rows for every state.
__device__ __noinline__ int improve_state_exact(const Game& G, const BatchOut& O, int mode, int64_t i,
                                                double tau, const double* v, double* res) {
    const int m1 = G.T.m1, m2 = G.T.m2;
    const int64_t x = G.x0 + i;
    const int64_t rb = G.row0 + i * G.R;
    const int acur = O.alpha[x];
    double Fa[kGameMaxM1];
    int changed = 0;
    for (int a = 0; a < m1; ++a) {
        if (mode == 1 && a != acur) continue;
        uint8_t& bref = O.beta[x * m1 + a];
        const int bcur = bref;
        double best = 0.0, fcur = 0.0;
        int first = 0;
        for (int b = 0; b < m2; ++b) {
            const double F = row_value(G, rb + a * m2 + b, v);
            if (b == 0 || F < best) { best = F; first = b; }
            if (b == bcur) fcur = F;
        }
        const int bnew = (fcur - best > tau) ? first : bcur;
        if (bnew != bcur) {
            bref = (uint8_t)bnew;
            if (mode == 1) changed = 1;
        }
        Fa[a] = best;
    }
    int anew = acur;
    if (mode == 0) {
        double fmax_ = Fa[0];
        int first = 0;
        for (int a = 1; a < m1; ++a)
            if (Fa[a] > fmax_) { fmax_ = Fa[a]; first = a; }
        anew = (fmax_ - Fa[acur] > tau) ? first : acur;
        changed = anew != acur;
        *res = fabs(fmax_ - v[i]);
        O.alpha[x] = (uint8_t)anew;
    }
    const int64_t row = rb + anew * m2 + O.beta[x * m1 + anew];
    O.sel[x] = row;
    O.rhs[x] = G.T.rew[row];
    return changed;
}

// Policy improvement at local state i (modes as for the Isaacs grid), screened
// in float32: every F(v; x, a, b) is first taken from the float32 copies of p
// and v, within err = 2^-18 (mu |v|_inf + |r|) of its float64 value (float32
// rounding of the inputs and of at most 10 operations, with a wide margin).
// A decision whose best candidate beats the second by more than 2 err + tau
// is the float64 one; otherwise the state takes the exact path.  float64 then
// only evaluates |F(v) - v| for the chosen row (outer mode).
// Returns the number of changed policy entries; *res gets |F(v) - v| (outer).
__device__ int improve_state(const Game& G, const BatchOut& O, int mode, int64_t i, double tau,
                             float tauf, float vmaxf, const double* v, double* res) {
    // games with many MAX actions (fine discretisations of continuous action
    // sets) take the float64 decisions directly
    if (G.T.m1 > kScreenMaxM1) return improve_state_exact(G, O, mode, i, tau, v, res);
    const int m1 = G.T.m1, m2 = G.T.m2;
    const int64_t x = G.x0 + i;
    const int64_t rb = G.row0 + i * G.R;
    const int acur = O.alpha[x];
    const float* v32 = O.v32 + G.x0;
    float Fa[kScreenMaxM1];
    int bsel[kScreenMaxM1];
    bool sure = true;
    for (int a = 0; a < m1 && sure; ++a) {
        if (mode == 1 && a != acur) continue;
        float best = INFINITY, second = INFINITY, rmax = 0.0f;
        int first = 0;
        for (int b = 0; b < m2; ++b) {
            const int64_t row = rb + a * m2 + b;
            const float F = row_value_f(G, row, v32);
            rmax = fmaxf(rmax, fabsf(f64_to_f32(G.T.rew[row])));
            if (F < best) {
                second = best;
                best = F;
                first = b;
            } else if (F < second) {
                second = F;
            }
        }
        const float err = 0x1p-18f * (G.mu_f * vmaxf + rmax);
        sure = m2 == 1 || second - best > 2.0f * err + tauf;
        Fa[a] = best;
        bsel[a] = first;
    }
    int anew = acur;
    if (sure && mode == 0) {
        float g1 = -INFINITY, g2 = -INFINITY;
        int first = 0;
        for (int a = 0; a < m1; ++a) {
            if (Fa[a] > g1) {
                g2 = g1;
                g1 = Fa[a];
                first = a;
            } else if (Fa[a] > g2) {
                g2 = Fa[a];
            }
        }
        float rmax = 0.0f;
        for (int r = 0; r < G.R; ++r) rmax = fmaxf(rmax, fabsf(f64_to_f32(G.T.rew[rb + r])));
        const float err = 0x1p-18f * (G.mu_f * vmaxf + rmax);
        sure = m1 == 1 || g1 - g2 > 2.0f * err + tauf;
        anew = first;
    }
    if (!sure) return improve_state_exact(G, O, mode, i, tau, v, res);
    int changed = 0;
    for (int a = 0; a < m1; ++a) {
        if (mode == 1 && a != acur) continue;
        uint8_t& bref = O.beta[x * m1 + a];
        if (bref != bsel[a]) {
            bref = (uint8_t)bsel[a];
            if (mode == 1) changed = 1;
        }
    }
    const int64_t row = rb + anew * m2 + O.beta[x * m1 + anew];
    if (mode == 0) {
        changed = anew != acur;
        *res = fabs(row_value(G, row, v) - v[i]);
        O.alpha[x] = (uint8_t)anew;
    }
    O.sel[x] = row;
    O.rhs[x] = G.T.rew[row];
    return changed;
}

// Transition probability k in the relaxation's precision.
template <typename T>
__device__ __forceinline__ T prob_at(const GameTables& tb, int64_t k) {
    if constexpr (sizeof(T) == 8) return tb.prob[k];
    else return tb.prob16 ? __bfloat162float(tb.prob16[k]) : tb.prob32[k];
}

// (A e)_i and the diagonal of A = I - mu M for the selected row, leakage form:
// (A e)_i = s_i e_i + mu sum_k p_k (e_i - e_col), s_i = 1 - mu sum_k p_k.
template <typename T>
__device__ __forceinline__ void apply_row(const Game& G, const BatchOut& O, int64_t i, const T* e,
                                          T* Ae, T* diag) {
    const int64_t row = O.sel[G.x0 + i];
    const T ei = e[i];
    const T mu = sizeof(T) == 4 ? (T)G.mu_f : (T)G.mu;
    const T leak = sizeof(T) == 4 ? (T)G.T.leak32[row] : (T)G.T.leak[row];
    T acc = leak * ei, off = 0;
    int64_t k0, k1;
    row_range(G.T, row, &k0, &k1);
    for (int64_t k = k0; k < k1; ++k) {
        const int32_t c = G.T.col[k];
        const T p = prob_at<T>(G.T, k);
        acc += mu * p * (ei - e[c]);
        if (c != i) off += mu * p;
    }
    *Ae = acc;
    *diag = leak + off;
}

// Diagonal of A for the selected row: s_i + mu sum_{k: col_k != i} p_k.
template <typename T>
__device__ __forceinline__ T diag_row(const Game& G, const BatchOut& O, int64_t i) {
    const int64_t row = O.sel[G.x0 + i];
    const T mu = sizeof(T) == 4 ? (T)G.mu_f : (T)G.mu;
    T off = 0;
    int64_t k0, k1;
    row_range(G.T, row, &k0, &k1);
    for (int64_t k = k0; k < k1; ++k)
        if (G.T.col[k] != i) off += mu * prob_at<T>(G.T, k);
    return (sizeof(T) == 4 ? (T)G.T.leak32[row] : (T)G.T.leak[row]) + off;
}

// The same row operations on the slot-major copy of the selected rows (same
// entries, same order: the same arithmetic).
// (KC > 0: rows of exactly KC entries, known at compile time, so that a
// row's loads are issued together; KC = 0: S.K at run time.)
template <int KC>
__device__ __forceinline__ double row_sum_c(const Compact& S, int64_t n, int64_t i, const double* v) {
    const int K = KC > 0 ? KC : S.K;
    double s0 = 0.0, s1 = 0.0;
    int k = 0;
#pragma unroll
    for (; k + 1 < K; k += 2) {
        s0 = fma(S.p64[k * n + i], v[S.col[k * n + i]], s0);
        s1 = fma(S.p64[(k + 1) * n + i], v[S.col[(k + 1) * n + i]], s1);
    }
    if (k < K) s0 = fma(S.p64[k * n + i], v[S.col[k * n + i]], s0);
    return s0 + s1;
}
template <typename T, int KC>
__device__ __forceinline__ void apply_row_c(const Game& G, const Compact& S, int64_t i, const T* e, T* Ae,
                                            T* diag) {
    const int K = KC > 0 ? KC : S.K;
    const int64_t n = G.n;
    const T ei = e[i];
    const T mu = sizeof(T) == 4 ? (T)G.mu_f : (T)G.mu;
    const T leak = sizeof(T) == 4 ? (T)S.leak32[i] : (T)S.leak64[i];
    T acc = leak * ei, off = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int32_t c = S.col[k * n + i];
        const T p = sizeof(T) == 4 ? (T)S.p32[k * n + i] : (T)S.p64[k * n + i];
        acc += mu * p * (ei - e[c]);
        if (c != i) off += mu * p;
    }
    *Ae = acc;
    *diag = leak + off;
}
template <typename T, int KC>
__device__ __forceinline__ T diag_row_c(const Game& G, const Compact& S, int64_t i) {
    const int K = KC > 0 ? KC : S.K;
    const int64_t n = G.n;
    const T mu = sizeof(T) == 4 ? (T)G.mu_f : (T)G.mu;
    T off = 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
        if (S.col[k * n + i] != i) off += mu * (sizeof(T) == 4 ? (T)S.p32[k * n + i] : (T)S.p64[k * n + i]);
    return (sizeof(T) == 4 ? (T)S.leak32[i] : (T)S.leak64[i]) + off;
}

// Execution context of one game's policy iteration: which threads share the
// work, how they synchronise, and where the correction vectors live.  The
// block context runs a game inside one thread block (vectors in shared
// memory); the grid context spreads one game over a cooperative grid (vectors
// in global memory, bounded grid barriers, reductions through per-block
// partials combined in a fixed order, so the result does not depend on timing).
template <typename T>
struct BlockCtx {
    T *r, *e, *t;      // correction right-hand side, correction, Jacobi work vector
    double* red_d;
    int* red_i;
    Compact cp{};      // not used: the rows are read in place
    __device__ size_t begin() const { return threadIdx.x; }
    __device__ size_t stride() const { return blockDim.x; }
    __device__ bool sync() { __syncthreads(); return true; }
    __device__ double max(double v) { return block_max(v, red_d); }
    __device__ double sum(double v) { return block_sum(v, red_d); }
    __device__ int sumi(int v) { return block_sum(v, red_i); }
    __device__ bool failed() const { return false; }
    __device__ bool leader() const { return threadIdx.x == 0; }
};

template <typename T>
struct GridCtx {
    T *r, *e, *t;
    double* part;      // [2][gridDim.x] per-block partials (alternating)
    GridBarrier* bar;
    Compact cp;        // slot-major selected rows (cp.col null: rows read in place)
    double* red_d;
    int flip;
    bool bad;
    __device__ size_t begin() const { return (size_t)blockIdx.x * blockDim.x + threadIdx.x; }
    __device__ size_t stride() const { return (size_t)gridDim.x * blockDim.x; }
    __device__ bool sync() {
        if (!bad) bad = !GridSync{bar, gridDim.x}.sync();
        return !bad;
    }
    __device__ double combine(double v, bool is_max) {
        v = is_max ? block_max(v, red_d) : block_sum(v, red_d);
        double* P = part + (size_t)flip * gridDim.x;
        flip ^= 1;
        if (threadIdx.x == 0) P[blockIdx.x] = v;
        if (!sync()) return 0.0;
        double acc = 0.0;
        for (unsigned k = threadIdx.x & 31; k < gridDim.x; k += 32) {
            const double p = __ldcg(P + k);
            acc = is_max ? fmax(acc, p) : acc + p;
        }
        return is_max ? warp_maxd(acc) : warp_sum(acc);
    }
    __device__ double max(double v) { return combine(v, true); }
    __device__ double sum(double v) { return combine(v, false); }
    __device__ int sumi(int v) { return (int)combine((double)v, false); }
    __device__ bool failed() const { return bad; }
    __device__ bool leader() const { return blockIdx.x == 0 && threadIdx.x == 0; }
};

// float64 residual rhs - (v - mu M v) -> C.r; returns |r|_inf, sets *vmax.
// With jacobi0, also the correction's first Jacobi sweep from zero,
// e = r / diag -> C.e (the V(1,1) cycle below starts from it).
template <typename T, class Ctx>
__device__ double check(const Game& G, const BatchOut& O, const double* v, Ctx& C, double* vmax,
                        bool jacobi0 = false) {
    // maxima on the bit patterns, conversions on the integer pipe
    unsigned long long rm = 0, vm = 0;
    const int cpt = C.cp.col == nullptr ? 0 : C.cp.K == 8 ? 2 : 1;   // 2: rows of 8 entries
    for (int64_t i = C.begin(); i < G.n; i += C.stride()) {
        const double Mv = cpt == 2   ? row_sum_c<8>(C.cp, G.n, i, v)
                          : cpt == 1 ? row_sum_c<0>(C.cp, G.n, i, v)
                                     : row_sum(G, O.sel[G.x0 + i], v);
        const double r = O.rhs[G.x0 + i] - (v[i] - G.mu * Mv);
        T rt;
        if constexpr (sizeof(T) == 4) rt = f64_to_f32(r);
        else rt = r;
        C.r[i] = rt;
        if (jacobi0)
            C.e[i] = rt / (cpt == 2   ? diag_row_c<T, 8>(G, C.cp, i)
                           : cpt == 1 ? diag_row_c<T, 0>(G, C.cp, i)
                                      : diag_row<T>(G, O, i));
        const unsigned long long rb = bits_of(r) & 0x7fffffffffffffffull;
        const unsigned long long vb = bits_of(v[i]) & 0x7fffffffffffffffull;
        rm = rb > rm ? rb : rm;
        vm = vb > vm ? vb : vm;
    }
    *vmax = C.max(from_bits(vm));
    return C.max(from_bits(rm));
}

// One two-level cycle on A e = r from e = 0, then v += e.  Returns false if a
// grid barrier gave up.
template <typename T, class Ctx>
__device__ bool cycle(const Game& G, const BatchOut& O, double* v, Ctx& C, T asum, int nu1, int nu2) {
    // pre-relaxation (Jacobi; the first sweep from zero)
    for (int k = 0; k < nu1; ++k) {
        for (int64_t i = C.begin(); i < G.n; i += C.stride()) {
            if (k == 0) {
                C.t[i] = C.r[i] / diag_row<T>(G, O, i);
            } else {
                T Ae, d;
                apply_row<T>(G, O, i, C.e, &Ae, &d);
                C.t[i] = C.e[i] + (C.r[i] - Ae) / d;
            }
        }
        if (!C.sync()) return false;
        T* sw = C.e; C.e = C.t; C.t = sw;
    }
    if (nu1 == 0) {
        for (int64_t i = C.begin(); i < G.n; i += C.stride()) C.e[i] = 0;
        if (!C.sync()) return false;
    }
    // coarse correction on the constant vector: e += (1^T (r - A e)) / (1^T A 1)
    double part = 0.0;
    for (int64_t i = C.begin(); i < G.n; i += C.stride()) {
        T Ae, d;
        apply_row<T>(G, O, i, C.e, &Ae, &d);
        if constexpr (sizeof(T) == 4) part += f32_to_f64(C.r[i] - Ae);
        else part += (double)(C.r[i] - Ae);
    }
    const double tot = C.sum(part);
    if (C.failed()) return false;
    const T c = asum != T(0) ? (T)(tot / (double)asum) : T(0);
    for (int64_t i = C.begin(); i < G.n; i += C.stride()) C.e[i] += c;
    if (!C.sync()) return false;
    // post-relaxation
    for (int k = 0; k < nu2; ++k) {
        for (int64_t i = C.begin(); i < G.n; i += C.stride()) {
            T Ae, d;
            apply_row<T>(G, O, i, C.e, &Ae, &d);
            C.t[i] = C.e[i] + (C.r[i] - Ae) / d;
        }
        if (!C.sync()) return false;
        T* sw = C.e; C.e = C.t; C.t = sw;
    }
    float* v32 = O.v32 + G.x0;
    for (int64_t i = C.begin(); i < G.n; i += C.stride()) {
        double vi = v[i];
        if constexpr (sizeof(T) == 4) vi += f32_to_f64(C.e[i]);
        else vi += C.e[i];
        v[i] = vi;
        v32[i] = f64_to_f32(vi);
    }
    return C.sync();
}

// The same two-level cycle for one Jacobi sweep before and after the coarse
// correction, in two passes over the rows (the first sweep e1 = r / diag came
// with the residual check): A e1 gives the coarse correction c (e2 = e1 + c)
// and, since A 1 is the leakage s of each row, A e2 = A e1 + c s without
// another product; the post-sweep e = e2 + (r - A e2) / diag and v += e close
// the cycle.  Same iteration as cycle() with nu1 = nu2 = 1.
template <typename T, class Ctx>
__device__ bool cycle11(const Game& G, const BatchOut& O, double* v, Ctx& C, T asum) {
    const int cpt = C.cp.col == nullptr ? 0 : C.cp.K == 8 ? 2 : 1;   // 2: rows of 8 entries
    double part = 0.0;
    for (int64_t i = C.begin(); i < G.n; i += C.stride()) {
        T Ae, d;
        if (cpt == 2) apply_row_c<T, 8>(G, C.cp, i, C.e, &Ae, &d);
        else if (cpt == 1) apply_row_c<T, 0>(G, C.cp, i, C.e, &Ae, &d);
        else apply_row<T>(G, O, i, C.e, &Ae, &d);
        const T q = C.r[i] - Ae;
        if constexpr (sizeof(T) == 4) part += f32_to_f64(q);
        else part += (double)q;
        C.r[i] = q;   // r - A e1 (r itself is not needed again)
        C.t[i] = d;
    }
    const double tot = C.sum(part);
    if (C.failed()) return false;
    const T c = asum != T(0) ? (T)(tot / (double)asum) : T(0);
    float* v32 = O.v32 + G.x0;
    for (int64_t i = C.begin(); i < G.n; i += C.stride()) {
        T s;
        if (cpt) {
            s = sizeof(T) == 4 ? (T)C.cp.leak32[i] : (T)C.cp.leak64[i];
        } else {
            const int64_t row = O.sel[G.x0 + i];
            s = sizeof(T) == 4 ? (T)G.T.leak32[row] : (T)G.T.leak[row];
        }
        const T e = C.e[i] + c + (C.r[i] - c * s) / C.t[i];
        double vi = v[i];
        if constexpr (sizeof(T) == 4) vi += f32_to_f64(e);
        else vi += e;
        v[i] = vi;
        v32[i] = f64_to_f32(vi);
    }
    return C.sync();
}

// Why a policy evaluation stopped.
enum { kEvalExact = 0, kEvalInexact = 1, kEvalCapped = 2 };

// Policy evaluation: cycles until the float64 floor / tolerance (kEvalExact),
// a residual drop by rel_tol (kEvalInexact) or max_cycles (kEvalCapped).
template <typename T, class Ctx>
__device__ int evaluate(const Game& G, const BatchOut& O, const BatchOpts& P, double* v, Ctx& C,
                        double rel_tol, int* cycles) {
    const bool v11 = P.nu1 == 1 && P.nu2 == 1;
    if (!v11) C.cp.col = nullptr;   // the general cycle reads the rows in place
    double part = 0.0;
    for (int64_t i = C.begin(); i < G.n; i += C.stride()) {
        const int64_t row = O.sel[G.x0 + i];
        part += G.T.leak[row];
        if (C.cp.col) {   // the selected rows, slot-major
            const Compact& S = C.cp;
            const int64_t k0 = row * S.K;
            for (int k = 0; k < S.K; ++k) {
                S.col[k * G.n + i] = G.T.col[k0 + k];
                S.p64[k * G.n + i] = G.T.prob[k0 + k];
                S.p32[k * G.n + i] = prob_at<float>(G.T, k0 + k);
            }
            S.leak64[i] = G.T.leak[row];
            S.leak32[i] = G.T.leak32[row];
        }
    }
    const T asum = (T)C.sum(part);   // (its barrier also publishes the gathered rows)
    double vm;
    double res = check<T>(G, O, v, C, &vm, v11);
    const double res0 = res;
    double prev = res;
    int slow = 0;
    for (int cyc = 0;; ++cyc) {
        if (C.failed()) return kEvalExact;   // a barrier gave up: the caller leaves
        if (res <= P.lin_tol * fmax(vm, 1e-300) || res == 0.0) return kEvalExact;
        if (cyc > 0) {
            slow = res > 0.5 * prev ? slow + 1 : 0;
            if (slow >= 2 && res < 1e-12 * fmax(vm, 1e-300)) return kEvalExact;
            if (res <= rel_tol * res0) return kEvalInexact;
            prev = fmin(prev, res);
        }
        if (cyc >= P.max_cycles) return kEvalCapped;
        if (!(v11 ? cycle11<T>(G, O, v, C, asum) : cycle<T>(G, O, v, C, asum, P.nu1, P.nu2)))
            return kEvalExact;
        ++*cycles;
        res = check<T>(G, O, v, C, &vm, v11);
    }
}

template <class Ctx>
__device__ int improve_all(const Game& G, const BatchOut& O, int mode, const double* v, Ctx& C,
                           double* res_out) {
    unsigned long long vb = 0;
    for (int64_t i = C.begin(); i < G.n; i += C.stride()) {
        const unsigned long long b = bits_of(v[i]) & 0x7fffffffffffffffull;
        vb = b > vb ? b : vb;
    }
    const double vm = C.max(from_bits(vb));
    const double tau = 1e-13 * fmax(1.0, vm);
    const float tauf = f64_to_f32(tau), vmaxf = f64_to_f32(vm);
    int changed = 0;
    unsigned long long rb = 0;
    for (int64_t i = C.begin(); i < G.n; i += C.stride()) {
        double r = 0.0;
        changed += improve_state(G, O, mode, i, tau, tauf, vmaxf, v, &r);
        const unsigned long long b = bits_of(r);
        rb = b > rb ? b : rb;
    }
    if (res_out) *res_out = C.max(from_bits(rb));
    return C.sumi(changed);
}

// Algorithm 2 with Algorithm 1 inside for game g (see the Isaacs driver for
// the stopping rules and the exact confirmation of inexact evaluations).
template <typename T, class Ctx>
__device__ void solve_game(const BatchArgs& B, int g, Ctx& C) {
    Game G;
    G.T = B.T;
    G.x0 = B.st_off[g];
    G.n = B.st_off[g + 1] - G.x0;
    G.R = B.T.m1 * B.T.m2;
    G.row0 = G.x0 * G.R;
    G.mu = B.mu[g];
    G.mu_f = f64_to_f32(G.mu);
    const BatchOut& O = B.out;
    const BatchOpts& P = B.opt;
    double* v = O.v + G.x0;
    const int a0 = P.default_alpha;
    for (int64_t i = C.begin(); i < G.n; i += C.stride()) {
        v[i] = 0.0;
        O.v32[G.x0 + i] = 0.0f;
        O.alpha[G.x0 + i] = (uint8_t)(a0 < G.T.m1 ? a0 : 0);
        for (int a = 0; a < G.T.m1; ++a) O.beta[(G.x0 + i) * G.T.m1 + a] = 0;
    }
    if (!C.sync()) return;
    improve_all(G, O, 2, v, C, (double*)nullptr);   // MIN's first reply, assembly
    if (!C.sync()) return;
    int outer = 0, systems = 0, cycles = 0, converged = 0;
    bool capped = false;   // an evaluation stopped at max_cycles: no decision may rest on it
    double res = 0.0;
    while (true) {
        for (int j = 0; j < P.max_inner; ++j) {
            const int why = evaluate<T>(G, O, P, v, C, P.pi_rtol, &cycles);
            ++systems;
            if (!C.sync()) return;
            if (why == kEvalCapped) {
                capped = true;
                break;
            }
            if (improve_all(G, O, 1, v, C, (double*)nullptr) != 0) continue;
            if (!C.sync()) return;
            if (why == kEvalInexact) {
                if (evaluate<T>(G, O, P, v, C, 0.0, &cycles) == kEvalCapped) capped = true;
                if (!C.sync()) return;
                if (capped) break;
                if (improve_all(G, O, 1, v, C, (double*)nullptr) != 0) continue;
                if (!C.sync()) return;
            }
            break;
        }
        ++outer;
        if (!C.sync()) return;
        const int ach = improve_all(G, O, 0, v, C, &res);
        if (!C.sync()) return;
        if (capped) break;   // unconverged; v is the best iterate, res its residual
        if (res <= P.eps || ach == 0) {
            converged = 1;
            break;
        }
        if (outer >= P.max_outer) break;
    }
    if (C.leader()) {
        O.gstats[4 * g + 0] = outer;
        O.gstats[4 * g + 1] = systems;
        O.gstats[4 * g + 2] = cycles;
        O.gstats[4 * g + 3] = converged;
        O.gres[g] = res;
    }
    C.sync();
}

// One thread block of NT threads per game; blocks take games from the queue
// in the order B.order gives (512 / NT blocks per SM fit the registers).
template <typename T, int NT>
__global__ void __launch_bounds__(NT, 512 / NT) k_games_pi(const __grid_constant__ BatchArgs B) {
    extern __shared__ __align__(16) char smem[];
    __shared__ int s_game;
    __shared__ double red_d[32];
    __shared__ int red_i[32];
    while (true) {
        if (threadIdx.x == 0) {
            const int q = atomicAdd(B.queue, 1);
            s_game = q < B.count ? B.order[q] : -1;
        }
        __syncthreads();
        const int g = s_game;
        __syncthreads();
        if (g < 0) break;
        BlockCtx<T> C;
        C.r = (T*)smem;
        C.e = C.r + B.max_n;
        C.t = C.e + B.max_n;
        C.red_d = red_d;
        C.red_i = red_i;
        if (B.cp.col) {   // this game's part of the slot-major rows
            const int64_t x0 = B.st_off[g], K = B.cp.K;
            C.cp = Compact{B.cp.col + x0 * K, B.cp.p32 + x0 * K, B.cp.p64 + x0 * K, B.cp.leak32 + x0,
                           B.cp.leak64 + x0, B.cp.K};
        }
        solve_game<T>(B, g, C);
    }
}

// One game over a cooperative grid (games too large for one block).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_game_pi_grid(const __grid_constant__ BatchArgs B,
                                                           GridWork W) {
    __shared__ double red_d[32];
    GridCtx<T> C;
    C.r = (T*)W.r;
    C.e = (T*)W.e;
    C.t = (T*)W.t;
    C.part = W.part;
    C.bar = W.bar;
    C.cp = W.cp;
    C.red_d = red_d;
    C.flip = 0;
    C.bad = false;
    solve_game<T>(B, 0, C);
}

// One policy improvement of game 0 over the whole grid (the algebraic
// multigrid path runs policy iteration from the host): keep-current
// tolerance from |v|_inf (bits at scal + 4), changed entries summed into
// scal[0], |F(v) - v|_inf (outer mode) as bits at scal + 2.
__global__ void k_game_improve_one(const __grid_constant__ BatchArgs B, int mode, int* scal) {
    Game G;
    G.T = B.T;
    G.x0 = 0;
    G.n = B.st_off[1];
    G.R = B.T.m1 * B.T.m2;
    G.row0 = 0;
    G.mu = B.mu[0];
    G.mu_f = f64_to_f32(G.mu);
    const double vm = from_bits(*reinterpret_cast<const unsigned long long*>(scal + 4));
    const double tau = 1e-13 * fmax(1.0, vm);
    const float tauf = f64_to_f32(tau), vmaxf = f64_to_f32(vm);
    int changed = 0;
    unsigned long long rb = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < G.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double r = 0.0;
        changed += improve_state(G, B.out, mode, i, tau, tauf, vmaxf, B.out.v, &r);
        const unsigned long long b = bits_of(r);
        rb = b > rb ? b : rb;
    }
    changed = warp_sum(changed);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, rb, o);
        rb = w > rb ? w : rb;
    }
    if ((threadIdx.x & 31) == 0) {
        if (changed) atomicAdd(scal, changed);
        atomicMax(reinterpret_cast<unsigned long long*>(scal + 2), rb);
    }
}

}  // namespace

void launch_game_improve_one(const BatchArgs& B, int mode, int64_t n, int* scal, cudaStream_t st) {
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
    k_game_improve_one<<<g, 256, 0, st>>>(B, mode, scal);
    GS_CHECK_LAUNCH();
}

void launch_game_validate(const GameTables& T, int count, const int64_t* st_off, int64_t rows,
                          int* bad, cudaStream_t st) {
    const unsigned g = (unsigned)std::min<int64_t>((rows + 255) / 256, 152 * 32);
    k_game_validate<<<std::max(1u, g), 256, 0, st>>>(T, count, st_off, bad);
    GS_CHECK_LAUNCH();
}

void launch_game_prepare(const GameTables& T, int count, const int64_t* st_off, int64_t rows,
                         const double* mu, double* leak, float* leak32, float* prob32,
                         __nv_bfloat16* prob16, cudaStream_t st) {
    const unsigned g = (unsigned)std::min<int64_t>((rows + 255) / 256, 152 * 32);
    k_game_prepare<<<std::max(1u, g), 256, 0, st>>>(T, count, st_off, mu, leak, leak32, prob32, prob16);
    GS_CHECK_LAUNCH();
}

int game_grid_blocks(int64_t n, int cap) {
    static int per_sm = 0, sms = 0;
    if (!per_sm) {
        int dev = 0;
        GS_CUDA(cudaGetDevice(&dev));
        GS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        int a = 0, b = 0;
        GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_game_pi_grid<float>, kThreads, 0));
        GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_game_pi_grid<double>, kThreads, 0));
        per_sm = std::max(1, std::min(a, b));
    }
    int blocks = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)per_sm * sms);
    if (cap > 0) blocks = std::min(blocks, cap);
    return std::max(1, blocks);
}

void launch_game_pi_grid(const BatchArgs& B, const GridWork& W, int blocks, bool mixed,
                         cudaStream_t st) {
    const void* fn = mixed ? (const void*)k_game_pi_grid<float> : (const void*)k_game_pi_grid<double>;
    void* args[] = {(void*)&B, (void*)&W};
    GS_CUDA(cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(kThreads), args, 0, st));
    note_launches(1);
}

size_t games_smem_bytes(int max_n, bool mixed) {
    return (size_t)3 * max_n * (mixed ? sizeof(float) : sizeof(double));
}

void launch_games_pi(const BatchArgs& B, bool mixed, int threads, cudaStream_t st) {
    const size_t smem = games_smem_bytes(B.max_n, mixed);
    const void* fn = threads == 256 ? (mixed ? (const void*)k_games_pi<float, 256>
                                             : (const void*)k_games_pi<double, 256>)
                                    : (mixed ? (const void*)k_games_pi<float, 512>
                                             : (const void*)k_games_pi<double, 512>);
    const int nt = threads == 256 ? 256 : 512;
    GS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, dev = 0, sms = 0;
    GS_CUDA(cudaGetDevice(&dev));
    GS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem));
    const int blocks = std::max(1, std::min(B.count, std::max(1, per_sm) * sms));
    void* args[] = {(void*)&B};
    GS_CUDA(cudaLaunchKernel(fn, dim3(blocks), dim3(nt), args, smem, st));
    note_launches(1);
}

}  // namespace gs
