// Two-sided stopping game on a line (Sec. 6.3, Eq. (exVI2stop)), solved on
// the device by one thread block: policy iteration (Algorithm 2 with
// Algorithm 1 inside, or FAMGpi, Algorithm 4) with every policy-fixed system
// solved by a one-dimensional algebraic multigrid (Galerkin coarse operators,
// C/F relaxation, Algorithm 3), all vectors and the hierarchy in shared memory.
//
// States x_1..x_n (n = 2^k - 1) of a uniform grid with end values v_0, v_{n+1};
// actions 0 = stop, 1 = continue for both players:
//   F(v; x, a, 0) = psi2(x)            MIN stops (also when both stop)
//   F(v; x, 0, 1) = psi1(x)            MAX stops alone
//   F(v; x, 1, 1) = (v(x-1) + v(x+1)) / 2 + c(x)   both continue (mu = 1)
// A grid two times coarser (FAMGpi) carries the same stop values at its points
// and the continuation reward 4 c (c = h^2 r for the generator's reward r).
#include <cstdint>

#include "common.cuh"
#include "line.cuh"

namespace gs {

namespace {

// Row kinds of the policy-fixed system: v = psi2, v = psi1, or continuation.
constexpr uint8_t kRowPsi2 = 0, kRowPsi1 = 1, kRowCont = 2;

struct LineLevel {
    int n;
    double *lo, *di, *up;   // tridiagonal operator (levels >= 1)
    double *u, *f;          // unknown and right-hand side
    double *wl, *wr;        // interpolation weights of the F points (levels < last)
};

struct LineShared {
    LineLevel L[kLineMaxLevels];
    int nlev;
};

// Operator row j of level 0 (implicit in the row kinds).
__device__ __forceinline__ void row0(const uint8_t* kind, int n, int j, double* lo, double* di,
                                     double* up) {
    if (kind[j] == kRowCont) {
        *lo = j > 0 ? -0.5 : 0.0;
        *up = j + 1 < n ? -0.5 : 0.0;
    } else {
        *lo = 0.0;
        *up = 0.0;
    }
    *di = 1.0;
}

__device__ __forceinline__ void row_of(const LineShared& S, const uint8_t* kind, int l, int j,
                                       double* lo, double* di, double* up) {
    if (l == 0) {
        row0(kind, S.L[0].n, j, lo, di, up);
    } else {
        *lo = S.L[l].lo[j];
        *di = S.L[l].di[j];
        *up = S.L[l].up[j];
    }
}

// Galerkin hierarchy of the current policy-fixed system: C points are the odd
// positions j = 2J + 1, an F point j = 2J interpolates from its C neighbours
// with w = -a(j, j -+ 1) / a(j, j), and A_{l+1} = P^T A_l P (tridiagonal).
__device__ void line_setup(LineShared& S, const uint8_t* kind) {
    for (int l = 0; l + 1 < S.nlev; ++l) {
        const LineLevel& F = S.L[l];
        LineLevel& C = S.L[l + 1];
        // weights of the F points 2J, J = 0..nc (nc + 1 of them)
        for (int J = threadIdx.x; J <= C.n; J += blockDim.x) {
            const int j = 2 * J;
            double wl = 0.0, wr = 0.0;
            if (j < F.n) {
                double lo, di, up;
                row_of(S, kind, l, j, &lo, &di, &up);
                if (di != 0.0) {
                    wl = j > 0 ? -lo / di : 0.0;
                    wr = j + 1 < F.n ? -up / di : 0.0;
                }
            }
            F.wl[J] = wl;
            F.wr[J] = wr;
        }
        __syncthreads();
        // coarse row J: fine rows 2J (weight wr of F point 2J), 2J + 1 (1), 2J + 2 (wl of 2J + 2)
        for (int J = threadIdx.x; J < C.n; J += blockDim.x) {
            double acc[3] = {0.0, 0.0, 0.0};   // towards J - 1, J, J + 1
            for (int t = 0; t < 3; ++t) {
                const int i = 2 * J + t;
                const double R = t == 0 ? F.wr[J] : t == 1 ? 1.0 : F.wl[J + 1];
                if (R == 0.0 || i >= F.n) continue;
                double a[3];
                row_of(S, kind, l, i, &a[0], &a[1], &a[2]);
                for (int d = 0; d < 3; ++d) {
                    const int k = i - 1 + d;
                    if (k < 0 || k >= F.n || a[d] == 0.0) continue;
                    const double v = R * a[d];
                    if (k & 1) {                       // C point (k - 1) / 2
                        acc[(k - 1) / 2 - J + 1] += v;
                    } else {                           // F point k = 2K: coarse K - 1 and K
                        const int K = k / 2;
                        if (K - 1 >= 0) acc[K - 1 - J + 1] += v * F.wl[K];
                        if (K < C.n) acc[K - J + 1] += v * F.wr[K];
                    }
                }
            }
            C.lo[J] = J > 0 ? acc[0] : 0.0;
            C.di[J] = acc[1];
            C.up[J] = J + 1 < C.n ? acc[2] : 0.0;
        }
        __syncthreads();
    }
}

// Gauss-Seidel on the points of one parity (C points: odd, F points: even).
__device__ void line_relax(const LineShared& S, const uint8_t* kind, int l, int parity) {
    const LineLevel& L = S.L[l];
    for (int j = 2 * threadIdx.x + parity; j < L.n; j += 2 * blockDim.x) {
        double lo, di, up;
        row_of(S, kind, l, j, &lo, &di, &up);
        double s = L.f[j];
        if (j > 0) s -= lo * L.u[j - 1];
        if (j + 1 < L.n) s -= up * L.u[j + 1];
        L.u[j] = s / di;
    }
    __syncthreads();
}

__device__ __forceinline__ double line_resid(const LineShared& S, const uint8_t* kind, int l, int j) {
    const LineLevel& L = S.L[l];
    double lo, di, up;
    row_of(S, kind, l, j, &lo, &di, &up);
    double Au = di * L.u[j];
    if (j > 0) Au += lo * L.u[j - 1];
    if (j + 1 < L.n) Au += up * L.u[j + 1];
    return L.f[j] - Au;
}

// One V-cycle on level l's system (Algorithm 3, C/F relaxation, gamma = 1).
__device__ void line_vcycle(LineShared& S, const uint8_t* kind, int nu1, int nu2) {
    const int Lc = S.nlev - 1;
    for (int l = 0; l < Lc; ++l) {
        for (int k = 0; k < nu1; ++k) {
            line_relax(S, kind, l, 1);
            line_relax(S, kind, l, 0);
        }
        const LineLevel& F = S.L[l];
        const LineLevel& C = S.L[l + 1];
        for (int J = threadIdx.x; J < C.n; J += blockDim.x) {
            const int i = 2 * J + 1;
            double r = line_resid(S, kind, l, i);
            r += F.wr[J] * line_resid(S, kind, l, i - 1);
            if (i + 1 < F.n) r += F.wl[J + 1] * line_resid(S, kind, l, i + 1);
            C.f[J] = r;
            C.u[J] = 0.0;
        }
        __syncthreads();
    }
    // coarsest: tridiagonal elimination by one thread
    if (threadIdx.x == 0) {
        const LineLevel& L = S.L[Lc];
        double cp[3], dp[3];
        const int n = L.n;
        for (int j = 0; j < n; ++j) {
            double lo, di, up;
            row_of(S, kind, Lc, j, &lo, &di, &up);
            const double m = j > 0 ? di - lo * cp[j - 1] : di;
            cp[j] = m != 0.0 ? up / m : 0.0;
            dp[j] = m != 0.0 ? (L.f[j] - (j > 0 ? lo * dp[j - 1] : 0.0)) / m : 0.0;
        }
        for (int j = n - 1; j >= 0; --j) L.u[j] = dp[j] - (j + 1 < n ? cp[j] * L.u[j + 1] : 0.0);
    }
    __syncthreads();
    for (int l = Lc - 1; l >= 0; --l) {
        const LineLevel& F = S.L[l];
        const LineLevel& C = S.L[l + 1];
        for (int j = threadIdx.x; j < F.n; j += blockDim.x) {
            if (j & 1) {
                F.u[j] += C.u[(j - 1) / 2];
            } else {
                const int J = j / 2;
                double e = 0.0;
                if (J - 1 >= 0) e += F.wl[J] * C.u[J - 1];
                if (J < C.n) e += F.wr[J] * C.u[J];
                F.u[j] += e;
            }
        }
        __syncthreads();
        for (int k = 0; k < nu2; ++k) {
            line_relax(S, kind, l, 1);
            line_relax(S, kind, l, 0);
        }
    }
}

// Block-wide maximum (every thread gets it).
__device__ double line_block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    __syncthreads();
    return m;
}

__device__ int line_block_sum(int v, int* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;
}

struct LineGrid {
    int n;
    double scale;          // continuation reward factor on this grid (4^s)
    int stride;            // fine index of point j: (j + 1) * stride - 1
};

__device__ __forceinline__ double c_at(const LineArgs& A, const LineGrid& G, int j) {
    return G.scale * A.c[(j + 1) * G.stride - 1];
}
__device__ __forceinline__ double psi1_at(const LineArgs& A, const LineGrid& G, int j) {
    return A.psi1[(j + 1) * G.stride - 1];
}
__device__ __forceinline__ double psi2_at(const LineArgs& A, const LineGrid& G, int j) {
    return A.psi2[(j + 1) * G.stride - 1];
}

// Continuation value at j from the level-0 vector v (end values outside).
__device__ __forceinline__ double cont_at(const LineArgs& A, const LineGrid& G, const double* v,
                                          int j) {
    const double vl = j > 0 ? v[j - 1] : A.v_left;
    const double vr = j + 1 < G.n ? v[j + 1] : A.v_right;
    return 0.5 * (vl + vr) + c_at(A, G, j);
}

// Policy improvement at v: mode 0 (MAX and MIN, |F(v) - v|), 1 (MIN at alpha),
// 2 (MIN's reply for both a), 3 (no change: the given policies' rows).
// Keep-current rule with tolerance tau.  Returns the number of changed policy
// entries; row kinds and right-hand side follow the (new) policies.
__device__ int line_improve(const LineArgs& A, const LineGrid& G, int mode, const double* v,
                            uint8_t* alpha, uint8_t* beta, uint8_t* kind, double* f, double tau,
                            double* res) {
    int changed = 0;
    double rm = 0.0;
    for (int j = threadIdx.x; j < G.n; j += blockDim.x) {
        const double p1 = psi1_at(A, G, j), p2 = psi2_at(A, G, j);
        const double q[2][2] = {{p2, p1}, {p2, cont_at(A, G, v, j)}};   // q[a][b]
        double Fa[2];
        const int acur = alpha[j];
        for (int a = 0; a < 2; ++a) {
            const int bc = beta[2 * j + a];
            const int first = q[a][1] < q[a][0] ? 1 : 0;
            const double m = q[a][first];
            Fa[a] = m;
            if (mode == 3 || (mode == 1 && a != acur)) continue;
            const int b = q[a][bc] - m > tau ? first : bc;
            if (b != bc) {
                beta[2 * j + a] = (uint8_t)b;
                if (mode == 1) changed = 1;
            }
        }
        int anew = acur;
        if (mode == 0) {
            const int first = Fa[1] > Fa[0] ? 1 : 0;
            anew = Fa[first] - Fa[acur] > tau ? first : acur;
            if (anew != acur) changed = 1;
            alpha[j] = (uint8_t)anew;
            rm = fmax(rm, fabs(Fa[first] - v[j]));
        }
        const int b = beta[2 * j + anew];
        const uint8_t k = b == 0 ? kRowPsi2 : anew == 0 ? kRowPsi1 : kRowCont;
        kind[j] = k;
        double rhs = k == kRowPsi2 ? p2 : k == kRowPsi1 ? p1 : c_at(A, G, j);
        if (k == kRowCont) {
            if (j == 0) rhs += 0.5 * A.v_left;
            if (j + 1 == G.n) rhs += 0.5 * A.v_right;
        }
        f[j] = rhs;
    }
    if (res) *res = rm;
    return changed;
}

// Solves the policy-fixed system to the float64 floor from the current v.
__device__ int line_evaluate(LineShared& S, const uint8_t* kind, const double* f, double* v,
                             const LineArgs& A, double* red, int max_cycles) {
    LineLevel& L0 = S.L[0];
    line_setup(S, kind);
    int cycles = 0;
    double prev = 0.0;
    int slow = 0;
    for (;; ++cycles) {
        // residual of v in float64; the correction equation A e = r on the hierarchy
        double rm = 0.0, vm = 0.0;
        for (int j = threadIdx.x; j < L0.n; j += blockDim.x) {
            double lo, di, up;
            row0(kind, L0.n, j, &lo, &di, &up);
            double Av = di * v[j];
            if (j > 0) Av += lo * v[j - 1];
            if (j + 1 < L0.n) Av += up * v[j + 1];
            const double r = f[j] - Av;
            L0.f[j] = r;
            L0.u[j] = 0.0;
            rm = fmax(rm, fabs(r));
            vm = fmax(vm, fabs(v[j]));
        }
        rm = line_block_max(rm, red);
        vm = line_block_max(vm, red);
        if (rm <= 1e-15 * fmax(vm, 1e-300) || rm == 0.0) break;
        if (cycles > 0) {
            slow = rm > 0.5 * prev ? slow + 1 : 0;
            if (slow >= 2) break;           // float64 floor
        }
        prev = cycles > 0 ? fmin(prev, rm) : rm;
        if (cycles >= max_cycles) break;
        line_vcycle(S, kind, A.nu1, A.nu2);
        for (int j = threadIdx.x; j < L0.n; j += blockDim.x) v[j] += L0.u[j];
        __syncthreads();
    }
    return cycles;
}

__global__ void __launch_bounds__(kLineThreads, 1) k_line_pi(const __grid_constant__ LineArgs A) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ LineShared S;
    __shared__ double red[kLineThreads / 32];
    __shared__ int redi[kLineThreads / 32];
    const int nmax = A.n;
    // carve: level-0 vectors (v, u, f, row kinds, alpha, beta), then each level
    double* v = (double*)sm;
    double* rhs = v + nmax;
    size_t off = 2 * (size_t)nmax * sizeof(double);
    auto take_d = [&](int cnt) {
        double* p = (double*)(sm + off);
        off += (size_t)cnt * sizeof(double);
        return p;
    };
    if (threadIdx.x == 0) {
        int nl = 0;
        for (int n = nmax; nl < kLineMaxLevels; n = (n - 1) / 2) {
            LineLevel& L = S.L[nl++];
            L.n = n;
            if (n <= 3) break;
        }
        S.nlev = nl;
    }
    __syncthreads();
    for (int l = 0; l < S.nlev; ++l) {
        LineLevel& L = S.L[l];
        const int n = L.n;
        double* u = take_d(n);
        double* f = take_d(n);
        double *lo = nullptr, *di = nullptr, *up = nullptr, *wl = nullptr, *wr = nullptr;
        if (l > 0) {
            lo = take_d(n);
            di = take_d(n);
            up = take_d(n);
        }
        if (l + 1 < S.nlev) {
            wl = take_d((n - 1) / 2 + 1);
            wr = take_d((n - 1) / 2 + 1);
        }
        if (threadIdx.x == 0) {
            L.u = u; L.f = f; L.lo = lo; L.di = di; L.up = up; L.wl = wl; L.wr = wr;
        }
    }
    uint8_t* kind = sm + off;
    uint8_t* alpha = kind + nmax;
    uint8_t* beta = alpha + nmax;
    __syncthreads();

    // grids of FAMGpi: interior sizes 1, 3, 7, ..., n (or n alone)
    int ngrids = 1;
    if (A.fmg)
        for (int m = nmax; m > 1; m = (m - 1) / 2) ++ngrids;
    int outer_total = 0, systems = 0, cycles = 0, converged = 0;
    double res = 0.0;
    for (int gi = 0; gi < ngrids; ++gi) {
        LineGrid G;
        G.stride = 1 << (ngrids - 1 - gi);
        G.n = (nmax + 1) / G.stride - 1;
        G.scale = (double)G.stride * (double)G.stride;
        const bool last = gi + 1 == ngrids;
        // this grid's hierarchy: the first levels of the full one
        if (threadIdx.x == 0) {
            int nl = 0;
            for (int n = G.n; nl < kLineMaxLevels; n = (n - 1) / 2) {
                S.L[nl++].n = n;
                if (n <= 3) break;
            }
            S.nlev = nl;
        }
        __syncthreads();
        if (gi == 0) {
            // default policies: MAX stops, MIN's reply; v = 0
            for (int j = threadIdx.x; j < G.n; j += blockDim.x) {
                v[j] = 0.0;
                alpha[j] = 0;
                beta[2 * j] = beta[2 * j + 1] = 0;
            }
            __syncthreads();
            // tolerance 1e-13 max(1, |v|_inf) at v = 0
            line_improve(A, G, 2, v, alpha, beta, kind, rhs, 1e-13, nullptr);
            __syncthreads();
        } else {
            line_improve(A, G, 3, v, alpha, beta, kind, rhs, 0.0, nullptr);   // assembly only
            __syncthreads();
        }
        const double h = 1.0 / (double)(G.n + 1);
        const double eps = last ? A.eps : A.fmg_c * h * h;
        int outer = 0;
        while (true) {
            for (int it = 0; it < A.max_inner; ++it) {
                cycles += line_evaluate(S, kind, rhs, v, A, red, A.max_cycles);
                ++systems;
                double vm = 0.0;
                for (int j = threadIdx.x; j < G.n; j += blockDim.x) vm = fmax(vm, fabs(v[j]));
                vm = line_block_max(vm, red);
                const int ch = line_block_sum(
                    line_improve(A, G, 1, v, alpha, beta, kind, rhs, 1e-13 * fmax(1.0, vm), nullptr),
                    redi);
                if (ch == 0) break;
            }
            ++outer;
            double vm = 0.0;
            for (int j = threadIdx.x; j < G.n; j += blockDim.x) vm = fmax(vm, fabs(v[j]));
            vm = line_block_max(vm, red);
            double r = 0.0;
            const int ch = line_block_sum(
                line_improve(A, G, 0, v, alpha, beta, kind, rhs, 1e-13 * fmax(1.0, vm), &r), redi);
            res = line_block_max(r, red);
            if (res <= eps || ch == 0) {
                converged = 1;
                break;
            }
            if (outer >= A.max_outer) {
                converged = 0;
                break;
            }
        }
        outer_total += outer;
        if (!last) {
            // value interpolation I and strategy interpolation U (Sec. 5.2) to the
            // next grid, in place from the top down: coarse point J is fine 2J + 1
            const int nf = 2 * G.n + 1;
            double vj[4];
            uint8_t aj[4], b0[4], b1[4];
            int cnt = 0;
            for (int j = threadIdx.x; j < nf && cnt < 4; j += blockDim.x, ++cnt) {
                if (j & 1) {
                    const int J = (j - 1) / 2;
                    vj[cnt] = v[J];
                    aj[cnt] = alpha[J];
                    b0[cnt] = beta[2 * J];
                    b1[cnt] = beta[2 * J + 1];
                } else {
                    const int J = j / 2;   // between coarse J - 1 and J
                    const double vl = J - 1 >= 0 ? v[J - 1] : A.v_left;
                    const double vr = J < G.n ? v[J] : A.v_right;
                    vj[cnt] = 0.5 * (vl + vr);
                    const int Js = J - 1 >= 0 ? J - 1 : J;   // lowest-index interior neighbour
                    aj[cnt] = alpha[Js];
                    b0[cnt] = beta[2 * Js];
                    b1[cnt] = beta[2 * Js + 1];
                }
            }
            __syncthreads();
            cnt = 0;
            for (int j = threadIdx.x; j < nf && cnt < 4; j += blockDim.x, ++cnt) {
                v[j] = vj[cnt];
                alpha[j] = aj[cnt];
                beta[2 * j] = b0[cnt];
                beta[2 * j + 1] = b1[cnt];
            }
            __syncthreads();
        }
    }
    for (int j = threadIdx.x; j < nmax; j += blockDim.x) {
        A.v_out[j] = v[j];
        A.alpha_out[j] = alpha[j];
        A.beta_out[2 * j] = beta[2 * j];
        A.beta_out[2 * j + 1] = beta[2 * j + 1];
    }
    if (threadIdx.x == 0) {
        A.stats[0] = outer_total;
        A.stats[1] = systems;
        A.stats[2] = cycles;
        A.stats[3] = converged;
        A.stats[4] = ngrids;
        *A.res_out = res;
    }
}

}  // namespace

size_t line_smem_bytes(int n) {
    size_t off = 2 * (size_t)n * sizeof(double);
    int nl = 0;
    for (int m = n; nl < kLineMaxLevels; m = (m - 1) / 2) {
        ++nl;
        off += 2 * (size_t)m * sizeof(double);            // u, f
        if (nl > 1) off += 3 * (size_t)m * sizeof(double);  // lo, di, up
        if (m > 3) off += 2 * (size_t)((m - 1) / 2 + 1) * sizeof(double);   // wl, wr
        if (m <= 3) break;
    }
    return off + 4 * (size_t)n;   // kind, alpha, beta (2 per state)
}

void launch_line_pi(const LineArgs& A, cudaStream_t st) {
    const size_t smem = line_smem_bytes(A.n);
    GS_CUDA(cudaFuncSetAttribute(k_line_pi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_line_pi<<<1, kLineThreads, smem, st>>>(A);
    GS_CHECK_LAUNCH();
}

}  // namespace gs
