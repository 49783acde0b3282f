// Fine-level kernels of the finite-difference Isaacs game (Sec. 3.3, Sec. 6.1):
// reward set-up, policy improvement (Eq. (eq1)/(ILPI)) fused with the
// policy-fixed assembly (Eq. (LSPI)), the implicit 5-point operator's
// relaxation/residual, its interpolation and Galerkin product, and the FAMGpi
// interpolations (Sec. 5.2).
#include "kernels.cuh"
#include "stencil.cuh"

namespace gs {

namespace {

constexpr int kBlock = 256;

// SplitMix64 (Steele, Lea & Flood 2014): output i of the stream `seed`.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_isaacs_r0(int side, double h, double kappa, NoiseSrc ns, double* __restrict__ r0) {
    const size_t n = (size_t)side * side;
    size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const int i = (int)(x % side), j = (int)(x / side);
    const size_t ii = (size_t)(i + 1) * ns.step - 1, jj = (size_t)(j + 1) * ns.step - 1;
    const size_t fx = jj * ns.fine_side + ii;
    double xi;
    if (ns.xi_fine) {
        xi = ns.xi_fine[fx];
    } else {
        const double u = (double)(splitmix64(ns.seed, fx) >> 11) * 0x1.0p-53;
        xi = __dsub_rn(__dmul_rn(u, 0.1), 0.05);   // 0.1 u - 0.05, no contraction
    }
    const double x1 = (i + 1) * h, x2 = (j + 1) * h;
    r0[x] = kappa * (sin(M_PI * x1) * sin(M_PI * x2) + xi);
}

__device__ __forceinline__ double obstacle_psi(int i, int j, double h) {
    const double x1 = (i + 1) * h - 0.5, x2 = (j + 1) * h - 0.5;
    return 0.2 - (x1 * x1 + x2 * x2);
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_isum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// F(v; x, a, b) = mu sum_y p(y|x,a,b) v(y) + r(x,a,b) for the stencil of (a, b).
struct Nbr {
    double vE, vW, vN, vS, vx;
};
__device__ __forceinline__ double shapley_ab(const IsaacsConsts* K, const Nbr& nb, double r0,
                                             int a, int b) {
    const double* p = K->p[4 * a + b];
    const double s = p[0] * nb.vE + p[1] * nb.vW + p[2] * nb.vN + p[3] * nb.vS + p[4] * nb.vx;
    return K->mu * s + (r0 + K->dr[a][b]);
}

// MIN's reply at fixed a with the keep-current rule: returns the new b and
// sets *fmin to min_b F(v; x, a, b).
__device__ __forceinline__ int reply_b(const IsaacsConsts* K, const Nbr& nb, double r0, int a,
                                       int bcur, double tau, double* fmin) {
    double F[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) F[b] = shapley_ab(K, nb, r0, a, b);
    double m = F[0];
    int first = 0;
#pragma unroll
    for (int b = 1; b < 4; ++b)
        if (F[b] < m) { m = F[b]; first = b; }
    *fmin = m;
    return (F[bcur] - m > tau) ? first : bcur;
}

template <int MODE>
__global__ void k_isaacs_improve(const IsaacsConsts* __restrict__ K, int side, int variant,
                                 const double* __restrict__ v, const double* __restrict__ r0,
                                 uint8_t* __restrict__ alpha, uint32_t* __restrict__ beta,
                                 uint8_t* __restrict__ code, double* __restrict__ rhs,
                                 double* __restrict__ fv, DevScalars* sc) {
    const size_t n = (size_t)side * side;
    const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = x < n;
    double res = 0.0;
    int changed = 0;
    if (active) {
        const int i = (int)(x % side), j = (int)(x / side);
        const double tau = 1e-13 * fmax(1.0, __longlong_as_double((long long)sc->vmax));
        Nbr nb;
        nb.vx = v[x];
        nb.vE = i + 1 < side ? v[x + 1] : 0.0;
        nb.vW = i > 0 ? v[x - 1] : 0.0;
        nb.vN = j + 1 < side ? v[x + side] : 0.0;
        nb.vS = j > 0 ? v[x - side] : 0.0;
        const double rx = r0[x];
        const int acur = alpha[x];
        const uint32_t bw = beta[x];
        uint32_t bnew = bw;
        int anew = acur;
        if (MODE == IMP_INNER) {
            if (acur < 4) {
                const int bc = (bw >> (8 * acur)) & 0xff;
                double fmin;
                const int b = reply_b(K, nb, rx, acur, bc, tau, &fmin);
                if (b != bc) {
                    changed = 1;
                    bnew = (bw & ~(0xffu << (8 * acur))) | ((uint32_t)b << (8 * acur));
                }
            }
        } else {
            double Fa[5];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int bc = (bw >> (8 * a)) & 0xff;
                const int b = reply_b(K, nb, rx, a, bc, tau, &Fa[a]);
                bnew = (bnew & ~(0xffu << (8 * a))) | ((uint32_t)b << (8 * a));
            }
            const int m1 = variant == 1 ? 5 : 4;
            if (m1 == 5) Fa[4] = obstacle_psi(i, j, K->h);
            if (MODE == IMP_OUTER) {
                double fmax_ = Fa[0];
                int first = 0;
                for (int a = 1; a < m1; ++a)
                    if (Fa[a] > fmax_) { fmax_ = Fa[a]; first = a; }
                anew = (fmax_ - Fa[acur] > tau) ? first : acur;
                changed = anew != acur;
                res = fabs(fmax_ - nb.vx);
                if (fv) fv[x] = fmax_;
                alpha[x] = (uint8_t)anew;
            }
        }
        beta[x] = bnew;
        // policy-fixed assembly for (alpha, beta(., alpha))
        if (anew == 4) {
            code[x] = kStopCode;
            rhs[x] = obstacle_psi(i, j, K->h);
        } else {
            const int b = (bnew >> (8 * anew)) & 0xff;
            code[x] = (uint8_t)(4 * anew + b);
            rhs[x] = rx + K->dr[anew][b];
        }
    }
    const double wres = warp_max(res);
    const double wsq = warp_sum(res * res);
    const int wch = warp_isum(changed);
    if ((threadIdx.x & 31) == 0) {
        if (MODE == IMP_OUTER) {
            atomic_max_nonneg(&sc->res, wres);
            atomicAdd(&sc->res_sq, wsq);
        }
        if (wch) atomicAdd(&sc->changed, wch);
    }
}

__global__ void k_isaacs_assemble(const IsaacsConsts* __restrict__ K, int side,
                                  const uint8_t* __restrict__ alpha, const uint32_t* __restrict__ beta,
                                  const double* __restrict__ r0, uint8_t* __restrict__ code,
                                  double* __restrict__ rhs) {
    const size_t n = (size_t)side * side;
    const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const int a = alpha[x];
    if (a == 4) {
        code[x] = kStopCode;
        rhs[x] = obstacle_psi((int)(x % side), (int)(x / side), K->h);
    } else {
        const int b = (beta[x] >> (8 * a)) & 0xff;
        code[x] = (uint8_t)(4 * a + b);
        rhs[x] = r0[x] + K->dr[a][b];
    }
}

__global__ void k_absmax(const double* __restrict__ v, size_t n, unsigned long long* out) {
    double m = 0.0;
    for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (size_t)gridDim.x * blockDim.x)
        m = fmax(m, fabs(v[x]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(out, m);
}

// Fine-level neighbour access with Dirichlet zero outside the grid.
template <typename T>
struct Fine5 {
    T c, w, e, s, nn;
};
template <typename T>
__device__ __forceinline__ Fine5<T> load5(const T* __restrict__ u, size_t x, int i, int j, int side) {
    Fine5<T> q;
    q.c = u[x];
    q.w = i > 0 ? u[x - 1] : T(0);
    q.e = i + 1 < side ? u[x + 1] : T(0);
    q.s = j > 0 ? u[x - side] : T(0);
    q.nn = j + 1 < side ? u[x + side] : T(0);
    return q;
}

// float64 residual r = f - A u of the implicit 5-point operator; |r|_inf.
template <bool TO32>
__global__ void k_l0_residual64(const IsaacsConsts* __restrict__ K, int side,
                                const uint8_t* __restrict__ code, const double* __restrict__ f,
                                const double* __restrict__ u, void* __restrict__ r,
                                unsigned long long* rmax) {
    const size_t n = (size_t)side * side;
    const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rx = 0.0;
    if (x < n) {
        const int i = (int)(x % side), j = (int)(x / side);
        const double* am = K->am[code[x]];
        const Fine5<double> q = load5(u, x, i, j, side);
        const double Au = am[0] * q.c + am[1] * q.w + am[2] * q.e + am[3] * q.s + am[4] * q.nn;
        rx = f[x] - Au;
        if (TO32) ((float*)r)[x] = (float)rx;
        else ((double*)r)[x] = rx;
    }
    if (rmax) {
        const double m = warp_max(fabs(rx));
        if ((threadIdx.x & 31) == 0) atomic_max_nonneg(rmax, m);
    }
}

// Red-black ordering of the 5-point operator: colour 0 = points with i + j
// even = the C points (odd, odd) and the cell corners (even, even), which are
// uncoupled; colour 1 = the edge F points.  Relaxing colour 0 then colour 1
// is the C/F relaxation (C points first, then F points).
__device__ __forceinline__ bool colour_point(int side, int color, size_t t, int* i, int* j) {
    const int hs = (side + 1) / 2;
    *j = (int)(t / hs);
    *i = ((*j + color) & 1) + 2 * (int)(t % hs);
    return *j < side && *i < side;
}

__global__ void k_l0_smooth64(const IsaacsConsts* __restrict__ K, int side,
                              const uint8_t* __restrict__ code, const double* __restrict__ f,
                              double* __restrict__ u, int color) {
    int i, j;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (!colour_point(side, color, t, &i, &j)) return;
    const size_t x = (size_t)j * side + i;
    const double* am = K->am[code[x]];
    double s = f[x];
    if (i > 0) s -= am[1] * u[x - 1];
    if (i + 1 < side) s -= am[2] * u[x + 1];
    if (j > 0) s -= am[3] * u[x - side];
    if (j + 1 < side) s -= am[4] * u[x + side];
    u[x] = s / am[0];
}

// Row sum of the fine row (the leakage 1 - mu sum_y p), float64.
__device__ __forceinline__ double l0_rowsum(const IsaacsConsts* K, int c, int i, int j, int side) {
    if (c == kStopCode) return 1.0;
    const double* am = K->am[c];
    double s = K->kappa;
    if (i == 0) s -= am[1];
    if (i + 1 == side) s -= am[2];
    if (j == 0) s -= am[3];
    if (j + 1 == side) s -= am[4];
    return s;
}

__global__ void k_l0_smooth32(const IsaacsConsts* __restrict__ K, int side,
                              const uint8_t* __restrict__ code, const float* __restrict__ f,
                              float* __restrict__ u, int color, bool zero_init) {
    int i, j;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (!colour_point(side, color, t, &i, &j)) return;
    const size_t x = (size_t)j * side + i;
    const int c = code[x];
    const float* am = K->amf[c];
    const float s_row = (float)l0_rowsum(K, c, i, j, side);
    float diag = s_row, acc = f[x];
    if (i > 0) { diag -= am[1]; if (!zero_init) acc -= am[1] * u[x - 1]; }
    if (i + 1 < side) { diag -= am[2]; if (!zero_init) acc -= am[2] * u[x + 1]; }
    if (j > 0) { diag -= am[3]; if (!zero_init) acc -= am[3] * u[x - side]; }
    if (j + 1 < side) { diag -= am[4]; if (!zero_init) acc -= am[4] * u[x + side]; }
    u[x] = acc / diag;
}

__global__ void k_l0_residual32(const IsaacsConsts* __restrict__ K, int side,
                                const uint8_t* __restrict__ code, const float* __restrict__ f,
                                const float* __restrict__ u, float* __restrict__ r) {
    const size_t n = (size_t)side * side;
    const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const int i = (int)(x % side), j = (int)(x / side);
    const int c = code[x];
    const float* am = K->amf[c];
    const Fine5<float> q = load5(u, x, i, j, side);
    // leakage form: (A u)_x = s_x u_x + sum_d a_d (u_d - u_x) over interior d
    float Au = (float)l0_rowsum(K, c, i, j, side) * q.c;
    if (i > 0) Au += am[1] * (q.w - q.c);
    if (i + 1 < side) Au += am[2] * (q.e - q.c);
    if (j > 0) Au += am[3] * (q.s - q.c);
    if (j + 1 < side) Au += am[4] * (q.nn - q.c);
    r[x] = f[x] - Au;
}

__global__ void k_axpy32(double* __restrict__ v, const float* __restrict__ e, size_t n) {
    const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) v[x] += (double)e[x];
}

// FAMGpi interpolation from side sc to sf = 2 sc + 1 (1-based fine (p, q),
// coarse (P, Q) at fine (2P, 2Q); P or Q in {0, sc+1} is the boundary).
__global__ void k_fmg_interp(int sc, const double* __restrict__ vc, const uint8_t* __restrict__ ac,
                             const uint32_t* __restrict__ bc, const uint8_t* __restrict__ b4c,
                             double* __restrict__ vf, uint8_t* __restrict__ af,
                             uint32_t* __restrict__ bf, uint8_t* __restrict__ b4f) {
    const int sf = 2 * sc + 1;
    const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= (size_t)sf * sf) return;
    const int p = (int)(x % sf) + 1, q = (int)(x / sf) + 1;
    auto V = [&](int P, int Q) -> double {
        return (P < 1 || Q < 1 || P > sc || Q > sc) ? 0.0 : vc[(size_t)(Q - 1) * sc + (P - 1)];
    };
    double val;
    int P, Q;   // source of the policies: lowest-index interior member of N(x)
    if (!(p & 1) && !(q & 1)) {
        P = p / 2; Q = q / 2;
        val = V(P, Q);
    } else if ((p & 1) && !(q & 1)) {
        Q = q / 2;
        val = (V((p - 1) / 2, Q) + V((p + 1) / 2, Q)) / 2.0;
        P = (p - 1) / 2 >= 1 ? (p - 1) / 2 : (p + 1) / 2;
    } else if (!(p & 1) && (q & 1)) {
        P = p / 2;
        val = (V(P, (q - 1) / 2) + V(P, (q + 1) / 2)) / 2.0;
        Q = (q - 1) / 2 >= 1 ? (q - 1) / 2 : (q + 1) / 2;
    } else {
        const int P0 = (p - 1) / 2, P1 = (p + 1) / 2, Q0 = (q - 1) / 2, Q1 = (q + 1) / 2;
        val = (V(P0, Q0) + V(P1, Q0) + V(P0, Q1) + V(P1, Q1)) / 4.0;
        Q = Q0 >= 1 ? Q0 : Q1;
        P = P0 >= 1 ? P0 : P1;
        if (P > sc) P = P0;
        if (Q > sc) Q = Q0;
    }
    if (P > sc) P = sc;
    if (Q > sc) Q = sc;
    const size_t src = (size_t)(Q - 1) * sc + (P - 1);
    vf[x] = val;
    af[x] = ac[src];
    bf[x] = bc[src];
    if (b4f) b4f[x] = b4c[src];
}

}  // namespace

void launch_isaacs_r0(const IsaacsConsts* K, int side, double kappa, NoiseSrc ns, double* r0,
                      cudaStream_t st) {
    (void)K;
    const size_t n = (size_t)side * side;
    k_isaacs_r0<<<div_up(n, kBlock), kBlock, 0, st>>>(side, 1.0 / (side + 1), kappa, ns, r0);
    GS_CHECK_LAUNCH();
}

void launch_isaacs_improve(ImproveMode mode, const IsaacsConsts* K, int side, int variant,
                           const double* v, const double* r0, uint8_t* alpha, uint32_t* beta,
                           uint8_t* code, double* rhs, double* fv, DevScalars* sc,
                           cudaStream_t st) {
    const size_t n = (size_t)side * side;
    const unsigned g = div_up(n, kBlock);
    switch (mode) {
    case IMP_OUTER:
        k_isaacs_improve<IMP_OUTER><<<g, kBlock, 0, st>>>(K, side, variant, v, r0, alpha, beta, code, rhs, fv, sc);
        break;
    case IMP_INNER:
        k_isaacs_improve<IMP_INNER><<<g, kBlock, 0, st>>>(K, side, variant, v, r0, alpha, beta, code, rhs, fv, sc);
        break;
    default:
        k_isaacs_improve<IMP_REPLY><<<g, kBlock, 0, st>>>(K, side, variant, v, r0, alpha, beta, code, rhs, fv, sc);
    }
    GS_CHECK_LAUNCH();
}

void launch_isaacs_assemble(const IsaacsConsts* K, int side, const uint8_t* alpha,
                            const uint32_t* beta, const double* r0, uint8_t* code, double* rhs,
                            cudaStream_t st) {
    const size_t n = (size_t)side * side;
    k_isaacs_assemble<<<div_up(n, kBlock), kBlock, 0, st>>>(K, side, alpha, beta, r0, code, rhs);
    GS_CHECK_LAUNCH();
}

void launch_absmax(const double* v, size_t n, unsigned long long* out, cudaStream_t st) {
    unsigned g = div_up(n, kBlock);
    if (g > 152 * 8) g = 152 * 8;
    k_absmax<<<g, kBlock, 0, st>>>(v, n, out);
    GS_CHECK_LAUNCH();
}

void launch_l0_residual64(const IsaacsConsts* K, int side, const uint8_t* code, const double* f,
                          const double* u, double* r, unsigned long long* rmax, cudaStream_t st) {
    const size_t n = (size_t)side * side;
    k_l0_residual64<false><<<div_up(n, kBlock), kBlock, 0, st>>>(K, side, code, f, u, r, rmax);
    GS_CHECK_LAUNCH();
}

void launch_l0_residual64_to32(const IsaacsConsts* K, int side, const uint8_t* code,
                               const double* f, const double* u, float* r32,
                               unsigned long long* rmax, cudaStream_t st) {
    const size_t n = (size_t)side * side;
    k_l0_residual64<true><<<div_up(n, kBlock), kBlock, 0, st>>>(K, side, code, f, u, r32, rmax);
    GS_CHECK_LAUNCH();
}

void launch_l0_smooth64(const IsaacsConsts* K, int side, const uint8_t* code, const double* f,
                        double* u, int color, cudaStream_t st) {
    const size_t cnt = (size_t)side * ((side + 1) / 2);
    k_l0_smooth64<<<div_up(cnt, kBlock), kBlock, 0, st>>>(K, side, code, f, u, color);
    GS_CHECK_LAUNCH();
}

void launch_l0_smooth32(const IsaacsConsts* K, int side, const uint8_t* code, const float* f,
                        float* u, int color, bool zero_init, cudaStream_t st) {
    const size_t cnt = (size_t)side * ((side + 1) / 2);
    k_l0_smooth32<<<div_up(cnt, kBlock), kBlock, 0, st>>>(K, side, code, f, u, color, zero_init);
    GS_CHECK_LAUNCH();
}

void launch_l0_residual32(const IsaacsConsts* K, int side, const uint8_t* code, const float* f,
                          const float* u, float* r, cudaStream_t st) {
    const size_t n = (size_t)side * side;
    k_l0_residual32<<<div_up(n, kBlock), kBlock, 0, st>>>(K, side, code, f, u, r);
    GS_CHECK_LAUNCH();
}

void launch_l0_interp(const IsaacsConsts* K, int side, const uint8_t* code, double* P, float* P32,
                      cudaStream_t st) {
    const int sc = (side - 1) / 2;
    const size_t ncell = (size_t)(sc + 1) * (sc + 1);
    Src5 src{K, code, side};
    k_interp_edges<<<div_up(ncell, kBlock), kBlock, 0, st>>>(src, sc, P, P32);
    k_interp_corners<<<div_up(ncell, kBlock), kBlock, 0, st>>>(src, sc, P, P32);
    GS_CHECK_LAUNCH_N(2);
}

void launch_l0_rap(const IsaacsConsts* K, int side, const uint8_t* code, const double* P,
                   double* Ac, cudaStream_t st) {
    const int sc = (side - 1) / 2;
    Src5 src{K, code, side};
    k_rap<<<div_up((size_t)sc * sc, kBlock), kBlock, 0, st>>>(src, sc, P, Ac);
    GS_CHECK_LAUNCH();
}

void launch_l0_coarse_invert(const IsaacsConsts* K, int side, const uint8_t* code, double* inv,
                             int* status, cudaStream_t st) {
    const int n = side * side;
    static bool attr = false;
    if (!attr) {
        GS_CUDA(cudaFuncSetAttribute(k_coarse_invert<Src5>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 128 * 8));
        attr = true;
    }
    Src5 src{K, code, side};
    k_coarse_invert<<<1, 256, (size_t)n * 2 * n * sizeof(double), st>>>(src, side, inv, status);
    GS_CHECK_LAUNCH();
}

void launch_axpy32(double* v, const float* e, size_t n, cudaStream_t st) {
    k_axpy32<<<div_up(n, kBlock), kBlock, 0, st>>>(v, e, n);
    GS_CHECK_LAUNCH();
}

void launch_fmg_interp(int sc, const double* v_c, const uint8_t* alpha_c, const uint32_t* beta_c,
                       const uint8_t* beta4_c, double* v_f, uint8_t* alpha_f, uint32_t* beta_f,
                       uint8_t* beta4_f, cudaStream_t st) {
    const int sf = 2 * sc + 1;
    k_fmg_interp<<<div_up((size_t)sf * sf, kBlock), kBlock, 0, st>>>(sc, v_c, alpha_c, beta_c,
                                                                     beta4_c, v_f, alpha_f, beta_f,
                                                                     beta4_f);
    GS_CHECK_LAUNCH();
}

}  // namespace gs
