// Fine-level kernels of the finite-difference Isaacs game (Sec. 3.3, Sec. 6.1):
// reward set-up, policy improvement (Eq. (eq1)/(ILPI)) fused with the
// policy-fixed assembly (Eq. (LSPI)), and the
// FAMGpi interpolations (Sec. 5.2).
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

// Maximum of non-negative doubles through their bit patterns (integer ops).
__device__ __forceinline__ unsigned long long warp_max_bits(double v) {
    unsigned long long b = bits_of(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, b, o);
        b = w > b ? w : b;
    }
    return b;
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

// Shapley rows of the Isaacs game, factored.  With S the sum of the four
// neighbour values, w0 = 1/(2 c0) the weight of a direction without drift and
// delta = h/(2 c0) the extra weight of half a unit of drift, the drift
// (e_a - e_b)/2 puts delta on direction a and on the direction opposite to b
// (both on a when b is opposite to a), and a == b puts 2 delta on x itself:
//   F(v; x, a, b) = base + A_a + T_b            (a != b)
//   F(v; x, a, a) = base + 2 g v(x)
// with g = mu delta, base = mu w0 S + r0(x), A_a = g v(x + e_a) + c a,
// T_b = g v(x - e_b) - c b and c = 0.1 (1 - mu).  For fixed a, F(v; x, a, .)
// is base + A_a + u_b with u_b = T_b (b != a) and u_a = 2 g v(x) - A_a, so the
// argmin over b and the keep-current test compare the u_b.
struct Nbr {
    double vE, vW, vN, vS, vx;
};

// MIN's reply at fixed a with the keep-current rule: returns the new b and
// sets *fmin to min_b F(v; x, a, b).
__device__ __forceinline__ int reply_b(const double T[4], double A, double D, double base, int a,
                                       int bcur, double tau, double* fmin) {
    double u[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) u[b] = (b == a) ? D - A : T[b];
    double m = u[0];
    int first = 0;
#pragma unroll
    for (int b = 1; b < 4; ++b)
        if (u[b] < m) { m = u[b]; first = b; }
    *fmin = base + A + m;
    return (u[bcur] - m > tau) ? first : bcur;
}

// MIN's reply at fixed a screened in float32: the float32 copies of the u_b
// are within err of the float64 values the exact path compares (err bounds
// the float32 rounding of the inputs and of every operation, with a wide
// margin), so when the smallest float32 u_b beats every other by more than
// 2 err + tau, the float64 comparisons pick the same index, and with the
// keep-current rule the reply is that index.  Returns false (undecided)
// otherwise.  *phi = A_a + min_b u_b in float32.
__device__ __forceinline__ bool screen_reply(const float Tf[4], float Af, float Df, int a, float err,
                                             float tauf, int* b_out, float* phi) {
    float u[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) u[b] = (b == a) ? Df - Af : Tf[b];
    float m1 = u[0], m2 = INFINITY;
    int first = 0;
#pragma unroll
    for (int b = 1; b < 4; ++b) {
        if (u[b] < m1) {
            m2 = m1;
            m1 = u[b];
            first = b;
        } else if (u[b] < m2) {
            m2 = u[b];
        }
    }
    *b_out = first;
    *phi = Af + m1;
    return m2 - m1 > 2.0f * err + tauf;
}

// Keep-current tolerance 1e-13 max(1, |v|_inf) from the reduced |v|_inf.
__device__ __noinline__ double tau_of_vmax(const DevScalars* sc) {
    return 1e-13 * fmax(1.0, __longlong_as_double((long long)sc->vmax));
}

// The exact float64 decisions of one state, for the states whose float32
// screen was not conclusive (near-ties).  Not inlined: the compiler must not
// evaluate these float64 rows speculatively for every state.
template <int MODE>
__device__ __noinline__ void improve_exact(const IsaacsConsts* __restrict__ K, const Nbr nb,
                                           double rx, int i, int j, int m1, int acur, uint32_t bw,
                                           double tau, uint32_t* bnew_out, int* anew_out,
                                           double* fmax_out) {
    const double g = K->gmu, c = K->c01;
    const double base = K->w0mu * (nb.vE + nb.vW + nb.vN + nb.vS) + rx;
    const double D = 2.0 * g * nb.vx;
    // T_b = g v(x - e_b) - c b for b = +x1, -x1, +x2, -x2
    const double T[4] = {g * nb.vW, g * nb.vE - c, g * nb.vS - 2.0 * c, g * nb.vN - 3.0 * c};
    // A_a = g v(x + e_a) + c a
    const double A[4] = {g * nb.vE, g * nb.vW + c, g * nb.vN + 2.0 * c, g * nb.vS + 3.0 * c};
    uint32_t bnew = bw;
    int anew = acur;
    if (MODE == IMP_INNER) {
        if (acur < 4) {
            const int bc = (bw >> (8 * acur)) & 0xff;
            double fmin;
            const int b = reply_b(T, A[acur], D, base, acur, bc, tau, &fmin);
            bnew = (bw & ~(0xffu << (8 * acur))) | ((uint32_t)b << (8 * acur));
        }
    } else {
        double Fa[5];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int bc = (bw >> (8 * a)) & 0xff;
            const int b = reply_b(T, A[a], D, base, a, bc, tau, &Fa[a]);
            bnew = (bnew & ~(0xffu << (8 * a))) | ((uint32_t)b << (8 * a));
        }
        if (m1 == 5) Fa[4] = obstacle_psi(i, j, K->h);
        if (MODE == IMP_OUTER) {
            double fmax_ = Fa[0];
            int first = 0;
            for (int a = 1; a < m1; ++a)
                if (Fa[a] > fmax_) { fmax_ = Fa[a]; first = a; }
            anew = (fmax_ - Fa[acur] > tau) ? first : acur;
            *fmax_out = fmax_;
        }
    }
    *bnew_out = bnew;
    *anew_out = anew;
}

template <int MODE>
__global__ void k_isaacs_improve(const IsaacsConsts* __restrict__ K, int side, int variant,
                                 const double* __restrict__ v, const double* __restrict__ r0,
                                 uint8_t* __restrict__ alpha, uint32_t* __restrict__ beta,
                                 uint8_t* __restrict__ code, double* __restrict__ rhs,
                                 double* __restrict__ fv, DevScalars* sc, double tau_host,
                                 float tau_host_f, int tau_from_vmax) {
    const size_t n = (size_t)side * side;
    const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = x < n;
    double res = 0.0;
    int changed = 0, code_changed = 0;
    if (active) {
        unsigned iu;
        const int j = (int)FastDiv((unsigned)side).divmod((unsigned)x, &iu), i = (int)iu;
        Nbr nb;
        nb.vx = v[x];
        nb.vE = load_or_zero(v, x + 1, i + 1 < side);
        nb.vW = load_or_zero(v, x - 1, i > 0);
        nb.vN = load_or_zero(v, x + side, j + 1 < side);
        nb.vS = load_or_zero(v, x - side, j > 0);
        const double rx = r0[x];
        const int acur = alpha[x];
        const uint32_t bw = beta[x];
        const int m1 = variant == 1 ? 5 : 4;

        // ---- float32 screen of every decision this mode takes
        const float fx = f64_to_f32(nb.vx), fE = f64_to_f32(nb.vE), fW = f64_to_f32(nb.vW),
                    fN = f64_to_f32(nb.vN), fS = f64_to_f32(nb.vS);
        const float gf = K->gmu_f, cf = K->c01_f;
        const float tauf = tau_from_vmax ? f64_to_f32(tau_of_vmax(sc)) : tau_host_f;
        const float Vm = fmaxf(fmaxf(fabsf(fx), fmaxf(fabsf(fE), fabsf(fW))), fmaxf(fabsf(fN), fabsf(fS)));
        const float err = 0x1p-18f * (3.0f * gf * Vm + 6.0f * cf);
        const float Tf[4] = {gf * fW, gf * fE - cf, gf * fS - 2.0f * cf, gf * fN - 3.0f * cf};
        const float Af[4] = {gf * fE, gf * fW + cf, gf * fN + 2.0f * cf, gf * fS + 3.0f * cf};
        const float Df = 2.0f * gf * fx;
        bool sure = true;
        uint32_t bnew = bw;
        int anew = acur, amax = acur;
        int bfirst[4] = {0, 0, 0, 0};
        if (MODE == IMP_INNER) {
            if (acur < 4) {
                float phi;
                // select, not index: a runtime index would put Af in local memory
                const float Aa = acur == 0 ? Af[0] : acur == 1 ? Af[1] : acur == 2 ? Af[2] : Af[3];
                sure = screen_reply(Tf, Aa, Df, acur, err, tauf, &bfirst[0], &phi);
                bnew = (bw & ~(0xffu << (8 * acur))) | ((uint32_t)bfirst[0] << (8 * acur));
            }
        } else {
            float G[5];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                sure &= screen_reply(Tf, Af[a], Df, a, err, tauf, &bfirst[a], &G[a]);
                bnew = (bnew & ~(0xffu << (8 * a))) | ((uint32_t)bfirst[a] << (8 * a));
            }
            if (MODE == IMP_OUTER && sure) {
                // F(v; x, a) = base + G_a: base cancels between the four moves,
                // not against the stop value psi
                float margin = 4.0f * err + tauf;
                G[4] = -INFINITY;
                if (m1 == 5) {
                    const float S = (fE + fW) + (fN + fS);
                    const float basef = K->w0mu_f * S + f64_to_f32(rx);
                    const float x1 = (i + 1) * K->h_f - 0.5f, x2 = (j + 1) * K->h_f - 0.5f;
                    const float psif = 0.2f - (x1 * x1 + x2 * x2);
#pragma unroll
                    for (int a = 0; a < 4; ++a) G[a] += basef;
                    G[4] = psif;
                    margin += 0x1p-17f * (K->w0mu_f * 4.0f * Vm + fabsf(basef) + fabsf(psif) + 1.0f);
                }
                float g1 = G[0], g2 = -INFINITY;
                int first = 0;
#pragma unroll
                for (int a = 1; a < 5; ++a) {
                    if (G[a] > g1) {
                        g2 = g1;
                        g1 = G[a];
                        first = a;
                    } else if (G[a] > g2) {
                        g2 = G[a];
                    }
                }
                sure = g1 - g2 > margin;
                amax = first;
                anew = first;
            }
        }

        double fmax_ = 0.0;
        if (sure) {
            // float64 only where a value is stored
            if (MODE == IMP_OUTER) {
                if (amax == 4) {
                    fmax_ = obstacle_psi(i, j, K->h);
                } else {
                    const double g = K->gmu, c = K->c01;
                    const double base = K->w0mu * (nb.vE + nb.vW + nb.vN + nb.vS) + rx;
                    const int b = amax == 0 ? bfirst[0] : amax == 1 ? bfirst[1] : amax == 2 ? bfirst[2] : bfirst[3];
                    const double vb = b == 0 ? nb.vW : b == 1 ? nb.vE : b == 2 ? nb.vS : nb.vN;
                    const double va = amax == 0 ? nb.vE : amax == 1 ? nb.vW : amax == 2 ? nb.vN : nb.vS;
                    const double Aa = g * va + c * (double)amax;
                    // u_b = g v(x - e_b) - c b, or 2 g v(x) - A_a when b == a (as reply_b forms them)
                    const double u = (b == amax) ? 2.0 * g * nb.vx - Aa : g * vb - c * (double)b;
                    fmax_ = base + Aa + u;
                }
            }
        } else {
            improve_exact<MODE>(K, nb, rx, i, j, m1, acur, bw, tau_from_vmax ? tau_of_vmax(sc) : tau_host,
                                &bnew, &anew, &fmax_);
        }
        if (MODE == IMP_OUTER) {
            changed = anew != acur;
            res = fabs(fmax_ - nb.vx);
            if (fv) fv[x] = fmax_;
            alpha[x] = (uint8_t)anew;
        } else if (MODE == IMP_INNER) {
            changed = bnew != bw;
        }
        beta[x] = bnew;
        // policy-fixed assembly for (alpha, beta(., alpha))
        const int old_code = code[x];
        int new_code;
        if (anew == 4) {
            new_code = kStopCode;
            rhs[x] = obstacle_psi(i, j, K->h);
        } else {
            const int b = (bnew >> (8 * anew)) & 0xff;
            new_code = 4 * anew + b;
            rhs[x] = rx + K->dr[anew][b];
        }
        code[x] = (uint8_t)new_code;
        code_changed = new_code != old_code;
    }
    const int wch = warp_isum(changed);
    const int wcc = warp_isum(code_changed);
    if (MODE == IMP_OUTER) {
        const unsigned long long wres = warp_max_bits(res);
        const double wsq = warp_sum(res * res);
        if ((threadIdx.x & 31) == 0) {
            atomicMax(&sc->res, wres);
            atomicAdd(&sc->res_sq, wsq);
        }
    }
    if ((threadIdx.x & 31) == 0) {
        if (wch) atomicAdd(&sc->changed, wch);
        if (wcc) atomicAdd(&sc->code_changed, wcc);
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
                           uint8_t* code, double* rhs, double* fv, DevScalars* sc, double tau,
                           cudaStream_t st) {
    const size_t n = (size_t)side * side;
    const unsigned g = div_up(n, kBlock);
    switch (mode) {
    case IMP_OUTER:
        k_isaacs_improve<IMP_OUTER><<<g, kBlock, 0, st>>>(K, side, variant, v, r0, alpha, beta, code, rhs, fv, sc, tau < 0.0 ? 0.0 : tau, (float)(tau < 0.0 ? 0.0 : tau), tau < 0.0 ? 1 : 0);
        break;
    case IMP_INNER:
        k_isaacs_improve<IMP_INNER><<<g, kBlock, 0, st>>>(K, side, variant, v, r0, alpha, beta, code, rhs, fv, sc, tau < 0.0 ? 0.0 : tau, (float)(tau < 0.0 ? 0.0 : tau), tau < 0.0 ? 1 : 0);
        break;
    default:
        k_isaacs_improve<IMP_REPLY><<<g, kBlock, 0, st>>>(K, side, variant, v, r0, alpha, beta, code, rhs, fv, sc, tau < 0.0 ? 0.0 : tau, (float)(tau < 0.0 ? 0.0 : tau), tau < 0.0 ? 1 : 0);
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
