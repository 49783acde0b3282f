// Coarse-level (9-point) multigrid kernels: C/F relaxation, residual,
// restriction R = P^T, prolongation/correction, coarsest solve (Algorithm 3).
#include "kernels.cuh"
#include "stencil.cuh"

namespace gs {

namespace {

constexpr int kBlock = 256;

// Coarse stencil storage: float64 A[d*n+x] holds the entries of A; the float32
// copy holds the row sum in slot 0 and the off-diagonal entries in slots 1..8,
// so the diagonal is re-formed as (row sum) - (off-diagonal sum) in float32
// and the small row sums that carry the discount survive the rounding.
template <typename T>
struct Row9;

template <>
struct Row9<double> {
    const double* A;
    size_t n;
    __device__ __forceinline__ double diag(size_t x) const { return A[x]; }
    __device__ __forceinline__ double off(int d, size_t x) const { return A[d * n + x]; }
    // (A u)_x given u_x and the neighbour sum sum_d off_d u_d
    __device__ __forceinline__ double apply(size_t x, double ux, double offsum) const {
        return A[x] * ux + offsum;
    }
};

template <>
struct Row9<float> {
    const float* A;
    size_t n;
    __device__ __forceinline__ float diag(size_t x) const {
        float s = A[x];
#pragma unroll
        for (int d = 1; d < 9; ++d) s -= A[d * n + x];
        return s;
    }
    __device__ __forceinline__ float off(int d, size_t x) const { return A[d * n + x]; }
};

// One colour of the C/F relaxation (C points, then the F points by type):
// Gauss-Seidel u_x <- (f_x - sum_{y != x} a_xy u_y) / a_xx over the points
// (ox + 2k, oy + 2m), which are mutually uncoupled in a 9-point stencil.
template <typename T>
__global__ void k_smooth9(Row9<T> A, int side, const T* __restrict__ f, T* __restrict__ u,
                          int ox, int oy, bool zero_init) {
    const int nx = (side - ox + 1) / 2, ny = (side - oy + 1) / 2;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)nx * ny) return;
    const int i = ox + 2 * (int)(t % nx), j = oy + 2 * (int)(t / nx);
    const size_t x = (size_t)j * side + i;
    T s = f[x];
    if (!zero_init) {
#pragma unroll
        for (int d = 1; d < 9; ++d) {
            const int gi = i + dir_di(d), gj = j + dir_dj(d);
            if (gi < 0 || gj < 0 || gi >= side || gj >= side) continue;
            s -= A.off(d, x) * u[(size_t)gj * side + gi];
        }
    }
    u[x] = s / A.diag(x);
}

template <typename T>
__global__ void k_residual9(Row9<T> A, int side, const T* __restrict__ f, const T* __restrict__ u,
                            T* __restrict__ r) {
    const size_t n = (size_t)side * side;
    size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const int i = (int)(x % side), j = (int)(x / side);
    const T ux = u[x];
    T acc;
    if constexpr (sizeof(T) == 8) {
        acc = A.A[x] * ux;
#pragma unroll
        for (int d = 1; d < 9; ++d) {
            const int gi = i + dir_di(d), gj = j + dir_dj(d);
            if (gi < 0 || gj < 0 || gi >= side || gj >= side) continue;
            acc += A.off(d, x) * u[(size_t)gj * side + gi];
        }
    } else {
        // leakage form: (A u)_x = s_x u_x + sum_d a_d (u_d - u_x)
        acc = A.A[x] * ux;
#pragma unroll
        for (int d = 1; d < 9; ++d) {
            const int gi = i + dir_di(d), gj = j + dir_dj(d);
            const T ud = (gi < 0 || gj < 0 || gi >= side || gj >= side) ? T(0)
                                                                       : u[(size_t)gj * side + gi];
            acc += A.off(d, x) * (ud - ux);
        }
    }
    r[x] = f[x] - acc;
}

// f_c(I, J) = sum over the 3x3 fine block of P(i, (I,J)) r(i).
template <typename T, typename W>
__global__ void k_restrict(const T* __restrict__ r, const W* __restrict__ P, int sc,
                           T* __restrict__ fc) {
    const size_t nc = (size_t)sc * sc;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc) return;
    const int I = (int)(t % sc), J = (int)(t / sc);
    const int sf = 2 * sc + 1;
    T acc = 0;
#pragma unroll
    for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
        for (int di = -1; di <= 1; ++di) {
            const W w = restrict_weight(P, sc, I, J, di, dj);
            acc += (T)w * r[(size_t)(2 * J + 1 + dj) * sf + (2 * I + 1 + di)];
        }
    fc[t] = acc;
}

// u_f += P u_c, one thread per coarse cell (its corner, edge and C points).
template <typename T, typename W>
__global__ void k_prolong(const T* __restrict__ uc, const W* __restrict__ P, int sc,
                          T* __restrict__ uf) {
    const int nc1 = sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell) return;
    const int I = (int)(t % nc1), J = (int)(t / nc1);
    const int sf = 2 * sc + 1;
    auto U = [&](int a, int b) -> T {
        return (a < 0 || b < 0 || a >= sc || b >= sc) ? T(0) : uc[(size_t)b * sc + a];
    };
    const T uSW = U(I - 1, J - 1), uSE = U(I, J - 1), uNW = U(I - 1, J), uNE = U(I, J);
    uf[(size_t)(2 * J) * sf + 2 * I] += (T)P[PSW * ncell + t] * uSW + (T)P[PSE * ncell + t] * uSE +
                                        (T)P[PNW * ncell + t] * uNW + (T)P[PNE * ncell + t] * uNE;
    if (J < sc)
        uf[(size_t)(2 * J + 1) * sf + 2 * I] += (T)P[PXW * ncell + t] * uNW + (T)P[PXE * ncell + t] * uNE;
    if (I < sc)
        uf[(size_t)(2 * J) * sf + 2 * I + 1] += (T)P[PYS * ncell + t] * uSE + (T)P[PYN * ncell + t] * uNE;
    if (I < sc && J < sc) uf[(size_t)(2 * J + 1) * sf + 2 * I + 1] += uNE;
}

template <typename T>
__global__ void k_coarse_apply(const double* __restrict__ inv, int n, const T* __restrict__ f,
                               T* __restrict__ u) {
    __shared__ double fs[64];
    for (int k = threadIdx.x; k < n; k += blockDim.x) fs[k] = (double)f[k];
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += inv[(size_t)r * n + k] * fs[k];
        u[r] = (T)acc;
    }
}

__global__ void k_stencil_to32(const double* __restrict__ A, size_t n, float* __restrict__ A32) {
    size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 9; ++d) s += A[d * n + x];
    A32[x] = (float)s;
#pragma unroll
    for (int d = 1; d < 9; ++d) A32[d * n + x] = (float)A[d * n + x];
}

}  // namespace

void launch_interp9(const double* A, int side, double* P, float* P32, cudaStream_t st) {
    const int sc = (side - 1) / 2;
    const size_t ncell = (size_t)(sc + 1) * (sc + 1);
    Src9 src{A, side, (size_t)side * side};
    k_interp_edges<<<div_up(ncell, kBlock), kBlock, 0, st>>>(src, sc, P, P32);
    k_interp_corners<<<div_up(ncell, kBlock), kBlock, 0, st>>>(src, sc, P, P32);
    GS_CHECK_LAUNCH_N(2);
}

void launch_rap9(const double* A, int side, const double* P, double* Ac, cudaStream_t st) {
    const int sc = (side - 1) / 2;
    Src9 src{A, side, (size_t)side * side};
    k_rap<<<div_up((size_t)sc * sc, kBlock), kBlock, 0, st>>>(src, sc, P, Ac);
    GS_CHECK_LAUNCH();
}

void launch_coarse_invert9(const double* A, int side, double* inv, int* status, cudaStream_t st) {
    const int n = side * side;
    const size_t smem = (size_t)n * 2 * n * sizeof(double);
    static bool attr = false;
    if (!attr) {
        GS_CUDA(cudaFuncSetAttribute(k_coarse_invert<Src9>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 128 * 8));
        attr = true;
    }
    Src9 src{A, side, (size_t)n};
    k_coarse_invert<<<1, 256, smem, st>>>(src, side, inv, status);
    GS_CHECK_LAUNCH();
}

void launch_stencil_to32(const double* A, size_t n, float* A32, cudaStream_t st) {
    k_stencil_to32<<<div_up(n, kBlock), kBlock, 0, st>>>(A, n, A32);
    GS_CHECK_LAUNCH();
}

static void phase_offsets(int phase, int* ox, int* oy) {
    // C/F relaxation order: C = (odd, odd), then F: corners (even, even),
    // x-edges (even, odd), y-edges (odd, even).
    static const int OX[4] = {1, 0, 0, 1}, OY[4] = {1, 0, 1, 0};
    *ox = OX[phase];
    *oy = OY[phase];
}

template <typename T>
void launch_smooth9(const void* A, int side, const T* f, T* u, int phase, bool zero_init,
                    cudaStream_t st) {
    int ox, oy;
    phase_offsets(phase, &ox, &oy);
    const size_t cnt = (size_t)((side - ox + 1) / 2) * ((side - oy + 1) / 2);
    Row9<T> R{(const T*)A, (size_t)side * side};
    k_smooth9<T><<<div_up(cnt, kBlock), kBlock, 0, st>>>(R, side, f, u, ox, oy, zero_init);
    GS_CHECK_LAUNCH();
}

template <typename T>
void launch_residual9(const void* A, int side, const T* f, const T* u, T* r, cudaStream_t st) {
    const size_t n = (size_t)side * side;
    Row9<T> R{(const T*)A, n};
    k_residual9<T><<<div_up(n, kBlock), kBlock, 0, st>>>(R, side, f, u, r);
    GS_CHECK_LAUNCH();
}

template <typename T>
void launch_restrict(const T* r, const double* P64, const float* P32, int side_f, T* fc,
                     cudaStream_t st) {
    const int sc = (side_f - 1) / 2;
    const size_t nc = (size_t)sc * sc;
    if constexpr (sizeof(T) == 8)
        k_restrict<T, double><<<div_up(nc, kBlock), kBlock, 0, st>>>(r, P64, sc, fc);
    else
        k_restrict<T, float><<<div_up(nc, kBlock), kBlock, 0, st>>>(r, P32, sc, fc);
    GS_CHECK_LAUNCH();
}

template <typename T>
void launch_prolong(const T* uc, const double* P64, const float* P32, int side_f, T* uf,
                    cudaStream_t st) {
    const int sc = (side_f - 1) / 2;
    const size_t ncell = (size_t)(sc + 1) * (sc + 1);
    if constexpr (sizeof(T) == 8)
        k_prolong<T, double><<<div_up(ncell, kBlock), kBlock, 0, st>>>(uc, P64, sc, uf);
    else
        k_prolong<T, float><<<div_up(ncell, kBlock), kBlock, 0, st>>>(uc, P32, sc, uf);
    GS_CHECK_LAUNCH();
}

template <typename T>
void launch_coarse_apply(const double* inv, int n, const T* f, T* u, cudaStream_t st) {
    k_coarse_apply<T><<<1, 64, 0, st>>>(inv, n, f, u);
    GS_CHECK_LAUNCH();
}

template void launch_smooth9<double>(const void*, int, const double*, double*, int, bool, cudaStream_t);
template void launch_smooth9<float>(const void*, int, const float*, float*, int, bool, cudaStream_t);
template void launch_residual9<double>(const void*, int, const double*, const double*, double*, cudaStream_t);
template void launch_residual9<float>(const void*, int, const float*, const float*, float*, cudaStream_t);
template void launch_restrict<double>(const double*, const double*, const float*, int, double*, cudaStream_t);
template void launch_restrict<float>(const float*, const double*, const float*, int, float*, cudaStream_t);
template void launch_prolong<double>(const double*, const double*, const float*, int, double*, cudaStream_t);
template void launch_prolong<float>(const float*, const double*, const float*, int, float*, cudaStream_t);
template void launch_coarse_apply<double>(const double*, int, const double*, double*, cudaStream_t);
template void launch_coarse_apply<float>(const double*, int, const float*, float*, cudaStream_t);

}  // namespace gs
