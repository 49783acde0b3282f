// Structured algebraic multigrid on 2^k - 1 grids: generic device code shared
// by the fine Isaacs level (implicit 5-point rows from policy codes) and the
// coarse levels (explicit 9-point rows).
//
// C/F splitting (Sec. 4.3): the coarse variables C of a level of side sf are
// its points (2I+1, 2J+1), I, J in [0, sc), sc = (sf-1)/2; the others are F.
// Interpolation P (Sec. 4.3, P^l_{l+1}) is operator dependent: an F point on
// an x-edge interpolates from its two C neighbours with the row collapsed
// along y, a y-edge point likewise, and a cell corner from the four diagonal C
// points through its own row and the edge weights.  Restriction is P^T and
// the coarse operator is the Galerkin product A^{l+1} = P^T A^l P.
#pragma once

#include "common.cuh"

namespace gs {

// Explicit 9-point rows A[d * n + x].
struct Src9 {
    const double* A;
    int side;
    size_t n;
    __device__ __forceinline__ void row(int i, int j, double a[9]) const {
        size_t x = (size_t)j * side + i;
#pragma unroll
        for (int d = 0; d < 9; ++d) a[d] = __ldg(A + d * n + x);
    }
};

// Implicit 5-point rows of the fine Isaacs level: the row of A = I - mu M for
// the policy code at the point, with couplings to boundary points dropped.
struct Src5 {
    const IsaacsConsts* K;
    const uint8_t* code;
    int side;
    __device__ __forceinline__ void row(int i, int j, double a[9]) const {
        int c = __ldg(code + (size_t)j * side + i);
        const double* am = K->am[c];
        a[DC] = am[0];
        a[DW] = i > 0 ? am[1] : 0.0;
        a[DE] = i + 1 < side ? am[2] : 0.0;
        a[DS] = j > 0 ? am[3] : 0.0;
        a[DN] = j + 1 < side ? am[4] : 0.0;
        a[DSW] = a[DSE] = a[DNW] = a[DNE] = 0.0;
    }
};

// Edge weights (F points on cell edges), one thread per cell (I, J) in [0, sc]^2.
template <class Src>
__global__ void k_interp_edges(Src src, int sc, double* __restrict__ P, float* __restrict__ P32) {
    const int nc1 = sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell) return;
    int I = (int)(t % nc1), J = (int)(t / nc1);
    double a[9];
    double wxW = 0, wxE = 0, wyS = 0, wyN = 0;
    if (J < sc) {          // x-edge point (2I, 2J+1): collapse the row along y
        src.row(2 * I, 2 * J + 1, a);
        double dC = a[DC] + a[DS] + a[DN];
        if (dC > 0) {
            wxW = -(a[DW] + a[DSW] + a[DNW]) / dC;
            wxE = -(a[DE] + a[DSE] + a[DNE]) / dC;
        }
    }
    if (I < sc) {          // y-edge point (2I+1, 2J): collapse the row along x
        src.row(2 * I + 1, 2 * J, a);
        double dC = a[DC] + a[DW] + a[DE];
        if (dC > 0) {
            wyS = -(a[DS] + a[DSW] + a[DSE]) / dC;
            wyN = -(a[DN] + a[DNW] + a[DNE]) / dC;
        }
    }
    P[PXW * ncell + t] = wxW;
    P[PXE * ncell + t] = wxE;
    P[PYS * ncell + t] = wyS;
    P[PYN * ncell + t] = wyN;
    if (P32) {
        P32[PXW * ncell + t] = (float)wxW;
        P32[PXE * ncell + t] = (float)wxE;
        P32[PYS * ncell + t] = (float)wyS;
        P32[PYN * ncell + t] = (float)wyN;
    }
}

// Corner weights: the corner point (2I, 2J) solves its own row for the value
// given the (already interpolated) values of its 8 neighbours.
template <class Src>
__global__ void k_interp_corners(Src src, int sc, double* __restrict__ P, float* __restrict__ P32) {
    const int nc1 = sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ncell) return;
    int I = (int)(t % nc1), J = (int)(t / nc1);
    double a[9];
    src.row(2 * I, 2 * J, a);
    size_t cW = t - 1, cS = t - nc1;
    // west neighbour (2I-1, 2J): y-edge of cell (I-1, J); east (2I+1, 2J): of cell (I, J)
    double yS_W = I >= 1 ? P[PYS * ncell + cW] : 0.0, yN_W = I >= 1 ? P[PYN * ncell + cW] : 0.0;
    double yS_E = I < sc ? P[PYS * ncell + t] : 0.0, yN_E = I < sc ? P[PYN * ncell + t] : 0.0;
    // south neighbour (2I, 2J-1): x-edge of cell (I, J-1); north (2I, 2J+1): of cell (I, J)
    double xW_S = J >= 1 ? P[PXW * ncell + cS] : 0.0, xE_S = J >= 1 ? P[PXE * ncell + cS] : 0.0;
    double xW_N = J < sc ? P[PXW * ncell + t] : 0.0, xE_N = J < sc ? P[PXE * ncell + t] : 0.0;
    double wSW = 0, wSE = 0, wNW = 0, wNE = 0;
    if (a[DC] > 0) {
        double inv = 1.0 / a[DC];
        wSW = -(a[DSW] + a[DW] * yS_W + a[DS] * xW_S) * inv;
        wSE = -(a[DSE] + a[DE] * yS_E + a[DS] * xE_S) * inv;
        wNW = -(a[DNW] + a[DW] * yN_W + a[DN] * xW_N) * inv;
        wNE = -(a[DNE] + a[DE] * yN_E + a[DN] * xE_N) * inv;
    }
    P[PSW * ncell + t] = wSW;
    P[PSE * ncell + t] = wSE;
    P[PNW * ncell + t] = wNW;
    P[PNE * ncell + t] = wNE;
    if (P32) {
        P32[PSW * ncell + t] = (float)wSW;
        P32[PSE * ncell + t] = (float)wSE;
        P32[PNW * ncell + t] = (float)wNW;
        P32[PNE * ncell + t] = (float)wNE;
    }
}

// Coarse points from which the fine point (gi, gj) interpolates, with weights.
template <typename W>
__device__ __forceinline__ int interp_of(const W* __restrict__ P, int sc, int gi, int gj,
                                         int cI[4], int cJ[4], W w[4]) {
    const int nc1 = sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    const int I = gi >> 1, J = gj >> 1;
    const size_t c = (size_t)J * nc1 + I;
    const int oi = gi & 1, oj = gj & 1;
    if (oi && oj) {
        cI[0] = I; cJ[0] = J; w[0] = W(1);
        return 1;
    }
    if (!oi && oj) {
        cI[0] = I - 1; cJ[0] = J; w[0] = P[PXW * ncell + c];
        cI[1] = I;     cJ[1] = J; w[1] = P[PXE * ncell + c];
        return 2;
    }
    if (oi && !oj) {
        cI[0] = I; cJ[0] = J - 1; w[0] = P[PYS * ncell + c];
        cI[1] = I; cJ[1] = J;     w[1] = P[PYN * ncell + c];
        return 2;
    }
    cI[0] = I - 1; cJ[0] = J - 1; w[0] = P[PSW * ncell + c];
    cI[1] = I;     cJ[1] = J - 1; w[1] = P[PSE * ncell + c];
    cI[2] = I - 1; cJ[2] = J;     w[2] = P[PNW * ncell + c];
    cI[3] = I;     cJ[3] = J;     w[3] = P[PNE * ncell + c];
    return 4;
}

// Weight of the fine point (2I+1+di, 2J+1+dj) towards the coarse point (I, J),
// i.e. the restriction coefficient R = P^T.
template <typename W>
__device__ __forceinline__ W restrict_weight(const W* __restrict__ P, int sc, int I, int J,
                                             int di, int dj) {
    const int nc1 = sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    if (di == 0 && dj == 0) return W(1);
    if (dj == 0)   // x-edge: (2I, .) is cell (I, J) east weight; (2I+2, .) cell (I+1, J) west weight
        return di < 0 ? P[PXE * ncell + (size_t)J * nc1 + I] : P[PXW * ncell + (size_t)J * nc1 + I + 1];
    if (di == 0)
        return dj < 0 ? P[PYN * ncell + (size_t)J * nc1 + I] : P[PYS * ncell + (size_t)(J + 1) * nc1 + I];
    if (dj < 0)
        return di < 0 ? P[PNE * ncell + (size_t)J * nc1 + I] : P[PNW * ncell + (size_t)J * nc1 + I + 1];
    return di < 0 ? P[PSE * ncell + (size_t)(J + 1) * nc1 + I]
                  : P[PSW * ncell + (size_t)(J + 1) * nc1 + I + 1];
}

// Galerkin coarse operator A_c = P^T A P (float64 accumulation), one thread per
// coarse point; the result is a 9-point stencil on the coarse grid.
template <class Src>
__global__ void k_rap(Src src, int sc, const double* __restrict__ P, double* __restrict__ Ac) {
    const size_t nc = (size_t)sc * sc;
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nc) return;
    const int I = (int)(t % sc), J = (int)(t / sc);
    const int sf = 2 * sc + 1;
    double acc[9];
#pragma unroll
    for (int d = 0; d < 9; ++d) acc[d] = 0.0;
    for (int dj = -1; dj <= 1; ++dj) {
        for (int di = -1; di <= 1; ++di) {
            const double R = restrict_weight(P, sc, I, J, di, dj);
            if (R == 0.0) continue;
            const int fi = 2 * I + 1 + di, fj = 2 * J + 1 + dj;
            double a[9];
            src.row(fi, fj, a);
#pragma unroll
            for (int d = 0; d < 9; ++d) {
                if (a[d] == 0.0) continue;
                const int gi = fi + dir_di(d), gj = fj + dir_dj(d);
                if (gi < 0 || gj < 0 || gi >= sf || gj >= sf) continue;
                const double RA = R * a[d];
                int cI[4], cJ[4];
                double w[4];
                const int m = interp_of(P, sc, gi, gj, cI, cJ, w);
                for (int k = 0; k < m; ++k) {
                    if (cI[k] < 0 || cJ[k] < 0 || cI[k] >= sc || cJ[k] >= sc) continue;
                    acc[dir_of(cI[k] - I, cJ[k] - J)] += RA * w[k];
                }
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 9; ++d) Ac[d * nc + t] = acc[d];
}

// Explicit inverse of the coarsest operator (n = side^2 <= 64) by Gauss-Jordan
// elimination with partial pivoting, in one thread block.  status[0] is set to
// 1 if a pivot vanished.
template <class Src>
__global__ void k_coarse_invert(Src src, int side, double* __restrict__ inv, int* status) {
    extern __shared__ double M[];   // n rows of 2n
    const int n = side * side, w = 2 * n;
    for (int e = threadIdx.x; e < n * w; e += blockDim.x) M[e] = 0.0;
    __syncthreads();
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        const int i = x % side, j = x / side;
        double a[9];
        src.row(i, j, a);
        for (int d = 0; d < 9; ++d) {
            const int gi = i + dir_di(d), gj = j + dir_dj(d);
            if (gi < 0 || gj < 0 || gi >= side || gj >= side) continue;
            M[x * w + gj * side + gi] += a[d];
        }
        M[x * w + n + x] = 1.0;
    }
    __syncthreads();
    __shared__ int piv;
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            int best = k;
            double bv = fabs(M[k * w + k]);
            for (int r = k + 1; r < n; ++r) {
                double v = fabs(M[r * w + k]);
                if (v > bv) { bv = v; best = r; }
            }
            piv = best;
            if (bv == 0.0) status[0] = 1;
        }
        __syncthreads();
        if (piv != k) {
            for (int c = threadIdx.x; c < w; c += blockDim.x) {
                double tmp = M[k * w + c];
                M[k * w + c] = M[piv * w + c];
                M[piv * w + c] = tmp;
            }
        }
        __syncthreads();
        const double d = M[k * w + k];
        const double dinv = d != 0.0 ? 1.0 / d : 0.0;
        __syncthreads();
        for (int c = threadIdx.x; c < w; c += blockDim.x) M[k * w + c] *= dinv;
        __syncthreads();
        for (int e = threadIdx.x; e < n * w; e += blockDim.x) {
            const int r = e / w, c = e % w;
            if (r == k || c == k) continue;
            M[e] -= M[r * w + k] * M[k * w + c];
        }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x)
            if (r != k) M[r * w + k] = 0.0;
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) inv[e] = M[(e / n) * w + n + (e % n)];
}

}  // namespace gs
