// Structured algebraic multigrid on 2^k - 1 grids: device code shared by the
// fine Isaacs level (implicit 5-point rows from policy codes) and the coarse
// levels (explicit 9-point rows).
//
// C/F splitting (Sec. 4.3): the coarse variables C of a level of side sf are
// its points (2I+1, 2J+1), I, J in [0, sc), sc = (sf-1)/2; the others are F.
// Interpolation P^l_{l+1} is operator dependent: an F point on an x-edge
// interpolates from its two C neighbours with its row collapsed along y, a
// y-edge point likewise along x, and a cell corner from the four diagonal C
// points through its own row and the edge weights.  Restriction is
// R = P^T and the coarse operator is the Galerkin product A^{l+1} = R A^l P.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace gs {

// ------------------------------------------------------------------ weight storage
// The V-cycle's operators and interpolation weights are stored in float64,
// float32 or bfloat16 and used in the cycle's arithmetic type: wval widens a
// stored weight (bfloat16 to float32, the others unchanged).
__device__ __forceinline__ double wval(double x) { return x; }
__device__ __forceinline__ float wval(float x) { return x; }
__device__ __forceinline__ float wval(__nv_bfloat16 x) { return __bfloat162float(x); }

// Destination of the set-up's rounded copies: float32, bfloat16 or none.
struct WOut {
    float* f32;
    __nv_bfloat16* b16;
    __device__ __forceinline__ bool any() const { return f32 || b16; }
    __device__ __forceinline__ void put(size_t k, double v) const {
        if (f32) f32[k] = (float)v;
        else if (b16) b16[k] = __double2bfloat16(v);
    }
};

// ------------------------------------------------------------------ rows
// Explicit 9-point rows A[d * n + x] (float64).
struct Src9 {
    static constexpr bool kFivePoint = false;
    const double* A;
    int side;
    size_t n;
    __device__ __forceinline__ void row(int i, int j, double a[9]) const {
        size_t x = (size_t)j * side + i;
#pragma unroll
        for (int d = 0; d < 9; ++d) a[d] = A[d * n + x];
    }
};

// Implicit 5-point rows of the fine Isaacs level: the row of A = I - mu M for
// the policy code at the point, couplings to boundary points dropped.
struct Src5 {
    static constexpr bool kFivePoint = true;   // the diagonal entries are zero
    const IsaacsConsts* K;
    const uint8_t* code;
    int side;
    __device__ __forceinline__ void row(int i, int j, double a[9]) const {
        int c = code[(size_t)j * side + i];
        const double* am = K->am[c];
        a[DC] = am[0];
        a[DW] = i > 0 ? am[1] : 0.0;
        a[DE] = i + 1 < side ? am[2] : 0.0;
        a[DS] = j > 0 ? am[3] : 0.0;
        a[DN] = j + 1 < side ? am[4] : 0.0;
        a[DSW] = a[DSE] = a[DNW] = a[DNE] = 0.0;
    }
};

// Row sum of an implicit fine row (the leakage 1 - mu sum_y p(y)) in float32
// for the float32 path: kappa plus the mass of the couplings dropped at the
// boundary (all terms non-negative).
__device__ __forceinline__ float l0_rowsum_f(const IsaacsConsts* K, int c, int i, int j, int side) {
    if (c == kStopCode) return 1.0f;
    const float* am = K->amf[c];
    float s = K->kappa_f;
    if (i == 0) s -= am[1];
    if (i + 1 == side) s -= am[2];
    if (j == 0) s -= am[3];
    if (j + 1 == side) s -= am[4];
    return s;
}

// ------------------------------------------------------------------ level operators
// Residual f - A u at (i, j) and one Gauss-Seidel update of u at (i, j).
// The float32 forms use the leakage representation: the row sum s is kept
// separately and the diagonal is re-formed as s - sum(off-diagonals), so that
// the small row sums carrying the discount survive the rounding.
template <typename T>
struct L0Op;

template <>
struct L0Op<double> {
    const IsaacsConsts* K;
    const uint8_t* code;
    int side;
    // Couplings to the boundary multiply +0 instead of being skipped: no
    // branch or select on doubles (both would take the float64 pipe).
    // Five fused multiply-adds from f (each float64 operation costs 64 cycles).
    __device__ __forceinline__ double resid(const double* f, const double* u, int i, int j) const {
        const size_t x = (size_t)j * side + i;
        const double* am = K->am[code[x]];
        double r = fma(-am[0], u[x], f[x]);
        r = fma(-am[1], load_or_zero(u, x - 1, i > 0), r);
        r = fma(-am[2], load_or_zero(u, x + 1, i + 1 < side), r);
        r = fma(-am[3], load_or_zero(u, x - side, j > 0), r);
        return fma(-am[4], load_or_zero(u, x + side, j + 1 < side), r);
    }
    // Gauss-Seidel value of u at (i, j) (neighbours from u; zero: u == 0).
    __device__ __forceinline__ double relaxed(const double* f, const double* u, int i, int j,
                                              bool zero) const {
        const size_t x = (size_t)j * side + i;
        const double* am = K->am[code[x]];
        double s = f[x];
        if (!zero) {
            if (i > 0) s -= am[1] * u[x - 1];
            if (i + 1 < side) s -= am[2] * u[x + 1];
            if (j > 0) s -= am[3] * u[x - side];
            if (j + 1 < side) s -= am[4] * u[x + side];
        }
        return s / am[0];
    }
    // The same update with the four neighbours' values given (W, E, S, N).
    __device__ __forceinline__ double relaxed_nb(const double* f, int i, int j, double uW, double uE,
                                                 double uS, double uN) const {
        const size_t x = (size_t)j * side + i;
        const double* am = K->am[code[x]];
        double s = f[x];
        if (i > 0) s -= am[1] * uW;
        if (i + 1 < side) s -= am[2] * uE;
        if (j > 0) s -= am[3] * uS;
        if (j + 1 < side) s -= am[4] * uN;
        return s / am[0];
    }
};

template <>
struct L0Op<float> {
    const IsaacsConsts* K;
    const uint8_t* code;
    int side;
    __device__ __forceinline__ float resid(const float* f, const float* u, int i, int j) const {
        const size_t x = (size_t)j * side + i;
        const int c = code[x];
        const float* am = K->amf[c];
        const float ux = u[x];
        float Au = l0_rowsum_f(K, c, i, j, side) * ux;
        if (i > 0) Au += am[1] * (u[x - 1] - ux);
        if (i + 1 < side) Au += am[2] * (u[x + 1] - ux);
        if (j > 0) Au += am[3] * (u[x - side] - ux);
        if (j + 1 < side) Au += am[4] * (u[x + side] - ux);
        return f[x] - Au;
    }
    // Diagonal of the row in the leakage form, as relaxed() forms it.
    __device__ __forceinline__ float diag(int i, int j) const {
        const int c = code[(size_t)j * side + i];
        const float* am = K->amf[c];
        float d = l0_rowsum_f(K, c, i, j, side);
        if (i > 0) d -= am[1];
        if (i + 1 < side) d -= am[2];
        if (j > 0) d -= am[3];
        if (j + 1 < side) d -= am[4];
        return d;
    }
    __device__ __forceinline__ float relaxed(const float* f, const float* u, int i, int j,
                                             bool zero) const {
        const size_t x = (size_t)j * side + i;
        const int c = code[x];
        const float* am = K->amf[c];
        float diag = l0_rowsum_f(K, c, i, j, side), s = f[x];
        if (i > 0) { diag -= am[1]; if (!zero) s -= am[1] * u[x - 1]; }
        if (i + 1 < side) { diag -= am[2]; if (!zero) s -= am[2] * u[x + 1]; }
        if (j > 0) { diag -= am[3]; if (!zero) s -= am[3] * u[x - side]; }
        if (j + 1 < side) { diag -= am[4]; if (!zero) s -= am[4] * u[x + side]; }
        return s / diag;
    }
    __device__ __forceinline__ float relaxed_nb(const float* f, int i, int j, float uW, float uE,
                                                float uS, float uN) const {
        const size_t x = (size_t)j * side + i;
        const int c = code[x];
        const float* am = K->amf[c];
        float diag = l0_rowsum_f(K, c, i, j, side), s = f[x];
        if (i > 0) { diag -= am[1]; s -= am[1] * uW; }
        if (i + 1 < side) { diag -= am[2]; s -= am[2] * uE; }
        if (j > 0) { diag -= am[3]; s -= am[3] * uS; }
        if (j + 1 < side) { diag -= am[4]; s -= am[4] * uN; }
        return s / diag;
    }
};

// 9-point levels: float64 rows hold the entries of A; float32 rows hold the
// row sum in slot 0 and the off-diagonal entries in slots 1..8.
template <typename T, typename W = T>
struct L9Op {
    const W* A;
    size_t n;
    int side;
    __device__ __forceinline__ T resid(const T* f, const T* u, int i, int j) const {
        const size_t x = (size_t)j * side + i;
        const T ux = u[x];
        T Au = (T)wval(A[x]) * ux;
#pragma unroll
        for (int d = 1; d < 9; ++d) {
            const int gi = i + dir_di(d), gj = j + dir_dj(d);
            const bool in = gi >= 0 && gj >= 0 && gi < side && gj < side;
            const T ud = in ? u[(size_t)gj * side + gi] : T(0);
            if constexpr (sizeof(T) == 8) Au += (T)wval(A[d * n + x]) * ud;
            else Au += (T)wval(A[d * n + x]) * (ud - ux);
        }
        return f[x] - Au;
    }
    // Gauss-Seidel value of u at (i, j) (neighbours from u; zero: u == 0).
    __device__ __forceinline__ T relaxed(const T* f, const T* u, int i, int j, bool zero) const {
        const size_t x = (size_t)j * side + i;
        T s = f[x];
        T diag = (T)wval(A[x]);
#pragma unroll
        for (int d = 1; d < 9; ++d) {
            const T a = (T)wval(A[d * n + x]);
            if constexpr (sizeof(T) == 4) diag -= a;
            if (zero) continue;
            const int gi = i + dir_di(d), gj = j + dir_dj(d);
            if (gi < 0 || gj < 0 || gi >= side || gj >= side) continue;
            s -= a * u[(size_t)gj * side + gi];
        }
        return s / diag;
    }
    // Diagonal of the row, as relaxed() forms it.
    __device__ __forceinline__ T diag(int i, int j) const {
        const size_t x = (size_t)j * side + i;
        T d = (T)wval(A[x]);
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int k = 1; k < 9; ++k) d -= (T)wval(A[k * n + x]);
        }
        return d;
    }
};

// ------------------------------------------------------------------ interpolation
// Edge weights of cell t = (I, J), I, J in [0, sc].
template <class Src>
__device__ __forceinline__ void interp_edges_item(const Src& src, int sc, size_t t, double* P,
                                                  const WOut& Pw) {
    const int nc1 = sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    const int I = (int)(t % nc1), J = (int)(t / nc1);
    double a[9];
    double wxW = 0, wxE = 0, wyS = 0, wyN = 0;
    if (J < sc) {          // x-edge point (2I, 2J+1): row collapsed along y
        src.row(2 * I, 2 * J + 1, a);
        const double dC = a[DC] + a[DS] + a[DN];
        if (dC > 0) {
            wxW = -(a[DW] + a[DSW] + a[DNW]) / dC;
            wxE = -(a[DE] + a[DSE] + a[DNE]) / dC;
        }
    }
    if (I < sc) {          // y-edge point (2I+1, 2J): row collapsed along x
        src.row(2 * I + 1, 2 * J, a);
        const double dC = a[DC] + a[DW] + a[DE];
        if (dC > 0) {
            wyS = -(a[DS] + a[DSW] + a[DSE]) / dC;
            wyN = -(a[DN] + a[DNW] + a[DNE]) / dC;
        }
    }
    P[PXW * ncell + t] = wxW;
    P[PXE * ncell + t] = wxE;
    P[PYS * ncell + t] = wyS;
    P[PYN * ncell + t] = wyN;
    if (Pw.any()) {
        Pw.put(PXW * ncell + t, wxW);
        Pw.put(PXE * ncell + t, wxE);
        Pw.put(PYS * ncell + t, wyS);
        Pw.put(PYN * ncell + t, wyN);
    }
}

// Corner weights: the corner point (2I, 2J) solves its own row given the
// interpolated values of its 8 neighbours (needs the edge weights).
template <class Src>
__device__ __forceinline__ void interp_corners_item(const Src& src, int sc, size_t t, double* P,
                                                    const WOut& Pw) {
    const int nc1 = sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    const int I = (int)(t % nc1), J = (int)(t / nc1);
    double a[9];
    src.row(2 * I, 2 * J, a);
    const size_t cW = t - 1, cS = t - nc1;
    // west neighbour (2I-1, 2J): y-edge of cell (I-1, J); east (2I+1, 2J): of cell (I, J)
    const double yS_W = I >= 1 ? P[PYS * ncell + cW] : 0.0, yN_W = I >= 1 ? P[PYN * ncell + cW] : 0.0;
    const double yS_E = I < sc ? P[PYS * ncell + t] : 0.0, yN_E = I < sc ? P[PYN * ncell + t] : 0.0;
    // south neighbour (2I, 2J-1): x-edge of cell (I, J-1); north (2I, 2J+1): of cell (I, J)
    const double xW_S = J >= 1 ? P[PXW * ncell + cS] : 0.0, xE_S = J >= 1 ? P[PXE * ncell + cS] : 0.0;
    const double xW_N = J < sc ? P[PXW * ncell + t] : 0.0, xE_N = J < sc ? P[PXE * ncell + t] : 0.0;
    double wSW = 0, wSE = 0, wNW = 0, wNE = 0;
    if (a[DC] > 0) {
        const double inv = 1.0 / a[DC];
        wSW = -(a[DSW] + a[DW] * yS_W + a[DS] * xW_S) * inv;
        wSE = -(a[DSE] + a[DE] * yS_E + a[DS] * xE_S) * inv;
        wNW = -(a[DNW] + a[DW] * yN_W + a[DN] * xW_N) * inv;
        wNE = -(a[DNE] + a[DE] * yN_E + a[DN] * xE_N) * inv;
    }
    P[PSW * ncell + t] = wSW;
    P[PSE * ncell + t] = wSE;
    P[PNW * ncell + t] = wNW;
    P[PNE * ncell + t] = wNE;
    if (Pw.any()) {
        Pw.put(PSW * ncell + t, wSW);
        Pw.put(PSE * ncell + t, wSE);
        Pw.put(PNW * ncell + t, wNW);
        Pw.put(PNE * ncell + t, wNE);
    }
}

// Weight of the fine point (2I+1+di, 2J+1+dj) towards the coarse point (I, J):
// the restriction coefficient R = P^T.
template <typename W>
__device__ __forceinline__ auto restrict_weight(const W* P, int sc, int I, int J, int di, int dj)
    -> decltype(wval(P[0])) {
    using R = decltype(wval(P[0]));
    const int nc1 = sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    if (di == 0 && dj == 0) return R(1);
    if (dj == 0)   // x-edge: (2I, .) is cell (I, J) east weight; (2I+2, .) cell (I+1, J) west weight
        return wval(di < 0 ? P[PXE * ncell + (size_t)J * nc1 + I] : P[PXW * ncell + (size_t)J * nc1 + I + 1]);
    if (di == 0)
        return wval(dj < 0 ? P[PYN * ncell + (size_t)J * nc1 + I]
                           : P[PYS * ncell + (size_t)(J + 1) * nc1 + I]);
    if (dj < 0)
        return wval(di < 0 ? P[PNE * ncell + (size_t)J * nc1 + I]
                           : P[PNW * ncell + (size_t)J * nc1 + I + 1]);
    return wval(di < 0 ? P[PSE * ncell + (size_t)(J + 1) * nc1 + I]
                       : P[PSW * ncell + (size_t)(J + 1) * nc1 + I + 1]);
}

// Adds v to the coarse stencil entry towards (I + tx, J + ty) if that point is
// an unknown (coarse boundary points carry the Dirichlet value 0).
template <typename V>
__device__ __forceinline__ void rap_add(V acc[9], int I, int J, int sc, int tx, int ty, V v) {
    if (I + tx >= 0 && I + tx < sc && J + ty >= 0 && J + ty < sc) acc[dir_of(tx, ty)] += v;
}

// Scatters RA = R(., i) A(i, g) along the interpolation row of the fine point g
// at offset (qx, qy) in [-2, 2]^2 from the coarse point's fine position
// (2I+1, 2J+1).  After unrolling, qx and qy are constants: the point's type
// (C, x-edge, y-edge, corner), its cell and its coarse targets fold away and
// acc stays in registers.
template <typename V>
__device__ __forceinline__ void rap_scatter(const V* P, int sc, int I, int J, int qx, int qy, V RA,
                                            V acc[9]) {
    const int nc1 = sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    const bool xC = (qx & 1) == 0, yC = (qy & 1) == 0;
    if (xC && yC) {
        rap_add(acc, I, J, sc, qx / 2, qy / 2, RA);
    } else if (!xC && yC) {                     // x-edge of cell (I + (1+qx)/2, J + qy/2)
        const int tx = (1 + qx) / 2, ty = qy / 2;
        const size_t c = (size_t)(J + ty) * nc1 + (I + tx);
        rap_add(acc, I, J, sc, tx - 1, ty, RA * P[PXW * ncell + c]);
        rap_add(acc, I, J, sc, tx, ty, RA * P[PXE * ncell + c]);
    } else if (xC && !yC) {                     // y-edge of cell (I + qx/2, J + (1+qy)/2)
        const int tx = qx / 2, ty = (1 + qy) / 2;
        const size_t c = (size_t)(J + ty) * nc1 + (I + tx);
        rap_add(acc, I, J, sc, tx, ty - 1, RA * P[PYS * ncell + c]);
        rap_add(acc, I, J, sc, tx, ty, RA * P[PYN * ncell + c]);
    } else {                                    // corner of cell (I + (1+qx)/2, J + (1+qy)/2)
        const int tx = (1 + qx) / 2, ty = (1 + qy) / 2;
        const size_t c = (size_t)(J + ty) * nc1 + (I + tx);
        rap_add(acc, I, J, sc, tx - 1, ty - 1, RA * P[PSW * ncell + c]);
        rap_add(acc, I, J, sc, tx, ty - 1, RA * P[PSE * ncell + c]);
        rap_add(acc, I, J, sc, tx - 1, ty, RA * P[PNW * ncell + c]);
        rap_add(acc, I, J, sc, tx, ty, RA * P[PNE * ncell + c]);
    }
}

// Galerkin coarse row A_c(t, .) = (P^T A P)(t, .) for the coarse point t
// (float64 accumulation); also its rounded leakage form (row sum, then the
// off-diagonal entries) when Aw has a destination.
template <class Src>
__device__ __forceinline__ void rap_item(const Src& src, int sc, size_t t, const double* P,
                                         double* Ac, const WOut& Aw) {
    const size_t nc = (size_t)sc * sc;
    const int I = (int)(t % sc), J = (int)(t / sc);
    const int sf = 2 * sc + 1;
    double acc[9];
#pragma unroll
    for (int d = 0; d < 9; ++d) acc[d] = 0.0;
#pragma unroll
    for (int oy = -1; oy <= 1; ++oy) {
#pragma unroll
        for (int ox = -1; ox <= 1; ++ox) {
            const double R = restrict_weight(P, sc, I, J, ox, oy);
            double a[9];
            src.row(2 * I + 1 + ox, 2 * J + 1 + oy, a);
#pragma unroll
            for (int d = 0; d < 9; ++d) {
                // The 5-point rows' diagonal entries are zero: skip them at
                // compile time.  No test on loaded values: it would make each
                // weight load below wait for the row's load.
                if constexpr (Src::kFivePoint)
                    if (d >= DSW) continue;
                const int qx = ox + dir_di(d), qy = oy + dir_dj(d);
                const int gi = 2 * I + 1 + qx, gj = 2 * J + 1 + qy;
                if (gi < 0 || gj < 0 || gi >= sf || gj >= sf) continue;
                rap_scatter(P, sc, I, J, qx, qy, R * a[d], acc);
            }
        }
    }
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 9; ++d) {
        Ac[d * nc + t] = acc[d];
        s += acc[d];
    }
    if (Aw.any()) {
        Aw.put(t, s);
#pragma unroll
        for (int d = 1; d < 9; ++d) Aw.put(d * nc + t, acc[d]);
    }
}

// ------------------------------------------------------------------ float32 set-up
// The mixed path builds its hierarchy in float32 (a float64 warp instruction
// costs 64 cycles of its SM sub-partition here, a float32 one under 5).  The
// V-cycle only needs float32 operators, but in the leakage form: each row's
// sum s (1 - mu sum p, O(h^2) against O(1) entries) must be accurate, and a
// sum of rounded float32 entries would lose it.  So s is carried separately
// and never formed by summing entries:
//  * a row is (a[9], s); a stored level holds (s, off[8]) and a[DC] = s - sum off;
//  * interpolation weights come from the rows as in float64, and the defect
//    of P on the constant vector, delta(g) = (P 1)(g) - 1 at each fine point g,
//    from identities free of cancellation:
//      edge point, row collapsed to dC:  w1 + w2 = 1 - s / dC,
//      cell corner:  sum of its 4 weights = 1 - (s + sum_dir a[dir] delta_dir) / a[DC]
//    (delta_dir of its four edge neighbours), less the weights towards coarse
//    points outside the grid (only next to the boundary, where delta is O(1));
//  * the Galerkin row sum is (P^T A P 1)(t) = sum_f R(t, f) (s_f + sum_g A(f, g) delta(g)),
//    small terms of one sign in the interior; the Galerkin off-diagonal
//    entries are accumulated in float32 as in float64.

// Fine level rows from the float32 table, with their row sums.
struct Src5f {
    static constexpr bool kFivePoint = true;
    const IsaacsConsts* K;
    const uint8_t* code;
    int side;
    __device__ __forceinline__ void row(int i, int j, float a[9], float* s) const {
        const int c = code[(size_t)j * side + i];
        const float* am = K->amf[c];
        a[DC] = am[0];
        a[DW] = i > 0 ? am[1] : 0.0f;
        a[DE] = i + 1 < side ? am[2] : 0.0f;
        a[DS] = j > 0 ? am[3] : 0.0f;
        a[DN] = j + 1 < side ? am[4] : 0.0f;
        a[DSW] = a[DSE] = a[DNW] = a[DNE] = 0.0f;
        *s = l0_rowsum_f(K, c, i, j, side);
    }
};

// Stored float32 leakage rows [9][n] (row sum, then the off-diagonal entries).
struct Src9f {
    static constexpr bool kFivePoint = false;
    const float* A;
    int side;
    size_t n;
    __device__ __forceinline__ void row(int i, int j, float a[9], float* s) const {
        const size_t x = (size_t)j * side + i;
        float d = A[x];
        *s = d;
#pragma unroll
        for (int k = 1; k < 9; ++k) {
            a[k] = A[k * n + x];
            d -= a[k];
        }
        a[DC] = d;
    }
};

// The same rows promoted to float64 (for the coarsest level's explicit inverse).
struct Src9fd {
    const float* A;
    int side;
    size_t n;
    __device__ __forceinline__ void row(int i, int j, double a[9]) const {
        const size_t x = (size_t)j * side + i;
        double d = A[x];
#pragma unroll
        for (int k = 1; k < 9; ++k) {
            a[k] = A[k * n + x];
            d -= a[k];
        }
        a[DC] = d;
    }
};

// Edge weights of cell t (as interp_edges_item) and delta (without the
// outside-the-grid correction) at its x- and y-edge points; delta is indexed
// like the fine level.
template <class Src>
__device__ __forceinline__ void interp_edges_item_f(const Src& src, int sc, unsigned t, float* P,
                                                    __nv_bfloat16* P16, float* delta) {
    const int nc1 = sc + 1, sf = 2 * sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    const int I = (int)(t % (unsigned)nc1), J = (int)(t / (unsigned)nc1);
    float a[9], s;
    float wxW = 0, wxE = 0, wyS = 0, wyN = 0;
    if (J < sc) {          // x-edge point (2I, 2J+1): row collapsed along y
        src.row(2 * I, 2 * J + 1, a, &s);
        const float dC = a[DC] + a[DS] + a[DN];
        float d = -1.0f;
        if (dC > 0) {
            wxW = -(a[DW] + a[DSW] + a[DNW]) / dC;
            wxE = -(a[DE] + a[DSE] + a[DNE]) / dC;
            d = -s / dC;
        }
        delta[(size_t)(2 * J + 1) * sf + 2 * I] = d;
    }
    if (I < sc) {          // y-edge point (2I+1, 2J): row collapsed along x
        src.row(2 * I + 1, 2 * J, a, &s);
        const float dC = a[DC] + a[DW] + a[DE];
        float d = -1.0f;
        if (dC > 0) {
            wyS = -(a[DS] + a[DSW] + a[DSE]) / dC;
            wyN = -(a[DN] + a[DNW] + a[DNE]) / dC;
            d = -s / dC;
        }
        delta[(size_t)(2 * J) * sf + 2 * I + 1] = d;
    }
    P[PXW * ncell + t] = wxW;
    P[PXE * ncell + t] = wxE;
    P[PYS * ncell + t] = wyS;
    P[PYN * ncell + t] = wyN;
    if (P16) {
        P16[PXW * ncell + t] = __float2bfloat16_rn(wxW);
        P16[PXE * ncell + t] = __float2bfloat16_rn(wxE);
        P16[PYS * ncell + t] = __float2bfloat16_rn(wyS);
        P16[PYN * ncell + t] = __float2bfloat16_rn(wyN);
    }
}

// Corner weights of cell t (as interp_corners_item), delta at the corner
// (from its edge neighbours' delta) and delta = 0 at the cell's C point.
template <class Src>
__device__ __forceinline__ void interp_corners_item_f(const Src& src, int sc, unsigned t, float* P,
                                                      __nv_bfloat16* P16, float* delta) {
    const int nc1 = sc + 1, sf = 2 * sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    const int I = (int)(t % (unsigned)nc1), J = (int)(t / (unsigned)nc1);
    float a[9], s;
    src.row(2 * I, 2 * J, a, &s);
    const size_t cW = t - 1, cS = t - nc1;
    const float yS_W = I >= 1 ? P[PYS * ncell + cW] : 0.0f, yN_W = I >= 1 ? P[PYN * ncell + cW] : 0.0f;
    const float yS_E = I < sc ? P[PYS * ncell + t] : 0.0f, yN_E = I < sc ? P[PYN * ncell + t] : 0.0f;
    const float xW_S = J >= 1 ? P[PXW * ncell + cS] : 0.0f, xE_S = J >= 1 ? P[PXE * ncell + cS] : 0.0f;
    const float xW_N = J < sc ? P[PXW * ncell + t] : 0.0f, xE_N = J < sc ? P[PXE * ncell + t] : 0.0f;
    // delta of the four edge neighbours (2I -+ 1, 2J) and (2I, 2J -+ 1)
    const float dW = I >= 1 ? delta[(size_t)(2 * J) * sf + 2 * I - 1] : 0.0f;
    const float dE = I < sc ? delta[(size_t)(2 * J) * sf + 2 * I + 1] : 0.0f;
    const float dS = J >= 1 ? delta[(size_t)(2 * J - 1) * sf + 2 * I] : 0.0f;
    const float dN = J < sc ? delta[(size_t)(2 * J + 1) * sf + 2 * I] : 0.0f;
    float wSW = 0, wSE = 0, wNW = 0, wNE = 0, d = -1.0f;
    if (a[DC] > 0) {
        const float inv = 1.0f / a[DC];
        wSW = -(a[DSW] + a[DW] * yS_W + a[DS] * xW_S) * inv;
        wSE = -(a[DSE] + a[DE] * yS_E + a[DS] * xE_S) * inv;
        wNW = -(a[DNW] + a[DW] * yN_W + a[DN] * xW_N) * inv;
        wNE = -(a[DNE] + a[DE] * yN_E + a[DN] * xE_N) * inv;
        d = -(s + a[DW] * dW + a[DE] * dE + a[DS] * dS + a[DN] * dN) * inv;
    }
    delta[(size_t)(2 * J) * sf + 2 * I] = d;
    if (I < sc && J < sc) delta[(size_t)(2 * J + 1) * sf + 2 * I + 1] = 0.0f;
    P[PSW * ncell + t] = wSW;
    P[PSE * ncell + t] = wSE;
    P[PNW * ncell + t] = wNW;
    P[PNE * ncell + t] = wNE;
    if (P16) {
        P16[PSW * ncell + t] = __float2bfloat16_rn(wSW);
        P16[PSE * ncell + t] = __float2bfloat16_rn(wSE);
        P16[PNW * ncell + t] = __float2bfloat16_rn(wNW);
        P16[PNE * ncell + t] = __float2bfloat16_rn(wNE);
    }
}

// delta(g) = (P 1)(g) - 1 at the fine point (gi, gj) in the grid: the stored
// value less the weights towards coarse points outside the grid.
__device__ __forceinline__ float delta_at(const float* P, const float* delta, int sc, int gi,
                                          int gj) {
    const int oi = gi & 1, oj = gj & 1;
    if (oi && oj) return 0.0f;   // C point: interpolates itself
    const int nc1 = sc + 1, sf = 2 * sc + 1;
    const size_t ncell = (size_t)nc1 * nc1;
    const int I = gi >> 1, J = gj >> 1;
    const size_t c = (size_t)J * nc1 + I;
    float d = delta[(size_t)gj * sf + gi];
    if (!oi) {
        if (oj) {            // x-edge: sources (I - 1, J) and (I, J)
            if (I == 0) d -= P[PXW * ncell + c];
            if (I == sc) d -= P[PXE * ncell + c];
        } else {             // corner: sources (I - 1 or I, J - 1 or J)
            const bool w = I == 0, e = I == sc, so = J == 0, no = J == sc;
            if (w || so) d -= P[PSW * ncell + c];
            if (e || so) d -= P[PSE * ncell + c];
            if (w || no) d -= P[PNW * ncell + c];
            if (e || no) d -= P[PNE * ncell + c];
        }
    } else {                 // y-edge: sources (I, J - 1) and (I, J)
        if (J == 0) d -= P[PYS * ncell + c];
        if (J == sc) d -= P[PYN * ncell + c];
    }
    return d;
}

// Galerkin coarse row t in float32 leakage form: Ac[t] = its row sum from
// R (s + A delta), Ac[d * nc + t] = its off-diagonal entries (and A16 their
// bfloat16 copy when given).
template <class Src>
__device__ __forceinline__ void rap_item_f(const Src& src, int sc, unsigned t, const float* P,
                                           const float* delta, float* Ac, __nv_bfloat16* A16) {
    const unsigned nc = (unsigned)sc * sc;
    const int I = (int)(t % (unsigned)sc), J = (int)(t / (unsigned)sc);
    const int sf = 2 * sc + 1;
    float dl[5][5];
#pragma unroll
    for (int qy = -2; qy <= 2; ++qy)
#pragma unroll
        for (int qx = -2; qx <= 2; ++qx) {
            const int gi = 2 * I + 1 + qx, gj = 2 * J + 1 + qy;
            const bool in = gi >= 0 && gj >= 0 && gi < sf && gj < sf;
            dl[qy + 2][qx + 2] = in ? delta_at(P, delta, sc, gi, gj) : 0.0f;
        }
    float acc[9];
#pragma unroll
    for (int d = 0; d < 9; ++d) acc[d] = 0.0f;
    float rowsum = 0.0f;
#pragma unroll
    for (int oy = -1; oy <= 1; ++oy) {
#pragma unroll
        for (int ox = -1; ox <= 1; ++ox) {
            const float R = restrict_weight(P, sc, I, J, ox, oy);
            float a[9], s;
            src.row(2 * I + 1 + ox, 2 * J + 1 + oy, a, &s);
            float inner = s;   // (A (P 1))(f) = s_f + sum_g A(f, g) delta(g)
#pragma unroll
            for (int d = 0; d < 9; ++d) {
                if constexpr (Src::kFivePoint)
                    if (d >= DSW) continue;
                const int qx = ox + dir_di(d), qy = oy + dir_dj(d);
                inner += a[d] * dl[qy + 2][qx + 2];
                const int gi = 2 * I + 1 + qx, gj = 2 * J + 1 + qy;
                if (gi < 0 || gj < 0 || gi >= sf || gj >= sf) continue;
                rap_scatter(P, sc, I, J, qx, qy, R * a[d], acc);
            }
            rowsum += R * inner;
        }
    }
    Ac[t] = rowsum;
#pragma unroll
    for (int d = 1; d < 9; ++d) Ac[d * nc + t] = acc[d];
    if (A16) {
        A16[t] = __float2bfloat16_rn(rowsum);
#pragma unroll
        for (int d = 1; d < 9; ++d) A16[d * nc + t] = __float2bfloat16_rn(acc[d]);
    }
}

// Explicit inverse of the coarsest operator (n = side^2 <= 64) by Gauss-Jordan
// elimination with partial pivoting, by one thread block; M is n x 2n shared
// memory.  *status is set to 1 if a pivot vanished.
template <class Src>
__device__ void coarse_invert_block(const Src& src, int side, double* M, double* inv, int* status) {
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
                const double v = fabs(M[r * w + k]);
                if (v > bv) { bv = v; best = r; }
            }
            piv = best;
            if (bv == 0.0) *status = 1;
        }
        __syncthreads();
        if (piv != k)
            for (int c = threadIdx.x; c < w; c += blockDim.x) {
                const double tmp = M[k * w + c];
                M[k * w + c] = M[piv * w + c];
                M[piv * w + c] = tmp;
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
    __syncthreads();
}

}  // namespace gs
