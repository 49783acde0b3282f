// Shared definitions of the CUDA path (kernels and host orchestration).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "../../include/gamesolve.h"

namespace gs {

// ---------------------------------------------------------------- errors
void set_last_error(const char* fmt, ...);

struct Error {
    gs_status st;
};

#define GS_CUDA(call)                                                           \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) {                                                \
            ::gs::set_last_error("%s:%d %s: %s", __FILE__, __LINE__, #call,     \
                                 cudaGetErrorString(e_));                       \
            throw ::gs::Error{GS_ECUDA};                                        \
        }                                                                       \
    } while (0)

// Counts kernels launched by the library (process-wide) for launch accounting.
void note_launches(int k);
#define GS_CHECK_LAUNCH_N(k)          \
    do {                              \
        ::gs::note_launches(k);       \
        GS_CUDA(cudaGetLastError());  \
    } while (0)
#define GS_CHECK_LAUNCH() GS_CHECK_LAUNCH_N(1)

// ---------------------------------------------------------------- stencils
// Directions of a 9-point stencil on a grid whose first index i (along x1) is
// the fast one: C centre, W (i-1), E (i+1), S (j-1), N (j+1) and diagonals.
enum Dir { DC = 0, DW = 1, DE = 2, DS = 3, DN = 4, DSW = 5, DSE = 6, DNW = 7, DNE = 8 };
__host__ __device__ constexpr int dir_di(int d) {
    return d == DW || d == DSW || d == DNW ? -1 : (d == DE || d == DSE || d == DNE ? 1 : 0);
}
__host__ __device__ constexpr int dir_dj(int d) {
    return d == DS || d == DSW || d == DSE ? -1 : (d == DN || d == DNW || d == DNE ? 1 : 0);
}
__host__ __device__ constexpr int dir_of(int di, int dj) {
    return dj == 0 ? (di == 0 ? DC : (di < 0 ? DW : DE))
                   : (dj < 0 ? (di == 0 ? DS : (di < 0 ? DSW : DSE))
                             : (di == 0 ? DN : (di < 0 ? DNW : DNE)));
}

// Interpolation weights of one coarse cell (I, J), I, J in [0, sc]: the fine
// points (2I, 2J+1) (x-edge, between coarse (I-1,J) and (I,J)), (2I+1, 2J)
// (y-edge, between (I,J-1) and (I,J)) and (2I, 2J) (cell corner, between the
// four coarse points around it).  Stored as P[k * ncell + cell].
enum PW { PXW = 0, PXE = 1, PYS = 2, PYN = 3, PSW = 4, PSE = 5, PNW = 6, PNE = 7 };

// Policy code of a fine Isaacs row: 4 a + b for a, b in {0..3}; 16 = stop.
constexpr int kStopCode = 16;
constexpr int kCodes = 17;

// Constants of one Isaacs grid, resident in device memory.
struct IsaacsConsts {
    int side;
    int variant;          // 0 plain, 1 obstacle
    double h, mu, kappa;  // kappa = 1 - mu, evaluated without cancellation
    // Row of A = I - mu M for each code, in direction order C, W, E, S, N.
    double am[kCodes][5];
    // Transition probabilities per code (a < 4) in the order of the neighbours
    // E (+x1), W (-x1), N (+x2), S (-x2), self.
    double p[16][5];
    // Reward offset (1 - mu) 0.1 (a - b).
    double dr[4][4];
    // float copies of the off-diagonal entries of am (index 1..4 used).
    float amf[kCodes][5];
    float kappa_f;        // kappa rounded to float
    // Factored Shapley rows: mu w0 (no-drift weight), mu delta (half-drift
    // weight), 0.1 kappa (reward per unit of a - b).
    double w0mu, gmu, c01;
    float w0mu_f, gmu_f, c01_f, h_f;   // the same and h rounded to float32 (screening)
};

// Device-side scalars: reductions written by kernels, read by the host once
// per decision.  Non-negative doubles are reduced as their bit patterns.
struct DevScalars {
    unsigned long long vmax;     // |v|_inf (bits)
    unsigned long long res;      // |F(v) - v|_inf or |b - A v|_inf (bits)
    double res_sq;               // sum of squares (statistics only)
    int changed;                 // policy entries changed by an improvement
    int code_changed;            // rows of the policy-fixed system that changed
};

// Quotient and remainder of x by d (1 <= d < 2^14, x < 2^28, so x / d < 2^20)
// from a float32 reciprocal: the float quotient's relative error is at most
// 3 * 2^-24 (rounding of x, of 1/d and of the product), under 0.2 in absolute
// terms, so the truncated quotient is off by at most one and one correction
// step makes it exact.  Replaces 64-bit integer division in the index
// arithmetic of every grid-stride loop.
struct FastDiv {
    unsigned d;
    float inv;
    __device__ __forceinline__ explicit FastDiv(unsigned d_) : d(d_), inv(1.0f / (float)d_) {}
    __device__ __forceinline__ unsigned divmod(unsigned x, unsigned* r) const {
        unsigned q = __float2uint_rz(__uint2float_rn(x) * inv);
        int rem = (int)(x - q * d);
        if (rem < 0) {
            --q;
            rem += (int)d;
        } else if (rem >= (int)d) {
            ++q;
            rem -= (int)d;
        }
        *r = (unsigned)rem;
        return q;
    }
};

// Conversions between binary64 and binary32 done on the integer pipe from
// the IEEE 754 encodings (a float64-pipe conversion costs as much as a float64
// operation on this part).  Both give exactly the hardware conversions'
// results; values whose binary32 image is subnormal, infinite or NaN take the
// hardware conversion, in a function that is not inlined so that the compiler
// cannot turn the rare branch into a conversion every lane executes.
static __device__ __noinline__ float f64_to_f32_hw(double x) { return (float)x; }

// The bit pattern of a double through an opaque move: integer tests on it
// must stay integer operations (a compiler may otherwise fold them back
// into float64 compares, which cost as much as float64 arithmetic here).
__device__ __forceinline__ unsigned long long bits_of(double x) {
    unsigned long long b;
    asm("mov.b64 %0, %1;" : "=l"(b) : "d"(x));
    return b;
}

__device__ __forceinline__ double from_bits(unsigned long long b) {
    double x;
    asm("mov.b64 %0, %1;" : "=d"(x) : "l"(b));
    return x;
}

// p[k] if `in`, else +0.0, chosen on the bit pattern: a select between two
// doubles would otherwise take the float64 pipe.
__device__ __forceinline__ double load_or_zero(const double* p, size_t k, bool in) {
    return from_bits(in ? reinterpret_cast<const unsigned long long*>(p)[k] : 0ull);
}
static __device__ __noinline__ double f32_to_f64_hw(float v) { return (double)v; }

// binary64 -> binary32, round to nearest, ties to even.
__device__ __forceinline__ float f64_to_f32(double x) {
    const unsigned long long b = bits_of(x);
    if ((b << 1) == 0) return __uint_as_float((unsigned)(b >> 32));   // signed zero
    const int e = (int)((b >> 52) & 0x7ff) - 1023 + 127;
    if (e <= 0 || e >= 255) return f64_to_f32_hw(x);
    const unsigned mant = (unsigned)((b >> 29) & 0x7fffff);
    const unsigned rest = (unsigned)(b & 0x1fffffff);   // the 29 bits dropped
    unsigned f = (unsigned)(b >> 32 & 0x80000000u) | ((unsigned)e << 23) | mant;
    if (rest > 0x10000000u || (rest == 0x10000000u && (mant & 1u))) ++f;   // may carry into the exponent
    return __uint_as_float(f);
}

// binary32 -> binary64 (exact).
__device__ __forceinline__ double f32_to_f64(float v) {
    const unsigned b = __float_as_uint(v);
    const unsigned e = (b >> 23) & 0xff;
    if ((b & 0x7fffffffu) == 0) return __hiloint2double((int)(b & 0x80000000u), 0);
    if (e == 0 || e == 255) return f32_to_f64_hw(v);
    const unsigned hi = (b & 0x80000000u) | ((e + (1023 - 127)) << 20) | ((b & 0x7fffffu) >> 3);
    return __hiloint2double((int)hi, (int)((b & 7u) << 29));
}

// Largest Isaacs grid side: keeps every level index below 2^28 (FastDiv).
constexpr int kIsaacsMaxSide = 16383;

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* dst, double v) {
    atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

inline double bits_to_double(unsigned long long b) {
    double d;
    static_assert(sizeof(d) == sizeof(b), "");
    __builtin_memcpy(&d, &b, sizeof d);
    return d;
}

inline unsigned int div_up(size_t a, size_t b) { return (unsigned int)((a + b - 1) / b); }

}  // namespace gs
