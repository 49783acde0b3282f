// Algebraic multigrid for the policy-fixed systems of finite games given by
// CSR tables (Sec. 4.3, Algorithm 3), and the policy iteration that uses it
// (AMGpi, Sec. 5.1) for one game on the whole GPU.
//
// Set-up, for the system (I - mu M^{alpha beta}) w = r^{alpha beta} of the
// current policies (its sparsity follows the policies, so every system gets
// its own hierarchy):
//  - strength: j strongly influences i when -a_ij >= theta max_{k != i} -a_ik
//    (the off-diagonal entries of I - mu M are <= 0);
//  - C/F splitting: a parallel maximal independent set of the strength graph
//    (PMIS: weight = number of points a point strongly influences plus a
//    hashed fraction; a local maximum becomes C, the points strongly
//    depending on a new C point become F); optionally followed by the
//    Ruge-Stueben second pass, which promotes to C every F point having a
//    strong F neighbour with which it shares no C point (Ruge-Stueben's
//    condition for interpolation);
//  - extended+i interpolation: an F point interpolates from its strong C
//    neighbours and those of its strong F neighbours, the F neighbours'
//    couplings distributed over the candidates (at most the 4 largest
//    weights kept, rescaled to the row's full sum); a C point copies its
//    coarse value;
//  - restriction R = P^T and the Galerkin coarse operator A_c = R A P,
//    accumulated in float64, each coarse row by one thread in a fixed order;
//  - down to at most 64 unknowns, solved by the coarsest operator's inverse.
// Cycles: V-cycles on the correction of the float64 iterate (float32 in the
// mixed path, rows in leakage form: row sum kept beside the off-diagonals),
// C/F Gauss-Seidel (the C points, then the F points, each set colour by
// colour of a greedy colouring of the matrix graph; reversed after the coarse
// correction), float64 residual and stopping test.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "amg.cuh"
#include "gridsync.cuh"
#include "solver.cuh"

namespace gs {

namespace {

constexpr int kAmgThreads = 256;

// ------------------------------------------------------------------ set-up kernels
// Rows of A = I - mu M for the selected rows (ELL, diagonal first, duplicate
// successors merged) and their float32 leakage copy (row sum in slot 0).
__global__ void k_amg_assemble(GameTables T, const int64_t* __restrict__ sel, double mu, int n, int W,
                               int* __restrict__ col, double* __restrict__ a64, float* __restrict__ a32) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int64_t row = sel[i];
        int64_t k0, k1;
        row_range(T, row, &k0, &k1);
        int* c = col + (size_t)i * W;
        double* a = a64 + (size_t)i * W;
        int m = 1;
        c[0] = i;
        a[0] = 1.0;
        for (int s = 1; s < W; ++s) { c[s] = -1; a[s] = 0.0; }
        for (int64_t k = k0; k < k1; ++k) {
            const int y = T.col[k];
            const double v = -mu * T.prob[k];
            int s = 0;
            while (s < m && c[s] != y) ++s;
            if (s == m) { c[m] = y; a[m] = 0.0; ++m; }
            a[s] += v;
        }
        float* af = a32 + (size_t)i * W;
        af[0] = (float)T.leak[row];
        for (int s = 1; s < W; ++s) af[s] = (float)a[s];
    }
}

// Strong couplings of each row as a bit mask over its ELL slots; lam[j]
// counts the points j strongly influences.
__global__ void k_amg_strength(int n, int W, const int* __restrict__ col, const double* __restrict__ a,
                               double theta, unsigned long long* __restrict__ S, int* __restrict__ lam) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int* c = col + (size_t)i * W;
        const double* v = a + (size_t)i * W;
        double m = 0.0;
        for (int s = 1; s < W; ++s)
            if (c[s] >= 0) m = fmax(m, -v[s]);
        unsigned long long mask = 0;
        if (m > 0.0)
            for (int s = 1; s < W; ++s)
                if (c[s] >= 0 && -v[s] >= theta * m && -v[s] > 0.0) {
                    mask |= 1ull << s;
                    atomicAdd(&lam[c[s]], 1);
                }
        S[i] = mask;
    }
}

// PMIS weight: points strongly influenced plus a fraction hashed from the index.
__device__ __forceinline__ double pmis_weight(int lam, int i) {
    unsigned long long z = (unsigned long long)i * 0x9e3779b97f4a7c15ull + 0x632be59bd9b4e019ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    return (double)lam + (double)(z >> 11) * 0x1.0p-53;
}

// state: 0 undecided, 1 C, 2 F.  Points with no strong coupling either way are F.
__global__ void k_pmis_init(int n, const unsigned long long* __restrict__ S, const int* __restrict__ lam,
                            int8_t* __restrict__ state, double* __restrict__ w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        state[i] = (S[i] == 0 && lam[i] == 0) ? 2 : 0;
        w[i] = pmis_weight(lam[i], i);
    }
}

// Along every strong edge between two undecided points, the one of smaller
// weight is not a local maximum.
__global__ void k_pmis_mark(int n, int W, const int* __restrict__ col, const unsigned long long* __restrict__ S,
                            const int8_t* __restrict__ state, const double* __restrict__ w,
                            int* __restrict__ notmax) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (state[i] != 0) continue;
        const unsigned long long m = S[i];
        for (int s = 1; s < W; ++s) {
            if (!(m >> s & 1ull)) continue;
            const int j = col[(size_t)i * W + s];
            if (state[j] != 0) continue;
            if (w[j] > w[i]) notmax[i] = 1;
            else notmax[j] = 1;
        }
    }
}

__global__ void k_pmis_select(int n, int8_t* __restrict__ state, int* __restrict__ notmax) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (state[i] == 0 && !notmax[i]) state[i] = 1;
        notmax[i] = 0;
    }
}

// Undecided points that strongly depend on a C point become F; counts the rest.
__global__ void k_pmis_fpass(int n, int W, const int* __restrict__ col, const unsigned long long* __restrict__ S,
                             int8_t* __restrict__ state, int* __restrict__ left) {
    int cnt = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (state[i] != 0) continue;
        const unsigned long long m = S[i];
        bool f = false;
        for (int s = 1; s < W && !f; ++s)
            if ((m >> s & 1ull) && state[col[(size_t)i * W + s]] == 1) f = true;
        if (f) state[i] = 2;
        else ++cnt;
    }
    if (cnt) atomicAdd(left, cnt);
}

// Ruge-Stueben second pass: an F point i with a strong F neighbour j that
// depends on none of i's strong C points violates the interpolation
// condition; the pair is resolved by making one of the two a C point (the
// one of larger index, so that both ends of a pair name the same point;
// flags, then applied).
__global__ void k_rs_second(int n, int W, const int* __restrict__ col, const unsigned long long* __restrict__ S,
                            const int8_t* __restrict__ state, int* __restrict__ promote) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (state[i] != 2) continue;
        const int* ci = col + (size_t)i * W;
        const unsigned long long mi = S[i];
        for (int s = 1; s < W; ++s) {
            if (!(mi >> s & 1ull)) continue;
            const int j = ci[s];
            if (state[j] != 2) continue;
            const int* cj = col + (size_t)j * W;
            const unsigned long long mj = S[j];
            // j must strongly depend on one of i's strong C points
            bool common = false;
            for (int p = 1; p < W && !common; ++p) {
                if (!(mi >> p & 1ull) || state[ci[p]] != 1) continue;
                for (int q = 1; q < W; ++q)
                    if ((mj >> q & 1ull) && cj[q] == ci[p]) { common = true; break; }
            }
            if (!common) promote[max(i, j)] = 1;
        }
    }
}

__global__ void k_rs_apply(int n, int8_t* __restrict__ state, int* __restrict__ promote) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (promote[i]) state[i] = 1;
        promote[i] = 0;
    }
}

// Colouring of the matrix graph for the Gauss-Seidel smoother (greedy
// independent sets, Jones-Plassmann): in round k every uncoloured point whose
// hashed weight beats all its uncoloured neighbours' (along either direction
// of a coupling) takes colour k.  Points of one colour are mutually
// uncoupled, so relaxing them together is exactly Gauss-Seidel in colour
// order.
__device__ __forceinline__ unsigned colour_weight(int i) {
    unsigned z = (unsigned)i * 0x9e3779b9u + 0x7f4a7c15u;
    z = (z ^ (z >> 16)) * 0x85ebca6bu;
    z = (z ^ (z >> 13)) * 0xc2b2ae35u;
    z ^= z >> 16;
    return z;
}
__device__ __forceinline__ bool colour_beats(int i, int j) {   // strict total order
    const unsigned wi = colour_weight(i), wj = colour_weight(j);
    return wi != wj ? wi > wj : i > j;
}

__global__ void k_colour_mark(int n, int W, const int* __restrict__ col, const int16_t* __restrict__ colour,
                              int* __restrict__ notmax) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (colour[i] >= 0) continue;
        for (int s = 1; s < W; ++s) {
            const int j = col[(size_t)i * W + s];
            if (j < 0 || j == i || colour[j] >= 0) continue;
            if (colour_beats(j, i)) notmax[i] = 1;
            else notmax[j] = 1;
        }
    }
}

// Round k: local maxima take colour k; counts per (colour, C/F) class and the
// points left uncoloured.
// The points of each smoother class (C or F, colour k) counted, then listed
// (class order: C colours, then F colours; order within a class is free: its
// points are mutually uncoupled).
__global__ void k_class_count(int n, int ncolour, const int16_t* __restrict__ colour,
                              const int8_t* __restrict__ cf, int* __restrict__ cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        atomicAdd(&cnt[(cf[i] == 1 ? 0 : ncolour) + colour[i]], 1);
}
__global__ void k_class_scatter(int n, int ncolour, const int16_t* __restrict__ colour,
                                const int8_t* __restrict__ cf, int* __restrict__ cursor, int* __restrict__ ord) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        ord[atomicAdd(&cursor[(cf[i] == 1 ? 0 : ncolour) + colour[i]], 1)] = i;
}

__global__ void k_colour_select(int n, int k, int16_t* __restrict__ colour, int* __restrict__ notmax,
                                const int8_t* __restrict__ cf, int* __restrict__ cls, int* __restrict__ left) {
    int lc = 0, nC = 0, nF = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (colour[i] < 0) {
            if (!notmax[i]) {
                colour[i] = (int16_t)k;
                if (cf[i] == 1) ++nC;
                else ++nF;
            } else {
                ++lc;
            }
        }
        notmax[i] = 0;
    }
    if (lc) atomicAdd(left, lc);
    if (nC) atomicAdd(&cls[0], nC);
    if (nF) atomicAdd(&cls[1], nF);
}

// Exclusive prefix sum of (state == C) in blocks of 1024, then over the blocks.
constexpr int kScanBlock = 1024;
__global__ void k_scan_local(int n, const int8_t* __restrict__ state, int* __restrict__ idx,
                             int* __restrict__ sums) {
    __shared__ int buf[kScanBlock];
    const int base = blockIdx.x * kScanBlock;
    const int i = base + threadIdx.x;
    buf[threadIdx.x] = i < n && state[i] == 1 ? 1 : 0;
    __syncthreads();
    for (int o = 1; o < kScanBlock; o <<= 1) {
        const int v = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
        __syncthreads();
        buf[threadIdx.x] += v;
        __syncthreads();
    }
    if (i < n) idx[i] = buf[threadIdx.x] - (state[i] == 1 ? 1 : 0);
    if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = buf[kScanBlock - 1];
}

// Block offsets (one block, sequential over at most a few thousand sums).
__global__ void k_scan_sums(int nb, int* __restrict__ sums, int* __restrict__ total) {
    if (threadIdx.x != 0) return;
    int acc = 0;
    for (int b = 0; b < nb; ++b) {
        const int v = sums[b];
        sums[b] = acc;
        acc += v;
    }
    *total = acc;
}

__global__ void k_scan_add(int n, const int8_t* __restrict__ state, const int* __restrict__ sums,
                           int* __restrict__ idx) {
    const int i = blockIdx.x * kScanBlock + threadIdx.x;
    if (i < n) idx[i] = state[i] == 1 ? idx[i] + sums[blockIdx.x] : -1;
}

// Interpolation rows keep at most this many weights: the largest, rescaled
// to the row's full sum (truncation keeps the coarse operators sparse).
constexpr int kPMax = 4;
constexpr int kInterpCap = 64;   // candidate C points of one F row

// Extended+i interpolation of F point i (the classical interpolation widened
// to distance two, for splittings that leave strong F-F couplings without a
// common C point, as PMIS does).  Candidates: i's strong C neighbours and
// those of its strong F neighbours k.  With abar_kl = min(a_kl, 0):
//   w_ij = -(a_ij + sum_k a_ik abar_kj / d_k) / a~_ii,
//   a~_ii = a_ii + sum_{weak, non-candidate m} a_im + sum_k a_ik abar_ki / d_k,
//   d_k = sum_{l candidate} abar_kl + abar_ki
// (a strong F neighbour with d_k = 0 is lumped into the diagonal).  Returns
// the number of candidates (keys/w hold them), -1 if they overflow.
__device__ int ext_interp_row(int i, int W, const int* __restrict__ col, const double* __restrict__ a,
                              const unsigned long long* __restrict__ S, const int8_t* __restrict__ state,
                              int* keys, double* w) {
    const int* ci = col + (size_t)i * W;
    const double* ai = a + (size_t)i * W;
    const unsigned long long mi = S[i];
    int m = 0;
    auto add = [&](int j) {
        for (int q = 0; q < m; ++q)
            if (keys[q] == j) return true;
        if (m == kInterpCap) return false;
        keys[m] = j;
        w[m] = 0.0;
        ++m;
        return true;
    };
    for (int s = 1; s < W; ++s) {
        const int j = ci[s];
        if (j < 0 || !(mi >> s & 1ull)) continue;
        if (state[j] == 1) {
            if (!add(j)) return -1;
        } else {
            const unsigned long long mk = S[j];
            for (int t = 1; t < W; ++t) {
                const int l = col[(size_t)j * W + t];
                if (l >= 0 && (mk >> t & 1ull) && state[l] == 1 && !add(l)) return -1;
            }
        }
    }
    if (m == 0) return 0;
    auto find = [&](int j) {
        for (int q = 0; q < m; ++q)
            if (keys[q] == j) return q;
        return -1;
    };
    double diag = ai[0];
    for (int s = 1; s < W; ++s) {
        const int j = ci[s];
        if (j < 0) continue;
        const int q = find(j);
        if (q >= 0) {
            w[q] += ai[s];
        } else if (!((mi >> s & 1ull) && state[j] != 1)) {
            diag += ai[s];   // weak coupling outside the candidates: lumped
        }
    }
    for (int s = 1; s < W; ++s) {
        const int k = ci[s];
        if (k < 0 || !(mi >> s & 1ull) || state[k] == 1) continue;
        const int* ck = col + (size_t)k * W;
        const double* ak = a + (size_t)k * W;
        double den = 0.0, aki = 0.0;
        for (int t = 1; t < W; ++t) {
            const int l = ck[t];
            if (l < 0) continue;
            const double ab = fmin(ak[t], 0.0);
            if (l == i) aki = ab;
            else if (find(l) >= 0) den += ab;
        }
        den += aki;
        if (den == 0.0) {
            diag += ai[s];
            continue;
        }
        for (int t = 1; t < W; ++t) {
            const int l = ck[t];
            if (l < 0 || l == i) continue;
            const int q = find(l);
            if (q >= 0) w[q] += ai[s] * fmin(ak[t], 0.0) / den;
        }
        diag += ai[s] * aki / den;
    }
    for (int q = 0; q < m; ++q) w[q] = -w[q] / diag;
    return m;
}

// Interpolation: count pass (entries per row after truncation; widest in
// *wmax; candidate overflow counted in *overflow).
__global__ void k_interp_count(int n, int W, const int* __restrict__ col, const double* __restrict__ a,
                               const unsigned long long* __restrict__ S, const int8_t* __restrict__ state,
                               int* __restrict__ wmax, int* __restrict__ overflow) {
    int mx = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int c = 1;
        if (state[i] != 1) {
            int keys[kInterpCap];
            double w[kInterpCap];
            c = ext_interp_row(i, W, col, a, S, state, keys, w);
            if (c < 0) {
                atomicAdd(overflow, 1);
                c = 0;
            }
        }
        mx = max(mx, min(c, kPMax));
    }
    if (mx) atomicMax(wmax, mx);
}

__global__ void k_interp_fill(int n, int W, const int* __restrict__ col, const double* __restrict__ a,
                              const unsigned long long* __restrict__ S, const int8_t* __restrict__ state,
                              const int* __restrict__ cidx, int WP, int* __restrict__ pcol,
                              double* __restrict__ p64, float* __restrict__ p32, int* __restrict__ rcount) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int* pc = pcol + (size_t)i * WP;
        double* pv = p64 + (size_t)i * WP;
        int m = 0;
        if (state[i] == 1) {
            pc[0] = cidx[i];
            pv[0] = 1.0;
            m = 1;
            atomicAdd(&rcount[cidx[i]], 1);
        } else {
            int keys[kInterpCap];
            double w[kInterpCap];
            const int c = ext_interp_row(i, W, col, a, S, state, keys, w);
            if (c > 0) {
                // the kPMax largest weights (ties: first candidate), rescaled to the full sum
                int keep[kPMax];
                int nk = 0;
                double total = 0.0;
                for (int q = 0; q < c; ++q) {
                    total += w[q];
                    if (nk < kPMax) {
                        keep[nk++] = q;
                    } else {
                        int lo = 0;
                        for (int t = 1; t < kPMax; ++t)
                            if (w[keep[t]] < w[keep[lo]]) lo = t;
                        if (w[q] > w[keep[lo]]) keep[lo] = q;
                    }
                }
                double kept = 0.0;
                for (int t = 0; t < nk; ++t) kept += w[keep[t]];
                const double scale = kept != 0.0 ? total / kept : 1.0;
                for (int t = 0; t < nk; ++t) {
                    pc[m] = cidx[keys[keep[t]]];
                    pv[m] = scale * w[keep[t]];
                    atomicAdd(&rcount[pc[m]], 1);
                    ++m;
                }
            }
        }
        for (int s = m; s < WP; ++s) { pc[s] = -1; pv[s] = 0.0; }
        for (int s = 0; s < WP; ++s) p32[(size_t)i * WP + s] = (float)pv[s];
    }
}

__global__ void k_max_int(int n, const int* __restrict__ v, int* __restrict__ out) {
    int m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = max(m, v[i]);
    if (m) atomicMax(out, m);
}

// R = P^T: rows of the coarse level listing (fine point, weight), then each
// row sorted by fine index so that every later sum runs in a fixed order.
__global__ void k_transpose_fill(int n, int WP, const int* __restrict__ pcol, const double* __restrict__ p64,
                                 int WR, int* __restrict__ fillc, int* __restrict__ rcol,
                                 double* __restrict__ r64) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int s = 0; s < WP; ++s) {
            const int J = pcol[(size_t)i * WP + s];
            if (J < 0) break;
            const int pos = atomicAdd(&fillc[J], 1);
            rcol[(size_t)J * WR + pos] = i;
            r64[(size_t)J * WR + pos] = p64[(size_t)i * WP + s];
        }
}

__global__ void k_transpose_sort(int nc, int WR, const int* __restrict__ cnt, int* __restrict__ rcol,
                                 double* __restrict__ r64, float* __restrict__ r32) {
    for (int J = blockIdx.x * blockDim.x + threadIdx.x; J < nc; J += gridDim.x * blockDim.x) {
        int* c = rcol + (size_t)J * WR;
        double* v = r64 + (size_t)J * WR;
        const int m = cnt[J];
        for (int a = 1; a < m; ++a) {
            const int kc = c[a];
            const double kv = v[a];
            int b = a - 1;
            while (b >= 0 && c[b] > kc) { c[b + 1] = c[b]; v[b + 1] = v[b]; --b; }
            c[b + 1] = kc;
            v[b + 1] = kv;
        }
        for (int a = m; a < WR; ++a) { c[a] = -1; v[a] = 0.0; }
        for (int a = 0; a < WR; ++a) r32[(size_t)J * WR + a] = (float)v[a];
    }
}

// Galerkin row I of A_c = R A P, accumulated in float64 in a fixed order:
// fine points of R's row ascending, then A's slots, then P's slots.  count
// pass (write == false): distinct columns only; fill pass: the row in ELL
// form with the diagonal first and the rest in order of first appearance.
// Threads per block of the Galerkin product and the size of each thread's
// hash table over its coarse row's columns (a power of two above the row cap).
constexpr int kRapThreads = 16;
constexpr int kRapHash = 128;
static_assert(kRapHash > kAmgRowCap, "hash table must exceed the row cap");

__global__ void __launch_bounds__(kRapThreads) k_rap(int nc, const AmgLevelArgs F, int Wc, bool write,
                                                     int* __restrict__ wmax, int* __restrict__ overflow,
                                                     int* __restrict__ ccol, double* __restrict__ c64,
                                                     float* __restrict__ c32) {
    // each thread's row lives in shared memory: its columns in order of first
    // appearance (keys, vals) and a hash table column -> position, so that
    // adding a product costs one probe instead of a scan of the row (the sums
    // are formed in the same order as by a scan: the same values)
    __shared__ int s_keys[kRapThreads][kAmgRowCap];
    __shared__ double s_vals[kRapThreads][kAmgRowCap];
    __shared__ int s_hk[kRapThreads][kRapHash];            // column + 1, 0 = empty
    __shared__ unsigned char s_hq[kRapThreads][kRapHash];  // its position in keys/vals
    int* keys = s_keys[threadIdx.x];
    double* vals = s_vals[threadIdx.x];
    int* hk = s_hk[threadIdx.x];
    unsigned char* hq = s_hq[threadIdx.x];
    auto slot = [&](int J) {
        unsigned h = ((unsigned)J * 2654435761u) >> (32 - 7);
        while (hk[h] != 0 && hk[h] != J + 1) h = (h + 1) & (kRapHash - 1);
        return h;
    };
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
        for (int h = 0; h < kRapHash; ++h) hk[h] = 0;
        int m = 1;
        keys[0] = I;
        vals[0] = 0.0;
        {
            const unsigned h = slot(I);
            hk[h] = I + 1;
            hq[h] = 0;
        }
        bool over = false;
        for (int r = 0; r < F.WR; ++r) {
            const int i = F.rcol[(size_t)I * F.WR + r];
            if (i < 0) break;
            const double wi = F.r64[(size_t)I * F.WR + r];
            for (int s = 0; s < F.W; ++s) {
                const int k = F.col[(size_t)i * F.W + s];
                if (k < 0) continue;
                const double wa = wi * F.a64[(size_t)i * F.W + s];
                for (int p = 0; p < F.WP; ++p) {
                    const int J = F.pcol[(size_t)k * F.WP + p];
                    if (J < 0) break;
                    const double add = wa * F.p64[(size_t)k * F.WP + p];
                    const unsigned h = slot(J);
                    int q;
                    if (hk[h] == 0) {
                        if (m == kAmgRowCap) {
                            over = true;
                            continue;
                        }
                        q = m++;
                        keys[q] = J;
                        vals[q] = 0.0;
                        hk[h] = J + 1;
                        hq[h] = (unsigned char)q;
                    } else {
                        q = hq[h];
                    }
                    vals[q] += add;
                }
            }
        }
        if (over) atomicAdd(overflow, 1);
        if (!write) {
            atomicMax(wmax, m);
            continue;
        }
        double rowsum = 0.0;
        for (int q = 0; q < m; ++q) rowsum += vals[q];
        for (int q = 0; q < Wc; ++q) {
            const bool in = q < m;
            ccol[(size_t)I * Wc + q] = in ? keys[q] : -1;
            c64[(size_t)I * Wc + q] = in ? vals[q] : 0.0;
            c32[(size_t)I * Wc + q] = q == 0 ? (float)rowsum : (in ? (float)vals[q] : 0.0f);
        }
    }
}

// Inverse of the coarsest operator (n <= 64) by Gauss-Jordan with partial
// pivoting in one block; status 1 if singular.
// Dynamic shared memory: the n x 2n augmented matrix.
struct Aug {
    double* m;
    int w;
    __device__ double& operator()(int r, int c) const { return m[r * w + c]; }
};

// The augmented matrix lives in shared memory (n <= kAmgInvSmem) or in the
// global scratch gm (larger coarsest levels).
__global__ void k_amg_coarse_inv(int n, int W, const int* __restrict__ col, const double* __restrict__ a,
                                 double* __restrict__ inv, int* __restrict__ status, double* gm) {
    extern __shared__ double msh[];
    const Aug M{gm ? gm : msh, 2 * n};
    __shared__ int piv;
    for (int k = threadIdx.x; k < n * 2 * n; k += blockDim.x) {
        const int r = k / (2 * n), c = k % (2 * n);
        M(r, c) = c >= n && c - n == r ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
        for (int s = 0; s < W; ++s) {
            const int c = col[(size_t)r * W + s];
            if (c >= 0) M(r, c) += a[(size_t)r * W + s];
        }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            int p = k;
            for (int r = k + 1; r < n; ++r)
                if (fabs(M(r, k)) > fabs(M(p, k))) p = r;
            piv = p;
            if (M(p, k) == 0.0) *status = 1;
        }
        __syncthreads();
        if (piv != k)
            for (int c = threadIdx.x; c < 2 * n; c += blockDim.x) {
                const double t = M(k, c);
                M(k, c) = M(piv, c);
                M(piv, c) = t;
            }
        __syncthreads();
        const double d = M(k, k);
        __syncthreads();
        for (int c = threadIdx.x; c < 2 * n; c += blockDim.x) M(k, c) /= d;
        __syncthreads();
        for (int idx = threadIdx.x; idx < n * 2 * n; idx += blockDim.x) {
            const int r = idx / (2 * n), c = idx % (2 * n);
            if (r != k) {
                const double fct = M(r, k);
                if (c != k) M(r, c) -= fct * M(k, c);
            }
        }
        __syncthreads();
        for (int r = threadIdx.x; r < n; r += blockDim.x)
            if (r != k) M(r, k) = 0.0;
        __syncthreads();
    }
    for (int k = threadIdx.x; k < n * n; k += blockDim.x) inv[k] = M(k / n, n + k % n);
}

// ------------------------------------------------------------------ cycles
// (A u)_i and the diagonal: float64 rows hold the entries, float32 rows the
// row sum in slot 0 and the off-diagonals (leakage form).
template <typename T>
__device__ __forceinline__ void amg_row(const AmgLevelArgs& L, int i, const T* u, T* Au, T* d) {
    const int* c = L.col + (size_t)i * L.W;
    if constexpr (sizeof(T) == 8) {
        const double* a = L.a64 + (size_t)i * L.W;
        double s = 0.0;
        for (int k = 0; k < L.W; ++k)
            if (c[k] >= 0) s = fma(a[k], u[c[k]], s);
        *Au = s;
        *d = a[0];
    } else {
        const float* a = L.a32 + (size_t)i * L.W;
        const float ui = u[i];
        float s = a[0] * ui, dg = a[0];
        for (int k = 1; k < L.W; ++k) {
            if (c[k] < 0) continue;
            s = fmaf(a[k], u[c[k]] - ui, s);
            dg -= a[k];
        }
        *Au = s;
        *d = dg;
    }
}

template <typename T>
__device__ __forceinline__ T pw(const AmgLevelArgs& L, size_t k) {
    if constexpr (sizeof(T) == 8) return L.p64[k];
    else return L.p32[k];
}
template <typename T>
__device__ __forceinline__ T rw(const AmgLevelArgs& L, size_t k) {
    if constexpr (sizeof(T) == 8) return L.r64[k];
    else return L.r32[k];
}

// Jacobi relaxation of the C points (which = 1), of the F points (which = 0)
// or of all points (which = 2) (u -> t, the others copied; the splitting
// marks C points 1, F points 2).
template <typename T>
__device__ void amg_relax(const AmgLevelArgs& L, const T* u, T* t, const T* f, int which, size_t gt, size_t gs) {
    for (size_t i = gt; i < (size_t)L.n; i += gs) {
        if (which != 2 && (L.cf[i] == 1) != (which == 1)) {
            t[i] = u[i];
            continue;
        }
        T Au, d;
        amg_row<T>(L, (int)i, u, &Au, &d);
        t[i] = u[i] + (f[i] - Au) / d;
    }
}

// Gauss-Seidel on the points of colour k in the C (which = 1) or F (which =
// 0) set, in place: they are mutually uncoupled.  The class's points are read
// from its list (thread index gt of gs).
template <typename T>
__device__ void amg_gs(const AmgLevelArgs& L, T* u, const T* f, int k, int which, size_t gt, size_t gs) {
    const int key = (which == 1 ? 0 : L.ncolour) + k;
    const size_t b = (size_t)L.kofs[key], e = (size_t)L.kofs[key + 1];
    for (size_t x = b + gt; x < e; x += gs) {
        const int i = L.ord[x];
        T Au, d;
        amg_row<T>(L, i, u, &Au, &d);
        u[i] += (f[i] - Au) / d;
    }
}

// One C/F Gauss-Seidel sweep, colour by colour (C points first when c_first).
// Who runs a phase and how it ends: the whole grid with a grid barrier, or
// thread block 0 alone with a block barrier (small levels).
// gx numbers the threads block-minor (thread t of block b is t * blocks + b),
// so that a short list is spread over all the blocks, not packed into the
// first few.
struct GridPh {
    const GridSync* G;
    size_t gt, gs, gx;
    __device__ bool sync() const { return G->sync(); }
};
struct BlockPh {
    size_t gt, gs, gx;
    __device__ bool sync() const {
        __syncthreads();
        return true;
    }
};

template <typename T, class Ph>
__device__ bool amg_sweep(const AmgLevelArgs& L, T* u, const T* f, bool c_first, const Ph& ph) {
    for (int half = 0; half < 2; ++half) {
        const int which = (half == 0) == c_first ? 1 : 0;
        for (int k = 0; k < L.ncolour; ++k) {
            const unsigned long long m = which ? L.cmaskC[k >> 6] : L.cmaskF[k >> 6];
            if (!(m >> (k & 63) & 1ull)) continue;   // no point of this set has colour k
            amg_gs<T>(L, u, f, k, which, ph.gx, ph.gs);
            if (!ph.sync()) return false;
        }
    }
    return true;
}

// Down leg of level l: C/F relaxation, residual, restriction f_{l+1} = R r_l,
// u_{l+1} = 0.
template <typename T, class Ph>
__device__ bool amg_down(const AmgSolveArgs& a, int l, T* const* u, T* const* t, const Ph& ph) {
    const AmgLevelArgs& L = a.L[l];
    const T* f = (const T*)L.f;
    for (int s = 0; s < a.nu1; ++s)
        if (!amg_sweep<T>(L, u[l], f, true, ph)) return false;
    for (size_t i = ph.gt; i < (size_t)L.n; i += ph.gs) {
        T Au, d;
        amg_row<T>(L, (int)i, u[l], &Au, &d);
        t[l][i] = f[i] - Au;
    }
    if (!ph.sync()) return false;
    const AmgLevelArgs& C = a.L[l + 1];
    T* fc = (T*)C.f;
    for (size_t I = ph.gt; I < (size_t)C.n; I += ph.gs) {
        T acc = 0;
        for (int r = 0; r < L.WR; ++r) {
            const int i = L.rcol[I * L.WR + r];
            if (i < 0) break;
            acc += rw<T>(L, I * L.WR + r) * t[l][i];
        }
        fc[I] = acc;
        u[l + 1][I] = T(0);
    }
    return ph.sync();
}

// Up leg of level l: u_l += P u_{l+1}, then F/C relaxation.
template <typename T, class Ph>
__device__ bool amg_up(const AmgSolveArgs& a, int l, T* const* u, const Ph& ph) {
    const AmgLevelArgs& L = a.L[l];
    const T* f = (const T*)L.f;
    for (size_t i = ph.gt; i < (size_t)L.n; i += ph.gs) {
        T acc = 0;
        for (int p = 0; p < L.WP; ++p) {
            const int J = L.pcol[i * L.WP + p];
            if (J < 0) break;
            acc += pw<T>(L, i * L.WP + p) * u[l + 1][J];
        }
        u[l][i] += acc;
    }
    if (!ph.sync()) return false;
    for (int s = 0; s < a.nu2; ++s)
        if (!amg_sweep<T>(L, u[l], f, false, ph)) return false;
    return true;
}

__device__ __forceinline__ unsigned long long abs_bits64(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// float64 residual of the fine system: rhs - A v, its and v's maxima; the
// correction's right-hand side f0 = r and u0 = 0.
template <typename T>
__device__ void amg_check(const AmgSolveArgs& a, int slot, T* f0, T* u0, size_t gt, size_t gs) {
    const AmgLevelArgs& L = a.L[0];
    unsigned long long rm = 0, vm = 0;
    for (size_t i = gt; i < (size_t)L.n; i += gs) {
        const int* c = L.col + i * L.W;
        const double* av = L.a64 + i * L.W;
        double s = a.rhs[i];
        for (int k = 0; k < L.W; ++k)
            if (c[k] >= 0) s = fma(-av[k], a.v[c[k]], s);
        f0[i] = (T)s;
        u0[i] = T(0);
        rm = max(rm, abs_bits64(s));
        vm = max(vm, abs_bits64(a.v[i]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rm = max(rm, __shfl_xor_sync(0xffffffffu, rm, o));
        vm = max(vm, __shfl_xor_sync(0xffffffffu, vm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&a.out->rmax[slot], rm);
        atomicMax(&a.out->vmax[slot], vm);
    }
}

// V-cycles on the correction of a.v, with the float64 stopping test between
// cycles (same rules as the Isaacs grids' kernel).
// The coarsest level: its inverse applied by the thread block that has
// `inverse_block` set (block 0), or (coarsening stopped early) Jacobi sweeps
// over the phase's threads.
template <typename T, class Ph>
__device__ bool amg_coarsest(const AmgSolveArgs& a, T** u, T** t, double* fs, const Ph& ph, bool inverse_block) {
    const int Lc = a.nlev - 1;
    const AmgLevelArgs& C = a.L[Lc];
    if (a.coarse_sweeps > 0) {
        for (size_t i = ph.gt; i < (size_t)C.n; i += ph.gs) u[Lc][i] = T(0);
        if (!ph.sync()) return false;
        for (int k = 0; k < a.coarse_sweeps; ++k) {
            amg_relax<T>(C, u[Lc], t[Lc], (const T*)C.f, 2, ph.gt, ph.gs);
            T* sw = u[Lc];
            u[Lc] = t[Lc];
            t[Lc] = sw;
            if (!ph.sync()) return false;
        }
        return true;
    }
    if (inverse_block) {
        const T* f = (const T*)C.f;
        for (int k = threadIdx.x; k < C.n; k += blockDim.x) fs[k] = (double)f[k];
        __syncthreads();
        for (int r = threadIdx.x; r < C.n; r += blockDim.x) {
            double acc = 0.0;
            for (int k = 0; k < C.n; ++k) acc += a.inv[(size_t)r * C.n + k] * fs[k];
            u[Lc][r] = (T)acc;
        }
        __syncthreads();
    }
    return true;
}

template <typename T>
__global__ void __launch_bounds__(kAmgThreads) k_amg_cycles(const __grid_constant__ AmgSolveArgs a) {
    __shared__ double fs[kAmgCoarsest];
    const GridSync G{a.bar, gridDim.x};
    const size_t gt = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gs = (size_t)gridDim.x * blockDim.x;
    T* u[kAmgMaxLevels];
    T* t[kAmgMaxLevels];
    for (int l = 0; l < a.nlev; ++l) {
        u[l] = (T*)a.L[l].u;
        t[l] = (T*)a.L[l].t;
    }
    const int Lc = a.nlev - 1;
    int slot = 0;
    amg_check<T>(a, slot, (T*)a.L[0].f, u[0], gt, gs);
    if (!G.sync()) return;
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
        // down legs of the grid-wide levels, then the small levels (a.tail
        // and below) by thread block 0 alone, then the up legs
        const GridPh gp{&G, gt, gs, (size_t)threadIdx.x * gridDim.x + blockIdx.x};
        const int tl = a.tail < Lc ? a.tail : Lc;
        for (int l = 0; l < tl; ++l)
            if (!amg_down<T>(a, l, u, t, gp)) return;
        if (a.tail <= Lc) {
            if (blockIdx.x == 0) {
                const BlockPh bp{threadIdx.x, blockDim.x, threadIdx.x};
                for (int l = a.tail; l < Lc; ++l) amg_down<T>(a, l, u, t, bp);
                amg_coarsest<T>(a, u, t, fs, bp, true);
                for (int l = Lc - 1; l >= a.tail; --l) amg_up<T>(a, l, u, bp);
            }
            if (!G.sync()) return;
        } else {
            if (!amg_coarsest<T>(a, u, t, fs, gp, blockIdx.x == 0)) return;
            if (!G.sync()) return;
        }
        for (int l = tl - 1; l >= 0; --l)
            if (!amg_up<T>(a, l, u, gp)) return;
        // v += e and the next residual check
        for (size_t i = gt; i < (size_t)a.L[0].n; i += gs) a.v[i] += (double)u[0][i];
        if (!G.sync()) return;
        slot ^= 1;
        amg_check<T>(a, slot, (T*)a.L[0].f, u[0], gt, gs);
        if (!G.sync()) return;
    }
}

// Longest row of the tables (entries), for the finest level's ELL width.
__global__ void k_max_rowlen(int64_t rows, const int64_t* __restrict__ row_ptr, int* __restrict__ out) {
    int m = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (int)(row_ptr[r + 1] - row_ptr[r]));
    if (m) atomicMax(out, m);
}

// float32 copy of the value (the improvement's screen reads it).
__global__ void k_v_to_f32(int64_t n, const double* __restrict__ v, float* __restrict__ v32) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v32[i] = f64_to_f32(v[i]);
}

}  // namespace

// ------------------------------------------------------------------ host
AmgHierarchy::AmgHierarchy() = default;
AmgHierarchy::~AmgHierarchy() = default;

namespace {

// Assembly of the policy-fixed system from given policies (warm start):
// sel[x] = row (x, alpha(x), beta(x, alpha(x))), rhs[x] = its reward.
__global__ void k_game_assemble(int64_t n, int m1, int m2, const uint8_t* __restrict__ alpha,
                                const uint8_t* __restrict__ beta, const double* __restrict__ rew,
                                int64_t* __restrict__ sel, double* __restrict__ rhs) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int a = alpha[x];
        const int64_t row = (x * m1 + a) * m2 + beta[x * m1 + a];
        sel[x] = row;
        rhs[x] = rew[row];
    }
}

unsigned grid_for(int64_t n) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
}

struct GamePI {
    int outer = 0, systems = 0, cycles = 0, levels = 0;
    double res = 0.0;
    bool converged = false;
};

// AMGpi (Sec. 5.1) on one finite game: Algorithm 2 with Algorithm 1 inside,
// every policy-fixed system solved by the algebraic multigrid above (its
// hierarchy rebuilt whenever the policies changed), inexact evaluations
// inside the inner loop confirmed at the float64 floor before any stopping
// decision, as on the other paths.  warm: start from the problem's v, alpha
// and beta (Algorithm 4 passes them down); else from v = 0, action 0 and
// MIN's best reply.  Stops when |F(v) - v|_inf <= eps or alpha is unchanged.
GamePI amgpi_game(gs_solver* s, Problem& P, double eps, bool warm) {
    GameProblem& G = *P.game;
    cudaStream_t st = s->st;
    const int64_t n = G.n_total;
    if (n > (int64_t)INT32_MAX / 64) {
        set_last_error("AMG: %lld states is more than this path takes", (long long)n);
        throw Error{GS_EINVAL};
    }
    if (!G.amg_scal) {
        G.amg_scal = P.arena.alloc<int>(8);
        GS_CUDA(cudaMemsetAsync(G.amg_scal, 0, 8 * sizeof(int), st));
        k_max_rowlen<<<grid_for(G.rows), 256, 0, st>>>(G.rows, G.row_ptr, G.amg_scal);
        GS_CHECK_LAUNCH();
        int m = 0;
        GS_CUDA(cudaMemcpyAsync(&m, G.amg_scal, sizeof m, cudaMemcpyDeviceToHost, st));
        GS_CUDA(cudaStreamSynchronize(st));
        G.amg_row_max = m;
    }
    const int W0 = 1 + G.amg_row_max;
    if (W0 > 64) {
        set_last_error("AMG: rows of up to 63 successors (this game has %d)", G.amg_row_max);
        throw Error{GS_EINVAL};
    }
    BatchArgs B{};
    B.T = G.tables();
    B.out = {G.v, G.v32, G.alpha, G.beta, G.sel, G.rhs, G.gstats, G.gres};
    B.count = 1;
    B.max_n = G.max_n;
    B.st_off = G.st_off;
    B.mu = G.mu;
    double mu = 0.0;
    GS_CUDA(cudaMemcpyAsync(&mu, G.mu, sizeof mu, cudaMemcpyDeviceToHost, st));
    int* sc = G.amg_scal;
    int hsc[8];
    auto absmax_v = [&]() {
        GS_CUDA(cudaMemsetAsync(sc + 4, 0, 2 * sizeof(int), st));
        launch_absmax(G.v, (size_t)n, reinterpret_cast<unsigned long long*>(sc + 4), st);
    };
    auto improve = [&](int mode) {
        GS_CUDA(cudaMemsetAsync(sc, 0, 4 * sizeof(int), st));
        launch_game_improve_one(B, mode, n, sc, st);
        GS_CUDA(cudaMemcpyAsync(hsc, sc, sizeof hsc, cudaMemcpyDeviceToHost, st));
        GS_CUDA(cudaStreamSynchronize(st));
        return hsc[0];
    };
    auto sync_v32 = [&]() {
        k_v_to_f32<<<grid_for(n), 256, 0, st>>>(n, G.v, G.v32);
        GS_CHECK_LAUNCH();
    };
    if (warm) {
        sync_v32();
        absmax_v();
        k_game_assemble<<<grid_for(n), 256, 0, st>>>(n, G.m1, G.m2, G.alpha, G.beta, G.rew, G.sel, G.rhs);
        GS_CHECK_LAUNCH();
    } else {
        GS_CUDA(cudaMemsetAsync(G.v, 0, sizeof(double) * n, st));
        GS_CUDA(cudaMemsetAsync(G.v32, 0, sizeof(float) * n, st));
        GS_CUDA(cudaMemsetAsync(G.alpha, 0, (size_t)n, st));
        GS_CUDA(cudaMemsetAsync(G.beta, 0, (size_t)n * G.m1, st));
        absmax_v();
        improve(2);   // MIN's first reply; assembles the first system
    }
    if (!G.amg) G.amg = std::make_unique<AmgHierarchy>();
    AmgHierarchy& H = *G.amg;
    MGState* mgd = s->mgd;
    AmgOut* dout = reinterpret_cast<AmgOut*>(&mgd->out);
    static_assert(sizeof(AmgOut) <= sizeof(SolveOut), "AmgOut lives in the multigrid state");
    AmgOut hout{};
    GamePI R;
    bool capped = false, built = false;
    double lin_res = 0.0, vmax = 0.0;
    auto evaluate = [&](double rel_tol) {
        if (!built) {
            H.build(B.T, G.sel, mu, (int)n, W0, s->opt, st);
            built = true;
        }
        const int why = H.solve(G.v, G.rhs, s->opt, rel_tol, &mgd->bar, dout, &hout, &R.cycles, &lin_res,
                                &vmax, st);
        sync_v32();
        absmax_v();
        return why;
    };
    while (true) {
        for (int j = 0; j < s->opt.max_inner; ++j) {
            const int why = evaluate(s->opt.pi_rtol);
            ++R.systems;
            if (why == 3) { capped = true; break; }
            if (improve(1) != 0) { built = false; continue; }
            if (why == 2) {
                if (evaluate(0.0) == 3) { capped = true; break; }
                if (improve(1) != 0) { built = false; continue; }
            }
            break;
        }
        ++R.outer;
        const int ach = improve(0);
        unsigned long long rb;
        std::memcpy(&rb, hsc + 2, sizeof rb);
        R.res = bits_to_double(rb);
        if (capped) break;
        if (R.res <= eps || ach == 0) {
            R.converged = true;
            break;
        }
        if (R.outer >= s->opt.max_outer) break;
        built = false;   // the outer improvement changed the policies: a new system
    }
    R.levels = (int)H.lv.size();
    return R;
}

}  // namespace

gs_status run_game_fmg(gs_solver* s, gs_solve_stats* stats);

gs_status run_game_amg(gs_solver* s, gs_solve_stats* stats) {
    if (s->opt.fmg) return run_game_fmg(s, stats);
    GameProblem& G = *s->prob->game;
    cudaStream_t st = s->st;
    cudaEvent_t e0, e1;
    GS_CUDA(cudaEventCreate(&e0));
    GS_CUDA(cudaEventCreate(&e1));
    GS_CUDA(cudaEventRecord(e0, st));
    const GamePI R = amgpi_game(s, *s->prob, s->opt.eps, false);
    GS_CUDA(cudaEventRecord(e1, st));
    GS_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    GS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    G.stats_h.assign({R.outer, R.systems, R.cycles, R.converged ? 1 : 0});
    G.res_h.assign({R.res});
    G.shape = 0;
    s->level_stats = {(int)G.n_total, R.outer, R.systems};
    reset_initial(s);
    if (stats) {
        stats->outer = R.outer;
        stats->systems = R.systems;
        stats->cycles = R.cycles;
        stats->levels = R.levels;
        stats->res_inf = R.res;
        stats->res_l2 = 0.0;
        stats->seconds = ms * 1e-3;
        stats->converged = R.converged ? 1 : 0;
        stats->fmg_levels = 0;
    }
    return R.converged ? GS_OK : GS_ENOTCONV;
}

// ------------------------------------------------------------------ algebraic FAMGpi
// Full multilevel policy iteration for a finite game given only by its tables
// (the question Sec. 7 leaves open: Algorithm 4 needs coarse discretisations,
// which a finite game does not have).  This build makes the coarse games
// algebraically, by aggregation:
//  - the mean transition operator of the game, P(x, y) averaged over all
//    action pairs, gives a strength graph; the C/F splitting above (PMIS and
//    the Ruge-Stueben second pass) picks the C points; an F point without a
//    strong C neighbour becomes C;
//  - every C point seeds an aggregate and every F point joins the aggregate
//    of its strongest C neighbour;
//  - the coarse game has the aggregates as states and the same actions and
//    discount: its row (I, a, b) is the average over the members x of I of
//    the row (x, a, b), with successors mapped to their aggregates, and its
//    reward the members' average reward;
//  - the interpolations copy a coarse state's value and policies to its
//    members (the analogues of I and U);
//  - AMGpi runs on every level from the coarsest up, each starting from the
//    interpolated value and policies; coarse levels to the policy fixed
//    point, the finest to options.eps.
// The fixed point reached on the finest level is the game's (it is unique,
// Sec. 2); the coarse levels only provide the starting point.
namespace {

constexpr int kFmgCoarse = 64;      // coarsen games down to about this many states
constexpr int kFmgMaxLevels = 16;

// Rows of the mean operator (diagonal 1, off-diagonals minus the mean
// transition probability), distinct successors merged; count pass first.
__global__ void k_mean_rows(GameTables T, int64_t n, int W, bool write, int* __restrict__ wmax,
                            int* __restrict__ overflow, int* __restrict__ col, double* __restrict__ a) {
    const int R = T.m1 * T.m2;
    const double inv = 1.0 / R;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        int keys[64];
        double vals[64];
        int m = 1;
        keys[0] = (int)x;
        vals[0] = 0.0;
        bool over = false;
        for (int r = 0; r < R; ++r) {
            int64_t k0, k1;
            row_range(T, x * R + r, &k0, &k1);
            for (int64_t k = k0; k < k1; ++k) {
                const int y = T.col[k];
                int q = 0;
                while (q < m && keys[q] != y) ++q;
                if (q == m) {
                    if (m == 64) { over = true; continue; }
                    keys[m] = y;
                    vals[m] = 0.0;
                    ++m;
                }
                vals[q] += T.prob[k] * inv;
            }
        }
        if (over) atomicAdd(overflow, 1);
        if (!write) {
            atomicMax(wmax, m);
            continue;
        }
        for (int q = 0; q < W; ++q) {
            col[x * W + q] = q < m ? keys[q] : -1;
            a[x * W + q] = q == 0 ? 1.0 : (q < m ? -vals[q] : 0.0);
        }
    }
}

// F points without a strong C neighbour become C (every point then has an aggregate).
__global__ void k_promote_lonely(int n, int W, const int* __restrict__ col, const unsigned long long* __restrict__ S,
                                 int8_t* __restrict__ state) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (state[i] == 1) continue;
        bool has = false;
        for (int s = 1; s < W && !has; ++s)
            if ((S[i] >> s & 1ull) && state[col[(size_t)i * W + s]] == 1) has = true;
        if (!has) state[i] = 1;
    }
}

// Aggregate of every point: its own (C) or its strongest strong C neighbour's (F).
__global__ void k_agg_map(int n, int W, const int* __restrict__ col, const double* __restrict__ a,
                          const unsigned long long* __restrict__ S, const int8_t* __restrict__ state,
                          const int* __restrict__ cidx, int* __restrict__ agg, int* __restrict__ cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int g = -1;
        if (state[i] == 1) {
            g = cidx[i];
        } else {
            double best = 0.0;
            for (int s = 1; s < W; ++s) {
                const int j = col[(size_t)i * W + s];
                if (!(S[i] >> s & 1ull) || state[j] != 1) continue;
                if (g < 0 || -a[(size_t)i * W + s] > best) {
                    best = -a[(size_t)i * W + s];
                    g = cidx[j];
                }
            }
        }
        agg[i] = g;
        atomicAdd(&cnt[g], 1);
    }
}

// Members of every aggregate (ELL, ascending).
__global__ void k_agg_fill(int n, const int* __restrict__ agg, int WA, int* __restrict__ fill,
                           int* __restrict__ mem) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int g = agg[i];
        mem[(size_t)g * WA + atomicAdd(&fill[g], 1)] = i;
    }
}

__global__ void k_agg_sort(int nc, int WA, const int* __restrict__ cnt, int* __restrict__ mem) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nc; g += gridDim.x * blockDim.x) {
        int* m = mem + (size_t)g * WA;
        const int c = cnt[g];
        for (int p = 1; p < c; ++p) {
            const int key = m[p];
            int q = p - 1;
            while (q >= 0 && m[q] > key) { m[q + 1] = m[q]; --q; }
            m[q + 1] = key;
        }
        for (int p = c; p < WA; ++p) m[p] = -1;
    }
}

// Row (I, a, b) of the coarse game: the members' rows averaged, successors
// mapped to aggregates (merged in order of first appearance); count pass,
// then fill in uniform-width CSR (padding: the row's own state, probability 0).
__global__ void k_coarse_game(GameTables T, int nc, int WA, const int* __restrict__ mem,
                              const int* __restrict__ cnt, const int* __restrict__ agg, int Wc, bool write,
                              int* __restrict__ wmax, int* __restrict__ overflow, int32_t* __restrict__ ccol,
                              double* __restrict__ cprob, double* __restrict__ crew) {
    const int R = T.m1 * T.m2;
    const int64_t rows = (int64_t)nc * R;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(row / R), r = (int)(row % R);
        const int c = cnt[I];
        const double w = 1.0 / c;
        int keys[64];
        double vals[64];
        int m = 0;
        bool over = false;
        double rew = 0.0;
        for (int p = 0; p < c; ++p) {
            const int64_t x = mem[(size_t)I * WA + p];
            const int64_t frow = x * R + r;
            rew += w * T.rew[frow];
            int64_t k0, k1;
            row_range(T, frow, &k0, &k1);
            for (int64_t k = k0; k < k1; ++k) {
                const int J = agg[T.col[k]];
                int q = 0;
                while (q < m && keys[q] != J) ++q;
                if (q == m) {
                    if (m == 64) { over = true; continue; }
                    keys[m] = J;
                    vals[m] = 0.0;
                    ++m;
                }
                vals[q] += w * T.prob[k];
            }
        }
        if (over) atomicAdd(overflow, 1);
        if (!write) {
            atomicMax(wmax, m);
            continue;
        }
        // an average of probabilities is at most one; the rounding of the
        // members' weights 1/c can leave it an ulp above (all successors in
        // one aggregate): clamped
        for (int q = 0; q < Wc; ++q) {
            ccol[row * Wc + q] = q < m ? keys[q] : I;
            cprob[row * Wc + q] = q < m ? fmin(vals[q], 1.0) : 0.0;
        }
        crew[row] = rew;
    }
}

__global__ void k_row_ptr_uniform(int64_t rows, int W, int64_t* __restrict__ rp) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= rows; r += (int64_t)gridDim.x * blockDim.x)
        rp[r] = r * W;
}

// The interpolations: every fine state takes its aggregate's value and policies.
__global__ void k_fmg_game_interp(int64_t n, int m1, const int* __restrict__ agg, const double* __restrict__ vc,
                                  const uint8_t* __restrict__ ac, const uint8_t* __restrict__ bc,
                                  double* __restrict__ vf, uint8_t* __restrict__ af, uint8_t* __restrict__ bf) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
        const int g = agg[x];
        vf[x] = vc[g];
        af[x] = ac[g];
        for (int a = 0; a < m1; ++a) bf[x * m1 + a] = bc[(size_t)g * m1 + a];
    }
}

}  // namespace

gs_status run_game_fmg(gs_solver* s, gs_solve_stats* stats) {
    cudaStream_t st = s->st;
    Arena tmp(0, 0, st);
    int* scal = tmp.alloc<int>(8);
    int hs[8];
    auto read_scal = [&]() {
        GS_CUDA(cudaMemcpyAsync(hs, scal, sizeof hs, cudaMemcpyDeviceToHost, st));
        GS_CUDA(cudaStreamSynchronize(st));
    };
    cudaEvent_t e0, e1;
    GS_CUDA(cudaEventCreate(&e0));
    GS_CUDA(cudaEventCreate(&e1));
    GS_CUDA(cudaEventRecord(e0, st));
    // coarse games, finest first
    std::vector<Problem*> lev{s->prob.get()};
    std::vector<std::unique_ptr<Problem>> owned;
    std::vector<int*> aggs;   // aggs[l]: aggregate (state of level l + 1) of each state of level l
    const double theta = s->opt.amg_theta > 0 ? s->opt.amg_theta : 0.25;
    while ((int)lev.size() < kFmgMaxLevels) {
        GameProblem& F = *lev.back()->game;
        const int64_t n = F.n_total;
        if (n <= kFmgCoarse) break;
        const GameTables T = F.tables();
        const unsigned g = grid_for(n);
        GS_CUDA(cudaMemsetAsync(scal, 0, sizeof(int) * 8, st));
        k_mean_rows<<<g, 128, 0, st>>>(T, n, 0, false, scal, scal + 1, nullptr, nullptr);
        GS_CHECK_LAUNCH();
        read_scal();
        if (hs[1] || hs[0] > 64) break;   // too many distinct successors for the strength masks
        const int W = hs[0];
        int* col = tmp.alloc<int>((size_t)n * W);
        double* a = tmp.alloc<double>((size_t)n * W);
        k_mean_rows<<<g, 128, 0, st>>>(T, n, W, true, scal, scal + 1, col, a);
        unsigned long long* S = tmp.alloc<unsigned long long>(n);
        int* lam = tmp.alloc<int>(n);
        double* w = tmp.alloc<double>(n);
        int* flag = tmp.alloc<int>(n);
        int8_t* cf = tmp.alloc<int8_t>(n);
        int* cidx = tmp.alloc<int>(n);
        GS_CUDA(cudaMemsetAsync(lam, 0, sizeof(int) * n, st));
        GS_CUDA(cudaMemsetAsync(flag, 0, sizeof(int) * n, st));
        k_amg_strength<<<g, 256, 0, st>>>((int)n, W, col, a, theta, S, lam);
        k_pmis_init<<<g, 256, 0, st>>>((int)n, S, lam, cf, w);
        GS_CHECK_LAUNCH_N(3);
        for (int it = 0; it < 200; ++it) {
            GS_CUDA(cudaMemsetAsync(scal, 0, sizeof(int) * 8, st));
            k_pmis_mark<<<g, 256, 0, st>>>((int)n, W, col, S, cf, w, flag);
            k_pmis_select<<<g, 256, 0, st>>>((int)n, cf, flag);
            k_pmis_fpass<<<g, 256, 0, st>>>((int)n, W, col, S, cf, scal + 2);
            GS_CHECK_LAUNCH_N(3);
            read_scal();
            if (hs[2] == 0) break;
        }
        k_rs_second<<<g, 256, 0, st>>>((int)n, W, col, S, cf, flag);
        k_rs_apply<<<g, 256, 0, st>>>((int)n, cf, flag);
        k_promote_lonely<<<g, 256, 0, st>>>((int)n, W, col, S, cf);
        const int nblk = (int)((n + kScanBlock - 1) / kScanBlock);
        int* sums = tmp.alloc<int>(nblk);
        GS_CUDA(cudaMemsetAsync(scal, 0, sizeof(int) * 8, st));
        k_scan_local<<<nblk, kScanBlock, 0, st>>>((int)n, cf, cidx, sums);
        k_scan_sums<<<1, 32, 0, st>>>(nblk, sums, scal + 3);
        k_scan_add<<<nblk, kScanBlock, 0, st>>>((int)n, cf, sums, cidx);
        GS_CHECK_LAUNCH_N(6);
        read_scal();
        const int nc = hs[3];
        if (nc == 0 || nc > n - n / 8) break;   // no useful coarsening
        int* agg = tmp.alloc<int>(n);
        int* cnt = tmp.alloc<int>(nc);
        GS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * nc, st));
        k_agg_map<<<g, 256, 0, st>>>((int)n, W, col, a, S, cf, cidx, agg, cnt);
        GS_CUDA(cudaMemsetAsync(scal, 0, sizeof(int) * 8, st));
        k_max_int<<<grid_for(nc), 256, 0, st>>>(nc, cnt, scal);
        GS_CHECK_LAUNCH_N(2);
        read_scal();
        const int WA = std::max(1, hs[0]);
        int* mem = tmp.alloc<int>((size_t)nc * WA);
        int* fill = tmp.alloc<int>(nc);
        GS_CUDA(cudaMemsetAsync(fill, 0, sizeof(int) * nc, st));
        k_agg_fill<<<g, 256, 0, st>>>((int)n, agg, WA, fill, mem);
        k_agg_sort<<<grid_for(nc), 256, 0, st>>>(nc, WA, cnt, mem);
        const int64_t crows = (int64_t)nc * F.m1 * F.m2;
        GS_CUDA(cudaMemsetAsync(scal, 0, sizeof(int) * 8, st));
        k_coarse_game<<<grid_for(crows), 128, 0, st>>>(T, nc, WA, mem, cnt, agg, 0, false, scal, scal + 1,
                                                       nullptr, nullptr, nullptr);
        GS_CHECK_LAUNCH_N(3);
        read_scal();
        if (hs[1]) break;   // a coarse row with too many successors: stop here
        const int Wc = std::max(1, hs[0]);
        int64_t* crp = tmp.alloc<int64_t>(crows + 1);
        int32_t* ccol = tmp.alloc<int32_t>((size_t)crows * Wc);
        double* cprob = tmp.alloc<double>((size_t)crows * Wc);
        double* crew = tmp.alloc<double>(crows);
        k_coarse_game<<<grid_for(crows), 128, 0, st>>>(T, nc, WA, mem, cnt, agg, Wc, true, scal, scal + 1,
                                                       ccol, cprob, crew);
        k_row_ptr_uniform<<<grid_for(crows + 1), 256, 0, st>>>(crows, Wc, crp);
        GS_CHECK_LAUNCH_N(2);
        const int64_t off[2] = {0, nc};
        owned.push_back(build_game_problem(s, 1, F.m1, F.m2, off, crp, ccol, cprob, crew, F.mu));
        lev.push_back(owned.back().get());
        aggs.push_back(agg);
    }
    // AMGpi from the coarsest level up
    const int L = (int)lev.size();
    GamePI R;
    s->level_stats.clear();
    std::vector<int> per;
    bool handed = false;   // the level below left a finite iterate to interpolate
    for (int l = L - 1; l >= 0; --l) {
        const bool finest = l == 0;
        if (handed) {
            GameProblem& C = *lev[l + 1]->game;
            GameProblem& F = *lev[l]->game;
            k_fmg_game_interp<<<grid_for(F.n_total), 256, 0, st>>>(F.n_total, F.m1, aggs[l], C.v, C.alpha,
                                                                  C.beta, F.v, F.alpha, F.beta);
            GS_CHECK_LAUNCH();
        }
        const GamePI r = amgpi_game(s, *lev[l], finest ? s->opt.eps : 0.0, handed);
        // a coarse game whose evaluation broke down (a policy pair without
        // exit on an undiscounted coarse game gives a singular system: its
        // iterate is not finite) hands nothing up: the next level starts
        // from the default start
        handed = std::isfinite(r.res);
        per.insert(per.end(), {(int)lev[l]->game->n_total, r.outer, r.systems});
        R.cycles += r.cycles;
        if (finest) {
            R.outer = r.outer;
            R.systems = r.systems;
            R.levels = r.levels;
            R.res = r.res;
            R.converged = r.converged;
        }
        // a coarse level that stops short of its fixed point still hands its
        // iterate up: the coarse games only provide the starting point
    }
    s->level_stats = per;
    GS_CUDA(cudaEventRecord(e1, st));
    GS_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    GS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    GameProblem& G = *s->prob->game;
    G.stats_h.assign({R.outer, R.systems, R.cycles, R.converged ? 1 : 0});
    G.res_h.assign({R.res});
    G.shape = 0;
    reset_initial(s);
    if (stats) {
        stats->outer = R.outer;
        stats->systems = R.systems;
        stats->cycles = R.cycles;
        stats->levels = R.levels;
        stats->res_inf = R.res;
        stats->res_l2 = 0.0;
        stats->seconds = ms * 1e-3;
        stats->converged = R.converged ? 1 : 0;
        stats->fmg_levels = L;
    }
    return R.converged ? GS_OK : GS_ENOTCONV;
}

void AmgHierarchy::build(const GameTables& T, const int64_t* sel, double mu, int n, int W0,
                         const gs_options& opt, cudaStream_t st) {
    const bool mixed = opt.precision != GS_PREC_FP64;
    const size_t tb = mixed ? sizeof(float) : sizeof(double);
    ar = std::make_unique<Arena>(0, 0, st);
    lv.clear();
    auto grid = [](size_t m) { return (unsigned)std::max<size_t>(1, std::min<size_t>((m + 255) / 256, 152 * 16)); };
    int* scal = ar->alloc<int>(8);   // [0] widest row, [1] overflow, [2] points left, [3] C points, [4] status
    int hs[8];
    auto read_scal = [&]() {
        GS_CUDA(cudaMemcpyAsync(hs, scal, sizeof hs, cudaMemcpyDeviceToHost, st));
        GS_CUDA(cudaStreamSynchronize(st));
    };
    // finest level: the selected rows
    AmgLevelMem L0;
    L0.n = n;
    L0.W = W0;
    L0.col = ar->alloc<int>((size_t)n * W0);
    L0.a64 = ar->alloc<double>((size_t)n * W0);
    L0.a32 = ar->alloc<float>((size_t)n * W0);
    k_amg_assemble<<<grid(n), 256, 0, st>>>(T, sel, mu, n, W0, L0.col, L0.a64, L0.a32);
    GS_CHECK_LAUNCH();
    lv.push_back(L0);
    const double theta = opt.amg_theta > 0 ? opt.amg_theta : 0.25;
    while (true) {
        AmgLevelMem& F = lv.back();
        const int nf = F.n;
        F.u = ar->raw_bytes((size_t)nf * tb);
        F.f = ar->raw_bytes((size_t)nf * tb);
        F.t = ar->raw_bytes((size_t)nf * tb);
        F.cf = ar->alloc<int8_t>(nf);
        // stop coarsening at a small level, at the level cap, or where a row is
        // too wide for the strength masks (that level is then relaxed instead
        // of inverted)
        if (nf <= kAmgCoarsest || (int)lv.size() == kAmgMaxLevels || F.W > 64) break;
        // strength, C/F splitting
        unsigned long long* S = ar->alloc<unsigned long long>(nf);
        int* lam = ar->alloc<int>(nf);
        double* w = ar->alloc<double>(nf);
        int* flag = ar->alloc<int>(nf);
        int* cidx = ar->alloc<int>(nf);
        GS_CUDA(cudaMemsetAsync(lam, 0, sizeof(int) * nf, st));
        GS_CUDA(cudaMemsetAsync(flag, 0, sizeof(int) * nf, st));
        k_amg_strength<<<grid(nf), 256, 0, st>>>(nf, F.W, F.col, F.a64, theta, S, lam);
        k_pmis_init<<<grid(nf), 256, 0, st>>>(nf, S, lam, F.cf, w);
        GS_CHECK_LAUNCH_N(2);
        for (int it = 0; it < 200; ++it) {
            GS_CUDA(cudaMemsetAsync(scal, 0, sizeof(int) * 8, st));
            k_pmis_mark<<<grid(nf), 256, 0, st>>>(nf, F.W, F.col, S, F.cf, w, flag);
            k_pmis_select<<<grid(nf), 256, 0, st>>>(nf, F.cf, flag);
            k_pmis_fpass<<<grid(nf), 256, 0, st>>>(nf, F.W, F.col, S, F.cf, scal + 2);
            GS_CHECK_LAUNCH_N(3);
            read_scal();
            if (hs[2] == 0) break;
        }
        if (opt.amg_coarsening == 1) {
            k_rs_second<<<grid(nf), 256, 0, st>>>(nf, F.W, F.col, S, F.cf, flag);
            k_rs_apply<<<grid(nf), 256, 0, st>>>(nf, F.cf, flag);
            GS_CHECK_LAUNCH_N(2);
        }
        // colouring for the Gauss-Seidel smoother, with the (colour, C/F) classes used
        colour_level(F, flag, scal, hs, read_scal, grid(nf), st);
        // coarse numbering and the interpolation's width
        const int nblk = (nf + kScanBlock - 1) / kScanBlock;
        int* sums = ar->alloc<int>(nblk);
        GS_CUDA(cudaMemsetAsync(scal, 0, sizeof(int) * 8, st));
        k_scan_local<<<nblk, kScanBlock, 0, st>>>(nf, F.cf, cidx, sums);
        k_scan_sums<<<1, 32, 0, st>>>(nblk, sums, scal + 3);
        k_scan_add<<<nblk, kScanBlock, 0, st>>>(nf, F.cf, sums, cidx);
        k_interp_count<<<grid(nf), 256, 0, st>>>(nf, F.W, F.col, F.a64, S, F.cf, scal, scal + 1);
        GS_CHECK_LAUNCH_N(4);
        read_scal();
        const int nc = hs[3];
        if (hs[1]) break;                      // interpolation candidates overflow: coarsest here
        if (nc == 0 || nc > nf - nf / 8) break;  // no useful coarser level: this one is the coarsest
        F.WP = std::max(1, hs[0]);
        F.pcol = ar->alloc<int>((size_t)nf * F.WP);
        F.p64 = ar->alloc<double>((size_t)nf * F.WP);
        F.p32 = ar->alloc<float>((size_t)nf * F.WP);
        int* rcount = ar->alloc<int>(nc);
        GS_CUDA(cudaMemsetAsync(rcount, 0, sizeof(int) * nc, st));
        k_interp_fill<<<grid(nf), 256, 0, st>>>(nf, F.W, F.col, F.a64, S, F.cf, cidx, F.WP, F.pcol,
                                                F.p64, F.p32, rcount);
        GS_CUDA(cudaMemsetAsync(scal, 0, sizeof(int) * 8, st));
        k_max_int<<<grid(nc), 256, 0, st>>>(nc, rcount, scal);
        GS_CHECK_LAUNCH_N(2);
        read_scal();
        F.WR = std::max(1, hs[0]);
        F.rcol = ar->alloc<int>((size_t)nc * F.WR);
        F.r64 = ar->alloc<double>((size_t)nc * F.WR);
        F.r32 = ar->alloc<float>((size_t)nc * F.WR);
        GS_CUDA(cudaMemsetAsync(rcount, 0, sizeof(int) * nc, st));
        k_transpose_fill<<<grid(nf), 256, 0, st>>>(nf, F.WP, F.pcol, F.p64, F.WR, rcount, F.rcol, F.r64);
        k_transpose_sort<<<grid(nc), 256, 0, st>>>(nc, F.WR, rcount, F.rcol, F.r64, F.r32);
        GS_CHECK_LAUNCH_N(2);
        // Galerkin coarse operator: count pass, then fill
        const AmgLevelArgs FA = args_of(F);
        GS_CUDA(cudaMemsetAsync(scal, 0, sizeof(int) * 8, st));
        const unsigned rap_blocks = (unsigned)std::max(1, std::min((nc + kRapThreads - 1) / kRapThreads, 152 * 64));
        k_rap<<<rap_blocks, kRapThreads, 0, st>>>(nc, FA, 0, false, scal, scal + 1, nullptr, nullptr, nullptr);
        GS_CHECK_LAUNCH();
        read_scal();
        if (hs[1]) break;   // a Galerkin row too wide: relax this level as the coarsest
        AmgLevelMem C;
        C.n = nc;
        C.W = hs[0];
        C.col = ar->alloc<int>((size_t)nc * C.W);
        C.a64 = ar->alloc<double>((size_t)nc * C.W);
        C.a32 = ar->alloc<float>((size_t)nc * C.W);
        k_rap<<<rap_blocks, kRapThreads, 0, st>>>(nc, FA, C.W, true, scal, scal + 1, C.col, C.a64, C.a32);
        GS_CHECK_LAUNCH();
        lv.push_back(C);
    }
    // coarsest level: its inverse, or relaxation sweeps where coarsening stopped early
    AmgLevelMem& Lc = lv.back();
    coarse_n = Lc.n;
    coarse_sweeps = 0;
    if (Lc.n > kAmgCoarsest) {
        coarse_sweeps = kAmgCoarseSweeps;
        inv = nullptr;
        return;
    }
    inv = ar->alloc<double>((size_t)Lc.n * Lc.n);
    GS_CUDA(cudaMemsetAsync(scal, 0, sizeof(int) * 8, st));
    static bool attr = false;
    if (!attr) {
        GS_CUDA(cudaFuncSetAttribute(k_amg_coarse_inv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(2 * kAmgInvSmem * kAmgInvSmem * sizeof(double))));
        attr = true;
    }
    const bool in_smem = Lc.n <= kAmgInvSmem;
    double* gm = in_smem ? nullptr : ar->alloc<double>(2 * (size_t)Lc.n * Lc.n);
    k_amg_coarse_inv<<<1, in_smem ? 256 : 1024, in_smem ? 2 * (size_t)Lc.n * Lc.n * sizeof(double) : 0, st>>>(
        Lc.n, Lc.W, Lc.col, Lc.a64, inv, scal + 4, gm);
    GS_CHECK_LAUNCH();
    read_scal();
    if (hs[4]) {
        set_last_error("AMG: the coarsest operator is singular");
        throw Error{GS_EINVAL};
    }
}

template <class Read>
void AmgHierarchy::colour_level(AmgLevelMem& F, int* flag, int* scal, int* hs, Read&& read_scal, unsigned g,
                                cudaStream_t st) {
    const int nf = F.n;
    F.colour = ar->alloc<int16_t>(nf);
    GS_CUDA(cudaMemsetAsync(F.colour, 0xff, sizeof(int16_t) * nf, st));   // -1: uncoloured
    GS_CUDA(cudaMemsetAsync(flag, 0, sizeof(int) * nf, st));
    std::memset(F.cmaskC, 0, sizeof F.cmaskC);
    std::memset(F.cmaskF, 0, sizeof F.cmaskF);
    F.ncolour = 0;
    for (int k = 0; k < kAmgMaxColours; ++k) {
        GS_CUDA(cudaMemsetAsync(scal, 0, sizeof(int) * 8, st));
        k_colour_mark<<<g, 256, 0, st>>>(nf, F.W, F.col, F.colour, flag);
        k_colour_select<<<g, 256, 0, st>>>(nf, k, F.colour, flag, F.cf, scal + 5, scal + 2);
        GS_CHECK_LAUNCH_N(2);
        read_scal();
        if (hs[5]) F.cmaskC[k >> 6] |= 1ull << (k & 63);
        if (hs[6]) F.cmaskF[k >> 6] |= 1ull << (k & 63);
        F.ncolour = k + 1;
        if (hs[2] == 0) break;
    }
    if (hs[2] != 0) {
        set_last_error("AMG: more than %d colours needed for the smoother", kAmgMaxColours);
        throw Error{GS_EINVAL};
    }
    // the points listed by class, so that a colour phase visits only its own
    const int nk = 2 * F.ncolour;
    int* cnt = ar->alloc<int>(nk);
    GS_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * nk, st));
    k_class_count<<<g, 256, 0, st>>>(nf, F.ncolour, F.colour, F.cf, cnt);
    GS_CHECK_LAUNCH();
    std::vector<int> hc(nk), ofs(nk + 1, 0);
    GS_CUDA(cudaMemcpyAsync(hc.data(), cnt, sizeof(int) * nk, cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < nk; ++k) ofs[k + 1] = ofs[k] + hc[k];
    F.kofs = ar->alloc<int>(nk + 1);
    F.ord = ar->alloc<int>(std::max(1, nf));
    GS_CUDA(cudaMemcpyAsync(F.kofs, ofs.data(), sizeof(int) * (nk + 1), cudaMemcpyHostToDevice, st));
    GS_CUDA(cudaMemcpyAsync(cnt, ofs.data(), sizeof(int) * nk, cudaMemcpyHostToDevice, st));
    k_class_scatter<<<g, 256, 0, st>>>(nf, F.ncolour, F.colour, F.cf, cnt, F.ord);
    GS_CHECK_LAUNCH();
    GS_CUDA(cudaStreamSynchronize(st));   // the host offsets' buffer is released on return
}

AmgLevelArgs AmgHierarchy::args_of(const AmgLevelMem& m) {
    AmgLevelArgs A{};
    A.n = m.n;
    A.W = m.W;
    A.col = m.col;
    A.a64 = m.a64;
    A.a32 = m.a32;
    A.WP = m.WP;
    A.pcol = m.pcol;
    A.p64 = m.p64;
    A.p32 = m.p32;
    A.WR = m.WR;
    A.rcol = m.rcol;
    A.r64 = m.r64;
    A.r32 = m.r32;
    A.cf = m.cf;
    A.ord = m.ord;
    A.kofs = m.kofs;
    A.ncolour = m.ncolour;
    A.cmaskC[0] = m.cmaskC[0];
    A.cmaskC[1] = m.cmaskC[1];
    A.cmaskF[0] = m.cmaskF[0];
    A.cmaskF[1] = m.cmaskF[1];
    A.u = m.u;
    A.f = m.f;
    A.t = m.t;
    return A;
}

int AmgHierarchy::solve(double* v, const double* rhs, const gs_options& opt, double rel_tol,
                        GridBarrier* bar_state, AmgOut* dout, AmgOut* hout, int* cycles, double* res,
                        double* vmax, cudaStream_t st) {
    const bool mixed = opt.precision != GS_PREC_FP64;
    AmgSolveArgs a{};
    a.nlev = (int)lv.size();
    a.nu1 = std::max(1, opt.nu1);
    a.nu2 = std::max(1, opt.nu2);
    a.max_cycles = opt.max_cycles;
    a.mixed = mixed;
    a.lin_tol = opt.lin_tol;
    a.rel_tol = rel_tol;
    a.rhs = rhs;
    a.v = v;
    a.inv = inv;
    a.coarse_sweeps = coarse_sweeps;
    // the small levels' phases are short: one block with block barriers beats
    // the grid barrier there (needs the coarsest inverse: the Jacobi sweeps
    // swap their vectors per thread)
    a.tail = a.nlev;
    if (coarse_sweeps == 0)
        while (a.tail > 0 && lv[a.tail - 1].n <= kAmgTailN) --a.tail;
    a.bar = bar_state;
    a.out = dout;
    for (int l = 0; l < a.nlev; ++l) a.L[l] = args_of(lv[l]);
    static int per_sm[2] = {0, 0}, sms = 0;
    if (!sms) {
        int dev = 0;
        GS_CUDA(cudaGetDevice(&dev));
        GS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[0], k_amg_cycles<float>, kAmgThreads, 0));
        GS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm[1], k_amg_cycles<double>, kAmgThreads, 0));
    }
    const int ps = std::max(1, per_sm[mixed ? 0 : 1]);
    int nb = (int)std::min<size_t>((size_t)ps * sms, ((size_t)lv[0].n + kAmgThreads - 1) / kAmgThreads);
    if (opt.grid_blocks > 0) nb = std::min(nb, opt.grid_blocks);
    if (a.tail == 0) nb = 1;   // the whole hierarchy is small
    nb = std::max(1, nb);
    GS_CUDA(cudaMemsetAsync(bar_state, 0, sizeof(GridBarrier), st));
    GS_CUDA(cudaMemsetAsync(dout, 0, sizeof(AmgOut), st));
    void* args[] = {(void*)&a};
    const void* fn = mixed ? (const void*)k_amg_cycles<float> : (const void*)k_amg_cycles<double>;
    GS_CUDA(cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(kAmgThreads), args, 0, st));
    note_launches(1);
    GridBarrier hb{};
    GS_CUDA(cudaMemcpyAsync(&hb, bar_state, sizeof hb, cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaMemcpyAsync(hout, dout, sizeof(AmgOut), cudaMemcpyDeviceToHost, st));
    GS_CUDA(cudaStreamSynchronize(st));
    if (hb.error) {
        set_last_error("AMG solve: a grid barrier wait timed out");
        throw Error{GS_ETIMEOUT};
    }
    *cycles += hout->cycles;
    *res = hout->res;
    *vmax = hout->vmax_final;
    return hout->reason;
}

}  // namespace gs
