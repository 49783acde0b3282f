// Launchers of the CUDA kernels (host-callable; all asynchronous on `st`).
#pragma once

#include "common.cuh"

namespace gs {

// ------------------------------------------------------------ Isaacs fine level
// xi source of a level whose points are the points (ii, jj) = ((i+1)step-1,
// (j+1)step-1) of a finest grid of side `fine_side`: xi_fine[jj*fine_side+ii]
// if xi_fine is not null, else the SplitMix64 stream `seed` at that index.
struct NoiseSrc {
    const double* xi_fine;
    uint64_t seed;
    int fine_side;
    int step;
};

void launch_isaacs_r0(const IsaacsConsts* K, int side, double kappa, NoiseSrc ns,
                      double* r0, cudaStream_t st);

enum ImproveMode { IMP_OUTER = 0, IMP_INNER = 1, IMP_REPLY = 2 };

// Policy improvement at v (Eq. (eq1)/(ILPI)).  alpha, beta (packed 4 x 8 bits
// per state: beta(x, a) for a = 0..3) are read and updated in place according
// to the mode; code/rhs receive the policy-fixed row codes and right-hand
// side r^{alpha beta} (assembly, Eq. (LSPI)); fv (may be null) receives F(v).
// tau >= 0 is the keep-current tolerance; tau < 0 takes 1e-13 max(1, sc->vmax).
void launch_isaacs_improve(ImproveMode mode, const IsaacsConsts* K, int side, int variant,
                           const double* v, const double* r0, uint8_t* alpha, uint32_t* beta,
                           uint8_t* code, double* rhs, double* fv, DevScalars* sc, double tau,
                           cudaStream_t st);

// Assembly only: code/rhs from alpha and beta.
void launch_isaacs_assemble(const IsaacsConsts* K, int side, const uint8_t* alpha,
                            const uint32_t* beta, const double* r0, uint8_t* code,
                            double* rhs, cudaStream_t st);

// |v|_inf into sc->vmax (sc->vmax must be cleared first).
void launch_absmax(const double* v, size_t n, unsigned long long* out, cudaStream_t st);

// FAMGpi interpolations (Sec. 5.2) from a coarse grid of side sc to 2 sc + 1.
void launch_fmg_interp(int sc, const double* v_c, const uint8_t* alpha_c,
                       const uint32_t* beta_c, const uint8_t* beta4_c, double* v_f,
                       uint8_t* alpha_f, uint32_t* beta_f, uint8_t* beta4_f, cudaStream_t st);

}  // namespace gs
