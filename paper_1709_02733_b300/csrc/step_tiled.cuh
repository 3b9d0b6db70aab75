// step_tiled.cuh -- host interface of the TMA-staged step kernels.
#pragma once
#include <cuda.h>

#include "pact_internal.cuh"

// one tensor map per array: u (3), sigma (6, Voigt), rho, lambda, mu, alpha
enum { TM_U0 = 0, TM_S0 = 3, TM_RHO = 9, TM_LAM = 10, TM_MU = 11, TM_ALPHA = 12, TM_N = 13 };

struct TmaSet {
    CUtensorMap m[TM_N];
};

// 0 on success; arrays[i] is the device base address of array i (order above)
int make_tma_set(TmaSet* out, float* const* arrays, int nx, int ny, int nz);
void launch_vel_tiled(bool adj, const StepParams& p, const TmaSet& tm, int* err, cudaStream_t st);
void launch_str_tiled(bool adj, const StepParams& p, const TmaSet& tm, int* err, cudaStream_t st);
