// tv.cu -- proximal step of a total-variation penalty with non-negativity,
// for the accelerated reconstruction (penalised least squares with the
// matched pair, the use the paper names in Sec. 8).
//
//   x = argmin_{x >= 0} 1/2 ||x - b||^2 + tau TV(x),
//   TV(x) = sum_i |grad x_i| (isotropic; forward differences, zero at the
//   last index of each axis),
//
// by the fast gradient projection of Beck and Teboulle on the dual field p
// (three components, |p| <= 1 pointwise): with x(r) = max(0, b + tau div r),
//   p_k = P(r_k + grad x(r_k) / (12 tau)),  r_{k+1} = p_k + c_k (p_k - p_{k-1}),
// c_k = (t_k - 1) / t_{k+1}, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, and the
// answer x(p_K).  div is minus the adjoint of grad.  Each inner iteration is
// two grid passes (x from r; p and r from x), coalesced along x.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "pact.h"

namespace {

__device__ __forceinline__ float div_at(const float* __restrict__ r, size_t N, int x, int y, int z, int nx, int ny,
                                        int nz, size_t i) {
    const size_t sy = nx, sz = (size_t)nx * ny;
    float d = 0.f;
    if (x < nx - 1) d += r[i];
    if (x > 0) d -= r[i - 1];
    if (y < ny - 1) d += r[N + i];
    if (y > 0) d -= r[N + i - sy];
    if (z < nz - 1) d += r[2 * N + i];
    if (z > 0) d -= r[2 * N + i - sz];
    return d;
}

// x = max(0, b + tau div r)
__global__ void k_tv_primal(const float* __restrict__ b, const float* __restrict__ r, float* __restrict__ x,
                            int nx, int ny, int nz, float tau) {
    const size_t N = (size_t)nx * ny * nz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const int xi = (int)(i % nx), yi = (int)((i / nx) % ny), zi = (int)(i / ((size_t)nx * ny));
        x[i] = fmaxf(0.f, b[i] + tau * div_at(r, N, xi, yi, zi, nx, ny, nz, i));
    }
}

// p = P(r + step grad x); r = p + c (p - p_prev); p_prev = p
__global__ void k_tv_dual(const float* __restrict__ x, float* __restrict__ r, float* __restrict__ pprev, int nx,
                          int ny, int nz, float step, float c) {
    const size_t N = (size_t)nx * ny * nz;
    const size_t sy = nx, sz = (size_t)nx * ny;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        const int xi = (int)(i % nx), yi = (int)((i / nx) % ny), zi = (int)(i / sz);
        const float xc = x[i];
        const float g0 = xi < nx - 1 ? x[i + 1] - xc : 0.f;
        const float g1 = yi < ny - 1 ? x[i + sy] - xc : 0.f;
        const float g2 = zi < nz - 1 ? x[i + sz] - xc : 0.f;
        const float q0 = r[i] + step * g0, q1 = r[N + i] + step * g1, q2 = r[2 * N + i] + step * g2;
        const float s = 1.0f / fmaxf(1.0f, sqrtf(q0 * q0 + q1 * q1 + q2 * q2));
        const float p0 = q0 * s, p1 = q1 * s, p2 = q2 * s;
        r[i] = p0 + c * (p0 - pprev[i]);
        r[N + i] = p1 + c * (p1 - pprev[N + i]);
        r[2 * N + i] = p2 + c * (p2 - pprev[2 * N + i]);
        pprev[i] = p0;
        pprev[N + i] = p1;
        pprev[2 * N + i] = p2;
    }
}

unsigned grid_for(size_t n) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (unsigned)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, (size_t)sms * 8));
}

}  // namespace

void pact_note_error(const std::string& msg);

extern "C" int pact_tv_prox_nn(const float* b, float* x, int nx, int ny, int nz, float tau, int iters, float* work,
                               void* stream) {
    if (!b || !x || !work || nx < 1 || ny < 1 || nz < 1 || iters < 0 || !(tau >= 0.f)) {
        pact_note_error("pact_tv_prox_nn: NULL pointer, empty grid, iters < 0 or tau < 0");
        return PACT_EINVAL;
    }
    const size_t N = (size_t)nx * ny * nz;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned g = grid_for(N);
    float* r = work;
    float* pprev = work + 3 * N;
    if (cudaMemsetAsync(work, 0, 6 * N * sizeof(float), st) != cudaSuccess) {
        pact_note_error("pact_tv_prox_nn: clearing the work array failed");
        return PACT_ECUDA;
    }
    if (tau > 0.f) {
        const float step = 1.0f / (12.0f * tau);
        double t = 1.0;
        for (int k = 0; k < iters; ++k) {
            const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
            k_tv_primal<<<g, 256, 0, st>>>(b, r, x, nx, ny, nz, tau);
            k_tv_dual<<<g, 256, 0, st>>>(x, r, pprev, nx, ny, nz, step, (float)((t - 1.0) / tn));
            t = tn;
        }
    }
    // the answer from the last dual iterate (zero when tau = 0 or no iteration: projection)
    k_tv_primal<<<g, 256, 0, st>>>(b, pprev, x, nx, ny, nz, tau);
    if (cudaGetLastError() != cudaSuccess) {
        pact_note_error("pact_tv_prox_nn: launch failed");
        return PACT_ECUDA;
    }
    return PACT_OK;
}
