// step_tiled.cu -- z-marching, TMA-staged step kernels of H and H^T.
//
// Each block owns a 32 x 8 column tile of the x-y plane and marches through a
// chunk of z planes.  For every plane, one thread issues TMA loads of the
// tile's halo box (40 x 13 points: x0-4..x0+35, y0-2..y0+10) of every input
// array into a ring of shared-memory stages (4 planes deep, so two planes are
// in flight while the block works).  TMA fills points outside the grid with
// zeros, which is exactly the zero padding of the difference operators.
// x and y differences read shared memory; z differences read per-thread
// register queues holding the thread's own column over four planes.
//
// The two kernel families share their stencils:
//   velocity family (3 outputs from 6 stress-like fields):
//     forward  u  <- J u + dt/rho (D+x s11 + D-y s12 + D-z s13, ...)     (Eq. (it) + C-PML)
//     adjoint  u  <- J u - (D+x Q_x + D-y S_xy + D-z S_xz, ...)           (Eq. (backwardstep))
//   stress family (6 outputs from 3 velocity-like fields):
//     forward  s  <- s + dt (lambda tr(e) I + 2 mu e)                     (Eq. (it) + C-PML)
//     adjoint  s  <- s - (D-x R_xx, D+y R_xy + D+x R_yx, ...)             (Eq. (backwardstep))
// where the adjoint fields Q, S (stress side) and R (velocity side) are the
// material-weighted fields of the gather form of the transposed operators
// (see step_direct.cu), computed once per point into shared memory.  The
// deferred J and B tails of the adjoint are as in step_direct.cu.
//
// Requirements: nx % 4 == 0 (TMA global strides are multiples of 16 bytes).
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "pact_internal.cuh"
#include "step_tiled.cuh"
#include "tma.cuh"

namespace tiled {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int BW = TX + 8;      // box columns x0-4 .. x0+TX+3
constexpr int BH = TY + 5;      // box rows    y0-2 .. y0+TY+2
constexpr int BOX = BW * BH;    // 520 floats
constexpr int BOXS = 544;       // box stride in floats (2176 B, 128-B aligned)
constexpr int OX = 4, OY = 2;   // own point offset inside the box
constexpr int D = 4;            // stage ring depth (planes)

template <bool ADJ> struct VelCfg {
    // stage boxes: 0..5 sigma (Voigt), 6 rho, 7 alpha, [8 lambda, 9 mu]
    static constexpr int NB = ADJ ? 10 : 8;
    static constexpr int NDER = ADJ ? 6 : 0;
    static constexpr size_t SMEM = (size_t)(D * NB + NDER) * BOXS * sizeof(float) + D * sizeof(uint64_t);
    __host__ __device__ static constexpr int tm(int b) {
        return b < 6 ? TM_S0 + b : (b == 6 ? TM_RHO : (b == 7 ? TM_ALPHA : (b == 8 ? TM_LAM : TM_MU)));
    }
};

template <bool ADJ> struct StrCfg {
    // stage boxes: 0..2 u; forward: 3 lambda, 4 mu; adjoint: 3 rho
    static constexpr int NB = ADJ ? 4 : 5;
    static constexpr int NDER = ADJ ? 6 : 0;
    static constexpr size_t SMEM = (size_t)(D * NB + NDER) * BOXS * sizeof(float) + D * sizeof(uint64_t);
    __host__ __device__ static constexpr int tm(int b) {
        return b < 3 ? TM_U0 + b : (ADJ ? TM_RHO : (b == 3 ? TM_LAM : TM_MU));
    }
};

// differences on a box (own index o) and on a register queue
__device__ __forceinline__ float dpx(const float* v, int o) {
    return PACT_C1 * (v[o + 1] - v[o]) - PACT_C2 * (v[o + 2] - v[o - 1]);
}
__device__ __forceinline__ float dmx(const float* v, int o) {
    return PACT_C1 * (v[o] - v[o - 1]) - PACT_C2 * (v[o + 1] - v[o - 2]);
}
__device__ __forceinline__ float dpy(const float* v, int o) {
    return PACT_C1 * (v[o + BW] - v[o]) - PACT_C2 * (v[o + 2 * BW] - v[o - BW]);
}
__device__ __forceinline__ float dmy(const float* v, int o) {
    return PACT_C1 * (v[o] - v[o - BW]) - PACT_C2 * (v[o + BW] - v[o - 2 * BW]);
}
// queue q[0..3] holds planes (z-2..z+1) for a half->integer difference or
// (z-1..z+2) for an integer->half difference; both reduce to this form
__device__ __forceinline__ float dq(const float* q) {
    return PACT_C1 * (q[2] - q[1]) - PACT_C2 * (q[3] - q[0]);
}
__device__ __forceinline__ void push(float* q, float h) {
    q[0] = q[1];
    q[1] = q[2];
    q[2] = q[3];
    q[3] = h;
}

__device__ __forceinline__ float frcp(float a) { return __fdividef(1.0f, a); }

// harmonic mean of four values; 0 if any is 0 (1/0 = inf makes the sum inf)
__device__ __forceinline__ float harm4f(float a, float b, float c, float d) {
    return __fdividef(4.0f, frcp(a) + frcp(b) + frcp(c) + frcp(d));
}

__device__ __forceinline__ bool in_slab_plane(int k, int n, int P) {
    return P > 0 && (k < P || k >= n - P - 1);
}

// C-PML table entry, runtime axis: which = 0 (a), 1 (b), 2 (chi)
__device__ __forceinline__ float tabv(const StepParams& p, int axis, int half, int which, int k) {
    return __ldg(p.tab[axis][half][which] + k);
}

// position (axis coordinate k) inside the slab of `axis`? returns slab index or -1
__device__ __forceinline__ long slab_at(const StepParams& p, int axis, int gx, int gy, int gz) {
    const int k = axis == 0 ? gx : (axis == 1 ? gy : gz);
    const int n = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
    const int l = slab_local(k, n, p.P);
    if (l < 0) return -1;
    return (long)slab_index(axis, gx, gy, gz, l, p);
}

struct Ring {
    float* base;
    int NB;
    int pfirst;
    __device__ __forceinline__ float* stage(int plane) const {
        return base + (size_t)(((plane - pfirst) & (D - 1)) * NB) * BOXS;
    }
};

// bounded drain of loads still in flight after a failed wait
__device__ __forceinline__ void drain(uint64_t* bar, int pfrom, int pto, int pfirst) {
    for (int pl = pfrom; pl <= pto; ++pl) {
        const int k = pl - pfirst;
        mbar_wait_bounded(&bar[k & (D - 1)], (k / D) & 1);
    }
}

}  // namespace tiled

using namespace tiled;

// ===========================================================================
// velocity family
// ===========================================================================
template <bool ADJ>
__global__ void __launch_bounds__(NT) k_vel_tiled(StepParams p, const __grid_constant__ TmaSet tm, int zc, int* err) {
    using Cfg = VelCfg<ADJ>;
    extern __shared__ __align__(128) float sm[];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zc0 = blockIdx.z * zc, zc1 = min(zc0 + zc, p.nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool own = x < p.nx && y < p.ny;
    const int pfirst = zc0 - 2, plast = zc1 + 1;
    const Ring ring{sm, Cfg::NB, pfirst};
    float* der = sm + (size_t)D * Cfg::NB * BOXS;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + (size_t)(D * Cfg::NB + Cfg::NDER) * BOXS);
    const int o = (ty + OY) * BW + tx + OX;
    const float dt = p.dt, h = p.inv_dx;
    const int P = p.P;
    const bool tpml = P > 0 && (x0 - 2 < P || x0 + TX + 2 >= p.nx - P - 1 || y0 - 2 < P || y0 + TY + 2 >= p.ny - P - 1);

    if (tid == 0) {
        for (int s = 0; s < D; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
        for (int b = 0; b < Cfg::NB; ++b) tma_prefetch_desc(&tm.m[Cfg::tm(b)]);
    }
    __syncthreads();
    auto issue = [&](int pl) {
        const int k = pl - pfirst;
        float* dst = ring.stage(pl);
        mbar_arrive_expect_tx(&bar[k & (D - 1)], Cfg::NB * BOX * sizeof(float));
        for (int b = 0; b < Cfg::NB; ++b) tma_load_3d(dst + b * BOXS, &tm.m[Cfg::tm(b)], x0 - 4, y0 - 2, pl, &bar[k & (D - 1)]);
    };
    if (tid == 0)
        for (int pl = pfirst; pl < pfirst + D && pl <= plast; ++pl) issue(pl);

    float q33[4] = {0, 0, 0, 0}, q13[4] = {0, 0, 0, 0}, q23[4] = {0, 0, 0, 0};
    const int xc1 = (x + 1 < p.nx) ? 1 : 0;        // clamped +x neighbour offset
    const int yc1 = (y + 1 < p.ny) ? BW : 0;       // clamped +y neighbour offset

    for (int pl = pfirst; pl <= plast; ++pl) {
        const int z = pl - 2;
        const bool out = z >= zc0;
        // own-point values of the output plane, loaded before the wait
        const unsigned g = own ? (unsigned)(((size_t)max(z, 0) * p.ny + y) * p.nx + x) : 0u;
        float u0 = 0.f, u1 = 0.f, u2 = 0.f;
        if (out && own) {
            u0 = p.u[0][g];
            u1 = p.u[1][g];
            u2 = p.u[2][g];
        }
        const int kk = pl - pfirst;
        const bool ok = mbar_wait_bounded(&bar[kk & (D - 1)], (kk / D) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, 1);
            drain(bar, pl, min(plast, max(pfirst + D - 1, pl - 3 + D)), pfirst);
            return;
        }
        const float* sp = ring.stage(pl);
        const float* spm = (pl - 1 >= pfirst) ? ring.stage(pl - 1) : nullptr;
        // ---- queue heads: integer->half field at plane pl, half->integer at pl-1
        if constexpr (!ADJ) {
            push(q33, sp[2 * BOXS + o]);
            push(q13, spm ? spm[4 * BOXS + o] : 0.f);
            push(q23, spm ? spm[3 * BOXS + o] : 0.f);
        } else {
            float h33 = 0.f, h13 = 0.f, h23 = 0.f;
            if (pl >= 0 && pl < p.nz) {
                const float s11 = sp[o], s22 = sp[BOXS + o], s33 = sp[2 * BOXS + o];
                const float lam = sp[8 * BOXS + o], mu2 = 2.0f * sp[9 * BOXS + o];
                const float ltr = lam * (s11 + s22 + s33);
                h33 = dt * (ltr + mu2 * s33);
                if (own && in_slab_plane(pl, p.nz, P)) {
                    const long si = slab_at(p, 2, x, y, pl);
                    const float a = tabv(p, 2, 0, 0, pl), chi = tabv(p, 2, 0, 2, pl);
                    h33 += a * (p.psi[2][2][si] + dt * (ltr + mu2 * chi * s33));
                }
            }
            const int zm = pl - 1;
            if (spm && zm >= 0 && zm < p.nz) {
                const float* mz = spm + 9 * BOXS;                       // mu at plane pl-1
                const float* mz1 = (pl < p.nz) ? sp + 9 * BOXS : mz;     // mu at plane pl (clamped)
                const float m13 = harm4f(mz[o], mz[o + xc1], mz1[o], mz1[o + xc1]);
                const float m23 = harm4f(mz[o], mz[o + yc1], mz1[o], mz1[o + yc1]);
                const float s13 = spm[4 * BOXS + o], s23 = spm[3 * BOXS + o];
                h13 = dt * m13 * s13;
                h23 = dt * m23 * s23;
                if (own && in_slab_plane(zm, p.nz, P)) {
                    const long si = slab_at(p, 2, x, y, zm);
                    const float a = tabv(p, 2, 1, 0, zm), chi = tabv(p, 2, 1, 2, zm);
                    h13 += a * (p.psi[0][2][si] + chi * h13);
                    h23 += a * (p.psi[1][2][si] + chi * h23);
                }
            }
            push(q33, h33);
            push(q13, h13);
            push(q23, h23);
        }

        if (out) {
            const float* sz = ring.stage(z);
            const float* sz1 = (z + 1 < p.nz) ? ring.stage(z + 1) : sz;
            const bool pml = tpml || in_slab_plane(z, p.nz, P);
            const float *XD0, *XD1, *XD2, *YD0, *YD1, *YD2;
            if constexpr (!ADJ) {
                XD0 = sz;             // s11
                XD1 = sz + 5 * BOXS;  // s12
                XD2 = sz + 4 * BOXS;  // s13
                YD0 = sz + 1 * BOXS;  // s22
                YD1 = sz + 5 * BOXS;  // s12
                YD2 = sz + 3 * BOXS;  // s23
            } else {
                // material-weighted stress fields of plane z into shared memory
                float* Qx = der;
                float* Syx = der + BOXS;
                float* Szx = der + 2 * BOXS;
                float* Qy = der + 3 * BOXS;
                float* Sxy = der + 4 * BOXS;
                float* Szy = der + 5 * BOXS;
                const float* m0 = sz + 9 * BOXS;
                const float* m1 = sz1 + 9 * BOXS;
                auto derive = [&](auto PMLT) {
                    constexpr bool PM = decltype(PMLT)::value;
                    // x-differenced: columns OX-2..OX+TX+1, rows OY..OY+TY-1
                    for (int i = tid; i < (TX + 4) * TY; i += NT) {
                        const int bx = OX - 2 + i % (TX + 4), by = OY + i / (TX + 4);
                        const int q = by * BW + bx;
                        const int gx = x0 - 4 + bx, gy = y0 - 2 + by;
                        const bool in = gx >= 0 && gx < p.nx && gy < p.ny;
                        const int qx1 = (gx + 1 < p.nx) ? q + 1 : q;
                        const int qy1 = (gy + 1 < p.ny) ? q + BW : q;
                        const float s11 = sz[q], s22 = sz[BOXS + q], s33 = sz[2 * BOXS + q];
                        const float lam = sz[8 * BOXS + q], mu2 = 2.0f * m0[q];
                        const float ltr = lam * (s11 + s22 + s33);
                        float vq = dt * (ltr + mu2 * s11);
                        const float m12 = harm4f(m0[q], m0[qx1], m0[qy1], m0[(gy + 1 < p.ny) ? qx1 + BW : qx1]);
                        const float m13 = harm4f(m0[q], m0[qx1], m1[q], m1[qx1]);
                        float v12 = dt * m12 * sz[5 * BOXS + q];
                        float v13 = dt * m13 * sz[4 * BOXS + q];
                        if constexpr (PM) {
                            if (in && slab_local(gx, p.nx, P) >= 0) {
                                const long si = slab_at(p, 0, gx, gy, z);
                                const float ai = tabv(p, 0, 0, 0, gx), ci = tabv(p, 0, 0, 2, gx);
                                const float ah = tabv(p, 0, 1, 0, gx), ch = tabv(p, 0, 1, 2, gx);
                                vq += ai * (p.psi[0][0][si] + dt * (ltr + mu2 * ci * s11));
                                v12 += ah * (p.psi[1][0][si] + ch * v12);
                                v13 += ah * (p.psi[2][0][si] + ch * v13);
                            }
                        }
                        Qx[q] = vq;
                        Syx[q] = v12;
                        Szx[q] = v13;
                    }
                    // y-differenced: columns OX..OX+TX-1, rows OY-2..OY+TY+1
                    for (int i = tid; i < TX * (TY + 4); i += NT) {
                        const int bx = OX + i % TX, by = OY - 2 + i / TX;
                        const int q = by * BW + bx;
                        const int gx = x0 - 4 + bx, gy = y0 - 2 + by;
                        const bool in = gx < p.nx && gy >= 0 && gy < p.ny;
                        const int qx1 = (gx + 1 < p.nx) ? q + 1 : q;
                        const int qy1 = (gy + 1 < p.ny) ? q + BW : q;
                        const float s11 = sz[q], s22 = sz[BOXS + q], s33 = sz[2 * BOXS + q];
                        const float lam = sz[8 * BOXS + q], mu2 = 2.0f * m0[q];
                        const float ltr = lam * (s11 + s22 + s33);
                        float vq = dt * (ltr + mu2 * s22);
                        const float m12 = harm4f(m0[q], m0[qx1], m0[qy1], m0[(gx + 1 < p.nx) ? qy1 + 1 : qy1]);
                        const float m23 = harm4f(m0[q], m0[qy1], m1[q], m1[qy1]);
                        float v12 = dt * m12 * sz[5 * BOXS + q];
                        float v23 = dt * m23 * sz[3 * BOXS + q];
                        if constexpr (PM) {
                            if (in && slab_local(gy, p.ny, P) >= 0) {
                                const long si = slab_at(p, 1, gx, gy, z);
                                const float ai = tabv(p, 1, 0, 0, gy), ci = tabv(p, 1, 0, 2, gy);
                                const float ah = tabv(p, 1, 1, 0, gy), ch = tabv(p, 1, 1, 2, gy);
                                vq += ai * (p.psi[1][1][si] + dt * (ltr + mu2 * ci * s22));
                                v12 += ah * (p.psi[0][1][si] + ch * v12);
                                v23 += ah * (p.psi[2][1][si] + ch * v23);
                            }
                        }
                        Qy[q] = vq;
                        Sxy[q] = v12;
                        Szy[q] = v23;
                    }
                };
                if (tpml) derive(std::true_type{});
                else derive(std::false_type{});
                __syncthreads();
                XD0 = Qx;
                XD1 = Syx;
                XD2 = Szx;
                YD0 = Qy;
                YD1 = Sxy;
                YD2 = Szy;
            }
            if (own) {
                // divergence terms of the three components
                float gx0 = dpx(XD0, o), gy0 = dmy(YD1, o), gz0 = dq(q13);   // u^x
                float gx1 = dmx(XD1, o), gy1 = dpy(YD0, o), gz1 = dq(q23);   // u^y
                float gx2 = dmx(XD2, o), gy2 = dmy(YD2, o), gz2 = dq(q33);   // u^z
                const float* r0 = sz + 6 * BOXS;
                const float* a0 = sz + 7 * BOXS;
                const float rb[3] = {0.5f * (r0[o] + r0[o + xc1]), 0.5f * (r0[o] + r0[o + yc1]),
                                     0.5f * (r0[o] + sz1[6 * BOXS + o])};
                const float ab[3] = {0.5f * (a0[o] + a0[o + xc1]), 0.5f * (a0[o] + a0[o + yc1]),
                                     0.5f * (a0[o] + sz1[7 * BOXS + o])};
                float uo[3] = {u0, u1, u2};
                float gsum[3][3] = {{gx0 * h, gy0 * h, gz0 * h}, {gx1 * h, gy1 * h, gz1 * h}, {gx2 * h, gy2 * h, gz2 * h}};
                const int co[3] = {x, y, z};
                const int nn[3] = {p.nx, p.ny, p.nz};
                float res[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    if constexpr (!ADJ) {
                        float acc = gsum[i][0] + gsum[i][1] + gsum[i][2];
                        if (pml) {
#pragma unroll
                            for (int j = 0; j < 3; ++j) {
                                const int l = slab_local(co[j], nn[j], P);
                                if (l >= 0) {
                                    const int hh = (i == j);
                                    const float a = tabv(p, j, hh, 0, co[j]), b = tabv(p, j, hh, 1, co[j]);
                                    const float c = tabv(p, j, hh, 2, co[j]);
                                    float* ph = p.phi[i][j] + slab_index(j, x, y, z, l, p);
                                    const float v = b * (*ph) + a * gsum[i][j];
                                    *ph = v;
                                    acc += c * v;
                                }
                            }
                        }
                        res[i] = (1.0f - dt * ab[i]) * uo[i] + __fdividef(dt, rb[i]) * acc;
                    } else {
                        const float w = __fdividef(dt, rb[i]) * uo[i];
                        if (pml) {
#pragma unroll
                            for (int j = 0; j < 3; ++j) {
                                const int l = slab_local(co[j], nn[j], P);
                                if (l >= 0) {
                                    const int hh = (i == j);
                                    const float b = tabv(p, j, hh, 1, co[j]), c = tabv(p, j, hh, 2, co[j]);
                                    float* ph = p.phi[i][j] + slab_index(j, x, y, z, l, p);
                                    *ph = b * (*ph + c * w);
                                }
                            }
                        }
                        res[i] = (1.0f - dt * ab[i]) * uo[i] - (gsum[i][0] + gsum[i][1] + gsum[i][2]);
                    }
                }
                p.u[0][g] = res[0];
                p.u[1][g] = res[1];
                p.u[2][g] = res[2];
            }
        }
        __syncthreads();
        if (tid == 0 && pl >= zc0 && pl - 2 + D <= plast) issue(pl - 2 + D);
    }
}

// ===========================================================================
// stress family
// ===========================================================================
template <bool ADJ>
__global__ void __launch_bounds__(NT) k_str_tiled(StepParams p, const __grid_constant__ TmaSet tm, int zc, int* err) {
    using Cfg = StrCfg<ADJ>;
    extern __shared__ __align__(128) float sm[];
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int zc0 = blockIdx.z * zc, zc1 = min(zc0 + zc, p.nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool own = x < p.nx && y < p.ny;
    const int pfirst = zc0 - 2, plast = zc1 + 1;
    const Ring ring{sm, Cfg::NB, pfirst};
    float* der = sm + (size_t)D * Cfg::NB * BOXS;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + (size_t)(D * Cfg::NB + Cfg::NDER) * BOXS);
    const int o = (ty + OY) * BW + tx + OX;
    const float dt = p.dt, h = p.inv_dx;
    const int P = p.P;
    const bool tpml = P > 0 && (x0 - 2 < P || x0 + TX + 2 >= p.nx - P - 1 || y0 - 2 < P || y0 + TY + 2 >= p.ny - P - 1);

    if (tid == 0) {
        for (int s = 0; s < D; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
        for (int b = 0; b < Cfg::NB; ++b) tma_prefetch_desc(&tm.m[Cfg::tm(b)]);
    }
    __syncthreads();
    auto issue = [&](int pl) {
        const int k = pl - pfirst;
        float* dst = ring.stage(pl);
        mbar_arrive_expect_tx(&bar[k & (D - 1)], Cfg::NB * BOX * sizeof(float));
        for (int b = 0; b < Cfg::NB; ++b) tma_load_3d(dst + b * BOXS, &tm.m[Cfg::tm(b)], x0 - 4, y0 - 2, pl, &bar[k & (D - 1)]);
    };
    if (tid == 0)
        for (int pl = pfirst; pl < pfirst + D && pl <= plast; ++pl) issue(pl);

    float qx[4] = {0, 0, 0, 0}, qy[4] = {0, 0, 0, 0}, qz[4] = {0, 0, 0, 0};
    const int xc1 = (x + 1 < p.nx) ? 1 : 0;
    const int yc1 = (y + 1 < p.ny) ? BW : 0;

    for (int pl = pfirst; pl <= plast; ++pl) {
        const int z = pl - 2;
        const bool out = z >= zc0;
        const unsigned g = own ? (unsigned)(((size_t)max(z, 0) * p.ny + y) * p.nx + x) : 0u;
        float so[6] = {0, 0, 0, 0, 0, 0};
        if (out && own) {
#pragma unroll
            for (int v = 0; v < 6; ++v) so[v] = p.s[v][g];
        }
        const int kk = pl - pfirst;
        const bool ok = mbar_wait_bounded(&bar[kk & (D - 1)], (kk / D) & 1);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, 1);
            drain(bar, pl, min(plast, max(pfirst + D - 1, pl - 3 + D)), pfirst);
            return;
        }
        const float* sp = ring.stage(pl);
        const float* spm = (pl - 1 >= pfirst) ? ring.stage(pl - 1) : nullptr;
        // ---- queue heads: d_z u^x, d_z u^y are integer->half (plane pl);
        //      d_z u^z is half->integer (plane pl-1)
        if constexpr (!ADJ) {
            push(qx, sp[o]);
            push(qy, sp[BOXS + o]);
            push(qz, spm ? spm[2 * BOXS + o] : 0.f);
        } else {
            float hx = 0.f, hy = 0.f, hz = 0.f;
            if (pl >= 0 && pl < p.nz) {
                const float* r = sp + 3 * BOXS;
                hx = __fdividef(2.0f * dt, r[o] + r[o + xc1]) * sp[o];
                hy = __fdividef(2.0f * dt, r[o] + r[o + yc1]) * sp[BOXS + o];
                if (own && in_slab_plane(pl, p.nz, P)) {
                    const long si = slab_at(p, 2, x, y, pl);
                    const float a = tabv(p, 2, 0, 0, pl), c = tabv(p, 2, 0, 2, pl);
                    hx += a * (p.phi[0][2][si] + c * hx);
                    hy += a * (p.phi[1][2][si] + c * hy);
                }
            }
            const int zm = pl - 1;
            if (spm && zm >= 0 && zm < p.nz) {
                const float* r = spm + 3 * BOXS;
                const float* r1 = (pl < p.nz) ? sp + 3 * BOXS : r;
                hz = __fdividef(2.0f * dt, r[o] + r1[o]) * spm[2 * BOXS + o];
                if (own && in_slab_plane(zm, p.nz, P)) {
                    const long si = slab_at(p, 2, x, y, zm);
                    const float a = tabv(p, 2, 1, 0, zm), c = tabv(p, 2, 1, 2, zm);
                    hz += a * (p.phi[2][2][si] + c * hz);
                }
            }
            push(qx, hx);
            push(qy, hy);
            push(qz, hz);
        }

        if (out) {
            const float* sz = ring.stage(z);
            const float* sz1 = (z + 1 < p.nz) ? ring.stage(z + 1) : sz;
            const bool pml = tpml || in_slab_plane(z, p.nz, P);
            const float *XD0, *XD1, *XD2, *YD0, *YD1, *YD2;
            if constexpr (!ADJ) {
                XD0 = sz;             // u^x  (D-x for s11)
                XD1 = sz + BOXS;      // u^y  (D+x for s12)
                XD2 = sz + 2 * BOXS;  // u^z  (D+x for s13)
                YD0 = sz + BOXS;      // u^y  (D-y for s22)
                YD1 = sz;             // u^x  (D+y for s12)
                YD2 = sz + 2 * BOXS;  // u^z  (D+y for s23)
            } else {
                float* Rxx = der;
                float* Ryx = der + BOXS;
                float* Rzx = der + 2 * BOXS;
                float* Ryy = der + 3 * BOXS;
                float* Rxy = der + 4 * BOXS;
                float* Rzy = der + 5 * BOXS;
                const float* r0 = sz + 3 * BOXS;
                const float* r1 = sz1 + 3 * BOXS;
                auto derive = [&](auto PMLT) {
                    constexpr bool PM = decltype(PMLT)::value;
                    for (int i = tid; i < (TX + 4) * TY; i += NT) {
                        const int bx = OX - 2 + i % (TX + 4), by = OY + i / (TX + 4);
                        const int q = by * BW + bx;
                        const int gx = x0 - 4 + bx, gy = y0 - 2 + by;
                        float wx = 0.f, wy = 0.f, wz = 0.f;
                        if (gx >= 0 && gx < p.nx && gy < p.ny) {
                            const int qx1 = (gx + 1 < p.nx) ? q + 1 : q;
                            const int qy1 = (gy + 1 < p.ny) ? q + BW : q;
                            wx = __fdividef(2.0f * dt, r0[q] + r0[qx1]) * sz[q];
                            wy = __fdividef(2.0f * dt, r0[q] + r0[qy1]) * sz[BOXS + q];
                            wz = __fdividef(2.0f * dt, r0[q] + r1[q]) * sz[2 * BOXS + q];
                            if constexpr (PM) {
                                if (slab_local(gx, p.nx, P) >= 0) {
                                    const long si = slab_at(p, 0, gx, gy, z);
                                    const float ah = tabv(p, 0, 1, 0, gx), ch = tabv(p, 0, 1, 2, gx);
                                    const float ai = tabv(p, 0, 0, 0, gx), ci = tabv(p, 0, 0, 2, gx);
                                    const float vx = wx + ah * (p.phi[0][0][si] + ch * wx);
                                    const float vy = wy + ai * (p.phi[1][0][si] + ci * wy);
                                    const float vz = wz + ai * (p.phi[2][0][si] + ci * wz);
                                    wx = vx;
                                    wy = vy;
                                    wz = vz;
                                }
                            }
                        }
                        Rxx[q] = wx;
                        Ryx[q] = wy;
                        Rzx[q] = wz;
                    }
                    for (int i = tid; i < TX * (TY + 4); i += NT) {
                        const int bx = OX + i % TX, by = OY - 2 + i / TX;
                        const int q = by * BW + bx;
                        const int gx = x0 - 4 + bx, gy = y0 - 2 + by;
                        float wx = 0.f, wy = 0.f, wz = 0.f;
                        if (gx < p.nx && gy >= 0 && gy < p.ny) {
                            const int qx1 = (gx + 1 < p.nx) ? q + 1 : q;
                            const int qy1 = (gy + 1 < p.ny) ? q + BW : q;
                            wx = __fdividef(2.0f * dt, r0[q] + r0[qx1]) * sz[q];
                            wy = __fdividef(2.0f * dt, r0[q] + r0[qy1]) * sz[BOXS + q];
                            wz = __fdividef(2.0f * dt, r0[q] + r1[q]) * sz[2 * BOXS + q];
                            if constexpr (PM) {
                                if (slab_local(gy, p.ny, P) >= 0) {
                                    const long si = slab_at(p, 1, gx, gy, z);
                                    const float ah = tabv(p, 1, 1, 0, gy), ch = tabv(p, 1, 1, 2, gy);
                                    const float ai = tabv(p, 1, 0, 0, gy), ci = tabv(p, 1, 0, 2, gy);
                                    const float vy = wy + ah * (p.phi[1][1][si] + ch * wy);
                                    const float vx = wx + ai * (p.phi[0][1][si] + ci * wx);
                                    const float vz = wz + ai * (p.phi[2][1][si] + ci * wz);
                                    wx = vx;
                                    wy = vy;
                                    wz = vz;
                                }
                            }
                        }
                        Ryy[q] = wy;
                        Rxy[q] = wx;
                        Rzy[q] = wz;
                    }
                };
                if (tpml) derive(std::true_type{});
                else derive(std::false_type{});
                __syncthreads();
                XD0 = Rxx;
                XD1 = Ryx;
                XD2 = Rzx;
                YD0 = Ryy;
                YD1 = Rxy;
                YD2 = Rzy;
            }
            if (own) {
                const float exx = dmx(XD0, o) * h, eyy = dmy(YD0, o) * h, ezz = dq(qz) * h;
                const float exy = dpy(YD1, o) * h;   // d_y of the u^x field
                const float eyx = dpx(XD1, o) * h;   // d_x of the u^y field
                const float exz = dq(qx) * h;        // d_z of the u^x field
                const float ezx = dpx(XD2, o) * h;   // d_x of the u^z field
                const float eyz = dq(qy) * h;        // d_z of the u^y field
                const float ezy = dpy(YD2, o) * h;   // d_y of the u^z field
                float res[6];
                if constexpr (!ADJ) {
                    const float* m0 = sz + 4 * BOXS;
                    const float* m1 = sz1 + 4 * BOXS;
                    const float lam = sz[3 * BOXS + o], mu2 = 2.0f * m0[o];
                    const int oxy = (x + 1 < p.nx) ? ((y + 1 < p.ny) ? o + 1 + BW : o + 1) : (o + yc1);
                    const float m12 = harm4f(m0[o], m0[o + xc1], m0[o + yc1], m0[oxy]);
                    const float m13 = harm4f(m0[o], m0[o + xc1], m1[o], m1[o + xc1]);
                    const float m23 = harm4f(m0[o], m0[o + yc1], m1[o], m1[o + yc1]);
                    float e[3] = {exx, eyy, ezz};
                    float ps[3] = {0.f, 0.f, 0.f}, cs[3] = {0.f, 0.f, 0.f};
                    // shear memory terms: (xy, yx), (xz, zx), (yz, zy)
                    float sh[6] = {exy, eyx, exz, ezx, eyz, ezy};
                    float shp[6] = {0, 0, 0, 0, 0, 0};
                    if (pml) {
                        const int co[3] = {x, y, z};
                        const int nn[3] = {p.nx, p.ny, p.nz};
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const int l = slab_local(co[k], nn[k], P);
                            if (l >= 0) {
                                const float a = tabv(p, k, 0, 0, co[k]), b = tabv(p, k, 0, 1, co[k]);
                                cs[k] = tabv(p, k, 0, 2, co[k]);
                                float* ps_ = p.psi[k][k] + slab_index(k, x, y, z, l, p);
                                const float v = b * (*ps_) + a * e[k];
                                *ps_ = v;
                                ps[k] = v;
                            }
                        }
                        // psi^{ij} on the axis-j slab, half lattice along j
                        const int pi_[6] = {0, 1, 0, 2, 1, 2};
                        const int pj_[6] = {1, 0, 2, 0, 2, 1};
#pragma unroll
                        for (int t = 0; t < 6; ++t) {
                            const int j = pj_[t];
                            const int l = slab_local(co[j], nn[j], P);
                            if (l >= 0) {
                                const float a = tabv(p, j, 1, 0, co[j]), b = tabv(p, j, 1, 1, co[j]);
                                const float c = tabv(p, j, 1, 2, co[j]);
                                float* ps_ = p.psi[pi_[t]][j] + slab_index(j, x, y, z, l, p);
                                const float v = b * (*ps_) + a * sh[t];
                                *ps_ = v;
                                shp[t] = c * v;
                            }
                        }
                    }
                    const float theta = exx + eyy + ezz + ps[0] + ps[1] + ps[2];
                    const float lt = lam * theta;
                    res[0] = so[0] + dt * (lt + mu2 * (exx + cs[0] * ps[0]));
                    res[1] = so[1] + dt * (lt + mu2 * (eyy + cs[1] * ps[1]));
                    res[2] = so[2] + dt * (lt + mu2 * (ezz + cs[2] * ps[2]));
                    res[3] = so[3] + dt * m23 * (eyz + ezy + shp[4] + shp[5]);
                    res[4] = so[4] + dt * m13 * (exz + ezx + shp[2] + shp[3]);
                    res[5] = so[5] + dt * m12 * (exy + eyx + shp[0] + shp[1]);
                } else {
                    if (pml) {
                        // psi <- B~ (psi + Delta^T sigma_old) at the own point
                        const int co[3] = {x, y, z};
                        const int nn[3] = {p.nx, p.ny, p.nz};
                        const float lam = __ldg(p.lam + g), mu2 = 2.0f * __ldg(p.mu + g);
                        const float ltr = lam * (so[0] + so[1] + so[2]);
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const int l = slab_local(co[k], nn[k], P);
                            if (l >= 0) {
                                const float b = tabv(p, k, 0, 1, co[k]), c = tabv(p, k, 0, 2, co[k]);
                                float* ps_ = p.psi[k][k] + slab_index(k, x, y, z, l, p);
                                *ps_ = b * (*ps_ + dt * (ltr + mu2 * c * so[k]));
                            }
                        }
                        const float msh[3] = {mu_shear<3>(x, y, z, p), mu_shear<4>(x, y, z, p), mu_shear<5>(x, y, z, p)};
                        // Voigt 3: (y,z), 4: (x,z), 5: (x,y)
                        const int vi[3] = {1, 0, 0}, vj[3] = {2, 2, 1};
#pragma unroll
                        for (int t = 0; t < 3; ++t) {
                            const float dms = dt * msh[t] * so[3 + t];
#pragma unroll
                            for (int side = 0; side < 2; ++side) {
                                const int i = side ? vj[t] : vi[t], j = side ? vi[t] : vj[t];
                                const int l = slab_local(co[j], nn[j], P);
                                if (l >= 0) {
                                    const float b = tabv(p, j, 1, 1, co[j]), c = tabv(p, j, 1, 2, co[j]);
                                    float* ps_ = p.psi[i][j] + slab_index(j, x, y, z, l, p);
                                    *ps_ = b * (*ps_ + c * dms);
                                }
                            }
                        }
                    }
                    res[0] = so[0] - exx;
                    res[1] = so[1] - eyy;
                    res[2] = so[2] - ezz;
                    res[3] = so[3] - (eyz + ezy);
                    res[4] = so[4] - (exz + ezx);
                    res[5] = so[5] - (exy + eyx);
                }
#pragma unroll
                for (int v = 0; v < 6; ++v) p.s[v][g] = res[v];
            }
        }
        __syncthreads();
        if (tid == 0 && pl >= zc0 && pl - 2 + D <= plast) issue(pl - 2 + D);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// z-chunk length: enough blocks for about two waves of resident blocks
static int chunk_len(const StepParams& p, size_t smem, const void* fn) {
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem);
    const long tiles = (long)((p.nx + TX - 1) / TX) * ((p.ny + TY - 1) / TY);
    const long want = 2L * sms * (per_sm > 0 ? per_sm : 1);
    long chunks = (want + tiles - 1) / tiles;
    chunks = std::max(1L, std::min(chunks, (long)std::max(1, p.nz / 16)));
    return (int)((p.nz + chunks - 1) / chunks);
}

// per (device, kernel, grid) launch configuration, computed once
struct LaunchCache {
    int dev;
    const void* fn;
    int nx, ny, nz;
    int zc;
};

template <class K>
static void launch_tiled(K kernel, size_t smem, const StepParams& p, const TmaSet& tm, int* err, cudaStream_t st) {
    static LaunchCache cache[64];
    static int ncache = 0;
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    int zc = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        for (int i = 0; i < ncache; ++i)
            if (cache[i].dev == dev && cache[i].fn == (const void*)kernel && cache[i].nx == p.nx &&
                cache[i].ny == p.ny && cache[i].nz == p.nz)
                zc = cache[i].zc;
        if (!zc) {
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            zc = chunk_len(p, smem, (const void*)kernel);
            cache[ncache % 64] = {dev, (const void*)kernel, p.nx, p.ny, p.nz, zc};
            ncache = std::min(ncache + 1, 64);
        }
    }
    dim3 grid((p.nx + TX - 1) / TX, (p.ny + TY - 1) / TY, (p.nz + zc - 1) / zc);
    kernel<<<grid, dim3(TX, TY, 1), smem, st>>>(p, tm, zc, err);
}

void launch_vel_tiled(bool adj, const StepParams& p, const TmaSet& tm, int* err, cudaStream_t st) {
    if (adj) launch_tiled(k_vel_tiled<true>, VelCfg<true>::SMEM, p, tm, err, st);
    else launch_tiled(k_vel_tiled<false>, VelCfg<false>::SMEM, p, tm, err, st);
}

void launch_str_tiled(bool adj, const StepParams& p, const TmaSet& tm, int* err, cudaStream_t st) {
    if (adj) launch_tiled(k_str_tiled<true>, StrCfg<true>::SMEM, p, tm, err, st);
    else launch_tiled(k_str_tiled<false>, StrCfg<false>::SMEM, p, tm, err, st);
}

// Tensor maps: one 3-D float32 map per array, box 40 x 13 x 1, zero fill.
int make_tma_set(TmaSet* out, float* const* arrays, int nx, int ny, int nz) {
    using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    if (nx % 4 != 0) return -2;
    const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
    const cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)BW, (cuuint32_t)BH, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    for (int i = 0; i < TM_N; ++i) {
        CUresult r = encode(&out->m[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, arrays[i], dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return -3 - i;
    }
    return 0;
}
