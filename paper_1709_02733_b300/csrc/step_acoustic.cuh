// step_acoustic.cuh -- bodies of the acoustic step kernels (one work item:
// a 32 x 8 tile over a z chunk), shared by the acoustic kernels of
// step_acoustic.cu and by the interior kernels of step_tiled.cu, which run
// them on the fluid work items of a medium-adaptive step.
//
// With mu = 0 at every node of an item's reach the elastic update of
// Eq. (it) keeps the three normal stresses equal (their increments
// dt lambda div u are the same) and the shear stresses at zero (the harmonic
// shear moduli vanish), so one stress-like field s = sigma^11 = sigma^22 =
// sigma^33 carries the state:
//   velocity: u^i <- (1 - dt alpha_i) u^i + dt / rho_i  D_i s
//   stress:   s   <- s + dt lambda (D-x u^1 + D-y u^2 + D-z u^3)
// and in the weighted adjoint variables (w = dt u~ / rho, Q^ii = lambda tr
// s~, equal for the three normal components):
//   w^i <- (1 - dt alpha_i) w^i - dt^2 / rho_i  D_i Q
//   Q   <- Q - lambda (D-x w^1 + D-y w^2 + D-z w^3).
// So that elastic neighbours read consistent fields, the stress body writes
// s to all three normal-stress arrays; the shear arrays stay zero.  Bytes
// per grid point: velocity 36 B (read s, u x3, rho, alpha; write u x3),
// stress 32 B (read u x3, s, lambda; write s x3), against 56 B and 68 B for
// the elastic interior bodies.
//
// Per plane one TMA load per array stages the tile's 40 x 13 halo box (the
// maps of the elastic kernels) into a 4-plane ring; x and y differences read
// the box, z differences a per-thread register queue.  Only the boxes a plane
// needs are staged: the velocity body loads s alone on the planes beyond the
// item that feed only its queue, and the stress body stages u^1 and u^2 on the
// item's planes and feeds the u^3 queue from own-point loads.  The bodies need whole tiles off the C-PML slabs
// (no own-point or edge-clamping checks).
#pragma once
#include "pact_internal.cuh"
#include "step_tiled.cuh"
#include "tma.cuh"

namespace acoustic {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int BW = TX + 8;      // box columns x0-4 .. x0+TX+3
constexpr int BH = TY + 5;      // box rows    y0-2 .. y0+TY+2
constexpr int BOX = BW * BH;    // 520 floats
constexpr int BOXS = 544;       // box stride (2176 B, a multiple of 128 B)
constexpr int OX = 4, OY = 2;   // own point offset inside the box
constexpr int D = 4;            // ring depth (planes)
constexpr int NB = 3;           // boxes per plane: velocity kernel s, rho, alpha; stress kernel u1, u2, u3
constexpr size_t SMEM = (size_t)D * NB * BOXS * sizeof(float) + D * sizeof(uint64_t);

constexpr float C1 = PACT_C1, C2 = PACT_C2;

__device__ __forceinline__ float dpx(const float* v, int o) { return C1 * (v[o + 1] - v[o]) - C2 * (v[o + 2] - v[o - 1]); }
__device__ __forceinline__ float dmx(const float* v, int o) { return C1 * (v[o] - v[o - 1]) - C2 * (v[o + 1] - v[o - 2]); }
__device__ __forceinline__ float dpy(const float* v, int o) {
    return C1 * (v[o + BW] - v[o]) - C2 * (v[o + 2 * BW] - v[o - BW]);
}
__device__ __forceinline__ float dmy(const float* v, int o) {
    return C1 * (v[o] - v[o - BW]) - C2 * (v[o + BW] - v[o - 2 * BW]);
}
// queue of four consecutive planes (either difference direction)
__device__ __forceinline__ float dq(const float* q) { return C1 * (q[2] - q[1]) - C2 * (q[3] - q[0]); }
__device__ __forceinline__ void push(float* q, float h) {
    q[0] = q[1];
    q[1] = q[2];
    q[2] = q[3];
    q[3] = h;
}

__device__ __forceinline__ void drain(uint64_t* bar, int pfrom, int pto, int pfirst) {
    for (int pl = pfrom; pl <= pto; ++pl) {
        const int k = pl - pfirst;
        mbar_wait_bounded(&bar[k & (D - 1)], (k / D) & 1);
    }
}


// own-point value of array a at plane z (0 off the grid, as the TMA fill)
__device__ __forceinline__ float own_at(const float* a, const StepParams& p, unsigned nxy, unsigned gxy, int z) {
    return (z >= 0 && z < p.nz) ? a[(unsigned)z * nxy + gxy] : 0.f;
}

// Velocity half: output plane z = pl - 2 for ring plane pl (the z queue of s
// holds planes z-1 .. z+2 for the integer->half difference).  The ring runs
// over planes zc0-1 .. zc1+1: the planes zc0 .. zc1 stage the s, rho (and
// alpha) boxes, the two outer planes the s box alone (only its own point
// enters the queue).
// alpha = false (an ITEM_NOALPHA item: alpha = 0 at every node it reads):
// the alpha box is not loaded, and the damping factors are 1 exactly
template <bool ADJ>
__device__ __forceinline__ bool ac_vel_body(const StepParams& p, const CUtensorMap* tmm, int tile_x, int tile_y,
                                            int zc0, int zc1, int* err, float* sm, bool alpha = true) {
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = tile_x * TX, y0 = tile_y * TY;
    const unsigned nxy = (unsigned)p.nx * p.ny, gxy = (unsigned)(y0 + ty) * p.nx + (unsigned)(x0 + tx);
    const int o = (ty + OY) * BW + tx + OX;
    const float dt = p.dt, h = p.inv_dx;
    const int pfirst = zc0 - 1, plast = zc1 + 1;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + (size_t)D * NB * BOXS);
    const CUtensorMap* maps[NB] = {&tmm[TM_S0], &tmm[TM_RHO], &tmm[TM_ALPHA]};
    if (tid == 0) {
        for (int s = 0; s < D; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
        for (int b = 0; b < NB; ++b) tma_prefetch_desc(maps[b]);
    }
    __syncthreads();
    auto stage = [&](int pl) { return sm + (size_t)(((pl - pfirst) & (D - 1)) * NB) * BOXS; };
    const int nb = alpha ? NB : NB - 1;  // the alpha box is the last one
    auto issue = [&](int pl) {
        const int k = pl - pfirst;
        const int n = (pl < zc0 || pl > zc1) ? 1 : nb;
        mbar_arrive_expect_tx(&bar[k & (D - 1)], n * BOX * sizeof(float));
        for (int b = 0; b < n; ++b) tma_load_3d(stage(pl) + b * BOXS, maps[b], x0 - 4, y0 - 2, pl, &bar[k & (D - 1)]);
    };
    if (tid == 0)
        for (int pl = pfirst; pl < pfirst + D && pl <= plast; ++pl) issue(pl);

    float qs[4] = {0, 0, 0, 0};
    float nu[3] = {0, 0, 0};
    auto prefetch = [&](int zn) {
        if (zn < zc0 || zn >= zc1) return;
        const unsigned g = (unsigned)zn * nxy + gxy;
        nu[0] = p.u[0][g];
        nu[1] = p.u[1][g];
        nu[2] = p.u[2][g];
    };
    for (int pl = pfirst; pl <= plast; ++pl) {
        const int z = pl - 2;
        const float cu[3] = {nu[0], nu[1], nu[2]};
        prefetch(z + 1);
        const int kk = pl - pfirst;
        const bool ok = mbar_wait_bounded(&bar[kk & (D - 1)], (kk / D) & 1);
        if (ok) push(qs, stage(pl)[o]);
        if (ok && z >= zc0) {
            const float* sz = stage(z);
            const float* sz1 = stage(z + 1);
            const float* r0 = sz + BOXS;
            const float* a0 = sz + 2 * BOXS;
            const float g[3] = {dpx(sz, o) * h, dpy(sz, o) * h, dq(qs) * h};
            const float rb[3] = {0.5f * (r0[o] + r0[o + 1]), 0.5f * (r0[o] + r0[o + BW]),
                                 0.5f * (r0[o] + sz1[BOXS + o])};
            const float ab[3] = {alpha ? 0.5f * (a0[o] + a0[o + 1]) : 0.f, alpha ? 0.5f * (a0[o] + a0[o + BW]) : 0.f,
                                 alpha ? 0.5f * (a0[o] + sz1[2 * BOXS + o]) : 0.f};
            const unsigned gi = (unsigned)z * nxy + gxy;
#pragma unroll
            for (int i = 0; i < 3; ++i)
                p.u_out[i][gi] = ADJ ? (1.0f - dt * ab[i]) * cu[i] - __fdividef(dt * dt, rb[i]) * g[i]
                                     : (1.0f - dt * ab[i]) * cu[i] + __fdividef(dt, rb[i]) * g[i];
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, 1);
            drain(bar, pl, min(plast, max(pfirst + D - 1, pl + 1)), pfirst);
            return false;
        }
        // the stage of plane z (= pl + 2 modulo the ring) is free once every
        // thread has passed the barrier above; planes up to pfirst + D - 1
        // were issued before the loop
        if (tid == 0 && pl + 2 >= pfirst + D && pl + 2 <= plast) issue(pl + 2);
    }
    if (tid == 0)
        for (int s = 0; s < D; ++s) mbar_inval(&bar[s]);
    return true;
}

// Stress half.  The ring stages the u^1 and u^2 boxes of the planes
// zc0 .. zc1-1 (the x and y differences); the z queue of u^3 holds planes
// z-2 .. z+1 (half->integer difference) of output plane z = pl - 2, from
// own-point loads three planes ahead (the u^3 box would only be read at the
// own point).
template <bool ADJ>
// all3 = false (an ITEM_DEEP item, no elastic reader): sigma^11 only
__device__ __forceinline__ bool ac_str_body(const StepParams& p, const CUtensorMap* tmm, int tile_x, int tile_y,
                                            int zc0, int zc1, int* err, float* sm, bool all3 = true) {
    constexpr int NS = 2;  // boxes per plane: u^1, u^2
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = tile_x * TX, y0 = tile_y * TY;
    const unsigned nxy = (unsigned)p.nx * p.ny, gxy = (unsigned)(y0 + ty) * p.nx + (unsigned)(x0 + tx);
    const int o = (ty + OY) * BW + tx + OX;
    const float h = p.inv_dx;
    const float ks = ADJ ? -1.0f : p.dt;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + (size_t)D * NB * BOXS);
    const CUtensorMap* maps[NS] = {&tmm[TM_U0], &tmm[TM_U0 + 1]};
    // u^3 of the next three queue planes (planes zc0-2 .. zc0 first), loaded
    // three iterations before they enter the queue
    const float* u3 = p.u[2];
    float f0 = own_at(u3, p, nxy, gxy, zc0 - 2), f1 = own_at(u3, p, nxy, gxy, zc0 - 1),
          f2 = own_at(u3, p, nxy, gxy, zc0);
    if (tid == 0) {
        for (int s = 0; s < D; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
        for (int b = 0; b < NS; ++b) tma_prefetch_desc(maps[b]);
    }
    __syncthreads();
    auto stage = [&](int z) { return sm + (size_t)(((z - zc0) & (D - 1)) * NS) * BOXS; };
    auto issue = [&](int z) {
        const int k = z - zc0;
        mbar_arrive_expect_tx(&bar[k & (D - 1)], NS * BOX * sizeof(float));
        for (int b = 0; b < NS; ++b) tma_load_3d(stage(z) + b * BOXS, maps[b], x0 - 4, y0 - 2, z, &bar[k & (D - 1)]);
    };
    if (tid == 0)
        for (int z = zc0; z < zc0 + D && z < zc1; ++z) issue(z);

    float qz[4] = {0, 0, 0, 0};
    float ns = 0.f, nl = 0.f;
    auto prefetch = [&](int zn) {
        if (zn < zc0 || zn >= zc1) return;
        const unsigned g = (unsigned)zn * nxy + gxy;
        ns = p.s[0][g];
        nl = __ldg(p.lam + g);
    };
    for (int pl = zc0 - 1; pl <= zc1 + 1; ++pl) {
        const int z = pl - 2;
        const float so = ns, lam = nl;
        prefetch(z + 1);
        push(qz, f0);  // plane pl - 1
        f0 = f1;
        f1 = f2;
        if (pl + 2 <= zc1) f2 = own_at(u3, p, nxy, gxy, pl + 2);
        bool ok = true;
        if (z >= zc0) {
            const int k = z - zc0;
            ok = mbar_wait_bounded(&bar[k & (D - 1)], (k / D) & 1);
            if (ok) {
                const float* sz = stage(z);
                const float theta = dmx(sz, o) * h + dmy(sz + BOXS, o) * h + dq(qz) * h;
                const float res = so + ks * (lam * theta);
                const unsigned gi = (unsigned)z * nxy + gxy;
                p.s_out[0][gi] = res;
                if (all3) {
                    p.s_out[1][gi] = res;
                    p.s_out[2][gi] = res;
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, 1);
            // planes issued and not yet waited for: z up to the last issued one
            drain(bar, z, min(zc1 - 1, max(zc0 + D - 1, z + D - 1)), zc0);
            return false;
        }
        if (tid == 0 && z >= zc0 && z + D < zc1) issue(z + D);
    }
    if (tid == 0)
        for (int s = 0; s < D; ++s) mbar_inval(&bar[s]);
    return true;
}

}  // namespace acoustic
