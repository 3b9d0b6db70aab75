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
// The two kernel families share their stencils, forward and adjoint alike:
//   velocity family (3 outputs from 6 stress-like fields):
//     forward  u <- J u + dt/rho (D+x s11 + D-y s12 + D-z s13, ...)        (Eq. (it) + C-PML)
//     adjoint  w <- J w - dt^2/rho (D+x F11 + D-y F12 + D-z F13, ...)      (Eq. (backwardstep))
//   stress family (6 outputs from 3 velocity-like fields):
//     forward  s <- s + dt C e(u)                                          (Eq. (it) + C-PML)
//     adjoint  Q <- Q - C e(E)                                             (Eq. (backwardstep))
// The adjoint runs on the weighted variables w = dt u~/rho and Q = C s~
// (step_direct.cu derives them); F and E are Q and w plus the C-PML memory
// terms, which are nonzero only on the slabs, so off the x / y layers the
// adjoint reads its boxes exactly as the forward does.  The deferred J and
// B tails of the adjoint are as in step_direct.cu.
//
// Every half-step is three launches over disjoint (tile, plane) regions: the
// frame of tiles whose halo touches an x or y C-PML slab (all planes; full
// C-PML code, per-thread x / y layer coefficients in registers), the z-slab
// planes of the other tiles (z-layer code only) and the rest (no layer code).
// Layer blocks load the own-point memory variables one plane ahead with the
// wavefield values.  The launches write disjoint points and read only the
// other family's fields, so the frame and z-slab launches may run on a second
// stream, concurrently with the interior one.
//
// Requirements: nx % 4 == 0 (TMA global strides are multiples of 16 bytes).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>
#include <type_traits>

#include "pact_internal.cuh"
#include "step_tiled.cuh"
#include "tma.cuh"

#include "tiled_common.cuh"

// ===========================================================================
// velocity family
// ===========================================================================
// One (tile, z chunk) work item; false if a bounded wait timed out.
//   forward: u <- J u + dt/rho (D sigma + chi phi),  phi <- b phi + a D sigma
//   adjoint: phi~ <- b (phi~ + chi w)  (the deferred tail of the previous
//            stress-family half, own point, old w), then
//            w <- J w - dt^2/rho D F,  F = Q + a (psi^ + chi Q) on the slabs
template <bool ADJ, int PM>
__device__ __forceinline__ bool vel_body(const StepParams& p, const CUtensorMap* maps, int tile_x, int tile_y, int zc0,
                                         int zc1, int* err, float* sm) {
    using Cfg = VelCfg<ADJ, PM>;
    constexpr bool PML = Cfg::PML, LX = Cfg::LX, LY = Cfg::LY, PXY = Cfg::PXY;
    constexpr int NV = mv_values(PM), YV = LX ? 3 : 0;  // buffered values per position; first y value
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = tile_x * TX, y0 = tile_y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = x < p.nx && y < p.ny;
    const int pfirst = zc0 - 2, plast = zc1 + 1;
    const Ring ring{sm, Cfg::NB, pfirst};
    float* der = sm + (size_t)D * Cfg::NB * BOXS;
    float* mvb = der + (size_t)Cfg::NDER * BOXS;
    uint64_t* bar = reinterpret_cast<uint64_t*>(mvb + Cfg::MV);
    const int o = (ty + OY) * BW + tx + OX;
    const float dt = p.dt, h = p.inv_dx;
    const int P = p.P;
    const unsigned nxy = (unsigned)p.nx * p.ny, gxy = own ? (unsigned)y * p.nx + x : 0u;
    PmlXY px{};
    if constexpr (PXY) pml_xy_init<LX, LY>(px, p, x, y, own);

    if (tid == 0) {
        for (int s = 0; s < D; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
        for (int b = 0; b < Cfg::NB; ++b) tma_prefetch_desc(&maps[Cfg::tm(b)]);
    }
    __syncthreads();
    // boxes a ring plane needs: the item's planes all of them; the planes
    // beyond it feed only the z queues (sigma^13 and sigma^23 of plane pl-1,
    // sigma^33 of plane pl) and, on plane zc1, the z averages of rho and alpha
    // (box order sigma^11, 22, 33, 23, 13, 12, rho, alpha)
    auto boxes = [&](int pl) -> unsigned {
        const unsigned m = pl < zc0 - 1 ? 0x18u : pl < zc0 ? 0x1cu : pl < zc1 ? 0xffu : pl == zc1 ? 0xdcu : 0x04u;
        return m & ((1u << Cfg::NB) - 1u);
    };
    auto issue = [&](int pl) {
        const int k = pl - pfirst;
        const unsigned m = boxes(pl);
        float* dst = ring.stage(pl);
        mbar_arrive_expect_tx(&bar[k & (D - 1)], __popc(m) * BOX * sizeof(float));
        for (int b = 0; b < Cfg::NB; ++b)
            if ((m >> b) & 1u) tma_load_3d(dst + b * BOXS, &maps[Cfg::tm(b)], x0 - 4, y0 - 2, pl, &bar[k & (D - 1)]);
    };
    if (tid == 0)
        for (int pl = pfirst; pl < pfirst + D && pl <= plast; ++pl) issue(pl);

    float q33[4] = {0, 0, 0, 0}, q13[4] = {0, 0, 0, 0}, q23[4] = {0, 0, 0, 0};
    const int xc1 = (x + 1 < p.nx) ? 1 : 0;   // clamped +x neighbour offset
    const int yc1 = (y + 1 < p.ny) ? BW : 0;  // clamped +y neighbour offset
    CrossPos cross{};
    CrossPml cpm{};
    float* cxt = nullptr;
    float* cyt = nullptr;
    if constexpr (ADJ && PXY) {
        cxt = frame_coef_tables();
        cyt = cxt + 4 * BW;
        cross_init(cross, tid, x0, y0, p.nx, p.ny);
        __syncthreads();  // a persistent block may still read the tables of its previous item
        cross_pml_init<LX, LY>(cpm, cxt, cyt, cross, tid, x0, y0, p);
        __syncthreads();
    }

    // own-point values of the next output plane, loaded one visit ahead
    float nu[3] = {0.f, 0.f, 0.f};
    float nph[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float na = 0.f;  // alpha of the own point on plane zn (bodies without the alpha box)
    auto prefetch = [&](int zn) {
        if constexpr (!Cfg::ABOX) {
            if (own && zn >= 0 && zn < p.nz) na = __ldg(p.alpha + (unsigned)zn * nxy + gxy);
        }
        if (!own || zn < zc0 || zn >= zc1) return;
        const unsigned g = (unsigned)zn * nxy + gxy;
        nu[0] = p.u[0][g];
        nu[1] = p.u[1][g];
        nu[2] = p.u[2][g];
        if constexpr (PML) {
            const int lz = zslab(zn, p);
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (in_axis<LX, LY>(j, px, lz)) {
                    const unsigned si = own_slab(j, px, lz, x, y, zn, p);
#pragma unroll
                    for (int i = 0; i < 3; ++i) nph[i][j] = p.phi[i][j][si];
                }
        }
    };
    // adjoint C-PML queue-head memory variables (psi^zz at plane pl, psi^xz and
    // psi^yz at plane pl-1), loaded one visit ahead
    float nhp[3] = {0.f, 0.f, 0.f};
    auto prefetch_heads = [&](int pn) {
        if constexpr (ADJ && PML) {
            if (!own) return;
            if (pn >= 0 && pn < p.nz) {
                const int l = zslab(pn, p);
                if (l >= 0) nhp[0] = p.psi[2][2][((unsigned)l * p.ny + y) * p.nx + x];
            }
            const int pm = pn - 1;
            if (pm >= 0 && pm < p.nz) {
                const int l = zslab(pm, p);
                if (l >= 0) {
                    const unsigned si = ((unsigned)l * p.ny + y) * p.nx + x;
                    nhp[1] = p.psi[0][2][si];
                    nhp[2] = p.psi[1][2][si];
                }
            }
        }
    };
    prefetch_heads(pfirst);

    for (int pl = pfirst; pl <= plast; ++pl) {
        const int z = pl - 2;
        const bool out = z >= zc0;
        const float cu[3] = {nu[0], nu[1], nu[2]};
        const float ca = na;  // alpha of the own point on plane z (prefetched a visit ago)
        float cph[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) cph[i][j] = nph[i][j];
        const float chp[3] = {nhp[0], nhp[1], nhp[2]};
        prefetch(z + 1);
        prefetch_heads(pl + 1);
        // full C-PML adjoint: copy psi^ at the cross positions of plane z + 1
        // into its buffer slot; the slot of plane z (copied one visit ago) is
        // complete after the wait
        if constexpr (ADJ && PXY) {
            const int zn = z + 1;
            if (zn >= zc0 && zn < zc1) {
                float* dst = mvb + (size_t)(zn & 1) * NV * NCROSS + tid;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (LX && cpm.sx[k] >= 0) {
                        const unsigned si = (unsigned)zn * p.ny * (2 * P + 1) + cpm.sx[k];
                        cp_async_4(dst + k * NT + 0 * NCROSS, p.psi[0][0] + si);
                        cp_async_4(dst + k * NT + 1 * NCROSS, p.psi[1][0] + si);
                        cp_async_4(dst + k * NT + 2 * NCROSS, p.psi[2][0] + si);
                    }
                    if (LY && cpm.sy[k] >= 0) {
                        const unsigned si = (unsigned)zn * (2 * P + 1) * p.nx + cpm.sy[k];
                        cp_async_4(dst + k * NT + (YV + 0) * NCROSS, p.psi[1][1] + si);
                        cp_async_4(dst + k * NT + (YV + 1) * NCROSS, p.psi[0][1] + si);
                        cp_async_4(dst + k * NT + (YV + 2) * NCROSS, p.psi[2][1] + si);
                    }
                }
            }
            cp_async_commit();
            cp_async_wait<1>();
        }
        const int kk = pl - pfirst;
        const bool ok = mbar_wait_bounded(&bar[kk & (D - 1)], (kk / D) & 1);
        const float* sp = ring.stage(pl);
        const float* spm = (pl - 1 >= pfirst) ? ring.stage(pl - 1) : nullptr;
        // ---- queue heads: integer->half field at plane pl, half->integer at
        //      pl-1 (zero outside the grid: the boxes are zero-filled there)
        if (ok) {
            float h33 = sp[2 * BOXS + o];
            float h13 = spm ? spm[4 * BOXS + o] : 0.f;
            float h23 = spm ? spm[3 * BOXS + o] : 0.f;
            if constexpr (ADJ && PML) {
                // z-layer terms of F33 (integer lattice, plane pl) and of F13,
                // F23 (half lattice, plane pl-1)
                if (own && pl >= 0 && pl < p.nz && zslab(pl, p) >= 0) {
                    const float a = tabv(p, 2, 0, 0, pl), chi = tabv(p, 2, 0, 2, pl);
                    h33 += a * (chp[0] + chi * h33);
                }
                const int zm = pl - 1;
                if (own && spm && zm >= 0 && zm < p.nz && zslab(zm, p) >= 0) {
                    const float a = tabv(p, 2, 1, 0, zm), chi = tabv(p, 2, 1, 2, zm);
                    h13 += a * (chp[1] + chi * h13);
                    h23 += a * (chp[2] + chi * h23);
                }
            }
            push(q33, h33);
            push(q13, h13);
            push(q23, h23);
        }

        if (out) {
            float* szw = ring.stage(z);
            const float* sz = szw;
            const float* sz1 = (z + 1 < p.nz) ? ring.stage(z + 1) : sz;
            // x-differenced fields (for u^x, u^y, u^z) and y-differenced ones
            const float* XD0 = sz;             // s11 / F11
            const float* XD1 = sz + 5 * BOXS;  // s12 / F21
            const float* XD2 = sz + 4 * BOXS;  // s13 / F31
            const float* YD0 = sz + 1 * BOXS;  // s22 / F22
            const float* YD1 = sz + 5 * BOXS;  // s12 / F12
            const float* YD2 = sz + 3 * BOXS;  // s23 / F32
            if constexpr (ADJ && PXY) {
                // F = Q + a (psi^ + chi Q) at the x-band (x layer) and y-row
                // (y layer) positions, in place; F21 goes to the extra box.
                float* E = der;
                if (ok) {
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const unsigned char f = cross.f[k];
                        if (!(f & CP_EXISTS)) continue;
                        const int q = cross.q[k];
                        const float q11 = sz[q], q22 = sz[BOXS + q], q23 = sz[3 * BOXS + q];
                        const float q13 = sz[4 * BOXS + q], q12 = sz[5 * BOXS + q];
                        float f11 = q11, f21 = q12, f31 = q13, f22 = q22, f12 = q12, f32 = q23;
                        const float* mv = mvb + (size_t)(z & 1) * NV * NCROSS + k * NT + tid;
                        if (LX && cpm.sx[k] >= 0) {
                            const float* t = cxt + cross.cxi[k];
                            f11 += t[0] * (mv[0] + t[BW] * q11);
                            f21 += t[2 * BW] * (mv[NCROSS] + t[3 * BW] * q12);
                            f31 += t[2 * BW] * (mv[2 * NCROSS] + t[3 * BW] * q13);
                        }
                        if (LY && cpm.sy[k] >= 0) {
                            const float* t = cyt + cross.cyi[k];
                            f22 += t[0] * (mv[YV * NCROSS] + t[BH] * q22);
                            f12 += t[2 * BH] * (mv[(YV + 1) * NCROSS] + t[3 * BH] * q12);
                            f32 += t[2 * BH] * (mv[(YV + 2) * NCROSS] + t[3 * BH] * q23);
                        }
                        if (f & CP_XB) {
                            szw[q] = f11;
                            E[q] = f21;
                            szw[4 * BOXS + q] = f31;
                        }
                        if (f & CP_YB) {
                            szw[BOXS + q] = f22;
                            szw[5 * BOXS + q] = f12;
                            szw[3 * BOXS + q] = f32;
                        }
                    }
                }
                __syncthreads();
                XD1 = E;
            }
            if (ok && own) {
                const float g[3][3] = {{dpx(XD0, o) * h, dmy(YD1, o) * h, dq(q13) * h},   // u^x
                                       {dmx(XD1, o) * h, dpy(YD0, o) * h, dq(q23) * h},   // u^y
                                       {dmx(XD2, o) * h, dmy(YD2, o) * h, dq(q33) * h}};  // u^z
                const float* r0 = sz + Cfg::BRHO * BOXS;
                const float rb[3] = {0.5f * (r0[o] + r0[o + xc1]), 0.5f * (r0[o] + r0[o + yc1]),
                                     0.5f * (r0[o] + sz1[Cfg::BRHO * BOXS + o])};
                float ab[3];
                if constexpr (Cfg::ABOX) {
                    const float* a0 = sz + Cfg::BALPHA * BOXS;
                    ab[0] = 0.5f * (a0[o] + a0[o + xc1]);
                    ab[1] = 0.5f * (a0[o] + a0[o + yc1]);
                    ab[2] = 0.5f * (a0[o] + sz1[Cfg::BALPHA * BOXS + o]);
                } else {
                    const float* ag = p.alpha + (unsigned)z * nxy + gxy;
                    ab[0] = 0.5f * (ca + __ldg(ag + xc1));
                    ab[1] = 0.5f * (ca + __ldg(ag + (yc1 ? p.nx : 0)));
                    ab[2] = 0.5f * (ca + (z + 1 < p.nz ? na : ca));
                }
                PmlZ pz{};
                if constexpr (PML) pml_z_init(pz, p, z);
                const unsigned gi = (unsigned)z * nxy + gxy;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float acc = g[i][0] + g[i][1] + g[i][2];
                    if constexpr (PML) {
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            if (in_axis<LX, LY>(j, px, pz.lz)) {
                                const int hh = (i == j);
                                float* ph = &p.phi[i][j][own_slab(j, px, pz.lz, x, y, z, p)];
                                if constexpr (!ADJ) {
                                    const float v = coef(j, hh, 1, px, pz) * cph[i][j] + coef(j, hh, 0, px, pz) * g[i][j];
                                    *ph = v;
                                    acc += coef(j, hh, 2, px, pz) * v;
                                } else {
                                    *ph = coef(j, hh, 1, px, pz) * (cph[i][j] + coef(j, hh, 2, px, pz) * cu[i]);
                                }
                            }
                    }
                    const float res = ADJ ? (1.0f - dt * ab[i]) * cu[i] - __fdividef(dt * dt, rb[i]) * acc
                                          : (1.0f - dt * ab[i]) * cu[i] + __fdividef(dt, rb[i]) * acc;
                    p.u_out[i][gi] = res;
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, 1);
            drain(bar, pl, min(plast, max(pfirst + D - 1, pl - 3 + D)), pfirst);
            if constexpr (ADJ && PXY) cp_async_wait<0>();
            return false;
        }
        if (tid == 0 && pl >= zc0 && pl - 2 + D <= plast) issue(pl - 2 + D);
    }
    // every issued plane has been waited for: retire the barriers so that a
    // persistent block can initialise them again for its next work item
    if constexpr (ADJ && PXY) cp_async_wait<0>();
    if (tid == 0)
        for (int s = 0; s < D; ++s) mbar_inval(&bar[s]);
    return true;
}

// ===========================================================================
// stress family
// ===========================================================================
// One (tile, z chunk) work item; false if a bounded wait timed out.
//   forward: psi <- b psi + a e(u),  sigma <- sigma + dt C (e(u) + chi psi)
//   adjoint: psi^ <- b (psi^ + chi Q)  (the deferred tail of the velocity-family
//            half, own point, old Q), then Q <- Q - C e(E),
//            E = w + a (phi~ + chi w) on the slabs
template <bool ADJ, int PM>
__device__ __forceinline__ bool str_body(const StepParams& p, const CUtensorMap* maps, int tile_x, int tile_y, int zc0,
                                         int zc1, int* err, float* sm) {
    using Cfg = StrCfg<ADJ, PM>;
    constexpr bool PML = Cfg::PML, LX = Cfg::LX, LY = Cfg::LY, PXY = Cfg::PXY;
    constexpr int NV = mv_values(PM), YV = LX ? 3 : 0;  // buffered values per position; first y value
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = tile_x * TX, y0 = tile_y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = x < p.nx && y < p.ny;
    const int pfirst = zc0 - 2, plast = zc1 + 1;
    const Ring ring{sm, Cfg::NB, pfirst};
    float* der = sm + (size_t)D * Cfg::NB * BOXS;
    float* mvb = der + (size_t)Cfg::NDER * BOXS;
    uint64_t* bar = reinterpret_cast<uint64_t*>(mvb + Cfg::MV);
    const int o = (ty + OY) * BW + tx + OX;
    const float dt = p.dt, h = p.inv_dx;
    const int P = p.P;
    const unsigned nxy = (unsigned)p.nx * p.ny, gxy = own ? (unsigned)y * p.nx + x : 0u;
    PmlXY px{};
    if constexpr (PXY) pml_xy_init<LX, LY>(px, p, x, y, own);

    if (tid == 0) {
        for (int s = 0; s < D; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
        for (int b = 0; b < Cfg::NB; ++b) tma_prefetch_desc(&maps[Cfg::tm(b)]);
    }
    __syncthreads();
    // lambda is read at the own point only: bodies without x or y layer take
    // it from own-point loads, the frame bodies (short of registers) from the
    // staged box
    constexpr bool LAMBOX = PXY;
    // boxes a ring plane needs: u^1, u^2, u^3, 1/mu (and lambda) on the item's
    // planes, u^1, u^2, u^3 and 1/mu on plane zc1 (the z averages of mu); the
    // planes beyond the item otherwise feed only the z queues (u^1 and u^2 of
    // plane pl, u^3 of plane pl-1) (box order u^1, u^2, u^3, lambda, 1/mu)
    auto boxes = [&](int pl) -> unsigned {
        return pl < zc0 - 1 ? 0x04u : pl < zc0 ? 0x07u : pl < zc1 ? (LAMBOX ? 0x1fu : 0x17u) : pl == zc1 ? 0x17u : 0x03u;
    };
    auto issue = [&](int pl) {
        const int k = pl - pfirst;
        const unsigned m = boxes(pl);
        float* dst = ring.stage(pl);
        mbar_arrive_expect_tx(&bar[k & (D - 1)], __popc(m) * BOX * sizeof(float));
        for (int b = 0; b < Cfg::NB; ++b)
            if ((m >> b) & 1u) tma_load_3d(dst + b * BOXS, &maps[Cfg::tm(b)], x0 - 4, y0 - 2, pl, &bar[k & (D - 1)]);
    };
    if (tid == 0)
        for (int pl = pfirst; pl < pfirst + D && pl <= plast; ++pl) issue(pl);

    float qx[4] = {0, 0, 0, 0}, qy[4] = {0, 0, 0, 0}, qz[4] = {0, 0, 0, 0};
    const int xc1 = (x + 1 < p.nx) ? 1 : 0;
    const int yc1 = (y + 1 < p.ny) ? BW : 0;
    const int oxy = o + xc1 + yc1;
    CrossPos cross{};
    CrossPml cpm{};
    float* cxt = nullptr;
    float* cyt = nullptr;
    if constexpr (ADJ && PXY) {
        cxt = frame_coef_tables();
        cyt = cxt + 4 * BW;
        cross_init(cross, tid, x0, y0, p.nx, p.ny);
        __syncthreads();  // a persistent block may still read the tables of its previous item
        cross_pml_init<LX, LY>(cpm, cxt, cyt, cross, tid, x0, y0, p);
        __syncthreads();
    }

    // own stresses, lambda and psi of the next output plane, loaded one visit ahead
    float ns[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float nl = 0.f;
    float nps[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    auto prefetch = [&](int zn) {
        if (!own || zn < zc0 || zn >= zc1) return;
        const unsigned g = (unsigned)zn * nxy + gxy;
#pragma unroll
        for (int v = 0; v < 6; ++v) ns[v] = p.s[v][g];
        if constexpr (!LAMBOX) nl = __ldg(p.lam + g);
        if constexpr (PML) {
            const int lz = zslab(zn, p);
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (in_axis<LX, LY>(j, px, lz)) {
                    const unsigned si = own_slab(j, px, lz, x, y, zn, p);
#pragma unroll
                    for (int i = 0; i < 3; ++i) nps[i][j] = p.psi[i][j][si];
                }
        }
    };
    // adjoint C-PML queue-head memory variables (phi^xz, phi^yz at plane pl,
    // phi^zz at plane pl-1), loaded one visit ahead
    float nhp[3] = {0.f, 0.f, 0.f};
    auto prefetch_heads = [&](int pn) {
        if constexpr (ADJ && PML) {
            if (!own) return;
            if (pn >= 0 && pn < p.nz) {
                const int l = zslab(pn, p);
                if (l >= 0) {
                    const unsigned si = ((unsigned)l * p.ny + y) * p.nx + x;
                    nhp[0] = p.phi[0][2][si];
                    nhp[1] = p.phi[1][2][si];
                }
            }
            const int pm = pn - 1;
            if (pm >= 0 && pm < p.nz) {
                const int l = zslab(pm, p);
                if (l >= 0) nhp[2] = p.phi[2][2][((unsigned)l * p.ny + y) * p.nx + x];
            }
        }
    };
    prefetch_heads(pfirst);

    for (int pl = pfirst; pl <= plast; ++pl) {
        const int z = pl - 2;
        const bool out = z >= zc0;
        float so[6];
#pragma unroll
        for (int v = 0; v < 6; ++v) so[v] = ns[v];
        const float lo = nl;  // lambda of plane z (own-point load, bodies without a lambda box)
        float cps[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) cps[i][j] = nps[i][j];
        const float chp[3] = {nhp[0], nhp[1], nhp[2]};
        prefetch(z + 1);
        prefetch_heads(pl + 1);
        // full C-PML adjoint: copy phi~ at the cross positions of plane z + 1
        // into its buffer slot; the slot of plane z (copied one visit ago) is
        // complete after the wait
        if constexpr (ADJ && PXY) {
            const int zn = z + 1;
            if (zn >= zc0 && zn < zc1) {
                float* dst = mvb + (size_t)(zn & 1) * NV * NCROSS + tid;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (LX && cpm.sx[k] >= 0) {
                        const unsigned si = (unsigned)zn * p.ny * (2 * P + 1) + cpm.sx[k];
                        cp_async_4(dst + k * NT + 0 * NCROSS, p.phi[0][0] + si);
                        cp_async_4(dst + k * NT + 1 * NCROSS, p.phi[1][0] + si);
                        cp_async_4(dst + k * NT + 2 * NCROSS, p.phi[2][0] + si);
                    }
                    if (LY && cpm.sy[k] >= 0) {
                        const unsigned si = (unsigned)zn * (2 * P + 1) * p.nx + cpm.sy[k];
                        cp_async_4(dst + k * NT + (YV + 0) * NCROSS, p.phi[1][1] + si);
                        cp_async_4(dst + k * NT + (YV + 1) * NCROSS, p.phi[0][1] + si);
                        cp_async_4(dst + k * NT + (YV + 2) * NCROSS, p.phi[2][1] + si);
                    }
                }
            }
            cp_async_commit();
            cp_async_wait<1>();
        }
        const int kk = pl - pfirst;
        const bool ok = mbar_wait_bounded(&bar[kk & (D - 1)], (kk / D) & 1);
        const float* sp = ring.stage(pl);
        const float* spm = (pl - 1 >= pfirst) ? ring.stage(pl - 1) : nullptr;
        // ---- queue heads: d_z of the x and y velocity-like fields is
        //      integer->half (plane pl); d_z of the z one is half->integer (pl-1)
        if (ok) {
            float hx = sp[o], hy = sp[BOXS + o];
            float hz = spm ? spm[2 * BOXS + o] : 0.f;
            if constexpr (ADJ && PML) {
                // z-layer terms of E13, E23 (integer lattice, plane pl) and E33
                // (half lattice, plane pl-1)
                if (own && pl >= 0 && pl < p.nz && zslab(pl, p) >= 0) {
                    const float a = tabv(p, 2, 0, 0, pl), c = tabv(p, 2, 0, 2, pl);
                    hx += a * (chp[0] + c * hx);
                    hy += a * (chp[1] + c * hy);
                }
                const int zm = pl - 1;
                if (own && spm && zm >= 0 && zm < p.nz && zslab(zm, p) >= 0) {
                    const float a = tabv(p, 2, 1, 0, zm), c = tabv(p, 2, 1, 2, zm);
                    hz += a * (chp[2] + c * hz);
                }
            }
            push(qx, hx);
            push(qy, hy);
            push(qz, hz);
        }

        if (out) {
            float* szw = ring.stage(z);
            const float* sz = szw;
            const float* sz1 = (z + 1 < p.nz) ? ring.stage(z + 1) : sz;
            // x-differenced fields and y-differenced ones
            const float* XD0 = sz;             // u^x / E11  (D-x for s11)
            const float* XD1 = sz + BOXS;      // u^y / E21  (D+x for s12)
            const float* XD2 = sz + 2 * BOXS;  // u^z / E31  (D+x for s13)
            const float* YD0 = sz + BOXS;      // u^y / E22  (D-y for s22)
            const float* YD1 = sz;             // u^x / E12  (D+y for s12)
            const float* YD2 = sz + 2 * BOXS;  // u^z / E32  (D+y for s23)
            if constexpr (ADJ && PXY) {
                // E = w + a (phi~ + chi w): the x-differenced fields in place at
                // the x-band (x layer) positions, the y-differenced ones at the
                // y-row (y layer) positions in the three extra boxes.
                float* E0 = der;
                float* E1 = der + BOXS;
                float* E2 = der + 2 * BOXS;
                if (ok) {
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const unsigned char f = cross.f[k];
                        if (!(f & CP_EXISTS)) continue;
                        const int q = cross.q[k];
                        const float wx = sz[q], wy = sz[BOXS + q], wz = sz[2 * BOXS + q];
                        float exx = wx, eyx = wy, ezx = wz, eyy = wy, exy = wx, ezy = wz;
                        const float* mv = mvb + (size_t)(z & 1) * NV * NCROSS + k * NT + tid;
                        if (LX && cpm.sx[k] >= 0) {
                            const float* t = cxt + cross.cxi[k];
                            exx += t[2 * BW] * (mv[0] + t[3 * BW] * wx);
                            eyx += t[0] * (mv[NCROSS] + t[BW] * wy);
                            ezx += t[0] * (mv[2 * NCROSS] + t[BW] * wz);
                        }
                        if (LY && cpm.sy[k] >= 0) {
                            const float* t = cyt + cross.cyi[k];
                            eyy += t[2 * BH] * (mv[YV * NCROSS] + t[3 * BH] * wy);
                            exy += t[0] * (mv[(YV + 1) * NCROSS] + t[BH] * wx);
                            ezy += t[0] * (mv[(YV + 2) * NCROSS] + t[BH] * wz);
                        }
                        if (f & CP_XB) {
                            szw[q] = exx;
                            szw[BOXS + q] = eyx;
                            szw[2 * BOXS + q] = ezx;
                        }
                        if (f & CP_YB) {
                            E0[q] = eyy;
                            E1[q] = exy;
                            E2[q] = ezy;
                        }
                    }
                }
                __syncthreads();
                YD0 = E0;
                YD1 = E1;
                YD2 = E2;
            }
            if (ok && own) {
                // du[i][j] = d_j of the u^i-like field
                const float du[3][3] = {{dmx(XD0, o) * h, dpy(YD1, o) * h, dq(qx) * h},
                                        {dpx(XD1, o) * h, dmy(YD0, o) * h, dq(qy) * h},
                                        {dpx(XD2, o) * h, dpy(YD2, o) * h, dq(qz) * h}};
                const unsigned gi = (unsigned)z * nxy + gxy;
                PmlZ pz{};
                if constexpr (PML) pml_z_init(pz, p, z);
                const float* m0 = sz + Cfg::BMU * BOXS;
                const float* m1 = sz1 + Cfg::BMU * BOXS;
                const float lam = LAMBOX ? sz[Cfg::BLAM * BOXS + o] : lo, mu2 = 2.0f * mu_of(m0[o]);
                const float m12 = harm_inv(m0[o], m0[o + xc1], m0[o + yc1], m0[oxy]);
                const float m13 = harm_inv(m0[o], m0[o + xc1], m1[o], m1[o + xc1]);
                const float m23 = harm_inv(m0[o], m0[o + yc1], m1[o], m1[o + yc1]);
                float res[6];
                if constexpr (!ADJ) {
                    // memory variables psi^{ij} (lattice: integer if i == j, else half)
                    float cp[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};  // chi * psi
                    float pd[3] = {0.f, 0.f, 0.f};                                         // psi^{kk}
                    if constexpr (PML) {
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            if (in_axis<LX, LY>(j, px, pz.lz)) {
                                const unsigned si = own_slab(j, px, pz.lz, x, y, z, p);
#pragma unroll
                                for (int i = 0; i < 3; ++i) {
                                    const int hh = (i != j);
                                    const float v =
                                        coef(j, hh, 1, px, pz) * cps[i][j] + coef(j, hh, 0, px, pz) * du[i][j];
                                    p.psi[i][j][si] = v;
                                    cp[i][j] = coef(j, hh, 2, px, pz) * v;
                                    if (i == j) pd[j] = v;
                                }
                            }
                    }
                    const float theta = du[0][0] + du[1][1] + du[2][2] + pd[0] + pd[1] + pd[2];
                    const float lt = lam * theta;
                    res[0] = so[0] + dt * (lt + mu2 * (du[0][0] + cp[0][0]));
                    res[1] = so[1] + dt * (lt + mu2 * (du[1][1] + cp[1][1]));
                    res[2] = so[2] + dt * (lt + mu2 * (du[2][2] + cp[2][2]));
                    res[3] = so[3] + dt * m23 * (du[1][2] + du[2][1] + cp[1][2] + cp[2][1]);
                    res[4] = so[4] + dt * m13 * (du[0][2] + du[2][0] + cp[0][2] + cp[2][0]);
                    res[5] = so[5] + dt * m12 * (du[0][1] + du[1][0] + cp[0][1] + cp[1][0]);
                } else {
                    if constexpr (PML) {
                        // psi^ <- b (psi^ + chi Q_old) at the own point
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            if (in_axis<LX, LY>(j, px, pz.lz)) {
                                const unsigned si = own_slab(j, px, pz.lz, x, y, z, p);
#pragma unroll
                                for (int i = 0; i < 3; ++i) {
                                    const int hh = (i != j);
                                    p.psi[i][j][si] =
                                        coef(j, hh, 1, px, pz) * (cps[i][j] + coef(j, hh, 2, px, pz) * so[voigt(i, j)]);
                                }
                            }
                    }
                    const float lt = lam * (du[0][0] + du[1][1] + du[2][2]);
                    res[0] = so[0] - (lt + mu2 * du[0][0]);
                    res[1] = so[1] - (lt + mu2 * du[1][1]);
                    res[2] = so[2] - (lt + mu2 * du[2][2]);
                    res[3] = so[3] - m23 * (du[1][2] + du[2][1]);
                    res[4] = so[4] - m13 * (du[0][2] + du[2][0]);
                    res[5] = so[5] - m12 * (du[0][1] + du[1][0]);
                }
#pragma unroll
                for (int v = 0; v < 6; ++v) p.s_out[v][gi] = res[v];
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, 1);
            drain(bar, pl, min(plast, max(pfirst + D - 1, pl - 3 + D)), pfirst);
            if constexpr (ADJ && PXY) cp_async_wait<0>();
            return false;
        }
        if (tid == 0 && pl >= zc0 && pl - 2 + D <= plast) issue(pl - 2 + D);
    }
    // every issued plane has been waited for: retire the barriers so that a
    // persistent block can initialise them again for its next work item
    if constexpr (ADJ && PXY) cp_async_wait<0>();
    if (tid == 0)
        for (int s = 0; s < D; ++s) mbar_inval(&bar[s]);
    return true;
}

// ===========================================================================
// kernels: one grid (single instance) and persistent (many instances)
// ===========================================================================
// Minimum resident blocks per SM of each instantiation (register budget)
// (0: no minimum; the velocity family is limited by its shared memory)
template <bool STR, bool ADJ, int PM>
constexpr int min_blocks() {
    return !STR ? ((ADJ && PM == PM_X) ? 3 : 0) : (PM == PM_NONE ? 4 : (PM == PM_FULL ? 2 : 3));
}
// the persistent kernels read their parameters from shared memory, which
// costs registers: give their velocity-family C-PML bodies an explicit budget
template <bool STR, bool ADJ, int PM>
constexpr int multi_min_blocks() {
    return PM == PM_X ? 3 : (PM == PM_FULL ? 2 : (!STR ? 0 : (ADJ ? 4 : 3)));
}

// One work item; a block runs the body of its region's kind.  The interior
// kernels (PM_NONE) run PM_NONE or PM_Z bodies, the edge kernels (PM_X) PM_X
// or PM_Y bodies, the corner kernels (PM_FULL) PM_FULL bodies; DISPATCH lets
// one kernel run any frame body.
template <bool ADJ, int PM, bool DISPATCH>
__device__ __forceinline__ bool vel_item(const StepParams& p, const CUtensorMap* maps, int kind, int tile_x,
                                         int tile_y, int zc0, int zc1, int* err, float* sm) {
    if constexpr (PM == PM_NONE) {
        if (kind == PM_Z) return vel_body<ADJ, PM_Z>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
        return vel_body<ADJ, PM_NONE>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
    } else if constexpr (DISPATCH) {
        if (kind == PM_X) return vel_body<ADJ, PM_X>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
        if (kind == PM_Y) return vel_body<ADJ, PM_Y>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
        return vel_body<ADJ, PM_FULL>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
    } else if constexpr (PM == PM_X) {
        if (kind == PM_Y) return vel_body<ADJ, PM_Y>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
        return vel_body<ADJ, PM_X>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
    } else {
        return vel_body<ADJ, PM>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
    }
}
template <bool ADJ, int PM, bool DISPATCH>
__device__ __forceinline__ bool str_item(const StepParams& p, const CUtensorMap* maps, int kind, int tile_x,
                                         int tile_y, int zc0, int zc1, int* err, float* sm) {
    if constexpr (PM == PM_NONE) {
        if (kind == PM_Z) return str_body<ADJ, PM_Z>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
        return str_body<ADJ, PM_NONE>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
    } else if constexpr (DISPATCH) {
        if (kind == PM_X) return str_body<ADJ, PM_X>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
        if (kind == PM_Y) return str_body<ADJ, PM_Y>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
        return str_body<ADJ, PM_FULL>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
    } else if constexpr (PM == PM_X) {
        if (kind == PM_Y) return str_body<ADJ, PM_Y>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
        return str_body<ADJ, PM_X>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
    } else {
        return str_body<ADJ, PM>(p, maps, tile_x, tile_y, zc0, zc1, err, sm);
    }
}

template <bool ADJ, int PM>
__global__ void __launch_bounds__(NT, (min_blocks<false, ADJ, PM>())) k_vel_tiled(StepParams p,
                                                                                 const __grid_constant__ TmaSet tm,
                                                                                 RegionList rl, int* err) {
    extern __shared__ __align__(128) float sm[];
    int tile_x, tile_y, zc0, zc1, kind;
    locate(rl, blockIdx.x, tile_x, tile_y, zc0, zc1, kind);
    vel_item<ADJ, PM, false>(p, tm.m, kind, tile_x, tile_y, zc0, zc1, err, sm);
}

template <bool ADJ, int PM>
__global__ void __launch_bounds__(NT, (min_blocks<true, ADJ, PM>())) k_str_tiled(StepParams p,
                                                                                const __grid_constant__ TmaSet tm,
                                                                                RegionList rl, int* err) {
    extern __shared__ __align__(128) float sm[];
    int tile_x, tile_y, zc0, zc1, kind;
    locate(rl, blockIdx.x, tile_x, tile_y, zc0, zc1, kind);
    str_item<ADJ, PM, false>(p, tm.m, kind, tile_x, tile_y, zc0, zc1, err, sm);
}

// Persistent multi-instance half steps: a fixed grid works through the work
// items of every unfinished instance of one direction in the table; each block
// takes the next item from an atomic counter (zeroed before the launch), so
// items of different cost (frame, z-slab and interior tiles of grids of any
// size) balance across the blocks.  STR selects the stress family, ADJ the
// direction: forward instances come first in the table, adjoint ones after
// them, so each kernel carries one body and the register budget of its
// single-grid twin.
template <bool STR, bool ADJ, int PM>
__global__ void __launch_bounds__(NT, (multi_min_blocks<STR, ADJ, PM>())) k_multi(const MultiTable* __restrict__ T,
                                                                                 int* err, int* next) {
    extern __shared__ __align__(128) float sm[];
    constexpr int WHICH = PM == PM_FULL ? ML_CORNER : (PM == PM_X ? ML_EDGE : ML_INNER);
    multi_loop<ADJ, WHICH>(T, err, next, sm,
                           [](const StepParams& sp, const CUtensorMap* maps, int kind, int tile_x, int tile_y, int zc0,
                              int zc1, int* e, float* smem) {
                               return STR ? str_item<ADJ, PM, false>(sp, maps, kind, tile_x, tile_y, zc0, zc1, e, smem)
                                          : vel_item<ADJ, PM, false>(sp, maps, kind, tile_x, tile_y, zc0, zc1, e, smem);
                           });
}

// ---------------------------------------------------------------------------
// host side: work regions and launches
// ---------------------------------------------------------------------------
namespace {

// Planes [za, zb) whose z-difference reach (two planes up and down, and the
// adjoint's z-layer-augmented fields) stays off the z layers; the z layers
// lie at the ends of the whole grid, which for a slab handle is larger.
void no_layer_planes(const StepParams& p, int& za, int& zb) {
    if (p.P <= 0) {
        za = 0;
        zb = p.nz;
        return;
    }
    za = std::min(std::max(p.P + 2 - p.z0g, 0), p.nz);
    zb = std::max(za, std::min(p.nzg - p.P - 3 - p.z0g, p.nz));
}

// tiles whose halo region (x0-2 .. x0+TX+2, y0-2 .. y0+TY+2) stays off the
// x and y layer slabs; returns false if there are none
bool interior_tiles(const StepParams& p, int& txlo, int& txhi, int& tylo, int& tyhi) {
    const int ntx = (p.nx + TX - 1) / TX, nty = (p.ny + TY - 1) / TY;
    const int P = p.P;
    txlo = ntx;
    txhi = -1;
    for (int t = 0; t < ntx; ++t) {
        const int a = t * TX;
        if (a - 2 >= P && a + TX + 2 < p.nx - P - 1) {
            txlo = std::min(txlo, t);
            txhi = std::max(txhi, t);
        }
    }
    tylo = nty;
    tyhi = -1;
    for (int t = 0; t < nty; ++t) {
        const int a = t * TY;
        if (a - 2 >= P && a + TY + 2 < p.ny - P - 1) {
            tylo = std::min(tylo, t);
            tyhi = std::max(tyhi, t);
        }
    }
    return txlo <= txhi && tylo <= tyhi;
}

int add_region(RegionList& rl, int tx0, int tx1, int ty0, int ty1, int za, int zb, int zc, int kind, int& blocks) {
    if (tx0 >= tx1 || ty0 >= ty1 || za >= zb) return 0;
    zc = std::max(1, std::min(zc, zb - za));
    Region& r = rl.r[rl.n++];
    r = {tx0, tx1, ty0, ty1, za, zb, zc, blocks, kind};
    const int chunks = (zb - za + zc - 1) / zc;
    blocks += (tx1 - tx0) * (ty1 - ty0) * chunks;
    return 1;
}

// z chunk length for `tiles` tile columns of zlen planes run by `slots`
// concurrently resident blocks: the chunk count that fills the last wave
// best, discounted by the `extra` planes every chunk loads beyond its own.
int chunk_planes(long tiles, int zlen, long slots, double extra = 3.0) {
    const int cmax = std::max(1, zlen / 16);
    int best = 1;
    double best_s = -1.0;
    for (int c = 1; c <= cmax; ++c) {
        const double w = (double)tiles * c / (double)std::max(1L, slots);
        const double sc = w / std::ceil(w) / (1.0 + extra * c / zlen);
        if (sc > best_s + 1e-9) {
            best_s = sc;
            best = c;
        }
    }
    return (zlen + best - 1) / best;
}

// Tiles and planes of the single-pass kernel: the whole reach of a tile
// (stress points x0-3 .. x0+TX+2, y0-3 .. y0+TY+2; velocity points within)
// inside [P, n-P-2] on x and y (the grid itself without a layer), and output
// planes [P+3, hi-2) whose reach (zs-3 .. zs+3) stays inside [P, hi] too.
struct FusedBox {
    int txlo, txhi, tylo, tyhi, za, zb;  // inclusive tile ranges, planes [za, zb)
};
bool fused_box(const StepParams& p, FusedBox& f) {
    if (p.z0g != 0 || p.nzg != p.nz) return false;  // whole grids only
    const int P = p.P;
    const int hx = P > 0 ? p.nx - P - 2 : p.nx - 1, hy = P > 0 ? p.ny - P - 2 : p.ny - 1;
    const int hz = P > 0 ? p.nz - P - 2 : p.nz - 1;
    const int ntx = (p.nx + TX - 1) / TX, nty = (p.ny + TY - 1) / TY;
    f.txlo = ntx;
    f.txhi = -1;
    for (int t = 0; t < ntx; ++t)
        if (t * TX - 3 >= P && t * TX + TX + 2 <= hx) {
            f.txlo = std::min(f.txlo, t);
            f.txhi = std::max(f.txhi, t);
        }
    f.tylo = nty;
    f.tyhi = -1;
    for (int t = 0; t < nty; ++t)
        if (t * TY - 3 >= P && t * TY + TY + 2 <= hy) {
            f.tylo = std::min(f.tylo, t);
            f.tyhi = std::max(f.tyhi, t);
        }
    f.za = P + 3;
    f.zb = hz - 2;
    return f.txlo <= f.txhi && f.tylo <= f.tyhi && f.zb - f.za >= 8;
}

// Work regions of one half step.  Interior launch: the interior tiles off
// the z slabs (no layer code; long chunks, first) and on the z slabs (z-layer
// code; one chunk per slab, last, so that they fill the launch's tail).
// Frame: the tiles around the interior ones, all planes, in up to eight
// rectangles: the edges (x layer only, y layer only; one launch) and the
// corners (both layers; a second launch), each chunked for its own launch.
// With P = 0 every tile is interior and there are no slabs.  With fb given,
// the tiles and planes of the single-pass kernel are left out of the
// interior launch, which then runs the rest of the interior tiles (z-layer
// code): the fused tiles' planes below and above the fused planes and every
// plane of the interior tiles beside the fused ones.
void make_regions(const StepParams& p, long slots_inner, long slots_edge, long slots_corner, RegionList& inner,
                  int& inner_blocks, RegionList& outer, int& outer_blocks, const FusedBox* fb = nullptr) {
    inner.n = outer.n = 0;
    inner_blocks = outer_blocks = 0;
    const int ntx = (p.nx + TX - 1) / TX, nty = (p.ny + TY - 1) / TY;
    const int P = p.P;
    int txlo = 0, txhi = ntx - 1, tylo = 0, tyhi = nty - 1;
    if (P > 0 && !interior_tiles(p, txlo, txhi, tylo, tyhi)) {
        add_region(outer, 0, ntx, 0, nty, 0, p.nz, chunk_planes((long)ntx * nty, p.nz, slots_corner), PM_FULL,
                   outer_blocks);
        return;
    }
    const long tiles = (long)(txhi + 1 - txlo) * (tyhi + 1 - tylo);
    const long frame = (long)ntx * nty - tiles;
    if (frame > 0) {
        // x-frame columns beside the interior rows (x layer), y-frame rows
        // beside the interior columns (y layer), and the four corners
        const long corners = (long)(ntx - (txhi + 1 - txlo)) * (nty - (tyhi + 1 - tylo));
        const int ze = chunk_planes(frame - corners, p.nz, slots_edge);
        const int zk = chunk_planes(corners, p.nz, slots_corner);
        add_region(outer, 0, txlo, tylo, tyhi + 1, 0, p.nz, ze, PM_X, outer_blocks);
        add_region(outer, txhi + 1, ntx, tylo, tyhi + 1, 0, p.nz, ze, PM_X, outer_blocks);
        add_region(outer, txlo, txhi + 1, 0, tylo, 0, p.nz, ze, PM_Y, outer_blocks);
        add_region(outer, txlo, txhi + 1, tyhi + 1, nty, 0, p.nz, ze, PM_Y, outer_blocks);
        add_region(outer, 0, txlo, 0, tylo, 0, p.nz, zk, PM_FULL, outer_blocks);
        add_region(outer, txhi + 1, ntx, 0, tylo, 0, p.nz, zk, PM_FULL, outer_blocks);
        add_region(outer, 0, txlo, tyhi + 1, nty, 0, p.nz, zk, PM_FULL, outer_blocks);
        add_region(outer, txhi + 1, ntx, tyhi + 1, nty, 0, p.nz, zk, PM_FULL, outer_blocks);
    }
    if (fb) {
        // the fused tiles lie inside the interior ones (their reach is wider)
        const FusedBox& f = *fb;
        const long ring = tiles - (long)(f.txhi + 1 - f.txlo) * (f.tyhi + 1 - f.tylo);
        const int zr = chunk_planes(std::max(1L, ring), p.nz, slots_inner);
        add_region(inner, f.txlo, f.txhi + 1, f.tylo, f.tyhi + 1, 0, f.za, f.za, PM_Z, inner_blocks);
        add_region(inner, f.txlo, f.txhi + 1, f.tylo, f.tyhi + 1, f.zb, p.nz, p.nz - f.zb, PM_Z, inner_blocks);
        add_region(inner, txlo, txhi + 1, tylo, f.tylo, 0, p.nz, zr, PM_Z, inner_blocks);
        add_region(inner, txlo, txhi + 1, f.tyhi + 1, tyhi + 1, 0, p.nz, zr, PM_Z, inner_blocks);
        add_region(inner, txlo, f.txlo, f.tylo, f.tyhi + 1, 0, p.nz, zr, PM_Z, inner_blocks);
        add_region(inner, f.txhi + 1, txhi + 1, f.tylo, f.tyhi + 1, 0, p.nz, zr, PM_Z, inner_blocks);
        return;
    }
    // Output planes [za, zb) run without layer code: their z differences reach
    // two planes up and down, and the adjoint differences fields that carry
    // z-layer terms on the slab planes, so the reach must stay off the slabs.
    int za, zb;
    no_layer_planes(p, za, zb);
    add_region(inner, txlo, txhi + 1, tylo, tyhi + 1, za, zb, chunk_planes(tiles, zb - za, slots_inner), PM_NONE,
               inner_blocks);
    add_region(inner, txlo, txhi + 1, tylo, tyhi + 1, 0, za, za, PM_Z, inner_blocks);
    add_region(inner, txlo, txhi + 1, tylo, tyhi + 1, zb, p.nz, p.nz - zb, PM_Z, inner_blocks);
}

struct LaunchPlan {
    int dev, nx, ny, nz, P, z0g, nzg, family, mode;
    RegionList inner, edge, corner;  // interior, frame edges (PM_X, PM_Y), frame corners (PM_FULL)
    int inner_blocks, edge_blocks, corner_blocks;
    RegionList ac;                   // STEP_ACOUSTIC: the no-layer interior region (acoustic kernels)
    int ac_blocks;
};

// the regions of the kinds in `kinds` (bit mask), renumbered from block 0
int select_kinds(const RegionList& all, unsigned kinds, RegionList& out) {
    out.n = 0;
    int blocks = 0;
    for (int k = 0; k < all.n; ++k) {
        if (!((kinds >> all.r[k].kind) & 1u)) continue;
        Region r = all.r[k];
        r.bstart = blocks;
        blocks += (r.tx1 - r.tx0) * (r.ty1 - r.ty0) * ((r.zb - r.za + r.zc - 1) / r.zc);
        out.r[out.n++] = r;
    }
    return blocks;
}

// kernel and dynamic shared memory of a family (0 vel fwd, 1 vel adj, 2 str
// fwd, 3 str adj) and C-PML mode
template <int PM>
const void* fam_fn(int f) {
    return f == 0 ? (const void*)k_vel_tiled<false, PM> : f == 1 ? (const void*)k_vel_tiled<true, PM>
         : f == 2 ? (const void*)k_str_tiled<false, PM> : (const void*)k_str_tiled<true, PM>;
}
template <int PM>
size_t fam_smem(int f) {
    return f == 0 ? VelCfg<false, PM>::SMEM : f == 1 ? VelCfg<true, PM>::SMEM
         : f == 2 ? StrCfg<false, PM>::SMEM : StrCfg<true, PM>::SMEM;
}
// pm: PM_NONE (interior kernel), PM_X (edge kernel) or PM_FULL (corner kernel)
const void* fam_fn(int f, int pm) {
    return pm == PM_FULL ? fam_fn<PM_FULL>(f) : pm == PM_X ? fam_fn<PM_X>(f) : fam_fn<PM_NONE>(f);
}
size_t fam_smem(int f, int pm) {
    return pm == PM_FULL ? fam_smem<PM_FULL>(f) : pm == PM_X ? fam_smem<PM_X>(f) : fam_smem<PM_NONE>(f);
}

// resident blocks of a kernel on the whole device
long device_slots(const void* fn, size_t smem, int dev) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // shared memory first in the unified L1 / shared array (TMA staging)
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int sms = 148, per_sm = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem);
    return (long)sms * std::max(1, per_sm);
}

LaunchPlan plan_for(int family, const StepParams& p, int mode) {
    static LaunchPlan plans[32];
    static int nplans = 0;
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < nplans; ++i) {
        const LaunchPlan& L = plans[i];
        if (L.dev == dev && L.family == family && L.mode == mode && L.nx == p.nx && L.ny == p.ny && L.nz == p.nz &&
            L.P == p.P && L.z0g == p.z0g && L.nzg == p.nzg)
            return L;
    }
    const long si = device_slots(fam_fn(family, PM_NONE), fam_smem(family, PM_NONE), dev);
    const long sc = device_slots(fam_fn(family, PM_FULL), fam_smem(family, PM_FULL), dev);
    const long se = device_slots(fam_fn(family, PM_X), fam_smem(family, PM_X), dev);
    LaunchPlan& L = plans[nplans % 32];
    L.dev = dev;
    L.family = family;
    L.mode = mode;
    L.nx = p.nx;
    L.ny = p.ny;
    L.nz = p.nz;
    L.P = p.P;
    L.z0g = p.z0g;
    L.nzg = p.nzg;
    RegionList outer;
    int outer_blocks = 0;
    FusedBox fb;
    const bool use_fb = mode == STEP_FUSED && fused_box(p, fb);
    make_regions(p, si, se, sc, L.inner, L.inner_blocks, outer, outer_blocks, use_fb ? &fb : nullptr);
    L.edge_blocks = select_kinds(outer, (1u << PM_X) | (1u << PM_Y), L.edge);
    L.corner_blocks = select_kinds(outer, 1u << PM_FULL, L.corner);
    L.ac.n = 0;
    L.ac_blocks = 0;
    if (mode == STEP_ACOUSTIC && p.P > 0) {
        // the no-layer region goes to the acoustic kernels, chunked for their
        // occupancy; the z-slab planes stay with the elastic interior kernel.
        // With a layer that region lies strictly inside the grid (its tiles
        // are whole and their reach, +1 neighbours included, is off the
        // slabs), which the acoustic kernels assume: they have no own-point
        // or edge-clamping checks.  Without a layer every tile is interior,
        // ragged ones included, and the elastic kernels keep them all.
        RegionList all = L.inner;
        L.inner_blocks = select_kinds(all, 1u << PM_Z, L.inner);
        RegionList none;
        select_kinds(all, 1u << PM_NONE, none);
        const bool str = family >= 2, adj = family == 1 || family == 3;
        const long sa = device_slots(acoustic_fn(str, adj), acoustic_smem(), dev);
        for (int k = 0; k < none.n; ++k) {
            const Region& r = none.r[k];
            const long tiles = (long)(r.tx1 - r.tx0) * (r.ty1 - r.ty0);
            add_region(L.ac, r.tx0, r.tx1, r.ty0, r.ty1, r.za, r.zb, chunk_planes(tiles, r.zb - r.za, sa), PM_NONE,
                       L.ac_blocks);
        }
    }
    nplans = std::min(nplans + 1, 32);
    return L;
}

long long region_points(const RegionList& rl, const StepParams& p) {
    long long n = 0;
    for (int k = 0; k < rl.n; ++k) {
        const Region& r = rl.r[k];
        const long long ex = std::min(r.tx1 * TX, p.nx) - r.tx0 * TX;
        const long long ey = std::min(r.ty1 * TY, p.ny) - r.ty0 * TY;
        n += ex * ey * (long long)(r.zb - r.za);
    }
    return n;
}

}  // namespace

// One half step of a medium-adaptive step: the frame items (edge and corner
// lists, elastic and fluid) on the frame streams between a fork and a join,
// the interior items (elastic, fluid z-slab, acoustic) on the main stream.
template <bool STR, bool ADJ>
static int launch_mixed_half(const StepParams& p, const TmaSet& tm, int* err, const SplitStreams& ss,
                             const MixedPlan& mp) {
    // the two-pass plan of the grid (cached) raises the dynamic shared-memory
    // limit of the elastic kernels launched below
    plan_for((STR ? 2 : 0) + (ADJ ? 1 : 0), p, STEP_TWO_PASS);
    const dim3 blk(TX, TY, 1);
    const int* nb = mp.blocks;
    // a stream for each list: with the four extra streams every list runs on
    // its own (in a captured step they become parallel branches of the
    // graph); otherwise the frame lists share aux / aux2 and the interior
    // lists the main stream.  The lists of a half write disjoint points and
    // read only the other family, so any order among them is correct.
    cudaStream_t sl[MX_N];
    for (int l = 0; l < MX_N; ++l) sl[l] = ss.st;
    const bool frame = nb[MX_EDGE_EL] || nb[MX_EDGE_FL] || nb[MX_CORNER_EL] || nb[MX_CORNER_FL];
    const bool inner = nb[MX_INT_EL] || nb[MX_INT_AC] || nb[MX_INT_FZ];
    cudaStream_t used[MX_N];
    cudaEvent_t joins[MX_N];
    int nused = 0;
    if (ss.aux && ss.aux2 && ss.more) {
        const cudaStream_t own[MX_N] = {ss.more[0], ss.st, ss.more[1], ss.aux, ss.more[2], ss.aux2, ss.more[3]};
        const cudaEvent_t oj[MX_N] = {ss.more_join[0], nullptr, ss.more_join[1], ss.join, ss.more_join[2],
                                      ss.join2, ss.more_join[3]};
        static_assert(MX_INT_EL == 0 && MX_INT_AC == 1 && MX_INT_FZ == 2 && MX_EDGE_EL == 3 && MX_EDGE_FL == 4 &&
                          MX_CORNER_EL == 5 && MX_CORNER_FL == 6,
                      "list order");
        int nonempty = 0;
        for (int l = 0; l < MX_N; ++l) nonempty += nb[l] > 0;
        if (nonempty > 1)
            for (int l = 0; l < MX_N; ++l)
                if (nb[l] && own[l] != ss.st) {
                    sl[l] = own[l];
                    used[nused] = own[l];
                    joins[nused++] = oj[l];
                }
    } else if (ss.aux && frame && inner) {
        sl[MX_EDGE_EL] = sl[MX_EDGE_FL] = sl[MX_CORNER_EL] = sl[MX_CORNER_FL] = ss.aux;
        used[nused] = ss.aux;
        joins[nused++] = ss.join;
        if (ss.aux2) {
            sl[MX_CORNER_EL] = sl[MX_CORNER_FL] = ss.aux2;
            used[nused] = ss.aux2;
            joins[nused++] = ss.join2;
        }
    }
    if (nused) {
        cudaEventRecord(ss.fork, ss.st);
        for (int k = 0; k < nused; ++k) cudaStreamWaitEvent(used[k], ss.fork, 0);
    }
    int n = 0;
    if (nb[MX_CORNER_EL]) {
        const cudaStream_t sc = sl[MX_CORNER_EL];
        if (STR)
            k_str_tiled<ADJ, PM_FULL><<<nb[MX_CORNER_EL], blk, StrCfg<ADJ, PM_FULL>::SMEM, sc>>>(p, tm, mp.list[MX_CORNER_EL], err);
        else
            k_vel_tiled<ADJ, PM_FULL><<<nb[MX_CORNER_EL], blk, VelCfg<ADJ, PM_FULL>::SMEM, sc>>>(p, tm, mp.list[MX_CORNER_EL], err);
        ++n;
    }
    if (nb[MX_CORNER_FL]) {
        launch_fluid(STR, ADJ, PM_FULL, p, tm, mp.list[MX_CORNER_FL], nb[MX_CORNER_FL], err, sl[MX_CORNER_FL]);
        ++n;
    }
    if (nb[MX_EDGE_EL]) {
        const cudaStream_t se = sl[MX_EDGE_EL];
        if (STR) k_str_tiled<ADJ, PM_X><<<nb[MX_EDGE_EL], blk, StrCfg<ADJ, PM_X>::SMEM, se>>>(p, tm, mp.list[MX_EDGE_EL], err);
        else k_vel_tiled<ADJ, PM_X><<<nb[MX_EDGE_EL], blk, VelCfg<ADJ, PM_X>::SMEM, se>>>(p, tm, mp.list[MX_EDGE_EL], err);
        ++n;
    }
    if (nb[MX_EDGE_FL]) {
        launch_fluid(STR, ADJ, PM_X, p, tm, mp.list[MX_EDGE_FL], nb[MX_EDGE_FL], err, sl[MX_EDGE_FL]);
        ++n;
    }
    if (nb[MX_INT_EL]) {
        const cudaStream_t si = sl[MX_INT_EL];
        if (STR)
            k_str_tiled<ADJ, PM_NONE><<<nb[MX_INT_EL], blk, StrCfg<ADJ, PM_NONE>::SMEM, si>>>(p, tm, mp.list[MX_INT_EL], err);
        else
            k_vel_tiled<ADJ, PM_NONE><<<nb[MX_INT_EL], blk, VelCfg<ADJ, PM_NONE>::SMEM, si>>>(p, tm, mp.list[MX_INT_EL], err);
        ++n;
    }
    if (nb[MX_INT_FZ]) {
        launch_fluid(STR, ADJ, PM_Z, p, tm, mp.list[MX_INT_FZ], nb[MX_INT_FZ], err, sl[MX_INT_FZ]);
        ++n;
    }
    if (nb[MX_INT_AC]) {
        launch_acoustic(STR, ADJ, p, tm, mp.list[MX_INT_AC], nb[MX_INT_AC], err, sl[MX_INT_AC]);
        ++n;
    }
    for (int k = 0; k < nused; ++k) {
        cudaEventRecord(joins[k], used[k]);
        cudaStreamWaitEvent(ss.st, joins[k], 0);
    }
    return n;
}

// The frame launch goes to `aux` (when given) between a fork and a join
// event, so that it overlaps the interior launch on `st`.
template <bool ADJ>
static int launch_vel_impl(const StepParams& p, const TmaSet& tm, int* err, const SplitStreams& ss, int mode,
                            const MixedPlan* mp) {
    if (mode == STEP_MIXED && mp) return launch_mixed_half<false, ADJ>(p, tm, err, ss, *mp);
    const LaunchPlan L = plan_for(ADJ ? 1 : 0, p, mode);
    const RegionList& inner = L.inner;
    const int inner_blocks = L.inner_blocks;
    const dim3 blk(TX, TY, 1);
    const int nframe = (L.edge_blocks > 0) + (L.corner_blocks > 0);
    const bool split = ss.aux && nframe && inner_blocks;
    cudaStream_t so = ss.st, sc = ss.st;
    const bool split2 = split && ss.aux2 && L.corner_blocks && L.edge_blocks;
    if (split) {
        cudaEventRecord(ss.fork, ss.st);
        cudaStreamWaitEvent(ss.aux, ss.fork, 0);
        so = sc = ss.aux;
        if (split2) {
            cudaStreamWaitEvent(ss.aux2, ss.fork, 0);
            sc = ss.aux2;
        }
    }
    if (L.corner_blocks)
        k_vel_tiled<ADJ, PM_FULL><<<L.corner_blocks, blk, VelCfg<ADJ, PM_FULL>::SMEM, sc>>>(p, tm, L.corner, err);
    if (L.edge_blocks)
        k_vel_tiled<ADJ, PM_X><<<L.edge_blocks, blk, VelCfg<ADJ, PM_X>::SMEM, so>>>(p, tm, L.edge, err);
    if (inner_blocks)
        k_vel_tiled<ADJ, PM_NONE><<<inner_blocks, blk, VelCfg<ADJ, PM_NONE>::SMEM, ss.st>>>(p, tm, inner, err);
    if (split) {
        cudaEventRecord(ss.join, ss.aux);
        cudaStreamWaitEvent(ss.st, ss.join, 0);
        if (split2) {
            cudaEventRecord(ss.join2, ss.aux2);
            cudaStreamWaitEvent(ss.st, ss.join2, 0);
        }
    }
    return nframe + (inner_blocks > 0);
}

template <bool ADJ>
static int launch_str_impl(const StepParams& p, const TmaSet& tm, int* err, const SplitStreams& ss, int mode,
                            const MixedPlan* mp) {
    if (mode == STEP_MIXED && mp) return launch_mixed_half<true, ADJ>(p, tm, err, ss, *mp);
    const LaunchPlan L = plan_for(ADJ ? 3 : 2, p, mode);
    const RegionList& inner = L.inner;
    const int inner_blocks = L.inner_blocks;
    const dim3 blk(TX, TY, 1);
    const int nframe = (L.edge_blocks > 0) + (L.corner_blocks > 0);
    const bool split = ss.aux && nframe && inner_blocks;
    cudaStream_t so = ss.st, sc = ss.st;
    const bool split2 = split && ss.aux2 && L.corner_blocks && L.edge_blocks;
    if (split) {
        cudaEventRecord(ss.fork, ss.st);
        cudaStreamWaitEvent(ss.aux, ss.fork, 0);
        so = sc = ss.aux;
        if (split2) {
            cudaStreamWaitEvent(ss.aux2, ss.fork, 0);
            sc = ss.aux2;
        }
    }
    if (L.corner_blocks)
        k_str_tiled<ADJ, PM_FULL><<<L.corner_blocks, blk, StrCfg<ADJ, PM_FULL>::SMEM, sc>>>(p, tm, L.corner, err);
    if (L.edge_blocks)
        k_str_tiled<ADJ, PM_X><<<L.edge_blocks, blk, StrCfg<ADJ, PM_X>::SMEM, so>>>(p, tm, L.edge, err);
    if (inner_blocks)
        k_str_tiled<ADJ, PM_NONE><<<inner_blocks, blk, StrCfg<ADJ, PM_NONE>::SMEM, ss.st>>>(p, tm, inner, err);
    if (split) {
        cudaEventRecord(ss.join, ss.aux);
        cudaStreamWaitEvent(ss.st, ss.join, 0);
        if (split2) {
            cudaEventRecord(ss.join2, ss.aux2);
            cudaStreamWaitEvent(ss.st, ss.join2, 0);
        }
    }
    return nframe + (inner_blocks > 0);
}

// ---- multi-instance (persistent) launches --------------------------------
template <bool STR, bool ADJ, int PM>
static size_t multi_smem() {
    return STR ? StrCfg<ADJ, PM>::SMEM : VelCfg<ADJ, PM>::SMEM;
}

template <bool STR, bool ADJ, int PM>
static int multi_grid() {
    static int grid[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!grid[dev])
        grid[dev] = (int)device_slots((const void*)k_multi<STR, ADJ, PM>, multi_smem<STR, ADJ, PM>(), dev);
    return grid[dev];
}

template <bool STR, bool ADJ, int PM>
static void launch_multi(const MultiTable* dT, int* err, int* next, cudaStream_t st) {
    k_multi<STR, ADJ, PM>
        <<<multi_grid<STR, ADJ, PM>(), dim3(TX, TY, 1), multi_smem<STR, ADJ, PM>(), st>>>(dT, err, next);
}

template <bool STR>
static void launch_multi_family(const MultiTable* dT, int* err, int* next, cudaStream_t st) {
    launch_multi<STR, false, PM_FULL>(dT, err, next + 0, st);
    launch_multi<STR, true, PM_FULL>(dT, err, next + 1, st);
    launch_multi<STR, false, PM_X>(dT, err, next + 2, st);
    launch_multi<STR, true, PM_X>(dT, err, next + 3, st);
    launch_multi<STR, false, PM_NONE>(dT, err, next + 4, st);
    launch_multi<STR, true, PM_NONE>(dT, err, next + 5, st);
}

// the elastic corner / edge / interior launches of both directions, then
// the fluid C-PML and acoustic ones (which find no items for instances
// without a medium-adaptive plan)
void launch_multi_step_half(bool str, const MultiTable* dT, int* err, int* next, cudaStream_t st) {
    if (str) launch_multi_family<true>(dT, err, next, st);
    else launch_multi_family<false>(dT, err, next, st);
    launch_multi_fl(str, false, dT, err, next + 6, st);
    launch_multi_fl(str, true, dT, err, next + 7, st);
    launch_multi_ac(str, false, dT, err, next + 8, st);
    launch_multi_ac(str, true, dT, err, next + 9, st);
}

// Region plan of one instance for the persistent kernels: z chunks of about
// `zc` planes so that work items of different instances are of similar size.
void plan_instance_regions(const StepParams& p, int zc, RegionList& inner, int& ninner, RegionList& edge,
                           int& nedge, RegionList& corner, int& ncorner) {
    RegionList outer;
    int nouter = 0;
    make_regions(p, 1, 1, 1, inner, ninner, outer, nouter);
    select_kinds(outer, (1u << PM_X) | (1u << PM_Y), edge);
    select_kinds(outer, 1u << PM_FULL, corner);
    auto rechunk = [zc](RegionList& rl) {
        int blocks = 0;
        for (int k = 0; k < rl.n; ++k) {
            Region& r = rl.r[k];
            r.zc = std::max(1, std::min(zc, r.zb - r.za));
            r.bstart = blocks;
            blocks += (r.tx1 - r.tx0) * (r.ty1 - r.ty0) * ((r.zb - r.za + r.zc - 1) / r.zc);
        }
        return blocks;
    };
    ninner = rechunk(inner);
    nedge = rechunk(edge);
    ncorner = rechunk(corner);
}

int launch_vel_tiled(bool adj, const StepParams& p, const TmaSet& tm, int* err, const SplitStreams& ss, int mode,
                     const MixedPlan* mp) {
    return adj ? launch_vel_impl<true>(p, tm, err, ss, mode, mp) : launch_vel_impl<false>(p, tm, err, ss, mode, mp);
}

int launch_str_tiled(bool adj, const StepParams& p, const TmaSet& tm, int* err, const SplitStreams& ss, int mode,
                     const MixedPlan* mp) {
    return adj ? launch_str_impl<true>(p, tm, err, ss, mode, mp) : launch_str_impl<false>(p, tm, err, ss, mode, mp);
}

// ---- medium-adaptive interior (STEP_MIXED) ---------------------------------
// out[z * ntiles + t] = 1 if mu > 0 (or, called on alpha, alpha > 0) at any
// node of tile t's x-y reach (x0-3 .. x0+TX+2, y0-3 .. y0+TY+2, clipped to
// the grid) on plane z.
__global__ void k_tile_solid(const float* __restrict__ mu, int nx, int ny, int txlo, int tylo, int ntx, int nty,
                             unsigned char* __restrict__ out) {
    const int t = blockIdx.x, z = blockIdx.y;
    const int x0 = (txlo + t % ntx) * TX, y0 = (tylo + t / ntx) * TY;
    constexpr int RW = TX + 6, RH = TY + 6;
    bool any = false;
    for (int i = threadIdx.x; i < RW * RH; i += blockDim.x) {
        const int x = x0 - 3 + i % RW, y = y0 - 3 + i / RW;
        if (x >= 0 && x < nx && y >= 0 && y < ny) any |= __ldg(mu + ((size_t)z * ny + y) * nx + x) > 0.0f;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) out[(size_t)z * ntx * nty + t] = any ? 1 : 0;
}

static_assert(TX == kTileX && TY == kTileY, "plan_deep's tile size");

void free_mixed_plan(MixedPlan* mp) {
    cudaFree(mp->mem);
    delete[] mp->deep;
    *mp = MixedPlan{};
}

int build_mixed_plan(const StepParams& p, const float* mu, const float* alpha, cudaStream_t st, MixedPlan* mp) {
    free_mixed_plan(mp);
    int txlo, txhi, tylo, tyhi;
    if (p.P <= 0 || !interior_tiles(p, txlo, txhi, tylo, tyhi)) return 0;
    const int ntx = (p.nx + TX - 1) / TX, nty = (p.ny + TY - 1) / TY, ntiles = ntx * nty;
    // the no-layer planes of the interior tiles (as in make_regions)
    int za, zb;
    no_layer_planes(p, za, zb);
    unsigned char* d_flag = nullptr;
    const size_t nflag = (size_t)p.nz * ntiles;
    if (cudaMalloc(&d_flag, nflag) != cudaSuccess) return 1;
    // the same reach test on alpha > 0 (absorbing nodes)
    k_tile_solid<<<dim3(ntiles, p.nz), 256, 0, st>>>(mu, p.nx, p.ny, 0, 0, ntx, nty, d_flag);
    std::vector<unsigned char> flag(nflag), aflag(nflag);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(flag.data(), d_flag, nflag, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) k_tile_solid<<<dim3(ntiles, p.nz), 256, 0, st>>>(alpha, p.nx, p.ny, 0, 0, ntx, nty, d_flag);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(aflag.data(), d_flag, nflag, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_flag);
    if (e != cudaSuccess) return 1;
    // absorb[z][t]: an absorbing node where the velocity body of plane z reads
    // alpha (planes z and z+1 of the reach); a fluid item without one is
    // ITEM_NOALPHA (PACT_NOALPHA=0: none is)
    std::vector<unsigned char> absorb(nflag, 1);
    const char* aenv = getenv("PACT_NOALPHA");
    if (!(aenv && std::strcmp(aenv, "0") == 0))
        for (int z = 0; z < p.nz; ++z)
            for (int t = 0; t < ntiles; ++t)
                absorb[(size_t)z * ntiles + t] =
                    aflag[(size_t)z * ntiles + t] | (z + 1 < p.nz ? aflag[(size_t)(z + 1) * ntiles + t] : 0);
    // solid[z][t]: a solid node within planes z-3 .. z+3 of tile t's reach;
    // on a slab of a larger grid the planes beyond its halo are unknown here,
    // so a reach that crosses a cut between slabs counts as solid
    std::vector<unsigned char> solid(nflag);
    const bool cut_lo = p.z0g > 0, cut_hi = p.z0g + p.nz < p.nzg;
    for (int t = 0; t < ntiles; ++t)
        for (int z = 0; z < p.nz; ++z) {
            unsigned char any = (cut_lo && z < 3) || (cut_hi && z > p.nz - 4);
            for (int k = std::max(0, z - 3); k <= std::min(p.nz - 1, z + 3); ++k) any |= flag[(size_t)k * ntiles + t];
            solid[(size_t)z * ntiles + t] = any;
        }
    // near[z][t]: an elastic item within one tile in x and y and three planes
    // in z, i.e. within reach of an elastic body's sigma^22 / sigma^33 reads
    // (two cells, two planes) with a margin.  A fluid item without it is
    // ITEM_DEEP (PACT_AC_DEEP=0: none is).
    std::vector<unsigned char> near(nflag, 1);
    const char* denv = getenv("PACT_AC_DEEP");
    if (!(denv && std::strcmp(denv, "0") == 0)) {
        std::vector<unsigned char> nxy(nflag);
        for (int z = 0; z < p.nz; ++z)
            for (int t = 0; t < ntiles; ++t) {
                const int tx = t % ntx, ty = t / ntx;
                unsigned char any = 0;
                for (int dy = -1; dy <= 1 && !any; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int ux = tx + dx, uy = ty + dy;
                        if (ux < 0 || ux >= ntx || uy < 0 || uy >= nty) continue;
                        any |= solid[(size_t)z * ntiles + uy * ntx + ux];
                    }
                nxy[(size_t)z * ntiles + t] = any;
            }
        for (int t = 0; t < ntiles; ++t)
            for (int z = 0; z < p.nz; ++z) {
                unsigned char any = 0;
                for (int k = std::max(0, z - 3); k <= std::min(p.nz - 1, z + 3); ++k) any |= nxy[(size_t)k * ntiles + t];
                near[(size_t)z * ntiles + t] = any;
            }
    }
    mp->ntx = ntx;
    mp->nty = nty;
    mp->deep = new (std::nothrow) unsigned char[nflag]();
    if (!mp->deep) return 1;
    // Segments of every tile over common z chunks (the z-slab planes below
    // and above the interior planes, then chunks of the interior planes),
    // chunk by chunk, so that the blocks resident at one time work on the
    // same planes of neighbouring tiles and find each other's halos in L2.
    std::vector<Region> lists[MX_N];
    long long pts[MX_N] = {};
    int blocks[MX_N] = {};
    auto add = [&](int li, int tx, int ty, int a, int b, int kind) {
        lists[li].push_back(Region{tx, tx + 1, ty, ty + 1, a, b, b - a, blocks[li], kind});
        blocks[li] += 1;
        const int ex = std::min(p.nx - tx * TX, TX), ey = std::min(p.ny - ty * TY, TY);
        pts[li] += (long long)ex * ey * (b - a);
    };
    // planes per work item: 32 where the tiles alone give the device enough
    // items (on B300 the skull-512 step pair took 4.58 ms at 32 against 4.68
    // at 48, 4.63 at 24 and 4.89 at 96); fewer (down to 8) on small grids,
    // whose few blocks would otherwise march many planes one after another
    // with most SMs idle (each block waits on its loads plane by plane)
    int sms = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long want = 4L * sms;
    const int kChunk = (int)std::min<long>(32, std::max<long>(8, (long)(zb - za) * ntiles / want));
    std::vector<int> cuts{0};
    if (za > 0) cuts.push_back(za);
    if (zb > za) {
        const int nchunk = (zb - za + kChunk - 1) / kChunk;
        const int zc = (zb - za + nchunk - 1) / nchunk;
        for (int c = za + zc; c < zb; c += zc) cuts.push_back(c);
        cuts.push_back(zb);
    }
    if (cuts.back() != p.nz) cuts.push_back(p.nz);
    for (size_t ci = 0; ci + 1 < cuts.size(); ++ci) {
        const int c0 = cuts[ci], c1 = cuts[ci + 1];
        const bool zslab = c0 < za || c0 >= zb;
        for (int t = 0; t < ntiles; ++t) {
            const int tx = t % ntx, ty = t / ntx;
            const bool inx = tx >= txlo && tx <= txhi, iny = ty >= tylo && ty <= tyhi;
            int kind, li_el, li_fl;
            if (inx && iny) {
                kind = zslab ? PM_Z : PM_NONE;
                li_el = MX_INT_EL;
                li_fl = zslab ? MX_INT_FZ : MX_INT_AC;
            } else if (inx || iny) {
                kind = iny ? PM_X : PM_Y;
                li_el = MX_EDGE_EL;
                li_fl = MX_EDGE_FL;
            } else {
                kind = PM_FULL;
                li_el = MX_CORNER_EL;
                li_fl = MX_CORNER_FL;
            }
            // runs of equal (solid, near, absorb) flags; near and absorb
            // only matter for the fluid items
            auto key = [&](int z) {
                const size_t i = (size_t)z * ntiles + t;
                const unsigned char f = solid[i];
                return (int)f * 4 + (!f ? (int)near[i] * 2 + (int)absorb[i] : 0);
            };
            int a = c0;
            while (a < c1) {
                const int kf = key(a);
                int b = a + 1;
                while (b < c1 && key(b) == kf) ++b;
                const bool f = kf >= 4;
                const bool deep = !f && (kf & 2) == 0, noalpha = !f && (kf & 1) == 0;
                add(f ? li_el : li_fl, tx, ty, a, b, kind | (deep ? ITEM_DEEP : 0) | (noalpha ? ITEM_NOALPHA : 0));
                const int ex = std::min(p.nx - tx * TX, TX), ey = std::min(p.ny - ty * TY, TY);
                if (deep) {
                    for (int z = a; z < b; ++z) mp->deep[(size_t)z * ntiles + t] = 1;
                    mp->deep_points += (long long)ex * ey * (b - a);
                }
                if (noalpha) mp->noalpha_points += (long long)ex * ey * (b - a);
                a = b;
            }
        }
    }
    // the fluid C-PML items once more in one list, for the persistent kernels
    std::vector<Region> ff;
    for (int l : {(int)MX_INT_FZ, (int)MX_EDGE_FL, (int)MX_CORNER_FL})
        for (Region r : lists[l]) {
            r.bstart = (int)ff.size();
            ff.push_back(r);
        }
    size_t n = ff.size();
    for (int l = 0; l < MX_N; ++l) n += lists[l].size();
    if (cudaMalloc(&mp->mem, n * sizeof(Region)) != cudaSuccess) return 1;
    std::vector<Region> all;
    all.reserve(n);
    for (int l = 0; l < MX_N; ++l) all.insert(all.end(), lists[l].begin(), lists[l].end());
    all.insert(all.end(), ff.begin(), ff.end());
    e = cudaMemcpyAsync(mp->mem, all.data(), n * sizeof(Region), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free_mixed_plan(mp);
        return 1;
    }
    size_t off = 0;
    for (int l = 0; l < MX_N; ++l) {
        mp->list[l].n = 0;
        mp->list[l].dev = lists[l].empty() ? nullptr : mp->mem + off;
        mp->list[l].dn = (int)lists[l].size();
        mp->blocks[l] = blocks[l];
        mp->points[l] = pts[l];
        off += lists[l].size();
    }
    mp->fluid_frame.n = 0;
    mp->fluid_frame.dev = ff.empty() ? nullptr : mp->mem + off;
    mp->fluid_frame.dn = (int)ff.size();
    mp->fluid_frame_blocks = (int)ff.size();
    return 0;
}

int launch_acoustic_step(bool str, bool adj, const StepParams& p, const TmaSet& tm, int* err, cudaStream_t st) {
    const LaunchPlan L = plan_for((str ? 2 : 0) + (adj ? 1 : 0), p, STEP_ACOUSTIC);
    if (L.ac_blocks <= 0) return 0;
    launch_acoustic(str, adj, p, tm, L.ac, L.ac_blocks, err, st);
    return 1;
}

// The fused region: one rectangle of tiles over the fused planes, in z
// chunks that fill the last wave of resident single-pass blocks best (every
// chunk computes four velocity planes and loads seven stress planes beyond
// its own).
bool fused_plan(const StepParams& p, RegionList& rl, int& blocks) {
    rl.n = 0;
    blocks = 0;
    FusedBox f;
    if (!fused_box(p, f)) return false;
    static long slots[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!slots[dev]) {
        // device_slots also raises the dynamic shared-memory limit of the kernel
        slots[dev] = device_slots(fused_fn(false), fused_smem(), dev);
        device_slots(fused_fn(true), fused_smem(), dev);
    }
    const long tiles = (long)(f.txhi + 1 - f.txlo) * (f.tyhi + 1 - f.tylo);
    add_region(rl, f.txlo, f.txhi + 1, f.tylo, f.tyhi + 1, f.za, f.zb, chunk_planes(tiles, f.zb - f.za, slots[dev], 6.0),
               PM_NONE, blocks);
    return blocks > 0;
}

int launch_fused_step(bool adj, const StepParams& p, const FusedMaps& fm, int* err, cudaStream_t st) {
    struct Cached {
        int dev, nx, ny, nz, P, blocks;
        RegionList rl;
    };
    static Cached cache[16];
    static int ncache = 0;
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    Cached c{};
    {
        std::lock_guard<std::mutex> lock(mu);
        int i = 0;
        for (; i < ncache; ++i)
            if (cache[i].dev == dev && cache[i].nx == p.nx && cache[i].ny == p.ny && cache[i].nz == p.nz &&
                cache[i].P == p.P)
                break;
        if (i == ncache) {
            Cached& n = cache[ncache % 16];
            n = {dev, p.nx, p.ny, p.nz, p.P, 0, {}};
            fused_plan(p, n.rl, n.blocks);
            i = ncache % 16;
            ncache = std::min(ncache + 1, 16);
        }
        c = cache[i];
    }
    if (c.blocks <= 0) return 0;
    launch_fused(adj, p, fm, c.rl, c.blocks, err, st);
    return 1;
}

long long role_points(int family, int mode, const StepParams& p) {
    if (family == 2) {
        RegionList rl;
        int blocks = 0;
        return fused_plan(p, rl, blocks) ? region_points(rl, p) : 0;
    }
    if (family == 3) return mode == STEP_ACOUSTIC ? region_points(plan_for(0, p, STEP_ACOUSTIC).ac, p) : 0;
    const LaunchPlan L = plan_for(family == 0 ? 0 : 2, p, mode);
    return region_points(L.inner, p) + region_points(L.edge, p) + region_points(L.corner, p);
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
