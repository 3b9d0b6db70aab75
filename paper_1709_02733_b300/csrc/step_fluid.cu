// step_fluid.cu -- C-PML frame and z-slab step kernels for fluid work items.
//
// In a work item whose reach (x0-3 .. x0+TX+2, y0-3 .. y0+TY+2, z-3 .. z+3)
// holds only fluid nodes (mu = 0), the elastic update with the C-PML of
// Appendix A.3 keeps sigma^11 = sigma^22 = sigma^33 (their increments are all
// dt lambda sum_k (D_k u^k + psi^kk)) and the shear stresses at zero (the
// harmonic shear moduli vanish), so one stress field s carries the state and
// only the memory variables the fluid drives change:
//   forward velocity  phi^ii <- b_i phi^ii + a_i D_i s   (u^i node, axis-i layer)
//                     u^i <- J u^i + dt/rho_i (D_i s + chi_i phi^ii)
//   forward stress    psi^kk <- b_k psi^kk + a_k D_k u^k  (integer node, axis-k layer)
//                     s <- s + dt lambda sum_k (D_k u^k + psi^kk)
// The off-diagonal phi^ij stay zero (they are driven by the shear stresses);
// the off-diagonal psi^ij act only on shear stresses of nodes whose shear
// modulus is zero, so they are not kept.  In the adjoint's weighted variables
// (the elastic kernels' w, Q; step_tiled.cu):
//   velocity  phi~^ii <- b_i (phi~^ii + chi_i w^i)  (the deferred tail), then
//             w^i <- J w^i - dt^2/rho_i D_i F^ii,  F^ii = Q + a_i (psi^^ii + chi_i Q)
//   stress    psi^^kk <- b_k (psi^^kk + chi_k Q)  (deferred tail, own point;
//             the off-diagonal psi^^ij stay zero, they are driven by the shear Q),
//             Q <- Q - lambda sum_k D_k E^kk,  E^kk = w^k + a_k (phi~^kk + chi_k w^k)
// F and E are formed at the cross positions of the x and y layers as in the
// elastic kernels, for the diagonal components only, but as each plane
// arrives, two planes before it is differenced, so that the end-of-plane
// barrier orders them and no barrier sits between forming and differencing.  The off-diagonal
// adjoint memory variables of a fluid item's nodes matter nowhere: psi^^ij
// and F^ij stay zero (the shear Q is zero), and phi~^ij enters only E^ij,
// which only the shear update of a node within two cells reads; every such
// node has a fluid node among its four neighbours (all of them lie in the
// item's reach), so its shear modulus, and the weight of E^ij, is zero.
//
// Bytes per grid point against the elastic frame bodies: the velocity body
// stages s, rho, alpha (3 boxes for 8; s alone on the two planes beyond the
// item that only feed its z queue), the stress body u^1 and u^2 (2 boxes for
// 5; u^3 and lambda are read at the own point only, and come from own-point
// loads) and writes three stresses instead of six.  The stress body writes s to
// all three normal-stress arrays so that elastic neighbours read consistent
// fields; the shear arrays stay zero.
#include <algorithm>

#include "tiled_common.cuh"

namespace {

template <bool ADJ, int PM> struct VelFl {
    static constexpr bool LX = has_x(PM), LY = has_y(PM), PXY = LX || LY;
    static constexpr int NB = 3, BS = 0, BRHO = 1, BALPHA = 2;  // s (or Q), rho, alpha
    static constexpr int NV = (LX ? 1 : 0) + (LY ? 1 : 0);      // psi^ values per cross position
    static constexpr int NDER = (ADJ && PXY) ? D * NV : 0;      // F11 / F22 boxes, one set per ring stage
    static constexpr int MV = ADJ ? 2 * NV * NCROSS : 0;
    static constexpr size_t SMEM = ((size_t)(D * NB + NDER) * BOXS + MV) * sizeof(float) + D * sizeof(uint64_t);
    __host__ __device__ static constexpr int tm(int b) { return b == 0 ? TM_S0 : (b == 1 ? TM_RHO : TM_ALPHA); }
};

template <bool ADJ, int PM> struct StrFl {
    static constexpr bool LX = has_x(PM), LY = has_y(PM), PXY = LX || LY;
    static constexpr int NB = 2;                                // u^1, u^2 (or w)
    static constexpr int NDER = 0;                              // E11, E22 formed in place
    static constexpr int NV = (LX ? 1 : 0) + (LY ? 1 : 0);      // phi~ values per cross position
    static constexpr int MV = ADJ ? 2 * NV * NCROSS : 0;
    static constexpr size_t SMEM = ((size_t)(D * NB + NDER) * BOXS + MV) * sizeof(float) + D * sizeof(uint64_t);
    __host__ __device__ static constexpr int tm(int b) { return TM_U0 + b; }
};

// the persistent kernel runs every fluid body with the corner layout
static_assert(VelFl<true, PM_FULL>::SMEM >= VelFl<true, PM_X>::SMEM && VelFl<true, PM_FULL>::SMEM >= VelFl<true, PM_Z>::SMEM &&
                  StrFl<true, PM_FULL>::SMEM >= StrFl<true, PM_X>::SMEM &&
                  StrFl<true, PM_FULL>::SMEM >= StrFl<true, PM_Z>::SMEM &&
                  VelFl<false, PM_FULL>::SMEM >= VelFl<false, PM_X>::SMEM &&
                  StrFl<false, PM_FULL>::SMEM >= StrFl<false, PM_X>::SMEM,
              "corner layout covers the other fluid bodies");
// the edge kernels run the PM_X and PM_Y bodies with one layout
static_assert(VelFl<true, PM_X>::SMEM == VelFl<true, PM_Y>::SMEM && StrFl<true, PM_X>::SMEM == StrFl<true, PM_Y>::SMEM &&
                  VelFl<false, PM_X>::SMEM == VelFl<false, PM_Y>::SMEM &&
                  StrFl<false, PM_X>::SMEM == StrFl<false, PM_Y>::SMEM,
              "edge bodies share one layout");

// ---------------------------------------------------------------------------
// velocity family
// ---------------------------------------------------------------------------
// alpha = false (an ITEM_NOALPHA item): no alpha box, damping factors 1
template <bool ADJ, int PM>
__device__ __forceinline__ bool vel_fluid_body(const StepParams& p, const CUtensorMap* maps, int tile_x, int tile_y,
                                               int zc0, int zc1, int* err, float* sm, bool alpha = true) {
    using Cfg = VelFl<ADJ, PM>;
    constexpr bool LX = Cfg::LX, LY = Cfg::LY, PXY = Cfg::PXY;
    constexpr int NV = Cfg::NV, YV = LX ? 1 : 0;  // buffered values per position; the y value
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = tile_x * TX, y0 = tile_y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = x < p.nx && y < p.ny;
    // ring planes zc0-1 .. zc1+1: the outer two feed only the z queue (their
    // s box alone is staged)
    const int pfirst = zc0 - 1, plast = zc1 + 1;
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
    static_assert(Cfg::BALPHA == Cfg::NB - 1 && Cfg::BS == 0, "s box first, alpha box last");
    const int nb = alpha ? Cfg::NB : Cfg::NB - 1;
    auto issue = [&](int pl) {
        const int k = pl - pfirst;
        const int n = (pl < zc0 || pl > zc1) ? 1 : nb;
        float* dst = ring.stage(pl);
        mbar_arrive_expect_tx(&bar[k & (D - 1)], n * BOX * sizeof(float));
        for (int b = 0; b < n; ++b)
            tma_load_3d(dst + b * BOXS, &maps[Cfg::tm(b)], x0 - 4, y0 - 2, pl, &bar[k & (D - 1)]);
    };
    if (tid == 0)
        for (int pl = pfirst; pl < pfirst + D && pl <= plast; ++pl) issue(pl);

    float qs[4] = {0, 0, 0, 0};  // s (adjoint: F33) at planes z-1 .. z+2
    const int xc1 = (x + 1 < p.nx) ? 1 : 0;
    const int yc1 = (y + 1 < p.ny) ? BW : 0;
    CrossPos cross{};
    CrossPml cpm{};
    float* cxt = nullptr;
    float* cyt = nullptr;
    if constexpr (ADJ && PXY) {
        cxt = frame_coef_tables();
        cyt = cxt + 4 * BW;
        cross_init(cross, tid, x0, y0, p.nx, p.ny);
        __syncthreads();
        cross_pml_init<LX, LY>(cpm, cxt, cyt, cross, tid, x0, y0, p);
        __syncthreads();
    }

    // own-point values of the next output plane, loaded one visit ahead:
    // the old velocity and phi^ii (forward) / phi~^ii (adjoint) on the layer
    // of axis i
    float nu[3] = {0.f, 0.f, 0.f};
    float nph[3] = {0.f, 0.f, 0.f};
    auto prefetch = [&](int zn) {
        if (!own || zn < zc0 || zn >= zc1) return;
        const unsigned g = (unsigned)zn * nxy + gxy;
        nu[0] = p.u[0][g];
        nu[1] = p.u[1][g];
        nu[2] = p.u[2][g];
        const int lz = zslab(zn, p);
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (in_axis<LX, LY>(j, px, lz)) nph[j] = p.phi[j][j][own_slab(j, px, lz, x, y, zn, p)];
    };
    // adjoint: psi^zz at plane pl (the z-layer term of the F33 queue head), one visit ahead
    float nhp = 0.f;
    auto prefetch_head = [&](int pn) {
        if constexpr (ADJ) {
            if (!own || pn < 0 || pn >= p.nz) return;
            const int l = zslab(pn, p);
            if (l >= 0) nhp = p.psi[2][2][((unsigned)l * p.ny + y) * p.nx + x];
        }
    };
    prefetch_head(pfirst);

    for (int pl = pfirst; pl <= plast; ++pl) {
        const int z = pl - 2;
        const bool out = z >= zc0;
        const float cu[3] = {nu[0], nu[1], nu[2]};
        const float cph[3] = {nph[0], nph[1], nph[2]};
        const float chp = nhp;
        prefetch(z + 1);
        prefetch_head(pl + 1);
        // adjoint layers: copy psi^xx (x band) and psi^yy (y rows) at the cross
        // positions of plane pl + 1 into its buffer slot (each thread reads
        // back only its own copies)
        if constexpr (ADJ && PXY) {
            const int zn = pl + 1;
            if (zn >= zc0 && zn < zc1) {
                float* dst = mvb + (size_t)(zn & 1) * NV * NCROSS + tid;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (LX && cpm.sx[k] >= 0)
                        cp_async_4(dst + k * NT, p.psi[0][0] + (unsigned)zn * p.ny * (2 * P + 1) + cpm.sx[k]);
                    if (LY && cpm.sy[k] >= 0)
                        cp_async_4(dst + k * NT + YV * NCROSS, p.psi[1][1] + (unsigned)zn * (2 * P + 1) * p.nx + cpm.sy[k]);
                }
            }
            cp_async_commit();
            cp_async_wait<1>();
        }
        const int kk = pl - pfirst;
        const bool ok = mbar_wait_bounded(&bar[kk & (D - 1)], (kk / D) & 1);
        if (ok) {
            float h33 = ring.stage(pl)[o];
            if constexpr (ADJ) {
                // z-layer term of F33 (integer lattice, plane pl)
                if (own && pl >= 0 && pl < p.nz && zslab(pl, p) >= 0) {
                    const float a = tabv(p, 2, 0, 0, pl), chi = tabv(p, 2, 0, 2, pl);
                    h33 += a * (chp + chi * h33);
                }
            }
            push(qs, h33);
            if constexpr (ADJ && PXY) {
                // F11 = Q + a (psi^xx + chi Q) at the x-band positions and
                // F22 = Q + a (psi^yy + chi Q) at the y-band ones of plane pl,
                // formed as the plane arrives into the extra boxes of its ring
                // stage (the Q box stays as loaded).  They are differenced two
                // planes later: the end-of-plane barriers in between order
                // these writes before every read.
                if (pl >= zc0 && pl < zc1) {
                    const float* sq = ring.stage(pl);
                    float* e = der + (size_t)(kk & (D - 1)) * NV * BOXS;
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const unsigned char f = cross.f[k];
                        const int q = cross.q[k];
                        const float* mv = mvb + (size_t)(pl & 1) * NV * NCROSS + k * NT + tid;
                        if (LX && (f & CP_XB)) {
                            const float qv = sq[q];
                            float f11 = qv;
                            if (cpm.sx[k] >= 0) {
                                const float* t = cxt + cross.cxi[k];
                                f11 += t[0] * (mv[0] + t[BW] * qv);
                            }
                            e[q] = f11;
                        }
                        if (LY && (f & CP_YB)) {
                            const float qv = sq[q];
                            float f22 = qv;
                            if (cpm.sy[k] >= 0) {
                                const float* t = cyt + cross.cyi[k];
                                f22 += t[0] * (mv[YV * NCROSS] + t[BH] * qv);
                            }
                            e[YV * BOXS + q] = f22;
                        }
                    }
                }
            }
        }
        if (out) {
            const float* sz = ring.stage(z);
            const float* sz1 = (z + 1 < p.nz) ? ring.stage(z + 1) : sz;
            const float* XD = sz;  // s / F11
            const float* YD = sz;  // s / F22
            if constexpr (ADJ && PXY) {
                const float* e = der + (size_t)((z - pfirst) & (D - 1)) * NV * BOXS;
                if constexpr (LX) XD = e;
                if constexpr (LY) YD = e + YV * BOXS;
            }
            if (ok && own) {
                const float g[3] = {dpx(XD, o) * h, dpy(YD, o) * h, dq(qs) * h};
                const float* r0 = sz + Cfg::BRHO * BOXS;
                const float* a0 = sz + Cfg::BALPHA * BOXS;
                const float rb[3] = {0.5f * (r0[o] + r0[o + xc1]), 0.5f * (r0[o] + r0[o + yc1]),
                                     0.5f * (r0[o] + sz1[Cfg::BRHO * BOXS + o])};
                const float ab[3] = {alpha ? 0.5f * (a0[o] + a0[o + xc1]) : 0.f,
                                     alpha ? 0.5f * (a0[o] + a0[o + yc1]) : 0.f,
                                     alpha ? 0.5f * (a0[o] + sz1[Cfg::BALPHA * BOXS + o]) : 0.f};
                PmlZ pz{};
                pml_z_init(pz, p, z);
                const unsigned gi = (unsigned)z * nxy + gxy;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float acc = g[i];
                    // phi^ii / phi~^ii (half lattice along axis i)
                    if (in_axis<LX, LY>(i, px, pz.lz)) {
                        float* ph = &p.phi[i][i][own_slab(i, px, pz.lz, x, y, z, p)];
                        if constexpr (!ADJ) {
                            const float v = coef(i, 1, 1, px, pz) * cph[i] + coef(i, 1, 0, px, pz) * g[i];
                            *ph = v;
                            acc += coef(i, 1, 2, px, pz) * v;
                        } else {
                            *ph = coef(i, 1, 1, px, pz) * (cph[i] + coef(i, 1, 2, px, pz) * cu[i]);
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
            drain(bar, pl, min(plast, max(pfirst + D - 1, pl + 1)), pfirst);
            if constexpr (ADJ && PXY) cp_async_wait<0>();
            return false;
        }
        // the stage of plane z (= pl + 2 modulo the ring) is free once every
        // thread has passed the barrier above; planes up to pfirst + D - 1
        // were issued before the loop
        if (tid == 0 && pl + 2 >= pfirst + D && pl + 2 <= plast) issue(pl + 2);
    }
    if constexpr (ADJ && PXY) cp_async_wait<0>();
    if (tid == 0)
        for (int s = 0; s < D; ++s) mbar_inval(&bar[s]);
    return true;
}

// ---------------------------------------------------------------------------
// stress family
// ---------------------------------------------------------------------------
template <bool ADJ, int PM>
// all3 = false (an ITEM_DEEP item, no elastic reader): sigma^11 only
__device__ __forceinline__ bool str_fluid_body(const StepParams& p, const CUtensorMap* maps, int tile_x, int tile_y,
                                               int zc0, int zc1, int* err, float* sm, bool all3 = true) {
    using Cfg = StrFl<ADJ, PM>;
    constexpr bool LX = Cfg::LX, LY = Cfg::LY, PXY = Cfg::PXY;
    constexpr int NV = Cfg::NV, YV = LX ? 1 : 0;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = tile_x * TX, y0 = tile_y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = x < p.nx && y < p.ny;
    // ring planes zc0 .. zc1-1, the planes differenced in x and y (u^1, u^2
    // boxes); the u^3 queue and lambda come from own-point loads
    const int pfirst = zc0, plast = zc1 - 1;
    const Ring ring{sm, Cfg::NB, pfirst};
    float* der = sm + (size_t)D * Cfg::NB * BOXS;
    float* mvb = der + (size_t)Cfg::NDER * BOXS;
    uint64_t* bar = reinterpret_cast<uint64_t*>(mvb + Cfg::MV);
    const int o = (ty + OY) * BW + tx + OX;
    const float dt = p.dt, h = p.inv_dx;
    const int P = p.P;
    const unsigned nxy = (unsigned)p.nx * p.ny, gxy = own ? (unsigned)y * p.nx + x : 0u;
    // u^3 (adjoint: w^3) at the own point of plane zq (0 off the grid, as the TMA fill)
    auto u3at = [&](int zq) {
        return (own && zq >= 0 && zq < p.nz) ? p.u[2][(unsigned)zq * nxy + gxy] : 0.f;
    };
    // u^3 of the next three queue planes (planes zc0-2 .. zc0 first), loaded
    // three iterations before they enter the queue
    float f0 = u3at(zc0 - 2), f1 = u3at(zc0 - 1), f2 = u3at(zc0);
    PmlXY px{};
    if constexpr (PXY) pml_xy_init<LX, LY>(px, p, x, y, own);

    if (tid == 0) {
        for (int s = 0; s < D; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
        for (int b = 0; b < Cfg::NB; ++b) tma_prefetch_desc(&maps[Cfg::tm(b)]);
    }
    __syncthreads();
    auto issue = [&](int pl) {
        const int k = pl - pfirst;
        float* dst = ring.stage(pl);
        mbar_arrive_expect_tx(&bar[k & (D - 1)], Cfg::NB * BOX * sizeof(float));
        for (int b = 0; b < Cfg::NB; ++b)
            tma_load_3d(dst + b * BOXS, &maps[Cfg::tm(b)], x0 - 4, y0 - 2, pl, &bar[k & (D - 1)]);
    };
    if (tid == 0)
        for (int pl = pfirst; pl < pfirst + D && pl <= plast; ++pl) issue(pl);

    float qz[4] = {0, 0, 0, 0};  // u^3 (adjoint: E33) at planes z-2 .. z+1
    CrossPos cross{};
    CrossPml cpm{};
    float* cxt = nullptr;
    float* cyt = nullptr;
    if constexpr (ADJ && PXY) {
        cxt = frame_coef_tables();
        cyt = cxt + 4 * BW;
        cross_init(cross, tid, x0, y0, p.nx, p.ny);
        __syncthreads();
        cross_pml_init<LX, LY>(cpm, cxt, cyt, cross, tid, x0, y0, p);
        __syncthreads();
    }

    // own-point values of the next output plane, loaded one visit ahead: the
    // old s (or Q), lambda and psi^kk (forward) / psi^^kk (adjoint) on the
    // layer of axis k
    float ns = 0.f, nl = 0.f;
    float nps[3] = {0.f, 0.f, 0.f};
    auto prefetch = [&](int zn) {
        if (!own || zn < zc0 || zn >= zc1) return;
        const unsigned g = (unsigned)zn * nxy + gxy;
        ns = p.s[0][g];
        nl = __ldg(p.lam + g);
        const int lz = zslab(zn, p);
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (in_axis<LX, LY>(j, px, lz)) nps[j] = p.psi[j][j][own_slab(j, px, lz, x, y, zn, p)];
    };
    // adjoint: phi~^zz at plane pl-1 (the z-layer term of the E33 queue head), one visit ahead
    float nhp = 0.f;
    auto prefetch_head = [&](int pn) {
        if constexpr (ADJ) {
            const int pm = pn - 1;
            if (!own || pm < 0 || pm >= p.nz) return;
            const int l = zslab(pm, p);
            if (l >= 0) nhp = p.phi[2][2][((unsigned)l * p.ny + y) * p.nx + x];
        }
    };
    prefetch_head(zc0 - 1);

    // queue plane pl - 1 enters at visit pl; output plane z = pl - 2
    for (int pl = zc0 - 1; pl <= zc1 + 1; ++pl) {
        const int z = pl - 2;
        const bool out = z >= zc0;
        const float so = ns, lam = nl;
        const float cps[3] = {nps[0], nps[1], nps[2]};
        const float chp = nhp;
        prefetch(z + 1);
        prefetch_head(pl + 1);
        float hz = f0;  // u^3 (adjoint: w^3) of plane pl - 1
        f0 = f1;
        f1 = f2;
        if (pl + 2 <= zc1) f2 = u3at(pl + 2);
        // adjoint layers: copy phi~^xx (x band) and phi~^yy (y rows) at the
        // cross positions of plane pl + 1 into its buffer slot (each thread
        // reads back only its own copies)
        if constexpr (ADJ && PXY) {
            const int zn = pl + 1;
            if (zn >= zc0 && zn < zc1) {
                float* dst = mvb + (size_t)(zn & 1) * NV * NCROSS + tid;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (LX && cpm.sx[k] >= 0)
                        cp_async_4(dst + k * NT, p.phi[0][0] + (unsigned)zn * p.ny * (2 * P + 1) + cpm.sx[k]);
                    if (LY && cpm.sy[k] >= 0)
                        cp_async_4(dst + k * NT + YV * NCROSS, p.phi[1][1] + (unsigned)zn * (2 * P + 1) * p.nx + cpm.sy[k]);
                }
            }
            cp_async_commit();
            cp_async_wait<1>();
        }
        const bool staged = pl >= zc0 && pl < zc1;
        bool ok = true;
        if (staged) {
            const int kk = pl - pfirst;
            ok = mbar_wait_bounded(&bar[kk & (D - 1)], (kk / D) & 1);
        }
        if (ok) {
            if constexpr (ADJ) {
                // z-layer term of E33 (half lattice, plane pl-1)
                const int zm = pl - 1;
                if (own && zm >= 0 && zm < p.nz && zslab(zm, p) >= 0) {
                    const float a = tabv(p, 2, 1, 0, zm), c = tabv(p, 2, 1, 2, zm);
                    hz += a * (chp + c * hz);
                }
            }
            push(qz, hz);
            if constexpr (ADJ && PXY) {
                // E11 = w1 + a (phi~xx + chi w1) in place in the w1 box at the
                // x-band positions and E22 = w2 + a (phi~yy + chi w2) in the w2
                // box at the y-band ones of plane pl, as the plane arrives (off
                // the layers E = w, which the boxes hold already; each box is
                // read by one difference only).  They are differenced two planes
                // later, after the end-of-plane barriers in between.
                if (staged) {
                    float* sw = ring.stage(pl);
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int q = cross.q[k];
                        const float* mv = mvb + (size_t)(pl & 1) * NV * NCROSS + k * NT + tid;
                        if (LX && cpm.sx[k] >= 0) {
                            const float wx = sw[q];
                            const float* t = cxt + cross.cxi[k];
                            sw[q] = wx + t[2 * BW] * (mv[0] + t[3 * BW] * wx);
                        }
                        if (LY && cpm.sy[k] >= 0) {
                            const float wy = sw[BOXS + q];
                            const float* t = cyt + cross.cyi[k];
                            sw[BOXS + q] = wy + t[2 * BH] * (mv[YV * NCROSS] + t[3 * BH] * wy);
                        }
                    }
                    // these generic writes precede the TMA load that refills the stage
                    fence_proxy_async_smem();
                }
            }
        }
        if (out) {
            const float* sz = ring.stage(z);
            const float* XD0 = sz;         // u^1 / E11 (D-x)
            const float* YD0 = sz + BOXS;  // u^2 / E22 (D-y)
            if (ok && own) {
                const float du[3] = {dmx(XD0, o) * h, dmy(YD0, o) * h, dq(qz) * h};
                PmlZ pz{};
                pml_z_init(pz, p, z);
                const unsigned gi = (unsigned)z * nxy + gxy;
                float res;
                if constexpr (!ADJ) {
                    float pd[3] = {0.f, 0.f, 0.f};  // new psi^kk
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        if (in_axis<LX, LY>(j, px, pz.lz)) {
                            const float v = coef(j, 0, 1, px, pz) * cps[j] + coef(j, 0, 0, px, pz) * du[j];
                            p.psi[j][j][own_slab(j, px, pz.lz, x, y, z, p)] = v;
                            pd[j] = v;
                        }
                    const float theta = du[0] + du[1] + du[2] + pd[0] + pd[1] + pd[2];
                    res = so + dt * (lam * theta);
                } else {
                    // psi^^kk <- b (psi^^kk + chi Q_old) at the own point
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        if (in_axis<LX, LY>(j, px, pz.lz))
                            p.psi[j][j][own_slab(j, px, pz.lz, x, y, z, p)] =
                                coef(j, 0, 1, px, pz) * (cps[j] + coef(j, 0, 2, px, pz) * so);
                    res = so - lam * (du[0] + du[1] + du[2]);
                }
                p.s_out[0][gi] = res;
                if (all3) {
                    p.s_out[1][gi] = res;
                    p.s_out[2][gi] = res;
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, 1);
            // a failed wait is on a staged plane pl; drain it and the later ones issued
            drain(bar, pl, min(plast, max(pfirst + D - 1, pl + 1)), pfirst);
            if constexpr (ADJ && PXY) cp_async_wait<0>();
            return false;
        }
        // the stage of plane z (= pl + 2 modulo the ring) is free once every
        // thread has passed the barrier above; planes up to pfirst + D - 1
        // were issued before the loop
        if (tid == 0 && pl + 2 >= pfirst + D && pl + 2 <= plast) issue(pl + 2);
    }
    if constexpr (ADJ && PXY) cp_async_wait<0>();
    if (tid == 0)
        for (int s = 0; s < D; ++s) mbar_inval(&bar[s]);
    return true;
}

// The fluid kernel of a layer kind runs the body of its item's kind: PM_Z
// (z layer only), PM_X or PM_Y (the edge kernel), PM_FULL (the corner kernel).
template <bool STR, bool ADJ, int PM>
__global__ void __launch_bounds__(NT) k_fluid(StepParams p, const __grid_constant__ TmaSet tm, RegionList rl, int* err) {
    extern __shared__ __align__(128) float sm[];
    int tile_x, tile_y, zc0, zc1, kind;
    locate_item(rl, blockIdx.x, tile_x, tile_y, zc0, zc1, kind);
    const bool all3 = !(kind & ITEM_DEEP), alpha = !(kind & ITEM_NOALPHA);
    kind &= ~ITEM_FLAGS;
    if constexpr (PM == PM_X) {
        if (kind == PM_Y) {
            if (STR) str_fluid_body<ADJ, PM_Y>(p, tm.m, tile_x, tile_y, zc0, zc1, err, sm, all3);
            else vel_fluid_body<ADJ, PM_Y>(p, tm.m, tile_x, tile_y, zc0, zc1, err, sm, alpha);
            return;
        }
    }
    if (STR) str_fluid_body<ADJ, PM>(p, tm.m, tile_x, tile_y, zc0, zc1, err, sm, all3);
    else vel_fluid_body<ADJ, PM>(p, tm.m, tile_x, tile_y, zc0, zc1, err, sm, alpha);
}

template <bool STR, bool ADJ, int PM>
size_t fluid_smem_of() {
    return STR ? StrFl<ADJ, PM>::SMEM : VelFl<ADJ, PM>::SMEM;
}

// Shared memory first in the unified L1 / shared-memory array (the bodies
// stage through TMA, not L1), so that shared memory does not cap the blocks
// per SM below the register limit, and the dynamic shared memory of each
// layout allowed (the adjoint corner layout is above the 48 KB default); set
// once per kernel and device.
template <bool STR, bool ADJ, int PM>
void fluid_attrs() {
    cudaFuncSetAttribute(k_fluid<STR, ADJ, PM>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_fluid<STR, ADJ, PM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fluid_smem_of<STR, ADJ, PM>());
}
template <bool STR, bool ADJ>
void prefer_shared() {
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    fluid_attrs<STR, ADJ, PM_Z>();
    fluid_attrs<STR, ADJ, PM_X>();
    fluid_attrs<STR, ADJ, PM_FULL>();
    done[dev] = true;
}

template <bool STR, bool ADJ>
void launch_fl(int pm, const StepParams& p, const TmaSet& tm, const RegionList& rl, int blocks, int* err,
               cudaStream_t st) {
    const dim3 blk(TX, TY, 1);
    prefer_shared<STR, ADJ>();
    if (pm == PM_Z)
        k_fluid<STR, ADJ, PM_Z><<<blocks, blk, fluid_smem_of<STR, ADJ, PM_Z>(), st>>>(p, tm, rl, err);
    else if (pm == PM_X)
        k_fluid<STR, ADJ, PM_X><<<blocks, blk, fluid_smem_of<STR, ADJ, PM_X>(), st>>>(p, tm, rl, err);
    else
        k_fluid<STR, ADJ, PM_FULL><<<blocks, blk, fluid_smem_of<STR, ADJ, PM_FULL>(), st>>>(p, tm, rl, err);
}

// Persistent multi-instance kernel over the fluid C-PML items (z-slab, edge
// and corner kinds, one list) of the medium-adaptive instances in a serving
// table; the dynamic shared memory covers the corner layout, the largest.
template <bool STR, bool ADJ>
__global__ void __launch_bounds__(NT) k_multi_fl(const MultiTable* __restrict__ T, int* err, int* next) {
    extern __shared__ __align__(128) float sm[];
    multi_loop<ADJ, ML_FL>(T, err, next, sm,
                           [](const StepParams& sp, const CUtensorMap* maps, int kind, int tile_x, int tile_y, int zc0,
                              int zc1, int* e, float* smem) {
                               const bool all3 = !(kind & ITEM_DEEP), alpha = !(kind & ITEM_NOALPHA);
                               kind &= ~ITEM_FLAGS;
                               if (kind == PM_Z)
                                   return STR ? str_fluid_body<ADJ, PM_Z>(sp, maps, tile_x, tile_y, zc0, zc1, e, smem, all3)
                                              : vel_fluid_body<ADJ, PM_Z>(sp, maps, tile_x, tile_y, zc0, zc1, e, smem, alpha);
                               if (kind == PM_X)
                                   return STR ? str_fluid_body<ADJ, PM_X>(sp, maps, tile_x, tile_y, zc0, zc1, e, smem, all3)
                                              : vel_fluid_body<ADJ, PM_X>(sp, maps, tile_x, tile_y, zc0, zc1, e, smem, alpha);
                               if (kind == PM_Y)
                                   return STR ? str_fluid_body<ADJ, PM_Y>(sp, maps, tile_x, tile_y, zc0, zc1, e, smem, all3)
                                              : vel_fluid_body<ADJ, PM_Y>(sp, maps, tile_x, tile_y, zc0, zc1, e, smem, alpha);
                               return STR ? str_fluid_body<ADJ, PM_FULL>(sp, maps, tile_x, tile_y, zc0, zc1, e, smem, all3)
                                          : vel_fluid_body<ADJ, PM_FULL>(sp, maps, tile_x, tile_y, zc0, zc1, e, smem, alpha);
                           });
}

template <bool STR, bool ADJ>
int multi_fl_grid() {
    static int grid[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!grid[dev]) {
        const size_t smem = fluid_smem_of<STR, ADJ, PM_FULL>();
        cudaFuncSetAttribute(k_multi_fl<STR, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_multi_fl<STR, ADJ>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        int sms = 148, per_sm = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi_fl<STR, ADJ>, NT, smem);
        grid[dev] = sms * std::max(1, per_sm);
    }
    return grid[dev];
}

template <bool STR, bool ADJ>
void launch_mfl(const MultiTable* dT, int* err, int* next, cudaStream_t st) {
    k_multi_fl<STR, ADJ><<<multi_fl_grid<STR, ADJ>(), dim3(TX, TY, 1), fluid_smem_of<STR, ADJ, PM_FULL>(), st>>>(dT, err,
                                                                                                            next);
}

}  // namespace

// Fluid C-PML items of kind pm (PM_Z, PM_X for the edges, PM_FULL) of one
// half step (str: stress family) on stream st.
void launch_fluid(bool str, bool adj, int pm, const StepParams& p, const TmaSet& tm, const RegionList& rl, int blocks,
                  int* err, cudaStream_t st) {
    if (blocks <= 0) return;
    if (str) {
        if (adj) launch_fl<true, true>(pm, p, tm, rl, blocks, err, st);
        else launch_fl<true, false>(pm, p, tm, rl, blocks, err, st);
    } else {
        if (adj) launch_fl<false, true>(pm, p, tm, rl, blocks, err, st);
        else launch_fl<false, false>(pm, p, tm, rl, blocks, err, st);
    }
}

void launch_multi_fl(bool str, bool adj, const MultiTable* dT, int* err, int* next, cudaStream_t st) {
    if (str) {
        if (adj) launch_mfl<true, true>(dT, err, next, st);
        else launch_mfl<true, false>(dT, err, next, st);
    } else {
        if (adj) launch_mfl<false, true>(dT, err, next, st);
        else launch_mfl<false, false>(dT, err, next, st);
    }
}
