// tiled_common.cuh -- tile geometry, C-PML work-item kinds, shared-memory
// layouts and device helpers of the TMA-staged step kernels, shared by the
// elastic kernels (step_tiled.cu) and the fluid C-PML kernels (step_fluid.cu).
#pragma once
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

// C-PML code of a work-item body:
//   PM_NONE  no layer (tiles and planes whose reach stays off every slab, or P = 0)
//   PM_FULL  x, y and z layers (corner tiles: halo on an x and a y slab)
//   PM_X     x and z layers (tiles whose halo touches an x slab only)
//   PM_Y     y and z layers (tiles whose halo touches a y slab only)
//   PM_Z     z layer only (the other tiles, planes on the z slabs)
// The frame tiles run in three launches (PM_X, PM_Y, PM_FULL); the interior
// launch (PM_NONE) runs, per block, the PM_NONE or the PM_Z body.
constexpr int PM_NONE = 0, PM_FULL = 1, PM_Z = 2, PM_X = 3, PM_Y = 4;
// A fluid work item of a medium-adaptive step (no layer code, the reach all
// fluid): the acoustic kernels run it.
constexpr int PM_AC = 5;
constexpr bool has_x(int pm) { return pm == PM_FULL || pm == PM_X; }
constexpr bool has_y(int pm) { return pm == PM_FULL || pm == PM_Y; }

// Frame adjoint blocks copy the memory variables at their threads' cross
// positions (two positions, three values per layer axis) one plane ahead with
// cp.async into two plane slots of shared memory.
constexpr int mv_values(int pm) { return (has_x(pm) ? 3 : 0) + (has_y(pm) ? 3 : 0); }
// Layout [slot][value][cross position]: a thread's positions are tid and
// tid + TX*TY (the second exists for the first 160 threads only).
constexpr int mv_floats(int pm) { return 2 * mv_values(pm) * ((TX + 4) * TY + 4 * TX); }

template <bool ADJ, int PM> struct VelCfg {
    static constexpr bool PML = PM != PM_NONE, LX = has_x(PM), LY = has_y(PM), PXY = LX || LY;
    // stage boxes 0..5: sigma (forward) or Q (adjoint), Voigt order; 6 rho,
    // 7 alpha.  Frame adjoint blocks form the layer-augmented fields F in
    // place and keep the x-differenced F^21, which differs from the
    // y-differenced F^12 inside the layers, in one extra box.  The adjoint
    // edge bodies read alpha through the cache instead (own point one plane
    // ahead, +x / +y neighbours from L1), which brings their layout under the
    // shared memory of three blocks per SM.
    static constexpr bool ABOX = !(ADJ && (PM == PM_X || PM == PM_Y));
    static constexpr int NB = ABOX ? 8 : 7;
    static constexpr int BRHO = 6, BALPHA = 7;
    static constexpr int NDER = (ADJ && PXY) ? 1 : 0;
    static constexpr int MV = ADJ ? mv_floats(PM) : 0;  // floats of the memory-variable buffer
    static constexpr size_t SMEM = ((size_t)(D * NB + NDER) * BOXS + MV) * sizeof(float) + D * sizeof(uint64_t);
    __host__ __device__ static constexpr int tm(int b) { return b < 6 ? TM_S0 + b : (b == BRHO ? TM_RHO : TM_ALPHA); }
};

template <bool ADJ, int PM> struct StrCfg {
    static constexpr bool PML = PM != PM_NONE, LX = has_x(PM), LY = has_y(PM), PXY = LX || LY;
    // stage boxes 0..2: u (forward) or w (adjoint); 3 lambda (staged for the
    // frame bodies only; the others read it at the own point from own-point
    // loads), 4 1/mu.  Full
    // C-PML adjoint blocks form the layer-augmented fields E in place (the
    // x-differenced ones) and keep the y-differenced ones, which differ inside
    // the layers, in three extra boxes.
    static constexpr int NB = 5;
    static constexpr int NDER = (ADJ && PXY) ? 3 : 0;
    static constexpr int MV = ADJ ? mv_floats(PM) : 0;  // floats of the memory-variable buffer
    static constexpr int BLAM = 3, BMU = 4;
    static constexpr size_t SMEM = ((size_t)(D * NB + NDER) * BOXS + MV) * sizeof(float) + D * sizeof(uint64_t);
    __host__ __device__ static constexpr int tm(int b) { return b < 3 ? TM_U0 + b : (b == 3 ? TM_LAM : TM_MU); }
};

// the edge kernel runs PM_X and PM_Y bodies with one shared-memory layout;
// the interior kernel runs PM_NONE and PM_Z bodies
static_assert(VelCfg<true, PM_X>::SMEM == VelCfg<true, PM_Y>::SMEM && StrCfg<true, PM_X>::SMEM == StrCfg<true, PM_Y>::SMEM &&
                  VelCfg<false, PM_X>::SMEM == VelCfg<false, PM_Y>::SMEM &&
                  StrCfg<false, PM_X>::SMEM == StrCfg<false, PM_Y>::SMEM,
              "edge bodies share one layout");
static_assert(VelCfg<true, PM_NONE>::SMEM == VelCfg<true, PM_Z>::SMEM &&
                  StrCfg<true, PM_NONE>::SMEM == StrCfg<true, PM_Z>::SMEM &&
                  VelCfg<false, PM_NONE>::SMEM == VelCfg<false, PM_Z>::SMEM &&
                  StrCfg<false, PM_NONE>::SMEM == StrCfg<false, PM_Z>::SMEM,
              "interior bodies share one layout");
// the persistent frame kernels run every frame body with the corner layout
static_assert(VelCfg<true, PM_FULL>::SMEM >= VelCfg<true, PM_X>::SMEM &&
                  StrCfg<true, PM_FULL>::SMEM >= StrCfg<true, PM_X>::SMEM &&
                  VelCfg<false, PM_FULL>::SMEM >= VelCfg<false, PM_X>::SMEM &&
                  StrCfg<false, PM_FULL>::SMEM >= StrCfg<false, PM_X>::SMEM,
              "corner layout covers the edge bodies");

__device__ __forceinline__ void locate(const RegionList& rl, int b, int& tile_x, int& tile_y, int& zc0, int& zc1,
                                       int& kind) {
    locate_item(rl, b, tile_x, tile_y, zc0, zc1, kind);
}
// the same for a list held inline (the persistent multi-instance kernels)
__device__ __forceinline__ void locate_inline(const RegionList& rl, int b, int& tile_x, int& tile_y, int& zc0,
                                              int& zc1, int& kind) {
    int r = 0;
    while (r + 1 < rl.n && b >= rl.r[r + 1].bstart) ++r;
    const Region& R = rl.r[r];
    const int lb = b - R.bstart;
    const int ntx = R.tx1 - R.tx0, nt = ntx * (R.ty1 - R.ty0);
    const int t = lb % nt, ch = lb / nt;
    tile_x = R.tx0 + t % ntx;
    tile_y = R.ty0 + t / ntx;
    zc0 = R.za + ch * R.zc;
    zc1 = min(zc0 + R.zc, R.zb);
    kind = R.kind;
}

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

// The TMA-staged kernels read r = 1/mu (+inf at fluid nodes).
// mu = 1/r (0 at fluid nodes); the harmonic mean of four mu is 4 / (r1+r2+r3+r4),
// which is 0 as soon as one node is fluid (the sum is +inf).
__device__ __forceinline__ float mu_of(float r) { return frcp(r); }
__device__ __forceinline__ float harm_inv(float a, float b, float c, float d) {
    return __fdividef(4.0f, a + b + c + d);
}

// The cross-shaped region the x and y differences read: the x band (rows
// OY..OY+TY-1, columns OX-2..OX+TX+1) and four y rows (OY-2, OY-1, OY+TY,
// OY+TY+1; columns OX..OX+TX-1): 416 positions, at most two per thread.  The
// positions a thread owns are the same on every plane, so their box index,
// clamped +x / +y neighbour offsets and band flags are computed once.  A
// thread's first position is its own point; the second, for the first 160
// threads, is one of the 32 x-halo positions (four columns by TY rows) or one
// of the 128 y-row positions, so that a warp's positions lie in one box row
// (no shared-memory bank conflicts) except on the x-halo warp.
constexpr int NCROSS = (TX + 4) * TY + 4 * TX;
static_assert(NCROSS == NT + 4 * TY + 4 * TX && NCROSS <= 2 * NT, "two cross positions per thread");
constexpr unsigned char CP_EXISTS = 1, CP_IN = 2, CP_XB = 4, CP_YB = 8;
struct CrossPos {
    int q[2];
    short dx[2], dy[2];
    short cxi[2], cyi[2];  // the position's box column / row (index into the coefficient tables)
    unsigned char f[2];
};

__device__ __forceinline__ void cross_init(CrossPos& c, int tid, int x0, int y0, int nx, int ny) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int i = tid + k * NT;
        c.q[k] = 0;
        c.dx[k] = c.dy[k] = 0;
        c.cxi[k] = c.cyi[k] = 0;
        c.f[k] = 0;
        if (i >= NCROSS) continue;
        int bx, by;
        bool inx, iny;
        if (i < NT) {  // own point
            bx = OX + i % TX;
            by = OY + i / TX;
            inx = iny = true;
        } else if (i < NT + 4 * TY) {  // x halo: columns OX-2, OX-1, OX+TX, OX+TX+1
            const int j = i - NT, c = j % 4;
            bx = c < 2 ? OX - 2 + c : OX + TX - 2 + c;
            by = OY + j / 4;
            inx = true;
            iny = false;
        } else {  // y rows
            const int j = i - NT - 4 * TY, r = j / TX;
            bx = OX + j % TX;
            by = r < 2 ? OY - 2 + r : OY + TY - 2 + r;
            inx = false;
            iny = true;
        }
        const int gx = x0 - 4 + bx, gy = y0 - 2 + by;
        const bool in = gx >= 0 && gx < nx && gy >= 0 && gy < ny;
        c.q[k] = by * BW + bx;
        c.cxi[k] = (short)bx;
        c.cyi[k] = (short)by;
        c.dx[k] = (gx + 1 < nx) ? 1 : 0;
        c.dy[k] = (gy + 1 < ny) ? BW : 0;
        c.f[k] = CP_EXISTS | (in ? CP_IN : 0) | (inx ? CP_XB : 0) | (iny ? CP_YB : 0);
    }
}

// C-PML data of the cross positions: per box column / row the layer
// coefficients (a and chi on the integer and half lattice) and, per position,
// the slab index base of the x slab (x-band positions) and y slab (y-band
// positions), -1 off the layer.
struct CrossPml {
    int sx[2], sy[2];
};

template <bool LX, bool LY>
__device__ __forceinline__ void cross_pml_init(CrossPml& c, float* cx, float* cy, const CrossPos& cp, int tid,
                                               int x0, int y0, const StepParams& p) {
    const int W = 2 * p.P + 1;
    for (int i = tid; i < BW + BH; i += NT) {
        // one array per coefficient (stride W = BW or BH between them), so
        // that a warp reading one coefficient of consecutive columns hits
        // consecutive banks
        const int axis = i < BW ? 0 : 1;
        const int W = axis == 0 ? BW : BH;
        float* t = axis == 0 ? cx + i : cy + (i - BW);
        const int g = i < BW ? x0 - 4 + i : y0 - 2 + (i - BW);
        const int n = axis == 0 ? p.nx : p.ny;
        const bool in = g >= 0 && g < n && slab_local(g, n, p.P) >= 0;
        t[0] = in ? __ldg(p.tab[axis][0][0] + g) : 0.f;      // a, integer lattice
        t[W] = in ? __ldg(p.tab[axis][0][2] + g) : 0.f;      // chi, integer lattice
        t[2 * W] = in ? __ldg(p.tab[axis][1][0] + g) : 0.f;  // a, half lattice
        t[3 * W] = in ? __ldg(p.tab[axis][1][2] + g) : 0.f;  // chi, half lattice
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        c.sx[k] = c.sy[k] = -1;
        const unsigned char f = cp.f[k];
        if (!(f & CP_IN)) continue;
        const int bx = cp.q[k] % BW, by = cp.q[k] / BW;
        const int gx = x0 - 4 + bx, gy = y0 - 2 + by;
        const int lx = slab_local(gx, p.nx, p.P), ly = slab_local(gy, p.ny, p.P);
        if (LX && (f & CP_XB) && lx >= 0) c.sx[k] = gy * W + lx;
        if (LY && (f & CP_YB) && ly >= 0) c.sy[k] = ly * p.nx + gx;
    }
}

// Shared tables of the layer coefficients of the cross positions (four
// arrays of BW floats over the box columns, then four of BH over the rows:
// a and chi on the integer lattice, a and chi on the half lattice).  One allocation per kernel,
// shared by all its C-PML bodies (a block runs one body at a time), so that a
// kernel that carries both edge bodies pays for the tables once.
__device__ __forceinline__ float* frame_coef_tables() {
    __shared__ float t[4 * BW + 4 * BH];
    return t;
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
    const int l = axis == 0 ? slab_local(gx, p.nx, p.P) : (axis == 1 ? slab_local(gy, p.ny, p.P) : zslab(gz, p));
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

// per-thread C-PML constants of the own column along x and y
struct PmlXY {
    int lx, ly;          // slab coordinate along x / y, -1 outside the layer
    float c[2][2][3];    // [axis x, y][lattice integer, half][a, b, chi]
};

template <bool LX, bool LY>
__device__ __forceinline__ void pml_xy_init(PmlXY& q, const StepParams& p, int x, int y, bool own) {
    q.lx = (LX && own) ? slab_local(x, p.nx, p.P) : -1;
    q.ly = (LY && own) ? slab_local(y, p.ny, p.P) : -1;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh)
#pragma unroll
        for (int w = 0; w < 3; ++w) {
            q.c[0][hh][w] = (LX && q.lx >= 0) ? tabv(p, 0, hh, w, x) : 0.f;
            q.c[1][hh][w] = (LY && q.ly >= 0) ? tabv(p, 1, hh, w, y) : 0.f;
        }
}

// C-PML coefficients of plane z along the z axis
struct PmlZ {
    int lz;
    float c[2][3];
};

__device__ __forceinline__ void pml_z_init(PmlZ& q, const StepParams& p, int z) {
    q.lz = (z >= 0 && z < p.nz) ? zslab(z, p) : -1;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh)
#pragma unroll
        for (int w = 0; w < 3; ++w) q.c[hh][w] = q.lz >= 0 ? tabv(p, 2, hh, w, z) : 0.f;
}

// slab index of the own point (x, y, z) on the slab of `axis`
__device__ __forceinline__ unsigned own_slab(int axis, const PmlXY& q, int lz, int x, int y, int z,
                                             const StepParams& p) {
    const unsigned W = 2 * p.P + 1;
    if (axis == 0) return ((unsigned)z * p.ny + y) * W + q.lx;
    if (axis == 1) return ((unsigned)z * W + q.ly) * p.nx + x;
    return ((unsigned)lz * p.ny + y) * p.nx + x;
}

// own point on the layer of axis j?  Layers without code in the body (LX or
// LY false) are absent, which the compiler sees for an unrolled j.
template <bool LX, bool LY>
__device__ __forceinline__ bool in_axis(int j, const PmlXY& q, int lz) {
    return j == 2 ? lz >= 0 : (j == 0 ? (LX && q.lx >= 0) : (LY && q.ly >= 0));
}

__device__ __forceinline__ float coef(int j, int hh, int w, const PmlXY& q, const PmlZ& qz) {
    return j < 2 ? q.c[j][hh][w] : qz.c[hh][w];
}

