// step_fused.cu -- single-pass step kernel of the interior tiles: the
// velocity update and the stress update of one time step of H (Eq. (it)) or
// of H^T (Eq. (backwardstep), in the weighted variables w = dt u~/rho,
// Q = C s~) in one z-march, on ping-pong wavefield buffers.
//
// Each block owns a 32 x 8 column tile and a chunk of z planes.  Per plane it
// stages, with one TMA load per array, the halo box (40 x 14 points:
// x0-4..x0+35, y0-3..y0+10) of the six stress-like fields and of rho, alpha of
// the INPUT buffer, and
//   1. computes the new velocity-like field at plane zu on its own points and
//      on the cross-shaped halo that the stress differences read (two columns
//      on each side of the tile rows, two rows above and below its columns;
//      only the components those differences use), from the staged boxes and
//      per-position register queues of the z-differenced fields;
//   2. writes the own points of the new velocity to the OUTPUT buffer and the
//      whole cross into a four-plane shared ring;
//   3. computes the new stress-like field at plane zs = zu - 2 from that ring
//      (x and y differences), per-thread queues of its own column (z
//      differences), the old stresses of its own points (a two-plane register
//      delay line) and lambda, 1/mu (read through the cache), and writes it
//      to the OUTPUT buffer.
// Each field of the input buffer is read once and each field of the output
// buffer written once per step: 72 B of wavefield and 16 B of medium per grid
// point, against 124 B for the velocity and stress passes run one after the
// other.  The price is the velocity recomputed on the halo cross (1.47x the
// velocity work of the tile).
//
// The tiles and planes this kernel takes have their whole reach -- every
// stress point read and every velocity point computed -- off the C-PML slabs
// and inside the grid, so they carry no layer code: x0-3 >= P, x0+34 <= hi,
// y0-3 >= P, y0+10 <= hi, planes [P+3, hi-2) with hi = n-P-2 (n-1 without a
// layer).  The other tiles and planes run the two-pass kernels of
// step_tiled.cu, which read the same input buffer and write the same output
// buffer.
#include <type_traits>

#include "pact_internal.cuh"
#include "step_tiled.cuh"
#include "tma.cuh"

namespace fused {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int BW = TX + 8;        // stress box columns x0-4 .. x0+TX+3
constexpr int BH = TY + 6;        // stress box rows    y0-3 .. y0+TY+2
constexpr int BOX = BW * BH;      // 560 floats
constexpr int BOXS = 576;         // box stride in floats (2304 B, a multiple of 128 B)
constexpr int OX = 4, OY = 3;     // own point offset inside the box
constexpr int NB = 8;             // boxes per plane: s11 s22 s33 s23 s13 s12 (Voigt), rho, alpha
constexpr int BRHO = 6, BALPHA = 7;
// Ring of D planes: an iteration reads three (pl-2 .. pl) while the next one
// is in flight.  (A fifth stage, two planes in flight, measured no faster.)
constexpr int D = 4;
constexpr int STG = NB * BOXS;    // floats per ring stage
constexpr int UW = TX + 4;        // velocity plane columns x0-2 .. x0+TX+1
constexpr int UH = TY + 4;        // velocity plane rows    y0-2 .. y0+TY+1
constexpr int US = UW * UH;       // 432 floats per component
constexpr int UO = 2;             // own point offset inside a velocity plane
constexpr int NU = 4;             // velocity planes kept (zs .. zs+2, and one being replaced)
constexpr int UPL = 3 * US;       // floats per velocity plane (3 components)
constexpr size_t SMEM = ((size_t)D * STG + (size_t)NU * UPL) * sizeof(float) + D * sizeof(uint64_t);
static_assert(SMEM <= 113 * 1024, "two blocks per SM");

constexpr float C1 = PACT_C1, C2 = PACT_C2;

// Raw (unscaled) differences: the integer->half form d(v, i) = C1 (v[i+s] -
// v[i]) - C2 (v[i+2s] - v[i-s]); the half->integer difference at i is the
// integer->half one at i - s.
template <int S>
__device__ __forceinline__ float dp(const float* v, int i) {
    return C1 * (v[i + S] - v[i]) - C2 * (v[i + 2 * S] - v[i - S]);
}

// A halo unit: one velocity component on one row (y band) or on up to three
// columns (x band) of the cross, computed by one warp.  Y-band units cover the
// 32 columns of the tile; x-band units the columns beside it, 8 rows each:
//   id  0..2  u1 at rows y0-1, y0+8, y0+9        (d+y u1 of s12 needs y-1..y+2)
//   id  3..5  u2 at rows y0-2, y0-1, y0+8        (d-y u2 of s22 needs y-2..y+1)
//   id  6..8  u3 at rows y0-1, y0+8, y0+9        (d+y u3 of s23 needs y-1..y+2)
//   id  9     u1 at columns x0-2, x0-1, x0+32    (d-x u1 of s11 needs x-2..x+1)
//   id 10, 11 u2, u3 at columns x0-1, x0+32, x0+33 (d+x of s12, s13 needs x-1..x+2)
// Warp w computes unit w and, for w < 4, unit 8 + w.  Every component is
//   u_c <- J u_c + k / rho_c (dp_x(X_c) + dp_y(Y_c) + dp_z(queue)),
// with X, Y the stress boxes (Voigt 0 s11, 1 s22, 2 s33, 3 s23, 4 s13, 5 s12)
// and shifts of the component (c = 0: s11 at q, s12 at q-BW; c = 1: s12 at
// q-1, s22 at q; c = 2: s13 at q-1, s23 at q-BW), its z queue fed from s13 /
// s23 of the previous plane (c = 0, 1) or s33 of the head plane (c = 2), and
// rho, alpha averaged with the +x, +y or next-plane node.  A unit stores the
// stage-relative indices of these reads, so its code has no branches.
struct Unit {
    int ix, iy, ih, irn;  // x-, y-difference bases, z-queue head, rho neighbour (stage-relative)
    int q;                // own box index
    int s;                // velocity-plane index (component * US + position)
    int c;                // component (-1: no unit)
    unsigned g;           // y * nx + x
};

__device__ __forceinline__ Unit make_unit(int id, int lane, int x0, int y0, int nx) {
    Unit u{0, 0, 0, 0, 0, 0, -1, 0u};
    int dx, dy;
    if (id < 9) {
        // rows per component: u1, u3 at -1, TY, TY+1; u2 at -2, -1, TY
        u.c = id / 3;
        const int r = id % 3;
        dx = lane;
        dy = u.c == 1 ? (r == 0 ? -2 : (r == 1 ? -1 : TY)) : (r == 0 ? -1 : (r == 1 ? TY : TY + 1));
    } else if (id < 12) {
        if (lane >= 24) return u;
        u.c = id - 9;
        const int c = lane >> 3;
        dx = u.c == 0 ? (c == 0 ? -2 : (c == 1 ? -1 : TX)) : (c == 0 ? -1 : (c == 1 ? TX : TX + 1));
        dy = lane & 7;
    } else {
        return u;
    }
    const int q = (dy + OY) * BW + dx + OX;
    u.q = q;
    u.ix = u.c == 0 ? q : (u.c == 1 ? 5 * BOXS + q - 1 : 4 * BOXS + q - 1);
    u.iy = u.c == 0 ? 5 * BOXS + q - BW : (u.c == 1 ? BOXS + q : 3 * BOXS + q - BW);
    u.ih = u.c == 0 ? 4 * BOXS + q : (u.c == 1 ? 3 * BOXS + q : 2 * BOXS + q);
    u.irn = BRHO * BOXS + q + (u.c == 0 ? 1 : (u.c == 1 ? BW : 0));
    u.s = u.c * US + (dy + UO) * UW + dx + UO;
    u.g = (unsigned)(y0 + dy) * nx + (unsigned)(x0 + dx);
    return u;
}

// dq of a four-plane register queue written cyclically: slot P holds the
// newest plane, slot (P+1)&3 the oldest
template <int P>
__device__ __forceinline__ float dqr(const float (&q)[4]) {
    return C1 * (q[(P + 3) & 3] - q[(P + 2) & 3]) - C2 * (q[P] - q[(P + 1) & 3]);
}

// one velocity component from stage-relative reads: a = stage of the plane,
// an = stage holding the rho / alpha neighbour
__device__ __forceinline__ float vcomp(const float* a, const float* an, int ix, int iy, int ir, int irn, float dz,
                                       float uo, float kv2, float hdt) {
    const float acc = dp<1>(a, ix) + dp<BW>(a, iy) + dz;
    const float r = a[ir] + an[irn];
    const float al = a[ir + (BALPHA - BRHO) * BOXS] + an[irn + (BALPHA - BRHO) * BOXS];
    return (1.0f - hdt * al) * uo + __fdividef(kv2, r) * acc;
}

// bounded drain of loads still in flight after a failed wait
__device__ __forceinline__ void drain(uint64_t* bar, int pfrom, int pto, int pfirst) {
    for (int pl = pfrom; pl <= pto; ++pl) {
        const int k = pl - pfirst;
        mbar_wait_bounded(&bar[k % D], (k / D) & 1);
    }
}

__device__ __forceinline__ void locate(const RegionList& rl, int b, int& tile_x, int& tile_y, int& zc0, int& zc1) {
    int kind;
    locate_item(rl, b, tile_x, tile_y, zc0, zc1, kind);
}

template <int P>
using Phase = std::integral_constant<int, P>;

}  // namespace fused

using namespace fused;

// p.u / p.s: input buffer (old values); p.u_out / p.s_out: output buffer.
// fm: stress-like fields of the input buffer (Voigt order), rho, alpha.
//
// The plane loop is unrolled four times: iteration pl runs phase
// (pl - pfirst) & 3, which fixes at compile time the ring stage of every
// plane it touches, the velocity plane it writes and reads, and the register
// slots of its queues (written cyclically, so no register is moved).
template <bool ADJ>
__global__ void __launch_bounds__(NT, 2) k_fused(StepParams p, const __grid_constant__ FusedMaps fm, RegionList rl,
                                                 int* err) {
    extern __shared__ __align__(128) float sm[];
    int tile_x, tile_y, zc0, zc1;
    fused::locate(rl, blockIdx.x, tile_x, tile_y, zc0, zc1);
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int x0 = tile_x * TX, y0 = tile_y * TY;
    const int nx = p.nx;
    const unsigned nxy = (unsigned)nx * p.ny;
    const unsigned gxy = (unsigned)(y0 + ty) * nx + (unsigned)(x0 + tx);
    const int o = (ty + OY) * BW + tx + OX;       // own stress-box index
    const int os = (ty + UO) * UW + tx + UO;      // own velocity-plane index
    const float dt = p.dt, h = p.inv_dx;
    // velocity: u <- (1 - dt alpha_bar) u + kv / rho_bar * (raw differences),
    // 1 / rho_bar = 2 / (rho + rho'), alpha_bar = (alpha + alpha') / 2
    const float kv2 = 2.0f * (ADJ ? -dt * dt * h : dt * h), hdt = 0.5f * dt;
    // stress: s <- s + ks * C e_raw (forward dt C e(u); adjoint -C e(w))
    const float ks = ADJ ? -h : dt * h;
    const int pfirst = zc0 - 4, plast = zc1 + 3;
    float* uring = sm + (size_t)D * STG;
    uint64_t* bar = reinterpret_cast<uint64_t*>(uring + (size_t)NU * UPL);

    if (tid == 0) {
        for (int s = 0; s < D; ++s) mbar_init(&bar[s], 1);
        mbar_fence_init();
        for (int b = 0; b < NB; ++b) tma_prefetch_desc(&fm.m[b]);
    }
    __syncthreads();
    // plane pl sits in stage (pl - pfirst) % D; its barrier completes phase
    // ((pl - pfirst) / D) & 1
    auto issue = [&](int pl) {
        const int k = (pl - pfirst) & (D - 1);
        float* st = sm + (size_t)k * STG;
        mbar_arrive_expect_tx(&bar[k], NB * BOX * sizeof(float));
        for (int b = 0; b < NB; ++b) tma_load_3d(st + b * BOXS, &fm.m[b], x0 - 4, y0 - 3, pl, &bar[k]);
    };
    if (tid == 0)
        for (int pl = pfirst; pl < pfirst + D && pl <= plast; ++pl) issue(pl);

    const int warp = tid >> 5, lane = tid & 31;
    const Unit ua = make_unit(warp, lane, x0, y0, nx);
    const Unit ub = make_unit(warp < 4 ? 8 + warp : 99, lane, x0, y0, nx);

    // z queues of the stress-like fields for the velocity (own column: s13,
    // s23, s33; the two halo units) and of the new velocity for the stress
    // (own column: u1, u2 for the integer->half differences, u3 for the
    // half->integer one, read before this plane's value enters)
    float q13[4] = {0, 0, 0, 0}, q23[4] = {0, 0, 0, 0}, q33[4] = {0, 0, 0, 0};
    float qa[4] = {0, 0, 0, 0}, qb[4] = {0, 0, 0, 0};
    float v1[4] = {0, 0, 0, 0}, v2[4] = {0, 0, 0, 0}, v3[4] = {0, 0, 0, 0};
    // old own stresses of the last two velocity planes (slot (pl-pfirst)&1)
    float sd[2][6] = {{0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0}};
    // 1/mu of the own point and its +x, +y, +xy neighbours: planes zs, zs+1
    float mu[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    // old velocity of planes zu and zu+1 (own components, unit a, unit b)
    float nu[2][3] = {{0, 0, 0}, {0, 0, 0}}, nua[2] = {0, 0}, nub[2] = {0, 0};
    {
        const unsigned base = (unsigned)(zc0 - 2) * nxy;
        nu[0][0] = p.u[0][base + gxy];
        nu[0][1] = p.u[1][base + gxy];
        nu[0][2] = p.u[2][base + gxy];
        if (ua.c >= 0) nua[0] = p.u[ua.c][base + ua.g];
        if (ub.c >= 0) nub[0] = p.u[ub.c][base + ub.g];
        const float* m = p.rmu + (size_t)zc0 * nxy + gxy;
        mu[0][0] = __ldg(m);
        mu[0][1] = __ldg(m + 1);
        mu[0][2] = __ldg(m + nx);
        mu[0][3] = __ldg(m + nx + 1);
    }

    int pl = pfirst;
    auto step = [&](auto phase) -> bool {
        constexpr int PH = decltype(phase)::value;
        constexpr int S0 = PH * STG;                 // stage of plane pl (z-queue head of s33)
        constexpr int S1 = ((PH + 3) & 3) * STG;     // stage of pl - 1 = zu + 1
        constexpr int S2 = ((PH + 2) & 3) * STG;     // stage of pl - 2 = zu
        constexpr int UZ = ((PH + 2) & 3) * UPL;     // velocity plane zu
        constexpr int UZS = PH * UPL;                // velocity plane zs = zu - 2
        constexpr int A = PH & 1, B = A ^ 1;         // two-slot rotations
        const int zu = pl - 2, zs = pl - 4;
        const bool have = pl <= plast;
        const bool vel = have && pl >= zc0;
        const bool str = zs >= zc0 && zs < zc1;
        // medium of the stress plane and old velocity of the next plane,
        // issued before the wait
        float lam = 0.f;
        if (str) {
            const unsigned g = (unsigned)zs * nxy + gxy;
            lam = __ldg(p.lam + g);
            const float* m = p.rmu + g + nxy;
            mu[B][0] = __ldg(m);
            mu[B][1] = __ldg(m + 1);
            mu[B][2] = __ldg(m + nx);
            mu[B][3] = __ldg(m + nx + 1);
        }
        if (vel && zu + 1 <= zc1 + 1) {
            const unsigned base = (unsigned)(zu + 1) * nxy;
            nu[B][0] = p.u[0][base + gxy];
            nu[B][1] = p.u[1][base + gxy];
            nu[B][2] = p.u[2][base + gxy];
            if (ua.c >= 0) nua[B] = p.u[ua.c][base + ua.g];
            if (ub.c >= 0) nub[B] = p.u[ub.c][base + ub.g];
        }
        bool ok = true;
        if (have) ok = mbar_wait_bounded(&bar[PH], ((pl - pfirst) / D) & 1);
        if (have && ok) {
            q33[PH] = sm[S0 + 2 * BOXS + o];
            q13[PH] = sm[S1 + 4 * BOXS + o];
            q23[PH] = sm[S1 + 3 * BOXS + o];
            if (ua.c >= 0) qa[PH] = sm[(ua.c == 2 ? S0 : S1) + ua.ih];
            if (ub.c >= 0) qb[PH] = sm[(ub.c == 2 ? S0 : S1) + ub.ih];
        }
        float n2 = 0.f;
        if (vel && ok) {
            const float* a = sm + S2;
            const float* an = sm + S1;
            float* uz = uring + UZ;
            constexpr int IR = BRHO * BOXS;
            const float n0 = vcomp(a, a, o, 5 * BOXS + o - BW, IR + o, IR + o + 1, dqr<PH>(q13), nu[A][0], kv2, hdt);
            const float n1 = vcomp(a, a, 5 * BOXS + o - 1, BOXS + o, IR + o, IR + o + BW, dqr<PH>(q23), nu[A][1], kv2,
                                   hdt);
            n2 = vcomp(a, an, 4 * BOXS + o - 1, 3 * BOXS + o - BW, IR + o, IR + o, dqr<PH>(q33), nu[A][2], kv2, hdt);
            uz[os] = n0;
            uz[US + os] = n1;
            uz[2 * US + os] = n2;
            if (zu >= zc0 && zu < zc1) {
                const unsigned gi = (unsigned)zu * nxy + gxy;
                p.u_out[0][gi] = n0;
                p.u_out[1][gi] = n1;
                p.u_out[2][gi] = n2;
            }
            v1[PH] = n0;
            v2[PH] = n1;
            if (ua.c >= 0)
                uz[ua.s] = vcomp(a, ua.c == 2 ? an : a, ua.ix, ua.iy, IR + ua.q, ua.irn, dqr<PH>(qa), nua[A], kv2, hdt);
            if (ub.c >= 0)
                uz[ub.s] = vcomp(a, ub.c == 2 ? an : a, ub.ix, ub.iy, IR + ub.q, ub.irn, dqr<PH>(qb), nub[A], kv2, hdt);
        }
        if (str && ok) {
            const float* uz = uring + UZS;
            // raw differences: e[i][j] = d_j of the velocity component i
            const float e00 = dp<1>(uz, os - 1), e01 = dp<UW>(uz, os), e02 = dqr<PH>(v1);
            const float e10 = dp<1>(uz + US, os), e11 = dp<UW>(uz + US, os - UW), e12 = dqr<PH>(v2);
            const float e20 = dp<1>(uz + 2 * US, os), e21 = dp<UW>(uz + 2 * US, os);
            // u3 queue before this plane's value: oldest in slot PH
            const float e22 = C1 * (v3[(PH + 2) & 3] - v3[(PH + 1) & 3]) - C2 * (v3[(PH + 3) & 3] - v3[PH]);
            const float* mc = mu[A];
            const float* mn = mu[B];
            const float mu2 = 2.0f * __fdividef(1.0f, mc[0]);
            const float m12 = __fdividef(4.0f, mc[0] + mc[1] + mc[2] + mc[3]);
            const float m13 = __fdividef(4.0f, mc[0] + mc[1] + mn[0] + mn[1]);
            const float m23 = __fdividef(4.0f, mc[0] + mc[2] + mn[0] + mn[2]);
            const float lt = lam * (e00 + e11 + e22);
            const float* so = sd[A];
            const unsigned gi = (unsigned)zs * nxy + gxy;
            p.s_out[0][gi] = so[0] + ks * (lt + mu2 * e00);
            p.s_out[1][gi] = so[1] + ks * (lt + mu2 * e11);
            p.s_out[2][gi] = so[2] + ks * (lt + mu2 * e22);
            p.s_out[3][gi] = so[3] + ks * m23 * (e12 + e21);
            p.s_out[4][gi] = so[4] + ks * m13 * (e02 + e20);
            p.s_out[5][gi] = so[5] + ks * m12 * (e01 + e10);
        }
        if (vel && ok) {
            // this plane's old own stresses replace those of zs; u3 enters its queue
#pragma unroll
            for (int v = 0; v < 6; ++v) sd[A][v] = sm[S2 + v * BOXS + o];
            v3[PH] = n2;
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicExch(err, 1);
            drain(bar, pl, min(plast, max(pfirst + D - 1, pl + 1)), pfirst);
            return false;
        }
        // the stage of pl - 2 is free: load plane pl + 2 into it
        if (tid == 0 && pl >= pfirst + 2 && pl + 2 <= plast) issue(pl + 2);
        ++pl;
        return true;
    };
    for (;;) {
        if (!step(Phase<0>{})) return;
        if (!step(Phase<1>{})) return;
        if (!step(Phase<2>{})) return;
        if (!step(Phase<3>{})) return;
        if (pl > plast) break;
    }
    if (tid == 0)
        for (int s = 0; s < D; ++s) mbar_inval(&bar[s]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t fused_smem() { return SMEM; }

const void* fused_fn(bool adj) { return adj ? (const void*)k_fused<true> : (const void*)k_fused<false>; }

void launch_fused(bool adj, const StepParams& p, const FusedMaps& fm, const RegionList& rl, int blocks, int* err,
                  cudaStream_t st) {
    if (blocks <= 0) return;
    const dim3 blk(TX, TY, 1);
    if (adj) k_fused<true><<<blocks, blk, SMEM, st>>>(p, fm, rl, err);
    else k_fused<false><<<blocks, blk, SMEM, st>>>(p, fm, rl, err);
}

// Tensor maps of the fused kernel: float32, box 40 x 14 x 1, zero fill.
int make_fused_maps(FusedMaps* out, float* const* arrays, int nx, int ny, int nz) {
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
    for (int i = 0; i < FM_N; ++i) {
        CUresult r = encode(&out->m[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, arrays[i], dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return -3 - i;
    }
    return 0;
}
