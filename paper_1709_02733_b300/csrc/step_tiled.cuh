// step_tiled.cuh -- host interface of the TMA-staged step kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "pact_internal.cuh"
#include "tma.cuh"

// one tensor map per array: u (3), sigma (6, Voigt), rho, lambda, mu, alpha
enum { TM_U0 = 0, TM_S0 = 3, TM_RHO = 9, TM_LAM = 10, TM_MU = 11, TM_ALPHA = 12, TM_N = 13 };

struct TmaSet {
    CUtensorMap m[TM_N];
};

// A rectangular block of work: tiles [tx0,tx1) x [ty0,ty1), planes [za,zb)
// in chunks of zc planes; bstart = first block (work item) of the region;
// kind = the C-PML code its blocks run (0 none, 1 full, 2 z layer only).
struct Region {
    int tx0, tx1, ty0, ty1, za, zb, zc, bstart, kind;
};
constexpr int kMaxRegions = 8;
// Up to kMaxRegions regions inline, or (dev set) dn regions in device memory,
// ordered by bstart.
struct RegionList {
    int n;
    Region r[kMaxRegions];
    const Region* dev = nullptr;
    int dn = 0;
};

// The region holding work item b: the last region whose first block is <= b.
__device__ __forceinline__ Region region_of(const RegionList& rl, int b) {
    if (rl.dev) {
        int lo = 0, hi = rl.dn - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&rl.dev[mid].bstart) <= b) lo = mid;
            else hi = mid - 1;
        }
        return rl.dev[lo];
    }
    int r = 0;
    while (r + 1 < rl.n && b >= rl.r[r + 1].bstart) ++r;
    return rl.r[r];
}

// tile, z chunk [zc0, zc1) and C-PML kind of work item b
__device__ __forceinline__ void locate_item(const RegionList& rl, int b, int& tile_x, int& tile_y, int& zc0,
                                            int& zc1, int& kind) {
    const Region R = region_of(rl, b);
    const int lb = b - R.bstart;
    const int ntx = R.tx1 - R.tx0, nt = ntx * (R.ty1 - R.ty0);
    const int t = lb % nt, ch = lb / nt;
    tile_x = R.tx0 + t % ntx;
    tile_y = R.ty0 + t / ntx;
    zc0 = R.za + ch * R.zc;
    zc1 = min(zc0 + R.zc, R.zb);
    kind = R.kind;
}

// One instance (a forward or adjoint solve on its own grid) of the
// persistent multi-instance step kernels.
struct alignas(128) InstDev {
    TmaSet tm;            // tensor maps of this instance's arrays
    StepParams p;
    RegionList inner;     // work items of the interior tiles (off and on the z slabs)
    RegionList edge;      // work items of the frame tiles with one layer (x or y)
    RegionList corner;    // work items of the frame corner tiles (both layers)
    RegionList ac;        // medium-adaptive handles: fluid no-layer items (acoustic body)
    RegionList fl;        // medium-adaptive handles: fluid C-PML items (z slab, edge and corner kinds)
    RecTable rec;
    const float* src;     // adjoint: traces to inject
    float* dst;           // forward: traces to sample into
    int adj;              // 0 forward, 1 adjoint
    int m;                // steps done (advanced on the device)
    int nsteps;
    int L;
};

constexpr int kMaxInst = 64;
struct MultiTable {
    int n_inst;
    int n_fwd;                     // instances [0, n_fwd) are forward, the rest adjoint
    int pre_inner[kMaxInst + 1];   // first work item of each instance
    int pre_edge[kMaxInst + 1];
    int pre_corner[kMaxInst + 1];
    int pre_ac[kMaxInst + 1];
    int pre_fl[kMaxInst + 1];
    InstDev inst[kMaxInst];
};

// 0 on success; arrays[i] is the device base address of array i (order above)
int make_tma_set(TmaSet* out, float* const* arrays, int nx, int ny, int nz);
// Streams of one half step: the interior launch goes to st; with aux set,
// the C-PML frame launch goes to aux between the events fork (recorded on st)
// and join (waited for by st), so that the two launches may overlap.
struct SplitStreams {
    cudaStream_t st;
    cudaStream_t aux;
    cudaEvent_t fork, join;
    cudaStream_t aux2;           // optional: the corner launch runs here (join2 recorded after it)
    cudaEvent_t join2;
    // optional (medium-adaptive step): four more streams, so that each of
    // the seven work lists of a half step runs on a stream of its own
    const cudaStream_t* more = nullptr;
    const cudaEvent_t* more_join = nullptr;
};
// Step modes of the TMA-staged kernels:
//   STEP_TWO_PASS  every tile runs the elastic velocity and stress kernels;
//   STEP_FUSED     the interior tiles and planes that the single-pass kernel
//                  takes (fused_plan) are left out: launch_vel_tiled,
//                  launch_fused_step, launch_str_tiled;
//   STEP_ACOUSTIC  (mu = 0 everywhere) the no-layer interior region runs the
//                  acoustic kernels: launch_vel_tiled + launch_acoustic_step
//                  (velocity), launch_str_tiled + launch_acoustic_step (stress).
//   STEP_MIXED     (mu > 0 somewhere) the interior work items whose whole
//                  reach is fluid run the acoustic kernels, the others the
//                  elastic ones, from a per-medium plan (MixedPlan).
enum { STEP_TWO_PASS = 0, STEP_FUSED = 1, STEP_ACOUSTIC = 2, STEP_MIXED = 3 };

// Work lists of a medium (STEP_MIXED), in device memory.  A tile and plane
// is fluid if mu = 0 at every integer node of its reach (x0-3 .. x0+TX+2,
// y0-3 .. y0+TY+2, z-3 .. z+3): there every stress and velocity the elastic
// update reads has sigma^11 = sigma^22 = sigma^33 and zero shear, so the
// acoustic update (no layer) or the fluid C-PML update (step_fluid.cu)
// computes the same operator.  Every list is one tile per region, ordered by
// z chunk.
enum {
    MX_INT_EL = 0,   // interior tiles with solid in reach: no-layer and z-slab planes (elastic)
    MX_INT_AC,       // interior tiles, fluid, no-layer planes (acoustic kernels)
    MX_INT_FZ,       // interior tiles, fluid, z-slab planes (fluid C-PML kernels)
    MX_EDGE_EL,      // frame edges (x or y layer) with solid in reach (elastic)
    MX_EDGE_FL,      // frame edges, fluid
    MX_CORNER_EL,    // frame corners (x and y layers), solid in reach (elastic)
    MX_CORNER_FL,    // frame corners, fluid
    MX_N
};
// Flag bit of Region.kind: a fluid item (acoustic or fluid C-PML) that no
// elastic item reads (no solid within one tile in x and y and three planes in
// z).  Only elastic bodies read sigma^22 and sigma^33 of other points, so the
// fluid stress bodies write sigma^11 alone there.  The other two hold stale
// values until launch_deep_fill copies sigma^11 into them (before an image
// read-out or a wavefield copy), and the receiver sampler reads 3 sigma^11 at
// such points.
constexpr int ITEM_DEEP = 0x100;
// Flag bit of Region.kind: a fluid item whose velocity body reads alpha = 0 at
// every node (the node and its +1 neighbours in x, y and z over the item's
// tiles and planes): it loads no alpha box and its damping factors are 1.
constexpr int ITEM_NOALPHA = 0x200;
constexpr int ITEM_FLAGS = ITEM_DEEP | ITEM_NOALPHA;

struct MixedPlan {
    RegionList list[MX_N];
    int blocks[MX_N] = {};
    long long points[MX_N] = {};
    RegionList fluid_frame;      // MX_INT_FZ, MX_EDGE_FL, MX_CORNER_FL in one list (serving)
    int fluid_frame_blocks = 0;
    Region* mem = nullptr;       // device allocation behind the lists
    // host map [z][tile] of the planes of ITEM_DEEP items (tile = ty * ntx + tx)
    unsigned char* deep = nullptr;
    int ntx = 0, nty = 0;
    long long deep_points = 0, noalpha_points = 0;
};
// Is grid point (x, y, z) in an ITEM_DEEP item of the plan?  (tiles of
// kTileX x kTileY points, the step kernels' tiles)
constexpr int kTileX = 32, kTileY = 8;
inline bool plan_deep(const MixedPlan& mp, int x, int y, int z) {
    if (!mp.deep) return false;
    return mp.deep[(size_t)z * mp.ntx * mp.nty + (size_t)(y / kTileY) * mp.ntx + x / kTileX] != 0;
}
// sigma^22 = sigma^33 = sigma^11 on the ITEM_DEEP items of list rl (blocks = its blocks)
void launch_deep_fill(const StepParams& p, const RegionList& rl, int blocks, cudaStream_t st);
// Build the plan of the grid of p for the medium's mu (device array);
// returns 0 on success (with no fluid item every list but the elastic ones is
// empty), nonzero on a CUDA error.  Synchronises st.
int build_mixed_plan(const StepParams& p, const float* mu, const float* alpha, cudaStream_t st, MixedPlan* mp);
void free_mixed_plan(MixedPlan* mp);

// Both return the number of kernels launched.  With mode STEP_MIXED, mp
// gives the work lists: on the main stream the elastic interior items, the
// fluid z-slab items and the acoustic items; on the frame streams the elastic
// and fluid edge and corner items.
int launch_vel_tiled(bool adj, const StepParams& p, const TmaSet& tm, int* err, const SplitStreams& ss,
                     int mode = STEP_TWO_PASS, const MixedPlan* mp = nullptr);
int launch_str_tiled(bool adj, const StepParams& p, const TmaSet& tm, int* err, const SplitStreams& ss,
                     int mode = STEP_TWO_PASS, const MixedPlan* mp = nullptr);

// Fluid C-PML kernels (step_fluid.cu): items of kind pm (PM_Z items with
// pm = 2, edge items (PM_X or PM_Y) with pm = 3, corner items with pm = 1).
void launch_fluid(bool str, bool adj, int pm, const StepParams& p, const TmaSet& tm, const RegionList& rl, int blocks,
                  int* err, cudaStream_t st);

// Acoustic interior kernels (step_acoustic.cu): the elastic tensor maps (the
// velocity kernel reads sigma^11, rho, alpha; the stress kernel u^1..u^3).
size_t acoustic_smem();
const void* acoustic_fn(bool str, bool adj);
void launch_acoustic(bool str, bool adj, const StepParams& p, const TmaSet& tm, const RegionList& rl, int blocks,
                     int* err, cudaStream_t st);
// the acoustic half step over the interior region; returns 1 if launched
int launch_acoustic_step(bool str, bool adj, const StepParams& p, const TmaSet& tm, int* err, cudaStream_t st);
// out[0] |= 1 if any mu > 0
void launch_any_shear(const float* mu, size_t n, unsigned int* out, cudaStream_t st);

// Single-pass (velocity + stress) kernel of the interior tiles (step_fused.cu).
// Its tensor maps: the six stress-like fields of the input buffer (Voigt
// order), rho, alpha; box 40 x 14.
enum { FM_N = 8 };
struct FusedMaps {
    CUtensorMap m[FM_N];
};
int make_fused_maps(FusedMaps* out, float* const* arrays, int nx, int ny, int nz);
size_t fused_smem();
const void* fused_fn(bool adj);
void launch_fused(bool adj, const StepParams& p, const FusedMaps& fm, const RegionList& rl, int blocks, int* err,
                  cudaStream_t st);
// the fused region of a grid (false if the grid has none)
bool fused_plan(const StepParams& p, RegionList& rl, int& blocks);
// returns 1 if the fused kernel was launched (0: the grid has no fused region)
int launch_fused_step(bool adj, const StepParams& p, const FusedMaps& fm, int* err, cudaStream_t st);
// grid points one launch set of a role updates: family 0 velocity (elastic
// kernels), 1 stress (elastic kernels), 2 fused, 3 acoustic interior
long long role_points(int family, int mode, const StepParams& p);
// persistent multi-instance half step (str = stress family) over a device
// table: six launches (two directions x corner / edge / interior), launch k
// taking its work items from the counter next[k], which must be zero beforehand
constexpr int kMultiLaunches = 10;
void launch_multi_step_half(bool str, const MultiTable* dT, int* err, int* next, cudaStream_t st);
void plan_instance_regions(const StepParams& p, int zc, RegionList& inner, int& ninner, RegionList& edge,
                           int& nedge, RegionList& corner, int& ncorner);

// ---- persistent multi-instance loop --------------------------------------
// The work lists of an instance that the persistent kernels walk.
enum { ML_INNER = 0, ML_EDGE = 1, ML_CORNER = 2, ML_AC = 3, ML_FL = 4 };
__device__ __forceinline__ const RegionList& inst_list(const InstDev& I, int which) {
    return which == ML_INNER ? I.inner
         : which == ML_EDGE  ? I.edge
         : which == ML_CORNER ? I.corner
         : which == ML_AC    ? I.ac
                             : I.fl;
}
__device__ __forceinline__ const int* table_pre(const MultiTable* T, int which) {
    return which == ML_INNER ? T->pre_inner
         : which == ML_EDGE  ? T->pre_edge
         : which == ML_CORNER ? T->pre_corner
         : which == ML_AC    ? T->pre_ac
                             : T->pre_fl;
}

// A fixed grid works through the items of list WHICH of every unfinished
// instance of one direction (ADJ) in the table; each block takes the next item
// from an atomic counter (zeroed before the launch).  body(p, maps, kind,
// tile_x, tile_y, zc0, zc1, err, sm) runs one item and returns false if a
// bounded wait gave up.  The instance's parameters are copied to shared memory.
template <bool ADJ, int WHICH, typename Body>
__device__ __forceinline__ void multi_loop(const MultiTable* __restrict__ T, int* err, int* next, float* sm,
                                           Body&& body) {
    __shared__ StepParams sp;
    __shared__ int s_item;
    const int nthreads = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int i0 = ADJ ? T->n_fwd : 0, i1 = ADJ ? T->n_inst : T->n_fwd;
    const int* pre = table_pre(T, WHICH);
    const int first = pre[i0], total = pre[i1];
    for (;;) {
        __syncthreads();  // the previous item is finished with s_item and sp
        if (tid == 0) s_item = first + atomicAdd(next, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) return;
        int i = i0;
        while (i + 1 < i1 && item >= pre[i + 1]) ++i;
        const InstDev& I = T->inst[i];
        if (I.m >= I.nsteps) continue;  // finished instance (uniform per block)
        int tile_x, tile_y, zc0, zc1, kind;
        locate_item(inst_list(I, WHICH), item - pre[i], tile_x, tile_y, zc0, zc1, kind);
        // a work item must lie inside its instance's grid and the instance
        // must be of this kernel's direction; otherwise record the
        // inconsistency and touch nothing
        if (tile_x < 0 || tile_x * 32 >= I.p.nx || tile_y < 0 || tile_y * 8 >= I.p.ny || zc0 < 0 || zc0 >= zc1 ||
            zc1 > I.p.nz || (I.adj != 0) != ADJ) {
            if (tid == 0) atomicExch(err, 2);
            continue;
        }
        for (int w = tid; w < (int)(sizeof(StepParams) / sizeof(int)); w += nthreads)
            reinterpret_cast<int*>(&sp)[w] = reinterpret_cast<const int*>(&I.p)[w];
        if (tid == 0)
            for (int b = 0; b < TM_N; ++b) tensormap_acquire(&I.tm.m[b]);
        __syncthreads();
        if (!body(sp, I.tm.m, kind, tile_x, tile_y, zc0, zc1, err, sm)) return;
    }
}

// persistent launches over the fluid lists of medium-adaptive instances:
// acoustic body (step_acoustic.cu) and fluid C-PML bodies (step_fluid.cu)
void launch_multi_ac(bool str, bool adj, const MultiTable* dT, int* err, int* next, cudaStream_t st);
void launch_multi_fl(bool str, bool adj, const MultiTable* dT, int* err, int* next, cudaStream_t st);
