// step_tiled.cuh -- host interface of the TMA-staged step kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "pact_internal.cuh"

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
struct RegionList {
    int n;
    Region r[kMaxRegions];
};

// One instance (a forward or adjoint solve on its own grid) of the
// persistent multi-instance step kernels.
struct alignas(128) InstDev {
    TmaSet tm;            // tensor maps of this instance's arrays
    StepParams p;
    RegionList inner;     // work items of the interior tiles (off and on the z slabs)
    RegionList edge;      // work items of the frame tiles with one layer (x or y)
    RegionList corner;    // work items of the frame corner tiles (both layers)
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
};
// Step modes of the TMA-staged kernels:
//   STEP_TWO_PASS  every tile runs the elastic velocity and stress kernels;
//   STEP_FUSED     the interior tiles and planes that the single-pass kernel
//                  takes (fused_plan) are left out: launch_vel_tiled,
//                  launch_fused_step, launch_str_tiled;
//   STEP_ACOUSTIC  (mu = 0 everywhere) the no-layer interior region runs the
//                  acoustic kernels: launch_vel_tiled + launch_acoustic_step
//                  (velocity), launch_str_tiled + launch_acoustic_step (stress).
enum { STEP_TWO_PASS = 0, STEP_FUSED = 1, STEP_ACOUSTIC = 2 };
// Both return the number of kernels launched.
int launch_vel_tiled(bool adj, const StepParams& p, const TmaSet& tm, int* err, const SplitStreams& ss,
                     int mode = STEP_TWO_PASS);
int launch_str_tiled(bool adj, const StepParams& p, const TmaSet& tm, int* err, const SplitStreams& ss,
                     int mode = STEP_TWO_PASS);

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
constexpr int kMultiLaunches = 6;
void launch_multi_step_half(bool str, const MultiTable* dT, int* err, int* next, cudaStream_t st);
void plan_instance_regions(const StepParams& p, int zc, RegionList& inner, int& ninner, RegionList& edge,
                           int& nedge, RegionList& corner, int& ncorner);
