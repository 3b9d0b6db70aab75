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
    RegionList outer;     // work items of the C-PML frame tiles
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
    int pre_outer[kMaxInst + 1];
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
};
// Both return the number of kernels launched.  With fz set the interior
// tiles and planes that the single-pass kernel takes (fused_plan) are left
// out: the step is then launch_vel_tiled, launch_fused_step, launch_str_tiled.
int launch_vel_tiled(bool adj, const StepParams& p, const TmaSet& tm, int* err, const SplitStreams& ss,
                     bool fz = false);
int launch_str_tiled(bool adj, const StepParams& p, const TmaSet& tm, int* err, const SplitStreams& ss,
                     bool fz = false);

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
// grid points one launch set of a role updates: family 0 velocity, 1 stress,
// 2 fused; fz as above
long long role_points(int family, bool fz, const StepParams& p);
// persistent multi-instance half step (str = stress family) over a device
// table: four launches (two directions x frame / interior), launch k taking
// its work items from the counter next[k], which must be zero beforehand
constexpr int kMultiLaunches = 4;
void launch_multi_step_half(bool str, const MultiTable* dT, int* err, int* next, cudaStream_t st);
void plan_instance_regions(const StepParams& p, int zc, RegionList& inner, int& ninner, RegionList& outer,
                           int& nouter);
