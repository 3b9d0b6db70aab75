// step_acoustic.cu -- interior step kernels of the acoustic operator pair
// H_{mu=0}, H^T_{mu=0} (the paper's elastic operator with the shear modulus
// set to zero, Sec. 7 ablation).
//
// The kernels of the all-fluid medium (mu = 0 at every node): each block
// runs the acoustic body (step_acoustic.cuh) on one work item of the
// interior tiles and planes; the C-PML frame and the z-slab planes keep
// running the elastic kernels, which compute the same operator when mu = 0.
#include <algorithm>

#include "pact_internal.cuh"
#include "step_tiled.cuh"
#include "tma.cuh"

#include "step_acoustic.cuh"

using namespace acoustic;

template <bool ADJ>
__global__ void __launch_bounds__(NT) k_ac_vel(StepParams p, const __grid_constant__ TmaSet tm, RegionList rl,
                                               int* err) {
    extern __shared__ __align__(128) float sm[];
    int tile_x, tile_y, zc0, zc1, kind;
    locate_item(rl, blockIdx.x, tile_x, tile_y, zc0, zc1, kind);
    ac_vel_body<ADJ>(p, tm.m, tile_x, tile_y, zc0, zc1, err, sm, !(kind & ITEM_NOALPHA));
}

template <bool ADJ>
__global__ void __launch_bounds__(NT) k_ac_str(StepParams p, const __grid_constant__ TmaSet tm, RegionList rl,
                                               int* err) {
    extern __shared__ __align__(128) float sm[];
    int tile_x, tile_y, zc0, zc1, kind;
    locate_item(rl, blockIdx.x, tile_x, tile_y, zc0, zc1, kind);
    ac_str_body<ADJ>(p, tm.m, tile_x, tile_y, zc0, zc1, err, sm, !(kind & ITEM_DEEP));
}

// Persistent multi-instance kernel over the fluid no-layer items of the
// medium-adaptive instances in a serving table (ADJ: the direction).
template <bool STR, bool ADJ>
__global__ void __launch_bounds__(NT) k_multi_ac(const MultiTable* __restrict__ T, int* err, int* next) {
    extern __shared__ __align__(128) float sm[];
    multi_loop<ADJ, ML_AC>(T, err, next, sm,
                           [](const StepParams& sp, const CUtensorMap* maps, int kind, int tile_x, int tile_y, int zc0,
                              int zc1, int* e, float* smem) {
                               return STR ? ac_str_body<ADJ>(sp, maps, tile_x, tile_y, zc0, zc1, e, smem,
                                                             !(kind & ITEM_DEEP))
                                          : ac_vel_body<ADJ>(sp, maps, tile_x, tile_y, zc0, zc1, e, smem,
                                                             !(kind & ITEM_NOALPHA));
                           });
}

// any mu > 0?  (out[0] |= 1)
__global__ void k_any_shear(const float* __restrict__ mu, size_t n, unsigned int* out) {
    bool any = false;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        any |= mu[i] > 0.0f;
    if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(out, 1u);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t acoustic_smem() { return SMEM; }
const void* acoustic_fn(bool str, bool adj) {
    return str ? (adj ? (const void*)k_ac_str<true> : (const void*)k_ac_str<false>)
               : (adj ? (const void*)k_ac_vel<true> : (const void*)k_ac_vel<false>);
}

// Shared memory first in the unified L1 / shared-memory array (the bodies
// stage through TMA), so that it does not cap the blocks per SM below the
// register limit; set once per device.
static void prefer_shared_ac() {
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    for (int k = 0; k < 4; ++k)
        cudaFuncSetAttribute(acoustic_fn(k & 2, k & 1), cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_multi_ac<false, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_multi_ac<false, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_multi_ac<true, false>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_multi_ac<true, true>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    done[dev] = true;
}

void launch_acoustic(bool str, bool adj, const StepParams& p, const TmaSet& tm, const RegionList& rl, int blocks,
                     int* err, cudaStream_t st) {
    if (blocks <= 0) return;
    prefer_shared_ac();
    const dim3 blk(TX, TY, 1);
    if (str) {
        if (adj) k_ac_str<true><<<blocks, blk, SMEM, st>>>(p, tm, rl, err);
        else k_ac_str<false><<<blocks, blk, SMEM, st>>>(p, tm, rl, err);
    } else {
        if (adj) k_ac_vel<true><<<blocks, blk, SMEM, st>>>(p, tm, rl, err);
        else k_ac_vel<false><<<blocks, blk, SMEM, st>>>(p, tm, rl, err);
    }
}

// sigma^22 = sigma^33 = sigma^11 on the ITEM_DEEP items of a list (one block
// per item; other items are left alone)
__global__ void __launch_bounds__(NT) k_deep_fill(const float* __restrict__ s0, float* s1, float* s2, int nx, int ny,
                                                  RegionList rl) {
    int tile_x, tile_y, zc0, zc1, kind;
    locate_item(rl, blockIdx.x, tile_x, tile_y, zc0, zc1, kind);
    if (!(kind & ITEM_DEEP)) return;
    const int x = tile_x * TX + threadIdx.x, y = tile_y * TY + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const size_t nxy = (size_t)nx * ny;
    for (int z = zc0; z < zc1; ++z) {
        const size_t g = (size_t)z * nxy + (size_t)y * nx + x;
        const float v = s0[g];
        s1[g] = v;
        s2[g] = v;
    }
}

void launch_deep_fill(const StepParams& p, const RegionList& rl, int blocks, cudaStream_t st) {
    if (blocks > 0) k_deep_fill<<<blocks, dim3(TX, TY, 1), 0, st>>>(p.s[0], p.s[1], p.s[2], p.nx, p.ny, rl);
}

void launch_any_shear(const float* mu, size_t n, unsigned int* out, cudaStream_t st) {
    const size_t b = std::min<size_t>((n + 255) / 256, 148 * 8);
    k_any_shear<<<(unsigned)std::max<size_t>(b, 1), 256, 0, st>>>(mu, n, out);
}

template <bool STR, bool ADJ>
static int multi_ac_grid() {
    static int grid[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!grid[dev]) {
        prefer_shared_ac();
        int sms = 148, per_sm = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi_ac<STR, ADJ>, NT, SMEM);
        grid[dev] = sms * std::max(1, per_sm);
    }
    return grid[dev];
}

void launch_multi_ac(bool str, bool adj, const MultiTable* dT, int* err, int* next, cudaStream_t st) {
    const dim3 blk(TX, TY, 1);
    if (str) {
        if (adj) k_multi_ac<true, true><<<multi_ac_grid<true, true>(), blk, SMEM, st>>>(dT, err, next);
        else k_multi_ac<true, false><<<multi_ac_grid<true, false>(), blk, SMEM, st>>>(dT, err, next);
    } else {
        if (adj) k_multi_ac<false, true><<<multi_ac_grid<false, true>(), blk, SMEM, st>>>(dT, err, next);
        else k_multi_ac<false, false><<<multi_ac_grid<false, false>(), blk, SMEM, st>>>(dT, err, next);
    }
}
