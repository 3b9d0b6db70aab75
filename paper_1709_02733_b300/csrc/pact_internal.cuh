// pact_internal.cuh -- device-side data layout and helpers shared by the step
// kernels of libpact.so.
//
// Layout in HBM (all float32, C order [z][y][x], N = nx*ny*nz):
//   wavefield : u1 u2 u3 s11 s22 s33 s23 s13 s12     (9 arrays of N)
//   medium    : rho lambda mu alpha                  (4 arrays of N, integer nodes)
//   C-PML     : per axis j, six arrays on the two layer slabs normal to j:
//               phi^{1j} phi^{2j} phi^{3j} psi^{1j} psi^{2j} psi^{3j}
//               slab coordinate l in [0, 2P]: l = k for k < P (low face),
//               l = P + k - (n-P-1) for k >= n-P-1 (high face; one extra plane
//               because half-lattice nodes k+1/2 with k = n-P-1 are in the layer)
//   tables    : per axis j and lattice h (0 integer, 1 half): a, b, chi (n_j each)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define PACT_C1 (9.0f / 8.0f)
#define PACT_C2 (1.0f / 24.0f)

// Voigt index of sigma^{ij} (Sec. 2.2 ordering 11, 22, 33, 23, 13, 12).
__host__ __device__ constexpr int voigt(int i, int j) {
    return i == j ? i : (i + j == 1 ? 5 : (i + j == 2 ? 4 : 3));
}

struct StepParams {
    int nx, ny, nz;
    int P;                      // C-PML thickness (0: none)
    // z-slab of a larger grid: this grid's plane k is plane z0g + k of a grid
    // of nzg planes, whose z layers lie at its own ends (z0g = 0, nzg = nz
    // for a whole grid)
    int z0g, nzg;
    float dt, inv_dx;
    float* u[3];                // velocity components (input of a step)
    float* s[6];                // stress, Voigt order (input of a step)
    float* u_out[3];            // where the TMA-staged kernels write the new values:
    float* s_out[6];            // u / s themselves (in place) or the other buffer
    const float* rho;
    const float* lam;
    const float* mu;
    const float* alpha;
    const float* rmu;           // 1/mu (+inf at fluid nodes)
    const float* tab[3][2][3];  // [axis][lattice][a, b, chi]
    float* phi[3][3];           // phi^{ij}: [i][j], slab of axis j
    float* psi[3][3];           // psi^{ij}: [i][j], slab of axis j
};

__device__ __forceinline__ size_t lin3(int x, int y, int z, int nx, int ny) {
    return ((size_t)z * ny + y) * nx + x;
}

__host__ __device__ __forceinline__ int slab_local(int k, int n, int P) {
    if (P <= 0) return -1;
    if (k < P) return k;
    int r = k - (n - P - 1);
    return r >= 0 ? P + r : -1;
}

// slab coordinate of plane z on the z layer (global position), -1 off it
__host__ __device__ __forceinline__ int zslab(int z, const StepParams& p) {
    return slab_local(z + p.z0g, p.nzg, p.P);
}

// slab coordinate of position k along axis A (z: global position)
template <int A>
__host__ __device__ __forceinline__ int axis_slab(int k, const StepParams& p) {
    return A == 2 ? zslab(k, p) : slab_local(k, A == 0 ? p.nx : p.ny, p.P);
}

__device__ __forceinline__ size_t slab_index(int axis, int x, int y, int z, int l, const StepParams& p) {
    const int W = 2 * p.P + 1;
    if (axis == 0) return ((size_t)z * p.ny + y) * W + l;
    if (axis == 1) return ((size_t)z * W + l) * p.nx + x;
    return ((size_t)l * p.ny + y) * p.nx + x;
}

template <int A>
__device__ __forceinline__ int coord(int x, int y, int z) {
    return A == 0 ? x : (A == 1 ? y : z);
}

template <int A>
__device__ __forceinline__ int extent(const StepParams& p) {
    return A == 0 ? p.nx : (A == 1 ? p.ny : p.nz);
}

// C-PML table entry along axis A on lattice `half`: which = 0 (a), 1 (b), 2 (chi)
template <int A>
__device__ __forceinline__ float ptab(const StepParams& p, int half, int which, int k) {
    return __ldg(p.tab[A][half][which] + k);
}

// value of a field with zero padding outside the grid
__device__ __forceinline__ float ldz(const float* __restrict__ f, int x, int y, int z, const StepParams& p) {
    return ((unsigned)x < (unsigned)p.nx && (unsigned)y < (unsigned)p.ny && (unsigned)z < (unsigned)p.nz)
               ? __ldg(f + lin3(x, y, z, p.nx, p.ny))
               : 0.0f;
}

// clamped read of a medium array (edge value past the last index)
__device__ __forceinline__ float ldc(const float* __restrict__ f, int x, int y, int z, const StepParams& p) {
    x = min(x, p.nx - 1);
    y = min(y, p.ny - 1);
    z = min(z, p.nz - 1);
    return __ldg(f + lin3(x, y, z, p.nx, p.ny));
}

// rho or alpha on the u^A node at (x,y,z): arithmetic mean along A
template <int A>
__device__ __forceinline__ float med_avg(const float* __restrict__ f, int x, int y, int z, const StepParams& p) {
    return 0.5f * (ldc(f, x, y, z, p) + ldc(f, x + (A == 0), y + (A == 1), z + (A == 2), p));
}

__device__ __forceinline__ float harm4(float a, float b, float c, float d) {
    if (a == 0.0f || b == 0.0f || c == 0.0f || d == 0.0f) return 0.0f;
    return 4.0f / (1.0f / a + 1.0f / b + 1.0f / c + 1.0f / d);
}

// the two axes spanned by the shear node of Voigt index V (3: 23, 4: 13, 5: 12)
template <int V> struct ShearAxes;
template <> struct ShearAxes<3> { static constexpr int I = 1, J = 2; };
template <> struct ShearAxes<4> { static constexpr int I = 0, J = 2; };
template <> struct ShearAxes<5> { static constexpr int I = 0, J = 1; };

// mu on the shear node of Voigt index V at (x,y,z): harmonic mean of 4 nodes
template <int V>
__device__ __forceinline__ float mu_shear(int x, int y, int z, const StepParams& p) {
    constexpr int I = ShearAxes<V>::I, J = ShearAxes<V>::J;
    const float* m = p.mu;
    return harm4(ldc(m, x, y, z, p), ldc(m, x + (I == 0), y + (I == 1), z + (I == 2), p),
                 ldc(m, x + (J == 0), y + (J == 1), z + (J == 2), p),
                 ldc(m, x + (I == 0) + (J == 0), y + (I == 1) + (J == 1), z + (I == 2) + (J == 2), p));
}

// Receiver tables (built on the host from the receiver positions).
struct RecTable {
    int L;
    const int* corner;      // [L][8] linear indices of the trilinear corners
    const float* weight;    // [L][8] trilinear weights
    // injection, owner-computes: distinct corner points and their contributions
    int ncorner;
    const int* inj_point;   // [ncorner] linear index
    const int* inj_off;     // [ncorner + 1] CSR offsets
    const int* inj_rec;     // [8L] receiver of each contribution
    const float* inj_w;     // [8L] weight of each contribution
};

// A solve advanced by CUDA graphs of whole steps: the graph's receiver
// kernels take the step count, the trace buffers and the receiver table from
// here, so that one captured graph serves every solve of its handle.  The
// last block of each receiver launch advances m.
struct SolveState {
    int m;                 // steps done
    unsigned int done;     // blocks of the running receiver launch that finished
    int nsteps;
    RecTable r;
    float* out;            // forward: traces, (nsteps+1) x L
    const float* in;       // adjoint: traces, (nsteps+1) x L
};
void launch_set_state(SolveState* st, const SolveState& v, cudaStream_t stream);
// Theta row m+1 (forward) / Theta^T row nsteps-(m+1) (adjoint), then m += 1
void launch_sample_state(const StepParams& p, SolveState* st, cudaStream_t stream);
void launch_inject_state(const StepParams& p, SolveState* st, cudaStream_t stream);
