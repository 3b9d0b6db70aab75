// noalloc.cu -- pact_forward_noalloc: the forward operator H for callers that
// cannot allocate device memory.
//
// Who needs it: code embedded in a host application that owns all device
// memory through its own pool and forbids outside cudaMalloc / cudaFree (an
// allocation there escapes its accounting, or fails once the pool has reserved
// the device), and latency-critical loops in which cudaMalloc / cudaFree would
// add implicit device synchronisation.  The regular entry points allocate a
// handle's working memory; this one takes all of it from one fixed array that
// the library declares at file scope, so it allocates nothing.  Each call reads
// the medium check back (it waits for the stream) and copies small tables from
// pageable host memory, so a call blocks the host until its stream reaches the
// check and cannot be captured in a CUDA graph.
//
// The array (PACT_NOALLOC_SCRATCH_BYTES, 64 MiB) is committed on a GPU when the
// module that holds it is loaded there -- at the latest by the first call of
// this entry point on that device, under CUDA's default lazy module loading --
// and stays there until the process exits.  It holds the wavefield,
// the C-PML memory variables, the C-PML profile tables, the receiver tables and
// a four-word medium reduction.  The medium, p0 and the traces stay in the
// caller's buffers.  All calls share the array: each call clears what must
// start at zero, and two calls that overlap on the GPU (different streams or
// host threads) race and corrupt each other's results.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "pact.h"
#include "pact_internal.cuh"

// launchers of the step kernels (step_direct.cu) and host helpers (pact_abi.cu)
void launch_fwd_velocity(const StepParams& p, cudaStream_t st);
void launch_fwd_stress(const StepParams& p, cudaStream_t st);
void launch_source(const float* p0, const StepParams& p, cudaStream_t st, unsigned long long* band_count);
void launch_sample(const StepParams& p, const RecTable& r, float* out, cudaStream_t st);
void launch_medium_check(const float* rho, const float* lam, const float* mu, const float* alpha, size_t n,
                         unsigned int* out, cudaStream_t st);
size_t slab_points(const pact_grid_desc& d, int axis);
int check_desc(const pact_grid_desc* d, std::string& why);
void pml_coef(int n, int P, double dx, double dt, double vmax, double R0, double f0, double pos, double& a,
              double& b, double& chi);
void pact_note_error(const std::string& msg);

// The scratch array.  In host code this name is only a stand-in for the device
// symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PACT_NOALLOC_SCRATCH_BYTES];

namespace {

int nerr(int code, const std::string& msg) {
    pact_note_error(msg);
    return code;
}

// Device address of the scratch array in the current context, looked up on
// every call (a cheap lookup) rather than cached per device ordinal: a host
// that binds its own CUDA context gets its own copy of the module, and with it
// another address.  The first lookup in a context loads the module that holds
// the array, which commits its 64 MiB on that device.
int scratch_address(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return nerr(PACT_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    *out = static_cast<unsigned char*>(p);
    return PACT_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

extern "C" int pact_forward_noalloc(const pact_grid_desc* desc, const float* rho, const float* lambda,
                                    const float* mu, const float* alpha, const float* p0, const float* rec_xyz,
                                    int L, int nsteps, float* traces, void* stream) {
    std::string why;
    int rc = check_desc(desc, why);
    if (rc) return nerr(rc, why);
    if (!rho || !lambda || !mu || !alpha || !p0 || !traces) return nerr(PACT_EINVAL, "NULL data pointer");
    if (!rec_xyz || L < 1) return nerr(PACT_EINVAL, "receivers: rec_xyz must be non-NULL and L >= 1");
    if (nsteps < 0) return nerr(PACT_EINVAL, "nsteps < 0");
    const pact_grid_desc& d = *desc;
    const size_t N = (size_t)d.nx * d.ny * d.nz;
    const int nmax = std::max(d.nx, std::max(d.ny, d.nz));
    size_t slab_n[3];
    for (int a = 0; a < 3; ++a) slab_n[a] = slab_points(d, a);

    // scratch layout, every segment 256-byte aligned
    size_t off = 0;
    const size_t o_fields = off;
    off += align256(9 * N * sizeof(float));
    size_t o_slab[3];
    for (int a = 0; a < 3; ++a) {
        o_slab[a] = off;
        off += align256(6 * slab_n[a] * sizeof(float));
    }
    const size_t o_tab = off;
    off += align256(18 * (size_t)nmax * sizeof(float));
    const size_t o_corner = off;
    off += align256(8 * (size_t)L * sizeof(int));
    const size_t o_weight = off;
    off += align256(8 * (size_t)L * sizeof(float));
    const size_t o_red = off;
    off += align256(4 * sizeof(unsigned int));
    if (off > (size_t)PACT_NOALLOC_SCRATCH_BYTES) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "pact_forward_noalloc: this grid and receiver set need %zu bytes of scratch; the fixed array "
                 "holds %zu (use pact_create_grid / pact_forward instead)",
                 off, (size_t)PACT_NOALLOC_SCRATCH_BYTES);
        return nerr(PACT_EINVAL, buf);
    }

    // receivers: validate on the host, build the trilinear corner table
    const int lim[3] = {d.nx - 2, d.ny - 2, d.nz - 2};
    std::vector<int> corner(8 * (size_t)L);
    std::vector<float> weight(8 * (size_t)L);
    for (int l = 0; l < L; ++l) {
        for (int a = 0; a < 3; ++a) {
            const float v = rec_xyz[3 * l + a];
            if (!std::isfinite(v) || v < 0.0f || v > (float)lim[a]) {
                char buf[160];
                snprintf(buf, sizeof buf, "receiver %d coordinate %d = %g outside [0, %d]", l, a, (double)v, lim[a]);
                return nerr(PACT_EINVAL, buf);
            }
        }
        const double x = rec_xyz[3 * l], y = rec_xyz[3 * l + 1], z = rec_xyz[3 * l + 2];
        const int i0 = std::min((int)std::floor(x), d.nx - 2);
        const int j0 = std::min((int)std::floor(y), d.ny - 2);
        const int k0 = std::min((int)std::floor(z), d.nz - 2);
        const double fx = x - i0, fy = y - j0, fz = z - k0;
        int c = 0;
        for (int cz = 0; cz < 2; ++cz)
            for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx, ++c) {
                    corner[8 * l + c] = ((k0 + cz) * d.ny + (j0 + cy)) * d.nx + (i0 + cx);
                    weight[8 * l + c] = (float)((cx ? fx : 1 - fx) * (cy ? fy : 1 - fy) * (cz ? fz : 1 - fz));
                }
    }

    unsigned char* base = nullptr;
    if ((rc = scratch_address(&base))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
#define NCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return nerr(PACT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

    // medium check (one 16-byte read back, which waits for the stream)
    unsigned int* red = reinterpret_cast<unsigned int*>(base + o_red);
    NCK(cudaMemsetAsync(red, 0, 4 * sizeof(unsigned int), st));
    launch_medium_check(rho, lambda, mu, alpha, N, red, st);
    NCK(cudaGetLastError());
    unsigned int hred[4] = {0, 0, 0, 0};
    NCK(cudaMemcpyAsync(hred, red, sizeof hred, cudaMemcpyDeviceToHost, st));
    NCK(cudaStreamSynchronize(st));
    if (hred[2] != 0) {
        char buf[192];
        snprintf(buf, sizeof buf,
                 "medium: %u nodes violate rho > 0, mu >= 0, lambda + 2 mu > 0, 3 lambda + 2 mu > 0, alpha >= 0",
                 hred[2]);
        return nerr(PACT_EINVAL, buf);
    }
    float c2, amax;
    memcpy(&c2, &hred[0], 4);
    memcpy(&amax, &hred[1], 4);
    const double cmax = std::sqrt((double)c2);
    if (!(cmax * d.dt / d.dx < 6.0 / (7.0 * std::sqrt(3.0)))) return nerr(PACT_ECFL, "CFL: c_max dt / dx >= 6/(7 sqrt 3)");
    if (!((double)amax * d.dt < 1.0)) return nerr(PACT_ECFL, "absorption: alpha_max dt >= 1");

    // C-PML tables and receiver tables into the scratch array
    const double vmax = d.pml_vmax > 0 ? d.pml_vmax : cmax;
    std::vector<float> tab(18 * (size_t)nmax, 0.0f);
    const int dims[3] = {d.nx, d.ny, d.nz};
    for (int a = 0; a < 3; ++a)
        for (int l = 0; l < 2; ++l)
            for (int k = 0; k < dims[a]; ++k) {
                double ca, cb, cc;
                pml_coef(dims[a], d.npml, d.dx, d.dt, vmax, d.pml_R0, d.pml_f0, k + 0.5 * l, ca, cb, cc);
                tab[((a * 2 + l) * 3 + 0) * (size_t)nmax + k] = (float)ca;
                tab[((a * 2 + l) * 3 + 1) * (size_t)nmax + k] = (float)cb;
                tab[((a * 2 + l) * 3 + 2) * (size_t)nmax + k] = (float)cc;
            }
    float* tables = reinterpret_cast<float*>(base + o_tab);
    int* dcorner = reinterpret_cast<int*>(base + o_corner);
    float* dweight = reinterpret_cast<float*>(base + o_weight);
    NCK(cudaMemcpyAsync(tables, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    NCK(cudaMemcpyAsync(dcorner, corner.data(), corner.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    NCK(cudaMemcpyAsync(dweight, weight.data(), weight.size() * sizeof(float), cudaMemcpyHostToDevice, st));

    // the wavefield and the memory variables start at zero on every call
    float* fields = reinterpret_cast<float*>(base + o_fields);
    NCK(cudaMemsetAsync(fields, 0, 9 * N * sizeof(float), st));
    for (int a = 0; a < 3; ++a)
        if (slab_n[a]) NCK(cudaMemsetAsync(base + o_slab[a], 0, 6 * slab_n[a] * sizeof(float), st));

    StepParams p{};
    p.nx = d.nx;
    p.ny = d.ny;
    p.nz = d.nz;
    p.P = d.npml;
    p.z0g = 0;
    p.nzg = d.nz;
    p.dt = (float)d.dt;
    p.inv_dx = (float)(1.0 / d.dx);
    for (int i = 0; i < 3; ++i) p.u[i] = fields + i * N;
    for (int v = 0; v < 6; ++v) p.s[v] = fields + (3 + v) * N;
    p.rho = rho;
    p.lam = lambda;
    p.mu = mu;
    p.alpha = alpha;
    for (int a = 0; a < 3; ++a)
        for (int l = 0; l < 2; ++l)
            for (int w = 0; w < 3; ++w) p.tab[a][l][w] = tables + ((a * 2 + l) * 3 + w) * (size_t)nmax;
    for (int j = 0; j < 3; ++j) {
        float* sl = slab_n[j] ? reinterpret_cast<float*>(base + o_slab[j]) : nullptr;
        for (int i = 0; i < 3; ++i) {
            p.phi[i][j] = sl ? sl + i * slab_n[j] : nullptr;
            p.psi[i][j] = sl ? sl + (3 + i) * slab_n[j] : nullptr;
        }
    }
    RecTable r{};
    r.L = L;
    r.corner = dcorner;
    r.weight = dweight;

    launch_source(p0, p, st, nullptr);
    launch_sample(p, r, traces, st);
    for (int m = 1; m <= nsteps; ++m) {
        launch_fwd_velocity(p, st);
        launch_fwd_stress(p, st);
        launch_sample(p, r, traces + (size_t)m * L, st);
    }
    NCK(cudaGetLastError());
#undef NCK
    return PACT_OK;
}
