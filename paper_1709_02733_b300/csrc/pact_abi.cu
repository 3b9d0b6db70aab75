// pact_abi.cu -- host side of the C ABI declared in include/pact.h.
//
// A handle owns, on one device: the wavefield (9 x N floats), a copy of the
// medium (4 x N), the C-PML memory variables on the layer slabs, the 1-D C-PML
// profile tables, the receiver tables and staging buffers for the host-pointer
// calls.  All work is queued on the handle's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pact.h"
#include "pact_internal.cuh"
#include "step_tiled.cuh"

void launch_fwd_velocity(const StepParams& p, cudaStream_t st);
void launch_fwd_stress(const StepParams& p, cudaStream_t st);
void launch_adj_a(const StepParams& p, cudaStream_t st);
void launch_adj_b(const StepParams& p, cudaStream_t st);
void launch_source(const float* p0, const StepParams& p, cudaStream_t st, unsigned long long* band_count);
void launch_readout(float* img, const StepParams& p, cudaStream_t st);
void launch_sample(const StepParams& p, const RecTable& r, float* out, cudaStream_t st);
void launch_inject(const StepParams& p, const RecTable& r, const float* ph, cudaStream_t st);
void launch_inv_mu(const float* mu, float* inv, size_t n, cudaStream_t st);
void launch_medium_check(const float* rho, const float* lam, const float* mu, const float* alpha, size_t n,
                         unsigned int* out, cudaStream_t st);

namespace {

thread_local std::string g_err;

struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct pact_grid {
    pact_grid_desc d{};
    cudaStream_t stream = nullptr;
    int device = 0;
    size_t N = 0;
    float* fields = nullptr;      // 9N
    float* medium = nullptr;      // 5N: rho, lambda, mu, alpha, 1/mu
    float* tables = nullptr;      // 3 axes x 2 lattices x 3 (a,b,chi) x nmax
    int nmax = 0;
    float* slabs[3] = {nullptr, nullptr, nullptr};  // 6 x slab size per axis
    size_t slab_n[3] = {0, 0, 0};
    unsigned int* scratch_u32 = nullptr;            // [0..2] medium check, [3] error word, [4] any mu > 0,
                                                    // [6..7] p0-near-the-layer count (64 bit)
    bool medium_set = false;
    double cmax = 0.0;
    // receivers
    std::vector<float> rec_host;
    long long rec_medium_gen = -1;  // medium_gen the device tables were built for
    int L = 0;
    int rec_cap = 0;
    int* rec_corner = nullptr;
    float* rec_weight = nullptr;
    int ncorner = 0;
    int* inj_point = nullptr;
    int* inj_off = nullptr;
    int* inj_rec = nullptr;
    float* inj_w = nullptr;
    // staging for *_host calls
    float* stage_a = nullptr;
    size_t stage_a_n = 0;
    float* stage_b = nullptr;
    size_t stage_b_n = 0;
    // launch accounting and optional per-launch events (pact_profile)
    long long launches[PACT_NKIND] = {};  // invocations of each role
    long long kernels = 0;                 // kernel launches of all roles
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;  // kind of the launch that ends at event i (-1: origin)
    // TMA-staged kernels (nx % 4 == 0) or the direct kernels
    bool tiled = false;
    TmaSet tm{};
    // single-pass interior kernel on two wavefield buffers: fields and
    // fields2 (allocated at the first solve); cur = the buffer holding the
    // state.  tmp[c] / fmp[c]: maps of a step whose input is buffer c (the
    // two-pass kernels read the stresses of buffer c and the velocities of
    // buffer 1-c; the single-pass kernel the stresses of buffer c).
    bool fused = false;
    // mu = 0 at every node: the interior runs the acoustic kernels
    bool acoustic = false;
    // mu > 0 somewhere: the fluid interior work items run the acoustic
    // kernels, the rest the elastic ones (plan built from the medium)
    bool mixed = false;
    MixedPlan mixed_plan{};
    long long medium_gen = 0;  // pact_set_medium calls (the receiver tables depend on the plan)
    // a slab of a larger grid (pact_create_slab): plane k is plane z0g + k of nzg
    int z0g = 0, nzg = 0;
    float* fields2 = nullptr;
    int cur = 0;
    TmaSet tmp[2]{};
    FusedMaps fmp[2]{};
    // the C-PML frame launches overlap the interior launches on this stream
    cudaStream_t aux = nullptr, aux2 = nullptr;   // frame edges / frame corners
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    // medium-adaptive step: four more streams, one per work list
    // (PACT_LISTSTREAMS=0 keeps the lists on the three streams above)
    cudaStream_t xs[4] = {};
    cudaEvent_t xj[4] = {};
    bool list_streams = false;
    // CUDA graphs of whole steps for pact_forward / pact_adjoint (two-pass
    // TMA-staged path, profiling off): graphs[adjoint][0] one step,
    // graphs[adjoint][1] kGraphSteps steps, captured on `cap` after one step
    // launched directly (which builds every launch plan the capture uses);
    // their receiver kernels read the solve from solve_dev.  Dropped when the
    // medium changes (the launch lists depend on it).
    struct StepGraph {
        cudaGraphExec_t exec = nullptr;
        long long kernels = 0;
        long long launches[PACT_NKIND] = {};
    };
    StepGraph graphs[2][2];
    bool graph_warm[2] = {false, false};
    bool graph_off = false;  // a capture failed: launch directly
    SolveState* solve_dev = nullptr;
    cudaStream_t cap = nullptr;
    // serving state (pact_begin / pact_advance / pact_poll)
    bool sv_active = false;
    bool sv_solo = false;  // advanced by its own step graphs, not the multi-instance kernels
    // pact_advance runs each such solve's steps on this stream, forked from
    // the caller's stream and joined back (solves overlap on the device)
    cudaStream_t sv_stream = nullptr;
    cudaEvent_t sv_fork = nullptr, sv_join = nullptr;
    int sv_adj = 0, sv_m = 0, sv_nsteps = 0;
    const float* sv_in = nullptr;
    float* sv_out = nullptr;
    RegionList sv_inner{}, sv_edge{}, sv_corner{}, sv_ac{}, sv_fl{};
    int sv_ninner = 0, sv_nedge = 0, sv_ncorner = 0, sv_nac = 0, sv_nfl = 0;
    std::string err;
};

int serve_run(const MultiTable& T, int ksteps, cudaStream_t st, std::string& why);

// message for pact_last_error(NULL) from calls that have no handle
void pact_note_error(const std::string& msg) { g_err = msg; }

static int fail(pact_handle h, int code, const std::string& msg) {
    if (h) h->err = msg;
    g_err = msg;
    return code;
}

#define CK(h, call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((h), e_ == cudaErrorMemoryAllocation ? PACT_ENOMEM : PACT_ECUDA,     \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                 \
    } while (0)

// Count a launch of `kind`; in profile mode record an event after it on the
// stream, so that the launch's duration is the time since the previous event.
static void mark(pact_handle h, int kind, int nkernels = 1) {
    if (kind >= 0) {
        h->launches[kind]++;
        h->kernels += nkernels;
    }
    if (!h->prof) return;
    const size_t i = h->ev_kind.size();
    if (i >= h->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            h->prof = false;
            return;
        }
        h->ev_pool.push_back(e);
    }
    cudaEventRecord(h->ev_pool[i], h->stream);
    h->ev_kind.push_back(kind);
}

size_t slab_points(const pact_grid_desc& d, int axis) {
    if (d.npml <= 0) return 0;
    const size_t W = 2 * (size_t)d.npml + 1;
    if (axis == 0) return (size_t)d.nz * d.ny * W;
    if (axis == 1) return (size_t)d.nz * W * d.nx;
    return W * d.ny * d.nx;
}

int check_desc(const pact_grid_desc* d, std::string& why) {
    if (!d) { why = "desc is NULL"; return PACT_EINVAL; }
    if (d->npml < 0) { why = "npml < 0"; return PACT_EINVAL; }
    const int need = std::max(4, 2 * d->npml + 2);
    if (d->nx < need || d->ny < need || d->nz < need) {
        why = "every grid dimension must be >= max(4, 2*npml+2)";
        return PACT_EINVAL;
    }
    if (!(d->dx > 0) || !(d->dt > 0) || !std::isfinite(d->dx) || !std::isfinite(d->dt)) {
        why = "dx and dt must be positive";
        return PACT_EINVAL;
    }
    if ((size_t)d->nx * d->ny * d->nz >= (size_t)1 << 31) {
        why = "grid too large (N must be < 2^31)";
        return PACT_EINVAL;
    }
    if (d->npml > 0 && (!(d->pml_R0 > 0 && d->pml_R0 < 1) || !(d->pml_f0 >= 0))) {
        why = "C-PML needs 0 < pml_R0 < 1 and pml_f0 >= 0";
        return PACT_EINVAL;
    }
    return PACT_OK;
}

static size_t desc_bytes(const pact_grid_desc& d, int L, int nsteps) {
    const size_t N = (size_t)d.nx * d.ny * d.nz;
    size_t b = 14 * N * sizeof(float);  // fields + medium (incl. 1/mu)
    for (int a = 0; a < 3; ++a) b += 6 * slab_points(d, a) * sizeof(float);
    const int nmax = std::max(d.nx, std::max(d.ny, d.nz));
    b += 18 * (size_t)nmax * sizeof(float) + 16;
    if (L > 0) b += (size_t)L * 8 * (4 + 4 + 4 + 4 + 4 + 4) + 4;  // corner, weight, inj tables
    if (L > 0 && nsteps >= 0) b += (N + (size_t)(nsteps + 1) * L) * sizeof(float);  // host-call staging
    return b;
}

// C-PML 1-D profile (Appendix A.1, kappa = 1) at grid coordinate pos on an axis of n nodes.
void pml_coef(int n, int P, double dx, double dt, double vmax, double R0, double f0, double pos,
                     double& a, double& b, double& chi) {
    a = 0.0;
    b = 1.0;
    chi = 0.0;
    if (P <= 0) return;
    double s = 0.0;
    if (pos < P) s = P - pos;
    else if (pos > n - 1 - P) s = pos - (n - 1 - P);
    if (s <= 0.0) return;
    s = std::min(s, (double)P);
    const double d0 = -3.0 * vmax * std::log(R0) / (2.0 * P * dx);
    const double r = s / P;
    const double dd = d0 * r * r;
    const double beta = M_PI * f0 * (1.0 - r);
    b = std::exp(-(dd + beta) * dt);
    a = (dd + beta) > 0.0 ? dd * (b - 1.0) / (dd + beta) : 0.0;
    chi = 1.0;
}

static float* buffer(pact_handle h, int c) { return c == 0 ? h->fields : h->fields2; }

// Parameters of a step reading wavefield buffer `in` and writing buffer
// `out` (out < 0: in place, which the direct, serving and small kernels use).
static StepParams make_params(pact_handle h, int in = 0, int out = -1) {
    StepParams p{};
    const pact_grid_desc& d = h->d;
    p.nx = d.nx;
    p.ny = d.ny;
    p.nz = d.nz;
    p.P = d.npml;
    p.z0g = h->z0g;
    p.nzg = h->nzg;
    p.dt = (float)d.dt;
    p.inv_dx = (float)(1.0 / d.dx);
    float* fi = buffer(h, in);
    float* fo = out < 0 ? fi : buffer(h, out);
    for (int i = 0; i < 3; ++i) p.u[i] = fi + i * h->N;
    for (int v = 0; v < 6; ++v) p.s[v] = fi + (3 + v) * h->N;
    for (int i = 0; i < 3; ++i) p.u_out[i] = fo + i * h->N;
    for (int v = 0; v < 6; ++v) p.s_out[v] = fo + (3 + v) * h->N;
    p.rho = h->medium;
    p.lam = h->medium + h->N;
    p.mu = h->medium + 2 * h->N;
    p.alpha = h->medium + 3 * h->N;
    p.rmu = h->medium + 4 * h->N;
    for (int a = 0; a < 3; ++a)
        for (int l = 0; l < 2; ++l)
            for (int w = 0; w < 3; ++w) p.tab[a][l][w] = h->tables + ((a * 2 + l) * 3 + w) * (size_t)h->nmax;
    for (int j = 0; j < 3; ++j)
        for (int i = 0; i < 3; ++i) {
            p.phi[i][j] = h->slabs[j] ? h->slabs[j] + i * h->slab_n[j] : nullptr;
            p.psi[i][j] = h->slabs[j] ? h->slabs[j] + (3 + i) * h->slab_n[j] : nullptr;
        }
    return p;
}

static RecTable make_rec(pact_handle h) {
    RecTable r{};
    r.L = h->L;
    r.corner = h->rec_corner;
    r.weight = h->rec_weight;
    r.ncorner = h->ncorner;
    r.inj_point = h->inj_point;
    r.inj_off = h->inj_off;
    r.inj_rec = h->inj_rec;
    r.inj_w = h->inj_w;
    return r;
}

static void free_rec(pact_handle h) {
    cudaFree(h->rec_corner);
    cudaFree(h->rec_weight);
    cudaFree(h->inj_point);
    cudaFree(h->inj_off);
    cudaFree(h->inj_rec);
    cudaFree(h->inj_w);
    h->rec_corner = nullptr;
    h->rec_weight = nullptr;
    h->inj_point = h->inj_off = h->inj_rec = nullptr;
    h->inj_w = nullptr;
    h->rec_cap = 0;
}

// sigma^22, sigma^33 (adjoint: Q^22, Q^33) of the ITEM_DEEP items hold
// stale values during a solve (only sigma^11 is written there); copy
// sigma^11 into them before anything reads the three (image read-out,
// wavefield copy)
static void ac_fill(pact_handle h, cudaStream_t st) {
    if (!h->mixed || h->mixed_plan.deep_points == 0) return;
    const MixedPlan& mp = h->mixed_plan;
    const StepParams p = make_params(h);
    for (int l : {(int)MX_INT_AC, (int)MX_INT_FZ, (int)MX_EDGE_FL, (int)MX_CORNER_FL})
        launch_deep_fill(p, mp.list[l], mp.blocks[l], st);
}

// Validate the HOST receiver array and (re)build the device tables when it changed.
static int set_receivers(pact_handle h, const float* rec, int L) {
    if (!rec || L < 1) return fail(h, PACT_EINVAL, "receivers: rec_xyz must be non-NULL and L >= 1");
    const pact_grid_desc& d = h->d;
    const int lim[3] = {d.nx - 2, d.ny - 2, d.nz - 2};
    for (int l = 0; l < L; ++l)
        for (int a = 0; a < 3; ++a) {
            const float v = rec[3 * l + a];
            if (!std::isfinite(v) || v < 0.0f || v > (float)lim[a]) {
                char buf[160];
                snprintf(buf, sizeof buf, "receiver %d coordinate %d = %g outside [0, %d]", l, a, (double)v, lim[a]);
                return fail(h, PACT_EINVAL, buf);
            }
        }
    if (L == h->L && !h->rec_host.empty() && h->rec_medium_gen == h->medium_gen &&
        std::memcmp(h->rec_host.data(), rec, sizeof(float) * 3 * L) == 0)
        return PACT_OK;
    // host tables
    std::vector<int> corner(8 * (size_t)L);
    std::vector<float> weight(8 * (size_t)L);
    struct Contrib {
        int point, rec;
        float w;
    };
    std::vector<Contrib> con(8 * (size_t)L);
    for (int l = 0; l < L; ++l) {
        const double x = rec[3 * l], y = rec[3 * l + 1], z = rec[3 * l + 2];
        const int i0 = std::min((int)std::floor(x), d.nx - 2);
        const int j0 = std::min((int)std::floor(y), d.ny - 2);
        const int k0 = std::min((int)std::floor(z), d.nz - 2);
        const double fx = x - i0, fy = y - j0, fz = z - k0;
        int c = 0;
        for (int cz = 0; cz < 2; ++cz)
            for (int cy = 0; cy < 2; ++cy)
                for (int cx = 0; cx < 2; ++cx, ++c) {
                    const double w = (cx ? fx : 1 - fx) * (cy ? fy : 1 - fy) * (cz ? fz : 1 - fz);
                    const int q = ((k0 + cz) * d.ny + (j0 + cy)) * d.nx + (i0 + cx);
                    // a corner in an ITEM_DEEP item is stored as ~q: the
                    // sampler reads 3 sigma^11 there (sigma^22, sigma^33 stale)
                    const bool deep = h->mixed && plan_deep(h->mixed_plan, i0 + cx, j0 + cy, k0 + cz);
                    corner[8 * l + c] = deep ? ~q : q;
                    weight[8 * l + c] = (float)w;
                    con[8 * l + c] = {q, l, (float)w};
                }
    }
    std::stable_sort(con.begin(), con.end(), [](const Contrib& a, const Contrib& b) { return a.point < b.point; });
    std::vector<int> ipoint, ioff, irec(con.size());
    std::vector<float> iw(con.size());
    for (size_t e = 0; e < con.size(); ++e) {
        if (e == 0 || con[e].point != con[e - 1].point) {
            ipoint.push_back(con[e].point);
            ioff.push_back((int)e);
        }
        irec[e] = con[e].rec;
        iw[e] = con[e].w;
    }
    ioff.push_back((int)con.size());
    // device tables (grow only; wait for queued work before freeing)
    if (L > h->rec_cap) {
        CK(h, cudaStreamSynchronize(h->stream));
        free_rec(h);
        const size_t E = 8 * (size_t)L;
        CK(h, cudaMalloc(&h->rec_corner, E * sizeof(int)));
        CK(h, cudaMalloc(&h->rec_weight, E * sizeof(float)));
        CK(h, cudaMalloc(&h->inj_point, E * sizeof(int)));
        CK(h, cudaMalloc(&h->inj_off, (E + 1) * sizeof(int)));
        CK(h, cudaMalloc(&h->inj_rec, E * sizeof(int)));
        CK(h, cudaMalloc(&h->inj_w, E * sizeof(float)));
        h->rec_cap = L;
    }
    cudaStream_t s = h->stream;
    CK(h, cudaMemcpyAsync(h->rec_corner, corner.data(), corner.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(h, cudaMemcpyAsync(h->rec_weight, weight.data(), weight.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(h, cudaMemcpyAsync(h->inj_point, ipoint.data(), ipoint.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(h, cudaMemcpyAsync(h->inj_off, ioff.data(), ioff.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(h, cudaMemcpyAsync(h->inj_rec, irec.data(), irec.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(h, cudaMemcpyAsync(h->inj_w, iw.data(), iw.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    // pageable sources: the copies are staged before return, but keep the order
    // explicit by waiting here (receivers change rarely)
    CK(h, cudaStreamSynchronize(s));
    h->ncorner = (int)ipoint.size();
    h->L = L;
    h->rec_host.assign(rec, rec + 3 * (size_t)L);
    h->rec_medium_gen = h->medium_gen;
    return PACT_OK;
}

static int zero_state(pact_handle h) {
    CK(h, cudaMemsetAsync(h->fields, 0, 9 * h->N * sizeof(float), h->stream));
    for (int a = 0; a < 3; ++a)
        if (h->slabs[a]) CK(h, cudaMemsetAsync(h->slabs[a], 0, 6 * h->slab_n[a] * sizeof(float), h->stream));
    return PACT_OK;
}

static int precheck(pact_handle h, const void* a, const void* b, int nsteps) {
    if (!h) return fail(nullptr, PACT_EINVAL, "handle is NULL");
    if (!h->medium_set) return fail(h, PACT_ESTATE, "pact_set_medium must be called first");
    if (!a || !b) return fail(h, PACT_EINVAL, "NULL data pointer");
    if (nsteps < 0) return fail(h, PACT_EINVAL, "nsteps < 0");
    CK(h, cudaSetDevice(h->device));
    return PACT_OK;
}

// a tiled kernel records a timed-out wait in scratch_u32[3]; read at sync points
static int device_status(pact_handle h) {
    unsigned int w = 0;
    CK(h, cudaMemcpyAsync(&w, h->scratch_u32 + 3, sizeof w, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (w) return fail(h, PACT_ETIMEOUT, "a step kernel gave up waiting for its TMA loads");
    return PACT_OK;
}

// One step of H (fwd) or of H^T: the velocity-family and stress-family
// launches, with the single-pass interior launch between them when the
// handle runs on two buffers (the step then reads buffer c and writes 1-c).
static int step_mode(pact_handle h) {
    return h->fused ? STEP_FUSED : (h->acoustic ? STEP_ACOUSTIC : (h->mixed ? STEP_MIXED : STEP_TWO_PASS));
}

static void tiled_step(pact_handle h, const StepParams& p, int c, bool adj, cudaStream_t st) {
    int* err = reinterpret_cast<int*>(h->scratch_u32 + 3);
    const bool fz = h->fused;
    const int mode = step_mode(h);
    const TmaSet& tm = fz ? h->tmp[c] : h->tm;
    const SplitStreams ss{st,          fz ? nullptr : h->aux, h->ev_fork, h->ev_join, fz ? nullptr : h->aux2,
                          h->ev_join2, h->list_streams ? h->xs : nullptr, h->xj};
    const MixedPlan* mp = h->mixed ? &h->mixed_plan : nullptr;
    mark(h, adj ? PACT_K_ADJ_A : PACT_K_FWD_VELOCITY, launch_vel_tiled(adj, p, tm, err, ss, mode, mp));
    if (h->acoustic)
        mark(h, adj ? PACT_K_ADJ_AC_A : PACT_K_FWD_AC_VEL, launch_acoustic_step(false, adj, p, tm, err, st));
    if (fz) mark(h, adj ? PACT_K_ADJ_FUSED : PACT_K_FWD_FUSED, launch_fused_step(adj, p, h->fmp[c], err, st));
    mark(h, adj ? PACT_K_ADJ_B : PACT_K_FWD_STRESS, launch_str_tiled(adj, p, tm, err, ss, mode, mp));
    if (h->acoustic)
        mark(h, adj ? PACT_K_ADJ_AC_B : PACT_K_FWD_AC_STR, launch_acoustic_step(true, adj, p, tm, err, st));
}

static void fwd_step(pact_handle h, const StepParams& p, int c) {
    if (h->tiled) {
        tiled_step(h, p, c, false, h->stream);
    } else {
        launch_fwd_velocity(p, h->stream);
        mark(h, PACT_K_FWD_VELOCITY);
        launch_fwd_stress(p, h->stream);
        mark(h, PACT_K_FWD_STRESS);
    }
}

static void adj_step(pact_handle h, const StepParams& p, int c) {
    if (h->tiled) {
        tiled_step(h, p, c, true, h->stream);
    } else {
        launch_adj_a(p, h->stream);
        mark(h, PACT_K_ADJ_A);
        launch_adj_b(p, h->stream);
        mark(h, PACT_K_ADJ_B);
    }
}

// The second wavefield buffer and the maps of both step parities, made at
// the first solve of a handle that runs the single-pass kernel.
static int ensure_pingpong(pact_handle h) {
    if (!h->fused || h->fields2) return PACT_OK;
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMalloc(&h->fields2, 9 * h->N * sizeof(float)));
    for (int c = 0; c < 2; ++c) {
        float* fi = buffer(h, c);
        float* fo = buffer(h, 1 - c);
        float* arrays[TM_N];
        for (int i = 0; i < 3; ++i) arrays[TM_U0 + i] = fo + i * h->N;
        for (int v = 0; v < 6; ++v) arrays[TM_S0 + v] = fi + (3 + v) * h->N;
        arrays[TM_RHO] = h->medium;
        arrays[TM_LAM] = h->medium + h->N;
        arrays[TM_MU] = h->medium + 4 * h->N;
        arrays[TM_ALPHA] = h->medium + 3 * h->N;
        float* farr[FM_N];
        for (int v = 0; v < 6; ++v) farr[v] = fi + (3 + v) * h->N;
        farr[6] = h->medium;
        farr[7] = h->medium + 3 * h->N;
        if (make_tma_set(&h->tmp[c], arrays, h->d.nx, h->d.ny, h->d.nz) != 0 ||
            make_fused_maps(&h->fmp[c], farr, h->d.nx, h->d.ny, h->d.nz) != 0) {
            cudaFree(h->fields2);
            h->fields2 = nullptr;
            return fail(h, PACT_ECUDA, "encoding the tensor maps of the second wavefield buffer failed");
        }
    }
    return PACT_OK;
}

// 64-bit counter of nonzero p0 entries near the faces, in scratch words 6..7 (8-byte aligned)
static unsigned long long* band_counter(pact_handle h) {
    return reinterpret_cast<unsigned long long*>(h->scratch_u32 + 6);
}

// ---- CUDA graphs of whole steps ---------------------------------------------
constexpr int kGraphSteps = 16;
// pact_advance steps grids of at least this many points on their own step
// graphs, the rest on the multi-instance kernels.  On B300 the step graphs
// ran every size measured (96^3 .. 320^3) at least as fast, and 40 requests
// advanced together at 40.2 G updates/s against 37.7 with 8 M points here
// and 31.8 with every solve on the multi-instance kernels: all solves take
// their own graphs (PACT_SERVE_SOLO_POINTS overrides the size).
constexpr long long kSoloPoints = 0;

static void drop_graphs(pact_handle h) {
    for (auto& dir : h->graphs)
        for (auto& g : dir) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g = pact_grid::StepGraph{};
        }
    h->graph_warm[0] = h->graph_warm[1] = false;
    h->graph_off = false;
}

static bool graphs_apply(pact_handle h) {
    const char* genv = getenv("PACT_GRAPHS");
    return h->tiled && !h->fused && !h->prof && h->cap && !(genv && std::strcmp(genv, "0") == 0);
}

// one step of the solve in h->solve_dev on stream st: the step kernels, then
// the receiver kernel that reads the step count from the device
static void state_step(pact_handle h, bool adj, cudaStream_t st) {
    const StepParams p = make_params(h, 0);
    tiled_step(h, p, 0, adj, st);
    if (!adj) {
        launch_sample_state(p, h->solve_dev, st);
        mark(h, PACT_K_SAMPLE);
    } else {
        launch_inject_state(p, h->solve_dev, st);
        mark(h, PACT_K_INJECT);
    }
}

// Capture (once) the graph of `steps` steps (1 or kGraphSteps); a capture
// that fails turns the graphs of this handle off (graph_off).
static void ensure_step_graph(pact_handle h, bool adj, int steps) {
    pact_grid::StepGraph& g = h->graphs[adj ? 1 : 0][steps == 1 ? 0 : 1];
    if (!g.exec && !h->graph_off) {
        // the capture only records launches: keep the launch counts of one
        // replay, and count them at each launch below
        long long l0[PACT_NKIND];
        std::memcpy(l0, h->launches, sizeof l0);
        const long long k0 = h->kernels;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            for (int k = 0; k < steps; ++k) state_step(h, adj, h->cap);
            e = cudaStreamEndCapture(h->cap, &graph);
        }
        for (int k = 0; k < PACT_NKIND; ++k) {
            g.launches[k] = h->launches[k] - l0[k];
            h->launches[k] = l0[k];
        }
        g.kernels = h->kernels - k0;
        h->kernels = k0;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            // not capturable here: this handle launches its steps directly
            g.exec = nullptr;
            cudaGetLastError();
            h->graph_off = true;
        }
    }
}

// Launch on st the graph of `steps` steps (captured first if need be).
static int launch_step_graph(pact_handle h, bool adj, int steps, cudaStream_t st) {
    ensure_step_graph(h, adj, steps);
    if (h->graph_off) return PACT_OK;
    const pact_grid::StepGraph& g = h->graphs[adj ? 1 : 0][steps == 1 ? 0 : 1];
    CK(h, cudaGraphLaunch(g.exec, st));
    for (int k = 0; k < PACT_NKIND; ++k) h->launches[k] += g.launches[k];
    h->kernels += g.kernels;
    return PACT_OK;
}

// Steps 1..nsteps of the solve set up in h->solve_dev: the first solve of a
// handle and direction runs its first step directly, later steps replay the
// graphs (kGraphSteps at a time, the rest one at a time).
static int graph_steps(pact_handle h, bool adj, int nsteps, cudaStream_t st) {
    int m = 0;
    if (nsteps > 0 && !h->graph_warm[adj ? 1 : 0]) {
        state_step(h, adj, st);
        CK(h, cudaGetLastError());
        h->graph_warm[adj ? 1 : 0] = true;
        m = 1;
        // both graphs now, whatever this solve's length: a capture only
        // records launches, and later solves then start on graphs at once
        if (graphs_apply(h)) {
            ensure_step_graph(h, adj, 1);
            ensure_step_graph(h, adj, kGraphSteps);
        }
    }
    int rc = PACT_OK;
    while (rc == PACT_OK && m < nsteps && !h->graph_off && graphs_apply(h)) {
        const int k = nsteps - m >= kGraphSteps ? kGraphSteps : 1;
        rc = launch_step_graph(h, adj, k, st);
        if (!h->graph_off) m += k;
    }
    for (; rc == PACT_OK && m < nsteps; ++m) state_step(h, adj, st);
    if (rc == PACT_OK) CK(h, cudaGetLastError());
    return rc;
}

static int run_forward(pact_handle h, const float* p0, float* traces, int nsteps) {
    int rc = ensure_pingpong(h);
    if (rc) return rc;
    h->cur = 0;
    rc = zero_state(h);
    if (rc) return rc;
    const RecTable r = make_rec(h);
    StepParams p = make_params(h, 0);
    mark(h, -1);
    CK(h, cudaMemsetAsync(h->scratch_u32 + 6, 0, sizeof(unsigned long long), h->stream));
    launch_source(p0, p, h->stream, band_counter(h));
    mark(h, PACT_K_SOURCE);
    launch_sample(p, r, traces, h->stream);
    mark(h, PACT_K_SAMPLE);
    if (graphs_apply(h)) {
        const SolveState v{0, 0u, nsteps, r, traces, nullptr};
        launch_set_state(h->solve_dev, v, h->stream);
        rc = graph_steps(h, false, nsteps, h->stream);
        if (rc) return rc;
        h->cur = 0;
        CK(h, cudaGetLastError());
        return PACT_OK;
    }
    int c = 0;
    for (int m = 1; m <= nsteps; ++m) {
        const int out = h->fused ? 1 - c : -1;
        fwd_step(h, make_params(h, c, out), c);
        if (out >= 0) c = out;
        p = make_params(h, c);
        launch_sample(p, r, traces + (size_t)m * h->L, h->stream);
        mark(h, PACT_K_SAMPLE);
    }
    h->cur = c;
    CK(h, cudaGetLastError());
    return PACT_OK;
}

static int run_adjoint(pact_handle h, const float* traces, float* image, int nsteps) {
    int rc = ensure_pingpong(h);
    if (rc) return rc;
    h->cur = 0;
    rc = zero_state(h);
    if (rc) return rc;
    const RecTable r = make_rec(h);
    StepParams p = make_params(h, 0);
    mark(h, -1);
    launch_inject(p, r, traces + (size_t)nsteps * h->L, h->stream);
    mark(h, PACT_K_INJECT, r.ncorner > 0);
    if (graphs_apply(h)) {
        const SolveState v{0, 0u, nsteps, r, nullptr, traces};
        launch_set_state(h->solve_dev, v, h->stream);
        rc = graph_steps(h, true, nsteps, h->stream);
        if (rc) return rc;
        ac_fill(h, h->stream);
        launch_readout(image, p, h->stream);
        mark(h, PACT_K_READOUT);
        h->cur = 0;
        CK(h, cudaGetLastError());
        return PACT_OK;
    }
    int c = 0;
    for (int m = nsteps; m >= 1; --m) {
        const int out = h->fused ? 1 - c : -1;
        adj_step(h, make_params(h, c, out), c);
        if (out >= 0) c = out;
        p = make_params(h, c);
        launch_inject(p, r, traces + (size_t)(m - 1) * h->L, h->stream);
        mark(h, PACT_K_INJECT, r.ncorner > 0);
    }
    ac_fill(h, h->stream);
    launch_readout(image, p, h->stream);
    mark(h, PACT_K_READOUT);
    h->cur = c;
    CK(h, cudaGetLastError());
    return PACT_OK;
}

static int ensure_stage(pact_handle h, float** buf, size_t* cap, size_t n) {
    if (*cap >= n) return PACT_OK;
    CK(h, cudaStreamSynchronize(h->stream));
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    CK(h, cudaMalloc(buf, n * sizeof(float)));
    *cap = n;
    return PACT_OK;
}

extern "C" {

// A handle for grid desc, which is planes [z0g, z0g + desc->nz) of a grid of
// nzg planes (z0g = 0, nzg = desc->nz for a whole grid); desc is checked by
// the caller.
static int create_handle(const pact_grid_desc* desc, int z0g, int nzg, void* stream, pact_handle* out) {
    *out = nullptr;
    pact_grid* h = new (std::nothrow) pact_grid();
    if (!h) return fail(nullptr, PACT_ENOMEM, "host allocation failed");
    h->d = *desc;
    h->z0g = z0g;
    h->nzg = nzg;
    h->stream = (cudaStream_t)stream;
    h->N = (size_t)desc->nx * desc->ny * desc->nz;
    h->nmax = std::max(desc->nx, std::max(desc->ny, desc->nz));
    auto bail = [&](int code) {
        g_err = h->err;
        pact_destroy(h);
        return code;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        h->err = "cudaGetDevice failed";
        return bail(PACT_ECUDA);
    }
    cudaError_t e = cudaMalloc(&h->fields, 9 * h->N * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->medium, 5 * h->N * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->tables, 18 * (size_t)h->nmax * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&h->scratch_u32, 8 * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&h->solve_dev, sizeof(SolveState));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
    for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
        h->slab_n[a] = slab_points(*desc, a);
        if (h->slab_n[a]) e = cudaMalloc(&h->slabs[a], 6 * h->slab_n[a] * sizeof(float));
    }
    if (e != cudaSuccess) {
        h->err = std::string("allocation: ") + cudaGetErrorString(e);
        return bail(e == cudaErrorMemoryAllocation ? PACT_ENOMEM : PACT_ECUDA);
    }
    if (cudaMemset(h->scratch_u32, 0, 8 * sizeof(unsigned int)) != cudaSuccess) {
        h->err = "cudaMemset of the status words failed";
        return bail(PACT_ECUDA);
    }
    // TMA-staged kernels need 16-byte row strides (nx % 4 == 0); PACT_KERNELS=direct
    // in the environment selects the one-thread-per-point kernels instead.
    const char* kenv = getenv("PACT_KERNELS");
    if (desc->nx % 4 == 0 && !(kenv && std::strcmp(kenv, "direct") == 0)) {
        float* arrays[TM_N];
        for (int i = 0; i < 9; ++i) arrays[i] = h->fields + i * h->N;
        arrays[TM_RHO] = h->medium;
        arrays[TM_LAM] = h->medium + h->N;
        arrays[TM_MU] = h->medium + 4 * h->N;  // the TMA-staged kernels read 1/mu
        arrays[TM_ALPHA] = h->medium + 3 * h->N;
        h->tiled = make_tma_set(&h->tm, arrays, desc->nx, desc->ny, desc->nz) == 0;
        // PACT_FUSED=1 runs the interior tiles on the single-pass kernel (two
        // wavefield buffers); by default every tile runs the in-place
        // two-pass kernels, which measured faster on B300
        const char* fenv = getenv("PACT_FUSED");
        if (h->tiled && fenv && std::strcmp(fenv, "1") == 0) {
            StepParams q{};
            q.nx = desc->nx;
            q.ny = desc->ny;
            q.nz = desc->nz;
            q.P = desc->npml;
            q.z0g = z0g;
            q.nzg = nzg;
            RegionList rl;
            int blocks = 0;
            h->fused = fused_plan(q, rl, blocks);
            // every grid point must be updated by exactly one launch of each
            // half: the regions are disjoint by construction, so their point
            // counts must add up to N
            if (h->fused) {
                const long long nf = role_points(2, STEP_FUSED, q);
                h->fused = role_points(0, STEP_FUSED, q) + nf == (long long)h->N &&
                           role_points(1, STEP_FUSED, q) + nf == (long long)h->N;
            }
        }
        // PACT_OVERLAP=0 runs the frame and interior launches one after the other
        const char* oenv = getenv("PACT_OVERLAP");
        if (h->tiled && !(oenv && std::strcmp(oenv, "0") == 0)) {
            if (cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamCreateWithFlags(&h->aux2, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->ev_join2, cudaEventDisableTiming) != cudaSuccess) {
                h->err = "creating the frame stream and its events failed";
                return bail(PACT_ECUDA);
            }
            const char* lenv = getenv("PACT_LISTSTREAMS");
            if (!(lenv && std::strcmp(lenv, "0") == 0)) {
                for (int k = 0; k < 4; ++k)
                    if (cudaStreamCreateWithFlags(&h->xs[k], cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&h->xj[k], cudaEventDisableTiming) != cudaSuccess) {
                        h->err = "creating the work-list streams failed";
                        return bail(PACT_ECUDA);
                    }
                h->list_streams = true;
            }
        }
    }
    *out = h;
    return PACT_OK;
}

int pact_create_grid(const pact_grid_desc* desc, void* stream, pact_handle* out) {
    std::string why;
    if (!out) return fail(nullptr, PACT_EINVAL, "out is NULL");
    *out = nullptr;
    const int rc = check_desc(desc, why);
    if (rc) return fail(nullptr, rc, why);
    return create_handle(desc, 0, desc->nz, stream, out);
}

int pact_create_slab(const pact_grid_desc* global, int z_lo, int z_hi, void* stream, pact_handle* out) {
    std::string why;
    if (!out) return fail(nullptr, PACT_EINVAL, "out is NULL");
    *out = nullptr;
    const int rc = check_desc(global, why);
    if (rc) return fail(nullptr, rc, why);
    if (z_lo < 0 || z_hi > global->nz || z_hi - z_lo < 5)
        return fail(nullptr, PACT_EINVAL, "pact_create_slab: need 0 <= z_lo, z_hi <= nz and z_hi - z_lo >= 5");
    pact_grid_desc d = *global;
    d.nz = z_hi - z_lo;
    return create_handle(&d, z_lo, global->nz, stream, out);
}

int pact_set_medium(pact_handle h, const float* rho, const float* lambda, const float* mu, const float* alpha) {
    if (!h) return fail(nullptr, PACT_EINVAL, "handle is NULL");
    if (!rho || !lambda || !mu || !alpha) return fail(h, PACT_EINVAL, "NULL medium pointer");
    CK(h, cudaSetDevice(h->device));
    const size_t N = h->N;
    cudaStream_t s = h->stream;
    CK(h, cudaStreamSynchronize(s));
    drop_graphs(h);
    CK(h, cudaMemcpyAsync(h->medium, rho, N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync(h->medium + N, lambda, N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync(h->medium + 2 * N, mu, N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync(h->medium + 3 * N, alpha, N * sizeof(float), cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemsetAsync(h->scratch_u32, 0, 8 * sizeof(unsigned int), s));
    launch_medium_check(h->medium, h->medium + N, h->medium + 2 * N, h->medium + 3 * N, N, h->scratch_u32, s);
    launch_any_shear(h->medium + 2 * N, N, h->scratch_u32 + 4, s);
    launch_inv_mu(h->medium + 2 * N, h->medium + 4 * N, N, s);
    CK(h, cudaGetLastError());
    unsigned int red[8];
    CK(h, cudaMemcpyAsync(red, h->scratch_u32, sizeof red, cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    h->medium_set = false;
    if (red[2] != 0) {
        char buf[192];
        snprintf(buf, sizeof buf,
                 "medium: %u nodes violate rho > 0, mu >= 0, lambda + 2 mu > 0, 3 lambda + 2 mu > 0, alpha >= 0",
                 red[2]);
        return fail(h, PACT_EINVAL, buf);
    }
    float c2, amax;
    std::memcpy(&c2, &red[0], 4);
    std::memcpy(&amax, &red[1], 4);
    const double cmax = std::sqrt((double)c2);
    const double courant = cmax * h->d.dt / h->d.dx;
    const double limit = 6.0 / (7.0 * std::sqrt(3.0));
    if (!(courant < limit)) {
        char buf[200];
        snprintf(buf, sizeof buf, "CFL: c_max dt / dx = %.4f >= 6/(7 sqrt 3) = %.4f (c_max = %.1f m/s)", courant,
                 limit, cmax);
        return fail(h, PACT_ECFL, buf);
    }
    if (!((double)amax * h->d.dt < 1.0)) return fail(h, PACT_ECFL, "absorption: alpha_max dt >= 1");
    h->cmax = cmax;
    // C-PML profile tables, double precision on the host, stored as float
    const pact_grid_desc& d = h->d;
    const double vmax = d.pml_vmax > 0 ? d.pml_vmax : cmax;
    std::vector<float> tab(18 * (size_t)h->nmax, 0.0f);
    // the z profile of a slab handle is the whole grid's at the slab's planes
    const int dims[3] = {d.nx, d.ny, d.nz};
    const int gdim[3] = {d.nx, d.ny, h->nzg}, goff[3] = {0, 0, h->z0g};
    for (int a = 0; a < 3; ++a)
        for (int l = 0; l < 2; ++l)
            for (int k = 0; k < dims[a]; ++k) {
                double ca, cb, cc;
                pml_coef(gdim[a], d.npml, d.dx, d.dt, vmax, d.pml_R0, d.pml_f0, goff[a] + k + 0.5 * l, ca, cb, cc);
                tab[((a * 2 + l) * 3 + 0) * (size_t)h->nmax + k] = (float)ca;
                tab[((a * 2 + l) * 3 + 1) * (size_t)h->nmax + k] = (float)cb;
                tab[((a * 2 + l) * 3 + 2) * (size_t)h->nmax + k] = (float)cc;
            }
    CK(h, cudaMemcpyAsync(h->tables, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(h, cudaStreamSynchronize(s));
    // mu = 0 everywhere (the acoustic operator pair of the paper's ablation):
    // the interior runs the acoustic kernels unless PACT_ACOUSTIC=0
    const char* aenv = getenv("PACT_ACOUSTIC");
    const bool ac_ok = h->tiled && !h->fused && !(aenv && std::strcmp(aenv, "0") == 0);
    // The medium-adaptive plan: the work items whose reach is all fluid run
    // the acoustic and fluid C-PML kernels (the same operator there), the rest
    // the elastic ones; with mu = 0 everywhere every item is fluid.
    // PACT_ACOUSTIC=0 keeps the elastic kernels everywhere.  Without a plan
    // (no C-PML layer, or no interior tile) a medium with mu = 0 everywhere
    // runs the no-layer region on the acoustic kernels when it can.
    h->mixed = false;
    h->acoustic = false;
    if (ac_ok) {
        if (build_mixed_plan(make_params(h), h->medium + 2 * h->N, h->medium + 3 * h->N, s, &h->mixed_plan) != 0)
            return fail(h, PACT_ECUDA, "building the fluid / solid work lists of the medium failed");
        const long long* np = h->mixed_plan.points;
        h->mixed = np[MX_INT_AC] + np[MX_INT_FZ] + np[MX_EDGE_FL] + np[MX_CORNER_FL] > 0;
    }
    if (!h->mixed)
        h->acoustic = ac_ok && red[4] == 0 && role_points(3, STEP_ACOUSTIC, make_params(h)) > 0;  // needs a layer (see plan_for)
    h->medium_gen++;
    h->medium_set = true;
    return PACT_OK;
}

int pact_forward(pact_handle h, const float* p0, const float* rec_xyz, int L, int nsteps, float* traces) {
    int rc = precheck(h, p0, traces, nsteps);
    if (rc) return rc;
    rc = set_receivers(h, rec_xyz, L);
    if (rc) return rc;
    return run_forward(h, p0, traces, nsteps);
}

int pact_adjoint(pact_handle h, const float* traces, const float* rec_xyz, int L, int nsteps, float* image) {
    int rc = precheck(h, traces, image, nsteps);
    if (rc) return rc;
    rc = set_receivers(h, rec_xyz, L);
    if (rc) return rc;
    return run_adjoint(h, traces, image, nsteps);
}

int pact_forward_host(pact_handle h, const float* p0, const float* rec_xyz, int L, int nsteps, float* traces) {
    int rc = precheck(h, p0, traces, nsteps);
    if (rc) return rc;
    rc = set_receivers(h, rec_xyz, L);
    if (rc) return rc;
    const size_t nt = (size_t)(nsteps + 1) * L;
    if ((rc = ensure_stage(h, &h->stage_a, &h->stage_a_n, h->N))) return rc;
    if ((rc = ensure_stage(h, &h->stage_b, &h->stage_b_n, nt))) return rc;
    CK(h, cudaMemcpyAsync(h->stage_a, p0, h->N * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    if ((rc = run_forward(h, h->stage_a, h->stage_b, nsteps))) return rc;
    CK(h, cudaMemcpyAsync(traces, h->stage_b, nt * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    return device_status(h);
}

int pact_adjoint_host(pact_handle h, const float* traces, const float* rec_xyz, int L, int nsteps, float* image) {
    int rc = precheck(h, traces, image, nsteps);
    if (rc) return rc;
    rc = set_receivers(h, rec_xyz, L);
    if (rc) return rc;
    const size_t nt = (size_t)(nsteps + 1) * L;
    if ((rc = ensure_stage(h, &h->stage_a, &h->stage_a_n, h->N))) return rc;
    if ((rc = ensure_stage(h, &h->stage_b, &h->stage_b_n, nt))) return rc;
    CK(h, cudaMemcpyAsync(h->stage_b, traces, nt * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    if ((rc = run_adjoint(h, h->stage_b, h->stage_a, nsteps))) return rc;
    CK(h, cudaMemcpyAsync(image, h->stage_a, h->N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    return device_status(h);
}

int pact_destroy(pact_handle h) {
    if (!h) return PACT_OK;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    cudaFree(h->fields);
    free_mixed_plan(&h->mixed_plan);
    cudaFree(h->fields2);
    cudaFree(h->medium);
    cudaFree(h->tables);
    cudaFree(h->scratch_u32);
    drop_graphs(h);
    cudaFree(h->solve_dev);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->sv_stream) cudaStreamDestroy(h->sv_stream);
    if (h->sv_fork) cudaEventDestroy(h->sv_fork);
    if (h->sv_join) cudaEventDestroy(h->sv_join);
    for (int a = 0; a < 3; ++a) cudaFree(h->slabs[a]);
    free_rec(h);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_join2) cudaEventDestroy(h->ev_join2);
    if (h->aux) cudaStreamDestroy(h->aux);
    if (h->aux2) cudaStreamDestroy(h->aux2);
    for (int k = 0; k < 4; ++k) {
        if (h->xs[k]) cudaStreamDestroy(h->xs[k]);
        if (h->xj[k]) cudaEventDestroy(h->xj[k]);
    }
    cudaFree(h->stage_a);
    cudaFree(h->stage_b);
    delete h;
    return PACT_OK;
}

const char* pact_last_error(pact_handle h) { return h ? h->err.c_str() : g_err.c_str(); }

int pact_query_bytes(const pact_grid_desc* desc, int L, int nsteps, size_t* bytes) {
    std::string why;
    if (!bytes) return fail(nullptr, PACT_EINVAL, "bytes is NULL");
    int rc = check_desc(desc, why);
    if (rc) return fail(nullptr, rc, why);
    *bytes = desc_bytes(*desc, L, nsteps);
    return PACT_OK;
}

int pact_get_wavefield(pact_handle h, float* host_out) {
    if (!h) return fail(nullptr, PACT_EINVAL, "handle is NULL");
    if (!host_out) return fail(h, PACT_EINVAL, "host_out is NULL");
    CK(h, cudaSetDevice(h->device));
    ac_fill(h, h->stream);
    CK(h, cudaMemcpyAsync(host_out, buffer(h, h->cur), 9 * h->N * sizeof(float), cudaMemcpyDeviceToHost,
                          h->stream));
    return device_status(h);
}

int pact_profile(pact_handle h, int enable) {
    if (!h) return fail(nullptr, PACT_EINVAL, "handle is NULL");
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    for (int k = 0; k < PACT_NKIND; ++k) h->launches[k] = 0;
    h->kernels = 0;
    h->ev_kind.clear();
    h->prof = enable != 0;
    return PACT_OK;
}

int pact_profile_read(pact_handle h, int kind, long long* launches, double* total_ms) {
    if (!h) return fail(nullptr, PACT_EINVAL, "handle is NULL");
    if (kind < 0 || kind > PACT_K_ALL || !launches || !total_ms) return fail(h, PACT_EINVAL, "bad kind or NULL");
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    *launches = kind == PACT_K_ALL ? h->kernels : h->launches[kind];
    double ms = 0.0;
    for (size_t i = 1; i < h->ev_kind.size(); ++i) {
        if (kind == PACT_K_ALL ? h->ev_kind[i] < 0 : h->ev_kind[i] != kind) continue;
        float t = 0.0f;
        CK(h, cudaEventElapsedTime(&t, h->ev_pool[i - 1], h->ev_pool[i]));
        ms += t;
    }
    *total_ms = ms;
    return device_status(h);
}

int pact_role_points(pact_handle h, int kind, long long* points, long long* slab_points) {
    if (!h) return fail(nullptr, PACT_EINVAL, "handle is NULL");
    if (!points || !slab_points) return fail(h, PACT_EINVAL, "NULL output");
    const bool vel = kind == PACT_K_FWD_VELOCITY || kind == PACT_K_ADJ_A;
    const bool str = kind == PACT_K_FWD_STRESS || kind == PACT_K_ADJ_B;
    const bool fz = kind == PACT_K_FWD_FUSED || kind == PACT_K_ADJ_FUSED;
    const bool ac = kind == PACT_K_FWD_AC_VEL || kind == PACT_K_FWD_AC_STR || kind == PACT_K_ADJ_AC_A ||
                    kind == PACT_K_ADJ_AC_B;
    if (!vel && !str && !fz && !ac) return fail(h, PACT_EINVAL, "kind is not a step role");
    CK(h, cudaSetDevice(h->device));
    const StepParams p = make_params(h);
    long long slabs = 0;
    for (int a = 0; a < 3; ++a) slabs += (long long)h->slab_n[a];
    if (fz || ac) {
        // the single-pass and acoustic regions lie off the slabs
        *points = fz ? (h->fused ? role_points(2, STEP_FUSED, p) : 0)
                     : (h->acoustic ? role_points(3, STEP_ACOUSTIC, p)
                                    : (h->mixed ? h->mixed_plan.points[MX_INT_AC] : 0));
        *slab_points = 0;
    } else if (h->tiled) {
        *points = h->mixed ? (long long)h->N - h->mixed_plan.points[MX_INT_AC]
                           : role_points(vel ? 0 : 1, step_mode(h), p);
        *slab_points = slabs;
    } else {
        *points = (long long)h->N;
        *slab_points = slabs;
    }
    return PACT_OK;
}

int pact_begin(pact_handle h, int is_adjoint, const float* in, const float* rec_xyz, int L, int nsteps, float* out) {
    int rc;
    if (L == 0) {
        // no receiver (a z-slab owning none): no traces, so the trace pointer
        // may be NULL; p0 (forward) or the image (adjoint) is still required
        const void* field = is_adjoint ? (const void*)out : (const void*)in;
        rc = precheck(h, field, field, nsteps);
        if (rc) return rc;
        h->L = 0;
        h->ncorner = 0;
        h->rec_host.clear();
    } else {
        rc = precheck(h, in, out, nsteps);
        if (rc) return rc;
        rc = set_receivers(h, rec_xyz, L);
        if (rc) return rc;
    }
    if (!h->tiled) return fail(h, PACT_EINVAL, "serving uses the TMA-staged kernels: nx must be a multiple of 4");
    h->cur = 0;
    rc = zero_state(h);
    if (rc) return rc;
    const StepParams p = make_params(h);
    const RecTable r = make_rec(h);
    h->sv_adj = is_adjoint ? 1 : 0;
    h->sv_m = 0;
    h->sv_nsteps = nsteps;
    h->sv_in = in;
    h->sv_out = out;
    if (!is_adjoint) {
        CK(h, cudaMemsetAsync(h->scratch_u32 + 6, 0, sizeof(unsigned long long), h->stream));
        launch_source(in, p, h->stream, band_counter(h));
        launch_sample(p, r, out, h->stream);
    } else {
        if (L > 0) launch_inject(p, r, in + (size_t)nsteps * L, h->stream);
        if (nsteps == 0) {
            ac_fill(h, h->stream);
            launch_readout(out, p, h->stream);
        }
    }
    if (h->mixed) {
        // a medium-adaptive handle serves its per-medium work lists
        const MixedPlan& mp = h->mixed_plan;
        h->sv_inner = mp.list[MX_INT_EL];
        h->sv_ninner = mp.blocks[MX_INT_EL];
        h->sv_edge = mp.list[MX_EDGE_EL];
        h->sv_nedge = mp.blocks[MX_EDGE_EL];
        h->sv_corner = mp.list[MX_CORNER_EL];
        h->sv_ncorner = mp.blocks[MX_CORNER_EL];
        h->sv_ac = mp.list[MX_INT_AC];
        h->sv_nac = mp.blocks[MX_INT_AC];
        h->sv_fl = mp.fluid_frame;
        h->sv_nfl = mp.fluid_frame_blocks;
    } else {
        plan_instance_regions(p, 64, h->sv_inner, h->sv_ninner, h->sv_edge, h->sv_nedge, h->sv_corner,
                              h->sv_ncorner);
        h->sv_ac = RegionList{};
        h->sv_ac.n = 0;
        h->sv_fl = h->sv_ac;
        h->sv_nac = h->sv_nfl = 0;
    }
    // a solve of kSoloPoints points or more advances on its own step graphs
    // (its state then lives in solve_dev), a smaller one on the multi-instance
    // kernels.  PACT_SERVE_SOLO_POINTS overrides the size (a negative value
    // sends every solve to the multi-instance kernels).
    long long solo_points = kSoloPoints;
    if (const char* senv = getenv("PACT_SERVE_SOLO_POINTS")) solo_points = std::atoll(senv);
    h->sv_solo = h->tiled && !h->fused && solo_points >= 0 && (long long)h->N >= solo_points;
    if (h->sv_solo && !h->sv_stream) {
        CK(h, cudaStreamCreateWithFlags(&h->sv_stream, cudaStreamNonBlocking));
        CK(h, cudaEventCreateWithFlags(&h->sv_fork, cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->sv_join, cudaEventDisableTiming));
    }
    if (h->sv_solo) {
        const SolveState v{0, 0u, nsteps, r, is_adjoint ? nullptr : out, is_adjoint ? in : nullptr};
        launch_set_state(h->solve_dev, v, h->stream);
    }
    h->sv_active = nsteps > 0;
    CK(h, cudaGetLastError());
    return PACT_OK;
}

int pact_advance(pact_handle* hs, int n, int ksteps, void* stream) {
    if (!hs || n < 0 || n > kMaxInst) return fail(nullptr, PACT_EINVAL, "pact_advance: 0 <= n <= 64 handles");
    if (ksteps < 1) return fail(nullptr, PACT_EINVAL, "pact_advance: ksteps >= 1");
    static thread_local MultiTable* T = nullptr;
    if (!T) T = new (std::nothrow) MultiTable();
    if (!T) return fail(nullptr, PACT_ENOMEM, "host allocation failed");
    int dev = -1, ni = 0;
    T->pre_inner[0] = T->pre_edge[0] = T->pre_corner[0] = T->pre_ac[0] = T->pre_fl[0] = 0;
    // forward instances first, then adjoint ones (each persistent kernel
    // serves one direction)
    for (int pass = 0; pass < 2; ++pass) {
        for (int k = 0; k < n; ++k) {
            pact_handle h = hs[k];
            if (!h) return fail(nullptr, PACT_EINVAL, "pact_advance: NULL handle");
            if (!h->sv_active || h->sv_adj != pass) continue;
            if (dev < 0) dev = h->device;
            if (h->sv_solo) {
                if (h->device != dev) return fail(h, PACT_EINVAL, "pact_advance: handles on different devices");
                continue;
            }
            if (h->device != dev) return fail(h, PACT_EINVAL, "pact_advance: handles on different devices");
            InstDev& e = T->inst[ni];
            e.tm = h->tm;
            e.p = make_params(h);
            e.inner = h->sv_inner;
            e.edge = h->sv_edge;
            e.corner = h->sv_corner;
            e.ac = h->sv_ac;
            e.fl = h->sv_fl;
            e.rec = make_rec(h);
            e.src = h->sv_adj ? h->sv_in : nullptr;
            e.dst = h->sv_adj ? nullptr : h->sv_out;
            e.adj = h->sv_adj;
            e.m = h->sv_m;
            e.nsteps = h->sv_nsteps;
            e.L = h->L;
            T->pre_inner[ni + 1] = T->pre_inner[ni] + h->sv_ninner;
            T->pre_edge[ni + 1] = T->pre_edge[ni] + h->sv_nedge;
            T->pre_corner[ni + 1] = T->pre_corner[ni] + h->sv_ncorner;
            T->pre_ac[ni + 1] = T->pre_ac[ni] + h->sv_nac;
            T->pre_fl[ni + 1] = T->pre_fl[ni] + h->sv_nfl;
            ++ni;
        }
        if (pass == 0) T->n_fwd = ni;
    }
    T->n_inst = ni;
    if (dev < 0) return PACT_OK;
    if (cudaSetDevice(dev) != cudaSuccess) return fail(nullptr, PACT_ECUDA, "cudaSetDevice failed");
    std::string why;
    cudaStream_t st = (cudaStream_t)stream;
    if (ni > 0) {
        const int rc = serve_run(*T, ksteps, st, why);
        if (rc) return fail(nullptr, rc, why);
    }
    // solves on their own step graphs: each on its stream, forked from st and
    // joined back, so that they overlap one another and the table's kernels
    for (int k = 0; k < n; ++k) {
        pact_handle h = hs[k];
        if (!h->sv_active || !h->sv_solo) continue;
        CK(h, cudaEventRecord(h->sv_fork, st));
        CK(h, cudaStreamWaitEvent(h->sv_stream, h->sv_fork, 0));
        const int rc = graph_steps(h, h->sv_adj != 0, std::min(ksteps, h->sv_nsteps - h->sv_m), h->sv_stream);
        if (rc) return rc;
        CK(h, cudaEventRecord(h->sv_join, h->sv_stream));
        CK(h, cudaStreamWaitEvent(st, h->sv_join, 0));
    }
    for (int k = 0; k < n; ++k) {
        pact_handle h = hs[k];
        if (!h->sv_active) continue;
        h->sv_m = std::min(h->sv_nsteps, h->sv_m + ksteps);
        if (h->sv_m == h->sv_nsteps) {
            h->sv_active = false;
            if (h->sv_adj) {
                const StepParams p = make_params(h);
                ac_fill(h, st);
                launch_readout(h->sv_out, p, st);
            }
        }
    }
    if (cudaGetLastError() != cudaSuccess) return fail(nullptr, PACT_ECUDA, "pact_advance: launch failed");
    return PACT_OK;
}

// ---- stepping a prepared solve one half step at a time ----------------------
// (the z-slab decomposition exchanges halo planes between the halves)
int pact_step_half(pact_handle h, int stress) {
    if (!h) return fail(nullptr, PACT_EINVAL, "handle is NULL");
    if (!h->sv_active) return fail(h, PACT_ESTATE, "pact_step_half: no unfinished solve (pact_begin first)");
    if (h->fused) return fail(h, PACT_EINVAL, "pact_step_half: not with the single-pass kernel (PACT_FUSED)");
    CK(h, cudaSetDevice(h->device));
    const bool adj = h->sv_adj != 0, str = stress != 0;
    const StepParams p = make_params(h);
    int* err = reinterpret_cast<int*>(h->scratch_u32 + 3);
    const SplitStreams ss{h->stream,   h->aux, h->ev_fork, h->ev_join, h->aux2,
                          h->ev_join2, h->list_streams ? h->xs : nullptr, h->xj};
    const MixedPlan* mp = h->mixed ? &h->mixed_plan : nullptr;
    const int mode = step_mode(h);
    if (!str) {
        mark(h, adj ? PACT_K_ADJ_A : PACT_K_FWD_VELOCITY, launch_vel_tiled(adj, p, h->tm, err, ss, mode, mp));
        if (h->acoustic)
            mark(h, adj ? PACT_K_ADJ_AC_A : PACT_K_FWD_AC_VEL, launch_acoustic_step(false, adj, p, h->tm, err, h->stream));
    } else {
        mark(h, adj ? PACT_K_ADJ_B : PACT_K_FWD_STRESS, launch_str_tiled(adj, p, h->tm, err, ss, mode, mp));
        if (h->acoustic)
            mark(h, adj ? PACT_K_ADJ_AC_B : PACT_K_FWD_AC_STR, launch_acoustic_step(true, adj, p, h->tm, err, h->stream));
    }
    CK(h, cudaGetLastError());
    return PACT_OK;
}

int pact_step_receivers(pact_handle h) {
    if (!h) return fail(nullptr, PACT_EINVAL, "handle is NULL");
    if (!h->sv_active) return fail(h, PACT_ESTATE, "pact_step_receivers: no unfinished solve (pact_begin first)");
    CK(h, cudaSetDevice(h->device));
    const StepParams p = make_params(h);
    const RecTable r = make_rec(h);
    const int m = h->sv_m + 1;  // the step just completed
    if (h->L > 0) {
        if (!h->sv_adj) {
            launch_sample(p, r, h->sv_out + (size_t)m * h->L, h->stream);
            mark(h, PACT_K_SAMPLE);
        } else {
            launch_inject(p, r, h->sv_in + (size_t)(h->sv_nsteps - m) * h->L, h->stream);
            mark(h, PACT_K_INJECT, r.ncorner > 0);
        }
    }
    h->sv_m = m;
    if (m == h->sv_nsteps) {
        h->sv_active = false;
        if (h->sv_adj) {
            ac_fill(h, h->stream);
            launch_readout(h->sv_out, p, h->stream);
            mark(h, PACT_K_READOUT);
        }
    }
    CK(h, cudaGetLastError());
    return PACT_OK;
}

int pact_field_ptr(pact_handle h, int field, float** out) {
    if (!h || !out) return fail(h, PACT_EINVAL, "pact_field_ptr: NULL argument");
    if (field < 0 || field > 8) return fail(h, PACT_EINVAL, "pact_field_ptr: field must be 0..8");
    if (h->fused) return fail(h, PACT_EINVAL, "pact_field_ptr: not with the single-pass kernel (PACT_FUSED)");
    *out = h->fields + (size_t)field * h->N;
    return PACT_OK;
}

int pact_item_points(pact_handle h, int item_class, long long* points) {
    if (!h || !points) return fail(h, PACT_EINVAL, "pact_item_points: NULL argument");
    if (item_class != PACT_ITEM_DEEP && item_class != PACT_ITEM_NOALPHA)
        return fail(h, PACT_EINVAL, "pact_item_points: item_class must be PACT_ITEM_DEEP or PACT_ITEM_NOALPHA");
    *points = !h->mixed ? 0 : (item_class == PACT_ITEM_DEEP ? h->mixed_plan.deep_points : h->mixed_plan.noalpha_points);
    return PACT_OK;
}

int pact_support_warning(pact_handle h, long long* n_points) {
    if (!h || !n_points) return fail(h, PACT_EINVAL, "pact_support_warning: NULL argument");
    unsigned long long c = 0;
    CK(h, cudaMemcpyAsync(&c, band_counter(h), sizeof c, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    *n_points = (long long)c;
    return PACT_OK;
}

int pact_poll(pact_handle h, int* steps_done) {
    if (!h || !steps_done) return fail(h, PACT_EINVAL, "pact_poll: NULL argument");
    *steps_done = h->sv_m;
    return PACT_OK;
}

}  // extern "C"
