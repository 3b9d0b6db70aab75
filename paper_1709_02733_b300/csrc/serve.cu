// serve.cu -- persistent multi-instance stepping behind pact_advance.
//
// Many solves (forward or adjoint, each on its own grid) advance together:
// per time step, the persistent velocity-family kernels, the persistent
// stress-family kernels and one receiver kernel each walk a device table of
// instances.  k steps are captured once into a CUDA graph per device and k;
// the graph reads the table from a fixed device address, so a changed set of
// admitted solves only needs a new table copy, not a new graph.
#include <cuda_runtime.h>

#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "pact.h"
#include "pact_internal.cuh"
#include "step_tiled.cuh"

// After one step of every unfinished instance: forward instances sample
// row m+1 of their traces (Theta), adjoint instances inject row nsteps-(m+1)
// (Theta^T into the weighted normal stresses Q, owner-computes as in
// k_inject); then the step counter advances.
__global__ void k_multi_receivers(MultiTable* T) {
    const int i = blockIdx.x;
    if (i >= T->n_inst) return;
    InstDev& I = T->inst[i];
    const int m = I.m;
    if (m >= I.nsteps) return;
    const StepParams& p = I.p;
    const RecTable& r = I.rec;
    if (!I.adj) {
        float* out = I.dst + (size_t)(m + 1) * I.L;
        for (int l = threadIdx.x; l < I.L; l += blockDim.x) {
            float acc = 0.0f;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                // a corner stored as ~q lies in an ITEM_DEEP item (3 sigma^11)
                const int q = r.corner[8 * l + c];
                acc += r.weight[8 * l + c] * (q >= 0 ? p.s[0][q] + p.s[1][q] + p.s[2][q] : 3.0f * p.s[0][~q]);
            }
            out[l] = -acc;
        }
    } else {
        const float* ph = I.src + (size_t)(I.nsteps - (m + 1)) * I.L;
        for (int c = threadIdx.x; c < r.ncorner; c += blockDim.x) {
            float acc = 0.0f;
            for (int e = r.inj_off[c]; e < r.inj_off[c + 1]; ++e) acc += r.inj_w[e] * ph[r.inj_rec[e]];
            const int q = r.inj_point[c];
            acc *= 3.0f * p.lam[q] + 2.0f * p.mu[q];  // Q = C sigma~ (see step_direct.cu)
            p.s[0][q] -= acc;
            p.s[1][q] -= acc;
            p.s[2][q] -= acc;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) I.m = m + 1;
}

namespace {

struct Server {
    MultiTable* dT = nullptr;
    int* err = nullptr;
    unsigned int* host_err = nullptr;  // pinned copy of the status word
    cudaStream_t cap = nullptr;
    // the last replay queued on this device: an advance queued on another
    // stream waits for it, since every replay reads the one table at dT
    cudaEvent_t last = nullptr;
    bool have_last = false;
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        int* next = nullptr;  // work-item counters of the graph's launches
    };
    std::map<int, Graph> graphs;
};

std::mutex g_serve_mu;
Server g_srv[64];

}  // namespace

// Copy the table (header + n instances) and replay the k-step graph on st.
int serve_run(const MultiTable& T, int ksteps, cudaStream_t st, std::string& why) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        why = "serve: no current device";
        return PACT_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_serve_mu);
    Server& S = g_srv[dev];
#define SCK(call)                                                                \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            why = std::string(#call) + ": " + cudaGetErrorString(e_);            \
            return e_ == cudaErrorMemoryAllocation ? PACT_ENOMEM : PACT_ECUDA;   \
        }                                                                        \
    } while (0)
    if (!S.dT) {
        SCK(cudaMalloc(&S.dT, sizeof(MultiTable)));
        SCK(cudaMalloc(&S.err, sizeof(int)));
        SCK(cudaMemset(S.err, 0, sizeof(int)));
        SCK(cudaMallocHost(&S.host_err, sizeof(unsigned int)));
        *S.host_err = 0;
        SCK(cudaStreamCreateWithFlags(&S.cap, cudaStreamNonBlocking));
        SCK(cudaEventCreateWithFlags(&S.last, cudaEventDisableTiming));
    }
    if (*S.host_err) {
        why = *S.host_err == 2 ? "serve: a multi-instance work item fell outside its grid (skipped)"
                               : "serve: a multi-instance step kernel gave up waiting for its TMA loads";
        return *S.host_err == 2 ? PACT_EINVAL : PACT_ETIMEOUT;
    }
    auto it = S.graphs.find(ksteps);
    if (it == S.graphs.end()) {
        // one counter per persistent launch of the k steps, zeroed by the
        // graph's first node on every replay
        const size_t ncount = (size_t)ksteps * 2 * kMultiLaunches;
        Server::Graph G;
        SCK(cudaMalloc(&G.next, ncount * sizeof(int)));
        cudaGraph_t g = nullptr;
        SCK(cudaStreamBeginCapture(S.cap, cudaStreamCaptureModeRelaxed));
        cudaMemsetAsync(G.next, 0, ncount * sizeof(int), S.cap);
        for (int k = 0; k < ksteps; ++k) {
            launch_multi_step_half(false, S.dT, S.err, G.next + (2 * k) * kMultiLaunches, S.cap);
            launch_multi_step_half(true, S.dT, S.err, G.next + (2 * k + 1) * kMultiLaunches, S.cap);
            k_multi_receivers<<<kMaxInst, 256, 0, S.cap>>>(S.dT);
        }
        SCK(cudaStreamEndCapture(S.cap, &g));
        SCK(cudaGraphInstantiate(&G.exec, g, 0));
        cudaGraphDestroy(g);
        it = S.graphs.emplace(ksteps, G).first;
    }
    const size_t bytes = offsetof(MultiTable, inst) + (size_t)T.n_inst * sizeof(InstDev);
    // the table copy must not overtake a replay still reading the table
    if (S.have_last) SCK(cudaStreamWaitEvent(st, S.last, 0));
    SCK(cudaMemcpyAsync(S.dT, &T, bytes, cudaMemcpyHostToDevice, st));
    SCK(cudaGraphLaunch(it->second.exec, st));
    SCK(cudaEventRecord(S.last, st));
    S.have_last = true;
    SCK(cudaMemcpyAsync(S.host_err, S.err, sizeof(int), cudaMemcpyDeviceToHost, st));
#undef SCK
    return PACT_OK;
}
