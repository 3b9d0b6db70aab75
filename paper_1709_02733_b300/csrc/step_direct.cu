// step_direct.cu -- one-thread-per-grid-point step kernels of H and H^T.
//
// Forward step (Appendix A.3, the four sub-updates after Eq. (opPML)), split in
// two in-place kernels so that no thread reads a value another thread writes:
//   k_fwd_velocity : phi <- B phi + E sigma ; u <- J u + Phi sigma + Gamma phi
//   k_fwd_stress   : psi <- B~ psi + E~ u   ; sigma <- sigma + Psi u + Delta psi
// Adjoint step W'^T = S1^T S2^T S3^T S4^T (Sec. 4, Eq. (backwardstep); Appendix
// A.3, Eq. (AdjupPML)) in gather form.  With zero padding (D+)^T = -(D-) and
// (D-)^T = -(D+), so every transposed difference is a difference of the
// complementary kind.  The adjoint state is kept in weighted variables
//   w = dt u~ / rho_bar   (velocity nodes),   Q = C sigma~   (stress nodes),
//   psi^ = psi~ / dt,     phi~ as is,
// where C is the stiffness of the stress update (lambda, mu at the normal
// nodes, the harmonic mean of mu at the shear nodes).  In these variables the
// transposed step has the form of the forward step with negated differences,
// so no material-weighted field has to be formed at neighbouring points:
//   k_adj_a : phi~ <- b (phi~ + chi w)      (tail of the previous S2^T / S1^T, own point)
//             w    <- J w - dt^2/rho_bar D F,   F = Q + a (psi^ + chi Q)   [S4^T, S3^T]
//   k_adj_b : psi^ <- b (psi^ + chi Q)      (tail of S4^T / S3^T, own point, old Q)
//             Q    <- Q - C e(E),           E = w + a (phi~ + chi w)      [S2^T, S1^T]
// with D, e(.) the difference patterns of the forward velocity and stress
// updates and a, b, chi the C-PML tables (the a-terms vanish off the slabs).
// The J and b factors are applied one kernel later because the next kernel
// still reads w, Q and the memory variables at neighbouring points.
// Source and read-out in these variables: the injection Theta^T p adds
// -(3 lambda + 2 mu) p to each normal Q (it adds -p to each normal sigma~), and
// tau^T sigma~ = -tr(sigma~)/3 = -tr(Q) / (3 (3 lambda + 2 mu)), which needs a
// positive bulk modulus 3 lambda + 2 mu at every node (checked with the medium).
#include "pact_internal.cuh"

// ---------------------------------------------------------------------------
// differences of a field along axis A at (x,y,z) (Sec. 2.2, Eq. (derivative))
// ---------------------------------------------------------------------------
template <int A>
__device__ __forceinline__ float tapz(const float* f, int x, int y, int z, int o, const StepParams& p) {
    return ldz(f, x + (A == 0) * o, y + (A == 1) * o, z + (A == 2) * o, p);
}

// integer lattice -> half lattice
template <int A>
__device__ __forceinline__ float Dplus(const float* f, int x, int y, int z, const StepParams& p) {
    return (PACT_C1 * (tapz<A>(f, x, y, z, 1, p) - tapz<A>(f, x, y, z, 0, p)) -
            PACT_C2 * (tapz<A>(f, x, y, z, 2, p) - tapz<A>(f, x, y, z, -1, p))) * p.inv_dx;
}

// half lattice -> integer lattice
template <int A>
__device__ __forceinline__ float Dminus(const float* f, int x, int y, int z, const StepParams& p) {
    return (PACT_C1 * (tapz<A>(f, x, y, z, 0, p) - tapz<A>(f, x, y, z, -1, p)) -
            PACT_C2 * (tapz<A>(f, x, y, z, 1, p) - tapz<A>(f, x, y, z, -2, p))) * p.inv_dx;
}

// the same two differences of a computed field g(x,y,z) (zero outside the grid)
template <int A, class G>
__device__ __forceinline__ float DplusF(G g, int x, int y, int z, const StepParams& p) {
    auto t = [&](int o) { return g(x + (A == 0) * o, y + (A == 1) * o, z + (A == 2) * o); };
    return (PACT_C1 * (t(1) - t(0)) - PACT_C2 * (t(2) - t(-1))) * p.inv_dx;
}

template <int A, class G>
__device__ __forceinline__ float DminusF(G g, int x, int y, int z, const StepParams& p) {
    auto t = [&](int o) { return g(x + (A == 0) * o, y + (A == 1) * o, z + (A == 2) * o); };
    return (PACT_C1 * (t(0) - t(-1)) - PACT_C2 * (t(1) - t(-2))) * p.inv_dx;
}

__device__ __forceinline__ bool inside(int x, int y, int z, const StepParams& p) {
    return (unsigned)x < (unsigned)p.nx && (unsigned)y < (unsigned)p.ny && (unsigned)z < (unsigned)p.nz;
}

// ===========================================================================
// forward
// ===========================================================================

// d_J sigma^{IJ} at the u^I node
template <int I, int J>
__device__ __forceinline__ float dsig(int x, int y, int z, const StepParams& p) {
    const float* f = p.s[voigt(I, J)];
    return I == J ? Dplus<J>(f, x, y, z, p) : Dminus<J>(f, x, y, z, p);
}

// one term of the velocity update: d_J sigma^{IJ} + chi_J phi^{IJ}, updating phi^{IJ}
template <int I, int J>
__device__ __forceinline__ float vel_term(int x, int y, int z, const StepParams& p) {
    const float g = dsig<I, J>(x, y, z, p);
    const int k = coord<J>(x, y, z);
    const int l = axis_slab<J>(k, p);
    if (l < 0) return g;
    constexpr int h = (I == J);  // u^I is on the half lattice along I only
    const float a = ptab<J>(p, h, 0, k), b = ptab<J>(p, h, 1, k), chi = ptab<J>(p, h, 2, k);
    float* ph = p.phi[I][J] + slab_index(J, x, y, z, l, p);
    const float v = b * (*ph) + a * g;
    *ph = v;
    return g + chi * v;
}

template <int I>
__device__ __forceinline__ void vel_update(int x, int y, int z, size_t idx, const StepParams& p) {
    const float acc = vel_term<I, 0>(x, y, z, p) + vel_term<I, 1>(x, y, z, p) + vel_term<I, 2>(x, y, z, p);
    const float rb = med_avg<I>(p.rho, x, y, z, p);
    const float ab = med_avg<I>(p.alpha, x, y, z, p);
    float* u = p.u[I] + idx;
    *u = (1.0f - p.dt * ab) * (*u) + p.dt / rb * acc;
}

__global__ void k_fwd_velocity(StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const size_t idx = lin3(x, y, z, p.nx, p.ny);
    vel_update<0>(x, y, z, idx, p);
    vel_update<1>(x, y, z, idx, p);
    vel_update<2>(x, y, z, idx, p);
}

// d_J u^I at the sigma^{IJ} node
template <int I, int J>
__device__ __forceinline__ float dvel(int x, int y, int z, const StepParams& p) {
    const float* f = p.u[I];
    return I == J ? Dminus<J>(f, x, y, z, p) : Dplus<J>(f, x, y, z, p);
}

// psi^{IJ} <- b psi^{IJ} + a g on the axis-J slab; returns the new value (0 off
// the slab) and the indicator chi_J there
template <int I, int J>
__device__ __forceinline__ float psi_step(float g, int x, int y, int z, const StepParams& p, float& chi) {
    chi = 0.0f;
    const int k = coord<J>(x, y, z);
    const int l = axis_slab<J>(k, p);
    if (l < 0) return 0.0f;
    constexpr int h = (I != J);  // sigma^{IJ}, I != J, is on the half lattice along J
    const float a = ptab<J>(p, h, 0, k), b = ptab<J>(p, h, 1, k);
    chi = ptab<J>(p, h, 2, k);
    float* ps = p.psi[I][J] + slab_index(J, x, y, z, l, p);
    const float v = b * (*ps) + a * g;
    *ps = v;
    return v;
}

template <int V>
__device__ __forceinline__ void shear_update(int x, int y, int z, size_t idx, const StepParams& p) {
    constexpr int I = ShearAxes<V>::I, J = ShearAxes<V>::J;
    const float eij = dvel<I, J>(x, y, z, p);  // d_J u^I
    const float eji = dvel<J, I>(x, y, z, p);  // d_I u^J
    float cj, ci;
    const float qij = psi_step<I, J>(eij, x, y, z, p, cj);
    const float qji = psi_step<J, I>(eji, x, y, z, p, ci);
    const float m = mu_shear<V>(x, y, z, p);
    p.s[V][idx] += p.dt * m * (eij + eji + cj * qij + ci * qji);
}

__global__ void k_fwd_stress(StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const size_t idx = lin3(x, y, z, p.nx, p.ny);
    const float e0 = dvel<0, 0>(x, y, z, p), e1 = dvel<1, 1>(x, y, z, p), e2 = dvel<2, 2>(x, y, z, p);
    float c0, c1, c2;
    const float q0 = psi_step<0, 0>(e0, x, y, z, p, c0);
    const float q1 = psi_step<1, 1>(e1, x, y, z, p, c1);
    const float q2 = psi_step<2, 2>(e2, x, y, z, p, c2);
    const float theta = e0 + e1 + e2 + q0 + q1 + q2;
    const float lam = __ldg(p.lam + idx), mu2 = 2.0f * __ldg(p.mu + idx);
    p.s[0][idx] += p.dt * (lam * theta + mu2 * (e0 + c0 * q0));
    p.s[1][idx] += p.dt * (lam * theta + mu2 * (e1 + c1 * q1));
    p.s[2][idx] += p.dt * (lam * theta + mu2 * (e2 + c2 * q2));
    shear_update<3>(x, y, z, idx, p);
    shear_update<4>(x, y, z, idx, p);
    shear_update<5>(x, y, z, idx, p);
}

// ===========================================================================
// adjoint
// ===========================================================================

// F for u^K differenced along K (normal node q): Q^KK + a_K (psi^KK + chi_K Q^KK)
template <int K>
__device__ __forceinline__ float adj_normal(int x, int y, int z, const StepParams& p) {
    if (!inside(x, y, z, p)) return 0.0f;
    const size_t q = lin3(x, y, z, p.nx, p.ny);
    const float qk = __ldg(p.s[K] + q);
    const int k = coord<K>(x, y, z);
    const int l = axis_slab<K>(k, p);
    if (l < 0) return qk;
    const float a = ptab<K>(p, 0, 0, k), chi = ptab<K>(p, 0, 2, k);
    return qk + a * (__ldg(p.psi[K][K] + slab_index(K, x, y, z, l, p)) + chi * qk);
}

// F for u^K differenced along J (shear node q): Q^KJ + a_J (psi^KJ + chi_J Q^KJ)
template <int K, int J>
__device__ __forceinline__ float adj_shear(int x, int y, int z, const StepParams& p) {
    if (!inside(x, y, z, p)) return 0.0f;
    const size_t q = lin3(x, y, z, p.nx, p.ny);
    const float qs = __ldg(p.s[voigt(K, J)] + q);
    const int k = coord<J>(x, y, z);
    const int l = axis_slab<J>(k, p);
    if (l < 0) return qs;
    const float a = ptab<J>(p, 1, 0, k), chi = ptab<J>(p, 1, 2, k);
    return qs + a * (__ldg(p.psi[K][J] + slab_index(J, x, y, z, l, p)) + chi * qs);
}

// deferred tail of S2^T / S1^T for phi^{KJ}: phi <- b (phi + chi w)
template <int K, int J>
__device__ __forceinline__ void phi_tail(float w, int x, int y, int z, const StepParams& p) {
    const int k = coord<J>(x, y, z);
    const int l = axis_slab<J>(k, p);
    if (l < 0) return;
    constexpr int h = (K == J);
    const float b = ptab<J>(p, h, 1, k), chi = ptab<J>(p, h, 2, k);
    float* ph = p.phi[K][J] + slab_index(J, x, y, z, l, p);
    *ph = b * (*ph + chi * w);
}

template <int K>
__device__ __forceinline__ void adj_a_update(int x, int y, int z, size_t idx, const StepParams& p) {
    constexpr int J1 = (K + 1) % 3, J2 = (K + 2) % 3;
    const float w = p.u[K][idx];
    phi_tail<K, 0>(w, x, y, z, p);
    phi_tail<K, 1>(w, x, y, z, p);
    phi_tail<K, 2>(w, x, y, z, p);
    const float g = DplusF<K>([&](int a, int b, int c) { return adj_normal<K>(a, b, c, p); }, x, y, z, p) +
                    DminusF<J1>([&](int a, int b, int c) { return adj_shear<K, J1>(a, b, c, p); }, x, y, z, p) +
                    DminusF<J2>([&](int a, int b, int c) { return adj_shear<K, J2>(a, b, c, p); }, x, y, z, p);
    p.u[K][idx] = (1.0f - p.dt * med_avg<K>(p.alpha, x, y, z, p)) * w - p.dt * p.dt / med_avg<K>(p.rho, x, y, z, p) * g;
}

__global__ void k_adj_a(StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const size_t idx = lin3(x, y, z, p.nx, p.ny);
    adj_a_update<0>(x, y, z, idx, p);
    adj_a_update<1>(x, y, z, idx, p);
    adj_a_update<2>(x, y, z, idx, p);
}

// E for the u^I node differenced along J: w^I + a_J (phi^IJ + chi_J w^I)
template <int I, int J>
__device__ __forceinline__ float adj_vel(int x, int y, int z, const StepParams& p) {
    if (!inside(x, y, z, p)) return 0.0f;
    const size_t q = lin3(x, y, z, p.nx, p.ny);
    const float w = __ldg(p.u[I] + q);
    const int k = coord<J>(x, y, z);
    const int l = axis_slab<J>(k, p);
    if (l < 0) return w;
    constexpr int h = (I == J);
    const float a = ptab<J>(p, h, 0, k), chi = ptab<J>(p, h, 2, k);
    return w + a * (__ldg(p.phi[I][J] + slab_index(J, x, y, z, l, p)) + chi * w);
}

// deferred tail of S4^T / S3^T for psi^{IJ}: psi^ <- b (psi^ + chi Q)
template <int I, int J>
__device__ __forceinline__ void psi_tail(float qv, int x, int y, int z, const StepParams& p) {
    const int k = coord<J>(x, y, z);
    const int l = axis_slab<J>(k, p);
    if (l < 0) return;
    constexpr int h = (I != J);
    const float b = ptab<J>(p, h, 1, k), chi = ptab<J>(p, h, 2, k);
    float* ps = p.psi[I][J] + slab_index(J, x, y, z, l, p);
    *ps = b * (*ps + chi * qv);
}

template <int V>
__device__ __forceinline__ void adj_b_shear(int x, int y, int z, size_t idx, const StepParams& p) {
    constexpr int I = ShearAxes<V>::I, J = ShearAxes<V>::J;
    const float qo = p.s[V][idx];
    psi_tail<I, J>(qo, x, y, z, p);
    psi_tail<J, I>(qo, x, y, z, p);
    const float g = DplusF<J>([&](int a, int b, int c) { return adj_vel<I, J>(a, b, c, p); }, x, y, z, p) +
                    DplusF<I>([&](int a, int b, int c) { return adj_vel<J, I>(a, b, c, p); }, x, y, z, p);
    p.s[V][idx] = qo - mu_shear<V>(x, y, z, p) * g;
}

__global__ void k_adj_b(StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const size_t idx = lin3(x, y, z, p.nx, p.ny);
    const float q0 = p.s[0][idx], q1 = p.s[1][idx], q2 = p.s[2][idx];
    psi_tail<0, 0>(q0, x, y, z, p);
    psi_tail<1, 1>(q1, x, y, z, p);
    psi_tail<2, 2>(q2, x, y, z, p);
    const float e0 = DminusF<0>([&](int a, int b, int c) { return adj_vel<0, 0>(a, b, c, p); }, x, y, z, p);
    const float e1 = DminusF<1>([&](int a, int b, int c) { return adj_vel<1, 1>(a, b, c, p); }, x, y, z, p);
    const float e2 = DminusF<2>([&](int a, int b, int c) { return adj_vel<2, 2>(a, b, c, p); }, x, y, z, p);
    const float lt = __ldg(p.lam + idx) * (e0 + e1 + e2), mu2 = 2.0f * __ldg(p.mu + idx);
    p.s[0][idx] = q0 - (lt + mu2 * e0);
    p.s[1][idx] = q1 - (lt + mu2 * e1);
    p.s[2][idx] = q2 - (lt + mu2 * e2);
    adj_b_shear<3>(x, y, z, idx, p);
    adj_b_shear<4>(x, y, z, idx, p);
    adj_b_shear<5>(x, y, z, idx, p);
}

// ===========================================================================
// source, sampler, injection, read-out, medium check
// ===========================================================================

// tau (Eq. (initialp0)): sigma^ii = -p0 / 3 (other fields already zero)
// With band_count set, the same pass counts the nonzero p0 entries at nodes
// within `band` nodes of a face: the C-PML memory variables start at zero
// (Appendix A.3), so the support of p0 should stay 2 nodes clear of the layer.
// The loop advances whole warps (blockDim is a multiple of 32) so that every
// lane takes part in the ballot; one atomic per warp with a hit.
__global__ void k_source(const float* __restrict__ p0, float* s0, float* s1, float* s2, size_t n, int nx, int ny,
                         int z0g, int nzg, int band, unsigned long long* band_count) {
    const unsigned lane = threadIdx.x & 31u;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t base = blockIdx.x * (size_t)blockDim.x + (threadIdx.x - lane); base < n; base += stride) {
        const size_t i = base + lane;
        bool hit = false;
        if (i < n) {
            const float q = __ldg(p0 + i);
            const float v = -q * (1.0f / 3.0f);
            s0[i] = v;
            s1[i] = v;
            s2[i] = v;
            if (band_count && q != 0.0f) {
                const int x = (int)(i % (size_t)nx);
                const size_t r = i / (size_t)nx;
                const int y = (int)(r % (size_t)ny);
                const int z = z0g + (int)(r / (size_t)ny);  // plane of the whole grid
                const int dmin = min(min(min(x, nx - 1 - x), min(y, ny - 1 - y)), min(z, nzg - 1 - z));
                hit = dmin < band;
            }
        }
        if (band_count) {
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            if (m && lane == 0) atomicAdd(band_count, (unsigned long long)__popc(m));
        }
    }
}

// tau^T: image = -(sigma~11 + sigma~22 + sigma~33) / 3 = -tr(Q) / (3 (3 lambda + 2 mu))
__global__ void k_readout(const float* __restrict__ s0, const float* __restrict__ s1, const float* __restrict__ s2,
                          const float* __restrict__ lam, const float* __restrict__ mu, float* img, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float k3 = 3.0f * (3.0f * __ldg(lam + i) + 2.0f * __ldg(mu + i));
        img[i] = -__fdividef(__ldg(s0 + i) + __ldg(s1 + i) + __ldg(s2 + i), k3);
    }
}

// sigma^11 + sigma^22 + sigma^33 at a receiver corner; a corner stored as ~q
// lies in an item that writes sigma^11 alone (ITEM_DEEP), where the three
// are equal: 3 sigma^11, bitwise the sum (s + s is exact, so both round 3 s once)
__device__ __forceinline__ float corner_trace(const float* __restrict__ s0, const float* __restrict__ s1,
                                              const float* __restrict__ s2, int q) {
    return q >= 0 ? __ldg(s0 + q) + __ldg(s1 + q) + __ldg(s2 + q) : 3.0f * __ldg(s0 + ~q);
}

// Theta (Eq. (interpgrid)): out[l] = -sum_c w_c (s11 + s22 + s33)(c)
__global__ void k_sample(const float* __restrict__ s0, const float* __restrict__ s1, const float* __restrict__ s2,
                         RecTable r, float* out) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= r.L) return;
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) acc += __ldg(r.weight + 8 * l + c) * corner_trace(s0, s1, s2, __ldg(r.corner + 8 * l + c));
    out[l] = -acc;
}

// Theta^T: sigma~^ii(point) -= sum over contributions w * p_hat[l], i.e.
// Q^ii(point) -= (3 lambda + 2 mu) * that sum; one thread per distinct corner
// point, contributions in a fixed order (deterministic)
__global__ void k_inject(float* s0, float* s1, float* s2, const float* __restrict__ lam, const float* __restrict__ mu,
                         RecTable r, const float* __restrict__ ph) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= r.ncorner) return;
    float acc = 0.0f;
    for (int e = __ldg(r.inj_off + c); e < __ldg(r.inj_off + c + 1); ++e)
        acc += __ldg(r.inj_w + e) * __ldg(ph + __ldg(r.inj_rec + e));
    const int q = __ldg(r.inj_point + c);
    acc *= 3.0f * __ldg(lam + q) + 2.0f * __ldg(mu + q);
    s0[q] -= acc;
    s1[q] -= acc;
    s2[q] -= acc;
}

// ---- receivers of a graph-launched solve (state in device memory) ----------
// Fixed grids with grid-stride loops: the captured launch serves any L.
constexpr int kRecBlocks = 16, kRecThreads = 256;

// After every thread of the launch has read st->m: the last block to finish
// advances the step count for the next step's launch.
__device__ __forceinline__ void step_done(SolveState* st) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&st->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        st->done = 0;
        st->m = st->m + 1;
        __threadfence();
    }
}

__global__ void k_set_state(SolveState* st, SolveState v) { *st = v; }

__global__ void k_sample_state(const float* __restrict__ s0, const float* __restrict__ s1,
                               const float* __restrict__ s2, SolveState* st) {
    const int m = *(volatile int*)&st->m;
    const RecTable r = st->r;
    float* out = st->out + (size_t)(m + 1) * r.L;
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < r.L; l += gridDim.x * blockDim.x) {
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            acc += __ldg(r.weight + 8 * l + c) * corner_trace(s0, s1, s2, __ldg(r.corner + 8 * l + c));
        out[l] = -acc;
    }
    step_done(st);
}

__global__ void k_inject_state(float* s0, float* s1, float* s2, const float* __restrict__ lam,
                               const float* __restrict__ mu, SolveState* st) {
    const int m = *(volatile int*)&st->m;
    const RecTable r = st->r;
    const float* ph = st->in + (size_t)(st->nsteps - (m + 1)) * r.L;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < r.ncorner; c += gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int e = __ldg(r.inj_off + c); e < __ldg(r.inj_off + c + 1); ++e)
            acc += __ldg(r.inj_w + e) * __ldg(ph + __ldg(r.inj_rec + e));
        const int q = __ldg(r.inj_point + c);
        acc *= 3.0f * __ldg(lam + q) + 2.0f * __ldg(mu + q);
        s0[q] -= acc;
        s1[q] -= acc;
        s2[q] -= acc;
    }
    step_done(st);
}

// 1/mu for the TMA-staged kernels (+inf at fluid nodes, where mu = 0)
__global__ void k_inv_mu(const float* __restrict__ mu, float* inv, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float m = mu[i];
        inv[i] = m > 0.0f ? 1.0f / m : __int_as_float(0x7f800000);
    }
}

// medium reduction: [0] max (lambda+2mu)/rho, [1] max alpha, as float bits
// (all values checked >= 0 before use); [2] count of invalid nodes
__global__ void k_medium_check(const float* __restrict__ rho, const float* __restrict__ lam,
                               const float* __restrict__ mu, const float* __restrict__ alpha, size_t n,
                               unsigned int* out) {
    float cmax = 0.0f, amax = 0.0f;
    unsigned int bad = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float r = rho[i], l = lam[i], m = mu[i], a = alpha[i];
        const float m2 = l + 2.0f * m;
        const bool ok = (r > 0.0f) && (m >= 0.0f) && (m2 > 0.0f) && (3.0f * l + 2.0f * m > 0.0f) && (a >= 0.0f) &&
                        isfinite(r) && isfinite(l) && isfinite(m) && isfinite(a);
        if (!ok) {
            ++bad;
            continue;
        }
        cmax = fmaxf(cmax, m2 / r);
        amax = fmaxf(amax, a);
    }
    for (int o = 16; o > 0; o >>= 1) {
        cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out + 0, __float_as_uint(cmax));
        atomicMax(out + 1, __float_as_uint(amax));
        atomicAdd(out + 2, bad);
    }
}

// ---------------------------------------------------------------------------
// launchers (host)
// ---------------------------------------------------------------------------
static dim3 step_grid(const StepParams& p, dim3 blk) {
    return dim3((p.nx + blk.x - 1) / blk.x, (p.ny + blk.y - 1) / blk.y, p.nz);
}

void launch_fwd_velocity(const StepParams& p, cudaStream_t st) {
    const dim3 blk(32, 8, 1);
    k_fwd_velocity<<<step_grid(p, blk), blk, 0, st>>>(p);
}

void launch_fwd_stress(const StepParams& p, cudaStream_t st) {
    const dim3 blk(32, 8, 1);
    k_fwd_stress<<<step_grid(p, blk), blk, 0, st>>>(p);
}

void launch_adj_a(const StepParams& p, cudaStream_t st) {
    const dim3 blk(32, 8, 1);
    k_adj_a<<<step_grid(p, blk), blk, 0, st>>>(p);
}

void launch_adj_b(const StepParams& p, cudaStream_t st) {
    const dim3 blk(32, 8, 1);
    k_adj_b<<<step_grid(p, blk), blk, 0, st>>>(p);
}

static int ew_blocks(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b < 148 * 16 ? b : 148 * 16);
}

// band_count: nullptr, or a zeroed device counter for the p0-near-the-layer warning
// (only counted when the grid has a C-PML: band = P + 2).
void launch_source(const float* p0, const StepParams& p, cudaStream_t st, unsigned long long* band_count) {
    const size_t n = (size_t)p.nx * p.ny * p.nz;
    unsigned long long* c = p.P > 0 ? band_count : nullptr;
    k_source<<<ew_blocks(n), 256, 0, st>>>(p0, p.s[0], p.s[1], p.s[2], n, p.nx, p.ny, p.z0g, p.nzg, p.P + 2, c);
}

void launch_readout(float* img, const StepParams& p, cudaStream_t st) {
    const size_t n = (size_t)p.nx * p.ny * p.nz;
    k_readout<<<ew_blocks(n), 256, 0, st>>>(p.s[0], p.s[1], p.s[2], p.lam, p.mu, img, n);
}

void launch_sample(const StepParams& p, const RecTable& r, float* out, cudaStream_t st) {
    if (r.L > 0) k_sample<<<(r.L + 127) / 128, 128, 0, st>>>(p.s[0], p.s[1], p.s[2], r, out);
}

void launch_inject(const StepParams& p, const RecTable& r, const float* ph, cudaStream_t st) {
    if (r.ncorner > 0) k_inject<<<(r.ncorner + 127) / 128, 128, 0, st>>>(p.s[0], p.s[1], p.s[2], p.lam, p.mu, r, ph);
}

void launch_set_state(SolveState* st, const SolveState& v, cudaStream_t stream) {
    k_set_state<<<1, 1, 0, stream>>>(st, v);
}

void launch_sample_state(const StepParams& p, SolveState* st, cudaStream_t stream) {
    k_sample_state<<<kRecBlocks, kRecThreads, 0, stream>>>(p.s[0], p.s[1], p.s[2], st);
}

void launch_inject_state(const StepParams& p, SolveState* st, cudaStream_t stream) {
    k_inject_state<<<kRecBlocks, kRecThreads, 0, stream>>>(p.s[0], p.s[1], p.s[2], p.lam, p.mu, st);
}

void launch_inv_mu(const float* mu, float* inv, size_t n, cudaStream_t st) {
    k_inv_mu<<<ew_blocks(n), 256, 0, st>>>(mu, inv, n);
}

void launch_medium_check(const float* rho, const float* lam, const float* mu, const float* alpha, size_t n,
                         unsigned int* out, cudaStream_t st) {
    k_medium_check<<<ew_blocks(n), 256, 0, st>>>(rho, lam, mu, alpha, n, out);
}
