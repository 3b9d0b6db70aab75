/*
 * pact.h -- C ABI of libpact.so: the elastic-wave photoacoustic forward
 * operator H and its exact discrete adjoint H^T on one NVIDIA B300 (sm_103a).
 *
 * The operator pair follows Mitsuhashi et al., "A forward-adjoint operator pair
 * based on the elastic wave equation for use in transcranial photoacoustic
 * computed tomography": H maps an initial pressure p0 to receiver traces
 * through the staggered-grid velocity-stress FDTD recursion with a
 * convolutional PML (Appendix A.3, Eq. (HPML)); H^T is its matrix transpose
 * applied by the backward recursion of Eq. (AdjupPML).
 *
 * Conventions shared by every call
 *  - Grid: nx * ny * nz vertices, spacing dx [m]; every 3-D array is float32,
 *    C order [z][y][x] (x fastest), N = nx*ny*nz entries.  This is the
 *    lexicographic order of the paper's field vectors (Sec. 2.2).
 *  - Staggering (Sec. 2.2): p0, rho, lambda, mu, alpha and the normal stresses
 *    at integer nodes (i,j,k); u^1 at (i+1/2,j,k), u^2 at (i,j+1/2,k),
 *    u^3 at (i,j,k+1/2); sigma^23, sigma^13, sigma^12 at the matching two-half
 *    positions.  rho and alpha are averaged arithmetically onto the velocity
 *    nodes, mu harmonically onto the shear nodes.  Values outside the grid are
 *    zero (zero padding).
 *  - Receivers: rec_xyz is a HOST array of L float triples (x, y, z) in
 *    grid-index units on the integer lattice; each must satisfy
 *    0 <= x <= nx-2 (same for y, z).  Sampling is trilinear (Eq. (interpgrid)).
 *  - Traces: float32 [(nsteps+1)][L], time-major: row m is p_hat_m, the
 *    negative sum of the three normal stresses at time m*dt (Sec. 2.3).
 *  - Source: sigma^11 = sigma^22 = sigma^33 = -p0/3 at t = 0, everything else
 *    zero (Eq. (Ini)); so row 0 of the traces is the trilinear interpolant of p0.
 *  - Device pointers (p0, traces, image, medium arrays) must be cudaMalloc'd or
 *    torch CUDA memory on the handle's device; the caller keeps ownership.
 *  - Every compute call is asynchronous and ordered on the handle's stream;
 *    host-pointer variants (*_host) copy in and out and return after the
 *    stream has finished.  A handle must not be used from two host threads at
 *    once.  No C++ exception crosses this interface.
 *  - Errors: every call returns a PACT_* code; pact_last_error(h) gives the
 *    message of the last failure on h (pact_last_error(NULL) the last failure
 *    of a call that had no valid handle).
 */
#ifndef PACT_H
#define PACT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PACT_OK 0
#define PACT_EINVAL 1   /* bad dimensions, pointers, receivers or sizes            */
#define PACT_ECFL 2     /* c_max * dt / dx >= 6 / (7 sqrt 3) (4th-order stability) */
#define PACT_ENOMEM 3   /* device allocation failed                                */
#define PACT_ECUDA 4    /* a CUDA runtime call failed (message has the detail)     */
#define PACT_ETIMEOUT 5 /* a bounded device wait expired                           */
#define PACT_ESTATE 6   /* call out of order (e.g. forward before set_medium)      */

typedef struct pact_grid* pact_handle;

/* Grid and time step of one operator pair.  C-PML (Appendix A.1-A.3, kappa = 1):
 * layer npml cells thick on every face; damping d(s) = d0 (s/npml)^2 with
 * d0 = -3 vmax ln(R0) / (2 npml dx), s the depth into the layer in cells;
 * frequency shift beta(s) = pi f0 (1 - s/npml).  pml_vmax <= 0 means "use the
 * largest compressional speed of the medium". */
typedef struct {
    int nx, ny, nz;   /* vertices per axis, each >= max(4, 2*npml + 2)             */
    double dx;        /* grid spacing [m]                                          */
    double dt;        /* time step [s]                                             */
    int npml;         /* C-PML thickness in cells (0: zero-padded boundary)        */
    double pml_R0;    /* nominal normal-incidence reflection, e.g. 1e-4            */
    double pml_f0;    /* CFS shift frequency [Hz], e.g. 1e6                        */
    double pml_vmax;  /* speed scaling the damping [m/s]; <= 0: medium maximum     */
} pact_grid_desc;

/* Create a handle for one grid (Sec. 2.2 discretisation).  Allocates the
 * wavefield (9 arrays of N floats), the medium copy (4 x N), the C-PML memory
 * variables (18 arrays, stored only on the layer slabs) and the profile tables
 * on the current CUDA device.  stream: a cudaStream_t (NULL = legacy default
 * stream) on which every later call of this handle is ordered.
 * Errors: PACT_EINVAL (bad desc or out == NULL), PACT_ENOMEM, PACT_ECUDA. */
int pact_create_grid(const pact_grid_desc* desc, void* stream, pact_handle* out);

/* Copy the medium into the handle: density rho [kg/m^3] > 0, Lame lambda and
 * mu [Pa] (mu >= 0, lambda + 2 mu > 0, bulk modulus 3 lambda + 2 mu > 0, which
 * the adjoint's read-out divides by), absorption alpha [1/s] >= 0, all
 * device arrays of N floats at the integer nodes (Sec. 2.1, Eq. (Elastic)).
 * Builds the C-PML profile tables.  Synchronises the stream (it reduces the
 * medium to check it).  Errors: PACT_EINVAL (NULL pointer or a value out of
 * range), PACT_ECFL (c_max dt / dx >= 6/(7 sqrt 3), or alpha dt >= 1),
 * PACT_ECUDA. */
int pact_set_medium(pact_handle h, const float* rho, const float* lambda, const float* mu,
                    const float* alpha);
/* (With mu = 0 at every node -- the acoustic operator pair H_{mu=0},
 * H^T_{mu=0} of the paper's ablation, Sec. 7 -- the three normal stresses stay
 * equal and the shear stresses zero; on TMA-staged grids the interior tiles
 * then run acoustic kernels that carry one stress field, and the C-PML frame
 * the elastic ones.  The results are those of the elastic operator with
 * mu = 0.  PACT_ACOUSTIC=0 in the environment keeps the elastic kernels.) */

/* p_hat = H p0 (Eq. (H); with the C-PML Eq. (HPML)): load sigma^ii = -p0/3,
 * sample p_hat_0, then nsteps times apply one leapfrog step (velocity and
 * memory variables phi, then stress and memory variables psi; Appendix A.3) and
 * sample.  p0: device, N floats.  traces: device, (nsteps+1)*L floats,
 * overwritten.  nsteps >= 0, L >= 1.  Errors: PACT_EINVAL, PACT_ESTATE (no
 * medium), PACT_ENOMEM, PACT_ECUDA.
 * With PACT_FUSED=1 in the environment at pact_create_grid, on grids with
 * nx % 4 == 0 whose interior holds a region off the C-PML slabs, the interior
 * tiles run one single-pass (velocity + stress) kernel per step on two
 * wavefield buffers; the first pact_forward / pact_adjoint on such a handle
 * then allocates the second buffer (9N floats).  By default every tile runs
 * the in-place velocity and stress kernels. */
int pact_forward(pact_handle h, const float* p0, const float* rec_xyz, int L, int nsteps, float* traces);

/* p_adj = H^T p_hat (Eq. (adjHPML)) by the backward recursion of Eq. (AdjupPML):
 * v = Theta^T p_hat_{nsteps}; for m = nsteps..1: v = W^T v + Theta^T p_hat_{m-1};
 * p_adj = tau^T v = -(sigma^11 + sigma^22 + sigma^33)/3.  W^T applies the
 * transposed sub-updates in reverse order (Sec. 4, Eq. (backwardstep)).
 * traces: device, (nsteps+1)*L floats (read only).  image: device, N floats,
 * overwritten.  Errors as pact_forward. */
int pact_adjoint(pact_handle h, const float* traces, const float* rec_xyz, int L, int nsteps, float* image);

/* Same as pact_forward / pact_adjoint with HOST p0 / traces / image buffers:
 * copies in, runs, copies out, and returns after the stream has finished.
 * Device staging buffers are owned by the handle and reused. */
int pact_forward_host(pact_handle h, const float* p0, const float* rec_xyz, int L, int nsteps, float* traces);
int pact_adjoint_host(pact_handle h, const float* traces, const float* rec_xyz, int L, int nsteps, float* image);

/* Warning, not an error, about the p0 of the last forward solve started on h
 * (pact_forward, pact_forward_host, or pact_begin with is_adjoint = 0): the
 * number of nonzero p0 entries at nodes within npml + 2 nodes of a face
 * (min(x, nx-1-x, y, ny-1-y, z, nz-1-z) < npml + 2).  The C-PML memory
 * variables start at zero (Appendix A.3), so the support of p0 should stay at
 * least 2 grid positions away from the layer; a nonzero count says it does not
 * (the solve ran regardless).  Always 0 when npml = 0.  The count is taken by
 * the source kernel in the same pass.  n_points: host.  Waits for the
 * handle's stream.  Errors: PACT_EINVAL (NULL argument), PACT_ECUDA. */
int pact_support_warning(pact_handle h, long long* n_points);

/* Release everything the handle owns (waits for its stream first). */
int pact_destroy(pact_handle h);

/* Message of the last failure on h (or of a handle-less call for h == NULL).
 * The pointer stays valid until the next failing call on the same handle. */
const char* pact_last_error(pact_handle h);

/* Device bytes a handle with this desc will allocate for serving (fields,
 * medium, C-PML slabs and tables, receiver tables for L receivers; pact_begin
 * runs in place on one wavefield buffer).  Used for admission against a
 * memory budget.  pact_forward / pact_adjoint may add a second wavefield
 * buffer of 9N floats (see pact_forward).  Errors: PACT_EINVAL. */
int pact_query_bytes(const pact_grid_desc* desc, int L, int nsteps, size_t* bytes);

/* Diagnostics: copy the current wavefield to HOST memory, 9*N floats in the
 * order u^1, u^2, u^3, sigma^11, sigma^22, sigma^33, sigma^23, sigma^13, sigma^12
 * (Sec. 2.2 vectors u_bar, sigma_bar) after pact_forward.  After pact_adjoint
 * the same slots hold the adjoint state in the library's weighted variables
 * w = dt u~ / rho_bar and Q = C sigma~ (C: the stiffness of the stress update).
 * Synchronises the stream. */
int pact_get_wavefield(pact_handle h, float* host_out);

/* ---- serving: many solves advanced together ------------------------------
 * A solve is prepared on its handle with pact_begin, then any set of prepared
 * handles (forward and adjoint, any grid sizes) is advanced together by
 * pact_advance.  Each solve advances on its own CUDA graphs of whole steps
 * (those of pact_forward / pact_adjoint) on a stream of its handle, so that
 * the solves of one advance overlap on the device; solves below a size
 * (PACT_SERVE_SOLO_POINTS in the environment at pact_begin; default 0, i.e.
 * none) instead go to persistent multi-instance kernels that walk a device
 * table of solves.  Both run the same step bodies, so a result is the same
 * alone and in a mix.  Not part of the paper: this is how the operator pair
 * is served to concurrent requests. */

/* Prepare one solve on h (queued on the handle's stream).  is_adjoint = 0:
 * forward, in = p0 (device, N floats), out = traces (device, (nsteps+1)*L),
 * row 0 is written now; is_adjoint = 1: adjoint, in = traces (device,
 * (nsteps+1)*L), out = image (device, N), written when the solve finishes.
 * Needs nx % 4 == 0 (TMA-staged kernels).  L = 0 is accepted here (a z-slab
 * that owns no receiver): no traces are read or written and the trace
 * pointer may be NULL.  Errors as pact_forward. */
int pact_begin(pact_handle h, int is_adjoint, const float* in, const float* rec_xyz, int L, int nsteps, float* out);

/* Advance every unfinished solve among hs[0..n-1] (n <= 64, one device) by
 * min(ksteps, steps left) time steps, queued on `stream` (cudaStream_t): the
 * step graphs of each solve on its handle's serving stream, forked from and
 * joined back to `stream`, and one replay of a captured CUDA graph of ksteps
 * multi-instance steps for the solves on the multi-instance kernels; a solve
 * that finishes gets its read-out.  Work queued on `stream` after the call
 * runs after all of it.  pact_begin of these handles must be ordered before
 * it (use the same stream).  All advances on one device share one device
 * table of solves and one set of work counters, so the library orders them:
 * an advance queued on a different stream than the previous advance on that
 * device first waits (cudaStreamWaitEvent) for the previous replay, and
 * table replays on one device therefore never run concurrently.  Errors:
 * PACT_EINVAL, PACT_ECUDA,
 * PACT_ETIMEOUT (an earlier advance on this device reported a timed-out
 * wait); message via pact_last_error(NULL). */
int pact_advance(pact_handle* hs, int n, int ksteps, void* stream);

/* Steps done by the solve prepared on h (host bookkeeping; never touches the
 * GPU).  Results are complete once steps_done == nsteps and the stream has
 * reached that point. */
int pact_poll(pact_handle h, int* steps_done);

/* ---- z-slab decomposition: one slab of a larger grid per handle ------------
 * The paper runs H and H^T on several GPUs (the CUDA + MPI implementation of
 * its implementation section) by splitting the grid; here a slab handle holds
 * planes [z_lo, z_hi) of the grid `global` (its own planes plus two halo planes
 * on each side that touches another slab), and the caller exchanges the halo
 * planes between the two half steps of every time step.  The C-PML z layer of
 * a slab handle lies at the whole grid's ends (Appendix A.3): a slab in the
 * middle has no z layer.  Medium, p0, traces, image and receiver coordinates of
 * a slab handle are those of its own grid of (z_hi - z_lo) planes (receiver z
 * relative to z_lo).  Errors: PACT_EINVAL (global fails the pact_create_grid
 * checks, 0 <= z_lo < z_hi <= global->nz violated, or fewer than 5 planes),
 * PACT_ENOMEM, PACT_ECUDA. */
int pact_create_slab(const pact_grid_desc* global, int z_lo, int z_hi, void* stream, pact_handle* out);

/* One half step of the solve prepared on h by pact_begin (any handle, a slab
 * handle included): stress = 0 the velocity-family half (forward: phi, u of
 * Eq. (it); adjoint: the transposes of the stress update, Eq. (backwardstep)),
 * stress = 1 the stress-family half.  A time step is the velocity half, the
 * stress half and pact_step_receivers, in that order.  Queued on the handle's
 * stream.  Errors: PACT_ESTATE (no unfinished solve), PACT_EINVAL (a handle
 * created with PACT_FUSED=1), PACT_ECUDA. */
int pact_step_half(pact_handle h, int stress);

/* Finish the time step of the solve prepared on h: forward, sample row m of
 * the traces (Theta, Eq. (interpgrid)); adjoint, inject row nsteps - m
 * (Theta^T); the adjoint's read-out (tau^T) follows the last step.  Advances
 * the step count that pact_poll reports.  Errors as pact_step_half. */
int pact_step_receivers(pact_handle h);

/* Device address of wavefield array `field` of h (0..8: u^1, u^2, u^3,
 * sigma^11, sigma^22, sigma^33, sigma^23, sigma^13, sigma^12; after an adjoint
 * pact_begin the same slots hold w and Q): N floats, [z][y][x], one z plane
 * of nx*ny floats contiguous.  For halo exchange between slab handles; the
 * library owns the memory.  During a solve on a medium with fluid and solid
 * nodes, sigma^22 and sigma^33 (Q^22, Q^33) of fluid points far from every
 * solid node hold stale values (the library writes sigma^11 alone there and
 * fills the other two before an image read-out or pact_get_wavefield); the
 * planes a slab exchanges are never such points.  Errors: PACT_EINVAL. */
int pact_field_ptr(pact_handle h, int field, float** out);

/* Forward operator H that allocates no device memory.  The paper has no
 * counterpart: this is a deployment variant of pact_forward for callers that
 * cannot call cudaMalloc -- code inside a host application that owns all device
 * memory through its own pool and forbids outside allocations (they would escape
 * its accounting, or fail once the pool has reserved the device).
 * All working memory (wavefield 9N floats, C-PML slabs, profile tables,
 * receiver tables: about 36 bytes per grid point plus the slabs) comes from one
 * fixed file-scope device array of PACT_NOALLOC_SCRATCH_BYTES (64 MiB); a grid
 * too large for it is rejected with PACT_EINVAL and a message giving the bytes
 * it would need (roughly up to 110^3 points with a thin layer).  The array is
 * committed on a device when the library's module holding it is loaded there;
 * under CUDA's default lazy module loading that is the first call of this
 * entry point on the device (with that device current), unless other work of
 * the library came first.  Make that first call at set-up time, before a pool
 * reserves the device; from then on the device holds the array until the
 * process exits, and later calls commit no device memory.
 * Inputs and outputs are the caller's: desc as for pact_create_grid; rho,
 * lambda, mu, alpha and p0 device arrays of N floats (read only); rec_xyz a
 * HOST array of L triples; traces a device array of (nsteps+1)*L floats,
 * overwritten, with the same values pact_forward produces.  stream:
 * cudaStream_t (NULL = legacy default).
 * Synchronisation: every call checks the medium on the device and reads the
 * result back (16 bytes), which waits for the stream, and copies the C-PML and
 * receiver tables from pageable host memory; so every call blocks the host
 * until the stream reaches that point, and a call cannot be captured in a CUDA
 * graph.  The steps are then queued asynchronously.  The array's device
 * address is looked up (cudaGetSymbolAddress) on every call in the current
 * context.  Every call reuses the same array and clears what must start at
 * zero; calls that overlap on the GPU (two streams or two host threads) race
 * and corrupt each other.  Unlike pact_forward, no count of p0 entries near
 * the absorbing layer is kept (pact_support_warning has no counterpart here).
 * Errors: PACT_EINVAL, PACT_ECFL, PACT_ECUDA; message via pact_last_error(NULL). */
#define PACT_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
int pact_forward_noalloc(const pact_grid_desc* desc, const float* rho, const float* lambda, const float* mu,
                         const float* alpha, const float* p0, const float* rec_xyz, int L, int nsteps,
                         float* traces, void* stream);

/* Proximal step of a total-variation penalty with non-negativity, for
 * penalised least-squares reconstruction with H and H^T (the use the paper
 * names in Sec. 8):  x = argmin_{x >= 0} 1/2 ||x - b||^2 + tau TV(x), with
 * TV(x) = sum_i |grad x_i| (isotropic; forward differences, zero at the last
 * index of each axis), by iters iterations of Beck and Teboulle's fast
 * gradient projection on the dual field.  b, x: device arrays of
 * N = nx*ny*nz floats, [z][y][x] (x fastest), x must not alias b; work: a
 * device array of 6N floats owned by the caller (the dual field and its
 * previous iterate; contents on entry are ignored).  tau >= 0 (tau = 0 or
 * iters = 0 gives max(0, b)).  Queued on stream (cudaStream_t, NULL = legacy
 * default), asynchronous.  Errors: PACT_EINVAL, PACT_ECUDA; message via
 * pact_last_error(NULL). */
int pact_tv_prox_nn(const float* b, float* x, int nx, int ny, int nz, float tau, int iters, float* work,
                    void* stream);

/* Linear time resampling of receiver traces, for data simulated with one time
 * step and reconstructed with another (the non-inverse-crime study of
 * Sec. 6.2).  in: device, m_in x L floats (time-major, as pact_forward writes
 * them); out: device, m_out x L floats, overwritten with
 * out[k][l] = in(s0 + k * ratio)[l], linear between neighbouring input
 * samples and zero outside [0, m_in - 1] (s0 and ratio in input samples).
 * Queued on stream (cudaStream_t), asynchronous.  Errors: PACT_EINVAL,
 * PACT_ECUDA; message via pact_last_error(NULL). */
int pact_resample_traces(const float* in, int m_in, float* out, int m_out, int L, double s0, double ratio,
                         void* stream);

/* Self-check of failure detection (not part of the method).  The TMA-staged
 * kernels bound every wait on an mbarrier (2 s of wall time), record a timed-out
 * wait in a status word and leave; the host reports it as PACT_ETIMEOUT.  This
 * call runs the same bounded wait on an mbarrier that nothing ever completes,
 * with a limit of limit_us microseconds (1 .. 2e6), on stream (cudaStream_t),
 * and waits for the stream.  Returns PACT_ETIMEOUT when the wait gave up as it
 * must (the context stays usable), PACT_OK if it did not, PACT_EINVAL for a
 * limit out of range, PACT_ENOMEM / PACT_ECUDA on a CUDA failure. */
int pact_check_bounded_wait(unsigned int limit_us, void* stream);

/* Measurement support (not part of the method).  Kernel roles counted and
 * timed by pact_profile / pact_profile_read. */
#define PACT_K_FWD_VELOCITY 0 /* velocity + phi update of one forward step        */
#define PACT_K_FWD_STRESS 1   /* stress + psi update of one forward step          */
#define PACT_K_ADJ_A 2        /* velocity-side half of one adjoint step           */
#define PACT_K_ADJ_B 3        /* stress-side half of one adjoint step             */
#define PACT_K_SAMPLE 4       /* receiver sampling Theta                          */
#define PACT_K_INJECT 5       /* receiver injection Theta^T                       */
#define PACT_K_SOURCE 6       /* source tau                                       */
#define PACT_K_READOUT 7      /* read-out tau^T                                   */
#define PACT_K_FWD_FUSED 8    /* single-pass velocity + stress kernel, forward    */
#define PACT_K_ADJ_FUSED 9    /* single-pass kernel of one adjoint step           */
#define PACT_K_FWD_AC_VEL 10  /* acoustic interior velocity kernel (mu = 0)       */
#define PACT_K_FWD_AC_STR 11  /* acoustic interior stress kernel (mu = 0)         */
#define PACT_K_ADJ_AC_A 12    /* acoustic interior kernel, adjoint half A         */
#define PACT_K_ADJ_AC_B 13    /* acoustic interior kernel, adjoint half B         */
#define PACT_NKIND 14
#define PACT_K_ALL 14         /* pact_profile_read only: every kernel launch     */

/* Reset this handle's launch counters and, if enable != 0, start recording a
 * CUDA event after every kernel launch on the handle's stream (so a launch's
 * device time is the time since the previous event; the stream is busy between
 * consecutive launches of one call).  Synchronises the stream. */
int pact_profile(pact_handle h, int enable);

/* Invocations of one kernel role since pact_profile (one step half of the
 * role may launch up to three kernels: C-PML frame, z-slab planes, interior),
 * and their summed device time in milliseconds (0 if recording was off).
 * kind = PACT_K_ALL gives the number of kernel launches of all roles and the
 * device time of all of them.  Synchronises the stream.
 * Errors: PACT_EINVAL (kind out of range or NULL output). */
int pact_profile_read(pact_handle h, int kind, long long* launches, double* total_ms);

/* Grid points that one invocation of a step role (PACT_K_FWD_VELOCITY,
 * PACT_K_FWD_STRESS, PACT_K_ADJ_A, PACT_K_ADJ_B, PACT_K_FWD_FUSED,
 * PACT_K_ADJ_FUSED, PACT_K_FWD_AC_VEL, PACT_K_FWD_AC_STR, PACT_K_ADJ_AC_A,
 * PACT_K_ADJ_AC_B) updates on this handle's grid, and the C-PML slab points
 * among them; 0 for a role that this grid does not run.  Used to turn a
 * role's device time into algorithmic bytes per second.  Errors: PACT_EINVAL. */
int pact_role_points(pact_handle h, int kind, long long* points, long long* slab_points);

/* Work-item classes of the medium-adaptive step (media with fluid nodes):
 * PACT_ITEM_DEEP, fluid points that no solid node's update reads, whose
 * stress-family update writes sigma^11 alone (sigma^22 and sigma^33 equal it
 * there and are filled in before they are read: 8 bytes fewer per point and
 * stress half); PACT_ITEM_NOALPHA, fluid points whose velocity-family update
 * reads alpha = 0 at every node and loads no alpha (4 bytes fewer per point
 * and velocity half).  *points = grid points of that class; 0 on media
 * without fluid nodes.  Errors: PACT_EINVAL (unknown class, NULL). */
#define PACT_ITEM_DEEP 1
#define PACT_ITEM_NOALPHA 2
int pact_item_points(pact_handle h, int item_class, long long* points);

#ifdef __cplusplus
}
#endif

#endif /* PACT_H */
