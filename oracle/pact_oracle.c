/*
 * pact_oracle.c -- FP64 CPU oracle for the elastic-wave forward operator H and
 * its discrete adjoint H^T (Mitsuhashi et al., "A forward-adjoint operator pair
 * based on the elastic wave equation for use in transcranial photoacoustic
 * computed tomography").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * only tests/, __graft_entry__.smoke() and the cpu_baseline / reference legs of
 * bench.py load it.  It shares no code, header, table or constant with the CUDA
 * library; both sides are written independently from the paper.
 *
 * Style: plain loops, double precision, zero padding outside the grid, every
 * operator evaluated from its definition.  The forward step is applied as the
 * four sub-updates of Appendix A.3, Eq. (PropagatePML) / the four-line update
 * after Eq. (opPML):
 *     S1: phi   <- B phi + E sigma                 (memory variables of d sigma)
 *     S2: u     <- J u + Phi sigma + Gamma phi     (velocity, Eq. (it) + C-PML)
 *     S3: psi   <- B~ psi + E~ u                   (memory variables of d u)
 *     S4: sigma <- sigma + Psi u + Delta psi       (stress, Eq. (it) + C-PML)
 * and the adjoint applies the literal transposes S1^T S2^T S3^T S4^T (S4^T
 * first), written in SCATTER form: every term "out(p) += c * in(q)" of a forward
 * sub-update becomes "adj_in(q) += c * adj_out(p)".  The oracle therefore never
 * relies on the identity (D+)^T = -(D-) that a gather-form adjoint would use.
 * Scatter loops run over z in five colour classes (z mod 5): a scatter from
 * plane z touches planes z-2..z+2 only, so within one class no two threads
 * write the same plane, and every target element receives its contributions
 * in the same (class) order whatever the thread count.
 *
 * Readings of the paper where it is silent or inconsistent (each one is listed
 * in the design notes of the repository):
 *  - staggered positions (Sec. 2.2; the figure is missing): sigma11,22,33, lambda,
 *    mu, rho, alpha, p0 at (i,j,k); u1 at (i+1/2,j,k), u2 at (i,j+1/2,k),
 *    u3 at (i,j,k+1/2); sigma23 at (i,j+1/2,k+1/2), sigma13 at (i+1/2,j,k+1/2),
 *    sigma12 at (i+1/2,j+1/2,k).  Each lattice has N = nx*ny*nz points.
 *  - 4th-order staggered difference (Sec. 2.2, Eq. (derivative)) in two forms:
 *      integer -> half   (Dp f)[k] = (9/8 (f[k+1]-f[k]) - 1/24 (f[k+2]-f[k-1]))/dx
 *      half -> integer   (Dm g)[k] = (9/8 (g[k]-g[k-1]) - 1/24 (g[k+1]-g[k-2]))/dx
 *    with every index outside [0,n) reading zero.
 *  - rho, alpha at velocity nodes: arithmetic mean of the two neighbouring
 *    integer nodes (Sec. 6.1 averages density and absorption at interfaces);
 *    the missing neighbour past the last index is clamped to the edge value.
 *  - mu at shear nodes: harmonic mean of the four surrounding integer nodes,
 *    zero if any of them is zero; out-of-range neighbours clamped.
 *  - source: sigma^ii_0 = -p0/3 (Eq. (Ini), tau of Eq. (initialp0)); the -I of
 *    tau' in Appendix A.3 is read as the same -1/3.
 *  - sampler: p_hat[l] = -R_l (sigma11 + sigma22 + sigma33) with trilinear R_l
 *    on the integer lattice (Eq. (interpgrid)); receiver coordinates are given
 *    in grid-index units.
 *  - C-PML coefficients (Appendix A.1-A.3, kappa = 1): phi^{ij} lives at the u^i
 *    node and psi^{ij} at the sigma^{ij} node, and both use the axis-j profile
 *    (a_j, b_j, chi_j) evaluated at that node's j coordinate.
 *  - C-PML profile (the paper gives only kappa = 1): s = depth into the layer
 *    in cells (clamped to npml), d = d0 (s/npml)^2 with
 *    d0 = -3 vmax ln(R0) / (2 npml dx), beta = pi f0 (1 - s/npml),
 *    b = exp(-(d + beta) dt), a = d (b - 1) / (d + beta), chi = 1; outside the
 *    layer d = beta = a = chi = 0 and b = 1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int nx, ny, nz;
    double dx, dt;
    int npml;
    double pml_R0, pml_f0, pml_vmax;
} or_desc;

/* Voigt order of the stress vector, Sec. 2.2: 11, 22, 33, 23, 13, 12. */
static const int VOIGT[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};

typedef struct {
    or_desc g;
    size_t n;
    /* staggered medium, Sec. 2.2 diagonals Q_i, A_i, Lambda, M */
    double *rho_u[3], *alpha_u[3]; /* at u^i nodes */
    double *lam, *mu;              /* at integer nodes (normal stresses) */
    double *mu_s[3];               /* shear nodes, order 23, 13, 12 */
    /* C-PML 1-D profiles per axis at integer [0] and half [1] positions */
    double *pa[3][2], *pb[3][2], *pchi[3][2], *pd[3][2], *pbeta[3][2];
} or_ctx;

/* State vector v'_m of Appendix A.3: [phi (9N), u (3N), psi (9N), sigma (6N)],
 * phi and psi in the order 11,12,13,21,22,23,31,32,33 (Eq. (auxPML)). */
#define PHI(st, i, j, N) ((st) + (size_t)(3 * (i) + (j)) * (N))
#define UU(st, i, N) ((st) + (size_t)(9 + (i)) * (N))
#define PSI(st, i, j, N) ((st) + (size_t)(12 + 3 * (i) + (j)) * (N))
#define SIG(st, v, N) ((st) + (size_t)(21 + (v)) * (N))

static inline size_t lin(const or_desc *g, int x, int y, int z) {
    return ((size_t)z * g->ny + y) * g->nx + x;
}

static inline int dim(const or_desc *g, int axis) {
    return axis == 0 ? g->nx : (axis == 1 ? g->ny : g->nz);
}

/* value of field f at (c[0],c[1],c[2]) with zero padding outside the grid */
static inline double at(const or_desc *g, const double *f, const int c[3]) {
    if (c[0] < 0 || c[0] >= g->nx || c[1] < 0 || c[1] >= g->ny || c[2] < 0 || c[2] >= g->nz)
        return 0.0;
    return f[lin(g, c[0], c[1], c[2])];
}

static inline double tap(const or_desc *g, const double *f, int x, int y, int z, int axis, int off) {
    int c[3] = {x, y, z};
    c[axis] += off;
    return at(g, f, c);
}

/* Eq. (derivative), integer lattice -> half lattice (result sits at k+1/2) */
static double Dp(const or_desc *g, const double *f, int x, int y, int z, int axis) {
    double c1 = tap(g, f, x, y, z, axis, 1) - tap(g, f, x, y, z, axis, 0);
    double c3 = tap(g, f, x, y, z, axis, 2) - tap(g, f, x, y, z, axis, -1);
    return (9.0 / 8.0 * c1 - 1.0 / 24.0 * c3) / g->dx;
}

/* Eq. (derivative), half lattice (index k <-> k+1/2) -> integer lattice */
static double Dm(const or_desc *g, const double *f, int x, int y, int z, int axis) {
    double c1 = tap(g, f, x, y, z, axis, 0) - tap(g, f, x, y, z, axis, -1);
    double c3 = tap(g, f, x, y, z, axis, 1) - tap(g, f, x, y, z, axis, -2);
    return (9.0 / 8.0 * c1 - 1.0 / 24.0 * c3) / g->dx;
}

static inline void add_at(const or_desc *g, double *f, int x, int y, int z, int axis, int off, double v) {
    int c[3] = {x, y, z};
    c[axis] += off;
    if (c[0] < 0 || c[0] >= g->nx || c[1] < 0 || c[1] >= g->ny || c[2] < 0 || c[2] >= g->nz)
        return; /* the forward read a zero-padded value here: nothing to transpose */
    f[lin(g, c[0], c[1], c[2])] += v;
}

/* transpose of "out(p) += c * (Dp f)(p)": scatter c into the four taps of f */
static void Dp_T(const or_desc *g, double *f, int x, int y, int z, int axis, double c) {
    double s = c / g->dx;
    add_at(g, f, x, y, z, axis, 1, 9.0 / 8.0 * s);
    add_at(g, f, x, y, z, axis, 0, -9.0 / 8.0 * s);
    add_at(g, f, x, y, z, axis, 2, -1.0 / 24.0 * s);
    add_at(g, f, x, y, z, axis, -1, 1.0 / 24.0 * s);
}

/* transpose of "out(p) += c * (Dm g)(p)" */
static void Dm_T(const or_desc *g, double *f, int x, int y, int z, int axis, double c) {
    double s = c / g->dx;
    add_at(g, f, x, y, z, axis, 0, 9.0 / 8.0 * s);
    add_at(g, f, x, y, z, axis, -1, -9.0 / 8.0 * s);
    add_at(g, f, x, y, z, axis, 1, -1.0 / 24.0 * s);
    add_at(g, f, x, y, z, axis, -2, 1.0 / 24.0 * s);
}

/* --------------------------------------------------------------------------
 * C-PML 1-D profile, Appendix A.1 (b and a of the memory-variable recursion)
 * with kappa = 1 (Appendix A.2).  pos is a grid-index coordinate (k or k+1/2).
 * ------------------------------------------------------------------------ */
static void pml_point(int n, int npml, double dx, double dt, double vmax, double R0, double f0,
                      double pos, double *d, double *beta, double *a, double *b, double *chi) {
    *d = 0.0; *beta = 0.0; *a = 0.0; *b = 1.0; *chi = 0.0;
    if (npml <= 0) return;
    double s = 0.0;
    if (pos < (double)npml) s = (double)npml - pos;
    else if (pos > (double)(n - 1 - npml)) s = pos - (double)(n - 1 - npml);
    if (s <= 0.0) return;
    if (s > (double)npml) s = (double)npml;
    double L = npml * dx;
    double d0 = -3.0 * vmax * log(R0) / (2.0 * L);
    double r = s / (double)npml;
    *d = d0 * r * r;
    *beta = M_PI * f0 * (1.0 - r);
    *b = exp(-(*d + *beta) * dt);
    *a = (*d + *beta) > 0.0 ? (*d) * (*b - 1.0) / (*d + *beta) : 0.0;
    *chi = 1.0;
}

void or_pml_profile(int n, int npml, double dx, double dt, double vmax, double R0, double f0, int half,
                    double *d, double *beta, double *a, double *b, double *chi) {
    for (int k = 0; k < n; ++k)
        pml_point(n, npml, dx, dt, vmax, R0, f0, k + (half ? 0.5 : 0.0), &d[k], &beta[k], &a[k], &b[k], &chi[k]);
}

/* --------------------------------------------------------------------------
 * Staggered medium (Sec. 2.2 matrices Q_i, A_i, Lambda_jk, M_jk)
 * ------------------------------------------------------------------------ */
static double clamp_at(const or_desc *g, const double *f, int x, int y, int z) {
    if (x > g->nx - 1) x = g->nx - 1;
    if (y > g->ny - 1) y = g->ny - 1;
    if (z > g->nz - 1) z = g->nz - 1;
    return f[lin(g, x, y, z)];
}

static double harmonic4(double m0, double m1, double m2, double m3) {
    if (m0 == 0.0 || m1 == 0.0 || m2 == 0.0 || m3 == 0.0) return 0.0;
    return 4.0 / (1.0 / m0 + 1.0 / m1 + 1.0 / m2 + 1.0 / m3);
}

or_ctx *or_create(const or_desc *g, const double *rho, const double *lam, const double *mu, const double *alpha) {
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    c->g = *g;
    size_t N = (size_t)g->nx * g->ny * g->nz;
    c->n = N;
    for (int i = 0; i < 3; ++i) {
        c->rho_u[i] = (double *)malloc(N * sizeof(double));
        c->alpha_u[i] = (double *)malloc(N * sizeof(double));
        c->mu_s[i] = (double *)malloc(N * sizeof(double));
    }
    c->lam = (double *)malloc(N * sizeof(double));
    c->mu = (double *)malloc(N * sizeof(double));
    memcpy(c->lam, lam, N * sizeof(double));
    memcpy(c->mu, mu, N * sizeof(double));
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t p = lin(g, x, y, z);
                int nb[3][3] = {{x + 1, y, z}, {x, y + 1, z}, {x, y, z + 1}};
                for (int i = 0; i < 3; ++i) {
                    c->rho_u[i][p] = 0.5 * (rho[p] + clamp_at(g, rho, nb[i][0], nb[i][1], nb[i][2]));
                    c->alpha_u[i][p] = 0.5 * (alpha[p] + clamp_at(g, alpha, nb[i][0], nb[i][1], nb[i][2]));
                }
                /* sigma23 at (x, y+1/2, z+1/2): the y-z plane square */
                c->mu_s[0][p] = harmonic4(mu[p], clamp_at(g, mu, x, y + 1, z), clamp_at(g, mu, x, y, z + 1),
                                          clamp_at(g, mu, x, y + 1, z + 1));
                /* sigma13 at (x+1/2, y, z+1/2): the x-z plane square */
                c->mu_s[1][p] = harmonic4(mu[p], clamp_at(g, mu, x + 1, y, z), clamp_at(g, mu, x, y, z + 1),
                                          clamp_at(g, mu, x + 1, y, z + 1));
                /* sigma12 at (x+1/2, y+1/2, z): the x-y plane square */
                c->mu_s[2][p] = harmonic4(mu[p], clamp_at(g, mu, x + 1, y, z), clamp_at(g, mu, x, y + 1, z),
                                          clamp_at(g, mu, x + 1, y + 1, z));
            }
    for (int ax = 0; ax < 3; ++ax)
        for (int h = 0; h < 2; ++h) {
            int n = dim(g, ax);
            c->pa[ax][h] = (double *)malloc(n * sizeof(double));
            c->pb[ax][h] = (double *)malloc(n * sizeof(double));
            c->pchi[ax][h] = (double *)malloc(n * sizeof(double));
            c->pd[ax][h] = (double *)malloc(n * sizeof(double));
            c->pbeta[ax][h] = (double *)malloc(n * sizeof(double));
            or_pml_profile(n, g->npml, g->dx, g->dt, g->pml_vmax, g->pml_R0, g->pml_f0, h, c->pd[ax][h],
                           c->pbeta[ax][h], c->pa[ax][h], c->pb[ax][h], c->pchi[ax][h]);
        }
    return c;
}

void or_free(or_ctx *c) {
    if (!c) return;
    for (int i = 0; i < 3; ++i) {
        free(c->rho_u[i]); free(c->alpha_u[i]); free(c->mu_s[i]);
    }
    free(c->lam); free(c->mu);
    for (int ax = 0; ax < 3; ++ax)
        for (int h = 0; h < 2; ++h) {
            free(c->pa[ax][h]); free(c->pb[ax][h]); free(c->pchi[ax][h]); free(c->pd[ax][h]); free(c->pbeta[ax][h]);
        }
    free(c);
}

/* copies of the staggered medium for tests: rho_u, alpha_u, mu_s are 3N each */
void or_get_stagger(const or_ctx *c, double *rho_u, double *alpha_u, double *mu_s) {
    for (int i = 0; i < 3; ++i) {
        memcpy(rho_u + i * c->n, c->rho_u[i], c->n * sizeof(double));
        memcpy(alpha_u + i * c->n, c->alpha_u[i], c->n * sizeof(double));
        memcpy(mu_s + i * c->n, c->mu_s[i], c->n * sizeof(double));
    }
}

/* PML profile value along `axis` for a point whose coordinate on that axis is
 * on the half lattice (half = 1) or the integer lattice (half = 0). */
static inline double PA(const or_ctx *c, int axis, int half, int x, int y, int z) {
    int k = axis == 0 ? x : (axis == 1 ? y : z);
    return c->pa[axis][half][k];
}
static inline double PB(const or_ctx *c, int axis, int half, int x, int y, int z) {
    int k = axis == 0 ? x : (axis == 1 ? y : z);
    return c->pb[axis][half][k];
}
static inline double PCHI(const or_ctx *c, int axis, int half, int x, int y, int z) {
    int k = axis == 0 ? x : (axis == 1 ? y : z);
    return c->pchi[axis][half][k];
}

/* u^i lies on the half lattice along axis i only; sigma^{ij} (i != j) on the
 * half lattice along i and j; sigma^{ii} on the integer lattice. */
static inline int u_half(int i, int axis) { return axis == i; }
static inline int s_half(int i, int j, int axis) { return i != j && (axis == i || axis == j); }

/* d_j sigma^{ij} evaluated at the u^i node (Sec. 2.2, Phi of Eq. (Operatordef)) */
static double dsig(const or_ctx *c, const double *st, int i, int j, int x, int y, int z) {
    const double *s = SIG(st, VOIGT[i][j], c->n);
    return (i == j) ? Dp(&c->g, s, x, y, z, j) : Dm(&c->g, s, x, y, z, j);
}

/* d_j u^i evaluated at the sigma^{ij} node (Psi of Eq. (Operatordef)) */
static double du(const or_ctx *c, const double *st, int i, int j, int x, int y, int z) {
    const double *u = UU(st, i, c->n);
    return (i == j) ? Dm(&c->g, u, x, y, z, j) : Dp(&c->g, u, x, y, z, j);
}

/* ========================= forward sub-updates ========================== */

/* S1: phi^{ij} <- b_j phi^{ij} + a_j d_j sigma^{ij}   (E_ij, B_ij of Eq. (opPML)) */
static void S1(const or_ctx *c, double *st) {
    const or_desc *g = &c->g;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t p = lin(g, x, y, z);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        int h = u_half(i, j);
                        double *ph = PHI(st, i, j, c->n);
                        ph[p] = PB(c, j, h, x, y, z) * ph[p] + PA(c, j, h, x, y, z) * dsig(c, st, i, j, x, y, z);
                    }
            }
}

/* S2: u^i <- (1 - dt alpha_i) u^i + dt/rho_i sum_j (d_j sigma^{ij} + chi_j phi^{ij})
 *     (J, Phi of Eq. (Operatordef); Gamma of Eq. (opPML)) */
static void S2(const or_ctx *c, double *st) {
    const or_desc *g = &c->g;
    double dt = g->dt;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t p = lin(g, x, y, z);
                for (int i = 0; i < 3; ++i) {
                    double acc = 0.0;
                    for (int j = 0; j < 3; ++j)
                        acc += dsig(c, st, i, j, x, y, z) +
                               PCHI(c, j, u_half(i, j), x, y, z) * PHI(st, i, j, c->n)[p];
                    double *u = UU(st, i, c->n);
                    u[p] = (1.0 - dt * c->alpha_u[i][p]) * u[p] + dt / c->rho_u[i][p] * acc;
                }
            }
}

/* S3: psi^{ij} <- b~_j psi^{ij} + a~_j d_j u^i   (E~_ij, B~_ij of Eq. (opPML)) */
static void S3(const or_ctx *c, double *st) {
    const or_desc *g = &c->g;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t p = lin(g, x, y, z);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        int h = s_half(i, j, j);
                        double *ps = PSI(st, i, j, c->n);
                        ps[p] = PB(c, j, h, x, y, z) * ps[p] + PA(c, j, h, x, y, z) * du(c, st, i, j, x, y, z);
                    }
            }
}

/* S4: sigma^{ii} += dt [lambda sum_k (d_k u^k + psi^{kk}) + 2 mu (d_i u^i + chi_i psi^{ii})]
 *     sigma^{ij} += dt mu_ij (d_i u^j + d_j u^i + chi_j psi^{ij} + chi_i psi^{ji})
 *     (Psi of Eq. (Operatordef); Delta of Eq. (opPML)) */
static void S4(const or_ctx *c, double *st) {
    const or_desc *g = &c->g;
    double dt = g->dt;
    size_t N = c->n;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t p = lin(g, x, y, z);
                double theta = 0.0;
                for (int k = 0; k < 3; ++k) theta += du(c, st, k, k, x, y, z) + PSI(st, k, k, N)[p];
                for (int i = 0; i < 3; ++i) {
                    double e = du(c, st, i, i, x, y, z) + PCHI(c, i, 0, x, y, z) * PSI(st, i, i, N)[p];
                    SIG(st, i, N)[p] += dt * (c->lam[p] * theta + 2.0 * c->mu[p] * e);
                }
                for (int i = 0; i < 3; ++i)
                    for (int j = i + 1; j < 3; ++j) {
                        int v = VOIGT[i][j];
                        double m = c->mu_s[v - 3][p];
                        double e = du(c, st, j, i, x, y, z) + du(c, st, i, j, x, y, z) +
                                   PCHI(c, j, 1, x, y, z) * PSI(st, i, j, N)[p] +
                                   PCHI(c, i, 1, x, y, z) * PSI(st, j, i, N)[p];
                        SIG(st, v, N)[p] += dt * m * e;
                    }
            }
}

/* ==================== transposed sub-updates (scatter) ==================== */

/* scatter form of d_j sigma^{ij} at the u^i node */
static void dsig_T(const or_ctx *c, double *st, int i, int j, int x, int y, int z, double v) {
    double *s = SIG(st, VOIGT[i][j], c->n);
    if (i == j) Dp_T(&c->g, s, x, y, z, j, v);
    else Dm_T(&c->g, s, x, y, z, j, v);
}

/* scatter form of d_j u^i at the sigma^{ij} node */
static void du_T(const or_ctx *c, double *st, int i, int j, int x, int y, int z, double v) {
    double *u = UU(st, i, c->n);
    if (i == j) Dm_T(&c->g, u, x, y, z, j, v);
    else Dp_T(&c->g, u, x, y, z, j, v);
}

/* S4^T: u += Psi^T sigma, psi += Delta^T sigma, sigma unchanged */
static void S4T(const or_ctx *c, double *st) {
    const or_desc *g = &c->g;
    double dt = g->dt;
    size_t N = c->n;
    for (int ph = 0; ph < 5; ++ph)
#pragma omp parallel for schedule(static)
    for (int z = ph; z < g->nz; z += 5)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t p = lin(g, x, y, z);
                for (int i = 0; i < 3; ++i) {
                    double s = SIG(st, i, N)[p];
                    /* terms dt*lambda*(d_k u^k + psi^kk) for every k */
                    for (int k = 0; k < 3; ++k) {
                        du_T(c, st, k, k, x, y, z, dt * c->lam[p] * s);
                        PSI(st, k, k, N)[p] += dt * c->lam[p] * s;
                    }
                    /* terms 2 dt mu (d_i u^i + chi_i psi^ii) */
                    du_T(c, st, i, i, x, y, z, 2.0 * dt * c->mu[p] * s);
                    PSI(st, i, i, N)[p] += 2.0 * dt * c->mu[p] * PCHI(c, i, 0, x, y, z) * s;
                }
                for (int i = 0; i < 3; ++i)
                    for (int j = i + 1; j < 3; ++j) {
                        int v = VOIGT[i][j];
                        double w = dt * c->mu_s[v - 3][p] * SIG(st, v, N)[p];
                        du_T(c, st, j, i, x, y, z, w);
                        du_T(c, st, i, j, x, y, z, w);
                        PSI(st, i, j, N)[p] += PCHI(c, j, 1, x, y, z) * w;
                        PSI(st, j, i, N)[p] += PCHI(c, i, 1, x, y, z) * w;
                    }
            }
}

/* S3^T: u += E~^T psi, then psi <- B~ psi */
static void S3T(const or_ctx *c, double *st) {
    const or_desc *g = &c->g;
    size_t N = c->n;
    for (int ph = 0; ph < 5; ++ph)
#pragma omp parallel for schedule(static)
    for (int z = ph; z < g->nz; z += 5)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t p = lin(g, x, y, z);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        int h = s_half(i, j, j);
                        du_T(c, st, i, j, x, y, z, PA(c, j, h, x, y, z) * PSI(st, i, j, N)[p]);
                    }
            }
#pragma omp parallel for schedule(static)
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t p = lin(g, x, y, z);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) PSI(st, i, j, N)[p] *= PB(c, j, s_half(i, j, j), x, y, z);
            }
}

/* S2^T: sigma += Phi^T u, phi += Gamma^T u, then u <- J u */
static void S2T(const or_ctx *c, double *st) {
    const or_desc *g = &c->g;
    double dt = g->dt;
    size_t N = c->n;
    for (int ph = 0; ph < 5; ++ph)
#pragma omp parallel for schedule(static)
    for (int z = ph; z < g->nz; z += 5)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t p = lin(g, x, y, z);
                for (int i = 0; i < 3; ++i) {
                    double w = dt / c->rho_u[i][p] * UU(st, i, N)[p];
                    for (int j = 0; j < 3; ++j) {
                        dsig_T(c, st, i, j, x, y, z, w);
                        PHI(st, i, j, N)[p] += PCHI(c, j, u_half(i, j), x, y, z) * w;
                    }
                }
            }
#pragma omp parallel for schedule(static)
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t p = lin(g, x, y, z);
                for (int i = 0; i < 3; ++i) UU(st, i, N)[p] *= (1.0 - dt * c->alpha_u[i][p]);
            }
}

/* S1^T: sigma += E^T phi, then phi <- B phi */
static void S1T(const or_ctx *c, double *st) {
    const or_desc *g = &c->g;
    size_t N = c->n;
    for (int ph = 0; ph < 5; ++ph)
#pragma omp parallel for schedule(static)
    for (int z = ph; z < g->nz; z += 5)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t p = lin(g, x, y, z);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        int h = u_half(i, j);
                        dsig_T(c, st, i, j, x, y, z, PA(c, j, h, x, y, z) * PHI(st, i, j, N)[p]);
                    }
            }
#pragma omp parallel for schedule(static)
    for (int z = 0; z < g->nz; ++z)
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x) {
                size_t p = lin(g, x, y, z);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) PHI(st, i, j, N)[p] *= PB(c, j, u_half(i, j), x, y, z);
            }
}

/* one sub-update k in {1,2,3,4}, forward (transpose = 0) or transposed */
void or_substep(const or_ctx *c, int k, int transpose, double *st) {
    if (!transpose) {
        if (k == 1) S1(c, st);
        else if (k == 2) S2(c, st);
        else if (k == 3) S3(c, st);
        else if (k == 4) S4(c, st);
    } else {
        if (k == 1) S1T(c, st);
        else if (k == 2) S2T(c, st);
        else if (k == 3) S3T(c, st);
        else if (k == 4) S4T(c, st);
    }
}

/* v'_{m+1} = W' v'_m (Appendix A.3) */
void or_step(const or_ctx *c, double *st) {
    S1(c, st); S2(c, st); S3(c, st); S4(c, st);
}

/* v <- W'^T v, i.e. S1^T S2^T S3^T S4^T applied right to left */
void or_step_T(const or_ctx *c, double *st) {
    S4T(c, st); S3T(c, st); S2T(c, st); S1T(c, st);
}

/* ====================== source, sampler, read-out ======================== */

/* tau' (Eq. (initialp0PML), read with -1/3): zero state, sigma^ii = -p0/3 */
void or_inject(const or_ctx *c, const double *p0, double *st) {
    size_t N = c->n;
    memset(st, 0, 27 * N * sizeof(double));
    for (int i = 0; i < 3; ++i)
        for (size_t p = 0; p < N; ++p) SIG(st, i, N)[p] = -p0[p] / 3.0;
}

/* tau'^T: image = -1/3 (sigma11 + sigma22 + sigma33) */
void or_readout(const or_ctx *c, const double *st, double *img) {
    size_t N = c->n;
    for (size_t p = 0; p < N; ++p)
        img[p] = -(SIG(st, 0, N)[p] + SIG(st, 1, N)[p] + SIG(st, 2, N)[p]) / 3.0;
}

/* trilinear weights R_l on the integer lattice: corner (cx,cy,cz) in {0,1}^3 */
static int corners(const or_desc *g, const double *r, size_t idx[8], double w[8]) {
    int i0 = (int)floor(r[0]), j0 = (int)floor(r[1]), k0 = (int)floor(r[2]);
    double fx = r[0] - i0, fy = r[1] - j0, fz = r[2] - k0;
    int q = 0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                int x = i0 + cx, y = j0 + cy, z = k0 + cz;
                double wt = (cx ? fx : 1.0 - fx) * (cy ? fy : 1.0 - fy) * (cz ? fz : 1.0 - fz);
                if (x < 0 || x >= g->nx || y < 0 || y >= g->ny || z < 0 || z >= g->nz) {
                    idx[q] = 0; w[q] = 0.0; /* zero padding; weight dropped */
                } else {
                    idx[q] = lin(g, x, y, z); w[q] = wt;
                }
                ++q;
            }
    return 8;
}

/* Theta': out[l] = -R_l (sigma11 + sigma22 + sigma33) (Eq. (interpgridPML)) */
void or_sample(const or_ctx *c, const double *rec, int L, const double *st, double *out) {
    size_t N = c->n;
    for (int l = 0; l < L; ++l) {
        size_t idx[8]; double w[8];
        corners(&c->g, rec + 3 * l, idx, w);
        double acc = 0.0;
        for (int q = 0; q < 8; ++q)
            acc += w[q] * (SIG(st, 0, N)[idx[q]] + SIG(st, 1, N)[idx[q]] + SIG(st, 2, N)[idx[q]]);
        out[l] = -acc;
    }
}

/* Theta'^T: sigma^ii(corner) += -w * p_hat[l] for i = 1,2,3 */
void or_sample_T(const or_ctx *c, const double *rec, int L, const double *ph, double *st) {
    size_t N = c->n;
    for (int l = 0; l < L; ++l) {
        size_t idx[8]; double w[8];
        corners(&c->g, rec + 3 * l, idx, w);
        for (int q = 0; q < 8; ++q)
            for (int i = 0; i < 3; ++i) SIG(st, i, N)[idx[q]] += -w[q] * ph[l];
    }
}

/* ========================== operators H and H^T ========================== */

/* p_hat = H p0 (Eq. (HPML)); traces is (nsteps+1) x L, time-major. */
void or_forward(const or_ctx *c, const double *p0, const double *rec, int L, int nsteps, double *traces) {
    double *st = (double *)malloc(27 * c->n * sizeof(double));
    or_inject(c, p0, st);
    or_sample(c, rec, L, st, traces);
    for (int m = 1; m <= nsteps; ++m) {
        or_step(c, st);
        or_sample(c, rec, L, st, traces + (size_t)m * L);
    }
    free(st);
}

/* p_adj = H^T p_hat (Eq. (adjHPML)) via the recursion of Eq. (AdjupPML):
 * v_{M-1} = Theta'^T p_{M-1};  v_{m-1} = Theta'^T p_{m-1} + W'^T v_m;
 * p_adj = tau'^T v_0. */
void or_adjoint(const or_ctx *c, const double *traces, const double *rec, int L, int nsteps, double *img) {
    double *st = (double *)calloc(27 * c->n, sizeof(double));
    or_sample_T(c, rec, L, traces + (size_t)nsteps * L, st);
    for (int m = nsteps; m >= 1; --m) {
        or_step_T(c, st);
        or_sample_T(c, rec, L, traces + (size_t)(m - 1) * L, st);
    }
    or_readout(c, st, img);
    free(st);
}

/* forward run that also returns the full state after `nsteps` steps */
void or_run_state(const or_ctx *c, const double *p0, int nsteps, double *st) {
    or_inject(c, p0, st);
    for (int m = 1; m <= nsteps; ++m) or_step(c, st);
}
