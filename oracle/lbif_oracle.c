/*
 * FP64 CPU oracle for the lattice Boltzmann method for inhomogeneous
 * hard-sphere fluids (Melchionna & Marconi, "Lattice Boltzmann method for
 * inhomogeneous fluids", EPL 2008).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA path is checked against. Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it. The product path never calls it
 * and shares no code, header, table or constant with it.
 *
 * Everything is FP64 and written as plain loops in the order the paper gives:
 *   1. moments n, u = j/n                      (Sec. Theory, moments of f)
 *   2. coarse-grained density nbar over a ball of radius sigma/2 and the
 *      contact value g2(etabar) at the midpoint r + sigma/2 (Sec. Methods,
 *      Fischer-Methfessel prescription)
 *   3. hard-sphere force C1 of Eq. LBHS with the 18-point sphere rule
 *      (6 on-lattice points, 12 off-lattice points bilinearly interpolated)
 *      and the wall regulariser (1 - exp(-|r - r_w|/sigma)) on the
 *      density-current term, at constant temperature
 *   4. optional mean-field attractive tail (Sec. Conclusions: attractive
 *      forces as a generalisation)
 *   5. BGK relaxation to the second-order equilibrium plus the first-order
 *      Hermite source w_i c_i.F / v_T^2 (forward-Euler update; C0 = 0)
 *   6. two-array push streaming, halfway bounce-back at the slit walls,
 *      periodic x and y.
 *
 * Readings of points the paper leaves open:
 *   - walls sit half-way, at z = -1/2 and z = nz - 1/2; all nz nodes are fluid
 *   - the ball is the lattice solid sphere |d|^2 <= (sigma/2)^2, normalised
 *     by its node count
 *   - g2 "as printed": (1 - e/2 + e^2/4)/(1 - e)^3; form 1 = Carnahan-Starling
 *   - off-lattice points interpolate the fields n, u (at r + sigma s) and
 *     g2 (at r + sigma s/2) separately; the products are formed afterwards
 *   - outside the fluid n = 0, u = 0, g2 = 0; x, y (and z when periodic)
 *     wrap, summed over displacements
 *   - source S_i = w_i c_i.F / c_s^2 (first Hermite order), u = j/n unshifted
 *   - regulariser distance = distance of node r to the nearest wall plane
 *   - initial density n0 (1 + a (2U - 1)), U from SplitMix64(seed ^ index)
 *
 * Units: lattice spacing 1, time step 1, m = 1, k_B T = v_T^2 = c_s^2 = 1/3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV 19 /* D3Q19 */
#define NS 18 /* sphere quadrature points */

/* ------------------------------------------------------------------------- */
/* D3Q19 velocity set, built from its definition: all c in {-1,0,1}^3 with    */
/* |c|^2 <= 2; Gauss-Hermite weights 1/3 (rest), 1/18 (|c|=1), 1/36 (|c|^2=2) */
/* ------------------------------------------------------------------------- */
static int    cv[NV][3];
static double wv[NV];
static int    opp[NV];

/* A&S 18-point rule on the unit sphere: 6 axis points (weight 1/30) and the
 * 12 face-diagonal points (+-1,+-1,0)/sqrt2 and permutations (weight 1/15).  */
static double sdir[NS][3];
static double swt[NS];

static void build_tables(void)
{
    int q = 0;
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                int s = cx * cx + cy * cy + cz * cz;
                if (s > 2) continue;
                cv[q][0] = cx; cv[q][1] = cy; cv[q][2] = cz;
                wv[q] = (s == 0) ? 1.0 / 3.0 : (s == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
                ++q;
            }
    for (int i = 0; i < NV; ++i)
        for (int j = 0; j < NV; ++j)
            if (cv[j][0] == -cv[i][0] && cv[j][1] == -cv[i][1] && cv[j][2] == -cv[i][2])
                opp[i] = j;

    q = 0;
    for (int a = 0; a < 3; ++a)
        for (int s = -1; s <= 1; s += 2) {
            sdir[q][0] = sdir[q][1] = sdir[q][2] = 0.0;
            sdir[q][a] = (double)s;
            swt[q] = 1.0 / 30.0;
            ++q;
        }
    const double h = 1.0 / sqrt(2.0);
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            for (int sa = -1; sa <= 1; sa += 2)
                for (int sb = -1; sb <= 1; sb += 2) {
                    sdir[q][0] = sdir[q][1] = sdir[q][2] = 0.0;
                    sdir[q][a] = sa * h;
                    sdir[q][b] = sb * h;
                    swt[q] = 1.0 / 15.0;
                    ++q;
                }
}

__attribute__((constructor)) static void oracle_init(void) { build_tables(); }

/* Copies of the tables for the isotropy and quadrature pins. */
void or_lattice(int* c, double* w)
{
    for (int i = 0; i < NV; ++i) {
        c[3 * i + 0] = cv[i][0]; c[3 * i + 1] = cv[i][1]; c[3 * i + 2] = cv[i][2];
        w[i] = wv[i];
    }
}

void or_sphere_rule(double* dir, double* w)
{
    for (int q = 0; q < NS; ++q) {
        dir[3 * q + 0] = sdir[q][0]; dir[3 * q + 1] = sdir[q][1]; dir[3 * q + 2] = sdir[q][2];
        w[q] = swt[q];
    }
}

/* ------------------------------------------------------------------------- */
/* geometry: x, y periodic; z periodic or bounded by two walls                */
/* ------------------------------------------------------------------------- */
typedef struct { int nx, ny, nz, zper; } geom;

static inline int wrapi(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

/* index of the fluid node at integer position, or -1 outside the slit */
static inline long node_at(const geom* g, int x, int y, int z)
{
    x = wrapi(x, g->nx);
    y = wrapi(y, g->ny);
    if (g->zper) z = wrapi(z, g->nz);
    else if (z < 0 || z >= g->nz) return -1;
    return ((long)z * g->ny + y) * g->nx + x;
}

static inline double field_at(const geom* g, const double* a, int x, int y, int z)
{
    long i = node_at(g, x, y, z);
    return i < 0 ? 0.0 : a[i];
}

/* linear interpolation at a real position from the surrounding lattice
 * nodes (the weights of a zero fractional part are skipped, so an
 * off-lattice point of the quadrature uses the four nodes of its plane)    */
static double interp(const geom* g, const double* a, double px, double py, double pz)
{
    double bx = floor(px), by = floor(py), bz = floor(pz);
    double tx = px - bx, ty = py - by, tz = pz - bz;
    double s = 0.0;
    for (int k = 0; k < 2; ++k)
        for (int j = 0; j < 2; ++j)
            for (int i = 0; i < 2; ++i) {
                double w = (i ? tx : 1.0 - tx) * (j ? ty : 1.0 - ty) * (k ? tz : 1.0 - tz);
                if (w == 0.0) continue;
                s += w * field_at(g, a, (int)bx + i, (int)by + j, (int)bz + k);
            }
    return s;
}

/* ------------------------------------------------------------------------- */
/* closures                                                                   */
/* ------------------------------------------------------------------------- */

/* contact value of the pair correlation, Sec. Methods (Fischer-Methfessel
 * paragraph); form 0 = as printed there, form 1 = Carnahan-Starling        */
/* threads the parallel loops below run on (1 without OpenMP) */
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the parallel loops from now on (n >= 1) */
void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

double or_g2(double eta, int form)
{
    double d = (1.0 - eta) * (1.0 - eta) * (1.0 - eta);
    if (form == 1) return (1.0 - 0.5 * eta) / d;
    return (1.0 - 0.5 * eta + 0.25 * eta * eta) / d;
}

/* number of lattice nodes in the ball |d|^2 <= (sigma/2)^2 */
int or_ball_count(int sigma)
{
    int r = sigma / 2, c = 0;
    for (int dz = -r; dz <= r; ++dz)
        for (int dy = -r; dy <= r; ++dy)
            for (int dx = -r; dx <= r; ++dx)
                if (dx * dx + dy * dy + dz * dz <= r * r) ++c;
    return c;
}

/* Fischer-Methfessel coarse-grained density: uniform average of n over the
 * ball of radius sigma/2 centred on each node.                             */
void or_coarse_density(int nx, int ny, int nz, int zper, int sigma, const double* n, double* nbar)
{
    geom g = {nx, ny, nz, zper};
    int r = sigma / 2;
    double inv = 1.0 / (double)or_ball_count(sigma);
    long N = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (long id = 0; id < N; ++id) {
        int x = (int)(id % nx), y = (int)((id / nx) % ny), z = (int)(id / ((long)nx * ny));
        double s = 0.0;
        for (int dz = -r; dz <= r; ++dz)
            for (int dy = -r; dy <= r; ++dy)
                for (int dx = -r; dx <= r; ++dx)
                    if (dx * dx + dy * dy + dz * dz <= r * r)
                        s += field_at(&g, n, x + dx, y + dy, z + dz);
        nbar[id] = s * inv;
    }
}

/* g2 field at every node from the coarse-grained packing fraction
 * etabar = pi sigma^3 nbar / 6 ; zero is used outside the fluid.           */
static void g2_field(long N, int sigma, int form, const double* nbar, double* G)
{
    double c = M_PI * (double)sigma * sigma * sigma / 6.0;
    for (long i = 0; i < N; ++i) G[i] = or_g2(c * nbar[i], form);
}

/* regulariser of the density-current term at node height z */
static double regulariser(const geom* g, int z, int sigma, int on)
{
    if (!on || g->zper) return 1.0;
    double dw = fmin(z + 0.5, g->nz - 0.5 - z);
    return 1.0 - exp(-dw / (double)sigma);
}

/* Hard-sphere collisional momentum source, Eq. LBHS at constant T:
 *   F(r) = -kT sigma^2 4pi sum_q W_q s_q G(r + sigma s_q/2) n(r) n(r + sigma s_q)
 *          x [1 - lambda(z) (2/(v_T sqrt(pi))) s_q.(u(r + sigma s_q) - u(r))]
 * with G the g2 field built from nbar. Also returns the local collisional
 * pressure (trace of the static part, divided by 3) when p != NULL, and,
 * when C2 != NULL, the energy source of Eq. C2eq at constant T,
 *   C2(r) = kT sigma^2 4pi sum_q W_q G(r + sigma s_q/2) n(r) n(r + sigma s_q)
 *           x ( - s_q.(u(r + sigma s_q) - u(r)) / 2 ).                      */
static void hs_force(const geom* g, int sigma, double kT, int coupling, int regularize,
                     const double* n, const double* ux, const double* uy, const double* uz,
                     const double* G, double* Fx, double* Fy, double* Fz, double* pc, double* C2)
{
    const double vT = sqrt(kT);
    const double kappa = 2.0 / (vT * sqrt(M_PI));
    const double pref = kT * (double)sigma * sigma * 4.0 * M_PI;
    const double s = (double)sigma;
    long N = (long)g->nx * g->ny * g->nz;
#pragma omp parallel for schedule(static)
    for (long id = 0; id < N; ++id) {
        int x = (int)(id % g->nx), y = (int)((id / g->nx) % g->ny), z = (int)(id / ((long)g->nx * g->ny));
        double lam = regulariser(g, z, sigma, regularize);
        double fx = 0.0, fy = 0.0, fz = 0.0, ps = 0.0, c2 = 0.0;
        for (int q = 0; q < NS; ++q) {
            double px = x + s * sdir[q][0], py = y + s * sdir[q][1], pz = z + s * sdir[q][2];
            double mx = x + 0.5 * s * sdir[q][0], my = y + 0.5 * s * sdir[q][1], mz = z + 0.5 * s * sdir[q][2];
            double nq = interp(g, n, px, py, pz);
            double Gq = interp(g, G, mx, my, mz);
            double bracket = 1.0;
            double du = 0.0;
            if (coupling || C2) {
                du = sdir[q][0] * (interp(g, ux, px, py, pz) - ux[id])
                   + sdir[q][1] * (interp(g, uy, px, py, pz) - uy[id])
                   + sdir[q][2] * (interp(g, uz, px, py, pz) - uz[id]);
            }
            if (coupling) bracket -= lam * kappa * du;
            double t = swt[q] * Gq * n[id] * nq;
            c2 += t * (-0.5 * du);
            fx += sdir[q][0] * t * bracket;
            fy += sdir[q][1] * t * bracket;
            fz += sdir[q][2] * t * bracket;
            ps += t;
        }
        Fx[id] = -pref * fx;
        Fy[id] = -pref * fy;
        Fz[id] = -pref * fz;
        /* P^c_aa/3 = (kT sigma^3/6) 4pi sum_q W_q G_q n n_q (static part) */
        if (pc) pc[id] = kT * s * s * s / 6.0 * 4.0 * M_PI * ps;
        if (C2) C2[id] = pref * c2;
    }
}

/* Mean-field attractive tail: F(r) = n(r) sum_d n(r+d) phi'(|d|) d/|d| over
 * sigma <= |d| <= rcut sigma, phi(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6].
 * phi'(|d|) and |d| depend on the displacement only: they are evaluated once
 * per displacement (same formula), and every node sums over the
 * displacements in the same order as a per-node evaluation would.          */
static void tail_force(const geom* g, int sigma, double eps, double rcut, const double* n,
                       double* Fx, double* Fy, double* Fz)
{
    const double s = (double)sigma, rmax = rcut * s;
    const int R = (int)ceil(rmax);
    const double s6 = pow(s, 6.0), s12 = s6 * s6;
    const int W = 2 * R + 1;
    double* dphi_t = (double*)malloc(sizeof(double) * (size_t)W * W * W);
    double* r_t = (double*)malloc(sizeof(double) * (size_t)W * W * W);
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                long k = ((long)(dz + R) * W + (dy + R)) * W + (dx + R);
                double r2 = (double)(dx * dx + dy * dy + dz * dz);
                double r = sqrt(r2);
                r_t[k] = r;
                dphi_t[k] = (r2 < s * s || r2 > rmax * rmax)
                                ? 0.0
                                : 4.0 * eps * (-12.0 * s12 / pow(r, 13.0) + 6.0 * s6 / pow(r, 7.0));
            }
    long N = (long)g->nx * g->ny * g->nz;
#pragma omp parallel for schedule(static)
    for (long id = 0; id < N; ++id) {
        int x = (int)(id % g->nx), y = (int)((id / g->nx) % g->ny), z = (int)(id / ((long)g->nx * g->ny));
        double fx = 0.0, fy = 0.0, fz = 0.0;
        for (int dz = -R; dz <= R; ++dz)
            for (int dy = -R; dy <= R; ++dy)
                for (int dx = -R; dx <= R; ++dx) {
                    double r2 = (double)(dx * dx + dy * dy + dz * dz);
                    if (r2 < s * s || r2 > rmax * rmax) continue;
                    double nd = field_at(g, n, x + dx, y + dy, z + dz);
                    if (nd == 0.0) continue;
                    long k = ((long)(dz + R) * W + (dy + R)) * W + (dx + R);
                    double r = r_t[k];
                    double dphi = dphi_t[k];
                    fx += nd * dphi * dx / r;
                    fy += nd * dphi * dy / r;
                    fz += nd * dphi * dz / r;
                }
        Fx[id] += n[id] * fx;
        Fy[id] += n[id] * fy;
        Fz[id] += n[id] * fz;
    }
    free(dphi_t);
    free(r_t);
}

/* second-order (low-Mach) local equilibrium, Sec. Methods */
void or_equilibrium(double n, const double* u, double* feq)
{
    const double cs2 = 1.0 / 3.0;
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < NV; ++i) {
        double cu = cv[i][0] * u[0] + cv[i][1] * u[1] + cv[i][2] * u[2];
        feq[i] = wv[i] * n * (1.0 + cu / cs2 + (cu * cu - cs2 * uu) / (2.0 * cs2 * cs2));
    }
}

/* BGK relaxation plus first-order Hermite source at one node */
void or_collide_node(const double* f, const double* F, double tau, double* fout)
{
    const double cs2 = 1.0 / 3.0;
    double n = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < NV; ++i) {
        n += f[i];
        for (int a = 0; a < 3; ++a) j[a] += cv[i][a] * f[i];
    }
    double u[3] = {j[0] / n, j[1] / n, j[2] / n};
    double feq[NV];
    or_equilibrium(n, u, feq);
    for (int i = 0; i < NV; ++i) {
        double cF = cv[i][0] * F[0] + cv[i][1] * F[1] + cv[i][2] * F[2];
        fout[i] = f[i] - (f[i] - feq[i]) / tau + wv[i] * cF / cs2;
    }
}

/* ------------------------------------------------------------------------- */
/* state                                                                      */
/* ------------------------------------------------------------------------- */
typedef struct {
    geom g;
    int sigma;
    double eta, tau, n0, kT;
    double body[3];
    int hs, coupling, regularize, g2form, tail;
    double eps, rcut;
    long N;
    double *f, *fn;                   /* [NV][N] */
    double *n, *ux, *uy, *uz;         /* moments */
    double *nbar, *G, *Fx, *Fy, *Fz, *pc;
    double *Lx, *Ly, *Lz;             /* lagged force (variant), NULL until used */
    int c2;                           /* energy source of Eq. C2eq on */
    double* C2f;                      /* its field, NULL until used */
    int lag_ok;                       /* Lx.. hold the force of the previous step */
    long t;
} or_state;

void* or_create(int nx, int ny, int nz, int zper, int sigma, double eta, double tau,
                const double* body, int hs, int coupling, int regularize, int g2form,
                int tail, double eps, double rcut)
{
    if (nx < 1 || ny < 1 || nz < 1 || sigma < 2 || (sigma % 2) || tau <= 0.5) return NULL;
    or_state* s = (or_state*)calloc(1, sizeof(or_state));
    s->g.nx = nx; s->g.ny = ny; s->g.nz = nz; s->g.zper = zper;
    s->sigma = sigma; s->eta = eta; s->tau = tau;
    s->kT = 1.0 / 3.0;
    s->n0 = 6.0 * eta / (M_PI * (double)sigma * sigma * sigma);
    for (int a = 0; a < 3; ++a) s->body[a] = body ? body[a] : 0.0;
    s->hs = hs; s->coupling = coupling; s->regularize = regularize; s->g2form = g2form;
    s->tail = tail; s->eps = eps; s->rcut = rcut;
    s->N = (long)nx * ny * nz;
    long N = s->N;
    s->f = (double*)calloc((size_t)NV * N, sizeof(double));
    s->fn = (double*)calloc((size_t)NV * N, sizeof(double));
    double** fields[] = {&s->n, &s->ux, &s->uy, &s->uz, &s->nbar, &s->G, &s->Fx, &s->Fy, &s->Fz, &s->pc};
    for (size_t k = 0; k < sizeof(fields) / sizeof(fields[0]); ++k)
        *fields[k] = (double*)calloc((size_t)N, sizeof(double));
    return s;
}

void or_destroy(void* h)
{
    or_state* s = (or_state*)h;
    if (!s) return;
    free(s->f); free(s->fn); free(s->n); free(s->ux); free(s->uy); free(s->uz);
    free(s->nbar); free(s->G); free(s->Fx); free(s->Fy); free(s->Fz); free(s->pc);
    free(s->Lx); free(s->Ly); free(s->Lz); free(s->C2f);
    free(s);
}

double or_n0(void* h) { return ((or_state*)h)->n0; }
long or_time(void* h) { return ((or_state*)h)->t; }

/* SplitMix64 (Steele, Lea & Flood 2014), applied once to seed ^ index */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* n(r) = n0 (1 + amp (2U - 1)) with U in [0,1) from the top 53 bits of
 * SplitMix64(seed ^ (offset + index)); populations start at f_eq(n, 0).   */
void or_init_noise(void* h, uint64_t seed, double amp, int64_t offset)
{
    or_state* s = (or_state*)h;
    for (long id = 0; id < s->N; ++id) {
        uint64_t r = splitmix64(seed ^ (uint64_t)(offset + id));
        double U = (double)(r >> 11) * (1.0 / 9007199254740992.0);
        double n = s->n0 * (1.0 + amp * (2.0 * U - 1.0));
        for (int i = 0; i < NV; ++i) s->f[(long)i * s->N + id] = wv[i] * n;
    }
    s->t = 0;
}

/* populations set to the local equilibrium of given n and u fields */
void or_init_fields(void* h, const double* n, const double* ux, const double* uy, const double* uz)
{
    or_state* s = (or_state*)h;
    for (long id = 0; id < s->N; ++id) {
        double u[3] = {ux ? ux[id] : 0.0, uy ? uy[id] : 0.0, uz ? uz[id] : 0.0};
        double feq[NV];
        or_equilibrium(n[id], u, feq);
        for (int i = 0; i < NV; ++i) s->f[(long)i * s->N + id] = feq[i];
    }
    s->t = 0;
}

static void compute_moments(or_state* s)
{
    long N = s->N;
    for (long id = 0; id < N; ++id) {
        double n = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
        for (int i = 0; i < NV; ++i) {
            double fi = s->f[(long)i * N + id];
            n += fi;
            jx += cv[i][0] * fi; jy += cv[i][1] * fi; jz += cv[i][2] * fi;
        }
        s->n[id] = n;
        s->ux[id] = jx / n; s->uy[id] = jy / n; s->uz[id] = jz / n;
    }
}

/* total force density at every node from the current moments */
static void compute_forces(or_state* s, int want_pressure)
{
    long N = s->N;
    for (long id = 0; id < N; ++id) {
        s->Fx[id] = s->n[id] * s->body[0];
        s->Fy[id] = s->n[id] * s->body[1];
        s->Fz[id] = s->n[id] * s->body[2];
    }
    if (s->hs || want_pressure) {
        or_coarse_density(s->g.nx, s->g.ny, s->g.nz, s->g.zper, s->sigma, s->n, s->nbar);
        g2_field(N, s->sigma, s->g2form, s->nbar, s->G);
    }
    if (s->hs) {
        double* hx = (double*)malloc(sizeof(double) * N);
        double* hy = (double*)malloc(sizeof(double) * N);
        double* hz = (double*)malloc(sizeof(double) * N);
        if (s->c2 && !s->C2f) s->C2f = (double*)calloc((size_t)N, sizeof(double));
        hs_force(&s->g, s->sigma, s->kT, s->coupling, s->regularize, s->n, s->ux, s->uy, s->uz,
                 s->G, hx, hy, hz, s->pc, s->c2 ? s->C2f : NULL);
        for (long id = 0; id < N; ++id) { s->Fx[id] += hx[id]; s->Fy[id] += hy[id]; s->Fz[id] += hz[id]; }
        free(hx); free(hy); free(hz);
    } else if (want_pressure) {
        for (long id = 0; id < N; ++id) s->pc[id] = 0.0;
    }
    if (s->tail) tail_force(&s->g, s->sigma, s->eps, s->rcut, s->n, s->Fx, s->Fy, s->Fz);
}

/* one forward-Euler LB update: collide every node, push to r + c_i,
 * halfway bounce-back at the walls (the population returns reversed)     */
static void collide_stream(or_state* s)
{
    long N = s->N;
    const geom* g = &s->g;
#pragma omp parallel for schedule(static)
    for (long id = 0; id < N; ++id) {
        int x = (int)(id % g->nx), y = (int)((id / g->nx) % g->ny), z = (int)(id / ((long)g->nx * g->ny));
        double f[NV], fo[NV], F[3] = {s->Fx[id], s->Fy[id], s->Fz[id]};
        for (int i = 0; i < NV; ++i) f[i] = s->f[(long)i * N + id];
        or_collide_node(f, F, s->tau, fo);
        if (s->c2 && s->hs) {
            /* second-order Hermite source of the scalar C2, read as the trace
             * of an isotropic C2_ab = C2 delta_ab / 3:
             *   w_i C2 (c_i^2 - 3 kT) / (6 kT^2)                             */
            const double kT = s->kT;
            for (int i = 0; i < NV; ++i) {
                double c2i = (double)(cv[i][0] * cv[i][0] + cv[i][1] * cv[i][1] + cv[i][2] * cv[i][2]);
                fo[i] += wv[i] * s->C2f[id] * (c2i - 3.0 * kT) / (6.0 * kT * kT);
            }
        }
        for (int i = 0; i < NV; ++i) {
            long t = node_at(g, x + cv[i][0], y + cv[i][1], z + cv[i][2]);
            if (t < 0) s->fn[(long)opp[i] * N + id] = fo[i];
            else s->fn[(long)i * N + t] = fo[i];
        }
    }
    double* tmp = s->f; s->f = s->fn; s->fn = tmp;
}

/* Collision and streaming with velocity-shifted (second-order) forcing, for
 * comparison with the paper's first-order source: the equilibrium takes
 * u = (j + F/2)/n and the source is
 *   (1 - 1/(2 tau)) w_i [ (c_i - u).F / c_s^2 + (c_i.u)(c_i.F) / c_s^4 ],
 * with F the force of the step (from the unshifted moments).              */
static void collide_stream_shifted(or_state* s)
{
    long N = s->N;
    const geom* g = &s->g;
    const double cs2 = 1.0 / 3.0, a = 1.0 - 0.5 / s->tau;
#pragma omp parallel for schedule(static)
    for (long id = 0; id < N; ++id) {
        int x = (int)(id % g->nx), y = (int)((id / g->nx) % g->ny), z = (int)(id / ((long)g->nx * g->ny));
        double f[NV], fo[NV], feq[NV], F[3] = {s->Fx[id], s->Fy[id], s->Fz[id]};
        double n = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < NV; ++i) {
            f[i] = s->f[(long)i * N + id];
            n += f[i];
            for (int c = 0; c < 3; ++c) j[c] += cv[i][c] * f[i];
        }
        double u[3] = {(j[0] + 0.5 * F[0]) / n, (j[1] + 0.5 * F[1]) / n, (j[2] + 0.5 * F[2]) / n};
        or_equilibrium(n, u, feq);
        for (int i = 0; i < NV; ++i) {
            double cu = cv[i][0] * u[0] + cv[i][1] * u[1] + cv[i][2] * u[2];
            double cF = cv[i][0] * F[0] + cv[i][1] * F[1] + cv[i][2] * F[2];
            double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
            fo[i] = f[i] - (f[i] - feq[i]) / s->tau + a * wv[i] * ((cF - uF) / cs2 + cu * cF / (cs2 * cs2));
        }
        for (int i = 0; i < NV; ++i) {
            long t = node_at(g, x + cv[i][0], y + cv[i][1], z + cv[i][2]);
            if (t < 0) s->fn[(long)opp[i] * N + id] = fo[i];
            else s->fn[(long)i * N + t] = fo[i];
        }
    }
    double* tmp = s->f; s->f = s->fn; s->fn = tmp;
}

/* steps with the velocity-shifted forcing. Reading: the force is evaluated
 * from the moments n, u = j/n of the pre-collision populations (as in the
 * paper's scheme), which keeps the step explicit when the force depends on
 * u (the density-current term of Eq. LBHS); only the equilibrium velocity
 * (j + F/2)/n and the source are shifted. -1 (nothing done) with the energy
 * source of Eq. C2eq on, which this variant does not add.                  */
int or_step_shifted(void* h, long nsteps)
{
    or_state* s = (or_state*)h;
    if (s->c2) return -1;
    for (long k = 0; k < nsteps; ++k) {
        compute_moments(s);
        compute_forces(s, 0);
        collide_stream_shifted(s);
        s->t += 1;
    }
    s->lag_ok = 0;
    return 0;
}

/* switch the energy source of Eq. C2eq (constant T) on or off */
void or_set_c2(void* h, int on) { ((or_state*)h)->c2 = on; }

/* the C2 field of the current state (NULL-safe: zeros when the source is off) */
void or_c2_field(void* h, double* out)
{
    or_state* s = (or_state*)h;
    int was = s->c2;
    s->c2 = 1;
    compute_moments(s);
    compute_forces(s, 0);
    for (long id = 0; id < s->N; ++id) out[id] = s->hs ? s->C2f[id] : 0.0;
    s->c2 = was;
}

void or_step(void* h, long nsteps)
{
    or_state* s = (or_state*)h;
    for (long k = 0; k < nsteps; ++k) {
        compute_moments(s);
        compute_forces(s, 0);
        collide_stream(s);
        s->t += 1;
    }
    s->lag_ok = 0;
}

/* Lagged-force variant of the step: the collision at step t uses the force
 * computed from the moments of step t - 1 (the first step after plain steps
 * or creation uses the current one). Same equilibrium, source and streaming;
 * a steady state of the plain step is a steady state of this one.          */
void or_step_lagged(void* h, long nsteps)
{
    or_state* s = (or_state*)h;
    long N = s->N;
    if (!s->Lx) {
        s->Lx = (double*)calloc((size_t)N, sizeof(double));
        s->Ly = (double*)calloc((size_t)N, sizeof(double));
        s->Lz = (double*)calloc((size_t)N, sizeof(double));
    }
    for (long k = 0; k < nsteps; ++k) {
        compute_moments(s);
        compute_forces(s, 0);                  /* F(t) */
        if (!s->lag_ok) {
            memcpy(s->Lx, s->Fx, sizeof(double) * N);
            memcpy(s->Ly, s->Fy, sizeof(double) * N);
            memcpy(s->Lz, s->Fz, sizeof(double) * N);
            s->lag_ok = 1;
        }
        /* collide with the lagged force, keep F(t) for the next step */
        double* t;
        t = s->Fx; s->Fx = s->Lx; s->Lx = t;
        t = s->Fy; s->Fy = s->Ly; s->Ly = t;
        t = s->Fz; s->Fz = s->Lz; s->Lz = t;
        collide_stream(s);
        s->t += 1;
    }
}

/* moments of the current populations; p = kT n + collisional static part.
 * Any output may be NULL.                                                  */
void or_moments(void* h, double* n, double* ux, double* uy, double* uz, double* p)
{
    or_state* s = (or_state*)h;
    compute_moments(s);
    long N = s->N;
    if (p) {
        compute_forces(s, 1);
        for (long id = 0; id < N; ++id) p[id] = s->kT * s->n[id] + s->pc[id];
    }
    for (long id = 0; id < N; ++id) {
        if (n) n[id] = s->n[id];
        if (ux) ux[id] = s->ux[id];
        if (uy) uy[id] = s->uy[id];
        if (uz) uz[id] = s->uz[id];
    }
}

/* total force density (body + hard sphere + tail) of the current state,
 * and the g2 field it used                                                 */
void or_forces(void* h, double* Fx, double* Fy, double* Fz, double* G)
{
    or_state* s = (or_state*)h;
    compute_moments(s);
    compute_forces(s, 1);
    for (long id = 0; id < s->N; ++id) {
        Fx[id] = s->Fx[id]; Fy[id] = s->Fy[id]; Fz[id] = s->Fz[id];
        if (G) G[id] = s->G[id];
    }
}

/* x,y-averaged density and streaming velocity profiles n(z), u_x(z) */
void or_profiles(void* h, double* nz_out, double* ux_out)
{
    or_state* s = (or_state*)h;
    compute_moments(s);
    long A = (long)s->g.nx * s->g.ny;
    for (int z = 0; z < s->g.nz; ++z) {
        double a = 0.0, b = 0.0;
        for (long k = 0; k < A; ++k) { a += s->n[z * A + k]; b += s->ux[z * A + k]; }
        nz_out[z] = a / A;
        ux_out[z] = b / A;
    }
}

/* total mass and momentum */
void or_totals(void* h, double* out4)
{
    or_state* s = (or_state*)h;
    long N = s->N;
    out4[0] = out4[1] = out4[2] = out4[3] = 0.0;
    for (long id = 0; id < N; ++id)
        for (int i = 0; i < NV; ++i) {
            double fi = s->f[(long)i * N + id];
            out4[0] += fi;
            out4[1] += cv[i][0] * fi; out4[2] += cv[i][1] * fi; out4[3] += cv[i][2] * fi;
        }
}

/* copy of the populations f[i][id] (NV x N, the layout of the state) */
void or_get_pops(void* h, double* out)
{
    or_state* s = (or_state*)h;
    memcpy(out, s->f, sizeof(double) * (size_t)NV * s->N);
}

/* replace the populations (same layout); the step counter is kept */
void or_set_pops(void* h, const double* in)
{
    or_state* s = (or_state*)h;
    memcpy(s->f, in, sizeof(double) * (size_t)NV * s->N);
    s->lag_ok = 0;
}

/* ------------------------------------------------------------------------- */
/* stateless entry points for field-level pins                               */
/* ------------------------------------------------------------------------- */

/* hard-sphere force and g2 field of given n, u fields (u may be NULL = 0) */
void or_hs_force_fields(int nx, int ny, int nz, int zper, int sigma, int coupling, int regularize,
                        int g2form, const double* n, const double* ux, const double* uy,
                        const double* uz, double* Fx, double* Fy, double* Fz, double* G, double* pc)
{
    geom g = {nx, ny, nz, zper};
    long N = (long)nx * ny * nz;
    double* zero = (double*)calloc((size_t)N, sizeof(double));
    double* nbar = (double*)malloc(sizeof(double) * N);
    double* Gl = G ? G : (double*)malloc(sizeof(double) * N);
    or_coarse_density(nx, ny, nz, zper, sigma, n, nbar);
    g2_field(N, sigma, g2form, nbar, Gl);
    hs_force(&g, sigma, 1.0 / 3.0, coupling, regularize, n, ux ? ux : zero, uy ? uy : zero,
             uz ? uz : zero, Gl, Fx, Fy, Fz, pc, NULL);
    if (!G) free(Gl);
    free(nbar);
    free(zero);
}

/* attractive tail force of a given n field */
void or_tail_force_field(int nx, int ny, int nz, int zper, int sigma, double eps, double rcut,
                         const double* n, double* Fx, double* Fy, double* Fz)
{
    geom g = {nx, ny, nz, zper};
    long N = (long)nx * ny * nz;
    for (long i = 0; i < N; ++i) Fx[i] = Fy[i] = Fz[i] = 0.0;
    tail_force(&g, sigma, eps, rcut, n, Fx, Fy, Fz);
}
