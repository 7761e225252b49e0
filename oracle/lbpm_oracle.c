/*
 * FP64 CPU oracle for the two-fluid color-gradient lattice Boltzmann step.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library. The product path (the
 * CUDA library and its Python binding) never links, imports or calls it, and
 * the two share no code, headers, tables or constant generators.
 *
 * The oracle is deliberately plain: fp64 throughout, a pore-site list, and the
 * canonical two-array "push" form of streaming (f_new[x + xi_q] = f*_q(x)).
 * Each timestep follows the paper's model in its own order:
 *
 *   1. phase field        phi = (Na - Nb) / (Na + Nb)           Sec. 3.1
 *   2. color gradient     C = grad(phi), solids give phi_s       Sec. 3.1, Eq. phi_s (Sec. 3.2)
 *   3. macroscopic        rho, j (and u = j / rho0)              Sec. 3.1 (MRT momentum LBE)
 *   4. relaxation rates   from the kinematic viscosity           Sec. 3.1
 *   5. equilibrium moments, with the alpha|C| terms              Sec. 3.1 (m1, m9, m11, m13-15)
 *   6. MRT collision + body force                                 Sec. 3.1 (MRT LBE)
 *   7. recoloring of the two D3Q7 component distributions         Eqs. LBE-mass-a, LBE-mass-b
 *   8. streaming with halfway bounce-back at solid voxels
 *   9. optional reservoir slabs at the z faces (unsteady protocol, Sec. 4.1)
 *
 * Readings taken where the paper is silent or garbled (each is listed, with
 * its reason, in the design notes):
 *   - sign order of xi inside each group of Eq. d3q19 (table XI below);
 *   - m1^eq = -11 rho + 19 j.j/rho0 - alpha|C| (the printed m1 line drops the
 *     -11 rho and the factor 19 of d'Humieres' energy moment);
 *   - the non-alpha equilibria are d'Humieres' incompressible ones;
 *   - s_nu = 1/tau on m1, m2, m9..m15; s_q = s_m = 8(2 - s_nu)/(8 - s_nu) on
 *     m4, m6, m8, m16..m18; tau = tau_b + (tau_a - tau_b)(1 + phi)/2;
 *   - the color gradient is the lattice stencil C = sum_q 18 t_q xi_q phi(x+xi_q)
 *     (unit face weights, half edge weights), which is 6 grad(phi) for smooth
 *     phi: with the printed alpha|C|/2 stress terms this is the scaling under
 *     which the paper's sigma_ab = 6 alpha holds;
 *   - n = C/|C|, and n = 0 when |C| = 0;
 *   - u = j / rho0 in the equilibria; the reported velocity adds F/2;
 *   - p = rho / 3; rho0 = 1;
 *   - phi = 0 where Na + Nb <= 0;
 *   - off-domain neighbours on a non-periodic axis are solid with phi_s = 0;
 *   - initial state: Na = (1+phi0)/2, Nb = (1-phi0)/2, A_q = w_q Na,
 *     B_q = w_q Nb, f_q = t_q (rho = 1, u = 0); the step counter starts at 0;
 *   - reservoir slabs (Sec. 4.1 names pressure reservoirs at inlet and
 *     outlet without giving a scheme): after streaming, the sites with
 *     z < 4 are reset to f = t_q rho_in, A = w_q, B = 0 and the sites with
 *     z >= nz - 4 to f = t_q rho_out, A = 0, B = w_q;
 *   - pressure boundary (reservoir_z = 2; Sec. 4.1 cites Zou and He's
 *     scheme for constant inlet / outlet pressure): after streaming (and on
 *     the initial state), at every pore site of the face z = 0 (density
 *     rho_in) or z = nz - 1 (rho_out), the populations entering from outside
 *     are rebuilt so that the site has that density and no tangential
 *     velocity, by bouncing back their non-equilibrium parts: with n the
 *     inward normal, S0 the sum over c.n = 0 and S_out the sum over
 *     c.n = -1, u_n = 1 - (S0 + 2 S_out) / rho and, for each entering q,
 *     f_q = f_qbar + 2 t_q rho u_n (c_q.n) / c_s^2 - c_t N_t, which is
 *     rho u_n / 3 for the normal and rho u_n / 6 for the four edges, with
 *     N_t = (1/2) sum_{c.n = 0} c_t f for t = x, y. The
 *     entering component population is the reservoir fluid's equilibrium at
 *     the face velocity: A = w rho_in (1 + 4.5 u_z) and B = 0 at the inlet,
 *     B = w rho_out (1 - 4.5 u_z) and A = 0 at the outlet;
 *   - flux inlet (reservoir_z = 3; Sec. 4.1's flux condition sets a total
 *     volumetric flow rate across the inlet): the inlet is a pressure face
 *     whose uniform density is chosen at every step so that the face
 *     velocities u_n = 1 - K_s / rho of its sites (K_s = S0 + 2 S_out) sum to
 *     the prescribed flux Q: rho = sum_s K_s / (n_in - Q); the outlet keeps
 *     the pressure rho_out.
 *
 * Parity status: every function here is pinned by the tests against closed
 * forms, physics or an independent dense implementation. The reservoir reset
 * is pinned by the exact reset state at every slab site after each step and
 * by the closed-form steady state it drives when both reservoirs have one
 * density (rest at that density, component densities exactly linear along a
 * walled duct between the slabs, with alpha = beta = 0); the pressure-driven
 * flow between different reservoir densities has no closed form (an entrance
 * region of the order of the duct width) and is checked for a monotonically
 * rising saturation and an advancing displacement front. The component
 * population entering at a pressure face (the reservoir fluid's equilibrium at
 * the face velocity) is pinned by a closed form: in a body-force-driven duct
 * between two faces at the same density, the total component density stays
 * that density at every site and carries the momentum lattice's mass flux.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q19 19
#define Q7 7
#define RHO0 1.0
#define GRAD_WEIGHT 18.0   /* C = 18 sum_q t_q xi_q phi(x + xi_q) */
#define RESERVOIR_DEPTH 4
#define NMEAS 30

/* D3Q19 velocity set, Eq. d3q19: rest, faces (q = 1..6), xy edges (7..10),
 * xz edges (11..14), yz edges (15..18). Opposites are adjacent pairs. */
static const int XI[Q19][3] = {
    {0, 0, 0},
    {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},  {-1, 1, 0},
    {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},
    {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};

/* D3Q19 weights t_q (c_s^2 = 1/3) and D3Q7 weights w_q (c_s^2 = 2/9), Sec. 3.1 */
static double T19[Q19];
static double W7[Q7];
static double M[Q19][Q19];     /* M[k][q]: moment k of distribution q */
static double MINV[Q19][Q19];  /* MINV[q][k] */
static int tables_ready = 0;

static int opposite(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }

/* d'Humieres et al. (2002) moment polynomials, ordered m0..m18 with
 * m13 = p_xy, m14 = p_yz, m15 = p_xz as the paper's equilibria imply. */
static double moment_poly(int k, const int c[3]) {
    const double x = c[0], y = c[1], z = c[2];
    const double c2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return 19.0 * c2 - 30.0;
    case 2: return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
    case 3: return x;
    case 4: return (5.0 * c2 - 9.0) * x;
    case 5: return y;
    case 6: return (5.0 * c2 - 9.0) * y;
    case 7: return z;
    case 8: return (5.0 * c2 - 9.0) * z;
    case 9: return 3.0 * x * x - c2;
    case 10: return (3.0 * c2 - 5.0) * (3.0 * x * x - c2);
    case 11: return y * y - z * z;
    case 12: return (3.0 * c2 - 5.0) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return (y * y - z * z) * x;
    case 17: return (z * z - x * x) * y;
    case 18: return (x * x - y * y) * z;
    }
    return 0.0;
}

static void build_tables(void) {
    if (tables_ready) return;
    T19[0] = 1.0 / 3.0;
    for (int q = 1; q <= 6; ++q) T19[q] = 1.0 / 18.0;
    for (int q = 7; q < Q19; ++q) T19[q] = 1.0 / 36.0;
    W7[0] = 1.0 / 3.0;
    for (int q = 1; q < Q7; ++q) W7[q] = 1.0 / 9.0;
    for (int k = 0; k < Q19; ++k)
        for (int q = 0; q < Q19; ++q) M[k][q] = moment_poly(k, XI[q]);
    /* rows are orthogonal, so M^-1 = M^T diag(1 / |row_k|^2) */
    for (int k = 0; k < Q19; ++k) {
        double nrm = 0.0;
        for (int q = 0; q < Q19; ++q) nrm += M[k][q] * M[k][q];
        for (int q = 0; q < Q19; ++q) MINV[q][k] = M[k][q] / nrm;
    }
    tables_ready = 1;
}

/* max |M * MINV - I| (should be round-off) */
double orc_lattice_check(void) {
    build_tables();
    double err = 0.0;
    for (int i = 0; i < Q19; ++i)
        for (int j = 0; j < Q19; ++j) {
            double s = 0.0;
            for (int q = 0; q < Q19; ++q) s += M[i][q] * MINV[q][j];
            double e = fabs(s - (i == j ? 1.0 : 0.0));
            if (e > err) err = e;
        }
    return err;
}

void orc_tables(double* xi, double* t19, double* w7, double* m, double* minv) {
    build_tables();
    for (int q = 0; q < Q19; ++q) {
        for (int a = 0; a < 3; ++a) xi[3 * q + a] = XI[q][a];
        t19[q] = T19[q];
    }
    for (int q = 0; q < Q7; ++q) w7[q] = W7[q];
    for (int k = 0; k < Q19; ++k)
        for (int q = 0; q < Q19; ++q) {
            m[k * Q19 + q] = M[k][q];
            minv[q * Q19 + k] = MINV[q][k];
        }
}

static int n_threads = 1;
void orc_set_threads(int n) { n_threads = n < 1 ? 1 : n; }
int orc_get_threads(void) { return n_threads; }
int orc_have_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

/* ------------------------------------------------------------------------ */
/* single-site operators (Sec. 3.1)                                          */
/* ------------------------------------------------------------------------ */

/* rate_mode 0: d'Humieres rates from tau; 1: every non-conserved rate 1/tau */
static void relaxation_rates(double tau, int rate_mode, double s[Q19]) {
    const double s_nu = 1.0 / tau;
    const double s_m = (rate_mode == 1) ? s_nu : 8.0 * (2.0 - s_nu) / (8.0 - s_nu);
    for (int k = 0; k < Q19; ++k) s[k] = s_nu;
    s[0] = s[3] = s[5] = s[7] = 0.0; /* conserved: rho, j */
    s[4] = s[6] = s[8] = s_m;
    s[16] = s[17] = s[18] = s_m;
}

static void equilibrium_moments(double rho, const double j[3], double alpha,
                                const double C[3], double meq[Q19]) {
    const double jx = j[0], jy = j[1], jz = j[2];
    const double jj = (jx * jx + jy * jy + jz * jz) / RHO0;
    const double cmag = sqrt(C[0] * C[0] + C[1] * C[1] + C[2] * C[2]);
    double nx = 0.0, ny = 0.0, nz = 0.0;
    if (cmag > 0.0) {
        nx = C[0] / cmag;
        ny = C[1] / cmag;
        nz = C[2] / cmag;
    }
    const double ac = alpha * cmag;
    meq[0] = rho;
    meq[1] = -11.0 * rho + 19.0 * jj - ac;
    meq[2] = 3.0 * rho - 5.5 * jj;
    meq[3] = jx;
    meq[4] = -2.0 / 3.0 * jx;
    meq[5] = jy;
    meq[6] = -2.0 / 3.0 * jy;
    meq[7] = jz;
    meq[8] = -2.0 / 3.0 * jz;
    meq[9] = (2.0 * jx * jx - jy * jy - jz * jz) / RHO0 + 0.5 * ac * (2.0 * nx * nx - ny * ny - nz * nz);
    meq[10] = -0.5 * (2.0 * jx * jx - jy * jy - jz * jz) / RHO0;
    meq[11] = (jy * jy - jz * jz) / RHO0 + 0.5 * ac * (ny * ny - nz * nz);
    meq[12] = -0.5 * (jy * jy - jz * jz) / RHO0;
    meq[13] = jx * jy / RHO0 + 0.5 * ac * nx * ny;
    meq[14] = jy * jz / RHO0 + 0.5 * ac * ny * nz;
    meq[15] = jx * jz / RHO0 + 0.5 * ac * nx * nz;
    meq[16] = 0.0;
    meq[17] = 0.0;
    meq[18] = 0.0;
}

/* MRT collision with the interfacial perturbation and the body force:
 * f*_q = f_q + sum_k MINV[q][k] s_k (m_k^eq - m_k) + t_q xi_q . F / c_s^2 */
void orc_collide_site(const double* f, const double* C, double tau, double alpha,
                      const double* F, int rate_mode, double* fout) {
    build_tables();
    double m[Q19], meq[Q19], s[Q19], dm[Q19];
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < Q19; ++q) {
        rho += f[q];
        for (int a = 0; a < 3; ++a) j[a] += XI[q][a] * f[q];
    }
    for (int k = 0; k < Q19; ++k) {
        double acc = 0.0;
        for (int q = 0; q < Q19; ++q) acc += M[k][q] * f[q];
        m[k] = acc;
    }
    equilibrium_moments(rho, j, alpha, C, meq);
    relaxation_rates(tau, rate_mode, s);
    for (int k = 0; k < Q19; ++k) dm[k] = s[k] * (meq[k] - m[k]);
    for (int q = 0; q < Q19; ++q) {
        double acc = 0.0;
        for (int k = 0; k < Q19; ++k) acc += MINV[q][k] * dm[k];
        const double xf = XI[q][0] * F[0] + XI[q][1] * F[1] + XI[q][2] * F[2];
        fout[q] = f[q] + acc + 3.0 * T19[q] * xf;
    }
}

/* Recoloring, Eqs. LBE-mass-a and LBE-mass-b (post-collision, pre-streaming) */
void orc_recolor_site(double Na, double Nb, const double* u, const double* C, double beta,
                      double* A, double* B) {
    build_tables();
    const double N = Na + Nb;
    const double cmag = sqrt(C[0] * C[0] + C[1] * C[1] + C[2] * C[2]);
    double n[3] = {0.0, 0.0, 0.0};
    if (cmag > 0.0)
        for (int a = 0; a < 3; ++a) n[a] = C[a] / cmag;
    const double fa = (N > 0.0) ? Nb / N : 0.0; /* weight of the A recoloring term */
    const double fb = (N > 0.0) ? Na / N : 0.0;
    for (int q = 0; q < Q7; ++q) {
        const double ux = u[0] * XI[q][0] + u[1] * XI[q][1] + u[2] * XI[q][2];
        const double nx = n[0] * XI[q][0] + n[1] * XI[q][1] + n[2] * XI[q][2];
        A[q] = W7[q] * Na * (1.0 + 4.5 * ux + beta * fa * nx);
        B[q] = W7[q] * Nb * (1.0 + 4.5 * ux - beta * fb * nx);
    }
}

/* ------------------------------------------------------------------------ */
/* the domain                                                                */
/* ------------------------------------------------------------------------ */

typedef struct orc {
    int nx, ny, nz;
    int periodic[3];
    long long V, N;
    int32_t* vox_site;  /* [V]: site id or -1 (solid) */
    int64_t* site_vox;  /* [N] */
    int32_t* sx;        /* [N] site coordinates */
    int32_t* sy;
    int32_t* sz;
    int32_t* nbr;       /* [18][N]: neighbour site along xi_q (q = 1..18), -1 if none */
    double* phis;       /* [V]: wetting affinity phi_s of solid voxels */
    double tau_a, tau_b, alpha, beta, F[3];
    int reservoir_z;
    double rho_in, rho_out;
    double flux_in;
    int rate_mode;
    double *f, *fn;     /* [N][19] */
    double *A, *An;     /* [N][7] */
    double *B, *Bn;
    double* phi;        /* [N] */
    long long step;
} orc_t;

static long long vox_index(const orc_t* o, int x, int y, int z) {
    return (long long)x + (long long)o->nx * ((long long)y + (long long)o->ny * z);
}

/* Wrap (x, y, z) into the domain; returns 0 if it leaves a non-periodic axis. */
static int wrap(const orc_t* o, int* x, int* y, int* z) {
    int c[3] = {*x, *y, *z};
    const int L[3] = {o->nx, o->ny, o->nz};
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0 || c[a] >= L[a]) {
            if (!o->periodic[a]) return 0;
            c[a] = ((c[a] % L[a]) + L[a]) % L[a];
        }
    }
    *x = c[0];
    *y = c[1];
    *z = c[2];
    return 1;
}

orc_t* orc_create(int nx, int ny, int nz, const uint16_t* labels, const float* affinity,
                  const int* periodic) {
    build_tables();
    orc_t* o = (orc_t*)calloc(1, sizeof(orc_t));
    o->nx = nx;
    o->ny = ny;
    o->nz = nz;
    for (int a = 0; a < 3; ++a) o->periodic[a] = periodic[a] ? 1 : 0;
    o->V = (long long)nx * ny * nz;
    o->vox_site = (int32_t*)malloc(sizeof(int32_t) * o->V);
    o->phis = (double*)malloc(sizeof(double) * o->V);
    /* lexicographic compaction: x fastest, then y, then z */
    long long n = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long long v = vox_index(o, x, y, z);
                if (labels[v] == 0) {
                    o->vox_site[v] = (int32_t)n++;
                    o->phis[v] = 0.0;
                } else {
                    o->vox_site[v] = -1;
                    o->phis[v] = affinity ? (double)affinity[v] : 0.0;
                }
            }
    o->N = n;
    const long long N = o->N;
    o->site_vox = (int64_t*)malloc(sizeof(int64_t) * (N ? N : 1));
    o->sx = (int32_t*)malloc(sizeof(int32_t) * (N ? N : 1));
    o->sy = (int32_t*)malloc(sizeof(int32_t) * (N ? N : 1));
    o->sz = (int32_t*)malloc(sizeof(int32_t) * (N ? N : 1));
    o->nbr = (int32_t*)malloc(sizeof(int32_t) * 18 * (N ? N : 1));
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long long v = vox_index(o, x, y, z);
                const int32_t s = o->vox_site[v];
                if (s < 0) continue;
                o->site_vox[s] = v;
                o->sx[s] = x;
                o->sy[s] = y;
                o->sz[s] = z;
                for (int q = 1; q < Q19; ++q) {
                    int xx = x + XI[q][0], yy = y + XI[q][1], zz = z + XI[q][2];
                    int32_t t = -1;
                    if (wrap(o, &xx, &yy, &zz)) t = o->vox_site[vox_index(o, xx, yy, zz)];
                    o->nbr[(long long)(q - 1) * N + s] = t;
                }
            }
    o->f = (double*)calloc((size_t)(N ? N : 1) * Q19, sizeof(double));
    o->fn = (double*)calloc((size_t)(N ? N : 1) * Q19, sizeof(double));
    o->A = (double*)calloc((size_t)(N ? N : 1) * Q7, sizeof(double));
    o->An = (double*)calloc((size_t)(N ? N : 1) * Q7, sizeof(double));
    o->B = (double*)calloc((size_t)(N ? N : 1) * Q7, sizeof(double));
    o->Bn = (double*)calloc((size_t)(N ? N : 1) * Q7, sizeof(double));
    o->phi = (double*)calloc((size_t)(N ? N : 1), sizeof(double));
    o->tau_a = o->tau_b = 1.0;
    o->rho_in = o->rho_out = 1.0;
    return o;
}

void orc_destroy(orc_t* o) {
    if (!o) return;
    free(o->vox_site); free(o->phis); free(o->site_vox);
    free(o->sx); free(o->sy); free(o->sz); free(o->nbr);
    free(o->f); free(o->fn); free(o->A); free(o->An); free(o->B); free(o->Bn);
    free(o->phi);
    free(o);
}

long long orc_num_sites(const orc_t* o) { return o->N; }
long long orc_step_count(const orc_t* o) { return o->step; }

void orc_get_index(const orc_t* o, int64_t* site_vox, int32_t* nbr) {
    memcpy(site_vox, o->site_vox, sizeof(int64_t) * o->N);
    memcpy(nbr, o->nbr, sizeof(int32_t) * 18 * o->N);
}

void orc_set_params(orc_t* o, double tau_a, double tau_b, double alpha, double beta,
                    const double* F, int reservoir_z, double rho_in, double rho_out, double flux_in) {
    o->tau_a = tau_a;
    o->tau_b = tau_b;
    o->alpha = alpha;
    o->beta = beta;
    for (int a = 0; a < 3; ++a) o->F[a] = F[a];
    o->reservoir_z = reservoir_z;
    o->rho_in = rho_in;
    o->rho_out = rho_out;
    o->flux_in = flux_in;
}

void orc_set_rate_mode(orc_t* o, int mode) { o->rate_mode = mode; }

static void reset_reservoirs(orc_t* o, double* f, double* A, double* B) {
    if (o->reservoir_z != 1) return;
    for (long long n = 0; n < o->N; ++n) {
        const int z = o->sz[n];
        int side = 0;
        if (z < RESERVOIR_DEPTH) side = 1;
        else if (z >= o->nz - RESERVOIR_DEPTH) side = 2;
        if (!side) continue;
        const double rho = side == 1 ? o->rho_in : o->rho_out;
        for (int q = 0; q < Q19; ++q) f[n * Q19 + q] = T19[q] * rho;
        for (int q = 0; q < Q7; ++q) {
            A[n * Q7 + q] = side == 1 ? W7[q] : 0.0;
            B[n * Q7 + q] = side == 1 ? 0.0 : W7[q];
        }
    }
}

/* Pressure boundary at the z faces (reservoir_z == 2), on a state in
 * canonical post-streaming form. */
static void pressure_faces(orc_t* o, double* f, double* A, double* B) {
    if (o->reservoir_z != 2 && o->reservoir_z != 3) return;
    double rho_in = o->rho_in;
    if (o->reservoir_z == 3) {
        /* flux inlet: the uniform inlet density whose Zou-He face velocities
         * u_n = 1 - K_s / rho sum to the flux, K_s = S0 + 2 S_out of site s */
        double K = 0.0;
        long long n_in = 0;
        for (long long n = 0; n < o->N; ++n) {
            if (o->sz[n] != 0) continue;
            const double* g = f + n * Q19;
            for (int q = 0; q < Q19; ++q) {
                if (XI[q][2] == 0) K += g[q];
                else if (XI[q][2] < 0) K += 2.0 * g[q];
            }
            ++n_in;
        }
        if (n_in > 0) rho_in = K / ((double)n_in - o->flux_in);
    }
    for (long long n = 0; n < o->N; ++n) {
        const int z = o->sz[n];
        int nrm;                                   /* inward normal along z */
        double rho;
        if (z == 0) { nrm = 1; rho = rho_in; }
        else if (z == o->nz - 1) { nrm = -1; rho = o->rho_out; }
        else continue;
        double* g = f + n * Q19;
        double s0 = 0.0, sout = 0.0, Nt[2] = {0.0, 0.0};
        for (int q = 0; q < Q19; ++q) {
            const int cn = XI[q][2] * nrm;
            if (cn == 0) {
                s0 += g[q];
                Nt[0] += XI[q][0] * g[q];
                Nt[1] += XI[q][1] * g[q];
            } else if (cn < 0) {
                sout += g[q];
            }
        }
        Nt[0] *= 0.5;
        Nt[1] *= 0.5;
        const double un = 1.0 - (s0 + 2.0 * sout) / rho;
        for (int q = 1; q < Q19; ++q) {
            if (XI[q][2] * nrm <= 0) continue;     /* only the entering directions */
            const int tang = abs(XI[q][0]) + abs(XI[q][1]);
            g[q] = g[opposite(q)] + rho * un * (tang ? 1.0 / 6.0 : 1.0 / 3.0) - XI[q][0] * Nt[0] - XI[q][1] * Nt[1];
        }
        const double uz = nrm * un;
        const int qin = nrm > 0 ? 5 : 6;           /* D3Q7 direction entering the face */
        const double eq = W7[qin] * rho * (1.0 + 4.5 * XI[qin][2] * uz);
        A[n * Q7 + qin] = nrm > 0 ? eq : 0.0;
        B[n * Q7 + qin] = nrm > 0 ? 0.0 : eq;
    }
}

/* Initial state consistent with a phase field phi0 (per voxel; pores read). */
void orc_init_fluids(orc_t* o, const float* phi0) {
    for (long long n = 0; n < o->N; ++n) {
        const double p = phi0[o->site_vox[n]];
        const double Na = 0.5 * (1.0 + p), Nb = 0.5 * (1.0 - p);
        for (int q = 0; q < Q19; ++q) o->f[n * Q19 + q] = T19[q] * RHO0;
        for (int q = 0; q < Q7; ++q) {
            o->A[n * Q7 + q] = W7[q] * Na;
            o->B[n * Q7 + q] = W7[q] * Nb;
        }
    }
    reset_reservoirs(o, o->f, o->A, o->B);
    pressure_faces(o, o->f, o->A, o->B);
    o->step = 0;
}

/* State exchange in canonical population-major order: f[q*N + n]. */
void orc_set_state(orc_t* o, const double* f, const double* A, const double* B, long long step) {
    const long long N = o->N;
    for (long long n = 0; n < N; ++n) {
        for (int q = 0; q < Q19; ++q) o->f[n * Q19 + q] = f[q * N + n];
        for (int q = 0; q < Q7; ++q) {
            o->A[n * Q7 + q] = A[q * N + n];
            o->B[n * Q7 + q] = B[q * N + n];
        }
    }
    o->step = step;
}

void orc_get_state(const orc_t* o, double* f, double* A, double* B) {
    const long long N = o->N;
    for (long long n = 0; n < N; ++n) {
        for (int q = 0; q < Q19; ++q) f[q * N + n] = o->f[n * Q19 + q];
        for (int q = 0; q < Q7; ++q) {
            A[q * N + n] = o->A[n * Q7 + q];
            B[q * N + n] = o->B[n * Q7 + q];
        }
    }
}

/* step 1: phase indicator at every pore site */
static void phase_field(orc_t* o) {
    const long long N = o->N;
#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (long long n = 0; n < N; ++n) {
        double Na = 0.0, Nb = 0.0;
        for (int q = 0; q < Q7; ++q) {
            Na += o->A[n * Q7 + q];
            Nb += o->B[n * Q7 + q];
        }
        const double Nt = Na + Nb;
        o->phi[n] = Nt > 0.0 ? (Na - Nb) / Nt : 0.0;
    }
}

/* phi seen by the gradient stencil at the neighbour of site n along xi_q */
static double phi_neighbour(const orc_t* o, long long n, int q) {
    const int32_t t = o->nbr[(long long)(q - 1) * o->N + n];
    if (t >= 0) return o->phi[t];
    int x = o->sx[n] + XI[q][0], y = o->sy[n] + XI[q][1], z = o->sz[n] + XI[q][2];
    if (!wrap(o, &x, &y, &z)) return 0.0;        /* outside a non-periodic face */
    return o->phis[vox_index(o, x, y, z)];        /* solid: wetting affinity, Eq. phi_s */
}

/* step 2: color gradient at site n (phase field must be current) */
static void color_gradient(const orc_t* o, long long n, double C[3]) {
    C[0] = C[1] = C[2] = 0.0;
    for (int q = 1; q < Q19; ++q) {
        const double p = phi_neighbour(o, n, q);
        for (int a = 0; a < 3; ++a) C[a] += GRAD_WEIGHT * T19[q] * XI[q][a] * p;
    }
}

void orc_phase_gradient(orc_t* o, double* phi, double* C) {
    phase_field(o);
    for (long long n = 0; n < o->N; ++n) {
        double c[3];
        color_gradient(o, n, c);
        phi[n] = o->phi[n];
        for (int a = 0; a < 3; ++a) C[a * o->N + n] = c[a];
    }
}

static void one_step(orc_t* o) {
    const long long N = o->N;
    phase_field(o);
#pragma omp parallel for num_threads(n_threads) schedule(static)
    for (long long n = 0; n < N; ++n) {
        const double* fs = o->f + n * Q19;
        double Na = 0.0, Nb = 0.0;
        for (int q = 0; q < Q7; ++q) {
            Na += o->A[n * Q7 + q];
            Nb += o->B[n * Q7 + q];
        }
        double C[3];
        color_gradient(o, n, C);
        double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < Q19; ++q) {
            rho += fs[q];
            for (int a = 0; a < 3; ++a) j[a] += XI[q][a] * fs[q];
        }
        const double u[3] = {j[0] / RHO0, j[1] / RHO0, j[2] / RHO0};
        const double tau = o->tau_b + (o->tau_a - o->tau_b) * 0.5 * (1.0 + o->phi[n]);
        double fpost[Q19], Apost[Q7], Bpost[Q7];
        orc_collide_site(fs, C, tau, o->alpha, o->F, o->rate_mode, fpost);
        orc_recolor_site(Na, Nb, u, C, o->beta, Apost, Bpost);
        /* step 8: push streaming, halfway bounce-back where the target is not a pore */
        o->fn[n * Q19 + 0] = fpost[0];
        for (int q = 1; q < Q19; ++q) {
            const int32_t t = o->nbr[(long long)(q - 1) * N + n];
            if (t >= 0) o->fn[(long long)t * Q19 + q] = fpost[q];
            else o->fn[n * Q19 + opposite(q)] = fpost[q];
        }
        o->An[n * Q7 + 0] = Apost[0];
        o->Bn[n * Q7 + 0] = Bpost[0];
        for (int q = 1; q < Q7; ++q) {
            const int32_t t = o->nbr[(long long)(q - 1) * N + n];
            if (t >= 0) {
                o->An[(long long)t * Q7 + q] = Apost[q];
                o->Bn[(long long)t * Q7 + q] = Bpost[q];
            } else {
                o->An[n * Q7 + opposite(q)] = Apost[q];
                o->Bn[n * Q7 + opposite(q)] = Bpost[q];
            }
        }
    }
    reset_reservoirs(o, o->fn, o->An, o->Bn);
    pressure_faces(o, o->fn, o->An, o->Bn);
    double* t;
    t = o->f; o->f = o->fn; o->fn = t;
    t = o->A; o->A = o->An; o->An = t;
    t = o->B; o->B = o->Bn; o->Bn = t;
    o->step += 1;
}

void orc_step(orc_t* o, int nsteps) {
    for (int s = 0; s < nsteps; ++s) one_step(o);
}

/* Per-site fields of the current state: phi, pressure p = rho/3, reported u. */
void orc_fields(const orc_t* o, double* phi, double* p, double* u) {
    const long long N = o->N;
    for (long long n = 0; n < N; ++n) {
        double Na = 0.0, Nb = 0.0, rho = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < Q7; ++q) {
            Na += o->A[n * Q7 + q];
            Nb += o->B[n * Q7 + q];
        }
        for (int q = 0; q < Q19; ++q) {
            rho += o->f[n * Q19 + q];
            for (int a = 0; a < 3; ++a) j[a] += XI[q][a] * o->f[n * Q19 + q];
        }
        const double Nt = Na + Nb;
        phi[n] = Nt > 0.0 ? (Na - Nb) / Nt : 0.0;
        p[n] = rho / 3.0;
        for (int a = 0; a < 3; ++a) u[a * N + n] = (j[a] + 0.5 * o->F[a]) / RHO0;
    }
}

/* Basic analysis (Sec. 4 intro) and integral measures (Sec. 3.4, table of
 * integral measures) of the current state, in fp64, summed in site order.
 * Output layout (NMEAS doubles):
 *  0 step, 1 sat_mass, 2 sat_count, 3 mass_a, 4 mass_b, 5 mass_total (sum rho),
 *  6-8 mom_a, 9-11 mom_b, 12-14 flux, 15-17 flux_a, 18-20 flux_b,
 *  21 ke_a, 22 ke_b, 23 p_a, 24 p_b, 25 vol_a, 26 vol_b, 27 Ca, 28 n_sites,
 *  29 status (0 ok, bit 0 a non-finite value, bit 1 a component density below
 *  -1e-2 or a non-positive total density). Small negative component densities
 *  (order 1e-5) occur in valid runs next to interfaces, where a recolored
 *  population can be negative, so they are not flagged. */
void orc_measure(const orc_t* o, double* out) {
    for (int i = 0; i < NMEAS; ++i) out[i] = 0.0;
    const long long N = o->N;
    double sNa = 0, sNb = 0, srho = 0, cnt_a = 0;
    double mom_a[3] = {0, 0, 0}, mom_b[3] = {0, 0, 0};
    double q[3] = {0, 0, 0}, qa[3] = {0, 0, 0}, qb[3] = {0, 0, 0};
    double Ma = 0, Mb = 0, ke_a = 0, ke_b = 0, pa = 0, pb = 0;
    int status = 0;
    for (long long n = 0; n < N; ++n) {
        double Na = 0, Nb = 0, rho = 0, j[3] = {0, 0, 0};
        for (int k = 0; k < Q7; ++k) {
            Na += o->A[n * Q7 + k];
            Nb += o->B[n * Q7 + k];
        }
        for (int k = 0; k < Q19; ++k) {
            const double fv = o->f[n * Q19 + k];
            if (!isfinite(fv)) status |= 1;
            rho += fv;
            for (int a = 0; a < 3; ++a) j[a] += XI[k][a] * fv;
        }
        if (!isfinite(Na) || !isfinite(Nb)) status |= 1;
        const double Nt = Na + Nb;
        if (Na < -1e-2 || Nb < -1e-2 || Nt <= 0.0 || rho <= 0.0) status |= 2;
        const double phi = Nt > 0.0 ? (Na - Nb) / Nt : 0.0;
        double u[3];
        for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * o->F[a]) / RHO0;
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double p = rho / 3.0;
        const double xa = Nt > 0.0 ? Na / Nt : 0.0, xb = Nt > 0.0 ? Nb / Nt : 0.0;
        sNa += Na;
        sNb += Nb;
        srho += rho;
        for (int a = 0; a < 3; ++a) {
            q[a] += u[a];
            qa[a] += xa * u[a];
            qb[a] += xb * u[a];
        }
        if (phi > 0.0) {
            cnt_a += 1.0;
            Ma += rho;
            for (int a = 0; a < 3; ++a) mom_a[a] += rho * u[a];
            ke_a += rho * uu;
            pa += p;
        } else {
            Mb += rho;
            for (int a = 0; a < 3; ++a) mom_b[a] += rho * u[a];
            ke_b += rho * uu;
            pb += p;
        }
    }
    const double V = (double)o->V;
    const double cnt_b = (double)N - cnt_a;
    out[0] = (double)o->step;
    out[1] = (sNa + sNb) > 0 ? sNa / (sNa + sNb) : 0.0;
    out[2] = N > 0 ? cnt_a / (double)N : 0.0;
    out[3] = sNa;
    out[4] = sNb;
    out[5] = srho;
    for (int a = 0; a < 3; ++a) {
        out[6 + a] = mom_a[a];
        out[9 + a] = mom_b[a];
        out[12 + a] = q[a] / V;
        out[15 + a] = qa[a] / V;
        out[18 + a] = qb[a] / V;
    }
    out[21] = ke_a;
    out[22] = ke_b;
    out[23] = cnt_a > 0 ? pa / cnt_a : 0.0;
    out[24] = cnt_b > 0 ? pb / cnt_b : 0.0;
    out[25] = cnt_a;
    out[26] = cnt_b;
    /* total capillary number, Eq. capillary_number, sigma = 6 alpha */
    double ca = 0.0;
    if (o->alpha > 0.0) {
        const double mu_a = RHO0 * (o->tau_a - 0.5) / 3.0, mu_b = RHO0 * (o->tau_b - 0.5) / 3.0;
        double ua = 0.0, ub = 0.0;
        if (Ma > 0) ua = sqrt(mom_a[0] * mom_a[0] + mom_a[1] * mom_a[1] + mom_a[2] * mom_a[2]) / Ma;
        if (Mb > 0) ub = sqrt(mom_b[0] * mom_b[0] + mom_b[1] * mom_b[1] + mom_b[2] * mom_b[2]) / Mb;
        ca = ((cnt_a / V) * mu_a * ua + (cnt_b / V) * mu_b * ub) / (6.0 * o->alpha);
    }
    out[27] = ca;
    out[28] = (double)N;
    out[29] = (double)status;
}
