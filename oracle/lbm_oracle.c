/* Oracle: plain FP64 CPU statement of the D3Q19 lattice Boltzmann method with
 * interpolated bounce-back (IBB) and direct-forcing immersed boundary (IBM)
 * no-slip walls, following Peng et al., arXiv:1906.05448 (Part II), Sec. 2.1
 * (pipe flow: body-force driving, linear IBB on the wall, IBM-U / IBM-B with
 * the Peskin 4-point delta and two extra forcing iterations, Table 1) and
 * Sec. 3.1 (particle-laden decaying turbulence: D3Q19 MRT with d'Humieres
 * rates, quadratic -> linear -> single-node bounce-back fallback, Galilean
 * invariant momentum exchange, Caiazzo refill, Kempe inner-fluid inertia,
 * normal-only soft-sphere collisions, particle release, Table 2).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path. It shares no code
 * with the CUDA library. Everything is done the slow, obvious way: dense
 * 19x19 moment matrices, brute-force geometry, scatter spreading, serial
 * reductions in a fixed order (only the per-cell stream-collide loop runs in
 * OpenMP threads, each cell independent). Compile with -ffp-contract=off.
 *
 * The paper defers every formula to the cited originals; the readings used
 * here are listed beside each function.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19
#define PI 3.14159265358979323846

/* D3Q19 velocity set: rest, 6 axis neighbours, 12 edge neighbours. Opposite
 * directions sit next to each other. */
static const int CV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double WT(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
static int OPP(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

void orc_lattice(int *c, double *w, int *opp)
{
    for (int i = 0; i < Q; i++) {
        for (int d = 0; d < 3; d++) c[3 * i + d] = CV[i][d];
        w[i] = WT(i);
        opp[i] = OPP(i);
    }
}

/* Moment basis of d'Humieres et al. (2002) for D3Q19 (the MRT model named in
 * Sec. 3.1), built by evaluating its 19 polynomials on the velocities:
 * rho, e, eps, jx, qx, jy, qy, jz, qz, 3pxx, 3pixx, pww, piww, pxy, pyz, pxz,
 * mx, my, mz. */
static void moment_matrix(double M[Q][Q])
{
    for (int i = 0; i < Q; i++) {
        double cx = CV[i][0], cy = CV[i][1], cz = CV[i][2];
        double c2 = cx * cx + cy * cy + cz * cz;
        M[0][i] = 1.0;
        M[1][i] = 19.0 * c2 - 30.0;
        M[2][i] = (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
        M[3][i] = cx;
        M[4][i] = (5.0 * c2 - 9.0) * cx;
        M[5][i] = cy;
        M[6][i] = (5.0 * c2 - 9.0) * cy;
        M[7][i] = cz;
        M[8][i] = (5.0 * c2 - 9.0) * cz;
        M[9][i] = 3.0 * cx * cx - c2;
        M[10][i] = (3.0 * c2 - 5.0) * (3.0 * cx * cx - c2);
        M[11][i] = cy * cy - cz * cz;
        M[12][i] = (3.0 * c2 - 5.0) * (cy * cy - cz * cz);
        M[13][i] = cx * cy;
        M[14][i] = cy * cz;
        M[15][i] = cx * cz;
        M[16][i] = (cy * cy - cz * cz) * cx;
        M[17][i] = (cz * cz - cx * cx) * cy;
        M[18][i] = (cx * cx - cy * cy) * cz;
    }
}

void orc_moment_matrix(double *Mout)
{
    double M[Q][Q];
    moment_matrix(M);
    memcpy(Mout, M, sizeof(M));
}

/* The rows are mutually orthogonal, so M^-1 = M^T diag(1/|row|^2). */
static void moment_inverse(double M[Q][Q], double Mi[Q][Q])
{
    for (int k = 0; k < Q; k++) {
        double n2 = 0.0;
        for (int i = 0; i < Q; i++) n2 += M[k][i] * M[k][i];
        for (int i = 0; i < Q; i++) Mi[i][k] = M[k][i] / n2;
    }
}

/* Relaxation rates. SRT: every non-conserved moment relaxes at 1/tau (the
 * single-parameter setting of the pipe solver, Sec. 2.1). DHUMIERES: the
 * multiple rates of d'Humieres et al. (2002) used for the particle-laden
 * runs (Sec. 3.1), with the shear moments at 1/tau. Conserved moments get 0. */
void orc_rates(int set, double tau, double *s)
{
    double om = 1.0 / tau;
    for (int k = 0; k < Q; k++) s[k] = om;
    if (set == ORC_RATES_DHUMIERES) {
        s[1] = 1.19;
        s[2] = 1.4;
        s[4] = s[6] = s[8] = 1.2;
        s[10] = s[12] = 1.4;
        s[16] = s[17] = s[18] = 1.98;
    }
    s[0] = s[3] = s[5] = s[7] = 0.0;
}

/* Second-order equilibrium f_i = w_i rho [1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u]. */
void orc_feq(double rho, const double *u, double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; i++) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        feq[i] = WT(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

/* Guo et al. (2002) forcing term F_i = w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F. */
static void guo_source(const double *u, const double *F, double *Fi)
{
    for (int i = 0; i < Q; i++) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        double s = 0.0;
        for (int d = 0; d < 3; d++) s += (3.0 * (CV[i][d] - u[d]) + 9.0 * cu * CV[i][d]) * F[d];
        Fi[i] = WT(i) * s;
    }
}

/* Pre-collision density and Guo velocity u = (sum f c + F/2) / rho. */
static void moments0(const double *f, const double *F, double *rho, double *u)
{
    double r = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; i++) {
        r += f[i];
        for (int d = 0; d < 3; d++) j[d] += f[i] * CV[i][d];
    }
    *rho = r;
    for (int d = 0; d < 3; d++) u[d] = (j[d] + 0.5 * F[d]) / r;
}

/* MRT collision with Guo forcing in moment space:
 *   m* = m - S (m - m_eq) + (I - S/2) M F_i,   f* = M^-1 m*,
 * with m_eq = M f_eq(rho, u). */
static void collide_mrt(double M[Q][Q], double Mi[Q][Q], const double *s,
                        const double *f, const double *F, double *out)
{
    double rho, u[3], feq[Q], Fi[Q];
    moments0(f, F, &rho, u);
    orc_feq(rho, u, feq);
    guo_source(u, F, Fi);
    double m[Q], meq[Q], mF[Q], ms[Q];
    for (int k = 0; k < Q; k++) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = 0; i < Q; i++) {
            a += M[k][i] * f[i];
            b += M[k][i] * feq[i];
            c += M[k][i] * Fi[i];
        }
        m[k] = a;
        meq[k] = b;
        mF[k] = c;
    }
    for (int k = 0; k < Q; k++) ms[k] = m[k] - s[k] * (m[k] - meq[k]) + (1.0 - 0.5 * s[k]) * mF[k];
    for (int i = 0; i < Q; i++) {
        double a = 0.0;
        for (int k = 0; k < Q; k++) a += Mi[i][k] * ms[k];
        out[i] = a;
    }
}

void orc_collide_mrt(const double *f, const double *F, int set, double tau, double *out)
{
    double M[Q][Q], Mi[Q][Q], s[Q];
    moment_matrix(M);
    moment_inverse(M, Mi);
    orc_rates(set, tau, s);
    collide_mrt(M, Mi, s, f, F, out);
}

/* BGK with Guo forcing, written directly in population space (used to pin
 * the MRT path: equal rates must reduce to this). */
void orc_collide_bgk(const double *f, const double *F, double tau, double *out)
{
    double rho, u[3], feq[Q], Fi[Q];
    moments0(f, F, &rho, u);
    orc_feq(rho, u, feq);
    guo_source(u, F, Fi);
    for (int i = 0; i < Q; i++) out[i] = f[i] - (f[i] - feq[i]) / tau + (1.0 - 0.5 / tau) * Fi[i];
}

/* Peskin (2002) 4-point regularised delta kernel (Sec. 2.1, Sec. 3.1). */
double orc_peskin_phi(double r)
{
    double a = fabs(r);
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
    return 0.0;
}

/* ------------------------------------------------------------------------ */

typedef struct {
    long long cell;
    int dir, scheme, pid;
    double q;
} link_t;

struct orc_sim {
    int nx, ny, nz;
    long long N;
    double tau, Fext[3];
    int rates;
    double M[Q][Q], Mi[Q][Q], s[Q];
    double *f, *fn;          /* post-collision populations (19*N) and the next buffer */
    double *fibm;            /* IBM force of the last collision (3*N) */
    unsigned char *solid;    /* geometry: cell inside a particle or outside the pipe */
    int *owner;              /* particle owning a solid cell (-1: pipe or none) */
    long long *link_start;   /* first link of a cell, -1 if none (links sorted by cell) */
    link_t *links;
    long long nlinks, cap_links;
    /* pipe */
    int has_pipe;
    double pipe_R, pipe_cx, pipe_cy;
    /* plane channel (test geometry of the bounce-back schemes) */
    int has_chan, chan_chain;
    double chan_ylo, chan_yhi, chan_u[2];
    /* particles (FP64) */
    int np, fixed;
    double dens;
    double *X, *U, *W, *R, *mass, *inertia;
    double *Fh, *Th, *Fprev, *Tprev, *Fc;
    int *has_prev;
    double *Iu, *Ir;          /* Kempe inner integrals of u and (x-X) x u */
    /* markers (IBM) */
    long long nm;
    double *mX, *mU, *mF, *mFacc, *mdV, *mUnit;
    int *mpid;
    double resid[3];
    int armed_bc;
    long long step;
};

static int nthreads_req = 0;
void orc_set_threads(int n) { nthreads_req = n; }
int orc_get_threads(void)
{
#ifdef _OPENMP
    return nthreads_req > 0 ? nthreads_req : omp_get_max_threads();
#else
    return 1;
#endif
}

static inline int wrapi(int a, int n) { a %= n; return a < 0 ? a + n : a; }
static inline long long cidx(const orc_sim *S, int x, int y, int z)
{
    return (long long)wrapi(x, S->nx) + (long long)S->nx * ((long long)wrapi(y, S->ny) + (long long)S->ny * wrapi(z, S->nz));
}
static inline void ccoord(const orc_sim *S, long long idx, int *x, int *y, int *z)
{
    *x = (int)(idx % S->nx);
    *y = (int)((idx / S->nx) % S->ny);
    *z = (int)(idx / ((long long)S->nx * S->ny));
}
/* minimum-image displacement along one periodic axis of length n */
static inline double mimg(double d, int n)
{
    if (d > 0.5 * n) d -= n;
    else if (d < -0.5 * n) d += n;
    return d;
}

/* The driving body force acts on the fluid only: cells inside a particle or
 * outside the pipe get none (for IBM this keeps the virtual fluid there
 * undriven). */
static double fext_at(const orc_sim *S, long long c, int d) { return S->solid[c] ? 0.0 : S->Fext[d]; }

void orc_set_group_rates(orc_sim *S, double s_e, double s_eps, double s_q, double s_pi, double s_m)
{
    S->s[1] = s_e;
    S->s[2] = s_eps;
    S->s[4] = S->s[6] = S->s[8] = s_q;
    S->s[10] = S->s[12] = s_pi;
    S->s[16] = S->s[17] = S->s[18] = s_m;
    S->rates = ORC_RATES_DHUMIERES;
}

orc_sim *orc_create(int nx, int ny, int nz, double tau, const double *F, int rates)
{
    orc_sim *S = (orc_sim *)calloc(1, sizeof(orc_sim));
    S->nx = nx; S->ny = ny; S->nz = nz;
    S->N = (long long)nx * ny * nz;
    S->tau = tau;
    for (int d = 0; d < 3; d++) S->Fext[d] = F ? F[d] : 0.0;
    S->rates = rates;
    moment_matrix(S->M);
    moment_inverse(S->M, S->Mi);
    orc_rates(rates, tau, S->s);
    S->f = (double *)calloc((size_t)(Q * S->N), sizeof(double));
    S->fn = (double *)calloc((size_t)(Q * S->N), sizeof(double));
    S->fibm = (double *)calloc((size_t)(3 * S->N), sizeof(double));
    S->solid = (unsigned char *)calloc((size_t)S->N, 1);
    S->owner = (int *)malloc(sizeof(int) * (size_t)S->N);
    S->link_start = (long long *)malloc(sizeof(long long) * (size_t)S->N);
    for (long long c = 0; c < S->N; c++) { S->owner[c] = -1; S->link_start[c] = -1; }
    S->armed_bc = -1;
    double u0[3] = {0, 0, 0}, feq[Q];
    orc_feq(1.0, u0, feq);
    for (int i = 0; i < Q; i++)
        for (long long c = 0; c < S->N; c++) S->f[i * S->N + c] = feq[i];
    return S;
}

void orc_destroy(orc_sim *S)
{
    if (!S) return;
    free(S->f); free(S->fn); free(S->fibm); free(S->solid); free(S->owner); free(S->link_start);
    free(S->links);
    free(S->X); free(S->U); free(S->W); free(S->R); free(S->mass); free(S->inertia);
    free(S->Fh); free(S->Th); free(S->Fprev); free(S->Tprev); free(S->Fc); free(S->has_prev);
    free(S->Iu); free(S->Ir);
    free(S->mX); free(S->mU); free(S->mF); free(S->mFacc); free(S->mdV); free(S->mUnit); free(S->mpid);
    free(S);
}

/* Initial state: populations at equilibrium f_eq(rho0, u). */
void orc_init_velocity(orc_sim *S, const double *u, double rho0)
{
    for (long long c = 0; c < S->N; c++) {
        double uc[3] = {u[c], u[S->N + c], u[2 * S->N + c]}, feq[Q];
        orc_feq(rho0, uc, feq);
        for (int i = 0; i < Q; i++) S->f[i * S->N + c] = feq[i];
    }
}

void orc_set_populations(orc_sim *S, const double *f) { memcpy(S->f, f, sizeof(double) * Q * S->N); }
void orc_get_populations(const orc_sim *S, double *f) { memcpy(f, S->f, sizeof(double) * Q * S->N); }

/* ---------------- geometry ---------------- */

/* Cell (x,y,z) inside particle p: |x - X_p|^2 <= R_p^2, squared distance
 * summed as ((dx^2 + dy^2) + dz^2) with minimum-image components. */
static int inside_particle(const orc_sim *S, int p, int x, int y, int z)
{
    double dx = mimg((double)x - S->X[3 * p], S->nx);
    double dy = mimg((double)y - S->X[3 * p + 1], S->ny);
    double dz = mimg((double)z - S->X[3 * p + 2], S->nz);
    double d2 = (dx * dx + dy * dy) + dz * dz;
    return d2 <= S->R[p] * S->R[p];
}

/* Cell outside the pipe wall: (x-cx)^2 + (y-cy)^2 >= R^2. */
static int outside_pipe(const orc_sim *S, int x, int y)
{
    double dx = (double)x - S->pipe_cx, dy = (double)y - S->pipe_cy;
    double d2 = dx * dx + dy * dy;
    return d2 >= S->pipe_R * S->pipe_R;
}

static void compute_solid(orc_sim *S)
{
    for (long long c = 0; c < S->N; c++) { S->solid[c] = 0; S->owner[c] = -1; }
    if (S->has_pipe) {
        for (long long c = 0; c < S->N; c++) {
            int x, y, z;
            ccoord(S, c, &x, &y, &z);
            if (outside_pipe(S, x, y)) S->solid[c] = 1;
        }
    }
    if (S->has_chan) {
        for (long long c = 0; c < S->N; c++) {
            int x, y, z;
            ccoord(S, c, &x, &y, &z);
            if ((double)y <= S->chan_ylo) { S->solid[c] = 1; S->owner[c] = -2; }
            else if ((double)y >= S->chan_yhi) { S->solid[c] = 1; S->owner[c] = -3; }
        }
    }
    for (int p = 0; p < S->np; p++) {
        int r = (int)ceil(S->R[p]) + 1;
        int bx = (int)floor(S->X[3 * p]), by = (int)floor(S->X[3 * p + 1]), bz = (int)floor(S->X[3 * p + 2]);
        for (int z = bz - r; z <= bz + r + 1; z++)
            for (int y = by - r; y <= by + r + 1; y++)
                for (int x = bx - r; x <= bx + r + 1; x++) {
                    int wx = wrapi(x, S->nx), wy = wrapi(y, S->ny), wz = wrapi(z, S->nz);
                    if (!inside_particle(S, p, wx, wy, wz)) continue;
                    long long c = cidx(S, wx, wy, wz);
                    S->solid[c] = 1;
                    if (S->owner[c] < 0 || p < S->owner[c]) S->owner[c] = p;
                }
    }
}

/* Wall position along a link: smallest t in (0,1] with |x_f + t c - X| = R
 * (sphere, x_f outside) or the exit root of the infinite cylinder (pipe, x_f
 * inside), from a t^2 + 2 b t + c0 = 0 with a = c.c, b = c.d, c0 = d.d - R^2,
 * d = x_f - X. Sums are taken left to right: b = (cx dx + cy dy) + cz dz. */
static double link_q_sphere(const orc_sim *S, int p, int x, int y, int z, int i)
{
    double dx = mimg((double)x - S->X[3 * p], S->nx);
    double dy = mimg((double)y - S->X[3 * p + 1], S->ny);
    double dz = mimg((double)z - S->X[3 * p + 2], S->nz);
    double a = (double)(CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2]);
    double b = (CV[i][0] * dx + CV[i][1] * dy) + CV[i][2] * dz;
    double c0 = ((dx * dx + dy * dy) + dz * dz) - S->R[p] * S->R[p];
    double disc = b * b - a * c0;
    if (disc < 0.0) disc = 0.0;
    double t = (-b - sqrt(disc)) / a;
    if (t > 1.0) t = 1.0;
    if (t < 0.0) t = 0.0;
    return t;
}

static double link_q_pipe(const orc_sim *S, int x, int y, int i)
{
    double dx = (double)x - S->pipe_cx, dy = (double)y - S->pipe_cy;
    double a = (double)(CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1]);
    double b = CV[i][0] * dx + CV[i][1] * dy;
    double c0 = (dx * dx + dy * dy) - S->pipe_R * S->pipe_R;
    double disc = b * b - a * c0;
    if (disc < 0.0) disc = 0.0;
    double t = (-b + sqrt(disc)) / a;
    if (t > 1.0) t = 1.0;
    if (t < 0.0) t = 0.0;
    return t;
}

/* Channel wall (owner -2: lower plane y = y_lo, -3: upper plane y = y_hi)
 * along a link from x_f: t = (y_w - y_f) / c_y. */
static double link_q_channel(const orc_sim *S, int y, int i, int pid)
{
    double yw = pid == -2 ? S->chan_ylo : S->chan_yhi;
    double t = (yw - (double)y) / (double)CV[i][1];
    if (t > 1.0) t = 1.0;
    if (t < 0.0) t = 0.0;
    return t;
}

/* Boundary links: every (x_f, i) with x_f fluid and x_f + c_i solid. The
 * scheme follows the fallback chain of Sec. 3.1 (quadratic, then linear, then
 * single-node bounce-back) on spheres; the pipe wall uses the linear scheme
 * (Sec. 2.1) with the same single-node fallback. Quadratic needs x_f - c_i
 * fluid, and x_f - 2 c_i as well when q < 1/2; linear needs x_f - c_i fluid
 * when q < 1/2. */
static void build_links(orc_sim *S)
{
    S->nlinks = 0;
    for (long long c = 0; c < S->N; c++) S->link_start[c] = -1;
    for (long long c = 0; c < S->N; c++) {
        if (S->solid[c]) continue;
        int x, y, z;
        ccoord(S, c, &x, &y, &z);
        for (int i = 1; i < Q; i++) {
            long long b = cidx(S, x + CV[i][0], y + CV[i][1], z + CV[i][2]);
            if (!S->solid[b]) continue;
            double q;
            int pid = S->owner[b];
            if (pid >= 0) q = link_q_sphere(S, pid, x, y, z, i);
            else if (pid <= -2) q = link_q_channel(S, y, i, pid);
            else q = link_q_pipe(S, x, y, i);
            int f1 = !S->solid[cidx(S, x - CV[i][0], y - CV[i][1], z - CV[i][2])];
            int f2 = !S->solid[cidx(S, x - 2 * CV[i][0], y - 2 * CV[i][1], z - 2 * CV[i][2])];
            int scheme, chain = pid >= 0 ? 0 : (pid <= -2 ? S->chan_chain : 1);
            if (chain == 0) {
                if (q < 0.5) scheme = (f1 && f2) ? ORC_SCHEME_QUAD : (f1 ? ORC_SCHEME_LINEAR : ORC_SCHEME_SINGLE);
                else scheme = f1 ? ORC_SCHEME_QUAD : ORC_SCHEME_LINEAR;
            } else if (chain == 1) {
                if (q < 0.5) scheme = f1 ? ORC_SCHEME_LINEAR : ORC_SCHEME_SINGLE;
                else scheme = ORC_SCHEME_LINEAR;
            } else {
                scheme = chain == 2 ? ORC_SCHEME_SINGLE : ORC_SCHEME_HALFWAY;
            }
            if (S->nlinks == S->cap_links) {
                S->cap_links = S->cap_links ? 2 * S->cap_links : 1024;
                S->links = (link_t *)realloc(S->links, sizeof(link_t) * (size_t)S->cap_links);
            }
            if (S->link_start[c] < 0) S->link_start[c] = S->nlinks;
            link_t *L = &S->links[S->nlinks++];
            L->cell = c; L->dir = i; L->scheme = scheme; L->pid = pid; L->q = q;
        }
    }
}

/* Plane channel, a test geometry for the bounce-back schemes: walls normal
 * to y at y = y_lo and y = y_hi (cells with y <= y_lo or y >= y_hi are
 * solid), moving along x at u_lo and u_hi. chain picks the schemes of its
 * links: 0 the sphere chain (quadratic, linear, single-node), 1 the pipe
 * chain (linear, single-node), 2 single-node only, 3 halfway only. */
void orc_set_channel(orc_sim *S, double y_lo, double y_hi, double u_lo, double u_hi, int chain)
{
    S->has_chan = 1;
    S->chan_ylo = y_lo;
    S->chan_yhi = y_hi;
    S->chan_u[0] = u_lo;
    S->chan_u[1] = u_hi;
    S->chan_chain = chain;
    compute_solid(S);
    build_links(S);
}

void orc_set_pipe(orc_sim *S, double R)
{
    S->has_pipe = 1;
    S->pipe_R = R;
    S->pipe_cx = 0.5 * (S->nx - 1);
    S->pipe_cy = 0.5 * (S->ny - 1);
    compute_solid(S);
    build_links(S);
}

/* Kempe et al. (2012) cell solid fraction from the level set phi = |x-X| - R
 * at the 8 cell corners: alpha = sum(-phi H(-phi)) / sum|phi|. */
double orc_solid_fraction(const double *x, const double *X, double R)
{
    double num = 0.0, den = 0.0;
    for (int m = 0; m < 8; m++) {
        double cx = x[0] + ((m & 1) ? 0.5 : -0.5) - X[0];
        double cy = x[1] + ((m & 2) ? 0.5 : -0.5) - X[1];
        double cz = x[2] + ((m & 4) ? 0.5 : -0.5) - X[2];
        double phi = sqrt(cx * cx + cy * cy + cz * cz) - R;
        if (phi < 0.0) num += -phi;
        den += fabs(phi);
    }
    return den > 0.0 ? num / den : 0.0;
}

static double cell_alpha(const orc_sim *S, int p, int x, int y, int z)
{
    double xr[3] = {S->X[3 * p] + mimg((double)x - S->X[3 * p], S->nx),
                    S->X[3 * p + 1] + mimg((double)y - S->X[3 * p + 1], S->ny),
                    S->X[3 * p + 2] + mimg((double)z - S->X[3 * p + 2], S->nz)};
    return orc_solid_fraction(xr, &S->X[3 * p], S->R[p]);
}

/* Velocity of a post-collision state: sum f c = rho u + F/2 after a Guo
 * collision, so u = (sum f c - F/2) / rho with the force of that collision. */
static void cell_macro(const orc_sim *S, long long c, double *rho, double *u)
{
    double r = 0.0, j[3] = {0, 0, 0};
    for (int i = 0; i < Q; i++) {
        double fi = S->f[i * S->N + c];
        r += fi;
        for (int d = 0; d < 3; d++) j[d] += fi * CV[i][d];
    }
    *rho = r;
    for (int d = 0; d < 3; d++) {
        double F = fext_at(S, c, d) + S->fibm[d * S->N + c];
        u[d] = r != 0.0 ? (j[d] - 0.5 * F) / r : 0.0;
    }
}

void orc_macro(const orc_sim *S, double *rho, double *u)
{
    int ibb = (S->armed_bc == ORC_BC_IBB);
    for (long long c = 0; c < S->N; c++) {
        double r, uc[3];
        if (ibb && S->solid[c]) { r = 0.0; uc[0] = uc[1] = uc[2] = 0.0; }
        else cell_macro(S, c, &r, uc);
        rho[c] = r;
        for (int d = 0; d < 3; d++) u[d * S->N + c] = uc[d];
    }
}

static void cross(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* Kempe inner integrals I_u = sum alpha u, I_r = sum alpha (x-X) x u over the
 * cells overlapping particle p, using the velocities of the current state. */
static void kempe_integrals(const orc_sim *S, int p, double *Iu, double *Ir)
{
    Iu[0] = Iu[1] = Iu[2] = Ir[0] = Ir[1] = Ir[2] = 0.0;
    int r = (int)ceil(S->R[p]) + 1;
    int bx = (int)floor(S->X[3 * p]), by = (int)floor(S->X[3 * p + 1]), bz = (int)floor(S->X[3 * p + 2]);
    for (int z = bz - r; z <= bz + r + 1; z++)
        for (int y = by - r; y <= by + r + 1; y++)
            for (int x = bx - r; x <= bx + r + 1; x++) {
                int wx = wrapi(x, S->nx), wy = wrapi(y, S->ny), wz = wrapi(z, S->nz);
                double a = cell_alpha(S, p, wx, wy, wz);
                if (a <= 0.0) continue;
                double rho, u[3], rr[3], ru[3];
                cell_macro(S, cidx(S, wx, wy, wz), &rho, u);
                rr[0] = mimg((double)wx - S->X[3 * p], S->nx);
                rr[1] = mimg((double)wy - S->X[3 * p + 1], S->ny);
                rr[2] = mimg((double)wz - S->X[3 * p + 2], S->nz);
                cross(rr, u, ru);
                for (int d = 0; d < 3; d++) { Iu[d] += a * u[d]; Ir[d] += a * ru[d]; }
            }
}

/* Particle release (Sec. 3.1): translation velocity = fluid velocity
 * averaged over the particle volume (weights alpha), rotation zero. */
static void release_velocity(const orc_sim *S, int p, double *U)
{
    double su[3] = {0, 0, 0}, sa = 0.0;
    int r = (int)ceil(S->R[p]) + 1;
    int bx = (int)floor(S->X[3 * p]), by = (int)floor(S->X[3 * p + 1]), bz = (int)floor(S->X[3 * p + 2]);
    for (int z = bz - r; z <= bz + r + 1; z++)
        for (int y = by - r; y <= by + r + 1; y++)
            for (int x = bx - r; x <= bx + r + 1; x++) {
                int wx = wrapi(x, S->nx), wy = wrapi(y, S->ny), wz = wrapi(z, S->nz);
                double a = cell_alpha(S, p, wx, wy, wz);
                if (a <= 0.0) continue;
                double rho, u[3];
                cell_macro(S, cidx(S, wx, wy, wz), &rho, u);
                for (int d = 0; d < 3; d++) su[d] += a * u[d];
                sa += a;
            }
    for (int d = 0; d < 3; d++) U[d] = sa > 0.0 ? su[d] / sa : 0.0;
}

int orc_add_spheres(orc_sim *S, int n, const double *X, const double *R, double density_ratio,
                    const double *U, const double *W, int fixed)
{
    if (S->has_pipe || S->np > 0 || n <= 0) return -1;
    S->np = n;
    S->fixed = fixed;
    S->dens = density_ratio;
#define ALLOC3(p) p = (double *)calloc((size_t)(3 * n), sizeof(double))
    ALLOC3(S->X); ALLOC3(S->U); ALLOC3(S->W); ALLOC3(S->Fh); ALLOC3(S->Th);
    ALLOC3(S->Fprev); ALLOC3(S->Tprev); ALLOC3(S->Fc); ALLOC3(S->Iu); ALLOC3(S->Ir);
#undef ALLOC3
    S->R = (double *)calloc((size_t)n, sizeof(double));
    S->mass = (double *)calloc((size_t)n, sizeof(double));
    S->inertia = (double *)calloc((size_t)n, sizeof(double));
    S->has_prev = (int *)calloc((size_t)n, sizeof(int));
    for (int p = 0; p < n; p++) {
        for (int d = 0; d < 3; d++) S->X[3 * p + d] = X[3 * p + d];
        S->R[p] = R[p];
        double vol = 4.0 / 3.0 * PI * R[p] * R[p] * R[p];
        S->mass[p] = density_ratio * vol;
        S->inertia[p] = 0.4 * S->mass[p] * R[p] * R[p];
    }
    for (int p = 0; p < n; p++) {
        if (U) for (int d = 0; d < 3; d++) S->U[3 * p + d] = U[3 * p + d];
        else release_velocity(S, p, &S->U[3 * p]);
        if (W) for (int d = 0; d < 3; d++) S->W[3 * p + d] = W[3 * p + d];
    }
    compute_solid(S);
    build_links(S);
    return 0;
}

/* ---------------- IBB stream-collide ---------------- */

static void wall_velocity(const orc_sim *S, int p, const double *xw, double *uw)
{
    if (p <= -2) { uw[0] = S->chan_u[p == -2 ? 0 : 1]; uw[1] = uw[2] = 0.0; return; }
    if (p < 0) { uw[0] = uw[1] = uw[2] = 0.0; return; }
    double r[3] = {mimg(xw[0] - S->X[3 * p], S->nx), mimg(xw[1] - S->X[3 * p + 1], S->ny),
                   mimg(xw[2] - S->X[3 * p + 2], S->nz)};
    double wr[3];
    cross(&S->W[3 * p], r, wr);
    for (int d = 0; d < 3; d++) uw[d] = S->U[3 * p + d] + wr[d];
}

/* Single-node bounce-back (the last fallback of Sec. 3.1, after Zhao & Yong
 * 2017; the formula is this build's reading, see single-node below): the
 * collision at x_f removed the departure d = M^-1 S (m - m_eq) from its
 * pre-collision populations. It is recovered here from the post-collision
 * populations alone, moment by moment:
 *   m~ = m - S (m - m_eq) + (I - S/2) M F_i
 *   =>  S (m - m_eq) = S (I - S)^-1 (m~ - m_eq - (I - S/2) M F_i),
 * with rho = sum f~ and u = (sum f~ c - F/2) / rho (the Guo velocity of that
 * collision). A moment with rate 0 (conserved) or exactly 1 contributes
 * nothing (a rate of 1 leaves no trace of its departure in f~). Returns
 * d_i + d_ibar. */
static double single_node_pair(const orc_sim *S, const double *A, long long c0, int i, int ib)
{
    double f[Q], r = 0.0, j[3] = {0, 0, 0}, F[3], u[3], feq[Q], Fi[Q], a[Q];
    for (int k = 0; k < Q; k++) {
        f[k] = A[k * S->N + c0];
        r += f[k];
        for (int d = 0; d < 3; d++) j[d] += f[k] * CV[k][d];
    }
    for (int d = 0; d < 3; d++) {
        F[d] = fext_at(S, c0, d);
        u[d] = (j[d] - 0.5 * F[d]) / r;
    }
    orc_feq(r, u, feq);
    guo_source(u, F, Fi);
    for (int k = 0; k < Q; k++) {
        double mt = 0.0, me = 0.0, mF = 0.0, sk = S->s[k];
        for (int m = 0; m < Q; m++) {
            mt += S->M[k][m] * f[m];
            me += S->M[k][m] * feq[m];
            mF += S->M[k][m] * Fi[m];
        }
        a[k] = (sk == 0.0 || sk == 1.0) ? 0.0 : sk / (1.0 - sk) * (mt - me - (1.0 - 0.5 * sk) * mF);
    }
    double di = 0.0, db = 0.0;
    for (int k = 0; k < Q; k++) {
        di += S->Mi[i][k] * a[k];
        db += S->Mi[ib][k] * a[k];
    }
    return di + db;
}

/* Population leaving the wall into x_f along -c_i at t+1 (Bouzidi et al.
 * 2001 quadratic / linear interpolation, the single-node scheme as the last
 * fallback; plain halfway bounce-back only for the channel tests), from
 * post-collision values at t. The moving-wall term D = 6 w_i rho_w
 * (c_ibar . u_w), rho_w = 1, rides on the f_i(x_f) weight. Single node:
 * halfway bounce-back plus (1 - 2q)/2 times the symmetric part d_i + d_ibar
 * of the departure its collision removed at x_f; for a steady flow whose
 * velocity is linear in space that departure is minus the change of f_eq
 * along c_i per unit length, so the value is exact there at any q, and at
 * q = 1/2 it is halfway bounce-back. */
static double ibb_value(const orc_sim *S, const double *A, const link_t *L)
{
    int i = L->dir, ib = OPP(i);
    int x, y, z;
    ccoord(S, L->cell, &x, &y, &z);
    long long c0 = L->cell;
    long long c1 = cidx(S, x - CV[i][0], y - CV[i][1], z - CV[i][2]);
    long long c2 = cidx(S, x - 2 * CV[i][0], y - 2 * CV[i][1], z - 2 * CV[i][2]);
    double q = L->q;
    double xw[3] = {x + q * CV[i][0], y + q * CV[i][1], z + q * CV[i][2]}, uw[3];
    wall_velocity(S, L->pid, xw, uw);
    double D = 6.0 * WT(i) * (CV[ib][0] * uw[0] + CV[ib][1] * uw[1] + CV[ib][2] * uw[2]);
    double fi0 = A[i * S->N + c0], fi1 = A[i * S->N + c1], fi2 = A[i * S->N + c2];
    double fb0 = A[ib * S->N + c0], fb1 = A[ib * S->N + c1];
    switch (L->scheme) {
    case ORC_SCHEME_QUAD:
        if (q < 0.5) return q * (1.0 + 2.0 * q) * fi0 + (1.0 - 4.0 * q * q) * fi1 - q * (1.0 - 2.0 * q) * fi2 + D;
        return fi0 / (q * (2.0 * q + 1.0)) + (2.0 * q - 1.0) / q * fb0 - (2.0 * q - 1.0) / (2.0 * q + 1.0) * fb1 +
               D / (q * (2.0 * q + 1.0));
    case ORC_SCHEME_LINEAR:
        if (q < 0.5) return 2.0 * q * fi0 + (1.0 - 2.0 * q) * fi1 + D;
        return fi0 / (2.0 * q) + (2.0 * q - 1.0) / (2.0 * q) * fb0 + D / (2.0 * q);
    case ORC_SCHEME_SINGLE:
        return fi0 + D + 0.5 * (1.0 - 2.0 * q) * single_node_pair(S, A, c0, i, ib);
    default:
        return fi0 + D;
    }
}

static const link_t *find_link(const orc_sim *S, long long c, int dir)
{
    long long s = S->link_start[c];
    if (s < 0) return NULL;
    for (long long k = s; k < S->nlinks && S->links[k].cell == c; k++)
        if (S->links[k].dir == dir) return &S->links[k];
    return NULL;
}

/* Pull streaming f_i(x, t+1) = f*_i(x - c_i, t); with IBB, a population
 * whose source is solid comes from the link formula instead. */
static void stream_collide(orc_sim *S, int ibb, const double *Fcell /* 3*N or NULL */)
{
    const double *A = S->f;
    double *B = S->fn;
    long long N = S->N;
    int nthr = orc_get_threads();
#pragma omp parallel for schedule(static) num_threads(nthr)
    for (int z = 0; z < S->nz; z++) {
        for (int y = 0; y < S->ny; y++)
            for (int x = 0; x < S->nx; x++) {
                long long c = cidx(S, x, y, z);
                if (ibb && S->solid[c]) continue;
                double fin[Q], fout[Q], F[3];
                for (int i = 0; i < Q; i++) {
                    long long src = cidx(S, x - CV[i][0], y - CV[i][1], z - CV[i][2]);
                    if (ibb && S->solid[src]) {
                        const link_t *L = find_link(S, c, OPP(i));
                        fin[i] = L ? ibb_value(S, A, L) : A[OPP(i) * N + c];
                    } else {
                        fin[i] = A[i * N + src];
                    }
                }
                for (int d = 0; d < 3; d++) F[d] = fext_at(S, c, d) + (Fcell ? Fcell[d * N + c] : 0.0);
                collide_mrt(S->M, S->Mi, S->s, fin, F, fout);
                for (int i = 0; i < Q; i++) B[i * N + c] = fout[i];
            }
    }
}

/* Galilean-invariant momentum exchange (Wen et al. 2014), per link:
 * dP = (c_i - u_w) f*_i(x_f, t) - (c_ibar - u_w) f_ibar(x_f, t+1);
 * force = sum dP, torque = sum (x_f + c_i/2 - X_p) x dP. The lever arm is the
 * link midpoint: with it a uniformly translating sphere in a uniform stream
 * feels neither force nor torque (with the wall point x_f + q c_i it would
 * pick up a spurious torque from the Galilean correction term). */
static void gimem(orc_sim *S)
{
    for (int p = 0; p < S->np; p++)
        for (int d = 0; d < 3; d++) S->Fh[3 * p + d] = S->Th[3 * p + d] = 0.0;
    for (long long k = 0; k < S->nlinks; k++) {
        const link_t *L = &S->links[k];
        int p = L->pid;
        if (p < 0) continue;
        int i = L->dir, ib = OPP(i), x, y, z;
        ccoord(S, L->cell, &x, &y, &z);
        double xw[3] = {x + L->q * CV[i][0], y + L->q * CV[i][1], z + L->q * CV[i][2]}, uw[3];
        wall_velocity(S, p, xw, uw);
        double fout = S->f[i * S->N + L->cell];
        double fin = ibb_value(S, S->f, L);
        double dP[3], r[3], t[3];
        for (int d = 0; d < 3; d++) dP[d] = (CV[i][d] - uw[d]) * fout - (CV[ib][d] - uw[d]) * fin;
        r[0] = mimg(x + 0.5 * CV[i][0] - S->X[3 * p], S->nx);
        r[1] = mimg(y + 0.5 * CV[i][1] - S->X[3 * p + 1], S->ny);
        r[2] = mimg(z + 0.5 * CV[i][2] - S->X[3 * p + 2], S->nz);
        cross(r, dP, t);
        for (int d = 0; d < 3; d++) { S->Fh[3 * p + d] += dP[d]; S->Th[3 * p + d] += t[d]; }
    }
}

/* Normal-only soft-sphere contact (Sec. 3.1): for a gap delta = |X_a - X_b|
 * - (R_a + R_b) below zeta = 1, a spring-dashpot force along the line of
 * centres, F = k_n (zeta - delta) - eta_n v_n, with k_n = m (pi^2 + ln^2 e) /
 * Tc^2, eta_n = -2 m ln e / Tc, m the reduced mass, e = 0.97, Tc = 10. */
static void contact_forces(orc_sim *S)
{
    const double zeta = 1.0, e = 0.97, Tc = 10.0;
    for (int p = 0; p < 3 * S->np; p++) S->Fc[p] = 0.0;
    for (int a = 0; a < S->np; a++)
        for (int b = a + 1; b < S->np; b++) {
            double d[3] = {mimg(S->X[3 * a] - S->X[3 * b], S->nx), mimg(S->X[3 * a + 1] - S->X[3 * b + 1], S->ny),
                           mimg(S->X[3 * a + 2] - S->X[3 * b + 2], S->nz)};
            double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double gap = dist - (S->R[a] + S->R[b]);
            if (gap >= zeta || dist <= 0.0) continue;
            double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
            double vn = (S->U[3 * a] - S->U[3 * b]) * n[0] + (S->U[3 * a + 1] - S->U[3 * b + 1]) * n[1] +
                        (S->U[3 * a + 2] - S->U[3 * b + 2]) * n[2];
            double meff = S->mass[a] * S->mass[b] / (S->mass[a] + S->mass[b]);
            double le = log(e);
            double kn = meff * (PI * PI + le * le) / (Tc * Tc);
            double eta = -2.0 * meff * le / Tc;
            double Fm = kn * (zeta - gap) - eta * vn;
            for (int k = 0; k < 3; k++) { S->Fc[3 * a + k] += Fm * n[k]; S->Fc[3 * b + k] -= Fm * n[k]; }
        }
}

/* Rigid-body update in FP64 (the paper does not give its integrator): the
 * hydrodynamic force and torque are averaged over the last two steps (first
 * step: the current value), the contact force enters at its current value,
 * the velocity is advanced first and the position with the new velocity
 * (symplectic Euler, which keeps the soft-sphere restitution at e):
 *   U^{n+1} = U^n + ((F_h^n + F_h^{n-1})/2 + F_c^n) / m,  X^{n+1} = X^n + U^{n+1},
 *   W^{n+1} = W^n + (T_h^n + T_h^{n-1}) / (2 I). */
static void particle_eom(orc_sim *S)
{
    int n[3] = {S->nx, S->ny, S->nz};
    for (int p = 0; p < S->np; p++) {
        for (int d = 0; d < 3; d++) {
            double Fh = S->Fh[3 * p + d], Th = S->Th[3 * p + d];
            double Fa = S->has_prev[p] ? 0.5 * (Fh + S->Fprev[3 * p + d]) : Fh;
            double Ta = S->has_prev[p] ? 0.5 * (Th + S->Tprev[3 * p + d]) : Th;
            double u1 = S->U[3 * p + d] + (Fa + S->Fc[3 * p + d]) / S->mass[p];
            S->U[3 * p + d] = u1;
            S->W[3 * p + d] += Ta / S->inertia[p];
            double x = S->X[3 * p + d] + u1;
            if (x >= n[d]) x -= n[d];
            if (x < 0.0) x += n[d];
            S->X[3 * p + d] = x;
            S->Fprev[3 * p + d] = Fh;
            S->Tprev[3 * p + d] = Th;
        }
        S->has_prev[p] = 1;
    }
}

/* Caiazzo (2008) refill of a node uncovered between t and t+1: density =
 * mean of its fluid neighbours, velocity = rigid-body velocity of the
 * particle that left it, non-equilibrium part copied from the fluid
 * neighbour best aligned with the outward normal (ties: lowest direction). */
static void refill(orc_sim *S, const unsigned char *solid_old, const int *owner_old)
{
    double *B = S->fn;
    long long N = S->N;
    for (long long c = 0; c < N; c++) {
        if (!solid_old[c] || S->solid[c]) continue;
        int p = owner_old[c];
        int x, y, z;
        ccoord(S, c, &x, &y, &z);
        double xr[3] = {(double)x, (double)y, (double)z}, uw[3];
        wall_velocity(S, p, xr, uw);
        double nrm[3] = {0, 0, 0};
        if (p >= 0) {
            nrm[0] = mimg(x - S->X[3 * p], S->nx);
            nrm[1] = mimg(y - S->X[3 * p + 1], S->ny);
            nrm[2] = mimg(z - S->X[3 * p + 2], S->nz);
            double l = sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
            if (l > 0) for (int d = 0; d < 3; d++) nrm[d] /= l;
        }
        double rsum = 0.0, best = -1e300;
        int cnt = 0;
        long long bestc = -1;
        for (int i = 1; i < Q; i++) {
            long long nb = cidx(S, x + CV[i][0], y + CV[i][1], z + CV[i][2]);
            if (solid_old[nb] || S->solid[nb]) continue;
            double r = 0.0;
            for (int k = 0; k < Q; k++) r += B[k * N + nb];
            rsum += r;
            cnt++;
            double cl = sqrt((double)(CV[i][0] * CV[i][0] + CV[i][1] * CV[i][1] + CV[i][2] * CV[i][2]));
            double al = (nrm[0] * CV[i][0] + nrm[1] * CV[i][1] + nrm[2] * CV[i][2]) / cl;
            if (al > best) { best = al; bestc = nb; }
        }
        double rho = cnt ? rsum / cnt : 1.0, feq[Q];
        orc_feq(rho, uw, feq);
        if (bestc >= 0) {
            double r = 0.0, j[3] = {0, 0, 0}, un[3], fe[Q];
            for (int k = 0; k < Q; k++) {
                double fk = B[k * N + bestc];
                r += fk;
                for (int d = 0; d < 3; d++) j[d] += fk * CV[k][d];
            }
            for (int d = 0; d < 3; d++) un[d] = (j[d] - 0.5 * fext_at(S, bestc, d)) / r;
            orc_feq(r, un, fe);
            for (int k = 0; k < Q; k++) B[k * N + c] = feq[k] + (B[k * N + bestc] - fe[k]);
        } else {
            for (int k = 0; k < Q; k++) B[k * N + c] = feq[k];
        }
    }
}

static void step_ibb(orc_sim *S)
{
    stream_collide(S, 1, NULL);
    if (S->np > 0) {
        gimem(S);
        if (!S->fixed) {
            contact_forces(S);
            particle_eom(S);
            unsigned char *so = (unsigned char *)malloc((size_t)S->N);
            int *oo = (int *)malloc(sizeof(int) * (size_t)S->N);
            memcpy(so, S->solid, (size_t)S->N);
            memcpy(oo, S->owner, sizeof(int) * (size_t)S->N);
            compute_solid(S);
            refill(S, so, oo);
            free(so);
            free(oo);
        }
    }
    double *t = S->f; S->f = S->fn; S->fn = t;
    if (S->np > 0 && !S->fixed) build_links(S);
}

/* ---------------- IBM ---------------- */

int orc_marker_count(double RL) { return (int)floor(PI / 3.0 * (12.0 * RL * RL + 1.0) + 0.5); }

/* Golden-spiral points on the unit sphere (the paper does not say how its
 * Lagrangian points are laid out; this gives near-uniform spacing). */
void orc_sphere_markers(double RL, int n, double *unit)
{
    (void)RL;
    double ga = PI * (3.0 - sqrt(5.0));
    for (int l = 0; l < n; l++) {
        double zz = 1.0 - (2.0 * l + 1.0) / n;
        double r = sqrt(1.0 - zz * zz);
        double th = ga * l;
        unit[3 * l] = r * cos(th);
        unit[3 * l + 1] = r * sin(th);
        unit[3 * l + 2] = zz;
    }
}

/* Lagrangian markers with a cell volume close to the Eulerian one (Sec. 2.1):
 * spheres at R_L = R - r_d with N_L = round(pi/3 (12 R_L^2 + 1)) points and
 * dV = pi (12 R_L^2 + 1) / (3 N_L) (a shell of unit thickness split evenly);
 * the pipe as a circle of N_c = round(2 pi R_L) points at R_L = R + r_d copied
 * to every z plane, dV = 2 pi R_L / N_c. r_d = 0.4 for IBM-B, 0 for IBM-U. */
static void build_markers(orc_sim *S, double rd)
{
    free(S->mX); free(S->mU); free(S->mF); free(S->mFacc); free(S->mdV); free(S->mUnit); free(S->mpid);
    long long nm = 0;
    if (S->has_pipe) {
        double RL = S->pipe_R + rd;
        int nc = (int)floor(2.0 * PI * RL + 0.5);
        nm = (long long)nc * S->nz;
        S->mX = (double *)calloc((size_t)(3 * nm), sizeof(double));
        S->mdV = (double *)calloc((size_t)nm, sizeof(double));
        S->mpid = (int *)calloc((size_t)nm, sizeof(int));
        S->mUnit = NULL;
        for (int z = 0; z < S->nz; z++)
            for (int j = 0; j < nc; j++) {
                long long l = (long long)z * nc + j;
                double th = 2.0 * PI * j / nc;
                S->mX[3 * l] = S->pipe_cx + RL * cos(th);
                S->mX[3 * l + 1] = S->pipe_cy + RL * sin(th);
                S->mX[3 * l + 2] = (double)z;
                S->mdV[l] = 2.0 * PI * RL / nc;
                S->mpid[l] = -1;
            }
    } else {
        for (int p = 0; p < S->np; p++) nm += orc_marker_count(S->R[p] - rd);
        S->mX = (double *)calloc((size_t)(3 * nm), sizeof(double));
        S->mUnit = (double *)calloc((size_t)(3 * nm), sizeof(double));
        S->mdV = (double *)calloc((size_t)nm, sizeof(double));
        S->mpid = (int *)calloc((size_t)nm, sizeof(int));
        long long l = 0;
        for (int p = 0; p < S->np; p++) {
            double RL = S->R[p] - rd;
            int n = orc_marker_count(RL);
            orc_sphere_markers(RL, n, &S->mUnit[3 * l]);
            for (int k = 0; k < n; k++, l++) {
                for (int d = 0; d < 3; d++) S->mUnit[3 * l + d] *= RL;
                S->mdV[l] = PI * (12.0 * RL * RL + 1.0) / (3.0 * n);
                S->mpid[l] = p;
            }
        }
    }
    S->nm = nm;
    S->mU = (double *)calloc((size_t)(3 * nm), sizeof(double));
    S->mF = (double *)calloc((size_t)(3 * nm), sizeof(double));
    S->mFacc = (double *)calloc((size_t)(3 * nm), sizeof(double));
}

static void place_markers(orc_sim *S)
{
    if (S->has_pipe) return;
    int n[3] = {S->nx, S->ny, S->nz};
    for (long long l = 0; l < S->nm; l++) {
        int p = S->mpid[l];
        for (int d = 0; d < 3; d++) {
            double x = S->X[3 * p + d] + S->mUnit[3 * l + d];
            if (x >= n[d]) x -= n[d];
            if (x < 0.0) x += n[d];
            S->mX[3 * l + d] = x;
        }
    }
}

/* Marker l's 4x4x4 stencil: nodes floor(X)-1 .. floor(X)+2 per axis, with
 * weight phi(x-X) phi(y-Y) phi(z-Z). */
typedef struct { long long c[64]; double w[64]; } stencil_t;
static void marker_stencil(const orc_sim *S, const double *X, stencil_t *st)
{
    int b[3] = {(int)floor(X[0]) - 1, (int)floor(X[1]) - 1, (int)floor(X[2]) - 1};
    double ph[3][4];
    for (int d = 0; d < 3; d++)
        for (int k = 0; k < 4; k++) ph[d][k] = orc_peskin_phi((double)(b[d] + k) - X[d]);
    int m = 0;
    for (int kz = 0; kz < 4; kz++)
        for (int ky = 0; ky < 4; ky++)
            for (int kx = 0; kx < 4; kx++, m++) {
                st->c[m] = cidx(S, b[0] + kx, b[1] + ky, b[2] + kz);
                st->w[m] = ph[0][kx] * ph[1][ky] * ph[2][kz];
            }
}

static void marker_desired_velocity(const orc_sim *S, long long l, double *Ud)
{
    int p = S->mpid[l];
    if (p < 0) { Ud[0] = Ud[1] = Ud[2] = 0.0; return; }
    wall_velocity(S, p, &S->mX[3 * l], Ud);
}

/* IBM step (Uhlmann 2005 direct forcing with the multi-direct-forcing
 * iterations of Breugem 2012; Sec. 2.1 / 3.1): stream; rho and
 * u* = (sum f c + F_ext/2)/rho; three passes of {interpolate U*_l, force
 * F_l = 2 rho_l (U_d - U*_l), spread F(x) = sum_l F_l delta dV_l,
 * u* += F/(2 rho)}; collide with F_ext + the accumulated IBM force. */
static void step_ibm(orc_sim *S)
{
    long long N = S->N;
    const double *A = S->f;
    double *fp = S->fn;
    /* stream */
    for (int z = 0; z < S->nz; z++)
        for (int y = 0; y < S->ny; y++)
            for (int x = 0; x < S->nx; x++) {
                long long c = cidx(S, x, y, z);
                for (int i = 0; i < Q; i++)
                    fp[i * N + c] = A[i * N + cidx(S, x - CV[i][0], y - CV[i][1], z - CV[i][2])];
            }
    double *rho = (double *)malloc(sizeof(double) * (size_t)N);
    double *us = (double *)malloc(sizeof(double) * (size_t)(3 * N));
    double *Fp = (double *)malloc(sizeof(double) * (size_t)(3 * N));
    for (long long c = 0; c < N; c++) {
        double r = 0.0, j[3] = {0, 0, 0};
        for (int i = 0; i < Q; i++) {
            double fi = fp[i * N + c];
            r += fi;
            for (int d = 0; d < 3; d++) j[d] += fi * CV[i][d];
        }
        rho[c] = r;
        for (int d = 0; d < 3; d++) us[d * N + c] = (j[d] + 0.5 * fext_at(S, c, d)) / r;
    }
    memset(S->fibm, 0, sizeof(double) * (size_t)(3 * N));
    for (long long l = 0; l < S->nm; l++)
        for (int d = 0; d < 3; d++) S->mFacc[3 * l + d] = 0.0;
    stencil_t st;
    for (int pass = 0; pass < 3; pass++) {
        double rmax = 0.0;
        for (long long l = 0; l < S->nm; l++) {
            marker_stencil(S, &S->mX[3 * l], &st);
            double U[3] = {0, 0, 0}, rl = 0.0, Ud[3];
            for (int m = 0; m < 64; m++) {
                rl += st.w[m] * rho[st.c[m]];
                for (int d = 0; d < 3; d++) U[d] += st.w[m] * us[d * N + st.c[m]];
            }
            marker_desired_velocity(S, l, Ud);
            for (int d = 0; d < 3; d++) {
                double r = fabs(Ud[d] - U[d]);
                if (r > rmax) rmax = r;
                S->mU[3 * l + d] = U[d];
                S->mF[3 * l + d] = 2.0 * rl * (Ud[d] - U[d]);
                S->mFacc[3 * l + d] += S->mF[3 * l + d];
            }
        }
        S->resid[pass] = rmax;
        memset(Fp, 0, sizeof(double) * (size_t)(3 * N));
        for (long long l = 0; l < S->nm; l++) {
            marker_stencil(S, &S->mX[3 * l], &st);
            for (int m = 0; m < 64; m++)
                for (int d = 0; d < 3; d++) Fp[d * N + st.c[m]] += S->mF[3 * l + d] * st.w[m] * S->mdV[l];
        }
        for (long long c = 0; c < N; c++)
            for (int d = 0; d < 3; d++) {
                us[d * N + c] += Fp[d * N + c] / (2.0 * rho[c]);
                S->fibm[d * N + c] += Fp[d * N + c];
            }
    }
    /* collide every cell with F_ext + F_IBM */
    double *B = (double *)malloc(sizeof(double) * (size_t)(Q * N));
    int nthr = orc_get_threads();
#pragma omp parallel for schedule(static) num_threads(nthr)
    for (long long c = 0; c < N; c++) {
        double fin[Q], fout[Q], F[3];
        for (int i = 0; i < Q; i++) fin[i] = fp[i * N + c];
        for (int d = 0; d < 3; d++) F[d] = fext_at(S, c, d) + S->fibm[d * N + c];
        collide_mrt(S->M, S->Mi, S->s, fin, F, fout);
        for (int i = 0; i < Q; i++) B[i * N + c] = fout[i];
    }
    memcpy(S->f, B, sizeof(double) * (size_t)(Q * N));
    free(B);
    /* particle force and torque: reaction of the marker forces plus the
     * Kempe et al. (2012) rate of change of the inner-fluid momentum */
    if (S->np > 0) {
        for (int p = 0; p < S->np; p++)
            for (int d = 0; d < 3; d++) S->Fh[3 * p + d] = S->Th[3 * p + d] = 0.0;
        for (long long l = 0; l < S->nm; l++) {
            int p = S->mpid[l];
            double F[3], r[3], t[3];
            for (int d = 0; d < 3; d++) F[d] = -S->mFacc[3 * l + d] * S->mdV[l];
            r[0] = mimg(S->mX[3 * l] - S->X[3 * p], S->nx);
            r[1] = mimg(S->mX[3 * l + 1] - S->X[3 * p + 1], S->ny);
            r[2] = mimg(S->mX[3 * l + 2] - S->X[3 * p + 2], S->nz);
            cross(r, F, t);
            for (int d = 0; d < 3; d++) { S->Fh[3 * p + d] += F[d]; S->Th[3 * p + d] += t[d]; }
        }
        for (int p = 0; p < S->np; p++) {
            double Iu[3], Ir[3];
            kempe_integrals(S, p, Iu, Ir);
            for (int d = 0; d < 3; d++) {
                S->Fh[3 * p + d] += Iu[d] - S->Iu[3 * p + d];
                S->Th[3 * p + d] += Ir[d] - S->Ir[3 * p + d];
                S->Iu[3 * p + d] = Iu[d];
                S->Ir[3 * p + d] = Ir[d];
            }
        }
        if (!S->fixed) {
            contact_forces(S);
            particle_eom(S);
            place_markers(S);
            compute_solid(S);
        }
    }
    free(rho); free(us); free(Fp);
}

/* First IBM step: markers, and the one-time overwrite of the velocity inside
 * each particle with its rigid-body motion at insertion (Sec. 3.1). */
static void arm_ibm(orc_sim *S, int bc)
{
    build_markers(S, bc == ORC_BC_IBM_B ? 0.4 : 0.0);
    place_markers(S);
    long long N = S->N;
    for (long long c = 0; c < N; c++) {
        int p = S->owner[c];
        if (p < 0 || !S->solid[c]) continue;
        int x, y, z;
        ccoord(S, c, &x, &y, &z);
        double xr[3] = {(double)x, (double)y, (double)z}, uw[3], rho, u[3], feq[Q];
        cell_macro(S, c, &rho, u);
        wall_velocity(S, p, xr, uw);
        orc_feq(rho, uw, feq);
        for (int i = 0; i < Q; i++) S->f[i * N + c] = feq[i];
    }
    for (int p = 0; p < S->np; p++) kempe_integrals(S, p, &S->Iu[3 * p], &S->Ir[3 * p]);
}

int orc_step(orc_sim *S, int nsteps, int bc)
{
    if (S->armed_bc < 0) {
        S->armed_bc = bc;
        if (bc == ORC_BC_IBM_U || bc == ORC_BC_IBM_B) arm_ibm(S, bc);
    } else if (S->armed_bc != bc) {
        return -1;
    }
    for (int n = 0; n < nsteps; n++) {
        if (bc == ORC_BC_IBM_U || bc == ORC_BC_IBM_B) {
            step_ibm(S);
        } else if (bc == ORC_BC_IBB) {
            step_ibb(S);
        } else {
            stream_collide(S, 0, NULL);
            double *t = S->f; S->f = S->fn; S->fn = t;
        }
        S->step++;
    }
    return 0;
}

/* Particle dynamics alone (no fluid): contact forces and the rigid-body
 * update with zero hydrodynamic force, for checking the integrator. */
void orc_particles_advance(orc_sim *S, int nsteps)
{
    for (int n = 0; n < nsteps; n++) {
        for (int k = 0; k < 3 * S->np; k++) S->Fh[k] = S->Th[k] = 0.0;
        contact_forces(S);
        particle_eom(S);
    }
}

/* ---------------- accessors ---------------- */

void orc_get_solid(const orc_sim *S, unsigned char *solid, int *owner)
{
    if (solid) memcpy(solid, S->solid, (size_t)S->N);
    if (owner) memcpy(owner, S->owner, sizeof(int) * (size_t)S->N);
}
long long orc_num_links(const orc_sim *S) { return S->nlinks; }
void orc_get_links(const orc_sim *S, long long *cell, int *dir, int *scheme, double *q, int *pid)
{
    for (long long k = 0; k < S->nlinks; k++) {
        cell[k] = S->links[k].cell;
        dir[k] = S->links[k].dir;
        scheme[k] = S->links[k].scheme;
        q[k] = S->links[k].q;
        pid[k] = S->links[k].pid;
    }
}
int orc_num_particles(const orc_sim *S) { return S->np; }
void orc_get_particles(const orc_sim *S, double *X, double *U, double *W, double *F, double *T)
{
    size_t b = sizeof(double) * (size_t)(3 * S->np);
    if (X) memcpy(X, S->X, b);
    if (U) memcpy(U, S->U, b);
    if (W) memcpy(W, S->W, b);
    if (F) memcpy(F, S->Fh, b);
    if (T) memcpy(T, S->Th, b);
}
long long orc_num_markers(const orc_sim *S) { return S->nm; }
void orc_get_markers(const orc_sim *S, double *X, double *F, double *dV, int *pid)
{
    if (X) memcpy(X, S->mX, sizeof(double) * (size_t)(3 * S->nm));
    if (F) memcpy(F, S->mFacc, sizeof(double) * (size_t)(3 * S->nm));
    if (dV) memcpy(dV, S->mdV, sizeof(double) * (size_t)S->nm);
    if (pid) memcpy(pid, S->mpid, sizeof(int) * (size_t)S->nm);
}
void orc_get_ibm_force(const orc_sim *S, double *F) { memcpy(F, S->fibm, sizeof(double) * (size_t)(3 * S->N)); }
double orc_marker_residual(const orc_sim *S, int pass) { return (pass >= 0 && pass < 3) ? S->resid[pass] : -1.0; }

/* ---------------- statistics ---------------- */

/* Statistics of Sec. 3.2 / Sec. 2.2 on the current state.
 * Masking (Sec. 3.2): cells inside a particle take its rigid-body velocity
 * (cells outside the pipe take the wall velocity, zero); IBB always masks,
 * IBM masks unless ORC_STATS_UNMASK. Velocity gradients by second-order
 * central differences on the periodic grid; dissipation 2 nu s_ij s_ij with
 * the zero-mean assumption of Sec. 3.2. Radial bins: fluid cells binned by
 * r / r_p of the nearest particle surface, r/r_p in [1, 3) by 0.05, each bin
 * mean normalised by the mean over all fluid cells. */
/* Velocity field of the statistics (Sec. 3.2): u of the post-collision
   state, with solid cells replaced by the rigid-body velocity of their
   particle (zero outside the pipe) unless IBM statistics are asked for
   unmasked. u: 3 N values, component-major. */
void orc_masked_velocity(const orc_sim *S, int flags, double *u)
{
    long long N = S->N;
    double *rho = (double *)malloc(sizeof(double) * (size_t)N);
    orc_macro(S, rho, u);
    free(rho);
    int ibm = (S->armed_bc == ORC_BC_IBM_U || S->armed_bc == ORC_BC_IBM_B);
    int mask = !(ibm && (flags & ORC_STATS_UNMASK));
    for (long long c = 0; c < N; c++) {
        if (!S->solid[c] || !mask) continue;
        int x, y, z;
        ccoord(S, c, &x, &y, &z);
        double xr[3] = {(double)x, (double)y, (double)z}, uw[3];
        wall_velocity(S, S->owner[c], xr, uw);
        for (int d = 0; d < 3; d++) u[d * N + c] = uw[d];
    }
}

void orc_stats(const orc_sim *S, int flags, orc_stats_t *o)
{
    long long N = S->N;
    memset(o, 0, sizeof(*o));
    double *rho = (double *)malloc(sizeof(double) * (size_t)N);
    double *u = (double *)malloc(sizeof(double) * (size_t)(3 * N));
    orc_macro(S, rho, u);
    orc_masked_velocity(S, flags, u);
    double nu = (S->tau - 0.5) / 3.0;
    double ke = 0.0, eps = 0.0, kef = 0.0, epsf = 0.0, ub = 0.0;
    long long nf = 0, nin = 0;
    double *epsc = (double *)malloc(sizeof(double) * (size_t)N);
    for (long long c = 0; c < N; c++) {
        int x, y, z;
        ccoord(S, c, &x, &y, &z);
        double g[3][3];
        for (int a = 0; a < 3; a++) {
            long long cp[3] = {cidx(S, x + 1, y, z), cidx(S, x, y + 1, z), cidx(S, x, y, z + 1)};
            long long cm[3] = {cidx(S, x - 1, y, z), cidx(S, x, y - 1, z), cidx(S, x, y, z - 1)};
            for (int b = 0; b < 3; b++) g[a][b] = 0.5 * (u[a * N + cp[b]] - u[a * N + cm[b]]);
        }
        double ss = 0.0;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double sab = 0.5 * (g[a][b] + g[b][a]);
                ss += sab * sab;
            }
        double e = 2.0 * nu * ss;
        double k = 0.5 * (u[c] * u[c] + u[N + c] * u[N + c] + u[2 * N + c] * u[2 * N + c]);
        epsc[c] = e;
        ke += k;
        eps += e;
        if (!S->solid[c]) {
            kef += k;
            epsf += e;
            nf++;
        }
        if (S->has_pipe && !S->solid[c]) { ub += u[2 * N + c]; nin++; }
    }
    /* mass and momentum over the cells that carry fluid: all cells for IBM
     * and for the plain periodic box, the non-solid ones for IBB */
    {
        double *uu = (double *)malloc(sizeof(double) * (size_t)(3 * N));
        orc_macro(S, rho, uu);
        for (long long c = 0; c < N; c++) {
            if (S->armed_bc == ORC_BC_IBB && S->solid[c]) continue;
            o->mass += rho[c];
            for (int d = 0; d < 3; d++) o->momentum[d] += rho[c] * uu[d * N + c];
        }
        free(uu);
    }
    o->kinetic_energy = ke / (double)N;
    o->dissipation = eps / (double)N;
    o->kinetic_energy_fluid = nf ? kef / nf : 0.0;
    o->dissipation_fluid = nf ? epsf / nf : 0.0;
    o->nfluid = nf;
    o->bulk_velocity = nin ? ub / nin : 0.0;
    for (int p = 0; p < S->np; p++) {
        double U2 = 0.0, W2 = 0.0;
        for (int d = 0; d < 3; d++) {
            U2 += S->U[3 * p + d] * S->U[3 * p + d];
            W2 += S->W[3 * p + d] * S->W[3 * p + d];
            o->force[d] += S->Fh[3 * p + d];
            o->torque[d] += S->Th[3 * p + d];
        }
        o->particle_ke += 0.5 * S->mass[p] * U2;
        o->particle_ake += 0.5 * S->inertia[p] * W2;
    }
    if ((flags & ORC_STATS_BINS) && S->np > 0) {
        double sk[ORC_NBINS] = {0}, se[ORC_NBINS] = {0};
        for (long long c = 0; c < N; c++) {
            if (S->solid[c]) continue;
            int x, y, z;
            ccoord(S, c, &x, &y, &z);
            double best = 1e300, ratio = 0.0;
            for (int p = 0; p < S->np; p++) {
                double dx = mimg(x - S->X[3 * p], S->nx), dy = mimg(y - S->X[3 * p + 1], S->ny),
                       dz = mimg(z - S->X[3 * p + 2], S->nz);
                double r = sqrt(dx * dx + dy * dy + dz * dz);
                if (r - S->R[p] < best) { best = r - S->R[p]; ratio = r / S->R[p]; }
            }
            int b = (int)floor((ratio - 1.0) / 0.05);
            if (b < 0 || b >= ORC_NBINS) continue;
            sk[b] += 0.5 * (u[c] * u[c] + u[N + c] * u[N + c] + u[2 * N + c] * u[2 * N + c]);
            se[b] += epsc[c];
            o->bin_count[b]++;
        }
        o->nbins = ORC_NBINS;
        for (int b = 0; b < ORC_NBINS; b++) {
            o->bin_r[b] = 1.0 + 0.05 * (b + 0.5);
            if (o->bin_count[b] > 0) {
                o->bin_tke[b] = (sk[b] / o->bin_count[b]) / (o->kinetic_energy_fluid > 0 ? o->kinetic_energy_fluid : 1.0);
                o->bin_eps[b] = (se[b] / o->bin_count[b]) / (o->dissipation_fluid > 0 ? o->dissipation_fluid : 1.0);
            }
        }
    }
    o->nlinks = S->nlinks;
    o->nmarkers = S->nm;
    o->step = S->step;
    free(rho); free(u); free(epsc);
}
