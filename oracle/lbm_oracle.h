/* Oracle for the D3Q19 lattice Boltzmann method with interpolated bounce-back
 * (IBB) and direct-forcing immersed boundary (IBM) no-slip walls, as compared
 * in Peng et al., "Comparative study of IBB and IBM in the lattice Boltzmann
 * method, Part II: turbulent flows" (arXiv:1906.05448).
 *
 * TEST INFRASTRUCTURE ONLY. A plain, slow, FP64 CPU statement of what the
 * CUDA library computes, written from the paper and the methods it cites.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may load it; it shares no code, header, table or helper with the CUDA
 * library.
 *
 * Layout: scalar fields idx = x + nx*(y + ny*z); populations f[i*N + idx];
 * vectors component-major v[c*N + idx]. Particle arrays are (n,3) row-major.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_sim orc_sim;

enum { ORC_BC_NONE = 0, ORC_BC_IBB = 1, ORC_BC_IBM_U = 2, ORC_BC_IBM_B = 3 };
enum { ORC_RATES_SRT = 0, ORC_RATES_DHUMIERES = 1 };
enum { ORC_SCHEME_QUAD = 0, ORC_SCHEME_LINEAR = 1, ORC_SCHEME_SINGLE = 2, ORC_SCHEME_HALFWAY = 3 };
enum { ORC_STATS_UNMASK = 1, ORC_STATS_BINS = 4 };

#define ORC_NBINS 40

typedef struct {
    double mass, momentum[3];
    double kinetic_energy, dissipation;         /* cell averages over the box */
    double kinetic_energy_fluid, dissipation_fluid; /* averages over fluid cells */
    double particle_ke, particle_ake;
    double force[3], torque[3];
    double bulk_velocity;
    int nbins;
    double bin_r[ORC_NBINS], bin_tke[ORC_NBINS], bin_eps[ORC_NBINS];
    long long bin_count[ORC_NBINS];
    long long nfluid, nlinks, nmarkers, step;
} orc_stats_t;

/* lattice and single-cell pieces */
void   orc_lattice(int *c, double *w, int *opp);
void   orc_moment_matrix(double *M);
void   orc_rates(int set, double tau, double *s);
void   orc_feq(double rho, const double *u, double *feq);
void   orc_collide_mrt(const double *f, const double *F, int set, double tau, double *out);
void   orc_collide_bgk(const double *f, const double *F, double tau, double *out);
double orc_peskin_phi(double r);
double orc_solid_fraction(const double *x, const double *X, double R);
int    orc_marker_count(double RL);
void   orc_sphere_markers(double RL, int n, double *unit);

/* simulation */
orc_sim *orc_create(int nx, int ny, int nz, double tau, const double *F, int rates);
/* Non-shear relaxation rates by d'Humieres group: energy e (bulk viscosity
 * (2/9)(1/s_e - 1/2)), energy square eps, energy flux q, pi_xx and pi_ww,
 * and the third-order m modes; the shear rate stays 1/tau. The paper's
 * solver has this knob for the bulk viscosity but leaves it off (Sec. 2.2). */
void  orc_set_group_rates(orc_sim *S, double s_e, double s_eps, double s_q, double s_pi, double s_m);
void  orc_destroy(orc_sim *S);
void  orc_set_threads(int n);
int   orc_get_threads(void);
void  orc_init_velocity(orc_sim *S, const double *u, double rho0);
void  orc_set_populations(orc_sim *S, const double *f);
void  orc_get_populations(const orc_sim *S, double *f);
void  orc_set_pipe(orc_sim *S, double R);
void  orc_set_channel(orc_sim *S, double y_lo, double y_hi, double u_lo, double u_hi, int chain);
int   orc_add_spheres(orc_sim *S, int n, const double *X, const double *R, double density_ratio,
                      const double *U, const double *W, int fixed);
int   orc_step(orc_sim *S, int nsteps, int bc);
void  orc_macro(const orc_sim *S, double *rho, double *u);
void  orc_get_solid(const orc_sim *S, unsigned char *solid, int *owner);
long long orc_num_links(const orc_sim *S);
void  orc_get_links(const orc_sim *S, long long *cell, int *dir, int *scheme, double *q, int *pid);
int   orc_num_particles(const orc_sim *S);
void  orc_get_particles(const orc_sim *S, double *X, double *U, double *W, double *F, double *T);
long long orc_num_markers(const orc_sim *S);
void  orc_get_markers(const orc_sim *S, double *X, double *F, double *dV, int *pid);
void  orc_get_ibm_force(const orc_sim *S, double *F);
void  orc_stats(const orc_sim *S, int flags, orc_stats_t *out);
void  orc_masked_velocity(const orc_sim *S, int flags, double *u);
double orc_marker_residual(const orc_sim *S, int pass);
void  orc_particles_advance(orc_sim *S, int nsteps);

#ifdef __cplusplus
}
#endif
#endif
