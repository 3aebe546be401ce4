/* lbm.h -- C ABI of the GB300 (sm_103a) lattice Boltzmann library with
 * interpolated bounce-back (IBB) and immersed boundary (IBM) no-slip walls.
 *
 * What it computes: the method compared in Peng et al., "Comparative study
 * of IBB and IBM in the lattice Boltzmann method, Part II: turbulent flows"
 * (arXiv:1906.05448): a D3Q19 MRT lattice Boltzmann fluid driven by a body
 * force (Sec. 2.1), with no-slip walls on a pipe (Sec. 2.1, Table 1) and on
 * moving spheres (Sec. 3.1, Table 2) realised either by interpolated
 * bounce-back (quadratic/linear Bouzidi with single-node fallback,
 * Galilean-invariant momentum exchange, refill of uncovered nodes) or by
 * direct-forcing IBM (Uhlmann, or Breugem with r_d = 0.4, Peskin 4-point
 * delta, two extra forcing iterations, Kempe inner-fluid inertia), with
 * particle motion in FP64 and the statistics of Secs. 2.2 and 3.2.
 *
 * Conventions for every call:
 *  - Lattice units (dx = dt = 1). Node (x,y,z) sits at coordinate (x,y,z).
 *  - Scalar fields: idx = x + nx*(y + ny*z). Vector fields: three planes,
 *    v[c*N + idx]. Populations: 19 planes, f[i*N + idx], velocity order
 *    0:(0,0,0) 1:(1,0,0) 2:(-1,0,0) 3:(0,1,0) 4:(0,-1,0) 5:(0,0,1) 6:(0,0,-1)
 *    7:(1,1,0) 8:(-1,-1,0) 9:(1,-1,0) 10:(-1,1,0) 11:(1,0,1) 12:(-1,0,-1)
 *    13:(1,0,-1) 14:(-1,0,1) 15:(0,1,1) 16:(0,-1,-1) 17:(0,1,-1) 18:(0,-1,1).
 *  - Particle arrays are (n,3) row-major FP64 on the host.
 *  - Host pointers are read during the call only and never retained.
 *  - Device memory: the caller owns one device buffer (the workspace) of at
 *    least lbm_workspace_bytes() bytes, 256-byte aligned, alive until
 *    lbm_destroy(). The library allocates no device memory of its own; it
 *    allocates a small pinned host block for status words.
 *  - Every kernel is launched on the caller's CUDA stream given at create.
 *    Calls that return host data synchronise that stream; lbm_step does not.
 *  - Errors: every call returns an lbm_status; lbm_last_error() gives a
 *    one-line reason. After LBM_EUNSTABLE or LBM_ECUDA the context accepts
 *    only lbm_stats / lbm_get_* / lbm_destroy (others return LBM_ESTATE).
 *  - One context per host thread at a time.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,      /* bad argument (sizes, pointers, enum values) */
    LBM_ENOMEM = 2,      /* workspace too small or a capacity exceeded */
    LBM_ECUDA = 3,       /* a CUDA call failed; detail in lbm_last_error */
    LBM_EUNSTABLE = 4,   /* the watchdog saw NaN/Inf, rho outside [0.5,2] or |u| > 0.3 */
    LBM_ETIMEOUT = 5,    /* a bounded host wait on the stream ran out */
    LBM_ESTATE = 6,      /* call not allowed in the current state */
    LBM_EUNSUPPORTED = 7, /* combination not built */
    LBM_EIO = 8           /* a checkpoint file could not be opened, read or written, or is truncated */
} lbm_status;

/* No-slip treatment used by lbm_step (Sec. 2.1, Sec. 3.1). */
typedef enum {
    LBM_BC_NONE = 0,  /* plain periodic box: geometry ignored */
    LBM_BC_IBB = 1,   /* interpolated bounce-back */
    LBM_BC_IBM_U = 2, /* direct-forcing IBM, markers on the surface (r_d = 0) */
    LBM_BC_IBM_B = 3  /* direct-forcing IBM, markers retracted by r_d = 0.4 */
} lbm_bc;

/* Population storage in HBM. F64/F32 store f_i - w_i in that precision;
 * F16S/BF16S store f_i - w_i in 16 bits (FP16 scaled by 2^10, or BF16),
 * always with FP32 collision arithmetic. */
typedef enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16S = 2, LBM_BF16S = 3 } lbm_storage;

/* Relaxation rates: SRT = all non-conserved moments at 1/tau (the
 * single-parameter setting of Sec. 2.1); DHUMIERES = the multiple rates of
 * d'Humieres et al. 2002 used in Sec. 3.1 (shear moments at 1/tau). */
typedef enum { LBM_RATES_SRT = 0, LBM_RATES_DHUMIERES = 1 } lbm_rates;

/* Sphere capacity limit: the statistics pack a particle id into 20 bits. */
#define LBM_MAX_PARTICLES 1048575

typedef struct {
    int nx, ny, nz;          /* grid, each >= 4, nx*ny*nz < 2^31 */
    int storage;             /* lbm_storage */
    int rates;               /* lbm_rates */
    int max_particles;       /* capacity for spheres (0: none; at most LBM_MAX_PARTICLES) */
    long long max_links;     /* IBB link capacity (0: derived from the grid and max_particles) */
    long long max_markers;   /* IBM marker capacity (0: derived) */
    long long max_sites;     /* boundary / support cell capacity (0: derived) */
    int lattice;             /* velocity set: 0 or 19 D3Q19 (every path); 27 D3Q27, the set of the
                                paper's pipe solver (Sec. 2.1): periodic box (LBM_BC_NONE), BGK
                                (LBM_RATES_SRT), FP64 or FP32 storage, and the pipe wall
                                (lbm_set_pipe, LBM_BC_IBB); spheres, IBM and the MRT rates answer
                                LBM_EUNSUPPORTED. Populations in and out (lbm_set_populations,
                                LBM_FIELD_POPS) then hold 27 planes: rest, 6 faces, 12 edges, 8
                                corners, each group in lexicographic order of (c_x, c_y, c_z) over
                                {-1, 0, 1}^3, c_x slowest. */
} lbm_grid;

/* Bytes of device workspace lbm_create needs for this grid. 0 on bad input. */
size_t lbm_workspace_bytes(const lbm_grid *grid);

/* Create a context (Sec. 2.1 problem statement: periodic box, relaxation
 * time tau > 0.5, uniform body force per unit volume `force` acting on the
 * fluid cells). Populations start at equilibrium with rho = 1, u = 0.
 * dev_workspace: caller-owned device buffer (see conventions);
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Errors: LBM_EINVAL (bad grid/tau/pointers), LBM_ENOMEM (bytes too small),
 * LBM_ECUDA. */
lbm_status lbm_create(const lbm_grid *grid, double tau, const double force[3], void *dev_workspace,
                      size_t bytes, void *cuda_stream, lbm_ctx **out);

/* Set every population to f_eq(rho0, u) from a host velocity field u
 * (3*N doubles, component-major). Synchronous. Only before the first step. */
lbm_status lbm_init_velocity(lbm_ctx *ctx, const double *u_host, double rho0);

/* Set the populations from a host array of 19*N doubles (unshifted f_i). */
lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f_host);

/* Pipe along z, centre ((nx-1)/2, (ny-1)/2), radius R: cells with
 * (x-cx)^2 + (y-cy)^2 >= R^2 are outside (Sec. 2.1). Exclusive with spheres. */
lbm_status lbm_set_pipe(lbm_ctx *ctx, double radius);

/* Add n spheres (Sec. 3.1): centres xyz (n,3), radii (n), particle/fluid
 * density ratio. vel/omega may be NULL: then the translation velocity is the
 * fluid velocity averaged over the particle volume and the rotation is zero
 * (the release of Sec. 3.1). fixed != 0 holds the particles in place (their
 * velocities still move the wall). Once per context, before the first step. */
lbm_status lbm_add_spheres(lbm_ctx *ctx, int n, const double *xyz, const double *radius, double density_ratio,
                           const double *vel, const double *omega, int fixed);

/* Advance nsteps time steps with no-slip treatment bc. The first call fixes
 * bc for the life of the context (another bc later returns LBM_ESTATE).
 * Asynchronous on the stream: instability found by the watchdog of one call
 * is reported by the next call that synchronises (lbm_step when the previous
 * check has completed, lbm_stats, lbm_get_*). */
lbm_status lbm_step(lbm_ctx *ctx, int nsteps, int bc);

/* Bound, in seconds, of the host waits on the stream: calls that return
 * host data first wait for the work already enqueued. Default 600 s. A wait
 * that runs out returns LBM_ETIMEOUT and leaves the context usable: the
 * work stays enqueued, and a later call waits for it again. seconds must be
 * positive and at most 1e6, else LBM_EINVAL. */
lbm_status lbm_set_wait_limit(lbm_ctx *ctx, double seconds);

/* Checkpoint and restart (Sec. 2.2: the IBM-U pipe run was restarted from
 * the IBM-B flow field). lbm_checkpoint writes to the file `path` everything
 * the next step reads: the populations in their storage format, the step
 * count, the wall treatment, the relaxation rates, the geometry (pipe radius,
 * or the spheres' centres, radii, density ratio and fixed flag), the FP64
 * particle state (U, W, the hydrodynamic force and torque of the last two
 * steps, the contact force, the inner-fluid integrals of the IBM), the IBM
 * force of the last step per support cell and per marker, and the closure
 * weights. Syncs.
 * lbm_restore reads such a file into a context created with the same grid
 * (nx, ny, nz, storage, lattice), tau and force, capacities at least as
 * large, and nothing set yet (no populations, geometry or step). The
 * restored context then steps bit for bit as the saved one would have.
 * Format: a fixed header and raw arrays in host byte order (not portable
 * across byte orders). Errors: LBM_EINVAL (null path; restore: a file of
 * another grid, tau or force), LBM_ESTATE (checkpoint of a context left
 * unusable by an error; restore into a context that is not fresh),
 * LBM_ENOMEM (capacities too small), LBM_EIO (open, read or write failed,
 * truncated file, not a checkpoint), LBM_ECUDA. */
lbm_status lbm_checkpoint(lbm_ctx *ctx, const char *path);
lbm_status lbm_restore(lbm_ctx *ctx, const char *path);

#define LBM_STATS_UNMASK 1   /* IBM: statistics on the raw virtual fluid inside particles */
#define LBM_STATS_BINS 4     /* radial profiles around particles (Sec. 3.2) */
#define LBM_STATS_CLOSURE 8  /* near-surface gradients from the learned closure (lbm_closure_set_weights) */
#define LBM_NBINS 40

typedef struct {
    double mass, momentum[3];
    double kinetic_energy, dissipation;             /* averages over all cells (masked velocity) */
    double kinetic_energy_fluid, dissipation_fluid; /* averages over cells outside solids */
    double particle_ke, particle_ake;               /* sum 1/2 m U^2, sum 1/2 I W^2 */
    double force[3], torque[3];                     /* summed hydrodynamic force / torque on particles */
    double bulk_velocity;                           /* pipe: mean u_z inside */
    int nbins;
    double bin_r[LBM_NBINS], bin_tke[LBM_NBINS], bin_eps[LBM_NBINS];
    long long bin_count[LBM_NBINS];
    long long nfluid, nlinks, nmarkers, step;
} lbm_stats_t;

/* Statistics of the current state (Sec. 3.2 masking, 2nd-order central
 * differences, dissipation 2 nu s_ij s_ij; Sec. 2.2 bulk velocity). Syncs. */
lbm_status lbm_stats(lbm_ctx *ctx, int flags, lbm_stats_t *out);

/* Three-dimensional spectra of kinetic energy and dissipation of the
 * current state (Sec. 3.2), on a periodic cube of side n = nx = ny = nz, n a
 * power of two in [8, 1024]:
 *   u_hat(k) = (1/N) sum_x u(x) exp(-2 pi i k.x / n), N = n^3, with the
 *   velocity of lbm_stats (solid cells masked with the rigid-body velocity
 *   unless IBM statistics are asked for with LBM_STATS_UNMASK in flags);
 *   E[K] = sum over wave vectors with round(|k|) = K of (1/2)|u_hat(k)|^2,
 *   summed over the three components (sum of E = mean kinetic energy);
 *   D[K] = the same sum of 2 nu (2 pi |k| / n)^2 (1/2)|u_hat(k)|^2, nu =
 *   (tau - 1/2)/3 (sum of D = spectral dissipation).
 * E and D: host arrays of nbins doubles (1 <= nbins <= LBM_SPECTRUM_MAX_BINS);
 * shells K >= nbins are left out. The transform runs in FP32 on the device
 * and the shell sums in FP64. Scratch: the population buffer that the next
 * step overwrites, so the call allocates nothing and must not overlap a
 * step on another stream. Syncs. Errors: LBM_EINVAL (arguments),
 * LBM_EUNSUPPORTED (not such a cube), LBM_ENOMEM (scratch too small). */
#define LBM_SPECTRUM_MAX_BINS 2048
lbm_status lbm_spectrum(lbm_ctx *ctx, int flags, int nbins, double *E, double *D);

/* Radial profiles of the pipe (Sec. 2.2: statistics against the distance
 * to the axis), for the cells inside the pipe, in nbins bins
 * b = floor(r nbins / R), r the distance to the axis (cells at
 * ((nx-1)/2, (ny-1)/2)). out: host array of nbins x LBM_PROF_NQ doubles,
 * bin-major; per bin the number of cells, then the means over its cells of
 * u_r, u_theta, u_z, u_r^2, u_theta^2, u_z^2, u_r u_z, u_r u_theta,
 * u_theta u_z, rho and 2 nu s_ij s_ij (central differences). The velocity is
 * that of lbm_stats (LBM_STATS_UNMASK in flags as there). One snapshot:
 * time averages are the caller's sums over calls. Scratch: the population
 * buffer that the next step overwrites. Syncs. Errors: LBM_EINVAL,
 * LBM_ESTATE (no pipe), LBM_ENOMEM. */
#define LBM_PROF_NQ 12
#define LBM_PROF_MAX_BINS 256
lbm_status lbm_pipe_profiles(lbm_ctx *ctx, int flags, int nbins, double *out);

/* Non-shear relaxation rates of the MRT collision by d'Humieres group:
 * energy e (bulk viscosity (2/9)(1/s_e - 1/2); the BGK value 2 nu / 3 at
 * s_e = 1/tau), energy square eps, energy flux q, pi_xx and pi_ww, and the
 * third-order m modes. The shear rate stays 1/tau. The paper's solver has
 * this knob for damping acoustic noise and leaves it off (Sec. 2.2). The
 * context switches to the multiple-relaxation-time collision; the rates
 * apply from the next step. Each rate must lie in (0, 2). Errors:
 * LBM_EINVAL. */
lbm_status lbm_set_mrt_rates(lbm_ctx *ctx, double s_e, double s_eps, double s_q, double s_pi, double s_m);

/* Component-wise TKE budget of the pipe (Eq. 1a-c, Sec. 2.2) of the current
 * snapshot, in the radial bins of lbm_pipe_profiles (cells with r > 0).
 * Averages are means over a bin's cells and fluctuations are departures
 * from them; velocity gradients are central differences of the statistics
 * velocity (LBM_STATS_UNMASK in flags as for lbm_stats) rotated into
 * (e_r, e_theta, e_z); p' = c_s^2 rho'; d/dr of a binned profile is a
 * central difference over the bin centres (b + 1/2) R / nbins, one-sided at
 * the ends. out: host array of nbins x LBM_BUDGET_NT doubles, bin-major:
 * the cell count, then E_Oz, E_Tz, E_Pz, E_Vz, E_Dz, E_Tr, E_Pr, E_Vr, E_Dr,
 * E_Ttheta, E_Ptheta, E_Vtheta, E_Dtheta (production, turbulent transport,
 * pressure work, viscous diffusion, dissipation); empty bins hold zeros.
 * One snapshot: time averages are the caller's. Scratch: the population
 * buffer that the next step overwrites. Syncs. Errors: LBM_EINVAL (bins
 * outside 1..LBM_PROF_MAX_BINS, null out), LBM_ESTATE (no pipe),
 * LBM_ENOMEM (scratch larger than that buffer). */
#define LBM_BUDGET_NT 14
lbm_status lbm_tke_budget(lbm_ctx *ctx, int flags, int nbins, double *out);

#define LBM_FIELD_RHO 0      /* N doubles */
#define LBM_FIELD_U 1        /* 3N doubles */
#define LBM_FIELD_POPS 2     /* 19N doubles, unshifted f_i (post-collision state) */
#define LBM_FIELD_FLAGS 3    /* N bytes: bit0 solid, bit1 IBB boundary cell, bit2 IBM support cell */
#define LBM_FIELD_IBM_FORCE 4 /* 3N doubles: IBM force of the last step */

/* Copy a field to host memory dst of `bytes` bytes. Syncs. Populations of
 * solid cells under IBB are undefined; rho and u report 0 there. */
lbm_status lbm_get_field(lbm_ctx *ctx, int which, void *dst, size_t bytes);

/* Number of IBB boundary links of the current geometry. */
lbm_status lbm_num_links(lbm_ctx *ctx, long long *n);

/* Boundary links sorted by (cell, dir): fluid cell, direction i with
 * cell + c_i solid, scheme (0 quadratic, 1 linear, 2 single-node), wall
 * fraction q in (0,1] (FP64), owning particle (-1 for the pipe). Each array
 * holds at least `capacity` entries. Syncs. */
lbm_status lbm_get_links(lbm_ctx *ctx, long long capacity, long long *cell, int *dir, int *scheme, double *q,
                         int *pid);

/* Number of spheres of the context (0 without particles). */
lbm_status lbm_num_particles(lbm_ctx *ctx, int *n);

/* Particle state (n,3) arrays; any pointer may be NULL. F/T are the
 * hydrodynamic force and torque of the last step. Syncs. */
lbm_status lbm_get_particles(lbm_ctx *ctx, double *X, double *U, double *W, double *F, double *T);

/* IBM markers of the current step: positions (m,3), accumulated force
 * density (m,3), volume (m), owner (m; -1 for the pipe). Syncs. */
lbm_status lbm_num_markers(lbm_ctx *ctx, long long *n);
lbm_status lbm_get_markers(lbm_ctx *ctx, long long capacity, double *X, double *F, double *dV, int *pid);

/* Per-kernel-group timing with CUDA events recorded on the library's stream
 * around each group of launches, and a count of every kernel launch.
 * Groups: 0 bulk stream-collide sweep, 1 IBB boundary cells, 2 IBM forcing
 * passes, 3 IBM support-cell collision, 4 particle force/motion, 5 geometry
 * update (flags, refill, link or support lists), 6 statistics, 7 other
 * (the IBM rigid-body overwrite), 8 the closure's tensor-core inference
 * inside lbm_stats (LBM_STATS_CLOSURE).
 * enable = 1 starts recording (and clears totals), 0 stops; out (nullable)
 * receives the totals since the last enable, after synchronising. */
#define LBM_NGROUPS 9
typedef struct {
    double ms[LBM_NGROUPS];
    long long spans[LBM_NGROUPS];     /* timed spans per group */
    long long launches[LBM_NGROUPS];  /* kernels launched per group */
    long long total_launches;         /* every kernel launched since create */
} lbm_profile_t;
lbm_status lbm_profile(lbm_ctx *ctx, int enable, lbm_profile_t *out);

/* ---------------------------------------------------------------------
 * Learned near-surface gradient closure. The paper finds that IBM cannot
 * resolve the velocity gradients inside its diffused interface, so the
 * local dissipation near particle surfaces comes out too low (Sec. 3.2,
 * Sec. 4). A perceptron 85 -> 64 -> 64 -> 64 (ReLU) -> 9 maps the IBM
 * velocity stencil around a near-surface node to its 9 velocity
 * gradients; it is trained on pairs produced by the method itself (IBM
 * features, IBB gradients from the same initial state). Tensor cores:
 * BF16 operands, FP32 accumulation, FP32 master weights.
 * Parameter vector (FP32, 14409 values): W1 (85x64, [in][out]), b1 (64),
 * W2 (64x64), b2, W3 (64x64), b3, W4 (64x9), b4 (9).
 * Features per node (85): u - u_rb at the 27 nodes x + (dx,dy,dz),
 * dz, dy, dx in -1..1 (dz outermost), 3 components each, divided by
 * u_scale; the distance to the nearest particle surface (lattice units);
 * u - u_rb at the node again (3). u_rb: rigid-body velocity of the nearest
 * particle. Outputs: du_a/dx_b at index 3a + b, times g_scale.
 * --------------------------------------------------------------------- */
#define LBM_MLP_NPARAM 14409

/* Device workspace for the lbm_mlp_* calls (caller-owned, 256-byte aligned). */
size_t lbm_mlp_workspace_bytes(void);
int lbm_mlp_num_params(void);

/* Y (n x 9) = network(X (n x 85)) for FP32 device arrays; w_dev: the FP32
 * parameter vector on the device. Asynchronous on `stream`. */
lbm_status lbm_mlp_forward(const float *X_dev, long long n, const float *w_dev, float *Y_dev, void *ws,
                           size_t ws_bytes, void *stream);

/* Mean squared error over the n samples and 9 outputs and its gradient
 * with respect to the parameters (grad_dev: 14409 floats). Synchronous when
 * loss != NULL. */
lbm_status lbm_mlp_loss_grad(const float *X_dev, const float *T_dev, long long n, const float *w_dev,
                             float *grad_dev, double *loss, void *ws, size_t ws_bytes, void *stream);

/* Adam (lr, beta = 0.9/0.999, eps = 1e-8) over consecutive mini-batches of
 * the given (pre-shuffled) samples, `epochs` times; w_dev is updated in
 * place. last_epoch_loss (nullable) receives the mean loss of the last
 * epoch's batches (evaluated before each update). */
lbm_status lbm_mlp_train(const float *X_dev, const float *T_dev, long long n, int epochs, int batch, double lr,
                         float *w_dev, void *ws, size_t ws_bytes, void *stream, double *last_epoch_loss);

/* Features of the near-surface fluid nodes (distance to the nearest
 * surface in (0, 2]) of the current state into X_dev (capacity x 85) and
 * their cell indices into cells_dev; *n receives the count (order not
 * fixed). LBM_ENOMEM when more than `capacity` nodes exist. Syncs. */
lbm_status lbm_closure_samples(lbm_ctx *ctx, double u_scale, float *X_dev, int *cells_dev, long long capacity,
                               long long *n);

/* Central-difference gradients of the current (rigid-body masked)
 * velocity at the given cells, times g_scale, into T_dev (n x 9); NaN where
 * the cell is solid in this state. Syncs. */
lbm_status lbm_closure_targets(lbm_ctx *ctx, const int *cells_dev, long long n, double g_scale, float *T_dev);

/* Weights (host FP32, 14409) and scales used by lbm_stats(LBM_STATS_CLOSURE):
 * near-surface nodes then take their gradients, hence their dissipation,
 * from the network. Needs max_particles > 0. */
lbm_status lbm_closure_set_weights(lbm_ctx *ctx, const float *w_host, int n, double u_scale, double g_scale);

/* Kinetic energy and dissipation of a velocity field already in device
 * memory, computed without allocating anything. The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc, e.g.
 * solvers whose device memory all belongs to another framework's pool (an
 * allocation beside it would escape that pool's accounting or exceed its
 * limit), or loops that must not pay cudaMalloc's implicit device
 * synchronisation.
 * u_dev: 3*N doubles (component-major, x fastest), N = nx*ny*nz, device.
 * nu: kinematic viscosity. out_dev: 2 doubles on the device, receiving the
 * box averages of 1/2 |u|^2 and 2 nu s_ij s_ij (periodic central
 * differences), the same quantities lbm_stats reports as kinetic_energy and
 * dissipation for an unmasked field. Launched on cuda_stream; asynchronous.
 * Scratch: a fixed 512 KiB device array inside the library (held by every
 * GPU that loads it until exit), shared by all calls: calls that overlap on
 * the GPU race on it. N above lbm_field_energy_noalloc_max_cells()
 * (134,217,728 = 512^3) is refused with LBM_ENOMEM; bad pointers or sizes
 * give LBM_EINVAL; a launch that fails gives LBM_ECUDA (an error left
 * pending by earlier, unrelated work is neither reported nor cleared). The
 * first call on a device looks the scratch address up
 * (cudaGetSymbolAddress); make that first call before any stream capture. */
lbm_status lbm_field_energy_noalloc(const double *u_dev, int nx, int ny, int nz, double nu, double *out_dev,
                                    void *cuda_stream);
long long lbm_field_energy_noalloc_max_cells(void);

const char *lbm_last_error(const lbm_ctx *ctx);
const char *lbm_status_string(int status);
void lbm_destroy(lbm_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
