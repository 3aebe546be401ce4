// Internal definitions of the GB300 lattice Boltzmann library: the context
// that the C ABI hands out, profiling groups and the launcher prototypes.
// Device-side definitions are in lbm_device.cuh.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <vector>

#include "lbm.h"
#include "lbm_device.cuh"

namespace lbmgb {

// ------------------------------------------------------------ context -----
struct Ctx {
    lbm_grid g;
    int nx, ny, nz;
    long long N;
    double tau, F[3];
    int storage, rates;
    int q = 19;  // velocity set: 19 (every path) or 27 (periodic box or pipe with IBB, BGK)
    unsigned *q27_colmask;  // D3Q27 pipe: per (x, y) column, the directions whose column is solid
    unsigned *q27_hmask;    // D3Q27 pipe: per column, the wall directions with q >= 1/2
    void *q27_coef;         // D3Q27 pipe: per column and direction, the two wall weights
    Rates rt;
    cudaStream_t stream;
    char *ws;
    size_t ws_bytes;
    // fields
    void *fA, *fB;
    uint8_t *flags;
    int *owner, *aux;
    // compact sites (IBB boundary cells or IBM support cells)
    long long max_sites;
    int *site_cell, *site_first;
    unsigned *site_mask;
    // IBM per site: (rho, u*) as 4 values, accumulated force, force of the
    // current pass, in the storage's arithmetic type (double for FP64, else float)
    void *sup_ru, *sup_F, *sup_Fp;
    // links
    long long max_links;
    int *link_cell, *link_pid;
    int8_t *link_dir, *link_scheme;
    double *link_q;
    void *link_dP, *link_dT;  // per-link momentum exchange and torque (arithmetic type of the storage)
    // row segments of the fluid extent (IBB walls with a solid margin)
    uint4 *seg;  // warp items of the pipe sweep (segments.h)
    long long nseg, max_seg;
    // static wall (pipe) links regrouped by direction for the ghost pass:
    // x = cell | scheme << 30, y = bits of q rounded to FP32
    uint2 *slink;
    int slink_off[20];  // first link of each direction, and the total
    int static_links;   // 1: the ghost pass uses slink (FP32-arithmetic storages)
    long long static_single;  // single-node (scheme 2) links of the static wall
    // wall cells' post-collision populations, written by the sweep for the
    // next ghost pass: 19 values (storage type) per wall cell in cell order
    int *slink_rank;    // per static link: rank of its wall cell
    uint4 *slink4;      // per static link: upstream cell | flags, two weights, wall-cell rank
    int slink4_ready;   // 1: the records hold every static link
    uint2 *seg_bnd;     // per sweep item: rank of its first wall cell, lane mask of wall cells
    void *bvals;
    long long max_bvals;
    // compact ghosts: the ghost pass stores the bounced values here (one per
    // link, storage type) instead of in the solid nodes' slots; per wall
    // cell (rank) a record {first value, mask of the directions it replaces}
    uint2 *wrec;
    int *gidx;          // per static link: index of its value
    void *gvals;
    int bvals_ready;    // the tables above are built
    int pipe_nowrap;    // no fluid cell on an x or y face: pulls wrap only in z (lean pipe sweep)
    // what the last sweep left for the next step's wall: 0 nothing (read
    // the populations), 1 bvals holds the wall cells' values of the current
    // state, 2 gvals holds the partial values p of the inline wall form
    int bvals_valid;
    uint2 *wcoef;       // inline wall form: per compact value k1, k2 (bit 31: q >= 1/2)
    unsigned short *wlane;  // inline wall form: per compact value its wall cell's sweep lane | direction << 5
    // the pair sweep of 16-bit storage (sweep_pair16.cu): items of up to 32
    // cell pairs, per item {first slot, links, 64-bit wall-cell mask}, per
    // compact value the cell of its item | direction << 6
    uint4 *pair_items, *pair_wall;
    unsigned short *wslot;
    long long npair_items;
    int pair_ready;
    int wcoef_ready;
    // compaction scratch
    int nblk;
    long long *blk_sites, *blk_links;
    long long *d_counts;  // [0] sites, [1] links, [2] refill nodes, [3] closure samples, [4] single-node links
    int *sn_list;         // links of the single-node scheme (link indices), d_counts[4] of them
    int *refill_list, *refill_pid;
    long long max_refill;
    long long nsites, nlinks;   // host copies (valid after a sync)
    long long nsites_hint;      // launch sizing: a bound on the device count
    long long nlinks_hint;
    // particles (FP64)
    int max_np, np, fixed;
    double dens;
    double *X, *Xold, *U, *W, *R, *mass, *inertia, *Fh, *Th, *Fprev, *Tprev, *Fc, *Iu, *Ir;
    int *has_prev;
    float4 *Xf;  // FP32 centre and radius (contact search)
    // markers
    long long max_markers, nm;
    double *mX, *mUnit, *mdV, *mFacc;
    void *mUd, *mFaccR;  // desired marker velocity, pass force sum (arithmetic type of the storage)
    void *mFr;  // marker forces of the pass in the arithmetic type (spreading)
    int *mB;    // per marker: first stencil node floor(X) - 1 (3 ints, wrapped)
    void *mE;   // per marker: X - floor(X) in the arithmetic type (3 values)
    int *mpid, *m_first;
    double rd;  // marker retraction (IBM-B: 0.4)
    double max_radius;
    // pipe IBM: ring markers per plane and, per (x, y) column, the ring
    // markers whose 4x4 footprint covers it with their x-y weights
    int pipe_nc;
    double pipe_dV;
    int *pipe_xy_start, *pipe_xy_j;
    void *pipe_xy_w;  // x-y weights in the storage's arithmetic type
    long long pipe_max_xy;
    // pipe interpolation: per ring marker, 16 (support site in a plane, x-y
    // weight) entries; pipe_sp = support sites per z plane (0: not built)
    int *pipe_it_k;
    void *pipe_it_w;  // arithmetic type of the storage
    int pipe_sp, pipe_max_ring;
    // statistics scratch
    double *rho_f, *u_f, *partials;
    unsigned long long *near_key;  // nearest particle surface per cell (diag.cu)
    // status
    unsigned *d_status;
    unsigned *h_status;
    cudaEvent_t ev_status;
    bool status_pending;
    double wait_limit_s;  // bound of the host waits on the stream (lbm_set_wait_limit)
    // geometry
    int has_pipe;
    double pipe_R, pipe_cx, pipe_cy;
    int armed_bc;
    long long step;
    bool broken;
    bool initialised_pops;
    char err[256];
    // learned closure: weights, scales and sample buffers
    float *cl_w, *cl_X, *cl_Y, *cl_eps;
    int *cl_cells;
    void *cl_pk;
    long long max_cl, cl_last_n;
    double cl_uscale, cl_gscale;
    int cl_ready;
    // profiling
    long long launches;                 // every kernel launched
    long long group_launches[LBM_NGROUPS];
    int prof_on;
    void *prof;                         // host-side event records (lbm_api.cu)
};

// every launcher calls this once per kernel it launches
inline void count_launch(Ctx &c, int group, int n = 1) {
    c.launches += n;
    c.group_launches[group] += n;
}
enum { G_BULK = 0, G_BND = 1, G_IBM = 2, G_IBMCOL = 3, G_PART = 4, G_GEOM = 5, G_STATS = 6, G_OTHER = 7, G_CLOSURE = 8 };

}  // namespace lbmgb

struct lbm_ctx {
    lbmgb::Ctx c;
};

// ------------------------------------------------ cross-file launchers ----
namespace lbmgb {
cudaError_t launch_init_equilibrium(Ctx &c, const double *u_dev, double rho0);
cudaError_t launch_set_populations(Ctx &c, const double *f_dev);
cudaError_t launch_get_populations(Ctx &c, double *f_dev);
cudaError_t launch_stream_collide(Ctx &c, int bc);
bool launch_pipe_sweep(Ctx &c, cudaError_t &err);  // sweep_pipe.cu: false when it does not apply
bool pipe_inline_walls(const Ctx &c);             // the lean sweep runs the inline wall form
bool launch_pair16_sweep(Ctx &c, cudaError_t &err);  // sweep_pair16.cu: false when it does not apply
bool build_pair16(Ctx &c, const uint8_t *fl, const std::vector<int> &bcells, const std::vector<uint2> &wr);
cudaError_t launch_pipe_wall_prime(Ctx &c);       // partial values p from the populations
cudaError_t launch_ibb_links(Ctx &c);
cudaEvent_t prof_event(Ctx &c);  // profiling event on the stream (null when off)
void prof_span(Ctx &c, int g, cudaEvent_t a, cudaEvent_t b);  // time from a to b into group g
cudaError_t launch_ibm_collide(Ctx &c);
cudaError_t launch_pipe_flags(Ctx &c);
cudaError_t launch_sphere_mark(Ctx &c, bool clear_old);
cudaError_t launch_refill(Ctx &c);
cudaError_t launch_finish_geometry(Ctx &c);
cudaError_t build_sites(Ctx &c, int mode);  // mode 1: IBB links, 2: IBM support
cudaError_t launch_gimem(Ctx &c);
cudaError_t launch_release(Ctx &c);
cudaError_t launch_particle_update(Ctx &c);
cudaError_t launch_markers_place(Ctx &c);
cudaError_t launch_marker_offsets(Ctx &c);
cudaError_t launch_support_mark(Ctx &c);
cudaError_t launch_ibm_passes(Ctx &c);
cudaError_t launch_ibm_particle_sums(Ctx &c, bool init_only);
cudaError_t launch_ibm_rigid_overwrite(Ctx &c);
cudaError_t launch_macro(Ctx &c, int mask_mode, float *u32 = nullptr);
cudaError_t launch_mask(Ctx &c);  // statistics velocity: solid cells take the rigid-body velocity
cudaError_t run_spectrum(Ctx &c, int flags, int nbins, double *E, double *D);
cudaError_t run_pipe_profiles(Ctx &c, int flags, int nbins, double *out);
size_t pipe_profile_scratch_bytes(int nbins);
cudaError_t run_tke_budget(Ctx &c, int flags, int nbins, double *out);
// D3Q27 periodic box (q27.cu)
cudaError_t launch_q27_step(Ctx &c);
cudaError_t launch_q27_init(Ctx &c, const double *u_dev, double rho0);
cudaError_t q27_plane_copy(Ctx &c, int i, bool to_f64);
cudaError_t launch_q27_macro(Ctx &c);
void q27_pipe_colmask(const Ctx &c, std::vector<unsigned> &mask);
cudaError_t launch_q27_coef(Ctx &c);
size_t tke_budget_scratch_bytes(int nbins);
size_t spectrum_scratch_bytes(long long N, int nbins);
cudaError_t run_stats(Ctx &c, int flags, lbm_stats_t *out);
cudaError_t closure_samples(Ctx &c, double u_scale, float *X, int *cells, long long cap, long long *n_out);
cudaError_t closure_targets(Ctx &c, const int *cells, long long n, double g_scale, float *T);
size_t mlp_pack_bytes();
cudaError_t mlp_pack_device(const float *w, void *pk, cudaStream_t s);
// tensor-core (tcgen05) closure inference, closure_tc.cu
cudaError_t mlp_forward_tc(const float *X, long long n, const float *w, const void *pk, float *Y, int *err,
                           cudaStream_t s);
cudaError_t mlp_train_tc(const float *X, const float *T, long long s0, long long s1, const float *w, const void *pk,
                         float *gpart, float *lpart, int max_blocks, int *err, cudaStream_t s, int *nblk_out);
cudaError_t closure_eps_tc(const Ctx &c, const float *u32, const int *cells, const int *pid, const long long *count,
                           long long cap, const void *pk, float *eps_o, int *err);
}  // namespace lbmgb
