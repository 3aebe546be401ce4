// Geometry kernels: solid flags of the pipe and of the spheres, refill of
// uncovered nodes, and the ordered compaction that lists IBB boundary cells
// with their links, or IBM support cells.
//
// Solid test and link fraction q are computed in FP64 with explicitly
// rounded operations (no fused multiply-add), in a fixed order, so that a
// given set of particle positions yields bit-identical link lists on every
// run (Sec. 3.1: a sharp interface found by ray-sphere intersection).
#include "lbm_internal.cuh"

namespace lbmgb {

__device__ __forceinline__ double gmimg(double d, int n) {
    if (d > 0.5 * n) d = __dsub_rn(d, (double)n);
    else if (d < -0.5 * n) d = __dadd_rn(d, (double)n);
    return d;
}
__device__ __forceinline__ int gwrap(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}
// |d|^2 summed as ((dx^2 + dy^2) + dz^2)
__device__ __forceinline__ double dist2(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// ------------------------------------------------------------ pipe -------
__global__ void pipe_flags_kernel(uint8_t *flags, int *owner, int nx, int ny, long long N, double pcx, double pcy,
                                  double R) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const int x = (int)(c % nx), y = (int)((c / nx) % ny);
    const double dx = __dsub_rn((double)x, pcx), dy = __dsub_rn((double)y, pcy);
    const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    flags[c] = d2 >= __dmul_rn(R, R) ? FL_SOLID : 0;
    owner[c] = NO_OWNER;
}

cudaError_t launch_pipe_flags(Ctx &c) {
    const unsigned nb = (unsigned)((c.N + 255) / 256);
    count_launch(c, G_GEOM);
    pipe_flags_kernel<<<nb, 256, 0, c.stream>>>(c.flags, c.owner, c.nx, c.ny, c.N, c.pipe_cx, c.pipe_cy, c.pipe_R);
    return cudaGetLastError();
}

// ---------------------------------------------------------- spheres ------
__device__ __forceinline__ void atomic_or_flag(uint8_t *flags, long long c, uint8_t bit) {
    unsigned *w = (unsigned *)(flags + (c & ~3LL));
    atomicOr(w, ((unsigned)bit) << (8 * (c & 3)));
}
__device__ __forceinline__ void atomic_and_flag(uint8_t *flags, long long c, uint8_t keep) {
    unsigned *w = (unsigned *)(flags + (c & ~3LL));
    const unsigned sh = 8 * (unsigned)(c & 3);
    atomicAnd(w, ~((unsigned)(uint8_t)~keep << sh));
}

struct SphereArgs {
    uint8_t *flags;
    int *owner, *aux;
    const double *X, *Xold, *R;
    int nx, ny, nz;
    int keep_owner;  // IBB: record the old owner in aux for the refill
};

// One block per particle over the box floor(X)-r .. floor(X)+r+1, r = ceil(R)+1.
// clear pass: cells owned by p at the old position lose SOLID, gain
// WAS_SOLID, and remember p in aux (needed by the refill).
// mark pass: cells inside p at the new position gain SOLID, owner = lowest id.
template <bool CLEAR>
__global__ void sphere_kernel(SphereArgs a) {
    const int p = blockIdx.x;
    const double *Xp = CLEAR ? a.Xold + 3 * p : a.X + 3 * p;
    const double R = a.R[p];
    const int r = (int)ceil(R) + 1;
    const int bx = (int)floor(Xp[0]) - r, by = (int)floor(Xp[1]) - r, bz = (int)floor(Xp[2]) - r;
    const int w = 2 * r + 2;
    const int total = w * w * w;
    const double R2 = __dmul_rn(R, R);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int x = gwrap(bx + t % w, a.nx), y = gwrap(by + (t / w) % w, a.ny), z = gwrap(bz + t / (w * w), a.nz);
        const long long c = (long long)x + (long long)a.nx * (y + (long long)a.ny * z);
        if (CLEAR) {
            if (a.owner[c] == p) {
                if (a.keep_owner) a.aux[c] = p;
                a.owner[c] = NO_OWNER;
                a.flags[c] = (uint8_t)((a.flags[c] & ~FL_SOLID) | FL_WAS_SOLID);
            }
        } else {
            const double dx = gmimg(__dsub_rn((double)x, Xp[0]), a.nx);
            const double dy = gmimg(__dsub_rn((double)y, Xp[1]), a.ny);
            const double dz = gmimg(__dsub_rn((double)z, Xp[2]), a.nz);
            if (dist2(dx, dy, dz) <= R2) {
                atomicMin(a.owner + c, p);
                atomic_or_flag(a.flags, c, FL_SOLID);
            }
        }
    }
}

cudaError_t launch_sphere_mark(Ctx &c, bool clear_old) {
    if (c.np == 0) return cudaSuccess;
    SphereArgs a{c.flags, c.owner, c.aux, c.X, c.Xold, c.R, c.nx, c.ny, c.nz, c.armed_bc == LBM_BC_IBB};
    count_launch(c, G_GEOM, clear_old ? 2 : 1);
    if (clear_old) sphere_kernel<true><<<c.np, 256, 0, c.stream>>>(a);
    sphere_kernel<false><<<c.np, 256, 0, c.stream>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------ refill ------
struct RefillArgs {
    void *B;
    const uint8_t *flags;
    const int *aux;
    const double *X, *U, *W, *R;
    int nx, ny, nz;
    long long N;
    double F[3];
};

template <typename R, int S>
__device__ double load_f(const void *B, size_t idx) {
    typedef typename Store<S>::T T;
    const T *p = (const T *)B + idx;
    if (S == LBM_F64) return *(const double *)p;
    if (S == LBM_F32) return (double)*(const float *)p;
    if (S == LBM_F16S) return (double)__half2float(*(const __half *)p) / (double)F16_SCALE;
    return (double)__bfloat162float(*(const __nv_bfloat16 *)p);
}

// Caiazzo (2008) refill (Sec. 3.1) of a node that the particle p uncovered:
// rho = mean over fluid neighbours, u = rigid-body velocity, and the
// non-equilibrium part of the fluid neighbour best aligned with the outward
// normal (ties: lowest direction index).
template <int S>
__global__ void refill_kernel(RefillArgs a) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R Rt;
    const int p = blockIdx.x;
    const double *Xp = a.X + 3 * p;
    const int r = (int)ceil(a.R[p]) + 3;
    const int bx = (int)floor(Xp[0]) - r, by = (int)floor(Xp[1]) - r, bz = (int)floor(Xp[2]) - r;
    const int w = 2 * r + 2;
    const int total = w * w * w;
    const size_t N = (size_t)a.N;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int x = gwrap(bx + t % w, a.nx), y = gwrap(by + (t / w) % w, a.ny), z = gwrap(bz + t / (w * w), a.nz);
        const long long c = (long long)x + (long long)a.nx * (y + (long long)a.ny * z);
        const uint8_t fl = a.flags[c];
        if (!(fl & FL_WAS_SOLID) || (fl & FL_SOLID) || a.aux[c] != p) continue;
        double rv[3] = {gmimg((double)x - Xp[0], a.nx), gmimg((double)y - Xp[1], a.ny),
                        gmimg((double)z - Xp[2], a.nz)};
        const double *Up = a.U + 3 * p, *Wp = a.W + 3 * p;
        double uw[3] = {Up[0] + (Wp[1] * rv[2] - Wp[2] * rv[1]), Up[1] + (Wp[2] * rv[0] - Wp[0] * rv[2]),
                        Up[2] + (Wp[0] * rv[1] - Wp[1] * rv[0])};
        const double l = sqrt(rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2]);
        double nrm[3] = {0, 0, 0};
        if (l > 0) {
            nrm[0] = rv[0] / l;
            nrm[1] = rv[1] / l;
            nrm[2] = rv[2] / l;
        }
        double rsum = 0.0, best = -1e300;
        int cnt = 0;
        long long bestc = -1;
#pragma unroll 1
        for (int i = 1; i < 19; i++) {
            const long long nb = (long long)gwrap(x + cx(i), a.nx) +
                                 (long long)a.nx * (gwrap(y + cy(i), a.ny) + (long long)a.ny * gwrap(z + cz(i), a.nz));
            if (a.flags[nb] & (FL_WAS_SOLID | FL_SOLID)) continue;
            double rr = 0.0;
            for (int k = 0; k < 19; k++) rr += load_f<Rt, S>(a.B, k * N + nb) + wgt(k);
            rsum += rr;
            cnt++;
            const double cl = sqrt((double)(cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i)));
            const double al = (nrm[0] * cx(i) + nrm[1] * cy(i) + nrm[2] * cz(i)) / cl;
            if (al > best) {
                best = al;
                bestc = nb;
            }
        }
        const double rho = cnt ? rsum / cnt : 1.0;
        double fe_nb[19];
        bool have = bestc >= 0;
        if (have) {
            double rn = 0.0, j[3] = {0, 0, 0};
            for (int k = 0; k < 19; k++) {
                const double fk = load_f<Rt, S>(a.B, k * N + bestc) + wgt(k);
                fe_nb[k] = fk;
                rn += fk;
                j[0] += fk * cx(k);
                j[1] += fk * cy(k);
                j[2] += fk * cz(k);
            }
            const double un[3] = {(j[0] - 0.5 * a.F[0]) / rn, (j[1] - 0.5 * a.F[1]) / rn, (j[2] - 0.5 * a.F[2]) / rn};
            const double un2 = un[0] * un[0] + un[1] * un[1] + un[2] * un[2];
            for (int k = 0; k < 19; k++) {
                const double cu = cx(k) * un[0] + cy(k) * un[1] + cz(k) * un[2];
                fe_nb[k] -= wgt(k) * rn * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * un2);  // f_neq of neighbour
            }
        }
        const double uw2 = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
        for (int k = 0; k < 19; k++) {
            const double cu = cx(k) * uw[0] + cy(k) * uw[1] + cz(k) * uw[2];
            double f = wgt(k) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uw2);
            if (have) f += fe_nb[k];
            Store<S>::st((T *)a.B + k * N + c, Rt(f - wgt(k)));
        }
    }
}

cudaError_t launch_refill(Ctx &c) {
    if (c.np == 0) return cudaSuccess;
    count_launch(c, G_GEOM);
    RefillArgs a{c.fB, c.flags, c.aux, c.X, c.U, c.W, c.R, c.nx, c.ny, c.nz, c.N, {c.F[0], c.F[1], c.F[2]}};
    switch (c.storage) {
    case LBM_F64: refill_kernel<LBM_F64><<<c.np, 128, 0, c.stream>>>(a); break;
    case LBM_F32: refill_kernel<LBM_F32><<<c.np, 128, 0, c.stream>>>(a); break;
    case LBM_F16S: refill_kernel<LBM_F16S><<<c.np, 128, 0, c.stream>>>(a); break;
    default: refill_kernel<LBM_BF16S><<<c.np, 128, 0, c.stream>>>(a); break;
    }
    return cudaGetLastError();
}

// clear WAS_SOLID around each particle after the refill
__global__ void finish_kernel(uint8_t *flags, const double *X, const double *R, int nx, int ny, int nz) {
    const int p = blockIdx.x;
    const int r = (int)ceil(R[p]) + 3;
    const int bx = (int)floor(X[3 * p]) - r, by = (int)floor(X[3 * p + 1]) - r, bz = (int)floor(X[3 * p + 2]) - r;
    const int w = 2 * r + 2;
    for (int t = threadIdx.x; t < w * w * w; t += blockDim.x) {
        const int x = gwrap(bx + t % w, nx), y = gwrap(by + (t / w) % w, ny), z = gwrap(bz + t / (w * w), nz);
        const long long c = (long long)x + (long long)nx * (y + (long long)ny * z);
        if (flags[c] & FL_WAS_SOLID) atomic_and_flag(flags, c, (uint8_t)~FL_WAS_SOLID);
    }
}

cudaError_t launch_finish_geometry(Ctx &c) {
    if (c.np == 0) return cudaSuccess;
    count_launch(c, G_GEOM);
    finish_kernel<<<c.np, 256, 0, c.stream>>>(c.flags, c.X, c.R, c.nx, c.ny, c.nz);
    return cudaGetLastError();
}

// ------------------------------------------------ site compaction --------
// Cells are processed in tiles of TILE consecutive indices; each tile's
// counts are scanned, so sites and links come out ordered by cell index and
// links of a cell by direction, independent of the launch configuration.
constexpr int CT = 256;        // threads per tile block
constexpr int CPT = 4;         // cells per thread
constexpr int TILE = CT * CPT;

struct SiteArgs {
    uint8_t *flags;
    const int *owner;
    int *aux;
    const double *X, *R;
    int nx, ny, nz;
    long long N;
    double pcx, pcy, pR;
    int mode;
    long long *blk_sites, *blk_links;
    long long *counts;
    int *site_cell, *site_first;
    unsigned *site_mask;
    int *link_cell, *link_pid;
    int8_t *link_dir, *link_scheme;
    double *link_q;
    long long max_sites, max_links;
    unsigned *status;
};

// solid-neighbour mask of a fluid cell (bit l: x + c_l solid)
__device__ __forceinline__ unsigned solid_mask(const SiteArgs &a, int x, int y, int z) {
    unsigned m = 0;
#pragma unroll
    for (int l = 1; l < 19; l++) {
        const int xs = gwrap(x + cx(l), a.nx), ys = gwrap(y + cy(l), a.ny), zs = gwrap(z + cz(l), a.nz);
        const long long nb = (long long)xs + (long long)a.nx * (ys + (long long)a.ny * zs);
        if (a.flags[nb] & FL_SOLID) m |= 1u << l;
    }
    return m;
}

__device__ __forceinline__ void cell_info(const SiteArgs &a, long long c, bool &site, unsigned &mask) {
    site = false;
    mask = 0;
    if (c >= a.N) return;
    const uint8_t fl = a.flags[c];
    if (a.mode == 1) {
        if (fl & FL_SOLID) return;
        const int x = (int)(c % a.nx), y = (int)((c / a.nx) % a.ny), z = (int)(c / ((long long)a.nx * a.ny));
        mask = solid_mask(a, x, y, z);
        site = mask != 0;
    } else {
        site = (fl & FL_SUP) != 0;
    }
}

template <typename V>
__device__ V block_exclusive_scan(V v, V *sh, V &total) {
    // simple two-level scan over CT threads (warp shuffles, then warp sums)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    V inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        V t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        V s = lane < CT / 32 ? sh[lane] : V(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            V t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < CT / 32) sh[lane] = s;
    }
    __syncthreads();
    const V before = wid > 0 ? sh[wid - 1] : V(0);
    total = sh[CT / 32 - 1];
    __syncthreads();
    return before + inc - v;
}

__global__ void __launch_bounds__(CT) site_count_kernel(SiteArgs a) {
    __shared__ long long sh[CT / 32];
    const long long base = (long long)blockIdx.x * TILE + (long long)threadIdx.x * CPT;
    long long ns = 0, nl = 0;
    for (int k = 0; k < CPT; k++) {
        bool site;
        unsigned mask;
        cell_info(a, base + k, site, mask);
        ns += site;
        nl += __popc(mask);
    }
    long long ts, tl;
    block_exclusive_scan<long long>(ns, sh, ts);
    block_exclusive_scan<long long>(nl, sh, tl);
    if (threadIdx.x == 0) {
        a.blk_sites[blockIdx.x] = ts;
        a.blk_links[blockIdx.x] = tl;
    }
}

// single block: exclusive scan of the per-tile counts
__global__ void __launch_bounds__(CT) site_scan_kernel(SiteArgs a, int nblk) {
    __shared__ long long sh[CT / 32];
    __shared__ long long carry_s, carry_l;
    if (threadIdx.x == 0) carry_s = carry_l = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblk; b0 += CT) {
        const int b = b0 + threadIdx.x;
        const long long vs = b < nblk ? a.blk_sites[b] : 0, vl = b < nblk ? a.blk_links[b] : 0;
        long long ts, tl;
        const long long es = block_exclusive_scan<long long>(vs, sh, ts);
        const long long el = block_exclusive_scan<long long>(vl, sh, tl);
        if (b < nblk) {
            a.blk_sites[b] = carry_s + es;
            a.blk_links[b] = carry_l + el;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_s += ts;
            carry_l += tl;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.counts[0] = carry_s;
        a.counts[1] = carry_l;
        if (carry_s > a.max_sites || carry_l > a.max_links) atomicOr(a.status, 2u);
    }
}

__device__ void link_geometry(const SiteArgs &a, int x, int y, int z, int l, double &q, int &pid, int &scheme) {
    const int xb = gwrap(x + cx(l), a.nx), yb = gwrap(y + cy(l), a.ny), zb = gwrap(z + cz(l), a.nz);
    const long long cb = (long long)xb + (long long)a.nx * (yb + (long long)a.ny * zb);
    const int own = a.owner[cb];
    const double cl0 = (double)cx(l), cl1 = (double)cy(l), cl2 = (double)cz(l);
    const double aa = (double)(cx(l) * cx(l) + cy(l) * cy(l) + cz(l) * cz(l));
    double t;
    if (own != NO_OWNER) {
        pid = own;
        const double *Xp = a.X + 3 * own;
        const double Rp = a.R[own];
        const double dx = gmimg(__dsub_rn((double)x, Xp[0]), a.nx);
        const double dy = gmimg(__dsub_rn((double)y, Xp[1]), a.ny);
        const double dz = gmimg(__dsub_rn((double)z, Xp[2]), a.nz);
        const double b = __dadd_rn(__dadd_rn(__dmul_rn(cl0, dx), __dmul_rn(cl1, dy)), __dmul_rn(cl2, dz));
        const double c0 = __dsub_rn(dist2(dx, dy, dz), __dmul_rn(Rp, Rp));
        double disc = __dsub_rn(__dmul_rn(b, b), __dmul_rn(aa, c0));
        if (disc < 0.0) disc = 0.0;
        t = __ddiv_rn(__dsub_rn(-b, __dsqrt_rn(disc)), aa);
    } else {
        pid = -1;
        const double a2 = (double)(cx(l) * cx(l) + cy(l) * cy(l));
        const double dx = __dsub_rn((double)x, a.pcx), dy = __dsub_rn((double)y, a.pcy);
        const double b = __dadd_rn(__dmul_rn(cl0, dx), __dmul_rn(cl1, dy));
        const double c0 = __dsub_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(a.pR, a.pR));
        double disc = __dsub_rn(__dmul_rn(b, b), __dmul_rn(a2, c0));
        if (disc < 0.0) disc = 0.0;
        t = __ddiv_rn(__dadd_rn(-b, __dsqrt_rn(disc)), a2);
    }
    if (t > 1.0) t = 1.0;
    if (t < 0.0) t = 0.0;
    q = t;
    const int x1 = gwrap(x - cx(l), a.nx), y1 = gwrap(y - cy(l), a.ny), z1 = gwrap(z - cz(l), a.nz);
    const int x2 = gwrap(x - 2 * cx(l), a.nx), y2 = gwrap(y - 2 * cy(l), a.ny), z2 = gwrap(z - 2 * cz(l), a.nz);
    const bool f1 = !(a.flags[(long long)x1 + (long long)a.nx * (y1 + (long long)a.ny * z1)] & FL_SOLID);
    const bool f2 = !(a.flags[(long long)x2 + (long long)a.nx * (y2 + (long long)a.ny * z2)] & FL_SOLID);
    if (pid >= 0) {
        if (q < 0.5) scheme = (f1 && f2) ? 0 : (f1 ? 1 : 2);
        else scheme = f1 ? 0 : 1;
    } else {
        if (q < 0.5) scheme = f1 ? 1 : 2;
        else scheme = 1;
    }
}

__global__ void __launch_bounds__(CT) site_emit_kernel(SiteArgs a) {
    __shared__ long long sh[CT / 32];
    const long long base = (long long)blockIdx.x * TILE + (long long)threadIdx.x * CPT;
    bool site[CPT];
    unsigned mask[CPT];
    long long ns = 0, nl = 0;
    for (int k = 0; k < CPT; k++) {
        cell_info(a, base + k, site[k], mask[k]);
        ns += site[k];
        nl += __popc(mask[k]);
    }
    long long ts, tl;
    long long s0 = block_exclusive_scan<long long>(ns, sh, ts) + a.blk_sites[blockIdx.x];
    long long l0 = block_exclusive_scan<long long>(nl, sh, tl) + a.blk_links[blockIdx.x];
    for (int k = 0; k < CPT; k++) {
        const long long c = base + k;
        if (c >= a.N) break;
        const int nl_c = __popc(mask[k]);
        // a site is written only if it and all its links fit the capacity;
        // otherwise the status word reports the overflow and the cell keeps
        // no BND flag, so no kernel reads a slot or link that was not written
        const bool fits = site[k] && s0 < a.max_sites && l0 + nl_c <= a.max_links;
        if (a.mode == 1) {
            const uint8_t fl = a.flags[c];
            const uint8_t nf = fits ? (uint8_t)(fl | FL_BND) : (uint8_t)(fl & ~FL_BND);
            if (nf != fl) a.flags[c] = nf;
        }
        if (!site[k]) continue;
        if (fits) {
            a.site_cell[s0] = (int)c;
            a.site_first[s0] = (int)l0;
            a.site_mask[s0] = mask[k];
            a.aux[c] = (int)s0;
            if (a.mode == 1) {
                const int x = (int)(c % a.nx), y = (int)((c / a.nx) % a.ny), z = (int)(c / ((long long)a.nx * a.ny));
                long long lk = l0;
                for (int l = 1; l < 19; l++) {
                    if (!((mask[k] >> l) & 1u)) continue;
                    double q;
                    int pid, sch;
                    link_geometry(a, x, y, z, l, q, pid, sch);
                    a.link_cell[lk] = (int)c;
                    a.link_dir[lk] = (int8_t)l;
                    a.link_scheme[lk] = (int8_t)sch;
                    a.link_q[lk] = q;
                    a.link_pid[lk] = pid;
                    lk++;
                }
            }
        } else if (a.mode == 2) {
            a.aux[c] = -1;  // support cell without a slot: skipped by every reader
        }
        l0 += nl_c;
        s0++;
    }
}

// Build the compact site list. mode 1: IBB boundary cells and their links
// (BND flags refreshed); mode 2: IBM support cells (SUP flags set before).
cudaError_t build_sites(Ctx &c, int mode) {
    SiteArgs a;
    a.flags = c.flags;
    a.owner = c.owner;
    a.aux = c.aux;
    a.X = c.X;
    a.R = c.R;
    a.nx = c.nx;
    a.ny = c.ny;
    a.nz = c.nz;
    a.N = c.N;
    a.pcx = c.pipe_cx;
    a.pcy = c.pipe_cy;
    a.pR = c.pipe_R;
    a.mode = mode;
    a.blk_sites = c.blk_sites;
    a.blk_links = c.blk_links;
    a.counts = c.d_counts;
    a.site_cell = c.site_cell;
    a.site_first = c.site_first;
    a.site_mask = c.site_mask;
    a.link_cell = c.link_cell;
    a.link_pid = c.link_pid;
    a.link_dir = c.link_dir;
    a.link_scheme = c.link_scheme;
    a.link_q = c.link_q;
    a.max_sites = c.max_sites;
    a.max_links = c.max_links;
    a.status = c.d_status;
    const int nblk = (int)((c.N + TILE - 1) / TILE);
    count_launch(c, G_GEOM, 3);
    site_count_kernel<<<nblk, CT, 0, c.stream>>>(a);
    site_scan_kernel<<<1, CT, 0, c.stream>>>(a, nblk);
    site_emit_kernel<<<nblk, CT, 0, c.stream>>>(a);
    return cudaGetLastError();
}

}  // namespace lbmgb
