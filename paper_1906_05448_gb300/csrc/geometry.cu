// Geometry kernels: solid flags of the pipe and of the spheres, refill of
// uncovered nodes, and the ordered compaction that lists IBB boundary cells
// with their links, or IBM support cells.
//
// Solid test and link fraction q are computed in FP64 with explicitly
// rounded operations (no fused multiply-add), in a fixed order, so that a
// given set of particle positions yields bit-identical link lists on every
// run (Sec. 3.1: a sharp interface found by ray-sphere intersection).
#include "lbm_internal.cuh"

#include <algorithm>

#ifndef LBM_LOCAL_SITES
#define LBM_LOCAL_SITES 1  // 1: particle boundary cells marked per particle box (see bnd_mark_kernel)
#endif

namespace lbmgb {

__device__ __forceinline__ double gmimg(double d, int n) {
    if (d > 0.5 * n) d = __dsub_rn(d, (double)n);
    else if (d < -0.5 * n) d = __dadd_rn(d, (double)n);
    return d;
}
// wrap a coordinate in [-n, 2n) into [0, n)
__device__ __forceinline__ int gwrap(int a, int n) {
    a = a < 0 ? a + n : a;
    return a >= n ? a - n : a;
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
// The inside test is decided in FP32 away from the surface and by the exact
// FP64 test (same operations and order as everywhere else) within a band of
// 0.01 in d^2 around R^2, far wider than the FP32 error of d^2 here
// (|d| < 2R + 4, coordinates below 2^16).
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
    const float R2f = (float)R2, band = 0.01f;
    const float X0 = (float)Xp[0], X1 = (float)Xp[1], X2 = (float)Xp[2];
    const FastDiv fw((unsigned)w);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int ix, iy, iz;
        box_coords(t, fw, w, ix, iy, iz);
        const int x = gwrap(bx + ix, a.nx), y = gwrap(by + iy, a.ny), z = gwrap(bz + iz, a.nz);
        const long long c = (long long)x + (long long)a.nx * (y + (long long)a.ny * z);
        if (CLEAR) {
            if (a.owner[c] == p) {
                if (a.keep_owner) a.aux[c] = p;
                a.owner[c] = NO_OWNER;
                a.flags[c] = (uint8_t)((a.flags[c] & ~FL_SOLID) | FL_WAS_SOLID);
            }
        } else {
            float fx = (float)x - X0, fy = (float)y - X1, fz = (float)z - X2;
            fx = fx > 0.5f * a.nx ? fx - a.nx : (fx < -0.5f * a.nx ? fx + a.nx : fx);
            fy = fy > 0.5f * a.ny ? fy - a.ny : (fy < -0.5f * a.ny ? fy + a.ny : fy);
            fz = fz > 0.5f * a.nz ? fz - a.nz : (fz < -0.5f * a.nz ? fz + a.nz : fz);
            const float d2f = fx * fx + fy * fy + fz * fz;
            bool inside;
            if (d2f < R2f - band) {
                inside = true;
            } else if (d2f > R2f + band) {
                inside = false;
            } else {
                const double dx = gmimg(__dsub_rn((double)x, Xp[0]), a.nx);
                const double dy = gmimg(__dsub_rn((double)y, Xp[1]), a.ny);
                const double dz = gmimg(__dsub_rn((double)z, Xp[2]), a.nz);
                inside = dist2(dx, dy, dz) <= R2;
            }
            if (inside) {
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
// Caiazzo (2008) refill (Sec. 3.1) of a node that the particle p uncovered:
// rho = mean over fluid neighbours, u = rigid-body velocity, and the
// non-equilibrium part of the fluid neighbour best aligned with the outward
// normal (ties: lowest direction index).
// refill_collect_kernel lists the uncovered nodes (one block per particle);
// refill_apply_kernel handles one node per warp, lane i on direction i.
struct RefillArgs {
    void *B;
    const uint8_t *flags;
    const int *aux;
    const double *X, *U, *W, *R, *Xold;
    int nx, ny, nz;
    long long N;
    double F[3];
    long long *count;  // device counter of listed nodes
    int *list, *list_pid;
    long long cap;
};

__global__ void refill_collect_kernel(RefillArgs a) {
    const int p = blockIdx.x;
    // uncovered nodes were solid at the old position: the box the clear pass swept
    const double *Xp = a.Xold + 3 * p;
    const int r = (int)ceil(a.R[p]) + 1;
    const int bx = (int)floor(Xp[0]) - r, by = (int)floor(Xp[1]) - r, bz = (int)floor(Xp[2]) - r;
    const int w = 2 * r + 2;
    const FastDiv fw((unsigned)w);
    for (int t = threadIdx.x; t < w * w * w; t += blockDim.x) {
        int ix, iy, iz;
        box_coords(t, fw, w, ix, iy, iz);
        const int x = gwrap(bx + ix, a.nx), y = gwrap(by + iy, a.ny), z = gwrap(bz + iz, a.nz);
        const long long c = (long long)x + (long long)a.nx * (y + (long long)a.ny * z);
        const uint8_t fl = a.flags[c];
        if (!(fl & FL_WAS_SOLID) || (fl & FL_SOLID) || a.aux[c] != p) continue;
        const long long k = atomicAdd((unsigned long long *)a.count, 1ULL);
        if (k < a.cap) {
            a.list[k] = (int)c;
            a.list_pid[k] = p;
        }
    }
}

template <int S>
__device__ __forceinline__ void refill_one(const RefillArgs &a, long long k) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R Rt;
    const int lane = threadIdx.x & 31;
    const size_t N = (size_t)a.N;
    T *B = (T *)a.B;
    const int c = a.list[k], p = a.list_pid[k];
    const int x = c % a.nx, y = (c / a.nx) % a.ny, z = c / (a.nx * a.ny);
    const double rv0 = gmimg((double)x - a.X[3 * p], a.nx), rv1 = gmimg((double)y - a.X[3 * p + 1], a.ny),
                 rv2 = gmimg((double)z - a.X[3 * p + 2], a.nz);
    const double *Up = a.U + 3 * p, *Wp = a.W + 3 * p;
    const Rt uw0 = Rt(Up[0] + (Wp[1] * rv2 - Wp[2] * rv1)), uw1 = Rt(Up[1] + (Wp[2] * rv0 - Wp[0] * rv2)),
             uw2 = Rt(Up[2] + (Wp[0] * rv1 - Wp[1] * rv0));
    const double l = sqrt(rv0 * rv0 + rv1 * rv1 + rv2 * rv2);
    const Rt n0 = l > 0 ? Rt(rv0 / l) : Rt(0), n1 = l > 0 ? Rt(rv1 / l) : Rt(0), n2 = l > 0 ? Rt(rv2 / l) : Rt(0);
    // lane i (1..18): neighbour x + c_i
    Rt rho_i = 0, j0 = 0, j1 = 0, j2 = 0, al = Rt(-1e30);
    int valid = 0;
    long long nb = -1;
    if (lane >= 1 && lane < 19) {
        const int i = lane;
        const int cxi = (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
                      : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
        const int cyi = (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
                      : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
        const int czi = (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
                      : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
        nb = (long long)gwrap(x + cxi, a.nx) + (long long)a.nx * (gwrap(y + cyi, a.ny) + (long long)a.ny * gwrap(z + czi, a.nz));
        if (!(a.flags[nb] & (FL_WAS_SOLID | FL_SOLID))) {
            valid = 1;
            Rt r = 0;
#pragma unroll
            for (int q = 0; q < 19; q++) {
                const Rt g = Store<S>::ld(B + q * N + nb);
                r += g;
                j0 += g * Rt(cx(q));
                j1 += g * Rt(cy(q));
                j2 += g * Rt(cz(q));
            }
            rho_i = Rt(1) + r;
            const Rt cl = sqrt(Rt(cxi * cxi + cyi * cyi + czi * czi));
            al = (n0 * Rt(cxi) + n1 * Rt(cyi) + n2 * Rt(czi)) / cl;
        }
    }
    // mean density of the fluid neighbours, and the best-aligned one
    Rt rsum = valid ? rho_i : Rt(0);
    int cnt = valid;
    Rt best = al;
    int bl = valid ? lane : 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        const Rt ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
        if (ob > best || (ob == best && ol < bl)) {
            best = ob;
            bl = ol;
        }
    }
    const Rt rho = cnt ? rsum / Rt(cnt) : Rt(1);
    const bool have = bl < 32;
    const int src = have ? bl : 0;
    const Rt rn = __shfl_sync(0xffffffffu, rho_i, src), k0 = __shfl_sync(0xffffffffu, j0, src),
             k1 = __shfl_sync(0xffffffffu, j1, src), k2 = __shfl_sync(0xffffffffu, j2, src);
    const long long nbb = __shfl_sync(0xffffffffu, nb, src);
    if (lane >= 19) return;
    const int q = lane;
    const Rt uu = uw0 * uw0 + uw1 * uw1 + uw2 * uw2;
    const Rt cuw = Rt(cx(q)) * uw0 + Rt(cy(q)) * uw1 + Rt(cz(q)) * uw2;
    Rt f = Rt(wgt(q)) * rho * (Rt(1) + Rt(3) * cuw + Rt(4.5) * cuw * cuw - Rt(1.5) * uu);
    if (have) {
        const Rt un0 = (k0 - Rt(0.5) * Rt(a.F[0])) / rn, un1 = (k1 - Rt(0.5) * Rt(a.F[1])) / rn,
                 un2 = (k2 - Rt(0.5) * Rt(a.F[2])) / rn;
        const Rt un = un0 * un0 + un1 * un1 + un2 * un2;
        const Rt cun = Rt(cx(q)) * un0 + Rt(cy(q)) * un1 + Rt(cz(q)) * un2;
        const Rt feq_nb = Rt(wgt(q)) * rn * (Rt(1) + Rt(3) * cun + Rt(4.5) * cun * cun - Rt(1.5) * un);
        const Rt fnb = Store<S>::ld(B + q * N + nbb) + Rt(wgt(q));
        f += fnb - feq_nb;
    }
    Store<S>::st(B + q * N + c, f - Rt(wgt(q)));
}

template <int S>
__global__ void __launch_bounds__(256) refill_apply_kernel(RefillArgs a) {
    const long long n = *a.count < a.cap ? *a.count : a.cap;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < n; k += warps)
        refill_one<S>(a, k);
}


cudaError_t launch_refill(Ctx &c) {
    if (c.np == 0) return cudaSuccess;
    count_launch(c, G_GEOM, 3);
    RefillArgs a{c.fB, c.flags, c.aux, c.X, c.U, c.W, c.R, c.Xold, c.nx, c.ny, c.nz, c.N, {c.F[0], c.F[1], c.F[2]},
                 c.d_counts + 2, c.refill_list, c.refill_pid, c.max_refill};
    cudaError_t e = cudaMemsetAsync(c.d_counts + 2, 0, sizeof(long long), c.stream);
    if (e != cudaSuccess) return e;
    refill_collect_kernel<<<c.np, 256, 0, c.stream>>>(a);
    // warp per node over the listed nodes (the count is on the device): a grid of a few blocks per SM
    const unsigned nb = (unsigned)std::min<long long>((c.max_refill * 32 + 255) / 256, 152LL * 8);
    switch (c.storage) {
    case LBM_F64: refill_apply_kernel<LBM_F64><<<nb, 256, 0, c.stream>>>(a); break;
    case LBM_F32: refill_apply_kernel<LBM_F32><<<nb, 256, 0, c.stream>>>(a); break;
    case LBM_F16S: refill_apply_kernel<LBM_F16S><<<nb, 256, 0, c.stream>>>(a); break;
    default: refill_apply_kernel<LBM_BF16S><<<nb, 256, 0, c.stream>>>(a); break;
    }
    return cudaGetLastError();
}

// clear WAS_SOLID after the refill: it was set in the box of the old position
__global__ void finish_kernel(uint8_t *flags, const double *X, const double *R, int nx, int ny, int nz) {
    const int p = blockIdx.x;
    const int r = (int)ceil(R[p]) + 1;
    const int bx = (int)floor(X[3 * p]) - r, by = (int)floor(X[3 * p + 1]) - r, bz = (int)floor(X[3 * p + 2]) - r;
    const int w = 2 * r + 2;
    const FastDiv fw((unsigned)w);
    for (int t = threadIdx.x; t < w * w * w; t += blockDim.x) {
        int ix, iy, iz;
        box_coords(t, fw, w, ix, iy, iz);
        const int x = gwrap(bx + ix, nx), y = gwrap(by + iy, ny), z = gwrap(bz + iz, nz);
        const long long c = (long long)x + (long long)nx * (y + (long long)ny * z);
        if (flags[c] & FL_WAS_SOLID) atomic_and_flag(flags, c, (uint8_t)~FL_WAS_SOLID);
    }
}

cudaError_t launch_finish_geometry(Ctx &c) {
    if (c.np == 0) return cudaSuccess;
    count_launch(c, G_GEOM);
    finish_kernel<<<c.np, 256, 0, c.stream>>>(c.flags, c.Xold, c.R, c.nx, c.ny, c.nz);
    return cudaGetLastError();
}

// ------------------------------------------------ site compaction --------
// Cells are processed in tiles of TILE consecutive indices; each tile's
// counts are scanned, so sites and links come out ordered by cell index and
// links of a cell by direction, independent of the launch configuration.
constexpr int CT = 256;        // threads per tile block
constexpr int CPT = 4;         // cells per thread
constexpr int TILE = CT * CPT;

struct __align__(32) SiteGeo {
    double dx, dy, dz, c0;
};

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
    FastDiv dx, dxy;  // division by nx and nx * ny
    double dn[3], hn[3];  // nx, ny, nz and their halves as doubles
    int *sn_list;         // links of the single-node scheme (appended, counts[4])
    // 32/16-bit storage with particles: per site, the offset d = x - X_p to
    // its first solid neighbour's particle and c0 = |d|^2 - R_p^2 (FP64),
    // and that particle; null otherwise (every link forms them itself)
    SiteGeo *site_geo;
    int *site_own;
};

// minimum image with the box size and its half given as doubles (no
// int-to-double conversion per call; the same values as gmimg)
__device__ __forceinline__ double gmimg_d(double d, double n, double h) {
    if (d > h) d = __dsub_rn(d, n);
    else if (d < -h) d = __dadd_rn(d, n);
    return d;
}

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
        const unsigned zq = a.dxy.div((unsigned)c), rem = (unsigned)c - zq * (unsigned)(a.nx * a.ny);
        const unsigned yq = a.dx.div(rem);
        mask = solid_mask(a, (int)(rem - yq * (unsigned)a.nx), (int)yq, (int)zq);
        site = mask != 0;
    } else {
        site = (fl & FL_SUP) != 0;
    }
}

// The CPT = 4 consecutive cells of a thread at once (mode 1, nx a multiple
// of 4, so that the group starts a 4-byte word and stays in one row): the
// solid bits of x0-1 .. x0+4 in each of the 9 rows y+dy, z+dz are read as
// one word and two bytes, and the 18-neighbour masks are cut from them.
__device__ __forceinline__ unsigned solid_bits6(const SiteArgs &a, long long rowbase, int x0) {
    const unsigned mid = __ldg((const unsigned *)(a.flags + rowbase + x0));
    const unsigned left = a.flags[rowbase + (x0 > 0 ? x0 - 1 : a.nx - 1)];
    const unsigned right = a.flags[rowbase + (x0 + 4 < a.nx ? x0 + 4 : 0)];
    const unsigned m = mid & 0x01010101u * FL_SOLID;
    const unsigned four = ((m >> 0) & 1u) | ((m >> 7) & 2u) | ((m >> 14) & 4u) | ((m >> 21) & 8u);
    return ((left & FL_SOLID) ? 1u : 0u) | (four << 1) | ((right & FL_SOLID) ? 32u : 0u);
}

// Solid bits around the 4 cells c0 .. c0+3 of one x-row word: rows[dz+1][dy+1]
// holds the cells x0-1 .. x0+4 of the row (y+dy, z+dz) in bits 0 .. 5.
__device__ __forceinline__ void solid_rows4(const SiteArgs &a, long long c0, unsigned rows[3][3]) {
    const unsigned zq = a.dxy.div((unsigned)c0), rem = (unsigned)c0 - zq * (unsigned)(a.nx * a.ny);
    const unsigned yq = a.dx.div(rem);
    const int x0 = (int)(rem - yq * (unsigned)a.nx), y = (int)yq, z = (int)zq;
#pragma unroll
    for (int dz = -1; dz <= 1; dz++)
#pragma unroll
        for (int dy = -1; dy <= 1; dy++) {
            if (dy != 0 && dz != 0) {
                rows[dz + 1][dy + 1] = 0;  // no D3Q19 velocity has both
                continue;
            }
            const int yy = gwrap(y + dy, a.ny), zz = gwrap(z + dz, a.nz);
            rows[dz + 1][dy + 1] = solid_bits6(a, ((long long)zz * a.ny + yy) * a.nx, x0);
        }
    // the edge rows of D3Q19 (dy, dz both nonzero) take only the centre cell
#pragma unroll
    for (int dz = -1; dz <= 1; dz += 2)
#pragma unroll
        for (int dy = -1; dy <= 1; dy += 2) {
            const int yy = gwrap(y + dy, a.ny), zz = gwrap(z + dz, a.nz);
            const unsigned w = __ldg((const unsigned *)(a.flags + ((long long)zz * a.ny + yy) * a.nx + x0));
            const unsigned m = w & 0x01010101u * FL_SOLID;
            rows[dz + 1][dy + 1] = (((m >> 0) & 1u) | ((m >> 7) & 2u) | ((m >> 14) & 4u) | ((m >> 21) & 8u)) << 1;
        }
}

// Direction-major neighbour bits of the 4 cells: bit k of v[l] is set when
// cell c0 + k is a fluid cell of the grid and its neighbour x + c_l is solid.
// Counting needs only popcounts of these 18 words; the per-cell masks are
// formed for the few cells that have a link.
__device__ __forceinline__ void link_bits4(const SiteArgs &a, long long c0, unsigned v[19]) {
    unsigned rows[3][3];
    solid_rows4(a, c0, rows);
    const long long left = a.N - c0;
    const unsigned valid = left >= CPT ? (1u << CPT) - 1u : (left > 0 ? (1u << left) - 1u : 0u);
    const unsigned fluid = ~(rows[1][1] >> 1) & valid;
    v[0] = 0;
#pragma unroll
    for (int l = 1; l < 19; l++) v[l] = (rows[cz(l) + 1][cy(l) + 1] >> (1 + cx(l))) & fluid;
}

__device__ __forceinline__ void cell_info4(const SiteArgs &a, long long c0, bool site[CPT], unsigned mask[CPT]) {
    unsigned v[19];
    link_bits4(a, c0, v);
    unsigned any = 0;
#pragma unroll
    for (int l = 1; l < 19; l++) any |= v[l];
#pragma unroll
    for (int k = 0; k < CPT; k++) {
        site[k] = (any >> k) & 1u;
        unsigned m = 0;
        if (site[k]) {
#pragma unroll
            for (int l = 1; l < 19; l++) m |= ((v[l] >> k) & 1u) << l;
        }
        mask[k] = m;
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
    if (a.mode == 1 && a.nx % 4 == 0 && base < a.N) {
        unsigned v[19], any = 0;
        link_bits4(a, base, v);
#pragma unroll
        for (int l = 1; l < 19; l++) {
            any |= v[l];
            nl += __popc(v[l]);
        }
        ns = __popc(any);
    } else {
        for (int k = 0; k < CPT; k++) {
            bool site;
            unsigned mask;
            cell_info(a, base + k, site, mask);
            ns += site;
            nl += __popc(mask);
        }
    }
    long long ts, tl;
    block_exclusive_scan<long long>(ns, sh, ts);
    block_exclusive_scan<long long>(nl, sh, tl);
    if (threadIdx.x == 0) {
        a.blk_sites[blockIdx.x] = ts;
        a.blk_links[blockIdx.x] = tl;
    }
}

// single block of ST threads: exclusive scan of the per-tile counts. Each
// thread sums a run of consecutive tiles, the thread sums are scanned in the
// block, and each run is written back from its thread's offset.
constexpr int ST = 1024;
__global__ void __launch_bounds__(ST) site_scan_kernel(SiteArgs a, int nblk) {
    __shared__ long long ws[ST / 32], wl[ST / 32];
    const int per = (nblk + ST - 1) / ST;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, nblk);
    long long ss = 0, sl = 0;
    for (int b = b0; b < b1; b++) {
        ss += a.blk_sites[b];
        sl += a.blk_links[b];
    }
    // block exclusive scan of (ss, sl)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long is = ss, il = sl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long ts = __shfl_up_sync(0xffffffffu, is, o), tl = __shfl_up_sync(0xffffffffu, il, o);
        if (lane >= o) {
            is += ts;
            il += tl;
        }
    }
    if (lane == 31) {
        ws[wid] = is;
        wl[wid] = il;
    }
    __syncthreads();
    if (wid == 0) {
        long long vs = ws[lane], vl = wl[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long ts = __shfl_up_sync(0xffffffffu, vs, o), tl = __shfl_up_sync(0xffffffffu, vl, o);
            if (lane >= o) {
                vs += ts;
                vl += tl;
            }
        }
        ws[lane] = vs;
        wl[lane] = vl;
    }
    __syncthreads();
    long long es = (wid > 0 ? ws[wid - 1] : 0) + is - ss, el = (wid > 0 ? wl[wid - 1] : 0) + il - sl;
    for (int b = b0; b < b1; b++) {
        const long long vs = a.blk_sites[b], vl = a.blk_links[b];
        a.blk_sites[b] = es;
        a.blk_links[b] = el;
        es += vs;
        el += vl;
    }
    if (threadIdx.x == ST - 1) {
        a.counts[0] = es;
        a.counts[1] = el;
        if (es > a.max_sites || el > a.max_links) atomicOr(a.status, 2u);
    }
}

// v / c2 for c2 = |c|^2 or its xy part: division by 1 or 2 is exact, so the
// scaling returns the correctly rounded quotient; 0 gives the IEEE result
__device__ __forceinline__ double exact_div_c2(double v, double c2) {
    return c2 == 1.0 ? v : (c2 == 2.0 ? v * 0.5 : __ddiv_rn(v, c2));
}

// q to FP32 accuracy (32/16-bit storage). The smaller root of
// a t^2 + 2 b t + c0 = 0 is (-b - s)/a = c0/(s - b), s = sqrt(b^2 - a c0);
// for a link into the sphere c0 > 0 and b < 0 (the quadratic falls from
// c0 at t = 0 to <= 0 at t = 1), so s - b adds two positive numbers and
// the quotient keeps FP32's relative accuracy: with the discriminant in
// FP64 as in the exact form, the error is below 3e-7. Within 1e-5 of 1/2,
// where q picks the scheme, the exact FP64 form decides, so the link lists
// are those of the exact q.
__device__ __forceinline__ double fast_root(double b, double disc, double c0, bool diag) {
    const float qf = (float)c0 / (sqrtf((float)disc) - (float)b);
    if (fabsf(qf - 0.5f) >= 1e-5f) return (double)qf;
    const double num = __dsub_rn(-b, __dsqrt_rn(disc));
    return diag ? num * 0.5 : num;
}

// per site: d and c0 of the particle that owns the site's first solid neighbour
__global__ void __launch_bounds__(256) site_geo_kernel(SiteArgs a) {
    const long long ns = a.counts[0] < a.max_sites ? a.counts[0] : a.max_sites;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < ns;
         s += (long long)gridDim.x * blockDim.x) {
        const unsigned c = (unsigned)a.site_cell[s];
        const unsigned m = a.site_mask[s];
        const unsigned zq = a.dxy.div(c), rem = c - zq * (unsigned)(a.nx * a.ny);
        const unsigned yq = a.dx.div(rem);
        const int x = (int)(rem - yq * (unsigned)a.nx), y = (int)yq, z = (int)zq;
        const int l = m ? __ffs(m) - 1 : 1;
        const int xb = gwrap(x + cx(l), a.nx), yb = gwrap(y + cy(l), a.ny), zb = gwrap(z + cz(l), a.nz);
        const int own = a.owner[(long long)xb + (long long)a.nx * (yb + (long long)a.ny * zb)];
        a.site_own[s] = own;
        if (own == NO_OWNER) continue;
        const double *Xp = a.X + 3 * own;
        const double Rp = a.R[own];
        const double dx = gmimg_d(__dsub_rn((double)x, Xp[0]), a.dn[0], a.hn[0]);
        const double dy = gmimg_d(__dsub_rn((double)y, Xp[1]), a.dn[1], a.hn[1]);
        const double dz = gmimg_d(__dsub_rn((double)z, Xp[2]), a.dn[2], a.hn[2]);
        a.site_geo[s] = SiteGeo{dx, dy, dz, __dsub_rn(dist2(dx, dy, dz), __dmul_rn(Rp, Rp))};
    }
}

__device__ void link_geometry(const SiteArgs &a, int x, int y, int z, int l, double &q, int &pid, int &scheme,
                              long long site = -1) {
    const int xb = gwrap(x + cx(l), a.nx), yb = gwrap(y + cy(l), a.ny), zb = gwrap(z + cz(l), a.nz);
    const long long cb = (long long)xb + (long long)a.nx * (yb + (long long)a.ny * zb);
    const int own = a.owner[cb];
    // FP64 issue is what this kernel costs on GB300, so c_l and |c_l|^2 come
    // from selects on constants rather than int-to-double conversions (the
    // values are the same)
    const int i0 = cx(l), i1 = cy(l), i2 = cz(l);
    const double cl0 = i0 > 0 ? 1.0 : (i0 < 0 ? -1.0 : 0.0);
    const double cl1 = i1 > 0 ? 1.0 : (i1 < 0 ? -1.0 : 0.0);
    const double cl2 = i2 > 0 ? 1.0 : (i2 < 0 ? -1.0 : 0.0);
    const bool diag = (i0 != 0) + (i1 != 0) + (i2 != 0) == 2;  // |c_l|^2 = 2
    const double aa = diag ? 2.0 : 1.0;
    double t;
    if (own != NO_OWNER) {
        pid = own;
        double dx, dy, dz, c0;
        if (site >= 0 && a.site_own[site] == own) {
            const SiteGeo g = a.site_geo[site];
            dx = g.dx;
            dy = g.dy;
            dz = g.dz;
            c0 = g.c0;
        } else {
            const double *Xp = a.X + 3 * own;
            const double Rp = a.R[own];
            dx = gmimg_d(__dsub_rn((double)x, Xp[0]), a.dn[0], a.hn[0]);
            dy = gmimg_d(__dsub_rn((double)y, Xp[1]), a.dn[1], a.hn[1]);
            dz = gmimg_d(__dsub_rn((double)z, Xp[2]), a.dn[2], a.hn[2]);
            c0 = __dsub_rn(dist2(dx, dy, dz), __dmul_rn(Rp, Rp));
        }
        // b = c_l . d as ((c0 dx + c1 dy) + c2 dz): with components in
        // {-1, 0, 1} this is the sum of the one or two nonzero terms, which
        // gives the same bits whenever that sum is not zero; a zero sum takes
        // the full form for the sign of zero
        const double u = i0 ? (i0 > 0 ? dx : -dx) : (i1 ? (i1 > 0 ? dy : -dy) : (i2 > 0 ? dz : -dz));
        const double v = !diag ? 0.0 : (i2 ? (i2 > 0 ? dz : -dz) : (i1 > 0 ? dy : -dy));
        double b = __dadd_rn(u, v);
        if (b == 0.0) b = __dadd_rn(__dadd_rn(__dmul_rn(cl0, dx), __dmul_rn(cl1, dy)), __dmul_rn(cl2, dz));
        double disc = __dsub_rn(__dmul_rn(b, b), __dmul_rn(aa, c0));
        if (disc < 0.0) disc = 0.0;
        if (site >= 0) {
            t = fast_root(b, disc, c0, diag);
        } else {
            const double num = __dsub_rn(-b, __dsqrt_rn(disc));
            t = diag ? num * 0.5 : num;  // division by |c_l|^2 = 1 or 2, exact
        }
    } else {
        pid = -1;
        const double a2 = (double)(cx(l) * cx(l) + cy(l) * cy(l));
        const double dx = __dsub_rn((double)x, a.pcx), dy = __dsub_rn((double)y, a.pcy);
        const double b = __dadd_rn(__dmul_rn(cl0, dx), __dmul_rn(cl1, dy));
        const double c0 = __dsub_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(a.pR, a.pR));
        double disc = __dsub_rn(__dmul_rn(b, b), __dmul_rn(a2, c0));
        if (disc < 0.0) disc = 0.0;
        t = exact_div_c2(__dadd_rn(-b, __dsqrt_rn(disc)), a2);
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
    if (a.mode == 1 && a.nx % 4 == 0 && base < a.N) {
        cell_info4(a, base, site, mask);
    } else {
        for (int k = 0; k < CPT; k++) cell_info(a, base + k, site[k], mask[k]);
    }
    for (int k = 0; k < CPT; k++) {
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
                // cell and direction only; link_geom_kernel fills in q, owner and scheme
                long long lk = l0;
                for (unsigned mm = mask[k] & ~1u; mm; mm &= mm - 1u, lk++) {  // set bits, ascending
                    a.link_cell[lk] = (int)c;
                    a.link_dir[lk] = (int8_t)(__ffs(mm) - 1);
                }
            }
        } else if (a.mode == 2) {
            a.aux[c] = -1;  // support cell without a slot: skipped by every reader
        }
        l0 += nl_c;
        s0++;
    }
}

// one thread per link: wall fraction q, owner and interpolation scheme
__global__ void __launch_bounds__(256) link_geom_kernel(SiteArgs a) {
    const long long nl = a.counts[1] < a.max_links ? a.counts[1] : a.max_links;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nl;
         k += (long long)gridDim.x * blockDim.x) {
        const unsigned c = (unsigned)a.link_cell[k];
        const int l = a.link_dir[k];
        const unsigned zq = a.dxy.div(c), rem = c - zq * (unsigned)(a.nx * a.ny);
        const unsigned yq = a.dx.div(rem);
        const int x = (int)(rem - yq * (unsigned)a.nx), y = (int)yq, z = (int)zq;
        double q;
        int pid, sch;
        link_geometry(a, x, y, z, l, q, pid, sch, a.site_geo ? (long long)a.aux[c] : -1LL);
        if (sch == 2) {  // listed for the single-node pass of the step
            const long long j = (long long)atomicAdd((unsigned long long *)(a.counts + 4), 1ULL);
            if (j < a.max_links) a.sn_list[j] = (int)k;
        }
        a.link_scheme[k] = (int8_t)sch;
        a.link_q[k] = q;
        a.link_pid[k] = pid;
    }
}

// ------------------------------------- particle boundary cells, locally --
// With particles, every boundary cell lies within one link of a particle
// (|x - X_p| <= R_p + sqrt 2), so the cells of the last list lose their BND
// flag, each particle's box marks its boundary cells again (BND flag, and
// the neighbour mask in aux), and the ordered compaction then reads only the
// grid's flag bytes, 16 per thread, instead of forming every cell's
// neighbour mask. Order and contents of the lists are those of the
// full-grid compaction.
constexpr int VT = 16;          // cells per thread (one 16-byte flag load)
constexpr int VTILE = CT * VT;  // cells per tile

__global__ void bnd_clear_kernel(uint8_t *flags, const int *site_cell, const long long *counts, long long max_sites) {
    const long long n = counts[0] < max_sites ? counts[0] : max_sites;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x)
        atomic_and_flag(flags, site_cell[s], (uint8_t)~FL_BND);
}

__global__ void __launch_bounds__(256) bnd_mark_kernel(SiteArgs a) {
    const int p = blockIdx.x;
    const int r = (int)ceil(a.R[p]) + 2;
    const int bx = (int)floor(a.X[3 * p]) - r, by = (int)floor(a.X[3 * p + 1]) - r, bz = (int)floor(a.X[3 * p + 2]) - r;
    const int w = 2 * r + 2;
    const FastDiv fw((unsigned)w);
    // a boundary cell of p lies in the shell R_p - 1 < |x - X_p| <= R_p + sqrt 2
    // (FP32 with margins: cells deeper inside are solid, farther out have no solid neighbour of p)
    const float Ro = (float)a.R[p] + 1.5f, Ri = fmaxf((float)a.R[p] - 1.5f, 0.f), ro2 = Ro * Ro, ri2 = Ri * Ri;
    const float fX0 = (float)a.X[3 * p] - bx, fX1 = (float)a.X[3 * p + 1] - by, fX2 = (float)a.X[3 * p + 2] - bz;
    for (int t = threadIdx.x; t < w * w * w; t += blockDim.x) {
        int ix, iy, iz;
        box_coords(t, fw, w, ix, iy, iz);
        const float ex = ix - fX0, ey = iy - fX1, ez = iz - fX2, e2 = ex * ex + ey * ey + ez * ez;
        if (e2 > ro2 || e2 < ri2) continue;
        const int x = gwrap(bx + ix, a.nx), y = gwrap(by + iy, a.ny), z = gwrap(bz + iz, a.nz);
        const long long c = (long long)x + (long long)a.nx * (y + (long long)a.ny * z);
        if (a.flags[c] & FL_SOLID) continue;
        const unsigned m = solid_mask(a, x, y, z);
        if (m == 0u) continue;
        a.aux[c] = (int)m;  // the same value from every box that holds the cell
        atomic_or_flag(a.flags, c, FL_BND);
    }
}

// bnd_mark_kernel with the solid bits of the particle's box and its one-cell
// rim staged in shared memory (a tile of side T, the same for every
// particle, T >= 2 (ceil R_p + 2) + 4): the 18 neighbour tests of a shell
// cell become loads at fixed offsets. The kernel changes only BND bits, so
// the staged solid bits stay those of the grid.
__global__ void __launch_bounds__(256) bnd_mark_tile_kernel(SiteArgs a, int T) {
    extern __shared__ uint8_t sol[];
    const int p = blockIdx.x;
    const int r = (int)ceil(a.R[p]) + 2;
    const int bx = (int)floor(a.X[3 * p]) - r, by = (int)floor(a.X[3 * p + 1]) - r, bz = (int)floor(a.X[3 * p + 2]) - r;
    const int w = 2 * r + 2;
    const FastDiv fT((unsigned)T), fw((unsigned)w);
    for (int t = threadIdx.x; t < T * T * T; t += blockDim.x) {
        int ix, iy, iz;
        box_coords(t, fT, T, ix, iy, iz);
        const int x = gwrap(bx - 1 + ix, a.nx), y = gwrap(by - 1 + iy, a.ny), z = gwrap(bz - 1 + iz, a.nz);
        sol[t] = a.flags[(long long)x + (long long)a.nx * (y + (long long)a.ny * z)] & FL_SOLID;
    }
    __syncthreads();
    const float Ro = (float)a.R[p] + 1.5f, Ri = fmaxf((float)a.R[p] - 1.5f, 0.f), ro2 = Ro * Ro, ri2 = Ri * Ri;
    const float fX0 = (float)a.X[3 * p] - bx, fX1 = (float)a.X[3 * p + 1] - by, fX2 = (float)a.X[3 * p + 2] - bz;
    for (int t = threadIdx.x; t < w * w * w; t += blockDim.x) {
        int ix, iy, iz;
        box_coords(t, fw, w, ix, iy, iz);
        const float ex = ix - fX0, ey = iy - fX1, ez = iz - fX2, e2 = ex * ex + ey * ey + ez * ez;
        if (e2 > ro2 || e2 < ri2) continue;
        const uint8_t *s = sol + (ix + 1) + T * ((iy + 1) + T * (iz + 1));
        if (*s) continue;
        unsigned m = 0;
#pragma unroll
        for (int l = 1; l < 19; l++)
            if (s[cx(l) + T * (cy(l) + T * cz(l))]) m |= 1u << l;
        if (m == 0u) continue;
        const int x = gwrap(bx + ix, a.nx), y = gwrap(by + iy, a.ny), z = gwrap(bz + iz, a.nz);
        const long long c = (long long)x + (long long)a.nx * (y + (long long)a.ny * z);
        a.aux[c] = (int)m;  // the same value from every box that holds the cell
        atomic_or_flag(a.flags, c, FL_BND);
    }
}

// the VT flag bytes of a thread's cells (zero past the grid's end)
__device__ __forceinline__ void load_flags16(const SiteArgs &a, long long base, uint8_t f[VT]) {
    if (base + VT <= a.N) {
        const uint4 v = __ldg((const uint4 *)(a.flags + base));
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < VT; k++) f[k] = (uint8_t)(w[k >> 2] >> (8 * (k & 3)));
    } else {
#pragma unroll
        for (int k = 0; k < VT; k++) f[k] = base + k < a.N ? a.flags[base + k] : (uint8_t)0;
    }
}

__global__ void __launch_bounds__(CT) bnd_count_kernel(SiteArgs a) {
    __shared__ long long sh[CT / 32];
    const long long base = (long long)blockIdx.x * VTILE + (long long)threadIdx.x * VT;
    long long ns = 0, nl = 0;
    if (base < a.N) {
        uint8_t f[VT];
        load_flags16(a, base, f);
#pragma unroll
        for (int k = 0; k < VT; k++)
            if (f[k] & FL_BND) {
                ns++;
                nl += __popc((unsigned)a.aux[base + k]);
            }
    }
    long long ts, tl;
    block_exclusive_scan<long long>(ns, sh, ts);
    block_exclusive_scan<long long>(nl, sh, tl);
    if (threadIdx.x == 0) {
        a.blk_sites[blockIdx.x] = ts;
        a.blk_links[blockIdx.x] = tl;
    }
}

__global__ void __launch_bounds__(CT) bnd_emit_kernel(SiteArgs a) {
    __shared__ long long sh[CT / 32];
    const long long base = (long long)blockIdx.x * VTILE + (long long)threadIdx.x * VT;
    uint8_t f[VT];
    long long ns = 0, nl = 0;
    unsigned bnd = 0;
    if (base < a.N) {
        load_flags16(a, base, f);
#pragma unroll
        for (int k = 0; k < VT; k++)
            if (f[k] & FL_BND) {
                bnd |= 1u << k;
                ns++;
                nl += __popc((unsigned)a.aux[base + k]);
            }
    }
    long long ts, tl;
    long long s0 = block_exclusive_scan<long long>(ns, sh, ts) + a.blk_sites[blockIdx.x];
    long long l0 = block_exclusive_scan<long long>(nl, sh, tl) + a.blk_links[blockIdx.x];
    while (bnd) {
        const int k = __ffs(bnd) - 1;
        bnd &= bnd - 1;
        const long long c = base + k;
        const unsigned m = (unsigned)a.aux[c];
        const int nl_c = __popc(m);
        // a site and its links are written only if they fit; otherwise the
        // status word reports the overflow and the cell loses its BND flag
        // (this thread owns these flag bytes here)
        if (s0 < a.max_sites && l0 + nl_c <= a.max_links) {
            a.site_cell[s0] = (int)c;
            a.site_first[s0] = (int)l0;
            a.site_mask[s0] = m;
            a.aux[c] = (int)s0;
            long long lk = l0;
            for (unsigned mm = m & ~1u; mm; mm &= mm - 1u, lk++) {  // set bits, ascending
                a.link_cell[lk] = (int)c;
                a.link_dir[lk] = (int8_t)(__ffs(mm) - 1);
            }
        } else {
            a.flags[c] = (uint8_t)(a.flags[c] & ~FL_BND);
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
    a.dx = FastDiv((unsigned)c.nx);
    a.dxy = FastDiv((unsigned)(c.nx * c.ny));
    a.sn_list = c.sn_list;
    // per-site geometry for 32/16-bit storage with particles, kept in the
    // IBM per-site arrays (unused by IBB)
    const bool fast_q = mode == 1 && c.np > 0 && c.storage != LBM_F64;
    a.site_geo = fast_q ? (SiteGeo *)c.sup_ru : nullptr;
    a.site_own = fast_q ? (int *)c.sup_F : nullptr;
    const int nd[3] = {c.nx, c.ny, c.nz};
    for (int d = 0; d < 3; d++) {
        a.dn[d] = (double)nd[d];
        a.hn[d] = 0.5 * (double)nd[d];
    }
    if (mode == 1 && c.np > 0 && LBM_LOCAL_SITES) {
        // particles: local marking, then the ordered compaction of the flags
        const int nblk = (int)((c.N + VTILE - 1) / VTILE);
        count_launch(c, G_GEOM, 6);  // with the link pass below
        bnd_clear_kernel<<<(unsigned)std::min<long long>(152LL * 8, (c.max_sites + 255) / 256), 256, 0, c.stream>>>(
            c.flags, c.site_cell, c.d_counts, c.max_sites);
        // the shared-memory tile of the largest particle's box and rim, when it is small
        const int T = 2 * ((int)ceil(c.max_radius) + 2) + 4;
        if ((long long)T * T * T <= 32768) bnd_mark_tile_kernel<<<c.np, 256, (size_t)T * T * T, c.stream>>>(a, T);
        else bnd_mark_kernel<<<c.np, 256, 0, c.stream>>>(a);
        bnd_count_kernel<<<nblk, CT, 0, c.stream>>>(a);
        site_scan_kernel<<<1, ST, 0, c.stream>>>(a, nblk);
        bnd_emit_kernel<<<nblk, CT, 0, c.stream>>>(a);
    } else {
        const int nblk = (int)((c.N + TILE - 1) / TILE);
        count_launch(c, G_GEOM, mode == 1 ? 4 : 3);
        site_count_kernel<<<nblk, CT, 0, c.stream>>>(a);
        site_scan_kernel<<<1, ST, 0, c.stream>>>(a, nblk);
        site_emit_kernel<<<nblk, CT, 0, c.stream>>>(a);
    }
    if (mode == 1) {
        cudaError_t e = cudaMemsetAsync(c.d_counts + 4, 0, sizeof(long long), c.stream);
        if (e != cudaSuccess) return e;
        long long n = c.nlinks_hint > 0 ? c.nlinks_hint : c.max_links;
        if (n > c.max_links) n = c.max_links;
        long long nb = (n + 255) / 256;
        if (nb < 1) nb = 1;
        if (nb > 152LL * 64) nb = 152LL * 64;
        if (a.site_geo) {
            long long sb = ((c.nlinks_hint > 0 ? c.nlinks_hint : c.max_sites) + 255) / 256;
            if (sb > 152LL * 16) sb = 152LL * 16;
            if (sb < 1) sb = 1;
            count_launch(c, G_GEOM);
            site_geo_kernel<<<(unsigned)sb, 256, 0, c.stream>>>(a);
        }
        link_geom_kernel<<<(unsigned)nb, 256, 0, c.stream>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace lbmgb
