// Fused pull-stream + collide sweeps (the dominant kernel of every step).
//
// stream_collide_bulk: one thread per cell, threads along x so that every
// population plane is read and written in coalesced rows; the 19 loads of a
// cell are independent and issued together. Cells that need a boundary
// treatment are left to the compact kernels below:
//   IBB: solid cells are skipped, boundary cells go to boundary_collide;
//   IBM: support cells only store rho and u* (first half of the direct
//        forcing, Sec. 2.1) and are collided later by ibm_collide.
// boundary_collide: interpolated bounce-back for the missing populations of
//   a boundary cell (Bouzidi et al. 2001 quadratic/linear, single-node
//   fallback; Sec. 3.1), then the same collision; it also records per link
//   the Galilean-invariant momentum exchange (Wen et al. 2014, Sec. 3.1).
// ibm_collide: collides support cells with the body force plus the IBM force
//   accumulated over the forcing passes.
#include "lbm_internal.cuh"

namespace lbmgb {

struct SweepArgs {
    const void *A;
    void *B;
    const uint8_t *flags;
    const int *aux;
    double *sup_rho, *sup_u;
    unsigned *status;
    long long max_sites;
    int nx, ny, nz;
    long long N;
    double F[3];
    Rates rt;
};

template <typename R>
__device__ __forceinline__ void watchdog(R rho, R ux, R uy, R uz, unsigned *status) {
    const R u2 = ux * ux + uy * uy + uz * uz;
    if (!(rho > R(0.5) && rho < R(2) && u2 < R(0.09))) atomicOr(status, 1u);
}

// BC: 0 periodic, 1 IBB, 2 IBM
template <int S, bool SRT, int BC, bool FORCE>
__global__ void __launch_bounds__(256) stream_collide_bulk(SweepArgs a) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const int rows = a.ny * a.nz;
    const int row = blockIdx.x * blockDim.y + threadIdx.y;
    if (row >= rows) return;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int y = row % ny, z = row / ny;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    // row offsets of the source rows (y - c_y, z - c_z)
    const int r00 = (y + ny * z) * nx;
    const int rM0 = (ym + ny * z) * nx, rP0 = (yp + ny * z) * nx;
    const int r0M = (y + ny * zm) * nx, r0P = (y + ny * zp) * nx;
    const int rMM = (ym + ny * zm) * nx, rPP = (yp + ny * zp) * nx;
    const int rMP = (ym + ny * zp) * nx, rPM = (yp + ny * zm) * nx;
    const T *__restrict__ A = (const T *)a.A;
    T *__restrict__ B = (T *)a.B;
    const size_t N = (size_t)a.N;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
        const int c = r00 + x;
        uint8_t fl = 0;
        if (BC != 0) {
            fl = a.flags[c];
            if (BC == 1 && (fl & (FL_SOLID | FL_BND))) continue;
        }
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        R g[19];
        // pull: f_i(x) = f*_i(x - c_i)
        g[0] = Store<S>::ld(A + c);
        g[1] = Store<S>::ld(A + 1 * N + r00 + xm);
        g[2] = Store<S>::ld(A + 2 * N + r00 + xp);
        g[3] = Store<S>::ld(A + 3 * N + rM0 + x);
        g[4] = Store<S>::ld(A + 4 * N + rP0 + x);
        g[5] = Store<S>::ld(A + 5 * N + r0M + x);
        g[6] = Store<S>::ld(A + 6 * N + r0P + x);
        g[7] = Store<S>::ld(A + 7 * N + rM0 + xm);
        g[8] = Store<S>::ld(A + 8 * N + rP0 + xp);
        g[9] = Store<S>::ld(A + 9 * N + rP0 + xm);
        g[10] = Store<S>::ld(A + 10 * N + rM0 + xp);
        g[11] = Store<S>::ld(A + 11 * N + r0M + xm);
        g[12] = Store<S>::ld(A + 12 * N + r0P + xp);
        g[13] = Store<S>::ld(A + 13 * N + r0P + xm);
        g[14] = Store<S>::ld(A + 14 * N + r0M + xp);
        g[15] = Store<S>::ld(A + 15 * N + rMM + x);
        g[16] = Store<S>::ld(A + 16 * N + rPP + x);
        g[17] = Store<S>::ld(A + 17 * N + rMP + x);
        g[18] = Store<S>::ld(A + 18 * N + rPM + x);
        const bool fluid = !(fl & FL_SOLID);
        if (BC == 2 && (fl & FL_SUP)) {
            // first half of direct forcing: rho and u* = (sum f c + F_ext/2)/rho
            R drho = g[0];
#pragma unroll
            for (int i = 1; i < 19; i++) drho += g[i];
            R jx = (g[1] - g[2]) + (g[7] - g[8]) + (g[9] - g[10]) + (g[11] - g[12]) + (g[13] - g[14]);
            R jy = (g[3] - g[4]) + (g[7] - g[8]) - (g[9] - g[10]) + (g[15] - g[16]) + (g[17] - g[18]);
            R jz = (g[5] - g[6]) + (g[11] - g[12]) - (g[13] - g[14]) + (g[15] - g[16]) - (g[17] - g[18]);
            if (FORCE && fluid) {
                jx += R(0.5) * R(a.F[0]);
                jy += R(0.5) * R(a.F[1]);
                jz += R(0.5) * R(a.F[2]);
            }
            const R rho = R(1) + drho;
            const int s = a.aux[c];
            if (s < 0 || s >= a.max_sites) continue;
            a.sup_rho[s] = double(rho);
            a.sup_u[3 * s + 0] = double(jx / rho);
            a.sup_u[3 * s + 1] = double(jy / rho);
            a.sup_u[3 * s + 2] = double(jz / rho);
            continue;
        }
        R rho, ux, uy, uz;
        if (FORCE && fluid)
            collide<R, true, SRT>(g, R(a.F[0]), R(a.F[1]), R(a.F[2]), a.rt, rho, ux, uy, uz);
        else
            collide<R, false, SRT>(g, R(0), R(0), R(0), a.rt, rho, ux, uy, uz);
        watchdog(rho, ux, uy, uz, a.status);
#pragma unroll
        for (int i = 0; i < 19; i++) Store<S>::st(B + i * N + c, g[i]);
    }
}

// ------------------------------------------------------------ IBB cells ----
struct BoundaryArgs {
    const void *A;
    void *B;
    const int *site_cell, *site_first;
    const unsigned *site_mask;
    const int8_t *link_scheme;
    const int *link_pid;
    const double *link_q;
    double *link_fin, *link_dP, *link_dT;
    const double *X, *U, *W;
    unsigned *status;
    const long long *counts;  // [0]: number of sites (device)
    long long max_sites;
    int nx, ny, nz;
    long long N;
    double F[3];
    Rates rt;
};

__device__ __forceinline__ double mimg(double d, int n) {
    if (d > 0.5 * n) d -= n;
    else if (d < -0.5 * n) d += n;
    return d;
}
__device__ __forceinline__ int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

template <int S, bool SRT, bool FORCE>
__global__ void __launch_bounds__(128) boundary_collide(BoundaryArgs a) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const long long ns = a.counts[0] < a.max_sites ? a.counts[0] : a.max_sites;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < ns;
         s += (long long)gridDim.x * blockDim.x) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int c = a.site_cell[s];
    const int first = a.site_first[s];
    const unsigned mask = a.site_mask[s];
    const int x = c % nx, y = (c / nx) % ny, z = c / (nx * ny);
    const T *__restrict__ A = (const T *)a.A;
    T *__restrict__ B = (T *)a.B;
    const size_t N = (size_t)a.N;
    R g[19];
#pragma unroll
    for (int i = 0; i < 19; i++) {
        const int l = opp(i);
        if (i > 0 && ((mask >> l) & 1u)) {
            // link l: x_f + c_l is solid; unknown population i = opp(l)
            const int k = first + __popc(mask & ((1u << l) - 1u));
            const int x1 = wrap(x + cx(i), nx), y1 = wrap(y + cy(i), ny), z1 = wrap(z + cz(i), nz);
            const int x2 = wrap(x1 + cx(i), nx), y2 = wrap(y1 + cy(i), ny), z2 = wrap(z1 + cz(i), nz);
            const int c1 = x1 + nx * (y1 + ny * z1), c2 = x2 + nx * (y2 + ny * z2);
            const R fl0 = Store<S>::ld(A + l * N + c);   // f*_l(x_f)
            const R fi0 = Store<S>::ld(A + i * N + c);   // f*_i(x_f)
            const double q = a.link_q[k];
            const int sch = a.link_scheme[k];
            const int pid = a.link_pid[k];
            double uw[3] = {0.0, 0.0, 0.0};
            if (pid >= 0) {
                const double r0 = mimg(x + q * cx(l) - a.X[3 * pid + 0], nx);
                const double r1 = mimg(y + q * cy(l) - a.X[3 * pid + 1], ny);
                const double r2 = mimg(z + q * cz(l) - a.X[3 * pid + 2], nz);
                const double *Wp = a.W + 3 * pid, *Up = a.U + 3 * pid;
                uw[0] = Up[0] + (Wp[1] * r2 - Wp[2] * r1);
                uw[1] = Up[1] + (Wp[2] * r0 - Wp[0] * r2);
                uw[2] = Up[2] + (Wp[0] * r1 - Wp[1] * r0);
            }
            const R D = R(6.0 * wgt(l) * (cx(i) * uw[0] + cy(i) * uw[1] + cz(i) * uw[2]));
            const R qq = R(q);
            R v;
            if (sch == 0) {
                if (qq < R(0.5)) {
                    const R fl1 = Store<S>::ld(A + l * N + c1), fl2 = Store<S>::ld(A + l * N + c2);
                    v = qq * (R(1) + R(2) * qq) * fl0 + (R(1) - R(4) * qq * qq) * fl1 -
                        qq * (R(1) - R(2) * qq) * fl2 + D;
                } else {
                    const R fi1 = Store<S>::ld(A + i * N + c1);
                    const R d = R(1) / (qq * (R(2) * qq + R(1)));
                    v = d * fl0 + (R(2) * qq - R(1)) / qq * fi0 - (R(2) * qq - R(1)) / (R(2) * qq + R(1)) * fi1 +
                        d * D;
                }
            } else if (sch == 1) {
                if (qq < R(0.5)) {
                    const R fl1 = Store<S>::ld(A + l * N + c1);
                    v = R(2) * qq * fl0 + (R(1) - R(2) * qq) * fl1 + D;
                } else {
                    const R h = R(1) / (R(2) * qq);
                    v = h * fl0 + (R(2) * qq - R(1)) * h * fi0 + h * D;
                }
            } else {
                v = fl0 + D;
            }
            g[i] = v;
            a.link_fin[k] = double(v);
            if (pid >= 0) {
                // momentum exchange on the link, unshifted f = g + w (w_l = w_i)
                const double fo = double(fl0) + wgt(l), fi = double(v) + wgt(i);
                double dP[3];
                dP[0] = (cx(l) - uw[0]) * fo - (cx(i) - uw[0]) * fi;
                dP[1] = (cy(l) - uw[1]) * fo - (cy(i) - uw[1]) * fi;
                dP[2] = (cz(l) - uw[2]) * fo - (cz(i) - uw[2]) * fi;
                const double m0 = mimg(x + 0.5 * cx(l) - a.X[3 * pid + 0], nx);
                const double m1 = mimg(y + 0.5 * cy(l) - a.X[3 * pid + 1], ny);
                const double m2 = mimg(z + 0.5 * cz(l) - a.X[3 * pid + 2], nz);
                a.link_dP[3 * k + 0] = dP[0];
                a.link_dP[3 * k + 1] = dP[1];
                a.link_dP[3 * k + 2] = dP[2];
                a.link_dT[3 * k + 0] = m1 * dP[2] - m2 * dP[1];
                a.link_dT[3 * k + 1] = m2 * dP[0] - m0 * dP[2];
                a.link_dT[3 * k + 2] = m0 * dP[1] - m1 * dP[0];
            }
        } else {
            const int xs = wrap(x - cx(i), nx), ys = wrap(y - cy(i), ny), zs = wrap(z - cz(i), nz);
            g[i] = Store<S>::ld(A + i * N + (xs + nx * (ys + ny * zs)));
        }
    }
    R rho, ux, uy, uz;
    if (FORCE)
        collide<R, true, SRT>(g, R(a.F[0]), R(a.F[1]), R(a.F[2]), a.rt, rho, ux, uy, uz);
    else
        collide<R, false, SRT>(g, R(0), R(0), R(0), a.rt, rho, ux, uy, uz);
    watchdog(rho, ux, uy, uz, a.status);
#pragma unroll
    for (int i = 0; i < 19; i++) Store<S>::st(B + i * N + c, g[i]);
    }
}

// ------------------------------------------------------------ IBM cells ----
struct IbmCollideArgs {
    const void *A;
    void *B;
    const int *site_cell;
    const uint8_t *flags;
    const double *sup_F;
    unsigned *status;
    const long long *counts;
    long long max_sites;
    int nx, ny, nz;
    long long N;
    double F[3];
    Rates rt;
};

template <int S, bool SRT>
__global__ void __launch_bounds__(128) ibm_collide(IbmCollideArgs a) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const long long ns = a.counts[0] < a.max_sites ? a.counts[0] : a.max_sites;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < ns;
         s += (long long)gridDim.x * blockDim.x) {
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int c = a.site_cell[s];
    const int x = c % nx, y = (c / nx) % ny, z = c / (nx * ny);
    const T *__restrict__ A = (const T *)a.A;
    T *__restrict__ B = (T *)a.B;
    const size_t N = (size_t)a.N;
    R g[19];
#pragma unroll
    for (int i = 0; i < 19; i++) {
        const int xs = wrap(x - cx(i), nx), ys = wrap(y - cy(i), ny), zs = wrap(z - cz(i), nz);
        g[i] = Store<S>::ld(A + i * N + (xs + nx * (ys + ny * zs)));
    }
    const bool fluid = !(a.flags[c] & FL_SOLID);
    const R Fx = R((fluid ? a.F[0] : 0.0) + a.sup_F[3 * s + 0]);
    const R Fy = R((fluid ? a.F[1] : 0.0) + a.sup_F[3 * s + 1]);
    const R Fz = R((fluid ? a.F[2] : 0.0) + a.sup_F[3 * s + 2]);
    R rho, ux, uy, uz;
    collide<R, true, SRT>(g, Fx, Fy, Fz, a.rt, rho, ux, uy, uz);
    watchdog(rho, ux, uy, uz, a.status);
#pragma unroll
    for (int i = 0; i < 19; i++) Store<S>::st(B + i * N + c, g[i]);
    }
}

// ------------------------------------------------------------- launchers ---
// Site kernels read the site count from device memory (it changes on the
// device when particles move) and stride over a grid sized by the smaller of
// the known count and the capacity.
static unsigned site_grid(const Ctx &c, int tb) {
    long long n = c.nsites_hint > 0 ? c.nsites_hint : c.max_sites;
    if (n > c.max_sites) n = c.max_sites;
    long long nb = (n + tb - 1) / tb;
    if (nb < 1) nb = 1;
    if (nb > 152LL * 64) nb = 152LL * 64;
    return (unsigned)nb;
}

template <int S, bool SRT, int BC>
static cudaError_t launch_bulk_t(Ctx &c, bool force) {
    SweepArgs a;
    a.A = c.fA;
    a.B = c.fB;
    a.flags = c.flags;
    a.aux = c.aux;
    a.sup_rho = c.sup_rho;
    a.sup_u = c.sup_u;
    a.status = c.d_status;
    a.max_sites = c.max_sites;
    a.nx = c.nx;
    a.ny = c.ny;
    a.nz = c.nz;
    a.N = c.N;
    for (int d = 0; d < 3; d++) a.F[d] = c.F[d];
    a.rt = c.rt;
    int bx = ((c.nx + 31) / 32) * 32;
    if (bx > 256) bx = 256;
    int by = 256 / bx;
    if (by < 1) by = 1;
    const int rows = c.ny * c.nz;
    dim3 block(bx, by), grid((rows + by - 1) / by);
    count_launch(c, G_BULK);
    if (force)
        stream_collide_bulk<S, SRT, BC, true><<<grid, block, 0, c.stream>>>(a);
    else
        stream_collide_bulk<S, SRT, BC, false><<<grid, block, 0, c.stream>>>(a);
    return cudaGetLastError();
}

template <int S>
static cudaError_t launch_bulk_s(Ctx &c, int bc, bool force) {
    const bool srt = c.rates == LBM_RATES_SRT;
    const int m = bc == LBM_BC_NONE ? 0 : (bc == LBM_BC_IBB ? 1 : 2);
    if (srt) {
        if (m == 0) return launch_bulk_t<S, true, 0>(c, force);
        if (m == 1) return launch_bulk_t<S, true, 1>(c, force);
        return launch_bulk_t<S, true, 2>(c, force);
    }
    if (m == 0) return launch_bulk_t<S, false, 0>(c, force);
    if (m == 1) return launch_bulk_t<S, false, 1>(c, force);
    return launch_bulk_t<S, false, 2>(c, force);
}

cudaError_t launch_stream_collide(Ctx &c, int bc) {
    const bool force = c.F[0] != 0.0 || c.F[1] != 0.0 || c.F[2] != 0.0;
    switch (c.storage) {
    case LBM_F64: return launch_bulk_s<LBM_F64>(c, bc, force);
    case LBM_F32: return launch_bulk_s<LBM_F32>(c, bc, force);
    case LBM_F16S: return launch_bulk_s<LBM_F16S>(c, bc, force);
    default: return launch_bulk_s<LBM_BF16S>(c, bc, force);
    }
}

template <int S>
static cudaError_t launch_boundary_s(Ctx &c) {
    if (c.max_sites == 0) return cudaSuccess;
    BoundaryArgs a;
    a.A = c.fA;
    a.B = c.fB;
    a.site_cell = c.site_cell;
    a.site_first = c.site_first;
    a.site_mask = c.site_mask;
    a.link_scheme = c.link_scheme;
    a.link_pid = c.link_pid;
    a.link_q = c.link_q;
    a.link_fin = c.link_fin;
    a.link_dP = c.link_dP;
    a.link_dT = c.link_dT;
    a.X = c.X;
    a.U = c.U;
    a.W = c.W;
    a.status = c.d_status;
    a.counts = c.d_counts;
    a.max_sites = c.max_sites;
    a.nx = c.nx;
    a.ny = c.ny;
    a.nz = c.nz;
    a.N = c.N;
    for (int d = 0; d < 3; d++) a.F[d] = c.F[d];
    a.rt = c.rt;
    const bool force = c.F[0] != 0.0 || c.F[1] != 0.0 || c.F[2] != 0.0;
    const int tb = 128;
    const unsigned nb = site_grid(c, tb);
    const bool srt = c.rates == LBM_RATES_SRT;
    count_launch(c, G_BND);
    if (srt) {
        if (force) boundary_collide<S, true, true><<<nb, tb, 0, c.stream>>>(a);
        else boundary_collide<S, true, false><<<nb, tb, 0, c.stream>>>(a);
    } else {
        if (force) boundary_collide<S, false, true><<<nb, tb, 0, c.stream>>>(a);
        else boundary_collide<S, false, false><<<nb, tb, 0, c.stream>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_boundary_collide(Ctx &c) {
    switch (c.storage) {
    case LBM_F64: return launch_boundary_s<LBM_F64>(c);
    case LBM_F32: return launch_boundary_s<LBM_F32>(c);
    case LBM_F16S: return launch_boundary_s<LBM_F16S>(c);
    default: return launch_boundary_s<LBM_BF16S>(c);
    }
}

template <int S>
static cudaError_t launch_ibm_s(Ctx &c) {
    if (c.max_sites == 0) return cudaSuccess;
    IbmCollideArgs a;
    a.A = c.fA;
    a.B = c.fB;
    a.site_cell = c.site_cell;
    a.flags = c.flags;
    a.sup_F = c.sup_F;
    a.status = c.d_status;
    a.counts = c.d_counts;
    a.max_sites = c.max_sites;
    a.nx = c.nx;
    a.ny = c.ny;
    a.nz = c.nz;
    a.N = c.N;
    for (int d = 0; d < 3; d++) a.F[d] = c.F[d];
    a.rt = c.rt;
    const int tb = 128;
    const unsigned nb = site_grid(c, tb);
    count_launch(c, G_IBMCOL);
    if (c.rates == LBM_RATES_SRT) ibm_collide<S, true><<<nb, tb, 0, c.stream>>>(a);
    else ibm_collide<S, false><<<nb, tb, 0, c.stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ibm_collide(Ctx &c) {
    switch (c.storage) {
    case LBM_F64: return launch_ibm_s<LBM_F64>(c);
    case LBM_F32: return launch_ibm_s<LBM_F32>(c);
    case LBM_F16S: return launch_ibm_s<LBM_F16S>(c);
    default: return launch_ibm_s<LBM_BF16S>(c);
    }
}

// ------------------------------------------------- population transfer ----
template <int S>
__global__ void set_pops_kernel(void *dst, const double *f, long long N) {
    typedef typename Store<S>::T T;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 19 * N) return;
    const int i = (int)(idx / N);
    Store<S>::st((T *)dst + idx, typename Store<S>::R(f[idx] - wgt(i)));
}

template <int S>
__global__ void get_pops_kernel(const void *src, double *f, long long N) {
    typedef typename Store<S>::T T;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 19 * N) return;
    const int i = (int)(idx / N);
    const T *p = (const T *)src + idx;
    double v;
    if (S == LBM_F64) v = (double)*(const double *)p;
    else if (S == LBM_F32) v = (double)*(const float *)p;
    else if (S == LBM_F16S) v = (double)__half2float(*(const __half *)p) / F16_SCALE;
    else v = (double)__bfloat162float(*(const __nv_bfloat16 *)p);
    f[idx] = v + wgt(i);
}

template <int S>
__global__ void init_eq_kernel(void *dst, const double *u, double rho0, long long N) {
    typedef typename Store<S>::T T;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const double ux = u[c], uy = u[N + c], uz = u[2 * N + c];
    const double u2 = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < 19; i++) {
        const double cu = cx(i) * ux + cy(i) * uy + cz(i) * uz;
        const double feq = wgt(i) * rho0 * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
        Store<S>::st((T *)dst + (size_t)i * N + c, typename Store<S>::R(feq - wgt(i)));
    }
}

cudaError_t launch_set_populations(Ctx &c, const double *f_dev) {
    const long long n = 19 * c.N;
    const unsigned nb = (unsigned)((n + 255) / 256);
    switch (c.storage) {
    case LBM_F64: set_pops_kernel<LBM_F64><<<nb, 256, 0, c.stream>>>(c.fA, f_dev, c.N); break;
    case LBM_F32: set_pops_kernel<LBM_F32><<<nb, 256, 0, c.stream>>>(c.fA, f_dev, c.N); break;
    case LBM_F16S: set_pops_kernel<LBM_F16S><<<nb, 256, 0, c.stream>>>(c.fA, f_dev, c.N); break;
    default: set_pops_kernel<LBM_BF16S><<<nb, 256, 0, c.stream>>>(c.fA, f_dev, c.N); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_get_populations(Ctx &c, double *f_dev) {
    const long long n = 19 * c.N;
    const unsigned nb = (unsigned)((n + 255) / 256);
    switch (c.storage) {
    case LBM_F64: get_pops_kernel<LBM_F64><<<nb, 256, 0, c.stream>>>(c.fA, f_dev, c.N); break;
    case LBM_F32: get_pops_kernel<LBM_F32><<<nb, 256, 0, c.stream>>>(c.fA, f_dev, c.N); break;
    case LBM_F16S: get_pops_kernel<LBM_F16S><<<nb, 256, 0, c.stream>>>(c.fA, f_dev, c.N); break;
    default: get_pops_kernel<LBM_BF16S><<<nb, 256, 0, c.stream>>>(c.fA, f_dev, c.N); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_init_equilibrium(Ctx &c, const double *u_dev, double rho0) {
    const unsigned nb = (unsigned)((c.N + 255) / 256);
    switch (c.storage) {
    case LBM_F64: init_eq_kernel<LBM_F64><<<nb, 256, 0, c.stream>>>(c.fA, u_dev, rho0, c.N); break;
    case LBM_F32: init_eq_kernel<LBM_F32><<<nb, 256, 0, c.stream>>>(c.fA, u_dev, rho0, c.N); break;
    case LBM_F16S: init_eq_kernel<LBM_F16S><<<nb, 256, 0, c.stream>>>(c.fA, u_dev, rho0, c.N); break;
    default: init_eq_kernel<LBM_BF16S><<<nb, 256, 0, c.stream>>>(c.fA, u_dev, rho0, c.N); break;
    }
    return cudaGetLastError();
}

}  // namespace lbmgb
