// Particle-side kernels, FP64 throughout:
//  - gimem_reduce: per-particle sum of the per-link momentum exchange
//    (Galilean-invariant form of Wen et al. 2014, Sec. 3.1);
//  - release_kernel: initial particle velocity = fluid velocity averaged
//    over the particle volume (Sec. 3.1);
//  - contact_kernel / eom_kernel: normal-only soft-sphere contacts and the
//    rigid-body update (Sec. 3.1);
//  - IBM: marker placement, support-cell marking, the three direct-forcing
//    passes (interpolate with the Peskin 4-point delta, force, spread;
//    Sec. 2.1 / 3.1) and the particle force with Kempe's inner-fluid term.
// All reductions are block trees in a fixed order (bitwise reproducible for
// a given launch configuration); only the IBM spreading uses FP64 atomics.
#include "lbm_internal.cuh"

namespace lbmgb {

__device__ __forceinline__ double pmimg(double d, int n) {
    if (d > 0.5 * n) d -= n;
    else if (d < -0.5 * n) d += n;
    return d;
}
// wrap a coordinate in [-n, 2n) into [0, n)
__device__ __forceinline__ int pwrap(int a, int n) {
    a = a < 0 ? a + n : a;
    return a >= n ? a - n : a;
}

constexpr int PB = 256;  // threads per particle block

// fixed-order block sum of NV doubles per thread; result valid in thread 0
template <int NV>
__device__ void block_sum(double v[NV], double *sh /* PB*NV */) {
    for (int k = 0; k < NV; k++) sh[k * PB + threadIdx.x] = v[k];
    __syncthreads();
    for (int s = PB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < NV; k++) sh[k * PB + threadIdx.x] += sh[k * PB + threadIdx.x + s];
        __syncthreads();
    }
    for (int k = 0; k < NV; k++) v[k] = sh[k * PB];
}

// ------------------------------------------------------------ GIMEM ------
struct GimemArgs {
    const uint8_t *flags;
    const int *aux, *site_first, *link_pid;
    const unsigned *site_mask;
    const void *link_dP, *link_dT;  // arithmetic type of the storage
    const double *X, *R;
    double *Fh, *Th;
    int nx, ny, nz;
    long long max_sites;
};

template <typename Rl>
__global__ void __launch_bounds__(PB) gimem_reduce_kernel(GimemArgs a) {
    const Rl *dP = (const Rl *)a.link_dP, *dT = (const Rl *)a.link_dT;
    __shared__ double sh[6 * PB];
    const int p = blockIdx.x;
    const int r = (int)ceil(a.R[p]) + 2;
    const int bx = (int)floor(a.X[3 * p]) - r, by = (int)floor(a.X[3 * p + 1]) - r, bz = (int)floor(a.X[3 * p + 2]) - r;
    const int w = 2 * r + 2;
    // per-thread partial sums in the storage's arithmetic type (a few links
    // each), then the fixed-order FP64 block sum
    Rl v[6] = {0, 0, 0, 0, 0, 0};
    const FastDiv fw((unsigned)w);
    // a link of p starts within R_p + sqrt 2 of its centre
    const float reach = (float)a.R[p] + 1.5f, reach2 = reach * reach;
    const float fX0 = (float)a.X[3 * p] - bx, fX1 = (float)a.X[3 * p + 1] - by, fX2 = (float)a.X[3 * p + 2] - bz;
    for (int t = threadIdx.x; t < w * w * w; t += PB) {
        int ix, iy, iz;
        box_coords(t, fw, w, ix, iy, iz);
        const float ex = ix - fX0, ey = iy - fX1, ez = iz - fX2;
        if (ex * ex + ey * ey + ez * ez > reach2) continue;
        const int x = pwrap(bx + ix, a.nx), y = pwrap(by + iy, a.ny), z = pwrap(bz + iz, a.nz);
        const long long c = (long long)x + (long long)a.nx * (y + (long long)a.ny * z);
        if (!(a.flags[c] & FL_BND)) continue;
        const int s = a.aux[c];
        if (s < 0 || s >= a.max_sites) continue;
        const int first = a.site_first[s];
        const int n = __popc(a.site_mask[s]);
        for (int k = first; k < first + n; k++) {
            if (a.link_pid[k] != p) continue;
            for (int d = 0; d < 3; d++) {
                v[d] += dP[3 * k + d];
                v[3 + d] += dT[3 * k + d];
            }
        }
    }
    double vd[6];
    for (int d = 0; d < 6; d++) vd[d] = double(v[d]);
    block_sum<6>(vd, sh);
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; d++) {
            a.Fh[3 * p + d] = vd[d];
            a.Th[3 * p + d] = vd[3 + d];
        }
}

cudaError_t launch_gimem(Ctx &c) {
    if (c.np == 0) return cudaSuccess;
    GimemArgs a{c.flags, c.aux, c.site_first, c.link_pid, c.site_mask, c.link_dP, c.link_dT,
                c.X, c.R, c.Fh, c.Th, c.nx, c.ny, c.nz, c.max_sites};
    count_launch(c, G_PART);
    if (c.storage == LBM_F64)
        gimem_reduce_kernel<double><<<c.np, PB, 0, c.stream>>>(a);
    else
        gimem_reduce_kernel<float><<<c.np, PB, 0, c.stream>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------- solid fraction ----
// Kempe et al. (2012): alpha = sum(-phi H(-phi)) / sum|phi| over the 8 cell
// corners, phi = |x - X| - R (x relative to the particle, minimum image),
// in the arithmetic type R of the storage.
template <typename R>
__device__ R solid_fraction(R rx, R ry, R rz, R Rp) {
    R num = 0, den = 0;
    for (int m = 0; m < 8; m++) {
        const R ax = rx + ((m & 1) ? R(0.5) : R(-0.5)), ay = ry + ((m & 2) ? R(0.5) : R(-0.5)),
                az = rz + ((m & 4) ? R(0.5) : R(-0.5));
        const R phi = sqrt(ax * ax + ay * ay + az * az) - Rp;
        if (phi < R(0)) num += -phi;
        den += fabs(phi);
    }
    return den > R(0) ? num / den : R(0);
}

// velocity of the post-collision state of cell c: (sum f c - F/2) / rho
template <int S>
__device__ void cell_velocity(const void *A, size_t N, long long c, double Fx, double Fy, double Fz, double &rho,
                              double u[3]) {
    typedef typename Store<S>::T T;
    const T *P = (const T *)A;
    double r = 0.0, j0 = 0.0, j1 = 0.0, j2 = 0.0;
    for (int i = 0; i < 19; i++) {
        double g;
        if (S == LBM_F64) g = *(const double *)(P + i * N + c);
        else if (S == LBM_F32) g = *(const float *)(P + i * N + c);
        else if (S == LBM_F16S) g = (double)__half2float(*(const __half *)(P + i * N + c)) / (double)F16_SCALE;
        else g = (double)__bfloat162float(*(const __nv_bfloat16 *)(P + i * N + c));
        r += g;
        j0 += g * cx(i);
        j1 += g * cy(i);
        j2 += g * cz(i);
    }
    rho = 1.0 + r;
    u[0] = (j0 - 0.5 * Fx) / rho;
    u[1] = (j1 - 0.5 * Fy) / rho;
    u[2] = (j2 - 0.5 * Fz) / rho;
}

struct VolArgs {
    const void *A;
    const uint8_t *flags;
    const int *aux;
    const void *sup_ru;  // (rho, u*) per support site, arithmetic type of the storage
    const double *X, *R;
    double *out_u, *out_r;  // per particle (3): sum alpha u and sum alpha r x u (or averages)
    int nx, ny, nz;
    long long N;
    double F[3];
    int mode;  // 0: release average from populations, 1: Kempe integrals from populations, 2: from sup_u
    long long max_sites;
};

template <int S>
__global__ void __launch_bounds__(PB) volume_kernel(VolArgs a) {
    typedef typename Store<S>::R Rt;
    __shared__ double sh[7 * PB];
    const int p = blockIdx.x;
    const double *Xp = a.X + 3 * p;
    const double Rp = a.R[p];
    const int r = (int)ceil(Rp) + 1;
    const int bx = (int)floor(Xp[0]) - r, by = (int)floor(Xp[1]) - r, bz = (int)floor(Xp[2]) - r;
    const int w = 2 * r + 2;
    // cell offsets relative to the particle: integer part exact, fraction in Rt
    const double fx = Xp[0] - floor(Xp[0]), fy = Xp[1] - floor(Xp[1]), fz = Xp[2] - floor(Xp[2]);
    Rt v[7] = {0, 0, 0, 0, 0, 0, 0};
    const Rt *su = (const Rt *)a.sup_ru;
    const FastDiv fw((unsigned)w);
    for (int t = threadIdx.x; t < w * w * w; t += PB) {
        int ix, iy, iz;
        box_coords(t, fw, w, ix, iy, iz);
        const int x = pwrap(bx + ix, a.nx), y = pwrap(by + iy, a.ny), z = pwrap(bz + iz, a.nz);
        const Rt rx = Rt(ix - r) - Rt(fx), ry = Rt(iy - r) - Rt(fy), rz = Rt(iz - r) - Rt(fz);
        const Rt al = solid_fraction<Rt>(rx, ry, rz, Rt(Rp));
        if (al <= Rt(0)) continue;
        const long long c = (long long)x + (long long)a.nx * (y + (long long)a.ny * z);
        Rt u[3];
        if (a.mode == 2) {
            const int s = a.aux[c];
            if (s < 0 || s >= a.max_sites) continue;
            u[0] = su[4 * s + 1];
            u[1] = su[4 * s + 2];
            u[2] = su[4 * s + 3];
        } else {
            double rho, ud[3];
            const bool fluid = a.mode == 0 ? true : !(a.flags[c] & FL_SOLID);
            cell_velocity<S>(a.A, (size_t)a.N, c, fluid ? a.F[0] : 0.0, fluid ? a.F[1] : 0.0, fluid ? a.F[2] : 0.0,
                             rho, ud);
            u[0] = Rt(ud[0]);
            u[1] = Rt(ud[1]);
            u[2] = Rt(ud[2]);
        }
        v[0] += al * u[0];
        v[1] += al * u[1];
        v[2] += al * u[2];
        v[3] += al * (ry * u[2] - rz * u[1]);
        v[4] += al * (rz * u[0] - rx * u[2]);
        v[5] += al * (rx * u[1] - ry * u[0]);
        v[6] += al;
    }
    double vd[7];
    for (int k = 0; k < 7; k++) vd[k] = double(v[k]);
    block_sum<7>(vd, sh);
    if (threadIdx.x == 0) {
        if (a.mode == 0) {
            for (int d = 0; d < 3; d++) a.out_u[3 * p + d] = vd[6] > 0.0 ? vd[d] / vd[6] : 0.0;
        } else {
            for (int d = 0; d < 3; d++) {
                a.out_u[3 * p + d] = vd[d];
                a.out_r[3 * p + d] = vd[3 + d];
            }
        }
    }
}

static cudaError_t launch_volume(Ctx &c, int mode, double *out_u, double *out_r) {
    if (c.np == 0) return cudaSuccess;
    count_launch(c, G_PART);
    VolArgs a{c.fA, c.flags, c.aux, c.sup_ru, c.X, c.R, out_u, out_r, c.nx, c.ny, c.nz, c.N,
              {c.F[0], c.F[1], c.F[2]}, mode, c.max_sites};
    switch (c.storage) {
    case LBM_F64: volume_kernel<LBM_F64><<<c.np, PB, 0, c.stream>>>(a); break;
    case LBM_F32: volume_kernel<LBM_F32><<<c.np, PB, 0, c.stream>>>(a); break;
    case LBM_F16S: volume_kernel<LBM_F16S><<<c.np, PB, 0, c.stream>>>(a); break;
    default: volume_kernel<LBM_BF16S><<<c.np, PB, 0, c.stream>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_release(Ctx &c) { return launch_volume(c, 0, c.U, nullptr); }

// ------------------------------------------------------- contacts, EOM ----
struct EomArgs {
    double *X, *Xold, *U, *W, *Fh, *Th, *Fprev, *Tprev, *Fc;
    const double *R, *mass, *inertia;
    int *has_prev;
    int np, nx, ny, nz;
    float4 *Xf;  // FP32 copies of the centres and radii for the contact search's cull
};

// FP32 centre and radius of every particle: the contact search culls pairs
// on these (one FP64-to-FP32 conversion per particle instead of per pair)
__global__ void xf_kernel(EomArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < a.np) a.Xf[p] = make_float4((float)a.X[3 * p], (float)a.X[3 * p + 1], (float)a.X[3 * p + 2], (float)a.R[p]);
}

// Normal-only soft-sphere contact (Sec. 3.1): for a gap below zeta = 1, a
// spring-dashpot along the line of centres, k_n = m (pi^2 + ln^2 e)/Tc^2,
// eta_n = -2 m ln e / Tc, m the reduced mass, e = 0.97, Tc = 10 steps.
// One warp per particle; lanes stride over partners, cull in FP32 with a
// margin and evaluate the few close pairs in FP64 (each pair as (a < b));
// the lane sums are reduced in a fixed butterfly order.
__global__ void __launch_bounds__(256) contact_kernel(EomArgs a) {
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= a.np) return;
    const double zeta = 1.0, e = 0.97, Tc = 10.0, PI = 3.14159265358979323846;
    const float hx = 0.5f * a.nx, hy = 0.5f * a.ny, hz = 0.5f * a.nz;
    const float4 P = a.Xf[p];
    double F[3] = {0.0, 0.0, 0.0};
    for (int q = lane; q < a.np; q += 32) {
        if (q == p) continue;
        const float4 Q = a.Xf[q];
        float dx = P.x - Q.x, dy = P.y - Q.y, dz = P.z - Q.z;
        dx = dx > hx ? dx - a.nx : (dx < -hx ? dx + a.nx : dx);
        dy = dy > hy ? dy - a.ny : (dy < -hy ? dy + a.ny : dy);
        dz = dz > hz ? dz - a.nz : (dz < -hz ? dz + a.nz : dz);
        const float reach = P.w + Q.w + (float)zeta + 0.01f;
        if (dx * dx + dy * dy + dz * dz >= reach * reach) continue;
        const int ia = q < p ? q : p, ib = q < p ? p : q;  // pair evaluated as (a < b)
        const double d0 = pmimg(a.X[3 * ia] - a.X[3 * ib], a.nx), d1 = pmimg(a.X[3 * ia + 1] - a.X[3 * ib + 1], a.ny),
                     d2 = pmimg(a.X[3 * ia + 2] - a.X[3 * ib + 2], a.nz);
        const double dist = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        const double gap = dist - (a.R[ia] + a.R[ib]);
        if (gap >= zeta || dist <= 0.0) continue;
        const double n0 = d0 / dist, n1 = d1 / dist, n2 = d2 / dist;
        const double vn = (a.U[3 * ia] - a.U[3 * ib]) * n0 + (a.U[3 * ia + 1] - a.U[3 * ib + 1]) * n1 +
                          (a.U[3 * ia + 2] - a.U[3 * ib + 2]) * n2;
        const double meff = a.mass[ia] * a.mass[ib] / (a.mass[ia] + a.mass[ib]);
        const double le = log(e);
        const double kn = meff * (PI * PI + le * le) / (Tc * Tc);
        const double eta = -2.0 * meff * le / Tc;
        const double Fm = kn * (zeta - gap) - eta * vn;
        const double sg = q < p ? -1.0 : 1.0;
        F[0] += sg * (Fm * n0);
        F[1] += sg * (Fm * n1);
        F[2] += sg * (Fm * n2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        for (int d = 0; d < 3; d++) F[d] += __shfl_xor_sync(0xffffffffu, F[d], o);
    if (lane == 0)
        for (int d = 0; d < 3; d++) a.Fc[3 * p + d] = F[d];
}

// U += ((F_h^n + F_h^{n-1})/2 + F_c)/m, W += (T^n + T^{n-1})/(2 I), X += U_new.
__global__ void eom_kernel(EomArgs a) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.np) return;
    const int n[3] = {a.nx, a.ny, a.nz};
    const bool hp = a.has_prev[p] != 0;
    for (int d = 0; d < 3; d++) {
        const double Fh = a.Fh[3 * p + d], Th = a.Th[3 * p + d];
        const double Fa = hp ? 0.5 * (Fh + a.Fprev[3 * p + d]) : Fh;
        const double Ta = hp ? 0.5 * (Th + a.Tprev[3 * p + d]) : Th;
        const double u1 = a.U[3 * p + d] + (Fa + a.Fc[3 * p + d]) / a.mass[p];
        a.U[3 * p + d] = u1;
        a.W[3 * p + d] += Ta / a.inertia[p];
        a.Xold[3 * p + d] = a.X[3 * p + d];
        double x = a.X[3 * p + d] + u1;
        if (x >= n[d]) x -= n[d];
        if (x < 0.0) x += n[d];
        a.X[3 * p + d] = x;
        a.Fprev[3 * p + d] = Fh;
        a.Tprev[3 * p + d] = Th;
    }
    a.has_prev[p] = 1;
}

cudaError_t launch_particle_update(Ctx &c) {
    if (c.np == 0) return cudaSuccess;
    EomArgs a{c.X, c.Xold, c.U, c.W, c.Fh, c.Th, c.Fprev, c.Tprev, c.Fc, c.R, c.mass, c.inertia, c.has_prev,
              c.np, c.nx, c.ny, c.nz, c.Xf};
    const int tb = 128, nb = (c.np + tb - 1) / tb;
    count_launch(c, G_PART, 3);
    xf_kernel<<<nb, tb, 0, c.stream>>>(a);
    contact_kernel<<<(c.np * 32 + 255) / 256, 256, 0, c.stream>>>(a);
    eom_kernel<<<nb, tb, 0, c.stream>>>(a);
    return cudaGetLastError();
}

// -------------------------------------------------------------- IBM ------
__device__ __forceinline__ double peskin(double r) {
    const double a = fabs(r);
    if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) * 0.125;
    if (a <= 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) * 0.125;
    return 0.0;
}

__global__ void markers_place_kernel(double *mX, const double *mUnit, const int *mpid, const double *X, long long nm,
                                     int nx, int ny, int nz) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nm) return;
    const int p = mpid[l];
    const int n[3] = {nx, ny, nz};
    for (int d = 0; d < 3; d++) {
        double x = X[3 * p + d] + mUnit[3 * l + d];
        if (x >= n[d]) x -= n[d];
        if (x < 0.0) x += n[d];
        mX[3 * l + d] = x;
    }
}

// per marker: first stencil node floor(X) - 1 (wrapped), X - floor(X), and
// the desired velocity U_d = U_p + Omega_p x (X_l - X_p) of the rigid body
// (zero for the pipe's ring markers), evaluated in FP64 once per step
template <typename R>
__global__ void marker_offsets_kernel(const double *mX, int *mB, R *mE, R *mUd, const int *mpid, const double *X,
                                      const double *U, const double *W, long long nm, int nx, int ny, int nz) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nm) return;
    const int n[3] = {nx, ny, nz};
    for (int d = 0; d < 3; d++) {
        const double x = mX[3 * l + d], f = floor(x);
        mB[3 * l + d] = pwrap((int)f - 1, n[d]);
        mE[3 * l + d] = R(x - f);
    }
    double Ud[3] = {0.0, 0.0, 0.0};
    const int p = mpid[l];
    if (p >= 0) {
        const double r0 = pmimg(mX[3 * l] - X[3 * p], nx), r1 = pmimg(mX[3 * l + 1] - X[3 * p + 1], ny),
                     r2 = pmimg(mX[3 * l + 2] - X[3 * p + 2], nz);
        const double *Wp = W + 3 * p, *Up = U + 3 * p;
        Ud[0] = Up[0] + (Wp[1] * r2 - Wp[2] * r1);
        Ud[1] = Up[1] + (Wp[2] * r0 - Wp[0] * r2);
        Ud[2] = Up[2] + (Wp[0] * r1 - Wp[1] * r0);
    }
    for (int d = 0; d < 3; d++) mUd[3 * l + d] = R(Ud[d]);
}

cudaError_t launch_marker_offsets(Ctx &c) {
    if (c.nm == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((c.nm + 255) / 256);
    count_launch(c, G_GEOM);
    if (c.storage == LBM_F64)
        marker_offsets_kernel<double><<<nb, 256, 0, c.stream>>>(c.mX, c.mB, (double *)c.mE, (double *)c.mUd, c.mpid,
                                                                c.X, c.U, c.W, c.nm, c.nx, c.ny, c.nz);
    else
        marker_offsets_kernel<float><<<nb, 256, 0, c.stream>>>(c.mX, c.mB, (float *)c.mE, (float *)c.mUd, c.mpid,
                                                               c.X, c.U, c.W, c.nm, c.nx, c.ny, c.nz);
    return cudaGetLastError();
}

cudaError_t launch_markers_place(Ctx &c) {
    if (c.np == 0 || c.nm == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((c.nm + 127) / 128);
    count_launch(c, G_GEOM);
    markers_place_kernel<<<nb, 128, 0, c.stream>>>(c.mX, c.mUnit, c.mpid, c.X, c.nm, c.nx, c.ny, c.nz);
    return cudaGetLastError();
}

__device__ __forceinline__ void flag_or(uint8_t *flags, long long c, uint8_t bit) {
    unsigned *w = (unsigned *)(flags + (c & ~3LL));
    atomicOr(w, ((unsigned)bit) << (8 * (c & 3)));
}

__global__ void clear_sup_kernel(uint8_t *flags, long long N) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const uint8_t f = flags[c];
    if (f & FL_SUP) flags[c] = (uint8_t)(f & ~FL_SUP);
}

// support = 4x4x4 stencil of every marker
__global__ void mark_stencil_kernel(uint8_t *flags, const double *mX, long long nm, int nx, int ny, int nz) {
    const long long l = (long long)blockIdx.x * (blockDim.x / 64) + threadIdx.x / 64;
    if (l >= nm) return;
    const int k = threadIdx.x & 63;
    const int ox = k & 3, oy = (k >> 2) & 3, oz = k >> 4;
    const int x = pwrap((int)floor(mX[3 * l]) - 1 + ox, nx), y = pwrap((int)floor(mX[3 * l + 1]) - 1 + oy, ny),
              z = pwrap((int)floor(mX[3 * l + 2]) - 1 + oz, nz);
    flag_or(flags, (long long)x + (long long)nx * (y + (long long)ny * z), FL_SUP);
}

// ... plus every cell overlapping a particle (|x - X| < R + 1), whose
// velocity enters the inner-fluid integrals
__global__ void mark_interior_kernel(uint8_t *flags, const double *X, const double *R, int nx, int ny, int nz) {
    const int p = blockIdx.x;
    const double Rp = R[p];
    const int r = (int)ceil(Rp) + 1;
    const int bx = (int)floor(X[3 * p]) - r, by = (int)floor(X[3 * p + 1]) - r, bz = (int)floor(X[3 * p + 2]) - r;
    const int w = 2 * r + 2;
    const FastDiv fw((unsigned)w);
    for (int t = threadIdx.x; t < w * w * w; t += blockDim.x) {
        int ix, iy, iz;
        box_coords(t, fw, w, ix, iy, iz);
        const int x = pwrap(bx + ix, nx), y = pwrap(by + iy, ny), z = pwrap(bz + iz, nz);
        const double rx = pmimg(x - X[3 * p], nx), ry = pmimg(y - X[3 * p + 1], ny), rz = pmimg(z - X[3 * p + 2], nz);
        if (rx * rx + ry * ry + rz * rz < (Rp + 1.0) * (Rp + 1.0))
            flag_or(flags, (long long)x + (long long)nx * (y + (long long)ny * z), FL_SUP);
    }
}

cudaError_t launch_support_mark(Ctx &c) {
    const unsigned nb = (unsigned)((c.N + 255) / 256);
    count_launch(c, G_GEOM, 1 + (c.nm > 0) + (c.np > 0));
    clear_sup_kernel<<<nb, 256, 0, c.stream>>>(c.flags, c.N);
    if (c.nm > 0) {
        const unsigned mb = (unsigned)((c.nm + 3) / 4);
        mark_stencil_kernel<<<mb, 256, 0, c.stream>>>(c.flags, c.mX, c.nm, c.nx, c.ny, c.nz);
    }
    if (c.np > 0) mark_interior_kernel<<<c.np, 256, 0, c.stream>>>(c.flags, c.X, c.R, c.nx, c.ny, c.nz);
    return cudaGetLastError();
}

// Peskin (2002) 4-point kernel in the arithmetic type R of the storage
template <typename R>
__device__ __forceinline__ R peskin_r(R r) {
    const R a = fabs(r);
    if (a <= R(1)) return (R(3) - R(2) * a + sqrt(R(1) + R(4) * a - R(4) * a * a)) * R(0.125);
    if (a <= R(2)) return (R(5) - R(2) * a - sqrt(R(-7) + R(12) * a - R(4) * a * a)) * R(0.125);
    return R(0);
}

// Support-cell data (rho, u*, accumulated force, force of the pass) and the
// marker forces used for spreading are held in R: double for FP64 storage,
// float otherwise (FP64 arithmetic is slow on this GPU and would dominate).
struct IbmArgs {
    const double *mX, *mdV;
    const int *mpid;
    double *mFacc;        // per-step marker force (sum of the passes), FP64
    const void *mUd;      // desired velocity U_d at the marker (R)
    void *mFaccR, *mFr;   // running sum of the passes' forces; F_l dV_l of this pass for the spreading (R)
    const int *mB;
    const void *mE;
    const int *aux;
    void *sup_ru, *sup_F, *sup_Fp;
    const double *X, *U, *W;
    long long nm;
    const long long *counts;
    long long max_sites;
    int nx, ny, nz;
    int pass, last;
};

// (rho, u*) of one support site: one 16-byte load in FP32
__device__ __forceinline__ void ld_site4(const float *p, float q[4]) {
    const float4 v = __ldg((const float4 *)p);
    q[0] = v.x;
    q[1] = v.y;
    q[2] = v.z;
    q[3] = v.w;
}
__device__ __forceinline__ void ld_site4(const double *p, double q[4]) {
    const double2 v0 = __ldg((const double2 *)p), v1 = __ldg((const double2 *)p + 1);
    q[0] = v0.x;
    q[1] = v0.y;
    q[2] = v1.x;
    q[3] = v1.y;
}

// Interpolation, one warp per marker: lane k takes stencil nodes k and k+32;
// U*_l = sum u* delta, rho_l = sum rho delta (fixed butterfly reduction);
// F_l = 2 rho_l (U_d - U*_l).
template <typename R>
__global__ void __launch_bounds__(256) ibm_interp_warp_kernel(IbmArgs a) {
    const long long l = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (l >= a.nm) return;
    const R *ru = (const R *)a.sup_ru;
    const R *E = (const R *)a.mE + 3 * l;
    const R e0 = E[0], e1 = E[1], e2 = E[2];  // X - floor(X)
    const int b0 = a.mB[3 * l], b1 = a.mB[3 * l + 1], b2 = a.mB[3 * l + 2];  // floor(X) - 1, wrapped
    // the 12 one-dimensional kernel values of the marker: lane 4 d + o holds
    // phi(o - 1 - e_d); every node's weight is a product of three of them
    R phi = R(0);
    if (lane < 12) {
        const int d = lane >> 2, o = lane & 3;
        phi = peskin_r<R>(R(o - 1) - (d == 0 ? e0 : (d == 1 ? e1 : e2)));
    }
    R U0 = 0, U1 = 0, U2 = 0, rl = 0;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int k = lane + 32 * h;
        const int kx = k & 3, ky = (k >> 2) & 3, kz = k >> 4;
        const R w = __shfl_sync(0xffffffffu, phi, kx) * __shfl_sync(0xffffffffu, phi, 4 + ky) *
                    __shfl_sync(0xffffffffu, phi, 8 + kz);
        const long long c = (long long)pwrap(b0 + kx, a.nx) +
                            (long long)a.nx * (pwrap(b1 + ky, a.ny) + (long long)a.ny * pwrap(b2 + kz, a.nz));
        const int s = a.aux[c];
        if (s < 0 || s >= a.max_sites) continue;
        R q[4];
        ld_site4(ru + 4 * (size_t)s, q);
        rl += w * q[0];
        U0 += w * q[1];
        U1 += w * q[2];
        U2 += w * q[3];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rl += __shfl_xor_sync(0xffffffffu, rl, o);
        U0 += __shfl_xor_sync(0xffffffffu, U0, o);
        U1 += __shfl_xor_sync(0xffffffffu, U1, o);
        U2 += __shfl_xor_sync(0xffffffffu, U2, o);
    }
    if (lane != 0) return;
    // F_l = 2 rho_l (U_d - U*_l) in the storage's arithmetic type; U_d was
    // evaluated once per step (marker_offsets_kernel)
    const R *Ud = (const R *)a.mUd + 3 * l;
    const R U[3] = {U0, U1, U2};
    R *mFr = (R *)a.mFr, *acc = (R *)a.mFaccR;
    const R dVl = R(a.mdV[l]);
    for (int d = 0; d < 3; d++) {
        const R Fl = R(2) * rl * (Ud[d] - U[d]);
        mFr[3 * l + d] = Fl * dVl;  // spread weight F_l dV_l
        const R s = a.pass == 0 ? Fl : acc[3 * l + d] + Fl;
        acc[3 * l + d] = s;
        if (a.last) a.mFacc[3 * l + d] = double(s);
    }
}

// Pipe wall tiles. The ring of markers is the same in every z plane and sits
// at integer z, so the z factor of the 4-point kernel takes the constants
// phi(0) = 1/2, phi(+-1) = 1/4 (phi(+-2) = 0), and the x-y factor of every
// (marker, site) pair is the same in all planes. A block takes 32 ring
// markers (or 32 sites of a plane) over PIPE_ZT consecutive planes: it forms
// the x-y sums once per plane, for its planes and one halo plane on each
// side, in shared memory, and combines three neighbouring planes per output.
// Each plane's x-y sum is gathered once instead of three times.
#ifndef LBM_PIPE_ZT
#define LBM_PIPE_ZT 6  // measured: 6, 14, 30 planes -> 0.165, 0.166, 0.176 ms for 3 passes
#endif
constexpr int PIPE_ZT = LBM_PIPE_ZT;
constexpr int PIPE_ZH = PIPE_ZT + 2;  // with the halo planes

__device__ __forceinline__ int zwrap(int z, int nz) {
    z %= nz;
    return z < 0 ? z + nz : z;
}

struct PipeInterpArgs {
    const int *it_k;
    const void *it_w;  // R
    const void *sup_ru;
    double *mFacc;
    void *mFaccR, *mFr;
    int nc, nz, sp, pass, last;
    double dV;  // ring marker volume
};

// U*_l = sum over planes dz = -1, 0, 1 of phi_z(dz) times the sum over the
// 16 column entries of ring marker j of w_xy u*(site) in plane z + dz (the
// 4-point delta interpolation, Sec. 3.1); then the direct-forcing force
// F_l = 2 rho_l (U_d - U*_l) with U_d = 0 on the fixed wall (Sec. 2.1)
template <typename R>
__global__ void __launch_bounds__(256) ibm_interp_pipe_kernel(PipeInterpArgs a) {
    __shared__ R P[PIPE_ZH][32][4];
    const int jj = threadIdx.x & 31, j = blockIdx.x * 32 + jj;
    const int z0 = blockIdx.y * PIPE_ZT;
    const R *ru = (const R *)a.sup_ru;
    const R *tw = (const R *)a.it_w + 16 * (size_t)j;
    const int *tk = a.it_k + 16 * (size_t)j;
    for (int pz = threadIdx.x >> 5; pz < PIPE_ZH; pz += blockDim.x >> 5) {
        R q[4] = {R(0), R(0), R(0), R(0)};
        if (j < a.nc) {
            // all 16 gathers in flight at once (an entry without a site has
            // weight 0 and index 0: its load is in bounds and not summed)
            const R *rp = ru + 4 * (size_t)zwrap(z0 - 1 + pz, a.nz) * a.sp;
            R v[16][4];
#pragma unroll
            for (int e = 0; e < 16; e++) ld_site4(rp + 4 * (size_t)tk[e], v[e]);
#pragma unroll
            for (int e = 0; e < 16; e++) {
                const R w = tw[e];
                if (w != R(0))
                    for (int d = 0; d < 4; d++) q[d] += w * v[e][d];
            }
        }
        for (int d = 0; d < 4; d++) P[pz][jj][d] = q[d];
    }
    __syncthreads();
    if (j >= a.nc) return;
    R *mFr = (R *)a.mFr, *acc = (R *)a.mFaccR;
    const R dVl = R(a.dV);
    for (int pz = threadIdx.x >> 5; pz < PIPE_ZT; pz += blockDim.x >> 5) {
        const int z = z0 + pz;
        if (z >= a.nz) break;
        const long long l = (long long)z * a.nc + j;
        R q[4];
        for (int d = 0; d < 4; d++) q[d] = R(0.25) * P[pz][jj][d] + R(0.5) * P[pz + 1][jj][d] + R(0.25) * P[pz + 2][jj][d];
        for (int d = 0; d < 3; d++) {
            const R Fl = R(2) * q[0] * (R(0) - q[1 + d]);
            mFr[3 * l + d] = Fl * dVl;  // spread weight F_l dV_l
            const R s = a.pass == 0 ? Fl : acc[3 * l + d] + Fl;
            acc[3 * l + d] = s;
            if (a.last) a.mFacc[3 * l + d] = double(s);
        }
    }
}

// generic spreading with global atomics (large particles only)
template <typename R>
__global__ void ibm_spread_kernel(IbmArgs a) {
    const long long l = (long long)blockIdx.x * (blockDim.x / 64) + threadIdx.x / 64;
    if (l >= a.nm) return;
    const int k = threadIdx.x & 63;
    const int kx = k & 3, ky = (k >> 2) & 3, kz = k >> 4;
    const R *E = (const R *)a.mE + 3 * l;
    const int b0 = a.mB[3 * l], b1 = a.mB[3 * l + 1], b2 = a.mB[3 * l + 2];
    const R w = peskin_r<R>(R(kx - 1) - E[0]) * peskin_r<R>(R(ky - 1) - E[1]) * peskin_r<R>(R(kz - 1) - E[2]);
    const long long c = (long long)pwrap(b0 + kx, a.nx) +
                        (long long)a.nx * (pwrap(b1 + ky, a.ny) + (long long)a.ny * pwrap(b2 + kz, a.nz));
    const int s = a.aux[c];
    if (s < 0 || s >= a.max_sites) return;
    const R *mFr = (const R *)a.mFr;
    R *Fp = (R *)a.sup_Fp;
    atomicAdd(Fp + 3 * s, mFr[3 * l] * w);
    atomicAdd(Fp + 3 * s + 1, mFr[3 * l + 1] * w);
    atomicAdd(Fp + 3 * s + 2, mFr[3 * l + 2] * w);
}

// u* += F/(2 rho); accumulate the IBM force; clear the pass buffer
template <typename R>
__global__ void ibm_update_kernel(IbmArgs a) {
    const long long ns = a.counts[0] < a.max_sites ? a.counts[0] : a.max_sites;
    R *ru = (R *)a.sup_ru, *sF = (R *)a.sup_F, *Fp = (R *)a.sup_Fp;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (long long)gridDim.x * blockDim.x) {
        const R ir = R(0.5) / ru[4 * s];
        for (int d = 0; d < 3; d++) {
            const R f = Fp[3 * s + d];
            ru[4 * s + 1 + d] += f * ir;
            sF[3 * s + d] = a.pass == 0 ? f : sF[3 * s + d] + f;
            Fp[3 * s + d] = R(0);
        }
    }
}

// Pipe wall: the ring of markers is the same in every z plane and sits at
// integer z, so the z weights of the 4-point kernel are the constants
// phi(0) = 1/2, phi(+-1) = 1/4 (phi(+-2) = 0). Each support cell gathers
// from a fixed list of ring markers of its (x, y) column in the planes
// z-1, z, z+1 -- no atomics, fixed order -- and applies the u* update.
struct PipeSpreadArgs {
    const int *site_cell;
    const int *xy_start, *xy_j;
    const void *xy_w;  // R
    const void *mFr;
    void *sup_ru, *sup_F;
    const long long *counts;
    long long max_sites;
    int nx, ny, nz, nc;
    int pass;
};

template <typename R>
__global__ void __launch_bounds__(256) ibm_spread_pipe_kernel(PipeSpreadArgs a) {
    const long long ns = a.counts[0] < a.max_sites ? a.counts[0] : a.max_sites;
    const R *mFr = (const R *)a.mFr;
    R *ru = (R *)a.sup_ru, *sF = (R *)a.sup_F;
    const int nxy = a.nx * a.ny;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (long long)gridDim.x * blockDim.x) {
        const int c = a.site_cell[s];
        const int z = c / nxy, xy = c - z * nxy;
        const int j0 = a.xy_start[xy], j1 = a.xy_start[xy + 1];
        R F0 = 0, F1 = 0, F2 = 0;
        for (int dz = -1; dz <= 1; dz++) {
            int zm = z - dz;
            zm = zm < 0 ? zm + a.nz : (zm >= a.nz ? zm - a.nz : zm);
            const R wz = R(dz == 0 ? 0.5 : 0.25);
            const R *Fp = mFr + 3 * (long long)zm * a.nc;
            for (int k = j0; k < j1; k++) {
                const R w = ((const R *)a.xy_w)[k] * wz;
                const int j = a.xy_j[k];
                F0 += Fp[3 * j] * w;
                F1 += Fp[3 * j + 1] * w;
                F2 += Fp[3 * j + 2] * w;
            }
        }
        const R ir = R(0.5) / ru[4 * s];
        ru[4 * s + 1] += F0 * ir;
        ru[4 * s + 2] += F1 * ir;
        ru[4 * s + 3] += F2 * ir;
        sF[3 * s] = a.pass == 0 ? F0 : sF[3 * s] + F0;
        sF[3 * s + 1] = a.pass == 0 ? F1 : sF[3 * s + 1] + F1;
        sF[3 * s + 2] = a.pass == 0 ? F2 : sF[3 * s + 2] + F2;
    }
}

// The same spreading on the z tiles (sites s = z sp + k, plane-invariant):
// the x-y sum Q(z', k) = sum over the ring markers of column k of
// w_xy F_l dV_l in plane z' is formed once per plane, then
// F(z, k) = Q(z+1, k)/4 + Q(z, k)/2 + Q(z-1, k)/4, followed by the u* update.
struct PipeSpreadTileArgs {
    const int *site_cell;  // the first sp sites (plane 0) give the (x, y) columns
    const int *xy_start, *xy_j;
    const void *xy_w;  // R
    const void *mFr;
    void *sup_ru, *sup_F;
    int nz, nc, sp, pass;
};

template <typename R>
__global__ void __launch_bounds__(256) ibm_spread_pipe_tiled_kernel(PipeSpreadTileArgs a) {
    __shared__ R Q[PIPE_ZH][32][3];
    const int kk = threadIdx.x & 31, k = blockIdx.x * 32 + kk;
    const int z0 = blockIdx.y * PIPE_ZT;
    const R *mFr = (const R *)a.mFr, *xw = (const R *)a.xy_w;
    int e0 = 0, e1 = 0;
    if (k < a.sp) {
        const int xy = a.site_cell[k];
        e0 = a.xy_start[xy];
        e1 = a.xy_start[xy + 1];
    }
    for (int pz = threadIdx.x >> 5; pz < PIPE_ZH; pz += blockDim.x >> 5) {
        const R *Fp = mFr + 3 * (size_t)zwrap(z0 - 1 + pz, a.nz) * a.nc;
        R q0 = R(0), q1 = R(0), q2 = R(0);
        for (int e = e0; e < e1; e++) {
            const R w = xw[e];
            const int j = a.xy_j[e];
            q0 += Fp[3 * j] * w;
            q1 += Fp[3 * j + 1] * w;
            q2 += Fp[3 * j + 2] * w;
        }
        Q[pz][kk][0] = q0;
        Q[pz][kk][1] = q1;
        Q[pz][kk][2] = q2;
    }
    __syncthreads();
    if (k >= a.sp) return;
    R *ru = (R *)a.sup_ru, *sF = (R *)a.sup_F;
    for (int pz = threadIdx.x >> 5; pz < PIPE_ZT; pz += blockDim.x >> 5) {
        const int z = z0 + pz;
        if (z >= a.nz) break;
        const size_t s = (size_t)z * a.sp + k;
        const R ir = R(0.5) / ru[4 * s];
        for (int d = 0; d < 3; d++) {
            const R F = R(0.25) * Q[pz + 2][kk][d] + R(0.5) * Q[pz + 1][kk][d] + R(0.25) * Q[pz][kk][d];
            ru[4 * s + 1 + d] += F * ir;
            sF[3 * s + d] = a.pass == 0 ? F : sF[3 * s + d] + F;
        }
    }
}

// Spheres: one block per particle accumulates the spread force of its
// markers in a shared-memory box around the particle, then adds the box to
// the support cells (global atomics only where boxes of nearby particles
// overlap).
struct ParticleSpreadArgs {
    const double *mX, *mdV;
    const void *mFr;
    const int *mB;
    const void *mE;
    const double *X, *R;
    const int *m_first, *aux;
    void *sup_Fp;
    long long max_sites;
    int nx, ny, nz;
    double rd;
};

template <typename R>
__global__ void __launch_bounds__(256) ibm_spread_particle_kernel(ParticleSpreadArgs a, int W) {
    extern __shared__ __align__(16) unsigned char box_raw[];
    R *box = (R *)box_raw;  // W^3 x 3
    const int p = blockIdx.x;
    const int nbox = W * W * W;
    for (int t = threadIdx.x; t < 3 * nbox; t += blockDim.x) box[t] = R(0);
    __syncthreads();
    const double RL = a.R[p] - a.rd;
    const int h = (int)ceil(RL) + 2;
    const double Xp0 = a.X[3 * p], Xp1 = a.X[3 * p + 1], Xp2 = a.X[3 * p + 2];
    const int o0 = (int)floor(Xp0) - h, o1 = (int)floor(Xp1) - h, o2 = (int)floor(Xp2) - h;
    const int l0 = a.m_first[p], l1 = a.m_first[p + 1];
    const R *mFr = (const R *)a.mFr;
    const int lane = threadIdx.x & 31;
    // 64 (marker, node) pairs per marker: a warp's 32 pairs share one marker
    // and every warp runs the same number of rounds (64 n is a multiple of 32)
    for (long long t = threadIdx.x; t < 64LL * (l1 - l0); t += blockDim.x) {
        const int l = l0 + (int)(t >> 6), k = (int)(t & 63);
        const int kx = k & 3, ky = (k >> 2) & 3, kz = k >> 4;
        const R *E = (const R *)a.mE + 3 * l;
        // the marker's 12 one-dimensional kernel values on lanes 0 .. 11
        R phi = R(0);
        if (lane < 12) phi = peskin_r<R>(R((lane & 3) - 1) - E[lane >> 2]);
        const R w = __shfl_sync(0xffffffffu, phi, kx) * __shfl_sync(0xffffffffu, phi, 4 + ky) *
                    __shfl_sync(0xffffffffu, phi, 8 + kz);
        // box-local node index; the marker base is wrapped, so unwrap the difference
        int i0 = a.mB[3 * l] + kx - o0, i1 = a.mB[3 * l + 1] + ky - o1, i2 = a.mB[3 * l + 2] + kz - o2;
        i0 = i0 < -a.nx / 2 ? i0 + a.nx : (i0 >= a.nx / 2 ? i0 - a.nx : i0);
        i1 = i1 < -a.ny / 2 ? i1 + a.ny : (i1 >= a.ny / 2 ? i1 - a.ny : i1);
        i2 = i2 < -a.nz / 2 ? i2 + a.nz : (i2 >= a.nz / 2 ? i2 - a.nz : i2);
        if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= W || i1 >= W || i2 >= W) continue;
        const int bi = i0 + W * (i1 + W * i2);
        atomicAdd(&box[3 * bi], mFr[3 * l] * w);
        atomicAdd(&box[3 * bi + 1], mFr[3 * l + 1] * w);
        atomicAdd(&box[3 * bi + 2], mFr[3 * l + 2] * w);
    }
    __syncthreads();
    R *Fp = (R *)a.sup_Fp;
    for (int bi = threadIdx.x; bi < nbox; bi += blockDim.x) {
        const R f0 = box[3 * bi], f1 = box[3 * bi + 1], f2 = box[3 * bi + 2];
        if (f0 == R(0) && f1 == R(0) && f2 == R(0)) continue;
        const int i0 = bi % W, i1 = (bi / W) % W, i2 = bi / (W * W);
        const long long c = (long long)pwrap(o0 + i0, a.nx) +
                            (long long)a.nx * (pwrap(o1 + i1, a.ny) + (long long)a.ny * pwrap(o2 + i2, a.nz));
        const int s = a.aux[c];
        if (s < 0 || s >= a.max_sites) continue;
        atomicAdd(Fp + 3 * s, f0);
        atomicAdd(Fp + 3 * s + 1, f1);
        atomicAdd(Fp + 3 * s + 2, f2);
    }
}

template <typename R>
static cudaError_t ibm_passes_t(Ctx &c) {
    IbmArgs a{c.mX, c.mdV, c.mpid, c.mFacc, c.mUd, c.mFaccR, c.mFr, c.mB, c.mE, c.aux, c.sup_ru, c.sup_F, c.sup_Fp,
              c.X, c.U, c.W, c.nm, c.d_counts, c.max_sites, c.nx, c.ny, c.nz, 0, 0};
    long long ns = c.nsites_hint > 0 ? c.nsites_hint : c.max_sites;
    if (ns > c.max_sites) ns = c.max_sites;
    long long ub = (ns + 255) / 256;
    if (ub < 1) ub = 1;
    if (ub > 152 * 32) ub = 152 * 32;
    const bool pipe_gather = c.has_pipe && c.nm > 0 && c.pipe_nc > 0;
    // sphere boxes in shared memory when they fit
    const double RLmax = c.max_radius - c.rd;
    const int W = 2 * (int)ceil(RLmax) + 6;
    const size_t smem = 3 * sizeof(R) * (size_t)W * W * W;
    const bool box_spread = !c.has_pipe && c.np > 0 && smem <= 200 * 1024;
    if (box_spread) {
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(ibm_spread_particle_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
            attr_set = true;
        }
    }
    for (int pass = 0; pass < 3; pass++) {
        a.pass = pass;
        a.last = pass == 2;
        const bool pipe_tiles = c.nm > 0 && pipe_gather && c.pipe_sp > 0 && c.nm == (long long)c.nz * c.pipe_nc &&
                                c.nz <= 65535LL * PIPE_ZT;
        const dim3 zt_grid((unsigned)((c.nz + PIPE_ZT - 1) / PIPE_ZT));
        if (pipe_tiles) {
            PipeInterpArgs pi{c.pipe_it_k, c.pipe_it_w, c.sup_ru, c.mFacc, c.mFaccR, c.mFr,
                              c.pipe_nc, c.nz, c.pipe_sp, pass, pass == 2, c.pipe_dV};
            count_launch(c, G_IBM);
            ibm_interp_pipe_kernel<R><<<dim3((unsigned)((c.pipe_nc + 31) / 32), zt_grid.x), 256, 0, c.stream>>>(pi);
        } else if (c.nm > 0) {
            count_launch(c, G_IBM);
            ibm_interp_warp_kernel<R><<<(unsigned)((c.nm * 32 + 255) / 256), 256, 0, c.stream>>>(a);
        }
        if (pipe_tiles) {
            PipeSpreadTileArgs ps{c.site_cell, c.pipe_xy_start, c.pipe_xy_j, c.pipe_xy_w, c.mFr, c.sup_ru,
                                  c.sup_F, c.nz, c.pipe_nc, c.pipe_sp, pass};
            count_launch(c, G_IBM);
            ibm_spread_pipe_tiled_kernel<R><<<dim3((unsigned)((c.pipe_sp + 31) / 32), zt_grid.x), 256, 0, c.stream>>>(ps);
            continue;
        }
        if (pipe_gather) {
            PipeSpreadArgs ps{c.site_cell, c.pipe_xy_start, c.pipe_xy_j, c.pipe_xy_w, c.mFr, c.sup_ru,
                              c.sup_F, c.d_counts, c.max_sites, c.nx, c.ny, c.nz, c.pipe_nc, pass};
            count_launch(c, G_IBM);
            ibm_spread_pipe_kernel<R><<<(unsigned)ub, 256, 0, c.stream>>>(ps);
            continue;
        }
        if (c.nm > 0) {
            count_launch(c, G_IBM);
            if (box_spread) {
                ParticleSpreadArgs pa{c.mX, c.mdV, c.mFr, c.mB, c.mE, c.X, c.R, c.m_first, c.aux, c.sup_Fp,
                                      c.max_sites, c.nx, c.ny, c.nz, c.rd};
                ibm_spread_particle_kernel<R><<<c.np, 256, smem, c.stream>>>(pa, W);
            } else {
                ibm_spread_kernel<R><<<(unsigned)((c.nm + 3) / 4), 256, 0, c.stream>>>(a);
            }
        }
        count_launch(c, G_IBM);
        ibm_update_kernel<R><<<(unsigned)ub, 256, 0, c.stream>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_ibm_passes(Ctx &c) {
    return c.storage == LBM_F64 ? ibm_passes_t<double>(c) : ibm_passes_t<float>(c);
}

// particle force/torque: -sum_l F_l dV_l (+ moment) plus the change of the
// inner-fluid momentum sum alpha u (Kempe et al. 2012)
struct SumArgs {
    const double *mX, *mdV, *mFacc;
    const int *m_first;
    const double *X;
    double *Fh, *Th, *Iu, *Ir;
    const double *Iu_new, *Ir_new;
    int nx, ny, nz;
};

__global__ void __launch_bounds__(PB) ibm_sum_kernel(SumArgs a) {
    __shared__ double sh[6 * PB];
    const int p = blockIdx.x;
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int l = a.m_first[p] + threadIdx.x; l < a.m_first[p + 1]; l += PB) {
        const double F0 = -a.mFacc[3 * l] * a.mdV[l], F1 = -a.mFacc[3 * l + 1] * a.mdV[l],
                     F2 = -a.mFacc[3 * l + 2] * a.mdV[l];
        const double r0 = pmimg(a.mX[3 * l] - a.X[3 * p], a.nx), r1 = pmimg(a.mX[3 * l + 1] - a.X[3 * p + 1], a.ny),
                     r2 = pmimg(a.mX[3 * l + 2] - a.X[3 * p + 2], a.nz);
        v[0] += F0;
        v[1] += F1;
        v[2] += F2;
        v[3] += r1 * F2 - r2 * F1;
        v[4] += r2 * F0 - r0 * F2;
        v[5] += r0 * F1 - r1 * F0;
    }
    block_sum<6>(v, sh);
    if (threadIdx.x == 0)
        for (int d = 0; d < 3; d++) {
            a.Fh[3 * p + d] = v[d] + (a.Iu_new[3 * p + d] - a.Iu[3 * p + d]);
            a.Th[3 * p + d] = v[3 + d] + (a.Ir_new[3 * p + d] - a.Ir[3 * p + d]);
            a.Iu[3 * p + d] = a.Iu_new[3 * p + d];
            a.Ir[3 * p + d] = a.Ir_new[3 * p + d];
        }
}

cudaError_t launch_ibm_particle_sums(Ctx &c, bool init_only) {
    if (c.np == 0) return cudaSuccess;
    if (init_only) return launch_volume(c, 1, c.Iu, c.Ir);
    // scratch for the new integrals: the contact-force buffer (2 x 3 doubles
    // per particle) is free until the contact kernel runs later in the step
    double *Iu_new = c.Fc, *Ir_new = c.Fc + 3 * c.max_np;
    cudaError_t e = launch_volume(c, 2, Iu_new, Ir_new);
    if (e != cudaSuccess) return e;
    SumArgs a{c.mX, c.mdV, c.mFacc, c.m_first, c.X, c.Fh, c.Th, c.Iu, c.Ir, Iu_new, Ir_new, c.nx, c.ny, c.nz};
    count_launch(c, G_PART);
    ibm_sum_kernel<<<c.np, PB, 0, c.stream>>>(a);
    return cudaGetLastError();
}

// one-time rigid-body overwrite inside the particles at insertion (Sec. 3.1)
template <int S>
__global__ void rigid_overwrite_kernel(void *A, const uint8_t *flags, const int *owner, const double *X,
                                       const double *U, const double *W, const double *R, int nx, int ny, int nz,
                                       long long N, double F0, double F1, double F2) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R Rt;
    const int p = blockIdx.x;
    const int r = (int)ceil(R[p]) + 1;
    const int bx = (int)floor(X[3 * p]) - r, by = (int)floor(X[3 * p + 1]) - r, bz = (int)floor(X[3 * p + 2]) - r;
    const int w = 2 * r + 2;
    const FastDiv fw((unsigned)w);
    for (int t = threadIdx.x; t < w * w * w; t += blockDim.x) {
        int ix, iy, iz;
        box_coords(t, fw, w, ix, iy, iz);
        const int x = pwrap(bx + ix, nx), y = pwrap(by + iy, ny), z = pwrap(bz + iz, nz);
        const long long c = (long long)x + (long long)nx * (y + (long long)ny * z);
        if (!(flags[c] & FL_SOLID) || owner[c] != p) continue;
        double rho, u[3];
        cell_velocity<S>(A, (size_t)N, c, 0.0, 0.0, 0.0, rho, u);  // solid cells feel no body force
        const double rx = pmimg(x - X[3 * p], nx), ry = pmimg(y - X[3 * p + 1], ny), rz = pmimg(z - X[3 * p + 2], nz);
        const double uw[3] = {U[3 * p] + (W[3 * p + 1] * rz - W[3 * p + 2] * ry),
                              U[3 * p + 1] + (W[3 * p + 2] * rx - W[3 * p] * rz),
                              U[3 * p + 2] + (W[3 * p] * ry - W[3 * p + 1] * rx)};
        const double u2 = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
        for (int i = 0; i < 19; i++) {
            const double cu = cx(i) * uw[0] + cy(i) * uw[1] + cz(i) * uw[2];
            const double feq = wgt(i) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
            Store<S>::st((T *)A + (size_t)i * N + c, Rt(feq - wgt(i)));
        }
    }
    (void)F0; (void)F1; (void)F2;
}

cudaError_t launch_ibm_rigid_overwrite(Ctx &c) {
    if (c.np == 0) return cudaSuccess;
    count_launch(c, G_OTHER);
    switch (c.storage) {
#define RO(S) rigid_overwrite_kernel<S><<<c.np, 256, 0, c.stream>>>(c.fA, c.flags, c.owner, c.X, c.U, c.W, c.R, \
                                                                      c.nx, c.ny, c.nz, c.N, 0, 0, 0)
    case LBM_F64: RO(LBM_F64); break;
    case LBM_F32: RO(LBM_F32); break;
    case LBM_F16S: RO(LBM_F16S); break;
    default: RO(LBM_BF16S); break;
#undef RO
    }
    return cudaGetLastError();
}

}  // namespace lbmgb
