// Diagnostics (Sec. 3.2, Sec. 2.2): macroscopic fields of the current state,
// rigid-body masking of particle regions, kinetic energy, dissipation
// 2 nu s_ij s_ij from second-order central differences, radial profiles
// around particles and the pipe bulk velocity. Sums are FP64 block partials
// reduced on the host in block order (deterministic).
#include "lbm_internal.cuh"

#include <vector>
#include <cstring>

namespace lbmgb {

__device__ __forceinline__ double dmimg(double d, int n) {
    if (d > 0.5 * n) d = __dsub_rn(d, (double)n);
    else if (d < -0.5 * n) d = __dadd_rn(d, (double)n);
    return d;
}
__device__ __forceinline__ int dwrap(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

// rho and u of the post-collision state: sum f c = rho u + F/2 after a Guo
// collision with total force F (body force on fluid cells + IBM force).
// u32, if not null, receives an FP32 copy of u, one 16-byte record (ux, uy,
// uz, 0) per cell (the closure's gather input).
template <int S>
__global__ void macro_kernel(const void *A, const uint8_t *flags, const int *aux, const void *sup_Fv, double *rho_o,
                             double *u_o, float *u32, long long N, double F0, double F1, double F2, int ibb, int ibm,
                             long long max_sites) {
    typedef typename Store<S>::T T;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const uint8_t fl = flags[c];
    if (ibb && (fl & FL_SOLID)) {
        rho_o[c] = 0.0;
        u_o[c] = u_o[N + c] = u_o[2 * N + c] = 0.0;
        if (u32) reinterpret_cast<float4 *>(u32)[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    // arithmetic type of the storage (FP32 for the 32- and 16-bit layouts)
    typedef typename Store<S>::R R;
    const T *P = (const T *)A;
    R r = R(0), j0 = R(0), j1 = R(0), j2 = R(0);
#pragma unroll
    for (int i = 0; i < 19; i++) {
        const R g = Store<S>::ld(P + (size_t)i * N + c);
        r += g;
        j0 += g * R(cx(i));
        j1 += g * R(cy(i));
        j2 += g * R(cz(i));
    }
    const bool fluid = !(fl & FL_SOLID);
    R Fx = fluid ? R(F0) : R(0), Fy = fluid ? R(F1) : R(0), Fz = fluid ? R(F2) : R(0);
    if (ibm && (fl & FL_SUP) && aux[c] >= 0 && aux[c] < max_sites) {
        const R *sup_F = (const R *)sup_Fv;
        const int s = aux[c];
        Fx += sup_F[3 * s];
        Fy += sup_F[3 * s + 1];
        Fz += sup_F[3 * s + 2];
    }
    const R rho = R(1) + r;
    const R ir = R(1) / rho;
    rho_o[c] = double(rho);
    const R ux = (j0 - R(0.5) * Fx) * ir, uy = (j1 - R(0.5) * Fy) * ir, uz = (j2 - R(0.5) * Fz) * ir;
    u_o[c] = double(ux);
    u_o[N + c] = double(uy);
    u_o[2 * N + c] = double(uz);
    if (u32) {
        reinterpret_cast<float4 *>(u32)[c] = make_float4(float(ux), float(uy), float(uz), 0.f);
    }
}

cudaError_t launch_macro(Ctx &c, int /*mask_mode*/, float *u32) {
    if (c.q == 27) return launch_q27_macro(c);
    count_launch(c, G_STATS);
    const unsigned nb = (unsigned)((c.N + 255) / 256);
    const int ibb = c.armed_bc == LBM_BC_IBB;
    const int ibm = c.armed_bc == LBM_BC_IBM_U || c.armed_bc == LBM_BC_IBM_B;
    switch (c.storage) {
#define MK(S) macro_kernel<S><<<nb, 256, 0, c.stream>>>(c.fA, c.flags, c.aux, c.sup_F, c.rho_f, c.u_f, u32, c.N, c.F[0], \
                                                           c.F[1], c.F[2], ibb, ibm, c.max_sites)
    case LBM_F64: MK(LBM_F64); break;
    case LBM_F32: MK(LBM_F32); break;
    case LBM_F16S: MK(LBM_F16S); break;
    default: MK(LBM_BF16S); break;
#undef MK
    }
    return cudaGetLastError();
}

constexpr int SB = 256;     // threads per statistics block
constexpr int SNB = 1024;   // statistics blocks (fixed: the reduction order does not depend on the grid)
constexpr int NP = 16;      // partial sums per block

template <int NV>
__device__ void sblock_sum(double v[NV], double *sh) {
    for (int k = 0; k < NV; k++) sh[k * SB + threadIdx.x] = v[k];
    __syncthreads();
    for (int s = SB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < NV; k++) sh[k * SB + threadIdx.x] += sh[k * SB + threadIdx.x + s];
        __syncthreads();
    }
    for (int k = 0; k < NV; k++) v[k] = sh[k * SB];
}

// partials: mass, momentum (3) over fluid-carrying cells
__global__ void __launch_bounds__(SB) mass_kernel(const double *rho, const double *u, const uint8_t *flags, long long N,
                                                  int ibb, double *part) {
    __shared__ double sh[4 * SB];
    double v[4] = {0, 0, 0, 0};
    for (long long c = (long long)blockIdx.x * SB + threadIdx.x; c < N; c += (long long)SNB * SB) {
        if (ibb && (flags[c] & FL_SOLID)) continue;
        v[0] += rho[c];
        v[1] += rho[c] * u[c];
        v[2] += rho[c] * u[N + c];
        v[3] += rho[c] * u[2 * N + c];
    }
    sblock_sum<4>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; k++) part[blockIdx.x * NP + k] = v[k];
}

// replace the velocity of solid cells by the rigid-body velocity
__global__ void mask_kernel(double *u, const uint8_t *flags, const int *owner, const double *X, const double *U,
                            const double *W, int nx, int ny, int nz, long long N) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    if (!(flags[c] & FL_SOLID)) return;
    const int p = owner[c];
    double uw[3] = {0, 0, 0};
    if (p != NO_OWNER) {
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        const double r0 = dmimg(x - X[3 * p], nx), r1 = dmimg(y - X[3 * p + 1], ny), r2 = dmimg(z - X[3 * p + 2], nz);
        uw[0] = U[3 * p] + (W[3 * p + 1] * r2 - W[3 * p + 2] * r1);
        uw[1] = U[3 * p + 1] + (W[3 * p + 2] * r0 - W[3 * p] * r2);
        uw[2] = U[3 * p + 2] + (W[3 * p] * r1 - W[3 * p + 1] * r0);
    }
    u[c] = uw[0];
    u[N + c] = uw[1];
    u[2 * N + c] = uw[2];
}

__device__ __forceinline__ double cell_eps(const double *u, int x, int y, int z, int nx, int ny, int nz, long long N,
                                           double nu) {
    const long long xp = dwrap(x + 1, nx) + (long long)nx * (y + (long long)ny * z);
    const long long xm = dwrap(x - 1, nx) + (long long)nx * (y + (long long)ny * z);
    const long long yp = x + (long long)nx * (dwrap(y + 1, ny) + (long long)ny * z);
    const long long ym = x + (long long)nx * (dwrap(y - 1, ny) + (long long)ny * z);
    const long long zp = x + (long long)nx * (y + (long long)ny * dwrap(z + 1, nz));
    const long long zm = x + (long long)nx * (y + (long long)ny * dwrap(z - 1, nz));
    double g[3][3];
    for (int a = 0; a < 3; a++) {
        const double *ua = u + a * N;
        g[a][0] = 0.5 * (ua[xp] - ua[xm]);
        g[a][1] = 0.5 * (ua[yp] - ua[ym]);
        g[a][2] = 0.5 * (ua[zp] - ua[zm]);
    }
    double ss = 0.0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            const double s = 0.5 * (g[a][b] + g[b][a]);
            ss += s * s;
        }
    return 2.0 * nu * ss;
}

// partials: ke, eps over all cells; ke, eps, count over fluid cells; pipe bulk
__global__ void __launch_bounds__(SB) energy_kernel(const double *u, const uint8_t *flags, int nx, int ny, int nz,
                                                    long long N, double nu, int pipe, double *part, const float *eps_o) {
    __shared__ double sh[7 * SB];
    double v[7] = {0, 0, 0, 0, 0, 0, 0};
    for (long long c = (long long)blockIdx.x * SB + threadIdx.x; c < N; c += (long long)SNB * SB) {
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        const double e = (eps_o && eps_o[c] >= 0.f) ? (double)eps_o[c] : cell_eps(u, x, y, z, nx, ny, nz, N, nu);
        const double k = 0.5 * (u[c] * u[c] + u[N + c] * u[N + c] + u[2 * N + c] * u[2 * N + c]);
        v[0] += k;
        v[1] += e;
        if (!(flags[c] & FL_SOLID)) {
            v[2] += k;
            v[3] += e;
            v[4] += 1.0;
            if (pipe) {
                v[5] += u[2 * N + c];
                v[6] += 1.0;
            }
        }
    }
    sblock_sum<7>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 7; k++) part[blockIdx.x * NP + 4 + k] = v[k];
}

// Nearest particle surface of the fluid cells with 0 < s <= reach, s = r -
// R_p (reach: the farthest distance a caller needs, the closure's 2 or the
// last radial bin), in one pass: the 64-bit key of a cell holds the bits
// of s (positive, so ordered as integers) with its low NEAR_PID_BITS bits
// replaced by the particle id, and atomicMin keeps the nearest. Particles
// whose s agree in the upper 44 bits (2^-44 relative) count as tied, and
// the lower id wins. Every particle that could be the nearest of such a
// cell has it in its box, so the minimum is over all of them; cells
// farther out keep the empty key. s is formed in FP32 from the split centre
// (integer part exact, FP32 fraction: error about 1e-6 lu), and in exact
// FP64 where it lies within 1e-4 of 0 or of reach, so every cell's
// membership (0 < s <= reach) is that of the FP64 distance; s itself, the
// order of two particles within 1e-6 of each other and the distance
// feature carry the FP32 error. The closure's own threshold (2) is decided
// the same way when the bins reach farther.
constexpr int NEAR_PID_BITS = 20;
constexpr unsigned long long NEAR_PID_MASK = (1ULL << NEAR_PID_BITS) - 1;
constexpr unsigned long long NEAR_EMPTY = ~0ULL;
__device__ __forceinline__ int near_pid_of(unsigned long long k) { return (int)(k & NEAR_PID_MASK); }
__device__ __forceinline__ double near_s_of(unsigned long long k) {
    return __longlong_as_double((long long)(k & ~NEAR_PID_MASK));
}

__global__ void near_key_kernel(unsigned long long *key, const uint8_t *flags, const double *X, const double *R,
                                int nx, int ny, int nz, double reach) {
    const int p = blockIdx.x;
    const double Rp = R[p];
    const int r = (int)ceil(Rp + reach) + 2;
    const double Xd = X[3 * p], Yd = X[3 * p + 1], Zd = X[3 * p + 2];
    const int bx = (int)floor(Xd) - r, by = (int)floor(Yd) - r, bz = (int)floor(Zd) - r;
    const int w = 2 * r + 2;
    const FastDiv fw((unsigned)w);
    // the centre relative to the box corner: integer part exact, fraction in FP32
    const float fX0 = (float)(Xd - bx), fX1 = (float)(Yd - by), fX2 = (float)(Zd - bz);
    const float Rf = (float)Rp, reachf = (float)reach;
    const float lo = fmaxf(Rf - 2e-3f, 0.f), hi = Rf + reachf + 2e-3f, lo2 = lo * lo, hi2 = hi * hi;
    for (int t = threadIdx.x; t < w * w * w; t += blockDim.x) {
        int ix, iy, iz;
        box_coords(t, fw, w, ix, iy, iz);
        const float ex = ix - fX0, ey = iy - fX1, ez = iz - fX2, e2 = ex * ex + ey * ey + ez * ez;
        if (e2 > hi2 || e2 < lo2) continue;
        const int x = dwrap(bx + ix, nx), y = dwrap(by + iy, ny),
                  z = dwrap(bz + iz, nz);
        const long long c = (long long)x + (long long)nx * (y + (long long)ny * z);
        if (flags[c] & FL_SOLID) continue;
        const float s32 = sqrtf(e2) - Rf;
        double sd;
        if (s32 < 1e-4f || fabsf(s32 - reachf) < 1e-4f || fabsf(s32 - 2.0f) < 1e-4f) {  // 2: the closure's band
            const double dx = dmimg(__dsub_rn((double)x, Xd), nx);
            const double dy = dmimg(__dsub_rn((double)y, Yd), ny);
            const double dz = dmimg(__dsub_rn((double)z, Zd), nz);
            const double rr = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
            sd = __dsub_rn(rr, Rp);
        } else {
            sd = (double)s32;
        }
        if (sd <= 0.0 || sd > reach) continue;
        const unsigned long long k = ((unsigned long long)__double_as_longlong(sd) & ~NEAR_PID_MASK) | (unsigned)p;
        atomicMin(key + c, k);
    }
}

// one counter increment per warp for the lanes with `take`; returns this lane's slot
__device__ __forceinline__ long long warp_slot(bool take, long long *count) {
    const unsigned m = __ballot_sync(__activemask(), take);
    if (!take) return -1;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd((unsigned long long *)count, (unsigned long long)__popc(m));
    base = __shfl_sync(m, base, leader);
    return (long long)base + __popc(m & ((1u << lane) - 1u));
}

constexpr int NBIN = LBM_NBINS;

__global__ void __launch_bounds__(SB) bins_kernel(const double *u, const uint8_t *flags, const unsigned long long *near_key,
                                                  const double *X, const double *R, int nx, int ny, int nz,
                                                  long long N, double nu, double *bpart, const float *eps_o) {
    __shared__ double sk[NBIN], se[NBIN], sc[NBIN];
    for (int b = threadIdx.x; b < NBIN; b += SB) sk[b] = se[b] = sc[b] = 0.0;
    __syncthreads();
    // accumulate per block in shared memory with FP64 atomics, then write
    // (per-bin sums of a few values each; order effects stay at round-off)
    for (long long c = (long long)blockIdx.x * SB + threadIdx.x; c < N; c += (long long)SNB * SB) {
        if (flags[c] & FL_SOLID) continue;
        const unsigned long long key = near_key[c];
        if (key == NEAR_EMPTY) continue;
        const int p = near_pid_of(key);
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        const double dx = dmimg(__dsub_rn((double)x, X[3 * p]), nx);
        const double dy = dmimg(__dsub_rn((double)y, X[3 * p + 1]), ny);
        const double dz = dmimg(__dsub_rn((double)z, X[3 * p + 2]), nz);
        const double rr = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
        const double ratio = __ddiv_rn(rr, R[p]);
        const int b = (int)floor(__ddiv_rn(__dsub_rn(ratio, 1.0), 0.05));
        if (b < 0 || b >= NBIN) continue;
        const double k = 0.5 * (u[c] * u[c] + u[N + c] * u[N + c] + u[2 * N + c] * u[2 * N + c]);
        atomicAdd(&sk[b], k);
        atomicAdd(&se[b], (eps_o && eps_o[c] >= 0.f) ? (double)eps_o[c] : cell_eps(u, x, y, z, nx, ny, nz, N, nu));
        atomicAdd(&sc[b], 1.0);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < NBIN; b += SB) {
        bpart[blockIdx.x * 3 * NBIN + b] = sk[b];
        bpart[blockIdx.x * 3 * NBIN + NBIN + b] = se[b];
        bpart[blockIdx.x * 3 * NBIN + 2 * NBIN + b] = sc[b];
    }
}

__global__ void fill_u64(unsigned long long *p, unsigned long long v, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// ------------------------------------------------------ learned closure --
// Near-surface fluid nodes (distance to the nearest particle surface in
// (0, 2]) and their 85 features: the 27-point stencil of u - u_rb (u_rb the
// rigid-body velocity of the nearest particle), scaled by 1/u_scale, the
// signed distance / h, and u - u_rb at the node.
__global__ void closure_sample_kernel(const double *u, const uint8_t *flags, const unsigned long long *near_key,
                                      const double *X, const double *U, const double *W, int nx, int ny, int nz,
                                      long long N, double inv_us, float *feat, int *cells, long long *count,
                                      long long cap) {
    // whole warps per round (the slot counter is taken once per warp)
    const long long span = (long long)gridDim.x * blockDim.x;
    for (long long c0 = (long long)blockIdx.x * blockDim.x; c0 < N; c0 += span) {
        const long long c = c0 + threadIdx.x;
        const unsigned long long key = c < N && !(flags[c] & FL_SOLID) ? near_key[c] : NEAR_EMPTY;
        const double d = near_s_of(key);  // r - R_p of the nearest particle
        const bool take = key != NEAR_EMPTY && d > 0.0 && d <= 2.0;
        const long long k = warp_slot(take, count);
        if (!take || k >= cap) continue;
        const int p = near_pid_of(key);
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        const double rx = dmimg(x - X[3 * p], nx), ry = dmimg(y - X[3 * p + 1], ny), rz = dmimg(z - X[3 * p + 2], nz);
        cells[k] = (int)c;
        float *f = feat + k * 85;
        int j = 0;
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    const long long q = (long long)dwrap(x + dx, nx) + (long long)nx * (dwrap(y + dy, ny) + (long long)ny * dwrap(z + dz, nz));
                    const double sx = rx + dx, sy = ry + dy, sz = rz + dz;
                    const double ub0 = U[3 * p] + (W[3 * p + 1] * sz - W[3 * p + 2] * sy);
                    const double ub1 = U[3 * p + 1] + (W[3 * p + 2] * sx - W[3 * p] * sz);
                    const double ub2 = U[3 * p + 2] + (W[3 * p] * sy - W[3 * p + 1] * sx);
                    f[j++] = (float)((u[q] - ub0) * inv_us);
                    f[j++] = (float)((u[N + q] - ub1) * inv_us);
                    f[j++] = (float)((u[2 * N + q] - ub2) * inv_us);
                }
        f[81] = (float)d;
        f[82] = f[3 * 13];
        f[83] = f[3 * 13 + 1];
        f[84] = f[3 * 13 + 2];
    }
}

// 9 velocity gradients du_a/dx_b (central differences) at listed cells,
// scaled by g_scale; NaN where the cell is solid in this state
__global__ void closure_target_kernel(const double *u, const uint8_t *flags, const int *cells, long long n, int nx,
                                      int ny, int nz, long long N, double gs, float *T) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const long long c = cells[k];
    float *t = T + k * 9;
    if (flags[c] & FL_SOLID) {
        for (int e = 0; e < 9; e++) t[e] = __int_as_float(0x7fc00000);
        return;
    }
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
    const long long nb[3][2] = {{dwrap(x + 1, nx) + (long long)nx * (y + (long long)ny * z), dwrap(x - 1, nx) + (long long)nx * (y + (long long)ny * z)},
                                {x + (long long)nx * (dwrap(y + 1, ny) + (long long)ny * z), x + (long long)nx * (dwrap(y - 1, ny) + (long long)ny * z)},
                                {x + (long long)nx * (y + (long long)ny * dwrap(z + 1, nz)), x + (long long)nx * (y + (long long)ny * dwrap(z - 1, nz))}};
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) t[3 * a + b] = (float)(0.5 * (u[a * N + nb[b][0]] - u[a * N + nb[b][1]]) * gs);
}

// the near-surface fluid nodes of the fused closure dissipation: cell and
// nearest particle (distance to the surface in (0, 2]); order not fixed
// One slot range per block and 256 consecutive cells, filled in cell
// order, so that neighbouring samples of the list are mostly neighbouring
// cells (their stencils share lines in the inference kernel's gather).
__global__ void __launch_bounds__(256) closure_list_kernel(const uint8_t *flags, const unsigned long long *near_key,
                                                           long long N, int *cells, int *pids, long long *count,
                                                           long long cap) {
    __shared__ unsigned wcnt[8];
    __shared__ unsigned long long base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long span = (long long)gridDim.x * blockDim.x;
    for (long long c0 = (long long)blockIdx.x * blockDim.x; c0 < N; c0 += span) {
        const long long c = c0 + threadIdx.x;
        const unsigned long long key = c < N && !(flags[c] & FL_SOLID) ? near_key[c] : NEAR_EMPTY;
        const double d = near_s_of(key);  // r - R_p of the nearest particle
        const bool take = key != NEAR_EMPTY && d > 0.0 && d <= 2.0;
        const unsigned m = __ballot_sync(0xffffffffu, take);
        if (lane == 0) wcnt[warp] = (unsigned)__popc(m);
        __syncthreads();
        unsigned before = 0, total = 0;
        for (int w = 0; w < 8; w++) {
            before += w < warp ? wcnt[w] : 0u;
            total += wcnt[w];
        }
        if (threadIdx.x == 0) base = total ? atomicAdd((unsigned long long *)count, (unsigned long long)total) : 0ull;
        __syncthreads();
        const long long k = (long long)base + before + __popc(m & ((1u << lane) - 1u));
        if (take && k < cap) {
            cells[k] = (int)c;
            pids[k] = near_pid_of(key);
        }
        __syncthreads();  // wcnt and base are rewritten next round
    }
}

// dissipation 2 nu s_ij s_ij from predicted gradients (scaled by g_scale)
__global__ void closure_eps_kernel(const float *Y, const int *cells, long long n, double inv_gs, double nu,
                                   float *eps_o) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double g[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) g[a][b] = (double)Y[k * 9 + 3 * a + b] * inv_gs;
    double ss = 0.0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            const double sab = 0.5 * (g[a][b] + g[b][a]);
            ss += sab * sab;
        }
    eps_o[cells[k]] = (float)(2.0 * nu * ss);
}

__global__ void fill_f32(float *p, float v, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}


// nearest particle and distance to its surface of the fluid cells within
// `reach` of a surface (key and pid; others NO_OWNER)
static void near_surface(Ctx &c, const unsigned nb, double reach) {
    count_launch(c, G_STATS, 2);
    fill_u64<<<nb, 256, 0, c.stream>>>(c.near_key, NEAR_EMPTY, c.N);
    near_key_kernel<<<c.np, 256, 0, c.stream>>>(c.near_key, c.flags, c.X, c.R, c.nx, c.ny, c.nz, reach);
}

cudaError_t closure_samples(Ctx &c, double u_scale, float *X, int *cells, long long cap, long long *n_out) {
    cudaError_t e;
    if ((e = launch_macro(c, 0)) != cudaSuccess) return e;
    const unsigned nb = (unsigned)((c.N + 255) / 256);
    near_surface(c, nb, 2.0);
    count_launch(c, G_STATS);
    if ((e = cudaMemsetAsync(c.d_counts + 3, 0, sizeof(long long), c.stream)) != cudaSuccess) return e;
    closure_sample_kernel<<<nb, 256, 0, c.stream>>>(c.u_f, c.flags, c.near_key, c.X, c.U, c.W, c.nx, c.ny, c.nz,
                                                    c.N, 1.0 / u_scale, X, cells, c.d_counts + 3, cap);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    long long n = 0;
    if ((e = cudaMemcpyAsync(&n, c.d_counts + 3, sizeof(long long), cudaMemcpyDeviceToHost, c.stream)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(c.stream)) != cudaSuccess) return e;
    *n_out = n;
    return cudaSuccess;
}

cudaError_t closure_targets(Ctx &c, const int *cells, long long n, double g_scale, float *T) {
    cudaError_t e;
    if ((e = launch_macro(c, 0)) != cudaSuccess) return e;
    const unsigned nb = (unsigned)((c.N + 255) / 256);
    count_launch(c, G_STATS, 2);
    mask_kernel<<<nb, 256, 0, c.stream>>>(c.u_f, c.flags, c.owner, c.X, c.U, c.W, c.nx, c.ny, c.nz, c.N);
    if (n > 0)
        closure_target_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(c.u_f, c.flags, cells, n, c.nx, c.ny,
                                                                              c.nz, c.N, g_scale, T);
    return cudaGetLastError();
}

// ------------------------------------------------ pipe radial profiles ----
// Per radial bin b = floor(r nbins / R) of the cells inside the pipe, the
// sums of 1, u_r, u_theta, u_z, their products, rho and 2 nu s_ij s_ij
// (statistics velocity, central differences); FP64 shared sums per block,
// the blocks added on the host in a fixed order. r and the bin use
// explicitly rounded operations so that a cell on a bin edge falls in the
// same bin everywhere.
constexpr int PROF_NQ = LBM_PROF_NQ;
constexpr int PROF_BLOCKS = 304;

__global__ void __launch_bounds__(SB) pipe_profile_kernel(const double *u, const double *rho, const uint8_t *flags,
                                                         int nx, int ny, int nz, long long N, double cx, double cy,
                                                         double R, int nbins, double nu, double *part) {
    extern __shared__ double sp[];  // nbins x PROF_NQ
    for (int i = threadIdx.x; i < nbins * PROF_NQ; i += blockDim.x) sp[i] = 0.0;
    __syncthreads();
    for (long long c = (long long)blockIdx.x * SB + threadIdx.x; c < N; c += (long long)gridDim.x * SB) {
        if (flags[c] & FL_SOLID) continue;
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        const double dx = __dsub_rn((double)x, cx), dy = __dsub_rn((double)y, cy);
        const double r = sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
        const int b = (int)floor(__ddiv_rn(__dmul_rn(r, (double)nbins), R));
        if (b < 0 || b >= nbins) continue;
        const double ux = u[c], uy = u[N + c], uz = u[2 * N + c];
        const double ur = r > 0.0 ? (ux * dx + uy * dy) / r : ux;
        const double ut = r > 0.0 ? (uy * dx - ux * dy) / r : uy;
        const double q[PROF_NQ] = {1.0,     ur,      ut,      uz,      ur * ur, ut * ut,
                                   uz * uz, ur * uz, ur * ut, ut * uz, rho[c],  cell_eps(u, x, y, z, nx, ny, nz, N, nu)};
        double *row = sp + b * PROF_NQ;
        for (int k = 0; k < PROF_NQ; k++) atomicAdd(row + k, q[k]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbins * PROF_NQ; i += blockDim.x) part[(size_t)blockIdx.x * nbins * PROF_NQ + i] = sp[i];
}

size_t pipe_profile_scratch_bytes(int nbins) { return sizeof(double) * (size_t)PROF_BLOCKS * nbins * PROF_NQ; }

// scratch: the population buffer that the next step overwrites
cudaError_t run_pipe_profiles(Ctx &c, int flags, int nbins, double *out) {
    cudaError_t e;
    if ((e = launch_macro(c, 0)) != cudaSuccess) return e;
    const int ibm = c.armed_bc == LBM_BC_IBM_U || c.armed_bc == LBM_BC_IBM_B;
    if (!(ibm && (flags & LBM_STATS_UNMASK)))
        if ((e = launch_mask(c)) != cudaSuccess) return e;
    double *part = (double *)c.fB;
    const double nu = (c.tau - 0.5) / 3.0;
    count_launch(c, G_STATS);
    pipe_profile_kernel<<<PROF_BLOCKS, SB, sizeof(double) * nbins * PROF_NQ, c.stream>>>(
        c.u_f, c.rho_f, c.flags, c.nx, c.ny, c.nz, c.N, c.pipe_cx, c.pipe_cy, c.pipe_R, nbins, nu, part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::vector<double> hp((size_t)PROF_BLOCKS * nbins * PROF_NQ);
    if ((e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, c.stream)) !=
        cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(c.stream)) != cudaSuccess) return e;
    for (int b = 0; b < nbins; b++) {
        double s[PROF_NQ] = {0};
        for (int blk = 0; blk < PROF_BLOCKS; blk++)  // fixed block order
            for (int k = 0; k < PROF_NQ; k++) s[k] += hp[((size_t)blk * nbins + b) * PROF_NQ + k];
        const double cnt = s[0];
        out[(size_t)b * PROF_NQ] = cnt;
        for (int k = 1; k < PROF_NQ; k++) out[(size_t)b * PROF_NQ + k] = cnt > 0.0 ? s[k] / cnt : 0.0;
    }
    return cudaSuccess;
}

cudaError_t launch_mask(Ctx &c) {
    count_launch(c, G_STATS);
    mask_kernel<<<(unsigned)((c.N + 255) / 256), 256, 0, c.stream>>>(c.u_f, c.flags, c.owner, c.X, c.U, c.W, c.nx,
                                                                     c.ny, c.nz, c.N);
    return cudaGetLastError();
}

cudaError_t run_stats(Ctx &c, int flags, lbm_stats_t *o) {
    cudaError_t e;
    memset(o, 0, sizeof(*o));
    const int ibb = c.armed_bc == LBM_BC_IBB;
    const int ibm = c.armed_bc == LBM_BC_IBM_U || c.armed_bc == LBM_BC_IBM_B;
    const bool closure = (flags & LBM_STATS_CLOSURE) && c.np > 0 && c.cl_ready && c.max_cl > 0 && c.q == 19;
    // the closure gathers an FP32 copy of u (16 B per cell), kept in the
    // population buffer that the next step overwrites (19 x 2 B per cell or more)
    float *u32 = closure ? (float *)c.fB : nullptr;
    if ((e = launch_macro(c, 0, u32)) != cudaSuccess) return e;
    count_launch(c, G_STATS, 3);
    mass_kernel<<<SNB, SB, 0, c.stream>>>(c.rho_f, c.u_f, c.flags, c.N, ibb, c.partials);
    const bool mask = !(ibm && (flags & LBM_STATS_UNMASK));
    const unsigned nb = (unsigned)((c.N + 255) / 256);
    const double nu = (c.tau - 0.5) / 3.0;
    const bool bins = (flags & LBM_STATS_BINS) && c.np > 0;
    const float *eps_o = nullptr;
    // the bins reach r/R_p = 1 + 0.05 NBIN; the closure 2 lattice units from the surface
    double reach = bins ? 0.05 * NBIN * c.max_radius : 0.0;
    if (closure && reach < 2.0) reach = 2.0;
    if (bins || closure) near_surface(c, nb, reach);
    if (closure) {
        // learned gradients at the near-surface nodes (unmasked velocity in):
        // list the nodes, then one tensor-core kernel gathers each node's
        // features, runs the network and writes the dissipation at the cell
        count_launch(c, G_STATS, 4);
        fill_f32<<<nb, 256, 0, c.stream>>>(c.cl_eps, -1.f, c.N);
        if ((e = cudaMemsetAsync(c.d_counts + 3, 0, sizeof(long long), c.stream)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(c.d_status + 1, 0, sizeof(unsigned), c.stream)) != cudaSuccess) return e;
        int *pids = (int *)c.cl_X;  // the feature buffer is not needed by the fused path
        closure_list_kernel<<<nb, 256, 0, c.stream>>>(c.flags, c.near_key, c.N, c.cl_cells, pids, c.d_counts + 3,
                                                      c.max_cl);
        if ((e = mlp_pack_device(c.cl_w, c.cl_pk, c.stream)) != cudaSuccess) return e;
        cudaEvent_t t0 = prof_event(c);
        count_launch(c, G_CLOSURE, 2);  // particle records, inference
        if ((e = closure_eps_tc(c, u32, c.cl_cells, pids, c.d_counts + 3, c.max_cl, c.cl_pk, c.cl_eps,
                                (int *)(c.d_status + 1))) != cudaSuccess)
            return e;
        prof_span(c, G_CLOSURE, t0, prof_event(c));
        eps_o = c.cl_eps;
    }
    if (mask) mask_kernel<<<nb, 256, 0, c.stream>>>(c.u_f, c.flags, c.owner, c.X, c.U, c.W, c.nx, c.ny, c.nz, c.N);
    energy_kernel<<<SNB, SB, 0, c.stream>>>(c.u_f, c.flags, c.nx, c.ny, c.nz, c.N, nu, c.has_pipe, c.partials, eps_o);
    double *bpart = c.partials + SNB * NP;
    if (bins) {
        count_launch(c, G_STATS);
        bins_kernel<<<SNB, SB, 0, c.stream>>>(c.u_f, c.flags, c.near_key, c.X, c.R, c.nx, c.ny, c.nz, c.N, nu, bpart,
                                              eps_o);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::vector<double> part((size_t)SNB * NP), bp(bins ? (size_t)SNB * 3 * NBIN : 0);
    if ((e = cudaMemcpyAsync(part.data(), c.partials, sizeof(double) * part.size(), cudaMemcpyDeviceToHost,
                             c.stream)) != cudaSuccess)
        return e;
    if (bins && (e = cudaMemcpyAsync(bp.data(), bpart, sizeof(double) * bp.size(), cudaMemcpyDeviceToHost,
                                     c.stream)) != cudaSuccess)
        return e;
    std::vector<double> P(3 * c.np), Uh(3 * c.np), Wh(3 * c.np), Fh(3 * c.np), Th(3 * c.np), mass(c.np), inertia(c.np);
    if (c.np > 0) {
        cudaMemcpyAsync(Uh.data(), c.U, sizeof(double) * 3 * c.np, cudaMemcpyDeviceToHost, c.stream);
        cudaMemcpyAsync(Wh.data(), c.W, sizeof(double) * 3 * c.np, cudaMemcpyDeviceToHost, c.stream);
        cudaMemcpyAsync(Fh.data(), c.Fh, sizeof(double) * 3 * c.np, cudaMemcpyDeviceToHost, c.stream);
        cudaMemcpyAsync(Th.data(), c.Th, sizeof(double) * 3 * c.np, cudaMemcpyDeviceToHost, c.stream);
        cudaMemcpyAsync(mass.data(), c.mass, sizeof(double) * c.np, cudaMemcpyDeviceToHost, c.stream);
        cudaMemcpyAsync(inertia.data(), c.inertia, sizeof(double) * c.np, cudaMemcpyDeviceToHost, c.stream);
    }
    unsigned tc_err = 0;
    if (closure && (e = cudaMemcpyAsync(&tc_err, c.d_status + 1, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                        c.stream)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(c.stream)) != cudaSuccess) return e;
    if (tc_err) return cudaErrorLaunchTimeout;  // a tensor-core wait of the closure ran out
    double s[NP] = {0};
    for (int b = 0; b < SNB; b++)
        for (int k = 0; k < 11; k++) s[k] += part[(size_t)b * NP + k];
    o->mass = s[0];
    o->momentum[0] = s[1];
    o->momentum[1] = s[2];
    o->momentum[2] = s[3];
    o->kinetic_energy = s[4] / (double)c.N;
    o->dissipation = s[5] / (double)c.N;
    o->nfluid = (long long)s[8];
    o->kinetic_energy_fluid = s[8] > 0 ? s[6] / s[8] : 0.0;
    o->dissipation_fluid = s[8] > 0 ? s[7] / s[8] : 0.0;
    o->bulk_velocity = s[10] > 0 ? s[9] / s[10] : 0.0;
    for (int p = 0; p < c.np; p++) {
        double U2 = 0, W2 = 0;
        for (int d = 0; d < 3; d++) {
            U2 += Uh[3 * p + d] * Uh[3 * p + d];
            W2 += Wh[3 * p + d] * Wh[3 * p + d];
            o->force[d] += Fh[3 * p + d];
            o->torque[d] += Th[3 * p + d];
        }
        o->particle_ke += 0.5 * mass[p] * U2;
        o->particle_ake += 0.5 * inertia[p] * W2;
    }
    if (bins) {
        double sk[NBIN] = {0}, se[NBIN] = {0}, sc[NBIN] = {0};
        for (int b = 0; b < SNB; b++)
            for (int k = 0; k < NBIN; k++) {
                sk[k] += bp[(size_t)b * 3 * NBIN + k];
                se[k] += bp[(size_t)b * 3 * NBIN + NBIN + k];
                sc[k] += bp[(size_t)b * 3 * NBIN + 2 * NBIN + k];
            }
        o->nbins = NBIN;
        for (int k = 0; k < NBIN; k++) {
            o->bin_r[k] = 1.0 + 0.05 * (k + 0.5);
            o->bin_count[k] = (long long)sc[k];
            if (sc[k] > 0) {
                const double kf = o->kinetic_energy_fluid > 0 ? o->kinetic_energy_fluid : 1.0;
                const double ef = o->dissipation_fluid > 0 ? o->dissipation_fluid : 1.0;
                o->bin_tke[k] = sk[k] / sc[k] / kf;
                o->bin_eps[k] = se[k] / sc[k] / ef;
            }
        }
    }
    o->nlinks = c.armed_bc == LBM_BC_IBB ? c.nlinks : 0;
    o->nmarkers = c.nm;
    o->step = c.step;
    return cudaSuccess;
}

size_t stats_partials_doubles() { return (size_t)SNB * NP + (size_t)SNB * 3 * NBIN; }

}  // namespace lbmgb
