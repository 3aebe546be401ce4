// D3Q27 on a periodic box: the velocity set of the paper's pipe solver
// (Sec. 2.1: D3Q27 MRT run with a single relaxation parameter, i.e. BGK).
// Same storage (shifted g = f - w_i, FP64 or FP32), pull streaming, Guo
// forcing and post-collision stored state as the D3Q19 path.
//
// Velocity order (the interface of populations in and out): rest, the 6
// faces, the 12 edges, the 8 corners; within a group the triples
// (c_x, c_y, c_z) over {-1, 0, 1}^3 in lexicographic order (c_x slowest).
// Weights 8/27, 2/27, 1/54, 1/216 by |c|^2 = 0 .. 3.
#include "lbm_internal.cuh"

#include <vector>

#ifndef LBM_Q27_MINB
#define LBM_Q27_MINB 0  // resident blocks of 256 per SM the pipe kernel's registers are sized for (0: per storage)
#endif

namespace lbmgb {

namespace {

// components as characters '0', '1', '2' for -1, 0, 1 (compile-time lookups)
__host__ __device__ constexpr int q27x(int i) { return "101111200001111222200002222"[i] - '1'; }
__host__ __device__ constexpr int q27y(int i) { return "110112101120022011200220022"[i] - '1'; }
__host__ __device__ constexpr int q27z(int i) { return "111021110210202102102020202"[i] - '1'; }
__host__ __device__ constexpr double q27w(int i) {
    return i == 0 ? 8.0 / 27.0 : (i <= 6 ? 2.0 / 27.0 : (i <= 18 ? 1.0 / 54.0 : 1.0 / 216.0));
}
static_assert(q27x(1) == -1 && q27y(1) == 0 && q27z(1) == 0, "first face");
static_assert(q27x(26) == 1 && q27y(26) == 1 && q27z(26) == 1, "last corner");
static_assert(q27x(7) * q27x(7) + q27y(7) * q27y(7) + q27z(7) * q27z(7) == 2, "first edge");
static_assert(q27x(19) * q27x(19) + q27y(19) * q27y(19) + q27z(19) * q27z(19) == 3, "first corner");

constexpr int Q27 = 27;

template <int S>
__global__ void q27_init_kernel(void *A, const double *u, double rho0, long long N) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const double ux = u[c], uy = u[N + c], uz = u[2 * N + c];
    const double u2 = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < Q27; i++) {
        const double cu = q27x(i) * ux + q27y(i) * uy + q27z(i) * uz;
        const double feq = q27w(i) * rho0 * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
        Store<S>::st((T *)A + (size_t)i * N + c, R(feq - q27w(i)));
    }
}

template <int S>
__global__ void q27_plane_kernel(void *A, double *v, long long N, int i, int to_f64) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    T *p = (T *)A + (size_t)i * N + c;
    const double w = q27w(i);
    if (to_f64) v[c] = (double)Store<S>::ld(p) + w;
    else Store<S>::st(p, R(v[c] - w));
}

// rho and u of the post-collision state: sum f c = rho u + F/2
template <int S>
__global__ void q27_macro_kernel(const void *A, double *rho_o, double *u_o, long long N, double F0, double F1,
                                 double F2) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const T *P = (const T *)A;
    R r = R(0), j0 = R(0), j1 = R(0), j2 = R(0);
#pragma unroll
    for (int i = 0; i < Q27; i++) {
        const R g = Store<S>::ld(P + (size_t)i * N + c);
        r += g;
        j0 += g * R(q27x(i));
        j1 += g * R(q27y(i));
        j2 += g * R(q27z(i));
    }
    const R rho = R(1) + r, ir = R(1) / rho;
    rho_o[c] = double(rho);
    u_o[c] = double((j0 - R(0.5) * R(F0)) * ir);
    u_o[N + c] = double((j1 - R(0.5) * R(F1)) * ir);
    u_o[2 * N + c] = double((j2 - R(0.5) * R(F2)) * ir);
}

struct Q27Args {
    const void *A;
    void *B;
    long long N;
    int nx, ny, nz;
    FastDiv fx, fxy;  // division by nx and nx * ny
    double om;        // 1 / tau
    double F[3];
    unsigned *status;
};

// one cell per thread: pull f_i(x) = f*_i(x - c_i) (periodic), BGK with the
// Guo source, store the post-collision values
template <int S, bool FORCE>
__global__ void __launch_bounds__(256) q27_sweep_kernel(Q27Args a) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.N) return;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const unsigned zq = a.fxy.div((unsigned)c), rem = (unsigned)c - zq * (unsigned)(nx * ny);
    const unsigned yq = a.fx.div(rem);
    const int z = (int)zq, y = (int)yq, x = (int)(rem - yq * (unsigned)nx);
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const T *__restrict__ A = (const T *)a.A;
    T *__restrict__ B = (T *)a.B;
    const size_t N = (size_t)a.N;
    R g[Q27];
#pragma unroll
    for (int i = 0; i < Q27; i++) {
        const int xs = q27x(i) > 0 ? xm : (q27x(i) < 0 ? xp : x);
        const int ys = q27y(i) > 0 ? ym : (q27y(i) < 0 ? yp : y);
        const int zs = q27z(i) > 0 ? zm : (q27z(i) < 0 ? zp : z);
        g[i] = Store<S>::ld(A + (i * N + (size_t)(xs + nx * (ys + ny * zs))));
    }
    R drho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int i = 0; i < Q27; i++) {
        drho += g[i];
        if (q27x(i)) jx += q27x(i) > 0 ? g[i] : -g[i];
        if (q27y(i)) jy += q27y(i) > 0 ? g[i] : -g[i];
        if (q27z(i)) jz += q27z(i) > 0 ? g[i] : -g[i];
    }
    const R Fx = FORCE ? R(a.F[0]) : R(0), Fy = FORCE ? R(a.F[1]) : R(0), Fz = FORCE ? R(a.F[2]) : R(0);
    const R rho = R(1) + drho, ir = R(1) / rho;
    const R ux = (jx + R(0.5) * Fx) * ir, uy = (jy + R(0.5) * Fy) * ir, uz = (jz + R(0.5) * Fz) * ir;
    const R u2 = ux * ux + uy * uy + uz * uz;
    // g_eq = f_eq - w = w (drho - 1.5 rho u^2 + c.u (3 rho + 4.5 rho c.u))
    const R om = R(a.om), c1 = R(1) - R(0.5) * om;
    const R base = drho - rho * R(1.5) * u2, r3 = R(3) * rho, r45 = R(4.5) * rho;
    const R uF3 = FORCE ? R(3) * (ux * Fx + uy * Fy + uz * Fz) : R(0);
#pragma unroll
    for (int i = 0; i < Q27; i++) {
        const R cu = R(q27x(i)) * ux + R(q27y(i)) * uy + R(q27z(i)) * uz;
        const R geq = R(q27w(i)) * (base + cu * (r3 + r45 * cu));
        R v = g[i] + om * (geq - g[i]);
        if (FORCE) {
            const R cF = R(q27x(i)) * Fx + R(q27y(i)) * Fy + R(q27z(i)) * Fz;
            v += (c1 * R(q27w(i))) * (R(3) * cF - uF3 + R(9) * cu * cF);
        }
        Store<S>::st(B + (i * N + (size_t)c), v);
    }
    watchdog(rho, ux, uy, uz, a.status);
}

__host__ __device__ constexpr int q27opp(int i) {
    // the opposite velocity has every component negated: search the table
    int o = 0;
    for (int j = 0; j < Q27; j++)
        if (q27x(j) == -q27x(i) && q27y(j) == -q27y(i) && q27z(j) == -q27z(i)) o = j;
    return o;
}
static_assert(q27opp(0) == 0 && q27opp(1) == 6 && q27opp(26) == 19, "opposites");

// The pipe wall of the paper's runs (Sec. 2.1) on D3Q27: cells with
// (x - c_x)^2 + (y - c_y)^2 >= R^2 are solid. A link (x_f, i) joins a fluid
// cell to a solid x_f + c_i; the wall sits at x_f + q c_i, q in (0, 1] the
// exit root of the cylinder equation along c_i (FP64). The population
// j = opp(i) that cannot be pulled from x_f + c_i is the linear
// interpolated bounce-back (Bouzidi et al. 2001) from post-collision values
// at the wall at rest:
//   q < 1/2: 2q f*_i(x_f) + (1 - 2q) f*_i(x_f - c_i), x_f - c_i fluid, else f*_i(x_f);
//   q >= 1/2: f*_i(x_f) / (2q) + (2q - 1)/(2q) f*_j(x_f).
// The geometry is the same in every z plane: per (x, y) column a 27-bit
// mask (bit i: the column x + c_i, y + c_i is solid; bit 0: the column
// itself) tells which pulls come from the wall. Solid cells are not swept.
// The weights of the two populations of each wall link are formed once, at
// set-up (q27_coef_kernel), per column and direction: (2q, 1 - 2q) with
// f*_i(x_f - c_i), (1, 0) for the halfway fallback, and
// (1/(2q), (2q - 1)/(2q)) with f*_j(x_f), the last flagged in hmask.
struct Q27PipeArgs {
    Q27Args b;
    const unsigned *colmask, *hmask;
    const void *coef;  // per column x 27 directions: two weights in the arithmetic type
    // when no fluid cell touches an x or y face: the pull of direction i
    // for cell c is Ap[i][c] (plus N or minus N across the z ends), its
    // store Bp[i][c]: one address operation per access
    int nowrap;
    const void *Ap[Q27];  // A + i N - (c_x + nx c_y + nx ny c_z)
    void *Bp[Q27];        // B + i N
};

template <typename R>
struct Q27Coef {
    R k1, k2;
};

template <int S>
__global__ void q27_coef_kernel(const unsigned *colmask, unsigned *hmask, void *coefv, int nx, int ny, double pcx,
                                double pcy, double R2) {
    typedef typename Store<S>::R R;
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= nx * ny) return;
    const unsigned m = colmask[col];
    Q27Coef<R> *coef = (Q27Coef<R> *)coefv + (size_t)col * Q27;
    unsigned h = 0;
    if (!(m & 1u) && m) {
        const int x = col % nx, y = col / nx;
        const double dx = (double)x - pcx, dy = (double)y - pcy;
        const double c0 = dx * dx + dy * dy - R2;
        for (int i = 1; i < Q27; i++) {
            if (!((m >> i) & 1u)) continue;
            const double aa = (double)(q27x(i) * q27x(i) + q27y(i) * q27y(i));
            const double b = q27x(i) * dx + q27y(i) * dy;
            const double q = (-b + sqrt(b * b - aa * c0)) / aa;
            Q27Coef<R> k;
            if (q < 0.5) {
                if ((m >> q27opp(i)) & 1u) {  // x_f - c_i solid too: halfway
                    k.k1 = R(1);
                    k.k2 = R(0);
                } else {
                    k.k1 = R(2.0 * q);
                    k.k2 = R(1.0 - 2.0 * q);
                }
            } else {
                k.k1 = R(1.0 / (2.0 * q));
                k.k2 = R((2.0 * q - 1.0) / (2.0 * q));
                h |= 1u << i;
            }
            coef[i] = k;
        }
    }
    hmask[col] = h;
}

// FP32: registers for 4 resident blocks of 256 per SM (64, no spills):
// 0.387 ms per step on the benchmark pipe against 0.477 ms at 80 registers
// (3 blocks), where only 13 of the 24 possible warps were active (the solid
// cells' threads end at once, their blocks stay resident)
constexpr int q27_min_blocks(int S) { return LBM_Q27_MINB > 0 ? LBM_Q27_MINB : (S == LBM_F32 ? 4 : 1); }

template <int S, bool FORCE>
__global__ void __launch_bounds__(256, q27_min_blocks(S)) q27_pipe_kernel(Q27PipeArgs pa) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const Q27Args &a = pa.b;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.N) return;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const unsigned zq = a.fxy.div((unsigned)c), rem = (unsigned)c - zq * (unsigned)(nx * ny);
    const unsigned yq = a.fx.div(rem);
    const int z = (int)zq, y = (int)yq, x = (int)(rem - yq * (unsigned)nx);
    const unsigned m = __ldg(pa.colmask + rem);
    if (m & 1u) return;  // solid: keeps its values, never read
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const T *__restrict__ A = (const T *)a.A;
    T *__restrict__ B = (T *)a.B;
    const size_t N = (size_t)a.N;
    R g[Q27];
    if (pa.nowrap) {
        const int zpl = z == 0 ? (int)N : 0, zmi = z == nz - 1 ? (int)N : 0;
#pragma unroll
        for (int i = 0; i < Q27; i++) {
            const int o = (int)c + (q27z(i) > 0 ? zpl : 0) - (q27z(i) < 0 ? zmi : 0);
            g[i] = Store<S>::ld((const T *)pa.Ap[i] + o);
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q27; i++) {
            const int xs = q27x(i) > 0 ? xm : (q27x(i) < 0 ? xp : x);
            const int ys = q27y(i) > 0 ? ym : (q27y(i) < 0 ? yp : y);
            const int zs = q27z(i) > 0 ? zm : (q27z(i) < 0 ? zp : z);
            g[i] = Store<S>::ld(A + (i * N + (size_t)(xs + nx * (ys + ny * zs))));
        }
    }
    if (m) {  // wall cell: the populations coming back from the wall
        const unsigned h = __ldg(pa.hmask + rem);
        const Q27Coef<R> *kc = (const Q27Coef<R> *)pa.coef + (size_t)rem * Q27;
#pragma unroll
        for (int i = 1; i < Q27; i++) {
            if (!((m >> i) & 1u)) continue;
            const int j = q27opp(i);
            const Q27Coef<R> k = kc[i];
            const R fi = Store<S>::ld(A + (i * N + (size_t)c));  // f*_i(x_f)
            // q < 1/2: f*_i(x_f - c_i), the regular pull of direction i
            // (weight 0 for the halfway fallback); q >= 1/2: f*_j(x_f)
            const R second = ((h >> i) & 1u) ? Store<S>::ld(A + (j * N + (size_t)c)) : g[i];
            // the bounce-back acts on f, the storage holds g = f - w with w_i = w_j
            g[j] = k.k1 * fi + k.k2 * second;
        }
    }
    R drho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int i = 0; i < Q27; i++) {
        drho += g[i];
        if (q27x(i)) jx += q27x(i) > 0 ? g[i] : -g[i];
        if (q27y(i)) jy += q27y(i) > 0 ? g[i] : -g[i];
        if (q27z(i)) jz += q27z(i) > 0 ? g[i] : -g[i];
    }
    const R Fx = FORCE ? R(a.F[0]) : R(0), Fy = FORCE ? R(a.F[1]) : R(0), Fz = FORCE ? R(a.F[2]) : R(0);
    const R rho = R(1) + drho, ir = R(1) / rho;
    const R ux = (jx + R(0.5) * Fx) * ir, uy = (jy + R(0.5) * Fy) * ir, uz = (jz + R(0.5) * Fz) * ir;
    const R u2 = ux * ux + uy * uy + uz * uz;
    const R om = R(a.om), c1 = R(1) - R(0.5) * om;
    const R base = drho - rho * R(1.5) * u2, r3 = R(3) * rho, r45 = R(4.5) * rho;
    const R uF3 = FORCE ? R(3) * (ux * Fx + uy * Fy + uz * Fz) : R(0);
#pragma unroll
    for (int i = 0; i < Q27; i++) {
        const R cu = R(q27x(i)) * ux + R(q27y(i)) * uy + R(q27z(i)) * uz;
        const R geq = R(q27w(i)) * (base + cu * (r3 + r45 * cu));
        R v = g[i] + om * (geq - g[i]);
        if (FORCE) {
            const R cF = R(q27x(i)) * Fx + R(q27y(i)) * Fy + R(q27z(i)) * Fz;
            v += (c1 * R(q27w(i))) * (R(3) * cF - uF3 + R(9) * cu * cF);
        }
        Store<S>::st(pa.nowrap ? (T *)pa.Bp[i] + c : B + (i * N + (size_t)c), v);
    }
    watchdog(rho, ux, uy, uz, a.status);
}

}  // namespace

template <int S>
static cudaError_t q27_step_s(Ctx &c, const Q27Args &a, bool force) {
    const unsigned nb = (unsigned)((c.N + 255) / 256);
    if (force) q27_sweep_kernel<S, true><<<nb, 256, 0, c.stream>>>(a);
    else q27_sweep_kernel<S, false><<<nb, 256, 0, c.stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_q27_step(Ctx &c) {
    Q27Args a;
    a.A = c.fA;
    a.B = c.fB;
    a.N = c.N;
    a.nx = c.nx;
    a.ny = c.ny;
    a.nz = c.nz;
    a.fx = FastDiv((unsigned)c.nx);
    a.fxy = FastDiv((unsigned)(c.nx * c.ny));
    a.om = 1.0 / c.tau;
    for (int d = 0; d < 3; d++) a.F[d] = c.F[d];
    a.status = c.d_status;
    const bool force = c.F[0] != 0.0 || c.F[1] != 0.0 || c.F[2] != 0.0;
    count_launch(c, G_BULK);
    if (c.has_pipe) {
        Q27PipeArgs pa;
        pa.b = a;
        pa.colmask = c.q27_colmask;
        pa.hmask = c.q27_hmask;
        pa.coef = c.q27_coef;
        pa.nowrap = c.pipe_nowrap && c.N < (1LL << 30);
        const size_t sb = storage_bytes(c.storage);
        for (int i = 0; i < Q27; i++) {
            const long long off = q27x(i) + (long long)c.nx * q27y(i) + (long long)c.nx * c.ny * q27z(i);
            pa.Ap[i] = (const void *)((const char *)c.fA + sb * (size_t)((long long)i * c.N - off));
            pa.Bp[i] = (void *)((char *)c.fB + sb * (size_t)((long long)i * c.N));
        }
        const unsigned nb = (unsigned)((c.N + 255) / 256);
        if (c.storage == LBM_F64) {
            if (force) q27_pipe_kernel<LBM_F64, true><<<nb, 256, 0, c.stream>>>(pa);
            else q27_pipe_kernel<LBM_F64, false><<<nb, 256, 0, c.stream>>>(pa);
        } else {
            if (force) q27_pipe_kernel<LBM_F32, true><<<nb, 256, 0, c.stream>>>(pa);
            else q27_pipe_kernel<LBM_F32, false><<<nb, 256, 0, c.stream>>>(pa);
        }
        return cudaGetLastError();
    }
    return c.storage == LBM_F64 ? q27_step_s<LBM_F64>(c, a, force) : q27_step_s<LBM_F32>(c, a, force);
}

// per (x, y) column: bit i set when the column (x + c_x, y + c_y) of
// direction i is outside the pipe (bit 0: the column itself); FP64 test as
// the D3Q19 pipe flags
void q27_pipe_colmask(const Ctx &c, std::vector<unsigned> &mask) {
    mask.assign((size_t)c.nx * c.ny, 0u);
    auto solid = [&](int x, int y) {
        x = (x % c.nx + c.nx) % c.nx;
        y = (y % c.ny + c.ny) % c.ny;
        const double dx = (double)x - c.pipe_cx, dy = (double)y - c.pipe_cy;
        return dx * dx + dy * dy >= c.pipe_R * c.pipe_R;
    };
    for (int y = 0; y < c.ny; y++)
        for (int x = 0; x < c.nx; x++) {
            unsigned m = 0;
            for (int i = 0; i < Q27; i++)
                if (solid(x + q27x(i), y + q27y(i))) m |= 1u << i;
            mask[(size_t)x + (size_t)c.nx * y] = m;
        }
}

// the wall weights of the pipe (after the column masks are uploaded)
cudaError_t launch_q27_coef(Ctx &c) {
    const unsigned nb = (unsigned)((c.nx * c.ny + 255) / 256);
    const double R2 = c.pipe_R * c.pipe_R;
    if (c.storage == LBM_F64)
        q27_coef_kernel<LBM_F64><<<nb, 256, 0, c.stream>>>(c.q27_colmask, c.q27_hmask, c.q27_coef, c.nx, c.ny,
                                                            c.pipe_cx, c.pipe_cy, R2);
    else
        q27_coef_kernel<LBM_F32><<<nb, 256, 0, c.stream>>>(c.q27_colmask, c.q27_hmask, c.q27_coef, c.nx, c.ny,
                                                            c.pipe_cx, c.pipe_cy, R2);
    return cudaGetLastError();
}

cudaError_t launch_q27_init(Ctx &c, const double *u_dev, double rho0) {
    const unsigned nb = (unsigned)((c.N + 255) / 256);
    if (c.storage == LBM_F64) q27_init_kernel<LBM_F64><<<nb, 256, 0, c.stream>>>(c.fA, u_dev, rho0, c.N);
    else q27_init_kernel<LBM_F32><<<nb, 256, 0, c.stream>>>(c.fA, u_dev, rho0, c.N);
    return cudaGetLastError();
}

// one population plane to or from the FP64 scratch c.rho_f (unshifted f)
cudaError_t q27_plane_copy(Ctx &c, int i, bool to_f64) {
    const unsigned nb = (unsigned)((c.N + 255) / 256);
    if (c.storage == LBM_F64) q27_plane_kernel<LBM_F64><<<nb, 256, 0, c.stream>>>(c.fA, c.rho_f, c.N, i, to_f64);
    else q27_plane_kernel<LBM_F32><<<nb, 256, 0, c.stream>>>(c.fA, c.rho_f, c.N, i, to_f64);
    return cudaGetLastError();
}

cudaError_t launch_q27_macro(Ctx &c) {
    count_launch(c, G_STATS);
    const unsigned nb = (unsigned)((c.N + 255) / 256);
    if (c.storage == LBM_F64)
        q27_macro_kernel<LBM_F64><<<nb, 256, 0, c.stream>>>(c.fA, c.rho_f, c.u_f, c.N, c.F[0], c.F[1], c.F[2]);
    else
        q27_macro_kernel<LBM_F32><<<nb, 256, 0, c.stream>>>(c.fA, c.rho_f, c.u_f, c.N, c.F[0], c.F[1], c.F[2]);
    return cudaGetLastError();
}

}  // namespace lbmgb
