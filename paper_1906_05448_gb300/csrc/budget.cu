// Component-wise TKE budget of the pipe (Eq. 1a-c, Sec. 2.2): production,
// turbulent transport, pressure work, viscous diffusion and dissipation of
// the streamwise, radial and azimuthal velocity fluctuations, per radial
// bin of one snapshot.
//
// The per-cell work runs in two passes over the cells inside the pipe
// (r > 0, bin b = floor(r nbins / R)): pass 1 sums 20 quantities per bin
// (velocity components, pressure, strain and gradient components in the
// local basis e_r, e_theta, e_z), pass 2 sums 20 products of their
// fluctuations about the bin means of pass 1. The sums are FP64, per block
// in shared memory and added over the blocks on the host in a fixed order.
// The host then takes the radial derivatives of the binned profiles
// (central differences over the bin centres, one-sided at the ends).
//
// Local quantities of a cell (statistics velocity, central differences):
//   G_ab = d u_a / d x_b, T_ij = e_i . G . e_j, s_ij = (T_ij + T_ji) / 2,
//   du_i/dr = T_ir, du_i/dz = T_iz, (1/r) du_z/dtheta = T_ztheta,
//   (1/r) du_r/dtheta = T_rtheta + u_theta / r,
//   (1/r) du_theta/dtheta = T_thetatheta - u_r / r,
//   p = c_s^2 rho.
#include "lbm_internal.cuh"

#include <vector>

namespace lbmgb {

namespace {

constexpr int BQ = 20;          // quantities per bin and pass
constexpr int BUD_BLOCKS = 304;  // 2 blocks per SM
constexpr int BUD_TB = 256;

// pass-1 quantities (bin means)
enum { M_ONE, M_UZ, M_UR, M_UT, M_P, M_SZR, M_SZT, M_SZZ, M_SRR, M_SRT, M_STT,
       M_DRZ, M_DTHZ, M_DZZ, M_DRR, M_DTHR, M_DZR, M_DRT, M_DTHT, M_DZT };
static_assert(M_DZT + 1 == BQ, "pass-1 table");

// one cell: its bin and its BQ local quantities; false outside the pipe,
// on the axis or beyond the last bin
__device__ bool budget_cell(const double *u, const double *rho, const uint8_t *flags, long long c, int nx, int ny,
                            int nz, long long N, double cx, double cy, double R, int nbins, int &b, double q[BQ]) {
    if (flags[c] & FL_SOLID) return false;
    const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
    // r and the bin with explicitly rounded operations, as the radial profiles
    const double dx = __dsub_rn((double)x, cx), dy = __dsub_rn((double)y, cy);
    const double r = sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    if (!(r > 0.0)) return false;
    b = (int)floor(__ddiv_rn(__dmul_rn(r, (double)nbins), R));
    if (b < 0 || b >= nbins) return false;
    // Cartesian gradient by central differences, periodic wrap
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const long long row = (long long)nx * ny;
    const long long cxm = c - x + xm, cxp = c - x + xp;
    const long long cym = c + (long long)(ym - y) * nx, cyp = c + (long long)(yp - y) * nx;
    const long long czm = c + (long long)(zm - z) * row, czp = c + (long long)(zp - z) * row;
    double G[3][3];
    for (int a = 0; a < 3; a++) {
        const double *ua = u + (long long)a * N;
        G[a][0] = 0.5 * (ua[cxp] - ua[cxm]);
        G[a][1] = 0.5 * (ua[cyp] - ua[cym]);
        G[a][2] = 0.5 * (ua[czp] - ua[czm]);
    }
    // local basis e_r, e_theta, e_z
    const double e[3][3] = {{dx / r, dy / r, 0.0}, {-dy / r, dx / r, 0.0}, {0.0, 0.0, 1.0}};
    double T[3][3];  // indices 0 r, 1 theta, 2 z
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double t = 0.0;
            for (int a = 0; a < 3; a++)
                for (int k = 0; k < 3; k++) t += e[i][a] * G[a][k] * e[j][k];
            T[i][j] = t;
        }
    const double ux = u[c], uy = u[N + c], uzv = u[2 * N + c];
    const double ur = e[0][0] * ux + e[0][1] * uy, ut = e[1][0] * ux + e[1][1] * uy;
    q[M_ONE] = 1.0;
    q[M_UZ] = uzv;
    q[M_UR] = ur;
    q[M_UT] = ut;
    q[M_P] = rho[c] * (1.0 / 3.0);  // p = c_s^2 rho
    q[M_SZR] = 0.5 * (T[2][0] + T[0][2]);
    q[M_SZT] = 0.5 * (T[2][1] + T[1][2]);
    q[M_SZZ] = T[2][2];
    q[M_SRR] = T[0][0];
    q[M_SRT] = 0.5 * (T[0][1] + T[1][0]);
    q[M_STT] = T[1][1];
    q[M_DRZ] = T[2][0];
    q[M_DTHZ] = T[2][1];
    q[M_DZZ] = T[2][2];
    q[M_DRR] = T[0][0];
    q[M_DTHR] = T[0][1] + ut / r;
    q[M_DZR] = T[0][2];
    q[M_DRT] = T[1][0];
    q[M_DTHT] = T[1][1] - ur / r;
    q[M_DZT] = T[1][2];
    return true;
}

// pass-2 products of fluctuations (bin means), in the order the terms use them
enum { P_ZR, P_ZZR, P_P_DZZ, P_Z_SZR, P_SZR_DRZ, P_SZT_DTHZ, P_SZZ_DZZ,
       P_RRR, P_R_P, P_P_DRR, P_R_SRR, P_SRR_DRR, P_SRT_DTHR, P_SZR_DZR,
       P_TTR, P_P_DTHT, P_T_SRT, P_STT_DTHT, P_SRT_DRT, P_SZT_DZT };
static_assert(P_SZT_DZT + 1 == BQ, "pass-2 table");

struct BudgetArgs {
    const double *u, *rho;
    const uint8_t *flags;
    const double *mean;  // pass 2: nbins x BQ bin means of pass 1
    double *part;        // BUD_BLOCKS x nbins x BQ block sums
    int nx, ny, nz;
    long long N;
    double cx, cy, R;
    int nbins;
};

template <int PASS>
__global__ void __launch_bounds__(BUD_TB) budget_kernel(BudgetArgs a) {
    extern __shared__ double sb[];  // nbins x BQ
    for (int i = threadIdx.x; i < a.nbins * BQ; i += blockDim.x) sb[i] = 0.0;
    __syncthreads();
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < a.N;
         c += (long long)gridDim.x * blockDim.x) {
        int b;
        double q[BQ];
        if (!budget_cell(a.u, a.rho, a.flags, c, a.nx, a.ny, a.nz, a.N, a.cx, a.cy, a.R, a.nbins, b, q)) continue;
        double *row = sb + b * BQ;
        if (PASS == 1) {
            for (int k = 0; k < BQ; k++) atomicAdd(row + k, q[k]);
        } else {
            const double *m = a.mean + b * BQ;
            double f[BQ];
            for (int k = 0; k < BQ; k++) f[k] = q[k] - m[k];
            const double v[BQ] = {f[M_UZ] * f[M_UR], f[M_UZ] * f[M_UZ] * f[M_UR], f[M_P] * f[M_DZZ],
                                  f[M_UZ] * f[M_SZR], f[M_SZR] * f[M_DRZ], f[M_SZT] * f[M_DTHZ],
                                  f[M_SZZ] * f[M_DZZ], f[M_UR] * f[M_UR] * f[M_UR], f[M_UR] * f[M_P],
                                  f[M_P] * f[M_DRR], f[M_UR] * f[M_SRR], f[M_SRR] * f[M_DRR],
                                  f[M_SRT] * f[M_DTHR], f[M_SZR] * f[M_DZR], f[M_UT] * f[M_UT] * f[M_UR],
                                  f[M_P] * f[M_DTHT], f[M_UT] * f[M_SRT], f[M_STT] * f[M_DTHT],
                                  f[M_SRT] * f[M_DRT], f[M_SZT] * f[M_DZT]};
            for (int k = 0; k < BQ; k++) atomicAdd(row + k, v[k]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.nbins * BQ; i += blockDim.x)
        a.part[(size_t)blockIdx.x * a.nbins * BQ + i] = sb[i];
}

// block sums -> bin means (fixed block order); cnt receives the counts
void bin_means(const std::vector<double> &hp, int nbins, std::vector<double> &mean, std::vector<double> &cnt,
               int count_col) {
    mean.assign((size_t)nbins * BQ, 0.0);
    if (count_col >= 0) cnt.assign(nbins, 0.0);
    for (int b = 0; b < nbins; b++) {
        double s[BQ] = {0};
        for (int blk = 0; blk < BUD_BLOCKS; blk++)
            for (int k = 0; k < BQ; k++) s[k] += hp[((size_t)blk * nbins + b) * BQ + k];
        if (count_col >= 0) cnt[b] = s[count_col];
        const double n = cnt[b];
        for (int k = 0; k < BQ; k++) mean[(size_t)b * BQ + k] = n > 0.0 ? s[k] / n : 0.0;
    }
}

template <int PASS>
cudaError_t budget_pass(Ctx &c, BudgetArgs &a, int nbins, std::vector<double> &hp) {
    count_launch(c, G_STATS);
    budget_kernel<PASS><<<BUD_BLOCKS, BUD_TB, sizeof(double) * nbins * BQ, c.stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    hp.resize((size_t)BUD_BLOCKS * nbins * BQ);
    if ((e = cudaMemcpyAsync(hp.data(), a.part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, c.stream)) !=
        cudaSuccess)
        return e;
    return cudaStreamSynchronize(c.stream);
}

}  // namespace

size_t tke_budget_scratch_bytes(int nbins) { return sizeof(double) * ((size_t)BUD_BLOCKS + 1) * nbins * BQ; }


// scratch: the population buffer that the next step overwrites (block sums,
// then the bin means of pass 1)
cudaError_t run_tke_budget(Ctx &c, int flags, int nbins, double *out) {
    cudaError_t e;
    if ((e = launch_macro(c, 0)) != cudaSuccess) return e;
    const int ibm = c.armed_bc == LBM_BC_IBM_U || c.armed_bc == LBM_BC_IBM_B;
    if (!(ibm && (flags & LBM_STATS_UNMASK)))
        if ((e = launch_mask(c)) != cudaSuccess) return e;
    BudgetArgs a{c.u_f, c.rho_f, c.flags, nullptr, (double *)c.fB, c.nx, c.ny, c.nz, c.N,
                 c.pipe_cx, c.pipe_cy, c.pipe_R, nbins};
    double *dmean = a.part + (size_t)BUD_BLOCKS * nbins * BQ;
    std::vector<double> hp, mean, prod, cnt;
    if ((e = budget_pass<1>(c, a, nbins, hp)) != cudaSuccess) return e;
    bin_means(hp, nbins, mean, cnt, M_ONE);
    if ((e = cudaMemcpyAsync(dmean, mean.data(), sizeof(double) * mean.size(), cudaMemcpyHostToDevice, c.stream)) !=
        cudaSuccess)
        return e;
    a.mean = dmean;
    if ((e = budget_pass<2>(c, a, nbins, hp)) != cudaSuccess) return e;
    bin_means(hp, nbins, prod, cnt, -1);

    // radial derivative over the bin centres r_b = (b + 1/2) R / nbins:
    // central differences, one-sided at the first and last bins
    const int n = nbins;
    const double R = c.pipe_R, h = R / n, nu = (c.tau - 0.5) / 3.0;
    std::vector<double> rb(n);
    for (int b = 0; b < n; b++) rb[b] = ((b + 0.5) * R) / n;
    auto ddr = [&](const std::vector<double> &F) {
        std::vector<double> g(n, 0.0);
        if (n > 1) {
            g[0] = (F[1] - F[0]) / h;
            g[n - 1] = (F[n - 1] - F[n - 2]) / h;
            for (int b = 1; b < n - 1; b++) g[b] = (F[b + 1] - F[b - 1]) / (2.0 * h);
        }
        return g;
    };
    auto div_r = [&](const std::vector<double> &F) {  // (1/r) d/dr (r F)
        std::vector<double> rF(n);
        for (int b = 0; b < n; b++) rF[b] = rb[b] * F[b];
        std::vector<double> g = ddr(rF);
        for (int b = 0; b < n; b++) g[b] /= rb[b];
        return g;
    };
    auto pm = [&](int k, double f) {  // f times a pass-2 column
        std::vector<double> v(n);
        for (int b = 0; b < n; b++) v[b] = f * prod[(size_t)b * BQ + k];
        return v;
    };
    auto P = [&](int b, int k) { return prod[(size_t)b * BQ + k]; };
    std::vector<double> uz_mean(n);
    for (int b = 0; b < n; b++) uz_mean[b] = mean[(size_t)b * BQ + M_UZ];
    const std::vector<double> dUz = ddr(uz_mean), Tz = div_r(pm(P_ZZR, 0.5)), Vz = div_r(pm(P_Z_SZR, 1.0)),
                              Tr = div_r(pm(P_RRR, 0.5)), dRP = ddr(pm(P_R_P, 1.0)), Vr = div_r(pm(P_R_SRR, 1.0)),
                              Tt = div_r(pm(P_TTR, 0.5)), Vt = div_r(pm(P_T_SRT, 1.0));
    for (int b = 0; b < n; b++) {
        double *o = out + (size_t)b * LBM_BUDGET_NT;
        o[0] = cnt[b];
        if (!(cnt[b] > 0.0)) {
            for (int k = 1; k < LBM_BUDGET_NT; k++) o[k] = 0.0;
            continue;
        }
        o[1] = -P(b, P_ZR) * dUz[b];
        o[2] = -Tz[b];
        o[3] = P(b, P_P_DZZ);
        o[4] = 2.0 * nu * Vz[b];
        o[5] = -2.0 * nu * (P(b, P_SZR_DRZ) + P(b, P_SZT_DTHZ) + P(b, P_SZZ_DZZ));
        o[6] = -Tr[b];
        o[7] = -dRP[b] + P(b, P_P_DRR);
        o[8] = 2.0 * nu * Vr[b];
        o[9] = -2.0 * nu * (P(b, P_SRR_DRR) + P(b, P_SRT_DTHR) + P(b, P_SZR_DZR));
        o[10] = -Tt[b];
        o[11] = P(b, P_P_DTHT);
        o[12] = 2.0 * nu * Vt[b];
        o[13] = -2.0 * nu * (P(b, P_STT_DTHT) + P(b, P_SRT_DRT) + P(b, P_SZT_DZT));
    }
    return cudaSuccess;
}

}  // namespace lbmgb
