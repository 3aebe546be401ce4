// Device definitions of the GB300 lattice Boltzmann library: D3Q19
// constants, population storage formats, the collision operators and small
// helpers shared by the sweep kernels. The method is the D3Q19 MRT LBM with
// Guo forcing of Peng et al., arXiv:1906.05448 (Sec. 2.1, Sec. 3.1); see
// lbm.h for the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "lbm.h"

namespace lbmgb {

// ---------------------------------------------------------------- flags ----
enum : uint8_t {
    FL_SOLID = 1,     // inside a particle / outside the pipe
    FL_BND = 2,       // IBB: fluid cell with at least one boundary link (sites list)
    FL_SUP = 4,       // IBM: cell handled by the compact forcing path
    FL_WAS_SOLID = 8, // transient during a geometry update
};

constexpr int NO_OWNER = 0x7fffffff;

// --------------------------------------------------------------- D3Q19 -----
// Velocity order (same as lbm.h): rest, +-x, +-y, +-z, then the edges in
// (+,+)/(-,-), (+,-)/(-,+) pairs for xy, xz, yz. Opposites are adjacent.
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr double wgt(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

// ------------------------------------------------------------- storage -----
// Populations are stored shifted, g_i = f_i - w_i, which keeps the stored
// numbers small and the rounding of the stored state well below that of f.
template <int S> struct Store;
template <> struct Store<LBM_F64> {
    typedef double T;
    typedef double R;  // arithmetic type
    static __device__ __forceinline__ double ld(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(T *p, double v) { *p = v; }
};
#ifndef LBM_STORE_CS
#define LBM_STORE_CS 0
#endif
template <> struct Store<LBM_F32> {
    typedef float T;
    typedef float R;
    static __device__ __forceinline__ float ld(const T *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(T *p, float v) {
        if (LBM_STORE_CS) __stcs(p, v);
        else *p = v;
    }
};
// FP16 holds g * 2^10 so that small departures from w_i stay normal numbers.
constexpr float F16_SCALE = 1024.0f;
template <> struct Store<LBM_F16S> {
    typedef __half T;
    typedef float R;
    static __device__ __forceinline__ float ld(const T *p) {
        return __half2float(__ldg(p)) * (1.0f / F16_SCALE);
    }
    static __device__ __forceinline__ void st(T *p, float v) { *p = __float2half_rn(v * F16_SCALE); }
    // the stored number itself (g * 2^10); the scale is a power of two, so
    // arithmetic on scaled numbers rounds exactly as on unscaled ones
    static __device__ __forceinline__ float ld_scaled(const T *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void st_scaled(T *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Store<LBM_BF16S> {
    typedef __nv_bfloat16 T;
    typedef float R;
    static __device__ __forceinline__ float ld(const T *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ void st(T *p, float v) { *p = __float2bfloat16_rn(v); }
};

inline size_t storage_bytes(int s) { return s == LBM_F64 ? 8 : (s == LBM_F32 ? 4 : 2); }

// Unsigned 32-bit division by a run-time constant with a multiply-high and
// shifts (Granlund & Montgomery 1994), valid for every 32-bit dividend.
struct FastDiv {
    unsigned d, m, s;
    __host__ __device__ FastDiv() : d(1), m(0), s(0) {}
    __host__ __device__ explicit FastDiv(unsigned dd) : d(dd) {
        unsigned l = 0;
        while ((1ull << l) < dd) l++;
        s = l;
        m = (unsigned)((((1ull << l) - dd) << 32) / dd + 1);
    }
    __host__ __device__ __forceinline__ unsigned div(unsigned n) const {
#ifdef __CUDA_ARCH__
        const unsigned t = __umulhi(n, m);
#else
        const unsigned t = (unsigned)(((unsigned long long)n * m) >> 32);
#endif
        return s == 0 ? n : (t + ((n - t) >> 1)) >> (s - 1);
    }
};

// t -> (ix, iy, iz) in a w x w x w box, x fastest (two multiply-shift
// divisions instead of integer division)
__device__ __forceinline__ void box_coords(int t, const FastDiv &fw, int w, int &ix, int &iy, int &iz) {
    const unsigned q1 = fw.div((unsigned)t), q2 = fw.div(q1);
    ix = t - (int)q1 * w;
    iy = (int)q1 - (int)q2 * w;
    iz = (int)q2;
}

// ------------------------------------------------------------ collision ----
struct Rates {
    float s_e, s_eps, s_q, s_nu, s_pi, s_m;  // d'Humieres groups (s_nu = 1/tau)
    double d_e, d_eps, d_q, d_nu, d_pi, d_m;
};

// Guo forcing term F_i = w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F.
template <typename R>
__host__ __device__ __forceinline__ R guo_term(int i, R ux, R uy, R uz, R Fx, R Fy, R Fz) {
    const R cu = R(cx(i)) * ux + R(cy(i)) * uy + R(cz(i)) * uz;
    const R a = (R(cx(i)) - ux) * Fx + (R(cy(i)) - uy) * Fy + (R(cz(i)) - uz) * Fz;
    const R b = R(cx(i)) * Fx + R(cy(i)) * Fy + R(cz(i)) * Fz;
    return R(wgt(i)) * (R(3) * a + R(9) * cu * b);
}

// BGK + Guo factors per weight class (rest, axis, edge) and direction, in
// the pair form, with the forcing folded into the departure (divided by
// omega); factors that scale populations carry the storage scale 2^SC.
struct PairK {
    float om;       // omega
    float q[2];     // 4.5 w (axis, edge)                 [x rho per cell]
    float t[2];     // 3 w (axis, edge), with 2 t_axis + 8 t_edge = 1 exactly  [x c_i.j']
    float w[3];     // w (rest, axis, edge)               [x (drho - 1.5 rho u^2)]
    float cw[3];    // (1 - omega/2) w / omega            [x 3 u.F]
    float K[19];    // 3 (1 - omega/2) w c_i.F / omega + t_i c_i.F / 2 (the force's share of the odd equilibrium)
    float L[19];    // 9 (1 - omega/2) w c_i.F / omega
    float hF[3];    // F / 2 (unscaled)
    float F3[3];    // 3 F (unscaled)
};

inline PairK make_pair_k(double omega, const double F[3]) {
    PairK k;
    const double c1 = (1.0 - 0.5 * omega) / omega;
    const double wcls[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    k.om = (float)omega;
    for (int j = 0; j < 2; j++) k.q[j] = (float)(4.5 * wcls[j + 1]);
    // 3 w in FP32 with the x-momentum sum 2 t_axis + 8 t_edge exactly 1, so
    // that the odd equilibrium part carries exactly the momentum j'
    k.t[1] = (float)(1.0 / 12.0);
    k.t[0] = (float)((1.0 - 8.0 * (double)k.t[1]) / 2.0);  // exact: 5592405 / 2^25
    for (int j = 0; j < 3; j++) {
        k.w[j] = (float)wcls[j];
        k.cw[j] = (float)(c1 * wcls[j]);
    }
    for (int i = 0; i < 19; i++) {
        const double cF = cx(i) * F[0] + cy(i) * F[1] + cz(i) * F[2];
        const double ti = i == 0 ? 0.0 : (double)k.t[i <= 6 ? 0 : 1];
        k.K[i] = (float)(3.0 * c1 * wgt(i) * cF + 0.5 * ti * cF);
        k.L[i] = (float)(9.0 * c1 * wgt(i) * cF);
    }
    for (int d = 0; d < 3; d++) {
        k.hF[d] = (float)(0.5 * F[d]);
        k.F3[d] = (float)(3.0 * F[d]);
    }
    return k;
}

// BGK + Guo on one cell over opposite pairs, g in/out (x 2^SC); returns rho
// and |u|^2. The new value is g + omega d with the departure
// d_i = g_eq,i + F_i / omega - g_i formed at its own (small) scale and
// rounded into g once. Two choices keep FP32 rounding from accumulating in
// a near-steady flow, where the same rounding recurs every step:
// - the odd equilibrium part 3 w_i c_i.(rho u) = 3 w_i c_i.(j + F/2) is
//   taken from the momentum j itself with FP32 factors whose momentum sum
//   is exactly 1, so the equilibrium carries exactly the cell's momentum
//   (with the rounded factors 3 w and rho u = rho (j'/rho), every collision
//   would add about 3e-8 of it); the force's share 3 w_i c_i.F/2 is a
//   per-direction constant (adding F/2 to j in FP32 would keep only a few
//   bits of a small force);
// - that odd part is subtracted from g_i in one fused step (it nearly
//   cancels g_i's odd part), and the even part and forcing are added to
//   the small remainder.
template <bool FORCE, int SC>
__device__ __forceinline__ void collide_pairs(float g[19], const PairK &k, float &rho_o, float &u2_o) {
    constexpr float down = 1.0f / float(1u << SC), up = float(1u << SC);
    const float s1 = g[1] + g[2], d1 = g[1] - g[2], s3 = g[3] + g[4], d3 = g[3] - g[4];
    const float s5 = g[5] + g[6], d5 = g[5] - g[6], s7 = g[7] + g[8], d7 = g[7] - g[8];
    const float s9 = g[9] + g[10], d9 = g[9] - g[10], s11 = g[11] + g[12], d11 = g[11] - g[12];
    const float s13 = g[13] + g[14], d13 = g[13] - g[14], s15 = g[15] + g[16], d15 = g[15] - g[16];
    const float s17 = g[17] + g[18], d17 = g[17] - g[18];
    float drho = g[0] + ((s1 + s3) + s5) + ((s7 + s9) + (s11 + s13)) + (s15 + s17);
    // momentum j at the scale of g; the Guo velocity is u = (j + F/2) / rho
    const float jx = d1 + (d7 + d9) + (d11 + d13);
    const float jy = d3 + (d7 - d9) + (d15 + d17);
    const float jz = d5 + (d11 - d13) + (d15 - d17);
    if (SC != 0) drho *= down;
    const float rho = 1.0f + drho;
    const float ir = __frcp_rn(rho) * down;
    const float ux = (FORCE ? fmaf(k.hF[0], up, jx) : jx) * ir;
    const float uy = (FORCE ? fmaf(k.hF[1], up, jy) : jy) * ir;
    const float uz = (FORCE ? fmaf(k.hF[2], up, jz) : jz) * ir;
    const float u2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    rho_o = rho;
    u2_o = u2;
    const float Bv = fmaf(-1.5f * rho, u2, drho);
    const float uF3 = FORCE ? fmaf(ux, k.F3[0], fmaf(uy, k.F3[1], uz * k.F3[2])) : 0.0f;
    // even part of the departure without its 4.5 w rho (c.u)^2 and L c.u terms, per class (x 2^SC)
    const float b0 = (FORCE ? fmaf(k.w[0], Bv, -k.cw[0] * uF3) : k.w[0] * Bv) * up;
    const float b1 = (FORCE ? fmaf(k.w[1], Bv, -k.cw[1] * uF3) : k.w[1] * Bv) * up;
    const float b2 = (FORCE ? fmaf(k.w[2], Bv, -k.cw[2] * uF3) : k.w[2] * Bv) * up;
    const float q1 = k.q[0] * rho * up, q2 = k.q[1] * rho * up;
    const float t1 = k.t[0], t2 = k.t[1];
    const float om = k.om;
    g[0] = fmaf(om, b0 - g[0], g[0]);
    // even part E = q (c.u)^2 + L c.u + b, odd part t c.j + K
    auto pair = [&](int i, float cu, float cj, float q, float t, float b) {
        const float E = FORCE ? fmaf(fmaf(q, cu, k.L[i] * up), cu, b) : fmaf(q * cu, cu, b);
        const float Ki = FORCE ? k.K[i] * up : 0.0f;
        const float hi = fmaf(t, cj, -g[i]), hb = fmaf(-t, cj, -g[i + 1]);
        g[i] = fmaf(om, (E + Ki) + hi, g[i]);
        g[i + 1] = fmaf(om, (E - Ki) + hb, g[i + 1]);
    };
    pair(1, ux, jx, q1, t1, b1);
    pair(3, uy, jy, q1, t1, b1);
    pair(5, uz, jz, q1, t1, b1);
    pair(7, ux + uy, jx + jy, q2, t2, b2);
    pair(9, ux - uy, jx - jy, q2, t2, b2);
    pair(11, ux + uz, jx + jz, q2, t2, b2);
    pair(13, ux - uz, jx - jz, q2, t2, b2);
    pair(15, uy + uz, jy + jz, q2, t2, b2);
    pair(17, uy - uz, jy - jz, q2, t2, b2);
}

// Collide one cell in place. g: shifted populations in, post-collision out.
// F: total force on the cell. Returns rho and u = (sum f c + F/2)/rho.
// The moment transform is the d'Humieres D3Q19 basis evaluated through
// opposite-pair sums (even moments) and differences (odd moments); the
// inverse uses the orthogonality of the basis (row norms below).
template <typename R, bool FORCE, bool SRT>
__host__ __device__ __forceinline__ void collide(R g[19], R Fx, R Fy, R Fz, const Rates &rt, R &rho_o, R &ux_o,
                                                 R &uy_o, R &uz_o) {
    R drho = g[0];
#pragma unroll
    for (int i = 1; i < 19; i++) drho += g[i];
    R jx = (g[1] - g[2]) + (g[7] - g[8]) + (g[9] - g[10]) + (g[11] - g[12]) + (g[13] - g[14]);
    R jy = (g[3] - g[4]) + (g[7] - g[8]) - (g[9] - g[10]) + (g[15] - g[16]) + (g[17] - g[18]);
    R jz = (g[5] - g[6]) + (g[11] - g[12]) - (g[13] - g[14]) + (g[15] - g[16]) - (g[17] - g[18]);
    const R rho = R(1) + drho;
    const R irho = R(1) / rho;
    const R jx0 = jx, jy0 = jy, jz0 = jz;  // momentum without the force's half (odd equilibrium part)
    if (FORCE) {
        jx += R(0.5) * Fx;
        jy += R(0.5) * Fy;
        jz += R(0.5) * Fz;
    }
    const R ux = jx * irho, uy = jy * irho, uz = jz * irho;
    rho_o = rho;
    ux_o = ux;
    uy_o = uy;
    uz_o = uz;
    const R uxx = ux * ux, uyy = uy * uy, uzz = uz * uz, u2 = uxx + uyy + uzz;
    if constexpr (SRT) {
        // BGK: g* = g + om d, d_i = g_eq,i + F_i / om - g_i with g_eq = f_eq - w
        // and F_i = (1 - om/2) w_i [3 c_i.F - 3 u.F + 9 (c_i.u)(c_i.F)], over
        // opposite pairs. The odd equilibrium part 3 w rho c_i.u, which nearly
        // cancels the odd part of g_i, is subtracted from g_i in one fused
        // step and d is rounded into g once (see collide_pairs).
        const R om = (sizeof(R) == 8) ? R(rt.d_nu) : R(rt.s_nu);
        const R c1 = (R(1) - R(0.5) * om) / om;
        const R Bv = drho - rho * R(1.5) * u2;
        const R uF3 = FORCE ? R(3) * (ux * Fx + uy * Fy + uz * Fz) : R(0);
        const R wr[3] = {R(1.0 / 3.0), R(1.0 / 18.0), R(1.0 / 36.0)};
        // odd part 3 w c.(j + F/2): t c.j with factors whose momentum sum
        // is exactly 1, and the force's share t c.F/2 beside it (see collide_pairs)
        const R tE = R(1.0 / 12.0), tA = sizeof(R) == 8 ? R(1.0 / 6.0) : R((1.0 - 8.0 * (double)float(1.0 / 12.0)) / 2.0);
        g[0] = g[0] + om * ((wr[0] * Bv - c1 * wr[0] * uF3) - g[0]);
        auto pair = [&](int i, R cu, R cj, R cF, int cls) {
            const R w = wr[cls];
            const R E = w * (Bv + R(4.5) * rho * cu * cu) + (FORCE ? c1 * w * (R(9) * cu * cF - uF3) : R(0));
            const R t = cls == 1 ? tA : tE;
            const R K = FORCE ? R(3) * c1 * w * cF + R(0.5) * t * cF : R(0);
            const R hi = fma(t, cj, -g[i]), hb = fma(-t, cj, -g[i + 1]);
            g[i] = fma(om, (E + K) + hi, g[i]);
            g[i + 1] = fma(om, (E - K) + hb, g[i + 1]);
        };
        pair(1, ux, jx0, Fx, 1);
        pair(3, uy, jy0, Fy, 1);
        pair(5, uz, jz0, Fz, 1);
        pair(7, ux + uy, jx0 + jy0, Fx + Fy, 2);
        pair(9, ux - uy, jx0 - jy0, Fx - Fy, 2);
        pair(11, ux + uz, jx0 + jz0, Fx + Fz, 2);
        pair(13, ux - uz, jx0 - jz0, Fx - Fz, 2);
        pair(15, uy + uz, jy0 + jz0, Fy + Fz, 2);
        pair(17, uy - uz, jy0 - jz0, Fy - Fz, 2);
    } else {
    // MRT: g* = g + F_i - M^-1 S (M (g + F_i/2) - (m_eq - M w)).
    R Fi[19];
    if (FORCE) {
#pragma unroll
        for (int i = 0; i < 19; i++) Fi[i] = guo_term<R>(i, ux, uy, uz, Fx, Fy, Fz);
    }
    R h[19];
#pragma unroll
    for (int i = 0; i < 19; i++) h[i] = FORCE ? g[i] + R(0.5) * Fi[i] : g[i];
    const R Sx = h[1] + h[2], Sy = h[3] + h[4], Sz = h[5] + h[6];
    const R Sa = h[7] + h[8], Sb = h[9] + h[10], Sc = h[11] + h[12], Sd = h[13] + h[14];
    const R Se = h[15] + h[16], Sf = h[17] + h[18];
    const R Dx = h[1] - h[2], Dy = h[3] - h[4], Dz = h[5] - h[6];
    const R Da = h[7] - h[8], Db = h[9] - h[10], Dc = h[11] - h[12], Dd = h[13] - h[14];
    const R De = h[15] - h[16], Df = h[17] - h[18];
    const R A = Sx + Sy + Sz;
    const R Exy = Sa + Sb, Exz = Sc + Sd, Eyz = Se + Sf;
    const R E = Exy + Exz + Eyz;
    const R pxx = R(2) * Sx - Sy - Sz + Exy + Exz - R(2) * Eyz;      // 3 p_xx
    const R pixx = R(-2) * (R(2) * Sx - Sy - Sz) + Exy + Exz - R(2) * Eyz;
    const R pww = Sy - Sz + Exy - Exz;
    const R piww = R(-2) * (Sy - Sz) + Exy - Exz;
    const R mee = R(-30) * h[0] - R(11) * A + R(8) * E;
    const R mep = R(12) * h[0] - R(4) * A + E;
    const R pxy = Sa - Sb, pyz = Se - Sf, pxz = Sc - Sd;
    const R qx = R(-4) * Dx + Da + Db + Dc + Dd;
    const R qy = R(-4) * Dy + Da - Db + De + Df;
    const R qz = R(-4) * Dz + Dc - Dd + De - Df;
    const R mx = (Da + Db) - (Dc + Dd);
    const R my = (De + Df) - (Da - Db);
    const R mz = (Dc - Dd) - (De - Df);
    // equilibrium moments minus those of w (rho = 1, u = 0)
    const R eq_e = R(-11) * drho + R(19) * rho * u2;
    const R eq_ep = R(3) * drho - R(5.5) * rho * u2;
    const R tx = R(2) * uxx - uyy - uzz;
    const R eq_pxx = rho * tx, eq_pixx = R(-0.5) * rho * tx;
    const R eq_pww = rho * (uyy - uzz), eq_piww = R(-0.5) * rho * (uyy - uzz);
    const R eq_q = R(-2.0 / 3.0) * rho;
    const bool dbl = sizeof(R) == 8;
    const R se = dbl ? R(rt.d_e) : R(rt.s_e), sep = dbl ? R(rt.d_eps) : R(rt.s_eps);
    const R sq = dbl ? R(rt.d_q) : R(rt.s_q), snu = dbl ? R(rt.d_nu) : R(rt.s_nu);
    const R spi = dbl ? R(rt.d_pi) : R(rt.s_pi), sm = dbl ? R(rt.d_m) : R(rt.s_m);
    // relaxed departures divided by the squared row norms of the basis
    const R a_e = se * (mee - eq_e) * R(1.0 / 2394.0);
    const R a_ep = sep * (mep - eq_ep) * R(1.0 / 252.0);
    const R a_pxx = snu * (pxx - eq_pxx) * R(1.0 / 36.0);
    const R a_pixx = spi * (pixx - eq_pixx) * R(1.0 / 72.0);
    const R a_pww = snu * (pww - eq_pww) * R(1.0 / 12.0);
    const R a_piww = spi * (piww - eq_piww) * R(1.0 / 24.0);
    const R a_pxy = snu * (pxy - rho * ux * uy) * R(0.25);
    const R a_pyz = snu * (pyz - rho * uy * uz) * R(0.25);
    const R a_pxz = snu * (pxz - rho * ux * uz) * R(0.25);
    const R a_qx = sq * (qx - eq_q * ux) * R(1.0 / 40.0);
    const R a_qy = sq * (qy - eq_q * uy) * R(1.0 / 40.0);
    const R a_qz = sq * (qz - eq_q * uz) * R(1.0 / 40.0);
    const R a_mx = sm * mx * R(0.125), a_my = sm * my * R(0.125), a_mz = sm * mz * R(0.125);
    // back-transform: even and odd parts per opposite pair
    const R c0 = R(-30) * a_e + R(12) * a_ep;
    const R ax = R(-11) * a_e - R(4) * a_ep;                 // common to the 6 axis directions
    const R ed = R(8) * a_e + a_ep;                          // common to the 12 edges
    const R evx = ax + R(2) * a_pxx - R(4) * a_pixx;
    const R evy = ax - a_pxx + R(2) * a_pixx + a_pww - R(2) * a_piww;
    const R evz = ax - a_pxx + R(2) * a_pixx - a_pww + R(2) * a_piww;
    const R exy = ed + a_pxx + a_pixx + a_pww + a_piww;
    const R exz = ed + a_pxx + a_pixx - a_pww - a_piww;
    const R eyz = ed - R(2) * a_pxx - R(2) * a_pixx;
    const R evA = exy + a_pxy, evB = exy - a_pxy;
    const R evC = exz + a_pxz, evD = exz - a_pxz;
    const R evE = eyz + a_pyz, evF = eyz - a_pyz;
    const R odx = R(-4) * a_qx, ody = R(-4) * a_qy, odz = R(-4) * a_qz;
    const R odA = a_qx + a_qy + a_mx - a_my;
    const R odB = a_qx - a_qy + a_mx + a_my;
    const R odC = a_qx + a_qz - a_mx + a_mz;
    const R odD = a_qx - a_qz - a_mx - a_mz;
    const R odE = a_qy + a_qz + a_my - a_mz;
    const R odF = a_qy - a_qz + a_my + a_mz;
    R corr[19];
    corr[0] = c0;
    corr[1] = evx + odx;  corr[2] = evx - odx;
    corr[3] = evy + ody;  corr[4] = evy - ody;
    corr[5] = evz + odz;  corr[6] = evz - odz;
    corr[7] = evA + odA;  corr[8] = evA - odA;
    corr[9] = evB + odB;  corr[10] = evB - odB;
    corr[11] = evC + odC; corr[12] = evC - odC;
    corr[13] = evD + odD; corr[14] = evD - odD;
    corr[15] = evE + odE; corr[16] = evE - odE;
    corr[17] = evF + odF; corr[18] = evF - odF;
#pragma unroll
    for (int i = 0; i < 19; i++) g[i] = FORCE ? g[i] + Fi[i] - corr[i] : g[i] - corr[i];
    }
}

// Single-node bounce-back, the last fallback of the scheme chain (Sec. 3.1,
// after Zhao & Yong 2017; the formula is a reading): halfway bounce-back
// plus (1 - 2q)/2 (d_l + d_ibar), where d = M^-1 S (m - m_eq) is the
// departure the collision at the boundary node x_f removed. It is recovered
// from the node's post-collision populations alone, moment by moment:
//   S (m - m_eq) = S (I - S)^-1 (m~ - m_eq - (I - S/2) M F_i),
// with rho and u = (sum f c - F/2)/rho those of that collision. Rates of 0
// or exactly 1 contribute nothing. Odd moments cancel in d_l + d_ibar, so
// only the even ones are formed. p: the 19 stored values of x_f, population
// k at p[k * stride]. Returns d_l + d_ibar.
template <int S>
__device__ __noinline__ typename Store<S>::R single_node_pair(const typename Store<S>::T *p, size_t stride, int l,
                                                              typename Store<S>::R Fx, typename Store<S>::R Fy,
                                                              typename Store<S>::R Fz, const Rates &rt) {
    typedef typename Store<S>::R R;
    R g[19];
#pragma unroll
    for (int k = 0; k < 19; k++) g[k] = Store<S>::ld(p + k * stride);
    R drho = g[0];
#pragma unroll
    for (int k = 1; k < 19; k++) drho += g[k];
    const R jx = (g[1] - g[2]) + (g[7] - g[8]) + (g[9] - g[10]) + (g[11] - g[12]) + (g[13] - g[14]);
    const R jy = (g[3] - g[4]) + (g[7] - g[8]) - (g[9] - g[10]) + (g[15] - g[16]) + (g[17] - g[18]);
    const R jz = (g[5] - g[6]) + (g[11] - g[12]) - (g[13] - g[14]) + (g[15] - g[16]) - (g[17] - g[18]);
    const R rho = R(1) + drho, ir = R(1) / rho;
    const R ux = (jx - R(0.5) * Fx) * ir, uy = (jy - R(0.5) * Fy) * ir, uz = (jz - R(0.5) * Fz) * ir;
    R Fi[19];
#pragma unroll
    for (int k = 0; k < 19; k++) Fi[k] = guo_term<R>(k, ux, uy, uz, Fx, Fy, Fz);
    // even d'Humieres moments (e, eps, 3p_xx, 3pi_xx, p_ww, pi_ww, p_xy, p_yz, p_xz) of h
    auto even = [](const R *h, R *m) {
        const R Sx = h[1] + h[2], Sy = h[3] + h[4], Sz = h[5] + h[6];
        const R Sa = h[7] + h[8], Sb = h[9] + h[10], Sc = h[11] + h[12], Sd = h[13] + h[14];
        const R Se = h[15] + h[16], Sf = h[17] + h[18];
        const R A = Sx + Sy + Sz, Exy = Sa + Sb, Exz = Sc + Sd, Eyz = Se + Sf, E = Exy + Exz + Eyz;
        m[0] = R(-30) * h[0] - R(11) * A + R(8) * E;
        m[1] = R(12) * h[0] - R(4) * A + E;
        m[2] = R(2) * Sx - Sy - Sz + Exy + Exz - R(2) * Eyz;
        m[3] = R(-2) * (R(2) * Sx - Sy - Sz) + Exy + Exz - R(2) * Eyz;
        m[4] = Sy - Sz + Exy - Exz;
        m[5] = R(-2) * (Sy - Sz) + Exy - Exz;
        m[6] = Sa - Sb;
        m[7] = Se - Sf;
        m[8] = Sc - Sd;
    };
    R m[9], mF[9];
    even(g, m);
    even(Fi, mF);
    // equilibrium moments minus those of w
    const R uxx = ux * ux, uyy = uy * uy, uzz = uz * uz, u2 = uxx + uyy + uzz, tx = R(2) * uxx - uyy - uzz;
    const R eq[9] = {R(-11) * drho + R(19) * rho * u2, R(3) * drho - R(5.5) * rho * u2, rho * tx, R(-0.5) * rho * tx,
                     rho * (uyy - uzz), R(-0.5) * rho * (uyy - uzz), rho * ux * uy, rho * uy * uz, rho * ux * uz};
    const bool dbl = sizeof(R) == 8;
    const R se = dbl ? R(rt.d_e) : R(rt.s_e), sep = dbl ? R(rt.d_eps) : R(rt.s_eps);
    const R snu = dbl ? R(rt.d_nu) : R(rt.s_nu), spi = dbl ? R(rt.d_pi) : R(rt.s_pi);
    const R s[9] = {se, sep, snu, spi, snu, spi, snu, snu, snu};
    const R norm[9] = {R(1.0 / 2394.0), R(1.0 / 252.0), R(1.0 / 36.0), R(1.0 / 72.0), R(1.0 / 12.0),
                       R(1.0 / 24.0), R(0.25), R(0.25), R(0.25)};
    R a[9];
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const R f = (s[k] == R(0) || s[k] == R(1)) ? R(0) : s[k] / (R(1) - s[k]);
        a[k] = f * (m[k] - eq[k] - (R(1) - R(0.5) * s[k]) * mF[k]) * norm[k];
    }
    // even part of the back-transform for the pair (l, ibar)
    const R ax = R(-11) * a[0] - R(4) * a[1];
    const R ed = R(8) * a[0] + a[1];
    R ev;
    switch ((l + 1) >> 1) {
    case 1: ev = ax + R(2) * a[2] - R(4) * a[3]; break;
    case 2: ev = ax - a[2] + R(2) * a[3] + a[4] - R(2) * a[5]; break;
    case 3: ev = ax - a[2] + R(2) * a[3] - a[4] + R(2) * a[5]; break;
    case 4: ev = ed + a[2] + a[3] + a[4] + a[5] + a[6]; break;
    case 5: ev = ed + a[2] + a[3] + a[4] + a[5] - a[6]; break;
    case 6: ev = ed + a[2] + a[3] - a[4] - a[5] + a[8]; break;
    case 7: ev = ed + a[2] + a[3] - a[4] - a[5] - a[8]; break;
    case 8: ev = ed - R(2) * a[2] - R(2) * a[3] + a[7]; break;
    default: ev = ed - R(2) * a[2] - R(2) * a[3] - a[7]; break;
    }
    return R(2) * ev;
}

// ------------------------------------------------------------- helpers ----
// body force component in the arithmetic type R
template <typename R, typename Args>
__device__ __forceinline__ R body_force(const Args &a, int d) {
    if constexpr (sizeof(R) == 8)
        return R(a.F[d]);
    else
        return R(a.Fs[d]);
}

template <typename R>
__device__ __forceinline__ void watchdog(R rho, R ux, R uy, R uz, unsigned *status) {
    const R u2 = ux * ux + uy * uy + uz * uz;
    if (!(rho > R(0.5) && rho < R(2) && u2 < R(0.09))) atomicOr(status, 1u);
}

}  // namespace lbmgb
