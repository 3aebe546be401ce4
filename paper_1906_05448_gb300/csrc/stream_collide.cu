// Boundary and IBM collision kernels around the sweep (sweep.cu).
//
// ibb_links: one thread per boundary link (x_f, l), x_f + c_l solid. It
//   evaluates the interpolated bounce-back (Bouzidi et al. 2001 quadratic /
//   linear, single-node fallback; Sec. 3.1, Sec. 2.1) from post-collision
//   values and stores the result in the solid node's slot of the population
//   that streams back into x_f -- the layer of nodes outside the wall that
//   holds the bounced populations (Sec. 2.1) -- so the sweep pulls it like
//   any other population. It also records the Galilean-invariant momentum
//   exchange of the link (Wen et al. 2014, Sec. 3.1).
// ibm_collide: collides support cells with the body force plus the IBM force
//   accumulated over the forcing passes.
// Population transfer and equilibrium initialisation kernels.

#include "lbm_internal.cuh"

#include <algorithm>

namespace lbmgb {

__device__ __forceinline__ double mimg(double d, int n) {
    if (d > 0.5 * n) d -= n;
    else if (d < -0.5 * n) d += n;
    return d;
}
__device__ __forceinline__ int wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// Population bounced back into the fluid node x_f along ibar = opp(l) at time
// t + 1 from post-collision values at t (Sec. 2.1): quadratic (sch 0) or
// linear (sch 1) interpolated bounce-back, split at q = 1/2, or the halfway
// rule (sch 2, to which the callers add the single-node correction of
// single_node_pair) where the interpolation nodes are not fluid. fl0 = f*_l(x_f),
// fi0 = f*_ibar(x_f); c1 = x_f - c_l, c2 = x_f - 2 c_l; D = moving-wall term.
template <int S>
__device__ __forceinline__ typename Store<S>::R ibb_value(const typename Store<S>::T *A, size_t N, int l, int i,
                                                          int sch, typename Store<S>::R qq, int c1, int c2,
                                                          typename Store<S>::R D, typename Store<S>::R fl0,
                                                          typename Store<S>::R fi0) {
    typedef typename Store<S>::R R;
    R v;
    if (sch == 0) {
        if (qq < R(0.5)) {
            const R fl1 = Store<S>::ld(A + (size_t)l * N + c1), fl2 = Store<S>::ld(A + (size_t)l * N + c2);
            v = qq * (R(1) + R(2) * qq) * fl0 + (R(1) - R(4) * qq * qq) * fl1 - qq * (R(1) - R(2) * qq) * fl2 + D;
        } else {
            const R fi1 = Store<S>::ld(A + (size_t)i * N + c1);
            const R d = R(1) / (qq * (R(2) * qq + R(1)));
            v = d * fl0 + (R(2) * qq - R(1)) / qq * fi0 - (R(2) * qq - R(1)) / (R(2) * qq + R(1)) * fi1 + d * D;
        }
    } else if (sch == 1) {
        if (qq < R(0.5)) {
            const R fl1 = Store<S>::ld(A + (size_t)l * N + c1);
            v = R(2) * qq * fl0 + (R(1) - R(2) * qq) * fl1 + D;
        } else {
            const R h = R(1) / (R(2) * qq);
            v = h * fl0 + (R(2) * qq - R(1)) * h * fi0 + h * D;
        }
    } else {
        v = fl0 + D;
    }
    return v;
}

// ------------------------------------------------------------ IBB links ----
struct LinkArgs {
    void *A;  // post-collision populations at t; ghost slots of solid nodes are written
    const int *link_cell, *link_pid;
    const int8_t *link_dir, *link_scheme;
    const double *link_q;
    void *link_dP, *link_dT;  // per-link momentum exchange and torque (arithmetic type of the storage)
    const double *X, *U, *W;
    const long long *counts;  // [1]: number of links (device)
    long long max_links;
    int nx, ny, nz;
    long long N;
    FastDiv dx, dxy;  // division by nx and nx*ny
    double F[3];      // body force on fluid cells (single-node fallback)
    float Fs[3];
    Rates rt;
    const int *sn_list;  // single-node links (counts[4] of them)
};


// PART: some links belong to moving walls (particles); the pipe wall alone
// needs neither the wall velocity nor the momentum exchange
template <int S, bool PART>
__global__ void __launch_bounds__(256) ibb_links(LinkArgs a) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const long long nl = a.counts[1] < a.max_links ? a.counts[1] : a.max_links;
    T *A = (T *)a.A;
    const size_t N = (size_t)a.N;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < nl;
         k += (long long)gridDim.x * blockDim.x) {
        const int c = a.link_cell[k];
        const int l = a.link_dir[k];
        const int sch = a.link_scheme[k];
        const int pid = PART ? a.link_pid[k] : -1;
        const double q = a.link_q[k];
        const unsigned zq = a.dxy.div((unsigned)c), rem = (unsigned)c - zq * (unsigned)(nx * ny);
        const unsigned yq = a.dx.div(rem);
        const int z = (int)zq, y = (int)yq, x = (int)(rem - yq * (unsigned)nx);
        const int lx = cx(l), ly = cy(l), lz = cz(l);
        // solid node x_f + c_l, and fluid nodes x_f - c_l, x_f - 2 c_l
        const int cb = wrap(x + lx, nx) + nx * (wrap(y + ly, ny) + ny * wrap(z + lz, nz));
        const int x1 = wrap(x - lx, nx), y1 = wrap(y - ly, ny), z1 = wrap(z - lz, nz);
        const int c1 = x1 + nx * (y1 + ny * z1);
        const int c2 = wrap(x1 - lx, nx) + nx * (wrap(y1 - ly, ny) + ny * wrap(z1 - lz, nz));
        const int i = opp(l);
        const R fl0 = Store<S>::ld(A + (size_t)l * N + c);  // f*_l(x_f), toward the wall
        const R fi0 = Store<S>::ld(A + (size_t)i * N + c);  // f*_ibar(x_f)
        // scheme 2 stores the halfway value here; single_node_fix adds the
        // single-node correction (and its momentum) afterwards
        if constexpr (!PART) {
            const R v = ibb_value<S>(A, N, l, i, sch, R(q), c1, c2, R(0), fl0, fi0);
            Store<S>::st(A + (size_t)i * N + cb, v);  // pulled by x_f as f_ibar(x_f, t+1)
        } else if constexpr (sizeof(R) == 8) {
            // FP64 storage: wall velocity and momentum exchange in FP64
            double uw[3] = {0.0, 0.0, 0.0};
            if (pid >= 0) {
                const double r0 = mimg(x + q * lx - a.X[3 * pid + 0], nx);
                const double r1 = mimg(y + q * ly - a.X[3 * pid + 1], ny);
                const double r2 = mimg(z + q * lz - a.X[3 * pid + 2], nz);
                const double *Wp = a.W + 3 * pid, *Up = a.U + 3 * pid;
                uw[0] = Up[0] + (Wp[1] * r2 - Wp[2] * r1);
                uw[1] = Up[1] + (Wp[2] * r0 - Wp[0] * r2);
                uw[2] = Up[2] + (Wp[0] * r1 - Wp[1] * r0);
            }
            // moving-wall term 6 w rho_w (c_ibar . u_w), rho_w = 1; c_ibar = -c_l
            const R Dw = pid >= 0 ? R(-6.0 * wgt(l) * (lx * uw[0] + ly * uw[1] + lz * uw[2])) : R(0);
            const R v = ibb_value<S>(A, N, l, i, sch, R(q), c1, c2, Dw, fl0, fi0);
            Store<S>::st(A + (size_t)i * N + cb, v);
            if (pid >= 0) {
                // momentum exchange with unshifted f = g + w (w_l = w_ibar)
                const double fo = double(fl0) + wgt(l), fi = double(v) + wgt(i);
                const double dP0 = (lx - uw[0]) * fo - (-lx - uw[0]) * fi;
                const double dP1 = (ly - uw[1]) * fo - (-ly - uw[1]) * fi;
                const double dP2 = (lz - uw[2]) * fo - (-lz - uw[2]) * fi;
                const double m0 = mimg(x + 0.5 * lx - a.X[3 * pid + 0], nx);
                const double m1 = mimg(y + 0.5 * ly - a.X[3 * pid + 1], ny);
                const double m2 = mimg(z + 0.5 * lz - a.X[3 * pid + 2], nz);
                double *dP = (double *)a.link_dP + 3 * k, *dT = (double *)a.link_dT + 3 * k;
                dP[0] = dP0;
                dP[1] = dP1;
                dP[2] = dP2;
                dT[0] = m1 * dP2 - m2 * dP1;
                dT[1] = m2 * dP0 - m0 * dP2;
                dT[2] = m0 * dP1 - m1 * dP0;
            }
        } else {
            // 32- and 16-bit storage: the same in FP32 after one FP64
            // difference x_f - X_p per component (FP64 stays in the sums)
            float d[3] = {0.0f, 0.0f, 0.0f}, uw[3] = {0.0f, 0.0f, 0.0f};
            const float qf = float(q);
            if (pid >= 0) {
                d[0] = float(mimg(double(x) - a.X[3 * pid + 0], nx));
                d[1] = float(mimg(double(y) - a.X[3 * pid + 1], ny));
                d[2] = float(mimg(double(z) - a.X[3 * pid + 2], nz));
                const float r0 = d[0] + qf * lx, r1 = d[1] + qf * ly, r2 = d[2] + qf * lz;
                const double *Wp = a.W + 3 * pid, *Up = a.U + 3 * pid;
                const float W0 = float(Wp[0]), W1 = float(Wp[1]), W2 = float(Wp[2]);
                uw[0] = float(Up[0]) + (W1 * r2 - W2 * r1);
                uw[1] = float(Up[1]) + (W2 * r0 - W0 * r2);
                uw[2] = float(Up[2]) + (W0 * r1 - W1 * r0);
            }
            const float w_l = float(wgt(l));
            const float Dw = pid >= 0 ? -6.0f * w_l * (lx * uw[0] + ly * uw[1] + lz * uw[2]) : 0.0f;
            const float v = ibb_value<S>(A, N, l, i, sch, qf, c1, c2, Dw, fl0, fi0);
            Store<S>::st(A + (size_t)i * N + cb, v);
            if (pid >= 0) {
                const float fo = fl0 + w_l, fi = v + w_l;
                const float dP0 = (lx - uw[0]) * fo - (-lx - uw[0]) * fi;
                const float dP1 = (ly - uw[1]) * fo - (-ly - uw[1]) * fi;
                const float dP2 = (lz - uw[2]) * fo - (-lz - uw[2]) * fi;
                const float m0 = d[0] + 0.5f * lx, m1 = d[1] + 0.5f * ly, m2 = d[2] + 0.5f * lz;
                float *dP = (float *)a.link_dP + 3 * k, *dT = (float *)a.link_dT + 3 * k;
                dP[0] = dP0;
                dP[1] = dP1;
                dP[2] = dP2;
                dT[0] = m1 * dP2 - m2 * dP1;
                dT[1] = m2 * dP0 - m0 * dP2;
                dT[2] = m0 * dP1 - m1 * dP0;
            }
        }
    }
}

// Single-node links (scheme 2): ibb_links stored their halfway value; this
// pass adds the single-node correction (1 - 2q)/2 (d_l + d_ibar) from the
// wall node's own post-collision values (single_node_pair), and for
// particle links the momentum the correction carries, (c_l + u_w) dv, and
// its torque. Kept out of ibb_links so that the rare scheme costs the
// common link pass no registers.
template <int S, bool PART>
__global__ void __launch_bounds__(256) single_node_fix(LinkArgs a) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    // the single-node links of the current list, as listed by the geometry pass
    const long long ns = a.counts[4] < a.max_links ? a.counts[4] : a.max_links;
    T *A = (T *)a.A;
    const size_t N = (size_t)a.N;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < ns;
         j += (long long)gridDim.x * blockDim.x) {
        const long long k = a.sn_list[j];
        const int c = a.link_cell[k];
        const int l = a.link_dir[k];
        const double q = a.link_q[k];
        const unsigned zq = a.dxy.div((unsigned)c), rem = (unsigned)c - zq * (unsigned)(nx * ny);
        const unsigned yq = a.dx.div(rem);
        const int z = (int)zq, y = (int)yq, x = (int)(rem - yq * (unsigned)nx);
        const int lx = cx(l), ly = cy(l), lz = cz(l), i = opp(l);
        const int cb = wrap(x + lx, nx) + nx * (wrap(y + ly, ny) + ny * wrap(z + lz, nz));
        const R qq = sizeof(R) == 8 ? R(q) : R(float(q));
        const R dv = R(0.5) * (R(1) - R(2) * qq) *
                     single_node_pair<S>(A + c, N, l, body_force<R>(a, 0), body_force<R>(a, 1), body_force<R>(a, 2), a.rt);
        T *slot = A + (size_t)i * N + cb;
        Store<S>::st(slot, Store<S>::ld(slot) + dv);
        if constexpr (PART) {
            const int pid = a.link_pid[k];
            if (pid < 0) continue;
            // the wall velocity and lever arm of ibb_links, in the same arithmetic
            R uw[3], m[3];
            if constexpr (sizeof(R) == 8) {
                const double r0 = mimg(x + q * lx - a.X[3 * pid + 0], nx);
                const double r1 = mimg(y + q * ly - a.X[3 * pid + 1], ny);
                const double r2 = mimg(z + q * lz - a.X[3 * pid + 2], nz);
                const double *Wp = a.W + 3 * pid, *Up = a.U + 3 * pid;
                uw[0] = Up[0] + (Wp[1] * r2 - Wp[2] * r1);
                uw[1] = Up[1] + (Wp[2] * r0 - Wp[0] * r2);
                uw[2] = Up[2] + (Wp[0] * r1 - Wp[1] * r0);
                m[0] = mimg(x + 0.5 * lx - a.X[3 * pid + 0], nx);
                m[1] = mimg(y + 0.5 * ly - a.X[3 * pid + 1], ny);
                m[2] = mimg(z + 0.5 * lz - a.X[3 * pid + 2], nz);
            } else {
                const float d0 = float(mimg(double(x) - a.X[3 * pid + 0], nx));
                const float d1 = float(mimg(double(y) - a.X[3 * pid + 1], ny));
                const float d2 = float(mimg(double(z) - a.X[3 * pid + 2], nz));
                const float qf = float(q);
                const float r0 = d0 + qf * lx, r1 = d1 + qf * ly, r2 = d2 + qf * lz;
                const double *Wp = a.W + 3 * pid, *Up = a.U + 3 * pid;
                const float W0 = float(Wp[0]), W1 = float(Wp[1]), W2 = float(Wp[2]);
                uw[0] = float(Up[0]) + (W1 * r2 - W2 * r1);
                uw[1] = float(Up[1]) + (W2 * r0 - W0 * r2);
                uw[2] = float(Up[2]) + (W0 * r1 - W1 * r0);
                m[0] = d0 + 0.5f * lx;
                m[1] = d1 + 0.5f * ly;
                m[2] = d2 + 0.5f * lz;
            }
            // dP = (c_l - u_w) f_out - (c_ibar - u_w) f_in: f_in grew by dv
            const R e0 = (R(lx) + uw[0]) * dv, e1 = (R(ly) + uw[1]) * dv, e2 = (R(lz) + uw[2]) * dv;
            R *dP = (R *)a.link_dP + 3 * k, *dT = (R *)a.link_dT + 3 * k;
            dP[0] += e0;
            dP[1] += e1;
            dP[2] += e2;
            dT[0] += m[1] * e2 - m[2] * e1;
            dT[1] += m[2] * e0 - m[0] * e2;
            dT[2] += m[0] * e1 - m[1] * e0;
        }
    }
}

// ------------------------------------------------------------ IBM cells ----
struct IbmCollideArgs {
    void *B;  // streamed populations of the support cells, collided in place
    const int *site_cell;
    const uint8_t *flags;
    const void *sup_F;  // arithmetic type of the storage
    unsigned *status;
    const long long *counts;
    long long max_sites;
    long long N;
    double F[3];
    float Fs[3];
    Rates rt;
};

template <int S, bool SRT>
__global__ void __launch_bounds__(256) ibm_collide(IbmCollideArgs a) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const long long ns = a.counts[0] < a.max_sites ? a.counts[0] : a.max_sites;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < ns;
         s += (long long)gridDim.x * blockDim.x) {
    const int c = a.site_cell[s];
    T *__restrict__ B = (T *)a.B;
    const size_t N = (size_t)a.N;
    // the bulk sweep left this cell's streamed populations f_i(x) = f*_i(x - c_i) in B
    R g[19];
#pragma unroll
    for (int i = 0; i < 19; i++) g[i] = Store<S>::ld(B + (i * N + c));
    const bool fluid = !(a.flags[c] & FL_SOLID);
    const R *sF = (const R *)a.sup_F;
    const R fs = fluid ? R(1) : R(0);
    const R Fx = fs * body_force<R>(a, 0) + sF[3 * s + 0];
    const R Fy = fs * body_force<R>(a, 1) + sF[3 * s + 1];
    const R Fz = fs * body_force<R>(a, 2) + sF[3 * s + 2];
    R rho, ux, uy, uz;
    collide<R, true, SRT>(g, Fx, Fy, Fz, a.rt, rho, ux, uy, uz);
    watchdog(rho, ux, uy, uz, a.status);
#pragma unroll
    for (int i = 0; i < 19; i++) Store<S>::st(B + (i * N + c), g[i]);
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

// Ghost pass of a static wall (no particle links), FP32 arithmetic: links
// regrouped by direction, blockIdx.y = direction l, so l, c_l and ibar are
// uniform over the block and neighbouring threads touch neighbouring cells.
struct StaticLinkArgs {
    void *A;
    const uint4 *slink4;  // link records of the kept-values pass (see ibb_links_kept)
    const uint2 *slink;  // x = cell | scheme << 30, y = FP32 bits of q
    const int *rank;     // wall-cell rank of each link
    const void *bvals;   // wall cells' values (19 per cell), or null: read A
    const int *gidx;     // compact ghost value of each link
    void *gvals;         // compact ghost values (null: store in the solid nodes' slots)
    int off[20];
    int nx, ny, nz;
    long long N;
    FastDiv dx, dxy;
    double F[3];  // body force on fluid cells (single-node fallback)
    float Fs[3];
    Rates rt;
};

// The ghost pass of the static wall from per-link records (16 bytes: the
// upstream cell x_f - c_l with the flags "second value is f_ibar(x_f)" and
// "single-node", the two FP32 weights, the wall cell's rank), grouped by
// direction as the links are:
//   v = k1 f*_l(x_f) + k2 f*_l(x_f - c_l)   (linear, q < 1/2)
//   v = k1 f*_l(x_f) + k2 f*_ibar(x_f)      (linear, q >= 1/2)
//   v = f*_l(x_f) + k2 (d_l + d_ibar)       (single-node, Sec. 3.1)
// The wall cell's own populations come from the values the last sweep kept
// (19 per wall cell), or, before the first sweep, from A at x_f (only z
// wraps between x_f - c_l and x_f: the walls of this pass touch no x or y
// face). No division or index decoding per link.
template <int S, bool SN>
__global__ void __launch_bounds__(256) ibb_links_kept(StaticLinkArgs a) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const int l = blockIdx.y;
    const int k0 = a.off[l], k1 = a.off[l + 1];
    const size_t N = (size_t)a.N;
    const T *A = (const T *)a.A + (size_t)l * N;  // plane l
    const int i = opp(l);
    const bool kept = a.bvals != nullptr;
    const long long offl = (long long)cx(l) + (long long)a.nx * (cy(l) + (long long)a.ny * cz(l));
    for (int k = k0 + blockIdx.x * blockDim.x + threadIdx.x; k < k1; k += gridDim.x * blockDim.x) {
        const uint4 m = __ldg(a.slink4 + k);
        const int gi = __ldg(a.gidx + k);
        const unsigned c1 = m.x & 0x3fffffffu;
        const bool own = (m.x >> 30) & 1u, single = m.x >> 31;
        const T *wv;
        size_t stride;
        if (kept) {
            wv = (const T *)a.bvals + (size_t)19 * m.w;
            stride = 1;
        } else {
            long long c = (long long)c1 + offl;
            c = c < 0 ? c + (long long)N : (c >= (long long)N ? c - (long long)N : c);
            wv = (const T *)a.A + c;
            stride = N;
        }
        const R fl0 = Store<S>::ld(wv + (size_t)l * stride);
        const R second = own ? Store<S>::ld(wv + (size_t)i * stride) : (single ? R(0) : Store<S>::ld(A + c1));
        R v = fmaf(R(__uint_as_float(m.y)), fl0, R(__uint_as_float(m.z)) * second);
        if (SN && single)
            v = fmaf(R(__uint_as_float(m.z)),
                     single_node_pair<S>(wv, stride, l, body_force<R>(a, 0), body_force<R>(a, 1), body_force<R>(a, 2),
                                         a.rt),
                     fl0);
        Store<S>::st((T *)a.gvals + gi, v);
    }
}

template <int S, bool SN>
__global__ void __launch_bounds__(256) ibb_links_static(StaticLinkArgs a) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const int l = blockIdx.y;
    const int k0 = a.off[l], k1 = a.off[l + 1];
    T *A = (T *)a.A;
    const size_t N = (size_t)a.N;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int lx = cx(l), ly = cy(l), lz = cz(l), i = opp(l);
    for (int k = k0 + blockIdx.x * blockDim.x + threadIdx.x; k < k1; k += gridDim.x * blockDim.x) {
        const uint2 m = __ldg(a.slink + k);
        const int c = (int)(m.x & 0x3fffffffu), sch = (int)(m.x >> 30);
        const R qq = R(__uint_as_float(m.y));
        const unsigned zq = a.dxy.div((unsigned)c), rem = (unsigned)c - zq * (unsigned)(nx * ny);
        const unsigned yq = a.dx.div(rem);
        const int z = (int)zq, y = (int)yq, x = (int)(rem - yq * (unsigned)nx);
        const int cb = wrap(x + lx, nx) + nx * (wrap(y + ly, ny) + ny * wrap(z + lz, nz));
        const int x1 = wrap(x - lx, nx), y1 = wrap(y - ly, ny), z1 = wrap(z - lz, nz);
        const int c1 = x1 + nx * (y1 + ny * z1);
        const int c2 = wrap(x1 - lx, nx) + nx * (wrap(y1 - ly, ny) + ny * wrap(z1 - lz, nz));
        R fl0, fi0;
        if (a.bvals) {  // the same values, kept contiguous by the last sweep
            const T *wv = (const T *)a.bvals + (size_t)19 * __ldg(a.rank + k);
            fl0 = Store<S>::ld(wv + l);
            fi0 = Store<S>::ld(wv + i);
        } else {
            fl0 = Store<S>::ld(A + (size_t)l * N + c);
            fi0 = Store<S>::ld(A + (size_t)i * N + c);
        }
        R v = ibb_value<S>(A, N, l, i, sch, qq, c1, c2, R(0), fl0, fi0);
        if (SN && sch == 2) {  // single-node fallback from the wall cell's own values
            const T *p = a.bvals ? (const T *)a.bvals + (size_t)19 * __ldg(a.rank + k) : A + c;
            v += R(0.5) * (R(1) - R(2) * qq) *
                 single_node_pair<S>(p, a.bvals ? 1 : N, l, body_force<R>(a, 0), body_force<R>(a, 1),
                                     body_force<R>(a, 2), a.rt);
        }
        if (a.gvals)
            Store<S>::st((T *)a.gvals + __ldg(a.gidx + k), v);  // read by the sweep in place of the pull
        else
            Store<S>::st(A + (size_t)i * N + cb, v);
    }
}

template <int S>
static cudaError_t launch_links_s(Ctx &c) {
    if (c.max_links == 0) return cudaSuccess;
    if (c.static_links && c.np == 0 && S != LBM_F64) {
        // the inline wall form: the last sweep left the partial values, or
        // they are formed once from the populations
        if (pipe_inline_walls(c)) return c.bvals_valid == 2 ? cudaSuccess : launch_pipe_wall_prime(c);
        StaticLinkArgs a;
        a.A = c.fA;
        a.slink4 = c.slink4;
        a.slink = c.slink;
        a.rank = c.slink_rank;
        a.bvals = c.bvals_valid == 1 ? c.bvals : nullptr;
        a.gidx = c.gidx;
        a.gvals = c.bvals_ready ? c.gvals : nullptr;
        for (int l = 0; l < 20; l++) a.off[l] = c.slink_off[l];
        a.nx = c.nx;
        a.ny = c.ny;
        a.nz = c.nz;
        a.N = c.N;
        a.dx = FastDiv((unsigned)c.nx);
        a.dxy = FastDiv((unsigned)(c.nx * c.ny));
        for (int d = 0; d < 3; d++) {
            a.F[d] = c.F[d];
            a.Fs[d] = (float)c.F[d];
        }
        a.rt = c.rt;
        int most = 0;
        for (int l = 0; l < 19; l++) most = std::max(most, c.slink_off[l + 1] - c.slink_off[l]);
        unsigned nbx = (unsigned)((most + 255) / 256);
        if (nbx < 1) nbx = 1;

        count_launch(c, G_BND);
        // the variant with the single-node scheme only for walls that have such links
        if (c.slink4_ready && a.gvals) {  // every step, so a restart repeats the same arithmetic
            if (c.static_single > 0) ibb_links_kept<S, true><<<dim3(nbx, 19), 256, 0, c.stream>>>(a);
            else ibb_links_kept<S, false><<<dim3(nbx, 19), 256, 0, c.stream>>>(a);
        } else if (c.static_single > 0) {
            ibb_links_static<S, true><<<dim3(nbx, 19), 256, 0, c.stream>>>(a);
        } else {
            ibb_links_static<S, false><<<dim3(nbx, 19), 256, 0, c.stream>>>(a);
        }
        return cudaGetLastError();
    }
    LinkArgs a{c.fA, c.link_cell, c.link_pid, c.link_dir, c.link_scheme, c.link_q, c.link_dP, c.link_dT,
               c.X, c.U, c.W, c.d_counts, c.max_links, c.nx, c.ny, c.nz, c.N,
               FastDiv((unsigned)c.nx), FastDiv((unsigned)(c.nx * c.ny)), {c.F[0], c.F[1], c.F[2]},
               {(float)c.F[0], (float)c.F[1], (float)c.F[2]}, c.rt, c.sn_list};
    long long n = c.nlinks_hint > 0 ? c.nlinks_hint : c.max_links;
    if (n > c.max_links) n = c.max_links;
    long long nb = (n + 255) / 256;
    if (nb < 1) nb = 1;
    if (nb > 152LL * 64) nb = 152LL * 64;
    count_launch(c, G_BND);
    if (c.np > 0) ibb_links<S, true><<<(unsigned)nb, 256, 0, c.stream>>>(a);
    else ibb_links<S, false><<<(unsigned)nb, 256, 0, c.stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // moving walls may have single-node links at any step; a static wall only if its list has some
    if (c.np > 0 || c.static_single > 0) {
        count_launch(c, G_BND);
        const unsigned nbs = 152u * 2u;  // a few single-node links: a small grid striding over the list
        if (c.np > 0) single_node_fix<S, true><<<nbs, 256, 0, c.stream>>>(a);
        else single_node_fix<S, false><<<nbs, 256, 0, c.stream>>>(a);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_ibb_links(Ctx &c) {
    switch (c.storage) {
    case LBM_F64: return launch_links_s<LBM_F64>(c);
    case LBM_F32: return launch_links_s<LBM_F32>(c);
    case LBM_F16S: return launch_links_s<LBM_F16S>(c);
    default: return launch_links_s<LBM_BF16S>(c);
    }
}

template <int S>
static cudaError_t launch_ibm_s(Ctx &c) {
    if (c.max_sites == 0) return cudaSuccess;
    IbmCollideArgs a;
    a.B = c.fB;
    a.site_cell = c.site_cell;
    a.flags = c.flags;
    a.sup_F = c.sup_F;
    a.status = c.d_status;
    a.counts = c.d_counts;
    a.max_sites = c.max_sites;
    a.N = c.N;
    for (int d = 0; d < 3; d++) {
        a.F[d] = c.F[d];
        a.Fs[d] = (float)c.F[d];
    }
    a.rt = c.rt;
    const int tb = 256;
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
    // arithmetic type of the storage: FP64 arithmetic is slow on GB300 and
    // buys nothing for 32- or 16-bit populations
    typedef typename Store<S>::R R;
    const R ux = R(u[c]), uy = R(u[N + c]), uz = R(u[2 * N + c]), r0 = R(rho0);
    const R u2 = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < 19; i++) {
        const R cu = R(cx(i)) * ux + R(cy(i)) * uy + R(cz(i)) * uz;
        // f_eq - w = w (rho0 - 1) + w rho0 (3 cu + 4.5 cu^2 - 1.5 u^2)
        const R geq = R(wgt(i)) * ((r0 - R(1)) + r0 * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * u2));
        Store<S>::st((T *)dst + (size_t)i * N + c, geq);
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
