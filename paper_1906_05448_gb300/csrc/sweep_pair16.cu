// The lean pipe sweep for 16-bit storage (FP16 x 2^10 or BF16) with two
// adjacent cells per lane: the pull-stream + BGK/Guo sweep of the static
// pipe wall (Sec. 2.1) in the inline wall form (see sweep_pipe.cu).
//
// - Work: runs of fluid cells cut at even cells into pieces of up to 32
//   pairs; a warp sweeps an item of up to two pieces, one pair per lane. A
//   run's first cell when odd and its last when even are solid cells that
//   the lane completes with zeros.
// - Pulls: a direction with c_x = 0 pulls both cells with one 4-byte load
//   (nx even, so both sources share an aligned word); the others with two
//   2-byte loads. Stores: one 4-byte store per direction and pair.
// - Collision: BGK with Guo forcing on both cells at once, in packed FP32
//   arithmetic (two lanes of every add, multiply and fused multiply-add).
// - Wall: every wall value goes through shared memory. The wall lanes put
//   their cells' pulled values there; one lane per link of the item (its
//   links are a contiguous range of ghost slots) replaces the value of the
//   link's direction by p + k2' f*_l(x_f - c_l), p from the ghost slot; the
//   wall lanes read them back before the collision. After it, they put
//   their post-collision values there, and one round later, while the next
//   item's pulls are in flight, one lane per link forms the next step's p.
#include "lbm_internal.cuh"

#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pairs.h"
#include "segments.h"

namespace lbmgb {

struct Pair16Args {
    const SweepItem *items;  // pair units: x and lanes count pairs
    const uint4 *iwall;      // per item: first ghost slot, links, 64-bit mask of wall cells
    long long nitems;
    void *gvals;                  // ghost slots: the partial values p
    const uint2 *wcoef;           // per slot: k1, k2 (bit 31: q >= 1/2)
    const unsigned short *wslot;  // per slot: cell of the item (0..63) | direction << 6
    unsigned *status;
    int nx;
    unsigned N;
    unsigned rz0, rz1;  // rows of the first plane: < rz0; of the last: >= rz1
    PairK k;
    const void *Ap[19];  // A + i N - (c_x + nx c_y + nx ny c_z)
    void *Bp[19];        // B + i N
};

#ifndef LBM_PAIR16_MINB
#define LBM_PAIR16_MINB 2  // resident blocks of 256 per SM the registers are sized for (128: no spills)
#endif

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b rounded once: b (-1) + a with the exact product
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

// collide_pairs (lbm_device.cuh) on two cells at once: the same operations
// in the same order, each on both lanes of a packed pair
template <bool FORCE, int SC>
__device__ __forceinline__ void collide_pairs2(float2 g[19], const PairK &k, float2 &rho_o, float2 &u2_o) {
    constexpr float down = 1.0f / float(1u << SC), up = float(1u << SC);
    const float2 s1 = add2(g[1], g[2]), d1 = sub2(g[1], g[2]), s3 = add2(g[3], g[4]), d3 = sub2(g[3], g[4]);
    const float2 s5 = add2(g[5], g[6]), d5 = sub2(g[5], g[6]), s7 = add2(g[7], g[8]), d7 = sub2(g[7], g[8]);
    const float2 s9 = add2(g[9], g[10]), d9 = sub2(g[9], g[10]), s11 = add2(g[11], g[12]), d11 = sub2(g[11], g[12]);
    const float2 s13 = add2(g[13], g[14]), d13 = sub2(g[13], g[14]), s15 = add2(g[15], g[16]),
                 d15 = sub2(g[15], g[16]);
    const float2 s17 = add2(g[17], g[18]), d17 = sub2(g[17], g[18]);
    float2 drho = add2(add2(add2(g[0], add2(add2(s1, s3), s5)), add2(add2(s7, s9), add2(s11, s13))), add2(s15, s17));
    const float2 jx = add2(add2(d1, add2(d7, d9)), add2(d11, d13));
    const float2 jy = add2(add2(d3, sub2(d7, d9)), add2(d15, d17));
    const float2 jz = add2(add2(d5, sub2(d11, d13)), sub2(d15, d17));
    if (SC != 0) drho = mul2(drho, f2(down));
    const float2 rho = add2(f2(1.0f), drho);
    const float2 ir = mul2(make_float2(__frcp_rn(rho.x), __frcp_rn(rho.y)), f2(down));
    const float2 ux = mul2(FORCE ? fma2(f2(k.hF[0]), f2(up), jx) : jx, ir);
    const float2 uy = mul2(FORCE ? fma2(f2(k.hF[1]), f2(up), jy) : jy, ir);
    const float2 uz = mul2(FORCE ? fma2(f2(k.hF[2]), f2(up), jz) : jz, ir);
    const float2 u2 = fma2(ux, ux, fma2(uy, uy, mul2(uz, uz)));
    rho_o = rho;
    u2_o = u2;
    const float2 Bv = fma2(mul2(f2(-1.5f), rho), u2, drho);
    const float2 uF3 = FORCE ? fma2(ux, f2(k.F3[0]), fma2(uy, f2(k.F3[1]), mul2(uz, f2(k.F3[2])))) : f2(0.0f);
    const float2 b0 = mul2(FORCE ? fma2(f2(k.w[0]), Bv, mul2(f2(-k.cw[0]), uF3)) : mul2(f2(k.w[0]), Bv), f2(up));
    const float2 b1 = mul2(FORCE ? fma2(f2(k.w[1]), Bv, mul2(f2(-k.cw[1]), uF3)) : mul2(f2(k.w[1]), Bv), f2(up));
    const float2 b2 = mul2(FORCE ? fma2(f2(k.w[2]), Bv, mul2(f2(-k.cw[2]), uF3)) : mul2(f2(k.w[2]), Bv), f2(up));
    const float2 q1 = mul2(mul2(f2(k.q[0]), rho), f2(up)), q2 = mul2(mul2(f2(k.q[1]), rho), f2(up));
    const float2 t1 = f2(k.t[0]), t2 = f2(k.t[1]), mt1 = f2(-k.t[0]), mt2 = f2(-k.t[1]);
    const float2 om = f2(k.om);
    g[0] = fma2(om, sub2(b0, g[0]), g[0]);
    auto pair = [&](int i, float2 cu, float2 cj, float2 q, float2 t, float2 mt, float2 b) {
        const float2 E = FORCE ? fma2(fma2(q, cu, f2(k.L[i] * up)), cu, b) : fma2(mul2(q, cu), cu, b);
        const float2 Ki = f2(FORCE ? k.K[i] * up : 0.0f);
        const float2 hi = fma2(t, cj, neg2(g[i])), hb = fma2(mt, cj, neg2(g[i + 1]));
        g[i] = fma2(om, add2(add2(E, Ki), hi), g[i]);
        g[i + 1] = fma2(om, add2(sub2(E, Ki), hb), g[i + 1]);
    };
    pair(1, ux, jx, q1, t1, mt1, b1);
    pair(3, uy, jy, q1, t1, mt1, b1);
    pair(5, uz, jz, q1, t1, mt1, b1);
    pair(7, add2(ux, uy), add2(jx, jy), q2, t2, mt2, b2);
    pair(9, sub2(ux, uy), sub2(jx, jy), q2, t2, mt2, b2);
    pair(11, add2(ux, uz), add2(jx, jz), q2, t2, mt2, b2);
    pair(13, sub2(ux, uz), sub2(jx, jz), q2, t2, mt2, b2);
    pair(15, add2(uy, uz), add2(jy, jz), q2, t2, mt2, b2);
    pair(17, sub2(uy, uz), sub2(jy, jz), q2, t2, mt2, b2);
}

// the two stored 16-bit numbers of a 32-bit word (low half first) as they
// enter the collision (FP16 keeps g x 2^10: no unscaling), and back
template <int S>
__device__ __forceinline__ float2 unpack2(unsigned v) {
    if constexpr (S == LBM_F16S) {
        __half2 h;
        memcpy(&h, &v, 4);
        return __half22float2(h);
    } else {
        __nv_bfloat162 h;
        memcpy(&h, &v, 4);
        return __bfloat1622float2(h);
    }
}
template <int S>
__device__ __forceinline__ unsigned pack2(float2 v) {
    unsigned r;
    if constexpr (S == LBM_F16S) {
        const __half2 h = __floats2half2_rn(v.x, v.y);
        memcpy(&r, &h, 4);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        memcpy(&r, &h, 4);
    }
    return r;
}
template <int S>
__device__ __forceinline__ float unpack1(unsigned short v) {
    return unpack2<S>((unsigned)v).x;
}

// the partial value p of a wall link (w: k1, k2 with bit 31 set for
// q >= 1/2) from the wall cell's own values f*_l and f*_ibar: the arithmetic
// of pipe_wall_prime and of the one-cell sweep, so that the two sweeps and
// a restart agree bit for bit
__device__ __forceinline__ float pair_wall_partial(uint2 w, float fl, float fi) {
    const float k1 = __uint_as_float(w.x);
    return (w.y >> 31) ? __fmaf_rn(k1, fl, __fmul_rn(__uint_as_float(w.y & 0x7fffffffu), fi)) : __fmul_rn(k1, fl);
}

template <int S, bool FORCE>
__global__ void __launch_bounds__(256, LBM_PAIR16_MINB) stream_collide_pair16(Pair16Args a) {
    typedef typename Store<S>::T T;
    constexpr int SC = S == LBM_F16S ? 10 : 0;
    const int lane = threadIdx.x & 31;
    const unsigned items = (unsigned)a.nitems;
    const unsigned gw = gridDim.x * (blockDim.x / 32);
    const unsigned N = a.N;
    // per warp: the wall cells' 19 values, slot 2 lane + h for cell h of the lane's pair
    __shared__ float gsm[8][19][64];
    float(*gs)[64] = gsm[threadIdx.x / 32];
    // the partial values p of a wall item's links [pb0, pb0 + pnum) from the
    // post-collision values in shared memory (run one round late)
    auto partials = [&](unsigned pb0, unsigned pnum) {
        for (unsigned k = lane; k < pnum; k += 32u) {
            const uint2 w = __ldg(a.wcoef + pb0 + k);
            const unsigned t = __ldg(a.wslot + pb0 + k);
            const int s = (int)(t & 63u), i = (int)(t >> 6);
            const float pv = pair_wall_partial(w, gs[opp(i)][s], gs[i][s]);
            ((unsigned short *)a.gvals)[pb0 + k] = (unsigned short)(pack2<S>(make_float2(pv, 0.0f)) & 0xffffu);
        }
        __syncwarp();
    };
    unsigned pb0 = 0u, pnum = 0u;
    const unsigned w0 = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    uint4 sgn = make_uint4(0u, 0u, 0u, 0u), wln = make_uint4(0u, 0u, 0u, 0u);
    if (w0 < items) {
        sgn = __ldg((const uint4 *)a.items + w0);
        wln = __ldg(a.iwall + w0);
    }
    for (unsigned w = w0; w < items; w += gw) {
        const uint4 sg = sgn, wl = wln;
        if (w + gw < items) {  // the next round's records
            sgn = __ldg((const uint4 *)a.items + w + gw);
            wln = __ldg(a.iwall + w + gw);
        }
        const int la = (int)((sg.y >> 16) & 0xff);
        const bool pa = lane < la;
        const unsigned wd = pa ? sg.y : sg.w, row = pa ? sg.x : sg.z;
        const int lp = pa ? lane : lane - la;
        const int len = (int)((wd >> 16) & 0xff), lead = (int)((wd >> 24) & 15), trail = (int)(wd >> 28);
        const bool active = lp < len;
        const unsigned c0 = row * (unsigned)a.nx + 2u * ((wd & 0xffffu) - (unsigned)lead + (unsigned)lp);
        const bool zero0 = lead && lp == 0, zero1 = trail && lp == len - 1;
        // pulls of both cells, as one 32-bit word per direction (low half: the even cell)
        unsigned raw[19];
        if (active) {
            const unsigned zp = row < a.rz0 ? N : 0u, zm = row >= a.rz1 ? N : 0u;
#pragma unroll
            for (int i = 0; i < 19; i++) {
                const int o = (int)c0 + (cz(i) > 0 ? (int)zp : 0) - (cz(i) < 0 ? (int)zm : 0);
                const T *p = (const T *)a.Ap[i] + o;
                if (cx(i) == 0) {
                    raw[i] = __ldg((const unsigned *)p);
                } else {
                    raw[i] = (unsigned)__ldg((const unsigned short *)p) |
                             ((unsigned)__ldg((const unsigned short *)p + 1) << 16);
                }
            }
        }
        // the wall: this item's links [lb0, lb0 + lnum), the first 32 one per lane
        const unsigned lb0 = wl.x, lnum = wl.y;
        const unsigned long long wmask = ((unsigned long long)wl.w << 32) | wl.z;
        const unsigned mine = (unsigned)(wmask >> (2 * lane)) & 3u;  // wall cells of this lane's pair
        unsigned lk = 0u, lt = 0u, lp16 = 0u;
        if ((unsigned)lane < lnum) {
            lk = __ldg(&a.wcoef[lb0 + lane].y);
            lt = __ldg(a.wslot + lb0 + lane);
            lp16 = __ldg((const unsigned short *)a.gvals + lb0 + lane);
        }
        if (pnum) {  // the last wall item's partial values
            partials(pb0, pnum);
            pnum = 0u;
        }
        float2 g[19];
#pragma unroll
        for (int i = 0; i < 19; i++) g[i] = active ? unpack2<S>(raw[i]) : f2(0.0f);
        if (lnum) {  // uniform over the warp
            if (mine) {
#pragma unroll
                for (int i = 0; i < 19; i++) {
                    gs[i][2 * lane] = g[i].x;
                    gs[i][2 * lane + 1] = g[i].y;
                }
            }
            __syncwarp();
            // f_ibar = p + k2' f*_l(x_f - c_l): a link with k2' != 0 has its
            // opposite direction pulled from a fluid cell, never replaced
            for (unsigned k = lane; k < lnum; k += 32u) {
                unsigned k2 = lk, t = lt, pv = lp16;
                if (k >= 32u) {  // items with more than 32 links (rows along the wall)
                    k2 = __ldg(&a.wcoef[lb0 + k].y);
                    t = __ldg(a.wslot + lb0 + k);
                    pv = __ldg((const unsigned short *)a.gvals + lb0 + k);
                }
                const int s = (int)(t & 63u), i = (int)(t >> 6);
                const float p = unpack1<S>((unsigned short)pv);
                gs[i][s] = (k2 >> 31) ? p : __fmaf_rn(__uint_as_float(k2), gs[opp(i)][s], p);
            }
            __syncwarp();
            if (mine) {
#pragma unroll
                for (int i = 1; i < 19; i++) g[i] = make_float2(gs[i][2 * lane], gs[i][2 * lane + 1]);
            }
        }
        float2 rho, u2;
        collide_pairs2<FORCE, SC>(g, a.k, rho, u2);
        if (active) {
            const bool bad0 = !zero0 && !(rho.x > 0.5f && rho.x < 2.0f && u2.x < 0.09f);
            const bool bad1 = !zero1 && !(rho.y > 0.5f && rho.y < 2.0f && u2.y < 0.09f);
            if (bad0 || bad1) atomicOr(a.status, 1u);
#pragma unroll
            for (int i = 0; i < 19; i++) {
                // zero cells (solid) complete the word
                const unsigned word = pack2<S>(make_float2(zero0 ? 0.0f : g[i].x, zero1 ? 0.0f : g[i].y));
                *((unsigned *)((T *)a.Bp[i] + c0)) = word;
                if (mine) {  // wall cells: the stored values, for the partial values p of the next step
                    const float2 r = unpack2<S>(word);
                    gs[i][2 * lane] = r.x;
                    gs[i][2 * lane + 1] = r.y;
                }
            }
        }
        if (lnum) {
            __syncwarp();
            pb0 = lb0;
            pnum = lnum;
        }
    }
    if (pnum) partials(pb0, pnum);
}

// ----------------------------------------------------------------- host --
// The pair work list and wall tables (pairs.h) of a static wall whose fluid
// runs the one-cell sweep already lists, uploaded to the workspace. Returns
// false (nothing built) when the form does not fit or the workspace holds
// too few items.
bool build_pair16(Ctx &c, const uint8_t *fl, const std::vector<int> &bcells, const std::vector<uint2> &wr) {
    c.pair_ready = 0;
    std::vector<SweepItem> items;
    std::vector<PairItemWall> iw;
    std::vector<unsigned short> ws;
    if (!build_pair_tables(fl, c.nx, c.ny, c.nz, FL_SOLID, bcells, wr, items, iw, ws)) return false;
    if ((long long)items.size() > c.max_seg) return false;
    static_assert(sizeof(SweepItem) == sizeof(uint4) && sizeof(PairItemWall) == sizeof(uint4), "item layout");
    if (cudaMemcpy(c.pair_items, items.data(), 16 * items.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c.pair_wall, iw.data(), 16 * iw.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c.wslot, ws.data(), 2 * ws.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
    c.npair_items = (long long)items.size();
    c.pair_ready = 1;
    return true;
}

#ifndef LBM_PAIR16
#define LBM_PAIR16 1  // 1: the pair sweep for 16-bit storage where it applies
#endif

template <int S>
static cudaError_t launch_pair16_t(Ctx &c, bool force) {
    Pair16Args a{};
    a.items = (const SweepItem *)c.pair_items;
    a.iwall = c.pair_wall;
    a.nitems = c.npair_items;
    a.gvals = c.gvals;
    a.wcoef = c.wcoef;
    a.wslot = c.wslot;
    a.status = c.d_status;
    a.nx = c.nx;
    a.N = (unsigned)c.N;
    a.rz0 = (unsigned)c.ny;
    a.rz1 = (unsigned)c.ny * (unsigned)(c.nz - 1);
    const long long nxy = (long long)c.nx * c.ny;
    for (int i = 0; i < 19; i++) {
        const long long off = cx(i) + (long long)c.nx * cy(i) + nxy * cz(i);
        a.Ap[i] = (const void *)((const char *)c.fA + 2 * (size_t)((long long)i * c.N - off));
        a.Bp[i] = (void *)((char *)c.fB + 2 * (size_t)((long long)i * c.N));
    }
    a.k = make_pair_k(c.rt.d_nu, c.F);
    static int resident[2];
    int &res = resident[force ? 1 : 0];
    if (res == 0) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (force) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_collide_pair16<S, true>, 256, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_collide_pair16<S, false>, 256, 0);
        res = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    long long nb = (c.npair_items + 7) / 8;
    if (nb > res) nb = res;
    if (nb < 1) nb = 1;
    count_launch(c, G_BULK);
    if (force) stream_collide_pair16<S, true><<<(unsigned)nb, 256, 0, c.stream>>>(a);
    else stream_collide_pair16<S, false><<<(unsigned)nb, 256, 0, c.stream>>>(a);
    return cudaGetLastError();
}

// The pair sweep serves the inline wall form on 16-bit storage once its
// tables are built. Returns false (nothing launched) otherwise.
bool launch_pair16_sweep(Ctx &c, cudaError_t &err) {
    if (!LBM_PAIR16 || !c.pair_ready || (c.storage != LBM_F16S && c.storage != LBM_BF16S) || !pipe_inline_walls(c))
        return false;
    const bool force = c.F[0] != 0.0 || c.F[1] != 0.0 || c.F[2] != 0.0;
    err = c.storage == LBM_F16S ? launch_pair16_t<LBM_F16S>(c, force) : launch_pair16_t<LBM_BF16S>(c, force);
    return true;
}

}  // namespace lbmgb
