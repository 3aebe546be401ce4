// Fused pull-stream + BGK/Guo collide sweep of a static IBB wall whose fluid
// cells never touch the x or y faces of the box (the pipe of Sec. 2.1):
// the dominant kernel of the pipe step, in a leaner form than the general
// sweep (sweep.cu).
//
// - Work: the fluid-run pieces of segments.h, items of up to two pieces,
//   persistent grid; a warp sweeps LBM_PIPE_ITEMS items per round (one by
//   default: two spill registers and measured slower), with the pulls of
//   all of them requested before any is collided, and the next round's
//   records loaded one round ahead.
// - Addresses: a pull is a per-direction base pointer (plane base minus
//   the direction's offset, a kernel parameter) plus the cell index; only
//   the periodic z ends need a correction (rows of the first and last
//   plane). Stores likewise from per-direction plane pointers.
// - Wall cells: an item without wall cells loads plain pulls; an item with
//   some (a warp-uniform branch) takes, at its wall lanes, the bounced
//   populations of the step from the compact ghost values in place of the
//   pulls from solid nodes. Two forms:
//   kept: a ghost pass before the sweep wrote the whole bounced values; the
//     sweep keeps the wall cells' 19 values for the next ghost pass;
//   inline (no single-node links, every weight known at set-up): the
//     linear interpolated bounce-back of link l (x_f + c_l solid, ibar =
//     opp(l) the unknown) is split at the step boundary,
//       f_ibar(x_f, t+1) = p + k2' f*_l(x_f - c_l),
//       p = k1 f*_l(x_f) + [q >= 1/2] k2 f*_ibar(x_f),
//       k2' = [q < 1/2] k2,
//     p from the wall cell's own post-collision values, written by this
//     sweep into the ghost slot, f*_l(x_f - c_l) the pull of direction l
//     that the next sweep makes at x_f anyway. The wall lanes put their 19
//     values in shared memory; one lane per link (an item's links are a
//     contiguous range of ghost slots) applies the weights, with coalesced
//     loads of the weights and stores of p. No ghost pass runs between
//     sweeps; pipe_wall_prime forms p from the stored populations when the
//     state was set otherwise (first step, restart).
// - Collision: BGK with Guo forcing (the single-relaxation setting of the
//   pipe runs, Sec. 2.1) written over opposite pairs: with cu_ibar = -cu_i
//   the equilibrium and forcing terms split into a part even and a part
//   odd under i -> ibar, each formed once per pair.
#include "lbm_internal.cuh"

namespace lbmgb {

struct PipeArgs {
    const void *A;
    void *B;
    const uint4 *seg;  // warp items (segments.h)
    long long nseg;
    const uint2 *seg_bnd;  // per item: rank of its first wall cell, wall-cell lanes
    void *bvals;           // wall cells' values for the next ghost pass, or null
    const uint2 *wrec;     // per wall cell: first compact ghost value, replaced directions
    void *gvals;           // compact ghost values of this step (inline: the partial values p)
    const uint2 *wcoef;    // inline: per ghost value k1, k2 (bit 31: q >= 1/2)
    const unsigned short *wlane;  // inline: per ghost value its wall cell's lane | direction << 5
    unsigned *status;
    int nx;
    unsigned N;        // cells; 19 N < 2^32
    unsigned rz0, rz1; // rows y + ny z of the first plane: < rz0; of the last: >= rz1
    PairK k;
    // per-direction base pointers: the pull of direction i for cell c is
    // Ap[i][c] (plus the z-end correction), its store Bp[i][c]; one address
    // operation per access (measured: sweep 0.2273 -> 0.2144 ms against
    // 32-bit offsets added to one base)
    const void *Ap[19];  // A + i N - (c_x + nx c_y + nx ny c_z)
    void *Bp[19];        // B + i N
};

// the inline wall form when it applies (0: always the ghost pass)
#ifndef LBM_PIPE_INLINE
#define LBM_PIPE_INLINE 1
#endif
// link offsets of the direction-grouped list and the box, for pipe_wall_prime
struct PipeLinkOff {
    int off[20];
    int nx, ny;
    long long N;
};

#ifndef LBM_PIPE_ITEMS
#define LBM_PIPE_ITEMS 1  // warp items a warp sweeps together (1 or 2)
#endif
#ifndef LBM_PIPE_MINB
#define LBM_PIPE_MINB 0  // resident blocks of 256 per SM the registers are sized for (0: per storage)
#endif
// measured on the benchmark pipe: with the ghost pass FP32 is fastest at 4
// blocks (64 registers), 16-bit storage at 5 (48 registers, more loads in
// flight); the inline wall form at 3 (80 registers; at 4 its sweep took
// 0.248 ms instead of 0.232 ms in FP32)
constexpr int pipe_min_blocks(int S, bool INL) {
    return LBM_PIPE_MINB > 0 ? LBM_PIPE_MINB : (INL ? 3 : (S == LBM_F32 ? 4 : 5));
}

// The stored numbers as the sweep computes on them (FP16 keeps g * 2^10;
// the scale is a power of two, so the arithmetic rounds as on g itself).
template <int S>
__device__ __forceinline__ float pipe_cvt(typename Store<S>::T v) {
    if constexpr (S == LBM_F32) return v;
    else if constexpr (S == LBM_F16S) return __half2float(v);
    else return __bfloat162float(v);
}
template <int S>
__device__ __forceinline__ void pipe_st(typename Store<S>::T *p, float v) {
    if constexpr (S == LBM_F16S) Store<LBM_F16S>::st_scaled(p, v);
    else Store<S>::st(p, v);
}
// v as it reads back from storage
template <int S>
__device__ __forceinline__ float pipe_round(float v) {
    if constexpr (S == LBM_F32) return v;
    else if constexpr (S == LBM_F16S) return __half2float(__float2half_rn(v));
    else return __bfloat162float(__float2bfloat16_rn(v));
}
// the partial value p of a wall link from the wall cell's own values f*_l
// and f*_ibar (the one arithmetic of the sweep's wall lanes and of
// pipe_wall_prime, so a restart repeats the uninterrupted run bit for bit)
// (w: k1, k2 with bit 31 set for q >= 1/2)
__device__ __forceinline__ float wall_partial(uint2 w, float fl, float fi) {
    const float k1 = __uint_as_float(w.x);
    return (w.y >> 31) ? __fmaf_rn(k1, fl, __fmul_rn(__uint_as_float(w.y & 0x7fffffffu), fi)) : __fmul_rn(k1, fl);
}

// NI warp items per warp and round: the records of the next round are
// loaded one round ahead, the populations of all NI items are requested
// before any of them is collided, so each thread has NI x 19 loads in flight.
// INL: the inline wall form (see above).
template <int S, bool FORCE, int NI, bool INL>
__global__ void __launch_bounds__(256, pipe_min_blocks(S, INL)) stream_collide_pipe(PipeArgs a) {
    typedef typename Store<S>::T T;
    // FP16 keeps g * 2^10: the collision runs on the stored numbers
    constexpr bool scaled = S == LBM_F16S;
    constexpr int SC = scaled ? 10 : 0;
    auto cvt = [](T v) -> float { return pipe_cvt<S>(v); };
    auto st = [](T *p, float v) { pipe_st<S>(p, v); };
    const int lane = threadIdx.x & 31;
    const unsigned items = (unsigned)a.nseg;  // < 2^32 (one item per 32 cells or fewer)
    const unsigned gw = gridDim.x * (blockDim.x / 32);  // warps in the grid
    const T *__restrict__ A = (const T *)a.A;
    const unsigned N = a.N;
    const bool keep_walls = !INL && a.bvals != nullptr;
    const bool walls = INL || keep_walls;  // compact ghost values and wall records in use
    auto wall_record = [&](uint2 bdv) -> uint2 {
        if (!((bdv.y >> lane) & 1u)) return make_uint2(0u, 0u);
        return __ldg(a.wrec + bdv.x + __popc(bdv.y & ((1u << lane) - 1u)));
    };
    uint4 sgn[NI];
    uint2 bdn[NI], wrn[NI];
    auto fetch = [&](unsigned w, int j) {
        sgn[j] = make_uint4(0u, 0u, 0u, 0u);
        bdn[j] = wrn[j] = make_uint2(0u, 0u);
        if (w < items) {
            sgn[j] = __ldg(a.seg + w);
            if (walls) {
                bdn[j] = __ldg(a.seg_bnd + w);
                wrn[j] = wall_record(bdn[j]);
            }
        }
    };
    // inline form: per warp, the wall lanes' 19 values in shared memory,
    // where one lane per wall link (an item's links are a contiguous range
    // of the compact values, in lane order) applies the link's weights
    static_assert(!INL || NI == 1, "the inline wall form takes one item per warp and round");
    __shared__ float gsm[INL ? 8 : 1][19][32];
    float(*gs)[32] = gsm[INL ? threadIdx.x / 32 : 0];
    // the partial values p of a wall item's links [pb0, pb0 + pnum) from the
    // wall lanes' post-collision values in shared memory; run one round
    // late, while the next item's pulls are in flight
    auto partials = [&](unsigned pb0, unsigned pnum) {
        for (unsigned k = lane; k < pnum; k += 32u) {
            const uint2 w = __ldg(a.wcoef + pb0 + k);
            const unsigned t = __ldg(a.wlane + pb0 + k);
            const int ln = (int)(t & 31u), i = (int)(t >> 5);
            st((T *)a.gvals + pb0 + k, wall_partial(w, gs[opp(i)][ln], gs[i][ln]));
        }
        __syncwarp();  // the slots are free for the next item
    };
    unsigned pb0 = 0u, pnum = 0u;  // the last wall item's links (uniform over the warp)
    const unsigned w0 = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
#pragma unroll
    for (int j = 0; j < NI; j++) fetch(w0 + j * gw, j);
    for (unsigned w = w0; w < items; w += NI * gw) {
        // this round's lanes: state 0 idle, 1 zero lane, 2 cell
        int state[NI];
        unsigned c[NI], row[NI];
        uint2 bd[NI], wr[NI];
#pragma unroll
        for (int j = 0; j < NI; j++) {
            const uint4 sg = sgn[j];
            bd[j] = bdn[j];
            wr[j] = wrn[j];
            const int la = (int)((sg.y >> 16) & 0xff);
            const bool pa = lane < la;
            const unsigned wd = pa ? sg.y : sg.w;
            row[j] = pa ? sg.x : sg.z;
            const int lp = pa ? lane : lane - la;
            const int len = (int)((wd >> 16) & 0xff), lead = (int)((wd >> 24) & 15), trail = (int)(wd >> 28);
            c[j] = row[j] * (unsigned)a.nx + ((wd & 0xffffu) - (unsigned)lead + (unsigned)lp);
            state[j] = (w + j * gw >= items || lp >= len) ? 0 : ((lp < lead || lp >= len - trail) ? 1 : 2);
        }
#pragma unroll
        for (int j = 0; j < NI; j++) fetch(w + (NI + j) * gw, j);
        // all pulls of the round
        T raw[NI][19];
#pragma unroll
        for (int j = 0; j < NI; j++) {
            if (state[j] != 2) continue;
            // periodic z ends: pulls with c_z = +1 from the first plane, c_z = -1 from the last
            const unsigned zp = row[j] < a.rz0 ? N : 0u, zm = row[j] >= a.rz1 ? N : 0u;
            const unsigned cj = c[j];
            auto pull = [&](int i) -> const T * {
                const int o = (int)cj + (cz(i) > 0 ? (int)zp : 0) - (cz(i) < 0 ? (int)zm : 0);
                return (const T *)a.Ap[i] + o;
            };
            if (bd[j].y == 0u) {  // no wall cell in this item (uniform over the warp)
#pragma unroll
                for (int i = 0; i < 19; i++) raw[j][i] = __ldg(pull(i));
            } else {
                const T *gv = walls ? (const T *)a.gvals + wr[j].x : A;
                const unsigned m = wr[j].y;
#pragma unroll
                for (int i = 0; i < 19; i++)
                    raw[j][i] = __ldg(((m >> i) & 1u) ? gv + __popc(m & ((1u << i) - 1u)) : pull(i));
            }
        }
        // inline form: an item's links are the ghost slots [lb0, lb0 + lnum)
        // in lane order; the first 32, one per lane (weights; wall lane |
        // direction << 5), load while the pulls are in flight
        unsigned lb0 = 0u, lnum = 0u;
        unsigned lk = 0u, li = 0u;  // k2 (bit 31: q >= 1/2), wall lane | direction << 5
        if (INL && bd[0].y != 0u) {  // uniform over the warp
            lb0 = __shfl_sync(0xffffffffu, wr[0].x, __ffs(bd[0].y) - 1);
            lnum = __reduce_add_sync(0xffffffffu, (unsigned)__popc(wr[0].y));
            if ((unsigned)lane < lnum) {
                lk = __ldg(&a.wcoef[lb0 + lane].y);
                li = __ldg(a.wlane + lb0 + lane);
            }
        }
        if (INL && pnum) {  // the last wall item's partial values
            partials(pb0, pnum);
            pnum = 0u;
        }
        if constexpr (!INL) {
#pragma unroll
            for (int j = 0; j < NI; j++) {
                if (state[j] == 0) continue;
                const unsigned cj = c[j];
                auto dst = [&](int i) -> T * { return (T *)a.Bp[i] + cj; };
                if (state[j] == 1) {
                    // zero lanes complete the run's end sectors (dead or ghost-overwritten slots)
#pragma unroll
                    for (int i = 0; i < 19; i++) st(dst(i), 0.0f);
                    continue;
                }
                float g[19];
#pragma unroll
                for (int i = 0; i < 19; i++) g[i] = cvt(raw[j][i]);
                float rho, u2;
                collide_pairs<FORCE, SC>(g, a.k, rho, u2);
                if (!(rho > 0.5f && rho < 2.0f && u2 < 0.09f)) atomicOr(a.status, 1u);
#pragma unroll
                for (int i = 0; i < 19; i++) st(dst(i), g[i]);
                if (keep_walls && ((bd[j].y >> lane) & 1u)) {
                    T *wv = (T *)a.bvals + (size_t)19 * (bd[j].x + __popc(bd[j].y & ((1u << lane) - 1u)));
#pragma unroll
                    for (int i = 0; i < 19; i++) st(wv + i, g[i]);
                }
            }
        } else {
            // one item (NI = 1); the warp-wide steps of the wall links sit
            // outside the per-lane branches
            const bool cell = state[0] == 2;
            const unsigned cj = c[0];
            auto dst = [&](int i) -> T * { return (T *)a.Bp[i] + cj; };
            if (state[0] == 1) {
#pragma unroll
                for (int i = 0; i < 19; i++) st(dst(i), 0.0f);
            }
            // every lane converts and collides (lanes without a cell on
            // zeros, results dropped): no per-lane branch around the warp-wide steps
            float g[19];
#pragma unroll
            for (int i = 0; i < 19; i++) g[i] = cell ? cvt(raw[0][i]) : 0.0f;
            const unsigned m = wr[0].y;  // replaced directions (wall lanes only)
            const bool wall_item = bd[0].y != 0u;  // uniform over the warp
            if (wall_item) {
                // f_ibar = p + k2' f*_l(x_f - c_l): a link with k2' != 0 has
                // its opposite direction pulled from a fluid cell, never replaced
                if (m) {
#pragma unroll
                    for (int i = 0; i < 19; i++) gs[i][lane] = g[i];
                }
                __syncwarp();
                for (unsigned k = lane; k < lnum; k += 32u) {
                    unsigned k2 = lk, t = li;
                    if (k >= 32u) {  // items with more than 32 links (rows along the wall)
                        k2 = __ldg(&a.wcoef[lb0 + k].y);
                        t = __ldg(a.wlane + lb0 + k);
                    }
                    const int ln = (int)(t & 31u), i = (int)(t >> 5);
                    if (!(k2 >> 31)) gs[i][ln] = __fmaf_rn(__uint_as_float(k2), gs[opp(i)][ln], gs[i][ln]);
                }
                __syncwarp();
                if (m) {
#pragma unroll
                    for (int i = 1; i < 19; i++) g[i] = gs[i][lane];
                }
            }
            {
                float rho, u2;
                collide_pairs<FORCE, SC>(g, a.k, rho, u2);
                if (cell && !(rho > 0.5f && rho < 2.0f && u2 < 0.09f)) atomicOr(a.status, 1u);
                if (cell) {
#pragma unroll
                    for (int i = 0; i < 19; i++) st(dst(i), g[i]);
                }
            }
            if (wall_item) {  // the values for the partial values p of the next step
                pb0 = lb0;
                pnum = lnum;
                if (m) {
#pragma unroll
                    for (int i = 0; i < 19; i++) gs[i][lane] = pipe_round<S>(g[i]);
                }
                __syncwarp();
            }
        }
    }
    if (INL && pnum) partials(pb0, pnum);
}

// The partial values p of every wall link from the stored populations (the
// state set by an initialisation or a restore): per link record of the
// direction-grouped list, x_f from the upstream cell x_f - c_l (only z
// wraps: the walls of the lean sweep touch no x or y face).
template <int S>
__global__ void __launch_bounds__(256) pipe_wall_prime(const void *Av, const uint4 *slink4, const int *gidx,
                                                        const uint2 *wcoef, void *gvals, PipeLinkOff o) {
    typedef typename Store<S>::T T;
    const int l = blockIdx.y;
    const T *A = (const T *)Av;
    const long long N = o.N;
    const long long offl = (long long)cx(l) + (long long)o.nx * (cy(l) + (long long)o.ny * cz(l));
    for (int k = o.off[l] + blockIdx.x * blockDim.x + threadIdx.x; k < o.off[l + 1]; k += gridDim.x * blockDim.x) {
        long long c = (long long)(__ldg(slink4 + k).x & 0x3fffffffu) + offl;
        c = c < 0 ? c + N : (c >= N ? c - N : c);
        const int gi = __ldg(gidx + k);
        const float fl = pipe_cvt<S>(__ldg(A + (size_t)l * N + c));
        const float fi = pipe_cvt<S>(__ldg(A + (size_t)opp(l) * N + c));
        pipe_st<S>((T *)gvals + gi, wall_partial(__ldg(wcoef + gi), fl, fi));
    }
}

template <int S>
static cudaError_t launch_prime_t(Ctx &c) {
    PipeLinkOff o;
    for (int l = 0; l < 20; l++) o.off[l] = c.slink_off[l];
    o.nx = c.nx;
    o.ny = c.ny;
    o.N = c.N;
    int most = 0;
    for (int l = 0; l < 19; l++) most = std::max(most, c.slink_off[l + 1] - c.slink_off[l]);
    const unsigned nbx = (unsigned)std::max(1, (most + 255) / 256);
    count_launch(c, G_BND);
    pipe_wall_prime<S><<<dim3(nbx, 19), 256, 0, c.stream>>>(c.fA, c.slink4, c.gidx, c.wcoef, c.gvals, o);
    return cudaGetLastError();
}

cudaError_t launch_pipe_wall_prime(Ctx &c) {
    switch (c.storage) {
    case LBM_F32: return launch_prime_t<LBM_F32>(c);
    case LBM_F16S: return launch_prime_t<LBM_F16S>(c);
    default: return launch_prime_t<LBM_BF16S>(c);
    }
}

template <int S, bool INL>
static cudaError_t launch_pipe_t(Ctx &c, bool force) {
    PipeArgs a{};
    a.A = c.fA;
    a.B = c.fB;
    a.seg = c.seg;
    a.nseg = c.nseg;
    a.seg_bnd = c.seg_bnd;
    a.bvals = (!INL && c.bvals_ready && c.static_links) ? c.bvals : nullptr;
    a.wrec = c.wrec;
    a.gvals = c.gvals;
    a.wcoef = c.wcoef;
    a.wlane = c.wlane;
    a.status = c.d_status;
    a.nx = c.nx;
    a.N = (unsigned)c.N;
    a.rz0 = (unsigned)c.ny;
    a.rz1 = (unsigned)c.ny * (unsigned)(c.nz - 1);
    const long long nxy = (long long)c.nx * c.ny;
    for (int i = 0; i < 19; i++) {
        const long long off = cx(i) + (long long)c.nx * cy(i) + nxy * cz(i);
        a.Ap[i] = (const void *)((const char *)c.fA + storage_bytes(c.storage) * (size_t)((long long)i * c.N - off));
        a.Bp[i] = (void *)((char *)c.fB + storage_bytes(c.storage) * (size_t)((long long)i * c.N));
    }
    a.k = make_pair_k(c.rt.d_nu, c.F);
    static int resident[4][2][2];
    int &res = resident[S][force ? 1 : 0][INL ? 1 : 0];
    if (res == 0) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (force)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_collide_pipe<S, true, LBM_PIPE_ITEMS, INL>,
                                                          256, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_collide_pipe<S, false, LBM_PIPE_ITEMS, INL>,
                                                          256, 0);
        res = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    long long nb = (c.nseg + 7) / 8;
    if (nb > res) nb = res;
    if (nb < 1) nb = 1;
    count_launch(c, G_BULK);
    if (force) stream_collide_pipe<S, true, LBM_PIPE_ITEMS, INL><<<(unsigned)nb, 256, 0, c.stream>>>(a);
    else stream_collide_pipe<S, false, LBM_PIPE_ITEMS, INL><<<(unsigned)nb, 256, 0, c.stream>>>(a);
    return cudaGetLastError();
}

static bool pipe_sweep_fits(const Ctx &c) {
    return c.pipe_nowrap && c.nseg > 0 && c.rates == LBM_RATES_SRT && c.storage != LBM_F64 && c.np == 0 &&
           19ULL * (unsigned long long)c.N + 64 < (1ULL << 32);
}

bool pipe_inline_walls(const Ctx &c) {
    return LBM_PIPE_INLINE && pipe_sweep_fits(c) && c.static_links && c.bvals_ready && c.slink4_ready &&
           c.wcoef_ready && c.static_single == 0;
}

// The lean sweep serves the static-wall IBB step with the single relaxation
// rate, 32- or 16-bit storage, a segment work list whose fluid cells do not
// touch the x or y faces, and 19 N < 2^32. Returns false (nothing launched)
// otherwise.
bool launch_pipe_sweep(Ctx &c, cudaError_t &err) {
    if (!pipe_sweep_fits(c)) return false;
    const bool force = c.F[0] != 0.0 || c.F[1] != 0.0 || c.F[2] != 0.0;
    const bool inl = pipe_inline_walls(c);
    switch (c.storage) {
    case LBM_F32: err = inl ? launch_pipe_t<LBM_F32, true>(c, force) : launch_pipe_t<LBM_F32, false>(c, force); break;
    case LBM_F16S: err = inl ? launch_pipe_t<LBM_F16S, true>(c, force) : launch_pipe_t<LBM_F16S, false>(c, force); break;
    default: err = inl ? launch_pipe_t<LBM_BF16S, true>(c, force) : launch_pipe_t<LBM_BF16S, false>(c, force); break;
    }
    return true;
}

}  // namespace lbmgb
