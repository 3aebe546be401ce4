// Fused pull-stream + collide sweep: the dominant kernel of every step.
//
// stream_collide_bulk: one thread per cell, threads along x so that every
// population plane is read and written in coalesced rows; the 19 loads of a
// cell are independent and issued together. IBB: solid cells are never
// swept (the pipe's fluid runs are listed as segments, see segments.h).
// IBM: support cells store rho and u* (first half of the direct forcing,
// Sec. 2.1) and their streamed populations, which ibm_collide later
// collides in place with the IBM force.
#include "lbm_internal.cuh"

#include <type_traits>

namespace lbmgb {

struct SweepArgs {
    const void *A;
    void *B;
    const uint4 *seg;  // optional warp items of fluid-run pieces (segments.h)
    long long nseg;
    FastDiv fd_ny;  // row -> (y, z)
    FastDiv fd_nx;     // cell -> (row, x) without a segment list
    long long nflat;   // without a segment list: items of blockDim.x consecutive cells
    const uint8_t *flags;
    const int *aux;
    void *sup_ru;  // (rho, u*) per support site, arithmetic type of the storage
    unsigned *status;
    long long max_sites;
    int nx, ny, nz;
    long long N;
    double F[3];
    float Fs[3];  // F in single precision (a double-to-single conversion per cell is costly on GB300)
    Rates rt;
    PairK pk;  // BGK + Guo factors in the pair form (FP32 arithmetic, uniform force)
    const uint2 *seg_bnd;  // per item: rank of its first wall cell, wall-cell lanes
    void *bvals;           // wall cells' populations for the next ghost pass (storage type), or null
    const uint2 *wrec;     // per wall cell: first compact ghost value, replaced directions
    const void *gvals;     // compact ghost values of this step (storage type)
    // plane bases A + i N and B + i N: one address operation per access
    // (as in the pipe sweep, where it cut the sweep from 0.2273 to 0.2144 ms)
    const void *Ap[19];
    void *Bp[19];
};

// BC: 0 periodic, 1 IBB, 2 IBM
// Resident blocks of 256 threads per SM the register allocation aims at
// (measured per variant: the BGK box fits 5 blocks without spilling; the
// pipe sweeps, which also handle the wall cells, and MRT are fastest at 4).
#ifndef LBM_BULK_MINB
#define LBM_BULK_MINB 0  // 0: per variant below
#endif
constexpr int bulk_min_blocks(int S, bool SRT, int BC) {
    return LBM_BULK_MINB > 0 ? LBM_BULK_MINB
                             : (!SRT || BC == 2 || S == LBM_F64) ? 4 : (BC == 0 ? 5 : 4);
}
#ifndef LBM_BULK_PERSIST
#define LBM_BULK_PERSIST 2  // persistent grid: 0 never, 1 always, 2 for segment sweeps
#endif
#ifndef LBM_BULK_SPEC
#define LBM_BULK_SPEC 0
#endif
#ifndef LBM_SRT_FOLDED
#define LBM_SRT_FOLDED 1
#endif
#ifndef LBM_IDX32
#define LBM_IDX32 1  // 32-bit element indices where they fit
#endif

// Work items: without a segment list, one item = blockDim.x consecutive
// cells in cell order, across row ends, so warps are full and start on a
// 32-cell boundary whatever nx is. With a segment list (IBB walls whose rows have a solid
// margin, e.g. the pipe), one warp = one segment of up to 32 consecutive
// cells inside the fluid extent of a row, so no lanes idle on the margin.
// The block walks its items with a grid stride and loads the flag byte of
// its next item before pulling the current one.
template <int S, bool SRT, int BC, bool FORCE, bool IDX32>
__global__ void __launch_bounds__(256, bulk_min_blocks(S, SRT, BC)) stream_collide_bulk(SweepArgs a) {
    typedef typename Store<S>::T T;
    typedef typename Store<S>::R R;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const bool segs = a.nseg > 0;  // one warp per item
    const int lane = threadIdx.x & 31;
    const long long items = segs ? a.nseg : a.nflat;
    const long long stride = segs ? (long long)gridDim.x * (blockDim.x / 32) : (long long)gridDim.x;
    const T *__restrict__ A = (const T *)a.A;
    // element index type: 32-bit when every index fits (19 N < 2^32), so an
    // address is one 32-bit add and one scaled add to the plane base
    typedef typename std::conditional<IDX32, unsigned, size_t>::type IX;
    const IX N = (IX)a.N;
    // FP16 with the folded BGK works on the stored (scaled) numbers
    static_assert(F16_SCALE == 1024.0f, "the scaled FP16 path assumes g * 2^10");
    constexpr bool scaled = S == LBM_F16S && SRT && BC != 2 && LBM_SRT_FOLDED;
    auto ld = [](const T *p) -> R {
        if constexpr (scaled) return Store<LBM_F16S>::ld_scaled(p);
        else return Store<S>::ld(p);
    };
    long long w = segs ? (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32 : (long long)blockIdx.x;
    // warp item: up to two pieces of fluid runs (row, word), see segments.h;
    // the next item is loaded one iteration ahead
    uint4 sg_next = make_uint4(0u, 0u, 0u, 0u);
    uint2 bd_next = make_uint2(0u, 0u), wr_next = make_uint2(0u, 0u);
    const bool keep_walls = BC == 1 && segs && a.bvals != nullptr;
    // the wall record of this lane's cell in the next item (its compact
    // ghost values replace the pulls from the solid nodes)
    auto wall_record = [&](uint2 bdv) -> uint2 {
        if (!((bdv.y >> lane) & 1u)) return make_uint2(0u, 0u);
        return __ldg(a.wrec + bdv.x + __popc(bdv.y & ((1u << lane) - 1u)));
    };
    if (segs && w < items) sg_next = __ldg(a.seg + w);
    if (keep_walls && w < items) {
        bd_next = __ldg(a.seg_bnd + w);
        wr_next = wall_record(bd_next);
    }
    auto cell_of = [&](long long item, int &x, int &row) {  // without a segment list
        // consecutive cells across row ends (N < 2^31): full warps for any nx
        const unsigned cc = (unsigned)item * blockDim.x + threadIdx.x;
        row = (int)a.fd_nx.div(cc);
        x = (int)(cc - (unsigned)row * (unsigned)nx);
        if (row >= ny * nz) x = nx;  // past the last cell
    };
    // segments cover fluid cells only: no flag byte is needed (IBB)
    const bool read_flags = BC != 0 && !(BC == 1 && segs);
    uint8_t fl_next = 0;
    if (read_flags && w < items) {
        int x, row;
        cell_of(w, x, row);
        if (x < nx) fl_next = a.flags[(size_t)row * nx + x];
    }
    for (; w < items; w += stride) {
        int x, row;
        bool zero = false;
        uint2 bd = make_uint2(0u, 0u), wr = make_uint2(0u, 0u);
        if (segs) {
            const uint4 sg = sg_next;
            bd = bd_next;
            wr = wr_next;
            if (w + stride < items) sg_next = __ldg(a.seg + w + stride);
            if (keep_walls && w + stride < items) {
                bd_next = __ldg(a.seg_bnd + w + stride);
                wr_next = wall_record(bd_next);
            }
            const int la = (int)((sg.y >> 16) & 0xff);
            const bool pa = lane < la;
            const unsigned wd = pa ? sg.y : sg.w;
            row = (int)(pa ? sg.x : sg.z);
            const int lp = pa ? lane : lane - la;  // lane within the piece
            const int len = (int)((wd >> 16) & 0xff), lead = (int)((wd >> 24) & 15), trail = (int)(wd >> 28);
            if (lp >= len) continue;
            x = (int)(wd & 0xffff) - lead + lp;
            // lanes on the solid cells that complete the 32-byte sectors at
            // either end of a fluid run write zeros (full-sector stores; the
            // slots are dead or rewritten as ghosts before they are read)
            zero = lp < lead || lp >= len - trail;
        } else {
            cell_of(w, x, row);
        }
        const uint8_t fl = fl_next;
        if (read_flags && w + stride < items) {
            int x2, row2;
            cell_of(w + stride, x2, row2);
            if (x2 < nx) fl_next = a.flags[(size_t)row2 * nx + x2];
        }
        if (zero) {
            const long long cz = (long long)row * nx + x;
#pragma unroll
            for (int i = 0; i < 19; i++) Store<S>::st((T *)a.Bp[i] + IX(cz), R(0));
            continue;
        }
        if (x >= nx) continue;
        if (!LBM_BULK_SPEC && BC == 1 && (fl & FL_SOLID)) continue;
        const int z = (int)a.fd_ny.div((unsigned)row), y = row - z * ny;
        const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
        const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
        // row offsets of the source rows (y - c_y, z - c_z)
        const int r00 = (y + ny * z) * nx;
        const int rM0 = (ym + ny * z) * nx, rP0 = (yp + ny * z) * nx;
        const int r0M = (y + ny * zm) * nx, r0P = (y + ny * zp) * nx;
        const int rMM = (ym + ny * zm) * nx, rPP = (yp + ny * zp) * nx;
        const int rMP = (ym + ny * zp) * nx, rPM = (yp + ny * zm) * nx;
        const int c = r00 + x;
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        R g[19];
        // pull: f_i(x) = f*_i(x - c_i); at a wall cell of the pipe, the
        // populations bounced at the wall are taken from the compact ghost
        // values of this step instead (one load either way)
        const T *gv = keep_walls ? (const T *)a.gvals + wr.x : A;
        auto pick = [&](int i, const T *pull) -> const T * {
            if constexpr (BC == 1)
                return ((wr.y >> i) & 1u) ? gv + __popc(wr.y & ((1u << i) - 1u)) : pull;
            else
                return pull;
        };
        g[0] = ld(A + IX(c));
        g[1] = ld(pick(1, (const T *)a.Ap[1] + IX(r00 + xm)));
        g[2] = ld(pick(2, (const T *)a.Ap[2] + IX(r00 + xp)));
        g[3] = ld(pick(3, (const T *)a.Ap[3] + IX(rM0 + x)));
        g[4] = ld(pick(4, (const T *)a.Ap[4] + IX(rP0 + x)));
        g[5] = ld(pick(5, (const T *)a.Ap[5] + IX(r0M + x)));
        g[6] = ld(pick(6, (const T *)a.Ap[6] + IX(r0P + x)));
        g[7] = ld(pick(7, (const T *)a.Ap[7] + IX(rM0 + xm)));
        g[8] = ld(pick(8, (const T *)a.Ap[8] + IX(rP0 + xp)));
        g[9] = ld(pick(9, (const T *)a.Ap[9] + IX(rP0 + xm)));
        g[10] = ld(pick(10, (const T *)a.Ap[10] + IX(rM0 + xp)));
        g[11] = ld(pick(11, (const T *)a.Ap[11] + IX(r0M + xm)));
        g[12] = ld(pick(12, (const T *)a.Ap[12] + IX(r0P + xp)));
        g[13] = ld(pick(13, (const T *)a.Ap[13] + IX(r0P + xm)));
        g[14] = ld(pick(14, (const T *)a.Ap[14] + IX(r0M + xp)));
        g[15] = ld(pick(15, (const T *)a.Ap[15] + IX(rMM + x)));
        g[16] = ld(pick(16, (const T *)a.Ap[16] + IX(rPP + x)));
        g[17] = ld(pick(17, (const T *)a.Ap[17] + IX(rMP + x)));
        g[18] = ld(pick(18, (const T *)a.Ap[18] + IX(rPM + x)));

        if (LBM_BULK_SPEC && BC == 1 && (fl & FL_SOLID)) continue;
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
                jx += R(0.5) * body_force<R>(a, 0);
                jy += R(0.5) * body_force<R>(a, 1);
                jz += R(0.5) * body_force<R>(a, 2);
            }
            const R rho = R(1) + drho;
            const int s = a.aux[c];
            if (s >= 0 && s < a.max_sites) {
                R *ru = (R *)a.sup_ru + 4 * (size_t)s;
                const R ir = R(1) / rho;
                ru[0] = rho;
                ru[1] = jx * ir;
                ru[2] = jy * ir;
                ru[3] = jz * ir;
            }
            // the streamed populations wait in B for the forced collision
            // (ibm_collide, in place), so every row of B is written whole
        } else {
            R rho, ux, uy, uz;
            const R fs = fluid ? R(1) : R(0);  // the body force acts on fluid cells only
            if constexpr (SRT && sizeof(R) == 4 && BC != 2 && LBM_SRT_FOLDED) {
                float u2;  // BC 0/1: only fluid cells collide
                collide_pairs<FORCE, scaled ? 10 : 0>(g, a.pk, rho, u2);
                if (!(rho > 0.5f && rho < 2.0f && u2 < 0.09f)) atomicOr(a.status, 1u);
            } else {
                collide<R, FORCE, SRT>(g, fs * body_force<R>(a, 0), fs * body_force<R>(a, 1), fs * body_force<R>(a, 2),
                                       a.rt, rho, ux, uy, uz);
                watchdog(rho, ux, uy, uz, a.status);
            }
        }
#pragma unroll
        for (int i = 0; i < 19; i++) {
            if constexpr (scaled) Store<LBM_F16S>::st_scaled((T *)a.Bp[i] + IX(c), g[i]);
            else Store<S>::st((T *)a.Bp[i] + IX(c), g[i]);
        }
        if (keep_walls && ((bd.y >> lane) & 1u)) {
            // a wall cell: the same 19 stored values, contiguous, for the ghost pass
            T *wv = (T *)a.bvals + (size_t)19 * (bd.x + __popc(bd.y & ((1u << lane) - 1u)));
#pragma unroll
            for (int i = 0; i < 19; i++) {
                if constexpr (scaled) Store<LBM_F16S>::st_scaled(wv + i, g[i]);
                else Store<S>::st(wv + i, g[i]);
            }
        }
    }
}

// ------------------------------------------------------------- launchers ---
template <int S, bool SRT, int BC>
static cudaError_t launch_bulk_t(Ctx &c, bool force) {
    SweepArgs a{};
    a.A = c.fA;
    a.B = c.fB;
    for (int i = 0; i < 19; i++) {
        a.Ap[i] = (const void *)((const char *)c.fA + storage_bytes(c.storage) * (size_t)i * (size_t)c.N);
        a.Bp[i] = (void *)((char *)c.fB + storage_bytes(c.storage) * (size_t)i * (size_t)c.N);
    }
    a.flags = c.flags;
    a.aux = c.aux;
    a.sup_ru = c.sup_ru;
    a.status = c.d_status;
    a.max_sites = c.max_sites;
    a.nx = c.nx;
    a.ny = c.ny;
    a.nz = c.nz;
    a.N = c.N;
    for (int d = 0; d < 3; d++) {
        a.F[d] = c.F[d];
        a.Fs[d] = (float)c.F[d];
    }
    a.rt = c.rt;
    a.pk = make_pair_k(c.rt.d_nu, c.F);
    const bool segs = BC == 1 && c.nseg > 0;
    a.seg_bnd = c.seg_bnd;
    a.bvals = (segs && c.bvals_ready && c.static_links && S != LBM_F64) ? c.bvals : nullptr;
    a.wrec = c.wrec;
    a.gvals = c.gvals;
    a.seg = c.seg;
    a.nseg = segs ? c.nseg : 0;
    a.fd_ny = FastDiv((unsigned)c.ny);
    a.fd_nx = FastDiv((unsigned)c.nx);
    const int bx = 256;  // 8 warps: one segment each, or 256 consecutive cells
    a.nflat = (c.N + bx - 1) / bx;
    long long nb = segs ? (c.nseg + 7) / 8 : a.nflat;
    if (LBM_BULK_PERSIST == 1 || (LBM_BULK_PERSIST == 2 && segs)) {
        // persistent grid: as many blocks as fit on the device at once
        static int resident[4][2][3][2];
        int &res = resident[S][SRT][BC][force ? 1 : 0];
        if (res == 0) {
            int per_sm = 0, dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (force)
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_collide_bulk<S, SRT, BC, true, true>, bx, 0);
            else
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_collide_bulk<S, SRT, BC, false, true>, bx, 0);
            res = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
        }
        if (nb > res) nb = res;
    }
    dim3 block(bx), grid((unsigned)nb);
    count_launch(c, G_BULK);
    const bool i32 = LBM_IDX32 && 19 * (unsigned long long)c.N + 64 < (1ULL << 32);
    if (force && i32)
        stream_collide_bulk<S, SRT, BC, true, true><<<grid, block, 0, c.stream>>>(a);
    else if (force)
        stream_collide_bulk<S, SRT, BC, true, false><<<grid, block, 0, c.stream>>>(a);
    else if (i32)
        stream_collide_bulk<S, SRT, BC, false, true><<<grid, block, 0, c.stream>>>(a);
    else
        stream_collide_bulk<S, SRT, BC, false, false><<<grid, block, 0, c.stream>>>(a);
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

#ifndef LBM_PIPE_SWEEP
#define LBM_PIPE_SWEEP 1  // 1: the lean static-wall sweep (sweep_pipe.cu) where it applies
#endif

cudaError_t launch_stream_collide(Ctx &c, int bc) {
    if (LBM_PIPE_SWEEP && bc == LBM_BC_IBB) {
        cudaError_t e = cudaSuccess;
        if (launch_pair16_sweep(c, e)) return e;
        if (launch_pipe_sweep(c, e)) return e;
    }
    const bool force = c.F[0] != 0.0 || c.F[1] != 0.0 || c.F[2] != 0.0;
    switch (c.storage) {
    case LBM_F64: return launch_bulk_s<LBM_F64>(c, bc, force);
    case LBM_F32: return launch_bulk_s<LBM_F32>(c, bc, force);
    case LBM_F16S: return launch_bulk_s<LBM_F16S>(c, bc, force);
    default: return launch_bulk_s<LBM_BF16S>(c, bc, force);
    }
}

}  // namespace lbmgb
