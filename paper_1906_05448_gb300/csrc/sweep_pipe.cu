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
//   pulls from solid nodes, and keeps the wall cells' 19 values for the
//   next ghost pass.
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
    const void *gvals;     // compact ghost values of this step
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

#ifndef LBM_PIPE_ITEMS
#define LBM_PIPE_ITEMS 1  // warp items a warp sweeps together (1 or 2)
#endif
#ifndef LBM_PIPE_MINB
#define LBM_PIPE_MINB 0  // resident blocks of 256 per SM the registers are sized for (0: per storage)
#endif
// measured on the benchmark pipe: FP32 is fastest at 4 blocks (64
// registers), 16-bit storage at 5 (48 registers, more loads in flight)
constexpr int pipe_min_blocks(int S) { return LBM_PIPE_MINB > 0 ? LBM_PIPE_MINB : (S == LBM_F32 ? 4 : 5); }

// NI warp items per warp and round: the records of the next round are
// loaded one round ahead, the populations of all NI items are requested
// before any of them is collided, so each thread has NI x 19 loads in flight.
template <int S, bool FORCE, int NI>
__global__ void __launch_bounds__(256, pipe_min_blocks(S)) stream_collide_pipe(PipeArgs a) {
    typedef typename Store<S>::T T;
    // FP16 keeps g * 2^10: the collision runs on the stored numbers
    constexpr bool scaled = S == LBM_F16S;
    constexpr int SC = scaled ? 10 : 0;
    auto cvt = [](T v) -> float {
        if constexpr (S == LBM_F32) return v;
        else if constexpr (scaled) return __half2float(v);
        else return __bfloat162float(v);
    };
    auto st = [](T *p, float v) {
        if constexpr (scaled) Store<LBM_F16S>::st_scaled(p, v);
        else Store<S>::st(p, v);
    };
    const int lane = threadIdx.x & 31;
    const long long items = a.nseg;
    const long long gw = (long long)gridDim.x * (blockDim.x / 32);  // warps in the grid
    const T *__restrict__ A = (const T *)a.A;
    const unsigned N = a.N;
    const bool keep_walls = a.bvals != nullptr;
    auto wall_record = [&](uint2 bdv) -> uint2 {
        if (!((bdv.y >> lane) & 1u)) return make_uint2(0u, 0u);
        return __ldg(a.wrec + bdv.x + __popc(bdv.y & ((1u << lane) - 1u)));
    };
    uint4 sgn[NI];
    uint2 bdn[NI], wrn[NI];
    auto fetch = [&](long long w, int j) {
        sgn[j] = make_uint4(0u, 0u, 0u, 0u);
        bdn[j] = wrn[j] = make_uint2(0u, 0u);
        if (w < items) {
            sgn[j] = __ldg(a.seg + w);
            if (keep_walls) {
                bdn[j] = __ldg(a.seg_bnd + w);
                wrn[j] = wall_record(bdn[j]);
            }
        }
    };
    const long long w0 = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
#pragma unroll
    for (int j = 0; j < NI; j++) fetch(w0 + j * gw, j);
    for (long long w = w0; w < items; w += NI * gw) {
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
                const T *gv = keep_walls ? (const T *)a.gvals + wr[j].x : A;
                const unsigned m = wr[j].y;
#pragma unroll
                for (int i = 0; i < 19; i++)
                    raw[j][i] = __ldg(((m >> i) & 1u) ? gv + __popc(m & ((1u << i) - 1u)) : pull(i));
            }
        }
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
    }
}

template <int S>
static cudaError_t launch_pipe_t(Ctx &c, bool force) {
    PipeArgs a{};
    a.A = c.fA;
    a.B = c.fB;
    a.seg = c.seg;
    a.nseg = c.nseg;
    a.seg_bnd = c.seg_bnd;
    a.bvals = (c.bvals_ready && c.static_links) ? c.bvals : nullptr;
    a.wrec = c.wrec;
    a.gvals = c.gvals;
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
    static int resident[4][2];
    int &res = resident[S][force ? 1 : 0];
    if (res == 0) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (force)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_collide_pipe<S, true, LBM_PIPE_ITEMS>, 256, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stream_collide_pipe<S, false, LBM_PIPE_ITEMS>, 256, 0);
        res = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    long long nb = (c.nseg + 7) / 8;
    if (nb > res) nb = res;
    if (nb < 1) nb = 1;
    count_launch(c, G_BULK);
    if (force) stream_collide_pipe<S, true, LBM_PIPE_ITEMS><<<(unsigned)nb, 256, 0, c.stream>>>(a);
    else stream_collide_pipe<S, false, LBM_PIPE_ITEMS><<<(unsigned)nb, 256, 0, c.stream>>>(a);
    return cudaGetLastError();
}

// The lean sweep serves the static-wall IBB step with the single relaxation
// rate, 32- or 16-bit storage, a segment work list whose fluid cells do not
// touch the x or y faces, and 19 N < 2^32. Returns false (nothing launched)
// otherwise.
bool launch_pipe_sweep(Ctx &c, cudaError_t &err) {
    if (!c.pipe_nowrap || c.nseg <= 0 || c.rates != LBM_RATES_SRT || c.storage == LBM_F64 || c.np > 0 ||
        19ULL * (unsigned long long)c.N + 64 >= (1ULL << 32))
        return false;
    const bool force = c.F[0] != 0.0 || c.F[1] != 0.0 || c.F[2] != 0.0;
    switch (c.storage) {
    case LBM_F32: err = launch_pipe_t<LBM_F32>(c, force); break;
    case LBM_F16S: err = launch_pipe_t<LBM_F16S>(c, force); break;
    default: err = launch_pipe_t<LBM_BF16S>(c, force); break;
    }
    return true;
}

}  // namespace lbmgb
