// Learned closure on the fifth-generation tensor cores (tcgen05): inference
// fused with the near-surface dissipation diagnostic, inference over a
// feature array, and training (loss, data and weight gradients; below).
//
// The closure (an 85-64-64-64-9 ReLU perceptron, see closure.cu) maps the
// IBM velocity stencil around a near-surface node to its 9 velocity
// gradients; the paper motivates it by IBM's underestimated dissipation
// inside the diffused interface (Sec. 3.2, Sec. 4).
//
// A CTA works on tiles of 128 samples (the MMA's M); over a feature array
// with 128 threads (a sample each, four CTAs per SM), fused with 256 in two
// roles (gather and layers, two CTAs per SM; see mlp_tc_field_ws_kernel):
// - inputs: either 85 FP32 features per sample read from memory
//   (lbm_mlp_forward), or, fused, gathered from an FP32 copy of the
//   velocity field at the listed near-surface cells (the 27-point stencil
//   of u - u_rb, the distance to the surface, u - u_rb at the node) -- no
//   feature array in HBM; rounded to BF16 into shared memory;
// - four layers, each: one elected thread issues tcgen05.mma (kind::f16,
//   BF16 operands from shared memory, FP32 accumulators in tensor memory)
//   over K in steps of 16 and commits to an mbarrier; the warps read the
//   accumulators back with tcgen05.ld (warp w: TMEM lanes 32 (w mod 4)..),
//   add the FP32 bias, apply ReLU and write the next layer's BF16 operand;
// - output: the 9 gradients (FP32), or, fused, the dissipation
//   2 nu s_ij s_ij of the predicted gradients at the cell.
// Operands use the no-swizzle K-major layout of 8 x 8 BF16 core matrices
// (128 B each): consecutive along K 128 B apart, along the rows K/8 x 128 B
// apart. The weights are the BF16 operand copies of closure.cu's packed
// block, rearranged into that layout once per CTA.
// Every wait on the mbarrier is bounded; a wait that runs out sets an error
// word, and the kernel frees its tensor memory and returns.
#include "lbm_internal.cuh"

namespace lbmgb {

size_t mlp_pack_bytes();

namespace {

constexpr int TM = 128, TK1 = 96, TKH = 64, TN4 = 16;
constexpr int TC_IN = 85, TC_H = 64, TC_OUT = 9;
// packed operand block of closure.cu: WT_l [out_pad][in_pad] (BF16)
constexpr int PW1 = 0, PW2 = PW1 + TC_H * TK1, PW3 = PW2 + TC_H * TC_H, PW4 = PW3 + TC_H * TC_H;
// flat FP32 parameter offsets of the biases
constexpr int OB1 = TC_IN * TC_H, OB2 = OB1 + TC_H + TC_H * TC_H, OB3 = OB2 + TC_H + TC_H * TC_H,
              OB4 = OB3 + TC_H + TC_H * TC_OUT;
constexpr long long TC_WAIT_LIMIT = 1LL << 24;  // polls of the mbarrier before giving up

struct __align__(128) TcSmem {
    unsigned short w1[TC_H * TK1];
    unsigned short w2[TC_H * TKH];
    unsigned short w3[TC_H * TKH];
    unsigned short w4[TN4 * TKH];
    unsigned short a[TM * TK1];  // the layer input (K = 96 for layer 1, 64 after)
    float b[208];                // b1 @0, b2 @64, b3 @128, b4 @192 (9 used)
    unsigned long long mbar;
    unsigned taddr;
    int err;
};

// element offset of (row r, column k) in the core-matrix layout of a K-wide operand
__device__ __forceinline__ int cm(int r, int k, int K) { return ((r >> 3) * (K >> 3) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K) and stride (row
// group) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(const void *p, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, N, M
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void tc_commit(void *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_wait(void *mbar, uint32_t parity) {
    const uint32_t m = smem_u32(mbar);
    for (long long it = 0; it < TC_WAIT_LIMIT; it++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(m), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t t, float v[32]) {
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(t));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t t, float v[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(t));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ unsigned bf2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&v);
}
// 8 values of one core-matrix row as one 16-byte store
__device__ __forceinline__ void put8(unsigned short *base, int off, const float *v) {
    *reinterpret_cast<uint4 *>(base + off) = make_uint4(bf2(v[0], v[1]), bf2(v[2], v[3]), bf2(v[4], v[5]), bf2(v[6], v[7]));
}


}  // namespace

struct TcArgs {
    const float *X;           // features (n x 85), or null: gather from the field
    float *Y;                 // outputs (n x 9), or null: dissipation at the cells
    const long long *count;   // device sample count (fused), else null
    long long n, cap;
    const float *w;           // FP32 parameters (biases)
    const unsigned short *pk; // packed BF16 operand block
    // fused: near-surface cells and their nearest particle
    const int *cells, *pid;
    const float4 *u;         // FP32 copy of the velocity field, (ux, uy, uz, 0) per cell
    const float4 *pf;        // per particle: closure_particle_kernel's record (4 float4)
    int nx, ny, nz;
    long long N;
    double inv_us, inv_gs, nu;
    float *eps_o;
    int *err;
};

// Per particle, for the gather: floor of the centre (int), the FP32
// offset of the centre from it, the radius, U and W (FP32). The features
// are rounded to BF16 (8 bits) at once, so FP32 is ample for them; the
// split centre keeps the offset to the particle exact to about 1e-7 lu at
// any box size (a plain FP32 centre would lose 3e-5 lu at 2^9).
__global__ void closure_particle_kernel(const double *X, const double *U, const double *W, const double *R, int np,
                                        float4 *pf) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const double x = X[3 * p], y = X[3 * p + 1], z = X[3 * p + 2];
    const double fx = floor(x), fy = floor(y), fz = floor(z);
    pf[4 * p] = make_float4(__int_as_float((int)fx), __int_as_float((int)fy), __int_as_float((int)fz), (float)R[p]);
    pf[4 * p + 1] = make_float4((float)(x - fx), (float)(y - fy), (float)(z - fz), 0.f);
    pf[4 * p + 2] = make_float4((float)U[3 * p], (float)U[3 * p + 1], (float)U[3 * p + 2], 0.f);
    pf[4 * p + 3] = make_float4((float)W[3 * p], (float)W[3 * p + 1], (float)W[3 * p + 2], 0.f);
}

__device__ __forceinline__ float fmimg(float d, int n) {
    const float h = 0.5f * (float)n;
    return d > h ? d - (float)n : (d < -h ? d + (float)n : d);
}

// The features of one sample, columns [48 H0, 48 H1) (H0 = 0, H1 = 2: all
// 96), BF16 into row `row` of the layer-1 operand, in two halves of 48
// columns: stencil points 0-15, then points 16-26, the distance to the
// surface, the node again and 11 zeros. Each half's 16-byte velocity loads
// are issued together.
template <int H0, int H1>
__device__ __forceinline__ void gather_put(const TcArgs &a, long long s, unsigned short *A, int row) {
    const unsigned c = (unsigned)a.cells[s];
    const int p = a.pid[s];
    const unsigned nxy = (unsigned)a.nx * (unsigned)a.ny;
    const unsigned z = c / nxy, rem = c - z * nxy, y = rem / (unsigned)a.nx, x = rem - y * (unsigned)a.nx;
    const float4 P0 = __ldg(a.pf + 4 * p), P1 = __ldg(a.pf + 4 * p + 1), Uv = __ldg(a.pf + 4 * p + 2),
                 Wv = __ldg(a.pf + 4 * p + 3);
    const float rx = fmimg((float)((int)x - __float_as_int(P0.x)) - P1.x, a.nx);
    const float ry = fmimg((float)((int)y - __float_as_int(P0.y)) - P1.y, a.ny);
    const float rz = fmimg((float)((int)z - __float_as_int(P0.z)) - P1.z, a.nz);
    const float ius = (float)a.inv_us;
    const int xm = x == 0 ? a.nx - 1 : (int)x - 1, xp = (int)x + 1 == a.nx ? 0 : (int)x + 1;
    const int ym = y == 0 ? a.ny - 1 : (int)y - 1, yp = (int)y + 1 == a.ny ? 0 : (int)y + 1;
    const int zm = z == 0 ? a.nz - 1 : (int)z - 1, zp = (int)z + 1 == a.nz ? 0 : (int)z + 1;
    auto addr = [&](int j) -> const float4 * {  // u at stencil point j (dz, dy, dx in -1..1, dz outermost)
        const int dx = j % 3 - 1, dy = (j / 3) % 3 - 1, dz = j / 9 - 1;
        const int xs = dx < 0 ? xm : (dx > 0 ? xp : (int)x), ys = dy < 0 ? ym : (dy > 0 ? yp : (int)y),
                  zs = dz < 0 ? zm : (dz > 0 ? zp : (int)z);
        return a.u + ((long long)xs + (long long)a.nx * (ys + (long long)a.ny * zs));
    };
    auto rel = [&](int j, const float4 &u, float *o) {  // u - u_rb at point j, scaled
        const float sx = rx + (float)(j % 3 - 1), sy = ry + (float)((j / 3) % 3 - 1), sz = rz + (float)(j / 9 - 1);
        o[0] = (u.x - (Uv.x + (Wv.y * sz - Wv.z * sy))) * ius;
        o[1] = (u.y - (Uv.y + (Wv.z * sx - Wv.x * sz))) * ius;
        o[2] = (u.z - (Uv.z + (Wv.x * sy - Wv.y * sx))) * ius;
    };
    // values go out 8 columns at a time (compile-time positions after unrolling)
    float buf[8];
    int fill = 0, col = 0;
    auto push = [&](float v) {
        buf[fill++] = v;
        if (fill == 8) {
            put8(A, cm(row, col, TK1), buf);
            col += 8;
            fill = 0;
        }
    };
    auto push_rel = [&](int j, const float4 &u) {
        float o[3];
        rel(j, u, o);
        push(o[0]);
        push(o[1]);
        push(o[2]);
    };
    if constexpr (H0 == 0) {
        float4 u[16];
#pragma unroll
        for (int t = 0; t < 16; t++) u[t] = __ldg(addr(t));
#pragma unroll
        for (int t = 0; t < 16; t++) push_rel(t, u[t]);
    }
    if constexpr (H1 == 2) {
        col = 48;
        float4 u[12];
#pragma unroll
        for (int t = 0; t < 11; t++) u[t] = __ldg(addr(16 + t));
        u[11] = __ldg(addr(13));
#pragma unroll
        for (int t = 0; t < 11; t++) push_rel(16 + t, u[t]);
        push(sqrtf(rx * rx + ry * ry + rz * rz) - P0.w);
        push_rel(13, u[11]);
#pragma unroll
        for (int k = 85; k < 96; k++) push(0.f);
    }
}

// Inference over a feature array (lbm_mlp_forward): 128 threads, a sample
// row each, four CTAs per SM (512 tensor-memory columns / 128 per CTA).
__global__ void __launch_bounds__(128, 4) mlp_tc_kernel(TcArgs a) {
    constexpr int TC_THREADS = 128;
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(tc_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long n = a.n;
    const long long tiles = (n + TM - 1) / TM;
    if ((long long)blockIdx.x >= tiles) return;  // the whole block leaves before any tensor memory is taken
    // weights into the core-matrix layout, biases
    for (int e = tid; e < TC_H * TK1; e += TC_THREADS) S.w1[cm(e / TK1, e % TK1, TK1)] = a.pk[PW1 + e];
    for (int e = tid; e < TC_H * TKH; e += TC_THREADS) {
        S.w2[cm(e / TKH, e % TKH, TKH)] = a.pk[PW2 + e];
        S.w3[cm(e / TKH, e % TKH, TKH)] = a.pk[PW3 + e];
    }
    for (int e = tid; e < TN4 * TKH; e += TC_THREADS) S.w4[cm(e / TKH, e % TKH, TKH)] = a.pk[PW4 + e];
    for (int i = tid; i < 208; i += TC_THREADS) {
        float v = 0.f;
        if (i < 64) v = a.w[OB1 + i];
        else if (i < 128) v = a.w[OB2 + i - 64];
        else if (i < 192) v = a.w[OB3 + i - 128];
        else if (i - 192 < TC_OUT) v = a.w[OB4 + i - 192];
        S.b[i] = v;
    }
    if (tid == 0) {
        S.err = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&S.taddr))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t T0 = S.taddr;                               // columns 0..63 and 64..127 of this CTA
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const int row = 32 * (warp & 3) + lane;                    // this thread's sample row in the tile
    uint32_t parity = 0;
    bool ok = true;
    // one layer: MMA over K into TMEM column base tc, then the epilogue of
    // 32 columns per thread into the next operand (K = 64)
    auto run_layer = [&](const unsigned short *w, int K, uint32_t tc, int N) {
        if (tid == 0) {
            fence_after();
            const uint32_t sbo = (uint32_t)(K / 8) * 128u;
            for (int s = 0; s < K / 16; s++)
                tc_mma(T0 + tc, sdesc(S.a + 128 * s, 128u, sbo), sdesc(w + 128 * s, 128u, sbo), idesc_bf16(TM, N),
                       s > 0 ? 1u : 0u);
            tc_commit(&S.mbar);
        }
        if (!mbar_wait(&S.mbar, parity)) ok = false;
        parity ^= 1u;
        fence_after();
    };
    // the MMA that read the operand has completed (its mbarrier), so the
    // epilogue overwrites the operand in place; 32 columns at a time
    auto hidden_out = [&](uint32_t tc, int boff) {
#pragma unroll
        for (int ch = 0; ch < 2; ch++) {
            const int c0 = 32 * ch;
            float v[32];
            tmem_ld32(T0 + lane_base + tc + c0, v);
#pragma unroll
            for (int j = 0; j < 32; j++) v[j] = fmaxf(v[j] + S.b[boff + c0 + j], 0.f);
#pragma unroll
            for (int g = 0; g < 4; g++) put8(S.a, cm(row, c0 + 8 * g, TKH), v + 8 * g);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
    };
    for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const long long s = tile * TM + row;
        // layer-1 operand: 85 features (BF16), zero padding to 96, zero rows past n
        {
            {
                // the tile's rows are one contiguous run of 85 x rows floats:
                // read it in coalesced 16-byte words (scalar where the words
                // would pass the array's end or the base is not 16-byte
                // aligned), each value to its (row, column) of the operand
                const long long r0 = tile * TM;
                const int rows = (int)(n - r0 < TM ? n - r0 : TM);
                const float *base = a.X + r0 * TC_IN;
                const int nv = rows * TC_IN;
                auto put1 = [&](int e, float v) {
                    const int r = e / TC_IN, k = e - r * TC_IN;
                    const __nv_bfloat16 b = __float2bfloat16_rn(v);
                    S.a[cm(r, k, TK1)] = *reinterpret_cast<const unsigned short *>(&b);
                };
                if ((reinterpret_cast<uintptr_t>(base) & 15) == 0) {
                    const float4 *b4 = reinterpret_cast<const float4 *>(base);
                    for (int f = tid; 4 * f + 3 < nv; f += TC_THREADS) {
                        const float4 v = __ldg(b4 + f);
                        put1(4 * f, v.x);
                        put1(4 * f + 1, v.y);
                        put1(4 * f + 2, v.z);
                        put1(4 * f + 3, v.w);
                    }
                    for (int e = (nv & ~3) + tid; e < nv; e += TC_THREADS) put1(e, __ldg(base + e));
                } else {
                    for (int e = tid; e < nv; e += TC_THREADS) put1(e, __ldg(base + e));
                }
                // zero padding columns 85..95, and whole rows past n
                for (int e = tid; e < TM * (TK1 - TC_IN); e += TC_THREADS) {
                    const int r = e / (TK1 - TC_IN), k = TC_IN + e % (TK1 - TC_IN);
                    S.a[cm(r, k, TK1)] = 0;
                }
                for (int e = rows * TC_IN + tid; e < TM * TC_IN; e += TC_THREADS) {
                    const int r = e / TC_IN, k = e - r * TC_IN;
                    S.a[cm(r, k, TK1)] = 0;
                }
            }
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        run_layer(S.w1, TK1, 0, TC_H);
        if (!ok) break;
        hidden_out(0, 0);
        run_layer(S.w2, TKH, 64, TC_H);
        if (!ok) break;
        hidden_out(64, 64);
        run_layer(S.w3, TKH, 0, TC_H);
        if (!ok) break;
        hidden_out(0, 128);
        run_layer(S.w4, TKH, 64, TN4);
        if (!ok) break;
        {
            float y[16];
            tmem_ld16(T0 + lane_base + 64, y);
            if (s < n) {
#pragma unroll
                for (int j = 0; j < TC_OUT; j++) a.Y[s * TC_OUT + j] = y[j] + S.b[192 + j];
            }
        }
        fence_before();
        __syncthreads();  // the next tile rewrites the operand and the accumulators
    }
    if (!ok && tid == 0) atomicExch(a.err, 1);
    fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(T0) : "memory");
}

// ------------------------------------------- fused inference, two roles --
// The fused diagnostic's form with the stencil gather overlapped with the
// layer chain: of the 256 threads, warps 4-7 gather tile t + 1 (a sample
// row each, all 28 points) into one of two input operands while warps 0-3
// (a TMEM lane each, 64 columns per epilogue) run the four layers of tile
// t from the other. Hand-off through mbarriers: full[b] (128 gather
// arrivals: the operand is written) and empty[b] (one arrival once the
// first layer's product has read it). Every wait is bounded; a wait that
// runs out sets the error word and its role stops, so the other role's
// waits run out too and the kernel frees its tensor memory and returns.
// (Measured: 0.154 ms per diagnostic of 1.26 M samples, 233 TFLOP/s,
// against 0.177 ms when every thread gathers and then runs the layers.)
namespace {
struct __align__(128) WsSmem {
    unsigned short w1[TC_H * TK1], w2[TC_H * TKH], w3[TC_H * TKH], w4[TN4 * TKH];
    unsigned short x[2][TM * TK1];  // input operands
    unsigned short h[TM * TKH];     // hidden operand
    float b[208];
    unsigned long long mma_bar, full[2], empty[2];
    unsigned taddr;
};
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
}  // namespace

__global__ void __launch_bounds__(256, 2) mlp_tc_field_ws_kernel(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char ws_smem_raw[];
    WsSmem &S = *reinterpret_cast<WsSmem *>(ws_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long n = *a.count < a.cap ? *a.count : a.cap;
    const long long tiles = (n + TM - 1) / TM;
    if ((long long)blockIdx.x >= tiles) return;  // the whole block leaves before any tensor memory is taken
    for (int e = tid; e < TC_H * TK1; e += 256) S.w1[cm(e / TK1, e % TK1, TK1)] = a.pk[PW1 + e];
    for (int e = tid; e < TC_H * TKH; e += 256) {
        S.w2[cm(e / TKH, e % TKH, TKH)] = a.pk[PW2 + e];
        S.w3[cm(e / TKH, e % TKH, TKH)] = a.pk[PW3 + e];
    }
    for (int e = tid; e < TN4 * TKH; e += 256) S.w4[cm(e / TKH, e % TKH, TKH)] = a.pk[PW4 + e];
    for (int i = tid; i < 208; i += 256) {
        float v = 0.f;
        if (i < 64) v = a.w[OB1 + i];
        else if (i < 128) v = a.w[OB2 + i - 64];
        else if (i < 192) v = a.w[OB3 + i - 128];
        else if (i - 192 < TC_OUT) v = a.w[OB4 + i - 192];
        S.b[i] = v;
    }
    if (tid == 0) {
        mbar_init(&S.mma_bar, 1);
        for (int b = 0; b < 2; b++) {
            mbar_init(&S.full[b], 128);
            mbar_init(&S.empty[b], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(smem_u32(&S.taddr))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t T0 = S.taddr;
    const int row = 32 * (warp & 3) + lane;
    bool ok = true;
    if (warp >= 4) {
        // gather role
        int k = 0;
        for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x, k++) {
            const int b = k & 1;
            if (k >= 2 && !mbar_wait(&S.empty[b], (uint32_t)(((k >> 1) - 1) & 1))) {
                ok = false;
                break;
            }
            const long long s = tile * TM + row;
            if (s < n) {
                gather_put<0, 2>(a, s, S.x[b], row);
            } else {
                const float f[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int g = 0; g < 12; g++) put8(S.x[b], cm(row, 8 * g, TK1), f);
            }
            fence_async_smem();  // the operand, to the tensor cores' proxy
            mbar_arrive(&S.full[b]);
        }
    } else {
        // layer role: thread `row` owns TMEM lane `row`
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        uint32_t mp = 0;
        auto layer = [&](const unsigned short *A, const unsigned short *W, int K, uint32_t tc, int N) -> bool {
            if (tid == 0) {
                fence_after();
                const uint32_t sbo = (uint32_t)(K / 8) * 128u;
                for (int st = 0; st < K / 16; st++)
                    tc_mma(T0 + tc, sdesc(A + 128 * st, 128u, sbo), sdesc(W + 128 * st, 128u, sbo), idesc_bf16(TM, N),
                           st > 0 ? 1u : 0u);
                tc_commit(&S.mma_bar);
            }
            const bool done = mbar_wait(&S.mma_bar, mp);
            mp ^= 1u;
            fence_after();
            return done;
        };
        auto hidden = [&](uint32_t tc, int boff) {
#pragma unroll
            for (int ch = 0; ch < 2; ch++) {
                float v[32];
                tmem_ld32(T0 + lane_base + tc + 32 * ch, v);
#pragma unroll
                for (int j = 0; j < 32; j++) v[j] = fmaxf(v[j] + S.b[boff + 32 * ch + j], 0.f);
#pragma unroll
                for (int g = 0; g < 4; g++) put8(S.h, cm(row, 32 * ch + 8 * g, TKH), v + 8 * g);
            }
            fence_async_smem();
            fence_before();
            consumers_sync();
        };
        int k = 0;
        for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x, k++) {
            const int b = k & 1;
            if (!mbar_wait(&S.full[b], (uint32_t)((k >> 1) & 1))) {
                ok = false;
                break;
            }
            fence_after();
            if (!layer(S.x[b], S.w1, TK1, 0, TC_H)) {
                ok = false;
                break;
            }
            if (tid == 0) mbar_arrive(&S.empty[b]);  // the input operand has been read
            hidden(0, 0);
            if (!layer(S.h, S.w2, TKH, 64, TC_H)) {
                ok = false;
                break;
            }
            hidden(64, 64);
            if (!layer(S.h, S.w3, TKH, 0, TC_H)) {
                ok = false;
                break;
            }
            hidden(0, 128);
            if (!layer(S.h, S.w4, TKH, 64, TN4)) {
                ok = false;
                break;
            }
            const long long s = tile * TM + row;
            float y[16];
            tmem_ld16(T0 + lane_base + 64, y);
            if (s < n) {
                const float igs = (float)a.inv_gs;
                float ss = 0.f;
#pragma unroll
                for (int p = 0; p < 3; p++)
#pragma unroll
                    for (int q = 0; q < 3; q++) {
                        const float sab = 0.5f * ((y[3 * p + q] + S.b[192 + 3 * p + q]) + (y[3 * q + p] + S.b[192 + 3 * q + p])) * igs;
                        ss = fmaf(sab, sab, ss);
                    }
                a.eps_o[a.cells[s]] = (float)(2.0 * a.nu) * ss;
            }
            fence_before();
            consumers_sync();  // the next tile's products rewrite the accumulators
        }
    }
    if (!ok) atomicExch(a.err, 1);
    fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(T0) : "memory");
}

static cudaError_t tc_launch(const TcArgs &a, bool field, long long max_tiles, cudaStream_t s) {
    static bool attr = false;
    const int smem = (int)sizeof(TcSmem), wsm = (int)sizeof(WsSmem);
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(mlp_tc_field_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, wsm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long nb = (long long)(field ? 2 : 4) * (sms > 0 ? sms : 1);
    if (nb > max_tiles) nb = max_tiles;
    if (nb < 1) nb = 1;
    if (field) mlp_tc_field_ws_kernel<<<(unsigned)nb, 256, wsm, s>>>(a);
    else mlp_tc_kernel<<<(unsigned)nb, 128, smem, s>>>(a);
    return cudaGetLastError();
}

// ------------------------------------------------------------ training --
// Loss and gradient of a batch on tcgen05. One CTA (128 threads, a sample
// row each; one CTA per SM: 185 KB of shared memory, all 512 tensor-memory
// columns) runs tiles of 128 samples:
// - forward as in inference, keeping the three hidden activations (BF16);
// - the output gradient dZ4 = 2 (Y - T) / (9 n), then per layer k = 4..1
//   the weight gradient  dW_k += [H_{k-1}; 1]^T dZ_k  (M = 128 input rows
//   with a row of ones whose product is the bias gradient, N = units,
//   K = the 128 samples) accumulated in tensor memory over the CTA's tiles,
//   and the data gradient dH_{k-1} = dZ_k W_k^T masked by the ReLU;
// - both products take BF16 operands (the activations, dZ_k and the
//   weights, as the tensor cores require) and add in FP32.
// The transposed operands are written by the epilogues (each thread holds
// one sample, so it writes one column of [H_{k-1}; 1]^T and of dZ_k^T).
// At the end every thread reads its row of the four accumulators and
// writes this CTA's gradient slot; the Adam kernel sums the slots in a
// fixed order.
// Tensor-memory columns: 0-63 the layer product, 64-127 dW1, 128-191 dW2,
// 192-255 dW3, 256-271 dW4.
namespace {
constexpr int PB2 = PW4 + TN4 * TKH, PB3 = PB2 + TC_H * TC_H, PB4 = PB3 + TC_H * TC_H;  // backward operand blocks
constexpr int TK_T = 128;  // K of the weight-gradient products (samples of a tile)

struct __align__(128) TrainTcSmem {
    unsigned short w1[TC_H * TK1], w2[TC_H * TKH], w3[TC_H * TKH], w4[TN4 * TKH];  // forward B: [out][in]
    unsigned short v2[TC_H * TC_H], v3[TC_H * TC_H], v4[TC_H * TN4];              // backward B: [in][out]
    unsigned short x0[TM * TK1];      // layer-1 operand
    unsigned short h[3][TM * TKH];    // hidden activations
    unsigned short at[TM * TK_T];     // [H_{k-1}; 1]^T, rows padded to 128 with zeros
    unsigned short dz[TM * TKH];      // dZ_k (A of the data gradient), K = units
    unsigned short dzt[TC_H * TK_T];  // dZ_k^T (B of the weight gradient), K = samples
    float b[208];
    unsigned long long mbar;
    unsigned taddr;
    float loss[4];
};

__device__ __forceinline__ unsigned short bf16_bits(float v) {
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    return *reinterpret_cast<const unsigned short *>(&b);
}
}  // namespace

struct TrainTcArgs {
    const float *X, *T;
    long long s0, s1;
    float inv;  // 2 / (9 n) of the batch
    const float *w;
    const unsigned short *pk;
    float *gpart, *lpart;
    int *err;
};

__global__ void __launch_bounds__(TM, 1) mlp_train_tc_kernel(TrainTcArgs a) {
    extern __shared__ __align__(1024) unsigned char tt_smem_raw[];
    TrainTcSmem &S = *reinterpret_cast<TrainTcSmem *>(tt_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long n = a.s1 - a.s0;
    const long long tiles = (n + TM - 1) / TM;
    for (int e = tid; e < TC_H * TK1; e += TM) S.w1[cm(e / TK1, e % TK1, TK1)] = a.pk[PW1 + e];
    for (int e = tid; e < TC_H * TKH; e += TM) {
        S.w2[cm(e / TKH, e % TKH, TKH)] = a.pk[PW2 + e];
        S.w3[cm(e / TKH, e % TKH, TKH)] = a.pk[PW3 + e];
        S.v2[cm(e / TC_H, e % TC_H, TC_H)] = a.pk[PB2 + e];
        S.v3[cm(e / TC_H, e % TC_H, TC_H)] = a.pk[PB3 + e];
    }
    for (int e = tid; e < TN4 * TKH; e += TM) {
        S.w4[cm(e / TKH, e % TKH, TKH)] = a.pk[PW4 + e];
        S.v4[cm(e / TN4, e % TN4, TN4)] = a.pk[PB4 + e];
    }
    for (int i = tid; i < 208; i += TM) {
        float v = 0.f;
        if (i < 64) v = a.w[OB1 + i];
        else if (i < 128) v = a.w[OB2 + i - 64];
        else if (i < 192) v = a.w[OB3 + i - 128];
        else if (i - 192 < TC_OUT) v = a.w[OB4 + i - 192];
        S.b[i] = v;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&S.taddr))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t T0 = S.taddr;
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const int row = tid;  // this thread's sample in the tile, and its row of the weight-gradient accumulators
    uint32_t parity = 0;
    bool ok = true;
    float lsum = 0.f;
    bool first = true;  // the CTA's first weight-gradient product overwrites the accumulators
    auto sync_operands = [&]() {  // generic shared-memory writes -> the tensor cores
        fence_async_smem();
        fence_before();
        __syncthreads();
    };
    auto wait_mma = [&]() {
        if (!mbar_wait(&S.mbar, parity)) ok = false;
        parity ^= 1u;
        fence_after();
    };
    // D (TMEM column tc) = A (K-major, K columns) x B^T (N rows, K-major)
    auto mma = [&](uint32_t tc, const unsigned short *A, const unsigned short *B, int K, int N, bool acc) {
        const uint32_t sbo = (uint32_t)(K / 8) * 128u;
        for (int s = 0; s < K / 16; s++)
            tc_mma(T0 + tc, sdesc(A + 128 * s, 128u, sbo), sdesc(B + 128 * s, 128u, sbo), idesc_bf16(TM, N),
                   (acc || s > 0) ? 1u : 0u);
    };
    auto issue = [&](auto &&body) {  // one thread issues, commits; all wait
        if (tid == 0) {
            fence_after();
            body();
            tc_commit(&S.mbar);
        }
        wait_mma();
    };
    // hidden epilogue: relu(D + b) -> h[k] (this thread's row)
    auto hidden = [&](unsigned short *H, int boff) {
#pragma unroll
        for (int ch = 0; ch < 2; ch++) {
            float v[32];
            tmem_ld32(T0 + lane_base + 32 * ch, v);
#pragma unroll
            for (int j = 0; j < 32; j++) v[j] = fmaxf(v[j] + S.b[boff + 32 * ch + j], 0.f);
#pragma unroll
            for (int g = 0; g < 4; g++) put8(H, cm(row, 32 * ch + 8 * g, TKH), v + 8 * g);
        }
        sync_operands();
    };
    // column `row` of [src; 1]^T (src: this thread's row of a K-major operand with `cols` columns)
    auto transpose_in = [&](const unsigned short *src, int cols, int ones_row) {
        for (int j0 = 0; j0 < cols; j0 += 8) {
            const uint4 q = *reinterpret_cast<const uint4 *>(src + cm(row, j0, cols));
            const unsigned w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int t = 0; t < 8; t++) S.at[cm(j0 + t, row, TK_T)] = (unsigned short)(w4[t >> 1] >> (16 * (t & 1)));
        }
        S.at[cm(ones_row, row, TK_T)] = bf16_bits(1.f);
        for (int j = ones_row + 1; j < TM; j++) S.at[cm(j, row, TK_T)] = 0;
    };
    // data-gradient epilogue: dZ = D masked by relu'(h) -> dz (unless last) and dz^T
    auto backward = [&](const unsigned short *H, bool keep_dz) {
#pragma unroll
        for (int ch = 0; ch < 2; ch++) {
            float v[32];
            tmem_ld32(T0 + lane_base + 32 * ch, v);
#pragma unroll
            for (int g = 0; g < 4; g++) {
                const int j0 = 32 * ch + 8 * g;
                const uint4 q = *reinterpret_cast<const uint4 *>(H + cm(row, j0, TKH));
                const unsigned w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int t = 0; t < 8; t++) {
                    const unsigned short hb = (unsigned short)(w4[t >> 1] >> (16 * (t & 1)));
                    if (hb == 0 || (hb & 0x8000u)) v[8 * g + t] = 0.f;  // relu'(h) = 0 where h <= 0
                    S.dzt[cm(j0 + t, row, TK_T)] = bf16_bits(v[8 * g + t]);
                }
                if (keep_dz) put8(S.dz, cm(row, j0, TKH), v + 8 * g);
            }
        }
    };
    for (long long tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const long long r0 = tile * TM;
        const int rows = (int)(n - r0 < TM ? n - r0 : TM);
        const long long srow = a.s0 + r0 + row;
        // layer-1 operand: coalesced 16-byte words when the rows start aligned
        {
            const float *base = a.X + (a.s0 + r0) * TC_IN;
            const int nv = rows * TC_IN;
            auto put1 = [&](int e, float v) {
                const int r = e / TC_IN, k = e - r * TC_IN;
                S.x0[cm(r, k, TK1)] = bf16_bits(v);
            };
            if ((reinterpret_cast<uintptr_t>(base) & 15) == 0) {
                const float4 *b4 = reinterpret_cast<const float4 *>(base);
                for (int f = tid; 4 * f + 3 < nv; f += TM) {
                    const float4 v = __ldg(b4 + f);
                    put1(4 * f, v.x);
                    put1(4 * f + 1, v.y);
                    put1(4 * f + 2, v.z);
                    put1(4 * f + 3, v.w);
                }
                for (int e = (nv & ~3) + tid; e < nv; e += TM) put1(e, __ldg(base + e));
            } else {
                for (int e = tid; e < nv; e += TM) put1(e, __ldg(base + e));
            }
            for (int k = TC_IN; k < TK1; k++) S.x0[cm(row, k, TK1)] = 0;
            if (row >= rows)
                for (int k = 0; k < TC_IN; k++) S.x0[cm(row, k, TK1)] = 0;
        }
        sync_operands();
        // forward
        issue([&] { mma(0, S.x0, S.w1, TK1, TC_H, false); });
        if (!ok) break;
        hidden(S.h[0], 0);
        issue([&] { mma(0, S.h[0], S.w2, TKH, TC_H, false); });
        if (!ok) break;
        hidden(S.h[1], 64);
        issue([&] { mma(0, S.h[1], S.w3, TKH, TC_H, false); });
        if (!ok) break;
        hidden(S.h[2], 128);
        issue([&] { mma(0, S.h[2], S.w4, TKH, TN4, false); });
        if (!ok) break;
        // output gradient of the tile (zero for rows past the batch)
        {
            float y[16], d[16];
            tmem_ld16(T0 + lane_base, y);
#pragma unroll
            for (int o = 0; o < 16; o++) {
                d[o] = 0.f;
                if (o < TC_OUT && row < rows) {
                    const float r = y[o] + S.b[192 + o] - __ldg(a.T + srow * TC_OUT + o);
                    lsum = fmaf(r, r, lsum);
                    d[o] = a.inv * r;
                }
            }
            put8(S.dz, cm(row, 0, TN4), d);
            put8(S.dz, cm(row, 8, TN4), d + 8);
#pragma unroll
            for (int o = 0; o < 16; o++) S.dzt[cm(o, row, TK_T)] = bf16_bits(d[o]);
            transpose_in(S.h[2], TKH, TC_H);
        }
        sync_operands();
        // layer 4: dW4 += [H3; 1]^T dZ4, dH3 = dZ4 W4^T
        issue([&] {
            mma(256, S.at, S.dzt, TK_T, TN4, !first);
            mma(0, S.dz, S.v4, TN4, TC_H, false);
        });
        if (!ok) break;
        backward(S.h[2], true);
        transpose_in(S.h[1], TKH, TC_H);
        sync_operands();
        // layer 3
        issue([&] {
            mma(192, S.at, S.dzt, TK_T, TC_H, !first);
            mma(0, S.dz, S.v3, TKH, TC_H, false);
        });
        if (!ok) break;
        backward(S.h[1], true);
        transpose_in(S.h[0], TKH, TC_H);
        sync_operands();
        // layer 2
        issue([&] {
            mma(128, S.at, S.dzt, TK_T, TC_H, !first);
            mma(0, S.dz, S.v2, TKH, TC_H, false);
        });
        if (!ok) break;
        backward(S.h[0], false);
        transpose_in(S.x0, TK1, TK1);  // the 85 inputs (zero-padded to 96), ones at row 96
        sync_operands();
        // layer 1
        issue([&] { mma(64, S.at, S.dzt, TK_T, TC_H, !first); });
        if (!ok) break;
        first = false;
    }
    // this CTA's gradient slot: thread `row` holds row `row` of each accumulator
    if (ok) {
        float *g = a.gpart + (size_t)blockIdx.x * (size_t)(OB4 + TC_OUT);
#pragma unroll 1
        for (int L = 0; L < 3; L++) {
            const int nin = L == 0 ? TC_IN : TC_H, ones = L == 0 ? TK1 : TC_H;
            const int offw = L == 0 ? 0 : (L == 1 ? OB1 + TC_H : OB2 + TC_H), offb = L == 0 ? OB1 : (L == 1 ? OB2 : OB3);
            for (int ch = 0; ch < 2; ch++) {
                float v[32];
                tmem_ld32(T0 + lane_base + 64 * (L + 1) + 32 * ch, v);
                if (row < nin)
                    for (int o = 0; o < 32; o++) g[offw + row * TC_H + 32 * ch + o] = first ? 0.f : v[o];
                else if (row == ones)
                    for (int o = 0; o < 32; o++) g[offb + 32 * ch + o] = first ? 0.f : v[o];
            }
        }
        {
            float v[16];
            tmem_ld16(T0 + lane_base + 256, v);
            if (row < TC_H)
                for (int o = 0; o < TC_OUT; o++) g[OB3 + TC_H + row * TC_OUT + o] = first ? 0.f : v[o];
            else if (row == TC_H)
                for (int o = 0; o < TC_OUT; o++) g[OB4 + o] = first ? 0.f : v[o];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) S.loss[warp] = lsum;
    if (!ok && tid == 0) atomicExch(a.err, 1);
    fence_before();
    __syncthreads();
    if (tid == 0) a.lpart[blockIdx.x] = S.loss[0] + S.loss[1] + S.loss[2] + S.loss[3];
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(T0) : "memory");
}

// Gradient slots (one per CTA) and loss partials of the batch [s0, s1).
cudaError_t mlp_train_tc(const float *X, const float *T, long long s0, long long s1, const float *w, const void *pk,
                         float *gpart, float *lpart, int max_blocks, int *err, cudaStream_t s, int *nblk_out) {
    static bool attr = false;
    const int smem = (int)sizeof(TrainTcSmem);
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(mlp_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long tiles = (s1 - s0 + TM - 1) / TM;
    int nb = (int)(tiles < max_blocks ? tiles : max_blocks);
    if (nb < 1) nb = 1;
    TrainTcArgs a;
    a.X = X;
    a.T = T;
    a.s0 = s0;
    a.s1 = s1;
    a.inv = 2.0f / (float)((double)(s1 - s0) * TC_OUT);
    a.w = w;
    a.pk = (const unsigned short *)pk;
    a.gpart = gpart;
    a.lpart = lpart;
    a.err = err;
    mlp_train_tc_kernel<<<nb, TM, smem, s>>>(a);
    *nblk_out = nb;
    return cudaGetLastError();
}

// Y (n x 9) = network(X (n x 85)); pk: the packed BF16 operand block of w.
cudaError_t mlp_forward_tc(const float *X, long long n, const float *w, const void *pk, float *Y, int *err,
                           cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    TcArgs a{};
    a.X = X;
    a.Y = Y;
    a.n = n;
    a.w = w;
    a.pk = (const unsigned short *)pk;
    a.err = err;
    return tc_launch(a, false, (n + TM - 1) / TM, s);
}

// dissipation 2 nu s_ij s_ij of the network's gradients (times 1/g_scale)
// at the listed near-surface cells into eps_o; the count is read on the device
cudaError_t closure_eps_tc(const Ctx &c, const float *u32, const int *cells, const int *pid, const long long *count,
                           long long cap, const void *pk, float *eps_o, int *err) {
    TcArgs a{};
    a.count = count;
    a.cap = cap;
    a.w = c.cl_w;
    a.pk = (const unsigned short *)pk;
    a.cells = cells;
    a.pid = pid;
    a.u = reinterpret_cast<const float4 *>(u32);
    // FP32 particle records in the closure's output buffer (unused by the fused path)
    float4 *pf = (float4 *)c.cl_Y;
    closure_particle_kernel<<<(c.np + 255) / 256, 256, 0, c.stream>>>(c.X, c.U, c.W, c.R, c.np, pf);
    a.pf = pf;
    a.nx = c.nx;
    a.ny = c.ny;
    a.nz = c.nz;
    a.N = c.N;
    a.inv_us = 1.0 / c.cl_uscale;
    a.inv_gs = 1.0 / c.cl_gscale;
    a.nu = (c.tau - 0.5) / 3.0;
    a.eps_o = eps_o;
    a.err = err;
    return tc_launch(a, true, (cap + TM - 1) / TM, c.stream);
}

}  // namespace lbmgb
