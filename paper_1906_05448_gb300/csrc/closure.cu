// Learned near-surface gradient closure: an 85-64-64-64-9 ReLU perceptron.
// Training on tensor cores with mma.sync m16n8k16 (BF16 operands, FP32
// accumulation); inference runs on tcgen05 (closure_tc.cu).
//
// The paper has no closure; it motivates one: inside IBM's diffused
// interface the velocity gradients, hence the dissipation, come out too low
// (Sec. 3.2, Sec. 4). The network maps the local IBM velocity stencil
// (relative to the particle's rigid-body motion), the signed distance to the
// surface and the relative velocity to the 9 velocity-gradient components.
//
// Flat FP32 parameter vector (same order as the oracle): W1 [85][64], b1,
// W2 [64][64], b2, W3 [64][64], b3, W4 [64][9], b4 -- each W stored
// [in][out]. Kernels take BF16 copies packed for the MMA operands:
//   forward B operands  WT_l [out_pad][in_pad]  (in padded 85 -> 96, out 9 -> 16)
//   backward B operands W_l  [in][out_pad]      (layers 2..4)
// Training: each block runs forward and backward on tiles of 64 samples
// (warp = 16 samples), accumulates its weight gradient in shared memory and
// writes it to its own slot; a second kernel sums the slots in a fixed order
// and applies Adam to the FP32 master weights (deterministic).
#include "lbm_internal.cuh"

#include <cstring>
#include <vector>

namespace lbmgb {

constexpr int MIN = 85, MIN_P = 96, MH = 64, MOUT = 9, MOUT_P = 16;
constexpr int NPARAM = MIN * MH + MH + 2 * (MH * MH + MH) + MH * MOUT + MOUT;  // 14409
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MIN * MH, OFF_W2 = OFF_B1 + MH, OFF_B2 = OFF_W2 + MH * MH,
              OFF_W3 = OFF_B2 + MH, OFF_B3 = OFF_W3 + MH * MH, OFF_W4 = OFF_B3 + MH, OFF_B4 = OFF_W4 + MH * MOUT;
// packed BF16 operand block (element offsets)
constexpr int PK_WT1 = 0, PK_WT2 = PK_WT1 + MH * MIN_P, PK_WT3 = PK_WT2 + MH * MH, PK_WT4 = PK_WT3 + MH * MH,
              PK_W2 = PK_WT4 + MOUT_P * MH, PK_W3 = PK_W2 + MH * MH, PK_W4 = PK_W3 + MH * MH,
              PK_TOTAL = PK_W4 + MH * MOUT_P;
constexpr int PK_FWD = PK_W2;  // forward needs only the WT blocks

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&v);
}

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// B fragment of a K x N operand stored as [N][K] (row length K)
__device__ __forceinline__ void load_b(const __nv_bfloat16 *B, int K, int ntile, int kstep, int lane, unsigned &b0,
                                       unsigned &b1) {
    const int n = ntile * 8 + (lane >> 2), k = kstep * 16 + (lane & 3) * 2;
    b0 = *reinterpret_cast<const unsigned *>(B + n * K + k);
    b1 = *reinterpret_cast<const unsigned *>(B + n * K + k + 8);
}

// C fragments (16 x 8 tiles, fp32) of an activation -> A fragments (bf16)
template <int NT>
__device__ __forceinline__ void c_to_a(const float c[NT][4], unsigned a[NT / 2][4]) {
#pragma unroll
    for (int kk = 0; kk < NT / 2; kk++) {
        a[kk][0] = pack_bf16(c[2 * kk][0], c[2 * kk][1]);
        a[kk][1] = pack_bf16(c[2 * kk][2], c[2 * kk][3]);
        a[kk][2] = pack_bf16(c[2 * kk + 1][0], c[2 * kk + 1][1]);
        a[kk][3] = pack_bf16(c[2 * kk + 1][2], c[2 * kk + 1][3]);
    }
}

// Forward of one warp tile of 16 samples (rows r0 = base + lane/4, r1 = r0 + 8).
// h1..h3: post-ReLU activations, y: outputs, all in C-fragment layout.
__device__ __forceinline__ void warp_forward(const float *X, long long n, long long base, const __nv_bfloat16 *sw,
                                             const float *sb, int lane, float h1[8][4], float h2[8][4], float h3[8][4],
                                             float y[2][4]) {
    const int gid = lane >> 2, tig = lane & 3;
    const long long r0 = base + gid, r1 = base + gid + 8;
    unsigned ax[6][4];
#pragma unroll
    for (int kk = 0; kk < 6; kk++) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int col = kk * 16 + tig * 2 + (e & 1) + ((e >> 2) ? 8 : 0);
            const long long row = (e & 2) ? r1 : r0;
            v[e] = (col < MIN && row < n) ? X[row * MIN + col] : 0.f;
        }
        ax[kk][0] = pack_bf16(v[0], v[1]);
        ax[kk][1] = pack_bf16(v[2], v[3]);
        ax[kk][2] = pack_bf16(v[4], v[5]);
        ax[kk][3] = pack_bf16(v[6], v[7]);
    }
    const int cb = tig * 2;
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < 6; kk++) {
            unsigned b0, b1;
            load_b(sw + PK_WT1, MIN_P, nt, kk, lane, b0, b1);
            mma_bf16(c, ax[kk], b0, b1);
        }
        const float bl = sb[nt * 8 + cb], bh = sb[nt * 8 + cb + 1];
        h1[nt][0] = fmaxf(c[0] + bl, 0.f);
        h1[nt][1] = fmaxf(c[1] + bh, 0.f);
        h1[nt][2] = fmaxf(c[2] + bl, 0.f);
        h1[nt][3] = fmaxf(c[3] + bh, 0.f);
    }
    unsigned a[4][4];
    c_to_a<8>(h1, a);
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            unsigned b0, b1;
            load_b(sw + PK_WT2, MH, nt, kk, lane, b0, b1);
            mma_bf16(c, a[kk], b0, b1);
        }
        const float bl = sb[64 + nt * 8 + cb], bh = sb[64 + nt * 8 + cb + 1];
        h2[nt][0] = fmaxf(c[0] + bl, 0.f);
        h2[nt][1] = fmaxf(c[1] + bh, 0.f);
        h2[nt][2] = fmaxf(c[2] + bl, 0.f);
        h2[nt][3] = fmaxf(c[3] + bh, 0.f);
    }
    c_to_a<8>(h2, a);
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            unsigned b0, b1;
            load_b(sw + PK_WT3, MH, nt, kk, lane, b0, b1);
            mma_bf16(c, a[kk], b0, b1);
        }
        const float bl = sb[128 + nt * 8 + cb], bh = sb[128 + nt * 8 + cb + 1];
        h3[nt][0] = fmaxf(c[0] + bl, 0.f);
        h3[nt][1] = fmaxf(c[1] + bh, 0.f);
        h3[nt][2] = fmaxf(c[2] + bl, 0.f);
        h3[nt][3] = fmaxf(c[3] + bh, 0.f);
    }
    c_to_a<8>(h3, a);
#pragma unroll
    for (int nt = 0; nt < 2; nt++) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < 4; kk++) {
            unsigned b0, b1;
            load_b(sw + PK_WT4, MH, nt, kk, lane, b0, b1);
            mma_bf16(c, a[kk], b0, b1);
        }
        const int col = nt * 8 + cb;
        const float bl = col < MOUT ? sb[192 + col] : 0.f, bh = col + 1 < MOUT ? sb[192 + col + 1] : 0.f;
        y[nt][0] = c[0] + bl;
        y[nt][1] = c[1] + bh;
        y[nt][2] = c[2] + bl;
        y[nt][3] = c[3] + bh;
    }
}

// biases of the four layers in shared memory: b1 @0, b2 @64, b3 @128, b4 @192
__device__ __forceinline__ void load_params(const __nv_bfloat16 *pk, const float *w, __nv_bfloat16 *sw, float *sb,
                                            int count) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) sw[i] = pk[i];
    for (int i = threadIdx.x; i < 208; i += blockDim.x) {
        float v;
        if (i < 64) v = w[OFF_B1 + i];
        else if (i < 128) v = w[OFF_B2 + i - 64];
        else if (i < 192) v = w[OFF_B3 + i - 128];
        else v = (i - 192) < MOUT ? w[OFF_B4 + i - 192] : 0.f;
        sb[i] = v;
    }
    __syncthreads();
}

// --------------------------------------------------------------- training --
constexpr int TB = 64;  // samples per block tile (4 warps x 16)

struct TrainSmem {
    __nv_bfloat16 w[PK_TOTAL];
    float b[208];
    float H[TB * MIN_P];    // staged layer input, row-major [sample][feature]
    float D[TB * MH];       // staged pre-activation gradient [sample][unit]
    float g[NPARAM];        // this block's gradient
    float loss[4];
};

// store a C-fragment activation block (16 rows x NT*8 cols) of warp `warp` to smem rows
template <int NT>
__device__ __forceinline__ void stage_c(float *S, int ld, const float c[NT][4], int warp, int lane) {
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
        const int col = nt * 8 + tig * 2;
        S[(warp * 16 + gid) * ld + col] = c[nt][0];
        S[(warp * 16 + gid) * ld + col + 1] = c[nt][1];
        S[(warp * 16 + gid + 8) * ld + col] = c[nt][2];
        S[(warp * 16 + gid + 8) * ld + col + 1] = c[nt][3];
    }
}

// g_W[i][o] += sum_s H[s][i] D[s][o] (i < nin, o < nout), g_b[o] += sum_s D[s][o]
__device__ __forceinline__ void accumulate_grad(TrainSmem &S, int ldh, int ldd, int nin, int nout, int offW, int offB) {
    for (int e = threadIdx.x; e < nin * nout; e += blockDim.x) {
        const int i = e / nout, o = e - i * nout;
        float acc = 0.f;
#pragma unroll 8
        for (int s = 0; s < TB; s++) acc += S.H[s * ldh + i] * S.D[s * ldd + o];
        S.g[offW + e] += acc;
    }
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
        float acc = 0.f;
        for (int s = 0; s < TB; s++) acc += S.D[s * ldd + o];
        S.g[offB + o] += acc;
    }
}

// dX = dZ . W^T : A = dZ (16 x nout, A fragments), B = W stored [in][nout_pad]
template <int KT>
__device__ __forceinline__ void back_data(const unsigned a[KT][4], const __nv_bfloat16 *W, int ld, int lane,
                                          float out[8][4]) {
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kk = 0; kk < KT; kk++) {
            unsigned b0, b1;
            load_b(W, ld, nt, kk, lane, b0, b1);
            mma_bf16(c, a[kk], b0, b1);
        }
#pragma unroll
        for (int e = 0; e < 4; e++) out[nt][e] = c[e];
    }
}

__global__ void __launch_bounds__(128) mlp_train_kernel(const float *X, const float *T, long long s0, long long s1,
                                                        long long ntot, const float *w, const __nv_bfloat16 *pk,
                                                        float *gpart, float *lpart) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
    load_params(pk, w, S.w, S.b, PK_TOTAL);
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) S.g[i] = 0.f;
    if (threadIdx.x < 4) S.loss[threadIdx.x] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gid = lane >> 2, tig = lane & 3;
    const long long tiles = (s1 - s0 + TB - 1) / TB;
    const float inv = 2.0f / (float)(ntot * MOUT);
    float lsum = 0.f;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
        const long long base = s0 + t * TB + warp * 16;
        float h1[8][4], h2[8][4], h3[8][4], y[2][4];
        warp_forward(X, s1, base, S.w, S.b, lane, h1, h2, h3, y);
        // output gradient dY = 2 (Y - T) / (n 9) on valid entries
        float d4[2][4];
#pragma unroll
        for (int nt = 0; nt < 2; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int col = nt * 8 + tig * 2 + (e & 1);
                const long long row = base + gid + ((e & 2) ? 8 : 0);
                float d = 0.f;
                if (col < MOUT && row < s1) {
                    const float r = y[nt][e] - T[row * MOUT + col];
                    lsum += r * r;
                    d = inv * r;
                }
                d4[nt][e] = d;
            }
        // layer 4
        stage_c<8>(S.H, MIN_P, h3, warp, lane);
        stage_c<2>(S.D, MH, d4, warp, lane);
        __syncthreads();
        accumulate_grad(S, MIN_P, MH, MH, MOUT, OFF_W4, OFF_B4);
        __syncthreads();
        unsigned a4[1][4];
        c_to_a<2>(d4, a4);
        float d3[8][4];
        back_data<1>(a4, S.w + PK_W4, MOUT_P, lane, d3);
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) d3[nt][e] = h3[nt][e] > 0.f ? d3[nt][e] : 0.f;
        // layer 3
        stage_c<8>(S.H, MIN_P, h2, warp, lane);
        stage_c<8>(S.D, MH, d3, warp, lane);
        __syncthreads();
        accumulate_grad(S, MIN_P, MH, MH, MH, OFF_W3, OFF_B3);
        __syncthreads();
        unsigned a3[4][4];
        c_to_a<8>(d3, a3);
        float d2[8][4];
        back_data<4>(a3, S.w + PK_W3, MH, lane, d2);
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) d2[nt][e] = h2[nt][e] > 0.f ? d2[nt][e] : 0.f;
        // layer 2
        stage_c<8>(S.H, MIN_P, h1, warp, lane);
        stage_c<8>(S.D, MH, d2, warp, lane);
        __syncthreads();
        accumulate_grad(S, MIN_P, MH, MH, MH, OFF_W2, OFF_B2);
        __syncthreads();
        unsigned a2[4][4];
        c_to_a<8>(d2, a2);
        float d1[8][4];
        back_data<4>(a2, S.w + PK_W2, MH, lane, d1);
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) d1[nt][e] = h1[nt][e] > 0.f ? d1[nt][e] : 0.f;
        // layer 1: stage the inputs (rounded to BF16 as the forward used them)
        for (int e = lane; e < 16 * MIN_P; e += 32) {
            const int r = e / MIN_P, col = e - r * MIN_P;
            const long long row = base + r;
            const float v = (col < MIN && row < s1) ? X[row * MIN + col] : 0.f;
            S.H[(warp * 16 + r) * MIN_P + col] = __bfloat162float(__float2bfloat16_rn(v));
        }
        stage_c<8>(S.D, MH, d1, warp, lane);
        __syncthreads();
        accumulate_grad(S, MIN_P, MH, MIN, MH, OFF_W1, OFF_B1);
        __syncthreads();
    }
    // block loss and gradient to this block's slots
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) S.loss[warp] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) lpart[blockIdx.x] = S.loss[0] + S.loss[1] + S.loss[2] + S.loss[3];
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) gpart[(size_t)blockIdx.x * NPARAM + i] = S.g[i];
}

// packed BF16 operand copies of the FP32 master weights
__device__ __forceinline__ void repack_one(const float *w, __nv_bfloat16 *pk, int p) {
    // find the layer of parameter p and write its packed copies
    int off, nin, nout, wt, wb, ldt, ldb;
    if (p < OFF_B1) { off = OFF_W1; nin = MIN; nout = MH; wt = PK_WT1; wb = -1; ldt = MIN_P; ldb = 0; }
    else if (p >= OFF_W2 && p < OFF_B2) { off = OFF_W2; nin = MH; nout = MH; wt = PK_WT2; wb = PK_W2; ldt = MH; ldb = MH; }
    else if (p >= OFF_W3 && p < OFF_B3) { off = OFF_W3; nin = MH; nout = MH; wt = PK_WT3; wb = PK_W3; ldt = MH; ldb = MH; }
    else if (p >= OFF_W4 && p < OFF_B4) { off = OFF_W4; nin = MH; nout = MOUT; wt = PK_WT4; wb = PK_W4; ldt = MH; ldb = MOUT_P; }
    else return;  // biases stay FP32
    const int e = p - off, i = e / nout, o = e - i * nout;
    (void)nin;
    const __nv_bfloat16 v = __float2bfloat16_rn(w[p]);
    pk[wt + o * ldt + i] = v;
    if (wb >= 0) pk[wb + i * ldb + o] = v;
}

__global__ void mlp_pack_kernel(const float *w, __nv_bfloat16 *pk) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < PK_TOTAL) pk[p] = __float2bfloat16_rn(0.f);
}
__global__ void mlp_pack2_kernel(const float *w, __nv_bfloat16 *pk) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NPARAM) repack_one(w, pk, p);
}

// sum the per-block gradients in block order; Adam on the FP32 master
__global__ void mlp_adam_kernel(float *w, float *m, float *v, const float *gpart, int nblk, int step, float lr,
                                float b1, float b2, float eps, __nv_bfloat16 *pk, float *gout) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    float g = 0.f;
    for (int b = 0; b < nblk; b++) g += gpart[(size_t)b * NPARAM + p];
    if (gout) {
        gout[p] = g;
        return;
    }
    const float mm = b1 * m[p] + (1.f - b1) * g;
    const float vv = b2 * v[p] + (1.f - b2) * g * g;
    m[p] = mm;
    v[p] = vv;
    const float mh = mm / (1.f - powf(b1, (float)step)), vh = vv / (1.f - powf(b2, (float)step));
    w[p] -= lr * mh / (sqrtf(vh) + eps);
    repack_one(w, pk, p);
}

constexpr int TRAIN_BLOCKS = 64;

size_t mlp_train_smem() { return sizeof(TrainSmem); }

}  // namespace lbmgb

using namespace lbmgb;

namespace {
// workspace: packed operands | Adam m | Adam v | block gradients | block losses
struct MlpWs {
    __nv_bfloat16 *pk;
    float *m, *v, *gpart, *lpart;
    int *err;  // set by the tensor-core forward when a wait runs out
};
size_t mlp_ws_bytes() {
    return (((size_t)PK_TOTAL * 2 + 255) / 256) * 256 + 2 * (((size_t)NPARAM * 4 + 255) / 256) * 256 +
           (((size_t)TRAIN_BLOCKS * NPARAM * 4 + 255) / 256) * 256 + 256 * 4 + 256;
}
MlpWs mlp_ws(void *ws) {
    char *b = (char *)ws;
    MlpWs W;
    size_t o = 0;
    W.pk = (__nv_bfloat16 *)(b + o);
    o += (((size_t)PK_TOTAL * 2 + 255) / 256) * 256;
    W.m = (float *)(b + o);
    o += (((size_t)NPARAM * 4 + 255) / 256) * 256;
    W.v = (float *)(b + o);
    o += (((size_t)NPARAM * 4 + 255) / 256) * 256;
    W.gpart = (float *)(b + o);
    o += (((size_t)TRAIN_BLOCKS * NPARAM * 4 + 255) / 256) * 256;
    W.lpart = (float *)(b + o);
    o += 256 * 4;
    W.err = (int *)(b + o);
    return W;
}
cudaError_t mlp_pack(const float *w, __nv_bfloat16 *pk, cudaStream_t s) {
    mlp_pack_kernel<<<(PK_TOTAL + 255) / 256, 256, 0, s>>>(w, pk);
    mlp_pack2_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(w, pk);
    return cudaGetLastError();
}
cudaError_t set_train_smem() {
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(TrainSmem));
    if (e == cudaSuccess) done = true;
    return e;
}
}  // namespace

namespace lbmgb {
// BF16 operand copies of the FP32 parameters (the layout described at the top)
cudaError_t mlp_pack_device(const float *w, void *pk, cudaStream_t s) { return mlp_pack(w, (__nv_bfloat16 *)pk, s); }
size_t mlp_pack_bytes() { return (size_t)PK_TOTAL * 2; }
}  // namespace lbmgb

extern "C" {

size_t lbm_mlp_workspace_bytes(void) { return mlp_ws_bytes(); }
int lbm_mlp_num_params(void) { return NPARAM; }

lbm_status lbm_mlp_forward(const float *X_dev, long long n, const float *w_dev, float *Y_dev, void *ws, size_t bytes,
                           void *stream) {
    if (!X_dev || !w_dev || !Y_dev || !ws || n < 0) return LBM_EINVAL;
    if (bytes < mlp_ws_bytes()) return LBM_ENOMEM;
    MlpWs W = mlp_ws(ws);
    cudaStream_t s = (cudaStream_t)stream;
    // tensor-core inference (closure_tc.cu); synchronous: the completion word is checked
    if (cudaMemsetAsync(W.err, 0, sizeof(int), s) != cudaSuccess || mlp_pack(w_dev, W.pk, s) != cudaSuccess ||
        mlp_forward_tc(X_dev, n, w_dev, W.pk, Y_dev, W.err, s) != cudaSuccess)
        return LBM_ECUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, W.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LBM_ECUDA;
    return err ? LBM_ETIMEOUT : LBM_OK;
}

lbm_status lbm_mlp_loss_grad(const float *X_dev, const float *T_dev, long long n, const float *w_dev, float *grad_dev,
                             double *loss, void *ws, size_t bytes, void *stream) {
    if (!X_dev || !T_dev || !w_dev || !grad_dev || !ws || n <= 0) return LBM_EINVAL;
    if (bytes < mlp_ws_bytes()) return LBM_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    MlpWs W = mlp_ws(ws);
    if (set_train_smem() != cudaSuccess || mlp_pack(w_dev, W.pk, s) != cudaSuccess) return LBM_ECUDA;
    long long tiles = (n + TB - 1) / TB;
    const int nblk = (int)(tiles < TRAIN_BLOCKS ? tiles : TRAIN_BLOCKS);
    mlp_train_kernel<<<nblk, 128, sizeof(TrainSmem), s>>>(X_dev, T_dev, 0, n, n, w_dev, W.pk, W.gpart, W.lpart);
    mlp_adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(nullptr, nullptr, nullptr, W.gpart, nblk, 1, 0.f, 0.f, 0.f,
                                                         0.f, W.pk, grad_dev);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    if (loss) {
        float lp[TRAIN_BLOCKS];
        if (cudaMemcpyAsync(lp, W.lpart, sizeof(float) * nblk, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return LBM_ECUDA;
        double L = 0;
        for (int b = 0; b < nblk; b++) L += lp[b];
        *loss = L / ((double)n * MOUT);
    }
    return LBM_OK;
}

lbm_status lbm_mlp_train(const float *X_dev, const float *T_dev, long long n, int epochs, int batch, double lr,
                         float *w_dev, void *ws, size_t bytes, void *stream, double *last_epoch_loss) {
    if (!X_dev || !T_dev || !w_dev || !ws || n <= 0 || epochs < 0 || batch <= 0 || !(lr > 0)) return LBM_EINVAL;
    if (bytes < mlp_ws_bytes()) return LBM_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    MlpWs W = mlp_ws(ws);
    if (set_train_smem() != cudaSuccess) return LBM_ECUDA;
    if (cudaMemsetAsync(W.m, 0, sizeof(float) * NPARAM, s) != cudaSuccess ||
        cudaMemsetAsync(W.v, 0, sizeof(float) * NPARAM, s) != cudaSuccess || mlp_pack(w_dev, W.pk, s) != cudaSuccess)
        return LBM_ECUDA;
    int step = 0;
    double epoch_loss = 0.0;
    std::vector<float> lp(TRAIN_BLOCKS);
    for (int ep = 0; ep < epochs; ep++) {
        const bool last = ep == epochs - 1;
        epoch_loss = 0.0;
        for (long long s0 = 0; s0 < n; s0 += batch) {
            const long long s1 = s0 + batch < n ? s0 + batch : n;
            const long long tiles = (s1 - s0 + TB - 1) / TB;
            const int nblk = (int)(tiles < TRAIN_BLOCKS ? tiles : TRAIN_BLOCKS);
            mlp_train_kernel<<<nblk, 128, sizeof(TrainSmem), s>>>(X_dev, T_dev, s0, s1, s1 - s0, w_dev, W.pk,
                                                                   W.gpart, W.lpart);
            step++;
            mlp_adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(w_dev, W.m, W.v, W.gpart, nblk, step, (float)lr,
                                                                 0.9f, 0.999f, 1e-8f, W.pk, nullptr);
            if (last) {
                if (cudaMemcpyAsync(lp.data(), W.lpart, sizeof(float) * nblk, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess)
                    return LBM_ECUDA;
                for (int b = 0; b < nblk; b++) epoch_loss += lp[b];
            }
        }
    }
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    if (last_epoch_loss) *last_epoch_loss = epochs > 0 ? epoch_loss / ((double)n * MOUT) : 0.0;
    return LBM_OK;
}

}  // extern "C"
