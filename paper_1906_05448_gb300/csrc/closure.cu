// Learned near-surface gradient closure: an 85-64-64-64-9 ReLU perceptron.
// Inference and training run on tcgen05 (closure_tc.cu): BF16 operands,
// FP32 accumulation in tensor memory; this file holds the parameter
// layout, the operand packing, Adam and the C ABI.
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
// Training (closure_tc.cu): each CTA runs forward and backward on tcgen05
// over tiles of 128 samples, accumulates its weight gradient in tensor
// memory and writes it to its own slot; a second kernel here sums the slots
// in a fixed order and applies Adam to the FP32 master weights
// (deterministic).
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

// packed BF16 operand copies of the FP32 master weights
__device__ __forceinline__ void repack_one(const float *w, __nv_bfloat16 *pk, int p) {
    // find the layer of parameter p and write its packed copies
    int off, nout, wt, wb, ldt, ldb;
    if (p < OFF_B1) { off = OFF_W1; nout = MH; wt = PK_WT1; wb = -1; ldt = MIN_P; ldb = 0; }
    else if (p >= OFF_W2 && p < OFF_B2) { off = OFF_W2; nout = MH; wt = PK_WT2; wb = PK_W2; ldt = MH; ldb = MH; }
    else if (p >= OFF_W3 && p < OFF_B3) { off = OFF_W3; nout = MH; wt = PK_WT3; wb = PK_W3; ldt = MH; ldb = MH; }
    else if (p >= OFF_W4 && p < OFF_B4) { off = OFF_W4; nout = MOUT; wt = PK_WT4; wb = PK_W4; ldt = MH; ldb = MOUT_P; }
    else return;  // biases stay FP32
    const int e = p - off, i = e / nout, o = e - i * nout;
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

constexpr int TRAIN_BLOCKS = 64;  // gradient slots: CTAs of one training launch at most

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
    int nblk = 0;
    if (cudaMemsetAsync(W.err, 0, sizeof(int), s) != cudaSuccess || mlp_pack(w_dev, W.pk, s) != cudaSuccess ||
        mlp_train_tc(X_dev, T_dev, 0, n, w_dev, W.pk, W.gpart, W.lpart, TRAIN_BLOCKS, W.err, s, &nblk) != cudaSuccess)
        return LBM_ECUDA;
    mlp_adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(nullptr, nullptr, nullptr, W.gpart, nblk, 1, 0.f, 0.f, 0.f,
                                                         0.f, W.pk, grad_dev);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    float lp[TRAIN_BLOCKS];
    int err = 0;
    if (cudaMemcpyAsync(lp, W.lpart, sizeof(float) * nblk, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&err, W.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LBM_ECUDA;
    if (err) return LBM_ETIMEOUT;
    if (loss) {
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
    if (cudaMemsetAsync(W.err, 0, sizeof(int), s) != cudaSuccess) return LBM_ECUDA;
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
            int nblk = 0;
            if (mlp_train_tc(X_dev, T_dev, s0, s1, w_dev, W.pk, W.gpart, W.lpart, TRAIN_BLOCKS, W.err, s, &nblk) !=
                cudaSuccess)
                return LBM_ECUDA;
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
    int err = 0;
    if (cudaMemcpyAsync(&err, W.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LBM_ECUDA;
    if (err) return LBM_ETIMEOUT;  // a tensor-core wait ran out
    if (last_epoch_loss) *last_epoch_loss = epochs > 0 ? epoch_loss / ((double)n * MOUT) : 0.0;
    return LBM_OK;
}

}  // extern "C"
