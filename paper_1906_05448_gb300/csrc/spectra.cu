// Three-dimensional spectra of kinetic energy and dissipation (Sec. 3.2:
// the paper compares IBB and IBM spectra with the velocity inside the
// particles masked or not).
//
// The velocity field of the statistics (masked as in lbm_stats) is
// transformed component by component with a hand-written radix-2 FFT in
// FP32: fft_lines_kernel transforms L lines of one axis per block in shared
// memory (bit-reversed load, Cooley-Tukey stages, twiddles from sincospif),
// lines along y and z are taken L at a time in consecutive x so that every
// load and store is coalesced. spectrum_bins_kernel adds (1/2)|u_hat|^2 and
// its dissipation 2 nu kappa^2 (1/2)|u_hat|^2 into integer shells round(|k|)
// with FP64 shared-memory sums per block; the host adds the blocks in a
// fixed order.
//
// Scratch: the population buffer that the next step overwrites (at least
// 38 bytes per cell) holds the complex field (8 bytes per cell) and the
// per-block sums, so the entry point needs no memory of its own.
#include "lbm_internal.cuh"

#include <vector>

namespace lbmgb {

constexpr int SPB = 256;          // threads per block
constexpr int SP_BLOCKS = 304;    // binning blocks (2 per SM)
constexpr int FFT_SMEM = 32768;   // shared bytes per FFT block

__global__ void load_component_kernel(const double *u, float2 *d, long long N) {
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x)
        d[c] = make_float2((float)u[c], 0.0f);
}

// axis 0: lines along x (contiguous); 1: along y; 2: along z. Line index
// ell = p + n q: axis 0 starts at ell n; axis 1 at p + q n^2 (p = x, q = z);
// axis 2 at p + q n (p = x, q = y).
__global__ void __launch_bounds__(SPB) fft_lines_kernel(float2 *d, int n, int logn, int axis, int logL) {
    extern __shared__ float2 sh[];
    const int L = 1 << logL;
    const long long first = (long long)blockIdx.x * L;
    const long long n2 = (long long)n * n;
    const long long stride = axis == 0 ? 1 : (axis == 1 ? n : n2);
    auto base = [&](long long line) -> long long {
        const long long p = line & (n - 1), q = line >> logn;
        return axis == 0 ? line * n : (axis == 1 ? p + q * n2 : p + q * n);
    };
    const int total = L << logn;
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int li, j;
        if (axis == 0) {
            li = t >> logn;
            j = t & (n - 1);
        } else {
            j = t >> logL;
            li = t & (L - 1);
        }
        const int r = (int)(__brev((unsigned)j) >> (32 - logn));
        sh[(li << logn) + r] = d[base(first + li) + j * stride];
    }
    __syncthreads();
    for (int s = 1; s <= logn; s++) {
        const int half = 1 << (s - 1);
        for (int t = threadIdx.x; t < total / 2; t += blockDim.x) {
            const int li = t >> (logn - 1), k = t & (n / 2 - 1);
            const int grp = k >> (s - 1), pos = k & (half - 1);
            const int i0 = (li << logn) + grp * 2 * half + pos, i1 = i0 + half;
            float sn, cs;
            sincospif(-(float)pos / (float)half, &sn, &cs);  // exp(-2 pi i pos / (2 half))
            const float2 a = sh[i0], b = sh[i1];
            const float2 bw = make_float2(b.x * cs - b.y * sn, b.x * sn + b.y * cs);
            sh[i0] = make_float2(a.x + bw.x, a.y + bw.y);
            sh[i1] = make_float2(a.x - bw.x, a.y - bw.y);
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int li, j;
        if (axis == 0) {
            li = t >> logn;
            j = t & (n - 1);
        } else {
            j = t >> logL;
            li = t & (L - 1);
        }
        d[base(first + li) + j * stride] = sh[(li << logn) + j];
    }
}

// shell K = round(|k|) of an integer squared norm k2, decided in integers:
// K^2 - K + 1 <= k2 <= K^2 + K
__device__ __forceinline__ int shell_of(int k2) {
    int K = (int)sqrtf((float)k2);
    while (K * K + K < k2) K++;
    while (K > 0 && K * K - K + 1 > k2) K--;
    return K;
}

__global__ void __launch_bounds__(SPB) spectrum_bins_kernel(const float2 *d, int n, int logn, double scale,
                                                          double dfac, int nbins, double *part) {
    extern __shared__ double sb[];  // E[nbins], D[nbins]
    for (int i = threadIdx.x; i < 2 * nbins; i += blockDim.x) sb[i] = 0.0;
    __syncthreads();
    const long long N = (long long)n * n * n;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(c & (n - 1)), j = (int)((c >> logn) & (n - 1)), l = (int)(c >> (2 * logn));
        const int kx = i < n / 2 ? i : i - n, ky = j < n / 2 ? j : j - n, kz = l < n / 2 ? l : l - n;
        const int k2 = kx * kx + ky * ky + kz * kz;
        const int K = shell_of(k2);
        if (K >= nbins) continue;
        const float2 v = d[c];
        const double e = scale * ((double)v.x * v.x + (double)v.y * v.y);  // (1/2)|u_hat|^2
        atomicAdd(&sb[K], e);
        atomicAdd(&sb[nbins + K], dfac * k2 * e);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 2 * nbins; k += blockDim.x) part[(size_t)blockIdx.x * 2 * nbins + k] += sb[k];
}

cudaError_t run_spectrum(Ctx &c, int flags, int nbins, double *E, double *D) {
    cudaError_t e;
    const int n = c.nx;
    int logn = 0;
    while ((1 << logn) < n) logn++;
    const long long N = c.N;
    float2 *field = (float2 *)c.fB;
    const size_t off = ((size_t)N * sizeof(float2) + 255) / 256 * 256;
    double *part = (double *)((char *)c.fB + off);
    if ((e = launch_macro(c, 0)) != cudaSuccess) return e;
    const int ibm = c.armed_bc == LBM_BC_IBM_U || c.armed_bc == LBM_BC_IBM_B;
    if (!(ibm && (flags & LBM_STATS_UNMASK)))
        if ((e = launch_mask(c)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(part, 0, sizeof(double) * 2 * nbins * SP_BLOCKS, c.stream)) != cudaSuccess) return e;
    int logL = 0;
    while ((2 << logL) * n * (int)sizeof(float2) <= FFT_SMEM && (2 << logL) <= n * n) logL++;
    const int L = 1 << logL;
    const unsigned fft_blocks = (unsigned)((long long)n * n / L);
    const size_t fft_smem = (size_t)L * n * sizeof(float2);
    const double nu = (c.tau - 0.5) / 3.0;
    const double scale = 0.5 / ((double)N * (double)N);
    const double two_pi_n = 2.0 * 3.141592653589793 / n;
    const double dfac = 2.0 * nu * two_pi_n * two_pi_n;
    for (int comp = 0; comp < 3; comp++) {
        count_launch(c, G_STATS, 5);
        load_component_kernel<<<1024, SPB, 0, c.stream>>>(c.u_f + comp * N, field, N);
        for (int axis = 0; axis < 3; axis++)
            fft_lines_kernel<<<fft_blocks, SPB, fft_smem, c.stream>>>(field, n, logn, axis, logL);
        spectrum_bins_kernel<<<SP_BLOCKS, SPB, 2 * nbins * sizeof(double), c.stream>>>(field, n, logn, scale, dfac,
                                                                                    nbins, part);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::vector<double> hp((size_t)2 * nbins * SP_BLOCKS);
    if ((e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, c.stream)) !=
        cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(c.stream)) != cudaSuccess) return e;
    for (int k = 0; k < nbins; k++) {
        double se = 0.0, sd = 0.0;
        for (int b = 0; b < SP_BLOCKS; b++) {  // fixed block order
            se += hp[(size_t)b * 2 * nbins + k];
            sd += hp[(size_t)b * 2 * nbins + nbins + k];
        }
        E[k] = se;
        D[k] = sd;
    }
    return cudaSuccess;
}

size_t spectrum_scratch_bytes(long long N, int nbins) {
    return ((size_t)N * sizeof(float2) + 255) / 256 * 256 + sizeof(double) * 2 * (size_t)nbins * SP_BLOCKS;
}

}  // namespace lbmgb
