// Kinetic energy and dissipation of a device velocity field without any
// allocation: the per-block partial sums live in a file-scope device array.
//
// This is a variant of the statistics reduction behind lbm_stats for
// callers that cannot allocate device memory: solvers whose device memory
// is entirely owned by another framework's pool (a cudaMalloc beside it
// would break that pool's accounting or fail under its limit), and loops
// that must not pay the implicit device synchronisation of
// cudaMalloc/cudaFree. The caller passes the field and a device output.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr long long NA_CELLS_PER_BLOCK = 4096;         // cells reduced by one block
constexpr int NA_MAX_BLOCKS = 32768;                    // capacity of the scratch array
constexpr long long NA_MAX_CELLS = NA_CELLS_PER_BLOCK * NA_MAX_BLOCKS;  // 134,217,728 = 512^3

// Two partial sums (kinetic energy, dissipation) per block: 512 KiB that
// every GPU which loads the library keeps until the process exits.
static __device__ __align__(256) double g_na_partials[2 * NA_MAX_BLOCKS];

std::mutex g_na_mutex;
void *g_na_ptr[128];     // device address of g_na_partials, per device
bool g_na_ready[128];

__device__ __forceinline__ int na_wrap(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// 1/2 |u|^2 and 2 nu s_ij s_ij with second-order central differences on the
// periodic grid, summed per block in a fixed tree order.
__global__ void __launch_bounds__(NA_THREADS) na_partial_kernel(const double *__restrict__ u, int nx, int ny, int nz,
                                                                  long long N, double nu, double *partials) {
    __shared__ double sk[NA_THREADS], se[NA_THREADS];
    const long long c0 = (long long)blockIdx.x * NA_CELLS_PER_BLOCK;
    long long c1 = c0 + NA_CELLS_PER_BLOCK;
    if (c1 > N) c1 = N;
    double k = 0.0, e = 0.0;
    for (long long c = c0 + threadIdx.x; c < c1; c += NA_THREADS) {
        const int x = (int)(c % nx), y = (int)((c / nx) % ny), z = (int)(c / ((long long)nx * ny));
        const long long xp = na_wrap(x + 1, nx) + (long long)nx * (y + (long long)ny * z);
        const long long xm = na_wrap(x - 1, nx) + (long long)nx * (y + (long long)ny * z);
        const long long yp = x + (long long)nx * (na_wrap(y + 1, ny) + (long long)ny * z);
        const long long ym = x + (long long)nx * (na_wrap(y - 1, ny) + (long long)ny * z);
        const long long zp = x + (long long)nx * (y + (long long)ny * na_wrap(z + 1, nz));
        const long long zm = x + (long long)nx * (y + (long long)ny * na_wrap(z - 1, nz));
        double g[3][3];
        for (int a = 0; a < 3; a++) {
            const double *ua = u + a * N;
            g[a][0] = 0.5 * (ua[xp] - ua[xm]);
            g[a][1] = 0.5 * (ua[yp] - ua[ym]);
            g[a][2] = 0.5 * (ua[zp] - ua[zm]);
        }
        double ss = 0.0;
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                const double s = 0.5 * (g[a][b] + g[b][a]);
                ss += s * s;
            }
        e += 2.0 * nu * ss;
        k += 0.5 * (u[c] * u[c] + u[N + c] * u[N + c] + u[2 * N + c] * u[2 * N + c]);
    }
    sk[threadIdx.x] = k;
    se[threadIdx.x] = e;
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sk[threadIdx.x] += sk[threadIdx.x + s];
            se[threadIdx.x] += se[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = sk[0];
        partials[2 * blockIdx.x + 1] = se[0];
    }
}

// One block: sum the partials of the first `nblk` blocks (each written by
// the kernel above in this call) and store the box averages.
__global__ void __launch_bounds__(NA_THREADS) na_final_kernel(const double *partials, int nblk, long long N,
                                                                double *out) {
    __shared__ double sk[NA_THREADS], se[NA_THREADS];
    double k = 0.0, e = 0.0;
    for (int b = threadIdx.x; b < nblk; b += NA_THREADS) {
        k += partials[2 * b];
        e += partials[2 * b + 1];
    }
    sk[threadIdx.x] = k;
    se[threadIdx.x] = e;
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sk[threadIdx.x] += sk[threadIdx.x + s];
            se[threadIdx.x] += se[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sk[0] / (double)N;
        out[1] = se[0] / (double)N;
    }
}

// Device address of the scratch array for the current device. Looked up
// once per device (with that device current) and cached.
cudaError_t na_scratch(void **ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ready[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_na_partials);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev] = p;
        g_na_ready[dev] = true;
    }
    *ptr = g_na_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" lbm_status lbm_field_energy_noalloc(const double *u_dev, int nx, int ny, int nz, double nu,
                                                double *out_dev, void *cuda_stream) {
    if (!u_dev || !out_dev || nx < 1 || ny < 1 || nz < 1 || !(nu >= 0.0)) return LBM_EINVAL;
    const long long N = (long long)nx * ny * nz;
    if (N > NA_MAX_CELLS) return LBM_ENOMEM;
    void *scratch = nullptr;
    if (na_scratch(&scratch) != cudaSuccess) return LBM_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int nblk = (int)((N + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
    // each launch reports its own status (cudaLaunchKernel), so an error left
    // pending on this thread by unrelated earlier work is neither reported
    // here nor cleared
    double *partials = (double *)scratch;
    void *a1[] = {(void *)&u_dev, (void *)&nx, (void *)&ny, (void *)&nz, (void *)&N, (void *)&nu, (void *)&partials};
    if (cudaLaunchKernel((const void *)na_partial_kernel, dim3((unsigned)nblk), dim3(NA_THREADS), a1, 0, s) !=
        cudaSuccess)
        return LBM_ECUDA;
    void *a2[] = {(void *)&partials, (void *)&nblk, (void *)&N, (void *)&out_dev};
    if (cudaLaunchKernel((const void *)na_final_kernel, dim3(1), dim3(NA_THREADS), a2, 0, s) != cudaSuccess)
        return LBM_ECUDA;
    return LBM_OK;
}

extern "C" long long lbm_field_energy_noalloc_max_cells(void) { return NA_MAX_CELLS; }
