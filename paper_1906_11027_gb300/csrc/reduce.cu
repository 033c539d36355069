// reduce.cu -- deterministic double-precision reductions shared by all lattices.
// Every sum is formed in a fixed order (per-thread strided partials, then a
// fixed shared-memory tree), so results are bit-identical run to run.
#include <cuda_runtime.h>

#include "internal.h"

namespace lbm {

// One block: res[i] = sum over blocks of partials[b*width + i] for i < width-1,
// and the max for i = width-1.
__global__ void __launch_bounds__(256) k_sum_partials(const double* __restrict__ partials, int nblocks, int width,
                                                      double* __restrict__ res)
{
    __shared__ double sh[256];
    for (int i = 0; i < width; ++i) {
        const bool is_max = (i == width - 1) && (width == kObsWidth);
        double acc = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const double v = partials[static_cast<long long>(b) * width + i];
            acc = is_max ? fmax(acc, v) : acc + v;
        }
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] = is_max ? fmax(sh[threadIdx.x], sh[threadIdx.x + s])
                                                          : sh[threadIdx.x] + sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) res[i] = sh[0];
        __syncthreads();
    }
}

cudaError_t launch_sum_partials(const double* partials, int nblocks, int width, double* res, cudaStream_t s)
{
    k_sum_partials<<<1, 256, 0, s>>>(partials, nblocks, width, res);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_block_sums(const double* __restrict__ x, long long n,
                                                    double* __restrict__ partials)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        acc += x[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void k_divide(double* res, double n) { res[0] = res[0] / n; }

// res[0] = (sum of x) / n, deterministic.
cudaError_t launch_mean(const double* x, long long n, double* partials, int nblocks_max, double* res,
                        cudaStream_t s)
{
    long long nb = (n + 255) / 256;
    if (nb > nblocks_max) nb = nblocks_max;
    if (nb < 1) nb = 1;
    k_block_sums<<<static_cast<int>(nb), 256, 0, s>>>(x, n, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_sum_partials(partials, static_cast<int>(nb), 1, res, s);
    if (e != cudaSuccess) return e;
    k_divide<<<1, 1, 0, s>>>(res, static_cast<double>(n));
    return cudaGetLastError();
}

__device__ __forceinline__ double centre_offset(int i, int n)
{
    double d = static_cast<double>(i) - static_cast<double>(n / 2);
    if (d > 0.5 * n) d -= n;
    if (d < -0.5 * n) d += n;
    return d;
}

__global__ void k_field_from_table(DevParams p, int dim, const float* __restrict__ table, int T, double dmax,
                                   double R, double* __restrict__ rho0)
{
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < p.N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % p.nx);
        const long long r = i / p.nx;
        const int y = static_cast<int>(r % p.ny);
        const int z = static_cast<int>(r / p.ny);
        const double dx = centre_offset(x, p.nx), dy = centre_offset(y, p.ny);
        const double dz = dim == 3 ? centre_offset(z, p.nz) : 0.0;
        double d = sqrt(dx * dx + dy * dy + dz * dz) - R;
        d = fmin(fmax(d, -dmax), dmax);
        const double u = (d + dmax) / (2.0 * dmax) * (T - 1);
        int k = static_cast<int>(floor(u));
        if (k > T - 2) k = T - 2;
        const double a = u - k;
        rho0[i] = (1.0 - a) * static_cast<double>(table[k]) + a * static_cast<double>(table[k + 1]);
    }
}

__global__ void k_add_constant(double* __restrict__ x, long long n, double c)
{
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x)
        x[i] += c;
}

cudaError_t launch_field_from_table(const DevParams& p, int dim, const float* table, int T, double dmax, double R,
                                    double* rho0, cudaStream_t s)
{
    const long long nb = (p.N + 255) / 256;
    k_field_from_table<<<static_cast<int>(nb < 2432 ? nb : 2432), 256, 0, s>>>(p, dim, table, T, dmax, R, rho0);
    return cudaGetLastError();
}

cudaError_t launch_add_constant(double* x, long long n, double c, cudaStream_t s)
{
    const long long nb = (n + 255) / 256;
    k_add_constant<<<static_cast<int>(nb < 2432 ? nb : 2432), 256, 0, s>>>(x, n, c);
    return cudaGetLastError();
}

}  // namespace lbm
