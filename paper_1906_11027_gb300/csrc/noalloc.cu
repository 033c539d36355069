// noalloc.cu -- lbm_moments_noalloc: the mass/momentum reduction of a population
// buffer with its block partials in a file-scope device array instead of
// memory from an allocator.
//
// Who needs it: callers that cannot allocate device memory when they want the
// totals, e.g. an application whose device memory is all reserved at start-up
// by another framework's pool, or a service that must not call cudaMalloc on
// its latency-critical path.  They pass the populations (for example the
// buffer lbm_device_state returns) and a host array for the result; this file
// supplies the scratch.
//
// The scratch, g_moments_scratch, is a static __device__ array of
// kNoAllocBlocks * 4 + 8 doubles (about 512 KiB) that every GPU loading the
// library keeps until the process exits.  It holds one partial per block of
// 1024 cells, so a call handles at most kNoAllocMaxCells = 16,777,216 cells and
// rejects larger domains.  In host code the array's name is only a host-side
// stand-in, so its device address is looked up with cudaGetSymbolAddress once
// per device, with that device current, on the first call there; make that
// first call before any stream capture.  All calls share the array, which keeps
// the last call's contents: every slot a call reads is written earlier in the
// same call, and calls whose kernels overlap on the GPU race on it.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/lbm.h"
#include "internal.h"
#include "kernels.cuh"

namespace lbm {

constexpr int kNoAllocBlocks = 16384;
constexpr int kNoAllocCellsPerBlock = 1024;  // 256 threads x 4 cells
constexpr long long kNoAllocMaxCells = static_cast<long long>(kNoAllocBlocks) * kNoAllocCellsPerBlock;
constexpr int kNoAllocWidth = 4;             // mass, momentum x, y, z
constexpr int kNoAllocResult = kNoAllocBlocks * kNoAllocWidth;  // offset of the final sums

static __device__ __align__(256) double g_moments_scratch[kNoAllocBlocks * kNoAllocWidth + 8];

// One partial per block: sums over its 1024 cells of rho and sum_b f_b c_b,
// reduced in a fixed order (warp shuffles, then warps in index order).  The
// buffer is summed as stored, A_b[i] for every direction b and cell i, with
// coalesced loads: the totals over the whole periodic box are the same as over
// the pulled populations f_b(x) = A_b(x - c_b), a permutation of the cells.
template <int LAT, class Real>
__global__ void __launch_bounds__(256) k_moments_partials(const Real* __restrict__ A, DevParams p,
                                                          double* __restrict__ scratch)
{
    using L = Lattice<LAT>;
    double v[kNoAllocWidth] = {0.0, 0.0, 0.0, 0.0};
    for (int k = 0; k < kNoAllocCellsPerBlock / 256; ++k) {
        const long long i = static_cast<long long>(blockIdx.x) * kNoAllocCellsPerBlock + k * 256 + threadIdx.x;
        if (i >= p.N) break;
        double s = 0.0, j[3] = {0.0, 0.0, 0.0};
        sfor<L::Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
            const double fb = static_cast<double>(A[static_cast<long long>(b) * p.N + i]);
            s += fb;
            j[0] += fb * cx;
            j[1] += fb * cy;
            j[2] += fb * cz;
        });
        v[0] += std::is_same<Real, float>::value ? p.rho_bar + s : s;
        v[1] += j[0];
        v[2] += j[1];
        v[3] += j[2];
    }
    __shared__ double sh[8][kNoAllocWidth];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < kNoAllocWidth; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < kNoAllocWidth; ++c) sh[warp][c] = v[c];
    __syncthreads();
    if (threadIdx.x < kNoAllocWidth) {
        double acc = 0.0;
        for (int w = 0; w < 8; ++w) acc += sh[w][threadIdx.x];
        scratch[static_cast<long long>(blockIdx.x) * kNoAllocWidth + threadIdx.x] = acc;
    }
}

// Sums the partials of nblocks blocks in a fixed order into scratch[kNoAllocResult..].
__global__ void __launch_bounds__(256) k_moments_final(double* __restrict__ scratch, int nblocks)
{
    __shared__ double sh[256];
    for (int c = 0; c < kNoAllocWidth; ++c) {
        double acc = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += 256) acc += scratch[static_cast<long long>(b) * kNoAllocWidth + c];
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int s = 128; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) scratch[kNoAllocResult + c] = sh[0];
        __syncthreads();
    }
}

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of g_moments_scratch on the current device, looked up once per
// device (with that device current) and cached.
cudaError_t scratch_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_moments_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

template <int LAT, class Real>
cudaError_t launch_moments(const void* f, const DevParams& p, double* scratch, int nblocks, cudaStream_t s)
{
    k_moments_partials<LAT, Real><<<nblocks, 256, 0, s>>>(static_cast<const Real*>(f), p, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_moments_final<<<1, 256, 0, s>>>(scratch, nblocks);
    return cudaGetLastError();
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_moments_noalloc(const void* f_dev, int lattice, int precision, int nx, int ny, int nz,
                                   double rho_bar, void* stream, double* out_host)
{
    using namespace lbm;
    if (!f_dev || !out_host) return set_last_error(LBM_EINVAL, "lbm_moments_noalloc: NULL buffer");
    const bool three_d = lattice == LBM_D3Q19;
    if (lattice < LBM_D2Q9 || lattice > LBM_D2Q25)
        return set_last_error(LBM_EINVAL, "lbm_moments_noalloc: unknown lattice");
    if (precision != LBM_FP64 && precision != LBM_FP32_SHIFTED)
        return set_last_error(LBM_EINVAL, "lbm_moments_noalloc: unknown precision");
    if (nx < 8 || ny < 8 || (three_d ? nz < 8 : nz != 1))
        return set_last_error(LBM_EINVAL, "lbm_moments_noalloc: every dimension must be >= 8 (nz = 1 in 2-D)");
    const long long n = static_cast<long long>(nx) * ny * nz;
    if (n > kNoAllocMaxCells) {
        char msg[160];
        std::snprintf(msg, sizeof(msg),
                      "lbm_moments_noalloc: %lld cells exceed the static scratch limit of %lld cells", n,
                      kNoAllocMaxCells);
        return set_last_error(LBM_EINVAL, msg);
    }
    double* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return set_last_error(LBM_ECUDA, cudaGetErrorString(e));
    DevParams p{};
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.N = n;
    p.rho_bar = precision == LBM_FP32_SHIFTED ? rho_bar : 0.0;
    const int nblocks = static_cast<int>((n + kNoAllocCellsPerBlock - 1) / kNoAllocCellsPerBlock);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const bool fp32 = precision == LBM_FP32_SHIFTED;
    switch (lattice) {
    case LBM_D2Q9:
        e = fp32 ? launch_moments<kLatD2Q9, float>(f_dev, p, scratch, nblocks, s)
                 : launch_moments<kLatD2Q9, double>(f_dev, p, scratch, nblocks, s);
        break;
    case LBM_D3Q19:
        e = fp32 ? launch_moments<kLatD3Q19, float>(f_dev, p, scratch, nblocks, s)
                 : launch_moments<kLatD3Q19, double>(f_dev, p, scratch, nblocks, s);
        break;
    case LBM_D2Q13:
        e = fp32 ? launch_moments<kLatD2Q13, float>(f_dev, p, scratch, nblocks, s)
                 : launch_moments<kLatD2Q13, double>(f_dev, p, scratch, nblocks, s);
        break;
    default:
        e = fp32 ? launch_moments<kLatD2Q25, float>(f_dev, p, scratch, nblocks, s)
                 : launch_moments<kLatD2Q25, double>(f_dev, p, scratch, nblocks, s);
        break;
    }
    if (e != cudaSuccess) return set_last_error(LBM_ECUDA, cudaGetErrorString(e));
    e = cudaMemcpyAsync(out_host, scratch + kNoAllocResult, sizeof(double) * kNoAllocWidth,
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_last_error(LBM_ECUDA, cudaGetErrorString(e));
    return LBM_OK;
}
