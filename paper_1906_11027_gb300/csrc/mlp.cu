// mlp.cu -- the learned warm start: a 5 -> 128 -> 128 -> 128 -> 128 -> 1 SiLU
// network trained and evaluated on the GPU by the library's own kernels (BF16
// operands on the tensor cores, FP32 accumulation, FP32 master weights, Adam),
// and lbm_init_droplet_learned, which starts a droplet from the network's
// steady-profile prediction instead of the tanh profile.
//
// Parameter vector (FP32, compact): W1 [5][128], b1, W2 [128][128], b2, W3, b3,
// W4, b4, W5 [128][1], b5; z_l = h_{l-1} W_l + b_l, h_l = silu(z_l), y = h_4 W_5 + b_5.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "internal.h"
#include "trace.h"

namespace lbm {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kIn = 5, kH = 128, kLayers = 5;
constexpr int kInPad = 16, kOutPad = 8;
constexpr int kFan[kLayers + 1] = {kIn, kH, kH, kH, kH, 1};

constexpr long long param_offset_w(int l)
{
    long long o = 0;
    for (int i = 0; i < l; ++i) o += (long long)kFan[i] * kFan[i + 1] + kFan[i + 1];
    return o;
}
constexpr long long param_offset_b(int l) { return param_offset_w(l) + (long long)kFan[l] * kFan[l + 1]; }
constexpr long long kNParam = param_offset_w(kLayers);
static_assert(kNParam == 50433, "parameter count");

// padded GEMM shapes of layer l: [K_l][N_l]
constexpr int kK[kLayers] = {kInPad, kH, kH, kH, kH};
constexpr int kN[kLayers] = {kH, kH, kH, kH, kOutPad};

// ---- BF16 tensor-core GEMM: C[M][N] (+)= op(A)[M][K] op(B)[K][N] -------------------
// op(A)[m][k] = ta ? A[k*lda + m] : A[m*lda + k];  op(B)[k][n] = tb ? B[n*ldb + k] : B[k*ldb + n].
// CTA tile 64x64, four warps of 32x32, K step 16; mma.sync m16n8k16 (row.col, bf16, f32 acc).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const bf16* __restrict__ A, int lda, int ta,
                                              const bf16* __restrict__ B, int ldb, int tb, float* __restrict__ C,
                                              int ldc, int accumulate)
{
    __shared__ __align__(16) bf16 As[64][24];  // [m][k]
    __shared__ __align__(16) bf16 Bs[64][24];  // [n][k]
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    const bf16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < K; k0 += 16) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int idx = threadIdx.x * 8 + e;
            const int r = idx >> 4, kk = idx & 15;
            const int gm = m0 + r, gk = k0 + kk, gn = n0 + r;
            As[r][kk] = (gm < M && gk < K) ? (ta ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk]) : zero;
            Bs[r][kk] = (gn < N && gk < K) ? (tb ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn]) : zero;
        }
        __syncthreads();
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
            uint32_t a[4];
            const int r0 = wm + mi * 16 + g;
            a[0] = *reinterpret_cast<const uint32_t*>(&As[r0][2 * t]);
            a[1] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][2 * t]);
            a[2] = *reinterpret_cast<const uint32_t*>(&As[r0][2 * t + 8]);
            a[3] = *reinterpret_cast<const uint32_t*>(&As[r0 + 8][2 * t + 8]);
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                uint32_t b[2];
                const int c0 = wn + ni * 8 + g;
                b[0] = *reinterpret_cast<const uint32_t*>(&Bs[c0][2 * t]);
                b[1] = *reinterpret_cast<const uint32_t*>(&Bs[c0][2 * t + 8]);
                mma_bf16(acc[mi][ni], a, b);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = m0 + wm + mi * 16 + g + ((e & 2) ? 8 : 0);
                const int c = n0 + wn + ni * 8 + 2 * t + (e & 1);
                if (r < M && c < N) {
                    float* p = C + (long long)r * ldc + c;
                    *p = accumulate ? *p + acc[mi][ni][e] : acc[mi][ni][e];
                }
            }
}

cudaError_t gemm(cudaStream_t s, int M, int N, int K, const bf16* A, int lda, int ta, const bf16* B, int ldb, int tb,
                 float* C, int ldc, int accumulate = 0)
{
    const dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<<<grid, 128, 0, s>>>(M, N, K, A, lda, ta, B, ldb, tb, C, ldc, accumulate);
    return cudaGetLastError();
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z)
{
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

// Z[r][c] += b[c]; H = bf16(silu(Z)) (or bf16(Z) for the output layer).
__global__ void k_bias_act(float* __restrict__ Z, const float* __restrict__ b, bf16* __restrict__ H, int rows,
                           int cols, int ncols_valid, int act)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * cols) return;
    const int c = (int)(i % cols);
    const float z = Z[i] + (c < ncols_valid ? b[c] : 0.f);
    Z[i] = z;
    if (H) H[i] = __float2bfloat16(act ? silu_f(z) : z);
}

// MSE: dY[r][0] = 2 (y_r - t_r) / B (padded to kInPad columns, bf16); per-block loss sums.
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ t, int rows, bf16* __restrict__ dY,
                      float* __restrict__ dY32, double* __restrict__ loss_part)
{
    __shared__ double sh[256];
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (r < rows) {
        const float e = Y[(long long)r * kOutPad] - t[r];
        l = (double)e * e;
        const float g = 2.f * e / rows;
        for (int c = 0; c < kInPad; ++c) dY[(long long)r * kInPad + c] = __float2bfloat16(c == 0 ? g : 0.f);
        dY32[r] = g;
    }
    sh[threadIdx.x] = l;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = sh[0];
}

// dZ = dH * silu'(Z): bf16 copy for the GEMMs, f32 copy for the bias gradient.
__global__ void k_silu_back(const float* __restrict__ dH, const float* __restrict__ Z, bf16* __restrict__ dZ,
                            float* __restrict__ dZ32, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = dH[i] * silu_grad_f(Z[i]);
    dZ[i] = __float2bfloat16(v);
    dZ32[i] = v;
}

// db[c] = sum_r dZ[r][c], fixed order (one thread per column).
__global__ void k_colsum(const float* __restrict__ dZ, int rows, int cols, int ld, float* __restrict__ db)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dZ[(long long)r * ld + c];
    db[c] = s;
}

// Copy a [K][N] block out of a padded [Kp][Np] f32 matrix into the compact vector.
__global__ void k_unpad(const float* __restrict__ src, int Np, int K, int N, float* __restrict__ dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K * N) return;
    dst[i] = src[(i / N) * Np + (i % N)];
}

// Adam (bias-corrected) on the FP32 master vector.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// BF16 padded weights [Kp][Np] from the compact master vector.
__global__ void k_pack_weights(const float* __restrict__ master, long long off, int K, int N, int Kp, int Np,
                               bf16* __restrict__ Wp)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Kp * Np) return;
    const int k = i / Np, n = i % Np;
    Wp[i] = __float2bfloat16((k < K && n < N) ? master[off + (long long)k * N + n] : 0.f);
}

// X (rows x 5 f32) -> padded bf16 rows x 16.
__global__ void k_pack_x(const float* __restrict__ X, int rows, bf16* __restrict__ Xp)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)rows * kInPad) return;
    const long long r = i / kInPad;
    const int c = (int)(i % kInPad);
    Xp[i] = __float2bfloat16(c < kIn ? X[r * kIn + c] : 0.f);
}

inline unsigned blocks(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Feature scaling of the warm-start network (shared by training data and inference).
// The radius enters as the curvature 10/R: the steady profile depends on R
// through the Laplace pressure sigma/R, and a droplet larger than any trained
// one then lies next to the trained range (curvature near 0) instead of far
// outside it.  The curvature is capped at that of R = 5, below the smallest
// trained droplets, so that the small radii the mass bisection tries stay in
// range.  d spans the interface and the bulk plateaus on both sides.
__host__ __device__ inline void mlp_features(double G, double tau, double order, double R, double d, float* x)
{
    const double kappa = R > 5.0 ? 10.0 / R : 2.0;
    x[0] = (float)((G + 4.9) / 0.6);
    x[1] = (float)((tau - 0.8) / 0.2);
    x[2] = (float)((order - 7.0) / 3.0);
    x[3] = (float)((kappa - 0.5) / 0.4);
    x[4] = (float)(d / kMlpDmax);
}

}  // namespace lbm

using namespace lbm;

struct lbm_mlp {
    int device;
    cudaStream_t stream;
    uint64_t seed;
    long long adam_t;
    float* master;   // [kNParam]
    float* grad;     // [kNParam]
    float* m;
    float* v;
    bf16* W[kLayers];   // padded bf16 weights [kK][kN]
    float* b[kLayers];  // views into master
    int bcap;           // work buffer capacity (rows)
    bf16* Xp;           // [bcap][16]
    float* Z[kLayers];  // [bcap][kN[l]]
    bf16* Hb[kLayers];  // activations h_l (bf16) [bcap][kN[l]]
    float* dH;          // [bcap][128]
    bf16* dZb;          // [bcap][128] (and [bcap][16] for the output)
    float* dZ32;        // [bcap][128]
    float* dW;          // [128][128] scratch
    float* tbuf;        // targets [bcap]
    double* loss_part;
};

namespace {

#define MCK(call)                                                                                        \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return set_last_error(LBM_ECUDA, cudaGetErrorString(e_));                 \
    } while (0)

void free_work(lbm_mlp* n)
{
    cudaFree(n->Xp);
    for (int l = 0; l < kLayers; ++l) {
        cudaFree(n->Z[l]);
        cudaFree(n->Hb[l]);
        n->Z[l] = nullptr;
        n->Hb[l] = nullptr;
    }
    cudaFree(n->dH);
    cudaFree(n->dZb);
    cudaFree(n->dZ32);
    cudaFree(n->tbuf);
    cudaFree(n->loss_part);
    n->Xp = nullptr;
    n->dH = nullptr;
    n->dZb = nullptr;
    n->dZ32 = nullptr;
    n->tbuf = nullptr;
    n->loss_part = nullptr;
    n->bcap = 0;
}

int ensure_work(lbm_mlp* n, int rows)
{
    if (rows <= n->bcap) return LBM_OK;
    free_work(n);
    const int cap = std::max(rows, 1024);
    bool ok = cudaMalloc(&n->Xp, sizeof(bf16) * cap * kInPad) == cudaSuccess;
    for (int l = 0; l < kLayers && ok; ++l) {
        ok = cudaMalloc(&n->Z[l], sizeof(float) * cap * kN[l]) == cudaSuccess &&
             cudaMalloc(&n->Hb[l], sizeof(bf16) * cap * kN[l]) == cudaSuccess;
    }
    ok = ok && cudaMalloc(&n->dH, sizeof(float) * cap * kH) == cudaSuccess &&
         cudaMalloc(&n->dZb, sizeof(bf16) * cap * kH) == cudaSuccess &&
         cudaMalloc(&n->dZ32, sizeof(float) * cap * kH) == cudaSuccess &&
         cudaMalloc(&n->tbuf, sizeof(float) * cap) == cudaSuccess &&
         cudaMalloc(&n->loss_part, sizeof(double) * blocks(cap)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_work(n);
        return set_last_error(LBM_ENOMEM, "MLP work buffers");
    }
    n->bcap = cap;
    return LBM_OK;
}

int pack_all(lbm_mlp* n)
{
    for (int l = 0; l < kLayers; ++l) {
        k_pack_weights<<<blocks(kK[l] * kN[l]), 256, 0, n->stream>>>(n->master, param_offset_w(l), kFan[l],
                                                                     kFan[l + 1], kK[l], kN[l], n->W[l]);
        MCK(cudaGetLastError());
    }
    return LBM_OK;
}

// Forward pass of `rows` packed inputs (n->Xp); output y in Z[4][r][0].
int forward(lbm_mlp* n, int rows)
{
    const bf16* h = n->Xp;
    int ldh = kInPad;
    for (int l = 0; l < kLayers; ++l) {
        MCK(gemm(n->stream, rows, kN[l], kK[l], h, ldh, 0, n->W[l], kN[l], 0, n->Z[l], kN[l]));
        k_bias_act<<<blocks((long long)rows * kN[l]), 256, 0, n->stream>>>(n->Z[l], n->b[l], n->Hb[l], rows, kN[l],
                                                                          kFan[l + 1], l < kLayers - 1);
        MCK(cudaGetLastError());
        h = n->Hb[l];
        ldh = kN[l];
    }
    return LBM_OK;
}

// Loss and gradient (into n->grad) of one batch already in n->Xp / n->tbuf.
int backward(lbm_mlp* n, int rows, double* loss)
{
    const unsigned nb = blocks(rows);
    k_mse<<<nb, 256, 0, n->stream>>>(n->Z[kLayers - 1], n->tbuf, rows, n->dZb, n->dZ32, n->loss_part);
    MCK(cudaGetLastError());
    // output layer: dZ5 = dY (rows x 1, padded to 16 columns in dZb)
    const bf16* dZ = n->dZb;
    int ldz = kInPad;  // padded width of dY
    int width = 1;     // valid columns of dZ
    for (int l = kLayers - 1; l >= 0; --l) {
        const bf16* hprev = (l == 0) ? n->Xp : n->Hb[l - 1];
        const int ldp = (l == 0) ? kInPad : kH;
        // dW_l = h_{l-1}^T dZ_l  ([K_l][N_l], K reduction over the rows)
        MCK(gemm(n->stream, kK[l], kN[l], rows, hprev, ldp, 1, dZ, ldz, 0, n->dW, kN[l]));
        k_unpad<<<blocks(kFan[l] * kFan[l + 1]), 256, 0, n->stream>>>(n->dW, kN[l], kFan[l], kFan[l + 1],
                                                                     n->grad + param_offset_w(l));
        MCK(cudaGetLastError());
        // db_l = column sums of dZ_l (f32 copy)
        if (l == kLayers - 1) {
            k_colsum<<<1, 32, 0, n->stream>>>(n->dZ32, rows, 1, 1, n->grad + param_offset_b(l));
        } else {
            k_colsum<<<1, kH, 0, n->stream>>>(n->dZ32, rows, kH, kH, n->grad + param_offset_b(l));
        }
        MCK(cudaGetLastError());
        if (l == 0) break;
        // dH_{l-1} = dZ_l W_l^T  ([rows][128]); K = N_l (16-padded for the output layer)
        // K = N_l: the padded output layer has 8 columns in W5 (dZ5 columns 1..15 are zero)
        MCK(gemm(n->stream, rows, kH, kN[l], dZ, ldz, 0, n->W[l], kN[l], 1, n->dH, kH));
        k_silu_back<<<blocks((long long)rows * kH), 256, 0, n->stream>>>(n->dH, n->Z[l - 1], n->dZb, n->dZ32,
                                                                         (long long)rows * kH);
        MCK(cudaGetLastError());
        dZ = n->dZb;
        ldz = kH;
        width = kH;
    }
    (void)width;
    if (loss) {
        std::vector<double> lp(nb);
        MCK(cudaMemcpyAsync(lp.data(), n->loss_part, sizeof(double) * nb, cudaMemcpyDeviceToHost, n->stream));
        MCK(cudaStreamSynchronize(n->stream));
        double s = 0.0;
        for (double v : lp) s += v;
        *loss = s / rows;
    }
    return LBM_OK;
}

// SplitMix64, a counter-based generator (deterministic initialisation).
uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

}  // namespace

extern "C" {

int lbm_mlp_num_params(void) { return (int)kNParam; }

int lbm_mlp_create(lbm_mlp** out, uint64_t seed)
{
    if (!out) return set_last_error(LBM_EINVAL, "NULL argument");
    lbm_mlp* n = new (std::nothrow) lbm_mlp();
    if (!n) return set_last_error(LBM_ENOMEM, "host allocation failed");
    cudaGetDevice(&n->device);
    n->seed = seed;
    bool ok = cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&n->master, sizeof(float) * kNParam) == cudaSuccess &&
              cudaMalloc(&n->grad, sizeof(float) * kNParam) == cudaSuccess &&
              cudaMalloc(&n->m, sizeof(float) * kNParam) == cudaSuccess &&
              cudaMalloc(&n->v, sizeof(float) * kNParam) == cudaSuccess &&
              cudaMalloc(&n->dW, sizeof(float) * kH * kH) == cudaSuccess;
    for (int l = 0; l < kLayers && ok; ++l) ok = cudaMalloc(&n->W[l], sizeof(bf16) * kK[l] * kN[l]) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        lbm_mlp_destroy(n);
        return set_last_error(LBM_ENOMEM, "MLP allocation failed");
    }
    for (int l = 0; l < kLayers; ++l) n->b[l] = n->master + param_offset_b(l);
    // He-uniform weights from SplitMix64, zero biases
    std::vector<float> p(kNParam, 0.f);
    uint64_t ctr = seed * 0x100000001B3ull;
    for (int l = 0; l < kLayers; ++l) {
        const double lim = std::sqrt(6.0 / kFan[l]);
        for (long long i = 0; i < (long long)kFan[l] * kFan[l + 1]; ++i) {
            const double u = (splitmix64(ctr++) >> 11) * (1.0 / 9007199254740992.0);
            p[param_offset_w(l) + i] = (float)((2.0 * u - 1.0) * lim);
        }
    }
    int rc = LBM_OK;
    if (cudaMemcpy(n->master, p.data(), sizeof(float) * kNParam, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(n->m, 0, sizeof(float) * kNParam) != cudaSuccess ||
        cudaMemset(n->v, 0, sizeof(float) * kNParam) != cudaSuccess)
        rc = set_last_error(LBM_ECUDA, "MLP upload failed");
    if (rc == LBM_OK) rc = pack_all(n);
    if (rc == LBM_OK && cudaStreamSynchronize(n->stream) != cudaSuccess) rc = set_last_error(LBM_ECUDA, "sync");
    if (rc != LBM_OK) {
        lbm_mlp_destroy(n);
        return rc;
    }
    *out = n;
    return LBM_OK;
}

int lbm_mlp_destroy(lbm_mlp* n)
{
    if (!n) return LBM_OK;
    cudaSetDevice(n->device);
    if (n->stream) cudaStreamSynchronize(n->stream);
    free_work(n);
    cudaFree(n->master);
    cudaFree(n->grad);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->dW);
    for (int l = 0; l < kLayers; ++l) cudaFree(n->W[l]);
    if (n->stream) cudaStreamDestroy(n->stream);
    delete n;
    return LBM_OK;
}

int lbm_mlp_get_params(const lbm_mlp* n, float* out)
{
    if (!n || !out) return set_last_error(LBM_EINVAL, "NULL argument");
    MCK(cudaSetDevice(n->device));
    MCK(cudaMemcpyAsync(out, n->master, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, n->stream));
    MCK(cudaStreamSynchronize(n->stream));
    return LBM_OK;
}

int lbm_mlp_set_params(lbm_mlp* n, const float* in)
{
    if (!n || !in) return set_last_error(LBM_EINVAL, "NULL argument");
    MCK(cudaSetDevice(n->device));
    MCK(cudaMemcpyAsync(n->master, in, sizeof(float) * kNParam, cudaMemcpyHostToDevice, n->stream));
    if (int rc = pack_all(n)) return rc;
    MCK(cudaStreamSynchronize(n->stream));
    return LBM_OK;
}

int lbm_mlp_features(const double* raw, int64_t n, float* out)
{
    if (!raw || !out || n < 0) return set_last_error(LBM_EINVAL, "bad argument");
    for (int64_t i = 0; i < n; ++i)
        mlp_features(raw[5 * i], raw[5 * i + 1], raw[5 * i + 2], raw[5 * i + 3], raw[5 * i + 4], out + 5 * i);
    return LBM_OK;
}

int lbm_mlp_predict(lbm_mlp* n, const float* X, int64_t rows, float* y)
{
    if (!n || !X || !y || rows < 0) return set_last_error(LBM_EINVAL, "bad argument");
    MCK(cudaSetDevice(n->device));
    const int chunk = 1 << 16;
    std::vector<float> out((size_t)chunk * kOutPad);
    float* Xd = nullptr;
    MCK(cudaMalloc(&Xd, sizeof(float) * (size_t)chunk * kIn));
    int rc = ensure_work(n, chunk);
    for (int64_t r0 = 0; r0 < rows && rc == LBM_OK; r0 += chunk) {
        const int m = (int)std::min<int64_t>(chunk, rows - r0);
        if (cudaMemcpyAsync(Xd, X + r0 * kIn, sizeof(float) * m * kIn, cudaMemcpyHostToDevice, n->stream)) {
            rc = set_last_error(LBM_ECUDA, "copy");
            break;
        }
        k_pack_x<<<blocks((long long)m * kInPad), 256, 0, n->stream>>>(Xd, m, n->Xp);
        if ((rc = forward(n, m)) != LBM_OK) break;
        if (cudaMemcpyAsync(out.data(), n->Z[kLayers - 1], sizeof(float) * m * kOutPad, cudaMemcpyDeviceToHost,
                            n->stream) != cudaSuccess ||
            cudaStreamSynchronize(n->stream) != cudaSuccess) {
            rc = set_last_error(LBM_ECUDA, "copy back");
            break;
        }
        for (int i = 0; i < m; ++i) y[r0 + i] = out[(size_t)i * kOutPad];
    }
    cudaFree(Xd);
    return rc;
}

// Loss and gradient of one batch (for checks against a reference).
int lbm_mlp_loss_grad(lbm_mlp* n, const float* X, const float* t, int rows, double* loss, float* grad)
{
    if (!n || !X || !t || rows < 1) return set_last_error(LBM_EINVAL, "bad argument");
    MCK(cudaSetDevice(n->device));
    if (int rc = ensure_work(n, rows)) return rc;
    float* Xd = nullptr;
    MCK(cudaMalloc(&Xd, sizeof(float) * rows * kIn));
    int rc = LBM_OK;
    if (cudaMemcpyAsync(Xd, X, sizeof(float) * rows * kIn, cudaMemcpyHostToDevice, n->stream) != cudaSuccess ||
        cudaMemcpyAsync(n->tbuf, t, sizeof(float) * rows, cudaMemcpyHostToDevice, n->stream) != cudaSuccess)
        rc = set_last_error(LBM_ECUDA, "copy");
    if (rc == LBM_OK) {
        k_pack_x<<<blocks((long long)rows * kInPad), 256, 0, n->stream>>>(Xd, rows, n->Xp);
        rc = forward(n, rows);
    }
    if (rc == LBM_OK) rc = backward(n, rows, loss);
    if (rc == LBM_OK && grad &&
        (cudaMemcpyAsync(grad, n->grad, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, n->stream) != cudaSuccess ||
         cudaStreamSynchronize(n->stream) != cudaSuccess))
        rc = set_last_error(LBM_ECUDA, "copy back");
    cudaFree(Xd);
    return rc;
}

// Adam on mini-batches of `batch` rows drawn without replacement (SplitMix64
// permutation per epoch).  *final_loss = mean loss of the last epoch.
int lbm_mlp_train(lbm_mlp* n, const float* X, const float* t, int64_t rows, int epochs, double lr, int batch,
                  double* final_loss)
{
    lbm::TraceRange trace("lbm_mlp_train");
    if (!n || !X || !t || rows < 1 || epochs < 0 || !(lr > 0.0) || batch < 16)
        return set_last_error(LBM_EINVAL, "bad argument");
    MCK(cudaSetDevice(n->device));
    if (int rc = ensure_work(n, batch)) return rc;
    float* Xb = nullptr;
    MCK(cudaMalloc(&Xb, sizeof(float) * batch * kIn));
    int rc = LBM_OK;
    std::vector<int64_t> perm(rows);
    for (int64_t i = 0; i < rows; ++i) perm[i] = i;
    std::vector<float> xb((size_t)batch * kIn), tb(batch);
    double epoch_loss = 0.0;
    uint64_t ctr = n->seed ^ 0xA5A5A5A5u;
    for (int ep = 0; ep < epochs && rc == LBM_OK; ++ep) {
        for (int64_t i = rows - 1; i > 0; --i) std::swap(perm[i], perm[splitmix64(ctr++) % (uint64_t)(i + 1)]);
        double lsum = 0.0;
        int64_t nb = 0;
        for (int64_t r0 = 0; r0 + batch <= rows && rc == LBM_OK; r0 += batch, ++nb) {
            for (int i = 0; i < batch; ++i) {
                const int64_t s = perm[r0 + i];
                std::memcpy(&xb[(size_t)i * kIn], X + s * kIn, sizeof(float) * kIn);
                tb[i] = t[s];
            }
            if (cudaMemcpyAsync(Xb, xb.data(), sizeof(float) * batch * kIn, cudaMemcpyHostToDevice, n->stream) ||
                cudaMemcpyAsync(n->tbuf, tb.data(), sizeof(float) * batch, cudaMemcpyHostToDevice, n->stream)) {
                rc = set_last_error(LBM_ECUDA, "batch copy");
                break;
            }
            k_pack_x<<<blocks((long long)batch * kInPad), 256, 0, n->stream>>>(Xb, batch, n->Xp);
            double l = 0.0;
            if ((rc = forward(n, batch)) != LBM_OK) break;
            if ((rc = backward(n, batch, &l)) != LBM_OK) break;
            ++n->adam_t;
            const float c1 = 1.f - std::pow(0.9f, (float)n->adam_t), c2 = 1.f - std::pow(0.999f, (float)n->adam_t);
            k_adam<<<blocks(kNParam), 256, 0, n->stream>>>(n->master, n->grad, n->m, n->v, kNParam, (float)lr, 0.9f,
                                                          0.999f, 1e-8f, c1, c2);
            if (cudaGetLastError() != cudaSuccess) {
                rc = set_last_error(LBM_ECUDA, "adam");
                break;
            }
            if ((rc = pack_all(n)) != LBM_OK) break;
            lsum += l;
        }
        epoch_loss = nb ? lsum / nb : 0.0;
    }
    if (rc == LBM_OK && cudaStreamSynchronize(n->stream) != cudaSuccess) rc = set_last_error(LBM_ECUDA, "sync");
    cudaFree(Xb);
    if (rc == LBM_OK && final_loss) *final_loss = epoch_loss;
    return rc;
}

int lbm_mlp_save(const lbm_mlp* n, const char* path)
{
    if (!n || !path) return set_last_error(LBM_EINVAL, "NULL argument");
    std::vector<float> p(kNParam);
    if (int rc = lbm_mlp_get_params(n, p.data())) return rc;
    FILE* f = std::fopen(path, "wb");
    if (!f) return set_last_error(LBM_EIO, "cannot open file");
    const uint32_t hdr[2] = {0x4d4c5031u, (uint32_t)kNParam};
    const bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1 && std::fwrite(p.data(), sizeof(float), kNParam, f) == (size_t)kNParam;
    if (std::fclose(f) != 0 || !ok) return set_last_error(LBM_EIO, "write failed");
    return LBM_OK;
}

int lbm_mlp_load(lbm_mlp** out, const char* path)
{
    if (!out || !path) return set_last_error(LBM_EINVAL, "NULL argument");
    FILE* f = std::fopen(path, "rb");
    if (!f) return set_last_error(LBM_EIO, "cannot open file");
    uint32_t hdr[2] = {0, 0};
    std::vector<float> p(kNParam);
    const bool ok = std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == 0x4d4c5031u && hdr[1] == (uint32_t)kNParam &&
                    std::fread(p.data(), sizeof(float), kNParam, f) == (size_t)kNParam;
    std::fclose(f);
    if (!ok) return set_last_error(LBM_EIO, "not an MLP file");
    lbm_mlp* n = nullptr;
    if (int rc = lbm_mlp_create(&n, 0)) return rc;
    if (int rc = lbm_mlp_set_params(n, p.data())) {
        lbm_mlp_destroy(n);
        return rc;
    }
    *out = n;
    return LBM_OK;
}

}  // extern "C"

// ---- evaluation of the network on a 1-D table of signed distances -------------
namespace lbm {

int mlp_profile_table(lbm_mlp* n, double G, double tau, double order, double R, int T, double dmax, float* table_dev)
{
    if (int rc = ensure_work(n, T)) return rc;
    std::vector<float> x((size_t)T * kIn);
    for (int k = 0; k < T; ++k) {
        const double d = -dmax + 2.0 * dmax * k / (T - 1);
        mlp_features(G, tau, order, R, d, &x[(size_t)k * kIn]);
    }
    float* Xd = nullptr;
    MCK(cudaMalloc(&Xd, sizeof(float) * T * kIn));
    int rc = LBM_OK;
    if (cudaMemcpyAsync(Xd, x.data(), sizeof(float) * T * kIn, cudaMemcpyHostToDevice, n->stream) != cudaSuccess)
        rc = set_last_error(LBM_ECUDA, "copy");
    if (rc == LBM_OK) {
        k_pack_x<<<blocks((long long)T * kInPad), 256, 0, n->stream>>>(Xd, T, n->Xp);
        rc = forward(n, T);
    }
    if (rc == LBM_OK)
        if (cudaMemcpy2DAsync(table_dev, sizeof(float), n->Z[kLayers - 1], sizeof(float) * kOutPad, sizeof(float), T,
                              cudaMemcpyDeviceToDevice, n->stream) != cudaSuccess)
            rc = set_last_error(LBM_ECUDA, "table copy");
    if (rc == LBM_OK && cudaStreamSynchronize(n->stream) != cudaSuccess) rc = set_last_error(LBM_ECUDA, "sync");
    cudaFree(Xd);
    return rc;
}

}  // namespace lbm
