// kernels.cuh -- device kernels of one pseudo-potential LB time step and its
// readbacks, templated on lattice, force-stencil order, collision and precision.
//
// Storage: the context keeps the post-collision, not yet streamed populations
// A_b(y) = f*_b(y, n-1) (pull scheme).  The pre-collision state of Eq. 3 is
// f_b(x, n) = A_b(x - c_b).  One step (two-pass schedule):
//   k_psi   : rho(x) = sum_b A_b(x - c_b),  psi(rho) -> ghosted psi buffer
//   k_fused : TMA-stage the psi tile + halo in shared memory; gather f(x);
//             rho, j = sum f c; F = -G psi(x) sum_a w_a psi(x + e_a) e_a (Eq. 1);
//             u = (j + F/2)/rho; Guo-forced BGK or MRT collision (Eqs. 3-4);
//             write B_b(x) = f*_b(x).
// FP32 storage keeps deviations f~ = f - w_b rho_bar (rho = rho_bar + sum f~).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <set>
#include <utility>
#include <type_traits>

#include "internal.h"
#include "lattice.cuh"

namespace lbm {

constexpr double kPrA = 2.0 / 49.0;  // Peng-Robinson a, b (R = 1), Sec. 3
constexpr double kPrB = 2.0 / 21.0;

// Sets a kernel's dynamic shared-memory limit to its request, once per (kernel,
// device): the attribute belongs to the device, and a process may drive several.
template <class K>
cudaError_t ensure_dyn_smem(K kern, size_t dyn)
{
    // The default limit (48 KB) covers static plus dynamic shared memory, so a
    // kernel whose dynamic part fits under 48 KB can still need the attribute
    // once its static arrays are added: set it for every dynamic request.
    if (dyn == 0) return cudaSuccess;
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    int dev = 0;
    if (cudaError_t e = cudaGetDevice(&dev); e != cudaSuccess) return e;
    const std::pair<const void*, int> key(reinterpret_cast<const void*>(kern), dev);
    std::lock_guard<std::mutex> lock(mu);
    if (done.count(key)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
    if (e == cudaSuccess) done.insert(key);
    return e;
}

// ---- small PTX helpers: shared-memory mbarrier and TMA ----------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait.  try_wait suspends for an interval the hardware chooses, so
// the bound is kept in time rather than in tries: the wait gives up once the
// global nanosecond timer has advanced kWaitLimitNs past its first failed try
// (no staged copy legitimately takes that long).  Returns false if it ran out.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

// Bulk global -> shared copy of `bytes` (16-byte aligned ends, multiple of 16)
// counted on an mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Orders this thread's earlier generic shared-memory accesses before its later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Asynchronous 4-byte global -> shared copies (cp.async, completion by groups).
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---- indexing -----------------------------------------------------------------
__device__ __forceinline__ long long cell_of(const DevParams& p, int x, int y, int z)
{
    return (static_cast<long long>(z) * p.ny + y) * p.nx + x;
}
template <int C>
__device__ __forceinline__ int shift_wrap(int i, int n)
{
    // i - C on a periodic axis, |C| <= 3 <= n
    int j = i - C;
    if (C > 0 && j < 0) j += n;
    if (C < 0 && j >= n) j -= n;
    return j;
}
template <int C>
__device__ __forceinline__ int shift_wrap_fwd(int i, int n)
{
    int j = i + C;
    if (C < 0 && j < 0) j += n;
    if (C > 0 && j >= n) j -= n;
    return j;
}

// Pull gather of the pre-collision populations f_b(x) = A_b(x - c_b).
template <int LAT, class Real>
__device__ __forceinline__ void gather(const Real* __restrict__ A, const DevParams& p, int x, int y, int z,
                                       Real (&f)[Lattice<LAT>::Q])
{
    using L = Lattice<LAT>;
    sfor<L::Q>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
        const int xs = shift_wrap<cx>(x, p.nx);
        const int ys = shift_wrap<cy>(y, p.ny);
        const int zs = (L::D == 3) ? shift_wrap<cz>(z, p.nz) : 0;
        f[b] = A[static_cast<long long>(b) * p.N + cell_of(p, xs, ys, zs)];
    });
}

// ---- psi -------------------------------------------------------------------------
__device__ __forceinline__ double psi_exp(double r) { return -expm1(-r); }
__device__ __forceinline__ float psi_exp(float r) { return -expm1f(-r); }

// psi = sqrt(2 (p_EOS - c_s^2 rho) / (G c_s'^2)) with the Peng-Robinson EOS (Sec. 3).
__device__ __forceinline__ double psi_pr(double rho, const DevParams& p, double cs2)
{
    const double pe = rho * p.pr_T / (1.0 - kPrB * rho)
                    - kPrA * p.pr_alpha * rho * rho / (1.0 + 2.0 * kPrB * rho - kPrB * kPrB * rho * rho);
    const double arg = 2.0 * (pe - cs2 * rho) / (p.G * cs2);
    if (!(arg >= 0.0)) atomicOr(p.err, kErrNegativeSqrt);
    return sqrt(arg);
}

template <int LAT, class Real>
__device__ __forceinline__ Real psi_of(Real rho, const DevParams& p)
{
    if (std::is_same<Real, double>::value && p.psi_kind == 1)
        return static_cast<Real>(psi_pr(static_cast<double>(rho), p, Lattice<LAT>::cs2));
    return psi_exp(rho);
}

// Writes psi of cell (x, y, z) and its periodic images into the ghosted buffer.
template <int D, class Real>
__device__ __forceinline__ void store_psi(Real* __restrict__ psi, const DevParams& p, int x, int y, int z, Real v)
{
    const int g = p.g;
    const int gz = (D == 3) ? g : 0;
    const int zlo = (D == 3) ? -1 : 0, zhi = (D == 3) ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz) {
        const int Z = z + dz * p.nz;
        if (Z < -gz || Z >= p.nz + gz) continue;
        for (int dy = -1; dy <= 1; ++dy) {
            const int Y = y + dy * p.ny;
            if (Y < -g || Y >= p.ny + g) continue;
            for (int dx = -1; dx <= 1; ++dx) {
                const int X = x + dx * p.nx;
                if (X < -kGhostX || X >= p.nx + kGhostX) continue;
                psi[(static_cast<long long>(Z + gz) * p.psy + (Y + g)) * p.psx + (X + kGhostX)] = v;
            }
        }
    }
}

// ---- force (Eq. 1) from a psi view with compile-time strides -------------------
template <int LAT, int ORD, class Real, int SX, int SY>
__device__ __forceinline__ void force_from(const Real* tc, Real G, Real (&F)[3])
{
    using L = Lattice<LAT>;
    using S = Stencil<L::D, ORD>;
    // Opposite stencil vectors are adjacent: each pair contributes
    // w e (psi(x + e) - psi(x - e)).
    Real ax = Real(0), ay = Real(0), az = Real(0);
    sfor<S::n / 2>([&](auto kI) {
        constexpr int a = 2 * decltype(kI)::value;
        constexpr int ex = S::T.v[a][0], ey = S::T.v[a][1], ez = S::T.v[a][2];
        constexpr double wt = S::T.w[a] * L::cs2;  // c_s^2-scaled force weight
        const Real d = tc[(ez * SY + ey) * SX + ex] - tc[-((ez * SY + ey) * SX + ex)];
        if (ex != 0) ax += Real(wt * ex) * d;
        if (ey != 0) ay += Real(wt * ey) * d;
        if (ez != 0) az += Real(wt * ez) * d;
    });
    const Real gp = -G * tc[0];
    F[0] = gp * ax;
    F[1] = gp * ay;
    F[2] = gp * az;
}

// ---- value helpers shared by the scalar and the packed-pair collision --------
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ double vmul(double a, double b) { return a * b; }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <class V> __device__ __forceinline__ V vsplat(double x);
template <> __device__ __forceinline__ double vsplat<double>(double x) { return x; }
template <> __device__ __forceinline__ float vsplat<float>(double x) { return static_cast<float>(x); }
template <> __device__ __forceinline__ float2 vsplat<float2>(double x)
{
    return make_float2(static_cast<float>(x), static_cast<float>(x));
}
// acc + C x for a compile-time integer C (no operation for C = 0)
template <int C, class V>
__device__ __forceinline__ V macc(V acc, V x)
{
    if constexpr (C == 0) return acc;
    else if constexpr (C == 1) return vadd(acc, x);
    else if constexpr (C == -1) return vsub(acc, x);
    else return vfma(vsplat<V>(double(C)), x, acc);
}
// A scalar parameter in the kernel's precision (FP32 kernels read the FP32 copy).
template <class Real>
__device__ __forceinline__ Real par(double d, float f)
{
    if constexpr (std::is_same<Real, float>::value) return f; else return d;
}

// ---- MRT as a correction of the BGK update -------------------------------------
// With m_eq := M feq and Guo's source in moment space, the MRT update is
//   m* = m - S (m - m_eq) + (I - S/2) m_src,
// and the BGK update is the same with S = omega I.  Their difference is
// (omega I - S)(m - m_eq + m_src/2), so
//   f*_b = f_BGK,b + sum_k M_kb t_k,  t_k = (omega - s_k)/|M_k|^2 m_k(g),  g = f - feq + src/2,
// where only the moments whose rate differs from omega contribute (the
// conserved ones have m_k(g) = 0: sum g = 0 and sum g c = j - rho u + F/2 = 0).
// m_k(f) comes from the pair sums P = f_b + f_b+1 (even rows) or differences
// D = f_b - f_b+1 (odd rows), b = 2p + 1; the equilibrium and source moments
// are closed forms in the compile-time tensors A, B, C of Mrt<LAT>::T:
//   even rows: m_k(g) = m_k(f) - A_k (rho' - u.v/(2 cs2)) - u.C_k.v/(2 cs4)
//   odd rows:  m_k(g) = m_k(f) - B_k.j/cs2
// with v = j - F/2 (= rho u - F) and rho' = rho, or rho - rho_bar for FP32
// deviations (whose m_k(f) lacks the rho_bar A_k of the stored offset).
template <int LAT, class V>
__device__ __forceinline__ void mrt_moments_g(V f0, const V (&P)[(Lattice<LAT>::Q - 1) / 2],
                                              const V (&D)[(Lattice<LAT>::Q - 1) / 2], V r0, const V (&j)[3],
                                              const V (&u)[3], const V (&v)[3], const V (&dm)[4],
                                              V (&t)[Lattice<LAT>::Q])
{
    using L = Lattice<LAT>;
    using MB = Mrt<LAT>;
    constexpr int Q = L::Q;
    constexpr int NP = (Q - 1) / 2;
    constexpr int DIM = L::D;
    constexpr double cs2 = L::cs2;
    V uv = vmul(u[0], v[0]);
    uv = vfma(u[1], v[1], uv);
    if constexpr (DIM == 3) uv = vfma(u[2], v[2], uv);
    const V e0 = vfma(uv, vsplat<V>(-0.5 / cs2), r0);
    sfor<Q>([&](auto kI) {
        constexpr int k = decltype(kI)::value;
        constexpr int rc = MB::B.rate_class[k];
        if constexpr (rc != 0) {
            constexpr int par_k = MB::T.parity[k];
            static_assert(par_k != 0, "every non-conserved MRT row is even or odd under c -> -c");
            V m = vsplat<V>(0.0);
            if constexpr (par_k > 0) {
                constexpr int m0 = static_cast<int>(MB::B.M[k][0]);
                static_assert(double(m0) == MB::B.M[k][0], "integer basis");
                m = macc<m0>(m, f0);
                sfor<NP>([&](auto pI) {
                    constexpr int pp = decltype(pI)::value;
                    constexpr int mk = static_cast<int>(MB::B.M[k][2 * pp + 1]);
                    static_assert(double(mk) == MB::B.M[k][2 * pp + 1], "integer basis");
                    m = macc<mk>(m, P[pp]);
                });
                constexpr double A = MB::T.A[k];
                if constexpr (A != 0.0) m = vfma(vsplat<V>(-A), e0, m);
                sfor<DIM>([&](auto iI) {
                    constexpr int i = decltype(iI)::value;
                    sfor<DIM>([&](auto jI) {
                        constexpr int jj = decltype(jI)::value;
                        constexpr double c = MB::T.C[k][i][jj];
                        if constexpr (c != 0.0) m = vfma(vsplat<V>(-0.5 * c / (cs2 * cs2)), vmul(u[i], v[jj]), m);
                    });
                });
            } else {
                sfor<NP>([&](auto pI) {
                    constexpr int pp = decltype(pI)::value;
                    constexpr int mk = static_cast<int>(MB::B.M[k][2 * pp + 1]);
                    static_assert(double(mk) == MB::B.M[k][2 * pp + 1], "integer basis");
                    m = macc<mk>(m, D[pp]);
                });
                sfor<DIM>([&](auto iI) {
                    constexpr int i = decltype(iI)::value;
                    constexpr double bc = MB::T.Bv[k][i];
                    if constexpr (bc != 0.0) m = vfma(vsplat<V>(-bc / cs2), j[i], m);
                });
            }
            constexpr double inv_norm = MB::B.inv_norm[k];
            t[k] = vmul(dm[rc], vmul(vsplat<V>(inv_norm), m));
        }
    });
}

// f_b += sum_k M_kb t_k over the non-conserved moments, by opposite pairs:
// f_b += E + O, f_b+1 += E - O with E from the even rows and O from the odd ones.
template <int LAT, class V>
__device__ __forceinline__ void mrt_apply(const V (&t)[Lattice<LAT>::Q], V (&f)[Lattice<LAT>::Q])
{
    using L = Lattice<LAT>;
    using MB = Mrt<LAT>;
    constexpr int Q = L::Q;
    {
        V e = vsplat<V>(0.0);
        sfor<Q>([&](auto kI) {
            constexpr int k = decltype(kI)::value;
            if constexpr (MB::B.rate_class[k] != 0 && MB::T.parity[k] > 0)
                e = macc<static_cast<int>(MB::B.M[k][0])>(e, t[k]);
        });
        f[0] = vadd(f[0], e);
    }
    sfor<(Q - 1) / 2>([&](auto pI) {
        constexpr int b = 2 * decltype(pI)::value + 1;
        V e = vsplat<V>(0.0), o = vsplat<V>(0.0);
        sfor<Q>([&](auto kI) {
            constexpr int k = decltype(kI)::value;
            if constexpr (MB::B.rate_class[k] != 0) {
                constexpr int mk = static_cast<int>(MB::B.M[k][b]);
                if constexpr (MB::T.parity[k] > 0) e = macc<mk>(e, t[k]);
                else o = macc<mk>(o, t[k]);
            }
        });
        f[b] = vadd(f[b], vadd(e, o));
        f[b + 1] = vadd(f[b + 1], vsub(e, o));
    });
}

// ---- collision (Eqs. 3-4) --------------------------------------------------------
// f holds pre-collision populations (FP32: deviations); on return the
// post-collision ones.  Returns nothing; rho, u computed inside.
template <int LAT, int COLL, class Real>
__device__ __forceinline__ void collide(Real (&f)[Lattice<LAT>::Q], const Real (&F)[3], const DevParams& p)
{
    using L = Lattice<LAT>;
    constexpr int NP = (L::Q - 1) / 2;
    constexpr bool kDev = std::is_same<Real, float>::value;  // deviation storage
    // Moments through the opposite pairs (b, b+1): sum f and sum (f_b - f_b+1) c_b.
    Real s = f[0], jx = Real(0), jy = Real(0), jz = Real(0);
    Real Pp[NP], Dp[NP];  // pair sums and differences (MRT)
    sfor<NP>([&](auto kI) {
        constexpr int b = 1 + 2 * decltype(kI)::value;
        constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
        Pp[decltype(kI)::value] = f[b] + f[b + 1];
        s += Pp[decltype(kI)::value];
        const Real d = f[b] - f[b + 1];
        Dp[decltype(kI)::value] = d;
        if (cx != 0) jx += Real(cx) * d;
        if (cy != 0) jy += Real(cy) * d;
        if (cz != 0) jz += Real(cz) * d;
    });
    const Real rho = kDev ? par<Real>(p.rho_bar, p.rho_bar_f) + s : s;
    const Real inv_rho = Real(1) / rho;
    const Real ux = (jx + Real(0.5) * F[0]) * inv_rho;
    const Real uy = (jy + Real(0.5) * F[1]) * inv_rho;
    const Real uz = (jz + Real(0.5) * F[2]) * inv_rho;
    constexpr double cs2 = L::cs2;
    const Real inv_cs2 = Real(1.0 / cs2);
    const Real inv_cs4 = Real(1.0 / (cs2 * cs2));
    const Real half_inv_cs4 = Real(0.5 / (cs2 * cs2));
    const Real usq = (ux * ux + uy * uy + uz * uz) * Real(0.5 / cs2);
    const Real uF = ux * F[0] + uy * F[1] + uz * F[2];
    const Real omega = par<Real>(p.omega, p.omega_f);
    const Real pref = par<Real>(p.pref, p.pref_f);
    if constexpr (COLL == 0 || COLL == 1) {
        // MRT: the moment-space correction is formed from the pre-collision state
        Real t[L::Q];
        if constexpr (COLL == 1) {
            const Real jv[3] = {jx, jy, jz};
            const Real uv3[3] = {ux, uy, uz};
            const Real vv[3] = {jx - Real(0.5) * F[0], jy - Real(0.5) * F[1], jz - Real(0.5) * F[2]};
            Real dm[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) dm[c] = par<Real>(p.dmrt[c], p.dmrt_f[c]);
            mrt_moments_g<LAT, Real>(f[0], Pp, Dp, kDev ? s : rho, jv, uv3, vv, dm, t);
        }
        // omega feq_b + pref src_b regrouped (Eq. 4):
        //   w_b [ A0 + (c.u)(c.V) + c.P ],
        //   A0 = omega rho (1 - u.u/(2 cs2)) - pref u.F / cs2   (FP32: omega (rho - rho_bar) in
        //        place of omega rho for the constant term),
        //   P  = (omega rho u + pref F) / cs2,   V = (omega rho u / 2 + pref F) / cs4;
        // the c.P term is odd under c -> -c, the rest even.
        const Real orho = omega * rho;
        const Real A0 = (kDev ? omega * s : orho) - orho * usq - pref * uF * inv_cs2;
        const Real Px = (orho * ux + pref * F[0]) * inv_cs2;
        const Real Py = (orho * uy + pref * F[1]) * inv_cs2;
        const Real Pz = (orho * uz + pref * F[2]) * inv_cs2;
        const Real h = Real(0.5) * orho;
        const Real Vx = (h * ux + pref * F[0]) * inv_cs4;
        const Real Vy = (h * uy + pref * F[1]) * inv_cs4;
        const Real Vz = (h * uz + pref * F[2]) * inv_cs4;
        const Real om1 = Real(1) - omega;
        {
            constexpr double w0 = L::T.w[0];
            f[0] = f[0] * om1 + Real(w0) * A0;
        }
        sfor<NP>([&](auto kI) {
            constexpr int b = 1 + 2 * decltype(kI)::value;
            constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
            static_assert(L::T.v[b + 1][0] == -cx && L::T.v[b + 1][1] == -cy && L::T.v[b + 1][2] == -cz,
                          "opposite velocities must be adjacent");
            constexpr double wb = L::T.w[b];
            const Real cu = Real(cx) * ux + Real(cy) * uy + Real(cz) * uz;
            const Real cV = Real(cx) * Vx + Real(cy) * Vy + Real(cz) * Vz;
            const Real cP = Real(cx) * Px + Real(cy) * Py + Real(cz) * Pz;
            const Real ev = cu * cV + A0;
            f[b] = f[b] * om1 + Real(wb) * (ev + cP);
            f[b + 1] = f[b + 1] * om1 + Real(wb) * (ev - cP);
        });
        if constexpr (COLL == 1) mrt_apply<LAT, Real>(t, f);
        (void)half_inv_cs4;
    } else {
        // Exact-difference forcing with BGK (the scheme of the paper's runs, Sec. 3):
        //   f* = feq(rho, v) + (1 - omega) (f - feq(rho, u')),  u' = j / rho, v = u' + F / rho,
        // regrouped as w_b [ A0 + q_b +- c.P ] with
        //   A0 = omega rho - rho (v.v - (1 - omega) u'.u') / (2 cs2)   (FP32: omega (rho - rho_bar)),
        //   P  = rho (v - (1 - omega) u') / cs2,
        //   q_b = rho ((c.v)^2 - (1 - omega) (c.u')^2) / (2 cs4)   (even under c -> -c).
        const Real upx = jx * inv_rho, upy = jy * inv_rho, upz = jz * inv_rho;
        const Real vx = (jx + F[0]) * inv_rho, vy = (jy + F[1]) * inv_rho, vz = (jz + F[2]) * inv_rho;
        const Real om1 = Real(1) - omega;
        const Real vv = vx * vx + vy * vy + vz * vz;
        const Real uu = upx * upx + upy * upy + upz * upz;
        const Real A0 = (kDev ? omega * s : omega * rho) - rho * (vv - om1 * uu) * Real(0.5 / cs2);
        const Real Px = rho * (vx - om1 * upx) * inv_cs2;
        const Real Py = rho * (vy - om1 * upy) * inv_cs2;
        const Real Pz = rho * (vz - om1 * upz) * inv_cs2;
        const Real hq = rho * half_inv_cs4;
        {
            constexpr double w0 = L::T.w[0];
            f[0] = f[0] * om1 + Real(w0) * A0;
        }
        sfor<(L::Q - 1) / 2>([&](auto kI) {
            constexpr int b = 1 + 2 * decltype(kI)::value;
            constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
            constexpr double wb = L::T.w[b];
            const Real cv = Real(cx) * vx + Real(cy) * vy + Real(cz) * vz;
            const Real cu = Real(cx) * upx + Real(cy) * upy + Real(cz) * upz;
            const Real cP = Real(cx) * Px + Real(cy) * Py + Real(cz) * Pz;
            const Real ev = A0 + hq * (cv * cv - om1 * cu * cu);
            f[b] = f[b] * om1 + Real(wb) * (ev + cP);
            f[b + 1] = f[b + 1] * om1 + Real(wb) * (ev - cP);
        });
        (void)ux; (void)uy; (void)uz; (void)usq; (void)uF; (void)pref;
    }
}

// Index of the velocity opposite to c_b (c_opp = -c_b).
template <int LAT>
__host__ __device__ constexpr int opposite(int b)
{
    using L = Lattice<LAT>;
    for (int k = 0; k < L::Q; ++k)
        if (L::T.v[k][0] == -L::T.v[b][0] && L::T.v[k][1] == -L::T.v[b][1] && L::T.v[k][2] == -L::T.v[b][2])
            return k;
    return -1;
}

// ---- kernels -------------------------------------------------------------------------

// rho and psi of every cell (pull gather), written with periodic ghosts.  A solid
// node (y < wall_rows) carries the psi of the wall's virtual density.
template <int LAT, class Real>
__global__ void __launch_bounds__(256) k_psi(const Real* __restrict__ A, Real* __restrict__ psi, DevParams p)
{
    using L = Lattice<LAT>;
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    if (y < p.wall_rows) {
        store_psi<L::D>(psi, p, x, y, z, static_cast<Real>(p.psi_w));
        return;
    }
    Real f[L::Q];
    gather<LAT>(A, p, x, y, z, f);
    Real s = Real(0);
    sfor<L::Q>([&](auto bI) { s += f[decltype(bI)::value]; });
    const Real rho = std::is_same<Real, float>::value ? Real(p.rho_bar) + s : s;
    store_psi<L::D>(psi, p, x, y, z, psi_of<LAT>(rho, p));
}

// Fused pull-stream / force / collide, psi tile staged by TMA.  (With a wall,
// k_bounce then rewrites the rows of the solid band.)
template <int LAT, int ORD, int COLL, class Real, int TY, int TZ>
__global__ void __launch_bounds__(32 * TY * TZ)
    k_fused(const __grid_constant__ CUtensorMap tmap, const Real* __restrict__ A, Real* __restrict__ B, DevParams p)
{
    using L = Lattice<LAT>;
    using S = Stencil<L::D, ORD>;
    constexpr int D = L::D;
    constexpr int R = S::radius;
    constexpr int SX = 32 + 2 * kGhostX;
    constexpr int SY = TY + 2 * R;
    constexpr int SZ = (D == 3) ? TZ + 2 * R : 1;
    __shared__ alignas(128) Real tile[SZ * SY * SX];
    __shared__ alignas(8) unsigned long long bar;

    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int tid = (tz * TY + ty) * 32 + tx;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * TY, z0 = (D == 3) ? blockIdx.z * TZ : 0;
    const uint32_t bar_a = smem_u32(&bar);
    const uint32_t tile_a = smem_u32(tile);
    if (tid == 0) {
        mbar_init(bar_a, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(bar_a, static_cast<uint32_t>(sizeof(tile)));
        // box origin in buffer coordinates = domain (x0 - kGhostX, y0 - R, z0 - R)
        if (D == 3)
            tma_load_3d(tile_a, &tmap, x0, y0, z0, bar_a);
        else
            tma_load_2d(tile_a, &tmap, x0, y0, bar_a);
    }
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    const bool active = x < p.nx && y < p.ny && (D == 2 || z < p.nz);
    Real f[L::Q];
    if (active) gather<LAT>(A, p, x, y, z, f);
    if (!mbar_wait(bar_a, 0)) {
        if (tid == 0) atomicOr(p.err, kErrTimeout);
        mbar_wait(bar_a, 0);  // never leave with the copy still landing in shared memory
        return;
    }
    if (!active) return;
    const Real* tc = tile + ((tz + (D == 3 ? R : 0)) * SY + (ty + R)) * SX + (tx + kGhostX);
    Real F[3];
    force_from<LAT, ORD, Real, SX, SY>(tc, par<Real>(p.G, p.G_f), F);
    collide<LAT, COLL>(f, F, p);
    const long long c = cell_of(p, x, y, z);
    sfor<L::Q>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        B[static_cast<long long>(b) * p.N + c] = f[b];
    });
}

// Standard bounce-back on the solid band y < wall_rows (2-D): a solid node takes
// no collision and sends every population back the way it came, f*_b = f_{-b}.
// Runs after k_fused on the same stream and overwrites what that kernel wrote
// for the band, so the fluid kernels carry no wall test.
template <int LAT, class Real>
__global__ void __launch_bounds__(256) k_bounce(const Real* __restrict__ A, Real* __restrict__ B, DevParams p)
{
    using L = Lattice<LAT>;
    const long long n = static_cast<long long>(p.nx) * p.wall_rows;
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % p.nx), y = static_cast<int>(i / p.nx);
        Real f[L::Q];
        gather<LAT>(A, p, x, y, 0, f);
        const long long c = cell_of(p, x, y, 0);
        sfor<L::Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int ob = opposite<LAT>(b);
            static_assert(ob >= 0, "velocity set without an opposite");
            B[static_cast<long long>(b) * p.N + c] = f[ob];
        });
    }
}

// ---- one-pass schedule ------------------------------------------------------------
// A CTA owns a tile of the plane normal to the marching axis (3-D: TX x TY cells
// of an xy plane, marching in z; 2-D: TX cells of an x line, marching in y) and
// a chunk of ZC slabs along the marching axis.  It keeps psi of the tile plus
// its stencil halo for the 2R+1 slabs around the current one in a shared-memory
// ring: before colliding slab m it computes psi of slab m + R (pull gather of
// the halo-extended tile), so psi never goes to HBM and each population is read
// from HBM once per step (the second gather for the collision hits L1/L2).
// Chunks are the slowest grid index, so co-resident CTAs hold neighbouring tiles
// at the same slabs and their halo reads are shared through L2.
// Ring slot of slab m (m >= -3): a modulo by a compile-time constant.
__host__ __device__ constexpr int ring_slot(int m, int ns)
{
    return static_cast<int>(static_cast<unsigned>(m + 4 * ns) % static_cast<unsigned>(ns));
}

__device__ __forceinline__ int wrap_any(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

template <int LAT, int ORD, class Real, int EX, int E, int NS>
__device__ __forceinline__ void force_ring(const Real* ring, int m, int cx, int cy, Real G, Real (&F)[3])
{
    using L = Lattice<LAT>;
    using S = Stencil<L::D, ORD>;
    constexpr int R = S::radius;
    const Real* base[2 * R + 1];
#pragma unroll
    for (int s = 0; s < 2 * R + 1; ++s) base[s] = ring + ring_slot(m - R + s, NS) * E + cy * EX + cx;
    Real ax = Real(0), ay = Real(0), az = Real(0);
    sfor<S::n / 2>([&](auto kI) {
        constexpr int a = 2 * decltype(kI)::value;
        constexpr int ex = S::T.v[a][0], ey = S::T.v[a][1], ez = S::T.v[a][2];
        constexpr int dm = (L::D == 3) ? ez : ey;  // offset along the marching axis
        constexpr int dq = (L::D == 3) ? ey : 0;   // in-plane offset of the second axis
        constexpr double wt = S::T.w[a] * L::cs2;
        const Real d = base[dm + R][dq * EX + ex] - base[R - dm][-(dq * EX + ex)];
        if (ex != 0) ax += Real(wt * ex) * d;
        if (ey != 0) ay += Real(wt * ey) * d;
        if (ez != 0) az += Real(wt * ez) * d;
    });
    const Real gp = -G * base[R][0];
    F[0] = gp * ax;
    F[1] = gp * ay;
    F[2] = gp * az;
}

// Per-direction base pointers of the population buffers, passed by value so
// they sit in the kernel's parameter (constant) bank: the address of f_b at
// cell offset o is one multiply-add on in[b].
template <class Real, int Q>
struct Pops {
    const Real* in[Q];
    Real* out[Q];
};

template <class Real, int Q>
Pops<Real, Q> make_pops(const void* fin, void* fout, long long N)
{
    Pops<Real, Q> P;
    for (int b = 0; b < Q; ++b) {
        P.in[b] = static_cast<const Real*>(fin) + static_cast<long long>(b) * N;
        P.out[b] = static_cast<Real*>(fout) + static_cast<long long>(b) * N;
    }
    return P;
}

// i - j on a periodic axis of length n for |j| <= 3 <= n, without a division.
__device__ __forceinline__ int wrap_near(int i, int n)
{
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

// o[j + RE] = wrap(i - j) * scale for j = -RE..RE, with i already in [0, n).
template <int RE>
__device__ __forceinline__ void axis_offsets(int i, int n, int scale, int (&o)[2 * RE + 1])
{
#pragma unroll
    for (int j = -RE; j <= RE; ++j) o[j + RE] = wrap_near(i - j, n) * scale;
}

// Pull gather through precomputed wrapped offsets: f_b = A_b[zo(cz) + yo(cy) + xo(cx)]
// where xo[j + RE] = wrap(x - j), yo[j + RE] = wrap(y - j) * nx, and zo likewise
// (RE = lattice reach).  All offsets are within one direction's array (< 2^31).
template <int LAT, class Real, int RE>
__device__ __forceinline__ void gather_off(const Pops<Real, Lattice<LAT>::Q>& P, const int (&xo)[2 * RE + 1],
                                           const int (&yo)[2 * RE + 1], const int (&zo)[2 * RE + 1],
                                           Real (&f)[Lattice<LAT>::Q])
{
    using L = Lattice<LAT>;
    sfor<L::Q>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
        f[b] = __ldg(P.in[b] + (zo[cz + RE] + yo[cy + RE] + xo[cx + RE]));
    });
}

// ST selects where the interior populations wait between their gather for psi
// (slab m + R) and their collision (R slabs later): 0 = gathered again (L1/L2),
// 1 = registers (R = 1 only), 2 = dynamic shared memory, [R + 1][Q][TX*TY].
template <int LAT, int ORD, int COLL, class Real, int TX, int TY, int ZC, int MINB, int ST>
__global__ void __launch_bounds__(TX * TY, MINB)
    k_onepass(const __grid_constant__ Pops<Real, Lattice<LAT>::Q> P, DevParams p, int ntx, int nty)
{
    using L = Lattice<LAT>;
    using S = Stencil<L::D, ORD>;
    constexpr int D = L::D;
    constexpr int R = S::radius;
    constexpr int RE = L::reach;
    constexpr int Q = L::Q;
    constexpr int NT = TX * TY;
    constexpr int EX = TX + 2 * R;
    constexpr int EY = (D == 3) ? TY + 2 * R : 1;
    constexpr int E = EX * EY;
    constexpr int H = E - NT;          // halo cells of the extended tile
    constexpr int NS = 2 * R + 2;      // ring depth: one spare slot, one barrier per slab
    constexpr bool kStash = (ST == 1);
    constexpr bool kSmem = (ST == 2);
    constexpr int NST = R + 1;         // shared-memory stash slots
    static_assert(H <= NT, "halo larger than the block");
    static_assert(ST != 1 || R == 1, "register stash needs a radius-1 stencil");
    __shared__ Real ring[NS * E];
    extern __shared__ unsigned char dyn_smem[];
    Real* stash = reinterpret_cast<Real*>(dyn_smem);  // [NST][Q][NT] when kSmem

    const int ncol = ntx * nty;
    const int col = blockIdx.x % ncol;
    const int chunk = blockIdx.x / ncol;
    const int x0 = (col % ntx) * TX;
    const int y0 = (D == 3) ? (col / ntx) * TY : 0;
    const int nm = (D == 3) ? p.nz : p.ny;
    const int m0 = chunk * ZC;
    const int m1 = (m0 + ZC < nm) ? m0 + ZC : nm;
    const int mscale = (D == 3) ? p.nx * p.ny : p.nx;  // offset of one slab
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;

    // interior cell of this thread (extended-tile position (tx + R, ty + R))
    const int ix = x0 + tx, iy = y0 + ty;
    int ixo[2 * RE + 1], iyo[2 * RE + 1];
    axis_offsets<RE>(wrap_any(ix, p.nx), p.nx, 1, ixo);
    if (D == 3) axis_offsets<RE>(wrap_any(iy, p.ny), p.ny, p.nx, iyo);
    const int i_slot = (D == 3 ? (ty + R) * EX : 0) + tx + R;

    // halo cell of this thread (tid < H): the ring of the extended tile
    const bool has_halo = tid < H;
    int hex = 0, hey = 0;
    if (D == 3) {
        if (tid < R * EX) {
            hex = tid % EX; hey = tid / EX;
        } else if (tid < 2 * R * EX) {
            hex = (tid - R * EX) % EX; hey = EY - R + (tid - R * EX) / EX;
        } else {
            const int h = tid - 2 * R * EX;
            const int k = h % (2 * R);
            hey = R + h / (2 * R);
            hex = (k < R) ? k : TX + k;
        }
    } else {
        hex = (tid < R) ? tid : TX + tid;
    }
    int hxo[2 * RE + 1], hyo[2 * RE + 1];
    axis_offsets<RE>(wrap_any(x0 - R + hex, p.nx), p.nx, 1, hxo);
    if (D == 3) axis_offsets<RE>(wrap_any(y0 - R + hey, p.ny), p.ny, p.nx, hyo);
    const int h_slot = hey * EX + hex;
    const int zero[2 * RE + 1] = {};

    Real fcur[Q], fnxt[Q];

    // psi of slab m for the extended tile; the interior populations go to fnxt
    auto psi_slab = [&](int m) {
        int mo[2 * RE + 1];
        axis_offsets<RE>(wrap_near(m, nm), nm, mscale, mo);
        Real* dst = ring + ring_slot(m, NS) * E;
        {
            if (D == 3)
                gather_off<LAT, Real, RE>(P, ixo, iyo, mo, fnxt);
            else
                gather_off<LAT, Real, RE>(P, ixo, mo, zero, fnxt);
            Real s = Real(0);
            sfor<Q>([&](auto bI) { s += fnxt[decltype(bI)::value]; });
            const Real rho = std::is_same<Real, float>::value ? Real(p.rho_bar) + s : s;
            dst[i_slot] = psi_of<LAT>(rho, p);
            if (kSmem) {
                Real* st = stash + static_cast<unsigned>(m + 4 * NST) % NST * (Q * NT) + tid;
                sfor<Q>([&](auto bI) {
                    constexpr int bb = decltype(bI)::value;
                    st[bb * NT] = fnxt[bb];
                });
            }
        }
        if (has_halo) {
            Real f[Q];
            if (D == 3)
                gather_off<LAT, Real, RE>(P, hxo, hyo, mo, f);
            else
                gather_off<LAT, Real, RE>(P, hxo, mo, zero, f);
            Real s = Real(0);
            sfor<Q>([&](auto bI) { s += f[decltype(bI)::value]; });
            const Real rho = std::is_same<Real, float>::value ? Real(p.rho_bar) + s : s;
            dst[h_slot] = psi_of<LAT>(rho, p);
        }
    };

    for (int m = m0 - R; m < m0 + R; ++m) {
        psi_slab(m);
        if (kStash && m == m0 + R - 1) {
#pragma unroll
            for (int b = 0; b < Q; ++b) fcur[b] = fnxt[b];
        }
    }
    const bool active = ix < p.nx && (D == 2 || iy < p.ny);
    const int cell_xy = (D == 3) ? iy * p.nx + ix : ix;
    for (int m = m0; m < m1; ++m) {
        psi_slab(m + R);
        __syncthreads();
        if (active) {
            if (kSmem) {
                const Real* st = stash + static_cast<unsigned>(m + 4 * NST) % NST * (Q * NT) + tid;
                sfor<Q>([&](auto bI) {
                    constexpr int bb = decltype(bI)::value;
                    fcur[bb] = st[bb * NT];
                });
            } else if (!kStash) {
                int mo[2 * RE + 1];
                axis_offsets<RE>(m, nm, mscale, mo);
                if (D == 3)
                    gather_off<LAT, Real, RE>(P, ixo, iyo, mo, fcur);
                else
                    gather_off<LAT, Real, RE>(P, ixo, mo, zero, fcur);
            }
            Real F[3];
            force_ring<LAT, ORD, Real, EX, E, NS>(ring, m, tx + R, (D == 3) ? ty + R : 0, par<Real>(p.G, p.G_f), F);
            collide<LAT, COLL>(fcur, F, p);
            const int c = m * mscale + cell_xy;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                P.out[b][c] = fcur[b];
            });
        }
        if (kStash) {
#pragma unroll
            for (int b = 0; b < Q; ++b) fcur[b] = fnxt[b];
        }
    }
}

// One-pass schedule for domains whose x-row fits in shared memory (3-D,
// radius-1 stencils): a tile is TY whole rows, so direction b's staged rows for
// slab s -- rows y0 - 1 - c_by .. y0 + TY - c_by of plane s - c_bz, all NX cells --
// are one contiguous range of global memory, copied by one cp.async.bulk (two
// where the range wraps in y).  The periodic x shift becomes an index wrap in
// shared memory, and the psi ring carries one wrapped column on each side.
// NSTG stages are in flight; the interior populations wait one slab in registers.
// PROD = 1 adds a 32-thread producer warp that only issues the copies (and takes
// part in the block barriers), so no compute warp carries the copy issue.
// PROD = 2 also marks the stored populations evict-first in L2 (they are not read
// again within the step), leaving L2 to the halo rows neighbouring tiles re-read.
template <int LAT, int ORD, int COLL, class Real, int NX, int TY, int ZC, int NSTG, int PROD>
__global__ void __launch_bounds__(NX * TY + (PROD ? 32 : 0), 1)
    k_onepass_row(const __grid_constant__ Pops<Real, Lattice<LAT>::Q> P, DevParams p, int zc_run)
{
    using L = Lattice<LAT>;
    using S = Stencil<3, ORD>;
    constexpr int R = S::radius;
    constexpr int Q = L::Q;
    static_assert(L::D == 3 && R == 1 && L::reach == 1, "row staging is written for 3-D radius-1 stencils");
    constexpr int NT = NX * TY;
    constexpr int EY = TY + 2 * R;
    constexpr int EX = NX + 2 * R;   // ring row: one wrapped psi column on each side
    constexpr int E = EX * EY;
    constexpr int NS = 2 * R + 2;
    constexpr int STG = Q * EY * NX;  // values per stage: [Q][EY][NX]
    static_assert(NT % 32 == 0 && NT <= 1024, "block");
    static_assert((NX * sizeof(Real)) % 16 == 0, "16-byte rows");
    __shared__ Real ring[NS * E];
    __shared__ alignas(8) unsigned long long bars[NSTG];
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    Real* stage = reinterpret_cast<Real*>(dyn_smem);  // [NSTG][STG]

    const int nty = (p.ny + TY - 1) / TY;
    const int trow = blockIdx.x % nty;
    const int chunk = blockIdx.x / nty;
    const int y0 = trow * TY;
    const int nm = p.nz;
    const int zc = ZC > 0 ? ZC : zc_run;  // ZC = 0: chunk length chosen at launch
    const int m0 = chunk * zc;
    const int m1 = (m0 + zc < nm) ? m0 + zc : nm;
    const int plane = NX * p.ny;
    const int tid = threadIdx.x;
    const int tx = tid % NX, ty = tid / NX;
    const int lane = tid & 31;
    const bool issuer = PROD ? tid >= NT : tid < 32;
    const bool compute = !PROD || tid < NT;

    if (tid == 0) {
        for (int k = 0; k < NSTG; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
    }
    __syncthreads();

    int cby = 0, cbz = 0;
    const Real* src_b = nullptr;
    sfor<Q>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        constexpr int vy = L::T.v[b][1], vz = L::T.v[b][2];
        if (lane == b) {
            cby = vy;
            cbz = vz;
            src_b = P.in[b];
        }
    });
    const int base = m0 - R;
    auto issue = [&](int s) {
        const int slot = (s - base) % NSTG;
        const uint32_t bar = smem_u32(&bars[slot]);
        if (lane == 0) mbar_expect_tx(bar, static_cast<uint32_t>(STG * sizeof(Real)));
        __syncwarp();
        if (lane < Q) {
            fence_proxy_async_smem();
            const Real* pl = src_b + static_cast<long long>(wrap_any(s - cbz, nm)) * plane;
            uint32_t dst = smem_u32(stage + slot * STG + lane * (EY * NX));
            int y = y0 - R - cby, left = EY;
            while (left > 0) {
                const int yw = wrap_any(y, p.ny);
                const int n = (p.ny - yw < left) ? p.ny - yw : left;
                bulk_g2s(dst, pl + static_cast<long long>(yw) * NX, static_cast<uint32_t>(n * NX * sizeof(Real)), bar);
                dst += static_cast<uint32_t>(n * NX * sizeof(Real));
                y += n;
                left -= n;
            }
        }
    };
    uint32_t phase = 0;
    bool ok = true;
    auto wait_stage = [&](int s) -> const Real* {
        const int slot = (s - base) % NSTG;
        if (ok && !mbar_wait(smem_u32(&bars[slot]), (phase >> slot) & 1u)) ok = false;  // after a timeout, stop waiting
        phase ^= 1u << slot;
        return stage + slot * STG;
    };

    // stage column of x - c_x for c_x = -1 and +1 (x periodic within the row)
    const int xm = (tx + 1 == NX) ? 0 : tx + 1;   // c_x = -1
    const int xp = (tx == 0) ? NX - 1 : tx - 1;   // c_x = +1
    // f of the cell in frame row fy of the stage (pull: row fy of direction b)
    auto load_cell = [&](const Real* st, int fy, Real (&f)[Q]) {
        const Real* r = st + fy * NX;
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int vx = L::T.v[b][0];
            const int c = vx == 0 ? tx : (vx > 0 ? xp : xm);
            f[b] = r[b * (EY * NX) + c];
        });
    };
    auto rho_psi = [&](const Real (&f)[Q]) {
        Real sum = Real(0);
        sfor<Q>([&](auto bI) { sum += f[decltype(bI)::value]; });
        const Real rho = std::is_same<Real, float>::value ? Real(p.rho_bar) + sum : sum;
        return psi_of<LAT>(rho, p);
    };
    Real fcur[Q], fnxt[Q];
    auto put_psi = [&](Real* dst, int fy, Real v) {
        Real* row = dst + fy * EX;
        row[tx + R] = v;
        if (tx == 0) row[NX + R] = v;       // wrapped column right of the row
        if (tx == NX - 1) row[0] = v;       // wrapped column left of the row
    };
    auto psi_slab = [&](int s) {
        const Real* st = wait_stage(s);
        Real* dst = ring + ring_slot(s, NS) * E;
        load_cell(st, ty + R, fnxt);
        put_psi(dst, ty + R, rho_psi(fnxt));
        // halo rows of the frame: fy = 0 and fy = EY - 1, NX cells each
        for (int k = ty; k < 2 * R; k += TY) {
            const int fy = (k < R) ? k : EY - 2 * R + k;
            Real f[Q];
            load_cell(st, fy, f);
            put_psi(dst, fy, rho_psi(f));
        }
    };

    int next = base;
    const int last = m1 - 1 + R;
    if (issuer)
        for (; next <= last && next < base + NSTG; ++next) issue(next);
    if (compute)
        for (int s = m0 - R; s < m0 + R; ++s) psi_slab(s);
#pragma unroll
    for (int b = 0; b < Q; ++b) fcur[b] = fnxt[b];
    __syncthreads();
    if (issuer)
        for (; next <= last && next < m0 + R + NSTG; ++next) issue(next);

    const bool active = compute && (y0 + ty) < p.ny;
    const int cell_xy = (y0 + ty) * NX + tx;
    for (int m = m0; m < m1; ++m) {
        if (compute) psi_slab(m + R);
        __syncthreads();
        if (issuer)
            for (; next <= last && next <= m + R + NSTG; ++next) issue(next);
        if (active) {
            Real F[3];
            force_ring<LAT, ORD, Real, EX, E, NS>(ring, m, tx + R, ty + R, par<Real>(p.G, p.G_f), F);
            collide<LAT, COLL>(fcur, F, p);
            const int c = m * plane + cell_xy;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                if (PROD == 2)
                    __stcs(P.out[b] + c, fcur[b]);
                else
                    P.out[b][c] = fcur[b];
            });
        }
#pragma unroll
        for (int b = 0; b < Q; ++b) fcur[b] = fnxt[b];
    }
    if (!ok && tid == 0) atomicOr(p.err, kErrTimeout);
}

// Persistent form of the whole-row schedule: one block per SM walks the
// (row pair, chunk) items chunk-major with stride gridDim.x, so the blocks that
// run at a time still cover neighbouring row pairs at similar z (their shared
// halo rows meet in L2).  The producer warp issues one global sequence of slabs
// across the block's items: as soon as the last slabs of an item are consumed it
// runs on into the next item's first slabs, which load while the current item's
// last rows collide, so the copy stream never restarts from empty.
template <int LAT, int ORD, int COLL, class Real, int NX, int TY, int NSTG>
__global__ void __launch_bounds__(NX * TY + 32, 1)
    k_onepass_rowp(const __grid_constant__ Pops<Real, Lattice<LAT>::Q> P, DevParams p, int zc, int nitems)
{
    using L = Lattice<LAT>;
    using S = Stencil<3, ORD>;
    constexpr int R = S::radius;
    constexpr int Q = L::Q;
    static_assert(L::D == 3 && R == 1 && L::reach == 1, "row staging is written for 3-D radius-1 stencils");
    constexpr int NT = NX * TY;
    constexpr int EY = TY + 2 * R;
    constexpr int EX = NX + 2 * R;
    constexpr int E = EX * EY;
    constexpr int NS = 2 * R + 2;
    constexpr int STG = Q * EY * NX;
    static_assert(NT % 32 == 0 && NT <= 1024 && NSTG >= 2 * R && NSTG <= 32, "block / stages");
    static_assert((NX * sizeof(Real)) % 16 == 0, "16-byte rows");
    __shared__ Real ring[NS * E];
    __shared__ alignas(8) unsigned long long bars[NSTG];
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    Real* stage = reinterpret_cast<Real*>(dyn_smem);  // [NSTG][STG]

    const int nty = (p.ny + TY - 1) / TY;
    const int nm = p.nz;
    const int plane = NX * p.ny;
    const int tid = threadIdx.x;
    const int tx = tid % NX, ty = tid / NX;
    const int lane = tid & 31;
    const bool producer = tid >= NT;

    if (tid == 0) {
        for (int k = 0; k < NSTG; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
    }
    __syncthreads();

    int cby = 0, cbz = 0;
    const Real* src_b = nullptr;
    sfor<Q>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        constexpr int vy = L::T.v[b][1], vz = L::T.v[b][2];
        if (lane == b) {
            cby = vy;
            cbz = vz;
            src_b = P.in[b];
        }
    });
    // producer: the next slab of the block's global sequence
    int p_it = blockIdx.x, p_y0 = 0, p_next = 0, p_last = -1;
    auto p_load_item = [&]() {
        if (p_it >= nitems) return;
        const int m0 = (p_it / nty) * zc;
        const int m1 = (m0 + zc < nm) ? m0 + zc : nm;
        p_y0 = (p_it % nty) * TY;
        p_next = m0 - R;
        p_last = m1 - 1 + R;
    };
    p_load_item();
    long long issued = 0;
    auto issue_next = [&]() {
        const int slot = static_cast<int>(issued % NSTG);
        const uint32_t bar = smem_u32(&bars[slot]);
        if (lane == 0) mbar_expect_tx(bar, static_cast<uint32_t>(STG * sizeof(Real)));
        __syncwarp();
        if (lane < Q) {
            fence_proxy_async_smem();
            const Real* pl = src_b + static_cast<long long>(wrap_any(p_next - cbz, nm)) * plane;
            uint32_t dst = smem_u32(stage + slot * STG + lane * (EY * NX));
            int y = p_y0 - R - cby, left = EY;
            while (left > 0) {
                const int yw = wrap_any(y, p.ny);
                const int n = (p.ny - yw < left) ? p.ny - yw : left;
                bulk_g2s(dst, pl + static_cast<long long>(yw) * NX, static_cast<uint32_t>(n * NX * sizeof(Real)), bar);
                dst += static_cast<uint32_t>(n * NX * sizeof(Real));
                y += n;
                left -= n;
            }
        }
        ++issued;
        if (++p_next > p_last) {
            p_it += gridDim.x;
            p_load_item();
        }
    };
    // a slot is refilled once the slab NSTG earlier in the sequence is consumed
    auto issue_upto = [&](long long consumed) {
        while (p_it < nitems && issued < consumed + NSTG) issue_next();
    };

    uint32_t phase = 0;
    bool ok = true;
    long long consumed = 0;  // the same count in every thread
    auto wait_seq = [&](long long q) -> const Real* {
        const int slot = static_cast<int>(q % NSTG);
        if (ok && !mbar_wait(smem_u32(&bars[slot]), (phase >> slot) & 1u)) ok = false;  // after a timeout, stop waiting
        phase ^= 1u << slot;
        return stage + slot * STG;
    };
    const int xm = (tx + 1 == NX) ? 0 : tx + 1;   // c_x = -1
    const int xp = (tx == 0) ? NX - 1 : tx - 1;   // c_x = +1
    auto load_cell = [&](const Real* st, int fy, Real (&f)[Q]) {
        const Real* r = st + fy * NX;
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int vx = L::T.v[b][0];
            const int c = vx == 0 ? tx : (vx > 0 ? xp : xm);
            f[b] = r[b * (EY * NX) + c];
        });
    };
    auto rho_psi = [&](const Real (&f)[Q]) {
        Real sum = Real(0);
        sfor<Q>([&](auto bI) { sum += f[decltype(bI)::value]; });
        const Real rho = std::is_same<Real, float>::value ? Real(p.rho_bar) + sum : sum;
        return psi_of<LAT>(rho, p);
    };
    Real fcur[Q], fnxt[Q];
    auto put_psi = [&](Real* dst, int fy, Real v) {
        Real* row = dst + fy * EX;
        row[tx + R] = v;
        if (tx == 0) row[NX + R] = v;
        if (tx == NX - 1) row[0] = v;
    };
    auto psi_slab = [&](int s, long long q) {
        const Real* st = wait_seq(q);
        Real* dst = ring + ring_slot(s, NS) * E;
        load_cell(st, ty + R, fnxt);
        put_psi(dst, ty + R, rho_psi(fnxt));
        for (int k = ty; k < 2 * R; k += TY) {
            const int fy = (k < R) ? k : EY - 2 * R + k;
            Real f[Q];
            load_cell(st, fy, f);
            put_psi(dst, fy, rho_psi(f));
        }
    };

    if (producer) issue_upto(0);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int y0 = (it % nty) * TY;
        const int m0 = (it / nty) * zc;
        const int m1 = (m0 + zc < nm) ? m0 + zc : nm;
        if (!producer)
            for (int s = m0 - R; s < m0 + R; ++s) psi_slab(s, consumed + (s - (m0 - R)));
        consumed += 2 * R;
#pragma unroll
        for (int b = 0; b < Q; ++b) fcur[b] = fnxt[b];
        __syncthreads();
        if (producer) issue_upto(consumed);
        const bool active = !producer && (y0 + ty) < p.ny;
        const int cell_xy = (y0 + ty) * NX + tx;
        for (int m = m0; m < m1; ++m) {
            if (!producer) psi_slab(m + R, consumed);
            ++consumed;
            __syncthreads();
            // every thread is past psi of slab m + R: its stage can be refilled, and
            // after the item's last slab the next item's first slabs start loading
            if (producer) issue_upto(consumed);
            if (active) {
                Real F[3];
                force_ring<LAT, ORD, Real, EX, E, NS>(ring, m, tx + R, ty + R, par<Real>(p.G, p.G_f), F);
                collide<LAT, COLL>(fcur, F, p);
                const int c = m * plane + cell_xy;
                sfor<Q>([&](auto bI) {
                    constexpr int b = decltype(bI)::value;
                    __stcs(P.out[b] + c, fcur[b]);
                });
            }
#pragma unroll
            for (int b = 0; b < Q; ++b) fcur[b] = fnxt[b];
        }
        __syncthreads();  // the ring is reused by the next item
    }
    if (!ok && tid == 0) atomicOr(p.err, kErrTimeout);
}

// One-pass schedule with bulk-copy staging for 2-D lattices of reach 1 (D2Q9),
// any force stencil up to radius 3.  A tile is TX cells of a row; the march runs
// along y.  For row s, direction b needs row s - c_by over x0 - XP .. x0 + TX + XP
// (XP = 16 bytes of values >= R + 1): one contiguous segment, copied by one
// cp.async.bulk (two where it crosses the periodic x edge).  A stage stays
// resident until the row collides, so the interior populations are read from
// shared memory twice (psi, then collision) and nothing waits in registers;
// stages hold NSTG rows, NSTG - R - 1 of them in flight.  A producer warp issues
// the copies.
template <int LAT, int ORD, int COLL, class Real, int TX, int ZC, int NSTG>
__global__ void __launch_bounds__(TX + 32, 1)
    k_onepass_seg(const __grid_constant__ Pops<Real, Lattice<LAT>::Q> P, DevParams p, int ntx)
{
    using L = Lattice<LAT>;
    using S = Stencil<2, ORD>;
    constexpr int R = S::radius;
    constexpr int Q = L::Q;
    static_assert(L::D == 2 && L::reach == 1, "segment staging is written for 2-D reach-1 lattices");
    constexpr int XP = 16 / static_cast<int>(sizeof(Real));
    static_assert(XP >= R + 1 && TX % XP == 0 && TX % 32 == 0, "x pad / tile");
    constexpr int W = TX + 2 * XP;   // staged segment length
    constexpr int EX = TX + 2 * R;   // psi ring row
    constexpr int NS = 2 * R + 2;
    constexpr int STG = Q * W;
    static_assert(NSTG >= R + 2 && NSTG >= 2 * R, "one row in flight; the 2R warm-up rows staged at once");
    __shared__ Real ring[NS * EX];
    __shared__ alignas(8) unsigned long long bars[NSTG];
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    Real* stage = reinterpret_cast<Real*>(dyn_smem);  // [NSTG][Q][W]

    const int tile = blockIdx.x % ntx;
    const int chunk = blockIdx.x / ntx;
    const int x0 = tile * TX;
    const int nm = p.ny;
    const int m0 = chunk * ZC;
    const int m1 = (m0 + ZC < nm) ? m0 + ZC : nm;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const bool producer = tid >= TX;

    if (tid == 0) {
        for (int k = 0; k < NSTG; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
    }
    __syncthreads();

    int cby = 0;
    const Real* src_b = nullptr;
    sfor<Q>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        constexpr int vy = L::T.v[b][1];
        if (lane == b) {
            cby = vy;
            src_b = P.in[b];
        }
    });
    const int base = m0 - R;
    auto issue = [&](int s) {
        const int slot = (s - base) % NSTG;
        const uint32_t bar = smem_u32(&bars[slot]);
        if (lane == 0) mbar_expect_tx(bar, static_cast<uint32_t>(STG * sizeof(Real)));
        __syncwarp();
        if (lane < Q) {
            fence_proxy_async_smem();
            const Real* row = src_b + static_cast<long long>(wrap_any(s - cby, nm)) * p.nx;
            uint32_t dst = smem_u32(stage + slot * STG + lane * W);
            int xs = x0 - XP, left = W;
            while (left > 0) {
                const int x = wrap_any(xs, p.nx);
                const int n = (p.nx - x < left) ? p.nx - x : left;
                bulk_g2s(dst, row + x, static_cast<uint32_t>(n * sizeof(Real)), bar);
                dst += static_cast<uint32_t>(n * sizeof(Real));
                xs += n;
                left -= n;
            }
        }
    };
    uint32_t phase = 0;
    bool ok = true;
    auto stage_of = [&](int s) { return stage + ((s - base) % NSTG) * STG; };
    auto wait_stage = [&](int s) {
        const int slot = (s - base) % NSTG;
        if (ok && !mbar_wait(smem_u32(&bars[slot]), (phase >> slot) & 1u)) ok = false;  // after a timeout, stop waiting
        phase ^= 1u << slot;
    };
    // f of the cell at tile offset cx (-R .. TX + R - 1) from stage st (pull)
    auto load_cell = [&](const Real* st, int cx, Real (&f)[Q]) {
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int vx = L::T.v[b][0];
            f[b] = st[b * W + cx + XP - vx];
        });
    };
    auto rho_psi = [&](const Real (&f)[Q]) {
        Real sum = Real(0);
        sfor<Q>([&](auto bI) { sum += f[decltype(bI)::value]; });
        const Real rho = std::is_same<Real, float>::value ? Real(p.rho_bar) + sum : sum;
        return psi_of<LAT>(rho, p);
    };
    auto psi_slab = [&](int s) {
        wait_stage(s);
        const Real* st = stage_of(s);
        Real* dst = ring + ring_slot(s, NS) * EX;
        Real f[Q];
        load_cell(st, tid, f);
        dst[tid + R] = rho_psi(f);
        if (tid < 2 * R) {
            const int cx = (tid < R) ? tid - R : TX + tid - R;
            load_cell(st, cx, f);
            dst[cx + R] = rho_psi(f);
        }
    };

    int next = base;
    const int last = m1 - 1 + R;
    if (producer)
        for (; next <= last && next < base + NSTG; ++next) issue(next);
    if (!producer)
        for (int s = m0 - R; s < m0 + R; ++s) psi_slab(s);
    __syncthreads();
    // slabs below m0 are consumed (psi only): slab k may refill slab k - NSTG's stage
    if (producer)
        for (; next <= last && next < m0 + NSTG; ++next) issue(next);

    const bool active = !producer && (x0 + tid) < p.nx;
    for (int m = m0; m < m1; ++m) {
        if (!producer) psi_slab(m + R);
        __syncthreads();
        // every thread is past the collision of row m - 1
        if (producer)
            for (; next <= last && next <= m - 1 + NSTG; ++next) issue(next);
        if (active) {
            Real f[Q];
            load_cell(stage_of(m), tid, f);
            Real F[3];
            force_ring<LAT, ORD, Real, EX, EX, NS>(ring, m, tid + R, 0, par<Real>(p.G, p.G_f), F);
            collide<LAT, COLL>(f, F, p);
            const int c = m * p.nx + x0 + tid;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                __stcs(P.out[b] + c, f[b]);
            });
        }
    }
    if (!ok && tid == 0) atomicOr(p.err, kErrTimeout);
}

// One-pass schedule with asynchronous staging (FP32 hot path): the populations
// of slab s (interior and halo cells of the tile) are copied global -> shared
// with cp.async one iteration before psi of slab s is formed, and the interior
// ones stay staged until slab s collides R iterations later.  Load latency is
// then off the critical path without holding registers.
// Shared memory: interior [R+2][Q][NT], halo [2][Q][H] (dynamic), psi ring (static).
template <int LAT, int ORD, int COLL, class Real, int TX, int TY, int ZC, int MINB>
__global__ void __launch_bounds__(TX * TY, MINB)
    k_onepass_async(const __grid_constant__ Pops<Real, Lattice<LAT>::Q> P, DevParams p, int ntx, int nty)
{
    using L = Lattice<LAT>;
    using S = Stencil<L::D, ORD>;
    constexpr int D = L::D;
    constexpr int R = S::radius;
    constexpr int RE = L::reach;
    constexpr int Q = L::Q;
    constexpr int NT = TX * TY;
    constexpr int EX = TX + 2 * R;
    constexpr int EY = (D == 3) ? TY + 2 * R : 1;
    constexpr int E = EX * EY;
    constexpr int H = E - NT;
    constexpr int NS = 2 * R + 2;
    constexpr int NI = R + 2;  // interior staging slots
    static_assert(H <= NT, "halo larger than the block");
    static_assert(sizeof(Real) == 4, "4-byte cp.async staging");
    __shared__ Real ring[NS * E];
    extern __shared__ unsigned char dyn_smem[];
    Real* stI = reinterpret_cast<Real*>(dyn_smem);  // [NI][Q][NT]
    Real* stH = stI + NI * Q * NT;                  // [2][Q][H]

    const int ncol = ntx * nty;
    const int col = blockIdx.x % ncol;
    const int chunk = blockIdx.x / ncol;
    const int x0 = (col % ntx) * TX;
    const int y0 = (D == 3) ? (col / ntx) * TY : 0;
    const int nm = (D == 3) ? p.nz : p.ny;
    const int m0 = chunk * ZC;
    const int m1 = (m0 + ZC < nm) ? m0 + ZC : nm;
    const int mscale = (D == 3) ? p.nx * p.ny : p.nx;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;

    const int ix = x0 + tx, iy = y0 + ty;
    int ixo[2 * RE + 1], iyo[2 * RE + 1];
    axis_offsets<RE>(wrap_any(ix, p.nx), p.nx, 1, ixo);
    if (D == 3) axis_offsets<RE>(wrap_any(iy, p.ny), p.ny, p.nx, iyo);
    const int i_slot = (D == 3 ? (ty + R) * EX : 0) + tx + R;

    const bool has_halo = tid < H;
    int hex = 0, hey = 0;
    if (D == 3) {
        if (tid < R * EX) {
            hex = tid % EX; hey = tid / EX;
        } else if (tid < 2 * R * EX) {
            hex = (tid - R * EX) % EX; hey = EY - R + (tid - R * EX) / EX;
        } else {
            const int h = tid - 2 * R * EX;
            const int k = h % (2 * R);
            hey = R + h / (2 * R);
            hex = (k < R) ? k : TX + k;
        }
    } else {
        hex = (tid < R) ? tid : TX + tid;
    }
    int hxo[2 * RE + 1], hyo[2 * RE + 1];
    axis_offsets<RE>(wrap_any(x0 - R + hex, p.nx), p.nx, 1, hxo);
    if (D == 3) axis_offsets<RE>(wrap_any(y0 - R + hey, p.ny), p.ny, p.nx, hyo);
    const int h_slot = hey * EX + hex;
    const int zero[2 * RE + 1] = {};
    const uint32_t stI_a = smem_u32(stI) + 4u * tid;
    const uint32_t stH_a = smem_u32(stH) + 4u * tid;

    // issue the copies of slab s (own interior cell, own halo cell) and commit
    auto stage = [&](int s) {
        int mo[2 * RE + 1];
        axis_offsets<RE>(wrap_near(s, nm), nm, mscale, mo);
        const int* yi = (D == 3) ? iyo : mo;
        const int* zi = (D == 3) ? mo : zero;
        const uint32_t di = stI_a + 4u * static_cast<uint32_t>(ring_slot(s, NI) * Q * NT);
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
            cp_async4(di + 4u * b * NT, P.in[b] + (zi[cz + RE] + yi[cy + RE] + ixo[cx + RE]));
        });
        if (has_halo) {
            const int* yh = (D == 3) ? hyo : mo;
            const uint32_t dh = stH_a + 4u * static_cast<uint32_t>((s & 1) * Q * H);
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
                cp_async4(dh + 4u * b * H, P.in[b] + (zi[cz + RE] + yh[cy + RE] + hxo[cx + RE]));
            });
        }
        cp_async_commit();
    };
    // psi of slab s from its staged populations
    auto psi_slab = [&](int s) {
        Real* dst = ring + ring_slot(s, NS) * E;
        const Real* fi = stI + ring_slot(s, NI) * Q * NT + tid;
        Real sum = Real(0);
        sfor<Q>([&](auto bI) { sum += fi[decltype(bI)::value * NT]; });
        const Real rho = Real(p.rho_bar) + sum;
        dst[i_slot] = psi_of<LAT>(rho, p);
        if (has_halo) {
            const Real* fh = stH + (s & 1) * Q * H + tid;
            Real sh = Real(0);
            sfor<Q>([&](auto bI) { sh += fh[decltype(bI)::value * H]; });
            dst[h_slot] = psi_of<LAT>(Real(p.rho_bar) + sh, p);
        }
    };

    for (int s = m0 - R; s < m0 + R; ++s) {
        stage(s);
        cp_async_wait<0>();
        psi_slab(s);
    }
    stage(m0 + R);  // psi of slab m + R is formed at iteration m from data staged one iteration earlier
    const bool active = ix < p.nx && (D == 2 || iy < p.ny);
    const int cell_xy = (D == 3) ? iy * p.nx + ix : ix;
    for (int m = m0; m < m1; ++m) {
        const bool more = m + R + 1 < m1 + R;  // the next psi slab exists
        if (more) stage(m + R + 1);
        if (more)
            cp_async_wait<1>();
        else
            cp_async_wait<0>();
        psi_slab(m + R);
        __syncthreads();
        if (active) {
            Real f[Q];
            const Real* fi = stI + ring_slot(m, NI) * Q * NT + tid;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                f[b] = fi[b * NT];
            });
            Real F[3];
            force_ring<LAT, ORD, Real, EX, E, NS>(ring, m, tx + R, (D == 3) ? ty + R : 0, par<Real>(p.G, p.G_f), F);
            collide<LAT, COLL>(f, F, p);
            const int c = m * mscale + cell_xy;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                P.out[b][c] = f[b];
            });
        }
    }
    cp_async_wait<0>();
}

// Extended-tile position of halo cell h (the ring around a TX x TY tile).
template <int D, int R, int TX, int EX, int EY>
__device__ __forceinline__ void halo_pos(int h, int& hex, int& hey)
{
    if (D == 3) {
        if (h < R * EX) {
            hex = h % EX; hey = h / EX;
        } else if (h < 2 * R * EX) {
            hex = (h - R * EX) % EX; hey = EY - R + (h - R * EX) / EX;
        } else {
            const int g = h - 2 * R * EX;
            const int k = g % (2 * R);
            hey = R + g / (2 * R);
            hex = (k < R) ? k : TX + k;
        }
    } else {
        hey = 0;
        hex = (h < R) ? h : TX + h;
    }
}

// One-pass schedule with lookahead: iteration m first issues the loads of slab
// m + R + 1, then collides slab m (its psi slabs were completed before the last
// barrier), and only then forms psi of slab m + R + 1 from the loaded values, so
// the load latency overlaps the collision.  Interior populations wait in a
// shared-memory stash of R + 2 slabs; the psi ring has 2R + 2 slots.
// HL = 1: the halo cells' loads also run ahead; HL = 0: only the interior ones
// (fewer registers), the halo is gathered after the collision.
template <int LAT, int ORD, int COLL, class Real, int TX, int TY, int ZC, int MINB, int HL>
__global__ void __launch_bounds__(TX * TY, MINB)
    k_onepass_la(const __grid_constant__ Pops<Real, Lattice<LAT>::Q> P, DevParams p, int ntx, int nty)
{
    using L = Lattice<LAT>;
    using S = Stencil<L::D, ORD>;
    constexpr int D = L::D;
    constexpr int R = S::radius;
    constexpr int RE = L::reach;
    constexpr int Q = L::Q;
    constexpr int NT = TX * TY;
    constexpr int EX = TX + 2 * R;
    constexpr int EY = (D == 3) ? TY + 2 * R : 1;
    constexpr int E = EX * EY;
    constexpr int H = E - NT;
    constexpr int NS = 2 * R + 2;
    constexpr int NST = R + 2;
    static_assert(H <= NT, "halo larger than the block");
    __shared__ Real ring[NS * E];
    extern __shared__ unsigned char dyn_smem[];
    Real* stash = reinterpret_cast<Real*>(dyn_smem);  // [NST][Q][NT]

    const int ncol = ntx * nty;
    const int col = blockIdx.x % ncol;
    const int chunk = blockIdx.x / ncol;
    const int x0 = (col % ntx) * TX;
    const int y0 = (D == 3) ? (col / ntx) * TY : 0;
    const int nm = (D == 3) ? p.nz : p.ny;
    const int m0 = chunk * ZC;
    const int m1 = (m0 + ZC < nm) ? m0 + ZC : nm;
    const int mscale = (D == 3) ? p.nx * p.ny : p.nx;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;

    const int ix = x0 + tx, iy = y0 + ty;
    int ixo[2 * RE + 1], iyo[2 * RE + 1];
    axis_offsets<RE>(wrap_any(ix, p.nx), p.nx, 1, ixo);
    if (D == 3) axis_offsets<RE>(wrap_any(iy, p.ny), p.ny, p.nx, iyo);
    const int i_slot = (D == 3 ? (ty + R) * EX : 0) + tx + R;
    const bool has_halo = tid < H;
    int hex, hey;
    halo_pos<D, R, TX, EX, EY>(has_halo ? tid : 0, hex, hey);
    int hxo[2 * RE + 1], hyo[2 * RE + 1];
    axis_offsets<RE>(wrap_any(x0 - R + hex, p.nx), p.nx, 1, hxo);
    if (D == 3) axis_offsets<RE>(wrap_any(y0 - R + hey, p.ny), p.ny, p.nx, hyo);
    const int h_slot = hey * EX + hex;
    const int zero[2 * RE + 1] = {};

    Real fl[Q], hl[Q];
    auto load_halo = [&](int m) {
        int mo[2 * RE + 1];
        axis_offsets<RE>(wrap_near(m, nm), nm, mscale, mo);
        if (D == 3) {
            if (has_halo) gather_off<LAT, Real, RE>(P, hxo, hyo, mo, hl);
        } else {
            if (has_halo) gather_off<LAT, Real, RE>(P, hxo, mo, zero, hl);
        }
    };
    auto load_slab = [&](int m) {
        int mo[2 * RE + 1];
        axis_offsets<RE>(wrap_near(m, nm), nm, mscale, mo);
        if (D == 3)
            gather_off<LAT, Real, RE>(P, ixo, iyo, mo, fl);
        else
            gather_off<LAT, Real, RE>(P, ixo, mo, zero, fl);
        if (HL) load_halo(m);
    };
    auto finish_slab = [&](int m) {
        if (!HL) load_halo(m);
        Real* dst = ring + ring_slot(m, NS) * E;
        Real sum = Real(0);
        sfor<Q>([&](auto bI) { sum += fl[decltype(bI)::value]; });
        dst[i_slot] = psi_of<LAT>(std::is_same<Real, float>::value ? Real(p.rho_bar) + sum : sum, p);
        Real* st = stash + ring_slot(m, NST) * (Q * NT) + tid;
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            st[b * NT] = fl[b];
        });
        if (has_halo) {
            Real sh = Real(0);
            sfor<Q>([&](auto bI) { sh += hl[decltype(bI)::value]; });
            dst[h_slot] = psi_of<LAT>(std::is_same<Real, float>::value ? Real(p.rho_bar) + sh : sh, p);
        }
    };

    for (int m = m0 - R; m <= m0 + R; ++m) {
        load_slab(m);
        finish_slab(m);
    }
    __syncthreads();
    const bool active = ix < p.nx && (D == 2 || iy < p.ny);
    const int cell_xy = (D == 3) ? iy * p.nx + ix : ix;
    for (int m = m0; m < m1; ++m) {
        const bool ahead = m + 1 < m1;  // psi of slab m + R + 1 is needed
        if (ahead) load_slab(m + R + 1);
        if (active) {
            Real f[Q];
            const Real* st = stash + ring_slot(m, NST) * (Q * NT) + tid;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                f[b] = st[b * NT];
            });
            Real F[3];
            force_ring<LAT, ORD, Real, EX, E, NS>(ring, m, tx + R, (D == 3) ? ty + R : 0, par<Real>(p.G, p.G_f), F);
            collide<LAT, COLL>(f, F, p);
            const int c = m * mscale + cell_xy;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                P.out[b][c] = f[b];
            });
        }
        if (ahead) finish_slab(m + R + 1);
        __syncthreads();
    }
}

// ---- one-pass schedule, two cells per thread, packed FP32 ---------------------
// FP32 BGK only.  A thread owns the x-adjacent cells (x, x+1), x even, so the
// directions with c_x = 0 are gathered with one 8-byte load and every store is
// one 8-byte store (longer DRAM row segments: a warp covers 64 cells), and all
// per-cell arithmetic runs on float2 pairs with the packed FP32 instructions
// (__ffma2_rn / __fadd2_rn / __fmul2_rn).  Needs an even nx.
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, p2(-1.f), a); }

// c . v for a compile-time integer vector c (components in -3..3)
template <int CX, int CY, int CZ>
__device__ __forceinline__ float2 cdot2(float2 vx, float2 vy, float2 vz)
{
    float2 r = p2(0.f);
    bool any = false;
    auto acc = [&](int c, float2 v) {
        if (c == 0) return;
        if (!any) {
            r = (c == 1) ? v : mul2(p2(float(c)), v);
            any = true;
        } else if (c == 1) {
            r = add2(r, v);
        } else if (c == -1) {
            r = sub2(r, v);
        } else {
            r = fma2(p2(float(c)), v, r);
        }
    };
    acc(CX, vx);
    acc(CY, vy);
    acc(CZ, vz);
    return r;
}

// Packed-pair collision: BGK (COLL = 0) or MRT (COLL = 1, the BGK update plus
// the moment-space correction of mrt_moments_g / mrt_apply), both Guo-forced.
template <int LAT, int COLL = 0>
__device__ __forceinline__ void collide2(float2 (&f)[Lattice<LAT>::Q], const float2 (&F)[3], const DevParams& p)
{
    static_assert(COLL == 0 || COLL == 1, "packed pairs: BGK or MRT");
    using L = Lattice<LAT>;
    constexpr int Q = L::Q;
    constexpr int NP = (Q - 1) / 2;
    float2 s = f[0], jx = p2(0.f), jy = p2(0.f), jz = p2(0.f);
    float2 Pp[NP], Dp[NP];
    sfor<NP>([&](auto kI) {
        constexpr int k = decltype(kI)::value;
        constexpr int b = 1 + 2 * k;
        constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
        Pp[k] = add2(f[b], f[b + 1]);
        s = add2(s, Pp[k]);
        const float2 d = sub2(f[b], f[b + 1]);
        Dp[k] = d;
        if (cx == 1) jx = add2(jx, d); else if (cx == -1) jx = sub2(jx, d); else if (cx != 0) jx = fma2(p2(float(cx)), d, jx);
        if (cy == 1) jy = add2(jy, d); else if (cy == -1) jy = sub2(jy, d); else if (cy != 0) jy = fma2(p2(float(cy)), d, jy);
        if (cz == 1) jz = add2(jz, d); else if (cz == -1) jz = sub2(jz, d); else if (cz != 0) jz = fma2(p2(float(cz)), d, jz);
    });
    const float2 rho = add2(p2(p.rho_bar_f), s);
    const float2 inv_rho = make_float2(1.f / rho.x, 1.f / rho.y);
    const float2 ux = mul2(fma2(p2(0.5f), F[0], jx), inv_rho);
    const float2 uy = mul2(fma2(p2(0.5f), F[1], jy), inv_rho);
    const float2 uz = mul2(fma2(p2(0.5f), F[2], jz), inv_rho);
    constexpr double cs2 = L::cs2;
    constexpr bool k3 = L::D == 3;  // 2-D: no z terms (u_z = F_z = 0)
    float2 t[Q];
    if constexpr (COLL == 1) {
        const float2 jv[3] = {jx, jy, jz};
        const float2 uv3[3] = {ux, uy, uz};
        const float2 vv[3] = {fma2(p2(-0.5f), F[0], jx), fma2(p2(-0.5f), F[1], jy), fma2(p2(-0.5f), F[2], jz)};
        const float2 dm[4] = {p2(p.dmrt_f[0]), p2(p.dmrt_f[1]), p2(p.dmrt_f[2]), p2(p.dmrt_f[3])};
        mrt_moments_g<LAT, float2>(f[0], Pp, Dp, s, jv, uv3, vv, dm, t);
    }
    const float2 usq = k3 ? mul2(fma2(ux, ux, fma2(uy, uy, mul2(uz, uz))), p2(float(0.5 / cs2)))
                          : mul2(fma2(ux, ux, mul2(uy, uy)), p2(float(0.5 / cs2)));
    const float2 uF = k3 ? fma2(ux, F[0], fma2(uy, F[1], mul2(uz, F[2]))) : fma2(ux, F[0], mul2(uy, F[1]));
    const float2 omega = p2(p.omega_f);
    const float2 pref = p2(p.pref_f);
    const float2 orho = mul2(omega, rho);
    // A0 = omega s - omega rho usq - pref uF / cs2
    const float2 A0 = fma2(mul2(pref, p2(float(-1.0 / cs2))), uF, fma2(orho, sub2(p2(0.f), usq), mul2(omega, s)));
    const float2 ic2 = p2(float(1.0 / cs2)), ic4 = p2(float(1.0 / (cs2 * cs2)));
    const float2 Px = mul2(fma2(orho, ux, mul2(pref, F[0])), ic2);
    const float2 Py = mul2(fma2(orho, uy, mul2(pref, F[1])), ic2);
    const float2 Pz = mul2(fma2(orho, uz, mul2(pref, F[2])), ic2);
    const float2 h = mul2(p2(0.5f), orho);
    const float2 Vx = mul2(fma2(h, ux, mul2(pref, F[0])), ic4);
    const float2 Vy = mul2(fma2(h, uy, mul2(pref, F[1])), ic4);
    const float2 Vz = mul2(fma2(h, uz, mul2(pref, F[2])), ic4);
    const float2 om1 = p2(p.om1_f);
    {
        constexpr double w0 = L::T.w[0];
        f[0] = fma2(f[0], om1, mul2(p2(float(w0)), A0));
    }
    sfor<NP>([&](auto kI) {
        constexpr int b = 1 + 2 * decltype(kI)::value;
        constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
        constexpr double wb = L::T.w[b];
        const float2 cu = cdot2<cx, cy, cz>(ux, uy, uz);
        const float2 cV = cdot2<cx, cy, cz>(Vx, Vy, Vz);
        const float2 cP = cdot2<cx, cy, cz>(Px, Py, Pz);
        const float2 ev = fma2(cu, cV, A0);
        f[b] = fma2(f[b], om1, mul2(p2(float(wb)), add2(ev, cP)));
        f[b + 1] = fma2(f[b + 1], om1, mul2(p2(float(wb)), sub2(ev, cP)));
    });
    if constexpr (COLL == 1) mrt_apply<LAT, float2>(t, f);
}

// Packed-pair form of the persistent whole-row schedule (FP32 BGK): a compute
// thread owns the x-adjacent cells (2t, 2t + 1) of one row, so the directions
// with c_x = 0 come from shared memory as one 8-byte load per pair, the force and
// collision run on float2 pairs with the packed FP32 instructions, and every
// store is one 8-byte store.  Staging, item walk and producer are those of
// k_onepass_rowp.  PRODW = false drops the dedicated producer warp: the last
// compute warp issues the stage copies right after each barrier and then
// computes.  With 12 compute warps that keeps three warps per SM sub-partition
// (a 13th warp would cap every thread at 128 registers).
template <int LAT, int ORD, int COLL, int NX, int TY, int NSTG, bool PRODW = true, int NXMAX = NX>
__global__ void __launch_bounds__((NXMAX / 2 * TY + 31) / 32 * 32 + (PRODW ? 32 : 0), 1)
    k_onepass_rowp2(const __grid_constant__ Pops<float, Lattice<LAT>::Q> P, DevParams p, int zc, int nitems)
{
    using L = Lattice<LAT>;
    using S = Stencil<3, ORD>;
    constexpr int R = S::radius;
    constexpr int Q = L::Q;
    static_assert(L::D == 3 && R == 1 && L::reach == 1, "row staging is written for 3-D radius-1 stencils");
    // NX > 0: rows of NX cells (compile time); NX = 0: the domain's own row
    // length p.nx (<= NXMAX, a multiple of 4), and the compute threads are
    // rounded up to whole warps, the lanes past the last row pair idle.
    constexpr int EY = TY + 2 * R;
    constexpr int NS = 2 * R + 2;
    static_assert(NX > 0 ? (NX / 2 * TY) % 32 == 0 && NX / 2 * TY + 32 <= 1024 && NX % 4 == 0
                         : (NXMAX / 2 * TY + 31) / 32 * 32 + 32 <= 1024 && NXMAX % 4 == 0,
                  "block shape");
    static_assert(NSTG >= 2 * R && NSTG <= 32, "stages");
    const int nx = NX > 0 ? NX : p.nx;
    const int half = nx / 2;
    const int NT = NX > 0 ? NX / 2 * TY : (half * TY + 31) / 32 * 32;  // compute threads, whole warps
    const int EX = nx + 2 * R;
    const int E = EX * EY;
    const int STG = Q * EY * nx;
    __shared__ float ring_s[NX > 0 ? NS * (NX + 2 * R) * EY : 1];
    __shared__ alignas(8) unsigned long long bars[NSTG];
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    float* stage = reinterpret_cast<float*>(dyn_smem);  // [NSTG][STG]
    float* ring = NX > 0 ? ring_s : stage + NSTG * STG;  // [NS][E]

    const int nty = (p.ny + TY - 1) / TY;
    const int nm = p.nz;
    const int plane = nx * p.ny;
    const int tid = threadIdx.x;
    const int tp = tid % half, ty = tid / half;  // pair index along x, row in the tile (ty >= TY: idle lane)
    const int x0 = 2 * tp;                               // first cell of the pair
    const int lane = tid & 31;
    const bool producer = PRODW && tid >= NT;
    // the warp that issues the stage copies: the producer warp, else the last compute warp
    const bool issuer = PRODW ? producer : (tid / 32 == NT / 32 - 1);

    if (tid == 0) {
        for (int k = 0; k < NSTG; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
    }
    __syncthreads();

    int cby = 0, cbz = 0;
    const float* src_b = nullptr;
    sfor<Q>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        constexpr int vy = L::T.v[b][1], vz = L::T.v[b][2];
        if (lane == b) {
            cby = vy;
            cbz = vz;
            src_b = P.in[b];
        }
    });
    int p_it = blockIdx.x, p_y0 = 0, p_next = 0, p_last = -1;
    auto p_load_item = [&]() {
        if (p_it >= nitems) return;
        const int m0 = (p_it / nty) * zc;
        const int m1 = (m0 + zc < nm) ? m0 + zc : nm;
        p_y0 = (p_it % nty) * TY;
        p_next = m0 - R;
        p_last = m1 - 1 + R;
    };
    p_load_item();
    long long issued = 0;
    auto issue_next = [&]() {
        const int slot = static_cast<int>(issued % NSTG);
        const uint32_t bar = smem_u32(&bars[slot]);
        if (lane == 0) mbar_expect_tx(bar, static_cast<uint32_t>(STG * sizeof(float)));
        __syncwarp();
        if (lane < Q) {
            fence_proxy_async_smem();
            const float* pl = src_b + static_cast<long long>(wrap_any(p_next - cbz, nm)) * plane;
            uint32_t dst = smem_u32(stage + slot * STG + lane * (EY * nx));
            int y = p_y0 - R - cby, left = EY;
            while (left > 0) {
                const int yw = wrap_any(y, p.ny);
                const int n = (p.ny - yw < left) ? p.ny - yw : left;
                bulk_g2s(dst, pl + static_cast<long long>(yw) * nx, static_cast<uint32_t>(n * nx * sizeof(float)), bar);
                dst += static_cast<uint32_t>(n * nx * sizeof(float));
                y += n;
                left -= n;
            }
        }
        __syncwarp();
        ++issued;
        if (++p_next > p_last) {
            p_it += gridDim.x;
            p_load_item();
        }
    };
    auto issue_upto = [&](long long consumed) {
        while (p_it < nitems && issued < consumed + NSTG) issue_next();
    };

    uint32_t phase = 0;
    bool ok = true;
    long long consumed = 0;
    auto wait_seq = [&](long long q) -> const float* {
        const int slot = static_cast<int>(q % NSTG);
        if (ok && !mbar_wait(smem_u32(&bars[slot]), (phase >> slot) & 1u)) ok = false;  // after a timeout, stop waiting
        phase ^= 1u << slot;
        return stage + slot * STG;
    };
    // pull columns of the pair for c_x = +1 (x - 1) and c_x = -1 (x + 1), periodic
    const int xl = (x0 == 0) ? nx - 1 : x0 - 1;        // left of the first cell
    const int xr = (x0 + 2 == nx) ? 0 : x0 + 2;        // right of the second cell
    auto load_pair = [&](const float* st, int fy, float2 (&f)[Q]) {
        const float* r = st + fy * nx;
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int vx = L::T.v[b][0];
            const float* rb = r + b * (EY * nx);
            if (vx == 0)
                f[b] = *reinterpret_cast<const float2*>(rb + x0);
            else if (vx > 0)
                f[b] = make_float2(rb[xl], rb[x0]);
            else
                f[b] = make_float2(rb[x0 + 1], rb[xr]);
        });
    };
    auto rho_psi2 = [&](const float2 (&f)[Q]) {
        float2 sum = p2(0.f);
        sfor<Q>([&](auto bI) { sum = add2(sum, f[decltype(bI)::value]); });
        const float rb = static_cast<float>(p.rho_bar);
        return make_float2(psi_of<LAT>(rb + sum.x, p), psi_of<LAT>(rb + sum.y, p));
    };
    float2 fcur[Q], fnxt[Q];
    auto put_psi2 = [&](float* dst, int fy, float2 v) {
        float* row = dst + fy * EX;
        row[x0 + R] = v.x;
        row[x0 + 1 + R] = v.y;
        if (x0 == 0) row[nx + R] = v.x;          // wrapped column right of the row
        if (x0 + 2 == nx) row[0] = v.y;          // wrapped column left of the row
    };
    auto psi_slab = [&](int s, long long q) {
        const float* st = wait_seq(q);
        if (NX == 0 && ty >= TY) return;  // idle lane: keeps the barrier phases only
        float* dst = ring + ring_slot(s, NS) * E;
        load_pair(st, ty + R, fnxt);
        put_psi2(dst, ty + R, rho_psi2(fnxt));
        for (int k = ty; k < 2 * R; k += TY) {
            const int fy = (k < R) ? k : EY - 2 * R + k;
            float2 f[Q];
            load_pair(st, fy, f);
            put_psi2(dst, fy, rho_psi2(f));
        }
    };

    if (issuer) issue_upto(0);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int y0 = (it % nty) * TY;
        const int m0 = (it / nty) * zc;
        const int m1 = (m0 + zc < nm) ? m0 + zc : nm;
        if (!producer)
            for (int s = m0 - R; s < m0 + R; ++s) psi_slab(s, consumed + (s - (m0 - R)));
        consumed += 2 * R;
#pragma unroll
        for (int b = 0; b < Q; ++b) fcur[b] = fnxt[b];
        __syncthreads();
        if (issuer) issue_upto(consumed);
        const bool active = !producer && ty < TY && (y0 + ty) < p.ny;
        const int cell_xy = (y0 + ty) * nx + x0;
        for (int m = m0; m < m1; ++m) {
            if (!producer) psi_slab(m + R, consumed);
            ++consumed;
            __syncthreads();
            if (issuer) issue_upto(consumed);
            if (active) {
                // force (Eq. 1) of both cells from the psi ring, opposite vectors paired
                const float* base[2 * R + 1];
#pragma unroll
                for (int k = 0; k < 2 * R + 1; ++k) base[k] = ring + ring_slot(m - R + k, NS) * E + (ty + R) * EX + x0 + R;
                float2 ax = p2(0.f), ay = p2(0.f), az = p2(0.f);
                sfor<S::n / 2>([&](auto kI) {
                    constexpr int a = 2 * decltype(kI)::value;
                    constexpr int ex = S::T.v[a][0], ey = S::T.v[a][1], ez = S::T.v[a][2];
                    constexpr double wt = S::T.w[a] * L::cs2;
                    const float* pp = base[ez + R] + ey * EX + ex;
                    const float* pm = base[R - ez] - ey * EX - ex;
                    const float2 d = sub2(make_float2(pp[0], pp[1]), make_float2(pm[0], pm[1]));
                    if (ex != 0) ax = fma2(p2(float(wt * ex)), d, ax);
                    if (ey != 0) ay = fma2(p2(float(wt * ey)), d, ay);
                    if (ez != 0) az = fma2(p2(float(wt * ez)), d, az);
                });
                const float2 gp = mul2(p2(-p.G_f), make_float2(base[R][0], base[R][1]));
                const float2 F[3] = {mul2(gp, ax), mul2(gp, ay), mul2(gp, az)};
                collide2<LAT, COLL>(fcur, F, p);
                const int c = m * plane + cell_xy;
                sfor<Q>([&](auto bI) {
                    constexpr int b = decltype(bI)::value;
                    __stcs(reinterpret_cast<float2*>(P.out[b] + c), fcur[b]);
                });
            }
#pragma unroll
            for (int b = 0; b < Q; ++b) fcur[b] = fnxt[b];
        }
        __syncthreads();
    }
    if (!ok && tid == 0) atomicOr(p.err, kErrTimeout);
}

// Whole-row packed-pair schedule for stencils of radius R >= 2 (D3Q19 with the
// 6th-order stencil): the staging, item walk and packed collision of
// k_onepass_rowp2, with the row length read at run time (nx <= NXMAX, a
// multiple of 4).  At radius 2 a slab's stage holds TY + 4 rows per direction,
// so a 256-cell row allows only few stages; with NSTG = 1 the copy of slab
// m + R + 1 starts right after every thread has formed psi of slab m + R and
// overlaps the force and collision of slab m.  Because fewer than 2R stages
// may exist, the 2R warm-up slabs of an item are consumed one at a time, each
// followed by a barrier after which the issuing warp refills the stage.  The
// interior populations wait R slabs in a register delay line (d0 collides
// next, d1 one slab later).  The psi ring keeps R wrapped columns on each side.
template <int LAT, int ORD, int COLL, int TY, int NSTG, bool PRODW, int NXMAX>
__global__ void __launch_bounds__((NXMAX / 2 * TY + 31) / 32 * 32 + (PRODW ? 32 : 0), 1)
    k_onepass_rowr(const __grid_constant__ Pops<float, Lattice<LAT>::Q> P, DevParams p, int zc, int nitems)
{
    using L = Lattice<LAT>;
    using S = Stencil<3, ORD>;
    constexpr int R = S::radius;
    constexpr int Q = L::Q;
    static_assert(L::D == 3 && R == 2 && L::reach == 1, "radius-2 row staging for 3-D reach-1 lattices");
    constexpr int EY = TY + 2 * R;
    constexpr int NS = 2 * R + 2;
    static_assert((NXMAX / 2 * TY + 31) / 32 * 32 + 32 <= 1024 && NXMAX % 4 == 0, "block shape");
    static_assert(NSTG >= 1 && NSTG <= 32, "stages");
    const int nx = p.nx;
    const int half = nx / 2;
    const int NT = (half * TY + 31) / 32 * 32;  // compute threads, whole warps
    const int EX = nx + 2 * R;
    const int E = EX * EY;
    const int STG = Q * EY * nx;
    __shared__ alignas(8) unsigned long long bars[NSTG];
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    float* stage = reinterpret_cast<float*>(dyn_smem);  // [NSTG][STG]
    float* ring = stage + NSTG * STG;                    // [NS][E]

    const int nty = (p.ny + TY - 1) / TY;
    const int nm = p.nz;
    const int plane = nx * p.ny;
    const int tid = threadIdx.x;
    const int tp = tid % half, ty = tid / half;  // pair index along x, row in the tile (ty >= TY: idle lane)
    const int x0 = 2 * tp;
    const int lane = tid & 31;
    const bool producer = PRODW && tid >= NT;
    const bool issuer = PRODW ? producer : (tid / 32 == NT / 32 - 1);

    if (tid == 0) {
        for (int k = 0; k < NSTG; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
    }
    __syncthreads();

    int cby = 0, cbz = 0;
    const float* src_b = nullptr;
    sfor<Q>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        constexpr int vy = L::T.v[b][1], vz = L::T.v[b][2];
        if (lane == b) {
            cby = vy;
            cbz = vz;
            src_b = P.in[b];
        }
    });
    // the copy sequence: for every item of this block, slabs m0 - R .. m1 - 1 + R
    int p_it = blockIdx.x, p_y0 = 0, p_next = 0, p_last = -1;
    auto p_load_item = [&]() {
        if (p_it >= nitems) return;
        const int m0 = (p_it / nty) * zc;
        const int m1 = (m0 + zc < nm) ? m0 + zc : nm;
        p_y0 = (p_it % nty) * TY;
        p_next = m0 - R;
        p_last = m1 - 1 + R;
    };
    p_load_item();
    long long issued = 0;
    auto issue_next = [&]() {
        const int slot = static_cast<int>(issued % NSTG);
        const uint32_t bar = smem_u32(&bars[slot]);
        if (lane == 0) mbar_expect_tx(bar, static_cast<uint32_t>(STG * sizeof(float)));
        __syncwarp();
        if (lane < Q) {
            fence_proxy_async_smem();
            const float* pl = src_b + static_cast<long long>(wrap_any(p_next - cbz, nm)) * plane;
            uint32_t dst = smem_u32(stage + slot * STG + lane * (EY * nx));
            int y = p_y0 - R - cby, left = EY;
            while (left > 0) {
                const int yw = wrap_any(y, p.ny);
                const int n = (p.ny - yw < left) ? p.ny - yw : left;
                bulk_g2s(dst, pl + static_cast<long long>(yw) * nx, static_cast<uint32_t>(n * nx * sizeof(float)), bar);
                dst += static_cast<uint32_t>(n * nx * sizeof(float));
                y += n;
                left -= n;
            }
        }
        __syncwarp();
        ++issued;
        if (++p_next > p_last) {
            p_it += gridDim.x;
            p_load_item();
        }
    };
    auto issue_upto = [&](long long consumed) {
        while (p_it < nitems && issued < consumed + NSTG) issue_next();
    };

    uint32_t phase = 0;
    bool ok = true;
    long long consumed = 0;
    auto wait_seq = [&](long long q) -> const float* {
        const int slot = static_cast<int>(q % NSTG);
        if (ok && !mbar_wait(smem_u32(&bars[slot]), (phase >> slot) & 1u)) ok = false;  // after a timeout, stop waiting
        phase ^= 1u << slot;
        return stage + slot * STG;
    };
    const int xl = (x0 == 0) ? nx - 1 : x0 - 1;  // pull column of c_x = +1 for the first cell
    const int xr = (x0 + 2 == nx) ? 0 : x0 + 2;  // pull column of c_x = -1 for the second cell
    auto load_pair = [&](const float* st, int fy, float2 (&f)[Q]) {
        const float* r = st + fy * nx;
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int vx = L::T.v[b][0];
            const float* rb = r + b * (EY * nx);
            if (vx == 0)
                f[b] = *reinterpret_cast<const float2*>(rb + x0);
            else if (vx > 0)
                f[b] = make_float2(rb[xl], rb[x0]);
            else
                f[b] = make_float2(rb[x0 + 1], rb[xr]);
        });
    };
    auto rho_psi2 = [&](const float2 (&f)[Q]) {
        float2 sum = p2(0.f);
        sfor<Q>([&](auto bI) { sum = add2(sum, f[decltype(bI)::value]); });
        return make_float2(psi_of<LAT>(p.rho_bar_f + sum.x, p), psi_of<LAT>(p.rho_bar_f + sum.y, p));
    };
    // psi of the pair into ring row fy, and into the R wrapped columns on each side
    auto put_psi2 = [&](float* dst, int fy, float2 v) {
        float* row = dst + fy * EX;
        row[x0 + R] = v.x;
        row[x0 + 1 + R] = v.y;
        if (x0 < R) {
            row[x0 + nx + R] = v.x;
            if (x0 + 1 < R) row[x0 + 1 + nx + R] = v.y;
        }
        if (x0 + 1 >= nx - R) {
            row[x0 + 1 - nx + R] = v.y;
            if (x0 >= nx - R) row[x0 - nx + R] = v.x;
        }
    };
    float2 fnxt[Q], d0[Q], d1[Q];
    auto psi_slab = [&](int s, long long q) {
        const float* st = wait_seq(q);
        if (ty >= TY) return;  // idle lane: keeps the barrier phases only
        float* dst = ring + ring_slot(s, NS) * E;
        load_pair(st, ty + R, fnxt);
        put_psi2(dst, ty + R, rho_psi2(fnxt));
        for (int k = ty; k < 2 * R; k += TY) {
            const int fy = (k < R) ? k : EY - 2 * R + k;
            float2 f[Q];
            load_pair(st, fy, f);
            put_psi2(dst, fy, rho_psi2(f));
        }
    };
    auto shift = [&]() {
#pragma unroll
        for (int b = 0; b < Q; ++b) {
            d0[b] = d1[b];
            d1[b] = fnxt[b];
        }
    };

    if (issuer) issue_upto(0);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int y0 = (it % nty) * TY;
        const int m0 = (it / nty) * zc;
        const int m1 = (m0 + zc < nm) ? m0 + zc : nm;
        // warm-up: psi of slabs m0 - R .. m0 + R - 1, one slab per barrier
        for (int k = 0; k < 2 * R; ++k) {
            if (!producer) {
                psi_slab(m0 - R + k, consumed);
                shift();
            }
            ++consumed;
            __syncthreads();
            if (issuer) issue_upto(consumed);
        }
        const bool active = !producer && ty < TY && (y0 + ty) < p.ny;
        const int cell_xy = (y0 + ty) * nx + x0;
        for (int m = m0; m < m1; ++m) {
            if (!producer) psi_slab(m + R, consumed);
            ++consumed;
            __syncthreads();
            if (issuer) issue_upto(consumed);
            if (active) {
                // force (Eq. 1) of both cells from the psi ring, opposite vectors paired
                const float* base[2 * R + 1];
#pragma unroll
                for (int k = 0; k < 2 * R + 1; ++k) base[k] = ring + ring_slot(m - R + k, NS) * E + (ty + R) * EX + x0 + R;
                float2 ax = p2(0.f), ay = p2(0.f), az = p2(0.f);
                sfor<S::n / 2>([&](auto kI) {
                    constexpr int a = 2 * decltype(kI)::value;
                    constexpr int ex = S::T.v[a][0], ey = S::T.v[a][1], ez = S::T.v[a][2];
                    constexpr double wt = S::T.w[a] * L::cs2;
                    const float* pp = base[ez + R] + ey * EX + ex;
                    const float* pm = base[R - ez] - ey * EX - ex;
                    const float2 d = sub2(make_float2(pp[0], pp[1]), make_float2(pm[0], pm[1]));
                    if (ex != 0) ax = fma2(p2(float(wt * ex)), d, ax);
                    if (ey != 0) ay = fma2(p2(float(wt * ey)), d, ay);
                    if (ez != 0) az = fma2(p2(float(wt * ez)), d, az);
                });
                const float2 gp = mul2(p2(-p.G_f), make_float2(base[R][0], base[R][1]));
                const float2 F[3] = {mul2(gp, ax), mul2(gp, ay), mul2(gp, az)};
                collide2<LAT, COLL>(d0, F, p);
                const int c = m * plane + cell_xy;
                sfor<Q>([&](auto bI) {
                    constexpr int b = decltype(bI)::value;
                    __stcs(reinterpret_cast<float2*>(P.out[b] + c), d0[b]);
                });
            }
            if (!producer) shift();
        }
        __syncthreads();
    }
    if (!ok && tid == 0) atomicOr(p.err, kErrTimeout);
}

// ---- whole-row schedule with a carried density ------------------------------
// Position of direction b among the directions with (c_x, c_y) != 0, which
// cross between the threads of a slab; -1 for the rest.
template <int LAT>
__host__ __device__ constexpr int xchg_index(int b)
{
    using L = Lattice<LAT>;
    int k = 0;
    for (int j = 0; j < b; ++j)
        if (L::T.v[j][0] != 0 || L::T.v[j][1] != 0) ++k;
    return (L::T.v[b][0] != 0 || L::T.v[b][1] != 0) ? k : -1;
}
template <int LAT>
__host__ __device__ constexpr int xchg_count()
{
    return xchg_index<LAT>(Lattice<LAT>::Q - 1) + 1;
}

// Carried density of the next step (k_onepass_rowc).  The density deviation
// rho(x, t+1) - rho_bar = sum_i g_i(x - c_i) of the post-collision values of
// step t is written by step t itself, so that step t+1 finds the psi of the
// halo rows without staging their populations.  Rows are grouped TY at a time;
// a block sums the sources inside its group ("own", one value per cell) and
// writes what its first and last rows send across the group boundary into two
// frames:
//   own  [nz][ny][nx]
//   lo   [nty][nz][nx]: sent by group g to row y0(g) - 1 (the last row of g - 1)
//   hi   [nty][nz][nx]: sent by group g to row y0(g) + rows(g) (the first of g + 1)
// and the density of row y is own + hi[g(y) - 1] (if y is the first row of its
// group) + lo[g(y) + 1] (if it is the last), summed in that order, with the
// group indices periodic.  k_carry_init starts a carry from populations: own
// is the whole sum and both frames are zero.
struct CarryView {
    const float* own;
    const float* lo;
    const float* hi;
};
__host__ __device__ inline long long carry_floats(long long N, int nty, int nz, int nx)
{
    return N + 2LL * nty * nz * nx;
}

template <int LAT>
__global__ void __launch_bounds__(256)
    k_carry_init(const __grid_constant__ Pops<float, Lattice<LAT>::Q> P, DevParams p, float* __restrict__ c, int nty)
{
    using L = Lattice<LAT>;
    const long long nfr = 2LL * nty * p.nz * p.nx;
    const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < p.N + nfr; i += stride) {
        if (i >= p.N) {
            c[i] = 0.f;
            continue;
        }
        const int x = static_cast<int>(i % p.nx);
        const int y = static_cast<int>((i / p.nx) % p.ny);
        const int z = static_cast<int>(i / (static_cast<long long>(p.nx) * p.ny));
        float s = 0.f;
        sfor<L::Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int vx = L::T.v[b][0], vy = L::T.v[b][1], vz = L::T.v[b][2];
            const int xs = wrap_any(x - vx, p.nx);
            const int ys = wrap_any(y - vy, p.ny);
            const int zs = wrap_any(z - vz, p.nz);
            s += P.in[b][(static_cast<long long>(zs) * p.ny + ys) * p.nx + xs];
        });
        c[i] = s;
    }
}

// Whole-row packed-pair schedule with a carried density (FP32, 3-D lattices of
// reach 1, any stencil radius R).  Staging, item walk and packed collision are
// those of k_onepass_rowp2, with three changes:
// - psi of slab m + R comes from the carried density of the step before: the
//   own values plus the frames of the group-boundary rows, loaded one slab
//   ahead into registers.  A stage holds only the TY rows of the item per
//   direction, whatever R, so two or three stages fit;
// - the staged populations collide at once: no delay line;
// - the block also collides the slab before and the slab after its chunk
//   (m0 - 1 and m1, not stored), so every slab of the chunk receives all its
//   sources from this block and no frame crosses a chunk boundary.
// After the collision of slab m the pairs of the directions that cross between
// threads go to an exchange buffer; each thread then sums, per c_z, what its two
// cells receive from slab m (sources outside the group come through the frames),
// and a two-slab delay in registers completes the carried density of slab m - 1.
template <int LAT, int ORD, int COLL, int TY, int NSTG, int NXMAX>
__global__ void __launch_bounds__((NXMAX / 2 * TY + 31) / 32 * 32, 1)
    k_onepass_rowc(const __grid_constant__ Pops<float, Lattice<LAT>::Q> P, DevParams p, CarryView cin,
                   float* __restrict__ cout, int zc, int nitems)
{
    using L = Lattice<LAT>;
    using S = Stencil<3, ORD>;
    constexpr int R = S::radius;
    constexpr int Q = L::Q;
    constexpr int NXD = xchg_count<LAT>();
    static_assert(L::D == 3 && L::reach == 1, "row staging for 3-D reach-1 lattices");
    constexpr int EY = TY + 2 * R;          // psi rows of the ring
    constexpr int NS = 2 * R + 1;           // psi slabs of the ring
    constexpr int KR = (EY + TY - 1) / TY;  // psi rows per thread, at most
    static_assert((NXMAX / 2 * TY + 31) / 32 * 32 <= 1024 && NXMAX % 4 == 0, "block shape");
    static_assert(NSTG >= 1 && NSTG <= 32, "stages");
    const int nx = p.nx;
    const int half = nx / 2;
    const int NT = (half * TY + 31) / 32 * 32;  // threads, whole warps
    const int EX = nx + 2 * R;
    const int E = EX * EY;
    const int STG = Q * TY * nx;
    __shared__ alignas(8) unsigned long long bars[NSTG];
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    float* stage = reinterpret_cast<float*>(dyn_smem);  // [NSTG][Q][TY][nx]
    float* ring = stage + NSTG * STG;                    // [NS][EY][EX]
    float* xch = ring + NS * E;                          // [NXD][TY][nx]

    const int nty = (p.ny + TY - 1) / TY;
    const int nm = p.nz;
    const int plane = nx * p.ny;
    const long long fsz = static_cast<long long>(nm) * nx;  // one group's frame
    float* cout_lo = cout + p.N;
    float* cout_hi = cout_lo + nty * fsz;
    const int tid = threadIdx.x;
    const int tp = tid % half, ty = tid / half;  // pair along x, row in the group (ty >= TY: idle lane)
    const int x0 = 2 * tp;
    const int lane = tid & 31;
    const bool issuer = tid / 32 == NT / 32 - 1;

    if (tid == 0) {
        for (int k = 0; k < NSTG; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
    }
    __syncthreads();

    int cby = 0, cbz = 0;
    const float* src_b = nullptr;
    sfor<Q>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        constexpr int vy = L::T.v[b][1], vz = L::T.v[b][2];
        if (lane == b) {
            cby = vy;
            cbz = vz;
            src_b = P.in[b];
        }
    });
    // the copy sequence: for every item of this block, slabs m0 - 1 .. m1
    int p_it = blockIdx.x, p_y0 = 0, p_next = 0, p_last = -1;
    auto p_load_item = [&]() {
        if (p_it >= nitems) return;
        const int m0 = (p_it / nty) * zc;
        p_y0 = (p_it % nty) * TY;
        p_next = m0 - 1;
        p_last = (m0 + zc < nm) ? m0 + zc : nm;
    };
    p_load_item();
    long long issued = 0;
    auto issue_next = [&]() {
        const int slot = static_cast<int>(issued % NSTG);
        const uint32_t bar = smem_u32(&bars[slot]);
        if (lane == 0) mbar_expect_tx(bar, static_cast<uint32_t>(STG * sizeof(float)));
        __syncwarp();
        if (lane < Q) {
            fence_proxy_async_smem();
            const float* pl = src_b + static_cast<long long>(wrap_any(p_next - cbz, nm)) * plane;
            uint32_t dst = smem_u32(stage + slot * STG + lane * (TY * nx));
            int y = p_y0 - cby, left = TY;
            while (left > 0) {
                const int yw = wrap_any(y, p.ny);
                const int n = (p.ny - yw < left) ? p.ny - yw : left;
                bulk_g2s(dst, pl + static_cast<long long>(yw) * nx, static_cast<uint32_t>(n * nx * sizeof(float)), bar);
                dst += static_cast<uint32_t>(n * nx * sizeof(float));
                y += n;
                left -= n;
            }
        }
        __syncwarp();
        ++issued;
        if (++p_next > p_last) {
            p_it += gridDim.x;
            p_load_item();
        }
    };
    auto issue_upto = [&](long long consumed) {
        while (p_it < nitems && issued < consumed + NSTG) issue_next();
    };

    uint32_t phase = 0;
    bool ok = true;
    long long consumed = 0;
    auto wait_seq = [&](long long q) -> const float* {
        const int slot = static_cast<int>(q % NSTG);
        if (ok && !mbar_wait(smem_u32(&bars[slot]), (phase >> slot) & 1u)) ok = false;  // after a timeout, stop waiting
        phase ^= 1u << slot;
        return stage + slot * STG;
    };
    const int xl = (x0 == 0) ? nx - 1 : x0 - 1;  // column x - 1 of the first cell
    const int xr = (x0 + 2 == nx) ? 0 : x0 + 2;  // column x + 1 of the second cell
    // the pair's values of a row shifted by -c_x (the pull source of direction c_x)
    auto pull_row = [&](const float* r, int vx) -> float2 {
        if (vx == 0) return *reinterpret_cast<const float2*>(r + x0);
        if (vx > 0) return make_float2(r[xl], r[x0]);
        return make_float2(r[x0 + 1], r[xr]);
    };
    // the three parts (own, frame from the group before, frame from the group
    // after) of the carried density of grid row yr, slab z, for the pair
    auto carry_load = [&](int yr, int z, float2 (&v)[3]) {
        const int gr = yr / TY;
        const int first = gr * TY;
        const int last = ((first + TY < p.ny) ? first + TY : p.ny) - 1;
        const long long fz = static_cast<long long>(z) * nx + x0;
        v[0] = __ldg(reinterpret_cast<const float2*>(cin.own + static_cast<long long>(z) * plane + yr * nx + x0));
        v[1] = p2(0.f);
        v[2] = p2(0.f);
        if (yr == first) v[1] = __ldg(reinterpret_cast<const float2*>(cin.hi + (gr == 0 ? nty - 1 : gr - 1) * fsz + fz));
        if (yr == last) v[2] = __ldg(reinterpret_cast<const float2*>(cin.lo + (gr + 1 == nty ? 0 : gr + 1) * fsz + fz));
    };
    // carried densities of the thread's psi rows (ring rows ty, ty + TY, ...) of slab s
    auto psi_load = [&](int y0, int s, float2 (&v)[KR][3]) {
        const int z = wrap_any(s, nm);
#pragma unroll
        for (int j = 0; j < KR; ++j) {
            const int k = ty + j * TY;
            if (k < EY) carry_load(wrap_any(y0 - R + k, p.ny), z, v[j]);
        }
    };
    // psi of the pair into ring row fy, and into the R wrapped columns on each side
    auto put_psi2 = [&](float* dst, int fy, float2 v) {
        float* row = dst + fy * EX;
        row[x0 + R] = v.x;
        row[x0 + 1 + R] = v.y;
        if (x0 < R) {
            row[x0 + nx + R] = v.x;
            if (x0 + 1 < R) row[x0 + 1 + nx + R] = v.y;
        }
        if (x0 + 1 >= nx - R) {
            row[x0 + 1 - nx + R] = v.y;
            if (x0 >= nx - R) row[x0 - nx + R] = v.x;
        }
    };
    auto psi_put = [&](int s, const float2 (&v)[KR][3]) {
        float* dst = ring + ring_slot(s, NS) * E;
#pragma unroll
        for (int j = 0; j < KR; ++j) {
            const int k = ty + j * TY;
            if (k < EY) {
                const float2 r = add2(add2(v[j][0], v[j][1]), v[j][2]);
                put_psi2(dst, k, make_float2(psi_of<LAT>(p.rho_bar_f + r.x, p), psi_of<LAT>(p.rho_bar_f + r.y, p)));
            }
        }
    };

    float2 pre[KR][3];
    if (issuer) issue_upto(0);
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int g = it % nty;
        const int y0 = g * TY;
        const int rows = (y0 + TY < p.ny) ? TY : p.ny - y0;
        const int m0 = (it / nty) * zc;
        const int m1 = (m0 + zc < nm) ? m0 + zc : nm;
        const bool act = ty < rows;
        const bool top = ty == 0, bot = ty == rows - 1;
        // warm-up: psi of slabs m0 - 1 - R .. m0 - 2 + R into the ring, slab
        // m0 - 1 + R into the registers (all loads issued before the first use)
        if (ty < TY) {
            float2 w[2 * R][KR][3];
#pragma unroll
            for (int k = 0; k < 2 * R; ++k) psi_load(y0, m0 - 1 - R + k, w[k]);
            psi_load(y0, m0 - 1 + R, pre);
#pragma unroll
            for (int k = 0; k < 2 * R; ++k) psi_put(m0 - 1 - R + k, w[k]);
        }
        float2 A0 = p2(0.f), A1 = p2(0.f), U0 = p2(0.f), U1 = p2(0.f), V0 = p2(0.f), V1 = p2(0.f);
        const long long cell_xy = static_cast<long long>(y0 + ty) * nx + x0;
        for (int m = m0 - 1; m <= m1; ++m) {
            if (ty < TY) {
                psi_put(m + R, pre);
                if (m < m1) psi_load(y0, m + R + 1, pre);
            }
            const float* st = wait_seq(consumed);
            float2 f[Q];
            if (act) {
                const float* r = st + ty * nx;
                sfor<Q>([&](auto bI) {
                    constexpr int b = decltype(bI)::value;
                    constexpr int vx = L::T.v[b][0];
                    f[b] = pull_row(r + b * (TY * nx), vx);
                });
            }
            ++consumed;
            __syncthreads();  // psi of slab m + R in the ring; the stage slot is free
            if (issuer) issue_upto(consumed);
            if (act) {
                // force (Eq. 1) of both cells from the psi ring, opposite vectors paired
                const float* base[2 * R + 1];
#pragma unroll
                for (int k = 0; k < 2 * R + 1; ++k) base[k] = ring + ring_slot(m - R + k, NS) * E + (ty + R) * EX + x0 + R;
                float2 ax = p2(0.f), ay = p2(0.f), az = p2(0.f);
                sfor<S::n / 2>([&](auto kI) {
                    constexpr int a = 2 * decltype(kI)::value;
                    constexpr int ex = S::T.v[a][0], ey = S::T.v[a][1], ez = S::T.v[a][2];
                    constexpr double wt = S::T.w[a] * L::cs2;
                    const float* pp = base[ez + R] + ey * EX + ex;
                    const float* pm = base[R - ez] - ey * EX - ex;
                    const float2 d = sub2(make_float2(pp[0], pp[1]), make_float2(pm[0], pm[1]));
                    if (ex != 0) ax = fma2(p2(float(wt * ex)), d, ax);
                    if (ey != 0) ay = fma2(p2(float(wt * ey)), d, ay);
                    if (ez != 0) az = fma2(p2(float(wt * ez)), d, az);
                });
                const float2 gp = mul2(p2(-p.G_f), make_float2(base[R][0], base[R][1]));
                const float2 F[3] = {mul2(gp, ax), mul2(gp, ay), mul2(gp, az)};
                collide2<LAT, COLL>(f, F, p);
                if (m >= m0 && m < m1) {
                    const long long c = static_cast<long long>(m) * plane + cell_xy;
                    sfor<Q>([&](auto bI) {
                        constexpr int b = decltype(bI)::value;
                        __stcs(reinterpret_cast<float2*>(P.out[b] + c), f[b]);
                    });
                }
                sfor<Q>([&](auto bI) {
                    constexpr int b = decltype(bI)::value;
                    constexpr int xi = xchg_index<LAT>(b);
                    if constexpr (xi >= 0) *reinterpret_cast<float2*>(xch + (xi * TY + ty) * nx + x0) = f[b];
                });
            }
            __syncthreads();  // the exchange buffer holds slab m
            if (act) {
                // what the pair receives from slab m, per c_z (T), and what rows
                // y0 - 1 (U) and y0 + rows (V) receive from the group's edge rows
                float2 T[3] = {p2(0.f), p2(0.f), p2(0.f)};
                float2 Uc[3] = {p2(0.f), p2(0.f), p2(0.f)};
                float2 Vc[3] = {p2(0.f), p2(0.f), p2(0.f)};
                sfor<Q>([&](auto bI) {
                    constexpr int b = decltype(bI)::value;
                    constexpr int vx = L::T.v[b][0], vy = L::T.v[b][1], vz = L::T.v[b][2];
                    constexpr int xi = xchg_index<LAT>(b);
                    if constexpr (xi < 0) {
                        T[vz + 1] = add2(T[vz + 1], f[b]);
                    } else {
                        const float* xb = xch + xi * TY * nx;
                        const int sy = ty - vy;
                        if (sy >= 0 && sy < rows) T[vz + 1] = add2(T[vz + 1], pull_row(xb + sy * nx, vx));
                        if (vy < 0 && top) Uc[vz + 1] = add2(Uc[vz + 1], pull_row(xb, vx));
                        if (vy > 0 && bot) Vc[vz + 1] = add2(Vc[vz + 1], pull_row(xb + (rows - 1) * nx, vx));
                    }
                });
                if (m - 1 >= m0 && m - 1 < m1) {  // slab m - 1 has received all its sources
                    const long long fo = static_cast<long long>(g) * fsz + static_cast<long long>(m - 1) * nx + x0;
                    *reinterpret_cast<float2*>(cout + static_cast<long long>(m - 1) * plane + cell_xy) = add2(A0, T[0]);
                    if (top) *reinterpret_cast<float2*>(cout_lo + fo) = add2(U0, Uc[0]);
                    if (bot) *reinterpret_cast<float2*>(cout_hi + fo) = add2(V0, Vc[0]);
                }
                A0 = add2(A1, T[1]);
                A1 = T[2];
                U0 = add2(U1, Uc[1]);
                U1 = Uc[2];
                V0 = add2(V1, Vc[1]);
                V1 = Vc[2];
            }
        }
    }
    if (!ok && tid == 0) atomicOr(p.err, kErrTimeout);
}

// Packed-pair form of the segment schedule k_onepass_seg (FP32 BGK, 2-D reach-1
// lattices): a compute thread owns the x-adjacent cells (2t, 2t + 1) of the
// tile, so the directions with c_x = 0 come from the staged segment as one
// 8-byte load per pair, psi, the force and the collision run on float2 pairs
// with the packed FP32 instructions, and every store is one 8-byte store.
// Staging, stage reuse and the producer warp are those of k_onepass_seg.
template <int LAT, int ORD, int COLL, int TX, int ZC, int NSTG>
__global__ void __launch_bounds__(TX / 2 + 32, 1)
    k_onepass_seg2(const __grid_constant__ Pops<float, Lattice<LAT>::Q> P, DevParams p, int ntx)
{
    using L = Lattice<LAT>;
    using S = Stencil<2, ORD>;
    constexpr int R = S::radius;
    constexpr int Q = L::Q;
    static_assert(L::D == 2 && L::reach == 1, "segment staging is written for 2-D reach-1 lattices");
    constexpr int NT = TX / 2;       // compute threads
    constexpr int XP = 4;            // 16 bytes of floats on each side of the tile
    static_assert(XP >= R + 1 && TX % XP == 0 && NT % 32 == 0, "x pad / tile");
    constexpr int W = TX + 2 * XP;   // staged segment length (even: the pairs stay 8-byte aligned)
    constexpr int EX = TX + 2 * R;   // psi ring row
    constexpr int NS = 2 * R + 2;
    constexpr int STG = Q * W;
    static_assert(NSTG >= R + 2 && NSTG >= 2 * R, "one row in flight; the 2R warm-up rows staged at once");
    __shared__ float ring[NS * EX];
    __shared__ alignas(8) unsigned long long bars[NSTG];
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    float* stage = reinterpret_cast<float*>(dyn_smem);  // [NSTG][Q][W]

    const int tile = blockIdx.x % ntx;
    const int chunk = blockIdx.x / ntx;
    const int x0 = tile * TX;
    const int nm = p.ny;
    const int m0 = chunk * ZC;
    const int m1 = (m0 + ZC < nm) ? m0 + ZC : nm;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const bool producer = tid >= NT;
    const int cx0 = 2 * tid;  // tile offset of the pair's first cell

    if (tid == 0) {
        for (int k = 0; k < NSTG; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
    }
    __syncthreads();

    int cby = 0;
    const float* src_b = nullptr;
    sfor<Q>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        constexpr int vy = L::T.v[b][1];
        if (lane == b) {
            cby = vy;
            src_b = P.in[b];
        }
    });
    const int base = m0 - R;
    auto issue = [&](int s) {
        const int slot = (s - base) % NSTG;
        const uint32_t bar = smem_u32(&bars[slot]);
        if (lane == 0) mbar_expect_tx(bar, static_cast<uint32_t>(STG * sizeof(float)));
        __syncwarp();
        if (lane < Q) {
            fence_proxy_async_smem();
            const float* row = src_b + static_cast<long long>(wrap_any(s - cby, nm)) * p.nx;
            uint32_t dst = smem_u32(stage + slot * STG + lane * W);
            int xs = x0 - XP, left = W;
            while (left > 0) {
                const int x = wrap_any(xs, p.nx);
                const int n = (p.nx - x < left) ? p.nx - x : left;
                bulk_g2s(dst, row + x, static_cast<uint32_t>(n * sizeof(float)), bar);
                dst += static_cast<uint32_t>(n * sizeof(float));
                xs += n;
                left -= n;
            }
        }
    };
    uint32_t phase = 0;
    bool ok = true;
    auto stage_of = [&](int s) { return stage + ((s - base) % NSTG) * STG; };
    auto wait_stage = [&](int s) {
        const int slot = (s - base) % NSTG;
        if (ok && !mbar_wait(smem_u32(&bars[slot]), (phase >> slot) & 1u)) ok = false;  // after a timeout, stop waiting
        phase ^= 1u << slot;
    };
    // f of the cell at tile offset cx (-R .. TX + R - 1) from stage st (pull)
    auto load_cell = [&](const float* st, int cx, float (&f)[Q]) {
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int vx = L::T.v[b][0];
            f[b] = st[b * W + cx + XP - vx];
        });
    };
    // f of the pair (cx0, cx0 + 1): c_x = 0 as one 8-byte load, shifted directions as two words
    auto load_pair = [&](const float* st, float2 (&f)[Q]) {
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int vx = L::T.v[b][0];
            const float* rb = st + b * W + XP + cx0;
            if (vx == 0)
                f[b] = *reinterpret_cast<const float2*>(rb);
            else
                f[b] = make_float2(rb[-vx], rb[1 - vx]);
        });
    };
    auto rho_psi = [&](const float (&f)[Q]) {
        float sum = 0.f;
        sfor<Q>([&](auto bI) { sum += f[decltype(bI)::value]; });
        return psi_of<LAT>(static_cast<float>(p.rho_bar) + sum, p);
    };
    auto psi_slab = [&](int s) {
        wait_stage(s);
        const float* st = stage_of(s);
        float* dst = ring + ring_slot(s, NS) * EX;
        float2 f[Q];
        load_pair(st, f);
        float2 sum = p2(0.f);
        sfor<Q>([&](auto bI) { sum = add2(sum, f[decltype(bI)::value]); });
        const float rb = static_cast<float>(p.rho_bar);
        dst[cx0 + R] = psi_of<LAT>(rb + sum.x, p);
        dst[cx0 + 1 + R] = psi_of<LAT>(rb + sum.y, p);
        if (tid < 2 * R) {
            const int cx = (tid < R) ? tid - R : TX + tid - R;
            float fs[Q];
            load_cell(st, cx, fs);
            dst[cx + R] = rho_psi(fs);
        }
    };

    int next = base;
    const int last = m1 - 1 + R;
    if (producer)
        for (; next <= last && next < base + NSTG; ++next) issue(next);
    if (!producer)
        for (int s = m0 - R; s < m0 + R; ++s) psi_slab(s);
    __syncthreads();
    // slabs below m0 are consumed (psi only): slab k may refill slab k - NSTG's stage
    if (producer)
        for (; next <= last && next < m0 + NSTG; ++next) issue(next);

    const bool active = !producer && (x0 + cx0) < p.nx;  // nx even: the pair's second cell is inside too
    for (int m = m0; m < m1; ++m) {
        if (!producer) psi_slab(m + R);
        __syncthreads();
        // every thread is past the collision of row m - 1
        if (producer)
            for (; next <= last && next <= m - 1 + NSTG; ++next) issue(next);
        if (active) {
            float2 f[Q];
            load_pair(stage_of(m), f);
            // force (Eq. 1) of both cells from the psi ring, opposite vectors paired
            const float* rowp[2 * R + 1];
#pragma unroll
            for (int k = 0; k < 2 * R + 1; ++k) rowp[k] = ring + ring_slot(m - R + k, NS) * EX + cx0 + R;
            float2 ax = p2(0.f), ay = p2(0.f);
            sfor<S::n / 2>([&](auto kI) {
                constexpr int a = 2 * decltype(kI)::value;
                constexpr int ex = S::T.v[a][0], ey = S::T.v[a][1];
                constexpr double wt = S::T.w[a] * L::cs2;
                const float* pp = rowp[ey + R] + ex;
                const float* pm = rowp[R - ey] - ex;
                const float2 d = sub2(make_float2(pp[0], pp[1]), make_float2(pm[0], pm[1]));
                if (ex != 0) ax = fma2(p2(float(wt * ex)), d, ax);
                if (ey != 0) ay = fma2(p2(float(wt * ey)), d, ay);
            });
            const float2 gp = mul2(p2(-p.G_f), make_float2(rowp[R][0], rowp[R][1]));
            const float2 F[3] = {mul2(gp, ax), mul2(gp, ay), p2(0.f)};
            collide2<LAT, COLL>(f, F, p);
            const int c = m * p.nx + x0 + cx0;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                __stcs(reinterpret_cast<float2*>(P.out[b] + c), f[b]);
            });
        }
    }
    if (!ok && tid == 0) atomicOr(p.err, kErrTimeout);
}

template <int LAT, int ORD, int TX2, int TY, int ZC, int MINB, int ST>
__global__ void __launch_bounds__(TX2 * TY, MINB)
    k_onepass_x2(const __grid_constant__ Pops<float, Lattice<LAT>::Q> P, DevParams p, int ntx, int nty)
{
    using L = Lattice<LAT>;
    using S = Stencil<L::D, ORD>;
    constexpr int D = L::D;
    constexpr int R = S::radius;
    constexpr int RE = L::reach;
    constexpr int Q = L::Q;
    constexpr int NT = TX2 * TY;
    constexpr int TX = 2 * TX2;
    constexpr int EX = TX + 2 * R;
    constexpr int EY = (D == 3) ? TY + 2 * R : 1;
    constexpr int E = EX * EY;
    constexpr int H = E - TX * TY;
    constexpr int NS = 2 * R + 2;
    constexpr int NST = R + 1;
    static_assert(H <= 2 * NT, "halo larger than two cells per thread");
    static_assert(ST == 2 || (ST == 1 && R == 1), "stash in shared memory, or registers for radius 1");
    __shared__ float ring[NS * E];
    extern __shared__ unsigned char dyn_smem[];
    float2* stash = reinterpret_cast<float2*>(dyn_smem);  // [NST][Q][NT] when ST == 2

    const int ncol = ntx * nty;
    const int col = blockIdx.x % ncol;
    const int chunk = blockIdx.x / ncol;
    const int x0 = (col % ntx) * TX;
    const int y0 = (D == 3) ? (col / ntx) * TY : 0;
    const int nm = (D == 3) ? p.nz : p.ny;
    const int m0 = chunk * ZC;
    const int m1 = (m0 + ZC < nm) ? m0 + ZC : nm;
    const int mscale = (D == 3) ? p.nx * p.ny : p.nx;
    const int tid = threadIdx.x;
    const int tx2 = tid % TX2, ty = tid / TX2;

    // interior pair (ix, ix + 1), ix even
    const int ix = x0 + 2 * tx2, iy = y0 + ty;
    const int ixw = wrap_any(ix, p.nx);
    int xa[2 * RE + 1], xb[2 * RE + 1], iyo[2 * RE + 1];
    axis_offsets<RE>(ixw, p.nx, 1, xa);
    axis_offsets<RE>(ixw + 1 < p.nx ? ixw + 1 : 0, p.nx, 1, xb);
    if (D == 3) axis_offsets<RE>(wrap_any(iy, p.ny), p.ny, p.nx, iyo);
    const int i_pos = (D == 3 ? (ty + R) * EX : 0) + 2 * tx2 + R;

    // up to two halo cells: h = tid and h = tid + NT
    int hx0[2 * RE + 1], hy0[2 * RE + 1], hx1[2 * RE + 1], hy1[2 * RE + 1];
    int hpos0 = 0, hpos1 = 0;
    const bool h0 = tid < H, h1 = tid + NT < H;
    {
        int ex, ey;
        halo_pos<D, R, TX, EX, EY>(h0 ? tid : 0, ex, ey);
        axis_offsets<RE>(wrap_any(x0 - R + ex, p.nx), p.nx, 1, hx0);
        if (D == 3) axis_offsets<RE>(wrap_any(y0 - R + ey, p.ny), p.ny, p.nx, hy0);
        hpos0 = ey * EX + ex;
        halo_pos<D, R, TX, EX, EY>(h1 ? tid + NT : 0, ex, ey);
        axis_offsets<RE>(wrap_any(x0 - R + ex, p.nx), p.nx, 1, hx1);
        if (D == 3) axis_offsets<RE>(wrap_any(y0 - R + ey, p.ny), p.ny, p.nx, hy1);
        hpos1 = ey * EX + ex;
    }
    const int zero[2 * RE + 1] = {};

    float2 fcur[Q], fnxt[Q];

    auto halo_psi = [&](const int (&hx)[2 * RE + 1], const int* yo, const int* zo, float* dst) {
        float sum = 0.f;
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
            sum += __ldg(P.in[b] + (zo[cz + RE] + yo[cy + RE] + hx[cx + RE]));
        });
        *dst = psi_exp(float(p.rho_bar) + sum);
    };

    auto psi_slab = [&](int m) {
        int mo[2 * RE + 1];
        axis_offsets<RE>(wrap_near(m, nm), nm, mscale, mo);
        const int* yi = (D == 3) ? iyo : mo;
        const int* zi = (D == 3) ? mo : zero;
        float* dst = ring + ring_slot(m, NS) * E;
        float2 sum = p2(0.f);
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
            const int base = zi[cz + RE] + yi[cy + RE];
            if (cx == 0) {
                fnxt[b] = __ldg(reinterpret_cast<const float2*>(P.in[b] + (base + xa[RE])));
            } else {
                fnxt[b] = make_float2(__ldg(P.in[b] + (base + xa[cx + RE])), __ldg(P.in[b] + (base + xb[cx + RE])));
            }
            sum = add2(sum, fnxt[b]);
        });
        const float2 rho = add2(p2(float(p.rho_bar)), sum);
        dst[i_pos] = psi_exp(rho.x);
        dst[i_pos + 1] = psi_exp(rho.y);
        if (ST == 2) {
            float2* st = stash + static_cast<unsigned>(m + 4 * NST) % NST * (Q * NT) + tid;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                st[b * NT] = fnxt[b];
            });
        }
        const int* yh0 = (D == 3) ? hy0 : mo;
        const int* yh1 = (D == 3) ? hy1 : mo;
        if (h0) halo_psi(hx0, yh0, zi, dst + hpos0);
        if (h1) halo_psi(hx1, yh1, zi, dst + hpos1);
    };

    for (int m = m0 - R; m < m0 + R; ++m) {
        psi_slab(m);
        if (ST == 1 && m == m0 + R - 1) {
#pragma unroll
            for (int b = 0; b < Q; ++b) fcur[b] = fnxt[b];
        }
    }
    const bool active = ix < p.nx && (D == 2 || iy < p.ny);
    const int cell_xy = (D == 3) ? iy * p.nx + ix : ix;
    for (int m = m0; m < m1; ++m) {
        psi_slab(m + R);
        __syncthreads();
        if (active) {
            if (ST == 2) {
                const float2* st = stash + static_cast<unsigned>(m + 4 * NST) % NST * (Q * NT) + tid;
                sfor<Q>([&](auto bI) {
                    constexpr int b = decltype(bI)::value;
                    fcur[b] = st[b * NT];
                });
            }
            // force (Eq. 1) of both cells from the psi ring, opposite vectors paired
            const float* base[2 * R + 1];
#pragma unroll
            for (int k = 0; k < 2 * R + 1; ++k) base[k] = ring + ring_slot(m - R + k, NS) * E + i_pos;
            float2 ax = p2(0.f), ay = p2(0.f), az = p2(0.f);
            sfor<S::n / 2>([&](auto kI) {
                constexpr int a = 2 * decltype(kI)::value;
                constexpr int ex = S::T.v[a][0], ey = S::T.v[a][1], ez = S::T.v[a][2];
                constexpr int dm = (D == 3) ? ez : ey;
                constexpr int dq = (D == 3) ? ey : 0;
                constexpr double wt = S::T.w[a] * L::cs2;
                const float* pp = base[dm + R] + dq * EX + ex;
                const float* pm = base[R - dm] - dq * EX - ex;
                const float2 d = sub2(make_float2(pp[0], pp[1]), make_float2(pm[0], pm[1]));
                if (ex != 0) ax = fma2(p2(float(wt * ex)), d, ax);
                if (ey != 0) ay = fma2(p2(float(wt * ey)), d, ay);
                if (ez != 0) az = fma2(p2(float(wt * ez)), d, az);
            });
            const float2 gp = mul2(p2(-p.G_f), make_float2(base[R][0], base[R][1]));
            const float2 F[3] = {mul2(gp, ax), mul2(gp, ay), mul2(gp, az)};
            collide2<LAT, 0>(fcur, F, p);
            const int c = m * mscale + cell_xy;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                *reinterpret_cast<float2*>(P.out[b] + c) = fcur[b];
            });
        }
        if (ST == 1) {
#pragma unroll
            for (int b = 0; b < Q; ++b) fcur[b] = fnxt[b];
        }
    }
}

// Deterministic block reduction of kObsWidth values (sums, last one a max).
__device__ __forceinline__ void block_reduce_obs(double (&v)[kObsWidth], double* out)
{
    __shared__ double sh[8][kObsWidth];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < kObsWidth - 1; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
        v[kObsWidth - 1] = fmax(v[kObsWidth - 1], __shfl_xor_sync(0xffffffffu, v[kObsWidth - 1], o));
    }
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < kObsWidth; ++i) sh[warp][i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        double acc[kObsWidth];
#pragma unroll
        for (int i = 0; i < kObsWidth; ++i) acc[i] = sh[0][i];
        for (int w = 1; w < nw; ++w) {
#pragma unroll
            for (int i = 0; i < kObsWidth - 1; ++i) acc[i] += sh[w][i];
            acc[kObsWidth - 1] = fmax(acc[kObsWidth - 1], sh[w][kObsWidth - 1]);
        }
#pragma unroll
        for (int i = 0; i < kObsWidth; ++i) out[i] = acc[i];
    }
}

// psi at (x + ex, y + ey, z + ez) from the ghosted buffer (|e| <= g).
template <int D, class Real>
__device__ __forceinline__ double psi_at(const Real* __restrict__ psi, const DevParams& p, int x, int y, int z)
{
    const int gz = (D == 3) ? p.g : 0;
    return static_cast<double>(psi[(static_cast<long long>(z + gz) * p.psy + (y + p.g)) * p.psx + (x + kGhostX)]);
}

// Density and momentum sums of one cell in FP64 (exact for FP32-stored values,
// so small currents keep their resolution); zero velocity components add nothing.
template <int LAT, class Real>
__device__ __forceinline__ void cell_sums(const Real* __restrict__ A, const DevParams& p, int x, int y, int z,
                                          double& rho, double (&j)[3])
{
    using L = Lattice<LAT>;
    Real f[L::Q];
    gather<LAT>(A, p, x, y, z, f);
    double s = 0.0;
    j[0] = j[1] = j[2] = 0.0;
    sfor<L::Q>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        const double fb = static_cast<double>(f[b]);
        s += fb;
        sfor<3>([&](auto iI) {
            constexpr int i = decltype(iI)::value;
            constexpr int c = L::T.v[b][i];
            if constexpr (c == 1) j[i] += fb;
            else if constexpr (c == -1) j[i] -= fb;
            else if constexpr (c != 0) j[i] += fb * c;
        });
    });
    rho = std::is_same<Real, float>::value ? p.rho_bar + s : s;
}

// Eq. 1 force of one cell in FP32 from an FP32 psi buffer (observables of FP32
// storage: relative error ~1e-7, off the slow FP64 pipe).
template <int LAT, int ORD>
__device__ __forceinline__ void cell_force_f32(const float* __restrict__ psi, const DevParams& p, int x, int y,
                                               int z, float (&F)[3])
{
    using L = Lattice<LAT>;
    using S = Stencil<L::D, ORD>;
    const int gz = (L::D == 3) ? p.g : 0;
    const float* c0 = psi + (static_cast<long long>(z + gz) * p.psy + (y + p.g)) * p.psx + (x + kGhostX);
    const long long sy = p.psx, sz = static_cast<long long>(p.psx) * p.psy;
    float ax = 0.f, ay = 0.f, az = 0.f;
    sfor<S::n / 2>([&](auto kI) {
        constexpr int a = 2 * decltype(kI)::value;
        constexpr int ex = S::T.v[a][0], ey = S::T.v[a][1], ez = S::T.v[a][2];
        constexpr float wt = static_cast<float>(S::T.w[a] * L::cs2);
        const long long o = ez * sz + ey * sy + ex;
        const float d = c0[o] - c0[-o];
        if (ex != 0) ax = fmaf(wt * ex, d, ax);
        if (ey != 0) ay = fmaf(wt * ey, d, ay);
        if (ez != 0) az = fmaf(wt * ez, d, az);
    });
    const float gp = -p.G_f * c0[0];
    F[0] = gp * ax;
    F[1] = gp * ay;
    F[2] = gp * az;
}

template <int LAT, int ORD, class Real>
__device__ __forceinline__ void cell_macro(const Real* __restrict__ A, const Real* __restrict__ psi,
                                           const DevParams& p, int x, int y, int z, double& rho, double (&mom)[3])
{
    using L = Lattice<LAT>;
    using S = Stencil<L::D, ORD>;
    double j[3];
    cell_sums<LAT>(A, p, x, y, z, rho, j);
    double acc[3] = {0.0, 0.0, 0.0};
    sfor<S::n>([&](auto aI) {
        constexpr int a = decltype(aI)::value;
        constexpr int ex = S::T.v[a][0], ey = S::T.v[a][1], ez = S::T.v[a][2];
        constexpr double wt = S::T.w[a] * L::cs2;
        const double wp = wt * psi_at<L::D>(psi, p, x + ex, y + ey, z + ez);
        acc[0] += wp * ex;
        acc[1] += wp * ey;
        acc[2] += wp * ez;
    });
    const double gp = -p.G * psi_at<L::D>(psi, p, x, y, z);
    for (int i = 0; i < 3; ++i) mom[i] = j[i] + 0.5 * (gp * acc[i]);
}

template <int LAT, int ORD, class Real>
__global__ void __launch_bounds__(256)
    k_obs(const Real* __restrict__ A, const Real* __restrict__ psi, DevParams p, double* __restrict__ partials)
{
    double v[kObsWidth] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < p.N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % p.nx);
        const long long r = i / p.nx;
        const int y = static_cast<int>(r % p.ny);
        const int z = static_cast<int>(r / p.ny);
        double rho, mom[3], um;
        if constexpr (std::is_same<Real, float>::value) {
            // FP32 storage: FP64 sums, FP32 force, 1/rho and |u|
            double j[3];
            cell_sums<LAT>(A, p, x, y, z, rho, j);
            float F[3];
            cell_force_f32<LAT, ORD>(psi, p, x, y, z, F);
            for (int k = 0; k < 3; ++k) mom[k] = j[k] + 0.5 * static_cast<double>(F[k]);
            const float inv = 1.0f / static_cast<float>(rho);
            const float ux = static_cast<float>(mom[0]) * inv, uy = static_cast<float>(mom[1]) * inv,
                        uz = static_cast<float>(mom[2]) * inv;
            um = static_cast<double>(sqrtf(ux * ux + uy * uy + uz * uz));
        } else {
            cell_macro<LAT, ORD>(A, psi, p, x, y, z, rho, mom);
            const double ux = mom[0] / rho, uy = mom[1] / rho, uz = mom[2] / rho;
            um = sqrt(ux * ux + uy * uy + uz * uz);
        }
        if (y < p.wall_rows) {  // solid: its populations count in the mass only
            if (!isfinite(rho)) bad = true;
            v[0] += rho;
            continue;
        }
        if (!isfinite(rho) || !isfinite(um)) bad = true;
        v[0] += rho;
        v[1] += mom[0];
        v[2] += mom[1];
        v[3] += mom[2];
        v[4] += um;
        v[5] = fmax(v[5], um);
    }
    if (bad) atomicOr(p.err, kErrNonFinite);
    block_reduce_obs(v, partials + static_cast<long long>(blockIdx.x) * kObsWidth);
}

// rho along the x line through the centre (threads 0..nx-1), at the vapour
// probe (thread nx) and at the liquid probe (thread nx+1).  Without a wall the
// probes are node 0 and the centre node; with one they are (0, ny-1, 0), the
// top fluid row, and (nx/2, wall_rows, nz/2), the first fluid node above the
// wall under the centre.
template <int LAT, class Real>
__global__ void k_probe(const Real* __restrict__ A, DevParams p, double* __restrict__ res)
{
    using L = Lattice<LAT>;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > p.nx + 1) return;
    const int zc = (L::D == 3) ? p.nz / 2 : 0;
    int x, y, z, slot;
    if (i < p.nx) {
        x = i; y = p.ny / 2; z = zc; slot = kResLine + i;
    } else if (i == p.nx) {
        x = 0; y = p.wall_rows ? p.ny - 1 : 0; z = 0; slot = kResRhoOrigin;
    } else {
        x = p.nx / 2; y = p.wall_rows ? p.wall_rows : p.ny / 2; z = zc; slot = kResRhoCentre;
    }
    Real f[L::Q];
    gather<LAT>(A, p, x, y, z, f);
    double s = 0.0;
    sfor<L::Q>([&](auto bI) { s += static_cast<double>(f[decltype(bI)::value]); });
    const double rho = std::is_same<Real, float>::value ? p.rho_bar + s : s;
    res[slot] = rho;
}

template <int LAT, int ORD, class Real>
__global__ void __launch_bounds__(256) k_fields(const Real* __restrict__ A, const Real* __restrict__ psi,
                                                DevParams p, double* __restrict__ rho_out, double* __restrict__ u_out)
{
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < p.N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % p.nx);
        const long long r = i / p.nx;
        const int y = static_cast<int>(r % p.ny);
        const int z = static_cast<int>(r / p.ny);
        double rho, mom[3];
        cell_macro<LAT, ORD>(A, psi, p, x, y, z, rho, mom);
        const bool solid = y < p.wall_rows;  // solid nodes report u = 0
        if (rho_out) rho_out[i] = rho;
        if (u_out)
            for (int k = 0; k < 3; ++k) u_out[3 * i + k] = solid ? 0.0 : mom[k] / rho;
    }
}

// Minimum-image distance of node index i to the centre node n/2.
__device__ __forceinline__ double min_image(int i, int n)
{
    double d = static_cast<double>(i) - static_cast<double>(n / 2);
    if (d > 0.5 * n) d -= n;
    if (d < -0.5 * n) d += n;
    return d;
}

// Tanh initial density (Sec. 3): droplet (mode 0) or flat slab (mode 1).
template <int D>
__global__ void k_init_profile(DevParams p, int mode, int axis, double rl, double rg, double R, double W,
                               double* __restrict__ rho0)
{
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < p.N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % p.nx);
        const long long r = i / p.nx;
        const int y = static_cast<int>(r % p.ny);
        const int z = static_cast<int>(r / p.ny);
        double dist, rad;
        if (mode == 0) {
            const double dx = min_image(x, p.nx), dy = min_image(y, p.ny);
            const double dz = (D == 3) ? min_image(z, p.nz) : 0.0;
            dist = sqrt(dx * dx + dy * dy + dz * dz);
            rad = R;
        } else {
            const int L = (axis == 0) ? p.nx : ((axis == 1) ? p.ny : p.nz);
            const int k = (axis == 0) ? x : ((axis == 1) ? y : z);
            dist = fabs(min_image(k, L));
            rad = 0.25 * L;
        }
        rho0[i] = 0.5 * (rl + rg) - 0.5 * (rl - rg) * tanh(2.0 * (dist - rad) / W);
    }
}

// A_b(y) = w_b rho0(y + c_b)  (FP32: w_b (rho0 - rho_bar)), so that the pulled
// state is f = feq(rho0, 0).
template <int LAT, class Real>
__global__ void __launch_bounds__(256) k_init_from_rho(const double* __restrict__ rho0, DevParams p, Real* __restrict__ A)
{
    using L = Lattice<LAT>;
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < p.N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % p.nx);
        const long long r = i / p.nx;
        const int y = static_cast<int>(r % p.ny);
        const int z = static_cast<int>(r / p.ny);
        sfor<L::Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
            const int xs = shift_wrap_fwd<cx>(x, p.nx), ys = shift_wrap_fwd<cy>(y, p.ny);
            const int zs = (L::D == 3) ? shift_wrap_fwd<cz>(z, p.nz) : 0;
            constexpr double wb = L::T.w[b];
            const double rv = rho0[cell_of(p, xs, ys, zs)];
            const double v = std::is_same<Real, float>::value ? wb * (rv - p.rho_bar) : wb * rv;
            A[static_cast<long long>(b) * p.N + i] = static_cast<Real>(v);
        });
    }
}

// Pre-collision populations in double, [Q][cell].
template <int LAT, class Real>
__global__ void __launch_bounds__(256) k_get_f(const Real* __restrict__ A, DevParams p, double* __restrict__ out)
{
    using L = Lattice<LAT>;
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < p.N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % p.nx);
        const long long r = i / p.nx;
        const int y = static_cast<int>(r % p.ny);
        const int z = static_cast<int>(r / p.ny);
        Real f[L::Q];
        gather<LAT>(A, p, x, y, z, f);
        sfor<L::Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr double wb = L::T.w[b];
            const double shift = std::is_same<Real, float>::value ? wb * p.rho_bar : 0.0;
            out[static_cast<long long>(b) * p.N + i] = static_cast<double>(f[b]) + shift;
        });
    }
}

template <int LAT, class Real>
__global__ void __launch_bounds__(256) k_set_f(const double* __restrict__ in, DevParams p, Real* __restrict__ A)
{
    using L = Lattice<LAT>;
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < p.N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % p.nx);
        const long long r = i / p.nx;
        const int y = static_cast<int>(r % p.ny);
        const int z = static_cast<int>(r / p.ny);
        sfor<L::Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1], cz = L::T.v[b][2];
            const int xs = shift_wrap_fwd<cx>(x, p.nx), ys = shift_wrap_fwd<cy>(y, p.ny);
            const int zs = (L::D == 3) ? shift_wrap_fwd<cz>(z, p.nz) : 0;
            constexpr double wb = L::T.w[b];
            const double shift = std::is_same<Real, float>::value ? wb * p.rho_bar : 0.0;
            A[static_cast<long long>(b) * p.N + i] =
                static_cast<Real>(in[static_cast<long long>(b) * p.N + cell_of(p, xs, ys, zs)] - shift);
        });
    }
}

// rho(x) = sum_b f_b(x) of a double population array in the pre-collision layout.
template <int LAT>
__global__ void __launch_bounds__(256) k_rho_of_f(const double* __restrict__ in, DevParams p, double* __restrict__ rho)
{
    using L = Lattice<LAT>;
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < p.N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        double s = 0.0;
        sfor<L::Q>([&](auto bI) { s += in[static_cast<long long>(decltype(bI)::value) * p.N + i]; });
        rho[i] = s;
    }
}

// ---- launchers ---------------------------------------------------------------------------
inline int grid_1d(long long n, int cap = 152 * 16)
{
    long long b = (n + 255) / 256;
    if (b < 1) b = 1;
    return static_cast<int>(b < cap ? b : cap);
}

template <int LAT, class Real>
cudaError_t launch_psi(const LaunchArgs& a, cudaStream_t s)
{
    const dim3 blk(32, 8, 1);
    const dim3 grd((a.p.nx + 31) / 32, (a.p.ny + 7) / 8, Lattice<LAT>::D == 3 ? a.p.nz : 1);
    k_psi<LAT, Real><<<grd, blk, 0, s>>>(static_cast<const Real*>(a.fin), static_cast<Real*>(a.psi), a.p);
    return cudaGetLastError();
}

template <int LAT, int ORD, int COLL, class Real, int TY, int TZ>
cudaError_t launch_fused(const LaunchArgs& a, cudaStream_t s)
{
    const dim3 blk(32, TY, TZ);
    const dim3 grd((a.p.nx + 31) / 32, (a.p.ny + TY - 1) / TY, Lattice<LAT>::D == 3 ? (a.p.nz + TZ - 1) / TZ : 1);
    k_fused<LAT, ORD, COLL, Real, TY, TZ><<<grd, blk, 0, s>>>(*a.tmap, static_cast<const Real*>(a.fin),
                                                             static_cast<Real*>(a.fout), a.p);
    if (Lattice<LAT>::D == 2 && a.p.wall_rows > 0) {
        const long long n = static_cast<long long>(a.p.nx) * a.p.wall_rows;
        k_bounce<LAT, Real><<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(
            static_cast<const Real*>(a.fin), static_cast<Real*>(a.fout), a.p);
    }
    return cudaGetLastError();
}

template <int LAT, int ORD, int COLL, class Real, int TX, int TY, int ZC, int MINB, int ST>
cudaError_t launch_onepass(const LaunchArgs& a, cudaStream_t s)
{
    constexpr int R = Stencil<Lattice<LAT>::D, ORD>::radius;
    constexpr size_t dyn = (ST == 2) ? sizeof(Real) * (R + 1) * Lattice<LAT>::Q * TX * TY : 0;
    auto kern = &k_onepass<LAT, ORD, COLL, Real, TX, TY, ZC, MINB, ST>;
    if (cudaError_t e = ensure_dyn_smem(kern, dyn); e != cudaSuccess) return e;
    constexpr bool k3 = Lattice<LAT>::D == 3;
    const int ntx = (a.p.nx + TX - 1) / TX;
    const int nty = k3 ? (a.p.ny + TY - 1) / TY : 1;
    const int nm = k3 ? a.p.nz : a.p.ny;
    const long long nblocks = static_cast<long long>(ntx) * nty * ((nm + ZC - 1) / ZC);
    const auto P = make_pops<Real, Lattice<LAT>::Q>(a.fin, a.fout, a.p.N);
    kern<<<static_cast<unsigned>(nblocks), TX * TY, dyn, s>>>(P, a.p, ntx, nty);
    return cudaGetLastError();
}

// Chunk length of the persistent whole-row schedules (one block per SM): the
// chunk count that minimises the largest number of slabs a block marches, its
// items x (chunk + the warm-up slabs, 2R).
inline int rowp_chunk(int nz, int nty, int nsm, int warm = 2)
{
    int zc = nz;
    long long best = -1;
    for (int nc = 1; nc <= nz; ++nc) {
        const int len = (nz + nc - 1) / nc;
        const int used = (nz + len - 1) / len;
        const long long per_block = (static_cast<long long>(nty) * used + nsm - 1) / nsm;
        const long long cost = per_block * (len + warm);
        if (best < 0 || cost < best) {
            best = cost;
            zc = len;
        }
    }
    return zc;
}

template <int LAT, int ORD, int COLL, int NX, int TY, int NSTG, bool PRODW = true>
cudaError_t launch_onepass_rowp2(const LaunchArgs& a, cudaStream_t s)
{
    constexpr size_t dyn = sizeof(float) * NSTG * Lattice<LAT>::Q * (TY + 2) * NX;
    auto kern = &k_onepass_rowp2<LAT, ORD, COLL, NX, TY, NSTG, PRODW>;
    if (cudaError_t e = ensure_dyn_smem(kern, dyn); e != cudaSuccess) return e;
    if (a.p.nx != NX) return cudaErrorInvalidValue;
    const int nty = (a.p.ny + TY - 1) / TY;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int zc = rowp_chunk(a.p.nz, nty, nsm);
    const int nitems = nty * ((a.p.nz + zc - 1) / zc);
    const int grid = nitems < nsm ? nitems : nsm;
    const auto P = make_pops<float, Lattice<LAT>::Q>(a.fin, a.fout, a.p.N);
    kern<<<grid, NX / 2 * TY + (PRODW ? 32 : 0), dyn, s>>>(P, a.p, zc, nitems);
    return cudaGetLastError();
}

// Whole-row packed-pair schedule for any row length nx <= NXMAX that is a
// multiple of 4 (16-byte rows for the bulk copies): the kernel reads nx from
// the domain, the psi ring moves into dynamic shared memory after the stages,
// and the compute threads are rounded up to whole warps.
template <int LAT, int ORD, int COLL, int NXMAX, int TY, int NSTG, bool PRODW>
cudaError_t launch_onepass_rowp2w(const LaunchArgs& a, cudaStream_t s)
{
    constexpr int Q = Lattice<LAT>::Q;
    constexpr int R = Stencil<3, ORD>::radius;
    constexpr int EY = TY + 2 * R;
    constexpr int NS = 2 * R + 2;
    auto dyn_of = [](int nx) {
        return sizeof(float) * (static_cast<size_t>(NSTG) * Q * EY * nx + static_cast<size_t>(NS) * (nx + 2 * R) * EY);
    };
    auto kern = &k_onepass_rowp2<LAT, ORD, COLL, 0, TY, NSTG, PRODW, NXMAX>;
    if (cudaError_t e = ensure_dyn_smem(kern, dyn_of(NXMAX)); e != cudaSuccess) return e;
    const int nx = a.p.nx;
    if (nx % 4 != 0 || nx < 8 || nx > NXMAX) return cudaErrorInvalidValue;
    const int nty = (a.p.ny + TY - 1) / TY;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int zc = rowp_chunk(a.p.nz, nty, nsm);
    const int nitems = nty * ((a.p.nz + zc - 1) / zc);
    const int grid = nitems < nsm ? nitems : nsm;
    const int threads = (nx / 2 * TY + 31) / 32 * 32 + (PRODW ? 32 : 0);
    const auto P = make_pops<float, Q>(a.fin, a.fout, a.p.N);
    kern<<<grid, threads, dyn_of(nx), s>>>(P, a.p, zc, nitems);
    return cudaGetLastError();
}

// Radius-2 whole-row schedule (k_onepass_rowr), any row length nx <= NXMAX
// that is a multiple of 4.
template <int LAT, int ORD, int COLL, int NXMAX, int TY, int NSTG, bool PRODW>
cudaError_t launch_onepass_rowr(const LaunchArgs& a, cudaStream_t s)
{
    constexpr int Q = Lattice<LAT>::Q;
    constexpr int R = Stencil<3, ORD>::radius;
    constexpr int EY = TY + 2 * R;
    constexpr int NS = 2 * R + 2;
    auto dyn_of = [](int nx) {
        return sizeof(float) * (static_cast<size_t>(NSTG) * Q * EY * nx + static_cast<size_t>(NS) * (nx + 2 * R) * EY);
    };
    auto kern = &k_onepass_rowr<LAT, ORD, COLL, TY, NSTG, PRODW, NXMAX>;
    if (cudaError_t e = ensure_dyn_smem(kern, dyn_of(NXMAX)); e != cudaSuccess) return e;
    const int nx = a.p.nx;
    if (nx % 4 != 0 || nx < 8 || nx > NXMAX) return cudaErrorInvalidValue;
    const int nty = (a.p.ny + TY - 1) / TY;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int zc = rowp_chunk(a.p.nz, nty, nsm, 2 * R);
    const int nitems = nty * ((a.p.nz + zc - 1) / zc);
    const int grid = nitems < nsm ? nitems : nsm;
    const int threads = (nx / 2 * TY + 31) / 32 * 32 + (PRODW ? 32 : 0);
    const auto P = make_pops<float, Q>(a.fin, a.fout, a.p.N);
    kern<<<grid, threads, dyn_of(nx), s>>>(P, a.p, zc, nitems);
    return cudaGetLastError();
}

// Whole-row schedule with a carried density (k_onepass_rowc), any row length
// nx <= NXMAX that is a multiple of 4.  Reads the carry of the current state
// (a.carry_in) and writes that of the next (a.carry_out).
template <int LAT, int ORD, int COLL, int NXMAX, int TY, int NSTG>
cudaError_t launch_onepass_rowc(const LaunchArgs& a, cudaStream_t s)
{
    constexpr int Q = Lattice<LAT>::Q;
    constexpr int R = Stencil<3, ORD>::radius;
    constexpr int EY = TY + 2 * R;
    constexpr int NS = 2 * R + 1;
    constexpr int NXD = xchg_count<LAT>();
    auto dyn_of = [](int nx) {
        return sizeof(float) * (static_cast<size_t>(NSTG) * Q * TY * nx + static_cast<size_t>(NS) * (nx + 2 * R) * EY +
                                static_cast<size_t>(NXD) * TY * nx);
    };
    auto kern = &k_onepass_rowc<LAT, ORD, COLL, TY, NSTG, NXMAX>;
    if (cudaError_t e = ensure_dyn_smem(kern, dyn_of(NXMAX)); e != cudaSuccess) return e;
    const int nx = a.p.nx;
    if (nx % 4 != 0 || nx < 8 || nx > NXMAX || !a.carry_in || !a.carry_out) return cudaErrorInvalidValue;
    const int nty = (a.p.ny + TY - 1) / TY;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int zc = rowp_chunk(a.p.nz, nty, nsm, 2);
    const int nitems = nty * ((a.p.nz + zc - 1) / zc);
    const int grid = nitems < nsm ? nitems : nsm;
    const int threads = (nx / 2 * TY + 31) / 32 * 32;
    const long long fr = static_cast<long long>(nty) * a.p.nz * nx;
    const CarryView cv{a.carry_in, a.carry_in + a.p.N, a.carry_in + a.p.N + fr};
    const auto P = make_pops<float, Q>(a.fin, a.fout, a.p.N);
    kern<<<grid, threads, dyn_of(nx), s>>>(P, a.p, cv, a.carry_out, zc, nitems);
    return cudaGetLastError();
}

// Starts the carry of the current state (a.fin) in a.carry_in for groups of ty
// rows: own = the whole pulled sum, frames zero.
template <int LAT>
cudaError_t launch_carry_init(const LaunchArgs& a, int ty, cudaStream_t s)
{
    if (!a.carry_in || ty < 1) return cudaErrorInvalidValue;
    const int nty = (a.p.ny + ty - 1) / ty;
    const auto P = make_pops<float, Lattice<LAT>::Q>(a.fin, a.fout, a.p.N);
    k_carry_init<LAT><<<grid_1d(carry_floats(a.p.N, nty, a.p.nz, a.p.nx)), 256, 0, s>>>(P, a.p, a.carry_in, nty);
    return cudaGetLastError();
}

template <int LAT, int ORD, int COLL, class Real, int NX, int TY, int NSTG>
cudaError_t launch_onepass_rowp(const LaunchArgs& a, cudaStream_t s)
{
    constexpr size_t dyn = sizeof(Real) * NSTG * Lattice<LAT>::Q * (TY + 2) * NX;
    auto kern = &k_onepass_rowp<LAT, ORD, COLL, Real, NX, TY, NSTG>;
    if (cudaError_t e = ensure_dyn_smem(kern, dyn); e != cudaSuccess) return e;
    if (a.p.nx != NX) return cudaErrorInvalidValue;
    const int nty = (a.p.ny + TY - 1) / TY;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int zc = rowp_chunk(a.p.nz, nty, nsm);
    const int nitems = nty * ((a.p.nz + zc - 1) / zc);
    const int grid = nitems < nsm ? nitems : nsm;
    const auto P = make_pops<Real, Lattice<LAT>::Q>(a.fin, a.fout, a.p.N);
    kern<<<grid, NX * TY + 32, dyn, s>>>(P, a.p, zc, nitems);
    return cudaGetLastError();
}

template <int LAT, int ORD, int COLL, class Real, int NX, int TY, int ZC, int NSTG, int PROD>
cudaError_t launch_onepass_row(const LaunchArgs& a, cudaStream_t s)
{
    constexpr size_t dyn = sizeof(Real) * NSTG * Lattice<LAT>::Q * (TY + 2) * NX;
    auto kern = &k_onepass_row<LAT, ORD, COLL, Real, NX, TY, ZC, NSTG, PROD>;
    if (cudaError_t e = ensure_dyn_smem(kern, dyn); e != cudaSuccess) return e;
    if (a.p.nx != NX) return cudaErrorInvalidValue;
    const int nty = (a.p.ny + TY - 1) / TY;
    int zc = ZC;
    if (ZC == 0) {
        // one block per SM (shared memory): pick the chunk count that minimises
        // waves x (slabs per chunk + the two warm-up slabs of every chunk)
        int dev = 0, nsm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        long long best = -1;
        for (int nc = 1; nc <= a.p.nz; ++nc) {
            const int len = (a.p.nz + nc - 1) / nc;
            const int used = (a.p.nz + len - 1) / len;  // chunks actually launched
            const long long waves = (static_cast<long long>(nty) * used + nsm - 1) / nsm;
            const long long cost = waves * (len + 2);
            if (best < 0 || cost < best) {
                best = cost;
                zc = len;
            }
        }
    }
    const long long nblocks = static_cast<long long>(nty) * ((a.p.nz + zc - 1) / zc);
    const auto P = make_pops<Real, Lattice<LAT>::Q>(a.fin, a.fout, a.p.N);
    kern<<<static_cast<unsigned>(nblocks), NX * TY + (PROD ? 32 : 0), dyn, s>>>(P, a.p, zc);
    return cudaGetLastError();
}

template <int LAT, int ORD, int COLL, class Real, int TX, int ZC, int NSTG>
cudaError_t launch_onepass_seg(const LaunchArgs& a, cudaStream_t s)
{
    constexpr int XP = 16 / static_cast<int>(sizeof(Real));
    constexpr size_t dyn = sizeof(Real) * NSTG * Lattice<LAT>::Q * (TX + 2 * XP);
    auto kern = &k_onepass_seg<LAT, ORD, COLL, Real, TX, ZC, NSTG>;
    if (cudaError_t e = ensure_dyn_smem(kern, dyn); e != cudaSuccess) return e;
    if (a.p.nx % XP != 0) return cudaErrorInvalidValue;
    const int ntx = (a.p.nx + TX - 1) / TX;
    const long long nblocks = static_cast<long long>(ntx) * ((a.p.ny + ZC - 1) / ZC);
    const auto P = make_pops<Real, Lattice<LAT>::Q>(a.fin, a.fout, a.p.N);
    kern<<<static_cast<unsigned>(nblocks), TX + 32, dyn, s>>>(P, a.p, ntx);
    return cudaGetLastError();
}

template <int LAT, int ORD, int COLL, int TX, int ZC, int NSTG>
cudaError_t launch_onepass_seg2(const LaunchArgs& a, cudaStream_t s)
{
    constexpr size_t dyn = sizeof(float) * NSTG * Lattice<LAT>::Q * (TX + 8);
    auto kern = &k_onepass_seg2<LAT, ORD, COLL, TX, ZC, NSTG>;
    if (cudaError_t e = ensure_dyn_smem(kern, dyn); e != cudaSuccess) return e;
    if (a.p.nx % 4 != 0) return cudaErrorInvalidValue;
    const int ntx = (a.p.nx + TX - 1) / TX;
    const long long nblocks = static_cast<long long>(ntx) * ((a.p.ny + ZC - 1) / ZC);
    const auto P = make_pops<float, Lattice<LAT>::Q>(a.fin, a.fout, a.p.N);
    kern<<<static_cast<unsigned>(nblocks), TX / 2 + 32, dyn, s>>>(P, a.p, ntx);
    return cudaGetLastError();
}

template <int LAT, int ORD, int COLL, class Real, int TX, int TY, int ZC, int MINB>
cudaError_t launch_onepass_async(const LaunchArgs& a, cudaStream_t s)
{
    using L = Lattice<LAT>;
    constexpr int R = Stencil<L::D, ORD>::radius;
    constexpr int EX = TX + 2 * R;
    constexpr int EY = (L::D == 3) ? TY + 2 * R : 1;
    constexpr int H = EX * EY - TX * TY;
    constexpr size_t dyn = sizeof(Real) * L::Q * ((R + 2) * TX * TY + 2 * H);
    auto kern = &k_onepass_async<LAT, ORD, COLL, Real, TX, TY, ZC, MINB>;
    if (cudaError_t e = ensure_dyn_smem(kern, dyn); e != cudaSuccess) return e;
    constexpr bool k3 = L::D == 3;
    const int ntx = (a.p.nx + TX - 1) / TX;
    const int nty = k3 ? (a.p.ny + TY - 1) / TY : 1;
    const int nm = k3 ? a.p.nz : a.p.ny;
    const long long nblocks = static_cast<long long>(ntx) * nty * ((nm + ZC - 1) / ZC);
    const auto P = make_pops<Real, L::Q>(a.fin, a.fout, a.p.N);
    kern<<<static_cast<unsigned>(nblocks), TX * TY, dyn, s>>>(P, a.p, ntx, nty);
    return cudaGetLastError();
}

template <int LAT, int ORD, int COLL, class Real, int TX, int TY, int ZC, int MINB, int HL>
cudaError_t launch_onepass_la(const LaunchArgs& a, cudaStream_t s)
{
    using L = Lattice<LAT>;
    constexpr int R = Stencil<L::D, ORD>::radius;
    constexpr size_t dyn = sizeof(Real) * (R + 2) * L::Q * TX * TY;
    auto kern = &k_onepass_la<LAT, ORD, COLL, Real, TX, TY, ZC, MINB, HL>;
    if (cudaError_t e = ensure_dyn_smem(kern, dyn); e != cudaSuccess) return e;
    constexpr bool k3 = L::D == 3;
    const int ntx = (a.p.nx + TX - 1) / TX;
    const int nty = k3 ? (a.p.ny + TY - 1) / TY : 1;
    const int nm = k3 ? a.p.nz : a.p.ny;
    const long long nblocks = static_cast<long long>(ntx) * nty * ((nm + ZC - 1) / ZC);
    const auto P = make_pops<Real, L::Q>(a.fin, a.fout, a.p.N);
    kern<<<static_cast<unsigned>(nblocks), TX * TY, dyn, s>>>(P, a.p, ntx, nty);
    return cudaGetLastError();
}

template <int LAT, int ORD, int TX2, int TY, int ZC, int MINB, int ST>
cudaError_t launch_onepass_x2(const LaunchArgs& a, cudaStream_t s)
{
    using L = Lattice<LAT>;
    constexpr int R = Stencil<L::D, ORD>::radius;
    constexpr size_t dyn = (ST == 2) ? sizeof(float2) * (R + 1) * L::Q * TX2 * TY : 0;
    auto kern = &k_onepass_x2<LAT, ORD, TX2, TY, ZC, MINB, ST>;
    if (cudaError_t e = ensure_dyn_smem(kern, dyn); e != cudaSuccess) return e;
    constexpr bool k3 = L::D == 3;
    constexpr int TX = 2 * TX2;
    const int ntx = (a.p.nx + TX - 1) / TX;
    const int nty = k3 ? (a.p.ny + TY - 1) / TY : 1;
    const int nm = k3 ? a.p.nz : a.p.ny;
    const long long nblocks = static_cast<long long>(ntx) * nty * ((nm + ZC - 1) / ZC);
    const auto P = make_pops<float, L::Q>(a.fin, a.fout, a.p.N);
    kern<<<static_cast<unsigned>(nblocks), TX2 * TY, dyn, s>>>(P, a.p, ntx, nty);
    return cudaGetLastError();
}

template <int LAT, int ORD, class Real>
cudaError_t launch_obs(const LaunchArgs& a, cudaStream_t s, int* nblocks)
{
    const int nb = grid_1d(a.p.N, a.nblocks_max);
    k_obs<LAT, ORD, Real><<<nb, 256, 0, s>>>(static_cast<const Real*>(a.fin), static_cast<const Real*>(a.psi),
                                             a.p, a.partials);
    *nblocks = nb;
    return cudaGetLastError();
}

template <int LAT, class Real>
cudaError_t launch_probe(const LaunchArgs& a, cudaStream_t s)
{
    const int n = a.p.nx + 2;
    k_probe<LAT, Real><<<(n + 127) / 128, 128, 0, s>>>(static_cast<const Real*>(a.fin), a.p, a.res);
    return cudaGetLastError();
}

template <int LAT, int ORD, class Real>
cudaError_t launch_fields(const LaunchArgs& a, cudaStream_t s)
{
    k_fields<LAT, ORD, Real><<<grid_1d(a.p.N), 256, 0, s>>>(static_cast<const Real*>(a.fin),
                                                           static_cast<const Real*>(a.psi), a.p, a.dbuf0, a.dbuf1);
    return cudaGetLastError();
}

template <int LAT>
cudaError_t launch_init_profile(const LaunchArgs& a, cudaStream_t s)
{
    k_init_profile<Lattice<LAT>::D><<<grid_1d(a.p.N), 256, 0, s>>>(a.p, a.mode, a.axis, a.a0, a.a1, a.a2, a.a3,
                                                                   a.dbuf0);
    return cudaGetLastError();
}

template <int LAT, class Real>
cudaError_t launch_init_from_rho(const LaunchArgs& a, cudaStream_t s)
{
    k_init_from_rho<LAT, Real><<<grid_1d(a.p.N), 256, 0, s>>>(a.dbuf0, a.p, static_cast<Real*>(a.fout));
    return cudaGetLastError();
}

template <int LAT, class Real>
cudaError_t launch_get_f(const LaunchArgs& a, cudaStream_t s)
{
    k_get_f<LAT, Real><<<grid_1d(a.p.N), 256, 0, s>>>(static_cast<const Real*>(a.fin), a.p, a.dbuf0);
    return cudaGetLastError();
}

template <int LAT, class Real>
cudaError_t launch_set_f(const LaunchArgs& a, cudaStream_t s)
{
    k_set_f<LAT, Real><<<grid_1d(a.p.N), 256, 0, s>>>(a.dbuf0, a.p, static_cast<Real*>(a.fout));
    return cudaGetLastError();
}

template <int LAT>
cudaError_t launch_rho_of_f(const LaunchArgs& a, cudaStream_t s)
{
    k_rho_of_f<LAT><<<grid_1d(a.p.N), 256, 0, s>>>(a.dbuf0, a.p, a.dbuf1);
    return cudaGetLastError();
}

// The one-pass variants offered to the autotuner for (LAT, ORD, COLL, Real):
// tile TX x TY (2-D: TX), chunk of ZC slabs, at least MINB resident blocks per
// SM (a register cap).  Built at compile time, so a list longer than the
// schedule table is a build error rather than a silently dropped variant.
struct VariantList {
    int n;
    bool overflow;
    StepVariant v[kMaxVariants];
};

template <int LAT, int ORD, int COLL, class Real>
constexpr VariantList make_variants()
{
    constexpr bool k3 = Lattice<LAT>::D == 3;
    VariantList k{};
    auto add = [&k](const char* name, cudaError_t (*fn)(const LaunchArgs&, cudaStream_t), int nx_mult = 1,
                    int nx_exact = 0, int nx_max = 0, int carry_rows = 0) {
        if (k.n >= kMaxVariants) {
            k.overflow = true;
            return;
        }
        k.v[k.n].name = name;
        k.v[k.n].fn = fn;
        k.v[k.n].nx_multiple = nx_mult;
        k.v[k.n].nx_exact = nx_exact;
        k.v[k.n].nx_max = nx_max;
        k.v[k.n].carry_rows = carry_rows;
        ++k.n;
    };
    constexpr bool r1 = Stencil<Lattice<LAT>::D, ORD>::radius == 1;
    constexpr bool hot = COLL == 0 && std::is_same<Real, float>::value;
    if constexpr (k3) {
        add("onepass_32x8_z16_b2_smem", &launch_onepass<LAT, ORD, COLL, Real, 32, 8, 16, 2, 2>);
        if constexpr (hot) {
            add("onepass_32x8_z16_b4_smem", &launch_onepass<LAT, ORD, COLL, Real, 32, 8, 16, 4, 2>);
            add("onepass_32x8_z16_b3_smem", &launch_onepass<LAT, ORD, COLL, Real, 32, 8, 16, 3, 2>);
            if constexpr (r1) add("onepass_32x8_z16_b3_reg", &launch_onepass<LAT, ORD, COLL, Real, 32, 8, 16, 3, 1>);
            add("onepass_32x8_z16_b4_regather", &launch_onepass<LAT, ORD, COLL, Real, 32, 8, 16, 4, 0>);
            add("onepass_async_32x8_z16_b2", &launch_onepass_async<LAT, ORD, COLL, Real, 32, 8, 16, 2>);
            add("onepass_async_32x8_z32_b2", &launch_onepass_async<LAT, ORD, COLL, Real, 32, 8, 32, 2>);
            if constexpr (r1) {
                add("onepass_async_64x4_z16_b2", &launch_onepass_async<LAT, ORD, COLL, Real, 64, 4, 16, 2>);
                add("onepass_64x4_z16_b4_smem", &launch_onepass<LAT, ORD, COLL, Real, 64, 4, 16, 4, 2>);
                add("onepass_row256x2_z32_s2", &launch_onepass_row<LAT, ORD, COLL, Real, 256, 2, 32, 2, 0>, 1, 256);
                add("onepass_row256x2_z32_s2_prod", &launch_onepass_row<LAT, ORD, COLL, Real, 256, 2, 32, 2, 1>, 1, 256);
                add("onepass_row256x2_zauto_s2_prod", &launch_onepass_row<LAT, ORD, COLL, Real, 256, 2, 0, 2, 1>, 1, 256);
                add("onepass_row256x2_zauto_s2_prod_cs", &launch_onepass_row<LAT, ORD, COLL, Real, 256, 2, 0, 2, 2>, 1, 256);
                add("onepass_rowp256x2_s2", &launch_onepass_rowp<LAT, ORD, COLL, Real, 256, 2, 2>, 1, 256);
                add("onepass_rowp2_256x2_s2", &launch_onepass_rowp2<LAT, ORD, 0, 256, 2, 2>, 1, 256);
                add("onepass_rowp2_256x3_s2", &launch_onepass_rowp2<LAT, ORD, 0, 256, 3, 2>, 1, 256);
                add("onepass_rowp2_256x3_s2_np", &launch_onepass_rowp2<LAT, ORD, 0, 256, 3, 2, false>, 1, 256);
                add("onepass_rowp2_w256x3_s2_np", &launch_onepass_rowp2w<LAT, ORD, 0, 256, 3, 2, false>, 4, 0, 256);
                add("onepass_rowp2_w224x3_s2", &launch_onepass_rowp2w<LAT, ORD, 0, 224, 3, 2, true>, 4, 0, 224);
                add("onepass_rowp2_w208x2_s3", &launch_onepass_rowp2w<LAT, ORD, 0, 208, 2, 3, true>, 4, 0, 208);
                add("onepass_rowp2_w344x2_s2", &launch_onepass_rowp2w<LAT, ORD, 0, 344, 2, 2, true>, 4, 0, 344);
                add("onepass_rowp2_w456x1_s2", &launch_onepass_rowp2w<LAT, ORD, 0, 456, 1, 2, true>, 4, 0, 456);
                add("onepass_row128x4_z32_s3", &launch_onepass_row<LAT, ORD, COLL, Real, 128, 4, 32, 3, 0>, 1, 128);
                add("onepass_row128x4_z32_s3_prod", &launch_onepass_row<LAT, ORD, COLL, Real, 128, 4, 32, 3, 1>, 1, 128);
                add("onepass_row128x4_zauto_s3_prod_cs", &launch_onepass_row<LAT, ORD, COLL, Real, 128, 4, 0, 3, 2>, 1, 128);
                add("onepass_x2_64x8_z16_b2_reg", &launch_onepass_x2<LAT, ORD, 32, 8, 16, 2, 1>, 2);
                add("onepass_128x4_z16_b2_smem", &launch_onepass<LAT, ORD, COLL, Real, 128, 4, 16, 2, 2>);
                add("onepass_64x4_z8_b4_smem", &launch_onepass<LAT, ORD, COLL, Real, 64, 4, 8, 4, 2>);
                add("onepass_64x4_z32_b4_smem", &launch_onepass<LAT, ORD, COLL, Real, 64, 4, 32, 4, 2>);
                add("onepass_la_64x4_z16_b2", &launch_onepass_la<LAT, ORD, COLL, Real, 64, 4, 16, 2, 1>);
                add("onepass_lai_64x4_z16_b3", &launch_onepass_la<LAT, ORD, COLL, Real, 64, 4, 16, 3, 0>);
                add("onepass_lai_64x4_z16_b4", &launch_onepass_la<LAT, ORD, COLL, Real, 64, 4, 16, 4, 0>);
                add("onepass_lai_64x4_z32_b3", &launch_onepass_la<LAT, ORD, COLL, Real, 64, 4, 32, 3, 0>);
            }
            if constexpr (Stencil<3, ORD>::radius == 2) {
                add("onepass_rowr_w256x2_s1", &launch_onepass_rowr<LAT, ORD, COLL, 256, 2, 1, true>, 4, 0, 256);
                add("onepass_rowr_w256x2_s1_np", &launch_onepass_rowr<LAT, ORD, COLL, 256, 2, 1, false>, 4, 0, 256);
                add("onepass_rowr_w256x3_s1_np", &launch_onepass_rowr<LAT, ORD, COLL, 256, 3, 1, false>, 4, 0, 256);
                add("onepass_rowr_w256x1_s2", &launch_onepass_rowr<LAT, ORD, COLL, 256, 1, 2, true>, 4, 0, 256);
            }
            if constexpr (Lattice<LAT>::reach == 1) {
                add("onepass_rowc_w256x3_s2", &launch_onepass_rowc<LAT, ORD, COLL, 256, 3, 2>, 4, 0, 256, 3);
                add("onepass_rowc_w256x2_s3", &launch_onepass_rowc<LAT, ORD, COLL, 256, 2, 3>, 4, 0, 256, 2);
            }
            add("onepass_la_32x8_z16_b2", &launch_onepass_la<LAT, ORD, COLL, Real, 32, 8, 16, 2, 1>);
            add("onepass_lai_32x8_z16_b3", &launch_onepass_la<LAT, ORD, COLL, Real, 32, 8, 16, 3, 0>);
            add("onepass_x2_64x8_z16_b2_smem", &launch_onepass_x2<LAT, ORD, 32, 8, 16, 2, 2>, 2);
        }
        // MRT in FP32: the packed-pair whole-row kernels (nx = 256)
        if constexpr (COLL == 1 && std::is_same<Real, float>::value && r1) {
            add("onepass_rowp2_256x3_s2_np", &launch_onepass_rowp2<LAT, ORD, 1, 256, 3, 2, false>, 1, 256);
            add("onepass_rowp2_256x2_s2", &launch_onepass_rowp2<LAT, ORD, 1, 256, 2, 2>, 1, 256);
            add("onepass_rowp2_256x3_s2", &launch_onepass_rowp2<LAT, ORD, 1, 256, 3, 2>, 1, 256);
            add("onepass_rowp2_w256x3_s2_np", &launch_onepass_rowp2w<LAT, ORD, 1, 256, 3, 2, false>, 4, 0, 256);
            add("onepass_rowp2_w224x3_s2", &launch_onepass_rowp2w<LAT, ORD, 1, 224, 3, 2, true>, 4, 0, 224);
            add("onepass_rowp2_w208x2_s3", &launch_onepass_rowp2w<LAT, ORD, 1, 208, 2, 3, true>, 4, 0, 208);
            add("onepass_rowp2_w344x2_s2", &launch_onepass_rowp2w<LAT, ORD, 1, 344, 2, 2, true>, 4, 0, 344);
            add("onepass_rowp2_w456x1_s2", &launch_onepass_rowp2w<LAT, ORD, 1, 456, 1, 2, true>, 4, 0, 456);
        }
        // MRT in FP32, any stencil radius: the carried-density whole-row kernels
        if constexpr (COLL == 1 && std::is_same<Real, float>::value && Lattice<LAT>::reach == 1) {
            add("onepass_rowc_w256x3_s2", &launch_onepass_rowc<LAT, ORD, 1, 256, 3, 2>, 4, 0, 256, 3);
            add("onepass_rowc_w256x2_s3", &launch_onepass_rowc<LAT, ORD, 1, 256, 2, 3>, 4, 0, 256, 2);
        }
        // MRT in FP32 with the radius-2 stencil: the radius-2 whole-row kernel
        if constexpr (COLL == 1 && std::is_same<Real, float>::value && Stencil<3, ORD>::radius == 2)
            add("onepass_rowr_w256x3_s1_np", &launch_onepass_rowr<LAT, ORD, 1, 256, 3, 1, false>, 4, 0, 256);
    } else {
        add("onepass_128_z16_b2_smem", &launch_onepass<LAT, ORD, COLL, Real, 128, 1, 16, 2, 2>);
        if constexpr (hot) {
            add("onepass_256_z16_b3_smem", &launch_onepass<LAT, ORD, COLL, Real, 256, 1, 16, 3, 2>);
            if constexpr (r1) add("onepass_256_z16_b3_reg", &launch_onepass<LAT, ORD, COLL, Real, 256, 1, 16, 3, 1>);
            add("onepass_async_256_z16_b2", &launch_onepass_async<LAT, ORD, COLL, Real, 256, 1, 16, 2>);
            add("onepass_x2_256_z16_b2_smem", &launch_onepass_x2<LAT, ORD, 128, 1, 16, 2, 2>, 2);
            if constexpr (Lattice<LAT>::reach == 1) {
                add("onepass_seg256_z64_s8", &launch_onepass_seg<LAT, ORD, COLL, Real, 256, 64, 8>, 4);
                add("onepass_seg256_z64_s6", &launch_onepass_seg<LAT, ORD, COLL, Real, 256, 64, 6>, 4);
                add("onepass_seg128_z64_s8", &launch_onepass_seg<LAT, ORD, COLL, Real, 128, 64, 8>, 4);
                add("onepass_seg512_z64_s6", &launch_onepass_seg<LAT, ORD, COLL, Real, 512, 64, 6>, 4);
                add("onepass_seg2_256_z64_s6", &launch_onepass_seg2<LAT, ORD, 0, 256, 64, 6>, 4);
                add("onepass_seg2_512_z64_s6", &launch_onepass_seg2<LAT, ORD, 0, 512, 64, 6>, 4);
                if constexpr (Stencil<2, ORD>::radius <= 2)
                    add("onepass_seg2_512_z64_s4", &launch_onepass_seg2<LAT, ORD, 0, 512, 64, 4>, 4);
            }
        }
        // MRT in FP32 (D2Q9): the packed-pair segment kernels
        if constexpr (COLL == 1 && std::is_same<Real, float>::value && Lattice<LAT>::reach == 1) {
            add("onepass_seg2_256_z64_s6", &launch_onepass_seg2<LAT, ORD, 1, 256, 64, 6>, 4);
            add("onepass_seg2_512_z64_s6", &launch_onepass_seg2<LAT, ORD, 1, 512, 64, 6>, 4);
        }
    }
    return k;
}

template <int LAT, int ORD, int COLL, class Real>
KernelSet make_set()
{
    constexpr bool k3 = Lattice<LAT>::D == 3;
    constexpr int TY = k3 ? 4 : 8;
    constexpr int TZ = k3 ? 2 : 1;
    KernelSet k{};
    k.tile_x = 32;
    k.tile_y = TY;
    k.tile_z = TZ;
    k.psi = &launch_psi<LAT, Real>;
    k.fused = &launch_fused<LAT, ORD, COLL, Real, TY, TZ>;
    constexpr VariantList V = make_variants<LAT, ORD, COLL, Real>();
    static_assert(!V.overflow, "more one-pass variants than the schedule table holds: raise kMaxVariants");
    k.n_onepass = V.n;
    for (int i = 0; i < V.n; ++i) k.onepass[i] = V.v[i];
    k.obs = &launch_obs<LAT, ORD, Real>;
    k.probe = &launch_probe<LAT, Real>;
    k.fields = &launch_fields<LAT, ORD, Real>;
    k.init_profile = &launch_init_profile<LAT>;
    k.init_from_rho = &launch_init_from_rho<LAT, Real>;
    k.get_f = &launch_get_f<LAT, Real>;
    k.set_f = &launch_set_f<LAT, Real>;
    k.rho_of_f = &launch_rho_of_f<LAT>;
    if constexpr (k3 && std::is_same<Real, float>::value) k.carry_init = &launch_carry_init<LAT>;
    return k;
}

}  // namespace lbm
