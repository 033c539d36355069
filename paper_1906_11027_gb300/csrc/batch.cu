// batch.cu -- many independent 2-D D2Q9 domains (uneven sizes, each with its own
// G, tau, stencil order and initial droplet) advanced together by one persistent
// kernel per step, captured in a CUDA graph together with a per-domain steady
// check; converged domains retire and drop out of the work list.
//
// Work item = (domain, tile of TX cells along x, chunk of ZC rows along y); the
// tile width and chunk length are picked per batch by an autotuner that times
// each compiled shape on the batch's own domains (all shapes perform the same
// per-cell arithmetic, so the choice changes speed only).  Each
// item runs the one-pass march of the single-domain kernels: psi of the tile and
// its halo is formed one row ahead into a shared-memory ring, the populations
// wait in a shared-memory stash, then force (Eq. 1), Guo-forced BGK collision
// (Eqs. 3-4) and the pull-streamed store.  The item count lives in device
// memory, so a captured graph stays valid while the list shrinks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "internal.h"
#include "trace.h"
#include "kernels.cuh"

namespace lbm {
namespace {

constexpr int kBMaxR = 3;  // largest stencil radius (10th order)
constexpr int kBNS = 2 * kBMaxR + 2;
constexpr int kQ9 = 9;

struct BatchDom {
    int nx, ny, order, ntx, nch, active;
    long long off;   // element offset of the domain in each population pool
    long long poff;  // element offset of the domain in the psi scratch field (two-pass shape)
    double G, omega, pref, rho_bar;
    float G_f, omega_f, pref_f, rho_bar_f;  // FP32 copies (set with the doubles on the host)
};

__device__ __forceinline__ DevParams dom_params(const BatchDom& d)
{
    DevParams p{};
    p.nx = d.nx;
    p.ny = d.ny;
    p.nz = 1;
    p.N = static_cast<long long>(d.nx) * d.ny;
    p.G = d.G;
    p.omega = d.omega;
    p.pref = d.pref;
    p.rho_bar = d.rho_bar;
    p.G_f = d.G_f;
    p.omega_f = d.omega_f;
    p.pref_f = d.pref_f;
    p.rho_bar_f = d.rho_bar_f;
    p.psi_kind = 0;
    return p;
}

// One (tile, chunk) of one domain: the 2-D one-pass march with a shared-memory
// stash.  ring: [NS][EX] psi, stash: [R + 1][Q][TX] populations.
template <int ORD, class Real, int TX, int ZC>
__device__ void batch_item(const Real* __restrict__ A, Real* __restrict__ Bo, const DevParams& p, int x0, int m0,
                           Real* ring, Real* stash)
{
    using L = Lattice<kLatD2Q9>;
    using S = Stencil<2, ORD>;
    constexpr int R = S::radius;
    constexpr int RE = 1;
    constexpr int Q = kQ9;
    constexpr int EX = TX + 2 * R;
    constexpr int E = EX;
    constexpr int NS = 2 * R + 2;
    constexpr int NST = R + 1;
    Pops<Real, Q> P;
#pragma unroll
    for (int b = 0; b < Q; ++b) {
        P.in[b] = A + static_cast<long long>(b) * p.N;
        P.out[b] = Bo + static_cast<long long>(b) * p.N;
    }
    const int nm = p.ny;
    const int m1 = (m0 + ZC < nm) ? m0 + ZC : nm;
    const int tid = threadIdx.x;
    const int ix = x0 + tid;
    int ixo[2 * RE + 1];
    axis_offsets<RE>(wrap_any(ix, p.nx), p.nx, 1, ixo);
    const bool has_halo = tid < 2 * R;
    const int hex = (tid < R) ? tid : TX + tid;
    int hxo[2 * RE + 1];
    axis_offsets<RE>(wrap_any(x0 - R + hex, p.nx), p.nx, 1, hxo);
    const int zero[2 * RE + 1] = {};

    auto psi_slab = [&](int m) {
        int mo[2 * RE + 1];
        axis_offsets<RE>(wrap_near(m, nm), nm, p.nx, mo);
        Real* dst = ring + ring_slot(m, NS) * E;
        Real f[Q];
        gather_off<kLatD2Q9, Real, RE>(P, ixo, mo, zero, f);
        Real s = Real(0);
        sfor<Q>([&](auto bI) { s += f[decltype(bI)::value]; });
        dst[tid + R] = psi_of<kLatD2Q9>(std::is_same<Real, float>::value ? Real(p.rho_bar) + s : s, p);
        Real* st = stash + static_cast<unsigned>(m + 4 * NST) % NST * (Q * TX) + tid;
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            st[b * TX] = f[b];
        });
        if (has_halo) {
            Real h[Q];
            gather_off<kLatD2Q9, Real, RE>(P, hxo, mo, zero, h);
            Real sh = Real(0);
            sfor<Q>([&](auto bI) { sh += h[decltype(bI)::value]; });
            dst[hex] = psi_of<kLatD2Q9>(std::is_same<Real, float>::value ? Real(p.rho_bar) + sh : sh, p);
        }
    };
    for (int m = m0 - R; m < m0 + R; ++m) psi_slab(m);
    const bool active = ix < p.nx;
    for (int m = m0; m < m1; ++m) {
        psi_slab(m + R);
        __syncthreads();
        if (active) {
            Real f[Q];
            const Real* st = stash + static_cast<unsigned>(m + 4 * NST) % NST * (Q * TX) + tid;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                f[b] = st[b * TX];
            });
            Real F[3];
            force_ring<kLatD2Q9, ORD, Real, EX, E, NS>(ring, m, tid + R, 0, par<Real>(p.G, p.G_f), F);
            collide<kLatD2Q9, 0>(f, F, p);
            const int c = m * p.nx + ix;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                P.out[b][c] = f[b];
            });
        }
    }
    (void)L::Q;
}

// Persistent step kernel: every CTA walks the work list with stride gridDim.x.
template <class Real, int TX, int ZC>
__global__ void __launch_bounds__(TX) k_batch_step(const BatchDom* __restrict__ doms, const int4* __restrict__ items,
                                                   const int* __restrict__ nitems, const Real* __restrict__ pool_in,
                                                   Real* __restrict__ pool_out)
{
    __shared__ Real ring[kBNS * (TX + 2 * kBMaxR)];
    __shared__ Real stash[(kBMaxR + 1) * kQ9 * TX];
    const int n = *nitems;
    for (int it = blockIdx.x; it < n; it += gridDim.x) {
        const int4 w = items[it];
        const BatchDom d = doms[w.x];
        const DevParams p = dom_params(d);
        const Real* A = pool_in + d.off;
        Real* Bo = pool_out + d.off;
        const int x0 = w.y * TX, m0 = w.z * ZC;
        switch (d.order) {
        case 4: batch_item<4, Real, TX, ZC>(A, Bo, p, x0, m0, ring, stash); break;
        case 6: batch_item<6, Real, TX, ZC>(A, Bo, p, x0, m0, ring, stash); break;
        case 8: batch_item<8, Real, TX, ZC>(A, Bo, p, x0, m0, ring, stash); break;
        default: batch_item<10, Real, TX, ZC>(A, Bo, p, x0, m0, ring, stash); break;
        }
        __syncthreads();  // shared memory is reused by the next item
    }
}

// Segment-staged work item (FP32; nx a multiple of 4): the bulk-copy pipeline of
// the single-domain 2-D kernel.  A producer warp (threads TX .. TX + 31) copies,
// per row s and direction b, the contiguous segment of row s - c_by over
// x0 - 4 .. x0 + TX + 4 into a stage (two copies where it crosses the periodic x
// edge); the stage stays resident until the row collides.  mbarrier phases run
// on across the items a block processes.
template <int ORD, int TX, int ZC, int NSTG>
__device__ __forceinline__ void batch_item_seg(const float* __restrict__ A, float* __restrict__ Bo, const DevParams& p, int x0,
                               int m0, float* ring, float* stage, unsigned long long* bars, uint32_t& phase, bool& ok)
{
    using L = Lattice<kLatD2Q9>;
    constexpr int R = Stencil<2, ORD>::radius;
    constexpr int Q = kQ9;
    constexpr int XP = 4;
    constexpr int W = TX + 2 * XP;
    constexpr int EX = TX + 2 * R;
    constexpr int NS = 2 * R + 2;
    constexpr int STG = Q * W;
    static_assert(NSTG >= R + 2 && NSTG >= 2 * R && XP >= R + 1, "stages / pad");
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const bool producer = tid >= TX;
    const int nm = p.ny;
    const int m1 = (m0 + ZC < nm) ? m0 + ZC : nm;
    const long long N = static_cast<long long>(p.nx) * p.ny;
    int cby = 0;
    sfor<Q>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        constexpr int vy = L::T.v[b][1];
        if (lane == b) cby = vy;
    });
    const float* src_b = A + static_cast<long long>(lane < Q ? lane : 0) * N;
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
    auto stage_of = [&](int s) { return stage + ((s - base) % NSTG) * STG; };
    auto wait_stage = [&](int s) {
        const int slot = (s - base) % NSTG;
        if (ok && !mbar_wait(smem_u32(&bars[slot]), (phase >> slot) & 1u)) ok = false;  // after a timeout, stop waiting
        phase ^= 1u << slot;
    };
    auto load_cell = [&](const float* st, int cx, float (&f)[Q]) {
        sfor<Q>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int vx = L::T.v[b][0];
            f[b] = st[b * W + cx + XP - vx];
        });
    };
    auto rho_psi = [&](const float (&f)[Q]) {
        float sum = 0.f;
        sfor<Q>([&](auto bI) { sum += f[decltype(bI)::value]; });
        return psi_of<kLatD2Q9>(static_cast<float>(p.rho_bar) + sum, p);
    };
    auto psi_slab = [&](int s) {
        wait_stage(s);
        const float* st = stage_of(s);
        float* dst = ring + ring_slot(s, NS) * EX;
        float f[Q];
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
    if (producer)
        for (; next <= last && next < m0 + NSTG; ++next) issue(next);
    const bool active = !producer && (x0 + tid) < p.nx;
    for (int m = m0; m < m1; ++m) {
        if (!producer) psi_slab(m + R);
        __syncthreads();
        if (producer)
            for (; next <= last && next <= m - 1 + NSTG; ++next) issue(next);
        if (active) {
            float f[Q];
            load_cell(stage_of(m), tid, f);
            float F[3];
            force_ring<kLatD2Q9, ORD, float, EX, EX, NS>(ring, m, tid + R, 0, p.G_f, F);
            collide<kLatD2Q9, 0>(f, F, p);
            const long long c = static_cast<long long>(m) * p.nx + x0 + tid;
            sfor<Q>([&](auto bI) {
                constexpr int b = decltype(bI)::value;
                __stcs(Bo + b * N + c, f[b]);
            });
        }
    }
}

template <int TX, int ZC, int NSTG>
__global__ void __launch_bounds__(TX + 32) k_batch_step_seg(const BatchDom* __restrict__ doms,
                                                            const int4* __restrict__ items,
                                                            const int* __restrict__ nitems,
                                                            const float* __restrict__ pool_in,
                                                            float* __restrict__ pool_out, unsigned* __restrict__ err)
{
    __shared__ float ring[kBNS * (TX + 2 * kBMaxR)];
    __shared__ alignas(8) unsigned long long bars[NSTG];
    extern __shared__ __align__(128) unsigned char dyn_smem[];
    float* stage = reinterpret_cast<float*>(dyn_smem);  // [NSTG][9][TX + 8]
    if (threadIdx.x == 0) {
        for (int k = 0; k < NSTG; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    bool ok = true;
    const int n = *nitems;
    for (int it = blockIdx.x; it < n; it += gridDim.x) {
        const int4 w = items[it];
        const BatchDom d = doms[w.x];
        const DevParams p = dom_params(d);
        const float* A = pool_in + d.off;
        float* Bo = pool_out + d.off;
        const int x0 = w.y * TX, m0 = w.z * ZC;
        switch (d.order) {
        case 4: batch_item_seg<4, TX, ZC, NSTG>(A, Bo, p, x0, m0, ring, stage, bars, phase, ok); break;
        case 6: batch_item_seg<6, TX, ZC, NSTG>(A, Bo, p, x0, m0, ring, stage, bars, phase, ok); break;
        case 8: batch_item_seg<8, TX, ZC, NSTG>(A, Bo, p, x0, m0, ring, stage, bars, phase, ok); break;
        default: batch_item_seg<10, TX, ZC, NSTG>(A, Bo, p, x0, m0, ring, stage, bars, phase, ok); break;
        }
        __syncthreads();  // stages and ring are reused by the next item
    }
    if (!ok && threadIdx.x == 0) atomicOr(err, kErrTimeout);
}

// Two-pass form of the batch step, for few active cells: the march of the other
// shapes runs its rows one after another, so a step cannot finish faster than
// one item's march however little work is left.  Here a step is two launches
// with one thread per cell and no sequential loop: k_batch_psi2 writes psi of
// every active cell to a scratch field, k_batch_fused2 gathers, takes the force
// from that field (the same pair order and arithmetic as the ring kernels, so the
// results are bitwise the same) and collides.  Work item = 256 consecutive cells
// of one domain.
template <int ORD, class Real>
__device__ __forceinline__ void force_global(const Real* __restrict__ psi, int nx, int ny, int x, int y, Real G,
                                             Real (&F)[3])
{
    using L = Lattice<kLatD2Q9>;
    using S = Stencil<2, ORD>;
    Real ax = Real(0), ay = Real(0), az = Real(0);
    sfor<S::n / 2>([&](auto kI) {
        constexpr int a = 2 * decltype(kI)::value;
        constexpr int ex = S::T.v[a][0], ey = S::T.v[a][1];
        constexpr double wt = S::T.w[a] * L::cs2;
        const Real d = psi[wrap_near(y + ey, ny) * nx + wrap_near(x + ex, nx)] -
                       psi[wrap_near(y - ey, ny) * nx + wrap_near(x - ex, nx)];
        if (ex != 0) ax += Real(wt * ex) * d;
        if (ey != 0) ay += Real(wt * ey) * d;
    });
    const Real gp = -G * psi[y * nx + x];
    F[0] = gp * ax;
    F[1] = gp * ay;
    F[2] = gp * az;
}

template <class Real>
__global__ void __launch_bounds__(256) k_batch_psi2(const BatchDom* __restrict__ doms, const int4* __restrict__ items,
                                                    const int* __restrict__ nitems, const Real* __restrict__ pool_in,
                                                    Real* __restrict__ psi_pool)
{
    const int n = *nitems;
    for (int it = blockIdx.x; it < n; it += gridDim.x) {
        const int4 w = items[it];
        const BatchDom d = doms[w.x];
        const DevParams p = dom_params(d);
        const long long i = static_cast<long long>(w.y) * 256 + threadIdx.x;
        if (i >= p.N) continue;
        const int x = static_cast<int>(i % p.nx), y = static_cast<int>(i / p.nx);
        Real f[kQ9];
        gather<kLatD2Q9>(pool_in + d.off, p, x, y, 0, f);
        Real s = Real(0);
        sfor<kQ9>([&](auto bI) { s += f[decltype(bI)::value]; });
        psi_pool[d.poff + i] = psi_of<kLatD2Q9>(std::is_same<Real, float>::value ? Real(p.rho_bar) + s : s, p);
    }
}

template <int ORD, class Real>
__device__ __forceinline__ void fused2_cell(const Real* __restrict__ A, const Real* __restrict__ psi,
                                            Real* __restrict__ Bo, const DevParams& p, long long i)
{
    const int x = static_cast<int>(i % p.nx), y = static_cast<int>(i / p.nx);
    Real f[kQ9];
    gather<kLatD2Q9>(A, p, x, y, 0, f);
    Real F[3];
    force_global<ORD, Real>(psi, p.nx, p.ny, x, y, par<Real>(p.G, p.G_f), F);
    collide<kLatD2Q9, 0>(f, F, p);
    sfor<kQ9>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        Bo[static_cast<long long>(b) * p.N + i] = f[b];
    });
}

template <class Real>
__global__ void __launch_bounds__(256) k_batch_fused2(const BatchDom* __restrict__ doms,
                                                      const int4* __restrict__ items, const int* __restrict__ nitems,
                                                      const Real* __restrict__ pool_in,
                                                      const Real* __restrict__ psi_pool, Real* __restrict__ pool_out)
{
    const int n = *nitems;
    for (int it = blockIdx.x; it < n; it += gridDim.x) {
        const int4 w = items[it];
        const BatchDom d = doms[w.x];
        const DevParams p = dom_params(d);
        const long long i = static_cast<long long>(w.y) * 256 + threadIdx.x;
        if (i >= p.N) continue;
        const Real* A = pool_in + d.off;
        const Real* psi = psi_pool + d.poff;
        Real* Bo = pool_out + d.off;
        switch (d.order) {
        case 4: fused2_cell<4, Real>(A, psi, Bo, p, i); break;
        case 6: fused2_cell<6, Real>(A, psi, Bo, p, i); break;
        case 8: fused2_cell<8, Real>(A, psi, Bo, p, i); break;
        default: fused2_cell<10, Real>(A, psi, Bo, p, i); break;
        }
    }
}

// Per-cell macroscopic values of domain d at cell i (pulled populations, psi of
// the neighbourhood recomputed from the populations; used by the observables).
template <int ORD, class Real>
__device__ void batch_cell_obs(const Real* __restrict__ A, const DevParams& p, int x, int y, double& rho,
                               double (&mom)[3])
{
    using L = Lattice<kLatD2Q9>;
    using S = Stencil<2, ORD>;
    auto rho_at = [&](int xx, int yy) {
        Real f[kQ9];
        gather<kLatD2Q9>(A, p, wrap_any(xx, p.nx), wrap_any(yy, p.ny), 0, f);
        Real s = Real(0);
        sfor<kQ9>([&](auto bI) { s += f[decltype(bI)::value]; });
        return std::is_same<Real, float>::value ? Real(p.rho_bar) + s : s;
    };
    Real f[kQ9];
    gather<kLatD2Q9>(A, p, x, y, 0, f);
    double s = 0.0, j[2] = {0.0, 0.0};
    sfor<kQ9>([&](auto bI) {
        constexpr int b = decltype(bI)::value;
        constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1];
        s += static_cast<double>(f[b]);
        j[0] += static_cast<double>(f[b]) * cx;
        j[1] += static_cast<double>(f[b]) * cy;
    });
    rho = std::is_same<Real, float>::value ? p.rho_bar + s : s;
    double acc[2] = {0.0, 0.0};
    sfor<S::n>([&](auto aI) {
        constexpr int a = decltype(aI)::value;
        constexpr int ex = S::T.v[a][0], ey = S::T.v[a][1];
        constexpr double wt = S::T.w[a] * L::cs2;
        const double ps = static_cast<double>(psi_of<kLatD2Q9>(rho_at(x + ex, y + ey), p));
        acc[0] += wt * ps * ex;
        acc[1] += wt * ps * ey;
    });
    const double gp = -p.G * static_cast<double>(psi_of<kLatD2Q9>(static_cast<Real>(rho), p));
    mom[0] = j[0] + 0.5 * (gp * acc[0]);
    mom[1] = j[1] + 0.5 * (gp * acc[1]);
    mom[2] = 0.0;
}

// Per-domain observables: one block per (domain, block slice); block partials
// are written per slice and summed per domain in a fixed order by k_batch_obs_final.
constexpr int kObsSlices = 8;
template <class Real>
__global__ void __launch_bounds__(256) k_batch_obs(const BatchDom* __restrict__ doms, const Real* __restrict__ pool,
                                                   const int* __restrict__ cur_of, const long long pool_stride,
                                                   double* __restrict__ partials, int ndom, int only_active)
{
    const int d = blockIdx.x / kObsSlices, slice = blockIdx.x % kObsSlices;
    if (d >= ndom) return;
    const BatchDom dm = doms[d];
    if (only_active && !dm.active) return;  // a retired domain keeps its last observables
    const DevParams p = dom_params(dm);
    const Real* A = pool + dm.off + (cur_of[d] ? pool_stride : 0);
    double v[kObsWidth] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    for (long long i = static_cast<long long>(slice) * blockDim.x + threadIdx.x; i < p.N;
         i += static_cast<long long>(kObsSlices) * blockDim.x) {
        const int x = static_cast<int>(i % p.nx), y = static_cast<int>(i / p.nx);
        double rho, mom[3];
        switch (dm.order) {
        case 4: batch_cell_obs<4, Real>(A, p, x, y, rho, mom); break;
        case 6: batch_cell_obs<6, Real>(A, p, x, y, rho, mom); break;
        case 8: batch_cell_obs<8, Real>(A, p, x, y, rho, mom); break;
        default: batch_cell_obs<10, Real>(A, p, x, y, rho, mom); break;
        }
        const double ux = mom[0] / rho, uy = mom[1] / rho, uz = 0.0;
        const double um = sqrt(ux * ux + uy * uy + uz * uz);
        if (!isfinite(rho) || !isfinite(um)) bad = true;
        v[0] += rho;
        v[1] += mom[0];
        v[2] += mom[1];
        v[4] += um;
        v[5] = fmax(v[5], um);
    }
    if (bad) v[5] = INFINITY;  // a diverged domain reports max|u| = inf (fmax would skip NaN)
    block_reduce_obs(v, partials + static_cast<long long>(blockIdx.x) * kObsWidth);
}

// res[d*8 + 0..5] = sums (max) over the slices; 6: rho at the centre, 7: rho at node 0.
template <class Real>
__global__ void k_batch_obs_final(const BatchDom* __restrict__ doms, const Real* __restrict__ pool,
                                  const int* __restrict__ cur_of, const long long pool_stride,
                                  const double* __restrict__ partials, double* __restrict__ res, int ndom,
                                  int only_active)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndom) return;
    if (only_active && !doms[d].active) return;
    double acc[kObsWidth];
    for (int k = 0; k < kObsWidth; ++k) acc[k] = partials[static_cast<long long>(d) * kObsSlices * kObsWidth + k];
    for (int s = 1; s < kObsSlices; ++s)
        for (int k = 0; k < kObsWidth; ++k) {
            const double v = partials[(static_cast<long long>(d) * kObsSlices + s) * kObsWidth + k];
            acc[k] = (k == kObsWidth - 1) ? fmax(acc[k], v) : acc[k] + v;
        }
    for (int k = 0; k < kObsWidth; ++k) res[d * 8 + k] = acc[k];
    const BatchDom dm = doms[d];
    const DevParams p = dom_params(dm);
    const Real* A = pool + dm.off + (cur_of[d] ? pool_stride : 0);
    auto rho_at = [&](int x, int y) {
        Real f[kQ9];
        gather<kLatD2Q9>(A, p, x, y, 0, f);
        double s = 0.0;
        for (int b = 0; b < kQ9; ++b) s += static_cast<double>(f[b]);
        return std::is_same<Real, float>::value ? p.rho_bar + s : s;
    };
    res[d * 8 + 6] = rho_at(p.nx / 2, p.ny / 2);
    res[d * 8 + 7] = rho_at(0, 0);
}

template <class Real>
__global__ void k_batch_init(const BatchDom* __restrict__ doms, const double* __restrict__ init, int ndom,
                             Real* __restrict__ pool)
{
    using L = Lattice<kLatD2Q9>;
    const int d = blockIdx.y;
    if (d >= ndom) return;
    const BatchDom dm = doms[d];
    const DevParams p = dom_params(dm);
    const double rl = init[4 * d], rg = init[4 * d + 1], R = init[4 * d + 2], W = init[4 * d + 3];
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < p.N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(i % p.nx), y = static_cast<int>(i / p.nx);
        sfor<kQ9>([&](auto bI) {
            constexpr int b = decltype(bI)::value;
            constexpr int cx = L::T.v[b][0], cy = L::T.v[b][1];
            constexpr double wb = L::T.w[b];
            // A_b(y) = w_b rho0(y + c_b): the pulled state is feq(rho0, 0)
            const int xs = shift_wrap_fwd<cx>(x, p.nx), ys = shift_wrap_fwd<cy>(y, p.ny);
            const double dx = min_image(xs, p.nx), dy = min_image(ys, p.ny);
            const double r = sqrt(dx * dx + dy * dy);
            const double rho0 = 0.5 * (rl + rg) - 0.5 * (rl - rg) * tanh(2.0 * (r - R) / W);
            const double v = std::is_same<Real, float>::value ? wb * (rho0 - p.rho_bar) : wb * rho0;
            pool[dm.off + static_cast<long long>(b) * p.N + i] = static_cast<Real>(v);
        });
    }
}

__global__ void k_batch_prev_init(const BatchDom* __restrict__ doms, const double* __restrict__ res,
                                  double* __restrict__ prev, int ndom)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < ndom && doms[d].active) prev[d] = res[d * 8 + 5];
}

// Steady check after a block of K steps: retire domain d when
// |max|u|(t) - max|u|(t-K)| / K < max(tol, floor * max|u| / K).
__global__ void k_batch_check(BatchDom* __restrict__ doms, const double* __restrict__ res, double* __restrict__ prev,
                              int ndom, double tol, double floor_rel, int K, int* __restrict__ newly)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndom) return;
    if (!doms[d].active) return;
    const double u = res[d * 8 + 5];
    if (!isfinite(u)) {  // diverged: retire it, its observables stay non-finite
        doms[d].active = 0;
        atomicAdd(newly, 1);
        return;
    }
    const double thr = fmax(tol, floor_rel * u / K);
    if (prev[d] >= 0.0 && fabs(u - prev[d]) / K < thr) {
        doms[d].active = 0;
        atomicAdd(newly, 1);
    }
    prev[d] = u;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_batch {
    int n;
    int fp32;
    int device;
    cudaStream_t stream;
    bool own_stream;
    lbm_params p0;
    std::vector<BatchDom> doms;
    std::vector<double> init;
    std::vector<int> cur_of;     // buffer holding each domain's state (0: pool A)
    std::vector<int64_t> steps;  // steps each domain has taken
    std::vector<int> retired_at_check;
    long long pool_elems;
    void* pool[2];
    void* psi_pool;  // psi of every cell, for the two-pass shape
    BatchDom* d_doms;
    int4* d_items;
    int* d_nitems;
    int* d_cur_of;
    double* d_init;
    double* d_partials;
    double* d_res;
    double* d_prev;
    int* d_newly;
    int* h_newly;  // pinned
    int nitems;
    int grid;
    int cur;  // global parity: pool[cur] holds the state of active domains
    int64_t global_step;
    cudaGraphExec_t graph[2];
    int graph_k;
    int graph_cur;  // parity the graph was captured from
    unsigned* d_err;  // device error word (a bounded wait that ran out)
    unsigned* h_err;  // pinned copy, read after every graph block
    int var;        // tile shape in use (index into the variant table)
    bool tuned;     // autotuner has run, or a shape was pinned
    bool pinned;    // a shape was pinned by lbm_batch_set_schedule (never re-tuned)
    long long tuned_cells;  // active cells when the shape was last tuned
    std::vector<double> tune_ms;  // ms per step of each shape (< 0: not timed)

    void* dalloc(size_t bytes)
    {
        if (p0.dev_alloc) return p0.dev_alloc(bytes, p0.alloc_ctx);
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    void dfree(void* p)
    {
        if (!p) return;
        if (p0.dev_free)
            p0.dev_free(p, p0.alloc_ctx);
        else
            cudaFree(p);
    }
};

namespace {

// Compiled tile shapes of the batch step kernel: TX cells per tile (= threads per
// CTA) by ZC rows per work item.
struct BatchVariant {
    const char* name;
    int tx, zc;
    cudaError_t (*launch)(lbm_batch* b, int parity);
    int (*occupancy)(int fp32);
    bool staged;   // bulk-copy staging: FP32 only, every nx a multiple of 4
    bool per_cell; // two-pass shape: items are 256 consecutive cells, not (tile, row chunk)
};

template <int TX, int ZC>
cudaError_t launch_variant(lbm_batch* b, int parity)
{
    if (b->fp32)
        k_batch_step<float, TX, ZC><<<b->grid, TX, 0, b->stream>>>(
            b->d_doms, b->d_items, b->d_nitems, static_cast<const float*>(b->pool[parity]),
            static_cast<float*>(b->pool[parity ^ 1]));
    else
        k_batch_step<double, TX, ZC><<<b->grid, TX, 0, b->stream>>>(
            b->d_doms, b->d_items, b->d_nitems, static_cast<const double*>(b->pool[parity]),
            static_cast<double*>(b->pool[parity ^ 1]));
    return cudaGetLastError();
}

template <int TX, int ZC>
int occupancy_variant(int fp32)
{
    int occ = 0;
    if (fp32)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_step<float, TX, ZC>, TX, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_step<double, TX, ZC>, TX, 0);
    return occ;
}

template <int TX, int ZC, int NSTG>
constexpr size_t seg_dyn_bytes()
{
    return sizeof(float) * NSTG * kQ9 * (TX + 8);
}

template <int TX, int ZC, int NSTG>
cudaError_t launch_seg(lbm_batch* b, int parity)
{
    auto kern = &k_batch_step_seg<TX, ZC, NSTG>;
    kern<<<b->grid, TX + 32, seg_dyn_bytes<TX, ZC, NSTG>(), b->stream>>>(
        b->d_doms, b->d_items, b->d_nitems, static_cast<const float*>(b->pool[parity]),
        static_cast<float*>(b->pool[parity ^ 1]), b->d_err);
    return cudaGetLastError();
}

template <int TX, int ZC, int NSTG>
int occupancy_seg(int)
{
    auto kern = &k_batch_step_seg<TX, ZC, NSTG>;
    constexpr size_t dyn = seg_dyn_bytes<TX, ZC, NSTG>();
    // the 48 KB default covers static plus dynamic shared memory: set the limit for any request
    if (dyn > 0) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(dyn));
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, TX + 32, dyn);
    return occ;
}

cudaError_t launch_twopass(lbm_batch* b, int parity)
{
    if (b->fp32) {
        k_batch_psi2<float><<<b->grid, 256, 0, b->stream>>>(b->d_doms, b->d_items, b->d_nitems,
                                                             static_cast<const float*>(b->pool[parity]),
                                                             static_cast<float*>(b->psi_pool));
        k_batch_fused2<float><<<b->grid, 256, 0, b->stream>>>(
            b->d_doms, b->d_items, b->d_nitems, static_cast<const float*>(b->pool[parity]),
            static_cast<const float*>(b->psi_pool), static_cast<float*>(b->pool[parity ^ 1]));
    } else {
        k_batch_psi2<double><<<b->grid, 256, 0, b->stream>>>(b->d_doms, b->d_items, b->d_nitems,
                                                              static_cast<const double*>(b->pool[parity]),
                                                              static_cast<double*>(b->psi_pool));
        k_batch_fused2<double><<<b->grid, 256, 0, b->stream>>>(
            b->d_doms, b->d_items, b->d_nitems, static_cast<const double*>(b->pool[parity]),
            static_cast<const double*>(b->psi_pool), static_cast<double*>(b->pool[parity ^ 1]));
    }
    return cudaGetLastError();
}

int occupancy_twopass(int fp32)
{
    int a = 0, c = 0;
    if (fp32) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch_psi2<float>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_batch_fused2<float>, 256, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_batch_psi2<double>, 256, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_batch_fused2<double>, 256, 0);
    }
    return std::min(a, c);
}

const BatchVariant kBatchVariants[] = {
    {"tile64_rows16", 64, 16, &launch_variant<64, 16>, &occupancy_variant<64, 16>, false, false},
    {"tile32_rows16", 32, 16, &launch_variant<32, 16>, &occupancy_variant<32, 16>, false, false},
    {"tile32_rows32", 32, 32, &launch_variant<32, 32>, &occupancy_variant<32, 32>, false, false},
    {"tile64_rows8", 64, 8, &launch_variant<64, 8>, &occupancy_variant<64, 8>, false, false},
    {"tile64_rows32", 64, 32, &launch_variant<64, 32>, &occupancy_variant<64, 32>, false, false},
    {"tile128_rows16", 128, 16, &launch_variant<128, 16>, &occupancy_variant<128, 16>, false, false},
    {"tile128_rows32", 128, 32, &launch_variant<128, 32>, &occupancy_variant<128, 32>, false, false},
    {"staged64_rows32", 64, 32, &launch_seg<64, 32, 8>, &occupancy_seg<64, 32, 8>, true, false},
    {"staged128_rows32", 128, 32, &launch_seg<128, 32, 8>, &occupancy_seg<128, 32, 8>, true, false},
    {"staged128_rows64", 128, 64, &launch_seg<128, 64, 8>, &occupancy_seg<128, 64, 8>, true, false},
    {"staged256_rows64", 256, 64, &launch_seg<256, 64, 8>, &occupancy_seg<256, 64, 8>, true, false},
    {"staged64_rows1024", 64, 1024, &launch_seg<64, 1024, 8>, &occupancy_seg<64, 1024, 8>, true, false},
    {"staged128_rows1024", 128, 1024, &launch_seg<128, 1024, 8>, &occupancy_seg<128, 1024, 8>, true, false},
    {"tile32_rows8", 32, 8, &launch_variant<32, 8>, &occupancy_variant<32, 8>, false, false},
    {"twopass_cells256", 256, 1, &launch_twopass, &occupancy_twopass, false, true},
};
constexpr int kNumBatchVariants = sizeof(kBatchVariants) / sizeof(kBatchVariants[0]);
constexpr int kMinTX = 32, kMinZC = 8;  // smallest tile and chunk of the table (item buffer size)

#define LBM_BCK(call)                                                                                  \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) {                                                                       \
            char m_[256];                                                                              \
            std::snprintf(m_, sizeof(m_), "%s: %s", #call, cudaGetErrorString(e_));                    \
            return set_last_error(LBM_ECUDA, m_);                                                      \
        }                                                                                              \
    } while (0)

int rebuild_items(lbm_batch* b)
{
    const BatchVariant& v = kBatchVariants[b->var];
    std::vector<int4> items;
    for (int d = 0; d < b->n; ++d) {
        BatchDom& m = b->doms[d];
        m.ntx = (m.nx + v.tx - 1) / v.tx;
        m.nch = (m.ny + v.zc - 1) / v.zc;
        if (!m.active) continue;
        if (v.per_cell) {
            const long long nb = (static_cast<long long>(m.nx) * m.ny + 255) / 256;
            for (long long k = 0; k < nb; ++k) items.push_back(make_int4(d, static_cast<int>(k), 0, 1));
            continue;
        }
        for (int c = 0; c < m.nch; ++c)
            for (int t = 0; t < m.ntx; ++t)
                items.push_back(make_int4(d, t, c, std::min(v.zc, m.ny - c * v.zc)));  // w: rows of the item
    }
    // longest items first: the persistent blocks take them in index order
    std::stable_sort(items.begin(), items.end(), [](const int4& a, const int4& c) { return a.w > c.w; });
    b->nitems = static_cast<int>(items.size());
    if (!items.empty())
        LBM_BCK(cudaMemcpyAsync(b->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice,
                                b->stream));
    LBM_BCK(cudaMemcpyAsync(b->d_nitems, &b->nitems, sizeof(int), cudaMemcpyHostToDevice, b->stream));
    LBM_BCK(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

cudaError_t launch_step(lbm_batch* b, int parity)
{
    return kBatchVariants[b->var].launch(b, parity);
}

// Makes shape v current: persistent grid = SMs x resident CTAs, work list rebuilt,
// captured graphs dropped (they hold the previous kernel).
int select_variant(lbm_batch* b, int v)
{
    b->var = v;
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, b->device);
    b->grid = std::max(1, nsm * std::max(1, kBatchVariants[v].occupancy(b->fp32)));
    for (int k = 0; k < 2; ++k)
        if (b->graph[k]) {
            cudaGraphExecDestroy(b->graph[k]);
            b->graph[k] = nullptr;
        }
    if (int rc = rebuild_items(b)) return rc;
    // no more persistent blocks than items: the work list only shrinks until the
    // next selection, and the blocks loop over whatever it holds
    b->grid = std::max(1, std::min(b->grid, b->nitems));
    return LBM_OK;
}

// Times every shape on the batch's current state (a few steps each, from a saved
// copy that is put back afterwards, so the state does not advance) and keeps the
// fastest.  Without room for the copy the default shape stays.
int autotune(lbm_batch* b, bool again = false)
{
    if (b->tuned && !(again && !b->pinned)) return LBM_OK;
    b->tuned = true;
    // the active domains' states are saved and put back (retired ones are not stepped)
    const size_t es = b->fp32 ? 4 : 8;
    size_t bytes = 0;
    long long cells = 0;
    for (const auto& m : b->doms)
        if (m.active) {
            bytes += es * kQ9 * static_cast<size_t>(m.nx) * m.ny;
            cells += static_cast<long long>(m.nx) * m.ny;
        }
    b->tuned_cells = cells;
    if (bytes == 0) return LBM_OK;
    char* save = static_cast<char*>(b->dalloc(bytes));
    if (!save) return LBM_OK;
    auto copy_states = [&](bool to_save) {
        size_t o = 0;
        for (const auto& m : b->doms) {
            if (!m.active) continue;
            const size_t n = es * kQ9 * static_cast<size_t>(m.nx) * m.ny;
            char* pool = static_cast<char*>(b->pool[b->cur]) + es * m.off;
            cudaError_t e = to_save ? cudaMemcpyAsync(save + o, pool, n, cudaMemcpyDeviceToDevice, b->stream)
                                    : cudaMemcpyAsync(pool, save + o, n, cudaMemcpyDeviceToDevice, b->stream);
            if (e != cudaSuccess) return e;
            o += n;
        }
        return cudaSuccess;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LBM_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == LBM_OK) rc = set_last_error(LBM_ECUDA, cudaGetErrorString(e));
    };
    ck(cudaEventCreate(&e0));
    ck(cudaEventCreate(&e1));
    ck(copy_states(true));
    constexpr int kWarm = 2, kTimed = 8;
    b->tune_ms.assign(kNumBatchVariants, -1.0);
    bool nx4 = true;
    for (const auto& m : b->doms) nx4 = nx4 && m.nx % 4 == 0;
    int best = 0;
    for (int v = 0; v < kNumBatchVariants && rc == LBM_OK; ++v) {
        if (kBatchVariants[v].staged && !(b->fp32 && nx4)) continue;
        if (int r = select_variant(b, v)) {
            rc = r;
            break;
        }
        for (int i = 0; i < kWarm; ++i) ck(launch_step(b, (b->cur + i) & 1));
        ck(cudaEventRecord(e0, b->stream));
        for (int i = 0; i < kTimed; ++i) ck(launch_step(b, (b->cur + kWarm + i) & 1));
        ck(cudaEventRecord(e1, b->stream));
        ck(cudaEventSynchronize(e1));
        float ms = 0.f;
        ck(cudaEventElapsedTime(&ms, e0, e1));
        b->tune_ms[v] = ms / kTimed;
        if (b->tune_ms[v] < b->tune_ms[best]) best = v;
        ck(copy_states(false));
    }
    ck(cudaStreamSynchronize(b->stream));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->dfree(save);
    if (rc != LBM_OK) return rc;
    return select_variant(b, best);
}

// Observables into d_res (the state pointed to by d_cur_of): of every domain, or
// (only_active, inside the steady-check graph) of the domains still stepping.
cudaError_t launch_obs(lbm_batch* b, int only_active = 0)
{
    const long long stride = static_cast<const char*>(b->pool[1]) - static_cast<const char*>(b->pool[0]);
    const long long es = b->fp32 ? 4 : 8;
    if (b->fp32) {
        k_batch_obs<float><<<b->n * kObsSlices, 256, 0, b->stream>>>(
            b->d_doms, static_cast<const float*>(b->pool[0]), b->d_cur_of, stride / es, b->d_partials, b->n,
            only_active);
        k_batch_obs_final<float><<<(b->n + 63) / 64, 64, 0, b->stream>>>(
            b->d_doms, static_cast<const float*>(b->pool[0]), b->d_cur_of, stride / es, b->d_partials, b->d_res,
            b->n, only_active);
    } else {
        k_batch_obs<double><<<b->n * kObsSlices, 256, 0, b->stream>>>(
            b->d_doms, static_cast<const double*>(b->pool[0]), b->d_cur_of, stride / es, b->d_partials, b->n,
            only_active);
        k_batch_obs_final<double><<<(b->n + 63) / 64, 64, 0, b->stream>>>(
            b->d_doms, static_cast<const double*>(b->pool[0]), b->d_cur_of, stride / es, b->d_partials,
            b->d_res, b->n, only_active);
    }
    return cudaGetLastError();
}

double pressure_exp(double rho, double G)
{
    const double ps = -std::expm1(-rho);
    return rho / 3.0 + 0.5 * G / 3.0 * ps * ps;
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_params* ps, const double* init, int n, lbm_batch** out)
{
    if (!ps || !init || !out || n < 1) return set_last_error(LBM_EINVAL, "lbm_batch_create: bad argument");
    const int fp32 = ps[0].precision == LBM_FP32_SHIFTED;
    for (int d = 0; d < n; ++d) {
        const lbm_params& p = ps[d];
        const int order = p.stencil == LBM_STENCIL_LATTICE ? 4 : p.stencil;
        if (p.lattice != LBM_D2Q9 || p.psi != LBM_PSI_EXP || p.collision != LBM_BGK || p.wall_rows != 0)
            return set_last_error(LBM_EUNSUPPORTED, "lbm_batch_create: batches are D2Q9, exp psi, BGK, no wall");
        if ((p.precision == LBM_FP32_SHIFTED) != (fp32 != 0))
            return set_last_error(LBM_EINVAL, "lbm_batch_create: one precision per batch");
        if (p.nx < 8 || p.ny < 8 || p.nz != 1 || !(p.tau > 0.5) ||
            !(order == 4 || order == 6 || order == 8 || order == 10))
            return set_last_error(LBM_EINVAL, "lbm_batch_create: bad domain parameters");
        if (!(init[4 * d + 3] > 0.0) || !(init[4 * d] > 0.0) || !(init[4 * d + 1] > 0.0))
            return set_last_error(LBM_EINVAL, "lbm_batch_create: bad initial droplet");
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return set_last_error(LBM_ENOMEM, "host allocation failed");
    b->n = n;
    b->fp32 = fp32;
    b->p0 = ps[0];
    b->init.assign(init, init + 4 * n);
    b->cur_of.assign(n, 0);
    b->steps.assign(n, 0);
    cudaGetDevice(&b->device);
    if (ps[0].stream) {
        b->stream = static_cast<cudaStream_t>(ps[0].stream);
    } else {
        cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = true;
    }
    long long off = 0, poff = 0;
    b->doms.resize(n);
    for (int d = 0; d < n; ++d) {
        const lbm_params& p = ps[d];
        BatchDom& m = b->doms[d];
        m.nx = p.nx;
        m.ny = p.ny;
        m.order = p.stencil == LBM_STENCIL_LATTICE ? 4 : p.stencil;
        m.ntx = (p.nx + kMinTX - 1) / kMinTX;  // item buffer sized for the finest shape
        m.nch = (p.ny + kMinZC - 1) / kMinZC;
        m.active = 1;
        m.off = off;
        m.G = p.G;
        m.omega = 1.0 / p.tau;
        m.pref = 1.0 - 1.0 / (2.0 * p.tau);
        // FP32 deviations from the mean initial density (rectangle-rule mean of the
        // tanh droplet, computed on the host in double)
        double sum = 0.0;
        if (fp32) {
            for (int y = 0; y < p.ny; ++y)
                for (int x = 0; x < p.nx; ++x) {
                    auto mi = [](int i, int nn) {
                        double v = (double)i - (double)(nn / 2);
                        if (v > 0.5 * nn) v -= nn;
                        if (v < -0.5 * nn) v += nn;
                        return v;
                    };
                    const double dx = mi(x, p.nx), dy = mi(y, p.ny);
                    const double r = std::sqrt(dx * dx + dy * dy);
                    sum += 0.5 * (init[4 * d] + init[4 * d + 1]) -
                           0.5 * (init[4 * d] - init[4 * d + 1]) * std::tanh(2.0 * (r - init[4 * d + 2]) / init[4 * d + 3]);
                }
            m.rho_bar = sum / ((double)p.nx * p.ny);
        }
        m.G_f = static_cast<float>(m.G);
        m.omega_f = static_cast<float>(m.omega);
        m.pref_f = static_cast<float>(m.pref);
        m.rho_bar_f = static_cast<float>(m.rho_bar);
        off += (long long)kQ9 * p.nx * p.ny;
        off = (off + 63) / 64 * 64;  // 256-byte aligned domains
        m.poff = poff;
        poff += ((long long)p.nx * p.ny + 63) / 64 * 64;
    }
    b->pool_elems = off;
    const size_t es = fp32 ? 4 : 8;
    long long items = 0;
    for (auto& m : b->doms) items += (long long)m.ntx * m.nch;
    b->pool[0] = b->dalloc(es * off);
    b->pool[1] = b->dalloc(es * off);
    b->psi_pool = b->dalloc(es * poff);
    b->d_doms = static_cast<BatchDom*>(b->dalloc(sizeof(BatchDom) * n));
    b->d_items = static_cast<int4*>(b->dalloc(sizeof(int4) * items));
    b->d_nitems = static_cast<int*>(b->dalloc(256));
    b->d_cur_of = static_cast<int*>(b->dalloc(sizeof(int) * n));
    b->d_init = static_cast<double*>(b->dalloc(sizeof(double) * 4 * n));
    b->d_partials = static_cast<double*>(b->dalloc(sizeof(double) * n * kObsSlices * kObsWidth));
    b->d_res = static_cast<double*>(b->dalloc(sizeof(double) * n * 8));
    b->d_prev = static_cast<double*>(b->dalloc(sizeof(double) * n));
    b->d_newly = static_cast<int*>(b->dalloc(256));
    b->d_err = static_cast<unsigned*>(b->dalloc(256));
    if (!b->pool[0] || !b->pool[1] || !b->psi_pool || !b->d_doms || !b->d_items || !b->d_nitems || !b->d_cur_of || !b->d_init ||
        !b->d_partials || !b->d_res || !b->d_prev || !b->d_newly || !b->d_err) {
        lbm_batch_destroy(b);
        return set_last_error(LBM_ENOMEM, "lbm_batch_create: device allocation failed");
    }
    if (cudaMallocHost(&b->h_newly, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&b->h_err, sizeof(unsigned)) != cudaSuccess) {
        lbm_batch_destroy(b);
        return set_last_error(LBM_ENOMEM, "pinned host allocation failed");
    }
    int rc = LBM_OK;
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == LBM_OK) rc = set_last_error(LBM_ECUDA, cudaGetErrorString(e));
    };
    ck(cudaMemcpyAsync(b->d_doms, b->doms.data(), sizeof(BatchDom) * n, cudaMemcpyHostToDevice, b->stream));
    ck(cudaMemcpyAsync(b->d_init, init, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, b->stream));
    ck(cudaMemsetAsync(b->d_cur_of, 0, sizeof(int) * n, b->stream));
    ck(cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), b->stream));
    std::vector<double> prev(n, -1.0);
    ck(cudaMemcpyAsync(b->d_prev, prev.data(), sizeof(double) * n, cudaMemcpyHostToDevice, b->stream));
    ck(cudaMemsetAsync(b->pool[1], 0, es * off, b->stream));
    int maxp = 1;
    for (auto& m : b->doms) maxp = std::max(maxp, m.nx * m.ny);
    const dim3 g((maxp + 255) / 256 < 1024 ? (maxp + 255) / 256 : 1024, n);
    if (fp32)
        k_batch_init<float><<<g, 256, 0, b->stream>>>(b->d_doms, b->d_init, n, static_cast<float*>(b->pool[0]));
    else
        k_batch_init<double><<<g, 256, 0, b->stream>>>(b->d_doms, b->d_init, n, static_cast<double*>(b->pool[0]));
    ck(cudaGetLastError());
    if (rc == LBM_OK) rc = select_variant(b, 0);
    if (rc != LBM_OK) {
        lbm_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBM_OK;
}

int lbm_batch_destroy(lbm_batch* b)
{
    if (!b) return LBM_OK;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (int k = 0; k < 2; ++k)
        if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    b->dfree(b->pool[0]);
    b->dfree(b->pool[1]);
    b->dfree(b->psi_pool);
    b->dfree(b->d_doms);
    b->dfree(b->d_items);
    b->dfree(b->d_nitems);
    b->dfree(b->d_cur_of);
    b->dfree(b->d_init);
    b->dfree(b->d_partials);
    b->dfree(b->d_res);
    b->dfree(b->d_prev);
    b->dfree(b->d_newly);
    b->dfree(b->d_err);
    if (b->h_newly) cudaFreeHost(b->h_newly);
    if (b->h_err) cudaFreeHost(b->h_err);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return LBM_OK;
}

// Advances every active domain by n steps (no steady check).
int lbm_batch_step(lbm_batch* b, int64_t n)
{
    lbm::TraceRange trace("lbm_batch_step");
    if (!b || n < 0) return set_last_error(LBM_EINVAL, "lbm_batch_step: bad argument");
    LBM_BCK(cudaSetDevice(b->device));
    if (n > 0)
        if (int rc = autotune(b)) return rc;
    for (int64_t i = 0; i < n; ++i) {
        LBM_BCK(launch_step(b, b->cur));
        b->cur ^= 1;
    }
    b->global_step += n;
    for (int d = 0; d < b->n; ++d)
        if (b->doms[d].active) {
            b->steps[d] += n;
            b->cur_of[d] = b->cur;
        }
    LBM_BCK(cudaMemcpyAsync(b->d_cur_of, b->cur_of.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, b->stream));
    return LBM_OK;
}

int lbm_batch_run_to_steady(lbm_batch* b, double tol, int64_t max_steps, int64_t check_every,
                            int64_t* steps_per_domain, lbm_obs* obs_per_domain)
{
    lbm::TraceRange trace("lbm_batch_run_to_steady");
    if (!b || !(tol > 0.0) || max_steps < 0 || check_every < 2 || check_every % 2)
        return set_last_error(LBM_EINVAL, "lbm_batch_run_to_steady: bad argument (check_every must be even)");
    LBM_BCK(cudaSetDevice(b->device));
    if (int rc = autotune(b)) return rc;
    const int K = static_cast<int>(check_every);
    const double floor_rel = b->fp32 ? 1e-6 : 0.0;
    // one graph per starting parity is not needed: K is even, so every block of K
    // steps starts from the same parity
    auto capture = [&]() -> int {
    if (!b->graph[0] || b->graph_k != K || b->graph_cur != b->cur) {
        if (b->graph[0]) cudaGraphExecDestroy(b->graph[0]);
        b->graph[0] = nullptr;
        cudaGraph_t g = nullptr;
        LBM_BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < K && e == cudaSuccess; ++i) e = launch_step(b, (b->cur + i) & 1);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_newly, 0, sizeof(int), b->stream);
        if (e == cudaSuccess) e = launch_obs(b, 1);
        if (e == cudaSuccess) {
            k_batch_check<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->d_doms, b->d_res, b->d_prev, b->n, tol,
                                                                    floor_rel, K, b->d_newly);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_newly, b->d_newly, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_err, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return set_last_error(LBM_ECUDA, cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&b->graph[0], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return set_last_error(LBM_ECUDA, cudaGetErrorString(e));
        b->graph_k = K;
        b->graph_cur = b->cur;
    }
    return LBM_OK;
    };
    if (int rc = capture()) return rc;
    // the observables inside the graph read cur_of: active domains end each block
    // on the same parity as they started (K even)
    for (int d = 0; d < b->n; ++d)
        if (b->doms[d].active) b->cur_of[d] = b->cur;
    LBM_BCK(cudaMemcpyAsync(b->d_cur_of, b->cur_of.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, b->stream));
    // the first check compares against max|u| of the state the run starts from
    LBM_BCK(launch_obs(b));
    k_batch_prev_init<<<(b->n + 127) / 128, 128, 0, b->stream>>>(b->d_doms, b->d_res, b->d_prev, b->n);
    LBM_BCK(cudaGetLastError());
    int64_t taken = 0;
    int nactive = 0;
    for (auto& m : b->doms) nactive += m.active;
    while (nactive > 0 && taken + K <= max_steps) {
        LBM_BCK(cudaGraphLaunch(b->graph[0], b->stream));
        LBM_BCK(cudaStreamSynchronize(b->stream));
        if (*b->h_err & kErrTimeout) return set_last_error(LBM_ETIMEOUT, "a bounded device wait ran out");
        taken += K;
        b->global_step += K;
        for (int d = 0; d < b->n; ++d)
            if (b->doms[d].active) b->steps[d] += K;
        if (*b->h_newly > 0) {
            std::vector<BatchDom> dv(b->n);
            LBM_BCK(cudaMemcpy(dv.data(), b->d_doms, sizeof(BatchDom) * b->n, cudaMemcpyDeviceToHost));
            for (int d = 0; d < b->n; ++d) b->doms[d].active = dv[d].active;
            nactive = 0;
            for (auto& m : b->doms) nactive += m.active;
            if (int rc = rebuild_items(b)) return rc;
            // when the active set has shrunk eightfold, finer items may fill the GPU
            // better: time the shapes again on what is left
            long long cells = 0;
            for (const auto& m : b->doms)
                if (m.active) cells += static_cast<long long>(m.nx) * m.ny;
            if (nactive > 0 && cells * 8 < b->tuned_cells) {
                if (int rc = autotune(b, true)) return rc;
                if (int rc = capture()) return rc;
            }
        }
    }
    LBM_BCK(launch_obs(b));
    std::vector<double> res(8 * (size_t)b->n);
    LBM_BCK(cudaMemcpyAsync(res.data(), b->d_res, sizeof(double) * 8 * b->n, cudaMemcpyDeviceToHost, b->stream));
    LBM_BCK(cudaStreamSynchronize(b->stream));
    for (int d = 0; d < b->n; ++d) {
        if (steps_per_domain) steps_per_domain[d] = b->steps[d];
        if (obs_per_domain) {
            lbm_obs o{};
            const double* r = &res[8 * (size_t)d];
            const double N = (double)b->doms[d].nx * b->doms[d].ny;
            o.mass = r[0];
            o.mom[0] = r[1];
            o.mom[1] = r[2];
            o.mean_u = r[4] / N;
            o.max_u = r[5];
            o.rho_l = r[6];
            o.rho_g = r[7];
            o.dp = pressure_exp(o.rho_l, b->doms[d].G) - pressure_exp(o.rho_g, b->doms[d].G);
            o.step = b->steps[d];
            obs_per_domain[d] = o;
        }
    }
    return nactive == 0 ? LBM_OK : set_last_error(LBM_ENOTCONVERGED, "some domains still changing at max_steps");
}

int lbm_batch_schedule_report(lbm_batch* b, char* buf, int len)
{
    if (!b || !buf || len < 1) return set_last_error(LBM_EINVAL, "lbm_batch_schedule_report: bad argument");
    LBM_BCK(cudaSetDevice(b->device));
    if (int rc = autotune(b)) return rc;
    std::string s = std::string("chosen=") + kBatchVariants[b->var].name;
    for (int v = 0; v < kNumBatchVariants && v < (int)b->tune_ms.size(); ++v) {
        if (b->tune_ms[v] < 0) continue;
        char t[96];
        std::snprintf(t, sizeof(t), ";%s=%.5f", kBatchVariants[v].name, b->tune_ms[v]);
        s += t;
    }
    std::snprintf(buf, len, "%s", s.c_str());
    return LBM_OK;
}

int lbm_batch_set_schedule(lbm_batch* b, const char* name)
{
    if (!b || !name) return set_last_error(LBM_EINVAL, "lbm_batch_set_schedule: bad argument");
    LBM_BCK(cudaSetDevice(b->device));
    bool nx4 = true;
    for (const auto& m : b->doms) nx4 = nx4 && m.nx % 4 == 0;
    for (int v = 0; v < kNumBatchVariants; ++v)
        if (std::strcmp(kBatchVariants[v].name, name) == 0) {
            if (kBatchVariants[v].staged && !(b->fp32 && nx4))
                return set_last_error(LBM_EINVAL, "lbm_batch_set_schedule: staged shapes need FP32 and nx % 4 == 0");
            b->tuned = true;
            b->pinned = true;
            return select_variant(b, v);
        }
    return set_last_error(LBM_EINVAL, "lbm_batch_set_schedule: unknown tile shape");
}

// Observables of every domain in its current state.
int lbm_batch_observables(lbm_batch* b, lbm_obs* obs_per_domain)
{
    if (!b || !obs_per_domain) return set_last_error(LBM_EINVAL, "lbm_batch_observables: bad argument");
    LBM_BCK(cudaSetDevice(b->device));
    LBM_BCK(cudaMemcpyAsync(b->d_cur_of, b->cur_of.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice, b->stream));
    LBM_BCK(launch_obs(b));
    std::vector<double> res(8 * (size_t)b->n);
    LBM_BCK(cudaMemcpyAsync(res.data(), b->d_res, sizeof(double) * 8 * b->n, cudaMemcpyDeviceToHost, b->stream));
    LBM_BCK(cudaStreamSynchronize(b->stream));
    for (int d = 0; d < b->n; ++d) {
        lbm_obs o{};
        const double* r = &res[8 * (size_t)d];
        const double N = (double)b->doms[d].nx * b->doms[d].ny;
        o.mass = r[0];
        o.mom[0] = r[1];
        o.mom[1] = r[2];
        o.mean_u = r[4] / N;
        o.max_u = r[5];
        o.rho_l = r[6];
        o.rho_g = r[7];
        o.dp = pressure_exp(o.rho_l, b->doms[d].G) - pressure_exp(o.rho_g, b->doms[d].G);
        o.step = b->steps[d];
        obs_per_domain[d] = o;
    }
    return LBM_OK;
}

// Sets domain d's pre-collision populations from a double host array [9][ny][nx]
// (in the pool buffer that holds its state).
int lbm_batch_set_populations(lbm_batch* b, int d, const double* f_host)
{
    if (!b || !f_host || d < 0 || d >= b->n) return set_last_error(LBM_EINVAL, "lbm_batch_set_populations: bad argument");
    LBM_BCK(cudaSetDevice(b->device));
    const BatchDom& m = b->doms[d];
    const long long N = (long long)m.nx * m.ny;
    const size_t es = b->fp32 ? 4 : 8;
    std::vector<unsigned char> raw(es * kQ9 * N);
    static const int cx[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    static const int cy[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
    static const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    // stream on the host: A_b(y) = f_b(y + c_b)
    for (int q = 0; q < kQ9; ++q)
        for (int y = 0; y < m.ny; ++y)
            for (int x = 0; x < m.nx; ++x) {
                const int xs = (x + cx[q] + m.nx) % m.nx, ys = (y + cy[q] + m.ny) % m.ny;
                const double v = f_host[(long long)q * N + (long long)ys * m.nx + xs];
                const long long i = (long long)q * N + (long long)y * m.nx + x;
                if (b->fp32) {
                    const float fv = static_cast<float>(v - w[q] * m.rho_bar);
                    std::memcpy(&raw[4 * i], &fv, 4);
                } else {
                    std::memcpy(&raw[8 * i], &v, 8);
                }
            }
    char* dst = static_cast<char*>(b->pool[b->cur_of[d]]) + es * m.off;
    LBM_BCK(cudaMemcpyAsync(dst, raw.data(), raw.size(), cudaMemcpyHostToDevice, b->stream));
    LBM_BCK(cudaStreamSynchronize(b->stream));
    return LBM_OK;
}

// Pre-collision populations of domain d in double, [9][ny][nx].
int lbm_batch_get_populations(lbm_batch* b, int d, double* f_host)
{
    if (!b || !f_host || d < 0 || d >= b->n) return set_last_error(LBM_EINVAL, "lbm_batch_get_populations: bad argument");
    LBM_BCK(cudaSetDevice(b->device));
    const BatchDom& m = b->doms[d];
    const long long N = (long long)m.nx * m.ny;
    const size_t es = b->fp32 ? 4 : 8;
    std::vector<unsigned char> raw(es * kQ9 * N);
    const char* src = static_cast<const char*>(b->pool[b->cur_of[d]]) + es * m.off;
    LBM_BCK(cudaMemcpyAsync(raw.data(), src, raw.size(), cudaMemcpyDeviceToHost, b->stream));
    LBM_BCK(cudaStreamSynchronize(b->stream));
    // un-stream on the host: f_b(x) = A_b(x - c_b)
    static const int cx[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    static const int cy[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
    static const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    for (int q = 0; q < kQ9; ++q)
        for (int y = 0; y < m.ny; ++y)
            for (int x = 0; x < m.nx; ++x) {
                const int xs = ((x - cx[q]) % m.nx + m.nx) % m.nx, ys = ((y - cy[q]) % m.ny + m.ny) % m.ny;
                const long long i = (long long)q * N + (long long)ys * m.nx + xs;
                double v;
                if (b->fp32) {
                    float fv;
                    std::memcpy(&fv, &raw[4 * i], 4);
                    v = (double)fv + w[q] * m.rho_bar;
                } else {
                    std::memcpy(&v, &raw[8 * i], 8);
                }
                f_host[(long long)q * N + (long long)y * m.nx + x] = v;
            }
    return LBM_OK;
}

}  // extern "C"
