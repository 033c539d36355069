// lattice.cuh -- compile-time velocity sets, force stencils and MRT moment bases.
//
// Lattices (Table 1 of arXiv:1906.11027 for D2Q9, D2Q13, D2Q25; the standard
// D3Q19): velocity order = rest, shells of increasing |c|^2, inside a shell the
// vectors whose first non-zero component is positive in decreasing
// lexicographic order, each followed by its opposite.
//
// Force stencils (Sec. 2, Eq. 2): unit-normalised weights (sum w e_x^2 = 1) on
// shells of integer vectors; each set is the unique solution of the isotropy
// conditions up to its order.  The kernels multiply them by the lattice's c_s^2,
// so c_s'^2 = c_s^2; the stencil "order 0" is the lattice itself (Sec. 3).
#pragma once

#include <cstdint>
#include <utility>

namespace lbm {

// ---- compile-time loop -----------------------------------------------------
template <class F, int... I>
__host__ __device__ __forceinline__ void sfor_impl(F&& f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__host__ __device__ __forceinline__ void sfor(F&& f)
{
    sfor_impl(f, std::make_integer_sequence<int, N>{});
}

// ---- shell sets ------------------------------------------------------------
struct VecSet {
    int n;          // number of vectors
    int dim;
    int radius;     // max |component|
    int v[64][3];
    double w[64];   // weight of each vector
};

struct ShellSpec {
    int dim;
    int nshell;
    int sq[8];
    double w[8];
};

// Every integer vector of each listed |v|^2, in the order described above.
constexpr VecSet expand(const ShellSpec& s)
{
    VecSet t{};
    t.dim = s.dim;
    t.n = 0;
    t.radius = 0;
    for (int k = 0; k < s.nshell; ++k) {
        if (s.sq[k] == 0) {
            t.v[t.n][0] = 0; t.v[t.n][1] = 0; t.v[t.n][2] = 0; t.w[t.n] = s.w[k]; ++t.n;
            continue;
        }
        const int zr = (s.dim == 3) ? 3 : 0;
        for (int a = 3; a >= -3; --a)
            for (int b = 3; b >= -3; --b)
                for (int c = zr; c >= -zr; --c) {
                    if (a * a + b * b + c * c != s.sq[k]) continue;
                    const int lead = (a != 0) ? a : ((b != 0) ? b : c);
                    if (lead <= 0) continue;
                    for (int sgn = 1; sgn >= -1; sgn -= 2) {
                        t.v[t.n][0] = sgn * a; t.v[t.n][1] = sgn * b; t.v[t.n][2] = sgn * c;
                        t.w[t.n] = s.w[k];
                        const int m = (a < 0 ? -a : a) > (b < 0 ? -b : b) ? (a < 0 ? -a : a) : (b < 0 ? -b : b);
                        const int mm = m > (c < 0 ? -c : c) ? m : (c < 0 ? -c : c);
                        if (mm > t.radius) t.radius = mm;
                        ++t.n;
                    }
                }
    }
    return t;
}

// ---- lattices ----------------------------------------------------------------
constexpr ShellSpec kD2Q9 = {2, 3, {0, 1, 2}, {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0}};
constexpr ShellSpec kD2Q13 = {2, 4, {0, 1, 2, 4}, {2.0 / 5.0, 8.0 / 75.0, 1.0 / 25.0, 1.0 / 300.0}};
constexpr ShellSpec kD2Q25 = {2, 6, {0, 1, 2, 4, 5, 8},
                              {72.0 / 245.0, 16.0 / 147.0, 16.0 / 315.0, 1.0 / 105.0, 8.0 / 2205.0, 1.0 / 8820.0}};
constexpr ShellSpec kD3Q19 = {3, 3, {0, 1, 2}, {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0}};

enum LatticeId { kLatD2Q9 = 0, kLatD3Q19 = 1, kLatD2Q13 = 2, kLatD2Q25 = 3 };

template <int ID> struct Lattice;

#define LBM_DEFINE_LATTICE(ID, SPEC, QV, CS2, ORDER)                       \
    template <> struct Lattice<ID> {                                        \
        static constexpr int id = ID;                                       \
        static constexpr VecSet T = expand(SPEC);                           \
        static constexpr int Q = QV;                                        \
        static constexpr int D = SPEC.dim;                                  \
        static constexpr int reach = T.radius;                              \
        static constexpr double cs2 = CS2;                                  \
        static constexpr int iso_order = ORDER;                             \
        static_assert(T.n == QV, "lattice size");                           \
    };

LBM_DEFINE_LATTICE(kLatD2Q9, kD2Q9, 9, 1.0 / 3.0, 4)
LBM_DEFINE_LATTICE(kLatD3Q19, kD3Q19, 19, 1.0 / 3.0, 4)
LBM_DEFINE_LATTICE(kLatD2Q13, kD2Q13, 13, 2.0 / 5.0, 6)
LBM_DEFINE_LATTICE(kLatD2Q25, kD2Q25, 25, 4.0 / 7.0, 8)
#undef LBM_DEFINE_LATTICE

// ---- force stencils (unit normalised) -----------------------------------------
constexpr ShellSpec kE4_2D = {2, 2, {1, 2}, {1.0 / 3.0, 1.0 / 12.0}};
constexpr ShellSpec kE6_2D = {2, 3, {1, 2, 4}, {4.0 / 15.0, 1.0 / 10.0, 1.0 / 120.0}};
constexpr ShellSpec kE8_2D = {2, 5, {1, 2, 4, 5, 8},
                              {4.0 / 21.0, 4.0 / 45.0, 1.0 / 60.0, 2.0 / 315.0, 1.0 / 5040.0}};
constexpr ShellSpec kE10_2D = {2, 7, {1, 2, 4, 5, 8, 9, 10},
                               {262.0 / 1785.0, 93.0 / 1190.0, 7.0 / 340.0, 6.0 / 595.0, 9.0 / 9520.0,
                                2.0 / 5355.0, 1.0 / 7140.0}};
constexpr ShellSpec kE4_3D = {3, 2, {1, 2}, {1.0 / 6.0, 1.0 / 12.0}};
constexpr ShellSpec kE6_3D = {3, 4, {1, 2, 3, 4}, {2.0 / 15.0, 1.0 / 15.0, 1.0 / 60.0, 1.0 / 120.0}};

template <int DIM, int ORDER> struct Stencil;

#define LBM_DEFINE_STENCIL(DIM, ORDER, SPEC, NV)                            \
    template <> struct Stencil<DIM, ORDER> {                                \
        static constexpr VecSet T = expand(SPEC);                           \
        static constexpr int n = NV;                                        \
        static constexpr int radius = T.radius;                             \
        static constexpr int order = ORDER;                                 \
        static_assert(T.n == NV, "stencil size");                           \
    };

LBM_DEFINE_STENCIL(2, 4, kE4_2D, 8)
LBM_DEFINE_STENCIL(2, 6, kE6_2D, 12)
LBM_DEFINE_STENCIL(2, 8, kE8_2D, 24)
LBM_DEFINE_STENCIL(2, 10, kE10_2D, 36)
LBM_DEFINE_STENCIL(3, 4, kE4_3D, 18)
LBM_DEFINE_STENCIL(3, 6, kE6_3D, 32)
#undef LBM_DEFINE_STENCIL

// ---- MRT moment bases ----------------------------------------------------------
// D2Q9: orthogonal basis of Lallemand & Luo (2000); D3Q19: d'Humieres et al. (2002).
// Row k evaluated at velocity c.  Rates per row are given by mrt_rate_class().
constexpr double basis_d2q9(int k, int x, int y)
{
    const double c2 = double(x * x + y * y);
    switch (k) {
    case 0: return 1.0;
    case 1: return 3.0 * c2 - 4.0;
    case 2: return (9.0 * c2 * c2 - 21.0 * c2 + 8.0) * 0.5;
    case 3: return double(x);
    case 4: return (3.0 * c2 - 5.0) * x;
    case 5: return double(y);
    case 6: return (3.0 * c2 - 5.0) * y;
    case 7: return double(x * x - y * y);
    default: return double(x * y);
    }
}
constexpr double basis_d3q19(int k, int x, int y, int z)
{
    const double c2 = double(x * x + y * y + z * z);
    switch (k) {
    case 0: return 1.0;
    case 1: return 19.0 * c2 - 30.0;
    case 2: return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) * 0.5;
    case 3: return double(x);
    case 4: return (5.0 * c2 - 9.0) * x;
    case 5: return double(y);
    case 6: return (5.0 * c2 - 9.0) * y;
    case 7: return double(z);
    case 8: return (5.0 * c2 - 9.0) * z;
    case 9: return 3.0 * x * x - c2;
    case 10: return (3.0 * c2 - 5.0) * (3.0 * x * x - c2);
    case 11: return double(y * y - z * z);
    case 12: return (3.0 * c2 - 5.0) * (y * y - z * z);
    case 13: return double(x * y);
    case 14: return double(y * z);
    case 15: return double(x * z);
    case 16: return double((y * y - z * z) * x);
    case 17: return double((z * z - x * x) * y);
    default: return double((x * x - y * y) * z);
    }
}

// Rate class of each moment: 0 = 1/tau (conserved and stress moments),
// 1 = s_e, 2 = s_eps, 3 = s_q.
constexpr int mrt_rate_class_d2q9(int k)
{
    switch (k) {
    case 1: return 1;
    case 2: return 2;
    case 4: case 6: return 3;
    default: return 0;
    }
}
constexpr int mrt_rate_class_d3q19(int k)
{
    switch (k) {
    case 1: return 1;
    case 2: case 10: case 12: return 2;
    case 4: case 6: case 8: case 16: case 17: case 18: return 3;
    default: return 0;
    }
}

struct MrtBasis {
    double M[25][25];
    double inv_norm[25];  // 1 / sum_b M_kb^2 (rows are orthogonal, so Minv = M^T diag(inv_norm))
    int rate_class[25];
};

template <int ID>
constexpr MrtBasis make_mrt()
{
    MrtBasis m{};
    constexpr VecSet T = Lattice<ID>::T;
    for (int k = 0; k < Lattice<ID>::Q; ++k) {
        double nrm = 0.0;
        for (int b = 0; b < Lattice<ID>::Q; ++b) {
            const double v = (ID == kLatD2Q9) ? basis_d2q9(k, T.v[b][0], T.v[b][1])
                                              : basis_d3q19(k, T.v[b][0], T.v[b][1], T.v[b][2]);
            m.M[k][b] = v;
            nrm += v * v;
        }
        m.inv_norm[k] = 1.0 / nrm;
        m.rate_class[k] = (ID == kLatD2Q9) ? mrt_rate_class_d2q9(k) : mrt_rate_class_d3q19(k);
    }
    return m;
}

// Moments of the equilibrium's building blocks for each basis row k:
//   A_k = sum_b M_kb w_b,  B_ki = sum_b M_kb w_b c_bi,  C_kij = sum_b M_kb w_b c_bi c_bj,
// so that for feq_b = w_b rho (1 + c.u/cs2 + (c.u)^2/(2 cs4) - u.u/(2 cs2)) and Guo's
// source src_b = w_b [(c - u)/cs2 + (c.u) c/cs4].F (Eq. 4):
//   m_k(feq) = rho [A_k + B_k.u/cs2 + u.C_k.u/(2 cs4) - A_k u.u/(2 cs2)],
//   m_k(src) = B_k.F/cs2 - A_k u.F/cs2 + u.C_k.F/cs4.
// parity[k] = +1 if row k is even under c -> -c (M_kb equal on opposite
// velocities), -1 if odd (opposite values, zero on the rest velocity).
struct MrtMoments {
    double A[25];
    double Bv[25][3];
    double C[25][3][3];
    int parity[25];
};

template <int ID>
constexpr MrtMoments make_mrt_moments()
{
    MrtMoments t{};
    constexpr VecSet T = Lattice<ID>::T;
    constexpr int Q = Lattice<ID>::Q;
    const MrtBasis m = make_mrt<ID>();
    for (int k = 0; k < Q; ++k) {
        for (int b = 0; b < Q; ++b) {
            const double mw = m.M[k][b] * T.w[b];
            t.A[k] += mw;
            for (int i = 0; i < 3; ++i) {
                t.Bv[k][i] += mw * T.v[b][i];
                for (int j = 0; j < 3; ++j) t.C[k][i][j] += mw * T.v[b][i] * T.v[b][j];
            }
        }
        bool even = true, odd = (m.M[k][0] == 0.0);
        for (int b = 1; b + 1 < Q; b += 2) {
            even = even && (m.M[k][b] == m.M[k][b + 1]);
            odd = odd && (m.M[k][b] == -m.M[k][b + 1]);
        }
        t.parity[k] = even ? 1 : (odd ? -1 : 0);
    }
    return t;
}

template <int ID> struct Mrt {
    static constexpr MrtBasis B = make_mrt<ID>();
    static constexpr MrtMoments T = make_mrt_moments<ID>();
};

}  // namespace lbm
