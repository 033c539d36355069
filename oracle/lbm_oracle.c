/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of the Shan-Chen pseudo-potential
 * multiphase lattice Boltzmann step studied in Peng, Ayala, Ayala & Wang,
 * "Isotropy and spurious currents in pseudo-potential multiphase lattice
 * Boltzmann models" (arXiv:1906.11027).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's CPU
 * baseline are the only users.  The GPU library never includes, links or calls
 * this file, and this file takes no table, constant or helper from it.
 *
 * State at step n: the pre-collision populations f_b(x, n) on a periodic box,
 * dt = dx = 1.  One step n -> n+1, in the paper's order:
 *   rho(x) = sum_b f_b(x)
 *   psi(x) = psi(rho(x))          1 - exp(-rho)  or the Peng-Robinson form (Sec. 3)
 *   F(x)   = -G psi(x) sum_a w_a psi(x + e_a) e_a                        (Eq. 1)
 *   u(x)   = (sum_b f_b c_b + F/2) / rho          (Guo's half-force velocity, Eq. 4)
 *   f*_b   = f_b - (f_b - feq_b)/tau + phi_b                       (Eqs. 3-4, BGK)
 *            or the moment-space (MRT) collision with the same feq and phi,
 *            or BGK with the exact-difference forcing the paper's runs use (Sec. 3):
 *            f*_b = f_b - (f_b - feq_b(rho, u'))/tau + feq_b(rho, u' + F/rho) - feq_b(rho, u'),
 *            u' = sum_b f_b c_b / rho (the physical velocity is still u' + F/(2 rho))
 *   f_b(x + c_b, n+1) = f*_b(x)                                    (Eq. 3, stream)
 *
 * Optional wall (Sec. 3, Fig. 6; or_set_wall): the rows y < wall_rows are solid.
 * A solid node takes no collision; it sends every population back the way it
 * came, f*_b = f_{-b} (standard, full-way bounce-back), and in Eq. 1 it carries
 * psi(rho_w), the wall's virtual density, which sets the wettability.
 *
 * Readings of the paper used here (each is also listed in the design notes):
 *  - Force weights w_a are stored unit-normalised (sum_a w_a e_ax^2 = 1) and are
 *    multiplied by the lattice's c_s^2, so c_s'^2 = c_s^2 on every lattice and
 *    the critical coupling of psi = 1 - exp(-rho) is G_c = -4 everywhere.
 *  - c_s^2 = sum_b w_b c_bi c_bi is read per component (no sum over i).
 *  - Initial populations are feq(rho0, u = 0).
 *  - MRT (not defined in the paper) uses m_eq := M feq and Guo's source in
 *    moment space, m* = m - S(m - m_eq) + (I - S/2) M phi~.
 *
 * Everything is double precision; build with -ffp-contract=off so no fused
 * multiply-add changes the rounding.  Per-cell work is independent, so the
 * optional OpenMP loops give results independent of the thread count;
 * reductions are serial, in index order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXQ 25
#define OR_MAXE 64

enum { OR_D2Q9 = 0, OR_D3Q19 = 1, OR_D2Q13 = 2, OR_D2Q25 = 3 };
enum { OR_PSI_EXP = 0, OR_PSI_PR = 1 };
enum { OR_BGK = 0, OR_MRT = 1, OR_EDM = 2 };

/* ------------------------------------------------------------------------ */
/* Shell tables: a velocity set or force stencil is every integer vector whose
 * squared length is one of the listed shells, weighted by the shell's weight. */

typedef struct {
    int dim;
    int nshell;
    int sq[8];     /* |c|^2 of each shell */
    double w[8];   /* weight of every vector of that shell */
} shell_set;

/* Table 1 of the paper: D2Q9, D2Q13, D2Q25, weights indexed by |c|^2. */
static shell_set lattice_shells(int lattice, double* cs2)
{
    shell_set s;
    memset(&s, 0, sizeof(s));
    switch (lattice) {
    case OR_D2Q9:
        s.dim = 2; s.nshell = 3;
        s.sq[0] = 0; s.w[0] = 4.0 / 9.0;
        s.sq[1] = 1; s.w[1] = 1.0 / 9.0;
        s.sq[2] = 2; s.w[2] = 1.0 / 36.0;
        *cs2 = 1.0 / 3.0;
        break;
    case OR_D2Q13:
        s.dim = 2; s.nshell = 4;
        s.sq[0] = 0; s.w[0] = 2.0 / 5.0;
        s.sq[1] = 1; s.w[1] = 8.0 / 75.0;
        s.sq[2] = 2; s.w[2] = 1.0 / 25.0;
        s.sq[3] = 4; s.w[3] = 1.0 / 300.0;
        *cs2 = 2.0 / 5.0;
        break;
    case OR_D2Q25:
        s.dim = 2; s.nshell = 6;
        s.sq[0] = 0; s.w[0] = 72.0 / 245.0;
        s.sq[1] = 1; s.w[1] = 16.0 / 147.0;
        s.sq[2] = 2; s.w[2] = 16.0 / 315.0;
        s.sq[3] = 4; s.w[3] = 1.0 / 105.0;
        s.sq[4] = 5; s.w[4] = 8.0 / 2205.0;
        s.sq[5] = 8; s.w[5] = 1.0 / 8820.0;
        *cs2 = 4.0 / 7.0;
        break;
    default: /* OR_D3Q19: the standard 3-D nearest-neighbour lattice */
        s.dim = 3; s.nshell = 3;
        s.sq[0] = 0; s.w[0] = 1.0 / 3.0;
        s.sq[1] = 1; s.w[1] = 1.0 / 18.0;
        s.sq[2] = 2; s.w[2] = 1.0 / 36.0;
        *cs2 = 1.0 / 3.0;
        break;
    }
    return s;
}

/* Unit-normalised isotropic force stencils (sum w e_x^2 = 1).  2-D orders 4, 6,
 * 8, 10 and 3-D orders 4, 6, each the unique solution of the isotropy
 * conditions on its shells (Sec. 2, Eq. 2).  Returns 0 if the pair is unknown. */
static int stencil_shells(int dim, int order, shell_set* s)
{
    memset(s, 0, sizeof(*s));
    s->dim = dim;
    if (dim == 2 && order == 4) {
        s->nshell = 2;
        s->sq[0] = 1; s->w[0] = 1.0 / 3.0;
        s->sq[1] = 2; s->w[1] = 1.0 / 12.0;
    } else if (dim == 2 && order == 6) {
        s->nshell = 3;
        s->sq[0] = 1; s->w[0] = 4.0 / 15.0;
        s->sq[1] = 2; s->w[1] = 1.0 / 10.0;
        s->sq[2] = 4; s->w[2] = 1.0 / 120.0;
    } else if (dim == 2 && order == 8) {
        s->nshell = 5;
        s->sq[0] = 1; s->w[0] = 4.0 / 21.0;
        s->sq[1] = 2; s->w[1] = 4.0 / 45.0;
        s->sq[2] = 4; s->w[2] = 1.0 / 60.0;
        s->sq[3] = 5; s->w[3] = 2.0 / 315.0;
        s->sq[4] = 8; s->w[4] = 1.0 / 5040.0;
    } else if (dim == 2 && order == 10) {
        s->nshell = 7;
        s->sq[0] = 1;  s->w[0] = 262.0 / 1785.0;
        s->sq[1] = 2;  s->w[1] = 93.0 / 1190.0;
        s->sq[2] = 4;  s->w[2] = 7.0 / 340.0;
        s->sq[3] = 5;  s->w[3] = 6.0 / 595.0;
        s->sq[4] = 8;  s->w[4] = 9.0 / 9520.0;
        s->sq[5] = 9;  s->w[5] = 2.0 / 5355.0;
        s->sq[6] = 10; s->w[6] = 1.0 / 7140.0;
    } else if (dim == 3 && order == 4) {
        s->nshell = 2;
        s->sq[0] = 1; s->w[0] = 1.0 / 6.0;
        s->sq[1] = 2; s->w[1] = 1.0 / 12.0;
    } else if (dim == 3 && order == 6) {
        s->nshell = 4;
        s->sq[0] = 1; s->w[0] = 2.0 / 15.0;
        s->sq[1] = 2; s->w[1] = 1.0 / 15.0;
        s->sq[2] = 3; s->w[2] = 1.0 / 60.0;
        s->sq[3] = 4; s->w[3] = 1.0 / 120.0;
    } else {
        return 0;
    }
    return 1;
}

/* Expand a shell set into vectors.  Order: shells by increasing |c|^2; inside
 * a shell, the vectors whose first non-zero component is positive in
 * decreasing lexicographic order, each followed by its opposite. */
static int expand_shells(const shell_set* s, int c[][3], double* w)
{
    int n = 0;
    for (int k = 0; k < s->nshell; ++k) {
        if (s->sq[k] == 0) {
            c[n][0] = c[n][1] = c[n][2] = 0; w[n] = s->w[k]; ++n;
            continue;
        }
        int zr = (s->dim == 3) ? 3 : 0;
        for (int a = 3; a >= -3; --a)
            for (int b = 3; b >= -3; --b)
                for (int d = zr; d >= -zr; --d) {
                    if (a * a + b * b + d * d != s->sq[k]) continue;
                    int first = (a != 0) ? a : ((b != 0) ? b : d);
                    if (first <= 0) continue;
                    c[n][0] = a; c[n][1] = b; c[n][2] = d; w[n] = s->w[k]; ++n;
                    c[n][0] = -a; c[n][1] = -b; c[n][2] = -d; w[n] = s->w[k]; ++n;
                }
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Peng-Robinson equation of state (Sec. 3): a = 2/49, b = 2/21, R = 1,
 * omega = 0.344, alpha(T) = [1 + k (1 - sqrt(T/Tc))]^2. */

static const double PR_A = 2.0 / 49.0;
static const double PR_B = 2.0 / 21.0;
static const double PR_R = 1.0;
static const double PR_OMEGA = 0.344;

static double pr_p(double rho, double T, double alpha)
{
    return rho * PR_R * T / (1.0 - PR_B * rho)
         - PR_A * alpha * rho * rho / (1.0 + 2.0 * PR_B * rho - PR_B * PR_B * rho * rho);
}

/* Critical temperature of the printed EOS with alpha = 1: the point where
 * dp/drho = d2p/drho2 = 0 (the paper does not print T_c).  The derivatives are
 * written out from the EOS:
 *   D      = 1 + 2 b rho - b^2 rho^2
 *   dp     = R T / (1 - b rho)^2 - 2 a rho (1 + b rho) / D^2
 *   d2p    = 2 b R T / (1 - b rho)^3
 *            - a [ (2 + 4 b rho) D - 8 b rho (1 + b rho)(1 - b rho) ] / D^3
 * For a trial T the density where d2p = 0 is found by bisection, and T is
 * bisected on the sign of dp there (negative below T_c). */
static double pr_d1(double rho, double T)
{
    double D = 1.0 + 2.0 * PR_B * rho - PR_B * PR_B * rho * rho;
    double q = 1.0 - PR_B * rho;
    return PR_R * T / (q * q) - 2.0 * PR_A * rho * (1.0 + PR_B * rho) / (D * D);
}
static double pr_d2(double rho, double T)
{
    double D = 1.0 + 2.0 * PR_B * rho - PR_B * PR_B * rho * rho;
    double q = 1.0 - PR_B * rho;
    return 2.0 * PR_B * PR_R * T / (q * q * q)
         - PR_A * ((2.0 + 4.0 * PR_B * rho) * D - 8.0 * PR_B * rho * (1.0 + PR_B * rho) * q) / (D * D * D);
}
static double pr_min_slope(double T)
{
    /* d2p < 0 below the inflection density and > 0 above it, for rho in (0.5, 8). */
    double lo = 0.5, hi = 8.0;
    for (int i = 0; i < 200; ++i) {
        double mid = 0.5 * (lo + hi);
        if (pr_d2(mid, T) < 0.0) lo = mid; else hi = mid;
    }
    return pr_d1(0.5 * (lo + hi), T);
}
double or_pr_critical_T(void)
{
    double lo = 0.05, hi = 0.1;
    for (int i = 0; i < 200; ++i) {
        double mid = 0.5 * (lo + hi);
        if (pr_min_slope(mid) < 0.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

double or_pr_alpha(double T_over_Tc)
{
    double k = 0.37464 + 1.54226 * PR_OMEGA - 0.26992 * PR_OMEGA * PR_OMEGA;
    double t = 1.0 + k * (1.0 - sqrt(T_over_Tc));
    return t * t;
}

double or_pr_pressure(double rho, double T_over_Tc, double Tc)
{
    return pr_p(rho, T_over_Tc * Tc, or_pr_alpha(T_over_Tc));
}

/* ------------------------------------------------------------------------ */

typedef struct {
    int nx, ny, nz, N, dim;
    int lattice, Q;
    int c[OR_MAXQ][3];
    double w[OR_MAXQ];
    double cs2;
    int ne;                 /* force stencil size */
    int e[OR_MAXE][3];
    double we[OR_MAXE];     /* scaled force weights: c_s^2 * unit weight */
    double cs2p;            /* c_s'^2 = sum_a we_a e_ax^2 */
    int psi_kind;
    double T_over_Tc, Tc, pr_alpha;
    double G, tau;
    int coll;
    double srate[OR_MAXQ];  /* MRT relaxation rate of each moment */
    double M[OR_MAXQ][OR_MAXQ], Minv[OR_MAXQ][OR_MAXQ];
    double *f, *ftmp, *rho, *psi;
    int64_t step;
    int wall_rows;          /* rows y < wall_rows are solid; 0 = no wall */
    double rho_w, psi_w;    /* the wall's virtual density and its psi */
    int opp[OR_MAXQ];       /* c_opp[b] = -c_b */
} or_sim;

/* ---- moment basis for MRT --------------------------------------------- */

/* D2Q9: orthogonal polynomial basis of Lallemand & Luo (2000), row k is the
 * polynomial evaluated at each c_b:
 *   1, 3|c|^2-4, (9|c|^4-21|c|^2+8)/2, cx, (3|c|^2-5)cx, cy, (3|c|^2-5)cy,
 *   cx^2-cy^2, cx cy.
 * D3Q19: the basis of d'Humieres et al. (2002):
 *   1, 19|c|^2-30, (21|c|^4-53|c|^2+24)/2, cx, (5|c|^2-9)cx, cy, (5|c|^2-9)cy,
 *   cz, (5|c|^2-9)cz, 3cx^2-|c|^2, (3|c|^2-5)(3cx^2-|c|^2), cy^2-cz^2,
 *   (3|c|^2-5)(cy^2-cz^2), cx cy, cy cz, cx cz, (cy^2-cz^2)cx, (cz^2-cx^2)cy,
 *   (cx^2-cy^2)cz. */
static double basis_row(int lattice, int k, const int* cv)
{
    double x = cv[0], y = cv[1], z = cv[2];
    double c2 = x * x + y * y + z * z;
    if (lattice == OR_D2Q9) {
        switch (k) {
        case 0: return 1.0;
        case 1: return 3.0 * c2 - 4.0;
        case 2: return (9.0 * c2 * c2 - 21.0 * c2 + 8.0) / 2.0;
        case 3: return x;
        case 4: return (3.0 * c2 - 5.0) * x;
        case 5: return y;
        case 6: return (3.0 * c2 - 5.0) * y;
        case 7: return x * x - y * y;
        default: return x * y;
        }
    }
    switch (k) {
    case 0: return 1.0;
    case 1: return 19.0 * c2 - 30.0;
    case 2: return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
    case 3: return x;
    case 4: return (5.0 * c2 - 9.0) * x;
    case 5: return y;
    case 6: return (5.0 * c2 - 9.0) * y;
    case 7: return z;
    case 8: return (5.0 * c2 - 9.0) * z;
    case 9: return 3.0 * x * x - c2;
    case 10: return (3.0 * c2 - 5.0) * (3.0 * x * x - c2);
    case 11: return y * y - z * z;
    case 12: return (3.0 * c2 - 5.0) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return (y * y - z * z) * x;
    case 17: return (z * z - x * x) * y;
    default: return (x * x - y * y) * z;
    }
}

/* Plain Gauss-Jordan inverse with partial pivoting. Returns 0 if singular. */
static int invert(int n, double A[][OR_MAXQ], double Ainv[][OR_MAXQ])
{
    double a[OR_MAXQ][2 * OR_MAXQ];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j)
            a[i][j] = (j < n) ? A[i][j] : ((j - n == i) ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return 0;
        if (piv != col)
            for (int j = 0; j < 2 * n; ++j) { double t = a[col][j]; a[col][j] = a[piv][j]; a[piv][j] = t; }
        double d = a[col][col];
        for (int j = 0; j < 2 * n; ++j) a[col][j] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            if (m == 0.0) continue;
            for (int j = 0; j < 2 * n; ++j) a[r][j] -= m * a[col][j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i][j] = a[i][j + n];
    return 1;
}

/* ---- creation ------------------------------------------------------------ */

/* stencil_order 0 selects the lattice itself as the force stencil (the
 * "consistent implementation" of Sec. 3): order 4 for D2Q9/D3Q19, 6 for D2Q13,
 * 8 for D2Q25.  mrt_rates: for D2Q9 (s_e, s_eps, s_q); for D3Q19 the same three
 * are applied to the energy, the fourth-order (eps and pi) and the
 * third-order (q and m) moments.  Returns NULL on an unsupported combination. */
or_sim* or_create(int lattice, int nx, int ny, int nz, int stencil_order, int psi_kind,
                  double T_over_Tc, double G, double tau, int coll,
                  double s_e, double s_eps, double s_q)
{
    if (lattice < 0 || lattice > 3 || nx < 1 || ny < 1 || nz < 1 || !(tau > 0.5)) return NULL;
    if (coll < OR_BGK || coll > OR_EDM) return NULL;
    or_sim* s = (or_sim*)calloc(1, sizeof(or_sim));
    s->lattice = lattice;
    shell_set ls = lattice_shells(lattice, &s->cs2);
    s->dim = ls.dim;
    s->Q = expand_shells(&ls, s->c, s->w);
    if (s->dim == 2) nz = 1;
    s->nx = nx; s->ny = ny; s->nz = nz; s->N = nx * ny * nz;
    int order = stencil_order;
    if (order == 0) order = (lattice == OR_D2Q13) ? 6 : ((lattice == OR_D2Q25) ? 8 : 4);
    shell_set es;
    if (!stencil_shells(s->dim, order, &es)) { free(s); return NULL; }
    double wunit[OR_MAXE];
    s->ne = expand_shells(&es, s->e, wunit);
    s->cs2p = 0.0;
    for (int a = 0; a < s->ne; ++a) {
        s->we[a] = s->cs2 * wunit[a];
        s->cs2p += s->we[a] * s->e[a][0] * s->e[a][0];
    }
    s->psi_kind = psi_kind;
    s->T_over_Tc = T_over_Tc;
    s->G = G; s->tau = tau; s->coll = coll;
    if (psi_kind == OR_PSI_PR) {
        s->Tc = or_pr_critical_T();
        s->pr_alpha = or_pr_alpha(T_over_Tc);
    }
    if (coll == OR_MRT) {
        if (lattice != OR_D2Q9 && lattice != OR_D3Q19) { free(s); return NULL; }
        for (int k = 0; k < s->Q; ++k)
            for (int b = 0; b < s->Q; ++b) s->M[k][b] = basis_row(lattice, k, s->c[b]);
        if (!invert(s->Q, s->M, s->Minv)) { free(s); return NULL; }
        double st = 1.0 / tau;
        if (lattice == OR_D2Q9) {
            double r[9] = { st, s_e, s_eps, st, s_q, st, s_q, st, st };
            for (int k = 0; k < 9; ++k) s->srate[k] = r[k];
        } else {
            double r[19] = { st, s_e, s_eps, st, s_q, st, s_q, st, s_q,
                             st, s_eps, st, s_eps, st, st, st, s_q, s_q, s_q };
            for (int k = 0; k < 19; ++k) s->srate[k] = r[k];
        }
    }
    s->f = (double*)calloc((size_t)s->Q * s->N, sizeof(double));
    s->ftmp = (double*)calloc((size_t)s->Q * s->N, sizeof(double));
    s->rho = (double*)calloc((size_t)s->N, sizeof(double));
    s->psi = (double*)calloc((size_t)s->N, sizeof(double));
    if (!s->f || !s->ftmp || !s->rho || !s->psi) {
        free(s->f); free(s->ftmp); free(s->rho); free(s->psi); free(s); return NULL;
    }
    return s;
}

void or_destroy(or_sim* s)
{
    if (!s) return;
    free(s->f); free(s->ftmp); free(s->rho); free(s->psi); free(s);
}

/* ---- tables (for the tests) ---------------------------------------------- */

int or_lattice_table(int lattice, int* c /* 25*3 */, double* w /* 25 */, double* cs2)
{
    int cc[OR_MAXQ][3];
    shell_set ls = lattice_shells(lattice, cs2);
    int q = expand_shells(&ls, cc, w);
    for (int b = 0; b < q; ++b) for (int i = 0; i < 3; ++i) c[3 * b + i] = cc[b][i];
    return q;
}

/* Unit-normalised stencil; returns the number of vectors or 0. */
int or_stencil_table(int dim, int order, int* e /* 64*3 */, double* w /* 64 */)
{
    shell_set es;
    int ee[OR_MAXE][3];
    if (!stencil_shells(dim, order, &es)) return 0;
    int n = expand_shells(&es, ee, w);
    for (int a = 0; a < n; ++a) for (int i = 0; i < 3; ++i) e[3 * a + i] = ee[a][i];
    return n;
}

int or_Q(const or_sim* s) { return s->Q; }
int or_N(const or_sim* s) { return s->N; }
double or_cs2(const or_sim* s) { return s->cs2; }
double or_cs2p(const or_sim* s) { return s->cs2p; }
int64_t or_step_count(const or_sim* s) { return s->step; }
int or_mrt_matrix(const or_sim* s, double* M, double* Minv)
{
    for (int k = 0; k < s->Q; ++k)
        for (int b = 0; b < s->Q; ++b) { M[k * s->Q + b] = s->M[k][b]; Minv[k * s->Q + b] = s->Minv[k][b]; }
    return s->Q;
}

/* ---- the pieces of the method -------------------------------------------- */

static int wrap(int i, int n)
{
    int r = i % n;
    return (r < 0) ? r + n : r;
}

static size_t cell_index(const or_sim* s, int x, int y, int z)
{
    return ((size_t)z * s->ny + y) * s->nx + x;
}

/* psi(rho): 1 - exp(-rho) (original Shan-Chen potential), evaluated as
 * -expm1(-rho); or psi = sqrt(2 (p_EOS - c_s^2 rho) / (G c_s'^2)) (Sec. 3). */
double or_psi_of_rho(const or_sim* s, double rho)
{
    if (s->psi_kind == OR_PSI_EXP) return -expm1(-rho);
    double p = pr_p(rho, s->T_over_Tc * s->Tc, s->pr_alpha);
    return sqrt(2.0 * (p - s->cs2 * rho) / (s->G * s->cs2p));
}

/* Bulk pressure: c_s^2 rho + (G c_s'^2 / 2) psi^2, which for the P-R potential
 * is exactly the EOS pressure. */
double or_pressure(const or_sim* s, double rho)
{
    if (s->psi_kind == OR_PSI_PR) return pr_p(rho, s->T_over_Tc * s->Tc, s->pr_alpha);
    double psi = or_psi_of_rho(s, rho);
    return s->cs2 * rho + 0.5 * s->G * s->cs2p * psi * psi;
}

/* Eq. 1 at one node, from a psi field. */
static void force_at(const or_sim* s, const double* psi, int x, int y, int z, double F[3])
{
    double acc[3] = { 0.0, 0.0, 0.0 };
    for (int a = 0; a < s->ne; ++a) {
        int xn = wrap(x + s->e[a][0], s->nx);
        int yn = wrap(y + s->e[a][1], s->ny);
        int zn = wrap(z + s->e[a][2], s->nz);
        double wp = s->we[a] * psi[cell_index(s, xn, yn, zn)];
        for (int i = 0; i < 3; ++i) acc[i] += wp * s->e[a][i];
    }
    double p0 = psi[cell_index(s, x, y, z)];
    for (int i = 0; i < 3; ++i) F[i] = -s->G * p0 * acc[i];
}

/* Force field of an arbitrary psi field (N values, x fastest) -> F (3N, xyz per cell). */
void or_force_field(const or_sim* s, const double* psi, double* F)
{
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) force_at(s, psi, x, y, z, &F[3 * cell_index(s, x, y, z)]);
}

/* Eq. 4: equilibrium. */
static double feq_b(const or_sim* s, int b, double rho, const double u[3])
{
    double cu = s->c[b][0] * u[0] + s->c[b][1] * u[1] + s->c[b][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return rho * s->w[b] * (1.0 + cu / s->cs2 + (cu * cu) / (2.0 * s->cs2 * s->cs2) - uu / (2.0 * s->cs2));
}

/* Eq. 4: Guo's source without the (1 - 1/(2 tau)) prefactor,
 * w_b [ (c_b - u)/c_s^2 + (c_b . u) c_b / c_s^4 ] . F */
static double guo_b(const or_sim* s, int b, const double u[3], const double F[3])
{
    double cu = s->c[b][0] * u[0] + s->c[b][1] * u[1] + s->c[b][2] * u[2];
    double sum = 0.0;
    for (int i = 0; i < 3; ++i)
        sum += ((s->c[b][i] - u[i]) / s->cs2 + cu * s->c[b][i] / (s->cs2 * s->cs2)) * F[i];
    return s->w[b] * sum;
}

/* The collision at one node: populations fin (pre-collision), force F ->
 * fout (post-collision).  Also returns rho and u if asked. */
void or_collide_cell(const or_sim* s, const double* fin, const double F[3], double* fout,
                     double* rho_out, double* u_out)
{
    double rho = 0.0, j[3] = { 0.0, 0.0, 0.0 };
    for (int b = 0; b < s->Q; ++b) {
        rho += fin[b];
        for (int i = 0; i < 3; ++i) j[i] += fin[b] * s->c[b][i];
    }
    double u[3];
    for (int i = 0; i < 3; ++i) u[i] = (j[i] + 0.5 * F[i]) / rho;
    double feq[OR_MAXQ], src[OR_MAXQ];
    for (int b = 0; b < s->Q; ++b) {
        feq[b] = feq_b(s, b, rho, u);
        src[b] = guo_b(s, b, u, F);
    }
    if (s->coll == OR_BGK) {
        double pref = 1.0 - 1.0 / (2.0 * s->tau);
        for (int b = 0; b < s->Q; ++b)
            fout[b] = fin[b] - (fin[b] - feq[b]) / s->tau + pref * src[b];
    } else if (s->coll == OR_EDM) {
        /* exact difference: relax towards feq at the force-free velocity u', then
         * add the change of feq that the velocity increment F/rho makes */
        double up[3], uv[3];
        for (int i = 0; i < 3; ++i) {
            up[i] = j[i] / rho;
            uv[i] = up[i] + F[i] / rho;
        }
        for (int b = 0; b < s->Q; ++b) {
            double e0 = feq_b(s, b, rho, up);
            double e1 = feq_b(s, b, rho, uv);
            fout[b] = fin[b] - (fin[b] - e0) / s->tau + (e1 - e0);
        }
    } else {
        double m[OR_MAXQ], meq[OR_MAXQ], ms[OR_MAXQ], mpost[OR_MAXQ];
        for (int k = 0; k < s->Q; ++k) {
            m[k] = meq[k] = ms[k] = 0.0;
            for (int b = 0; b < s->Q; ++b) {
                m[k] += s->M[k][b] * fin[b];
                meq[k] += s->M[k][b] * feq[b];
                ms[k] += s->M[k][b] * src[b];
            }
            mpost[k] = m[k] - s->srate[k] * (m[k] - meq[k]) + (1.0 - 0.5 * s->srate[k]) * ms[k];
        }
        for (int b = 0; b < s->Q; ++b) {
            fout[b] = 0.0;
            for (int k = 0; k < s->Q; ++k) fout[b] += s->Minv[b][k] * mpost[k];
        }
    }
    if (rho_out) *rho_out = rho;
    if (u_out) for (int i = 0; i < 3; ++i) u_out[i] = u[i];
}

static int is_solid(const or_sim* s, int y) { return y < s->wall_rows; }

static void update_rho_psi(or_sim* s)
{
    #pragma omp parallel for schedule(static)
    for (int n = 0; n < s->N; ++n) {
        double r = 0.0;
        for (int b = 0; b < s->Q; ++b) r += s->f[(size_t)b * s->N + n];
        s->rho[n] = r;
        s->psi[n] = is_solid(s, (n / s->nx) % s->ny) ? s->psi_w : or_psi_of_rho(s, r);
    }
}

/* Solid band y < rows with virtual wall density rho_w (Sec. 3, Fig. 6).  The
 * box stays periodic in y, so the band is the floor of the fluid and the
 * ceiling of its periodic image: it must be at least as thick as the lattice's
 * reach and the force stencil's radius so that no population and no term of
 * Eq. 1 crosses it, and it must leave fluid rows.  Returns 1, or 0 (nothing
 * changed) for a band that breaks these rules or a psi(rho_w) that is not
 * finite. */
int or_set_wall(or_sim* s, int rows, double rho_w)
{
    int reach = 0, radius = 0;
    for (int b = 0; b < s->Q; ++b)
        for (int i = 0; i < 3; ++i) reach = abs(s->c[b][i]) > reach ? abs(s->c[b][i]) : reach;
    for (int a = 0; a < s->ne; ++a)
        for (int i = 0; i < 3; ++i) radius = abs(s->e[a][i]) > radius ? abs(s->e[a][i]) : radius;
    if (rows != 0 && (rows < reach || rows < radius || rows >= s->ny)) return 0;
    double pw = or_psi_of_rho(s, rho_w);
    if (rows != 0 && !isfinite(pw)) return 0;
    for (int b = 0; b < s->Q; ++b) {
        s->opp[b] = -1;
        for (int k = 0; k < s->Q; ++k)
            if (s->c[k][0] == -s->c[b][0] && s->c[k][1] == -s->c[b][1] && s->c[k][2] == -s->c[b][2]) s->opp[b] = k;
        if (s->opp[b] < 0) return 0;
    }
    s->wall_rows = rows;
    s->rho_w = rho_w;
    s->psi_w = pw;
    return 1;
}

/* n time steps. */
void or_step(or_sim* s, int64_t nsteps)
{
    for (int64_t it = 0; it < nsteps; ++it) {
        update_rho_psi(s);
        #pragma omp parallel for schedule(static) collapse(2)
        for (int z = 0; z < s->nz; ++z)
            for (int y = 0; y < s->ny; ++y)
                for (int x = 0; x < s->nx; ++x) {
                    size_t n = cell_index(s, x, y, z);
                    double fin[OR_MAXQ], fout[OR_MAXQ], F[3];
                    for (int b = 0; b < s->Q; ++b) fin[b] = s->f[(size_t)b * s->N + n];
                    if (is_solid(s, y)) {
                        for (int b = 0; b < s->Q; ++b) fout[b] = fin[s->opp[b]];
                    } else {
                        force_at(s, s->psi, x, y, z, F);
                        or_collide_cell(s, fin, F, fout, NULL, NULL);
                    }
                    for (int b = 0; b < s->Q; ++b) {
                        size_t dst = cell_index(s, wrap(x + s->c[b][0], s->nx),
                                               wrap(y + s->c[b][1], s->ny),
                                               wrap(z + s->c[b][2], s->nz));
                        s->ftmp[(size_t)b * s->N + dst] = fout[b];
                    }
                }
        double* t = s->f; s->f = s->ftmp; s->ftmp = t;
        s->step += 1;
    }
}

/* ---- initial conditions --------------------------------------------------- */

/* f_b = feq_b(rho0, u = 0) = w_b rho0. */
void or_init_from_rho(or_sim* s, const double* rho0)
{
    for (int n = 0; n < s->N; ++n)
        for (int b = 0; b < s->Q; ++b) s->f[(size_t)b * s->N + n] = s->w[b] * rho0[n];
    s->step = 0;
}

/* Minimum-image distance along one axis from node i to the centre node n/2. */
static double min_image(int i, int n)
{
    double d = (double)i - (double)(n / 2);
    if (d > 0.5 * n) d -= n;
    if (d < -0.5 * n) d += n;
    return d;
}

/* Tanh droplet (Sec. 3): rho0 = (rl + rg)/2 - (rl - rg)/2 tanh(2 (r - R) / W),
 * r the periodic distance to the centre node (nx/2, ny/2, nz/2). */
void or_init_droplet(or_sim* s, double rho_l, double rho_g, double R, double W)
{
    double* r0 = (double*)malloc(sizeof(double) * s->N);
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                double dx = min_image(x, s->nx), dy = min_image(y, s->ny);
                double dz = (s->dim == 3) ? min_image(z, s->nz) : 0.0;
                double r = sqrt(dx * dx + dy * dy + dz * dz);
                r0[cell_index(s, x, y, z)] =
                    0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * tanh(2.0 * (r - R) / W);
            }
    or_init_from_rho(s, r0);
    free(r0);
}

/* Flat liquid slab centred on the middle node of `axis`, occupying
 * [L/4, 3L/4): the same tanh profile with r = |x_axis - L/2| and R = L/4. */
void or_init_flat(or_sim* s, double rho_l, double rho_g, double W, int axis)
{
    int L = (axis == 0) ? s->nx : ((axis == 1) ? s->ny : s->nz);
    double* r0 = (double*)malloc(sizeof(double) * s->N);
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                int i = (axis == 0) ? x : ((axis == 1) ? y : z);
                double r = fabs(min_image(i, L));
                r0[cell_index(s, x, y, z)] =
                    0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * tanh(2.0 * (r - 0.25 * L) / W);
            }
    or_init_from_rho(s, r0);
    free(r0);
}

void or_set_f(or_sim* s, const double* f) { memcpy(s->f, f, sizeof(double) * (size_t)s->Q * s->N); }
void or_get_f(const or_sim* s, double* f) { memcpy(f, s->f, sizeof(double) * (size_t)s->Q * s->N); }

/* ---- macroscopic fields and observables -------------------------------- */

/* rho, psi, F (3 per cell) and u (3 per cell) of the current state; any output
 * may be NULL.  Solid nodes report F = u = 0 (rho is the sum of the populations
 * they hold, psi the wall's). */
void or_fields(or_sim* s, double* rho, double* psi, double* F, double* u)
{
    update_rho_psi(s);
    for (int z = 0; z < s->nz; ++z)
        for (int y = 0; y < s->ny; ++y)
            for (int x = 0; x < s->nx; ++x) {
                size_t n = cell_index(s, x, y, z);
                double Fl[3], j[3] = { 0.0, 0.0, 0.0 };
                const int solid = is_solid(s, y);
                force_at(s, s->psi, x, y, z, Fl);
                for (int b = 0; b < s->Q; ++b)
                    for (int i = 0; i < 3; ++i) j[i] += s->f[(size_t)b * s->N + n] * s->c[b][i];
                if (rho) rho[n] = s->rho[n];
                if (psi) psi[n] = s->psi[n];
                for (int i = 0; i < 3; ++i) {
                    if (F) F[3 * n + i] = solid ? 0.0 : Fl[i];
                    if (u) u[3 * n + i] = solid ? 0.0 : (j[i] + 0.5 * Fl[i]) / s->rho[n];
                }
            }
}

/* out[0..10] = rho_l (centre node), rho_g (node 0), dp = p(rho_l) - p(rho_g),
 * max|u|, mean|u|, mass, momentum x, y, z (sum of rho u), thickness (number
 * of nodes along the x line through the centre with 1.05 rho_g <= rho <=
 * 0.95 rho_l; meaningful for flat interfaces), step.
 * With a wall: rho_l is read at (nx/2, wall_rows, nz/2), the first fluid node
 * above the wall under the centre, rho_g at (0, ny - 1, 0), the top fluid row;
 * max|u|, mean|u| and the momentum run over fluid nodes only (the mean divides
 * by their number); mass still sums every node, which the scheme conserves. */
void or_observables(or_sim* s, double* out)
{
    double* u = (double*)malloc(sizeof(double) * 3 * s->N);
    or_fields(s, NULL, NULL, NULL, u);
    double mass = 0.0, mom[3] = { 0.0, 0.0, 0.0 }, umax = 0.0, usum = 0.0;
    int nfluid = 0;
    for (int n = 0; n < s->N; ++n) {
        mass += s->rho[n];
        if (is_solid(s, (n / s->nx) % s->ny)) continue;
        nfluid += 1;
        double m2 = 0.0;
        for (int i = 0; i < 3; ++i) {
            mom[i] += s->rho[n] * u[3 * n + i];
            m2 += u[3 * n + i] * u[3 * n + i];
        }
        double um = sqrt(m2);
        usum += um;
        if (um > umax) umax = um;
    }
    size_t centre = cell_index(s, s->nx / 2, s->wall_rows ? s->wall_rows : s->ny / 2, s->nz / 2);
    size_t far = s->wall_rows ? cell_index(s, 0, s->ny - 1, 0) : 0;
    double rl = s->rho[centre], rg = s->rho[far];
    double thick = 0.0;
    for (int x = 0; x < s->nx; ++x) {
        double r = s->rho[cell_index(s, x, s->ny / 2, s->nz / 2)];
        if (r >= 1.05 * rg && r <= 0.95 * rl) thick += 1.0;
    }
    out[0] = rl;
    out[1] = rg;
    out[2] = or_pressure(s, rl) - or_pressure(s, rg);
    out[3] = umax;
    out[4] = usum / nfluid;
    out[5] = mass;
    out[6] = mom[0]; out[7] = mom[1]; out[8] = mom[2];
    out[9] = thick;
    out[10] = (double)s->step;
    free(u);
}
