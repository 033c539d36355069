// internal.h -- interface between the C-ABI layer (api.cu) and the kernel
// instantiations (one translation unit per lattice).  Not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace lbm {

// Error bits raised by kernels in the device error word.
enum : unsigned {
    kErrNonFinite = 1u,   // NaN/Inf density or velocity
    kErrNegativeSqrt = 2u,  // Peng-Robinson psi argument below zero
    kErrTimeout = 4u,     // a bounded wait (mbarrier) gave up
};

// psi buffer: periodic ghost layers, kGhostX cells on each side in x (so that
// every TMA box starts on a 16-byte boundary) and `g` = stencil radius in y, z.
constexpr int kGhostX = 4;

// Runtime constants of one domain, passed by value to every kernel.
struct DevParams {
    int nx, ny, nz;
    long long N;         // cells
    int g;               // ghost width of psi in y (and z)
    int psx;             // psi row pitch in elements
    int psy;             // psi rows per z plane (ny + 2g)
    double G;
    double omega;        // 1 / tau
    double pref;         // 1 - 1/(2 tau)
    double rho_bar;      // reference density of FP32 deviation storage (0 in FP64)
    int psi_kind;        // 0 exp, 1 Peng-Robinson
    double pr_T;         // Peng-Robinson temperature T_over_Tc * T_c
    double pr_alpha;     // alpha(T)
    double rate[4];      // MRT rates by class: 1/tau, s_e, s_eps, s_q
    unsigned* err;       // device error word
    int wall_rows;       // rows y < wall_rows are solid (bounce-back); 0 = no wall
    double psi_w;        // psi of the wall's virtual density
    // Derived by finish_params(): the MRT correction factors omega - s per rate
    // class (class 0 relaxes at omega, so its factor is 0), and FP32 copies of
    // the scalars the FP32 kernels use, so they convert nothing per cell.
    double dmrt[4];
    float omega_f, pref_f, rho_bar_f, G_f;
    float om1_f;  // 1 - omega, rounded once from double
    float dmrt_f[4];
};

// Fills the derived fields of p from the others; call after any change to
// omega, pref, rho_bar, G or rate.
__host__ __device__ inline void finish_params(DevParams& p)
{
    for (int c = 0; c < 4; ++c) {
        p.dmrt[c] = (c == 0) ? 0.0 : p.omega - p.rate[c];
        p.dmrt_f[c] = static_cast<float>(p.dmrt[c]);
    }
    p.omega_f = static_cast<float>(p.omega);
    p.pref_f = static_cast<float>(p.pref);
    p.rho_bar_f = static_cast<float>(p.rho_bar);
    p.G_f = static_cast<float>(p.G);
    p.om1_f = static_cast<float>(1.0 - p.omega);
}

// Everything a launcher may need; unused fields are ignored.
struct LaunchArgs {
    DevParams p;
    const void* fin;       // populations read (current state)
    void* fout;            // populations written
    void* psi;             // ghosted psi buffer (base of the allocation)
    const CUtensorMap* tmap;  // TMA descriptor of the psi buffer
    double* partials;      // reduction scratch
    int nblocks_max;       // capacity of partials (blocks)
    double* res;           // reduction result (see api.cu for the slots)
    double* dbuf0;         // double work buffers (N or Q*N)
    double* dbuf1;
    int mode;              // init profile: 0 droplet, 1 flat
    int axis;
    double a0, a1, a2, a3; // init parameters (rho_l, rho_g, R, width)
    float* carry_in;       // carried density of the current state (schedules with carry_rows > 0)
    float* carry_out;      // carried density of the state written
};

// One compiled variant of the one-pass step kernel (tile shape, chunk length,
// minimum resident blocks); the autotuner picks among them.
struct StepVariant {
    const char* name;
    cudaError_t (*fn)(const LaunchArgs&, cudaStream_t);
    int nx_multiple;     // nx must be a multiple of this (two cells per thread, 16-byte rows)
    int nx_exact;        // nonzero: the variant is compiled for this nx only (whole rows in shared memory)
    int nx_max;          // nonzero: the variant takes rows of at most this many cells (shared-memory size)
    int carry_rows;      // nonzero: the step reads and writes a carried density for groups of this many rows
};
constexpr int kMaxVariants = 48;

// One set of launchers per (lattice, stencil order, collision, precision).
struct KernelSet {
    int tile_x, tile_y, tile_z;  // fused-kernel tile (TMA box minus halo)
    cudaError_t (*psi)(const LaunchArgs&, cudaStream_t);
    cudaError_t (*fused)(const LaunchArgs&, cudaStream_t);
    int n_onepass;                          // 0: no one-pass schedule
    StepVariant onepass[kMaxVariants];
    cudaError_t (*obs)(const LaunchArgs&, cudaStream_t, int* nblocks);
    cudaError_t (*probe)(const LaunchArgs&, cudaStream_t);
    cudaError_t (*fields)(const LaunchArgs&, cudaStream_t);
    cudaError_t (*init_profile)(const LaunchArgs&, cudaStream_t);
    cudaError_t (*init_from_rho)(const LaunchArgs&, cudaStream_t);
    cudaError_t (*get_f)(const LaunchArgs&, cudaStream_t);
    cudaError_t (*set_f)(const LaunchArgs&, cudaStream_t);
    cudaError_t (*rho_of_f)(const LaunchArgs&, cudaStream_t);
    cudaError_t (*carry_init)(const LaunchArgs&, int rows, cudaStream_t);  // null: no carried-density schedule
};

// Records msg as the calling thread's lbm_last_error() text and returns code.
int set_last_error(int code, const char* msg);

// Shared reduction helpers (reduce.cu).
cudaError_t launch_sum_partials(const double* partials, int nblocks, int width, double* res,
                                cudaStream_t s);
cudaError_t launch_mean(const double* x, long long n, double* partials, int nblocks_max,
                        double* res, cudaStream_t s);

// Failure-detection check (diag.cu): one block waits on an mbarrier that nothing
// completes, through the step kernels' bounded wait, and sets kErrTimeout in *err.
cudaError_t launch_wait_probe(unsigned* err, cudaStream_t s);

// Warm-start network (mlp.cu): evaluates the network's density at T signed
// distances evenly spaced over [-dmax, dmax] for (G, tau, order, R) into table_dev.
// The network's distance input spans |d| <= kMlpDmax.
constexpr double kMlpDmax = 24.0;
}  // namespace lbm
struct lbm_mlp;
namespace lbm {
int mlp_profile_table(lbm_mlp* n, double G, double tau, double order, double R, int T, double dmax,
                      float* table_dev);

// Density field from a radial profile table (reduce.cu): rho0(cell) = table(r - R)
// with r the periodic distance to the centre node, linear interpolation, clamped.
cudaError_t launch_field_from_table(const DevParams& p, int dim, const float* table, int T, double dmax, double R,
                                    double* rho0, cudaStream_t s);
cudaError_t launch_add_constant(double* x, long long n, double c, cudaStream_t s);

// Per-lattice lookup (defined in kernels_<lattice>.cu). Returns false if the
// combination is not instantiated.
bool kernels_d2q9(int order, int coll, int fp32, KernelSet* ks);
bool kernels_d3q19(int order, int coll, int fp32, KernelSet* ks);
bool kernels_d2q13(int order, int coll, int fp32, KernelSet* ks);
bool kernels_d2q25(int order, int coll, int fp32, KernelSet* ks);

// Slots of the reduction result array `res`.
enum ResSlot {
    kResMass = 0, kResMomX, kResMomY, kResMomZ, kResSumU, kResMaxU, kResCount,
    kResRhoCentre = 8, kResRhoOrigin = 9, kResLine = 16  // then nx values
};
constexpr int kObsWidth = 6;

}  // namespace lbm
