// api.cu -- the C ABI of include/lbm.h: context life cycle, initial conditions,
// stepping (CUDA-graph replay of the step kernels), observables and I/O.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "internal.h"
#include "trace.h"

using namespace lbm;

namespace {

thread_local char g_last_error[512] = "";

int fail(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

#define LBM_CK(call)                                                                                 \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(LBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));      \
    } while (0)

// Peng-Robinson constants (Sec. 3) and the critical temperature of the printed
// EOS with alpha = 1.  Eliminating T between dp/drho = 0 and d2p/drho2 = 0
// leaves eta^3 + eta^2 + eta - 1/3 = 0 for eta = b rho_c; then
// R T_c = 2 a rho_c (1 + eta)(1 - eta)^2 / (1 + 2 eta - eta^2)^2.
constexpr double kA = 2.0 / 49.0, kB = 2.0 / 21.0, kR = 1.0, kOmega = 0.344;

double pr_critical_temperature()
{
    double eta = 0.25;
    for (int i = 0; i < 60; ++i) {
        const double g = ((eta + 1.0) * eta + 1.0) * eta - 1.0 / 3.0;
        const double dg = (3.0 * eta + 2.0) * eta + 1.0;
        const double step = g / dg;
        eta -= step;
        if (std::fabs(step) < 1e-17) break;
    }
    const double rho_c = eta / kB;
    const double d = 1.0 + 2.0 * eta - eta * eta;
    return 2.0 * kA * rho_c * (1.0 + eta) * (1.0 - eta) * (1.0 - eta) / (d * d) / kR;
}

double pr_alpha(double t_over_tc)
{
    const double k = 0.37464 + 1.54226 * kOmega - 0.26992 * kOmega * kOmega;
    const double s = 1.0 + k * (1.0 - std::sqrt(t_over_tc));
    return s * s;
}

double pr_pressure(double rho, double T, double alpha)
{
    return rho * kR * T / (1.0 - kB * rho) - kA * alpha * rho * rho / (1.0 + 2.0 * kB * rho - kB * kB * rho * rho);
}

struct LatInfo {
    int Q, D, reach, iso_order;
    double cs2;
};

bool lattice_info(int lattice, LatInfo* li)
{
    switch (lattice) {
    case LBM_D2Q9: *li = {9, 2, 1, 4, 1.0 / 3.0}; return true;
    case LBM_D3Q19: *li = {19, 3, 1, 4, 1.0 / 3.0}; return true;
    case LBM_D2Q13: *li = {13, 2, 2, 6, 2.0 / 5.0}; return true;
    case LBM_D2Q25: *li = {25, 2, 2, 8, 4.0 / 7.0}; return true;
    default: return false;
    }
}

int stencil_radius(int dim, int order)
{
    if (dim == 2) return order == 4 ? 1 : (order == 6 || order == 8) ? 2 : order == 10 ? 3 : -1;
    return order == 4 ? 1 : order == 6 ? 2 : -1;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

constexpr int kGraphSteps = 16;   // steps per captured graph (even)
// Couplings weaker than this use the tanh start in lbm_init_droplet_learned:
// within ~0.65 of G_c = -4 a droplet may dissolve, persist or settle with
// another current depending on the initial state, so a learned start need not
// reach the plain run's steady state.
constexpr double kWarmStartMaxG = -4.65;
constexpr int kNBlocksMax = 152 * 16;
constexpr uint32_t kMagic = 0x4c424d31u;  // "LBM1"

}  // namespace

int lbm::set_last_error(int code, const char* msg) { return fail(code, "%s", msg); }

struct lbm_ctx {
    lbm_params prm;
    LatInfo li;
    int order;   // resolved stencil order
    int g;       // stencil radius = psi ghost width
    int device;
    cudaStream_t stream;
    bool own_stream;
    bool graphs_ok;
    size_t elem;  // bytes per population value
    long long N;
    void* buf[2];
    int cur;      // index of the buffer holding the current state
    void* psi;
    size_t psi_bytes;
    double* partials;
    double* res;
    unsigned* err;
    double* host_res;  // pinned
    size_t res_len;
    CUtensorMap tmap;
    KernelSet ks;
    DevParams dp;
    int64_t step;
    cudaGraphExec_t graph;
    bool graph_valid;
    int variant;       // step schedule: -1 two-pass (psi + fused TMA kernel), else one-pass variant
    bool tuned;        // schedule chosen (the autotuner runs on the first step)
    int n_cand;
    int cand[kMaxVariants + 1];       // candidate schedules of the autotuner
    double cand_ms[kMaxVariants + 1]; // their measured milliseconds per step
    float* carry[2];   // carried density of buf[0] / buf[1] (schedules with carry_rows > 0)
    int carry_tag[2];  // rows per group of the carry layout in carry[i]; 0: not the density of buf[i]

    void* dalloc(size_t bytes)
    {
        if (bytes == 0) bytes = 256;
        if (prm.dev_alloc) return prm.dev_alloc(bytes, prm.alloc_ctx);
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
        if (prm.dev_free)
            prm.dev_free(p, prm.alloc_ctx);
        else
            cudaFree(p);
    }
    LaunchArgs args() const
    {
        LaunchArgs a{};
        a.p = dp;
        finish_params(a.p);
        a.fin = buf[cur];
        a.fout = buf[cur ^ 1];
        a.carry_in = carry[cur];
        a.carry_out = carry[cur ^ 1];
        a.psi = psi;
        a.tmap = &tmap;
        a.partials = partials;
        a.nblocks_max = kNBlocksMax;
        a.res = res;
        return a;
    }
};

namespace {

// RAII device scratch from the context's allocator.
struct Scratch {
    lbm_ctx* c;
    void* p;
    Scratch(lbm_ctx* ctx, size_t bytes) : c(ctx), p(ctx->dalloc(bytes)) {}
    ~Scratch() { c->dfree(p); }
    double* d() const { return static_cast<double*>(p); }
};

int set_device(lbm_ctx* c)
{
    LBM_CK(cudaSetDevice(c->device));
    return LBM_OK;
}

// A schedule with a carried density (carry_rows > 0) reads the density of the
// current state from carry[cur] and writes that of the next into carry[cur^1].
// Makes carry[cur] hold the density of buf[cur] in schedule v's layout: the
// buffers are allocated on first use (for the smallest group among the
// candidates), and k_carry_init starts a carry whenever carry_tag says that
// carry[cur] is stale or in another layout.
int ensure_carry(lbm_ctx* c, int v)
{
    const int rows = v >= 0 ? c->ks.onepass[v].carry_rows : 0;
    if (rows == 0) return LBM_OK;
    if (!c->ks.carry_init) return fail(LBM_EUNSUPPORTED, "no carried-density kernel for this case");
    if (!c->carry[0]) {
        int rmin = rows;
        for (int i = 0; i < c->n_cand; ++i) {
            const int r = c->cand[i] >= 0 ? c->ks.onepass[c->cand[i]].carry_rows : 0;
            if (r > 0 && r < rmin) rmin = r;
        }
        const long long nty = (c->prm.ny + rmin - 1) / rmin;
        const size_t bytes = sizeof(float) * (size_t)(c->N + 2LL * nty * c->prm.nz * c->prm.nx);
        for (int i = 0; i < 2; ++i) {
            c->carry[i] = static_cast<float*>(c->dalloc(bytes));
            if (!c->carry[i]) return fail(LBM_ENOMEM, "carried-density allocation failed");
        }
    }
    if (c->carry_tag[c->cur] != rows) {
        LBM_CK(c->ks.carry_init(c->args(), rows, c->stream));
        c->carry_tag[c->cur] = rows;
    }
    return LBM_OK;
}

// Launches schedule v (-1 two-pass, else one-pass variant v) from buffer cur to cur^1.
int launch_schedule(lbm_ctx* c, int v)
{
    if (int rc = ensure_carry(c, v)) return rc;
    const LaunchArgs a = c->args();
    if (v >= 0) {
        LBM_CK(c->ks.onepass[v].fn(a, c->stream));
    } else {
        LBM_CK(c->ks.psi(a, c->stream));
        LBM_CK(c->ks.fused(a, c->stream));
    }
    c->carry_tag[c->cur ^ 1] = v >= 0 ? c->ks.onepass[v].carry_rows : 0;
    return LBM_OK;
}

int one_step(lbm_ctx* c)
{
    if (int rc = launch_schedule(c, c->variant)) return rc;
    c->cur ^= 1;
    return LBM_OK;
}

// Times every candidate schedule on the context's current state (cur -> cur^1,
// without advancing it: each trial recomputes the same step) with CUDA events on
// the context's stream, and keeps the fastest.  All candidates perform the same
// arithmetic, so the choice changes speed only.
int autotune(lbm_ctx* c)
{
    if (c->tuned) return LBM_OK;
    cudaEvent_t e0, e1;
    LBM_CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(LBM_ECUDA, "event creation failed");
    }
    constexpr int kReps = 3;
    int rc = LBM_OK;
    int best = -1;
    for (int i = 0; i < c->n_cand && rc == LBM_OK; ++i) {
        const int v = c->cand[i];
        rc = launch_schedule(c, v);  // warm-up (and the start of a carried density)
        if (rc == LBM_OK && cudaEventRecord(e0, c->stream) != cudaSuccess) rc = fail(LBM_ECUDA, "event record");
        for (int r = 0; r < kReps && rc == LBM_OK; ++r) rc = launch_schedule(c, v);
        if (rc == LBM_OK && cudaEventRecord(e1, c->stream) != cudaSuccess) rc = fail(LBM_ECUDA, "event record");
        if (rc == LBM_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(LBM_ECUDA, "event sync");
        float ms = 0.f;
        if (rc == LBM_OK) cudaEventElapsedTime(&ms, e0, e1);
        c->cand_ms[i] = ms / kReps;
        if (rc == LBM_OK && (best < 0 || c->cand_ms[i] < c->cand_ms[best])) best = i;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LBM_OK) return rc;
    c->variant = c->cand[best];
    c->tuned = true;
    return LBM_OK;
}

int build_graph(lbm_ctx* c)
{
    // Captured from cur == 0; after an even number of steps cur is 0 again.
    cudaGraph_t g = nullptr;
    LBM_CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = LBM_OK;
    for (int i = 0; i < kGraphSteps && rc == LBM_OK; ++i) rc = one_step(c);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(LBM_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(LBM_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    c->graph_valid = true;
    return LBM_OK;
}

double psi_host(const lbm_ctx* c, double rho)
{
    if (c->prm.psi == LBM_PSI_EXP) return -std::expm1(-rho);
    const double arg = 2.0 * (pr_pressure(rho, c->dp.pr_T, c->dp.pr_alpha) - c->li.cs2 * rho) / (c->prm.G * c->li.cs2);
    return std::sqrt(arg);
}

double pressure_host(const lbm_ctx* c, double rho)
{
    if (c->prm.psi == LBM_PSI_PENG_ROBINSON) return pr_pressure(rho, c->dp.pr_T, c->dp.pr_alpha);
    const double ps = psi_host(c, rho);
    return c->li.cs2 * rho + 0.5 * c->prm.G * c->li.cs2 * ps * ps;
}

int check_err_word(lbm_ctx* c, unsigned* word_out)
{
    unsigned w = 0;
    LBM_CK(cudaMemcpyAsync(&w, c->err, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(cudaStreamSynchronize(c->stream));
    if (w) LBM_CK(cudaMemsetAsync(c->err, 0, sizeof(unsigned), c->stream));
    *word_out = w;
    return LBM_OK;
}

int err_code_of(unsigned w)
{
    if (w & kErrTimeout) return fail(LBM_ETIMEOUT, "a bounded device wait ran out");
    if (w & kErrNegativeSqrt) return fail(LBM_ENONFINITE, "Peng-Robinson psi argument below zero");
    if (w & kErrNonFinite) return fail(LBM_ENONFINITE, "non-finite density or velocity");
    return LBM_OK;
}

// rho_bar := mean of the double field x (FP32 storage only), returned in *mean.
int field_mean(lbm_ctx* c, const double* x, double* mean)
{
    LBM_CK(launch_mean(x, c->N, c->partials, kNBlocksMax, c->res, c->stream));
    LBM_CK(cudaMemcpyAsync(c->host_res, c->res, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(cudaStreamSynchronize(c->stream));
    *mean = c->host_res[0];
    return LBM_OK;
}

// Kernel parameters (rho_bar) are baked into the captured graph: drop it
// whenever they change.
void invalidate_graph(lbm_ctx* c)
{
    c->carry_tag[0] = c->carry_tag[1] = 0;  // every caller changes the state or the schedule
    if (c->graph_valid) {
        cudaGraphExecDestroy(c->graph);
        c->graph_valid = false;
    }
}

// Populates buffer 0 from the double density field rho0 (device, N values).
int init_from_device_rho(lbm_ctx* c, double* rho0)
{
    invalidate_graph(c);
    c->dp.rho_bar = 0.0;
    if (c->prm.precision == LBM_FP32_SHIFTED) {
        int rc = field_mean(c, rho0, &c->dp.rho_bar);
        if (rc) return rc;
    }
    c->cur = 0;
    LaunchArgs a = c->args();
    a.dbuf0 = rho0;
    a.fout = c->buf[0];
    LBM_CK(c->ks.init_from_rho(a, c->stream));
    c->step = 0;
    return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_strerror(int code)
{
    switch (code) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_EUNSUPPORTED: return "unsupported combination";
    case LBM_ENOMEM: return "device allocation failed";
    case LBM_ECUDA: return "CUDA error";
    case LBM_ENONFINITE: return "non-finite value in the fields";
    case LBM_ETIMEOUT: return "device wait timed out";
    case LBM_ENOTCONVERGED: return "not converged";
    case LBM_EIO: return "file I/O error";
    default: return "unknown error";
    }
}

const char* lbm_last_error(void) { return g_last_error; }

int lbm_params_default(lbm_params* p)
{
    if (!p) return fail(LBM_EINVAL, "NULL params");
    std::memset(p, 0, sizeof(*p));
    p->nx = 64;
    p->ny = 64;
    p->nz = 1;
    p->lattice = LBM_D2Q9;
    p->stencil = LBM_STENCIL_LATTICE;
    p->psi = LBM_PSI_EXP;
    p->T_over_Tc = 0.0;
    p->G = -5.0;
    p->tau = 1.0;
    p->collision = LBM_BGK;
    p->s_e = 1.64;
    p->s_eps = 1.54;
    p->s_q = 1.9;
    p->precision = LBM_FP64;
    p->path = LBM_PATH_AUTO;
    p->wall_rows = 0;
    p->rho_w = 1.0;
    return LBM_OK;
}

int lbm_create(const lbm_params* p, lbm_ctx** out)
{
    if (!p || !out) return fail(LBM_EINVAL, "NULL argument");
    LatInfo li;
    if (!lattice_info(p->lattice, &li)) return fail(LBM_EINVAL, "unknown lattice %d", p->lattice);
    const int nz = (li.D == 2) ? 1 : p->nz;
    if (p->nx < 8 || p->ny < 8 || (li.D == 3 && nz < 8))
        return fail(LBM_EINVAL, "every dimension must be >= 8 (got %d x %d x %d)", p->nx, p->ny, nz);
    if (li.D == 2 && p->nz != 1) return fail(LBM_EINVAL, "2-D lattice needs nz = 1");
    if ((long long)p->nx * p->ny * nz > (1LL << 31) / 32) return fail(LBM_EINVAL, "domain too large");
    if (!(p->tau > 0.5)) return fail(LBM_EINVAL, "tau must exceed 1/2");
    if (!std::isfinite(p->G)) return fail(LBM_EINVAL, "G not finite");
    if (p->psi != LBM_PSI_EXP && p->psi != LBM_PSI_PENG_ROBINSON) return fail(LBM_EINVAL, "unknown psi");
    if (p->collision != LBM_BGK && p->collision != LBM_MRT && p->collision != LBM_BGK_EDM)
        return fail(LBM_EINVAL, "unknown collision");
    if (p->precision != LBM_FP64 && p->precision != LBM_FP32_SHIFTED) return fail(LBM_EINVAL, "unknown precision");
    if (p->path < LBM_PATH_AUTO || p->path > LBM_PATH_ONE_PASS) return fail(LBM_EINVAL, "unknown path");
    int order = p->stencil == LBM_STENCIL_LATTICE ? li.iso_order : p->stencil;
    if (order != 4 && order != 6 && order != 8 && order != 10) return fail(LBM_EINVAL, "unknown stencil %d", p->stencil);
    const int g = stencil_radius(li.D, order);
    if (g < 0) return fail(LBM_EUNSUPPORTED, "no %d-D stencil of order %d", li.D, order);
    if (p->collision == LBM_MRT && !(p->lattice == LBM_D2Q9 || p->lattice == LBM_D3Q19))
        return fail(LBM_EUNSUPPORTED, "MRT is provided for D2Q9 and D3Q19 only");
    if (p->collision == LBM_BGK_EDM && li.D != 2)
        return fail(LBM_EUNSUPPORTED, "exact-difference forcing is provided for the 2-D lattices");
    if (p->collision == LBM_MRT) {
        const double r[3] = {p->s_e, p->s_eps, p->s_q};
        for (double v : r)
            if (!(v > 0.0 && v < 2.0)) return fail(LBM_EINVAL, "MRT rates must lie in (0, 2)");
    }
    if (p->psi == LBM_PSI_PENG_ROBINSON) {
        if (p->precision != LBM_FP64) return fail(LBM_EUNSUPPORTED, "Peng-Robinson psi needs FP64 storage");
        if (!(p->G < 0.0)) return fail(LBM_EINVAL, "Peng-Robinson psi needs G < 0");
        if (!(p->T_over_Tc > 0.0 && p->T_over_Tc < 1.0)) return fail(LBM_EINVAL, "T_over_Tc must lie in (0, 1)");
    }
    if ((p->dev_alloc == nullptr) != (p->dev_free == nullptr))
        return fail(LBM_EINVAL, "dev_alloc and dev_free must be given together");
    if (p->wall_rows != 0) {
        if (li.D != 2) return fail(LBM_EUNSUPPORTED, "the wall is provided for the 2-D lattices");
        if (p->path == LBM_PATH_ONE_PASS) return fail(LBM_EUNSUPPORTED, "the wall runs on the two-pass schedule");
        const int need = li.reach > g ? li.reach : g;
        if (p->wall_rows < need || p->wall_rows >= p->ny)
            return fail(LBM_EINVAL, "wall_rows must lie in [%d, ny) (lattice reach and force radius)", need);
        if (!(p->rho_w > 0.0) || !std::isfinite(p->rho_w)) return fail(LBM_EINVAL, "rho_w must be positive");
    }

    KernelSet ks{};
    const int fp32 = p->precision == LBM_FP32_SHIFTED;
    bool ok = false;
    switch (p->lattice) {
    case LBM_D2Q9: ok = kernels_d2q9(order, p->collision, fp32, &ks); break;
    case LBM_D3Q19: ok = kernels_d3q19(order, p->collision, fp32, &ks); break;
    case LBM_D2Q13: ok = kernels_d2q13(order, p->collision, fp32, &ks); break;
    case LBM_D2Q25: ok = kernels_d2q25(order, p->collision, fp32, &ks); break;
    }
    if (!ok) return fail(LBM_EUNSUPPORTED, "combination not instantiated");
    if (p->path == LBM_PATH_ONE_PASS && ks.n_onepass == 0)
        return fail(LBM_EUNSUPPORTED, "one-pass schedule not built for this case");

    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(LBM_ENOMEM, "host allocation failed");
    c->prm = *p;
    c->prm.nz = nz;
    c->li = li;
    c->order = order;
    c->g = g;
    c->ks = ks;
    c->elem = fp32 ? 4 : 8;
    c->N = (long long)p->nx * p->ny * nz;
    c->n_cand = 0;
    if (p->path != LBM_PATH_ONE_PASS) c->cand[c->n_cand++] = -1;
    if (p->path != LBM_PATH_TWO_PASS && p->wall_rows == 0)
        for (int v = 0; v < ks.n_onepass; ++v)
            if (p->nx % ks.onepass[v].nx_multiple == 0 &&
                (ks.onepass[v].nx_exact == 0 || ks.onepass[v].nx_exact == p->nx) &&
                (ks.onepass[v].nx_max == 0 || p->nx <= ks.onepass[v].nx_max))
                c->cand[c->n_cand++] = v;
    if (c->n_cand == 0) {
        delete c;
        return fail(LBM_EUNSUPPORTED, "no one-pass variant applies to this domain");
    }
    c->variant = c->cand[0];
    c->tuned = c->n_cand == 1;

    auto cleanup = [&](int code) {
        lbm_destroy(c);
        return code;
    };
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return fail(LBM_ECUDA, "no current CUDA device");
    }
    if (p->stream) {
        c->stream = static_cast<cudaStream_t>(p->stream);
        c->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(LBM_ECUDA, "stream creation failed");
        }
        c->own_stream = true;
    }
    // Special handles (legacy / per-thread default stream) cannot be captured.
    c->graphs_ok = !(p->stream == reinterpret_cast<void*>(1) || p->stream == reinterpret_cast<void*>(2));

    const int gz = (li.D == 3) ? g : 0;
    int psx = p->nx + 2 * kGhostX;
    psx = (psx + 3) / 4 * 4;  // 16-byte row pitch for both element sizes
    const int psy = p->ny + 2 * g;
    c->psi_bytes = (size_t)psx * psy * (nz + 2 * gz) * c->elem;
    const size_t fbytes = (size_t)li.Q * c->N * c->elem;
    c->buf[0] = c->dalloc(fbytes);
    c->buf[1] = c->dalloc(fbytes);
    c->psi = c->dalloc(c->psi_bytes);
    c->partials = static_cast<double*>(c->dalloc(sizeof(double) * kNBlocksMax * kObsWidth));
    c->res_len = kResLine + p->nx + 8;
    c->res = static_cast<double*>(c->dalloc(sizeof(double) * c->res_len));
    c->err = static_cast<unsigned*>(c->dalloc(256));
    if (!c->buf[0] || !c->buf[1] || !c->psi || !c->partials || !c->res || !c->err)
        return cleanup(fail(LBM_ENOMEM, "device allocation of %zu bytes failed", 2 * fbytes + c->psi_bytes));
    if (cudaMallocHost(&c->host_res, sizeof(double) * c->res_len) != cudaSuccess)
        return cleanup(fail(LBM_ENOMEM, "pinned host allocation failed"));
    if (cudaMemsetAsync(c->buf[0], 0, fbytes, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->buf[1], 0, fbytes, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->psi, 0, c->psi_bytes, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->err, 0, 256, c->stream) != cudaSuccess)
        return cleanup(fail(LBM_ECUDA, "memset failed"));

    DevParams& d = c->dp;
    d.nx = p->nx;
    d.ny = p->ny;
    d.nz = nz;
    d.N = c->N;
    d.g = g;
    d.psx = psx;
    d.psy = psy;
    d.G = p->G;
    d.omega = 1.0 / p->tau;
    d.pref = 1.0 - 1.0 / (2.0 * p->tau);
    d.rho_bar = 0.0;
    d.psi_kind = p->psi;
    if (p->psi == LBM_PSI_PENG_ROBINSON) {
        d.pr_T = p->T_over_Tc * pr_critical_temperature();
        d.pr_alpha = pr_alpha(p->T_over_Tc);
    }
    d.rate[0] = 1.0 / p->tau;
    d.rate[1] = p->s_e;
    d.rate[2] = p->s_eps;
    d.rate[3] = p->s_q;
    d.err = c->err;
    d.wall_rows = p->wall_rows;
    if (p->wall_rows) {
        d.psi_w = psi_host(c, p->rho_w);
        if (!std::isfinite(d.psi_w))
            return cleanup(fail(LBM_EINVAL, "psi of the wall density rho_w is not finite (Peng-Robinson argument below zero)"));
    }

    // TMA descriptor of the ghosted psi buffer; the box is one fused-kernel
    // tile plus the halo (x: kGhostX each side, y/z: the stencil radius).
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode_fn();
    if (!enc) return cleanup(fail(LBM_ECUDA, "cuTensorMapEncodeTiled unavailable"));
    const CUtensorMapDataType dt = fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    cuuint64_t dims[3] = {(cuuint64_t)(p->nx + 2 * kGhostX), (cuuint64_t)psy, (cuuint64_t)(nz + 2 * gz)};
    cuuint64_t strides[2] = {(cuuint64_t)psx * c->elem, (cuuint64_t)psx * psy * c->elem};
    cuuint32_t box[3] = {(cuuint32_t)(ks.tile_x + 2 * kGhostX), (cuuint32_t)(ks.tile_y + 2 * g),
                         (cuuint32_t)(ks.tile_z + 2 * gz)};
    cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t rank = li.D == 3 ? 3 : 2;
    CUresult cr = enc(&c->tmap, dt, rank, c->psi, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cleanup(fail(LBM_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr));
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cleanup(fail(LBM_ECUDA, "create sync failed"));
    *out = c;
    return LBM_OK;
}

int lbm_destroy(lbm_ctx* c)
{
    if (!c) return LBM_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph_valid) cudaGraphExecDestroy(c->graph);
    c->dfree(c->buf[0]);
    c->dfree(c->buf[1]);
    c->dfree(c->carry[0]);
    c->dfree(c->carry[1]);
    c->dfree(c->psi);
    c->dfree(c->partials);
    c->dfree(c->res);
    c->dfree(c->err);
    if (c->host_res) cudaFreeHost(c->host_res);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return LBM_OK;
}

int lbm_init_droplet(lbm_ctx* c, double rho_l, double rho_g, double R, double width)
{
    if (!c) return fail(LBM_EINVAL, "NULL context");
    if (!(width > 0.0) || !(R >= 0.0) || !std::isfinite(rho_l) || !std::isfinite(rho_g) || !(rho_l > 0.0) ||
        !(rho_g > 0.0))
        return fail(LBM_EINVAL, "bad droplet parameters");
    if (int rc = set_device(c)) return rc;
    Scratch rho0(c, sizeof(double) * c->N);
    if (!rho0.p) return fail(LBM_ENOMEM, "scratch allocation failed");
    LaunchArgs a = c->args();
    a.dbuf0 = rho0.d();
    a.mode = 0;
    a.a0 = rho_l; a.a1 = rho_g; a.a2 = R; a.a3 = width;
    LBM_CK(c->ks.init_profile(a, c->stream));
    int rc = init_from_device_rho(c, rho0.d());
    LBM_CK(cudaStreamSynchronize(c->stream));
    return rc;
}

int lbm_init_flat(lbm_ctx* c, double rho_l, double rho_g, double width, int axis)
{
    if (!c) return fail(LBM_EINVAL, "NULL context");
    if (!(width > 0.0) || !(rho_l > 0.0) || !(rho_g > 0.0) || axis < 0 || axis > (c->li.D - 1))
        return fail(LBM_EINVAL, "bad flat-interface parameters");
    if (int rc = set_device(c)) return rc;
    Scratch rho0(c, sizeof(double) * c->N);
    if (!rho0.p) return fail(LBM_ENOMEM, "scratch allocation failed");
    LaunchArgs a = c->args();
    a.dbuf0 = rho0.d();
    a.mode = 1;
    a.axis = axis;
    a.a0 = rho_l; a.a1 = rho_g; a.a2 = 0.0; a.a3 = width;
    LBM_CK(c->ks.init_profile(a, c->stream));
    int rc = init_from_device_rho(c, rho0.d());
    LBM_CK(cudaStreamSynchronize(c->stream));
    return rc;
}

// Learned warm start: rho0(r) = network(G, tau, order, R_eff, r - R_eff), R_eff bisected
// so that the mass equals the tanh droplet's (rho_l, rho_g, R, width), the rest
// of the mass difference removed by a uniform shift.  Falls back to the tanh
// profile if the network gives a non-finite or non-positive density.
int lbm_init_droplet_learned(lbm_ctx* c, lbm_mlp* net, double R, double rho_l, double rho_g, double width,
                             int* used_fallback, double* R_eff_out)
{
    if (!c || !net || !(R > 0.0) || !(width > 0.0) || !(rho_l > 0.0) || !(rho_g > 0.0))
        return fail(LBM_EINVAL, "bad argument");
    if (c->prm.psi != LBM_PSI_EXP) return fail(LBM_EUNSUPPORTED, "the warm-start network models psi = 1 - exp(-rho)");
    if (int rc = set_device(c)) return rc;
    if (used_fallback) *used_fallback = 0;
    if (c->prm.G > kWarmStartMaxG) {  // near the critical coupling the steady state depends on the start
        if (used_fallback) *used_fallback = 1;
        if (R_eff_out) *R_eff_out = R;
        return lbm_init_droplet(c, rho_l, rho_g, R, width);
    }
    Scratch rho0(c, sizeof(double) * c->N);
    constexpr int T = 1024;
    constexpr double kDmax = kMlpDmax;
    Scratch table(c, sizeof(float) * T);
    if (!rho0.p || !table.p) return fail(LBM_ENOMEM, "scratch allocation failed");
    // target mass of the tanh start
    LaunchArgs a = c->args();
    a.dbuf0 = rho0.d();
    a.mode = 0;
    a.a0 = rho_l; a.a1 = rho_g; a.a2 = R; a.a3 = width;
    LBM_CK(c->ks.init_profile(a, c->stream));
    double m0 = 0.0;
    if (int rc = field_mean(c, rho0.d(), &m0)) return rc;
    const int dim = c->li.D;
    // The network holds 2-D profiles, whose Laplace jump is sigma/R; a 3-D
    // droplet's is 2 sigma/R, the jump of a 2-D droplet of radius R/2, so a 3-D
    // droplet's profile is taken at that radius (and placed at R).
    const double r_in = (dim == 3) ? 0.5 : 1.0;
    auto mass_at = [&](double Re, double* mean) -> int {
        if (int rc = mlp_profile_table(net, c->prm.G, c->prm.tau, (double)c->order, r_in * Re, T, kDmax,
                                       static_cast<float*>(table.p)))
            return rc;
        LBM_CK(launch_field_from_table(c->dp, dim, static_cast<const float*>(table.p), T, kDmax, Re, rho0.d(),
                                       c->stream));
        return field_mean(c, rho0.d(), mean);
    };
    // the steady radius can differ much from R when the tanh densities are far
    // from coexistence (small droplet, large box): bracket the whole box
    int nmin = std::min(c->prm.nx, c->prm.ny);
    if (dim == 3) nmin = std::min(nmin, c->prm.nz);
    double lo = 1.0, hi = 0.5 * nmin, mlo = 0.0, mhi = 0.0;
    int rc = mass_at(lo, &mlo);
    if (rc == LBM_OK) rc = mass_at(hi, &mhi);
    if (rc != LBM_OK) return rc;
    bool ok = std::isfinite(mlo) && std::isfinite(mhi) && (mlo - m0) * (mhi - m0) < 0.0;
    double Re = R;
    // 36 halvings of a bracket of at most a few hundred cells leave R_eff within
    // 1e-8; the uniform shift below removes the remaining mass difference
    for (int it = 0; ok && it < 36; ++it) {
        Re = 0.5 * (lo + hi);
        double mm = 0.0;
        if (int r2 = mass_at(Re, &mm)) return r2;
        if (!std::isfinite(mm)) {
            ok = false;
            break;
        }
        if ((mm - m0) * (mlo - m0) > 0.0) {
            lo = Re;
            mlo = mm;
        } else {
            hi = Re;
        }
    }
    if (ok) {
        double mm = 0.0;
        if (int r2 = mass_at(Re, &mm)) return r2;
        LBM_CK(launch_add_constant(rho0.d(), c->N, m0 - mm, c->stream));
        // the shifted field must stay a valid density
        std::vector<float> tab(T);
        LBM_CK(cudaMemcpyAsync(tab.data(), table.p, sizeof(float) * T, cudaMemcpyDeviceToHost, c->stream));
        LBM_CK(cudaStreamSynchronize(c->stream));
        for (float v : tab)
            if (!std::isfinite(v) || v + (m0 - mm) <= 0.0) ok = false;
    }
    if (!ok) {  // fallback: the plain tanh droplet
        if (used_fallback) *used_fallback = 1;
        LBM_CK(c->ks.init_profile(a, c->stream));
        Re = R;
    }
    if (R_eff_out) *R_eff_out = Re;
    rc = init_from_device_rho(c, rho0.d());
    LBM_CK(cudaStreamSynchronize(c->stream));
    return rc;
}

int lbm_init_from_rho(lbm_ctx* c, const double* rho_host)
{
    if (!c || !rho_host) return fail(LBM_EINVAL, "NULL argument");
    if (int rc = set_device(c)) return rc;
    Scratch rho0(c, sizeof(double) * c->N);
    if (!rho0.p) return fail(LBM_ENOMEM, "scratch allocation failed");
    LBM_CK(cudaMemcpyAsync(rho0.p, rho_host, sizeof(double) * c->N, cudaMemcpyHostToDevice, c->stream));
    int rc = init_from_device_rho(c, rho0.d());
    LBM_CK(cudaStreamSynchronize(c->stream));
    return rc;
}

int lbm_get_populations(lbm_ctx* c, double* f_host)
{
    if (!c || !f_host) return fail(LBM_EINVAL, "NULL argument");
    if (int rc = set_device(c)) return rc;
    const size_t bytes = sizeof(double) * c->li.Q * c->N;
    Scratch f(c, bytes);
    if (!f.p) return fail(LBM_ENOMEM, "scratch allocation failed");
    LaunchArgs a = c->args();
    a.dbuf0 = f.d();
    LBM_CK(c->ks.get_f(a, c->stream));
    LBM_CK(cudaMemcpyAsync(f_host, f.p, bytes, cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, const double* f_host)
{
    if (!c || !f_host) return fail(LBM_EINVAL, "NULL argument");
    if (int rc = set_device(c)) return rc;
    const size_t bytes = sizeof(double) * c->li.Q * c->N;
    Scratch f(c, bytes);
    Scratch rho(c, sizeof(double) * c->N);
    if (!f.p || !rho.p) return fail(LBM_ENOMEM, "scratch allocation failed");
    LBM_CK(cudaMemcpyAsync(f.p, f_host, bytes, cudaMemcpyHostToDevice, c->stream));
    invalidate_graph(c);
    c->dp.rho_bar = 0.0;
    if (c->prm.precision == LBM_FP32_SHIFTED) {
        LaunchArgs a = c->args();
        a.dbuf0 = f.d();
        a.dbuf1 = rho.d();
        LBM_CK(c->ks.rho_of_f(a, c->stream));
        if (int rc = field_mean(c, rho.d(), &c->dp.rho_bar)) return rc;
    }
    c->cur = 0;
    LaunchArgs a = c->args();
    a.dbuf0 = f.d();
    a.fout = c->buf[0];
    LBM_CK(c->ks.set_f(a, c->stream));
    LBM_CK(cudaStreamSynchronize(c->stream));
    c->step = 0;
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int64_t n)
{
    lbm::TraceRange trace("lbm_step");
    if (!c || n < 0) return fail(LBM_EINVAL, "bad argument");
    if (int rc = set_device(c)) return rc;
    if (n > 0)
        if (int rc = autotune(c)) return rc;
    while (n > 0) {
        if (c->graphs_ok && n >= kGraphSteps && c->cur == 0) {
            if (!c->graph_valid) {
                if (int rc = ensure_carry(c, c->variant)) return rc;  // outside the capture
                if (int rc = build_graph(c)) return rc;
            }
            LBM_CK(cudaGraphLaunch(c->graph, c->stream));
            n -= kGraphSteps;
            c->step += kGraphSteps;
        } else {
            if (int rc = one_step(c)) return rc;
            n -= 1;
            c->step += 1;
        }
    }
    return LBM_OK;
}

int lbm_step_timed(lbm_ctx* c, int64_t n, double* mean_ms, int max_kernels, int* nkernels)
{
    if (!c || n < 1 || !mean_ms || max_kernels < 2) return fail(LBM_EINVAL, "bad argument");
    if (int rc = set_device(c)) return rc;
    if (int rc = autotune(c)) return rc;
    const int K = c->variant >= 0 ? 1 : 2;  // onepass | psi, fused
    if (int rc = ensure_carry(c, c->variant)) return rc;
    std::vector<cudaEvent_t> ev((size_t)n * K + 1);
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(LBM_ECUDA, "event creation failed");
    int rc = LBM_OK;
    LBM_CK(cudaEventRecord(ev[0], c->stream));
    for (int64_t i = 0; i < n && rc == LBM_OK; ++i) {
        LaunchArgs a = c->args();
        if (c->variant >= 0) {
            if (cudaError_t e = c->ks.onepass[c->variant].fn(a, c->stream))
                rc = fail(LBM_ECUDA, "onepass: %s", cudaGetErrorString(e));
            if (rc == LBM_OK) cudaEventRecord(ev[i + 1], c->stream);
        } else {
            if (cudaError_t e = c->ks.psi(a, c->stream)) rc = fail(LBM_ECUDA, "psi: %s", cudaGetErrorString(e));
            if (rc == LBM_OK) cudaEventRecord(ev[i * K + 1], c->stream);
            if (rc == LBM_OK)
                if (cudaError_t e = c->ks.fused(a, c->stream))
                    rc = fail(LBM_ECUDA, "fused: %s", cudaGetErrorString(e));
            if (rc == LBM_OK) cudaEventRecord(ev[i * K + 2], c->stream);
        }
        c->carry_tag[c->cur ^ 1] = c->variant >= 0 ? c->ks.onepass[c->variant].carry_rows : 0;
        c->cur ^= 1;
        c->step += 1;
    }
    if (rc == LBM_OK && cudaEventSynchronize(ev.back()) != cudaSuccess) rc = fail(LBM_ECUDA, "event sync failed");
    if (rc == LBM_OK) {
        for (int k = 0; k < K; ++k) {
            double sum = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[i * K + k], ev[i * K + k + 1]);
                sum += ms;
            }
            mean_ms[k] = sum / (double)n;
        }
        if (nkernels) *nkernels = K;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return rc;
}

const char* lbm_step_kernel_name(const lbm_ctx* c, int i)
{
    if (c && c->variant >= 0) return i == 0 ? "k_onepass" : "";
    return i == 0 ? "k_psi" : (i == 1 ? "k_fused" : "");
}

int lbm_schedule_report(lbm_ctx* c, char* buf, int len)
{
    if (!c || !buf || len < 1) return fail(LBM_EINVAL, "bad argument");
    if (int rc = set_device(c)) return rc;
    if (int rc = autotune(c)) return rc;
    auto name = [c](int v) { return v >= 0 ? c->ks.onepass[v].name : "two_pass"; };
    int off = std::snprintf(buf, (size_t)len, "chosen=%s", name(c->variant));
    for (int i = 0; i < c->n_cand && off < len; ++i)
        off += std::snprintf(buf + off, (size_t)(len - off), ";%s=%.5f", name(c->cand[i]),
                             c->n_cand > 1 ? c->cand_ms[i] : -1.0);
    return LBM_OK;
}

int lbm_set_schedule(lbm_ctx* c, const char* name)
{
    if (!c || !name) return fail(LBM_EINVAL, "NULL argument");
    for (int i = 0; i < c->n_cand; ++i) {
        const int v = c->cand[i];
        const char* nm = v >= 0 ? c->ks.onepass[v].name : "two_pass";
        if (std::strcmp(nm, name) == 0) {
            invalidate_graph(c);
            c->variant = v;
            c->tuned = true;
            return LBM_OK;
        }
    }
    return fail(LBM_EINVAL, "schedule %s is not a candidate of this context", name);
}

int lbm_observables(lbm_ctx* c, lbm_obs* out)
{
    lbm::TraceRange trace("lbm_observables");
    if (!c || !out) return fail(LBM_EINVAL, "NULL argument");
    if (int rc = set_device(c)) return rc;
    LaunchArgs a = c->args();
    LBM_CK(c->ks.psi(a, c->stream));
    int nb = 0;
    LBM_CK(c->ks.obs(a, c->stream, &nb));
    LBM_CK(launch_sum_partials(c->partials, nb, kObsWidth, c->res, c->stream));
    LBM_CK(c->ks.probe(a, c->stream));
    LBM_CK(cudaMemcpyAsync(c->host_res, c->res, sizeof(double) * (kResLine + c->prm.nx), cudaMemcpyDeviceToHost,
                           c->stream));
    unsigned w = 0;
    if (int rc = check_err_word(c, &w)) return rc;
    if (int rc = err_code_of(w)) return rc;
    const double* r = c->host_res;
    lbm_obs o{};
    o.mass = r[kResMass];
    o.mom[0] = r[kResMomX];
    o.mom[1] = r[kResMomY];
    o.mom[2] = r[kResMomZ];
    o.mean_u = r[kResSumU] / (double)(c->N - (long long)c->prm.wall_rows * c->prm.nx * c->prm.nz);
    o.max_u = r[kResMaxU];
    o.rho_l = r[kResRhoCentre];
    o.rho_g = r[kResRhoOrigin];
    o.dp = pressure_host(c, o.rho_l) - pressure_host(c, o.rho_g);
    double th = 0.0;
    for (int i = 0; i < c->prm.nx; ++i) {
        const double v = r[kResLine + i];
        if (v >= 1.05 * o.rho_g && v <= 0.95 * o.rho_l) th += 1.0;
    }
    o.thickness = th;
    o.step = c->step;
    if (!std::isfinite(o.mass) || !std::isfinite(o.max_u)) return fail(LBM_ENONFINITE, "non-finite observables");
    *out = o;
    return LBM_OK;
}

int lbm_reference_density(lbm_ctx* c, double* rho_bar)
{
    if (!c || !rho_bar) return fail(LBM_EINVAL, "NULL argument");
    *rho_bar = c->dp.rho_bar;
    return LBM_OK;
}

int lbm_diag_wait_timeout(lbm_ctx* c)
{
    if (!c) return fail(LBM_EINVAL, "NULL argument");
    if (int rc = set_device(c)) return rc;
    LBM_CK(launch_wait_probe(c->err, c->stream));
    unsigned w = 0;
    if (int rc = check_err_word(c, &w)) return rc;
    if (int rc = err_code_of(w)) return rc;
    return fail(LBM_ECUDA, "the probe's wait on a barrier that nothing completes did not give up");
}

int lbm_run_to_steady(lbm_ctx* c, double tol, int64_t max_steps, int64_t check_every, int64_t* steps_out)
{
    lbm::TraceRange trace("lbm_run_to_steady");
    if (!c || !(tol > 0.0) || max_steps < 0 || check_every < 1) return fail(LBM_EINVAL, "bad argument");
    lbm_obs o;
    if (int rc = lbm_observables(c, &o)) return rc;
    double prev = o.max_u;
    int64_t taken = 0;
    const bool fp32 = c->prm.precision == LBM_FP32_SHIFTED;
    while (taken < max_steps) {
        const int64_t k = (max_steps - taken < check_every) ? (max_steps - taken) : check_every;
        if (int rc = lbm_step(c, k)) return rc;
        taken += k;
        if (int rc = lbm_observables(c, &o)) return rc;
        double thr = tol;
        if (fp32) thr = std::fmax(tol, 1e-6 * o.max_u / (double)k);
        if (std::fabs(o.max_u - prev) / (double)k < thr) {
            if (steps_out) *steps_out = taken;
            return LBM_OK;
        }
        prev = o.max_u;
    }
    if (steps_out) *steps_out = taken;
    return fail(LBM_ENOTCONVERGED, "max|u| still changing after %lld steps", (long long)taken);
}

int lbm_get_fields(lbm_ctx* c, double* rho_host, double* u_host)
{
    if (!c) return fail(LBM_EINVAL, "NULL context");
    if (int rc = set_device(c)) return rc;
    Scratch rho(c, sizeof(double) * c->N);
    Scratch u(c, sizeof(double) * 3 * c->N);
    if (!rho.p || !u.p) return fail(LBM_ENOMEM, "scratch allocation failed");
    LaunchArgs a = c->args();
    a.dbuf0 = rho.d();
    a.dbuf1 = u.d();
    LBM_CK(c->ks.psi(a, c->stream));
    LBM_CK(c->ks.fields(a, c->stream));
    if (rho_host)
        LBM_CK(cudaMemcpyAsync(rho_host, rho.p, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
    if (u_host)
        LBM_CK(cudaMemcpyAsync(u_host, u.p, sizeof(double) * 3 * c->N, cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_device_state(lbm_ctx* c, const void** f_dev, int* Q, int64_t* ncells, int* elem_bytes)
{
    if (!c) return fail(LBM_EINVAL, "NULL context");
    if (f_dev) *f_dev = c->buf[c->cur];
    if (Q) *Q = c->li.Q;
    if (ncells) *ncells = c->N;
    if (elem_bytes) *elem_bytes = (int)c->elem;
    return LBM_OK;
}

double lbm_bytes_per_update(const lbm_ctx* c)
{
    if (!c) return 0.0;
    return 2.0 * c->li.Q * c->elem + 2.0 * c->elem;
}

struct CkptHeader {
    uint32_t magic, version;
    int32_t nx, ny, nz, lattice, order, collision, precision, psi;
    double G, tau, T_over_Tc, rho_bar;
    int64_t step;
    uint64_t bytes;
};

int lbm_save(lbm_ctx* c, const char* path)
{
    if (!c || !path) return fail(LBM_EINVAL, "NULL argument");
    if (int rc = set_device(c)) return rc;
    const size_t bytes = (size_t)c->li.Q * c->N * c->elem;
    std::vector<unsigned char> host(bytes);
    LBM_CK(cudaMemcpyAsync(host.data(), c->buf[c->cur], bytes, cudaMemcpyDeviceToHost, c->stream));
    LBM_CK(cudaStreamSynchronize(c->stream));
    CkptHeader h{kMagic, 1u, c->prm.nx, c->prm.ny, c->prm.nz, c->prm.lattice, c->order, c->prm.collision,
                 c->prm.precision, c->prm.psi, c->prm.G, c->prm.tau, c->prm.T_over_Tc, c->dp.rho_bar, c->step,
                 (uint64_t)bytes};
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(LBM_EIO, "cannot open %s", path);
    const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 && std::fwrite(host.data(), 1, bytes, f) == bytes;
    if (std::fclose(f) != 0 || !ok) return fail(LBM_EIO, "write to %s failed", path);
    return LBM_OK;
}

int lbm_load(lbm_ctx* c, const char* path)
{
    if (!c || !path) return fail(LBM_EINVAL, "NULL argument");
    if (int rc = set_device(c)) return rc;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(LBM_EIO, "cannot open %s", path);
    CkptHeader h{};
    const size_t bytes = (size_t)c->li.Q * c->N * c->elem;
    std::vector<unsigned char> host(bytes);
    const bool ok = std::fread(&h, sizeof(h), 1, f) == 1 && h.magic == kMagic && h.version == 1u &&
                    h.bytes == bytes && std::fread(host.data(), 1, bytes, f) == bytes;
    std::fclose(f);
    if (!ok) return fail(LBM_EIO, "%s is not a checkpoint of this size", path);
    if (h.nx != c->prm.nx || h.ny != c->prm.ny || h.nz != c->prm.nz || h.lattice != c->prm.lattice ||
        h.order != c->order || h.collision != c->prm.collision || h.precision != c->prm.precision ||
        h.psi != c->prm.psi || h.G != c->prm.G || h.tau != c->prm.tau || h.T_over_Tc != c->prm.T_over_Tc)
        return fail(LBM_EINVAL, "checkpoint parameters differ from the context's");
    invalidate_graph(c);
    c->cur = 0;
    LBM_CK(cudaMemcpyAsync(c->buf[0], host.data(), bytes, cudaMemcpyHostToDevice, c->stream));
    LBM_CK(cudaStreamSynchronize(c->stream));
    c->dp.rho_bar = h.rho_bar;
    c->step = h.step;
    return LBM_OK;
}

}  // extern "C"
