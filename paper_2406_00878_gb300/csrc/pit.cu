// pit.cu -- host side of libpit.so: the C ABI declared in include/pit.h.
//
// A context owns the problem data (u^0, Dirichlet data, sources), the residual,
// the Jacobi-scaled Jacobian planes of all levels and the chain kernel's team
// workspace. Every entry point enqueues work on the context's stream; norms and
// statistics are read back with small device-to-host copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>

#include "pit.h"
#include "pit_internal.h"
#include "pit_teams.h"
#include "pit_kernels.cuh"

using namespace pit;

namespace {
constexpr int kNT = 256;        // threads per CTA of every kernel
constexpr int kMinLocal = 256;  // auto team size: at least this many unknowns per CTA
}  // namespace

struct pit_ctx {
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    cudaStream_t stream = nullptr;
    pit_grid grid{};
    int M = 0;
    double dt = 0.0;
    pit_params params{};
    pit_options opt{};
    OpConst oc{};
    bool conv = false, nlv = false;
    long long Ns = 0, DOF = 0;
    int nb = 0;  // boundary values per level

    // problem data and workspaces (device)
    double* u0 = nullptr;
    double* bc = nullptr;    // nullptr = zero Dirichlet data
    double* q = nullptr;     // nullptr = no source
    bool has_bc = false, has_q = false;
    double* R = nullptr;     // [M][Ns]
    double* coef = nullptr;  // [5][M][Ns] scaled planes
    double* Uh = nullptr;    // [M][Ns] iterate of pit_solve_host
    unsigned long long* keys = nullptr;  // [0] ||R||_inf key, [1..M] Gershgorin keys, [M+1..2M] nonsymmetric flags

    // chain team workspace
    int G = 0, rows_base = 0, rows_rem = 0;
    size_t chain_smem = 0;
    double* pub = nullptr;
    double* red_part = nullptr;
    unsigned long long* sync_words = nullptr;  // flags[G], red_cnt[4]
    int* ints = nullptr;                       // abort, status, level_iters[M], level_method[M]
    double* cta_sumsq = nullptr;               // [G]
    unsigned long long* timers = nullptr;      // [4] chain kernel, CTA 0

    // Newton wavefront (pit_solve): K teams of Gw CTAs, the middle ones larger where SMs are left over
    int K = 0, Gw = 0, w_rows_base = 0, w_rows_rem = 0, kcap = 0;
    int Gs = 0, w_ctas = 0;                 // CTAs of the largest team (workspace stride), of the launch
    int* w_geom = nullptr;                  // [K][4] teams of different sizes (see WaveArgs::tgeom), or null
    size_t wave_smem = 0;
    double* w_pub = nullptr;
    unsigned long long* w_tpub = nullptr;   // tagged publication words: one-exchange SOR sweeps (rows_base >= 3)
    unsigned long long* w_tred = nullptr;   // tagged reduction words (with w_tpub)
    size_t w_tpub_n = 0, w_tred_n = 0;
    double* w_red = nullptr;
    unsigned long long* w_sync = nullptr;  // flags[K*Gs], prog[K*Gs], red_cnt[K*4]
    int* w_ints = nullptr;                  // abort, status, stop[2]
    double* w_res = nullptr;                // [kcap]
    double* w_prefix = nullptr;             // [kcap][M]
    int* w_cell = nullptr;                  // [kcap][M]
    double* w_sumsq = nullptr;              // [kcap][Gs]
    unsigned long long* w_timers = nullptr; // [K][kWaveTimers]
    std::vector<double> h_wres, h_wsumsq;
    std::vector<int> h_wcell;
    std::vector<unsigned long long> h_wtimers;

    // host mirrors
    std::vector<int> h_ints;
    std::vector<double> h_sumsq;
    unsigned long long h_timers[4] = {0, 0, 0, 0};
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};

    char err[512] = "";
};

// ------------------------------------------------------------------- helpers

static pit_status fail(pit_ctx* c, pit_status s, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? PIT_ENOMEM : PIT_ECUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                               \
    } while (0)

#define CHECK_RET(expr)             \
    do {                            \
        pit_status s_ = (expr);     \
        if (s_ != PIT_OK) return s_; \
    } while (0)

template <typename T>
static cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

static double key_to_double(unsigned long long k) {
    double d;
    std::memcpy(&d, &k, sizeof(d));
    return d;
}

extern "C" void pit_default_options(pit_options* o) {
    if (!o) return;
    o->newton_max = 30;
    o->tol_res = 1e-12;
    o->lin_solver = PIT_LIN_AUTO;
    o->eta_max = 1e-2;
    o->eta_gamma = 1.0;
    o->lin_atol = 1e-15;
    o->lin_max_iter = 4000;
    o->sor_rho_max = 0.999;
    o->team_ctas = 0;
    o->wait_budget = 1ll << 26;
    o->wave_teams = 0;
    o->precision = PIT_FP64;
    o->window = 0;
    o->batch_wave_nodes = 65536;
    o->window_start = PIT_START_PLAIN;
}

extern "C" const char* pit_status_string(pit_status s) {
    switch (s) {
        case PIT_OK: return "PIT_OK";
        case PIT_EINVAL: return "PIT_EINVAL";
        case PIT_ECUDA: return "PIT_ECUDA";
        case PIT_ENOMEM: return "PIT_ENOMEM";
        case PIT_ENOCONV: return "PIT_ENOCONV";
        case PIT_EDIVERGED: return "PIT_EDIVERGED";
        case PIT_ETIMEOUT: return "PIT_ETIMEOUT";
        case PIT_EUNSUPPORTED: return "PIT_EUNSUPPORTED";
        case PIT_EBOUNDS: return "PIT_EBOUNDS";
    }
    return "PIT_UNKNOWN";
}

// ------------------------------------------------------- bounds-checking build

namespace {
constexpr int kMaxBoundsReaders = 128;
int (*g_bounds_readers[kMaxBoundsReaders])();
int g_n_bounds_readers = 0;
}  // namespace

namespace pit {
// Called from static initialisers of the check build's translation units (one thread, at
// load time).
void register_bounds_reader(int (*reader)()) {
    if (g_n_bounds_readers < kMaxBoundsReaders) g_bounds_readers[g_n_bounds_readers++] = reader;
}
}  // namespace pit

extern "C" pit_status pit_bounds_status(int* enabled, int* first_id) {
    if (!enabled || !first_id) return PIT_EINVAL;
#ifdef PIT_CHECK_BOUNDS
    *enabled = 1;
#else
    *enabled = 0;
#endif
    *first_id = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return PIT_ECUDA;
    bool failed = false;
    for (int i = 0; i < g_n_bounds_readers; ++i) {
        const int v = g_bounds_readers[i]();
        if (v < 0) failed = true;
        else if (v > 0 && *first_id == 0) *first_id = v;
    }
    if (failed) return PIT_ECUDA;
    return *first_id ? PIT_EBOUNDS : PIT_OK;
}

extern "C" const char* pit_last_error(const pit_ctx* ctx) { return ctx ? ctx->err : "null context"; }

// ------------------------------------------------------------ kernel dispatch

// Residual of a window of levels [s, s + oc.M): u_prev is u^{s-1} (u^0 when s = 0);
// U, bc, q, R point at level s.
template <bool CONV, bool NLV>
static void launch_residual(pit_ctx* c, const OpConst& oc, const double* u_prev, const double* U, const double* bc,
                            const double* q, double* R) {
    dim3 grid((unsigned)((c->Ns + kNT - 1) / kNT), (unsigned)oc.M);
    residual_kernel<CONV, NLV, kNT><<<grid, kNT, 0, c->stream>>>(oc, u_prev, U, bc, q, R, c->keys);
}

static pit_status enqueue_residual_range(pit_ctx* ctx, int s, int Mw, const double* U, double* R) {
    OpConst oc = ctx->oc;
    oc.M = Mw;
    const double* u_prev = s == 0 ? ctx->u0 : U + (size_t)(s - 1) * ctx->Ns;
    const double* bc = ctx->has_bc ? ctx->bc + (size_t)s * ctx->nb : nullptr;
    const double* q = ctx->has_q ? ctx->q + (size_t)s * ctx->Ns : nullptr;
    const double* Uw = U + (size_t)s * ctx->Ns;
    double* Rw = R + (size_t)s * ctx->Ns;
    CK(cudaMemsetAsync(ctx->keys, 0, sizeof(unsigned long long), ctx->stream));
    if (ctx->conv) {
        if (ctx->nlv) launch_residual<true, true>(ctx, oc, u_prev, Uw, bc, q, Rw);
        else launch_residual<true, false>(ctx, oc, u_prev, Uw, bc, q, Rw);
    } else {
        if (ctx->nlv) launch_residual<false, true>(ctx, oc, u_prev, Uw, bc, q, Rw);
        else launch_residual<false, false>(ctx, oc, u_prev, Uw, bc, q, Rw);
    }
    CK(cudaGetLastError());
    return PIT_OK;
}

template <bool CONV, bool NLV, bool SCALED>
static void launch_assemble(pit_ctx* c, const double* U, double* coef) {
    dim3 grid((unsigned)((c->Ns + kNT - 1) / kNT), (unsigned)c->M);
    assemble_kernel<CONV, NLV, SCALED, kNT><<<grid, kNT, 0, c->stream>>>(c->oc, U, c->has_bc ? c->bc : nullptr, coef,
                                                                         c->keys + 1);
}

static pit_status enqueue_residual(pit_ctx* ctx, const double* U, double* R) {
    return enqueue_residual_range(ctx, 0, ctx->M, U, R);
}

static pit_status read_res_inf(pit_ctx* ctx, double* out) {
    unsigned long long k = 0;
    CK(cudaMemcpyAsync(&k, ctx->keys, sizeof(k), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *out = key_to_double(k);
    return PIT_OK;
}

template <bool SCALED>
static pit_status enqueue_assemble(pit_ctx* ctx, const double* U, double* coef) {
    if (SCALED) CK(cudaMemsetAsync(ctx->keys + 1, 0, sizeof(unsigned long long) * 2 * ctx->M, ctx->stream));
    if (ctx->conv) {
        if (ctx->nlv) launch_assemble<true, true, SCALED>(ctx, U, coef);
        else launch_assemble<true, false, SCALED>(ctx, U, coef);
    } else {
        if (ctx->nlv) launch_assemble<false, true, SCALED>(ctx, U, coef);
        else launch_assemble<false, false, SCALED>(ctx, U, coef);
    }
    CK(cudaGetLastError());
    return PIT_OK;
}

// Run the level chain on the scaled planes in ctx->coef with right-hand sides R.
// update_U: U += dU; dU (may be null) receives the solution. Fills the statistics.
static pit_status run_chain(pit_ctx* ctx, const double* R, double* U, double* dU, double eta, double sor_tol_abs,
                            pit_step_info* info) {
    const int G = ctx->G, M = ctx->M;
    CK(cudaMemsetAsync(ctx->sync_words, 0, sizeof(unsigned long long) * (G + 4), ctx->stream));
    CK(cudaMemsetAsync(ctx->ints, 0, sizeof(int) * (2 + 2 * (size_t)M), ctx->stream));
    ChainArgs a{};
    a.nx = ctx->grid.nx;
    a.ny = ctx->grid.ny;
    a.M = M;
    a.G = G;
    a.rows_base = ctx->rows_base;
    a.rows_rem = ctx->rows_rem;
    a.R = R;
    a.coef = ctx->coef;
    a.rho_key = ctx->keys + 1;
    a.U = U;
    a.dU = dU;
    a.update_U = U != nullptr;
    a.method = ctx->opt.lin_solver;
    a.sor_rho_max = ctx->opt.sor_rho_max;
    a.eta = eta;
    a.sor_tol_abs = sor_tol_abs;
    a.atol = ctx->opt.lin_atol;
    a.max_iter = ctx->opt.lin_max_iter;
    a.wait_budget = ctx->opt.wait_budget;
    a.pub = ctx->pub;
    a.flags = ctx->sync_words;
    a.red_cnt = ctx->sync_words + G;
    a.red_part = ctx->red_part;
    a.abort_flag = ctx->ints;
    a.status = ctx->ints + 1;
    a.level_iters = ctx->ints + 2;
    a.level_method = ctx->ints + 2 + M;
    a.cta_sumsq = ctx->cta_sumsq;
    a.timers = ctx->timers;
    void* args[] = {&a};
    CK(cudaEventRecord(ctx->ev[2], ctx->stream));
    CK(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(chain_kernel<kNT>), dim3(G), dim3(kNT), args,
                                   ctx->chain_smem, ctx->stream));
    CK(cudaEventRecord(ctx->ev[3], ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_ints.data(), ctx->ints, sizeof(int) * (2 + 2 * (size_t)M), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_sumsq.data(), ctx->cta_sumsq, sizeof(double) * G, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_timers, ctx->timers, sizeof(ctx->h_timers), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int status = ctx->h_ints[1];
    if (info) {
        long long tot = 0;
        int mx = 0, nsor = 0, ncap = 0;
        for (int n = 0; n < M; ++n) {
            const int it = ctx->h_ints[2 + n];
            tot += it;
            mx = std::max(mx, it);
            nsor += ctx->h_ints[2 + M + n] == 1;
            ncap += it >= ctx->opt.lin_max_iter;
        }
        double ss = 0.0;
        for (int b = 0; b < G; ++b) ss += ctx->h_sumsq[b];
        info->upd_rms = std::sqrt(ss / (double)ctx->DOF);
        info->lin_iters_mean = (double)tot / M;
        info->lin_iters_max = mx;
        info->levels_sor = nsor;
        info->levels_capped = ncap;
        info->us_halo_wait = (float)(ctx->h_timers[0] * 1e-3);
        info->us_reduce_wait = (float)(ctx->h_timers[1] * 1e-3);
        info->us_chain = (float)(ctx->h_timers[2] * 1e-3);
    }
    if (status == ST_ETIMEOUT) return fail(ctx, PIT_ETIMEOUT, "chain kernel: a device wait ran out of budget");
    if (status == ST_EDIVERGED) return fail(ctx, PIT_EDIVERGED, "chain kernel: NaN/Inf in a level solve");
    if (status == ST_ENOCONV) return fail(ctx, PIT_ENOCONV, "chain kernel: a level solve hit lin_max_iter");
    return PIT_OK;
}

static bool finite_positive(double v) { return std::isfinite(v) && v > 0.0; }

// The wavefront kernel for a closure and a level-solve precision.
static const void* wave_fn(bool conv, bool nlv, bool fp32) {
    if (fp32) {
        if (conv) return nlv ? reinterpret_cast<const void*>(wave_kernel<kNT, true, true, float>)
                             : reinterpret_cast<const void*>(wave_kernel<kNT, true, false, float>);
        return nlv ? reinterpret_cast<const void*>(wave_kernel<kNT, false, true, float>)
                   : reinterpret_cast<const void*>(wave_kernel<kNT, false, false, float>);
    }
    if (conv) return nlv ? reinterpret_cast<const void*>(wave_kernel<kNT, true, true, double>)
                         : reinterpret_cast<const void*>(wave_kernel<kNT, true, false, double>);
    return nlv ? reinterpret_cast<const void*>(wave_kernel<kNT, false, true, double>)
               : reinterpret_cast<const void*>(wave_kernel<kNT, false, false, double>);
}

// ------------------------------------------------------------------ the ABI

extern "C" pit_status pit_create(const pit_grid* grid, int M, double dt, const pit_params* params,
                                 const pit_options* opt, void* stream, pit_ctx** out) {
    pit_ctx* ctx = nullptr;
    if (!out) return PIT_EINVAL;
    *out = nullptr;
    if (!grid || !params) return PIT_EINVAL;
    if (grid->nx < 1 || grid->ny < 1 || M < 1 || M > 65535 || !finite_positive(dt)) return PIT_EINVAL;
    if (!(grid->xr > grid->xl) || !(grid->yr > grid->yl) || !std::isfinite(grid->xr - grid->xl) ||
        !std::isfinite(grid->yr - grid->yl))
        return PIT_EINVAL;
    if (params->equation != PIT_HEAT && params->equation != PIT_BURGERS) return PIT_EINVAL;
    if (!(params->mu_a >= 0.0) || !(params->mu_b >= 0.0) || !std::isfinite(params->mu_a) ||
        !std::isfinite(params->mu_b))
        return PIT_EINVAL;
    if ((long long)grid->nx * grid->ny > (1ll << 31)) return PIT_EUNSUPPORTED;

    ctx = new (std::nothrow) pit_ctx();
    if (!ctx) return PIT_ENOMEM;
    pit_default_options(&ctx->opt);
    if (opt) ctx->opt = *opt;
    const pit_options& o = ctx->opt;
    if (o.newton_max < 0 || o.newton_max > PIT_MAX_NEWTON || !(o.tol_res >= 0.0) || o.lin_solver < 0 ||
        o.lin_solver > 2 || !(o.eta_max > 0.0) || !(o.eta_gamma >= 0.0) || !(o.lin_atol >= 0.0) ||
        o.lin_max_iter < 1 || !(o.sor_rho_max > 0.0) || o.team_ctas < 0 || o.wait_budget < 1 || o.wave_teams < -1 ||
        o.wave_teams > 64 || (o.precision != PIT_FP64 && o.precision != PIT_FP32_INNER) || o.window < 0 ||
        (o.window_start != PIT_START_PLAIN && o.window_start != PIT_START_GIVEN)) {
        delete ctx;
        return PIT_EINVAL;
    }
    ctx->grid = *grid;
    ctx->M = M;
    ctx->dt = dt;
    ctx->params = *params;
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->Ns = (long long)grid->nx * grid->ny;
    ctx->DOF = ctx->Ns * M;
    ctx->nb = 2 * grid->nx + 2 * grid->ny;
    ctx->conv = params->equation == PIT_BURGERS;
    ctx->nlv = params->mu_b != 0.0;
    const double hx = (grid->xr - grid->xl) / (grid->nx + 1), hy = (grid->yr - grid->yl) / (grid->ny + 1);
    OpConst& c = ctx->oc;
    c.nx = grid->nx;
    c.ny = grid->ny;
    c.M = M;
    c.Ns = ctx->Ns;
    c.dt = dt;
    c.cx = dt / (4.0 * hx);
    c.cy = dt / (4.0 * hy);
    c.jx = dt / (2.0 * hx);
    c.jy = dt / (2.0 * hy);
    c.vx = dt / (hx * hx);
    c.vy = dt / (hy * hy);
    c.mu_a = params->mu_a;
    c.mu_b = params->mu_b;
    c.vmx = c.mu_a * c.vx;
    c.vmy = c.mu_a * c.vy;
    c.kcen = 1.0 + 2.0 * (c.vmx + c.vmy);

    pit_status st = PIT_OK;
    auto setup = [&]() -> pit_status {
        CK(cudaGetDevice(&ctx->device));
        CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device));
        int optin = 0, coop = 0;
        CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
        CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
        if (!coop) return fail(ctx, PIT_EUNSUPPORTED, "device lacks cooperative launch");
        ctx->smem_optin = (size_t)optin;
        // team of G CTAs per level: row strips of rows_per rows
        const int nx = grid->nx, ny = grid->ny;
        int rows_per;
        if (o.team_ctas > 0) {
            const int G = std::min(o.team_ctas, ny);
            rows_per = (ny + G - 1) / G;
        } else {
            rows_per = std::max((ny + ctx->num_sms - 1) / ctx->num_sms, (kMinLocal + nx - 1) / nx);
        }
        rows_per = std::min(rows_per, ny);
        for (;;) {
            const size_t bytes = sizeof(double) * chain_smem_doubles(rows_per * nx, nx);
            if (bytes <= ctx->smem_optin) {
                ctx->chain_smem = bytes;
                break;
            }
            if (rows_per == 1) return fail(ctx, PIT_EUNSUPPORTED, "one grid row (nx = %d) exceeds shared memory", nx);
            rows_per = (rows_per + 1) / 2;  // more, thinner strips
        }
        ctx->G = (ny + rows_per - 1) / rows_per;
        ctx->rows_base = ny / ctx->G;
        ctx->rows_rem = ny % ctx->G;
        // The limit is a property of the kernel, shared by every context in the process:
        // raise it to the device maximum (never lower it to this context's need, which
        // would break the launches of a context created earlier with larger strips).
        {
            cudaFuncAttributes fa;
            CK(cudaFuncGetAttributes(&fa, chain_kernel<kNT>));
            CK(cudaFuncSetAttribute(reinterpret_cast<const void*>(chain_kernel<kNT>),
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(ctx->smem_optin - fa.sharedSizeBytes)));
        }
        int per_sm = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chain_kernel<kNT>, kNT, ctx->chain_smem));
        if ((long long)per_sm * ctx->num_sms < ctx->G)
            return fail(ctx, PIT_EUNSUPPORTED, "team of %d CTAs cannot be co-resident (%d per SM x %d SMs)", ctx->G,
                        per_sm, ctx->num_sms);
        // wavefront teams: K teams of Gw CTAs, one CTA per SM, level strips in shared memory
        if (o.wave_teams >= 0) {
            const bool fp32 = o.precision == PIT_FP32_INNER;
            const void* wf = wave_fn(ctx->conv, ctx->nlv, fp32);
            cudaFuncAttributes fa;
            CK(cudaFuncGetAttributes(&fa, wf));
            const size_t dyn_max = ctx->smem_optin - fa.sharedSizeBytes;
            int K = o.wave_teams == 0 ? 6 : o.wave_teams;  // auto: the most teams (<= 6) that fit
            K = std::max(1, std::min(K, std::max(1, o.newton_max)));
            const int rows_min = (kMinLocal + nx - 1) / nx;
            for (; K >= 1; --K) {
                int Gw = std::min(ctx->num_sms / K, (ny + rows_min - 1) / rows_min);
                if (o.team_ctas > 0) Gw = std::min(Gw, o.team_ctas);
                Gw = std::max(1, std::min(Gw, ny));
                const int rows = (ny + Gw - 1) / Gw;
                Gw = (ny + rows - 1) / rows;
                const size_t bytes = fp32 ? wave_smem_bytes<float>(rows * nx, nx) : wave_smem_bytes<double>(rows * nx, nx);
                if (bytes <= dyn_max && K * Gw <= ctx->num_sms) {
                    ctx->K = K;
                    ctx->Gw = Gw;
                    ctx->w_rows_base = ny / Gw;
                    ctx->w_rows_rem = ny % Gw;
                    ctx->wave_smem = bytes;
                    break;
                }
            }
            // the SMs that K teams of Gw CTAs leave over go to the middle teams (pit_teams.h)
            std::vector<int> geom;
            if (ctx->K > 0) {
                const int K = ctx->K, Gw = ctx->Gw;
                std::vector<int> G(K, Gw);
                ctx->w_ctas = pit_wave_team_sizes(K, Gw, nx, ny, ctx->num_sms, kMinLocal, ny, o.team_ctas, G.data());
                ctx->Gs = *std::max_element(G.begin(), G.end());
                if (ctx->w_ctas != K * Gw) {
                    int first = 0;
                    for (int t = 0; t < K; ++t) {
                        geom.insert(geom.end(), {first, G[t], ny / G[t], ny % G[t]});
                        first += G[t];
                    }
                }
            }
            if (ctx->K > 0) {
                CK(cudaFuncSetAttribute(wf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max));
                int per = 0;
                CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, wf, kNT, ctx->wave_smem));
                if ((long long)per * ctx->num_sms < (long long)ctx->w_ctas) ctx->K = 0;  // fall back
            }
            if (ctx->K > 0) {
                const int K = ctx->K, Gw = ctx->Gw, Gs = ctx->Gs;
                ctx->kcap = std::max(1, o.newton_max);
                if (!geom.empty()) {
                    CK(cudaMalloc(&ctx->w_geom, sizeof(int) * geom.size()));
                    CK(cudaMemcpy(ctx->w_geom, geom.data(), sizeof(int) * geom.size(), cudaMemcpyHostToDevice));
                }
                CK(dalloc(&ctx->w_pub, (size_t)K * 2 * Gs * 2 * nx));
                if (ctx->w_rows_base >= 3 && Gw >= 2) {
                    ctx->w_tpub_n = (size_t)K * 2 * Gs * kDeepSlotRows * nx * 2;
                    ctx->w_tred_n = (size_t)K * 4 * Gs * kTagRedWords;
                    CK(dalloc(&ctx->w_tpub, ctx->w_tpub_n));
                    CK(dalloc(&ctx->w_tred, ctx->w_tred_n));
                }
                CK(dalloc(&ctx->w_red, (size_t)K * 4 * Gs * 4));
                CK(dalloc(&ctx->w_sync, (size_t)K * Gs * 2 + (size_t)K * 4));
                CK(dalloc(&ctx->w_ints, 4));
                CK(dalloc(&ctx->w_res, (size_t)ctx->kcap));
                CK(dalloc(&ctx->w_prefix, (size_t)ctx->kcap * M));
                CK(dalloc(&ctx->w_cell, (size_t)ctx->kcap * M));
                CK(dalloc(&ctx->w_sumsq, (size_t)ctx->kcap * Gs));
                CK(dalloc(&ctx->w_timers, (size_t)K * kWaveTimers));
                ctx->h_wres.assign(ctx->kcap, 0.0);
                ctx->h_wcell.assign((size_t)ctx->kcap * M, 0);
                ctx->h_wsumsq.assign((size_t)ctx->kcap * Gs, 0.0);
                ctx->h_wtimers.assign((size_t)K * kWaveTimers, 0);
            }
        }
        CK(dalloc(&ctx->u0, ctx->Ns));
        CK(cudaMemsetAsync(ctx->u0, 0, sizeof(double) * ctx->Ns, ctx->stream));
        CK(dalloc(&ctx->R, ctx->DOF));
        CK(dalloc(&ctx->coef, 5 * (size_t)ctx->DOF));
        CK(dalloc(&ctx->Uh, ctx->DOF));
        CK(dalloc(&ctx->keys, 2 * (size_t)M + 1));
        CK(dalloc(&ctx->pub, (size_t)2 * ctx->G * 2 * nx));
        CK(dalloc(&ctx->red_part, (size_t)4 * ctx->G * 4));
        CK(dalloc(&ctx->sync_words, (size_t)ctx->G + 4));
        CK(dalloc(&ctx->ints, 2 + 2 * (size_t)M));
        CK(dalloc(&ctx->cta_sumsq, (size_t)ctx->G));
        CK(dalloc(&ctx->timers, 4));
        CK(cudaMemsetAsync(ctx->timers, 0, sizeof(unsigned long long) * 4, ctx->stream));
        ctx->h_ints.assign(2 + 2 * (size_t)M, 0);
        ctx->h_sumsq.assign(ctx->G, 0.0);
        for (auto& e : ctx->ev) CK(cudaEventCreate(&e));
        CK(cudaStreamSynchronize(ctx->stream));
        return PIT_OK;
    };
    st = setup();
    if (st != PIT_OK) {
        fprintf(stderr, "pit_create: %s\n", ctx->err);
        pit_destroy(ctx);
        return st;
    }
    *out = ctx;
    return PIT_OK;
}

extern "C" void pit_destroy(pit_ctx* ctx) {
    if (!ctx) return;
    cudaFree(ctx->u0);
    cudaFree(ctx->bc);
    cudaFree(ctx->q);
    cudaFree(ctx->R);
    cudaFree(ctx->coef);
    cudaFree(ctx->Uh);
    cudaFree(ctx->keys);
    cudaFree(ctx->pub);
    cudaFree(ctx->red_part);
    cudaFree(ctx->sync_words);
    cudaFree(ctx->ints);
    cudaFree(ctx->cta_sumsq);
    cudaFree(ctx->timers);
    cudaFree(ctx->w_pub);
    cudaFree(ctx->w_geom);
    cudaFree(ctx->w_tpub);
    cudaFree(ctx->w_tred);
    cudaFree(ctx->w_red);
    cudaFree(ctx->w_sync);
    cudaFree(ctx->w_ints);
    cudaFree(ctx->w_res);
    cudaFree(ctx->w_prefix);
    cudaFree(ctx->w_cell);
    cudaFree(ctx->w_sumsq);
    cudaFree(ctx->w_timers);
    for (auto& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    delete ctx;
}

extern "C" pit_status pit_set_data(pit_ctx* ctx, const double* u0_dev, const double* bc_dev, const double* q_dev) {
    if (!ctx) return PIT_EINVAL;
    if (!u0_dev) return fail(ctx, PIT_EINVAL, "pit_set_data: u0 is required");
    CK(cudaMemcpyAsync(ctx->u0, u0_dev, sizeof(double) * ctx->Ns, cudaMemcpyDeviceToDevice, ctx->stream));
    if (bc_dev) {
        if (!ctx->bc) CK(dalloc(&ctx->bc, (size_t)ctx->M * ctx->nb));
        CK(cudaMemcpyAsync(ctx->bc, bc_dev, sizeof(double) * ctx->M * ctx->nb, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    ctx->has_bc = bc_dev != nullptr;
    if (q_dev) {
        if (!ctx->q) CK(dalloc(&ctx->q, (size_t)ctx->DOF));
        CK(cudaMemcpyAsync(ctx->q, q_dev, sizeof(double) * ctx->DOF, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    ctx->has_q = q_dev != nullptr;
    return PIT_OK;
}

void pit_internal_view(const pit_ctx* ctx, PitProblemView* v) {
    v->grid = ctx->grid;
    v->M = ctx->M;
    v->dt = ctx->dt;
    v->params = ctx->params;
    v->opt = ctx->opt;
    v->u0 = ctx->u0;
    v->bc = ctx->has_bc ? ctx->bc : nullptr;
    v->q = ctx->has_q ? ctx->q : nullptr;
    v->stream = ctx->stream;
    v->wave_teams = ctx->K;
    v->wave_team_ctas = ctx->Gw;
}

pit_status pit_internal_fail(pit_ctx* ctx, pit_status s, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

extern "C" pit_status pit_fill_plain_guess(pit_ctx* ctx, double* U_dev) {
    if (!ctx) return PIT_EINVAL;
    if (!U_dev) return fail(ctx, PIT_EINVAL, "pit_fill_plain_guess: U is NULL");
    const int blocks = std::max(1, std::min(ctx->num_sms * 8, (int)((ctx->DOF + kNT - 1) / kNT)));
    plain_guess_kernel<<<blocks, kNT, 0, ctx->stream>>>(ctx->u0, U_dev, ctx->Ns, ctx->M);
    CK(cudaGetLastError());
    return PIT_OK;
}

extern "C" pit_status pit_residual(pit_ctx* ctx, const double* U_dev, double* R_dev, double* res_inf) {
    if (!ctx) return PIT_EINVAL;
    if (!U_dev || !R_dev || U_dev == R_dev) return fail(ctx, PIT_EINVAL, "pit_residual: bad U/R pointers");
    CHECK_RET(enqueue_residual(ctx, U_dev, R_dev));
    if (res_inf) CHECK_RET(read_res_inf(ctx, res_inf));
    return PIT_OK;
}

extern "C" pit_status pit_assemble(pit_ctx* ctx, const double* U_dev, double* coef_dev) {
    if (!ctx) return PIT_EINVAL;
    if (!U_dev || !coef_dev) return fail(ctx, PIT_EINVAL, "pit_assemble: NULL pointer");
    return enqueue_assemble<false>(ctx, U_dev, coef_dev);
}

extern "C" pit_status pit_block_solve(pit_ctx* ctx, const double* U_dev, const double* R_dev, double* dU_dev,
                                      double eta, pit_step_info* info) {
    if (!ctx) return PIT_EINVAL;
    if (!U_dev || !R_dev || !dU_dev) return fail(ctx, PIT_EINVAL, "pit_block_solve: NULL pointer");
    if (!(eta > 0.0)) return fail(ctx, PIT_EINVAL, "pit_block_solve: eta must be > 0");
    if (info) std::memset(info, 0, sizeof(*info));
    CHECK_RET(enqueue_assemble<true>(ctx, U_dev, ctx->coef));
    return run_chain(ctx, R_dev, nullptr, dU_dev, eta, 0.0, info);
}

// One Newton update given that ctx->R holds the residual of U and res its max norm.
static pit_status newton_update(pit_ctx* ctx, double* U, double res, pit_step_info* info) {
    // inexact-Newton forcing: relative eta for BiCGStab, absolute eta*||R||_inf for SOR
    const double eta = std::max(std::min(ctx->opt.eta_max, ctx->opt.eta_gamma * res), 1e-300);
    const double sor_tol = std::max(ctx->opt.lin_atol, eta * res);
    CK(cudaEventRecord(ctx->ev[1], ctx->stream));
    CHECK_RET(enqueue_assemble<true>(ctx, U, ctx->coef));
    pit_status st = run_chain(ctx, ctx->R, U, nullptr, eta, sor_tol, info);  // records ev[2], ev[3] around the launch
    if (info) {
        CK(cudaEventSynchronize(ctx->ev[3]));
        CK(cudaEventElapsedTime(&info->ms_residual, ctx->ev[0], ctx->ev[1]));
        CK(cudaEventElapsedTime(&info->ms_assemble, ctx->ev[1], ctx->ev[2]));
        CK(cudaEventElapsedTime(&info->ms_solve, ctx->ev[2], ctx->ev[3]));
    }
    return st;
}

extern "C" pit_status pit_newton_step(pit_ctx* ctx, double* U_dev, pit_step_info* info) {
    if (!ctx) return PIT_EINVAL;
    if (!U_dev) return fail(ctx, PIT_EINVAL, "pit_newton_step: U is NULL");
    if (info) std::memset(info, 0, sizeof(*info));
    CK(cudaEventRecord(ctx->ev[0], ctx->stream));
    CHECK_RET(enqueue_residual(ctx, U_dev, ctx->R));
    double res = 0.0;
    CHECK_RET(read_res_inf(ctx, &res));
    if (info) info->res_inf = res;
    if (!std::isfinite(res)) return fail(ctx, PIT_EDIVERGED, "pit_newton_step: residual is not finite");
    return newton_update(ctx, U_dev, res, info);
}

// One wavefront launch running Newton iterations k_begin <= k < k_end on U. Fills
// info->steps[k] and res_inf[k] for the iterations that completed; *k_done receives
// one past the last completed iteration, *stopped whether a converged iteration
// raised the stop flag.
static pit_status run_wave(pit_ctx* ctx, int s, int Mw, double* Uall, int k_begin, int k_end, pit_solve_info* inf,
                           int* k_done, bool* stopped) {
    const int K = ctx->K, Gs = ctx->Gs, M = Mw;
    double* U = Uall + (size_t)s * ctx->Ns;
    const size_t nsync = (size_t)K * Gs * 2 + (size_t)K * 4;
    CK(cudaMemsetAsync(ctx->w_sync, 0, sizeof(unsigned long long) * nsync, ctx->stream));
    CK(cudaMemsetAsync(ctx->w_ints, 0, sizeof(int) * 3, ctx->stream));
    CK(cudaMemsetAsync(ctx->w_ints + 3, 0x7f, sizeof(int), ctx->stream));  // stop[1] = first converged k: large
    CK(cudaMemsetAsync(ctx->w_cell, 0, sizeof(int) * (size_t)ctx->kcap * M, ctx->stream));
    CK(cudaMemsetAsync(ctx->w_timers, 0, sizeof(unsigned long long) * K * kWaveTimers, ctx->stream));
    // slots of CTAs a smaller team does not have stay zero
    CK(cudaMemsetAsync(ctx->w_sumsq, 0, sizeof(double) * (size_t)ctx->kcap * Gs, ctx->stream));
    if (ctx->w_tpub) {  // tag 0 is never published: stale words of an earlier launch cannot match
        CK(cudaMemsetAsync(ctx->w_tpub, 0, sizeof(unsigned long long) * ctx->w_tpub_n, ctx->stream));
        CK(cudaMemsetAsync(ctx->w_tred, 0, sizeof(unsigned long long) * ctx->w_tred_n, ctx->stream));
    }
    WaveArgs a{};
    a.c = ctx->oc;
    a.c.M = Mw;
    a.u0 = s == 0 ? ctx->u0 : Uall + (size_t)(s - 1) * ctx->Ns;
    a.bc = ctx->has_bc ? ctx->bc + (size_t)s * ctx->nb : nullptr;
    a.q = ctx->has_q ? ctx->q + (size_t)s * ctx->Ns : nullptr;
    a.U = U;
    a.K = K;
    a.G = Gs;
    a.rows_base = ctx->w_rows_base;  // the largest strip (smallest team)
    a.rows_rem = ctx->w_rows_rem;
    a.tgeom = ctx->w_geom;
    a.k_begin = k_begin;
    a.k_end = k_end;
    // bulk copies of the level strips need 16-byte aligned rows: nx even, U aligned
    a.bulk_u = (ctx->grid.nx % 2 == 0) && (reinterpret_cast<uintptr_t>(U) % 16 == 0);
    a.tol_res = ctx->opt.tol_res;
    a.eta_max = ctx->opt.eta_max;
    a.eta_gamma = ctx->opt.eta_gamma;
    a.atol = ctx->opt.lin_atol;
    a.sor_rho_max = ctx->opt.sor_rho_max;
    a.method = ctx->opt.lin_solver;
    a.max_iter = ctx->opt.lin_max_iter;
    a.wait_budget = ctx->opt.wait_budget;
    a.pub = ctx->w_pub;
    a.tpub = ctx->w_tpub;
    a.tred = ctx->w_tred;
    a.red_part = ctx->w_red;
    a.flags = ctx->w_sync;
    a.prog = ctx->w_sync + (size_t)K * Gs;
    a.red_cnt = ctx->w_sync + (size_t)K * Gs * 2;
    a.abort_flag = ctx->w_ints;
    a.status = ctx->w_ints + 1;
    a.stop = ctx->w_ints + 2;
    a.kconv = nullptr;
    a.res_inf = ctx->w_res;
    a.cell_prefix = ctx->w_prefix;
    a.cell_iters = ctx->w_cell;
    a.cta_sumsq = ctx->w_sumsq;
    a.timers = ctx->w_timers;
    void* args[] = {&a};
    const void* kf = wave_fn(ctx->conv, ctx->nlv, ctx->opt.precision == PIT_FP32_INNER);
    CK(cudaEventRecord(ctx->ev[2], ctx->stream));
    CK(cudaLaunchCooperativeKernel(kf, dim3(ctx->w_ctas), dim3(kNT), args, ctx->wave_smem, ctx->stream));
    CK(cudaEventRecord(ctx->ev[3], ctx->stream));
    int hi[4];
    CK(cudaMemcpyAsync(hi, ctx->w_ints, sizeof(hi), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_wres.data(), ctx->w_res, sizeof(double) * ctx->kcap, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_wcell.data(), ctx->w_cell, sizeof(int) * (size_t)ctx->kcap * M, cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_wsumsq.data(), ctx->w_sumsq, sizeof(double) * (size_t)ctx->kcap * Gs,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_wtimers.data(), ctx->w_timers, sizeof(unsigned long long) * K * kWaveTimers,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev[2], ctx->ev[3]));
    inf->ms_wave += ms;
    inf->wave_launches += 1;
    inf->us_pred_wait += (float)(ctx->h_wtimers[2] * 1e-3);
    inf->us_halo_wait += (float)(ctx->h_wtimers[0] * 1e-3);
    inf->us_reduce_wait += (float)(ctx->h_wtimers[1] * 1e-3);
    inf->us_setup += (float)(ctx->h_wtimers[4] * 1e-3);
    inf->us_level_solve += (float)(ctx->h_wtimers[5] * 1e-3);
    inf->us_update += (float)(ctx->h_wtimers[6] * 1e-3);
    *stopped = hi[2] != 0 && hi[3] < k_end;
    // completed iterations: every level of iteration k ran (cell statistics all set)
    int done = k_begin;
    for (int k = k_begin; k < k_end; ++k) {
        bool full = true;
        for (int n = 0; n < M && full; ++n) full = ctx->h_wcell[(size_t)k * M + n] != 0;
        if (!full) break;
        done = k + 1;
        pit_step_info& st = inf->steps[k];
        std::memset(&st, 0, sizeof(st));
        st.res_inf = ctx->h_wres[k];
        inf->res_inf[k] = ctx->h_wres[k];
        long long tot = 0;
        int mx = 0, nsor = 0;
        for (int n = 0; n < M; ++n) {
            const int c = ctx->h_wcell[(size_t)k * M + n];
            const int it = (c < 0 ? -c : c) - 1;
            tot += it;
            mx = std::max(mx, it);
            nsor += c > 0;
        }
        double ss = 0.0;
        for (int b = 0; b < Gs; ++b) ss += ctx->h_wsumsq[(size_t)k * Gs + b];
        st.upd_rms = std::sqrt(ss / (double)((size_t)Mw * ctx->Ns));
        st.lin_iters_mean = (double)tot / M;
        st.lin_iters_max = mx;
        st.levels_sor = nsor;
        if (*stopped && k >= hi[3]) break;
    }
    *k_done = done;
    const int status = hi[1];
    if (status == ST_ETIMEOUT) return fail(ctx, PIT_ETIMEOUT, "wavefront kernel: a device wait ran out of budget");
    if (status == ST_EDIVERGED) return fail(ctx, PIT_EDIVERGED, "wavefront kernel: NaN/Inf in a residual or solve");
    return PIT_OK;  // a capped level solve (ST_ENOCONV) is not fatal: Newton continues
}

// Newton for one window of levels [s, s + Mw) with the wavefront kernel, until the
// window's residual is <= tol_res (the window's first level uses the converged
// level s - 1, or u^0).
static pit_status solve_window(pit_ctx* ctx, double* U_dev, int s, int Mw, pit_solve_info* inf, int* iters) {
    int k = 0;
    for (;;) {
        int k_done = k;
        bool stopped = false;
        if (k < ctx->opt.newton_max) CHECK_RET(run_wave(ctx, s, Mw, U_dev, k, ctx->opt.newton_max, inf, &k_done, &stopped));
        CHECK_RET(enqueue_residual_range(ctx, s, Mw, U_dev, ctx->R));
        double res = 0.0;
        CHECK_RET(read_res_inf(ctx, &res));
        inf->res_inf[k_done] = res;
        *iters = k_done;
        if (!std::isfinite(res))
            return fail(ctx, PIT_EDIVERGED, "pit_solve: residual of levels %d..%d is not finite", s, s + Mw - 1);
        if (res <= ctx->opt.tol_res) return PIT_OK;
        if (k_done >= ctx->opt.newton_max || k_done == k)
            return fail(ctx, PIT_ENOCONV, "pit_solve: ||R||_inf = %.3e > %.3e on levels %d..%d after %d Newton updates",
                        res, ctx->opt.tol_res, s, s + Mw - 1, k_done);
        k = k_done;  // continue Newton from the current iterate
    }
}

static pit_status fill_window_guess(pit_ctx* ctx, double* U_dev, int s, int Mw) {
    const double* from = s == 0 ? ctx->u0 : U_dev + (size_t)(s - 1) * ctx->Ns;
    const int blocks = std::max(1, std::min(ctx->num_sms * 8, (int)(((size_t)Mw * ctx->Ns + kNT - 1) / kNT)));
    plain_guess_kernel<<<blocks, kNT, 0, ctx->stream>>>(from, U_dev + (size_t)s * ctx->Ns, ctx->Ns, Mw);
    CK(cudaGetLastError());
    return PIT_OK;
}

// Levels in windows (all M at once when window = 0). A window whose Newton diverges
// or does not converge is halved and restarted from the plain guess at its first
// level (the solution is the same: the system is block lower-triangular in time);
// after a success the window grows back toward its nominal length.
static pit_status solve_wave(pit_ctx* ctx, double* U_dev, pit_solve_info* inf) {
    inf->wave_teams = ctx->K;
    inf->wave_team_ctas = ctx->Gw;
    inf->wave_ctas = ctx->K > 0 ? ctx->w_ctas : 0;
    const int M = ctx->M;
    const int Wn = ctx->opt.window > 0 ? std::min(ctx->opt.window, M) : M;
    int w = Wn;
    // the caller's iterate is the start of the first attempt over all levels, and of every
    // window with PIT_START_GIVEN, except on levels a failed attempt has overwritten
    const bool given = Wn == M || ctx->opt.window_start == PIT_START_GIVEN;
    int clean_from = 0;  // levels >= clean_from still hold the caller's iterate
    bool whole = false;  // one window over all levels converged: its residual is the final one
    for (int s = 0; s < M;) {
        const int Mw = std::min(w, M - s);
        if (!(given && s >= clean_from)) CHECK_RET(fill_window_guess(ctx, U_dev, s, Mw));
        int iters = 0;
        const pit_status st = solve_window(ctx, U_dev, s, Mw, inf, &iters);
        whole = st == PIT_OK && s == 0 && Mw == M;
        if (st != PIT_OK) clean_from = std::max(clean_from, s + Mw);
        inf->windows += 1;
        inf->newton_iters_total += iters;
        inf->newton_iters = std::max(inf->newton_iters, iters);
        if (st == PIT_OK) {
            inf->windows_converged += 1;
            s += Mw;
            w = std::min(Wn, 2 * w);
        } else if ((st == PIT_ENOCONV || st == PIT_EDIVERGED) && Mw > 1) {
            w = std::max(1, Mw / 2);
        } else {
            return st;
        }
    }
    // the residual of the whole final iterate decides convergence (already computed, on the
    // same iterate, when one window spanned every level)
    if (whole) {
        inf->converged = 1;
        return PIT_OK;
    }
    CHECK_RET(enqueue_residual(ctx, U_dev, ctx->R));
    double res = 0.0;
    CHECK_RET(read_res_inf(ctx, &res));
    inf->res_inf[inf->newton_iters] = res;
    if (!std::isfinite(res)) return fail(ctx, PIT_EDIVERGED, "pit_solve: final residual is not finite");
    if (res <= ctx->opt.tol_res) {
        inf->converged = 1;
        return PIT_OK;
    }
    return fail(ctx, PIT_ENOCONV, "pit_solve: final ||R||_inf = %.3e > %.3e", res, ctx->opt.tol_res);
}

extern "C" pit_status pit_solve(pit_ctx* ctx, double* U_dev, pit_solve_info* info) {
    if (!ctx) return PIT_EINVAL;
    if (!U_dev) return fail(ctx, PIT_EINVAL, "pit_solve: U is NULL");
    if (ctx->K > 0) {
        pit_solve_info local;
        pit_solve_info* inf = info ? info : &local;
        std::memset(inf, 0, sizeof(*inf));
        cudaEvent_t t0 = nullptr, t1 = nullptr;
        CK(cudaEventCreate(&t0));
        CK(cudaEventCreate(&t1));
        CK(cudaEventRecord(t0, ctx->stream));
        pit_status st = solve_wave(ctx, U_dev, inf);
        CK(cudaEventRecord(t1, ctx->stream));
        CK(cudaEventSynchronize(t1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, t0, t1));
        inf->ms_total = ms;
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        return st;
    }
    pit_solve_info local;
    pit_solve_info* inf = info ? info : &local;
    std::memset(inf, 0, sizeof(*inf));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    CK(cudaEventCreate(&t0));
    CK(cudaEventCreate(&t1));
    CK(cudaEventRecord(t0, ctx->stream));
    pit_status st = PIT_OK;
    for (int k = 0;; ++k) {
        CK(cudaEventRecord(ctx->ev[0], ctx->stream));
        st = enqueue_residual(ctx, U_dev, ctx->R);
        double res = 0.0;
        if (st == PIT_OK) st = read_res_inf(ctx, &res);
        if (st != PIT_OK) break;
        inf->res_inf[k] = res;
        if (!std::isfinite(res)) {
            st = fail(ctx, PIT_EDIVERGED, "pit_solve: residual is not finite at Newton iteration %d", k);
            break;
        }
        if (res <= ctx->opt.tol_res) {
            inf->converged = 1;
            break;
        }
        if (k >= ctx->opt.newton_max) {
            st = fail(ctx, PIT_ENOCONV, "pit_solve: ||R||_inf = %.3e > %.3e after %d Newton updates", res,
                      ctx->opt.tol_res, k);
            break;
        }
        inf->steps[k].res_inf = res;
        st = newton_update(ctx, U_dev, res, &inf->steps[k]);
        inf->newton_iters = k + 1;
        if (st == PIT_ENOCONV) st = PIT_OK;  // a capped level solve: Newton carries on
        if (st != PIT_OK) break;
    }
    inf->windows = 1;
    inf->windows_converged = inf->converged;
    inf->newton_iters_total = inf->newton_iters;
    CK(cudaEventRecord(t1, ctx->stream));
    CK(cudaEventSynchronize(t1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, t0, t1));
    inf->ms_total = ms;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return st;
}

extern "C" int pit_wave_timers(const pit_ctx* ctx, unsigned long long* out, int n) {
    if (!ctx || !out || n < 0) return -1;
    const int have = (int)ctx->h_wtimers.size();
    for (int i = 0; i < n && i < have; ++i) out[i] = ctx->h_wtimers[i];
    return have;
}

extern "C" pit_status pit_solve_host(pit_ctx* ctx, const double* u0_host, double* U_host, pit_solve_info* info) {
    if (!ctx) return PIT_EINVAL;
    if (!u0_host || !U_host) return fail(ctx, PIT_EINVAL, "pit_solve_host: NULL pointer");
    CK(cudaMemcpyAsync(ctx->u0, u0_host, sizeof(double) * ctx->Ns, cudaMemcpyHostToDevice, ctx->stream));
    CHECK_RET(pit_fill_plain_guess(ctx, ctx->Uh));
    pit_status st = pit_solve(ctx, ctx->Uh, info);
    CK(cudaMemcpyAsync(U_host, ctx->Uh, sizeof(double) * ctx->DOF, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return st;
}
