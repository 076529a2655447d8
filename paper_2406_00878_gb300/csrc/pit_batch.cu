// pit_batch.cu -- many independent problems in one persistent cooperative launch.
//
// Each problem is a job of the launch (batch_kernel in pit_kernels.cuh): the level
// chain (nested block inverse of eq. 7) with Newton iterations per window of levels
// until the window's residual is below tol_res, then a final FP64 residual pass.
// A problem on a large grid is a wavefront job: K teams of G CTAs, nearly the whole
// GPU, keep K Newton iterations of its window in flight, and such jobs run one after
// another at the start of the launch. Every other problem gets a single team, and
// teams of different sizes run side by side on the remaining SMs and afterwards.
// Here: the routing, the autotuner that picks a team size per packed problem from
// short timed runs, the list schedule that places the jobs on the SMs, the workspace
// pools, and the launch, which is captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <map>
#include <numeric>
#include <cstdlib>
#include <vector>

#include "pit.h"
#include "pit_kernels.cuh"
#include "pit_teams.h"

using namespace pit;

namespace {
constexpr int kNT = kBatchThreads;
constexpr int kMaxTeam = 160;
constexpr int kMinLocal = 256;   // wavefront teams: at least this many unknowns per CTA
constexpr int kMaxWaveTeams = 6;
}

struct pit_batch {
    int count = 0;
    pit_options opt{};
    cudaStream_t stream = nullptr;       // the batch's own stream (capturable)
    cudaStream_t user_stream = nullptr;  // the caller's stream: the batch's work is ordered after it
    cudaEvent_t ev_user = nullptr;
    int num_sms = 0;
    size_t dyn_max = 0;
    bool fp32 = false;
    std::vector<pit_instance> in;
    std::vector<int> team_of;          // CTAs per team, per problem
    std::vector<int> teams_of;         // teams per problem: K for a wavefront job, 1 otherwise
    int wave_jobs = 0;
    int closures = 0;                  // set of the problems' closures (closure_bit)
    const void* kfn = nullptr;         // the batched kernel compiled for that set
    // device data
    BatchInstance* d_inst = nullptr;
    BatchJob* d_jobs = nullptr;
    int* d_job_off = nullptr;
    BatchTeamWs* d_ws = nullptr;
    int* d_geom = nullptr;             // team sizes of the wavefront jobs whose teams differ (BatchTeamWs::tgeom)
    unsigned char* pool = nullptr;     // job workspaces
    size_t pool_bytes = 0, sync_bytes = 0;  // sync region (zeroed per launch) at the start of the pool
    double* d_res = nullptr;
    int* d_iters = nullptr;            // [count] iters, [count] converged windows
    int* d_ctl = nullptr;              // abort, status
    int ctas = 0;
    size_t smem = 0;
    // results (pinned)
    double* h_res = nullptr;
    int* h_iters = nullptr;
    int* h_ctl = nullptr;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool graph_ok = true;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double est_ms = 0.0, ms_tuning = 0.0;
    int min_team = 0, max_team = 0;
    bool calibrating = false;          // autotuner runs: plain starts on scratch iterates
    // problems of several closures or kinds: one batch per closure and kind (wavefront job or
    // single team), solved one after another (a kernel holding several closures' wave bodies
    // ran each job 20-25 % slower than the kernel of its own closure); problem i is problem
    // where[i].second of parts[where[i].first]
    std::vector<pit_batch*> parts;
    std::vector<std::pair<int, int>> where;
    char err[512] = "";
};

static pit_status bfail(pit_batch* b, pit_status s, const char* fmt, ...) {
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define BCK(call)                                                                                          \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? PIT_ENOMEM : PIT_ECUDA, "%s: %s (%s:%d)", #call, \
                         cudaGetErrorString(e_), __FILE__, __LINE__);                                      \
    } while (0)

#define BRET(expr)                  \
    do {                            \
        pit_status s_ = (expr);     \
        if (s_ != PIT_OK) return s_; \
    } while (0)

// The batched kernel of every precision and closure, one per compilation of
// pit_batch_kernels.cu: pit_batch_kernel_<fp32>_<closure bit>(). A batch holds problems of
// one closure (pit_batch_create splits mixed sets).
#define PIT_BK_SETS(X, f) X(f, 1) X(f, 2) X(f, 4) X(f, 8)
#define PIT_BK_DECL(f, c) __attribute__((visibility("hidden"))) const void* pit_batch_kernel_##f##_##c();
PIT_BK_SETS(PIT_BK_DECL, 0)
PIT_BK_SETS(PIT_BK_DECL, 1)

static const void* batch_fn(bool fp32, int closures) {
    switch (closures) {
#define PIT_BK_CASE(f, c) \
    case c:               \
        return fp32 ? pit_batch_kernel_1_##c() : pit_batch_kernel_0_##c();
        PIT_BK_SETS(PIT_BK_CASE, 0)
#undef PIT_BK_CASE
        default:
            return nullptr;
    }
}

static size_t team_smem(bool fp32, int nx, int ny, int G) {
    const int rows = (ny + G - 1) / G;
    return fp32 ? wave_smem_bytes<float>(rows * nx, nx) : wave_smem_bytes<double>(rows * nx, nx);
}

// Bytes of one job's workspace (K teams of G CTAs): sync part (job barrier; kconv,
// stop and abort words; flags, prog, red_cnt; tagged words; zeroed before each
// launch) and data part (halo rows, reduction partials, per-cell running maxima).
struct WsSize {
    size_t sync_head, sync, data;
};
static size_t tagged_words(int K, int G, int nx) {
    return (size_t)K * ((size_t)2 * G * kDeepSlotRows * nx * 2 + (size_t)4 * G * kTagRedWords);
}
static WsSize ws_size(int K, int G, int nx, int newton_max, int window) {
    WsSize w;
    w.sync_head = align_up(sizeof(unsigned long long) * (5 + (size_t)K * G * 2 + (size_t)K * 4), 256);
    w.sync = w.sync_head + align_up(sizeof(unsigned long long) * tagged_words(K, G, nx), 256);
    w.data = align_up(sizeof(double) * ((size_t)K * 2 * G * 2 * nx + (size_t)K * 4 * G * 4 + (size_t)newton_max * window),
                      256);
    return w;
}

// Wavefront shape of a large problem: the most teams (<= 6, <= newton_max) whose
// strips of at least kMinLocal unknowns fit in shared memory with K * G <= SMs.
static bool wave_shape(const pit_batch* b, const pit_instance& I, int* K_out, int* G_out) {
    const int nx = I.grid.nx, ny = I.grid.ny;
    const int rows_min = (kMinLocal + nx - 1) / nx;
    for (int K = std::min(kMaxWaveTeams, std::max(1, b->opt.newton_max)); K >= 2; --K) {
        int G = std::min(b->num_sms / K, (ny + rows_min - 1) / rows_min);
        G = std::max(1, std::min({G, ny, kMaxTeam}));
        const int rows = (ny + G - 1) / G;
        G = (ny + rows - 1) / rows;
        if (team_smem(b->fp32, nx, ny, G) <= b->dyn_max && K * G <= b->num_sms) {
            *K_out = K;
            *G_out = G;
            return true;
        }
    }
    return false;
}

struct Job {
    int inst, G, K;
    double start, dur;
    std::vector<int> size, first;  // per team: CTAs (G, or more for the middle teams of a wavefront
                                   // job where SMs are left over) and the first one's index
    int width = 0, Gs = 0;         // CTAs of the job, the largest team's size
    std::vector<int> ctas;         // team tk, rank r -> ctas[first[tk] + r]
};

// Team sizes of a job of K teams of G CTAs on P SMs: the SMs the teams leave over go to the
// middle teams, as in the single-problem wavefront launch (pit_teams.h).
static void team_sizes(Job& j, int nx, int ny, int P, int fixed) {
    j.size.assign(j.K, j.G);
    j.width = pit_wave_team_sizes(j.K, j.G, nx, ny, P, kMinLocal, kMaxTeam, fixed, j.size.data());
    j.first.assign(j.K, 0);
    j.Gs = 0;
    for (int t = 0, f = 0; t < j.K; ++t) {
        j.first[t] = f;
        f += j.size[t];
        j.Gs = std::max(j.Gs, j.size[t]);
    }
}

// Build jobs, workspace and device descriptors for problems `in` with K[i] teams of
// G[i] CTAs each (K[i] > 1: a wavefront job, placed first on CTAs 0 .. K G - 1, one
// after another; the other jobs are list-scheduled over the SMs after them, longest
// first);
// problem i reports into result slot gid[i] (calibration runs use one problem with
// truncated levels and slot 0).
static pit_status build_launch(pit_batch* b, const std::vector<pit_instance>& in, const std::vector<int>& team,
                               const std::vector<int>& teams, const std::vector<double>& cost,
                               const std::vector<int>& gid) {
    const int n = (int)in.size();
    const int P = b->num_sms;
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        if ((teams[a] > 1) != (teams[c] > 1)) return teams[a] > 1;  // wavefront jobs first
        return cost[a] > cost[c];
    });
    std::vector<double> free_at(P, 0.0);
    std::vector<Job> jobs;
    bool wave_phase = true;
    for (int i : order) {
        if (wave_phase && teams[i] == 1) {
            // the single teams start when the wavefront jobs are done, on every SM: their
            // cost estimates are rough, and teams packed beside them on the few SMs left
            // over would form a tail
            wave_phase = false;
            const double t0 = *std::max_element(free_at.begin(), free_at.end());
            std::fill(free_at.begin(), free_at.end(), t0);
        }
        Job j;
        j.inst = i;
        j.G = team[i];
        j.K = teams[i];
        team_sizes(j, in[i].grid.nx, in[i].grid.ny, P, b->opt.team_ctas);
        const int width = j.width;
        if (j.K > 1) {
            j.ctas.resize(width);
            std::iota(j.ctas.begin(), j.ctas.end(), 0);
        } else {
            // a team takes the G CTAs that free up earliest
            std::vector<int> idx(P);
            std::iota(idx.begin(), idx.end(), 0);
            std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return free_at[a] < free_at[c]; });
            j.ctas.assign(idx.begin(), idx.begin() + width);
            std::sort(j.ctas.begin(), j.ctas.end());
        }
        double start = 0.0;
        for (int c : j.ctas) start = std::max(start, free_at[c]);
        j.start = start;
        j.dur = cost[i];
        for (int c : j.ctas) free_at[c] = start + cost[i];
        jobs.push_back(j);
    }
    b->est_ms = *std::max_element(free_at.begin(), free_at.end());
    // CTAs used and their job lists, in the global (assignment) order
    int used = 0;
    for (const Job& j : jobs)
        for (int c : j.ctas) used = std::max(used, c + 1);
    std::vector<std::vector<BatchJob>> per(used);
    std::vector<WsSize> wss(jobs.size());
    size_t sync_total = 0, data_total = 0;
    const int W = b->opt.window > 0 ? b->opt.window : 32;
    for (size_t q = 0; q < jobs.size(); ++q) {
        const Job& j = jobs[q];
        const pit_instance& I = in[j.inst];
        wss[q] = ws_size(j.K, j.Gs, I.grid.nx, b->opt.newton_max, std::min(W, I.M));
        sync_total += wss[q].sync;
        data_total += wss[q].data;
        for (int tk = 0; tk < j.K; ++tk)
            for (int r = 0; r < j.size[tk]; ++r)
                per[j.ctas[(size_t)j.first[tk] + r]].push_back(
                    BatchJob{j.inst, r, j.size[tk], (int)q, j.K, tk, j.first[tk], j.width, j.Gs});
    }
    // the geometry of the jobs whose teams differ in size (first CTA, CTAs, strips)
    std::vector<int> geom;
    std::vector<long long> geom_at(jobs.size(), -1);
    for (size_t q = 0; q < jobs.size(); ++q) {
        const Job& j = jobs[q];
        if (j.K < 2 || j.width == j.K * j.G) continue;
        const int ny = in[j.inst].grid.ny;
        geom_at[q] = (long long)geom.size();
        for (int t = 0; t < j.K; ++t) geom.insert(geom.end(), {j.first[t], j.size[t], ny / j.size[t], ny % j.size[t]});
    }
    // device buffers (freed and rebuilt for every build)
    cudaFree(b->pool);
    cudaFree(b->d_jobs);
    cudaFree(b->d_job_off);
    cudaFree(b->d_ws);
    cudaFree(b->d_inst);
    cudaFree(b->d_geom);
    b->pool = nullptr;
    b->d_jobs = nullptr;
    b->d_job_off = nullptr;
    b->d_ws = nullptr;
    b->d_inst = nullptr;
    b->d_geom = nullptr;
    if (!geom.empty()) {
        BCK(cudaMalloc(&b->d_geom, sizeof(int) * geom.size()));
        BCK(cudaMemcpy(b->d_geom, geom.data(), sizeof(int) * geom.size(), cudaMemcpyHostToDevice));
    }
    b->pool_bytes = sync_total + data_total;
    b->sync_bytes = sync_total;
    BCK(cudaMalloc(&b->pool, b->pool_bytes));
    std::vector<BatchTeamWs> ws(jobs.size());
    size_t so = 0, dof = sync_total;
    for (size_t q = 0; q < jobs.size(); ++q) {
        const int K = jobs[q].K, G = jobs[q].Gs, nx = in[jobs[q].inst].grid.nx;  // G: the workspace stride
        unsigned long long* sw = reinterpret_cast<unsigned long long*>(b->pool + so);
        ws[q].jbar = sw;
        ws[q].jres = sw + 1;
        ws[q].kconv = reinterpret_cast<int*>(sw + 2);  // kconv, stop[2], jabort, jstatus
        ws[q].stop = ws[q].kconv + 1;
        ws[q].jabort = ws[q].kconv + 3;
        ws[q].jstatus = ws[q].kconv + 4;
        ws[q].flags = sw + 5;
        ws[q].prog = sw + 5 + (size_t)K * G;
        ws[q].red_cnt = sw + 5 + (size_t)2 * K * G;
        ws[q].sync_words = sw + 5;
        ws[q].sync_count = wss[q].sync / sizeof(unsigned long long) - 5;
        unsigned long long* tw = reinterpret_cast<unsigned long long*>(b->pool + so + wss[q].sync_head);
        ws[q].tpub = tw;
        ws[q].tred = tw + (size_t)K * 2 * G * kDeepSlotRows * nx * 2;
        so += wss[q].sync;
        double* dw = reinterpret_cast<double*>(b->pool + dof);
        ws[q].pub = dw;
        ws[q].red_part = dw + (size_t)K * 2 * G * 2 * nx;
        ws[q].cell_prefix = ws[q].red_part + (size_t)K * 4 * G * 4;
        ws[q].tgeom = geom_at[q] >= 0 ? b->d_geom + geom_at[q] : nullptr;
        dof += wss[q].data;
    }
    std::vector<BatchJob> flat;
    std::vector<int> off(used + 1, 0);
    for (int c = 0; c < used; ++c) {
        off[c] = (int)flat.size();
        flat.insert(flat.end(), per[c].begin(), per[c].end());
    }
    off[used] = (int)flat.size();
    std::vector<BatchInstance> bi(n);
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
        const pit_instance& I = in[i];
        const double hx = (I.grid.xr - I.grid.xl) / (I.grid.nx + 1), hy = (I.grid.yr - I.grid.yl) / (I.grid.ny + 1);
        OpConst& c = bi[i].c;
        c.nx = I.grid.nx;
        c.ny = I.grid.ny;
        c.M = I.M;
        c.Ns = (long long)I.grid.nx * I.grid.ny;
        c.dt = I.dt;
        c.cx = I.dt / (4.0 * hx);
        c.cy = I.dt / (4.0 * hy);
        c.jx = I.dt / (2.0 * hx);
        c.jy = I.dt / (2.0 * hy);
        c.vx = I.dt / (hx * hx);
        c.vy = I.dt / (hy * hy);
        c.mu_a = I.params.mu_a;
        c.mu_b = I.params.mu_b;
        c.vmx = c.mu_a * c.vx;
        c.vmy = c.mu_a * c.vy;
        c.kcen = 1.0 + 2.0 * (c.vmx + c.vmy);
        bi[i].conv = I.params.equation == PIT_BURGERS;
        bi[i].nlv = I.params.mu_b != 0.0;
        bi[i].window = std::min(W, I.M);
        bi[i].bulk_u = (I.grid.nx % 2 == 0) && (reinterpret_cast<uintptr_t>(I.U_dev) % 16 == 0);
        bi[i].u0 = I.u0_dev;
        bi[i].bc = I.bc_dev;
        bi[i].q = I.q_dev;
        bi[i].U = I.U_dev;
        bi[i].res_inf = b->d_res + gid[i];
        bi[i].newton_iters = b->d_iters + gid[i];
        bi[i].converged_windows = b->d_iters + b->count + gid[i];
        smem = std::max(smem, team_smem(b->fp32, I.grid.nx, I.grid.ny, team[i]));
    }
    b->smem = smem;
    b->ctas = used;
    BCK(cudaMalloc(&b->d_inst, sizeof(BatchInstance) * n));
    BCK(cudaMalloc(&b->d_jobs, sizeof(BatchJob) * std::max<size_t>(flat.size(), 1)));
    BCK(cudaMalloc(&b->d_job_off, sizeof(int) * (used + 1)));
    BCK(cudaMalloc(&b->d_ws, sizeof(BatchTeamWs) * std::max<size_t>(ws.size(), 1)));
    BCK(cudaMemcpy(b->d_inst, bi.data(), sizeof(BatchInstance) * n, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_jobs, flat.data(), sizeof(BatchJob) * flat.size(), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_job_off, off.data(), sizeof(int) * (used + 1), cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->d_ws, ws.data(), sizeof(BatchTeamWs) * ws.size(), cudaMemcpyHostToDevice));
    b->min_team = *std::min_element(team.begin(), team.end());
    b->max_team = 0;
    for (const Job& j : jobs) b->max_team = std::max(b->max_team, j.Gs);
    return PIT_OK;
}

static pit_status enqueue_launch(pit_batch* b, bool timed) {
    BCK(cudaMemsetAsync(b->pool, 0, b->sync_bytes, b->stream));
    BCK(cudaMemsetAsync(b->d_ctl, 0, sizeof(int) * 2, b->stream));
    BatchArgs a{};
    a.inst = b->d_inst;
    a.jobs = b->d_jobs;
    a.job_off = b->d_job_off;
    a.ws = b->d_ws;
    a.abort_flag = b->d_ctl;
    a.status = b->d_ctl + 1;
    a.newton_max = b->opt.newton_max;
    a.tol_res = b->opt.tol_res;
    a.eta_max = b->opt.eta_max;
    a.eta_gamma = b->opt.eta_gamma;
    a.atol = b->opt.lin_atol;
    a.sor_rho_max = b->opt.sor_rho_max;
    a.method = b->opt.lin_solver;
    a.max_iter = b->opt.lin_max_iter;
    a.wait_budget = b->opt.wait_budget;
    a.start_given = b->opt.window_start == PIT_START_GIVEN && !b->calibrating;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(b->ctas);
    cfg.blockDim = dim3(kNT);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (timed) BCK(cudaEventRecord(b->e0, b->stream));
    BCK(cudaLaunchKernelEx(&cfg, reinterpret_cast<void (*)(BatchArgs)>(const_cast<void*>(b->kfn)), a));
    if (timed) BCK(cudaEventRecord(b->e1, b->stream));
    BCK(cudaMemcpyAsync(b->h_res, b->d_res, sizeof(double) * b->count, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaMemcpyAsync(b->h_iters, b->d_iters, sizeof(int) * 2 * b->count, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(int) * 2, cudaMemcpyDeviceToHost, b->stream));
    return PIT_OK;
}

static pit_status run_direct(pit_batch* b, double* ms) {
    BRET(enqueue_launch(b, true));
    BCK(cudaStreamSynchronize(b->stream));
    float f = 0.f;
    BCK(cudaEventElapsedTime(&f, b->e0, b->e1));
    *ms = f;
    if (b->h_ctl[1] == ST_ETIMEOUT) return bfail(b, PIT_ETIMEOUT, "batch kernel: a device wait ran out of budget");
    if (b->h_ctl[1] == ST_EDIVERGED) return bfail(b, PIT_EDIVERGED, "batch kernel: NaN/Inf in a problem");
    return PIT_OK;
}

extern "C" pit_status pit_batch_create(const pit_instance* inst, int count, const pit_options* opt, void* stream,
                                       pit_batch** out) {
    if (!out) return PIT_EINVAL;
    *out = nullptr;
    if (!inst || count < 1) return PIT_EINVAL;
    pit_batch* b = new (std::nothrow) pit_batch();
    if (!b) return PIT_ENOMEM;
    pit_default_options(&b->opt);
    if (opt) b->opt = *opt;
    if (b->opt.window <= 0) b->opt.window = 32;
    if (b->opt.window_start != PIT_START_PLAIN && b->opt.window_start != PIT_START_GIVEN) {
        delete b;
        return PIT_EINVAL;
    }
    b->count = count;
    b->user_stream = static_cast<cudaStream_t>(stream);
    b->fp32 = b->opt.precision == PIT_FP32_INNER;
    b->in.assign(inst, inst + count);
    {
        // several closures, or wavefront jobs beside single teams: a batch per closure and
        // kind, solved one after another (one launch mixing them measured slower than the
        // separate launches together: 2019 against 1412 + 427 ms on the 64-problem workload)
        auto key = [&](const pit_instance& I) {
            const int bit = closure_bit(I.params.equation == PIT_BURGERS, I.params.mu_b != 0.0);
            const bool wave = b->opt.batch_wave_nodes > 0 && (long long)I.grid.nx * I.grid.ny >= b->opt.batch_wave_nodes;
            return 2 * bit + (wave ? 1 : 0);
        };
        unsigned long long keys = 0;  // bit 2 * closure_bit + wave: at most 2 * 8 + 1 = 17
        for (int i = 0; i < count; ++i) {
            const pit_instance& I = inst[i];
            if (I.params.equation != PIT_HEAT && I.params.equation != PIT_BURGERS) {
                delete b;
                return PIT_EINVAL;
            }
            keys |= 1ull << key(I);
        }
        if (keys & (keys - 1)) {
            b->where.resize(count);
            for (int k = 0; k < 64; ++k) {
                if (!(keys >> k & 1)) continue;
                std::vector<pit_instance> sub;
                for (int i = 0; i < count; ++i)
                    if (key(inst[i]) == k) {
                        b->where[i] = {(int)b->parts.size(), (int)sub.size()};
                        sub.push_back(inst[i]);
                    }
                pit_batch* part = nullptr;
                const pit_status st = pit_batch_create(sub.data(), (int)sub.size(), opt, stream, &part);
                if (st != PIT_OK) {
                    for (pit_batch* q : b->parts) pit_batch_destroy(q);
                    delete b;
                    return st;
                }
                b->parts.push_back(part);
            }
            for (pit_batch* q : b->parts) {
                b->wave_jobs += q->wave_jobs;
                b->ms_tuning += q->ms_tuning;
                b->est_ms += q->est_ms;
                b->ctas = std::max(b->ctas, q->ctas);
                b->min_team = b->min_team ? std::min(b->min_team, q->min_team) : q->min_team;
                b->max_team = std::max(b->max_team, q->max_team);
            }
            *out = b;
            return PIT_OK;
        }
    }
    const auto t_start = std::chrono::steady_clock::now();
    auto setup = [&]() -> pit_status {
        if (b->opt.newton_max < 1 || b->opt.newton_max > PIT_MAX_NEWTON || b->opt.lin_max_iter < 1 ||
            b->opt.wait_budget < 1 || b->opt.team_ctas < 0)
            return bfail(b, PIT_EINVAL, "invalid options");
        for (int i = 0; i < count; ++i) {
            const pit_instance& I = inst[i];
            if (I.grid.nx < 1 || I.grid.ny < 1 || I.M < 1 || !(I.dt > 0.0) || !(I.grid.xr > I.grid.xl) ||
                !(I.grid.yr > I.grid.yl) || !I.u0_dev || !I.U_dev || !(I.params.mu_a >= 0.0) ||
                !(I.params.mu_b >= 0.0) || (I.params.equation != PIT_HEAT && I.params.equation != PIT_BURGERS))
                return bfail(b, PIT_EINVAL, "problem %d: invalid grid, levels, step, parameters or pointers", i);
        }
        int dev = 0, optin = 0, coop = 0;
        BCK(cudaGetDevice(&dev));
        BCK(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev));
        BCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        BCK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        if (!coop) return bfail(b, PIT_EUNSUPPORTED, "device lacks cooperative launch");
        // the kernel compiled for exactly this batch's closures
        for (int i = 0; i < count; ++i)
            b->closures |= closure_bit(inst[i].params.equation == PIT_BURGERS, inst[i].params.mu_b != 0.0);
        b->kfn = batch_fn(b->fp32, b->closures);
        if (!b->kfn) return bfail(b, PIT_EUNSUPPORTED, "no batched kernel for closure set %d", b->closures);
        cudaFuncAttributes fa;
        BCK(cudaFuncGetAttributes(&fa, b->kfn));
        b->dyn_max = (size_t)optin - fa.sharedSizeBytes;
        BCK(cudaFuncSetAttribute(b->kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->dyn_max));
        int per = 0;
        BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, b->kfn, kNT, b->dyn_max));
        if (per < 1) return bfail(b, PIT_EUNSUPPORTED, "batch kernel does not fit on an SM");
        BCK(cudaMalloc(&b->d_res, sizeof(double) * count));
        BCK(cudaMalloc(&b->d_iters, sizeof(int) * 2 * count));
        BCK(cudaMalloc(&b->d_ctl, sizeof(int) * 2));
        BCK(cudaMallocHost(&b->h_res, sizeof(double) * count));
        BCK(cudaMallocHost(&b->h_iters, sizeof(int) * 2 * count));
        BCK(cudaMallocHost(&b->h_ctl, sizeof(int) * 2));
        BCK(cudaEventCreate(&b->e0));
        BCK(cudaEventCreate(&b->e1));
        BCK(cudaEventCreateWithFlags(&b->ev_user, cudaEventDisableTiming));
        BCK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        BCK(cudaEventRecord(b->ev_user, b->user_stream));
        BCK(cudaStreamWaitEvent(b->stream, b->ev_user, 0));
        // routing: a large grid becomes a wavefront job when a wavefront shape fits
        b->teams_of.assign(count, 1);
        std::vector<int> team(count, 0);
        for (int i = 0; i < count; ++i) {
            const pit_instance& I = inst[i];
            const long long nodes = (long long)I.grid.nx * I.grid.ny;
            int K = 0, G = 0;
            if (b->opt.batch_wave_nodes > 0 && nodes >= b->opt.batch_wave_nodes && wave_shape(b, I, &K, &G)) {
                b->teams_of[i] = K;
                team[i] = G;
                ++b->wave_jobs;
            }
        }
        const std::vector<int>& teams = b->teams_of;
        // smallest team whose strips fit in shared memory, per packed problem
        std::vector<int> gmin(count, 1);
        for (int i = 0; i < count; ++i) {
            if (teams[i] > 1) continue;
            const pit_instance& I = inst[i];
            int g = 1;
            while (g <= std::min(I.grid.ny, kMaxTeam) && team_smem(b->fp32, I.grid.nx, I.grid.ny, g) > b->dyn_max) ++g;
            if (g > std::min(I.grid.ny, std::min(kMaxTeam, b->num_sms)))
                return bfail(b, PIT_EUNSUPPORTED, "problem %d: a level strip does not fit in shared memory", i);
            gmin[i] = g;
        }
        std::vector<double> cost(count, 1.0);
        if (b->opt.team_ctas > 0) {
            for (int i = 0; i < count; ++i)
                if (teams[i] == 1) team[i] = std::max(gmin[i], std::min({b->opt.team_ctas, inst[i].grid.ny, b->num_sms}));
            for (int i = 0; i < count; ++i)
                cost[i] = (double)inst[i].M * inst[i].grid.nx * inst[i].grid.ny / ((double)team[i] * teams[i]);
        } else {
            // autotuner: per distinct grid, time candidate team sizes on the first problem of
            // that grid truncated to a few levels; per-level time t(G) -> cost = t(G) * M.
            // A wavefront grid is timed at its team size; its cost counts the iterations in
            // flight as halving the time (only the schedule of the packed teams uses it).
            std::map<std::pair<int, int>, int> rep;
            std::map<std::pair<int, int>, std::vector<int>> cand;
            for (int i = 0; i < count; ++i) {
                const auto key = std::make_pair(inst[i].grid.nx, inst[i].grid.ny);
                rep.emplace(key, i);
                std::vector<int>& cs = cand[key];
                if (teams[i] > 1) {
                    if (std::find(cs.begin(), cs.end(), team[i]) == cs.end()) cs.push_back(team[i]);
                    continue;
                }
                const int gmax = std::min({inst[i].grid.ny, kMaxTeam, b->num_sms});
                for (double f : {1.0, 1.5, 2.0, 3.0, 4.0, 6.0}) {
                    const int g = std::min(gmax, std::max(gmin[i], (int)std::lround(gmin[i] * f)));
                    if (std::find(cs.begin(), cs.end(), g) == cs.end()) cs.push_back(g);
                }
            }
            std::map<std::pair<int, int>, std::vector<std::pair<int, double>>> table;
            // the calibration runs solve on a scratch iterate, so the problems' U_dev (which
            // may hold the caller's starting iterate) stay untouched
            size_t cal_n = 0;
            for (auto& kv : rep) cal_n = std::max(cal_n, (size_t)std::min(inst[kv.second].M, 8) * kv.first.first * kv.first.second);
            double* cal_U = nullptr;
            BCK(cudaMalloc(&cal_U, sizeof(double) * std::max<size_t>(cal_n, 1)));
            struct CalGuard {
                pit_batch* b;
                double* p;
                ~CalGuard() {
                    cudaFree(p);
                    b->calibrating = false;
                }
            } guard{b, cal_U};
            b->calibrating = true;
            for (auto& kv : rep) {
                pit_instance cal = inst[kv.second];
                cal.M = std::min(cal.M, 8);
                cal.U_dev = cal_U;
                for (int g : cand[kv.first]) {
                    std::vector<pit_instance> one{cal};
                    double best = 1e300;
                    BRET(build_launch(b, one, std::vector<int>{g}, std::vector<int>{1}, std::vector<double>{1.0},
                                      std::vector<int>{0}));
                    // results land in slot 0 of the real arrays; harmless before the real solve
                    for (int rep2 = 0; rep2 < 2; ++rep2) {
                        double ms = 0.0;
                        BRET(run_direct(b, &ms));
                        best = std::min(best, ms);
                    }
                    table[kv.first].push_back({g, best / cal.M});
                }
            }
            // per packed problem: the team size with the least SM time (t * G), then give
            // the longest problems more CTAs while they bound the makespan
            for (int i = 0; i < count; ++i) {
                const auto& tb = table[std::make_pair(inst[i].grid.nx, inst[i].grid.ny)];
                if (teams[i] > 1) {
                    for (auto& e : tb)
                        if (e.first == team[i]) cost[i] = e.second * inst[i].M / 2.0;
                    continue;
                }
                double bestv = 1e300;
                for (auto& e : tb) {
                    if (e.first >= gmin[i] && e.second * e.first < bestv) {
                        bestv = e.second * e.first;
                        team[i] = e.first;
                        cost[i] = e.second * inst[i].M;
                    }
                }
            }
            for (int round = 0; round < 64; ++round) {
                double total = 0.0, worst = 0.0;
                int wi = -1;
                for (int i = 0; i < count; ++i) {
                    total += cost[i] * team[i] * teams[i];
                    if (teams[i] == 1 && cost[i] > worst) {
                        worst = cost[i];
                        wi = i;
                    }
                }
                if (wi < 0 || worst <= total / b->num_sms) break;
                const auto& tb = table[std::make_pair(inst[wi].grid.nx, inst[wi].grid.ny)];
                bool grew = false;
                for (auto& e : tb) {
                    if (e.first > team[wi] && e.second * inst[wi].M < cost[wi]) {
                        team[wi] = e.first;
                        cost[wi] = e.second * inst[wi].M;
                        grew = true;
                        break;
                    }
                }
                if (!grew) break;
            }
        }
        b->team_of = team;
        std::vector<int> gid(count);
        std::iota(gid.begin(), gid.end(), 0);
        BRET(build_launch(b, b->in, team, teams, cost, gid));
        return PIT_OK;
    };
    pit_status st = setup();
    b->ms_tuning = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    if (st != PIT_OK) {
        fprintf(stderr, "pit_batch_create: %s\n", b->err);
        pit_batch_destroy(b);
        return st;
    }
    *out = b;
    return PIT_OK;
}

extern "C" pit_status pit_batch_solve(pit_batch* b, pit_batch_info* info) {
    if (!b) return PIT_EINVAL;
    if (!b->parts.empty()) {
        // one batch per closure, one after another; times and counts add up
        pit_batch_info pi{}, sum{};
        bool all_graph = true;
        pit_status worst = PIT_OK;
        for (pit_batch* q : b->parts) {
            const pit_status st = pit_batch_solve(q, &pi);
            if (st != PIT_OK && st != PIT_ENOCONV) {
                snprintf(b->err, sizeof(b->err), "%s", q->err);
                return st;
            }
            if (st == PIT_ENOCONV) worst = PIT_ENOCONV;
            sum.ms += pi.ms;
            sum.converged += pi.converged;
            all_graph = all_graph && pi.graph;
        }
        if (info) {
            info->count = b->count;
            info->ctas = b->ctas;
            info->teams = b->count;
            info->min_team = b->min_team;
            info->max_team = b->max_team;
            info->converged = sum.converged;
            info->graph = all_graph ? 1 : 0;
            info->ms = sum.ms;
            info->est_makespan_ms = b->est_ms;
            info->ms_tuning = b->ms_tuning;
            info->wave_jobs = b->wave_jobs;
        }
        if (worst != PIT_OK)
            return bfail(b, worst, "%d of %d problems did not reach tol_res", b->count - sum.converged, b->count);
        return PIT_OK;
    }
    double ms = 0.0;
    bool used_graph = false;
    // the caller's stream may hold the producers of the problems' data
    BCK(cudaEventRecord(b->ev_user, b->user_stream));
    BCK(cudaStreamWaitEvent(b->stream, b->ev_user, 0));
    if (b->graph_ok && !b->exec) {
        // capture the launch sequence once
        cudaStreamCaptureStatus cs;
        if (cudaStreamIsCapturing(b->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone &&
            cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const pit_status s = enqueue_launch(b, false);  // events in a graph cannot be timed
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
            if (s == PIT_OK && e == cudaSuccess && g &&
                cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess) {
                b->graph = g;
            } else {
                if (g) cudaGraphDestroy(g);
                b->exec = nullptr;
                b->graph_ok = false;
                cudaGetLastError();
            }
        } else {
            b->graph_ok = false;
            cudaGetLastError();
        }
    }
    if (b->exec) {
        BCK(cudaEventRecord(b->e0, b->stream));
        BCK(cudaGraphLaunch(b->exec, b->stream));
        BCK(cudaEventRecord(b->e1, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
        float f = 0.f;
        BCK(cudaEventElapsedTime(&f, b->e0, b->e1));
        ms = f;
        used_graph = true;
        if (b->h_ctl[1] == ST_ETIMEOUT) return bfail(b, PIT_ETIMEOUT, "batch kernel: a device wait ran out of budget");
        if (b->h_ctl[1] == ST_EDIVERGED) return bfail(b, PIT_EDIVERGED, "batch kernel: NaN/Inf in a problem");
    } else {
        BRET(run_direct(b, &ms));
    }
    int conv = 0;
    for (int i = 0; i < b->count; ++i) conv += (b->h_res[i] <= b->opt.tol_res);
    if (info) {
        info->count = b->count;
        info->ctas = b->ctas;
        info->teams = b->count;
        info->min_team = b->min_team;
        info->max_team = b->max_team;
        info->converged = conv;
        info->graph = used_graph ? 1 : 0;
        info->ms = ms;
        info->est_makespan_ms = b->est_ms;
        info->ms_tuning = b->ms_tuning;
        info->wave_jobs = b->wave_jobs;
    }
    if (conv < b->count) return bfail(b, PIT_ENOCONV, "%d of %d problems did not reach tol_res", b->count - conv, b->count);
    return PIT_OK;
}

extern "C" pit_status pit_batch_result(const pit_batch* b, int i, double* res_inf, int* newton_iters,
                                       int* windows_converged, int* team_ctas) {
    if (!b || i < 0 || i >= b->count) return PIT_EINVAL;
    if (!b->parts.empty())
        return pit_batch_result(b->parts[b->where[i].first], b->where[i].second, res_inf, newton_iters,
                                windows_converged, team_ctas);
    if (res_inf) *res_inf = b->h_res[i];
    if (newton_iters) *newton_iters = b->h_iters[i];
    if (windows_converged) *windows_converged = b->h_iters[b->count + i];
    if (team_ctas) *team_ctas = b->team_of.empty() ? 0 : b->team_of[i];
    return PIT_OK;
}

extern "C" pit_status pit_batch_placement(const pit_batch* b, int i, int* teams, int* team_ctas) {
    if (!b || i < 0 || i >= b->count) return PIT_EINVAL;
    if (!b->parts.empty()) return pit_batch_placement(b->parts[b->where[i].first], b->where[i].second, teams, team_ctas);
    if (teams) *teams = b->teams_of.empty() ? 0 : b->teams_of[i];
    if (team_ctas) *team_ctas = b->team_of.empty() ? 0 : b->team_of[i];
    return PIT_OK;
}

extern "C" const char* pit_batch_last_error(const pit_batch* b) { return b ? b->err : "null batch"; }

extern "C" void pit_batch_destroy(pit_batch* b) {
    if (!b) return;
    for (pit_batch* q : b->parts) pit_batch_destroy(q);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_inst);
    cudaFree(b->d_jobs);
    cudaFree(b->d_job_off);
    cudaFree(b->d_ws);
    cudaFree(b->d_geom);
    cudaFree(b->pool);
    cudaFree(b->d_res);
    cudaFree(b->d_iters);
    cudaFree(b->d_ctl);
    cudaFreeHost(b->h_res);
    cudaFreeHost(b->h_iters);
    cudaFreeHost(b->h_ctl);
    if (b->e0) cudaEventDestroy(b->e0);
    if (b->e1) cudaEventDestroy(b->e1);
    if (b->ev_user) cudaEventDestroy(b->ev_user);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}
