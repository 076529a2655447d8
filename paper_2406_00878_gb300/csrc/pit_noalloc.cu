// pit_noalloc.cu -- pit_block_solve_noalloc: the nested block inverse (row a3)
// for callers that cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc or anything that allocates
// on the device -- a host thread that works from a fixed, pre-sized memory
// budget, a real-time loop where an allocation's implicit device
// synchronisation is not allowed, or an embedding that owns every byte of GPU
// memory itself. Such a caller still owns and passes every input and output;
// the only memory this entry point touches besides them is the chain kernel's
// team workspace, which lives in the file-scope device array below.
//
// The array is a static __device__ object of this library: every GPU on which
// the library's kernels are loaded holds it (about 2.7 MB) until the process
// exits. In host code its name is only a host-side stand-in, not a device
// address, so the device address is fetched with cudaGetSymbolAddress once per
// device, with that device current, the first time the entry point runs there.
// Every call reads its status back into host memory and synchronises the stream,
// so no call may be made while the stream is being captured into a CUDA graph:
// such a call is refused with PIT_EUNSUPPORTED. Every call on a device shares
// the one array and it keeps the last call's contents: the counters that must
// start at zero are cleared at the start of each call, on the caller's stream.
// Calls that overlap on the GPU (other streams, other host threads) race on the
// array -- serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "pit.h"
#include "pit_kernels.cuh"

using namespace pit;

namespace {

constexpr int kNT = 256;
constexpr int kMinLocal = 256;
constexpr int kMaxDevices = 64;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Layout of the scratch array (bytes).
constexpr size_t kPubBytes = sizeof(double) * 2 * PIT_NOALLOC_MAX_TEAM * 2 * PIT_NOALLOC_MAX_NX;
constexpr size_t kRedBytes = sizeof(double) * 4 * PIT_NOALLOC_MAX_TEAM * 4;
constexpr size_t kSumBytes = sizeof(double) * PIT_NOALLOC_MAX_TEAM;
constexpr size_t kSyncBytes = sizeof(unsigned long long) * (PIT_NOALLOC_MAX_TEAM + 4);
constexpr size_t kTimerBytes = sizeof(unsigned long long) * 4;
constexpr size_t kIntBytes = sizeof(int) * (2 + 2 * (size_t)PIT_NOALLOC_MAX_LEVELS);
constexpr size_t kOffPub = 0;
constexpr size_t kOffRed = align256(kOffPub + kPubBytes);
constexpr size_t kOffSum = align256(kOffRed + kRedBytes);
constexpr size_t kOffSync = align256(kOffSum + kSumBytes);  // sync words, timers, ints: cleared per call
constexpr size_t kOffTimer = kOffSync + kSyncBytes;
constexpr size_t kOffInt = kOffTimer + kTimerBytes;
constexpr size_t kClearBytes = kSyncBytes + kTimerBytes + kIntBytes;
constexpr size_t kScratchBytes = align256(kOffInt + kIntBytes);

std::mutex g_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};  // device address of the array, per device
size_t g_smem_set[kMaxDevices] = {};             // dynamic shared memory opted in, per device

pit_status report(char* err, int err_len, pit_status s, const char* fmt, ...) {
    if (err && err_len > 0) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, (size_t)err_len, fmt, ap);
        va_end(ap);
    }
    return s;
}

}  // namespace

// The team workspace of pit_block_solve_noalloc (see the file comment).
static __device__ __align__(256) unsigned char g_pit_noalloc_scratch[kScratchBytes];

extern "C" pit_status pit_block_solve_noalloc(int nx, int ny, int M, const double* coef_dev, const double* R_dev,
                                              double* dU_dev, double eta, const pit_options* opt, void* stream,
                                              char* err, int err_len) {
    if (err && err_len > 0) err[0] = '\0';
    if (nx < 1 || ny < 1 || M < 1) return report(err, err_len, PIT_EINVAL, "nx, ny, M must be >= 1");
    if (!coef_dev || !R_dev || !dU_dev) return report(err, err_len, PIT_EINVAL, "NULL coef/R/dU pointer");
    if (!(eta > 0.0)) return report(err, err_len, PIT_EINVAL, "eta must be > 0");
    if (nx > PIT_NOALLOC_MAX_NX)
        return report(err, err_len, PIT_EUNSUPPORTED, "nx = %d exceeds the scratch limit PIT_NOALLOC_MAX_NX = %d", nx,
                      PIT_NOALLOC_MAX_NX);
    if (M > PIT_NOALLOC_MAX_LEVELS)
        return report(err, err_len, PIT_EUNSUPPORTED, "M = %d exceeds the scratch limit PIT_NOALLOC_MAX_LEVELS = %d",
                      M, PIT_NOALLOC_MAX_LEVELS);
    pit_options o;
    pit_default_options(&o);
    if (opt) o = *opt;
    if (o.lin_solver < 0 || o.lin_solver > 2 || !(o.lin_atol >= 0.0) || o.lin_max_iter < 1 || o.wait_budget < 1 ||
        o.team_ctas < 0 || !(o.sor_rho_max > 0.0))
        return report(err, err_len, PIT_EINVAL, "invalid options");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    {
        // the status read-back and the synchronisation below are illegal in a capture
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        const cudaError_t e = cudaStreamIsCapturing(st, &cap);
        if (e != cudaSuccess) return report(err, err_len, PIT_ECUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
        if (cap != cudaStreamCaptureStatusNone)
            return report(err, err_len, PIT_EUNSUPPORTED,
                          "the stream is being captured: this call reads its status back and synchronises");
    }

#define NA_CK(call)                                                                                            \
    do {                                                                                                       \
        cudaError_t e_ = (call);                                                                               \
        if (e_ != cudaSuccess)                                                                                 \
            return report(err, err_len, PIT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));                   \
    } while (0)

    int dev = 0, sms = 0, optin = 0, coop = 0;
    NA_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return report(err, err_len, PIT_EUNSUPPORTED, "device index %d", dev);
    NA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    NA_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    NA_CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return report(err, err_len, PIT_EUNSUPPORTED, "device lacks cooperative launch");

    // team of G CTAs per level, row strips (the same rule as pit_create)
    int rows_per;
    if (o.team_ctas > 0) {
        const int G = std::min(o.team_ctas, ny);
        rows_per = (ny + G - 1) / G;
    } else {
        rows_per = std::max((ny + sms - 1) / sms, (kMinLocal + nx - 1) / nx);
    }
    rows_per = std::min(rows_per, ny);
    size_t smem = 0;
    for (;;) {
        smem = sizeof(double) * chain_smem_doubles(rows_per * nx, nx);
        if (smem <= (size_t)optin) break;
        if (rows_per == 1) return report(err, err_len, PIT_EUNSUPPORTED, "one grid row (nx = %d) exceeds shared memory", nx);
        rows_per = (rows_per + 1) / 2;
    }
    const int G = (ny + rows_per - 1) / rows_per;
    if (G > PIT_NOALLOC_MAX_TEAM)
        return report(err, err_len, PIT_EUNSUPPORTED,
                      "team of %d CTAs exceeds the scratch limit PIT_NOALLOC_MAX_TEAM = %d (set team_ctas)", G,
                      PIT_NOALLOC_MAX_TEAM);

    unsigned char* scratch = nullptr;
    {
        // once per device, with that device current: the array's device address and
        // the kernel's shared-memory opt-in
        std::lock_guard<std::mutex> lock(g_mutex);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            NA_CK(cudaGetSymbolAddress(&p, g_pit_noalloc_scratch));
            cudaFuncAttributes fa;
            NA_CK(cudaFuncGetAttributes(&fa, chain_kernel<kNT, true>));
            const int dyn_max = optin - (int)fa.sharedSizeBytes;
            NA_CK(cudaFuncSetAttribute(reinterpret_cast<const void*>(chain_kernel<kNT, true>),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
            g_smem_set[dev] = (size_t)dyn_max;
            g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    if (smem > g_smem_set[dev]) return report(err, err_len, PIT_EUNSUPPORTED, "level strip exceeds shared memory");
    int per_sm = 0;
    NA_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chain_kernel<kNT, true>, kNT, smem));
    if ((long long)per_sm * sms < G)
        return report(err, err_len, PIT_EUNSUPPORTED, "team of %d CTAs cannot be co-resident", G);

    NA_CK(cudaMemsetAsync(scratch + kOffSync, 0, kClearBytes, st));
    ChainArgs a{};
    a.nx = nx;
    a.ny = ny;
    a.M = M;
    a.G = G;
    a.rows_base = ny / G;
    a.rows_rem = ny % G;
    a.R = R_dev;
    a.coef = coef_dev;
    a.rho_key = nullptr;
    a.U = nullptr;
    a.dU = dU_dev;
    a.update_U = 0;
    a.method = o.lin_solver;
    a.sor_rho_max = o.sor_rho_max;
    a.eta = eta;
    a.sor_tol_abs = 0.0;
    a.atol = o.lin_atol;
    a.max_iter = o.lin_max_iter;
    a.wait_budget = o.wait_budget;
    a.pub = reinterpret_cast<double*>(scratch + kOffPub);
    a.red_part = reinterpret_cast<double*>(scratch + kOffRed);
    a.cta_sumsq = reinterpret_cast<double*>(scratch + kOffSum);
    a.flags = reinterpret_cast<unsigned long long*>(scratch + kOffSync);
    a.red_cnt = a.flags + G;
    a.timers = reinterpret_cast<unsigned long long*>(scratch + kOffTimer);
    int* ints = reinterpret_cast<int*>(scratch + kOffInt);
    a.abort_flag = ints;
    a.status = ints + 1;
    a.level_iters = ints + 2;
    a.level_method = ints + 2 + M;
    void* args[] = {&a};
    NA_CK(cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(chain_kernel<kNT, true>), dim3(G), dim3(kNT),
                                      args, smem, st));
    int h[2] = {0, 0};
    NA_CK(cudaMemcpyAsync(h, ints, sizeof(h), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
    if (h[1] == ST_ETIMEOUT) return report(err, err_len, PIT_ETIMEOUT, "a device wait ran out of budget");
    if (h[1] == ST_EDIVERGED) return report(err, err_len, PIT_EDIVERGED, "NaN/Inf in a level solve");
    if (h[1] == ST_ENOCONV) return report(err, err_len, PIT_ENOCONV, "a level solve hit lin_max_iter");
    return PIT_OK;
}
