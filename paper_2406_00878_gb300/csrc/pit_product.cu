// pit_product.cu -- the paper's literal decoupled form (Theorem 1, eq. 8) and the
// recursion of Sec. 5 that builds it:
//
//   P^1 = A_1,  P^n = P^{n-1} A_n,   r~^1 = r^1,  r~^n = P^{n-1} r^n + r~^{n-1},
//   P^n du^n = r~^n  for every level n, independently.
//
// Storage: P^n in diagonal-offset form. Its row k couples node (i, j) to the nodes
// (i + dx, j + dy) with |dx| + |dy| <= n -- the 2n^2 + 2n + 1 diagonals of Remark 2 --
// and plane o of P^n holds, for every row k, the entry in offset o (zero where the
// neighbour lies outside the grid). Offsets are ordered by dy, then dx. P^0 = I is
// stored as one plane of ones so that every level follows the same product rule
//
//   P^n[o](k) = sum over the 5-point stencil s of  P^{n-1}[o - s](k) * A_n[s](k + o - s)
//
// which is the row-partitioned sparse product of eq. 10 with one thread per entry.
//
// Solve: every row of P^n and of r~^n is divided by the diagonal entry of P^n (the
// diagonal preconditioner of Sec. 7), the result is scattered into a dense band of
// half width n * nx and factored by banded LU without pivoting (the direct solver of
// Sec. 8), a team of CTAs per level, levels in parallel. The product's condition number grows
// like K^n with the per-level condition K (eq. 15): past the bound of eq. 15 the
// computed du^n loses its digits, which is why the library's main path applies the
// same inverse in nested form (eq. 7) instead.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "pit.h"
#include "pit_internal.h"

namespace {

constexpr int kT = 256;
constexpr int kLuThreads = 512;
constexpr int kMaxProductLevels = 180;  // 2n^2 + 2n + 1 offsets must fit a grid dimension

__host__ __device__ inline long long diag_count(int n) { return 2ll * n * n + 2ll * n + 1; }

// (dx, dy) of offset index oi in the ordering of { |dx| + |dy| <= n } by dy, then dx.
// Rows dy < 0 occupy the first n^2 indices ((n + dy)^2 of them lie before row dy); the
// ordering is centrally symmetric, so rows dy > 0 mirror rows dy < 0.
__device__ inline void offset_of(int oi, int n, int* dx, int* dy) {
    const int n2 = n * n;
    auto low = [&](int idx, int* ox, int* oy) {
        int r = (int)sqrt((double)idx);
        while (r * r > idx) --r;
        while ((r + 1) * (r + 1) <= idx) ++r;
        *oy = r - n;
        *ox = idx - r * r - r;
    };
    if (oi < n2) {
        low(oi, dx, dy);
    } else if (oi <= n2 + 2 * n) {
        *dy = 0;
        *dx = oi - n2 - n;
    } else {
        int mx, my;
        low((int)diag_count(n) - 1 - oi, &mx, &my);
        *dx = -mx;
        *dy = -my;
    }
}

// Index of offset (dx, dy), |dx| + |dy| <= n, in that ordering.
__device__ inline int offset_index(int dx, int dy, int n) {
    const int ady = dy < 0 ? -dy : dy;
    const int before = dy <= 0 ? (n + dy) * (n + dy) : n * n + dy * (2 * n + 2 - dy);
    return before + dx + (n - ady);
}

__global__ void identity_plane_kernel(double* P0, size_t Ns) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < Ns; k += (size_t)gridDim.x * blockDim.x)
        P0[k] = 1.0;
}

// P^n from P^{n-1} and the 5 coefficient planes of A_n (C, W, E, S, N at [5][M][Ns]).
// Grid: x over rows k, y over the offsets of P^n.
__global__ void product_kernel(const double* __restrict__ Pprev, double* __restrict__ Pn,
                               const double* __restrict__ coef, int n, int nx, int ny, int M) {
    const size_t Ns = (size_t)nx * ny, plane = (size_t)M * Ns;
    const double* A = coef + (size_t)(n - 1) * Ns;  // plane s of A_n at A + s * plane
    int dx, dy;
    offset_of(blockIdx.y, n, &dx, &dy);
    const int sx[5] = {0, -1, 1, 0, 0}, sy[5] = {0, 0, 0, -1, 1};
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < Ns; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / nx), i = (int)(k - (size_t)j * nx);
        double acc = 0.0;
        if (i + dx >= 0 && i + dx < nx && j + dy >= 0 && j + dy < ny) {
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const int px = dx - sx[s], py = dy - sy[s];  // offset of the P^{n-1} factor
                if ((px < 0 ? -px : px) + (py < 0 ? -py : py) > n - 1) continue;
                const int mi = i + px, mj = j + py;  // the intermediate node m = k + (o - s)
                if (mi < 0 || mi >= nx || mj < 0 || mj >= ny) continue;
                acc += Pprev[(size_t)offset_index(px, py, n - 1) * Ns + k] * A[s * plane + (size_t)mj * nx + mi];
            }
        }
        Pn[(size_t)blockIdx.y * Ns + k] = acc;
    }
}

// r~^n = P^{n-1} r^n + r~^{n-1} (r~^0 = 0), one thread per row.
__global__ void rhs_kernel(const double* __restrict__ Pprev, const double* __restrict__ r, const double* rt_prev,
                           double* __restrict__ rt, int n, int nx, int ny) {
    const size_t Ns = (size_t)nx * ny;
    const int m = n - 1;  // P^{n-1} has offsets |dx| + |dy| <= m
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < Ns; k += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / nx), i = (int)(k - (size_t)j * nx);
        double acc = 0.0;
        int oi = 0;
        for (int dy = -m; dy <= m; ++dy) {
            const int w = m - (dy < 0 ? -dy : dy);
            for (int dx = -w; dx <= w; ++dx, ++oi) {
                const int ti = i + dx, tj = j + dy;
                if (ti < 0 || ti >= nx || tj < 0 || tj >= ny) continue;
                acc += Pprev[(size_t)oi * Ns + k] * r[(size_t)tj * nx + ti];
            }
        }
        rt[k] = acc + (rt_prev ? rt_prev[k] : 0.0);
    }
}

// Scatter the diagonally scaled P^n and r~^n of levels [n0, n0 + count) into dense
// bands: band[l][k][d], d = col - k + b_n, width 2 b_n + 1, b_n = n nx. Grid: x over rows,
// y over levels in the batch.
__global__ void scatter_kernel(const double* __restrict__ Pall, const long long* __restrict__ pbase,
                               const double* __restrict__ rt_all, double* __restrict__ band,
                               const long long* __restrict__ bbase, double* __restrict__ rhs, int n0, int nx, int ny) {
    const size_t Ns = (size_t)nx * ny;
    const int n = n0 + blockIdx.y;
    const int b = n * nx;
    const size_t W = 2 * (size_t)b + 1;
    const double* P = Pall + pbase[n];
    double* B = band + bbase[blockIdx.y];
    const long long D = diag_count(n);
    const size_t center = (size_t)offset_index(0, 0, n);
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < Ns; k += (size_t)gridDim.x * blockDim.x) {
        const double inv = 1.0 / P[center * Ns + k];
        const int j = (int)(k / nx), i = (int)(k - (size_t)j * nx);
        for (long long oi = 0; oi < D; ++oi) {
            int dx, dy;
            offset_of((int)oi, n, &dx, &dy);
            if (i + dx < 0 || i + dx >= nx || j + dy < 0 || j + dy >= ny) continue;
            const long long d = (long long)dx + (long long)dy * nx + b;
            B[k * W + d] = P[(size_t)oi * Ns + k] * inv;
        }
        rhs[(size_t)blockIdx.y * Ns + k] = rt_all[(size_t)(n - 1) * Ns + k] * inv;
    }
}

// Banded LU without pivoting and the two triangular solves of every level of a batch:
// the rhs is overwritten by the solution, which goes to dU[n - 1].
// Team version: G CTAs per level share the elimination. Rows are dealt out cyclically
// (row k + 1 + t to CTA t mod G), every step ends with a team barrier (the pivot row and
// rhs entry of the next step are then final), and the back substitution runs the same
// way. Barriers are counters in global memory with bounded waits and an abort flag: a
// time-out raises *status and ends every CTA of the launch.
__device__ __forceinline__ unsigned long long lu_ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int lu_ld_acquire_s32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ bool lu_team_sync(unsigned long long* cnt, unsigned long long target, int* abort,
                                             int* status, long long budget, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(cnt, 1ull);
        int ok = 1;
        long long spins = 0;
        while (lu_ld_acquire(cnt) < target) {
            if (lu_ld_acquire_s32(abort)) {
                ok = 0;
                break;
            }
            if (++spins > budget) {
                atomicCAS(status, 0, 1);
                atomicExch(abort, 1);
                ok = 0;
                break;
            }
            if (spins > 1024) __nanosleep(32);
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

__global__ void __launch_bounds__(kLuThreads) band_lu_team_kernel(double* __restrict__ band,
                                                                  const long long* __restrict__ bbase,
                                                                  double* __restrict__ rhs, double* __restrict__ dU,
                                                                  double* __restrict__ min_pivot, int n0, int nx,
                                                                  int ny, int G, unsigned long long* cnt, int* abort,
                                                                  int* status, long long budget) {
    __shared__ int s_flag;
    const size_t Ns = (size_t)nx * ny;
    const int lvl = blockIdx.x / G, g = blockIdx.x - lvl * G;
    const int n = n0 + lvl;
    const int b = n * nx;
    const size_t W = 2 * (size_t)b + 1;
    double* B = band + bbase[lvl];
    double* r = rhs + (size_t)lvl * Ns;
    unsigned long long* c = cnt + lvl;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    unsigned long long sync = 0;
    double pmin = INFINITY;
    for (size_t k = 0; k < Ns; ++k) {
        const double* prow = B + k * W + b + 1;  // prow[jj] = B(k, k + 1 + jj)
        const double piv = B[k * W + b];
        const int span = (int)((size_t)b < Ns - 1 - k ? (size_t)b : Ns - 1 - k);
        if (threadIdx.x == 0) pmin = fmin(pmin, fabs(piv));
        const double inv = 1.0 / piv;
        const double rk = r[k];
        for (int t = g + warp * G; t < span; t += nwarps * G) {
            const size_t i = k + 1 + t;
            double* row = B + i * W + (b - 1 - t);  // row[0] = B(i, k), row[1 + jj] = B(i, k + 1 + jj)
            const double l = row[0] * inv;
            __syncwarp();
            for (int jj = lane; jj < span; jj += 32) row[jj + 1] = fma(-l, prow[jj], row[jj + 1]);
            if (lane == 0) {
                row[0] = l;
                r[i] = fma(-l, rk, r[i]);
            }
        }
        if (!lu_team_sync(c, (unsigned long long)G * ++sync, abort, status, budget, &s_flag)) return;
    }
    // back substitution U x = y
    for (size_t kk = Ns; kk-- > 0;) {
        const double xk = r[kk] / B[kk * W + b];
        const int span = (int)((size_t)b < kk ? (size_t)b : kk);
        for (int t = g + (int)threadIdx.x * G; t < span; t += (int)blockDim.x * G) {
            const size_t i = kk - 1 - t;
            r[i] = fma(-B[i * W + (b + 1 + t)], xk, r[i]);  // B(i, kk): column offset kk - i = 1 + t
        }
        if (g == 0 && threadIdx.x == 0) dU[(size_t)(n - 1) * Ns + kk] = xk;
        if (!lu_team_sync(c, (unsigned long long)G * ++sync, abort, status, budget, &s_flag)) return;
    }
    if (g == 0 && threadIdx.x == 0) min_pivot[n - 1] = pmin;
}

__global__ void axpy_kernel(double* __restrict__ U, const double* __restrict__ dU, size_t N, double* sumsq) {
    double s = 0.0;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (size_t)gridDim.x * blockDim.x) {
        U[k] += dU[k];
        s += dU[k] * dU[k];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sumsq, s);
}

unsigned grid_for(size_t work) {
    const size_t b = (work + kT - 1) / kT;
    return (unsigned)std::max<size_t>(1, std::min<size_t>(b, 152u * 32u));
}

// Workspace of one product-form solve.
struct ProductWs {
    int M = 0, nx = 0, ny = 0;
    size_t Ns = 0;
    std::vector<long long> pbase;   // start of P^n, n = 0..M, in doubles
    double* P = nullptr;            // all P^n
    double* rt = nullptr;           // r~^n, [M][Ns]
    double* coef = nullptr;         // [5][M][Ns]
    long long* d_pbase = nullptr;
    double* band = nullptr;         // dense bands of one batch of levels
    long long* d_bbase = nullptr;   // per batch slot
    double* rhs = nullptr;          // [batch][Ns]
    double* pmin = nullptr;         // [M]
    unsigned long long* lu_cnt = nullptr;  // [batch] team barrier counters of the LU launch
    int* lu_flags = nullptr;        // [2] abort, status
    int lu_G = 1;                   // CTAs per level in the LU launch
    int batch = 0;
    size_t band_doubles = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};

    ~ProductWs() {
        for (void* p : {(void*)P, (void*)rt, (void*)coef, (void*)d_pbase, (void*)band, (void*)d_bbase, (void*)rhs,
                        (void*)pmin, (void*)lu_cnt, (void*)lu_flags})
            cudaFree(p);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
};

size_t band_doubles_of(int n, int nx, size_t Ns) { return (2 * (size_t)n * nx + 1) * Ns; }

pit_status ws_init(pit_ctx* ctx, const PitProblemView& v, ProductWs& w) {
    w.M = v.M;
    w.nx = v.grid.nx;
    w.ny = v.grid.ny;
    w.Ns = (size_t)w.nx * w.ny;
    if (w.M > kMaxProductLevels)
        return pit_internal_fail(ctx, PIT_EUNSUPPORTED, "product form: M = %d levels above the supported %d", w.M,
                                 kMaxProductLevels);
    w.pbase.assign(w.M + 2, 0);
    for (int n = 0; n <= w.M; ++n) w.pbase[n + 1] = w.pbase[n] + diag_count(n) * (long long)w.Ns;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 0;
    const size_t p_bytes = sizeof(double) * (size_t)w.pbase[w.M + 1];
    const size_t budget = free_b / 2;
    if (p_bytes > budget)
        return pit_internal_fail(ctx, PIT_ENOMEM, "product form: the products P^1..P^M need %.2f GB, %.2f GB free",
                                 p_bytes * 1e-9, free_b * 1e-9);
    // levels per factorization batch: as many as fit a quarter of the remaining memory
    const size_t band_budget = std::max<size_t>((free_b - p_bytes) / 4, band_doubles_of(w.M, w.nx, w.Ns) * 8);
    size_t acc = 0;
    int batch = 0;
    for (int n = w.M; n >= 1; --n) {
        const size_t bd = band_doubles_of(n, w.nx, w.Ns);
        if (batch > 0 && (acc + bd) * sizeof(double) > band_budget) break;
        acc += bd;
        ++batch;
    }
    w.batch = std::max(1, batch);
    w.band_doubles = acc;
    auto al = [&](void** p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 8)); };
    cudaError_t e = al((void**)&w.P, p_bytes);
    if (e == cudaSuccess) e = al((void**)&w.rt, sizeof(double) * w.M * w.Ns);
    if (e == cudaSuccess) e = al((void**)&w.coef, sizeof(double) * 5 * w.M * w.Ns);
    if (e == cudaSuccess) e = al((void**)&w.d_pbase, sizeof(long long) * (w.M + 2));
    if (e == cudaSuccess) e = al((void**)&w.band, sizeof(double) * w.band_doubles);
    if (e == cudaSuccess) e = al((void**)&w.d_bbase, sizeof(long long) * w.batch);
    if (e == cudaSuccess) e = al((void**)&w.rhs, sizeof(double) * w.batch * w.Ns);
    if (e == cudaSuccess) e = al((void**)&w.pmin, sizeof(double) * w.M);
    if (e == cudaSuccess) e = al((void**)&w.lu_cnt, sizeof(unsigned long long) * w.batch);
    if (e == cudaSuccess) e = al((void**)&w.lu_flags, sizeof(int) * 2);
    {   // CTAs per level: the batch's levels side by side on (about) one CTA per SM each
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
            w.lu_G = std::max(1, std::min(32, (sms - 4) / std::max(1, w.batch)));
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w.d_pbase, w.pbase.data(), sizeof(long long) * (w.M + 2), cudaMemcpyHostToDevice,
                            v.stream);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&w.ev[i]);
    if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);  // pbase is a host temporary
    if (e != cudaSuccess)
        return pit_internal_fail(ctx, e == cudaErrorMemoryAllocation ? PIT_ENOMEM : PIT_ECUDA, "product form: %s",
                                 cudaGetErrorString(e));
    return PIT_OK;
}

// One product-form block solve on the context's stream: dU = (product form)^{-1} R for
// the Jacobians at U.
pit_status product_solve(pit_ctx* ctx, const PitProblemView& v, ProductWs& w, const double* U, const double* R,
                         double* dU, pit_product_info* info) {
    cudaStream_t st = v.stream;
    const size_t Ns = w.Ns;
    cudaError_t e = cudaEventRecord(w.ev[0], st);
    pit_status s = pit_assemble(ctx, U, w.coef);
    if (s != PIT_OK) return s;
    if (e == cudaSuccess) e = cudaEventRecord(w.ev[1], st);
    identity_plane_kernel<<<grid_for(Ns), kT, 0, st>>>(w.P, Ns);
    for (int n = 1; n <= w.M; ++n) {
        const double* Pprev = w.P + w.pbase[n - 1];
        dim3 g(std::min<unsigned>(grid_for(Ns), 64u), (unsigned)diag_count(n));
        product_kernel<<<g, kT, 0, st>>>(Pprev, w.P + w.pbase[n], w.coef, n, w.nx, w.ny, w.M);
        rhs_kernel<<<grid_for(Ns), kT, 0, st>>>(Pprev, R + (size_t)(n - 1) * Ns,
                                                 n > 1 ? w.rt + (size_t)(n - 2) * Ns : nullptr,
                                                 w.rt + (size_t)(n - 1) * Ns, n, w.nx, w.ny);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(w.ev[2], st);
    // factor and solve, levels in batches (highest levels have the widest bands)
    std::vector<long long> bbase(w.batch);
    for (int hi = w.M; hi >= 1 && e == cudaSuccess;) {
        int count = 0;
        size_t acc = 0;
        while (hi - count >= 1 && count < w.batch) {
            const size_t bd = band_doubles_of(hi - count, w.nx, Ns);
            if (acc + bd > w.band_doubles) break;
            acc += bd;
            ++count;
        }
        const int n0 = hi - count + 1;
        acc = 0;
        for (int l = 0; l < count; ++l) {
            bbase[l] = (long long)acc;
            acc += band_doubles_of(n0 + l, w.nx, Ns);
        }
        e = cudaMemcpyAsync(w.d_bbase, bbase.data(), sizeof(long long) * count, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.band, 0, sizeof(double) * acc, st);
        if (e != cudaSuccess) break;
        scatter_kernel<<<dim3(std::min<unsigned>(grid_for(Ns), 64u), count), kT, 0, st>>>(
            w.P, w.d_pbase, w.rt, w.band, w.d_bbase, w.rhs, n0, w.nx, w.ny);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.lu_cnt, 0, sizeof(unsigned long long) * count, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(w.lu_flags, 0, sizeof(int) * 2, st);
        if (e != cudaSuccess) break;
        {
            int G = w.lu_G;
            const long long budget = v.opt.wait_budget;
            int* abort_flag = w.lu_flags;
            int* status = w.lu_flags + 1;
            void* args[] = {&w.band, &w.d_bbase, &w.rhs, &dU, &w.pmin, (void*)&n0, &w.nx, &w.ny, &G, &w.lu_cnt,
                            &abort_flag, &status, (void*)&budget};
            e = cudaLaunchCooperativeKernel((const void*)band_lu_team_kernel, dim3(count * G), dim3(kLuThreads), args, 0,
                                            st);
        }
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // bbase is a host temporary reused by the next batch
        if (e == cudaSuccess) {
            int fl[2] = {0, 0};
            e = cudaMemcpy(fl, w.lu_flags, sizeof(fl), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && fl[1])
                return pit_internal_fail(ctx, PIT_ETIMEOUT, "product form: a team barrier of the LU ran out of budget");
        }
        hi = n0 - 1;
    }
    if (e == cudaSuccess) e = cudaEventRecord(w.ev[3], st);
    if (e == cudaSuccess) e = cudaEventSynchronize(w.ev[3]);
    if (e != cudaSuccess)
        return pit_internal_fail(ctx, e == cudaErrorMemoryAllocation ? PIT_ENOMEM : PIT_ECUDA, "product form: %s",
                                 cudaGetErrorString(e));
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->levels = w.M;
        info->diagonals = diag_count(w.M);
        info->half_band = (long long)w.M * w.nx;
        std::vector<double> pm(w.M);
        if (cudaMemcpy(pm.data(), w.pmin, sizeof(double) * w.M, cudaMemcpyDeviceToHost) == cudaSuccess) {
            double mn = INFINITY;
            for (double x : pm) mn = std::min(mn, x);
            info->min_pivot = mn;
        }
        cudaEventElapsedTime(&info->ms_assemble, w.ev[0], w.ev[1]);
        cudaEventElapsedTime(&info->ms_products, w.ev[1], w.ev[2]);
        cudaEventElapsedTime(&info->ms_factor, w.ev[2], w.ev[3]);
    }
    return PIT_OK;
}

}  // namespace

extern "C" pit_status pit_product_form_solve(pit_ctx* ctx, const double* U_dev, const double* R_dev, double* dU_dev,
                                             pit_product_info* info) {
    if (!ctx) return PIT_EINVAL;
    if (!U_dev || !R_dev || !dU_dev) return pit_internal_fail(ctx, PIT_EINVAL, "pit_product_form_solve: NULL pointer");
    PitProblemView v;
    pit_internal_view(ctx, &v);
    ProductWs w;
    pit_status s = ws_init(ctx, v, w);
    if (s != PIT_OK) return s;
    return product_solve(ctx, v, w, U_dev, R_dev, dU_dev, info);
}

extern "C" pit_status pit_solve_product(pit_ctx* ctx, double* U_dev, pit_solve_info* info) {
    if (!ctx) return PIT_EINVAL;
    if (!U_dev) return pit_internal_fail(ctx, PIT_EINVAL, "pit_solve_product: U is NULL");
    PitProblemView v;
    pit_internal_view(ctx, &v);
    pit_solve_info local;
    pit_solve_info* inf = info ? info : &local;
    std::memset(inf, 0, sizeof(*inf));
    inf->windows = 1;
    ProductWs w;
    pit_status s = ws_init(ctx, v, w);
    if (s != PIT_OK) return s;
    const size_t N = (size_t)v.M * w.Ns;
    double *R = nullptr, *dU = nullptr, *sumsq = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e = cudaMalloc(&R, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMalloc(&dU, sizeof(double) * N);
    if (e == cudaSuccess) e = cudaMalloc(&sumsq, sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e == cudaSuccess) e = cudaEventRecord(t0, v.stream);
    const int kmax = std::min(v.opt.newton_max, PIT_MAX_NEWTON);
    s = e == cudaSuccess ? PIT_OK
                         : pit_internal_fail(ctx, e == cudaErrorMemoryAllocation ? PIT_ENOMEM : PIT_ECUDA,
                                             "pit_solve_product: %s", cudaGetErrorString(e));
    for (int k = 0; s == PIT_OK; ++k) {
        double res = 0.0;
        s = pit_residual(ctx, U_dev, R, &res);
        if (s != PIT_OK) break;
        inf->res_inf[k] = res;
        inf->newton_iters = k;
        if (res <= v.opt.tol_res) {
            inf->converged = 1;
            break;
        }
        if (!std::isfinite(res) || res > 1e10) {
            s = pit_internal_fail(ctx, PIT_EDIVERGED, "pit_solve_product: residual %g at iteration %d", res, k);
            break;
        }
        if (k == kmax) {
            s = pit_internal_fail(ctx, PIT_ENOCONV, "pit_solve_product: residual %g after %d iterations", res, k);
            break;
        }
        pit_product_info pinfo;
        s = product_solve(ctx, v, w, U_dev, R, dU, &pinfo);
        if (s != PIT_OK) break;
        e = cudaMemsetAsync(sumsq, 0, sizeof(double), v.stream);
        axpy_kernel<<<grid_for(N), kT, 0, v.stream>>>(U_dev, dU, N, sumsq);
        double ss = 0.0;
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ss, sumsq, sizeof(double), cudaMemcpyDeviceToHost, v.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
        if (e != cudaSuccess) {
            s = pit_internal_fail(ctx, PIT_ECUDA, "pit_solve_product: %s", cudaGetErrorString(e));
            break;
        }
        pit_step_info& si = inf->steps[k];
        si.res_inf = res;
        si.upd_rms = std::sqrt(ss / (double)N);
        si.ms_assemble = pinfo.ms_assemble;
        si.ms_solve = pinfo.ms_products + pinfo.ms_factor;
    }
    inf->newton_iters_total = inf->newton_iters;
    if (t1 && cudaEventRecord(t1, v.stream) == cudaSuccess && cudaEventSynchronize(t1) == cudaSuccess) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess) inf->ms_total = ms;
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(R);
    cudaFree(dU);
    cudaFree(sumsq);
    return s;
}
