// pit_coarse.cu -- the paper's initial iterate (Sec. 4): solve the problem on a grid
// coarsened by c_f in each spatial direction and in time, then carry the coarse
// solution to the fine space-time grid with 1-D cubic splines.
//
// Coarse problem: nx_c = (nx + 1) / c_f - 1 interior nodes in x (likewise y) on the same
// domain, M_c = M / c_f levels of step M dt / M_c (same end time). Its data are sampled
// from the fine data: u^0 and the sources bilinearly between fine interior nodes, the
// Dirichlet data linearly along each edge, sources and Dirichlet data linearly in time
// between fine levels (injection wherever coarse and fine nodes meet). It is solved by
// pit_solve, whose converged result is the sequential BDF1 solution the paper computes.
//
// Interpolation: natural cubic splines (zero second derivative at both ends) on the
// uniform knots of each direction, in index units -- x through the west edge value, the
// coarse nodes and the east edge value; y through the south edge value, the x-splined
// rows and the north edge value; t through u^0 at t = 0 and the coarse levels. Each
// direction takes two kernels: one thread per line solves the spline's tridiagonal
// system (m_{k-1} + 4 m_k + m_{k+1} = 6 (y_{k+1} - 2 y_k + y_{k-1}), Thomas algorithm,
// pivots precomputed once: they depend on the line length only), then one thread per
// output value evaluates the spline, so every large array is read and written with
// consecutive threads on consecutive addresses.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "pit.h"
#include "pit_internal.h"

namespace {

constexpr int kT = 256;

// Reciprocal pivots of the Thomas algorithm for the natural-spline system with n knots:
// c_1 = 1/4, c_k = 1 / (4 - c_{k-1}), k = 2..n-2 (entries 0 and n-1 unused).
__global__ void spline_pivots_kernel(double* c, int n) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    c[0] = 0.0;
    double prev = 0.0;
    for (int k = 1; k <= n - 2; ++k) {
        prev = 1.0 / (4.0 - prev);
        c[k] = prev;
    }
    c[n - 1] = 0.0;
}

// Knot values of one line come from a functor y(k), k = 0..n-1; the second derivatives
// go to m(k) (the caller's addressing picks the stride).
template <typename Y, typename Mref>
__device__ void spline_solve_line(const Y& y, const Mref& m, const double* __restrict__ c, int n) {
    m(0) = 0.0;
    m(n - 1) = 0.0;
    if (n < 3) return;
    double dp = 0.0, ym = y(0), y0 = y(1);
    for (int k = 1; k <= n - 2; ++k) {
        const double yp = y(k + 1);
        dp = (6.0 * (yp - 2.0 * y0 + ym) - dp) * c[k];
        m(k) = dp;
        ym = y0;
        y0 = yp;
    }
    double next = 0.0;
    for (int k = n - 2; k >= 1; --k) {
        next = m(k) - c[k] * next;
        m(k) = next;
    }
}

__device__ __forceinline__ double spline_at(double yk, double yk1, double mk, double mk1, double t) {
    const double u = 1.0 - t;
    return u * yk + t * yk1 + ((u * u * u - u) * mk + (t * t * t - t) * mk1) * (1.0 / 6.0);
}

// Interval of a position s in [0, n - 1] on n knots, and the offset inside it.
__device__ __forceinline__ int spline_interval(double s, int n, double* t) {
    int k = (int)floor(s);
    k = max(0, min(k, n - 2));
    *t = s - k;
    return k;
}

// Linear interpolation weights of position s on the index range [0, n - 1].
struct Lin {
    int i0, i1;
    double w;
};
__device__ __forceinline__ Lin lin_at(double s, int n) {
    Lin r;
    r.i0 = max(0, min((int)floor(s), n - 1));
    r.i1 = min(r.i0 + 1, n - 1);
    r.w = fmin(1.0, fmax(0.0, s - r.i0));
    return r;
}
// Coarse interior node kc of nc, placed on the fine interior index range of n nodes.
__device__ __forceinline__ Lin space_pos(int kc, int nc, int n) {
    return lin_at((double)(kc + 1) * (n + 1) / (nc + 1) - 1.0, n);
}
// Coarse level l (1-based, time l T / M_c) on the fine levels (index n - 1 <-> time n dt).
__device__ __forceinline__ Lin time_pos(int l, int Mc, int M) {
    return lin_at((double)l * M / Mc - 1.0, M);
}

// ------------------------------------------------------------------ restriction

// out[l][jc][ic] = bilinear sample of f at coarse interior node (jc, ic), linear in time
// between fine levels when Mc > 0 (Mc == 0: f is a single level).
__global__ void restrict_interior_kernel(const double* __restrict__ f, double* __restrict__ out, int nx, int ny,
                                         int nxc, int nyc, int Mc, int M) {
    const size_t Nsc = (size_t)nxc * nyc, Ns = (size_t)nx * ny;
    const size_t total = Nsc * (size_t)(Mc > 0 ? Mc : 1);
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(k / Nsc);
        const size_t r = k - (size_t)l * Nsc;
        const int jc = (int)(r / nxc), ic = (int)(r - (size_t)jc * nxc);
        const Lin px = space_pos(ic, nxc, nx), py = space_pos(jc, nyc, ny);
        auto at = [&](const double* g) {
            const double a = (1.0 - px.w) * g[(size_t)py.i0 * nx + px.i0] + px.w * g[(size_t)py.i0 * nx + px.i1];
            const double b = (1.0 - px.w) * g[(size_t)py.i1 * nx + px.i0] + px.w * g[(size_t)py.i1 * nx + px.i1];
            return (1.0 - py.w) * a + py.w * b;
        };
        double v;
        if (Mc > 0) {
            const Lin pt = time_pos(l + 1, Mc, M);
            v = (1.0 - pt.w) * at(f + (size_t)pt.i0 * Ns) + pt.w * at(f + (size_t)pt.i1 * Ns);
        } else {
            v = at(f);
        }
        out[k] = v;
    }
}

// Dirichlet data bcc[l][e], e over the coarse edges (south nx_c, north nx_c, west ny_c,
// east ny_c), linear along the fine edge and in time.
__global__ void restrict_edges_kernel(const double* __restrict__ bf, double* __restrict__ bcc, int nx, int ny, int nxc,
                                      int nyc, int Mc, int M) {
    const int nbc = 2 * nxc + 2 * nyc, nbf = 2 * nx + 2 * ny;
    const size_t total = (size_t)Mc * nbc;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(k / nbc), e = (int)(k - (size_t)l * nbc);
        int base, pos, nc, nf;
        if (e < nxc) {
            base = 0; pos = e; nc = nxc; nf = nx;
        } else if (e < 2 * nxc) {
            base = nx; pos = e - nxc; nc = nxc; nf = nx;
        } else if (e < 2 * nxc + nyc) {
            base = 2 * nx; pos = e - 2 * nxc; nc = nyc; nf = ny;
        } else {
            base = 2 * nx + ny; pos = e - 2 * nxc - nyc; nc = nyc; nf = ny;
        }
        const Lin ps = space_pos(pos, nc, nf), pt = time_pos(l + 1, Mc, M);
        auto at = [&](int lf) {
            const double* b = bf + (size_t)lf * nbf + base;
            return (1.0 - ps.w) * b[ps.i0] + ps.w * b[ps.i1];
        };
        bcc[k] = (1.0 - pt.w) * at(pt.i0) + pt.w * at(pt.i1);
    }
}

// ------------------------------------------------------------------ x splines

struct XKnots {  // knots of coarse row (l, jc): west edge, coarse row, east edge
    const double* Uc;
    const double* bcc;  // coarse Dirichlet data (zeros when the problem has none)
    int nxc, nyc;
    __device__ double operator()(int l, int jc, int k) const {
        const size_t nbc = 2 * (size_t)nxc + 2 * (size_t)nyc;
        if (k == 0) return bcc[(size_t)l * nbc + 2 * nxc + jc];
        if (k == nxc + 1) return bcc[(size_t)l * nbc + 2 * nxc + nyc + jc];
        return Uc[((size_t)l * nyc + jc) * nxc + (k - 1)];
    }
};

// mx[(l, jc)][k], k = 0..nxc+1: one thread per coarse row.
__global__ void spline_x_solve_kernel(XKnots kn, const double* __restrict__ c, double* __restrict__ mx, int Mc) {
    const int n = kn.nxc + 2;
    const size_t lines = (size_t)Mc * kn.nyc;
    for (size_t line = (size_t)blockIdx.x * blockDim.x + threadIdx.x; line < lines;
         line += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(line / kn.nyc), jc = (int)(line - (size_t)l * kn.nyc);
        double* m = mx + line * n;
        spline_solve_line([&](int k) { return kn(l, jc, k); }, [&](int k) -> double& { return m[k]; }, c, n);
    }
}

// tx[l][jc][i]: the x spline of coarse row (l, jc) at fine column i.
__global__ void spline_x_eval_kernel(XKnots kn, const double* __restrict__ mx, double* __restrict__ tx, int Mc,
                                     int nx) {
    const int n = kn.nxc + 2;
    const size_t total = (size_t)Mc * kn.nyc * nx;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const size_t line = k / nx;
        const int i = (int)(k - line * nx);
        const int l = (int)(line / kn.nyc), jc = (int)(line - (size_t)l * kn.nyc);
        double t;
        const int a = spline_interval((double)(i + 1) * (kn.nxc + 1) / (nx + 1), n, &t);
        const double* m = mx + line * n;
        tx[k] = spline_at(kn(l, jc, a), kn(l, jc, a + 1), m[a], m[a + 1], t);
    }
}

// ------------------------------------------------------------------ y splines

struct YKnots {  // knots of fine column (l, i): south edge at t_l, x-splined rows, north edge at t_l
    const double* tx;
    const double* bf;  // fine Dirichlet data [M][2nx+2ny] (zeros when the problem has none)
    int nx, ny, nyc, Mc, M;
    __device__ double edge(int l, int idx) const {
        const Lin pt = time_pos(l + 1, Mc, M);
        const size_t nbf = 2 * (size_t)nx + 2 * (size_t)ny;
        return (1.0 - pt.w) * bf[(size_t)pt.i0 * nbf + idx] + pt.w * bf[(size_t)pt.i1 * nbf + idx];
    }
    __device__ double operator()(int l, int i, int k) const {
        if (k == 0) return edge(l, i);
        if (k == nyc + 1) return edge(l, nx + i);
        return tx[((size_t)l * nyc + (k - 1)) * nx + i];
    }
};

// my[l][k][i], k = 0..nyc+1: one thread per fine column (consecutive i on consecutive threads).
__global__ void spline_y_solve_kernel(YKnots kn, const double* __restrict__ c, double* __restrict__ my) {
    const int n = kn.nyc + 2;
    const size_t lines = (size_t)kn.Mc * kn.nx;
    for (size_t line = (size_t)blockIdx.x * blockDim.x + threadIdx.x; line < lines;
         line += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(line / kn.nx), i = (int)(line - (size_t)l * kn.nx);
        double* m = my + (size_t)l * n * kn.nx + i;
        spline_solve_line([&](int k) { return kn(l, i, k); },
                          [&](int k) -> double& { return m[(size_t)k * kn.nx]; }, c, n);
    }
}

// ty[l][j][i]: the y spline of column (l, i) at fine row j.
__global__ void spline_y_eval_kernel(YKnots kn, const double* __restrict__ my, double* __restrict__ ty) {
    const int n = kn.nyc + 2;
    const size_t Ns = (size_t)kn.nx * kn.ny, total = (size_t)kn.Mc * Ns;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(k / Ns);
        const size_t r = k - (size_t)l * Ns;
        const int j = (int)(r / kn.nx), i = (int)(r - (size_t)j * kn.nx);
        double t;
        const int a = spline_interval((double)(j + 1) * (kn.nyc + 1) / (kn.ny + 1), n, &t);
        const double* m = my + (size_t)l * n * kn.nx + i;
        ty[k] = spline_at(kn(l, i, a), kn(l, i, a + 1), m[(size_t)a * kn.nx], m[(size_t)(a + 1) * kn.nx], t);
    }
}

// ------------------------------------------------------------------ t splines

struct TKnots {  // knots of fine node p: u^0, then the Mc y-splined levels
    const double* u0;
    const double* ty;
    size_t Ns;
    __device__ double operator()(size_t p, int k) const { return k == 0 ? u0[p] : ty[(size_t)(k - 1) * Ns + p]; }
};

// mt[k][p], k = 0..Mc: one thread per fine node.
__global__ void spline_t_solve_kernel(TKnots kn, const double* __restrict__ c, double* __restrict__ mt, int Mc) {
    const int n = Mc + 1;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < kn.Ns; p += (size_t)gridDim.x * blockDim.x) {
        double* m = mt + p;
        spline_solve_line([&](int k) { return kn(p, k); }, [&](int k) -> double& { return m[(size_t)k * kn.Ns]; }, c,
                          n);
    }
}

// U[lv][p]: the t spline of node p at time (lv + 1) dt, i.e. knot position (lv + 1) Mc / M.
__global__ void spline_t_eval_kernel(TKnots kn, const double* __restrict__ mt, double* __restrict__ U, int Mc, int M) {
    const int nk = Mc + 1;
    const size_t total = (size_t)M * kn.Ns;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int lv = (int)(k / kn.Ns);
        const size_t p = k - (size_t)lv * kn.Ns;
        double t;
        const int a = spline_interval((double)(lv + 1) * Mc / M, nk, &t);
        U[k] = spline_at(kn(p, a), kn(p, a + 1), mt[(size_t)a * kn.Ns + p], mt[(size_t)(a + 1) * kn.Ns + p], t);
    }
}

unsigned grid_for(size_t work) {
    const size_t b = (work + kT - 1) / kT;
    return (unsigned)std::max<size_t>(1, std::min<size_t>(b, 152u * 64u));
}

}  // namespace

extern "C" pit_status pit_coarse_guess(pit_ctx* ctx, int cf, double* U_dev, pit_solve_info* coarse_info) {
    if (!ctx) return PIT_EINVAL;
    if (!U_dev) return pit_internal_fail(ctx, PIT_EINVAL, "pit_coarse_guess: U is NULL");
    PitProblemView v;
    pit_internal_view(ctx, &v);
    const int nx = v.grid.nx, ny = v.grid.ny, M = v.M;
    if (cf < 2) return pit_internal_fail(ctx, PIT_EINVAL, "pit_coarse_guess: coarsening factor %d < 2", cf);
    const int nxc = (nx + 1) / cf - 1, nyc = (ny + 1) / cf - 1, Mc = M / cf;
    if (nxc < 1 || nyc < 1 || Mc < 1)
        return pit_internal_fail(ctx, PIT_EINVAL, "pit_coarse_guess: grid %dx%dx%d too small to coarsen by %d", nx,
                                 ny, M, cf);
    cudaStream_t st = v.stream;
    const size_t Ns = (size_t)nx * ny, Nsc = (size_t)nxc * nyc;
    const int nbc = 2 * nxc + 2 * nyc;
    double *u0c = nullptr, *bcc = nullptr, *qc = nullptr, *Uc = nullptr, *tx = nullptr, *ty = nullptr;
    double *mx = nullptr, *my = nullptr, *mt = nullptr, *cx = nullptr, *cy = nullptr, *ctt = nullptr;
    double* bz = nullptr;  // zero Dirichlet data for the spline knots when the problem has none
    pit_ctx* cctx = nullptr;
    pit_status status = PIT_OK;
    char where[400] = "";
    auto ck = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && status == PIT_OK) {
            status = e == cudaErrorMemoryAllocation ? PIT_ENOMEM : PIT_ECUDA;
            snprintf(where, sizeof(where), "%s: %s", what, cudaGetErrorString(e));
        }
        return e == cudaSuccess;
    };
    auto alloc = [&](double** p, size_t n) {
        return ck(cudaMalloc(reinterpret_cast<void**>(p), sizeof(double) * std::max<size_t>(n, 1)), "cudaMalloc");
    };
    const bool ok = alloc(&u0c, Nsc) && alloc(&Uc, Nsc * Mc) && alloc(&tx, (size_t)Mc * nyc * nx) &&
                    alloc(&ty, (size_t)Mc * Ns) && alloc(&mx, (size_t)Mc * nyc * (nxc + 2)) &&
                    alloc(&my, (size_t)Mc * (nyc + 2) * nx) && alloc(&mt, (size_t)(Mc + 1) * Ns) &&
                    alloc(&cx, nxc + 2) && alloc(&cy, nyc + 2) && alloc(&ctt, Mc + 1) &&
                    alloc(&bcc, (size_t)Mc * nbc) && (v.bc || alloc(&bz, (size_t)M * (2 * nx + 2 * ny))) &&
                    (!v.q || alloc(&qc, Nsc * Mc));
    if (ok) {
        // coarse data
        restrict_interior_kernel<<<grid_for(Nsc), kT, 0, st>>>(v.u0, u0c, nx, ny, nxc, nyc, 0, M);
        if (v.bc) {
            restrict_edges_kernel<<<grid_for((size_t)Mc * nbc), kT, 0, st>>>(v.bc, bcc, nx, ny, nxc, nyc, Mc, M);
        } else {
            ck(cudaMemsetAsync(bcc, 0, sizeof(double) * Mc * nbc, st), "cudaMemsetAsync");
            ck(cudaMemsetAsync(bz, 0, sizeof(double) * M * (2 * nx + 2 * ny), st), "cudaMemsetAsync");
        }
        if (v.q) restrict_interior_kernel<<<grid_for(Nsc * Mc), kT, 0, st>>>(v.q, qc, nx, ny, nxc, nyc, Mc, M);
        ck(cudaGetLastError(), "restriction kernels");
        // coarse solve: the context's options, team sizes chosen afresh for the coarse grid
        pit_grid gc = v.grid;
        gc.nx = nxc;
        gc.ny = nyc;
        pit_options o = v.opt;
        o.team_ctas = 0;
        o.wave_teams = 0;
        if (status == PIT_OK) {
            status = pit_create(&gc, Mc, v.dt * M / Mc, &v.params, &o, st, &cctx);
            if (status != PIT_OK) snprintf(where, sizeof(where), "coarse context: %s", pit_status_string(status));
        }
        if (status == PIT_OK) status = pit_set_data(cctx, u0c, v.bc ? bcc : nullptr, qc);
        if (status == PIT_OK) status = pit_fill_plain_guess(cctx, Uc);
        if (status != PIT_OK && !where[0] && cctx) snprintf(where, sizeof(where), "%s", pit_last_error(cctx));
        pit_solve_info local;
        if (status == PIT_OK) {
            status = pit_solve(cctx, Uc, coarse_info ? coarse_info : &local);
            if (status != PIT_OK) snprintf(where, sizeof(where), "coarse solve: %s", pit_last_error(cctx));
        }
        if (status == PIT_OK) {
            spline_pivots_kernel<<<1, 1, 0, st>>>(cx, nxc + 2);
            spline_pivots_kernel<<<1, 1, 0, st>>>(cy, nyc + 2);
            spline_pivots_kernel<<<1, 1, 0, st>>>(ctt, Mc + 1);
            const XKnots kx{Uc, bcc, nxc, nyc};
            spline_x_solve_kernel<<<grid_for((size_t)Mc * nyc), kT, 0, st>>>(kx, cx, mx, Mc);
            spline_x_eval_kernel<<<grid_for((size_t)Mc * nyc * nx), kT, 0, st>>>(kx, mx, tx, Mc, nx);
            const YKnots ky{tx, v.bc ? v.bc : bz, nx, ny, nyc, Mc, M};
            spline_y_solve_kernel<<<grid_for((size_t)Mc * nx), kT, 0, st>>>(ky, cy, my);
            spline_y_eval_kernel<<<grid_for((size_t)Mc * Ns), kT, 0, st>>>(ky, my, ty);
            const TKnots kt{v.u0, ty, Ns};
            spline_t_solve_kernel<<<grid_for(Ns), kT, 0, st>>>(kt, ctt, mt, Mc);
            spline_t_eval_kernel<<<grid_for((size_t)M * Ns), kT, 0, st>>>(kt, mt, U_dev, Mc, M);
            ck(cudaGetLastError(), "spline kernels");
        }
    }
    ck(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    pit_destroy(cctx);
    for (double* p : {u0c, bcc, qc, Uc, tx, ty, mx, my, mt, cx, cy, ctt, bz}) cudaFree(p);
    if (status != PIT_OK) return pit_internal_fail(ctx, status, "pit_coarse_guess: %s", where[0] ? where : "failed");
    return PIT_OK;
}
