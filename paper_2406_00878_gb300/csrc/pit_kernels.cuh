// pit_kernels.cuh -- sm_103a kernels of the all-at-once BDF1 Newton iteration
// (arXiv 2406.00878, eq. 3-7).
//
//   residual_kernel   row (a1): r^n for all M levels at once (eq. 3-5) + ||R||_inf
//   assemble_kernel   row (a2): the 5 entries per row of A_n = I + tau dF/du for all
//                     levels at once (eq. 5-6), raw or Jacobi-scaled, + per-level
//                     Gershgorin bound of the scaled block
//   chain_kernel      row (a3): the exact block inverse of eq. 7 in nested form,
//                     du^n = A_n^{-1}(r^n + du^{n-1}), as one persistent cooperative
//                     launch that walks the level chain; a team of G CTAs shares each
//                     level (row strips), keeping the level's data in shared memory.
//
// Arithmetic is FP64 throughout. Closures: f = g = beta u^2/2 (CONV = Burgers),
// mu(u) = mu_a + mu_b u^2 (NLV when mu_b != 0), mid-point viscosity
// mu_{i+1/2} = mu((u_i + u_{i+1})/2).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pit_check.cuh"

namespace pit {

// ------------------------------------------------------------------ constants

struct OpConst {
    int nx, ny, M;
    long long Ns;
    double dt;
    double cx, cy;    // dt / (4 h_x), dt / (4 h_y): tau * (f_E - f_W)/(2h) with f = u^2/2
    double jx, jy;    // dt / (2 h_x), dt / (2 h_y): tau * f'(u)/(2h)
    double vx, vy;    // dt / h_x^2, dt / h_y^2
    double mu_a, mu_b;
    double vmx, vmy, kcen;  // mu_a dt / h_x^2, mu_a dt / h_y^2, 1 + 2 (vmx + vmy): constant-viscosity folds
};

// Status codes shared with the host (values of pit_status).
enum : int { ST_OK = 0, ST_ENOCONV = 4, ST_EDIVERGED = 5, ST_ETIMEOUT = 6 };

// A Newton residual above this (or not finite) counts as divergence.
constexpr double kDiverged = 1e10;
// A Newton iteration k >= 1 whose residual at a level exceeds this many times the first
// iteration's running residual there (or tol_res, if larger) counts as diverging too:
// from a poor start Newton on these problems was seen to grow the residual up to ~70x
// and still converge, while runs that grew it past ~1000x never did and burned capped
// level solves; the window is then retried shorter (same solution, block triangular).
constexpr double kGrowth = 1e3;

// --------------------------------------------------------- memory primitives

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_s32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// ---------------------------------------------- bulk copies (TMA) into shared memory
// One thread copies a contiguous global range into shared memory with cp.async.bulk and
// an mbarrier that counts the bytes; the CTA waits on the barrier's phase.

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Arrive (count one) and expect `bytes` of transactions in the current phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}
__device__ __forceinline__ bool mbar_test_parity(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Poll the phase with the given parity, at most `polls` times.
__device__ __forceinline__ bool mbar_wait_parity(unsigned long long* bar, unsigned parity, long long polls) {
    for (long long i = 0; i < polls; ++i)
        if (mbar_test_parity(bar, parity)) return true;
    return false;
}
// Generic-proxy accesses to shared memory before this point are ordered before later
// async-proxy (TMA) writes (after a barrier that covers every thread's accesses).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Global -> shared bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned),
// completing on bar's transaction count.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
constexpr long long kBulkWaitPolls = 1ll << 24;

// |x| as an order-preserving key: non-negative doubles compare like their bits,
// and NaN (sign cleared, 0x7ff8...) sorts above +Inf so it propagates through max.
// The sign bit is masked on the integer pipe (GB300's FP64 pipe is the scarce one).
__device__ __forceinline__ unsigned long long abs_key(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ double key_val(unsigned long long k) { return __longlong_as_double((long long)k); }

// x * y < 0 for nonzero finite x, y, decided on the sign and magnitude bits (integer pipe).
__device__ __forceinline__ bool opposite_nonzero(double x, double y) {
    const long long bx = __double_as_longlong(x), by = __double_as_longlong(y);
    const long long mag = 0x7fffffffffffffffll;
    return ((bx ^ by) < 0) && (bx & mag) != 0 && (by & mag) != 0;
}

__device__ __forceinline__ bool opposite_nonzero(float x, float y) {
    const int bx = __float_as_int(x), by = __float_as_int(y);
    const int mag = 0x7fffffff;
    return ((bx ^ by) < 0) && (bx & mag) != 0 && (by & mag) != 0;
}

// Maxima of four keys over the CTA, valid on thread 0 only (one barrier); red holds
// NT/32 * 4 keys.
template <int NT>
__device__ __forceinline__ void block_max4_to0(unsigned long long (&k)[4], unsigned long long* red) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, k[q], o);
            k[q] = w > k[q] ? w : k[q];
        }
    if ((threadIdx.x & 31) == 0)
        for (int q = 0; q < 4; ++q) red[(threadIdx.x >> 5) * 4 + q] = k[q];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < NT / 32; ++w)
            for (int q = 0; q < 4; ++q) k[q] = red[w * 4 + q] > k[q] ? red[w * 4 + q] : k[q];
}

template <int NT>
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* red) {
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < NT / 32 ? red[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w > v ? w : v;
        }
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    v = red[0];
    __syncthreads();
    return v;
}

// Sum of K doubles over the block in a fixed order (deterministic).
template <int NT, int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double* red) {
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) red[wid * K + k] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = lane < NT / 32 ? red[lane * K + k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) red[k] = s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = red[k];
    __syncthreads();
}

// ------------------------------------------------------------ stencil access

// Value of level vector u at (j, i), j in [-1, ny], i in [-1, nx]; off-interior
// nodes read the level's Dirichlet data (zero when bnd == nullptr).
template <typename PU, typename PB>
__device__ __forceinline__ double node_value(const PU& u, const PB& bnd, int nx, int ny, int j, int i) {
    if (i >= 0 && i < nx && j >= 0 && j < ny) return u[(long long)j * nx + i];
    if (!bnd) return 0.0;
    if (j < 0) return bnd[i];
    if (j >= ny) return bnd[nx + i];
    if (i < 0) return bnd[2 * nx + j];
    return bnd[2 * nx + ny + j];
}

// tau * F(u) at one node (eq. 3 without the time term), from the five stencil values.
template <bool CONV, bool NLV>
__device__ __forceinline__ double tau_F(const OpConst& c, double uC, double uW, double uE, double uS, double uN) {
    double t = 0.0;
    if (CONV) t = c.cx * ((uE - uW) * (uE + uW)) + c.cy * ((uN - uS) * (uN + uS));
    if (NLV) {
        const double ae = 0.5 * (uC + uE), aw = 0.5 * (uC + uW), an = 0.5 * (uC + uN), as = 0.5 * (uC + uS);
        const double me = fma(c.mu_b, ae * ae, c.mu_a), mw = fma(c.mu_b, aw * aw, c.mu_a);
        const double mn = fma(c.mu_b, an * an, c.mu_a), ms = fma(c.mu_b, as * as, c.mu_a);
        const double fx = me * (uE - uC) - mw * (uC - uW);
        const double fy = mn * (uN - uC) - ms * (uC - uS);
        t -= c.vx * fx + c.vy * fy;
    } else {
        t -= c.mu_a * (c.vx * ((uE - uC) - (uC - uW)) + c.vy * ((uN - uC) - (uC - uS)));
    }
    return t;
}

// The five entries of row C of A = I + tau dF/du (eq. 5-6).
template <bool CONV, bool NLV>
__device__ __forceinline__ void jac_row(const OpConst& c, double uC, double uW, double uE, double uS, double uN,
                                        double& aC, double& aW, double& aE, double& aS, double& aN) {
    if (NLV) {
        const double ae = 0.5 * (uC + uE), aw = 0.5 * (uC + uW), an = 0.5 * (uC + uN), as = 0.5 * (uC + uS);
        const double me = fma(c.mu_b, ae * ae, c.mu_a), mw = fma(c.mu_b, aw * aw, c.mu_a);
        const double mn = fma(c.mu_b, an * an, c.mu_a), ms = fma(c.mu_b, as * as, c.mu_a);
        // d mu_{e} / d u = mu'(a_e)/2 = mu_b a_e
        const double de = c.mu_b * ae, dw = c.mu_b * aw, dn = c.mu_b * an, ds = c.mu_b * as;
        aE = -c.vx * (me + de * (uE - uC));
        aW = -c.vx * (mw - dw * (uC - uW));
        aN = -c.vy * (mn + dn * (uN - uC));
        aS = -c.vy * (ms - ds * (uC - uS));
        aC = 1.0 + c.vx * (me + mw - de * (uE - uC) + dw * (uC - uW)) + c.vy * (mn + ms - dn * (uN - uC) + ds * (uC - uS));
    } else {
        aE = -c.vx * c.mu_a;
        aW = aE;
        aN = -c.vy * c.mu_a;
        aS = aN;
        aC = 1.0 + 2.0 * c.mu_a * (c.vx + c.vy);
    }
    if (CONV) {
        aE += c.jx * uE;
        aW -= c.jx * uW;
        aN += c.jy * uN;
        aS -= c.jy * uS;
    }
}

// --------------------------------------------------------------- (a1) residual

// One thread per node, all levels at once: grid (ceil(Ns/NT), M). Writes R and
// folds |r| into *rinf_key (order-preserving max key, see abs_key).
template <bool CONV, bool NLV, int NT>
__global__ void __launch_bounds__(NT) residual_kernel(OpConst c, const double* __restrict__ u0,
                                                      const double* __restrict__ U, const double* __restrict__ bc,
                                                      const double* __restrict__ q, double* __restrict__ R,
                                                      unsigned long long* __restrict__ rinf_key) {
    __shared__ unsigned long long red[NT / 32];
    const int n = blockIdx.y;  // level index 0..M-1 <-> u^{n+1}
    const long long k = (long long)blockIdx.x * NT + threadIdx.x;
    unsigned long long key = 0;
    const long long nb = 2 * c.nx + 2 * c.ny, tot = (long long)c.M * c.Ns;
    const auto Uc = chk(U, tot, kChkU);
    const auto bcc = chk(bc, c.M * nb, kChkBc);
    const auto qc = chk(q, tot, kChkQ);
    const auto Rc = chk(R, tot, kChkR);
    if (k < c.Ns) {
        const int j = (int)(k / c.nx), i = (int)(k - (long long)j * c.nx);
        const auto u = Uc + (long long)n * c.Ns;
        const auto up = (n == 0) ? chk(u0, c.Ns, kChkU0) : Uc + (long long)(n - 1) * c.Ns;
        const auto bnd = bc ? bcc + (long long)n * nb : bcc;
        const double uC = u[k];
        const double uW = node_value(u, bnd, c.nx, c.ny, j, i - 1);
        const double uE = node_value(u, bnd, c.nx, c.ny, j, i + 1);
        const double uS = node_value(u, bnd, c.nx, c.ny, j - 1, i);
        const double uN = node_value(u, bnd, c.nx, c.ny, j + 1, i);
        double r;
        if (CONV && !NLV) {
            // constant-viscosity Burgers with the constants folded (nine FP64 operations):
            // r = u^{n-1} - kcen uC - uE (cx uE - vmx) + uW (cx uW + vmx) - (the same in y)
            r = fma(-c.kcen, uC, up[k]);
            r = fma(-uE, fma(c.cx, uE, -c.vmx), r);
            r = fma(uW, fma(c.cx, uW, c.vmx), r);
            r = fma(-uN, fma(c.cy, uN, -c.vmy), r);
            r = fma(uS, fma(c.cy, uS, c.vmy), r);
        } else {
            r = (up[k] - uC) - tau_F<CONV, NLV>(c, uC, uW, uE, uS, uN);
        }
        if (q) r = fma(c.dt, qc[(long long)n * c.Ns + k], r);
        Rc[(long long)n * c.Ns + k] = r;
        key = abs_key(r);
    }
    key = block_max_u64<NT>(key, red);
    if (threadIdx.x == 0 && key) atomicMax(rinf_key, key);
}

// ------------------------------------------------------------ (a2) assembly

// One thread per node, all levels at once. SCALED = false writes the raw entries
// coef[5][M][Ns] = C, W, E, S, N of A_n. SCALED = true writes the Jacobi-scaled
// planes used by the level solver: 1/C, W/C, E/C, S/C, N/C, and folds the row sum
// |W|+|E|+|S|+|N| over |C| into rho_key[n] (Gershgorin bound of I - D^{-1}A_n) and
// sets rho_key[M + n] when a row has opposite-signed couplings in x or y.
template <bool CONV, bool NLV, bool SCALED, int NT>
__global__ void __launch_bounds__(NT) assemble_kernel(OpConst c, const double* __restrict__ U,
                                                      const double* __restrict__ bc, double* __restrict__ coef,
                                                      unsigned long long* __restrict__ rho_key) {
    __shared__ unsigned long long red[NT / 32];
    const int n = blockIdx.y;
    const long long k = (long long)blockIdx.x * NT + threadIdx.x;
    const long long plane = (long long)c.M * c.Ns;
    unsigned long long key = 0;
    const long long nb = 2 * c.nx + 2 * c.ny;
    const auto Uc = chk(U, plane, kChkU);
    const auto bcc = chk(bc, c.M * nb, kChkBc);
    const auto coefc = chk(coef, 5 * plane, kChkCoef);
    if (k < c.Ns) {
        const int j = (int)(k / c.nx), i = (int)(k - (long long)j * c.nx);
        const auto u = Uc + (long long)n * c.Ns;
        const auto bnd = bc ? bcc + (long long)n * nb : bcc;
        const double uC = u[k];
        const double uW = node_value(u, bnd, c.nx, c.ny, j, i - 1);
        const double uE = node_value(u, bnd, c.nx, c.ny, j, i + 1);
        const double uS = node_value(u, bnd, c.nx, c.ny, j - 1, i);
        const double uN = node_value(u, bnd, c.nx, c.ny, j + 1, i);
        double aC, aW, aE, aS, aN;
        jac_row<CONV, NLV>(c, uC, uW, uE, uS, uN, aC, aW, aE, aS, aN);
        if (i == 0) aW = 0.0;
        if (i == c.nx - 1) aE = 0.0;
        if (j == 0) aS = 0.0;
        if (j == c.ny - 1) aN = 0.0;
        const auto o = coefc + ((long long)n * c.Ns + k);
        if (SCALED) {
            const double d = 1.0 / aC;
            aW *= d;
            aE *= d;
            aS *= d;
            aN *= d;
            o[0] = d;
            key = abs_key(fabs(aW) + fabs(aE) + fabs(aS) + fabs(aN));
            if (aW * aE < 0.0 || aS * aN < 0.0) atomicMax(rho_key + c.M + n, 1ull);
        } else {
            o[0] = aC;
        }
        o[plane] = aW;
        o[2 * plane] = aE;
        o[3 * plane] = aS;
        o[4 * plane] = aN;
    }
    if (SCALED) {
        key = block_max_u64<NT>(key, red);
        if (threadIdx.x == 0 && key) atomicMax(rho_key + n, key);
    }
}

// -------------------------------------------- copy u^0 into every level (guess)

static __global__ void plain_guess_kernel(const double* __restrict__ u0, double* __restrict__ U, long long Ns, int M) {
    const long long total = Ns * (long long)M;
    const auto Uc = chk(U, total, kChkU);
    const auto u0c = chk(u0, Ns, kChkU0);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
        Uc[t] = u0c[t % Ns];
}

// ------------------------------------------------------ (a3) the level chain

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Control words shared by every CTA of a launch that uses the team protocol.
struct TeamCtl {
    int* abort_flag;        // raised by the first CTA that gives up; every wait watches it
    int* status;            // first error code (ST_*)
    long long wait_budget;  // spin iterations before a wait gives up
    int max_iter;           // cap on sweeps / iterations per level solve
};

// Per-CTA state of the team protocol: a team of G CTAs shares one level as row
// strips; CTA b owns rows [r0, r0 + nrows). The team's workspace:
//   pub      [2][G][2][nx] published first/last rows (double-buffered by sequence)
//   flags    [G]           publication counters
//   red_part [4][G][4]     reduction partials (4 slots in rotation)
//   red_cnt  [4]           arrival counters of the slots
struct Team {
    int b, G, nx;
    int rows_base;                // the team's strips: rows_base rows, one more for the first ones
    int r0, nrows, nloc;
    long long Ns;
    double* pub;
    unsigned long long* flags;
    double* red_part;
    unsigned long long* red_cnt;
    unsigned long long pub_seq;   // publications so far by this CTA
    unsigned long long red_seq;   // counter-based reductions started so far
    unsigned long long tag_seq;   // sequence-tagged reductions started so far
    unsigned long long t_halo;    // ns spent waiting for neighbours (thread 0)
    unsigned long long t_red;     // ns spent waiting for team reductions (thread 0)
};

__device__ __forceinline__ void team_init(Team& t, int b, int G, int nx, int ny, int rows_base, int rows_rem,
                                          double* pub, unsigned long long* flags, double* red_part,
                                          unsigned long long* red_cnt) {
    t.b = b;
    t.G = G;
    t.nx = nx;
    t.rows_base = rows_base;
    t.nrows = rows_base + (b < rows_rem ? 1 : 0);
    t.r0 = b * rows_base + (b < rows_rem ? b : rows_rem);
    t.nloc = t.nrows * nx;
    t.Ns = (long long)nx * ny;
    t.pub = pub;
    t.flags = flags;
    t.red_part = red_part;
    t.red_cnt = red_cnt;
    t.pub_seq = 0;
    t.red_seq = 0;
    t.tag_seq = 0;
    t.t_halo = 0;
    t.t_red = 0;
}

// Give up on a wait: record the status once and raise the abort flag.
__device__ __forceinline__ void team_fail(const TeamCtl& c, int code) {
    atomicCAS(c.status, 0, code);
    atomicExch(c.abort_flag, 1);
}

// Spin (one thread) until *p >= target, the abort flag is raised, or the budget is spent.
__device__ __forceinline__ bool wait_geq(const TeamCtl& c, const unsigned long long* p, unsigned long long target) {
    long long spins = 0;
    while (ld_acquire_u64(p) < target) {
        if (ld_acquire_s32(c.abort_flag)) return false;
        if (++spins > c.wait_budget) {
            team_fail(c, ST_ETIMEOUT);
            return false;
        }
        if (spins > 4096) __nanosleep(64);
    }
    return true;
}

// Thread 0: make this CTA's publication at `seq` visible (release), then wait until
// both neighbours have published `seq` (acquire). Writes the outcome to *s_ok.
__device__ __forceinline__ void publish_and_wait(const TeamCtl& c, Team& t, unsigned long long seq, int* s_ok) {
    __threadfence();
    st_release_u64(t.flags + t.b, seq);
    const unsigned long long t0 = global_ns();
    bool ok = true;
    if (t.b > 0) ok = wait_geq(c, t.flags + t.b - 1, seq);
    if (ok && t.b + 1 < t.G) ok = wait_geq(c, t.flags + t.b + 1, seq);
    __threadfence();
    *s_ok = ok ? 1 : 0;
    t.t_halo += global_ns() - t0;
}

// Publish the first and last local rows of v for the neighbours; then fetch the
// neighbours' rows published at the same step into haloS (row r0-1) and haloN
// (row r0+nrows). Rows outside the domain are zero (the correction vanishes on
// the Dirichlet boundary). Returns false when the launch aborted.
template <int NT, typename T>
__device__ bool exchange_halo(const TeamCtl& c, Team& t, const sptr<const T> v, const sptr<T> haloS, const sptr<T> haloN,
                              int* s_ok) {
    const int nx = t.nx;
    const unsigned long long seq = ++t.pub_seq;
    T* const pubT = reinterpret_cast<T*>(t.pub);
    T* mine = pubT + ((size_t)(seq & 1) * t.G + t.b) * 2 * nx;
    for (int i = threadIdx.x; i < nx; i += NT) {
        __stcg(mine + i, v[i]);
        __stcg(mine + nx + i, v[(t.nrows - 1) * nx + i]);
    }
    __syncthreads();
    if (threadIdx.x == 0) publish_and_wait(c, t, seq, s_ok);
    __syncthreads();
    if (!*s_ok) return false;
    const T* par = pubT + (size_t)(seq & 1) * t.G * 2 * nx;
    if (t.b > 0) {  // neighbour below: its last row
        const T* lo = par + (size_t)(t.b - 1) * 2 * nx + nx;
        for (int i = threadIdx.x; i < nx; i += NT) haloS[i] = __ldcg(lo + i);
    } else {
        for (int i = threadIdx.x; i < nx; i += NT) haloS[i] = T(0);
    }
    if (t.b + 1 < t.G) {  // neighbour above: its first row
        const T* hi = par + (size_t)(t.b + 1) * 2 * nx;
        for (int i = threadIdx.x; i < nx; i += NT) haloN[i] = __ldcg(hi + i);
    } else {
        for (int i = threadIdx.x; i < nx; i += NT) haloN[i] = T(0);
    }
    __syncthreads();
    return true;
}

// Rows of the two neighbours that let red-black SOR run on one exchange per sweep: the
// scaled couplings and rhs of rows r0-1 and r0+nrows (cS, cN: cw ce cs cn bs, exchanged
// once per level) and the iterate two rows away (xS2, xN2). With these a CTA updates the
// red points of its halo rows itself -- the same arithmetic on the same values as their
// owner -- so the black half-sweep needs no second exchange.
//
// These exchanges, and the team reductions of the same launches, use sequence-tagged
// words: every published 32-bit piece travels in a 64-bit word whose high half is the
// sequence number of the publication (single-copy atomic), so a reader polls the data
// itself -- no release/acquire flag and no fence on the critical path. tpub: the team's
// publication words, [2][G][kDeepSlotRows][nx][words per value]; tred: the team's
// reduction words, [4][G][kTagRedWords]; both zero before the launch (tag 0 is never used).
constexpr int kDeepSlotRows = 10;
constexpr int kTagRedWords = 8;
template <typename T>
struct Deep {
    unsigned long long* tpub;
    unsigned long long* tred;
    sptr<T> cS[5];
    sptr<T> cN[5];
    sptr<T> xS2;
    sptr<T> xN2;
};

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
// Two adjacent tagged words (16-byte aligned) in one access: each 8-byte word is still
// single-copy atomic, and each carries its own tag.
__device__ __forceinline__ void st_relaxed_v2(unsigned long long* p, unsigned long long a, unsigned long long b) {
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void ld_relaxed_v2(const unsigned long long* p, unsigned long long& a, unsigned long long& b) {
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ unsigned long long tagged(unsigned tag, unsigned payload) {
    return ((unsigned long long)tag << 32) | payload;
}

// 32-bit pieces of a value (one for float, two for double).
template <typename T>
struct Pieces;
template <>
struct Pieces<float> {
    static constexpr int n = 1;
    __device__ static unsigned get(float v, int) { return __float_as_uint(v); }
    __device__ static float make(const unsigned (&w)[2]) { return __uint_as_float(w[0]); }
};
template <>
struct Pieces<double> {
    static constexpr int n = 2;
    __device__ static unsigned get(double v, int k) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(v);
        return k ? (unsigned)(b >> 32) : (unsigned)b;
    }
    __device__ static double make(const unsigned (&w)[2]) {
        return __longlong_as_double((long long)(((unsigned long long)w[1] << 32) | w[0]));
    }
};

// Complete a batch of N tagged words: the first loads are issued together (one L2 round
// trip for the batch); words whose tag is not yet `tag` are polled again. false after the
// wait budget or when the launch aborts (checked every 256 rounds).
template <int N>
__device__ __forceinline__ bool wait_tagged(const TeamCtl& c, const unsigned long long* const (&src)[N],
                                            unsigned long long (&w)[N], unsigned tag) {
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] = src[k] ? ld_relaxed_u64(src[k]) : tagged(tag, 0u);
    for (long long spins = 0;; ++spins) {
        bool all = true;
#pragma unroll
        for (int k = 0; k < N; ++k)
            if ((unsigned)(w[k] >> 32) != tag) {
                all = false;
                w[k] = ld_relaxed_u64(src[k]);
            }
        if (all) return true;
        if ((spins & 255) == 255 && ld_acquire_s32(c.abort_flag)) return false;
        if (spins > c.wait_budget) return false;
    }
}

// wait_tagged for N pairs of adjacent words (16-byte aligned), loaded two at a time.
template <int N>
__device__ __forceinline__ bool wait_tagged_pairs(const TeamCtl& c, const unsigned long long* const (&src)[N],
                                                  unsigned long long (&w)[2 * N], unsigned tag) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
        if (src[k]) ld_relaxed_v2(src[k], w[2 * k], w[2 * k + 1]);
        else w[2 * k] = w[2 * k + 1] = tagged(tag, 0u);
    }
    for (long long spins = 0;; ++spins) {
        bool all = true;
#pragma unroll
        for (int k = 0; k < N; ++k)
            if ((unsigned)(w[2 * k] >> 32) != tag || (unsigned)(w[2 * k + 1] >> 32) != tag) {
                all = false;
                ld_relaxed_v2(src[k], w[2 * k], w[2 * k + 1]);
            }
        if (all) return true;
        if ((spins & 255) == 255 && ld_acquire_s32(c.abort_flag)) return false;
        if (spins > c.wait_budget) return false;
    }
}

// Publish H rows for each neighbour -- lo[h] (this CTA's first rows) for the CTA below and
// hi[h] (its last rows) for the CTA above -- as sequence-tagged words. Returns the
// publication's sequence number, which fetch_rows_tagged takes. No barrier: the caller
// makes the rows final before (a __syncthreads) and may compute on until it fetches.
template <int NT, typename T, int H>
__device__ __forceinline__ unsigned long long publish_rows_tagged(Team& t, unsigned long long* tpub,
                                                                  const sptr<const T> (&lo)[H],
                                                                  const sptr<const T> (&hi)[H]) {
    static_assert(2 * H <= kDeepSlotRows, "slot too small");
    constexpr int P = Pieces<T>::n;
    const int nx = t.nx;
    const unsigned long long seq = ++t.pub_seq;
    const unsigned tag = (unsigned)seq;
    const size_t row_w = (size_t)nx * P, slot_w = (size_t)kDeepSlotRows * row_w;
    unsigned long long* mine = tpub + ((size_t)(seq & 1) * t.G + t.b) * slot_w;
#pragma unroll
    for (int h = 0; h < H; ++h)
        for (int i = threadIdx.x; i < nx; i += NT) {
            if constexpr (P == 2) {
                // both words of a double in one 16-byte store
                st_relaxed_v2(mine + h * row_w + (size_t)i * 2, tagged(tag, Pieces<T>::get(lo[h][i], 0)),
                              tagged(tag, Pieces<T>::get(lo[h][i], 1)));
                st_relaxed_v2(mine + (H + h) * row_w + (size_t)i * 2, tagged(tag, Pieces<T>::get(hi[h][i], 0)),
                              tagged(tag, Pieces<T>::get(hi[h][i], 1)));
            } else {
                st_relaxed_u64(mine + h * row_w + (size_t)i, tagged(tag, Pieces<T>::get(lo[h][i], 0)));
                st_relaxed_u64(mine + (H + h) * row_w + (size_t)i, tagged(tag, Pieces<T>::get(hi[h][i], 0)));
            }
        }
    return seq;
}

// Fetch the CTA below's hi rows of publication `seq` into fromS and the CTA above's lo rows
// into fromN (zeros off the domain); ends with a barrier. Returns false when a wait timed
// out (the launch is then aborted) or the launch aborted.
template <int NT, typename T, int H>
__device__ bool fetch_rows_tagged(const TeamCtl& c, const Team& t, const unsigned long long* tpub,
                                  unsigned long long seq, const sptr<T> (&fromS)[H], const sptr<T> (&fromN)[H]) {
    constexpr int P = Pieces<T>::n;
    const int nx = t.nx;
    const unsigned tag = (unsigned)seq;
    const size_t row_w = (size_t)nx * P, slot_w = (size_t)kDeepSlotRows * row_w;
    const unsigned long long* par = tpub + (size_t)(seq & 1) * t.G * slot_w;
    const unsigned long long* srcS = t.b > 0 ? par + (size_t)(t.b - 1) * slot_w + H * row_w : nullptr;
    const unsigned long long* srcN = t.b + 1 < t.G ? par + (size_t)(t.b + 1) * slot_w : nullptr;
    bool ok = true;
    for (int i0 = 0; i0 < nx && ok; i0 += NT) {
        const int i = i0 + threadIdx.x;
        if (i >= nx) continue;
        unsigned long long w[2 * H * P];
        if constexpr (P == 2) {
            const unsigned long long* src[2 * H];
#pragma unroll
            for (int h = 0; h < H; ++h) {
                src[h] = srcS ? srcS + h * row_w + (size_t)i * 2 : nullptr;
                src[H + h] = srcN ? srcN + h * row_w + (size_t)i * 2 : nullptr;
            }
            ok = wait_tagged_pairs<2 * H>(c, src, w, tag);
        } else {
            const unsigned long long* src[2 * H * P];
#pragma unroll
            for (int h = 0; h < H; ++h)
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    src[(h * P + k)] = srcS ? srcS + h * row_w + (size_t)i * P + k : nullptr;
                    src[(H + h) * P + k] = srcN ? srcN + h * row_w + (size_t)i * P + k : nullptr;
                }
            ok = wait_tagged<2 * H * P>(c, src, w, tag);
        }
#pragma unroll
        for (int h = 0; h < H; ++h) {
            unsigned pS[2] = {0u, 0u}, pN[2] = {0u, 0u};
#pragma unroll
            for (int k = 0; k < P; ++k) {
                pS[k] = (unsigned)w[h * P + k];
                pN[k] = (unsigned)w[(H + h) * P + k];
            }
            fromS[h][i] = srcS ? Pieces<T>::make(pS) : T(0);
            fromN[h][i] = srcN ? Pieces<T>::make(pN) : T(0);
        }
    }
    const bool failed = __syncthreads_or(!ok) != 0;
    if (failed) {
        if (threadIdx.x == 0 && !ld_acquire_s32(c.abort_flag)) team_fail(c, ST_ETIMEOUT);
        return false;
    }
    return true;
}

// Publish, then fetch at once (no work in between).
template <int NT, typename T, int H>
__device__ bool exchange_rows_tagged(const TeamCtl& c, Team& t, unsigned long long* tpub,
                                     const sptr<const T> (&lo)[H], const sptr<const T> (&hi)[H],
                                     const sptr<T> (&fromS)[H], const sptr<T> (&fromN)[H]) {
    const unsigned long long seq = publish_rows_tagged<NT, T, H>(t, tpub, lo, hi);
    return fetch_rows_tagged<NT, T, H>(c, t, tpub, seq, fromS, fromN);
}

// Team reduction over sequence-tagged words. Arrive: thread 0 publishes this CTA's K
// values for reduction `use` (slot use & 3, tag use + 1). Finish: warp 0 polls every
// CTA's words, lanes fold in CTA order with a fixed shuffle tree (max or sum, NaN
// propagates); the result goes to out on thread 0 (lane 0) only. A CTA publishes
// reduction use + 1 only after finishing use - 1, which needs every CTA's arrival at
// use - 1, so four slots are never overwritten while still being read.
template <int K>
__device__ __forceinline__ void tagged_arrive(Team& t, unsigned long long* tred, unsigned long long use,
                                              const double (&vals)[K]) {
    static_assert(2 * K <= kTagRedWords, "too many values");
    unsigned long long* w = tred + ((size_t)(use & 3) * t.G + t.b) * kTagRedWords;
    const unsigned tag = (unsigned)(use + 1);
#pragma unroll
    for (int k = 0; k < K; ++k)
        st_relaxed_v2(w + 2 * k, tagged(tag, Pieces<double>::get(vals[k], 0)), tagged(tag, Pieces<double>::get(vals[k], 1)));
}

// Warp 0 only. Returns false when a wait timed out or the launch aborted. MAXOP is for
// non-negative values (magnitudes and flags, NaN included): their bit patterns order
// like the values, so the maximum is taken on the integer pipe (NaN, above +Inf, wins).
template <int K, bool MAXOP>
__device__ __forceinline__ bool tagged_finish(const TeamCtl& c, const Team& t, const unsigned long long* tred,
                                              unsigned long long use, double (&out)[K]) {
    const int lane = threadIdx.x & 31;
    const unsigned tag = (unsigned)(use + 1);
    const unsigned long long* base = tred + (size_t)(use & 3) * t.G * kTagRedWords;
    double acc[K];
    unsigned long long kmax[K];
    bool nan[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        acc[k] = 0.0;
        kmax[k] = 0ull;
        nan[k] = false;
    }
    bool ok = true;
    for (int b = lane; b < t.G && ok; b += 32) {
        const unsigned long long* src[K];
        unsigned long long w[2 * K];
#pragma unroll
        for (int k = 0; k < K; ++k) src[k] = base + (size_t)b * kTagRedWords + 2 * k;
        ok = wait_tagged_pairs<K>(c, src, w, tag);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (MAXOP) {
                const unsigned long long bits = ((w[2 * k + 1] & 0xffffffffull) << 32) | (w[2 * k] & 0xffffffffull);
                kmax[k] = bits > kmax[k] ? bits : kmax[k];
            } else {
                const unsigned pw[2] = {(unsigned)w[2 * k], (unsigned)w[2 * k + 1]};
                const double v = Pieces<double>::make(pw);
                acc[k] += v;
                nan[k] |= (v != v);
            }
        }
    }
    ok = __all_sync(0xffffffffu, ok);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if (MAXOP) {
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long w = __shfl_xor_sync(0xffffffffu, kmax[k], o);
                kmax[k] = w > kmax[k] ? w : kmax[k];
            }
            out[k] = key_val(kmax[k]);
        } else {
            for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
            const bool any_nan = __any_sync(0xffffffffu, nan[k]);
            out[k] = any_nan ? __longlong_as_double(0x7ff8000000000000ll) : acc[k];
        }
    }
    return ok;
}

// Start a team reduction of K <= 4 values (this CTA's partials already block-reduced
// into vals). Deterministic: every CTA later combines the G partials in CTA order.
template <int K>
__device__ __forceinline__ unsigned long long reduce_arrive(Team& t, const double (&vals)[K]) {
    const unsigned long long use = t.red_seq++;
    const int slot = (int)(use & 3);
    if (threadIdx.x == 0) {
        double* part = t.red_part + ((size_t)slot * t.G + t.b) * 4;
#pragma unroll
        for (int k = 0; k < K; ++k) __stcg(part + k, vals[k]);
        __threadfence();
        atomicAdd(t.red_cnt + slot, 1ull);
    }
    return use;
}

// Finish reduction `use`: wait for all G arrivals, then one warp sums the partials
// (lane l takes CTAs l, l+32, ... in order, then a fixed xor-shuffle tree), or takes
// their max when MAXOP. Every CTA performs the identical sequence of operations, so
// all CTAs obtain the same value. Result is broadcast to every thread.
template <int K, bool MAXOP>
__device__ __forceinline__ bool reduce_finish(const TeamCtl& c, Team& t, unsigned long long use, double (&out)[K],
                                              double* s_bcast, int* s_ok) {
    const int slot = (int)(use & 3);
    if (threadIdx.x == 0) {
        const unsigned long long target = (unsigned long long)t.G * ((use >> 2) + 1);
        const unsigned long long t0 = global_ns();
        *s_ok = wait_geq(c, t.red_cnt + slot, target) ? 1 : 0;
        __threadfence();
        t.t_red += global_ns() - t0;
    }
    __syncthreads();
    const bool ok = *s_ok != 0;
    if (ok && threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const double* part = t.red_part + (size_t)slot * t.G * 4;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            bool nan = false;
            for (int b = lane; b < t.G; b += 32) {
                const double v = __ldcg(part + (size_t)b * 4 + k);
                s = MAXOP ? fmax(s, v) : s + v;
                nan |= (v != v);
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double w = __shfl_xor_sync(0xffffffffu, s, o);
                s = MAXOP ? fmax(s, w) : s + w;
            }
            nan = __any_sync(0xffffffffu, nan);
            if (lane == 0) s_bcast[k] = nan ? __longlong_as_double(0x7ff8000000000000ll) : s;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] = s_bcast[k];
    __syncthreads();
    return ok;
}

// Machine epsilon of the level-solve precision.
template <typename T> struct Eps;
template <> struct Eps<double> { static constexpr double value = 1.1102230246251565e-16; };
template <> struct Eps<float> { static constexpr double value = 5.9604644775390625e-08; };

// Shared-memory arrays of one CTA (cap elements each, cap = largest rows x nx). T is
// the precision of the level solve: double, or float for FP32 inner solves.
template <typename T>
struct Smem {
    sptr<T> cw, ce, cs, cn, bs, x;           // scaled couplings, scaled rhs, iterate
    sptr<T> r, rh, p, v, t;                  // BiCGStab vectors (s shares r)
    sptr<T> haloS, haloN;                    // neighbour rows of the exchanged vector
    double* red;                             // 64 doubles: block reductions [0,32), broadcast [32,48), flags [48,64)
                                             // (addressed by constant offsets and warp numbers only)
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Byte offset of the 64-double reduction area after the solver arrays and halos.
template <typename T>
__host__ __device__ inline size_t smem_red_offset(int cap, int nx) {
    return align_up(sizeof(T) * (11 * (size_t)cap + 2 * (size_t)nx), 16);
}

// Carve the layout: cw ce cs cn bs x r rh p v t | haloS haloN | red.
template <typename T>
__device__ __forceinline__ Smem<T> smem_layout(unsigned char* base, int cap, int nx) {
    Smem<T> m;
    T* b = reinterpret_cast<T*>(base);
    m.cw = chk(b, cap, kChkSmem + 0);
    m.ce = chk(b + cap, cap, kChkSmem + 1);
    m.cs = chk(b + 2 * cap, cap, kChkSmem + 2);
    m.cn = chk(b + 3 * cap, cap, kChkSmem + 3);
    m.bs = chk(b + 4 * cap, cap, kChkSmem + 4);
    m.x = chk(b + 5 * cap, cap, kChkSmem + 5);
    m.r = chk(b + 6 * cap, cap, kChkSmem + 6);
    m.rh = chk(b + 7 * cap, cap, kChkSmem + 7);
    m.p = chk(b + 8 * cap, cap, kChkSmem + 8);
    m.v = chk(b + 9 * cap, cap, kChkSmem + 9);
    m.t = chk(b + 10 * cap, cap, kChkSmem + 10);
    m.haloS = chk(b + 11 * cap, nx, kChkSmem + 11);
    m.haloN = chk(b + 11 * cap + nx, nx, kChkSmem + 12);
    m.red = reinterpret_cast<double*>(base + smem_red_offset<T>(cap, nx));
    return m;
}

// y = (D^{-1} A) v on the local rows (unit diagonal), halos of v in haloS/haloN.
template <int NT, typename T>
__device__ __forceinline__ void local_spmv(const Team& t, const Smem<T>& m, const sptr<const T> v, const sptr<T> y) {
    const int nx = t.nx;
    for (int k = threadIdx.x; k < t.nloc; k += NT) {
        const int jl = k / nx, i = k - jl * nx;
        const T vW = i > 0 ? v[k - 1] : T(0);
        const T vE = i < nx - 1 ? v[k + 1] : T(0);
        const T vS = jl > 0 ? v[k - nx] : m.haloS[i];
        const T vN = jl < t.nrows - 1 ? v[k + nx] : m.haloN[i];
        y[k] = v[k] + m.cw[k] * vW + m.ce[k] * vE + m.cs[k] * vS + m.cn[k] * vN;
    }
}

// Order-preserving key of |x| in an integer (max on the integer pipe; NaN sorts above +Inf).
__device__ __forceinline__ unsigned long long mag_key(double x) { return abs_key(x); }
__device__ __forceinline__ unsigned long long mag_key(float x) {
    return static_cast<unsigned long long>(__float_as_uint(x) & 0x7fffffffu);
}
template <typename T>
__device__ __forceinline__ double mag_val(unsigned long long k);
template <>
__device__ __forceinline__ double mag_val<double>(unsigned long long k) { return key_val(k); }
template <>
__device__ __forceinline__ double mag_val<float>(unsigned long long k) { return (double)__uint_as_float((unsigned)k); }

// One SOR point update on the Jacobi-scaled level system
// x + cw xW + ce xE + cs xS + cn xN = bs: t = x - bs + (cw xW + ce xE + cs xS + cn xN) is
// minus the point's residual and x' = x - omega t, so the point moves by omega |t|. Six FP64
// operations and no per-level scaling of the couplings. Shared by the owner of a point
// and by a neighbour that recomputes it, so both get the same bits.
template <typename T>
__device__ __forceinline__ T sor_point(T xk, T bs, T cw, T ce, T cs, T cn, T xW, T xE, T xS, T xN, T om, T& t) {
    T acc = xk - bs;
    acc = fma(cw, xW, acc);
    acc = fma(ce, xE, acc);
    acc = fma(cs, xS, acc);
    acc = fma(cn, xN, acc);
    t = acc;
    return fma(-om, acc, xk);
}

// Thread 0's stopping decision after sweep `sweep`, given d = the team's largest change
// of sweep - 1 (NaN flagged in nan): -1 abort, 0 continue, 1 converged or capped, 2 NaN.
// prev / prev2 carry the largest changes of the two sweeps before. With
// rho = max(omega - 1, d_{s-1} / d_{s-2}), d_{s-1} rho / (1 - rho) estimates the error after
// sweep s - 1, and sweep s, already done, shrinks it by rho once more: stop when
// d_{s-1} rho^2 <= tol (1 - rho). Written with A = rho d_{s-2} so that it needs no FP64
// division (a long dependent chain on GB300, while the other warps wait at a barrier):
// rho < 1 <=> A < d_{s-2}, and the test <=> d_{s-1} A^2 <= tol d_{s-2} (d_{s-2} - A).
// All changes may be scaled by one factor f > 0 if tol is divided by f.
__device__ __forceinline__ int sor_decision(bool nan, double d, double omega, double tol, int sweep, int max_iter,
                                            double& prev, double& prev2) {
    if (nan) return 2;
    prev2 = prev;
    prev = d;
    if (prev == 0.0 || sweep >= max_iter) return 1;
    if (!(prev2 > 0.0)) return 0;
    const double A = fmax((omega - 1.0) * prev2, prev);
    return (A < prev2 && prev * A * A <= tol * prev2 * (prev2 - A)) ? 1 : 0;
}

// Red-black SOR on the scaled level system x + W x_W + E x_E + S x_S + N x_N = bs,
// starting from x. Stops when the error estimate d_s rho / (1 - rho) <= tol, where
// d_s is the largest change of a sweep and rho = max(d_s / d_{s-1}, omega - 1); the
// global d_s is known one sweep late (lagged team reduction), so every CTA takes
// the same decision at the same sweep. Threads walk the points of one colour only
// (every lane of a warp does useful work). Scalar decisions are taken by thread 0
// and broadcast. The largest change of a sweep is omega times the largest |t| of its
// point updates (see sor_point). This form exchanges the halo before each half-sweep
// (flag protocol); teams with deep rows use level_sor_deep. Returns the sweep count
// (< 0 on abort).
template <int NT, typename T>
__device__ int level_sor(const TeamCtl& c, Team& t, const Smem<T>& m, double omega, double tol, int* s_ok) {
    const int nx = t.nx;
    const int half = (nx + 1) >> 1;            // points of one colour per row, at most
    const int npts = t.nrows * half;
    const T om = (T)omega;
    double prev = -1.0, prev2 = -1.0;          // global max change of sweeps s-1 and s-2 (thread 0)
    unsigned long long pending = 0;
    bool have_pending = false;
    int* s_flag = reinterpret_cast<int*>(m.red + 48);
    for (int sweep = 1;; ++sweep) {
        unsigned long long key = 0;
        for (int color = 0; color < 2; ++color) {
            if (!exchange_halo<NT, T>(c, t, m.x, m.haloS, m.haloN, s_ok)) return -1;
            for (int q = threadIdx.x; q < npts; q += NT) {
                const int jl = q / half;
                const int i = ((t.r0 + jl + color) & 1) + 2 * (q - jl * half);
                if (i >= nx) continue;
                const int k = jl * nx + i;
                const T xW = i > 0 ? m.x[k - 1] : T(0);
                const T xE = i < nx - 1 ? m.x[k + 1] : T(0);
                const T xS = jl > 0 ? m.x[k - nx] : m.haloS[i];
                const T xN = jl < t.nrows - 1 ? m.x[k + nx] : m.haloN[i];
                T tk;
                m.x[k] = sor_point<T>(m.x[k], m.bs[k], m.cw[k], m.ce[k], m.cs[k], m.cn[k], xW, xE, xS, xN, om, tk);
                const unsigned long long kk = mag_key(tk);
                key = kk > key ? kk : key;
            }
            __syncthreads();
        }
        // this CTA's max change (warp maxima, folded by thread 0), then arrive at the team
        // reduction of this sweep
        const unsigned long long use = t.red_seq++;
        {
            unsigned long long* wred = reinterpret_cast<unsigned long long*>(m.red);
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long w = __shfl_xor_sync(0xffffffffu, key, o);
                key = w > key ? w : key;
            }
            if ((threadIdx.x & 31) == 0) wred[threadIdx.x >> 5] = key;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned long long kmax = wred[0];
                for (int w = 1; w < NT / 32; ++w) kmax = wred[w] > kmax ? wred[w] : kmax;
                double* part = t.red_part + ((size_t)(use & 3) * t.G + t.b) * 4;
                __stcg(part, mag_val<T>(kmax) * omega);
                __threadfence();
                atomicAdd(t.red_cnt + (use & 3), 1ull);
            }
        }
        if (have_pending) {
            // warp 0 finishes the previous sweep's reduction; thread 0 decides
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                const int slot = (int)(pending & 3);
                int ok = 1;
                double d = 0.0;
                bool nan = false;
                const unsigned long long t0 = lane == 0 ? global_ns() : 0ull;
                if (lane == 0) {
                    const unsigned long long target = (unsigned long long)t.G * ((pending >> 2) + 1);
                    ok = wait_geq(c, t.red_cnt + slot, target) ? 1 : 0;
                    __threadfence();
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (ok) {
                    const double* part = t.red_part + (size_t)slot * t.G * 4;
                    for (int b = lane; b < t.G; b += 32) {
                        const double v = __ldcg(part + (size_t)b * 4);
                        d = fmax(d, v);
                        nan |= (v != v);
                    }
                    for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_xor_sync(0xffffffffu, d, o));
                    nan = __any_sync(0xffffffffu, nan);
                }
                if (lane == 0) t.t_red += global_ns() - t0;
                int decision = -1;  // -1 abort, 0 continue, 1 converged / capped, 2 NaN
                if (ok) {
                    decision = 0;
                    if (lane == 0) decision = sor_decision(nan, d, omega, tol, sweep, c.max_iter, prev, prev2);
                }
                if (lane == 0) *s_flag = decision;
            }
            __syncthreads();
            // s_flag is written again only after the next sweep's barriers
            const int decision = *s_flag;
            if (decision < 0) {
                if (threadIdx.x == 0 && !ld_acquire_s32(c.abort_flag)) team_fail(c, ST_ETIMEOUT);
                *s_ok = 0;
                return -1;
            }
            if (decision) {
                if (decision == 2 && threadIdx.x == 0) atomicCAS(c.status, 0, ST_EDIVERGED);
                // consume the outstanding reduction so the counter sequence stays aligned
                double h[1];
                if (!reduce_finish<1, true>(c, t, use, h, m.red + 32, s_ok)) return -1;
                return sweep;
            }
        }
        pending = use;
        have_pending = true;
    }
}

// Red-black SOR for a team with deep rows (see Deep), the same iteration and stopping
// rule as level_sor with one exchange per sweep, arranged so that the team's latencies
// overlap arithmetic:
//   1. the CTA publishes its first two and last two rows (as of the start of the sweep),
//   2. warp 0 issues the loads of the previous sweep's reduction words,
//   3. colour 0 on the interior rows, which need no halo, while both are in flight,
//   4. the neighbours' rows are fetched (normally already there),
//   5. colour 0 on the first and last rows, and the red points of the two halo rows as
//      their owners compute them (same arithmetic on the same values, same bits),
//   6. colour 1 on every row,
//   7. warp 0 completes the previous sweep's reduction from the prefetched words and
//      decides; one barrier; thread 0 publishes this sweep's largest change.
// The neighbours' boundary rows of the level system (deep->cS, deep->cN) must already be
// in place (the caller exchanges them once per level). The team reduces max |t| (the change
// over omega), so the tolerance comes as tol_w = tol / omega. Returns the sweep count (< 0
// on abort).
template <int NT, typename T>
__device__ int level_sor_deep(const TeamCtl& c, Team& t, const Smem<T>& m, double omega, double tol_w, int* s_ok,
                              const Deep<T>& deep) {
    // thread 0 adds each step's cycles to counters in shared memory (m.red[56..63]); the
    // counter reads also keep the compiler from moving work across the steps, which measured
    // faster than any schedule it picked on its own
    unsigned long long* const cyc = reinterpret_cast<unsigned long long*>(m.red + 56);
    const int nx = t.nx;
    const int half = (nx + 1) >> 1;            // points of one colour per row, at most
    const int nrows = t.nrows;
    const int last = (nrows - 1) * nx;
    const T om = (T)omega;
    const bool has_s = t.b > 0, has_n = t.b + 1 < t.G;
    const int lane = threadIdx.x & 31;
    double prev = -1.0, prev2 = -1.0;          // global max change of sweeps s-1 and s-2 (thread 0)
    unsigned long long pending = 0;
    bool have_pending = false;
    int* s_flag = reinterpret_cast<int*>(m.red + 48);
    unsigned long long* wred = reinterpret_cast<unsigned long long*>(m.red);
    const sptr<const T> lo[2] = {m.x, m.x + nx};
    const sptr<const T> hi[2] = {m.x + last, m.x + last - nx};
    const sptr<T> fS[2] = {m.haloS, deep.xS2};
    const sptr<T> fN[2] = {m.haloN, deep.xN2};
    // one point of a colour: local row jl, qi-th point of that colour in the row
    auto update = [&](int jl, int qi, int color, unsigned long long& key) {
        const int i = ((t.r0 + jl + color) & 1) + 2 * qi;
        if (i >= nx) return;
        const int k = jl * nx + i;
        const T xW = i > 0 ? m.x[k - 1] : T(0);
        const T xE = i < nx - 1 ? m.x[k + 1] : T(0);
        const T xS = jl > 0 ? m.x[k - nx] : m.haloS[i];
        const T xN = jl < nrows - 1 ? m.x[k + nx] : m.haloN[i];
        T tk;
        m.x[k] = sor_point<T>(m.x[k], m.bs[k], m.cw[k], m.ce[k], m.cs[k], m.cn[k], xW, xE, xS, xN, om, tk);
        const unsigned long long kk = mag_key(tk);
        key = kk > key ? kk : key;
    };
    // thread's first point (row, index in row) and the step of NT points, found once: the
    // sweep loops then walk their points without an integer division per point
    const int q_first = NT - 1 - (int)threadIdx.x;
    const int r_first = q_first / half, qi_first = q_first - r_first * half;
    const int dr = NT / half, dqi = NT - dr * half;
    for (int sweep = 1;; ++sweep) {
        unsigned long long key = 0;
        const long long c0 = clock64();
        // 1.
        const unsigned long long seq = publish_rows_tagged<NT, T, 2>(t, deep.tpub, lo, hi);
        const long long c1 = clock64();
        // 3. (the highest-numbered threads take the odd points out, so warp 0, which has the
        //    serial work of steps 4 and 7, finishes its share first)
        {
            int r = r_first, qi = qi_first;  // point NT - 1 - threadIdx.x, then NT points on
            for (int q = NT - 1 - threadIdx.x; q < (nrows - 2) * half; q += NT) {
                update(1 + r, qi, 0, key);
                qi += dqi;
                r += dr;
                if (qi >= half) {
                    qi -= half;
                    ++r;
                }
            }
        }
        const long long c2 = clock64();
        // 4.
        if (!fetch_rows_tagged<NT, T, 2>(c, t, deep.tpub, seq, fS, fN)) {
            *s_ok = 0;
            return -1;
        }
        const long long c3 = clock64();
        // 5.
        const int r_s = t.r0 - 1, r_n = t.r0 + nrows;
        for (int q = threadIdx.x; q < 4 * half; q += NT) {
            if (q < 2 * half) {
                if (q < half) update(0, q, 0, key);
                else if (nrows > 1) update(nrows - 1, q - half, 0, key);
            } else {
                const int qh = q - 2 * half;
                const bool south = qh < half;
                if (south ? !has_s : !has_n) continue;
                const int row = south ? r_s : r_n;
                const int i = (row & 1) + 2 * (south ? qh : qh - half);
                if (i >= nx) continue;
                const sptr<T> h = south ? m.haloS : m.haloN;
                const sptr<T>* cc = south ? deep.cS : deep.cN;
                const T xS = south ? deep.xS2[i] : m.x[last + i];
                const T xN = south ? m.x[i] : deep.xN2[i];
                const T xW = i > 0 ? h[i - 1] : T(0);
                const T xE = i < nx - 1 ? h[i + 1] : T(0);
                T unused;
                h[i] = sor_point<T>(h[i], cc[4][i], cc[0][i], cc[1][i], cc[2][i], cc[3][i], xW, xE, xS, xN, om, unused);
            }
        }
        const long long c4a = clock64();
        __syncthreads();
        const long long c4 = clock64();
        // 2. (issued here: by now every CTA has arrived at the previous sweep's reduction;
        //    teams of up to 32 CTAs, one word pair per lane; wider teams poll in step 7)
        unsigned long long pw0 = 0, pw1 = 0;
        const bool prefetched = have_pending && t.G <= 32;
        if (prefetched && threadIdx.x < 32 && lane < t.G)
            ld_relaxed_v2(deep.tred + ((size_t)(pending & 3) * t.G + lane) * kTagRedWords, pw0, pw1);
        // 6.
        {
            int r = r_first, qi = qi_first;
            for (int q = NT - 1 - threadIdx.x; q < nrows * half; q += NT) {
                update(r, qi, 1, key);
                qi += dqi;
                r += dr;
                if (qi >= half) {
                    qi -= half;
                    ++r;
                }
            }
        }
        const long long c5 = clock64();
        // 7.
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, key, o);
            key = w > key ? w : key;
        }
        if (lane == 0) wred[threadIdx.x >> 5] = key;
        if (have_pending && threadIdx.x < 32) {
            const unsigned long long t0 = lane == 0 ? global_ns() : 0ull;
            bool ok = true;
            double d = 0.0;
            bool nan = false;
            if (prefetched) {
                unsigned long long dk = 0ull;
                if (lane < t.G) {
                    const unsigned tag = (unsigned)(pending + 1);
                    unsigned long long w[2] = {pw0, pw1};
                    if ((unsigned)(w[0] >> 32) != tag || (unsigned)(w[1] >> 32) != tag) {
                        const unsigned long long* src[1] = {deep.tred + ((size_t)(pending & 3) * t.G + lane) *
                                                                            kTagRedWords};
                        ok = wait_tagged_pairs<1>(c, src, w, tag);
                    }
                    dk = ((w[1] & 0xffffffffull) << 32) | (w[0] & 0xffffffffull);
                }
                ok = __all_sync(0xffffffffu, ok);
                // non-negative values (or NaN): the maximum of the bit patterns, integer pipe
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long w = __shfl_xor_sync(0xffffffffu, dk, o);
                    dk = w > dk ? w : dk;
                }
                d = key_val(dk);
                nan = d != d;
            } else {
                double g1[1];
                ok = tagged_finish<1, true>(c, t, deep.tred, pending, g1);
                d = g1[0];
                nan = d != d;
            }
            if (lane == 0) {
                t.t_red += global_ns() - t0;
                *s_flag = ok ? sor_decision(nan, d, omega, tol_w, sweep, c.max_iter, prev, prev2) : -1;
            }
        }
        const long long c6a = clock64();
        __syncthreads();
        const long long c6 = clock64();
        if (threadIdx.x == 0) {
            cyc[0] += c1 - c0;   // 1-2 publish
            cyc[1] += c2 - c1;   // 3 interior colour 0
            cyc[2] += c3 - c2;   // 4 fetch
            cyc[3] += c4a - c3;  // 5 boundary rows and halo points
            cyc[4] += c4 - c4a;  //   barrier
            cyc[5] += c5 - c4;   // 6 colour 1
            cyc[6] += c6a - c5;  // 7 reduction and decision
            cyc[7] += c6 - c6a;  //   barrier
        }
        const unsigned long long use = t.tag_seq++;
        if (threadIdx.x == 0) {
            unsigned long long kmax = wred[0];
            for (int w = 1; w < NT / 32; ++w) kmax = wred[w] > kmax ? wred[w] : kmax;
            const double v1[1] = {mag_val<T>(kmax)};  // max |t|: the change is omega times it
            tagged_arrive<1>(t, deep.tred, use, v1);
        }
        if (have_pending) {
            // s_flag and wred are written again only after the next sweep's barriers
            const int decision = *s_flag;
            if (decision < 0) {
                if (threadIdx.x == 0 && !ld_acquire_s32(c.abort_flag)) team_fail(c, ST_ETIMEOUT);
                *s_ok = 0;
                return -1;
            }
            if (decision) {
                if (decision == 2 && threadIdx.x == 0) atomicCAS(c.status, 0, ST_EDIVERGED);
                return sweep;
            }
        }
        pending = use;
        have_pending = true;
    }
}

// Broadcast a double computed by thread 0 to every thread of the CTA.
__device__ __forceinline__ double bcast0(double v, double* slot) {
    if (threadIdx.x == 0) *slot = v;
    __syncthreads();
    v = *slot;
    __syncthreads();
    return v;
}

// Jacobi-preconditioned BiCGStab (van der Vorst 1992) on the scaled level system,
// from x = 0; s shares storage with r. Vectors in precision T, dot products and
// recurrence scalars in FP64. Stops when ||r||_2 <= max(eta, 16 eps_T) ||bs||_2. Scalars are formed by thread 0 and broadcast (FP64 division
// is costly on this part). Returns the iteration count (< 0 on abort).
template <int NT, typename T>
__device__ int level_bicgstab(const TeamCtl& c, Team& t, const Smem<T>& m, double eta, double atol, int* s_ok) {
    double* sb = m.red + 32;
    double* slot = m.red + 48;
    const int nloc = t.nloc;
    // r = bs, rh = bs, x = 0, p = v = 0
    double one[1] = {0.0};
    for (int k = threadIdx.x; k < nloc; k += NT) {
        const T b = m.bs[k];
        m.x[k] = T(0);
        m.r[k] = b;
        m.rh[k] = b;
        m.p[k] = T(0);
        m.v[k] = T(0);
        one[0] += (double)b * (double)b;
    }
    block_sum<NT, 1>(one, m.red);
    double g1[1];
    if (!reduce_finish<1, false>(c, t, reduce_arrive<1>(t, one), g1, sb, s_ok)) return -1;
    // thread 0 keeps the recurrence scalars; others receive what they need
    double tol = 0.0, rho_old = 1.0, alpha = 1.0, omega = 1.0, rho = g1[0];
    if (threadIdx.x == 0) {
        // relative to the scaled rhs only: an absolute floor would act on a residual that
        // the Jacobi scaling has divided by the diagonal
        const double bn = sqrt(g1[0]);
        tol = fmax(eta * bn, 16.0 * Eps<T>::value * bn);
    }
    if (bcast0(threadIdx.x == 0 ? (sqrt(g1[0]) <= tol ? 1.0 : 0.0) : 0.0, slot) != 0.0) return 0;
    for (int it = 1; it <= c.max_iter; ++it) {
        double beta = 0.0;
        if (threadIdx.x == 0) beta = (rho / rho_old) * (alpha / omega);
        const T beta_t = (T)bcast0(beta, slot);
        const T om_b = (T)bcast0(omega, slot);
        for (int k = threadIdx.x; k < nloc; k += NT) m.p[k] = m.r[k] + beta_t * (m.p[k] - om_b * m.v[k]);
        __syncthreads();
        if (!exchange_halo<NT, T>(c, t, m.p, m.haloS, m.haloN, s_ok)) return -1;
        local_spmv<NT, T>(t, m, m.p, m.v);
        double d1[1] = {0.0};
        for (int k = threadIdx.x; k < nloc; k += NT) d1[0] += (double)m.rh[k] * (double)m.v[k];
        block_sum<NT, 1>(d1, m.red);
        if (!reduce_finish<1, false>(c, t, reduce_arrive<1>(t, d1), d1, sb, s_ok)) return -1;
        // code: 0 go on, 1 NaN, 2 breakdown
        double code = 0.0;
        if (threadIdx.x == 0) {
            if (d1[0] != d1[0]) code = 1.0;
            else if (d1[0] == 0.0) code = 2.0;
            else alpha = rho / d1[0];
        }
        code = bcast0(code, slot);
        if (code != 0.0) {
            if (threadIdx.x == 0) atomicCAS(c.status, 0, code == 1.0 ? ST_EDIVERGED : ST_ENOCONV);
            return it;
        }
        const T al_b = (T)bcast0(alpha, slot);
        for (int k = threadIdx.x; k < nloc; k += NT) m.r[k] -= al_b * m.v[k];  // r holds s
        __syncthreads();
        if (!exchange_halo<NT, T>(c, t, m.r, m.haloS, m.haloN, s_ok)) return -1;
        local_spmv<NT, T>(t, m, m.r, m.t);
        double d2[2] = {0.0, 0.0};
        for (int k = threadIdx.x; k < nloc; k += NT) {
            d2[0] += (double)m.t[k] * (double)m.r[k];
            d2[1] += (double)m.t[k] * (double)m.t[k];
        }
        block_sum<NT, 2>(d2, m.red);
        if (!reduce_finish<2, false>(c, t, reduce_arrive<2>(t, d2), d2, sb, s_ok)) return -1;
        if (threadIdx.x == 0) omega = d2[1] > 0.0 ? d2[0] / d2[1] : 0.0;
        const T om2 = (T)bcast0(omega, slot);
        double d3[2] = {0.0, 0.0};
        for (int k = threadIdx.x; k < nloc; k += NT) {
            const T sk = m.r[k];
            m.x[k] += al_b * m.p[k] + om2 * sk;
            const T rk = sk - om2 * m.t[k];
            m.r[k] = rk;
            d3[0] += (double)m.rh[k] * (double)rk;
            d3[1] += (double)rk * (double)rk;
        }
        block_sum<NT, 2>(d3, m.red);
        if (!reduce_finish<2, false>(c, t, reduce_arrive<2>(t, d3), d3, sb, s_ok)) return -1;
        // code: 0 go on, 1 NaN, 2 breakdown, 3 converged
        code = 0.0;
        if (threadIdx.x == 0) {
            const double rnorm = sqrt(d3[1]);
            if (rnorm != rnorm) code = 1.0;
            else if (rnorm <= tol) code = 3.0;
            else if (omega == 0.0 || d3[0] == 0.0) code = 2.0;
            rho_old = rho;
            rho = d3[0];
        }
        code = bcast0(code, slot);
        if (code == 3.0) return it;
        if (code != 0.0) {
            if (threadIdx.x == 0) atomicCAS(c.status, 0, code == 1.0 ? ST_EDIVERGED : ST_ENOCONV);
            return it;
        }
    }
    if (threadIdx.x == 0) atomicCAS(c.status, 0, ST_ENOCONV);
    return c.max_iter;
}

// Thread 0: SOR's omega for a level with Jacobi-scaled Gershgorin bound rho_g (< 1), in
// FP32 (a few digits suffice, and GB300's FP32 square root and division are short):
// omega = 2 / (1 + sqrt(1 - rho^2)) (Young), capped below 2 / (1 + rho) when some row has
// opposite-signed couplings (see level_solve).
__device__ __forceinline__ double sor_omega(double rho_g, bool nonsym) {
    if (!(rho_g < 1.0)) return 1.0;
    const float rc = (float)fmin(rho_g, 0.999999);
    float w = 2.0f / (1.0f + sqrtf(1.0f - rc * rc));
    if (nonsym) w = fmaxf(1.0f, fminf(w, 0.99f * 2.0f / (1.0f + (float)rho_g)));
    return (double)w;
}

// Solve the scaled level system in m with the method chosen from the level's
// Gershgorin bound rho_g; SOR's omega = 2/(1 + sqrt(1 - rho^2)) is formed by
// thread 0. Returns iterations (< 0 on abort) and the method used (1 SOR, 2 BiCGStab).
// When some row has opposite-signed couplings in x or y (a cell Peclet number
// above 2) the Jacobi spectrum may be complex and Young's omega may diverge; omega is
// then capped below 2/(1 + rho), the bound under which SOR converges for any
// strictly diagonally dominant matrix with Jacobi row sums <= rho.
template <int NT, typename T>
__device__ __forceinline__ int level_solve(const TeamCtl& c, Team& t, const Smem<T>& m, int method, double sor_rho_max,
                                           double rho_g, bool nonsym, double sor_tol, double eta, double atol,
                                           int* s_ok, int* used, const Deep<T>* deep = nullptr) {
    const bool use_sor = method == 1 || (method == 0 && rho_g < sor_rho_max);
    *used = use_sor ? 1 : 2;
    if (use_sor) {
        double omega = 1.0;
        if (threadIdx.x == 0) omega = sor_omega(rho_g, nonsym);
        omega = bcast0(omega, m.red + 48);
        return deep ? level_sor_deep<NT, T>(c, t, m, omega, sor_tol / omega, s_ok, *deep)
                    : level_sor<NT, T>(c, t, m, omega, sor_tol, s_ok);
    }
    return level_bicgstab<NT, T>(c, t, m, eta, atol, s_ok);
}

// level_solve for the wavefront kernel: the method, omega and the tolerances come decided
// (thread 0 forms them with the forcing term and broadcasts them in one barrier).
template <int NT, typename T>
__device__ __forceinline__ int level_solve_decided(const TeamCtl& c, Team& t, const Smem<T>& m, bool use_sor,
                                                   double omega, double sor_tol_w, double eta, double atol, int* s_ok,
                                                   const Deep<T>* deep) {
    if (use_sor)
        return deep ? level_sor_deep<NT, T>(c, t, m, omega, sor_tol_w, s_ok, *deep)
                    : level_sor<NT, T>(c, t, m, omega, sor_tol_w * omega, s_ok);
    return level_bicgstab<NT, T>(c, t, m, eta, atol, s_ok);
}

// Number of doubles of dynamic shared memory per CTA of chain_kernel.
__host__ __device__ inline size_t chain_smem_doubles(int nloc, int nx) {
    return smem_red_offset<double>(nloc, nx) / sizeof(double) + 64;
}

struct ChainArgs {
    int nx, ny, M;
    int G;                                  // CTAs per level (team size), = gridDim.x
    int rows_base, rows_rem;                // CTA b owns rows_base + (b < rows_rem) rows
    const double* R;                        // [M][Ns] right-hand sides r^n
    const double* coef;                     // [5][M][Ns] scaled planes (raw entries when RAW)
    const unsigned long long* rho_key;      // [2M] Gershgorin bound, then nonsymmetric-row flag, per level (unused when RAW)
    double* U;                              // [M][Ns] iterate, += dU when update_U
    double* dU;                             // [M][Ns] receives dU, or nullptr
    int update_U;
    int method;                             // 0 auto, 1 SOR, 2 BiCGStab
    double sor_rho_max;
    double eta;                             // relative tolerance of every level solve
    double sor_tol_abs;                     // > 0: absolute SOR tolerance instead of eta*||b||_inf
    double atol;                            // absolute floor of the tolerance
    int max_iter;                           // cap per level
    long long wait_budget;
    // team communication (zeroed before each launch by the host)
    double* pub;                            // [2][G][2][nx] published boundary rows
    unsigned long long* flags;              // [G] publication counters
    double* red_part;                       // [4][G][4] reduction partials
    unsigned long long* red_cnt;            // [4] arrival counters
    int* abort_flag;
    int* status;
    // statistics
    int* level_iters;                       // [M] sweeps / iterations of each level
    int* level_method;                      // [M] 1 = SOR, 2 = BiCGStab
    double* cta_sumsq;                      // [G] sum of dU^2 over the CTA's rows, all levels
    unsigned long long* timers;             // [4] CTA 0: ns waiting on halos, on reductions, total
};

// The chain: for n = 1..M, rhs = r^n + du^{n-1}; solve the level; U^n += du^n.
// Must be launched cooperatively with gridDim.x = G (all CTAs co-resident).
// RAW = false: a.coef holds the Jacobi-scaled planes and a.rho_key the Gershgorin
// bound of every level (both from assemble_kernel<SCALED>). RAW = true: a.coef
// holds the raw entries C, W, E, S, N of A_n; each level is scaled on load and its
// bound is formed by a team max-reduction.
template <int NT, bool RAW = false>
__global__ void __launch_bounds__(NT) chain_kernel(ChainArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_ok;
    TeamCtl c{a.abort_flag, a.status, a.wait_budget, a.max_iter};
    Team t;
    team_init(t, blockIdx.x, a.G, a.nx, a.ny, a.rows_base, a.rows_rem, a.pub, a.flags, a.red_part, a.red_cnt);
    const unsigned long long t_start = global_ns();
    const int nloc = t.nloc;
    const int cap = (a.rows_base + (a.rows_rem ? 1 : 0)) * a.nx;  // largest nloc of the team
    const Smem<double> m = smem_layout<double>(smem, cap, a.nx);

    const long long Ns = t.Ns;
    const long long plane = (long long)a.M * Ns;
    const long long off0 = (long long)t.r0 * a.nx;
    double sumsq = 0.0;
    const auto coefg = chk(a.coef, 5 * plane, kChkCoef);
    const auto Rg = chk(a.R, plane, kChkR);
    const auto Ug = chk(a.U, plane, kChkU);
    const auto dUg = chk(a.dU, plane, kChkDU);
    const auto rho_keyg = chk(a.rho_key, 2 * (long long)a.M, kChkLevel);

    // du^0 = 0 lives in x
    for (int k = threadIdx.x; k < nloc; k += NT) m.x[k] = 0.0;
    __syncthreads();

    for (int n = 0; n < a.M; ++n) {
        const long long lo = (long long)n * Ns + off0;
        const auto cd = coefg + lo;
        // rhs b = r^n + du^{n-1}, scaled by 1/C; load the couplings
        double rho_g;
        bool nonsym;
        if (!RAW) {
            for (int k = threadIdx.x; k < nloc; k += NT) {
                const double d = cd[k];
                m.cw[k] = cd[plane + k];
                m.ce[k] = cd[2 * plane + k];
                m.cs[k] = cd[3 * plane + k];
                m.cn[k] = cd[4 * plane + k];
                const double b = Rg[lo + k] + m.x[k];
                m.bs[k] = d * b;
                m.x[k] = b;  // SOR start: unscaled rhs (exact for the smooth modes where A ~ I)
            }
            __syncthreads();
            rho_g = key_val(rho_keyg[n]);
            nonsym = rho_keyg[a.M + n] != 0ull;
        } else {
            // row sums folded as order-preserving keys: a NaN entry gives a NaN bound
            // (above +Inf), so the level goes to BiCGStab, which reports it
            unsigned long long rs = 0ull;
            bool ns = false;
            for (int k = threadIdx.x; k < nloc; k += NT) {
                const double d = 1.0 / cd[k];
                const double w = cd[plane + k] * d, e = cd[2 * plane + k] * d;
                const double sv = cd[3 * plane + k] * d, nv = cd[4 * plane + k] * d;
                m.cw[k] = w;
                m.ce[k] = e;
                m.cs[k] = sv;
                m.cn[k] = nv;
                const double b = Rg[lo + k] + m.x[k];
                m.bs[k] = d * b;
                m.x[k] = b;
                const unsigned long long kr = abs_key(fabs(w) + fabs(e) + fabs(sv) + fabs(nv));
                rs = kr > rs ? kr : rs;
                ns |= (w * e < 0.0 || sv * nv < 0.0);
            }
            double v[2];
            v[0] = key_val(block_max_u64<NT>(rs, reinterpret_cast<unsigned long long*>(m.red)));
            v[1] = key_val(block_max_u64<NT>(ns ? abs_key(1.0) : 0ull, reinterpret_cast<unsigned long long*>(m.red)));
            double g[2];
            if (!reduce_finish<2, true>(c, t, reduce_arrive<2>(t, v), g, m.red + 32, &s_ok)) return;
            rho_g = g[0];
            nonsym = g[1] != 0.0;
        }
        double sor_tol = a.sor_tol_abs;
        const bool sor_here = a.method == 1 || (a.method == 0 && rho_g < a.sor_rho_max);
        if (sor_here && !(sor_tol > 0.0)) {
            // tolerance relative to the level's unscaled ||b||_inf (team max reduction)
            double bl = 0.0;
            for (int k = threadIdx.x; k < nloc; k += NT) bl = fmax(bl, fabs(m.x[k]));
            unsigned long long key = block_max_u64<NT>(abs_key(bl), reinterpret_cast<unsigned long long*>(m.red));
            double v[1] = {key_val(key)};
            double g[1];
            if (!reduce_finish<1, true>(c, t, reduce_arrive<1>(t, v), g, m.red + 32, &s_ok)) return;
            sor_tol = fmax(a.eta * g[0], a.atol);
        }
        int used = 0;
        const int iters = level_solve<NT, double>(c, t, m, a.method, a.sor_rho_max, rho_g, nonsym, sor_tol, a.eta,
                                                  a.atol, &s_ok, &used);
        if (iters < 0) return;  // aborted
        // du^n = x: update the iterate and keep x as du^{n-1} of the next level
        for (int k = threadIdx.x; k < nloc; k += NT) {
            const double dx = m.x[k];
            if (a.update_U) Ug[lo + k] += dx;
            if (a.dU) dUg[lo + k] = dx;
            sumsq += dx * dx;
        }
        if (t.b == 0 && threadIdx.x == 0) {
            chk(a.level_iters, a.M, kChkLevel)[n] = iters;
            chk(a.level_method, a.M, kChkLevel)[n] = used;
            if (iters >= a.max_iter) atomicCAS(a.status, 0, ST_ENOCONV);
        }
        __syncthreads();
    }
    double ss[1] = {sumsq};
    block_sum<NT, 1>(ss, m.red);
    if (threadIdx.x == 0) chk(a.cta_sumsq, a.G, kChkSumsq)[t.b] = ss[0];
    if (t.b == 0 && threadIdx.x == 0) {
        a.timers[0] = t.t_halo;
        a.timers[1] = t.t_red;
        a.timers[2] = global_ns() - t_start;
    }
}

// --------------------------------------- the Newton wavefront (a1 + a2 + a3 + a4)

// All Newton iterations of the all-at-once system in one cooperative launch.
// K teams of G CTAs; team t runs iterations k = k_begin + t, k_begin + t + K, ...
// Cell (k, n) -- Newton iteration k at level n -- needs u^n_k, final once cell
// (k-1, n) has updated it, and du^{n-1}_k, which the same team produced one level
// earlier and still holds in shared memory. So iteration k walks the levels right
// behind iteration k - 1: up to K iterations are in flight, and the latency of
// one level solve is overlapped with the others. Per cell, the team computes the
// residual r^n_k (eq. 3-5) and the scaled Jacobian entries (eq. 5-6) of its rows
// from u^n_k (global, own and halo rows) and u^{n-1}_k (shared memory), then
// solves A_n du^n = r^n + du^{n-1} (eq. 7 nested) and updates U^n. The iterates are
// those of plain Newton; the forcing term uses the running max of ||r^j_k||_inf
// over the levels j <= n seen so far. Cell (k, n) is skipped (du^n_k = 0) when the
// previous iteration's running max at level n is already <= tol_res: the levels
// 0..n have converged and, the system being block lower-triangular in time, need
// no further update. The rule depends only on finished cells, so the result is
// the same on every run. When an iteration ends with a running max <= tol_res,
// every later cell is a skip; the team raises a stop flag so the others leave early.
// The mbarrier of a CTA's bulk copies and the parity of its current phase. Initialised
// once per launch (mbarrier.init on a live barrier is undefined), carried through every
// wavefront body the CTA runs; every copy is waited for before the next is issued.
struct BulkBar {
    unsigned long long* bar;
    unsigned phase;
};

struct WaveArgs {
    OpConst c;
    const double* u0;
    const double* bc;
    const double* q;
    double* U;
    int K, G, rows_base, rows_rem;      // G: CTAs per team and stride of the team workspaces;
                                        // rows_base/rows_rem: the strips of a G-CTA team
    const int* tgeom;                   // [K][4] per team (first block, CTAs <= G, rows_base, rows_rem),
                                        // or null: every team has G CTAs. Either way the largest
                                        // strip has rows_base + (rows_rem > 0) rows.
    int k_begin, k_end;                 // iterations k_begin <= k < k_end may run
    int bulk_u;                         // u^n_k strips by bulk copy (nx even, U 16-byte aligned)
    unsigned long long cell_base;       // added to every progress value (monotonic across calls)
    double tol_res, eta_max, eta_gamma, atol, sor_rho_max;
    int method;
    int max_iter;
    long long wait_budget;
    // workspace, zeroed by the host before the launch (stop[1] set to INT_MAX)
    double* pub;                        // [K][2][G][2][nx]
    unsigned long long* tpub;           // [K][2][G][kDeepSlotRows][nx][2] tagged words (one-exchange SOR), or nullptr
    unsigned long long* tred;           // [K][4][G][kTagRedWords] tagged reduction words (with tpub)
    unsigned long long* flags;          // [K][G]
    double* red_part;                   // [K][4][G][4]
    unsigned long long* red_cnt;        // [K][4]
    unsigned long long* prog;           // [K][G] cells completed: k * M + n + 1
    int* abort_flag;
    int* status;
    int* stop;                          // [0] stop flag, [1] first converged iteration (K > 1; may be null)
    int* kconv;                         // one team (K = 1): CTA 0 writes the converged iteration; several
                                        // teams of a batch: -2 marks a diverged window (may be null)
    // per iteration records, indexed by k
    double* res_inf;                    // [k_end] ||R_k||_inf
    double* cell_prefix;                // [k_end][M] max_{j <= n} ||r^j_k||_inf (written by CTA 0 of the team)
    int* cell_iters;                    // [k_end][M] 1 + sweeps (SOR) or -(1 + iterations) (BiCGStab); 0 = not run
    double* cta_sumsq;                  // [k_end][G] sum of du_k^2 over the CTA's rows
    unsigned long long* timers;         // [K][kWaveTimers] CTA 0 of each team (see kWaveTimers)
};

// Phase timers of CTA 0 of every team of a wavefront launch, per team (ns unless noted):
// 0 halo waits (flag protocol), 1 team-reduction waits, 2 waits for the previous Newton
// iteration, 3 total, 4 level setup (all of it), 5 level solves, 6 updates and progress
// publication, 7 setup: loading u^n_k, 8 setup: team reduction and boundary-row exchange,
// 9 cells solved (count), 10 sweeps or iterations (count), 11 unused, 12..19 cycles of
// CTA 0's thread 0 in the steps of the deep SOR sweeps (see level_sor_deep): publish,
// interior colour 0, fetch, boundary rows and halo points, barrier, colour 1, reduction and
// decision, barrier; 20..24 cycles of CTA 0's thread 0 in the steps of the level setup: the
// node loop (residual, couplings, rhs), the block reduction, publishing the boundary rows of
// the level system, the team reduction (arrive, wait, broadcast), fetching the neighbours'
// boundary rows.
constexpr int kWaveTimers = 25;

// u^n_k with its halo rows ((cap + 2 nx) doubles) shares the BiCGStab scratch r..t
// when it fits there; otherwise it follows uprev.
template <typename T>
__host__ __device__ inline bool wave_u_aliases(int cap, int nx) {
    return (size_t)(cap + 2 * (size_t)nx) * sizeof(double) <= 5 * (size_t)cap * sizeof(T);
}

// Dynamic shared memory of wave_kernel<T>: solver arrays, halos, reduction area,
// uprev (cap doubles) and, unless aliased, u.
template <typename T>
__host__ __device__ inline size_t wave_smem_bytes(int cap, int nx) {
    size_t bytes = smem_red_offset<T>(cap, nx) + 64 * sizeof(double) + sizeof(double) * (size_t)cap;
    if (!wave_u_aliases<T>(cap, nx)) bytes += sizeof(double) * (cap + 2 * (size_t)nx);
    return bytes;
}

// The work of CTA b of team `team` in a wavefront launch (or one window of one
// instance of a batched launch). t is the CTA's team state, already initialised
// with the team's workspace; its sequence counters carry over between calls.
template <int NT, bool CONV, bool NLV, typename T>
__device__ void wave_body(const WaveArgs& a, int team, int b, Team& t, unsigned char* smem, int& s_ok, BulkBar& bb) {
    const OpConst& oc = a.c;
    const int nx = oc.nx, ny = oc.ny, M = oc.M;
    TeamCtl c{a.abort_flag, a.status, a.wait_budget, a.max_iter};
    const unsigned long long t_start = global_ns();
    unsigned long long t_pred = 0, t_setup = 0, t_solve = 0, t_upd = 0, t_mark = 0;
    unsigned long long t_load = 0, t_sred = 0, n_cells = 0, n_sweeps = 0;
    const int nloc = t.nloc;
    const int cap = (a.rows_base + (a.rows_rem ? 1 : 0)) * nx;
    const Smem<T> m = smem_layout<T>(smem, cap, nx);
    // u^{n-1}_k, own rows (cap doubles), after the reduction area
    double* const uprev_p = reinterpret_cast<double*>(smem + smem_red_offset<T>(cap, nx) + 64 * sizeof(double));
    const sptr<double> uprev = chk(uprev_p, cap, kChkUprev);
    // u^n_k with one halo row each side: (nrows + 2) x nx doubles
    const sptr<double> u = chk(wave_u_aliases<T>(cap, nx) ? reinterpret_cast<double*>(static_cast<T*>(m.r)) : uprev_p + cap,
                               cap + 2 * nx, kChkUstrip);
    const long long Ns = t.Ns;
    const long long off0 = (long long)t.r0 * nx;
    const int nb = 2 * nx + 2 * ny;
    // the problem's arrays (levels 0..M-1 of this call) and the per-iteration records
    const auto Ug = chk(a.U, (long long)M * Ns, kChkU);
    const auto u0g = chk(a.u0, Ns, kChkU0);
    const auto bcg = chk(a.bc, (long long)M * nb, kChkBc);
    const auto qg = chk(a.q, (long long)M * Ns, kChkQ);
    const auto prefixg = chk(a.cell_prefix, (long long)a.k_end * M, kChkPrefix);
    const auto itersg = chk(a.cell_iters, (long long)a.k_end * M, kChkCellIters);
    const int pred_team = (team + a.K - 1) % a.K;
    const auto pred_prog = chk(a.prog, (long long)a.K * a.G, kChkProg) + (long long)pred_team * a.G;
    // the predecessor team's CTAs that own rows r0-1 .. r0+nrows (its strips may differ from ours)
    int p_lo = b - 1, p_hi = b + 1;
    if (a.tgeom) {
        const int prb = a.tgeom[4 * pred_team + 2], prr = a.tgeom[4 * pred_team + 3];
        const int big = prr * (prb + 1);  // rows of its longer strips, which come first
        const int rlo = max(t.r0 - 1, 0), rhi = min(t.r0 + t.nrows, ny - 1);
        p_lo = rlo < big ? rlo / (prb + 1) : prr + (rlo - big) / prb;
        p_hi = rhi < big ? rhi / (prb + 1) : prr + (rhi - big) / prb;
    }
    const int p_cnt = a.tgeom ? a.tgeom[4 * pred_team + 1] : a.G;
    const auto my_prog = chk(a.prog, (long long)a.K * a.G, kChkProg) + (long long)team * a.G;
    double* slot = m.red + 48;
    // Burgers-type closures with constant viscosity have a constant diagonal 1 + 2 mu_a (vx + vy)
    const double dconst = 1.0 / (1.0 + 2.0 * oc.mu_a * (oc.vx + oc.vy));
    // their folded constants: viscous mu_a tau / h^2, and the scaled couplings
    const double vmu_x = oc.vmx, vmu_y = oc.vmy;
    const double kcen = oc.kcen;
    const double sjx = oc.jx * dconst, sjy = oc.jy * dconst, svx = vmu_x * dconst, svy = vmu_y * dconst;
    // the same in the level-solve precision (FP32 solves form their couplings in FP32)
    const T sjx_t = (T)sjx, sjy_t = (T)sjy, svx_t = (T)svx, svy_t = (T)svy, dconst_t = (T)dconst;
    // neighbour rows for one-exchange SOR sweeps: in the BiCGStab scratch r..t (5 cap values),
    // which SOR leaves unused and u^n_k no longer needs once the level's system is formed.
    // The conditions are the same on every CTA of the team (cap and rows_base are team-wide).
    Deep<T> deep_rows;
    const Deep<T>* deep = nullptr;
    if (a.tpub && a.tred && t.G >= 2 && t.rows_base >= 2 && 12 * (size_t)nx <= 5 * (size_t)cap) {
        T* const d0 = static_cast<T*>(m.r);
        for (int h = 0; h < 5; ++h) {
            deep_rows.cS[h] = chk(d0 + (size_t)h * nx, nx, kChkDeep);
            deep_rows.cN[h] = chk(d0 + (size_t)(5 + h) * nx, nx, kChkDeep);
        }
        deep_rows.xS2 = chk(d0 + (size_t)10 * nx, nx, kChkDeep);
        deep_rows.xN2 = chk(d0 + (size_t)11 * nx, nx, kChkDeep);
        deep_rows.tpub = a.tpub + (size_t)team * 2 * a.G * kDeepSlotRows * nx * 2;
        deep_rows.tred = a.tred + (size_t)team * 4 * a.G * kTagRedWords;
        deep = &deep_rows;
    }

    unsigned long long* const ubar = bb.bar;
    // thread 0's cycle counters: the deep sweeps' steps in m.red[56..63], the setup's in m.red[50..54]
    unsigned long long* const scyc = reinterpret_cast<unsigned long long*>(m.red + 50);
    if (threadIdx.x == 0) {
        for (int q = 0; q < 8; ++q) reinterpret_cast<unsigned long long*>(m.red + 56)[q] = 0ull;
        for (int q = 0; q < 5; ++q) scyc[q] = 0ull;
    }
    __syncthreads();
    for (int k = a.k_begin + team; k < a.k_end; k += a.K) {
        for (int i = threadIdx.x; i < nloc; i += NT) {
            m.x[i] = T(0);              // du^{-1} = 0
            uprev[i] = u0g[off0 + i];   // u^0
        }
        double prefix = 0.0;            // running max of ||r^j_k||_inf, j <= n (thread 0)
        double sumsq = 0.0;
        float sumsq_f = 0.0f;
        bool uprev_valid = true;        // uprev holds u^{n-1}_k (false after a skipped level)
        double first_res = 1.0 / 0.0;   // iteration 0's running residual at the current level
        __syncthreads();
        for (int n = 0; n < M; ++n) {
            // 1. wait until iteration k - 1 has finished level n on rows r0-1 .. r0+nrows and
            //    on CTA 0 (which publishes its running residual max): lanes of warp 0 poll the
            //    progress words of the predecessor's CTAs p_lo..p_hi (b-1, b, b+1 when the
            //    teams' strips match) and lane 31 its CTA 0, at once (acquire)
            const int pl = p_lo <= 0 ? -p_lo : 31;  // the lane that polls CTA 0
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                bool stop_seen = false;
                if (k > a.k_begin) {
                    const unsigned long long target = a.cell_base + (unsigned long long)(k - 1) * M + n + 1;
                    const unsigned long long t0 = lane == 0 ? global_ns() : 0ull;
                    int nbr = p_lo + lane <= p_hi ? p_lo + lane : (lane == 31 && p_lo > 0 ? 0 : -1);
                    if (nbr >= p_cnt) nbr = -1;
                    if (nbr >= 0) {
                        long long spins = 0;
                        while (ld_acquire_u64(&pred_prog[nbr]) < target) {
                            if ((a.stop && ld_acquire_s32(a.stop)) || ld_acquire_s32(a.abort_flag)) {
                                stop_seen = true;
                                break;
                            }
                            if (++spins > a.wait_budget) {
                                team_fail(c, ST_ETIMEOUT);
                                stop_seen = true;
                                break;
                            }
                            if (spins > 4096) __nanosleep(64);
                        }
                        __threadfence();
                    }
                    stop_seen = __any_sync(0xffffffffu, stop_seen);
                    if (lane == 0) t_pred += global_ns() - t0;
                }
                if (lane == 0)
                    s_ok = (stop_seen || (a.stop && ld_acquire_s32(a.stop)) || ld_acquire_s32(a.abort_flag)) ? 1 : 0;
            }
            __syncthreads();
            const int stop_local = s_ok;
            // every later cell is a skip once the stop flag is up (or the launch aborts)
            if (stop_local) goto done;
            if (threadIdx.x == 0) t_mark = global_ns();
            // 2. the previous iteration's running max (lane pl: it acquired CTA 0's progress), and
            //    in the same round trip u^{n-1}_k when the previous level was skipped (the global,
            //    final iterate) and u^n_k (below)
            if (threadIdx.x == pl) {
                slot[0] = k > a.k_begin ? ldcg(prefixg + ((long long)(k - 1) * M + n)) : 1.0 / 0.0;
                // the first iteration's running residual at this level (finished long before)
                slot[1] = k > 0 ? ldcg(prefixg + n) : 1.0 / 0.0;
            }
            const bool reload_prev = !uprev_valid;
            if (reload_prev) {
                const auto up = n == 0 ? u0g + off0 : Ug + ((long long)(n - 1) * Ns + off0);
                for (int i = threadIdx.x; i < nloc; i += NT) uprev[i] = ldcg(up + i);
                uprev_valid = true;
            }
            // u^n_k: own rows and one halo row each side (Dirichlet data off the domain)
            const auto Un = Ug + (long long)n * Ns;
            const auto bnd = a.bc ? bcg + (long long)n * nb : bcg;
            // maxima as integer keys (abs_key), so the bookkeeping stays off the FP64 pipe
            unsigned long long krmax = 0, krs = 0, kbmax = 0;
            bool ns = false;
            {
                if (a.bulk_u) {
                    // the strip's rows inside the domain are contiguous in U: one bulk copy
                    // (TMA) issued by thread 0 -- every thread finished with this shared memory
                    // at the barrier above; the rows off the domain take the Dirichlet data
                    const int j0 = t.r0 > 0 ? t.r0 - 1 : 0;
                    const int j1 = t.r0 + t.nrows < ny ? t.r0 + t.nrows : ny - 1;
                    if (threadIdx.x == 0) {
                        const unsigned bytes = (unsigned)((size_t)(j1 - j0 + 1) * nx * sizeof(double));
                        const auto dst = u + (long long)(j0 - (t.r0 - 1)) * nx;
                        const auto src = Un + (long long)j0 * nx;
                        bool issue = true;
#ifdef PIT_CHECK_BOUNDS
                        // the copy's ranges and alignment; a bad copy is not issued (the phase
                        // then completes on the arrival alone)
                        issue = dst.lo <= 0 && (long long)(j1 - j0 + 1) * nx <= dst.hi && src.lo <= 0 &&
                                (long long)(j1 - j0 + 1) * nx <= src.hi && (bytes & 15u) == 0 &&
                                ((size_t)static_cast<double*>(dst) & 15) == 0 &&
                                ((size_t)static_cast<const double*>(src) & 15) == 0;
                        if (!issue) bounds_fail(kChkBulk);
#endif
                        fence_proxy_async_smem();
                        mbar_arrive_expect_tx(ubar, issue ? bytes : 0u);
                        if (issue) bulk_copy_g2s(dst, src, bytes, ubar);
                    }
                    if (t.r0 == 0)
                        for (int i = threadIdx.x; i < nx; i += NT) u[i] = bnd ? bnd[i] : 0.0;
                    if (t.r0 + t.nrows == ny)
                        for (int i = threadIdx.x; i < nx; i += NT) u[(size_t)(t.nrows + 1) * nx + i] = bnd ? bnd[nx + i] : 0.0;
                    int landed = 1;
                    if (threadIdx.x == 0) {
                        landed = mbar_wait_parity(ubar, bb.phase, kBulkWaitPolls) ? 1 : 0;
                        if (!landed) {
                            // give up: raise the abort, and let the copy land before leaving
                            team_fail(c, ST_ETIMEOUT);
                            mbar_wait_parity(ubar, bb.phase, kBulkWaitPolls);
                        }
                    }
                    bb.phase ^= 1u;
                    if (!__syncthreads_and(landed)) return;
                } else {
#pragma unroll 4
                    for (int i = threadIdx.x; i < (t.nrows + 2) * nx; i += NT) {
                        const int jr = i / nx, ii = i - jr * nx, j = t.r0 - 1 + jr;
                        double val;
                        if (j < 0) val = bnd ? bnd[ii] : 0.0;
                        else if (j >= ny) val = bnd ? bnd[nx + ii] : 0.0;
                        else val = ldcg(Un + ((long long)j * nx + ii));
                        u[i] = val;
                    }
                    __syncthreads();
                }
                if (threadIdx.x == 0) t_load += global_ns() - t_mark;
                const double pred_prefix = slot[0];
                first_res = slot[1];
                if (pred_prefix <= a.tol_res) {
                    // levels 0..n converged in iteration k - 1: du^n_k = 0, nothing to solve
                    __syncthreads();  // slot[0] read by every thread
                    for (int i = threadIdx.x; i < nloc; i += NT) m.x[i] = T(0);
                    uprev_valid = false;
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        prefix = pred_prefix;
                        __threadfence();
                        if (b == 0) {
                            stcg(prefixg + ((long long)k * M + n), prefix);
                            if (a.cell_iters) itersg[(long long)k * M + n] = 1;
                            __threadfence();
                        }
                        st_release_u64(&my_prog[b], a.cell_base + (unsigned long long)k * M + n + 1);
                    }
                    continue;
                }
                // 3. residual r^n_k, scaled couplings, rhs; uprev <- u^n_k
                const auto qn = a.q ? qg + ((long long)n * Ns + off0) : qg;
                float gmax_f = 0.0f;  // FP32 solves: largest FP32 row sum of this thread's rows
                struct NodeIn {
                    double uC, uW, uE, uS, uN, up, x, q;
                };
                struct NodeOut {
                    double r, bval, d;
                    T aW, aE, aS, aN;  // Jacobi-scaled couplings, in the level-solve precision
                };
                auto load_node = [&](int i, int jl, int ii) {
                    const int j = t.r0 + jl;
                    const int ku = (jl + 1) * nx + ii;
                    NodeIn v;
                    v.uC = u[ku];
                    v.uW = ii > 0 ? u[ku - 1] : (bnd ? bnd[2 * nx + j] : 0.0);
                    v.uE = ii < nx - 1 ? u[ku + 1] : (bnd ? bnd[2 * nx + ny + j] : 0.0);
                    v.uS = u[ku - nx];
                    v.uN = u[ku + nx];
                    v.up = uprev[i];
                    v.x = (double)m.x[i];
                    v.q = qn ? qn[i] : 0.0;
                    return v;
                };
                auto form_node = [&](int jl, int ii, const NodeIn& v) {
                    const int j = t.r0 + jl;
                    NodeOut o;
                    if (CONV && !NLV) {
                        // Burgers with constant viscosity: eq. 3-5 and the Jacobian with the
                        // constants folded (the diagonal 1/d is constant). With mu tau/h^2 = vmu:
                        //   r = u^{n-1} - kcen uC - uE (cx uE - vmu_x) + uW (cx uW + vmu_x)
                        //                         - uN (cy uN - vmu_y) + uS (cy uS + vmu_y),
                        // kcen = 1 + 2 (vmu_x + vmu_y): nine FP64 operations
                        double r = fma(-kcen, v.uC, v.up);
                        r = fma(-v.uE, fma(oc.cx, v.uE, -vmu_x), r);
                        r = fma(v.uW, fma(oc.cx, v.uW, vmu_x), r);
                        r = fma(-v.uN, fma(oc.cy, v.uN, -vmu_y), r);
                        o.r = fma(v.uS, fma(oc.cy, v.uS, vmu_y), r);
                        o.d = dconst;
                        if constexpr (sizeof(T) == 4) {
                            // FP32 level solves: the couplings are formed in FP32 from u in
                            // FP32 (they are stored in FP32 anyway); only r and the rhs are FP64
                            o.aE = fmaf(sjx_t, (float)v.uE, -svx_t);
                            o.aW = fmaf(-sjx_t, (float)v.uW, -svx_t);
                            o.aN = fmaf(sjy_t, (float)v.uN, -svy_t);
                            o.aS = fmaf(-sjy_t, (float)v.uS, -svy_t);
                        } else {
                            o.aE = fma(sjx, v.uE, -svx);
                            o.aW = fma(-sjx, v.uW, -svx);
                            o.aN = fma(sjy, v.uN, -svy);
                            o.aS = fma(-sjy, v.uS, -svy);
                        }
                    } else {
                        o.r = (v.up - v.uC) - tau_F<CONV, NLV>(oc, v.uC, v.uW, v.uE, v.uS, v.uN);
                        double aC, aW, aE, aS, aN;
                        jac_row<CONV, NLV>(oc, v.uC, v.uW, v.uE, v.uS, v.uN, aC, aW, aE, aS, aN);
                        o.d = NLV ? 1.0 / aC : dconst;
                        o.aW = (T)(aW * o.d);
                        o.aE = (T)(aE * o.d);
                        o.aS = (T)(aS * o.d);
                        o.aN = (T)(aN * o.d);
                    }
                    if (qn) o.r = fma(oc.dt, v.q, o.r);
                    if (ii == 0) o.aW = T(0);
                    if (ii == nx - 1) o.aE = T(0);
                    if (j == 0) o.aS = T(0);
                    if (j == ny - 1) o.aN = T(0);
                    o.bval = o.r + v.x;  // r^n + du^{n-1}
                    return o;
                };
                auto store_node = [&](int i, const NodeIn& v, const NodeOut& o) {
                    m.cw[i] = o.aW;
                    m.ce[i] = o.aE;
                    m.cs[i] = o.aS;
                    m.cn[i] = o.aN;
                    const T xt = (T)o.bval;
                    if constexpr (sizeof(T) == 4 && CONV && !NLV) m.bs[i] = xt * dconst_t;  // FP32 product
                    else m.bs[i] = (T)(o.d * o.bval);
                    m.x[i] = xt;      // SOR start
                    uprev[i] = v.uC;  // u^n_k for the next level's time difference
                    const unsigned long long kr = abs_key(o.r), kb = abs_key(o.bval);
                    krmax = kr > krmax ? kr : krmax;
                    kbmax = kb > kbmax ? kb : kbmax;
                    // Gershgorin row sum of the couplings as stored (FP32 sums for FP32 solves;
                    // biased upward once per thread below so it stays an upper bound)
                    if constexpr (sizeof(T) == 4) {
                        gmax_f = fmaxf(gmax_f, fabsf(o.aW) + fabsf(o.aE) + fabsf(o.aS) + fabsf(o.aN));
                    } else {
                        const unsigned long long kg = abs_key(fabs(o.aW) + fabs(o.aE) + fabs(o.aS) + fabs(o.aN));
                        krs = kg > krs ? kg : krs;
                    }
                    ns |= opposite_nonzero(o.aW, o.aE) || opposite_nonzero(o.aS, o.aN);
                };
                // node i = (local row jl, column ii), stepped by NT without a division per node
                int jl = (int)threadIdx.x / nx, ii = (int)threadIdx.x - jl * nx;
                const int djl = NT / nx, dii = NT - djl * nx;
                const long long s0 = clock64();
#pragma unroll 2
                for (int i = threadIdx.x; i < nloc; i += NT) {
                    const NodeIn v = load_node(i, jl, ii);
                    store_node(i, v, form_node(jl, ii, v));
                    ii += dii;
                    jl += djl;
                    if (ii >= nx) {
                        ii -= nx;
                        ++jl;
                    }
                }
                // four FP32 magnitudes summed in FP32 err by at most 3 units in 2^-24 of the sum:
                // the bias 2^-20 keeps the bound above the exact sum of the stored couplings
                // (a NaN in u shows in max |r|, which ends the window before any solve)
                if constexpr (sizeof(T) == 4) krs = abs_key((double)gmax_f * (1.0 + 0x1p-20));
                if (threadIdx.x == 0) scyc[0] += clock64() - s0;
            }
            // 4. team reduction: max |r|, Gershgorin bound, 2 stop + nonsymmetric-row flag, max |rhs|
            //    (every CTA of the team takes the same decisions from these)
            const int flags_local = (stop_local ? 2 : 0) + (ns ? 1 : 0);
            double v3[4];
            const long long s1 = clock64();
            {
                unsigned long long kk[4] = {krmax, krs, abs_key((double)flags_local), kbmax};
                block_max4_to0<NT>(kk, reinterpret_cast<unsigned long long*>(m.red));
                for (int q = 0; q < 4; ++q) v3[q] = key_val(kk[q]);  // meaningful on thread 0 only
            }
            const long long s2 = clock64();
            // deep rows: the neighbours' boundary rows of the level system travel while the
            // team reduction does (publish now, fetch after it)
            unsigned long long cseq = 0;
            const unsigned long long t_sr0 = threadIdx.x == 0 ? global_ns() : 0ull;
            if (deep) {
                const int last = (t.nrows - 1) * nx;
                const sptr<const T> lo[5] = {m.cw, m.ce, m.cs, m.cn, m.bs};
                const sptr<const T> hi[5] = {m.cw + last, m.ce + last, m.cs + last, m.cn + last, m.bs + last};
                cseq = publish_rows_tagged<NT, T, 5>(t, deep->tpub, lo, hi);
            }
            const long long s3 = clock64();
            double g3[4];
            if (deep) {
                const unsigned long long use = t.tag_seq++;
                if (threadIdx.x == 0) tagged_arrive<4>(t, deep->tred, use, v3);
                if (threadIdx.x < 32) {
                    const unsigned long long t0 = threadIdx.x == 0 ? global_ns() : 0ull;
                    const bool okr = tagged_finish<4, true>(c, t, deep->tred, use, g3);
                    if (threadIdx.x == 0) {
                        t.t_red += global_ns() - t0;
                        for (int q = 0; q < 4; ++q) m.red[32 + q] = g3[q];
                        if (!okr && !ld_acquire_s32(c.abort_flag)) team_fail(c, ST_ETIMEOUT);
                        s_ok = okr ? 1 : 0;
                    }
                }
                __syncthreads();
                for (int q = 0; q < 4; ++q) g3[q] = m.red[32 + q];
                const bool okr = s_ok != 0;
                __syncthreads();
                if (!okr) return;
            } else if (!reduce_finish<4, true>(c, t, reduce_arrive<4>(t, v3), g3, m.red + 32, &s_ok)) {
                return;
            }
            const long long s4 = clock64();
            if (g3[2] >= 2.0) goto done;  // another iteration has converged (or the launch aborts)
            if (!(g3[0] < kDiverged) || g3[0] > kGrowth * fmax(first_res, a.tol_res)) {
                // NaN/Inf or a runaway residual: Newton diverges on this range of levels. One
                // team (a batch problem) ends its window and lets the caller retry a shorter
                // one; several teams end the launch with PIT_EDIVERGED.
                if (threadIdx.x == 0) {
                    if (a.K == 1) {
                        if (b == 0 && a.kconv) *a.kconv = -2;
                    } else if (a.kconv) {
                        // several teams on one problem of a batch, whose abort word is the
                        // job's own: mark the window diverged and end it for every team
                        // (every wait watches that word); the batch retries a shorter window
                        *a.kconv = -2;
                        __threadfence();
                        atomicExch(a.abort_flag, 1);
                    } else {
                        team_fail(c, ST_EDIVERGED);
                    }
                }
                goto done;
            }
            if (deep) {
                const sptr<T> fS[5] = {deep->cS[0], deep->cS[1], deep->cS[2], deep->cS[3], deep->cS[4]};
                const sptr<T> fN[5] = {deep->cN[0], deep->cN[1], deep->cN[2], deep->cN[3], deep->cN[4]};
                if (!fetch_rows_tagged<NT, T, 5>(c, t, deep->tpub, cseq, fS, fN)) return;
            }
            if (threadIdx.x == 0) {
                scyc[1] += s2 - s1;
                scyc[2] += s3 - s2;
                scyc[3] += s4 - s3;
                scyc[4] += clock64() - s4;
            }
            if (threadIdx.x == 0) t_sred += global_ns() - t_sr0;
            {
                // 5. forcing from the running max; SOR tolerance absolute (as tol / omega, see
                //    level_sor_deep), BiCGStab relative; method and omega from the level's bound.
                //    Thread 0 forms them all, one barrier broadcasts them.
                const bool use_sor = a.method == 1 || (a.method == 0 && g3[1] < a.sor_rho_max);
                double* sc = m.red + 36;
                if (threadIdx.x == 0) {
                    prefix = fmax(prefix, g3[0]);
                    const double eta = fmax(fmin(a.eta_max, a.eta_gamma * prefix), 1e-300);
                    // absolute, not below the level-solve precision's round-off of the rhs
                    const double sor_tol = fmax(fmax(a.atol, eta * prefix), 16.0 * Eps<T>::value * g3[3]);
                    const double omega = use_sor ? sor_omega(g3[1], g3[2] != 0.0) : 1.0;
                    sc[0] = eta;
                    sc[1] = omega;
                    sc[2] = sor_tol / omega;
                    const unsigned long long now = global_ns();
                    t_setup += now - t_mark;
                    t_mark = now;
                }
                __syncthreads();
                const double eta = sc[0], omega = sc[1], sor_tol_w = sc[2];
                const int used = use_sor ? 1 : 2;
                const int iters =
                    level_solve_decided<NT, T>(c, t, m, use_sor, omega, sor_tol_w, eta, a.atol, &s_ok, deep);
                if (iters < 0) return;  // aborted
                if (threadIdx.x == 0) {
                    const unsigned long long now = global_ns();
                    t_solve += now - t_mark;
                    t_mark = now;
                    n_cells += 1;
                    n_sweeps += (unsigned long long)(iters > 0 ? iters : 0);
                }
                // 6. U^n += du^n; du^n stays in x for the next level
                const auto Uw = Ug + ((long long)n * Ns + off0);
                for (int i = threadIdx.x; i < nloc; i += NT) {
                    const T xt = m.x[i];
                    const double dx = (double)xt;
                    stcg(Uw + i, uprev[i] + dx);
                    // the update norm is a statistic: with FP32 level solves it is summed in
                    // FP32, which leaves the scarce FP64 pipe to the arithmetic of the method
                    if constexpr (sizeof(T) == 4) sumsq_f = fmaf(xt, xt, sumsq_f);
                    else sumsq += dx * dx;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    if (b == 0) {
                        stcg(prefixg + ((long long)k * M + n), prefix);
                        if (a.cell_iters) itersg[(long long)k * M + n] = used == 1 ? iters + 1 : -(iters + 1);
                    }
                    __threadfence();
                    st_release_u64(&my_prog[b], a.cell_base + (unsigned long long)k * M + n + 1);
                    if (iters >= c.max_iter) atomicCAS(a.status, 0, ST_ENOCONV);
                    t_upd += global_ns() - t_mark;
                }
            }
        }
        {
            // iteration k done on every level
            double ss[1] = {sumsq + (double)sumsq_f};
            sumsq_f = 0.0f;
            block_sum<NT, 1>(ss, m.red);
            if (threadIdx.x == 0) {
                if (a.cta_sumsq) chk(a.cta_sumsq, (long long)a.k_end * a.G, kChkSumsq)[(long long)k * a.G + b] = ss[0];
                if (b == 0) {
                    if (a.res_inf) chk(a.res_inf, a.k_end, kChkLevel)[k] = prefix;
                    if (prefix <= a.tol_res && a.K > 1 && a.stop) {
                        atomicMin(a.stop + 1, k);
                        __threadfence();
                        atomicExch(a.stop, 1);
                    }
                }
            }
            // one team: every CTA holds the same running max and leaves by itself
            const double fin = bcast0(prefix, slot);
            if (a.K == 1 && fin <= a.tol_res) {
                if (threadIdx.x == 0 && b == 0 && a.kconv) *a.kconv = k;
                goto done;
            }
        }
    }
done:
    if (b == 0 && threadIdx.x == 0 && a.timers) {
        unsigned long long* tm = a.timers + (size_t)team * kWaveTimers;
        tm[0] = t.t_halo;
        tm[1] = t.t_red;
        tm[2] = t_pred;
        tm[3] = global_ns() - t_start;
        tm[4] = t_setup;
        tm[5] = t_solve;
        tm[6] = t_upd;
        tm[7] = t_load;
        tm[8] = t_sred;
        tm[9] = n_cells;
        tm[10] = n_sweeps;
        const unsigned long long* cyc = reinterpret_cast<const unsigned long long*>(m.red + 56);
        for (int q = 0; q < 8; ++q) tm[12 + q] = cyc[q];
        const unsigned long long* sc5 = reinterpret_cast<const unsigned long long*>(m.red + 50);
        for (int q = 0; q < 5; ++q) tm[20 + q] = sc5[q];
    }
    __syncthreads();
}

template <int NT, bool CONV, bool NLV, typename T = double>
__global__ void __launch_bounds__(NT) wave_kernel(WaveArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_ok;
    int team = blockIdx.x / a.G, b = blockIdx.x - team * a.G, G = a.G, rb = a.rows_base, rr = a.rows_rem;
    if (a.tgeom) {  // teams of their own sizes, in block order
        team = 0;
        while (team + 1 < a.K && (int)blockIdx.x >= a.tgeom[4 * (team + 1)]) ++team;
        b = blockIdx.x - a.tgeom[4 * team];
        G = a.tgeom[4 * team + 1];
        rb = a.tgeom[4 * team + 2];
        rr = a.tgeom[4 * team + 3];
    }
    Team t;
    team_init(t, b, G, a.c.nx, a.c.ny, rb, rr, a.pub + (size_t)team * 2 * a.G * 2 * a.c.nx,
              a.flags + (size_t)team * a.G, a.red_part + (size_t)team * 4 * a.G * 4, a.red_cnt + (size_t)team * 4);
    __shared__ __align__(8) unsigned long long s_ubar;
    if (threadIdx.x == 0) mbar_init(&s_ubar, 1);
    __syncthreads();
    BulkBar bb{&s_ubar, 0u};
    wave_body<NT, CONV, NLV, T>(a, team, b, t, smem, s_ok, bb);
}

// ------------------------------------------------ batched instances (one launch)

// One problem of a batch and its results.
struct BatchInstance {
    OpConst c;                          // grid, all M levels, dt, closure
    int conv, nlv;                      // closure: Burgers convection, u-dependent viscosity
    int window;                         // levels per window
    int bulk_u;                         // level strips by bulk copy (nx even, U 16-byte aligned)
    const double* u0;
    const double* bc;
    const double* q;
    double* U;                          // [M][Ns] solution (the plain guess is filled in here)
    double* res_inf;                    // out: ||R||_inf of the final U
    int* newton_iters;                  // out: Newton updates summed over windows
    int* converged_windows;             // out
};

// Job of one CTA: CTA `rank` of team `tk` of K teams of G CTAs on instance `inst`
// (K = 1: one team runs the Newton iterations of a window one after another; K > 1:
// a wavefront job, team tk runs iterations tk, tk + K, ... with several in flight).
// Jobs are listed per CTA in one global order, so the lowest unfinished job always
// has all of its CTAs (no cyclic waits). The job's workspace is given by offsets
// into the pools.
struct BatchJob {
    int inst, rank, G;                  // G: CTAs of this CTA's team
    int team;                           // index of the job's workspace
    int K, tk;
    int first;                          // the team's first CTA among the job's CTAs
    int jctas;                          // CTAs of the job (sum of its teams' sizes)
    int Gs;                             // the largest team's size: stride of the team workspaces
};

struct BatchTeamWs {
    double* pub;                        // [K][2][G][2][nx]
    unsigned long long* flags;          // [K][G]
    double* red_part;                   // [K][4][G][4]
    unsigned long long* red_cnt;        // [K][4]
    unsigned long long* prog;           // [K][G]
    double* cell_prefix;                // [newton_max][window]
    int* kconv;                         // K = 1: converged iteration of the current window (CTA 0 only);
                                        // K > 1: -2 when the window diverged
    int* stop;                          // K > 1: [0] stop flag, [1] first converged iteration
    int* jabort;                        // K > 1: the job's abort word (a diverged window, or a wait that gave up)
    int* jstatus;                       // the job's status word: a level solve that breaks down or produces
                                        // NaN ends its window (retried shorter), not the launch
    unsigned long long* jbar;           // K > 1: arrivals at the job-wide barrier
    unsigned long long* jres;           // K > 1: final ||R||_inf as an order-preserving key (max over teams)
    unsigned long long* tpub;           // [K][2][G][kDeepSlotRows][nx][2] tagged words (zeroed per launch)
    unsigned long long* tred;           // [K][4][G][kTagRedWords] tagged reduction words (zeroed per launch)
    unsigned long long* sync_words;     // flags, prog, red_cnt and the tagged words: zeroed again after a
    size_t sync_count;                  // window that ended on the job's abort word
    const int* tgeom;                   // K > 1: [K][4] teams of different sizes (WaveArgs::tgeom), or null
};

struct BatchArgs {
    const BatchInstance* inst;
    const BatchJob* jobs;               // jobs of CTA c: jobs[job_off[c] .. job_off[c+1])
    const int* job_off;
    const BatchTeamWs* ws;
    int* abort_flag;
    int* status;
    int newton_max;
    double tol_res, eta_max, eta_gamma, atol, sor_rho_max;
    int method, max_iter;
    long long wait_budget;
    int start_given;                    // windows start from the iterate already in U (else the plain guess)
};

// A team-wide barrier built on the team reduction (every CTA of the team passes it
// only after all have arrived).
template <int NT>
__device__ __forceinline__ bool team_barrier(const TeamCtl& c, Team& t, double* red, int* s_ok) {
    double v[1] = {0.0};
    return reduce_finish<1, true>(c, t, reduce_arrive<1>(t, v), v, red + 32, s_ok);
}

// Barrier over all CTAs of a wavefront job: arrival count `target` = (barriers
// passed so far + 1) x CTAs of the job. The fences order each CTA's earlier writes
// before its arrival and the others' writes before its departure.
__device__ __forceinline__ bool job_barrier(const TeamCtl& c, unsigned long long* cnt, unsigned long long target,
                                            int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(cnt, 1ull);
        *s_ok = wait_geq(c, cnt, target) ? 1 : 0;
        __threadfence();
    }
    __syncthreads();
    return *s_ok != 0;
}

// Closures of a batched launch as a set: bit (2 conv + nlv). A batched kernel is compiled
// for one set and holds only those closures' wave bodies: holding all four made every
// job's code measurably slower than the dedicated wavefront kernel's (a heat problem:
// 99.6 ms with all four, 81.3 ms with its own only, 78.0 ms in the wavefront kernel).
__host__ __device__ constexpr int closure_bit(bool conv, bool nlv) { return 1 << ((conv ? 2 : 0) + (nlv ? 1 : 0)); }
constexpr int kBatchThreads = 256;  // threads per CTA of every batched kernel

template <int NT, int CLOSURES, typename T>
__device__ __forceinline__ void wave_body_of(const WaveArgs& a, int bit, int team, int b, Team& t, unsigned char* smem,
                                             int& s_ok, BulkBar& bb) {
    if constexpr ((CLOSURES & closure_bit(true, true)) != 0)
        if (bit == closure_bit(true, true)) return wave_body<NT, true, true, T>(a, team, b, t, smem, s_ok, bb);
    if constexpr ((CLOSURES & closure_bit(true, false)) != 0)
        if (bit == closure_bit(true, false)) return wave_body<NT, true, false, T>(a, team, b, t, smem, s_ok, bb);
    if constexpr ((CLOSURES & closure_bit(false, true)) != 0)
        if (bit == closure_bit(false, true)) return wave_body<NT, false, true, T>(a, team, b, t, smem, s_ok, bb);
    if constexpr ((CLOSURES & closure_bit(false, false)) != 0)
        if (bit == closure_bit(false, false)) return wave_body<NT, false, false, T>(a, team, b, t, smem, s_ok, bb);
}

template <int NT, int CLOSURES, typename T>
__device__ void batch_instance(const BatchArgs& ba, const BatchJob& job, unsigned char* smem, int& s_ok, BulkBar& bb) {
    const BatchInstance& in = ba.inst[job.inst];
    const BatchTeamWs& ws = ba.ws[job.team];
    const OpConst& oc = in.c;
    const int nx = oc.nx, ny = oc.ny, M = oc.M;
    const int G = job.G, b = job.rank, K = job.K, tk = job.tk, Gs = job.Gs;
    const int rows_base = ny / G, rows_rem = ny % G;
    TeamCtl c{ba.abort_flag, ba.status, ba.wait_budget, ba.max_iter};
    Team t;
    team_init(t, b, G, nx, ny, rows_base, rows_rem, ws.pub + (size_t)tk * 2 * Gs * 2 * nx, ws.flags + (size_t)tk * Gs,
              ws.red_part + (size_t)tk * 4 * Gs * 4, ws.red_cnt + (size_t)tk * 4);
    const long long Ns = t.Ns;
    const long long off0 = (long long)t.r0 * nx;
    const int nloc = t.nloc;
    const int cap = (rows_base + (rows_rem ? 1 : 0)) * nx;
    double* red = smem_layout<T>(smem, cap, nx).red;
    const int W = in.window > 0 ? in.window : M;
    const int nb = 2 * nx + 2 * ny;
    const auto Ug = chk(in.U, (long long)M * Ns, kChkU);
    const auto u0g = chk(in.u0, Ns, kChkU0);
    const auto bcg = chk(in.bc, (long long)M * nb, kChkBc);
    const auto qg = chk(in.q, (long long)M * Ns, kChkQ);
    const bool lead = tk == 0 && b == 0;          // reports the results
    const unsigned long long job_ctas = (unsigned long long)job.jctas;
    unsigned long long jep = 0;                   // job-wide barriers passed (K > 1)
    unsigned long long base = 0;
    int iters_total = 0, conv_windows = 0;
    __shared__ int s_kdone;
    // Windows adapt: a window whose Newton diverges or does not converge is halved and
    // restarted from the plain guess at its first level; after a success the window
    // length grows back toward W.
    int w = W;
    int clean_from = 0;                           // levels >= clean_from still hold the caller's iterate
    for (int s = 0; s < M;) {
        const int Mw = min(w, M - s);
        const auto from = s == 0 ? u0g : Ug + (long long)(s - 1) * Ns;
        // the same decision on every CTA of the job (s and clean_from are job-wide)
        if (!(ba.start_given && s >= clean_from)) {
            // plain guess for the window from its previous level: own rows only, levels
            // tk, tk + K, ... by team tk
            for (int n = tk; n < Mw; n += K) {
                const auto dst = Ug + ((long long)(s + n) * Ns + off0);
                for (int i = threadIdx.x; i < nloc; i += NT) dst[i] = ldcg(from + (off0 + i));
            }
        }
        if (threadIdx.x == 0 && lead) {
            if (K > 1) {
                ws.stop[0] = 0;
                ws.stop[1] = 0x7fffffff;
                *ws.jabort = 0;
            }
            *ws.kconv = -1;
            *ws.jstatus = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) __threadfence();
        if (K == 1) {
            if (!team_barrier<NT>(c, t, red, &s_ok)) return;  // neighbours' rows are filled
        } else if (!job_barrier(c, ws.jbar, job_ctas * ++jep, &s_ok)) {
            return;
        }
        WaveArgs a{};
        a.c = oc;
        a.c.M = Mw;
        a.u0 = from;
        a.bc = in.bc ? in.bc + (long long)s * (2 * nx + 2 * ny) : nullptr;
        a.q = in.q ? in.q + (long long)s * Ns : nullptr;
        a.U = in.U + (long long)s * Ns;
        a.K = K;
        a.G = Gs;
        a.rows_base = rows_base;  // this team's strips: the shared-memory layout above
        a.rows_rem = rows_rem;
        a.tgeom = K > 1 ? ws.tgeom : nullptr;
        a.k_begin = 0;
        a.k_end = ba.newton_max;
        a.bulk_u = in.bulk_u;
        a.cell_base = base;
        a.tol_res = ba.tol_res;
        a.eta_max = ba.eta_max;
        a.eta_gamma = ba.eta_gamma;
        a.atol = ba.atol;
        a.sor_rho_max = ba.sor_rho_max;
        a.method = ba.method;
        a.max_iter = ba.max_iter;
        a.wait_budget = ba.wait_budget;
        a.pub = ws.pub;
        // one-exchange sweeps and tagged reductions for wide teams; small teams (thick
        // strips, little halo traffic) measured faster with the flag protocol
        a.tpub = G >= 8 ? ws.tpub : nullptr;
        a.tred = G >= 8 ? ws.tred : nullptr;
        a.flags = ws.flags;
        a.red_part = ws.red_part;
        a.red_cnt = ws.red_cnt;
        a.prog = ws.prog;
        // several teams: the job's own abort word, so that a diverged window ends every
        // team's waits without ending the launch
        a.abort_flag = K > 1 ? ws.jabort : ba.abort_flag;
        a.status = ws.jstatus;
        a.stop = K > 1 ? ws.stop : nullptr;
        a.res_inf = nullptr;
        a.cell_prefix = ws.cell_prefix;
        a.cell_iters = nullptr;
        a.cta_sumsq = nullptr;
        a.timers = nullptr;
        // K = 1: CTA 0 writes the converged iteration (or -1 / -2 for not converged /
        // diverged); K > 1: any CTA marks a diverged window, the stop words give the
        // first converged iteration
        a.kconv = (K > 1 || b == 0) ? ws.kconv : nullptr;
        // the host launches a kernel whose set holds every problem's closure
        wave_body_of<NT, CLOSURES, T>(a, closure_bit(in.conv != 0, in.nlv != 0), tk, b, t, smem, s_ok, bb);
        if (threadIdx.x == 0) {
            // a wait that gave up is the launch's failure; other codes are the window's
            if (ld_acquire_s32(ws.jstatus) == ST_ETIMEOUT) atomicCAS(ba.status, 0, ST_ETIMEOUT);
            s_ok = ld_acquire_s32(ba.abort_flag);
            s_kdone = b == 0 ? *ws.kconv : 0;
        }
        __syncthreads();
        if (s_ok) return;  // the launch aborts (read once per CTA)
        int kdone;
        if (K == 1) {
            // the decision must be the same on every CTA: CTA 0's result, shared by max
            double kv[1] = {b == 0 ? (double)(s_kdone + 3) : 0.0};
            double kg[1];
            if (!reduce_finish<1, true>(c, t, reduce_arrive<1>(t, kv), kg, red + 32, &s_ok)) return;
            kdone = (int)kg[0] - 3;
        } else {
            // every team has left the window: the flags are final; read them, then let
            // the lead CTA reset them only after everyone has read
            if (!job_barrier(c, ws.jbar, job_ctas * ++jep, &s_ok)) return;
            if (threadIdx.x == 0) {
                const int kc = ld_acquire_s32(ws.kconv);
                const int st = ld_acquire_s32(ws.stop);
                const int k1 = ld_acquire_s32(ws.stop + 1);
                const int ja = ld_acquire_s32(ws.jabort);
                // the job's abort word without a diverged window: a wait gave up (fatal)
                s_kdone = ja ? (kc == -2 ? -2 : -3) : (kc == -2 ? -2 : (st != 0 && k1 != 0x7fffffff ? k1 : -1));
                s_ok = ja;
            }
            __syncthreads();
            kdone = s_kdone;
            const bool reset = s_ok != 0;
            __syncthreads();
            if (kdone == -3) {
                if (threadIdx.x == 0 && lead) team_fail(c, ST_ETIMEOUT);
                return;
            }
            if (reset) {
                // the teams left the window at different points: restart the job's
                // synchronisation from a clean state (zeroed words, fresh counters)
                const size_t per = (ws.sync_count + job_ctas - 1) / job_ctas;
                const size_t r = (size_t)job.first + b;
                const size_t lo = r * per, hi = lo + per < ws.sync_count ? lo + per : ws.sync_count;
                for (size_t i = lo + threadIdx.x; i < hi; i += NT) ws.sync_words[i] = 0ull;
            }
            if (!job_barrier(c, ws.jbar, job_ctas * ++jep, &s_ok)) return;
            if (reset)
                team_init(t, b, G, nx, ny, rows_base, rows_rem, ws.pub + (size_t)tk * 2 * Gs * 2 * nx,
                          ws.flags + (size_t)tk * Gs, ws.red_part + (size_t)tk * 4 * Gs * 4, ws.red_cnt + (size_t)tk * 4);
        }
        base += (unsigned long long)ba.newton_max * Mw + 1;
        if (kdone < 0) clean_from = max(clean_from, s + Mw);  // the failed attempt overwrote these levels
        if (kdone >= 0) {
            iters_total += kdone + 1;
            ++conv_windows;
            s += Mw;
            w = min(W, 2 * w);
        } else {
            iters_total += ba.newton_max;
            if (Mw > 1) {
                w = max(1, Mw / 2);  // retry the same first level with a shorter window
            } else {
                s += 1;              // a single level that does not converge: go on
                w = 1;
            }
        }
        __syncthreads();
    }
    // final residual of the whole solution, all levels (needs the neighbours' last
    // updates; with several teams every team's updates): team tk takes the levels
    // tk, tk + K, ...
    if (threadIdx.x == 0) __threadfence();
    if (K > 1) {
        if (!job_barrier(c, ws.jbar, job_ctas * ++jep, &s_ok)) return;
    } else if (!team_barrier<NT>(c, t, red, &s_ok)) {
        return;
    }
    double rmax = 0.0;
    for (int n = tk; n < M; n += K) {
        const auto Un = Ug + (long long)n * Ns;
        const auto Up = n == 0 ? u0g : Ug + (long long)(n - 1) * Ns;
        const auto bnd = in.bc ? bcg + (long long)n * nb : bcg;
        for (int i = threadIdx.x; i < nloc; i += NT) {
            const int jl = i / nx, ii = i - jl * nx, j = t.r0 + jl;
            const long long k = (long long)j * nx + ii;
            const double uC = ldcg(Un + k);
            const double uW = ii > 0 ? ldcg(Un + (k - 1)) : (bnd ? bnd[2 * nx + j] : 0.0);
            const double uE = ii < nx - 1 ? ldcg(Un + (k + 1)) : (bnd ? bnd[2 * nx + ny + j] : 0.0);
            const double uS = j > 0 ? ldcg(Un + (k - nx)) : (bnd ? bnd[ii] : 0.0);
            const double uN = j < ny - 1 ? ldcg(Un + (k + nx)) : (bnd ? bnd[nx + ii] : 0.0);
            double tf;
            if (in.conv) tf = in.nlv ? tau_F<true, true>(oc, uC, uW, uE, uS, uN) : tau_F<true, false>(oc, uC, uW, uE, uS, uN);
            else tf = in.nlv ? tau_F<false, true>(oc, uC, uW, uE, uS, uN) : tau_F<false, false>(oc, uC, uW, uE, uS, uN);
            double r = (ldcg(Up + k) - uC) - tf;
            if (in.q) r = fma(oc.dt, qg[(long long)n * Ns + k], r);
            rmax = fmax(rmax, fabs(r));
            if (r != r) rmax = r;
        }
    }
    double v[1] = {key_val(block_max_u64<NT>(abs_key(rmax), reinterpret_cast<unsigned long long*>(red)))};
    double g[1];
    if (!reduce_finish<1, true>(c, t, reduce_arrive<1>(t, v), g, red + 32, &s_ok)) return;
    if (K > 1) {
        // the teams' maxima meet in one key word
        if (threadIdx.x == 0 && b == 0) atomicMax(ws.jres, abs_key(g[0]));
        if (!job_barrier(c, ws.jbar, job_ctas * ++jep, &s_ok)) return;
        if (threadIdx.x == 0 && lead) g[0] = key_val(ld_acquire_u64(ws.jres));
    }
    if (lead && threadIdx.x == 0) {
        *in.res_inf = g[0];
        *in.newton_iters = iters_total;
        *in.converged_windows = conv_windows;
    }
    __syncthreads();
}

// Persistent launch over a batch: CTA c works through its job list in order. CLOSURES is
// the set of closures (closure_bit) this instance can run.
template <int NT, typename T, int CLOSURES>
__global__ void __launch_bounds__(NT, 1) batch_kernel(BatchArgs ba) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_ok;
    __shared__ __align__(8) unsigned long long s_ubar;
    if (threadIdx.x == 0) mbar_init(&s_ubar, 1);
    __syncthreads();
    BulkBar bb{&s_ubar, 0u};
    const int c = blockIdx.x;
    for (int j = ba.job_off[c]; j < ba.job_off[c + 1]; ++j) {
        const BatchJob job = ba.jobs[j];
        batch_instance<NT, CLOSURES, T>(ba, job, smem, s_ok, bb);
        __syncthreads();
        if (threadIdx.x == 0) s_ok = ld_acquire_s32(ba.abort_flag);
        __syncthreads();
        if (s_ok) return;
    }
}

}  // namespace pit
