// pit_tc.cuh -- 3x3 convolution (NHWC, BF16) as an implicit GEMM on the 5th-generation
// tensor cores: tcgen05.mma with the FP32 accumulator in tensor memory (TMEM).
//
// GEMM view: rows = 128 pixels of one image row (n, h, w0..w0+127), columns = up to 128
// output channels, K = 9 taps x Cin input channels, taken 16 at a time (one tap, one
// 16-channel chunk per MMA instruction: M = 128, N = nt, K = 16). A CTA computes kRows
// consecutive output rows h0..h0+kRows-1 with one accumulator each in TMEM, so every
// staged weight chunk serves kRows rows and every staged input row up to three.
//
// Operands sit in shared memory in the canonical K-major layout without swizzle: a core
// matrix is 8 rows x 16 bytes (8 BF16 K values per row), rows 16 bytes apart. For each
// 16-channel chunk the CTA stages the input rows h0-1..h0+kRows (130 columns, zeros
// outside the image) as two planes of 8 channels each -- pixel c of a plane at 16 c
// bytes -- so the A operand of tap (r, s) is simply the plane of row r starting at
// column s: 8 consecutive pixels are always one core matrix (stride between core
// matrices along M: 128 bytes; between the two K halves: the plane size). The weights
// of the chunk (9 taps x nt channels) are staged the same way.
//
// Pipeline: two staging buffers. Every thread loads chunk c into buffer c & 1 while the
// MMAs of chunk c - 1 run; thread 0 issues the 9 x kRows MMAs of a chunk and commits them
// to the buffer's mbarrier, which the CTA waits on before refilling that buffer two
// chunks later. After the last chunk the accumulators are read from TMEM (tcgen05.ld,
// each warp its 32 lanes = 32 pixels) for the epilogue: bias, optional residual, optional
// ReLU, BF16. Every mbarrier wait is bounded: on time-out the CTA raises *err, waits (bounded)
// for its MMAs in flight, frees its TMEM and returns without writing.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace pit_tc {

typedef __nv_bfloat16 bf16;

constexpr int kM = 128;          // pixels per output row segment (TMEM lanes)
constexpr int kNMax = 128;       // output channels per CTA
constexpr int kRows = 4;         // output rows per CTA (accumulators: kRows x nt <= 512 TMEM columns)
constexpr int kInRows = kRows + 2;
constexpr int kCols = kM + 2;    // staged columns of an input row (one halo column each side)
constexpr int kThreads = 256;   // 8 warps; warps w and w + 4 read the same TMEM lane quarter
constexpr long long kWaitPolls = 1ll << 22;

// staging buffer: A [kInRows rows][2 halves][kCols][8] then B [9 taps][2 halves][nb][8], BF16,
// nb = min(Cout, kNMax) rows per weight plane
constexpr int kABytes = kInRows * 2 * kCols * 16;
__host__ __device__ constexpr int buf_bytes(int nb) { return kABytes + 9 * 2 * nb * 16; }
// Dynamic shared memory of a launch: two buffers, three mbarriers and the TMEM address
// slot. When one CTA's accumulators take all 512 TMEM columns the request is raised so
// that only one CTA fits on an SM (a second would wait in tcgen05.alloc).
__host__ __device__ constexpr int smem_bytes(int nb) {
    return (nb > 64 ? (2 * buf_bytes(nb) + 32 > 116 * 1024 ? 2 * buf_bytes(nb) + 32 : 116 * 1024)
                    : 2 * buf_bytes(nb) + 32);
}
constexpr int kSmemMax = smem_bytes(kNMax);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Poll until the phase with the given parity has completed, at most kWaitPolls times.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (long long i = 0; i < kWaitPolls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 16-byte asynchronous copy global -> shared (zero-filled when `valid` is false), and the
// wait for all of this thread's outstanding copies.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Whole warp: allocate ncols TMEM columns (power of two >= 32); the address goes to *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor, K-major without swizzle: start address, byte offset
// between the core matrices adjacent in K (lbo) and in M/N (sbo), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive once on bar when every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Store 16 consecutive FP32 columns of this thread's TMEM lane (completion: tcgen05.wait::st).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

// Sixteen BF16 values from two 16-byte words.
__device__ __forceinline__ void load_bf16x16(const bf16* p, float (&f)[16]) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
    for (int e2 = 0; e2 < 2; ++e2) {
        const uint4 u = q[e2];
        const unsigned uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            f[e2 * 8 + 2 * e] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(uu[e] & 0xffff)));
            f[e2 * 8 + 2 * e + 1] = __bfloat162float(__ushort_as_bfloat16((unsigned short)(uu[e] >> 16)));
        }
    }
}

// The epilogue with the residual and mask values already loaded (r, m; null when absent).
__device__ __forceinline__ void epilogue16_loaded(float (&v)[16], const float* r, const float* m, int relu,
                                                  bf16* out) {
    if (r)
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += r[j];
    if (relu)
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
    if (m)
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (!(m[j] > 0.f)) v[j] = 0.f;
    uint32_t packed[8];
#pragma unroll
    for (int e = 0; e < 8; ++e)
        packed[e] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(v[2 * e])) |
                    ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(v[2 * e + 1])) << 16);
    uint4* o = reinterpret_cast<uint4*>(out);
    o[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    o[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
}

// Epilogue of 16 output channels of one pixel: v (accumulator + bias) + residual, then ReLU,
// then the mask (zero where mask <= 0: back through a ReLU whose output was mask), rounded
// to BF16 and stored as two 16-byte words. res and mask may be null.
__device__ __forceinline__ void epilogue16(float (&v)[16], const bf16* res, const bf16* mask, int relu, bf16* out) {
    if (res) {
        float r[16];
        load_bf16x16(res, r);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += r[j];
    }
    if (relu)
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
    if (mask) {
        float m[16];
        load_bf16x16(mask, m);
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (!(m[j] > 0.f)) v[j] = 0.f;
    }
    uint32_t packed[8];
#pragma unroll
    for (int e = 0; e < 8; ++e)
        packed[e] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(v[2 * e])) |
                    ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(v[2 * e + 1])) << 16);
    uint4* o = reinterpret_cast<uint4*>(out);
    o[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    o[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
}

// Y[n][h][w][co] = act(bias[co] + sum_{tap, ci} X[n][h+r-1][w+s-1][ci] W[co][tap][ci] (+ residual)).
// Grid: x = N * ceil(H / kRows) * ceil(W / 128) row-group segments, y = ceil(Cout / 128);
// 128 threads; kSmemBytes of dynamic shared memory. Cin and Cout are multiples of 16.
__global__ void __launch_bounds__(kThreads) conv3x3_fwd_tc_kernel(const bf16* __restrict__ X,
                                                                  const bf16* __restrict__ Wt,
                                                                  const float* __restrict__ bias,
                                                                  const bf16* residual, const bf16* mask,
                                                                  bf16* Y,  // may alias residual (in place)
                                                                  int N, int H, int W, int Cin,
                                                                  int Cout, int relu, int* err) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int nb = Cout < kNMax ? Cout : kNMax;  // weight rows per staged plane
    const int bufb = buf_bytes(nb);
    unsigned char* buf[2] = {sm, sm + bufb};
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * bufb);  // [0], [1] buffers, [2] final
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);

    const int tiles_w = (W + kM - 1) / kM;
    const int groups_h = (H + kRows - 1) / kRows;
    const int grp = blockIdx.x / tiles_w;  // n * groups_h + g
    const int w0 = (blockIdx.x - grp * tiles_w) * kM;
    const int n = grp / groups_h, h0 = (grp - n * groups_h) * kRows;
    const int co0 = blockIdx.y * kNMax;
    const int nt = Cout - co0 < kNMax ? Cout - co0 : kNMax;  // multiple of 16, <= nb
    const int ntp = nt <= 32 ? 32 : (nt <= 64 ? 64 : 128);   // TMEM columns per accumulator
    const uint32_t ncols = (uint32_t)(ntp * kRows);          // power of two, <= 512
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) tmem_alloc(tslot, ncols);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tslot;
    const uint32_t idesc = idesc_bf16(kM, nt);

    // issue the copies of chunk c into buffer c & 1 (one cp.async group; zero fill outside the image)
    auto stage = [&](int c) {
        bf16* sA = reinterpret_cast<bf16*>(buf[c & 1]);
        bf16* sB = reinterpret_cast<bf16*>(buf[c & 1] + kABytes);
        const int ci0 = c * 16;
        for (int t = threadIdx.x; t < kInRows * kCols * 2; t += kThreads) {
            const int half = t & 1, pc = t >> 1;
            const int r = pc / kCols, col = pc - r * kCols;
            const int hh = h0 + r - 1, ww = w0 + col - 1;
            const bool in = hh >= 0 && hh < H && ww >= 0 && ww < W;
            const bf16* src = in ? X + (((size_t)n * H + hh) * W + ww) * Cin + ci0 + half * 8 : X;
            cp_async16(sA + ((size_t)(r * 2 + half) * kCols + col) * 8, src, in);
        }
        for (int t = threadIdx.x; t < nt * 9 * 2; t += kThreads) {
            const int half = t & 1, ot = t >> 1;
            const int o = ot / 9, tap = ot - o * 9;
            cp_async16(sB + ((size_t)(tap * 2 + half) * nb + o) * 8,
                       Wt + ((size_t)(co0 + o) * 9 + tap) * Cin + ci0 + half * 8, true);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    const int nchunks = Cin / 16;
    bool ok = true;
    stage(0);
    for (int c = 0; c < nchunks; ++c) {
        const int b = c & 1;
        if (c + 1 < nchunks) {
            if (c >= 1) {  // buffer (c + 1) & 1: the MMAs of chunk c - 1 have finished reading it
                const bool got = mbar_wait(&bar[(c + 1) & 1], (uint32_t)(((c - 1) >> 1) & 1));
                ok = __syncthreads_and(got) != 0;
                if (!ok) break;
            }
            stage(c + 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");  // chunk c has landed
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        fence_async_smem();  // the copies feed the tensor cores (async proxy)
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(buf[b]), b0 = smem_u32(buf[b] + kABytes);
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int r = tap / 3, s = tap - r * 3;
                const uint64_t bd = smem_desc(b0 + (uint32_t)(tap * 2 * nb * 16), (uint32_t)(nb * 16), 128);
#pragma unroll
                for (int q = 0; q < kRows; ++q) {  // output row h0 + q reads input row h0 + q + r - 1
                    const uint64_t ad =
                        smem_desc(a0 + (uint32_t)(((q + r) * 2 * kCols + s) * 16), kCols * 16, 128);
                    mma_bf16(taddr + (uint32_t)(q * ntp), ad, bd, idesc, (c > 0 || tap > 0) ? 1u : 0u);
                }
            }
            mma_commit(&bar[b]);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");  // no copy left in flight (also after a time-out)
    // every MMA issued has completed (also after a time-out: bounded)
    if (threadIdx.x == 0) mma_commit(&bar[2]);
    const bool fin = mbar_wait(&bar[2], 0);
    ok = (__syncthreads_and(fin) != 0) && ok;
    tc_fence_after();
    if (ok) {
        const int quarter = warp & 3;             // TMEM lanes 32 quarter .. 32 quarter + 31
        const int p = w0 + quarter * 32 + lane;   // this thread's pixel
        for (int q = warp >> 2; q < kRows; q += kThreads / 128) {
            const int h = h0 + q;
            const size_t ybase = (((size_t)n * H + h) * W + p) * Cout + co0;
            for (int j0 = 0; j0 < nt; j0 += 16) {
                uint32_t r[16];
                tmem_ld16(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(q * ntp + j0), r);
                if (p < W && h < H) {
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]) + bias[co0 + j0 + j];
                    epilogue16(v, residual ? residual + ybase + j0 : nullptr, mask ? mask + ybase + j0 : nullptr, relu,
                               Y + ybase + j0);
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, ncols);
}

}  // namespace pit_tc

namespace pit_tc {

// ------------------------------------------------------------------ weight gradients
//
// dW[co][tap][ci] = sum over pixels p of X[p + tap][ci] dY[p][co] (zero outside the image),
// as GEMMs on the tensor cores with dY as the shared operand: B = dY (N = 64 output
// channels), K = pixels, 64 per staged segment of an image row (4 MMAs of K = 16). The
// 128 rows of A hold two taps at once -- rows 0..63 the input channels of tap 2g shifted
// by that tap, rows 64..127 those of tap 2g + 1 -- so five accumulators (taps 0-1, 2-3,
// 4-5, 6-7, 8) cover all nine taps and every dY segment is staged once. A CTA covers a
// 64 x 64 channel tile pair and a split of the image rows and writes FP32 partial sums;
// a second pass adds them over the splits in a fixed order.
//
// Both operands come from NHWC activations, where channels are contiguous and pixels are
// not; staging transposes them into the K-major core-matrix layout: a thread loads an
// 8-pixel x 8-channel block (8 x 16 bytes), exchanges 16-bit halves between pixel pairs
// (16 byte permutes), and after that the rows of the transposed block are a renaming of
// the registers -- each is one 16-byte row of a core matrix (8 channels x 8 pixels, 128
// contiguous bytes). Plane j of a staged operand holds pixels 8j..8j+7 of all its rows,
// so MMA k reads planes 2k and 2k+1 (byte offset between K-adjacent core matrices: the
// plane size; between row groups: 128 bytes).
constexpr int kWK = 64;                            // pixels per staged segment
constexpr int kWPlanes = kWK / 8;
constexpr int kWCi = 64;                           // input channels per tap half of A
constexpr int kWCo = 64;                           // output channels (N)
constexpr int kWGroups = 5;                        // tap pairs
constexpr int kWAGroupBytes = kWPlanes * 128 * 16;  // one group: 128 rows
constexpr int kWABytes = kWGroups * kWAGroupBytes;
constexpr int kWBBytes = kWPlanes * kWCo * 16;
constexpr int kWBufBytes = kWABytes + kWBBytes;
constexpr int kWSmemBytes = 2 * kWBufBytes + 32;
constexpr int kWBlk = 3;                           // 8x8 blocks per thread and segment, at most (<= 640)

// Transpose an 8 x 8 block of 16-bit values held as 8 rows of 4 words (row i = pixel i,
// word k = channels 2k, 2k+1) into 8 rows of 4 words indexed by channel (word a = pixels
// 2a, 2a+1).
__device__ __forceinline__ void transpose8x8_b16(const uint32_t (&in)[8][4], uint32_t (&out)[8][4]) {
    uint32_t w[8][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            w[2 * a][k] = __byte_perm(in[2 * a][k], in[2 * a + 1][k], 0x5410);      // channel 2k of pixels 2a, 2a+1
            w[2 * a + 1][k] = __byte_perm(in[2 * a][k], in[2 * a + 1][k], 0x7632);  // channel 2k+1
        }
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int a = 0; a < 4; ++a) out[c][a] = w[2 * a + (c & 1)][c >> 1];
}

// Grid: x = splits of the N*H image rows (rows_per_split each), y = ceil(Cin / 64),
// z = ceil(Cout / 64); 128 threads; kWSmemBytes of dynamic shared memory.
// part[split][co][tap][ci] receives the CTA's sums. Cin and Cout are multiples of 16.
__global__ void __launch_bounds__(kThreads) conv3x3_bwdw_tc_kernel(const bf16* __restrict__ X,
                                                                   const bf16* __restrict__ dY,
                                                                   float* __restrict__ part, int N, int H, int W,
                                                                   int Cin, int Cout, int rows_per_split, int* err) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int ci0 = blockIdx.y * kWCi, co0 = blockIdx.z * kWCo;
    const int cw = Cin - ci0 < kWCi ? Cin - ci0 : kWCi;   // real rows per tap half (multiple of 16)
    const int nco = Cout - co0 < kWCo ? Cout - co0 : kWCo; // N (multiple of 16)
    unsigned char* buf[2] = {sm, sm + kWBufBytes};
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * kWBufBytes);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 3);
    const int ntp = nco <= 32 ? 32 : 64;                    // TMEM columns per accumulator
    const uint32_t ncols = ntp * kWGroups <= 256 ? 256u : 512u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // A rows that never receive data stay zero in both buffers: rows cw..63 of every tap
    // half, and the upper half of the last group (there is no tenth tap)
    for (int b = 0; b < 2; ++b)
        for (int t = threadIdx.x; t < kWGroups * kWPlanes * 128; t += kThreads) {
            const int row = t & 127, gp = t >> 7;  // gp = group * kWPlanes + plane
            const int grp = gp / kWPlanes;
            const bool empty = (row & 63) >= cw || (grp == kWGroups - 1 && row >= 64);
            if (empty) *reinterpret_cast<uint4*>(buf[b] + (size_t)gp * 128 * 16 + (size_t)row * 16) = make_uint4(0, 0, 0, 0);
        }
    if (warp == 0) tmem_alloc(tslot, ncols);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tslot;
    const uint32_t idesc = idesc_bf16(kM, nco);

    const int row_begin = blockIdx.x * rows_per_split;
    const int row_end = min(row_begin + rows_per_split, N * H);
    const int segs_w = (W + kWK - 1) / kWK;
    const int nseg = (row_end > row_begin ? row_end - row_begin : 0) * segs_w;
    // 8x8 blocks per segment: A, 9 taps x cw/8 channel groups x 8 planes; B, nco/8 x 8
    const int cg8 = cw / 8, nA = 9 * cg8 * kWPlanes, nB = (nco / 8) * kWPlanes;

    uint4 in[kWBlk][8];
    auto load = [&](int sg) {
        const int rowi = row_begin + sg / segs_w;
        const int w0 = (sg % segs_w) * kWK;
        const int n = rowi / H, h = rowi - n * H;
#pragma unroll
        for (int u = 0; u < kWBlk; ++u) {
            const int blk = threadIdx.x + u * kThreads;
            const bool isA = blk < nA;
            int tap = 0, cg, j;
            if (isA) {
                tap = blk / (cg8 * kWPlanes);
                const int q = blk - tap * cg8 * kWPlanes;
                j = q / cg8;
                cg = q - j * cg8;
            } else {
                const int q = blk - nA;
                j = q / (nco / 8);
                cg = q - j * (nco / 8);
            }
            const int r = tap / 3, s = tap - r * 3, hh = h + r - 1;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int w = w0 + j * 8 + i;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (blk < nA + nB && w < W) {
                    if (isA) {
                        const int ww = w + s - 1;
                        if (hh >= 0 && hh < H && ww >= 0 && ww < W)
                            v = *reinterpret_cast<const uint4*>(X + (((size_t)n * H + hh) * W + ww) * Cin + ci0 + cg * 8);
                    } else {
                        v = *reinterpret_cast<const uint4*>(dY + (((size_t)n * H + h) * W + w) * Cout + co0 + cg * 8);
                    }
                }
                in[u][i] = v;
            }
        }
    };
    auto store = [&](unsigned char* sA, unsigned char* sB) {
#pragma unroll
        for (int u = 0; u < kWBlk; ++u) {
            const int blk = threadIdx.x + u * kThreads;
            if (blk >= nA + nB) continue;
            const bool isA = blk < nA;
            int tap = 0, cg, j;
            if (isA) {
                tap = blk / (cg8 * kWPlanes);
                const int q = blk - tap * cg8 * kWPlanes;
                j = q / cg8;
                cg = q - j * cg8;
            } else {
                const int q = blk - nA;
                j = q / (nco / 8);
                cg = q - j * (nco / 8);
            }
            uint32_t w8[8][4], out[8][4];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                w8[i][0] = in[u][i].x;
                w8[i][1] = in[u][i].y;
                w8[i][2] = in[u][i].z;
                w8[i][3] = in[u][i].w;
            }
            transpose8x8_b16(w8, out);
            unsigned char* dst = isA ? sA + (size_t)((tap >> 1) * kWPlanes + j) * 128 * 16 +
                                           (size_t)((tap & 1) * 64 + cg * 8) * 16
                                     : sB + (size_t)j * kWCo * 16 + (size_t)cg * 128;
            // Core matrices of neighbouring threads sit 128 bytes apart, i.e. on the same four
            // banks: thread-dependent row order (rotated by rot) spreads one store instruction
            // of a warp over all 32 banks. The rotation is done on registers in three steps.
            const int rot = (cg + j) & 7;
#pragma unroll
            for (int st = 1; st < 8; st <<= 1) {
                if (rot & st) {
                    uint32_t tmp[8][4];
#pragma unroll
                    for (int c = 0; c < 8; ++c)
#pragma unroll
                        for (int a = 0; a < 4; ++a) tmp[c][a] = out[(c + st) & 7][a];
#pragma unroll
                    for (int c = 0; c < 8; ++c)
#pragma unroll
                        for (int a = 0; a < 4; ++a) out[c][a] = tmp[c][a];
                }
            }
#pragma unroll
            for (int c = 0; c < 8; ++c)  // out[c] now holds transposed row (c + rot) & 7
                *reinterpret_cast<uint4*>(dst + ((c + rot) & 7) * 16) =
                    make_uint4(out[c][0], out[c][1], out[c][2], out[c][3]);
        }
    };

    bool ok = true;
    if (nseg > 0) load(0);
    for (int sg = 0; sg < nseg; ++sg) {
        const int b = sg & 1;
        if (sg >= 2) {
            const bool got = mbar_wait(&bar[b], (uint32_t)(((sg - 2) >> 1) & 1));
            ok = __syncthreads_and(got) != 0;
            if (!ok) break;
        }
        unsigned char* sA = buf[b];
        unsigned char* sB = buf[b] + kWABytes;
        store(sA, sB);
        if (sg + 1 < nseg) load(sg + 1);
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int k = 0; k < kWPlanes / 2; ++k) {
                const uint64_t bd = smem_desc(b0 + (uint32_t)(2 * k * kWCo * 16), kWCo * 16, 128);
#pragma unroll
                for (int g = 0; g < kWGroups; ++g) {
                    const uint64_t ad =
                        smem_desc(a0 + (uint32_t)((g * kWPlanes + 2 * k) * 128 * 16), 128 * 16, 128);
                    mma_bf16(taddr + (uint32_t)(g * ntp), ad, bd, idesc, (sg > 0 || k > 0) ? 1u : 0u);
                }
            }
            mma_commit(&bar[b]);
        }
    }
    if (threadIdx.x == 0) mma_commit(&bar[2]);
    const bool fin = mbar_wait(&bar[2], 0);
    ok = (__syncthreads_and(fin) != 0) && ok;
    tc_fence_after();
    if (ok) {
        // TMEM lane = A row: rows 0..63 tap 2g, rows 64..127 tap 2g + 1; column = output channel
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane, ci = ci0 + (row & 63);
        float* P = part + (size_t)blockIdx.x * Cout * 9 * Cin;
        for (int g = warp >> 2; g < kWGroups; g += kThreads / 128) {
            const int tap = 2 * g + (row >> 6);
            for (int j0 = 0; j0 < nco; j0 += 16) {
                uint32_t v[16];
                tmem_ld16(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(g * ntp + j0), v);
                if (tap < 9 && (row & 63) < cw) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        P[((size_t)(co0 + j0 + j) * 9 + tap) * Cin + ci] = nseg > 0 ? __uint_as_float(v[j]) : 0.f;
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(taddr, ncols);
}

}  // namespace pit_tc
