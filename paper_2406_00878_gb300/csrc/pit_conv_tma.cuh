// pit_conv_tma.cuh -- 3x3 convolution (NHWC, BF16) on the tcgen05 tensor cores with TMA
// tile loads: a persistent, warp-specialised form of the implicit GEMM of pit_tc.cuh for
// layers whose weights fit in shared memory.
//
// Each CTA owns one SM and one tile of up to 256 output channels, keeps that tile's weights
// (9 taps x Cin x nco, one TMA tensor load) resident in shared memory, and walks a
// contiguous range of output rows (image row h of image n, 128-pixel segment w0). An output
// row needs input rows h-1, h, h+1; they stream through a ring of `ring` staged rows,
// each loaded by one TMA tensor copy (cp.async.bulk.tensor, zero fill off the image) into
// the canonical K-major layout without swizzle: plane g (channels 8g..8g+7) of a staged row
// holds its 130 pixels (w0-1 .. w0+128) at 16 bytes each, so the A operand of tap (r, s)
// and channel chunk kc is the staged row h+r-1 starting at pixel s of planes 2kc, 2kc+1
// (byte offset between the K halves: the plane size; between 8-pixel groups: 128 bytes).
// Consecutive output rows share two of their three input rows, so a range of R rows
// stages R + 2 rows per image it touches.
//
// Warp roles (192 threads):
//   warp 0, one lane   TMA producer: the weights once, then the input rows in order;
//                      a ring slot is refilled when the MMAs that read it have completed
//                      (tcgen05.commit on the slot's `empty` barrier)
//   warp 1, one lane   MMA issuer: per output row 9 taps x Cin/16 MMAs (M = 128 pixels,
//                      N = nco, K = 16) into one of two TMEM accumulators, committed to the
//                      accumulator's `full` barrier; then it releases the slots no later
//                      row reads
//   warps 2..5         epilogue: tcgen05.ld of the accumulator (each warp its TMEM lane
//                      quarter = 32 pixels), bias, optional residual, optional ReLU, BF16
//                      stores; then they free the accumulator for the row after next
// With two accumulators the epilogue of row i overlaps the MMAs of row i + 1.
//
// Every mbarrier wait is bounded. A wait that runs out raises the CTA's abort word and the
// launch's error flag; every role leaves its loop, the CTA waits (bounded) for its MMAs
// and its TMA copies in flight, frees its TMEM and returns without further writes.
#pragma once

#include <cuda.h>

#include "pit_tc.cuh"

namespace pit_tc {

constexpr int kFThreads = 192;
constexpr int kFRingMax = 8;
constexpr int kFNMax = 256;  // output channels per CTA tile (N of one MMA)

// Bytes of one staged input row (Cin channels x kCols pixels), and its slot. Swizzled rows
// (Cin a multiple of 64): one 128-byte-swizzled block per 64 channels, kCols rows of 128
// bytes rounded up to whole 1024-byte swizzle atoms; otherwise 128-byte aligned.
constexpr int kSwBlockBytes = (kCols + 7) / 8 * 1024;
__host__ __device__ constexpr int fwd_row_bytes(int cin) { return cin * kCols * 2; }
__host__ __device__ constexpr int fwd_slot_bytes(int cin, int sw) {
    return sw ? cin / 64 * kSwBlockBytes : (fwd_row_bytes(cin) + 127) / 128 * 128;
}
__host__ __device__ constexpr int fwd_w_bytes(int cin, int nco) { return 9 * cin * nco * 2; }
// Dynamic shared memory: alignment slack, weights, ring, bias (kFNMax floats), barriers and
// the TMEM slot.
__host__ __device__ constexpr int fwd_smem_bytes(int cin, int nco, int ring, int sw) {
    return 1024 + fwd_w_bytes(cin, nco) + ring * fwd_slot_bytes(cin, sw) + kFNMax * 4 + 512;
}

struct FwdTmaArgs {
    const float* bias;        // [Cout]
    const bf16* residual;     // [N][H][W][Cout] or null
    const bf16* mask;         // [N][H][W][Cout] or null: outputs zeroed where mask <= 0
    bf16* Y;                  // [N][H][W][Cout]
    int N, H, W, Cin, Cout;
    int relu;
    int nco;                  // output channels of a CTA tile (multiple of 16, <= kFNMax)
    int ntp;                  // TMEM columns per accumulator: power of two >= max(nco, 32)
    int ring;                 // staged input rows, 3..kFRingMax
    int ctas_per_tile;        // CTAs sharing one output-channel tile
    int sw;                   // input rows as 128-byte-swizzled 64-channel blocks (Cin % 64 == 0)
    int* err;                 // raised when a wait timed out
};

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

// TMA tensor tile loads into shared memory, completing on bar's transaction count.
__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait that also gives up when another role of the CTA has raised the abort word.
__device__ __forceinline__ bool fwd_wait(uint64_t* bar, uint32_t parity, volatile int* abort_word) {
    for (long long i = 0; i < kWaitPolls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && *abort_word) return false;
    }
    *abort_word = 1;
    return false;
}

// Output row q of a CTA tile: q = (segment_w * N + n) * H + h.
struct FwdRow {
    int wt, n, h;
};
__device__ __forceinline__ FwdRow fwd_row(long long q, int N, int H) {
    FwdRow r;
    r.h = (int)(q % H);
    const long long t = q / H;
    r.n = (int)(t % N);
    r.wt = (int)(t / N);
    return r;
}

// Shared-memory descriptor of a K-major operand in 128-byte-swizzled rows (8-row atoms of
// 1024 bytes; stride between 8-row groups 1024 bytes); base_offset fills bits 49-51. The
// tensor cores apply the swizzle to absolute shared-memory addresses (atoms 1024-byte
// aligned), so an operand may start at any 128-byte row of an atom (a pixel shift) or at a
// 32-byte K step inside a row with base offset 0 -- checked element-wise against the oracle
// by the layer tests.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr, uint32_t base_offset) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(base_offset & 7) << 49;
    d |= (uint64_t)2 << 61;
    return d;
}

// X map, unswizzled rows: dims (8 channels, W pixels, Cin/8 planes, H, N), box (8, kCols,
// Cin/8, 1, 1). Swizzled rows: dims (Cin, W, H, N), box (64, kCols, 1, 1), 128-byte swizzle.
// W map: dims (8 channels, Cout, Cin/8 planes, 9 taps), box (8, nco, Cin/8, 9).
// Grid: co_tiles x ctas_per_tile; kFThreads threads; fwd_smem_bytes(Cin, nco, ring) bytes.
__global__ void __launch_bounds__(kFThreads, 1) conv3x3_fwd_tma_kernel(const __grid_constant__ CUtensorMap xmap,
                                                                       const __grid_constant__ CUtensorMap wmap,
                                                                       FwdTmaArgs a) {
    extern __shared__ __align__(128) unsigned char sm_raw[];
    // 1024-byte aligned base (swizzle atoms; TMA destinations)
    unsigned char* sm = sm_raw + ((1024 - (smem_u32(sm_raw) & 1023)) & 1023);
    const int G = a.Cin / 8, nco = a.nco, ring = a.ring;
    unsigned char* sW = sm;
    unsigned char* sRing = sm + fwd_w_bytes(a.Cin, nco);
    const int slot_bytes = fwd_slot_bytes(a.Cin, a.sw);
    float* s_bias = reinterpret_cast<float*>(sRing + ring * slot_bytes);
    uint64_t* full = reinterpret_cast<uint64_t*>(s_bias + kFNMax);
    uint64_t* empty = full + kFRingMax;
    uint64_t* acc_full = empty + kFRingMax;  // [2]
    uint64_t* acc_empty = acc_full + 2;      // [2]
    uint64_t* wfull = acc_empty + 2;
    uint64_t* fin = wfull + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort_word = reinterpret_cast<volatile int*>(tslot + 1);

    const int tile = blockIdx.x / a.ctas_per_tile, part = blockIdx.x - tile * a.ctas_per_tile;
    const int co0 = tile * kFNMax;
    const int nt = a.Cout - co0 < nco ? a.Cout - co0 : nco;  // this tile's channels (multiple of 16)
    const int w_tiles = (a.W + kM - 1) / kM;
    const long long T = (long long)w_tiles * a.N * a.H;
    const long long q0 = T * part / a.ctas_per_tile, q1 = T * (part + 1) / a.ctas_per_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t ncols = (uint32_t)(2 * a.ntp);

    if (warp == 0) tmem_alloc(tslot, ncols);
    if (threadIdx.x == 0) {
        for (int s = 0; s < ring; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
        }
        mbar_init(wfull, 1);
        mbar_init(fin, 1);
        *abort_word = 0;
        fence_mbar_init();
    }
    for (int j = threadIdx.x; j < kFNMax; j += kFThreads) s_bias[j] = j < nt ? a.bias[co0 + j] : 0.f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tslot;
    const uint32_t row_tx = (uint32_t)fwd_row_bytes(a.Cin);
    long long loads = 0;  // producer: input rows issued

    if (warp == 0) {
        if (lane == 0) {
            mbar_arrive_tx(wfull, (uint32_t)(9 * G * nco * 16));
            if (a.sw) {
                // tap t, channel block kb: nco rows of 64 channels, 128-byte swizzled
                for (int t = 0; t < 9; ++t)
                    for (int kb = 0; kb < a.Cin / 64; ++kb)
                        tma_load_3d(sW + (size_t)(t * (a.Cin / 64) + kb) * nco * 128, &wmap, kb * 64, t, co0, wfull);
            } else {
                tma_load_4d(sW, &wmap, 0, co0, 0, 0, wfull);
            }
            for (long long q = q0; q < q1 && !*abort_word; ++q) {
                const FwdRow r = fwd_row(q, a.N, a.H);
                const bool first = q == q0 || r.h == 0;
                for (int hh = first ? r.h - 1 : r.h + 1; hh <= r.h + 1; ++hh) {
                    const int s = (int)(loads % ring);
                    if (loads >= ring && !fwd_wait(&empty[s], (uint32_t)((loads / ring - 1) & 1), abort_word)) break;
                    mbar_arrive_tx(&full[s], row_tx);
                    unsigned char* dst = sRing + (size_t)s * slot_bytes;
                    if (a.sw) {
                        for (int kb = 0; kb < a.Cin / 64; ++kb)
                            tma_load_4d(dst + (size_t)kb * kSwBlockBytes, &xmap, kb * 64, r.wt * kM - 1, hh, r.n, &full[s]);
                    } else {
                        tma_load_5d(dst, &xmap, 0, r.wt * kM - 1, 0, hh, r.n, &full[s]);
                    }
                    ++loads;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kM, nco);
            const uint32_t w0a = smem_u32(sW), r0a = smem_u32(sRing);
            bool ok = fwd_wait(wfull, 0, abort_word);
            long long L = 0, released = 0;
            int i = 0;
            for (long long q = q0; q < q1 && ok; ++q, ++i) {
                const FwdRow r = fwd_row(q, a.N, a.H);
                const bool first = q == q0 || r.h == 0;
                const long long ai = first ? L : L - 2;  // load of input row h - 1
                L += first ? 3 : 1;
                const int acc = i & 1, use = i >> 1;
                if (use >= 1 && !(ok = fwd_wait(&acc_empty[acc], (uint32_t)((use - 1) & 1), abort_word))) break;
                for (int j = 0; j < 3 && ok; ++j) {
                    const long long l = ai + j;
                    ok = fwd_wait(&full[l % ring], (uint32_t)((l / ring) & 1), abort_word);
                }
                if (!ok) break;
                tc_fence_after();
                for (int tap = 0; tap < 9; ++tap) {
                    const int rr = tap / 3, ss = tap - rr * 3;
                    const uint32_t sbase = r0a + (uint32_t)(((ai + rr) % ring) * slot_bytes);
                    const uint32_t abase = sbase + (uint32_t)(ss * 16);
                    for (int kc = 0; kc < G / 2; ++kc) {
                        // swizzled: block kc / 4, rows from pixel ss (ss * 128 bytes), K step of
                        // 32 bytes inside the 128-byte row; else plane pair 2 kc from pixel ss
                        const uint64_t ad =
                            a.sw ? smem_desc_sw128(sbase + (uint32_t)((kc >> 2) * kSwBlockBytes + ss * 128 + (kc & 3) * 32),
                                                   0u)
                                 : smem_desc(abase + (uint32_t)(2 * kc * kCols * 16), kCols * 16, 128);
                        const uint64_t bd =
                            a.sw ? smem_desc_sw128(w0a + (uint32_t)((tap * (G / 8) + (kc >> 2)) * nco * 128 + (kc & 3) * 32), 0u)
                                 : smem_desc(w0a + (uint32_t)((tap * G + 2 * kc) * nco * 16), (uint32_t)(nco * 16), 128);
                        mma_bf16(taddr + (uint32_t)(acc * a.ntp), ad, bd, idesc, (tap > 0 || kc > 0) ? 1u : 0u);
                    }
                }
                mma_commit(&acc_full[acc]);
                // free the slots no later row reads (all three at the end of an image or range)
                const bool next_first = q + 1 >= q1 || fwd_row(q + 1, a.N, a.H).h == 0;
                const long long upto = next_first ? ai + 3 : ai + 1;
                for (; released < upto; ++released) mma_commit(&empty[released % ring]);
            }
            if (!ok) atomicExch(a.err, 1);
            mma_commit(fin);  // arrives once every MMA issued above has completed
        }
    } else {
        // epilogue: warps 2..5 cover the TMEM lane quarters 2, 3, 0, 1
        const int quarter = warp & 3;
        int i = 0;
        for (long long q = q0; q < q1; ++q, ++i) {
            const int acc = i & 1, use = i >> 1;
            // one decision per warp (tcgen05.ld below is warp-wide)
            if (!__all_sync(0xffffffffu, fwd_wait(&acc_full[acc], (uint32_t)(use & 1), abort_word))) {
                if (lane == 0) {
                    *abort_word = 1;
                    atomicExch(a.err, 1);
                }
                break;
            }
            tc_fence_after();
            const FwdRow r = fwd_row(q, a.N, a.H);
            const int p = r.wt * kM + quarter * 32 + lane;  // this thread's pixel
            const size_t ybase = (((size_t)r.n * a.H + r.h) * a.W + p) * a.Cout + co0;
            for (int j0 = 0; j0 < nt; j0 += 16) {
                uint32_t v32[16];
                tmem_ld16(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * a.ntp + j0), v32);
                if (p < a.W) {
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(v32[j]) + s_bias[j0 + j];
                    epilogue16(v, a.residual ? a.residual + ybase + j0 : nullptr, a.mask ? a.mask + ybase + j0 : nullptr,
                               a.relu, a.Y + ybase + j0);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive1(&acc_empty[acc]);
        }
    }
    __syncthreads();
    // drain: the MMAs (fin) and every TMA copy still in flight, bounded, before TMEM and
    // shared memory are given up
    if (warp == 1 && lane == 0) {
        bool done = false;
        for (long long k = 0; k < kWaitPolls && !done; ++k) done = mbar_try_wait(fin, 0);
        if (!done) atomicExch(a.err, 1);
    }
    if (warp == 0 && lane == 0) {
        const long long from = loads > ring ? loads - ring : 0;
        for (long long l = from; l < loads; ++l) {
            bool done = false;
            for (long long k = 0; k < kWaitPolls && !done; ++k) done = mbar_try_wait(&full[l % ring], (uint32_t)((l / ring) & 1));
            if (!done) atomicExch(a.err, 1);
        }
        bool wdone = false;
        for (long long k = 0; k < kWaitPolls && !wdone; ++k) wdone = mbar_try_wait(wfull, 0);
        if (!wdone) atomicExch(a.err, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(taddr, ncols);
}


// ---------------------------------------------------------- row-stationary form
//
// A bf16 tcgen05.mma with K = 16 takes about the same time for every N up to 256 (M = 128),
// so a layer with 64 output channels leaves three quarters of each instruction idle in the
// form above. Here every staged input row j is read once per pixel shift s and multiplied
// by the weights of its three row taps stacked along N: B = [W(0,s); W(1,s); W(2,s)], N =
// 3 nco. Row tap r of input row j feeds output row j + 1 - r, so one MMA adds into three
// output rows at once. Their accumulators (nco TMEM columns each) are laid out so that the
// three are adjacent: output row i of the CTA's sequence owns block NB - 1 - (i mod NB) of
// NB = 512 / nco blocks, i.e. later rows sit at lower columns. A run of rows that wraps
// around the ring (or would exceed N = 256) is split into two MMAs. Blocks are zeroed by
// the epilogue after it has read them (and once at the start), so every MMA accumulates.
//
// Per output row (steady state, 64 input channels): 3 shifts x 4 K steps = 12 MMAs of
// N = 192 instead of 36 of N = 64.
//
// Warp roles (320 threads): warp 0 one lane, TMA producer (weights, then input rows);
// warp 1 one lane, MMA issuer; warps 2..9 epilogue, two per TMEM lane quarter (warp w reads
// quarter w % 4 and every other 16-column chunk), which also zero the blocks they read.
//
// Weights in shared memory: for shift s and channel block kb, the B tile holds rows
// r * nco + co (r = 0, 1, 2) of 64 channels, 128-byte swizzled: 9 TMA boxes per block.
// Input rows: as above (swizzled 64-channel blocks of kCols pixels).
constexpr int kRThreads = 320;  // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue (two per lane quarter)

template <int KB>
__global__ void __launch_bounds__(kRThreads, 1) conv3x3_fwd_rows_kernel(const __grid_constant__ CUtensorMap xmap,
                                                                        const __grid_constant__ CUtensorMap wmap,
                                                                        FwdTmaArgs a) {
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char* sm = sm_raw + ((1024 - (smem_u32(sm_raw) & 1023)) & 1023);
    const int nco = a.nco, ring = a.ring;
    // accumulator blocks in TMEM: a power of two, 4..8 (nco <= 128)
    const int NB = nco <= 64 ? 8 : 4;
    unsigned char* sW = sm;
    unsigned char* sRing = sm + fwd_w_bytes(a.Cin, nco);
    const int slot_bytes = fwd_slot_bytes(a.Cin, 1);
    float* s_bias = reinterpret_cast<float*>(sRing + ring * slot_bytes);
    uint64_t* full = reinterpret_cast<uint64_t*>(s_bias + kFNMax);  // [kFRingMax] input rows landed
    uint64_t* empty = full + kFRingMax;                               // [kFRingMax] input rows consumed
    uint64_t* bfull = empty + kFRingMax;                              // [8] output row complete
    uint64_t* bempty = bfull + 8;                                     // [8] block read and zeroed
    uint64_t* wfull = bempty + 8;
    uint64_t* fin = wfull + 1;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort_word = reinterpret_cast<volatile int*>(tslot + 1);

    const int tile = blockIdx.x / a.ctas_per_tile, part = blockIdx.x - tile * a.ctas_per_tile;
    const int co0 = tile * nco;
    const int nt = a.Cout - co0 < nco ? a.Cout - co0 : nco;
    const int w_tiles = (a.W + kM - 1) / kM;
    const long long T = (long long)w_tiles * a.N * a.H;
    const long long q0 = T * part / a.ctas_per_tile, q1 = T * (part + 1) / a.ctas_per_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) tmem_alloc(tslot, 512);
    if (threadIdx.x == 0) {
        for (int s = 0; s < ring; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NB; ++b) {
            mbar_init(&bfull[b], 1);
            mbar_init(&bempty[b], 8);
        }
        mbar_init(wfull, 1);
        mbar_init(fin, 1);
        *abort_word = 0;
        fence_mbar_init();
    }
    for (int j = threadIdx.x; j < kFNMax; j += kRThreads) s_bias[j] = j < nt ? a.bias[co0 + j] : 0.f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tslot;
    if (warp >= 2) {
        // every accumulator block starts at zero (the two warps of a lane quarter take
        // alternate 16-column chunks)
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        uint32_t z[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) z[k] = 0u;
        for (int c = half * 16; c < 512; c += 32) tmem_st16(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c, z);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t row_tx = (uint32_t)fwd_row_bytes(a.Cin);
    long long loads = 0;  // producer: input rows issued

    if (warp == 0) {
        if (lane == 0) {
            mbar_arrive_tx(wfull, (uint32_t)(9 * KB * 64 * nco * 2));
            for (int t = 0; t < 9; ++t) {
                const int r = t / 3, sh = t - 3 * r;
                for (int kb = 0; kb < KB; ++kb)
                    tma_load_3d(sW + (size_t)((sh * KB + kb) * 3 + r) * nco * 128, &wmap, kb * 64, t, co0, wfull);
            }
            // input rows of each segment (one image's rows ha..hb of the range): ha-1 .. hb+1 on the image
            for (long long q = q0; q < q1 && !*abort_word;) {
                const FwdRow r0 = fwd_row(q, a.N, a.H);
                const long long qe = min(q1, q + (a.H - r0.h));  // end of the segment
                const int ha = r0.h, hb = r0.h + (int)(qe - q) - 1;
                for (int j = max(ha - 1, 0); j <= min(hb + 1, a.H - 1) && !*abort_word; ++j) {
                    const int s = (int)(loads % ring);
                    if (loads >= ring && !fwd_wait(&empty[s], (uint32_t)((loads / ring - 1) & 1), abort_word)) break;
                    mbar_arrive_tx(&full[s], row_tx);
                    unsigned char* dst = sRing + (size_t)s * slot_bytes;
#pragma unroll
                    for (int kb = 0; kb < KB; ++kb)
                        tma_load_4d(dst + (size_t)kb * kSwBlockBytes, &xmap, kb * 64, r0.wt * kM - 1, j, r0.n, &full[s]);
                    ++loads;
                }
                q = qe;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc0 = idesc_bf16(kM, 16) & ~(0x3Fu << 17);  // N filled per MMA
            const uint64_t a0 = smem_desc_sw128(smem_u32(sRing), 0u);
            const uint64_t b0 = smem_desc_sw128(smem_u32(sW), 0u);
            const uint32_t btile = (uint32_t)nco * 128;                   // bytes of one r block of B
            bool ok = fwd_wait(wfull, 0, abort_word);
            long long l = 0;
            int ibase = 0;  // sequence index of the segment's first output row
            for (long long q = q0; q < q1 && ok;) {
                const FwdRow r0 = fwd_row(q, a.N, a.H);
                const long long qe = min(q1, q + (a.H - r0.h));
                const int ha = r0.h, hb = r0.h + (int)(qe - q) - 1;
                for (int j = max(ha - 1, 0); j <= min(hb + 1, a.H - 1) && ok; ++j, ++l) {
                    // output rows that start here wait until their block is free (read and zeroed)
                    for (int h = (j == 0 ? 0 : j + 1); h <= j + 1 && ok; ++h) {
                        if (h < ha || h > hb) continue;
                        const int i = ibase + (h - ha);
                        const int u = i / NB;
                        if (u >= 1) ok = fwd_wait(&bempty[i & (NB - 1)], (uint32_t)((u - 1) & 1), abort_word);
                    }
                    if (ok) ok = fwd_wait(&full[l % ring], (uint32_t)((l / ring) & 1), abort_word);
                    if (!ok) break;
                    tc_fence_after();
                    const int rlo = max(0, j + 1 - hb), rhi = min(2, j + 1 - ha);
                    const uint64_t arow = a0 + (uint64_t)(((l % ring) * slot_bytes) >> 4);
                    // runs of adjacent accumulator blocks: r = rlo..rhi <-> output rows j+1-r,
                    // sequence indices i decreasing, columns increasing unless the ring wraps;
                    // per run: D column, instruction descriptor, B descriptor of its first r
                    uint32_t rcol[3], ridesc[3];
                    uint64_t rb[3];
                    int nr = 0;
                    for (int r = rlo; r <= rhi;) {
                        int e = r;
                        while (e + 1 <= rhi && ((ibase + (j + 1 - e - ha)) & (NB - 1)) != 0 && (e + 2 - r) * nco <= 256) ++e;
                        const int i = ibase + (j + 1 - r - ha);
                        rcol[nr] = taddr + (uint32_t)((NB - 1 - (i & (NB - 1))) * nco);
                        ridesc[nr] = idesc0 | ((uint32_t)((e - r + 1) * nco) >> 3 << 17);
                        rb[nr] = b0 + (uint64_t)((r * btile) >> 4);
                        ++nr;
                        r = e + 1;
                    }
#pragma unroll
                    for (int sh = 0; sh < 3; ++sh)
#pragma unroll
                        for (int kc = 0; kc < 4 * KB; ++kc) {
                            const uint64_t ad =
                                arow + (uint64_t)(((kc >> 2) * kSwBlockBytes + sh * 128 + (kc & 3) * 32) >> 4);
                            const uint64_t boff = (uint64_t)((((sh * KB + (kc >> 2)) * 3) * btile + (kc & 3) * 32) >> 4);
                            mma_bf16(rcol[0], ad, rb[0] + boff, ridesc[0], 1u);
                            if (nr > 1) mma_bf16(rcol[1], ad, rb[1] + boff, ridesc[1], 1u);
                            if (nr > 2) mma_bf16(rcol[2], ad, rb[2] + boff, ridesc[2], 1u);
                        }
                    mma_commit(&empty[l % ring]);
                    // output rows finished by this input row: j - 1, and j itself on the last image row
                    for (int h = j - 1; h <= j; ++h) {
                        if (h < ha || h > hb || (h == j && j != a.H - 1)) continue;
                        mma_commit(&bfull[(ibase + (h - ha)) & (NB - 1)]);
                    }
                }
                ibase += hb - ha + 1;
                q = qe;
            }
            if (!ok) atomicExch(a.err, 1);
            mma_commit(fin);
        }
    } else {
        // epilogue: warps 2..9 -- warp w reads TMEM lane quarter w % 4 (32 pixels) and the
        // 16-column chunks 16 h, 16 h + 32, ... with h = (w - 2) / 4
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        int i = 0;
        for (long long q = q0; q < q1; ++q, ++i) {
            const int blk = i & (NB - 1);
            const FwdRow r = fwd_row(q, a.N, a.H);
            const int p = r.wt * kM + quarter * 32 + lane;  // this thread's pixel
            const size_t ybase = (((size_t)r.n * a.H + r.h) * a.W + p) * a.Cout + co0;
            // the residual and mask of this thread's first two chunks do not depend on the
            // accumulator: load them before waiting for it
            float rv[2][16], mv[2][16];
            const bool pix = p < a.W;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int j0 = half * 16 + 32 * c;
                if (pix && j0 < nt) {
                    if (a.residual) load_bf16x16(a.residual + ybase + j0, rv[c]);
                    if (a.mask) load_bf16x16(a.mask + ybase + j0, mv[c]);
                }
            }
            if (!__all_sync(0xffffffffu, fwd_wait(&bfull[blk], (uint32_t)((i / NB) & 1), abort_word))) {
                if (lane == 0) {
                    *abort_word = 1;
                    atomicExch(a.err, 1);
                }
                break;
            }
            tc_fence_after();
            const uint32_t tcol = taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((NB - 1 - blk) * nco);
            uint32_t z[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) z[k] = 0u;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int j0 = half * 16 + 32 * c;
                if (j0 < nco) {
                    uint32_t v32[16];
                    tmem_ld16(tcol + (uint32_t)j0, v32);
                    tmem_st16(tcol + (uint32_t)j0, z);  // the block starts the next row at zero
                    if (pix && j0 < nt) {
                        float v[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(v32[j]) + s_bias[j0 + j];
                        epilogue16_loaded(v, a.residual ? rv[c] : nullptr, a.mask ? mv[c] : nullptr, a.relu,
                                          a.Y + ybase + j0);
                    }
                }
            }
            for (int j0 = half * 16 + 64; j0 < nco; j0 += 32) {
                uint32_t v32[16];
                tmem_ld16(tcol + (uint32_t)j0, v32);
                tmem_st16(tcol + (uint32_t)j0, z);
                if (pix && j0 < nt) {
                    float v[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(v32[j]) + s_bias[j0 + j];
                    epilogue16(v, a.residual ? a.residual + ybase + j0 : nullptr, a.mask ? a.mask + ybase + j0 : nullptr,
                               a.relu, a.Y + ybase + j0);
                }
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive1(&bempty[blk]);
        }
    }
    __syncthreads();
    // drain: the MMAs (fin) and every TMA copy still in flight, bounded, before TMEM and
    // shared memory are given up
    if (warp == 1 && lane == 0) {
        bool done = false;
        for (long long k = 0; k < kWaitPolls && !done; ++k) done = mbar_try_wait(fin, 0);
        if (!done) atomicExch(a.err, 1);
    }
    if (warp == 0 && lane == 0) {
        const long long from = loads > ring ? loads - ring : 0;
        for (long long l = from; l < loads; ++l) {
            bool done = false;
            for (long long k = 0; k < kWaitPolls && !done; ++k) done = mbar_try_wait(&full[l % ring], (uint32_t)((l / ring) & 1));
            if (!done) atomicExch(a.err, 1);
        }
        bool wdone = false;
        for (long long k = 0; k < kWaitPolls && !wdone; ++k) wdone = mbar_try_wait(wfull, 0);
        if (!wdone) atomicExch(a.err, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(taddr, 512);
}


// ------------------------------------------------------------------ weight gradients
//
// dW[co][r][s][ci] = sum over images n, output rows h, pixels w of
//                    dY[n][h][w][co] X[n][h + r - 1][w + s - 1][ci]       (zero off the image)
// regrouped by input row j = h + r - 1: input row j meets output rows j + 1, j, j - 1 through
// row taps r = 0, 1, 2. Per input row (a 128-pixel segment), the CTA stages with TMA the X row
// (kCols pixels, w0-1 .. w0+128) and the three dY rows j-1, j+1, j (one 64-channel block of
// dY: a tile of 64 output channels), all 128-byte swizzled, and the tensor cores read them as
// MN-major operands -- the NHWC rows as they are, no transposition:
//   A (M = 128, K = 16 pixels) = [dY row j+1 ; dY row j]   or   [dY row j-1 ; dY row j+1]
//       (two 64-channel blocks, byte offset between them (LBO) = one dY slot)
//   B (N = 192, K = 16 pixels) = the X row from pixel s, s = 0, 1, 2
//       (three 64-channel blocks 128 bytes apart: block s starts s pixels later)
// so D1[(r, co)][(s, ci)] (r = 0 in lanes 0-63, r = 1 in lanes 64-127) and D2 (r = 2 in lanes
// 0-63; lanes 64-127 repeat r = 0 and are not read) accumulate every tap of the CTA's rows:
// per 16 pixels two MMAs of N = 192. The epilogue writes the CTA's FP32 partial sums
// part[split][co][tap][ci]; a second pass adds them over the splits in a fixed order.
// The epilogue warps, idle until then, also sum each staged dY row j over its pixels (the
// bias gradient; each output row is row j of exactly one input row).
// Requires Cin = 64 and Cout a multiple of 64 (tiles of 64 output channels).
constexpr int kWRThreads = 192;
constexpr int kWRYBytes = kM * 128;                       // one staged dY row block (128 px x 64 ch)
constexpr int kWRTile = kSwBlockBytes + 3 * kWRYBytes;    // X row + 3 dY rows
__host__ __device__ constexpr int bwdw_rows_smem_bytes(int ring) { return 1024 + ring * kWRTile + 512 + 128 * 4; }

struct BwdwArgs {
    float* part;              // [splits][Cout][9][64] partial sums
    float* bias_part;         // [splits][Cout] partial bias gradients
    int N, H, W, Cout;
    int ring;                 // staged row tiles (>= 2)
    int ctas_per_tile;        // CTAs (splits) per 64-channel output tile
    int* err;
};

__device__ __forceinline__ uint64_t smem_desc_sw128_mn(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// X map: (64 channels, W, H, N), box (64, kCols, 1, 1); dY map: (Cout, W, H, N), box (64, 128, 1, 1);
// both 128-byte swizzled. Grid: Cout/64 tiles x ctas_per_tile; kWRThreads threads.
__global__ void __launch_bounds__(kWRThreads, 1) conv3x3_bwdw_rows_kernel(const __grid_constant__ CUtensorMap xmap,
                                                                          const __grid_constant__ CUtensorMap ymap,
                                                                          BwdwArgs a) {
    extern __shared__ __align__(128) unsigned char sm_raw[];
    unsigned char* sm = sm_raw + ((1024 - (smem_u32(sm_raw) & 1023)) & 1023);
    const int ring = a.ring;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + ring * kWRTile);  // [kFRingMax]
    uint64_t* empty = full + kFRingMax;                                 // [kFRingMax]
    uint64_t* fin = empty + kFRingMax;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
    volatile int* abort_word = reinterpret_cast<volatile int*>(tslot + 1);
    float* s_bias = reinterpret_cast<float*>(sm + ring * kWRTile + 512);  // [128] bias halves

    const int tile = blockIdx.x / a.ctas_per_tile, split = blockIdx.x - tile * a.ctas_per_tile;
    const int co0 = tile * 64;
    const int w_tiles = (a.W + kM - 1) / kM;
    const long long T = (long long)w_tiles * a.N * a.H;
    const long long q0 = T * split / a.ctas_per_tile, q1 = T * (split + 1) / a.ctas_per_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) tmem_alloc(tslot, 512);
    if (threadIdx.x == 0) {
        for (int s = 0; s < ring; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 5);  // the MMAs' commit and the four bias warps
        }
        mbar_init(fin, 1);
        *abort_word = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = *tslot;
    long long loads = 0;

    if (warp == 0) {
        if (lane == 0) {
            for (long long q = q0; q < q1 && !*abort_word; ++q) {
                const FwdRow r = fwd_row(q, a.N, a.H);
                const int s = (int)(loads % ring);
                if (loads >= ring && !fwd_wait(&empty[s], (uint32_t)((loads / ring - 1) & 1), abort_word)) break;
                mbar_arrive_tx(&full[s], (uint32_t)(fwd_row_bytes(64) + 3 * kWRYBytes));
                unsigned char* t = sm + (size_t)s * kWRTile;
                tma_load_4d(t, &xmap, 0, r.wt * kM - 1, r.h, r.n, &full[s]);
                // dY slots in the order j-1, j+1, j (A pairs: [j+1 ; j] and [j-1 ; j+1])
                tma_load_4d(t + kSwBlockBytes, &ymap, co0, r.wt * kM, r.h - 1, r.n, &full[s]);
                tma_load_4d(t + kSwBlockBytes + kWRYBytes, &ymap, co0, r.wt * kM, r.h + 1, r.n, &full[s]);
                tma_load_4d(t + kSwBlockBytes + 2 * kWRYBytes, &ymap, co0, r.wt * kM, r.h, r.n, &full[s]);
                ++loads;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // F32 accumulate, BF16 A and B, both MN-major, N = 192, M = 128
            const uint32_t idesc = idesc_bf16(kM, 192) | (1u << 15) | (1u << 16);
            bool ok = true;
            long long l = 0;
            for (long long q = q0; q < q1 && ok; ++q, ++l) {
                ok = fwd_wait(&full[l % ring], (uint32_t)((l / ring) & 1), abort_word);
                if (!ok) break;
                tc_fence_after();
                const uint32_t t = smem_u32(sm) + (uint32_t)((l % ring) * kWRTile);
                const uint32_t xs = t, ys = t + kSwBlockBytes;
#pragma unroll
                for (int k = 0; k < kM / 16; ++k) {
                    const uint64_t b = smem_desc_sw128_mn(xs + k * 2048, 128, 1024);
                    const uint64_t a1 = smem_desc_sw128_mn(ys + kWRYBytes + k * 2048, kWRYBytes, 1024);
                    const uint64_t a2 = smem_desc_sw128_mn(ys + k * 2048, kWRYBytes, 1024);
                    const uint32_t acc = (q > q0 || k > 0) ? 1u : 0u;
                    mma_bf16(taddr, a1, b, idesc, acc);
                    mma_bf16(taddr + 192, a2, b, idesc, acc);
                }
                mma_commit(&empty[l % ring]);
            }
            if (!ok) atomicExch(a.err, 1);
            mma_commit(fin);
        }
    } else {
        // bias: thread t sums channel t & 63 of the staged dY row j over pixels 64 (t >> 6) .. +63
        const int t = threadIdx.x - 64, c = t & 63, p0 = (t >> 6) * 64;
        float bsum = 0.f;
        long long l = 0;
        bool ok = true;
        for (long long q = q0; q < q1; ++q, ++l) {
            ok = __all_sync(0xffffffffu, fwd_wait(&full[l % ring], (uint32_t)((l / ring) & 1), abort_word));
            if (!ok) break;
            const unsigned char* y = sm + (size_t)(l % ring) * kWRTile + kSwBlockBytes + 2 * kWRYBytes;
#pragma unroll 8
            for (int p = p0; p < p0 + 64; ++p) {
                // 128-byte swizzle: 16-byte chunk (c / 8) of pixel row p sits at chunk (c / 8) ^ (p % 8)
                const unsigned off = (unsigned)p * 128u + ((((unsigned)c >> 3) ^ ((unsigned)p & 7u)) << 4) + ((unsigned)c & 7u) * 2u;
                bsum += __bfloat162float(*reinterpret_cast<const bf16*>(y + off));
            }
            __syncwarp();
            if (lane == 0) mbar_arrive1(&empty[l % ring]);
        }
        if (!ok && lane == 0) {
            *abort_word = 1;
            atomicExch(a.err, 1);
        }
        // the accumulators are final once every MMA has completed
        const bool done = ok && __all_sync(0xffffffffu, fwd_wait(fin, 0, abort_word));
        tc_fence_after();
        const int quarter = warp & 3, row = quarter * 32 + lane;
        const int co = co0 + (row & 63);
        float* P = a.part + ((size_t)split * a.Cout + co) * 9 * 64;
        // D1: lanes 0-63 tap row r = 0, 64-127 r = 1; D2: lanes 0-63 r = 2
        for (int d = 0; d < 2; ++d) {
            const int r = d == 0 ? (row >> 6) : 2;
            for (int j0 = 0; j0 < 192; j0 += 16) {
                uint32_t v[16];
                tmem_ld16(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(d * 192 + j0), v);
                if (done && (d == 0 || row < 64)) {
                    float4* o = reinterpret_cast<float4*>(P + r * 192 + j0);  // taps r*3 + s, s = j0 / 64
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        o[e] = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                                           __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
                }
            }
        }
        s_bias[t] = bsum;
        asm volatile("bar.sync 1, 128;" ::: "memory");  // the four bias warps
        if (t < 64 && done) a.bias_part[(size_t)split * a.Cout + co0 + t] = s_bias[t] + s_bias[t + 64];
        if (!done && lane == 0) atomicExch(a.err, 1);
    }
    __syncthreads();
    if (warp == 1 && lane == 0) {
        bool done = false;
        for (long long k = 0; k < kWaitPolls && !done; ++k) done = mbar_try_wait(fin, 0);
        if (!done) atomicExch(a.err, 1);
    }
    if (warp == 0 && lane == 0) {
        const long long from = loads > ring ? loads - ring : 0;
        for (long long l = from; l < loads; ++l) {
            bool done = false;
            for (long long k = 0; k < kWaitPolls && !done; ++k) done = mbar_try_wait(&full[l % ring], (uint32_t)((l / ring) & 1));
            if (!done) atomicExch(a.err, 1);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(taddr, 512);
}

}  // namespace pit_tc
