// pit_net.cu -- the learned initial guess: a small residual conv net that maps
// (u^0, log10 nu) on the grid to the corrections u^n - u^0 of all M levels, used as
// the starting iterate of Newton in place of the plain guess u^n = u^0.
//
//   z0 = conv(in); x = relu(z0); per block: h = relu(conv(x)); x = x + conv(h);
//   out = conv(x)                                   (3x3 convs, zero padding, bias)
//
// Activations are BF16 NHWC, weights BF16 [Cout][9][Cin] with FP32 master copies,
// products accumulate in FP32 on the tensor cores: the convolutions (forward, and data
// gradients through the same kernel on flipped, transposed weights) and the weight
// gradients (split over pixels, deterministic two-pass reduction) are tcgen05 GEMMs with
// TMEM accumulators (pit_tc.cuh). The input
// has 2 channels, padded to 16 for the tensor-core K step. Training: MSE loss, manual
// backward, Adam on the FP32 masters.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "pit.h"
#include "pit_conv_tma.cuh"
#include "pit_tc.cuh"

namespace {

typedef __nv_bfloat16 bf16;
constexpr int kCinPad0 = 64;   // input channels padded to one 64-channel block (the TMA convolutions' unit)
constexpr int kMaxSplits = 160;  // pixel splits of the weight-gradient GEMMs, at most

// Sum the split partials (deterministic): a CTA takes 64 outputs; thread group g (of four)
// adds splits g, g + 4, ... in order, and the four sums are added in group order.
__global__ void __launch_bounds__(256) sum_partials_kernel(const float* __restrict__ part, float* __restrict__ out,
                                                           int splits, size_t n) {
    __shared__ float red[4][64];
    const int o = threadIdx.x & 63, g = threadIdx.x >> 6;
    const size_t i = (size_t)blockIdx.x * 64 + o;
    float s = 0.f;
    if (i < n) {
#pragma unroll 8
        for (int k = g; k < splits; k += 4) s += __ldg(part + (size_t)k * n + i);
    }
    red[g][o] = s;
    __syncthreads();
    if (g == 0 && i < n) out[i] = ((red[0][o] + red[1][o]) + red[2][o]) + red[3][o];
}
static int sum_partials_grid(size_t n) { return (int)((n + 63) / 64); }

// out[c] = sum over k of part[k][c] for few columns c and many rows k: one CTA per column,
// threads take rows in a fixed stride and fold in a fixed tree (deterministic).
__global__ void __launch_bounds__(256) sum_rows_kernel(const float* __restrict__ part, float* __restrict__ out,
                                                       int rows, int cols) {
    __shared__ float red[256];
    const int c = blockIdx.x;
    float s = 0.f;
#pragma unroll 4
    for (int k = threadIdx.x; k < rows; k += 256) s += __ldg(part + (size_t)k * cols + c);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
}

// Bias gradient, first pass: CTA b sums dY[pix][o] over its range of pixels for every
// channel o (threads: pixel lanes x channels, so reads are coalesced), lanes folded in a
// fixed order; part[b][o]. The second pass (sum_partials_kernel) adds the CTAs in order.
constexpr int kBiasBlocks = 2048;
__global__ void __launch_bounds__(256) bias_grad_partial_kernel(const bf16* __restrict__ dY, float* __restrict__ part,
                                                                size_t pixels, int Cout, size_t per_block) {
    __shared__ float red[256];
    const size_t p0 = (size_t)blockIdx.x * per_block;
    const size_t p1 = p0 + per_block < pixels ? p0 + per_block : pixels;
    for (int c0 = 0; c0 < Cout; c0 += 256) {
        const int cw = Cout - c0 < 256 ? Cout - c0 : 256;
        const int lanes = 256 / cw;
        const int c = threadIdx.x % cw, pl = threadIdx.x / cw;
        float acc = 0.f;
        if (pl < lanes) {
#pragma unroll 8
            for (size_t p = p0 + pl; p < p1; p += lanes) acc += __bfloat162float(dY[p * Cout + c0 + c]);
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        if (threadIdx.x < cw) {
            float t = 0.f;
            for (int l = 0; l < lanes; ++l) t += red[l * cw + threadIdx.x];
            part[(size_t)blockIdx.x * Cout + c0 + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

// W'[c][8 - tap][o] = W[o][tap][c]: the weights of the data-gradient convolution.
__global__ void flip_transpose_kernel(const bf16* __restrict__ Wt, bf16* __restrict__ Wf, int Cout, int Cin) {
    const size_t n = (size_t)Cout * 9 * Cin;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % Cin);
        const int tap = (int)((i / Cin) % 9);
        const int o = (int)(i / ((size_t)9 * Cin));
        Wf[((size_t)c * 9 + (8 - tap)) * Cout + o] = Wt[i];
    }
}

// d *= (act > 0): back through a ReLU whose output was act.
__global__ void relu_back_kernel(bf16* __restrict__ d, const bf16* __restrict__ act, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(act[i]) > 0.f)) d[i] = __float2bfloat16(0.f);
}

// Network input: channel 0 = u0, channel 1 = log10 nu, channels 2..kCinPad0-1 = 0; one
// pixel's kCinPad0 channels written as 16-byte words.
__global__ void input_kernel(const double* __restrict__ u0, const float* __restrict__ lognu, bf16* __restrict__ X,
                             int N, size_t Ns) {
    static_assert(kCinPad0 % 8 == 0, "whole 16-byte words per pixel");
    const size_t n_total = (size_t)N * Ns;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_total; i += (size_t)gridDim.x * blockDim.x) {
        const int n = (int)(i / Ns);
        uint4* x = reinterpret_cast<uint4*>(X + i * kCinPad0);
        const uint32_t w0 = (uint32_t)__bfloat16_as_ushort(__float2bfloat16((float)u0[i])) |
                            ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(lognu[n])) << 16);
        x[0] = make_uint4(w0, 0u, 0u, 0u);
#pragma unroll
        for (int k = 1; k < kCinPad0 / 8; ++k) x[k] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// U_init[n][m][pix] = u0[n][pix] + out[n][pix][m] (solver layout, FP64).
__global__ void output_kernel(const bf16* __restrict__ out, const double* __restrict__ u0, double* __restrict__ U,
                              int N, int M, size_t Ns) {
    const size_t total = (size_t)N * M * Ns;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t pix = i % Ns;
        const int m = (int)((i / Ns) % M);
        const int n = (int)(i / (Ns * M));
        U[i] = u0[(size_t)n * Ns + pix] + (double)__bfloat162float(out[((size_t)n * Ns + pix) * M + m]);
    }
}

// Training target of one solution: T[pix][m] = U[m][pix] - u0[pix] in BF16.
__global__ void target_kernel(const double* __restrict__ U, const double* __restrict__ u0, bf16* __restrict__ T,
                              int M, size_t Ns) {
    const size_t total = (size_t)M * Ns;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i % M);
        const size_t pix = i / M;
        T[i] = __float2bfloat16((float)(U[(size_t)m * Ns + pix] - u0[pix]));
    }
}

// dout = 2 (out - target) / count and per-CTA partial sums of (out - target)^2.
__global__ void mse_kernel(const bf16* __restrict__ out, const bf16* __restrict__ target, bf16* __restrict__ dout,
                           float* __restrict__ partial, size_t n, float scale, int vec) {
    __shared__ float red[256];
    float s = 0.f;
    // eight values (16 bytes) per step when every buffer is 16-byte aligned (vec); the rest
    // one by one
    const size_t n8 = vec ? n / 8 : 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n8; k += stride) {
        const uint4 uo = reinterpret_cast<const uint4*>(out)[k], ut = reinterpret_cast<const uint4*>(target)[k];
        const unsigned wo[4] = {uo.x, uo.y, uo.z, uo.w}, wt[4] = {ut.x, ut.y, ut.z, ut.w};
        unsigned wd[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float d0 = __bfloat162float(__ushort_as_bfloat16((unsigned short)(wo[e] & 0xffff))) -
                             __bfloat162float(__ushort_as_bfloat16((unsigned short)(wt[e] & 0xffff)));
            const float d1 = __bfloat162float(__ushort_as_bfloat16((unsigned short)(wo[e] >> 16))) -
                             __bfloat162float(__ushort_as_bfloat16((unsigned short)(wt[e] >> 16)));
            s += d0 * d0 + d1 * d1;
            wd[e] = (unsigned)__bfloat16_as_ushort(__float2bfloat16(2.f * d0 * scale)) |
                    ((unsigned)__bfloat16_as_ushort(__float2bfloat16(2.f * d1 * scale)) << 16);
        }
        reinterpret_cast<uint4*>(dout)[k] = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    }
    for (size_t i = n8 * 8 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float d = __bfloat162float(out[i]) - __bfloat162float(target[i]);
        s += d * d;
        dout[i] = __float2bfloat16(2.f * d * scale);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// Adam on the FP32 masters (bias-corrected), then refresh the BF16 weights.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ a, bf16* __restrict__ b, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16(a[i]);
}

int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

}  // namespace

// ------------------------------------------------------------------ the network

struct Layer {
    int cin, cout;          // cin as stored (input layer padded to 16)
    int cin_public;         // cin in the public parameter layout
    size_t w_off, b_off;    // offsets of weights [cout][9][cin] and bias in the FP32 master buffer
};

struct pit_net {
    pit_net_shape shape{};
    cudaStream_t stream = nullptr;
    std::vector<Layer> layers;
    size_t nparam = 0;       // stored parameters (padded input layer)
    size_t nparam_public = 0;
    float* p = nullptr;      // FP32 masters
    float* g = nullptr;      // gradients
    float* m = nullptr;
    float* v = nullptr;
    bf16* wb = nullptr;      // BF16 weights (same offsets)
    bf16* wf = nullptr;      // flipped/transposed weights of one layer (scratch)
    float* part = nullptr;   // split partials of the weight gradient
    size_t part_n = 0;
    float* loss_part = nullptr;
    int step = 0;
    // activations for max_batch images
    bf16* in = nullptr;                 // [B][H][W][16]
    std::vector<bf16*> xs;              // x after the lift and after each block: blocks + 1
    std::vector<bf16*> hs;              // h inside each block
    bf16* out = nullptr;                // [B][H][W][M]
    bf16* d0 = nullptr;                 // gradient buffers
    bf16* d1 = nullptr;
    bf16* d2 = nullptr;
    bf16* dout = nullptr;
    float* lognu = nullptr;
    int* tc_err = nullptr;   // raised by a tensor-core conv whose mbarrier wait timed out
    float* bias_part = nullptr;  // [kBiasBlocks][max channels] bias-gradient partials
    char err[512] = "";
};

static pit_status nfail(pit_net* net, pit_status s, const char* fmt, ...) {
    if (net) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(net->err, sizeof(net->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define NCK(call)                                                                                            \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess)                                                                               \
            return nfail(net, e_ == cudaErrorMemoryAllocation ? PIT_ENOMEM : PIT_ECUDA, "%s: %s (%s:%d)", #call, \
                         cudaGetErrorString(e_), __FILE__, __LINE__);                                        \
    } while (0)

extern "C" long long pit_net_param_count(const pit_net_shape* s) {
    if (!s) return -1;
    const long long C = s->channels, M = s->levels;
    return (C * 9 * 2 + C) + 2LL * s->blocks * (C * 9 * C + C) + (M * 9 * C + M);
}

// ------------------------------------------------- TMA tensor maps (driver entry point)

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda);
// null when the CUDA driver does not offer it.
static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Maps of the TMA convolution (pit_conv_tma.cuh): activations [B][H][W][Cin] as (8 channels,
// W, Cin/8, H, B) with box (8, 130, Cin/8, 1, 1), weights [Cout][9][Cin] as (8 channels, Cout,
// Cin/8, 9) with box (8, nco, Cin/8, 9). Off-tensor elements read as zero.
static bool encode_conv_maps(CUtensorMap* xm, CUtensorMap* wm, const bf16* X, const bf16* Wt, int B, int H, int W,
                             int Cin, int Cout, int nco, int sw) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t G = (cuuint64_t)(Cin / 8), cb = (cuuint64_t)Cin * 2;
    const cuuint32_t ones[5] = {1, 1, 1, 1, 1};
    if (sw) {
        // rows of 64 channels (128 bytes), contiguous in NHWC: 128-byte swizzle
        const cuuint64_t xdim[4] = {(cuuint64_t)Cin, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        const cuuint64_t xstr[3] = {cb, cb * W, cb * W * H};
        const cuuint32_t xbox[4] = {64, (cuuint32_t)pit_tc::kCols, 1, 1};
        if (enc(xm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(X), xdim, xstr, xbox, ones,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    } else {
        const cuuint64_t xdim[5] = {8, (cuuint64_t)W, G, (cuuint64_t)H, (cuuint64_t)B};
        const cuuint64_t xstr[4] = {cb, 16, cb * W, cb * W * H};
        const cuuint32_t xbox[5] = {8, (cuuint32_t)pit_tc::kCols, (cuuint32_t)G, 1, 1};
        if (enc(xm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<bf16*>(X), xdim, xstr, xbox, ones,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    if (sw) {
        // [Cout][9][Cin] as (Cin, 9, Cout): a box is 64 channels of one tap for nco outputs
        const cuuint64_t wdim[3] = {(cuuint64_t)Cin, 9, (cuuint64_t)Cout};
        const cuuint64_t wstr[2] = {cb, 9 * cb};
        const cuuint32_t wbox[3] = {64, 1, (cuuint32_t)nco};
        return enc(wm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(Wt), wdim, wstr, wbox, ones,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    const cuuint64_t wdim[4] = {8, (cuuint64_t)Cout, G, 9};
    const cuuint64_t wstr[3] = {9 * cb, 16, cb};
    const cuuint32_t wbox[4] = {8, (cuuint32_t)nco, (cuuint32_t)G, 9};
    return enc(wm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(Wt), wdim, wstr, wbox, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

constexpr int kConvSmemLimit = 227 * 1024;

// An NHWC activation [B][H][W][C] as (C, W, H, B) with 128-byte-swizzled boxes of 64
// channels x box_w pixels (one image row segment).
static bool encode_rows_map(CUtensorMap* m, const bf16* base, int B, int H, int W, int C, int box_w) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
    const cuuint64_t cb = (cuuint64_t)C * 2;
    const cuuint64_t dim[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t str[3] = {cb, cb * W, cb * W * H};
    const cuuint32_t box[4] = {64, (cuuint32_t)box_w, 1, 1};
    const cuuint32_t ones[4] = {1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(base), dim, str, box, ones,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The row-stationary TMA convolution (Cin = 64 or 128, weights and two staged rows fit in
// shared memory); false = not applicable.
static bool launch_conv_rows(pit_net* net, const bf16* X, const bf16* Wt, const float* bias, const bf16* res,
                             const bf16* mask, bf16* Y, int B, int H, int W, int Cin, int Cout, int relu,
                             cudaError_t* cerr) {
    *cerr = cudaSuccess;
    if (Cin != 64 && Cin != 128) return false;
    const int nco = Cout < 128 ? Cout : 128;
    // four staged rows measured fastest (2: 1.346, 3: 1.336, 4: 1.331, 6: 1.351, 8: 1.376 ms
    // per training step of the 64-channel network on 16 images of 128 x 128)
    int ring = 4;
    while (ring >= 2 && pit_tc::fwd_smem_bytes(Cin, nco, ring, 1) > kConvSmemLimit) --ring;
    if (ring < 2 || (reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(Wt) & 15)) return false;
    CUtensorMap xm, wm;
    if (!encode_conv_maps(&xm, &wm, X, Wt, B, H, W, Cin, Cout, nco, 1)) return false;
    static int sms = 0;
    static bool attr_set = false;  // the limit belongs to the kernel; raising it again is harmless
    if (!attr_set) {
        int dev = 0;
        if ((*cerr = cudaGetDevice(&dev)) != cudaSuccess) return true;
        if ((*cerr = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return true;
        if ((*cerr = cudaFuncSetAttribute(pit_tc::conv3x3_fwd_rows_kernel<1>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmemLimit)) != cudaSuccess)
            return true;
        if ((*cerr = cudaFuncSetAttribute(pit_tc::conv3x3_fwd_rows_kernel<2>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmemLimit)) != cudaSuccess)
            return true;
        attr_set = true;
    }
    const int co_tiles = (Cout + nco - 1) / nco;
    const long long rows = (long long)((W + pit_tc::kM - 1) / pit_tc::kM) * B * H;
    const int per = (int)std::max(1LL, std::min((long long)std::max(1, sms / co_tiles), rows));
    pit_tc::FwdTmaArgs a;
    a.bias = bias;
    a.residual = res;
    a.mask = mask;
    a.Y = Y;
    a.N = B;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    a.Cout = Cout;
    a.relu = relu;
    a.nco = nco;
    a.ntp = 0;
    a.ring = ring;
    a.ctas_per_tile = per;
    a.sw = 1;
    a.err = net->tc_err;
    const int smem = pit_tc::fwd_smem_bytes(Cin, nco, ring, 1);
    if (Cin == 64)
        pit_tc::conv3x3_fwd_rows_kernel<1><<<co_tiles * per, pit_tc::kRThreads, smem, net->stream>>>(xm, wm, a);
    else
        pit_tc::conv3x3_fwd_rows_kernel<2><<<co_tiles * per, pit_tc::kRThreads, smem, net->stream>>>(xm, wm, a);
    *cerr = cudaGetLastError();
    return true;
}

// The TMA convolution when the layer's weight tile and a ring of at least four input rows
// fit in shared memory (and the maps encode); false = use the staged kernel.
static bool launch_conv_tma(pit_net* net, const bf16* X, const bf16* Wt, const float* bias, const bf16* res,
                            const bf16* mask, bf16* Y, int B, int H, int W, int Cin, int Cout, int relu,
                            cudaError_t* cerr) {
    *cerr = cudaSuccess;
    if (launch_conv_rows(net, X, Wt, bias, res, mask, Y, B, H, W, Cin, Cout, relu, cerr)) return true;
    const int nco = Cout < pit_tc::kFNMax ? Cout : pit_tc::kFNMax;
    const int sw = Cin % 64 == 0 ? 1 : 0;
    int ring = pit_tc::kFRingMax;
    while (ring >= 4 && pit_tc::fwd_smem_bytes(Cin, nco, ring, sw) > kConvSmemLimit) --ring;
    if (ring < 4 || (reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(Wt) & 15)) return false;
    CUtensorMap xm, wm;
    if (!encode_conv_maps(&xm, &wm, X, Wt, B, H, W, Cin, Cout, nco, sw)) return false;
    static int sms = 0;
    static bool attr_set = false;  // the limit belongs to the kernel; raising it again is harmless
    if (!attr_set) {
        int dev = 0;
        if ((*cerr = cudaGetDevice(&dev)) != cudaSuccess) return true;
        if ((*cerr = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return true;
        if ((*cerr = cudaFuncSetAttribute(pit_tc::conv3x3_fwd_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          kConvSmemLimit)) != cudaSuccess)
            return true;
        attr_set = true;
    }
    const int co_tiles = (Cout + nco - 1) / nco;
    const long long rows = (long long)((W + pit_tc::kM - 1) / pit_tc::kM) * B * H;
    const int per = (int)std::max(1LL, std::min((long long)std::max(1, sms / co_tiles), rows));
    pit_tc::FwdTmaArgs a;
    a.bias = bias;
    a.residual = res;
    a.mask = mask;
    a.Y = Y;
    a.N = B;
    a.H = H;
    a.W = W;
    a.Cin = Cin;
    a.Cout = Cout;
    a.relu = relu;
    a.nco = nco;
    a.ntp = nco <= 32 ? 32 : (nco <= 64 ? 64 : (nco <= 128 ? 128 : 256));
    a.ring = ring;
    a.ctas_per_tile = per;
    a.sw = sw;
    a.err = net->tc_err;
    pit_tc::conv3x3_fwd_tma_kernel<<<co_tiles * per, pit_tc::kFThreads, pit_tc::fwd_smem_bytes(Cin, nco, ring, sw),
                                     net->stream>>>(xm, wm, a);
    *cerr = cudaGetLastError();
    return true;
}

// Y = act(conv3x3(X; Wt) + bias (+ res)) on the tcgen05 tensor cores: the TMA kernel
// (pit_conv_tma.cuh) when the layer fits it, else the staged kernel (pit_tc.cuh).
static pit_status launch_conv_tc(pit_net* net, const bf16* X, const bf16* Wt, const float* bias, const bf16* res,
                                 bf16* Y, int B, int Cin, int Cout, int relu, const bf16* mask = nullptr) {
    const pit_net_shape& s = net->shape;
    if (Cin % 16 != 0 || Cout % 16 != 0) return nfail(net, PIT_EINVAL, "conv channels must be multiples of 16");
    {
        cudaError_t e = cudaSuccess;
        if (launch_conv_tma(net, X, Wt, bias, res, mask, Y, B, s.height, s.width, Cin, Cout, relu, &e)) {
            NCK(e);
            return PIT_OK;
        }
    }
    static bool attr_set = false;  // the limit belongs to the kernel; raising it again is harmless
    if (!attr_set) {
        NCK(cudaFuncSetAttribute(pit_tc::conv3x3_fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 pit_tc::kSmemMax));
        attr_set = true;
    }
    const int smem = pit_tc::smem_bytes(Cout < pit_tc::kNMax ? Cout : pit_tc::kNMax);
    dim3 grid((unsigned)(B * ((s.height + pit_tc::kRows - 1) / pit_tc::kRows) * ((s.width + pit_tc::kM - 1) / pit_tc::kM)),
              (unsigned)((Cout + pit_tc::kNMax - 1) / pit_tc::kNMax));
    pit_tc::conv3x3_fwd_tc_kernel<<<grid, pit_tc::kThreads, smem, net->stream>>>(
        X, Wt, bias, res, mask, Y, B, s.height, s.width, Cin, Cout, relu, net->tc_err);
    NCK(cudaGetLastError());
    return PIT_OK;
}

static pit_status conv_fwd(pit_net* net, const bf16* X, const Layer& L, const bf16* res, bf16* Y, int B, int relu) {
    return launch_conv_tc(net, X, net->wb + L.w_off, net->p + L.b_off, res, Y, B, L.cin, L.cout, relu);
}

// A tensor-core conv that timed out on an mbarrier raises tc_err; report it (synchronises).
static pit_status check_tc(pit_net* net) {
    int flag = 0;
    NCK(cudaMemcpyAsync(&flag, net->tc_err, sizeof(int), cudaMemcpyDeviceToHost, net->stream));
    NCK(cudaStreamSynchronize(net->stream));
    if (flag) {
        NCK(cudaMemsetAsync(net->tc_err, 0, sizeof(int), net->stream));
        return nfail(net, PIT_ETIMEOUT, "tensor-core convolution: an mbarrier wait timed out");
    }
    return PIT_OK;
}

// dX = conv(dY, flipped W) without bias (+ dx_res, then zeroed where dx_mask <= 0: the
// residual branch's gradient and the backward ReLU, fused into the epilogue; dx_res may be
// dX itself); dW, db into net->g.
static pit_status conv_bwd(pit_net* net, const bf16* X, const bf16* dY, const Layer& L, bf16* dX, int B,
                           const bf16* dx_res = nullptr, const bf16* dx_mask = nullptr) {
    const pit_net_shape& s = net->shape;
    // the data-gradient convolution reads L.cout input channels in chunks of 16
    if (L.cin % 16 != 0 || L.cout % 16 != 0) return nfail(net, PIT_EINVAL, "conv channels must be multiples of 16");
    {
        // the MN-major TMA kernel (pit_conv_tma.cuh) for 64 input channels and 64k outputs
        CUtensorMap xm, ym;
        if (L.cin == 64 && L.cout % 64 == 0 &&
            encode_rows_map(&xm, X, B, s.height, s.width, 64, pit_tc::kCols) &&
            encode_rows_map(&ym, dY, B, s.height, s.width, L.cout, pit_tc::kM)) {
            static int sms = 0;
            static bool rattr = false;  // the limit belongs to the kernel; raising it again is harmless
            if (!rattr) {
                int dev = 0;
                NCK(cudaGetDevice(&dev));
                NCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
                NCK(cudaFuncSetAttribute(pit_tc::conv3x3_bwdw_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kConvSmemLimit));
                rattr = true;
            }
            const int co_tiles = L.cout / 64;
            const long long T = (long long)((s.width + pit_tc::kM - 1) / pit_tc::kM) * B * s.height;
            const int per = (int)std::max(1LL, std::min({(long long)std::max(1, sms / co_tiles), T, (long long)kMaxSplits}));
            pit_tc::BwdwArgs ba;
            ba.part = net->part;
            ba.bias_part = net->bias_part;
            ba.N = B;
            ba.H = s.height;
            ba.W = s.width;
            ba.Cout = L.cout;
            ba.ring = 3;
            ba.ctas_per_tile = per;
            ba.err = net->tc_err;
            pit_tc::conv3x3_bwdw_rows_kernel<<<co_tiles * per, pit_tc::kWRThreads, pit_tc::bwdw_rows_smem_bytes(3),
                                               net->stream>>>(xm, ym, ba);
            NCK(cudaGetLastError());
            const size_t nw = (size_t)L.cout * 9 * L.cin;
            sum_partials_kernel<<<sum_partials_grid(nw), 256, 0, net->stream>>>(net->part, net->g + L.w_off, per, nw);
            sum_rows_kernel<<<L.cout, 256, 0, net->stream>>>(net->bias_part, net->g + L.b_off, per, L.cout);
            if (dX) {
                flip_transpose_kernel<<<grid_for(nw), 256, 0, net->stream>>>(net->wb + L.w_off, net->wf, L.cout, L.cin);
                if (pit_status st = launch_conv_tc(net, dY, net->wf, net->loss_part + 1024, dx_res, dX, B, L.cout,
                                                   L.cin, 0, dx_mask))
                    return st;
            }
            NCK(cudaGetLastError());
            return PIT_OK;
        }
    }
    const int rows = B * s.height;
    // one CTA per split and channel tile pair, about one per SM
    const int tiles = ((L.cin + pit_tc::kWCi - 1) / pit_tc::kWCi) * ((L.cout + pit_tc::kWCo - 1) / pit_tc::kWCo);
    const int want = std::max(1, std::min(kMaxSplits, 148 / tiles));
    const int rows_per_split = std::max(1, (rows + want - 1) / want);
    const int splits = (rows + rows_per_split - 1) / rows_per_split;
    static bool wattr_set = false;  // the limit belongs to the kernel; raising it again is harmless
    if (!wattr_set) {
        NCK(cudaFuncSetAttribute(pit_tc::conv3x3_bwdw_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 pit_tc::kWSmemBytes));
        wattr_set = true;
    }
    dim3 grid((unsigned)splits, (unsigned)((L.cin + pit_tc::kWCi - 1) / pit_tc::kWCi),
              (unsigned)((L.cout + pit_tc::kWCo - 1) / pit_tc::kWCo));
    pit_tc::conv3x3_bwdw_tc_kernel<<<grid, pit_tc::kThreads, pit_tc::kWSmemBytes, net->stream>>>(
        X, dY, net->part, B, s.height, s.width, L.cin, L.cout, rows_per_split, net->tc_err);
    NCK(cudaGetLastError());
    const size_t nw = (size_t)L.cout * 9 * L.cin;
    sum_partials_kernel<<<sum_partials_grid(nw), 256, 0, net->stream>>>(net->part, net->g + L.w_off, splits, nw);
    {
        const size_t pixels = (size_t)B * s.height * s.width;
        const size_t per = (pixels + kBiasBlocks - 1) / kBiasBlocks;
        const int blocks = (int)((pixels + per - 1) / per);
        bias_grad_partial_kernel<<<blocks, 256, 0, net->stream>>>(dY, net->bias_part, pixels, L.cout, per);
        sum_rows_kernel<<<L.cout, 256, 0, net->stream>>>(net->bias_part, net->g + L.b_off, blocks, L.cout);
    }
    if (dX) {
        flip_transpose_kernel<<<grid_for(nw), 256, 0, net->stream>>>(net->wb + L.w_off, net->wf, L.cout, L.cin);
        // zero bias for the data gradient: the zero tail of the loss buffer
        if (pit_status st =
                launch_conv_tc(net, dY, net->wf, net->loss_part + 1024, dx_res, dX, B, L.cout, L.cin, 0, dx_mask))
            return st;
    }
    NCK(cudaGetLastError());
    return PIT_OK;
}

static pit_status forward(pit_net* net, const double* u0, const float* lognu_dev, int B) {
    const pit_net_shape& s = net->shape;
    const size_t Ns = (size_t)s.height * s.width;
    input_kernel<<<grid_for(B * Ns), 256, 0, net->stream>>>(u0, lognu_dev, net->in, B, Ns);
    NCK(cudaGetLastError());
    const int nb = s.blocks;
    if (pit_status st = conv_fwd(net, net->in, net->layers[0], nullptr, net->xs[0], B, 1)) return st;
    for (int k = 0; k < nb; ++k) {
        if (pit_status st = conv_fwd(net, net->xs[k], net->layers[1 + 2 * k], nullptr, net->hs[k], B, 1)) return st;
        if (pit_status st = conv_fwd(net, net->hs[k], net->layers[2 + 2 * k], net->xs[k], net->xs[k + 1], B, 0))
            return st;
    }
    return conv_fwd(net, net->xs[nb], net->layers.back(), nullptr, net->out, B, 0);
}

extern "C" pit_status pit_net_create(const pit_net_shape* shape, unsigned long long seed, void* stream,
                                     pit_net** out) {
    if (!out) return PIT_EINVAL;
    *out = nullptr;
    if (!shape || shape->height < 1 || shape->width < 1 || shape->levels < 1 || shape->levels > 4096 ||
        shape->channels < 16 || shape->channels % 16 != 0 || shape->channels > 4096 || shape->blocks < 0 ||
        shape->max_batch < 1 || shape->levels % 16 != 0)
        return PIT_EINVAL;
    pit_net* net = new (std::nothrow) pit_net();
    if (!net) return PIT_ENOMEM;
    net->shape = *shape;
    net->stream = static_cast<cudaStream_t>(stream);
    const int C = shape->channels, M = shape->levels;
    auto add = [&](int cin, int cout, int cin_pub) {
        Layer L;
        L.cin = cin;
        L.cout = cout;
        L.cin_public = cin_pub;
        L.w_off = net->nparam;
        net->nparam += (size_t)cout * 9 * cin;
        L.b_off = net->nparam;
        net->nparam += cout;
        net->layers.push_back(L);
    };
    add(kCinPad0, C, 2);
    for (int k = 0; k < shape->blocks; ++k) {
        add(C, C, C);
        add(C, C, C);
    }
    add(C, M, C);
    net->nparam_public = (size_t)pit_net_param_count(shape);
    auto setup = [&]() -> pit_status {
        const size_t B = shape->max_batch, Ns = (size_t)shape->height * shape->width;
        NCK(cudaMalloc(&net->p, sizeof(float) * net->nparam));
        NCK(cudaMalloc(&net->g, sizeof(float) * net->nparam));
        NCK(cudaMalloc(&net->m, sizeof(float) * net->nparam));
        NCK(cudaMalloc(&net->v, sizeof(float) * net->nparam));
        NCK(cudaMalloc(&net->wb, sizeof(bf16) * net->nparam));
        size_t wmax = 0;
        for (auto& L : net->layers) wmax = std::max(wmax, (size_t)L.cout * 9 * L.cin);
        NCK(cudaMalloc(&net->wf, sizeof(bf16) * wmax));
        net->part_n = (size_t)kMaxSplits * wmax;
        NCK(cudaMalloc(&net->part, sizeof(float) * net->part_n));
        NCK(cudaMalloc(&net->loss_part, sizeof(float) * (1024 + 4096)));
        NCK(cudaMalloc(&net->tc_err, sizeof(int)));
        NCK(cudaMalloc(&net->bias_part, sizeof(float) * kBiasBlocks * std::max<size_t>(C, M)));
        NCK(cudaMemsetAsync(net->tc_err, 0, sizeof(int), net->stream));
        NCK(cudaMemsetAsync(net->loss_part, 0, sizeof(float) * (1024 + 4096), net->stream));
        NCK(cudaMalloc(&net->in, sizeof(bf16) * B * Ns * kCinPad0));
        for (int k = 0; k <= shape->blocks; ++k) {
            bf16* x;
            NCK(cudaMalloc(&x, sizeof(bf16) * B * Ns * C));
            net->xs.push_back(x);
        }
        for (int k = 0; k < shape->blocks; ++k) {
            bf16* hbuf;
            NCK(cudaMalloc(&hbuf, sizeof(bf16) * B * Ns * C));
            net->hs.push_back(hbuf);
        }
        const size_t cm = std::max<size_t>(C, M);
        NCK(cudaMalloc(&net->out, sizeof(bf16) * B * Ns * M));
        NCK(cudaMalloc(&net->dout, sizeof(bf16) * B * Ns * M));
        NCK(cudaMalloc(&net->d0, sizeof(bf16) * B * Ns * cm));
        NCK(cudaMalloc(&net->d1, sizeof(bf16) * B * Ns * cm));
        NCK(cudaMalloc(&net->d2, sizeof(bf16) * B * Ns * std::max<size_t>(cm, kCinPad0)));
        NCK(cudaMalloc(&net->lognu, sizeof(float) * B));
        // He-normal init (seeded) for hidden layers, zero head: the untrained net predicts
        // zero corrections, i.e. the plain guess
        std::vector<float> h(net->nparam, 0.f);
        std::mt19937_64 rng(seed);
        for (size_t li = 0; li < net->layers.size(); ++li) {
            const Layer& L = net->layers[li];
            if (li + 1 == net->layers.size()) break;
            std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (9.f * L.cin_public)));
            for (int o = 0; o < L.cout; ++o)
                for (int t = 0; t < 9; ++t)
                    for (int c = 0; c < L.cin; ++c)
                        h[L.w_off + ((size_t)o * 9 + t) * L.cin + c] = c < L.cin_public ? nd(rng) : 0.f;
        }
        // residual branches start small so each block begins near the identity
        for (int k = 0; k < shape->blocks; ++k) {
            const Layer& L = net->layers[2 + 2 * k];
            for (size_t i = 0; i < (size_t)L.cout * 9 * L.cin; ++i) h[L.w_off + i] *= 0.1f;
        }
        NCK(cudaMemcpyAsync(net->p, h.data(), sizeof(float) * net->nparam, cudaMemcpyHostToDevice, net->stream));
        NCK(cudaMemsetAsync(net->m, 0, sizeof(float) * net->nparam, net->stream));
        NCK(cudaMemsetAsync(net->v, 0, sizeof(float) * net->nparam, net->stream));
        to_bf16_kernel<<<grid_for(net->nparam), 256, 0, net->stream>>>(net->p, net->wb, net->nparam);
        NCK(cudaGetLastError());
        NCK(cudaStreamSynchronize(net->stream));
        return PIT_OK;
    };
    const pit_status st = setup();
    if (st != PIT_OK) {
        fprintf(stderr, "pit_net_create: %s\n", net->err);
        pit_net_destroy(net);
        return st;
    }
    *out = net;
    return PIT_OK;
}

extern "C" void pit_net_destroy(pit_net* net) {
    if (!net) return;
    cudaFree(net->p);
    cudaFree(net->g);
    cudaFree(net->m);
    cudaFree(net->v);
    cudaFree(net->wb);
    cudaFree(net->wf);
    cudaFree(net->part);
    cudaFree(net->loss_part);
    cudaFree(net->tc_err);
    cudaFree(net->bias_part);
    cudaFree(net->in);
    for (auto x : net->xs) cudaFree(x);
    for (auto x : net->hs) cudaFree(x);
    cudaFree(net->out);
    cudaFree(net->dout);
    cudaFree(net->d0);
    cudaFree(net->d1);
    cudaFree(net->d2);
    cudaFree(net->lognu);
    delete net;
}

extern "C" const char* pit_net_last_error(const pit_net* net) { return net ? net->err : "null network"; }

// Public flat layout <-> stored layout (the input layer stores 16 channels, 2 public).
static void public_to_stored(const pit_net* net, const float* pub, std::vector<float>& st) {
    st.assign(net->nparam, 0.f);
    size_t o = 0;
    for (const Layer& L : net->layers) {
        for (int co = 0; co < L.cout; ++co)
            for (int t = 0; t < 9; ++t)
                for (int c = 0; c < L.cin_public; ++c) st[L.w_off + ((size_t)co * 9 + t) * L.cin + c] = pub[o++];
        for (int co = 0; co < L.cout; ++co) st[L.b_off + co] = pub[o++];
    }
}

static void stored_to_public(const pit_net* net, const std::vector<float>& st, float* pub) {
    size_t o = 0;
    for (const Layer& L : net->layers) {
        for (int co = 0; co < L.cout; ++co)
            for (int t = 0; t < 9; ++t)
                for (int c = 0; c < L.cin_public; ++c) pub[o++] = st[L.w_off + ((size_t)co * 9 + t) * L.cin + c];
        for (int co = 0; co < L.cout; ++co) pub[o++] = st[L.b_off + co];
    }
}

extern "C" pit_status pit_net_get_params(pit_net* net, float* params_host) {
    if (!net || !params_host) return PIT_EINVAL;
    std::vector<float> st(net->nparam);
    NCK(cudaMemcpyAsync(st.data(), net->p, sizeof(float) * net->nparam, cudaMemcpyDeviceToHost, net->stream));
    NCK(cudaStreamSynchronize(net->stream));
    stored_to_public(net, st, params_host);
    return PIT_OK;
}

extern "C" pit_status pit_net_set_params(pit_net* net, const float* params_host) {
    if (!net || !params_host) return PIT_EINVAL;
    std::vector<float> st;
    public_to_stored(net, params_host, st);
    NCK(cudaMemcpyAsync(net->p, st.data(), sizeof(float) * net->nparam, cudaMemcpyHostToDevice, net->stream));
    to_bf16_kernel<<<grid_for(net->nparam), 256, 0, net->stream>>>(net->p, net->wb, net->nparam);
    NCK(cudaGetLastError());
    NCK(cudaStreamSynchronize(net->stream));
    return PIT_OK;
}

static pit_status set_lognu(pit_net* net, const float* lognu_host, int B) {
    NCK(cudaMemcpyAsync(net->lognu, lognu_host, sizeof(float) * B, cudaMemcpyHostToDevice, net->stream));
    return PIT_OK;
}

extern "C" pit_status pit_net_guess(pit_net* net, const double* u0_dev, const float* lognu_host, int B,
                                    double* U_dev) {
    if (!net || !u0_dev || !lognu_host || !U_dev || B < 1 || B > net->shape.max_batch) return PIT_EINVAL;
    if (pit_status st = set_lognu(net, lognu_host, B)) return st;
    if (pit_status st = forward(net, u0_dev, net->lognu, B)) return st;
    const size_t Ns = (size_t)net->shape.height * net->shape.width;
    output_kernel<<<grid_for((size_t)B * net->shape.levels * Ns), 256, 0, net->stream>>>(net->out, u0_dev, U_dev, B,
                                                                                       net->shape.levels, Ns);
    NCK(cudaGetLastError());
    return check_tc(net);
}

extern "C" pit_status pit_net_make_target(pit_net* net, const double* u0_dev, const double* U_dev, void* target_dev) {
    if (!net || !u0_dev || !U_dev || !target_dev) return PIT_EINVAL;
    const size_t Ns = (size_t)net->shape.height * net->shape.width;
    target_kernel<<<grid_for((size_t)net->shape.levels * Ns), 256, 0, net->stream>>>(
        U_dev, u0_dev, static_cast<bf16*>(target_dev), net->shape.levels, Ns);
    NCK(cudaGetLastError());
    return PIT_OK;
}

// Loss and gradients of one batch (targets: BF16 [B][H][W][M]).
static pit_status loss_grad(pit_net* net, const double* u0_dev, const float* lognu_host, const void* target_dev,
                            int B, float* loss_out) {
    const pit_net_shape& s = net->shape;
    const size_t Ns = (size_t)s.height * s.width;
    if (pit_status st = set_lognu(net, lognu_host, B)) return st;
    if (pit_status st = forward(net, u0_dev, net->lognu, B)) return st;
    const size_t nout = (size_t)B * Ns * s.levels;
    const int blocks = std::min(1024, grid_for(nout));
    const int vec = (reinterpret_cast<uintptr_t>(target_dev) & 15) == 0 ? 1 : 0;
    mse_kernel<<<blocks, 256, 0, net->stream>>>(net->out, static_cast<const bf16*>(target_dev), net->dout,
                                                net->loss_part, nout, 1.f / (float)nout, vec);
    NCK(cudaGetLastError());
    // backward: head, blocks in reverse, lift
    const int nb = s.blocks;
    bf16* dx = net->d0;
    if (pit_status st = conv_bwd(net, net->xs[nb], net->dout, net->layers.back(), dx, B)) return st;
    for (int k = nb - 1; k >= 0; --k) {
        // x_{k+1} = x_k + conv2(h_k): gradient dx flows to conv2 and straight to x_k.
        // dh = (conv2's data gradient) zeroed where h_k <= 0 (h_k = relu(conv1(x_k)));
        // dx += conv1's data gradient of dh, in place -- and for k = 0 zeroed where x_0 <= 0
        // (x_0 = relu(lift(in))), the gradient the lift's weights need
        bf16* dh = net->d1;
        if (pit_status st = conv_bwd(net, net->hs[k], dx, net->layers[2 + 2 * k], dh, B, nullptr, net->hs[k]))
            return st;
        if (pit_status st = conv_bwd(net, net->xs[k], dh, net->layers[1 + 2 * k], dx, B, dx, k == 0 ? net->xs[0] : nullptr))
            return st;
        NCK(cudaGetLastError());
    }
    if (nb == 0)
        relu_back_kernel<<<grid_for(B * Ns * s.channels), 256, 0, net->stream>>>(dx, net->xs[0], B * Ns * s.channels);
    if (pit_status st = conv_bwd(net, net->in, dx, net->layers[0], nullptr, B)) return st;
    if (loss_out) {
        std::vector<float> part(blocks);
        NCK(cudaMemcpyAsync(part.data(), net->loss_part, sizeof(float) * blocks, cudaMemcpyDeviceToHost, net->stream));
        NCK(cudaStreamSynchronize(net->stream));
        double sum = 0.0;
        for (float f : part) sum += f;
        *loss_out = (float)(sum / (double)nout);
    }
    return PIT_OK;
}

extern "C" pit_status pit_net_gradients(pit_net* net, const double* u0_dev, const float* lognu_host,
                                        const void* target_dev, int B, float* loss_out, float* grads_host) {
    if (!net || !u0_dev || !lognu_host || !target_dev || B < 1 || B > net->shape.max_batch) return PIT_EINVAL;
    if (pit_status st = loss_grad(net, u0_dev, lognu_host, target_dev, B, loss_out)) return st;
    if (pit_status st = check_tc(net)) return st;
    if (grads_host) {
        std::vector<float> st(net->nparam);
        NCK(cudaMemcpyAsync(st.data(), net->g, sizeof(float) * net->nparam, cudaMemcpyDeviceToHost, net->stream));
        NCK(cudaStreamSynchronize(net->stream));
        stored_to_public(net, st, grads_host);
    }
    return PIT_OK;
}

extern "C" pit_status pit_net_train_step(pit_net* net, const double* u0_dev, const float* lognu_host,
                                         const void* target_dev, int B, float lr, float* loss_out) {
    if (!net || !u0_dev || !lognu_host || !target_dev || B < 1 || B > net->shape.max_batch || !(lr > 0.f))
        return PIT_EINVAL;
    if (pit_status st = loss_grad(net, u0_dev, lognu_host, target_dev, B, loss_out)) return st;
    net->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
    adam_kernel<<<grid_for(net->nparam), 256, 0, net->stream>>>(net->p, net->g, net->m, net->v, net->nparam, lr, b1,
                                                                b2, 1e-8f, c1, c2);
    to_bf16_kernel<<<grid_for(net->nparam), 256, 0, net->stream>>>(net->p, net->wb, net->nparam);
    NCK(cudaGetLastError());
    return loss_out ? check_tc(net) : PIT_OK;
}

// ------------------------------------------------- one convolution layer, context-free
//
// The network's own tensor-core convolution kernels (the forward conv, the weight
// gradient and the data gradient through the flipped weights), run on one layer's
// operands. A scratch pit_net carries the shape, the stream and the temporaries of
// the calls above; it owns nothing of the caller's.

namespace {
struct ScratchNet {
    pit_net n;
    ~ScratchNet() {
        cudaFree(n.wf);
        cudaFree(n.part);
        cudaFree(n.g);
        cudaFree(n.bias_part);
        cudaFree(n.loss_part);
        cudaFree(n.tc_err);
    }
};

bool conv_args_ok(int B, int H, int Wd, int Cin, int Cout) {
    return B >= 1 && H >= 1 && Wd >= 1 && Cin >= 16 && Cout >= 16 && Cin % 16 == 0 && Cout % 16 == 0 &&
           Cin <= 4096 && Cout <= 4096;
}
}  // namespace

extern "C" pit_status pit_conv3x3_forward(const void* X_dev, const void* W_dev, const float* bias_dev,
                                          const void* res_dev, void* Y_dev, int B, int H, int Wd, int Cin, int Cout,
                                          int relu, void* stream) {
    if (!X_dev || !W_dev || !bias_dev || !Y_dev || !conv_args_ok(B, H, Wd, Cin, Cout)) return PIT_EINVAL;
    ScratchNet s;
    pit_net* net = &s.n;
    net->shape.height = H;
    net->shape.width = Wd;
    net->stream = static_cast<cudaStream_t>(stream);
    NCK(cudaMalloc(&net->tc_err, sizeof(int)));
    NCK(cudaMemsetAsync(net->tc_err, 0, sizeof(int), net->stream));
    if (pit_status st = launch_conv_tc(net, static_cast<const bf16*>(X_dev), static_cast<const bf16*>(W_dev), bias_dev,
                                       static_cast<const bf16*>(res_dev), static_cast<bf16*>(Y_dev), B, Cin, Cout,
                                       relu ? 1 : 0))
        return st;
    return check_tc(net);
}

extern "C" pit_status pit_conv3x3_backward(const void* X_dev, const void* W_dev, const void* dY_dev, void* dX_dev,
                                           float* dW_dev, float* db_dev, int B, int H, int Wd, int Cin, int Cout,
                                           void* stream) {
    if (!X_dev || !W_dev || !dY_dev || !dW_dev || !db_dev || !conv_args_ok(B, H, Wd, Cin, Cout)) return PIT_EINVAL;
    ScratchNet s;
    pit_net* net = &s.n;
    net->shape.height = H;
    net->shape.width = Wd;
    net->stream = static_cast<cudaStream_t>(stream);
    const size_t nw = (size_t)Cout * 9 * Cin;
    NCK(cudaMalloc(&net->tc_err, sizeof(int)));
    NCK(cudaMalloc(&net->wf, sizeof(bf16) * nw));
    NCK(cudaMalloc(&net->part, sizeof(float) * kMaxSplits * nw));
    NCK(cudaMalloc(&net->g, sizeof(float) * (nw + Cout)));
    NCK(cudaMalloc(&net->bias_part, sizeof(float) * kBiasBlocks * (size_t)Cout));
    NCK(cudaMalloc(&net->loss_part, sizeof(float) * (1024 + 4096)));  // zero bias of the data gradient at +1024
    NCK(cudaMemsetAsync(net->tc_err, 0, sizeof(int), net->stream));
    NCK(cudaMemsetAsync(net->loss_part, 0, sizeof(float) * (1024 + 4096), net->stream));
    net->wb = const_cast<bf16*>(static_cast<const bf16*>(W_dev));  // read only
    Layer L;
    L.cin = Cin;
    L.cout = Cout;
    L.cin_public = Cin;
    L.w_off = 0;
    L.b_off = nw;
    if (pit_status st = conv_bwd(net, static_cast<const bf16*>(X_dev), static_cast<const bf16*>(dY_dev), L,
                                 static_cast<bf16*>(dX_dev), B))
        return st;
    NCK(cudaMemcpyAsync(dW_dev, net->g, sizeof(float) * nw, cudaMemcpyDeviceToDevice, net->stream));
    NCK(cudaMemcpyAsync(db_dev, net->g + nw, sizeof(float) * Cout, cudaMemcpyDeviceToDevice, net->stream));
    return check_tc(net);
}
