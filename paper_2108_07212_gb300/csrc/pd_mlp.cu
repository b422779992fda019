// pd_mlp.cu -- the surrogate's multilayer perceptron on the tensor cores.
//
// y = W3 gelu(W2 gelu(W1 x + b1) + b2) + b3, 32 -> 128 -> 128 -> 32, with
// BF16 weights and activations as MMA operands and FP32 accumulation in tensor
// memory (tcgen05.mma kind::f16).  The forward pass of a 128-sample tile is
// one fused kernel: the three layers chain through shared memory and TMEM
// without touching global memory.  Training (loss gradients and Adam) uses the
// same fused forward, a tcgen05 GEMM for the backward products and small
// elementwise kernels; FP32 master weights, BF16 copies for the MMAs.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pd_internal.h"
#include "pd_mlp_tile.cuh"
#include "pd_tc.cuh"
#include "peridem.h"

namespace pd {
namespace mlp {
constexpr long long kSpins = 1LL << 24;      // bounded mbarrier waits (~0.5 s)
constexpr int kFwdSmem = 160 * 1024;        // generous: no operand read can leave the allocation
constexpr int kGemmSmem = 96 * 1024;
constexpr int kChunk = 64;                  // K chunk of the GEMM

struct Net {
    float *p, *g, *m, *v;                       // FP32 parameters, gradients, Adam moments
    __nv_bfloat16 *W1, *W2, *W3, *W2t, *W3t;    // BF16 weights [out][in] and transposed [in][out]
    float *Z1, *Z2, *Y, *dH, *C;                // training buffers (FP32, Bp rows)
    __nv_bfloat16 *Xt, *H1t, *H2t;              // feature-major activations [feature][Bp]
    __nv_bfloat16 *dY, *dYt, *dZ, *dZt;         // gradients: sample-major [Bp][n] and feature-major [n][Bp]
    float *loss;
    int *err;
};

__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

// ---------------------------------------------------------------------------
// fused forward of one 128-sample tile

// Rows [row0, row0 + 128) of X (rows >= B are zero) through the network whose
// BF16 weights are W1, W2, W3 and FP32 parameters p (biases); with train,
// the activations are kept in the training buffers of n.
__device__ __forceinline__ void fwd_tile(const __nv_bfloat16 *__restrict__ W1, const __nv_bfloat16 *__restrict__ W2,
                                         const __nv_bfloat16 *__restrict__ W3, const float *__restrict__ P,
                                         const float *__restrict__ X, float *__restrict__ Yout, int row0, int B,
                                         int Bp, int train, const Net &n, int *err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    uint8_t *sA = sm;                     // X tile   128 x 32  (8 KB)
    uint8_t *sW1 = sm + 8 * 1024;         // W1       128 x 32  (8 KB)
    uint8_t *sH = sm + 16 * 1024;         // H tile   128 x 128 (32 KB)
    uint8_t *sW2 = sm + 48 * 1024;        // W2       128 x 128 (32 KB)
    uint8_t *sW3 = sm + 80 * 1024;        // W3        32 x 128 (8 KB)
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = row0 + tid;
    if (warp == 0) tc::tmem_alloc(&tmem_base, 128);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    // operands -> canonical K-major shared layout, 8 values (one 16-byte core
    // matrix row) per store
    const bool x16 = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
    // the thread's whole input row is loaded before any store
    float x[IN];
    if (row < B && x16) {
#pragma unroll
        for (int k4 = 0; k4 < IN; k4 += 4) {
            const float4 a = *reinterpret_cast<const float4 *>(X + (size_t)row * IN + k4);
            x[k4] = a.x, x[k4 + 1] = a.y, x[k4 + 2] = a.z, x[k4 + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int q = 0; q < IN; ++q) x[q] = (row < B) ? X[(size_t)row * IN + q] : 0.f;
    }
#pragma unroll
    for (int k8 = 0; k8 < IN; k8 += 8) {
        __align__(16) __nv_bfloat16 xb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            xb[q] = __float2bfloat16(x[k8 + q]);
            if (train) n.Xt[(size_t)(k8 + q) * Bp + row] = xb[q];
        }
        *reinterpret_cast<uint4 *>(sA + tc::kmajor_off(tid, k8, TILE)) = *reinterpret_cast<const uint4 *>(xb);
    }
    {
        // the three weight matrices, 16 bytes per load: every load of the thread
        // is issued before the first store, so the copy costs one L2 (or DRAM)
        // latency instead of one per row chunk
        static_assert((HID * IN / 8) % 128 == 0 && (HID * HID / 8) % 128 == 0 && (OUT * HID / 8) % 128 == 0,
                      "weight chunks must divide over the 128 threads");
        constexpr int n1 = HID * IN / 8 / 128, n2 = HID * HID / 8 / 128, n3 = OUT * HID / 8 / 128;
        uint4 w1[n1], w2[n2], w3[n3];
#pragma unroll
        for (int q = 0; q < n1; ++q) {
            const int e = tid + q * 128, r = e / (IN / 8), k8 = (e % (IN / 8)) * 8;
            w1[q] = *reinterpret_cast<const uint4 *>(W1 + (size_t)r * IN + k8);
        }
#pragma unroll
        for (int q = 0; q < n2; ++q) {
            const int e = tid + q * 128, r = e / (HID / 8), k8 = (e % (HID / 8)) * 8;
            w2[q] = *reinterpret_cast<const uint4 *>(W2 + (size_t)r * HID + k8);
        }
#pragma unroll
        for (int q = 0; q < n3; ++q) {
            const int e = tid + q * 128, r = e / (HID / 8), k8 = (e % (HID / 8)) * 8;
            w3[q] = *reinterpret_cast<const uint4 *>(W3 + (size_t)r * HID + k8);
        }
#pragma unroll
        for (int q = 0; q < n1; ++q) {
            const int e = tid + q * 128, r = e / (IN / 8), k8 = (e % (IN / 8)) * 8;
            *reinterpret_cast<uint4 *>(sW1 + tc::kmajor_off(r, k8, HID)) = w1[q];
        }
#pragma unroll
        for (int q = 0; q < n2; ++q) {
            const int e = tid + q * 128, r = e / (HID / 8), k8 = (e % (HID / 8)) * 8;
            *reinterpret_cast<uint4 *>(sW2 + tc::kmajor_off(r, k8, HID)) = w2[q];
        }
#pragma unroll
        for (int q = 0; q < n3; ++q) {
            const int e = tid + q * 128, r = e / (HID / 8), k8 = (e % (HID / 8)) * 8;
            *reinterpret_cast<uint4 *>(sW3 + tc::kmajor_off(r, k8, OUT)) = w3[q];
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    bool ok = true;
    uint32_t phase = 0;

    for (int layer = 0; layer < 3 && ok; ++layer) {
        const int K = layer == 0 ? IN : HID;
        const int N = layer == 2 ? OUT : HID;
        uint8_t *a = layer == 0 ? sA : sH;
        uint8_t *b = layer == 0 ? sW1 : (layer == 1 ? sW2 : sW3);
        const uint32_t lbo_a = tc::kmajor_lbo(TILE), lbo_b = tc::kmajor_lbo(N);
        if (tid == 0) {
            const uint32_t idesc = tc::idesc_bf16(TILE, N);
            for (int ks = 0; ks < K / 16; ++ks) {
                const uint64_t ad = tc::smem_desc(tc::smem_addr(a) + ks * 2 * lbo_a, lbo_a, tc::kSbo);
                const uint64_t bd = tc::smem_desc(tc::smem_addr(b) + ks * 2 * lbo_b, lbo_b, tc::kSbo);
                tc::mma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
            }
            tc::mma_commit(&mbar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&mbar, phase, kSpins)) != 0;   // uniform outcome
        phase ^= 1;
        if (!ok) break;
        tc::fence_after_sync();
        const float *bias = P + (layer == 0 ? OB1 : (layer == 1 ? OB2 : OB3));
        for (int c0 = 0; c0 < N; c0 += 16) {
            float acc[16];
            tc::tmem_ld16(tmem + lane_base + (uint32_t)c0, acc);
            __align__(16) __nv_bfloat16 hb[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int c = c0 + q;
                const float z = acc[q] + bias[c];
                if (layer == 2) {
                    if (row < B) Yout[(size_t)row * OUT + c] = z;
                    if (train) n.Y[(size_t)row * OUT + c] = z;
                } else {
                    if (train) (layer == 0 ? n.Z1 : n.Z2)[(size_t)row * HID + c] = z;
                    hb[q] = __float2bfloat16(gelu(z));
                    if (train) (layer == 0 ? n.H1t : n.H2t)[(size_t)c * Bp + row] = hb[q];
                }
            }
            if (layer < 2) {
                *reinterpret_cast<uint4 *>(sH + tc::kmajor_off(tid, c0, TILE)) = *reinterpret_cast<const uint4 *>(hb);
                *reinterpret_cast<uint4 *>(sH + tc::kmajor_off(tid, c0 + 8, TILE)) =
                    *reinterpret_cast<const uint4 *>(hb + 8);
            }
        }
        tc::fence_before_sync();
        tc::fence_async_smem();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (!ok) {
        // the MMAs committed on the phase that timed out may still be writing the
        // accumulator: one more bounded wait on that phase before the columns are
        // released (the outputs of a timed-out tile are invalid either way: err is set)
        tc::mbar_wait(&mbar, phase ^ 1, kSpins);
        if (tid == 0) atomicExch(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem_base, 128);
}

__global__ void __launch_bounds__(128) k_mlp_fwd(Net n, const float *__restrict__ X, float *__restrict__ Yout,
                                                 int B, int Bp, int train) {
    fwd_tile(n.W1, n.W2, n.W3, n.p, X, Yout, blockIdx.x * TILE, B, Bp, train, n, n.err);
}

// Inference of several networks in one launch (the surrogate's step): tile
// blockIdx.x is rows [w.y, min(w.y + 128, w.z)) of X / Y through network
// refs[w.x].  The MMAs are those of fwd_tile; operand staging and the layer
// epilogues are spread over four warpgroups: warp w reads TMEM lanes
// 32 (w % 4) .. 32 (w % 4) + 31 (its quarter of the rows) and warpgroup g
// takes the g-th quarter of a hidden layer's columns, so four warps per
// scheduler hide the latency of the activation chains and of the loads.  The
// activation is the GELU with the error function of Abramowitz & Stegun
// 7.1.26 (branch-free; its 1.5e-7 error is far below the BF16 rounding of
// the activations).  With r.lin the output is the surrogate's modal force
// f = net(q) - Lambda q.
constexpr int kInferThreads = 512;
constexpr int kInferGroups = kInferThreads / TILE;

__global__ void __launch_bounds__(kInferThreads) k_mlp_infer(const MlpRef *__restrict__ refs,
                                                             const int4 *__restrict__ work,
                                                             const float *__restrict__ X, float *__restrict__ Y,
                                                             int *err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    uint8_t *sA = sm;                     // X tile   128 x 32  (8 KB)
    uint8_t *sW1 = sm + 8 * 1024;         // W1       128 x 32  (8 KB)
    uint8_t *sH = sm + 16 * 1024;         // H tile   128 x 128 (32 KB)
    uint8_t *sW2 = sm + 48 * 1024;        // W2       128 x 128 (32 KB)
    uint8_t *sW3 = sm + 80 * 1024;        // W3        32 x 128 (8 KB)
    const int4 wk = work[blockIdx.x];
    const MlpRef r = refs[wk.x];
    const float *P = r.p, *lin = r.lin;
    const int B = wk.z;
    const int tid = threadIdx.x, warp = tid >> 5, wg = warp >> 2;
    const int lrow = tid & 127;           // = 32 (warp % 4) + lane: the TMEM lane of the thread
    const int row = wk.y + lrow;
    if (tid == 0) tc::mbar_init(&mbar, 1);
    static_assert(IN == 8 * kInferGroups, "one 8-column piece of the input row per warpgroup");
    float *sX = reinterpret_cast<float *>(sm + 88 * 1024);   // input rows in FP32, 128 x 32 (16 KB)
    {
        // every load first: the thread's pieces of the three weight matrices
        // (while the kernel that writes the inputs may still run), then the
        // row's input columns 8 wg .. 8 wg + 7; then the stores
        WeightStage<IN, HID, kInferThreads> w1;
        WeightStage<HID, HID, kInferThreads> w2;
        WeightStage<HID, OUT, kInferThreads> w3;
        w1.load(static_cast<const __nv_bfloat16 *>(r.W1), tid);
        w2.load(static_cast<const __nv_bfloat16 *>(r.W2), tid);
        w3.load(static_cast<const __nv_bfloat16 *>(r.W3), tid);
        tc::grid_dep_wait();
        if (warp == 0) tc::tmem_alloc(&tmem_base, 128);
        float4 x0 = make_float4(0.f, 0.f, 0.f, 0.f), x1 = x0;
        if (row < B) {
            const float4 *src = reinterpret_cast<const float4 *>(X + (size_t)row * IN + 8 * wg);
            x0 = src[0];
            x1 = src[1];
        }
        const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        __align__(16) __nv_bfloat16 xb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            xb[q] = __float2bfloat16(x[q]);
            sX[lrow * IN + 8 * wg + q] = x[q];
        }
        *reinterpret_cast<uint4 *>(sA + tc::kmajor_off(lrow, 8 * wg, TILE)) = *reinterpret_cast<const uint4 *>(xb);
        w1.store(sW1, tid);
        w2.store(sW2, tid);
        w3.store(sW3, tid);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tc::grid_dep_launch();
    const uint32_t tmem = tmem_base;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    constexpr int kCols = HID / kInferGroups;            // hidden columns per warpgroup
    static_assert(kCols % 16 == 0 && OUT / 16 <= kInferGroups, "16-column TMEM loads");
    bool ok = true;
    uint32_t phase = 0;
    for (int layer = 0; layer < 3 && ok; ++layer) {
        const int K = layer == 0 ? IN : HID;
        const int N = layer == 2 ? OUT : HID;
        uint8_t *a = layer == 0 ? sA : sH;
        uint8_t *b = layer == 0 ? sW1 : (layer == 1 ? sW2 : sW3);
        if (tid == 0) {
            const uint32_t lbo_a = tc::kmajor_lbo(TILE), lbo_b = tc::kmajor_lbo(N);
            const uint32_t idesc = tc::idesc_bf16(TILE, N);
            for (int ks = 0; ks < K / 16; ++ks) {
                const uint64_t ad = tc::smem_desc(tc::smem_addr(a) + ks * 2 * lbo_a, lbo_a, tc::kSbo);
                const uint64_t bd = tc::smem_desc(tc::smem_addr(b) + ks * 2 * lbo_b, lbo_b, tc::kSbo);
                tc::mma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
            }
            tc::mma_commit(&mbar);
        }
        ok = __syncthreads_and(tc::mbar_wait(&mbar, phase, kSpins)) != 0;   // uniform outcome
        phase ^= 1;
        if (!ok) break;
        tc::fence_after_sync();
        const float *bias = P + (layer == 0 ? OB1 : (layer == 1 ? OB2 : OB3));
        if (layer < 2) {
            // hidden layer: columns kCols wg .. kCols (wg + 1) of the thread's row
#pragma unroll
            for (int c0 = kCols * wg; c0 < kCols * (wg + 1); c0 += 16) {
                float acc[16];
                tc::tmem_ld16(tmem + lane_base + (uint32_t)c0, acc);
                __align__(16) __nv_bfloat16 hb[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) hb[q] = __float2bfloat16(gelu_fast(acc[q] + bias[c0 + q]));
                *reinterpret_cast<uint4 *>(sH + tc::kmajor_off(lrow, c0, TILE)) = *reinterpret_cast<const uint4 *>(hb);
                *reinterpret_cast<uint4 *>(sH + tc::kmajor_off(lrow, c0 + 8, TILE)) =
                    *reinterpret_cast<const uint4 *>(hb + 8);
            }
        } else if (wg < OUT / 16) {
            // output layer: 16 columns per warpgroup (the first OUT / 16 groups; warp-uniform)
            const int c0 = 16 * wg;
            float acc[16];
            tc::tmem_ld16(tmem + lane_base + (uint32_t)c0, acc);
            if (row < B) {
                // y = z - lin (.) x with x from the staged rows; 16-byte stores
                float y[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = c0 + q;
                    const float z = acc[q] + bias[c];
                    y[q] = lin ? z - lin[c] * sX[lrow * IN + c] : z;
                }
                float4 *dst = reinterpret_cast<float4 *>(Y + (size_t)row * OUT + c0);
#pragma unroll
                for (int q = 0; q < 16; q += 4) dst[q / 4] = make_float4(y[q], y[q + 1], y[q + 2], y[q + 3]);
            }
        }
        tc::fence_before_sync();
        tc::fence_async_smem();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (!ok) {
        // the MMAs committed on the phase that timed out may still be writing the
        // accumulator: one more bounded wait on that phase before the columns are
        // released (the outputs of a timed-out tile are invalid either way: err is set)
        tc::mbar_wait(&mbar, phase ^ 1, kSpins);
        if (tid == 0) atomicExch(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem_base, 128);
}

// ---------------------------------------------------------------------------
// C[M x N] (+)= A[M x K] * B[N x K]^T, BF16 operands stored K-contiguous, FP32
// result.  One CTA per (128-row tile, K split); split partials are added
// atomically into C (which the caller cleared).  M multiple of 128, N in
// {32, 64, 128}, K a multiple of 16 per split.
__global__ void __launch_bounds__(128) k_gemm(const __nv_bfloat16 *__restrict__ A, int lda,
                                              const __nv_bfloat16 *__restrict__ Bm, int ldb, float *C, int ldc, int N,
                                              int K, int kper, int ksplit, int *err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    uint8_t *sA = sm;                 // 128 x 64 (16 KB)
    uint8_t *sB = sm + 16 * 1024;     // N x 64 (<= 16 KB)
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * TILE;
    const int k_lo = blockIdx.y * kper, k_hi = min(K, k_lo + kper);
    if (warp == 0) tc::tmem_alloc(&tmem_base, 128);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;
    bool ok = true;
    uint32_t phase = 0;
    int issued = 0;
    for (int k0 = k_lo; k0 < k_hi && ok; k0 += kChunk) {
        const int kc = min(kChunk, k_hi - k0);   // multiple of 16
        for (int e = tid; e < TILE * kc; e += 128) {
            const int r = e / kc, k = e % kc;
            *reinterpret_cast<__nv_bfloat16 *>(sA + tc::kmajor_off(r, k, TILE)) = A[(size_t)(m0 + r) * lda + k0 + k];
        }
        for (int e = tid; e < N * kc; e += 128) {
            const int r = e / kc, k = e % kc;
            *reinterpret_cast<__nv_bfloat16 *>(sB + tc::kmajor_off(r, k, N)) = Bm[(size_t)r * ldb + k0 + k];
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            const uint32_t lbo_a = tc::kmajor_lbo(TILE), lbo_b = tc::kmajor_lbo(N);
            const uint32_t idesc = tc::idesc_bf16(TILE, N);
            for (int ks = 0; ks < kc / 16; ++ks) {
                const uint64_t ad = tc::smem_desc(tc::smem_addr(sA) + ks * 2 * lbo_a, lbo_a, tc::kSbo);
                const uint64_t bd = tc::smem_desc(tc::smem_addr(sB) + ks * 2 * lbo_b, lbo_b, tc::kSbo);
                tc::mma_bf16(tmem, ad, bd, idesc, issued > 0 ? 1u : 0u);
                ++issued;
            }
            tc::mma_commit(&mbar);
        }
        // the tiles are reused by the next chunk; the outcome is made uniform
        ok = __syncthreads_and(tc::mbar_wait(&mbar, phase, kSpins)) != 0;
        phase ^= 1;
        tc::fence_after_sync();
    }
    if (ok && k_lo < k_hi) {
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        const int row = m0 + tid;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float acc[16];
            tc::tmem_ld16(tmem + lane_base + (uint32_t)c0, acc);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                float *dst = &C[(size_t)row * ldc + c0 + q];
                if (ksplit > 1) atomicAdd(dst, acc[q]);
                else *dst = acc[q];
            }
        }
    }
    if (!ok) {
        // the MMAs committed on the phase that timed out may still be writing the
        // accumulator: one more bounded wait on that phase before the columns are
        // released (the outputs of a timed-out tile are invalid either way: err is set)
        tc::mbar_wait(&mbar, phase ^ 1, kSpins);
        if (tid == 0) atomicExch(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem_base, 128);
}

// ---------------------------------------------------------------------------
// elementwise pieces of the backward pass and the optimiser

// dY = dL/dY for L = mean over samples and outputs of (Y - T)^2; also the loss.
__global__ void k_out_grad(Net n, const float *__restrict__ T, int B, int Bp) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Bp * OUT) return;
    const int r = idx / OUT, c = idx % OUT;
    float d = 0.f;
    if (r < B) {
        const float e = n.Y[(size_t)r * OUT + c] - T[(size_t)r * OUT + c];
        d = 2.f * e / (float)(B * OUT);
        atomicAdd(n.loss, e * e / (float)(B * OUT));
        atomicAdd(&n.g[OB3 + c], d);
    }
    const __nv_bfloat16 db = __float2bfloat16(d);
    n.dY[(size_t)r * OUT + c] = db;
    n.dYt[(size_t)c * Bp + r] = db;
}

// dZ = dH * gelu'(Z) (rows beyond the batch are zero), bias gradient.
__global__ void k_hidden_grad(Net n, const float *__restrict__ Z, int B, int Bp, int ob) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Bp * HID) return;
    const int r = idx / HID, c = idx % HID;
    float d = 0.f;
    if (r < B) {
        d = n.dH[(size_t)r * HID + c] * gelu_grad(Z[(size_t)r * HID + c]);
        atomicAdd(&n.g[ob + c], d);
    }
    const __nv_bfloat16 db = __float2bfloat16(d);
    n.dZ[(size_t)r * HID + c] = db;
    n.dZt[(size_t)c * Bp + r] = db;
}

// gradient blocks computed transposed (or into scratch) -> parameter layout
__global__ void k_scatter_grad(Net n, const float *__restrict__ src, int rows, int cols, int dst_off, int transpose) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int r = idx / cols, c = idx % cols;
    const int d = transpose ? c * rows + r : idx;
    n.g[dst_off + d] += src[idx];
}

__global__ void k_adam(Net n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float g = n.g[i];
    const float m = b1 * n.m[i] + (1.f - b1) * g;
    const float v = b2 * n.v[i] + (1.f - b2) * g * g;
    n.m[i] = m;
    n.v[i] = v;
    n.p[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// BF16 copies of the weights for the MMAs: [out][in] and transposed [in][out].
__global__ void k_to_bf16(Net n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < HID * IN) n.W1[i] = __float2bfloat16(n.p[OW1 + i]);
    if (i < HID * HID) {
        const int o = i / HID, k = i % HID;
        const __nv_bfloat16 w = __float2bfloat16(n.p[OW2 + i]);
        n.W2[i] = w;
        n.W2t[k * HID + o] = w;
    }
    if (i < OUT * HID) {
        const int o = i / HID, k = i % HID;
        const __nv_bfloat16 w = __float2bfloat16(n.p[OW3 + i]);
        n.W3[i] = w;
        n.W3t[k * OUT + o] = w;
    }
}

}  // namespace mlp
}  // namespace pd

// ===========================================================================
// host side

using namespace pd::mlp;

struct pd_mlp {
    cudaStream_t stream = nullptr;
    int max_batch = 0, Bp = 0;
    Net n{};
    bool bound = false;
    int adam_t = 0;
};

namespace {

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

template <class T>
void carve(char *base, size_t &off, T *&p, size_t count) {
    p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off = al(off + sizeof(T) * std::max<size_t>(count, 1));
}

size_t mlp_layout(pd_mlp *m, char *base) {
    size_t off = 0, Bp = (size_t)m->Bp;
    Net &n = m->n;
    carve(base, off, n.p, NPARAM);
    carve(base, off, n.g, NPARAM);
    carve(base, off, n.m, NPARAM);
    carve(base, off, n.v, NPARAM);
    carve(base, off, n.W1, HID * IN);
    carve(base, off, n.W2, HID * HID);
    carve(base, off, n.W3, OUT * HID);
    carve(base, off, n.W2t, HID * HID);
    carve(base, off, n.W3t, OUT * HID);
    carve(base, off, n.Z1, Bp * HID);
    carve(base, off, n.Z2, Bp * HID);
    carve(base, off, n.Y, Bp * OUT);
    carve(base, off, n.dH, Bp * HID);
    carve(base, off, n.C, HID * HID);
    carve(base, off, n.Xt, IN * Bp);
    carve(base, off, n.H1t, HID * Bp);
    carve(base, off, n.H2t, HID * Bp);
    carve(base, off, n.dY, Bp * OUT);
    carve(base, off, n.dYt, OUT * Bp);
    carve(base, off, n.dZ, Bp * HID);
    carve(base, off, n.dZt, HID * Bp);
    carve(base, off, n.loss, 1);
    carve(base, off, n.err, 1);
    return off;
}

#define MLP_CUDA(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return pd::set_error(PD_ECUDA, cudaGetErrorString(e_));          \
    } while (0)

int check_err(pd_mlp *m) {
    int err = 0;
    MLP_CUDA(cudaMemcpyAsync(&err, m->n.err, 4, cudaMemcpyDeviceToHost, m->stream));
    MLP_CUDA(cudaStreamSynchronize(m->stream));
    if (err) return pd::set_error(PD_ETIMEOUT, "tensor-core wait timed out");
    return PD_OK;
}

// K is split into pieces of a multiple of 64 columns; with more than one
// piece the partial products are added atomically into C (cleared by the caller).
cudaError_t gemm(pd_mlp *m, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, float *C, int ldc,
                 int M, int N, int K, int ksplit) {
    int kper = (K + ksplit - 1) / ksplit;
    kper = ((kper + kChunk - 1) / kChunk) * kChunk;
    ksplit = (K + kper - 1) / kper;
    dim3 grid(M / TILE, ksplit);
    pd::mlp::k_gemm<<<grid, 128, kGemmSmem, m->stream>>>(A, lda, B, ldb, C, ldc, N, K, kper, ksplit, m->n.err);
    return cudaGetLastError();
}

int forward(pd_mlp *m, const float *x, float *y, int batch, int train) {
    if (batch < 0 || batch > m->max_batch) return pd::set_error(PD_EINVAL, "batch exceeds max_batch");
    if (batch == 0) return PD_OK;
    const int tiles = (batch + TILE - 1) / TILE;
    pd::mlp::k_mlp_fwd<<<tiles, 128, kFwdSmem, m->stream>>>(m->n, x, y, batch, m->Bp, train);
    MLP_CUDA(cudaGetLastError());
    return PD_OK;
}

// forward + backward into n.g (cleared first); loss into n.loss.
int backward(pd_mlp *m, const float *x, const float *t, int batch) {
    Net &n = m->n;
    const int Bp = m->Bp;
    cudaStream_t s = m->stream;
    MLP_CUDA(cudaMemsetAsync(n.g, 0, sizeof(float) * NPARAM, s));
    MLP_CUDA(cudaMemsetAsync(n.loss, 0, sizeof(float), s));
    // clear the padded rows/columns of the feature-major activations
    MLP_CUDA(cudaMemsetAsync(n.Xt, 0, sizeof(__nv_bfloat16) * IN * Bp, s));
    if (int r = forward(m, x, n.Y, batch, 1)) return r;
    const int Mp = ((batch + TILE - 1) / TILE) * TILE;   // rows actually produced
    const int ks = std::max(1, std::min(64, Mp / 512));
    const int K = Mp;
    pd::mlp::k_out_grad<<<(Mp * OUT + 255) / 256, 256, 0, s>>>(n, t, batch, Bp);
    MLP_CUDA(cudaGetLastError());
    // dW3^T [HID x OUT] = H2^T . dY
    MLP_CUDA(cudaMemsetAsync(n.C, 0, sizeof(float) * HID * OUT, s));
    MLP_CUDA(gemm(m, n.H2t, Bp, n.dYt, Bp, n.C, OUT, HID, OUT, K, ks));
    pd::mlp::k_scatter_grad<<<(HID * OUT + 255) / 256, 256, 0, s>>>(n, n.C, HID, OUT, OW3, 1);
    // dH2 = dY . W3  (B operand: W3^T [HID][OUT])
    MLP_CUDA(gemm(m, n.dY, OUT, n.W3t, OUT, n.dH, HID, Mp, HID, OUT, 1));
    pd::mlp::k_hidden_grad<<<(Mp * HID + 255) / 256, 256, 0, s>>>(n, n.Z2, batch, Bp, OB2);
    // dW2 = dZ2^T . H1
    MLP_CUDA(cudaMemsetAsync(n.C, 0, sizeof(float) * HID * HID, s));
    MLP_CUDA(gemm(m, n.dZt, Bp, n.H1t, Bp, n.C, HID, HID, HID, K, ks));
    pd::mlp::k_scatter_grad<<<(HID * HID + 255) / 256, 256, 0, s>>>(n, n.C, HID, HID, OW2, 0);
    // dH1 = dZ2 . W2  (B operand: W2^T)
    MLP_CUDA(gemm(m, n.dZ, HID, n.W2t, HID, n.dH, HID, Mp, HID, HID, 1));
    pd::mlp::k_hidden_grad<<<(Mp * HID + 255) / 256, 256, 0, s>>>(n, n.Z1, batch, Bp, OB1);
    // dW1 = dZ1^T . X
    MLP_CUDA(cudaMemsetAsync(n.C, 0, sizeof(float) * HID * IN, s));
    MLP_CUDA(gemm(m, n.dZt, Bp, n.Xt, Bp, n.C, IN, HID, IN, K, ks));
    pd::mlp::k_scatter_grad<<<(HID * IN + 255) / 256, 256, 0, s>>>(n, n.C, HID, IN, OW1, 0);
    MLP_CUDA(cudaGetLastError());
    return PD_OK;
}

}  // namespace

int pd::mlp_ref(pd_mlp *m, MlpRef *out) {
    if (!m || !m->bound || !out) return pd::set_error(PD_ESTATE, "mlp not bound");
    out->W1 = m->n.W1;
    out->W2 = m->n.W2;
    out->W3 = m->n.W3;
    out->p = m->n.p;
    out->lin = nullptr;
    return PD_OK;
}

cudaError_t pd::launch_mlp_grouped(const MlpRef *refs, const int4 *work, int n_work, const float *x, float *y,
                                   int *err, cudaStream_t s, bool pdl) {
    if (n_work == 0) return cudaSuccess;
    static_assert(sizeof(MlpRef) == 40, "MlpRef layout");
    static_assert(88 * 1024 + 128 * PD_MLP_IN * 4 <= kFwdSmem, "inference tile and its input rows fit");
    // rows of 32 floats: 16-byte aligned when the arrays are
    if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) & 15) return cudaErrorMisalignedAddress;
    return launch_ex(pd::mlp::k_mlp_infer, dim3(n_work), dim3(pd::mlp::kInferThreads), kFwdSmem, s, pdl, refs, work,
                     x, y, err);
}

cudaError_t pd::mlp_init_attributes() {
    return cudaFuncSetAttribute(pd::mlp::k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem);
}

int pd::mlp_forward_stream(pd_mlp *m, const float *x, float *y, int batch, cudaStream_t s) {
    if (!m || !m->bound) return pd::set_error(PD_ESTATE, "mlp not bound");
    if (batch < 0 || batch > m->max_batch) return pd::set_error(PD_EINVAL, "batch exceeds max_batch");
    if (batch == 0) return PD_OK;
    const int tiles = (batch + TILE - 1) / TILE;
    pd::mlp::k_mlp_fwd<<<tiles, 128, kFwdSmem, s>>>(m->n, x, y, batch, m->Bp, 0);
    MLP_CUDA(cudaGetLastError());
    return PD_OK;
}

extern "C" {

int pd_mlp_create(pd_mlp **out, int max_batch, void *cuda_stream) {
    if (!out || max_batch < 1 || max_batch > (1 << 22)) return pd::set_error(PD_EINVAL, "max_batch in [1, 4194304]");
    pd_mlp *m = new (std::nothrow) pd_mlp();
    if (!m) return pd::set_error(PD_ENOMEM, "out of host memory");
    m->stream = (cudaStream_t)cuda_stream;
    m->max_batch = max_batch;
    m->Bp = ((max_batch + TILE - 1) / TILE) * TILE;
    *out = m;
    return PD_OK;
}

int pd_mlp_destroy(pd_mlp *m) {
    if (m) {
        if (m->bound) cudaStreamSynchronize(m->stream);
        delete m;
    }
    return PD_OK;
}

int pd_mlp_arena_bytes(pd_mlp *m, size_t *bytes) {
    if (!m || !bytes) return pd::set_error(PD_EINVAL, "null argument");
    *bytes = mlp_layout(m, nullptr);
    return PD_OK;
}

int pd_mlp_bind_arena(pd_mlp *m, void *dev, size_t bytes) {
    if (!m || !dev || ((uintptr_t)dev & 255)) return pd::set_error(PD_EINVAL, "arena null or not 256-byte aligned");
    if (bytes < mlp_layout(m, nullptr)) return pd::set_error(PD_EINVAL, "arena too small");
    mlp_layout(m, (char *)dev);
    MLP_CUDA(cudaFuncSetAttribute(pd::mlp::k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kFwdSmem));
    MLP_CUDA(cudaFuncSetAttribute(pd::mlp::k_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem));
    MLP_CUDA(cudaMemsetAsync(dev, 0, bytes, m->stream));
    m->bound = true;
    return PD_OK;
}

int pd_mlp_set_params(pd_mlp *m, const float *params) {
    if (!m || !m->bound || !params) return pd::set_error(PD_ESTATE, "mlp not bound or null params");
    MLP_CUDA(cudaMemcpyAsync(m->n.p, params, sizeof(float) * NPARAM, cudaMemcpyHostToDevice, m->stream));
    MLP_CUDA(cudaMemsetAsync(m->n.m, 0, sizeof(float) * NPARAM, m->stream));
    MLP_CUDA(cudaMemsetAsync(m->n.v, 0, sizeof(float) * NPARAM, m->stream));
    pd::mlp::k_to_bf16<<<(HID * HID + 255) / 256, 256, 0, m->stream>>>(m->n);
    MLP_CUDA(cudaGetLastError());
    MLP_CUDA(cudaStreamSynchronize(m->stream));
    m->adam_t = 0;
    return PD_OK;
}

int pd_mlp_get_params(pd_mlp *m, float *params) {
    if (!m || !m->bound || !params) return pd::set_error(PD_ESTATE, "mlp not bound or null params");
    MLP_CUDA(cudaMemcpyAsync(params, m->n.p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, m->stream));
    MLP_CUDA(cudaStreamSynchronize(m->stream));
    return PD_OK;
}

int pd_mlp_forward(pd_mlp *m, const float *x, float *y, int batch) {
    if (!m || !m->bound) return pd::set_error(PD_ESTATE, "mlp not bound");
    if (batch > 0 && (!x || !y)) return pd::set_error(PD_EINVAL, "null input/output");
    return forward(m, x, y, batch, 0);
}

int pd_mlp_loss_grad(pd_mlp *m, const float *x, const float *t, int batch, float *loss, float *grad) {
    if (!m || !m->bound) return pd::set_error(PD_ESTATE, "mlp not bound");
    if (batch < 1 || batch > m->max_batch || !x || !t) return pd::set_error(PD_EINVAL, "bad batch or null input");
    if (int r = backward(m, x, t, batch)) return r;
    if (loss) MLP_CUDA(cudaMemcpyAsync(loss, m->n.loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
    if (grad) MLP_CUDA(cudaMemcpyAsync(grad, m->n.g, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, m->stream));
    return check_err(m);
}

int pd_mlp_train_step(pd_mlp *m, const float *x, const float *t, int batch, float lr, float *loss) {
    if (!m || !m->bound) return pd::set_error(PD_ESTATE, "mlp not bound");
    if (batch < 1 || batch > m->max_batch || !x || !t) return pd::set_error(PD_EINVAL, "bad batch or null input");
    if (int r = backward(m, x, t, batch)) return r;
    m->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
    pd::mlp::k_adam<<<(NPARAM + 255) / 256, 256, 0, m->stream>>>(m->n, lr, b1, b2, 1e-8f, c1, c2);
    pd::mlp::k_to_bf16<<<(HID * HID + 255) / 256, 256, 0, m->stream>>>(m->n);
    MLP_CUDA(cudaGetLastError());
    if (loss) {
        MLP_CUDA(cudaMemcpyAsync(loss, m->n.loss, sizeof(float), cudaMemcpyDeviceToHost, m->stream));
        return check_err(m);
    }
    return PD_OK;
}

}  // extern "C"
