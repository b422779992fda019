// pd_mlp_tile.cuh -- the surrogate network's layout, its activations and the
// staging of its weights for the tensor cores (the training and inference
// kernels of pd_mlp.cu).
//
// y = W3 gelu(W2 gelu(W1 x + b1) + b2) + b3, 32 -> 128 -> 128 -> 32; BF16
// weights and activations as MMA operands (tcgen05.mma kind::f16), FP32
// accumulation in tensor memory.
#pragma once

#include <cuda_bf16.h>

#include "pd_internal.h"
#include "pd_tc.cuh"
#include "peridem.h"

namespace pd {
namespace mlp {

constexpr int IN = PD_MLP_IN, HID = PD_MLP_HIDDEN, OUT = PD_MLP_OUT, TILE = 128;
// FP32 parameter vector: W1 [HID][IN], b1, W2 [HID][HID], b2, W3 [OUT][HID], b3
constexpr int OW1 = 0, OB1 = OW1 + HID * IN, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
              OB3 = OW3 + OUT * HID, NPARAM = OB3 + OUT;
static_assert(NPARAM == PD_MLP_NPARAMS, "parameter layout");

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// The error function by Abramowitz & Stegun, Handbook of Mathematical
// Functions, eq. 7.1.26: erf(x) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5)
// exp(-x^2), t = 1 / (1 + p x) for x >= 0 (odd continuation), |error| <=
// 1.5e-7; branch-free, two special-function instructions.  Its error in the
// GELU (<= 1e-7 |z|) is far below the BF16 rounding of the activations.
__device__ __forceinline__ float erf_as(float x) {
    const float ax = fabsf(x);
    const float t = __fdividef(1.0f, fmaf(0.3275911f, ax, 1.0f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    return copysignf(1.0f - poly * __expf(-ax * ax), x);
}

__device__ __forceinline__ float gelu_fast(float z) { return 0.5f * z * (1.0f + erf_as(z * 0.70710678118654752f)); }

// The 16-byte pieces (8 BF16) of a [ROWS][K] weight matrix, staged into the
// K-major shared layout over NT threads in two halves, so that the loads of
// several matrices can all be in flight before any store: load() fills the
// thread's registers, store() writes them.
template <int K, int ROWS, int NT>
struct WeightStage {
    static constexpr int count = ROWS * K / 8, per = (count + NT - 1) / NT;
    uint4 v[per];
    __device__ __forceinline__ void load(const __nv_bfloat16 *__restrict__ W, int tid) {
#pragma unroll
        for (int q = 0; q < per; ++q) {
            const int e = tid + q * NT, rr = e / (K / 8), k8 = (e % (K / 8)) * 8;
            if (e < count) v[q] = *reinterpret_cast<const uint4 *>(W + (size_t)rr * K + k8);
        }
    }
    __device__ __forceinline__ void store(uint8_t *dst, int tid) const {
#pragma unroll
        for (int q = 0; q < per; ++q) {
            const int e = tid + q * NT, rr = e / (K / 8), k8 = (e % (K / 8)) * 8;
            if (e < count) *reinterpret_cast<uint4 *>(dst + tc::kmajor_off(rr, k8, ROWS)) = v[q];
        }
    }
};

}  // namespace mlp
}  // namespace pd
