// pd_surrogate.cu -- kernels of the learned per-grain modal surrogate.
//
// A grain whose bond network is a template (same shape, same lattice) is
// described in its co-rotated lattice frame: centroid c and rotation phi fit
// the current positions to the reference ones (2D Kabsch: phi = atan2(sum
// X' x p', sum X' . p')), the local deformation is
// w_i = R(-theta) (R(-phi) (p_i - c) - (X_i - Xbar)), and its modal
// coefficients q = Phi^T w / h on the template's basis Phi (lowest modes of the
// linearised bond operator K, K Phi = Phi Lambda).  The modal bond force
// f = Phi^T F / (E h) is the linear part -Lambda q plus a network's nonlinear
// correction: f = -Lambda q + net(q); the force kernel then puts
// R(theta + phi) Phi f E h in place of the bond loop.  Every judge_every steps
// the full bond kernel runs instead and the judge compares it with the
// surrogate force and checks the largest stretch, switching a grain back to
// the full bond force for good when it nears damage or the surrogate error
// grows.
//
// Per template the two basis products are dense GEMMs over all of its grains
// and run on the tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// tensor memory): the projection Q = W Phi (rows: grains, K: the 2 n_t node
// coordinates, split in chunks of kSurChunk whose partial sums are added in a
// fixed order) and the expansion F = Y Phi^T (rows: grains, N: node
// coordinates in tiles of kSurExpandRows, K: the modes).  FP32 accuracy comes
// from splitting every operand x = hi + lo into two BF16 numbers and adding
// the three products hi*hi + hi*lo + lo*hi (the split-precision scheme of
// Henry, Tang & Heinecke, "Leveraging the bfloat16 artificial intelligence
// datatype for higher-precision computations", ARITH 2019): relative error
// about 2^-16 per product, far inside the surrogate's 1e-3 tolerance.
#include <cuda_bf16.h>

#include "pd_device.cuh"
#include "pd_tc.cuh"

namespace pd {

constexpr int kSurThreads = 128;
constexpr int kMaxModes = 32;
constexpr long long kSurSpins = 1LL << 24;   // bounded mbarrier waits

__device__ __forceinline__ double block_sum_d(double v, double *sm) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kSurThreads / 32; ++w) t += sm[w];
    return t;
}

__device__ __forceinline__ float block_max_f(float v, float *sm) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < kSurThreads / 32; ++w) t = fmaxf(t, sm[w]);
    return t;
}

// Sum over the block of 32 per-thread mode accumulators; thread m < M gets
// the total of mode m.
__device__ __forceinline__ float block_sum_modes(const float (&acc)[kMaxModes], float (*sm)[kSurThreads], int M) {
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kMaxModes; ++m) sm[m][threadIdx.x] = acc[m];
    __syncthreads();
    float v = 0.f;
    if ((int)threadIdx.x < M)
        for (int q = 0; q < kSurThreads; ++q) v += sm[threadIdx.x][q];
    return v;
}

// Padded basis rows of template t (a multiple of kSurExpandRows).
__device__ __forceinline__ int tmpl_rows_pad(const DevPtrs &d, int t) { return d.tmpl_rows[t + 1] - d.tmpl_rows[t]; }

// ---------------------------------------------------------------------------
// co-rotated frame and local deformation

__device__ __forceinline__ float block_sum_f(float v, float *sm) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < kSurThreads / 32; ++w) t += sm[w];
    return t;
}

// (ah + al) * (bh + bl) as a float-float pair (the al * bl term is below the pair's precision).
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float &ph, float &pl) {
    float e;
    two_prod(ah, bh, ph, e);
    pl = e + (ah * bl + al * bh);
}

// Co-rotated frame of grain blockIdx.x and its local deformation w / h per node
// (into sur_w).  Grains without a template, or not active (unless
// all_templated), are skipped.
//
// Everything runs on the FP32 pipe.  The frame (centroid c, rotation phi)
// needs no more than float accuracy: an error in it adds a rigid translation
// or rotation to w, and the basis, orthogonal to the rigid modes, projects it
// out.  The deformation itself is a small difference of two quantities of the
// size of the grain, so positions relative to the grain's first node are
// float-float pairs (exact high-part differences of the shifted positions
// plus the low parts), and the rotation R(-theta - phi) and the reference
// offset h (lattice index - lattice centroid) are applied in float-float.
__global__ void __launch_bounds__(kSurThreads) k_sur_frame(DevPtrs d, KParams k, int all_templated) {
    __shared__ float frame[6];
    tc::grid_dep_launch();     // the projection may begin staging its basis chunks
    const int g = blockIdx.x;
    const int t = d.g_tmpl[g];
    if (t < 0 || (!all_templated && !d.sur_active[g])) return;
    const int s0 = d.g_start[g], s1 = d.g_start[g + 1], n = s1 - s0;
    const float4 fc = d.sur_fc[g];                 // (h hi, h lo, lattice centroid i, j)
    const float4 q0 = d.pq[s0];
    const float2 ph0 = make_float2(q0.x, q0.y), pl0 = make_float2(q0.z, q0.w);
    // one pass: centroid and the best-fit rotation sums in the lattice frame,
    // A = sum l . d, B = sum l x d (l: centred lattice index, d = p - p_first)
    float sx = 0.f, sy = 0.f, sa = 0.f, sb = 0.f;
    // nodes in batches of kFrameBatch per thread, all loads of a batch first
    // (the per-thread order of the sums is unchanged)
    constexpr int kFrameBatch = 4;
    for (int i0 = s0 + threadIdx.x; i0 < s1; i0 += kFrameBatch * kSurThreads) {
      float4 qb[kFrameBatch];
      int2 lb[kFrameBatch];
#pragma unroll
      for (int m = 0; m < kFrameBatch; ++m) {
          const int i = min(i0 + m * kSurThreads, s1 - 1);
          qb[m] = d.pq[i];
          lb[m] = d.lat[i];
      }
#pragma unroll
      for (int m = 0; m < kFrameBatch; ++m) {
        if (i0 + m * kSurThreads >= s1) break;
        const float4 qn = qb[m];
        const float2 ph = make_float2(qn.x, qn.y), pl = make_float2(qn.z, qn.w);
        const int2 li = lb[m];
        const float dx = __fsub_rn(ph.x, ph0.x) + (pl.x - pl0.x), dy = __fsub_rn(ph.y, ph0.y) + (pl.y - pl0.y);
        const float lx = (float)li.x - fc.z, ly = (float)li.y - fc.w;
        sx += dx;
        sy += dy;
        sa += lx * dx + ly * dy;
        sb += lx * dy - ly * dx;
      }
    }
    // the four sums in one block reduction
    __shared__ float4 sm4[kSurThreads / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, off);
        sy += __shfl_xor_sync(0xffffffffu, sy, off);
        sa += __shfl_xor_sync(0xffffffffu, sa, off);
        sb += __shfl_xor_sync(0xffffffffu, sb, off);
    }
    if ((threadIdx.x & 31) == 0) sm4[threadIdx.x >> 5] = make_float4(sx, sy, sa, sb);
    __syncthreads();
    if (threadIdx.x == 0) {
        float Sx = 0.f, Sy = 0.f, A = 0.f, Bs = 0.f;
        for (int w = 0; w < kSurThreads / 32; ++w) {
            Sx += sm4[w].x;
            Sy += sm4[w].y;
            A += sm4[w].z;
            Bs += sm4[w].w;
        }
        // reference offsets X' = R(theta) h l: sum X' . p' = cos A + sin B, sum X' x p' = cos B - sin A,
        // so the best-fit phi = atan2(cos B - sin A, cos A + sin B), and the angle sum reduces to
        // (cos, sin)(theta + phi) = (A, B) / |(A, B)|: no trigonometry on the block's critical path
        const double Ad = A, Bd = Bs, r2 = Ad * Ad + Bd * Bd;
        double cr, sr;
        if (r2 > 0.0) {
            const double ir = 1.0 / sqrt(r2);
            cr = Ad * ir;
            sr = Bd * ir;
        } else {
            sincos(d.g_theta[g], &sr, &cr);      // no deformation information: phi = 0
        }
        d.sur_rot[g] = make_float2((float)cr, (float)sr);
        const float ch = (float)cr, sh = (float)sr;
        frame[0] = ch;
        frame[1] = (float)(cr - (double)ch);
        frame[2] = sh;
        frame[3] = (float)(sr - (double)sh);
        frame[4] = Sx / (float)n;                  // centroid, relative to the first node
        frame[5] = Sy / (float)n;
    }
    __syncthreads();
    const float ch = frame[0], cl = frame[1], sh = frame[2], sl = frame[3], cx = frame[4], cy = frame[5];
    const float hinv = 1.0f / fc.x;
    for (int i0 = s0 + threadIdx.x; i0 < s1; i0 += kFrameBatch * kSurThreads) {
      float4 qb[kFrameBatch];
      int2 lb[kFrameBatch];
#pragma unroll
      for (int m = 0; m < kFrameBatch; ++m) {
          const int i = min(i0 + m * kSurThreads, s1 - 1);
          qb[m] = d.pq[i];
          lb[m] = d.lat[i];
      }
#pragma unroll
      for (int m = 0; m < kFrameBatch; ++m) {
        const int i = i0 + m * kSurThreads;
        if (i >= s1) break;
        const float4 qn = qb[m];
        const float2 ph = make_float2(qn.x, qn.y), pl = make_float2(qn.z, qn.w);
        const int2 li = lb[m];
        // e = p - c as float-float pairs
        float exh, exe, eyh, eye;
        two_sum(__fsub_rn(ph.x, ph0.x), -cx, exh, exe);
        two_sum(__fsub_rn(ph.y, ph0.y), -cy, eyh, eye);
        const float exl = exe + (pl.x - pl0.x), eyl = eye + (pl.y - pl0.y);
        // u = R(-theta - phi) e
        float p1h, p1l, p2h, p2l, q1h, q1l, q2h, q2l;
        ff_mul(ch, cl, exh, exl, p1h, p1l);        // c ex
        ff_mul(sh, sl, eyh, eyl, p2h, p2l);        // s ey
        ff_mul(sh, sl, exh, exl, q1h, q1l);        // s ex
        ff_mul(ch, cl, eyh, eyl, q2h, q2l);        // c ey
        float uxh, uxe, uyh, uye;
        two_sum(p1h, p2h, uxh, uxe);
        two_sum(q2h, -q1h, uyh, uye);
        const float uxl = uxe + (p1l + p2l), uyl = uye + (q2l - q1l);
        // reference offset h l as float-float pairs
        const float lx = (float)li.x - fc.z, ly = (float)li.y - fc.w;
        float rxh, rxe, ryh, rye;
        two_prod(fc.x, lx, rxh, rxe);
        two_prod(fc.x, ly, ryh, rye);
        const float rxl = rxe + fc.y * lx, ryl = rye + fc.y * ly;
        const float wx = __fsub_rn(uxh, rxh) + (uxl - rxl), wy = __fsub_rn(uyh, ryh) + (uyl - ryl);
        d.sur_w[i] = make_float2(wx * hinv, wy * hinv);
      }
    }
}

// ---------------------------------------------------------------------------
// CUDA-core projection (sampling and checks): out[g] = Phi^T v for every
// templated grain, v = sur_w, or v = R(-theta - phi) F / (E h) when F is given.

__global__ void __launch_bounds__(kSurThreads) k_sur_project_cc(DevPtrs d, KParams k, const double2 *F,
                                                                 float *out) {
    __shared__ float smq[kMaxModes][kSurThreads];
    const int g = blockIdx.x;
    const int t = d.g_tmpl[g];
    if (t < 0) return;
    const int s0 = d.g_start[g], s1 = d.g_start[g + 1];
    const int M = k.n_modes;
    const int rp = tmpl_rows_pad(d, t);
    const float2 rot = d.sur_rot[g];
    const float scale = 1.0f / (k.E * __ldg(&d.gq[__ldg(&d.grain[s0])]).x);
    const float *B = d.basis + (size_t)d.tmpl_rows[t] * M;
    float acc[kMaxModes];
#pragma unroll
    for (int m = 0; m < kMaxModes; ++m) acc[m] = 0.f;
    for (int i = s0 + threadIdx.x; i < s1; i += kSurThreads) {
        float lx, ly;
        if (F) {
            const double2 f = F[i];
            const float fx = (float)f.x * scale, fy = (float)f.y * scale;
            lx = rot.x * fx + rot.y * fy;
            ly = -rot.y * fx + rot.x * fy;
        } else {
            const float2 w = d.sur_w[i];
            lx = w.x;
            ly = w.y;
        }
        const int r = 2 * (i - s0);
#pragma unroll
        for (int m = 0; m < kMaxModes; ++m)
            if (m < M) {
                const float2 b = *reinterpret_cast<const float2 *>(B + (size_t)m * rp + r);
                acc[m] += b.x * lx + b.y * ly;
            }
    }
    const float v = block_sum_modes(acc, smq, M);
    if ((int)threadIdx.x < M) out[(size_t)g * M + threadIdx.x] = v;
}

// ---------------------------------------------------------------------------
// tensor-core basis products

__device__ __forceinline__ uint32_t split_pack(float a, float b, uint32_t &lo) {
    const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
    const __nv_bfloat16 al = __float2bfloat16_rn(a - __bfloat162float(ah));
    const __nv_bfloat16 bl = __float2bfloat16_rn(b - __bfloat162float(bh));
    lo = (uint32_t)__bfloat16_as_ushort(al) | ((uint32_t)__bfloat16_as_ushort(bl) << 16);
    return (uint32_t)__bfloat16_as_ushort(ah) | ((uint32_t)__bfloat16_as_ushort(bh) << 16);
}

// hi*hi + hi*lo + lo*hi over K/16 steps into the TMEM accumulator; one thread.
__device__ __forceinline__ void split_mma(uint32_t tmem, const uint8_t *ahi, const uint8_t *alo, const uint8_t *bhi,
                                          const uint8_t *blo, int arows, int brows, int K, uint32_t idesc) {
    const uint32_t lbo_a = tc::kmajor_lbo(arows), lbo_b = tc::kmajor_lbo(brows);
    uint32_t acc = 0;
    for (int ks = 0; ks < K / 16; ++ks) {
        const uint32_t oa = (uint32_t)ks * 2 * lbo_a, ob = (uint32_t)ks * 2 * lbo_b;
        const uint64_t a_h = tc::smem_desc(tc::smem_addr(ahi) + oa, lbo_a, tc::kSbo);
        const uint64_t a_l = tc::smem_desc(tc::smem_addr(alo) + oa, lbo_a, tc::kSbo);
        const uint64_t b_h = tc::smem_desc(tc::smem_addr(bhi) + ob, lbo_b, tc::kSbo);
        const uint64_t b_l = tc::smem_desc(tc::smem_addr(blo) + ob, lbo_b, tc::kSbo);
        tc::mma_bf16(tmem, a_h, b_h, idesc, acc);
        acc = 1;
        tc::mma_bf16(tmem, a_h, b_l, idesc, 1);
        tc::mma_bf16(tmem, a_l, b_h, idesc, 1);
    }
}

constexpr int kProjSmem = 96 * 1024;     // A hi/lo 128 x 128, B hi/lo 32 x 128 (80 KB used)
// A hi/lo 128 x 32, B hi/lo 128 x 32 (32 KB) and the store staging, 4 x 128 rows of 32 + 1 floats (66 KB)
constexpr int kExpSmem = 100 * 1024;
// Threads of the expansion tile: four warpgroups.  Warp w reads TMEM lanes
// 32 (w % 4) .. 32 (w % 4) + 31, so the thread's TMEM lane (its grain row of
// the tile) is tid % 128 and warpgroup tid / 128 takes a quarter of the
// operand staging and of the accumulator columns.
constexpr int kExpThreads = 512;
constexpr int kExpGroups = kExpThreads / kSurTile;

// Projection tile: network rows [s0, s0 + 128) of template t times basis rows
// [r0, r0 + kSurChunk): partial modal coefficients into sur_xpart[chunk].
__global__ void __launch_bounds__(128) k_sur_project_tc(DevPtrs d, KParams k) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    constexpr int KC = kSurChunk, MR = kSurTile, NM = kMaxModes;
    uint8_t *sAh = sm, *sAl = sm + MR * KC * 2, *sBh = sm + 2 * MR * KC * 2, *sBl = sBh + NM * KC * 2;
    const int4 wk = d.proj_work[blockIdx.x];
    const int t = wk.x, s0 = wk.y, r0 = wk.z, chunk = wk.w;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int M = k.n_modes;
    const int slot0 = d.tmpl_slot[t], Gt = d.tmpl_slot[t + 1] - slot0;
    const int rows2 = 2 * (d.tmpl_node[t + 1] - d.tmpl_node[t]);
    const int rp = tmpl_rows_pad(d, t);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    // B (the basis chunk, mode-major, 16-byte pieces) and A (local deformation
    // rows of the tile's grains, zero outside) staged with their loads in flight
    // together: the B pieces and the first half of the row, then the second half
    {
        const uint16_t *bh = d.bmm_hi + (size_t)d.tmpl_rows[t] * M;
        const uint16_t *bl = d.bmm_lo + (size_t)d.tmpl_rows[t] * M;
        constexpr int nb = NM * (KC / 8) / 128;
        static_assert(NM * (KC / 8) % 128 == 0, "basis pieces must divide over the 128 threads");
        uint4 vh[nb], vl[nb];
#pragma unroll
        for (int q = 0; q < nb; ++q) {
            const int e = tid + q * 128, m = e / (KC / 8), k8 = (e % (KC / 8)) * 8;
            vh[q] = vl[q] = make_uint4(0, 0, 0, 0);
            if (m < M) {
                vh[q] = *reinterpret_cast<const uint4 *>(bh + (size_t)m * rp + r0 + k8);
                vl[q] = *reinterpret_cast<const uint4 *>(bl + (size_t)m * rp + r0 + k8);
            }
        }
        const int s = s0 + tid;
        int g = -1;
        if (s < Gt) {
            g = d.slot_grain[slot0 + s];
            if (!d.sur_active[g]) g = -1;
        }
        const float *w = g >= 0 ? reinterpret_cast<const float *>(d.sur_w) + 2 * (size_t)d.g_start[g] : nullptr;
        // the frame kernel's deformation rows are read only after it has finished
        tc::grid_dep_wait();
        if (warp == 0) tc::tmem_alloc(&tmem_base, 32);
        constexpr int kLoadBatch = 16;                   // pairs per batch: four batches per chunk
        static_assert(KC % (2 * kLoadBatch) == 0, "chunk must hold whole batches");
#pragma unroll 1
        for (int kb = 0; kb < KC; kb += 2 * kLoadBatch) {
            float2 v[kLoadBatch];
#pragma unroll
            for (int q = 0; q < kLoadBatch; ++q) {
                const int r = r0 + kb + 2 * q;
                v[q] = (w && r < rows2) ? *reinterpret_cast<const float2 *>(w + r) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < kLoadBatch; ++q) {
                const int kk = kb + 2 * q;
                uint32_t lo;
                const uint32_t hi = split_pack(v[q].x, v[q].y, lo);
                *reinterpret_cast<uint32_t *>(sAh + tc::kmajor_off(tid, kk, MR)) = hi;
                *reinterpret_cast<uint32_t *>(sAl + tc::kmajor_off(tid, kk, MR)) = lo;
            }
        }
#pragma unroll
        for (int q = 0; q < nb; ++q) {
            const int e = tid + q * 128, m = e / (KC / 8), k8 = (e % (KC / 8)) * 8;
            *reinterpret_cast<uint4 *>(sBh + tc::kmajor_off(m, k8, NM)) = vh[q];
            *reinterpret_cast<uint4 *>(sBl + tc::kmajor_off(m, k8, NM)) = vl[q];
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tc::grid_dep_launch();
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        split_mma(tmem, sAh, sAl, sBh, sBl, MR, NM, KC, tc::idesc_bf16(MR, NM));
        tc::mma_commit(&mbar);
    }
    const bool ok = __syncthreads_and(tc::mbar_wait(&mbar, 0, kSurSpins)) != 0;
    if (ok) {
        tc::fence_after_sync();
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        const int s = s0 + tid;
        float *dst = d.sur_xpart + ((size_t)chunk * k.G + slot0 + s) * M;
        for (int c0 = 0; c0 < NM; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
            if (s < Gt)
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (c0 + q < M) dst[c0 + q] = v[q];
        }
    } else {
        // drain the timed-out phase before the columns are released; the tile's
        // results are invalid and the surrogate is not used from now on
        tc::mbar_wait(&mbar, 0, kSurSpins);
        if (tid == 0) atomicAdd(&d.status[PD_STATUS_TIMEOUT], 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem_base, 32);
}

// Network input rows: sum of the projection partials in chunk order.
__global__ void k_sur_reduce(DevPtrs d, KParams k) {
    const int row = blockIdx.x;                  // network row
    const int m = threadIdx.x;
    tc::grid_dep_launch();                       // the networks may begin staging their weights
    if (m >= k.n_modes) return;
    const int g = d.slot_grain[row];
    const int t = d.g_tmpl[g];
    const int nch = tmpl_rows_pad(d, t) / kSurChunk;
    tc::grid_dep_wait();                         // the projection's partials
    // eight partials in flight at a time, added in chunk order
    constexpr int kBatch = 8;
    float v = 0.f;
    for (int c0 = 0; c0 < nch; c0 += kBatch) {
        float p[kBatch];
#pragma unroll
        for (int j = 0; j < kBatch; ++j)
            p[j] = c0 + j < nch ? d.sur_xpart[((size_t)(c0 + j) * k.G + row) * k.n_modes + m] : 0.f;
#pragma unroll
        for (int j = 0; j < kBatch; ++j)
            if (c0 + j < nch) v += p[j];
    }
    d.sur_x[(size_t)row * k.n_modes + m] = v;
}

// Expansion tile: network rows [s0, s0 + 128) of template t times basis rows
// [r0, r0 + kSurExpandRows): surrogate bond force / (E h) of the tile's nodes
// in the lattice frame, into sur_f (active grains only).
__global__ void __launch_bounds__(kExpThreads) k_sur_expand_tc(DevPtrs d, KParams k) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    constexpr int NR = kSurExpandRows, MR = kSurTile, KM = kMaxModes;
    uint8_t *sAh = sm, *sAl = sm + MR * KM * 2, *sBh = sm + 2 * MR * KM * 2, *sBl = sBh + NR * KM * 2;
    const int4 wk = d.exp_work[blockIdx.x];
    const int t = wk.x, s0 = wk.y, r0 = wk.z;
    const int tid = threadIdx.x, warp = tid >> 5, wg = warp >> 2, lrow = tid & (MR - 1), lane = tid & 31;
    const int M = k.n_modes;
    const int slot0 = d.tmpl_slot[t], Gt = d.tmpl_slot[t + 1] - slot0;
    const int rows2 = 2 * (d.tmpl_node[t + 1] - d.tmpl_node[t]);
    if (tid == 0) tc::mbar_init(&mbar, 1);
    const int s = s0 + lrow;
    int g = -1;
    if (s < Gt) {
        g = d.slot_grain[slot0 + s];
        if (!d.sur_active[g]) g = -1;
    }
    // first node coordinate of the row's grain in the per-node arrays (-1: none)
    const int fbase = g >= 0 ? 2 * d.g_start[g] : -1;
    // A (network outputs of the tile's grains, modes [KM/4 wg, KM/4 (wg + 1)) per
    // warpgroup) and B (basis rows, node-major: each row the modes of one node
    // coordinate): every load before the first store
    {
        constexpr int kPer = KM / kExpGroups;
        static_assert(kPer % 2 == 0 && KM % kExpGroups == 0, "whole pairs per warpgroup");
        constexpr int nb = NR * (KM / 8) / kExpThreads;
        static_assert(NR * (KM / 8) % kExpThreads == 0, "basis pieces must divide over the threads");
        const float *y = g >= 0 ? d.sur_y + (size_t)(slot0 + s) * M : nullptr;
        const uint16_t *bh = d.bnm_hi + ((size_t)d.tmpl_rows[t] + r0) * M;
        const uint16_t *bl = d.bnm_lo + ((size_t)d.tmpl_rows[t] + r0) * M;
        float yv[kPer];
        uint4 vh[nb], vl[nb];
#pragma unroll
        for (int q = 0; q < nb; ++q) {
            const int e = tid + q * kExpThreads, r = e / (KM / 8), k8 = (e % (KM / 8)) * 8;
            vh[q] = vl[q] = make_uint4(0, 0, 0, 0);
            if (k8 < M) {
                vh[q] = *reinterpret_cast<const uint4 *>(bh + (size_t)r * M + k8);
                vl[q] = *reinterpret_cast<const uint4 *>(bl + (size_t)r * M + k8);
            }
        }
        // the network outputs only after the networks have finished
        tc::grid_dep_wait();
        if (warp == 0) tc::tmem_alloc(&tmem_base, NR);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int kk = kPer * wg + q;
            yv[q] = (y && kk < M) ? y[kk] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < kPer; q += 2) {
            const int kk = kPer * wg + q;
            uint32_t lo;
            const uint32_t hi = split_pack(yv[q], yv[q + 1], lo);
            *reinterpret_cast<uint32_t *>(sAh + tc::kmajor_off(lrow, kk, MR)) = hi;
            *reinterpret_cast<uint32_t *>(sAl + tc::kmajor_off(lrow, kk, MR)) = lo;
        }
#pragma unroll
        for (int q = 0; q < nb; ++q) {
            const int e = tid + q * kExpThreads, r = e / (KM / 8), k8 = (e % (KM / 8)) * 8;
            *reinterpret_cast<uint4 *>(sBh + tc::kmajor_off(r, k8, NR)) = vh[q];
            *reinterpret_cast<uint4 *>(sBl + tc::kmajor_off(r, k8, NR)) = vl[q];
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    tc::grid_dep_launch();
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        split_mma(tmem, sAh, sAl, sBh, sBl, MR, NR, KM, tc::idesc_bf16(MR, NR));
        tc::mma_commit(&mbar);
    }
    const bool ok = __syncthreads_and(tc::mbar_wait(&mbar, 0, kSurSpins)) != 0;
    if (ok) {
        tc::fence_after_sync();
        // columns [NR/4 wg, NR/4 (wg + 1)) of the thread's row, staged in shared
        // memory so that a warp stores one grain's 32 consecutive values per
        // instruction (the warp's rows are its own threads' rows: no block barrier)
        constexpr int kCols = NR / kExpGroups, kStride = kCols + 1;
        static_assert(kCols == 32, "one column per lane in the coalesced store");
        static_assert(2 * MR * KM * 2 + 2 * NR * KM * 2 + kExpGroups * MR * kStride * 4 <= kExpSmem,
                      "operands and staging fit the shared memory");
        float *stage = reinterpret_cast<float *>(sm + 2 * MR * KM * 2 + 2 * NR * KM * 2) + (size_t)wg * MR * kStride;
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
#pragma unroll
        for (int c0 = 0; c0 < kCols; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + lane_base + (uint32_t)(kCols * wg + c0), v);
#pragma unroll
            for (int q = 0; q < 16; ++q) stage[lrow * kStride + c0 + q] = v[q];
        }
        __syncwarp();
        const int rw0 = (warp & 3) * 32;
        const int r = r0 + kCols * wg + lane;
        float *sf = reinterpret_cast<float *>(d.sur_f);
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const int bj = __shfl_sync(0xffffffffu, fbase, j);    // no load in the store loop
            if (bj >= 0 && r < rows2) sf[(size_t)bj + r] = stage[(rw0 + j) * kStride + lane];
        }
    } else {
        // drain the timed-out phase before the columns are released; the tile's
        // results are invalid and the surrogate is not used from now on
        tc::mbar_wait(&mbar, 0, kSurSpins);
        if (tid == 0) atomicAdd(&d.status[PD_STATUS_TIMEOUT], 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem_base, NR);
}

// ---------------------------------------------------------------------------
// judge

// Judge (every judge_every steps): relative error of the surrogate nodal bond
// force against the full one (floored at the grain's weight), relative error
// of the modal bond force (what the network predicts), and the largest
// |s| / s0 over the grain's intact bonds; a grain that exceeds the stretch
// gate or the nodal error tolerance leaves the surrogate for good.
__device__ __forceinline__ void judge_grain(const DevPtrs &d, const KParams &k, int g) {
    __shared__ double smd[kSurThreads / 32];
    __shared__ float smf[kSurThreads / 32];
    __shared__ float smq[kMaxModes][kSurThreads];
    if (d.g_tmpl[g] < 0 || !d.sur_active[g]) return;
    const int t = d.g_tmpl[g];
    const int s0 = d.g_start[g], s1 = d.g_start[g + 1], n = s1 - s0;
    const int M = k.n_modes;
    const int rp = tmpl_rows_pad(d, t);
    const int gi = d.grain[s0];
    const float4 gq = d.gq[gi];
    const float Eh = k.E * gq.x;
    const float2 rot = d.sur_rot[g];
    const float *B = d.basis + (size_t)d.tmpl_rows[t] * M;
    const float *y = d.sur_y + (size_t)(d.tmpl_slot[t] + d.g_slot[g]) * M;
    const float s0g = (float)d.g_s0[gi];
    double e2 = 0.0, r2 = 0.0;
    float maxs = 0.f;
    float acc[kMaxModes];
#pragma unroll
    for (int m = 0; m < kMaxModes; ++m) acc[m] = 0.f;
    for (int i = s0 + threadIdx.x; i < s1; i += kSurThreads) {
        const float2 fl = d.sur_f[i];
        const float sx = (rot.x * fl.x - rot.y * fl.y) * Eh, sy = (rot.y * fl.x + rot.x * fl.y) * Eh;
        const float2 full = d.sur_fb[i];
        e2 += (double)(sx - full.x) * (sx - full.x) + (double)(sy - full.y) * (sy - full.y);
        r2 += (double)full.x * full.x + (double)full.y * full.y;
        // modal projection of the full bond force
        const float fx = full.x / Eh, fy = full.y / Eh;
        const float lx = rot.x * fx + rot.y * fy, ly = -rot.y * fx + rot.x * fy;
        const int r = 2 * (i - s0);
#pragma unroll
        for (int m = 0; m < kMaxModes; ++m)
            if (m < M) {
                const float2 b = *reinterpret_cast<const float2 *>(B + (size_t)m * rp + r);
                acc[m] += b.x * lx + b.y * ly;
            }
        // largest stretch of the node's intact bonds (float-float, as the force kernel)
        const float4 qi = d.pq[i];
        const float2 phi = make_float2(qi.x, qi.y), pli = make_float2(qi.z, qi.w);
        const int2 li = d.lat[i];
        const int r0 = d.row_ptr[i], r1 = d.row_ptr[i + 1];
        for (int b = r0; b < r1; ++b) {
            const int kk = b - r0;
            if ((d.bits[(size_t)i * k.wpn + (kk >> 5)] >> (kk & 31)) & 1u) continue;
            const int j = d.col[b];
            const float4 qj = d.pq[j];
            const float2 phj = make_float2(qj.x, qj.y), plj = make_float2(qj.z, qj.w);
            const int2 lj = d.lat[j];
            float L2h, L2l;
            len2_ff(__fsub_rn(phj.x, phi.x), plj.x - pli.x, __fsub_rn(phj.y, phi.y), plj.y - pli.y, L2h, L2l);
            const int di = lj.x - li.x, dj = lj.y - li.y;
            const float nn = (float)(di * di + dj * dj);
            float q, eq;
            two_prod(nn, gq.y, q, eq);
            const float xi = gq.x * sqrtf(nn);
            const float s = ff_diff(L2h, L2l, q, eq + nn * gq.z) / (xi * (sqrtf(L2h) + xi));
            maxs = fmaxf(maxs, fabsf(s) / s0g);
        }
    }
    const float fm = block_sum_modes(acc, smq, M);
    const float dm = (int)threadIdx.x < M ? fm - y[threadIdx.x] : 0.f;
    const double M2 = block_sum_d((double)dm * dm, smd);
    const double F2 = block_sum_d((int)threadIdx.x < M ? (double)fm * fm : 0.0, smd);
    const double E2 = block_sum_d(e2, smd);
    const double R2 = block_sum_d(r2, smd);
    const float mx = block_max_f(maxs, smf);
    if (threadIdx.x == 0) {
        const double floor_f = k.rho * (double)gq.w * fmax(sqrt(k.gx * k.gx + k.gy * k.gy), 100.0);
        const double err = sqrt(E2 / fmax(R2, (double)n * floor_f * floor_f));
        const double floor_m = floor_f / (double)Eh;
        const double merr = sqrt(M2 / fmax(F2, (double)n * floor_m * floor_m));
        d.sur_err[g] = (float)err;
        d.sur_merr[g] = (float)merr;
        d.sur_maxs[g] = mx;
        if (mx > k.gate || err > k.err_tol) d.sur_active[g] = 0;
    }
}

// One block per grain in a grid stride (the launch is in every step's graph;
// between judge steps it returns at once).
__global__ void __launch_bounds__(kSurThreads) k_sur_judge(DevPtrs d, KParams k) {
    if (!sur_healthy(d)) {
        // a tensor-core wait gave up: every grain leaves the surrogate
        if (threadIdx.x == 0)
            for (int g = blockIdx.x; g < k.G; g += gridDim.x) d.sur_active[g] = 0;
        return;
    }
    if ((*d.step) % k.judge_every != 0) return;
    for (int g = blockIdx.x; g < k.G; g += gridDim.x) {
        judge_grain(d, k, g);
        __syncthreads();          // shared scratch reused by the next grain
    }
}

// ---------------------------------------------------------------------------
// launchers

cudaError_t launch_sur_frame(const DevPtrs &d, const KParams &k, int all_templated, cudaStream_t s) {
    k_sur_frame<<<k.G, kSurThreads, 0, s>>>(d, k, all_templated);
    return cudaGetLastError();
}

cudaError_t launch_sur_project_cc(const DevPtrs &d, const KParams &k, const double2 *F, float *out, cudaStream_t s) {
    k_sur_project_cc<<<k.G, kSurThreads, 0, s>>>(d, k, F, out);
    return cudaGetLastError();
}

cudaError_t sur_init_attributes() {
    cudaError_t e = cudaFuncSetAttribute(k_sur_project_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kProjSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_sur_expand_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kExpSmem);
}

cudaError_t launch_sur_project_tc(const DevPtrs &d, const KParams &k, cudaStream_t s, bool pdl) {
    if (k.n_proj_work == 0) return cudaSuccess;
    return launch_ex(k_sur_project_tc, dim3(k.n_proj_work), dim3(128), kProjSmem, s, pdl, d, k);
}

cudaError_t launch_sur_reduce(const DevPtrs &d, const KParams &k, cudaStream_t s, bool pdl) {
    if (k.n_rows == 0) return cudaSuccess;
    return launch_ex(k_sur_reduce, dim3(k.n_rows), dim3(32), 0, s, pdl, d, k);
}

cudaError_t launch_sur_expand_tc(const DevPtrs &d, const KParams &k, cudaStream_t s, bool pdl) {
    if (k.n_exp_work == 0) return cudaSuccess;
    return launch_ex(k_sur_expand_tc, dim3(k.n_exp_work), dim3(kExpThreads), kExpSmem, s, pdl, d, k);
}

cudaError_t launch_sur_judge(const DevPtrs &d, const KParams &k, cudaStream_t s) {
    k_sur_judge<<<k.G < 152 * 8 ? k.G : 152 * 8, kSurThreads, 0, s>>>(d, k);
    return cudaGetLastError();
}

}  // namespace pd
