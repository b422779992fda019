// pd_common.cu -- precision-independent kernels of the multi-kernel step path:
// displacement update and positions (Algorithm 1), contact binning (hash-grid
// counting sort: bucket counts, device-wide exclusive scan, scatter),
// positions for readout and the diagnostics reductions; plus the launch
// dispatchers.  Compiled without FMA contraction.
#include <algorithm>
#include <cstring>

#include "pd_device.cuh"

namespace pd {

// u <- u + dt v + dt^2/2 a ; p = X + u (Algorithm 1).  Thread 0 also advances
// the step counter and sets the time of the force evaluation that follows:
// t_{n+1} = (n+1) dt.  A node that moved kSkinTrigger * skin since the last
// rebuild raises the rebuild flag; the last block to finish hands the flag to
// the conditional node of the step graph (use_cond), which runs the rebuild
// kernels only when it is set.
__global__ void __launch_bounds__(kBlock) k_predict(DevPtrs d, KParams k, int vin, int advance,
                                                    cudaGraphConditionalHandle cond, int use_cond) {
    __shared__ bool last;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    prefetch_force_inputs(d, k, i, (long long)gridDim.x * blockDim.x);
    if (blockIdx.x == 0) {
        const long long st = *d.step + (advance ? 1 : 0);
        __syncthreads();                   // every thread of block 0 has read the counter
        if (threadIdx.x == 0) {
            *d.t_now = (double)st * k.dt;
            if (advance) *d.step = st;
            // the persistent kernel's prediction of the next step no longer holds
            *d.pred_ok = 0;
        }
        wall_cells(d, k, (double)st * k.dt);
    }
    const bool need = i < k.N && predict_node<false>(d, k, i, vin, advance);
    if (__any_sync(0xffffffffu, need) && (threadIdx.x & 31) == 0) {
        *(volatile int *)d.rebuild = 1;
        __threadfence();
    }
    if (!use_cond) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(d.pred_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const int f = *(volatile int *)d.rebuild;
        *d.pred_done = 0u;
        cudaGraphSetConditional(cond, f ? 1u : 0u);
    }
}

// Rebuild of the contact candidate lists: bucket counts, a device-wide
// exclusive scan of the counts (reduce, top, apply), the counting-sort
// scatter and the lists (the list kernel clears the counts for the next
// rebuild).  Every
// kernel returns at once when the rebuild flag is clear.
__global__ void __launch_bounds__(kBlock) k_bin(DevPtrs d, KParams k) {
    if (!*(volatile int *)d.rebuild) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k.N) bin_node<false>(d, k, i);
}

__global__ void __launch_bounds__(kBlock) k_build_list(DevPtrs d, KParams k) {
    if (!*(volatile int *)d.rebuild) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) atomicAdd(&d.status[PD_STATUS_REBUILDS], 1);
    // the bucket counts were consumed by the scan: zero them for the next
    // rebuild (the grid covers max(N, T / 4) threads: one int4 per thread)
    if ((unsigned)i < k.T / 4) reinterpret_cast<int4 *>(d.count)[i] = make_int4(0, 0, 0, 0);
    if (i < k.N) build_list_node<false>(d, k, i);
}

// Block-wide exclusive scan of kScanItems values per thread.
__device__ __forceinline__ int block_exclusive_scan(int (&v)[kScanItems], int *smem_warp) {
    int local = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        int t = v[q];
        v[q] = local;
        local += t;
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) smem_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = (lane < (int)(blockDim.x / 32)) ? smem_warp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        smem_warp[lane] = wi - w;           // exclusive warp offsets
        if (lane == 31) smem_warp[32] = wi; // block total
    }
    __syncthreads();
    int base = smem_warp[warp] + (incl - local);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) v[q] += base;
    int total = smem_warp[32];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int *__restrict__ count, int *blocksums, unsigned T,
                                                              const int *flag) {
    if (!*(volatile const int *)flag) return;
    __shared__ int sm[33];
    static_assert(kScanItems == 4, "one int4 per thread");
    const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
    const int4 c4 = base < T ? *reinterpret_cast<const int4 *>(count + base) : make_int4(0, 0, 0, 0);
    int v[kScanItems] = {c4.x, c4.y, c4.z, c4.w};
    int total = block_exclusive_scan(v, sm);
    if (threadIdx.x == 0) blocksums[blockIdx.x] = total;
}

// Exclusive scan of the per-tile sums in place, kScanTile at a time with a
// running carry (any number of tiles; one block).
__global__ void __launch_bounds__(kScanThreads) k_scan_top(int *blocksums, int nblocks, const int *flag) {
    if (!*(volatile const int *)flag) return;
    __shared__ int sm[33];
    int carry = 0;
    for (int base = 0; base < nblocks; base += kScanTile) {
        int v[kScanItems];
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            const int idx = base + threadIdx.x * kScanItems + q;
            v[q] = idx < nblocks ? blocksums[idx] : 0;
        }
        const int total = block_exclusive_scan(v, sm);
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            const int idx = base + threadIdx.x * kScanItems + q;
            if (idx < nblocks) blocksums[idx] = v[q] + carry;
        }
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(int *count, const int *__restrict__ blocksums,
                                                             int *start, int *cursor, unsigned T, int N,
                                                             const int *flag) {
    if (!*(volatile const int *)flag) return;
    __shared__ int sm[33];
    // T is a power of two >= 1024 and bases are multiples of 4: whole int4 per thread
    const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
    int4 c4 = make_int4(0, 0, 0, 0);
    if (base < T) {
        c4 = *reinterpret_cast<const int4 *>(count + base);
    }
    int v[kScanItems] = {c4.x, c4.y, c4.z, c4.w};
    block_exclusive_scan(v, sm);
    const int off = blocksums[blockIdx.x];
    if (base < T) {
        const int4 st = make_int4(v[0] + off, v[1] + off, v[2] + off, v[3] + off);
        *reinterpret_cast<int4 *>(start + base) = st;
        *reinterpret_cast<int4 *>(cursor + base) = st;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) start[T] = N;
}

__global__ void __launch_bounds__(kBlock) k_scatter(DevPtrs d, KParams k) {
    if (!*(volatile int *)d.rebuild) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k.N) return;
    scatter_node<false>(d, k, i);
}

__global__ void __launch_bounds__(kBlock) k_positions(DevPtrs d, KParams k) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k.N) return;
    double2 X = d.X[i], u = d.u[i];
    d.p[i] = make_double2(X.x + u.x, X.y + u.y);
}

// Single-wall contact potential (Sec. 4.5): the energy whose derivative along
// the wall normal is minus the repulsion K_n V_x |S_l| (R_c - |c_l - p|) of
// eq. (wall-repulsive).  With the segment half-angle theta (d = R_c cos theta),
// |S_l| (R_c - |c_l - p|) = R_c^3 g(theta) and the potential is
// K_n V_x R_c^4 J(theta), J = int_0^theta g(t) sin t dt
//   = sin th - th cos th - sin^3 th / 3 - th / 4 + sin(2 th) / 6 - sin(4 th) / 48.
// J starts at th^7 / 35 and those terms cancel below th = 1; there J is
// summed from its Taylor series, J / th^7 = sum_{m>=3} C_m th^(2m-6) with
// C_m = (-1)^m c_m / (2m+1)!, c_m = 1 - (2m+1) - (3 - 3^(2m+1)) / 12
// + 2^(2m+1) / 6 - 4^(2m+1) / 48, coefficients evaluated at compile time.
__host__ __device__ constexpr double wall_energy_coef(int m) {
    double p2 = 2.0, p3 = 3.0, p4 = 4.0, fact = 1.0;
    for (int q = 1; q <= m; ++q) {
        p2 *= 4.0;
        p3 *= 9.0;
        p4 *= 16.0;
    }
    for (int q = 2; q <= 2 * m + 1; ++q) fact *= (double)q;
    const double c = 1.0 - (2.0 * m + 1.0) - (3.0 - p3) / 12.0 + p2 / 6.0 - p4 / 48.0;
    return ((m & 1) ? -c : c) / fact;
}
template <int M, int MMAX>
__device__ __forceinline__ double wall_energy_horner(double t2) {
    constexpr double c = wall_energy_coef(M);
    if constexpr (M == MMAX) return c;
    else return fma(wall_energy_horner<M + 1, MMAX>(t2), t2, c);
}
// R^4 J(theta) of a node at distance d from a wall (d < 0: taken at 0, as the force).
__device__ __forceinline__ double wall_energy_r4j(double d, double R) {
    if (!(d < R)) return 0.0;
    d = fmax(d, 0.0);
    const double th = atan2(sqrt((R - d) * (R + d)), d);
    double J;
    if (th < 1.0) {
        const double t2 = th * th;
        J = (th * t2 * t2 * t2) * wall_energy_horner<3, 22>(t2);
    } else {
        double sn, cs;
        sincos(th, &sn, &cs);
        J = sn - th * cs - sn * sn * sn / 3.0 - th / 4.0 + sin(2.0 * th) / 6.0 - sin(4.0 * th) / 48.0;
    }
    const double R2 = R * R;
    return R2 * R2 * J;
}

// Diagnostics: per-block partial sums (grid-stride, fixed order), then one
// block adds the partials in block order -- deterministic for a given grid.
// The contact potentials walk the candidate lists, which must be current (the
// caller rebuilds them first).
__global__ void __launch_bounds__(kBlock) k_diag_partial(DevPtrs d, KParams k, int vcur) {
    double acc[PD_DIAG_COUNT];
#pragma unroll
    for (int q = 0; q < PD_DIAG_COUNT; ++q) acc[q] = 0.0;
    const double2 *v = d.v[vcur];
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < k.N; x += gridDim.x * blockDim.x) {
        int g = d.grain[x];
        double m = (k.mat ? d.g_rho[g] : k.rho) * d.V[x];
        double2 vx = v[x], X = d.X[x], u = d.u[x];
        double px = X.x + u.x, py = X.y + u.y;
        acc[PD_DIAG_KE] += 0.5 * m * (vx.x * vx.x + vx.y * vx.y);
        acc[PD_DIAG_PX] += m * vx.x;
        acc[PD_DIAG_PY] += m * vx.y;
        acc[PD_DIAG_LZ] += m * (px * vx.y - py * vx.x);
        double cw = d.g_cw[g], eps = d.g_eps[g];
        int r0 = d.row_ptr[x], r1 = d.row_ptr[x + 1];
        for (int b = r0; b < r1; ++b) {
            int kk = b - r0;
            if ((d.bits[(size_t)x * k.wpn + (kk >> 5)] >> (kk & 31)) & 1u) {
                acc[PD_DIAG_NBROKEN] += 1.0;
                continue;
            }
            int y = d.col[b];
            double xi = d.xi[b];
            double2 Xy = d.X[y], uy = d.u[y];
            double dx = (Xy.x + uy.x) - px, dy = (Xy.y + uy.y) - py;
            double L = sqrt(dx * dx + dy * dy);
            double s = (L - xi) / xi;
            double c = k.micro ? cw * (1.0 - xi / eps) : cw;
            acc[PD_DIAG_EBOND] += 0.25 * c * s * s * xi * d.V[x] * d.V[y];
        }
        // contact potentials (Secs. 4.1, 4.4): 1/2 K_n V_x V_y (R_c - d)^2 between
        // grains; between unbonded nodes of one grain 1/2 (c_w / R_c) V_x V_y
        // (R_c - d)^2 for |xi| >= R_c and 1/2 (c_w / |xi|) V_x V_y (|xi| - d)^2
        // while d < |xi| < R_c.  Every pair is met from both of its nodes: each
        // adds half.
        const int ag = d.g_agg[g];
        const AggParams &A = d.agg[ag];
        const double Rc = A.Rc, Vx = d.V[x];
        const int nc = d.nbr_cnt[x];
        for (int q = 0; q < nc; ++q) {
            const int y = d.nbr[(size_t)q * k.N + x];
            const double2 Xy = d.X[y], uy = d.u[y];
            const double dx = (Xy.x + uy.x) - px, dy = (Xy.y + uy.y) - py;
            const double dd = sqrt(dx * dx + dy * dy);
            if (!(dd < Rc)) continue;
            const int gy = d.grain[y];
            if (gy != g) {
                const double Kn = k.mat ? 18.0 * harmonic64(d.g_k[g], d.g_k[gy]) / A.pe5 : A.Kn;
                acc[PD_DIAG_ECONTACT] += 0.25 * Kn * Vx * d.V[y] * (Rc - dd) * (Rc - dd);
                continue;
            }
            if (bonded_intact(d, k, x, r0, r1, y)) continue;
            const double xix = Xy.x - X.x, xiy = Xy.y - X.y;
            const double xi = sqrt(xix * xix + xiy * xiy);
            if (xi < Rc) {
                if (dd < xi) acc[PD_DIAG_ECONTACT] += 0.25 * (cw / xi) * Vx * d.V[y] * (xi - dd) * (xi - dd);
            } else {
                acc[PD_DIAG_ECONTACT] += 0.25 * (cw / Rc) * Vx * d.V[y] * (Rc - dd) * (Rc - dd);
            }
        }
        // single-wall potentials (Sec. 4.5) with the walls at the current time;
        // corner regions carry none (their term of eq. wall-total is not the
        // gradient of a potential)
        if (!far_from_walls<false>(d, x, ag)) {
            const double t = *d.t_now;
            const double Kn = k.mat ? 18.0 * d.g_k[g] / A.pe5 : A.Kn;
            const double dl[4] = {px - (A.w0[0] + A.wv[0] * t), (A.w0[1] + A.wv[1] * t) - px,
                                  py - (A.w0[2] + A.wv[2] * t), (A.w0[3] + A.wv[3] * t) - py};
            double e = 0.0;
#pragma unroll
            for (int l = 0; l < 4; ++l) e += wall_energy_r4j(dl[l], Rc);
            acc[PD_DIAG_EWALL] += Kn * Vx * e;
        }
    }
    __shared__ double sm[PD_DIAG_COUNT][kBlock];
#pragma unroll
    for (int q = 0; q < PD_DIAG_COUNT; ++q) sm[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < PD_DIAG_COUNT; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < PD_DIAG_COUNT) d.diag_part[blockIdx.x * PD_DIAG_COUNT + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void k_diag_final(DevPtrs d, int nblocks) {
    int q = threadIdx.x;
    if (q >= PD_DIAG_COUNT) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += d.diag_part[b * PD_DIAG_COUNT + q];
    d.diag_out[q] = s;
}

// ---------------------------------------------------------------------------

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

cudaError_t launch_predict(const DevPtrs &d, const KParams &k, int vin, int advance, cudaStream_t s,
                           cudaGraphConditionalHandle cond, int use_cond) {
    k_predict<<<nblk(k.N, kBlock), kBlock, 0, s>>>(d, k, vin, advance, cond, use_cond);
    return cudaGetLastError();
}

__global__ void k_widen(const float2 *__restrict__ src, double2 *__restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = make_double2((double)src[i].x, (double)src[i].y);
}

__global__ void k_narrow(const double2 *__restrict__ src, float2 *__restrict__ dst, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = make_float2(__double2float_rn(src[i].x), __double2float_rn(src[i].y));
}

cudaError_t launch_widen(const float2 *src, double2 *dst, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_widen<<<(unsigned)std::min<size_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_narrow(const double2 *src, float2 *dst, size_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_narrow<<<(unsigned)std::min<size_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_rebuild(const DevPtrs &d, const KParams &k, cudaStream_t s) {
    const int nb = nblk(k.T, kScanTile), nn = nblk(k.N, kBlock);
    k_bin<<<nn, kBlock, 0, s>>>(d, k);
    k_scan_reduce<<<nb, kScanThreads, 0, s>>>(d.count, d.blocksums, k.T, d.rebuild);
    k_scan_top<<<1, kScanThreads, 0, s>>>(d.blocksums, nb, d.rebuild);
    k_scan_apply<<<nb, kScanThreads, 0, s>>>(d.count, d.blocksums, d.start, d.cursor, k.T, k.N, d.rebuild);
    k_scatter<<<nn, kBlock, 0, s>>>(d, k);
    k_build_list<<<nblk(std::max<long long>(k.N, k.T / 4), kBlock), kBlock, 0, s>>>(d, k);
    return cudaGetLastError();
}

cudaError_t launch_force(const DevPtrs &d, const KParams &k, int vin, int update_v, cudaStream_t s, int phase) {
    return k.fp32 ? launch_force32(d, k, vin, update_v, s, phase) : launch_force64(d, k, vin, update_v, s, phase);
}

cudaError_t launch_persistent(const DevPtrs &d, const KParams &k, int vin, int nsteps, int block, cudaStream_t s) {
    return k.fp32 ? launch_persistent32(d, k, vin, nsteps, block, s)
                  : launch_persistent64(d, k, vin, nsteps, block, s);
}

cudaError_t launch_positions(const DevPtrs &d, const KParams &k, cudaStream_t s) {
    k_positions<<<nblk(k.N, kBlock), kBlock, 0, s>>>(d, k);
    return cudaGetLastError();
}

// Particle damage (Sec. 6): mean over the grain's nodes of the node damage
// broken / reference bonds (Sec. 3.1); one block per grain.
__global__ void __launch_bounds__(kBlock) k_grain_damage(DevPtrs d, KParams k, double *out) {
    __shared__ double sm[kBlock / 32];
    const int g = blockIdx.x;
    const int s0 = d.g_start[g], s1 = d.g_start[g + 1];
    double sum = 0.0;
    for (int i = s0 + threadIdx.x; i < s1; i += kBlock) {
        const int r0 = d.row_ptr[i], r1 = d.row_ptr[i + 1];
        int broken = 0;
        for (int kk = 0; kk < r1 - r0; kk += 32) {
            uint32_t w = d.bits[(size_t)i * k.wpn + (kk >> 5)];
            const int rest = r1 - r0 - kk;
            if (rest < 32) w &= (1u << rest) - 1u;
            broken += __popc(w);
        }
        if (r1 > r0) sum += (double)broken / (double)(r1 - r0);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) t += sm[w];
        out[g] = s1 > s0 ? t / (double)(s1 - s0) : 0.0;
    }
}

// Sums per aggregate of the wall terms of all nodes near a wall at the
// current state: out[16 a + 2 l + c] own segment of wall l, out[16 a + 8 + 2 q + c]
// corner q (the order of wall_terms64).
__global__ void __launch_bounds__(kBlock) k_wall_sums(DevPtrs d, KParams k, int vcur, double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k.N) return;
    const int ag = d.g_agg[d.grain[i]];
    if (far_from_walls<false>(d, i, ag)) return;
    const double2 p = d.p[i], v = d.v[vcur][i];
    const int g = d.grain[i];
    const AggParams &A = d.agg[ag];
    double single[4][2], corner[4][2];
    wall_terms64(k, A, k.mat ? 18.0 * d.g_k[g] / A.pe5 : A.Kn, k.mat ? d.g_rho[g] : k.rho, *d.t_now, p.x, p.y, v.x,
                 v.y, d.V[i], single, corner, nullptr);
    double *o = out + 16 * (size_t)ag;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (single[l][0] != 0.0) atomicAdd(&o[2 * l], single[l][0]);
        if (single[l][1] != 0.0) atomicAdd(&o[2 * l + 1], single[l][1]);
        if (corner[l][0] != 0.0) atomicAdd(&o[8 + 2 * l], corner[l][0]);
        if (corner[l][1] != 0.0) atomicAdd(&o[8 + 2 * l + 1], corner[l][1]);
    }
}

cudaError_t launch_observables(const DevPtrs &d, const KParams &k, int vcur, double *gdam, double *wsum,
                               cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(wsum, 0, sizeof(double) * 16 * (size_t)k.n_agg, s);
    if (e != cudaSuccess) return e;
    // positions, cells and wall cells of the current state (no advance, forced rebuild)
    if ((e = launch_predict(d, k, vcur, 0, s, 0, 0)) != cudaSuccess) return e;
    if ((e = launch_positions(d, k, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d.rebuild, 1, sizeof(int), s)) != cudaSuccess) return e;
    if ((e = launch_rebuild(d, k, s)) != cudaSuccess) return e;
    k_grain_damage<<<k.G, kBlock, 0, s>>>(d, k, gdam);
    k_wall_sums<<<nblk(k.N, kBlock), kBlock, 0, s>>>(d, k, vcur, wsum);
    return cudaGetLastError();
}

// Check of the integer square root of the FP64 bond loop: n pseudo-random
// positive doubles (splitmix64 of seed + i * golden ratio; exponents 2^-80 ..
// 2^20, uniform significands; every other one the exact square of a 26-bit
// significand) against the hardware's IEEE square root.
// out[0] counts mismatches, out[1] holds the bits of the first one found.
__global__ void k_check_sqrt(long long n, unsigned long long seed, unsigned long long *out) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        unsigned long long z = seed + (unsigned long long)i * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const unsigned long long e = 943ull + (z >> 52) % 101ull;
        double x = __longlong_as_double((long long)((e << 52) | (z & 0xFFFFFFFFFFFFFull)));
        if (i & 1) {
            // every other input an exact square: y with a 26-bit significand, y^2 exact
            const double y = __longlong_as_double((long long)(((1023ull - 40ull + (z >> 52) % 50ull) << 52) |
                                                              (z & 0xFFFFFF8000000ull)));
            x = __dmul_rn(y, y);
        }
        if (__double_as_longlong(sqrt_rn_int(x)) != __double_as_longlong(__dsqrt_rn(x))) {
            if (atomicAdd(&out[0], 1ull) == 0ull) out[1] = (unsigned long long)__double_as_longlong(x);
        }
    }
}

cudaError_t launch_diagnostics(const DevPtrs &d, const KParams &k, int vcur, cudaStream_t s) {
    // positions, cells and candidate lists of the current state (no advance, forced rebuild)
    cudaError_t e = launch_predict(d, k, vcur, 0, s, 0, 0);
    if (e != cudaSuccess) return e;
    if ((e = launch_positions(d, k, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(d.rebuild, 1, sizeof(int), s)) != cudaSuccess) return e;
    if ((e = launch_rebuild(d, k, s)) != cudaSuccess) return e;
    k_diag_partial<<<k.n_diag_blocks, kBlock, 0, s>>>(d, k, vcur);
    k_diag_final<<<1, 32, 0, s>>>(d, k.n_diag_blocks);
    return cudaGetLastError();
}

}  // namespace pd

extern "C" int pd_check_sqrt(long long n, unsigned long long seed, void *cuda_stream, long long *mismatches,
                             double *first_mismatch) {
    if (n < 0 || !mismatches) return pd::set_error(PD_EINVAL, "pd_check_sqrt: n >= 0 and a result pointer required");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    unsigned long long *dev = nullptr, host[2] = {0ull, 0ull};
    if (cudaMalloc(&dev, sizeof(host)) != cudaSuccess) return pd::set_error(PD_ECUDA, "pd_check_sqrt: cudaMalloc");
    cudaError_t e = cudaMemsetAsync(dev, 0, sizeof(host), s);
    if (e == cudaSuccess) {
        pd::k_check_sqrt<<<152 * 8, 256, 0, s>>>(n, seed, dev);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, dev, sizeof(host), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dev);
    if (e != cudaSuccess) return pd::set_error(PD_ECUDA, cudaGetErrorString(e));
    *mismatches = (long long)host[0];
    if (first_mismatch) {
        long long bits = (long long)host[1];
        std::memcpy(first_mismatch, &bits, sizeof(bits));
    }
    return PD_OK;
}
