// pd_noalloc.cu -- diagnostics reduction that allocates no device memory.
//
// Some host applications hand this library only device buffers they have
// already allocated and do not let it call cudaMalloc themselves: the
// allocation would synchronise the device inside their time loop, their
// memory is carved from a fixed budget, or device memory is owned by another
// runtime.  pd_diagnostics_noalloc serves them: the caller passes the state
// arrays and the output buffer, and the reduction's scratch (one row of
// partial sums per thread block) lives in a fixed file-scope device array.
#include "pd_internal.h"
#include "peridem.h"

#include <mutex>

namespace {

constexpr int kNaThreads = 128;
constexpr int kNaNodesPerBlock = 2048;                           // 16 nodes per thread
constexpr int kNaMaxBlocks = PD_NOALLOC_MAX_NODES / kNaNodesPerBlock;
constexpr int kNaMaxDevices = 64;

// Scratch: per-block partial sums.  Every GPU that loads the library holds it
// (64 KiB) until the process exits.  All calls share it.
static __device__ __align__(256) double g_na_partials[kNaMaxBlocks * PD_DIAG_COUNT];

std::mutex g_na_mutex;
double *g_na_ptr[kNaMaxDevices] = {};

__global__ void __launch_bounds__(kNaThreads)
    k_na_partial(int n, const double2 *__restrict__ X, const double2 *__restrict__ u, const double2 *__restrict__ v,
                 const double *__restrict__ V, const int *__restrict__ grain, const int *__restrict__ row_ptr,
                 const int *__restrict__ col, const uint8_t *__restrict__ broken, const double *__restrict__ g_cw,
                 const double *__restrict__ g_eps, double rho, int micro, double *partials) {
    double acc[PD_DIAG_COUNT];
#pragma unroll
    for (int q = 0; q < PD_DIAG_COUNT; ++q) acc[q] = 0.0;
    const int x0 = blockIdx.x * kNaNodesPerBlock;
    const int x1 = min(n, x0 + kNaNodesPerBlock);
    for (int x = x0 + (int)threadIdx.x; x < x1; x += kNaThreads) {
        const double m = rho * V[x];
        const double2 vx = v[x], Xx = X[x], ux = u[x];
        const double px = Xx.x + ux.x, py = Xx.y + ux.y;
        acc[PD_DIAG_KE] += 0.5 * m * (vx.x * vx.x + vx.y * vx.y);
        acc[PD_DIAG_PX] += m * vx.x;
        acc[PD_DIAG_PY] += m * vx.y;
        acc[PD_DIAG_LZ] += m * (px * vx.y - py * vx.x);
        const int g = grain[x];
        const double cw = g_cw[g], eps = g_eps[g];
        for (int b = row_ptr[x]; b < row_ptr[x + 1]; ++b) {
            if (broken[b]) {
                acc[PD_DIAG_NBROKEN] += 1.0;
                continue;
            }
            const int y = col[b];
            const double2 Xy = X[y], uy = u[y];
            const double rx = Xy.x - Xx.x, ry = Xy.y - Xx.y;
            const double xi = sqrt(rx * rx + ry * ry);
            const double dx = (Xy.x + uy.x) - px, dy = (Xy.y + uy.y) - py;
            const double s = (sqrt(dx * dx + dy * dy) - xi) / xi;
            const double c = micro ? cw * (1.0 - xi / eps) : cw;
            acc[PD_DIAG_EBOND] += 0.25 * c * s * s * xi * V[x] * V[y];
        }
    }
    __shared__ double sm[PD_DIAG_COUNT][kNaThreads];
#pragma unroll
    for (int q = 0; q < PD_DIAG_COUNT; ++q) sm[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = kNaThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int q = 0; q < PD_DIAG_COUNT; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + w];
        __syncthreads();
    }
    // every block overwrites its own row: nothing of an earlier call is read
    if (threadIdx.x < PD_DIAG_COUNT) partials[blockIdx.x * PD_DIAG_COUNT + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void k_na_final(const double *partials, int nblocks, double *out) {
    const int q = threadIdx.x;
    if (q >= PD_DIAG_COUNT) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partials[b * PD_DIAG_COUNT + q];
    out[q] = s;
}

}  // namespace

extern "C" int pd_diagnostics_noalloc(int n_nodes, const double *X, const double *u, const double *v, const double *V,
                                      const int32_t *grain, const int32_t *row_ptr, const int32_t *col,
                                      const uint8_t *broken, const double *g_cw, const double *g_eps, double rho,
                                      int micromodulus, double *out, void *cuda_stream) {
    if (n_nodes < 0 || n_nodes > PD_NOALLOC_MAX_NODES)
        return pd::set_error(PD_EINVAL, "pd_diagnostics_noalloc: n_nodes must be in [0, PD_NOALLOC_MAX_NODES = 2097152]");
    if (!out) return pd::set_error(PD_EINVAL, "pd_diagnostics_noalloc: null output");
    if (n_nodes > 0 && (!X || !u || !v || !V || !grain || !row_ptr || !col || !broken || !g_cw || !g_eps))
        return pd::set_error(PD_EINVAL, "pd_diagnostics_noalloc: null input array");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return pd::set_error(PD_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kNaMaxDevices) return pd::set_error(PD_EINVAL, "pd_diagnostics_noalloc: device index too large");
    double *scratch;
    {
        // once per device, with that device current: the device address of the
        // scratch array (its name is only a host-side stand-in in host code)
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_na_partials);
            if (e != cudaSuccess) return pd::set_error(PD_ECUDA, cudaGetErrorString(e));
            g_na_ptr[dev] = (double *)p;
        }
        scratch = g_na_ptr[dev];
    }
    const int nblocks = n_nodes > 0 ? (n_nodes + kNaNodesPerBlock - 1) / kNaNodesPerBlock : 1;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    k_na_partial<<<nblocks, kNaThreads, 0, s>>>(n_nodes, (const double2 *)X, (const double2 *)u, (const double2 *)v, V,
                                                grain, row_ptr, col, broken, g_cw, g_eps, rho, micromodulus, scratch);
    k_na_final<<<1, 32, 0, s>>>(scratch, nblocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return pd::set_error(PD_ECUDA, cudaGetErrorString(e));
    return PD_OK;
}
