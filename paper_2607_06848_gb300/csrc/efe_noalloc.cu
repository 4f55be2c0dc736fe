// Quadrature integral without any device allocation, for callers that cannot
// call cudaMalloc while they run: code inside a region whose memory is owned
// by another allocator, or a host that must not grow device memory after
// start-up.  Same value as efe_integrate; the per-cell partial sums live in a
// fixed, file-scope device array instead of a buffer allocated by the library.
#include "efe_internal.cuh"
#include "efe_funcs.cuh"

#include <atomic>
#include <cstdio>
#include <mutex>

namespace {

// One double per cell plus one slot for the total.  Every GPU that loads the
// library holds this array (512 KB + 8 B) until the process exits.
constexpr int kNoallocMaxCells = 65536;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocMaxCells + 1];

// Per-device address of g_noalloc_scratch.  In host code the symbol's name is
// only a host-side stand-in; the device address comes from
// cudaGetSymbolAddress with that device current, once per device, and is
// cached for the life of the process (the lookup is serialised by a mutex so
// that two host threads making their first call at once do not race).
constexpr int kMaxDevices = 64;
std::atomic<double *> g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

// Address of the array on `dev` (the context's device), current device unchanged on return.
cudaError_t scratch_address(int dev, double **out) {
    double *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (p) {
        *out = p;
        return cudaSuccess;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        int cur = 0;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return e;
        if (cur != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return e;
        e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_scratch);
        if (cur != dev) cudaSetDevice(cur);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return cudaSuccess;
}

// Makes `dev` current for the scope of one call and restores the caller's device.
struct DeviceScope {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceScope(int dev) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
        else if (err == cudaSuccess) prev = -1;
    }
    ~DeviceScope() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// scratch[c] = sum over the Gauss points of cell c of w_q J a(q) [b(q)]
__global__ void k_cell_integrals(MeshDev m, Tables1D T, const double *a, const double *b, double *scratch) {
    __shared__ double red[32];
    const int c = blockIdx.x;
    const double J = 0.125 * m.h * m.h * m.h;
    double s = 0.0;
    for (int q = threadIdx.x; q < m.nq3; q += blockDim.x) {
        const int qx = q % m.nq, qy = (q / m.nq) % m.nq, qz = q / (m.nq * m.nq);
        const size_t i = (size_t)c * m.nq3 + q;
        s += T.wq[qx] * T.wq[qy] * T.wq[qz] * J * a[i] * (b ? b[i] : 1.0);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        scratch[c] = t;
    }
}

// scratch[ncells] = sum of the per-cell values (one block, fixed order)
__global__ void k_sum_cells(int ncells, double *scratch) {
    __shared__ double red[32];
    double s = 0.0;
    for (int c = threadIdx.x; c < ncells; c += blockDim.x) s += scratch[c];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        scratch[ncells] = t;
    }
}

}  // namespace

extern "C" efe_status efe_integrate_noalloc(efe_ctx *ctx, const double *a_q, const double *b_q, double *out) {
    if (!ctx || !a_q || !out) return EFE_ERR_ARG;
    const MeshDev &m = ctx->m;
    const long long ncells = (long long)m.nx * m.ny * m.nz;
    if (ncells > kNoallocMaxCells) {
        ctx->err = "efe_integrate_noalloc: " + std::to_string(ncells) + " cells exceed the fixed scratch of " +
                   std::to_string(kNoallocMaxCells) + " cells; use efe_integrate";
        return EFE_ERR_ARG;
    }
    const int dev = ctx->device;   // the device the context (and its stream) was made on
    if (dev < 0 || dev >= kMaxDevices) {
        ctx->err = "efe_integrate_noalloc: device index out of range";
        return EFE_ERR_ARG;
    }
    // the launches below go to ctx->stream, so they run with the context's device current
    DeviceScope scope(dev);
    EFE_CUDA(ctx, scope.err);
    double *scratch = nullptr;
    // first call on a device: the address lookup (make it before any stream capture)
    EFE_CUDA(ctx, scratch_address(dev, &scratch));
    Tables1D T = make_tables(ctx);
    k_cell_integrals<<<(unsigned)ncells, 256, 0, ctx->stream>>>(m, T, a_q, b_q, scratch);
    EFE_TRY(efe_check_launch(ctx, "k_cell_integrals"));
    k_sum_cells<<<1, 1024, 0, ctx->stream>>>((int)ncells, scratch);
    EFE_TRY(efe_check_launch(ctx, "k_sum_cells"));
    EFE_CUDA(ctx, cudaMemcpyAsync(out, scratch + ncells, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    EFE_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return EFE_OK;
}
