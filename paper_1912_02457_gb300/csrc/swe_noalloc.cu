// swe_noalloc.cu -- mass and energy diagnostics that allocate nothing.
//
// For callers that cannot allocate device memory at the point where they
// need the diagnostics: code that runs while a stream is being captured
// into a CUDA graph (cudaMalloc is not allowed there), code inside a host
// framework that owns every device buffer through its own pool, and
// real-time loops where an allocation may block. The caller passes its own
// state planes and its own output; the per-row partial sums live in the
// file-scope device array below, which every GPU that loads the library
// holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/swe.h"

namespace {

constexpr int kMaxRows = SWE_NOALLOC_MAX_ROWS;       // 16384 rows
constexpr int kMaxDevices = 64;

// Two FP64 partial sums (mass, energy) per grid row: 256 KiB.
static __device__ __align__(256) double g_row_partials[2 * kMaxRows];

std::mutex g_mu;
double *g_partials_addr[kMaxDevices] = {nullptr};  // device address, per device

// One block per row: FP64 sums of eta and of (hu^2 + hv^2)/(2|h*|) + g eta^2/2
// over the row's water cells (a cell with a SWE_LAND corner is land).
__global__ void row_sums_kernel(const float *eta, const float *hu, const float *hv, const float *H,
                                int nx, int ny, long long pitch, long long cpitch, double g,
                                double kappa, double *partials) {
    __shared__ double sm[2][32];
    const int j = blockIdx.x;
    double m = 0.0, en = 0.0;
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const float *c = H + (long long)j * cpitch + i;
        float c00 = c[0], c10 = c[1], c01 = c[cpitch], c11 = c[cpitch + 1];
        if (c00 == SWE_LAND || c10 == SWE_LAND || c01 == SWE_LAND || c11 == SWE_LAND) continue;
        const long long s = (long long)j * pitch + i;
        double e = eta[s], u = hu[s], v = hv[s];
        double h = e + 0.25 * ((double)c00 + (double)c10 + (double)c01 + (double)c11);
        double hs = fmax(fabs(h), fmin(h * h / (2.0 * kappa) + 0.5 * kappa, kappa));
        m += e;
        en += 0.5 * (u * u + v * v) / hs + 0.5 * g * e * e;
    }
    for (int o = 16; o > 0; o >>= 1) {
        m += __shfl_xor_sync(0xffffffffu, m, o);
        en += __shfl_xor_sync(0xffffffffu, en, o);
    }
    if ((threadIdx.x & 31) == 0) { sm[0][threadIdx.x >> 5] = m; sm[1][threadIdx.x >> 5] = en; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) { a += sm[0][w]; b += sm[1][w]; }
        partials[2 * j] = a;
        partials[2 * j + 1] = b;
    }
}

// Sum the row partials in a fixed order (deterministic), scale by the cell area.
__global__ void rows_total_kernel(const double *partials, int ny, double area, double *out) {
    __shared__ double sm[2][32];
    double m = 0.0, e = 0.0;
    for (int j = threadIdx.x; j < ny; j += 32) { m += partials[2 * j]; e += partials[2 * j + 1]; }
    sm[0][threadIdx.x] = m;
    sm[1][threadIdx.x] = e;
    __syncwarp();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 32; w++) { a += sm[0][w]; b += sm[1][w]; }
        out[0] = a * area;
        out[1] = b * area;
    }
}

// Device address of the scratch array on the current device, looked up once
// per device (cudaGetSymbolAddress with that device current).
int scratch_on_current_device(double **ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return SWE_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SWE_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_partials_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_row_partials);
        if (e != cudaSuccess || !p) return SWE_ERR_CUDA;
        g_partials_addr[dev] = static_cast<double *>(p);
    }
    *ptr = g_partials_addr[dev];
    return SWE_OK;
}

}  // namespace

extern "C" {

int swe_diagnostics_noalloc(const float *eta, const float *hu, const float *hv, const float *H,
                            int nx, int ny, long long pitch, long long cpitch, double dx, double dy,
                            double g, double kappa, double *out, void *stream) {
    if (!eta || !hu || !hv || !H || !out) return SWE_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || pitch < nx || cpitch < (long long)nx + 1) return SWE_ERR_INVALID_ARG;
    if (ny > kMaxRows) return SWE_ERR_INVALID_ARG;     // beyond the static scratch
    if (!(dx > 0) || !(dy > 0) || !(g > 0) || !(kappa > 0)) return SWE_ERR_INVALID_ARG;
    double *partials = nullptr;
    int rc = scratch_on_current_device(&partials);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // launched through cudaLaunchKernel, whose status is that of this launch
    // alone (an error the caller left pending is neither reported nor cleared)
    double area = dx * dy;
    void *row_args[] = {&eta, &hu, &hv, &H, &nx, &ny, &pitch, &cpitch, &g, &kappa, &partials};
    if (cudaLaunchKernel((const void *)row_sums_kernel, dim3(ny), dim3(256), row_args, 0, st) != cudaSuccess)
        return SWE_ERR_CUDA;
    void *total_args[] = {&partials, &ny, &area, &out};
    if (cudaLaunchKernel((const void *)rows_total_kernel, dim3(1), dim3(32), total_args, 0, st) != cudaSuccess)
        return SWE_ERR_CUDA;
    return SWE_OK;
}

}  // extern "C"
