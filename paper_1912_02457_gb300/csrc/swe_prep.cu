// swe_prep.cu -- grid pre-processing of libswe (Sections 3.8 and 3.9):
// corner bathymetry from cell averages, land erosion, refinement and
// coarsening by two. Memory-bound stencils, one thread per output point,
// 32-wide rows for coalesced access; the neighbours of a point come
// through L1. Nothing here allocates.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "../../include/swe.h"
#include "swe_kernels.h"

namespace {

using swe::kLand;

constexpr int kMaxIter = 4096;           // iterations whose statistics fit the work area
constexpr int kBX = 32, kBY = 8;

int prep_fail(cudaError_t e) { return swe::record_cuda_error(e); }

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

dim3 grid_for(long long nx, long long ny) {
    return dim3((unsigned)((nx + kBX - 1) / kBX), (unsigned)((ny + kBY - 1) / kBY));
}

// Generalised minmod (Section 3.1), written so that exactly the cases of
// the definition select: the smallest of three positives, the largest of
// three negatives, else zero.
template <typename T>
__device__ __forceinline__ T gminmod(T a, T b, T c) {
    const T lo = fmin(a, fmin(b, c)), hi = fmax(a, fmax(b, c));
    return (a > T(0) && b > T(0) && c > T(0)) ? lo : ((a < T(0) && b < T(0) && c < T(0)) ? hi : T(0));
}

// Non-negative floats order like their bit patterns.
__device__ __forceinline__ void atomic_max_nonneg(unsigned int *acc, float v) {
    atomicMax(acc, __float_as_uint(v));
}

// Block maximum of v over the threads with `have`, one atomic per block
// (every thread of the block must call it).
__device__ __forceinline__ void block_max_to(unsigned int *acc, float v, bool have) {
    __shared__ float part[kBX * kBY / 32];
    v = have ? v : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0 && acc) {
        float m = 0.f;
        for (int w = 0; w < kBX * kBY / 32; w++) m = fmaxf(m, part[w]);
        atomic_max_nonneg(acc, m);
    }
}

// ---------------------------------------------------------------------------
// corner bathymetry (Section 3.8), FP32: GB300's FP64 rate is a small
// fraction of its FP32 rate, and the corners feed the FP32 stage kernels

// dH = Hm - H*(i, j), H* the mean of the cell's four corners; the largest
// |dH| goes to *acc when acc != NULL.
__global__ void __launch_bounds__(kBX * kBY) residual_kernel(const float *Hm, long long pitch,
                                                             const float *Hc, long long cpitch,
                                                             int nx, int ny, float *dH, long long wp,
                                                             unsigned int *acc) {
    const int i = blockIdx.x * kBX + threadIdx.x % kBX;
    const int j = blockIdx.y * kBY + threadIdx.x / kBX;
    const bool in = i < nx && j < ny;
    float r = 0.f;
    if (in) {
        const float *c = Hc + (long long)j * cpitch + i;
        const float mid = 0.25f * (((c[0] + c[1]) + c[cpitch]) + c[cpitch + 1]);
        r = Hm[(long long)j * pitch + i] - mid;
        dH[(long long)j * wp + i] = r;
    }
    block_max_to(acc, fabsf(r), in);
}

// eqn:recon_1: limited x and y slopes of field F per cell width; beyond the
// edge a neighbour is the linear extrapolation 2 F_0 - F_1 (a single cell
// along an axis has slope zero there).
__global__ void __launch_bounds__(kBX * kBY) slope_kernel(const float *F, long long fp, int nx, int ny,
                                                          float theta, float *sx, float *sy,
                                                          long long wp) {
    const int i = blockIdx.x * kBX + threadIdx.x % kBX;
    const int j = blockIdx.y * kBY + threadIdx.x / kBX;
    if (i >= nx || j >= ny) return;
    const float *p = F + (long long)j * fp + i;
    const float c = p[0];
    float w, e, s, n;
    if (nx == 1) { w = e = c; }
    else {
        w = i > 0 ? p[-1] : 2.f * c - p[1];
        e = i < nx - 1 ? p[1] : 2.f * c - p[-1];
    }
    if (ny == 1) { s = n = c; }
    else {
        s = j > 0 ? p[-fp] : 2.f * c - p[fp];
        n = j < ny - 1 ? p[fp] : 2.f * c - p[-fp];
    }
    const float bx = c - w, fx = e - c, by = c - s, fy = n - c;
    sx[(long long)j * wp + i] = gminmod(theta * bx, 0.5f * (bx + fx), theta * fx);
    sy[(long long)j * wp + i] = gminmod(theta * by, 0.5f * (by + fy), theta * fy);
}

// eqn:recon_2 and eqn:recon_3: corner (J, I) is the mean of the planar
// estimates of the (up to four) cells that meet there; out = base + mean
// (base NULL: the mean alone).
__global__ void __launch_bounds__(kBX * kBY) corner_kernel(const float *F, long long fp, const float *sx,
                                                           const float *sy, long long wp, int nx, int ny,
                                                           const float *base, long long cpitch,
                                                           float *out, long long op) {
    const int I = blockIdx.x * kBX + threadIdx.x % kBX;
    const int J = blockIdx.y * kBY + threadIdx.x / kBX;
    if (I > nx || J > ny) return;
    float total = 0.f;
    int count = 0;
    // the cells in the order: corner below-left of the centre (cell (J, I)),
    // below-right (cell (J, I-1)), above-left (J-1, I), above-right (J-1, I-1)
    for (int k = 0; k < 4; k++) {
        const int gy = k < 2 ? -1 : 1, gx = (k & 1) ? 1 : -1;
        const int j = gy < 0 ? J : J - 1, i = gx < 0 ? I : I - 1;
        if (i < 0 || i >= nx || j < 0 || j >= ny) continue;
        const long long c = (long long)j * wp + i;
        const float est = (F[(long long)j * fp + i] + 0.5f * gx * sx[c]) + 0.5f * gy * sy[c];
        total += est;
        count++;
    }
    // 1, 2 or 4 estimates: the mean is an exact scaling
    const float mean = total * (count == 4 ? 0.25f : (count == 2 ? 0.5f : 1.f));
    out[(long long)J * op + I] = base ? base[(long long)J * cpitch + I] + mean : mean;
}

// Hc := (1 - w) T + w (mean of T's four neighbour corners, linearly
// extrapolated beyond the edge); the largest |Hc_new - Hc_old| -> *acc.
__global__ void __launch_bounds__(kBX * kBY) smooth_kernel(const float *T, long long tp, float *Hc,
                                                           long long cpitch, int ncx, int ncy, float wgt,
                                                           unsigned int *acc) {
    const int I = blockIdx.x * kBX + threadIdx.x % kBX;
    const int J = blockIdx.y * kBY + threadIdx.x / kBX;
    const bool in = I < ncx && J < ncy;
    float change = 0.f;
    if (in) {
        const float *p = T + (long long)J * tp + I;
        const float c = p[0];
        const float W = I > 0 ? p[-1] : 2.f * c - p[1];
        const float E = I < ncx - 1 ? p[1] : 2.f * c - p[-1];
        const float S = J > 0 ? p[-tp] : 2.f * c - p[tp];
        const float N = J < ncy - 1 ? p[tp] : 2.f * c - p[-tp];
        const float v = (1.f - wgt) * c + wgt * 0.25f * (((W + E) + S) + N);
        float *h = Hc + (long long)J * cpitch + I;
        change = fabsf(v - *h);
        *h = v;
    }
    block_max_to(acc, change, in);
}

struct BathyWork {
    float *dH, *sx, *sy, *tmp;
    unsigned int *stats;
    long long wp, tp;
};

BathyWork bathy_layout(void *work, int nx, int ny) {
    BathyWork w;
    w.wp = round_up(nx, 32);
    w.tp = round_up((long long)nx + 1, 32);
    char *p = static_cast<char *>(work);
    const size_t plane = (size_t)round_up((long long)w.wp * ny * 4, 256);
    w.dH = reinterpret_cast<float *>(p);
    w.sx = reinterpret_cast<float *>(p + plane);
    w.sy = reinterpret_cast<float *>(p + 2 * plane);
    w.tmp = reinterpret_cast<float *>(p + 3 * plane);
    const size_t cplane = (size_t)round_up((long long)w.tp * (ny + 1) * 4, 256);
    w.stats = reinterpret_cast<unsigned int *>(p + 3 * plane + cplane);
    return w;
}

size_t bathy_bytes(int nx, int ny) {
    const long long wp = round_up(nx, 32), tp = round_up((long long)nx + 1, 32);
    return (size_t)(3 * round_up(wp * ny * 4, 256) + round_up(tp * (ny + 1) * 4, 256)) +
           2 * kMaxIter * sizeof(unsigned int);
}

// ---------------------------------------------------------------------------
// land erosion (Section 3.8)

__global__ void __launch_bounds__(kBX * kBY) erode_kernel(const unsigned char *land, const float *eta,
                                                          const float *Hm, long long pitch, int nx,
                                                          int ny, float land_depth, unsigned char *land_out,
                                                          float *eta_out, float *Hm_out) {
    const int i = blockIdx.x * kBX + threadIdx.x % kBX;
    const int j = blockIdx.y * kBY + threadIdx.x / kBX;
    if (i >= nx || j >= ny) return;
    const long long s = (long long)j * pitch + i;
    const bool l = land[s] != 0;
    // outside the domain counts as land
    const bool lw = i == 0 || land[s - 1] != 0, le = i == nx - 1 || land[s + 1] != 0;
    const bool ls = j == 0 || land[s - pitch] != 0, ln = j == ny - 1 || land[s + pitch] != 0;
    const bool stays = l && lw && le && ls && ln;
    const bool opened = l && !stays;
    float e = eta[s], h = Hm[s];
    if (opened) {
        // gray dilation: the largest eta among the water 4-neighbours
        float m = -INFINITY;
        if (!lw) m = fmaxf(m, eta[s - 1]);
        if (!le) m = fmaxf(m, eta[s + 1]);
        if (!ls) m = fmaxf(m, eta[s - pitch]);
        if (!ln) m = fmaxf(m, eta[s + pitch]);
        e = m;
        h = land_depth;
    }
    land_out[s] = stays ? 1 : 0;
    eta_out[s] = e;
    Hm_out[s] = h;
}

// ---------------------------------------------------------------------------
// refinement and coarsening by two (Section 3.9), FP32

__device__ __forceinline__ bool corner_land(const float *H, long long cp, int j, int i) {
    const float *c = H + (long long)j * cp + i;
    return (c[0] == kLand) | (c[1] == kLand) | (c[cp] == kLand) | (c[cp + 1] == kLand);
}

struct Planes3 {
    const float *q[3];
};
struct OutPlanes3 {
    float *q[3];
};

__global__ void __launch_bounds__(kBX * kBY) refine_cells_kernel(Planes3 in, long long pitch, const float *H,
                                                                 long long cp, int nx, int ny, float theta,
                                                                 OutPlanes3 out, long long fp) {
    const int i = blockIdx.x * kBX + threadIdx.x % kBX;
    const int j = blockIdx.y * kBY + threadIdx.x / kBX;
    if (i >= nx || j >= ny) return;
    const bool land = corner_land(H, cp, j, i);
    // a neighbour that is land or outside gives a zero one-sided difference
    const bool nw = i > 0 && !corner_land(H, cp, j, i - 1);
    const bool ne = i < nx - 1 && !corner_land(H, cp, j, i + 1);
    const bool ns = j > 0 && !corner_land(H, cp, j - 1, i);
    const bool nn = j < ny - 1 && !corner_land(H, cp, j + 1, i);
    const long long s = (long long)j * pitch + i;
    const long long f0 = (long long)(2 * j) * fp + 2 * i;
    for (int v = 0; v < 3; v++) {
        float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
        if (!land) {
            const float *p = in.q[v] + s;
            const float c = p[0];
            const float bx = nw ? c - p[-1] : 0.f, fx = ne ? p[1] - c : 0.f;
            const float by = ns ? c - p[-pitch] : 0.f, fy = nn ? p[pitch] - c : 0.f;
            const float sx = gminmod(theta * bx, 0.5f * (bx + fx), theta * fx);
            const float sy = gminmod(theta * by, 0.5f * (by + fy), theta * fy);
            // children at x +- 1/4, y +- 1/4 of the cell
            lo.x = (c - 0.25f * sx) - 0.25f * sy;
            lo.y = (c + 0.25f * sx) - 0.25f * sy;
            hi.x = (c - 0.25f * sx) + 0.25f * sy;
            hi.y = (c + 0.25f * sx) + 0.25f * sy;
        }
        *reinterpret_cast<float2 *>(out.q[v] + f0) = lo;
        *reinterpret_cast<float2 *>(out.q[v] + f0 + fp) = hi;
    }
}

// Fine intersections owned by coarse corner (J, I): (2J, 2I) and, where they
// exist, the edge midpoints (2J, 2I+1), (2J+1, 2I) and the centre (2J+1, 2I+1).
__global__ void __launch_bounds__(kBX * kBY) refine_corners_kernel(const float *H, long long cp, int nx, int ny,
                                                                   float *F, long long fcp) {
    const int I = blockIdx.x * kBX + threadIdx.x % kBX;
    const int J = blockIdx.y * kBY + threadIdx.x / kBX;
    if (I > nx || J > ny) return;
    const float *c = H + (long long)J * cp + I;
    float *o = F + (long long)(2 * J) * fcp + 2 * I;
    const float a = c[0];
    o[0] = a;
    if (I < nx) {
        const float b = c[1];
        o[1] = (a == kLand || b == kLand) ? kLand : 0.5f * (a + b);
    }
    if (J < ny) {
        const float b = c[cp];
        o[fcp] = (a == kLand || b == kLand) ? kLand : 0.5f * (a + b);
    }
    if (I < nx && J < ny) {
        const float c10 = c[1], c01 = c[cp], c11 = c[cp + 1];
        const bool l = (a == kLand) | (c10 == kLand) | (c01 == kLand) | (c11 == kLand);
        o[fcp + 1] = l ? kLand : 0.25f * (((a + c10) + c01) + c11);
    }
}

__global__ void __launch_bounds__(kBX * kBY) coarsen_cells_kernel(Planes3 fin, long long fp, const float *Hf,
                                                                  long long fcp, int nx, int ny, OutPlanes3 out,
                                                                  long long pitch) {
    const int i = blockIdx.x * kBX + threadIdx.x % kBX;
    const int j = blockIdx.y * kBY + threadIdx.x / kBX;
    if (i >= nx || j >= ny) return;
    // the coarse cell is land if one of its sampled corners is
    const float *cc = Hf + (long long)(2 * j) * fcp + 2 * i;
    const bool cland = (cc[0] == kLand) | (cc[2] == kLand) | (cc[2 * fcp] == kLand) | (cc[2 * fcp + 2] == kLand);
    bool wet[4];
    float n_wet = 0.f;
    for (int b = 0; b < 2; b++)
        for (int a = 0; a < 2; a++) {
            wet[2 * b + a] = !corner_land(Hf, fcp, 2 * j + b, 2 * i + a);
            n_wet += wet[2 * b + a] ? 1.f : 0.f;
        }
    const long long f0 = (long long)(2 * j) * fp + 2 * i;
    for (int v = 0; v < 3; v++) {
        const float2 lo = *reinterpret_cast<const float2 *>(fin.q[v] + f0);
        const float2 hi = *reinterpret_cast<const float2 *>(fin.q[v] + f0 + fp);
        const float s = (((wet[0] ? lo.x : 0.f) + (wet[1] ? lo.y : 0.f)) + (wet[2] ? hi.x : 0.f)) +
                        (wet[3] ? hi.y : 0.f);
        out.q[v][(long long)j * pitch + i] = (cland || n_wet == 0.f) ? 0.f : s / n_wet;
    }
}

__global__ void __launch_bounds__(kBX * kBY) coarsen_corners_kernel(const float *Hf, long long fcp, int nx, int ny,
                                                                    float *H, long long cp) {
    const int I = blockIdx.x * kBX + threadIdx.x % kBX;
    const int J = blockIdx.y * kBY + threadIdx.x / kBX;
    if (I > nx || J > ny) return;
    H[(long long)J * cp + I] = Hf[(long long)(2 * J) * fcp + 2 * I];
}

bool aligned8(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

}  // namespace

extern "C" {

size_t swe_bathymetry_work_bytes(int nx, int ny) {
    if (nx < 1 || ny < 1) return 0;
    return bathy_bytes(nx, ny);
}

int swe_bathymetry_reconstruct(const float *Hm, long long pitch, int nx, int ny, float *Hc,
                               long long cpitch, void *work, int n_iter, double theta,
                               double smooth, double *stats, void *stream) {
    if (!Hm || !Hc || !work || nx < 1 || ny < 1 || pitch < nx || cpitch < (long long)nx + 1)
        return SWE_ERR_INVALID_ARG;
    if (n_iter < 0 || n_iter > kMaxIter || !(theta >= 1.0 && theta <= 2.0) ||
        !(smooth >= 0.0 && smooth <= 1.0))
        return SWE_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(work) & 255u) != 0) return SWE_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const BathyWork w = bathy_layout(work, nx, ny);
    const dim3 blk(kBX * kBY), gc = grid_for(nx, ny), gk = grid_for(nx + 1, ny + 1);
    const float th = (float)theta, sm = (float)smooth;
    cudaError_t e = cudaMemsetAsync(w.stats, 0, 2 * kMaxIter * sizeof(unsigned int), st);
    if (e != cudaSuccess) return prep_fail(e);
    // initial guess from the cell averages themselves
    slope_kernel<<<gc, blk, 0, st>>>(Hm, pitch, nx, ny, th, w.sx, w.sy, w.wp);
    corner_kernel<<<gk, blk, 0, st>>>(Hm, pitch, w.sx, w.sy, w.wp, nx, ny, nullptr, 0, Hc, cpitch);
    for (int k = 0; k < n_iter; k++) {
        // misfit of the previous iteration's corners (none for the initial guess)
        residual_kernel<<<gc, blk, 0, st>>>(Hm, pitch, Hc, cpitch, nx, ny, w.dH, w.wp,
                                            k > 0 ? w.stats + 2 * (k - 1) : nullptr);
        slope_kernel<<<gc, blk, 0, st>>>(w.dH, w.wp, nx, ny, th, w.sx, w.sy, w.wp);
        corner_kernel<<<gk, blk, 0, st>>>(w.dH, w.wp, w.sx, w.sy, w.wp, nx, ny, Hc, cpitch, w.tmp, w.tp);
        smooth_kernel<<<gk, blk, 0, st>>>(w.tmp, w.tp, Hc, cpitch, nx + 1, ny + 1, sm,
                                          w.stats + 2 * k + 1);
    }
    if (n_iter > 0)
        residual_kernel<<<gc, blk, 0, st>>>(Hm, pitch, Hc, cpitch, nx, ny, w.dH, w.wp,
                                            w.stats + 2 * (n_iter - 1));
    if ((e = cudaGetLastError()) != cudaSuccess) return prep_fail(e);
    if (stats && n_iter > 0) {
        unsigned int bits[2 * kMaxIter];
        e = cudaMemcpyAsync(bits, w.stats, 2 * (size_t)n_iter * sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return prep_fail(e);
        for (int k = 0; k < 2 * n_iter; k++) {
            float f;
            memcpy(&f, &bits[k], sizeof f);
            stats[k] = f;
        }
    }
    return SWE_OK;
}

int swe_land_erode(const unsigned char *land, const float *eta, const float *Hm,
                   long long pitch, int nx, int ny, double land_depth,
                   unsigned char *land_out, float *eta_out, float *Hm_out, void *stream) {
    if (!land || !eta || !Hm || !land_out || !eta_out || !Hm_out || nx < 1 || ny < 1 || pitch < nx)
        return SWE_ERR_INVALID_ARG;
    if ((const void *)land_out == (const void *)land || eta_out == eta || Hm_out == Hm)
        return SWE_ERR_INVALID_ARG;
    if (!(land_depth >= 0.0)) return SWE_ERR_INVALID_ARG;
    erode_kernel<<<grid_for(nx, ny), kBX * kBY, 0, (cudaStream_t)stream>>>(
        land, eta, Hm, pitch, nx, ny, (float)land_depth, land_out, eta_out, Hm_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SWE_OK : prep_fail(e);
}

int swe_refine2(const float *eta, const float *hu, const float *hv, long long pitch,
                const float *H, long long cpitch, int nx, int ny, double theta,
                float *eta_f, float *hu_f, float *hv_f, long long fpitch, float *H_f,
                long long fcpitch, void *stream) {
    if (!eta || !hu || !hv || !H || !eta_f || !hu_f || !hv_f || !H_f) return SWE_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536 || pitch < nx || cpitch < (long long)nx + 1)
        return SWE_ERR_INVALID_ARG;
    if (fpitch < 2LL * nx || (fpitch & 1) || fcpitch < 2LL * nx + 1) return SWE_ERR_INVALID_ARG;
    if (!aligned8(eta_f) || !aligned8(hu_f) || !aligned8(hv_f)) return SWE_ERR_INVALID_ARG;
    if (!(theta >= 1.0 && theta <= 2.0)) return SWE_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Planes3 in{{eta, hu, hv}};
    OutPlanes3 out{{eta_f, hu_f, hv_f}};
    refine_cells_kernel<<<grid_for(nx, ny), kBX * kBY, 0, st>>>(in, pitch, H, cpitch, nx, ny, (float)theta,
                                                                out, fpitch);
    refine_corners_kernel<<<grid_for(nx + 1, ny + 1), kBX * kBY, 0, st>>>(H, cpitch, nx, ny, H_f, fcpitch);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SWE_OK : prep_fail(e);
}

int swe_coarsen2(const float *eta_f, const float *hu_f, const float *hv_f, long long fpitch,
                 const float *H_f, long long fcpitch, int nx, int ny, float *eta, float *hu,
                 float *hv, long long pitch, float *H, long long cpitch, void *stream) {
    if (!eta_f || !hu_f || !hv_f || !H_f || !eta || !hu || !hv || !H) return SWE_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536 || pitch < nx || cpitch < (long long)nx + 1)
        return SWE_ERR_INVALID_ARG;
    if (fpitch < 2LL * nx || (fpitch & 1) || fcpitch < 2LL * nx + 1) return SWE_ERR_INVALID_ARG;
    if (!aligned8(eta_f) || !aligned8(hu_f) || !aligned8(hv_f)) return SWE_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Planes3 fin{{eta_f, hu_f, hv_f}};
    OutPlanes3 out{{eta, hu, hv}};
    coarsen_cells_kernel<<<grid_for(nx, ny), kBX * kBY, 0, st>>>(fin, fpitch, H_f, fcpitch, nx, ny, out, pitch);
    coarsen_corners_kernel<<<grid_for(nx + 1, ny + 1), kBX * kBY, 0, st>>>(H_f, fcpitch, nx, ny, H, cpitch);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SWE_OK : prep_fail(e);
}

}  // extern "C"
