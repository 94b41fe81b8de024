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

// max |Hm - H*(i, j)| over the cells -> *acc, H* the mean of the cell's four
// corners (the misfit of the final corners).
__global__ void __launch_bounds__(kBX * kBY) residual_kernel(const float *Hm, long long pitch,
                                                             const float *Hc, long long cpitch,
                                                             int nx, int ny, unsigned int *acc) {
    const int i = blockIdx.x * kBX + threadIdx.x % kBX;
    const int j = blockIdx.y * kBY + threadIdx.x / kBX;
    const bool in = i < nx && j < ny;
    float r = 0.f;
    if (in) {
        const float *c = Hc + (long long)j * cpitch + i;
        const float mid = 0.25f * (((c[0] + c[1]) + c[cpitch]) + c[cpitch + 1]);
        r = Hm[(long long)j * pitch + i] - mid;
    }
    block_max_to(acc, fabsf(r), in);
}

// One iteration of the corner reconstruction (or, with X == NULL, the
// initial guess) for a tile of kTY x kTX output corners, every intermediate
// in shared memory, so an iteration reads Hm and the corners X and writes
// the corners Y once (halo re-reads come from L2):
//   A  the field F whose slopes are taken: Hm itself for the initial guess,
//      else the residual dH = Hm - H*(i, j) of X (cells on a 3-cell halo);
//   B  eqn:recon_1: the limited slopes of F (cells on a 2-cell halo; beyond
//      an edge a value is linearly extrapolated);
//   C  eqn:recon_2, eqn:recon_3: T = X + the mean of the planar estimates of
//      the cells meeting at a corner (corners on a 1-corner halo);
//   D  the smoothing pass Y = (1 - w) T + w (mean of T's 4 neighbours,
//      extrapolated beyond an edge); the initial guess is T as it stands.
// The misfit max|dH| of X and the largest change max|Y - X| go to misfit
// and change.
constexpr int kTX = 64, kTY = 32, kTileThreads = 256;

__global__ void __launch_bounds__(kTileThreads) bathy_tile_kernel(const float *Hm, long long pitch, int nx,
                                                                  int ny, const float *X, long long xp,
                                                                  float *Y, long long yp, float theta,
                                                                  float wgt, unsigned int *misfit,
                                                                  unsigned int *change) {
    __shared__ float D[kTY + 5][kTX + 5];
    __shared__ float SX[kTY + 3][kTX + 3], SY[kTY + 3][kTX + 3];
    __shared__ float T[kTY + 2][kTX + 2];
    __shared__ float part[2][kTileThreads / 32];
    const int I0 = blockIdx.x * kTX, J0 = blockIdx.y * kTY;
    const bool init = X == nullptr;
    float mis = 0.f, chg = 0.f;

    // A: F on cells [J0-3, J0+kTY+2) x [I0-3, I0+kTX+2)
    for (int k = threadIdx.x; k < (kTY + 5) * (kTX + 5); k += kTileThreads) {
        const int a = k / (kTX + 5), b = k % (kTX + 5);
        const int j = J0 - 3 + a, i = I0 - 3 + b;
        float v = 0.f;
        if (j >= 0 && j < ny && i >= 0 && i < nx) {
            v = Hm[(long long)j * pitch + i];
            if (!init) {
                const float *c = X + (long long)j * xp + i;
                v = v - 0.25f * (((c[0] + c[1]) + c[xp]) + c[xp + 1]);
                if (a >= 3 && a < 3 + kTY && b >= 3 && b < 3 + kTX) mis = fmaxf(mis, fabsf(v));
            }
        }
        D[a][b] = v;
    }
    __syncthreads();

    // B: slopes of the cells [J0-2, J0+kTY+1) x [I0-2, I0+kTX+1)
    for (int k = threadIdx.x; k < (kTY + 3) * (kTX + 3); k += kTileThreads) {
        const int a = k / (kTX + 3), b = k % (kTX + 3);
        const int j = J0 - 2 + a, i = I0 - 2 + b;
        float sx = 0.f, sy = 0.f;
        if (j >= 0 && j < ny && i >= 0 && i < nx) {
            const float c = D[a + 1][b + 1];
            float w = c, e = c, s = c, n = c;
            if (nx > 1) {
                w = i > 0 ? D[a + 1][b] : 2.f * c - D[a + 1][b + 2];
                e = i < nx - 1 ? D[a + 1][b + 2] : 2.f * c - D[a + 1][b];
            }
            if (ny > 1) {
                s = j > 0 ? D[a][b + 1] : 2.f * c - D[a + 2][b + 1];
                n = j < ny - 1 ? D[a + 2][b + 1] : 2.f * c - D[a][b + 1];
            }
            const float bx = c - w, fx = e - c, by = c - s, fy = n - c;
            sx = gminmod(theta * bx, 0.5f * (bx + fx), theta * fx);
            sy = gminmod(theta * by, 0.5f * (by + fy), theta * fy);
        }
        SX[a][b] = sx;
        SY[a][b] = sy;
    }
    __syncthreads();

    // C: T on the corners [J0-1, J0+kTY] x [I0-1, I0+kTX]
    for (int k = threadIdx.x; k < (kTY + 2) * (kTX + 2); k += kTileThreads) {
        const int a = k / (kTX + 2), b = k % (kTX + 2);
        const int J = J0 - 1 + a, I = I0 - 1 + b;
        float t = 0.f;
        if (J >= 0 && J <= ny && I >= 0 && I <= nx) {
            float total = 0.f;
            int count = 0;
            // the cells in the order: corner below-left of the centre (cell
            // (J, I)), below-right (J, I-1), above-left (J-1, I), above-right (J-1, I-1)
            for (int q = 0; q < 4; q++) {
                const int gy = q < 2 ? -1 : 1, gx = (q & 1) ? 1 : -1;
                const int j = gy < 0 ? J : J - 1, i = gx < 0 ? I : I - 1;
                if (i < 0 || i >= nx || j < 0 || j >= ny) continue;
                const int sa = j - J0 + 2, sb = i - I0 + 2;
                total += (D[sa + 1][sb + 1] + 0.5f * gx * SX[sa][sb]) + 0.5f * gy * SY[sa][sb];
                count++;
            }
            // 1, 2 or 4 estimates: the mean is an exact scaling
            const float mean = total * (count == 4 ? 0.25f : (count == 2 ? 0.5f : 1.f));
            t = init ? mean : X[(long long)J * xp + I] + mean;
        }
        T[a][b] = t;
    }
    __syncthreads();

    // D: the tile's own corners
    for (int k = threadIdx.x; k < kTY * kTX; k += kTileThreads) {
        const int a = k / kTX, b = k % kTX;
        const int J = J0 + a, I = I0 + b;
        if (J > ny || I > nx) continue;
        const float c = T[a + 1][b + 1];
        float v = c;
        if (!init) {
            const float W = I > 0 ? T[a + 1][b] : 2.f * c - T[a + 1][b + 2];
            const float E = I < nx ? T[a + 1][b + 2] : 2.f * c - T[a + 1][b];
            const float S = J > 0 ? T[a][b + 1] : 2.f * c - T[a + 2][b + 1];
            const float N = J < ny ? T[a + 2][b + 1] : 2.f * c - T[a][b + 1];
            v = (1.f - wgt) * c + wgt * 0.25f * (((W + E) + S) + N);
            chg = fmaxf(chg, fabsf(v - X[(long long)J * xp + I]));
        }
        Y[(long long)J * yp + I] = v;
    }
    if (init) return;                       // block-uniform
    // block maxima of the misfit and the change, one atomic each
    for (int o = 16; o > 0; o >>= 1) {
        mis = fmaxf(mis, __shfl_xor_sync(0xffffffffu, mis, o));
        chg = fmaxf(chg, __shfl_xor_sync(0xffffffffu, chg, o));
    }
    if ((threadIdx.x & 31) == 0) { part[0][threadIdx.x >> 5] = mis; part[1][threadIdx.x >> 5] = chg; }
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f, c = 0.f;
        for (int w = 0; w < kTileThreads / 32; w++) { m = fmaxf(m, part[0][w]); c = fmaxf(c, part[1][w]); }
        if (misfit) atomic_max_nonneg(misfit, m);
        atomic_max_nonneg(change, c);
    }
}

// Work area: one corner plane (the iterations alternate between it and the
// caller's corners, ending in the caller's) and the per-iteration statistics.
struct BathyWork {
    float *corners;
    unsigned int *stats;
    long long tp;
};

BathyWork bathy_layout(void *work, int nx, int ny) {
    BathyWork w;
    w.tp = round_up((long long)nx + 1, 32);
    char *p = static_cast<char *>(work);
    w.corners = reinterpret_cast<float *>(p);
    w.stats = reinterpret_cast<unsigned int *>(p + round_up(w.tp * (ny + 1) * 4, 256));
    return w;
}

size_t bathy_bytes(int nx, int ny) {
    const long long tp = round_up((long long)nx + 1, 32);
    return (size_t)round_up(tp * (ny + 1) * 4, 256) + 2 * kMaxIter * sizeof(unsigned int);
}

// ---------------------------------------------------------------------------
// land erosion (Section 3.8)

// One cell (i, j) of the erosion step (shared by the one-cell kernel and the
// ragged end of a row in the four-cell kernel).
__device__ __forceinline__ void erode_cell(const unsigned char *land, const float *eta, const float *Hm,
                                           long long pitch, int nx, int ny, float land_depth, int i, int j,
                                           unsigned char *land_out, float *eta_out, float *Hm_out) {
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

__global__ void __launch_bounds__(kBX * kBY) erode_kernel(const unsigned char *land, const float *eta,
                                                          const float *Hm, long long pitch, int nx,
                                                          int ny, float land_depth, unsigned char *land_out,
                                                          float *eta_out, float *Hm_out) {
    const int i = blockIdx.x * kBX + threadIdx.x % kBX;
    const int j = blockIdx.y * kBY + threadIdx.x / kBX;
    if (i >= nx || j >= ny) return;
    erode_cell(land, eta, Hm, pitch, nx, ny, land_depth, i, j, land_out, eta_out, Hm_out);
}

// The same step, four consecutive cells per thread with vector loads and
// stores (pitch a multiple of 4, float planes 16-byte and byte planes
// 4-byte aligned): five byte-plane loads and two float4 loads for four
// cells instead of twenty-eight scalar loads. The same selections and the
// same order of maxima as erode_cell, so the same bits.
__global__ void __launch_bounds__(kBX * kBY) erode4_kernel(const unsigned char *land, const float *eta,
                                                           const float *Hm, long long pitch, int nx,
                                                           int ny, float land_depth, unsigned char *land_out,
                                                           float *eta_out, float *Hm_out) {
    const int i0 = 4 * (blockIdx.x * kBX + threadIdx.x % kBX);
    const int j = blockIdx.y * kBY + threadIdx.x / kBX;
    if (i0 >= nx || j >= ny) return;
    if (i0 + 4 > nx) {                          // the ragged end of a row
        for (int i = i0; i < nx; i++)
            erode_cell(land, eta, Hm, pitch, nx, ny, land_depth, i, j, land_out, eta_out, Hm_out);
        return;
    }
    const long long s = (long long)j * pitch + i0;
    const uchar4 one = make_uchar4(1, 1, 1, 1);
    const uchar4 L = *reinterpret_cast<const uchar4 *>(land + s);
    const uchar4 LS = j > 0 ? *reinterpret_cast<const uchar4 *>(land + s - pitch) : one;
    const uchar4 LN = j < ny - 1 ? *reinterpret_cast<const uchar4 *>(land + s + pitch) : one;
    const bool lW = i0 == 0 || land[s - 1] != 0;
    const bool lE = i0 + 4 >= nx || land[s + 4] != 0;
    const float4 E = *reinterpret_cast<const float4 *>(eta + s);
    const float4 D = *reinterpret_cast<const float4 *>(Hm + s);
    const bool l[4] = {L.x != 0, L.y != 0, L.z != 0, L.w != 0};
    const bool ls[4] = {LS.x != 0, LS.y != 0, LS.z != 0, LS.w != 0};
    const bool ln[4] = {LN.x != 0, LN.y != 0, LN.z != 0, LN.w != 0};
    const float ein[4] = {E.x, E.y, E.z, E.w};
    float e[4] = {E.x, E.y, E.z, E.w}, h[4] = {D.x, D.y, D.z, D.w};
    unsigned char stay[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const bool lw = k == 0 ? lW : l[k - 1], le = k == 3 ? lE : l[k + 1];
        const bool stays = l[k] && lw && le && ls[k] && ln[k];
        if (l[k] && !stays) {
            float m = -INFINITY;
            if (!lw) m = fmaxf(m, k == 0 ? eta[s - 1] : ein[k - 1]);
            if (!le) m = fmaxf(m, k == 3 ? eta[s + 4] : ein[k + 1]);
            if (!ls[k]) m = fmaxf(m, eta[s + k - pitch]);
            if (!ln[k]) m = fmaxf(m, eta[s + k + pitch]);
            e[k] = m;
            h[k] = land_depth;
        }
        stay[k] = stays ? 1 : 0;
    }
    *reinterpret_cast<uchar4 *>(land_out + s) = make_uchar4(stay[0], stay[1], stay[2], stay[3]);
    *reinterpret_cast<float4 *>(eta_out + s) = make_float4(e[0], e[1], e[2], e[3]);
    *reinterpret_cast<float4 *>(Hm_out + s) = make_float4(h[0], h[1], h[2], h[3]);
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

// The four children of a water cell with value c and one-sided
// differences bx, fx (x) and by, fy (y): limited slopes, children at
// x +- 1/4, y +- 1/4 of the cell (lo: the lower row of children).
__device__ __forceinline__ void refine_children(float c, float bx, float fx, float by, float fy, float theta,
                                                float2 &lo, float2 &hi) {
    const float sx = gminmod(theta * bx, 0.5f * (bx + fx), theta * fx);
    const float sy = gminmod(theta * by, 0.5f * (by + fy), theta * fy);
    lo.x = (c - 0.25f * sx) - 0.25f * sy;
    lo.y = (c + 0.25f * sx) - 0.25f * sy;
    hi.x = (c - 0.25f * sx) + 0.25f * sy;
    hi.y = (c + 0.25f * sx) + 0.25f * sy;
}

// One coarse cell (i, j) of the refinement (the one-cell kernel, and the odd
// last cell of a row in the two-cell kernel).
__device__ __forceinline__ void refine_cell(const Planes3 &in, long long pitch, const float *H, long long cp,
                                            int nx, int ny, float theta, const OutPlanes3 &out, long long fp,
                                            int i, int j) {
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
            refine_children(c, nw ? c - p[-1] : 0.f, ne ? p[1] - c : 0.f, ns ? c - p[-pitch] : 0.f,
                            nn ? p[pitch] - c : 0.f, theta, lo, hi);
        }
        *reinterpret_cast<float2 *>(out.q[v] + f0) = lo;
        *reinterpret_cast<float2 *>(out.q[v] + f0 + fp) = hi;
    }
}

__global__ void __launch_bounds__(kBX * kBY) refine_cells_kernel(Planes3 in, long long pitch, const float *H,
                                                                 long long cp, int nx, int ny, float theta,
                                                                 OutPlanes3 out, long long fp) {
    const int i = blockIdx.x * kBX + threadIdx.x % kBX;
    const int j = blockIdx.y * kBY + threadIdx.x / kBX;
    if (i >= nx || j >= ny) return;
    refine_cell(in, pitch, H, cp, nx, ny, theta, out, fp, i, j);
}

// The same refinement, two coarse cells (i0, i0 + 1) per thread (coarse
// pitch even and coarse planes 8-byte aligned; fine pitch a multiple of 4
// and fine planes 16-byte aligned): float2 loads of the cells and their
// y-neighbours, the land of the six cells around them from one read of
// their corners, and one float4 store per row of children. The same
// selections and arithmetic as refine_cell, so the same bits.
__global__ void __launch_bounds__(kBX * kBY) refine2_cells_kernel(Planes3 in, long long pitch, const float *H,
                                                                  long long cp, int nx, int ny, float theta,
                                                                  OutPlanes3 out, long long fp) {
    const int i0 = 2 * (blockIdx.x * kBX + threadIdx.x % kBX);
    const int j = blockIdx.y * kBY + threadIdx.x / kBX;
    if (i0 >= nx || j >= ny) return;
    if (i0 + 1 >= nx) {                          // the odd last cell of a row
        refine_cell(in, pitch, H, cp, nx, ny, theta, out, fp, i0, j);
        return;
    }
    // corners of rows j, j + 1 at columns i0 - 1 .. i0 + 3 (where they exist)
    const float *c = H + (long long)j * cp + i0;
    const bool has_w = i0 > 0, has_e = i0 + 2 < nx, has_s = j > 0, has_n = j < ny - 1;
    bool a[5], b[5];                             // corner is LAND, rows j and j + 1
#pragma unroll
    for (int x = 0; x < 5; x++) {
        const bool ok = (x > 0 || has_w) && (x < 4 || has_e);
        a[x] = ok && c[x - 1] == kLand;
        b[x] = ok && c[cp + x - 1] == kLand;
    }
    const bool landW = a[0] | a[1] | b[0] | b[1], land0 = a[1] | a[2] | b[1] | b[2];
    const bool land1 = a[2] | a[3] | b[2] | b[3], landE = a[3] | a[4] | b[3] | b[4];
    bool landS0 = true, landS1 = true, landN0 = true, landN1 = true;
    if (has_s) {
        const float *d = c - cp;
        const bool s0 = d[0] == kLand, s1 = d[1] == kLand, s2 = d[2] == kLand;
        landS0 = s0 | s1 | a[1] | a[2];
        landS1 = s1 | s2 | a[2] | a[3];
    }
    if (has_n) {
        const float *d = c + 2 * cp;
        const bool n0 = d[0] == kLand, n1 = d[1] == kLand, n2 = d[2] == kLand;
        landN0 = b[1] | b[2] | n0 | n1;
        landN1 = b[2] | b[3] | n1 | n2;
    }
    const bool nw0 = has_w && !landW, ne0 = !land1, ns0 = has_s && !landS0, nn0 = has_n && !landN0;
    const bool nw1 = !land0, ne1 = has_e && !landE, ns1 = has_s && !landS1, nn1 = has_n && !landN1;
    const long long s = (long long)j * pitch + i0;
    const long long f0 = (long long)(2 * j) * fp + 2 * i0;
    for (int v = 0; v < 3; v++) {
        const float *p = in.q[v] + s;
        const float2 P = *reinterpret_cast<const float2 *>(p);
        const float pw = has_w ? p[-1] : 0.f, pe = has_e ? p[2] : 0.f;
        const float2 S = has_s ? *reinterpret_cast<const float2 *>(p - pitch) : make_float2(0.f, 0.f);
        const float2 N = has_n ? *reinterpret_cast<const float2 *>(p + pitch) : make_float2(0.f, 0.f);
        float2 lo0 = make_float2(0.f, 0.f), hi0 = lo0, lo1 = lo0, hi1 = lo0;
        if (!land0)
            refine_children(P.x, nw0 ? P.x - pw : 0.f, ne0 ? P.y - P.x : 0.f, ns0 ? P.x - S.x : 0.f,
                            nn0 ? N.x - P.x : 0.f, theta, lo0, hi0);
        if (!land1)
            refine_children(P.y, nw1 ? P.y - P.x : 0.f, ne1 ? pe - P.y : 0.f, ns1 ? P.y - S.y : 0.f,
                            nn1 ? N.y - P.y : 0.f, theta, lo1, hi1);
        *reinterpret_cast<float4 *>(out.q[v] + f0) = make_float4(lo0.x, lo0.y, lo1.x, lo1.y);
        *reinterpret_cast<float4 *>(out.q[v] + f0 + fp) = make_float4(hi0.x, hi0.y, hi1.x, hi1.y);
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

// One coarse cell (i, j) of the coarsening (the one-cell kernel, and the odd
// last cell of a row in the two-cell kernel).
__device__ __forceinline__ void coarsen_cell(const Planes3 &fin, long long fp, const float *Hf, long long fcp,
                                             const OutPlanes3 &out, long long pitch, int i, int j) {
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

__global__ void __launch_bounds__(kBX * kBY) coarsen_cells_kernel(Planes3 fin, long long fp, const float *Hf,
                                                                  long long fcp, int nx, int ny, OutPlanes3 out,
                                                                  long long pitch) {
    const int i = blockIdx.x * kBX + threadIdx.x % kBX;
    const int j = blockIdx.y * kBY + threadIdx.x / kBX;
    if (i >= nx || j >= ny) return;
    coarsen_cell(fin, fp, Hf, fcp, out, pitch, i, j);
}

// The same coarsening, two coarse cells (i0, i0 + 1) per thread (fine pitch
// a multiple of 4 and fine planes 16-byte aligned; coarse pitch even and
// coarse planes 8-byte aligned): one read of the 3 x 5 fine corners they
// share, float4 loads of the children, one float2 store per plane. The same
// selections and arithmetic as coarsen_cell, so the same bits.
__global__ void __launch_bounds__(kBX * kBY) coarsen2_cells_kernel(Planes3 fin, long long fp, const float *Hf,
                                                                   long long fcp, int nx, int ny, OutPlanes3 out,
                                                                   long long pitch) {
    const int i0 = 2 * (blockIdx.x * kBX + threadIdx.x % kBX);
    const int j = blockIdx.y * kBY + threadIdx.x / kBX;
    if (i0 >= nx || j >= ny) return;
    if (i0 + 1 >= nx) {                          // the odd last cell of a row
        coarsen_cell(fin, fp, Hf, fcp, out, pitch, i0, j);
        return;
    }
    // fine corners of rows 2j .. 2j + 2, columns 2 i0 .. 2 i0 + 4: LAND?
    const float *cc = Hf + (long long)(2 * j) * fcp + 2 * i0;
    bool L[3][5];
#pragma unroll
    for (int b = 0; b < 3; b++)
#pragma unroll
        for (int x = 0; x < 5; x++) L[b][x] = cc[b * fcp + x] == kLand;
    bool cland[2], wet[2][4];
    float n_wet[2];
#pragma unroll
    for (int k = 0; k < 2; k++) {
        cland[k] = L[0][2 * k] | L[0][2 * k + 2] | L[2][2 * k] | L[2][2 * k + 2];
        n_wet[k] = 0.f;
#pragma unroll
        for (int b = 0; b < 2; b++)
#pragma unroll
            for (int a = 0; a < 2; a++) {
                const int x = 2 * k + a;
                wet[k][2 * b + a] = !(L[b][x] | L[b][x + 1] | L[b + 1][x] | L[b + 1][x + 1]);
                n_wet[k] += wet[k][2 * b + a] ? 1.f : 0.f;
            }
    }
    const long long f0 = (long long)(2 * j) * fp + 2 * i0;
    for (int v = 0; v < 3; v++) {
        const float4 lo = *reinterpret_cast<const float4 *>(fin.q[v] + f0);
        const float4 hi = *reinterpret_cast<const float4 *>(fin.q[v] + f0 + fp);
        const float s0 = (((wet[0][0] ? lo.x : 0.f) + (wet[0][1] ? lo.y : 0.f)) + (wet[0][2] ? hi.x : 0.f)) +
                         (wet[0][3] ? hi.y : 0.f);
        const float s1 = (((wet[1][0] ? lo.z : 0.f) + (wet[1][1] ? lo.w : 0.f)) + (wet[1][2] ? hi.z : 0.f)) +
                         (wet[1][3] ? hi.w : 0.f);
        *reinterpret_cast<float2 *>(out.q[v] + (long long)j * pitch + i0) =
            make_float2((cland[0] || n_wet[0] == 0.f) ? 0.f : s0 / n_wet[0],
                        (cland[1] || n_wet[1] == 0.f) ? 0.f : s1 / n_wet[1]);
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
    swe::TraceRange trace("swe_bathymetry_reconstruct");
    if (!Hm || !Hc || !work || nx < 1 || ny < 1 || pitch < nx || cpitch < (long long)nx + 1)
        return SWE_ERR_INVALID_ARG;
    if (n_iter < 0 || n_iter > kMaxIter || !(theta >= 1.0 && theta <= 2.0) ||
        !(smooth >= 0.0 && smooth <= 1.0))
        return SWE_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(work) & 255u) != 0) return SWE_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const BathyWork w = bathy_layout(work, nx, ny);
    const dim3 tiles((unsigned)((nx + 1 + kTX - 1) / kTX), (unsigned)((ny + 1 + kTY - 1) / kTY));
    const float th = (float)theta, sm = (float)smooth;
    cudaError_t e = cudaMemsetAsync(w.stats, 0, 2 * kMaxIter * sizeof(unsigned int), st);
    if (e != cudaSuccess) return prep_fail(e);
    // corners after k iterations live in plane (n_iter - k) % 2: 0 the caller's, 1 the work area's
    float *plane[2] = {Hc, w.corners};
    const long long pp[2] = {cpitch, w.tp};
    int cur = n_iter % 2;
    bathy_tile_kernel<<<tiles, kTileThreads, 0, st>>>(Hm, pitch, nx, ny, nullptr, 0, plane[cur], pp[cur], th,
                                                      sm, nullptr, nullptr);
    for (int k = 0; k < n_iter; k++) {
        // the misfit of the previous iteration's corners (none for the initial guess)
        bathy_tile_kernel<<<tiles, kTileThreads, 0, st>>>(Hm, pitch, nx, ny, plane[cur], pp[cur],
                                                          plane[cur ^ 1], pp[cur ^ 1], th, sm,
                                                          k > 0 ? w.stats + 2 * (k - 1) : nullptr,
                                                          w.stats + 2 * k + 1);
        cur ^= 1;
    }
    if (n_iter > 0)
        residual_kernel<<<grid_for(nx, ny), kBX * kBY, 0, st>>>(Hm, pitch, Hc, cpitch, nx, ny,
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
    swe::TraceRange trace("swe_land_erode");
    if (!land || !eta || !Hm || !land_out || !eta_out || !Hm_out || nx < 1 || ny < 1 || pitch < nx)
        return SWE_ERR_INVALID_ARG;
    if ((const void *)land_out == (const void *)land || eta_out == eta || Hm_out == Hm)
        return SWE_ERR_INVALID_ARG;
    if (!(land_depth >= 0.0)) return SWE_ERR_INVALID_ARG;
    auto al = [](const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; };
    if (pitch % 4 == 0 && al(land, 4) && al(land_out, 4) && al(eta, 16) && al(Hm, 16) && al(eta_out, 16) &&
        al(Hm_out, 16))
        erode4_kernel<<<grid_for(((long long)nx + 3) / 4, ny), kBX * kBY, 0, (cudaStream_t)stream>>>(
            land, eta, Hm, pitch, nx, ny, (float)land_depth, land_out, eta_out, Hm_out);
    else
        erode_kernel<<<grid_for(nx, ny), kBX * kBY, 0, (cudaStream_t)stream>>>(
            land, eta, Hm, pitch, nx, ny, (float)land_depth, land_out, eta_out, Hm_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SWE_OK : prep_fail(e);
}

int swe_refine2(const float *eta, const float *hu, const float *hv, long long pitch,
                const float *H, long long cpitch, int nx, int ny, double theta,
                float *eta_f, float *hu_f, float *hv_f, long long fpitch, float *H_f,
                long long fcpitch, void *stream) {
    swe::TraceRange trace("swe_refine2");
    if (!eta || !hu || !hv || !H || !eta_f || !hu_f || !hv_f || !H_f) return SWE_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536 || pitch < nx || cpitch < (long long)nx + 1)
        return SWE_ERR_INVALID_ARG;
    if (fpitch < 2LL * nx || (fpitch & 1) || fcpitch < 2LL * nx + 1) return SWE_ERR_INVALID_ARG;
    if (!aligned8(eta_f) || !aligned8(hu_f) || !aligned8(hv_f)) return SWE_ERR_INVALID_ARG;
    if (!(theta >= 1.0 && theta <= 2.0)) return SWE_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Planes3 in{{eta, hu, hv}};
    OutPlanes3 out{{eta_f, hu_f, hv_f}};
    auto al = [](const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; };
    if (pitch % 2 == 0 && fpitch % 4 == 0 && al(eta, 8) && al(hu, 8) && al(hv, 8) && al(eta_f, 16) &&
        al(hu_f, 16) && al(hv_f, 16))
        refine2_cells_kernel<<<grid_for(((long long)nx + 1) / 2, ny), kBX * kBY, 0, st>>>(
            in, pitch, H, cpitch, nx, ny, (float)theta, out, fpitch);
    else
        refine_cells_kernel<<<grid_for(nx, ny), kBX * kBY, 0, st>>>(in, pitch, H, cpitch, nx, ny, (float)theta,
                                                                    out, fpitch);
    refine_corners_kernel<<<grid_for(nx + 1, ny + 1), kBX * kBY, 0, st>>>(H, cpitch, nx, ny, H_f, fcpitch);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SWE_OK : prep_fail(e);
}

int swe_coarsen2(const float *eta_f, const float *hu_f, const float *hv_f, long long fpitch,
                 const float *H_f, long long fcpitch, int nx, int ny, float *eta, float *hu,
                 float *hv, long long pitch, float *H, long long cpitch, void *stream) {
    swe::TraceRange trace("swe_coarsen2");
    if (!eta_f || !hu_f || !hv_f || !H_f || !eta || !hu || !hv || !H) return SWE_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536 || pitch < nx || cpitch < (long long)nx + 1)
        return SWE_ERR_INVALID_ARG;
    if (fpitch < 2LL * nx || (fpitch & 1) || fcpitch < 2LL * nx + 1) return SWE_ERR_INVALID_ARG;
    if (!aligned8(eta_f) || !aligned8(hu_f) || !aligned8(hv_f)) return SWE_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    Planes3 fin{{eta_f, hu_f, hv_f}};
    OutPlanes3 out{{eta, hu, hv}};
    auto al = [](const void *p, uintptr_t a) { return ((uintptr_t)p & (a - 1)) == 0; };
    if (fpitch % 4 == 0 && pitch % 2 == 0 && al(eta_f, 16) && al(hu_f, 16) && al(hv_f, 16) && al(eta, 8) &&
        al(hu, 8) && al(hv, 8))
        coarsen2_cells_kernel<<<grid_for(((long long)nx + 1) / 2, ny), kBX * kBY, 0, st>>>(
            fin, fpitch, H_f, fcpitch, nx, ny, out, pitch);
    else
        coarsen_cells_kernel<<<grid_for(nx, ny), kBX * kBY, 0, st>>>(fin, fpitch, H_f, fcpitch, nx, ny, out,
                                                                     pitch);
    coarsen_corners_kernel<<<grid_for(nx + 1, ny + 1), kBX * kBY, 0, st>>>(H_f, fcpitch, nx, ny, H, cpitch);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SWE_OK : prep_fail(e);
}

}  // extern "C"
