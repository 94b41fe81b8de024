// swe_stage_fast.cu -- the FP32 stage kernels of libswe (the fast path).
//
// Same arithmetic as the reference stage kernel (swe_device.cuh), organised
// for GB300:
//  * one warp marches up a strip of 28 output columns (32 lanes: two halo
//    columns on each side), one row per iteration, keeping a three-row
//    sliding window of cell primitives in registers: every cell's
//    primitives, reconstructions and face fluxes are computed once, and the
//    x-neighbours come from warp shuffles;
//  * loads of a row are coalesced 128-byte transactions of each plane;
//  * the CFL reduction is a warp/block max, and the last block of stage 2 to
//    finish advances the device clock (t, dt, forcing brackets), so a step
//    is two launches and needs no host round trip;
//  * this translation unit is built with approximate FP32 reciprocal and
//    square root (-prec-div=false -prec-sqrt=false): ~1 ulp, far inside the
//    parity tolerance, and exact zeros stay exact (lake at rest is still
//    bit-exact).
#include "swe_device.cuh"
#include "swe_kernels.h"

namespace swe {

namespace {

constexpr int kStrip = 28;           // output columns per warp
constexpr int kWarps = 4;            // warps per block

__device__ __forceinline__ void bnd_pos_f(int k, int n, int nb, int &k0, int &k1, float &w) {
    float p = (k + 0.5f) * (float)nb / (float)n - 0.5f;
    p = fminf(fmaxf(p, 0.0f), (float)(nb - 1));
    int q = (int)floorf(p);
    if (q > nb - 1) q = nb - 1;
    k0 = q;
    k1 = q + 1 < nb ? q + 1 : nb - 1;
    w = p - q;
}

// External solution (Section 3.6) in FP32 arithmetic: the time weight was
// computed in FP64 by the clock and is rounded once here.
__device__ __forceinline__ void bnd_state_f(const StageArgs<float> &a, int e, int r, int k,
                                            int stage, float &v0, float &v1, float &v2) {
    const ForcingDev &F = a.bnd;
    int nb = e < 2 ? F.n1 : F.n2;
    int n = e < 2 ? a.nx : a.ny;
    long long off = (e >= 1 ? 6LL * F.n1 : 0) + (e >= 2 ? 6LL * F.n1 : 0) + (e >= 3 ? 6LL * F.n2 : 0);
    int k0, k1;
    float w;
    bnd_pos_f(k, n, nb, k0, k1, w);
    int fk = a.ctl->bk[stage];
    float s = (float)a.ctl->bs[stage];
    long long fs = 12LL * (F.n1 + F.n2);
    const float *A = F.frames + (long long)fk * fs + off + (long long)(r * 3) * nb;
    const float *B = F.n > 1 ? A + fs : A;
    float out[3];
    for (int v = 0; v < 3; v++) {
        float va = (1.f - w) * A[v * nb + k0] + w * A[v * nb + k1];
        float vb = (1.f - w) * B[v * nb + k0] + w * B[v * nb + k1];
        out[v] = (1.f - s) * va + s * vb;
    }
    v0 = out[0]; v1 = out[1]; v2 = out[2];
}

// Cell (i, r) with its primitives; Q* = Q^n + D1 in stage 2. Outside a
// wall the cell is land; outside a nested edge it is the ghost of
// Section 3.6 (mirrored statics, external state).
template <int STAGE>
__device__ __forceinline__ void load_cell_f(const StageArgs<float> &a, int i, int r, Cell<float> &c) {
    const int nx = a.nx, ny = a.ny;
    int si = i, sj = r, e = -1, row = 0;
    const bool ox = i < 0 || i >= nx, oy = r < 0 || r >= ny;
    c.land = true;
    c.eta = c.hu = c.hv = c.Hbar = c.HE = c.HW = c.HN = c.HS = 0.f;
    c.f = c.ct = c.st = c.hbar = c.hs = c.u = c.v = c.fvx = c.fuy = 0.f;
    if (ox && oy) return;                           // ghost-ghost corner: unused
    if (i < -2 || i > nx + 1) return;               // beyond the halo of the last strip
    if (i < 0)        { e = EDGE_W; si = -i - 1;         row = -i - 1; }
    else if (i >= nx) { e = EDGE_E; si = 2 * nx - 1 - i; row = i - nx; }
    else if (r < 0)   { e = EDGE_S; sj = -r - 1;         row = -r - 1; }
    else if (r >= ny) { e = EDGE_N; sj = 2 * ny - 1 - r; row = r - ny; }
    if (e >= 0 && a.bc[e] == BC_WALL) return;
    const long long cp = a.cpitch;
    const float *H = a.H + (long long)sj * cp + si;
    float c00 = H[0], c10 = H[1], c01 = H[cp], c11 = H[cp + 1];
    if ((c00 == kLand) | (c10 == kLand) | (c01 == kLand) | (c11 == kLand)) return;
    c.land = false;
    c.Hbar = 0.25f * (c00 + c10 + c01 + c11);
    float HE = 0.5f * (c10 + c11), HW = 0.5f * (c00 + c01);
    float HN = 0.5f * (c01 + c11), HS = 0.5f * (c00 + c10);
    if (e == EDGE_W || e == EDGE_E) { float t = HE; HE = HW; HW = t; }
    if (e == EDGE_S || e == EDGE_N) { float t = HN; HN = HS; HS = t; }
    c.HE = HE; c.HW = HW; c.HN = HN; c.HS = HS;
    const long long s = (long long)sj * a.pitch + si;
    c.f = a.f ? __ldg(a.f + s) : a.f_const;
    float th = a.th ? __ldg(a.th + s) : a.th_const;
    __sincosf(th, &c.st, &c.ct);
    if (e < 0) {
        c.eta = a.qin[0][s]; c.hu = a.qin[1][s]; c.hv = a.qin[2][s];
        if (STAGE == 2) { c.eta += a.d1[0][s]; c.hu += a.d1[1][s]; c.hv += a.d1[2][s]; }
    } else {
        int k = e >= EDGE_W ? r : i;
        bnd_state_f(a, e, row, k, STAGE - 1, c.eta, c.hu, c.hv);
    }
    make_prim(c, a.kappa, a.half_inv_kappa);
}

// The part of a cell the y-reconstruction of later rows needs.
struct RowCell {
    bool land;
    float eta, hu, hv, fuy, HN, HS, hbar, Hbar;
};

__device__ __forceinline__ RowCell keep_row(const Cell<float> &c) {
    RowCell k;
    k.land = c.land;
    k.eta = c.eta; k.hu = c.hu; k.hv = c.hv; k.fuy = c.fuy;
    k.HN = c.HN; k.HS = c.HS; k.hbar = c.hbar; k.Hbar = c.Hbar;
    return k;
}

__device__ __forceinline__ Cell<float> as_cell(const RowCell &k) {
    Cell<float> c;
    c.land = k.land;
    c.eta = k.eta; c.hu = k.hu; c.hv = k.hv; c.fuy = k.fuy; c.fvx = 0.f;
    c.HN = k.HN; c.HS = k.HS; c.hbar = k.hbar; c.Hbar = k.Hbar;
    c.HE = c.HW = 0.f;
    return c;
}

__device__ __forceinline__ float shfl_up1(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn1(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }

__device__ __forceinline__ Face<float> shfl_dn_face(const Face<float> &F) {
    Face<float> G;
    G.h = 0.f;
    G.eta = shfl_dn1(F.eta); G.hu = shfl_dn1(F.hu); G.hv = shfl_dn1(F.hv);
    G.u = shfl_dn1(F.u); G.v = shfl_dn1(F.v); G.c = shfl_dn1(F.c);
    return G;
}

// Advance the device clock after the last block of stage 2 (see
// clock_update in swe_kernels.cu).
__device__ void finish_step(const StageArgs<float> &a, float block_speed) {
    __shared__ unsigned int last;
    if (threadIdx.x == 0) {
        atomicMax(&a.ctl->speed32, __float_as_uint(block_speed));
        __threadfence();
        unsigned int prev = atomicAdd(&a.ctl->blocks_done, 1u);
        last = (prev == (unsigned int)a.nblocks - 1u);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        unsigned int bits = atomicExch(&a.ctl->speed32, 0u);
        a.ctl->blocks_done = 0u;
        clock_update(a.ctl, a.clk, a.bnd, a.wind, (double)__uint_as_float(bits), 1);
        __threadfence();
    }
}

}  // namespace

template <int STAGE, bool KAHAN>
__global__ void __launch_bounds__(kWarps * 32, 4) stage_fast_kernel(StageArgs<float> a, int rows) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int strip = blockIdx.x * kWarps + warp;
    const int i = strip * kStrip - 2 + lane;
    const int j0 = blockIdx.y * rows;
    const int j1 = min(j0 + rows, a.ny);
    const bool strip_live = strip * kStrip < a.nx;
    const bool out_lane = lane >= 2 && lane < 2 + kStrip && i < a.nx;
    const float g = a.g, kappa = a.kappa, hik = a.half_inv_kappa;
    const float dt = (float)a.ctl->dt;
    const float rho_ratio = (float)a.clk.rho_ratio;
    float speed = 0.f;

    // y-window: rows r-2 (A), r-1 (B), r (current); x-results of rows r-1, r-2
    RowCell A, B;
    A.land = B.land = true;
    float acc1[3] = {0.f, 0.f, 0.f}, acc2[3] = {0.f, 0.f, 0.f};
    float S1 = 0.f, S2 = 0.f;
    Face<float> savedN;            // finished north face of row r-2
    savedN.h = savedN.eta = savedN.hu = savedN.hv = savedN.u = savedN.v = savedN.c = 0.f;
    float Gprev[3] = {0.f, 0.f, 0.f};

    if (strip_live) {
        for (int r = j0 - 2; r <= j1 + 1; r++) {
            Cell<float> c;
            load_cell_f<STAGE>(a, i, r, c);
            float acc0[3] = {0.f, 0.f, 0.f}, S0 = 0.f;

            // ---- x: reconstruction, fluxes and cell sources of row r
            if (r >= j0 && r < j1) {
                Cell<float> L, R;
                L.land = __shfl_up_sync(0xffffffffu, c.land, 1);
                L.eta = shfl_up1(c.eta); L.hu = shfl_up1(c.hu); L.hv = shfl_up1(c.hv);
                L.fvx = shfl_up1(c.fvx);
                R.land = __shfl_down_sync(0xffffffffu, c.land, 1);
                R.eta = shfl_dn1(c.eta); R.hu = shfl_dn1(c.hu); R.hv = shfl_dn1(c.hv);
                R.fvx = shfl_dn1(c.fvx);
                Face<float> pE, pW;
                pE.h = pE.eta = pE.hu = pE.hv = pW.h = pW.eta = pW.hu = pW.hv = 0.f;
                if (!c.land) reconstruct<float, 0>(L, c, R, a.kx, a.tm, pE, pW);
                const float etaE = pE.eta, etaW = pW.eta;
                finish_face(pE, g, kappa, hik);
                finish_face(pW, g, kappa, hik);
                // east face of this lane: (own E face | west face of lane + 1)
                Face<float> nW = shfl_dn_face(pW);
                const float HWr = shfl_dn1(c.HW);
                float Fe[3] = {0.f, 0.f, 0.f};
                if (!(c.land && R.land)) {
                    Face<float> lf = c.land ? mirror<float, 0>(nW) : pE;
                    Face<float> rf = R.land ? mirror<float, 0>(pE) : nW;
                    cu_flux<float, 0>(lf, rf, c.land ? HWr : c.HE, g, Fe);
                }
                float Fw[3];
                Fw[0] = shfl_up1(Fe[0]); Fw[1] = shfl_up1(Fe[1]); Fw[2] = shfl_up1(Fe[2]);
                acc0[0] = -(Fe[0] - Fw[0]) * a.inv_dx;
                acc0[1] = -(Fe[1] - Fw[1]) * a.inv_dx + g * 0.5f * (etaE + etaW) * (c.HE - c.HW) * a.inv_dx;
                acc0[2] = -(Fe[2] - Fw[2]) * a.inv_dx;
                // Coriolis with the north vector (Section 3.7) and wind stress
                float hue = c.ct * c.hu - c.st * c.hv;
                float hvn = c.st * c.hu + c.ct * c.hv;
                acc0[1] += c.f * (c.ct * hvn - c.st * hue);
                acc0[2] += c.f * (-c.st * hvn - c.ct * hue);
                if (a.wind.n > 0) {
                    if (a.clk.wind_uniform) {
                        acc0[1] += (float)a.ctl->tau[STAGE - 1][0];
                        acc0[2] += (float)a.ctl->tau[STAGE - 1][1];
                    } else {
                        float tx, ty;
                        wind_at(a, i < 0 ? 0 : (i >= a.nx ? a.nx - 1 : i), r, STAGE - 1, rho_ratio, tx, ty);
                        acc0[1] += tx;
                        acc0[2] += ty;
                    }
                }
                S0 = c.land ? 0.f : a.cd * sqrtf(c.u * c.u + c.v * c.v) / fabsf(c.hs);
            }

            // ---- y: reconstruction of row r-1, flux across its south face
            const int ry = r - 1;
            float Gcur[3] = {0.f, 0.f, 0.f};
            if (ry >= j0 - 1 && ry <= j1) {
                Cell<float> cA = as_cell(A), cB = as_cell(B), cC;
                cC.land = c.land; cC.eta = c.eta; cC.hu = c.hu; cC.hv = c.hv; cC.fuy = c.fuy;
                Face<float> pN, pS;
                pN.h = pN.eta = pN.hu = pN.hv = pS.h = pS.eta = pS.hu = pS.hv = 0.f;
                if (!B.land) reconstruct<float, 1>(cA, cB, cC, a.ky, a.tm, pN, pS);
                const float etaN = pN.eta, etaS = pS.eta;
                finish_face(pN, g, kappa, hik);
                finish_face(pS, g, kappa, hik);
                if (ry >= j0) {
                    // face between rows ry-1 (A, its north face savedN) and ry (B)
                    if (!(A.land && B.land)) {
                        Face<float> lf = A.land ? mirror<float, 1>(pS) : savedN;
                        Face<float> rf = B.land ? mirror<float, 1>(savedN) : pS;
                        cu_flux<float, 1>(lf, rf, B.land ? A.HN : B.HS, g, Gcur);
                    }
                }
                if (ry >= j0 && ry < j1)
                    acc1[2] += g * 0.5f * (etaN + etaS) * (B.HN - B.HS) * a.inv_dy;
                savedN = pN;
            }

            // ---- output row r-2
            const int ro = r - 2;
            if (ro >= j0 && ro < j1 && out_lane && !A.land) {
                float m0 = acc2[0] - (Gcur[0] - Gprev[0]) * a.inv_dy;
                float m1 = acc2[1] - (Gcur[1] - Gprev[1]) * a.inv_dy;
                float m2 = acc2[2] - (Gcur[2] - Gprev[2]) * a.inv_dy;
                const long long s = (long long)ro * a.pitch + i;
                if (STAGE == 1) {
                    float den = 1.f / (1.f + dt * S2);
                    a.d1[0][s] = dt * m0;
                    a.d1[1][s] = (dt * m1 - dt * S2 * A.hu) * den;
                    a.d1[2][s] = (dt * m2 - dt * S2 * A.hv) * den;
                } else {
                    float q0 = a.qin[0][s], q1 = a.qin[1][s], q2 = a.qin[2][s];
                    float D0 = a.d1[0][s], D1 = a.d1[1][s], D2 = a.d1[2][s];
                    float den = 1.f / (1.f + 0.5f * dt * S2);
                    float de0 = 0.5f * (D0 + dt * m0);
                    float de1 = 0.5f * (D1 + dt * m1 - dt * S2 * q1) * den;
                    float de2 = 0.5f * (D2 + dt * m2 - dt * S2 * q2) * den;
                    float c0 = 0.f, c1 = 0.f, c2 = 0.f;
                    if (KAHAN) {
                        c0 = a.comp[0][s]; c1 = a.comp[1][s]; c2 = a.comp[2][s];
                        kahan_add(q0, c0, de0); kahan_add(q1, c1, de1); kahan_add(q2, c2, de2);
                    } else {
                        q0 += de0; q1 += de1; q2 += de2;
                    }
                    // flow relaxation, eq:frs, nested edges in the order S, N, W, E
                    for (int e = 0; e < 4; e++) {
                        if (a.bc[e] != BC_NESTED) continue;
                        int d = e == EDGE_S ? ro : e == EDGE_N ? a.ny - 1 - ro : e == EDGE_W ? i : a.nx - 1 - i;
                        if (d >= a.frs_width) continue;
                        float al = (float)a.frs_alpha[d];
                        float x0, x1, x2;
                        bnd_state_f(a, e, 0, e >= EDGE_W ? ro : i, 1, x0, x1, x2);
                        if (KAHAN) {
                            kahan_add(q0, c0, al * (x0 - q0));
                            kahan_add(q1, c1, al * (x1 - q1));
                            kahan_add(q2, c2, al * (x2 - q2));
                        } else {
                            q0 += al * (x0 - q0); q1 += al * (x1 - q1); q2 += al * (x2 - q2);
                        }
                    }
                    a.qout[0][s] = q0; a.qout[1][s] = q1; a.qout[2][s] = q2;
                    if (KAHAN) { a.comp[0][s] = c0; a.comp[1][s] = c1; a.comp[2][s] = c2; }
                    if (!(isfinite(q0) && isfinite(q1) && isfinite(q2))) flag_error(a.ctl, ro * a.nx + i);
                    speed = fmaxf(speed, cell_speed(a, q0, q1, q2, A.Hbar));
                }
            }

            // ---- shift the window
            Gprev[0] = Gcur[0]; Gprev[1] = Gcur[1]; Gprev[2] = Gcur[2];
            acc2[0] = acc1[0]; acc2[1] = acc1[1]; acc2[2] = acc1[2]; S2 = S1;
            acc1[0] = acc0[0]; acc1[1] = acc0[1]; acc1[2] = acc0[2]; S1 = S0;
            A = B;
            B = keep_row(c);
        }
    }

    if (STAGE == 2) {
        __shared__ float sh[kWarps];
        for (int o = 16; o > 0; o >>= 1) speed = fmaxf(speed, __shfl_xor_sync(0xffffffffu, speed, o));
        if (lane == 0) sh[warp] = speed;
        __syncthreads();
        float bs = 0.f;
        if (threadIdx.x == 0)
            for (int w = 0; w < kWarps; w++) bs = fmaxf(bs, sh[w]);
        finish_step(a, bs);
    }
}

// ---------------------------------------------------------------------------
// launch configuration

int fast_rows(int nx, int ny) {
    // enough warps to fill 152 SMs at ~16 resident warps each before growing
    // the strips (halo rows cost 4 loads and 2 reconstructions per strip)
    long long strips = (nx + kStrip - 1) / kStrip;
    int rows = 64;
    while (rows > 8 && strips * ((ny + rows - 1) / rows) < 152LL * 16) rows >>= 1;
    return rows;
}

dim3 fast_grid(int nx, int ny, int rows) {
    int strips = (nx + kStrip - 1) / kStrip;
    return dim3((strips + kWarps - 1) / kWarps, (ny + rows - 1) / rows);
}

int fast_step_parts() { return 2; }

const char *fast_part_name(int part) {
    static const char *names[2] = {"stage1", "stage2"};
    return part >= 0 && part < 2 ? names[part] : "";
}

cudaError_t launch_step_fast_part(const StageArgs<float> &a0, cudaStream_t st, int part, bool kahan) {
    StageArgs<float> a = a0;
    int rows = fast_rows(a.nx, a.ny);
    dim3 g = fast_grid(a.nx, a.ny, rows);
    a.nblocks = (int)(g.x * g.y);
    dim3 b(kWarps * 32);
    if (part == 0) stage_fast_kernel<1, false><<<g, b, 0, st>>>(a, rows);
    else if (kahan) stage_fast_kernel<2, true><<<g, b, 0, st>>>(a, rows);
    else stage_fast_kernel<2, false><<<g, b, 0, st>>>(a, rows);
    return cudaGetLastError();
}

}  // namespace swe
