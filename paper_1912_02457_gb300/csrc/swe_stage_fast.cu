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
//  * ghosts of nested edges read an edge-state buffer that stage 1 fills for
//    the next time level; periodic ghosts read their periodic image;
//  * one kernel serves single domains (arguments in the launch's parameter
//    space) and batches (a device tile table), a warp per item of the
//    domain's work plan;
//  * this translation unit is built with approximate FP32 reciprocal and
//    square root (-prec-div=false -prec-sqrt=false): ~2 ulp, far inside the
//    parity tolerance, and exact zeros stay exact (lake at rest is still
//    bit-exact); denormal results flush to zero (-ftz=true: values below
//    1.2e-38, far below anything the scheme resolves).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <queue>
#include <vector>

#include "swe_device.cuh"
#include "swe_kernels.h"

namespace swe {

namespace {

constexpr int kStrip = kStripColumns;   // output columns per warp (28)
constexpr int kWarps = 4;            // warps per block
#ifndef SWE_MIN_BLOCKS
#define SWE_MIN_BLOCKS 4             // resident blocks per SM the register budget targets
#endif
#ifndef SWE_FORCE_ROWS
#define SWE_FORCE_ROWS 0             // > 0: fixed tile height (tuning builds)
#endif
#ifndef SWE_UNROLL
#define SWE_UNROLL 1                 // row iterations unrolled in the march
#endif
#define SWE_STR(x) #x
#define SWE_UNROLL_PRAGMA(n) _Pragma(SWE_STR(unroll n))

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
    // a window samples the edge at the whole domain's positions
    int n = e < 2 ? a.gnx : a.gny;
    long long off = (e >= 1 ? 6LL * F.n1 : 0) + (e >= 2 ? 6LL * F.n1 : 0) + (e >= 3 ? 6LL * F.n2 : 0);
    int k0, k1;
    float w;
    bnd_pos_f(k + (e < 2 ? a.off_x : a.off_y), n, nb, k0, k1, w);
    int fk = a.ctl->bk[stage];
    float s = a.ctl->bs_f[stage];
    long long fs = 12LL * (F.n1 + F.n2);
    const long long oa = (long long)fk * fs + off + (long long)(r * 3) * nb;
    const long long ob = F.n > 1 ? oa + fs : oa;
    auto ld = [&](long long o) { return SWE_CHECK(a, o, a.n_bnd) ? F.frames[o] : 0.f; };
    float out[3];
    for (int v = 0; v < 3; v++) {
        float va = (1.f - w) * ld(oa + v * nb + k0) + w * ld(oa + v * nb + k1);
        float vb = (1.f - w) * ld(ob + v * nb + k0) + w * ld(ob + v * nb + k1);
        out[v] = (1.f - s) * va + s * vb;
    }
    v0 = out[0]; v1 = out[1]; v2 = out[2];
}

// Offset of edge e within one time level of the edge-state buffer.
__device__ __forceinline__ int edge_base(int e, int nx, int ny) {
    return e == EDGE_S ? 0 : e == EDGE_N ? 6 * nx : e == EDGE_W ? 12 * nx : 12 * nx + 6 * ny;
}

// Evaluate the external state (bnd_state_f, stage brackets `stage`) on both
// ghost rings of every nested edge into time level `slot` of the edge-state
// buffer; entries idx, idx + stride, ... of the 4 (nx + ny) (edge, ring,
// position) entries. Every later ghost or relaxation read of that time
// level is one load of these values instead of a bracket and frame lookup.
__device__ void edge_fill(const StageArgs<float> &a, int slot, int stage, int idx, int stride) {
    if (!a.edge || a.bnd.n <= 0) return;
    const int nx = a.nx, ny = a.ny;
    const int total = 4 * (nx + ny);
    const long long base = (long long)slot * 12 * (nx + ny);
    for (; idx < total; idx += stride) {
        int e, q = idx;
        if (q < 2 * nx) e = EDGE_S;
        else if ((q -= 2 * nx) < 2 * nx) e = EDGE_N;
        else if ((q -= 2 * nx) < 2 * ny) e = EDGE_W;
        else { q -= 2 * ny; e = EDGE_E; }
        if (a.bc[e] != BC_NESTED) continue;
        const int n = e < 2 ? nx : ny;
        const int r = q / n, k = q - r * n;
        float v0, v1, v2;
        bnd_state_f(a, e, r, k, stage, v0, v1, v2);
        const long long o = base + edge_base(e, nx, ny) + 3 * r * n + k;
        if (SWE_CHECK(a, o, a.n_edge) && SWE_CHECK(a, o + 2 * n, a.n_edge)) {
            a.edge[o] = v0; a.edge[o + n] = v1; a.edge[o + 2 * n] = v2;
        }
    }
}

// Raw loads of one cell, issued one iteration ahead of use so their latency
// hides behind the current row's arithmetic. Interior cells and the ghosts
// of nested edges (Section 3.6: statics mirrored from the cells inside the
// edge, external state from the edge-state buffer) take the same loads;
// cells outside a wall, the ghost-ghost corners and lanes beyond the halo
// of the last strip are land (all four corners LAND); a ghost of a periodic
// edge is the periodic image of an interior cell. Stage 2 adds the increment
// D1 to interior cells; a ghost adds -0.0f, which leaves every value as it
// is.
template <int STAGE>
struct RawCell {
    float c00, c10, c01, c11, f, q0, q1, q2, d0, d1, d2;
};

template <int STAGE>
__device__ __forceinline__ void fetch_cell(const StageArgs<float> &a, int par, int i, int r,
                                           bool interior, RawCell<STAGE> &w,
                                           const RawCell<STAGE> *below = nullptr) {
    if (interior) {
        // the warp's whole item and its halo lie inside the domain: plain
        // loads of the cell's corners, Coriolis parameter and state; the
        // lower corners are the upper corners of the cell below when the
        // march has it
        const int cp = (int)a.cpitch;
        const int h0 = r * cp + i;
        const int s = r * (int)a.pitch + i;
        if (!(SWE_CHECK(a, h0, a.n_corner) && SWE_CHECK(a, h0 + cp + 1, a.n_corner) &&
              SWE_CHECK(a, s, a.n_plane))) {
            w.c00 = w.c10 = w.c01 = w.c11 = kLand;
            return;
        }
        const float *H = a.H + h0;
        if (below) { w.c00 = below->c01; w.c10 = below->c11; }
        else       { w.c00 = __ldg(H); w.c10 = __ldg(H + 1); }
        w.c01 = __ldg(H + cp); w.c11 = __ldg(H + cp + 1);
        w.f = a.f ? __ldg(a.f + s) : a.f_const;
        w.q0 = __ldg(a.q[par][0] + s); w.q1 = __ldg(a.q[par][1] + s); w.q2 = __ldg(a.q[par][2] + s);
        if (STAGE == 2) { w.d0 = __ldg(a.d1[0] + s); w.d1 = __ldg(a.d1[1] + s); w.d2 = __ldg(a.d1[2] + s); }
        return;
    }
    const int nx = a.nx, ny = a.ny;
    const bool ox = (unsigned)i >= (unsigned)nx, oy = (unsigned)r >= (unsigned)ny;
    int si = i, sj = r, e = -1, ring = 0;
    if (i < 0)        { e = EDGE_W; si = -i - 1;         ring = si; }
    else if (i >= nx) { e = EDGE_E; si = 2 * nx - 1 - i; ring = i - nx; }
    else if (r < 0)   { e = EDGE_S; sj = -r - 1;         ring = sj; }
    else if (r >= ny) { e = EDGE_N; sj = 2 * ny - 1 - r; ring = r - ny; }
    if (e >= 0 && a.bc[e] == BC_PERIODIC) {
        // the periodic image of an interior cell (at most two cells past the edge)
        si = i; sj = r;
        if (e >= EDGE_W) { si += si < 0 ? nx : -nx; si += si < 0 ? nx : (si >= nx ? -nx : 0); }
        else             { sj += sj < 0 ? ny : -ny; sj += sj < 0 ? ny : (sj >= ny ? -ny : 0); }
        e = -1;
    }
    if ((ox && oy) || i < -2 || i > nx + 1 || (e >= 0 && a.bc[e] != BC_NESTED)) {
        w.c00 = w.c10 = w.c01 = w.c11 = kLand;
        return;
    }
    // offsets fit in 32 bits (checked when the domain is created)
    const int cp = (int)a.cpitch;
    const int h0 = sj * cp + si;
    const int s = sj * (int)a.pitch + si;
    // an interior cell reads the state planes; a ghost reads its edge's values,
    // stage 1 at the time level of Q^n (slot par), stage 2 at the next one
    int pe = 0, ne = 0;
    if (e >= 0) {
        ne = e < 2 ? nx : ny;
        pe = (STAGE != 2 ? par : par ^ 1) * 12 * (nx + ny) + edge_base(e, nx, ny) + 3 * ring * ne +
             (e >= EDGE_W ? r : i);
    }
    if (!(SWE_CHECK(a, h0, a.n_corner) && SWE_CHECK(a, h0 + cp + 1, a.n_corner) && SWE_CHECK(a, s, a.n_plane) &&
          (e < 0 || (SWE_CHECK(a, pe, a.n_edge) && SWE_CHECK(a, pe + 2 * ne, a.n_edge))))) {
        w.c00 = w.c10 = w.c01 = w.c11 = kLand;
        return;
    }
    const float *H = a.H + h0;
    w.c00 = __ldg(H); w.c10 = __ldg(H + 1); w.c01 = __ldg(H + cp); w.c11 = __ldg(H + cp + 1);
    w.f = a.f ? __ldg(a.f + s) : a.f_const;
    const float *p0 = a.q[par][0] + s, *p1 = a.q[par][1] + s, *p2 = a.q[par][2] + s;
    if (e >= 0) {
        p0 = a.edge + pe;
        p1 = p0 + ne;
        p2 = p1 + ne;
    }
    w.q0 = __ldg(p0); w.q1 = __ldg(p1); w.q2 = __ldg(p2);
    if (STAGE == 2) {
        w.d0 = w.d1 = w.d2 = -0.0f;
        if (e < 0) { w.d0 = __ldg(a.d1[0] + s); w.d1 = __ldg(a.d1[1] + s); w.d2 = __ldg(a.d1[2] + s); }
    }
}

template <int STAGE>
__device__ __forceinline__ void decode_cell(const StageArgs<float> &a, int i, int r,
                                            const RawCell<STAGE> &w, Cell<float> &c) {
    c.land = (w.c00 == kLand) | (w.c10 == kLand) | (w.c01 == kLand) | (w.c11 == kLand);
    if (c.land) {
        c.eta = c.hu = c.hv = c.Hbar = c.HE = c.HW = c.HN = c.HS = 0.f;
        c.f = c.hbar = c.hs = c.u = c.v = c.fvx = c.fuy = 0.f;
        return;
    }
    c.Hbar = 0.25f * (w.c00 + w.c10 + w.c01 + w.c11);
    float HE = 0.5f * (w.c10 + w.c11), HW = 0.5f * (w.c00 + w.c01);
    float HN = 0.5f * (w.c01 + w.c11), HS = 0.5f * (w.c00 + w.c10);
    // a nested ghost's statics are mirrored across its edge (a periodic
    // ghost is its periodic image, unmirrored)
    const bool swap_x = (unsigned)i >= (unsigned)a.nx && a.bc[EDGE_W] != BC_PERIODIC;
    const bool swap_y = (unsigned)r >= (unsigned)a.ny && a.bc[EDGE_S] != BC_PERIODIC;
    c.HE = swap_x ? HW : HE; c.HW = swap_x ? HE : HW;
    c.HN = swap_y ? HS : HN; c.HS = swap_y ? HN : HS;
    c.f = w.f;
    c.eta = w.q0; c.hu = w.q1; c.hv = w.q2;
    if (STAGE == 2) { c.eta += w.d0; c.hu += w.d1; c.hv += w.d2; }
    // primitives (Sections 3.1, 3.2, 3.7): hbar, h*, u = hu/h*, v = hv/h*.
    // The north-vector projection of Section 3.7 enters the reconstruction
    // as f x.[v^n, -u^e] and -f y.[v^n, -u^e]; rotating (u, v) into the
    // local east/north frame and back is the identity for every angle, so
    // these are f v and f u and the north angle is not read.
    c.hbar = c.eta + c.Hbar;
    c.hs = desing(c.hbar, a.kappa, a.half_inv_kappa);
    const float rcp = 1.f / c.hs;
    c.u = c.hu * rcp;
    c.v = c.hv * rcp;
    c.fvx = c.f * c.v;
    c.fuy = c.f * c.u;
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

// Advance the device clock after the last block of stage 2 (clock_update in
// swe_device.cuh).
__device__ void finish_step(const StageArgs<float> &a, float block_speed, int nblocks, int mode) {
    if (threadIdx.x != 0) return;
    atomicMax(&a.ctl->speed32, __float_as_uint(block_speed));
    // a sub-domain leaves its maximum for the clock of all sub-domains
    if (mode == 5) return;
    __threadfence();                           // the block's maximum lands before its count
    // every block loads the clock's inputs while its count is in flight;
    // the last one then needs no further round trip to memory
    ClockIn c;
    clock_load_state(a.ctl, c, mode);
    const unsigned int prev = atomicAdd(&a.ctl->blocks_done, 1u);
    clock_load_forcing(a.clk, a.bnd, a.wind, c);
    if (prev != (unsigned int)nblocks - 1u) return;
    // atomics are performed at L2, so the exchange sees every block's
    // maximum; the next kernel sees the clock's writes (kernel boundary)
    const unsigned int bits = atomicExch(&a.ctl->speed32, 0u);
    a.ctl->blocks_done = 0u;
    clock_advance(a.ctl, a.clk, a.bnd, a.wind, (double)__uint_as_float(bits), mode, c);
}

}  // namespace

// Per-warp constants of one strip.
struct StripCtx {
    int lane, i, j0, j1, par;
    bool out_lane, frs_tile, wind_on;
    float dt, taux, tauy, rho_ratio;
};

// The sliding window carried from row to row.
struct Window {
    RowCell A, B;                  // rows r-2 and r-1
    float acc1[3], acc2[3];        // x-part of rows r-1 and r-2 (+ bed term in y)
    float S1, S2;                  // drag rate of rows r-1 and r-2
    Face<float> savedN;            // finished north face of row r-2
    float Gprev[3];                // y-flux across the south face of row r-2
    float speed;                   // running CFL maximum (stage 2)
    float fx, fy;                  // largest one-sided face speeds along x and y (speed pass)
};

// One row of the march: the x-part of row r (X), the y-reconstruction of
// row r-1 (Y) and the flux across its south face (G), and the update of row
// r-2 (OUT); the flags are warp-uniform. This body is instantiated once per
// kernel and wind kind on purpose: every cell of a domain then runs the same
// machine code wherever it sits in a strip, alone, in a batch or in a
// window, so results do not depend on the tiling (bit for bit, which the
// batch and split tests check). Land cells compute harmless values that
// selects discard. GW: the domain's wind is a grid sampled per cell (else
// uniform or none); uniform-wind domains carry no code of the gridded path
// in their march (with it, the coastal 1024^2 step measured 1.5% slower
// although that branch is never taken).
template <int STAGE, bool GW>
__device__ __forceinline__ void march_row(const StageArgs<float> &a, const StripCtx &k, int r,
                                          const Cell<float> &c, Window &w, const bool KAHAN,
                                          const bool X, const bool Y, const bool G, const bool OUT) {
    const float g = a.g, kappa = a.kappa, hik = a.half_inv_kappa;
    float acc0[3] = {0.f, 0.f, 0.f}, S0 = 0.f;

    // the loads of the output row are issued first so that their latency
    // hides behind the x and y work of this iteration
    const int s_out = (r - 2) * (int)a.pitch + k.i;
    const bool write = OUT && k.out_lane && !w.A.land && SWE_CHECK(a, s_out, a.n_plane);
    float oq[3] = {0.f, 0.f, 0.f}, oD[3] = {0.f, 0.f, 0.f}, oc[3] = {0.f, 0.f, 0.f};
    if (STAGE == 2 && write) {
        for (int v = 0; v < 3; v++) {
            oq[v] = __ldg(a.q[k.par][v] + s_out);
            oD[v] = __ldg(a.d1[v] + s_out);
        }
        if (KAHAN)
            for (int v = 0; v < 3; v++) oc[v] = a.comp[v][s_out];
    }

    // ---- x: reconstruction, fluxes and cell sources of row r
    float Fe[3] = {0.f, 0.f, 0.f}, etaE = 0.f, etaW = 0.f;
    if (X) {
        Cell<float> L, R;
        L.land = __shfl_up_sync(0xffffffffu, c.land, 1);
        L.eta = shfl_up1(c.eta); L.hu = shfl_up1(c.hu); L.hv = shfl_up1(c.hv);
        L.fvx = shfl_up1(c.fvx);
        R.land = __shfl_down_sync(0xffffffffu, c.land, 1);
        R.eta = shfl_dn1(c.eta); R.hu = shfl_dn1(c.hu); R.hv = shfl_dn1(c.hv);
        R.fvx = shfl_dn1(c.fvx);
        Face<float> pE, pW;
        reconstruct<float, 0>(L, c, R, a.kx, a.tm, pE, pW);
        etaE = pE.eta;
        etaW = pW.eta;
        finish_face(pE, g, kappa, hik);
        finish_face(pW, g, kappa, hik);
        // east face of this lane: (own E face | west face of lane + 1)
        Face<float> nW = shfl_dn_face(pW);
        const float HWr = shfl_dn1(c.HW);
        Face<float> lf = c.land ? mirror<float, 0>(nW) : pE;
        Face<float> rf = R.land ? mirror<float, 0>(pE) : nW;
        float sp;
        cu_flux<float, 0>(lf, rf, c.land ? HWr : c.HE, g, Fe, &sp);
        const bool none = c.land && R.land;
        Fe[0] = none ? 0.f : Fe[0]; Fe[1] = none ? 0.f : Fe[1]; Fe[2] = none ? 0.f : Fe[2];
        if (STAGE == 0) {
            // the speed pass: the east faces of lanes 1 .. 29 are the strip's
            // x-faces, those of cells -1 .. nx-1 the domain's (a face with
            // land on both sides carries no flux and no speed)
            const bool face = k.lane >= 1 && k.lane <= kStrip + 1 && k.i >= -1 && k.i < a.nx && !none;
            w.fx = fmaxf(w.fx, face ? sp : 0.f);
        }
    }
    // the x-flux difference and the cell sources (not in the speed pass)
    if (STAGE != 0 && X) {
        float Fw[3];
        Fw[0] = shfl_up1(Fe[0]); Fw[1] = shfl_up1(Fe[1]); Fw[2] = shfl_up1(Fe[2]);
        acc0[0] = -(Fe[0] - Fw[0]) * a.inv_dx;
        acc0[1] = -(Fe[1] - Fw[1]) * a.inv_dx + g * 0.5f * (etaE + etaW) * (c.HE - c.HW) * a.inv_dx;
        acc0[2] = -(Fe[2] - Fw[2]) * a.inv_dx;
        // Coriolis (Section 3.7: f x.[hv^n, -hu^e] = f hv and
        // f y.[hv^n, -hu^e] = -f hu for every north angle) and wind stress
        acc0[1] += c.f * c.hv;
        acc0[2] -= c.f * c.hu;
        if (k.wind_on) {
            if (!GW) {
                acc0[1] += k.taux;
                acc0[2] += k.tauy;
            } else {
                float tx, ty;
                wind_at(a, k.i < 0 ? 0 : (k.i >= a.nx ? a.nx - 1 : k.i), r, STAGE - 1, k.rho_ratio, tx, ty);
                acc0[1] += tx;
                acc0[2] += ty;
            }
        }
        S0 = c.land ? 0.f : a.cd * sqrtf(c.u * c.u + c.v * c.v) / fabsf(c.hs);
    }

    // ---- y: reconstruction of row r-1, flux across its south face
    float Gcur[3] = {0.f, 0.f, 0.f};
    if (Y) {
        Cell<float> cA = as_cell(w.A), cB = as_cell(w.B), cC;
        cC.land = c.land; cC.eta = c.eta; cC.hu = c.hu; cC.hv = c.hv; cC.fuy = c.fuy;
        Face<float> pN, pS;
        reconstruct<float, 1>(cA, cB, cC, a.ky, a.tm, pN, pS);
        const float etaN = pN.eta, etaS = pS.eta;
        finish_face(pN, g, kappa, hik);
        finish_face(pS, g, kappa, hik);
        if (G) {
            // face between rows r-2 (A, north face savedN) and r-1 (B)
            Face<float> lf = w.A.land ? mirror<float, 1>(pS) : w.savedN;
            Face<float> rf = w.B.land ? mirror<float, 1>(w.savedN) : pS;
            float sp;
            cu_flux<float, 1>(lf, rf, w.B.land ? w.A.HN : w.B.HS, g, Gcur, &sp);
            const bool none = w.A.land && w.B.land;
            Gcur[0] = none ? 0.f : Gcur[0]; Gcur[1] = none ? 0.f : Gcur[1]; Gcur[2] = none ? 0.f : Gcur[2];
            if (STAGE == 0) {
                // the speed pass: the faces below the item's rows and above
                // them (rows j0-1 | j0 .. j1-1 | j1) of the strip's own
                // columns inside the domain
                const bool face = k.out_lane && k.i >= 0 && !none;
                w.fy = fmaxf(w.fy, face ? sp : 0.f);
            }
        }
        // bed term of row r-1 in y (it is an output row whenever G and r-1 < j1)
        if (STAGE != 0 && G && r - 1 < k.j1)
            w.acc1[2] += g * 0.5f * (etaN + etaS) * (w.B.HN - w.B.HS) * a.inv_dy;
        w.savedN = pN;
    }

    // ---- output row r-2
    if (OUT) {
        const int ro = r - 2;
        const float m0 = w.acc2[0] - (Gcur[0] - w.Gprev[0]) * a.inv_dy;
        const float m1 = w.acc2[1] - (Gcur[1] - w.Gprev[1]) * a.inv_dy;
        const float m2 = w.acc2[2] - (Gcur[2] - w.Gprev[2]) * a.inv_dy;
        const int s = s_out;
        const float dt = k.dt, S2 = w.S2;
        if (STAGE == 1) {
            float den = 1.f / (1.f + dt * S2);
            if (write) {
                a.d1[0][s] = dt * m0;
                a.d1[1][s] = (dt * m1 - dt * S2 * w.A.hu) * den;
                a.d1[2][s] = (dt * m2 - dt * S2 * w.A.hv) * den;
            }
        } else if (write) {
            const int par = k.par;
            float q0 = oq[0], q1 = oq[1], q2 = oq[2];
            const float D0 = oD[0], D1 = oD[1], D2 = oD[2];
            float den = 1.f / (1.f + 0.5f * dt * S2);
            float de0 = 0.5f * (D0 + dt * m0);
            float de1 = 0.5f * (D1 + dt * m1 - dt * S2 * q1) * den;
            float de2 = 0.5f * (D2 + dt * m2 - dt * S2 * q2) * den;
            float c0 = oc[0], c1 = oc[1], c2 = oc[2];
            if (KAHAN) {
                kahan_add(q0, c0, de0); kahan_add(q1, c1, de1); kahan_add(q2, c2, de2);
            } else {
                q0 += de0; q1 += de1; q2 += de2;
            }
            // flow relaxation, eq:frs, nested edges in the order S, N, W, E
            for (int e = 0; k.frs_tile && e < 4; e++) {
                if (a.bc[e] != BC_NESTED) continue;
                int d = e == EDGE_S ? ro : e == EDGE_N ? a.ny - 1 - ro : e == EDGE_W ? k.i : a.nx - 1 - k.i;
                if (d >= a.frs_width) continue;
                float al = a.frs_alpha_f[d];
                // external state at the new time level, ring 0
                const int n = e < 2 ? a.nx : a.ny;
                const int pe = (par ^ 1) * 12 * (a.nx + a.ny) + edge_base(e, a.nx, a.ny) + (e >= EDGE_W ? ro : k.i);
                if (!(SWE_CHECK(a, pe, a.n_edge) && SWE_CHECK(a, pe + 2 * n, a.n_edge))) continue;
                const float *E = a.edge + pe;
                const float x0 = __ldg(E), x1 = __ldg(E + n), x2 = __ldg(E + 2 * n);
                if (KAHAN) {
                    kahan_add(q0, c0, al * (x0 - q0));
                    kahan_add(q1, c1, al * (x1 - q1));
                    kahan_add(q2, c2, al * (x2 - q2));
                } else {
                    q0 += al * (x0 - q0); q1 += al * (x1 - q1); q2 += al * (x2 - q2);
                }
            }
            a.q[par ^ 1][0][s] = q0; a.q[par ^ 1][1][s] = q1; a.q[par ^ 1][2][s] = q2;
            if (KAHAN) { a.comp[0][s] = c0; a.comp[1][s] = c1; a.comp[2][s] = c2; }
            if (!(isfinite(q0) && isfinite(q1) && isfinite(q2))) flag_error(a.ctl, ro * a.nx + k.i);
            w.speed = fmaxf(w.speed, cell_speed(a, q0, q1, q2, w.A.Hbar));
        }
    }

    // ---- shift the window
    w.Gprev[0] = Gcur[0]; w.Gprev[1] = Gcur[1]; w.Gprev[2] = Gcur[2];
    w.acc2[0] = w.acc1[0]; w.acc2[1] = w.acc1[1]; w.acc2[2] = w.acc1[2]; w.S2 = w.S1;
    w.acc1[0] = acc0[0]; w.acc1[1] = acc0[1]; w.acc1[2] = acc0[2]; w.S1 = S0;
    w.A = w.B;
    w.B = keep_row(c);
}

// One block of one domain: its kWarps warps take the warp items
// blk*kWarps .. blk*kWarps+kWarps-1 of the domain, item = band*strips + strip,
// each a strip of 28 output columns by `rows` rows. Numbering items
// linearly (instead of giving a block a 2-D tile) leaves no idle warps at
// the right edge and lets the tile height be chosen to fill whole waves.
// `nblocks`: blocks of this domain in this launch (the last of them to
// finish stage 2 advances the domain's clock).
template <int STAGE, bool GW>
__device__ __forceinline__ void stage_tile(const StageArgs<float> &a, int blk, int rows, int strips,
                                           int nblocks, const bool KAHAN) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    // warp slot -> warp item: from the domain's plan, or (without one) the
    // item-th strip of `rows`-row bands
    const int slot = blk * kWarps + warp;
    bool strip_live;
    int strip = 0, j0 = 0, j1 = 0;
    if (a.items) {
        strip_live = slot < a.n_items;
        if (strip_live && SWE_CHECK(a, slot, a.n_items)) {
            const uint2 it = __ldg(a.items + slot);
            strip = (int)it.x;
            j0 = (int)(it.y & 0xffffu);
            j1 = min(j0 + (int)(it.y >> 16), a.ny);
        }
    } else {
        const int bands = (a.ny + rows - 1) / rows;
        strip_live = slot < strips * bands;
        if (strip_live) { strip = slot % strips; j0 = slot / strips * rows; j1 = min(j0 + rows, a.ny); }
    }
    // everything above reads what no kernel writes (arguments, the plan);
    // from here on the previous kernel's results are needed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const StepCtl *ctl = a.ctl;
    const int done = ctl->done, par = ctl->parity;
    const double dt = ctl->dt;
    const float taux = STAGE == 0 ? 0.f : ctl->tau_f[STAGE - 1][0];
    const float tauy = STAGE == 0 ? 0.f : ctl->tau_f[STAGE - 1][1];
    if (done) return;                              // forecast horizon reached (block-uniform)
    StripCtx k;
    k.lane = lane;
    k.i = strip * kStrip - 2 + lane;
    k.j0 = j0;
    k.j1 = j1;
    k.par = par;
    // stage 1 also evaluates the external edge state of the next time level
    // (used by stage 2 and by stage 1 of the next step); the interior
    // blocks of the middle of the domain take it
    if (STAGE == 1) {
        const int b = blk + nblocks / 2 < nblocks ? blk + nblocks / 2 : blk + nblocks / 2 - nblocks;
        edge_fill(a, k.par ^ 1, 1, b * (kWarps * 32) + threadIdx.x, nblocks * (kWarps * 32));
    }
    k.out_lane = lane >= 2 && lane < 2 + kStrip && k.i < a.nx;
    k.dt = (float)dt;
    k.rho_ratio = (float)a.clk.rho_ratio;
    k.wind_on = a.wind.n > 0;
    k.taux = taux;
    k.tauy = tauy;
    // does any cell of this warp's strip lie in a flow-relaxation zone?
    {
        const int c0 = strip * kStrip, c1 = c0 + kStrip, fw = a.frs_width;
        k.frs_tile = STAGE == 2 &&
            ((a.bc[EDGE_S] == BC_NESTED && k.j0 < fw) || (a.bc[EDGE_N] == BC_NESTED && k.j1 > a.ny - fw) ||
             (a.bc[EDGE_W] == BC_NESTED && c0 < fw) || (a.bc[EDGE_E] == BC_NESTED && c1 > a.nx - fw));
    }
    Window w;
    w.A.land = w.B.land = true;
    w.A.eta = w.A.hu = w.A.hv = w.A.fuy = w.A.HN = w.A.HS = w.A.hbar = w.A.Hbar = 0.f;
    w.B = w.A;
    for (int q = 0; q < 3; q++) w.acc1[q] = w.acc2[q] = w.Gprev[q] = 0.f;
    w.S1 = w.S2 = 0.f;
    w.savedN.h = w.savedN.eta = w.savedN.hu = w.savedN.hv = w.savedN.u = w.savedN.v = w.savedN.c = 0.f;
    w.speed = 0.f;
    w.fx = w.fy = 0.f;

    if (strip_live) {
        const int i = k.i, j0 = k.j0, j1 = k.j1, par = k.par;
        RawCell<STAGE> cur, nxt;
        // warp-uniform: every cell the march loads is an interior cell
        const bool interior = strip * kStrip - 2 >= 0 && strip * kStrip + 29 < a.nx && j0 - 2 >= 0 &&
                              j1 + 1 < a.ny;
        fetch_cell<STAGE>(a, par, i, j0 - 2, interior, cur);
        // the two rows below the item only fill the window
        for (int r = j0 - 2; r < j0; r++) {
            fetch_cell<STAGE>(a, par, i, r + 1, interior, nxt, &cur);
            Cell<float> c;
            decode_cell<STAGE>(a, i, r, cur, c);
            march_row<STAGE, GW>(a, k, r, c, w, KAHAN, false, false, false, false);
            cur = nxt;
        }
        // then each row runs its x part, the y part of the row below, the
        // flux between them and the update of row r - 2. In stage 2 the
        // first three run on every row as one straight-line body, so the two
        // independent chains can interleave (the x parts of rows j1 and
        // j1 + 1 and the first flux reach no output; stage 2 measured 42.9 ->
        // 40.9 us on the coastal 1024 step, stage 1 1% slower, so it keeps
        // the exact flags)
        SWE_UNROLL_PRAGMA(SWE_UNROLL)
        for (int r = j0; r <= j1 + 1; r++) {
            if (r <= j1) fetch_cell<STAGE>(a, par, i, r + 1, interior, nxt, &cur);
            Cell<float> c;
            decode_cell<STAGE>(a, i, r, cur, c);
            march_row<STAGE, GW>(a, k, r, c, w, KAHAN, STAGE == 2 || r < j1, true, STAGE == 2 || r >= j0 + 1,
                             STAGE != 0 && r >= j0 + 2);
            cur = nxt;
        }
    }

    if (STAGE == 0 || STAGE == 2) {
        // stage 2: the CFL maximum of the cells (eq:cfl with the cell
        // averages); the speed pass: the largest face speed over the cell
        // size (eq:cfl with the faces' one-sided speeds)
        __shared__ float sh[kWarps];
        // a window of a larger domain takes the maximum over its own cells:
        // its halo rows are not in its plan, and the lanes of its halo
        // columns (written, then overwritten by the halo exchange) drop out
        // here, once, rather than in every row
        const bool own_col = (unsigned)(k.i - a.own_x0) < (unsigned)(a.own_x1 - a.own_x0);
        float speed = STAGE == 0 ? fmaxf(w.fx * a.inv_dx, w.fy * a.inv_dy) : (own_col ? w.speed : 0.f);
        for (int o = 16; o > 0; o >>= 1) speed = fmaxf(speed, __shfl_xor_sync(0xffffffffu, speed, o));
        if (lane == 0) sh[warp] = speed;
        __syncthreads();
        float bs = 0.f;
        if (threadIdx.x == 0)
            for (int q = 0; q < kWarps; q++) bs = fmaxf(bs, sh[q]);
        finish_step(a, bs, nblocks, STAGE == 0 ? 3 : a.clk.split ? 5 : (a.clk.cfl_faces ? 4 : 1));
    }
}

// Batch kernel: block t takes tile t of the tile table of all domains
// (tile t belongs to the domain d = tile_dom[t], tile_start[d] <= t <
// tile_start[d+1]; a grid smaller than the table walks it with a stride).
// One block per tile lets the hardware scheduler balance uneven tiles (7%
// faster than a persistent grid on a 64-domain ensemble); the table lives
// in device memory, so a captured graph stays valid while domains come and
// go with an unchanged tile count. A single domain comes
// with the launch instead (`one`, tiles > 0): its arguments sit in the
// kernel's parameter space, so a launch does not start with a chain of
// table lookups in global memory. Either way the tile work below is the one
// call site of stage_tile, so a domain computes the same bits alone or in
// a batch. GW: the kernel for domains with gridded wind (a batch with any
// such domain launches it for all of them; uniform-wind domains alone and
// in uniform batches launch the other).
template <int STAGE, bool GW>
__global__ void __launch_bounds__(kWarps * 32, SWE_MIN_BLOCKS)
stage_batch_kernel(const BatchTable tab, const __grid_constant__ OneDomain one) {
    // the domain's arguments, staged once per block in shared memory (they
    // are read uniformly by every thread)
    __shared__ StageArgs<float> sa;
    // the next stage kernel may start its prologue while this one drains
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const bool single = one.tiles > 0;
    const int n_dom = single ? 1 : *tab.n_domains;
    const int total = single ? one.tiles : (n_dom > 0 ? tab.tile_start[n_dom] : 0);
    int have = -1;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int d = 0, first = 0, ntiles = one.tiles, rows = one.rows, strips = one.strips;
        if (!single) {
            d = tab.tile_dom[t];
            first = tab.tile_start[d];
            ntiles = tab.tile_start[d + 1] - first;
            rows = tab.rows[d];
            strips = tab.grid_x[d];
        }
        if (d != have) {
            const int *src = single ? reinterpret_cast<const int *>(&one.args)
                                    : reinterpret_cast<const int *>(tab.args + d);
            int *dst = reinterpret_cast<int *>(&sa);
            for (int k = threadIdx.x; k < (int)(sizeof(StageArgs<float>) / sizeof(int)); k += blockDim.x)
                dst[k] = src[k];
            __syncthreads();
            have = d;
        }
        stage_tile<STAGE, GW>(sa, t - first, rows, strips, ntiles, sa.comp[0] != nullptr);
        __syncthreads();                        // shared scratch reused by the next tile
    }
}

// ---------------------------------------------------------------------------
// launch configuration

static int warp_slots() {
    static int slots = 0;
    if (!slots) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, stage_batch_kernel<2, false>, kWarps * 32, 0);
        slots = (sms > 0 ? sms : 152) * (per_sm > 0 ? per_sm : 4) * kWarps;
    }
    return slots;
}

// ---------------------------------------------------------------------------
// work planning: warp items of variable height
//
// A warp item is a strip of 28 output columns by a run of rows
// [j0, j0 + n), packed as {strip, j0 | n << 16}. A row costs about the same
// everywhere except where the march takes the general load path (the
// strips whose lanes reach past the west or east edge, and the items at the
// south and north edges: ~17% more per row), in the strips whose outer
// lanes are ghosts of a nested edge (another ~20%: the edge-state loads)
// and, in stage 2, in flow-relaxation zones (~8%). The weights are fitted
// to per-warp times of both stages on the coastal 1024 x 1024 step (per-row
// cost over an interior row, stage 1 / stage 2: east wall strip 1.20 /
// 1.16, south and north edge items 1.21 / 1.29, nested west strip 1.38 /
// 1.43); the earlier weights (ghost strips +10%, relaxation +13%, no
// general-path term) left the west strip's items ending ~5 us after the
// median warp of stage 2, and refitting took stage 2 from 38.9 to 36.8 us
// and the step from 18.1e9 to 18.9e9 cell-updates/s back to back. The
// four halo rows a march adds cost about a quarter of a row each (weighed
// at a third before: the coastal step measured 1.7% faster flushed with a
// quarter, the size sweep unchanged). Rows without a wet cell in the
// strip are left out (land cells are never written and never enter the CFL
// maximum, and a march recomputes its own halo): each strip falls into
// segments of wet rows, split where a land run is longer than a halo. A
// budget (kPlanUnit per plain row) cuts a segment of cost C into
// ceil(C / budget) items of equal cost, so the item count follows the
// budget smoothly and fast_budget can fill the GPU's resident warp slots.

namespace {

constexpr int kNonIntCost = 17, kGhostCost = 20, kFrsCost = 8, kHaloCost = 100;
constexpr int kEdgeRows = 12;

struct PlanCtx {
    int nx, ny, strips, fw;
    bool nest[4];
    const unsigned char *wet;       // strips x ny, strip-major; NULL: all wet
    bool is_wet(int j, int s) const { return !wet || wet[(size_t)s * ny + j] != 0; }
    // the strips whose lanes reach past the west or east edge march on the
    // general load path (ghost handling on every row)
    bool cols_edge(int s) const { return s * kStrip - 2 < 0 || s * kStrip + 29 >= nx; }
    int strip_extra(int s) const {
        int c = cols_edge(s) ? kNonIntCost : 0;
        if ((s == 0 && nest[EDGE_W]) || (s == strips - 1 && nest[EDGE_E])) c += kGhostCost;
        const int c0 = s * kStrip, c1 = std::min(c0 + kStrip, nx);
        if ((nest[EDGE_W] && c0 < fw) || (nest[EDGE_E] && c1 > nx - fw)) c += kFrsCost;
        return c;
    }
    int row_cost(int j, int s, int xs) const {
        const bool frs = is_wet(j, s) && ((nest[EDGE_S] && j < fw) || (nest[EDGE_N] && j >= ny - fw));
        // the first and last item of a strip (about kEdgeRows rows) march on
        // the general load path too
        const bool edge = !cols_edge(s) && (j < kEdgeRows || j >= ny - kEdgeRows);
        return kPlanUnit + xs + (frs ? kFrsCost : 0) + (edge ? kNonIntCost : 0);
    }
};

struct Segment {
    int strip, start, rows;
    long long cost;
};

PlanCtx plan_ctx(int nx, int ny, const unsigned char *wet, const int bc[4], int frs_width) {
    PlanCtx p;
    p.nx = nx; p.ny = ny; p.strips = (nx + kStrip - 1) / kStrip; p.fw = frs_width; p.wet = wet;
    for (int e = 0; e < 4; e++) p.nest[e] = bc[e] == BC_NESTED;
    return p;
}

std::vector<Segment> plan_segments(const PlanCtx &p) {
    std::vector<Segment> seg;
    for (int s = 0; s < p.strips; s++) {
        const int xs = p.strip_extra(s);
        int j = 0;
        for (;;) {
            while (j < p.ny && !p.is_wet(j, s)) j++;
            if (j >= p.ny) break;
            const int start = j;
            int end = j;                // one past the last wet row
            while (j < p.ny) {
                if (p.is_wet(j, s)) { end = ++j; continue; }
                int L = 0;
                while (j + L < p.ny && !p.is_wet(j + L, s)) L++;
                if (j + L >= p.ny || L * kPlanUnit >= kHaloCost) break;
                j += L;
            }
            long long c = 0;
            for (int r = start; r < end; r++) c += p.row_cost(r, s, xs);
            seg.push_back({s, start, end - start, c});
            j = end;
        }
    }
    return seg;
}

// items of one segment under a budget
long long seg_items(const Segment &g, int budget) {
    return std::min<long long>(g.rows, std::max<long long>(1, (g.cost + budget - 1) / budget));
}

}  // namespace

int fast_strips(int nx) { return (nx + kStrip - 1) / kStrip; }

int fast_budget(int nx, int ny, const unsigned char *wet, const int bc[4], int frs_width) {
    if (SWE_FORCE_ROWS > 0) return SWE_FORCE_ROWS * kPlanUnit;
    const std::vector<Segment> seg = plan_segments(plan_ctx(nx, ny, wet, bc, frs_width));
    // Score: the fraction of the last wave filled (items / whole waves of
    // resident warps) times the share of the work that is not halo. Items
    // are kept to 32 rows or fewer: longer marches measured slower on every
    // domain that needs them (2048^2 to 8192^2 coastal: 6-12%), even where
    // they would fill the slots exactly. Small domains take items down to two
    // rows: a warp's march is a chain of dependent row iterations, so short
    // items on more warps finish sooner (350^2: 35%, 512^2: 20% faster than
    // items of eight rows or more).
    const double slots = warp_slots();
    int best = 2 * kPlanUnit;
    double best_score = -1.0;
    for (int b = 2 * kPlanUnit; b <= 32 * kPlanUnit; b += kPlanUnit / 20) {
        long long n = 0, work = 0;
        for (const Segment &g : seg) {
            const long long k = seg_items(g, b);
            n += k;
            work += g.cost + k * kHaloCost;
        }
        if (n == 0) return 8 * kPlanUnit;      // all land: one no-op item whatever the budget
        const double waves = (double)n / slots;
        const double fill = waves / (waves <= 1.0 ? 1.0 : std::ceil(waves - 1e-9));
        const double useful = (double)(work - n * kHaloCost) / (double)work;
        const double score = fill * useful;
        if (score > best_score + 1e-12) { best_score = score; best = b; }
    }
    return best;
}

void fast_plan(int nx, int ny, const unsigned char *wet, const int bc[4], int frs_width, int budget,
               bool alone, std::vector<uint2> &items) {
    items.clear();
    const PlanCtx p = plan_ctx(nx, ny, wet, bc, frs_width);
    std::vector<long long> pref, cost;
    for (const Segment &g : plan_segments(p)) {
        const int xs = p.strip_extra(g.strip);
        pref.assign((size_t)g.rows + 1, 0);
        for (int r = 0; r < g.rows; r++) pref[r + 1] = pref[r] + p.row_cost(g.start + r, g.strip, xs);
        const int k = (int)seg_items(g, budget);
        // cut where the cost prefix is nearest to cost * q / k, each item
        // keeping at least one row
        int r0 = 0;
        for (int q = 1; q <= k; q++) {
            int r1 = g.rows;
            if (q < k) {
                const long long target = g.cost * q / k;
                r1 = r0 + 1;
                while (r1 < g.rows - (k - q) && pref[r1] < target) r1++;
                if (r1 - 1 > r0 && target - pref[r1 - 1] < pref[r1] - target) r1--;
            }
            items.push_back(make_uint2((unsigned)g.strip, (unsigned)(g.start + r0) | ((unsigned)(r1 - r0) << 16)));
            cost.push_back(pref[r1] - pref[r0] + kHaloCost);
            r0 = r1;
        }
    }
    if (items.empty()) { items.push_back(make_uint2(0u, 1u << 16)); cost.push_back(1); }
    const int n = (int)items.size(), nb = (n + kWarps - 1) / kWarps;
    const auto row_major = [&](int a, int c) {
        const unsigned ja = items[a].y & 0xffffu, jc = items[c].y & 0xffffu;
        return ja != jc ? ja < jc : items[a].x < items[c].x;
    };
    std::vector<int> order(n);
    for (int k = 0; k < n; k++) order[k] = k;
    std::vector<uint2> out;
    out.reserve(n);
    if (!alone || n > warp_slots() || budget < 8 * kPlanUnit) {
        // part of a batch, several waves, or short items: row-major order,
        // a block's warps taking neighbouring strips of the same rows (they
        // share halo lines in L1, which short items and later waves depend
        // on; measured 1-2% faster than balanced blocks there)
        std::sort(order.begin(), order.end(), row_major);
        for (int k : order) out.push_back(items[k]);
        items.swap(out);
        return;
    }
    // one wave of long items: blocks of kWarps items with equal total cost
    // (largest item first to the lightest block with room), so that the SMs,
    // whichever blocks they get, carry equal work (coastal 1024^2: +2.6%);
    // within a block, row-major order. (When the item count is not a
    // multiple of kWarps a packed block other than the last may hold fewer
    // items, and the launch's blocks then straddle packed blocks after it;
    // keeping every short block last measured no different.)
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    typedef std::pair<long long, int> Load;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int b = 0; b < nb; b++) heap.push(Load(0, b));
    std::vector<std::vector<int>> blk(nb);
    for (int k : order) {
        Load l = heap.top();
        heap.pop();
        blk[l.second].push_back(k);
        if ((int)blk[l.second].size() < kWarps) heap.push(Load(l.first + cost[k], l.second));
    }
    for (int b = 0; b < nb; b++) {
        std::sort(blk[b].begin(), blk[b].end(), row_major);
        for (int k : blk[b]) out.push_back(items[k]);
    }
    items.swap(out);
}

int fast_step_parts(bool faces) { return faces ? 3 : 2; }

const char *fast_part_name(int part, bool faces) {
    static const char *names[3] = {"speed", "stage1", "stage2"};
    if (faces) return part >= 0 && part < 3 ? names[part] : "";
    return part >= 0 && part < 2 ? names[part + 1] : "";
}

// Blocks (of kWarps warp items) a launch over n_items items needs.
int fast_tiles(int n_items) { return (n_items + kWarps - 1) / kWarps; }

// Per 28-column strip s and row j (out[s * ny + j], strip-major for the
// planner's walk down each strip): does the strip hold a wet cell of row j
// (a cell is land when any of its corners is LAND, as in decode_cell)?
__global__ void wet_strips_kernel(const float *__restrict__ H, long long cpitch, int nx, int ny, int strips,
                                  unsigned char *__restrict__ out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)ny * strips) return;
    const int j = (int)(t / strips), s = (int)(t % strips);
    const int c0 = s * kStrip, c1 = min(c0 + kStrip, nx);
    const float *r0 = H + (long long)j * cpitch, *r1 = r0 + cpitch;
    bool wet = false;
    for (int i = c0; i < c1 && !wet; i++)
        wet = !(r0[i] == kLand || r0[i + 1] == kLand || r1[i] == kLand || r1[i + 1] == kLand);
    out[(long long)s * ny + j] = wet ? 1 : 0;
}

cudaError_t launch_wet_strips(const float *H, long long cpitch, int nx, int ny, unsigned char *out,
                              cudaStream_t st) {
    const int strips = fast_strips(nx);
    const long long n = (long long)ny * strips;
    wet_strips_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(H, cpitch, nx, ny, strips, out);
    return cudaGetLastError();
}

// The external edge state of the current time level (stage-1 brackets).
__global__ void __launch_bounds__(256) edge_fill_kernel(const StageArgs<float> a) {
    edge_fill(a, a.ctl->parity, 0, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

long long edge_floats(int nx, int ny) { return 2LL * 12 * ((long long)nx + ny); }

cudaError_t launch_edge_fill(const StageArgs<float> &a, cudaStream_t st) {
    if (!a.edge || a.bnd.n <= 0) return cudaSuccess;
    const int total = 4 * (a.nx + a.ny);
    edge_fill_kernel<<<(total + 255) / 256, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// Stage launches carry the programmatic-stream-serialisation attribute: a
// stage kernel that follows another stage kernel in the stream (or in a
// captured graph) is scheduled while that kernel drains (it triggers its
// dependents at its start); its blocks stage their arguments and load
// their items, which no kernel writes, and then wait in
// griddepcontrol.wait for the previous kernel's completion and its writes
// (back-to-back steps 2.2% faster on the coastal 1024^2 step). After any
// other stream work a launch is ordered as usual.
static cudaError_t launch_stage(int stage, int blocks, const BatchTable &tab, const OneDomain &one,
                                bool gridded, cudaStream_t st) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kWarps * 32);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = stage == 0 ? cudaLaunchKernelEx(&cfg, stage_batch_kernel<0, false>, tab, one)
                    : stage == 1 ? (gridded ? cudaLaunchKernelEx(&cfg, stage_batch_kernel<1, true>, tab, one)
                                            : cudaLaunchKernelEx(&cfg, stage_batch_kernel<1, false>, tab, one))
                                 : (gridded ? cudaLaunchKernelEx(&cfg, stage_batch_kernel<2, true>, tab, one)
                                            : cudaLaunchKernelEx(&cfg, stage_batch_kernel<2, false>, tab, one));
    return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_batch_stage(const BatchTable &tab, int blocks, int stage, bool gridded, cudaStream_t st) {
    OneDomain none;
    memset(&none, 0, sizeof none);
    return launch_stage(stage, blocks, tab, none, gridded, st);
}

cudaError_t launch_domain_stage(const OneDomain &one, int stage, cudaStream_t st) {
    BatchTable tab;
    memset(&tab, 0, sizeof tab);
    return launch_stage(stage, one.tiles, tab, one, one.args.wind.n > 0 && !one.args.clk.wind_uniform, st);
}

}  // namespace swe
