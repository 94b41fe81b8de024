// swe_kernels.cu -- stage, reduction, clock and diagnostic kernels of libswe.
//
// One time step is two launches of the stage kernel (eq:rk2_semiimp) and a
// one-thread clock kernel:
//   stage 1: M(Q^n), S(Q^n) at time t        -> D1 = Q* - Q^n
//   stage 2: M(Q*),  S(Q*)  at time t + dt   -> Q^{n+1}, flow relaxation,
//            block-max of the CFL wave speed (atomicMax into the clock)
//   clock:   t += dt, next dt from the max speed (eq:cfl), forcing brackets.
// The reference stage kernel here maps one thread to one cell and reads its
// radius-2 plus-shaped stencil straight from global memory.
#include "swe_device.cuh"
#include "swe_kernels.h"

namespace swe {

// ---------------------------------------------------------------------------
// stencil loads

template <typename T>
__device__ __forceinline__ void sincos_t(T x, T *s, T *c);
template <>
__device__ __forceinline__ void sincos_t<float>(float x, float *s, float *c) { sincosf(x, s, c); }
template <>
__device__ __forceinline__ void sincos_t<double>(double x, double *s, double *c) { sincos(x, s, c); }

// Cell (i, j) of the stencil, i and j possibly one or two cells outside the
// domain. Outside a wall edge the cell is land (a wall is the land-mask
// wall of Section 3.4, which equals the ghost mirror of Section 3.3).
// Outside a nested edge it is a ghost cell: bathymetry, f and theta of the
// mirrored interior cell (faces swapped), state from the external frames
// at the stage time (Section 3.6). Outside a periodic edge it is the
// periodic image of an interior cell (Section 3.3).
template <typename T, int STAGE>
__device__ __forceinline__ void load_cell(const StageArgs<T> &a, int par, int i, int j, Cell<T> &c) {
    const int nx = a.nx, ny = a.ny;
    int si = i, sj = j, e = -1, row = 0;
    if (i < 0)        { e = EDGE_W; si = -i - 1;         row = -i - 1; }
    else if (i >= nx) { e = EDGE_E; si = 2 * nx - 1 - i; row = i - nx; }
    else if (j < 0)   { e = EDGE_S; sj = -j - 1;         row = -j - 1; }
    else if (j >= ny) { e = EDGE_N; sj = 2 * ny - 1 - j; row = j - ny; }
    if (e >= 0 && a.bc[e] == BC_WALL) { c.land = true; return; }
    if (e >= 0 && a.bc[e] == BC_PERIODIC) {
        // the periodic image of an interior cell, statics and state alike
        // (the stencil reaches at most two cells past an edge)
        si = i; sj = j;
        if (e >= EDGE_W) { si += si < 0 ? nx : -nx; si += si < 0 ? nx : (si >= nx ? -nx : 0); }
        else             { sj += sj < 0 ? ny : -ny; sj += sj < 0 ? ny : (sj >= ny ? -ny : 0); }
        e = -1;
    }
    const long long cp = a.cpitch;
    const T *H = a.H + (long long)sj * cp + si;
    T c00 = H[0], c10 = H[1], c01 = H[cp], c11 = H[cp + 1];
    const T L = T(kLand);
    c.land = (c00 == L) | (c10 == L) | (c01 == L) | (c11 == L);
    if (c.land) return;
    c.Hbar = T(0.25) * (c00 + c10 + c01 + c11);
    T HE = T(0.5) * (c10 + c11), HW = T(0.5) * (c00 + c01);
    T HN = T(0.5) * (c01 + c11), HS = T(0.5) * (c00 + c10);
    if (e == EDGE_W || e == EDGE_E) { T t = HE; HE = HW; HW = t; }
    if (e == EDGE_S || e == EDGE_N) { T t = HN; HN = HS; HS = t; }
    c.HE = HE; c.HW = HW; c.HN = HN; c.HS = HS;
    const long long s = (long long)sj * a.pitch + si;
    c.f = a.f ? a.f[s] : a.f_const;
    T th = a.th ? a.th[s] : a.th_const;
    sincos_t(th, &c.st, &c.ct);
    if (e < 0) {
        c.eta = a.q[par][0][s]; c.hu = a.q[par][1][s]; c.hv = a.q[par][2][s];
        if (STAGE == 2) { c.eta += a.d1[0][s]; c.hu += a.d1[1][s]; c.hv += a.d1[2][s]; }
    } else {
        int k = e >= EDGE_W ? j : i;
        c.eta = bnd_value(a, e, row, 0, k, STAGE - 1);
        c.hu = bnd_value(a, e, row, 1, k, STAGE - 1);
        c.hv = bnd_value(a, e, row, 2, k, STAGE - 1);
    }
    make_prim(c, a.kappa, a.half_inv_kappa);
}

// ---------------------------------------------------------------------------
// block reductions

template <typename T>
__device__ __forceinline__ T block_max(T v, T *sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    int tid = threadIdx.x + threadIdx.y * blockDim.x;
    int nw = (blockDim.x * blockDim.y + 31) >> 5;
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        v = tid < nw ? sh[tid] : T(0);
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

__device__ __forceinline__ void speed_atomic_max(StepCtl *ctl, float v) {
    atomicMax(&ctl->speed32, __float_as_uint(v));
}
__device__ __forceinline__ void speed_atomic_max(StepCtl *ctl, double v) {
    atomicMax(&ctl->speed64, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// the reference stage kernel: one thread per cell

template <typename T, int STAGE, bool KAHAN>
__global__ void __launch_bounds__(256) stage_ref_kernel(StageArgs<T> a) {
    __shared__ T sh[32];
    if (a.ctl->done) return;                      // forecast horizon reached
    const int par = a.ctl->parity;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const bool act = i < a.nx && j < a.ny;
    T speed = T(0);
    Cell<T> C;
    C.land = true;
    if (act) load_cell<T, STAGE>(a, par, i, j, C);
    if (act && !C.land) {
        const T g = a.g, kappa = a.kappa, hik = a.half_inv_kappa;
        Cell<T> W2, W1, E1, E2, S2, S1, N1, N2;
        load_cell<T, STAGE>(a, par, i - 2, j, W2);
        load_cell<T, STAGE>(a, par, i - 1, j, W1);
        load_cell<T, STAGE>(a, par, i + 1, j, E1);
        load_cell<T, STAGE>(a, par, i + 2, j, E2);
        load_cell<T, STAGE>(a, par, i, j - 2, S2);
        load_cell<T, STAGE>(a, par, i, j - 1, S1);
        load_cell<T, STAGE>(a, par, i, j + 1, N1);
        load_cell<T, STAGE>(a, par, i, j + 2, N2);

        Face<T> cE, cW, cN, cS, L, R;
        T Fw[3], Fe[3], Gs[3], Gn[3];
        reconstruct<T, 0>(W1, C, E1, a.kx, a.tm, cE, cW);
        reconstruct<T, 1>(S1, C, N1, a.ky, a.tm, cN, cS);
        const T etaE = cE.eta, etaW = cW.eta, etaN = cN.eta, etaS = cS.eta;
        // west face
        R = cW; finish_face(R, g, kappa, hik);
        if (W1.land) L = mirror<T, 0>(R);
        else { Face<T> p, m; reconstruct<T, 0>(W2, W1, C, a.kx, a.tm, p, m); L = p; finish_face(L, g, kappa, hik); }
        cu_flux<T, 0>(L, R, C.HW, g, Fw);
        // east face
        L = cE; finish_face(L, g, kappa, hik);
        if (E1.land) R = mirror<T, 0>(L);
        else { Face<T> p, m; reconstruct<T, 0>(C, E1, E2, a.kx, a.tm, p, m); R = m; finish_face(R, g, kappa, hik); }
        cu_flux<T, 0>(L, R, C.HE, g, Fe);
        // south face
        R = cS; finish_face(R, g, kappa, hik);
        if (S1.land) L = mirror<T, 1>(R);
        else { Face<T> p, m; reconstruct<T, 1>(S2, S1, C, a.ky, a.tm, p, m); L = p; finish_face(L, g, kappa, hik); }
        cu_flux<T, 1>(L, R, C.HS, g, Gs);
        // north face
        L = cN; finish_face(L, g, kappa, hik);
        if (N1.land) R = mirror<T, 1>(L);
        else { Face<T> p, m; reconstruct<T, 1>(C, N1, N2, a.ky, a.tm, p, m); R = m; finish_face(R, g, kappa, hik); }
        cu_flux<T, 1>(L, R, C.HN, g, Gn);

        // M(Q) = -dF/dx - dG/dy + B + C + W (eq:sw_semidiscrete)
        T m0 = -(Fe[0] - Fw[0]) * a.inv_dx - (Gn[0] - Gs[0]) * a.inv_dy;
        T m1 = -(Fe[1] - Fw[1]) * a.inv_dx - (Gn[1] - Gs[1]) * a.inv_dy;
        T m2 = -(Fe[2] - Fw[2]) * a.inv_dx - (Gn[2] - Gs[2]) * a.inv_dy;
        m1 += g * T(0.5) * (etaE + etaW) * (C.HE - C.HW) * a.inv_dx;   // bed, eta form
        m2 += g * T(0.5) * (etaN + etaS) * (C.HN - C.HS) * a.inv_dy;
        T hue = C.ct * C.hu - C.st * C.hv;                               // Coriolis
        T hvn = C.st * C.hu + C.ct * C.hv;
        m1 += C.f * (C.ct * hvn - C.st * hue);
        m2 += C.f * (-C.st * hvn - C.ct * hue);
        T tx, ty;
        wind_at(a, i, j, STAGE - 1, T(a.clk.rho_ratio), tx, ty);
        m1 += tx;
        m2 += ty;
        T S = a.cd * sqrt(C.u * C.u + C.v * C.v) / fabs(C.hs);          // drag rate

        const T dt = T(a.ctl->dt);
        const long long s = (long long)j * a.pitch + i;
        if (STAGE == 1) {
            T den = T(1) / (T(1) + dt * S);
            a.d1[0][s] = dt * m0;
            a.d1[1][s] = (dt * m1 - dt * S * C.hu) * den;
            a.d1[2][s] = (dt * m2 - dt * S * C.hv) * den;
        } else {
            // Q^{n+1} - Q^n = (D1 + dt M(Q*) - dt S Q^n) / 2 / (1 + dt S / 2)
            T q0 = a.q[par][0][s], q1 = a.q[par][1][s], q2 = a.q[par][2][s];
            T D0 = a.d1[0][s], D1 = a.d1[1][s], D2 = a.d1[2][s];
            T den = T(1) / (T(1) + T(0.5) * dt * S);
            T de0 = T(0.5) * (D0 + dt * m0);
            T de1 = T(0.5) * (D1 + dt * m1 - dt * S * q1) * den;
            T de2 = T(0.5) * (D2 + dt * m2 - dt * S * q2) * den;
            T c0 = 0, c1 = 0, c2 = 0;
            if (KAHAN) {
                c0 = a.comp[0][s]; c1 = a.comp[1][s]; c2 = a.comp[2][s];
                kahan_add(q0, c0, de0);
                kahan_add(q1, c1, de1);
                kahan_add(q2, c2, de2);
            } else {
                q0 += de0; q1 += de1; q2 += de2;
            }
            // flow relaxation, eq:frs, nested edges in the order S, N, W, E
            for (int e = 0; e < 4; e++) {
                if (a.bc[e] != BC_NESTED) continue;
                int d = e == EDGE_S ? j : e == EDGE_N ? a.ny - 1 - j : e == EDGE_W ? i : a.nx - 1 - i;
                if (d >= a.frs_width) continue;
                int k = e >= EDGE_W ? j : i;
                T al = T(a.frs_alpha[d]);
                T x0 = bnd_value(a, e, 0, 0, k, 1), x1 = bnd_value(a, e, 0, 1, k, 1),
                  x2 = bnd_value(a, e, 0, 2, k, 1);
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
            if (!(isfinite(q0) && isfinite(q1) && isfinite(q2))) flag_error(a.ctl, j * a.nx + i);
            speed = cell_speed(a, q0, q1, q2, C.Hbar);
        }
    }
    if (STAGE == 2) {
        speed = block_max(speed, sh);
        if (threadIdx.x == 0 && threadIdx.y == 0) speed_atomic_max(a.ctl, speed);
    }
}

// Max CFL speed of the current state (used at creation and on set_clock).
template <typename T>
__global__ void __launch_bounds__(256) speed_kernel(StageArgs<T> a) {
    __shared__ T sh[32];
    const int par = a.ctl->parity;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    T speed = T(0);
    // the domain's own cells (all of them unless it is a window)
    if (i >= a.own_x0 && i < a.own_x1 && j >= a.own_y0 && j < a.own_y1) {
        const long long cp = a.cpitch;
        const T *H = a.H + (long long)j * cp + i;
        T c00 = H[0], c10 = H[1], c01 = H[cp], c11 = H[cp + 1];
        const T L = T(kLand);
        if (!((c00 == L) | (c10 == L) | (c01 == L) | (c11 == L))) {
            const long long s = (long long)j * a.pitch + i;
            speed = cell_speed(a, a.q[par][0][s], a.q[par][1][s], a.q[par][2][s],
                               T(0.25) * (c00 + c10 + c01 + c11));
        }
    }
    speed = block_max(speed, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) speed_atomic_max(a.ctl, speed);
}

// ---------------------------------------------------------------------------
// the clock: t, dt, forcing brackets (FP64), one thread per domain

template <typename T>
__global__ void clock_kernel(StepCtl *ctl, ClockParams clk, ForcingDev bnd, ForcingDev wind, int mode) {
    if (mode == 1 && ctl->done) return;
    double speed = sizeof(T) == 4 ? (double)__uint_as_float(ctl->speed32)
                                  : __longlong_as_double((long long)ctl->speed64);
    ctl->speed32 = 0u;
    ctl->speed64 = 0ull;
    clock_update(ctl, clk, bnd, wind, speed, mode);
}

// One clock evaluation for the sub-domains of a decomposed domain, from
// the largest of their CFL maxima (each FP32 sub-domain's stage 2 or speed
// pass left its own in speed32; the maximum is taken over the bit patterns
// of these non-negative floats, as the atomics of a whole domain take it):
// every clock advances with the same speed, so to the same t, dt and
// forcing brackets.
__global__ void split_clock_kernel(SplitClocks c, int mode) {
    __shared__ unsigned int bits;
    if (threadIdx.x == 0) {
        unsigned int m = 0u;
        for (int k = 0; k < c.n; k++) m = max(m, c.ctl[k]->speed32);
        bits = m;
    }
    __syncthreads();
    const int k = threadIdx.x;
    if (k >= c.n) return;
    StepCtl *ctl = c.ctl[k];
    if (mode == 1 && ctl->done) return;
    ctl->speed32 = 0u;
    ctl->speed64 = 0ull;
    clock_update(ctl, c.clk, c.bnd[k], c.wind[k], (double)__uint_as_float(bits), mode);
}

// The halo exchange of a decomposed domain: copy c of the table moves the
// cells of a box (whole-domain coordinates) from the sub-domain that owns
// them into another's window; what = 0: the current state (each
// sub-domain's buffer chosen by its device-side parity), 1: the stage-1
// increment.
__global__ void __launch_bounds__(256) halo_copy_kernel(HaloTable t, int what) {
    const HaloCopy c = t.copy[blockIdx.y];
    const SplitPlanes &D = t.dom[c.dst], &S = t.dom[c.src];
    const int w = c.x1 - c.x0, n = w * (c.y1 - c.y0);
    const int dp = what == 0 ? D.ctl->parity : 0, sp = what == 0 ? S.ctl->parity : 0;
    float *const *dst = what == 0 ? D.q[dp] : D.d1;
    const float *const *src = what == 0 ? S.q[sp] : S.d1;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int x = c.x0 + k % w, y = c.y0 + k / w;
        const long long so = (long long)(y - S.wy0) * S.pitch + (x - S.wx0);
        const long long dof = (long long)(y - D.wy0) * D.pitch + (x - D.wx0);
        for (int v = 0; v < 3; v++) dst[v][dof] = src[v][so];
    }
}

__global__ void set_clock_kernel(StepCtl *ctl, double t, double dt, long long step) {
    ctl->t = t;
    ctl->step = step;
    ctl->done = 0;
    if (dt > 0.0) ctl->dt = dt;
    ctl->speed32 = 0u;
    ctl->speed64 = 0ull;
    ctl->blocks_done = 0u;
}

__global__ void init_ctl_kernel(StepCtl *ctl, double t0) {
    StepCtl z = {};
    z.t = t0;
    z.err_cell = -1;
    *ctl = z;
}

// Copy one plane of the current state (buffer chosen by the device-side
// parity) into a dense nx*ny destination.
template <typename T>
__global__ void read_plane_kernel(const StepCtl *ctl, const T *q0, const T *q1, long long pitch,
                                  int nx, int ny, T *dst) {
    const T *src = ctl->parity ? q1 : q0;
    long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        long long j = k / nx, i = k - j * nx;
        dst[k] = src[j * pitch + i];
    }
}

__global__ void set_end_kernel(StepCtl *ctl, double t_end) {
    ctl->t_end = t_end;
    ctl->done = 0;
}

// ---------------------------------------------------------------------------
// FP64 diagnostics: deterministic two-pass block sums

template <typename T>
__global__ void __launch_bounds__(256) diag_partial_kernel(StageArgs<T> a, double *partials) {
    __shared__ double sh[2][8];
    const int par = a.ctl->parity;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    double m = 0.0, en = 0.0;
    if (i < a.nx && j < a.ny) {
        const long long cp = a.cpitch;
        const T *H = a.H + (long long)j * cp + i;
        T c00 = H[0], c10 = H[1], c01 = H[cp], c11 = H[cp + 1];
        const T L = T(kLand);
        if (!((c00 == L) | (c10 == L) | (c01 == L) | (c11 == L))) {
            const long long s = (long long)j * a.pitch + i;
            double e = (double)a.q[par][0][s], u = (double)a.q[par][1][s], v = (double)a.q[par][2][s];
            double Hb = 0.25 * ((double)c00 + (double)c10 + (double)c01 + (double)c11);
            double k = (double)a.kappa;
            double h = e + Hb;
            double mm = fmin(h * h / (2.0 * k) + 0.5 * k, k);
            double hs = fmax(fabs(h), mm);
            m = e;
            en = 0.5 * (u * u + v * v) / hs + 0.5 * (double)a.g * e * e;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        m += __shfl_xor_sync(0xffffffffu, m, o);
        en += __shfl_xor_sync(0xffffffffu, en, o);
    }
    int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if ((tid & 31) == 0) { sh[0][tid >> 5] = m; sh[1][tid >> 5] = en; }
    __syncthreads();
    if (tid == 0) {
        double sm = 0.0, se = 0.0;
        for (int w = 0; w < 8; w++) { sm += sh[0][w]; se += sh[1][w]; }
        int b = blockIdx.y * gridDim.x + blockIdx.x;
        partials[2 * b] = sm;
        partials[2 * b + 1] = se;
    }
}

__global__ void diag_final_kernel(const double *partials, int n, double area, double *out) {
    __shared__ double sh[2][32];
    double m = 0.0, e = 0.0;
    // fixed assignment of partials to lanes, fixed combination order
    for (int b = threadIdx.x; b < n; b += 32) { m += partials[2 * b]; e += partials[2 * b + 1]; }
    sh[0][threadIdx.x] = m;
    sh[1][threadIdx.x] = e;
    __syncwarp();
    if (threadIdx.x == 0) {
        double sm = 0.0, se = 0.0;
        for (int w = 0; w < 32; w++) { sm += sh[0][w]; se += sh[1][w]; }
        out[0] = sm * area;
        out[1] = se * area;
    }
}

// ---------------------------------------------------------------------------
// launchers

static dim3 ref_block() { return dim3(32, 8); }
static dim3 ref_grid(int nx, int ny) { return dim3((nx + 31) / 32, (ny + 7) / 8); }

int ref_step_parts() { return 3; }

const char *ref_part_name(int part) {
    static const char *names[3] = {"stage1", "stage2", "clock"};
    return part >= 0 && part < 3 ? names[part] : "";
}

// One launch of the reference step: 0 = stage 1, 1 = stage 2, 2 = clock.
template <typename T>
cudaError_t launch_step_ref_part(const StageArgs<T> &a, cudaStream_t st, int part, bool kahan) {
    dim3 b = ref_block(), g = ref_grid(a.nx, a.ny);
    if (part == 0) {
        stage_ref_kernel<T, 1, false><<<g, b, 0, st>>>(a);
    } else if (part == 1) {
        if (kahan) stage_ref_kernel<T, 2, true><<<g, b, 0, st>>>(a);
        else stage_ref_kernel<T, 2, false><<<g, b, 0, st>>>(a);
    } else {
        clock_kernel<T><<<1, 1, 0, st>>>(a.ctl, a.clk, a.bnd, a.wind, 1);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_clock(const StageArgs<T> &a, cudaStream_t st, double t, double dt,
                              long long step) {
    set_clock_kernel<<<1, 1, 0, st>>>(a.ctl, t, dt, step);
    if (dt > 0.0) {
        clock_kernel<T><<<1, 1, 0, st>>>(a.ctl, a.clk, a.bnd, a.wind, 2);
    } else {
        speed_kernel<T><<<ref_grid(a.nx, a.ny), ref_block(), 0, st>>>(a);
        clock_kernel<T><<<1, 1, 0, st>>>(a.ctl, a.clk, a.bnd, a.wind, 0);
    }
    return cudaGetLastError();
}

cudaError_t launch_speed(const StageArgs<float> &a, cudaStream_t st) {
    speed_kernel<float><<<ref_grid(a.nx, a.ny), ref_block(), 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_split_clock(const SplitClocks &c, int mode, cudaStream_t st) {
    split_clock_kernel<<<1, 32, 0, st>>>(c, mode);
    return cudaGetLastError();
}

cudaError_t launch_halo_copy(const HaloTable &t, int what, cudaStream_t st) {
    if (t.n_copies <= 0) return cudaSuccess;
    int most = 0;
    for (int k = 0; k < t.n_copies; k++)
        most = std::max(most, (t.copy[k].x1 - t.copy[k].x0) * (t.copy[k].y1 - t.copy[k].y0));
    const int blocks = std::min(64, std::max(1, (most + 255) / 256));
    halo_copy_kernel<<<dim3(blocks, t.n_copies), 256, 0, st>>>(t, what);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_refresh_brackets(const StageArgs<T> &a, cudaStream_t st) {
    clock_kernel<T><<<1, 1, 0, st>>>(a.ctl, a.clk, a.bnd, a.wind, 2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_read_plane(const StepCtl *ctl, const T *q0, const T *q1, long long pitch,
                              int nx, int ny, T *dst, cudaStream_t st) {
    long long n = (long long)nx * ny;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    read_plane_kernel<T><<<blocks, 256, 0, st>>>(ctl, q0, q1, pitch, nx, ny, dst);
    return cudaGetLastError();
}
template cudaError_t launch_read_plane<float>(const StepCtl *, const float *, const float *, long long, int, int, float *, cudaStream_t);
template cudaError_t launch_read_plane<double>(const StepCtl *, const double *, const double *, long long, int, int, double *, cudaStream_t);

cudaError_t launch_set_end(StepCtl *ctl, double t_end, cudaStream_t st) {
    set_end_kernel<<<1, 1, 0, st>>>(ctl, t_end);
    return cudaGetLastError();
}

cudaError_t launch_ctl_init(StepCtl *ctl, double t0, cudaStream_t st) {
    init_ctl_kernel<<<1, 1, 0, st>>>(ctl, t0);
    return cudaGetLastError();
}

int diag_blocks(int nx, int ny) {
    dim3 g = ref_grid(nx, ny);
    return (int)(g.x * g.y);
}

template <typename T>
cudaError_t launch_diagnostics(const StageArgs<T> &a, double *partials, double *out,
                               cudaStream_t st) {
    dim3 g = ref_grid(a.nx, a.ny);
    diag_partial_kernel<T><<<g, ref_block(), 0, st>>>(a, partials);
    diag_final_kernel<<<1, 32, 0, st>>>(partials, (int)(g.x * g.y), (double)a.dx * (double)a.dy, out);
    return cudaGetLastError();
}

template cudaError_t launch_step_ref_part<float>(const StageArgs<float> &, cudaStream_t, int, bool);
template cudaError_t launch_step_ref_part<double>(const StageArgs<double> &, cudaStream_t, int, bool);
template cudaError_t launch_init_clock<float>(const StageArgs<float> &, cudaStream_t, double, double, long long);
template cudaError_t launch_init_clock<double>(const StageArgs<double> &, cudaStream_t, double, double, long long);
template cudaError_t launch_refresh_brackets<float>(const StageArgs<float> &, cudaStream_t);
template cudaError_t launch_refresh_brackets<double>(const StageArgs<double> &, cudaStream_t);
template cudaError_t launch_diagnostics<float>(const StageArgs<float> &, double *, double *, cudaStream_t);
template cudaError_t launch_diagnostics<double>(const StageArgs<double> &, double *, double *, cudaStream_t);

}  // namespace swe
