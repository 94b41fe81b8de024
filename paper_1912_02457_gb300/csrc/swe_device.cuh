// swe_device.cuh -- per-cell arithmetic of the well-balanced central-upwind
// scheme (Brodtkorb & Holm, arXiv 1912.02457), shared by every stage kernel
// of libswe. Templated on the arithmetic type T (float or double).
#pragma once

#include "swe_internal.h"

namespace swe {

// Desingularised depth, eq:desing_ours (Section 3.2):
// h* = sign(h) max(|h|, min(h^2/(2 kappa) + kappa/2, kappa)), sign(0) = +1.
template <typename T>
__device__ __forceinline__ T desing(T h, T kappa, T half_inv_kappa) {
    T m = fmin(h * h * half_inv_kappa + T(0.5) * kappa, kappa);
    T r = fmax(fabs(h), m);
    return h < T(0) ? -r : r;
}

// Generalised minmod of (theta*backward, central, theta*forward): the
// smallest when all three are positive, the largest when all are negative,
// else zero. Written branch-free as max(0, min3) + min(0, max3), which gives
// exactly those values (one of the two terms is always an exact zero).
template <typename T>
__device__ __forceinline__ T minmod3(T a, T b, T c) {
    const T lo = fmin(a, fmin(b, c)), hi = fmax(a, fmax(b, c));
    return fmax(T(0), lo) + fmin(T(0), hi);
}

// One cell as seen by the stencil: state, bilinear bathymetry at the cell
// average and face midpoints, Coriolis parameter and north angle, and the
// derived primitives of the reconstruction.
template <typename T>
struct Cell {
    bool land;
    T eta, hu, hv;
    T Hbar, HE, HW, HN, HS;
    T f, ct, st;
    T hbar, hs, u, v;
    T fvx, fuy;        // f x.[v^n,-u^e] and -f y.[v^n,-u^e] (Section 3.7)
};

// Face state before (raw) and after desingularisation.
template <typename T>
struct Face {
    T h, eta, hu, hv, u, v, c;
};

// Cell averages and north-vector-projected Coriolis terms (Sections 3.1,
// 3.2 and 3.7): hbar = eta + Hbar, u = hu/h*, v = hv/h*,
// u^e = e.[u,v], v^n = n.[u,v] with e = [cos,-sin], n = [sin,cos];
// the x-reconstruction uses f x.[v^n,-u^e] (= f v), the y-reconstruction
// -f y.[v^n,-u^e] (= f u), with x = [cos, sin] and y = [-sin, cos].
template <typename T>
__device__ __forceinline__ void make_prim(Cell<T> &c, T kappa, T hik) {
    c.hbar = c.eta + c.Hbar;
    c.hs = desing(c.hbar, kappa, hik);
    T r = T(1) / c.hs;
    c.u = c.hu * r;
    c.v = c.hv * r;
    T ue = c.ct * c.u - c.st * c.v;
    T vn = c.st * c.u + c.ct * c.v;
    T xs = c.ct * vn - c.st * ue;
    T ys = -c.st * vn - c.ct * ue;
    c.fvx = c.f * xs;
    c.fuy = -c.f * ys;
}

// Reconstruction of the centre cell `c` along x (DIR 0) or y (DIR 1),
// Section 3.1 in its local form (eq:Kbackwards, eq:hE): with
// phi = (dx/2g) f v (x) or -(dy/2g) f u (y),
//   bw = (eta_c - eta_l) - (phi_l + phi_c), fw = (eta_r - eta_c) - (phi_c + phi_r),
//   s  = minmod(theta bw, (bw+fw)/2, theta fw),
//   eta+ = eta_c + s/2 + phi_c, eta- = eta_c - s/2 - phi_c.
// Land neighbours are the mirror of the centre cell (Section 3.4).
// Wet-dry (eq:KxE_adjust): a negative face is re-sloped to zero depth and
// the other face gets 2 hbar; a cell with hbar <= 0 is dry on both faces.
// Momentum faces: minmod-limited slopes of hu and hv.
template <typename T, int DIR>
__device__ __forceinline__ void reconstruct(const Cell<T> &l, const Cell<T> &c,
                                            const Cell<T> &r, T k, T tm,
                                            Face<T> &plus, Face<T> &minus) {
    const T sg = DIR == 0 ? T(1) : T(-1);
    T phc = sg * k * (DIR == 0 ? c.fvx : c.fuy);
    T el, ml1, ml2, phl, er, mr1, mr2, phr;
    if (l.land) {
        el = c.eta; phl = -phc;
        ml1 = DIR == 0 ? -c.hu : c.hu;
        ml2 = DIR == 0 ? c.hv : -c.hv;
    } else {
        el = l.eta; ml1 = l.hu; ml2 = l.hv;
        phl = sg * k * (DIR == 0 ? l.fvx : l.fuy);
    }
    if (r.land) {
        er = c.eta; phr = -phc;
        mr1 = DIR == 0 ? -c.hu : c.hu;
        mr2 = DIR == 0 ? c.hv : -c.hv;
    } else {
        er = r.eta; mr1 = r.hu; mr2 = r.hv;
        phr = sg * k * (DIR == 0 ? r.fvx : r.fuy);
    }
    T bw = (c.eta - el) - (phl + phc);
    T fw = (er - c.eta) - (phc + phr);
    T sK = minmod3(tm * bw, T(0.5) * (bw + fw), tm * fw);
    T b1 = c.hu - ml1, f1 = mr1 - c.hu;
    T s1 = minmod3(tm * b1, T(0.5) * (b1 + f1), tm * f1);
    T b2 = c.hv - ml2, f2 = mr2 - c.hv;
    T s2 = minmod3(tm * b2, T(0.5) * (b2 + f2), tm * f2);

    T Hp = DIR == 0 ? c.HE : c.HN;
    T Hm = DIR == 0 ? c.HW : c.HS;
    T etap = c.eta + T(0.5) * sK + phc;
    T etam = c.eta - T(0.5) * sK - phc;
    T hp = etap + Hp, hm = etam + Hm;
    if (c.hbar <= T(0)) {
        etap = -Hp; etam = -Hm; hp = T(0); hm = T(0);
    } else if (hp < T(0)) {
        etap = -Hp; hp = T(0);
        etam = T(2) * c.eta + Hp; hm = etam + Hm;
    } else if (hm < T(0)) {
        etam = -Hm; hm = T(0);
        etap = T(2) * c.eta + Hm; hp = etap + Hp;
    }
    plus.h = fmax(hp, T(0));  plus.eta = etap;
    minus.h = fmax(hm, T(0)); minus.eta = etam;
    plus.hu = c.hu + T(0.5) * s1;  minus.hu = c.hu - T(0.5) * s1;
    plus.hv = c.hv + T(0.5) * s2;  minus.hv = c.hv - T(0.5) * s2;
}

// Desingularised face velocities; face momenta reset to h u, h v so that a
// dry face carries none; gravity-wave speed sqrt(g h).
template <typename T>
__device__ __forceinline__ void finish_face(Face<T> &F, T g, T kappa, T hik) {
    T hs = desing(F.h, kappa, hik);
    T r = T(1) / hs;
    F.u = F.hu * r;
    F.v = F.hv * r;
    F.hu = F.h * F.u;
    F.hv = F.h * F.v;
    F.c = sqrt(g * F.h);
}

template <typename T, int DIR>
__device__ __forceinline__ Face<T> mirror(Face<T> F) {
    if (DIR == 0) { F.hu = -F.hu; F.u = -F.u; }
    else          { F.hv = -F.hv; F.v = -F.v; }
    return F;
}

// Central-upwind flux eqn:numerical_flux in the eta variables (pressure
// g eta (eta + 2 H_f)/2; the constant g H_f^2/2 of the h form cancels
// against the matching part of the bed term). out = flux along DIR.
template <typename T, int DIR>
__device__ __forceinline__ void cu_flux(const Face<T> &L, const Face<T> &R, T Hf, T g,
                                        T out[3], T *speed = nullptr) {
    T unL = DIR == 0 ? L.u : L.v, unR = DIR == 0 ? R.u : R.v;
    T ap = fmax(fmax(unL + L.c, unR + R.c), T(0));
    T am = fmin(fmin(unL - L.c, unR - R.c), T(0));
    if (speed) *speed = fmax(ap, -am);      // the face's largest one-sided speed
    T den = ap - am;
    T pL = T(0.5) * g * L.eta * (L.eta + T(2) * Hf);
    T pR = T(0.5) * g * R.eta * (R.eta + T(2) * Hf);
    // two dry faces at rest (a+ = a- = 0): the h-form flux is zero, i.e. the
    // eta-form normal momentum flux is the dry pressure -g H_f^2/2 (= pL = pR).
    // Selected at the end rather than branched to, so the flux has no
    // divergent path.
    const bool rest = den == T(0);
    T rd = T(1) / (rest ? T(1) : den);
    T FL0, FL1, FL2, FR0, FR1, FR2;
    if (DIR == 0) {
        FL0 = L.hu; FL1 = L.hu * L.u + pL; FL2 = L.hu * L.v;
        FR0 = R.hu; FR1 = R.hu * R.u + pR; FR2 = R.hu * R.v;
    } else {
        FL0 = L.hv; FL1 = L.hv * L.u; FL2 = L.hv * L.v + pL;
        FR0 = R.hv; FR1 = R.hv * R.u; FR2 = R.hv * R.v + pR;
    }
    T apam = ap * am;
    const T o0 = (ap * FL0 - am * FR0 + apam * (R.eta - L.eta)) * rd;
    const T o1 = (ap * FL1 - am * FR1 + apam * (R.hu - L.hu)) * rd;
    const T o2 = (ap * FL2 - am * FR2 + apam * (R.hv - L.hv)) * rd;
    out[0] = rest ? T(0) : o0;
    out[1] = rest ? (DIR == 0 ? pL : T(0)) : o1;
    out[2] = rest ? (DIR == 0 ? T(0) : pL) : o2;
}

// Large & Pond wind stress (Section 3.5).
template <typename T>
__device__ __forceinline__ void wind_stress(T wx, T wy, T rho_ratio, T &tx, T &ty) {
    T w = sqrt(wx * wx + wy * wy);
    T cdrag = (w < T(11)) ? T(1.2e-3) : (T(0.49) + T(0.065) * w) * T(1e-3);
    T k = rho_ratio * cdrag * w;
    tx = k * wx;
    ty = k * wy;
}

// Kahan-compensated s += x; the represented value is s - c.
template <typename T>
__device__ __forceinline__ void kahan_add(T &s, T &c, T x) {
    T y = x - c;
    T t = s + y;
    c = (t - s) - y;
    s = t;
}

// Texture-like sampling position of cell k of n on nb samples.
__device__ __forceinline__ void axis_pos(int k, int n, int nb, int &k0, int &k1, double &w) {
    double p = (k + 0.5) * (double)nb / (double)n - 0.5;
    p = fmin(fmax(p, 0.0), (double)(nb - 1));
    int a = (int)floor(p);
    if (a > nb - 1) a = nb - 1;
    k0 = a;
    k1 = a + 1 < nb ? a + 1 : nb - 1;
    w = p - a;
}

// External solution of edge e, ghost row r, variable v at along-edge cell k,
// interpolated along the edge and in time with the stage's frame bracket.
template <typename T>
__device__ T bnd_value(const StageArgs<T> &a, int e, int r, int v, int k, int stage) {
    const ForcingDev &F = a.bnd;
    int nb = e < 2 ? F.n1 : F.n2;
    // a window samples the edge at the whole domain's positions
    int n = e < 2 ? a.gnx : a.gny;
    k += e < 2 ? a.off_x : a.off_y;
    long long off = (e >= 1 ? 6LL * F.n1 : 0) + (e >= 2 ? 6LL * F.n1 : 0) + (e >= 3 ? 6LL * F.n2 : 0);
    int k0, k1;
    double w;
    axis_pos(k, n, nb, k0, k1, w);
    int fk = a.ctl->bk[stage];
    double s = a.ctl->bs[stage];
    long long fs = 12LL * (F.n1 + F.n2);
    const float *A = F.frames + (long long)fk * fs + off + (long long)(r * 3 + v) * nb;
    const float *B = F.n > 1 ? A + fs : A;
    double va = (1.0 - w) * A[k0] + w * A[k1];
    double vb = (1.0 - w) * B[k0] + w * B[k1];
    return T((1.0 - s) * va + s * vb);
}


__device__ __forceinline__ void axis_pos_f(int k, int n, int nb, int &k0, int &k1, float &w) {
    float p = (k + 0.5f) * (float)nb / (float)n - 0.5f;
    p = fminf(fmaxf(p, 0.0f), (float)(nb - 1));
    int q = (int)floorf(p);
    if (q > nb - 1) q = nb - 1;
    k0 = q;
    k1 = q + 1 < nb ? q + 1 : nb - 1;
    w = p - q;
}

// Wind stress at cell (i, j) at the stage time (Section 3.5): uniform
// frames use the stress the clock kernel computed; gridded frames are
// sampled bilinearly at the cell centre and lerped in time here, in the
// domain's precision.
// Bounds checks of the debug builds (-DSWE_DEBUG_BOUNDS): SWE_CHECK(a, off,
// n) is true when 0 <= off < n; otherwise it records SWE_ERR_BOUNDS (with
// the source line in err_cell) and the caller skips the access. In product
// builds it is the constant true and costs nothing.
#ifdef SWE_DEBUG_BOUNDS
static __device__ __noinline__ void flag_bounds(StepCtl *ctl, int line) {
    atomicExch(&ctl->err, (int)ERR_BOUNDS);
    atomicCAS(&ctl->err_cell, -1, line);
}
__device__ __forceinline__ bool in_bounds(StepCtl *ctl, long long off, long long n, int line) {
    if (off >= 0 && off < n) return true;
    flag_bounds(ctl, line);
    return false;
}
#define SWE_CHECK(a, off, n) ::swe::in_bounds((a).ctl, (long long)(off), (long long)(n), __LINE__)
#else
#define SWE_CHECK(a, off, n) true
#endif

template <typename T>
__device__ __forceinline__ void wind_at(const StageArgs<T> &a, int i, int j, int stage,
                                        T rho_ratio, T &tx, T &ty) {
    if (a.wind.n <= 0) { tx = T(0); ty = T(0); return; }
    if (a.clk.wind_uniform) {
        tx = T(a.ctl->tau[stage][0]);
        ty = T(a.ctl->tau[stage][1]);
        return;
    }
    const ForcingDev &F = a.wind;
    // sampling positions and weights in the domain's precision (an FP64
    // domain interpolates in FP64, like its nesting frames); a window
    // samples at the whole domain's positions
    int x0, x1, y0, y1;
    T wx, wy;
    if constexpr (sizeof(T) == sizeof(double)) {
        double px, py;
        axis_pos(i + a.off_x, a.gnx, F.n1, x0, x1, px);
        axis_pos(j + a.off_y, a.gny, F.n2, y0, y1, py);
        wx = T(px); wy = T(py);
    } else {
        float px, py;
        axis_pos_f(i + a.off_x, a.gnx, F.n1, x0, x1, px);
        axis_pos_f(j + a.off_y, a.gny, F.n2, y0, y1, py);
        wx = T(px); wy = T(py);
    }
    int fk = a.ctl->wk[stage];
    T s = T(a.ctl->ws[stage]);
    long long fs = 2LL * F.n1 * F.n2;
    const long long oa = fk * fs, ob = F.n > 1 ? oa + fs : oa;
    auto A = [&](long long o) { return T(SWE_CHECK(a, oa + o, a.n_wind) ? F.frames[oa + o] : 0.f); };
    auto B = [&](long long o) { return T(SWE_CHECK(a, ob + o, a.n_wind) ? F.frames[ob + o] : 0.f); };
    T W[2];
    for (int c = 0; c < 2; c++) {
        T a0 = (T(1) - wx) * A((y0 * F.n1 + x0) * 2 + c) + wx * A((y0 * F.n1 + x1) * 2 + c);
        T a1 = (T(1) - wx) * A((y1 * F.n1 + x0) * 2 + c) + wx * A((y1 * F.n1 + x1) * 2 + c);
        T b0 = (T(1) - wx) * B((y0 * F.n1 + x0) * 2 + c) + wx * B((y0 * F.n1 + x1) * 2 + c);
        T b1 = (T(1) - wx) * B((y1 * F.n1 + x0) * 2 + c) + wx * B((y1 * F.n1 + x1) * 2 + c);
        W[c] = (T(1) - s) * ((T(1) - wy) * a0 + wy * a1) + s * ((T(1) - wy) * b0 + wy * b1);
    }
    wind_stress<T>(W[0], W[1], rho_ratio, tx, ty);
}

// CFL wave speed of one cell, eq:cfl: max((|u| + sqrt(g hbar+))/dx,
// (|v| + sqrt(g hbar+))/dy) with desingularised cell velocities.
template <typename T>
__device__ __forceinline__ T cell_speed(const StageArgs<T> &a, T eta, T hu, T hv, T Hbar) {
    T hbar = eta + Hbar;
    T hs = desing(hbar, a.kappa, a.half_inv_kappa);
    T c = sqrt(a.g * fmax(hbar, T(0)));
    T r = T(1) / hs;
    T sx = (fabs(hu * r) + c) * a.inv_dx;
    T sy = (fabs(hv * r) + c) * a.inv_dy;
    return fmax(sx, sy);
}

__device__ inline void flag_error(StepCtl *ctl, int cell) {
    if (atomicCAS(&ctl->err_cell, -1, cell) == -1) {
        ctl->err = ERR_NUMERIC;
        ctl->err_step = ctl->step;
    }
}

// The clock (one thread per domain): t and dt in FP64; frame brackets with
// their weights in the precision of the domain.
// The FP32 clock arithmetic uses explicitly rounded operations: the clock
// runs in translation units built with different division, square-root and
// contraction settings, and must give the same bits in all of them (a
// resumed run replays the clock of an uninterrupted one).
// The frame weight: in FP64, or (fp32) as the FP32 quotient of the FP64
// offset and interval rounded once each; *sf holds it in FP32 either way.
__device__ __forceinline__ void frame_weight(double off, double len, bool fp32, double *s, float *sf) {
    if (fp32) {
        *sf = __fdiv_rn((float)off, (float)len);
        *s = (double)*sf;
    } else {
        *s = off / len;
        *sf = (float)*s;
    }
}

__device__ __forceinline__ void bracket(const double *times, int n, double t, int *k, double *s,
                                        float *sf, bool fp32) {
    *sf = 0.f;
    if (n <= 1) { *k = 0; *s = 0.0; return; }
    if (t <= times[0]) { *k = 0; *s = 0.0; return; }
    if (t >= times[n - 1]) { *k = n - 2; *s = 1.0; *sf = 1.f; return; }
    int lo = 0, hi = n - 1;            // times[lo] <= t < times[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (times[mid] <= t) lo = mid; else hi = mid;
    }
    *k = lo;
    frame_weight(t - times[lo], times[lo + 1] - times[lo], fp32, s, sf);
}

// The clock's inputs: its state of the previous step and the forcing values
// around the previous brackets. They do not change while a stage kernel
// runs (only the clock writes them, and it runs after every other block of
// the domain has finished), so a stage-2 block can load them before it
// knows whether it is the last one: the loads overlap its atomics.
struct ClockIn {
    double t, dt, t_end;
    long long step;
    int parity, done;
    int bhint, whint;          // bracket of the previous stage-2 time
    // the brackets and uniform wind stress at this step's stage-1 time as
    // the previous evaluation left them (see clock_advance)
    int ck_b, ck_w;
    double cs_b, cs_w, ctau[2];
    float cs_b_f, ctau_f[2];
    double bt0, bt1;           // boundary times[bhint], times[bhint + 1] (if a bracket)
    double wt0, wt1;           // wind times around whint (if a bracket)
    int wk_pre;                // wind frame whose uniform values follow (-1: none)
    float wa[2], wb[2];        // uniform wind frames wk_pre and the next one
};

__device__ __forceinline__ bool hint_ok(const ForcingDev &F, int hint) {
    return F.n > 1 && hint >= 0 && hint < F.n - 1;
}

// First level: the clock state (one round of independent loads). `mode` as
// in clock_advance: the values at the stage-1 time of the step it sets up
// are the previous stage-2 ones (modes 1, 4) or stage-1 ones (mode 3).
__device__ __forceinline__ void clock_load_state(const StepCtl *ctl, ClockIn &c, int mode) {
    c.t = ctl->t;
    c.dt = ctl->dt;
    c.t_end = ctl->t_end;
    c.step = ctl->step;
    c.parity = ctl->parity;
    c.done = ctl->done;
    c.bhint = ctl->bk[1];
    c.whint = ctl->wk[1];
    const int src = mode == 3 ? 0 : 1;
    c.ck_b = ctl->bk[src];
    c.ck_w = ctl->wk[src];
    c.cs_b = ctl->bs[src];
    c.cs_w = ctl->ws[src];
    c.ctau[0] = ctl->tau[src][0];
    c.ctau[1] = ctl->tau[src][1];
    c.cs_b_f = ctl->bs_f[src];
    c.ctau_f[0] = ctl->tau_f[src][0];
    c.ctau_f[1] = ctl->tau_f[src][1];
}

// Second level: the frame times around the previous brackets and the
// uniform wind frames there.
__device__ __forceinline__ void clock_load_forcing(const ClockParams &clk, const ForcingDev &bnd,
                                                   const ForcingDev &wind, ClockIn &c) {
    c.bt0 = c.bt1 = c.wt0 = c.wt1 = 0.0;
    if (hint_ok(bnd, c.bhint)) { c.bt0 = bnd.times[c.bhint]; c.bt1 = bnd.times[c.bhint + 1]; }
    const bool wh = hint_ok(wind, c.whint);
    if (wh) { c.wt0 = wind.times[c.whint]; c.wt1 = wind.times[c.whint + 1]; }
    c.wk_pre = -1;
    c.wa[0] = c.wa[1] = c.wb[0] = c.wb[1] = 0.f;
    if (wind.n > 0 && clk.wind_uniform && (wh || wind.n == 1)) {
        c.wk_pre = wh ? c.whint : 0;
        const float *A = wind.frames + 2LL * c.wk_pre;
        const float *B = wind.n > 1 ? A + 2 : A;
        c.wa[0] = A[0]; c.wa[1] = A[1]; c.wb[0] = B[0]; c.wb[1] = B[1];
    }
}

// bracket(), trying the interval `hint` (bounded by the preloaded t0, t1)
// first: the forcing time only moves forward, so the interval of the
// previous evaluation nearly always holds (the frame times are strictly
// increasing, so the interval is unique and both routes give the same k
// and s). With fp32 the weight is the FP32 quotient of the FP64 offset and
// interval (all an FP32 domain uses; the FP64 division is slow on GB300),
// and s holds it widened.
__device__ __forceinline__ void bracket_pre(const double *times, int n, double t, int hint, double t0,
                                            double t1, int *k, double *s, float *sf, bool fp32) {
    if (n > 1 && hint >= 0 && hint < n - 1 && t0 <= t && t < t1) {
        *k = hint;
        frame_weight(t - t0, t1 - t0, fp32, s, sf);
        return;
    }
    bracket(times, n, t, k, s, sf, fp32);
}

// The clock from its loaded inputs, on one thread; the state is written
// once at the end. Modes: 0 set up (dt from `speed`); 1 end of a step (t +=
// dt, the next dt from `speed`, the cell-average reading of eq:cfl); 2
// brackets only; 3 the face-speed reading of eq:cfl, before a step (dt from
// `speed` = the largest face speed over the cell size, no advance); 4 end of
// a step whose next dt comes from a mode-3 pass (t += dt only).
__device__ inline void clock_advance(StepCtl *ctl, const ClockParams &clk, const ForcingDev &bnd,
                                     const ForcingDev &wind, double speed, int mode, const ClockIn &c) {
    double t = c.t, dt = c.dt;
    long long step = c.step;
    int parity = c.parity, done = c.done;
    const double t_end = c.t_end;
    const bool fp32 = clk.fp32 != 0;
    bool bad_speed = false;
    if (mode == 1 || mode == 4) { t += dt; step += 1; parity ^= 1; }
    if (clk.dt_fixed > 0.0) {
        dt = clk.dt_fixed;
    } else if (mode == 0 || ((mode == 1 || mode == 3) && (clk.dt_every == 1 || step % clk.dt_every == 0))) {
        // eq:cfl, the FP64 quotient. (An FP32 quotient saves ~0.2 us of the
        // stage-2 tail but moved the 24 h static-coast run from 7.8e-6 to
        // 1.2e-4 m off the oracle: dt is kept exact.)
        if (speed > 0.0 && isfinite(speed)) dt = clk.courant * 0.25 / speed;
        else bad_speed = true;
    }
    // a forecast horizon: clip the last step to land on t_end, then stop
    if (t_end > 0.0) {
        if (t >= t_end * (1.0 - 1e-14)) done = 1;
        else if (t + dt > t_end) dt = t_end - t;
    }
    int bk[2], wk[2];
    double bs[2], ws[2], tau[2][2];
    float bs_f[2], ws_f[2], tau_f[2][2];
    // The stage-1 time of the step being set up is the time at which the
    // previous evaluation took its stage-2 values (modes 1, 4: the new t is
    // the same FP64 sum t + dt that evaluation formed) or its stage-1 values
    // (mode 3: t does not move). Brackets, weights and stress at a given
    // time are unique, so they are carried over, bit for bit, and only the
    // stage-2 time, which depends on the new dt, is evaluated here. (Forcing
    // replaced in between goes through mode 2, which evaluates both.)
    const bool carry = mode == 1 || mode == 3 || mode == 4;
    if (carry) {
        bk[0] = c.ck_b; bs[0] = c.cs_b; bs_f[0] = c.cs_b_f;
        wk[0] = c.ck_w; ws[0] = c.cs_w; ws_f[0] = 0.f;
        tau[0][0] = c.ctau[0]; tau[0][1] = c.ctau[1];
        tau_f[0][0] = c.ctau_f[0]; tau_f[0][1] = c.ctau_f[1];
    }
    for (int q = carry ? 1 : 0; q < 2; q++) {
        const double tt = t + (q ? dt : 0.0);
        bracket_pre(bnd.times, bnd.n, tt, c.bhint, c.bt0, c.bt1, &bk[q], &bs[q], &bs_f[q], fp32);
        bracket_pre(wind.times, wind.n, tt, c.whint, c.wt0, c.wt1, &wk[q], &ws[q], &ws_f[q], fp32);
        tau[q][0] = tau[q][1] = 0.0;
        tau_f[q][0] = tau_f[q][1] = 0.f;
        if (wind.n > 0 && clk.wind_uniform) {
            float a0 = c.wa[0], a1 = c.wa[1], b0 = c.wb[0], b1 = c.wb[1];
            if (wk[q] != c.wk_pre) {
                const float *A = wind.frames + 2LL * wk[q];
                const float *B = wind.n > 1 ? A + 2 : A;
                a0 = A[0]; a1 = A[1]; b0 = B[0]; b1 = B[1];
            }
            if (fp32) {
                // Large & Pond stress (Section 3.5) in the precision the FP32
                // stage kernels use it in
                const float w = ws_f[q], w1 = __fsub_rn(1.f, w);
                const float wx = __fadd_rn(__fmul_rn(w1, a0), __fmul_rn(w, b0));
                const float wy = __fadd_rn(__fmul_rn(w1, a1), __fmul_rn(w, b1));
                const float sp = __fsqrt_rn(__fadd_rn(__fmul_rn(wx, wx), __fmul_rn(wy, wy)));
                const float cdrag = sp < 11.f ? 1.2e-3f : __fmul_rn(__fadd_rn(0.49f, __fmul_rn(0.065f, sp)), 1e-3f);
                const float k = __fmul_rn(__fmul_rn((float)clk.rho_ratio, cdrag), sp);
                tau_f[q][0] = __fmul_rn(k, wx);
                tau_f[q][1] = __fmul_rn(k, wy);
                tau[q][0] = (double)tau_f[q][0];
                tau[q][1] = (double)tau_f[q][1];
            } else {
                double w = ws[q];
                double wx = (1.0 - w) * a0 + w * b0;
                double wy = (1.0 - w) * a1 + w * b1;
                double sp = sqrt(wx * wx + wy * wy);
                double cdrag = sp < 11.0 ? 1.2e-3 : (0.49 + 0.065 * sp) * 1e-3;
                double k = clk.rho_ratio * cdrag * sp;
                tau[q][0] = k * wx;
                tau[q][1] = k * wy;
                tau_f[q][0] = (float)tau[q][0];
                tau_f[q][1] = (float)tau[q][1];
            }
        }
    }
    ctl->last_speed = speed;
    ctl->t = t;
    ctl->dt = dt;
    ctl->step = step;
    ctl->parity = parity;
    ctl->done = done;
    // a non-finite or zero CFL maximum is an error unless one is recorded
    // already (the sticky code is read here only, on this rare path)
    if (bad_speed && ctl->err == ERR_NONE) { ctl->err = ERR_NUMERIC; ctl->err_step = step; }
    for (int q = 0; q < 2; q++) {
        ctl->bk[q] = bk[q]; ctl->bs[q] = bs[q];
        ctl->wk[q] = wk[q]; ctl->ws[q] = ws[q];
        ctl->tau[q][0] = tau[q][0]; ctl->tau[q][1] = tau[q][1];
        ctl->bs_f[q] = bs_f[q];
        ctl->tau_f[q][0] = tau_f[q][0];
        ctl->tau_f[q][1] = tau_f[q][1];
    }
}

__device__ inline void clock_update(StepCtl *ctl, const ClockParams &clk, const ForcingDev &bnd,
                                    const ForcingDev &wind, double speed, int mode) {
    ClockIn c;
    clock_load_state(ctl, c, mode);
    clock_load_forcing(clk, bnd, wind, c);
    clock_advance(ctl, clk, bnd, wind, speed, mode, c);
}


}  // namespace swe
