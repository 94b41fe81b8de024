/*
 * swe_oracle.c -- FP64 CPU oracle of the well-balanced central-upwind scheme
 * for the rotating shallow-water equations of Brodtkorb & Holm, "Real-World
 * Oceanographic Simulations on the GPU using a Two-Dimensional Finite-Volume
 * Scheme" (arXiv 1912.02457).
 *
 * TEST INFRASTRUCTURE. This file is the parity authority for the CUDA path
 * and nothing else: only the test suite, the package smoke check and the
 * benchmark's CPU-baseline / reference arm load it. It shares no code,
 * header, table or constant with the CUDA library, and the product path
 * never calls it.
 *
 * It is written to be checked against the paper by eye: plain loops over a
 * ghost-padded grid, every quantity in double precision, no fusion or
 * reordering beyond what the equations state, one function per step of
 * the method, each citing the passage it follows. Where the paper is
 * silent the reading taken is stated at the point of use.
 *
 * Grid conventions: cells (i, j), 0 <= i < nx, 0 <= j < ny, stored row-major
 * with x fastest. Bathymetry H lives at the (nx+1) x (ny+1) cell corners
 * (Section 2: "the bathymetry is defined at the cell intersections"). A
 * corner equal to the no-data value ORC_LAND is land (Section 3.4); a cell
 * is land when any of its corners is.
 *
 * Parity pins (tests/test_oracle_*.py): lake at rest with and without land
 * (bit-exact zero change for eta = 0), geostrophic balance, mass
 * conservation under walls, mirror/transpose/rotation equivariance,
 * wall == land ring, north-vector invariance, the local reformulation
 * against the recursive prefix-sum form, inertial oscillation against the
 * exact discrete propagator, friction and wind closed forms, the CFL
 * closed form, nesting with constant frames, and second-order
 * self-convergence on the peaks benchmark.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LAND ((double)FLT_MAX)

enum { ORC_S = 0, ORC_N = 1, ORC_W = 2, ORC_E = 3 };
enum { ORC_WALL = 0, ORC_NESTED = 1, ORC_PERIODIC = 2 };

typedef struct {
    int nx, ny;
    double dx, dy;
    double g;           /* gravitational acceleration */
    double theta_mm;    /* generalised-minmod parameter */
    double kappa;       /* desingularisation depth, eq:desing_ours */
    double cd;          /* quadratic bottom-drag coefficient */
    double rho_air, rho_water;
    double frs_d0;      /* flow-relaxation fall-off d0, eq:frs */
    int frs_width;      /* cells of the relaxation zone */
    int bc[4];          /* S, N, W, E: ORC_WALL, ORC_NESTED or ORC_PERIODIC
                           (periodic edges come in opposite pairs) */
    const double *H;    /* (ny+1)*(nx+1) corner depths */
    const double *f;    /* ny*nx Coriolis parameter */
    const double *theta;/* ny*nx north angle */
    /* wind: wind_n frames of (nfy, nfx, 2) at wind_t */
    int wind_n, wind_nfx, wind_nfy;
    const double *wind_t, *wind;
    /* nesting frames: bnd_n frames of 12*(nbx+nby) at bnd_t */
    int bnd_n, bnd_nbx, bnd_nby;
    const double *bnd_t, *bnd;
    /* 1: round the stored state to float32 after every stage (the storage
     * precision of the paper's GPU code, Section 3.2); arithmetic stays FP64.
     * Used to measure how sensitive a solution is to float32 storage. */
    int round_state_f32;
    /* Which speeds bound the time step in eq:cfl. 0 (the reading of the
     * scheme, and what the CUDA path implements): the cell-average
     * velocities and depths of the current state. 1: the one-sided local
     * speeds a+, a- of the faces of the current state's reconstruction, the
     * condition under which Kurganov & Petrova's wet-dry reconstruction keeps
     * every cell depth non-negative (used by the pins that show why the
     * cell-average reading does not). */
    int cfl_faces;
    /* A window of a larger domain (the domain decomposition of the stencil
     * of Section 3: sub-domains that exchange a two-cell halo per stage):
     * cell (0, 0) of this domain is cell (off_x, off_y) of a gnx x gny
     * domain, and the forcing (wind grid, nesting frames along an edge) is
     * sampled at the whole domain's positions. gnx = gny = 0: the domain is
     * whole (off_x = off_y = 0). */
    int off_x, off_y, gnx, gny;
} orc_domain;

/* the whole domain's extent along x and y */
static int whole_nx(const orc_domain *d) { return d->gnx > 0 ? d->gnx : d->nx; }
static int whole_ny(const orc_domain *d) { return d->gny > 0 ? d->gny : d->ny; }

/* ------------------------------------------------------------------------ */
/* small pieces of the method                                               */
/* ------------------------------------------------------------------------ */

/* Desingularised depth, Section 3.2, eq:desing_ours:
 * h* = sign(h) max(|h|, min(h^2/(2 kappa) + kappa/2, kappa)).
 * Reading: sign(0) = +1, so that h*(0) = kappa/2 and never zero. */
double orc_desing(double h, double kappa)
{
    double a = fabs(h);
    double m = fmin(h * h / (2.0 * kappa) + 0.5 * kappa, kappa);
    double r = fmax(a, m);
    return h < 0.0 ? -r : r;
}

/* Generalised minmod of three slopes (Section 3.1, the limiter applied to
 * the backward, central and forward differences). The caller passes the
 * outer arguments already scaled by theta. */
double orc_minmod(double a, double b, double c)
{
    if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
    if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
    return 0.0;
}

/* Large & Pond wind stress, Section 3.5:
 * tau = rho_a/rho_w C_D |W| W, C_D = 1e-3 * (1.2 if |W| < 11 else
 * 0.49 + 0.065 |W|). */
void orc_wind_stress(double wx, double wy, double rho_air, double rho_water,
                     double *tx, double *ty)
{
    double w = sqrt(wx * wx + wy * wy);
    double cdrag = (w < 11.0) ? 1.2e-3 : (0.49 + 0.065 * w) * 1e-3;
    double k = rho_air / rho_water * cdrag * w;
    *tx = k * wx;
    *ty = k * wy;
}

/* Linear interpolation weight in time, eq:windstress_interpol:
 * s = (t - t_a)/(t_b - t_a) for the frame pair bracketing t.
 * Reading: outside the frames the nearest frame is held. */
static void time_bracket(const double *times, int n, double t, int *k, double *s)
{
    if (n <= 1) { *k = 0; *s = 0.0; return; }
    if (t <= times[0]) { *k = 0; *s = 0.0; return; }
    if (t >= times[n - 1]) { *k = n - 2; *s = 1.0; return; }
    int a = 0;
    while (a + 1 < n - 1 && times[a + 1] <= t) a++;
    *k = a;
    *s = (t - times[a]) / (times[a + 1] - times[a]);
}

/* Texture-like linear interpolation along one axis: the value of a field
 * stored at nb samples, evaluated at the centre of cell k of n. */
static void axis_lerp(int k, int n, int nb, int *k0, int *k1, double *w)
{
    double p = (k + 0.5) * (double)nb / (double)n - 0.5;
    if (p < 0.0) p = 0.0;
    if (p > nb - 1) p = nb - 1;
    int a = (int)floor(p);
    if (a > nb - 1) a = nb - 1;
    *k0 = a;
    *k1 = (a + 1 < nb) ? a + 1 : nb - 1;
    *w = p - a;
}

/* Wind at the centre of cell (i, j) at time t: bilinear in space, linear in
 * time ("trilinearly interpolated wind stress", Section 3.5). Returns the
 * stress. */
static void wind_at(const orc_domain *d, int i, int j, double t,
                    double *tx, double *ty)
{
    *tx = 0.0; *ty = 0.0;
    if (d->wind_n <= 0) return;
    int k; double s;
    time_bracket(d->wind_t, d->wind_n, t, &k, &s);
    int x0, x1, y0, y1; double wx, wy;
    axis_lerp(i + d->off_x, whole_nx(d), d->wind_nfx, &x0, &x1, &wx);
    axis_lerp(j + d->off_y, whole_ny(d), d->wind_nfy, &y0, &y1, &wy);
    double W[2];
    for (int c = 0; c < 2; c++) {
        double v[2];
        for (int q = 0; q < 2; q++) {
            int fk = (d->wind_n == 1) ? 0 : k + q;
            const double *F = d->wind + (size_t)fk * d->wind_nfy * d->wind_nfx * 2;
#define WV(yy, xx) F[((size_t)(yy) * d->wind_nfx + (xx)) * 2 + c]
            double a = (1.0 - wx) * WV(y0, x0) + wx * WV(y0, x1);
            double b = (1.0 - wx) * WV(y1, x0) + wx * WV(y1, x1);
#undef WV
            v[q] = (1.0 - wy) * a + wy * b;
        }
        W[c] = (1.0 - s) * v[0] + s * v[1];
    }
    orc_wind_stress(W[0], W[1], d->rho_air, d->rho_water, tx, ty);
}

/* External (nesting) value of variable v (0 eta, 1 hu, 2 hv) in ghost row r
 * (0 touching the domain) of edge e at along-edge cell k and time t:
 * linear in time between the bracketing frames and linear along the edge
 * (Section 3.6: the boundary data is interpolated like the wind). A window
 * samples the edge at the whole domain's cell k + offset. */
static double bnd_value(const orc_domain *d, int e, int r, int v, int k, double t)
{
    int nbx = d->bnd_nbx, nby = d->bnd_nby;
    int nb = (e == ORC_S || e == ORC_N) ? nbx : nby;
    int n = (e == ORC_S || e == ORC_N) ? whole_nx(d) : whole_ny(d);
    k += (e == ORC_S || e == ORC_N) ? d->off_x : d->off_y;
    size_t off = 0;
    if (e >= ORC_N) off += (size_t)6 * nbx;
    if (e >= ORC_W) off += (size_t)6 * nbx;
    if (e >= ORC_E) off += (size_t)6 * nby;
    int fk; double s;
    time_bracket(d->bnd_t, d->bnd_n, t, &fk, &s);
    int k0, k1; double w;
    axis_lerp(k, n, nb, &k0, &k1, &w);
    double val[2];
    for (int q = 0; q < 2; q++) {
        int ff = (d->bnd_n == 1) ? 0 : fk + q;
        const double *B = d->bnd + (size_t)ff * 12 * (nbx + nby) + off
                        + (size_t)(r * 3 + v) * nb;
        val[q] = (1.0 - w) * B[k0] + w * B[k1];
    }
    return (1.0 - s) * val[0] + s * val[1];
}

/* ------------------------------------------------------------------------ */
/* the ghost-padded grid                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nx, ny;
    int px;          /* padded cells per row: nx + 4, cells i in [-2, nx+1] */
    int kx;          /* padded corners per row: nx + 5, corners in [-2, nx+2] */
    double *Hc;      /* padded corners */
    double *f, *ct, *st;
    unsigned char *land;
    double *HE, *HW, *HN, *HS, *Hbar;
} statics;

#define CI(S, i, j) ((size_t)((j) + 2) * (S)->px + (size_t)((i) + 2))
#define KI(S, i, j) ((size_t)((j) + 2) * (S)->kx + (size_t)((i) + 2))

/* Corner reflection about the boundary corner lines (reading: the
 * bathymetry continues evenly into the ghost region). Reflected again
 * while outside, so that a domain one cell wide stays defined. */
static int refl(int i, int n)
{
    while (i < 0 || i > n) i = i < 0 ? -i : 2 * n - i;
    return i;
}

/* Periodic boundaries (Section 3.3 names them beside walls): the padded
 * corner i is the periodic image i mod n of the input corner line (the input's
 * last corner line repeats its first), and a ghost cell is the periodic image
 * of an interior cell with all its statics and state. */
static int corner_src(int i, int n, int periodic)
{
    if (!periodic) return refl(i, n);
    while (i < 0) i += n;
    while (i > n) i -= n;
    return i;
}

static int wrap(int i, int n)
{
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}

static void statics_free(statics *S)
{
    free(S->Hc); free(S->f); free(S->ct); free(S->st); free(S->land);
    free(S->HE); free(S->HW); free(S->HN); free(S->HS); free(S->Hbar);
}

/* Mirror source cell of ghost cell (i, j) and the edge it belongs to, or -1
 * when (i, j) is interior or a ghost-ghost corner (unused by the plus-shaped
 * stencil). The first ghost row mirrors the first interior row; the second
 * mirrors the padded cell one further in, which is itself a ghost of the
 * opposite edge when the domain is a single cell wide (so ghosts are filled
 * row 1 on every edge before row 2). */
static int ghost_source(int nx, int ny, int i, int j, int *si, int *sj, int *row)
{
    int gx = (i < 0) || (i >= nx), gy = (j < 0) || (j >= ny);
    if (gx && gy) return -2;
    if (!gx && !gy) return -1;
    if (i < 0)   { *si = -i - 1;         *sj = j; *row = -i - 1;   return ORC_W; }
    if (i >= nx) { *si = 2 * nx - 1 - i; *sj = j; *row = i - nx;   return ORC_E; }
    if (j < 0)   { *si = i; *sj = -j - 1;         *row = -j - 1;   return ORC_S; }
    *si = i; *sj = 2 * ny - 1 - j; *row = j - ny; return ORC_N;
}

static int statics_build(const orc_domain *d, statics *S)
{
    int nx = d->nx, ny = d->ny;
    S->nx = nx; S->ny = ny; S->px = nx + 4; S->kx = nx + 5;
    size_t nc = (size_t)(nx + 4) * (ny + 4), nk = (size_t)(nx + 5) * (ny + 5);
    S->Hc = malloc(nk * sizeof(double));
    S->f = malloc(nc * sizeof(double));
    S->ct = malloc(nc * sizeof(double));
    S->st = malloc(nc * sizeof(double));
    S->land = malloc(nc);
    S->HE = malloc(nc * sizeof(double)); S->HW = malloc(nc * sizeof(double));
    S->HN = malloc(nc * sizeof(double)); S->HS = malloc(nc * sizeof(double));
    S->Hbar = malloc(nc * sizeof(double));
    if (!S->Hc || !S->f || !S->ct || !S->st || !S->land || !S->HE || !S->HW ||
        !S->HN || !S->HS || !S->Hbar) { statics_free(S); return -1; }

    const int px = d->bc[ORC_W] == ORC_PERIODIC, py = d->bc[ORC_S] == ORC_PERIODIC;
    if (px != (d->bc[ORC_E] == ORC_PERIODIC) || py != (d->bc[ORC_N] == ORC_PERIODIC)) {
        statics_free(S);
        return -1;                              /* a periodic edge needs its opposite */
    }
    for (int j = -2; j <= ny + 2; j++)
        for (int i = -2; i <= nx + 2; i++)
            S->Hc[KI(S, i, j)] = d->H[(size_t)corner_src(j, ny, py) * (nx + 1) + corner_src(i, nx, px)];

    for (int j = -2; j <= ny + 1; j++)
        for (int i = -2; i <= nx + 1; i++) {
            size_t c = CI(S, i, j);
            double c00 = S->Hc[KI(S, i, j)], c10 = S->Hc[KI(S, i + 1, j)];
            double c01 = S->Hc[KI(S, i, j + 1)], c11 = S->Hc[KI(S, i + 1, j + 1)];
            int L = (c00 == ORC_LAND) || (c10 == ORC_LAND) ||
                    (c01 == ORC_LAND) || (c11 == ORC_LAND);
            S->land[c] = (unsigned char)L;
            /* Bilinear bathymetry (Sections 2 and 3.9): at a face midpoint the
             * surface is the mean of the face's two corners, and its cell
             * average is the mean of the four corners. */
            if (!L) {
                S->HE[c] = 0.5 * (c10 + c11);
                S->HW[c] = 0.5 * (c00 + c01);
                S->HN[c] = 0.5 * (c01 + c11);
                S->HS[c] = 0.5 * (c00 + c10);
                S->Hbar[c] = 0.25 * (c00 + c10 + c01 + c11);
            } else {
                S->HE[c] = S->HW[c] = S->HN[c] = S->HS[c] = S->Hbar[c] = NAN;
            }
            int si, sj, row;
            int e = ghost_source(nx, ny, i, j, &si, &sj, &row);
            if (e == -1) {
                S->f[c] = d->f[(size_t)j * nx + i];
                S->ct[c] = d->theta[(size_t)j * nx + i];   /* angle for now */
            } else {
                S->f[c] = NAN; S->ct[c] = NAN;
            }
        }
    /* ghost f and angle, first ghost row of every edge, then the second */
    for (int ring = 0; ring < 2; ring++)
        for (int j = -2; j <= ny + 1; j++)
            for (int i = -2; i <= nx + 1; i++) {
                int si, sj, row;
                int e = ghost_source(nx, ny, i, j, &si, &sj, &row);
                if (e < 0 || row != ring) continue;
                size_t c = CI(S, i, j), s = CI(S, si, sj);
                if (d->bc[e] == ORC_PERIODIC) s = CI(S, wrap(i, nx), wrap(j, ny));
                /* Section 3.3: at a wall the Coriolis parameter is odd,
                 * f(-x) = -f(x), so that K_x = 0 across the wall. Nested
                 * edges continue f evenly (reading); a periodic ghost is its
                 * periodic image. */
                S->f[c] = d->bc[e] == ORC_WALL ? -S->f[s] : S->f[s];
                S->ct[c] = S->ct[s];
            }
    for (size_t c = 0; c < (size_t)(nx + 4) * (ny + 4); c++) {
        double th = S->ct[c];
        S->ct[c] = cos(th);
        S->st[c] = sin(th);
    }
    return 0;
}

/* Ghost cells of the state at time t (Sections 3.3 and 3.6): walls mirror
 * the first two interior cells (eta even, normal momentum odd, tangential
 * momentum even, eq:tradWallBCx); nested edges take the external solution
 * interpolated in time and along the edge; periodic edges take the periodic
 * image. */
static void fill_ghosts(const orc_domain *d, const statics *S,
                        double *eta, double *hu, double *hv, double t)
{
    int nx = d->nx, ny = d->ny;
    for (int ring = 0; ring < 2; ring++)
    for (int j = -2; j <= ny + 1; j++)
        for (int i = -2; i <= nx + 1; i++) {
            int si, sj, row;
            int e = ghost_source(nx, ny, i, j, &si, &sj, &row);
            size_t c = CI(S, i, j);
            if (e == -1) continue;
            if (e == -2) { eta[c] = hu[c] = hv[c] = NAN; continue; }
            if (row != ring) continue;
            size_t s = CI(S, si, sj);
            if (d->bc[e] == ORC_PERIODIC) {
                s = CI(S, wrap(i, nx), wrap(j, ny));
                eta[c] = eta[s]; hu[c] = hu[s]; hv[c] = hv[s];
            } else if (d->bc[e] == ORC_WALL) {
                eta[c] = eta[s];
                if (e == ORC_W || e == ORC_E) { hu[c] = -hu[s]; hv[c] = hv[s]; }
                else                          { hu[c] = hu[s];  hv[c] = -hv[s]; }
            } else {
                int k = (e == ORC_W || e == ORC_E) ? j : i;
                eta[c] = bnd_value(d, e, row, 0, k, t);
                hu[c] = bnd_value(d, e, row, 1, k, t);
                hv[c] = bnd_value(d, e, row, 2, k, t);
            }
        }
}

/* ------------------------------------------------------------------------ */
/* one evaluation of the right-hand side M(Q) and friction rate S(Q)        */
/* ------------------------------------------------------------------------ */

typedef struct { double h, eta, hu, hv; } raw_face;
typedef struct { double h, eta, hu, hv, u, v, c; } face;

/* Face velocities with the desingularised depth (eq:desing_ours applied at
 * the face); the face momenta are reset to h u and h v so that a dry face
 * carries none (reading, after Kurganov & Petrova). */
static face finish_face(raw_face r, double g, double kappa)
{
    face F;
    double hs = orc_desing(r.h, kappa);
    F.h = r.h;
    F.eta = r.eta;
    F.u = r.hu / hs;
    F.v = r.hv / hs;
    F.hu = r.h * F.u;
    F.hv = r.h * F.v;
    F.c = sqrt(g * r.h);
    return F;
}

/* Central-upwind flux, eqn:numerical_flux, in the eta variables:
 * the pressure is g eta (eta + 2 H_f)/2, i.e. g h^2/2 without the constant
 * g H_f^2/2 that the central-upwind combination returns unchanged.
 * dir 0: x-face (F), dir 1: y-face (G). */
static void cu_flux(face L, face R, double Hf, double g, int dir, double out[3],
                    double *speed)
{
    double unL = dir == 0 ? L.u : L.v, unR = dir == 0 ? R.u : R.v;
    double ap = fmax(fmax(unL + L.c, unR + R.c), 0.0);
    double am = fmin(fmin(unL - L.c, unR - R.c), 0.0);
    *speed = fmax(ap, -am);
    double pL = 0.5 * g * L.eta * (L.eta + 2.0 * Hf);
    double pR = 0.5 * g * R.eta * (R.eta + 2.0 * Hf);
    if (ap - am == 0.0) {
        /* a+ = a- = 0 only between two dry faces at rest; there the h-form
         * flux is zero, which in eta variables is the pressure
         * -g H_f^2 / 2 (= pL = pR) in the normal momentum. */
        out[0] = 0.0;
        out[1] = dir == 0 ? pL : 0.0;
        out[2] = dir == 0 ? 0.0 : pL;
        return;
    }
    double FL[3], FR[3];
    if (dir == 0) {
        FL[0] = L.hu; FL[1] = L.hu * L.u + pL; FL[2] = L.hu * L.v;
        FR[0] = R.hu; FR[1] = R.hu * R.u + pR; FR[2] = R.hu * R.v;
    } else {
        FL[0] = L.hv; FL[1] = L.hv * L.u; FL[2] = L.hv * L.v + pL;
        FR[0] = R.hv; FR[1] = R.hv * R.u; FR[2] = R.hv * R.v + pR;
    }
    double QL[3] = { L.eta, L.hu, L.hv }, QR[3] = { R.eta, R.hu, R.hv };
    for (int k = 0; k < 3; k++)
        out[k] = (ap * FL[k] - am * FR[k]) / (ap - am)
               + ap * am / (ap - am) * (QR[k] - QL[k]);
}

/* Mirror of a face state across a wall or land face: normal momentum and
 * velocity flip sign (eq:tradWallBCx; Section 3.4 uses the same wall for
 * the land mask). */
static face mirror_face(face F, int dir)
{
    if (dir == 0) { F.hu = -F.hu; F.u = -F.u; }
    else          { F.hv = -F.hv; F.v = -F.v; }
    return F;
}

/* Per-cell values needed by the reconstruction: the cell average depth
 * hbar = eta + Hbar, the desingularised velocities, and the Coriolis terms
 * of the potential energies projected through the local north vector
 * (Section 3.7): fvx = f x.[v^n, -u^e] for K and fuy = -f y.[v^n, -u^e]
 * for L (both reduce to f v and f u). */
typedef struct { double hbar, hs, u, v, fvx, fuy; } prim;

static prim make_prim(const statics *S, size_t c, double eta, double hu,
                      double hv, double kappa)
{
    prim p;
    p.hbar = eta + S->Hbar[c];
    p.hs = orc_desing(p.hbar, kappa);
    p.u = hu / p.hs;
    p.v = hv / p.hs;
    double ct = S->ct[c], st = S->st[c];
    double ue = ct * p.u - st * p.v;   /* e = [cos, -sin] */
    double vn = st * p.u + ct * p.v;   /* n = [sin,  cos] */
    double xs = ct * vn + st * (-ue);  /* x = [cos, sin]  */
    double ys = -st * vn + ct * (-ue); /* y = [-sin, cos] */
    p.fvx = S->f[c] * xs;
    p.fuy = -S->f[c] * ys;
    return p;
}

/* Reconstruction of one cell along x (dir 0) or y (dir 1), Section 3.1.
 *
 * The limited slope of K (resp. L) uses the local differences of
 * eq:Kbackwards: with phi = dx/(2g) f v,
 *   backward  = (eta_i - eta_{i-1}) - (phi_{i-1} + phi_i)
 *   forward   = (eta_{i+1} - eta_i) - (phi_i + phi_{i+1})
 *   central   = (backward + forward)/2,
 * and sK = minmod(theta*backward, central, theta*forward) = dx K_x / g.
 * The face values follow eq:hE: h^E = eta + H_E + sK/2 + phi and
 * h^W = eta + H_W - sK/2 - phi. Along y the same holds with L = g(eta + U):
 * psi = dy/(2g) f u enters with the opposite sign.
 *
 * A land neighbour is replaced by the mirror of this cell (wall following
 * the land mask, Section 3.4), giving zero K-slope across the coast.
 *
 * Wet-dry (Section 3.4, eq:KxE_adjust): if h^E < 0 the slope is re-set so
 * that h^E = 0, which gives h^W = 2 hbar (because H_E + H_W = 2 Hbar);
 * likewise if h^W < 0. Reading: E is tested before W, and a cell with
 * hbar <= 0 gets dry faces on both sides.
 *
 * Momentum faces use minmod-limited slopes of hu and hv (reading: the
 * scheme reconstructs h, hu and hv). */
static void reconstruct(const orc_domain *d, const statics *S,
                        const double *eta, const double *hu, const double *hv,
                        const prim *P, int i, int j, int dir,
                        raw_face *plus, raw_face *minus)
{
    double tm = d->theta_mm;
    size_t c = CI(S, i, j);
    size_t cl = dir == 0 ? CI(S, i - 1, j) : CI(S, i, j - 1);
    size_t cr = dir == 0 ? CI(S, i + 1, j) : CI(S, i, j + 1);
    double dl = dir == 0 ? d->dx : d->dy;
    double k = dl / (2.0 * d->g);

    /* phi: the Coriolis-primitive increment of this direction, signed so
     * that the face value is eta + sK/2 + phi on the plus side. */
    double sgn = dir == 0 ? 1.0 : -1.0;
    double phic = sgn * k * (dir == 0 ? P[c].fvx : P[c].fuy);

    double e[3], m1[3], m2[3], ph[3];
    size_t idx[3] = { cl, c, cr };
    for (int q = 0; q < 3; q++) {
        size_t n = idx[q];
        if (q != 1 && S->land[n]) {
            /* mirror of this cell across the land face */
            e[q] = eta[c];
            m1[q] = dir == 0 ? -hu[c] : hu[c];
            m2[q] = dir == 0 ? hv[c] : -hv[c];
            ph[q] = -phic;
        } else {
            e[q] = eta[n];
            m1[q] = hu[n];
            m2[q] = hv[n];
            ph[q] = sgn * k * (dir == 0 ? P[n].fvx : P[n].fuy);
        }
    }
    double bw = (e[1] - e[0]) - (ph[0] + ph[1]);
    double fw = (e[2] - e[1]) - (ph[1] + ph[2]);
    double sK = orc_minmod(tm * bw, 0.5 * (bw + fw), tm * fw);

    double b1 = m1[1] - m1[0], f1 = m1[2] - m1[1];
    double s1 = orc_minmod(tm * b1, 0.5 * (b1 + f1), tm * f1);
    double b2 = m2[1] - m2[0], f2 = m2[2] - m2[1];
    double s2 = orc_minmod(tm * b2, 0.5 * (b2 + f2), tm * f2);

    double Hp = dir == 0 ? S->HE[c] : S->HN[c];
    double Hm = dir == 0 ? S->HW[c] : S->HS[c];
    double etap = e[1] + 0.5 * sK + phic;
    double etam = e[1] - 0.5 * sK - phic;
    double hp = etap + Hp, hm = etam + Hm;
    double hbar = P[c].hbar;
    if (hbar <= 0.0) {
        etap = -Hp; etam = -Hm; hp = 0.0; hm = 0.0;
    } else if (hp < 0.0) {
        etap = -Hp; hp = 0.0;
        etam = 2.0 * e[1] + Hp; hm = etam + Hm;
    } else if (hm < 0.0) {
        etam = -Hm; hm = 0.0;
        etap = 2.0 * e[1] + Hm; hp = etap + Hp;
    }
    if (hp < 0.0) hp = 0.0;
    if (hm < 0.0) hm = 0.0;
    plus->h = hp; plus->eta = etap;
    minus->h = hm; minus->eta = etam;
    plus->hu = hu[c] + 0.5 * s1;
    minus->hu = hu[c] - 0.5 * s1;
    plus->hv = hv[c] + 0.5 * s2;
    minus->hv = hv[c] - 0.5 * s2;
}

/* Work arrays of one right-hand-side evaluation, allocated once per run. */
typedef struct {
    double *eta, *hu, *hv;          /* padded state */
    prim *P;
    double *Fx, *Gy;                /* face fluxes */
    raw_face *xp, *xm, *yp, *ym;    /* reconstructed faces */
} work;

static void work_free(work *W)
{
    free(W->eta); free(W->hu); free(W->hv); free(W->P); free(W->Fx); free(W->Gy);
    free(W->xp); free(W->xm); free(W->yp); free(W->ym);
    memset(W, 0, sizeof(*W));
}

static int work_alloc(const statics *S, work *W)
{
    int nx = S->nx, ny = S->ny;
    size_t nc = (size_t)S->px * (ny + 4);
    memset(W, 0, sizeof(*W));
    W->eta = malloc(nc * sizeof(double));
    W->hu = malloc(nc * sizeof(double));
    W->hv = malloc(nc * sizeof(double));
    W->P = malloc(nc * sizeof(prim));
    W->Fx = malloc(3 * (size_t)(nx + 1) * ny * sizeof(double));
    W->Gy = malloc(3 * (size_t)nx * (ny + 1) * sizeof(double));
    W->xp = malloc(nc * sizeof(raw_face)); W->xm = malloc(nc * sizeof(raw_face));
    W->yp = malloc(nc * sizeof(raw_face)); W->ym = malloc(nc * sizeof(raw_face));
    if (!W->eta || !W->hu || !W->hv || !W->P || !W->Fx || !W->Gy ||
        !W->xp || !W->xm || !W->yp || !W->ym) { work_free(W); return -1; }
    return 0;
}

/* M(Q) and S(Q) over the interior at time t: eq:sw_semidiscrete with the
 * Kurganov-Levy bed term in eta form, the north-vector Coriolis term of
 * Section 3.7, the wind stress of Section 3.5 and the friction rate of
 * the semi-implicit update (reading: S = C_d |u| / |h*|, the quadratic
 * drag -C_d u|u| of eq:swe with a dimensionless coefficient).
 * eta/hu/hv are nx*ny interior arrays; M is 3 planes of nx*ny. *ax, *ay
 * receive the largest one-sided local speed max(a+, -a-) over the x- and
 * y-faces that carry a flux. */
static void rhs(const orc_domain *d, const statics *S, work *W,
                const double *eta_in, const double *hu_in, const double *hv_in,
                double t, double *M, double *Sf, double *ax, double *ay)
{
    int nx = d->nx, ny = d->ny;
    double *eta = W->eta, *hu = W->hu, *hv = W->hv;
    prim *P = W->P;
    double *Fx = W->Fx, *Gy = W->Gy;
    raw_face *xp = W->xp, *xm = W->xm, *yp = W->yp, *ym = W->ym;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t c = CI(S, i, j), s = (size_t)j * nx + i;
            eta[c] = eta_in[s]; hu[c] = hu_in[s]; hv[c] = hv_in[s];
        }
    fill_ghosts(d, S, eta, hu, hv, t);

    /* primitives on the plus-shaped padded region */
#pragma omp parallel for schedule(static)
    for (int j = -2; j <= ny + 1; j++)
        for (int i = -2; i <= nx + 1; i++) {
            int gx = (i < 0) || (i >= nx), gy = (j < 0) || (j >= ny);
            size_t c = CI(S, i, j);
            if ((gx && gy) || S->land[c]) continue;
            P[c] = make_prim(S, c, eta[c], hu[c], hv[c], d->kappa);
        }

    /* x-reconstructions for cells -1..nx of each row, y for rows -1..ny */
#pragma omp parallel for schedule(static)
    for (int j = -1; j <= ny; j++)
        for (int i = -1; i <= nx; i++) {
            int inx = (i >= 0 && i < nx), iny = (j >= 0 && j < ny);
            size_t c = CI(S, i, j);
            if (S->land[c]) continue;
            if (iny) reconstruct(d, S, eta, hu, hv, P, i, j, 0, &xp[c], &xm[c]);
            if (inx) reconstruct(d, S, eta, hu, hv, P, i, j, 1, &yp[c], &ym[c]);
        }

    /* fluxes across x-faces i+1/2, i = -1..nx-1 */
    double sx = 0.0, sy = 0.0;
#pragma omp parallel for schedule(static) reduction(max: sx)
    for (int j = 0; j < ny; j++)
        for (int i = -1; i < nx; i++) {
            size_t a = CI(S, i, j), b = CI(S, i + 1, j);
            double *out = Fx + 3 * ((size_t)j * (nx + 1) + (i + 1));
            if (S->land[a] && S->land[b]) { out[0] = out[1] = out[2] = 0.0; continue; }
            double Hf = 0.5 * (S->Hc[KI(S, i + 1, j)] + S->Hc[KI(S, i + 1, j + 1)]);
            face L, R;
            if (!S->land[a]) L = finish_face(xp[a], d->g, d->kappa);
            if (!S->land[b]) R = finish_face(xm[b], d->g, d->kappa);
            if (S->land[a]) L = mirror_face(R, 0);
            if (S->land[b]) R = mirror_face(L, 0);
            double sp;
            cu_flux(L, R, Hf, d->g, 0, out, &sp);
            sx = fmax(sx, sp);
        }
#pragma omp parallel for schedule(static) reduction(max: sy)
    for (int j = -1; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t a = CI(S, i, j), b = CI(S, i, j + 1);
            double *out = Gy + 3 * ((size_t)(j + 1) * nx + i);
            if (S->land[a] && S->land[b]) { out[0] = out[1] = out[2] = 0.0; continue; }
            double Hf = 0.5 * (S->Hc[KI(S, i, j + 1)] + S->Hc[KI(S, i + 1, j + 1)]);
            face L, R;
            if (!S->land[a]) L = finish_face(yp[a], d->g, d->kappa);
            if (!S->land[b]) R = finish_face(ym[b], d->g, d->kappa);
            if (S->land[a]) L = mirror_face(R, 1);
            if (S->land[b]) R = mirror_face(L, 1);
            double sp;
            cu_flux(L, R, Hf, d->g, 1, out, &sp);
            sy = fmax(sy, sp);
        }
    *ax = sx;
    *ay = sy;

    /* assemble M = -dF/dx - dG/dy + B + C + W, and S */
    size_t np = (size_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t c = CI(S, i, j), s = (size_t)j * nx + i;
            if (S->land[c]) { M[s] = M[np + s] = M[2 * np + s] = 0.0; Sf[s] = 0.0; continue; }
            const double *fe = Fx + 3 * ((size_t)j * (nx + 1) + i + 1);
            const double *fw = Fx + 3 * ((size_t)j * (nx + 1) + i);
            const double *gn = Gy + 3 * ((size_t)(j + 1) * nx + i);
            const double *gs = Gy + 3 * ((size_t)j * nx + i);
            double m[3];
            for (int k = 0; k < 3; k++)
                m[k] = -(fe[k] - fw[k]) / d->dx - (gn[k] - gs[k]) / d->dy;
            /* bed slope (Kurganov & Levy), eta form */
            m[1] += d->g * 0.5 * (xp[c].eta + xm[c].eta) * (S->HE[c] - S->HW[c]) / d->dx;
            m[2] += d->g * 0.5 * (yp[c].eta + ym[c].eta) * (S->HN[c] - S->HS[c]) / d->dy;
            /* Coriolis with the local north vector, Section 3.7 */
            double ct = S->ct[c], st = S->st[c], fc = S->f[c];
            double hue = ct * hu[c] - st * hv[c];
            double hvn = st * hu[c] + ct * hv[c];
            m[1] += fc * (ct * hvn + st * (-hue));
            m[2] += fc * (-st * hvn + ct * (-hue));
            /* wind stress */
            double tx, ty;
            wind_at(d, i, j, t, &tx, &ty);
            m[1] += tx;
            m[2] += ty;
            M[s] = m[0]; M[np + s] = m[1]; M[2 * np + s] = m[2];
            Sf[s] = d->cd * sqrt(P[c].u * P[c].u + P[c].v * P[c].v) / fabs(P[c].hs);
        }
}

/* Public single evaluation of M(Q) and S(Q) (used by the tests). */
int orc_rhs(const orc_domain *d, const double *eta, const double *hu,
            const double *hv, double t, double *M, double *Sf)
{
    statics S;
    work W;
    if (statics_build(d, &S)) return -1;
    if (work_alloc(&S, &W)) { statics_free(&S); return -1; }
    double ax, ay;
    rhs(d, &S, &W, eta, hu, hv, t, M, Sf, &ax, &ay);
    work_free(&W);
    statics_free(&S);
    return 0;
}

/* The largest one-sided local speeds max(a+, -a-) over the x-faces and the
 * y-faces of one right-hand-side evaluation at time t (out[0], out[1]);
 * eq:cfl read at the faces bounds the time step by them. */
int orc_face_speeds(const orc_domain *d, const double *eta, const double *hu,
                    const double *hv, double t, double *out)
{
    size_t np = (size_t)d->nx * d->ny;
    statics S;
    work W;
    if (statics_build(d, &S)) return -1;
    if (work_alloc(&S, &W)) { statics_free(&S); return -1; }
    double *M = malloc(3 * np * sizeof(double)), *Sf = malloc(np * sizeof(double));
    int rc = (!M || !Sf) ? -1 : 0;
    if (!rc) rhs(d, &S, &W, eta, hu, hv, t, M, Sf, &out[0], &out[1]);
    free(M); free(Sf);
    work_free(&W);
    statics_free(&S);
    return rc;
}

/* The ghost-padded state after the ghost fill at time t (exported for the
 * pins of the boundary interpolation of Section 3.6): out holds 3 planes
 * (eta, hu, hv) of (ny+4) x (nx+4) cells, cell (i, j) at (j+2)(nx+4)+(i+2);
 * the ghost-ghost corners, which no stencil reads, are NaN. */
int orc_ghosts(const orc_domain *d, const double *eta_in, const double *hu_in,
               const double *hv_in, double t, double *out)
{
    int nx = d->nx, ny = d->ny;
    statics S;
    if (statics_build(d, &S)) return -1;
    size_t nc = (size_t)S.px * (ny + 4);
    double *eta = out, *hu = out + nc, *hv = out + 2 * nc;
    for (size_t c = 0; c < nc; c++) eta[c] = hu[c] = hv[c] = NAN;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t c = CI(&S, i, j), s = (size_t)j * nx + i;
            eta[c] = eta_in[s]; hu[c] = hu_in[s]; hv[c] = hv_in[s];
        }
    fill_ghosts(d, &S, eta, hu, hv, t);
    statics_free(&S);
    return 0;
}

/* One face flux from raw face states (h, eta, hu, hv) on both sides, the
 * face depth H_f and the direction: desingularised and combined exactly as
 * in the right-hand side (exported for the eta-form vs h-form test). */
void orc_face_flux(const double *left, const double *right, double Hf, double g,
                   double kappa, int dir, double *out)
{
    raw_face a = { left[0], left[1], left[2], left[3] };
    raw_face b = { right[0], right[1], right[2], right[3] };
    double speed;
    cu_flux(finish_face(a, g, kappa), finish_face(b, g, kappa), Hf, g, dir, out, &speed);
}

/* Face values of the x-reconstruction of every interior cell (eta^E, eta^W,
 * h^E, h^W), for the test of the local reformulation against the recursive
 * form of eq:recursiveV / eq:hOnFaces_E. Ghosts are filled at time t. */
int orc_recon_x(const orc_domain *d, const double *eta_in, const double *hu_in,
                const double *hv_in, double t, double *out /* 4*nx*ny */)
{
    int nx = d->nx, ny = d->ny;
    statics S;
    if (statics_build(d, &S)) return -1;
    size_t nc = (size_t)S.px * (ny + 4), np = (size_t)nx * ny;
    double *eta = malloc(nc * sizeof(double)), *hu = malloc(nc * sizeof(double));
    double *hv = malloc(nc * sizeof(double));
    prim *P = malloc(nc * sizeof(prim));
    if (!eta || !hu || !hv || !P) { free(eta); free(hu); free(hv); free(P); statics_free(&S); return -1; }
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t c = CI(&S, i, j), s = (size_t)j * nx + i;
            eta[c] = eta_in[s]; hu[c] = hu_in[s]; hv[c] = hv_in[s];
        }
    fill_ghosts(d, &S, eta, hu, hv, t);
    for (int j = -2; j <= ny + 1; j++)
        for (int i = -2; i <= nx + 1; i++) {
            int gx = (i < 0) || (i >= nx), gy = (j < 0) || (j >= ny);
            size_t c = CI(&S, i, j);
            if ((gx && gy) || S.land[c]) continue;
            P[c] = make_prim(&S, c, eta[c], hu[c], hv[c], d->kappa);
        }
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t c = CI(&S, i, j), s = (size_t)j * nx + i;
            raw_face p, m;
            if (S.land[c]) { out[s] = out[np + s] = out[2 * np + s] = out[3 * np + s] = NAN; continue; }
            reconstruct(d, &S, eta, hu, hv, P, i, j, 0, &p, &m);
            out[s] = p.eta; out[np + s] = m.eta; out[2 * np + s] = p.h; out[3 * np + s] = m.h;
        }
    free(eta); free(hu); free(hv); free(P); statics_free(&S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* time stepping                                                            */
/* ------------------------------------------------------------------------ */

static int is_land_cell(const orc_domain *d, int i, int j)
{
    int nx = d->nx;
    const double *H = d->H;
    return H[(size_t)j * (nx + 1) + i] == ORC_LAND ||
           H[(size_t)j * (nx + 1) + i + 1] == ORC_LAND ||
           H[(size_t)(j + 1) * (nx + 1) + i] == ORC_LAND ||
           H[(size_t)(j + 1) * (nx + 1) + i + 1] == ORC_LAND;
}

/* Flow-relaxation scheme, eq:frs: Q = (1 - alpha) Q + alpha Q^ext with
 * alpha = 1 - tanh(d/d0), d the distance in cells to the external boundary.
 * Readings: d = 0 at the outermost interior cell, the zone is frs_width
 * cells deep, Q^ext is the external solution of the ghost row touching the
 * domain at the same along-edge position, the relaxation follows each full
 * step, and nested edges are applied in the order S, N, W, E. */
static void apply_frs(const orc_domain *d, double *eta, double *hu, double *hv, double t)
{
    int nx = d->nx, ny = d->ny;
    for (int e = 0; e < 4; e++) {
        if (d->bc[e] != ORC_NESTED) continue;
#pragma omp parallel for schedule(static)
        for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
                int dist = e == ORC_S ? j : e == ORC_N ? ny - 1 - j : e == ORC_W ? i : nx - 1 - i;
                if (dist >= d->frs_width || is_land_cell(d, i, j)) continue;
                int k = (e == ORC_S || e == ORC_N) ? i : j;
                double a = 1.0 - tanh((double)dist / d->frs_d0);
                size_t s = (size_t)j * nx + i;
                eta[s] = (1.0 - a) * eta[s] + a * bnd_value(d, e, 0, 0, k, t);
                hu[s] = (1.0 - a) * hu[s] + a * bnd_value(d, e, 0, 1, k, t);
                hv[s] = (1.0 - a) * hv[s] + a * bnd_value(d, e, 0, 2, k, t);
            }
    }
}

/* The flow relaxation of eq:frs at time t (what follows each step). */
void orc_frs(const orc_domain *d, double *eta, double *hu, double *hv, double t)
{
    apply_frs(d, eta, hu, hv, t);
}

/* One time step of the semi-implicit SSP-RK2 scheme, eq:rk2_semiimp:
 *   Q*      = (Q^n + dt M(Q^n)) / (1 + dt S(Q^n))
 *   Q^{n+1} = (Q^n + Q* + dt M(Q*)) / 2 / (1 + dt S(Q*)/2)
 * with S acting on the momenta only; land cells are not updated. Stage one
 * sees the forcing at t, stage two at t + dt; the flow relaxation follows
 * at t + dt. M, Sf, qs: caller-provided scratch of 3, 1 and 3 planes. */
static void step(const orc_domain *d, const statics *S, work *W,
                 double *eta, double *hu, double *hv, double t, double dt,
                 double *M, double *Sf, double *qs)
{
    int nx = d->nx, ny = d->ny;
    size_t np = (size_t)nx * ny;
    double ax, ay;
    rhs(d, S, W, eta, hu, hv, t, M, Sf, &ax, &ay);
    for (size_t s = 0; s < np; s++) {
        qs[s] = eta[s] + dt * M[s];
        qs[np + s] = (hu[s] + dt * M[np + s]) / (1.0 + dt * Sf[s]);
        qs[2 * np + s] = (hv[s] + dt * M[2 * np + s]) / (1.0 + dt * Sf[s]);
    }
    if (d->round_state_f32)
        for (size_t s = 0; s < 3 * np; s++) qs[s] = (double)(float)qs[s];
    rhs(d, S, W, qs, qs + np, qs + 2 * np, t + dt, M, Sf, &ax, &ay);
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t s = (size_t)j * nx + i;
            if (S->land[CI(S, i, j)]) continue;
            eta[s] = 0.5 * (eta[s] + qs[s] + dt * M[s]);
            hu[s] = 0.5 * (hu[s] + qs[np + s] + dt * M[np + s]) / (1.0 + 0.5 * dt * Sf[s]);
            hv[s] = 0.5 * (hv[s] + qs[2 * np + s] + dt * M[2 * np + s]) / (1.0 + 0.5 * dt * Sf[s]);
        }
    apply_frs(d, eta, hu, hv, t + dt);
    if (d->round_state_f32)
        for (size_t s = 0; s < np; s++) {
            eta[s] = (double)(float)eta[s];
            hu[s] = (double)(float)hu[s];
            hv[s] = (double)(float)hv[s];
        }
}

int orc_step(const orc_domain *d, double *eta, double *hu, double *hv,
             double t, double dt)
{
    size_t np = (size_t)d->nx * d->ny;
    statics S;
    work W;
    if (statics_build(d, &S)) return -1;
    if (work_alloc(&S, &W)) { statics_free(&S); return -1; }
    double *M = malloc(3 * np * sizeof(double)), *Sf = malloc(np * sizeof(double));
    double *qs = malloc(3 * np * sizeof(double));
    int rc = (!M || !Sf || !qs) ? -1 : 0;
    if (!rc) step(d, &S, &W, eta, hu, hv, t, dt, M, Sf, qs);
    free(M); free(Sf); free(qs);
    work_free(&W);
    statics_free(&S);
    return rc;
}

/* Largest inverse CFL time over the wet cells, eq:cfl:
 * max over cells of max((|u| + sqrt(g hbar))/dx, (|v| + sqrt(g hbar))/dy),
 * with u, v the desingularised cell velocities and hbar clamped at 0. */
double orc_max_speed(const orc_domain *d, const double *eta, const double *hu,
                     const double *hv)
{
    int nx = d->nx, ny = d->ny;
    double best = 0.0;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            if (is_land_cell(d, i, j)) continue;
            size_t s = (size_t)j * nx + i;
            const double *H = d->H;
            double Hbar = 0.25 * (H[(size_t)j * (nx + 1) + i] + H[(size_t)j * (nx + 1) + i + 1] +
                                  H[(size_t)(j + 1) * (nx + 1) + i] + H[(size_t)(j + 1) * (nx + 1) + i + 1]);
            double hbar = eta[s] + Hbar;
            double hs = orc_desing(hbar, d->kappa);
            double c = sqrt(d->g * fmax(hbar, 0.0));
            double sx = (fabs(hu[s] / hs) + c) / d->dx;
            double sy = (fabs(hv[s] / hs) + c) / d->dy;
            double m = fmax(sx, sy);
            if (m > best || m != m) best = m;
        }
    return best;
}

/* dt = courant * 1/4 * min(dx / max|u +- c|, dy / max|v +- c|), eq:cfl with
 * the Courant number of Section 5 (reading: the factor 1/4 of eq:cfl is
 * kept; the P100 timings with dt ~ 0.92 s at 800 m only fit with it). */
double orc_cfl_dt(const orc_domain *d, const double *eta, const double *hu,
                  const double *hv, double courant)
{
    return courant * 0.25 / orc_max_speed(d, eta, hu, hv);
}

/* Advance n steps from time *t (steps past t_end > 0 are skipped, and the
 * step that would pass it is shortened to end on it). dt policy: a fixed
 * dt when dt_fixed > 0,
 * otherwise dt is recomputed from the current state before every step whose
 * global index (step0 + k) is a multiple of dt_every, and held in between
 * (Section 5 recomputes it every 20 simulated minutes). *dt carries the
 * held value in and out; dts (optional) receives each step's dt. */
int orc_run(const orc_domain *d, double *eta, double *hu, double *hv,
            double *t, double *dt, long step0, int n, double courant,
            double dt_fixed, int dt_every, double *dts, double t_end)
{
    size_t np = (size_t)d->nx * d->ny;
    if (dt_every < 1) dt_every = 1;
    statics S;
    work W;
    if (statics_build(d, &S)) return -1;
    if (work_alloc(&S, &W)) { statics_free(&S); return -1; }
    double *M = malloc(3 * np * sizeof(double)), *Sf = malloc(np * sizeof(double));
    double *qs = malloc(3 * np * sizeof(double));
    int rc = (!M || !Sf || !qs) ? -1 : 0;
    for (int k = 0; k < n && !rc; k++) {
        long s = step0 + k;
        /* past the forecast horizon every further step is a no-op */
        if (t_end > 0.0 && *t >= t_end * (1.0 - 1e-14)) { if (dts) dts[k] = 0.0; continue; }
        if (dt_fixed > 0.0) *dt = dt_fixed;
        else if (s % dt_every == 0 || !(*dt > 0.0)) {
            if (d->cfl_faces) {
                /* eq:cfl at the faces: the local speeds of the current
                 * state's reconstruction (one extra evaluation) */
                double ax, ay;
                rhs(d, &S, &W, eta, hu, hv, *t, M, Sf, &ax, &ay);
                *dt = courant * 0.25 / fmax(ax / d->dx, ay / d->dy);
            } else {
                *dt = orc_cfl_dt(d, eta, hu, hv, courant);
            }
        }
        if (!(*dt > 0.0) || !isfinite(*dt)) { rc = -2; break; }
        /* a forecast horizon: the step that would pass t_end ends on it */
        if (t_end > 0.0 && *t + *dt > t_end) *dt = t_end - *t;
        step(d, &S, &W, eta, hu, hv, *t, *dt, M, Sf, qs);
        if (dts) dts[k] = *dt;
        *t += *dt;
    }
    free(M); free(Sf); free(qs);
    work_free(&W);
    statics_free(&S);
    return rc;
}

/* Mass and energy over the wet cells: sum eta dx dy and
 * sum [ (hu^2 + hv^2)/(2 |h*|) + g eta^2 / 2 ] dx dy. */
void orc_diagnostics(const orc_domain *d, const double *eta, const double *hu,
                     const double *hv, double *mass, double *energy)
{
    int nx = d->nx, ny = d->ny;
    double m = 0.0, e = 0.0;
    for (int j = 0; j < ny; j++) {
        double mr = 0.0, er = 0.0;
        for (int i = 0; i < nx; i++) {
            if (is_land_cell(d, i, j)) continue;
            size_t s = (size_t)j * nx + i;
            const double *H = d->H;
            double Hbar = 0.25 * (H[(size_t)j * (nx + 1) + i] + H[(size_t)j * (nx + 1) + i + 1] +
                                  H[(size_t)(j + 1) * (nx + 1) + i] + H[(size_t)(j + 1) * (nx + 1) + i + 1]);
            double hs = fabs(orc_desing(eta[s] + Hbar, d->kappa));
            mr += eta[s];
            er += 0.5 * (hu[s] * hu[s] + hv[s] * hv[s]) / hs + 0.5 * d->g * eta[s] * eta[s];
        }
        m += mr; e += er;
    }
    *mass = m * d->dx * d->dy;
    *energy = e * d->dx * d->dy;
}

/* Threads of the parallel loops from now on (the CPU baseline also times
 * the oracle on one core). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
