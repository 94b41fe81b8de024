// swe_internal.h -- device-side data structures shared by the kernels and
// the C-ABI host code of libswe. Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace swe {

constexpr int kMaxFrs = 32;          // deepest flow-relaxation zone supported
constexpr float kLand = 3.40282346638528859812e+38f;  // FLT_MAX corner marker
enum { EDGE_S = 0, EDGE_N = 1, EDGE_W = 2, EDGE_E = 3 };
enum { BC_WALL = 0, BC_NESTED = 1, BC_PERIODIC = 2 };
enum { ERR_NONE = 0, ERR_NUMERIC = -4, ERR_BOUNDS = -6 };

// Device-resident clock of one domain. The stage kernels read dt and the
// forcing brackets from here and the end-of-step reduction writes the next
// dt here, so a sequence of steps needs no host round trip.
struct StepCtl {
    double t;                 // simulated time of the current state
    double dt;                // dt of the next step
    long long step;           // steps taken
    double tau[2][2];         // uniform wind stress at stage-1 / stage-2 time
    double bs[2];             // boundary frame weight s at stage-1 / stage-2 time
    float bs_f[2];            // the same, rounded once for FP32 kernels
    float tau_f[2][2];        // uniform wind stress rounded once for FP32 kernels
    double ws[2];             // wind frame weight s
    int bk[2];                // boundary frame index at stage-1 / stage-2 time
    int wk[2];                // wind frame index
    double last_speed;        // last CFL reduction result
    unsigned int speed32;     // atomicMax target (float bits)
    unsigned int blocks_done; // last-block-done counter of the fused finalise
    unsigned long long speed64;  // atomicMax target (double bits)
    int err;                  // sticky error code
    int err_cell;             // first offending cell, -1 if none
    long long err_step;
    int parity;               // which state buffer holds Q^n (flipped per step)
    int done;                 // 1 once t reached t_end: steps become no-ops
    double t_end;             // end of the forecast (0: none); the last dt is clipped
};

// Clock policy, copied by value into the finalise kernels.
struct ClockParams {
    double courant;
    double dt_fixed;
    int dt_every;
    int wind_uniform;         // wind frames are 1x1: precompute tau per stage
    double rho_ratio;         // rho_air / rho_water
    int fp32;                 // an FP32 domain: frame weights and wind stress in FP32
    int cfl_faces;            // dt from the faces' one-sided speeds (a speed pass per step)
    int split;                // a sub-domain: stage 2 leaves its CFL maximum for a shared clock
};

struct ForcingDev {
    const float *frames;      // device frames (layout in swe.h)
    const double *times;      // device times
    int n, n1, n2;            // frames, samples along x / y (or grid size)
};

template <typename T>
struct StageArgs {
    int nx, ny;
    long long pitch;          // elements per row of cell planes
    long long cpitch;         // elements per row of the corner plane
    T dx, dy, inv_dx, inv_dy;
    T kx, ky;                 // dx/(2g), dy/(2g)
    T g, kappa, half_inv_kappa, tm, cd;
    int bc[4];
    const T *H, *f, *th;      // corner depths; f/theta planes or NULL
    T f_const, th_const;
    T *q[2][3];               // ping-pong state buffers; ctl->parity selects Q^n
    T *d1[3];                 // stage-1 increment Q* - Q^n
    T *comp[3];               // Kahan compensation (F32_KAHAN) or NULL
    ForcingDev bnd, wind;
    int frs_width;
    double frs_alpha[kMaxFrs];
    float frs_alpha_f[kMaxFrs];   // the same weights rounded once for FP32 kernels
    StepCtl *ctl;
    ClockParams clk;
    // FP32 fast path: the external state of Section 3.6 on the two ghost
    // rings of every nested edge, one copy per time level (two levels,
    // selected by the step parity); NULL on the other paths. A level holds
    // 12 (nx + ny) floats: edge S at 0, N at 6 nx, W at 12 nx, E at
    // 12 nx + 6 ny; within an edge of length n, value v of ring r at
    // position k sits at (3 r + v) n + k.
    float *edge;
    // FP32 fast path: the warp items a launch covers, {strip, j0 | rows << 16}
    // (rows without a wet cell in the strip are left out: land cells are
    // never written). NULL: every strip of `rows`-row bands.
    const uint2 *items;
    int n_items;
    // elements of each buffer (checked by the bounds-checked debug builds)
    long long n_plane, n_corner, n_edge, n_bnd, n_wind;
    // a window of a larger domain: cell (0, 0) is the whole domain's cell
    // (off_x, off_y), which has gnx x gny cells (forcing is sampled at the
    // whole domain's positions); the CFL maximum covers the own cells
    // [own_x0, own_x1) x [own_y0, own_y1). A whole domain: offsets 0,
    // gnx = nx, gny = ny, every cell its own.
    int off_x, off_y, gnx, gny;
    int own_x0, own_x1, own_y0, own_y1;
};

// A single FP32 domain handed to the stage kernel with the launch (kernel
// parameter space): tiles > 0 selects it over the batch table.
struct OneDomain {
    StageArgs<float> args;
    int tiles, rows, strips;
};

// Device-resident tile table of a batch of FP32 domains (one block per tile).
struct BatchTable {
    const StageArgs<float> *args;   // per domain
    const int *tile_start;          // n+1 prefix sums of tiles per domain
    const int *tile_dom;            // domain of each tile
    const int *grid_x;              // 28-column strips per row of each domain
    const int *rows;                // tile height of each domain
    const int *n_domains;           // current number of domains (device)
};

}  // namespace swe
