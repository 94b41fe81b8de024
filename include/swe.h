/*
 * swe.h -- C ABI of libswe, a GB300 (sm_103a) implementation of one time
 * step of the well-balanced central-upwind finite-volume scheme for the
 * rotating shallow-water equations of Brodtkorb & Holm, "Real-World
 * Oceanographic Simulations on the GPU using a Two-Dimensional
 * Finite-Volume Scheme" (arXiv 1912.02457).
 *
 * Every function returns SWE_OK (0) or a negative swe_status; none aborts
 * and no C++ exception crosses the ABI. A handle may be used from one
 * thread at a time; different handles may be used from different threads.
 * All kernels of a domain run on the CUDA stream given at creation, in
 * stream order, without host synchronisation unless a function says so.
 *
 * Grid conventions (Section 2): cell-average state (eta, hu, hv) on an
 * nx x ny grid, row-major with x fastest; eta = h - H is the sea-surface
 * deviation (eq:eta), hu and hv the momenta. The equilibrium depth H is
 * given at the (nx+1) x (ny+1) cell corners and is piecewise bilinear
 * (Section 3.9); a corner equal to SWE_LAND marks land (Section 3.4: the
 * land mask is a no-data value of the bathymetry), and a cell with any
 * SWE_LAND corner is land. Edges are numbered S, N, W, E = 0..3
 * (S: j = 0, W: i = 0).
 */
#ifndef SWE_H
#define SWE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SWE_LAND 3.40282346638528859812e+38f  /* FLT_MAX: land corner */
#define SWE_ABI_VERSION 2

typedef enum {
    SWE_OK = 0,
    SWE_ERR_INVALID_ARG = -1,  /* bad pointer, size, enum or ordering */
    SWE_ERR_OOM = -2,          /* device or host allocation failed */
    SWE_ERR_CUDA = -3,         /* a CUDA call failed; see swe_last_cuda_error */
    SWE_ERR_NUMERIC = -4,      /* non-finite state or time step (sticky) */
    SWE_ERR_UNSUPPORTED = -5,  /* option not built into this library */
    SWE_ERR_BOUNDS = -6        /* a kernel access outside its buffer was caught
                                  and skipped (bounds-checked debug builds only;
                                  sticky; swe_info.error_cell = source line) */
} swe_status;

typedef enum {
    SWE_F32 = 0,        /* FP32 state and arithmetic */
    SWE_F32_KAHAN = 1,  /* FP32 arithmetic, Kahan-compensated RK update */
    SWE_F64 = 2         /* FP64 everywhere (parity build, not a fast path) */
} swe_precision;

/* Boundary of one edge. WALL: reflective (Section 3.3). NESTED: ghosts from
 * the boundary frames with flow relaxation (Section 3.6). PERIODIC (Section
 * 3.3): the opposite edge must be PERIODIC too, and the corner plane's last
 * row (for S/N) or column (for W/E) must repeat its first. */
typedef enum { SWE_BC_WALL = 0, SWE_BC_NESTED = 1, SWE_BC_PERIODIC = 2 } swe_bc;
typedef enum { SWE_FORCING_WIND = 0, SWE_FORCING_BOUNDARY = 1 } swe_forcing_kind;

typedef enum {
    SWE_ETA = 0, SWE_HU = 1, SWE_HV = 2,            /* state planes, nx*ny */
    SWE_COMP_ETA = 3, SWE_COMP_HU = 4, SWE_COMP_HV = 5  /* Kahan terms */
} swe_field;

/* Scheme parameters (Sections 2-3). Fill with swe_default_params first. */
typedef struct {
    double g;               /* gravitational acceleration, 9.81 */
    double theta_mm;        /* generalised-minmod parameter, 1.3 */
    double kappa;           /* desingularisation depth of eq:desing_ours, 1e-2 m */
    double cd;              /* quadratic bottom drag C_d (S = C_d |u| / |h*|) */
    double courant;         /* Courant number of eq:cfl (dt = C/4 * min(...)) */
    double frs_d0;          /* flow relaxation fall-off d0 of eq:frs, 2.5 */
    int frs_width;          /* relaxation zone depth in cells (<= 32), 10 */
    int dt_update_every;    /* recompute dt every k steps (Section 5), 1 */
    double dt_fixed;        /* > 0: fixed dt, no CFL reduction */
    double rho_air;         /* 1.225 (Section 3.5) */
    double rho_water;       /* 1025 */
    double t0;              /* initial simulated time, s */
    int kernel;             /* 0 (use this): the kernels of the precision,
                               the sliding-window stage kernels for FP32
                               domains and the one-thread-per-cell kernels
                               for FP64 ones; 1: test instrument only, FP32
                               domains on the one-thread-per-cell kernels
                               (slower, not batchable), kept so that tests
                               can cross-check the two FP32 kernel sets */
    int cfl_faces;          /* 0: eq:cfl with the cell-average velocities and
                               depths of the state (the reading of the scheme);
                               1: eq:cfl with the faces' one-sided speeds a+, a-
                               of the state's reconstruction (Kurganov &
                               Petrova's condition for non-negative depths over
                               moving wet-dry fronts; an extra launch per step
                               and, on drying shelves, much shorter steps).
                               FP32 domains on the default kernels only, not
                               batchable (SWE_ERR_UNSUPPORTED otherwise) */
    /* Domain decomposition. Each RK stage of the scheme (Section 3:
       reconstruction from two cells on each side, fluxes between them)
       reads two cells along x and along y, so sub-domains that hold a
       two-cell halo of their neighbours' cells, refreshed after every
       stage, update their own cells exactly as the whole domain would.
       whole_nx = whole_ny = 0 (the default): this domain is whole and the
       other fields below are 0. Otherwise it is the window of a
       whole_nx x whole_ny domain whose cell (0, 0) is the whole domain's
       cell (window_x0, window_y0): wind and nesting frames are sampled at
       the whole domain's positions; it owns the cells [own_x0, own_x1) x
       [own_y0, own_y1) of the window (window coordinates), and its other
       cells are halo cells that swe_split_step overwrites from the
       sub-domains owning them (an edge of the window that faces a
       neighbour is given as a wall: what it does to the halo cells next
       to it is never used). Its CFL maximum covers its own cells only.
       FP32 domains on the default kernels with cfl_faces 0 and no
       periodic edge (SWE_ERR_UNSUPPORTED otherwise); not batchable. */
    int window_x0, window_y0, whole_nx, whole_ny;
    int own_x0, own_x1, own_y0, own_y1;
} swe_params;

/* Domain description. Arrays are read once by swe_create_domain and
 * copied; the caller keeps ownership. Element type of eta/hu/hv/H/f/theta
 * is float for SWE_F32 and SWE_F32_KAHAN, double for SWE_F64. */
typedef struct {
    int nx, ny;             /* cells, 1 <= nx, ny <= 65536, nx*ny < 2^31;
                               >= 2 across a nested edge */
    double dx, dy;          /* cell size, m */
    int precision;          /* swe_precision */
    int bc[4];              /* swe_bc per edge S, N, W, E */
    const void *eta, *hu, *hv;  /* nx*ny initial state */
    const void *H;          /* (nx+1)*(ny+1) corner depths, SWE_LAND = land */
    const void *f;          /* nx*ny Coriolis parameter, or NULL: f_const */
    const void *theta;      /* nx*ny north angle (rad), or NULL: theta_const */
    double f_const, theta_const;
    int src_is_device;      /* 1: the pointers above are device pointers */
} swe_domain_desc;

typedef struct {
    double t;               /* simulated time of the current state, s */
    double dt;              /* time step the next step will take, s */
    long long step;         /* steps taken since creation */
    int error;              /* sticky swe_status of the device, 0 if none */
    int error_cell;         /* first offending cell (j*nx+i), -1 if none */
    long long error_step;   /* step at which it was found */
    double max_speed;       /* last CFL reduction: max (|u|+c)/dx, (|v|+c)/dy */
    long long launches;     /* kernel launches issued by swe_step* so far */
    int done;               /* 1 once t reached the end time: steps are no-ops */
    double t_end;           /* end time set by swe_set_end_time, 0 if none */
} swe_info;

typedef struct swe_domain *swe_handle;

/* Optional device allocator (e.g. a framework's caching allocator). When
 * set, every device buffer of domains created afterwards comes from it and
 * is returned to it by swe_destroy_domain. ctx is passed through. */
typedef void *(*swe_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*swe_free_fn)(void *ptr, void *stream, void *ctx);
int swe_set_allocator(swe_alloc_fn alloc, swe_free_fn release, void *ctx);

/* Defaults of the readings the paper leaves open: g = 9.81, theta = 1.3,
 * kappa = 1e-2 m, C_d = 0, Courant 0.8 (Section 5), d0 = 2.5, zone 10
 * cells, dt every step, rho_air 1.225, rho_water 1025, t0 = 0, kernel 0. */
void swe_default_params(swe_params *p);

/* Create a domain: validate the description, allocate its device planes,
 * upload state and statics, and compute the first time step from the
 * initial state by the CFL condition eq:cfl (Section 2), all on `stream`
 * (a cudaStream_t, NULL = legacy default stream).
 * Errors: SWE_ERR_INVALID_ARG (sizes, enums, NULL pointers, frs_width),
 * SWE_ERR_OOM, SWE_ERR_CUDA. On error *out is NULL and nothing leaks. */
int swe_create_domain(const swe_domain_desc *d, const swe_params *p,
                      void *stream, swe_handle *out);

/* Set the forcing time series (Section 3.5 wind, Section 3.6 nesting).
 * times: n_frames increasing host doubles (s); frames: host floats.
 *   SWE_FORCING_WIND:     frames = n_frames x n2 x n1 x 2 wind at 10 m
 *                         (grid axes, m/s) on an n1 x n2 grid spanning the
 *                         domain, bilinear in space (cell centres),
 *                         linear in time (eq:windstress_interpol).
 *   SWE_FORCING_BOUNDARY: frames = n_frames x 12*(n1+n2): per frame edges
 *                         S, N (n1 samples each) then W, E (n2 samples),
 *                         each edge as [ghost row r][var v][k], r = 0 the
 *                         ghost row touching the domain, v = eta, hu, hv;
 *                         linear along the edge and in time; used by the
 *                         ghost cells of nested edges and as Q^ext of the
 *                         flow relaxation eq:frs.
 * Outside [times[0], times[n-1]] the nearest frame is held. Data are
 * copied (stream-ordered); the previous series is released after the
 * stream reaches this call. Errors: SWE_ERR_INVALID_ARG, SWE_ERR_OOM. */
int swe_set_forcing(swe_handle h, int kind, int n_frames, const double *times,
                    const float *frames, int n1, int n2);

/* Advance n_steps >= 0 steps of the semi-implicit SSP-RK2 scheme
 * eq:rk2_semiimp with the central-upwind fluxes eqn:numerical_flux,
 * asynchronously on the domain's stream. Each step: stage 1 at t, stage 2
 * at t + dt, flow relaxation, then the fused CFL reduction sets the next
 * dt on the device (no host synchronisation). Runs of 16 steps replay one
 * CUDA graph and the remaining steps a one-step graph (both captured on
 * first use, rebuilt after swe_set_forcing).
 * Numerical failures are reported through swe_get_info / the next
 * synchronising call.
 * Errors: SWE_ERR_INVALID_ARG, SWE_ERR_CUDA (launch), SWE_ERR_NUMERIC
 * (a sticky device error was already observed). */
int swe_step(swe_handle h, int n_steps);

/* Forecast horizon: the step that would pass t_end is shortened to end
 * exactly at t_end, after which steps leave the state and clock unchanged
 * (swe_info.done = 1). t_end = 0 removes the horizon. Stream-ordered. */
int swe_set_end_time(swe_handle h, double t_end);

/* Kernel launches one step issues, and the name of launch `part` of a step
 * ("stage1", "stage2", ...). For measurement tools. */
int swe_launches_per_step(swe_handle h);
const char *swe_launch_name(swe_handle h, int part);

/* swe_step with a CUDA event recorded before and after every kernel
 * launch; synchronises at the end and writes each launch's device time in
 * ms to ms[0 .. n_steps * swe_launches_per_step(h) - 1], in launch order.
 * capacity: elements of ms. Same numerics as swe_step. */
int swe_step_profiled(swe_handle h, int n_steps, float *ms, int capacity);

/* Copy one field of the current state (nx*ny, row-major, element type of
 * the domain's precision) to dst, host or device memory. Stream-ordered;
 * for a host dst the call synchronises the stream before returning. */
int swe_read_state(swe_handle h, int field, void *dst, int dst_is_device);

/* Overwrite one field of the current state from src (same layout). Land
 * cells keep whatever the caller writes. Writing a state field clears the
 * matching Kahan term. Stream-ordered; the source must stay valid until
 * the stream passes the call when src_is_device, and is copied before
 * return for a host src. */
int swe_write_state(swe_handle h, int field, const void *src, int src_is_device);

/* Set the clock: time t, step counter, and dt (dt <= 0: recompute it from
 * the current state by eq:cfl). Used to resume from a checkpoint. */
int swe_set_clock(swe_handle h, double t, double dt, long long step);

/* Synchronise the domain's stream and report clock, dt and the sticky
 * device error (swe_info). Returns SWE_ERR_NUMERIC when a device error is
 * set, SWE_ERR_CUDA when the stream failed. */
int swe_get_info(swe_handle h, swe_info *out);

/* Mass and energy over the wet cells, accumulated in FP64 on the device:
 * out[0] = sum eta dx dy, out[1] = sum [(hu^2+hv^2)/(2|h*|) + g eta^2/2] dx dy.
 * Synchronises the stream. */
int swe_diagnostics(swe_handle h, double out[2]);

/* Release every resource of the domain after its stream drains. */
int swe_destroy_domain(swe_handle h);

/* ---- batches: ensembles and served forecasts --------------------------
 * A batch advances many FP32 domains (of any sizes, each with its own
 * clock, dt, forcing and horizon) by ONE launch per RK stage: a block per
 * tile of a device-resident table of tiles covering all domains, and each
 * domain's CFL reduction and clock update are done by its own last tile.
 * Runs of 8 batch steps replay one CUDA graph; because the tables,
 * parities, clocks and horizons live on the device, the graph stays valid
 * when domains are added or removed without changing the tile count (it
 * is recaptured otherwise). The result of every domain is bitwise
 * the same as stepping it alone (the per-cell arithmetic does not depend on
 * the tiling). While in a batch a domain must be stepped only through it;
 * read its state after swe_batch_sync. A domain that reached its end time
 * (swe_set_end_time) is skipped at no cost. */
typedef struct swe_batch *swe_batch_handle;

/* Create an empty batch working on `stream`, with table room for
 * max_domains domains. Allocates device memory. */
int swe_batch_create(void *stream, int max_domains, swe_batch_handle *out);
/* Add / remove a domain (FP32 or FP32_KAHAN with the fast kernels;
 * SWE_ERR_UNSUPPORTED otherwise). Both drain the streams involved. */
int swe_batch_add(swe_batch_handle b, swe_handle d);
int swe_batch_remove(swe_batch_handle b, swe_handle d);
int swe_batch_size(swe_batch_handle b);
/* Tile height: the work budget of a warp item in rows (items are 28
 * columns wide, four to a block; each domain's wet rows are cut into items
 * of about this cost, land left out). 0 = autotune:
 * the first swe_batch_step of >= 16 steps times 2 steps with each of the
 * heights 8, 16, 32, 64 and keeps the fastest (these are real steps).
 * Every height a domain is stepped with keeps its work plan (a few bytes
 * per item) on the device until the domain is destroyed.
 * swe_batch_rows returns the current choice (0 until tuned). */
int swe_batch_set_rows(swe_batch_handle b, int rows);
int swe_batch_rows(swe_batch_handle b);
/* Advance every domain of the batch n_steps steps (asynchronous). */
int swe_batch_step(swe_batch_handle b, int n_steps);
/* The same steps launched the plain way, domain after domain, two kernels
 * per domain per step (the baseline the batched path is measured against). */
int swe_batch_step_serial(swe_batch_handle b, int n_steps);
int swe_batch_sync(swe_batch_handle b);
/* Synchronise, then report per domain (in add order) whether it reached
 * its end time and its simulated time. capacity >= swe_batch_size. */
int swe_batch_poll(swe_batch_handle b, int *done, double *t, int capacity);
/* Kernel launches issued by this batch so far. */
long long swe_batch_launches(swe_batch_handle b);
int swe_batch_destroy(swe_batch_handle b);

/* ---- domain decomposition on one device --------------------------------
 * n sub-domains (windows created with whole_nx > 0, see swe_params) whose
 * own cells tile the whole domain exactly once, whose windows hold two
 * cells beyond their own cells on every side that does not lie on the
 * whole domain's edge, and whose halo cells each lie in another
 * sub-domain's own cells, all on one stream, with the same
 * whole domain, cell size, precision and clock parameters; at most
 * SWE_SPLIT_MAX of them. Both calls are asynchronous on that stream.
 * swe_split_sync: one clock for all of them: the CFL maximum of eq:cfl
 * over every sub-domain's own cells sets one initial time step (their
 * clocks must hold the same t; call it after creating them, and after
 * swe_set_clock or swe_set_forcing on them).
 * swe_split_step: n_steps steps of the whole domain: stage 1 of every
 * sub-domain, the exchange of the stage-1 increment's halo cells, stage 2
 * of every sub-domain, one clock evaluation from the largest of their CFL
 * maxima (eq:cfl; every sub-domain gets the same t, dt and forcing
 * brackets), the exchange of the new state's halo cells. The own cells
 * end bit for bit where the whole domain's steps put them. The exchanges
 * are device copies between the sub-domains' planes; the same sequence
 * across devices would exchange through peer copies or messages (not
 * provided: one device).
 * Errors: SWE_ERR_INVALID_ARG (NULL, n out of range, not a tiling,
 * different streams or parameters, a domain that is not a window),
 * SWE_ERR_NUMERIC (a sticky device error observed before), SWE_ERR_CUDA. */
#define SWE_SPLIT_MAX 16
int swe_split_sync(const swe_handle *doms, int n);
int swe_split_step(const swe_handle *doms, int n, int n_steps);

/* ---- diagnostics for callers that cannot allocate ----------------------
 * The paper has no counterpart to this function; it is a service of this
 * library. It computes what swe_diagnostics computes (FP64 mass and
 * energy over the water cells) from caller-owned FP32 device planes, and
 * allocates nothing, for callers that cannot allocate device memory where
 * they need the numbers: code running while a stream is captured into a
 * CUDA graph (cudaMalloc is not allowed there), code inside a framework
 * that owns every device buffer through its own pool, real-time loops in
 * which an allocation may block.
 *   eta, hu, hv: device planes, ny rows of `pitch` floats (pitch >= nx);
 *   H: device corner depths, ny+1 rows of `cpitch` floats (cpitch >= nx+1),
 *      SWE_LAND at land corners; dx, dy, g, kappa as in swe_params;
 *   out: device pointer to 2 doubles, written stream-ordered on `stream`.
 * Scratch: per-row partial sums in a fixed device array of
 * SWE_NOALLOC_MAX_ROWS rows (256 KiB) that every GPU loading the library
 * keeps until the process exits; ny > SWE_NOALLOC_MAX_ROWS is rejected with
 * SWE_ERR_INVALID_ARG. The first call on each device looks the array's
 * device address up (cudaGetSymbolAddress), so make that first call before
 * any stream capture. Every call writes the partials it reads, so nothing
 * carries over between calls, but all calls share the one array: calls
 * that overlap on the GPU (other streams, other host threads) race, so
 * order them on one stream. Devices with an ordinal of 64 or more are not
 * supported (SWE_ERR_UNSUPPORTED); SWE_ERR_CUDA reports a failed address
 * lookup or a failed launch of this call (an error left pending by earlier
 * calls is neither reported nor cleared). */
#define SWE_NOALLOC_MAX_ROWS 16384
int swe_diagnostics_noalloc(const float *eta, const float *hu, const float *hv, const float *H,
                            int nx, int ny, long long pitch, long long cpitch, double dx,
                            double dy, double g, double kappa, double *out, void *stream);

/* ---- grid pre-processing (Sections 3.8 and 3.9) -------------------------
 * Run once before a simulation; all planes are device memory, row-major with
 * the given row pitch in elements, and the work is stream-ordered on
 * `stream`. Nothing is allocated. Corner planes carry SWE_LAND at land
 * intersections where stated. Errors: SWE_ERR_INVALID_ARG for a NULL
 * pointer, a size < 1, a pitch shorter than its row, or a parameter out of
 * range; SWE_ERR_CUDA for a failed launch or copy. */

/* Corner (bilinear) bathymetry from cell averages, Section 3.8 (FP32, the
 * precision of the stage kernels that read the corners): the initial
 * guess of eqn:recon_1 - eqn:recon_3 (limited cell slopes, each cell's plane
 * at its corners, the mean of the estimates meeting at an intersection),
 * then n_iter iterations of: dH = Hm - (mean of each cell's corners), add
 * the eqn:recon_1 - eqn:recon_3 corner estimate of dH, smooth the corners.
 *   Hm:    ny x nx cell averages (FP32), pitch >= nx;
 *   Hc:    (ny+1) x (nx+1) corners (FP32 output), cpitch >= nx+1;
 *   work:  swe_bathymetry_work_bytes(nx, ny) bytes of device scratch,
 *          256-byte aligned;
 *   theta: generalised-minmod parameter of the slopes, 1 <= theta <= 2;
 *   smooth: weight w of the smoothing pass Hc := (1-w) Hc + w (mean of the
 *          4 neighbour corners), 0 <= w <= 1; beyond an edge a cell or a
 *          corner is linearly extrapolated, so a linear surface is exact;
 *   stats: NULL, or a host array of 2 n_iter doubles that receives, per
 *          iteration, max|Hm - cell mean of Hc| and max|corner change|
 *          (the call then synchronises `stream`). */
size_t swe_bathymetry_work_bytes(int nx, int ny);
int swe_bathymetry_reconstruct(const float *Hm, long long pitch, int nx, int ny, float *Hc,
                               long long cpitch, void *work, int n_iter, double theta,
                               double smooth, double *stats, void *stream);

/* One step of land erosion for narrow straits, Section 3.8: a land cell
 * stays land only if its four neighbours are land (outside the domain
 * counts as land); a cell it opens takes the largest eta of its water
 * neighbours (gray dilation) and the depth land_depth (5 m in the paper).
 *   land, land_out: ny x nx bytes (nonzero = land); eta, Hm in, eta_out,
 *   Hm_out out (FP32); every plane has row pitch `pitch` elements; outputs
 *   must not alias inputs. */
int swe_land_erode(const unsigned char *land, const float *eta, const float *Hm,
                   long long pitch, int nx, int ny, double land_depth,
                   unsigned char *land_out, float *eta_out, float *Hm_out, void *stream);

/* Refinement by two, Section 3.9 (FP32): every water cell's slope-limited
 * reconstruction (generalised minmod with theta; a land or out-of-domain
 * neighbour gives a zero difference) evaluated at its four children's
 * centres; the corner surface evaluated at the fine intersections (coarse
 * corner, mean of two, mean of four; SWE_LAND if any of them is). Children
 * of land cells are land with zero state.
 *   eta, hu, hv: ny x nx, pitch; H: (ny+1) x (nx+1) corners, cpitch;
 *   eta_f, hu_f, hv_f: 2ny x 2nx, fpitch (even); H_f: (2ny+1) x (2nx+1),
 *   fcpitch. Fine outputs start on 8-byte boundaries. */
int swe_refine2(const float *eta, const float *hu, const float *hv, long long pitch,
                const float *H, long long cpitch, int nx, int ny, double theta,
                float *eta_f, float *hu_f, float *hv_f, long long fpitch, float *H_f,
                long long fcpitch, void *stream);

/* Coarsening by two, Section 3.9 (FP32): a coarse cell is the mean of its
 * water children (zero if it is land, i.e. one of its sampled corners is
 * SWE_LAND, or has none); the coarse corners are the even fine corners.
 *   fine: 2ny x 2nx planes with fpitch (even), (2ny+1) x (2nx+1) corners with
 *   fcpitch; coarse outputs ny x nx with pitch, (ny+1) x (nx+1) with cpitch.
 *   Fine planes start on 8-byte boundaries. */
int swe_coarsen2(const float *eta_f, const float *hu_f, const float *hv_f, long long fpitch,
                 const float *H_f, long long fcpitch, int nx, int ny, float *eta, float *hu,
                 float *hv, long long pitch, float *H, long long cpitch, void *stream);

/* The last CUDA error string recorded by this thread, or "". */
const char *swe_last_cuda_error(void);
const char *swe_status_string(int status);
int swe_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SWE_H */
