// swe_kernels.h -- launchers of the libswe kernels (internal).
#pragma once
#include <vector>

#include "swe_internal.h"

namespace swe {

int ref_step_parts();
const char *ref_part_name(int part);
template <typename T>
cudaError_t launch_step_ref_part(const StageArgs<T> &a, cudaStream_t st, int part, bool kahan);
template <typename T>
cudaError_t launch_init_clock(const StageArgs<T> &a, cudaStream_t st, double t, double dt,
                              long long step);
template <typename T>
cudaError_t launch_refresh_brackets(const StageArgs<T> &a, cudaStream_t st);
template <typename T>
cudaError_t launch_diagnostics(const StageArgs<T> &a, double *partials, double *out,
                               cudaStream_t st);
cudaError_t launch_ctl_init(StepCtl *ctl, double t0, cudaStream_t st);
cudaError_t launch_set_end(StepCtl *ctl, double t_end, cudaStream_t st);
template <typename T>
cudaError_t launch_read_plane(const StepCtl *ctl, const T *q0, const T *q1, long long pitch,
                              int nx, int ny, T *dst, cudaStream_t st);

// FP32 sliding-window stage kernels (swe_stage_fast.cu): stage 1, then
// stage 2 with the fused CFL reduction and clock update (stage 0: the speed
// pass of the face-speed time step). A single domain
// runs through the same kernel as a batch, its arguments in the launch's
// parameter space.
// With faces: a speed pass (the faces' one-sided speeds of the state, dt)
// before the two stages.
int fast_step_parts(bool faces);
const char *fast_part_name(int part, bool faces);
// Work planning (swe_stage_fast.cu): a warp item is a strip of 28 output
// columns by a run of rows, packed as {strip, j0 | rows << 16}; a launch
// covers the items of the domain's plan. Budgets cap the cost of an item in
// kPlanUnit per plain row. wet: strips x ny flags of launch_wet_strips
// (strip-major) on the host, or NULL (every cell wet).
constexpr int kPlanUnit = 100;
constexpr int kStripColumns = 28;        // output columns of a warp item
int fast_strips(int nx);
int fast_budget(int nx, int ny, const unsigned char *wet, const int bc[4], int frs_width);
// alone: the plan of a domain launched by itself (a batch launches many)
void fast_plan(int nx, int ny, const unsigned char *wet, const int bc[4], int frs_width, int budget,
               bool alone, std::vector<uint2> &items);
int fast_tiles(int n_items);
cudaError_t launch_wet_strips(const float *H, long long cpitch, int nx, int ny, unsigned char *out,
                              cudaStream_t st);
// gridded: some domain of the batch has gridded wind (the kernel with the
// per-cell wind sampling); a single domain's launch decides by its own wind.
cudaError_t launch_batch_stage(const BatchTable &tab, int blocks, int stage, bool gridded, cudaStream_t st);
// The same kernel for one domain whose arguments travel with the launch.
cudaError_t launch_domain_stage(const OneDomain &one, int stage, cudaStream_t st);
// Fill the external edge state of the current time level (after the clock
// or the forcing was set); stage 1 of every step fills the next level.
cudaError_t launch_edge_fill(const StageArgs<float> &a, cudaStream_t st);
long long edge_floats(int nx, int ny);   // both time levels

// Domain decomposition on one device (swe_kernels.cu): the largest CFL
// maximum of the own cells of every sub-domain (launch_speed, once per
// sub-domain, at set-up), one clock evaluation for all of them
// (launch_split_clock; mode as in clock_advance), and the halo exchange
// between their planes (launch_halo_copy; what 0: the current state, 1:
// the stage-1 increment).
constexpr int kSplitMax = 16;            // SWE_SPLIT_MAX
constexpr int kHaloCopies = 48;          // copies per launch
struct SplitClocks {
    int n;
    StepCtl *ctl[kSplitMax];
    ClockParams clk;
    ForcingDev bnd[kSplitMax], wind[kSplitMax];
};
struct SplitPlanes {
    float *q[2][3];
    float *d1[3];
    const StepCtl *ctl;
    long long pitch;
    int wx0, wy0;                        // window origin in the whole domain
};
struct HaloCopy {
    int dst, src;                        // sub-domain indices
    int x0, x1, y0, y1;                  // box in whole-domain cells
};
struct HaloTable {
    int n_copies;
    SplitPlanes dom[kSplitMax];
    HaloCopy copy[kHaloCopies];
};
cudaError_t launch_speed(const StageArgs<float> &a, cudaStream_t st);
cudaError_t launch_split_clock(const SplitClocks &c, int mode, cudaStream_t st);
cudaError_t launch_halo_copy(const HaloTable &t, int what, cudaStream_t st);
int diag_blocks(int nx, int ny);

// Record e for swe_last_cuda_error and return SWE_ERR_CUDA (swe_capi.cu).
int record_cuda_error(cudaError_t e);

// An NVTX range over a host entry point (a no-op unless a profiler that
// collects NVTX is attached): the library's calls show up by name in nsys /
// ncu timelines beside the kernels they enqueue.
struct TraceRange {
    explicit TraceRange(const char *name);
    ~TraceRange();
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace swe
