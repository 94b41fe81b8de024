// swe_kernels.h -- launchers of the libswe kernels (internal).
#pragma once
#include "swe_internal.h"

namespace swe {

template <typename T>
cudaError_t launch_step_ref(const StageArgs<T> &a, cudaStream_t st, bool kahan);
template <typename T>
cudaError_t launch_init_clock(const StageArgs<T> &a, cudaStream_t st, double t, double dt,
                              long long step);
template <typename T>
cudaError_t launch_refresh_brackets(const StageArgs<T> &a, cudaStream_t st);
template <typename T>
cudaError_t launch_diagnostics(const StageArgs<T> &a, double *partials, double *out,
                               cudaStream_t st);
cudaError_t launch_ctl_init(StepCtl *ctl, double t0, cudaStream_t st);
int diag_blocks(int nx, int ny);

}  // namespace swe
