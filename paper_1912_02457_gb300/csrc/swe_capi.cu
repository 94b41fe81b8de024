// swe_capi.cu -- host implementation of the libswe C ABI (include/swe.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/swe.h"
#include "swe_kernels.h"

using swe::StageArgs;
using swe::StepCtl;

namespace {

thread_local char g_cuda_err[256] = "";
swe_alloc_fn g_alloc = nullptr;
swe_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;

int cuda_fail(cudaError_t e) {
    snprintf(g_cuda_err, sizeof g_cuda_err, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return SWE_ERR_CUDA;
}

#define CK(x)                                    \
    do {                                         \
        cudaError_t _e = (x);                    \
        if (_e != cudaSuccess) return cuda_fail(_e); \
    } while (0)

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

}  // namespace

struct swe_domain {
    int nx = 0, ny = 0, prec = 0;
    size_t esz = 4;
    long long pitch = 0, cpitch = 0;   // elements
    double dx = 0, dy = 0;
    swe_params p{};
    int bc[4] = {0, 0, 0, 0};
    cudaStream_t stream = nullptr;
    swe_alloc_fn alloc = nullptr;
    swe_free_fn release = nullptr;
    void *alloc_ctx = nullptr;
    std::vector<void *> owned;
    void *q[2][3] = {{nullptr}};
    void *d1[3] = {nullptr};
    void *comp[3] = {nullptr};
    void *H = nullptr, *f = nullptr, *th = nullptr;
    double f_const = 0, th_const = 0;
    int cur = 0;
    StepCtl *ctl = nullptr;
    float *bnd = nullptr;
    double *bnd_t = nullptr;
    int bnd_n = 0, bnd_n1 = 0, bnd_n2 = 0;
    float *wind = nullptr;
    double *wind_t = nullptr;
    int wind_n = 0, wind_n1 = 0, wind_n2 = 0;
    double *diag_partials = nullptr;
    double *diag_out = nullptr;
    bool sticky_numeric = false;
    long long launches = 0;
    std::vector<cudaEvent_t> events;   // profiling pool, grown on demand

    bool fast() const { return prec != SWE_F64 && p.kernel == 0; }
    int parts() const { return fast() ? swe::fast_step_parts() : swe::ref_step_parts(); }

    void *dalloc(size_t bytes) {
        void *ptr = nullptr;
        if (alloc) {
            ptr = alloc(bytes, stream, alloc_ctx);
        } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            ptr = nullptr;
        }
        if (ptr) owned.push_back(ptr);
        return ptr;
    }
    void dfree(void *ptr) {
        if (!ptr) return;
        for (size_t k = 0; k < owned.size(); k++)
            if (owned[k] == ptr) { owned.erase(owned.begin() + (long)k); break; }
        if (release) release(ptr, stream, alloc_ctx);
        else cudaFree(ptr);
    }
    void free_all() {
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        events.clear();
        for (void *ptr : owned) {
            if (release) release(ptr, stream, alloc_ctx);
            else cudaFree(ptr);
        }
        owned.clear();
    }
    size_t plane_bytes() const { return (size_t)pitch * ny * esz; }
};

namespace {

template <typename T>
StageArgs<T> make_args(const swe_domain *d) {
    StageArgs<T> a;
    memset(&a, 0, sizeof a);
    a.nx = d->nx;
    a.ny = d->ny;
    a.pitch = d->pitch;
    a.cpitch = d->cpitch;
    a.dx = T(d->dx);
    a.dy = T(d->dy);
    a.inv_dx = T(1.0 / d->dx);
    a.inv_dy = T(1.0 / d->dy);
    a.kx = T(d->dx / (2.0 * d->p.g));
    a.ky = T(d->dy / (2.0 * d->p.g));
    a.g = T(d->p.g);
    a.kappa = T(d->p.kappa);
    a.half_inv_kappa = T(0.5 / d->p.kappa);
    a.tm = T(d->p.theta_mm);
    a.cd = T(d->p.cd);
    for (int e = 0; e < 4; e++) a.bc[e] = d->bc[e];
    a.H = (const T *)d->H;
    a.f = (const T *)d->f;
    a.th = (const T *)d->th;
    a.f_const = T(d->f_const);
    a.th_const = T(d->th_const);
    for (int k = 0; k < 3; k++) {
        a.qin[k] = (const T *)d->q[d->cur][k];
        a.qout[k] = (T *)d->q[1 - d->cur][k];
        a.d1[k] = (T *)d->d1[k];
        a.comp[k] = (T *)d->comp[k];
    }
    a.bnd = swe::ForcingDev{d->bnd, d->bnd_t, d->bnd_n, d->bnd_n1, d->bnd_n2};
    a.wind = swe::ForcingDev{d->wind, d->wind_t, d->wind_n, d->wind_n1, d->wind_n2};
    a.frs_width = d->p.frs_width;
    for (int k = 0; k < swe::kMaxFrs; k++)
        a.frs_alpha[k] = k < d->p.frs_width ? 1.0 - std::tanh((double)k / d->p.frs_d0) : 0.0;
    a.ctl = d->ctl;
    a.clk.courant = d->p.courant;
    a.clk.dt_fixed = d->p.dt_fixed;
    a.clk.dt_every = d->p.dt_update_every < 1 ? 1 : d->p.dt_update_every;
    a.clk.wind_uniform = (d->wind_n1 == 1 && d->wind_n2 == 1) ? 1 : 0;
    a.clk.rho_ratio = d->p.rho_air / d->p.rho_water;
    return a;
}

int upload_plane(swe_domain *d, void *dst, const void *src, int rows, int cols,
                 long long dpitch, int src_is_device) {
    CK(cudaMemcpy2DAsync(dst, (size_t)dpitch * d->esz, src, (size_t)cols * d->esz,
                         (size_t)cols * d->esz, (size_t)rows,
                         src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         d->stream));
    return SWE_OK;
}

int init_clock(swe_domain *d, double t, double dt, long long step) {
    cudaError_t e;
    if (d->prec == SWE_F64) e = swe::launch_init_clock(make_args<double>(d), d->stream, t, dt, step);
    else e = swe::launch_init_clock(make_args<float>(d), d->stream, t, dt, step);
    return e == cudaSuccess ? SWE_OK : cuda_fail(e);
}

int refresh_brackets(swe_domain *d) {
    cudaError_t e;
    if (d->prec == SWE_F64) e = swe::launch_refresh_brackets(make_args<double>(d), d->stream);
    else e = swe::launch_refresh_brackets(make_args<float>(d), d->stream);
    return e == cudaSuccess ? SWE_OK : cuda_fail(e);
}

int create_impl(const swe_domain_desc *dd, const swe_params *p, void *stream, swe_domain *d) {
    d->nx = dd->nx;
    d->ny = dd->ny;
    d->prec = dd->precision;
    d->esz = d->prec == SWE_F64 ? 8 : 4;
    d->dx = dd->dx;
    d->dy = dd->dy;
    d->p = *p;
    for (int e = 0; e < 4; e++) d->bc[e] = dd->bc[e];
    d->stream = (cudaStream_t)stream;
    d->alloc = g_alloc;
    d->release = g_free;
    d->alloc_ctx = g_alloc_ctx;
    // rows padded to 128 bytes; one spare row and column for the corner plane
    long long align = 128 / (long long)d->esz;
    d->pitch = round_up(d->nx, align);
    d->cpitch = round_up(d->nx + 1, align);
    const size_t pb = d->plane_bytes();
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++)
            if (!(d->q[b][k] = d->dalloc(pb))) return SWE_ERR_OOM;
    for (int k = 0; k < 3; k++)
        if (!(d->d1[k] = d->dalloc(pb))) return SWE_ERR_OOM;
    if (d->prec == SWE_F32_KAHAN)
        for (int k = 0; k < 3; k++) {
            if (!(d->comp[k] = d->dalloc(pb))) return SWE_ERR_OOM;
            CK(cudaMemsetAsync(d->comp[k], 0, pb, d->stream));
        }
    if (!(d->H = d->dalloc((size_t)d->cpitch * (d->ny + 1) * d->esz))) return SWE_ERR_OOM;
    if (dd->f && !(d->f = d->dalloc(pb))) return SWE_ERR_OOM;
    if (dd->theta && !(d->th = d->dalloc(pb))) return SWE_ERR_OOM;
    d->f_const = dd->f_const;
    d->th_const = dd->theta_const;
    if (!(d->ctl = (StepCtl *)d->dalloc(sizeof(StepCtl)))) return SWE_ERR_OOM;
    int nb = swe::diag_blocks(d->nx, d->ny);
    if (!(d->diag_partials = (double *)d->dalloc((size_t)nb * 2 * sizeof(double)))) return SWE_ERR_OOM;
    if (!(d->diag_out = (double *)d->dalloc(2 * sizeof(double)))) return SWE_ERR_OOM;

    const void *src[3] = {dd->eta, dd->hu, dd->hv};
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) {
            CK(cudaMemsetAsync(d->q[b][k], 0, pb, d->stream));
            int rc = upload_plane(d, d->q[b][k], src[k], d->ny, d->nx, d->pitch, dd->src_is_device);
            if (rc) return rc;
        }
    for (int k = 0; k < 3; k++) CK(cudaMemsetAsync(d->d1[k], 0, pb, d->stream));
    int rc = upload_plane(d, d->H, dd->H, d->ny + 1, d->nx + 1, d->cpitch, dd->src_is_device);
    if (rc) return rc;
    if (d->f && (rc = upload_plane(d, d->f, dd->f, d->ny, d->nx, d->pitch, dd->src_is_device))) return rc;
    if (d->th && (rc = upload_plane(d, d->th, dd->theta, d->ny, d->nx, d->pitch, dd->src_is_device))) return rc;
    cudaError_t e = swe::launch_ctl_init(d->ctl, p->t0, d->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    if ((rc = init_clock(d, p->t0, p->dt_fixed > 0 ? p->dt_fixed : 0.0, 0))) return rc;
    if (dd->src_is_device == 0) CK(cudaStreamSynchronize(d->stream));
    return SWE_OK;
}

int validate(const swe_domain_desc *d, const swe_params *p) {
    if (!d || !p) return SWE_ERR_INVALID_ARG;
    if (d->nx < 1 || d->ny < 1 || d->nx > 65536 || d->ny > 65536) return SWE_ERR_INVALID_ARG;
    if (!(d->dx > 0) || !(d->dy > 0)) return SWE_ERR_INVALID_ARG;
    if (d->precision < SWE_F32 || d->precision > SWE_F64) return SWE_ERR_INVALID_ARG;
    for (int e = 0; e < 4; e++)
        if (d->bc[e] != SWE_BC_WALL && d->bc[e] != SWE_BC_NESTED) return SWE_ERR_INVALID_ARG;
    if ((long long)d->nx * d->ny >= (1LL << 31)) return SWE_ERR_INVALID_ARG;
    // a nested edge mirrors the two cells next to it for the ghost statics
    if ((d->bc[2] == SWE_BC_NESTED || d->bc[3] == SWE_BC_NESTED) && d->nx < 2) return SWE_ERR_INVALID_ARG;
    if ((d->bc[0] == SWE_BC_NESTED || d->bc[1] == SWE_BC_NESTED) && d->ny < 2) return SWE_ERR_INVALID_ARG;
    if (!d->eta || !d->hu || !d->hv || !d->H) return SWE_ERR_INVALID_ARG;
    if (p->frs_width < 0 || p->frs_width > swe::kMaxFrs) return SWE_ERR_INVALID_ARG;
    if (!(p->g > 0) || !(p->kappa > 0) || !(p->courant > 0) || !(p->frs_d0 > 0)) return SWE_ERR_INVALID_ARG;
    if (p->cd < 0 || p->theta_mm < 1.0 || p->theta_mm > 2.0) return SWE_ERR_INVALID_ARG;
    if (p->dt_fixed < 0 || !(p->rho_water > 0) || p->rho_air < 0) return SWE_ERR_INVALID_ARG;
    if (p->kernel != 0 && p->kernel != 1) return SWE_ERR_INVALID_ARG;
    return SWE_OK;
}

void *plane_of(swe_domain *d, int field) {
    if (field >= SWE_ETA && field <= SWE_HV) return d->q[d->cur][field];
    if (field >= SWE_COMP_ETA && field <= SWE_COMP_HV) return d->comp[field - SWE_COMP_ETA];
    return nullptr;
}

}  // namespace

extern "C" {

int swe_abi_version(void) { return SWE_ABI_VERSION; }

const char *swe_last_cuda_error(void) { return g_cuda_err; }

const char *swe_status_string(int s) {
    switch (s) {
        case SWE_OK: return "ok";
        case SWE_ERR_INVALID_ARG: return "invalid argument";
        case SWE_ERR_OOM: return "out of memory";
        case SWE_ERR_CUDA: return "CUDA error";
        case SWE_ERR_NUMERIC: return "non-finite state or time step";
        case SWE_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

int swe_set_allocator(swe_alloc_fn alloc, swe_free_fn release, void *ctx) {
    if ((alloc == nullptr) != (release == nullptr)) return SWE_ERR_INVALID_ARG;
    g_alloc = alloc;
    g_free = release;
    g_alloc_ctx = ctx;
    return SWE_OK;
}

void swe_default_params(swe_params *p) {
    if (!p) return;
    p->g = 9.81;
    p->theta_mm = 1.3;
    p->kappa = 1e-2;
    p->cd = 0.0;
    p->courant = 0.8;
    p->frs_d0 = 2.5;
    p->frs_width = 10;
    p->dt_update_every = 1;
    p->dt_fixed = 0.0;
    p->rho_air = 1.225;
    p->rho_water = 1025.0;
    p->t0 = 0.0;
    p->kernel = 0;
}

int swe_create_domain(const swe_domain_desc *d, const swe_params *p, void *stream, swe_handle *out) {
    if (!out) return SWE_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = validate(d, p);
    if (rc) return rc;
    swe_domain *dom = new (std::nothrow) swe_domain();
    if (!dom) return SWE_ERR_OOM;
    rc = create_impl(d, p, stream, dom);
    if (rc) {
        cudaStreamSynchronize(dom->stream);
        dom->free_all();
        delete dom;
        return rc;
    }
    *out = dom;
    return SWE_OK;
}

int swe_set_forcing(swe_handle h, int kind, int n_frames, const double *times, const float *frames,
                    int n1, int n2) {
    if (!h || n_frames < 0 || (n_frames > 0 && (!times || !frames))) return SWE_ERR_INVALID_ARG;
    if (kind != SWE_FORCING_WIND && kind != SWE_FORCING_BOUNDARY) return SWE_ERR_INVALID_ARG;
    if (n_frames > 0 && (n1 < 1 || n2 < 1)) return SWE_ERR_INVALID_ARG;
    for (int k = 1; k < n_frames; k++)
        if (!(times[k] > times[k - 1])) return SWE_ERR_INVALID_ARG;
    size_t per = kind == SWE_FORCING_WIND ? (size_t)2 * n1 * n2 : (size_t)12 * (n1 + n2);
    float *nf = nullptr;
    double *nt = nullptr;
    if (n_frames > 0) {
        nf = (float *)h->dalloc(per * n_frames * sizeof(float));
        nt = (double *)h->dalloc((size_t)n_frames * sizeof(double));
        if (!nf || !nt) { h->dfree(nf); h->dfree(nt); return SWE_ERR_OOM; }
        CK(cudaMemcpyAsync(nf, frames, per * n_frames * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(nt, times, (size_t)n_frames * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    }
    // the old series may still be read by queued kernels: drain first
    CK(cudaStreamSynchronize(h->stream));
    if (kind == SWE_FORCING_WIND) {
        h->dfree(h->wind); h->dfree(h->wind_t);
        h->wind = nf; h->wind_t = nt; h->wind_n = n_frames; h->wind_n1 = n1; h->wind_n2 = n2;
    } else {
        h->dfree(h->bnd); h->dfree(h->bnd_t);
        h->bnd = nf; h->bnd_t = nt; h->bnd_n = n_frames; h->bnd_n1 = n1; h->bnd_n2 = n2;
    }
    int rc = refresh_brackets(h);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));
    return SWE_OK;
}

namespace {

int step_check(swe_handle h, int n_steps) {
    if (!h || n_steps < 0) return SWE_ERR_INVALID_ARG;
    if (h->sticky_numeric) return SWE_ERR_NUMERIC;
    if ((h->bc[0] == SWE_BC_NESTED || h->bc[1] == SWE_BC_NESTED || h->bc[2] == SWE_BC_NESTED ||
         h->bc[3] == SWE_BC_NESTED) && h->bnd_n == 0)
        return SWE_ERR_INVALID_ARG;
    return SWE_OK;
}

int launch_part(swe_handle h, int part) {
    cudaError_t e;
    if (h->prec == SWE_F64) e = swe::launch_step_ref_part(make_args<double>(h), h->stream, part, false);
    else if (h->fast()) e = swe::launch_step_fast_part(make_args<float>(h), h->stream, part, h->prec == SWE_F32_KAHAN);
    else e = swe::launch_step_ref_part(make_args<float>(h), h->stream, part, h->prec == SWE_F32_KAHAN);
    if (e != cudaSuccess) return cuda_fail(e);
    h->launches++;
    return SWE_OK;
}

}  // namespace

int swe_step(swe_handle h, int n_steps) {
    int rc = step_check(h, n_steps);
    if (rc) return rc;
    const int parts = h->parts();
    for (int s = 0; s < n_steps; s++) {
        for (int p = 0; p < parts; p++)
            if ((rc = launch_part(h, p))) return rc;
        h->cur ^= 1;
    }
    return SWE_OK;
}

int swe_launches_per_step(swe_handle h) {
    if (!h) return SWE_ERR_INVALID_ARG;
    return h->parts();
}

const char *swe_launch_name(swe_handle h, int part) {
    if (!h) return "";
    return h->fast() ? swe::fast_part_name(part) : swe::ref_part_name(part);
}

int swe_step_profiled(swe_handle h, int n_steps, float *ms, int capacity) {
    int rc = step_check(h, n_steps);
    if (rc) return rc;
    const int parts = h->parts();
    if (!ms || capacity < n_steps * parts) return SWE_ERR_INVALID_ARG;
    const size_t need = (size_t)2 * n_steps * parts;
    while (h->events.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        h->events.push_back(e);
    }
    size_t k = 0;
    for (int s = 0; s < n_steps; s++) {
        for (int p = 0; p < parts; p++) {
            CK(cudaEventRecord(h->events[k++], h->stream));
            if ((rc = launch_part(h, p))) return rc;
            CK(cudaEventRecord(h->events[k++], h->stream));
        }
        h->cur ^= 1;
    }
    CK(cudaEventSynchronize(h->events[need - 1]));
    for (size_t q = 0; q < need / 2; q++) CK(cudaEventElapsedTime(&ms[q], h->events[2 * q], h->events[2 * q + 1]));
    return SWE_OK;
}

int swe_read_state(swe_handle h, int field, void *dst, int dst_is_device) {
    if (!h || !dst) return SWE_ERR_INVALID_ARG;
    void *src = plane_of(h, field);
    if (!src) return field >= SWE_COMP_ETA && field <= SWE_COMP_HV ? SWE_ERR_UNSUPPORTED : SWE_ERR_INVALID_ARG;
    CK(cudaMemcpy2DAsync(dst, (size_t)h->nx * h->esz, src, (size_t)h->pitch * h->esz,
                         (size_t)h->nx * h->esz, (size_t)h->ny,
                         dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    if (!dst_is_device) CK(cudaStreamSynchronize(h->stream));
    return SWE_OK;
}

int swe_write_state(swe_handle h, int field, const void *src, int src_is_device) {
    if (!h || !src) return SWE_ERR_INVALID_ARG;
    if (field >= SWE_ETA && field <= SWE_HV) {
        for (int b = 0; b < 2; b++) {
            int rc = upload_plane(h, h->q[b][field], src, h->ny, h->nx, h->pitch, src_is_device);
            if (rc) return rc;
        }
        if (h->comp[field]) CK(cudaMemsetAsync(h->comp[field], 0, h->plane_bytes(), h->stream));
    } else if (field >= SWE_COMP_ETA && field <= SWE_COMP_HV) {
        if (!h->comp[field - SWE_COMP_ETA]) return SWE_ERR_UNSUPPORTED;
        int rc = upload_plane(h, h->comp[field - SWE_COMP_ETA], src, h->ny, h->nx, h->pitch, src_is_device);
        if (rc) return rc;
    } else {
        return SWE_ERR_INVALID_ARG;
    }
    if (!src_is_device) CK(cudaStreamSynchronize(h->stream));
    return SWE_OK;
}

int swe_set_clock(swe_handle h, double t, double dt, long long step) {
    if (!h || step < 0 || !std::isfinite(t)) return SWE_ERR_INVALID_ARG;
    return init_clock(h, t, dt, step);
}

int swe_get_info(swe_handle h, swe_info *out) {
    if (!h || !out) return SWE_ERR_INVALID_ARG;
    StepCtl c;
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(&c, h->ctl, sizeof c, cudaMemcpyDeviceToHost));
    out->t = c.t;
    out->dt = c.dt;
    out->step = c.step;
    out->error = c.err;
    out->error_cell = c.err_cell;
    out->error_step = c.err_step;
    out->max_speed = c.last_speed;
    out->launches = h->launches;
    if (c.err != 0) {
        h->sticky_numeric = true;
        return SWE_ERR_NUMERIC;
    }
    return SWE_OK;
}

int swe_diagnostics(swe_handle h, double out[2]) {
    if (!h || !out) return SWE_ERR_INVALID_ARG;
    cudaError_t e;
    if (h->prec == SWE_F64) e = swe::launch_diagnostics(make_args<double>(h), h->diag_partials, h->diag_out, h->stream);
    else e = swe::launch_diagnostics(make_args<float>(h), h->diag_partials, h->diag_out, h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    CK(cudaMemcpyAsync(out, h->diag_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return SWE_OK;
}

int swe_destroy_domain(swe_handle h) {
    if (!h) return SWE_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    h->free_all();
    delete h;
    return e == cudaSuccess ? SWE_OK : cuda_fail(e);
}

}  // extern "C"
