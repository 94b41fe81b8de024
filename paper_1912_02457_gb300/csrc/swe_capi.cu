// swe_capi.cu -- host implementation of the libswe C ABI (include/swe.h).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdlib>
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

int swe::record_cuda_error(cudaError_t e) { return cuda_fail(e); }

swe::TraceRange::TraceRange(const char *name) { nvtxRangePushA(name); }
swe::TraceRange::~TraceRange() { nvtxRangePop(); }

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
    StepCtl *ctl = nullptr;
    float *edge = nullptr;             // external edge state, two time levels (fast path)
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

    // graphs of kGraphSteps steps and of one step, captured on a private
    // stream and replayed on `stream`; every kernel reads the parity and
    // clock from the device, so a graph serves every step until the forcing
    // buffers change
    static constexpr int kGraphSteps = 16;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr, graph1 = nullptr;

    void drop_graph() {
        if (graph) cudaGraphExecDestroy(graph);
        if (graph1) cudaGraphExecDestroy(graph1);
        graph = graph1 = nullptr;
    }

    // the FP32 fast path: the domain's tiling and arguments, handed to the
    // stage kernel (the one batches use) with every launch
    swe::OneDomain one{};
    // per 28-column strip and row: does it hold a wet cell (the land mask
    // is fixed at creation); the work budget of the domain alone; the
    // device plans (warp items) per budget, kept until the domain is
    // destroyed (captured graphs and batch tables point at them)
    std::vector<unsigned char> wet;
    int budget = 0;
    struct ItemList { int budget; bool alone; int n; uint2 *dev; };
    std::vector<ItemList> item_lists;

    bool fast() const { return prec != SWE_F64 && p.kernel == 0; }
    int parts() const { return fast() ? swe::fast_step_parts(p.cfl_faces != 0) : swe::ref_step_parts(); }

    void *dalloc(size_t bytes) {
        void *ptr = nullptr;
        if (alloc) {
            ptr = alloc(bytes, stream, alloc_ctx);
        } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            ptr = nullptr;
        }
        if (ptr) {
            try {
                owned.push_back(ptr);
            } catch (...) {                      // no exception crosses the C ABI
                if (release) release(ptr, stream, alloc_ctx);
                else cudaFree(ptr);
                ptr = nullptr;
            }
        }
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
        drop_graph();
        if (capture_stream) cudaStreamDestroy(capture_stream);
        capture_stream = nullptr;
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
        a.q[0][k] = (T *)d->q[0][k];
        a.q[1][k] = (T *)d->q[1][k];
        a.d1[k] = (T *)d->d1[k];
        a.comp[k] = (T *)d->comp[k];
    }
    a.bnd = swe::ForcingDev{d->bnd, d->bnd_t, d->bnd_n, d->bnd_n1, d->bnd_n2};
    a.wind = swe::ForcingDev{d->wind, d->wind_t, d->wind_n, d->wind_n1, d->wind_n2};
    a.frs_width = d->p.frs_width;
    for (int k = 0; k < swe::kMaxFrs; k++) {
        a.frs_alpha[k] = k < d->p.frs_width ? 1.0 - std::tanh((double)k / d->p.frs_d0) : 0.0;
        a.frs_alpha_f[k] = (float)a.frs_alpha[k];
    }
    a.ctl = d->ctl;
    a.edge = d->edge;
    a.n_plane = d->pitch * d->ny;
    a.n_corner = d->cpitch * (d->ny + 1);
    a.n_edge = d->edge ? swe::edge_floats(d->nx, d->ny) : 0;
    a.n_bnd = (long long)d->bnd_n * 12 * (d->bnd_n1 + d->bnd_n2);
    a.n_wind = (long long)d->wind_n * 2 * d->wind_n1 * d->wind_n2;
#ifdef SWE_DEBUG_BOUNDS
    // test knob of the bounds-checked build: declare the last rows of every
    // state plane out of bounds (the allocation itself is untouched, so an
    // access the checks let through still lands inside it)
    if (const char *v = getenv("SWE_DEBUG_SHRINK_PLANE_ROWS")) a.n_plane -= atoll(v) * d->pitch;
#endif
    a.clk.courant = d->p.courant;
    a.clk.dt_fixed = d->p.dt_fixed;
    a.clk.dt_every = d->p.dt_update_every < 1 ? 1 : d->p.dt_update_every;
    a.clk.wind_uniform = (d->wind_n1 == 1 && d->wind_n2 == 1) ? 1 : 0;
    a.clk.rho_ratio = d->p.rho_air / d->p.rho_water;
    a.clk.fp32 = d->prec == SWE_F64 ? 0 : 1;
    a.clk.cfl_faces = d->p.cfl_faces;
    // a window of a larger domain, or the whole domain
    const bool win = d->p.whole_nx > 0;
    a.clk.split = win ? 1 : 0;
    a.off_x = win ? d->p.window_x0 : 0;
    a.off_y = win ? d->p.window_y0 : 0;
    a.gnx = win ? d->p.whole_nx : d->nx;
    a.gny = win ? d->p.whole_ny : d->ny;
    a.own_x0 = win ? d->p.own_x0 : 0;
    a.own_x1 = win ? d->p.own_x1 : d->nx;
    a.own_y0 = win ? d->p.own_y0 : 0;
    a.own_y1 = win ? d->p.own_y1 : d->ny;
    return a;
}

// The wet flags of the fast path's strips (once per domain).
int ensure_wet(swe_domain *d) {
    if (!d->wet.empty()) return SWE_OK;
    const size_t n = (size_t)swe::fast_strips(d->nx) * d->ny;
    try {
        d->wet.resize(n);
    } catch (...) {
        return SWE_ERR_OOM;
    }
    unsigned char *dev = (unsigned char *)d->dalloc(n);
    if (!dev) { d->wet.clear(); return SWE_ERR_OOM; }
    cudaError_t e = swe::launch_wet_strips((const float *)d->H, d->cpitch, d->nx, d->ny, dev, d->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d->wet.data(), dev, n, cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    d->dfree(dev);
    if (e != cudaSuccess) { d->wet.clear(); return cuda_fail(e); }
    if (d->p.whole_nx > 0) {
        // a window plans its own rows only, and no strip without an own
        // column: those cells are never written, the halo exchange fills
        // them (the halo columns of the strips it does march are written
        // and overwritten, and left out of its CFL maximum)
        const int strips = swe::fast_strips(d->nx), S = swe::kStripColumns;
        for (int st = 0; st < strips; st++) {
            const bool cols = st * S < d->p.own_x1 && st * S + S > d->p.own_x0;
            for (int j = 0; j < d->ny; j++)
                if (!cols || j < d->p.own_y0 || j >= d->p.own_y1) d->wet[(size_t)st * d->ny + j] = 0;
        }
    }
    return SWE_OK;
}

// The device plan of the fast path for a work budget, for the domain
// launched alone or in a batch (built once).
int domain_items(swe_domain *d, int budget, bool alone, const uint2 **dev, int *n) {
    for (const auto &l : d->item_lists)
        if (l.budget == budget && l.alone == alone) { *dev = l.dev; *n = l.n; return SWE_OK; }
    int rc = ensure_wet(d);
    if (rc) return rc;
    std::vector<uint2> items;
    try {
        swe::fast_plan(d->nx, d->ny, d->wet.data(), d->bc, d->p.frs_width, budget, alone, items);
    } catch (...) {
        return SWE_ERR_OOM;
    }
    uint2 *p = (uint2 *)d->dalloc(items.size() * sizeof(uint2));
    if (!p) return SWE_ERR_OOM;
    cudaError_t e = cudaMemcpyAsync(p, items.data(), items.size() * sizeof(uint2), cudaMemcpyHostToDevice,
                                    d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) { d->dfree(p); return cuda_fail(e); }
    try {
        d->item_lists.push_back({budget, alone, (int)items.size(), p});
    } catch (...) {
        d->dfree(p);
        return SWE_ERR_OOM;
    }
    *dev = p;
    *n = (int)items.size();
    return SWE_OK;
}

// Arguments of the fast path for a work budget, its plan and the blocks a
// launch over it takes.
int fast_args(swe_domain *d, int budget, bool alone, StageArgs<float> *a, int *tiles) {
    const uint2 *items = nullptr;
    int n = 0;
    int rc = domain_items(d, budget, alone, &items, &n);
    if (rc) return rc;
    *a = make_args<float>(d);
    a->items = items;
    a->n_items = n;
    *tiles = swe::fast_tiles(n);
    return SWE_OK;
}

// (Re)compute the fast path's tiling and launch arguments (after creation
// and whenever the forcing buffers change).
int upload_table(swe_domain *d) {
    if (!d->fast()) return SWE_OK;
    int rc = ensure_wet(d);
    if (rc) return rc;
    if (!d->budget) {
        try {
            d->budget = swe::fast_budget(d->nx, d->ny, d->wet.data(), d->bc, d->p.frs_width);
        } catch (...) {
            return SWE_ERR_OOM;                     // no exception crosses the C ABI
        }
    }
    d->one.rows = d->budget / swe::kPlanUnit;
    d->one.strips = swe::fast_strips(d->nx);
    return fast_args(d, d->budget, true, &d->one.args, &d->one.tiles);
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
    // the fast path reads the ghosts of the current time level from the edge buffer
    if (e == cudaSuccess && d->fast()) e = swe::launch_edge_fill(make_args<float>(d), d->stream);
    return e == cudaSuccess ? SWE_OK : cuda_fail(e);
}

int refresh_brackets(swe_domain *d) {
    cudaError_t e;
    if (d->prec == SWE_F64) e = swe::launch_refresh_brackets(make_args<double>(d), d->stream);
    else e = swe::launch_refresh_brackets(make_args<float>(d), d->stream);
    if (e == cudaSuccess && d->fast()) e = swe::launch_edge_fill(make_args<float>(d), d->stream);
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
    if (d->cpitch * (d->ny + 1) >= (1LL << 31)) return SWE_ERR_INVALID_ARG;   // 32-bit offsets
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
    if (d->fast()) {
        const size_t eb = (size_t)swe::edge_floats(d->nx, d->ny) * sizeof(float);
        if (!(d->edge = (float *)d->dalloc(eb))) return SWE_ERR_OOM;
        CK(cudaMemsetAsync(d->edge, 0, eb, d->stream));
    }
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
    if ((rc = upload_table(d))) return rc;
    if (dd->src_is_device == 0) CK(cudaStreamSynchronize(d->stream));
    return SWE_OK;
}

int validate(const swe_domain_desc *d, const swe_params *p) {
    if (!d || !p) return SWE_ERR_INVALID_ARG;
    if (d->nx < 1 || d->ny < 1 || d->nx > 65536 || d->ny > 65536) return SWE_ERR_INVALID_ARG;
    if (!(d->dx > 0) || !(d->dy > 0)) return SWE_ERR_INVALID_ARG;
    if (d->precision < SWE_F32 || d->precision > SWE_F64) return SWE_ERR_INVALID_ARG;
    for (int e = 0; e < 4; e++)
        if (d->bc[e] != SWE_BC_WALL && d->bc[e] != SWE_BC_NESTED && d->bc[e] != SWE_BC_PERIODIC)
            return SWE_ERR_INVALID_ARG;
    // periodic edges pair up (S with N, W with E)
    if ((d->bc[0] == SWE_BC_PERIODIC) != (d->bc[1] == SWE_BC_PERIODIC) ||
        (d->bc[2] == SWE_BC_PERIODIC) != (d->bc[3] == SWE_BC_PERIODIC))
        return SWE_ERR_INVALID_ARG;
    if ((long long)d->nx * d->ny >= (1LL << 31)) return SWE_ERR_INVALID_ARG;
    // a nested edge mirrors the two cells next to it for the ghost statics
    if ((d->bc[2] == SWE_BC_NESTED || d->bc[3] == SWE_BC_NESTED) && d->nx < 2) return SWE_ERR_INVALID_ARG;
    if ((d->bc[0] == SWE_BC_NESTED || d->bc[1] == SWE_BC_NESTED) && d->ny < 2) return SWE_ERR_INVALID_ARG;
    if (!d->eta || !d->hu || !d->hv || !d->H) return SWE_ERR_INVALID_ARG;
    // a periodic axis needs a corner plane whose last line repeats its first
    // (checked where the plane is host memory)
    if (!d->src_is_device) {
        const size_t w = (size_t)d->nx + 1;
        if (d->precision == SWE_F64) {
            const double *H = static_cast<const double *>(d->H);
            if (d->bc[2] == SWE_BC_PERIODIC)
                for (int j = 0; j <= d->ny; j++)
                    if (H[j * w] != H[j * w + d->nx]) return SWE_ERR_INVALID_ARG;
            if (d->bc[0] == SWE_BC_PERIODIC)
                for (int i = 0; i <= d->nx; i++)
                    if (H[i] != H[(size_t)d->ny * w + i]) return SWE_ERR_INVALID_ARG;
        } else {
            const float *H = static_cast<const float *>(d->H);
            if (d->bc[2] == SWE_BC_PERIODIC)
                for (int j = 0; j <= d->ny; j++)
                    if (H[j * w] != H[j * w + d->nx]) return SWE_ERR_INVALID_ARG;
            if (d->bc[0] == SWE_BC_PERIODIC)
                for (int i = 0; i <= d->nx; i++)
                    if (H[i] != H[(size_t)d->ny * w + i]) return SWE_ERR_INVALID_ARG;
        }
    }
    if (p->frs_width < 0 || p->frs_width > swe::kMaxFrs) return SWE_ERR_INVALID_ARG;
    if (!(p->g > 0) || !(p->kappa > 0) || !(p->courant > 0) || !(p->frs_d0 > 0)) return SWE_ERR_INVALID_ARG;
    if (p->cd < 0 || p->theta_mm < 1.0 || p->theta_mm > 2.0) return SWE_ERR_INVALID_ARG;
    if (p->dt_fixed < 0 || !(p->rho_water > 0) || p->rho_air < 0) return SWE_ERR_INVALID_ARG;
    if (p->kernel != 0 && p->kernel != 1) return SWE_ERR_INVALID_ARG;
    if (p->cfl_faces != 0 && p->cfl_faces != 1) return SWE_ERR_INVALID_ARG;
    if (p->cfl_faces && (d->precision == SWE_F64 || p->kernel != 0)) return SWE_ERR_UNSUPPORTED;
    // a window of a larger domain: inside it, with its own cells inside the window
    if (p->whole_nx == 0 && p->whole_ny == 0) {
        if (p->window_x0 || p->window_y0 || p->own_x0 || p->own_x1 || p->own_y0 || p->own_y1)
            return SWE_ERR_INVALID_ARG;
    } else {
        if (p->whole_nx < 1 || p->whole_ny < 1 || p->window_x0 < 0 || p->window_y0 < 0 ||
            (long long)p->window_x0 + d->nx > p->whole_nx || (long long)p->window_y0 + d->ny > p->whole_ny ||
            p->own_x0 < 0 || p->own_x0 >= p->own_x1 || p->own_x1 > d->nx ||
            p->own_y0 < 0 || p->own_y0 >= p->own_y1 || p->own_y1 > d->ny)
            return SWE_ERR_INVALID_ARG;
        for (int e = 0; e < 4; e++)
            if (d->bc[e] == SWE_BC_PERIODIC) return SWE_ERR_UNSUPPORTED;
        if (d->precision == SWE_F64 || p->kernel != 0 || p->cfl_faces) return SWE_ERR_UNSUPPORTED;
    }
    return SWE_OK;
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
    p->cfl_faces = 0;
    p->window_x0 = p->window_y0 = p->whole_nx = p->whole_ny = 0;
    p->own_x0 = p->own_x1 = p->own_y0 = p->own_y1 = 0;
}

int swe_create_domain(const swe_domain_desc *d, const swe_params *p, void *stream, swe_handle *out) {
    swe::TraceRange trace("swe_create_domain");
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
    swe::TraceRange trace("swe_set_forcing");
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
    h->drop_graph();
    if (kind == SWE_FORCING_WIND) {
        h->dfree(h->wind); h->dfree(h->wind_t);
        h->wind = nf; h->wind_t = nt; h->wind_n = n_frames; h->wind_n1 = n1; h->wind_n2 = n2;
    } else {
        h->dfree(h->bnd); h->dfree(h->bnd_t);
        h->bnd = nf; h->bnd_t = nt; h->bnd_n = n_frames; h->bnd_n1 = n1; h->bnd_n2 = n2;
    }
    int rc = refresh_brackets(h);
    if (rc) return rc;
    if ((rc = upload_table(h))) return rc;      // new forcing pointers
    CK(cudaStreamSynchronize(h->stream));
    return SWE_OK;
}

namespace {

int split_step_check(swe_handle h, int n_steps);

int step_check(swe_handle h, int n_steps) {
    // a window's clock advances only with its sub-domains (swe_split_step)
    if (h && h->p.whole_nx > 0) return SWE_ERR_UNSUPPORTED;
    return split_step_check(h, n_steps);
}

int split_step_check(swe_handle h, int n_steps) {
    if (!h || n_steps < 0) return SWE_ERR_INVALID_ARG;
    if (h->sticky_numeric) return SWE_ERR_NUMERIC;
    if ((h->bc[0] == SWE_BC_NESTED || h->bc[1] == SWE_BC_NESTED || h->bc[2] == SWE_BC_NESTED ||
         h->bc[3] == SWE_BC_NESTED) && h->bnd_n == 0)
        return SWE_ERR_INVALID_ARG;
    return SWE_OK;
}

int launch_part_on(swe_handle h, int part, cudaStream_t st) {
    cudaError_t e;
    if (h->prec == SWE_F64) e = swe::launch_step_ref_part(make_args<double>(h), st, part, false);
    else if (h->fast()) e = swe::launch_domain_stage(h->one, h->p.cfl_faces ? part : part + 1, st);
    else e = swe::launch_step_ref_part(make_args<float>(h), st, part, h->prec == SWE_F32_KAHAN);
    if (e != cudaSuccess) return cuda_fail(e);
    return SWE_OK;
}

int launch_part(swe_handle h, int part) {
    int rc = launch_part_on(h, part, h->stream);
    if (!rc) h->launches++;
    return rc;
}

int ensure_graph(swe_handle h, int steps, cudaGraphExec_t *out) {
    if (*out) return SWE_OK;
    if (!h->capture_stream) CK(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal));
    int rc = SWE_OK;
    for (int s = 0; s < steps && !rc; s++)
        for (int p = 0; p < h->parts() && !rc; p++) rc = launch_part_on(h, p, h->capture_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->capture_stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { *out = nullptr; return cuda_fail(e); }
    return SWE_OK;
}

}  // namespace

int swe_step(swe_handle h, int n_steps) {
    swe::TraceRange trace("swe_step");
    int rc = step_check(h, n_steps);
    if (rc) return rc;
    const int parts = h->parts();
    const int G = swe_domain::kGraphSteps;
    if (n_steps >= G) {
        if ((rc = ensure_graph(h, G, &h->graph))) return rc;
        for (; n_steps >= G; n_steps -= G) {
            CK(cudaGraphLaunch(h->graph, h->stream));
            h->launches += (long long)G * parts;
        }
    }
    // the remaining steps replay the one-step graph (its launches follow
    // each other without a host round trip between them)
    if (n_steps > 0 && (rc = ensure_graph(h, 1, &h->graph1))) return rc;
    for (; n_steps > 0; n_steps--) {
        CK(cudaGraphLaunch(h->graph1, h->stream));
        h->launches += parts;
    }
    return SWE_OK;
}

int swe_launches_per_step(swe_handle h) {
    if (!h) return SWE_ERR_INVALID_ARG;
    return h->parts();
}

const char *swe_launch_name(swe_handle h, int part) {
    if (!h) return "";
    return h->fast() ? swe::fast_part_name(part, h->p.cfl_faces != 0) : swe::ref_part_name(part);
}

int swe_step_profiled(swe_handle h, int n_steps, float *ms, int capacity) {
    swe::TraceRange trace("swe_step_profiled");
    int rc = step_check(h, n_steps);
    if (rc) return rc;
    const int parts = h->parts();
    if (!ms || capacity < n_steps * parts) return SWE_ERR_INVALID_ARG;
    const size_t need = (size_t)2 * n_steps * parts;
    while (h->events.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        try {
            h->events.push_back(e);
        } catch (...) {
            cudaEventDestroy(e);
            return SWE_ERR_OOM;
        }
    }
    size_t k = 0;
    for (int s = 0; s < n_steps; s++) {
        for (int p = 0; p < parts; p++) {
            CK(cudaEventRecord(h->events[k++], h->stream));
            if ((rc = launch_part(h, p))) return rc;
            CK(cudaEventRecord(h->events[k++], h->stream));
        }
    }
    CK(cudaEventSynchronize(h->events[need - 1]));
    for (size_t q = 0; q < need / 2; q++) CK(cudaEventElapsedTime(&ms[q], h->events[2 * q], h->events[2 * q + 1]));
    return SWE_OK;
}

int swe_read_state(swe_handle h, int field, void *dst, int dst_is_device) {
    swe::TraceRange trace("swe_read_state");
    if (!h || !dst) return SWE_ERR_INVALID_ARG;
    const void *src = nullptr;
    if (field >= SWE_COMP_ETA && field <= SWE_COMP_HV) {
        src = h->comp[field - SWE_COMP_ETA];
        if (!src) return SWE_ERR_UNSUPPORTED;
    } else if (field < SWE_ETA || field > SWE_HV) {
        return SWE_ERR_INVALID_ARG;
    }
    if (src) {
        CK(cudaMemcpy2DAsync(dst, (size_t)h->nx * h->esz, src, (size_t)h->pitch * h->esz,
                             (size_t)h->nx * h->esz, (size_t)h->ny,
                             dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    } else if (dst_is_device) {
        // the current buffer is known only to the device: copy by kernel
        cudaError_t e = h->prec == SWE_F64
            ? swe::launch_read_plane<double>(h->ctl, (const double *)h->q[0][field], (const double *)h->q[1][field],
                                             h->pitch, h->nx, h->ny, (double *)dst, h->stream)
            : swe::launch_read_plane<float>(h->ctl, (const float *)h->q[0][field], (const float *)h->q[1][field],
                                            h->pitch, h->nx, h->ny, (float *)dst, h->stream);
        if (e != cudaSuccess) return cuda_fail(e);
    } else {
        int par = 0;
        CK(cudaStreamSynchronize(h->stream));
        CK(cudaMemcpy(&par, &h->ctl->parity, sizeof par, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy2D(dst, (size_t)h->nx * h->esz, h->q[par & 1][field], (size_t)h->pitch * h->esz,
                        (size_t)h->nx * h->esz, (size_t)h->ny, cudaMemcpyDeviceToHost));
    }
    if (!dst_is_device) CK(cudaStreamSynchronize(h->stream));
    return SWE_OK;
}

int swe_set_end_time(swe_handle h, double t_end) {
    if (!h || !(t_end >= 0.0) || !std::isfinite(t_end)) return SWE_ERR_INVALID_ARG;
    cudaError_t e = swe::launch_set_end(h->ctl, t_end, h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    return refresh_brackets(h);
}

int swe_write_state(swe_handle h, int field, const void *src, int src_is_device) {
    swe::TraceRange trace("swe_write_state");
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
    out->done = c.done;
    out->t_end = c.t_end;
    if (c.err != 0) {
        h->sticky_numeric = true;
        return c.err == swe::ERR_BOUNDS ? SWE_ERR_BOUNDS : SWE_ERR_NUMERIC;
    }
    return SWE_OK;
}

int swe_diagnostics(swe_handle h, double out[2]) {
    swe::TraceRange trace("swe_diagnostics");
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

// ===========================================================================
// batches: many FP32 domains advanced by one launch per stage

struct swe_batch {
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    int cap = 0;
    std::vector<swe_handle> doms;
    std::vector<int> budget;        // work budget per domain (swe::kPlanUnit per row)
    int rows_choice = 0;            // 0: autotune on the next long step
    bool tuned = false;
    // device tables (capacity `cap`)
    swe::StageArgs<float> *d_args = nullptr;
    int *d_tile_start = nullptr, *d_grid_x = nullptr, *d_rows = nullptr, *d_n = nullptr;
    int *d_tile_dom = nullptr;      // domain of each tile (capacity tile_dom_cap)
    int tile_dom_cap = 0;
    int *d_done = nullptr;
    double *d_t = nullptr;
    int blocks = 0;
    bool gridded = false;           // some domain has gridded wind (which stage kernel)
    cudaGraphExec_t graph = nullptr;
    static constexpr int kGraphSteps = 8;
    long long launches = 0;
    std::vector<cudaEvent_t> events;
};

namespace {

const int kTuneRows[] = {8, 16, 32, 64};

int batch_upload_impl(swe_batch *b);

// (no exception crosses the C ABI: a failed host allocation is SWE_ERR_OOM)
int batch_upload(swe_batch *b) {
    try {
        return batch_upload_impl(b);
    } catch (...) {
        return SWE_ERR_OOM;
    }
}

int batch_upload_impl(swe_batch *b) {
    const int n = (int)b->doms.size();
    std::vector<swe::StageArgs<float>> args(n);
    std::vector<int> start(n + 1, 0), gx(n), rows(n);
    for (int k = 0; k < n; k++) {
        rows[k] = b->budget[k] / swe::kPlanUnit;
        int tiles = 0;
        int rc = fast_args(b->doms[k], b->budget[k], false, &args[k], &tiles);
        if (rc) return rc;
        gx[k] = swe::fast_strips(b->doms[k]->nx);
        start[k + 1] = start[k] + tiles;
    }
    // synchronous copies: the graph reads these tables; nothing is in flight
    CK(cudaStreamSynchronize(b->stream));
    if (n) {
        CK(cudaMemcpy(b->d_args, args.data(), sizeof(args[0]) * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b->d_grid_x, gx.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(b->d_rows, rows.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(b->d_tile_start, start.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(b->d_n, &n, sizeof(int), cudaMemcpyHostToDevice));
    // one block per tile: a new tile count (or table) needs a new graph,
    // and so does a change of the stage kernel (gridded wind or not)
    const int blocks = start[n] > 0 ? start[n] : 1;
    bool gridded = false;
    for (int k = 0; k < n; k++) gridded |= args[k].wind.n > 0 && !args[k].clk.wind_uniform;
    bool regraph = blocks != b->blocks || gridded != b->gridded;
    b->gridded = gridded;
    if (start[n] > b->tile_dom_cap) {
        int *p = nullptr;
        CK(cudaMalloc(&p, sizeof(int) * (size_t)start[n]));
        cudaFree(b->d_tile_dom);
        b->d_tile_dom = p;
        b->tile_dom_cap = start[n];
        regraph = true;
    }
    if (start[n] > 0) {
        std::vector<int> dom((size_t)start[n]);
        for (int k = 0; k < n; k++)
            for (int t = start[k]; t < start[k + 1]; t++) dom[(size_t)t] = k;
        CK(cudaMemcpy(b->d_tile_dom, dom.data(), sizeof(int) * dom.size(), cudaMemcpyHostToDevice));
    }
    if (regraph) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->blocks = blocks;
    }
    return SWE_OK;
}

swe::BatchTable batch_table(const swe_batch *b) {
    swe::BatchTable t;
    t.args = b->d_args;
    t.tile_start = b->d_tile_start;
    t.tile_dom = b->d_tile_dom;
    t.grid_x = b->d_grid_x;
    t.rows = b->d_rows;
    t.n_domains = b->d_n;
    return t;
}

int batch_launch_step(swe_batch *b, cudaStream_t st) {
    for (int stage = 1; stage <= 2; stage++) {
        cudaError_t e = swe::launch_batch_stage(batch_table(b), b->blocks, stage, b->gridded, st);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return SWE_OK;
}

int batch_ensure_graph(swe_batch *b) {
    if (b->graph) return SWE_OK;
    if (!b->capture_stream) CK(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
    int rc = SWE_OK;
    for (int s = 0; s < swe_batch::kGraphSteps && !rc; s++) rc = batch_launch_step(b, b->capture_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->capture_stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->graph = nullptr; return cuda_fail(e); }
    return SWE_OK;
}

int batch_set_rows_all(swe_batch *b, int rows) {
    for (size_t k = 0; k < b->doms.size(); k++)
        b->budget[k] = rows > 0 ? rows * swe::kPlanUnit : b->doms[k]->budget;
    return batch_upload(b);
}

// Autotuner: time two batch steps with every candidate tile height and keep
// the fastest. The steps are real steps of the forecast (the result does
// not depend on the tiling), so tuning costs no extra simulation.
int batch_tune(swe_batch *b, int *steps_used) {
    *steps_used = 0;
    if (b->doms.empty()) return SWE_OK;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int best_rows = kTuneRows[0];
    for (int rows : kTuneRows) {
        int rc = batch_set_rows_all(b, rows);
        if (!rc) rc = batch_launch_step(b, b->stream);      // settle
        if (!rc) CK(cudaEventRecord(e0, b->stream));
        if (!rc) rc = batch_launch_step(b, b->stream);
        if (!rc) CK(cudaEventRecord(e1, b->stream));
        if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        *steps_used += 2;
        b->launches += 4;
        if (ms < best) { best = ms; best_rows = rows; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->rows_choice = best_rows;
    b->tuned = true;
    return batch_set_rows_all(b, best_rows);
}

}  // namespace

extern "C" {

int swe_batch_create(void *stream, int max_domains, swe_batch_handle *out) {
    if (!out || max_domains < 1 || max_domains > (1 << 20)) return SWE_ERR_INVALID_ARG;
    *out = nullptr;
    swe_batch *b = new (std::nothrow) swe_batch();
    if (!b) return SWE_ERR_OOM;
    b->stream = (cudaStream_t)stream;
    b->cap = max_domains;
    bool ok = cudaMalloc(&b->d_args, sizeof(swe::StageArgs<float>) * max_domains) == cudaSuccess &&
              cudaMalloc(&b->d_tile_start, sizeof(int) * (max_domains + 1)) == cudaSuccess &&
              cudaMalloc(&b->d_grid_x, sizeof(int) * max_domains) == cudaSuccess &&
              cudaMalloc(&b->d_rows, sizeof(int) * max_domains) == cudaSuccess &&
              cudaMalloc(&b->d_n, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&b->d_done, sizeof(int) * max_domains) == cudaSuccess &&
              cudaMalloc(&b->d_t, sizeof(double) * max_domains) == cudaSuccess;
    if (ok) ok = batch_upload(b) == SWE_OK;
    if (!ok) {
        cudaFree(b->d_args); cudaFree(b->d_tile_start); cudaFree(b->d_grid_x); cudaFree(b->d_rows);
        cudaFree(b->d_n); cudaFree(b->d_done); cudaFree(b->d_t); cudaFree(b->d_tile_dom);
        delete b;
        return SWE_ERR_OOM;
    }
    *out = b;
    return SWE_OK;
}

int swe_batch_add(swe_batch_handle b, swe_handle d) {
    if (!b || !d) return SWE_ERR_INVALID_ARG;
    if (d->prec == SWE_F64 || !d->fast() || d->p.cfl_faces || d->p.whole_nx > 0) return SWE_ERR_UNSUPPORTED;
    if ((int)b->doms.size() >= b->cap) return SWE_ERR_INVALID_ARG;
    for (swe_handle x : b->doms)
        if (x == d) return SWE_ERR_INVALID_ARG;
    if (step_check(d, 0)) return step_check(d, 0);
    CK(cudaStreamSynchronize(d->stream));      // creation and uploads finished
    try {
        b->doms.push_back(d);
        b->budget.push_back(b->rows_choice > 0 ? b->rows_choice * swe::kPlanUnit : d->budget);
    } catch (...) {
        if (b->doms.size() > b->budget.size()) b->doms.pop_back();
        return SWE_ERR_OOM;
    }
    return batch_upload(b);
}

int swe_batch_remove(swe_batch_handle b, swe_handle d) {
    if (!b || !d) return SWE_ERR_INVALID_ARG;
    for (size_t k = 0; k < b->doms.size(); k++)
        if (b->doms[k] == d) {
            b->doms.erase(b->doms.begin() + (long)k);
            b->budget.erase(b->budget.begin() + (long)k);
            return batch_upload(b);             // also drains the batch stream
        }
    return SWE_ERR_INVALID_ARG;
}

int swe_batch_size(swe_batch_handle b) { return b ? (int)b->doms.size() : SWE_ERR_INVALID_ARG; }

int swe_batch_set_rows(swe_batch_handle b, int rows) {
    if (!b || rows < 0 || rows > 1024) return SWE_ERR_INVALID_ARG;
    b->rows_choice = rows;
    b->tuned = rows > 0;
    return batch_set_rows_all(b, rows);
}

int swe_batch_rows(swe_batch_handle b) { return b ? b->rows_choice : SWE_ERR_INVALID_ARG; }

int swe_batch_step(swe_batch_handle b, int n_steps) {
    swe::TraceRange trace("swe_batch_step");
    if (!b || n_steps < 0) return SWE_ERR_INVALID_ARG;
    if (b->doms.empty() || n_steps == 0) return SWE_OK;
    int rc;
    const int ncand = (int)(sizeof kTuneRows / sizeof kTuneRows[0]);
    if (!b->tuned && n_steps >= 4 * ncand) {
        int used = 0;
        if ((rc = batch_tune(b, &used))) return rc;
        n_steps -= used;
    }
    const int G = swe_batch::kGraphSteps;
    if (n_steps >= G) {
        if ((rc = batch_ensure_graph(b))) return rc;
        for (; n_steps >= G; n_steps -= G) {
            CK(cudaGraphLaunch(b->graph, b->stream));
            b->launches += 2LL * G;
        }
    }
    for (; n_steps > 0; n_steps--) {
        if ((rc = batch_launch_step(b, b->stream))) return rc;
        b->launches += 2;
    }
    return SWE_OK;
}

int swe_batch_step_serial(swe_batch_handle b, int n_steps) {
    swe::TraceRange trace("swe_batch_step_serial");
    if (!b || n_steps < 0) return SWE_ERR_INVALID_ARG;
    for (int s = 0; s < n_steps; s++)
        for (swe_handle d : b->doms)
            for (int p = 0; p < d->parts(); p++) {
                int rc = launch_part_on(d, p, b->stream);
                if (rc) return rc;
                b->launches++;
            }
    return SWE_OK;
}

int swe_batch_sync(swe_batch_handle b) {
    if (!b) return SWE_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(b->stream));
    return SWE_OK;
}

int swe_batch_poll(swe_batch_handle b, int *done, double *t, int capacity) {
    if (!b || capacity < (int)b->doms.size()) return SWE_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(b->stream));
    for (size_t k = 0; k < b->doms.size(); k++) {
        swe::StepCtl c;
        CK(cudaMemcpy(&c, b->doms[k]->ctl, sizeof c, cudaMemcpyDeviceToHost));
        if (done) done[k] = c.done;
        if (t) t[k] = c.t;
    }
    return SWE_OK;
}

long long swe_batch_launches(swe_batch_handle b) { return b ? b->launches : SWE_ERR_INVALID_ARG; }

int swe_batch_destroy(swe_batch_handle b) {
    if (!b) return SWE_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    cudaFree(b->d_args); cudaFree(b->d_tile_start); cudaFree(b->d_grid_x); cudaFree(b->d_rows);
    cudaFree(b->d_n); cudaFree(b->d_done); cudaFree(b->d_t); cudaFree(b->d_tile_dom);
    delete b;
    return e == cudaSuccess ? SWE_OK : cuda_fail(e);
}

// ---------------------------------------------------------------------------
// domain decomposition on one device

namespace {

struct Box { long long x0, x1, y0, y1; };

Box own_box(const swe_domain *d) {
    return {d->p.window_x0 + (long long)d->p.own_x0, d->p.window_x0 + (long long)d->p.own_x1,
            d->p.window_y0 + (long long)d->p.own_y0, d->p.window_y0 + (long long)d->p.own_y1};
}

Box window_box(const swe_domain *d) {
    return {d->p.window_x0, d->p.window_x0 + (long long)d->nx, d->p.window_y0, d->p.window_y0 + (long long)d->ny};
}

bool overlap(const Box &a, const Box &b, Box *out) {
    Box o{std::max(a.x0, b.x0), std::min(a.x1, b.x1), std::max(a.y0, b.y0), std::min(a.y1, b.y1)};
    if (o.x0 >= o.x1 || o.y0 >= o.y1) return false;
    if (out) *out = o;
    return true;
}

long long area(const Box &b) { return (b.x1 - b.x0) * (b.y1 - b.y0); }

// The sub-domains form a decomposition: windows of one whole domain with
// the same cell size, precision, stream and clock parameters, own cells
// that tile the whole domain once, every halo cell owned by another one.
int split_check(const swe_handle *doms, int n) {
    if (!doms || n < 1 || n > swe::kSplitMax) return SWE_ERR_INVALID_ARG;
    const swe_domain *a = doms[0];
    for (int i = 0; i < n; i++) {
        const swe_domain *d = doms[i];
        if (!d || d->p.whole_nx <= 0 || !d->fast()) return SWE_ERR_INVALID_ARG;
        for (int j = 0; j < i; j++)
            if (doms[j] == d) return SWE_ERR_INVALID_ARG;
        if (d->p.whole_nx != a->p.whole_nx || d->p.whole_ny != a->p.whole_ny || d->stream != a->stream ||
            d->prec != a->prec || d->dx != a->dx || d->dy != a->dy || d->p.courant != a->p.courant ||
            d->p.dt_fixed != a->p.dt_fixed || d->p.dt_update_every != a->p.dt_update_every)
            return SWE_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; i++) {
        // every own cell's two neighbours on each side lie in the window,
        // or outside the whole domain (the stencil of a stage)
        const swe_domain *d = doms[i];
        const Box o = own_box(d);
        if ((o.x0 > 0 && d->p.own_x0 < 2) || (o.x1 < d->p.whole_nx && d->nx - d->p.own_x1 < 2) ||
            (o.y0 > 0 && d->p.own_y0 < 2) || (o.y1 < d->p.whole_ny && d->ny - d->p.own_y1 < 2))
            return SWE_ERR_INVALID_ARG;
    }
    long long owned = 0;
    for (int i = 0; i < n; i++) {
        const Box oi = own_box(doms[i]);
        owned += area(oi);
        long long halo = 0;
        for (int j = 0; j < n; j++) {
            Box o;
            if (j == i) continue;
            if (overlap(oi, own_box(doms[j]), nullptr)) return SWE_ERR_INVALID_ARG;
            if (overlap(window_box(doms[i]), own_box(doms[j]), &o)) halo += area(o);
        }
        if (halo != area(window_box(doms[i])) - area(oi)) return SWE_ERR_INVALID_ARG;
    }
    if (owned != (long long)a->p.whole_nx * a->p.whole_ny) return SWE_ERR_INVALID_ARG;
    return SWE_OK;
}

swe::SplitClocks split_clocks(const swe_handle *doms, int n) {
    swe::SplitClocks c;
    memset(&c, 0, sizeof c);
    c.n = n;
    const StageArgs<float> a0 = make_args<float>(doms[0]);
    c.clk = a0.clk;
    for (int k = 0; k < n; k++) {
        const StageArgs<float> a = make_args<float>(doms[k]);
        c.ctl[k] = a.ctl;
        c.bnd[k] = a.bnd;
        c.wind[k] = a.wind;
    }
    return c;
}

// Every (sub-domain, owner) pair whose window and own cells overlap, in
// launches of at most kHaloCopies copies.
int split_exchange(const swe_handle *doms, int n, int what, cudaStream_t st, long long *launches) {
    swe::HaloTable t;
    memset(&t, 0, sizeof t);
    for (int k = 0; k < n; k++) {
        const swe_domain *d = doms[k];
        swe::SplitPlanes &P = t.dom[k];
        for (int v = 0; v < 3; v++) {
            P.q[0][v] = (float *)d->q[0][v];
            P.q[1][v] = (float *)d->q[1][v];
            P.d1[v] = (float *)d->d1[v];
        }
        P.ctl = d->ctl;
        P.pitch = d->pitch;
        P.wx0 = d->p.window_x0;
        P.wy0 = d->p.window_y0;
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            Box o;
            if (i == j || !overlap(window_box(doms[i]), own_box(doms[j]), &o)) continue;
            t.copy[t.n_copies++] = swe::HaloCopy{i, j, (int)o.x0, (int)o.x1, (int)o.y0, (int)o.y1};
            if (t.n_copies == swe::kHaloCopies) {
                cudaError_t e = swe::launch_halo_copy(t, what, st);
                if (e != cudaSuccess) return cuda_fail(e);
                ++*launches;
                t.n_copies = 0;
            }
        }
    if (t.n_copies > 0) {
        cudaError_t e = swe::launch_halo_copy(t, what, st);
        if (e != cudaSuccess) return cuda_fail(e);
        ++*launches;
    }
    return SWE_OK;
}

}  // namespace

int swe_split_sync(const swe_handle *doms, int n) {
    swe::TraceRange trace("swe_split_sync");
    int rc = split_check(doms, n);
    if (rc) return rc;
    cudaStream_t st = doms[0]->stream;
    for (int k = 0; k < n; k++) {
        cudaError_t e = swe::launch_speed(make_args<float>(doms[k]), st);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    cudaError_t e = swe::launch_split_clock(split_clocks(doms, n), 0, st);
    for (int k = 0; k < n && e == cudaSuccess; k++) e = swe::launch_edge_fill(make_args<float>(doms[k]), st);
    return e == cudaSuccess ? SWE_OK : cuda_fail(e);
}

int swe_split_step(const swe_handle *doms, int n, int n_steps) {
    swe::TraceRange trace("swe_split_step");
    int rc = split_check(doms, n);
    if (rc) return rc;
    for (int k = 0; k < n; k++)
        if ((rc = split_step_check(doms[k], n_steps))) return rc;
    cudaStream_t st = doms[0]->stream;
    const swe::SplitClocks clocks = split_clocks(doms, n);
    long long launches = 0;
    for (int s = 0; s < n_steps; s++) {
        for (int k = 0; k < n; k++) {
            cudaError_t e = swe::launch_domain_stage(doms[k]->one, 1, st);
            if (e != cudaSuccess) return cuda_fail(e);
        }
        if ((rc = split_exchange(doms, n, 1, st, &launches))) return rc;
        for (int k = 0; k < n; k++) {
            cudaError_t e = swe::launch_domain_stage(doms[k]->one, 2, st);
            if (e != cudaSuccess) return cuda_fail(e);
        }
        cudaError_t e = swe::launch_split_clock(clocks, 1, st);
        if (e != cudaSuccess) return cuda_fail(e);
        if ((rc = split_exchange(doms, n, 0, st, &launches))) return rc;
        for (int k = 0; k < n; k++) doms[k]->launches += 2;
        doms[0]->launches += 1;
    }
    doms[0]->launches += launches;
    return SWE_OK;
}

}  // extern "C"
