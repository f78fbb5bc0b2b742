// C ABI of libsal.so: argument checks, workspace layout and launches (declared in sal.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <new>

#include "sal_internal.cuh"

namespace sal {

void make_tables(int L, SpecTables *t)
{
    memset(t, 0, sizeof(*t));
    const double pi = 3.14159265358979323846264338327950288;
    for (int n = 0; n < L && n < 16; ++n) {
        t->cs[n] = (float)cos(2.0 * pi * n / L);
        t->sn[n] = (float)sin(2.0 * pi * n / L);
    }
    // Eq. 1-4 with centred indices: w_t = |(nu, om)| / rho, w_x = |(mu, om)| / rho, w_y = |(mu, nu)| / rho
    const int h = (L - 1) / 2;
    for (int mu = 0; mu <= h; ++mu)
        for (int nu = 0; nu <= h; ++nu)
            for (int om = 0; om <= h; ++om) {
                float *w = &t->w[((mu * kMaxHalf + nu) * kMaxHalf + om) * 3];
                const double rho = sqrt((double)(mu * mu + nu * nu + om * om));
                if (rho == 0.0) {
                    w[0] = w[1] = w[2] = 0.f;
                } else {
                    w[0] = (float)(sqrt((double)(nu * nu + om * om)) / rho);
                    w[1] = (float)(sqrt((double)(mu * mu + om * om)) / rho);
                    w[2] = (float)(sqrt((double)(mu * mu + nu * nu)) / rho);
                }
            }
    const double n3 = (double)L * L * L;
    t->escale = (float)(2.0 / ((n3 - 1.0) * n3));
}

namespace {
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
std::once_flag g_ctx_once;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
}  // namespace

cudaError_t current_context_id(unsigned long long *id)
{
    std::call_once(g_ctx_once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!g_ctx_get_current || !g_ctx_get_id) return cudaErrorNotSupported;
    void *ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return cudaErrorInitializationError;
    return g_ctx_get_id(ctx, id) == 0 ? cudaSuccess : cudaErrorInitializationError;
}

// Status word the tensor-core kernels set when a bounded wait runs out (one per device).
static __device__ int g_device_status;

namespace {
std::atomic<int> g_stall{0};
}  // namespace

// Device address of the status word in the current context.  Looked up on every call (the
// lookup allocates nothing), so it stays right after a device reset.
int *device_status_ptr()
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return nullptr;
    return static_cast<int *>(p);
}

TcControl tc_control()
{
    const int stall = g_stall.load();
    return TcControl{device_status_ptr(), stall, stall ? 20000000ull : 1000000000ull};
}

void set_test_stall(int on) { g_stall.store(on ? 1 : 0); }

}  // namespace sal

namespace {

thread_local char g_err[512];

sal_status fail(sal_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

sal_status ok()
{
    g_err[0] = 0;
    return SAL_OK;
}

sal_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(SAL_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

sal_status check_dims(sal_dims d)
{
    if (d.T < 1 || d.X < 1 || d.Y < 1) return fail(SAL_ERR_INVALID_ARG, "dims must be >= 1 (got %lld x %lld x %lld)",
                                                   (long long)d.T, (long long)d.X, (long long)d.Y);
    const double n = (double)d.T * (double)d.X * (double)d.Y;
    if (n > 4.0e12) return fail(SAL_ERR_INVALID_ARG, "volume too large");
    return SAL_OK;
}

sal_status check_L(int L)
{
    if (L < 3 || L > sal::kMaxL) return fail(SAL_ERR_INVALID_ARG, "L must be in [3, %d] (got %d)", sal::kMaxL, L);
    if ((L & 1) == 0) return fail(SAL_ERR_UNSUPPORTED, "even L has no centre voxel (got %d)", L);
    return SAL_OK;
}

sal_status check_params(const sal_params *p)
{
    if (!p) return fail(SAL_ERR_INVALID_ARG, "params is NULL");
    sal_status s = check_L(p->L);
    if (s) return s;
    if (p->precision < SAL_PREC_FP32 || p->precision > SAL_PREC_BF16)
        return fail(SAL_ERR_INVALID_ARG, "bad precision %d", p->precision);
    if (p->boundary != SAL_BND_REFLECT && p->boundary != SAL_BND_PERIODIC)
        return fail(SAL_ERR_INVALID_ARG, "bad boundary %d", p->boundary);
    if (p->stencil != SAL_STENCIL_26 && p->stencil != SAL_STENCIL_LINE && p->stencil != SAL_STENCIL_DIAG_TX)
        return fail(SAL_ERR_INVALID_ARG, "bad stencil %d", p->stencil);
    if (!(p->sigma > 0.f) || !isfinite(p->sigma)) return fail(SAL_ERR_INVALID_ARG, "sigma must be finite and > 0");
    if (p->stride < 0 || p->stride > (p->L - 1) / 2)
        return fail(SAL_ERR_INVALID_ARG, "stride must be 0, 1 or at most (L-1)/2 = %d (cubes overlapping by more than half; got %d)",
                    (p->L - 1) / 2, p->stride);
    if (!isfinite(p->a) || !isfinite(p->b) || !isfinite(p->c)) return fail(SAL_ERR_INVALID_ARG, "a, b, c must be finite");
    if (!(p->eps >= 0.0) || !isfinite(p->eps)) return fail(SAL_ERR_INVALID_ARG, "eps must be finite and >= 0");
    return SAL_OK;
}

// Entry points that compute energies one cube per voxel only (their scratch has no room for
// the lattice energies of a coarse stride).
sal_status check_unit_stride(const sal_params *p, const char *what)
{
    if (p->stride > 1)
        return fail(SAL_ERR_UNSUPPORTED, "%s computes one cube per voxel; stride %d is served by sal_saliency and by "
                                         "sal_lattice_energy + sal_interpolate_lattice", what, p->stride);
    return SAL_OK;
}

size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

struct WsLayout {
    size_t E, Sm, partials, stats, total;
};

WsLayout saliency_layout(sal_dims d)
{
    const size_t N = (size_t)(d.T * d.X * d.Y);
    WsLayout w;
    w.E = 0;
    w.Sm = round256(w.E + 3 * N * sizeof(float));
    w.partials = round256(w.Sm + 3 * N * sizeof(float));
    w.stats = round256(w.partials + 9 * (size_t)sal::dcs_num_partials(d) * sizeof(double));
    w.total = round256(w.stats + SAL_STATS_LEN * sizeof(double));
    return w;
}

size_t dcs_ws_bytes(sal_dims d) { return round256(9 * (size_t)sal::dcs_num_partials(d) * sizeof(double)); }

// Planes of V a slab needs beyond its own on each side: h for the energies of the E planes
// its comparisons read, plus the comparison's reach along t.
int64_t slab_halo_planes(const sal_params *p)
{
    const int64_t h = (p->L - 1) / 2;
    const int64_t rt = p->stencil == SAL_STENCIL_26 ? 1 : h;   // LINE (map t) and DIAG_TX reach h planes
    return h + rt;
}

// Workspace of a slab: E of the given planes, then the reduction partials.
WsLayout slab_layout(sal_dims ext)
{
    const size_t N = (size_t)(ext.T * ext.X * ext.Y);
    WsLayout w;
    w.E = 0;
    w.Sm = 0;
    w.partials = round256(3 * N * sizeof(float));
    w.stats = round256(w.partials + 9 * (size_t)sal::dcs_num_partials(ext) * sizeof(double));
    w.total = w.stats;
    return w;
}

sal_status energy_dispatch(const float *V, sal_dims d, const sal_params *p, float *E, cudaStream_t s)
{
    sal_status st = check_unit_stride(p, "this call");
    if (st) return st;
    if (p->precision != SAL_PREC_FP32) {
        if (!sal::energy_tc_supported(p->L, p->precision))
            return fail(SAL_ERR_UNSUPPORTED, "precision %d is not available for L = %d", p->precision, p->L);
        const sal::TcControl c = sal::tc_control();
        if (!c.status) return fail(SAL_ERR_CUDA, "device status word unavailable");
        sal::EVolDesc v{V, E, d.T, d.X, d.Y};
        cudaError_t e = sal::launch_energy_tc(&v, 1, p->L, p->boundary, p->precision, false, c, s);
        return e == cudaSuccess ? SAL_OK : cuda_fail(e, "tensor-core spectral energy launch");
    }
    const int shape = sal::autotune_lookup(p->L, p->precision, sal::size_class_of(d.T * d.X * d.Y));
    sal::EVolDesc v{V, E, d.T, d.X, d.Y};
    cudaError_t e = sal::launch_energy_fp32_batch(&v, 1, p->L, p->boundary, shape, false, s);
    return e == cudaSuccess ? SAL_OK : cuda_fail(e, "spectral energy launch");
}

// Workspace of the host-buffer entry point: two V buffers, E, S_m, two S buffers, the
// reduction partials and the statistics, each 256-byte aligned.
struct HostLayout {
    size_t V[2], E, Sm, S[2], partials, stats, total;
};

HostLayout host_layout(sal_dims d)
{
    const size_t N = (size_t)(d.T * d.X * d.Y), f = sizeof(float);
    HostLayout h;
    h.V[0] = 0;
    h.V[1] = round256(h.V[0] + N * f);
    h.E = round256(h.V[1] + N * f);
    h.Sm = round256(h.E + 3 * N * f);
    h.S[0] = round256(h.Sm + 3 * N * f);
    h.S[1] = round256(h.S[0] + N * f);
    h.partials = round256(h.S[1] + N * f);
    h.stats = round256(h.partials + 9 * (size_t)sal::dcs_num_partials(d) * sizeof(double));
    h.total = round256(h.stats + SAL_STATS_LEN * sizeof(double));
    return h;
}

// Streams and events that order the calls on one workspace: the V copy of a call waits for
// the kernels of the call that last read the same V buffer, the combine of a call for the
// copy-back of the call that last wrote the same S buffer.
constexpr int kHostChunks = 4;   // pieces of V (along t) whose copies overlap the first kernels

struct HostPipe {
    int dev = -1;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t v_free[2] = {nullptr, nullptr}, s_free[2] = {nullptr, nullptr};
    cudaEvent_t v_ready = nullptr, s_ready = nullptr, s_done = nullptr;
    cudaEvent_t chunk[kHostChunks] = {};
    int parity = 0;
};
std::mutex g_pipe_mu;
std::map<const void *, HostPipe> g_pipes;

cudaError_t pipe_create(HostPipe &hp, int dev)
{
    hp.dev = dev;
    cudaError_t e = cudaStreamCreateWithFlags(&hp.h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hp.d2h, cudaStreamNonBlocking);
    cudaEvent_t *evs[] = {&hp.v_free[0], &hp.v_free[1], &hp.s_free[0], &hp.s_free[1], &hp.v_ready, &hp.s_ready,
                          &hp.s_done};
    for (cudaEvent_t *ev : evs)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    for (cudaEvent_t &ev : hp.chunk)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    return e;
}

void pipe_destroy(HostPipe &hp)
{
    if (hp.h2d) cudaStreamSynchronize(hp.h2d);
    if (hp.d2h) cudaStreamSynchronize(hp.d2h);
    cudaEvent_t evs[] = {hp.v_free[0], hp.v_free[1], hp.s_free[0], hp.s_free[1], hp.v_ready, hp.s_ready, hp.s_done};
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : hp.chunk)
        if (ev) cudaEventDestroy(ev);
    if (hp.h2d) cudaStreamDestroy(hp.h2d);
    if (hp.d2h) cudaStreamDestroy(hp.d2h);
    hp = HostPipe{};
}

// Workspace layout of a batch: per volume E [3N] floats, S_m [3N] floats and its [9][tiles]
// reduction records, each 256-byte aligned; then n * 9 statistics.
struct BatchLayout {
    size_t E[SAL_BATCH_MAX], Sm[SAL_BATCH_MAX], part[SAL_BATCH_MAX], stats, total;
};

sal_status check_batch(const sal_volume *vols, int32_t n, const sal_params *p, bool need_ptrs)
{
    if (!vols) return fail(SAL_ERR_INVALID_ARG, "vols is NULL");
    if (n < 1 || n > SAL_BATCH_MAX) return fail(SAL_ERR_INVALID_ARG, "batch size must be in [1, %d]", SAL_BATCH_MAX);
    sal_status s = check_params(p);
    if (!s) s = check_unit_stride(p, "the batched path");
    if (s) return s;
    if (p->precision != SAL_PREC_FP32 && !sal::energy_tc_supported(p->L, p->precision))
        return fail(SAL_ERR_UNSUPPORTED, "precision %d is not available for L = %d", p->precision, p->L);
    for (int i = 0; i < n; ++i) {
        s = check_dims(sal_dims{vols[i].T, vols[i].X, vols[i].Y});
        if (s) return s;
        if (need_ptrs && (!vols[i].V || !vols[i].S)) return fail(SAL_ERR_INVALID_ARG, "volume %d: NULL pointer", i);
        if (need_ptrs && (!aligned16(vols[i].V) || !aligned16(vols[i].S)))
            return fail(SAL_ERR_INVALID_ARG, "volume %d: pointers must be 16-byte aligned", i);
    }
    return SAL_OK;
}

BatchLayout batch_layout(const sal_volume *vols, int32_t n)
{
    BatchLayout b;
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const size_t N = (size_t)(vols[i].T * vols[i].X * vols[i].Y);
        b.E[i] = off;
        b.Sm[i] = round256(off + 3 * N * sizeof(float));
        b.part[i] = round256(b.Sm[i] + 3 * N * sizeof(float));
        off = round256(b.part[i] + 9 * (size_t)sal::dcs_num_tiles(sal_dims{vols[i].T, vols[i].X, vols[i].Y}) * sizeof(double));
    }
    b.stats = off;
    b.total = round256(off + 9 * (size_t)n * sizeof(double));
    return b;
}

void energy_descs(const sal_volume *vols, int32_t n, const BatchLayout &b, char *base, sal::EVolDesc *ev)
{
    for (int i = 0; i < n; ++i) ev[i] = sal::EVolDesc{vols[i].V, (float *)(base + b.E[i]), vols[i].T, vols[i].X, vols[i].Y};
}

int batch_shape(const sal_volume *vols, int32_t n, const sal_params *p)
{
    int64_t nmax = 0;
    for (int i = 0; i < n; ++i) nmax = vols[i].T * vols[i].X * vols[i].Y > nmax ? vols[i].T * vols[i].X * vols[i].Y : nmax;
    return sal::autotune_lookup(p->L, p->precision, sal::size_class_of(nmax));
}

// Enqueues the four launches of a batch on `s`.
sal_status enqueue_batch(const sal_volume *vols, int32_t n, const sal_params *p, double *stats, char *base,
                         const BatchLayout &b, cudaStream_t s)
{
    sal::EVolDesc ev[SAL_BATCH_MAX];
    sal::DVolDesc dv[SAL_BATCH_MAX];
    sal::BatchVolDesc bv[SAL_BATCH_MAX];
    energy_descs(vols, n, b, base, ev);
    for (int i = 0; i < n; ++i) {
        float *Sm = (float *)(base + b.Sm[i]);
        double *part = (double *)(base + b.part[i]);
        dv[i] = sal::DVolDesc{ev[i].E, Sm, part, vols[i].T, vols[i].X, vols[i].Y};
        bv[i] = sal::BatchVolDesc{Sm, vols[i].S, part,
                                  sal::dcs_num_records(sal_dims{vols[i].T, vols[i].X, vols[i].Y}),
                                  vols[i].T * vols[i].X * vols[i].Y};
    }
    cudaError_t e;
    if (p->precision == SAL_PREC_FP32) {
        e = sal::launch_energy_fp32_batch(ev, n, p->L, p->boundary, batch_shape(vols, n, p), true, s);
    } else {
        const sal::TcControl c = sal::tc_control();
        if (!c.status) return fail(SAL_ERR_CUDA, "device status word unavailable");
        e = sal::launch_energy_tc(ev, n, p->L, p->boundary, p->precision, true, c, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batched spectral energy launch");
    e = sal::launch_dcs_items(dv, n, p, s);
    if (e != cudaSuccess) return cuda_fail(e, "batched directional compare launch");
    e = sal::launch_batch_stats_combine(bv, n, p, stats ? stats : (double *)(base + b.stats), s);
    if (e != cudaSuccess) return cuda_fail(e, "batched statistics / combine launch");
    return SAL_OK;
}

sal_tile_choice choice_of(int L, int precision, int cls, int shape, float ms)
{
    const sal::TileShape t = sal::energy_shape(L, shape);
    return sal_tile_choice{L, precision, cls, shape, t.bt, t.bx, t.by, t.mode, ms};
}

}  // namespace

extern "C" {

sal_status sal_params_default(sal_params *p)
{
    if (!p) return fail(SAL_ERR_INVALID_ARG, "params is NULL");
    memset(p, 0, sizeof(*p));
    p->L = 7;
    p->precision = SAL_PREC_FP32;
    p->boundary = SAL_BND_REFLECT;
    p->stencil = SAL_STENCIL_26;
    p->sigma = 1.0f;
    p->a = p->b = p->c = 1.0 / 3.0;
    p->eps = 1e-6;
    return ok();
}

sal_status sal_workspace_size(sal_dims dims, const sal_params *p, size_t *bytes)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!bytes) return fail(SAL_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = saliency_layout(dims).total;
    return ok();
}

sal_status sal_dcs_workspace_size(sal_dims dims, const sal_params *p, size_t *bytes)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!bytes) return fail(SAL_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = dcs_ws_bytes(dims);
    return ok();
}

sal_status sal_local_spectra(const float *V, sal_dims dims, const sal_params *p, const int64_t roi_lo[3],
                             const int64_t roi_ext[3], float *mag, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!V || !mag || !roi_lo || !roi_ext) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(V) || !aligned16(mag)) return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    const int64_t D[3] = {dims.T, dims.X, dims.Y};
    for (int i = 0; i < 3; ++i)
        if (roi_lo[i] < 0 || roi_ext[i] < 0 || roi_lo[i] + roi_ext[i] > D[i])
            return fail(SAL_ERR_INVALID_ARG, "region of interest leaves the volume on axis %d", i);
    cudaError_t e = sal::launch_local_spectra(V, dims, p->L, p->boundary, roi_lo, roi_ext, mag, (cudaStream_t)stream);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_local_spectra");
}

sal_status sal_project(const float *mag, int64_t n_vox, int32_t L, float *E, void *stream)
{
    sal_status s = check_L(L);
    if (s) return s;
    if (n_vox < 0) return fail(SAL_ERR_INVALID_ARG, "n_vox < 0");
    if (n_vox > 0 && (!mag || !E)) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(mag) || !aligned16(E)) return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    cudaError_t e = sal::launch_project(mag, n_vox, L, E, (cudaStream_t)stream);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_project");
}

sal_status sal_spectral_energy(const float *V, sal_dims dims, const sal_params *p, float *E, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!V || !E) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(V) || !aligned16(E)) return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    s = energy_dispatch(V, dims, p, E, (cudaStream_t)stream);
    return s ? s : ok();
}

sal_status sal_lattice_dims(sal_dims dims, const sal_params *p, sal_dims *lattice)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!lattice) return fail(SAL_ERR_INVALID_ARG, "lattice is NULL");
    const int st = p->stride > 1 ? p->stride : 1;
    *lattice = sal_dims{sal::lattice_size(dims.T, st), sal::lattice_size(dims.X, st), sal::lattice_size(dims.Y, st)};
    return ok();
}

sal_status sal_lattice_energy(const float *V, sal_dims dims, const sal_params *p, float *Ec, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (p->precision != SAL_PREC_FP32) return fail(SAL_ERR_UNSUPPORTED, "lattice energies are computed in FP32 only");
    if (!V || !Ec) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(V) || !aligned16(Ec)) return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    cudaError_t e = sal::launch_lattice_energy(V, dims, p->L, p->boundary, p->stride > 1 ? p->stride : 1, Ec,
                                               (cudaStream_t)stream);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_lattice_energy");
}

sal_status sal_interpolate_lattice(const float *Ec, sal_dims dims, const sal_params *p, float *E, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!Ec || !E) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(Ec) || !aligned16(E)) return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    cudaError_t e = sal::launch_interp_lattice(Ec, dims, p->stride > 1 ? p->stride : 1, E, (cudaStream_t)stream);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_interpolate_lattice");
}

sal_status sal_directional_compare(const float *E, sal_dims dims, const sal_params *p, float *Sm, double *stats,
                                   void *ws, size_t ws_bytes, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!E || !Sm || !stats || !ws) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(E) || !aligned16(Sm) || !aligned16(stats) || !aligned16(ws))
        return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    const size_t need = dcs_ws_bytes(dims);
    if (ws_bytes < need) return fail(SAL_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, need);
    cudaError_t e = sal::launch_dcs(E, dims, p, Sm, (double *)ws, stats, (cudaStream_t)stream);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_directional_compare");
}

sal_status sal_directional_compare_static(const float *E, sal_dims dims, const sal_params *p, float *Sm,
                                          double *stats, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!E || !Sm || !stats) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(E) || !aligned16(Sm) || !aligned16(stats))
        return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    const int64_t tiles = sal::dcs_num_tiles(dims);
    if (tiles > SAL_DCS_STATIC_MAX_TILES)
        return fail(SAL_ERR_WORKSPACE, "volume needs %lld tiles of fixed scratch; at most %d fit",
                    (long long)tiles, SAL_DCS_STATIC_MAX_TILES);
    double *scratch = nullptr;
    cudaError_t e = sal::dcs_static_scratch(&scratch);
    if (e != cudaSuccess) return cuda_fail(e, "fixed scratch address");
    e = sal::launch_dcs(E, dims, p, Sm, scratch, stats, (cudaStream_t)stream);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_directional_compare_static");
}

sal_status sal_directional_compare_user(const float *E, sal_dims dims, const sal_params *p, const sal_user_stencil *st,
                                        float *Sm, double *stats, void *ws, size_t ws_bytes, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!E || !Sm || !stats || !ws || !st) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(E) || !aligned16(Sm) || !aligned16(stats) || !aligned16(ws))
        return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    for (int m = 0; m < 3; ++m) {
        if (st->count[m] < 1 || st->count[m] > SAL_STENCIL_MAX_OFFSETS)
            return fail(SAL_ERR_INVALID_ARG, "map %d: count must be in [1, %d] (got %d)", m, SAL_STENCIL_MAX_OFFSETS,
                        st->count[m]);
        for (int k = 0; k < st->count[m]; ++k) {
            const int32_t *o = st->offset[m][k];
            for (int a = 0; a < 3; ++a)
                if (o[a] < -SAL_STENCIL_MAX_RADIUS || o[a] > SAL_STENCIL_MAX_RADIUS)
                    return fail(SAL_ERR_INVALID_ARG, "map %d offset %d: component %d outside [-%d, %d]", m, k, a,
                                SAL_STENCIL_MAX_RADIUS, SAL_STENCIL_MAX_RADIUS);
            if (!o[0] && !o[1] && !o[2]) return fail(SAL_ERR_INVALID_ARG, "map %d offset %d is (0, 0, 0)", m, k);
            if (!isfinite(st->weight[m][k])) return fail(SAL_ERR_INVALID_ARG, "map %d weight %d is not finite", m, k);
        }
    }
    const size_t need = dcs_ws_bytes(dims);
    if (ws_bytes < need) return fail(SAL_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, need);
    cudaError_t e = sal::launch_dcs(E, dims, p, Sm, (double *)ws, stats, (cudaStream_t)stream, st);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_directional_compare_user");
}

sal_status sal_slab_halo(const sal_params *p, int64_t *planes)
{
    sal_status s = check_params(p);
    if (s) return s;
    if (!planes) return fail(SAL_ERR_INVALID_ARG, "planes is NULL");
    *planes = slab_halo_planes(p);
    return ok();
}

sal_status sal_slab_workspace_size(int64_t ext_planes, int64_t X, int64_t Y, const sal_params *p, size_t *bytes)
{
    sal_status s = check_dims(sal_dims{ext_planes, X, Y});
    if (!s) s = check_params(p);
    if (s) return s;
    if (!bytes) return fail(SAL_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = slab_layout(sal_dims{ext_planes, X, Y}).total;
    return ok();
}

sal_status sal_slab_maps(const float *V_ext, sal_dims dims, int64_t ext_lo, int64_t ext_hi, int64_t own_lo, int64_t own_hi,
                         const sal_params *p, float *Sm_own, double *stats_local, void *ws, size_t ws_bytes, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!V_ext || !Sm_own || !stats_local || !ws) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(V_ext) || !aligned16(Sm_own) || !aligned16(stats_local) || !aligned16(ws))
        return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    if (own_lo < 0 || own_hi > dims.T || own_lo >= own_hi)
        return fail(SAL_ERR_INVALID_ARG, "own planes [%lld, %lld) must be a non-empty part of [0, %lld)",
                    (long long)own_lo, (long long)own_hi, (long long)dims.T);
    const int64_t H = slab_halo_planes(p);
    const int64_t want_lo = own_lo - H > 0 ? own_lo - H : 0, want_hi = own_hi + H < dims.T ? own_hi + H : dims.T;
    if (ext_lo != want_lo || ext_hi != want_hi)
        return fail(SAL_ERR_INVALID_ARG, "planes of V must be [%lld, %lld) for own planes [%lld, %lld) (halo %lld)",
                    (long long)want_lo, (long long)want_hi, (long long)own_lo, (long long)own_hi, (long long)H);
    if (p->boundary == SAL_BND_PERIODIC && (ext_lo != 0 || ext_hi != dims.T))
        return fail(SAL_ERR_UNSUPPORTED, "PERIODIC wraps t across the volume: a slab must hold every plane");
    const sal_dims ext{ext_hi - ext_lo, dims.X, dims.Y};
    const WsLayout w = slab_layout(ext);
    if (ws_bytes < w.total) return fail(SAL_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, w.total);
    char *base = (char *)ws;
    float *E = (float *)(base + w.E);
    const cudaStream_t st = (cudaStream_t)stream;
    s = energy_dispatch(V_ext, ext, p, E, st);
    if (s) return s;
    cudaError_t e = sal::launch_dcs(E, ext, p, Sm_own, (double *)(base + w.partials), stats_local, st, nullptr,
                                    own_lo - ext_lo, own_hi - ext_lo);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_slab_maps");
}

sal_status sal_probe_fma_rate(float *out, int64_t n_threads, int32_t iters, int32_t packed, void *stream)
{
    if (!out) return fail(SAL_ERR_INVALID_ARG, "out is NULL");
    if (n_threads < 256 || n_threads % 256 != 0 || n_threads / 256 > 0x7fffffffLL)
        return fail(SAL_ERR_INVALID_ARG, "n_threads must be a positive multiple of 256 (got %lld)", (long long)n_threads);
    if (iters < 16 || iters % 16 != 0) return fail(SAL_ERR_INVALID_ARG, "iters must be a positive multiple of 16 (got %d)", iters);
    cudaError_t e = sal::launch_fma_probe(out, n_threads, iters, packed != 0, (cudaStream_t)stream);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_probe_fma_rate");
}

sal_status sal_stats_merge(const double *stats, int32_t n, double *out, void *stream)
{
    if (!stats || !out) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (n < 1) return fail(SAL_ERR_INVALID_ARG, "n must be >= 1 (got %d)", n);
    if (!aligned16(stats) || !aligned16(out)) return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    cudaError_t e = sal::launch_stats_merge(stats, n, out, (cudaStream_t)stream);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_stats_merge");
}

sal_status sal_combine(const float *Sm, const double *stats, sal_dims dims, const sal_params *p, float *S, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!Sm || !stats || !S) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(Sm) || !aligned16(stats) || !aligned16(S))
        return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    cudaError_t e = sal::launch_combine(Sm, stats, dims, p, S, (cudaStream_t)stream);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_combine");
}

sal_status sal_saliency(const float *V, sal_dims dims, const sal_params *p, float *S, double *stats, void *ws,
                        size_t ws_bytes, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!V || !S || !ws) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(V) || !aligned16(S) || !aligned16(ws) || (stats && !aligned16(stats)))
        return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    const WsLayout w = saliency_layout(dims);
    if (ws_bytes < w.total) return fail(SAL_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, w.total);
    char *base = (char *)ws;
    float *E = (float *)(base + w.E);
    float *Sm = (float *)(base + w.Sm);
    double *part = (double *)(base + w.partials);
    double *st = stats ? stats : (double *)(base + w.stats);
    cudaStream_t cs = (cudaStream_t)stream;
    if (p->stride > 1) {
        // coarse stride: the lattice energies go to the S_m region (3 Nc <= 3 N floats, not yet
        // in use), are interpolated into E, and S_m then overwrites them in stream order
        if (p->precision != SAL_PREC_FP32)
            return fail(SAL_ERR_UNSUPPORTED, "stride > 1 is computed in FP32 on the CUDA cores only");
        cudaError_t e = sal::launch_lattice_energy(V, dims, p->L, p->boundary, p->stride, Sm, cs);
        if (e == cudaSuccess) e = sal::launch_interp_lattice(Sm, dims, p->stride, E, cs);
        if (e != cudaSuccess) return cuda_fail(e, "lattice energy / interpolation launch");
    } else {
        s = energy_dispatch(V, dims, p, E, cs);
        if (s) return s;
    }
    cudaError_t e = sal::launch_dcs(E, dims, p, Sm, part, st, cs);
    if (e != cudaSuccess) return cuda_fail(e, "directional compare launch");
    e = sal::launch_combine(Sm, st, dims, p, S, cs);
    if (e != cudaSuccess) return cuda_fail(e, "combine launch");
    return ok();
}

sal_status sal_host_workspace_size(sal_dims dims, const sal_params *p, size_t *bytes)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!bytes) return fail(SAL_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = host_layout(dims).total;
    return ok();
}

sal_status sal_saliency_host(const float *V_host, sal_dims dims, const sal_params *p, float *S_host, double *stats,
                             void *ws, size_t ws_bytes, void *stream, void *done_event)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (p->stride > 1 && p->precision != SAL_PREC_FP32)
        return fail(SAL_ERR_UNSUPPORTED, "stride > 1 is computed in FP32 on the CUDA cores only");
    if (!V_host || !S_host || !ws) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(ws) || (stats && !aligned16(stats)))
        return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    if (p->precision != SAL_PREC_FP32 && !sal::energy_tc_supported(p->L, p->precision))
        return fail(SAL_ERR_UNSUPPORTED, "precision %d is not available for L = %d", p->precision, p->L);
    const HostLayout h = host_layout(dims);
    if (ws_bytes < h.total) return fail(SAL_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, h.total);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");

    std::lock_guard<std::mutex> lock(g_pipe_mu);
    HostPipe &hp = g_pipes[ws];
    if (hp.dev < 0) {
        e = pipe_create(hp, dev);
        if (e != cudaSuccess) {
            pipe_destroy(hp);
            g_pipes.erase(ws);
            return cuda_fail(e, "stream / event creation");
        }
    } else if (hp.dev != dev) {
        return fail(SAL_ERR_INVALID_ARG, "workspace was first used on device %d, not %d", hp.dev, dev);
    }
    const int b = hp.parity;
    char *base = (char *)ws;
    float *Vd = (float *)(base + h.V[b]), *Sd = (float *)(base + h.S[b]);
    float *E = (float *)(base + h.E), *Sm = (float *)(base + h.Sm);
    double *part = (double *)(base + h.partials);
    double *st = stats ? stats : (double *)(base + h.stats);
    const size_t bytes = (size_t)(dims.T * dims.X * dims.Y) * sizeof(float);
    cudaStream_t cs = (cudaStream_t)stream;

    // host -> device, once the kernels of the call that last read this V buffer are done
    e = cudaStreamWaitEvent(hp.h2d, hp.v_free[b], 0);
    if (e != cudaSuccess) return cuda_fail(e, "copy of V to the device");
    const int64_t XY = dims.X * dims.Y;
    if (p->precision == SAL_PREC_FP32 && dims.T >= 64 && p->stride <= 1) {
        // V in pieces of whole planes (multiples of 16, so of every tile height); the energies
        // of a piece's output planes start once it and the next piece (its halo) are in
        int64_t lo[kHostChunks + 1];
        int64_t ct = (dims.T + kHostChunks - 1) / kHostChunks;
        ct = (ct + 15) / 16 * 16;
        int nch = 0;
        for (int64_t t = 0; t < dims.T && nch < kHostChunks; t += ct) lo[nch++] = t;
        lo[nch] = dims.T;
        for (int c = 0; c < nch && e == cudaSuccess; ++c) {
            e = cudaMemcpyAsync(Vd + lo[c] * XY, V_host + lo[c] * XY, (size_t)((lo[c + 1] - lo[c]) * XY) * sizeof(float),
                                cudaMemcpyHostToDevice, hp.h2d);
            if (e == cudaSuccess) e = cudaEventRecord(hp.chunk[c], hp.h2d);
        }
        if (e != cudaSuccess) return cuda_fail(e, "copy of V to the device");
        const int shape = sal::autotune_lookup(p->L, p->precision, sal::size_class_of(dims.T * XY));
        for (int c = 0; c < nch; ++c) {
            e = cudaStreamWaitEvent(cs, hp.chunk[c], 0);
            if (e == cudaSuccess && c + 1 < nch) e = cudaStreamWaitEvent(cs, hp.chunk[c + 1], 0);
            // a periodic extension reads the far end of the volume at the first and last planes
            if (e == cudaSuccess && c == 0 && p->boundary == SAL_BND_PERIODIC)
                e = cudaStreamWaitEvent(cs, hp.chunk[nch - 1], 0);
            if (e != cudaSuccess) return cuda_fail(e, "stream wait");
            sal::EVolDesc v{Vd, E, dims.T, dims.X, dims.Y, lo[c], lo[c + 1]};
            e = sal::launch_energy_fp32_batch(&v, 1, p->L, p->boundary, shape, false, cs);
            if (e != cudaSuccess) return cuda_fail(e, "spectral energy launch");
        }
    } else {
        e = cudaMemcpyAsync(Vd, V_host, bytes, cudaMemcpyHostToDevice, hp.h2d);
        if (e == cudaSuccess) e = cudaEventRecord(hp.v_ready, hp.h2d);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, hp.v_ready, 0);
        if (e != cudaSuccess) return cuda_fail(e, "copy of V to the device");
        if (p->stride > 1) {
            // lattice energies in the S_m region (free until the compare), interpolated into E
            e = sal::launch_lattice_energy(Vd, dims, p->L, p->boundary, p->stride, Sm, cs);
            if (e == cudaSuccess) e = sal::launch_interp_lattice(Sm, dims, p->stride, E, cs);
            if (e != cudaSuccess) return cuda_fail(e, "lattice energy / interpolation launch");
        } else {
            s = energy_dispatch(Vd, dims, p, E, cs);
            if (s) return s;
        }
    }
    e = cudaEventRecord(hp.v_free[b], cs);
    if (e == cudaSuccess) e = sal::launch_dcs(E, dims, p, Sm, part, st, cs);
    if (e != cudaSuccess) return cuda_fail(e, "directional compare launch");
    // S buffer b is free once the copy-back of the call that last wrote it is done
    e = cudaStreamWaitEvent(cs, hp.s_free[b], 0);
    if (e == cudaSuccess) e = sal::launch_combine(Sm, st, dims, p, Sd, cs);
    if (e != cudaSuccess) return cuda_fail(e, "combine launch");
    e = cudaEventRecord(hp.s_ready, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hp.d2h, hp.s_ready, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S_host, Sd, bytes, cudaMemcpyDeviceToHost, hp.d2h);
    if (e == cudaSuccess) e = cudaEventRecord(hp.s_free[b], hp.d2h);
    if (e == cudaSuccess) {
        if (done_event) {
            e = cudaEventRecord((cudaEvent_t)done_event, hp.d2h);
        } else {
            e = cudaEventRecord(hp.s_done, hp.d2h);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, hp.s_done, 0);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "copy of S to the host");
    hp.parity ^= 1;
    return ok();
}

sal_status sal_host_release(void *ws)
{
    if (!ws) return fail(SAL_ERR_INVALID_ARG, "ws is NULL");
    std::lock_guard<std::mutex> lock(g_pipe_mu);
    auto it = g_pipes.find(ws);
    if (it == g_pipes.end()) return ok();
    pipe_destroy(it->second);
    g_pipes.erase(it);
    return ok();
}

sal_status sal_batch_workspace_size(const sal_volume *vols, int32_t n, const sal_params *p, size_t *bytes)
{
    sal_status s = check_batch(vols, n, p, false);
    if (s) return s;
    if (!bytes) return fail(SAL_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = batch_layout(vols, n).total;
    return ok();
}

sal_status sal_saliency_batched(const sal_volume *vols, int32_t n, const sal_params *p, double *stats, void *ws,
                                size_t ws_bytes, void *stream)
{
    sal_status s = check_batch(vols, n, p, true);
    if (s) return s;
    if (!ws || !aligned16(ws) || (stats && !aligned16(stats)))
        return fail(SAL_ERR_INVALID_ARG, "ws must be non-NULL and 16-byte aligned (stats too)");
    const BatchLayout b = batch_layout(vols, n);
    if (ws_bytes < b.total) return fail(SAL_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, b.total);
    s = enqueue_batch(vols, n, p, stats, (char *)ws, b, (cudaStream_t)stream);
    return s ? s : ok();
}

}  // extern "C"

struct sal_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" {

sal_status sal_graph_create_batched(const sal_volume *vols, int32_t n, const sal_params *p, double *stats, void *ws,
                                    size_t ws_bytes, void *stream, sal_graph **out)
{
    sal_status s = check_batch(vols, n, p, true);
    if (s) return s;
    if (!out) return fail(SAL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ws || !aligned16(ws) || (stats && !aligned16(stats)))
        return fail(SAL_ERR_INVALID_ARG, "ws must be non-NULL and 16-byte aligned (stats too)");
    const BatchLayout b = batch_layout(vols, n);
    if (ws_bytes < b.total) return fail(SAL_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, b.total);
    char *base = (char *)ws;
    int64_t nmax = 0;
    for (int i = 0; i < n; ++i) nmax = vols[i].T * vols[i].X * vols[i].Y > nmax ? vols[i].T * vols[i].X * vols[i].Y : nmax;
    const int cls = sal::size_class_of(nmax);
    cudaError_t e = cudaSuccess;
    // first use for this (L, precision, size class): choose the tile shape on this batch
    float cached_ms = 0.f;
    if (p->precision == SAL_PREC_FP32 && !sal::autotune_get_ms(p->L, p->precision, cls, &cached_ms)) {
        sal::EVolDesc ev[SAL_BATCH_MAX];
        energy_descs(vols, n, b, base, ev);
        int best = 0;
        float ms = 0.f;
        e = sal::autotune_run(ev, n, p->L, p->boundary, p->precision, (cudaStream_t)stream, &best, &ms);
        if (e != cudaSuccess) return cuda_fail(e, "autotune before capture");
    }
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cap);
        return cuda_fail(e, "begin capture");
    }
    s = enqueue_batch(vols, n, p, stats, base, b, cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    cudaStreamDestroy(cap);
    if (s) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(e, "graph instantiate");
    }
    sal_graph *g = new (std::nothrow) sal_graph{graph, exec};
    if (!g) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return fail(SAL_ERR_INTERNAL, "out of host memory");
    }
    *out = g;
    return ok();
}

sal_status sal_graph_launch(sal_graph *g, void *stream)
{
    if (!g) return fail(SAL_ERR_INVALID_ARG, "graph is NULL");
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? ok() : cuda_fail(e, "graph launch");
}

sal_status sal_graph_destroy(sal_graph *g)
{
    if (!g) return ok();
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return ok();
}

sal_status sal_autotune(const float *V, sal_dims dims, const sal_params *p, float *E, void *stream, sal_tile_choice *out)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (!s) s = check_unit_stride(p, "sal_autotune");
    if (s) return s;
    if (!V || !E || !out) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(V) || !aligned16(E)) return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    if (p->precision != SAL_PREC_FP32)
        return fail(SAL_ERR_UNSUPPORTED, "only the FP32 kernel has several tile shapes (precision %d)", p->precision);
    sal::EVolDesc v{V, E, dims.T, dims.X, dims.Y};
    int best = 0;
    float ms = 0.f;
    cudaError_t e = sal::autotune_run(&v, 1, p->L, p->boundary, p->precision, (cudaStream_t)stream, &best, &ms);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    *out = choice_of(p->L, p->precision, sal::size_class_of(dims.T * dims.X * dims.Y), best, ms);
    return ok();
}

sal_status sal_autotune_batched(const sal_volume *vols, int32_t n, const sal_params *p, void *ws, size_t ws_bytes,
                                void *stream, sal_tile_choice *out)
{
    sal_status s = check_batch(vols, n, p, true);
    if (s) return s;
    if (p->precision != SAL_PREC_FP32)
        return fail(SAL_ERR_UNSUPPORTED, "only the FP32 kernel has several tile shapes (precision %d)", p->precision);
    if (!ws || !out || !aligned16(ws)) return fail(SAL_ERR_INVALID_ARG, "ws and out must be non-NULL (ws 16-byte aligned)");
    const BatchLayout b = batch_layout(vols, n);
    if (ws_bytes < b.total) return fail(SAL_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, b.total);
    sal::EVolDesc ev[SAL_BATCH_MAX];
    energy_descs(vols, n, b, (char *)ws, ev);
    int best = 0;
    float ms = 0.f;
    cudaError_t e = sal::autotune_run(ev, n, p->L, p->boundary, p->precision, (cudaStream_t)stream, &best, &ms);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    int64_t nmax = 0;
    for (int i = 0; i < n; ++i) nmax = vols[i].T * vols[i].X * vols[i].Y > nmax ? vols[i].T * vols[i].X * vols[i].Y : nmax;
    *out = choice_of(p->L, p->precision, sal::size_class_of(nmax), best, ms);
    return ok();
}

sal_status sal_autotune_query(int32_t L, int32_t precision, int64_t n_vox, sal_tile_choice *out)
{
    sal_status s = check_L(L);
    if (s) return s;
    if (!out || precision < 0 || precision > 2 || n_vox < 0) return fail(SAL_ERR_INVALID_ARG, "bad argument");
    const int cls = sal::size_class_of(n_vox);
    const int shape = sal::autotune_lookup(L, precision, cls);
    float ms = 0.f;
    sal::autotune_get_ms(L, precision, cls, &ms);
    *out = choice_of(L, precision, cls, shape, ms);
    return ok();
}

sal_status sal_autotune_save(const char *path)
{
    if (!path) return fail(SAL_ERR_INVALID_ARG, "path is NULL");
    return sal::autotune_save(path) == 0 ? ok() : fail(SAL_ERR_INVALID_ARG, "cannot write %s", path);
}

sal_status sal_autotune_load(const char *path)
{
    if (!path) return fail(SAL_ERR_INVALID_ARG, "path is NULL");
    const int r = sal::autotune_load(path);
    if (r == -1) return fail(SAL_ERR_INVALID_ARG, "cannot read %s", path);
    if (r < 0) return fail(SAL_ERR_INVALID_ARG, "malformed autotune cache %s (nothing loaded)", path);
    return ok();
}

sal_status sal_autotune_clear(void)
{
    sal::autotune_clear();
    return ok();
}

sal_status sal_surrogate_param_count(int64_t *n)
{
    if (!n) return fail(SAL_ERR_INVALID_ARG, "n is NULL");
    *n = sal::surrogate_param_count();
    return ok();
}

sal_status sal_surrogate_workspace_size(sal_dims dims, int32_t training, size_t *bytes)
{
    sal_status s = check_dims(dims);
    if (s) return s;
    if (!bytes) return fail(SAL_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = sal::surrogate_ws_bytes(dims, training != 0);
    return ok();
}

sal_status sal_surrogate_forward(const float *V, sal_dims dims, const sal_params *p, const float *params, float *E,
                                 int32_t training, void *ws, size_t ws_bytes, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!V || !params || !ws || (!E && !training)) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(V) || !aligned16(params) || !aligned16(ws) || (E && !aligned16(E)))
        return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    const size_t need = sal::surrogate_ws_bytes(dims, training != 0);
    if (ws_bytes < need) return fail(SAL_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, need);
    const sal::TcControl c = sal::tc_control();
    if (!training && p->precision == SAL_PREC_BF16 && !c.status) return fail(SAL_ERR_CUDA, "device status word unavailable");
    cudaError_t e = sal::surrogate_forward(V, dims, p->boundary, params, E, training != 0, ws, (cudaStream_t)stream,
                                           p->precision, &c);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_surrogate_forward");
}

sal_status sal_surrogate_backward(const float *V, sal_dims dims, const sal_params *p, const float *params,
                                  const float *E_target, int32_t margin, float *grads, double *loss, void *ws,
                                  size_t ws_bytes, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!V || !params || !E_target || !grads || !ws) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (margin < SAL_SURR_LAYERS) return fail(SAL_ERR_INVALID_ARG, "margin must be >= %d", SAL_SURR_LAYERS);
    if (dims.T <= 2 * margin || dims.X <= 2 * margin || dims.Y <= 2 * margin)
        return fail(SAL_ERR_INVALID_ARG, "the margin leaves no voxel in the loss");
    const size_t need = sal::surrogate_ws_bytes(dims, true);
    if (ws_bytes < need) return fail(SAL_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, need);
    cudaError_t e = sal::surrogate_backward(V, dims, p->boundary, params, E_target, margin, grads, loss, ws,
                                            (cudaStream_t)stream);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_surrogate_backward");
}

sal_status sal_surrogate_infer_workspace_size(sal_dims dims, const sal_params *p, size_t *bytes)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (s) return s;
    if (!bytes) return fail(SAL_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = sal::surrogate_infer_ws_bytes(dims, p->L);
    return ok();
}

sal_status sal_surrogate_infer(const float *V, sal_dims dims, const sal_params *p, const float *params, float *E,
                               float threshold, int32_t *counts, void *ws, size_t ws_bytes, void *stream)
{
    sal_status s = check_dims(dims);
    if (!s) s = check_params(p);
    if (!s) s = check_unit_stride(p, "sal_surrogate_infer");
    if (s) return s;
    if (!V || !params || !E || !ws) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (!aligned16(V) || !aligned16(E) || !aligned16(ws) || !aligned16(params))
        return fail(SAL_ERR_INVALID_ARG, "device pointers must be 16-byte aligned");
    if (!(threshold >= 0.f)) return fail(SAL_ERR_INVALID_ARG, "threshold must be >= 0");
    const size_t need = sal::surrogate_infer_ws_bytes(dims, p->L);
    if (ws_bytes < need) return fail(SAL_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, need);
    const sal::TcControl c = sal::tc_control();
    if (p->precision == SAL_PREC_BF16 && !c.status) return fail(SAL_ERR_CUDA, "device status word unavailable");
    cudaError_t e = sal::surrogate_infer(V, dims, p->L, p->boundary, params, E, threshold, counts, ws,
                                         (cudaStream_t)stream, p->precision, &c);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_surrogate_infer");
}

sal_status sal_surrogate_adam_step(float *params, const float *grads, float *m, float *v, int32_t step, float lr,
                                   float beta1, float beta2, float eps, void *stream)
{
    if (!params || !grads || !m || !v) return fail(SAL_ERR_INVALID_ARG, "NULL pointer argument");
    if (step < 1 || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return fail(SAL_ERR_INVALID_ARG, "bad Adam hyper-parameters");
    cudaError_t e = sal::surrogate_adam(params, grads, m, v, sal::surrogate_param_count(), step, lr, beta1, beta2, eps,
                                        (cudaStream_t)stream);
    return e == cudaSuccess ? ok() : cuda_fail(e, "sal_surrogate_adam_step");
}

sal_status sal_device_status(void *stream)
{
    int *p = sal::device_status_ptr();
    if (!p) return fail(SAL_ERR_CUDA, "device status word unavailable");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before reading the status word");
    int v = 0;
    const int zero = 0;
    e = cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(p, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "status word");
    if (v == SAL_ERR_TIMEOUT) return fail(SAL_ERR_TIMEOUT, "a bounded device-side wait ran out");
    return v == 0 ? ok() : fail(SAL_ERR_INTERNAL, "device status %d", v);
}

sal_status sal_test_stall_tensor_cores(int32_t on)
{
    sal::set_test_stall(on);
    return ok();
}

const char *sal_status_string(sal_status s)
{
    switch (s) {
        case SAL_OK: return "SAL_OK";
        case SAL_ERR_INVALID_ARG: return "SAL_ERR_INVALID_ARG";
        case SAL_ERR_UNSUPPORTED: return "SAL_ERR_UNSUPPORTED";
        case SAL_ERR_WORKSPACE: return "SAL_ERR_WORKSPACE";
        case SAL_ERR_CUDA: return "SAL_ERR_CUDA";
        case SAL_ERR_TIMEOUT: return "SAL_ERR_TIMEOUT";
        case SAL_ERR_INTERNAL: return "SAL_ERR_INTERNAL";
    }
    return "SAL_ERR_UNKNOWN";
}

const char *sal_last_error(void) { return g_err; }

}  // extern "C"
