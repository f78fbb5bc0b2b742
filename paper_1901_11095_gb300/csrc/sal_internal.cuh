// Internal declarations shared by the CUDA translation units of libsal.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sal.h"

namespace sal {

constexpr int kMaxL = 15;
constexpr int kMaxH = (kMaxL - 1) / 2;
constexpr int kMaxHalf = kMaxH + 1;

// Per-L tables the kernels read from the parameter constant bank.
//   cs[n], sn[n] = cos(2 pi n / L), sin(2 pi n / L), n = 0..L-1
//   w[((mu*kMaxHalf + |nu|)*kMaxHalf + |om|)*3 + m] = projection weight of Eq. 1-4 for
//   map m at (mu, +-nu, +-om), mu >= 0 (the weights depend on squares only)
//   escale = 2 / ((L^3 - 1) L^3): DFT normalisation L^-3, the non-DC mean (L^3-1)^-1 and
//   the factor 2 of the half spectrum (|F(-k)| = |F(k)| for real input)
struct SpecTables {
    float cs[16];
    float sn[16];
    float w[kMaxHalf * kMaxHalf * kMaxHalf * 3];
    float escale;
};

// Fills the tables on the host (double precision, then rounded).
void make_tables(int L, SpecTables *t);

// Boundary extension of one coordinate onto 0..n-1 (REFLECT: whole-sample symmetric,
// edge not repeated; PERIODIC: wrap).  Valid for any integer i; coordinates at most one
// reflection or wrap away take a division-free path.
__host__ __device__ __forceinline__ int64_t ext_index(int64_t i, int64_t n, int bnd)
{
    if (i >= 0 && i < n) return i;
    if (bnd == SAL_BND_PERIODIC) {
        if (i < 0 && i >= -n) return i + n;
        if (i >= n && i < 2 * n) return i - n;
        int64_t r = i % n;
        return r < 0 ? r + n : r;
    }
    if (n == 1) return 0;
    if (i < 0 && i > -n) return -i;
    if (i >= n && i <= 2 * n - 2) return 2 * (n - 1) - i;
    int64_t period = 2 * (n - 1);
    int64_t r = i % period;
    if (r < 0) r += period;
    return r < n ? r : period - r;
}

constexpr int kMaxBatch = SAL_BATCH_MAX;

// One volume of a (possibly batched) spectral-energy launch.
struct EVolDesc {
    const float *V;
    float *E;
    int64_t T, X, Y;
    // FP32 kernel, single volume only: compute the output planes [t_lo, t_hi) (both multiples
    // of every candidate BT, or t_hi = T); t_hi < 0 means the whole volume
    int64_t t_lo = 0, t_hi = -1;
};

// Tile shapes of the spectral-energy kernel that the autotuner chooses among.
struct TileShape {
    int bt, bx, by, mode;   // mode: how the spectra of a tile are held in shared memory (0..3)
};
constexpr int kMaxShapes = 6;
int energy_num_shapes(int L);
TileShape energy_shape(int L, int idx);

// Control of the tensor-core kernels: where a timed-out wait is recorded, the test hook
// that withholds every product, and the bound of one wait.
struct TcControl {
    int *status;
    int stall;
    unsigned long long limit_ns;
};
bool energy_tc_supported(int L, int prec);
// Unique id of the CUDA context current on this thread (driver cuCtxGetId, reached through the
// runtime's driver entry points); a device reset or a new primary context gives a new id, so
// device addresses cached per (device, id) are never reused from a destroyed context.
cudaError_t current_context_id(unsigned long long *id);
int *device_status_ptr();
TcControl tc_control();
void set_test_stall(int on);
cudaError_t launch_energy_tc(const EVolDesc *vols, int n, int L, int bnd, int prec, bool persistent,
                             const TcControl &c, cudaStream_t s);

cudaError_t launch_energy_fp32_list(const float *V, sal_dims d, int L, int bnd, const int64_t *list, const int *count,
                                    float *E, cudaStream_t s);

// Opts a kernel into `bytes` of dynamic shared memory and asks for the largest shared-memory
// carveout, so that several CTAs of a large-tile kernel can be resident on one SM.
template <class F>
inline cudaError_t set_smem(F fn, size_t bytes)
{
    cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    return e;
}

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_energy_fp32_batch(const EVolDesc *vols, int n, int L, int bnd, int shape_idx, bool persistent,
                                     cudaStream_t s);
cudaError_t launch_energy_fp32(const float *V, sal_dims d, int L, int bnd, float *E, cudaStream_t s);
cudaError_t launch_local_spectra(const float *V, sal_dims d, int L, int bnd, const int64_t lo[3],
                                 const int64_t ext[3], float *mag, cudaStream_t s);
// E_m at a list of voxels coords[k] = (t, x, y) (device, [n][3]): E[m * n + k].
cudaError_t launch_energy_points(const float *V, sal_dims d, int L, int bnd, const int64_t *coords, int64_t n, float *E,
                                 cudaStream_t s);
cudaError_t launch_project(const float *mag, int64_t n, int L, float *E, cudaStream_t s);

// One volume of a (possibly batched) directional-compare launch; `part` receives the
// volume's [9][tiles] partial records.
// Output planes [o_lo, o_hi) of E's T planes (o_hi < 0: all of them); Sm holds the output
// planes only, [3][o_hi - o_lo][X][Y].
struct DVolDesc {
    const float *E;
    float *Sm;
    double *part;
    int64_t T, X, Y;
    int64_t o_lo = 0, o_hi = -1;
};
// `user` (offset lists per map) replaces p->stencil when not NULL.
cudaError_t launch_dcs_items(const DVolDesc *vols, int n, const sal_params *p, cudaStream_t s,
                             const sal_user_stencil *user = nullptr);
// The t-x diagonal line of side L as an offset list, and the largest |dt| of a list.
sal_user_stencil diag_tx_stencil(const sal_params *p);
int dcs_user_radius_t(const sal_user_stencil &st);
// Merges n statistics records [n][9] into one (min, max, FP64 sum).
cudaError_t launch_stats_merge(const double *in, int n, double *out, cudaStream_t s);

// Directional compare: capacity of partial records in the workspace (per map, any stencil,
// plus the first reduction pass), and the records one map of a launch writes.
int64_t dcs_num_partials(sal_dims d);
int64_t dcs_num_records(sal_dims d);
cudaError_t launch_dcs(const float *E, sal_dims d, const sal_params *p, float *Sm, double *partials,
                       double *stats, cudaStream_t s, const sal_user_stencil *user = nullptr, int64_t o_lo = 0,
                       int64_t o_hi = -1);
// Fixed-scratch variant of the directional compare (no allocation by caller or library).
int64_t dcs_num_tiles(sal_dims d);
cudaError_t dcs_static_scratch(double **out);
// Per-volume statistics and Eq. 6 for a batch (one launch each).
struct BatchVolDesc {
    const float *Sm;
    float *S;
    const double *part;
    int64_t tiles, N;
};
cudaError_t launch_batch_stats_combine(const BatchVolDesc *vols, int n, const sal_params *p, double *stats,
                                       cudaStream_t s);

// Autotuner cache of spectral-energy tile shapes, keyed by (L, precision, size class).
int size_class_of(int64_t n_vox);
int autotune_lookup(int L, int precision, int size_class);
bool autotune_get_ms(int L, int precision, int size_class, float *ms);
void autotune_store(int L, int precision, int size_class, int shape, float ms);
// Times every candidate shape on the given volumes (batched when n > 1), stores and
// returns the fastest; synchronises the stream.
cudaError_t autotune_run(const EVolDesc *vols, int n, int L, int bnd, int precision, cudaStream_t s, int *best,
                         float *best_ms);
int autotune_save(const char *path);
int autotune_load(const char *path);
void autotune_clear();

// Learned surrogate of the spectral energies.
int64_t surrogate_param_count();
size_t surrogate_ws_bytes(sal_dims d, bool training);
cudaError_t surrogate_forward(const float *V, sal_dims d, int bnd, const float *params, float *E, bool training,
                              void *ws, cudaStream_t s, int prec = SAL_PREC_FP32, const TcControl *tc = nullptr);
cudaError_t surrogate_backward(const float *V, sal_dims d, int bnd, const float *params, const float *Etarget,
                               int margin, float *grads, double *loss, void *ws, cudaStream_t s);
size_t surrogate_infer_ws_bytes(sal_dims d, int L);
cudaError_t surrogate_infer(const float *V, sal_dims d, int L, int bnd, const float *params, float *E, float thr,
                            int *counts, void *ws, cudaStream_t s, int prec = SAL_PREC_FP32, const TcControl *tc = nullptr);
cudaError_t surrogate_adam(float *params, const float *grads, float *m, float *v, int64_t n, int step, float lr,
                           float b1, float b2, float eps, cudaStream_t s);

// Coarse-stride cubes: lattice size along an axis, E at the lattice points, interpolation back.
int64_t lattice_size(int64_t n, int s);
cudaError_t launch_lattice_energy(const float *V, sal_dims d, int L, int bnd, int s, float *Ec, cudaStream_t st);
cudaError_t launch_interp_lattice(const float *Ec, sal_dims d, int s, float *E, cudaStream_t st);

// FP32 FMA-rate probe: n_threads / 256 blocks, SAL_PROBE_CHAINS chains of `iters` FMAs per thread.
cudaError_t launch_fma_probe(float *out, int64_t n_threads, int iters, bool packed, cudaStream_t stream);

cudaError_t launch_combine(const float *Sm, const double *stats, sal_dims d, const sal_params *p, float *S,
                           cudaStream_t s);

}  // namespace sal
