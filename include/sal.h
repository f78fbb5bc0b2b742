/*
 * sal.h - C ABI of the GB300 seismic saliency library (libsal.so).
 *
 * The method is the one of Shafiq, Long, Alshawi and AlRegib, "Saliency detection for
 * seismic applications using multi-dimensional spectral projections and directional
 * comparisons" (ICIP 2017), Sec. 2 and Fig. 1:
 *   (1) a local 3D DFT of an L x L x L cube around every voxel (the DFT printed below Eq. 2),
 *   (2) projection of each spectral point onto the three planes (Eq. 1-4), DC excluded,
 *   (3) the absolute mean of each projected cube: spectral energies E_t, E_x, E_y,
 *   (4) directional centre-surround comparison of each E_m (Eq. 5): maps S_t, S_x, S_y,
 *   (5) their weighted combination (Eq. 6) into the saliency map S, the size of V.
 *
 * Conventions shared by every call
 *  - Volumes are float32, C order [t][x][y] (t = time/depth, x = crossline, y = inline,
 *    y contiguous), T*X*Y voxels.  Per-map arrays are planar: [3][T*X*Y] for m = t, x, y.
 *  - Every data pointer is a DEVICE pointer owned by the caller.  The library allocates
 *    and frees nothing; scratch goes in the caller's workspace `ws` (size from the
 *    matching *_workspace_size query).  Device pointers must be 16-byte aligned.
 *  - Calls are asynchronous on the caller's CUDA stream `stream` (a cudaStream_t passed
 *    as void*; NULL = the legacy default stream).  They return once work is enqueued.
 *  - Arguments are checked on the host before anything is launched; a bad argument
 *    returns SAL_ERR_INVALID_ARG (or SAL_ERR_UNSUPPORTED, SAL_ERR_WORKSPACE) and launches
 *    nothing.  A CUDA launch error returns SAL_ERR_CUDA.  sal_last_error() gives a
 *    thread-local message for the last failing call.  No C++ exception crosses the ABI.
 *  - Readings of the paper that these calls implement:
 *      centred signed frequency indices -h..h (h = (L-1)/2) in Eq. 1-4, so the DC point
 *      is the cube centre; features use |F|; the energy is the mean over the L^3 - 1
 *      non-DC points; one cube per voxel, centred on it, odd L; samples outside the
 *      volume come from the boundary extension (REFLECT: whole-sample symmetric without
 *      repeating the edge; PERIODIC: wrap); Eq. 5 is taken literally with Gaussian
 *      weights g(o) = exp(-|o|^2 / (2 sigma^2)) on the neighbour; each S_m is min-max
 *      normalised with its global min and max before Eq. 6, and a map whose range
 *      hi - lo <= eps * max(|hi|, |lo|) becomes 0.
 */
#ifndef SAL_H
#define SAL_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SAL_API __attribute__((visibility("default")))
#else
#define SAL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SAL_OK = 0,
    SAL_ERR_INVALID_ARG = 1,  /* null pointer, bad size, misaligned pointer, bad enum */
    SAL_ERR_UNSUPPORTED = 2,  /* valid request this build does not implement (e.g. even L) */
    SAL_ERR_WORKSPACE = 3,    /* workspace smaller than the size query returned */
    SAL_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed; see sal_last_error() */
    SAL_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out */
    SAL_ERR_INTERNAL = 6
} sal_status;

typedef enum { SAL_PREC_FP32 = 0, SAL_PREC_TF32 = 1, SAL_PREC_BF16 = 2 } sal_precision;
typedef enum { SAL_BND_REFLECT = 0, SAL_BND_PERIODIC = 1 } sal_boundary;
/* SAL_STENCIL_26: the 26 voxels around the centre (Q = 26).
 * SAL_STENCIL_LINE: the paper's d x 1 window of side d = L along axis m for map m
 * (offsets +-1..+-h, Q = L - 1), Sec. 2 text after Eq. 5.
 * SAL_STENCIL_DIAG_TX: the d x 1 window of side d = L along the t-x diagonal (Fig. 3), the
 * same for every map: offsets (k, k, 0), k = +-1..+-h, Q = L - 1, weights
 * g = exp(-2 k^2 / (2 sigma^2)).
 * Any other neighbourhood (orientation, size and weights tuned as the text after Eq. 5
 * allows) goes through sal_directional_compare_user. */
typedef enum { SAL_STENCIL_26 = 0, SAL_STENCIL_LINE = 1, SAL_STENCIL_DIAG_TX = 2 } sal_stencil;

typedef struct { int64_t T, X, Y; } sal_dims;

typedef struct {
    int32_t L;          /* local cube side, odd, 3..15 (Sec. 2: "L defines the size of the local data cube") */
    int32_t precision;  /* sal_precision of the DFT stage: FP32 on the CUDA cores (any L); the
                           y-stage on the tensor cores with BF16 (any L) or TF32 (L <= 11)
                           operands and FP32 accumulation; SAL_ERR_UNSUPPORTED otherwise */
    int32_t boundary;   /* sal_boundary */
    int32_t stencil;    /* sal_stencil */
    float sigma;        /* Gaussian width of the Eq. 5 weights, in voxels (> 0) */
    int32_t stride;     /* cube centres (Sec. 2, first step: the cube slides with more than 50 %
                           overlap): 0 or 1 = one cube per voxel; s in 2..(L-1)/2 = cubes centred
                           on the lattice min(i s, n - 1) of every axis, E interpolated
                           trilinearly back to every voxel (sal_saliency, sal_saliency_host
                           and the split calls sal_lattice_energy / sal_interpolate_lattice;
                           FP32 only; the other energy entry points return
                           SAL_ERR_UNSUPPORTED for s > 1) */
    double a, b, c;     /* Eq. 6 weights of S_t, S_x, S_y (equal in the paper) */
    double eps;         /* relative range below which a map counts as constant */
} sal_params;

/* Largest number of volumes one batched call takes. */
#define SAL_BATCH_MAX 128

/* Number of doubles in a stats array: (min, max, sum) of S_t, S_x, S_y in that order. */
#define SAL_STATS_LEN 9

/* Fill *p with the defaults: L = 7, FP32, REFLECT, 26-neighbourhood, sigma = 1,
 * a = b = c = 1/3 (the paper's equal weights, Sec. 2 after Eq. 6), eps = 1e-6. */
SAL_API sal_status sal_params_default(sal_params *p);

/* Workspace bytes needed by sal_saliency for this volume and these parameters. */
SAL_API sal_status sal_workspace_size(sal_dims dims, const sal_params *p, size_t *bytes);

/* Workspace bytes needed by sal_directional_compare. */
SAL_API sal_status sal_dcs_workspace_size(sal_dims dims, const sal_params *p, size_t *bytes);

/*
 * Local magnitude spectra (Sec. 2 first step; the DFT printed below Eq. 2, normalised by
 * L^-3) of the voxels of a region of interest: roi_lo[3] = first voxel (t, x, y),
 * roi_ext[3] = extent; the region must lie inside the volume.  `mag` receives
 * [roi voxels in C order][L][L][L] float32, frequency slots in centred order
 * (slot s holds signed index s - h); the DC slot holds |mean of the cube|.
 * Meant for inspection and tests (L^3 floats per voxel): keep the region small.
 */
SAL_API sal_status sal_local_spectra(const float *V, sal_dims dims, const sal_params *p,
                             const int64_t roi_lo[3], const int64_t roi_ext[3],
                             float *mag, void *stream);

/*
 * Spectral energies from magnitude spectra (Eq. 1-4 and the third step of Sec. 2):
 * E_m[v] = (L^3 - 1)^-1 sum over non-DC points of w_m |F|.  `mag` is [n_vox][L][L][L] in the
 * layout sal_local_spectra writes; `E` receives [3][n_vox].
 */
SAL_API sal_status sal_project(const float *mag, int64_t n_vox, int32_t L, float *E, void *stream);

/*
 * Fused steps 1-3 for a whole volume: E [3][T*X*Y] straight from V, no spectrum stored.
 * p->precision selects the DFT arithmetic (FP32 CUDA cores, or TF32/BF16 tensor cores
 * with FP32 accumulation).
 */
SAL_API sal_status sal_spectral_energy(const float *V, sal_dims dims, const sal_params *p, float *E,
                               void *stream);

/*
 * Coarse-stride cubes (p->stride = s > 1; Sec. 2, first step).  Along an axis of n samples
 * the cube centres are c_i = min(i s, n - 1), i = 0 .. n_c - 1, n_c = ceil((n - 1) / s) + 1
 * (n_c = 1 for n = 1).  sal_lattice_dims gives (Tc, Xc, Yc); sal_lattice_energy writes E_m of
 * the cube centred on every lattice point, Ec [3][Tc][Xc][Yc] (device); sal_interpolate_lattice
 * writes E [3][T][X][Y] (device), each voxel the trilinear interpolation of the 2 x 2 x 2
 * lattice energies around it (exact at the lattice points).  FP32 on the CUDA cores; with
 * s = 0 or 1 the lattice is every voxel.  The interpolation keeps a table of the lattice
 * segment of every t, x and y in shared memory: T + X + Y up to about 24,000 (beyond,
 * SAL_ERR_CUDA from the launch).
 * Asynchronous; errors as the other calls.
 */
SAL_API sal_status sal_lattice_dims(sal_dims dims, const sal_params *p, sal_dims *lattice);
SAL_API sal_status sal_lattice_energy(const float *V, sal_dims dims, const sal_params *p, float *Ec, void *stream);
SAL_API sal_status sal_interpolate_lattice(const float *Ec, sal_dims dims, const sal_params *p, float *E, void *stream);

/*
 * Directional centre-surround comparison, Eq. 5, of each E_m: Sm [3][T*X*Y], plus the
 * global (min, max, sum) of each S_m in `stats` (device, SAL_STATS_LEN doubles; the
 * reductions are FP64).  `ws` must hold sal_dcs_workspace_size bytes.  The line and
 * offset-list stencils address a plane by 32-bit offsets: with them X * Y must stay below
 * 2^31 (beyond, SAL_ERR_CUDA from the launch), in every call that runs the compare.
 */
SAL_API sal_status sal_directional_compare(const float *E, sal_dims dims, const sal_params *p,
                                   float *Sm, double *stats, void *ws, size_t ws_bytes,
                                   void *stream);

/*
 * Caller-given neighbourhoods for Eq. 5 (the text after Eq. 5: the comparison window can be
 * tuned in orientation, size and weights; Fig. 3 shows lines along t, x and the t-x diagonal).
 * For map m: count[m] offsets offset[m][k] = (dt, dx, dy) with weights weight[m][k], and
 *   S_m[v] = count[m]^-1 sum_k | E_m[v] - weight[m][k] E_m[v + offset[m][k]] |.
 * Limits: 1 <= count[m] <= SAL_STENCIL_MAX_OFFSETS; every component in
 * [-SAL_STENCIL_MAX_RADIUS, SAL_STENCIL_MAX_RADIUS]; no offset (0, 0, 0); finite weights.
 * Host memory, read during the call only.
 */
#define SAL_STENCIL_MAX_OFFSETS 64
#define SAL_STENCIL_MAX_RADIUS 7
typedef struct {
    int32_t count[3];
    int32_t offset[3][SAL_STENCIL_MAX_OFFSETS][3];
    float weight[3][SAL_STENCIL_MAX_OFFSETS];
} sal_user_stencil;

/*
 * sal_directional_compare with the neighbourhood of `st` instead of p->stencil (p gives the
 * boundary extension; its other fields are checked but unused).  Outputs and workspace as
 * for sal_directional_compare (sal_dcs_workspace_size bytes).  SAL_ERR_INVALID_ARG for a
 * stencil outside the limits above.
 */
SAL_API sal_status sal_directional_compare_user(const float *E, sal_dims dims, const sal_params *p,
                                                const sal_user_stencil *st, float *Sm, double *stats, void *ws,
                                                size_t ws_bytes, void *stream);

/*
 * Weighted combination, Eq. 6, of the min-max normalised maps:
 * S = a N_t + b N_x + c N_y with N_m = (S_m - min_m) / (max_m - min_m).  `stats` is the
 * device array sal_directional_compare wrote.
 */
SAL_API sal_status sal_combine(const float *Sm, const double *stats, sal_dims dims, const sal_params *p,
                       float *S, void *stream);

/*
 * The whole method of Fig. 1 on one volume: V -> S.  `stats` (device, SAL_STATS_LEN
 * doubles) may be NULL; otherwise it receives the S_m statistics.  `ws` must hold
 * sal_workspace_size bytes (it holds E, S_m and the reduction partials).
 */
SAL_API sal_status sal_saliency(const float *V, sal_dims dims, const sal_params *p, float *S,
                        double *stats, void *ws, size_t ws_bytes, void *stream);

/*
 * The whole method of Fig. 1 on a volume in HOST memory: copies V_host to the device,
 * computes S as sal_saliency does, and copies S back to S_host.  Successive calls on the
 * same workspace overlap: the copy of the next call's V, this call's kernels and the copy
 * of the previous call's S run on separate streams (V and S are double-buffered inside the
 * workspace), so a sequence of calls runs at the speed of the kernels when the copies are
 * shorter.
 *   V_host, S_host: host memory, T*X*Y floats each; page-locked memory (cudaHostAlloc,
 *     cudaHostRegister) is needed for the overlap, pageable memory works but copies
 *     synchronously.  V_host may be reused as soon as the stream has passed the copy
 *     (the library does not read it later).
 *   stats: device, SAL_STATS_LEN doubles, or NULL.
 *   ws: device workspace of sal_host_workspace_size bytes, owned by the caller; one
 *     sequence of calls per workspace at a time (the library keeps, per workspace pointer,
 *     the parity of its double buffers and the events that order them).
 *   done_event: a cudaEvent_t created by the caller, or NULL.  If NULL, `stream` waits for
 *     the copy of S (S_host is ready once `stream` completes).  Otherwise the event is
 *     recorded after the copy of S and `stream` does not wait for it, so the next call's
 *     kernels can run during this copy; S_host is ready once the event completes.
 * Not for use during stream capture.  Errors as sal_saliency; SAL_ERR_CUDA for a failed
 * copy, stream or event call.
 */
SAL_API sal_status sal_host_workspace_size(sal_dims dims, const sal_params *p, size_t *bytes);
SAL_API sal_status sal_saliency_host(const float *V_host, sal_dims dims, const sal_params *p, float *S_host,
                                     double *stats, void *ws, size_t ws_bytes, void *stream, void *done_event);
/* Waits for and destroys the streams and events kept for workspace ws (none: no-op). */
SAL_API sal_status sal_host_release(void *ws);

/* ---- Slabs along t ------------------------------------------------------------------------
 * One volume of T planes split into slabs that run on different GPUs (one process per GPU)
 * or on one GPU in turn.  The method's only global step is the normalisation before Eq. 6,
 * which needs the (min, max) of each S_m over the whole volume: every other value depends on
 * a bounded neighbourhood.  E at a voxel needs V within h = (L-1)/2 planes, and S_m needs E
 * within r_t planes (r_t = 1 for the 26-neighbourhood, h for the line and t-x diagonal
 * stencils).  So a slab that owns the planes [own_lo, own_hi) is given the planes
 * [ext_lo, ext_hi) of V, ext_lo = max(0, own_lo - H), ext_hi = min(T, own_hi + H), with
 * H = h + r_t from sal_slab_halo, and:
 *   1. sal_slab_maps: steps 1-4 on those planes; S_m of its own planes into Sm_own
 *      ([3][own_hi - own_lo][X][Y]) and their (min, max, sum) into stats_local (9 doubles);
 *   2. the 9 doubles of every slab are gathered (between ranks: one all-gather of 9 doubles
 *      per rank, the only exchange) and merged by sal_stats_merge;
 *   3. sal_combine(Sm_own, merged stats, {own_hi - own_lo, X, Y}) gives the slab's S.
 * S_m and S equal those of sal_saliency on the whole volume bit for bit when both use the
 * same spectral-energy tile shape (the autotuner's choice per L, precision and size class:
 * each value is then computed from the same samples in the same order), else within
 * rounding; the sums differ only in rounding.
 * PERIODIC wraps t from the last plane to the first, which a slab does not hold: with it a
 * slab must be the whole volume (SAL_ERR_UNSUPPORTED otherwise).
 */
SAL_API sal_status sal_slab_halo(const sal_params *p, int64_t *planes);
/* Workspace of sal_slab_maps for a slab given ext_planes = ext_hi - ext_lo planes of V. */
SAL_API sal_status sal_slab_workspace_size(int64_t ext_planes, int64_t X, int64_t Y, const sal_params *p,
                                           size_t *bytes);
/* dims: the WHOLE volume (T, X, Y).  V_ext: device, the planes [ext_lo, ext_hi) of V
 * (ext_lo, ext_hi exactly as above, else SAL_ERR_INVALID_ARG).  Sm_own, stats_local: device
 * outputs (sizes above); ws: device, sal_slab_workspace_size bytes.  Asynchronous. */
SAL_API sal_status sal_slab_maps(const float *V_ext, sal_dims dims, int64_t ext_lo, int64_t ext_hi, int64_t own_lo,
                                 int64_t own_hi, const sal_params *p, float *Sm_own, double *stats_local, void *ws,
                                 size_t ws_bytes, void *stream);
/* Merges n statistics records (device, [n][9], (min, max, sum) per map) into out (device,
 * 9 doubles): min of the minima, max of the maxima, FP64 sum of the sums in record order. */
SAL_API sal_status sal_stats_merge(const double *stats, int32_t n, double *out, void *stream);

/*
 * Directional compare for callers that cannot allocate device memory.
 *
 * The same computation and kernels as sal_directional_compare, but without a workspace
 * argument: the scratch for the per-tile reduction records is a fixed array inside the
 * library.  It serves callers that may not allocate device memory themselves, for example
 * a plug-in whose host application owns the whole GPU memory budget and forbids
 * allocations by its plug-ins, or a processing loop that must never enter the allocator.
 * The paper has no counterpart of this call; it is an interface convenience.
 *
 * Limits and behaviour:
 *  - the volume may need at most SAL_DCS_STATIC_MAX_TILES tiles of 8 x 8 x 64 voxels
 *    (ceil(T/8) * ceil(X/8) * ceil(Y/64)); a larger volume returns SAL_ERR_WORKSPACE and
 *    launches nothing.  The array takes 9 * (SAL_DCS_STATIC_MAX_TILES + 160) doubles,
 *    about 9.4 MB, on every GPU that loads the library, until the process exits;
 *  - the first call on a device looks up the array's device address (a one-time set-up
 *    for that device, repeated only if the device's context changes, e.g. after
 *    cudaDeviceReset); make that first call before any stream capture;
 *  - every call shares the one array and overwrites every record it reads, so nothing has
 *    to be cleared between calls; two calls whose kernels overlap on the GPU (different
 *    streams, or different host threads on one device) race on it and must be ordered by
 *    the caller;
 *  - E, Sm and stats are the caller's device memory, as for sal_directional_compare;
 *    this entry point calls no allocation routine.
 */
#define SAL_DCS_STATIC_MAX_TILES 131072
SAL_API sal_status sal_directional_compare_static(const float *E, sal_dims dims, const sal_params *p,
                                                  float *Sm, double *stats, void *stream);

/* ---- Many uneven volumes at once --------------------------------------------------------
 * One volume of a batch: device pointers owned by the caller (V input, S output), both
 * float32 C order [T][X][Y] and 16-byte aligned. */
typedef struct {
    const float *V;
    float *S;
    int64_t T, X, Y;
} sal_volume;

/* Workspace bytes for sal_saliency_batched / sal_graph_create_batched over these volumes
 * (per volume: E and S_m, 24 bytes per voxel, and its reduction records). */
SAL_API sal_status sal_batch_workspace_size(const sal_volume *vols, int32_t n, const sal_params *p,
                                            size_t *bytes);

/*
 * The whole method (Fig. 1) on n <= SAL_BATCH_MAX independent volumes of any sizes, each
 * stage as ONE persistent launch over the tiles of all volumes: spectral energies,
 * directional compare, per-volume FP64 statistics, combination.  Results equal those of
 * sal_saliency on each volume.  `vols` is a host array; `stats` (device, n * 9 doubles,
 * volume-major) may be NULL.  The spectral-energy tile shape is the autotuner's choice
 * for (L, precision, size class of the largest volume) when one is cached, else the default.
 */
SAL_API sal_status sal_saliency_batched(const sal_volume *vols, int32_t n, const sal_params *p,
                                        double *stats, void *ws, size_t ws_bytes, void *stream);

/*
 * The same batch captured once into a CUDA graph and replayed with sal_graph_launch.
 * Creation may run the autotuner first (when no tile shape is cached for the batch), which
 * times candidate launches on `stream` and synchronises it; the capture itself runs on a
 * private stream.  The graph keeps the pointers it was built with: the volumes, `stats`
 * and `ws` must stay valid and unchanged in size until sal_graph_destroy.  Host memory for
 * the graph object is the only allocation; no device memory is allocated by the library.
 */
typedef struct sal_graph sal_graph;
SAL_API sal_status sal_graph_create_batched(const sal_volume *vols, int32_t n, const sal_params *p,
                                            double *stats, void *ws, size_t ws_bytes, void *stream,
                                            sal_graph **out);
/* Replays the captured batch on `stream` (asynchronous). */
SAL_API sal_status sal_graph_launch(sal_graph *g, void *stream);
SAL_API sal_status sal_graph_destroy(sal_graph *g);

/* ---- Autotuner of the spectral-energy tile shape ----------------------------------------
 * A choice: cube side, precision, size class (0: fewer than 16 Mi voxels per volume,
 * 1: larger), candidate index, its BT x BX x BY output tile and staging mode (0: all
 * intermediate spectra of a mu in shared memory; 1: the lines of one (mu, |nu|) at a time;
 * 2: as 1, with stage t rerun per mu; 3: as 0, the next tile's halo copied while the current
 * one is computed; 4: as 0, the spectra of a mu in batches of a few lines, so that one more
 * CTA fits an SM (L = 7, 9)), and its measured time. */
typedef struct {
    int32_t L, precision, size_class, shape;
    int32_t bt, bx, by, mode;
    float ms;
} sal_tile_choice;

/* Times every candidate tile shape of the spectral-energy kernel on this volume (E is a
 * device buffer of 3 * T * X * Y floats it may overwrite), caches the fastest for the
 * process and returns it.  Synchronises `stream`: not for use during stream capture. */
SAL_API sal_status sal_autotune(const float *V, sal_dims dims, const sal_params *p, float *E, void *stream,
                                sal_tile_choice *out);
/* The same over a batch (times the persistent batched launch; ws as for the batch). */
SAL_API sal_status sal_autotune_batched(const sal_volume *vols, int32_t n, const sal_params *p, void *ws,
                                        size_t ws_bytes, void *stream, sal_tile_choice *out);
/* The shape the calls would use now for a volume of n_vox voxels (the default when none is cached). */
SAL_API sal_status sal_autotune_query(int32_t L, int32_t precision, int64_t n_vox, sal_tile_choice *out);
/* Saves / loads the cache as text; a malformed file is refused (SAL_ERR_INVALID_ARG) and
 * leaves the cache unchanged.  clear empties it. */
SAL_API sal_status sal_autotune_save(const char *path);
SAL_API sal_status sal_autotune_load(const char *path);
SAL_API sal_status sal_autotune_clear(void);

/* ---- Learned surrogate of the spectral energies ------------------------------------------
 * SAL_SURR_LAYERS layers of 3x3x3 convolution (1 -> SAL_SURR_WIDTH -> ... -> 3 channels), GELU
 * after all but the last, predicting E_t, E_x, E_y from the amplitudes.  Input and target are
 * divided by the volume's RMS amplitude inside (E scales with the amplitude, so the network
 * sees one scale).  Parameters: one flat FP32 array, layer by layer, weights
 * [Cout][Cin][3][3][3] then biases [Cout]; the kernels round the weights to BF16 as they read
 * them and accumulate in FP32.  The paper has no learned part: this is an added surrogate
 * whose errors are measured against the method it imitates. */
#define SAL_SURR_LAYERS 5
#define SAL_SURR_WIDTH 24
SAL_API sal_status sal_surrogate_param_count(int64_t *n);
/* Workspace for sal_surrogate_forward (training = 0: BF16 activations, 48 B/voxel; training
 * = 1: every FP32 activation kept for the backward pass, 972 B/voxel). */
SAL_API sal_status sal_surrogate_workspace_size(sal_dims dims, int32_t training, size_t *bytes);
/* E [3][T*X*Y] predicted from V (device pointers).  With training = 1 the activations stay in
 * `ws` for sal_surrogate_backward (FP32 activations, CUDA cores).  With training = 0 the
 * activations are BF16; p->precision = SAL_PREC_BF16 then runs layers 2..5 (24 input
 * channels) as tcgen05 products (BF16 operands, FP32 accumulation; bounded waits, a timeout
 * reported by sal_device_status), any other precision keeps every layer on the CUDA cores.
 * sal_surrogate_infer follows the same rule. */
SAL_API sal_status sal_surrogate_forward(const float *V, sal_dims dims, const sal_params *p, const float *params,
                                         float *E, int32_t training, void *ws, size_t ws_bytes, void *stream);
/* Gradient of L = 0.5 / count * sum (E_pred - E_target)^2 / rms^2 over voxels at least
 * `margin` (>= SAL_SURR_LAYERS) from every face, for the activations of the last training
 * forward in `ws`.  grads (FP32, param_count) is overwritten; *loss (device double) receives L. */
SAL_API sal_status sal_surrogate_backward(const float *V, sal_dims dims, const sal_params *p, const float *params,
                                          const float *E_target, int32_t margin, float *grads, double *loss,
                                          void *ws, size_t ws_bytes, void *stream);
/*
 * Inference with the plain method as the judge and the fallback: E predicted for the whole
 * volume, then, for every check block of 16 x 16 x 32 voxels, E computed exactly (FP32
 * path) at 8 sample voxels; a block whose largest error, relative to each map's mean
 * magnitude over all samples, exceeds `threshold` (e.g. 2e-2) is recomputed exactly.
 * counts (device, 2 ints, nullable) receives (blocks recomputed, blocks checked).
 */
SAL_API sal_status sal_surrogate_infer_workspace_size(sal_dims dims, const sal_params *p, size_t *bytes);
SAL_API sal_status sal_surrogate_infer(const float *V, sal_dims dims, const sal_params *p, const float *params,
                                       float *E, float threshold, int32_t *counts, void *ws, size_t ws_bytes,
                                       void *stream);
/* One Adam step (bias-corrected, step >= 1) on the FP32 parameters with moments m, v. */
SAL_API sal_status sal_surrogate_adam_step(float *params, const float *grads, float *m, float *v, int32_t step,
                                           float lr, float beta1, float beta2, float eps, void *stream);

/*
 * Synchronises `stream`, then reads and clears the library's device status word on the
 * current device: SAL_OK, or SAL_ERR_TIMEOUT when a bounded device-side wait of a
 * tensor-core kernel (precision TF32 or BF16) ran out since the last call; the outputs of
 * such a launch are undefined.
 */
SAL_API sal_status sal_device_status(void *stream);

/* Test hook: while on, the tensor-core kernels withhold every product, so each of their
 * bounded waits runs out (after about 20 ms) and sal_device_status reports
 * SAL_ERR_TIMEOUT.  Off by default; never needed in normal use. */
SAL_API sal_status sal_test_stall_tensor_cores(int32_t on);

/*
 * Measurement helper, not part of the method: the FP32 FMA rate of this GPU, the denominator
 * of the spectral-energy kernel's ALU roofline.  Launches n_threads / 256 blocks of 256
 * threads; each thread runs SAL_PROBE_CHAINS independent chains of `iters` FMAs
 * (x <- x * a + b) and writes one float to out[thread] (device, n_threads floats, so nothing
 * is optimised away).  packed = 0 issues scalar FFMA, packed = 1 the fma.rn.f32x2 form
 * (two chains per instruction).  FP32 flops of one launch = 2 * SAL_PROBE_CHAINS * iters *
 * n_threads; time it with events on `stream`.  n_threads must be a positive multiple of 256
 * and iters a positive multiple of 16, else SAL_ERR_INVALID_ARG; SAL_ERR_CUDA if the launch
 * fails.  Asynchronous on `stream`; allocates nothing.
 */
#define SAL_PROBE_CHAINS 8
SAL_API sal_status sal_probe_fma_rate(float *out, int64_t n_threads, int32_t iters, int32_t packed, void *stream);

/* Static text for a status code. */
SAL_API const char *sal_status_string(sal_status s);
/* Thread-local detail of the last failing call on this thread ("" if none). */
SAL_API const char *sal_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SAL_H */
