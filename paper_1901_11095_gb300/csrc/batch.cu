// Batched form of the path for many uneven volumes: the per-volume FP64 statistics and the
// normalised combination (Eq. 6) over a whole batch, each as one persistent launch.  The
// spectral-energy and directional-compare launches of a batch are the batched forms of
// their single-volume kernels (one persistent grid walks every tile of every volume).
#include <float.h>

#include "sal_internal.cuh"

namespace sal {

namespace {

struct RVol {
    const double *part;   // [9][tiles]
    int64_t tiles;
};
struct RBatch {
    int n;
    RVol v[kMaxBatch];
};

// Block v reduces the partial records of volume v into stats[9 v .. 9 v + 8] (FP64, fixed order).
__global__ void __launch_bounds__(256) reduce_volumes_kernel(const __grid_constant__ RBatch rb, double *__restrict__ stats)
{
    __shared__ double red[8][9];
    const int vi = blockIdx.x;
    if (vi >= rb.n) return;
    const RVol &v = rb.v[vi];
    double acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = q % 3 == 0 ? DBL_MAX : (q % 3 == 1 ? -DBL_MAX : 0.0);
    for (int64_t i = threadIdx.x; i < v.tiles; i += blockDim.x)
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const double u = v.part[q * v.tiles + i];
            acc[q] = q % 3 == 0 ? fmin(acc[q], u) : (q % 3 == 1 ? fmax(acc[q], u) : acc[q] + u);
        }
#pragma unroll
    for (int q = 0; q < 9; ++q)
        for (int o = 16; o; o >>= 1) {
            const double u = __shfl_xor_sync(0xffffffffu, acc[q], o);
            acc[q] = q % 3 == 0 ? fmin(acc[q], u) : (q % 3 == 1 ? fmax(acc[q], u) : acc[q] + u);
        }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int q = 0; q < 9; ++q) red[warp][q] = acc[q];
    __syncthreads();
    if (threadIdx.x < 9) {
        const int q = threadIdx.x;
        double r = red[0][q];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            r = q % 3 == 0 ? fmin(r, red[w][q]) : (q % 3 == 1 ? fmax(r, red[w][q]) : r + red[w][q]);
        stats[9 * vi + q] = r;
    }
}

constexpr int CCH = 1024;   // voxels per chunk of the combination: 256 threads x 4

struct CVol {
    const float *Sm;   // [3][N]
    float *S;
    int64_t N;
    int64_t chunk0;    // first chunk of this volume
};
struct CBatch {
    int n;
    double a, b, c, eps;
    int64_t chunks;
    CVol v[kMaxBatch];
};

// Eq. 6 on the min-max normalised maps of every volume of the batch, in one launch: each
// block first forms every volume's offsets and factors (FP64, once per block, into shared
// memory), then walks the chunks of 1024 consecutive voxels of all volumes (a chunk's volume
// by binary search), each thread loading its four voxels' three maps before any store.
__global__ void __launch_bounds__(256) combine_batch_kernel(const __grid_constant__ CBatch cb,
                                                            const double *__restrict__ stats)
{
    __shared__ float coef[kMaxBatch][6];   // lo[0..2], al[0..2] of each volume
    const double wts[3] = {cb.a, cb.b, cb.c};
    for (int e = threadIdx.x; e < 3 * cb.n; e += blockDim.x) {
        const int vi = e / 3, m = e - 3 * vi;
        const double l = stats[9 * vi + 3 * m], h = stats[9 * vi + 3 * m + 1];
        const double mag = fmax(fabs(l), fabs(h));
        const double scale = (h - l) <= cb.eps * mag ? 0.0 : 1.0 / (h - l);
        coef[vi][m] = (float)l;
        coef[vi][3 + m] = (float)(wts[m] * scale);
    }
    __syncthreads();
    for (int64_t c = blockIdx.x; c < cb.chunks; c += gridDim.x) {
        int lo = 0, hi = cb.n - 1;   // last volume whose first chunk is <= c
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (cb.v[mid].chunk0 <= c) lo = mid; else hi = mid - 1;
        }
        const CVol &v = cb.v[lo];
        const float *cf = coef[lo];
        const int64_t base = (c - v.chunk0) * CCH + threadIdx.x;
        const float *s0 = v.Sm, *s1 = v.Sm + v.N, *s2 = v.Sm + 2 * v.N;
        float x0[CCH / 256], x1[CCH / 256], x2[CCH / 256];
#pragma unroll
        for (int k = 0; k < CCH / 256; ++k) {
            const int64_t i = base + k * 256;
            x0[k] = i < v.N ? __ldg(s0 + i) : 0.f;
            x1[k] = i < v.N ? __ldg(s1 + i) : 0.f;
            x2[k] = i < v.N ? __ldg(s2 + i) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < CCH / 256; ++k) {
            const int64_t i = base + k * 256;
            if (i < v.N) v.S[i] = fmaf(cf[5], x2[k] - cf[2], fmaf(cf[4], x1[k] - cf[1], cf[3] * (x0[k] - cf[0])));
        }
    }
}

}  // namespace

cudaError_t launch_batch_stats_combine(const BatchVolDesc *vols, int n, const sal_params *p, double *stats,
                                       cudaStream_t s)
{
    if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
    RBatch rb;
    CBatch cb;
    rb.n = cb.n = n;
    cb.a = p->a;
    cb.b = p->b;
    cb.c = p->c;
    cb.eps = p->eps;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        rb.v[i].part = vols[i].part;
        rb.v[i].tiles = vols[i].tiles;
        cb.v[i].Sm = vols[i].Sm;
        cb.v[i].S = vols[i].S;
        cb.v[i].N = vols[i].N;
        cb.v[i].chunk0 = total;
        total += (vols[i].N + CCH - 1) / CCH;
    }
    cb.chunks = total;
    reduce_volumes_kernel<<<n, 256, 0, s>>>(rb, stats);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = total;                         // chunks
    const int64_t cap = (int64_t)nsm * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    combine_batch_kernel<<<(unsigned)blocks, 256, 0, s>>>(cb, stats);
    return cudaGetLastError();
}

}  // namespace sal
