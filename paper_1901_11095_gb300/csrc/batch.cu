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

struct CVol {
    const float *Sm;   // [3][N]
    float *S;
    int64_t N;
};
struct CBatch {
    int n;
    double a, b, c, eps;
    CVol v[kMaxBatch];
};

// Eq. 6 on the min-max normalised maps of every volume of the batch; one grid-stride pass
// per volume, all in one launch.
__global__ void __launch_bounds__(256) combine_batch_kernel(const __grid_constant__ CBatch cb,
                                                            const double *__restrict__ stats)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const double wts[3] = {cb.a, cb.b, cb.c};
    for (int vi = 0; vi < cb.n; ++vi) {
        const CVol &v = cb.v[vi];
        float lo[3], al[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const double l = stats[9 * vi + 3 * m], h = stats[9 * vi + 3 * m + 1];
            const double mag = fmax(fabs(l), fabs(h));
            const double scale = (h - l) <= cb.eps * mag ? 0.0 : 1.0 / (h - l);
            lo[m] = (float)l;
            al[m] = (float)(wts[m] * scale);
        }
        const float *s0 = v.Sm, *s1 = v.Sm + v.N, *s2 = v.Sm + 2 * v.N;
        for (int64_t i = i0; i < v.N; i += stride)
            v.S[i] = fmaf(al[2], s2[i] - lo[2], fmaf(al[1], s1[i] - lo[1], al[0] * (s0[i] - lo[0])));
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
        total += vols[i].N;
    }
    reduce_volumes_kernel<<<n, 256, 0, s>>>(rb, stats);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (total / n + 255) / 256;
    const int64_t cap = (int64_t)nsm * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    combine_batch_kernel<<<(unsigned)blocks, 256, 0, s>>>(cb, stats);
    return cudaGetLastError();
}

}  // namespace sal
