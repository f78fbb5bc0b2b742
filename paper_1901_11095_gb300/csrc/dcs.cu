// Directional centre-surround comparison (Eq. 5), the FP64 global statistics of the
// S_m maps, and the normalised weighted combination of Eq. 6.
//
//   S_m[v] = Q^-1 sum_{o in N_m} | E_m[v] - g(o) E_m[v + o] |,  g(o) = exp(-|o|^2 / (2 sigma^2))
//
// N_m is the 26-neighbourhood or the d x 1 line of side d = L along axis m (Sec. 2 text
// after Eq. 5).  E outside the volume comes from the boundary extension.  Each CTA stages
// its halo tile of E_m in shared memory (each value read from HBM about once), every
// thread produces four consecutive outputs along y, and the CTA reduces its min, max and
// sum (warp shuffles, then FP64 across warps) into one partial record; two small passes
// finish the FP64 reduction.
#include <float.h>

#include "sal_internal.cuh"

namespace sal {

namespace {

constexpr int DT = 4, DX = 8, DY = 32, DR = 4;          // output tile and outputs per thread
constexpr int DNT = DT * DX * (DY / DR);                // 256 threads
constexpr int DSMEM = (DT + 2 * kMaxH) * DX * DY;       // largest halo tile (LINE along t, h = 7)
constexpr int kRedBlocks = 160;                         // first pass of the partial reduction

struct DcsConsts {
    float g[3];            // 26-neighbourhood weights for |o|^2 = 1, 2, 3
    float gl[kMaxH + 1];   // line weights for offset k = 1..h
    float invQ;
    int stencil, h;
};

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(DNT) dcs_kernel(const float *__restrict__ E, int64_t T, int64_t X, int64_t Y,
                                                  int bnd, int tiles_x, int tiles_y, float *__restrict__ Sm,
                                                  double *__restrict__ partials, int64_t nparts,
                                                  const __grid_constant__ DcsConsts k)
{
    __shared__ __align__(16) float sE[DSMEM];
    __shared__ double red[DNT / 32][9];
    const int64_t tile = blockIdx.x;
    const int ty = (int)(tile % tiles_y);
    const int tx = (int)((tile / tiles_y) % tiles_x);
    const int64_t tt = tile / ((int64_t)tiles_y * tiles_x);
    const int64_t t0 = tt * DT, x0 = (int64_t)tx * DX, y0 = (int64_t)ty * DY;
    const int64_t N = T * X * Y;

    const int j = threadIdx.x % (DY / DR), row = threadIdx.x / (DY / DR);
    const int t = row / DX, x = row - t * DX;
    const int64_t gt = t0 + t, gx = x0 + x, gy = y0 + DR * j;
    const bool row_ok = gt < T && gx < X;

    float st_min[3], st_max[3], st_sum[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const int rt = k.stencil == SAL_STENCIL_26 ? 1 : (m == 0 ? k.h : 0);
        const int rx = k.stencil == SAL_STENCIL_26 ? 1 : (m == 1 ? k.h : 0);
        const int ry = k.stencil == SAL_STENCIL_26 ? 1 : (m == 2 ? k.h : 0);
        const int PX = DX + 2 * rx, PYr = DY + 2 * ry, n = (DT + 2 * rt) * PX * PYr;
        const float *Em = E + m * N;
        for (int i = threadIdx.x; i < n; i += DNT) {
            const int r = i / PYr, yy = i - r * PYr;
            const int a = r / PX, xx = r - a * PX;
            const int64_t et = ext_index(t0 - rt + a, T, bnd);
            const int64_t ex = ext_index(x0 - rx + xx, X, bnd);
            const int64_t ey = ext_index(y0 - ry + yy, Y, bnd);
            sE[i] = __ldg(Em + (et * X + ex) * Y + ey);
        }
        __syncthreads();

        float out[DR];
        if (k.stencil == SAL_STENCIL_26) {
            // window rows (t + a, x + b), columns y0-1 .. y0+4 of this thread
            const float *base = sE + ((t + 1) * PX + (x + 1)) * PYr + (DR * j + 1);
            float c[DR];
#pragma unroll
            for (int r = 0; r < DR; ++r) { c[r] = base[r]; out[r] = 0.f; }
#pragma unroll
            for (int a = -1; a <= 1; ++a)
#pragma unroll
                for (int b = -1; b <= 1; ++b) {
                    const float2 *p = reinterpret_cast<const float2 *>(base + (a * PX + b) * PYr - 1);
                    float w[DR + 2];
#pragma unroll
                    for (int q = 0; q < (DR + 2) / 2; ++q) {
                        const float2 v = p[q];
                        w[2 * q] = v.x;
                        w[2 * q + 1] = v.y;
                    }
#pragma unroll
                    for (int r = 0; r < DR; ++r)
#pragma unroll
                        for (int cc = -1; cc <= 1; ++cc) {
                            const int d2 = a * a + b * b + cc * cc;
                            if (d2 == 0) continue;
                            out[r] += fabsf(fmaf(-k.g[d2 - 1], w[r + 1 + cc], c[r]));
                        }
                }
        } else {
            const int stride = m == 0 ? PX * PYr : (m == 1 ? PYr : 1);
            const float *base = sE + ((t + rt) * PX + (x + rx)) * PYr + (DR * j + ry);
#pragma unroll
            for (int r = 0; r < DR; ++r) {
                const float c = base[r];
                float s = 0.f;
                for (int q = 1; q <= k.h; ++q) {
                    s += fabsf(fmaf(-k.gl[q], base[r + q * stride], c));
                    s += fabsf(fmaf(-k.gl[q], base[r - q * stride], c));
                }
                out[r] = s;
            }
        }

        float mn = FLT_MAX, mx = -FLT_MAX, sm = 0.f;
        if (row_ok) {
            float *o = Sm + m * N + (gt * X + gx) * Y + gy;
#pragma unroll
            for (int r = 0; r < DR; ++r) {
                out[r] *= k.invQ;
                if (gy + r < Y) {
                    mn = fminf(mn, out[r]);
                    mx = fmaxf(mx, out[r]);
                    sm += out[r];
                }
            }
            if (gy + DR <= Y && (Y & 3) == 0) {
                *reinterpret_cast<float4 *>(o) = make_float4(out[0], out[1], out[2], out[3]);
            } else {
#pragma unroll
                for (int r = 0; r < DR; ++r)
                    if (gy + r < Y) o[r] = out[r];
            }
        }
        st_min[m] = warp_min(mn);
        st_max[m] = warp_max(mx);
        st_sum[m] = warp_sum(sm);
        __syncthreads();   // sE is reloaded for the next map
    }

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int m = 0; m < 3; ++m) {
            red[warp][3 * m] = st_min[m];
            red[warp][3 * m + 1] = st_max[m];
            red[warp][3 * m + 2] = st_sum[m];
        }
    __syncthreads();
    if (threadIdx.x < 9) {
        const int q = threadIdx.x, kind = q % 3;
        double v = red[0][q];
        for (int w = 1; w < DNT / 32; ++w) {
            const double u = red[w][q];
            v = kind == 0 ? fmin(v, u) : (kind == 1 ? fmax(v, u) : v + u);
        }
        partials[q * nparts + blockIdx.x] = v;
    }
}

// Reduces `n` partial records [9][n] into gridDim.x records [9][gridDim.x] (FP64, fixed order).
__global__ void __launch_bounds__(256) reduce_partials_kernel(const double *__restrict__ in, int64_t n,
                                                              double *__restrict__ out, int64_t nout)
{
    __shared__ double red[8][9];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = blockIdx.x * chunk, b1 = b0 + chunk < n ? b0 + chunk : n;
    double v[9];
    for (int q = 0; q < 9; ++q) v[q] = q % 3 == 0 ? DBL_MAX : (q % 3 == 1 ? -DBL_MAX : 0.0);
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x)
        for (int q = 0; q < 9; ++q) {
            const double u = in[q * n + i];
            v[q] = q % 3 == 0 ? fmin(v[q], u) : (q % 3 == 1 ? fmax(v[q], u) : v[q] + u);
        }
    for (int q = 0; q < 9; ++q)
        for (int o = 16; o; o >>= 1) {
            const double u = __shfl_xor_sync(0xffffffffu, v[q], o);
            v[q] = q % 3 == 0 ? fmin(v[q], u) : (q % 3 == 1 ? fmax(v[q], u) : v[q] + u);
        }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int q = 0; q < 9; ++q) red[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x < 9) {
        const int q = threadIdx.x;
        double r = red[0][q];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            r = q % 3 == 0 ? fmin(r, red[w][q]) : (q % 3 == 1 ? fmax(r, red[w][q]) : r + red[w][q]);
        out[q * nout + blockIdx.x] = r;
    }
}

// Eq. 6 on min-max normalised maps: S = sum_m w_m (S_m - lo_m) / (hi_m - lo_m).
__global__ void __launch_bounds__(256) combine_kernel(const float *__restrict__ Sm, const double *__restrict__ stats,
                                                      int64_t N, double a, double b, double c, double eps,
                                                      float *__restrict__ S)
{
    const double wts[3] = {a, b, c};
    float lo[3], al[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const double l = stats[3 * m], h = stats[3 * m + 1];
        const double mag = fmax(fabs(l), fabs(h));
        const double scale = (h - l) <= eps * mag ? 0.0 : 1.0 / (h - l);
        lo[m] = (float)l;
        al[m] = (float)(wts[m] * scale);
    }
    const int64_t n4 = ((N & 3) == 0) ? N / 4 : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 s0 = __ldg(reinterpret_cast<const float4 *>(Sm) + i);
        const float4 s1 = __ldg(reinterpret_cast<const float4 *>(Sm + N) + i);
        const float4 s2 = __ldg(reinterpret_cast<const float4 *>(Sm + 2 * N) + i);
        float4 o;
        o.x = fmaf(al[2], s2.x - lo[2], fmaf(al[1], s1.x - lo[1], al[0] * (s0.x - lo[0])));
        o.y = fmaf(al[2], s2.y - lo[2], fmaf(al[1], s1.y - lo[1], al[0] * (s0.y - lo[0])));
        o.z = fmaf(al[2], s2.z - lo[2], fmaf(al[1], s1.z - lo[1], al[0] * (s0.z - lo[0])));
        o.w = fmaf(al[2], s2.w - lo[2], fmaf(al[1], s1.w - lo[1], al[0] * (s0.w - lo[0])));
        reinterpret_cast<float4 *>(S)[i] = o;
    }
    for (int64_t i = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride)
        S[i] = fmaf(al[2], Sm[2 * N + i] - lo[2], fmaf(al[1], Sm[N + i] - lo[1], al[0] * (Sm[i] - lo[0])));
}

void dcs_tiles(sal_dims d, int64_t *nt, int64_t *nx, int64_t *ny)
{
    *nt = (d.T + DT - 1) / DT;
    *nx = (d.X + DX - 1) / DX;
    *ny = (d.Y + DY - 1) / DY;
}

}  // namespace

int64_t dcs_num_partials(sal_dims d)
{
    int64_t nt, nx, ny;
    dcs_tiles(d, &nt, &nx, &ny);
    return nt * nx * ny + kRedBlocks;   // per-tile records, then the first reduction pass
}

cudaError_t launch_dcs(const float *E, sal_dims d, const sal_params *p, float *Sm, double *partials, double *stats,
                       cudaStream_t s)
{
    int64_t nt, nx, ny;
    dcs_tiles(d, &nt, &nx, &ny);
    const int64_t tiles = nt * nx * ny;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    DcsConsts k;
    const double s2 = 2.0 * (double)p->sigma * (double)p->sigma;
    for (int i = 0; i < 3; ++i) k.g[i] = (float)exp(-(double)(i + 1) / s2);
    const int h = (p->L - 1) / 2;
    for (int i = 0; i <= kMaxH; ++i) k.gl[i] = (float)exp(-(double)(i * i) / s2);
    k.stencil = p->stencil;
    k.h = h;
    k.invQ = (float)(1.0 / (p->stencil == SAL_STENCIL_26 ? 26.0 : (double)(2 * h)));
    dcs_kernel<<<(unsigned)tiles, DNT, 0, s>>>(E, d.T, d.X, d.Y, p->boundary, (int)nx, (int)ny, Sm, partials, tiles, k);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double *second = partials + 9 * tiles;
    reduce_partials_kernel<<<kRedBlocks, 256, 0, s>>>(partials, tiles, second, kRedBlocks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_partials_kernel<<<1, 256, 0, s>>>(second, kRedBlocks, stats, 1);
    return cudaGetLastError();
}

cudaError_t launch_combine(const float *Sm, const double *stats, sal_dims d, const sal_params *p, float *S,
                           cudaStream_t s)
{
    const int64_t N = d.T * d.X * d.Y;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (N / 4 + 255) / 256;
    const int64_t cap = (int64_t)nsm * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    combine_kernel<<<(unsigned)blocks, 256, 0, s>>>(Sm, stats, N, p->a, p->b, p->c, p->eps, S);
    return cudaGetLastError();
}

}  // namespace sal
