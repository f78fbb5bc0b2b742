// Learned surrogate of the spectral energies: 5 layers of 3x3x3 convolution (1 -> 24 -> 24 ->
// 24 -> 24 -> 3 channels), GELU after the first four, predicting E_t, E_x, E_y (divided by
// the volume's RMS amplitude, which makes the prediction as scale-covariant as E itself)
// from the amplitudes (divided by the same RMS).  Weights are BF16, accumulation FP32.
// Kernels: forward (FP32 or BF16 activations), input gradient (fused with the GELU
// derivative), weight gradient, masked MSE gradient, Adam, and the RMS reduction.
//
// Layout: activations planar [C][T][X][Y]; parameters flat, layer by layer, weights
// [Cout][Cin][3][3][3] then biases [Cout] (the same layout as the CPU reference).
//
// The backward pass implements the adjoint of the convolution for voxels whose receptive
// field stays inside the volume; the loss mask keeps a margin of at least one voxel per
// layer from every face, so the gradient never reaches the boundary extension and the
// result is exact.
#include <string.h>

#include <cuda_bf16.h>

#include "energy_tc.cuh"   // tcgen05 helpers: descriptors, bounded mbarrier wait, tensor-memory load
#include "sal_internal.cuh"

namespace sal {

namespace {

constexpr int ST = 2, SX = 8, SY = 32, SNT = 256;          // output tile, threads (2 outputs along y each)
constexpr int HT = ST + 2, HXX = SX + 2, HYY = SY + 2, HN = HT * HXX * HYY;
constexpr int CC = 8;                                        // input channels staged at once
constexpr int kLayers = SAL_SURR_LAYERS, kWidth = SAL_SURR_WIDTH;
constexpr int kWidths[kLayers + 1] = {1, kWidth, kWidth, kWidth, kWidth, 3};

// BF16 activations of the tensor-core layers, grouped: for every line (t, x) the channel groups
// of 8 one after another, each [y][8 channels] (16 bytes per voxel), so that a line's group is
// one contiguous run of 16-byte rows (the layout the products read, copied in bulk).
__host__ __device__ __forceinline__ int64_t gidx(int64_t line, int64_t Y, int64_t y, int o)
{
    return ((line * (kWidth / 8) + (o >> 3)) * Y + y) * 8 + (o & 7);
}

__device__ __forceinline__ float ldf(const float *p) { return *p; }
__device__ __forceinline__ float ldf(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void stf(float *p, float v) { *p = v; }
__device__ __forceinline__ void stf(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// GELU x * Phi(x) and its derivative, from CUDA's erff / expf
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

enum { FWD_HIDDEN = 0, FWD_OUTPUT = 1, BWD_DATA = 2 };

// One convolution layer over a tile of ST x SX x SY outputs.
//   FWD_HIDDEN: z = conv(in * in_scale) + b; optionally z stored (FP32), GELU(z) stored as TOUT
//   FWD_OUTPUT: (conv(in) + b) * out_scale stored as float
//   BWD_DATA:   in = dL/dz of the next layer, weights transposed and flipped (the adjoint),
//               samples outside the volume are zero; out = result * gelu'(zprev)
// Weights are the FP32 master parameters rounded to BF16 as they are staged.  ILV: BF16
// activations (input or output) in the grouped layout of the tensor-core layers (gidx)
// instead of planar [channel][voxel].
template <int CI, int CO, typename TIN, typename TOUT, int MODE, bool ILV = false>
__global__ void __launch_bounds__(SNT) conv_kernel(const TIN *__restrict__ in, int64_t T, int64_t X, int64_t Y,
                                                   int bnd, const float *__restrict__ in_scale_p,
                                                   const float *__restrict__ w, const float *__restrict__ b,
                                                   float *__restrict__ zout, TOUT *__restrict__ out,
                                                   const float *__restrict__ out_scale_p,
                                                   const float *__restrict__ zprev, int tiles_x, int tiles_y)
{
    extern __shared__ __align__(16) float sm[];
    float *ws = sm;                       // [CO][CI][27]
    float *xs = sm + CO * CI * 27;        // [CC][HN]
    const float in_scale = in_scale_p ? *in_scale_p : 1.f, out_scale = out_scale_p ? *out_scale_p : 1.f;
    // weights: forward as stored; adjoint: ws[o][i][tap] = w[i][o][26 - tap]
    for (int e = threadIdx.x; e < CO * CI * 27; e += SNT) {
        const int tap = e % 27, i = (e / 27) % CI, o = e / (27 * CI);
        const float v = MODE == BWD_DATA ? w[((int64_t)i * CO + o) * 27 + (26 - tap)] : w[e];
        ws[e] = __bfloat162float(__float2bfloat16_rn(v));
    }
    const int64_t tile = blockIdx.x;
    const int ty = (int)(tile % tiles_y), tx = (int)((tile / tiles_y) % tiles_x);
    const int64_t t0 = (tile / ((int64_t)tiles_y * tiles_x)) * ST, x0 = (int64_t)tx * SX, y0 = (int64_t)ty * SY;
    const int64_t N = T * X * Y;
    const int row = threadIdx.x >> 4, yp = threadIdx.x & 15;
    const int t = row / SX, x = row - t * SX;
    float acc[CO][2];
#pragma unroll
    for (int o = 0; o < CO; ++o) acc[o][0] = acc[o][1] = (MODE == BWD_DATA || !b) ? 0.f : b[o];

    for (int c0 = 0; c0 < CI; c0 += CC) {
        const int nc = CI - c0 < CC ? CI - c0 : CC;
        __syncthreads();
        for (int e = threadIdx.x; e < nc * HN; e += SNT) {
            const int c = e / HN, r = e - c * HN;
            const int a = r / (HXX * HYY), xx = (r / HYY) % HXX, yy = r % HYY;
            const int64_t gt0 = t0 - 1 + a, gx0 = x0 - 1 + xx, gy0 = y0 - 1 + yy;
            float v;
            if (MODE == BWD_DATA) {
                v = (gt0 >= 0 && gt0 < T && gx0 >= 0 && gx0 < X && gy0 >= 0 && gy0 < Y)
                        ? ldf(in + (c0 + c) * N + (gt0 * X + gx0) * Y + gy0) : 0.f;
            } else {
                const int64_t gt = ext_index(gt0, T, bnd), gx = ext_index(gx0, X, bnd), gy = ext_index(gy0, Y, bnd);
                const int64_t vox = (gt * X + gx) * Y + gy;
                const bool ilv_in = ILV && sizeof(TIN) == 2;
                v = ldf(in + (ilv_in ? gidx(gt * X + gx, Y, gy, c0 + c) : (c0 + c) * N + vox)) * in_scale;
            }
            xs[e] = v;
        }
        __syncthreads();
        for (int c = 0; c < nc; ++c) {
            float win[3][3][4];
            const float *base = xs + c * HN + (t * HXX + x) * HYY + 2 * yp;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int q = 0; q < 3; ++q)
#pragma unroll
                    for (int d = 0; d < 4; ++d) win[a][q][d] = base[(a * HXX + q) * HYY + d];
            const float *wc = ws + (c0 + c) * 27;
#pragma unroll
            for (int o = 0; o < CO; ++o) {
                const float *wo = wc + o * CI * 27;
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int q = 0; q < 3; ++q)
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const float wv = wo[(a * 3 + q) * 3 + d];
                            acc[o][0] = fmaf(wv, win[a][q][d], acc[o][0]);
                            acc[o][1] = fmaf(wv, win[a][q][d + 1], acc[o][1]);
                        }
            }
        }
    }
    const int64_t gt = t0 + t, gx = x0 + x;
    if (gt >= T || gx >= X) return;
    if constexpr (MODE == FWD_HIDDEN && ILV && sizeof(TOUT) == 2 && CO % 8 == 0) {
        // interleaved BF16 activations: the thread's two voxels are adjacent along y, so their
        // 2 x CO channels are one contiguous run written as 16-byte vectors (the warp's 32
        // voxels form one contiguous span)
        if (!zout) {
            const int64_t gy = y0 + 2 * yp;
            if (gy >= Y) return;
            const int nr = gy + 1 < Y ? 2 : 1;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                if (r >= nr) break;
#pragma unroll
                for (int g = 0; g < CO / 8; ++g) {
                    uint32_t p[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const __nv_bfloat162 h = __floats2bfloat162_rn(gelu(acc[8 * g + 2 * j][r]), gelu(acc[8 * g + 2 * j + 1][r]));
                        memcpy(&p[j], &h, 4);
                    }
                    *reinterpret_cast<uint4 *>(out + gidx(gt * X + gx, Y, gy + r, 8 * g)) = make_uint4(p[0], p[1], p[2], p[3]);
                }
            }
            return;
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int64_t gy = y0 + 2 * yp + r;
        if (gy >= Y) break;
        const int64_t v = (gt * X + gx) * Y + gy;
#pragma unroll
        for (int o = 0; o < CO; ++o) {
            const float z = acc[o][r];
            if (MODE == FWD_HIDDEN) {
                if (zout) zout[o * N + v] = z;
                const bool ilv_out = ILV && sizeof(TOUT) == 2;
                stf(out + (ilv_out ? gidx(gt * X + gx, Y, gy, o) : o * N + v), gelu(z));
            } else if (MODE == FWD_OUTPUT) {
                stf(out + o * N + v, z * out_scale);
            } else {
                stf(out + o * N + v, z * gelu_grad(zprev[o * N + v]));
            }
        }
    }
}

// Weight and bias gradients of one layer: dW[o][i][tap] += sum_v g[o][v] a[i][ext(v + off)].
// blockIdx.y selects a chunk of CC input channels; the grid walks the tiles persistently and
// every thread keeps its (o, i, tap) sums in registers until one atomic add at the end.
template <int CI, int CO>
__global__ void __launch_bounds__(SNT) wgrad_kernel(const float *__restrict__ a, const float *__restrict__ a_scale_p,
                                                    const float *__restrict__ g, int64_t T, int64_t X, int64_t Y,
                                                    int bnd, int tiles_x, int tiles_y, int64_t ntiles,
                                                    float *__restrict__ dw, float *__restrict__ db)
{
    const float a_scale = a_scale_p ? *a_scale_p : 1.f;
    constexpr int NE = CO * CC * 27, PER = (NE + SNT - 1) / SNT;
    extern __shared__ __align__(16) float sm[];
    float *gs = sm;                       // [CO][ST*SX*SY]
    float *as = sm + CO * ST * SX * SY;   // [CC][HN]
    const int c0 = blockIdx.y * CC;
    const int nc = CI - c0 < CC ? CI - c0 : CC;
    const int64_t N = T * X * Y;
    float accw[PER], accb = 0.f;
#pragma unroll
    for (int k = 0; k < PER; ++k) accw[k] = 0.f;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int ty = (int)(tile % tiles_y), tx = (int)((tile / tiles_y) % tiles_x);
        const int64_t t0 = (tile / ((int64_t)tiles_y * tiles_x)) * ST, x0 = (int64_t)tx * SX, y0 = (int64_t)ty * SY;
        __syncthreads();
        for (int e = threadIdx.x; e < CO * ST * SX * SY; e += SNT) {
            const int o = e / (ST * SX * SY), r = e - o * (ST * SX * SY);
            const int tt = r / (SX * SY), xx = (r / SY) % SX, yy = r % SY;
            const int64_t gt = t0 + tt, gx = x0 + xx, gy = y0 + yy;
            gs[e] = (gt < T && gx < X && gy < Y) ? g[o * N + (gt * X + gx) * Y + gy] : 0.f;
        }
        for (int e = threadIdx.x; e < nc * HN; e += SNT) {
            const int c = e / HN, r = e - c * HN;
            const int aa = r / (HXX * HYY), xx = (r / HYY) % HXX, yy = r % HYY;
            const int64_t gt = ext_index(t0 - 1 + aa, T, bnd), gx = ext_index(x0 - 1 + xx, X, bnd),
                          gy = ext_index(y0 - 1 + yy, Y, bnd);
            as[e] = a[(c0 + c) * N + (gt * X + gx) * Y + gy] * a_scale;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = threadIdx.x + k * SNT;
            if (e >= NE) break;
            const int tap = e % 27, c = (e / 27) % CC, o = e / (27 * CC);
            if (c >= nc) continue;
            const int da = tap / 9, dq = (tap / 3) % 3, dd = tap % 3;
            const float *gp = gs + o * (ST * SX * SY);
            const float *ap = as + c * HN + (da * HXX + dq) * HYY + dd;
            float s = 0.f;
            for (int tt = 0; tt < ST; ++tt)
                for (int xx = 0; xx < SX; ++xx) {
                    const float *gr = gp + (tt * SX + xx) * SY;
                    const float *ar = ap + (tt * HXX + xx) * HYY;
#pragma unroll 8
                    for (int yy = 0; yy < SY; ++yy) s = fmaf(gr[yy], ar[yy], s);
                }
            accw[k] += s;
        }
        if (blockIdx.y == 0 && threadIdx.x < CO) {
            const float *gp = gs + threadIdx.x * (ST * SX * SY);
            float s = 0.f;
            for (int i = 0; i < ST * SX * SY; ++i) s += gp[i];
            accb += s;
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * SNT;
        if (e >= NE) break;
        const int tap = e % 27, c = (e / 27) % CC, o = e / (27 * CC);
        if (c >= nc) continue;
        atomicAdd(&dw[((int64_t)o * CI + c0 + c) * 27 + tap], accw[k]);
    }
    if (blockIdx.y == 0 && threadIdx.x < CO) atomicAdd(&db[threadIdx.x], accb);
}

// dL/dout for L = 0.5 / count * sum over voxels at least `margin` from every face and the
// 3 channels of (out - target)^2; the loss itself is added to *loss (FP64).
__global__ void __launch_bounds__(256) loss_grad_kernel(const float *__restrict__ out, const float *__restrict__ target,
                                                        const float *__restrict__ tscale_p, int64_t T, int64_t X,
                                                        int64_t Y, int margin, float inv_count,
                                                        float *__restrict__ g, double *loss)
{
    const int64_t N = T * X * Y;
    const float tscale = *tscale_p;
    double part = 0.0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t y = v % Y, x = (v / Y) % X, t = v / (X * Y);
        const bool in = t >= margin && t < T - margin && x >= margin && x < X - margin && y >= margin && y < Y - margin;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float d = in ? out[c * N + v] - target[c * N + v] * tscale : 0.f;
            g[c * N + v] = d * inv_count;
            part += 0.5 * (double)d * d * inv_count;
        }
    }
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
}

__global__ void __launch_bounds__(256) scale_kernel(const float *__restrict__ in, int64_t n, const float *__restrict__ sp,
                                                    float *__restrict__ out)
{
    const float sc = *sp;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = in[i] * sc;
}

__global__ void __launch_bounds__(256) sumsq_kernel(const float *__restrict__ V, int64_t N, double *out)
{
    double part = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = V[i];
        part += v * v;
    }
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, part);
}

// RMS scale on the device: scale[0] = 1 / rms (input), scale[1] = rms (output)
__global__ void rms_kernel(const double *sumsq, int64_t N, float *scale)
{
    const double r = sqrt(*sumsq / (double)N);
    scale[0] = r > 0.0 ? (float)(1.0 / r) : 1.f;
    scale[1] = r > 0.0 ? (float)r : 1.f;
}

// Adam on the FP32 master parameters (the kernels round the weights to BF16 as they read them).
__global__ void __launch_bounds__(256) adam_kernel(float *__restrict__ w, const float *__restrict__ g,
                                                   float *__restrict__ m, float *__restrict__ v, int64_t n, float lr,
                                                   float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        w[i] = wi;
    }
}

// ---- per-block check of the prediction and exact recomputation where it fails ----------
constexpr int FB_T = 16, FB_X = 16, FB_Y = 32, FB_S = 8;   // check block (voxels) and samples per block

__device__ __forceinline__ uint32_t mix32(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return (uint32_t)k;
}

// FB_S sample voxels per check block at fixed pseudo-random positions inside it.
__global__ void sample_coords_kernel(int64_t T, int64_t X, int64_t Y, int64_t nbx, int64_t nby, int64_t nb,
                                     int64_t *__restrict__ coords)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nb * FB_S; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = k / FB_S;
        const int64_t by = b % nby, bx = (b / nby) % nbx, bt = b / (nby * nbx);
        const int64_t t0 = bt * FB_T, x0 = bx * FB_X, y0 = by * FB_Y;
        const int64_t et = T - t0 < FB_T ? T - t0 : FB_T, ex = X - x0 < FB_X ? X - x0 : FB_X, ey = Y - y0 < FB_Y ? Y - y0 : FB_Y;
        coords[3 * k] = t0 + mix32(3 * k + 1) % et;
        coords[3 * k + 1] = x0 + mix32(3 * k + 2) % ex;
        coords[3 * k + 2] = y0 + mix32(3 * k + 3) % ey;
    }
}

__global__ void sample_sums_kernel(const float *__restrict__ Eex, int64_t n, float *__restrict__ sums)
{
    float a[3] = {0.f, 0.f, 0.f};
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        for (int m = 0; m < 3; ++m) a[m] += fabsf(Eex[m * n + k]);
    for (int m = 0; m < 3; ++m) {
        for (int o = 16; o; o >>= 1) a[m] += __shfl_xor_sync(0xffffffffu, a[m], o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&sums[m], a[m]);
    }
}

// One thread per check block: the largest error of its samples, relative to each map's mean
// magnitude over all samples; a block above `thr` queues its energy tiles for recomputation.
__global__ void block_check_kernel(const float *__restrict__ Epred, int64_t T, int64_t X, int64_t Y,
                                   const int64_t *__restrict__ coords, const float *__restrict__ Eex, int64_t nb,
                                   const float *__restrict__ sums, float thr, int bt_, int bx_, int64_t tiles_t,
                                   int64_t tiles_x, int64_t tiles_y, int64_t nbx, int64_t nby,
                                   int64_t *__restrict__ list, int *__restrict__ count, int *__restrict__ nbad)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b == 0) nbad[1] = (int)nb;   // blocks checked, next to the count of blocks recomputed
    if (b >= nb) return;
    const int64_t N = T * X * Y, ns = nb * FB_S;
    float scale[3];
    for (int m = 0; m < 3; ++m) scale[m] = fmaxf(sums[m] / (float)ns, 1e-30f);
    float err = 0.f;
    for (int j = 0; j < FB_S; ++j) {
        const int64_t k = b * FB_S + j;
        const int64_t v = (coords[3 * k] * X + coords[3 * k + 1]) * Y + coords[3 * k + 2];
        for (int m = 0; m < 3; ++m) err = fmaxf(err, fabsf(Epred[m * N + v] - Eex[m * ns + k]) / scale[m]);
    }
    if (!(err <= thr)) {   // NaN counts as a failure
        atomicAdd(nbad, 1);
        const int64_t by = b % nby, bx = (b / nby) % nbx, bt = b / (nby * nbx);
        const int64_t t_lo = bt * (FB_T / bt_), t_hi = t_lo + FB_T / bt_ < tiles_t ? t_lo + FB_T / bt_ : tiles_t;
        const int64_t x_lo = bx * (FB_X / bx_), x_hi = x_lo + FB_X / bx_ < tiles_x ? x_lo + FB_X / bx_ : tiles_x;
        const int n = (int)((t_hi - t_lo) * (x_hi - x_lo));
        int64_t at = atomicAdd(count, n);
        for (int64_t tt = t_lo; tt < t_hi; ++tt)
            for (int64_t tx = x_lo; tx < x_hi; ++tx) list[at++] = (tt * tiles_x + tx) * tiles_y + by;
    }
}

int64_t param_offset(int l)
{
    int64_t o = 0;
    for (int k = 0; k < l; ++k) o += (int64_t)kWidths[k + 1] * kWidths[k] * 27 + kWidths[k + 1];
    return o;
}

void conv_tiles(sal_dims d, int *tx, int *ty, int64_t *n)
{
    const int64_t nt = (d.T + ST - 1) / ST, nx = (d.X + SX - 1) / SX, ny = (d.Y + SY - 1) / SY;
    *tx = (int)nx;
    *ty = (int)ny;
    *n = nt * nx * ny;
}

template <int CI, int CO, typename TIN, typename TOUT, int MODE, bool ILV = false>
cudaError_t launch_conv(const TIN *in, sal_dims d, int bnd, const float *in_scale, const float *w, const float *b,
                        float *zout, TOUT *out, const float *out_scale, const float *zprev, cudaStream_t s)
{
    int tx, ty;
    int64_t n;
    conv_tiles(d, &tx, &ty, &n);
    if (n > 0x7fffffffLL) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * ((size_t)CO * CI * 27 + (size_t)CC * HN);
    auto k = conv_kernel<CI, CO, TIN, TOUT, MODE, ILV>;
    cudaError_t e = set_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)n, SNT, smem, s>>>(in, d.T, d.X, d.Y, bnd, in_scale, w, b, zout, out, out_scale, zprev, tx, ty);
    return cudaGetLastError();
}

template <int CI, int CO>
cudaError_t launch_wgrad(const float *a, const float *a_scale, const float *g, sal_dims d, int bnd, float *dw, float *db,
                         cudaStream_t s)
{
    int tx, ty;
    int64_t n;
    conv_tiles(d, &tx, &ty, &n);
    const size_t smem = sizeof(float) * ((size_t)CO * ST * SX * SY + (size_t)CC * HN);
    auto k = wgrad_kernel<CI, CO>;
    cudaError_t e = set_smem(k, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t gx = (int64_t)nsm * 2;
    if (gx > n) gx = n;
    dim3 grid((unsigned)gx, (CI + CC - 1) / CC);
    k<<<grid, SNT, smem, s>>>(a, a_scale, g, d.T, d.X, d.Y, bnd, tx, ty, n, dw, db);
    return cudaGetLastError();
}

// ---- layers 2..5 on the tensor cores (inference) ------------------------------------------
// Implicit GEMM per tap: for an output line (t, x, y0 .. y0 + 127),
//     D[y][o] += sum_c A_tap[y][c] W[o][c][tap],  A_tap[y][c] = act[t + dt][x + dx][y + dy][c],
// 27 taps x 2 products of K = 16 (channels 0..15 and 16..31, 24..31 meeting zero weights),
// M = 128, BF16 operands, FP32 accumulation in tensor memory.  CO = 24: hidden layer (N = 32,
// bias, GELU, BF16 grouped out); CO = 3: output layer (N = 16, outputs 3..15 zero; bias and
// the RMS scale applied, FP32 E written planar [3][voxel]).  Activations in the grouped
// layout (gidx).
//
// The halo lines of a tile sit in shared memory as [line][channel group of 8][y][8 channels]:
// K-major core matrices of 8 rows x 16 bytes, 8-row groups 128 bytes apart, channel groups
// 2176 bytes apart.  The operand of every tap is a line's buffer at a byte offset added to
// the descriptor's start address, so no operand is rebuilt per tap.  Only the three real
// channel groups are kept: the second k-step's upper group reads the next t-line's first
// group (or a zero pad after the last one), which meets the zero weights of channels 24..31.
// Likewise the hidden layer's B tiles keep their 24 real rows (768 bytes each): the 4th 8-row
// group a product reads is the next tile's first and lands in outputs 24..31, never used.
// Each (line, group) is one contiguous run of the grouped activations, copied in bulk and
// counted in bytes on an mbarrier (a tensor-map load of boxes of 8 channels moves 16 bytes per
// row: it took about 7,000 cycles per 9-line halo).  The kernel is persistent (one CTA per SM)
// and warp-specialised, and tiles along x share their halo lines (see conv_tc2_kernel).
// Every wait is bounded; on expiry the status word gets SAL_ERR_TIMEOUT.
constexpr int TCY = 128, TCH = TCY + 2;                     // outputs per line tile, halo rows
constexpr int TC1_GRP = 17 * 128;                           // bytes of one channel group of a line

// A line tile: its output plane t, row x and first column y0 (32-bit: the launcher checks
// that T, X, Y and the tile count fit).
struct TileC {
    int t, x, y0;
};

// Boundary extension of one coordinate in 32 bits (one reflection or wrap; wider cases take
// the general routine).
__device__ __forceinline__ int ext32(int i, int n, int bnd)
{
    if (i >= 0 && i < n) return i;
    if (bnd == SAL_BND_PERIODIC) {
        if (i < 0 && i >= -n) return i + n;
        if (i >= n && i < 2 * n) return i - n;
    } else {
        if (n == 1) return 0;
        if (i < 0 && i > -n) return -i;
        if (i >= n && i <= 2 * n - 2) return 2 * (n - 1) - i;
    }
    return (int)ext_index(i, n, bnd);
}

__device__ __forceinline__ void tc_mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem), "l"(a), "l"(b),
                 "r"(idesc), "r"(acc));
}

// Bias, GELU, BF16 and store of the hidden layer's accumulator `acc` for the 32 voxels of lane
// quadrant q (rows = y) and channel half h (channels 0..15 or 16..23).
__device__ __forceinline__ void tc_epilogue_hidden(uint32_t acc, int q, int h, TileC c, int X, int Y, const float *sb,
                                                   __nv_bfloat16 *__restrict__ out)
{
    float v[16];
    energy_detail::tmem_ld16(acc + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * h), v);
    const int y = c.y0 + 32 * q + (threadIdx.x & 31);
    if (y >= Y) return;
    const int64_t line = (int64_t)c.t * X + c.x;
    uint32_t pk[8];
    const int npairs = h == 0 ? 8 : (kWidth - 16) / 2;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j >= npairs) break;
        const float a = gelu(v[2 * j] + sb[16 * h + 2 * j]);
        const float bb = gelu(v[2 * j + 1] + sb[16 * h + 2 * j + 1]);
        const __nv_bfloat162 p2 = __floats2bfloat162_rn(a, bb);
        pk[j] = *reinterpret_cast<const uint32_t *>(&p2);
    }
    *reinterpret_cast<uint4 *>(out + gidx(line, Y, y, 16 * h)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    if (h == 0) *reinterpret_cast<uint4 *>(out + gidx(line, Y, y, 8)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
}

// Warp roles of the pipelined layer: warp 0 stages halo lines, warp 1 issues the products,
// warps 2..9 run the epilogue (warp w reads tensor-memory lane quadrant w % 4, channel half
// (w - 2) / 4).  A CTA walks runs of up to XC consecutive tiles along x at one (t, y0), so
// that each tile brings in only the three lines (t - 1..t + 1) at x + 1 and reuses the other
// six from its neighbours: a "line step" stages the lines of one x (3 t-lines x 3 channel
// groups = 9 bulk copies) into one of RS slots, tile j of a run reads the slots of line steps
// j, j + 1, j + 2, and each slot is refilled once the last tile reading it has finished its
// products.  Two accumulators: while the products of one tile run, the epilogue of the
// previous one drains the other.
constexpr int TC2_EPI = 8;                                    // epilogue warps
constexpr int TC2_NT = 32 * (2 + TC2_EPI);
constexpr int TC2_RS = 6;                                     // line-step slots
constexpr int TC2_TLINE = 3 * TC1_GRP;                        // one t-line: 3 channel groups
constexpr int TC2_SLOT = 3 * TC2_TLINE;                       // one line step: 3 t-lines
constexpr int TC2_PAD = (TCH * 16 + 127) / 128 * 128;         // read by the last t-line's upper group

template <int CO>
constexpr size_t tc2_wbytes() { return (size_t)27 * 2 * (CO > 16 ? 768 : 512) + (CO > 16 ? 256 : 0); }
template <int CO>
constexpr size_t tc2_smem() { return tc2_wbytes<CO>() + (size_t)TC2_RS * TC2_SLOT + TC2_PAD + (2 * TC2_RS + 4) * 8 + 16; }

// A run of tiles: plane t, first output column y0, first x and its length n.
struct TcRun {
    int t, y0, x0, n;
};
__device__ __forceinline__ TcRun tc_run(long long k, int X, int ny, int nxc, int XC)
{
    const unsigned kk = (unsigned)k, q = kk / (unsigned)nxc, xc = kk - q * (unsigned)nxc;
    TcRun r;
    r.t = (int)(q / (unsigned)ny);
    r.y0 = (int)(q - (unsigned)r.t * (unsigned)ny) * TCY;
    r.x0 = (int)xc * XC;
    r.n = X - r.x0 < XC ? X - r.x0 : XC;
    return r;
}

// Line step l of run r into `slot`: lanes 0..8 copy (t-line, group) e in bulk (rows inside
// the volume along y, counted in bytes on `bar`, armed first by lane 0), lanes 0..17 store the
// y-extension rows (y = -1 when y0 = 0, y = Y when the halo passes Y), which the copies never
// write; the stores are made visible to the tensor cores before lane 0's arrival.
__device__ __forceinline__ void tc2_stage_line(const __nv_bfloat16 *__restrict__ in, int T, int X, int Y, int bnd,
                                               const TcRun &r, int l, unsigned char *slot, uint32_t bar)
{
    const int lane = threadIdx.x & 31;
    const int gx = ext32(r.x0 - 1 + l, X, bnd);
    const int ys = r.y0 >= 1 ? r.y0 - 1 : 0, ye = r.y0 + TCY + 1 < Y ? r.y0 + TCY + 1 : Y;
    const uint32_t bytes = (uint32_t)(ye - ys) * 16u;
    if (lane == 0) asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(9u * bytes) : "memory");
    __syncwarp();
    if (lane < 9) {
        const int tl = lane / 3, g = lane - tl * 3;
        const int gt = ext32(r.t + tl - 1, T, bnd);
        const __nv_bfloat16 *src = in + gidx((int64_t)gt * X + gx, Y, ys, 8 * g);
        const uint32_t dst = energy_detail::smem_u32(slot + tl * TC2_TLINE + g * TC1_GRP + (ys - (r.y0 - 1)) * 16);
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                     "l"(src), "r"(bytes), "r"(bar)
                     : "memory");
    }
    if (lane < 18) {
        const int side = lane / 9, piece = lane - side * 9, tl = piece / 3, g = piece - tl * 3;
        const int row = side == 0 ? 0 : Y - r.y0 + 1;
        if (side == 0 ? r.y0 == 0 : row < TCH) {
            const int gt = ext32(r.t + tl - 1, T, bnd), gy = ext32(side == 0 ? -1 : Y, Y, bnd);
            *reinterpret_cast<uint4 *>(slot + tl * TC2_TLINE + g * TC1_GRP + row * 16) =
                *reinterpret_cast<const uint4 *>(in + gidx((int64_t)gt * X + gx, Y, gy, 8 * g));
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int CO>
__global__ void __launch_bounds__(TC2_NT, 1) conv_tc2_kernel(const __nv_bfloat16 *__restrict__ in, int T, int X,
                                                             int Y, int bnd, const float *__restrict__ w,
                                                             const float *__restrict__ b, __nv_bfloat16 *__restrict__ out,
                                                             float *__restrict__ E,
                                                             const float *__restrict__ out_scale_p, int *status,
                                                             int stall, uint64_t limit_ns, int XC)
{
    constexpr int NB = CO > 16 ? 32 : 16;       // N of the products
    constexpr int BT = CO > 16 ? 768 : 512;     // bytes between B tiles (24 or 16 stored rows x 16 BF16)
    constexpr int WB = (int)tc2_wbytes<CO>();   // + the 4th group the last tile reads
    static_assert(WB % 128 == 0 && TC2_SLOT % 128 == 0, "slots on 128-byte boundaries");
    using energy_detail::mbar_wait;
    using energy_detail::smem_u32;
    extern __shared__ __align__(128) unsigned char tc_sm[];
    unsigned char *sW = tc_sm, *sL = tc_sm + WB;                  // slot s at sL + s * TC2_SLOT, then the pad
    uint64_t *bar = reinterpret_cast<uint64_t *>(sL + TC2_RS * TC2_SLOT + TC2_PAD);
    // lfull[s]: line step in slot s landed (bytes + the producer's arrival); lfree[s]: its last
    // tile's products done; bacc[a]: accumulator a full; bdrain[a]: drained (one arrival per
    // epilogue warp).  Line step L uses slot L % RS (its L / RS-th use), tile G accumulator G % 2.
    uint64_t *lfull = bar, *lfree = bar + TC2_RS, *bacc = bar + 2 * TC2_RS, *bdrain = bar + 2 * TC2_RS + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2 * TC2_RS + 4);
    __shared__ float sb[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    constexpr int NS = BT / 32;                 // stored rows per B tile
    for (int e = threadIdx.x; e < 27 * 2 * NS * 16; e += TC2_NT) {
        const int kk = e & 15, n = (e >> 4) % NS, ts = e / (16 * NS), tap = ts >> 1, ks = ts & 1;
        const int cin = ks * 16 + kk;
        const float v = (n < CO && cin < kWidth) ? w[((int64_t)n * kWidth + cin) * 27 + tap] : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(sW + ts * BT + ((n >> 3) * 2 + (kk >> 3)) * 128 + (n & 7) * 16 + (kk & 7) * 2) =
            __float2bfloat16_rn(v);
    }
    for (int e = threadIdx.x; e < (WB - 27 * 2 * BT) / 16; e += TC2_NT)   // finite rows after the last tile
        *reinterpret_cast<uint4 *>(sW + 27 * 2 * BT + e * 16) = make_uint4(0, 0, 0, 0);
    if (threadIdx.x < 32) sb[threadIdx.x] = threadIdx.x < CO ? b[threadIdx.x] : 0.f;
    // slots and pad start at zero: every byte a product reads is finite (the upper group of a
    // t-line's second k-step is the next t-line's first group, or the pad, at zero weights)
    for (int e = threadIdx.x; e < (TC2_RS * TC2_SLOT + TC2_PAD) / 16; e += TC2_NT)
        *reinterpret_cast<uint4 *>(sL + e * 16) = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2 * TC2_RS + 4; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar + i)),
                         "r"(i >= 2 * TC2_RS + 2 ? TC2_EPI : 1)
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(tslot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    const int ny = (Y + TCY - 1) / TCY, nxc = (X + XC - 1) / XC;
    const long long nruns = (long long)T * ny * nxc;
    bool ok = true;

    if (warp == 0) {
        // ---- line steps, in run order, each once its slot's previous line step is released
        int L = 0;
        for (long long k = blockIdx.x; k < nruns && ok; k += gridDim.x) {
            const TcRun r = tc_run(k, X, ny, nxc, XC);
            for (int l = 0; l < r.n + 2; ++l, ++L) {
                const int s = L % TC2_RS, u = L / TC2_RS;
                if (u >= 1) {
                    const bool got = lane == 0 ? mbar_wait(smem_u32(lfree + s), (u - 1) & 1, limit_ns) : true;
                    if (!__shfl_sync(0xffffffffu, got ? 1 : 0, 0)) {
                        ok = false;
                        break;
                    }
                }
                tc2_stage_line(in, T, X, Y, bnd, r, l, sL + s * TC2_SLOT, smem_u32(lfull + s));
            }
        }
        // copies still in flight after a timeout land before the CTA exits
        if (lane == 0)
            for (int i = L - TC2_RS; i < L; ++i)
                if (i >= 0) mbar_wait(smem_u32(lfull + i % TC2_RS), (i / TC2_RS) & 1, limit_ns);
    } else if (warp == 1) {
        // ---- products: 27 taps x 2 k-steps of tile j from the slots of line steps j .. j + 2
        if (lane == 0) {
            constexpr uint32_t idesc = energy_detail::instr_desc(1, 128, NB);
            const uint64_t b0 = energy_detail::smem_desc(smem_u32(sW), 128, 256);
            int Lw = 0, Lb = 0, G = 0, last = -1;   // line steps waited for, first of the run, tiles
            for (long long k = blockIdx.x; k < nruns && ok; k += gridDim.x) {
                const TcRun r = tc_run(k, X, ny, nxc, XC);
                for (int j = 0; j < r.n; ++j, ++G) {
                    const int a = G & 1;
                    for (; Lw <= Lb + j + 2 && ok; ++Lw)
                        ok = mbar_wait(smem_u32(lfull + Lw % TC2_RS), (Lw / TC2_RS) & 1, limit_ns);
                    if (ok && G >= 2) ok = mbar_wait(smem_u32(bdrain + a), ((G >> 1) - 1) & 1, limit_ns);
                    if (!ok) break;
                    if (stall) continue;   // test hook: no products, so every later wait runs out
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t acc = tmem + (uint32_t)(32 * a);
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const uint64_t a0 =
                            energy_detail::smem_desc(smem_u32(sL + ((Lb + j + dx) % TC2_RS) * TC2_SLOT), TC1_GRP, 128);
#pragma unroll
                        for (int dt = 0; dt < 3; ++dt)
#pragma unroll
                            for (int dy = 0; dy < 3; ++dy)
#pragma unroll
                                for (int ks = 0; ks < 2; ++ks) {
                                    const int tap = (dt * 3 + dx) * 3 + dy;
                                    const uint32_t aoff = (dt * TC2_TLINE + dy * 16 + ks * 2 * TC1_GRP) >> 4;
                                    const uint32_t boff = ((tap * 2 + ks) * BT) >> 4;
                                    tc_mma_bf16(acc, a0 + aoff, b0 + boff, idesc, (tap | ks) != 0);
                                }
                    }
                    // tile j is the last reader of line step j (and of the run's last two)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(lfree + (Lb + j) % TC2_RS))
                                 : "memory");
                    if (j == r.n - 1)
                        for (int e = 1; e <= 2; ++e)
                            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                             smem_u32(lfree + (Lb + j + e) % TC2_RS))
                                         : "memory");
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(bacc + a))
                                 : "memory");
                    last = G;
                }
                Lb += r.n + 2;
            }
            // products still running after a timeout finish before the accumulators are freed
            if (last >= 0) mbar_wait(smem_u32(bacc + (last & 1)), (last >> 1) & 1, limit_ns);
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    } else {
        // ---- epilogue: accumulator G % 2 of tile G
        const int q = warp & 3, h = (warp - 2) >> 2;
        const float out_scale = out_scale_p ? *out_scale_p : 1.f;
        const long long Nv = (long long)T * X * Y;
        int G = 0;
        for (long long k = blockIdx.x; k < nruns && ok; k += gridDim.x) {
            const TcRun r = tc_run(k, X, ny, nxc, XC);
            for (int j = 0; j < r.n; ++j, ++G) {
                const int a = G & 1;
                const bool got = lane == 0 ? mbar_wait(smem_u32(bacc + a), (G >> 1) & 1, limit_ns) : true;
                if (!__shfl_sync(0xffffffffu, got ? 1 : 0, 0)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const TileC c{r.t, r.x0 + j, r.y0};
                const uint32_t acc = tmem + (uint32_t)(32 * a);
                if (CO == kWidth) {
                    tc_epilogue_hidden(acc, q, h, c, X, Y, sb, out);
                } else if (h == 0) {   // N = 16: one load per lane quadrant
                    float v[16];
                    energy_detail::tmem_ld16(acc + ((uint32_t)(32 * q) << 16), v);
                    const int y = c.y0 + 32 * q + lane;
                    if (y < Y) {
                        const long long vox = ((long long)c.t * X + c.x) * Y + y;
#pragma unroll
                        for (int ch = 0; ch < CO; ++ch) E[ch * Nv + vox] = (v[ch] + sb[ch]) * out_scale;
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bdrain + a)) : "memory");
            }
        }
    }
    if (!ok && lane == 0) atomicExch(status, (int)SAL_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

// One layer on the tensor cores: CO = 24 (hidden) or 3 (output, writes E).
template <int CO>
cudaError_t launch_conv_tc(const __nv_bfloat16 *in, sal_dims d, int bnd, const float *w, const float *b,
                           __nv_bfloat16 *out, float *E, const float *out_scale, const TcControl &c, cudaStream_t s)
{
    const int64_t ny = (d.Y + TCY - 1) / TCY, ntiles = d.T * d.X * ny;
    if (ntiles <= 0) return cudaSuccess;
    // tile coordinates and indices travel in 32 bits
    if (d.T > 0x7fffffff || d.X > 0x7fffffff || d.Y > 0x7fffffff || ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    constexpr size_t smem = tc2_smem<CO>();
    cudaError_t e = set_smem(conv_tc2_kernel<CO>, smem);
    if (e != cudaSuccess) return e;
    // runs along x of at most 64 tiles, shorter where that leaves fewer than 8 runs per SM
    int64_t XC = ntiles / ((int64_t)nsm * 8);
    XC = XC < 4 ? 4 : (XC > 64 ? 64 : XC);
    if (XC > d.X) XC = d.X;
    const int64_t nruns = d.T * ny * ((d.X + XC - 1) / XC);
    int64_t grid = nsm;                              // one CTA per SM (shared memory), persistent
    if (grid > nruns) grid = nruns;
    conv_tc2_kernel<CO><<<(unsigned)grid, TC2_NT, smem, s>>>(in, (int)d.T, (int)d.X, (int)d.Y, bnd, w, b, out, E,
                                                            out_scale, c.status, c.stall, c.limit_ns, (int)XC);
    return cudaGetLastError();
}

#define SAL_TRY(x)                          \
    do {                                    \
        cudaError_t e_ = (x);               \
        if (e_ != cudaSuccess) return e_;   \
    } while (0)

}  // namespace

int64_t surrogate_param_count() { return param_offset(kLayers); }

// Workspace: a 256-byte head (sum of squares, loss, the two scales), then
//   inference: two BF16 buffers of kWidth channels (ping-pong activations);
//   training:  Z[4][kWidth][N] pre-activations, A[4][kWidth][N] inputs of layers 1..4,
//              out[3][N] prediction, two gradient buffers [kWidth][N] (all FP32).
size_t surrogate_ws_bytes(sal_dims d, bool training)
{
    const size_t N = (size_t)(d.T * d.X * d.Y);
    if (!training) return 256 + 2 * (size_t)kWidth * N * sizeof(__nv_bfloat16);
    return 256 + ((size_t)8 * kWidth + 3 + 2 * (size_t)kWidth) * N * sizeof(float);
}

namespace {
struct SurrWs {
    double *sumsq, *loss;
    float *scale;          // [0] = 1 / rms, [1] = rms
    unsigned char *data;
};
SurrWs carve(void *ws)
{
    SurrWs w;
    w.sumsq = (double *)ws;
    w.loss = w.sumsq + 1;
    w.scale = (float *)(w.sumsq + 2);
    w.data = (unsigned char *)ws + 256;
    return w;
}
struct TrainBufs {
    float *Z[4], *A[4], *out, *g0, *g1;
};
TrainBufs train_bufs(const SurrWs &w, int64_t N)
{
    TrainBufs b;
    float *p = (float *)w.data;
    for (int l = 0; l < 4; ++l) b.Z[l] = p + (int64_t)l * kWidth * N;
    p += (int64_t)4 * kWidth * N;
    for (int l = 0; l < 4; ++l) b.A[l] = p + (int64_t)l * kWidth * N;
    p += (int64_t)4 * kWidth * N;
    b.out = p;
    p += 3 * N;
    b.g0 = p;
    b.g1 = p + (int64_t)kWidth * N;
    return b;
}
const float *Wp(const float *params, int l) { return params + param_offset(l); }
const float *Bp(const float *params, int l) { return params + param_offset(l) + (int64_t)kWidths[l + 1] * kWidths[l] * 27; }
float *Wg(float *grads, int l) { return grads + param_offset(l); }
float *Bg(float *grads, int l) { return grads + param_offset(l) + (int64_t)kWidths[l + 1] * kWidths[l] * 27; }
}  // namespace

cudaError_t surrogate_forward(const float *V, sal_dims d, int bnd, const float *params, float *E, bool training,
                              void *ws, cudaStream_t s, int prec, const TcControl *tc)
{
    const int64_t N = d.T * d.X * d.Y;
    SurrWs w = carve(ws);
    SAL_TRY(cudaMemsetAsync(w.sumsq, 0, 2 * sizeof(double), s));
    sumsq_kernel<<<1024, 256, 0, s>>>(V, N, w.sumsq);
    SAL_TRY(cudaGetLastError());
    rms_kernel<<<1, 1, 0, s>>>(w.sumsq, N, w.scale);
    SAL_TRY(cudaGetLastError());
    const float *P = params;
    if (!training && prec == SAL_PREC_BF16) {
        // layers 2..5 on the tensor cores (layer 1 has a single input channel); activations
        // interleaved [voxel][24]
        if (!tc || !tc->status) return cudaErrorInvalidValue;
        __nv_bfloat16 *a0 = (__nv_bfloat16 *)w.data, *a1 = a0 + (int64_t)kWidth * N;
        SAL_TRY((launch_conv<1, kWidth, float, __nv_bfloat16, FWD_HIDDEN, true>(V, d, bnd, w.scale, Wp(P, 0), Bp(P, 0), nullptr, a0, nullptr, nullptr, s)));
        SAL_TRY(launch_conv_tc<kWidth>(a0, d, bnd, Wp(P, 1), Bp(P, 1), a1, nullptr, nullptr, *tc, s));
        SAL_TRY(launch_conv_tc<kWidth>(a1, d, bnd, Wp(P, 2), Bp(P, 2), a0, nullptr, nullptr, *tc, s));
        SAL_TRY(launch_conv_tc<kWidth>(a0, d, bnd, Wp(P, 3), Bp(P, 3), a1, nullptr, nullptr, *tc, s));
        SAL_TRY(launch_conv_tc<3>(a1, d, bnd, Wp(P, 4), Bp(P, 4), nullptr, E, w.scale + 1, *tc, s));
        return cudaSuccess;
    }
    if (!training) {
        __nv_bfloat16 *a0 = (__nv_bfloat16 *)w.data, *a1 = a0 + (int64_t)kWidth * N;
        SAL_TRY((launch_conv<1, kWidth, float, __nv_bfloat16, FWD_HIDDEN>(V, d, bnd, w.scale, Wp(P, 0), Bp(P, 0), nullptr, a0, nullptr, nullptr, s)));
        SAL_TRY((launch_conv<kWidth, kWidth, __nv_bfloat16, __nv_bfloat16, FWD_HIDDEN>(a0, d, bnd, nullptr, Wp(P, 1), Bp(P, 1), nullptr, a1, nullptr, nullptr, s)));
        SAL_TRY((launch_conv<kWidth, kWidth, __nv_bfloat16, __nv_bfloat16, FWD_HIDDEN>(a1, d, bnd, nullptr, Wp(P, 2), Bp(P, 2), nullptr, a0, nullptr, nullptr, s)));
        SAL_TRY((launch_conv<kWidth, kWidth, __nv_bfloat16, __nv_bfloat16, FWD_HIDDEN>(a0, d, bnd, nullptr, Wp(P, 3), Bp(P, 3), nullptr, a1, nullptr, nullptr, s)));
        SAL_TRY((launch_conv<kWidth, 3, __nv_bfloat16, float, FWD_OUTPUT>(a1, d, bnd, nullptr, Wp(P, 4), Bp(P, 4), nullptr, E, w.scale + 1, nullptr, s)));
        return cudaSuccess;
    }
    TrainBufs b = train_bufs(w, N);
    SAL_TRY((launch_conv<1, kWidth, float, float, FWD_HIDDEN>(V, d, bnd, w.scale, Wp(P, 0), Bp(P, 0), b.Z[0], b.A[0], nullptr, nullptr, s)));
    for (int l = 1; l < 4; ++l)
        SAL_TRY((launch_conv<kWidth, kWidth, float, float, FWD_HIDDEN>(b.A[l - 1], d, bnd, nullptr, Wp(P, l), Bp(P, l), b.Z[l], b.A[l], nullptr, nullptr, s)));
    SAL_TRY((launch_conv<kWidth, 3, float, float, FWD_OUTPUT>(b.A[3], d, bnd, nullptr, Wp(P, 4), Bp(P, 4), nullptr, b.out, nullptr, nullptr, s)));
    if (E) {
        scale_kernel<<<1024, 256, 0, s>>>(b.out, 3 * N, w.scale + 1, E);   // back to the units of E
        SAL_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

cudaError_t surrogate_backward(const float *V, sal_dims d, int bnd, const float *params, const float *Etarget,
                               int margin, float *grads, double *loss, void *ws, cudaStream_t s)
{
    const int64_t N = d.T * d.X * d.Y;
    SurrWs w = carve(ws);
    TrainBufs b = train_bufs(w, N);
    const float *P = params;
    const int64_t cnt = (d.T - 2 * margin) * (d.X - 2 * margin) * (d.Y - 2 * margin);
    if (cnt <= 0) return cudaErrorInvalidValue;
    SAL_TRY(cudaMemsetAsync(grads, 0, surrogate_param_count() * sizeof(float), s));
    SAL_TRY(cudaMemsetAsync(w.loss, 0, sizeof(double), s));
    float *g = b.g0, *gn = b.g1;
    loss_grad_kernel<<<1024, 256, 0, s>>>(b.out, Etarget, w.scale, d.T, d.X, d.Y, margin, 1.f / (3.f * (float)cnt), g, w.loss);
    SAL_TRY(cudaGetLastError());
    SAL_TRY((launch_wgrad<kWidth, 3>(b.A[3], nullptr, g, d, bnd, Wg(grads, 4), Bg(grads, 4), s)));
    SAL_TRY((launch_conv<3, kWidth, float, float, BWD_DATA>(g, d, bnd, nullptr, Wp(P, 4), nullptr, nullptr, gn, nullptr, b.Z[3], s)));
    for (int l = 3; l >= 1; --l) {
        float *t = g;
        g = gn;
        gn = t;
        SAL_TRY((launch_wgrad<kWidth, kWidth>(b.A[l - 1], nullptr, g, d, bnd, Wg(grads, l), Bg(grads, l), s)));
        SAL_TRY((launch_conv<kWidth, kWidth, float, float, BWD_DATA>(g, d, bnd, nullptr, Wp(P, l), nullptr, nullptr, gn, nullptr, b.Z[l - 1], s)));
    }
    SAL_TRY((launch_wgrad<1, kWidth>(V, w.scale, gn, d, bnd, Wg(grads, 0), Bg(grads, 0), s)));
    if (loss) SAL_TRY(cudaMemcpyAsync(loss, w.loss, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return cudaSuccess;
}

// ---- inference with the per-block fallback -----------------------------------------------
namespace {
struct InferLayout {
    size_t fwd, coords, eex, sums, list, counters, total;
    int64_t nb, nbx, nby, ntiles;
    int bt, bx;
    int64_t tiles_t, tiles_x, tiles_y;
};
size_t r256(size_t v) { return (v + 255) & ~(size_t)255; }
InferLayout infer_layout(sal_dims d, int L)
{
    InferLayout w;
    const TileShape sh = energy_shape(L, 0);
    w.bt = sh.bt;
    w.bx = sh.bx;
    w.tiles_t = (d.T + w.bt - 1) / w.bt;
    w.tiles_x = (d.X + w.bx - 1) / w.bx;
    w.tiles_y = (d.Y + 31) / 32;
    w.ntiles = w.tiles_t * w.tiles_x * w.tiles_y;
    const int64_t nbt = (d.T + FB_T - 1) / FB_T;
    w.nbx = (d.X + FB_X - 1) / FB_X;
    w.nby = (d.Y + FB_Y - 1) / FB_Y;
    w.nb = nbt * w.nbx * w.nby;
    w.fwd = 0;
    w.coords = r256(surrogate_ws_bytes(d, false));
    w.eex = r256(w.coords + (size_t)w.nb * FB_S * 3 * sizeof(int64_t));
    w.sums = r256(w.eex + (size_t)w.nb * FB_S * 3 * sizeof(float));
    w.list = r256(w.sums + 4 * sizeof(float));
    w.counters = r256(w.list + (size_t)w.ntiles * sizeof(int64_t));
    w.total = r256(w.counters + 4 * sizeof(int));
    return w;
}
}  // namespace

size_t surrogate_infer_ws_bytes(sal_dims d, int L) { return infer_layout(d, L).total; }

cudaError_t surrogate_infer(const float *V, sal_dims d, int L, int bnd, const float *params, float *E, float thr,
                            int *counts, void *ws, cudaStream_t s, int prec, const TcControl *tc)
{
    const InferLayout w = infer_layout(d, L);
    if (w.bt <= 0 || FB_T % w.bt || FB_X % w.bx) return cudaErrorInvalidValue;
    unsigned char *base = (unsigned char *)ws;
    int64_t *coords = (int64_t *)(base + w.coords);
    float *eex = (float *)(base + w.eex), *sums = (float *)(base + w.sums);
    int64_t *list = (int64_t *)(base + w.list);
    int *ctr = (int *)(base + w.counters);          // [0] tiles queued, [1] blocks recomputed, [2] checked
    SAL_TRY(surrogate_forward(V, d, bnd, params, E, false, base + w.fwd, s, prec, tc));
    const int64_t ns = w.nb * FB_S;
    sample_coords_kernel<<<(unsigned)((ns + 255) / 256 < 4096 ? (ns + 255) / 256 : 4096), 256, 0, s>>>(d.T, d.X, d.Y, w.nbx,
                                                                                                      w.nby, w.nb, coords);
    SAL_TRY(cudaGetLastError());
    SAL_TRY(launch_energy_points(V, d, L, bnd, coords, ns, eex, s));
    SAL_TRY(cudaMemsetAsync(sums, 0, 4 * sizeof(float), s));
    SAL_TRY(cudaMemsetAsync(ctr, 0, 4 * sizeof(int), s));
    sample_sums_kernel<<<256, 256, 0, s>>>(eex, ns, sums);
    SAL_TRY(cudaGetLastError());
    block_check_kernel<<<(unsigned)((w.nb + 255) / 256), 256, 0, s>>>(E, d.T, d.X, d.Y, coords, eex, w.nb, sums, thr, w.bt,
                                                                      w.bx, w.tiles_t, w.tiles_x, w.tiles_y, w.nbx,
                                                                      w.nby, list, ctr, ctr + 1);
    SAL_TRY(cudaGetLastError());
    SAL_TRY(launch_energy_fp32_list(V, d, L, bnd, list, ctr, E, s));
    if (counts) SAL_TRY(cudaMemcpyAsync(counts, ctr + 1, 2 * sizeof(int), cudaMemcpyDeviceToDevice, s));
    return cudaSuccess;
}

cudaError_t surrogate_adam(float *params, const float *grads, float *m, float *v, int64_t n, int step, float lr,
                           float b1, float b2, float eps, cudaStream_t s)
{
    const float c1 = 1.f / (1.f - powf(b1, (float)step)), c2 = 1.f / (1.f - powf(b2, (float)step));
    adam_kernel<<<256, 256, 0, s>>>(params, grads, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace sal
