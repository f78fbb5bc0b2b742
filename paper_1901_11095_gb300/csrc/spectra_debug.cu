// Materialised intermediate stages, for inspection and per-stage tests:
//   local_spectra: |F| of the full L^3 local spectrum of each voxel of a region (Sec. 2,
//                  the DFT printed below Eq. 2, normalised by L^-3), centred slot order;
//   project:       spectra -> E_t, E_x, E_y (Eq. 1-4 and the third step of Sec. 2).
// The fused energy kernel computes the same quantities without storing the spectra.
#include "sal_internal.cuh"

namespace sal {

namespace {

__device__ __forceinline__ int mod_l(int v, int L)
{
    int r = v % L;
    return r < 0 ? r + L : r;
}

// One CTA per voxel of the region; the three mode products run on the whole cube in
// shared memory.  Samples are taken relative to the cube's centre sample, which changes
// no off-DC coefficient and makes a constant cube's off-DC spectrum exactly zero.
// POINTS = false: voxels of the box lt.. + et.. (C order), |F| written to `mag`;
// POINTS = true: voxels coords[k] (t, x, y), E_m written to E[m * n + k] (Eq. 1-4 and the
// non-DC mean), via the same spectrum.
template <bool POINTS>
__global__ void __launch_bounds__(256) local_spectra_kernel(const float *__restrict__ V, int64_t T, int64_t X,
                                                            int64_t Y, int L, int bnd, int64_t lt, int64_t lx,
                                                            int64_t ly, int64_t et, int64_t ex, int64_t ey,
                                                            const int64_t *__restrict__ coords, int64_t npts,
                                                            float *__restrict__ mag, float *__restrict__ Eout,
                                                            const __grid_constant__ SpecTables tw)
{
    extern __shared__ __align__(16) float2 dyn[];   // g1[n3], g2[n3], f[n3]
    __shared__ float red[8];
    __shared__ float redE[8][3];
    const int64_t v = blockIdx.x;
    int64_t t, x, y;
    if (POINTS) {
        t = coords[3 * v];
        x = coords[3 * v + 1];
        y = coords[3 * v + 2];
    } else {
        const int64_t vy = v % ey, vx = (v / ey) % ex, vt = v / (ey * ex);
        t = lt + vt;
        x = lx + vx;
        y = ly + vy;
    }
    const int h = (L - 1) / 2, n3 = L * L * L;
    float2 *g1 = dyn, *g2 = dyn + n3;
    float *f = reinterpret_cast<float *>(dyn + 2 * n3);

    float part = 0.f;
    for (int i = threadIdx.x; i < n3; i += blockDim.x) {
        const int p = i / (L * L), q = (i / L) % L, r = i % L;
        const int64_t gt = ext_index(t - h + p, T, bnd), gx = ext_index(x - h + q, X, bnd),
                      gy = ext_index(y - h + r, Y, bnd);
        const float s = V[(gt * X + gx) * Y + gy];
        f[i] = s;
        part += s;
    }
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    const float centre = f[(h * L + h) * L + h];
    __syncthreads();
    for (int i = threadIdx.x; i < n3; i += blockDim.x) f[i] -= centre;
    __syncthreads();

    // stage t: g1[a][q][r] = sum_p f[p][q][r] e^{-i th mu (p-h)}, mu = a - h
    for (int i = threadIdx.x; i < n3; i += blockDim.x) {
        const int a = i / (L * L), q = (i / L) % L, r = i % L, mu = a - h;
        float re = 0.f, im = 0.f;
        for (int p = 0; p < L; ++p) {
            const int k = mod_l(mu * (p - h), L);
            const float s = f[(p * L + q) * L + r];
            re = fmaf(s, tw.cs[k], re);
            im = fmaf(-s, tw.sn[k], im);
        }
        g1[i] = make_float2(re, im);
    }
    __syncthreads();
    // stage x: g2[a][b][r] = sum_q g1[a][q][r] e^{-i th nu (q-h)}
    for (int i = threadIdx.x; i < n3; i += blockDim.x) {
        const int a = i / (L * L), b = (i / L) % L, r = i % L, nu = b - h;
        float re = 0.f, im = 0.f;
        for (int q = 0; q < L; ++q) {
            const int k = mod_l(nu * (q - h), L);
            const float2 z = g1[(a * L + q) * L + r];
            re += z.x * tw.cs[k] + z.y * tw.sn[k];
            im += z.y * tw.cs[k] - z.x * tw.sn[k];
        }
        g2[i] = make_float2(re, im);
    }
    __syncthreads();
    // stage y and magnitude
    const float inv = 1.f / (float)n3;
    float *out = POINTS ? nullptr : mag + v * n3;
    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
    for (int i = threadIdx.x; i < n3; i += blockDim.x) {
        const int a = i / (L * L), b = (i / L) % L, c = i % L, om = c - h;
        float re = 0.f, im = 0.f;
        for (int r = 0; r < L; ++r) {
            const int k = mod_l(om * (r - h), L);
            const float2 z = g2[(a * L + b) * L + r];
            re += z.x * tw.cs[k] + z.y * tw.sn[k];
            im += z.y * tw.cs[k] - z.x * tw.sn[k];
        }
        const float m = sqrtf(re * re + im * im) * inv;
        if (POINTS) {
            const float *w = &tw.w[((abs(a - h) * kMaxHalf + abs(b - h)) * kMaxHalf + abs(om)) * 3];   // 0 at DC
            e0 = fmaf(w[0], m, e0);
            e1 = fmaf(w[1], m, e1);
            e2 = fmaf(w[2], m, e2);
        } else {
            out[i] = m;
        }
    }
    if (POINTS) {
        for (int o = 16; o; o >>= 1) {
            e0 += __shfl_xor_sync(0xffffffffu, e0, o);
            e1 += __shfl_xor_sync(0xffffffffu, e1, o);
            e2 += __shfl_xor_sync(0xffffffffu, e2, o);
        }
        if ((threadIdx.x & 31) == 0) {
            redE[threadIdx.x >> 5][0] = e0;
            redE[threadIdx.x >> 5][1] = e1;
            redE[threadIdx.x >> 5][2] = e2;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            float s = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += redE[w][threadIdx.x];
            Eout[threadIdx.x * npts + v] = s / (float)(n3 - 1);
        }
    } else if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        out[(h * L + h) * L + h] = fabsf(s) * inv;
    }
}

// One warp per voxel: E_m = (L^3 - 1)^-1 sum_{non-DC} w_m |F|.
__global__ void __launch_bounds__(256) project_kernel(const float *__restrict__ mag, int64_t n, int L,
                                                      float *__restrict__ E, const __grid_constant__ SpecTables tb)
{
    const int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= n) return;
    const int h = (L - 1) / 2, n3 = L * L * L;
    const float *m = mag + v * n3;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int i = lane; i < n3; i += 32) {
        const int a = abs(i / (L * L) - h), b = abs((i / L) % L - h), c = abs(i % L - h);
        const float *w = &tb.w[((a * kMaxHalf + b) * kMaxHalf + c) * 3];   // 0 at DC
        const float f = m[i];
        s0 = fmaf(w[0], f, s0);
        s1 = fmaf(w[1], f, s1);
        s2 = fmaf(w[2], f, s2);
    }
    for (int o = 16; o; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        const float inv = 1.f / (float)(n3 - 1);
        E[v] = s0 * inv;
        E[n + v] = s1 * inv;
        E[2 * n + v] = s2 * inv;
    }
}

}  // namespace

cudaError_t launch_local_spectra(const float *V, sal_dims d, int L, int bnd, const int64_t lo[3], const int64_t ext[3],
                                 float *mag, cudaStream_t s)
{
    const int64_t n = ext[0] * ext[1] * ext[2];
    if (n <= 0) return cudaSuccess;
    if (n > 0x7fffffffLL) return cudaErrorInvalidValue;
    SpecTables tb;
    make_tables(L, &tb);
    const size_t smem = (size_t)L * L * L * (2 * sizeof(float2) + sizeof(float));
    cudaError_t e = set_smem(local_spectra_kernel<false>, smem);
    if (e != cudaSuccess) return e;
    local_spectra_kernel<false><<<(unsigned)n, 256, smem, s>>>(V, d.T, d.X, d.Y, L, bnd, lo[0], lo[1], lo[2], ext[0],
                                                            ext[1], ext[2], nullptr, 0, mag, nullptr, tb);
    return cudaGetLastError();
}

cudaError_t launch_energy_points(const float *V, sal_dims d, int L, int bnd, const int64_t *coords, int64_t n, float *E,
                                 cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (n > 0x7fffffffLL) return cudaErrorInvalidValue;
    SpecTables tb;
    make_tables(L, &tb);
    const size_t smem = (size_t)L * L * L * (2 * sizeof(float2) + sizeof(float));
    cudaError_t e = set_smem(local_spectra_kernel<true>, smem);
    if (e != cudaSuccess) return e;
    local_spectra_kernel<true><<<(unsigned)n, 256, smem, s>>>(V, d.T, d.X, d.Y, L, bnd, 0, 0, 0, 1, 1, 1, coords, n,
                                                           nullptr, E, tb);
    return cudaGetLastError();
}

cudaError_t launch_project(const float *mag, int64_t n, int L, float *E, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    SpecTables tb;
    make_tables(L, &tb);
    const int64_t blocks = (n * 32 + 255) / 256;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    project_kernel<<<(unsigned)blocks, 256, 0, s>>>(mag, n, L, E, tb);
    return cudaGetLastError();
}

}  // namespace sal
