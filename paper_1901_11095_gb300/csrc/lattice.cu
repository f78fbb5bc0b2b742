// Coarse-stride cubes (Sec. 2, first step: the local cube slides "with more than 50 %
// overlap").  With a stride s > 1 the cubes are centred on the lattice c_i = min(i s, n - 1)
// of every axis (the last sample always a centre), E_m is computed for those cubes only, and
// every voxel takes the trilinear interpolation of the 2 x 2 x 2 lattice energies around it.
//
// lattice_energy_kernel: one CTA per lattice plane i and block of BJ x BK lattice points.
// The CTA stages the V region their cubes cover (L planes around the plane's centre, the x
// and y ranges of its points plus h on each side), then per mu = 0..h:
//   stage t: G1(x', y') = sum_p V(p, x', y') e^{-i th mu (p-h)} for every column of the region;
//   stage x: G2(nu, j, y') = sum_q G1(x_j - h + q, y') e^{-i th nu (q-h)} at the lattice x_j;
//   stage y: F(nu, omega) at the lattice y_k by the folded DFT (one pass gives +-omega), then
//            |F| weighted by the projections of Eq. 1-4 into per-(point, nu) sums.
// mu > 0 counts twice (|F(-k)| = |F(k)| for real input); the DC point has weight 0.  Every
// sample is taken relative to one reference value of the region (no coefficient off DC
// changes), so a constant region has an exactly zero spectrum.
#include <algorithm>

#include "sal_internal.cuh"

namespace sal {

namespace {

constexpr int kLatThreads = 256;

__host__ __device__ __forceinline__ int64_t lattice_coord(int64_t i, int64_t n, int s)
{
    const int64_t c = i * (int64_t)s;
    return c < n - 1 ? c : n - 1;
}

struct LatGeo {
    int s, BJ, BK, RXM, RYM;   // stride, lattice points per CTA along x and y, region bounds
    int nbj, nbk;              // CTA blocks along x and y
    int64_t Tc, Xc, Yc;
};

// Shared memory of one CTA, in floats: the V region (rounded up to 16 bytes so the complex
// arrays after it stay aligned), G1 and G2 (complex), the per-(point, nu) sums of three maps.
__host__ __device__ inline size_t lat_region_floats(int L, int RXM, int RYM) { return ((size_t)L * RXM * RYM + 3) & ~(size_t)3; }
inline size_t lat_smem_bytes(int L, int BJ, int BK, int RXM, int RYM)
{
    return sizeof(float) * (lat_region_floats(L, RXM, RYM) + 2 * (size_t)RXM * RYM + 2 * (size_t)L * BJ * RYM +
                            3 * (size_t)BJ * BK * L);
}

template <int L>
__global__ void __launch_bounds__(kLatThreads) lattice_energy_kernel(const float *__restrict__ V, int64_t T, int64_t X,
                                                                     int64_t Y, int bnd, const LatGeo g,
                                                                     float *__restrict__ Ec,
                                                                     const __grid_constant__ SpecTables tb)
{
    constexpr int H = (L - 1) / 2;
    extern __shared__ __align__(16) float smem[];
    const int tid = threadIdx.x;
    int64_t b = blockIdx.x;
    const int kb = (int)(b % g.nbk);
    b /= g.nbk;
    const int jb = (int)(b % g.nbj);
    const int64_t i = b / g.nbj;
    const int64_t j0 = (int64_t)jb * g.BJ, k0 = (int64_t)kb * g.BK;
    const int nj = (int)min((int64_t)g.BJ, g.Xc - j0), nk = (int)min((int64_t)g.BK, g.Yc - k0);
    const int64_t tc = lattice_coord(i, T, g.s);
    const int64_t xlo = lattice_coord(j0, X, g.s) - H, ylo = lattice_coord(k0, Y, g.s) - H;
    const int RX = (int)(lattice_coord(j0 + nj - 1, X, g.s) + H - xlo + 1);
    const int RY = (int)(lattice_coord(k0 + nk - 1, Y, g.s) + H - ylo + 1);
    const int P = g.RYM;                                   // row pitch of the region (floats / float2)

    float *sV = smem;                                      // [L][RXM][P]
    float2 *sG1 = reinterpret_cast<float2 *>(sV + lat_region_floats(L, g.RXM, P));   // [RXM][P]
    float2 *sG2 = sG1 + (size_t)g.RXM * P;                 // [L (nu)][BJ][P]
    float *acc = reinterpret_cast<float *>(sG2 + (size_t)L * g.BJ * P);      // [3][BJ * BK * L]
    const int nitems = nj * nk * L;                        // (point, nu) items of stage y
    const int accn = g.BJ * g.BK * L;

    // the region of V, relative to one sample of it, with the boundary extension
    const float ref = V[(tc * X + (xlo + H)) * Y + (ylo + H)];
    for (int e = tid; e < L * RX * RY; e += kLatThreads) {
        const int p = e / (RX * RY), rem = e - p * (RX * RY), q = rem / RY, r = rem - q * RY;
        const int64_t gt = ext_index(tc - H + p, T, bnd), gx = ext_index(xlo + q, X, bnd), gy = ext_index(ylo + r, Y, bnd);
        sV[(p * g.RXM + q) * P + r] = V[(gt * X + gx) * Y + gy] - ref;
    }
    for (int e = tid; e < 3 * accn; e += kLatThreads) acc[e] = 0.f;
    __syncthreads();

    for (int mu = 0; mu <= H; ++mu) {
        // stage t: G1 of every column of the region
        for (int e = tid; e < RX * RY; e += kLatThreads) {
            const int q = e / RY, r = e - q * RY;
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int p = 0; p < L; ++p) {
                const int k = ((mu * (p - H)) % L + L) % L;       // e^{-i th k} = cs[k] - i sn[k]
                const float v = sV[(p * g.RXM + q) * P + r];
                re = fmaf(v, tb.cs[k], re);
                im = fmaf(-v, tb.sn[k], im);
            }
            sG1[q * P + r] = make_float2(re, im);
        }
        __syncthreads();
        // stage x: G2 of every nu at the lattice x of this CTA, every column y'
        for (int e = tid; e < L * nj * RY; e += kLatThreads) {
            const int nu = e / (nj * RY), rem = e - nu * (nj * RY), j = rem / RY, r = rem - j * RY;
            const int xq = (int)(lattice_coord(j0 + j, X, g.s) - H - xlo);
            const int nus = nu - H;
            float re = 0.f, im = 0.f;
#pragma unroll
            for (int q = 0; q < L; ++q) {
                const int k = ((nus * (q - H)) % L + L) % L;
                const float2 z = sG1[(xq + q) * P + r];
                const float c = tb.cs[k], sn = tb.sn[k];
                re = fmaf(z.x, c, fmaf(z.y, sn, re));            // (zr + i zi)(c - i s)
                im = fmaf(z.y, c, fmaf(-z.x, sn, im));
            }
            sG2[(nu * g.BJ + j) * P + r] = make_float2(re, im);
        }
        __syncthreads();
        // stage y: the folded DFT of each (point, nu) line at the lattice y, |F|, weights
        const float mult = mu == 0 ? 1.f : 2.f;
        for (int it = tid; it < nitems; it += kLatThreads) {
            const int nu = it % L, pt = it / L, j = pt / nk, k = pt - j * nk;
            const int yq = (int)(lattice_coord(k0 + k, Y, g.s) - H - ylo);
            const float2 *line = sG2 + (nu * g.BJ + j) * P + yq;
            const float2 z0 = line[H];
            float2 U[H + 1], D[H + 1];
            float2 s0 = z0;
#pragma unroll
            for (int r = 1; r <= H; ++r) {
                const float2 a = line[H + r], c = line[H - r];
                U[r] = make_float2(a.x + c.x, a.y + c.y);
                D[r] = make_float2(a.x - c.x, a.y - c.y);
                s0.x += U[r].x;
                s0.y += U[r].y;
            }
            const int anu = nu >= H ? nu - H : H - nu;
            const float *w0 = tb.w + ((mu * kMaxHalf + anu) * kMaxHalf) * 3;
            float et = 0.f, ex = 0.f, ey = 0.f;
            {
                const float m0 = sqrtf(fmaf(s0.x, s0.x, s0.y * s0.y));
                et = fmaf(w0[0], m0, et);
                ex = fmaf(w0[1], m0, ex);
                ey = fmaf(w0[2], m0, ey);
            }
#pragma unroll
            for (int om = 1; om <= H; ++om) {
                float2 A = z0, B = make_float2(0.f, 0.f);
#pragma unroll
                for (int r = 1; r <= H; ++r) {
                    const int k = (om * r) % L;
                    A.x = fmaf(U[r].x, tb.cs[k], A.x);
                    A.y = fmaf(U[r].y, tb.cs[k], A.y);
                    B.x = fmaf(D[r].x, tb.sn[k], B.x);
                    B.y = fmaf(D[r].y, tb.sn[k], B.y);
                }
                // F(+om) = A - iB, F(-om) = A + iB
                const float pr = A.x + B.y, pi = A.y - B.x, qr = A.x - B.y, qi = A.y + B.x;
                const float m = sqrtf(fmaf(pr, pr, pi * pi)) + sqrtf(fmaf(qr, qr, qi * qi));
                const float *w = w0 + om * 3;
                et = fmaf(w[0], m, et);
                ex = fmaf(w[1], m, ex);
                ey = fmaf(w[2], m, ey);
            }
            const int slot = (j * g.BK + k) * L + nu;
            acc[slot] = fmaf(mult, et, acc[slot]);
            acc[accn + slot] = fmaf(mult, ex, acc[accn + slot]);
            acc[2 * accn + slot] = fmaf(mult, ey, acc[2 * accn + slot]);
        }
        __syncthreads();
    }

    // E_m of each point: the sum over nu, times L^-3 (DFT) and (L^3 - 1)^-1 (non-DC mean)
    const float scale = tb.escale * 0.5f;   // escale holds the half-spectrum factor 2, applied above
    const int64_t Nc = g.Tc * g.Xc * g.Yc;
    for (int e = tid; e < 3 * nj * nk; e += kLatThreads) {
        const int m = e / (nj * nk), pt = e - m * (nj * nk), j = pt / nk, k = pt - j * nk;
        const float *a = acc + m * accn + (j * g.BK + k) * L;
        float sum = 0.f;
#pragma unroll
        for (int nu = 0; nu < L; ++nu) sum += a[nu];
        Ec[m * Nc + (i * g.Xc + (j0 + j)) * g.Yc + (k0 + k)] = sum * scale;
    }
}

// Trilinear interpolation of the lattice energies back to every voxel: one CTA row walk per
// (t, x) row, the t and x segments computed once per row, y along the threads.
__global__ void __launch_bounds__(256) interp_kernel(const float *__restrict__ Ec, int64_t T, int64_t X, int64_t Y,
                                                     int s, int64_t Tc, int64_t Xc, int64_t Yc, float *__restrict__ E)
{
    const int64_t N = T * X * Y, Nc = Tc * Xc * Yc;
    for (int64_t row = blockIdx.x; row < T * X; row += gridDim.x) {
        const int64_t t = row / X, x = row - t * X;
        int64_t it = Tc > 1 ? min(t / s, Tc - 2) : 0, ix = Xc > 1 ? min(x / s, Xc - 2) : 0;
        float ft = 0.f, fx = 0.f;
        if (Tc > 1) {
            const int64_t lo = lattice_coord(it, T, s), hi = lattice_coord(it + 1, T, s);
            ft = (float)(t - lo) / (float)(hi - lo);
        }
        if (Xc > 1) {
            const int64_t lo = lattice_coord(ix, X, s), hi = lattice_coord(ix + 1, X, s);
            fx = (float)(x - lo) / (float)(hi - lo);
        }
        const int64_t it1 = Tc > 1 ? it + 1 : it, ix1 = Xc > 1 ? ix + 1 : ix;
        const float w00 = (1.f - ft) * (1.f - fx), w01 = (1.f - ft) * fx, w10 = ft * (1.f - fx), w11 = ft * fx;
        const int64_t r00 = (it * Xc + ix) * Yc, r01 = (it * Xc + ix1) * Yc, r10 = (it1 * Xc + ix) * Yc,
                      r11 = (it1 * Xc + ix1) * Yc;
        for (int64_t y = threadIdx.x; y < Y; y += blockDim.x) {
            const int64_t iy = Yc > 1 ? min(y / s, Yc - 2) : 0, iy1 = Yc > 1 ? iy + 1 : iy;
            float fy = 0.f;
            if (Yc > 1) {
                const int64_t lo = lattice_coord(iy, Y, s), hi = lattice_coord(iy + 1, Y, s);
                fy = (float)(y - lo) / (float)(hi - lo);
            }
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const float *c = Ec + m * Nc;
                const float a = fmaf(fy, c[r00 + iy1] - c[r00 + iy], c[r00 + iy]);
                const float bq = fmaf(fy, c[r01 + iy1] - c[r01 + iy], c[r01 + iy]);
                const float cq = fmaf(fy, c[r10 + iy1] - c[r10 + iy], c[r10 + iy]);
                const float d = fmaf(fy, c[r11 + iy1] - c[r11 + iy], c[r11 + iy]);
                E[m * N + row * Y + y] = w00 * a + w01 * bq + w10 * cq + w11 * d;
            }
        }
    }
}

template <int L>
cudaError_t launch_lattice_L(const float *V, sal_dims d, int bnd, const LatGeo &g, float *Ec, cudaStream_t st)
{
    SpecTables tb;
    make_tables(L, &tb);
    const size_t smem = lat_smem_bytes(L, g.BJ, g.BK, g.RXM, g.RYM);
    cudaError_t e = set_smem(lattice_energy_kernel<L>, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = g.Tc * g.nbj * g.nbk;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    lattice_energy_kernel<L><<<(unsigned)blocks, kLatThreads, smem, st>>>(V, d.T, d.X, d.Y, bnd, g, Ec, tb);
    return cudaGetLastError();
}

}  // namespace

int64_t lattice_size(int64_t n, int s) { return n <= 1 ? 1 : (n - 2) / s + 2; }

cudaError_t launch_lattice_energy(const float *V, sal_dims d, int L, int bnd, int s, float *Ec, cudaStream_t st)
{
    LatGeo g;
    g.s = s;
    g.Tc = lattice_size(d.T, s);
    g.Xc = lattice_size(d.X, s);
    g.Yc = lattice_size(d.Y, s);
    // the largest BJ x BK block (from 8 x 16) whose region fits 200 KB of shared memory
    g.BJ = 8;
    g.BK = 16;
    for (;;) {
        g.RXM = (g.BJ - 1) * s + L;
        g.RYM = (g.BK - 1) * s + L;
        const size_t need = lat_smem_bytes(L, g.BJ, g.BK, g.RXM, g.RYM);
        if (need <= 200 * 1024 || (g.BJ == 1 && g.BK == 1)) break;
        if (g.BK >= g.BJ && g.BK > 1) g.BK /= 2; else g.BJ /= 2;
    }
    g.nbj = (int)((g.Xc + g.BJ - 1) / g.BJ);
    g.nbk = (int)((g.Yc + g.BK - 1) / g.BK);
    switch (L) {
    case 3: return launch_lattice_L<3>(V, d, bnd, g, Ec, st);
    case 5: return launch_lattice_L<5>(V, d, bnd, g, Ec, st);
    case 7: return launch_lattice_L<7>(V, d, bnd, g, Ec, st);
    case 9: return launch_lattice_L<9>(V, d, bnd, g, Ec, st);
    case 11: return launch_lattice_L<11>(V, d, bnd, g, Ec, st);
    case 13: return launch_lattice_L<13>(V, d, bnd, g, Ec, st);
    case 15: return launch_lattice_L<15>(V, d, bnd, g, Ec, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_interp_lattice(const float *Ec, sal_dims d, int s, float *E, cudaStream_t st)
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int64_t rows = d.T * d.X, grid = (int64_t)nsm * 8;
    if (grid > rows) grid = rows;
    const int threads = d.Y >= 256 ? 256 : (int)((d.Y + 31) / 32 * 32);
    interp_kernel<<<(unsigned)grid, threads, 0, st>>>(Ec, d.T, d.X, d.Y, s, lattice_size(d.T, s), lattice_size(d.X, s),
                                                      lattice_size(d.Y, s), E);
    return cudaGetLastError();
}

}  // namespace sal
