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

struct LatGeo {
    int s, BJ, BK, RXM, RYM;   // stride, lattice points per CTA along x and y, region bounds
    int nbj, nbk;              // CTA blocks along x and y
    int64_t Tc, Xc, Yc;
};

// Shared memory of one CTA, in floats: G1 of every mu (complex), then a region that first
// holds the V samples and, once stage t has consumed them, G2 of one mu (complex); both
// rounded up to 16 bytes.
__host__ __device__ constexpr size_t lat_g1_floats(int L, int RXM, int RYM) { return 2 * (size_t)((L + 1) / 2) * RXM * RYM; }
__host__ __device__ constexpr size_t lat_reg_floats(int L, int BJ, int RXM, int RYM)
{
    return (((size_t)L * RXM * RYM > 2 * (size_t)L * BJ * RYM ? (size_t)L * RXM * RYM : 2 * (size_t)L * BJ * RYM) + 3) &
           ~(size_t)3;
}
__host__ __device__ constexpr size_t lat_smem_bytes(int L, int BJ, int BK, int RXM, int RYM)
{
    return sizeof(float) * (lat_g1_floats(L, RXM, RYM) + lat_reg_floats(L, BJ, RXM, RYM) + 3 * (size_t)BJ * BK * L);
}

// The lattice block of a CTA (BJ x BK points): the largest from 8 x 8 whose shared memory fits
// two CTAs per SM (110 KB) and whose stage-y (BJ BK L) and stage-x (BJ RYM) items are at most 4
// and 2 per thread.
struct LatBlock {
    int BJ, BK;
};
__host__ __device__ constexpr LatBlock lat_choose(int L, int s)
{
    int BJ = 8, BK = 8;
    for (;;) {
        const int RXM = (BJ - 1) * s + L, RYM = (BK - 1) * s + L;
        if ((lat_smem_bytes(L, BJ, BK, RXM, RYM) <= 110 * 1024 && BJ * BK * L <= 4 * kLatThreads &&
             BJ * RYM <= 2 * kLatThreads) ||
            (BJ == 1 && BK == 1))
            return LatBlock{BJ, BK};
        if (BK >= BJ && BK > 1) BK /= 2; else BJ /= 2;
    }
}

// |F| from |F|^2: the hardware approximate square root (one MUFU operation, a relative error
// of a few ulp, far inside the path's tolerance), as the stride-1 energy kernel uses.
__device__ __forceinline__ float lat_sqrt(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// cos and sin of 2 pi k / L for k = 0..L-1 (compile-time indices once unrolled).
template <int L>
struct LatTw {
    float c[L], s[L];
    __device__ __forceinline__ void load(const SpecTables &tb)
    {
#pragma unroll
        for (int k = 0; k < L; ++k) {
            c[k] = tb.cs[k];
            s[k] = tb.sn[k];
        }
    }
};

// Folded length-L DFT of the complex samples z[0..L-1] (centre z[H]): out[H + f] = F(f) =
// sum_r z[r] e^{-i th f (r - H)}, f = -H..H.  U_r = z(+r) + z(-r), D_r = z(+r) - z(-r);
// F(+-f) = A -+ iB with A = z0 + sum U_r cos(th f r), B = sum D_r sin(th f r).
template <int L>
__device__ __forceinline__ void folded_dft(const float2 (&z)[L], const LatTw<L> &tw, float2 (&out)[L])
{
    constexpr int H = (L - 1) / 2;
    float2 U[H + 1], D[H + 1];
    float2 s0 = z[H];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
        U[r] = make_float2(z[H + r].x + z[H - r].x, z[H + r].y + z[H - r].y);
        D[r] = make_float2(z[H + r].x - z[H - r].x, z[H + r].y - z[H - r].y);
        s0.x += U[r].x;
        s0.y += U[r].y;
    }
    out[H] = s0;
#pragma unroll
    for (int f = 1; f <= H; ++f) {
        float2 A = z[H], B = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            const int k = (f * r) % L;
            A.x = fmaf(U[r].x, tw.c[k], A.x);
            A.y = fmaf(U[r].y, tw.c[k], A.y);
            B.x = fmaf(D[r].x, tw.s[k], B.x);
            B.y = fmaf(D[r].y, tw.s[k], B.y);
        }
        out[H + f] = make_float2(A.x + B.y, A.y - B.x);   // A - iB
        out[H - f] = make_float2(A.x - B.y, A.y + B.x);   // A + iB
    }
}

// S_ > 0: the stride and hence the block geometry are compile-time constants (common cube
// sizes and strides): every region spans the full RXM x RYM (columns past a block's last
// lattice point are read, through the boundary extension at a face, and not used), so every
// loop bound and shared-memory pitch is a constant.  S_ = 0: run-time geometry from g.
template <int L, int S_ = 0>
__global__ void __launch_bounds__(kLatThreads) lattice_energy_kernel(const float *__restrict__ V, int64_t T, int64_t X,
                                                                     int64_t Y, int bnd, const LatGeo g,
                                                                     float *__restrict__ Ec,
                                                                     const __grid_constant__ SpecTables tb)
{
    constexpr int H = (L - 1) / 2;
    constexpr int MAXIT = 4;   // stage-y items per thread (checked by the launcher)
    constexpr bool CT = S_ > 0;
    constexpr LatBlock CB = lat_choose(L, CT ? S_ : 1);
    extern __shared__ __align__(16) float smem[];
    const int tid = threadIdx.x;
    // block -> (lattice plane, x block, y block) in 32 bits (the launcher keeps the grid below 2^31)
    unsigned b = blockIdx.x;
    const int kb = (int)(b % (unsigned)g.nbk);
    b /= (unsigned)g.nbk;
    const int jb = (int)(b % (unsigned)g.nbj);
    const int64_t i = b / (unsigned)g.nbj;
    // lattice coordinates in 32 bits (the launcher checks that every axis fits)
    const int Xi = (int)X, Yi32 = (int)Y, s = CT ? S_ : g.s;
    const int BJ = CT ? CB.BJ : g.BJ, BK = CT ? CB.BK : g.BK;
    const int RXM = CT ? (CB.BJ - 1) * S_ + L : g.RXM, RYM = CT ? (CB.BK - 1) * S_ + L : g.RYM;
    auto coord = [s](int idx, int n) { return min(idx * s, n - 1); };
    const int j0 = jb * BJ, k0 = kb * BK;
    const int nj = min(BJ, (int)g.Xc - j0), nk = min(BK, (int)g.Yc - k0);
    const int64_t tc = coord((int)i, (int)T);
    const int xlo = coord(j0, Xi) - H, ylo = coord(k0, Yi32) - H;
    const int RX = CT ? RXM : coord(j0 + nj - 1, Xi) + H - xlo + 1;
    const int RY = CT ? RYM : coord(k0 + nk - 1, Yi32) + H - ylo + 1;
    const int P = RYM;                                     // row pitch (floats or float2)
    const int PL = RXM * P;                                // plane pitch of the V region / one G1 mu

    float2 *sG1 = reinterpret_cast<float2 *>(smem);                                   // [H+1][RXM][P]
    float *sV = smem + lat_g1_floats(L, RXM, RYM);                                    // [L][RXM][P]
    float2 *sG2 = reinterpret_cast<float2 *>(sV);                                     // [L (nu)][BJ][P], after stage t
    float *sacc = sV + lat_reg_floats(L, BJ, RXM, RYM);                               // [3][BJ * BK * L]
    const int nitems = CT ? BJ * BK * L : nj * nk * L;     // compile-time geometry: every point of the block
    const int accn = BJ * BK * L;
    const int BJP = BJ * P;                                // G2 stride between nu lines

    LatTw<L> tw;
    tw.load(tb);

    // the V region, relative to one sample of it, by asynchronous 4-byte copies.  Regions
    // inside the volume: whole rows (plane p, row q) per warp, lanes along y, the source offset
    // advanced per row; regions at a face: element by element with the boundary extension
    const float ref = V[(tc * X + (xlo + H)) * Y + (ylo + H)];
    {
        const bool inside = tc - H >= 0 && tc + H < T && xlo >= 0 && xlo + RX <= X && ylo >= 0 && ylo + RY <= Y &&
                            (int64_t)L * X * Y < 0x7fffffffLL;
        if (inside) {
            const int warp = tid >> 5, lane = tid & 31, nw = kLatThreads / 32;
            const float *src = V + ((tc - H) * X + xlo) * Y + ylo;
            const int Yi = (int)Y, XYi = (int)(X * Y);
            int q = warp % RX, p = warp / RX;
            for (int row = warp; row < L * RX; row += nw) {
                const int off = p * XYi + q * Yi;
                const unsigned dst = (unsigned)__cvta_generic_to_shared(sV + p * PL + q * P);
                for (int r = lane; r < RY; r += 32)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst + 4u * r), "l"(src + off + r) : "memory");
                q += nw;
                while (q >= RX) {
                    q -= RX;
                    ++p;
                }
            }
        } else {
            int r = tid % RY, q = (tid / RY) % RX, p = tid / (RX * RY);
            const int dr = kLatThreads % RY, dq = (kLatThreads / RY) % RX, dp = kLatThreads / (RX * RY);
            for (int e = tid; e < L * RX * RY; e += kLatThreads) {
                int64_t gt = tc - H + p, gx = xlo + q, gy = ylo + r;
                if ((uint64_t)gt >= (uint64_t)T) gt = ext_index(gt, T, bnd);
                if ((uint64_t)gx >= (uint64_t)X) gx = ext_index(gx, X, bnd);
                if ((uint64_t)gy >= (uint64_t)Y) gy = ext_index(gy, Y, bnd);
                const unsigned dst = (unsigned)__cvta_generic_to_shared(sV + p * PL + q * P + r);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(V + (gt * X + gx) * Y + gy) : "memory");
                r += dr;
                q += dq;
                p += dp;
                if (r >= RY) {
                    r -= RY;
                    ++q;
                }
                if (q >= RX) {
                    q -= RX;
                    ++p;
                }
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncthreads();

    // stage t, every mu at once: G1[mu](x', y') for each column of the region (real input:
    // folded, G1(mu) = A - iB with A = sum_p (a(+p) + a(-p) - 2 a0) cos, B = sum (a(+p) - a(-p)) sin)
    {
        int r = tid % RY, q = tid / RY;
        const int dr = kLatThreads % RY, dq = kLatThreads / RY;
        for (int e = tid; e < RX * RY; e += kLatThreads) {
            float a[L];
            const float *src = sV + q * P + r;
#pragma unroll
            for (int p = 0; p < L; ++p, src += PL) a[p] = *src - ref;
            float U[H + 1], D[H + 1], s0 = a[H];
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                U[k] = a[H + k] + a[H - k];
                D[k] = a[H + k] - a[H - k];
                s0 += U[k];
            }
            float2 *o = sG1 + q * P + r;
            o[0] = make_float2(s0, 0.f);
#pragma unroll
            for (int mu = 1; mu <= H; ++mu) {
                float A = a[H], B = 0.f;
#pragma unroll
                for (int k = 1; k <= H; ++k) {
                    A = fmaf(U[k], tw.c[(mu * k) % L], A);
                    B = fmaf(D[k], tw.s[(mu * k) % L], B);
                }
                o[mu * PL] = make_float2(A, -B);
            }
            r += dr;
            q += dq;
            if (r >= RY) {
                r -= RY;
                ++q;
            }
        }
    }
    __syncthreads();

    // stage-y items of this thread (the same for every mu): item it = nu * npts + point, so
    // the lanes of a warp read neighbouring points of one line (few shared-memory bank
    // conflicts); line offset into sG2 (without the nu part) and the weight row
    const int npts = CT ? BJ * BK : nj * nk, pnk = CT ? BK : nk;
    float acc[MAXIT][3];
    int ioff[MAXIT], inu[MAXIT];
#pragma unroll
    for (int kk = 0; kk < MAXIT; ++kk) {
        acc[kk][0] = acc[kk][1] = acc[kk][2] = 0.f;
        const int it = tid + kk * kLatThreads;
        const int nu = it / npts, pt = it - nu * npts, j = pt / pnk, k = pt - j * pnk;
        inu[kk] = nu;
        ioff[kk] = j * P + (coord(k0 + min(k, nk - 1), Yi32) - H - ylo);
    }

    // stage-x items of this thread (the same for every mu): column (j, r) of the lattice x
    // j; offsets into G1 (first tap) and into G2 (line nu = 0)
    constexpr int MAXX = 2;
    int xin[MAXX], xout[MAXX];
    const int nxit = CT ? BJ * RY : nj * RY;
#pragma unroll
    for (int kk = 0; kk < MAXX; ++kk) {
        const int e = tid + kk * kLatThreads;
        const int j = e / RY, r = e - j * RY;
        xin[kk] = (coord(j0 + min(j, nj - 1), Xi) - H - xlo) * P + r;
        xout[kk] = j * P + r;
    }

#pragma unroll 1
    for (int mu = 0; mu <= H; ++mu) {
        // stage x at the lattice x of this CTA: every nu of a column window at once
        const float2 *g1 = sG1 + mu * PL;
#pragma unroll
        for (int kk = 0; kk < MAXX; ++kk) {
            if (tid + kk * kLatThreads >= nxit) break;
            float2 z[L], out[L];
            const float2 *src = g1 + xin[kk];
#pragma unroll
            for (int q = 0; q < L; ++q, src += P) z[q] = *src;
            folded_dft<L>(z, tw, out);
            float2 *dst = sG2 + xout[kk];
#pragma unroll
            for (int nu = 0; nu < L; ++nu, dst += BJP) *dst = out[nu];
        }
        __syncthreads();
        // stage y: the folded DFT of each (point, nu) line at the lattice y, |F|, weights
        const float mult = mu == 0 ? 1.f : 2.f;
#pragma unroll
        for (int kk = 0; kk < MAXIT; ++kk) {
            if (tid + kk * kLatThreads >= nitems) break;
            const int nu = inu[kk];
            const float2 *line = sG2 + nu * BJP + ioff[kk];
            float2 z[L], F[L];
#pragma unroll
            for (int r = 0; r < L; ++r) z[r] = line[r];
            folded_dft<L>(z, tw, F);
            const int anu = nu >= H ? nu - H : H - nu;
            const float *w0 = tb.w + ((mu * kMaxHalf + anu) * kMaxHalf) * 3;
            float et = 0.f, ex = 0.f, ey = 0.f;
#pragma unroll
            for (int om = 0; om <= H; ++om) {
                float m = lat_sqrt(fmaf(F[H + om].x, F[H + om].x, F[H + om].y * F[H + om].y));
                if (om) m += lat_sqrt(fmaf(F[H - om].x, F[H - om].x, F[H - om].y * F[H - om].y));
                const float *w = w0 + om * 3;
                et = fmaf(w[0], m, et);
                ex = fmaf(w[1], m, ex);
                ey = fmaf(w[2], m, ey);
            }
            acc[kk][0] = fmaf(mult, et, acc[kk][0]);
            acc[kk][1] = fmaf(mult, ex, acc[kk][1]);
            acc[kk][2] = fmaf(mult, ey, acc[kk][2]);
        }
        __syncthreads();
    }

    // E_m of each point: the sum over nu, times L^-3 (DFT) and (L^3 - 1)^-1 (non-DC mean)
#pragma unroll
    for (int kk = 0; kk < MAXIT; ++kk) {
        const int it = tid + kk * kLatThreads;
        if (it >= nitems) break;
        const int nu = inu[kk], pt = it - nu * npts, j = pt / pnk, k = pt - j * pnk;
        const int slot = (j * BK + k) * L + nu;
        sacc[slot] = acc[kk][0];
        sacc[accn + slot] = acc[kk][1];
        sacc[2 * accn + slot] = acc[kk][2];
    }
    __syncthreads();
    const float scale = tb.escale * 0.5f;   // escale holds the half-spectrum factor 2, applied above
    const int64_t Nc = g.Tc * g.Xc * g.Yc;
    for (int e = tid; e < 3 * nj * nk; e += kLatThreads) {
        const int m = e / (nj * nk), pt = e - m * (nj * nk), j = pt / nk, k = pt - j * nk;
        const float *a = sacc + m * accn + (j * BK + k) * L;
        float sum = 0.f;
#pragma unroll
        for (int nu = 0; nu < L; ++nu) sum += a[nu];
        Ec[m * Nc + (i * g.Xc + (j0 + j)) * g.Yc + (k0 + k)] = sum * scale;
    }
}

// Trilinear interpolation of the lattice energies back to every voxel.  Every CTA first
// tabulates, once, the lattice segment and the fraction of the way of every t, x and y (the
// same for every row); it then walks rows (t, x) on a 2-D grid (no division per row): the four
// lattice rows around a row are blended along t and x into shared memory, and every voxel y
// blends its two neighbouring lattice values along y with a coalesced store.
__device__ __forceinline__ float2 lattice_segment(int v, int n, int nc, int s)
{
    if (nc <= 1) return make_float2(__int_as_float(0), 0.f);
    const int k = min(v / s, nc - 2);
    const int lo = k * s, hi = min((k + 1) * s, n - 1);
    return make_float2(__int_as_float(k), (float)(v - lo) / (float)(hi - lo));
}

__global__ void __launch_bounds__(256) interp_kernel(const float *__restrict__ Ec, int T, int X, int Y, int s, int Tc,
                                                     int Xc, int Yc, float *__restrict__ E)
{
    extern __shared__ float smem_i[];
    float *srow = smem_i;                                                     // [3][Yc]
    float2 *ytab = reinterpret_cast<float2 *>(smem_i + ((3 * Yc + 1) & ~1));  // [Y]
    float2 *ttab = ytab + Y;                                                  // [T]
    float2 *xtab = ttab + T;                                                  // [X]
    const int64_t N = (int64_t)T * X * Y, Nc = (int64_t)Tc * Xc * Yc;
    for (int v = threadIdx.x; v < Y; v += blockDim.x) ytab[v] = lattice_segment(v, Y, Yc, s);
    for (int v = threadIdx.x; v < T; v += blockDim.x) ttab[v] = lattice_segment(v, T, Tc, s);
    for (int v = threadIdx.x; v < X; v += blockDim.x) xtab[v] = lattice_segment(v, X, Xc, s);
    const int dt = Tc > 1 ? 1 : 0, dx = Xc > 1 ? 1 : 0, dk = Yc > 1 ? 1 : 0;
    for (int t = blockIdx.y; t < T; t += gridDim.y) {
        for (int x = blockIdx.x; x < X; x += gridDim.x) {
            __syncthreads();                      // tables ready; the previous row's blends consumed
            const float2 tt = ttab[t], xx = xtab[x];
            const int it = __float_as_int(tt.x), ix = __float_as_int(xx.x);
            const float ft = tt.y, fx = xx.y;
            const float w00 = (1.f - ft) * (1.f - fx), w01 = (1.f - ft) * fx, w10 = ft * (1.f - fx), w11 = ft * fx;
            const float *c00 = Ec + ((int64_t)it * Xc + ix) * Yc;
            const float *c01 = c00 + (int64_t)dx * Yc, *c10 = c00 + (int64_t)dt * Xc * Yc;
            const float *c11 = c10 + (int64_t)dx * Yc;
            for (int e = threadIdx.x; e < 3 * Yc; e += blockDim.x) {
                const int m = e >= Yc ? (e >= 2 * Yc ? 2 : 1) : 0;
                const int64_t o = m * Nc + (e - m * Yc);
                srow[e] = w00 * c00[o] + w01 * c01[o] + w10 * c10[o] + w11 * c11[o];
            }
            __syncthreads();
            float *e0 = E + ((int64_t)t * X + x) * Y, *e1 = e0 + N, *e2 = e1 + N;
            for (int y = threadIdx.x; y < Y; y += blockDim.x) {
                const float2 tf = ytab[y];
                const int ky = __float_as_int(tf.x);
                const float fy = tf.y;
                const float a0 = srow[ky], a1 = srow[Yc + ky], a2 = srow[2 * Yc + ky];
                e0[y] = fmaf(fy, srow[ky + dk] - a0, a0);
                e1[y] = fmaf(fy, srow[Yc + ky + dk] - a1, a1);
                e2[y] = fmaf(fy, srow[2 * Yc + ky + dk] - a2, a2);
            }
        }
    }
}

template <int L, int S = 0>
cudaError_t launch_lattice_L(const float *V, sal_dims d, int bnd, const LatGeo &g, float *Ec, cudaStream_t st)
{
    SpecTables tb;
    make_tables(L, &tb);
    const size_t smem = lat_smem_bytes(L, g.BJ, g.BK, g.RXM, g.RYM);
    if (g.BJ * g.BK * L > 4 * kLatThreads || g.BJ * g.RYM > 2 * kLatThreads)
        return cudaErrorInvalidValue;   // the kernel's stage-y and stage-x items per thread
    if (d.T > 0x3fffffffLL || d.X > 0x3fffffffLL || d.Y > 0x3fffffffLL) return cudaErrorInvalidValue;   // 32-bit coordinates
    cudaError_t e = set_smem(lattice_energy_kernel<L, S>, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = g.Tc * g.nbj * g.nbk;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    lattice_energy_kernel<L, S><<<(unsigned)blocks, kLatThreads, smem, st>>>(V, d.T, d.X, d.Y, bnd, g, Ec, tb);
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
    const LatBlock lb = lat_choose(L, s);
    g.BJ = lb.BJ;
    g.BK = lb.BK;
    g.RXM = (g.BJ - 1) * s + L;
    g.RYM = (g.BK - 1) * s + L;
    g.nbj = (int)((g.Xc + g.BJ - 1) / g.BJ);
    g.nbk = (int)((g.Yc + g.BK - 1) / g.BK);
    switch (L) {
    case 3: return launch_lattice_L<3>(V, d, bnd, g, Ec, st);
    case 5: return s == 2 ? launch_lattice_L<5, 2>(V, d, bnd, g, Ec, st) : launch_lattice_L<5>(V, d, bnd, g, Ec, st);
    case 7:
        return s == 2   ? launch_lattice_L<7, 2>(V, d, bnd, g, Ec, st)
               : s == 3 ? launch_lattice_L<7, 3>(V, d, bnd, g, Ec, st)
                        : launch_lattice_L<7>(V, d, bnd, g, Ec, st);
    case 9:
        return s == 2   ? launch_lattice_L<9, 2>(V, d, bnd, g, Ec, st)
               : s == 3 ? launch_lattice_L<9, 3>(V, d, bnd, g, Ec, st)
               : s == 4 ? launch_lattice_L<9, 4>(V, d, bnd, g, Ec, st)
                        : launch_lattice_L<9>(V, d, bnd, g, Ec, st);
    case 11: return launch_lattice_L<11>(V, d, bnd, g, Ec, st);
    case 13: return launch_lattice_L<13>(V, d, bnd, g, Ec, st);
    case 15: return launch_lattice_L<15>(V, d, bnd, g, Ec, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_interp_lattice(const float *Ec, sal_dims d, int s, float *E, cudaStream_t st)
{
    if (d.T > 0x7fffffffLL || d.X > 0x7fffffffLL || d.Y > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int Yc = (int)lattice_size(d.Y, s);
    const size_t smem = ((3 * (size_t)Yc + 1) & ~(size_t)1) * sizeof(float) +
                        (size_t)(d.Y + d.T + d.X) * sizeof(float2);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(interp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int threads = d.Y >= 256 ? 256 : (int)((d.Y + 31) / 32 * 32);
    const unsigned gx = (unsigned)(d.X < 64 ? d.X : 64), gy = (unsigned)(d.T < 40 ? d.T : 40);
    interp_kernel<<<dim3(gx, gy), threads, smem, st>>>(Ec, (int)d.T, (int)d.X, (int)d.Y, s, (int)lattice_size(d.T, s),
                                                      (int)lattice_size(d.X, s), Yc, E);
    return cudaGetLastError();
}

}  // namespace sal
