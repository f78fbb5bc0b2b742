// Fused local spectra -> spectral energies, FP32 on the CUDA cores.
//
// For every voxel v the method takes the L^3 cube centred on v, its DFT (Sec. 2, the
// transform printed below Eq. 2), weights |F| by the plane projections of Eq. 1-4 and
// averages over the non-DC points (third step of Sec. 2), giving E_t, E_x, E_y.
//
// The DFT is separable, so a CTA computes it for a tile of BT x BX x BY output voxels
// in three mode products that share work between neighbouring cubes:
//   stage t: every (t, x', y') column of the halo tile -> G1[mu], mu = 0..h (real input,
//            so the half spectrum mu >= 0 suffices: |F(-k)| = |F(k)|);
//   stage x: G1[mu](x-h..x+h) -> G2[mu, nu], nu = -h..h, for every (t, x, y');
//   stage y: G2[mu, nu](y-h..y+h) -> F[mu, nu, omega] for each output voxel, held in
//            registers only, then |F|, the projection weights and the mean.
// Each length-L transform folds the sample pairs +-k (U_k = z_k + z_-k, D_k = z_k - z_-k)
// so that one pass gives both +omega and -omega, and subtracts the centre sample from the
// pairs for the non-zero frequencies (which changes nothing there since the twiddles of a
// non-zero frequency sum to zero) so that a constant cube has an exactly zero spectrum.
// Indices are taken relative to the cube centre; that multiplies each coefficient by a
// unit phase, which |F| does not see.
#pragma once
#include "sal_internal.cuh"

namespace sal {
namespace energy_detail {

template <int L_, int BT_, int BX_>
struct EGeo {
    static constexpr int L = L_, H = (L_ - 1) / 2, BT = BT_, BX = BX_;
    static constexpr int BY = 32, R = 4, SY = BY / R;
    static constexpr int ROWS = BT * BX;               // output rows (t, x) per tile
    static constexpr int NT = ROWS * SY;                // threads
    static constexpr int HX = BX + 2 * H;               // halo rows along x
    static constexpr int PY = BY + 2 * H;               // halo columns along y
    // complex pitch of a G2 line: keeps 16-byte alignment and makes the stride between
    // output rows an odd multiple of 16 bytes (conflict-free 128-bit shared loads)
    static constexpr int PY2 = ((PY / 2) % 2 == 0) ? PY + 2 : PY;
    static constexpr int NV = (BT + 2 * H) * HX * PY;   // floats of the V halo tile
    static constexpr int NG1 = (BT * HX * L * PY + 3) / 4 * 4;
    static constexpr int NG2 = ROWS * L * PY2;          // float2 of one mu-slice of G2
    static constexpr int NALIAS = (NV * 4 > NG2 * 8) ? NV : NG2 * 2;
    static constexpr size_t SMEM = sizeof(float) * (size_t)(NG1 + NALIAS);
};

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// Magnitudes of one complex line of the y transform, window centred at Z[C]:
// m[0] = |F(0)|, m[w] = |F(w)| + |F(-w)| for w = 1..H.
template <int L, int C, int NZ>
__device__ __forceinline__ void line_mags(const float2 (&Z)[NZ], const SpecTables &tb, float (&m)[(L + 1) / 2])
{
    constexpr int H = (L - 1) / 2;
    const float2 z0 = Z[C];
    float2 U[H + 1], D[H + 1];
    float2 s = z0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        float2 p = f2add(Z[C + k], Z[C - k]);
        s = f2add(s, p);
        U[k] = make_float2(fmaf(-2.f, z0.x, p.x), fmaf(-2.f, z0.y, p.y));
        D[k] = f2sub(Z[C + k], Z[C - k]);
    }
    m[0] = sqrtf(fmaf(s.x, s.x, s.y * s.y));
#pragma unroll
    for (int w = 1; w <= H; ++w) {
        float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const float c = tb.cs[(w * k) % L], sn = tb.sn[(w * k) % L];
            A.x = fmaf(U[k].x, c, A.x);
            A.y = fmaf(U[k].y, c, A.y);
            B.x = fmaf(D[k].x, sn, B.x);
            B.y = fmaf(D[k].y, sn, B.y);
        }
        const float pr = A.x + B.y, pi = A.y - B.x;   // F(+w) = A - iB
        const float qr = A.x - B.y, qi = A.y + B.x;   // F(-w) = A + iB
        m[w] = sqrtf(fmaf(pr, pr, pi * pi)) + sqrtf(fmaf(qr, qr, qi * qi));
    }
}

// Real line (the mu = 0, nu = 0 line): m[w] = |F(w)| for w = 1..H (the -w point is the
// conjugate mirror, counted by the half-spectrum factor).
template <int L, int C, int NZ>
__device__ __forceinline__ void line_mags_real(const float2 (&Z)[NZ], const SpecTables &tb, float (&m)[(L + 1) / 2])
{
    constexpr int H = (L - 1) / 2;
    const float z0 = Z[C].x;
    float U[H + 1], D[H + 1];
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        U[k] = fmaf(-2.f, z0, Z[C + k].x + Z[C - k].x);
        D[k] = Z[C + k].x - Z[C - k].x;
    }
    m[0] = 0.f;
#pragma unroll
    for (int w = 1; w <= H; ++w) {
        float A = 0.f, B = 0.f;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            A = fmaf(U[k], tb.cs[(w * k) % L], A);
            B = fmaf(D[k], tb.sn[(w * k) % L], B);
        }
        m[w] = sqrtf(fmaf(A, A, B * B));
    }
}

template <class G>
__device__ __forceinline__ void load_line(const float2 *sG2, int row, int nu, int j, float2 (&Z)[G::R + 2 * G::H])
{
    static_assert((G::R + 2 * G::H) % 2 == 0, "even window");
    const float4 *p = reinterpret_cast<const float4 *>(sG2 + ((row * G::L + nu + G::H) * G::PY2 + G::R * j));
#pragma unroll
    for (int k = 0; k < (G::R + 2 * G::H) / 2; ++k) {
        const float4 v = p[k];
        Z[2 * k] = make_float2(v.x, v.y);
        Z[2 * k + 1] = make_float2(v.z, v.w);
    }
}

template <class G, int MU, int NU>
__device__ __forceinline__ void accum(const float (&m)[G::H + 1], const SpecTables &tb, float &et, float &ex, float &ey,
                                      int wfirst)
{
#pragma unroll
    for (int w = 0; w <= G::H; ++w) {
        if (w < wfirst) continue;
        const float *wt = &tb.w[((MU * kMaxHalf + NU) * kMaxHalf + w) * 3];
        et = fmaf(wt[0], m[w], et);
        ex = fmaf(wt[1], m[w], ex);
        ey = fmaf(wt[2], m[w], ey);
    }
}

// y stage for one mu: every thread owns R consecutive outputs of one (t, x) row.
template <class G, int MU>
__device__ __forceinline__ void y_stage(const float2 *sG2, int row, int j, const SpecTables &tb,
                                        float (&et)[G::R], float (&ex)[G::R], float (&ey)[G::R])
{
    constexpr int H = G::H, R = G::R, NZ = R + 2 * H;
    if (MU == 0) {
        {   // nu = 0: real line, omega > 0 only
            float2 Z[NZ];
            load_line<G>(sG2, row, 0, j, Z);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float m[H + 1];
                switch (r) {  // compile-time centre
                    case 0: line_mags_real<G::L, H + 0>(Z, tb, m); break;
                    case 1: line_mags_real<G::L, H + 1>(Z, tb, m); break;
                    case 2: line_mags_real<G::L, H + 2>(Z, tb, m); break;
                    default: line_mags_real<G::L, H + 3>(Z, tb, m); break;
                }
                accum<G, 0, 0>(m, tb, et[r], ex[r], ey[r], 1);
            }
        }
#pragma unroll
        for (int nu = 1; nu <= H; ++nu) {   // nu > 0: all omega; the nu < 0 lines are conjugate mirrors
            float2 Z[NZ];
            load_line<G>(sG2, row, nu, j, Z);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float m[H + 1];
                switch (r) {
                    case 0: line_mags<G::L, H + 0>(Z, tb, m); break;
                    case 1: line_mags<G::L, H + 1>(Z, tb, m); break;
                    case 2: line_mags<G::L, H + 2>(Z, tb, m); break;
                    default: line_mags<G::L, H + 3>(Z, tb, m); break;
                }
#pragma unroll
                for (int w = 0; w <= H; ++w) {
                    const float *wt = &tb.w[((0 * kMaxHalf + nu) * kMaxHalf + w) * 3];
                    et[r] = fmaf(wt[0], m[w], et[r]);
                    ex[r] = fmaf(wt[1], m[w], ex[r]);
                    ey[r] = fmaf(wt[2], m[w], ey[r]);
                }
            }
        }
    } else {
        {   // nu = 0
            float2 Z[NZ];
            load_line<G>(sG2, row, 0, j, Z);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float m[H + 1];
                switch (r) {
                    case 0: line_mags<G::L, H + 0>(Z, tb, m); break;
                    case 1: line_mags<G::L, H + 1>(Z, tb, m); break;
                    case 2: line_mags<G::L, H + 2>(Z, tb, m); break;
                    default: line_mags<G::L, H + 3>(Z, tb, m); break;
                }
                accum<G, MU, 0>(m, tb, et[r], ex[r], ey[r], 0);
            }
        }
#pragma unroll
        for (int nu = 1; nu <= H; ++nu) {   // the +nu and -nu lines share their weights
            float2 Zp[NZ], Zm[NZ];
            load_line<G>(sG2, row, nu, j, Zp);
            load_line<G>(sG2, row, -nu, j, Zm);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float mp[H + 1], mm[H + 1];
                switch (r) {
                    case 0: line_mags<G::L, H + 0>(Zp, tb, mp); line_mags<G::L, H + 0>(Zm, tb, mm); break;
                    case 1: line_mags<G::L, H + 1>(Zp, tb, mp); line_mags<G::L, H + 1>(Zm, tb, mm); break;
                    case 2: line_mags<G::L, H + 2>(Zp, tb, mp); line_mags<G::L, H + 2>(Zm, tb, mm); break;
                    default: line_mags<G::L, H + 3>(Zp, tb, mp); line_mags<G::L, H + 3>(Zm, tb, mm); break;
                }
#pragma unroll
                for (int w = 0; w <= H; ++w) {
                    const float s = mp[w] + mm[w];
                    const float *wt = &tb.w[((MU * kMaxHalf + nu) * kMaxHalf + w) * 3];
                    et[r] = fmaf(wt[0], s, et[r]);
                    ex[r] = fmaf(wt[1], s, ex[r]);
                    ey[r] = fmaf(wt[2], s, ey[r]);
                }
            }
        }
    }
}

// x stage for one mu: G1[mu](x-h..x+h, y') -> G2[mu, nu](x, y') for the BT x BX x PY items.
template <class G, int MU>
__device__ __forceinline__ void x_stage(const float *sG1, float2 *sG2, const SpecTables &tb)
{
    constexpr int L = G::L, H = G::H, PY = G::PY, NITEM = G::ROWS * PY;
    for (int i = threadIdx.x; i < NITEM; i += G::NT) {
        const int row = i / PY, yy = i - row * PY;
        const int t = row / G::BX, x = row - t * G::BX;
        const float *g = sG1 + ((t * G::HX + x) * L) * PY + yy;   // column x' = x + k, k = 0..L-1
        float2 *o = sG2 + (row * L + H) * G::PY2 + yy;            // slot of nu = 0
        if (MU == 0) {
            float z[L];
#pragma unroll
            for (int k = 0; k < L; ++k) z[k] = g[k * L * PY];
            const float z0 = z[H];
            float s = z0, U[H + 1], D[H + 1];
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const float p = z[H + k] + z[H - k];
                s += p;
                U[k] = fmaf(-2.f, z0, p);
                D[k] = z[H + k] - z[H - k];
            }
            o[0] = make_float2(s, 0.f);
#pragma unroll
            for (int nu = 1; nu <= H; ++nu) {
                float A = 0.f, B = 0.f;
#pragma unroll
                for (int k = 1; k <= H; ++k) {
                    A = fmaf(U[k], tb.cs[(nu * k) % L], A);
                    B = fmaf(D[k], tb.sn[(nu * k) % L], B);
                }
                o[nu * G::PY2] = make_float2(A, -B);
            }
        } else {
            float2 z[L];
#pragma unroll
            for (int k = 0; k < L; ++k)
                z[k] = make_float2(g[k * L * PY + (2 * MU - 1) * PY], g[k * L * PY + (2 * MU) * PY]);
            const float2 z0 = z[H];
            float2 s = z0, U[H + 1], D[H + 1];
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const float2 p = f2add(z[H + k], z[H - k]);
                s = f2add(s, p);
                U[k] = make_float2(fmaf(-2.f, z0.x, p.x), fmaf(-2.f, z0.y, p.y));
                D[k] = f2sub(z[H + k], z[H - k]);
            }
            o[0] = s;
#pragma unroll
            for (int nu = 1; nu <= H; ++nu) {
                float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 1; k <= H; ++k) {
                    const float c = tb.cs[(nu * k) % L], sn = tb.sn[(nu * k) % L];
                    A.x = fmaf(U[k].x, c, A.x);
                    A.y = fmaf(U[k].y, c, A.y);
                    B.x = fmaf(D[k].x, sn, B.x);
                    B.y = fmaf(D[k].y, sn, B.y);
                }
                o[nu * G::PY2] = make_float2(A.x + B.y, A.y - B.x);    // G2(+nu) = A - iB
                o[-nu * G::PY2] = make_float2(A.x - B.y, A.y + B.x);   // G2(-nu) = A + iB
            }
        }
    }
}

template <class G, int MU>
struct MuLoop {
    __device__ __forceinline__ static void run(const float *sG1, float2 *sG2, int row, int j, const SpecTables &tb,
                                               float (&et)[G::R], float (&ex)[G::R], float (&ey)[G::R])
    {
        x_stage<G, MU>(sG1, sG2, tb);
        __syncthreads();
        y_stage<G, MU>(sG2, row, j, tb, et, ex, ey);
        __syncthreads();
        MuLoop<G, MU + 1>::run(sG1, sG2, row, j, tb, et, ex, ey);
    }
};
template <class G>
struct MuLoop<G, G::H + 1> {
    __device__ __forceinline__ static void run(const float *, float2 *, int, int, const SpecTables &, float (&)[G::R],
                                               float (&)[G::R], float (&)[G::R]) {}
};

template <class G>
__global__ void __launch_bounds__(G::NT) energy_fp32_kernel(const float *__restrict__ V, int64_t T, int64_t X,
                                                            int64_t Y, int bnd, int tiles_x, int tiles_y,
                                                            float *__restrict__ E,
                                                            const __grid_constant__ SpecTables tb)
{
    static_assert(G::R == 4, "y_stage unrolls four outputs per thread");
    constexpr int L = G::L, H = G::H, PY = G::PY;
    extern __shared__ __align__(16) float smem[];
    float *sG1 = smem;
    float2 *sG2 = reinterpret_cast<float2 *>(smem + G::NG1);
    float *sV = smem + G::NG1;   // aliases sG2: dead once stage t is done

    const int64_t tile = blockIdx.x;
    const int ty = (int)(tile % tiles_y);
    const int tx = (int)((tile / tiles_y) % tiles_x);
    const int64_t tt = tile / ((int64_t)tiles_y * tiles_x);
    const int64_t t0 = tt * G::BT, x0 = (int64_t)tx * G::BX, y0 = (int64_t)ty * G::BY;

    // halo tile of V, boundary-extended (every address maps inside the volume)
    for (int i = threadIdx.x; i < G::NV; i += G::NT) {
        const int r = i / PY, yy = i - r * PY;
        const int a = r / G::HX, xx = r - a * G::HX;
        const int64_t gt = ext_index(t0 - H + a, T, bnd);
        const int64_t gx = ext_index(x0 - H + xx, X, bnd);
        const int64_t gy = ext_index(y0 - H + yy, Y, bnd);
        sV[i] = __ldg(V + (gt * X + gx) * Y + gy);
    }
    __syncthreads();

    // stage t: (t, x', y') -> G1 components [Re G1(0), Re G1(1), Im G1(1), ...]
    for (int i = threadIdx.x; i < G::BT * G::HX * PY; i += G::NT) {
        const int r = i / PY, yy = i - r * PY;
        const int t = r / G::HX, xx = r - t * G::HX;
        float a[L];
#pragma unroll
        for (int k = 0; k < L; ++k) a[k] = sV[((t + k) * G::HX + xx) * PY + yy];
        const float a0 = a[H];
        float s = a0, U[H + 1], D[H + 1];
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const float p = a[H + k] + a[H - k];
            s += p;
            U[k] = fmaf(-2.f, a0, p);
            D[k] = a[H + k] - a[H - k];
        }
        float *o = sG1 + ((t * G::HX + xx) * L) * PY + yy;
        o[0] = s;
#pragma unroll
        for (int mu = 1; mu <= H; ++mu) {
            float A = 0.f, B = 0.f;
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                A = fmaf(U[k], tb.cs[(mu * k) % L], A);
                B = fmaf(D[k], tb.sn[(mu * k) % L], B);
            }
            o[(2 * mu - 1) * PY] = A;     // G1(mu) = A - iB
            o[(2 * mu) * PY] = -B;
        }
    }
    __syncthreads();

    const int row = threadIdx.x % G::ROWS, j = threadIdx.x / G::ROWS;
    float et[G::R], ex[G::R], ey[G::R];
#pragma unroll
    for (int r = 0; r < G::R; ++r) et[r] = ex[r] = ey[r] = 0.f;
    MuLoop<G, 0>::run(sG1, sG2, row, j, tb, et, ex, ey);

    const int t = row / G::BX, x = row - t * G::BX;
    const int64_t gt = t0 + t, gx = x0 + x, gy = y0 + G::R * j;
    if (gt >= T || gx >= X) return;
    const int64_t N = T * X * Y;
    float *e0 = E + (gt * X + gx) * Y + gy;
    if (gy + G::R <= Y && (reinterpret_cast<uintptr_t>(e0) & 15) == 0 && (Y & 3) == 0) {
        *reinterpret_cast<float4 *>(e0) =
            make_float4(et[0] * tb.escale, et[1] * tb.escale, et[2] * tb.escale, et[3] * tb.escale);
        *reinterpret_cast<float4 *>(e0 + N) =
            make_float4(ex[0] * tb.escale, ex[1] * tb.escale, ex[2] * tb.escale, ex[3] * tb.escale);
        *reinterpret_cast<float4 *>(e0 + 2 * N) =
            make_float4(ey[0] * tb.escale, ey[1] * tb.escale, ey[2] * tb.escale, ey[3] * tb.escale);
    } else {
#pragma unroll
        for (int r = 0; r < G::R; ++r) {
            if (gy + r < Y) {
                e0[r] = et[r] * tb.escale;
                e0[r + N] = ex[r] * tb.escale;
                e0[r + 2 * N] = ey[r] * tb.escale;
            }
        }
    }
}

template <class G>
cudaError_t launch_energy_impl(const float *V, sal_dims d, int bnd, float *E, cudaStream_t s)
{
    SpecTables tb;
    make_tables(G::L, &tb);
    const int64_t nt = (d.T + G::BT - 1) / G::BT;
    const int64_t nx = (d.X + G::BX - 1) / G::BX;
    const int64_t ny = (d.Y + G::BY - 1) / G::BY;
    const int64_t tiles = nt * nx * ny;
    if (tiles <= 0) return cudaSuccess;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    auto kern = energy_fp32_kernel<G>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)tiles, G::NT, G::SMEM, s>>>(V, d.T, d.X, d.Y, bnd, (int)nx, (int)ny, E, tb);
    return cudaGetLastError();
}

}  // namespace energy_detail
}  // namespace sal
