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
//
// Complex values travel as packed pairs (re, im) and use the f32x2 add/sub/fma forms of
// sm_100-family GPUs, one instruction per complex add or complex-by-real FMA.  The loops
// over mu and nu stay rolled so the hot loop fits the instruction cache; the loops inside
// one length-L transform, whose indices select twiddles and registers, are unrolled.
#pragma once
#include "sal_internal.cuh"

namespace sal {
namespace energy_detail {

// Tile geometry.  MODE selects how the intermediate spectra are held in shared memory:
//   0: G1 of every mu, and the whole G2 slice of one mu (every nu line);
//   1: G1 of every mu, and G2 only for the lines +|nu|, -|nu| of one (mu, |nu|) batch;
//   2: G1 of one mu at a time (stage t rerun per mu from the staged V halo) and the
//      G2 batch of mode 1.
//   3: as 0, in two regions that swap roles every tile, so that the V halo of the next tile
//      is copied asynchronously (cp.async) while the current tile finishes.
// Modes 1 and 2 trade some recomputation in stages t and x for a smaller footprint, i.e.
// more resident CTAs per SM to hide the latencies of the y stage.
template <int L_, int BT_, int BX_, int MODE_ = 0, int R_ = 4>
struct EGeo {
    static constexpr int L = L_, H = (L_ - 1) / 2, BT = BT_, BX = BX_, MODE = MODE_;
    static constexpr int BY = 32, R = R_, SY = BY / R;     // R consecutive outputs along y per thread
    static_assert(R == 4 || R == 8, "strip of 4 or 8 outputs");
    static constexpr int ROWS = BT * BX;               // output rows (t, x) per tile
    static constexpr int NT = ROWS * SY;                // threads
    static constexpr int HX = BX + 2 * H;               // halo rows along x
    static constexpr int PY = BY + 2 * H;               // halo columns along y
    // complex pitch of a G2 line: keeps 16-byte alignment and makes the stride between
    // output rows an odd multiple of 16 bytes (conflict-free 128-bit shared loads)
    static constexpr int PY2 = ((PY / 2) % 2 == 0) ? PY + 2 : PY;
    static constexpr int NV = (BT + 2 * H) * HX * PY;   // floats of the V halo tile
    static constexpr int NVR = (NV + 3) / 4 * 4;
    static constexpr int NG1 = (BT * HX * L * PY + 3) / 4 * 4;
    static constexpr int NG2 = ROWS * L * PY2;          // float2 of one mu-slice of G2
    static constexpr int NALIAS = (NV * 4 > NG2 * 8) ? NV : NG2 * 2;
    static constexpr int NW = ((H + 1) * (H + 1) * (H + 1) * 3 + 3) / 4 * 4;   // projection weights
    static constexpr int NZ = R + 2 * H;                // window of one thread's R outputs
    // mu > 0 pairs (+nu, -nu) interleaved in G2 and walked as transposed pairs (fewer
    // instructions; above L = 11 the extra live state costs more than it saves)
    static constexpr bool PAIR4 = L_ <= 11;
    // mu = 0: the single lines nu = 1, 2 (3, 4, ...) stored and walked as pairs too (measured:
    // L = 9 -2 %, L = 11 unchanged, L = 5 and 7 slower, their extra live state not paid back)
    static constexpr bool PAIR0 = L_ == 9 || L_ == 11;
    // batched modes: G2 lines [s][row][y'] (s = 0: +|nu|, 1: -|nu|), row stride = PY2 float2
    static constexpr int NG2B = 2 * ROWS * PY2;         // float2
    static constexpr int NG1M = BT * HX * 2 * PY;       // floats: [(t, x')][re, im][y'] of one mu
    // mode 3: each region holds G1, a G2 slice or a V halo tile
    static constexpr int NREG_RAW = NG1 > 2 * NG2 ? (NG1 > NVR ? NG1 : NVR) : (2 * NG2 > NVR ? 2 * NG2 : NVR);
    static constexpr int NREG = (NREG_RAW + 3) / 4 * 4;
    // mode 4: G2 slices in batches of at most NSL line slots per output row (mu = 0 in one
    // batch: its H + 1 lines, or with paired single lines its nu = 0 line and pairs; mu > 0: the
    // nu = 0 line and the pairs 1..P0, then the pairs P0 + 1..H), RSB float2 per output row (an
    // odd multiple of 16 bytes, as PY2 is an odd multiple of 16 bytes)
    static constexpr int NSL = PAIR0 ? 1 + 2 * (H / 2) + (H & 1) : H + 1;
    static constexpr int P0 = (NSL - 1) / 2;
    static constexpr int RSB = NSL * PY2 + ((NSL & 1) ? 0 : 2);
    static constexpr int NG2Q = ROWS * RSB;             // float2
    static constexpr int NALIASQ = (NV * 4 > NG2Q * 8) ? NV : NG2Q * 2;
    static constexpr size_t SMEM =
        sizeof(float) * (size_t)(MODE == 0   ? NG1 + NALIAS + NW
                                 : MODE == 1 ? NG1 + (NVR > 2 * NG2B ? NVR : 2 * NG2B) + NW
                                 : MODE == 2 ? NVR + NG1M + 2 * NG2B + NW
                                 : MODE == 4 ? NG1 + NALIASQ + NW
                                             : 2 * NREG + NW);
    static_assert(MODE >= 0 && MODE <= 4, "tile mode");
    static_assert(MODE != 4 || (PAIR4 && (L_ == 7 || L_ == 9) && 2 * (H - P0) <= NSL && RSB % 2 == 0),
                  "mode 4 is laid out for L = 7 and 9");
};

// ---- packed pairs of floats -------------------------------------------------------------
typedef unsigned long long f2x;   // .x in the low word, .y in the high word

__device__ __forceinline__ f2x pk(float x, float y)
{
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ float lo(f2x v)
{
    float x;
    asm("{ .reg .f32 t; mov.b64 {%0, t}, %1; }" : "=f"(x) : "l"(v));
    return x;
}
__device__ __forceinline__ float hi(f2x v)
{
    float y;
    asm("{ .reg .f32 t; mov.b64 {t, %0}, %1; }" : "=f"(y) : "l"(v));
    return y;
}
__device__ __forceinline__ f2x add2(f2x a, f2x b)
{
    f2x r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b)
{
    f2x r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2x fma2(f2x a, f2x b, f2x c)
{
    f2x r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2x mul2(f2x a, f2x b)
{
    f2x r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// |F| of the magnitude stage: the hardware approximate square root (relative error of a
// few ulp, far inside the path's tolerance).
__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Twiddles of one cube size in registers, as broadcast pairs: c2[k] = (cos, cos) and
// s2[k] = (sin, sin) of 2 pi k / L, k = 0..L-1.
template <int L>
struct Tw {
    f2x c2[L], s2[L];
    __device__ __forceinline__ void load(const SpecTables &tb)
    {
#pragma unroll
        for (int k = 0; k < L; ++k) {
            c2[k] = pk(tb.cs[k], tb.cs[k]);
            s2[k] = pk(tb.sn[k], tb.sn[k]);
        }
    }
};

// Magnitudes of one complex line of the y transform, window centred at Z[c]:
// m[0] = |F(0)|, m[w] = |F(w)| + |F(-w)| for w = 1..H.
template <int L, int NZ>
__device__ __forceinline__ void line_mags(const f2x (&Z)[NZ], int c, const Tw<L> &tw, float (&m)[(L + 1) / 2])
{
    constexpr int H = (L - 1) / 2;
    const f2x z0 = Z[c];
    const f2x m2 = pk(-2.f, -2.f);
    f2x U[H + 1], D[H + 1];
    f2x s = z0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        const f2x p = add2(Z[c + k], Z[c - k]);
        s = add2(s, p);
        U[k] = fma2(z0, m2, p);
        D[k] = sub2(Z[c + k], Z[c - k]);
    }
    {
        const float sx = lo(s), sy = hi(s);
        m[0] = sqrt_approx(fmaf(sx, sx, sy * sy));
    }
#pragma unroll
    for (int w = 1; w <= H; ++w) {
        f2x A = mul2(U[1], tw.c2[w % L]);
        f2x B = mul2(D[1], tw.s2[w % L]);
#pragma unroll
        for (int k = 2; k <= H; ++k) {
            A = fma2(U[k], tw.c2[(w * k) % L], A);
            B = fma2(D[k], tw.s2[(w * k) % L], B);
        }
        const float ax = lo(A), ay = hi(A), bx = lo(B), by = hi(B);
        const float pr = ax + by, pi = ay - bx;   // F(+w) = A - iB
        const float qr = ax - by, qi = ay + bx;   // F(-w) = A + iB
        m[w] = sqrt_approx(fmaf(pr, pr, pi * pi)) + sqrt_approx(fmaf(qr, qr, qi * qi));
    }
}

// Real line (the mu = 0, nu = 0 line; the imaginary halves are zero): m[w] = |F(w)| for
// w = 1..H (the -w point is the conjugate mirror, counted by the half-spectrum factor).
template <int L, int NZ>
__device__ __forceinline__ void line_mags_real(const f2x (&Z)[NZ], int c, const Tw<L> &tw, float (&m)[(L + 1) / 2])
{
    constexpr int H = (L - 1) / 2;
    const float z0 = lo(Z[c]);
    float U[H + 1], D[H + 1];
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        U[k] = fmaf(-2.f, z0, lo(Z[c + k]) + lo(Z[c - k]));
        D[k] = lo(Z[c + k]) - lo(Z[c - k]);
    }
    m[0] = 0.f;
#pragma unroll
    for (int w = 1; w <= H; ++w) {
        float A = 0.f, B = 0.f;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            A = fmaf(U[k], lo(tw.c2[(w * k) % L]), A);
            B = fmaf(D[k], lo(tw.s2[(w * k) % L]), B);
        }
        m[w] = sqrt_approx(fmaf(A, A, B * B));
    }
}

// P := P + d * e^{-i 2 pi k / L} for the twiddle index k (packed complex, dsw = (d.im, -d.re)).
template <int L>
__device__ __forceinline__ f2x rot_acc(f2x P, f2x d, f2x dsw, const Tw<L> &tw, int k)
{
    return fma2(dsw, tw.s2[k], fma2(d, tw.c2[k], P));
}

__device__ __forceinline__ f2x swapneg(f2x d) { return pk(hi(d), -lo(d)); }

// Twiddle index of w * j modulo L in 0..L-1 for any sign of j (compile-time when w, j are).
template <int L>
__host__ __device__ constexpr int tw_index(int w, int j)
{
    return ((w * j) % L + L) % L;
}

__device__ __forceinline__ float cabs2(f2x v)
{
    const f2x q = mul2(v, v);
    return lo(q) + hi(q);
}

// Magnitudes of the R consecutive windows of one complex line, window r centred at
// Z[H + r], handed to put(r, w, m) as each is formed, w = 0..H in order for every window:
// m = |F_r(0)| for w = 0, |F_r(w)| + |F_r(-w)| otherwise.  Window 0 by the folded direct
// DFT; the others by a sliding recurrence on Q_r(w) = e^{-i th w r} F_r(w) (|Q_r| = |F_r|):
// Q_{r+1} = Q_r + (Z[r+2h+1] - Z[r]) e^{-i th w (r-h)}, because the twiddles of a whole
// period are equal; Q_0 = F_0 needs no rotation.
template <int L, int NZ>
struct LineWalk {
    static constexpr int H = (L - 1) / 2;
    f2x P[L];   // Q_r(w) at P[H + w], w = -H..H

    // window 0: m[0] = |F_0(0)|, m[w] = |F_0(w)| + |F_0(-w)|
    __device__ __forceinline__ void start(const f2x (&Z)[NZ], const Tw<L> &tw, float (&m)[H + 1])
    {
        const f2x z0 = Z[H];
        const f2x m2 = pk(-2.f, -2.f);
        f2x U[H + 1], D[H + 1];
        f2x s = z0;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const f2x p = add2(Z[H + k], Z[H - k]);
            s = add2(s, p);
            U[k] = fma2(z0, m2, p);
            D[k] = sub2(Z[H + k], Z[H - k]);
        }
        P[H] = s;
        m[0] = sqrt_approx(cabs2(s));
#pragma unroll
        for (int w = 1; w <= H; ++w) {
            f2x A = mul2(U[1], tw.c2[w % L]);
            f2x B = mul2(D[1], tw.s2[w % L]);
#pragma unroll
            for (int k = 2; k <= H; ++k) {
                A = fma2(U[k], tw.c2[(w * k) % L], A);
                B = fma2(D[k], tw.s2[(w * k) % L], B);
            }
            const float ax = lo(A), ay = hi(A), bx = lo(B), by = hi(B);
            const f2x Fp = pk(ax + by, ay - bx);   // F(+w) = A - iB
            const f2x Fm = pk(ax - by, ay + bx);   // F(-w) = A + iB
            m[w] = sqrt_approx(cabs2(Fp)) + sqrt_approx(cabs2(Fm));
            P[H + w] = Fp;
            P[H - w] = Fm;
        }
    }

    // window r + 1 from window r (r a compile-time constant once unrolled)
    __device__ __forceinline__ void step(const f2x (&Z)[NZ], const Tw<L> &tw, int r, float (&m)[H + 1])
    {
        const f2x d = sub2(Z[r + 2 * H + 1], Z[r]);
        const f2x dsw = swapneg(d);
        P[H] = add2(P[H], d);
#pragma unroll
        for (int w = 1; w <= H; ++w) {
            P[H + w] = rot_acc<L>(P[H + w], d, dsw, tw, tw_index<L>(w, r - H));
            P[H - w] = rot_acc<L>(P[H - w], d, dsw, tw, tw_index<L>(-w, r - H));
        }
        m[0] = sqrt_approx(cabs2(P[H]));
#pragma unroll
        for (int w = 1; w <= H; ++w) m[w] = sqrt_approx(cabs2(P[H + w])) + sqrt_approx(cabs2(P[H - w]));
    }
};

// Magnitudes of the R consecutive windows of one complex line, window r centred at
// Z[H + r], handed to put(r, w, m), w = 0..H in order for every window: m = |F_r(0)| for
// w = 0, |F_r(w)| + |F_r(-w)| otherwise.  Window 0 by the folded direct DFT; the others by a
// sliding recurrence on Q_r(w) = e^{-i th w r} F_r(w) (|Q_r| = |F_r|):
// Q_{r+1} = Q_r + (Z[r+2h+1] - Z[r]) e^{-i th w (r-h)}, because the twiddles of a whole
// period are equal; Q_0 = F_0 needs no rotation.
template <int L, int R, int NZ, class Put>
__device__ __forceinline__ void line_mags_strip(const f2x (&Z)[NZ], const Tw<L> &tw, Put &&put)
{
    constexpr int H = (L - 1) / 2;
    LineWalk<L, NZ> lw;
    float m[H + 1];
    lw.start(Z, tw, m);
#pragma unroll
    for (int w = 0; w <= H; ++w) put(0, w, m[w]);
#pragma unroll
    for (int r = 0; r + 1 < R; ++r) {
        lw.step(Z, tw, r, m);
#pragma unroll
        for (int w = 0; w <= H; ++w) put(r + 1, w, m[w]);
    }
}

// Two lines walked window by window together (independent work for the scheduler to
// interleave): put(r, w, ma, mb) with each line's magnitudes as in line_mags_strip.
template <int L, int R, int NZ, class Put>
__device__ __forceinline__ void line_mags_strip2(const f2x (&Za)[NZ], const f2x (&Zb)[NZ], const Tw<L> &tw, Put &&put)
{
    constexpr int H = (L - 1) / 2;
    LineWalk<L, NZ> la, lb;
    float ma[H + 1], mb[H + 1];
    la.start(Za, tw, ma);
    lb.start(Zb, tw, mb);
#pragma unroll
    for (int w = 0; w <= H; ++w) put(0, w, ma[w], mb[w]);
#pragma unroll
    for (int r = 0; r + 1 < R; ++r) {
        la.step(Za, tw, r, ma);
        lb.step(Zb, tw, r, mb);
#pragma unroll
        for (int w = 0; w <= H; ++w) put(r + 1, w, ma[w], mb[w]);
    }
}

// Two lines a, b walked together in transposed pairs: X = (Re a, Re b), Y = (Im a, Im b) of
// every sample and every recurrence state, so that one packed multiply and one packed FMA give
// the squared magnitudes of both lines.  Per line: ma[w] = |Fa(w)| + |Fa(-w)|, ma[0] = |Fa(0)|
// (and mb for line b).
template <int L, int NZ>
struct PairWalk {
    static constexpr int H = (L - 1) / 2;
    f2x X[L], Y[L];   // Q_r(w) of both lines at [H + w], w = -H..H

    __device__ __forceinline__ static void mags(f2x xp, f2x yp, f2x xm, f2x ym, float &ma, float &mb)
    {
        const f2x qp = fma2(yp, yp, mul2(xp, xp)), qm = fma2(ym, ym, mul2(xm, xm));
        ma = sqrt_approx(lo(qp)) + sqrt_approx(lo(qm));
        mb = sqrt_approx(hi(qp)) + sqrt_approx(hi(qm));
    }
    __device__ __forceinline__ static void mag0(f2x x, f2x y, float &ma, float &mb)
    {
        const f2x q = fma2(y, y, mul2(x, x));
        ma = sqrt_approx(lo(q));
        mb = sqrt_approx(hi(q));
    }

    __device__ __forceinline__ void start(const f2x (&ZX)[NZ], const f2x (&ZY)[NZ], const Tw<L> &tw,
                                          float (&ma)[H + 1], float (&mb)[H + 1])
    {
        const f2x m2 = pk(-2.f, -2.f);
        f2x UX[H + 1], UY[H + 1], DX[H + 1], DY[H + 1];
        f2x sx = ZX[H], sy = ZY[H];
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const f2x px = add2(ZX[H + k], ZX[H - k]), py = add2(ZY[H + k], ZY[H - k]);
            sx = add2(sx, px);
            sy = add2(sy, py);
            UX[k] = fma2(ZX[H], m2, px);
            UY[k] = fma2(ZY[H], m2, py);
            DX[k] = sub2(ZX[H + k], ZX[H - k]);
            DY[k] = sub2(ZY[H + k], ZY[H - k]);
        }
        X[H] = sx;
        Y[H] = sy;
        mag0(sx, sy, ma[0], mb[0]);
#pragma unroll
        for (int w = 1; w <= H; ++w) {
            f2x ax = mul2(UX[1], tw.c2[w % L]), ay = mul2(UY[1], tw.c2[w % L]);
            f2x bx = mul2(DX[1], tw.s2[w % L]), by = mul2(DY[1], tw.s2[w % L]);
#pragma unroll
            for (int k = 2; k <= H; ++k) {
                ax = fma2(UX[k], tw.c2[(w * k) % L], ax);
                ay = fma2(UY[k], tw.c2[(w * k) % L], ay);
                bx = fma2(DX[k], tw.s2[(w * k) % L], bx);
                by = fma2(DY[k], tw.s2[(w * k) % L], by);
            }
            X[H + w] = add2(ax, by);   // F(+w) = A - iB
            Y[H + w] = sub2(ay, bx);
            X[H - w] = sub2(ax, by);   // F(-w) = A + iB
            Y[H - w] = add2(ay, bx);
            mags(X[H + w], Y[H + w], X[H - w], Y[H - w], ma[w], mb[w]);
        }
    }

    // window r + 1 from window r (r a compile-time constant once unrolled): each state gains
    // d e^{-i th k} = (dX c + dY s, dY c - dX s)
    __device__ __forceinline__ void step(const f2x (&ZX)[NZ], const f2x (&ZY)[NZ], const Tw<L> &tw, int r,
                                         float (&ma)[H + 1], float (&mb)[H + 1])
    {
        const f2x dx = sub2(ZX[r + 2 * H + 1], ZX[r]), dy = sub2(ZY[r + 2 * H + 1], ZY[r]);
        X[H] = add2(X[H], dx);
        Y[H] = add2(Y[H], dy);
#pragma unroll
        for (int w = -H; w <= H; ++w) {
            if (w == 0) continue;
            const int k = tw_index<L>(w, r - H), kn = (L - k) % L;   // s2[kn] = -s2[k]
            X[H + w] = fma2(dy, tw.s2[k], fma2(dx, tw.c2[k], X[H + w]));
            Y[H + w] = fma2(dx, tw.s2[kn], fma2(dy, tw.c2[k], Y[H + w]));
        }
        mag0(X[H], Y[H], ma[0], mb[0]);
#pragma unroll
        for (int w = 1; w <= H; ++w) mags(X[H + w], Y[H + w], X[H - w], Y[H - w], ma[w], mb[w]);
    }
};

// The same for the real mu = 0, nu = 0 line: put(r, w, |F_r(w)|) for w = 1..H only (the -w
// point is the conjugate mirror, counted by the half-spectrum factor; w = 0 is the DC term).
template <int L, int R, int NZ, class Put>
__device__ __forceinline__ void line_mags_strip_real(const f2x (&Z)[NZ], const Tw<L> &tw, Put &&put)
{
    constexpr int H = (L - 1) / 2;
    const float z0 = lo(Z[H]);
    float U[H + 1], D[H + 1];
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        U[k] = fmaf(-2.f, z0, lo(Z[H + k]) + lo(Z[H - k]));
        D[k] = lo(Z[H + k]) - lo(Z[H - k]);
    }
    f2x P[H + 1];
#pragma unroll
    for (int w = 1; w <= H; ++w) {
        float A = 0.f, B = 0.f;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            A = fmaf(U[k], lo(tw.c2[(w * k) % L]), A);
            B = fmaf(D[k], lo(tw.s2[(w * k) % L]), B);
        }
        const f2x F = pk(A, -B);                 // F(w) = A - iB
        put(0, w, sqrt_approx(fmaf(A, A, B * B)));
        P[w] = F;
    }
#pragma unroll
    for (int r = 0; r + 1 < R; ++r) {
        const f2x d = pk(lo(Z[r + 2 * H + 1]) - lo(Z[r]), 0.f);
        const f2x dsw = swapneg(d);
#pragma unroll
        for (int w = 1; w <= H; ++w) {
            P[w] = rot_acc<L>(P[w], d, dsw, tw, tw_index<L>(w, r - H));
            put(r + 1, w, sqrt_approx(cabs2(P[w])));
        }
    }
}

// The NZ samples of one G2 line behind this thread's R outputs (128-bit shared loads).
template <class G>
__device__ __forceinline__ void load_line(const float2 *line, int j, f2x (&Z)[G::NZ])
{
    static_assert(G::NZ % 2 == 0, "even window");
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(line + G::R * j);
#pragma unroll
    for (int k = 0; k < G::NZ / 2; ++k) {
        const ulonglong2 v = p[k];
        Z[2 * k] = v.x;
        Z[2 * k + 1] = v.y;
    }
}

// Projection weights of the (mu, |nu|) group for omega = 0..H, from the shared copy
// sW[((mu * (H+1) + nu) * (H+1) + omega) * 3 + m].
template <class G>
__device__ __forceinline__ void load_w(const float *sW, int mu, int nu, float (&w)[G::H + 1][3])
{
    const float *src = sW + ((mu * (G::H + 1) + nu) * (G::H + 1)) * 3;
#pragma unroll
    for (int om = 0; om <= G::H; ++om) {
        w[om][0] = src[om * 3];
        w[om][1] = src[om * 3 + 1];
        w[om][2] = src[om * 3 + 2];
    }
}

// Copies the weights of this cube size from the parameter bank into sW.
template <class G>
__device__ __forceinline__ void fill_w(float *sW, const SpecTables &tb)
{
    constexpr int HP = G::H + 1;
    for (int e = threadIdx.x; e < HP * HP * HP * 3; e += G::NT) {
        const int m = e % 3, om = (e / 3) % HP, nu = (e / (3 * HP)) % HP, mu = e / (3 * HP * HP);
        sW[e] = tb.w[((mu * kMaxHalf + nu) * kMaxHalf + om) * 3 + m];
    }
}

// One magnitude (or folded pair of magnitudes) into an output's three energies.
__device__ __forceinline__ void wsum(const float (&w)[3], float m, float &et, float &ex, float &ey)
{
    et = fmaf(w[0], m, et);
    ex = fmaf(w[1], m, ex);
    ey = fmaf(w[2], m, ey);
}

// One complex line (weights of group (mu, nu)) for the thread's R outputs.
template <class G>
__device__ __forceinline__ void y_single(const float2 *line, int j, int mu, int nu, const float *sW,
                                         const Tw<G::L> &tw, float (&et)[G::R], float (&ex)[G::R], float (&ey)[G::R])
{
    f2x Z[G::NZ];
    load_line<G>(line, j, Z);
    float w[G::H + 1][3];
    load_w<G>(sW, mu, nu, w);
    line_mags_strip<G::L, G::R>(Z, tw, [&](int r, int om, float m) { wsum(w[om], m, et[r], ex[r], ey[r]); });
}

// The +nu and -nu lines of one mu > 0, which share their weights.
template <class G>
__device__ __forceinline__ void y_pair(const float2 *lp, const float2 *lm, int j, int mu, int nu, const float *sW,
                                       const Tw<G::L> &tw, float (&et)[G::R], float (&ex)[G::R], float (&ey)[G::R])
{
    float w[G::H + 1][3];
    load_w<G>(sW, mu, nu, w);
    f2x Zp[G::NZ], Zm[G::NZ];
    load_line<G>(lp, j, Zp);
    load_line<G>(lm, j, Zm);
    line_mags_strip2<G::L, G::R>(Zp, Zm, tw, [&](int r, int om, float mp, float mm) {
        wsum(w[om], mp + mm, et[r], ex[r], ey[r]);   // |F(+nu)| + |F(-nu)| share the weights
    });
}

// The +nu and -nu lines of one mu > 0 as stage x interleaves them (a float4 per column:
// Re +nu, Re -nu, Im +nu, Im -nu), which share their weights.
template <class G>
__device__ __forceinline__ void y_pair4(const float4 *line, int j, int mu, int nu, const float *sW,
                                        const Tw<G::L> &tw, float (&et)[G::R], float (&ex)[G::R], float (&ey)[G::R])
{
    float w[G::H + 1][3];
    load_w<G>(sW, mu, nu, w);
    f2x ZX[G::NZ], ZY[G::NZ];
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(line + G::R * j);
#pragma unroll
    for (int n = 0; n < G::NZ; ++n) {
        const ulonglong2 v = p[n];
        ZX[n] = v.x;
        ZY[n] = v.y;
    }
    PairWalk<G::L, G::NZ> pw;
    float ma[G::H + 1], mb[G::H + 1];   // |F(+nu)| and |F(-nu)| terms, summed in that order
    pw.start(ZX, ZY, tw, ma, mb);
#pragma unroll
    for (int om = 0; om <= G::H; ++om) wsum(w[om], ma[om] + mb[om], et[0], ex[0], ey[0]);
#pragma unroll
    for (int r = 0; r + 1 < G::R; ++r) {
        pw.step(ZX, ZY, tw, r, ma, mb);
#pragma unroll
        for (int om = 0; om <= G::H; ++om) wsum(w[om], ma[om] + mb[om], et[r + 1], ex[r + 1], ey[r + 1]);
    }
}

// Two single lines (mu, nua) and (mu, nub) stored interleaved like a pair (Re a, Re b, Im a,
// Im b per column), each with its own weights (line a's terms first in every output).
template <class G>
__device__ __forceinline__ void y_single_pair4(const float4 *line, int j, int mu, int nua, int nub, const float *sW,
                                               const Tw<G::L> &tw, float (&et)[G::R], float (&ex)[G::R],
                                               float (&ey)[G::R])
{
    float wa[G::H + 1][3], wb[G::H + 1][3];
    load_w<G>(sW, mu, nua, wa);
    load_w<G>(sW, mu, nub, wb);
    f2x ZX[G::NZ], ZY[G::NZ];
    const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(line + G::R * j);
#pragma unroll
    for (int n = 0; n < G::NZ; ++n) {
        const ulonglong2 v = p[n];
        ZX[n] = v.x;
        ZY[n] = v.y;
    }
    PairWalk<G::L, G::NZ> pw;
    float ma[G::H + 1], mb[G::H + 1];
    pw.start(ZX, ZY, tw, ma, mb);
#pragma unroll
    for (int om = 0; om <= G::H; ++om) wsum(wa[om], ma[om], et[0], ex[0], ey[0]);
#pragma unroll
    for (int om = 0; om <= G::H; ++om) wsum(wb[om], mb[om], et[0], ex[0], ey[0]);
#pragma unroll
    for (int r = 0; r + 1 < G::R; ++r) {
        pw.step(ZX, ZY, tw, r, ma, mb);
#pragma unroll
        for (int om = 0; om <= G::H; ++om) wsum(wa[om], ma[om], et[r + 1], ex[r + 1], ey[r + 1]);
#pragma unroll
        for (int om = 0; om <= G::H; ++om) wsum(wb[om], mb[om], et[r + 1], ex[r + 1], ey[r + 1]);
    }
}

// The real mu = 0, nu = 0 line, omega > 0 only.
template <class G>
__device__ __forceinline__ void y_real(const float2 *line, int j, const float *sW, const Tw<G::L> &tw,
                                       float (&et)[G::R], float (&ex)[G::R], float (&ey)[G::R])
{
    f2x Z[G::NZ];
    load_line<G>(line, j, Z);
    float w[G::H + 1][3];
    load_w<G>(sW, 0, 0, w);
    line_mags_strip_real<G::L, G::R>(Z, tw, [&](int r, int om, float m) { wsum(w[om], m, et[r], ex[r], ey[r]); });
}

// x stage for one mu: G1[mu](x-h..x+h, y') -> G2[mu, nu](x, y') for the BT x BX x PY items.
template <class G>
__device__ __forceinline__ void x_stage(const float *sG1, float2 *sG2, int mu, const Tw<G::L> &tw)
{
    constexpr int L = G::L, H = G::H, PY = G::PY, NITEM = G::ROWS * PY;
    if (mu == 0) {
        for (int i = threadIdx.x; i < NITEM; i += G::NT) {
            const int row = i / PY, yy = i - row * PY;
            const int t = row / G::BX, x = row - t * G::BX;
            const float *g = sG1 + ((t * G::HX + x) * L) * PY + yy;
            float2 *o = sG2 + (row * L + H) * G::PY2 + yy;
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
                    A = fmaf(U[k], lo(tw.c2[(nu * k) % L]), A);
                    B = fmaf(D[k], lo(tw.s2[(nu * k) % L]), B);
                }
                o[nu * G::PY2] = make_float2(A, -B);   // G2(+nu) = A - iB; nu < 0 is its mirror
            }
        }
    } else {
        const int cre = (2 * mu - 1) * PY, cim = 2 * mu * PY;
        const f2x m2 = pk(-2.f, -2.f);
        for (int i = threadIdx.x; i < NITEM; i += G::NT) {
            const int row = i / PY, yy = i - row * PY;
            const int t = row / G::BX, x = row - t * G::BX;
            const float *g = sG1 + ((t * G::HX + x) * L) * PY + yy;
            f2x *o = reinterpret_cast<f2x *>(sG2 + (row * L + H) * G::PY2 + yy);
            f2x z[L];
#pragma unroll
            for (int k = 0; k < L; ++k) z[k] = pk(g[k * L * PY + cre], g[k * L * PY + cim]);
            const f2x z0 = z[H];
            f2x s = z0, U[H + 1], D[H + 1];
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const f2x p = add2(z[H + k], z[H - k]);
                s = add2(s, p);
                U[k] = fma2(z0, m2, p);
                D[k] = sub2(z[H + k], z[H - k]);
            }
            o[0] = s;
#pragma unroll
            for (int nu = 1; nu <= H; ++nu) {
                f2x A = mul2(U[1], tw.c2[nu % L]);
                f2x B = mul2(D[1], tw.s2[nu % L]);
#pragma unroll
                for (int k = 2; k <= H; ++k) {
                    A = fma2(U[k], tw.c2[(nu * k) % L], A);
                    B = fma2(D[k], tw.s2[(nu * k) % L], B);
                }
                const float ax = lo(A), ay = hi(A), bx = lo(B), by = hi(B);
                o[nu * G::PY2] = pk(ax + by, ay - bx);    // G2(+nu) = A - iB
                o[-nu * G::PY2] = pk(ax - by, ay + bx);   // G2(-nu) = A + iB
            }
        }
    }
}

// Stage x by a sliding recurrence along x: one thread per (t, y') column of the tile walks
// the BX output positions.  Window 0 by the folded direct DFT; window r >= 1 by
// Q_r(nu) = Q_{r-1}(nu) + (z[r+2h] - z[r-1]) e^{-i th nu (r-1-h)} with Q_0 = F_0, so that
// Q_r(nu) = e^{-i th nu r} F_r(nu).  That unit factor depends on (nu, x) only, the same for
// every y' of a G2 line, so the y transform carries it unchanged into F and |F| does not
// see it.  mu = 0 (real input) writes lines nu = 0..h.  Layout of a G2 row (L x PY2 float2):
// modes 0 and 3 with PAIR4 (L <= 11) put the line nu = 0 first and then, for mu > 0, each
// pair (+nu, -nu) as PY2 float4 columns (Re +nu, Re -nu, Im +nu, Im -nu); with PAIR0 (L = 9,
// 11) the mu = 0 lines nu = 1, 2 (3, 4, ...) are paired the same way and an odd last line
// follows alone; otherwise line nu sits at slot h + nu.
template <class G>
__device__ __forceinline__ void x_stage_slide(const float *sG1, float2 *sG2, int mu, const Tw<G::L> &tw)
{
    constexpr int L = G::L, H = G::H, PY = G::PY, BX = G::BX, NZX = BX + 2 * H;
    constexpr int XS = L * PY;           // G1 stride between x'
    constexpr int RS = L * G::PY2;       // G2 stride between output rows x
    for (int i = threadIdx.x; i < G::BT * PY; i += G::NT) {
        const int t = i / PY, yy = i - t * PY;
        const float *g = sG1 + (t * G::HX * L) * PY + yy;
        float2 *o = sG2 + ((t * BX) * L + H) * G::PY2 + yy;   // line nu = 0 of output row (t, x = 0)
        if (mu == 0 && G::PAIR0) {
            // real input, lines nu = 0..H; row = [nu = 0: PY2 float2][pairs (1, 2), (3, 4), ...:
            // PY2 float4 each, (Re a, Re b, Im a, Im b)][nu = H alone when H is odd: PY2 float2]
            float z[NZX];
#pragma unroll
            for (int n = 0; n < NZX; ++n) z[n] = g[n * XS];
            const float z0 = z[H];
            float sum = z0, U[H + 1], D[H + 1];
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const float p = z[H + k] + z[H - k];
                sum += p;
                U[k] = fmaf(-2.f, z0, p);
                D[k] = z[H + k] - z[H - k];
            }
            float2 *r0 = sG2 + (t * BX) * RS + yy;
            float4 *q0 = reinterpret_cast<float4 *>(sG2 + (t * BX) * RS + G::PY2) + yy;
            float pr[H + 1], pi[H + 1];
#pragma unroll
            for (int nu = 1; nu <= H; ++nu) {
                float A = 0.f, B = 0.f;
#pragma unroll
                for (int k = 1; k <= H; ++k) {
                    A = fmaf(U[k], lo(tw.c2[(nu * k) % L]), A);
                    B = fmaf(D[k], lo(tw.s2[(nu * k) % L]), B);
                }
                pr[nu] = A;   // F_0(nu) = A - iB = Q_0(nu)
                pi[nu] = -B;
            }
#pragma unroll
            for (int r = 0; r < BX; ++r) {
                if (r > 0) {
                    const float d = z[r + 2 * H] - z[r - 1];
                    sum += d;
#pragma unroll
                    for (int nu = 1; nu <= H; ++nu) {
                        const int k = tw_index<L>(nu, r - 1 - H);
                        pr[nu] = fmaf(d, lo(tw.c2[k]), pr[nu]);    // + d e^{-i th k}
                        pi[nu] = fmaf(-d, lo(tw.s2[k]), pi[nu]);
                    }
                }
                r0[r * RS] = make_float2(sum, 0.f);
#pragma unroll
                for (int q = 0; q < H / 2; ++q)
                    q0[r * (RS / 2) + q * G::PY2] = make_float4(pr[2 * q + 1], pr[2 * q + 2], pi[2 * q + 1], pi[2 * q + 2]);
                if (H & 1) r0[r * RS + H * G::PY2] = make_float2(pr[H], pi[H]);
            }
        } else if (mu == 0) {
            float z[NZX];
#pragma unroll
            for (int n = 0; n < NZX; ++n) z[n] = g[n * XS];
            const float z0 = z[H];
            float sum = z0, U[H + 1], D[H + 1];
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const float p = z[H + k] + z[H - k];
                sum += p;
                U[k] = fmaf(-2.f, z0, p);
                D[k] = z[H + k] - z[H - k];
            }
            o[0] = make_float2(sum, 0.f);
            float pr[H + 1], pi[H + 1];
#pragma unroll
            for (int nu = 1; nu <= H; ++nu) {
                float A = 0.f, B = 0.f;
#pragma unroll
                for (int k = 1; k <= H; ++k) {
                    A = fmaf(U[k], lo(tw.c2[(nu * k) % L]), A);
                    B = fmaf(D[k], lo(tw.s2[(nu * k) % L]), B);
                }
                o[nu * G::PY2] = make_float2(A, -B);   // F_0(nu) = A - iB = Q_0(nu)
                pr[nu] = A;
                pi[nu] = -B;
            }
#pragma unroll
            for (int r = 1; r < BX; ++r) {
                const float d = z[r + 2 * H] - z[r - 1];
                sum += d;
                float2 *orow = o + r * RS;
                orow[0] = make_float2(sum, 0.f);
#pragma unroll
                for (int nu = 1; nu <= H; ++nu) {
                    const int k = tw_index<L>(nu, r - 1 - H);
                    pr[nu] = fmaf(d, lo(tw.c2[k]), pr[nu]);    // + d e^{-i th k}
                    pi[nu] = fmaf(-d, lo(tw.s2[k]), pi[nu]);
                    orow[nu * G::PY2] = make_float2(pr[nu], pi[nu]);
                }
            }
        } else if constexpr (G::PAIR4) {
            // mu > 0: row = [line nu = 0: PY2 float2][pair |nu| = 1..H: PY2 float4 each], a pair
            // column holding (Re G2(+nu), Re G2(-nu), Im G2(+nu), Im G2(-nu)) so that stage y
            // reads both lines of a pair with one 128-bit load, already transposed
            const int cre = (2 * mu - 1) * PY, cim = 2 * mu * PY;
            const f2x m2 = pk(-2.f, -2.f);
            f2x z[NZX];
#pragma unroll
            for (int n = 0; n < NZX; ++n) z[n] = pk(g[n * XS + cre], g[n * XS + cim]);
            const f2x z0 = z[H];
            f2x sum = z0, U[H + 1], D[H + 1];
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const f2x p = add2(z[H + k], z[H - k]);
                sum = add2(sum, p);
                U[k] = fma2(z0, m2, p);
                D[k] = sub2(z[H + k], z[H - k]);
            }
            f2x *o2 = reinterpret_cast<f2x *>(sG2 + (t * BX) * RS) + yy;              // line nu = 0, row x = 0
            float4 *o4 = reinterpret_cast<float4 *>(sG2 + (t * BX) * RS + G::PY2) + yy;   // pair 1, row x = 0
            o2[0] = sum;
            f2x Pp[H + 1], Pm[H + 1];   // P(+nu), P(-nu)
#pragma unroll
            for (int nu = 1; nu <= H; ++nu) {
                f2x A = mul2(U[1], tw.c2[nu % L]);
                f2x B = mul2(D[1], tw.s2[nu % L]);
#pragma unroll
                for (int k = 2; k <= H; ++k) {
                    A = fma2(U[k], tw.c2[(nu * k) % L], A);
                    B = fma2(D[k], tw.s2[(nu * k) % L], B);
                }
                const float ax = lo(A), ay = hi(A), bx = lo(B), by = hi(B);
                const f2x Fp = pk(ax + by, ay - bx);   // F_0(+nu) = A - iB
                const f2x Fm = pk(ax - by, ay + bx);   // F_0(-nu) = A + iB
                o4[(nu - 1) * G::PY2] = make_float4(lo(Fp), lo(Fm), hi(Fp), hi(Fm));
                Pp[nu] = Fp;
                Pm[nu] = Fm;
            }
#pragma unroll
            for (int r = 1; r < BX; ++r) {
                const f2x d = sub2(z[r + 2 * H], z[r - 1]);
                const f2x dsw = swapneg(d);
                sum = add2(sum, d);
                o2[r * RS] = sum;
#pragma unroll
                for (int nu = 1; nu <= H; ++nu) {
                    const int k = tw_index<L>(nu, r - 1 - H);
                    Pp[nu] = rot_acc<L>(Pp[nu], d, dsw, tw, k);
                    Pm[nu] = rot_acc<L>(Pm[nu], d, dsw, tw, (L - k) % L);
                    o4[r * (RS / 2) + (nu - 1) * G::PY2] = make_float4(lo(Pp[nu]), lo(Pm[nu]), hi(Pp[nu]), hi(Pm[nu]));
                }
            }
        } else {
            // mu > 0, lines nu = -H..H at slot H + nu
            const int cre = (2 * mu - 1) * PY, cim = 2 * mu * PY;
            const f2x m2 = pk(-2.f, -2.f);
            f2x z[NZX];
#pragma unroll
            for (int n = 0; n < NZX; ++n) z[n] = pk(g[n * XS + cre], g[n * XS + cim]);
            const f2x z0 = z[H];
            f2x sum = z0, U[H + 1], D[H + 1];
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const f2x p = add2(z[H + k], z[H - k]);
                sum = add2(sum, p);
                U[k] = fma2(z0, m2, p);
                D[k] = sub2(z[H + k], z[H - k]);
            }
            f2x *o2 = reinterpret_cast<f2x *>(o);
            o2[0] = sum;
            f2x Pp[H + 1], Pm[H + 1];   // P(+nu), P(-nu)
#pragma unroll
            for (int nu = 1; nu <= H; ++nu) {
                f2x A = mul2(U[1], tw.c2[nu % L]);
                f2x B = mul2(D[1], tw.s2[nu % L]);
#pragma unroll
                for (int k = 2; k <= H; ++k) {
                    A = fma2(U[k], tw.c2[(nu * k) % L], A);
                    B = fma2(D[k], tw.s2[(nu * k) % L], B);
                }
                const float ax = lo(A), ay = hi(A), bx = lo(B), by = hi(B);
                const f2x Fp = pk(ax + by, ay - bx);   // F_0(+nu) = A - iB
                const f2x Fm = pk(ax - by, ay + bx);   // F_0(-nu) = A + iB
                o2[nu * G::PY2] = Fp;
                o2[-nu * G::PY2] = Fm;
                Pp[nu] = Fp;
                Pm[nu] = Fm;
            }
#pragma unroll
            for (int r = 1; r < BX; ++r) {
                const f2x d = sub2(z[r + 2 * H], z[r - 1]);
                const f2x dsw = swapneg(d);
                sum = add2(sum, d);
                f2x *orow = o2 + r * RS;
                orow[0] = sum;
#pragma unroll
                for (int nu = 1; nu <= H; ++nu) {
                    const int k = tw_index<L>(nu, r - 1 - H);
                    Pp[nu] = rot_acc<L>(Pp[nu], d, dsw, tw, k);
                    Pm[nu] = rot_acc<L>(Pm[nu], d, dsw, tw, (L - k) % L);
                    orow[nu * G::PY2] = Pp[nu];
                    orow[-nu * G::PY2] = Pm[nu];
                }
            }
        }
    }
}

// Asynchronous 4-byte copy global -> shared (completion by cp.async.wait_*).
__device__ __forceinline__ void cp_async_f32(float *dst, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}

// Issues the asynchronous 4-byte copies of one tile's V halo into sV ([plane][row][column],
// NV floats); outside the volume the boundary extension supplies the samples.  Element
// i = (a, x', y') advances by NT elements at a time, NT / PY rows and NT % PY columns further,
// so no element needs a division.  Interior tiles address the volume by 32-bit offsets from
// the halo's first sample; tiles at a face extend each coordinate (a range check, the
// extension only outside).  G provides BT, BX, BY, H, HX, PY, NV and NT.
template <class G>
__device__ __forceinline__ void issue_v_copies(const float *__restrict__ V, int64_t T, int64_t X, int64_t Y, int bnd,
                                               int64_t t0, int64_t x0, int64_t y0, float *sV)
{
    constexpr int H = G::H, PY = G::PY, HX = G::HX;
    constexpr int DRS = G::NT / PY, DYS = G::NT - DRS * PY;
    static_assert(DRS + 1 < HX, "one step crosses at most one plane");
    int yy = threadIdx.x % PY, r = threadIdx.x / PY;
    int xx = r % HX, a = r / HX;
    auto advance = [&]() {
        yy += DYS;
        int dr = DRS;
        if (yy >= PY) {
            yy -= PY;
            ++dr;
        }
        xx += dr;
        if (xx >= HX) {
            xx -= HX;
            ++a;
        }
    };
    const bool inside = t0 - H >= 0 && t0 + G::BT + H <= T && x0 - H >= 0 && x0 + G::BX + H <= X && y0 - H >= 0 &&
                        y0 + G::BY + H <= Y && (int64_t)(G::BT + 2 * H) * X * Y < 0x7fffffffLL;
    if (inside) {
        // whole rows (plane a, halo row xx) per warp, lanes along the row: the row's source
        // offset and destination advance by a fixed step per row, so each copy costs a couple of
        // additions; lanes below PY - 32 take the row's last columns too
        constexpr int NW_ = G::NT / 32, ROWS_ = (G::BT + 2 * H) * HX;
        static_assert(NW_ < HX && PY > 32 && PY <= 64, "row walk: one plane step per row step, two copies per lane");
        (void)advance;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int Yi = (int)Y, XYi = (int)(X * Y);
        const float *src = V + ((t0 - H) * X + (x0 - H)) * Y + (y0 - H) + lane;
        int rx = warp;                                       // halo row of the current plane
        int off = warp * Yi;                                 // source offset of row `warp`
        unsigned dst = (unsigned)__cvta_generic_to_shared(sV + warp * PY + lane);
        const int wrap = XYi - HX * Yi;                      // extra source step into the next plane
        const bool two = lane < PY - 32;
        for (int r = warp; r < ROWS_; r += NW_) {
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src + off) : "memory");
            if (two) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst + 128u), "l"(src + off + 32) : "memory");
            dst += NW_ * PY * (unsigned)sizeof(float);
            off += NW_ * Yi;
            rx += NW_;
            if (rx >= HX) {
                rx -= HX;
                off += wrap;
            }
        }
    } else {
        for (int i = threadIdx.x; i < G::NV; i += G::NT) {
            int64_t gt = t0 - H + a, gx = x0 - H + xx, gy = y0 - H + yy;
            if ((uint64_t)gt >= (uint64_t)T) gt = ext_index(gt, T, bnd);
            if ((uint64_t)gx >= (uint64_t)X) gx = ext_index(gx, X, bnd);
            if ((uint64_t)gy >= (uint64_t)Y) gy = ext_index(gy, Y, bnd);
            cp_async_f32(sV + i, V + (gt * X + gx) * Y + gy);
            advance();
        }
    }
}

// Halo tile of V in shared memory, complete and visible to the thread on return (the caller
// synchronises the CTA).
template <class G>
__device__ __forceinline__ void stage_v(const float *__restrict__ V, int64_t T, int64_t X, int64_t Y, int bnd,
                                        int64_t t0, int64_t x0, int64_t y0, float *sV)
{
    issue_v_copies<G>(V, T, X, Y, bnd, t0, x0, y0, sV);
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Stage t: every (t, x', y') column of the halo tile -> G1 components
// [Re G1(0), Re G1(1), Im G1(1), ..., Re G1(h), Im G1(h)] in sG1[(t, x')][component][y'].
template <class G>
__device__ __forceinline__ void t_stage(const float *sV, float *sG1, const Tw<G::L> &tw)
{
    constexpr int L = G::L, H = G::H, PY = G::PY;
    // item i = (row r = (t, x'), column y') of the output planes; its samples along t are
    // the halo elements i + k HX PY.  (r, y') advance by NT items at a time.
    constexpr int DRS = G::NT / PY, DYS = G::NT - DRS * PY;
    int r = threadIdx.x / PY, yy = threadIdx.x - r * PY;
    for (int i = threadIdx.x; i < G::BT * G::HX * PY; i += G::NT) {
        float a[L];
#pragma unroll
        for (int k = 0; k < L; ++k) a[k] = sV[i + k * G::HX * PY];
        const float a0 = a[H];
        float s = a0, U[H + 1], D[H + 1];
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const float p = a[H + k] + a[H - k];
            s += p;
            U[k] = fmaf(-2.f, a0, p);
            D[k] = a[H + k] - a[H - k];
        }
        float *o = sG1 + (r * L) * PY + yy;
        o[0] = s;
#pragma unroll
        for (int mu = 1; mu <= H; ++mu) {
            float A = 0.f, B = 0.f;
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                A = fmaf(U[k], lo(tw.c2[(mu * k) % L]), A);
                B = fmaf(D[k], lo(tw.s2[(mu * k) % L]), B);
            }
            o[(2 * mu - 1) * PY] = A;     // G1(mu) = A - iB
            o[(2 * mu) * PY] = -B;
        }
        yy += DYS;
        r += DRS;
        if (yy >= PY) {
            yy -= PY;
            ++r;
        }
    }
}

// Writes this thread's R outputs of E_t, E_x, E_y (scaled by the mean's factor).
template <class G>
__device__ __forceinline__ void store_outputs(float *__restrict__ E, int64_t T, int64_t X, int64_t Y, int64_t t0,
                                              int64_t x0, int64_t y0, int row, int j, float sc,
                                              const float (&et)[G::R], const float (&ex)[G::R],
                                              const float (&ey)[G::R])
{
    const int t = row / G::BX, x = row - t * G::BX;
    const int64_t gt = t0 + t, gx = x0 + x, gy = y0 + G::R * j;
    if (gt >= T || gx >= X) return;
    const int64_t N = T * X * Y;
    float *e0 = E + (gt * X + gx) * Y + gy;
    if (gy + G::R <= Y && (reinterpret_cast<uintptr_t>(e0) & 15) == 0 && (Y & 3) == 0) {
#pragma unroll
        for (int c = 0; c < G::R; c += 4) {
            *reinterpret_cast<float4 *>(e0 + c) = make_float4(et[c] * sc, et[c + 1] * sc, et[c + 2] * sc, et[c + 3] * sc);
            *reinterpret_cast<float4 *>(e0 + c + N) =
                make_float4(ex[c] * sc, ex[c + 1] * sc, ex[c + 2] * sc, ex[c + 3] * sc);
            *reinterpret_cast<float4 *>(e0 + c + 2 * N) =
                make_float4(ey[c] * sc, ey[c + 1] * sc, ey[c + 2] * sc, ey[c + 3] * sc);
        }
        return;
    }
    {
#pragma unroll
        for (int r = 0; r < G::R; ++r) {
            if (gy + r < Y) {
                e0[r] = et[r] * sc;
                e0[r + N] = ex[r] * sc;
                e0[r + 2 * N] = ey[r] * sc;
            }
        }
    }
}

// One output tile of one volume.  Every thread of the CTA calls it with the same tile.
// Stage y of one mu for this thread's strip j of output row `row`: every line of the G2 slice
// that x_stage_slide left in sG2.
template <class G>
__device__ __forceinline__ void y_stage_mu(const float2 *sG2, int row, int j, int mu, const float *sW,
                                           const Tw<G::L> &tw, float (&et)[G::R], float (&ex)[G::R],
                                           float (&ey)[G::R])
{
    constexpr int L = G::L, H = G::H;
    if (mu == 0 && G::PAIR0) {
        const float2 *l0 = sG2 + row * L * G::PY2;         // nu = 0, the pairs (1, 2), ..., nu = H if odd
        y_real<G>(l0, j, sW, tw, et, ex, ey);
        const float4 *l4 = reinterpret_cast<const float4 *>(l0 + G::PY2);
#pragma unroll 1
        for (int q = 0; q < H / 2; ++q) y_single_pair4<G>(l4 + q * G::PY2, j, 0, 2 * q + 1, 2 * q + 2, sW, tw, et, ex, ey);
        if (H & 1) y_single<G>(l0 + H * G::PY2, j, 0, H, sW, tw, et, ex, ey);
    } else if constexpr (G::PAIR4 && G::PAIR0) {
        const float2 *l0 = sG2 + row * L * G::PY2;         // line nu = 0, then the pairs |nu| = 1..H
        y_single<G>(l0, j, mu, 0, sW, tw, et, ex, ey);
        const float4 *l4 = reinterpret_cast<const float4 *>(l0 + G::PY2);
#pragma unroll 1
        for (int nu = 1; nu <= H; ++nu) y_pair4<G>(l4 + (nu - 1) * G::PY2, j, mu, nu, sW, tw, et, ex, ey);
    } else if constexpr (G::PAIR4) {
        // single lines from one call site (mu = 0: nu = 1..H after the real line; mu > 0: the
        // nu = 0 line before the pairs), so the walker is inlined once
        const float2 *sl = sG2 + row * L * G::PY2;         // mu > 0: line nu = 0, then the pairs
        int s0 = 0, s1 = 0;
        if (mu == 0) {
            sl = sG2 + (row * L + H) * G::PY2;             // line nu = 0 of this row
            y_real<G>(sl, j, sW, tw, et, ex, ey);
            s0 = 1;
            s1 = H;
        }
#pragma unroll 1
        for (int nu = s0; nu <= s1; ++nu) y_single<G>(sl + nu * G::PY2, j, mu, nu, sW, tw, et, ex, ey);
        if (mu > 0) {
            const float4 *l4 = reinterpret_cast<const float4 *>(sl + G::PY2);
#pragma unroll 1
            for (int nu = 1; nu <= H; ++nu) y_pair4<G>(l4 + (nu - 1) * G::PY2, j, mu, nu, sW, tw, et, ex, ey);
        }
    } else if (mu == 0) {
        const float2 *l0 = sG2 + (row * L + H) * G::PY2;   // line nu = 0 of this row
        y_real<G>(l0, j, sW, tw, et, ex, ey);
#pragma unroll 1
        for (int nu = 1; nu <= H; ++nu) y_single<G>(l0 + nu * G::PY2, j, 0, nu, sW, tw, et, ex, ey);
    } else {
        const float2 *l0 = sG2 + (row * L + H) * G::PY2;   // line nu = 0 of this row
        y_single<G>(l0, j, mu, 0, sW, tw, et, ex, ey);
#pragma unroll 1
        for (int nu = 1; nu <= H; ++nu) y_pair<G>(l0 + nu * G::PY2, l0 - nu * G::PY2, j, mu, nu, sW, tw, et, ex, ey);
    }
}

template <class G>
__device__ __forceinline__ void energy_tile(const float *__restrict__ V, int64_t T, int64_t X, int64_t Y, int bnd,
                                            int64_t tile, int tiles_x, int tiles_y, float *__restrict__ E,
                                            const SpecTables &tb, float *smem)
{
    constexpr int L = G::L, H = G::H;
    float *sG1 = smem;
    float2 *sG2 = reinterpret_cast<float2 *>(smem + G::NG1);
    float *sV = smem + G::NG1;   // aliases sG2: dead once stage t is done
    float *sW = smem + G::NG1 + G::NALIAS;

    fill_w<G>(sW, tb);
    const int ty = (int)(tile % tiles_y);
    const int tx = (int)((tile / tiles_y) % tiles_x);
    const int64_t tt = tile / ((int64_t)tiles_y * tiles_x);
    const int64_t t0 = tt * G::BT, x0 = (int64_t)tx * G::BX, y0 = (int64_t)ty * G::BY;

    stage_v<G>(V, T, X, Y, bnd, t0, x0, y0, sV);
    __syncthreads();
    Tw<L> tw;
    tw.load(tb);
    t_stage<G>(sV, sG1, tw);
    __syncthreads();

    const int row = threadIdx.x % G::ROWS, j = threadIdx.x / G::ROWS;
    const bool ylive = y0 + G::R * j < Y;   // strips wholly past the last column sit out stage y
    float et[G::R], ex[G::R], ey[G::R];
#pragma unroll
    for (int r = 0; r < G::R; ++r) et[r] = ex[r] = ey[r] = 0.f;

#pragma unroll 1
    for (int mu = 0; mu <= H; ++mu) {
        x_stage_slide<G>(sG1, sG2, mu, tw);
        __syncthreads();
        if (ylive) y_stage_mu<G>(sG2, row, j, mu, sW, tw, et, ex, ey);
        __syncthreads();
    }

    store_outputs<G>(E, T, X, Y, t0, x0, y0, row, j, tb.escale, et, ex, ey);
}

// ---- batched modes (1, 2) -------------------------------------------------------------
// Twiddles of one runtime frequency index a: c[k] = cos(2 pi a k / L), s[k] = sin(...),
// k = 1..H, read from the parameter bank (a register array cannot be indexed at run time).
template <int L>
struct TwRow {
    static constexpr int H = (L - 1) / 2;
    float c[H + 1], s[H + 1];
    __device__ __forceinline__ void load(const SpecTables &tb, int a)
    {
        int idx = 0;
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            idx += a;
            if (idx >= L) idx -= L;
            c[k] = tb.cs[idx];
            s[k] = tb.sn[idx];
        }
    }
};

// Stage t for one mu: G1(mu) of every (t, x', y') column of the tile into
// sG1m[((t * HX + x') * 2 + part) * PY + y'] (part 0 = Re, 1 = Im; mu = 0 writes Re only).
template <class G>
__device__ __forceinline__ void t_stage_mu(const float *sV, float *sG1m, int mu, const TwRow<G::L> &tr)
{
    constexpr int L = G::L, H = G::H, PY = G::PY;
    // item i = (row r = (t, x'), column y') of the output planes; its samples along t are
    // the halo elements i + k HX PY.  (r, y') advance by NT items at a time.
    constexpr int DRS = G::NT / PY, DYS = G::NT - DRS * PY;
    int r = threadIdx.x / PY, yy = threadIdx.x - r * PY;
    for (int i = threadIdx.x; i < G::BT * G::HX * PY; i += G::NT) {
        float a[L];
#pragma unroll
        for (int k = 0; k < L; ++k) a[k] = sV[i + k * G::HX * PY];
        float *o = sG1m + (2 * r) * PY + yy;
        if (mu == 0) {
            float sum = a[H];
#pragma unroll
            for (int k = 1; k <= H; ++k) sum += a[H + k] + a[H - k];
            o[0] = sum;
        } else {
            const float a0 = a[H];
            float A = 0.f, B = 0.f;
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                A = fmaf(fmaf(-2.f, a0, a[H + k] + a[H - k]), tr.c[k], A);
                B = fmaf(a[H + k] - a[H - k], tr.s[k], B);
            }
            o[0] = A;       // G1(mu) = A - iB
            o[PY] = -B;
        }
        yy += DYS;
        r += DRS;
        if (yy >= PY) {
            yy -= PY;
            ++r;
        }
    }
}

// Stage x for the lines nu = +a and nu = -a of one mu: reads G1(mu) at x' = x - h .. x + h
// (column pointer g1 + (t * HX + x') * xs + y', real part at +ore, imaginary at +oim) and
// writes G2 line s (0: +a, 1: -a) of output row `row` at sG2b[(s * ROWS + row) * PY2 + y'].
// mu = 0 (real input) writes only line +a.
template <class G>
__device__ __forceinline__ void x_stage_b(const float *g1, int xs, int ore, int oim, float2 *sG2b, int mu, int a,
                                          const TwRow<G::L> &tr)
{
    constexpr int L = G::L, H = G::H, PY = G::PY, NITEM = G::ROWS * PY;
    for (int i = threadIdx.x; i < NITEM; i += G::NT) {
        const int row = i / PY, yy = i - row * PY;
        const int t = row / G::BX, x = row - t * G::BX;
        const float *g = g1 + (t * G::HX + x) * xs + yy;
        float2 *o = sG2b + row * G::PY2 + yy;
        if (mu == 0) {
            float z[L];
#pragma unroll
            for (int k = 0; k < L; ++k) z[k] = g[k * xs + ore];
            if (a == 0) {
                float sum = z[H];
#pragma unroll
                for (int k = 1; k <= H; ++k) sum += z[H + k] + z[H - k];
                o[0] = make_float2(sum, 0.f);
            } else {
                const float z0 = z[H];
                float A = 0.f, B = 0.f;
#pragma unroll
                for (int k = 1; k <= H; ++k) {
                    A = fmaf(fmaf(-2.f, z0, z[H + k] + z[H - k]), tr.c[k], A);
                    B = fmaf(z[H + k] - z[H - k], tr.s[k], B);
                }
                o[0] = make_float2(A, -B);
            }
        } else {
            f2x z[L];
#pragma unroll
            for (int k = 0; k < L; ++k) z[k] = pk(g[k * xs + ore], g[k * xs + oim]);
            f2x *o2 = reinterpret_cast<f2x *>(o);
            if (a == 0) {
                f2x sum = z[H];
#pragma unroll
                for (int k = 1; k <= H; ++k) sum = add2(sum, add2(z[H + k], z[H - k]));
                o2[0] = sum;
            } else {
                const f2x m2 = pk(-2.f, -2.f), z0 = z[H];
                f2x A = pk(0.f, 0.f), B = pk(0.f, 0.f);
#pragma unroll
                for (int k = 1; k <= H; ++k) {
                    A = fma2(fma2(z0, m2, add2(z[H + k], z[H - k])), pk(tr.c[k], tr.c[k]), A);
                    B = fma2(sub2(z[H + k], z[H - k]), pk(tr.s[k], tr.s[k]), B);
                }
                const float ax = lo(A), ay = hi(A), bx = lo(B), by = hi(B);
                o2[0] = pk(ax + by, ay - bx);                 // G2(+a) = A - iB
                o2[G::ROWS * G::PY2] = pk(ax - by, ay + bx);  // G2(-a) = A + iB
            }
        }
    }
}

// One output tile in a batched mode: per mu (and, in mode 2, its own stage t), per |nu|
// batch the x stage of the lines +-|nu| into the small G2 buffer, then their y stage.
template <class G>
__device__ __forceinline__ void energy_tile_b(const float *__restrict__ V, int64_t T, int64_t X, int64_t Y, int bnd,
                                              int64_t tile, int tiles_x, int tiles_y, float *__restrict__ E,
                                              const SpecTables &tb, float *smem)
{
    constexpr int L = G::L, H = G::H, PY = G::PY;
    float *sV, *sG1;
    float2 *sG2b;
    float *sW;
    if (G::MODE == 1) {
        sG1 = smem;
        sV = smem + G::NG1;   // aliases the G2 batch: dead once stage t is done
        sG2b = reinterpret_cast<float2 *>(smem + G::NG1);
        sW = smem + G::NG1 + (G::NVR > 2 * G::NG2B ? G::NVR : 2 * G::NG2B);
    } else {
        sV = smem;
        sG1 = smem + G::NVR;
        sG2b = reinterpret_cast<float2 *>(smem + G::NVR + G::NG1M);
        sW = smem + G::NVR + G::NG1M + 2 * G::NG2B;
    }

    fill_w<G>(sW, tb);
    const int ty = (int)(tile % tiles_y);
    const int tx = (int)((tile / tiles_y) % tiles_x);
    const int64_t tt = tile / ((int64_t)tiles_y * tiles_x);
    const int64_t t0 = tt * G::BT, x0 = (int64_t)tx * G::BX, y0 = (int64_t)ty * G::BY;

    stage_v<G>(V, T, X, Y, bnd, t0, x0, y0, sV);
    __syncthreads();
    Tw<L> tw;
    tw.load(tb);
    if (G::MODE == 1) {
        t_stage<G>(sV, sG1, tw);
        __syncthreads();
    }

    const int row = threadIdx.x % G::ROWS, j = threadIdx.x / G::ROWS;
    float et[G::R], ex[G::R], ey[G::R];
#pragma unroll
    for (int r = 0; r < G::R; ++r) et[r] = ex[r] = ey[r] = 0.f;
    const float2 *lp = sG2b + row * G::PY2, *lm = lp + G::ROWS * G::PY2;

#pragma unroll 1
    for (int mu = 0; mu <= H; ++mu) {
        int xs, ore, oim;
        if (G::MODE == 1) {
            xs = L * PY;
            ore = mu == 0 ? 0 : (2 * mu - 1) * PY;
            oim = 2 * mu * PY;
        } else {
            TwRow<L> trm;
            trm.load(tb, mu);
            t_stage_mu<G>(sV, sG1, mu, trm);
            __syncthreads();
            xs = 2 * PY;
            ore = 0;
            oim = PY;
        }
#pragma unroll 1
        for (int a = 0; a <= H; ++a) {
            TwRow<L> tr;
            tr.load(tb, a);
            x_stage_b<G>(sG1, xs, ore, oim, sG2b, mu, a, tr);
            __syncthreads();
            if (mu == 0) {
                if (a == 0)
                    y_real<G>(lp, j, sW, tw, et, ex, ey);
                else
                    y_single<G>(lp, j, 0, a, sW, tw, et, ex, ey);
            } else {
                if (a == 0)
                    y_single<G>(lp, j, mu, 0, sW, tw, et, ex, ey);
                else
                    y_pair<G>(lp, lm, j, mu, a, sW, tw, et, ex, ey);
            }
            __syncthreads();
        }
    }
    store_outputs<G>(E, T, X, Y, t0, x0, y0, row, j, tb.escale, et, ex, ey);
}

// ---- mode 4: the G2 slice of a mu in batches of at most NSL line slots --------------------
// Rows of RSB float2 (an odd multiple of 16 bytes apart).  mu = 0 (batch 0 only): lines
// nu = 0..H at slots 0..H, or, with paired single lines (L = 9), the nu = 0 line at slot 0 and
// the pairs (1, 2), (3, 4) at slots 1-2, 3-4.  mu > 0, batch 0: the nu = 0 line at slot 0 and the
// pairs |nu| = 1..P0 from slot 1; batch 1: the pairs P0 + 1..H from slot 0 (pairs interleaved
// per column as in mode 0).  Stage x walks a column once per batch (its loads and differences
// twice per mu > 0, the per-frequency work once), so a CTA needs less shared memory (L = 7:
// 50 KB instead of 65 KB, four CTAs per SM instead of three; L = 9: 74 KB instead of 94 KB,
// three instead of two); the arithmetic and its order are mode 0's.
template <class G, int B>
__device__ __forceinline__ void x_stage_q(const float *sG1, float2 *sG2, int mu, const Tw<G::L> &tw)
{
    constexpr int L = G::L, H = G::H, PY = G::PY, BX = G::BX, NZX = BX + 2 * H;
    constexpr int XS = L * PY;           // G1 stride between x'
    constexpr int RS = G::RSB;           // G2 stride between output rows x (float2)
    constexpr int NLO = B == 0 ? 1 : G::P0 + 1, NHI = B == 0 ? G::P0 : H;   // pairs of this batch (mu > 0)
    for (int i = threadIdx.x; i < G::BT * PY; i += G::NT) {
        const int t = i / PY, yy = i - t * PY;
        const float *g = sG1 + (t * G::HX * L) * PY + yy;
        float2 *o = sG2 + (t * BX) * RS + yy;   // slot 0 of output row (t, x = 0)
        if (mu == 0 && G::PAIR0) {
            // real input: the nu = 0 line at slot 0, the pairs (1, 2), (3, 4), ... from slot 1
            // (Re a, Re b, Im a, Im b per column), nu = H alone after them when H is odd
            float z[NZX];
#pragma unroll
            for (int n = 0; n < NZX; ++n) z[n] = g[n * XS];
            const float z0 = z[H];
            float sum = z0, U[H + 1], D[H + 1];
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const float p = z[H + k] + z[H - k];
                sum += p;
                U[k] = fmaf(-2.f, z0, p);
                D[k] = z[H + k] - z[H - k];
            }
            float4 *q0 = reinterpret_cast<float4 *>(sG2 + (t * BX) * RS + G::PY2) + yy;
            float pr[H + 1], pi[H + 1];
#pragma unroll
            for (int nu = 1; nu <= H; ++nu) {
                float A = 0.f, Bs = 0.f;
#pragma unroll
                for (int k = 1; k <= H; ++k) {
                    A = fmaf(U[k], lo(tw.c2[(nu * k) % L]), A);
                    Bs = fmaf(D[k], lo(tw.s2[(nu * k) % L]), Bs);
                }
                pr[nu] = A;   // F_0(nu) = A - iB = Q_0(nu)
                pi[nu] = -Bs;
            }
#pragma unroll
            for (int r = 0; r < BX; ++r) {
                if (r > 0) {
                    const float d = z[r + 2 * H] - z[r - 1];
                    sum += d;
#pragma unroll
                    for (int nu = 1; nu <= H; ++nu) {
                        const int k = tw_index<L>(nu, r - 1 - H);
                        pr[nu] = fmaf(d, lo(tw.c2[k]), pr[nu]);    // + d e^{-i th k}
                        pi[nu] = fmaf(-d, lo(tw.s2[k]), pi[nu]);
                    }
                }
                o[r * RS] = make_float2(sum, 0.f);
#pragma unroll
                for (int q = 0; q < H / 2; ++q)
                    q0[r * (RS / 2) + q * G::PY2] = make_float4(pr[2 * q + 1], pr[2 * q + 2], pi[2 * q + 1], pi[2 * q + 2]);
                if (H & 1) o[r * RS + H * G::PY2] = make_float2(pr[H], pi[H]);
            }
        } else if (mu == 0) {
            float z[NZX];
#pragma unroll
            for (int n = 0; n < NZX; ++n) z[n] = g[n * XS];
            const float z0 = z[H];
            float sum = z0, U[H + 1], D[H + 1];
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const float p = z[H + k] + z[H - k];
                sum += p;
                U[k] = fmaf(-2.f, z0, p);
                D[k] = z[H + k] - z[H - k];
            }
            o[0] = make_float2(sum, 0.f);
            float pr[H + 1], pi[H + 1];
#pragma unroll
            for (int nu = 1; nu <= H; ++nu) {
                float A = 0.f, Bs = 0.f;
#pragma unroll
                for (int k = 1; k <= H; ++k) {
                    A = fmaf(U[k], lo(tw.c2[(nu * k) % L]), A);
                    Bs = fmaf(D[k], lo(tw.s2[(nu * k) % L]), Bs);
                }
                o[nu * G::PY2] = make_float2(A, -Bs);   // F_0(nu) = A - iB = Q_0(nu)
                pr[nu] = A;
                pi[nu] = -Bs;
            }
#pragma unroll
            for (int r = 1; r < BX; ++r) {
                const float d = z[r + 2 * H] - z[r - 1];
                sum += d;
                float2 *orow = o + r * RS;
                orow[0] = make_float2(sum, 0.f);
#pragma unroll
                for (int nu = 1; nu <= H; ++nu) {
                    const int k = tw_index<L>(nu, r - 1 - H);
                    pr[nu] = fmaf(d, lo(tw.c2[k]), pr[nu]);    // + d e^{-i th k}
                    pi[nu] = fmaf(-d, lo(tw.s2[k]), pi[nu]);
                    orow[nu * G::PY2] = make_float2(pr[nu], pi[nu]);
                }
            }
        } else {
            const int cre = (2 * mu - 1) * PY, cim = 2 * mu * PY;
            const f2x m2 = pk(-2.f, -2.f);
            f2x z[NZX];
#pragma unroll
            for (int n = 0; n < NZX; ++n) z[n] = pk(g[n * XS + cre], g[n * XS + cim]);
            const f2x z0 = z[H];
            f2x sum = z0, U[H + 1], D[H + 1];
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const f2x p = add2(z[H + k], z[H - k]);
                sum = add2(sum, p);
                U[k] = fma2(z0, m2, p);
                D[k] = sub2(z[H + k], z[H - k]);
            }
            f2x *o2 = reinterpret_cast<f2x *>(o);
            // first pair of the batch: a pair line holds one float4 per column y'
            float4 *o4 = reinterpret_cast<float4 *>(sG2 + (t * BX) * RS + (B == 0 ? G::PY2 : 0)) + yy;
            if (B == 0) o2[0] = sum;
            f2x Pp[H + 1], Pm[H + 1];   // P(+nu), P(-nu)
#pragma unroll
            for (int nu = NLO; nu <= NHI; ++nu) {
                f2x A = mul2(U[1], tw.c2[nu % L]);
                f2x Bs = mul2(D[1], tw.s2[nu % L]);
#pragma unroll
                for (int k = 2; k <= H; ++k) {
                    A = fma2(U[k], tw.c2[(nu * k) % L], A);
                    Bs = fma2(D[k], tw.s2[(nu * k) % L], Bs);
                }
                const float ax = lo(A), ay = hi(A), bx = lo(Bs), by = hi(Bs);
                const f2x Fp = pk(ax + by, ay - bx);   // F_0(+nu) = A - iB
                const f2x Fm = pk(ax - by, ay + bx);   // F_0(-nu) = A + iB
                o4[(nu - NLO) * G::PY2] = make_float4(lo(Fp), lo(Fm), hi(Fp), hi(Fm));
                Pp[nu] = Fp;
                Pm[nu] = Fm;
            }
#pragma unroll
            for (int r = 1; r < BX; ++r) {
                const f2x d = sub2(z[r + 2 * H], z[r - 1]);
                const f2x dsw = swapneg(d);
                if (B == 0) {
                    sum = add2(sum, d);
                    o2[r * RS] = sum;
                }
#pragma unroll
                for (int nu = NLO; nu <= NHI; ++nu) {
                    const int k = tw_index<L>(nu, r - 1 - H);
                    Pp[nu] = rot_acc<L>(Pp[nu], d, dsw, tw, k);
                    Pm[nu] = rot_acc<L>(Pm[nu], d, dsw, tw, (L - k) % L);
                    o4[r * (RS / 2) + (nu - NLO) * G::PY2] = make_float4(lo(Pp[nu]), lo(Pm[nu]), hi(Pp[nu]), hi(Pm[nu]));
                }
            }
        }
    }
}

// Stage y of batch b of one mu (the lines x_stage_q<G, b> left in sG2), in mode 0's order;
// rolled loops over the step's single lines and pairs, so each walker is inlined once.
template <class G>
__device__ __forceinline__ void y_stage_q(const float2 *sG2, int row, int j, int mu, int b, const float *sW,
                                          const Tw<G::L> &tw, float (&et)[G::R], float (&ex)[G::R], float (&ey)[G::R])
{
    constexpr int H = G::H;
    const float2 *l0 = sG2 + row * G::RSB;
    if constexpr (G::PAIR0) {
        if (mu == 0) {   // the real line, then the paired single lines (and nu = H alone if odd)
            y_real<G>(l0, j, sW, tw, et, ex, ey);
            const float4 *q4 = reinterpret_cast<const float4 *>(l0 + G::PY2);
#pragma unroll 1
            for (int q = 0; q < H / 2; ++q)
                y_single_pair4<G>(q4 + q * G::PY2, j, 0, 2 * q + 1, 2 * q + 2, sW, tw, et, ex, ey);
            if (H & 1) y_single<G>(l0 + H * G::PY2, j, 0, H, sW, tw, et, ex, ey);
            return;
        }
    }
    // single lines: mu = 0, nu = 1..H (after the real line nu = 0); mu > 0, batch 0: nu = 0
    int s0 = 0, s1 = b == 0 ? 0 : -1;
    if (!G::PAIR0 && mu == 0) {
        y_real<G>(l0, j, sW, tw, et, ex, ey);
        s0 = 1;
        s1 = H;
    }
#pragma unroll 1
    for (int nu = s0; nu <= s1; ++nu) y_single<G>(l0 + nu * G::PY2, j, mu, nu, sW, tw, et, ex, ey);
    if (mu == 0) return;
    // pairs: batch 0 the pairs 1..P0 after the single line, batch 1 the pairs P0 + 1..H
    const int p0 = b == 0 ? 1 : G::P0 + 1, p1 = b == 0 ? G::P0 : H;
    const float4 *l4 = reinterpret_cast<const float4 *>(l0 + (b == 0 ? G::PY2 : 0));
#pragma unroll 1
    for (int nu = p0; nu <= p1; ++nu) y_pair4<G>(l4 + (nu - p0) * G::PY2, j, mu, nu, sW, tw, et, ex, ey);
}

template <class G>
__device__ __forceinline__ void energy_tile_q(const float *__restrict__ V, int64_t T, int64_t X, int64_t Y, int bnd,
                                              int64_t tile, int tiles_x, int tiles_y, float *__restrict__ E,
                                              const SpecTables &tb, float *smem)
{
    constexpr int L = G::L, H = G::H;
    float *sG1 = smem;
    float2 *sG2 = reinterpret_cast<float2 *>(smem + G::NG1);
    float *sV = smem + G::NG1;   // aliases sG2: dead once stage t is done
    float *sW = smem + G::NG1 + G::NALIASQ;

    fill_w<G>(sW, tb);
    const int ty = (int)(tile % tiles_y);
    const int tx = (int)((tile / tiles_y) % tiles_x);
    const int64_t tt = tile / ((int64_t)tiles_y * tiles_x);
    const int64_t t0 = tt * G::BT, x0 = (int64_t)tx * G::BX, y0 = (int64_t)ty * G::BY;

    stage_v<G>(V, T, X, Y, bnd, t0, x0, y0, sV);
    __syncthreads();
    Tw<L> tw;
    tw.load(tb);
    t_stage<G>(sV, sG1, tw);
    __syncthreads();

    const int row = threadIdx.x % G::ROWS, j = threadIdx.x / G::ROWS;
    const bool ylive = y0 + G::R * j < Y;   // strips wholly past the last column sit out stage y
    float et[G::R], ex[G::R], ey[G::R];
#pragma unroll
    for (int r = 0; r < G::R; ++r) et[r] = ex[r] = ey[r] = 0.f;

    // (mu, batch) steps in order, one call site each so that stage y is inlined once
#pragma unroll 1
    for (int step = 0; step < 2 * H + 1; ++step) {
        const int mu = (step + 1) >> 1, b = step > 0 && !(step & 1);
        if (b == 0)
            x_stage_q<G, 0>(sG1, sG2, mu, tw);
        else
            x_stage_q<G, 1>(sG1, sG2, mu, tw);
        __syncthreads();
        if (ylive) y_stage_q<G>(sG2, row, j, mu, b, sW, tw, et, ex, ey);
        __syncthreads();
    }

    store_outputs<G>(E, T, X, Y, t0, x0, y0, row, j, tb.escale, et, ex, ey);
}

template <class G>
__device__ __forceinline__ void energy_tile_any(const float *__restrict__ V, int64_t T, int64_t X, int64_t Y, int bnd,
                                                int64_t tile, int tiles_x, int tiles_y, float *__restrict__ E,
                                                const SpecTables &tb, float *smem)
{
    if constexpr (G::MODE == 0)
        energy_tile<G>(V, T, X, Y, bnd, tile, tiles_x, tiles_y, E, tb, smem);
    else if constexpr (G::MODE == 4)
        energy_tile_q<G>(V, T, X, Y, bnd, tile, tiles_x, tiles_y, E, tb, smem);
    else
        energy_tile_b<G>(V, T, X, Y, bnd, tile, tiles_x, tiles_y, E, tb, smem);
}

// ---- mode 3: the next tile's V halo in flight while the current tile finishes -----------

// Issues the asynchronous copies of one tile's V halo into sV (same layout as stage_v) and
// commits them as one group.
template <class G>
__device__ __forceinline__ void stage_v_async(const float *__restrict__ V, int64_t T, int64_t X, int64_t Y, int bnd,
                                              int64_t t0, int64_t x0, int64_t y0, float *sV)
{
    issue_v_copies<G>(V, T, X, Y, bnd, t0, x0, y0, sV);
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// One tile of a volume: origin and the volume it belongs to.
struct TileRef {
    const float *V;
    float *E;
    int64_t T, X, Y, t0, x0, y0;
};

// One mode-3 tile.  Its V halo is in sV (copies complete and visible); sO is the other
// region.  When `nx` is given, the next tile's V halo is copied into sO once G1 is dead.
template <class G>
__device__ __forceinline__ void energy_tile_pf(const TileRef &c, const TileRef *nx, int bnd, const SpecTables &tb,
                                               float *sV, float *sO, const float *sW)
{
    constexpr int L = G::L, H = G::H;
    float *sG1 = sO;
    float2 *sG2 = reinterpret_cast<float2 *>(sV);   // V is dead once stage t is done
    Tw<L> tw;
    tw.load(tb);
    t_stage<G>(sV, sG1, tw);
    __syncthreads();

    const int row = threadIdx.x % G::ROWS, j = threadIdx.x / G::ROWS;
    const bool ylive = c.y0 + G::R * j < c.Y;   // strips wholly past the last column sit out stage y
    float et[G::R], ex[G::R], ey[G::R];
#pragma unroll
    for (int r = 0; r < G::R; ++r) et[r] = ex[r] = ey[r] = 0.f;

#pragma unroll 1
    for (int mu = 0; mu <= H; ++mu) {
        x_stage_slide<G>(sG1, sG2, mu, tw);
        __syncthreads();
        if (mu == H && nx) stage_v_async<G>(nx->V, nx->T, nx->X, nx->Y, bnd, nx->t0, nx->x0, nx->y0, sO);
        if (ylive) y_stage_mu<G>(sG2, row, j, mu, sW, tw, et, ex, ey);
        __syncthreads();
    }
    store_outputs<G>(c.E, c.T, c.X, c.Y, c.t0, c.x0, c.y0, row, j, tb.escale, et, ex, ey);
}

// Volumes of one launch: a single volume, or a batch of uneven volumes walked by a
// persistent grid (tile k of the launch belongs to the volume whose tile0 range holds it).
struct EVol {
    const float *V;
    float *E;
    int64_t T, X, Y;
    int64_t tile0;
    int tiles_x, tiles_y;
};
struct EBatch {
    int n, bnd;
    int64_t total;
    EVol v[kMaxBatch];
};

template <class G>
__device__ __forceinline__ TileRef locate_tile(const EBatch &bt, int64_t k)
{
    int lo = 0, hi = bt.n - 1;      // last volume whose first tile is <= k
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bt.v[mid].tile0 <= k) lo = mid; else hi = mid - 1;
    }
    const EVol &v = bt.v[lo];
    const int64_t tile = k - v.tile0;
    const int ty = (int)(tile % v.tiles_y);
    const int tx = (int)((tile / v.tiles_y) % v.tiles_x);
    const int64_t tt = tile / ((int64_t)v.tiles_y * v.tiles_x);
    return TileRef{v.V, v.E, v.T, v.X, v.Y, tt * G::BT, (int64_t)tx * G::BX, (int64_t)ty * G::BY};
}

template <class G>
__global__ void __launch_bounds__(G::NT) energy_fp32_kernel(const __grid_constant__ EBatch bt,
                                                            const __grid_constant__ SpecTables tb)
{
    extern __shared__ __align__(16) float smem[];
    if constexpr (G::MODE == 3) {
        // persistent walk with the next tile's halo prefetched; regions swap every tile
        float *R0 = smem, *R1 = smem + G::NREG, *sW = smem + 2 * G::NREG;
        fill_w<G>(sW, tb);
        int64_t k = blockIdx.x;
        if (k >= bt.total) return;
        TileRef cur = locate_tile<G>(bt, k);
        stage_v_async<G>(cur.V, cur.T, cur.X, cur.Y, bt.bnd, cur.t0, cur.x0, cur.y0, R0);
        int p = 0;
        for (; k < bt.total; k += gridDim.x) {
            const int64_t kn = k + gridDim.x;
            TileRef nxt = cur;
            if (kn < bt.total) nxt = locate_tile<G>(bt, kn);
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
            energy_tile_pf<G>(cur, kn < bt.total ? &nxt : nullptr, bt.bnd, tb, p ? R1 : R0, p ? R0 : R1, sW);
            __syncthreads();
            cur = nxt;
            p ^= 1;
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else {
        for (int64_t k = blockIdx.x; k < bt.total; k += gridDim.x) {
            int lo = 0, hi = bt.n - 1;      // last volume whose first tile is <= k
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (bt.v[mid].tile0 <= k) lo = mid; else hi = mid - 1;
            }
            const EVol &v = bt.v[lo];
            energy_tile_any<G>(v.V, v.T, v.X, v.Y, bt.bnd, k - v.tile0, v.tiles_x, v.tiles_y, v.E, tb, smem);
            __syncthreads();
        }
    }
}

// The same kernel over a device-side list of tiles of one volume (count read on the device),
// e.g. the tiles that a check found wrong; the grid walks the list persistently.
template <class G>
__global__ void __launch_bounds__(G::NT) energy_fp32_list_kernel(const float *__restrict__ V, int64_t T, int64_t X,
                                                                 int64_t Y, int bnd, int tiles_x, int tiles_y,
                                                                 const int64_t *__restrict__ list,
                                                                 const int *__restrict__ count, float *__restrict__ E,
                                                                 const __grid_constant__ SpecTables tb)
{
    extern __shared__ __align__(16) float smem[];
    const int n = *count;
    for (int64_t k = blockIdx.x; k < n; k += gridDim.x) {
        energy_tile<G>(V, T, X, Y, bnd, list[k], tiles_x, tiles_y, E, tb, smem);
        __syncthreads();
    }
}

template <class G>
int64_t energy_tiles(int64_t T, int64_t X, int64_t Y, int *tx, int *ty)
{
    const int64_t nt = (T + G::BT - 1) / G::BT, nx = (X + G::BX - 1) / G::BX, ny = (Y + G::BY - 1) / G::BY;
    *tx = (int)nx;
    *ty = (int)ny;
    return nt * nx * ny;
}

// Launches over `n` volumes.  persistent: grid = resident CTAs of the whole GPU (walks all
// tiles); otherwise one CTA per tile.
template <class G>
cudaError_t launch_energy_impl(const EVolDesc *vols, int n, int bnd, bool persistent, cudaStream_t s)
{
    if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
    SpecTables tb;
    make_tables(G::L, &tb);
    EBatch bt;
    bt.n = n;
    bt.bnd = bnd;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        EVol &v = bt.v[i];
        v.V = vols[i].V;
        v.E = vols[i].E;
        v.T = vols[i].T;
        v.X = vols[i].X;
        v.Y = vols[i].Y;
        v.tile0 = total;
        const int64_t tiles = energy_tiles<G>(v.T, v.X, v.Y, &v.tiles_x, &v.tiles_y);
        if (vols[i].t_hi >= 0) {
            // a range of output planes: tiles are numbered t-major, so the range is contiguous
            if (n != 1 || vols[i].t_lo < 0 || vols[i].t_lo % G::BT != 0 || vols[i].t_hi > v.T ||
                (vols[i].t_hi % G::BT != 0 && vols[i].t_hi != v.T))
                return cudaErrorInvalidValue;
            const int64_t per_t = (int64_t)v.tiles_x * v.tiles_y;
            const int64_t k0 = vols[i].t_lo / G::BT * per_t;
            const int64_t k1 = (vols[i].t_hi + G::BT - 1) / G::BT * per_t;
            v.tile0 = -k0;                        // launch tile k is volume tile k + k0
            total = k1 > k0 ? k1 - k0 : 0;
        } else {
            total += tiles;
        }
    }
    bt.total = total;
    if (total <= 0) return cudaSuccess;
    auto kern = energy_fp32_kernel<G>;
    cudaError_t e = set_smem(kern, G::SMEM);
    if (e != cudaSuccess) return e;
    int64_t grid = total;
    if (persistent || G::MODE == 3) {
        int dev = 0, nsm = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::NT, G::SMEM);
        if (e != cudaSuccess) return e;
        // the occupancy query can answer for a smaller carveout than the launch gets: take
        // the larger of it and the per-SM shared-memory and register limits
        int smem_sm = 0, regs_sm = 0;
        cudaFuncAttributes fa;
        if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) == cudaSuccess &&
            cudaFuncGetAttributes(&fa, kern) == cudaSuccess && fa.numRegs > 0) {
            const int by_smem = smem_sm / (int)(G::SMEM + 1024);
            const int by_regs = regs_sm / (((fa.numRegs + 7) / 8 * 8) * G::NT);
            const int by_threads = 2048 / G::NT;
            int lim = by_smem < by_regs ? by_smem : by_regs;
            lim = lim < by_threads ? lim : by_threads;
            if (lim > per_sm) per_sm = lim;
        }
        const int64_t resident = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
        if (grid > resident) grid = resident;
    }
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    kern<<<(unsigned)grid, G::NT, G::SMEM, s>>>(bt, tb);
    return cudaGetLastError();
}

template <class G>
cudaError_t launch_energy_list_impl(const float *V, sal_dims d, int bnd, const int64_t *list, const int *count, float *E,
                                    cudaStream_t s)
{
    SpecTables tb;
    make_tables(G::L, &tb);
    int tx, ty;
    energy_tiles<G>(d.T, d.X, d.Y, &tx, &ty);
    auto kern = energy_fp32_list_kernel<G>;
    cudaError_t e = set_smem(kern, G::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::NT, G::SMEM);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)(nsm * (per_sm > 0 ? per_sm : 1)), G::NT, G::SMEM, s>>>(V, d.T, d.X, d.Y, bnd, tx, ty, list, count, E,
                                                                         tb);
    return cudaGetLastError();
}

}  // namespace energy_detail
}  // namespace sal
