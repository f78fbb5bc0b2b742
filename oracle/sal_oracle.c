/*
 * Plain FP64 CPU oracle of the seismic saliency method (Shafiq, Long, Alshawi, AlRegib,
 * "Saliency detection for seismic applications using multi-dimensional spectral
 * projections and directional comparisons", ICIP 2017, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this
 * file: only the tests, the smoke check and the benchmark's CPU-baseline leg do.  It
 * shares no code, header, table or helper with the CUDA library; every quantity here is
 * computed from its definition, in double precision, with plain loops and libm.
 *
 * Readings of the paper where it is silent or ambiguous (each is repeated where used):
 *  R1  frequency indices in the projection weights are centred signed indices -h..h
 *      (h = (L-1)/2), so that i = j = k = 0 is the centre of the spectral cube (Sec. 2,
 *      text after Eq. 4) and the weights are symmetric;
 *  R2  features use |F| (the magnitude spectrum); the weights are >= 0, so |F_m| = w_m |F|;
 *  R3  "absolute mean over each local cube" (Sec. 2, third step) is the mean of |F_m| over
 *      the L^3 - 1 non-DC points (the DC point is excluded, text after Eq. 4);
 *  R4  one cube per voxel (stride 1), the voxel at offset h inside its cube, odd L;
 *  R5  samples outside the volume come from a boundary extension: REFLECT (whole-sample
 *      symmetric, edge not repeated: ... c b | a b c d | c b a ...) or PERIODIC (wrap);
 *  R6  Eq. 5 is taken literally, w on the neighbour inside |.|, with Gaussian weights
 *      g(o) = exp(-|o|^2 / (2 sigma^2)); E outside the volume uses the same extension;
 *  R7  neighbourhoods: the 26 voxels around the centre (Q = 26), or the paper's d x 1
 *      line of side d = L along axis m for map m (offsets +-1..+-h, Q = L - 1), or the
 *      d x 1 line along the t-x diagonal of Fig. 3 for every map (offsets (k, k, 0),
 *      k = +-1..+-h, Q = L - 1), or a caller-given list of offsets with explicit weights
 *      per map (the text after Eq. 5 lets orientation, size and weights be tuned; Q is the
 *      number of offsets);
 *  R8  before Eq. 6 each S_m is min-max normalised with global min and max; a map whose
 *      range hi - lo <= eps * max(|hi|, |lo|) is treated as constant and becomes 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_REFLECT 0
#define ORC_PERIODIC 1
#define ORC_STENCIL_26 0
#define ORC_STENCIL_LINE 1
#define ORC_STENCIL_DIAG_TX 2

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* R5: map any integer coordinate i onto 0..n-1. */
long orc_ext_index(long i, long n, int bnd)
{
    if (bnd == ORC_PERIODIC) {
        long r = i % n;
        return r < 0 ? r + n : r;
    }
    if (n == 1) return 0;
    long period = 2 * (n - 1);
    long r = i % period;
    if (r < 0) r += period;
    return r < n ? r : period - r;
}

static double vol_at(const float *V, long T, long X, long Y, int bnd, long t, long x, long y)
{
    long te = orc_ext_index(t, T, bnd), xe = orc_ext_index(x, X, bnd), ye = orc_ext_index(y, Y, bnd);
    return (double)V[(te * X + xe) * Y + ye];
}

/* The local cube f[p][q][r] = V[t-h+p][x-h+q][y-h+r] (R4, R5), with its mean removed.
 * Removing the mean changes no DFT coefficient off DC (the DFT of a constant is zero
 * there); it makes the off-DC spectrum of a constant cube exactly zero in floating point.
 * The DC coefficient is never used (text after Eq. 4). */
static void load_cube(const float *V, long T, long X, long Y, int L, int bnd,
                      long t, long x, long y, double *f)
{
    int h = (L - 1) / 2;
    double s = 0.0;
    for (int p = 0; p < L; ++p)
        for (int q = 0; q < L; ++q)
            for (int r = 0; r < L; ++r) {
                double v = vol_at(V, T, X, Y, bnd, t - h + p, x - h + q, y - h + r);
                f[(p * L + q) * L + r] = v;
                s += v;
            }
    double mean = s / (double)(L * L * L);
    for (int i = 0; i < L * L * L; ++i) f[i] -= mean;
}

/* Centred signed frequency index of storage slot s (R1): s = 0..L-1 -> -h..h. */
static int freq_of_slot(int s, int L) { return s - (L - 1) / 2; }

/* exp(-2 pi i n k / L) with the product reduced mod L first, so the angle is exact. */
static void twiddle(int n, int k, int L, double *c, double *s)
{
    long m = ((long)n * (long)k) % L;
    if (m < 0) m += L;
    double a = -2.0 * ORC_PI * (double)m / (double)L;
    *c = cos(a);
    *s = sin(a);
}

/*
 * |F[mu,nu,omega]| of one local cube by the direct triple sum of the DFT printed in Sec. 2
 * (below Eq. 2):  F = L^-3 sum_{p,q,r} f[p,q,r] exp(-2 pi i (p mu + q nu + r omega) / L).
 * Output mag[(mu+h)][(nu+h)][(omega+h)] for mu, nu, omega in -h..h (R1).  O(L^6).
 */
int oracle_local_spectrum_brute(const float *V, long T, long X, long Y, int L, int bnd,
                                long t, long x, long y, double *mag)
{
    if (L < 1 || (L % 2) == 0) return -1;
    int n3 = L * L * L;
    double *f = (double *)malloc(sizeof(double) * n3);
    if (!f) return -2;
    load_cube(V, T, X, Y, L, bnd, t, x, y, f);
    double inv = 1.0 / (double)n3;
    for (int a = 0; a < L; ++a)
        for (int b = 0; b < L; ++b)
            for (int c = 0; c < L; ++c) {
                int mu = freq_of_slot(a, L), nu = freq_of_slot(b, L), om = freq_of_slot(c, L);
                double re = 0.0, im = 0.0;
                for (int p = 0; p < L; ++p)
                    for (int q = 0; q < L; ++q)
                        for (int r = 0; r < L; ++r) {
                            long m = ((long)p * mu + (long)q * nu + (long)r * om) % L;
                            if (m < 0) m += L;
                            double ang = -2.0 * ORC_PI * (double)m / (double)L;
                            double v = f[(p * L + q) * L + r];
                            re += v * cos(ang);
                            im += v * sin(ang);
                        }
                mag[(a * L + b) * L + c] = sqrt(re * re + im * im) * inv;
            }
    /* DC slot: the mean was removed, so report the DC magnitude of the original cube. */
    {
        int h = (L - 1) / 2;
        double s = 0.0;
        for (int p = 0; p < L; ++p)
            for (int q = 0; q < L; ++q)
                for (int r = 0; r < L; ++r)
                    s += vol_at(V, T, X, Y, bnd, t - h + p, x - h + q, y - h + r);
        mag[(h * L + h) * L + h] = fabs(s) * inv;
    }
    free(f);
    return 0;
}

/*
 * The same spectrum with the DFT applied one axis at a time (the transform is separable:
 * the exponential factors into one term per axis).  Stage 1 along t, stage 2 along x,
 * stage 3 along y; each stage is a product with the L x L DFT matrix.  O(3 L^4).
 */
static void spectrum_separable_from_cube(const double *f, int L, double *mag)
{
    int n3 = L * L * L;
    double *g1r = (double *)calloc(n3, sizeof(double)), *g1i = (double *)calloc(n3, sizeof(double));
    double *g2r = (double *)calloc(n3, sizeof(double)), *g2i = (double *)calloc(n3, sizeof(double));
    double *cs = (double *)malloc(sizeof(double) * L * L), *sn = (double *)malloc(sizeof(double) * L * L);
    for (int a = 0; a < L; ++a)
        for (int p = 0; p < L; ++p) twiddle(freq_of_slot(a, L), p, L, &cs[a * L + p], &sn[a * L + p]);
    /* stage 1: G1[mu][q][r] = sum_p f[p][q][r] e^{-2 pi i p mu / L} */
    for (int a = 0; a < L; ++a)
        for (int q = 0; q < L; ++q)
            for (int r = 0; r < L; ++r) {
                double re = 0.0, im = 0.0;
                for (int p = 0; p < L; ++p) {
                    double v = f[(p * L + q) * L + r];
                    re += v * cs[a * L + p];
                    im += v * sn[a * L + p];
                }
                g1r[(a * L + q) * L + r] = re;
                g1i[(a * L + q) * L + r] = im;
            }
    /* stage 2: G2[mu][nu][r] = sum_q G1[mu][q][r] e^{-2 pi i q nu / L} */
    for (int a = 0; a < L; ++a)
        for (int b = 0; b < L; ++b)
            for (int r = 0; r < L; ++r) {
                double re = 0.0, im = 0.0;
                for (int q = 0; q < L; ++q) {
                    double xr = g1r[(a * L + q) * L + r], xi = g1i[(a * L + q) * L + r];
                    double c = cs[b * L + q], s = sn[b * L + q];
                    re += xr * c - xi * s;
                    im += xr * s + xi * c;
                }
                g2r[(a * L + b) * L + r] = re;
                g2i[(a * L + b) * L + r] = im;
            }
    /* stage 3: F[mu][nu][omega] = L^-3 sum_r G2[mu][nu][r] e^{-2 pi i r omega / L} */
    double inv = 1.0 / (double)n3;
    for (int a = 0; a < L; ++a)
        for (int b = 0; b < L; ++b)
            for (int c3 = 0; c3 < L; ++c3) {
                double re = 0.0, im = 0.0;
                for (int r = 0; r < L; ++r) {
                    double xr = g2r[(a * L + b) * L + r], xi = g2i[(a * L + b) * L + r];
                    double c = cs[c3 * L + r], s = sn[c3 * L + r];
                    re += xr * c - xi * s;
                    im += xr * s + xi * c;
                }
                mag[(a * L + b) * L + c3] = sqrt(re * re + im * im) * inv;
            }
    free(g1r); free(g1i); free(g2r); free(g2i); free(cs); free(sn);
}

int oracle_local_spectrum_separable(const float *V, long T, long X, long Y, int L, int bnd,
                                    long t, long x, long y, double *mag)
{
    if (L < 1 || (L % 2) == 0) return -1;
    int n3 = L * L * L, h = (L - 1) / 2;
    double *f = (double *)malloc(sizeof(double) * n3);
    if (!f) return -2;
    load_cube(V, T, X, Y, L, bnd, t, x, y, f);
    spectrum_separable_from_cube(f, L, mag);
    double s = 0.0;
    for (int p = 0; p < L; ++p)
        for (int q = 0; q < L; ++q)
            for (int r = 0; r < L; ++r) s += vol_at(V, T, X, Y, bnd, t - h + p, x - h + q, y - h + r);
    mag[(h * L + h) * L + h] = fabs(s) / (double)n3;
    free(f);
    return 0;
}

/*
 * Projection weights of Eq. 1-4, stored w[m][(mu+h)][(nu+h)][(omega+h)] for m = t, x, y:
 *   w_t = sqrt(nu^2 + omega^2) / rho,  w_x = sqrt(mu^2 + omega^2) / rho,
 *   w_y = sqrt(mu^2 + nu^2) / rho,     rho = sqrt(mu^2 + nu^2 + omega^2)
 * (i, j, k of the paper are mu, nu, omega here, reading R1).  The DC point, where the
 * ratios are 0/0, gets weight 0: it is excluded from the features (text after Eq. 4).
 */
void oracle_weights(int L, double *w)
{
    int n3 = L * L * L;
    for (int a = 0; a < L; ++a)
        for (int b = 0; b < L; ++b)
            for (int c = 0; c < L; ++c) {
                double i = freq_of_slot(a, L), j = freq_of_slot(b, L), k = freq_of_slot(c, L);
                int idx = (a * L + b) * L + c;
                double rho = sqrt(i * i + j * j + k * k);
                if (rho == 0.0) {
                    w[idx] = w[n3 + idx] = w[2 * n3 + idx] = 0.0;
                } else {
                    w[idx] = sqrt(j * j + k * k) / rho;
                    w[n3 + idx] = sqrt(i * i + k * k) / rho;
                    w[2 * n3 + idx] = sqrt(i * i + j * j) / rho;
                }
            }
}

/* Spectral energies (Sec. 2, third step, readings R2, R3): E_m = (L^3-1)^-1 sum_{!=DC} w_m |F|. */
void oracle_project(const double *mag, long n_vox, int L, double *E)
{
    int n3 = L * L * L;
    double *w = (double *)malloc(sizeof(double) * 3 * n3);
    oracle_weights(L, w);
    int h = (L - 1) / 2, dc = (h * L + h) * L + h;
    for (long v = 0; v < n_vox; ++v)
        for (int m = 0; m < 3; ++m) {
            double s = 0.0;
            for (int i = 0; i < n3; ++i)
                if (i != dc) s += w[m * n3 + i] * mag[v * n3 + i];
            E[m * n_vox + v] = s / (double)(n3 - 1);
        }
    free(w);
}

/*
 * E_t, E_x, E_y for every voxel of V (steps one to three of Sec. 2).  E is [3][T*X*Y].
 * `brute` selects the direct DFT sum; otherwise the separable one.  OpenMP over t.
 */
int oracle_energy(const float *V, long T, long X, long Y, int L, int bnd, int brute,
                  int nthreads, double *E)
{
    if (L < 1 || (L % 2) == 0 || T < 1 || X < 1 || Y < 1) return -1;
    long N = T * X * Y;
    int n3 = L * L * L, h = (L - 1) / 2, dc = (h * L + h) * L + h;
    double *w = (double *)malloc(sizeof(double) * 3 * n3);
    oracle_weights(L, w);
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (long t = 0; t < T; ++t) {
        double *mag = (double *)malloc(sizeof(double) * n3);
        for (long x = 0; x < X; ++x)
            for (long y = 0; y < Y; ++y) {
                int rc = brute ? oracle_local_spectrum_brute(V, T, X, Y, L, bnd, t, x, y, mag)
                               : oracle_local_spectrum_separable(V, T, X, Y, L, bnd, t, x, y, mag);
                if (rc) err = rc;
                long v = (t * X + x) * Y + y;
                for (int m = 0; m < 3; ++m) {
                    double s = 0.0;
                    for (int i = 0; i < n3; ++i)
                        if (i != dc) s += w[m * n3 + i] * mag[i];
                    E[m * N + v] = s / (double)(n3 - 1);
                }
            }
        free(mag);
    }
    free(w);
    return err;
}

/* E_m at selected voxels only (separable DFT), for checks on volumes too large to sweep. */
int oracle_energy_at(const float *V, long T, long X, long Y, int L, int bnd,
                     const int64_t *coords /* [n][3] */, long n, int nthreads, double *E /* [3][n] */)
{
    if (L < 1 || (L % 2) == 0) return -1;
    int n3 = L * L * L, h = (L - 1) / 2, dc = (h * L + h) * L + h;
    double *w = (double *)malloc(sizeof(double) * 3 * n3);
    oracle_weights(L, w);
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
    for (long k = 0; k < n; ++k) {
        double *mag = (double *)malloc(sizeof(double) * n3);
        oracle_local_spectrum_separable(V, T, X, Y, L, bnd, coords[3 * k], coords[3 * k + 1],
                                        coords[3 * k + 2], mag);
        for (int m = 0; m < 3; ++m) {
            double s = 0.0;
            for (int i = 0; i < n3; ++i)
                if (i != dc) s += w[m * n3 + i] * mag[i];
            E[m * n + k] = s / (double)(n3 - 1);
        }
        free(mag);
    }
    free(w);
    return 0;
}

/*
 * Coarse-stride cubes (Sec. 2, first step: the local cube slides "with more than 50 %
 * overlap"; reading R4 with a stride s > 1).  Along an axis of n samples the cube centres
 * form the lattice c_i = min(i s, n - 1), i = 0 .. n_c - 1, n_c = ceil((n - 1) / s) + 1: step
 * s, and the last sample always a centre, so every voxel lies between two centres.
 */
long oracle_lattice_size(long n, int s) { return n <= 1 ? 1 : (n - 2) / s + 2; }

static long lattice_coord(long i, long n, int s)
{
    long c = i * (long)s;
    return c < n - 1 ? c : n - 1;
}

/* Ec [3][Tc][Xc][Yc]: E_m of the cube centred on every lattice point (separable DFT). */
int oracle_energy_lattice(const float *V, long T, long X, long Y, int L, int bnd, int s, int nthreads, double *Ec)
{
    if (L < 1 || (L % 2) == 0 || s < 1) return -1;
    long Tc = oracle_lattice_size(T, s), Xc = oracle_lattice_size(X, s), Yc = oracle_lattice_size(Y, s);
    long Nc = Tc * Xc * Yc;
    int64_t *coords = (int64_t *)malloc(sizeof(int64_t) * 3 * Nc);
    for (long i = 0; i < Tc; ++i)
        for (long j = 0; j < Xc; ++j)
            for (long k = 0; k < Yc; ++k) {
                long v = (i * Xc + j) * Yc + k;
                coords[3 * v] = lattice_coord(i, T, s);
                coords[3 * v + 1] = lattice_coord(j, X, s);
                coords[3 * v + 2] = lattice_coord(k, Y, s);
            }
    int rc = oracle_energy_at(V, T, X, Y, L, bnd, coords, Nc, nthreads, Ec);
    free(coords);
    return rc;
}

/* The two lattice centres around coordinate v and v's fraction of the way between them. */
static void lattice_segment(long v, long n, int s, long *i0, double *f)
{
    long nc = oracle_lattice_size(n, s);
    if (nc == 1) {
        *i0 = 0;
        *f = 0.0;
        return;
    }
    long i = v / s;
    if (i > nc - 2) i = nc - 2;
    long lo = lattice_coord(i, n, s), hi = lattice_coord(i + 1, n, s);
    *i0 = i;
    *f = (double)(v - lo) / (double)(hi - lo);
}

/* Trilinear interpolation of lattice values Ec [C][Tc][Xc][Yc] back to every voxel: out [C][T][X][Y]. */
void oracle_interp_lattice(const double *Ec, int C, long T, long X, long Y, int s, double *out)
{
    long Tc = oracle_lattice_size(T, s), Xc = oracle_lattice_size(X, s), Yc = oracle_lattice_size(Y, s);
    long N = T * X * Y, Nc = Tc * Xc * Yc;
    for (int m = 0; m < C; ++m)
        for (long t = 0; t < T; ++t)
            for (long x = 0; x < X; ++x)
                for (long y = 0; y < Y; ++y) {
                    long i, j, k;
                    double ft, fx, fy;
                    lattice_segment(t, T, s, &i, &ft);
                    lattice_segment(x, X, s, &j, &fx);
                    lattice_segment(y, Y, s, &k, &fy);
                    double acc = 0.0;
                    for (int a = 0; a < 2; ++a)
                        for (int b = 0; b < 2; ++b)
                            for (int c = 0; c < 2; ++c) {
                                double wgt = (a ? ft : 1.0 - ft) * (b ? fx : 1.0 - fx) * (c ? fy : 1.0 - fy);
                                if (wgt == 0.0) continue;   /* also keeps the index inside a 1-point lattice */
                                acc += wgt * Ec[m * Nc + ((i + a) * Xc + (j + b)) * Yc + (k + c)];
                            }
                    out[m * N + (t * X + x) * Y + y] = acc;
                }
}

/* E of every voxel with cubes on the lattice of stride s, interpolated back (s = 1: oracle_energy). */
int oracle_energy_strided(const float *V, long T, long X, long Y, int L, int bnd, int s, int nthreads, double *E)
{
    long Nc = oracle_lattice_size(T, s) * oracle_lattice_size(X, s) * oracle_lattice_size(Y, s);
    double *Ec = (double *)malloc(sizeof(double) * 3 * Nc);
    int rc = oracle_energy_lattice(V, T, X, Y, L, bnd, s, nthreads, Ec);
    if (!rc) oracle_interp_lattice(Ec, 3, T, X, Y, s, E);
    free(Ec);
    return rc;
}

/* Offsets of the neighbourhood of map m (reading R7); returns Q. */
static int neighbourhood(int stencil, int m, int L, int off[][3])
{
    int Q = 0;
    if (stencil == ORC_STENCIL_26) {
        for (int a = -1; a <= 1; ++a)
            for (int b = -1; b <= 1; ++b)
                for (int c = -1; c <= 1; ++c) {
                    if (a == 0 && b == 0 && c == 0) continue;
                    off[Q][0] = a; off[Q][1] = b; off[Q][2] = c; ++Q;
                }
    } else if (stencil == ORC_STENCIL_DIAG_TX) {
        int h = (L - 1) / 2;
        for (int k = -h; k <= h; ++k) {
            if (k == 0) continue;
            off[Q][0] = k;
            off[Q][1] = k;
            off[Q][2] = 0;
            ++Q;
        }
    } else {
        int h = (L - 1) / 2;
        for (int k = -h; k <= h; ++k) {
            if (k == 0) continue;
            off[Q][0] = off[Q][1] = off[Q][2] = 0;
            off[Q][m] = k;
            ++Q;
        }
    }
    return Q;
}

/*
 * Directional centre-surround comparison, Eq. 5 (reading R6):
 *   S_m[v] = Q^-1 sum_{o in N_m} | E_m[v] - g(o) E_m[v + o] |,  g(o) = exp(-|o|^2 / (2 sigma^2)).
 * E and Sm are [3][T*X*Y].
 */
int oracle_dcs(const double *E, long T, long X, long Y, int bnd, int stencil, int L,
               double sigma, int nthreads, double *Sm)
{
    if (T < 1 || X < 1 || Y < 1 || sigma <= 0.0) return -1;
    if (stencil != ORC_STENCIL_26 && (L < 3 || (L % 2) == 0)) return -1;
    long N = T * X * Y;
    for (int m = 0; m < 3; ++m) {
        int off[64][3];
        int Q = neighbourhood(stencil, m, L, off);
        double g[64];
        for (int k = 0; k < Q; ++k) {
            double d2 = (double)(off[k][0] * off[k][0] + off[k][1] * off[k][1] + off[k][2] * off[k][2]);
            g[k] = exp(-d2 / (2.0 * sigma * sigma));
        }
        const double *Em = E + m * N;
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1)
        for (long t = 0; t < T; ++t)
            for (long x = 0; x < X; ++x)
                for (long y = 0; y < Y; ++y) {
                    double c = Em[(t * X + x) * Y + y];
                    double s = 0.0;
                    for (int k = 0; k < Q; ++k) {
                        long tn = orc_ext_index(t + off[k][0], T, bnd);
                        long xn = orc_ext_index(x + off[k][1], X, bnd);
                        long yn = orc_ext_index(y + off[k][2], Y, bnd);
                        s += fabs(c - g[k] * Em[(tn * X + xn) * Y + yn]);
                    }
                    Sm[m * N + (t * X + x) * Y + y] = s / (double)Q;
                }
    }
    return 0;
}

/*
 * Eq. 5 with a caller-given neighbourhood per map (reading R7, user stencils):
 *   S_m[v] = Q_m^-1 sum_{k < Q_m} | E_m[v] - w_m[k] E_m[v + o_m[k]] |
 * off is [3][qmax][3] (dt, dx, dy), w is [3][qmax], Q[m] the number of offsets of map m.
 * E outside the volume comes from the boundary extension, as for the built-in stencils.
 */
int oracle_dcs_user(const double *E, long T, long X, long Y, int bnd, const int *Q, const int *off,
                    const double *w, int qmax, int nthreads, double *Sm)
{
    if (T < 1 || X < 1 || Y < 1 || qmax < 1) return -1;
    for (int m = 0; m < 3; ++m)
        if (Q[m] < 1 || Q[m] > qmax) return -1;
    long N = T * X * Y;
    for (int m = 0; m < 3; ++m) {
        const double *Em = E + m * N;
        const int *o = off + (long)m * qmax * 3;
        const double *wm = w + (long)m * qmax;
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1)
        for (long t = 0; t < T; ++t)
            for (long x = 0; x < X; ++x)
                for (long y = 0; y < Y; ++y) {
                    double c = Em[(t * X + x) * Y + y];
                    double s = 0.0;
                    for (int k = 0; k < Q[m]; ++k) {
                        long tn = orc_ext_index(t + o[3 * k], T, bnd);
                        long xn = orc_ext_index(x + o[3 * k + 1], X, bnd);
                        long yn = orc_ext_index(y + o[3 * k + 2], Y, bnd);
                        s += fabs(c - wm[k] * Em[(tn * X + xn) * Y + yn]);
                    }
                    Sm[m * N + (t * X + x) * Y + y] = s / (double)Q[m];
                }
    }
    return 0;
}

/* Global min, max and sum of each S_m: stats[3m + 0..2]. */
void oracle_stats(const double *Sm, long N, double *stats)
{
    for (int m = 0; m < 3; ++m) {
        double lo = Sm[m * N], hi = Sm[m * N], s = 0.0;
        for (long v = 0; v < N; ++v) {
            double a = Sm[m * N + v];
            if (a < lo) lo = a;
            if (a > hi) hi = a;
            s += a;
        }
        stats[3 * m] = lo;
        stats[3 * m + 1] = hi;
        stats[3 * m + 2] = s;
    }
}

/* Eq. 6 on min-max normalised maps (reading R8): S = a N_t + b N_x + c N_y. */
void oracle_combine(const double *Sm, const double *stats, long N, double a, double b, double c,
                    double eps, double *S)
{
    double wts[3] = {a, b, c};
    double lo[3], scale[3];
    for (int m = 0; m < 3; ++m) {
        double l = stats[3 * m], hgh = stats[3 * m + 1];
        double mag = fabs(hgh) > fabs(l) ? fabs(hgh) : fabs(l);
        lo[m] = l;
        scale[m] = (hgh - l) <= eps * mag ? 0.0 : 1.0 / (hgh - l);
    }
    for (long v = 0; v < N; ++v) {
        double s = 0.0;
        for (int m = 0; m < 3; ++m) s += wts[m] * (Sm[m * N + v] - lo[m]) * scale[m];
        S[v] = s;
    }
}

/* The whole method (Fig. 1): energies, DCS, normalisation and Eq. 6.  Optional outputs may be NULL. */
int oracle_saliency(const float *V, long T, long X, long Y, int L, int bnd, int stencil,
                    double sigma, double a, double b, double c, double eps, int nthreads,
                    double *S, double *E_out, double *Sm_out, double *stats_out)
{
    long N = T * X * Y;
    double *E = E_out ? E_out : (double *)malloc(sizeof(double) * 3 * N);
    double *Sm = Sm_out ? Sm_out : (double *)malloc(sizeof(double) * 3 * N);
    double st[9];
    int rc = oracle_energy(V, T, X, Y, L, bnd, 0, nthreads, E);
    if (!rc) rc = oracle_dcs(E, T, X, Y, bnd, stencil, L, sigma, nthreads, Sm);
    if (!rc) {
        oracle_stats(Sm, N, st);
        oracle_combine(Sm, st, N, a, b, c, eps, S);
        if (stats_out) memcpy(stats_out, st, sizeof(st));
    }
    if (!E_out) free(E);
    if (!Sm_out) free(Sm);
    return rc;
}

/* The whole method with cubes on the lattice of stride s (E interpolated back to every
 * voxel before Eq. 5); s = 1 is oracle_saliency. */
int oracle_saliency_strided(const float *V, long T, long X, long Y, int L, int bnd, int stencil, int s,
                            double sigma, double a, double b, double c, double eps, int nthreads,
                            double *S, double *E_out, double *Sm_out, double *stats_out)
{
    long N = T * X * Y;
    double *E = E_out ? E_out : (double *)malloc(sizeof(double) * 3 * N);
    double *Sm = Sm_out ? Sm_out : (double *)malloc(sizeof(double) * 3 * N);
    double st[9];
    int rc = oracle_energy_strided(V, T, X, Y, L, bnd, s, nthreads, E);
    if (!rc) rc = oracle_dcs(E, T, X, Y, bnd, stencil, L, sigma, nthreads, Sm);
    if (!rc) {
        oracle_stats(Sm, N, st);
        oracle_combine(Sm, st, N, a, b, c, eps, S);
        if (stats_out) memcpy(stats_out, st, sizeof(st));
    }
    if (!E_out) free(E);
    if (!Sm_out) free(Sm);
    return rc;
}

/* E_m and S_m (Eq. 5) at selected voxels only: the energies of each voxel's neighbours are
 * computed from their own cubes, so no full-volume sweep is needed.  For checks on
 * volumes too large for the whole-volume oracle. */
int oracle_maps_at(const float *V, long T, long X, long Y, int L, int bnd, int stencil, double sigma,
                   const int64_t *coords /* [n][3] */, long n, int nthreads, double *E /* [3][n] */,
                   double *Sm /* [3][n] */)
{
    if (L < 3 || (L % 2) == 0 || sigma <= 0.0) return -1;
    int n3 = L * L * L, h = (L - 1) / 2, dc = (h * L + h) * L + h;
    double *w = (double *)malloc(sizeof(double) * 3 * n3);
    oracle_weights(L, w);
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
    for (long k = 0; k < n; ++k) {
        double *mag = (double *)malloc(sizeof(double) * n3);
        long t = coords[3 * k], x = coords[3 * k + 1], y = coords[3 * k + 2];
        for (int m = 0; m < 3; ++m) {
            int off[64][3];
            int Q = neighbourhood(stencil, m, L, off);
            double e[65];
            for (int q = 0; q <= Q; ++q) {
                long tn = t, xn = x, yn = y;
                if (q < Q) {
                    tn = orc_ext_index(t + off[q][0], T, bnd);
                    xn = orc_ext_index(x + off[q][1], X, bnd);
                    yn = orc_ext_index(y + off[q][2], Y, bnd);
                }
                oracle_local_spectrum_separable(V, T, X, Y, L, bnd, tn, xn, yn, mag);
                double s = 0.0;
                for (int i = 0; i < n3; ++i)
                    if (i != dc) s += w[m * n3 + i] * mag[i];
                e[q] = s / (double)(n3 - 1);
            }
            double c = e[Q], s = 0.0;
            for (int q = 0; q < Q; ++q) {
                double d2 = (double)(off[q][0] * off[q][0] + off[q][1] * off[q][1] + off[q][2] * off[q][2]);
                s += fabs(c - exp(-d2 / (2.0 * sigma * sigma)) * e[q]);
            }
            E[m * n + k] = c;
            Sm[m * n + k] = s / (double)Q;
        }
        free(mag);
    }
    free(w);
    return 0;
}

/* ==== Learned surrogate: plain FP64 reference of its layers (test infrastructure) ====
 * A 3x3x3 convolution (cross-correlation, as the layers compute it) with bias, the GELU
 * activation x * Phi(x) (Phi the standard normal CDF, via erf), and the gradients of both
 * by the chain rule.  Arrays are planar [C][T][X][Y]; weights [Cout][Cin][3][3][3].  Samples
 * outside the volume come from the same boundary extension as the method (R5). */

void oracle_conv3d(const double *in, long T, long X, long Y, int cin, int cout, const double *w,
                   const double *b, int bnd, double *out)
{
    long N = T * X * Y;
#pragma omp parallel for
    for (long t = 0; t < T; ++t)
        for (long x = 0; x < X; ++x)
            for (long y = 0; y < Y; ++y)
                for (int co = 0; co < cout; ++co) {
                    double s = b ? b[co] : 0.0;
                    for (int ci = 0; ci < cin; ++ci)
                        for (int a = 0; a < 3; ++a)
                            for (int c = 0; c < 3; ++c)
                                for (int d = 0; d < 3; ++d) {
                                    long tt = orc_ext_index(t + a - 1, T, bnd), xx = orc_ext_index(x + c - 1, X, bnd),
                                         yy = orc_ext_index(y + d - 1, Y, bnd);
                                    s += w[(((long)co * cin + ci) * 3 + a) * 9 + c * 3 + d] *
                                         in[ci * N + (tt * X + xx) * Y + yy];
                                }
                    out[co * N + (t * X + x) * Y + y] = s;
                }
}

double oracle_gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
double oracle_gelu_grad(double x)
{
    const double phi = exp(-0.5 * x * x) / sqrt(2.0 * ORC_PI);
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * phi;
}

/* Gradients of out = conv(in) w.r.t. weights, bias and input, given gout = dL/dout.
 * gin may be NULL.  Accumulates nothing: every output is overwritten. */
void oracle_conv3d_grad(const double *in, long T, long X, long Y, int cin, int cout, const double *w,
                        int bnd, const double *gout, double *gw, double *gb, double *gin)
{
    long N = T * X * Y;
    for (int i = 0; i < cout * cin * 27; ++i) gw[i] = 0.0;
    for (int co = 0; co < cout; ++co) gb[co] = 0.0;
    if (gin)
        for (long i = 0; i < (long)cin * N; ++i) gin[i] = 0.0;
    for (long t = 0; t < T; ++t)
        for (long x = 0; x < X; ++x)
            for (long y = 0; y < Y; ++y)
                for (int co = 0; co < cout; ++co) {
                    double g = gout[co * N + (t * X + x) * Y + y];
                    gb[co] += g;
                    for (int ci = 0; ci < cin; ++ci)
                        for (int a = 0; a < 3; ++a)
                            for (int c = 0; c < 3; ++c)
                                for (int d = 0; d < 3; ++d) {
                                    long tt = orc_ext_index(t + a - 1, T, bnd), xx = orc_ext_index(x + c - 1, X, bnd),
                                         yy = orc_ext_index(y + d - 1, Y, bnd);
                                    long wi = (((long)co * cin + ci) * 3 + a) * 9 + c * 3 + d;
                                    long ii = ci * N + (tt * X + xx) * Y + yy;
                                    gw[wi] += g * in[ii];
                                    if (gin) gin[ii] += g * w[wi];
                                }
                }
}

/* The surrogate network: n layers of 3x3x3 convolution, GELU after all but the last.
 * widths[0..n] are the channel counts (widths[0] = 1 input, widths[n] = 3 outputs);
 * params holds, layer by layer, the weights then the biases.  acts (optional) receives
 * every layer's pre-activation, [sum of widths[1..n]][N]. */
int oracle_surrogate_forward(const double *x, long T, long X, long Y, int n, const int *widths,
                             const double *params, int bnd, double *out, double *acts)
{
    long N = T * X * Y;
    int wmax = 0;
    for (int l = 0; l <= n; ++l) wmax = widths[l] > wmax ? widths[l] : wmax;
    double *a = (double *)malloc(sizeof(double) * wmax * N), *z = (double *)malloc(sizeof(double) * wmax * N);
    memcpy(a, x, sizeof(double) * widths[0] * N);
    const double *p = params;
    long aoff = 0;
    for (int l = 0; l < n; ++l) {
        const double *w = p, *b = p + (long)widths[l + 1] * widths[l] * 27;
        p = b + widths[l + 1];
        oracle_conv3d(a, T, X, Y, widths[l], widths[l + 1], w, b, bnd, z);
        if (acts) memcpy(acts + aoff, z, sizeof(double) * widths[l + 1] * N);
        aoff += (long)widths[l + 1] * N;
        if (l + 1 < n) {
            for (long i = 0; i < (long)widths[l + 1] * N; ++i) a[i] = oracle_gelu(z[i]);
        } else {
            memcpy(out, z, sizeof(double) * widths[l + 1] * N);
        }
    }
    free(a);
    free(z);
    return 0;
}

/* Gradient of L = sum over outputs of 0.5 * mask * (out - target)^2 w.r.t. every parameter
 * (same layout as params).  mask may be NULL (all ones).  Returns L. */
double oracle_surrogate_loss_grad(const double *x, long T, long X, long Y, int n, const int *widths,
                                  const double *params, int bnd, const double *target, const double *mask,
                                  double *grads)
{
    long N = T * X * Y;
    long tot = 0;
    for (int l = 0; l < n; ++l) tot += widths[l + 1];
    double *acts = (double *)malloc(sizeof(double) * tot * N);
    double *out = (double *)malloc(sizeof(double) * widths[n] * N);
    oracle_surrogate_forward(x, T, X, Y, n, widths, params, bnd, out, acts);
    int wmax = 0;
    for (int l = 0; l <= n; ++l) wmax = widths[l] > wmax ? widths[l] : wmax;
    double *g = (double *)malloc(sizeof(double) * wmax * N), *gin = (double *)malloc(sizeof(double) * wmax * N);
    double *a = (double *)malloc(sizeof(double) * wmax * N);
    double loss = 0.0;
    for (long i = 0; i < (long)widths[n] * N; ++i) {
        double m = mask ? mask[i % N] : 1.0, d = out[i] - target[i];
        loss += 0.5 * m * d * d;
        g[i] = m * d;
    }
    /* parameter offsets per layer */
    long offs[64];
    long o = 0;
    for (int l = 0; l < n; ++l) {
        offs[l] = o;
        o += (long)widths[l + 1] * widths[l] * 27 + widths[l + 1];
    }
    long aoff_end = tot * N;
    for (int l = n - 1; l >= 0; --l) {
        long aoff = aoff_end - (long)widths[l + 1] * N;      /* this layer's pre-activation */
        /* the layer's input: x for l = 0, else GELU of the previous pre-activation */
        if (l == 0) {
            memcpy(a, x, sizeof(double) * widths[0] * N);
        } else {
            long poff = aoff - (long)widths[l] * N;
            for (long i = 0; i < (long)widths[l] * N; ++i) a[i] = oracle_gelu(acts[poff + i]);
        }
        const double *w = params + offs[l];
        double *gw = grads + offs[l], *gb = gw + (long)widths[l + 1] * widths[l] * 27;
        oracle_conv3d_grad(a, T, X, Y, widths[l], widths[l + 1], w, bnd, g, gw, gb, l > 0 ? gin : NULL);
        if (l > 0) {
            long poff = aoff - (long)widths[l] * N;
            for (long i = 0; i < (long)widths[l] * N; ++i) g[i] = gin[i] * oracle_gelu_grad(acts[poff + i]);
        }
        aoff_end = aoff;
    }
    free(acts);
    free(out);
    free(g);
    free(gin);
    free(a);
    return loss;
}
