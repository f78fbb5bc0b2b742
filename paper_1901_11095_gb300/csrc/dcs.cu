// Directional centre-surround comparison (Eq. 5), the FP64 global statistics of the
// S_m maps, and the normalised weighted combination of Eq. 6.
//
//   S_m[v] = Q^-1 sum_{o in N_m} | E_m[v] - g(o) E_m[v + o] |,  g(o) = exp(-|o|^2 / (2 sigma^2))
//
// N_m is the 26-neighbourhood, the d x 1 line of side d = L along axis m (Sec. 2 text
// after Eq. 5), the t-x diagonal line of Fig. 3 or a caller-given offset list.  E outside
// the volume comes from the boundary extension.  A CTA walks a chunk of planes along t for
// one 8 x 64 column block, the halo planes of E_m passing through a ring of shared-memory
// slots (each value read from HBM about once); every thread produces 4 x 4 outputs per step
// (4 planes, 4 consecutive columns along y), and the CTA reduces its min, max and sum (warp
// shuffles, then FP64 across warps) into one partial record per chunk; two small passes
// finish the FP64 reduction.
#include <float.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "sal_internal.cuh"

namespace sal {

namespace {

// Column block of one CTA and the step along t: DT planes x DX rows x DY columns.  Every
// thread owns a 4 x 4 block (4 planes along t, 4 columns along y) at one x.
constexpr int DT = 8, DX = 8, DY = 64, QT = 4, QY = 4;
constexpr int DNT = (DT / QT) * DX * (DY / QY);         // 256 threads
constexpr int kRedBlocks = 160;                         // first pass of the partial reduction

struct DcsConsts {
    float g[4];            // 26-neighbourhood weights for |o|^2 = 0 (unused), 1, 2, 3
    float gl[kMaxH + 1];   // line weights for offset k = 0..h
    float invQ;
    int h;
};

// Halo geometry of one map: radii along t, x, y and the shared-memory pitches.  Column c
// of the halo row (c = 0 is y0 - ry) is stored at c + off, with off chosen so that the
// tile's first output column y0 lands on a 16-byte boundary.
struct Halo {
    int rt, rx, ry, PX, PP, off, pitch, planes;
    __host__ __device__ constexpr Halo(int rt_, int rx_, int ry_)
        : rt(rt_), rx(rx_), ry(ry_), PX(0), PP(0), off(0), pitch(0), planes(0)
    {
        PX = DX + 2 * rx_;
        off = ((ry_ + 3) & ~3) - ry_;
        pitch = (off + DY + 2 * ry_ + 3) & ~3;
        PP = PX * pitch;
        planes = DT + 2 * rt_;
    }
    // shared memory of a ring holding the step's planes and the next step's DT planes
    __host__ __device__ constexpr int ring_floats() const { return (planes + DT) * PP; }
};

__host__ __device__ inline Halo halo_for(int stencil, int m, int h)
{
    if (stencil == SAL_STENCIL_26) return Halo(1, 1, 1);
    return Halo(m == 0 ? h : 0, m == 1 ? h : 0, m == 2 ? h : 0);
}

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

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }


// Volumes of one launch; work item k of the launch is (volume, map, record), map-major
// within each volume (a record: one chunk of SC planes of one column block).  Output planes [o_lo, o_hi) of E's T planes (the whole volume unless
// the launch serves a slab).
struct DVol {
    const float *E;
    float *Sm;
    double *part;          // [9][tiles] records of this volume (tiles = records per map)
    int64_t T, X, Y;
    int64_t o_lo, o_hi;
    int64_t item0, tiles;
    int tiles_x, tiles_y;
};
struct DBatch {
    int n, bnd;
    int64_t total;
    DVol v[kMaxBatch];
};

__device__ __forceinline__ const DVol &find_volume(const DBatch &bt, int64_t it)
{
    int lo = 0, hi = bt.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bt.v[mid].item0 <= it) lo = mid; else hi = mid - 1;
    }
    return bt.v[lo];
}

// ---- 26-neighbourhood, planes streamed along t ------------------------------------------
// One work item = (volume, map, chunk of SC planes along t, 8 x 64 column block (x, y)).  The
// CTA walks its chunk in steps of DT = 8 output planes.  The halo planes of E_m (10 rows x
// 66 columns each) pass through a ring of RING plane slots in shared memory: the 8 planes of
// the next step are copied asynchronously while the current step is computed, each halo
// value is read once per chunk (plus the two boundary planes of the chunk), and the boundary
// extension and index set-up are paid once per item instead of once per copy.
constexpr int SC = 128;                         // output planes per chunk
constexpr int RING = 18;                        // plane slots: 10 being read + 8 in flight
constexpr int PROW = 72;                        // slot row pitch (floats); halo column c at c + 3
constexpr int PSLOT = (DX + 2) * PROW;          // one plane slot (floats)
constexpr int PEL = (DX + 2) * (DY + 2);        // halo elements of one plane
constexpr int KEL = (PEL + DNT - 1) / DNT;      // copies per thread and plane
constexpr size_t kSmem26 = (size_t)RING * PSLOT * sizeof(float);
static_assert(SC % DT == 0, "a chunk is whole steps");
static_assert(RING >= DT + 2 + DT, "ring holds a step's planes and the next step's");

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Reduces the CTA's (min, max, sum) into record `rec` of map m (FP64 across warps).
__device__ __forceinline__ void write_record(float mn, float mx, float sm, double (*red)[3], double *__restrict__ part,
                                             int m, int64_t nrec, int64_t rec)
{
    mn = warp_min(mn);
    mx = warp_max(mx);
    sm = warp_sum(sm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[warp][0] = mn;
        red[warp][1] = mx;
        red[warp][2] = sm;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int q = threadIdx.x;
        double v = red[0][q];
        for (int w = 1; w < DNT / 32; ++w) {
            const double u = red[w][q];
            v = q == 0 ? fmin(v, u) : (q == 1 ? fmax(v, u) : v + u);
        }
        part[(3 * m + q) * nrec + rec] = v;
    }
}

// Scales a thread's 4 x 4 block of sums by 1 / Q, folds the values inside the output (the
// first nt planes, ny columns) into its running (min, max, sum) and stores them at o (plane
// stride `plane`).  A whole block takes the widest stores its row start's alignment allows.
__device__ __forceinline__ void emit_block(float (&out)[QT][QY], float invQ, float *o, int64_t plane, int nt, int ny,
                                           float &mn, float &mx, float &sm)
{
    if (nt == QT && ny == QY) {
#pragma unroll
        for (int to = 0; to < QT; ++to) {
#pragma unroll
            for (int yo = 0; yo < QY; ++yo) {
                out[to][yo] *= invQ;
                mn = fminf(mn, out[to][yo]);
                mx = fmaxf(mx, out[to][yo]);
                sm += out[to][yo];
            }
            float *q = o + to * plane;
            const unsigned a = (unsigned)(reinterpret_cast<uintptr_t>(q) & 15);
            if (a == 0) {
                *reinterpret_cast<float4 *>(q) = make_float4(out[to][0], out[to][1], out[to][2], out[to][3]);
            } else if (a == 8) {
                *reinterpret_cast<float2 *>(q) = make_float2(out[to][0], out[to][1]);
                *reinterpret_cast<float2 *>(q + 2) = make_float2(out[to][2], out[to][3]);
            } else {   // 4 or 12: q + 1 is 8-byte aligned
                q[0] = out[to][0];
                *reinterpret_cast<float2 *>(q + 1) = make_float2(out[to][1], out[to][2]);
                q[3] = out[to][3];
            }
        }
    } else {
#pragma unroll
        for (int to = 0; to < QT; ++to) {
            if (to >= nt) break;
#pragma unroll
            for (int yo = 0; yo < QY; ++yo) {
                out[to][yo] *= invQ;
                if (yo < ny) {
                    mn = fminf(mn, out[to][yo]);
                    mx = fmaxf(mx, out[to][yo]);
                    sm += out[to][yo];
                    o[to * plane + yo] = out[to][yo];
                }
            }
        }
    }
}

__global__ void __launch_bounds__(DNT, 4) dcs26_kernel(const __grid_constant__ DBatch bt, const __grid_constant__ DcsConsts k)
{
    extern __shared__ __align__(16) float sE[];
    __shared__ double red[DNT / 32][3];
    const float g1 = k.g[1], g2 = k.g[2], g3 = k.g[3];
    const int tid = threadIdx.x;
    for (int64_t it = blockIdx.x; it < bt.total; it += gridDim.x) {
        const DVol &v = find_volume(bt, it);
        // item -> (map, chunk, x block, y block) in 32 bits (the launcher checks 3 x records)
        const unsigned local = (unsigned)(it - v.item0), ntile = (unsigned)v.tiles;
        const int m = (int)(local / ntile);
        const unsigned rec = local - (unsigned)m * ntile, q1 = rec / (unsigned)v.tiles_y, q2 = q1 / (unsigned)v.tiles_x;
        const int ty = (int)(rec - q1 * (unsigned)v.tiles_y);
        const int tx = (int)(q1 - q2 * (unsigned)v.tiles_x);
        const int64_t ck = q2;
        const int64_t T = v.T, X = v.X, Y = v.Y, XY = X * Y;
        const int64_t o_lo = v.o_lo, o_hi = v.o_hi;      // output planes of E's T planes
        const int64_t t0 = o_lo + ck * SC, x0 = (int64_t)tx * DX, y0 = (int64_t)ty * DY;
        const float *Em = v.E + m * T * XY;
        float *Sm = v.Sm + m * (o_hi - o_lo) * XY;

        // this thread's copies within one plane: source pointer of its element in plane 0 of
        // the map and its byte offset in a slot (a shared-memory address is 32 bits)
        const float *srcq[KEL];
        int soff[KEL];
#pragma unroll
        for (int q = 0; q < KEL; ++q) {
            const int e = tid + q * DNT;
            const int b = e / (DY + 2), c = e - b * (DY + 2);
            srcq[q] = Em + (e < PEL ? ext_index(x0 - 1 + b, X, bt.bnd) * Y + ext_index(y0 - 1 + c, Y, bt.bnd) : 0);
            soff[q] = e < PEL ? (b * PROW + 3 + c) * (int)sizeof(float) : -1;
        }
        const unsigned sbase = (unsigned)__cvta_generic_to_shared(sE);
        // copies halo planes r0 .. r1 - 1 of the chunk (plane r is t0 - 1 + r) into their slots;
        // planes inside the volume skip the boundary extension, and only the last of a thread's
        // KEL copies can fall outside the plane's PEL elements
        auto stage = [&](int r0, int r1) {
            int slot = r0 % RING;
            for (int r = r0; r < r1; ++r) {
                int64_t gt = t0 - 1 + r;
                if ((uint64_t)gt >= (uint64_t)T) gt = ext_index(gt, T, bt.bnd);
                const int64_t poff = gt * XY;
                const unsigned dst = sbase + (unsigned)(slot * PSLOT * (int)sizeof(float));
#pragma unroll
                for (int q = 0; q < KEL; ++q)
                    if ((q + 1) * DNT <= PEL || soff[q] >= 0)
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst + (unsigned)soff[q]),
                                     "l"(srcq[q] + poff)
                                     : "memory");
                slot = slot + 1 == RING ? 0 : slot + 1;
            }
            cp_async_commit();
        };

        const int64_t left = o_hi - t0;
        const int nsteps = (int)(((left < SC ? left : SC) + DT - 1) / DT);
        // thread -> (t quarter, x row, y quad) of the block; a block at the last columns of the
        // volume packs its nyq < 16 live quads into the first threads, so that whole warps sit
        // out the arithmetic instead of computing columns past Y
        const int64_t left_y = Y - y0;
        const int nyq = left_y >= DY ? DY / QY : (int)((left_y + QY - 1) / QY);
        const int yq = tid % nyq, x = (tid / nyq) % DX, tq = tid / (nyq * DX);
        const bool live = tq < DT / QT;
        const int64_t gx = x0 + x, gy = y0 + QY * yq;
        float mn = FLT_MAX, mx = -FLT_MAX, sm = 0.f;

        // one barrier per step: it publishes the step's planes and also ends every thread's
        // reads of the previous step, whose first DT slots the next step's copies then reuse
        stage(0, DT + 2);
        for (int st = 0; st < nsteps; ++st) {
            cp_async_wait<0>();
            __syncthreads();
            if (st + 1 < nsteps) stage(DT * st + DT + 2, DT * st + 2 * DT + 2);

            if (live) {
                // halo planes rb .. rb + 5 of this thread's 4 output planes, rows x .. x + 2,
                // columns 4 yq .. 4 yq + 5 (stored at + 3)
                const int rb = DT * st + QT * tq;
                int sl[QT + 2];
                {
                    int sp = rb % RING;
#pragma unroll
                    for (int p = 0; p < QT + 2; ++p) {
                        sl[p] = sp * PSLOT + x * PROW + QY * yq + 3;
                        sp = sp + 1 == RING ? 0 : sp + 1;
                    }
                }
                float cen[QT][QY], out[QT][QY];
#pragma unroll
                for (int to = 0; to < QT; ++to) {
                    const float4 c4 = *reinterpret_cast<const float4 *>(sE + sl[to + 1] + PROW + 1);
                    cen[to][0] = c4.x; cen[to][1] = c4.y; cen[to][2] = c4.z; cen[to][3] = c4.w;
#pragma unroll
                    for (int yo = 0; yo < QY; ++yo) out[to][yo] = 0.f;
                }
#pragma unroll
                for (int p = 0; p < QT + 2; ++p)
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const float *row = sE + sl[p] + b * PROW;
                        float w[QY + 2];
                        w[0] = row[0];
                        const float4 mid = *reinterpret_cast<const float4 *>(row + 1);
                        w[1] = mid.x; w[2] = mid.y; w[3] = mid.z; w[4] = mid.w;
                        w[5] = row[5];
#pragma unroll
                        for (int to = 0; to < QT; ++to) {
                            const int dt = p - (to + 1);
                            if (dt < -1 || dt > 1) continue;
#pragma unroll
                            for (int yo = 0; yo < QY; ++yo)
#pragma unroll
                                for (int cc = -1; cc <= 1; ++cc) {
                                    const int d2 = dt * dt + (b - 1) * (b - 1) + cc * cc;
                                    if (d2 == 0) continue;
                                    const float g = d2 == 1 ? g1 : (d2 == 2 ? g2 : g3);
                                    out[to][yo] += fabsf(fmaf(-g, w[yo + 1 + cc], cen[to][yo]));
                                }
                        }
                    }

                if (gx < X) {
                    const int64_t lt = o_hi - (t0 + rb), ly = Y - gy;
                    emit_block(out, k.invQ, Sm + ((t0 - o_lo + rb) * X + gx) * Y + gy, X * Y,
                               (int)(lt < QT ? lt : QT), (int)(ly < QY ? ly : QY), mn, mx, sm);
                }
            }
        }
        write_record(mn, mx, sm, red, v.part, m, v.tiles, rec);
        __syncthreads();
    }
}

// ---- line and offset-list stencils, planes streamed along t --------------------------------
// The same walk as the 26-neighbourhood kernel: one work item = (volume, map, chunk of SC
// planes, 8 x 64 column block), halo planes of the map's own stencil passing through a ring
// of `ring` = (DT + 2 rt) + DT plane slots (the step's halo planes, and the next step's DT
// planes in flight).  Slot s holds one halo plane (PX rows x pitch floats, geometry of
// Halo) at s * PP.  A thread's copies within a plane (row b, column c of the halo, at most
// KMAX) are set up once per item with their boundary extension; a plane then costs one
// offset and KMAX copies.  The in-plane source offsets are 32-bit (the launcher checks
// X * Y < 2^31).

// Slot of halo plane sb + j (sb < ring, j < ring).
__device__ __forceinline__ int wrap_slot(int s, int ring) { return s >= ring ? s - ring : s; }

// d x 1 lines of half-width H along each axis (Sec. 2): out = sum_{q=1..H} |c - g(q) n(+q)|
// + |c - g(q) n(-q)|.  Along t and x the neighbours of a thread's 4 outputs are 4 aligned
// columns of another plane or row; along y the thread reads the window of columns
// -4 ceil(H/4) .. 3 + 4 ceil(H/4) once per plane.
template <int H>
struct LineStencil {
    DcsConsts k;
    // copies per thread and plane: the largest halo plane is (DX + 2H) rows x DY columns
    static constexpr int KMAX = ((DX + 2 * H) * DY + DNT - 1) / DNT;
    // resident CTAs the register budget is cut for (the ring of the x line, the largest,
    // leaves room for 3 CTAs per SM up to H = 3 and 2 beyond)
    static constexpr int MINB = H <= 3 ? 3 : 2;
    __device__ Halo halo(int m) const { return halo_for(SAL_STENCIL_LINE, m, H); }
    __device__ float invQ(int) const { return k.invQ; }
    // sb: slot of halo plane rb, the first plane any of the thread's neighbours lie in
    __device__ __forceinline__ void compute(const float *sE, const Halo &hl, int ring, int m, int sb, int x, int yq,
                                            float (&out)[QT][QY]) const
    {
        if (m == 0) {
            int pb[QT + 2 * H];   // float offsets of the thread's column quad in halo planes rb + j
#pragma unroll
            for (int j = 0; j < QT + 2 * H; ++j) pb[j] = wrap_slot(sb + j, ring) * hl.PP + x * hl.pitch + QY * yq;
#pragma unroll
            for (int to = 0; to < QT; ++to) {
                const float4 cv = lds4(sE + pb[to + H]);
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
                for (int q = 1; q <= H; ++q) {
                    const float g = k.gl[q];
                    const float4 a = lds4(sE + pb[to + H + q]), b = lds4(sE + pb[to + H - q]);
                    s0 += fabsf(fmaf(-g, a.x, cv.x));
                    s0 += fabsf(fmaf(-g, b.x, cv.x));
                    s1 += fabsf(fmaf(-g, a.y, cv.y));
                    s1 += fabsf(fmaf(-g, b.y, cv.y));
                    s2 += fabsf(fmaf(-g, a.z, cv.z));
                    s2 += fabsf(fmaf(-g, b.z, cv.z));
                    s3 += fabsf(fmaf(-g, a.w, cv.w));
                    s3 += fabsf(fmaf(-g, b.w, cv.w));
                }
                out[to][0] = s0;
                out[to][1] = s1;
                out[to][2] = s2;
                out[to][3] = s3;
            }
        } else if (m == 1) {
#pragma unroll
            for (int to = 0; to < QT; ++to) {
                const float *c = sE + wrap_slot(sb + to, ring) * hl.PP + (x + H) * hl.pitch + QY * yq;
                const float4 cv = lds4(c);
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
                for (int q = 1; q <= H; ++q) {
                    const float g = k.gl[q];
                    const float4 a = lds4(c + q * hl.pitch), b = lds4(c - q * hl.pitch);
                    s0 += fabsf(fmaf(-g, a.x, cv.x));
                    s0 += fabsf(fmaf(-g, b.x, cv.x));
                    s1 += fabsf(fmaf(-g, a.y, cv.y));
                    s1 += fabsf(fmaf(-g, b.y, cv.y));
                    s2 += fabsf(fmaf(-g, a.z, cv.z));
                    s2 += fabsf(fmaf(-g, b.z, cv.z));
                    s3 += fabsf(fmaf(-g, a.w, cv.w));
                    s3 += fabsf(fmaf(-g, b.w, cv.w));
                }
                out[to][0] = s0;
                out[to][1] = s1;
                out[to][2] = s2;
                out[to][3] = s3;
            }
        } else {
            constexpr int W0 = (H + 3) / 4;   // 16-byte groups left (and right) of the centre's
            float w[4 * (2 * W0 + 1)];
#pragma unroll
            for (int to = 0; to < QT; ++to) {
                const float *c = sE + wrap_slot(sb + to, ring) * hl.PP + x * hl.pitch + hl.off + H + QY * yq;
#pragma unroll
                for (int j = 0; j <= 2 * W0; ++j) {
                    const float4 v = lds4(c + 4 * (j - W0));
                    w[4 * j] = v.x;
                    w[4 * j + 1] = v.y;
                    w[4 * j + 2] = v.z;
                    w[4 * j + 3] = v.w;
                }
#pragma unroll
                for (int yo = 0; yo < QY; ++yo) {
                    const float cv = w[4 * W0 + yo];
                    float s = 0.f;
#pragma unroll
                    for (int q = 1; q <= H; ++q) {
                        s += fabsf(fmaf(-k.gl[q], w[4 * W0 + yo + q], cv));
                        s += fabsf(fmaf(-k.gl[q], w[4 * W0 + yo - q], cv));
                    }
                    out[to][yo] = s;
                }
            }
        }
    }
};

// Offset-list neighbourhood of every map (the t-x diagonal, caller-given stencils): halo
// radii, each neighbour's plane offset dt and in-plane shared-memory offset dx * pitch + dy
// (for that map's halo geometry), its weight, and 1 / Q.
struct UserStencil {
    int Q[3];
    int rt[3], rx[3], ry[3];
    int dt[3][SAL_STENCIL_MAX_OFFSETS];
    int delta[3][SAL_STENCIL_MAX_OFFSETS];
    float w[3][SAL_STENCIL_MAX_OFFSETS];
    float iq[3];
    static constexpr int KMAX =
        ((DX + 2 * SAL_STENCIL_MAX_RADIUS) * (DY + 2 * SAL_STENCIL_MAX_RADIUS) + DNT - 1) / DNT;
    static constexpr int MINB = 2;
    __device__ Halo halo(int m) const { return Halo(rt[m], rx[m], ry[m]); }
    __device__ float invQ(int m) const { return iq[m]; }
    // out = sum_q |c - w_q n(dt_q, delta_q)|.  delta_q mod 4 is the neighbour's y offset mod 4
    // (the same for every thread), so the 4 neighbours of a thread's outputs are one aligned
    // 16-byte load, or two and a shift.
    __device__ __forceinline__ void compute(const float *sE, const Halo &hl, int ring, int m, int sb, int x, int yq,
                                            float (&out)[QT][QY]) const
    {
        const int col = (x + hl.rx) * hl.pitch + hl.off + hl.ry + QY * yq;   // centre column quad in a plane
        float4 cv[QT];
#pragma unroll
        for (int to = 0; to < QT; ++to) {
            cv[to] = lds4(sE + wrap_slot(sb + hl.rt + to, ring) * hl.PP + col);
#pragma unroll
            for (int yo = 0; yo < QY; ++yo) out[to][yo] = 0.f;
        }
        for (int q = 0; q < Q[m]; ++q) {
            const int d = delta[m][q], da = d & ~3, sh = d - da;
            const int s0 = sb + hl.rt + dt[m][q];   // slot of the neighbour plane of output plane 0
            const float wq = w[m][q];
#pragma unroll
            for (int to = 0; to < QT; ++to) {
                const float *p = sE + wrap_slot(s0 + to, ring) * hl.PP + col + da;
                const float4 a = lds4(p);
                float4 n = a;
                if (sh != 0) {
                    const float4 b = lds4(p + 4);
                    n = sh == 1 ? make_float4(a.y, a.z, a.w, b.x)
                                : (sh == 2 ? make_float4(a.z, a.w, b.x, b.y) : make_float4(a.w, b.x, b.y, b.z));
                }
                out[to][0] += fabsf(fmaf(-wq, n.x, cv[to].x));
                out[to][1] += fabsf(fmaf(-wq, n.y, cv[to].y));
                out[to][2] += fabsf(fmaf(-wq, n.z, cv[to].z));
                out[to][3] += fabsf(fmaf(-wq, n.w, cv[to].w));
            }
        }
    }
};

template <class St>
__global__ void __launch_bounds__(DNT, St::MINB) dcs_stream_kernel(const __grid_constant__ DBatch bt,
                                                            const __grid_constant__ St sp)
{
    constexpr int KMAX = St::KMAX;
    extern __shared__ __align__(16) float sE[];
    __shared__ double red[DNT / 32][3];
    const int tid = threadIdx.x;
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(sE);
    for (int64_t it = blockIdx.x; it < bt.total; it += gridDim.x) {
        const DVol &v = find_volume(bt, it);
        // item -> (map, chunk, x block, y block) in 32 bits (the launcher checks 3 x records)
        const unsigned local = (unsigned)(it - v.item0), ntile = (unsigned)v.tiles;
        const int m = (int)(local / ntile);
        const unsigned rec = local - (unsigned)m * ntile, q1 = rec / (unsigned)v.tiles_y, q2 = q1 / (unsigned)v.tiles_x;
        const int ty = (int)(rec - q1 * (unsigned)v.tiles_y);
        const int tx = (int)(q1 - q2 * (unsigned)v.tiles_x);
        const int64_t T = v.T, X = v.X, Y = v.Y, XY = X * Y;
        const int64_t o_lo = v.o_lo, o_hi = v.o_hi;
        const int64_t t0 = o_lo + (int64_t)q2 * SC, x0 = (int64_t)tx * DX, y0 = (int64_t)ty * DY;
        const float *Em = v.E + m * T * XY;
        const Halo hl = sp.halo(m);
        const int ring = hl.planes + DT, W = DY + 2 * hl.ry, PE = hl.PX * W;

        // this thread's copies within a halo plane: in-plane source offset (boundary extension
        // along x and y applied) and byte offset in a slot, -1 past the plane's PE elements
        int srco[KMAX], dsto[KMAX];
#pragma unroll
        for (int q = 0; q < KMAX; ++q) {
            const int e = tid + q * DNT;
            srco[q] = 0;
            dsto[q] = -1;
            if (e < PE) {
                const int b = e / W, c = e - b * W;
                int64_t gx = x0 - hl.rx + b, gy = y0 - hl.ry + c;
                if ((uint64_t)gx >= (uint64_t)X) gx = ext_index(gx, X, bt.bnd);
                if ((uint64_t)gy >= (uint64_t)Y) gy = ext_index(gy, Y, bt.bnd);
                srco[q] = (int)(gx * Y + gy);
                dsto[q] = (b * hl.pitch + hl.off + c) * (int)sizeof(float);
            }
        }
        // copies halo planes r0 .. r1 - 1 of the chunk (plane r is t0 - rt + r) into their slots
        auto stage = [&](int r0, int r1) {
            int slot = r0 % ring;
            for (int r = r0; r < r1; ++r) {
                int64_t gt = t0 - hl.rt + r;
                if ((uint64_t)gt >= (uint64_t)T) gt = ext_index(gt, T, bt.bnd);
                const float *pl = Em + gt * XY;
                const unsigned dst = sbase + (unsigned)(slot * hl.PP * (int)sizeof(float));
#pragma unroll
                for (int q = 0; q < KMAX; ++q)
                    if (dsto[q] >= 0)
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst + (unsigned)dsto[q]),
                                     "l"(pl + srco[q])
                                     : "memory");
                slot = slot + 1 == ring ? 0 : slot + 1;
            }
            cp_async_commit();
        };

        const int64_t left = o_hi - t0;
        const int nsteps = (int)(((left < SC ? left : SC) + DT - 1) / DT);
        // thread -> (t quarter, x row, y quad); a block at the last columns packs its live quads
        // into the first threads (see the 26-neighbourhood kernel)
        const int64_t left_y = Y - y0;
        const int nyq = left_y >= DY ? DY / QY : (int)((left_y + QY - 1) / QY);
        const int yq = tid % nyq, x = (tid / nyq) % DX, tq = tid / (nyq * DX);
        const bool live = tq < DT / QT;
        const int64_t gx = x0 + x, gy = y0 + QY * yq;
        float mn = FLT_MAX, mx = -FLT_MAX, sm = 0.f;

        // one barrier per step, as in the 26-neighbourhood kernel
        stage(0, hl.planes);
        for (int st = 0; st < nsteps; ++st) {
            cp_async_wait<0>();
            __syncthreads();
            if (st + 1 < nsteps) stage(DT * st + hl.planes, DT * st + hl.planes + DT);
            if (live) {
                const int rb = DT * st + QT * tq;
                float out[QT][QY];
                sp.compute(sE, hl, ring, m, rb % ring, x, yq, out);
                if (gx < X) {
                    const int64_t lt = o_hi - (t0 + rb), ly = Y - gy;
                    emit_block(out, sp.invQ(m), v.Sm + m * (o_hi - o_lo) * XY + ((t0 - o_lo + rb) * X + gx) * Y + gy,
                               XY, (int)(lt < QT ? lt : QT), (int)(ly < QY ? ly : QY), mn, mx, sm);
                }
            }
        }
        write_record(mn, mx, sm, red, v.part, m, v.tiles, rec);
        __syncthreads();
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
    // vector width: 4 when every plane starts on a 16-byte boundary (N % 4 == 0), else 2
    // when N is even (planes 8-byte aligned), else scalar; the tail is scalar
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if ((N & 3) == 0) {
        const int64_t n4 = N / 4;
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
        done = 4 * n4;
    } else if ((N & 1) == 0) {
        const int64_t n2 = N / 2;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n2; i += stride) {
            const float2 s0 = __ldg(reinterpret_cast<const float2 *>(Sm) + i);
            const float2 s1 = __ldg(reinterpret_cast<const float2 *>(Sm + N) + i);
            const float2 s2 = __ldg(reinterpret_cast<const float2 *>(Sm + 2 * N) + i);
            float2 o;
            o.x = fmaf(al[2], s2.x - lo[2], fmaf(al[1], s1.x - lo[1], al[0] * (s0.x - lo[0])));
            o.y = fmaf(al[2], s2.y - lo[2], fmaf(al[1], s1.y - lo[1], al[0] * (s0.y - lo[0])));
            reinterpret_cast<float2 *>(S)[i] = o;
        }
        done = 2 * n2;
    }
    for (int64_t i = done + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += stride)
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

DcsConsts dcs_consts(const sal_params *p)
{
    DcsConsts k;
    const double s2 = 2.0 * (double)p->sigma * (double)p->sigma;
    for (int i = 0; i < 4; ++i) k.g[i] = (float)exp(-(double)i / s2);
    const int h = (p->L - 1) / 2;
    for (int i = 0; i <= kMaxH; ++i) k.gl[i] = (float)exp(-(double)(i * i) / s2);
    k.h = h;
    k.invQ = (float)(1.0 / (p->stencil == SAL_STENCIL_26 ? 26.0 : (double)(2 * h)));
    return k;
}

int64_t dcs_num_records(sal_dims d)
{
    int64_t nt, nx, ny;
    dcs_tiles(d, &nt, &nx, &ny);
    nt = (d.T + SC - 1) / SC;
    return nt * nx * ny;
}

// The t-x diagonal of Fig. 3 as an offset list: (k, k, 0), k = +-1..+-h, weights
// g = exp(-2 k^2 / (2 sigma^2)), the same line for every map.
sal_user_stencil diag_tx_stencil(const sal_params *p)
{
    sal_user_stencil u;
    memset(&u, 0, sizeof(u));
    const int h = (p->L - 1) / 2;
    const double s2 = 2.0 * (double)p->sigma * (double)p->sigma;
    for (int m = 0; m < 3; ++m) {
        int q = 0;
        for (int k = -h; k <= h; ++k) {
            if (!k) continue;
            u.offset[m][q][0] = k;
            u.offset[m][q][1] = k;
            u.offset[m][q][2] = 0;
            u.weight[m][q] = (float)exp(-(double)(2 * k * k) / s2);
            ++q;
        }
        u.count[m] = q;
    }
    return u;
}

namespace {

UserStencil user_consts(const sal_user_stencil &st)
{
    UserStencil u;
    memset(&u, 0, sizeof(u));
    for (int m = 0; m < 3; ++m) {
        int rt = 0, rx = 0, ry = 0;
        for (int q = 0; q < st.count[m]; ++q) {
            rt = abs(st.offset[m][q][0]) > rt ? abs(st.offset[m][q][0]) : rt;
            rx = abs(st.offset[m][q][1]) > rx ? abs(st.offset[m][q][1]) : rx;
            ry = abs(st.offset[m][q][2]) > ry ? abs(st.offset[m][q][2]) : ry;
        }
        const Halo hl(rt, rx, ry);
        u.Q[m] = st.count[m];
        u.rt[m] = rt;
        u.rx[m] = rx;
        u.ry[m] = ry;
        for (int q = 0; q < st.count[m]; ++q) {
            u.dt[m][q] = st.offset[m][q][0];
            u.delta[m][q] = st.offset[m][q][1] * hl.pitch + st.offset[m][q][2];
            u.w[m][q] = st.weight[m][q];
        }
        u.iq[m] = (float)(1.0 / (double)st.count[m]);
    }
    return u;
}

template <class St>
cudaError_t launch_stream(const DBatch &bt, const St &sp, int smem, int64_t total, cudaStream_t s)
{
    const void *fn = (const void *)dcs_stream_kernel<St>;
    int dev = 0, nsm = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = set_smem(fn, smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, DNT, smem);
    if (e != cudaSuccess) return e;
    const int64_t resident = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
    const int64_t grid = total < resident ? total : resident;
    if (grid <= 0) return cudaSuccess;
    dcs_stream_kernel<St><<<(unsigned)grid, DNT, smem, s>>>(bt, sp);
    return cudaGetLastError();
}

}  // namespace

int dcs_user_radius_t(const sal_user_stencil &st)
{
    int r = 0;
    for (int m = 0; m < 3; ++m)
        for (int q = 0; q < st.count[m]; ++q) r = abs(st.offset[m][q][0]) > r ? abs(st.offset[m][q][0]) : r;
    return r;
}

// Launches the compare over n volumes as one persistent grid (resident CTAs walk every
// (volume, map, tile) item).  `user` (offset lists per map) replaces p->stencil when
// given; p->stencil == SAL_STENCIL_DIAG_TX builds the diagonal's list.
cudaError_t launch_dcs_items(const DVolDesc *vols, int n, const sal_params *p, cudaStream_t s,
                             const sal_user_stencil *user)
{
    if (n < 1 || n > kMaxBatch) return cudaErrorInvalidValue;
    sal_user_stencil diag;
    if (!user && p->stencil == SAL_STENCIL_DIAG_TX) {
        diag = diag_tx_stencil(p);
        user = &diag;
    }
    const bool s26 = !user && p->stencil == SAL_STENCIL_26;
    const int h = (p->L - 1) / 2;
    if (!user && !s26 && (h < 1 || h > kMaxH)) return cudaErrorInvalidValue;
    DBatch bt;
    bt.n = n;
    bt.bnd = p->boundary;
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        DVol &v = bt.v[i];
        int64_t nt, nx, ny;
        const sal_dims d{vols[i].T, vols[i].X, vols[i].Y};
        const int64_t o_lo = vols[i].o_lo, o_hi = vols[i].o_hi < 0 ? d.T : vols[i].o_hi;
        if (o_lo < 0 || o_hi > d.T || o_lo >= o_hi) return cudaErrorInvalidValue;
        // the line and offset-list kernels hold in-plane offsets in 32 bits
        if (!s26 && d.X * d.Y > 0x7fffffffLL) return cudaErrorInvalidValue;
        const sal_dims dout{o_hi - o_lo, d.X, d.Y};
        dcs_tiles(dout, &nt, &nx, &ny);
        v.E = vols[i].E;
        v.Sm = vols[i].Sm;
        v.part = vols[i].part;
        v.T = d.T;
        v.X = d.X;
        v.Y = d.Y;
        v.o_lo = o_lo;
        v.o_hi = o_hi;
        v.tiles = dcs_num_records(dout);
        if (3 * v.tiles > 0x7fffffffLL) return cudaErrorInvalidValue;   // items of a volume in 32 bits
        v.tiles_x = (int)nx;
        v.tiles_y = (int)ny;
        v.item0 = total;
        total += 3 * v.tiles;
    }
    bt.total = total;
    const DcsConsts k = dcs_consts(p);
    if (s26) {
        const void *fn = (const void *)dcs26_kernel;
        int dev = 0, nsm = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = set_smem(fn, (int)kSmem26);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, DNT, (int)kSmem26);
        if (e != cudaSuccess) return e;
        const int64_t resident = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
        const int64_t grid = total < resident ? total : resident;
        if (grid <= 0) return cudaSuccess;
        dcs26_kernel<<<(unsigned)grid, DNT, kSmem26, s>>>(bt, k);
        return cudaGetLastError();
    }
    if (user) {
        const UserStencil u = user_consts(*user);
        int smem = 0;
        for (int m = 0; m < 3; ++m) {
            const int f = Halo(u.rt[m], u.rx[m], u.ry[m]).ring_floats() * (int)sizeof(float);
            smem = f > smem ? f : smem;
        }
        return launch_stream(bt, u, smem, total, s);
    }
    int smem = 0;
    for (int m = 0; m < 3; ++m) {
        const int f = halo_for(SAL_STENCIL_LINE, m, h).ring_floats() * (int)sizeof(float);
        smem = f > smem ? f : smem;
    }
    switch (h) {
        case 1: return launch_stream(bt, LineStencil<1>{k}, smem, total, s);
        case 2: return launch_stream(bt, LineStencil<2>{k}, smem, total, s);
        case 3: return launch_stream(bt, LineStencil<3>{k}, smem, total, s);
        case 4: return launch_stream(bt, LineStencil<4>{k}, smem, total, s);
        case 5: return launch_stream(bt, LineStencil<5>{k}, smem, total, s);
        case 6: return launch_stream(bt, LineStencil<6>{k}, smem, total, s);
        default: return launch_stream(bt, LineStencil<7>{k}, smem, total, s);
    }
}

cudaError_t launch_dcs(const float *E, sal_dims d, const sal_params *p, float *Sm, double *partials, double *stats,
                       cudaStream_t s, const sal_user_stencil *user, int64_t o_lo, int64_t o_hi)
{
    if (o_hi < 0) o_hi = d.T;
    const int64_t tiles = dcs_num_records(sal_dims{o_hi - o_lo, d.X, d.Y});
    if (3 * tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    DVolDesc v{E, Sm, partials, d.T, d.X, d.Y, o_lo, o_hi};
    cudaError_t e = launch_dcs_items(&v, 1, p, s, user);
    if (e != cudaSuccess) return e;
    double *second = partials + 9 * tiles;
    reduce_partials_kernel<<<kRedBlocks, 256, 0, s>>>(partials, tiles, second, kRedBlocks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_partials_kernel<<<1, 256, 0, s>>>(second, kRedBlocks, stats, 1);
    return cudaGetLastError();
}

// Merges n statistics records [n][9] (device) into one: min of the minima, max of the
// maxima, FP64 sum of the sums, in record order.
__global__ void stats_merge_kernel(const double *__restrict__ in, int n, double *__restrict__ out)
{
    const int q = threadIdx.x;
    if (q >= 9) return;
    double v = in[q];
    for (int i = 1; i < n; ++i) {
        const double u = in[9 * i + q];
        v = q % 3 == 0 ? fmin(v, u) : (q % 3 == 1 ? fmax(v, u) : v + u);
    }
    out[q] = v;
}

cudaError_t launch_stats_merge(const double *in, int n, double *out, cudaStream_t s)
{
    stats_merge_kernel<<<1, 32, 0, s>>>(in, n, out);
    return cudaGetLastError();
}

cudaError_t launch_combine(const float *Sm, const double *stats, sal_dims d, const sal_params *p, float *S,
                           cudaStream_t s)
{
    const int64_t N = d.T * d.X * d.Y;
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (N / 2 + 255) / 256;
    const int64_t cap = (int64_t)nsm * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    combine_kernel<<<(unsigned)blocks, 256, 0, s>>>(Sm, stats, N, p->a, p->b, p->c, p->eps, S);
    return cudaGetLastError();
}

// ---- directional compare with fixed scratch --------------------------------------------
// Scratch for the partial records of sal_directional_compare_static: a file-scope device
// array, so that entry point allocates nothing.  Its size is fixed at build time; every
// GPU that loads the library holds it until the process exits.
static __device__ __align__(256) double g_dcs_static_scratch[9 * (SAL_DCS_STATIC_MAX_TILES + kRedBlocks)];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
struct StaticSlot {
    unsigned long long ctx = 0;   // id of the context the address belongs to
    double *ptr = nullptr;
};
StaticSlot g_static_slot[kMaxDevices];
}  // namespace

int64_t dcs_num_tiles(sal_dims d)
{
    int64_t nt, nx, ny;
    dcs_tiles(d, &nt, &nx, &ny);
    return nt * nx * ny;
}

// Device address of the fixed scratch on the current device.  In host code the array's
// name is only a host-side stand-in, so the address comes from cudaGetSymbolAddress: once per
// device (with that device current), cached together with the id of the context it belongs
// to.  A device reset (or any new primary context) changes that id, and the next call looks
// the address up again instead of using one from the destroyed context.
cudaError_t dcs_static_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_static_mu);
    StaticSlot &sl = g_static_slot[dev];
    unsigned long long ctx = 0;
    const bool have_ctx = current_context_id(&ctx) == cudaSuccess;
    if (!sl.ptr || !have_ctx || sl.ctx != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dcs_static_scratch);   // creates the primary context if needed
        if (e != cudaSuccess) return e;
        e = current_context_id(&ctx);
        if (e != cudaSuccess) return e;
        sl.ptr = static_cast<double *>(p);
        sl.ctx = ctx;
    }
    *out = sl.ptr;
    return cudaSuccess;
}

}  // namespace sal
