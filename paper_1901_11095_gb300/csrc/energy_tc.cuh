// Spectral energies with the y-stage DFT on the tensor cores (tcgen05, BF16 or TF32 operands,
// FP32 accumulation in tensor memory).
//
// Stages t and x run on the CUDA cores in FP32 exactly as in the FP32 kernel.  Stage y, the
// length-L DFT of every sliding window of every (mu, nu) line (three quarters of the
// work), becomes a dense product: each row of A holds the 8 + 2h consecutive samples of
// one line that the 8 outputs of a segment need (re/im interleaved, K padded to the
// instruction K), and B is the banded Toeplitz DFT matrix that maps such a run to the L
// frequencies of each of the 8 windows:
//     D[(row, segment), (o, omega, re/im)] = sum_k A[(row, segment), k] B[(o, omega, re/im), k].
// The band zeros cost (8 + 2h) / L times the algorithmic MACs; they are not counted as work.
// One M = 128 product takes two lines at once (64 (row, segment) pairs each).  The epilogue
// reads D from tensor memory (one lane per row), forms |F|, applies the projection weights of
// Eq. 1-4 and accumulates each output's energies in registers across all lines.
//
// Samples of a line are taken relative to a reference sample of their segment (its first
// window's centre) before rounding to the operand type: that changes no coefficient off
// omega = 0 (twiddles of a non-zero frequency sum to zero), restores omega = 0 exactly in
// FP32 (+ L * reference), keeps a constant line exactly zero, and shrinks the rounded values.
//
// Every wait on the tensor cores is bounded (about one second of GPU time); on expiry the
// CTA records SAL_ERR_TIMEOUT in a status word, releases its tensor memory and returns.
#pragma once
#include <cuda_bf16.h>

#include "energy_fp32.cuh"

namespace sal {
namespace energy_detail {

struct OpBF16 {
    static constexpr int ESZ = 2, KI = 16, KG = 8, FMT = 1;
};
struct OpTF32 {
    static constexpr int ESZ = 4, KI = 8, KG = 4, FMT = 2;
};

template <int L_, int BT_, int BX_, class OP_>
struct TGeo {
    using OP = OP_;
    static constexpr int L = L_, H = (L_ - 1) / 2, BT = BT_, BX = BX_;
    static constexpr int BY = 32, P = 8, SEG = BY / P, ROWS = BT * BX;
    static_assert(ROWS * SEG == 64, "64 (row, segment) pairs fill one half of an M = 128 product");
    static constexpr int NT = 256;                                  // two warpgroups share the epilogue
    static constexpr int HX = BX + 2 * H, PY = BY + 2 * H;
    static constexpr int NV = (BT + 2 * H) * HX * PY;
    static constexpr int NG1 = (BT * HX * L * PY + 31) / 32 * 32;   // floats (128-byte multiple)
    static constexpr int RUN = P + 2 * H;                           // samples behind one segment
    static constexpr int KP = (2 * RUN + OP::KI - 1) / OP::KI * OP::KI;
    static constexpr int KGR = KP / OP::KG;                         // core matrices along K
    static constexpr int N = 2 * P * L;
    static constexpr int NPAIR = H + 1;                             // products per mu
    static constexpr int PAIR_BYTES = 128 * KP * OP::ESZ;
    static constexpr int A_BYTES = NPAIR * PAIR_BYTES;
    static constexpr int AV_RAW = A_BYTES > NV * 4 ? A_BYTES : NV * 4;
    static constexpr int AV_BYTES = (AV_RAW + 127) / 128 * 128;
    static constexpr int B_BYTES = (N * KP * OP::ESZ + 127) / 128 * 128;
    static constexpr int REF_BYTES = NPAIR * 128 * 8;
    // three partial sets meet the fourth at the end of a tile, in the stage-t buffer (free by
    // then) where it fits, else in a region of their own
    static constexpr int XCH_BYTES = 3 * 64 * 3 * P * 4;
    static constexpr bool XCH_IN_G1 = XCH_BYTES <= NG1 * 4;
    static constexpr int OFF_A = NG1 * 4, OFF_B = OFF_A + AV_BYTES, OFF_REF = OFF_B + B_BYTES;
    static constexpr int NW = ((H + 1) * (H + 1) * (H + 1) * 3 + 3) / 4 * 4;
    static constexpr int OFF_X = XCH_IN_G1 ? 0 : OFF_REF + REF_BYTES;
    static constexpr int OFF_W = OFF_REF + REF_BYTES + (XCH_IN_G1 ? 0 : XCH_BYTES), OFF_BAR = OFF_W + NW * 4;
    static constexpr size_t SMEM = OFF_BAR + 16;
    static constexpr int PPR = (256 / N < NPAIR) ? (256 / N > 0 ? 256 / N : 1) : NPAIR;  // products per round
    static constexpr int TCOLS_RAW = PPR * N;
    static constexpr int TMEM_COLS = TCOLS_RAW <= 32 ? 32 : TCOLS_RAW <= 64 ? 64 : TCOLS_RAW <= 128 ? 128
                                     : TCOLS_RAW <= 256 ? 256 : 512;
    static_assert(N <= 256 && N % 16 == 0, "N of one product");
    static_assert(SMEM <= 227 * 1024, "shared memory of one CTA");
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle, K-major core matrices of 8 rows x 16 bytes:
// lbo = bytes between core matrices adjacent along K, sbo = between adjacent 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: FP32 accumulator, A and B of format `fmt`, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int fmt, int m, int n)
{
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(m >> 4) << 24);
}

// Byte offset of element (row, k) of a K-major operand tile with KGR core matrices along K.
template <class G>
__device__ __forceinline__ int cm_off(int row, int k)
{
    return ((row >> 3) * G::KGR + k / G::OP::KG) * 128 + (row & 7) * 16 + (k % G::OP::KG) * G::OP::ESZ;
}

// Stores the complex value (re, im) at K positions (2j, 2j + 1) of operand row `row`.
template <class G>
__device__ __forceinline__ void put_pair(unsigned char *tile, int row, int j, float re, float im)
{
    unsigned char *p = tile + cm_off<G>(row, 2 * j);
    if (G::OP::ESZ == 2) {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(re, im);
    } else {
        // round to the TF32 grid (nearest, ties away) instead of letting the unit truncate
        uint32_t a, b;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(a) : "f"(re));
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b) : "f"(im));
        *reinterpret_cast<uint2 *>(p) = make_uint2(a, b);
    }
}

// Lines of one mu in product order: mu = 0: nu = 0..h; mu > 0: nu = 0, +1, -1, +2, -2, ...
__device__ __forceinline__ int nlines(int mu, int L) { return mu == 0 ? (L + 1) / 2 : L; }
__device__ __forceinline__ int nu_of_line(int li, int mu) { return mu == 0 ? li : (li == 0 ? 0 : ((li & 1) ? (li + 1) / 2 : -(li / 2))); }

// Stage x at one column (row, y'): every line of this mu, in product order.
template <class G>
__device__ __forceinline__ void x_column(const float *sG1, int row, int yy, int mu, const Tw<G::L> &tw,
                                         float2 (&g)[G::L])
{
    constexpr int L = G::L, H = G::H, PY = G::PY;
    const int t = row / G::BX, x = row - t * G::BX;
    const float *col = sG1 + ((t * G::HX + x) * L) * PY + yy;
    if (mu == 0) {
        float z[L];
#pragma unroll
        for (int k = 0; k < L; ++k) z[k] = col[k * L * PY];
        const float z0 = z[H];
        float s = z0, U[H + 1], D[H + 1];
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const float p = z[H + k] + z[H - k];
            s += p;
            U[k] = fmaf(-2.f, z0, p);
            D[k] = z[H + k] - z[H - k];
        }
        g[0] = make_float2(s, 0.f);
#pragma unroll
        for (int nu = 1; nu <= H; ++nu) {
            float A = 0.f, B = 0.f;
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                A = fmaf(U[k], lo(tw.c2[(nu * k) % L]), A);
                B = fmaf(D[k], lo(tw.s2[(nu * k) % L]), B);
            }
            g[nu] = make_float2(A, -B);
        }
#pragma unroll
        for (int li = H + 1; li < L; ++li) g[li] = make_float2(0.f, 0.f);
    } else {
        const int cre = (2 * mu - 1) * PY, cim = 2 * mu * PY;
        const f2x m2 = pk(-2.f, -2.f);
        f2x z[L];
#pragma unroll
        for (int k = 0; k < L; ++k) z[k] = pk(col[k * L * PY + cre], col[k * L * PY + cim]);
        const f2x z0 = z[H];
        f2x s = z0, U[H + 1], D[H + 1];
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const f2x p = add2(z[H + k], z[H - k]);
            s = add2(s, p);
            U[k] = fma2(z0, m2, p);
            D[k] = sub2(z[H + k], z[H - k]);
        }
        g[0] = make_float2(lo(s), hi(s));
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
            g[2 * nu - 1] = make_float2(ax + by, ay - bx);   // G2(+nu) = A - iB
            g[2 * nu] = make_float2(ax - by, ay + bx);       // G2(-nu) = A + iB
        }
    }
}

// Builds the A operands of one mu: references first (the sample at the first window centre
// of each segment), then every sample relative to its segment's reference.
template <class G>
__device__ __forceinline__ void build_a(const float *sG1, unsigned char *sA, float2 *ref, int mu, const Tw<G::L> &tw)
{
    constexpr int L = G::L, H = G::H, PY = G::PY;
    const int nl = nlines(mu, L);
    for (int i = threadIdx.x; i < G::ROWS * G::SEG; i += G::NT) {
        const int row = i / G::SEG, s = i - row * G::SEG;
        float2 g[L];
        x_column<G>(sG1, row, G::P * s + H, mu, tw, g);
#pragma unroll
        for (int li = 0; li < L; ++li)
            if (li < nl) ref[(li >> 1) * 128 + (li & 1) * 64 + row * G::SEG + s] = g[li];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < G::ROWS * PY; i += G::NT) {
        const int row = i / PY, yy = i - row * PY;
        float2 g[L];
        x_column<G>(sG1, row, yy, mu, tw, g);
        const int s_hi = yy / G::P < G::SEG ? yy / G::P : G::SEG - 1;
#pragma unroll
        for (int ds = 0; ds < 3; ++ds) {
            const int s = s_hi - ds, j = yy - G::P * s;
            if (s < 0 || j < 0 || j >= G::RUN) continue;
#pragma unroll
            for (int li = 0; li < L; ++li) {
                if (li >= nl) continue;
                const int arow = (li & 1) * 64 + row * G::SEG + s;
                const float2 c = ref[(li >> 1) * 128 + arow];
                put_pair<G>(sA + (li >> 1) * G::PAIR_BYTES, arow, j, g[li].x - c.x, g[li].y - c.y);
            }
        }
    }
}

// The banded Toeplitz DFT operand: row n = (o, omega, re/im), K position 2j + re/im for the
// run sample j; window o covers samples o..o+2h, phase measured from its centre.
template <class G>
__device__ __forceinline__ void build_b(unsigned char *sB, const SpecTables &tb)
{
    constexpr int L = G::L, H = G::H;
    for (int e = threadIdx.x; e < G::N * (G::KP / 2); e += G::NT) {
        const int n = e / (G::KP / 2), j = e - n * (G::KP / 2);
        const int c = n & 1, om = (n >> 1) % L, o = (n >> 1) / L;
        float vre = 0.f, vim = 0.f;   // coefficients of the sample's re and im parts
        const int d = j - o - H;
        if (j < G::RUN && d >= -H && d <= H) {
            int k = ((om - H) * d) % L;
            if (k < 0) k += L;
            const float cs = tb.cs[k], sn = tb.sn[k];
            // F = sum z e^{-i phi}: re = zr cos + zi sin, im = zi cos - zr sin
            vre = c == 0 ? cs : -sn;
            vim = c == 0 ? sn : cs;
        }
        put_pair<G>(sB, n, j, vre, vim);
    }
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
    return done != 0;
}

// Bounded wait for phase `parity` of the mbarrier; false when the limit ran out.  A phase
// that has already completed returns without reading the clock.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

template <class G>
__device__ __forceinline__ void issue_mma(uint32_t tmem, uint32_t a_addr, uint32_t b_addr)
{
    constexpr uint32_t idesc = instr_desc(G::OP::FMT, 128, G::N);
#pragma unroll
    for (int ks = 0; ks < G::KP / G::OP::KI; ++ks) {
        const uint64_t da = smem_desc(a_addr + ks * 256, 128, G::KGR * 128);
        const uint64_t db = smem_desc(b_addr + ks * 256, 128, G::KGR * 128);
        const uint32_t acc = ks > 0 ? 1u : 0u;
        if (G::OP::ESZ == 2)
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                         "l"(da), "l"(db), "r"(idesc), "r"(acc));
        else
            asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                         "l"(da), "l"(db), "r"(idesc), "r"(acc));
    }
}

// Arrives on the mbarrier once every product issued so far by this thread has completed.
__device__ __forceinline__ void commit_mma(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcCtl {
    int *status;        // set to SAL_ERR_TIMEOUT when a wait runs out
    int stall;          // test hook: no product is issued, so every wait must run out
    uint64_t limit_ns;  // bound of one wait
};

// One output tile on the tensor-core path.  Returns false when a wait ran out.
template <class G>
__device__ __forceinline__ bool energy_tile_tc(const float *__restrict__ V, int64_t T, int64_t X, int64_t Y, int bnd,
                                               int64_t tile, int tiles_x, int tiles_y, float *__restrict__ E,
                                               const SpecTables &tb, unsigned char *smem, uint32_t tmem,
                                               uint32_t &phase, const TcCtl &ctl)
{
    constexpr int L = G::L, H = G::H, P = G::P;
    float *sG1 = reinterpret_cast<float *>(smem);
    unsigned char *sA = smem + G::OFF_A;
    float *sV = reinterpret_cast<float *>(smem + G::OFF_A);   // aliases the operands until stage t is done
    float2 *ref = reinterpret_cast<float2 *>(smem + G::OFF_REF);
    float *xch = reinterpret_cast<float *>(smem + G::OFF_X);
    float *sW = reinterpret_cast<float *>(smem + G::OFF_W);
    fill_w<G>(sW, tb);
    const uint32_t bar = smem_u32(smem + G::OFF_BAR);
    const uint32_t a_addr = smem_u32(sA), b_addr = smem_u32(smem + G::OFF_B);

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
    // operand padding (K beyond the run, empty lines) must read as zero
    for (int i = threadIdx.x; i < G::A_BYTES / 16; i += G::NT) reinterpret_cast<uint4 *>(sA)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();

    // warpgroup g takes every other product of a round; within it, warp quarter q reads
    // tensor-memory lanes 32q..32q+31 = operand rows: line half, output row, segment
    const int g = threadIdx.x >> 7, q = (threadIdx.x >> 5) & 3;
    const int lane_row = threadIdx.x & 127;
    const int half = lane_row >> 6, rs = lane_row & 63;
    const uint32_t tq = tmem + ((uint32_t)(q * 32) << 16);
    float et[P], ex[P], ey[P];
#pragma unroll
    for (int o = 0; o < P; ++o) et[o] = ex[o] = ey[o] = 0.f;
    bool ok = true;

#pragma unroll 1
    for (int mu = 0; mu <= H && ok; ++mu) {
        build_a<G>(sG1, sA, ref, mu, tw);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        const int nl = nlines(mu, L), np = (nl + 1) / 2;
#pragma unroll 1
        for (int p0 = 0; p0 < np; p0 += G::PPR) {
            const int pend = p0 + G::PPR < np ? p0 + G::PPR : np;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (threadIdx.x == 0 && !ctl.stall) {
                for (int pr = p0; pr < pend; ++pr)
                    issue_mma<G>(tmem + (uint32_t)((pr - p0) * G::N), a_addr + pr * G::PAIR_BYTES, b_addr);
                commit_mma(bar);
            }
            // one thread watches the barrier (bounded); the others sleep in the CTA barrier
            // instead of taking issue slots from the co-resident CTA with polling
            const bool done = threadIdx.x == 0 ? mbar_wait(bar, phase, ctl.limit_ns) : true;
            if (__syncthreads_or(!done)) {
                ok = false;
                // products that were issued may still be in flight: give them one more bounded
                // wait before the caller releases the tensor memory
                if (!ctl.stall && threadIdx.x == 0) mbar_wait(bar, phase, ctl.limit_ns);
                break;
            }
            phase ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
            for (int pr = p0 + g; pr < pend; pr += 2) {
                const int li = 2 * pr + half;
                const bool valid = li < nl;                    // uniform per warp
                const int nu = nu_of_line(li, mu);
                const int anu = nu < 0 ? -nu : nu;
                const bool dc_line = mu == 0 && nu == 0;       // count omega > 0 only (its mirror is the factor 2)
                const float2 c = ref[pr * 128 + lane_row];
                // |F| summed over the signs of omega per (output, |omega|), then the weights
                float ms[P][H + 1];
#pragma unroll
                for (int o = 0; o < P; ++o)
#pragma unroll
                    for (int aw = 0; aw <= H; ++aw) ms[o][aw] = 0.f;
                const uint32_t taddr = tq + (uint32_t)((pr - p0) * G::N);
#pragma unroll
                for (int ch = 0; ch < L; ++ch) {
                    float v[16];
                    tmem_ld16(taddr + 16 * ch, v);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int idx = 8 * ch + u, o = idx / L, om = idx % L;
                        float re = v[2 * u], im = v[2 * u + 1];
                        if (om == H) {
                            re = fmaf((float)L, c.x, re);
                            im = fmaf((float)L, c.y, im);
                        }
                        const float mag = sqrt_approx(fmaf(re, re, im * im));
                        const int aw = om >= H ? om - H : H - om;
                        ms[o][aw] += (dc_line && om <= H) ? 0.f : mag;
                    }
                }
                if (valid) {
                    float w[H + 1][3];
                    load_w<G>(sW, mu, anu, w);
#pragma unroll
                    for (int o = 0; o < P; ++o)
#pragma unroll
                        for (int aw = 0; aw <= H; ++aw) {
                            et[o] = fmaf(w[aw][0], ms[o][aw], et[o]);
                            ex[o] = fmaf(w[aw][1], ms[o][aw], ex[o]);
                            ey[o] = fmaf(w[aw][2], ms[o][aw], ey[o]);
                        }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }
    if (!ok) return false;

    // four partial sets per (row, segment): two line halves x two warpgroups
    const int set = g * 2 + half;   // 0 writes the result
    if (set != 0) {
        float *xs = xch + (set - 1) * (3 * P * 64);
#pragma unroll
        for (int o = 0; o < P; ++o) {
            xs[(0 * P + o) * 64 + rs] = et[o];
            xs[(1 * P + o) * 64 + rs] = ex[o];
            xs[(2 * P + o) * 64 + rs] = ey[o];
        }
    }
    __syncthreads();
    if (set == 0) {
        const int row = rs / G::SEG, s = rs - row * G::SEG;
        const int t = row / G::BX, x = row - t * G::BX;
        const int64_t gt = t0 + t, gx = x0 + x, gy = y0 + P * s;
        if (gt < T && gx < X) {
            const int64_t N = T * X * Y;
            const float sc = tb.escale;
            float *e0 = E + (gt * X + gx) * Y + gy;
#pragma unroll
            for (int o = 0; o < P; ++o) {
                if (gy + o >= Y) break;
                float a0 = et[o], a1 = ex[o], a2 = ey[o];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float *xs = xch + k * (3 * P * 64);
                    a0 += xs[(0 * P + o) * 64 + rs];
                    a1 += xs[(1 * P + o) * 64 + rs];
                    a2 += xs[(2 * P + o) * 64 + rs];
                }
                e0[o] = a0 * sc;
                e0[o + N] = a1 * sc;
                e0[o + 2 * N] = a2 * sc;
            }
        }
    }
    __syncthreads();
    return true;
}

template <class G>
__global__ void __launch_bounds__(G::NT, 2) energy_tc_kernel(const __grid_constant__ EBatch bt,
                                                          const __grid_constant__ SpecTables tb, TcCtl ctl)
{
    extern __shared__ __align__(128) float tc_smem_f[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(tc_smem_f);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + G::OFF_BAR + 8);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(smem + G::OFF_BAR)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(G::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    build_b<G>(smem + G::OFF_B, tb);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    uint32_t phase = 0;
    for (int64_t k = blockIdx.x; k < bt.total; k += gridDim.x) {
        int lo = 0, hi = bt.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bt.v[mid].tile0 <= k) lo = mid; else hi = mid - 1;
        }
        const EVol &v = bt.v[lo];
        if (!energy_tile_tc<G>(v.V, v.T, v.X, v.Y, bt.bnd, k - v.tile0, v.tiles_x, v.tiles_y, v.E, tb, smem, tmem,
                               phase, ctl)) {
            if (threadIdx.x == 0) atomicExch(ctl.status, (int)SAL_ERR_TIMEOUT);
            break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::TMEM_COLS) : "memory");
}

template <class G>
cudaError_t launch_energy_tc_impl(const EVolDesc *vols, int n, int bnd, bool persistent, const TcCtl &ctl,
                                  cudaStream_t s)
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
        total += energy_tiles<G>(v.T, v.X, v.Y, &v.tiles_x, &v.tiles_y);
    }
    bt.total = total;
    if (total <= 0) return cudaSuccess;
    auto kern = energy_tc_kernel<G>;
    cudaError_t e = set_smem(kern, G::SMEM);
    if (e != cudaSuccess) return e;
    // one CTA per tile is far more than can be resident; walk the tiles persistently from
    // the resident CTAs (each holds its tensor memory for the whole launch)
    int dev = 0, nsm = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G::NT, G::SMEM);
    if (e != cudaSuccess) return e;
    (void)persistent;
    // the occupancy query can answer for a smaller shared-memory carveout than the launch
    // gets; size the persistent grid from the per-SM limits directly: shared memory (228 KB
    // per SM, 1 KB reserved per CTA), registers, and the 512 tensor-memory columns
    int smem_per_sm = 0, regs_per_sm = 0;
    cudaDeviceGetAttribute(&smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaFuncAttributes fa;
    int by_regs = 4;
    if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess && fa.numRegs > 0)
        by_regs = regs_per_sm / (((fa.numRegs + 7) / 8 * 8) * G::NT);
    const int by_smem = smem_per_sm > 0 ? smem_per_sm / (int)(G::SMEM + 1024) : 1;
    const int by_tmem = 512 / G::TMEM_COLS;
    per_sm = by_smem < by_regs ? by_smem : by_regs;
    if (per_sm > by_tmem) per_sm = by_tmem;
    int64_t grid = (int64_t)nsm * (per_sm > 0 ? per_sm : 1);
    if (grid > total) grid = total;
    kern<<<(unsigned)grid, G::NT, G::SMEM, s>>>(bt, tb, ctl);
    return cudaGetLastError();
}

}  // namespace energy_detail
}  // namespace sal
