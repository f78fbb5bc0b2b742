// Internal declarations shared by the CUDA translation units of libsal.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sal.h"

namespace sal {

constexpr int kMaxL = 15;
constexpr int kMaxH = (kMaxL - 1) / 2;
constexpr int kMaxHalf = kMaxH + 1;

// Per-L tables the kernels read from the parameter constant bank.
//   cs[n], sn[n] = cos(2 pi n / L), sin(2 pi n / L), n = 0..L-1
//   w[((mu*kMaxHalf + |nu|)*kMaxHalf + |om|)*3 + m] = projection weight of Eq. 1-4 for
//   map m at (mu, +-nu, +-om), mu >= 0 (the weights depend on squares only)
//   escale = 2 / ((L^3 - 1) L^3): DFT normalisation L^-3, the non-DC mean (L^3-1)^-1 and
//   the factor 2 of the half spectrum (|F(-k)| = |F(k)| for real input)
struct SpecTables {
    float cs[16];
    float sn[16];
    float w[kMaxHalf * kMaxHalf * kMaxHalf * 3];
    float escale;
};

// Fills the tables on the host (double precision, then rounded).
void make_tables(int L, SpecTables *t);

// Boundary extension of one coordinate onto 0..n-1 (REFLECT: whole-sample symmetric,
// edge not repeated; PERIODIC: wrap).  Valid for any integer i.
__host__ __device__ __forceinline__ int64_t ext_index(int64_t i, int64_t n, int bnd)
{
    if (i >= 0 && i < n) return i;
    if (bnd == SAL_BND_PERIODIC) {
        int64_t r = i % n;
        return r < 0 ? r + n : r;
    }
    if (n == 1) return 0;
    int64_t period = 2 * (n - 1);
    int64_t r = i % period;
    if (r < 0) r += period;
    return r < n ? r : period - r;
}

// Launchers (return cudaGetLastError() of the launch).
cudaError_t launch_energy_fp32(const float *V, sal_dims d, int L, int bnd, float *E, cudaStream_t s);
cudaError_t launch_local_spectra(const float *V, sal_dims d, int L, int bnd, const int64_t lo[3],
                                 const int64_t ext[3], float *mag, cudaStream_t s);
cudaError_t launch_project(const float *mag, int64_t n, int L, float *E, cudaStream_t s);

// Directional compare: number of per-CTA partial records written to the workspace.
int64_t dcs_num_partials(sal_dims d);
cudaError_t launch_dcs(const float *E, sal_dims d, const sal_params *p, float *Sm, double *partials,
                       double *stats, cudaStream_t s);
// Fixed-scratch variant of the directional compare (no allocation by caller or library).
int64_t dcs_num_tiles(sal_dims d);
cudaError_t dcs_static_scratch(double **out);
cudaError_t launch_combine(const float *Sm, const double *stats, sal_dims d, const sal_params *p, float *S,
                           cudaStream_t s);

}  // namespace sal
