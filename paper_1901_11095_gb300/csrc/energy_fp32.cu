// Dispatch of the FP32 spectral-energy kernel on the cube side L.
#include "sal_internal.cuh"

namespace sal {

cudaError_t launch_energy_fp32_l3(const float *V, sal_dims d, int bnd, float *E, cudaStream_t s);
cudaError_t launch_energy_fp32_l5(const float *V, sal_dims d, int bnd, float *E, cudaStream_t s);
cudaError_t launch_energy_fp32_l7(const float *V, sal_dims d, int bnd, float *E, cudaStream_t s);
cudaError_t launch_energy_fp32_l9(const float *V, sal_dims d, int bnd, float *E, cudaStream_t s);
cudaError_t launch_energy_fp32_l11(const float *V, sal_dims d, int bnd, float *E, cudaStream_t s);
cudaError_t launch_energy_fp32_l13(const float *V, sal_dims d, int bnd, float *E, cudaStream_t s);
cudaError_t launch_energy_fp32_l15(const float *V, sal_dims d, int bnd, float *E, cudaStream_t s);

cudaError_t launch_energy_fp32(const float *V, sal_dims d, int L, int bnd, float *E, cudaStream_t s)
{
    switch (L) {
        case 3: return launch_energy_fp32_l3(V, d, bnd, E, s);
        case 5: return launch_energy_fp32_l5(V, d, bnd, E, s);
        case 7: return launch_energy_fp32_l7(V, d, bnd, E, s);
        case 9: return launch_energy_fp32_l9(V, d, bnd, E, s);
        case 11: return launch_energy_fp32_l11(V, d, bnd, E, s);
        case 13: return launch_energy_fp32_l13(V, d, bnd, E, s);
        case 15: return launch_energy_fp32_l15(V, d, bnd, E, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sal
