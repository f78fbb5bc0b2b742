// FP32 spectral-energy kernel instantiated for L = 7 (one translation unit per cube size).
#include "energy_fp32.cuh"

namespace sal {

cudaError_t launch_energy_fp32_l7(const float *V, sal_dims d, int bnd, float *E, cudaStream_t s)
{
    return energy_detail::launch_energy_impl<energy_detail::EGeo<7, 2, 8>>(V, d, bnd, E, s);
}

}  // namespace sal
