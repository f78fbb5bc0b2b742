// FP32 spectral-energy kernel instantiated for L = 9, one kernel per candidate (tile shape,
// staging mode) in the order of the shape table (one translation unit per cube size).
#include "energy_fp32.cuh"

namespace sal {

cudaError_t launch_energy_fp32_l9(const EVolDesc *vols, int n, int bnd, int shape, bool persistent, cudaStream_t s)
{
    switch (shape) {
        case 0: return energy_detail::launch_energy_impl<energy_detail::EGeo<9, 2, 8, 4>>(vols, n, bnd, persistent, s);
        case 1: return energy_detail::launch_energy_impl<energy_detail::EGeo<9, 2, 8>>(vols, n, bnd, persistent, s);
        case 2: return energy_detail::launch_energy_impl<energy_detail::EGeo<9, 2, 16>>(vols, n, bnd, persistent, s);
        case 3: return energy_detail::launch_energy_impl<energy_detail::EGeo<9, 1, 16>>(vols, n, bnd, persistent, s);
        default: return cudaErrorInvalidValue;
    }
}

// The tiles of a device-side list use candidate 0's geometry (the tile numbering of energy_shape(L, 0);
// mode 0 staging, the same tiles as candidate 0's mode 4).
cudaError_t launch_energy_fp32_list_l9(const float *V, sal_dims d, int bnd, const int64_t *list, const int *count,
                                        float *E, cudaStream_t s)
{
    return energy_detail::launch_energy_list_impl<energy_detail::EGeo<9, 2, 8>>(V, d, bnd, list, count, E, s);
}

}  // namespace sal
