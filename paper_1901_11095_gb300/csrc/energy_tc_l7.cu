// Tensor-core spectral-energy kernel instantiated for L = 7 (BF16 and TF32 operands).
#include "energy_tc.cuh"

namespace sal {

cudaError_t launch_energy_tc_l7(const EVolDesc *vols, int n, int bnd, int prec, bool persistent, const TcControl &c,
                                 cudaStream_t s)
{
    const energy_detail::TcCtl ctl{c.status, c.stall, c.limit_ns};
    switch (prec) {
        case SAL_PREC_BF16: return energy_detail::launch_energy_tc_impl<energy_detail::TGeo<7, 2, 8, energy_detail::OpBF16>>(vols, n, bnd, persistent, ctl, s);
        case SAL_PREC_TF32: return energy_detail::launch_energy_tc_impl<energy_detail::TGeo<7, 2, 8, energy_detail::OpTF32>>(vols, n, bnd, persistent, ctl, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sal
