// FDM RHS pass / FDM-form pass 1, complex128 element arithmetic.
#include "ddh_k_fdm.cuh"

namespace ddh {

template void launch_pass1<double>(const DevModel&, const void*, const void*, const double2*, double, const double2*, int, void*, void*, int, const int*, cudaStream_t, const FdmCfg&);
template void set_pass1_limits<double>(int, int);

}  // namespace ddh
