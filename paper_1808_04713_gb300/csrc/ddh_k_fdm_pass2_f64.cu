// FDM recovery / FDM-form pass 2, complex128 element arithmetic.
#include "ddh_k_fdm.cuh"

namespace ddh {

template void launch_pass2<double>(const DevModel&, const void*, const void*, const double2*, const void*, void*, int, const double2*, int, double2*, int, const int*, cudaStream_t, const FdmCfg&);
template void set_pass2_limits<double>(int, int);

}  // namespace ddh
