// FDM RHS pass / FDM-form pass 1, complex64 element arithmetic.
#include "ddh_k_fdm.cuh"

namespace ddh {

template void launch_pass1<float>(const DevModel&, const void*, const void*, const double2*, double, const double2*, int, void*, void*, int, const int*, cudaStream_t, const FdmCfg&);
template void set_pass1_limits<float>(int, int);
int fdm_qb_max(int pmax, int rb, bool fp64) { return fp64 ? fdm_qb<double>(pmax, rb) : fdm_qb<float>(pmax, rb); }

}  // namespace ddh
