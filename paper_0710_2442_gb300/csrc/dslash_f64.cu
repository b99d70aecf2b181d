// dslash_f64.cu -- instantiates the hopping-term kernels for one storage
// precision family (see dslash_impl.cuh), so that the families compile in
// parallel.
#include "dslash_impl.cuh"

namespace wl {
template void launch_hop_prec<P_F64, P_F64, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_prec<P_F64, P_F64, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
}  // namespace wl
