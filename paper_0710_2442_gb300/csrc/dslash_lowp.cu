// dslash_lowp.cu -- instantiates the hopping-term kernels for one storage
// precision family (see dslash_impl.cuh), so that the families compile in
// parallel.
#include "dslash_impl.cuh"

namespace wl {
template void launch_hop_prec<P_F16, P_F16, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_prec<P_BF16, P_BF16, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_prec<P_F16, P_F16, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_prec<P_BF16, P_BF16, 18>(const HopParams&, int, int, int, bool, int, cudaStream_t);
}  // namespace wl
