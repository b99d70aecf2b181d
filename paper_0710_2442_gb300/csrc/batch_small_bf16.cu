// batch_small_bf16.cu -- instantiates the CTA-resident small-lattice solver
// of the batch for BF16 inner storage (batch_impl.cuh).
#include "batch_impl.cuh"

namespace wl {
namespace bt {
template void launch_small_ip<P_BF16>(bool, const BatchArgs&, const int*, const BatchGlobal*, unsigned long long,
                                   int, cudaStream_t);
}  // namespace bt
}  // namespace wl
