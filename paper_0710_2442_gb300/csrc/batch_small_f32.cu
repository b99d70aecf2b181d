// batch_small_f32.cu -- instantiates the CTA-resident small-lattice solver
// of the batch for F32 inner storage (batch_impl.cuh).
#include "batch_impl.cuh"

namespace wl {
namespace bt {
template void launch_small_ip<P_F32>(bool, const BatchArgs&, const int*, const BatchGlobal*, unsigned long long,
                                   int, cudaStream_t);
}  // namespace bt
}  // namespace wl
