// batch_hop_lo.cu -- instantiates the batched hop kernels for F32, F16 and
// BF16 spinors (batch_impl.cuh).
#include "batch_impl.cuh"

namespace wl {
namespace bt {
template void launch_bhop<P_F32, P_F32>(const BatchArgs&, const BOp&, int, int, int, int, cudaStream_t);
template void launch_bhop<P_F16, P_F16>(const BatchArgs&, const BOp&, int, int, int, int, cudaStream_t);
template void launch_bhop<P_BF16, P_BF16>(const BatchArgs&, const BOp&, int, int, int, int, cudaStream_t);
}  // namespace bt
}  // namespace wl
