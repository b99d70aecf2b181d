// batch_hop_64.cu -- instantiates the batched hop kernels for FP64 spinors
// (batch_impl.cuh).
#include "batch_impl.cuh"

namespace wl {
namespace bt {
template void launch_bhop<P_F64, P_F64>(const BatchArgs&, const BOp&, int, int, int, int, cudaStream_t);
}  // namespace bt
}  // namespace wl
