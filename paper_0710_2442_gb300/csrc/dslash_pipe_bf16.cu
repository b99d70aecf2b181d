// dslash_pipe_bf16.cu -- instantiates the pipelined hopping-term kernels
// (dslash_pipe.cuh) for BF16 storage in their own translation unit.
#include "dslash_pipe.cuh"

namespace wl {

template void launch_hop_pipe<P_BF16>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_pipe2<P_BF16>(const HopParams&, int, int, int, bool, int, cudaStream_t);

}  // namespace wl
