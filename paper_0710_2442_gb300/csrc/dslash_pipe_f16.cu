// dslash_pipe_f16.cu -- instantiates the pipelined hopping-term kernels
// (dslash_pipe.cuh) for F16 storage in their own translation unit.
#include "dslash_pipe.cuh"

namespace wl {

template void launch_hop_pipe<P_F16>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_pipe2<P_F16>(const HopParams&, int, int, int, bool, int, cudaStream_t);

}  // namespace wl
