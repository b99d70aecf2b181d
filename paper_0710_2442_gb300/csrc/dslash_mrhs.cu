// dslash_mrhs.cu -- instantiates the register-blocked multi-RHS hopping-term
// kernels (see dslash_impl.cuh) in their own translation unit, so that they
// compile in parallel with the single-RHS families.
#include "dslash_impl.cuh"

namespace wl {

template <int SP, int GP, int R>
void launch_hop_mrhs(const HopParams& P, int block, int site_blocks, int ny, bool dag, int variant,
                     cudaStream_t st) {
    switch (variant) {
        case 6: launch_hop_mrhs_v<SP, GP, R, 6>(P, block, site_blocks, ny, dag, st); break;
        case 7: launch_hop_mrhs_v<SP, GP, R, 7>(P, block, site_blocks, ny, dag, st); break;
        case 8: launch_hop_mrhs_v<SP, GP, R, 8>(P, block, site_blocks, ny, dag, st); break;
        case 9: launch_hop_mrhs_v<SP, GP, R, 9>(P, block, site_blocks, ny, dag, st); break;
        case 10: launch_hop_rl_v<SP, GP, R, 10>(P, block, site_blocks, ny, dag, st); break;
        case 18:
        case 19:
            if constexpr (SP == P_F16) {
                if (variant == 18) launch_hop_mrhs_v<SP, GP, R, 18>(P, block, site_blocks, ny, dag, st);
                else launch_hop_mrhs_v<SP, GP, R, 19>(P, block, site_blocks, ny, dag, st);
                break;
            }
            throw Error(7, "the packed-projection multi-RHS variants need F16 spinors");
        case kHopMmaVariant:
            if constexpr ((SP == P_F16 || SP == P_BF16) && GP == SP && R == 12) {
                launch_hop_mma<SP>(P, block, site_blocks, ny, dag, st);
                break;
            }
            throw Error(7, "the tensor-core hop variant needs F16/BF16 spinors and 12-real links");
        default: throw Error(7, "unknown register-blocked hop variant");
    }
}

template void launch_hop_mrhs<P_F32, P_F32, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_mrhs<P_F16, P_F16, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);
template void launch_hop_mrhs<P_BF16, P_BF16, 12>(const HopParams&, int, int, int, bool, int, cudaStream_t);

}  // namespace wl
