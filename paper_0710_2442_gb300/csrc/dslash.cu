// dslash.cu -- host-side dispatch of the hopping-term kernels (device code in
// dslash_impl.cuh): picks the instantiation for the storage precisions and
// link format, and the launch configuration from the autotuner.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "dslash_impl.cuh"

namespace wl {

int device_sm_count() {
    static int sms[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!sms[dev]) {
        int n = 0;
        WL_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
        sms[dev] = n > 0 ? n : 1;
    }
    return sms[dev];
}

bool pdl_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("WILSON_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

int hop_grid_blocks(const Geom& g, int block, int grid_cap) {
    int blocks = (g.Vh + block - 1) / block;
    if (grid_cap > 0 && blocks > grid_cap) blocks = grid_cap;
    return blocks < 1 ? 1 : blocks;
}

static void dispatch(const HopParams& P, Prec sp, Prec gp, int R, int block, int site_blocks, int ny, bool dag,
                     int variant, cudaStream_t st) {
    const int blocks = site_blocks;
    if (sp == P_F64 && gp == P_F64 && R == 18) launch_hop_prec<P_F64, P_F64, 18>(P, block, blocks, ny, dag, variant, st);
    else if (sp == P_F64 && gp == P_F64 && R == 12) launch_hop_prec<P_F64, P_F64, 12>(P, block, blocks, ny, dag, variant, st);
    else if (sp == P_F32 && gp == P_F32 && R == 12) launch_hop_prec<P_F32, P_F32, 12>(P, block, blocks, ny, dag, variant, st);
    else if (sp == P_F32 && gp == P_F32 && R == 18) launch_hop_prec<P_F32, P_F32, 18>(P, block, blocks, ny, dag, variant, st);
    else if (sp == P_F16 && gp == P_F16 && R == 12) launch_hop_prec<P_F16, P_F16, 12>(P, block, blocks, ny, dag, variant, st);
    else if (sp == P_BF16 && gp == P_BF16 && R == 12) launch_hop_prec<P_BF16, P_BF16, 12>(P, block, blocks, ny, dag, variant, st);
    else if (sp == P_F16 && gp == P_F16 && R == 18) launch_hop_prec<P_F16, P_F16, 18>(P, block, blocks, ny, dag, variant, st);
    else if (sp == P_BF16 && gp == P_BF16 && R == 18) launch_hop_prec<P_BF16, P_BF16, 18>(P, block, blocks, ny, dag, variant, st);
    else throw Error(7, "unsupported spinor/gauge precision and link-storage combination");
}

void launch_hop(const HopLaunch& L, cudaStream_t st) {
    const GaugeField& gf = *L.gauge;
    HopParams P;
    P.out = static_cast<char*>(L.out);
    P.in = static_cast<const char*>(L.in);
    P.x = static_cast<const char*>(L.x);
    P.out_pstep = L.out_pstep;
    P.in_pstep = L.in_pstep;
    P.x_pstep = L.x_pstep;
    P.nrhs = L.nrhs > 1 ? L.nrhs : 1;
    P.out_rstep = L.out_rstep;
    P.in_rstep = L.in_rstep;
    P.x_rstep = L.x_rstep;
    P.skip_stride = L.skip_stride;
    P.gauge = gf.buf.as<const char>();
    P.g = gf.g;
    P.out_parity = L.out_parity;
    P.full = L.full;
    P.xpay = L.xpay;
    P.a = L.a;
    P.reduce = 0;
    P.red = RedArgs{};
    P.skip = L.skip;
    WL_REQUIRE(!L.xpay || L.x, "xpay needs a field");
    const int ny = L.full ? 2 : 1;
    const bool dag = L.dagger != 0;
    const Prec sp = L.sprec, gp = gf.prec;
    const int R = gf.recon;
    // the t-slab kernel takes one parity and one RHS, in tiles that divide the slice
    auto slab_ok = [&](int block) { return P.nrhs == 1 && !L.full && hop_slab_fits(P.g, block); };

    // The grid of a launch.  A reducing launch walks the lattice with a capped
    // grid (one partial per block, summed by the last block in a fixed
    // order): one resident wave of the block size, the blocks that the
    // variant's register budget guarantees on every SM, so no tail wave.
    auto grid_of = [&](const LaunchConfig& c) {
        int cap = 0;
        if (L.red) {
            const int per_sm = std::max(1, hop_variant_minb(c.variant, sp) * 256 / c.block);
            cap = std::min(L.grid_cap, device_sm_count() * per_sm);
        }
        return hop_grid_blocks(P.g, c.block * hop_variant_spt(c.variant), cap);
    };
    // the link-staged, tensor-core and t-slab kernels have no fused reduction
    auto reduces = [](int v) { return v != kHopStagedVariant && v != kHopMmaVariant && v != kHopSlabVariant; };

    LaunchConfig cfg;
    const char* forced = std::getenv("WILSON_HOP_VARIANT");  // pins the kernel (tests of each variant)
    if (L.block > 0) {
        cfg.block = L.block;
        cfg.variant = L.variant;
    } else if (forced && *forced) {
        cfg.variant = std::atoi(forced);
        const char* fb = std::getenv("WILSON_HOP_BLOCK");
        cfg.block = fb && std::atoi(fb) > 0 ? std::atoi(fb) : 128;
        WL_REQUIRE(cfg.variant >= 0 && cfg.variant < kHopVariants, "WILSON_HOP_VARIANT out of range");
        // a blocked variant that does not fit this launch falls back to variant 3
        if (!hop_variant_valid(cfg.variant, sp, R, P.nrhs)) cfg.variant = 3;
        if (cfg.variant == kHopSlabVariant && !slab_ok(cfg.block)) cfg.variant = 3;
        WL_REQUIRE(cfg.block == 64 || cfg.block == 128 || cfg.block == 256, "WILSON_HOP_BLOCK must be 64, 128 or 256");
    } else {
        // Reducing launches are their own launch kind (key suffix ":red"):
        // their grid is one capped wave, and the variant that streams best
        // over the whole lattice need not walk it best in a wave.
        char key[170];
        snprintf(key, sizeof(key), "hop:s%d:g%d:r%d:d%d:f%d:x%d:n%d:%dx%dx%dx%d%s", (int)sp, (int)gp, R, (int)dag,
                 L.full, L.xpay, P.nrhs, P.g.L[0], P.g.L[1], P.g.L[2], P.g.L[3], L.red ? ":red" : "");
        // tuning launches never reduce (the finishers are not idempotent):
        // a reducing launch is timed as its non-reducing copy on its own grid
        const HopParams Pt = P;
        std::vector<LaunchConfig> cands;
        for (const LaunchConfig& c : hop_candidates())  // FP64 has three register budgets, not six
            if (!wide_regs(sp) || c.variant < 3) cands.push_back(c);
        // two sites per thread, the F16 packed projection and pipeline, the
        // prefetching variants and the t-slab kernel where its tiles fit
        for (int block : {64, 128, 256})
            for (int v = kHopSptVariant; v < kHopVariants; v++)
                if ((hop_variant_is_ps(v) || hop_variant_is_pf(v) || (v == kHopSlabVariant && slab_ok(block))) &&
                    hop_variant_valid(v, sp, R, P.nrhs))
                    cands.push_back(LaunchConfig{block, v});
        if (P.nrhs > 1)
            for (int block : {64, 128, 256})
                for (int v = kHopBaseVariants; v < kHopVariants; v++)
                    if (!hop_variant_is_ps(v) && !hop_variant_is_pf(v) && v != kHopSlabVariant &&
                        hop_variant_valid(v, sp, R, P.nrhs))
                        cands.push_back(LaunchConfig{block, v});
        if (L.red) cands.erase(std::remove_if(cands.begin(), cands.end(),
                                              [&](const LaunchConfig& c) { return !reduces(c.variant); }),
                               cands.end());
        if (L.no_tune)
            cfg = tune_lookup(key, cands, LaunchConfig{});
        else
            cfg = tune_launch(key, cands, LaunchConfig{}, st, [&](const LaunchConfig& c) {
                dispatch(Pt, sp, gp, R, c.block, grid_of(c), ny, dag, c.variant, st);
            });
    }
    WL_REQUIRE(hop_variant_valid(cfg.variant, sp, R, P.nrhs), "hop variant does not fit this launch");
    // a pinned variant without a fused reduction: the paired kernel, same block
    if (L.red && !reduces(cfg.variant)) cfg.variant = 3;
    if (L.tune_only) return;
    if (L.red) {
        P.reduce = 1;
        P.red = *L.red;
        WL_REQUIRE(!L.full, "reducing hop launches are single-parity");
    }
    const int site_blocks = grid_of(cfg);
    WL_REQUIRE(!L.red || site_blocks <= L.red->slot_cap, "reduction capacity below the grid size");
    dispatch(P, sp, gp, R, cfg.block, site_blocks, ny, dag, cfg.variant, st);
    WL_LAUNCH_CHECK();
}

}  // namespace wl
