// dslash_slab.cu -- the t-slab streaming even-odd hop (variant 26): the
// GPU form of the paper's main-memory layout with multiple buffering
// (Sec. 5, "Data in off-chip main memory"): the lattice is swept along the
// fourth direction and the input slices next to the one being computed stay
// in on-chip memory, so each input slice is fetched once for its two t-hops.
//
// A block owns a tile of T = blockDim.x consecutive half sites of one
// 3-d slice (T divides Lx Ly Lz / 2, so every tile lies in one slice and a
// site's t-neighbours sit at the same tile position one slice up or down:
// half index h +- Lx Ly Lz / 2) and sweeps tt consecutive slices.  Its shared
// memory holds a ring of four slices of the input field's tile, each the
// field's SoA rows for the tile (16-byte chunk rows, then the F16/BF16 scale
// row), filled by bulk asynchronous copies (cp.async.bulk, the TMA engine)
// that one thread issues and an mbarrier per slot completes.  Computing slice
// tc needs slices tc - 1 and tc + 1; when it is done, slice tc - 1's slot is
// refilled with slice tc + 3, two steps before it is needed.  The x, y and z
// hops read global memory as the plain kernel does; all eight links are
// prefetched into L2 when a thread takes its site.
//
// Every wait on an mbarrier is bounded (kWaitLimit polls with a 1 us
// suspend hint, about a second in all).  A thread whose wait gives up counts
// it in g_stage_timeouts (read by wilson_stage_timeouts) and stores NaN at its
// site, and the block stops its sweep after that step; thread 0 then waits,
// bounded again, for the copies it still has in flight before the block
// exits, so that no copy lands in shared memory the next block owns.  The
// failure-detection test sets WILSON_TEST_STAGE_TIMEOUT=1: the slots are then
// armed for their bytes but no copy is issued (a phase that nothing
// completes, with nothing in flight) and the waits give up after 4096 polls.
#include <cstdlib>

#include "dslash_impl.cuh"

namespace wl {

__device__ unsigned long long g_stage_timeouts = 0;

namespace {

constexpr int kSlots = 4;
constexpr int kWaitLimit = 1 << 20;
constexpr int kTestWaitLimit = 1 << 12;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
// One poll: true once the phase with the given parity has completed.
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(1000u)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, int limit) {
    for (int i = 0; i < limit; i++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// bytes (a multiple of 16) from global src to shared dst (both 16-byte
// aligned), completing transaction bytes on bar
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// The tile's stored spinor at position t of a slot (rows of T chunks), as
// the paired kernels hold it.
template <int SP>
__device__ __forceinline__ void slot_load(const unsigned char* slot, int T, int t, PSpinor& q, float& sc) {
    if constexpr (SP == P_F32) {
        const float4* b = reinterpret_cast<const float4*>(slot) + t;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float4 lo = b[(2 * c) * T], hi = b[(2 * c + 1) * T];
            q.re01[c] = make_float2(lo.x, lo.y);
            q.im01[c] = make_float2(lo.z, lo.w);
            q.re23[c] = make_float2(hi.x, hi.y);
            q.im23[c] = make_float2(hi.z, hi.w);
        }
        sc = 1.0f;
    } else {
        using LT = LowT<SP>;
        const uint4* b = reinterpret_cast<const uint4*>(slot) + t;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const uint4 d = b[c * T];
            q.re01[c] = LT::to_f2(d.x);
            q.im01[c] = LT::to_f2(d.y);
            q.re23[c] = LT::to_f2(d.z);
            q.im23[c] = LT::to_f2(d.w);
        }
        sc = reinterpret_cast<const float*>(slot + 48 * T)[t];
    }
}

// The two t-hops of an output site from the staged neighbour slices (the
// arithmetic of hop_dir_p for MU = 3).
template <int SP, int GP, int R, bool DAG>
__device__ __forceinline__ void hop_t_staged(PSpinor& acc, const HopParams& P, const unsigned char* up,
                                             const unsigned char* down, int T, int t, int p, int h, const int c[4],
                                             int s) {
    using GF = GaugeFmt<GP, R>;
    const Geom& g = P.g;
    const int Lt = g.L[3];
    const int smu = g.L[0] * g.L[1] * g.L[2];
    constexpr int SF_ = DAG ? -1 : 1;
    {
        PSpinor q;
        PHalf hh, w;
        cpx<float> U[3][3];
        float sc;
        slot_load<SP>(up, T, t, q, sc);
        GF::load(P.gauge, g.stride, p * 4 + 3, h, U);
        project_p<3, SF_>(q, hh);
        if (c[3] == Lt - 1) {
            const float er = (float)g.ph[3][0], ei = (float)g.ph[3][1];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float2 r = hh.re[k], m = hh.im[k];
                hh.re[k] = fma2(bc2(-ei), m, mul2(bc2(er), r));
                hh.im[k] = fma2(bc2(ei), r, mul2(bc2(er), m));
            }
        }
        su3_mul_p<false>(U, hh, w);
        expand_p<3, SF_, false>(acc, w, sc);
    }
    {
        const bool wrap = c[3] == 0;
        const int hn = (wrap ? s + (Lt - 1) * smu : s - smu) >> 1;
        PSpinor q;
        PHalf hh, w;
        cpx<float> U[3][3];
        float sc;
        slot_load<SP>(down, T, t, q, sc);
        GF::load(P.gauge, g.stride, (1 - p) * 4 + 3, hn, U);
        project_p<3, -SF_>(q, hh);
        if (wrap) {
            const float er = (float)g.ph[3][0], ei = -(float)g.ph[3][1];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float2 r = hh.re[k], m = hh.im[k];
                hh.re[k] = fma2(bc2(-ei), m, mul2(bc2(er), r));
                hh.im[k] = fma2(bc2(ei), r, mul2(bc2(er), m));
            }
        }
        su3_mul_p<true>(U, hh, w);
        expand_p<3, -SF_, false>(acc, w, sc);
    }
}

template <int SP>
constexpr unsigned slot_bytes_per_site() {
    return SpinorFmt<SP>::nchunk * SpinorFmt<SP>::chunk_bytes + (SpinorFmt<SP>::scaled ? 4 : 0);
}

// Grid: blockIdx.x = chunk * tiles + tile; chunk c sweeps slices [c tt, (c + 1) tt).
template <int SP, int GP, int R, bool DAG>
__global__ void __launch_bounds__(256, 2) hop_kernel_slab(const HopParams P, int tt, int wait_limit,
                                                           int no_copy) {
    using SF = SpinorFmt<SP>;
    constexpr int NS = SF::nchunk;
    extern __shared__ __align__(128) unsigned char slab_smem[];
    __shared__ __align__(8) unsigned long long bars[kSlots];
    __shared__ int abort_sweep;
    const int T = blockDim.x, t = threadIdx.x;
    const Geom& g = P.g;
    const int Lt = g.L[3];
    const int vs2 = g.L[0] * g.L[1] * (g.L[2] / 2);  // half sites per slice
    const int tiles = vs2 / T;
    const int tile = blockIdx.x % tiles;
    const int t0 = (blockIdx.x / tiles) * tt;
    const int p = P.out_parity;
    const unsigned slot_bytes = slot_bytes_per_site<SP>() * (unsigned)T;
    pdl_wait();
    if (P.skip && __ldcg(P.skip)) return;  // a converged right-hand side (block-uniform)
    const char* in = P.in;
    if (t == 0) {
        for (int i = 0; i < kSlots; i++) mbar_init(&bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_sweep = 0;
    }
    __syncthreads();
    // Slice ts of the input tile into slot (ts - t0 + 1) % 4 (thread 0 only);
    // fills[] counts each slot's fills, so its n-th fill completes phase n - 1.
    int fills[kSlots] = {0, 0, 0, 0};
    auto issue = [&](int ts) {
        const int rel = ts - t0 + 1;
        const int k = rel & (kSlots - 1);
        const int tw = (ts + Lt) % Lt;
        const long long h0 = (long long)tw * vs2 + (long long)tile * T;
        unsigned char* dst = slab_smem + (size_t)k * slot_bytes;
        mbar_expect_tx(&bars[k], slot_bytes);
        fills[k]++;
        if (no_copy) return;
#pragma unroll
        for (int r = 0; r < NS; r++)
            bulk_copy(dst + (size_t)r * 16 * T, in + ((long long)r * g.stride + h0) * 16, 16u * T, &bars[k]);
        if constexpr (SF::scaled)
            bulk_copy(dst + (size_t)NS * 16 * T, in + (long long)NS * 16 * g.stride + h0 * 4, 4u * T, &bars[k]);
    };
    if (t == 0)
        for (int ts = t0 - 1; ts <= t0 + 2 && ts <= t0 + tt; ts++) issue(ts);
    const char* x = P.x;
    const float a = (float)P.a;
    for (int tc = t0; tc < t0 + tt; tc++) {
        const int rdown = tc - t0, rup = tc - t0 + 2;  // slot-relative indices of slices tc -+ 1
        const unsigned char* down = slab_smem + (size_t)(rdown & (kSlots - 1)) * slot_bytes;
        const unsigned char* up = slab_smem + (size_t)(rup & (kSlots - 1)) * slot_bytes;
        const int h = tc * vs2 + tile * T + t;
        int c[4], s;
        site_of_half(h, p, g, c, s);
        hop_prefetch<SP, GP, R, 1>(P, in, p, h, c, s);
        PSpinor acc;
        hop_dir_p<SP, GP, R, DAG, 0, true>(acc, P, in, p, h, c, s);
        hop_dir_p<SP, GP, R, DAG, 1, false>(acc, P, in, p, h, c, s);
        hop_dir_p<SP, GP, R, DAG, 2, false>(acc, P, in, p, h, c, s);
        const bool ok = mbar_wait_bounded(&bars[rdown & (kSlots - 1)], (rdown >> 2) & 1, wait_limit) &&
                        mbar_wait_bounded(&bars[rup & (kSlots - 1)], (rup >> 2) & 1, wait_limit);
        if (ok) {
            hop_t_staged<SP, GP, R, DAG>(acc, P, up, down, T, t, p, h, c, s);
            if (P.xpay) {
                PSpinor xq;
                float xs;
                SF::load_packed(x, g.stride, h, xq, xs);
                const float2 A = bc2(a), X = bc2(xs);
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    acc.re01[cc] = fma2(A, acc.re01[cc], mul2(X, xq.re01[cc]));
                    acc.im01[cc] = fma2(A, acc.im01[cc], mul2(X, xq.im01[cc]));
                    acc.re23[cc] = fma2(A, acc.re23[cc], mul2(X, xq.re23[cc]));
                    acc.im23[cc] = fma2(A, acc.im23[cc], mul2(X, xq.im23[cc]));
                }
            } else if (P.a != 1.0) {
                const float2 A = bc2(a);
#pragma unroll
                for (int cc = 0; cc < 3; cc++) {
                    acc.re01[cc] = mul2(A, acc.re01[cc]);
                    acc.im01[cc] = mul2(A, acc.im01[cc]);
                    acc.re23[cc] = mul2(A, acc.re23[cc]);
                    acc.im23[cc] = mul2(A, acc.im23[cc]);
                }
            }
        } else {
            atomicAdd(&g_stage_timeouts, 1ULL);
            abort_sweep = 1;
            const float2 nan2 = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
#pragma unroll
            for (int cc = 0; cc < 3; cc++) acc.re01[cc] = acc.im01[cc] = acc.re23[cc] = acc.im23[cc] = nan2;
        }
        SF::store_packed(P.out, g.stride, h, acc);
        __syncthreads();  // every thread is done with slice tc - 1's slot
        if (abort_sweep) break;
        if (t == 0 && tc + 3 <= t0 + tt) issue(tc + 3);
    }
    pdl_trigger();
    // copies still in flight (only after an abandoned sweep): wait for them,
    // bounded, before the block's shared memory is released
    if (t == 0)
        for (int k = 0; k < kSlots; k++)
            if (fills[k] > 0) (void)mbar_wait_bounded(&bars[k], (fills[k] - 1) & 1, wait_limit);
}

}  // namespace

// Slices per block: the largest of 8, 4, 2 dividing Lt.
int slab_slices_per_block(const Geom& g) { return g.L[3] % 8 == 0 ? 8 : g.L[3] % 4 == 0 ? 4 : 2; }

bool hop_slab_fits(const Geom& g, int block) {
    const long long vs2 = (long long)g.L[0] * g.L[1] * g.L[2] / 2;
    return (block == 64 || block == 128 || block == 256) && vs2 % block == 0 && g.L[3] >= 2;
}

template <int SP, int GP, int R>
void launch_hop_slab(const HopParams& P, int block, bool dag, cudaStream_t st) {
    WL_REQUIRE(hop_slab_fits(P.g, block), "the slab hop needs a tile that divides the 3-d slice");
    WL_REQUIRE(P.nrhs == 1 && !P.full && !P.reduce, "the slab hop takes one parity and one RHS, unreduced");
    const int tt = slab_slices_per_block(P.g);
    const int tiles = P.g.L[0] * P.g.L[1] * (P.g.L[2] / 2) / block;
    const dim3 grid(tiles * (P.g.L[3] / tt));
    const size_t smem = (size_t)kSlots * slot_bytes_per_site<SP>() * block;
    auto k = dag ? hop_kernel_slab<SP, GP, R, true> : hop_kernel_slab<SP, GP, R, false>;
    static bool opted[64][2] = {};  // the larger dynamic shared memory, once per device and dagger
    int dev = 0;
    WL_CUDA(cudaGetDevice(&dev));
    WL_REQUIRE(dev >= 0 && dev < 64, "device ordinal out of range");
    if (!opted[dev][dag]) {
        WL_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kSlots * slot_bytes_per_site<SP>() * 256)));
        opted[dev][dag] = true;
    }
    const char* test = std::getenv("WILSON_TEST_STAGE_TIMEOUT");
    const bool short_fill = test && std::atoi(test) == 1;
    launch_dep_smem(k, grid, dim3(block), smem, st, P, tt, short_fill ? kTestWaitLimit : kWaitLimit,
                    short_fill ? 1 : 0);
}

#define WL_SLAB(SP, R) template void launch_hop_slab<SP, SP, R>(const HopParams&, int, bool, cudaStream_t);
WL_SLAB(P_F32, 12)
WL_SLAB(P_F32, 18)
WL_SLAB(P_F16, 12)
WL_SLAB(P_F16, 18)
WL_SLAB(P_BF16, 12)
WL_SLAB(P_BF16, 18)
#undef WL_SLAB

unsigned long long stage_timeouts(cudaStream_t st) {
    unsigned long long v = 0;
    WL_CUDA(cudaMemcpyFromSymbolAsync(&v, g_stage_timeouts, sizeof(v), 0, cudaMemcpyDeviceToHost, st));
    WL_CUDA(cudaStreamSynchronize(st));
    return v;
}

}  // namespace wl

extern "C" int wilson_stage_timeouts(unsigned long long* count, void* stream) {
    try {
        WL_REQUIRE(count != nullptr, "count is NULL");
        wl::check_device();
        *count = wl::stage_timeouts(static_cast<cudaStream_t>(stream));
        wl::record_error("");
        return WILSON_OK;
    } catch (const wl::Error& e) {
        wl::record_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        wl::record_error(e.what());
        return WILSON_ERR_CUDA;
    }
}
