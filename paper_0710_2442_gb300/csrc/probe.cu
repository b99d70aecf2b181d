// probe.cu -- measurement probes: wilson_probe_fma_peak, the peak FP
// throughput of the device for one kind of fused multiply-add, and
// wilson_probe_hop_access, the time of the even-odd hop's memory accesses
// with the arithmetic taken out.
//
// The paper's efficiency measure (Sec. 3, Eq. 2 and the text after it) sets
// the execution time against T_peak, the time the FP operations would take
// at the machine's peak FP rate.  The FP64 and FP32 rates of a GB300 are not
// published in a form this library can trust (FP64 runs at a small fraction
// of the FP32 rate on this part), so the library measures them: every
// thread of a grid of resident blocks on every SM runs eight independent
// FMA chains (enough to cover the pipeline latency) for a fixed number of
// iterations, and the rate is the FMA count x 2 flops (x 2 lanes for the
// paired FP32 instruction) over the kernel's CUDA-event time.  The chains
// feed one store per thread, so nothing folds away.  Every loop is bounded.
#include <algorithm>
#include <cstdio>
#include <string>

#include "../../include/wilson.h"
#include "internal.h"

using namespace wl;

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) fma_probe_f64(double* out, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma_probe_f32(float* out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = 1.0f + 1e-3f * (threadIdx.x + k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma_probe_f32x2(float* out, int iters, float a, float b) {
    float2 x[kChains];
    const float2 A = make_float2(a, a), B = make_float2(b, b);
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = make_float2(1.0f + 1e-3f * (threadIdx.x + k), 1.0f - 1e-3f * k);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = __ffma2_rn(x[k], A, B);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k].x + x[k].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The memory-access pattern of the even-odd hop (Eq. 3), with trivial
// arithmetic.  The paper benchmarked the access pattern of Eq. 3 on its
// hardware and found it within 20 % of its model's memory time T_mem
// (Sec. 5, after Table 1); this is the same benchmark on a GPU.  Each thread
// takes one output site of parity p, exactly as the hop kernels do: the eight
// neighbours' spinor rows of parity 1 - p (periodic wrap) through the
// read-only path, the eight links (the site's forward links, the neighbours'
// backward ones) as streaming loads, one store of the output site's rows.
// Every loaded word is folded by XOR or add into one accumulator per output
// word (as the hop accumulates one output spinor), so no load is dead and
// the loads of different rows stay independent; the accumulators are stored
// in place of the spinor.  Like the hop, the probe comes in register budgets
// (MINB resident 256-thread blocks per SM; 0: no bound), since the budget
// decides how many loads a thread keeps in flight; the call reports the
// fastest budget and block size.
//
// Field rows (bytes per site, SoA, stride g.stride sites between rows):
//   spinor: NS16 rows of 16 bytes, then SC4 rows of 4 (the F16/BF16 scale);
//   link block blk = parity * 4 + mu: NL16 rows of 16, NL8 of 8, NL4 of 4.
template <int NS16, int SC4, int NL16, int NL8, int NL4, int MINB>
__global__ void __launch_bounds__(256, MINB) hop_access_probe(char* out, const char* in, const char* gauge,
                                                              const Geom g, int p) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    constexpr long long kLinkBytes = 16 * NL16 + 8 * NL8 + 4 * NL4;
    const long long stride = g.stride;
    int c[4], s;
    site_of_half(h, p, g, c, s);
    uint4 acc[NS16];
#pragma unroll
    for (int k = 0; k < NS16; k++) acc[k] = make_uint4(0u, 0u, 0u, 0u);
    unsigned la = 0, lb = 0;
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
        const int L = g.L[mu];
        const int smu = mu == 0 ? 1 : mu == 1 ? g.L[0] : mu == 2 ? g.L[0] * g.L[1] : g.L[0] * g.L[1] * g.L[2];
#pragma unroll
        for (int d = 0; d < 2; d++) {
            const bool fwd = d == 0;
            const bool wrap = fwd ? c[mu] == L - 1 : c[mu] == 0;
            const int n = (fwd ? (wrap ? s - (L - 1) * smu : s + smu) : (wrap ? s + (L - 1) * smu : s - smu)) >> 1;
#pragma unroll
            for (int k = 0; k < NS16; k++) {
                const uint4 v = __ldg(reinterpret_cast<const uint4*>(in + 16 * k * stride) + n);
                acc[k].x ^= v.x, acc[k].y ^= v.y, acc[k].z ^= v.z, acc[k].w ^= v.w;
            }
            if (SC4) la += __ldg(reinterpret_cast<const unsigned*>(in + 16 * NS16 * stride) + n);
            const char* lk = gauge + ((fwd ? p : 1 - p) * 4 + mu) * kLinkBytes * stride;
            const int li = fwd ? h : n;
#pragma unroll
            for (int k = 0; k < NL16; k++) {
                const uint4 v = __ldcs(reinterpret_cast<const uint4*>(lk + 16 * k * stride) + li);
                acc[k % NS16].x += v.x, acc[k % NS16].y += v.y, acc[k % NS16].z += v.z, acc[k % NS16].w += v.w;
            }
#pragma unroll
            for (int k = 0; k < NL8; k++) {
                const uint2 v = __ldcs(reinterpret_cast<const uint2*>(lk + (16 * NL16 + 8 * k) * stride) + li);
                acc[k % NS16].x += v.x, acc[k % NS16].y += v.y;
            }
#pragma unroll
            for (int k = 0; k < NL4; k++)
                lb += __ldcs(reinterpret_cast<const unsigned*>(lk + (16 * NL16 + 8 * NL8 + 4 * k) * stride) + li);
        }
    }
    acc[0].x += lb;
#pragma unroll
    for (int k = 0; k < NS16; k++) reinterpret_cast<uint4*>(out + 16 * k * stride)[h] = acc[k];
    if (SC4) reinterpret_cast<unsigned*>(out + 16 * NS16 * stride)[h] = la;
}

using AccessKernel = void (*)(char*, const char*, const char*, const Geom, int);

// The probe instances whose rows are those of a field of precision sp with
// recon-real links (the layouts of the spinor and gauge formats), at register
// budget index b: no bound, then 4, 3 and 2 blocks per SM (64, 80, 128
// registers).
constexpr int kAccessBudgets = 4;
template <int NS16, int SC4, int NL16, int NL8, int NL4>
AccessKernel access_budget(int b) {
    return b == 0   ? hop_access_probe<NS16, SC4, NL16, NL8, NL4, 0>
           : b == 1 ? hop_access_probe<NS16, SC4, NL16, NL8, NL4, 4>
           : b == 2 ? hop_access_probe<NS16, SC4, NL16, NL8, NL4, 3>
                    : hop_access_probe<NS16, SC4, NL16, NL8, NL4, 2>;
}
AccessKernel access_kernel(Prec sp, int recon, int b) {
    switch (sp) {
        case P_F64: return recon == 12 ? access_budget<12, 0, 6, 0, 0>(b) : access_budget<12, 0, 9, 0, 0>(b);
        case P_F32: return recon == 12 ? access_budget<6, 0, 3, 0, 0>(b) : access_budget<6, 0, 0, 9, 0>(b);
        default: return recon == 12 ? access_budget<3, 1, 0, 3, 0>(b) : access_budget<3, 1, 2, 0, 1>(b);
    }
}

}  // namespace

extern "C" int wilson_probe_hop_access(wilson_spinor* out, const wilson_gauge* gh, const wilson_spinor* in, int reps,
                                       double* seconds, void* stream) {
    try {
        WL_REQUIRE(out && gh && in && seconds, "NULL argument");
        WL_REQUIRE(out != in, "out must not be in");
        WL_REQUIRE(reps >= 1 && reps <= 100000, "reps must be in [1, 100000]");
        const GaugeField& gf = gh->f;
        const SpinorField& a = in->f;
        const SpinorField& b = out->f;
        for (int mu = 0; mu < 4; mu++)
            WL_REQUIRE(a.g.L[mu] == gf.g.L[mu] && b.g.L[mu] == gf.g.L[mu], "lattice mismatch");
        WL_REQUIRE(a.prec == b.prec && gf.prec == a.prec, "gauge, in and out precisions differ");
        WL_REQUIRE(a.nrhs == 1 && b.nrhs == 1, "the probe takes one right-hand side");
        WL_REQUIRE(a.subset != 2 && b.subset == 1 - a.subset, "the probe maps parity 1-p to parity p");
        WL_REQUIRE(gf.recon == 12 || gf.recon == 18, "links must have 12 or 18 reals");
        check_device();
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const Geom& g = gf.g;
        const int p = b.subset;
        char* o = static_cast<char*>(b.block(p));
        const char* i = static_cast<const char*>(a.block(a.subset));
        const char* u = gf.buf.as<const char>();
        cudaEvent_t e0, e1;
        WL_CUDA(cudaEventCreate(&e0));
        WL_CUDA(cudaEventCreate(&e1));
        double best = 1e30;
        for (int budget = 0; budget < kAccessBudgets; budget++) {
            const AccessKernel k = access_kernel(a.prec, gf.recon, budget);
            for (int block : {64, 128, 256}) {
                const int grid = (g.Vh + block - 1) / block;
                for (int w = 0; w < 3; w++) k<<<grid, block, 0, st>>>(o, i, u, g, p);
                WL_LAUNCH_CHECK();
                WL_CUDA(cudaEventRecord(e0, st));
                for (int r = 0; r < reps; r++) k<<<grid, block, 0, st>>>(o, i, u, g, p);
                WL_CUDA(cudaEventRecord(e1, st));
                WL_CUDA(cudaEventSynchronize(e1));
                WL_LAUNCH_CHECK();
                float ms = 0.f;
                WL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                best = std::min(best, ms * 1e-3 / reps);
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *seconds = best;
        record_error("");
        return WILSON_OK;
    } catch (const Error& e) {
        record_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        record_error(e.what());
        return WILSON_ERR_CUDA;
    }
}

extern "C" int wilson_probe_fma_peak(int kind, double* gflops, void* stream) {
    try {
        WL_REQUIRE(gflops != nullptr, "gflops is NULL");
        WL_REQUIRE(kind >= WILSON_PROBE_FMA_F64 && kind <= WILSON_PROBE_FMA_F32X2, "unknown probe kind");
        check_device();
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const int sms = device_sm_count();
        const int threads = 256, blocks = sms * 8;  // 2048 threads per SM: full occupancy
        // iterations per thread: about 50-100 ms per launch at the expected rates
        const int iters = kind == WILSON_PROBE_FMA_F64 ? 40000 : kind == WILSON_PROBE_FMA_F32 ? 400000 : 300000;
        DevBuf out((size_t)blocks * threads * sizeof(double));
        cudaEvent_t e0, e1;
        WL_CUDA(cudaEventCreate(&e0));
        WL_CUDA(cudaEventCreate(&e1));
        auto launch = [&] {
            if (kind == WILSON_PROBE_FMA_F64)
                fma_probe_f64<<<blocks, threads, 0, st>>>(out.as<double>(), iters, 0.999999, 1e-6);
            else if (kind == WILSON_PROBE_FMA_F32)
                fma_probe_f32<<<blocks, threads, 0, st>>>(out.as<float>(), iters, 0.999999f, 1e-6f);
            else
                fma_probe_f32x2<<<blocks, threads, 0, st>>>(out.as<float>(), iters, 0.999999f, 1e-6f);
        };
        launch();  // warm-up
        WL_LAUNCH_CHECK();
        float best = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
            WL_CUDA(cudaEventRecord(e0, st));
            launch();
            WL_CUDA(cudaEventRecord(e1, st));
            WL_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            WL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) best = ms;
        }
        WL_LAUNCH_CHECK();
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        const double lanes = kind == WILSON_PROBE_FMA_F32X2 ? 2.0 : 1.0;
        const double flops = 2.0 * lanes * kChains * (double)iters * threads * (double)blocks;
        *gflops = flops / (best * 1e-3) / 1e9;
        record_error("");
        return WILSON_OK;
    } catch (const Error& e) {
        record_error(e.what());
        return e.code;
    } catch (const std::exception& e) {
        record_error(e.what());
        return WILSON_ERR_CUDA;
    }
}
