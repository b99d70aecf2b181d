// probe.cu -- wilson_probe_fma_peak: the peak FP throughput of the device
// for one kind of fused multiply-add, measured by a throughput kernel.
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

}  // namespace

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
