// layout.cu -- canonical complex128 fields <-> the library's SoA formats.
//
// Canonical: spinor [site][spin][colour], gauge [site][mu][row][col], complex
// as (re, im) doubles, site s = x + Lx*(y + Ly*(z + Lz*t)); half fields hold
// the sites of one parity at index s >> 1.
//
// Spinors: F64 (12 x 16 B chunks), F32 (6 x 16 B), F16/BF16 (3 x 16 B plus an
// FP32 per-site scale = the largest |component|; the stored values are
// component / scale rounded to nearest even).  Links: rows 0 and 1 only for
// 12-real storage (row 2 is rebuilt in the kernels, exact for SU(3)); links
// are never scaled (|U_ij| <= 1).
#include "internal.h"

namespace wl {

Geom make_geom(const int dims[4], const double ph[4][2]) {
    Geom g;
    long long V = 1;
    for (int mu = 0; mu < 4; mu++) {
        g.L[mu] = dims[mu];
        V *= dims[mu];
        g.ph[mu][0] = ph[mu][0];
        g.ph[mu][1] = ph[mu][1];
    }
    g.Vh = (int)(V / 2);
    g.stride = round_up(g.Vh, 64);
    for (int k = 0; k < 3; k++) div_magic(dims[k], g.dm[k], g.ds[k]);
    return g;
}

long long spinor_field_bytes(Prec p, int stride) {
    switch (p) {
        case P_F64: return SpinorFmt<P_F64>::field_bytes(stride);
        case P_F32: return SpinorFmt<P_F32>::field_bytes(stride);
        default: return SpinorFmt<P_F16>::field_bytes(stride);
    }
}

long long gauge_block_bytes(Prec p, int recon, int stride) {
    int per_link = (p == P_F64 ? 8 : p == P_F32 ? 4 : 2) * recon;
    return (long long)per_link * stride;
}

long long gauge_bytes(Prec p, int recon, int stride) { return 8 * gauge_block_bytes(p, recon, stride); }

void SpinorField::alloc(Prec p, int sub, int nr, const Geom& geom) {
    prec = p;
    subset = sub;
    nrhs = nr;
    g = geom;
    pbytes = (spinor_field_bytes(p, g.stride) + 255) / 256 * 256;
    buf.alloc((size_t)pbytes * nparity() * nrhs);
}

// ---------------------------------------------------------------------------
// spinors
// ---------------------------------------------------------------------------
__device__ __forceinline__ void site_coords_full(long long s, const Geom& g, int c[4]) {
    long long r = s;
    c[0] = (int)(r % g.L[0]); r /= g.L[0];
    c[1] = (int)(r % g.L[1]); r /= g.L[1];
    c[2] = (int)(r % g.L[2]); r /= g.L[2];
    c[3] = (int)r;
}

template <int SP>
__global__ void pack_spinor_kernel(const double2* __restrict__ canon, char* base, long long pbytes, int subset,
                                   Geom g) {
    using SF = SpinorFmt<SP>;
    using T = typename SF::real;
    const long long n = subset == 2 ? 2LL * g.Vh : (long long)g.Vh;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int p = 0;
        long long h = i;
        if (subset == 2) {
            int c[4];
            site_coords_full(i, g, c);
            p = (c[0] + c[1] + c[2] + c[3]) & 1;
            h = i >> 1;
        }
        cpx<T> v[12];
        const double2* src = canon + i * 12;
#pragma unroll
        for (int k = 0; k < 12; k++) {
            double2 d = src[k];
            v[k] = {(T)d.x, (T)d.y};
        }
        SF::store(base + (subset == 2 ? p * pbytes : 0), g.stride, (int)h, v);
    }
}

// Each block converts its sites into shared memory and then writes their
// canonical 192 bytes as one contiguous run (consecutive threads, consecutive
// 16-byte words), instead of 12 strided stores per thread.
constexpr int kUnpackBlock = 128;

template <int SP>
__global__ void __launch_bounds__(kUnpackBlock) unpack_spinor_kernel(double2* __restrict__ canon, const char* base,
                                                                     long long pbytes, int subset, Geom g) {
    using SF = SpinorFmt<SP>;
    using T = typename SF::real;
    __shared__ double2 stage[kUnpackBlock * 12];
    const long long n = subset == 2 ? 2LL * g.Vh : (long long)g.Vh;
    // block-uniform trip count: every thread reaches both barriers
    for (long long i0 = (long long)blockIdx.x * kUnpackBlock; i0 < n; i0 += (long long)gridDim.x * kUnpackBlock) {
        const long long i = i0 + threadIdx.x;
        if (i < n) {
            int p = 0;
            long long h = i;
            if (subset == 2) {
                int c[4];
                site_coords_full(i, g, c);
                p = (c[0] + c[1] + c[2] + c[3]) & 1;
                h = i >> 1;
            }
            cpx<T> v[12];
            SF::load(base + (subset == 2 ? p * pbytes : 0), g.stride, (int)h, v);
#pragma unroll
            for (int k = 0; k < 12; k++) stage[threadIdx.x * 12 + k] = make_double2((double)v[k].re, (double)v[k].im);
        }
        __syncthreads();
        const long long words = (n - i0 < kUnpackBlock ? n - i0 : kUnpackBlock) * 12;
        double2* dst = canon + i0 * 12;
        for (int e = threadIdx.x; e < words; e += kUnpackBlock) dst[e] = stage[e];
        __syncthreads();
    }
}

static int grid_for(long long n, int block) {
    long long b = (n + block - 1) / block;
    long long cap = 64LL * device_sm_count();
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

void pack_spinor(const SpinorField& f, int rhs, const double* canon, cudaStream_t st) {
    const long long n = f.subset == 2 ? 2LL * f.g.Vh : (long long)f.g.Vh;
    const int block = 256, grid = grid_for(n, block);
    char* base = static_cast<char*>(f.block(f.subset == 2 ? 0 : f.subset, rhs));
    const double2* src = reinterpret_cast<const double2*>(canon);
    switch (f.prec) {
        case P_F64: pack_spinor_kernel<P_F64><<<grid, block, 0, st>>>(src, base, f.pbytes, f.subset, f.g); break;
        case P_F32: pack_spinor_kernel<P_F32><<<grid, block, 0, st>>>(src, base, f.pbytes, f.subset, f.g); break;
        case P_F16: pack_spinor_kernel<P_F16><<<grid, block, 0, st>>>(src, base, f.pbytes, f.subset, f.g); break;
        case P_BF16: pack_spinor_kernel<P_BF16><<<grid, block, 0, st>>>(src, base, f.pbytes, f.subset, f.g); break;
    }
    WL_LAUNCH_CHECK();
}

void unpack_spinor(const SpinorField& f, int rhs, double* canon, cudaStream_t st) {
    const long long n = f.subset == 2 ? 2LL * f.g.Vh : (long long)f.g.Vh;
    const int block = kUnpackBlock, grid = grid_for(n, block);
    const char* base = static_cast<const char*>(f.block(f.subset == 2 ? 0 : f.subset, rhs));
    double2* dst = reinterpret_cast<double2*>(canon);
    switch (f.prec) {
        case P_F64: unpack_spinor_kernel<P_F64><<<grid, block, 0, st>>>(dst, base, f.pbytes, f.subset, f.g); break;
        case P_F32: unpack_spinor_kernel<P_F32><<<grid, block, 0, st>>>(dst, base, f.pbytes, f.subset, f.g); break;
        case P_F16: unpack_spinor_kernel<P_F16><<<grid, block, 0, st>>>(dst, base, f.pbytes, f.subset, f.g); break;
        case P_BF16: unpack_spinor_kernel<P_BF16><<<grid, block, 0, st>>>(dst, base, f.pbytes, f.subset, f.g); break;
    }
    WL_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// links
// ---------------------------------------------------------------------------
template <int GP, int R>
__device__ __forceinline__ void store_link(char* base, int stride, int blk, int i, const double2 u[9]) {
    if (GP == P_F64) {
        double2* b = reinterpret_cast<double2*>(base) + (size_t)blk * (R / 2) * stride + i;
#pragma unroll
        for (int c = 0; c < R / 2; c++) b[(size_t)c * stride] = u[c];
    } else if (GP == P_F32 && R == 18) {
        float2* b = reinterpret_cast<float2*>(base) + (size_t)blk * 9 * stride + i;
#pragma unroll
        for (int c = 0; c < 9; c++) b[(size_t)c * stride] = make_float2((float)u[c].x, (float)u[c].y);
    } else if (GP == P_F32 && R == 12) {
        float4* b = reinterpret_cast<float4*>(base) + (size_t)blk * 3 * stride + i;
#pragma unroll
        for (int c = 0; c < 3; c++)
            b[(size_t)c * stride] = make_float4((float)u[2 * c].x, (float)u[2 * c].y, (float)u[2 * c + 1].x,
                                                (float)u[2 * c + 1].y);
    } else if (R == 18) {  // F16 / BF16, 18 reals: rows of 16, 16 and 4 bytes
        using LT = LowT<GP == P_F16 ? P_F16 : P_BF16>;
        char* b = base + (size_t)blk * 36 * stride;
        unsigned int w[9];
#pragma unroll
        for (int k = 0; k < 9; k++) w[k] = LT::from_f2((float)u[k].x, (float)u[k].y);
        reinterpret_cast<uint4*>(b)[i] = make_uint4(w[0], w[1], w[2], w[3]);
        reinterpret_cast<uint4*>(b + 16LL * stride)[i] = make_uint4(w[4], w[5], w[6], w[7]);
        reinterpret_cast<unsigned int*>(b + 32LL * stride)[i] = w[8];
    } else {  // F16 / BF16, 12 reals
        using LT = LowT<GP == P_F16 ? P_F16 : P_BF16>;
        uint2* b = reinterpret_cast<uint2*>(base) + (size_t)blk * 3 * stride + i;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            uint2 d;
            d.x = LT::from_f2((float)u[2 * c].x, (float)u[2 * c].y);
            d.y = LT::from_f2((float)u[2 * c + 1].x, (float)u[2 * c + 1].y);
            b[(size_t)c * stride] = d;
        }
    }
}

template <int GP, int R>
__global__ void pack_gauge_kernel(const double2* __restrict__ canon, char* base, Geom g) {
    const long long V = 2LL * g.Vh;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < V; s += (long long)gridDim.x * blockDim.x) {
        int c[4];
        site_coords_full(s, g, c);
        const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
        const int h = (int)(s >> 1);
#pragma unroll
        for (int mu = 0; mu < 4; mu++) {
            double2 u[9];
            const double2* src = canon + (s * 4 + mu) * 9;
#pragma unroll
            for (int k = 0; k < 9; k++) u[k] = src[k];
            store_link<GP, R>(base, g.stride, p * 4 + mu, h, u);
        }
    }
}

void pack_gauge(GaugeField& gf, const double* canon, cudaStream_t st) {
    const long long V = 2LL * gf.g.Vh;
    const int block = 256, grid = grid_for(V, block);
    const double2* src = reinterpret_cast<const double2*>(canon);
    char* base = gf.buf.as<char>();
    const Prec p = gf.prec;
    const int R = gf.recon;
    if (p == P_F64 && R == 18) pack_gauge_kernel<P_F64, 18><<<grid, block, 0, st>>>(src, base, gf.g);
    else if (p == P_F64 && R == 12) pack_gauge_kernel<P_F64, 12><<<grid, block, 0, st>>>(src, base, gf.g);
    else if (p == P_F32 && R == 18) pack_gauge_kernel<P_F32, 18><<<grid, block, 0, st>>>(src, base, gf.g);
    else if (p == P_F32 && R == 12) pack_gauge_kernel<P_F32, 12><<<grid, block, 0, st>>>(src, base, gf.g);
    else if (p == P_F16 && R == 12) pack_gauge_kernel<P_F16, 12><<<grid, block, 0, st>>>(src, base, gf.g);
    else if (p == P_BF16 && R == 12) pack_gauge_kernel<P_BF16, 12><<<grid, block, 0, st>>>(src, base, gf.g);
    else if (p == P_F16 && R == 18) pack_gauge_kernel<P_F16, 18><<<grid, block, 0, st>>>(src, base, gf.g);
    else if (p == P_BF16 && R == 18) pack_gauge_kernel<P_BF16, 18><<<grid, block, 0, st>>>(src, base, gf.g);
    else throw Error(7, "unsupported link precision / storage");
    WL_LAUNCH_CHECK();
}

}  // namespace wl
