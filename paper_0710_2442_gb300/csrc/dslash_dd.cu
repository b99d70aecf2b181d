// dslash_dd.cu -- the even-odd hopping term of one sub-lattice of a lattice
// split along t, with the t-neighbours across the split taken from halo
// buffers: the GPU form of the paper's domain decomposition over SPEs and
// Cell nodes (Sec. 5), whose external communication T_ext carries projected
// half spinors, 12 reals per boundary site and face (Table 1).
//
// Split.  The global lattice Lx x Ly x Lz x Lt is cut into sub-lattices of
// Lr consecutive t-slices, Lr even, so that every sub-lattice starts at an
// even t and its local site parity equals the global one.  The t-slice tau
// of a sub-lattice's parity field is the contiguous half-site range
// [tau * Vs/2, (tau + 1) * Vs/2) with Vs = Lx Ly Lz, and the face site f of
// a slice has the same (x, y, z) in every slice, so a face buffer is indexed
// by f in [0, Vs/2) on both sides.
//
// Pack (the sender, from its input field of parity 1 - p):
//   to the previous sub-lattice: h = (1 - S g_4) psi on its first slice,
//     the projected half spinor that the receiver's forward t-hop needs;
//   to the next sub-lattice: W = U^dag_{y,4} (1 + S g_4) psi(y) on its last
//     slice; the link of that hop lives on the sender, so the sender applies
//     it and ships the product.
// Hop (the receiver): x, y, z hops and the interior t-hops as the single-
// GPU kernel; the forward t-hop of the last slice takes h from the buffer
// received from the next sub-lattice (times the boundary phase if this is
// the last sub-lattice of the lattice) and applies the local link; the
// backward t-hop of the first slice takes W from the buffer received from the
// previous sub-lattice (times the conjugate phase if this is the first).
// Between the two the caller moves the buffers: a device copy when the
// sub-lattices share a GPU, NCCL send/recv or a peer copy between GPUs.
//
// Halo storage: face stride round_up(Vs/2, 64); F64: 6 rows of double2
// (half spin * 3 + colour); F32: 3 rows of float4, colour c holding
// (h0.re, h1.re, h0.im, h1.im).  96 or 48 bytes per face site.
#include <cmath>
#include <cstdio>
#include <vector>

#include "dslash_impl.cuh"

namespace wl {

namespace {

template <int SP>
struct HaloFmt;
template <>
struct HaloFmt<P_F64> {
    static constexpr long long bytes_per_site = 96;
    __device__ static __forceinline__ void store(void* base, int fst, int f, const cpx<double> h[6]) {
        double2* b = static_cast<double2*>(base) + f;
#pragma unroll
        for (int k = 0; k < 6; k++) b[(size_t)k * fst] = make_double2(h[k].re, h[k].im);
    }
    __device__ static __forceinline__ void load(const void* base, int fst, int f, cpx<double> h[6]) {
        const double2* b = static_cast<const double2*>(base) + f;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const double2 d = __ldg(b + (size_t)k * fst);
            h[k] = {d.x, d.y};
        }
    }
};
template <>
struct HaloFmt<P_F32> {
    static constexpr long long bytes_per_site = 48;
    __device__ static __forceinline__ void store(void* base, int fst, int f, const cpx<float> h[6]) {
        float4* b = static_cast<float4*>(base) + f;
#pragma unroll
        for (int c = 0; c < 3; c++) b[(size_t)c * fst] = make_float4(h[c].re, h[3 + c].re, h[c].im, h[3 + c].im);
    }
    __device__ static __forceinline__ void load(const void* base, int fst, int f, cpx<float> h[6]) {
        const float4* b = static_cast<const float4*>(base) + f;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const float4 d = __ldg(b + (size_t)c * fst);
            h[c] = {d.x, d.z};
            h[3 + c] = {d.y, d.w};
        }
    }
};

struct DDArgs {
    const char* in;        // input parity block (parity pin)
    char* out;             // output parity block (parity p), hop only
    const char* gauge;
    Geom g;                // the sub-lattice's geometry
    int p;                 // output parity
    int nface;             // Vs / 2
    int fst;               // face stride
    void* send_prev;
    void* send_next;
    const void* recv_next;
    const void* recv_prev;
    int first, last;       // the sub-lattice holds the lattice's first / last t-slice
    int part;              // hop: 0 every site, 1 the interior t-slices, 2 the two face slices
    int count;             // hop: sites of the part
};

// The i-th site of a hop part (i < A.count).
__device__ __forceinline__ int dd_site(const DDArgs& A, int i, int Lt) {
    if (A.part == 1) return A.nface + i;                         // slices 1 .. Lt-2
    if (A.part == 2) return i < A.nface ? i : i + (Lt - 2) * A.nface;  // slices 0 and Lt-1
    return i;
}

template <int SP, int GP, int R, bool DAG>
__global__ void __launch_bounds__(256) dd_pack_kernel(const DDArgs A) {
    using SF = SpinorFmt<SP>;
    using GF = GaugeFmt<GP, R>;
    using T = typename SF::real;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= A.nface) return;
    constexpr int SF_ = DAG ? -1 : 1;
    const Geom& g = A.g;
    const int pin = 1 - A.p;
    {   // first slice -> previous sub-lattice: (1 - S g_4) psi
        cpx<T> v[12], hs[6];
        SF::load(A.in, g.stride, f, v);
        project<3, SF_>(v, hs);
        HaloFmt<SP>::store(A.send_prev, A.fst, f, hs);
    }
    {   // last slice -> next sub-lattice: U^dag_{y,4} (1 + S g_4) psi(y)
        const int h = (g.L[3] - 1) * A.nface + f;
        cpx<T> v[12], hs[6], w[6], U[3][3];
        SF::load(A.in, g.stride, h, v);
        project<3, -SF_>(v, hs);
        GF::load(A.gauge, g.stride, pin * 4 + 3, h, U);
        su3_mul<true>(U, hs, w);
        HaloFmt<SP>::store(A.send_next, A.fst, f, w);
    }
}

template <int SP, int GP, int R, bool DAG>
__global__ void __launch_bounds__(256, 2) dd_hop_kernel(const HopParams P, const DDArgs A) {
    using SF = SpinorFmt<SP>;
    using GF = GaugeFmt<GP, R>;
    using T = typename SF::real;
    constexpr int SF_ = DAG ? -1 : 1;
    const Geom& g = P.g;
    const int p = A.p;
    const int Lt = g.L[3];
    const int smu = g.L[0] * g.L[1] * g.L[2];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.count; i += gridDim.x * blockDim.x) {
        const int h = dd_site(A, i, Lt);
        int c[4], s;
        site_of_half(h, p, g, c, s);
        if constexpr (SP == P_F32) {
            // the site's links, all at once (L2 prefetches, as the undecomposed
            // F32 hop's prefetching variants): x, y, z as in hop_dir, the
            // forward t link, and the backward one unless it lies across the face
#pragma unroll
            for (int mu = 0; mu < 3; mu++) {
                const int L = g.L[mu];
                const int sm = mu == 0 ? 1 : mu == 1 ? g.L[0] : g.L[0] * g.L[1];
                prefetch_link<GP, R>(P.gauge, g.stride, p * 4 + mu, h);
                prefetch_link<GP, R>(P.gauge, g.stride, (1 - p) * 4 + mu,
                                     (c[mu] == 0 ? s + (L - 1) * sm : s - sm) >> 1);
            }
            prefetch_link<GP, R>(A.gauge, g.stride, p * 4 + 3, h);
            if (c[3] != 0) prefetch_link<GP, R>(A.gauge, g.stride, (1 - p) * 4 + 3, (s - smu) >> 1);
        }
        cpx<T> acc[12];
        hop_dir<SP, GP, R, DAG, 0, true>(acc, P, A.in, p, h, c, s);
        hop_dir<SP, GP, R, DAG, 1, false>(acc, P, A.in, p, h, c, s);
        hop_dir<SP, GP, R, DAG, 2, false>(acc, P, A.in, p, h, c, s);
        // t, forward: (1 - S g_4) eta U_{x,4} psi_{x+4}
        {
            cpx<T> hs[6], w[6], U[3][3];
            if (c[3] == Lt - 1) {
                HaloFmt<SP>::load(A.recv_next, A.fst, h - (Lt - 1) * A.nface, hs);
                if (A.last) {
                    const cpx<T> eta = {(T)g.ph[3][0], (T)g.ph[3][1]};
#pragma unroll
                    for (int k = 0; k < 6; k++) hs[k] = cmul(eta, hs[k]);
                }
            } else {
                cpx<T> v[12];
                SF::load(A.in, g.stride, (s + smu) >> 1, v);
                project<3, SF_>(v, hs);
            }
            GF::load(A.gauge, g.stride, p * 4 + 3, h, U);
            su3_mul<false>(U, hs, w);
            expand<3, SF_, false>(acc, w, (T)1);
        }
        // t, backward: (1 + S g_4) eta* U^dag_{x-4,4} psi_{x-4}
        {
            cpx<T> w[6];
            if (c[3] == 0) {
                HaloFmt<SP>::load(A.recv_prev, A.fst, h, w);
                if (A.first) {
                    const cpx<T> eta = {(T)g.ph[3][0], -(T)g.ph[3][1]};
#pragma unroll
                    for (int k = 0; k < 6; k++) w[k] = cmul(eta, w[k]);
                }
            } else {
                const int hn = (s - smu) >> 1;
                cpx<T> v[12], hs[6], U[3][3];
                SF::load(A.in, g.stride, hn, v);
                project<3, -SF_>(v, hs);
                GF::load(A.gauge, g.stride, (1 - p) * 4 + 3, hn, U);
                su3_mul<true>(U, hs, w);
            }
            expand<3, -SF_, false>(acc, w, (T)1);
        }
        SF::store(A.out, g.stride, h, acc);
    }
}

int face_stride(const Geom& g) { return round_up(g.L[0] * g.L[1] * g.L[2] / 2, 64); }

// Pack, or one part of the hop with the block size `block`.  (A paired-FP32
// form of the hop for F32 fields measured slower: 119 against 115.8 us for
// the two halves of 32^3 x 64, as the scalar stencil also wins the tuner's
// choice for the single-lattice F32 hop.)
template <int SP, int GP, int R>
void launch_dd(bool pack, bool dag, const HopParams& P, const DDArgs& A, int block, cudaStream_t st) {
    if (pack) {
        const int blocks = (A.nface + 127) / 128;
        if (dag) dd_pack_kernel<SP, GP, R, true><<<blocks, 128, 0, st>>>(A);
        else dd_pack_kernel<SP, GP, R, false><<<blocks, 128, 0, st>>>(A);
    } else if (A.count > 0) {
        const int blocks = (A.count + block - 1) / block;
        if (dag) dd_hop_kernel<SP, GP, R, true><<<blocks, block, 0, st>>>(P, A);
        else dd_hop_kernel<SP, GP, R, false><<<blocks, block, 0, st>>>(P, A);
    }
    WL_LAUNCH_CHECK();
}

void dispatch_dd(bool pack, bool dag, Prec sp, int recon, const HopParams& P, const DDArgs& A, int block,
                 cudaStream_t st) {
    if (sp == P_F64 && recon == 18) launch_dd<P_F64, P_F64, 18>(pack, dag, P, A, block, st);
    else if (sp == P_F64 && recon == 12) launch_dd<P_F64, P_F64, 12>(pack, dag, P, A, block, st);
    else if (sp == P_F32 && recon == 12) launch_dd<P_F32, P_F32, 12>(pack, dag, P, A, block, st);
    else if (sp == P_F32 && recon == 18) launch_dd<P_F32, P_F32, 18>(pack, dag, P, A, block, st);
    else throw Error(WILSON_ERR_UNSUPPORTED, "the decomposed hop takes F64 or F32 fields");
}

// The sites of a hop part: 0 all, 1 the interior t-slices, 2 the two faces.
int dd_count(const DDArgs& A, int part) {
    const int Lt = A.g.L[3];
    return part == 0 ? A.g.Vh : part == 1 ? (Lt - 2) * A.nface : 2 * A.nface;
}

long long halo_bytes(Prec sp, const Geom& g) {
    WL_REQUIRE(sp == P_F64 || sp == P_F32, "the decomposed hop takes F64 or F32 fields");
    return (sp == P_F64 ? HaloFmt<P_F64>::bytes_per_site : HaloFmt<P_F32>::bytes_per_site) * face_stride(g);
}

template <class F>
int guarded_dd(F&& f) {
    try {
        f();
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

// The arguments common to pack and hop; in: the input field (one parity).
DDArgs dd_args(const wilson_gauge* gh, const wilson_spinor* in, int out_parity) {
    WL_REQUIRE(gh && in, "NULL handle");
    const GaugeField& gf = gh->f;
    const SpinorField& a = in->f;
    WL_REQUIRE(a.subset == 0 || a.subset == 1, "the input is one parity of the sub-lattice");
    WL_REQUIRE(a.nrhs == 1, "the decomposed hop takes one right-hand side");
    WL_REQUIRE(gf.prec == a.prec, "gauge and spinor precision differ");
    for (int mu = 0; mu < 4; mu++) WL_REQUIRE(a.g.L[mu] == gf.g.L[mu], "lattice mismatch");
    WL_REQUIRE(out_parity == 1 - a.subset, "the hop maps parity 1-p to parity p");
    DDArgs A{};
    A.in = static_cast<const char*>(a.block(a.subset));
    A.gauge = gf.buf.as<const char>();
    A.g = gf.g;
    A.p = out_parity;
    A.nface = gf.g.L[0] * gf.g.L[1] * gf.g.L[2] / 2;
    A.fst = face_stride(gf.g);
    (void)halo_bytes(a.prec, gf.g);
    return A;
}

}  // namespace

}  // namespace wl

using namespace wl;

extern "C" long long wilson_dd_halo_bytes(const wilson_lattice* L, int prec) {
    long long out = -1;
    const int rc = guarded_dd([&] {
        const Geom g = checked_geom(L);
        WL_REQUIRE(prec == WILSON_F64 || prec == WILSON_F32, "the decomposed hop takes F64 or F32 fields");
        out = halo_bytes(static_cast<Prec>(prec), g);
    });
    return rc == WILSON_OK ? out : -1;
}

extern "C" int wilson_dd_pack(void* send_prev, void* send_next, const wilson_gauge* g, const wilson_spinor* in,
                              int dagger, void* stream) {
    return guarded_dd([&] {
        check_ptr(send_prev, "send_prev");
        check_ptr(send_next, "send_next");
        WL_REQUIRE(send_prev != send_next, "the two face buffers must differ");
        WL_REQUIRE(in != nullptr, "NULL handle");
        DDArgs A = dd_args(g, in, 1 - in->f.subset);
        WL_REQUIRE(is_device_ptr(send_prev) && is_device_ptr(send_next), "face buffers must be device memory");
        A.send_prev = send_prev;
        A.send_next = send_next;
        HopParams P{};
        P.g = A.g;
        dispatch_dd(true, dagger != 0, in->f.prec, g->f.recon, P, A, 128, static_cast<cudaStream_t>(stream));
    });
}

extern "C" int wilson_dd_hop(wilson_spinor* out, const wilson_gauge* g, const wilson_spinor* in,
                             const void* recv_next, const void* recv_prev, int dagger, int t_first, int t_last,
                             int part, void* stream) {
    return guarded_dd([&] {
        WL_REQUIRE(out && in && out != in, "NULL handle, or out is in");
        WL_REQUIRE(part == WILSON_DD_ALL || part == WILSON_DD_INTERIOR || part == WILSON_DD_FACES,
                   "part must be WILSON_DD_ALL, WILSON_DD_INTERIOR or WILSON_DD_FACES");
        if (part != WILSON_DD_INTERIOR) {
            check_ptr(recv_next, "recv_next");
            check_ptr(recv_prev, "recv_prev");
            WL_REQUIRE(is_device_ptr(recv_next) && is_device_ptr(recv_prev), "face buffers must be device memory");
        }
        DDArgs A = dd_args(g, in, out->f.subset);
        const SpinorField& b = out->f;
        WL_REQUIRE(b.prec == in->f.prec && b.nrhs == 1, "out must match in (precision, one right-hand side)");
        for (int mu = 0; mu < 4; mu++) WL_REQUIRE(b.g.L[mu] == A.g.L[mu], "lattice mismatch");
        A.out = static_cast<char*>(b.block(b.subset));
        A.recv_next = recv_next;
        A.recv_prev = recv_prev;
        A.first = t_first != 0;
        A.last = t_last != 0;
        HopParams P{};
        P.gauge = A.gauge;
        P.g = A.g;
        P.out_parity = A.p;
        P.a = 1.0;
        P.nrhs = 1;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        const Prec sp = in->f.prec;
        const int recon = g->f.recon;
        const bool dag = dagger != 0;
        // block size: tuned by the first ALL call on the caller's own fields
        // (the hop only writes out, so the repeated launches are harmless)
        LaunchConfig cfg{128, 0};
        char key[128];
        snprintf(key, sizeof(key), "ddhop:s%d:r%d:d%d:%dx%dx%dx%d", (int)sp, recon, (int)dag, A.g.L[0], A.g.L[1],
                 A.g.L[2], A.g.L[3]);
        const std::vector<LaunchConfig> cands = {{64, 0}, {128, 0}, {256, 0}};
        if (part == WILSON_DD_ALL) {
            DDArgs At = A;
            At.part = 0;
            At.count = dd_count(A, 0);
            cfg = tune_launch(key, cands, cfg, st,
                              [&](const LaunchConfig& c) { dispatch_dd(false, dag, sp, recon, P, At, c.block, st); });
        } else {
            cfg = tune_lookup(key, cands, cfg);
        }
        A.part = part;
        A.count = dd_count(A, part);
        dispatch_dd(false, dag, sp, recon, P, A, cfg.block, st);
    });
}
