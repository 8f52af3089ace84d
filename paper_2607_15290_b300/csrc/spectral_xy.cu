// spectral_xy.cu -- the three-pass plan of a 3D FP32 Fourier round trip: the x and y
// transforms of each z-plane run in one thread-block cluster whose CTAs hold the
// plane's rows in their shared memory.
//
//   xy forward : one cluster per plane z.  CTA q of CS runs the x-pass forward (nodal
//                prologue, packed transforms, half spectra) of rows [q R, (q+1) R),
//                R = n1 / CS, and stores every spectral value straight into the
//                shared memory of the CTA that owns its column (distributed shared
//                memory); after one cluster barrier each CTA transforms its columns
//                along y from its own shared memory and stores them to the spectrum.
//   z pass     : unchanged (forward FFT, multiplier, inverse FFT along z).
//   xy inverse : CTA q loads its columns, transforms them along y and writes each
//                row's part into the slab of the CTA that owns the row; after a
//                cluster barrier each CTA runs the x-pass inverse (nodal epilogue) of
//                its rows from its slab.
//
// The y passes of the five-pass plan each read and write the whole spectrum (3 words
// per node each way); here the spectrum crosses HBM only between the xy passes and
// the z pass, so an application moves 23 words per node instead of 35.  The spectral
// layout in HBM is the five-pass plan's, and the row bodies are the compile-time
// x-pass bodies of spectral_ct.cuh with their spectrum redirected to the slab.
#include <cooperative_groups.h>
#include "spectral_ct.cuh"
#include "spectral_xy.h"

namespace cg = cooperative_groups;

namespace llg {
namespace xy {

template <int LOGN0, int LOGN1, int CS, int NT>
struct Plan {
    static constexpr int N0 = 1 << LOGN0, N1 = 1 << LOGN1;
    static constexpr int E0 = ct::LineE<float, LOGN0>::value, P0 = N0 / E0;
    static constexpr int E1 = ct::LineE<float, LOGN1>::value, P1 = N1 / E1;
    static constexpr int R = N1 / CS;                 // plane rows per CTA
    static constexpr int LIVE = N0 + N0 / 2 + 1;      // spectral columns that carry data
    static constexpr int LINES = NT / P0;             // x-phase lines per block
    static constexpr int TWA = NT / P1;               // y-phase columns per round
    static constexpr int CC = (LIVE + CS - 1) / CS;   // columns per CTA
    static constexpr int YR = (CC + TWA - 1) / TWA;   // y-phase rounds
    static constexpr int LS0 = ct::RowL<LOGN0>::size;
    // row pairs per x round: the largest G with 3 G lines that divides the CTA's pairs
    static constexpr int pick_g(int g) { return (g <= 1 || ((R / 2) % g == 0)) ? (g < 1 ? 1 : g) : pick_g(g - 1); }
    static constexpr int G = pick_g(LINES / 3 < R / 2 ? LINES / 3 : R / 2);
    // slab row stride: the TWA columns of two consecutive rows start 2 TWA banks apart
    static constexpr int pick_sp(int s) { return ((2 * s) % 32 == (2 * TWA) % 32) ? s : pick_sp(s + 1); }
    static constexpr int SP = pick_sp(LIVE);
    // forward: a column buffer of N1 rows x CC columns (row stride CCP, odd to spread banks);
    // inverse: a slab of R rows x LIVE columns (row stride SP); the larger of the two
    static constexpr int CCP = CC | 1;
    static constexpr size_t cbuf_bytes = (size_t)N1 * CCP * sizeof(float2);
    static constexpr size_t slab_bytes_inv = (size_t)R * SP * sizeof(float2);
    static constexpr size_t slab_bytes = cbuf_bytes > slab_bytes_inv ? cbuf_bytes : slab_bytes_inv;
    static constexpr size_t xbuf_bytes = (size_t)2 * LINES * LS0 * sizeof(float2);
    static constexpr bool YDB = (size_t)2 * N1 * TWA * sizeof(float2) <= 96 * 1024;
    static constexpr size_t ybuf_bytes = (size_t)(YDB ? 2 : 1) * N1 * TWA * sizeof(float2);
    static constexpr size_t smem = slab_bytes + (xbuf_bytes > ybuf_bytes ? xbuf_bytes : ybuf_bytes);
    static_assert(NT % P0 == 0 && NT % P1 == 0, "block size must hold whole lines and columns");
    static_assert(R % 2 == 0 && 3 * G <= LINES, "plan shape");
    static_assert(smem <= 227 * 1024, "shared memory per CTA");
};

template <int LOGN0, int LOGN1, int CS, int NT, typename TIn, typename TOut, int IN>
__global__ void __launch_bounds__(NT) xy_fwd(RowArgs<float, TIn, TOut> a, const float2 *__restrict__ tw1) {
    using PL = Plan<LOGN0, LOGN1, CS, NT>;
    pdl_wait();
    if (a.io.skip && *a.io.skip) return;   // uniform over the cluster: every CTA reads the same flag
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *cbuf = reinterpret_cast<float2 *>(smraw);   // N1 rows x CC columns of this CTA
    unsigned char *work = smraw + PL::slab_bytes;
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank();
    const long long z = blockIdx.x / CS;
    // x phase: rows [q R, (q+1) R) of plane z, each value pushed to its column's owner
    RowArgs<float, TIn, TOut> ra = a;
    ra.G = PL::G;
    const long long lp0 = (z * PL::N1 + (long long)q * PL::R) / 2;
    const long long row0 = z * PL::N1;
    auto sink = [&](long long row, int col, float2 v) {
        const int owner = col / PL::CC;
        float2 *dst = cl.map_shared_rank(cbuf, owner);
        dst[(row - row0) * PL::CCP + (col - owner * PL::CC)] = v;
    };
    for (int pg = 0; pg < PL::R / 2; pg += PL::G) {
        ct::row_fwd_ct_body_to<float, TIn, TOut, LOGN0, IN>(ra, (lp0 + pg) / PL::G, work, sink);
        __syncthreads();
    }
    cl.sync();   // every CTA's column buffer is complete; nothing remote is touched after this
    // y phase: this CTA's columns [q CC, (q+1) CC) from its own buffer
    const int c = threadIdx.x % PL::TWA, t = threadIdx.x / PL::TWA;
    float2 *yb0 = reinterpret_cast<float2 *>(work);
    float2 *yb1 = PL::YDB ? yb0 + PL::N1 * PL::TWA : yb0;
    const int col_lo = q * PL::CC, col_hi = min(PL::LIVE, col_lo + PL::CC);
    for (int rd = 0; rd < PL::YR; ++rd) {
        const int cl_local = rd * PL::TWA + c, col = col_lo + cl_local;
        const bool live = col < col_hi;
        float2 v[PL::E1];
#pragma unroll
        for (int s = 0; s < PL::E1; ++s)
            v[s] = live ? cbuf[(t + PL::P1 * s) * PL::CCP + cl_local] : make_float2(0.f, 0.f);
        ct::fft<LOGN1, PL::E1, -1, ct::ColL<PL::TWA>, 0, PL::YDB>(v, yb0 + c, yb1 + c, t, tw1);
        if (live) {
            float2 *dst = a.spec + row0 * (long long)a.S + col;
#pragma unroll
            for (int s = 0; s < PL::E1; ++s) dst[(long long)(t + PL::P1 * s) * a.S] = v[s];
        }
        __syncthreads();
    }
}

template <int LOGN0, int LOGN1, int CS, int NT, typename TIn, typename TOut, int OUT>
__global__ void __launch_bounds__(NT) xy_inv(RowArgs<float, TIn, TOut> a, const float2 *__restrict__ tw1) {
    using PL = Plan<LOGN0, LOGN1, CS, NT>;
    pdl_wait();
    if (a.io.skip && *a.io.skip) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *slab = reinterpret_cast<float2 *>(smraw);
    unsigned char *work = smraw + PL::slab_bytes;
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank();
    const long long z = blockIdx.x / CS;
    // y phase: inverse transform of this CTA's columns, each row scattered to its owner's slab
    const int c = threadIdx.x % PL::TWA, t = threadIdx.x / PL::TWA;
    float2 *yb0 = reinterpret_cast<float2 *>(work);
    float2 *yb1 = PL::YDB ? yb0 + PL::N1 * PL::TWA : yb0;
    const int col_lo = q * PL::CC, col_hi = min(PL::LIVE, col_lo + PL::CC);
    for (int rd = 0; rd < PL::YR; ++rd) {
        const int col = col_lo + rd * PL::TWA + c;
        const bool live = col < col_hi;
        float2 v[PL::E1];
        const float2 *src = a.spec + (z * PL::N1) * (long long)a.S + col;
#pragma unroll
        for (int s = 0; s < PL::E1; ++s)
            v[s] = live ? src[(long long)(t + PL::P1 * s) * a.S] : make_float2(0.f, 0.f);
        ct::fft<LOGN1, PL::E1, +1, ct::ColL<PL::TWA>, 0, PL::YDB>(v, yb0 + c, yb1 + c, t, tw1);
        if (live) {
#pragma unroll
            for (int s = 0; s < PL::E1; ++s) {
                const int y = t + PL::P1 * s;
                float2 *dst = cl.map_shared_rank(slab, y / PL::R);
                dst[(y % PL::R) * PL::SP + col] = v[s];
            }
        }
        __syncthreads();
    }
    cl.sync();   // every CTA's slab is complete
    // x phase: rows [q R, (q+1) R) of plane z from the slab, nodal epilogue to the outputs
    RowArgs<float, TIn, TOut> ra = a;
    ra.G = PL::G;
    const long long lp0 = (z * PL::N1 + (long long)q * PL::R) / 2;
    for (int pg = 0; pg < PL::R / 2; pg += PL::G) {
        ct::row_inv_ct_body<float, TIn, TOut, LOGN0, OUT>(ra, (lp0 + pg) / PL::G, work, slab, lp0, PL::SP);
        __syncthreads();
    }
}

// launch with the cluster shape and as a programmatic dependent of the previous kernel
template <typename... KP, typename... A>
static cudaError_t launch_xy(void (*k)(KP...), int CS, int clusters, int NT, size_t smem, cudaStream_t st,
                             A... args) {
    cudaError_t e = set_smem(k, smem);
    if (e == cudaSuccess && CS > 8) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * CS);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// the compiled plans: (log2 n0, log2 n1, cluster size, threads)
#define LLG_XY_PLANS(X) X(7, 7, 8, 400) X(8, 8, 16, 416)

template <int LOGN0, int LOGN1, int CS, int NT, typename TIn, typename TOut>
static cudaError_t fwd_plan(llg_ctx *c, int in_mode, const RowArgs<float, TIn, TOut> &a, const float2 *tw1) {
    using PL = Plan<LOGN0, LOGN1, CS, NT>;
    if (in_mode != IN_V) return cudaErrorNotSupported;
    return launch_xy(xy_fwd<LOGN0, LOGN1, CS, NT, TIn, TOut, IN_V>, CS, c->geo.n[2], NT, PL::smem, c->stream, a, tw1);
}

template <int LOGN0, int LOGN1, int CS, int NT, typename TIn, typename TOut>
static cudaError_t inv_plan(llg_ctx *c, int out_mode, const RowArgs<float, TIn, TOut> &a, const float2 *tw1) {
    using PL = Plan<LOGN0, LOGN1, CS, NT>;
    if (out_mode == OUT_APPLY)
        return launch_xy(xy_inv<LOGN0, LOGN1, CS, NT, TIn, TOut, OUT_APPLY>, CS, c->geo.n[2], NT, PL::smem, c->stream,
                         a, tw1);
    if (out_mode == OUT_MATVEC)
        return launch_xy(xy_inv<LOGN0, LOGN1, CS, NT, TIn, TOut, OUT_MATVEC>, CS, c->geo.n[2], NT, PL::smem, c->stream,
                         a, tw1);
    return cudaErrorNotSupported;
}

bool available(const llg_ctx *c, int in_mode, int out_mode) {
    const SpecGeom &g = c->geo;
    if (g.dim != 3 || in_mode != IN_V || (out_mode != OUT_APPLY && out_mode != OUT_MATVEC)) return false;
#define LLG_XY_HAS(L0, L1, CS, NT) if (g.logn[0] == L0 && g.logn[1] == L1) return true;
    LLG_XY_PLANS(LLG_XY_HAS)
#undef LLG_XY_HAS
    return false;
}

template <typename TIn, typename TOut>
cudaError_t forward(llg_ctx *c, int in_mode, const RowArgs<float, TIn, TOut> &a) {
    const SpecGeom &g = c->geo;
#define LLG_XY_F(L0, L1, CS, NT) \
    if (g.logn[0] == L0 && g.logn[1] == L1) return fwd_plan<L0, L1, CS, NT, TIn, TOut>(c, in_mode, a, c->tw32[1]);
    LLG_XY_PLANS(LLG_XY_F)
#undef LLG_XY_F
    return cudaErrorNotSupported;
}

template <typename TIn, typename TOut>
cudaError_t inverse(llg_ctx *c, int out_mode, const RowArgs<float, TIn, TOut> &a) {
    const SpecGeom &g = c->geo;
#define LLG_XY_I(L0, L1, CS, NT) \
    if (g.logn[0] == L0 && g.logn[1] == L1) return inv_plan<L0, L1, CS, NT, TIn, TOut>(c, out_mode, a, c->tw32[1]);
    LLG_XY_PLANS(LLG_XY_I)
#undef LLG_XY_I
    return cudaErrorNotSupported;
}

template cudaError_t forward<double, float>(llg_ctx *, int, const RowArgs<float, double, float> &);
template cudaError_t forward<float, double>(llg_ctx *, int, const RowArgs<float, float, double> &);
template cudaError_t forward<float, float>(llg_ctx *, int, const RowArgs<float, float, float> &);
template cudaError_t inverse<double, float>(llg_ctx *, int, const RowArgs<float, double, float> &);
template cudaError_t inverse<float, double>(llg_ctx *, int, const RowArgs<float, float, double> &);
template cudaError_t inverse<float, float>(llg_ctx *, int, const RowArgs<float, float, float> &);

}  // namespace xy
}  // namespace llg
