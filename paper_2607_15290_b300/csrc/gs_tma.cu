// gs_tma.cu -- the Gram--Schmidt passes of flexible solves in FP32-pair arithmetic (the same
// arithmetic and data layout as arnoldi_pass_pair in krylov.cu), with their operands staged
// in shared memory by bulk copies.
//
// Each persistent block walks its share of the vectors in chunks through a ring of NS stages
// in shared memory, run as a producer/consumer pipeline: one producer warp fills a stage with
// the bulk copies of a chunk (the FP32 hi plane of w, in pass C also its lo plane, the FP64
// first basis vector and the hi and lo planes of every later one; cp.async.bulk, completion
// on the stage's "full" mbarrier) as soon as the consumers have released it (its "empty"
// mbarrier, one arrival per consumer warp); eight consumer warps wait on "full", compute, and
// release.  No block-wide barrier sits in the loop, so warps drift by up to the ring's depth
// instead of meeting after every chunk, and NS - 1 chunks stay in flight per block.
//
// Every mbarrier wait is bounded (about 1 s of clock).  A wait that runs out raises the
// error word in host-mapped memory (the host reports LLG_ERR_TIMEOUT at its next check); the
// warp stops, the block waits (bounded) for every copy it issued, and still stores its
// partial sums and counts its arrival, so the pass's last-block bookkeeping stays consistent.
#include <algorithm>
#include "spectral_kernels.cuh"
#include "krylov_dev.cuh"
#include "f32pair.cuh"
#include "tma_ptx.cuh"
#include "gs_tma.h"

namespace llg {
namespace gst {

using namespace llg::tma;

constexpr int NCW = 8;                    // consumer warps
constexpr int NC = NCW * 32;              // consumer threads (RB_THREADS: the block reduction's width)
constexpr int NT = NC + 32;               // + one producer warp
static_assert(NC == RB_THREADS, "consumer threads = reduction width");

// ring shape: up to 12 basis vectors two blocks per SM with two 48 KB stages each (measured
// at 128^3 against three 32, three 36 and four 24 KB stages: 75.5 against 78.1, 78.8 and
// 79.7 us a pass); beyond that (more registers a thread) one block per SM with four 48 KB
// stages
template <int MAXV> struct Ring {
    static constexpr int BLOCKS = MAXV <= 12 ? 2 : 1;
    static constexpr int NS = MAXV <= 12 ? 2 : 4;
    static constexpr int TARGET = 48 * 1024;
};

// bytes staged per vector element: w hi (+ w lo in pass C), V_0 (FP64), 8 per later vector
__host__ __device__ constexpr int elem_bytes(int nv, int mode) { return 4 + (mode == PASS_UPD_NRM ? 4 : 0) + 8 * nv; }

// chunk layout in a stage: [w hi][w lo (pass C)][V_0][V_1 hi][V_1 lo] ... each CH long
struct ChunkLayout {
    int CH;
    __host__ __device__ size_t stage_bytes(int nv, int mode) const {
        return ((size_t)CH * elem_bytes(nv, mode) + 127) / 128 * 128;
    }
};

template <int MAXV, int MODE>
__global__ void __launch_bounds__(NT, Ring<MAXV>::BLOCKS)
    gs_pass_staged(const double *__restrict__ V, long long ldv, int nv, GmresDev *gd, const float *w_hi,
                   const float *w_lo, float *o_hi, float *o_lo, long long n, ChunkLayout lay,
                   double *__restrict__ partials, volatile int *err) {
    constexpr int NS = Ring<MAXV>::NS;
    pdl_wait();
    if (gd->done) return;
    constexpr bool WLO = MODE == PASS_UPD_NRM;
    extern __shared__ __align__(128) unsigned char smraw[];
    unsigned char *ring = smraw + ((128u - (smem_addr(smraw) & 127u)) & 127u);
    __shared__ __align__(8) unsigned long long full[NS], empty[NS];
    __shared__ f32x2v2 coef[MAXV];   // the coefficient pair in both lanes
    __shared__ double red[NCW][MAXV];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int CH = lay.CH;
    const size_t SB = lay.stage_bytes(nv, MODE);
    if (tid < nv) {
        const double h = (MODE == PASS_UPD_DOT) ? gd->h1[tid] : ((MODE == PASS_UPD_NRM) ? gd->h2[tid] : 0.0);
        const f32x2 c = split_f64(h * gd->scale[tid]);
        coef[tid].hi = v2_pack(c.hi, c.hi);
        coef[tid].lo = v2_pack(c.lo, c.lo);
    }
    if (tid == 0) {
        for (int st = 0; st < NS; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], NCW);
        }
        mbar_init_fence();
    }
    __syncthreads();
    const long long nchunks = (n + CH - 1) / CH;
    const long long first = blockIdx.x, stride = gridDim.x;
    auto w_h_s = [&](int st) { return reinterpret_cast<float *>(ring + st * SB); };
    auto w_l_s = [&](int st) { return w_h_s(st) + CH; };
    auto v0_s = [&](int st) { return reinterpret_cast<double *>(w_h_s(st) + (WLO ? 2 : 1) * CH); };
    auto vh_s = [&](int st, int i) { return reinterpret_cast<float *>(v0_s(st) + CH) + (size_t)2 * (i - 1) * CH; };
    bool failed = false;
    f32x2v2 acc[MAXV];
#pragma unroll
    for (int i = 0; i < MAXV; ++i) acc[i] = f32x2v2{0ull, 0ull};

    if (warp == NCW) {
        // producer: lane 0 arms the stage's barrier, then the lanes share its copies
        long long issued = 0;
        for (long long chunk = first; chunk < nchunks; chunk += stride, ++issued) {
            const int st = (int)(issued % NS);
            if (issued >= NS) {
                // the consumers released this stage's previous chunk
                const bool ok = mbar_wait_bounded(&empty[st], (unsigned)(((issued / NS) - 1) & 1));
                if (__any_sync(0xffffffffu, !ok)) { failed = true; break; }
            }
            const long long e0 = chunk * CH;
            const unsigned len = (unsigned)std::min<long long>(CH, n - e0);
            if (lane == 0) mbar_expect_tx(&full[st], len * (unsigned)elem_bytes(nv, MODE));
            __syncwarp();
            // copy q: 0 w hi, 1 w lo (pass C), 2 V_0, 3 + 2 (i - 1) (+1) the hi (lo) plane of V_i
            for (int q = lane; q < 3 + 2 * (nv - 1); q += 32) {
                if (q == 0) bulk_load(w_h_s(st), w_hi + e0, len * 4u, &full[st]);
                else if (q == 1) { if (WLO) bulk_load(w_l_s(st), w_lo + e0, len * 4u, &full[st]); }
                else if (q == 2) bulk_load(v0_s(st), V + e0, len * 8u, &full[st]);
                else {
                    const int i = 1 + (q - 3) / 2, lo = (q - 3) & 1;
                    const float *b = reinterpret_cast<const float *>(V + i * ldv) + (lo ? n : 0);
                    bulk_load(vh_s(st, i) + (lo ? CH : 0), b + e0, len * 4u, &full[st]);
                }
            }
        }
        if (failed && lane == 0) {
            *err = 1;
            __threadfence_system();
        }
        // copies still in flight land in this block's shared memory: wait for them (bounded)
        if (lane == 0)
            for (long long k = std::max(0LL, issued - NS); k < issued; ++k)
                mbar_wait_bounded(&full[k % NS], (unsigned)((k / NS) & 1));
    } else {
        long long k = 0;
        for (long long chunk = first; chunk < nchunks; chunk += stride, ++k) {
            const int st = (int)(k % NS);
            if (__any_sync(0xffffffffu, !mbar_wait_bounded(&full[st], (unsigned)((k / NS) & 1)))) {
                failed = true;
                break;
            }
            const long long e0 = chunk * CH;
            const int len = (int)std::min<long long>(CH, n - e0);
            const float *wh = w_h_s(st), *wl = w_l_s(st);
            const double *v0 = v0_s(st);
            // two adjacent elements a thread, in the two lanes of packed registers (len is even);
            // the basis values are read from the stage where they are used (no array of them
            // held across the loops)
            for (int r = 2 * tid; r < len; r += 2 * NC) {
                f32x2v2 w;
                w.hi = *reinterpret_cast<const f32v2 *>(wh + r);
                w.lo = WLO ? *reinterpret_cast<const f32v2 *>(wl + r) : 0ull;
                f32x2v2 v0p;
                {
                    const double2 d = *reinterpret_cast<const double2 *>(v0 + r);
                    const f32x2 s0 = split_f64(d.x), s1 = split_f64(d.y);
                    v0p.hi = v2_pack(s0.hi, s1.hi);
                    v0p.lo = v2_pack(s0.lo, s1.lo);
                }
                auto vload = [&](int i) {
                    const float *b = vh_s(st, i);
                    f32x2v2 q;
                    q.hi = *reinterpret_cast<const f32v2 *>(b + r);
                    q.lo = *reinterpret_cast<const f32v2 *>(b + CH + r);
                    return q;
                };
                if (MODE == PASS_DOT) {
                    fma_acc_v2(v0p, w, acc[0]);
#pragma unroll
                    for (int i = 1; i < MAXV; ++i)
                        if (i < nv) fma_acc_v2(vload(i), w, acc[i]);
                } else {
                    f32x2v2 u{0ull, 0ull};
                    fma_acc_v2(coef[0], v0p, u);
#pragma unroll
                    for (int i = 1; i < MAXV; ++i)
                        if (i < nv) fma_acc_v2(coef[i], vload(i), u);
                    const f32x2v2 wn = sub_pair_v2(w, u);
                    *reinterpret_cast<f32v2 *>(o_hi + e0 + r) = wn.hi;
                    *reinterpret_cast<f32v2 *>(o_lo + e0 + r) = wn.lo;
                    if (MODE == PASS_UPD_DOT) {
                        fma_acc_v2(v0p, wn, acc[0]);
#pragma unroll
                        for (int i = 1; i < MAXV; ++i)
                            if (i < nv) fma_acc_v2(vload(i), wn, acc[i]);
                    } else {
                        fma_acc_v2(wn, wn, acc[0]);
                    }
                }
            }
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&empty[st])) : "memory");
        }
        if (failed && lane == 0) {
            *err = 1;
            __threadfence_system();
        }
    }
    // block reduction over the consumer warps (the producer's accumulators are zero)
    const int nout = MODE == PASS_UPD_NRM ? 1 : nv;
    if (warp < NCW) {
#pragma unroll
        for (int i = 0; i < MAXV; ++i) {
            if (i < nout) {
                double v = failed ? 0.0 : pair_v2_to_f64(acc[i]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane == 0) red[warp][i] = v;
            }
        }
    }
    __syncthreads();
    double *out = partials + (long long)blockIdx.x * RB_STRIDE;
    for (int i = tid; i < nout; i += NT) {
        double t = 0.0;
        for (int w = 0; w < NCW; ++w) t += red[w][i];
        out[i] = t;
    }
    if (last_block_arrived(&gd->arrived)) arnoldi_finish(partials, gridDim.x, nv, gd, MODE, nv - 1);
}

template <int MAXV, int MODE>
static cudaError_t launch_one(llg_ctx *c, const double *V, long long ldv, int nv, const float *wh, const float *wl,
                              float *oh, float *ol, long long n) {
    ChunkLayout lay;
    lay.CH = std::max(4, (Ring<MAXV>::TARGET / elem_bytes(nv, MODE)) / 4 * 4);
    if (lay.CH > n) lay.CH = (int)((n + 3) / 4 * 4);
    const size_t sm = Ring<MAXV>::NS * lay.stage_bytes(nv, MODE) + 128;
    auto k = gs_pass_staged<MAXV, MODE>;
    cudaError_t e = set_smem(k, sm);
    if (e != cudaSuccess) return e;
    int per = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, NT, sm)) != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    const long long nchunks = (n + lay.CH - 1) / lay.CH;
    const int blocks = (int)std::min<long long>(nchunks, std::min(per * c->sm_count, partial_capacity(c)));
    return launch_pdl(k, dim3(blocks), dim3(NT), sm, c->stream, V, ldv, nv, c->gdev, wh, wl, oh, ol, n, lay, c->red,
                      c->dprog + KERR_WORD);
}

template <int MAXV>
static cudaError_t launch_nv(llg_ctx *c, int mode, const double *V, long long ldv, int nv, const float *wh,
                             const float *wl, float *oh, float *ol, long long n) {
    if (mode == PASS_DOT) return launch_one<MAXV, PASS_DOT>(c, V, ldv, nv, wh, wl, oh, ol, n);
    if (mode == PASS_UPD_DOT) return launch_one<MAXV, PASS_UPD_DOT>(c, V, ldv, nv, wh, wl, oh, ol, n);
    return launch_one<MAXV, PASS_UPD_NRM>(c, V, ldv, nv, wh, wl, oh, ol, n);
}

bool available(const llg_ctx *c, long long n) { return c->dprog != nullptr && n % 4 == 0; }

cudaError_t pass(llg_ctx *c, int mode, const double *V, long long ldv, int nv, const float *wh, const float *wl,
                 float *oh, float *ol, long long n) {
#define LLG_GSN(K) case K: return launch_nv<K>(c, mode, V, ldv, nv, wh, wl, oh, ol, n);
    switch (nv) {
        LLG_GSN(1) LLG_GSN(2) LLG_GSN(3) LLG_GSN(4) LLG_GSN(5) LLG_GSN(6) LLG_GSN(7) LLG_GSN(8)
        LLG_GSN(9) LLG_GSN(10) LLG_GSN(11) LLG_GSN(12) LLG_GSN(13) LLG_GSN(14) LLG_GSN(15) LLG_GSN(16)
        LLG_GSN(17) LLG_GSN(18) LLG_GSN(19) LLG_GSN(20) LLG_GSN(21) LLG_GSN(22) LLG_GSN(23) LLG_GSN(24)
        LLG_GSN(25) LLG_GSN(26) LLG_GSN(27) LLG_GSN(28) LLG_GSN(29) LLG_GSN(30) LLG_GSN(31) LLG_GSN(32)
        default: break;
    }
#undef LLG_GSN
    return cudaErrorInvalidValue;
}

}  // namespace gst
}  // namespace llg
