// col_tma.cu -- FP32 axis passes (y forward, z with the multiplier, y inverse; the y pass
// of 2D grids) as persistent kernels whose tiles move between HBM and shared memory by
// the tensor memory accelerator.
//
// A tile is TW adjacent spectral columns of one batch (all n points of each line).  Each
// block walks its share of the tiles through a three-stage ring in shared memory: while
// it transforms tile i, the load of tile i+1 (cp.async.bulk.tensor, completion
// on an mbarrier) and the store of tile i-1 (cp.async.bulk.tensor from shared memory)
// are in flight, so the memory traffic of one tile overlaps the arithmetic of another
// within the block, and the register kernels' load -> transform -> store sequence no
// longer leaves the memory system idle.
//
// Every wait on an mbarrier is bounded by a clock budget.  A wait that runs out raises
// the error word in host-mapped memory (the host reports LLG_ERR_TIMEOUT), waits (again
// bounded) for the block's loads in flight and drains its stores, and the block returns.
#include <algorithm>
#include <cuda.h>
#include "spectral_ct.cuh"
#include "col_tma.h"
#include "tma_ptx.cuh"

namespace llg {
namespace tma {

constexpr int STAGES = 3;

// The round trip of the z pass (forward, multiplier, inverse) exchanges through a fourth
// tile beside the ring (one barrier per stage instead of two; measured 7% faster at 256^3);
// the one-way y passes transform in place, where the smaller footprint keeps one more block
// per SM resident (measured 6% faster than with the exchange tile).
__host__ __device__ constexpr bool uses_exchange(int mode) { return mode == 7; }
__host__ __device__ constexpr int tiles_held(int mode) { return STAGES + (uses_exchange(mode) ? 1 : 0); }

// tile t -> tensor coordinates: column block bx (x = 2 TW bx floats), batch b along the
// axis that is not transformed (y for the z pass, z for y passes)
struct TileMap {
    int tiles_x, ntiles, axis_z;
};

// E points of a line per thread: 8 (radix-8 stages) or 16 (radix-16 stages: half the
// shared-memory exchanges of a 256-point line)
template <int LOGN, int TW, int MODE, int E>
__global__ void __launch_bounds__(TW *((1 << LOGN) / E)) col_tma_kernel(const __grid_constant__ CUtensorMap map,
                                                                        ColArgs<float> a, TileMap tm, volatile int *err) {
    constexpr int N = 1 << LOGN, P = N / E, LR = E == 16 ? 4 : 3;
    constexpr int TILE = N * TW;                         // float2 elements
    constexpr unsigned BYTES = TILE * sizeof(float2);
    using L = ct::ColL<TW>;
    constexpr bool XB = uses_exchange(MODE);
    extern __shared__ __align__(128) unsigned char smraw[];
    // bulk tensor copies want 128-byte aligned shared addresses (one spare line is allocated)
    float2 *ring = reinterpret_cast<float2 *>(smraw + ((128u - (smem_addr(smraw) & 127u)) & 127u));
    __shared__ __align__(8) unsigned long long bar[STAGES];
    __shared__ int s_ok;
    pdl_wait();
    if (a.skip && *a.skip) return;
    const int tid = threadIdx.x, c = tid % TW, t = tid / TW;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
        // the initialised barriers are visible to the copy engine
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async();
    }
    __syncthreads();
    auto coords = [&](int tile, int &x, int &y, int &z) {
        const int bx = tile % tm.tiles_x, b = tile / tm.tiles_x;
        x = 2 * TW * bx;
        y = tm.axis_z ? b : 0;
        z = tm.axis_z ? 0 : b;
    };
    const int first = blockIdx.x, stride = gridDim.x;
    if (tid == 0 && first < tm.ntiles) {
        int x, y, z;
        coords(first, x, y, z);
        mbar_expect_tx(&bar[0], BYTES);
        tma_load(ring, &map, &bar[0], x, y, z);
    }
    bool failed = false;
    int it = 0;
    for (int tile = first; tile < tm.ntiles; tile += stride, ++it) {
        const int s = it % STAGES;
        const unsigned parity = (unsigned)((it / STAGES) & 1);
        if (tid == 0) {
            const int next = tile + stride;
            if (next < tm.ntiles) {
                // the stage of the next tile was last used by tile it-2, whose store must
                // have read it (at most the store of tile it-1 may still be pending)
                const int sn = (it + 1) % STAGES;
                bulk_wait_read_1();
                int x, y, z;
                coords(next, x, y, z);
                mbar_expect_tx(&bar[sn], BYTES);
                tma_load(ring + sn * TILE, &map, &bar[sn], x, y, z);
            }
            s_ok = mbar_wait_bounded(&bar[s], parity) ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) { failed = true; break; }
        // every thread acquires the completed phase (it completed already: no wait); the
        // decision to give up stays uniform over the block
        if (__syncthreads_or(mbar_wait_bounded(&bar[s], parity) ? 0 : 1)) { failed = true; break; }
        float2 *T = ring + s * TILE + c;
        float2 v[E];
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = T[(t + P * q) * TW];
        const int bx = tile % tm.tiles_x, b = tile / tm.tiles_x;
        if constexpr (XB) {
            // round trip: stage 0 stores into the exchange tile X, so no thread waits for the
            // others' loads of T, and the two buffers alternate with one barrier per stage
            float2 *X = ring + STAGES * TILE + c;
            ct::fft<LOGN, E, -1, L, 1, true, LR>(v, T, X, t, a.tw);
            ct::apply_symbol<float, LOGN, E, L>(v, a, bx * TW + c, b, t);
            ct::fft<LOGN, E, +1, L, ct::FreeBuf<LOGN, E, 1, LR>::value, true, LR>(v, T, X, t, a.tw);
        } else {
            if constexpr ((MODE & 1) != 0) ct::fft<LOGN, E, -1, L, 0, false, LR>(v, T, T, t, a.tw);
            if constexpr ((MODE & 4) != 0) ct::apply_symbol<float, LOGN, E, L>(v, a, bx * TW + c, b, t);
            if constexpr ((MODE & 2) != 0) ct::fft<LOGN, E, +1, L, 0, false, LR>(v, T, T, t, a.tw);
        }
        __syncthreads();   // every load of the last stage precedes the write-back
#pragma unroll
        for (int q = 0; q < E; ++q) T[(t + P * q) * TW] = v[q];
        fence_proxy_async();   // this thread's writes are visible to the copy engine
        __syncthreads();
        if (tid == 0) {
            int x, y, z;
            coords(tile, x, y, z);
            tma_store(&map, ring + s * TILE, x, y, z);
            bulk_commit();
        }
    }
    if (tid == 0) {
        if (failed) {
            *err = 1;
            __threadfence_system();
            // loads still in flight land in this block's shared memory: wait for them (bounded)
            for (int k = 0; k < 2; ++k) {   // tile it and the one issued after it
                const int idx = it + k;
                if (first + idx * stride < tm.ntiles) mbar_wait_bounded(&bar[idx % STAGES], (unsigned)((idx / STAGES) & 1));
            }
        }
        bulk_wait_all();
    }
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

bool available(const llg_ctx *c, int nl) {
    return c->dprog != nullptr && (nl == 128 || nl == 256) && encoder() != nullptr;
}

template <int LOGN, int TW, int MODE, int E>
static cudaError_t launch_one(llg_ctx *c, const CUtensorMap &map, const ColArgs<float> &a, TileMap tm) {
    constexpr int N = 1 << LOGN, threads = TW * (N / E);
    constexpr size_t sm = (size_t)tiles_held(MODE) * N * TW * sizeof(float2) + 128;
    auto k = col_tma_kernel<LOGN, TW, MODE, E>;
    cudaError_t e = set_smem(k, sm);
    if (e != cudaSuccess) return e;
    int per = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, sm)) != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    const int blocks = std::min(tm.ntiles, per * sms);
    return launch_pdl(k, dim3(blocks), dim3(threads), sm, c->stream, map, a, tm, c->dprog + KERR_WORD);
}

template <int LOGN, int TW, int E>
static cudaError_t launch_mode(llg_ctx *c, int mode, const CUtensorMap &map, const ColArgs<float> &a, TileMap tm) {
    if (mode == 1) return launch_one<LOGN, TW, 1, E>(c, map, a, tm);
    if (mode == 2) return launch_one<LOGN, TW, 2, E>(c, map, a, tm);
    if (mode == 7) return launch_one<LOGN, TW, 7, E>(c, map, a, tm);
    return cudaErrorInvalidValue;
}

template <int LOGN, int TW>
static cudaError_t launch_e(llg_ctx *c, int mode, int E, const CUtensorMap &map, const ColArgs<float> &a, TileMap tm) {
    return E == 16 ? launch_mode<LOGN, TW, 16>(c, mode, map, a, tm) : launch_mode<LOGN, TW, 8>(c, mode, map, a, tm);
}

cudaError_t col_launch(llg_ctx *c, int mode, const ColArgs<float> &a, int batches, int TW, int E) {
    const SpecGeom &g = c->geo;
    EncodeTiled enc = encoder();
    if (!enc || !c->dprog || (a.nl != 128 && a.nl != 256) || (TW != 8 && TW != 16) || (E != 8 && E != 16))
        return cudaErrorNotSupported;
    // the spectrum as a 3D tensor of floats: (2 S, n1, n2), rows of S complex slots
    const bool axis_z = a.ls != (long long)g.S;   // the z pass steps n1 S between line points
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * g.S), (cuuint64_t)g.n[1], (cuuint64_t)(g.dim == 3 ? g.n[2] : 1)};
    const cuuint64_t strides[2] = {(cuuint64_t)g.S * sizeof(float2), (cuuint64_t)g.n[1] * g.S * sizeof(float2)};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * TW), axis_z ? 1u : (cuuint32_t)a.nl, axis_z ? (cuuint32_t)a.nl : 1u};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap map;
    const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)a.spec, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    TileMap tm;
    tm.tiles_x = g.S / TW;
    tm.ntiles = tm.tiles_x * batches;
    tm.axis_z = axis_z ? 1 : 0;
    if (a.nl == 128) return TW == 16 ? launch_e<7, 16>(c, mode, E, map, a, tm) : launch_e<7, 8>(c, mode, E, map, a, tm);
    return TW == 16 ? launch_e<8, 16>(c, mode, E, map, a, tm) : launch_e<8, 8>(c, mode, E, map, a, tm);
}

}  // namespace tma
}  // namespace llg
