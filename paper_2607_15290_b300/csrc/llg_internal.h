// llg_internal.h -- context, workspace and launcher declarations shared by the
// CUDA translation units of the library (not part of the public C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <functional>
#include <vector>
#include "../../include/llg.h"
#include "fpair.cuh"

namespace llg {

// Programmatic dependent launch.  A kernel launched with launch_pdl may be launched before
// the kernel ahead of it in the stream has retired, which hides most of the launch latency
// between the many short dependent passes of a GMRES step.  Such a kernel must call
// pdl_wait() before it touches any memory: it returns once the preceding kernel has
// completed and its writes are visible (in a plain launch it is a no-op).  No kernel
// signals its dependents early: letting the next grid's blocks onto the SMs while this
// grid's last wave still runs made the FP64 passes of mid-size grids up to 20% slower.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Hint: move [p, p + bytes) of global memory into L2 (one bulk prefetch; p 16-byte aligned,
// bytes rounded down to a multiple of 16).  No completion to wait for, no effect on results.
__device__ __forceinline__ void l2_prefetch_bulk(const void *p, unsigned long long bytes) {
    const unsigned b = (unsigned)(bytes & ~15ull);
    if (b) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(b) : "memory");
}

template <typename... KP, typename... A>
inline cudaError_t launch_pdl(void (*k)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// Spectral buffer layout.  For every grid row (fixed y, z) the x-axis transform
// stores S complex slots: [0, n0) the full spectrum of the packed pair
// (c1 + i c2), [n0, n0 + n0/2] the half spectrum of the real component c3,
// and zero padding up to S (a multiple of 16 so that column tiles are uniform).
struct SpecGeom {
    int n[3];
    int logn[3];
    int dim;
    long long N;      // nodes
    long long rows;   // n1 * n2
    int S;            // complex slots per row
};

// Prologue (what is transformed) and epilogue (what is written) of a spectral
// chain: forward x-pass, axis passes with the symbol, inverse x-pass.
enum InMode {
    IN_V = 0,       // c = s * (v1, v2, v3)
    IN_FUSED = 1,   // c = s * (m x v + m r - lambda v)         [left-preconditioned operator]
    IN_M = 2,       // c = (m1, m2, m3)                          [Laplacian of the nodal field]
    IN_NODAL_T = 3, // (z, zr) = (S~ + lambda)^{-T} s x; c = z; y_r = zr / lambda   [M^{-T}]
};
enum OutMode {
    OUT_APPLY = 0,   // y = (S~ + lambda)^{-1} (w, s r / lambda)
    OUT_FUSED = 1,   // y = (S~ + lambda)^{-1} (s v + w, -s (m.v) / lambda)
    OUT_MATVEC = 2,  // y_v = w + s (m x v + m r), y_r = -s m.v     (transpose: signs of the skew part flip)
    OUT_FIELD = 3,   // y_v = w + fld, y_r = 0
    OUT_PLAIN = 4,   // y_v = w (y_r untouched)
    OUT_JT = 5,      // adjoint Jacobian transpose of a midpoint step (see api.cu)
};

// Pointwise Fourier multiplier: scale * (a + b sigma) or scale / (a + b sigma)
struct Symbol {
    double a, b, scale;
    int invert;
    int exchange;   // which sigma table
};

// storage of the nodal fields a chain of compute type T reads (FP32-pair chains read FP64)
template <typename T> struct nodal_store { using type = T; };
template <> struct nodal_store<fpair> { using type = double; };
template <typename T> using nodal_t = typename nodal_store<T>::type;

template <typename TIn, typename TOut, typename T>
struct NodalIO {
    const nodal_t<T> *m;   // nodal field used by the prologue/epilogue (3 planes)
    const TIn *x;          // input planes (4 planes; 3 for IN_M)
    TOut *y;               // output planes (4)
    const double *scale;   // optional device scalar s (NULL = 1)
    T lam;
    T fld[3];
    int transpose;         // OUT_MATVEC: use A^T
    // OUT_JT only
    const nodal_t<T> *mn;  // m^n (3 planes)
    const nodal_t<T> *vf;  // forward velocity v (3 planes) and r (1 plane, at vf + 3N)
    T half_k;              // k / 2
    // OUT_APPLY / OUT_FUSED: 1 = skip the nodal 4x4 inverse (the shifted symmetric-part
    // preconditioner (lambda I + H)^{-1} alone)
    int plain_nodal;
    // OUT_FIELD only: optional per-node field added as hs * hf (3 FP64 planes)
    const double *hf;
    double hs;
    // optional device flag: when set, every pass of the chain returns at once (operators
    // queued inside a GMRES cycle that has already converged)
    const int *skip;
};

// word of the host-mapped progress block that a kernel raises when one of its bounded
// waits runs out (the host reports LLG_ERR_TIMEOUT at its next check)
constexpr int KERR_WORD = 8;

struct Workspace {
    int restart = 0;
    long long n = 0;          // 4 N
    double *V = nullptr;      // (restart + 1) * n
    float *Z = nullptr;       // restart * n (flexible GMRES)
    double *W = nullptr;      // n
    double *T = nullptr;      // n
    double *R = nullptr;      // n
    const double *last_res = nullptr;   // final true residual of the last solve (T or V_0)
    bool pairs = false;       // the last solve stored V_1.. and w as planar FP32 pairs
};

struct GmresDev;   // device-side Arnoldi state (krylov.cu)

// launch shape of an axis pass: kind 0 = register kernel (E elements per thread, TW
// columns per block); kind 1 = staged kernel (TW = tile columns, CB = columns per
// compute sub-batch, E = 8); kind 3 = FP32 register kernel with two adjacent columns
// per thread (16-byte accesses; TW columns per tile)
// launch shape of an axis pass: kind 0 register kernel (E points per thread, TW columns),
// 1 staged tile (TW columns, CB per sub-batch), 3 two columns per thread, 4 persistent
// kernel fed by the tensor memory accelerator (TW columns per tile)
struct ColCfg {
    int kind, E, TW, CB;
};
// axis-pass slots: 2D y pass; 3D y forward, z (with multiplier), y inverse
enum { SLOT_2D = 0, SLOT_Y_FWD = 1, SLOT_Z = 2, SLOT_Y_INV = 3, NSLOT = 4 };

}  // namespace llg

struct llg_ctx {
    llg_grid grid;
    cudaStream_t stream = nullptr;
    llg::SpecGeom geo;
    // per-axis twiddle tables exp(-2 pi i j / n_axis), FP64 and FP32
    double2 *tw64[3] = {nullptr, nullptr, nullptr};
    float2 *tw32[3] = {nullptr, nullptr, nullptr};
    // per-axis symbol tables sigma_axis(index) for [spectral, fd2]
    double *sig64[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    float *sig32[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    // the same twiddle and symbol tables as FP32 pairs (FP64-accurate chains on the FP32 pipes)
    llg::cfpair *twp[3] = {nullptr, nullptr, nullptr};
    llg::fpair *sigp[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    double2 *spec64 = nullptr;   // spectral scratch, rows * S
    float2 *spec32 = nullptr;
    double *red = nullptr;       // reduction partials
    double *dsc = nullptr;       // small device scalars (norms, flags)
    double *hsc = nullptr;       // pinned host mirror of dsc
    llg::GmresDev *gdev = nullptr;
    void *ghost = nullptr;       // pinned host mirror of gdev
    volatile int *hprog = nullptr;   // host-mapped progress words of the running GMRES cycle
    volatile int *dprog = nullptr;   // the same words as the device addresses them
    int cycle_epoch = 0;         // cycles started through this context
    llg::Workspace ws;
    float *m32 = nullptr;        // FP32 copy of the nodal field (mixed precision)
    double *aux = nullptr;       // 12 N doubles of stepper scratch
    int sm_count = 148;
    int sync_every = 4;          // blocking-poll interval when hprog is unavailable
    int pass_plan = LLG_PLAN_FIVE;      // 3D FP32 round trips: LLG_PLAN_FIVE or LLG_PLAN_CLUSTER
    long long launches = 0;      // kernels launched through this context
    llg::ColCfg colcfg[2][llg::NSLOT];   // [FP32, FP64][slot] axis-pass shapes
    bool tuned[2] = {false, false};      // set by llg_autotune
    std::string err;
    // live per-kernel-class timing (llg_profile_begin/end): one event pair per launch
    struct ProfEntry { cudaEvent_t a, b; double bytes, flops; int tag; int valid; int count; };
    int prof_class = 0;
    std::vector<ProfEntry> prof;
    size_t prof_used = 0;
    int prof_open = -1;
    std::vector<std::pair<const void *, int>> occ;   // grid size per Arnoldi kernel (one full wave)
    double *dem_tab = nullptr;   // demagnetising wavevector tables (xi, xi' per axis)
};

namespace llg {

llg_status set_error(llg_ctx *c, llg_status s, const std::string &msg);
llg_status cuda_check(llg_ctx *c, cudaError_t e, const char *what);

// live profiling of one kernel class: call prof_begin right before a launch and
// prof_end right after it; both are no-ops unless that class is being profiled.
enum KClass { K_NONE = 0, K_XFWD = 1, K_AXIS = 2, K_XINV = 3, K_ARNOLDI = 4 };
// count: launches the timed interval covers (the Arnoldi passes of a step are timed as one
// interval, so that no events sit between their launches)
void prof_begin(llg_ctx *c, int cls, double bytes, double flops, int tag = -1, int count = 1);
void prof_end(llg_ctx *c);
void prof_discard(llg_ctx *c, size_t first, int min_tag);

// spectral.cu
llg_status autotune(llg_ctx *c, int prec_mask, std::string *report);
llg_status set_axis_shape(llg_ctx *c, int fp32, int slot, const ColCfg &f);
// FP64 Fourier transform along axis 1 (3D y) of every spectral column, no multiplier
llg_status plain_axis_pass64(llg_ctx *c, int axis, bool forward);
// every axis of the grid has a compile-time-length pass (the FP32-pair chains need one)
bool pair_chains_available(const llg_ctx *c);

// demag.cu: h = periodic zero-mean demagnetising field of m (3 planes, FP64; uses the FP64
// spectral buffer); h += 2 k_an (e . m) e
llg_status demag_field(llg_ctx *c, const double *m, double *h);
llg_status anisotropy_add(llg_ctx *c, const double *m, double kan, const double e_an[3], double *h);
template <typename T, typename TIn, typename TOut>
llg_status spectral_chain(llg_ctx *c, int in_mode, int out_mode, const NodalIO<TIn, TOut, T> &io,
                          const Symbol &sym);
// z = M^{-1} (s v) (IN_V, OUT_APPLY) then w = A z (IN_V unscaled, OUT_MATVEC), FP32, the first
// chain's x-pass inverse fused with the second's x-pass forward (nine passes, z still written)
bool chain_pm_available(const llg_ctx *c);
template <typename TIn1>
llg_status spectral_chain_pm(llg_ctx *c, const NodalIO<TIn1, float, float> &io1, const Symbol &sym1,
                             const NodalIO<float, float, float> &io2, const Symbol &sym2);

// reductions.cu / krylov.cu
int reduction_blocks(llg_ctx *c);
int partial_capacity(llg_ctx *c);   // blocks the partial-sum buffer red holds
llg_status dot_async(llg_ctx *c, const double *a, const double *b, long long n, double *dst_dev);

}  // namespace llg
