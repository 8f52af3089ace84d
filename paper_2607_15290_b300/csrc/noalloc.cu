// noalloc.cu -- llg_ffthss_apply_noalloc: the FFT--HSS preconditioner application
// for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: a time-critical loop that has
// promised no allocation after start-up, an application whose device memory is
// fully reserved by another allocator (a framework's caching allocator or a fixed
// pool, where an extra cudaMalloc fails or fragments), or a plug-in environment that
// is not allowed to create device allocations.  llg_create allocates tables and
// scratch, so those callers cannot use the context API.  This entry point needs no
// context: its spectral scratch, twiddle and symbol tables live in one file-scope
// static device array of fixed size, which every GPU that loads the library holds
// until the process exits.  The caller still passes the inputs and the output.
//
// In host code the array's name is only a host-side stand-in, not a device
// address, so every call fetches the device address for the current device with
// cudaGetSymbolAddress (which allocates nothing; a fetch per call also keeps a
// device reset from leaving a stale address behind) and the kernels get that
// address.  The first call on a device also loads the module there, so it should
// come before any stream capture.
// All calls share the array and it keeps the last call's contents: each call
// rewrites the tables and clears the spectral region it uses, and calls that
// overlap on the GPU (other streams or threads) race on it.
#include <cmath>
#include <cstring>
#include "spectral_kernels.cuh"

namespace {

using namespace llg;

// tables: 3 twiddle tables of up to 1024 complex values, then 3 symbol tables of up
// to 1024 doubles (stored two per slot); the spectral scratch follows
constexpr long long TW_SLOTS = 3 * 1024;
constexpr long long SIG_SLOTS = 3 * 1024 / 2;
constexpr long long TABLE_SLOTS = TW_SLOTS + SIG_SLOTS;
constexpr long long SPEC_SLOTS = LLG_NOALLOC_MAX_SPECTRAL;

static __device__ __align__(256) double2 g_noalloc_scratch[TABLE_SLOTS + SPEC_SLOTS];

// with the device current: the device address of the static array and the SM count
llg_status device_scratch(double2 **ptr, int *sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return LLG_ERR_CUDA; }
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) { cudaGetLastError(); return LLG_ERR_CUDA; }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
        cudaGetLastError();
        return LLG_ERR_CUDA;
    }
    *ptr = static_cast<double2 *>(p);
    *sms = n;
    return LLG_OK;
}

// per-axis twiddles exp(-2 pi i j / n) and symbols of -Lap_N for this grid
__global__ void k_noalloc_tables(double2 *tw, double *sig, int dim, int n0, int n1, int n2, double L0, double L1,
                                 double L2, int exchange) {
    const int axis = blockIdx.x;
    const int n = axis == 0 ? n0 : (axis == 1 ? n1 : n2);
    const double L = axis == 0 ? L0 : (axis == 1 ? L1 : L2);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)i / (double)n, &s, &c);
        tw[axis * 1024 + i] = make_double2(c, -s);
        const int kw = i < n / 2 ? i : i - n;
        double v = 0.0;
        if (axis < dim) {
            if (exchange == LLG_EX_FD2) {
                const double h = L / n, sn = sinpi((double)kw / (double)n);
                v = 4.0 / (h * h) * sn * sn;
            } else {
                const double xi = 2.0 * 3.141592653589793238462643383279502884 * (double)kw / L;
                v = xi * xi;
            }
        }
        sig[axis * 1024 + i] = v;
    }
}

template <int E>
cudaError_t launch_rows(bool fwd, bool transpose, RowArgs<double, double, double> a, int blocks, int threads,
                        size_t sm, cudaStream_t st) {
    if (fwd) {
        auto k = transpose ? row_fwd_kernel<double, double, double, E, IN_NODAL_T>
                           : row_fwd_kernel<double, double, double, E, IN_V>;
        cudaError_t e = set_smem(k, sm);
        if (e != cudaSuccess) return e;
        k<<<blocks, threads, sm, st>>>(a);
    } else {
        auto k = transpose ? row_inv_kernel<double, double, double, E, OUT_PLAIN>
                           : row_inv_kernel<double, double, double, E, OUT_APPLY>;
        cudaError_t e = set_smem(k, sm);
        if (e != cudaSuccess) return e;
        k<<<blocks, threads, sm, st>>>(a);
    }
    return cudaGetLastError();
}

template <int E, int TW>
cudaError_t launch_cols_ETW(int mode, const ColArgs<double> &a, dim3 grid, cudaStream_t st) {
    const size_t sm = (size_t)a.nl * TW * sizeof(double2);
    const int threads = TW * (a.nl / E);
    auto k = mode == 1 ? col_kernel<double, E, TW, 1> : (mode == 2 ? col_kernel<double, E, TW, 2> : col_kernel<double, E, TW, 7>);
    cudaError_t e = set_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<grid, threads, sm, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_cols(int mode, const ColArgs<double> &a, dim3 grid, cudaStream_t st) {
    const ColPlan p = col_plan<double>(a.nl);
    if (p.E == 2 && p.TW == 8) return launch_cols_ETW<2, 8>(mode, a, grid, st);
    if (p.E == 4 && p.TW == 8) return launch_cols_ETW<4, 8>(mode, a, grid, st);
    if (p.E == 8 && p.TW == 8) return launch_cols_ETW<8, 8>(mode, a, grid, st);
    if (p.E == 8 && p.TW == 4) return launch_cols_ETW<8, 4>(mode, a, grid, st);
    return cudaErrorInvalidValue;
}

bool pow2_ok(int n) { return n >= 2 && n <= 1024 && (n & (n - 1)) == 0; }

}  // namespace

extern "C" llg_status llg_ffthss_apply_noalloc(const llg_grid *grid, const llg_params *prm, const double *m,
                                               const double *p, double *z, int transpose, void *cuda_stream) {
    if (!grid || !prm || !m || !p || !z) return LLG_ERR_INVALID_ARG;
    if (grid->dim != 2 && grid->dim != 3) return LLG_ERR_INVALID_ARG;
    int n[3] = {1, 1, 1};
    double Lc[3] = {1.0, 1.0, 1.0};
    for (int l = 0; l < grid->dim; ++l) {
        if (!pow2_ok(grid->n[l])) return LLG_ERR_UNSUPPORTED_SIZE;
        if (!(grid->L[l] > 0) || !std::isfinite(grid->L[l])) return LLG_ERR_INVALID_ARG;
        n[l] = grid->n[l];
        Lc[l] = grid->L[l];
    }
    const double vals[] = {prm->alpha, prm->c_ex, prm->k, prm->theta, prm->lambda};
    for (double d : vals)
        if (!std::isfinite(d)) return LLG_ERR_INVALID_ARG;
    if (!(prm->alpha > 0) || !(prm->c_ex > 0) || !(prm->lambda > 0) || prm->k < 0 || !(prm->theta > 0))
        return LLG_ERR_INVALID_ARG;
    if (prm->exchange != LLG_EX_SPECTRAL && prm->exchange != LLG_EX_FD2) return LLG_ERR_INVALID_ARG;
    const long long rows = (long long)n[1] * n[2];
    const int S = ((n[0] + n[0] / 2 + 1) + 15) / 16 * 16;
    if (rows * S > SPEC_SLOTS) return LLG_ERR_UNSUPPORTED_SIZE;   // beyond the static scratch

    double2 *base = nullptr;
    int sms = 0;
    llg_status st = device_scratch(&base, &sms);
    if (st != LLG_OK) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    double2 *tw = base;
    double *sig = reinterpret_cast<double *>(base + TW_SLOTS);
    double2 *spec = base + TABLE_SLOTS;

    k_noalloc_tables<<<3, 256, 0, stream>>>(tw, sig, grid->dim, n[0], n[1], n[2], Lc[0], Lc[1], Lc[2], prm->exchange);
    if (cudaGetLastError() != cudaSuccess) return LLG_ERR_CUDA;
    if (cudaMemsetAsync(spec, 0, sizeof(double2) * rows * S, stream) != cudaSuccess) { cudaGetLastError(); return LLG_ERR_CUDA; }

    const long long N = rows * n[0];
    const double chat = (1.0 + prm->alpha * prm->alpha) * prm->c_ex;
    const int logn[3] = {(int)std::lround(std::log2((double)n[0])), (int)std::lround(std::log2((double)n[1])),
                         (int)std::lround(std::log2((double)n[2]))};

    // x-passes: same launch shape as the context path
    const int E = row_E<double>(n[0]), P = n[0] / E;
    const long long pairs = rows / 2;
    int G = 256 / (3 * P);
    if (G < 1) G = 1;
    const long long want = pairs / (2LL * sms);
    if (want < G) G = (int)(want < 1 ? 1 : want);
    const int blocks = (int)((pairs + G - 1) / G), threads = 3 * G * P;
    const size_t smr = (size_t)3 * G * RowLayout::size(n[0]) * sizeof(double2);
    RowArgs<double, double, double> ra;
    ra.spec = spec; ra.tw0 = tw; ra.n0 = n[0]; ra.logn0 = logn[0]; ra.S = S; ra.G = G; ra.rows = rows; ra.N = N;
    std::memset(&ra.io, 0, sizeof(ra.io));
    ra.io.m = m; ra.io.x = p; ra.io.y = z; ra.io.scale = nullptr; ra.io.lam = prm->lambda;

    // axis passes with the shifted exchange symbol 1 / (alpha + lambda + theta k Chat sigma), 1/N_g folded in
    ColArgs<double> ca{};
    ca.spec = spec; ca.n0 = n[0]; ca.S = S; ca.tx = sig;
    ca.sa = prm->alpha + prm->lambda; ca.sb = prm->theta * prm->k * chat; ca.sscale = 1.0 / (double)N; ca.sinv = 1;

    auto rows_pass = [&](bool fwd) -> cudaError_t {
        switch (E) {
            case 2: return launch_rows<2>(fwd, transpose != 0, ra, blocks, threads, smr, stream);
            case 4: return launch_rows<4>(fwd, transpose != 0, ra, blocks, threads, smr, stream);
            default: return launch_rows<8>(fwd, transpose != 0, ra, blocks, threads, smr, stream);
        }
    };
    auto tiles = [&](int nl) { return S / col_plan<double>(nl).TW; };
    if (rows_pass(true) != cudaSuccess) return LLG_ERR_CUDA;
    if (grid->dim == 2) {
        ca.tw = tw + 1024; ca.nl = n[1]; ca.logn = logn[1]; ca.ls = S; ca.bs = 0;
        ca.tl = sig + 1024; ca.tb = nullptr;
        if (launch_cols(7, ca, dim3(tiles(n[1]), 1), stream) != cudaSuccess) return LLG_ERR_CUDA;
    } else {
        ColArgs<double> cy = ca;
        cy.tw = tw + 1024; cy.nl = n[1]; cy.logn = logn[1]; cy.ls = S; cy.bs = (long long)n[1] * S;
        cy.tl = nullptr; cy.tb = nullptr;
        ColArgs<double> cz = ca;
        cz.tw = tw + 2048; cz.nl = n[2]; cz.logn = logn[2]; cz.ls = (long long)n[1] * S; cz.bs = S;
        cz.tl = sig + 2048; cz.tb = sig + 1024;
        if (launch_cols(1, cy, dim3(tiles(n[1]), n[2]), stream) != cudaSuccess) return LLG_ERR_CUDA;
        if (launch_cols(7, cz, dim3(tiles(n[2]), n[1]), stream) != cudaSuccess) return LLG_ERR_CUDA;
        if (launch_cols(2, cy, dim3(tiles(n[1]), n[2]), stream) != cudaSuccess) return LLG_ERR_CUDA;
    }
    if (rows_pass(false) != cudaSuccess) return LLG_ERR_CUDA;
    return LLG_OK;
}
