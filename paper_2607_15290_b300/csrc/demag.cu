// demag.cu -- the periodic zero-mean demagnetising field and the uniaxial anisotropy
// field of the lower-order field h_low (Sec. 2.1-2.2; the test problem of Sec. 4.6):
//
//   h_dem^(xi) = -xi' (xi' . m^(xi)) / |xi|^2  (xi != 0),  h_dem^(0) = 0,
//   xi = 2 pi k / L per axis, xi' = xi with the Nyquist component set to zero
//   (the first-derivative wavevector, which keeps the field real);
//   h_ani = 2 k_an (e . m) e.
//
// The demagnetising multiplier couples the three components at one mode, so this
// Fourier round trip transforms every component on its own: the x pass packs two grid
// rows of ONE component into a complex line (c[ya] + i c[yb]) and splits the result
// into the two half spectra, stored per row at slots [c H, c H + H) with H = n0/2 + 1
// (3H <= S for every supported n0).  The middle axis (3D) is transformed by the
// ordinary axis passes; the last axis pass loads the three components' lines of the
// same (kx, ky), transforms them, applies the multiplier mode by mode and transforms
// back.  FP64 only: the field is evaluated once per Picard iteration, outside GMRES.
#include <algorithm>
#include <vector>
#include "spectral_kernels.cuh"

namespace llg {

struct DemagRowArgs {
    double2 *spec;
    const double2 *tw0;
    int n0, logn0, S, G;
    long long rows, N;
    const double *m;   // 3 planes (x pass forward)
    double *h;         // 3 planes (x pass inverse)
};

// x pass forward: line 3g + c of the block holds component c of rows 2g (real part)
// and 2g + 1 (imaginary part) of the block's g-th row pair.
template <int E>
__global__ void __launch_bounds__(512) k_demag_xfwd(DemagRowArgs a) {
    using C = double2;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    constexpr int LE = E >= 8 ? 3 : (E >= 4 ? 2 : (E >= 2 ? 1 : 0));
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int n0 = a.n0, ln0 = a.logn0, P = n0 >> LE, lP = ln0 - LE, LS = RowLayout::size(n0), H = n0 / 2 + 1;
    const long long N = a.N, npairs = a.rows / 2, pair0 = (long long)blockIdx.x * a.G;
    const int total = 2 * a.G * n0;
    for (int idx = tid; idx < total; idx += nthr) {
        const int gp = idx >> (ln0 + 1), rr = (idx >> ln0) & 1, xx = idx & (n0 - 1);
        if (pair0 + gp >= npairs) continue;
        const long long j = (2 * (pair0 + gp) + rr) * n0 + xx;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            reinterpret_cast<double *>(&sm[(3 * gp + c) * LS + RowLayout::idx(xx, 1)])[rr] = a.m[c * N + j];
    }
    __syncthreads();
    const int line = tid >> lP, t = tid & (P - 1);
    const int gp = line / 3, comp = line % 3;
    const long long pair = pair0 + gp;
    const bool valid = gp < a.G && pair < npairs;
    C v[E];
#pragma unroll
    for (int q = 0; q < E; ++q) v[q] = sm[line * LS + RowLayout::idx(t + P * q, 1)];
    line_fft<E, -1, RowLayout>(v, sm + line * LS, 1, n0, ln0, t, P, a.tw0);
#pragma unroll
    for (int q = 0; q < E; ++q) sm[line * LS + RowLayout::idx(t + P * q, 1)] = v[q];
    __syncthreads();
    if (!valid) return;
    // U = FFT(c[ya] + i c[yb]):  C_a = (U_k + conj U_{-k}) / 2,  C_b = (U_k - conj U_{-k}) / (2i)
    C *da = a.spec + (2 * pair) * (long long)a.S + comp * H;
    C *db = da + a.S;
    for (int k = t; k < H; k += P) {
        const C uk = sm[line * LS + RowLayout::idx(k, 1)];
        const C um = sm[line * LS + RowLayout::idx((n0 - k) & (n0 - 1), 1)];
        da[k] = make_double2(0.5 * (uk.x + um.x), 0.5 * (uk.y - um.y));
        db[k] = make_double2(0.5 * (uk.y + um.y), -0.5 * (uk.x - um.x));
    }
}

// x pass inverse: rebuild U = C_a + i C_b of each component from its two half spectra,
// transform back and write the two rows of the field.
template <int E>
__global__ void __launch_bounds__(512) k_demag_xinv(DemagRowArgs a) {
    using C = double2;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    constexpr int LE = E >= 8 ? 3 : (E >= 4 ? 2 : (E >= 2 ? 1 : 0));
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int n0 = a.n0, ln0 = a.logn0, P = n0 >> LE, lP = ln0 - LE, LS = RowLayout::size(n0), H = n0 / 2 + 1;
    const long long N = a.N, npairs = a.rows / 2, pair0 = (long long)blockIdx.x * a.G;
    const int line = tid >> lP, t = tid & (P - 1);
    const int gp = line / 3, comp = line % 3;
    const long long pair = pair0 + gp;
    const bool valid = gp < a.G && pair < npairs;
    C v[E];
    if (valid) {
        const C *sa = a.spec + (2 * pair) * (long long)a.S + comp * H;
        const C *sb = sa + a.S;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int k = t + P * q;
            const bool lower = k <= n0 / 2;
            const int kk = lower ? k : n0 - k;
            C ca = sa[kk], cb = sb[kk];
            if (!lower) { ca.y = -ca.y; cb.y = -cb.y; }
            v[q] = make_double2(ca.x - cb.y, ca.y + cb.x);
        }
    } else {
#pragma unroll
        for (int q = 0; q < E; ++q) v[q] = make_double2(0.0, 0.0);
    }
    line_fft<E, +1, RowLayout>(v, sm + line * LS, 1, n0, ln0, t, P, a.tw0);
#pragma unroll
    for (int q = 0; q < E; ++q) sm[line * LS + RowLayout::idx(t + P * q, 1)] = v[q];
    __syncthreads();
    const int total = 2 * a.G * n0;
    for (int idx = tid; idx < total; idx += nthr) {
        const int g2 = idx >> (ln0 + 1), rr = (idx >> ln0) & 1, xx = idx & (n0 - 1);
        if (pair0 + g2 >= npairs) continue;
        const long long j = (2 * (pair0 + g2) + rr) * n0 + xx;
#pragma unroll
        for (int c = 0; c < 3; ++c)
            a.h[c * N + j] = reinterpret_cast<const double *>(&sm[(3 * g2 + c) * LS + RowLayout::idx(xx, 1)])[rr];
    }
}

struct DemagColArgs {
    double2 *spec;
    const double2 *tw;     // twiddles of the last axis
    long long ls, bs;      // stride between line elements; between batches (3D: y rows)
    int nl, logn, H, dim;
    const double *xi[3], *xp[3];   // per axis: 2 pi k / L, and the same with Nyquist zeroed
    double scale;          // 1 / N: normalisation of the round trip
};

// Last-axis pass with the demagnetising multiplier: TW columns kx of the half spectrum
// per block, each with the lines of its three components (slots kx, H + kx, 2H + kx).
// Wavevector per component c: x from the column, y from the batch (3D) or the line (2D),
// z from the line (3D) or absent (2D).
template <int E, int TW>
__global__ void __launch_bounds__(256) k_demag_last(DemagColArgs a) {
    using C = double2;
    extern __shared__ __align__(16) unsigned char smraw[];
    C *sm = reinterpret_cast<C *>(smraw);
    const int cl = threadIdx.x % TW, t = threadIdx.x / TW;
    const int P = a.nl / E;
    const int kx = blockIdx.x * TW + cl, by = blockIdx.y;
    const bool live = kx < a.H;
    C v[3][E];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const C *src = a.spec + (long long)by * a.bs + c * a.H + kx;
#pragma unroll
        for (int q = 0; q < E; ++q) v[c][q] = live ? src[(long long)(t + P * q) * a.ls] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) line_fft<E, -1, ColLayout>(v[c], sm + c * TW + cl, 3 * TW, a.nl, a.logn, t, P, a.tw);
    const double wx = live ? a.xi[0][kx] : 0.0, wxp = live ? a.xp[0][kx] : 0.0;
    const double wb = a.dim == 3 ? a.xi[1][by] : 0.0, wbp = a.dim == 3 ? a.xp[1][by] : 0.0;
    const int la = a.dim == 3 ? 2 : 1;   // axis of the line
#pragma unroll
    for (int q = 0; q < E; ++q) {
        const int e = t + P * q;
        const double wl = a.xi[la][e], wlp = a.xp[la][e];
        const double wy = a.dim == 3 ? wb : wl, wyp = a.dim == 3 ? wbp : wlp;
        const double wz = a.dim == 3 ? wl : 0.0, wzp = a.dim == 3 ? wlp : 0.0;
        const double s2 = wx * wx + wy * wy + wz * wz;
        const double f = s2 > 0.0 ? -a.scale / s2 : 0.0;
        const double dr = wxp * v[0][q].x + wyp * v[1][q].x + wzp * v[2][q].x;
        const double di = wxp * v[0][q].y + wyp * v[1][q].y + wzp * v[2][q].y;
        v[0][q] = make_double2(f * wxp * dr, f * wxp * di);
        v[1][q] = make_double2(f * wyp * dr, f * wyp * di);
        v[2][q] = make_double2(f * wzp * dr, f * wzp * di);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) line_fft<E, +1, ColLayout>(v[c], sm + c * TW + cl, 3 * TW, a.nl, a.logn, t, P, a.tw);
    if (!live) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        C *dst = a.spec + (long long)by * a.bs + c * a.H + kx;
#pragma unroll
        for (int q = 0; q < E; ++q) dst[(long long)(t + P * q) * a.ls] = v[c][q];
    }
}

// h = 2 k_an (e . m) e (+ h0 when given), three planes
__global__ void k_anisotropy_add(const double *__restrict__ m, double kan, double e0, double e1, double e2,
                                 double *h, long long N) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
        const double em = 2.0 * kan * (e0 * m[j] + e1 * m[N + j] + e2 * m[2 * N + j]);
        h[j] += em * e0;
        h[N + j] += em * e1;
        h[2 * N + j] += em * e2;
    }
}

// per-axis wavevector tables (xi, xi'), built once per context
static llg_status demag_tables(llg_ctx *c) {
    if (c->dem_tab) return LLG_OK;
    const SpecGeom &g = c->geo;
    std::vector<double> h;
    for (int l = 0; l < 3; ++l) {
        const int n = g.n[l];
        const double L = l < g.dim ? c->grid.L[l] : 1.0;
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i < n; ++i) {
                const int kw = i < n / 2 ? i : i - n;
                const double xi = l < g.dim ? 6.283185307179586476925286766559 * kw / L : 0.0;
                const bool nyq = (n % 2 == 0) && i == n / 2;
                h.push_back(pass == 1 && nyq ? 0.0 : xi);
            }
    }
    cudaError_t e = cudaMalloc(&c->dem_tab, sizeof(double) * h.size());
    if (e == cudaSuccess) e = cudaMemcpy(c->dem_tab, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(c->dem_tab);
        c->dem_tab = nullptr;
        return cuda_check(c, e, "demagnetising tables");
    }
    return LLG_OK;
}

template <int E>
static cudaError_t launch_demag_rows(llg_ctx *c, bool fwd, const DemagRowArgs &a, int blocks, int threads, size_t sm) {
    auto k = fwd ? k_demag_xfwd<E> : k_demag_xinv<E>;
    cudaError_t e = set_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<blocks, threads, sm, c->stream>>>(a);
    return cudaGetLastError();
}

template <int E, int TW>
static cudaError_t launch_demag_last(llg_ctx *c, const DemagColArgs &a, int batches) {
    const dim3 grid((a.H + TW - 1) / TW, batches);
    const size_t sm = (size_t)3 * TW * a.nl * sizeof(double2);
    auto k = k_demag_last<E, TW>;
    cudaError_t e = set_smem(k, sm);
    if (e != cudaSuccess) return e;
    k<<<grid, TW * (a.nl / E), sm, c->stream>>>(a);
    return cudaGetLastError();
}

llg_status demag_field(llg_ctx *c, const double *m, double *h) {
    llg_status st = demag_tables(c);
    if (st != LLG_OK) return st;
    const SpecGeom &g = c->geo;
    const int n0 = g.n[0], E = row_E<double>(n0), P = n0 / E;
    const long long pairs = g.rows / 2;
    int G = std::max(1, 256 / (3 * P));
    const long long want = pairs / (2LL * c->sm_count);
    if (want < G) G = (int)std::max(1LL, want);
    const int blocks = (int)((pairs + G - 1) / G), threads = 3 * G * P;
    const size_t smr = (size_t)3 * G * RowLayout::size(n0) * sizeof(double2);
    DemagRowArgs ra;
    ra.spec = c->spec64; ra.tw0 = c->tw64[0];
    ra.n0 = n0; ra.logn0 = g.logn[0]; ra.S = g.S; ra.G = G;
    ra.rows = g.rows; ra.N = g.N; ra.m = m; ra.h = h;
    auto rows = [&](bool fwd) -> cudaError_t {
        switch (E) {
            case 1: return launch_demag_rows<1>(c, fwd, ra, blocks, threads, smr);
            case 2: return launch_demag_rows<2>(c, fwd, ra, blocks, threads, smr);
            case 4: return launch_demag_rows<4>(c, fwd, ra, blocks, threads, smr);
            default: return launch_demag_rows<8>(c, fwd, ra, blocks, threads, smr);
        }
    };
    cudaError_t e = rows(true);
    c->launches++;
    if (e != cudaSuccess) return cuda_check(c, e, "demag x-pass forward");
    if (g.dim == 3 && (st = plain_axis_pass64(c, 1, true)) != LLG_OK) return st;
    DemagColArgs ca;
    const int la = g.dim == 3 ? 2 : 1;
    ca.spec = c->spec64; ca.tw = c->tw64[la];
    ca.nl = g.n[la]; ca.logn = g.logn[la]; ca.H = n0 / 2 + 1; ca.dim = g.dim;
    ca.ls = g.dim == 3 ? (long long)g.n[1] * g.S : g.S;
    ca.bs = g.dim == 3 ? g.S : 0;
    for (int l = 0; l < 3; ++l) {
        long long off = 0;
        for (int q = 0; q < l; ++q) off += 2LL * g.n[q];
        ca.xi[l] = c->dem_tab + off;
        ca.xp[l] = c->dem_tab + off + g.n[l];
    }
    ca.scale = 1.0 / (double)g.N;
    const int batches = g.dim == 3 ? g.n[1] : 1, El = ca.nl >= 8 ? 8 : ca.nl;
    // at most 256 threads (TW nl / 8) and 3 TW nl FP64 complex of shared memory (96 KB)
    const int TW = ca.nl >= 256 ? 2048 / ca.nl : 8;
    switch (El) {
        case 1: e = launch_demag_last<1, 8>(c, ca, batches); break;
        case 2: e = launch_demag_last<2, 8>(c, ca, batches); break;
        case 4: e = launch_demag_last<4, 8>(c, ca, batches); break;
        default:
            e = TW == 2 ? launch_demag_last<8, 2>(c, ca, batches)
                        : (TW == 4 ? launch_demag_last<8, 4>(c, ca, batches) : launch_demag_last<8, 8>(c, ca, batches));
            break;
    }
    c->launches++;
    if (e != cudaSuccess) return cuda_check(c, e, "demag last-axis pass");
    if (g.dim == 3 && (st = plain_axis_pass64(c, 1, false)) != LLG_OK) return st;
    e = rows(false);
    c->launches++;
    return cuda_check(c, e, "demag x-pass inverse");
}

llg_status anisotropy_add(llg_ctx *c, const double *m, double kan, const double e_an[3], double *h) {
    k_anisotropy_add<<<4 * c->sm_count, 256, 0, c->stream>>>(m, kan, e_an[0], e_an[1], e_an[2], h, c->geo.N);
    c->launches++;
    return cuda_check(c, cudaGetLastError(), "anisotropy field");
}

}  // namespace llg
