// Host side of libarkcos: ring geometry, kernel band tables, workspace layout and the
// C-ABI entry points declared in include/arkcos.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <new>

#include "arkcos_impl.cuh"

using namespace arkcos;

struct arkcos_grid_s {
    Grid g;
};
struct arkcos_kernel_s {
    Kernel k;
};

namespace {

thread_local char g_err[512] = "";

arkcos_status fail(arkcos_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

arkcos_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(ARKCOS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

bool is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }
int ilog2(int64_t n)
{
    int l = 0;
    while ((int64_t(1) << l) < n) ++l;
    return l;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

template <class T>
arkcos_status upload(T **dst, const std::vector<T> &src)
{
    *dst = nullptr;
    if (src.empty()) return ARKCOS_OK;
    CK(cudaMalloc((void **)dst, src.size() * sizeof(T)));
    CK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return ARKCOS_OK;
}

void free_grid_dev(Grid &g)
{
    cudaFree(g.d_n);
    cudaFree(g.d_hs);
    cudaFree(g.d_poff);
    cudaFree(g.d_soff);
    cudaFree(g.d_w);
    cudaFree(g.d_theta);
    cudaFree(g.d_tw);
    cudaFree(g.d_s2);
    cudaFree(g.d_s2f);
    cudaFree(g.d_ctab);
    cudaFree(g.d_ctabP);
    cudaFree(g.d_fb);
    cudaFree(g.d_fboff);
    for (auto &c : g.fft) cudaFree(c.reps);
    g.fft.clear();
}

// TF32 rounding (to nearest, ties away from zero), as cvt.rna.tf32.f32 does on the device.
float tf32_rna(float x)
{
    uint32_t u;
    memcpy(&u, &x, 4);
    u = (u + 0x1000u) & 0xFFFFE000u;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

// Cosine table of the tensor-core coefficient generation: for every block of 128 modes, sample
// offset f in {0, 1}, chunk of 32 samples and part (TF32 hi, lo), a 16 KiB tile of
// cos(pi m (2k + f) / N) in the no-swizzle K-major core-matrix layout (8 x 16-byte core
// matrices; K neighbours 128 bytes apart, row-octet neighbours 1024 bytes apart).  Angles are
// reduced exactly in integers and evaluated in FP64.
arkcos_status build_cos_table(Grid &g)
{
    const int NH = g.N / 2 + 1, nmb = (NH + 127) / 128, nkc = 4;
    g.nkc_tab = nkc;
    std::vector<float> tab((size_t)nmb * 2 * nkc * 2 * 4096, 0.f);
    for (int mb = 0; mb < nmb; ++mb)
        for (int f = 0; f < 2; ++f)
            for (int kc = 0; kc < nkc; ++kc) {
                float *hi = &tab[((((size_t)mb * 2 + f) * nkc + kc) * 2) * 4096];
                float *lo = hi + 4096;
                for (int r = 0; r < 128; ++r) {
                    const int64_t m = (int64_t)mb * 128 + r;
                    if (m >= NH) continue;
                    for (int k = 0; k < 32; ++k) {
                        const int64_t kk = (int64_t)kc * 32 + k;
                        const int64_t ang = (m * (2 * kk + f)) % (2 * (int64_t)g.N);
                        const double v = cos(M_PI * (double)ang / (double)g.N);
                        const float h = tf32_rna((float)v);
                        const float l = tf32_rna((float)(v - (double)h));
                        const size_t off = (size_t)((r >> 3) * 256 + (k >> 2) * 32 + (r & 7) * 4 + (k & 3));
                        hi[off] = h;
                        lo[off] = l;
                    }
                }
            }
    arkcos_status st = upload(&g.d_ctab, tab);
    if (st != ARKCOS_OK) return st;
    // the knot-projection table: chunk c of 32 modes m = 32 c + k, rows r = 128 f + t:
    // cos(pi m (2t + f) / N) (zero past N/2)
    const int nmc = (NH + 31) / 32;
    g.nmc_p = nmc;
    std::vector<float> tp((size_t)nmc * 2 * 8192, 0.f);
    for (int c = 0; c < nmc; ++c) {
        float *hi = &tp[(size_t)c * 2 * 8192], *lo = hi + 8192;
        for (int r = 0; r < 256; ++r) {
            const int64_t t = r & 127, f = r >> 7;
            for (int k = 0; k < 32; ++k) {
                const int64_t m = (int64_t)c * 32 + k;
                if (m >= NH) continue;
                const int64_t ang = (m * (2 * t + f)) % (2 * (int64_t)g.N);
                const double v = cos(M_PI * (double)ang / (double)g.N);
                const float h = tf32_rna((float)v);
                const float l = tf32_rna((float)(v - (double)h));
                const size_t off = (size_t)((r >> 3) * 256 + (k >> 2) * 32 + (r & 7) * 4 + (k & 3));
                hi[off] = h;
                lo[off] = l;
            }
        }
    }
    return upload(&g.d_ctabP, tp);
}

// Ring table -> offsets, FFT classes, twiddles and device copies.
arkcos_status finish_grid(Grid &g)
{
    g.R = (int)g.theta.size();
    g.nrep = (g.R + 1) / 2;
    g.poff.resize(g.R);
    g.soff.resize(g.R);
    int64_t po = 0, so = 0;
    for (int r = 0; r < g.R; ++r) {
        g.poff[r] = po;
        g.soff[r] = so;
        po += g.n[r];
        so += g.n[r] / 2 + 1;
    }
    g.npix = po;
    g.nspec = so;
    std::vector<float> wf(g.wgt.begin(), g.wgt.end());
    arkcos_status st;
    if ((st = upload(&g.d_n, g.n)) != ARKCOS_OK) return st;
    if ((st = upload(&g.d_hs, g.hs)) != ARKCOS_OK) return st;
    if ((st = upload(&g.d_poff, g.poff)) != ARKCOS_OK) return st;
    if ((st = upload(&g.d_soff, g.soff)) != ARKCOS_OK) return st;
    if ((st = upload(&g.d_w, wf)) != ARKCOS_OK) return st;
    if ((st = upload(&g.d_theta, g.theta)) != ARKCOS_OK) return st;
    // FFT launch classes by buffer size.  A ring of n pixels is transformed as the complex
    // sequence of its h = n/2 pixel pairs, two mirror rings at a time: buffer h (a power of
    // two) or the Bluestein size >= 2h - 1; buffers up to 1024 share one launch.  Rings whose
    // buffer would exceed kMaxFftM are split as n = 4q into four q-point Bluestein transforms
    // (class kSplitClass)
    std::vector<std::vector<int>> cls(kSplitClass + 1);
    int maxM = 2, maxpow2 = 2;
    auto buffer_of = [](int64_t l) {  // power-of-two buffer of an l-point transform (>= 2)
        if (l >= 2 && is_pow2(l)) return l;
        return std::max<int64_t>(2, int64_t(1) << ilog2(2 * l - 1));
    };
    auto bluestein = [](int64_t l) { return l < 2 || !is_pow2(l); };
    for (int j = 0; j < g.nrep; ++j) {
        const int n = g.n[j];
        const int64_t M = buffer_of(n / 2);
        if (is_pow2(n)) maxpow2 = std::max(maxpow2, n);
        if (M <= kMaxFftM) {
            cls[std::max(ilog2(M), 10)].push_back(j);
            maxM = std::max<int>(maxM, (int)M);
        } else if (n % 4 == 0 && !is_pow2(n / 4) && buffer_of(n / 4) <= kMaxSplitM) {
            cls[kSplitClass].push_back(j);
            maxM = std::max<int>(maxM, (int)buffer_of(n / 4));
        } else {
            return fail(ARKCOS_EUNSUPPORTED, "ring of %d pixels needs an FFT buffer of %lld > %d",
                        n, (long long)M, kMaxFftM);
        }
    }
    for (int l = 0; l <= kSplitClass; ++l) {
        if (cls[l].empty()) continue;
        FftClass c;
        int mx = 0;
        for (int j : cls[l]) {
            const int n = g.n[j];
            if (l == kSplitClass) {
                // buffer of the q-point transforms | the n-point spectrum | the chirp of q
                mx = std::max(mx, (int)buffer_of(n / 4));
                c.tab = std::max(c.tab, n + n / 8 + 1);
                continue;
            }
            const int M = (int)buffer_of(n / 2);
            mx = std::max(mx, M);
            if (4 * n < g.N) c.stage_c = 1;
            // the chirp of h (h/2 + 1, Bluestein rings) and exp(-+ i pi m / n), m <= n/2
            c.tab = std::max(c.tab, (bluestein(n / 2) ? (n / 2) / 2 + 1 : 0) + n / 2 + 1);
        }
        c.split = l == kSplitClass;
        c.M = mx;
        c.logM = ilog2(mx);
        c.threads = std::min(512, std::max(c.split ? 64 : 256, c.M / 16));  // as ring::ClassShape
        c.count = (int)cls[l].size();
        // staging the coefficients of short rings is an optimisation: drop it where it does not
        // fit beside the transform buffer (long kernel grids)
        if (c.stage_c && fft_smem_bytes(c.M, g.N, true, c.tab, c.threads, c.split) > 227 * 1024) c.stage_c = 0;
        const size_t smem = fft_smem_bytes(c.M, g.N, c.stage_c != 0, c.tab, c.threads, c.split);
        if (smem > 227 * 1024)
            return fail(ARKCOS_EUNSUPPORTED, "ring FFT class of buffer %d needs %zu bytes of shared memory",
                        c.M, smem);
        if ((st = upload(&c.reps, cls[l])) != ARKCOS_OK) return st;
        g.fft.push_back(c);
    }
    // stage twiddles tw[h + p] = exp(-2 pi i p / (2h)): the transform passes, the kernel-grid
    // transforms of N points and, at tw[n + m], exp(-i pi m / n) for power-of-two rings
    int twM = 2;
    while (twM < std::max({maxM, 2 * maxpow2, g.N})) twM <<= 1;
    g.twM = twM;
    std::vector<float2> tw(twM);
    tw[0] = make_float2(1.f, 0.f);
    for (int h = 1; h < twM; h <<= 1)
        for (int p = 0; p < h; ++p) {
            const double a = -M_PI * (double)p / (double)h;
            tw[h + p] = make_float2((float)cos(a), (float)sin(a));
        }
    if ((st = upload(&g.d_tw, tw)) != ARKCOS_OK) return st;
    // Bluestein chirp spectra of the representative rings, computed once on the device
    {
        std::vector<int> fboff(g.R, -1);
        int64_t tot = 0;
        for (const auto &c : g.fft) {
            std::vector<int> reps(c.count);
            if (cudaMemcpy(reps.data(), c.reps, c.count * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
                return fail(ARKCOS_ECUDA, "reading the FFT class table");
            for (int j : reps) {
                // the chirp of the ring's pair sequence, or of its quarter for split rings
                const int64_t l = c.split ? g.n[j] / 4 : g.n[j] / 2;
                if (!bluestein(l)) continue;
                fboff[j] = (int)tot;
                tot += buffer_of(l);
            }
        }
        if (tot > (int64_t)0x7fffffff) return fail(ARKCOS_EUNSUPPORTED, "chirp spectra too large");
        if ((st = upload(&g.d_fboff, fboff)) != ARKCOS_OK) return st;
        if (tot > 0) {
            cudaError_t e = cudaMalloc(&g.d_fb, (size_t)tot * sizeof(float2));
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(chirp spectra)");
            for (const auto &c : g.fft) {
                FftFwdArgs a;
                memset(&a, 0, sizeof(a));
                a.rd = g.dev();
                a.tw = g.d_tw;
                a.reps = c.reps;
                a.M = c.M;
                a.split = c.split;
                e = launch_chirp_spectra(a, g.d_fb, c.count, c.threads, 0);
                if (e != cudaSuccess) return cuda_fail(e, "chirp spectra");
            }
            e = cudaStreamSynchronize(0);
            if (e != cudaSuccess) return cuda_fail(e, "chirp spectra");
        }
    }
    std::vector<double> s2(g.N + 1);
    for (int t = 0; t <= g.N; ++t) {
        const double s = sin(M_PI * (double)t / (2.0 * g.N));
        s2[t] = s * s;
    }
    if ((st = upload(&g.d_s2, s2)) != ARKCOS_OK) return st;
    std::vector<float> s2f(s2.begin(), s2.end());
    if ((st = upload(&g.d_s2f, s2f)) != ARKCOS_OK) return st;
    if ((st = build_cos_table(g)) != ARKCOS_OK) return st;
    return ARKCOS_OK;
}

// Last tap k (0..kmax) with squared chord <= umax for samples x_k = pi (2k + f) / N, or -1.
int support_taps(const Grid &g, const std::vector<double> &s2, double A, double B, int f, double umax)
{
    const int N = g.N;
    const int kmax = f ? N / 2 - 1 : N / 2;
    auto u_of = [&](int k) {
        const int t = 2 * k + f;
        return 4.0 * (B * s2[N - t] + A * s2[t]);
    };
    if (u_of(0) > umax) return -1;
    if (u_of(kmax) <= umax) return kmax;
    int lo = 0, hi = kmax;  // u(lo) <= umax < u(hi)
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (u_of(mid) <= umax) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- stage timing
enum Stage { ST_TAPS, ST_FFT_FWD, ST_CONTRACT, ST_FFT_INV, ST_POLE, ST_POLE_ADJ, ST_KNOT_Q,
             ST_KNOT_PROJ, ST_KNOT_POLE, ST_KNOT_REDUCE, ST_COUNT };
const char *kStageNames[ST_COUNT] = {"taps", "fft_fwd", "contract", "fft_inv", "pole", "pole_adj",
                                     "knot_q", "knot_proj", "knot_pole", "knot_reduce"};

struct TimingRec {
    int stage;
    int launches;
    cudaEvent_t a, b;
};
std::mutex g_tmu;
bool g_timing = false;
std::vector<TimingRec> g_recs;

void timing_clear()
{
    for (auto &r : g_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_recs.clear();
}

// RAII scope: records an event pair around one stage when timing is on.
struct StageScope {
    int stage, launches;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    bool on;
    StageScope(int s, int nl, cudaStream_t stream) : stage(s), launches(nl), st(stream)
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        on = g_timing;
        if (on && cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess)
            cudaEventRecord(a, st);
        else
            on = false;
    }
    ~StageScope()
    {
        if (!on) return;
        cudaEventRecord(b, st);
        std::lock_guard<std::mutex> lk(g_tmu);
        g_recs.push_back(TimingRec{stage, launches, a, b});
    }
};

struct Layout {
    size_t taps_off[kMaxKernelsPerLaunch * 8];
    size_t spec = 0, gspec = 0, cbuf = 0, q = 0, xproj = 0, partial = 0, total = 0;
    size_t csum = 0;  // arkcos_convolve_multi with weights: the summed coefficients
    size_t prho = 0, prho_stride = 0;  // tabulated polar coefficients, per kernel
};

// Distinct kernels in call order (nkernels == 1 or nmaps).
bool layout_for(const Grid &g, const arkcos_kernel *ks, int64_t nk, int64_t nmaps, bool backward,
                bool want_knots, Layout &L)
{
    size_t off = 0;
    if (nk > (int64_t)(sizeof(L.taps_off) / sizeof(L.taps_off[0]))) return false;
    for (int64_t k = 0; k < nk; ++k) {
        L.taps_off[k] = off;
        off = align256(off + (size_t)ks[k]->k.ntaps * sizeof(float));
    }
    int maxpolar = 0;
    for (int64_t k = 0; k < nk; ++k) maxpolar = std::max(maxpolar, ks[k]->k.polar_pairs);
    L.prho = off;
    L.prho_stride = align256((size_t)maxpolar * (g.N / 2 + 1) * sizeof(float));
    off = align256(off + (size_t)nk * L.prho_stride);
    const size_t spec_bytes = (size_t)nmaps * g.nrep * (g.N / 2 + 1) * sizeof(float4);
    L.spec = off;
    off = align256(off + spec_bytes);
    if (backward) {
        L.gspec = off;
        off = align256(off + spec_bytes);
    }
    L.cbuf = off;
    off = align256(off + (size_t)nmaps * g.R * (g.N / 2 + 1) * sizeof(float2));
    if (backward && want_knots) {
        int maxpairs = 0, maxT = 0;
        for (int64_t k = 0; k < nk; ++k) {
            maxpairs = std::max(maxpairs, ks[k]->k.npairs);
            maxT = std::max(maxT, ks[k]->k.T);
        }
        L.q = off;
        off = align256(off + (size_t)maxpairs * (g.N / 2 + 1) * sizeof(float));
        L.xproj = off;
        off = align256(off + (size_t)maxpairs * 128 * sizeof(float));
        int maxfft = 0;
        for (int64_t k = 0; k < nk; ++k) maxfft = std::max(maxfft, ks[k]->k.knot_fft_pairs);
        L.partial = off;
        const int64_t rows = knot_proj_blocks() + 8 * nmaps + maxfft;
        off = align256(off + (size_t)rows * maxT * sizeof(double));
    }
    L.total = off;
    return true;
}

// Workspace of arkcos_convolve_multi: the samples and polar tables of the K kernels, the
// spectra of the nmaps inputs, the coefficients of the nmaps x K outputs and, with weights,
// their weighted sums.
void layout_multi(const Grid &g, const arkcos_kernel *ks, int64_t K, int64_t nmaps, bool weighted, Layout &L)
{
    size_t off = 0;
    int maxpolar = 0;
    for (int64_t k = 0; k < K; ++k) {
        L.taps_off[k] = off;
        off = align256(off + (size_t)ks[k]->k.ntaps * sizeof(float));
        maxpolar = std::max(maxpolar, ks[k]->k.polar_pairs);
    }
    const size_t NH = (size_t)(g.N / 2 + 1);
    L.prho = off;
    L.prho_stride = align256((size_t)maxpolar * NH * sizeof(float));
    off = align256(off + (size_t)K * L.prho_stride);
    L.spec = off;
    off = align256(off + (size_t)nmaps * g.nrep * NH * sizeof(float4));
    L.cbuf = off;
    off = align256(off + (size_t)nmaps * K * g.R * NH * sizeof(float2));
    L.csum = off;
    if (weighted) off = align256(off + (size_t)nmaps * g.R * NH * sizeof(float2));
    L.total = off;
}

arkcos_status check_multi(arkcos_grid grid, const arkcos_kernel *ks, int64_t K, int64_t nmaps, uint32_t flags,
                          bool weighted)
{
    if (!grid) return fail(ARKCOS_EINVAL, "grid is NULL");
    if (!ks) return fail(ARKCOS_EINVAL, "kernels is NULL");
    if (nmaps < 1) return fail(ARKCOS_EINVAL, "nmaps must be >= 1 (got %lld)", (long long)nmaps);
    const int64_t kmax = weighted ? kMaxKernelsPerLaunch : kMaxKernelsPerLaunch * 8;
    if (K < 1 || K > kmax)
        return fail(ARKCOS_EINVAL, "nkernels must be in [1, %lld] (got %lld)", (long long)kmax, (long long)K);
    if (nmaps * K > kMaxKernelsPerLaunch * 8)
        return fail(ARKCOS_EUNSUPPORTED, "at most %d outputs (nmaps x nkernels) per call", kMaxKernelsPerLaunch * 8);
    for (int64_t k = 0; k < K; ++k) {
        if (!ks[k]) return fail(ARKCOS_EINVAL, "kernels[%lld] is NULL", (long long)k);
        if (ks[k]->k.g != &grid->g) return fail(ARKCOS_EINVAL, "kernels[%lld] belongs to another grid", (long long)k);
    }
    if (flags & ~(ARKCOS_FLAG_BASIC | ARKCOS_FLAG_NO_SHIFT_FIX | ARKCOS_FLAG_NO_POLE_FIX | ARKCOS_FLAG_3XTF32))
        return fail(ARKCOS_EINVAL, "unknown flag bits 0x%x", flags);
    return ARKCOS_OK;
}

arkcos_status check_common(arkcos_grid grid, const arkcos_kernel *ks, int64_t nk, int64_t nmaps,
                           uint32_t flags)
{
    if (!grid) return fail(ARKCOS_EINVAL, "grid is NULL");
    if (!ks) return fail(ARKCOS_EINVAL, "kernels is NULL");
    if (nmaps < 1) return fail(ARKCOS_EINVAL, "nmaps must be >= 1 (got %lld)", (long long)nmaps);
    if (nk != 1 && nk != nmaps)
        return fail(ARKCOS_EINVAL, "nkernels must be 1 or nmaps (got %lld for %lld maps)",
                    (long long)nk, (long long)nmaps);
    if (nk > 256) return fail(ARKCOS_EUNSUPPORTED, "at most 256 per-map kernels per call");
    for (int64_t k = 0; k < nk; ++k) {
        if (!ks[k]) return fail(ARKCOS_EINVAL, "kernels[%lld] is NULL", (long long)k);
        if (ks[k]->k.g != &grid->g) return fail(ARKCOS_EINVAL, "kernels[%lld] belongs to another grid", (long long)k);
    }
    if (flags & ~(ARKCOS_FLAG_BASIC | ARKCOS_FLAG_NO_SHIFT_FIX | ARKCOS_FLAG_NO_POLE_FIX | ARKCOS_FLAG_3XTF32))
        return fail(ARKCOS_EINVAL, "unknown flag bits 0x%x", flags);
    return ARKCOS_OK;
}

// Map buffers are read and written as pixel pairs (8-byte accesses).
bool misaligned(const void *p) { return ((uintptr_t)p & 7) != 0; }

bool overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + nb && y < x + na;
}

// ---------------------------------------------------------------- pipeline pieces
arkcos_status run_taps(const Grid &g, const arkcos_kernel *ks, int64_t nk, char *ws, const Layout &L,
                       bool shift_fix, cudaStream_t st)
{
    StageScope sc(ST_TAPS, (int)nk, st);
    for (int64_t k = 0; k < nk; ++k) {
        TapArgs a;
        a.kd = ks[k]->k.kd;
        a.s2 = g.d_s2;
        a.s2f = g.d_s2f;
        a.taps = (float *)(ws + L.taps_off[k]);
        a.N = g.N;
        a.shift_fix = shift_fix;
        CK(launch_taps(a, ks[k]->k.npairs, st));
    }
    return ARKCOS_OK;
}

// Launch shape of one call: how many CTAs share the maps of a ring pair in the FFTs (a
// multiplier of the default split), and how many maps one contraction CTA takes (0: all).
struct Shape {
    int fft_split = 1;
    int map_chunk = 0;
    int tc_form = 0;  // tensor-core contraction: 0 default; blocks of 8 rings in groups of two
                      // with 1 / 2: one / two staging buffers; 3: blocks of 16 rings (one CTA
                      // per SM) in groups of two; 4 / 5: blocks of 8 / 16 in groups of four
};

// Shapes chosen by arkcos_autotune, per (grid, kernels, maps, flags).
struct TuneKey {
    const void *grid;
    std::vector<const void *> kernels;
    int64_t nmaps;
    uint32_t flags;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(grid, kernels, nmaps, flags) < std::tie(o.grid, o.kernels, o.nmaps, o.flags);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, Shape> g_tuned;

TuneKey tune_key(arkcos_grid grid, const arkcos_kernel *ks, int64_t nk, int64_t nmaps, uint32_t flags)
{
    TuneKey k{grid, std::vector<const void *>(ks, ks + nk), nmaps, flags};
    return k;
}

Shape tuned_shape(arkcos_grid grid, const arkcos_kernel *ks, int64_t nk, int64_t nmaps, uint32_t flags)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(tune_key(grid, ks, nk, nmaps, flags));
    return it == g_tuned.end() ? Shape{} : it->second;
}

arkcos_status run_fft_fwd(const Grid &g, const float *map, float2 *spec, float4 *spec4, int64_t nmaps,
                          bool weight, bool zero_poles, bool basic, cudaStream_t st, const Shape &sh = Shape{})
{
    StageScope sc(ST_FFT_FWD, (int)g.fft.size(), st);
    // classes from the largest buffers down: each later class starts in the last wave of the
    // one before it (programmatic dependent launch, see launch_fft_fwd)
    for (size_t ci = g.fft.size(); ci-- > 0;) {
        const FftClass &c = g.fft[ci];
        const bool after_prev = ci + 1 < g.fft.size();
        FftFwdArgs a;
        a.rd = g.dev();
        a.tw = g.d_tw;
        a.map = map;
        a.spec = spec;
        a.spec4 = spec4;
        a.ext4 = spec4 != nullptr;
        a.nrep = g.nrep;
        a.NH = g.N / 2 + 1;
        a.basic = basic;
        a.reps = c.reps;
        a.M = c.M;
        a.logM = c.logM;
        a.R = g.R;
        a.N = g.N;
        a.B = (int)nmaps;
        a.mchunk = fft_map_chunk(c.count, (int)nmaps, sh.fft_split);
        a.npix = g.npix;
        a.nspec = g.nspec;
        a.weight = weight;
        a.zero_poles = zero_poles;
        a.tab = c.tab;
        a.split = c.split;
        if (c.split) CK(launch_fft_fwd_split(a, c.count, c.threads, st, after_prev));
        else CK(launch_fft_fwd(a, c.count, c.threads, st, after_prev));
    }
    return ARKCOS_OK;
}

arkcos_status run_fft_inv(const Grid &g, const float2 *cbuf, float *map, int64_t nmaps, bool weight,
                          bool basic, bool skip_poles, cudaStream_t st, const Shape &sh = Shape{})
{
    StageScope sc(ST_FFT_INV, (int)g.fft.size(), st);
    for (size_t ci = g.fft.size(); ci-- > 0;) {  // as run_fft_fwd
        const FftClass &c = g.fft[ci];
        const bool after_prev = ci + 1 < g.fft.size();
        FftInvArgs a;
        a.rd = g.dev();
        a.tw = g.d_tw;
        a.c = cbuf;
        a.map = map;
        a.reps = c.reps;
        a.M = c.M;
        a.logM = c.logM;
        a.R = g.R;
        a.N = g.N;
        a.NH = g.N / 2 + 1;
        a.B = (int)nmaps;
        a.mchunk = fft_map_chunk(c.count, (int)nmaps, sh.fft_split);
        a.npix = g.npix;
        a.weight = weight;
        a.basic = basic;
        a.skip_poles = skip_poles;
        a.stage_c = c.stage_c;
        a.tab = c.tab;
        if (c.split) CK(launch_fft_inv_split(a, c.count, c.threads, st, after_prev));
        else CK(launch_fft_inv(a, c.count, c.threads, st, after_prev));
    }
    return ARKCOS_OK;
}

// Band contraction of nmaps maps (the kernel-grid coefficients of every ring into cbuf).  With
// kdiv > 0 the nmaps maps are virtual: map v uses kernel ks[v % kdiv] (nk == kdiv distinct
// kernels, whose samples and polar tables the layout holds once) and the spectra of input
// v / kdiv of spec4.
arkcos_status run_contract(const Grid &g, const arkcos_kernel *ks, int64_t nk, char *ws,
                           const Layout &L, const float4 *spec4, float2 *cbuf, int64_t nmaps,
                           bool basic, bool shift_fix, bool tf32, cudaStream_t st, const Shape &sh = Shape{},
                           bool polar_table = true, int64_t kdiv = 0)
{
    const int H = contract_ring_block();
    int maxband = 0, maxunion = 0, maxunion2 = 0, maxunion4 = 0;
    int srows[2][2] = {{0, 0}, {0, 0}};  // [16-ring blocks][groups of four]
    for (int64_t k = 0; k < nk; ++k) {
        const Kernel &K = ks[k]->k;
        maxband = std::max(maxband, K.maxband);
        maxunion = std::max(maxunion, K.max_union8);
        maxunion2 = std::max(maxunion2, K.max_union2);
        maxunion4 = std::max(maxunion4, K.max_union4);
        srows[0][0] = std::max(srows[0][0], K.max_stage_rows);
        srows[0][1] = std::max(srows[0][1], K.max_stage_rows_g4);
        srows[1][0] = std::max(srows[1][0], K.max_stage_rows16);
        srows[1][1] = std::max(srows[1][1], K.max_stage_rows16_g4);
    }
    // the register-resident fast path covers bands of up to contract_band_limit() rings
    const bool fast = maxband <= contract_band_limit() && 2 * maxunion * 64 * 16 <= 200 * 1024;
    const bool tc = tf32 && maxunion2 <= contract_band_limit() && contract_tc_smem(8, 2, srows[0][0], 0) <= 200 * 1024;
    // tensor-core form: groups of four rings when their union bands fit the 32 slots, blocks of
    // 16 rings when two staging buffers fit beside one CTA per SM; the autotuner's choice, else
    // the default: for a shared beam groups of four in blocks of 16 where they fit; for per-map
    // beams (every CTA generates its own coefficients for one map) blocks of 8, two CTAs per SM,
    // so that one CTA's generation overlaps the other's contraction
    const bool g4_ok = maxunion4 <= contract_band_limit();
    const bool b16_ok[2] = {contract_tc_nbuf(16, 2, srows[1][0], 0) == 2, contract_tc_nbuf(16, 4, srows[1][1], 0) == 2};
    int tc_rb = 8, tc_gs = g4_ok ? 4 : 2, tc_want = 0;
    const int form = sh.tc_form != 0 ? sh.tc_form : (nk > 1 ? 4 : 5);
    switch (form) {
    case 1: case 2: tc_gs = 2; tc_want = form; break;
    case 3: if (b16_ok[0]) { tc_rb = 16; tc_gs = 2; } break;
    case 4: break;
    default: if (g4_ok && b16_ok[1]) tc_rb = 16; break;
    }
    const int tc_srows = srows[tc_rb == 16][tc_gs == 4];
    int pair_chunk = std::min(H * maxband, 192);
    pair_chunk = std::max(pair_chunk, 1);
    const size_t smem = (size_t)pair_chunk * kModeBlock * sizeof(float);
    const bool per_map = nk > 1 || kdiv > 0;
    auto kof = [&](int64_t v) { return kdiv > 0 ? v % kdiv : v; };  // kernel of map v
    const int64_t groups = per_map ? (nmaps + kMaxKernelsPerLaunch - 1) / kMaxKernelsPerLaunch : 1;
    StageScope sc(ST_CONTRACT, (int)groups, st);
    if (kdiv > 0 && polar_table && (tc || fast)) {
        // several maps share each kernel: its polar coefficient table is computed once
        for (int64_t k0 = 0; k0 < kdiv; k0 += kMaxKernelsPerLaunch) {
            ContractArgs a;
            memset(&a, 0, sizeof(a));
            a.rd = g.dev();
            const int64_t cnt = std::min<int64_t>(kMaxKernelsPerLaunch, kdiv - k0);
            int maxpolar = 0;
            for (int64_t k = 0; k < cnt; ++k) {
                a.kd[k] = ks[k0 + k]->k.kd;
                a.taps[k] = (const float *)(ws + L.taps_off[k0 + k]);
                a.prho[k] = (const float *)(ws + L.prho + (k0 + k) * L.prho_stride);
                maxpolar = std::max(maxpolar, ks[k0 + k]->k.polar_pairs);
            }
            a.R = g.R;
            a.N = g.N;
            a.NH = g.N / 2 + 1;
            a.nrep = g.nrep;
            a.shift_fix = shift_fix;
            if (maxpolar > 0) {
                CK(launch_polar_rho(a, (int)cnt, maxpolar, g.d_tw, g.twM, st));
                ++sc.launches;
            }
        }
    }
    for (int64_t gi = 0; gi < groups; ++gi) {
        ContractArgs a;
        memset(&a, 0, sizeof(a));
        a.rd = g.dev();
        const int64_t base = per_map ? gi * kMaxKernelsPerLaunch : 0;
        const int64_t cnt = per_map ? std::min<int64_t>(kMaxKernelsPerLaunch, nmaps - base) : 1;
        int maxpolar = 0;
        for (int64_t k = 0; k < cnt; ++k) {
            const int64_t kk = kof(base + k);
            a.kd[k] = ks[kk]->k.kd;
            a.taps[k] = (const float *)(ws + L.taps_off[kk]);
            a.prho[k] = (const float *)(ws + L.prho + kk * L.prho_stride);
            maxpolar = std::max(maxpolar, ks[kk]->k.polar_pairs);
        }
        a.spec4 = spec4;
        a.c = cbuf;
        a.R = g.R;
        a.N = g.N;
        a.NH = g.N / 2 + 1;
        a.nrep = g.nrep;
        a.B = (int)(per_map ? base + cnt : nmaps);
        a.nspec = g.nspec;
        const int64_t chunk = per_map ? 1 : (sh.map_chunk > 0 ? std::min<int64_t>(sh.map_chunk, nmaps) : nmaps);
        a.maps_per_chunk = (int)chunk;
        a.per_map = per_map;
        a.map_base = (int)base;
        a.basic = basic;
        a.shift_fix = shift_fix;
        a.pair_chunk = pair_chunk;
        a.withhold_mma = test_withhold_mma();
        // chunks cover maps [base, base + cnt) for per-map kernels, all maps otherwise
        const int nchunks = per_map ? (int)cnt : (int)((nmaps + chunk - 1) / chunk);
        if (per_map) {
            // blockIdx.z indexes maps relative to the launch; shift the spectra and outputs
            if (kdiv > 0) {
                a.vbase = (int)base;
                a.vdiv = (int)kdiv;
            } else {
                a.spec4 = spec4 + base * (int64_t)g.nrep * (g.N / 2 + 1);
            }
            a.c = cbuf + base * (int64_t)g.R * (g.N / 2 + 1);
            a.B = (int)cnt;
            a.map_base = 0;
        }
        if ((tc || fast) && polar_table && kdiv == 0 && maxpolar > 0) {
            CK(launch_polar_rho(a, (int)cnt, maxpolar, g.d_tw, g.twM, st));
            ++sc.launches;
        }
        if (tc) CK(launch_contract_tc(a, tc_rb, tc_gs, nchunks, g.d_ctab, g.nkc_tab, tc_srows, tc_want, st));
        else if (fast) CK(launch_contract_band(a, nchunks, maxunion, st));
        else CK(launch_contract(a, nchunks, smem, st));
    }
    return ARKCOS_OK;
}

PoleArgs pole_args(const Grid &g, const arkcos_kernel *ks, int64_t base, int64_t cnt, bool per_map,
                   const float *in, float *out)
{
    PoleArgs a;
    memset(&a, 0, sizeof(a));
    a.rd = g.dev();
    for (int64_t k = 0; k < (per_map ? cnt : 1); ++k) a.kd[k] = ks[base + k]->k.kd;
    a.map = in + base * g.npix;
    a.out = out + base * g.npix;
    a.R = g.R;
    a.B = (int)cnt;
    a.per_map = per_map;
    a.map_base = 0;
    a.npix = g.npix;
    return a;
}

// ---------------------------------------------------------------- host-buffer pipeline
// Device buffers of arkcos_convolve_host: two input and two output chunks, then the forward
// workspace of the largest chunk.
struct HostLayout {
    int64_t chunk = 0;
    size_t map_bytes = 0, in[2] = {0, 0}, out[2] = {0, 0}, conv = 0, conv_bytes = 0, total = 0;
};

arkcos_status host_layout(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels, int64_t nmaps,
                          int64_t maps_per_chunk, uint32_t flags, HostLayout &H)
{
    if (maps_per_chunk < 1) return fail(ARKCOS_EINVAL, "maps_per_chunk %lld < 1", (long long)maps_per_chunk);
    const Grid &g = grid->g;
    const bool per_map = nkernels > 1;
    H.chunk = std::min(maps_per_chunk, nmaps);
    H.map_bytes = align256((size_t)H.chunk * g.npix * sizeof(float));
    size_t off = 0;
    for (int q = 0; q < 2; ++q) {
        H.in[q] = off;
        off += H.map_bytes;
        H.out[q] = off;
        off += H.map_bytes;
    }
    H.conv = off;
    H.conv_bytes = 0;
    for (int64_t c0 = 0; c0 < nmaps; c0 += H.chunk) {
        const int64_t cnt = std::min(H.chunk, nmaps - c0);
        size_t b = 0;
        arkcos_status st = arkcos_workspace_size(grid, kernels + (per_map ? c0 : 0), per_map ? cnt : 1, cnt,
                                                 flags, 0, &b);
        if (st != ARKCOS_OK) return st;
        H.conv_bytes = std::max(H.conv_bytes, b);
        if (!per_map) break;  // every chunk but a shorter last one needs the same
    }
    H.total = off + align256(H.conv_bytes);
    return ARKCOS_OK;
}

}  // namespace

int arkcos::device_sms()
{
    static std::mutex mu;
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    std::lock_guard<std::mutex> lk(mu);
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 152;
        cache[dev] = n;
    }
    return cache[dev];
}

int arkcos::test_withhold_mma()
{
    const char *v = getenv("ARKCOS_TEST_WITHHOLD_MMA");
    return (v && atoi(v) != 0) ? 1 : 0;
}

void arkcos::set_last_error(const char *msg)
{
    snprintf(g_err, sizeof(g_err), "%s", msg);
}

// ====================================================================== C ABI
extern "C" {

const char *arkcos_last_error(void) { return g_err; }
const char *arkcos_version(void) { return "arkcos-gb300 0.1 (sm_103a)"; }

arkcos_status arkcos_create_grid_healpix(int64_t nside, arkcos_grid *out)
{
    g_err[0] = 0;
    if (!out) return fail(ARKCOS_EINVAL, "out is NULL");
    *out = nullptr;
    if (nside < 1 || nside > 8192) return fail(ARKCOS_EINVAL, "nside %lld out of range [1, 8192]", (long long)nside);
    arkcos_grid h = new (std::nothrow) arkcos_grid_s;
    if (!h) return fail(ARKCOS_ENOMEM, "host allocation failed");
    Grid &g = h->g;
    g.kind = 0;
    g.nside = nside;
    g.N = (int)(4 * nside);
    const int64_t R = 4 * nside - 1;
    const double ns = (double)nside, w = 4.0 * M_PI / (12.0 * ns * ns);
    for (int64_t r = 1; r <= R; ++r) {
        double th;
        int n, hs;
        if (r < nside) {  // north polar cap: z = 1 - r^2 / (3 nside^2)
            n = (int)(4 * r);
            th = 2.0 * asin((double)r / (sqrt(6.0) * ns));
            hs = 1;
        } else if (r <= 3 * nside) {  // equatorial belt: z = 4/3 - 2r / (3 nside)
            n = (int)(4 * nside);
            th = acos(4.0 / 3.0 - 2.0 * (double)r / (3.0 * ns));
            hs = ((r - nside) % 2 == 0) ? 1 : 0;
        } else {  // south polar cap, mirror of the north
            const int64_t i = 4 * nside - r;
            n = (int)(4 * i);
            th = M_PI - 2.0 * asin((double)i / (sqrt(6.0) * ns));
            hs = 1;
        }
        g.theta.push_back(th);
        g.n.push_back(n);
        g.hs.push_back(hs);
        g.wgt.push_back(w);
    }
    arkcos_status st = finish_grid(g);
    if (st != ARKCOS_OK) {
        free_grid_dev(g);
        delete h;
        return st;
    }
    *out = h;
    return ARKCOS_OK;
}

arkcos_status arkcos_create_grid_ecp(int64_t ntheta, int64_t nphi, arkcos_grid *out)
{
    g_err[0] = 0;
    if (!out) return fail(ARKCOS_EINVAL, "out is NULL");
    *out = nullptr;
    if (ntheta < 1 || ntheta > 65536 || nphi < 2 || nphi > 65536 || (nphi % 2))
        return fail(ARKCOS_EINVAL, "ECP grid %lld x %lld invalid (ntheta >= 1, even nphi >= 2, both <= 65536)",
                    (long long)ntheta, (long long)nphi);
    arkcos_grid h = new (std::nothrow) arkcos_grid_s;
    if (!h) return fail(ARKCOS_ENOMEM, "host allocation failed");
    Grid &g = h->g;
    g.kind = 1;
    g.ntheta = ntheta;
    g.nphi = nphi;
    g.N = (int)nphi;
    for (int64_t r = 0; r < ntheta; ++r) {
        const double th = (r + 0.5) * M_PI / (double)ntheta;
        // Fejer's first rule (Waldvogel 2006): w = (2/n)[1 - 2 sum_{k<=n/2} cos(2k th)/(4k^2-1)]
        double s = 0.0;
        for (int64_t k = 1; k <= ntheta / 2; ++k) s += cos(2.0 * k * th) / (4.0 * (double)k * k - 1.0);
        g.theta.push_back(th);
        g.n.push_back((int)nphi);
        g.hs.push_back(0);
        g.wgt.push_back((2.0 / (double)ntheta) * (1.0 - 2.0 * s) * (2.0 * M_PI / (double)nphi));
    }
    arkcos_status st = finish_grid(g);
    if (st != ARKCOS_OK) {
        free_grid_dev(g);
        delete h;
        return st;
    }
    *out = h;
    return ARKCOS_OK;
}

arkcos_status arkcos_destroy_grid(arkcos_grid grid)
{
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto it = g_tuned.begin(); it != g_tuned.end();)
            it = it->first.grid == grid ? g_tuned.erase(it) : std::next(it);
    }
    g_err[0] = 0;
    if (!grid) return ARKCOS_OK;
    if (grid->g.live_kernels > 0)
        return fail(ARKCOS_EINVAL, "grid still has %d live kernels", grid->g.live_kernels);
    free_grid_dev(grid->g);
    delete grid;
    return ARKCOS_OK;
}

arkcos_status arkcos_grid_info(arkcos_grid grid, int64_t *nrings, int64_t *npix, int64_t *nlon)
{
    g_err[0] = 0;
    if (!grid) return fail(ARKCOS_EINVAL, "grid is NULL");
    if (nrings) *nrings = grid->g.R;
    if (npix) *npix = grid->g.npix;
    if (nlon) *nlon = grid->g.N;
    return ARKCOS_OK;
}

arkcos_status arkcos_set_kernel(arkcos_grid grid, const double *knots, int64_t nknots, double gamma_max,
                                uint32_t flags, arkcos_kernel *out)
{
    g_err[0] = 0;
    if (!out) return fail(ARKCOS_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !knots) return fail(ARKCOS_EINVAL, "grid or knots is NULL");
    if (nknots < 2 || nknots > 4096) return fail(ARKCOS_EINVAL, "nknots %lld not in [2, 4096]", (long long)nknots);
    if (!(gamma_max > 0.0) || gamma_max > M_PI / 2)
        return fail(ARKCOS_EINVAL, "gamma_max %g not in (0, pi/2]", gamma_max);
    if (flags != 0) return fail(ARKCOS_EINVAL, "set_kernel flags are reserved (pass 0)");
    for (int64_t t = 0; t < nknots; ++t)
        if (!isfinite(knots[t])) return fail(ARKCOS_EINVAL, "knot %lld is not finite", (long long)t);
    const Grid &g = grid->g;
    arkcos_kernel h = new (std::nothrow) arkcos_kernel_s;
    if (!h) return fail(ARKCOS_ENOMEM, "host allocation failed");
    Kernel &K = h->k;
    K.g = &grid->g;
    K.T = (int)nknots;
    K.gmax = gamma_max;
    std::vector<double> ut(nknots), kn(knots, knots + nknots);
    for (int64_t t = 0; t < nknots; ++t) {
        const double s = sin(0.5 * gamma_max * (double)t / (double)(nknots - 1));
        ut[t] = 4.0 * s * s;
    }
    K.umax = ut[nknots - 1];
    std::vector<double> s2(g.N + 1);
    for (int t = 0; t <= g.N; ++t) {
        const double s = sin(M_PI * (double)t / (2.0 * g.N));
        s2[t] = s * s;
    }
    // band tables for the representative output rings
    std::vector<int> pstart, jlo, jhi, S0, S1, fl, toff;
    std::vector<double> A, B;
    int j0 = 0;
    int64_t taps = 0;
    for (int i = 0; i < g.nrep; ++i) {
        while (j0 < g.R && g.theta[j0] < g.theta[i] - gamma_max) ++j0;
        int j1 = j0;
        while (j1 + 1 < g.R && g.theta[j1 + 1] <= g.theta[i] + gamma_max) ++j1;
        pstart.push_back((int)S0.size());
        jlo.push_back(j0);
        jhi.push_back(j1);
        K.maxband = std::max(K.maxband, j1 - j0 + 1);
        for (int j = j0; j <= j1; ++j) {
            const double sp = sin(0.5 * (g.theta[i] + g.theta[j]));
            const double sm = sin(0.5 * (g.theta[i] - g.theta[j]));
            const double a = sp * sp, b = sm * sm;
            const int f = (g.n[i] == g.n[j] && g.hs[i] != g.hs[j]) ? 1 : 0;
            const int s0 = support_taps(g, s2, a, b, 0, K.umax);
            const int s1 = support_taps(g, s2, a, b, 1, K.umax);
            A.push_back(a);
            B.push_back(b);
            S0.push_back(s0);
            S1.push_back(s1);
            fl.push_back(f);
            toff.push_back((int)taps);
            const int slots = (std::max(s0, s1) + 1 + 3) & ~3;
            taps += slots;
            K.maxS = std::max(K.maxS, std::max(s0, s1));
            K.sum_taps_fix += (f ? s1 : s0) + 1;
        }
    }
    pstart.push_back((int)S0.size());
    toff.push_back((int)taps);
    K.pole_band = jhi[0] - jlo[0] + 1;
    for (int r0 = 0; r0 < g.nrep; r0 += 8) {
        const int r1 = std::min(g.nrep, r0 + 8) - 1;
        K.max_union8 = std::max(K.max_union8, jhi[r1] - jlo[r0] + 1);
        for (int q = r0; q <= r1; q += 2) {
            K.max_union2 = std::max(K.max_union2, jhi[std::min(q + 1, r1)] - jlo[q] + 1);
            K.max_stage_rows = std::max(K.max_stage_rows, jlo[q] - jlo[r0] + 32);
        }
        K.max_stage_rows = std::max(K.max_stage_rows, jhi[r1] - jlo[r0] + 1);
    }
    // the same for tensor-core blocks of 8 and 16 rings with groups of two or four rings
    for (int rb : {8, 16})
        for (int gs : {2, 4})
            for (int r0 = 0; r0 < g.nrep; r0 += rb) {
                const int r1 = std::min(g.nrep, r0 + rb) - 1;
                int &rows = rb == 8 ? (gs == 2 ? K.max_stage_rows : K.max_stage_rows_g4)
                                    : (gs == 2 ? K.max_stage_rows16 : K.max_stage_rows16_g4);
                for (int q = r0; q <= r1; q += gs) {
                    rows = std::max(rows, jlo[q] - jlo[r0] + 32);
                    if (gs == 4) K.max_union4 = std::max(K.max_union4, jhi[std::min(q + 3, r1)] - jlo[q] + 1);
                }
                rows = std::max(rows, jhi[r1] - jlo[r0] + 1);
            }
    if (taps > (int64_t)0x7fffffff) {
        delete h;
        return fail(ARKCOS_EUNSUPPORTED, "kernel support too large (%lld samples)", (long long)taps);
    }
    K.npairs = (int)S0.size();
    K.ntaps = taps;
    // the leading ring blocks (next to the poles) whose pairs have more samples than the
    // tensor-core cosine table covers get their coefficients tabulated per call, when they
    // are few enough; the tabulated rings are whole blocks of 16, so that they also cover
    // the tensor-core blocks of 16 rings
    {
        const int kcap = g.nkc_tab * 32;
        int last = -1;
        for (int r0 = 0; r0 < g.nrep; r0 += 16) {
            int mx = 0;
            for (int p = pstart[r0]; p < pstart[std::min(g.nrep, r0 + 16)]; ++p)
                mx = std::max(mx, std::max(S0[p], S1[p]) + 1);
            if (mx <= kcap) break;
            last = r0 / 16;
        }
        const int pp = last < 0 ? 0 : pstart[std::min(g.nrep, 16 * (last + 1))];
        K.polar_pairs = pp <= kMaxPolarPairs ? pp : 0;
    }
    // tensor-core columns of each block of 8 representative rings: rings go in groups of two
    // (first table) or four (second table), column 32 l + u holds the pair of ring l with
    // input ring jlo(first ring of l's group) + u
    const int nblk8 = (g.nrep + 7) / 8;
    std::vector<int> coltab((size_t)2 * nblk8 * 256 * 4);
    for (int y = 0; y < 2 * nblk8; ++y) {
        const int gmask = y < nblk8 ? ~1 : ~3;
        const int r0 = 8 * (y % nblk8), nr = std::min(8, g.nrep - r0);
        for (int c = 0; c < 256; ++c) {
            const int l = c / 32, u = c % 32;
            int *e = &coltab[((size_t)y * 256 + c) * 4];
            e[0] = -1;
            e[1] = 0;
            e[2] = -1;
            e[3] = -2;
            if (l >= nr) continue;
            const int sl = u + jlo[r0 + (l & gmask)] - jlo[r0 + l];
            if (sl < 0 || sl > jhi[r0 + l] - jlo[r0 + l]) continue;
            const int p = pstart[r0 + l] + sl;
            e[0] = p;
            e[1] = toff[p];
            e[2] = S0[p];
            e[3] = 2 * S1[p] + fl[p];
        }
    }
    // the polar pairs' knot-gradient projection runs by FFT where the kernel grid allows;
    // the work units of the direct projection: (pair, first of knot_proj_taps() taps)
    K.knot_fft_pairs = (K.polar_pairs > 0 && is_pow2(g.N) && g.N >= 1024 && g.N <= 16384 && g.N <= g.twM)
                           ? K.polar_pairs : 0;
    {
        int mx = 0;
        for (int p = K.knot_fft_pairs; p < K.npairs; ++p) mx = std::max(mx, std::max(S0[p], S1[p]) + 1);
        K.proj_tc_ok = mx <= 128;
    }
    std::vector<int> ufix, unofix;
    const int ut_step = knot_proj_taps();
    for (int p = K.knot_fft_pairs; p < K.npairs; ++p) {
        const int nf = (fl[p] ? S1[p] : S0[p]) + 1, nn = S0[p] + 1;
        for (int k = 0; k < nf; k += ut_step) ufix.insert(ufix.end(), {p, k});
        for (int k = 0; k < nn; k += ut_step) unofix.insert(unofix.end(), {p, k});
    }
    // one device block holding every table
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_ps = take(pstart.size() * 4), o_jl = take(jlo.size() * 4), o_jh = take(jhi.size() * 4);
    const size_t o_s0 = take(S0.size() * 4), o_s1 = take(S1.size() * 4), o_fl = take(fl.size() * 4);
    const size_t o_to = take(toff.size() * 4), o_a = take(A.size() * 8), o_b = take(B.size() * 8);
    const size_t o_kn = take(kn.size() * 8), o_ut = take(ut.size() * 8);
    const size_t o_uf = take(ufix.size() * 4), o_un = take(unofix.size() * 4);
    const size_t o_ct = take(coltab.size() * 4);
    std::vector<char> host(off);
    memcpy(host.data() + o_ct, coltab.data(), coltab.size() * 4);
    memcpy(host.data() + o_uf, ufix.data(), ufix.size() * 4);
    memcpy(host.data() + o_un, unofix.data(), unofix.size() * 4);
    memcpy(host.data() + o_ps, pstart.data(), pstart.size() * 4);
    memcpy(host.data() + o_jl, jlo.data(), jlo.size() * 4);
    memcpy(host.data() + o_jh, jhi.data(), jhi.size() * 4);
    memcpy(host.data() + o_s0, S0.data(), S0.size() * 4);
    memcpy(host.data() + o_s1, S1.data(), S1.size() * 4);
    memcpy(host.data() + o_fl, fl.data(), fl.size() * 4);
    memcpy(host.data() + o_to, toff.data(), toff.size() * 4);
    memcpy(host.data() + o_a, A.data(), A.size() * 8);
    memcpy(host.data() + o_b, B.data(), B.size() * 8);
    memcpy(host.data() + o_kn, kn.data(), kn.size() * 8);
    memcpy(host.data() + o_ut, ut.data(), ut.size() * 8);
    cudaError_t e = cudaMalloc(&K.dmem, off);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaMalloc(kernel tables)");
    }
    e = cudaMemcpy(K.dmem, host.data(), off, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(K.dmem);
        delete h;
        return cuda_fail(e, "cudaMemcpy(kernel tables)");
    }
    char *d = (char *)K.dmem;
    K.kd.pstart = (const int *)(d + o_ps);
    K.kd.jlo = (const int *)(d + o_jl);
    K.kd.jhi = (const int *)(d + o_jh);
    K.kd.S0 = (const int *)(d + o_s0);
    K.kd.S1 = (const int *)(d + o_s1);
    K.kd.fl = (const int *)(d + o_fl);
    K.kd.toff = (const int *)(d + o_to);
    K.kd.A = (const double *)(d + o_a);
    K.kd.B = (const double *)(d + o_b);
    K.kd.knots = (const double *)(d + o_kn);
    K.kd.ut = (const double *)(d + o_ut);
    K.kd.coltab = (const int4 *)(d + o_ct);
    K.kd.coltab4 = K.kd.coltab + (size_t)nblk8 * 256;
    K.kd.unit_fix = (const int2 *)(d + o_uf);
    K.kd.unit_nofix = (const int2 *)(d + o_un);
    K.kd.nunit_fix = (int)(ufix.size() / 2);
    K.kd.nunit_nofix = (int)(unofix.size() / 2);
    K.kd.T = K.T;
    K.kd.npairs = K.npairs;
    K.kd.polar_pairs = K.polar_pairs;
    K.kd.umax = K.umax;
    K.kd.gscale = (double)(K.T - 1) / gamma_max;
    grid->g.live_kernels++;
    *out = h;
    return ARKCOS_OK;
}

arkcos_status arkcos_kernel_update_knots(arkcos_kernel kernel, const double *knots, int on_device, void *stream)
{
    g_err[0] = 0;
    if (!kernel || !knots) return fail(ARKCOS_EINVAL, "kernel or knots is NULL");
    double *dst = const_cast<double *>(kernel->k.kd.knots);
    const size_t bytes = (size_t)kernel->k.T * sizeof(double);
    if (on_device) {
        CK(cudaMemcpyAsync(dst, knots, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    } else {
        for (int t = 0; t < kernel->k.T; ++t)
            if (!isfinite(knots[t])) return fail(ARKCOS_EINVAL, "knot %d is not finite", t);
        CK(cudaMemcpy(dst, knots, bytes, cudaMemcpyHostToDevice));
    }
    return ARKCOS_OK;
}

arkcos_status arkcos_destroy_kernel(arkcos_kernel kernel)
{
    g_err[0] = 0;
    if (!kernel) return ARKCOS_OK;
    cudaError_t e = cudaFree(kernel->k.dmem);
    kernel->k.g->live_kernels--;
    delete kernel;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFree(kernel tables)");
    return ARKCOS_OK;
}

arkcos_status arkcos_workspace_size(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                                    int64_t nmaps, uint32_t flags, int backward, size_t *bytes)
{
    g_err[0] = 0;
    if (!bytes) return fail(ARKCOS_EINVAL, "bytes is NULL");
    arkcos_status st = check_common(grid, kernels, nkernels, nmaps, flags);
    if (st != ARKCOS_OK) return st;
    Layout L;
    if (!layout_for(grid->g, kernels, nkernels, nmaps, backward != 0, true, L))
        return fail(ARKCOS_EINVAL, "too many kernels");
    *bytes = L.total;
    return ARKCOS_OK;
}

// The forward convolution; with setup == false the beam's samples and polar coefficient table
// are taken as already in the workspace (written by an earlier call with the same grid, kernel,
// flags and workspace on the same stream).
arkcos_status convolve_impl(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels, const float *map_in,
                            float *map_out, int64_t nmaps, void *workspace, size_t ws_bytes, void *stream,
                            uint32_t flags, bool setup)
{
    g_err[0] = 0;
    arkcos_status st = check_common(grid, kernels, nkernels, nmaps, flags);
    if (st != ARKCOS_OK) return st;
    if (!map_in || !map_out) return fail(ARKCOS_EINVAL, "map_in or map_out is NULL");
    if (misaligned(map_in) || misaligned(map_out)) return fail(ARKCOS_EINVAL, "map buffers must be 8-byte aligned");
    const Grid &g = grid->g;
    const size_t mbytes = (size_t)nmaps * g.npix * sizeof(float);
    if (overlap(map_in, mbytes, map_out, mbytes)) return fail(ARKCOS_EINVAL, "map_in and map_out overlap");
    Layout L;
    if (!layout_for(g, kernels, nkernels, nmaps, false, false, L)) return fail(ARKCOS_EINVAL, "too many kernels");
    if (!workspace || ((uintptr_t)workspace & 255))
        return fail(ARKCOS_EWORKSPACE, "workspace is NULL or not 256-byte aligned");
    if (ws_bytes < L.total)
        return fail(ARKCOS_EWORKSPACE, "workspace of %zu bytes < %zu required", ws_bytes, L.total);
    cudaStream_t s = (cudaStream_t)stream;
    const bool basic = flags & ARKCOS_FLAG_BASIC;
    const bool shift_fix = !(flags & ARKCOS_FLAG_NO_SHIFT_FIX);
    const bool pole_fix = g.kind == 0 && !(flags & ARKCOS_FLAG_NO_POLE_FIX);
    char *ws = (char *)workspace;
    float4 *spec = (float4 *)(ws + L.spec);
    float2 *cbuf = (float2 *)(ws + L.cbuf);
    if (setup && (st = run_taps(g, kernels, nkernels, ws, L, shift_fix, s)) != ARKCOS_OK) return st;
    const Shape sh = tuned_shape(grid, kernels, nkernels, nmaps, flags);
    if ((st = run_fft_fwd(g, map_in, nullptr, spec, nmaps, true, false, basic, s, sh)) != ARKCOS_OK) return st;
    if ((st = run_contract(g, kernels, nkernels, ws, L, spec, cbuf, nmaps, basic, shift_fix,
                           (flags & ARKCOS_FLAG_3XTF32) != 0, s, sh, setup)) != ARKCOS_OK)
        return st;
    if ((st = run_fft_inv(g, cbuf, map_out, nmaps, false, basic, pole_fix, s, sh)) != ARKCOS_OK) return st;
    if (pole_fix) {
        const bool per_map = nkernels > 1;
        StageScope sc(ST_POLE, (int)((nmaps + kMaxKernelsPerLaunch - 1) / kMaxKernelsPerLaunch), s);
        for (int64_t base = 0; base < nmaps; base += kMaxKernelsPerLaunch) {
            const int64_t cnt = std::min<int64_t>(kMaxKernelsPerLaunch, nmaps - base);
            PoleArgs a = pole_args(g, kernels, per_map ? base : 0, cnt, per_map, map_in, map_out);
            a.map = map_in + base * g.npix;
            a.out = map_out + base * g.npix;
            CK(launch_pole_fwd(a, s));
        }
    }
    return ARKCOS_OK;
}

arkcos_status arkcos_convolve(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                              const float *map_in, float *map_out, int64_t nmaps, void *workspace,
                              size_t ws_bytes, void *stream, uint32_t flags)
{
    return convolve_impl(grid, kernels, nkernels, map_in, map_out, nmaps, workspace, ws_bytes, stream, flags, true);
}

arkcos_status arkcos_multi_workspace_size(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                                          int64_t nmaps, int weighted, uint32_t flags, size_t *bytes)
{
    g_err[0] = 0;
    if (!bytes) return fail(ARKCOS_EINVAL, "bytes is NULL");
    arkcos_status st = check_multi(grid, kernels, nkernels, nmaps, flags, weighted != 0);
    if (st != ARKCOS_OK) return st;
    Layout L;
    layout_multi(grid->g, kernels, nkernels, nmaps, weighted != 0, L);
    *bytes = L.total;
    return ARKCOS_OK;
}

arkcos_status arkcos_convolve_multi(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                                    const double *weights, const float *map_in, float *map_out, int64_t nmaps,
                                    void *workspace, size_t ws_bytes, void *stream, uint32_t flags)
{
    g_err[0] = 0;
    const bool weighted = weights != nullptr;
    arkcos_status st = check_multi(grid, kernels, nkernels, nmaps, flags, weighted);
    if (st != ARKCOS_OK) return st;
    if (!map_in || !map_out) return fail(ARKCOS_EINVAL, "map_in or map_out is NULL");
    if (misaligned(map_in) || misaligned(map_out)) return fail(ARKCOS_EINVAL, "map buffers must be 8-byte aligned");
    const Grid &g = grid->g;
    const int64_t K = nkernels, V = nmaps * K;  // outputs before the weighted sum
    const size_t ibytes = (size_t)nmaps * g.npix * sizeof(float);
    const size_t obytes = (size_t)(weighted ? nmaps : V) * g.npix * sizeof(float);
    if (overlap(map_in, ibytes, map_out, obytes)) return fail(ARKCOS_EINVAL, "map_in and map_out overlap");
    Layout L;
    layout_multi(g, kernels, K, nmaps, weighted, L);
    if (!workspace || ((uintptr_t)workspace & 255))
        return fail(ARKCOS_EWORKSPACE, "workspace is NULL or not 256-byte aligned");
    if (ws_bytes < L.total)
        return fail(ARKCOS_EWORKSPACE, "workspace of %zu bytes < %zu required", ws_bytes, L.total);
    cudaStream_t s = (cudaStream_t)stream;
    const bool basic = flags & ARKCOS_FLAG_BASIC;
    const bool shift_fix = !(flags & ARKCOS_FLAG_NO_SHIFT_FIX);
    const bool pole_fix = g.kind == 0 && !(flags & ARKCOS_FLAG_NO_POLE_FIX);
    const bool tf32 = (flags & ARKCOS_FLAG_3XTF32) != 0;
    char *ws = (char *)workspace;
    float4 *spec = (float4 *)(ws + L.spec);
    float2 *cbuf = (float2 *)(ws + L.cbuf);
    if ((st = run_taps(g, kernels, K, ws, L, shift_fix, s)) != ARKCOS_OK) return st;
    // one ring analysis per input map, shared by every kernel
    if ((st = run_fft_fwd(g, map_in, nullptr, spec, nmaps, true, false, basic, s)) != ARKCOS_OK) return st;
    if (K == 1) {
        if ((st = run_contract(g, kernels, 1, ws, L, spec, cbuf, nmaps, basic, shift_fix, tf32, s)) != ARKCOS_OK)
            return st;
    } else if ((st = run_contract(g, kernels, K, ws, L, spec, cbuf, V, basic, shift_fix, tf32, s, Shape{}, true,
                                  K)) != ARKCOS_OK) {
        return st;
    }
    const int64_t per_map = (int64_t)g.R * (g.N / 2 + 1);
    if (weighted) {
        float2 *csum = (float2 *)(ws + L.csum);
        {
            StageScope sc(ST_CONTRACT, 1, s);
            CK(launch_weighted_sum(cbuf, csum, nmaps, (int)K, weights, per_map, s));
        }
        if ((st = run_fft_inv(g, csum, map_out, nmaps, false, basic, pole_fix, s)) != ARKCOS_OK) return st;
        if (pole_fix) {
            StageScope sc(ST_POLE, 1, s);
            PoleArgs a;
            memset(&a, 0, sizeof(a));
            a.rd = g.dev();
            for (int64_t k = 0; k < K; ++k) {
                a.kd[k] = kernels[k]->k.kd;
                a.wsum[k] = weights[k];
            }
            a.nsum = (int)K;
            a.map = map_in;
            a.out = map_out;
            a.R = g.R;
            a.B = (int)nmaps;
            a.npix = g.npix;
            CK(launch_pole_fwd(a, s));
        }
        return ARKCOS_OK;
    }
    if ((st = run_fft_inv(g, cbuf, map_out, V, false, basic, pole_fix, s)) != ARKCOS_OK) return st;
    if (pole_fix) {
        StageScope sc(ST_POLE, (int)((V + kMaxKernelsPerLaunch - 1) / kMaxKernelsPerLaunch), s);
        for (int64_t base = 0; base < V; base += kMaxKernelsPerLaunch) {
            const int64_t cnt = std::min<int64_t>(kMaxKernelsPerLaunch, V - base);
            PoleArgs a;
            memset(&a, 0, sizeof(a));
            a.rd = g.dev();
            for (int64_t t = 0; t < cnt; ++t) a.kd[t] = kernels[(base + t) % K]->k.kd;
            a.out = map_out + base * g.npix;
            a.R = g.R;
            a.B = (int)cnt;
            a.per_map = 1;
            a.npix = g.npix;
            if (K > 1) {  // output v of the call reads input v / K
                a.map = map_in;
                a.vbase = (int)base;
                a.vdiv = (int)K;
            } else {
                a.map = map_in + base * g.npix;
            }
            CK(launch_pole_fwd(a, s));
        }
    }
    return ARKCOS_OK;
}

arkcos_status arkcos_autotune(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                              const float *map_in, float *map_out, int64_t nmaps, void *workspace,
                              size_t ws_bytes, void *stream, uint32_t flags, int64_t *out)
{
    g_err[0] = 0;
    arkcos_status st = check_common(grid, kernels, nkernels, nmaps, flags);
    if (st != ARKCOS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const TuneKey key = tune_key(grid, kernels, nkernels, nmaps, flags);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned.erase(key);
    }
    // candidate shapes: FFT split multipliers x contraction map chunks (shared beams only)
    std::vector<Shape> cand;
    std::vector<int> chunks{0};
    if (nkernels == 1)
        for (int d : {2, 4})
            if (nmaps / d >= 1 && (nmaps + d - 1) / d < nmaps) chunks.push_back((int)((nmaps + d - 1) / d));
    const bool tf32 = (flags & ARKCOS_FLAG_3XTF32) != 0;
    for (int fs : {1, 2, 4, 8, 16})
        for (int ch : chunks)
            for (int tf : {0, 1, 2, 3, 4, 5})
                if (tf32 || tf == 0) cand.push_back(Shape{fs, ch, tf});
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    Shape best_sh;
    for (const Shape &sh : cand) {
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[key] = sh;
        }
        float ms = 1e30f;
        for (int rep = 0; rep < 3 && st == ARKCOS_OK; ++rep) {
            cudaEventRecord(e0, s);
            st = arkcos_convolve(grid, kernels, nkernels, map_in, map_out, nmaps, workspace, ws_bytes, stream, flags);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = ARKCOS_ECUDA;
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) ms = std::min(ms, t);  // the first run of a shape warms it up
        }
        if (st != ARKCOS_OK) break;
        if (ms < best) {
            best = ms;
            best_sh = sh;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (st == ARKCOS_OK) g_tuned[key] = best_sh;
        else g_tuned.erase(key);
    }
    if (st != ARKCOS_OK) return st;
    if (out) {
        out[0] = best_sh.fft_split;
        out[1] = best_sh.map_chunk ? best_sh.map_chunk : nmaps;
        out[2] = (int64_t)cand.size();
        out[3] = (int64_t)(best * 1000.0f);
        out[4] = best_sh.tc_form;
    }
    return ARKCOS_OK;
}

arkcos_status arkcos_set_launch_shape(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                                     int64_t nmaps, uint32_t flags, const int64_t *shape)
{
    g_err[0] = 0;
    arkcos_status st = check_common(grid, kernels, nkernels, nmaps, flags);
    if (st != ARKCOS_OK) return st;
    if (!shape) return fail(ARKCOS_EINVAL, "shape is NULL");
    if (shape[0] != 1 && shape[0] != 2 && shape[0] != 4 && shape[0] != 8 && shape[0] != 16)
        return fail(ARKCOS_EINVAL, "FFT split multiplier %lld not in {1, 2, 4, 8, 16}", (long long)shape[0]);
    if (shape[1] < 0 || shape[1] > nmaps)
        return fail(ARKCOS_EINVAL, "maps per contraction CTA %lld not in [0, nmaps]", (long long)shape[1]);
    if (shape[2] < 0 || shape[2] > 5)
        return fail(ARKCOS_EINVAL, "contraction form %lld not in [0, 5]", (long long)shape[2]);
    const Shape sh{(int)shape[0], (int)shape[1], (int)shape[2]};
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[tune_key(grid, kernels, nkernels, nmaps, flags)] = sh;
    return ARKCOS_OK;
}

arkcos_status arkcos_host_workspace_size(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                                         int64_t nmaps, int64_t maps_per_chunk, uint32_t flags,
                                         size_t *bytes)
{
    g_err[0] = 0;
    if (!bytes) return fail(ARKCOS_EINVAL, "bytes is NULL");
    arkcos_status st = check_common(grid, kernels, nkernels, nmaps, flags);
    if (st != ARKCOS_OK) return st;
    HostLayout H;
    if ((st = host_layout(grid, kernels, nkernels, nmaps, maps_per_chunk, flags, H)) != ARKCOS_OK) return st;
    *bytes = H.total;
    return ARKCOS_OK;
}

arkcos_status arkcos_convolve_host(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                                   const float *host_in, float *host_out, int64_t nmaps, int64_t maps_per_chunk,
                                   void *workspace, size_t ws_bytes, void *stream, uint32_t flags)
{
    g_err[0] = 0;
    arkcos_status st = check_common(grid, kernels, nkernels, nmaps, flags);
    if (st != ARKCOS_OK) return st;
    if (!host_in || !host_out) return fail(ARKCOS_EINVAL, "host_in or host_out is NULL");
    const Grid &g = grid->g;
    const size_t mbytes = (size_t)nmaps * g.npix * sizeof(float);
    if (overlap(host_in, mbytes, host_out, mbytes)) return fail(ARKCOS_EINVAL, "host_in and host_out overlap");
    HostLayout H;
    if ((st = host_layout(grid, kernels, nkernels, nmaps, maps_per_chunk, flags, H)) != ARKCOS_OK) return st;
    if (!workspace || ((uintptr_t)workspace & 255))
        return fail(ARKCOS_EWORKSPACE, "workspace is NULL or not 256-byte aligned");
    if (ws_bytes < H.total) return fail(ARKCOS_EWORKSPACE, "workspace of %zu bytes < %zu required", ws_bytes, H.total);
    const bool per_map = nkernels > 1;
    char *ws = (char *)workspace;
    cudaStream_t s = (cudaStream_t)stream, up = nullptr, down = nullptr;
    cudaEvent_t ev[7] = {};  // start, in[2], conv[2], out[2]
    auto cleanup = [&]() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        if (up) cudaStreamDestroy(up);
        if (down) cudaStreamDestroy(down);
    };
#define HK(call)                                          \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) {                          \
            cleanup();                                    \
            return cuda_fail(e_, #call);                  \
        }                                                 \
    } while (0)
    HK(cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking));
    HK(cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking));
    for (auto &e : ev) HK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaEvent_t &ev_start = ev[0], *ev_in = ev + 1, *ev_conv = ev + 3, *ev_out = ev + 5;
    // both copy streams start after the work already queued on the caller's stream
    HK(cudaEventRecord(ev_start, s));
    HK(cudaStreamWaitEvent(up, ev_start, 0));
    HK(cudaStreamWaitEvent(down, ev_start, 0));
    // chunks: half a chunk first and last (the first upload and the last download are the parts
    // of the pipeline that nothing overlaps), full chunks between
    std::vector<int64_t> sizes;
    {
        const int64_t h = (H.chunk + 1) / 2;
        if (nmaps <= H.chunk) {
            sizes.push_back(nmaps);
        } else {
            sizes.push_back(h);
            const int64_t tail = std::min(h, nmaps - h);
            int64_t mid = nmaps - h - tail;
            while (mid > 0) {
                sizes.push_back(std::min(H.chunk, mid));
                mid -= sizes.back();
            }
            if (tail > 0) sizes.push_back(tail);
        }
    }
    int64_t c0 = 0;
    for (int64_t c = 0; c < (int64_t)sizes.size(); c0 += sizes[c], ++c) {
        const int q = (int)(c & 1);
        const int64_t cnt = sizes[c];
        const size_t bytes = (size_t)cnt * g.npix * sizeof(float);
        float *din = (float *)(ws + H.in[q]), *dout = (float *)(ws + H.out[q]);
        // upload chunk c once the convolution of chunk c - 2 has read this input buffer
        if (c >= 2) HK(cudaStreamWaitEvent(up, ev_conv[q], 0));
        HK(cudaMemcpyAsync(din, host_in + c0 * g.npix, bytes, cudaMemcpyHostToDevice, up));
        HK(cudaEventRecord(ev_in[q], up));
        // convolve once it has arrived and the download of chunk c - 2 has read this output
        HK(cudaStreamWaitEvent(s, ev_in[q], 0));
        if (c >= 2) HK(cudaStreamWaitEvent(s, ev_out[q], 0));
        // a shared beam's samples and polar table are computed by the first chunk only
        st = convolve_impl(grid, kernels + (per_map ? c0 : 0), per_map ? cnt : 1, din, dout, cnt, ws + H.conv,
                           H.conv_bytes, stream, flags, per_map || c == 0);
        if (st != ARKCOS_OK) {
            char msg[sizeof(g_err)];
            snprintf(msg, sizeof(msg), "%s", g_err);
            cleanup();
            return fail(st, "%s", msg);
        }
        HK(cudaEventRecord(ev_conv[q], s));
        HK(cudaStreamWaitEvent(down, ev_conv[q], 0));
        HK(cudaMemcpyAsync(host_out + c0 * g.npix, dout, bytes, cudaMemcpyDeviceToHost, down));
        HK(cudaEventRecord(ev_out[q], down));
    }
    // the caller's stream continues after the last download
    HK(cudaEventRecord(ev_start, down));
    HK(cudaStreamWaitEvent(s, ev_start, 0));
#undef HK
    cleanup();  // destruction waits for nothing: the streams and events are released when done
    return ARKCOS_OK;
}

arkcos_status arkcos_convolve_backward(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                                       const float *map_in, const float *grad_out, float *grad_in,
                                       double *grad_knots, int64_t nmaps, void *workspace, size_t ws_bytes,
                                       void *stream, uint32_t flags)
{
    g_err[0] = 0;
    arkcos_status st = check_common(grid, kernels, nkernels, nmaps, flags);
    if (st != ARKCOS_OK) return st;
    if (!grad_out) return fail(ARKCOS_EINVAL, "grad_out is NULL");
    if (grad_knots && !map_in) return fail(ARKCOS_EINVAL, "map_in is required for grad_knots");
    if (misaligned(map_in) || misaligned(grad_out) || misaligned(grad_in))
        return fail(ARKCOS_EINVAL, "map buffers must be 8-byte aligned");
    const Grid &g = grid->g;
    const size_t mbytes = (size_t)nmaps * g.npix * sizeof(float);
    if (grad_in && (overlap(grad_in, mbytes, grad_out, mbytes) || (map_in && overlap(grad_in, mbytes, map_in, mbytes))))
        return fail(ARKCOS_EINVAL, "grad_in overlaps grad_out or map_in");
    Layout L;
    if (!layout_for(g, kernels, nkernels, nmaps, true, grad_knots != nullptr, L))
        return fail(ARKCOS_EINVAL, "too many kernels");
    if (!workspace || ((uintptr_t)workspace & 255))
        return fail(ARKCOS_EWORKSPACE, "workspace is NULL or not 256-byte aligned");
    if (ws_bytes < L.total)
        return fail(ARKCOS_EWORKSPACE, "workspace of %zu bytes < %zu required", ws_bytes, L.total);
    cudaStream_t s = (cudaStream_t)stream;
    const bool basic = flags & ARKCOS_FLAG_BASIC;
    const bool shift_fix = !(flags & ARKCOS_FLAG_NO_SHIFT_FIX);
    const bool pole_fix = g.kind == 0 && !(flags & ARKCOS_FLAG_NO_POLE_FIX);
    char *ws = (char *)workspace;
    float4 *aspec = (float4 *)(ws + L.spec);
    float4 *gspec = (float4 *)(ws + L.gspec);
    float2 *cbuf = (float2 *)(ws + L.cbuf);
    if ((st = run_taps(g, kernels, nkernels, ws, L, shift_fix, s)) != ARKCOS_OK) return st;
    // spectra of the output gradient; the pole rings' hybrid outputs are overwritten by the
    // pole fix, so their gradient enters only through the transposed direct sum
    if ((st = run_fft_fwd(g, grad_out, nullptr, gspec, nmaps, false, pole_fix, basic, s)) != ARKCOS_OK)
        return st;
    const bool per_map = nkernels > 1;
    if (grad_in) {
        // L^T = W L W^{-1}: the same band sum with the ring weight on the output side
        if ((st = run_contract(g, kernels, nkernels, ws, L, gspec, cbuf, nmaps, basic, shift_fix,
                               (flags & ARKCOS_FLAG_3XTF32) != 0, s)) != ARKCOS_OK)
            return st;
        if ((st = run_fft_inv(g, cbuf, grad_in, nmaps, true, basic, false, s)) != ARKCOS_OK) return st;
        if (pole_fix) {
            int maxb = 0;
            for (int64_t k = 0; k < nkernels; ++k) maxb = std::max(maxb, kernels[k]->k.pole_band);
            StageScope sc(ST_POLE_ADJ, (int)((nmaps + kMaxKernelsPerLaunch - 1) / kMaxKernelsPerLaunch), s);
            for (int64_t base = 0; base < nmaps; base += kMaxKernelsPerLaunch) {
                const int64_t cnt = std::min<int64_t>(kMaxKernelsPerLaunch, nmaps - base);
                PoleArgs a = pole_args(g, kernels, per_map ? base : 0, cnt, per_map, grad_out, grad_in);
                a.map = grad_out + base * g.npix;
                a.out = grad_in + base * g.npix;
                CK(launch_pole_adj(a, maxb, s));
            }
        }
    }
    if (grad_knots) {
        if ((st = run_fft_fwd(g, map_in, nullptr, aspec, nmaps, true, false, basic, s)) != ARKCOS_OK)
            return st;
        float *Q = (float *)(ws + L.q);
        double *partial = (double *)(ws + L.partial);
        for (int64_t k = 0; k < nkernels; ++k) {
            const int64_t map0 = per_map ? k : 0;
            const int64_t nm = per_map ? 1 : nmaps;
            KnotGradArgs a;
            memset(&a, 0, sizeof(a));
            a.rd = g.dev();
            a.kd = kernels[k]->k.kd;
            a.spec4 = aspec;
            a.gspec4 = gspec;
            a.s2 = g.d_s2;
            a.tw = g.d_tw;
            a.partial = partial;
            a.R = g.R;
            a.N = g.N;
            a.NH = g.N / 2 + 1;
            a.nrep = g.nrep;
            a.B = (int)nmaps;
            a.map0 = (int)map0;
            a.nmaps = (int)nm;
            a.nspec = g.nspec;
            a.basic = basic;
            a.shift_fix = shift_fix;
            a.pole_fix = pole_fix;
            a.withhold_mma = test_withhold_mma();
            const Kernel &K = kernels[k]->k;
            {
                StageScope sc(ST_KNOT_Q, 1, s);
                CK(launch_knot_grad_q(a, Q, K.maxband, K.max_union8, K.max_union2, K.max_stage_rows, s));
            }
            {
                // 3xTF32 form: the cosine sums of the pairs past the FFT-projected ones as one
                // tensor-core product, then the deposits; otherwise both on the CUDA cores
                StageScope sc(ST_KNOT_PROJ, 1, s);
                const bool tc = (flags & ARKCOS_FLAG_3XTF32) && K.proj_tc_ok;
                float *X = (float *)(ws + L.xproj);
                if (tc) {
                    CK(launch_knot_proj_tc(a, Q, g.d_ctabP, g.nmc_p, K.knot_fft_pairs, X, s));
                    ++sc.launches;
                }
                CK(launch_knot_grad_proj(a, Q, tc ? X : nullptr, K.knot_fft_pairs, s));
            }
            int rows = knot_proj_blocks();
            if (kernels[k]->k.knot_fft_pairs > 0) {
                StageScope sc(ST_KNOT_PROJ, 1, s);
                CK(launch_knot_grad_proj_fft(a, Q, kernels[k]->k.knot_fft_pairs, rows, s));
                rows += kernels[k]->k.knot_fft_pairs;
            }
            if (pole_fix) {
                StageScope sc(ST_KNOT_POLE, 1, s);
                CK(launch_knot_grad_pole(a, map_in, grad_out, g.npix, rows, s));
                rows += 8 * (int)nm;
            }
            StageScope sc(ST_KNOT_REDUCE, 1, s);
            CK(launch_knot_reduce(partial, rows, kernels[k]->k.T, grad_knots + k * kernels[k]->k.T, s));
        }
    }
    return ARKCOS_OK;
}

arkcos_status arkcos_batch_workspace_size(const arkcos_job *jobs, int64_t njobs, size_t *bytes)
{
    g_err[0] = 0;
    if (!jobs || njobs < 1 || !bytes) return fail(ARKCOS_EINVAL, "jobs, njobs or bytes invalid");
    size_t tot = 0;
    for (int64_t q = 0; q < njobs; ++q) {
        size_t b = 0;
        arkcos_status st = arkcos_workspace_size(jobs[q].grid, jobs[q].kernels, jobs[q].nkernels,
                                                 jobs[q].nmaps, jobs[q].flags, 0, &b);
        if (st != ARKCOS_OK) return st;
        tot += align256(b);
    }
    *bytes = tot;
    return ARKCOS_OK;
}

arkcos_status arkcos_convolve_batch(const arkcos_job *jobs, int64_t njobs, void *workspace, size_t ws_bytes,
                                    void *stream)
{
    g_err[0] = 0;
    size_t need = 0;
    arkcos_status st = arkcos_batch_workspace_size(jobs, njobs, &need);
    if (st != ARKCOS_OK) return st;
    if (!workspace || ((uintptr_t)workspace & 255))
        return fail(ARKCOS_EWORKSPACE, "workspace is NULL or not 256-byte aligned");
    if (ws_bytes < need) return fail(ARKCOS_EWORKSPACE, "workspace of %zu bytes < %zu required", ws_bytes, need);
    // validate every job before enqueuing anything
    for (int64_t q = 0; q < njobs; ++q) {
        const arkcos_job &J = jobs[q];
        if ((st = check_common(J.grid, J.kernels, J.nkernels, J.nmaps, J.flags)) != ARKCOS_OK) return st;
        if (!J.map_in || !J.map_out) return fail(ARKCOS_EINVAL, "job %lld: map_in or map_out is NULL", (long long)q);
        if (misaligned(J.map_in) || misaligned(J.map_out))
            return fail(ARKCOS_EINVAL, "job %lld: map buffers must be 8-byte aligned", (long long)q);
        const size_t mb = (size_t)J.nmaps * J.grid->g.npix * sizeof(float);
        if (overlap(J.map_in, mb, J.map_out, mb))
            return fail(ARKCOS_EINVAL, "job %lld: map_in and map_out overlap", (long long)q);
    }
    char *ws = (char *)workspace;
    for (int64_t q = 0; q < njobs; ++q) {
        const arkcos_job &J = jobs[q];
        size_t b = 0;
        arkcos_workspace_size(J.grid, J.kernels, J.nkernels, J.nmaps, J.flags, 0, &b);
        st = arkcos_convolve(J.grid, J.kernels, J.nkernels, J.map_in, J.map_out, J.nmaps, ws, b, stream,
                             J.flags);
        if (st != ARKCOS_OK) {
            char msg[400];
            snprintf(msg, sizeof(msg), "job %lld: %s", (long long)q, g_err);
            snprintf(g_err, sizeof(g_err), "%s", msg);
            return st;
        }
        ws += align256(b);
    }
    return ARKCOS_OK;
}

arkcos_status arkcos_ring_analysis(arkcos_grid grid, const float *map_in, float *spec_out, int64_t nmaps,
                                   void *stream)
{
    g_err[0] = 0;
    if (!grid || !map_in || !spec_out) return fail(ARKCOS_EINVAL, "grid, map_in or spec_out is NULL");
    if (nmaps < 1) return fail(ARKCOS_EINVAL, "nmaps must be >= 1");
    if (misaligned(map_in) || misaligned(spec_out)) return fail(ARKCOS_EINVAL, "buffers must be 8-byte aligned");
    return run_fft_fwd(grid->g, map_in, (float2 *)spec_out, nullptr, nmaps, false, false, false,
                       (cudaStream_t)stream);
}

arkcos_status arkcos_ring_synthesis(arkcos_grid grid, const float *coeffs, float *map_out, int64_t nmaps,
                                    uint32_t flags, void *stream)
{
    g_err[0] = 0;
    if (!grid || !coeffs || !map_out) return fail(ARKCOS_EINVAL, "grid, coeffs or map_out is NULL");
    if (nmaps < 1) return fail(ARKCOS_EINVAL, "nmaps must be >= 1");
    if (misaligned(coeffs) || misaligned(map_out)) return fail(ARKCOS_EINVAL, "buffers must be 8-byte aligned");
    if (flags & ~ARKCOS_FLAG_BASIC) return fail(ARKCOS_EINVAL, "only ARKCOS_FLAG_BASIC applies to synthesis");
    return run_fft_inv(grid->g, (const float2 *)coeffs, map_out, nmaps, false, (flags & ARKCOS_FLAG_BASIC) != 0,
                       false, (cudaStream_t)stream);
}

arkcos_status arkcos_kernel_info(arkcos_kernel kernel, int64_t *pairs, int64_t *samples, int64_t *max_band)
{
    g_err[0] = 0;
    if (!kernel) return fail(ARKCOS_EINVAL, "kernel is NULL");
    if (pairs) *pairs = kernel->k.npairs;
    if (samples) *samples = kernel->k.sum_taps_fix;
    if (max_band) *max_band = kernel->k.maxband;
    return ARKCOS_OK;
}

arkcos_status arkcos_stage_timing(int enable)
{
    g_err[0] = 0;
    std::lock_guard<std::mutex> lk(g_tmu);
    timing_clear();
    g_timing = enable != 0;
    return ARKCOS_OK;
}

arkcos_status arkcos_stage_report(int64_t stage, const char **name, double *ms, int64_t *executions,
                                  int64_t *launches)
{
    g_err[0] = 0;
    if (stage < 0 || stage >= ST_COUNT) return fail(ARKCOS_EINVAL, "stage %lld out of range", (long long)stage);
    std::lock_guard<std::mutex> lk(g_tmu);
    double tot = 0.0;
    int64_t ex = 0, nl = 0;
    for (auto &r : g_recs) {
        if (r.stage != stage) continue;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float t = 0.f;
        e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        tot += t;
        ++ex;
        nl += r.launches;
    }
    if (name) *name = kStageNames[stage];
    if (ms) *ms = tot;
    if (executions) *executions = ex;
    if (launches) *launches = nl;
    return ARKCOS_OK;
}

arkcos_status arkcos_sync_status(void *stream)
{
    g_err[0] = 0;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetLastError");
    int tc_err = 0;
    e = take_tc_error(&tc_err);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device error word");
    if (tc_err)
        return fail(ARKCOS_ETIMEOUT, "a tensor-core completion wait expired (results of that call are invalid)");
    return ARKCOS_OK;
}

}  // extern "C"
