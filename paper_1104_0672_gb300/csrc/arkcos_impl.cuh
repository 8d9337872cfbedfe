// Internal declarations of libarkcos (not installed; the public ABI is include/arkcos.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "arkcos.h"

namespace arkcos {

constexpr int kMaxKernelsPerLaunch = 32;  // per-map beams handled per contraction launch
constexpr int kMaxPolarPairs = 16384;      // most pairs whose coefficients are tabulated per call
constexpr int kModeBlock = 128;           // modes per contraction CTA (one per thread)
constexpr int kMaxFftM = 8192;            // largest in-shared-memory ring FFT buffer (complex pairs)
constexpr int kMaxSplitM = 8192;          // buffer of the quarter transforms of split rings
constexpr int kSplitClass = 15;           // FFT class index of the split rings

// Ring table on the device (structure of arrays, R entries each).
struct RingDev {
    const int *n;         // pixels in the ring (even)
    const int *hs;        // 1: first pixel at phi0 = pi / n (half-pixel offset); 0: phi0 = 0
    const int64_t *poff;  // offset of the ring's first pixel in a map
    const int64_t *soff;  // offset of the ring's half spectrum (n/2 + 1 complex)
    const float *w;       // pixel solid-angle weight
    const double *theta;  // colatitude (FP64)
    const float2 *fb;     // Bluestein chirp spectra of the representative rings
    const int *fboff;     // [R] offset of a ring's chirp spectrum in fb (-1: power-of-two ring)
};

// One class of ring-pair representatives sharing an FFT buffer size M.
struct FftClass {
    int M = 0;            // largest buffer of the class (rings pick their own size <= M)
    int logM = 0;
    int threads = 0;
    int count = 0;
    int stage_c = 0;      // some ring of the class is shorter than N / 4
    int split = 0;        // rings of n = 4q pixels transformed as four q-point Bluestein DFTs
    int tab = 0;          // largest chirp + phase table of the class (complex words)
    int *reps = nullptr;  // device array of representative (northern) ring indices
};

struct Grid {
    int kind = 0;  // 0 HEALPix, 1 ECP
    int64_t nside = 0, ntheta = 0, nphi = 0;
    int R = 0;         // rings
    int N = 0;         // kernel longitude grid length
    int nrep = 0;      // ring-pair representatives (northern rings incl. the middle one)
    int64_t npix = 0;  // pixels per map
    int64_t nspec = 0; // complex half-spectrum entries per map, sum (n/2 + 1)
    std::vector<double> theta, wgt;
    std::vector<int> n, hs;
    std::vector<int64_t> poff, soff;
    // device copies
    int *d_n = nullptr, *d_hs = nullptr;
    int64_t *d_poff = nullptr, *d_soff = nullptr;
    float *d_w = nullptr;
    double *d_theta = nullptr;
    float2 *d_tw = nullptr;     // stage twiddles: tw[h + p] = exp(-2 pi i p / (2h)), p < h
    int twM = 0;
    double *d_s2 = nullptr;     // sin^2(pi t / (2N)) for t = 0..N
    float *d_s2f = nullptr;     // the same rounded to FP32 (the knot-segment search)
    float *d_ctab = nullptr;    // tensor-core cosine table (TF32 hi/lo, core-matrix layout)
    int nkc_tab = 0;            // 32-sample chunks the cosine table covers
    float *d_ctabP = nullptr;   // knot-projection cosine table: per chunk of 32 modes, 128 taps of
                                // each flavour (TF32 hi/lo, core-matrix layout)
    int nmc_p = 0;              // its chunks of 32 modes
    std::vector<FftClass> fft;  // forward/inverse FFT launch classes
    int live_kernels = 0;
    float2 *d_fb = nullptr;     // Bluestein chirp spectra (DIF order) of the representative rings
    int *d_fboff = nullptr;
    RingDev dev() const { return RingDev{d_n, d_hs, d_poff, d_soff, d_w, d_theta, d_fb, d_fboff}; }
};

// Device view of one kernel's ring-pair tables.  Pairs are listed per representative
// output ring i (i <= R-1-i), with input rings j = jlo[i]..jhi[i] in order.
struct KernDev {
    const int *pstart;   // [nrep + 1] first pair of each representative
    const int *jlo;      // [nrep]
    const int *jhi;      // [nrep]
    const int *S0;       // [npairs] last in-support tap, integer-offset samples (-1 none)
    const int *S1;       // [npairs] last in-support tap, half-offset samples (-1 none)
    const int *fl;       // [npairs] 1 when the pair samples at half offsets (shift fix)
    const int *toff;     // [npairs + 1] tap offsets (multiples of 4)
    const double *A;     // [npairs] sin^2((theta_i + theta_j)/2)
    const double *B;     // [npairs] sin^2((theta_i - theta_j)/2)
    const double *knots; // [T]
    const double *ut;    // [T] u_t = 4 sin^2(gamma_t / 2)
    const int4 *coltab;  // [ceil(nrep / 8)][256] tensor-core columns of each block of 8 rings:
                         // (pair or -1, tap offset, S0, 2 S1 + fl), rings in groups of two
    const int4 *coltab4; // the same with the rings in groups of four
    const int2 *unit_fix;   // knot-gradient work units (pair, first tap), with the shift fix
    const int2 *unit_nofix; // ... and without it
    int nunit_fix, nunit_nofix;
    int T;
    int npairs;
    int polar_pairs;     // pairs [0, polar_pairs) (rings next to the poles with many samples)
                         // take their coefficients from a table computed before the contraction
    double umax;
    double gscale;       // (T - 1) / gamma_max, for the first guess of the knot segment
};

struct Kernel {
    Grid *g = nullptr;
    int T = 0;
    double gmax = 0, umax = 0;
    int npairs = 0;
    int64_t ntaps = 0;  // padded tap slots
    int maxband = 0;
    int maxS = 0;
    int pole_band = 0;         // input rings inside the support of ring 0
    int max_union8 = 0;        // largest union band of 8 consecutive representative rings
    int max_union2 = 0;        // largest union band of rings 2g, 2g+1 of those blocks of 8
    int max_stage_rows = 0;    // staged rows a tensor-core block of 8 rings needs: its union
                               // band, and every group's first ring + 32 slots
    int max_stage_rows16 = 0;  // the same for blocks of 16 rings
    int max_union4 = 0;        // largest union band of rings 4g .. 4g+3
    int max_stage_rows_g4 = 0, max_stage_rows16_g4 = 0;  // staged rows with groups of four
    int polar_pairs = 0;       // leading pairs whose coefficients are tabulated per call
    int knot_fft_pairs = 0;    // leading pairs whose knot-gradient projection runs by FFT
    bool proj_tc_ok = false;   // the other pairs have at most 128 samples (tensor-core projection)
    int64_t sum_taps_fix = 0;  // in-support tap count with the shift fix (for reporting)
    void *dmem = nullptr;      // one device allocation holding every table
    KernDev kd{};
};

// ------------------------------------------------------------------ launch arguments
struct TapArgs {
    KernDev kd;
    const double *s2;
    const float *s2f;
    float *taps;   // [ntaps]
    int N;
    int shift_fix;
};

struct FftFwdArgs {
    RingDev rd;
    const float2 *tw;
    const float *map;   // [B][npix]
    float2 *spec;       // [B][nspec] half spectra (ext4 == 0)
    float4 *spec4;      // [B][nrep][NH] extended spectra of ring and mirror (ext4 == 1)
    int ext4, nrep, NH, basic;
    const int *reps;
    int M, logM, R, N, B;
    int mchunk;         // maps per CTA: CTA (ring pair, blockIdx.y) takes maps [y mchunk, ...)
    int64_t npix, nspec;
    int weight;         // multiply spectra by the ring weight
    int zero_poles;     // treat rings 0 and R-1 as zero (adjoint input)
    int tab;            // shared-memory words for the per-ring chirp and phase tables
    int split;          // the class holds split rings (n = 4q, see FftClass)
};

struct FftInvArgs {
    RingDev rd;
    const float2 *tw;
    const float2 *c;    // [B][R][NH]
    float *map;         // [B][npix]
    const int *reps;
    int M, logM, R, N, NH, B;
    int mchunk;         // maps per CTA: CTA (ring pair, blockIdx.y) takes maps [y mchunk, ...)
    int64_t npix;
    int weight;         // multiply by the ring weight
    int basic;
    int skip_poles;     // leave rings 0 and R-1 untouched (written by the pole kernel)
    int stage_c;        // stage coefficients in shared memory for rings with 4 n < N
    int tab;            // shared-memory words for the per-ring chirp and phase tables
};

struct ContractArgs {
    RingDev rd;
    KernDev kd[kMaxKernelsPerLaunch];
    const float *taps[kMaxKernelsPerLaunch];
    const float *prho[kMaxKernelsPerLaunch];  // [polar_pairs][NH] tabulated coefficients
    const float4 *spec4; // [B][nrep][NH]: (a_m(j), a_m(R-1-j)) for representative j
    float2 *c;          // [B][R][NH]
    int R, N, NH, nrep, B;
    int64_t nspec;
    int maps_per_chunk; // maps sharing one generation pass
    int per_map;        // 1: map b uses kd[b - map_base]
    int map_base;
    int basic, shift_fix;
    int pair_chunk;     // pairs whose coefficients fit in shared memory at once
    int withhold_mma;   // test knob: issue no tensor-core MMA, so the completion waits expire
    int vbase, vdiv;    // vdiv > 1 (several kernels on one input): map b of the launch reads the
                        // spectra of input (vbase + b) / vdiv of spec4; else those of map b
};

// Extended spectra of map b of a contraction launch.
__device__ __forceinline__ const float4 *map_spec4(const ContractArgs &a, int b)
{
    const int s = a.vdiv > 1 ? (a.vbase + b) / a.vdiv : b;
    return a.spec4 + (int64_t)s * a.nrep * a.NH;
}

struct PoleArgs {
    RingDev rd;
    KernDev kd[kMaxKernelsPerLaunch];
    const float *map;   // input (forward) or gradient (adjoint)
    float *out;
    int R, B, per_map, map_base;
    int64_t npix;
    int vbase, vdiv;    // vdiv > 1: output map b reads input map (vbase + b) / vdiv of `map`
    int nsum;           // > 0 (forward only): output map b is the sum over kernels k < nsum of
    double wsum[kMaxKernelsPerLaunch];  // wsum[k] x the direct sum of kd[k] over input map b
};

struct KnotGradArgs {
    RingDev rd;
    KernDev kd;
    const float4 *spec4;  // weighted extended spectra of the input maps [B][nrep][NH]
    const float4 *gspec4; // extended spectra of the output gradients [B][nrep][NH]
    const double *s2;
    const float2 *tw;    // stage twiddles of the grid (FFT projection of the polar pairs)
    double *partial;     // [rows][T] per-CTA partial sums
    int R, N, NH, nrep, B, map0, nmaps;
    int64_t nspec;
    int basic, shift_fix;
    int pole_fix;        // pole rings' hybrid outputs are replaced (skip their g)
    int withhold_mma;    // test knob: issue no tensor-core MMA, so the completion waits expire
};

// Extended spectrum of ring j at mode m from the paired layout: the representative row of j
// holds (a(rep), a(R-1-rep)); swap the halves for rings of the southern half.
__device__ __forceinline__ float4 paired_coeff(const float4 *__restrict__ sp4, int j, int R, int NH, int m)
{
    const int jm = R - 1 - j;
    const bool south = j > jm;
    float4 v = __ldg(&sp4[(int64_t)(south ? jm : j) * NH + m]);
    if (south) v = make_float4(v.z, v.w, v.x, v.y);
    return v;
}

// ------------------------------------------------------------------ launchers (return cuda error)
cudaError_t launch_taps(const TapArgs &a, int npairs, cudaStream_t st);
cudaError_t launch_polar_rho(const ContractArgs &a, int nk, int max_polar_pairs, const float2 *tw, int twM,
                             cudaStream_t st);
size_t fft_smem_bytes(int M, int N, bool stage_c, int tab, int threads, bool split);  // shared memory of a ring FFT class
cudaError_t launch_chirp_spectra(const FftFwdArgs &a, float2 *fb, int count, int threads, cudaStream_t st);
// Ring FFT class launches.  after_prev: the previous kernel on the stream is the previous class
// of the same stage, and this launch may begin while it still runs (ring_common.cuh
// stage_allow_next / stage_wait_prev).
cudaError_t launch_fft_fwd(const FftFwdArgs &a, int count, int threads, cudaStream_t st, bool after_prev);
cudaError_t launch_fft_fwd_split(const FftFwdArgs &a, int count, int threads, cudaStream_t st, bool after_prev);
int fft_map_chunk(int count, int nmaps, int split_mult);  // maps per CTA of a ring FFT launch over `count` ring pairs
cudaError_t launch_fft_inv(const FftInvArgs &a, int count, int threads, cudaStream_t st, bool after_prev);
cudaError_t launch_fft_inv_split(const FftInvArgs &a, int count, int threads, cudaStream_t st, bool after_prev);

// Launch of kernel(a) with the programmatic-serialization attribute when after_prev.
template <class Args>
cudaError_t launch_class_kernel(void (*kernel)(Args), dim3 grid, int threads, size_t smem, cudaStream_t st,
                                bool after_prev, const Args &a)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = after_prev ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}
cudaError_t launch_contract(const ContractArgs &a, int nchunks, size_t smem, cudaStream_t st);
cudaError_t launch_pole_fwd(const PoleArgs &a, cudaStream_t st);
// csum[b] = sum_k w[k] c[b K + k] for b < nmaps ([R][NH] complex coefficient arrays), the sum
// taken in order of k
cudaError_t launch_weighted_sum(const float2 *c, float2 *csum, int64_t nmaps, int K, const double *w,
                                int64_t per_map, cudaStream_t st);
cudaError_t launch_pole_adj(const PoleArgs &a, int max_band_rings, cudaStream_t st);
cudaError_t launch_knot_grad_q(const KnotGradArgs &a, float *Q, int max_band, int max_union, int max_union2,
                               int srows, cudaStream_t st);
cudaError_t launch_knot_grad_proj(const KnotGradArgs &a, const float *Q, const float *X, int pfirst,
                                  cudaStream_t st);
cudaError_t launch_knot_proj_tc(const KnotGradArgs &a, const float *Q, const float *ctabP, int nmc, int pfirst,
                                float *X, cudaStream_t st);
cudaError_t launch_knot_grad_proj_fft(const KnotGradArgs &a, const float *Q, int npairs, int row0, cudaStream_t st);
cudaError_t launch_knot_grad_pole(const KnotGradArgs &a, const float *map, const float *gout,
                                  int64_t npix, int row0, cudaStream_t st);
int knot_proj_blocks();
int knot_proj_taps();
cudaError_t launch_knot_reduce(const double *partial, int nrows, int T, double *out,
                               cudaStream_t st);
int contract_ring_block();
void set_last_error(const char *msg);  // sets the message arkcos_last_error() returns
int contract_band_limit();
int contract_band_rings();
cudaError_t launch_contract_band(const ContractArgs &a, int nchunks, int max_union, cudaStream_t st);
// tensor-core contraction over blocks of rb (8 or 16) representative rings, a thread taking
// a group of gs (2 or 4) rings
cudaError_t launch_contract_tc(const ContractArgs &a, int rb, int gs, int nchunks, const float *ctab, int nkc_tab,
                               int srows, int want_nbuf, cudaStream_t st);
int contract_tc_nbuf(int rb, int gs, int srows, int want_nbuf);
size_t contract_tc_smem(int rb, int gs, int srows, int want_nbuf);
int contract_tc_modes();
cudaError_t take_tc_error(int *out);
// Failure-detection test knob, read on every call: when the environment variable
// ARKCOS_TEST_WITHHOLD_MMA is set to a non-zero integer, the tensor-core kernels issue no MMA,
// so their bounded completion waits run out and the call reports ETIMEOUT through
// arkcos_sync_status.  Nothing is in flight when the waits give up.
int test_withhold_mma();
// Streaming multiprocessors of the current device (queried once per device; 152 if the query
// fails), for grid sizes that cover the GPU.
int device_sms();

}  // namespace arkcos
