// Tensor-core form of the ring-pair coefficient generation (3xTF32 on tcgen05), fused with
// the band contraction; and the tensor-core knot-gradient projection of the backward pass.
//
// For a block of RB (8 or 16) representative output rings x 128 modes the coefficients are a
// dense product  rho[m, col] = sum_k C_f[m, k] T[k, col]  with C_f[m, k] = cos(pi m (2k + f) / N)
// (f = the pair's sample offset, see contract.cu) and T the FP32 kernel samples.  The CTA
// stages C (an exact FP64 table split into TF32 hi + lo parts, prepared per grid in the
// tensor-core layout) and T (split into hi + lo on the fly) in shared memory, chunk by chunk of
// 32 samples with the next chunk's loads in flight, and one thread issues tcgen05.mma
// kind::tf32 with the accumulator in tensor memory:
//     D = C_hi T_hi + C_hi T_lo + C_lo T_hi      (3xTF32, FP32 accumulation).
// Pairs of the two offsets accumulate into the same columns with the other offset's samples
// zeroed.  The rings of the block go in groups of G (2 or 4) consecutive rings; column
// 32 (G g + t) + u holds the pair of ring G g + t with input ring jlo(G g) + u (zero when that
// ring is outside its band), so the rings of a group index one common run of 32 input rings.
// Each thread (mode, group) reads slices of its G x 32 coefficients of D with tcgen05.ld and
// contracts every staged input coefficient into all G rings' outputs.  Waits on the MMA
// completion barriers are bounded: on expiry the kernel records an error (reported by
// arkcos_sync_status) and still frees its tensor memory.
#include <stdint.h>

#include "tcgen05.cuh"

namespace arkcos {

__device__ int g_tc_error = 0;

namespace {

using namespace tc;

constexpr int kTcModes = 128;          // M of the MMA: modes per CTA (TMEM lanes)
constexpr int kTcBand = 32;            // input-ring slots per group (columns per ring)
constexpr int kTcNTile = 256;          // N of one MMA: 8 rings x 32 slots
constexpr int kTcKChunk = 32;          // taps per shared-memory chunk (4 MMA K-steps of 8)

// A CTA takes RB representative output rings (8 or 16) x kTcModes modes: RB / G ring groups
// of G (2 or 4) consecutive rings, one warp per group and lane quarter; RB x 32 tensor-memory
// columns, filled by RB / 8 MMAs of N = 256 per K-step.
template <int RB, int G>
struct TcShape {
    static constexpr int kRings = RB, kGroups = RB / G, kThreads = kTcModes * kGroups;
    static constexpr int kN = RB * kTcBand, kTiles = kN / kTcNTile, kTmemCols = kN;
    static constexpr size_t kAB = 2 * 16384 + 2 * (size_t)kN / 8 * kSBO;  // A hi | lo, B hi | lo
};

// acc += c v for the four lanes of v, as two packed two-lane FMAs (each lane rounds as fmaf)
__device__ __forceinline__ void fma4(float4 &acc, float c, const float4 &v)
{
    const float2 cc = make_float2(c, c);
    const float2 lo = __ffma2_rn(cc, make_float2(v.x, v.y), make_float2(acc.x, acc.y));
    const float2 hi = __ffma2_rn(cc, make_float2(v.z, v.w), make_float2(acc.z, acc.w));
    acc = make_float4(lo.x, lo.y, hi.x, hi.y);
}

template <int RB, int G>
__global__ void __launch_bounds__(TcShape<RB, G>::kThreads, 16 / RB)
k_contract_tc(ContractArgs a, const float *__restrict__ ctab, int nkc_tab, int srows, int nbuf)
{
    using Sh = TcShape<RB, G>;
    constexpr int kTcRings = Sh::kRings, kTcN = Sh::kN, kTcTmemCols = Sh::kTmemCols;
    extern __shared__ __align__(1024) unsigned char smem[];
    // A hi | A lo (16 KiB each) and B hi | B lo (32 KiB each), then reused for the
    // staged spectra; the last 16 bytes hold the MMA barrier and the tensor-memory address
    const size_t stage_bytes = (size_t)nbuf * srows * kTcModes * sizeof(float4);
    const size_t ab_bytes = Sh::kAB;
    const size_t ctl = ((stage_bytes > ab_bytes ? stage_bytes : ab_bytes) + 15) & ~size_t(15);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + ctl);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + ctl + 8);
    unsigned char *Ahi = smem, *Alo = smem + 16384;
    unsigned char *Bhi = smem + 32768, *Blo = Bhi + kTcN / 8 * kSBO;
    float4 *sh4 = reinterpret_cast<float4 *>(smem);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q4 = warp & 3, grp = warp >> 2;  // lane quarter of TMEM, ring group
    const int mrow = q4 * 32 + lane;           // mode within the block
    const int m = blockIdx.x * kTcModes + mrow;
    const bool mv = m < a.NH;
    const int r0 = blockIdx.y * kTcRings;
    const int nr = min(kTcRings, a.nrep - r0);
    if (a.basic) {
        // BASIC variant: output ring i keeps only its modes m <= n_i / 2 (Sec. 4.1 truncation;
        // the inverse transform reads no others), so a block of modes above the Nyquist
        // frequency of every ring of the block (and of their mirrors) has nothing to compute
        int nmax = 0;
        for (int t = 0; t < nr; ++t) nmax = max(nmax, __ldg(&a.rd.n[r0 + t]));
        if ((int)blockIdx.x * kTcModes > nmax / 2) return;
    }
    const int b0 = blockIdx.z * a.maps_per_chunk;
    const int b1 = min(a.B, b0 + a.maps_per_chunk);
    const int kid = a.per_map ? (b0 - a.map_base) : 0;
    const KernDev &kd = a.kd[kid];
    const float *taps = a.taps[kid];
    // this thread's rings i0 + t (t < G, valid while G grp + t < nr), i0 = r0 + G grp, whose
    // run starts at input ring jg0
    const int i0 = r0 + G * grp;
    const bool v0 = G * grp < nr;
    const int jg0 = v0 ? kd.jlo[i0] : 0;
    const int ju0 = kd.jlo[r0];
    const int nu = kd.jhi[r0 + nr - 1] - ju0 + 1;

    // ---- tensor memory and the completion barrier
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"((uint32_t)__cvta_generic_to_shared(tslot)), "r"(kTcTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;"
                     ::"r"((uint32_t)__cvta_generic_to_shared(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t mbar_s = (uint32_t)__cvta_generic_to_shared(mbar);

    // per pair slot: sample offset in `taps`, last sample and offset flavour (S = -1: empty);
    // and the largest sample count of the block's pairs per flavour
    __shared__ int s_kmax[2];
    __shared__ int s_toff[kTcN], s_S[kTcN], s_f[kTcN], s_p[kTcN];
    if (tid < 2) s_kmax[tid] = 0;
    __syncthreads();
    for (int c = tid; c < kTcN; c += blockDim.x) {
        // column c: ring l = c / 32 of the block, input ring jlo(first ring of l's group) + c % 32;
        // the table is laid out per block of 8 rings
        const int blk8 = blockIdx.y * (RB / 8) + c / kTcNTile;
        const int4 *ct = G == 2 ? kd.coltab : kd.coltab4;
        const int4 e = 8 * blk8 < a.nrep ? __ldg(&ct[(size_t)blk8 * kTcNTile + c % kTcNTile])
                                         : make_int4(-1, 0, -1, -2);
        int toff = 0, S = -1, f = 0, p = 0;
        if (e.x >= 0) {
            p = e.x;
            toff = e.y;
            f = a.shift_fix ? (e.w & 1) : 0;
            S = f ? (e.w >> 1) : e.z;
            atomicMax(&s_kmax[f], S + 1);
        }
        s_toff[c] = toff;
        s_S[c] = S;
        s_f[c] = f;
        s_p[c] = p;
    }
    __syncthreads();
    const int kmax0 = s_kmax[0], kmax1 = s_kmax[1];
    const int kcap = nkc_tab * kTcKChunk;  // samples the cosine table covers
    // blocks whose pairs all have tabulated coefficients read them (whatever the block size,
    // so both block sizes give the same result); the others generate theirs on the tensor
    // cores when the cosine table covers their samples
    const bool tabulated = kd.pstart[r0 + nr] <= kd.polar_pairs;
    const bool use_tc = !tabulated && kmax0 <= kcap && kmax1 <= kcap;
    // the coefficients stay in tensor memory: lane = mode, column 32 l + u (see above)
    const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16);
    const uint32_t colg = lane_base + (uint32_t)(G * grp * kTcBand);  // the group's first column
    bool have_rho = kmax0 + kmax1 > 0;  // CTA-uniform: some column has samples
    if (use_tc) {
        // once any CTA has seen an expired wait the results are invalid anyway: skip the MMAs
        bool ok = *((volatile int *)&g_tc_error) == 0;
        ok = __syncthreads_and(ok);
        uint32_t phase = 0;
        bool first = true;  // meaningful in the issuing thread only
        const uint32_t idesc = tf32_idesc(kTcModes, kTcNTile);
        // the chunks of 32 samples, flavour 0 first: the samples of chunk i + 1 are loaded into
        // registers while the MMAs of chunk i run, and its cosine tile is copied asynchronously
        // while its samples are split into the B operand
        const int n0 = (kmax0 + kTcKChunk - 1) / kTcKChunk, nch = n0 + (kmax1 + kTcKChunk - 1) / kTcKChunk;
        constexpr int kUnits = Sh::kN * 2 / Sh::kThreads;  // (column, 16 samples) units per thread
        float4 pre[kUnits][4];
        // a thread takes 16 consecutive samples of one column, loaded four at a time (tap
        // offsets are multiples of 4 and each pair's slots are padded to 4, so a float4 that
        // starts at or before the last sample stays inside the pair); others read as zero
        auto load_taps = [&](int i) {
            const int f = i < n0 ? 0 : 1, kc = f ? i - n0 : i;
#pragma unroll
            for (int u = 0; u < kUnits; ++u) {
                const int e = tid + u * blockDim.x, c = e >> 1, k0 = (e & 1) * 16;
                const int S = s_f[c] == f ? s_S[c] : -1;
                const float *tp = taps + s_toff[c];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int kk = kc * kTcKChunk + k0 + 4 * q;
                    pre[u][q] = kk <= S ? __ldg(reinterpret_cast<const float4 *>(tp + kk))
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        };
        if (nch > 0) load_taps(0);
        for (int i = 0; i < nch; ++i) {
            const int f = i < n0 ? 0 : 1, kc = f ? i - n0 : i;
            const int kf = f ? kmax1 : kmax0;
            const int ksteps = min(4, (kf - kc * kTcKChunk + 7) / 8);
            // A: this mode block's cosine chunk (hi, lo), prepared in the core layout
            const float *src = ctab + ((((size_t)blockIdx.x * 2 + f) * nkc_tab + kc) * 2) * 4096;
            for (int e = tid; e < 2 * 1024; e += blockDim.x) cp_async16(Ahi + 16 * e, src + 4 * e, 16);
            cp_async_commit();
            // B: the samples of every column of the block for this flavour, split hi / lo
#pragma unroll
            for (int u = 0; u < kUnits; ++u) {
                const int e = tid + u * blockDim.x, c = e >> 1, k0 = (e & 1) * 16;
                const int S = s_f[c] == f ? s_S[c] : -1;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int kk = kc * kTcKChunk + k0 + 4 * q;
                    const float v[4] = {pre[u][q].x, pre[u][q].y, pre[u][q].z, pre[u][q].w};
                    float4 hi4, lo4;
                    float *hp = &hi4.x, *lp = &lo4.x;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float x = kk + j <= S ? v[j] : 0.f;
                        hp[j] = tf32_round(x);
                        lp[j] = tf32_round(x - hp[j]);
                    }
                    const uint32_t off = core_offset(c, k0 + 4 * q);
                    *reinterpret_cast<float4 *>(Bhi + off) = hi4;
                    *reinterpret_cast<float4 *>(Blo + off) = lo4;
                }
            }
            if (i + 1 < nch) load_taps(i + 1);
            asm volatile("cp.async.wait_all;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            // CTA-uniform: whether this chunk's MMAs and their commit are issued (the test
            // knob withholds them, so that the wait below runs out)
            const bool issued = ok && !a.withhold_mma;
            if (tid == 0 && issued) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa_hi = (uint32_t)__cvta_generic_to_shared(Ahi);
                const uint32_t sa_lo = (uint32_t)__cvta_generic_to_shared(Alo);
                const uint32_t sb_hi = (uint32_t)__cvta_generic_to_shared(Bhi);
                const uint32_t sb_lo = (uint32_t)__cvta_generic_to_shared(Blo);
                for (int ks = 0; ks < ksteps; ++ks) {
                    const uint32_t o = ks * 2 * kLBO;  // 8 TF32 values = two core columns
#pragma unroll
                    for (int t = 0; t < Sh::kTiles; ++t) {
                        // tile t: columns [256 t, 256 t + 256), its B rows 32 KiB further on
                        const uint32_t d = tmem + (uint32_t)(t * kTcNTile);
                        const uint32_t ob = o + (uint32_t)t * (kTcNTile / 8) * kSBO;
                        mma_tf32(d, smem_desc(sa_hi + o), smem_desc(sb_hi + ob), idesc, first ? 0 : 1);
                        mma_tf32(d, smem_desc(sa_hi + o), smem_desc(sb_lo + ob), idesc, 1);
                        mma_tf32(d, smem_desc(sa_lo + o), smem_desc(sb_hi + ob), idesc, 1);
                    }
                    first = false;
                }
                mma_commit(mbar_s);
            }
            // every thread waits for the MMAs before the next chunk reuses shared memory; a
            // wait that expires is recorded and stops further MMAs.  An issued commit is
            // waited for once more (bounded) before anything reuses the memory its MMAs use;
            // nothing is in flight when the issue was withheld
            if (ok) {
                bool done = mbar_wait(mbar_s, phase);
                if (!done && issued) done = mbar_wait(mbar_s, phase);
                ok = done;
            }
            ok = __syncthreads_and(ok);
            if (!ok && tid == 0) atomicOr(&g_tc_error, 1);
            phase ^= 1;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        have_rho = have_rho && ok;
    } else {
        // blocks next to the poles have more samples per pair than the cosine table holds:
        // their coefficients were tabulated before this launch, or are generated here on the
        // CUDA cores; either way they go to the same tensor-memory columns, 16 at a time
        const bool tab = tabulated;
        const float *pr = a.prho[kid];
#pragma unroll 1
        for (int h = 0; h < G * kTcBand; h += 16) {
            const int cb = G * grp * kTcBand + h;  // first of 16 columns (one ring's half)
            float r[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int c = cb + u;
                float x = 0.f;
                if (mv && s_S[c] >= 0)
                    x = tab ? __ldg(&pr[(int64_t)s_p[c] * a.NH + m])
                            : gen_rho(reinterpret_cast<const float4 *>(taps + s_toff[c]), s_S[c], s_f[c], m, a.N);
                r[u] = x;
            }
            tmem_st16(colg + (uint32_t)h, r);
        }
    }
    const int joff = jg0 - ju0;  // the group's first input ring within the staged band
    __syncthreads();

    // ---- band contraction.  The union band of each map goes to shared memory by 16-byte
    // asynchronous copies that every thread issues (the copy engine of one thread per CTA
    // cannot keep enough bytes in flight); rows beyond the band stay zero, so every group
    // runs its 32 slots unpredicated (its coefficients are zero there).  nbuf == 2: the next
    // map is copied while this one is contracted; nbuf == 1: one buffer (the 8-ring form that
    // keeps two CTAs on an SM, or bands too wide for two).
    const int mid = (a.R - 1) / 2;
    const bool crosses = ju0 + nu - 1 > mid;
    const int sstar = mid - jg0 + 1;  // first slot of the group's run that is a southern ring
    const size_t bufsz = (size_t)srows * kTcModes;
    const int m0 = blockIdx.x * kTcModes;
    for (size_t e = tid; e < (size_t)nbuf * bufsz; e += blockDim.x) sh4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    auto issue = [&](int bb, int q) {
        stage_band_async(sh4 + q * bufsz, map_spec4(a, bb), ju0, nu, m0, kTcModes, a.R, a.NH);
    };
    if (b0 < b1) issue(b0, 0);
    for (int b = b0; b < b1; ++b) {
        const int cur = nbuf == 2 ? (b - b0) & 1 : 0;
        if (nbuf == 2 && b + 1 < b1) {
            issue(b + 1, cur ^ 1);
            cp_async_wait1();  // this map's copies (all but the newest group) have landed
        } else {
            asm volatile("cp.async.wait_all;" ::: "memory");
        }
        __syncthreads();
        float4 acc[G];
#pragma unroll
        for (int t = 0; t < G; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (v0 && have_rho) {  // warp-uniform: the tensor-memory loads are warp-collective
            const float4 *col = sh4 + cur * bufsz + joff * kTcModes + mrow;
            // slots in chunks of CH: the chunk's coefficients of the G rings, then CH staged
            // values, each used by all G rings
            constexpr int CH = G == 2 ? 16 : 8;
#pragma unroll
            for (int h = 0; h < kTcBand; h += CH) {
                uint32_t cr[G][CH];
#pragma unroll
                for (int t = 0; t < G; ++t) tmem_ld_async(colg + (uint32_t)(t * kTcBand + h), cr[t]);
                tmem_wait_ld();
                if (!crosses) {
#pragma unroll
                    for (int u = 0; u < CH; ++u) {
                        const float4 v = col[(h + u) * kTcModes];
#pragma unroll
                        for (int t = 0; t < G; ++t) fma4(acc[t], __uint_as_float(cr[t][u]), v);
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < CH; ++u) {
                        float4 v = col[(h + u) * kTcModes];
                        if (h + u >= sstar) v = make_float4(v.z, v.w, v.x, v.y);
#pragma unroll
                        for (int t = 0; t < G; ++t) fma4(acc[t], __uint_as_float(cr[t][u]), v);
                    }
                }
            }
        }
        if (mv) {
            float2 *cb = a.c + (int64_t)b * a.R * a.NH + m;
#pragma unroll
            for (int t = 0; t < G; ++t) {
                const int i = i0 + t;
                if (G * grp + t < nr) {
                    cb[(int64_t)i * a.NH] = make_float2(acc[t].x, acc[t].y);
                    if (a.R - 1 - i != i) cb[(int64_t)(a.R - 1 - i) * a.NH] = make_float2(acc[t].z, acc[t].w);
                }
            }
        }
        __syncthreads();
        if (nbuf == 1 && b + 1 < b1) issue(b + 1, 0);
    }

    // ---- release tensor memory
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols));
}

// Knot-gradient projection on the tensor cores (the 3xTF32 form of the backward pass):
//     X[p][k] = sum_m Q_m(p) cos(pi m (2k + f) / N),   k < 128, f = 0 and 1,
// a dense product of the Q rows of 128 ring pairs (A, M = 128, split hi/lo on the fly) and a
// per-grid table of the cosines of 128 taps of each flavour (B, N = 256, K = 32 modes per
// chunk, hi/lo in the core layout).  The sum over the modes is long (N/2 + 1 terms) and the
// cosines make it cancel, so it is not left to the tensor core's accumulator, whose additions
// do not round to nearest: every chunk's twelve MMAs start from zero in one of two 256-column
// accumulators, and once a chunk is complete its 128 x 256 partial sums are added in FP32
// (round to nearest) into registers of the epilogue threads while the next chunk's MMAs fill
// the other accumulator.  Two stages of shared memory: chunk c + 1 is staged while the MMAs of
// chunk c run, each stage (and its accumulator) released by its own completion barrier
// (bounded waits).  Each pair's row of its own flavour's 128 values goes to X; the hat-weight
// deposits follow in k_knot_proj.
constexpr int kPjPairs = 128, kPjThreads = 256;
constexpr uint32_t kPjA = 16384, kPjB = 32768, kPjStage = 2 * kPjA + 2 * kPjB;  // 96 KiB per stage
constexpr uint32_t kPjCols = 256;                                              // per accumulator

__global__ void __launch_bounds__(kPjThreads, 1)
k_knot_proj_tc(KnotGradArgs a, const float *__restrict__ Q, const float *__restrict__ ctabP, int nmc, int pfirst,
               float *X)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * kPjStage);  // [2] stage barriers
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + 2 * kPjStage + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int pbase = pfirst + blockIdx.x * kPjPairs;
    const int npairs = a.kd.npairs;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"((uint32_t)__cvta_generic_to_shared(tslot)), "r"(2 * kPjCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int q = 0; q < 2; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;"
                         ::"r"((uint32_t)__cvta_generic_to_shared(bar + q)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t bar_s = (uint32_t)__cvta_generic_to_shared(bar);
    bool ok = *((volatile int *)&g_tc_error) == 0;
    ok = __syncthreads_and(ok);
    uint32_t ph = 0;    // bit s: parity of the next completion of stage s
    uint32_t pend = 0;  // bit s: stage s has an issued commit not yet seen complete
    const uint32_t idesc = tf32_idesc(kTcModes, 2 * kTcModes);
    // epilogue role of the thread: warp (lane quarter, column half), lane = pair, columns =
    // the half's 128 taps; it sums every chunk's partials of those columns in registers
    const int er = (warp & 3) * 32 + lane, ehalf = warp >> 2;
    float acc[128];
#pragma unroll
    for (int j = 0; j < 128; ++j) acc[j] = 0.f;
    // adds the completed partial sums of accumulator `buf` (after its completion wait)
    auto drain = [&](int buf) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)buf * kPjCols +
                              (uint32_t)(ehalf * 128);
#pragma unroll
        for (int h = 0; h < 128; h += 16) {
            uint32_t v[16];
            tmem_ld_async(base + (uint32_t)h, v);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[h + j] += __uint_as_float(v[j]);
        }
    };
    // A: a thread takes four units of (pair row r, 4 consecutive modes from k4); the eight
    // lanes of a quarter-warp hold eight consecutive rows, so their 16-byte stores land in
    // distinct bank groups of the core layout.  The next chunk's values are loaded into
    // registers while the current chunk's MMAs run.
    float pre[4][4];
    auto load_a = [&](int c) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int U = tid + kPjThreads * i;
            const int r = (U & 7) + 8 * (U >> 6), k4 = ((U >> 3) & 7) * 4;
            const int p = pbase + r;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int m = 32 * c + k4 + j;
                pre[i][j] = (p < npairs && m < a.NH) ? __ldg(&Q[(int64_t)p * a.NH + m]) : 0.f;
            }
        }
    };
    if (nmc > 0) load_a(0);
    for (int c = 0; c < nmc; ++c) {
        const int st = c & 1;
        unsigned char *Ahi = smem + st * kPjStage, *Alo = Ahi + kPjA, *Bhi = Ahi + 2 * kPjA, *Blo = Bhi + kPjB;
        if (c >= 2) {  // the MMAs of chunk c - 2 read this stage and wrote this accumulator
            if (ok) {
                ok = mbar_wait(bar_s + 8u * st, (ph >> st) & 1);
                if (ok) pend &= ~(1u << st);
            }
            ph ^= 1u << st;
            if (ok) drain(st);
        }
        // B: the chunk's cosine tile (hi then lo, 64 KiB)
        const float *src = ctabP + (size_t)c * 2 * 8192;
        for (int e = tid; e < 4096; e += kPjThreads) cp_async16(Bhi + 16 * e, src + 4 * e, 16);
        cp_async_commit();
        // A: the Q rows of the block's pairs at the chunk's 32 modes, split hi / lo
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int U = tid + kPjThreads * i;
            const int r = (U & 7) + 8 * (U >> 6), k4 = ((U >> 3) & 7) * 4;
            float4 hi4, lo4;
            float *hp = &hi4.x, *lp = &lo4.x;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                hp[j] = tf32_round(pre[i][j]);
                lp[j] = tf32_round(pre[i][j] - hp[j]);
            }
            const uint32_t off = core_offset(r, k4);
            *reinterpret_cast<float4 *>(Ahi + off) = hi4;
            *reinterpret_cast<float4 *>(Alo + off) = lo4;
        }
        if (c + 1 < nmc) load_a(c + 1);
        asm volatile("cp.async.wait_all;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        // the accumulator's reads (drain) are ordered before the MMAs that overwrite it
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        ok = __syncthreads_and(ok);
        // CTA-uniform: the MMAs and commit of this chunk are issued (the test knob withholds
        // them, so that the completion wait runs out)
        const bool issued = ok && !a.withhold_mma;
        if (issued) pend |= 1u << st;
        if (tid == 0 && issued) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t sa_hi = (uint32_t)__cvta_generic_to_shared(Ahi);
            const uint32_t sa_lo = (uint32_t)__cvta_generic_to_shared(Alo);
            const uint32_t sb_hi = (uint32_t)__cvta_generic_to_shared(Bhi);
            const uint32_t sb_lo = (uint32_t)__cvta_generic_to_shared(Blo);
            const uint32_t d = tmem + (uint32_t)st * kPjCols;
            for (int ks = 0; ks < 4; ++ks) {
                const uint32_t o = ks * 2 * kLBO;
                mma_tf32(d, smem_desc(sa_hi + o), smem_desc(sb_hi + o), idesc, ks == 0 ? 0 : 1);
                mma_tf32(d, smem_desc(sa_hi + o), smem_desc(sb_lo + o), idesc, 1);
                mma_tf32(d, smem_desc(sa_lo + o), smem_desc(sb_hi + o), idesc, 1);
            }
            mma_commit(bar_s + 8u * st);
        }
    }
    // the last (up to) two chunks
    for (int c = max(0, nmc - 2); c < nmc; ++c) {
        const int st = c & 1;
        if (ok) {
            ok = mbar_wait(bar_s + 8u * st, (ph >> st) & 1);
            if (ok) pend &= ~(1u << st);
        }
        ph ^= 1u << st;
        if (ok) drain(st);
    }
    ok = __syncthreads_and(ok);
    if (!ok && tid == 0) atomicOr(&g_tc_error, 4);
    // after an expired wait: every issued commit not yet seen complete is waited for once more
    // (bounded) before the tensor memory and shared memory its MMAs use are released; a
    // withheld issue left nothing in flight
    if (!ok)
        for (int st = 0; st < 2; ++st)
            if (pend & (1u << st)) (void)mbar_wait(bar_s + 8u * st, (ph >> st) & 1);
    // a pair keeps the half of its own flavour
    {
        const int p = pbase + er;
        const bool pv = ok && p < npairs;
        const int f = pv && a.shift_fix ? a.kd.fl[p] : 0;
        if (pv && f == ehalf) {
            float *xr = X + (int64_t)(p - pfirst) * 128;
#pragma unroll
            for (int j = 0; j < 128; j += 4)
                *reinterpret_cast<float4 *>(xr + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kPjCols));
}

}  // namespace

int contract_tc_kchunks(int max_taps) { return (max_taps + kTcKChunk - 1) / kTcKChunk; }
int contract_tc_modes() { return kTcModes; }

constexpr size_t kTcSmemLimit = 216 * 1024;  // dynamic shared memory of a one-CTA-per-SM launch

// Staging buffers of srows rows for blocks of rb rings in groups of gs.  Two CTAs per SM
// (rb == 8): by default two buffers when they fit in the operand area, else one; `want` (1 or
// 2) overrides when it fits in 200 KiB.  One CTA per SM (rb == 16): two when they fit.
int contract_tc_nbuf(int rb, int gs, int srows, int want)
{
    const size_t row = (size_t)kTcModes * sizeof(float4);
    if (rb == 16) return 2 * srows * row + 32 <= kTcSmemLimit ? 2 : 1;
    if (want == 1) return 1;
    if (want == 2 && 2 * srows * row + 32 <= 200 * 1024) return 2;
    return 2 * srows * row <= (gs == 2 ? TcShape<8, 2>::kAB : TcShape<8, 4>::kAB) ? 2 : 1;
}

size_t contract_tc_smem(int rb, int gs, int srows, int want_nbuf)
{
    const size_t stage_bytes = (size_t)contract_tc_nbuf(rb, gs, srows, want_nbuf) * srows * kTcModes * sizeof(float4);
    const size_t ab_bytes = rb == 16 ? TcShape<16, 2>::kAB : TcShape<8, 2>::kAB;
    return (((stage_bytes > ab_bytes ? stage_bytes : ab_bytes) + 15) & ~size_t(15)) + 32;
}

template <int RB, int G>
cudaError_t launch_tc(const ContractArgs &a, int nchunks, const float *ctab, int nkc_tab, int srows, int nbuf,
                      size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute((const void *)k_contract_tc<RB, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.NH + kTcModes - 1) / kTcModes, (a.nrep + RB - 1) / RB, nchunks);
    k_contract_tc<RB, G><<<grid, TcShape<RB, G>::kThreads, smem, st>>>(a, ctab, nkc_tab, srows, nbuf);
    return cudaGetLastError();
}

cudaError_t launch_contract_tc(const ContractArgs &a, int rb, int gs, int nchunks, const float *ctab, int nkc_tab,
                               int srows, int want_nbuf, cudaStream_t st)
{
    const size_t smem = contract_tc_smem(rb, gs, srows, want_nbuf);
    const int nbuf = contract_tc_nbuf(rb, gs, srows, want_nbuf);
    if (rb == 16)
        return gs == 4 ? launch_tc<16, 4>(a, nchunks, ctab, nkc_tab, srows, nbuf, smem, st)
                       : launch_tc<16, 2>(a, nchunks, ctab, nkc_tab, srows, nbuf, smem, st);
    return gs == 4 ? launch_tc<8, 4>(a, nchunks, ctab, nkc_tab, srows, nbuf, smem, st)
                   : launch_tc<8, 2>(a, nchunks, ctab, nkc_tab, srows, nbuf, smem, st);
}

// Knot-gradient projection of pairs [pfirst, npairs) into X [npairs - pfirst][128] (rows of
// 128 taps of each pair's own flavour); ctabP holds nmc chunks of 32 modes.
cudaError_t launch_knot_proj_tc(const KnotGradArgs &a, const float *Q, const float *ctabP, int nmc, int pfirst,
                                float *X, cudaStream_t st)
{
    const int n = a.kd.npairs - pfirst;
    if (n <= 0) return cudaSuccess;
    const size_t smem = 2 * (size_t)kPjStage + 32;
    cudaError_t e = cudaFuncSetAttribute((const void *)k_knot_proj_tc,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_knot_proj_tc<<<(n + kPjPairs - 1) / kPjPairs, kPjThreads, smem, st>>>(a, Q, ctabP, nmc, pfirst, X);
    return cudaGetLastError();
}

// Host-side reset/readout of the device error word (bounded waits that expired).
cudaError_t take_tc_error(int *out)
{
    int v = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int));
    if (e != cudaSuccess) return e;
    *out = v;
    if (v) {
        const int z = 0;
        e = cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
    }
    return e;
}

}  // namespace arkcos
