// Tensor-core form of the ring-pair coefficient generation (3xTF32 on tcgen05), fused with
// the band contraction.
//
// For a block of 8 representative output rings x 128 modes the coefficients are a dense
// product  rho[m, pair] = sum_k C_f[m, k] T[k, pair]  with C_f[m, k] = cos(pi m (2k + f) / N)
// (f = the pair's sample offset, see contract.cu) and T the FP32 kernel samples.  The CTA
// stages C (an exact FP64 table split into TF32 hi + lo parts, prepared per grid in the
// tensor-core layout) and T (split into hi + lo on the fly) in shared memory and one thread
// issues tcgen05.mma kind::tf32 with the accumulator in tensor memory:
//     D = C_hi T_hi + C_hi T_lo + C_lo T_hi      (3xTF32, FP32 accumulation).
// Pairs of the two offsets accumulate into the same columns with the other offset's samples
// zeroed.  Each warp then reads its 32 modes x 32 pairs of D with tcgen05.ld, and the band
// contraction proceeds as in the CUDA-core fast path.  Waits on the MMA completion barrier
// are bounded: on expiry the kernel records an error (reported by arkcos_sync_status) and
// still frees its tensor memory.
#include <stdint.h>

#include "device_common.cuh"

namespace arkcos {

__device__ int g_tc_error = 0;

namespace {

constexpr int kTcModes = 128;          // M of the MMA: modes per CTA (TMEM lanes)
constexpr int kTcRings = 8;            // representative output rings per CTA
constexpr int kTcBand = 32;            // pair slots per output ring (columns per ring)
constexpr int kTcN = kTcRings * kTcBand;  // 256 = N of the MMA
constexpr int kTcKChunk = 32;          // taps per shared-memory chunk (4 MMA K-steps of 8)
constexpr int kTcTmemCols = 256;
constexpr uint32_t kTcTimeout = 1u << 16;  // polls of the completion barrier before giving up

// no-swizzle K-major tensor-core layout: 8-row x 16-byte core matrices, contiguous; core
// matrices adjacent in K are 128 bytes apart (LBO), adjacent in M/N 1024 bytes apart (SBO)
constexpr uint32_t kLBO = 128, kSBO = 1024;

__device__ __forceinline__ uint32_t core_offset(int row, int k)
{
    return (uint32_t)((row >> 3) * kSBO + (k >> 2) * kLBO + (row & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    return d;                // base offset 0, no swizzle
}

// kind::tf32 instruction descriptor: FP32 accumulator, TF32 A and B, both K-major.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ float tf32_round(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase)
{
    for (uint32_t it = 0; it < kTcTimeout; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(mbar), "r"(phase) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}


__global__ void __launch_bounds__(kTcModes *kTcRings, 1)
k_contract_tc(ContractArgs a, const float *__restrict__ ctab, int nkc_tab, int max_union)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    // A hi | A lo (16 KiB each) and B hi | B lo (32 KiB each), then reused for the
    // staged spectra; the last 16 bytes hold the mbarrier and the tensor-memory address
    const size_t stage_bytes = 2 * (size_t)max_union * kTcModes * sizeof(float4);
    const size_t ab_bytes = 2 * 16384 + 2 * (size_t)kTcN / 8 * kSBO;
    const size_t ctl = ((stage_bytes > ab_bytes ? stage_bytes : ab_bytes) + 15) & ~size_t(15);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + ctl);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + ctl + 8);
    unsigned char *Ahi = smem, *Alo = smem + 16384;
    unsigned char *Bhi = smem + 32768, *Blo = Bhi + kTcN / 8 * kSBO;
    float4 *sh4 = reinterpret_cast<float4 *>(smem);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q4 = warp & 3, li = warp >> 2;  // lane quarter of TMEM, output ring
    const int mrow = q4 * 32 + lane;           // mode within the block
    const int m = blockIdx.x * kTcModes + mrow;
    const bool mv = m < a.NH;
    const int r0 = blockIdx.y * kTcRings;
    const int nr = min(kTcRings, a.nrep - r0);
    const bool lv = li < nr;
    const int b0 = blockIdx.z * a.maps_per_chunk;
    const int b1 = min(a.B, b0 + a.maps_per_chunk);
    const int kid = a.per_map ? (b0 - a.map_base) : 0;
    const KernDev &kd = a.kd[kid];
    const float *taps = a.taps[kid];
    const int i = r0 + (lv ? li : 0);
    const int jl = kd.jlo[i];
    const int blen = lv ? kd.jhi[i] - jl + 1 : 0;
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
    __shared__ int s_toff[kTcN], s_S[kTcN], s_f[kTcN];
    if (tid < 2) s_kmax[tid] = 0;
    __syncthreads();
    for (int c = tid; c < kTcN; c += blockDim.x) {
        const int l = c / kTcBand, s = c % kTcBand;
        int toff = 0, S = -1, f = 0;
        if (l < nr && s <= kd.jhi[r0 + l] - kd.jlo[r0 + l]) {
            const int p = kd.pstart[r0 + l] + s;
            f = a.shift_fix ? kd.fl[p] : 0;
            S = f ? kd.S1[p] : kd.S0[p];
            toff = kd.toff[p];
            atomicMax(&s_kmax[f], S + 1);
        }
        s_toff[c] = toff;
        s_S[c] = S;
        s_f[c] = f;
    }
    __syncthreads();
    const int kmax0 = s_kmax[0], kmax1 = s_kmax[1];
    const int kcap = nkc_tab * kTcKChunk;  // samples the cosine table covers
    const bool use_tc = kmax0 <= kcap && kmax1 <= kcap;
    float rho[32];
#pragma unroll
    for (int s = 0; s < 32; ++s) rho[s] = 0.f;
    if (use_tc) {
        // once any CTA has seen an expired wait the results are invalid anyway: skip the MMAs
        bool ok = *((volatile int *)&g_tc_error) == 0;
        ok = __syncthreads_and(ok);
        uint32_t phase = 0;
        bool first = true;  // meaningful in the issuing thread only
        const uint32_t idesc = tf32_idesc(kTcModes, kTcN);
        for (int f = 0; f < 2; ++f) {
            const int kf = f ? kmax1 : kmax0;
            for (int kc = 0; kc * kTcKChunk < kf; ++kc) {
                const int ksteps = min(4, (kf - kc * kTcKChunk + 7) / 8);
                // A: this mode block's cosine chunk (hi, lo), prepared in the core layout
                const float4 *src = reinterpret_cast<const float4 *>(
                    ctab + ((((size_t)blockIdx.x * 2 + f) * nkc_tab + kc) * 2) * 4096);
                float4 *dstA = reinterpret_cast<float4 *>(Ahi);
                for (int e = tid; e < 2 * 1024; e += blockDim.x) dstA[e] = __ldg(&src[e]);
                // B: samples of every pair slot of the block for this flavour (others zero)
                for (int e = tid; e < kTcN * kTcKChunk; e += blockDim.x) {
                    const int c = e / kTcKChunk, k = e % kTcKChunk;
                    const int kk = kc * kTcKChunk + k;
                    float v = 0.f;
                    if (s_f[c] == f && kk <= s_S[c]) v = __ldg(&taps[s_toff[c] + kk]);
                    const float hi = tf32_round(v);
                    const float lo = tf32_round(v - hi);
                    const uint32_t off = core_offset(c, k);
                    *reinterpret_cast<float *>(Bhi + off) = hi;
                    *reinterpret_cast<float *>(Blo + off) = lo;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (tid == 0 && ok) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa_hi = (uint32_t)__cvta_generic_to_shared(Ahi);
                    const uint32_t sa_lo = (uint32_t)__cvta_generic_to_shared(Alo);
                    const uint32_t sb_hi = (uint32_t)__cvta_generic_to_shared(Bhi);
                    const uint32_t sb_lo = (uint32_t)__cvta_generic_to_shared(Blo);
                    for (int ks = 0; ks < ksteps; ++ks) {
                        const uint32_t o = ks * 2 * kLBO;  // 8 TF32 values = two core columns
                        mma_tf32(tmem, smem_desc(sa_hi + o), smem_desc(sb_hi + o), idesc, first ? 0 : 1);
                        mma_tf32(tmem, smem_desc(sa_hi + o), smem_desc(sb_lo + o), idesc, 1);
                        mma_tf32(tmem, smem_desc(sa_lo + o), smem_desc(sb_hi + o), idesc, 1);
                        first = false;
                    }
                    mma_commit(mbar_s);
                }
                // every thread waits for the MMAs before the next chunk reuses shared memory;
                // a wait that expires is recorded, retried once, and stops further MMAs
                if (ok) {
                    bool done = mbar_wait(mbar_s, phase);
                    if (!done) done = mbar_wait(mbar_s, phase);
                    ok = done;
                }
                ok = __syncthreads_and(ok);
                if (!ok && tid == 0) atomicOr(&g_tc_error, 1);
                phase ^= 1;
            }
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // ---- this thread's 32 coefficients from tensor memory (warp-collective load)
        if ((kmax0 + kmax1) > 0 && ok)
            tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(li * kTcBand), rho);
    } else {
        // blocks next to the poles have more samples per pair than the table holds: generate
        // their coefficients on the CUDA cores
        const int ps = kd.pstart[i];
#pragma unroll
        for (int s = 0; s < kTcBand; ++s) {
            if (s < blen && mv) {
                const int p = ps + s;
                const int f = a.shift_fix ? kd.fl[p] : 0;
                const int S = f ? kd.S1[p] : kd.S0[p];
                rho[s] = gen_rho(reinterpret_cast<const float4 *>(taps + kd.toff[p]), S, f, m, a.N);
            }
        }
    }
    if (!mv || !lv) {
#pragma unroll
        for (int s = 0; s < 32; ++s) rho[s] = 0.f;
    }
    const int joff = jl - ju0;
    __syncthreads();

    // ---- band contraction, as in the CUDA-core fast path (double-buffered async staging)
    const int mid = (a.R - 1) / 2;
    const bool crosses = ju0 + nu - 1 > mid;
    const int sstar = mid - jl + 1;
    const size_t bufsz = (size_t)nu * kTcModes;
    const int m0 = blockIdx.x * kTcModes;
    if (b0 < b1) stage_band_async(sh4, a.spec4 + (int64_t)b0 * a.nrep * a.NH, ju0, nu, m0, kTcModes, a.R, a.NH);
    for (int b = b0; b < b1; ++b) {
        const int cur = (b - b0) & 1;
        if (b + 1 < b1)
            stage_band_async(sh4 + (cur ^ 1) * bufsz, a.spec4 + (int64_t)(b + 1) * a.nrep * a.NH, ju0, nu, m0,
                             kTcModes, a.R, a.NH);
        else
            cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        if (lv && mv) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 *col = sh4 + cur * bufsz + joff * kTcModes + mrow;
            if (!crosses) {
#pragma unroll
                for (int s = 0; s < kTcBand; ++s) {
                    if (s < blen) {
                        const float4 v = col[s * kTcModes];
                        acc.x = fmaf(rho[s], v.x, acc.x);
                        acc.y = fmaf(rho[s], v.y, acc.y);
                        acc.z = fmaf(rho[s], v.z, acc.z);
                        acc.w = fmaf(rho[s], v.w, acc.w);
                    }
                }
            } else {
#pragma unroll
                for (int s = 0; s < kTcBand; ++s) {
                    if (s < blen) {
                        float4 v = col[s * kTcModes];
                        if (s >= sstar) v = make_float4(v.z, v.w, v.x, v.y);
                        acc.x = fmaf(rho[s], v.x, acc.x);
                        acc.y = fmaf(rho[s], v.y, acc.y);
                        acc.z = fmaf(rho[s], v.z, acc.z);
                        acc.w = fmaf(rho[s], v.w, acc.w);
                    }
                }
            }
            const int im = a.R - 1 - i;
            a.c[((int64_t)b * a.R + i) * a.NH + m] = make_float2(acc.x, acc.y);
            if (im != i) a.c[((int64_t)b * a.R + im) * a.NH + m] = make_float2(acc.z, acc.w);
        }
        __syncthreads();
    }

    // ---- release tensor memory
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols));
}

}  // namespace

int contract_tc_kchunks(int max_taps) { return (max_taps + kTcKChunk - 1) / kTcKChunk; }
int contract_tc_modes() { return kTcModes; }

size_t contract_tc_smem(int max_union)
{
    const size_t stage_bytes = 2 * (size_t)max_union * kTcModes * sizeof(float4);
    const size_t ab_bytes = 2 * 16384 + 2 * (size_t)kTcN / 8 * kSBO;
    return (((stage_bytes > ab_bytes ? stage_bytes : ab_bytes) + 15) & ~size_t(15)) + 16;
}

cudaError_t launch_contract_tc(const ContractArgs &a, int nchunks, const float *ctab, int nkc_tab,
                               int max_union, cudaStream_t st)
{
    const size_t smem = contract_tc_smem(max_union);
    cudaError_t e = cudaFuncSetAttribute((const void *)k_contract_tc,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((a.NH + kTcModes - 1) / kTcModes, (a.nrep + kTcRings - 1) / kTcRings, nchunks);
    k_contract_tc<<<grid, kTcModes * kTcRings, smem, st>>>(a, ctab, nkc_tab, max_union);
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
