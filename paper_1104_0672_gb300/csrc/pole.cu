// Pole-ring correction (Sec. 4.2, last paragraph): the first and last HEALPix ring (4 pixels
// each) are recomputed by the true-profile direct sum s_p = sum_q w_q f(gamma_pq) r_q over
// the input rings inside the support, and the adjoint adds the transposed sum.  FP64 squared
// chords and profile values, FP64 accumulation, deterministic block reductions.
#include "device_common.cuh"

namespace arkcos {

namespace {

// Squared chord between pixel p of ring i and pixel q of ring j (exact longitudes
// pi (2p + hs) / n reduced as rationals before the FP64 sincospi).
__device__ __forceinline__ double pixel_chord2(const RingDev &rd, int i, int p, int j, int q)
{
    const int ni = rd.n[i], nj = rd.n[j];
    const double y = (double)(2 * p + rd.hs[i]) / (2.0 * ni) - (double)(2 * q + rd.hs[j]) / (2.0 * nj);
    double sy, cy;
    sincospi(y, &sy, &cy);  // x/2 = pi y
    const double ti = rd.theta[i], tj = rd.theta[j];
    const double sd = sin(0.5 * (ti - tj)), ss = sin(0.5 * (ti + tj));
    return 4.0 * (sd * sd * cy * cy + ss * ss * sy * sy);
}

__device__ double block_sum(double v, double *red)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    __syncthreads();
    return s;
}

// Direct sum of kernel kd at pixel p of pole ring i over input map mp (this thread's share).
__device__ double pole_sum(const PoleArgs &a, const KernDev &kd, const float *mp, int i, int p, int e)
{
    const int jl = kd.jlo[0], jh = kd.jhi[0];
    double acc = 0.0;
    for (int jj = jl; jj <= jh; ++jj) {
        const int j = e == 0 ? jj : a.R - 1 - jj;
        const int nj = a.rd.n[j];
        const double wj = (double)a.rd.w[j];
        for (int q = threadIdx.x; q < nj; q += blockDim.x) {
            const double u = pixel_chord2(a.rd, i, p, j, q);
            if (u <= kd.umax)
                acc += wj * profile_eval(u, kd.ut, kd.knots, kd.T, kd.gscale) *
                       (double)__ldg(&mp[a.rd.poff[j] + q]);
        }
    }
    return acc;
}

// grid: (pixel p of the pole ring, pole e in {0: ring 0, 1: ring R-1}, map b)
__global__ void __launch_bounds__(256) k_pole_fwd(PoleArgs a)
{
    __shared__ double red[8];
    const int p = blockIdx.x, e = blockIdx.y, b = blockIdx.z;
    const int i = e == 0 ? 0 : a.R - 1;
    if (p >= a.rd.n[i]) return;
    const int src = a.vdiv > 1 ? (a.vbase + b) / a.vdiv : b;
    const float *mp = a.map + (int64_t)src * a.npix;
    double acc = 0.0;
    if (a.nsum > 0) {
        // the weighted sum over several kernels of one input map, in kernel order
        for (int k = 0; k < a.nsum; ++k) acc += a.wsum[k] * block_sum(pole_sum(a, a.kd[k], mp, i, p, e), red);
    } else {
        acc = block_sum(pole_sum(a, a.kd[a.per_map ? b - a.map_base : 0], mp, i, p, e), red);
    }
    if (threadIdx.x == 0) a.out[(int64_t)b * a.npix + a.rd.poff[i] + p] = (float)acc;
}

// grid: (ring index within the pole band, side e, map b); adds the transposed direct sum of
// both pole rings to every pixel of the band rings.
__global__ void __launch_bounds__(256) k_pole_adj(PoleArgs a)
{
    const int jj = blockIdx.x, e = blockIdx.y, b = blockIdx.z;
    const KernDev &kd = a.kd[a.per_map ? b - a.map_base : 0];
    const int jl = kd.jlo[0], jh = kd.jhi[0];
    if (jj > jh - jl) return;
    const int j = e == 0 ? jl + jj : a.R - 1 - (jl + jj);
    // a ring inside both pole bands (tiny grids) is handled once, from the north side
    if (e == 1 && a.R - 1 - j <= jh && j <= jh) return;
    const int nj = a.rd.n[j];
    const double wj = (double)a.rd.w[j];
    const float *g = a.map + (int64_t)b * a.npix;
    float *o = a.out + (int64_t)b * a.npix + a.rd.poff[j];
    for (int q = threadIdx.x; q < nj; q += blockDim.x) {
        double acc = 0.0;
        for (int side = 0; side < 2; ++side) {
            const int i = side == 0 ? 0 : a.R - 1;
            const int jn = side == 0 ? j : a.R - 1 - j;  // distance in rings from that pole
            if (jn < jl || jn > jh) continue;
            for (int p = 0; p < a.rd.n[i]; ++p) {
                const double u = pixel_chord2(a.rd, i, p, j, q);
                if (u <= kd.umax)
                    acc += wj * profile_eval(u, kd.ut, kd.knots, kd.T, kd.gscale) *
                           (double)__ldg(&g[a.rd.poff[i] + p]);
            }
        }
        o[q] += (float)acc;
    }
}

}  // namespace

cudaError_t launch_pole_fwd(const PoleArgs &a, cudaStream_t st)
{
    dim3 grid(4, 2, a.B);
    k_pole_fwd<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pole_adj(const PoleArgs &a, int max_band_rings, cudaStream_t st)
{
    dim3 grid(max_band_rings, 2, a.B);
    k_pole_adj<<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace arkcos
