/*
 * arkcos.h -- C ABI of the GB300 ring-band sphere convolution library (libarkcos.so).
 *
 * The library computes the hybrid Fourier / direct-space convolution of isolatitude-ring
 * sphere maps with a compact radial kernel described in Elsner & Wandelt 2011, "ARKCoS"
 * (Sec. 4): an FFT along every ring, ring-pair kernel Fourier coefficients generated on the
 * fly from the tabulated radial profile (never stored), a contraction over the input rings
 * inside the kernel support, and inverse ring FFTs, plus the adjoint of that operator and
 * its gradient with respect to the profile knots.
 *
 * Conventions shared by every entry point:
 *   - All functions return an arkcos_status; they never throw or abort.  On failure a
 *     thread-local message is available from arkcos_last_error().
 *   - Map and gradient buffers are DEVICE pointers owned by the caller, FP32, laid out as
 *     [nmaps][npix] with pixels in ring order (HEALPix RING ordering; ECP row-major with
 *     theta_r = (r + 1/2) pi / ntheta, phi_k = 2 pi k / nphi), 8-byte aligned (the kernels move
 *     pixel pairs; EINVAL otherwise).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Work is
 *     enqueued on it; the convolution calls do not synchronise the host.
 *   - arkcos_convolve / arkcos_convolve_backward allocate nothing: the caller provides a
 *     device workspace of at least arkcos_workspace_size() bytes (256-byte aligned).
 *   - Handles (grids, kernels) own device tables allocated at creation and freed by the
 *     matching destroy call.  A kernel handle references its grid, which must outlive it.
 *   - Handles are not thread-safe for concurrent mutation; concurrent convolve calls that
 *     use distinct workspaces are fine.
 */
#ifndef ARKCOS_H
#define ARKCOS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct arkcos_grid_s *arkcos_grid;
typedef struct arkcos_kernel_s *arkcos_kernel;

typedef enum {
    ARKCOS_OK = 0,
    ARKCOS_EINVAL = 1,       /* bad argument (null pointer, size, aliasing, range) */
    ARKCOS_ENOMEM = 2,       /* host or device allocation failed at handle creation */
    ARKCOS_ECUDA = 3,        /* a CUDA runtime call failed; message has the CUDA error */
    ARKCOS_EWORKSPACE = 4,   /* workspace missing, misaligned or too small */
    ARKCOS_ETIMEOUT = 5,     /* a bounded device wait expired (reported by sync_status) */
    ARKCOS_EUNSUPPORTED = 6  /* valid request this build does not implement */
} arkcos_status;

/* Option bits for arkcos_convolve / arkcos_convolve_backward / arkcos_workspace_size.
 * flags == 0 selects the paper's default enhanced operator in plain FP32. */
#define ARKCOS_FLAG_BASIC 1u          /* Sec. 4.1 basic variant: zero-padded input spectra and
                                         output truncated at each ring's Nyquist frequency,
                                         instead of the Sec. 4.3 periodic extension / fold */
#define ARKCOS_FLAG_NO_SHIFT_FIX 2u   /* disable the Sec. 4.3 equatorial shift fix (kernel
                                         sampled at phi - phi0 on equal-length ring pairs) */
#define ARKCOS_FLAG_NO_POLE_FIX 4u    /* disable the Sec. 4.2 direct-sum recomputation of the
                                         first and last HEALPix ring */
#define ARKCOS_FLAG_3XTF32 8u         /* generate the ring-pair coefficients on the tensor cores
                                         (tcgen05, 3xTF32 split precision, FP32 accumulation);
                                         bands wider than 32 rings use the FP32 path */

/* HEALPix grid in RING ordering (Sec. 4.1): 4 nside - 1 rings; cap ring i has 4i pixels
 * starting at longitude pi/(4i); equatorial rings have 4 nside pixels, every other one
 * offset by pi/(4 nside).  Ring colatitudes per Gorski et al. 2005.  nside in [1, 8192].
 * Errors: EINVAL (nside out of range, out == NULL), ENOMEM, ECUDA. */
arkcos_status arkcos_create_grid_healpix(int64_t nside, arkcos_grid *out);

/* Equidistant-cylindrical grid (Sec. 4.3, last paragraph): ntheta rings at
 * theta_r = (r + 1/2) pi / ntheta with nphi pixels each, phi_k = 2 pi k / nphi; pixel
 * weights are Fejer first-rule latitude weights times 2 pi / nphi.  nphi must be even.
 * Errors: EINVAL (ntheta < 1, nphi < 2 or odd, sizes above 65536), ENOMEM, ECUDA. */
arkcos_status arkcos_create_grid_ecp(int64_t ntheta, int64_t nphi, arkcos_grid *out);

/* Frees the grid's device tables.  Kernels created on it must be destroyed first.
 * Accepts NULL.  Errors: ECUDA. */
arkcos_status arkcos_destroy_grid(arkcos_grid grid);

/* Number of rings, total pixels and kernel longitude-grid length N (4 nside or nphi).
 * Any output pointer may be NULL.  Errors: EINVAL (grid NULL). */
arkcos_status arkcos_grid_info(arkcos_grid grid, int64_t *nrings, int64_t *npix, int64_t *nlon);

/* Radial profile (Sec. 4.1, the tabulated kernel): HOST array of nknots FP64 values
 * f_t = f(gamma_t) at gamma_t = t * gamma_max / (nknots - 1).  The profile is linear in the
 * squared chord u = 2(1 - cos gamma) between knots (the exact form of Eq. kernel_angle) and
 * zero for gamma > gamma_max.  Builds the ring-pair band tables (which input rings each
 * output ring sees, and how many kernel samples each ring pair has) on the host in FP64 and
 * uploads them.  2 <= nknots <= 4096, 0 < gamma_max <= pi/2.  flags is reserved (pass 0).
 * Errors: EINVAL, ENOMEM, ECUDA. */
arkcos_status arkcos_set_kernel(arkcos_grid grid, const double *knots, int64_t nknots,
                                double gamma_max, uint32_t flags, arkcos_kernel *out);

/* Replaces the knot values of an existing kernel (same nknots and gamma_max), e.g. while
 * fitting a beam.  `knots` is a DEVICE pointer when on_device != 0 (copied on `stream`),
 * else a host pointer (copied synchronously).  Errors: EINVAL, ECUDA. */
arkcos_status arkcos_kernel_update_knots(arkcos_kernel kernel, const double *knots,
                                         int on_device, void *stream);

/* Frees the kernel's device tables.  Accepts NULL.  Errors: ECUDA. */
arkcos_status arkcos_destroy_kernel(arkcos_kernel kernel);

/* Workspace bytes needed by arkcos_convolve (backward = 0) or arkcos_convolve_backward
 * (backward = 1) for `nmaps` maps using the given kernels (nkernels == 1 or nmaps).
 * Errors: EINVAL. */
arkcos_status arkcos_workspace_size(arkcos_grid grid, const arkcos_kernel *kernels,
                                    int64_t nkernels, int64_t nmaps, uint32_t flags,
                                    int backward, size_t *bytes);

/* Forward convolution (Sec. 4.1 steps with the Sec. 4.3 enhancements and the Sec. 4.2 pole
 * fix):  map_out[b] = L(kernel_b) map_in[b] for b < nmaps, where kernel_b = kernels[0] when
 * nkernels == 1 and kernels[b] when nkernels == nmaps.  map_in and map_out are DEVICE FP32
 * [nmaps][npix] and must not overlap.  Enqueued on `stream`; no host synchronisation and
 * no allocation.  Errors: EINVAL (nulls, nmaps < 1, nkernels not 1 or nmaps, kernels of
 * another grid, overlapping maps), EWORKSPACE, EUNSUPPORTED (flag not built), ECUDA (launch
 * failure). */
arkcos_status arkcos_convolve(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                              const float *map_in, float *map_out, int64_t nmaps,
                              void *workspace, size_t ws_bytes, void *stream, uint32_t flags);

/* Adjoint / gradient pass of arkcos_convolve for J = sum_b <grad_out[b], map_out[b]>:
 *   grad_in[b]      = L(kernel_b)^T grad_out[b]            (transposed ring-band sum), and
 *   grad_knots[k][t] = dJ / d f_t of kernel k               (FP64, summed over the maps
 *                                                            that use kernel k).
 * Ring FFTs of map_in are recomputed, not taken from the forward pass.  grad_in (DEVICE FP32
 * [nmaps][npix]) and grad_knots (DEVICE FP64 [nkernels][nknots], overwritten) may each be
 * NULL to skip that output; map_in may be NULL when grad_knots is NULL.  With
 * ARKCOS_FLAG_3XTF32 the transposed contraction and the knot-gradient cosine sums run on the
 * tensor cores (3xTF32, FP32 accumulation); the hat-weight deposits and the reduction over
 * pairs are deterministic (bitwise reproducible) in either form.  Errors as for
 * arkcos_convolve. */
arkcos_status arkcos_convolve_backward(arkcos_grid grid, const arkcos_kernel *kernels,
                                       int64_t nkernels, const float *map_in,
                                       const float *grad_out, float *grad_in,
                                       double *grad_knots, int64_t nmaps, void *workspace,
                                       size_t ws_bytes, void *stream, uint32_t flags);

/* Workspace bytes of arkcos_convolve_multi for nmaps input maps and nkernels kernels, with
 * (weighted != 0) or without the weighted sum.  Errors: EINVAL, EUNSUPPORTED (as
 * arkcos_convolve_multi's argument checks). */
arkcos_status arkcos_multi_workspace_size(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                                          int64_t nmaps, int weighted, uint32_t flags, size_t *bytes);

/* Several radial kernels applied to the same maps (Sec. 5: an asymmetric beam handled as
 * O(10) symmetric convolutions of one input, the decomposition of ASYMFAST; also multi-scale
 * symmetric wavelet analyses).  Every input map is ring-analysed once and its spectra are
 * contracted with the on-the-fly coefficients of each of the nkernels kernels (all created on
 * `grid`):
 *   weights == NULL:  map_out[b][k] = L(kernels[k]) map_in[b]          ([nmaps][nkernels][npix]);
 *   weights != NULL:  map_out[b] = sum_k weights[k] L(kernels[k]) map_in[b]   ([nmaps][npix]),
 *                     weights a HOST array of nkernels FP64 values (used as FP32), the sum
 *                     formed on the kernel-grid coefficients in kernel order before one
 *                     inverse ring transform per map (the pole rings sum the kernels' direct
 *                     sums the same way).
 * map_in and map_out are DEVICE FP32 and must not overlap.  1 <= nkernels <= 256 (32 with
 * weights), nmaps x nkernels <= 256.  The workspace (DEVICE, 256-byte aligned) holds at least
 * arkcos_multi_workspace_size() bytes.  Enqueued on `stream`, no host synchronisation, no
 * allocation.  Errors: EINVAL, EUNSUPPORTED, EWORKSPACE, ECUDA as arkcos_convolve. */
arkcos_status arkcos_convolve_multi(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                                    const double *weights, const float *map_in, float *map_out, int64_t nmaps,
                                    void *workspace, size_t ws_bytes, void *stream, uint32_t flags);

/* One convolution of a batch job: maps of one grid with one shared kernel or one per map. */
typedef struct {
    arkcos_grid grid;
    const arkcos_kernel *kernels; /* nkernels == 1 or nmaps, all created on `grid` */
    int64_t nkernels;
    const float *map_in;          /* DEVICE [nmaps][npix of grid] */
    float *map_out;               /* DEVICE [nmaps][npix of grid] */
    int64_t nmaps;
    uint32_t flags;
} arkcos_job;

/* Workspace bytes for arkcos_convolve_batch (the jobs' forward workspaces, each 256-byte
 * aligned, laid end to end).  Errors: EINVAL. */
arkcos_status arkcos_batch_workspace_size(const arkcos_job *jobs, int64_t njobs, size_t *bytes);

/* Batched forward convolution of maps on grids of different resolutions (the batching form of
 * the spec workload: many maps of mixed nside, each with its own beam): every job is
 * validated first, then all are enqueued back to back on `stream` with disjoint parts of the
 * workspace, so the whole batch is one stream-ordered sequence of kernel launches with no host
 * synchronisation and no allocation -- one CUDA-graph capture of this call replays the batch
 * with a single graph launch.  Errors: as arkcos_convolve for any job (nothing is enqueued
 * when validation fails), EWORKSPACE. */
arkcos_status arkcos_convolve_batch(const arkcos_job *jobs, int64_t njobs, void *workspace,
                                    size_t ws_bytes, void *stream);

/* Autotuning of launch shapes (no counterpart in the paper; the tile choice is left open by
 * it): times arkcos_convolve on the caller's buffers with every candidate shape -- how many
 * CTAs share the maps of a ring pair in the ring FFTs (1x, 2x, 4x, 8x, 16x the default split), for a
 * shared beam how many maps one contraction CTA takes (all, half, a quarter) -- three runs
 * each, and keeps the fastest for this (grid, kernels, nmaps, flags); later arkcos_convolve
 * calls with the same arguments use it (the choice is dropped with the grid).  Every shape
 * computes bitwise the same result.  map_out is overwritten; `stream` is synchronised; not
 * for stream capture.  With ARKCOS_FLAG_3XTF32 the form of the tensor-core contraction is a
 * third choice: a thread takes a group of 2 or 4 output rings, a CTA a block of 8 rings (two
 * CTAs per SM) or 16 (one CTA per SM, two staging buffers) -- 1 / 2 = blocks of 8, groups of 2,
 * one / two staging buffers; 3 = blocks of 16, groups of 2; 4 / 5 = blocks of 8 / 16, groups of
 * 4 (when the union band of every 4 rings fits 32 input rings); 0 = the default (for one
 * shared kernel form 5 where it fits, else blocks of 8 in groups of 2; for per-map kernels
 * form 4 where it fits, else 1).  out (HOST int64[5], nullable) receives the FFT split
 * multiplier, the maps per contraction CTA, the number of candidates, the best time in
 * microseconds and the contraction form.
 * Errors: as arkcos_convolve. */
arkcos_status arkcos_autotune(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                              const float *map_in, float *map_out, int64_t nmaps, void *workspace,
                              size_t ws_bytes, void *stream, uint32_t flags, int64_t *out);

/* Installs a launch shape for later arkcos_convolve calls with these (grid, kernels, nmaps,
 * flags), in place of an autotuned or default one (no counterpart in the paper): shape (HOST
 * int64[3]) = the FFT split multiplier (1, 2, 4, 8 or 16), the maps per contraction CTA for a shared
 * beam (0 = all; ignored for per-map kernels) and the tensor-core contraction form (0..5, as
 * arkcos_autotune reports it; ignored without ARKCOS_FLAG_3XTF32; a form whose tiles do not fit
 * the kernels falls back as the default does).  Every shape computes bitwise the same result.
 * Errors: as arkcos_convolve's argument checks, EINVAL (shape NULL or a value out of range). */
arkcos_status arkcos_set_launch_shape(arkcos_grid grid, const arkcos_kernel *kernels, int64_t nkernels,
                                      int64_t nmaps, uint32_t flags, const int64_t *shape);

/* Device workspace bytes of arkcos_convolve_host for nmaps maps in chunks of maps_per_chunk:
 * two input and two output chunk buffers plus the forward workspace of one chunk.
 * Errors: EINVAL (as arkcos_workspace_size; maps_per_chunk < 1). */
arkcos_status arkcos_host_workspace_size(arkcos_grid grid, const arkcos_kernel *kernels,
                                         int64_t nkernels, int64_t nmaps, int64_t maps_per_chunk,
                                         uint32_t flags, size_t *bytes);

/* arkcos_convolve on HOST buffers (the end-to-end form of the Sec. 4 convolution; the paper
 * has no separate counterpart): host_in and host_out are HOST FP32 [nmaps][npix], pinned
 * (page-locked) for the copies to overlap -- pageable buffers work but serialise.  The maps go
 * in chunks of maps_per_chunk (the first and the last chunk half as large, since nothing
 * overlaps the first upload and the last download): the upload of chunk c + 1 and the
 * download of chunk c - 1 run on two internal streams while chunk c is convolved on `stream`,
 * with the chunk buffers of `workspace` (DEVICE, 256-byte aligned, >= arkcos_host_workspace_size
 * bytes) double-buffered.  With one shared kernel its samples and polar table are computed
 * once, by the first chunk.
 * Everything is ordered after the work already on `stream`, and `stream` is ordered after the
 * last download: host_out is complete when the stream reaches that point.  The caller keeps
 * host_in, host_out and workspace alive until then.  Not for stream capture (the internal
 * streams and events are created per call).  Errors: as arkcos_convolve, EINVAL (host_in or
 * host_out NULL or overlapping, maps_per_chunk < 1), EWORKSPACE, ECUDA. */
arkcos_status arkcos_convolve_host(arkcos_grid grid, const arkcos_kernel *kernels,
                                   int64_t nkernels, const float *host_in, float *host_out,
                                   int64_t nmaps, int64_t maps_per_chunk, void *workspace,
                                   size_t ws_bytes, void *stream, uint32_t flags);

/* Allocation-free variant of arkcos_convolve (no counterpart in the paper).  For callers that
 * cannot pass a device workspace -- e.g. a host program whose device memory belongs to another
 * framework's pool, or a loop that must not call cudaMalloc, which can synchronise the device,
 * while it runs.  Same arguments and result as arkcos_convolve, minus the workspace: the
 * scratch is a fixed 32 MiB device array inside the library, which every GPU that loads the
 * library reserves until the process exits.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress, with the device current), so make the first call on
 * each device before any stream capture.  That address is kept for the life of the process
 * and does not survive cudaDeviceReset: do not use this entry point on a device after resetting
 * it.  The entry point allocates no device memory.  All calls share the one array and it keeps
 * the last call's contents (nothing in it needs to start at zero): calls whose work overlaps on
 * the GPU -- e.g. on two streams at once -- race and corrupt each other; serialise them.
 * Errors: as arkcos_convolve, plus EWORKSPACE (with a message) when the call needs more than
 * 32 MiB of scratch (arkcos_workspace_size), e.g. a single HEALPix map at nside 1024. */
arkcos_status arkcos_convolve_static(arkcos_grid grid, const arkcos_kernel *kernels,
                                     int64_t nkernels, const float *map_in, float *map_out,
                                     int64_t nmaps, void *stream, uint32_t flags);

/* Ring analysis alone (Sec. 4.1, first step): spec_out[b] receives, for every ring j in order,
 * the half spectrum a_m(j) = sum_q r_jq exp(-i m phi_jq), m = 0..n_j/2, as interleaved FP32
 * (re, im) pairs -- sum_j (n_j/2 + 1) complex values per map.  DEVICE buffers, no allocation.
 * Errors: EINVAL (nulls, nmaps < 1), ECUDA. */
arkcos_status arkcos_ring_analysis(arkcos_grid grid, const float *map_in, float *spec_out,
                                   int64_t nmaps, void *stream);

/* Ring synthesis alone (Sec. 4.1 last step with the Sec. 4.3 fold): coeffs[b][i][m], m = 0..N/2,
 * interleaved FP32 (re, im), are the kernel-grid Fourier coefficients c_m of output ring i; the
 * ring receives s_ip = sum'_{|m|<=N/2} c_m exp(i m phi_ip) (sum' halves |m| = N/2; c_{-m} =
 * conj c_m; only Re c_0 is used, as the rings are real), or with ARKCOS_FLAG_BASIC only
 * |m| <= n_i/2 with the ring-Nyquist terms halved.
 * DEVICE buffers, no allocation.  Errors: EINVAL, ECUDA. */
arkcos_status arkcos_ring_synthesis(arkcos_grid grid, const float *coeffs, float *map_out,
                                    int64_t nmaps, uint32_t flags, void *stream);

/* Ring-pair statistics of a kernel: representative ring pairs (N-S mirror pairs counted once),
 * in-support kernel samples over those pairs (with the equatorial shift fix, each sample
 * counted once for +k and -k), and the largest number of input rings one output ring sees.
 * Any output may be NULL.  Errors: EINVAL. */
arkcos_status arkcos_kernel_info(arkcos_kernel kernel, int64_t *pairs, int64_t *samples,
                                 int64_t *max_band);

/* Per-stage device timing (instrumentation, not part of the computation).  While enabled,
 * every arkcos_convolve / arkcos_convolve_backward call records a CUDA event pair around each
 * of its stages on its stream and counts the kernels each stage launches; this creates CUDA
 * events (host-side driver objects) but no device memory.  enable != 0 turns it on and clears
 * the records; 0 turns it off.  Errors: none. */
arkcos_status arkcos_stage_timing(int enable);

/* Totals since arkcos_stage_timing(1) for stage index `stage` (0-based; returns EINVAL past the
 * last stage): its name, summed milliseconds (synchronises on the recorded events), number of
 * recorded executions of the stage and total kernel launches in it.  Stages: "taps",
 * "fft_fwd", "contract", "fft_inv", "pole", "pole_adj", "knot_q", "knot_proj", "knot_pole",
 * "knot_reduce".  Errors: EINVAL, ECUDA. */
arkcos_status arkcos_stage_report(int64_t stage, const char **name, double *ms,
                                  int64_t *executions, int64_t *launches);

/* Stream-ordered status check: synchronises `stream` and reports device-side failures
 * recorded by earlier calls on it (bounded waits that expired -> ETIMEOUT, CUDA errors ->
 * ECUDA).  Clears the recorded device error.  Errors: ETIMEOUT, ECUDA.
 * Every wait of the tensor-core kernels (ARKCOS_FLAG_3XTF32) on the completion of their own
 * MMAs gives up after about one second; the kernel then records the error, issues no further
 * MMA, waits once more (bounded) for any MMA it did issue, frees its tensor memory and returns,
 * and the outputs of that call are invalid.  To exercise this path without a fault, set the
 * environment variable ARKCOS_TEST_WITHHOLD_MMA to 1 (read on every call): the tensor-core
 * kernels then issue no MMA at all, so their waits run out with nothing in flight. */
arkcos_status arkcos_sync_status(void *stream);

/* Thread-local description of the last error returned on this thread ("" if none). */
const char *arkcos_last_error(void);

/* Library version string. */
const char *arkcos_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ARKCOS_H */
