/*
 * Plain FP64 CPU oracle for the ARKCoS hybrid Fourier / direct-space radial
 * kernel convolution of isolatitude-ring sphere maps (Elsner & Wandelt 2011,
 * "ARKCoS", Sections 2-4).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; it has its own ring geometry, its own
 * kernel-profile lookup and its own naive DFTs.
 *
 * Every step is written as the plain definition, in the order of the paper's
 * Section 4.1, with no blocking or fusion:
 *   (1) ring DFT  a_m(j) = sum_q r_jq exp(-i m phi_jq)            (Sec. 4.1, Eq. fftrot)
 *   (2) kernel samples on the N-point longitude grid and their DFT
 *       kappa_m(i,j) = (1/N) sum_k K_k exp(-2 pi i m k / N)        (Sec. 4.1, Eq. kernel_angle)
 *   (3) ring-pair sum c_m(i) = sum_j w_j kappa_m e^{-i m delta} a_m(j)
 *   (4) synthesis s_ip = Re sum'_m c_m(i) exp(i m phi_ip)          (Sec. 4.1 / 4.3)
 *   (5) pole-ring direct-sum fix                                     (Sec. 4.2, last paragraph)
 * Readings of the paper used here (all stated in the design notes):
 *   - direct sum carries pixel weights: s_p = sum_q w_q f(gamma_pq) r_q (Sec. 2 Eq. def, Sec. 3.1 Eq. direct);
 *   - the squared chord u = 2(1 - cos gamma) is the exact form of Eq. kernel_angle;
 *     the profile is tabulated at gamma_t = t*gamma_max/(T-1) and K(u) is linear in u
 *     between u_t = 4 sin^2(gamma_t/2); K = 0 for u > u_max (Sec. 4.1, bias-compensated table);
 *   - ENHANCED variant (default): the input spectrum is the periodic extension of
 *     each ring's DFT to |m| <= N/2 and the output sums all |m| <= N/2 (Sec. 4.3);
 *     the equatorial shift fix samples the kernel at phi - phi0 for equal-length ring
 *     pairs (delta_ij = phi0_i - phi0_j) and applies no phase there (Sec. 4.3);
 *   - BASIC variant: input truncated at |m| <= n_j/2 and output at |m| <= n_i/2, with the
 *     ring-Nyquist terms halved (Sec. 4.1, zero padding and Nyquist truncation);
 *   - sum' halves the |m| = N/2 terms (trigonometric interpolation of the N samples).
 * Parity status: the BASIC variant's polar caps have no independent closed form
 * ("parity unpinned" beyond the oracle's own brute-force restatement).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_HEALPIX 0
#define OR_ECP 1

/* option bits understood by this oracle (its own definitions) */
#define OR_OPT_BASIC 1u       /* BASIC variant instead of ENHANCED */
#define OR_OPT_NO_SHIFT 2u    /* disable the equatorial shift fix */
#define OR_OPT_NO_POLE 4u     /* disable the pole-ring direct sum */

typedef struct {
    int kind;
    long R;      /* number of rings */
    long N;      /* kernel longitude grid length (4 nside, or nphi) */
    long npix;
    double *theta, *phi0, *w;
    long *n, *off;
} ogeom;

typedef struct {
    long T;
    const double *f;
    double *u;
    double umax;
} okern;

static void ogeom_free(ogeom *g)
{
    free(g->theta); free(g->phi0); free(g->w); free(g->n); free(g->off);
    memset(g, 0, sizeof(*g));
}

/* HEALPix ring geometry (Gorski et al. 2005, as cited in Sec. 4.1): 2(nside-1) cap
 * rings with 4i pixels and first-pixel longitude pi/(4i); 2nside+1 equatorial rings
 * with 4nside pixels, offset pi/(4nside) on every other ring.  Equal pixel areas.
 * ECP: theta_r = (r+1/2) pi / ntheta, nphi pixels per ring starting at phi = 0,
 * Fejer first-rule latitude weights times 2 pi / nphi. */
static int ogeom_init(ogeom *g, int kind, long a, long b)
{
    memset(g, 0, sizeof(*g));
    g->kind = kind;
    if (kind == OR_HEALPIX) {
        long ns = a;
        if (ns < 1) return -1;
        g->R = 4 * ns - 1;
        g->N = 4 * ns;
    } else if (kind == OR_ECP) {
        if (a < 1 || b < 2 || (b % 2)) return -1;
        g->R = a;
        g->N = b;
    } else {
        return -1;
    }
    long R = g->R;
    g->theta = malloc(R * sizeof(double));
    g->phi0 = malloc(R * sizeof(double));
    g->w = malloc(R * sizeof(double));
    g->n = malloc(R * sizeof(long));
    g->off = malloc((R + 1) * sizeof(long));
    if (kind == OR_HEALPIX) {
        long ns = a;
        double npix = 12.0 * (double)ns * (double)ns;
        for (long r = 1; r <= R; ++r) {
            long k = r - 1;
            if (r < ns) {
                g->n[k] = 4 * r;
                g->theta[k] = 2.0 * asin((double)r / (sqrt(6.0) * (double)ns));
                g->phi0[k] = M_PI / (4.0 * (double)r);
            } else if (r <= 3 * ns) {
                g->n[k] = 4 * ns;
                g->theta[k] = acos(4.0 / 3.0 - 2.0 * (double)r / (3.0 * (double)ns));
                g->phi0[k] = ((r - ns) % 2 == 0) ? M_PI / (4.0 * (double)ns) : 0.0;
            } else {
                long i = 4 * ns - r;
                g->n[k] = 4 * i;
                g->theta[k] = M_PI - 2.0 * asin((double)i / (sqrt(6.0) * (double)ns));
                g->phi0[k] = M_PI / (4.0 * (double)i);
            }
            g->w[k] = 4.0 * M_PI / npix;
        }
    } else {
        long nt = a, np = b;
        for (long r = 0; r < R; ++r) {
            double th = (r + 0.5) * M_PI / (double)nt;
            double s = 0.0;
            for (long j = 1; j <= nt / 2; ++j)
                s += cos(2.0 * j * th) / (4.0 * (double)j * (double)j - 1.0);
            g->theta[r] = th;
            g->n[r] = np;
            g->phi0[r] = 0.0;
            g->w[r] = (2.0 / (double)nt) * (1.0 - 2.0 * s) * (2.0 * M_PI / (double)np);
        }
    }
    g->off[0] = 0;
    for (long r = 0; r < R; ++r) g->off[r + 1] = g->off[r] + g->n[r];
    g->npix = g->off[R];
    return 0;
}

static int okern_init(okern *k, const double *f, long T, double gmax)
{
    if (T < 2 || !(gmax > 0.0) || gmax > M_PI) return -1;
    k->T = T;
    k->f = f;
    k->u = malloc(T * sizeof(double));
    for (long t = 0; t < T; ++t) {
        double g = gmax * (double)t / (double)(T - 1);
        double s = sin(0.5 * g);
        k->u[t] = 4.0 * s * s;
    }
    k->umax = k->u[T - 1];
    return 0;
}

static void okern_free(okern *k) { free(k->u); k->u = NULL; }

/* Tabulated radial profile as a function of the squared chord u (linear in u between
 * knots, zero beyond the support). */
static double okern_eval(const okern *k, double u)
{
    if (u > k->umax) return 0.0;
    long T = k->T;
    if (u >= k->u[T - 1]) return k->f[T - 1];
    long lo = 0, hi = T - 1;
    while (hi - lo > 1) {
        long mid = (lo + hi) / 2;
        if (k->u[mid] <= u) lo = mid; else hi = mid;
    }
    double lam = (u - k->u[lo]) / (k->u[hi] - k->u[lo]);
    return k->f[lo] + lam * (k->f[hi] - k->f[lo]);
}

/* d K(u) / d f_t as the pair (t0, 1-lam), (t0+1, lam); returns t0 or -1 outside support. */
static long okern_hat(const okern *k, double u, double *lam_out)
{
    if (u > k->umax) return -1;
    long T = k->T;
    if (u >= k->u[T - 1]) { *lam_out = 1.0; return T - 2; }
    long lo = 0, hi = T - 1;
    while (hi - lo > 1) {
        long mid = (lo + hi) / 2;
        if (k->u[mid] <= u) lo = mid; else hi = mid;
    }
    *lam_out = (u - k->u[lo]) / (k->u[hi] - k->u[lo]);
    return lo;
}

/* Squared chord between (theta_a, 0) and (theta_b, x): the exact form of the paper's
 * Eq. kernel_angle, 2(1 - cos gamma) = 4[sin^2(dtheta/2) cos^2(x/2) + sin^2(stheta/2) sin^2(x/2)]. */
static double ochord2(double ta, double tb, double x)
{
    double sd = sin(0.5 * (ta - tb)), ss = sin(0.5 * (ta + tb));
    double cx = cos(0.5 * x), sx = sin(0.5 * x);
    return 4.0 * (sd * sd * cx * cx + ss * ss * sx * sx);
}

static long omod(long a, long n) { long r = a % n; return r < 0 ? r + n : r; }

/* Offset between rings used in the kernel sampling (Sec. 4.3 equatorial fix). */
static double odelta(const ogeom *g, long i, long j, unsigned opt)
{
    if ((opt & OR_OPT_NO_SHIFT) || g->n[i] != g->n[j]) return 0.0;
    return g->phi0[i] - g->phi0[j];
}

/* Step (1): a_m(j) = sum_q r_jq exp(-i m phi_jq), phi_jq = phi0_j + 2 pi q / n_j, for
 * m = 0..M (M = N/2).  For m > n_j/2 this is the periodic extension the ENHANCED
 * variant uses; BASIC weights it by the trigonometric-interpolation window.  Negative
 * m follow by conjugation (real input). */
static void oring_dft(const ogeom *g, long j, const double *map, long M, unsigned opt, double *out)
{
    long n = g->n[j];
    const double *r = map + g->off[j];
    double *ct = malloc(n * sizeof(double)), *st = malloc(n * sizeof(double));
    for (long t = 0; t < n; ++t) {
        ct[t] = cos(2.0 * M_PI * (double)t / (double)n);
        st[t] = sin(2.0 * M_PI * (double)t / (double)n);
    }
    for (long m = 0; m <= M; ++m) {
        double re = 0.0, im = 0.0;
        for (long q = 0; q < n; ++q) {
            long t = (m * q) % n;
            re += r[q] * ct[t];
            im -= r[q] * st[t];
        }
        double c = cos((double)m * g->phi0[j]), s = sin((double)m * g->phi0[j]);
        double ore = re * c + im * s, oim = im * c - re * s;
        if (opt & OR_OPT_BASIC) {
            double h = 1.0;
            if (2 * m > n) h = 0.0;
            else if (2 * m == n && n < g->N) h = 0.5;
            ore *= h; oim *= h;
        }
        out[2 * m] = ore;
        out[2 * m + 1] = oim;
    }
    free(ct); free(st);
}

/* Which rings lie inside the kernel support of ring i (|theta_i - theta_j| <= gamma_max). */
static int oin_band(const ogeom *g, long i, long j, double gmax)
{
    return fabs(g->theta[i] - g->theta[j]) <= gmax;
}

/* Step (2): kappa_m(i,j) for m = -N/2..N/2 (index m + N/2), from the N kernel samples
 * at x_k = delta + 2 pi k / N; samples outside the support are zero and skipped. */
static void okappa(const ogeom *g, const okern *kn, long i, long j, double delta,
                   const double *cN, const double *sN, double *kre, double *kim,
                   long *kidx, double *kval)
{
    long N = g->N, nz = 0;
    for (long k = 0; k < N; ++k) {
        double x = delta + 2.0 * M_PI * (double)k / (double)N;
        double v = okern_eval(kn, ochord2(g->theta[i], g->theta[j], x));
        if (v != 0.0) { kidx[nz] = k; kval[nz] = v; ++nz; }
    }
    for (long m = -N / 2; m <= N / 2; ++m) {
        double re = 0.0, im = 0.0;
        for (long z = 0; z < nz; ++z) {
            long t = omod(m * kidx[z], N);
            re += kval[z] * cN[t];
            im -= kval[z] * sN[t];
        }
        kre[m + N / 2] = re / (double)N;
        kim[m + N / 2] = im / (double)N;
    }
}

/* True-profile direct sum (Sec. 3.1 Eq. direct with pixel weights) for one output pixel. */
static double odirect_pixel(const ogeom *g, const okern *kn, const double *map, long i, long p)
{
    double phip = g->phi0[i] + 2.0 * M_PI * (double)p / (double)g->n[i];
    double gmax = 2.0 * asin(0.5 * sqrt(kn->umax));
    double acc = 0.0;
    for (long j = 0; j < g->R; ++j) {
        if (!oin_band(g, i, j, gmax + 1e-12)) continue;
        const double *r = map + g->off[j];
        for (long q = 0; q < g->n[j]; ++q) {
            double phiq = g->phi0[j] + 2.0 * M_PI * (double)q / (double)g->n[j];
            double v = okern_eval(kn, ochord2(g->theta[i], g->theta[j], phip - phiq));
            acc += g->w[j] * v * r[q];
        }
    }
    return acc;
}

static int opole_fixed(const ogeom *g, long i, unsigned opt)
{
    return g->kind == OR_HEALPIX && !(opt & OR_OPT_NO_POLE) && (i == 0 || i == g->R - 1);
}

/* Per-output-ring hybrid result (steps 2-4) written to out (n_i values). */
static void ohybrid_ring(const ogeom *g, const okern *kn, double gmax, unsigned opt,
                         double **ahat, long i, const double *cN, const double *sN, double *out)
{
    long N = g->N, M = N / 2;
    double *cre = calloc(N + 1, sizeof(double)), *cim = calloc(N + 1, sizeof(double));
    double *kre = malloc((N + 1) * sizeof(double)), *kim = malloc((N + 1) * sizeof(double));
    long *kidx = malloc(N * sizeof(long));
    double *kval = malloc(N * sizeof(double));
    for (long j = 0; j < g->R; ++j) {
        if (!oin_band(g, i, j, gmax)) continue;
        double delta = odelta(g, i, j, opt);
        okappa(g, kn, i, j, delta, cN, sN, kre, kim, kidx, kval);
        for (long m = -M; m <= M; ++m) {
            long am = m < 0 ? -m : m;
            double are = ahat[j][2 * am], aim = ahat[j][2 * am + 1];
            if (m < 0) aim = -aim;
            double pc = cos((double)m * delta), ps = -sin((double)m * delta);
            /* w_j * kappa_m * e^{-i m delta} * a_m(j) */
            double tre = kre[m + M] * pc - kim[m + M] * ps;
            double tim = kre[m + M] * ps + kim[m + M] * pc;
            cre[m + M] += g->w[j] * (tre * are - tim * aim);
            cim[m + M] += g->w[j] * (tre * aim + tim * are);
        }
    }
    long n = g->n[i];
    long lim = (opt & OR_OPT_BASIC) ? n / 2 : M;
    for (long p = 0; p < n; ++p) {
        double acc = 0.0;
        for (long m = -lim; m <= lim; ++m) {
            double h = (m == lim || m == -lim) ? 0.5 : 1.0;
            double ph = (double)m * g->phi0[i] + 2.0 * M_PI * (double)omod(m * p, n) / (double)n;
            acc += h * (cre[m + M] * cos(ph) - cim[m + M] * sin(ph));
        }
        out[p] = acc;
    }
    free(cre); free(cim); free(kre); free(kim); free(kidx); free(kval);
}

static double **oalloc_ahat(const ogeom *g) { return calloc(g->R, sizeof(double *)); }
static void ofree_ahat(const ogeom *g, double **a)
{
    for (long j = 0; j < g->R; ++j) free(a[j]);
    free(a);
}

static void otables(long N, double **cN, double **sN)
{
    *cN = malloc(N * sizeof(double));
    *sN = malloc(N * sizeof(double));
    for (long t = 0; t < N; ++t) {
        (*cN)[t] = cos(2.0 * M_PI * (double)t / (double)N);
        (*sN)[t] = sin(2.0 * M_PI * (double)t / (double)N);
    }
}

static void oset_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* ---------------------------------------------------------------- public API */

long oracle_nrings(int kind, long a, long b)
{
    ogeom g;
    if (ogeom_init(&g, kind, a, b)) return -1;
    long R = g.R;
    ogeom_free(&g);
    return R;
}

/* Ring table export: theta, phi0, weight, pixel count, first-pixel offset (R entries). */
int oracle_geometry(int kind, long a, long b, double *theta, double *phi0, double *w,
                    long *n, long *off)
{
    ogeom g;
    if (ogeom_init(&g, kind, a, b)) return -1;
    for (long r = 0; r < g.R; ++r) {
        theta[r] = g.theta[r]; phi0[r] = g.phi0[r]; w[r] = g.w[r];
        n[r] = g.n[r]; off[r] = g.off[r];
    }
    ogeom_free(&g);
    return 0;
}

/* Forward operator for one map.  Only the output rings listed in rings[0..nr) are
 * written (all rings if rings == NULL); the input rings they need are transformed. */
int oracle_convolve(int kind, long a, long b, const double *knots, long T, double gmax,
                    unsigned opt, const double *map_in, double *map_out,
                    const long *rings, long nr, int nthreads)
{
    ogeom g;
    okern kn;
    if (ogeom_init(&g, kind, a, b)) return -1;
    if (okern_init(&kn, knots, T, gmax)) { ogeom_free(&g); return -1; }
    oset_threads(nthreads);
    long R = g.R, N = g.N, M = N / 2;
    long nout = rings ? nr : R;
    long *outl = malloc(nout * sizeof(long));
    for (long z = 0; z < nout; ++z) outl[z] = rings ? rings[z] : z;
    char *need = calloc(R, 1);
    for (long z = 0; z < nout; ++z)
        for (long j = 0; j < R; ++j)
            if (oin_band(&g, outl[z], j, gmax)) need[j] = 1;
    long *nl = malloc(R * sizeof(long)), nn = 0;
    for (long j = 0; j < R; ++j) if (need[j]) nl[nn++] = j;
    double **ahat = oalloc_ahat(&g);
    for (long z = 0; z < nn; ++z) ahat[nl[z]] = malloc(2 * (M + 1) * sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (long z = 0; z < nn; ++z) oring_dft(&g, nl[z], map_in, M, opt, ahat[nl[z]]);
    double *cN, *sN;
    otables(N, &cN, &sN);
#pragma omp parallel for schedule(dynamic, 1)
    for (long z = 0; z < nout; ++z) {
        long i = outl[z];
        double *out = map_out + g.off[i];
        if (opole_fixed(&g, i, opt)) {
            for (long p = 0; p < g.n[i]; ++p) out[p] = odirect_pixel(&g, &kn, map_in, i, p);
        } else {
            ohybrid_ring(&g, &kn, gmax, opt, ahat, i, cN, sN, out);
        }
    }
    free(cN); free(sN);
    ofree_ahat(&g, ahat);
    free(nl); free(need); free(outl);
    okern_free(&kn);
    ogeom_free(&g);
    return 0;
}

/* True-profile direct sum for every pixel of the listed output rings (a reference
 * the hybrid matches exactly on ECP grids and on equal-length HEALPix ring pairs). */
int oracle_direct(int kind, long a, long b, const double *knots, long T, double gmax,
                  const double *map_in, double *map_out, const long *rings, long nr,
                  int nthreads)
{
    ogeom g;
    okern kn;
    if (ogeom_init(&g, kind, a, b)) return -1;
    if (okern_init(&kn, knots, T, gmax)) { ogeom_free(&g); return -1; }
    oset_threads(nthreads);
    long nout = rings ? nr : g.R;
#pragma omp parallel for schedule(dynamic, 1)
    for (long z = 0; z < nout; ++z) {
        long i = rings ? rings[z] : z;
        for (long p = 0; p < g.n[i]; ++p)
            map_out[g.off[i] + p] = odirect_pixel(&g, &kn, map_in, i, p);
    }
    okern_free(&kn);
    ogeom_free(&g);
    return 0;
}

/* Adjoint of the forward operator (transpose of steps 1-5 taken in reverse order):
 *   g_hat_m(i) = sum_p g_ip exp(-i m phi_ip) with the synthesis window (sum' weights),
 *   abar_m(j)  = sum_i w_j kappa_m(i,j) e^{-i m delta_ij} conj(g_hat_m(i)),
 *   rbar_jq    = Re sum_m abar_m(j) exp(-i m phi_jq) (with the input window for BASIC),
 * plus the transpose of the pole-ring direct sum.  Only the listed input rings are written. */
int oracle_adjoint(int kind, long a, long b, const double *knots, long T, double gmax,
                   unsigned opt, const double *gmap, double *rbar, const long *rings, long nr,
                   int nthreads)
{
    ogeom g;
    okern kn;
    if (ogeom_init(&g, kind, a, b)) return -1;
    if (okern_init(&kn, knots, T, gmax)) { ogeom_free(&g); return -1; }
    oset_threads(nthreads);
    long R = g.R, N = g.N, M = N / 2;
    long nin = rings ? nr : R;
    long *inl = malloc(nin * sizeof(long));
    for (long z = 0; z < nin; ++z) inl[z] = rings ? rings[z] : z;
    char *need = calloc(R, 1);
    for (long z = 0; z < nin; ++z)
        for (long i = 0; i < R; ++i)
            if (oin_band(&g, i, inl[z], gmax) && !opole_fixed(&g, i, opt)) need[i] = 1;
    /* g_hat over m = -M..M including the synthesis window h(m) */
    double **gh = calloc(R, sizeof(double *));
    long *nl = malloc(R * sizeof(long)), nn = 0;
    for (long i = 0; i < R; ++i) if (need[i]) nl[nn++] = i;
#pragma omp parallel for schedule(dynamic, 1)
    for (long z = 0; z < nn; ++z) {
        long i = nl[z], n = g.n[i];
        long lim = (opt & OR_OPT_BASIC) ? n / 2 : M;
        double *o = calloc(2 * (N + 1), sizeof(double));
        const double *gi = gmap + g.off[i];
        for (long m = -lim; m <= lim; ++m) {
            double h = (m == lim || m == -lim) ? 0.5 : 1.0;
            double re = 0.0, im = 0.0;
            for (long p = 0; p < n; ++p) {
                double ph = (double)m * g.phi0[i] + 2.0 * M_PI * (double)omod(m * p, n) / (double)n;
                re += gi[p] * cos(ph);
                im -= gi[p] * sin(ph);
            }
            o[2 * (m + M)] = h * re;
            o[2 * (m + M) + 1] = h * im;
        }
        gh[i] = o;
    }
    double *cN, *sN;
    otables(N, &cN, &sN);
#pragma omp parallel for schedule(dynamic, 1)
    for (long z = 0; z < nin; ++z) {
        long j = inl[z], n = g.n[j];
        double *abr = calloc(N + 1, sizeof(double)), *abi = calloc(N + 1, sizeof(double));
        double *kre = malloc((N + 1) * sizeof(double)), *kim = malloc((N + 1) * sizeof(double));
        long *kidx = malloc(N * sizeof(long));
        double *kval = malloc(N * sizeof(double));
        for (long i = 0; i < R; ++i) {
            if (!gh[i] || !oin_band(&g, i, j, gmax)) continue;
            double delta = odelta(&g, i, j, opt);
            okappa(&g, &kn, i, j, delta, cN, sN, kre, kim, kidx, kval);
            for (long m = -M; m <= M; ++m) {
                double pc = cos((double)m * delta), ps = -sin((double)m * delta);
                double tre = kre[m + M] * pc - kim[m + M] * ps;
                double tim = kre[m + M] * ps + kim[m + M] * pc;
                double gre = gh[i][2 * (m + M)], gim = -gh[i][2 * (m + M) + 1];
                abr[m + M] += g.w[j] * (tre * gre - tim * gim);
                abi[m + M] += g.w[j] * (tre * gim + tim * gre);
            }
        }
        double *out = rbar + g.off[j];
        for (long q = 0; q < n; ++q) {
            double acc = 0.0;
            for (long m = -M; m <= M; ++m) {
                double hw = 1.0;
                if (opt & OR_OPT_BASIC) {
                    long am = m < 0 ? -m : m;
                    if (2 * am > n) hw = 0.0;
                    else if (2 * am == n && n < N) hw = 0.5;
                }
                if (hw == 0.0) continue;
                double ph = -((double)m * g.phi0[j] + 2.0 * M_PI * (double)omod(m * q, n) / (double)n);
                acc += hw * (abr[m + M] * cos(ph) - abi[m + M] * sin(ph));
            }
            out[q] = acc;
        }
        /* transpose of the pole-ring direct sum */
        if (g.kind == OR_HEALPIX && !(opt & OR_OPT_NO_POLE)) {
            long pr[2] = {0, R - 1};
            for (int e = 0; e < 2; ++e) {
                long i = pr[e];
                if (!oin_band(&g, i, j, gmax + 1e-12)) continue;
                for (long p = 0; p < g.n[i]; ++p) {
                    double phip = g.phi0[i] + 2.0 * M_PI * (double)p / (double)g.n[i];
                    double gp = gmap[g.off[i] + p];
                    for (long q = 0; q < n; ++q) {
                        double phiq = g.phi0[j] + 2.0 * M_PI * (double)q / (double)n;
                        out[q] += g.w[j] * okern_eval(&kn, ochord2(g.theta[i], g.theta[j], phip - phiq)) * gp;
                    }
                }
            }
        }
        free(abr); free(abi); free(kre); free(kim); free(kidx); free(kval);
    }
    free(cN); free(sN);
    for (long i = 0; i < R; ++i) free(gh[i]);
    free(gh); free(nl); free(need); free(inl);
    okern_free(&kn);
    ogeom_free(&g);
    return 0;
}

/* Gradient of <g, L r> with respect to the profile knots f_t.  K_k(i,j) is linear in the
 * knots through the hat weights of the lookup, so
 *   d<g,Lr>/dK_k(i,j) = (w_j/N) Re sum'_m e^{-i m x_k} a_m(j) conj(g_hat_m(i)),
 * with x_k = delta_ij + 2 pi k / N and g_hat including the synthesis window; the pole
 * rings contribute through their true-profile direct sum.  Sums over all ring pairs. */
int oracle_knot_grad(int kind, long a, long b, const double *knots, long T, double gmax,
                     unsigned opt, const double *map_in, const double *gmap, double *grad,
                     int nthreads)
{
    ogeom g;
    okern kn;
    if (ogeom_init(&g, kind, a, b)) return -1;
    if (okern_init(&kn, knots, T, gmax)) { ogeom_free(&g); return -1; }
    oset_threads(nthreads);
    long R = g.R, N = g.N, M = N / 2;
    double **ahat = oalloc_ahat(&g);
#pragma omp parallel for schedule(dynamic, 1)
    for (long j = 0; j < R; ++j) {
        ahat[j] = malloc(2 * (M + 1) * sizeof(double));
        oring_dft(&g, j, map_in, M, opt, ahat[j]);
    }
    double **gh = calloc(R, sizeof(double *));
#pragma omp parallel for schedule(dynamic, 1)
    for (long i = 0; i < R; ++i) {
        if (opole_fixed(&g, i, opt)) continue;
        long n = g.n[i];
        long lim = (opt & OR_OPT_BASIC) ? n / 2 : M;
        double *o = calloc(2 * (N + 1), sizeof(double));
        const double *gi = gmap + g.off[i];
        for (long m = -lim; m <= lim; ++m) {
            double h = (m == lim || m == -lim) ? 0.5 : 1.0;
            double re = 0.0, im = 0.0;
            for (long p = 0; p < n; ++p) {
                double ph = (double)m * g.phi0[i] + 2.0 * M_PI * (double)omod(m * p, n) / (double)n;
                re += gi[p] * cos(ph);
                im -= gi[p] * sin(ph);
            }
            o[2 * (m + M)] = h * re;
            o[2 * (m + M) + 1] = h * im;
        }
        gh[i] = o;
    }
    double *cN, *sN;
    otables(N, &cN, &sN);
    for (long t = 0; t < T; ++t) grad[t] = 0.0;
#pragma omp parallel
    {
        double *loc = calloc(T, sizeof(double));
        double *pre = malloc((N + 1) * sizeof(double)), *pim = malloc((N + 1) * sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (long i = 0; i < R; ++i) {
            if (!gh[i]) continue;
            for (long j = 0; j < R; ++j) {
                if (!oin_band(&g, i, j, gmax)) continue;
                double delta = odelta(&g, i, j, opt);
                for (long m = -M; m <= M; ++m) {
                    long am = m < 0 ? -m : m;
                    double are = ahat[j][2 * am], aim = ahat[j][2 * am + 1];
                    if (m < 0) aim = -aim;
                    double gre = gh[i][2 * (m + M)], gim = -gh[i][2 * (m + M) + 1];
                    pre[m + M] = are * gre - aim * gim;
                    pim[m + M] = are * gim + aim * gre;
                }
                for (long k = 0; k < N; ++k) {
                    double x = delta + 2.0 * M_PI * (double)k / (double)N;
                    double u = ochord2(g.theta[i], g.theta[j], x);
                    double lam;
                    long t0 = okern_hat(&kn, u, &lam);
                    if (t0 < 0) continue;
                    double X = 0.0;
                    for (long m = -M; m <= M; ++m) {
                        double pc = cos((double)m * delta), ps = -sin((double)m * delta);
                        long tt = omod(m * k, N);
                        double ere = cN[tt] * pc + sN[tt] * ps;   /* e^{-i m x_k} real part */
                        double eim = -sN[tt] * pc + cN[tt] * ps;  /* imaginary part */
                        X += ere * pre[m + M] - eim * pim[m + M];
                    }
                    X *= g.w[j] / (double)N;
                    loc[t0] += (1.0 - lam) * X;
                    loc[t0 + 1] += lam * X;
                }
            }
        }
        if (g.kind == OR_HEALPIX && !(opt & OR_OPT_NO_POLE)) {
            long pr[2] = {0, R - 1};
#pragma omp for schedule(dynamic, 1)
            for (long e = 0; e < 2; ++e) {
                long i = pr[e];
                for (long p = 0; p < g.n[i]; ++p) {
                    double phip = g.phi0[i] + 2.0 * M_PI * (double)p / (double)g.n[i];
                    double gp = gmap[g.off[i] + p];
                    for (long j = 0; j < R; ++j) {
                        if (!oin_band(&g, i, j, gmax + 1e-12)) continue;
                        for (long q = 0; q < g.n[j]; ++q) {
                            double phiq = g.phi0[j] + 2.0 * M_PI * (double)q / (double)g.n[j];
                            double lam;
                            long t0 = okern_hat(&kn, ochord2(g.theta[i], g.theta[j], phip - phiq), &lam);
                            if (t0 < 0) continue;
                            double X = g.w[j] * gp * map_in[g.off[j] + q];
                            loc[t0] += (1.0 - lam) * X;
                            loc[t0 + 1] += lam * X;
                        }
                    }
                }
            }
        }
#pragma omp critical
        for (long t = 0; t < T; ++t) grad[t] += loc[t];
        free(loc); free(pre); free(pim);
    }
    free(cN); free(sN);
    for (long i = 0; i < R; ++i) free(gh[i]);
    free(gh);
    ofree_ahat(&g, ahat);
    okern_free(&kn);
    ogeom_free(&g);
    return 0;
}
