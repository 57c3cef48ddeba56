/*
 * bisp_oracle.c -- plain FP64 CPU oracle for the FFT estimator of the
 * redshift-space bispectrum multipoles B_l^m(k1, mu, t) of Gill & Bharadwaj,
 * "Brisk estimator for the angular multipoles of the redshift space
 * bispectrum" (arXiv:2405.14513).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or constant with the CUDA implementation; both sides see the
 * same seeded input fields and nothing else.
 *
 * Everything here is the plain definition written out in double precision,
 * on the full N_g x N_g plane, enumerating every ordered plane pair (n1, n2)
 * with both signs (no half-space folding, no coarse grids, no fusion):
 *
 *   forward transform   Delta(k) = (V / N_g^3) sum_x delta(x) exp(-i k.x),
 *                       Delta(0) = 0                      (Sec. II, Eq. bs)
 *   rings               widths 2^floor((r-1)/10) grid units from radius 0,
 *                       outer radius capped at N_g/3          (Sec. II)
 *   D fields            D(r,n,x) = sum_{u in r} Delta(u,n) exp(-i u.x)
 *                                                             (Eq. iFT)
 *   unit fields         I(r,x)   = sum_{u in r} exp(-i u.x)  (Eq. 2FT)
 *   triangle counts     N_tri = N_g^-2 sum_x I1 I2 I3 (Eq. Ntri2), or the
 *                       direct count (Eq. Ntri1)
 *   per combination     S = sum_x D1 D2 D3 (Eq. fftbs: Bhat = S/(V N_tri N_g^2)),
 *                       or N_g^2 sum_{u,v,w} Delta Delta Delta delta_K(u+v+w)
 *                       (Eq. binbs)
 *   shape, orientation  t = k2/k1, mu = -k1.k2/(k1 k2) (Eq. shape); p from
 *                       mu_1 = p_z, mu_2 = -mu p_z + sqrt(1-mu^2) p_x
 *                       (Eq. orient)
 *   multipoles          B_l^m = sqrt((2l+1)/4pi) sum Y* Bhat N_tri /
 *                       sum |Y|^2 N_tri                       (Eq. bs_lm2_1)
 *
 * Readings where the paper is silent (each one is listed with its reason in
 * the design notes of the repository):
 *   - ring r is {u : e_{r-1} <= |u| < e_r}, e_0 = 0, the last ring is cut at
 *     N_g/3; its radius k_perp,r is the mean of |u| over its modes;
 *   - planes |n| <= floor(N_g/3); k1 edges must lie at or below (N_g/3) k_f,
 *     so every side of every accepted triangle is alias free;
 *   - a combination is accepted when N_tri > 0, K1 >= K2 >= K3 > 0 with
 *     K_i^2 = k_perp,ri^2 + n_i^2 (grid units), and K1 falls in a k1 bin;
 *     ties are accepted once per valid labelling;
 *   - mu = (K1^2+K2^2-K3^2)/(2 K1 K2), which lies in [1/2, 1] when
 *     K1 >= K2 >= K3 (clamped there against rounding); t = K2/K1;
 *   - mu and t bins are uniform on [0.5, 1]: bin j holds
 *     1/2 + j/(2n) <= x < 1/2 + (j+1)/(2n), top edge closed; t < 0.5 is
 *     dropped;
 *   - the two chiralities (p_y = +/-) of every combination are averaged;
 *     p_y = +sqrt(max(0, 1 - p_z^2 - p_x^2)); for mu >= 1 - 1e-12 the
 *     azimuth is undefined and Y* is averaged over it;
 *   - Y_l^m is orthonormal with the Condon-Shortley phase;
 *   - empty bins are reported as NaN.
 *
 * Built with -ffp-contract=off so that every floating-point operation is the
 * IEEE operation written here, on every host.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define BO_MAX_RINGS 256
#define BO_TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------------ */
/* Parameters of one estimate.                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    int ng;                  /* grid points per side                         */
    double box_len;          /* L; V = L^3, k_f = 2 pi / L                   */
    int n_k1;                /* number of k1 bins                            */
    const double *k1_edges;  /* n_k1 + 1 ascending edges (same units as k_f) */
    int n_mu, n_t;           /* uniform bins on [0.5, 1]                     */
    int l_max;               /* moments 0 <= m <= l <= l_max (all l)          */
    int mode;                /* 0: FFT form (Eqs. fftbs, Ntri2); 1: direct    */
                             /*    sums (Eqs. binbs, Ntri1)                   */
    int nthreads;            /* OpenMP threads, 0 = default                  */
} bo_desc;

static void set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* One-dimensional DFT, X_k = sum_j x_j exp(-2 pi i j k / n).                */
/* Radix-2 decimation in time for powers of two, the defining sum otherwise. */
/* ------------------------------------------------------------------------ */
static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static void dft_definition(cplx *x, int n, cplx *tmp)
{
    for (int k = 0; k < n; ++k) {
        cplx s = 0;
        for (int j = 0; j < n; ++j) {
            long jk = ((long)j * k) % n;
            double a = -BO_TWO_PI * (double)jk / (double)n;
            s += x[j] * (cos(a) + I * sin(a));
        }
        tmp[k] = s;
    }
    memcpy(x, tmp, sizeof(cplx) * (size_t)n);
}

static void fft_radix2(cplx *x, int n)
{
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2;
        for (int k = 0; k < half; ++k) {
            double a = -BO_TWO_PI * (double)k / (double)len;
            cplx w = cos(a) + I * sin(a);
            for (int s = 0; s < n; s += len) {
                cplx u = x[s + k], v = x[s + k + half] * w;
                x[s + k] = u + v;
                x[s + k + half] = u - v;
            }
        }
    }
}

/* n = 3 m, m a power of two: the sum over j split by j mod 3,
 * X_k = sum_{q=0..2} exp(-2 pi i q k / n) F_q(k mod m), F_q the m-point DFT
 * of x_{3j+q}. */
static void fft_radix3_2(cplx *x, int n, cplx *tmp)
{
    const int m = n / 3;
    for (int q = 0; q < 3; ++q) {
        for (int j = 0; j < m; ++j) tmp[q * m + j] = x[3 * j + q];
        fft_radix2(tmp + q * m, m);
    }
    for (int k = 0; k < n; ++k) {
        cplx s = tmp[k % m];
        for (int q = 1; q < 3; ++q) {
            double a = -BO_TWO_PI * (double)((q * k) % n) / (double)n;
            s += (cos(a) + I * sin(a)) * tmp[q * m + k % m];
        }
        x[k] = s;
    }
}

static void dft1(cplx *x, int n, cplx *tmp)
{
    if (is_pow2(n)) fft_radix2(x, n);
    else if (n % 3 == 0 && is_pow2(n / 3)) fft_radix3_2(x, n, tmp);
    else dft_definition(x, n, tmp);
}

/* In-place DFT of n-point lines with the given stride; nlines lines start at
 * base + line_offset(l). */
static void dft_lines(cplx *a, int n, long stride, long nlines,
                      long (*offset)(long, int), int ng)
{
#pragma omp parallel
    {
        cplx *buf = malloc(sizeof(cplx) * (size_t)n);
        cplx *tmp = malloc(sizeof(cplx) * (size_t)n);
#pragma omp for schedule(static)
        for (long l = 0; l < nlines; ++l) {
            long o = offset(l, ng);
            for (int j = 0; j < n; ++j) buf[j] = a[o + j * stride];
            dft1(buf, n, tmp);
            for (int j = 0; j < n; ++j) a[o + j * stride] = buf[j];
        }
        free(buf);
        free(tmp);
    }
}

static long off_z(long l, int ng) { return l * ng; }                       /* lines along z: (x,y) */
static long off_y(long l, int ng) { return (l / ng) * (long)ng * ng + (l % ng); } /* along y: (x,z) */
static long off_x(long l, int ng) { (void)ng; return l; }                  /* along x: (y,z) */
static long off_row(long l, int ng) { return l * ng; }                     /* 2D rows */
static long off_col(long l, int ng) { (void)ng; return l; }                /* 2D columns */

/* Forward 3D DFT of a real field delta[x][y][z] (z fastest), n^3 points. */
static void dft3(cplx *a, int ng)
{
    long ng2 = (long)ng * ng;
    dft_lines(a, ng, 1, ng2, off_z, ng);
    dft_lines(a, ng, ng, ng2, off_y, ng);
    dft_lines(a, ng, ng2, ng2, off_x, ng);
}

/* Forward 2D DFT of an ng x ng plane p[a][b] (b fastest). */
static void dft2(cplx *p, int ng)
{
    dft_lines(p, ng, 1, ng, off_row, ng);
    dft_lines(p, ng, ng, ng, off_col, ng);
}

/* exported: forward DFT of one line (for pinning the transform itself) */
void bo_dft(double *re_im, int n)
{
    cplx *x = malloc(sizeof(cplx) * (size_t)n), *tmp = malloc(sizeof(cplx) * (size_t)n);
    for (int j = 0; j < n; ++j) x[j] = re_im[2 * j] + I * re_im[2 * j + 1];
    dft1(x, n, tmp);
    for (int j = 0; j < n; ++j) { re_im[2 * j] = creal(x[j]); re_im[2 * j + 1] = cimag(x[j]); }
    free(x);
    free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Rings (Sec. II): width 2^floor((r-1)/10) grid units, starting at radius 0, */
/* outer radius capped at N_g/3.  Edges are kept as 3*e_r, which are exact    */
/* integers, so membership e_{r-1} <= |u| < e_r is the integer test           */
/* (3 e_{r-1})^2 <= 9 |u|^2 < (3 e_r)^2.                                      */
/* ------------------------------------------------------------------------ */
static int ring_edges3(int ng, long *e3)
{
    int r = 0;
    e3[0] = 0;
    while (e3[r] < ng) {
        ++r;
        if (r >= BO_MAX_RINGS) return -1;
        long w = 3L << ((r - 1) / 10);
        e3[r] = (e3[r - 1] + w < ng) ? e3[r - 1] + w : ng;
    }
    return r;
}

static int ring_of(int nr, const long *e3, long i, long j)
{
    long q9 = 9 * (i * i + j * j);
    for (int r = 0; r < nr; ++r)
        if (e3[r] * e3[r] <= q9 && q9 < e3[r + 1] * e3[r + 1]) return r;
    return -1;
}

typedef struct {
    int ng, nr, nz;
    long e3[BO_MAX_RINGS + 1];
    double kperp[BO_MAX_RINGS];   /* mode-averaged |u|, grid units */
    long count[BO_MAX_RINGS];
    int *ringidx;                 /* [(i+h)*ng + (j+h)], -1 outside rings */
} rings_t;

static int rings_build(int ng, rings_t *R)
{
    int h = ng / 2;
    R->ng = ng;
    R->nz = ng / 3;
    R->nr = ring_edges3(ng, R->e3);
    if (R->nr < 0) return -1;
    R->ringidx = malloc(sizeof(int) * (size_t)ng * ng);
    double sum[BO_MAX_RINGS];
    for (int r = 0; r < R->nr; ++r) { sum[r] = 0; R->count[r] = 0; }
    for (long i = -h; i < h; ++i)
        for (long j = -h; j < h; ++j) {
            int r = ring_of(R->nr, R->e3, i, j);
            R->ringidx[(i + h) * ng + (j + h)] = r;
            if (r >= 0) { sum[r] += sqrt((double)(i * i + j * j)); R->count[r] += 1; }
        }
    for (int r = 0; r < R->nr; ++r)
        R->kperp[r] = R->count[r] > 0 ? sum[r] / (double)R->count[r]
                                      : 0.5 * (double)(R->e3[r] + R->e3[r + 1]) / 3.0;
    return 0;
}

static int rings_at(const rings_t *R, long i, long j)
{
    int h = R->ng / 2;
    if (i < -h || i >= h || j < -h || j >= h) return -1;
    return R->ringidx[(i + h) * R->ng + (j + h)];
}

static long signed_freq(long a, int ng) { return a < ng / 2 ? a : a - ng; }

/* exported: ring table.  edges3 gets nr+1 entries (3 x edge radius in grid
 * units); kperp and count get nr entries.  Returns nr. */
int bo_rings(int ng, long *edges3, double *kperp, long *count)
{
    rings_t R;
    if (ng < 4 || rings_build(ng, &R)) return -1;
    for (int r = 0; r <= R.nr; ++r) edges3[r] = R.e3[r];
    for (int r = 0; r < R.nr; ++r) { kperp[r] = R.kperp[r]; count[r] = R.count[r]; }
    free(R.ringidx);
    return R.nr;
}

/* ------------------------------------------------------------------------ */
/* Forward transform of the data cube (Sec. II): Delta(k) = (V/N_g^3) DFT,   */
/* with Delta(0) = 0 (the mean density carries no triangle).                 */
/* out: complex [ng][ng][ng] (kx, ky, kz FFT-index order, kz fastest).        */
/* ------------------------------------------------------------------------ */
static cplx *forward_cube(int ng, double box_len, const double *delta)
{
    long n3 = (long)ng * ng * ng;
    cplx *a = malloc(sizeof(cplx) * (size_t)n3);
    if (!a) return NULL;
    for (long i = 0; i < n3; ++i) a[i] = delta[i];
    dft3(a, ng);
    double V = box_len * box_len * box_len;
    double s = V / (double)n3;
    for (long i = 0; i < n3; ++i) a[i] *= s;
    a[0] = 0;
    return a;
}

int bo_forward(int ng, double box_len, const double *delta, double *out_re_im)
{
    cplx *a = forward_cube(ng, box_len, delta);
    if (!a) return -1;
    long n3 = (long)ng * ng * ng;
    for (long i = 0; i < n3; ++i) { out_re_im[2 * i] = creal(a[i]); out_re_im[2 * i + 1] = cimag(a[i]); }
    free(a);
    return 0;
}

/* Plane n of the transformed cube (kz = n mod ng), ring-masked, then the 2D
 * sum of Eq. iFT.  out[x][y] (y fastest). */
static void dfield_from_cube(const rings_t *R, const cplx *cube, int r, int n, cplx *out)
{
    int ng = R->ng;
    long kz = ((n % ng) + ng) % ng;
    for (long a = 0; a < ng; ++a)
        for (long b = 0; b < ng; ++b) {
            int q = rings_at(R, signed_freq(a, ng), signed_freq(b, ng));
            out[a * ng + b] = (q == r) ? cube[(a * ng + b) * ng + kz] : 0;
        }
    dft2(out, ng);
}

/* Unit field of Eq. 2FT: the same sum with Delta = 1 on the ring. */
static void ifield(const rings_t *R, int r, cplx *out)
{
    int ng = R->ng;
    for (long a = 0; a < ng; ++a)
        for (long b = 0; b < ng; ++b)
            out[a * ng + b] = (rings_at(R, signed_freq(a, ng), signed_freq(b, ng)) == r) ? 1.0 : 0.0;
    dft2(out, ng);
}

/* exported: D(r, n, x) for one ring and plane of a field (Eq. iFT). */
int bo_dfield(int ng, double box_len, const double *delta, int r, int n, double *out_re_im)
{
    rings_t R;
    if (rings_build(ng, &R)) return -1;
    cplx *cube = forward_cube(ng, box_len, delta);
    cplx *d = malloc(sizeof(cplx) * (size_t)ng * ng);
    dfield_from_cube(&R, cube, r, n, d);
    for (long i = 0; i < (long)ng * ng; ++i) { out_re_im[2 * i] = creal(d[i]); out_re_im[2 * i + 1] = cimag(d[i]); }
    free(d);
    free(cube);
    free(R.ringidx);
    return 0;
}

/* exported: D(r, n, x) of Eq. iFT at the M x M points x = (N_g/M) y, y
 * integer: sum over the ring's members u of Delta(u, n) exp(-2 pi i u.y / M),
 * summed directly (one axis after the other) for any M >= 1.  out [M][M][2]. */
int bo_dfield_at(int ng, double box_len, const double *delta, int r, int n, int M, double *out_re_im)
{
    if (M < 1) return -1;
    rings_t R;
    if (rings_build(ng, &R)) return -1;
    cplx *cube = forward_cube(ng, box_len, delta);
    long kz = ((n % ng) + ng) % ng;
    /* e[a][y] = exp(-2 pi i u_a y / M), u_a the signed frequency of index a */
    cplx *e = malloc(sizeof(cplx) * (size_t)ng * M);
    for (long a = 0; a < ng; ++a)
        for (long y = 0; y < M; ++y) {
            double ph = -BO_TWO_PI * (double)((signed_freq(a, ng) * y) % M) / (double)M;
            e[a * M + y] = cos(ph) + I * sin(ph);
        }
    cplx *t = calloc((size_t)ng * M, sizeof(cplx));     /* t[a][y_y] */
    for (long a = 0; a < ng; ++a)
        for (long b = 0; b < ng; ++b) {
            if (rings_at(&R, signed_freq(a, ng), signed_freq(b, ng)) != r) continue;
            cplx v = cube[(a * ng + b) * ng + kz];
            for (long y = 0; y < M; ++y) t[a * M + y] += v * e[b * M + y];
        }
    for (long yx = 0; yx < M; ++yx)
        for (long yy = 0; yy < M; ++yy) {
            cplx s = 0;
            for (long a = 0; a < ng; ++a) s += e[a * M + yx] * t[a * M + yy];
            out_re_im[2 * (yx * M + yy)] = creal(s);
            out_re_im[2 * (yx * M + yy) + 1] = cimag(s);
        }
    free(t);
    free(e);
    free(cube);
    free(R.ringidx);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Triangle counts: Eq. Ntri2 (FFT of unit fields) or Eq. Ntri1 (count).     */
/* table[(r1*nr + r2)*nr + r3].                                              */
/* ------------------------------------------------------------------------ */
static double ntri_fft(const rings_t *R, long *table)
{
    int ng = R->ng, nr = R->nr;
    long np = (long)ng * ng;
    cplx *If = malloc(sizeof(cplx) * (size_t)nr * np);
    for (int r = 0; r < nr; ++r) ifield(R, r, If + r * np);
    double worst = 0;
    /* N_tri is symmetric in its three rings: evaluate r1 <= r2 <= r3 only */
#pragma omp parallel for schedule(dynamic) reduction(max : worst)
    for (long t = 0; t < (long)nr * nr * nr; ++t) {
        int r1 = (int)(t / ((long)nr * nr)), r2 = (int)((t / nr) % nr), r3 = (int)(t % nr);
        if (!(r1 <= r2 && r2 <= r3)) continue;
        const cplx *a = If + r1 * np, *b = If + r2 * np, *c = If + r3 * np;
        cplx s = 0;
        for (long x = 0; x < np; ++x) s += a[x] * b[x] * c[x];
        double v = creal(s) / (double)np;
        double rv = nearbyint(v);
        double res = fabs(v - rv) + fabs(cimag(s)) / (double)np;
        if (res > worst) worst = res;
        const int p[6][3] = {{r1, r2, r3}, {r1, r3, r2}, {r2, r1, r3}, {r2, r3, r1}, {r3, r1, r2}, {r3, r2, r1}};
        for (int q = 0; q < 6; ++q) table[((long)p[q][0] * nr + p[q][1]) * nr + p[q][2]] = (long)rv;
    }
    free(If);
    return worst;
}

typedef struct { int n; long *i; long *j; } members_t;

static void members_build(const rings_t *R, members_t *m)
{
    int ng = R->ng, h = ng / 2;
    for (int r = 0; r < R->nr; ++r) {
        m[r].n = 0;
        m[r].i = malloc(sizeof(long) * (size_t)(R->count[r] + 1));
        m[r].j = malloc(sizeof(long) * (size_t)(R->count[r] + 1));
    }
    for (long i = -h; i < h; ++i)
        for (long j = -h; j < h; ++j) {
            int r = rings_at(R, i, j);
            if (r >= 0) { m[r].i[m[r].n] = i; m[r].j[m[r].n] = j; m[r].n++; }
        }
}

static void members_free(const rings_t *R, members_t *m)
{
    for (int r = 0; r < R->nr; ++r) { free(m[r].i); free(m[r].j); }
}

static void ntri_direct(const rings_t *R, long *table)
{
    int nr = R->nr;
    members_t *m = malloc(sizeof(members_t) * (size_t)nr);
    members_build(R, m);
#pragma omp parallel for schedule(dynamic)
    for (long t = 0; t < (long)nr * nr * nr; ++t) {
        int r1 = (int)(t / ((long)nr * nr)), r2 = (int)((t / nr) % nr), r3 = (int)(t % nr);
        long c = 0;
        for (int a = 0; a < m[r1].n; ++a)
            for (int b = 0; b < m[r2].n; ++b)
                if (rings_at(R, -m[r1].i[a] - m[r2].i[b], -m[r1].j[a] - m[r2].j[b]) == r3) ++c;
        table[t] = c;
    }
    members_free(R, m);
    free(m);
}

/* exported: triangle-count table; mode 0 = Eq. Ntri2, 1 = Eq. Ntri1.
 * Returns the largest distance of an Eq. Ntri2 value from its integer
 * (0 for the direct count), or a negative value on error. */
double bo_ntri(int ng, int mode, int nthreads, long *table)
{
    rings_t R;
    set_threads(nthreads);
    if (rings_build(ng, &R)) return -1;
    double worst = 0;
    if (mode == 0) worst = ntri_fft(&R, table);
    else ntri_direct(&R, table);
    free(R.ringidx);
    return worst;
}

/* ------------------------------------------------------------------------ */
/* Spherical harmonics, orthonormal, Condon-Shortley phase.                  */
/* ------------------------------------------------------------------------ */
static double assoc_legendre(int l, int m, double x)
{
    /* P_m^m = (-1)^m (2m-1)!! (1-x^2)^{m/2}; then the upward recurrence in l */
    double pmm = 1.0;
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    for (int k = 1; k <= m; ++k) pmm *= -(2.0 * k - 1.0) * s;
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pm1;
    double p0 = pmm, p1 = pm1, p2 = 0;
    for (int ll = m + 2; ll <= l; ++ll) {
        p2 = ((2.0 * ll - 1.0) * x * p1 - (ll + m - 1.0) * p0) / (double)(ll - m);
        p0 = p1;
        p1 = p2;
    }
    return p2;
}

static double ylm_norm(int l, int m)
{
    double r = 1.0; /* (l-m)!/(l+m)! */
    for (int k = l - m + 1; k <= l + m; ++k) r /= (double)k;
    return sqrt((2.0 * l + 1.0) / (2.0 * BO_TWO_PI) * r);
}

/* Y_l^m at cos(theta) = z and azimuth with (cos phi, sin phi). */
static cplx ylm(int l, int m, double z, double cphi, double sphi)
{
    /* cos(m phi) + i sin(m phi) by repeated multiplication */
    cplx e = 1.0, e1 = cphi + I * sphi;
    for (int k = 0; k < m; ++k) e *= e1;
    return ylm_norm(l, m) * assoc_legendre(l, m, z) * e;
}

/* exported for pinning: Y_l^m(theta, phi) given cos(theta), cos(phi), sin(phi) */
void bo_ylm(int l, int m, double z, double cphi, double sphi, double *re_im)
{
    cplx y = ylm(l, m, z, cphi, sphi);
    re_im[0] = creal(y);
    re_im[1] = cimag(y);
}

static int n_moments_all(int l_max) { return (l_max + 1) * (l_max + 2) / 2; }
static int lm_index(int l, int m) { return l * (l + 1) / 2 + m; }

/* ------------------------------------------------------------------------ */
/* Geometry of one ring/plane combination (Eqs. shape, orient; Sec. II).     */
/* ------------------------------------------------------------------------ */
typedef struct {
    double K1, t, mu, mu1, mu2, mu3;
    double pz, px, py, cphi, sphi;
    int degenerate;
    int ib, im, it;
    int bin;
} geom_t;

/* Inverse of Eq. orient: p_z = mu_1 and, from mu_2 = -mu p_z + sqrt(1-mu^2) p_x,
 * p_x = (mu_2 + mu mu_1) / sqrt(1 - mu^2). */
static void orient_inverse(double mu1, double mu2, double mu, double *pz, double *px)
{
    *pz = mu1;
    *px = (mu2 + mu * mu1) / sqrt(1.0 - mu * mu);
}

/* Bin of x among n uniform bins of [1/2, 1]: bin j holds
 * 1/2 + j/(2n) <= x < 1/2 + (j+1)/(2n), and the top edge x = 1 belongs to
 * the last bin. */
static int half_unit_bin(double x, int n)
{
    int j = 0;
    while (j + 1 < n && 0.5 + (double)(j + 1) / (2.0 * n) <= x) ++j;
    return j;
}

/* Returns 1 when the combination is accepted into a (k1, mu, t) bin. */
static int combo_geometry(const bo_desc *d, double kp1, double kp2, double kp3,
                          int n1, int n2, int n3, geom_t *g)
{
    double k1sq = kp1 * kp1 + (double)n1 * n1;
    double k2sq = kp2 * kp2 + (double)n2 * n2;
    double k3sq = kp3 * kp3 + (double)n3 * n3;
    if (!(k1sq >= k2sq && k2sq >= k3sq && k3sq > 0.0)) return 0;
    double kf = BO_TWO_PI / d->box_len;
    double s1 = sqrt(k1sq), s2 = sqrt(k2sq), s3 = sqrt(k3sq);
    g->K1 = kf * s1;
    int ib = -1;
    for (int b = 0; b < d->n_k1; ++b)
        if (d->k1_edges[b] <= g->K1 && g->K1 < d->k1_edges[b + 1]) { ib = b; break; }
    if (ib < 0 && g->K1 == d->k1_edges[d->n_k1]) ib = d->n_k1 - 1;
    if (ib < 0) return 0;
    g->t = s2 / s1;
    /* law of cosines; sqrt(k1sq*k2sq) is exactly k1sq when the two sides are
     * equal, so equilateral triangles give mu = 1/2 exactly.  With
     * K1 >= K2 >= K3 the value lies in [1/2, 1]; the clamp removes rounding. */
    double mu = (k1sq + k2sq - k3sq) / (2.0 * sqrt(k1sq * k2sq));
    if (mu > 1.0) mu = 1.0;
    if (mu < 0.5) mu = 0.5;
    g->mu = mu;
    if (g->t < 0.5) return 0;
    int it = half_unit_bin(g->t, d->n_t);
    int im = half_unit_bin(g->mu, d->n_mu);
    g->ib = ib;
    g->im = im;
    g->it = it;
    g->bin = (ib * d->n_mu + im) * d->n_t + it;
    g->mu1 = (double)n1 / s1;
    g->mu2 = (double)n2 / s2;
    g->mu3 = (double)n3 / s3;
    g->pz = g->mu1;
    g->degenerate = (mu >= 1.0 - 1e-12);
    if (g->degenerate) {
        g->px = 0;
        g->py = 0;
        g->cphi = 1;
        g->sphi = 0;
    } else {
        orient_inverse(g->mu1, g->mu2, mu, &g->pz, &g->px);
        double q = 1.0 - g->pz * g->pz - g->px * g->px;
        g->py = sqrt(q > 0.0 ? q : 0.0);
        double rho = sqrt(g->px * g->px + g->py * g->py);
        if (rho > 0.0) { g->cphi = g->px / rho; g->sphi = g->py / rho; }
        else { g->cphi = 1.0; g->sphi = 0.0; }
    }
    return 1;
}

/* Chirality-averaged conjugate harmonic of a combination: every combination
 * holds the mirror image (p_y -> -p_y) of each of its triangles, so the
 * weight of Eq. bs_lm2_1 is the mean of Y* over the two; for a linear
 * triangle (undefined azimuth) it is the azimuthal mean of Y*. */
static cplx combo_ystar(int l, int m, const geom_t *g)
{
    if (g->degenerate) return m == 0 ? ylm_norm(l, 0) * assoc_legendre(l, 0, g->pz) : 0.0;
    cplx yp = ylm(l, m, g->pz, g->cphi, g->sphi);
    cplx ym = ylm(l, m, g->pz, g->cphi, -g->sphi);
    return 0.5 * (conj(yp) + conj(ym));
}

static double combo_y2(int l, int m, const geom_t *g)
{
    double p = ylm_norm(l, m) * assoc_legendre(l, m, g->pz);
    return p * p;
}

/* ------------------------------------------------------------------------ */
/* Combination list (every ordered plane pair, both signs).                  */
/* ------------------------------------------------------------------------ */
typedef struct { int n1, n2, n3, r1, r2, r3; long ntri; geom_t g; } combo_t;

static int desc_check(const bo_desc *d)
{
    if (d->ng < 4 || d->box_len <= 0 || d->n_k1 < 1 || !d->k1_edges || d->n_mu < 1 || d->n_t < 1 || d->l_max < 0)
        return -1;
    for (int b = 0; b < d->n_k1; ++b)
        if (!(d->k1_edges[b] < d->k1_edges[b + 1])) return -1;
    double kf = BO_TWO_PI / d->box_len;
    if (d->k1_edges[d->n_k1] > (d->ng / 3.0) * kf * (1.0 + 1e-12)) return -1;
    return 0;
}

static long combos_build(const bo_desc *d, const rings_t *R, const long *ntri, combo_t **out)
{
    int nr = R->nr, nz = R->nz;
    long cap = 1024, n = 0;
    combo_t *c = malloc(sizeof(combo_t) * (size_t)cap);
    for (int n1 = -nz; n1 <= nz; ++n1)
        for (int n2 = -nz; n2 <= nz; ++n2) {
            int n3 = -(n1 + n2);
            if (n3 < -nz || n3 > nz) continue;
            for (int r1 = 0; r1 < nr; ++r1)
                for (int r2 = 0; r2 < nr; ++r2)
                    for (int r3 = 0; r3 < nr; ++r3) {
                        long nt = ntri[((long)r1 * nr + r2) * nr + r3];
                        if (nt <= 0) continue;
                        geom_t g;
                        if (!combo_geometry(d, R->kperp[r1], R->kperp[r2], R->kperp[r3], n1, n2, n3, &g)) continue;
                        if (n == cap) { cap *= 2; c = realloc(c, sizeof(combo_t) * (size_t)cap); }
                        c[n].n1 = n1; c[n].n2 = n2; c[n].n3 = n3;
                        c[n].r1 = r1; c[n].r2 = r2; c[n].r3 = r3;
                        c[n].ntri = nt;
                        c[n].g = g;
                        ++n;
                    }
        }
    *out = c;
    return n;
}

/* ------------------------------------------------------------------------ */
/* Per-combination sums S = sum_x D1 D2 D3.                                  */
/* ------------------------------------------------------------------------ */
static void sums_fft(const rings_t *R, const cplx *cube, const combo_t *c, long nc, cplx *S)
{
    int ng = R->ng, nr = R->nr, nz = R->nz;
    long np = (long)ng * ng;
    long nfield = (long)(2 * nz + 1) * nr;
    cplx *D = malloc(sizeof(cplx) * (size_t)nfield * np);
#pragma omp parallel for schedule(dynamic)
    for (long f = 0; f < nfield; ++f) {
        int n = (int)(f / nr) - nz, r = (int)(f % nr);
        dfield_from_cube(R, cube, r, n, D + f * np);
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (long k = 0; k < nc; ++k) {
        const cplx *a = D + ((long)(c[k].n1 + nz) * nr + c[k].r1) * np;
        const cplx *b = D + ((long)(c[k].n2 + nz) * nr + c[k].r2) * np;
        const cplx *e = D + ((long)(c[k].n3 + nz) * nr + c[k].r3) * np;
        cplx s = 0;
        for (long x = 0; x < np; ++x) s += a[x] * b[x] * e[x];
        S[k] = s;
    }
    free(D);
}

static cplx cube_at(const cplx *cube, int ng, long i, long j, long n)
{
    long a = (i % ng + ng) % ng, b = (j % ng + ng) % ng, z = (n % ng + ng) % ng;
    return cube[(a * ng + b) * ng + z];
}

static void sums_direct(const rings_t *R, const cplx *cube, const combo_t *c, long nc, cplx *S)
{
    int ng = R->ng, nr = R->nr;
    members_t *m = malloc(sizeof(members_t) * (size_t)nr);
    members_build(R, m);
#pragma omp parallel for schedule(dynamic, 4)
    for (long k = 0; k < nc; ++k) {
        const members_t *m1 = &m[c[k].r1], *m2 = &m[c[k].r2];
        cplx s = 0;
        for (int a = 0; a < m1->n; ++a)
            for (int b = 0; b < m2->n; ++b) {
                long wi = -m1->i[a] - m2->i[b], wj = -m1->j[a] - m2->j[b];
                if (rings_at(R, wi, wj) != c[k].r3) continue;
                s += cube_at(cube, ng, m1->i[a], m1->j[a], c[k].n1) *
                     cube_at(cube, ng, m2->i[b], m2->j[b], c[k].n2) *
                     cube_at(cube, ng, wi, wj, c[k].n3);
            }
        S[k] = s * (double)ng * (double)ng;   /* sum_x exp(-i s.x) = N_g^2 delta_K (Eq. kdelta) */
    }
    members_free(R, m);
    free(m);
}

/* ------------------------------------------------------------------------ */
/* The estimator (Eq. bs_lm2_1).                                             */
/*   B[bin][lm] (all l <= l_max, 0 <= m <= l, lm = l(l+1)/2 + m), NaN where  */
/*   the denominator is 0; num_re/num_im/den the two sums of Eq. bs_lm2_1    */
/*   (numerator already divided by V N_g^2).  Returns the number of accepted */
/*   combinations, or -1.                                                    */
/* ------------------------------------------------------------------------ */
/* Share `part` of `nparts` (bo_estimate_part): the numerator sums only the
 * combinations whose ordered plane pair (n1, n2) has index
 * (n1 + nz)(2 nz + 1) + (n2 + nz) congruent to `part` modulo `nparts`; the
 * denominator sums all of them.  The numerator being a plain sum over
 * combinations, the shares' B add up to the whole B.  (nparts = 1: every
 * combination.) */
static long estimate_share(const bo_desc *d, const double *delta, int part, int nparts, double *B, double *num_re,
                           double *num_im, double *den)
{
    if (desc_check(d)) return -1;
    set_threads(d->nthreads);
    rings_t R;
    if (rings_build(d->ng, &R)) return -1;
    int nr = R.nr;
    long *ntri = malloc(sizeof(long) * (size_t)nr * nr * nr);
    if (d->mode == 0) ntri_fft(&R, ntri);
    else ntri_direct(&R, ntri);
    combo_t *c;
    long nc = combos_build(d, &R, ntri, &c);
    cplx *cube = forward_cube(d->ng, d->box_len, delta);
    cplx *S = malloc(sizeof(cplx) * (size_t)(nc > 0 ? nc : 1));
    if (d->mode == 0) sums_fft(&R, cube, c, nc, S);
    else sums_direct(&R, cube, c, nc, S);

    int nlm = n_moments_all(d->l_max);
    long nbin = (long)d->n_k1 * d->n_mu * d->n_t;
    cplx *num = calloc((size_t)nbin * nlm, sizeof(cplx));
    double *dn = calloc((size_t)nbin * nlm, sizeof(double));
    double V = d->box_len * d->box_len * d->box_len;
    double norm = 1.0 / (V * (double)d->ng * (double)d->ng);
    for (long k = 0; k < nc; ++k) {
        const geom_t *g = &c[k].g;
        const long pair = (long)(c[k].n1 + R.nz) * (2 * R.nz + 1) + (c[k].n2 + R.nz);
        const int mine = pair % nparts == part;
        for (int l = 0; l <= d->l_max; ++l)
            for (int m = 0; m <= l; ++m) {
                long o = (long)g->bin * nlm + lm_index(l, m);
                if (mine) num[o] += combo_ystar(l, m, g) * S[k] * norm;
                dn[o] += (double)c[k].ntri * combo_y2(l, m, g);
            }
    }
    for (long b = 0; b < nbin; ++b)
        for (int l = 0; l <= d->l_max; ++l)
            for (int m = 0; m <= l; ++m) {
                long o = b * nlm + lm_index(l, m);
                if (num_re) num_re[o] = creal(num[o]);
                if (num_im) num_im[o] = cimag(num[o]);
                if (den) den[o] = dn[o];
                B[o] = dn[o] > 0 ? sqrt((2.0 * l + 1.0) / (2.0 * BO_TWO_PI)) * creal(num[o]) / dn[o] : NAN;
            }
    free(num);
    free(dn);
    free(S);
    free(cube);
    free(c);
    free(ntri);
    free(R.ringidx);
    return nc;
}

long bo_estimate(const bo_desc *d, const double *delta, double *B, double *num_re, double *num_im, double *den)
{
    return estimate_share(d, delta, 0, 1, B, num_re, num_im, den);
}

long bo_estimate_part(const bo_desc *d, const double *delta, int part, int nparts, double *B)
{
    if (nparts < 1 || part < 0 || part >= nparts) return -1;
    return estimate_share(d, delta, part, nparts, B, NULL, NULL, NULL);
}

/* ------------------------------------------------------------------------ */
/* The estimate of bo_estimate for grids whose D fields do not all fit in    */
/* memory (N_g = 512: 341 planes x 42 rings x N_g^2 complex doubles, 60 GB), */
/* in slabs of n1 with a checkpoint after each slab.                         */
/*                                                                          */
/* Two facts of the definitions let it keep the planes n >= 0 only:          */
/*  - delta is real, so Delta(-k) = conj Delta(k); a ring is symmetric under */
/*    u -> -u (its radius stays below N_g/3, short of the Nyquist index), so */
/*    Eq. iFT gives D(r, -n, x) = conj D(r, n, x);                           */
/*  - so the combination (-n1, -n2, -n3; r1, r2, r3) has the sum conj S of   */
/*    (n1, n2, n3; r1, r2, r3) in Eq. fftbs, and the same acceptance and bin */
/*    (these depend on n_i^2 only); its weight Y* is its own (p_z and p_x    */
/*    change sign), computed by combo_geometry like every other.            */
/* Slab n1 (n1 = 0, 1, .., floor(N_g/3)) forms S for every accepted          */
/* (n1, n2; r1, r2, r3), n2 over all planes, and adds to num and den both   */
/* that combination and, for n1 > 0, its mirror with conj S: every ordered  */
/* combination of bo_estimate is counted once.  Each S is the running sum   */
/* S += (D1 D2) D3 over x in increasing order, as in bo_estimate; x is cut  */
/* into chunks and D1 D2 of a chunk is formed once for the r3 that share    */
/* (r1, r2), which changes no operation of any one sum.  The accumulation   */
/* into num and den differs from bo_estimate's only in order.               */
/*                                                                          */
/* ckpt (may be NULL): after every slab, num, den and the next slab are      */
/* written there (via a temporary file and a rename); a later call with the */
/* same parameters and field resumes after the last finished slab.  The    */
/* field is identified by a weighted sum of its values stored in the file. */
/* Outputs as bo_estimate.  Returns the number of accepted ordered          */
/* combinations, or -1 (bad parameters, no memory, unreadable checkpoint). */
/* max_slabs > 0 stops after that many slabs of this call and returns -2   */
/* once their checkpoint is written (the outputs are then not set).        */
/* verbose: one line per slab on stderr.                                    */
/* ------------------------------------------------------------------------ */
#define BO_CKPT_MAGIC 0x31304b4350434f42L  /* "BOCPCK01" */

typedef struct { int n2, n3, r1, r2, r3; long ntri; } stream_combo_t;

static double field_tag(const double *delta, long n)
{
    double s = 0;
    for (long i = 0; i < n; ++i) s += delta[i] * (double)(1 + i % 1021);
    return s;
}

static int ckpt_header_ok(FILE *f, const bo_desc *d, double tag)
{
    long magic;
    int h[5];
    double bl, tg;
    if (fread(&magic, sizeof magic, 1, f) != 1 || magic != BO_CKPT_MAGIC) return 0;
    if (fread(h, sizeof(int), 5, f) != 5) return 0;
    if (h[0] != d->ng || h[1] != d->n_k1 || h[2] != d->n_mu || h[3] != d->n_t || h[4] != d->l_max) return 0;
    if (fread(&bl, sizeof bl, 1, f) != 1 || bl != d->box_len) return 0;
    for (int b = 0; b <= d->n_k1; ++b) {
        double e;
        if (fread(&e, sizeof e, 1, f) != 1 || e != d->k1_edges[b]) return 0;
    }
    if (fread(&tg, sizeof tg, 1, f) != 1 || tg != tag) return 0;
    return 1;
}

static int ckpt_write(const char *path, const bo_desc *d, double tag, int next_slab, long ncombo,
                      const cplx *num, const double *dn, long nel)
{
    size_t len = strlen(path);
    char *tmp = malloc(len + 8);
    memcpy(tmp, path, len);
    memcpy(tmp + len, ".tmp", 5);
    FILE *f = fopen(tmp, "wb");
    if (!f) { free(tmp); return -1; }
    long magic = BO_CKPT_MAGIC;
    int h[5] = {d->ng, d->n_k1, d->n_mu, d->n_t, d->l_max};
    int ok = fwrite(&magic, sizeof magic, 1, f) == 1 && fwrite(h, sizeof(int), 5, f) == 5 &&
             fwrite(&d->box_len, sizeof(double), 1, f) == 1 &&
             fwrite(d->k1_edges, sizeof(double), (size_t)d->n_k1 + 1, f) == (size_t)d->n_k1 + 1 &&
             fwrite(&tag, sizeof tag, 1, f) == 1 && fwrite(&next_slab, sizeof(int), 1, f) == 1 &&
             fwrite(&ncombo, sizeof(long), 1, f) == 1 &&
             fwrite(num, sizeof(cplx), (size_t)nel, f) == (size_t)nel &&
             fwrite(dn, sizeof(double), (size_t)nel, f) == (size_t)nel;
    ok = (fclose(f) == 0) && ok;
    if (ok) ok = rename(tmp, path) == 0;
    free(tmp);
    return ok ? 0 : -1;
}

/* The accepted combinations of the ordered plane pair (n1, n2), in (r1, r2, r3) order. */
static long pair_combos(const bo_desc *d, const rings_t *R, const long *ntri, int n1, int n2,
                        stream_combo_t *out)
{
    int nr = R->nr, n3 = -(n1 + n2);
    long k = 0;
    for (int r1 = 0; r1 < nr; ++r1)
        for (int r2 = 0; r2 < nr; ++r2)
            for (int r3 = 0; r3 < nr; ++r3) {
                long nt = ntri[((long)r1 * nr + r2) * nr + r3];
                if (nt <= 0) continue;
                geom_t g;
                if (!combo_geometry(d, R->kperp[r1], R->kperp[r2], R->kperp[r3], n1, n2, n3, &g)) continue;
                out[k].n2 = n2; out[k].n3 = n3;
                out[k].r1 = r1; out[k].r2 = r2; out[k].r3 = r3;
                out[k].ntri = nt;
                ++k;
            }
    return k;
}

/* D(r, n) of the store of planes n >= 0, conjugated for n < 0 (cj = 1). */
static const cplx *stored_field(const cplx *D, int nr, long np, int r, int n, int *cj)
{
    *cj = n < 0;
    return D + ((long)(n < 0 ? -n : n) * nr + r) * np;
}

/* Sums S_k = sum_x D(r1,n1) D(r2,n2) D(r3,n3) of one plane pair's combinations. */
static void pair_sums(const cplx *D, int nr, long np, int n1, const stream_combo_t *c, long nc, cplx *S, cplx *P)
{
    enum { XC = 512 };
    for (long k = 0; k < nc; ++k) S[k] = 0;
    for (long x0 = 0; x0 < np; x0 += XC) {
        long xn = np - x0 < XC ? np - x0 : XC;
        long k = 0;
        while (k < nc) {
            long kend = k;
            while (kend < nc && c[kend].r1 == c[k].r1 && c[kend].r2 == c[k].r2) ++kend;
            int ca, cb;
            const cplx *a = stored_field(D, nr, np, c[k].r1, n1, &ca) + x0;
            const cplx *b = stored_field(D, nr, np, c[k].r2, c[k].n2, &cb) + x0;
            for (long x = 0; x < xn; ++x) {
                cplx av = ca ? conj(a[x]) : a[x], bv = cb ? conj(b[x]) : b[x];
                P[x] = av * bv;
            }
            /* up to four r3 at a time, each its own running sum: the
             * product P e written out as (pr er - pi ei) + i (pr ei + pi er),
             * the operations of the complex product, with ei negated (exact)
             * for a conjugated field */
            while (k < kend) {
                const int nk = kend - k < 4 ? (int)(kend - k) : 4;
                const double *e[4];
                double sr[4], si[4], sg = 1.0;
                for (int j = 0; j < 4; ++j) {
                    int ce;
                    const int kk = j < nk ? (int)(k + j) : (int)k;
                    e[j] = (const double *)(stored_field(D, nr, np, c[kk].r3, c[kk].n3, &ce) + x0);
                    sg = ce ? -1.0 : 1.0;           /* the same n3 for every combination of the pair */
                    sr[j] = creal(S[kk]);
                    si[j] = cimag(S[kk]);
                }
                const double *p = (const double *)P;
                if (nk == 4) {
                    for (long x = 0; x < xn; ++x) {
                        const double pr = p[2 * x], pi = p[2 * x + 1];
                        for (int j = 0; j < 4; ++j) {
                            const double er = e[j][2 * x], ei = sg * e[j][2 * x + 1];
                            sr[j] = sr[j] + (pr * er - pi * ei);
                            si[j] = si[j] + (pr * ei + pi * er);
                        }
                    }
                } else {
                    for (long x = 0; x < xn; ++x) {
                        const double pr = p[2 * x], pi = p[2 * x + 1];
                        for (int j = 0; j < nk; ++j) {
                            const double er = e[j][2 * x], ei = sg * e[j][2 * x + 1];
                            sr[j] = sr[j] + (pr * er - pi * ei);
                            si[j] = si[j] + (pr * ei + pi * er);
                        }
                    }
                }
                for (int j = 0; j < nk; ++j) S[k + j] = CMPLX(sr[j], si[j]);
                k += nk;
            }
        }
    }
}

static void add_combo(const bo_desc *d, const rings_t *R, int n1, const stream_combo_t *c, cplx S, double norm,
                      int nlm, cplx *num, double *dn)
{
    geom_t g;
    combo_geometry(d, R->kperp[c->r1], R->kperp[c->r2], R->kperp[c->r3], n1, c->n2, c->n3, &g);
    for (int l = 0; l <= d->l_max; ++l)
        for (int m = 0; m <= l; ++m) {
            long o = (long)g.bin * nlm + lm_index(l, m);
            num[o] += combo_ystar(l, m, &g) * S * norm;
            dn[o] += (double)c->ntri * combo_y2(l, m, &g);
        }
}

long bo_estimate_stream(const bo_desc *d, const double *delta, const char *ckpt, int max_slabs, int verbose,
                        double *B, double *num_re, double *num_im, double *den)
{
    if (desc_check(d) || d->mode != 0 || (max_slabs > 0 && !ckpt)) return -1;
    set_threads(d->nthreads);
    rings_t R;
    if (rings_build(d->ng, &R)) return -1;
    int ng = d->ng, nr = R.nr, nz = R.nz;
    long np = (long)ng * ng;
    int nlm = n_moments_all(d->l_max);
    long nbin = (long)d->n_k1 * d->n_mu * d->n_t, nel = nbin * nlm;
    double V = d->box_len * d->box_len * d->box_len;
    double norm = 1.0 / (V * (double)ng * (double)ng);
    double tag = field_tag(delta, np * ng);

    cplx *num = calloc((size_t)nel, sizeof(cplx));
    double *dn = calloc((size_t)nel, sizeof(double));
    long ncombo = 0;
    int slab0 = 0;
    if (ckpt) {
        FILE *f = fopen(ckpt, "rb");
        if (f) {
            int ok = ckpt_header_ok(f, d, tag) && fread(&slab0, sizeof(int), 1, f) == 1 &&
                     fread(&ncombo, sizeof(long), 1, f) == 1 &&
                     fread(num, sizeof(cplx), (size_t)nel, f) == (size_t)nel &&
                     fread(dn, sizeof(double), (size_t)nel, f) == (size_t)nel;
            fclose(f);
            if (!ok) { free(num); free(dn); free(R.ringidx); return -1; }
            if (verbose) fprintf(stderr, "stream: resuming at slab %d of %d\n", slab0, nz + 1);
        }
    }

    long *ntri = malloc(sizeof(long) * (size_t)nr * nr * nr);
    ntri_fft(&R, ntri);
    cplx *D = NULL;
    if (slab0 <= nz) {
        cplx *cube = forward_cube(ng, d->box_len, delta);
        D = cube ? malloc(sizeof(cplx) * (size_t)(nz + 1) * nr * np) : NULL;
        if (!D) { free(cube); free(ntri); free(num); free(dn); free(R.ringidx); return -1; }
#pragma omp parallel for schedule(dynamic)
        for (long f = 0; f < (long)(nz + 1) * nr; ++f)
            dfield_from_cube(&R, cube, (int)(f % nr), (int)(f / nr), D + f * np);
        free(cube);
        if (verbose) fprintf(stderr, "stream: %ld D fields ready\n", (long)(nz + 1) * nr);
    }

    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    cplx *tnum = calloc((size_t)nth * nel, sizeof(cplx));
    double *tdn = calloc((size_t)nth * nel, sizeof(double));
    long cap = (long)nr * nr * nr;
    int failed = 0, stopped = 0;
    for (int n1 = slab0; n1 <= nz && !failed; ++n1) {
        if (max_slabs > 0 && n1 - slab0 >= max_slabs) { stopped = 1; break; }
        double t0 = 0;
#ifdef _OPENMP
        t0 = omp_get_wtime();
#endif
        long slab_combos = 0;
        memset(tnum, 0, sizeof(cplx) * (size_t)nth * nel);
        memset(tdn, 0, sizeof(double) * (size_t)nth * nel);
#pragma omp parallel reduction(+ : slab_combos)
        {
            int me = 0;
#ifdef _OPENMP
            me = omp_get_thread_num();
#endif
            stream_combo_t *c = malloc(sizeof(stream_combo_t) * (size_t)cap);
            cplx *S = malloc(sizeof(cplx) * (size_t)cap);
            cplx *P = malloc(sizeof(cplx) * 512);
            cplx *mynum = tnum + (long)me * nel;
            double *mydn = tdn + (long)me * nel;
            /* round robin over n2: for a given thread count every thread
             * sums the same pairs in the same order, so a resumed run ends
             * with the bits of an uninterrupted one */
#pragma omp for schedule(static, 1)
            for (int n2 = -nz; n2 <= nz; ++n2) {
                int n3 = -(n1 + n2);
                if (n3 < -nz || n3 > nz) continue;
                long nc = pair_combos(d, &R, ntri, n1, n2, c);
                if (nc == 0) continue;
                pair_sums(D, nr, np, n1, c, nc, S, P);
                for (long k = 0; k < nc; ++k) {
                    add_combo(d, &R, n1, &c[k], S[k], norm, nlm, mynum, mydn);
                    slab_combos += 1;
                    if (n1 > 0) {
                        stream_combo_t m = c[k];
                        m.n2 = -c[k].n2;
                        m.n3 = -c[k].n3;
                        add_combo(d, &R, -n1, &m, conj(S[k]), norm, nlm, mynum, mydn);
                        slab_combos += 1;
                    }
                }
            }
            free(c);
            free(S);
            free(P);
        }
        for (int t = 0; t < nth; ++t)
            for (long o = 0; o < nel; ++o) {
                num[o] += tnum[(long)t * nel + o];
                dn[o] += tdn[(long)t * nel + o];
            }
        ncombo += slab_combos;
        if (ckpt && ckpt_write(ckpt, d, tag, n1 + 1, ncombo, num, dn, nel)) failed = 1;
        if (verbose) {
            double t1 = 0;
#ifdef _OPENMP
            t1 = omp_get_wtime();
#endif
            fprintf(stderr, "stream: slab %d/%d  %ld combinations  %.1f s\n", n1, nz, slab_combos, t1 - t0);
        }
    }
    free(tnum);
    free(tdn);
    free(D);
    free(ntri);
    if (!failed && !stopped)
        for (long b = 0; b < nbin; ++b)
            for (int l = 0; l <= d->l_max; ++l)
                for (int m = 0; m <= l; ++m) {
                    long o = b * nlm + lm_index(l, m);
                    if (num_re) num_re[o] = creal(num[o]);
                    if (num_im) num_im[o] = cimag(num[o]);
                    if (den) den[o] = dn[o];
                    B[o] = dn[o] > 0 ? sqrt((2.0 * l + 1.0) / (2.0 * BO_TWO_PI)) * creal(num[o]) / dn[o] : NAN;
                }
    free(num);
    free(dn);
    free(R.ringidx);
    return failed ? -1 : stopped ? -2 : ncombo;
}

/* ------------------------------------------------------------------------ */
/* Combination table export.  half_space = 1 keeps one of each pair          */
/* (n1,n2) / (-n1,-n2): n1 > 0, or n1 == 0 and n2 >= 0.                      */
/* ints[k][6] = n1,n2,n3,r1,r2,r3; bins[k] = flat (k1,mu,t) bin;             */
/* geo[k][6] = K1, t, mu, p_z, cos phi (chirality-free), degenerate flag.    */
/* Returns the count (all of it, even beyond cap).                           */
/* ------------------------------------------------------------------------ */
long bo_combos(const bo_desc *d, int half_space, long cap, int *ints, long *ntri_out, int *bins, double *geo)
{
    if (desc_check(d)) return -1;
    set_threads(d->nthreads);
    rings_t R;
    if (rings_build(d->ng, &R)) return -1;
    int nr = R.nr;
    long *ntri = malloc(sizeof(long) * (size_t)nr * nr * nr);
    if (d->mode == 0) ntri_fft(&R, ntri);
    else ntri_direct(&R, ntri);
    combo_t *c;
    long nc = combos_build(d, &R, ntri, &c);
    long k = 0;
    for (long i = 0; i < nc; ++i) {
        if (half_space && !(c[i].n1 > 0 || (c[i].n1 == 0 && c[i].n2 >= 0))) continue;
        if (k < cap) {
            int *p = ints + 6 * k;
            p[0] = c[i].n1; p[1] = c[i].n2; p[2] = c[i].n3;
            p[3] = c[i].r1; p[4] = c[i].r2; p[5] = c[i].r3;
            ntri_out[k] = c[i].ntri;
            bins[k] = c[i].g.bin;
            double *q = geo + 6 * k;
            q[0] = c[i].g.K1; q[1] = c[i].g.t; q[2] = c[i].g.mu; q[3] = c[i].g.pz;
            q[4] = c[i].g.cphi; q[5] = c[i].g.degenerate;
        }
        ++k;
    }
    free(c);
    free(ntri);
    free(R.ringidx);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Sums S = sum_x D1 D2 D3 (Eq. fftbs) for a given list of combinations,     */
/* computing only the planes and D fields the list needs.  ints[k][6] as in  */
/* bo_combos.  S_re_im[k][2].  For spot checks at large N_g.  times (may be  */
/* NULL) gets the wall seconds of the three stages: [0] the needed planes of */
/* the forward transform, [1] the D fields, [2] the triple sums.             */
/* ------------------------------------------------------------------------ */
int bo_combo_sums(int ng, double box_len, const double *delta, long nc, const int *ints, int nthreads,
                  double *S_re_im, double *times)
{
    set_threads(nthreads);
    rings_t R;
    if (rings_build(ng, &R)) return -1;
    int nr = R.nr, nz = R.nz;
    long np = (long)ng * ng;
    long nfield = (long)(2 * nz + 1) * nr;
    for (long k = 0; k < nc; ++k)
        for (int s = 0; s < 3; ++s) {
            int n = ints[6 * k + s], r = ints[6 * k + 3 + s];
            if (n < -nz || n > nz || r < 0 || r >= nr) { free(R.ringidx); return -1; }
        }
    cplx **D = calloc((size_t)nfield, sizeof(cplx *));
    char *need_plane = calloc((size_t)(2 * nz + 1), 1);
    char *need_field = calloc((size_t)nfield, 1);
    for (long k = 0; k < nc; ++k)
        for (int s = 0; s < 3; ++s) {
            int n = ints[6 * k + s], r = ints[6 * k + 3 + s];
            need_plane[n + nz] = 1;
            need_field[(long)(n + nz) * nr + r] = 1;
        }
    double t0 = 0, t1 = 0, t2 = 0, t3 = 0;
#ifdef _OPENMP
    t0 = omp_get_wtime();
#endif
    /* planes: the DFT of every (x, y) column along z, kept at the needed n,
     * then (V/N_g^3) times the 2D DFT over (x, y) */
    double V = box_len * box_len * box_len, scale = V / ((double)np * ng);
    cplx **plane = calloc((size_t)(2 * nz + 1), sizeof(cplx *));
    for (int pi = 0; pi < 2 * nz + 1; ++pi)
        if (need_plane[pi]) plane[pi] = malloc(sizeof(cplx) * (size_t)np);
#pragma omp parallel
    {
        cplx *col = malloc(sizeof(cplx) * (size_t)ng), *tmp = malloc(sizeof(cplx) * (size_t)ng);
#pragma omp for schedule(static)
        for (long xy = 0; xy < np; ++xy) {
            for (long z = 0; z < ng; ++z) col[z] = delta[xy * ng + z];
            dft1(col, ng, tmp);
            for (int pi = 0; pi < 2 * nz + 1; ++pi)
                if (plane[pi]) plane[pi][xy] = col[((pi - nz) % ng + ng) % ng];
        }
        free(col);
        free(tmp);
    }
    for (int pi = 0; pi < 2 * nz + 1; ++pi) {
        if (!plane[pi]) continue;
        dft2(plane[pi], ng);
        for (long i = 0; i < np; ++i) plane[pi][i] *= scale;
        if (pi == nz) plane[pi][0] = 0;
    }
#ifdef _OPENMP
    t1 = omp_get_wtime();
#endif
    for (long f = 0; f < nfield; ++f) {
        if (!need_field[f]) continue;
        int n = (int)(f / nr) - nz, r = (int)(f % nr);
        const cplx *p = plane[n + nz];
        cplx *o = malloc(sizeof(cplx) * (size_t)np);
        for (long a = 0; a < ng; ++a)
            for (long b = 0; b < ng; ++b)
                o[a * ng + b] = (rings_at(&R, signed_freq(a, ng), signed_freq(b, ng)) == r) ? p[a * ng + b] : 0;
        dft2(o, ng);
        D[f] = o;
    }
#ifdef _OPENMP
    t2 = omp_get_wtime();
#endif
#pragma omp parallel for schedule(dynamic)
    for (long k = 0; k < nc; ++k) {
        const int *q = ints + 6 * k;
        const cplx *a = D[(long)(q[0] + nz) * nr + q[3]];
        const cplx *b = D[(long)(q[1] + nz) * nr + q[4]];
        const cplx *e = D[(long)(q[2] + nz) * nr + q[5]];
        cplx s = 0;
        for (long x = 0; x < np; ++x) s += a[x] * b[x] * e[x];
        S_re_im[2 * k] = creal(s);
        S_re_im[2 * k + 1] = cimag(s);
    }
#ifdef _OPENMP
    t3 = omp_get_wtime();
#endif
    if (times) { times[0] = t1 - t0; times[1] = t2 - t1; times[2] = t3 - t2; }
    for (long f = 0; f < nfield; ++f) free(D[f]);
    for (int pi = 0; pi < 2 * nz + 1; ++pi) free(plane[pi]);
    free(plane);
    free(D);
    free(need_plane);
    free(need_field);
    free(R.ringidx);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Analytic model of Sec. III: B^r = 2 f_NG (P1P2 + P2P3 + P3P1) (Eq.        */
/* mod_bs) with P(k) = A k^index, times prod_i (1 + beta mu_i^2) (Eq.         */
/* rsd_bs).                                                                  */
/* ------------------------------------------------------------------------ */
static double model_bs(double A, double index, double f_ng, double beta,
                       double k1, double k2, double k3, double mu1, double mu2, double mu3)
{
    double P1 = A * pow(k1, index), P2 = A * pow(k2, index), P3 = A * pow(k3, index);
    double Br = 2.0 * f_ng * (P1 * P2 + P2 * P3 + P3 * P1);
    return (1.0 + beta * mu1 * mu1) * (1.0 + beta * mu2 * mu2) * (1.0 + beta * mu3 * mu3) * Br;
}

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n. */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(0.5 * BO_TWO_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
            double pn = (n == 1) ? z : p1, pn1 = (n == 1) ? 1.0 : p0;
            double dp = n * (z * pn - pn1) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
        double pn = (n == 1) ? z : p1, pn1 = (n == 1) ? 1.0 : p0;
        double dp = n * (z * pn - pn1) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

void bo_gauss_legendre(int n, double *x, double *w) { gauss_legendre(n, x, w); }

/* Continuum multipoles [B_l^m]_c of Eq. bs_lm for the model above, at one
 * (k1, mu, t): Gauss-Legendre in p_z times a uniform rule in the azimuth of
 * p.  The integrand is a polynomial in (p_x, p_z) of degree 6 times Y*, so
 * n_gl >= (6 + l_max)/2 + 1 and n_phi >= 6 + l_max + 1 make it exact.
 * out[lm][2] for all l <= l_max, 0 <= m <= l.  Which factors of Eq. rsd_bs
 * enter is set by the bits of factor_mask (1: mu_1, 2: mu_2, 4: mu_3).
 * axis selects the polar axis of Y_l^m in the triangle frame of Eq. orient
 * (z' along k1, x' in the triangle plane): 0 = z' (the estimator's
 * reading), 1 = x' with the azimuth measured from z'.  With axis 0 the
 * moments l = 6, m = 5, 6 of this model vanish identically (p_x enters at
 * most to the fourth power); with axis 1 all sixteen even-l moments are
 * non-zero, which is the count the paper states. */
void bo_continuum(double A, double index, double f_ng, double beta, int factor_mask, int axis,
                  double k1, double mu, double t, int l_max, int n_gl, int n_phi, double *out)
{
    double *x = malloc(sizeof(double) * (size_t)n_gl), *w = malloc(sizeof(double) * (size_t)n_gl);
    gauss_legendre(n_gl, x, w);
    int nlm = n_moments_all(l_max);
    cplx *acc = calloc((size_t)nlm, sizeof(cplx));
    double k2 = t * k1, k3 = k1 * sqrt(1.0 - 2.0 * t * mu + t * t);
    double sm = sqrt(1.0 - mu * mu), den3 = sqrt(1.0 - 2.0 * t * mu + t * t);
    for (int i = 0; i < n_gl; ++i) {
        double c = x[i], st = sqrt(fmax(0.0, 1.0 - c * c));   /* polar cosine about the axis */
        for (int j = 0; j < n_phi; ++j) {
            double phi = BO_TWO_PI * (double)j / (double)n_phi;
            double cp = cos(phi), sp = sin(phi);
            /* components of p in the triangle frame of Eq. orient */
            double pz = (axis == 1) ? st * cp : c;
            double px = (axis == 1) ? c : st * cp;
            double mu1 = pz;
            double mu2 = -mu * pz + sm * px;
            double mu3 = -((1.0 - t * mu) * pz + t * sm * px) / den3;
            double b1 = (factor_mask & 1) ? beta : 0.0, b2 = (factor_mask & 2) ? beta : 0.0, b3 = (factor_mask & 4) ? beta : 0.0;
            double P1 = A * pow(k1, index), P2 = A * pow(k2, index), P3 = A * pow(k3, index);
            double Br = 2.0 * f_ng * (P1 * P2 + P2 * P3 + P3 * P1);
            double Bs = (1.0 + b1 * mu1 * mu1) * (1.0 + b2 * mu2 * mu2) * (1.0 + b3 * mu3 * mu3) * Br;
            double dOmega = w[i] * BO_TWO_PI / (double)n_phi;
            for (int l = 0; l <= l_max; ++l)
                for (int m = 0; m <= l; ++m)
                    acc[lm_index(l, m)] += conj(ylm(l, m, c, cp, sp)) * Bs * dOmega;
        }
    }
    for (int l = 0; l <= l_max; ++l)
        for (int m = 0; m <= l; ++m) {
            cplx v = sqrt((2.0 * l + 1.0) / (2.0 * BO_TWO_PI)) * acc[lm_index(l, m)];
            out[2 * lm_index(l, m)] = creal(v);
            out[2 * lm_index(l, m) + 1] = cimag(v);
        }
    free(acc);
    free(x);
    free(w);
}

/* Discrete analytic prediction [B_l^m]_d of Sec. III.C: the model of Eq.
 * rsd_bs at each combination's mean (K_i, mu_i), binned exactly as the
 * estimator (Eq. bs_lm2_1 with Bhat replaced by the model).  B[bin][lm] as
 * in bo_estimate.  Returns the number of combinations. */
long bo_discrete_model(const bo_desc *d, double A, double index, double f_ng, double beta, double *B)
{
    if (desc_check(d)) return -1;
    set_threads(d->nthreads);
    rings_t R;
    if (rings_build(d->ng, &R)) return -1;
    int nr = R.nr;
    long *ntri = malloc(sizeof(long) * (size_t)nr * nr * nr);
    if (d->mode == 0) ntri_fft(&R, ntri);
    else ntri_direct(&R, ntri);
    combo_t *c;
    long nc = combos_build(d, &R, ntri, &c);
    int nlm = n_moments_all(d->l_max);
    long nbin = (long)d->n_k1 * d->n_mu * d->n_t;
    cplx *num = calloc((size_t)nbin * nlm, sizeof(cplx));
    double *dn = calloc((size_t)nbin * nlm, sizeof(double));
    double kf = BO_TWO_PI / d->box_len;
    for (long k = 0; k < nc; ++k) {
        const geom_t *g = &c[k].g;
        double K[3], kp[3] = {R.kperp[c[k].r1], R.kperp[c[k].r2], R.kperp[c[k].r3]};
        int n[3] = {c[k].n1, c[k].n2, c[k].n3};
        for (int s = 0; s < 3; ++s) K[s] = kf * sqrt(kp[s] * kp[s] + (double)n[s] * n[s]);
        double bs = model_bs(A, index, f_ng, beta, K[0], K[1], K[2], g->mu1, g->mu2, g->mu3);
        for (int l = 0; l <= d->l_max; ++l)
            for (int m = 0; m <= l; ++m) {
                long o = (long)g->bin * nlm + lm_index(l, m);
                num[o] += combo_ystar(l, m, g) * bs * (double)c[k].ntri;
                dn[o] += (double)c[k].ntri * combo_y2(l, m, g);
            }
    }
    for (long b = 0; b < nbin; ++b)
        for (int l = 0; l <= d->l_max; ++l)
            for (int m = 0; m <= l; ++m) {
                long o = b * nlm + lm_index(l, m);
                B[o] = dn[o] > 0 ? sqrt((2.0 * l + 1.0) / (2.0 * BO_TWO_PI)) * creal(num[o]) / dn[o] : NAN;
            }
    free(num);
    free(dn);
    free(c);
    free(ntri);
    free(R.ringidx);
    return nc;
}

/* Orientation inverse used by the estimator, exposed for pinning: from the
 * side cosines (mu_1, mu_2) and the shape mu, p_z and p_x of Eq. orient. */
void bo_orientation(double mu1, double mu2, double mu, double *pz, double *px)
{
    orient_inverse(mu1, mu2, mu, pz, px);
}

/* ======================================================================== */
/* Spherical-shell estimator of the m = 0 multipoles.                       */
/*                                                                          */
/* The FFT estimators the paper builds on (Sec. I) bin k in spherical        */
/* shells; with the weight of each mode's own direction they reach the m = 0 */
/* moments only.  Written out here as a comparison for that subset:          */
/*   shells     s = {k : e_s <= |k| < e_{s+1}} with |k| the 3D length and the */
/*              ring edges e (the same width rule); shell 0 = {0} is unused;  */
/*              K_s = mean |k| over the shell                                */
/*   triples    s1 >= s2 >= s3 >= 1 (then K1 >= K2 >= K3), binned in          */
/*              (k1, mu, t) from (K1, K2, K3) like a combination with n = 0;  */
/*              kept when N_tri > 0                                          */
/*   sums       over closed triangles k1 + k2 + k3 = 0, k_i in s_i:           */
/*                num_l = sum Y_l0(k1) Delta(k1) Delta(k2) Delta(k3)          */
/*                den_l = sum Y_l0(k1)^2,   N_tri = sum 1                     */
/*              Y_l0(k) = sqrt((2l+1)/4pi) P_l(k_z / |k|); even l            */
/*   FFT form   num_l = N^-3 sum_x F_{s1,l} D_{s2} D_{s3}, with               */
/*              F_{s,l}(x) = sum_{k in s} Y_l0(k) Delta(k) e^{-ik.x},         */
/*              D_s the same without Y; den_l and N_tri alike from            */
/*              sum_{k in s} Y_l0^2 e^{-ik.x} and sum_{k in s} e^{-ik.x}      */
/*   result     B_l^0 = sqrt((2l+1)/4pi) sum Re num_l / (V sum den_l) over    */
/*              the bin's triples; NaN where sum den_l = 0                   */
/* mode 0: FFT form; 1: the direct sums over mode pairs.                    */
/* ======================================================================== */
typedef struct {
    int ng, ns;
    long e3[BO_MAX_RINGS + 1];
    double K[BO_MAX_RINGS];
    int *idx;          /* shell of cube point (FFT index order, kz fastest), -1 outside */
} shells_t;

static int shells_build(int ng, shells_t *S)
{
    S->ng = ng;
    S->ns = ring_edges3(ng, S->e3);
    if (S->ns < 0) return -1;
    long n3 = (long)ng * ng * ng;
    S->idx = malloc(sizeof(int) * (size_t)n3);
    double sum[BO_MAX_RINGS];
    long cnt[BO_MAX_RINGS];
    for (int s = 0; s < S->ns; ++s) { sum[s] = 0; cnt[s] = 0; }
    for (long a = 0; a < ng; ++a)
        for (long b = 0; b < ng; ++b)
            for (long c = 0; c < ng; ++c) {
                long i = signed_freq(a, ng), j = signed_freq(b, ng), n = signed_freq(c, ng);
                long q9 = 9 * (i * i + j * j + n * n);
                int sh = -1;
                for (int s = 0; s < S->ns; ++s)
                    if (S->e3[s] * S->e3[s] <= q9 && q9 < S->e3[s + 1] * S->e3[s + 1]) { sh = s; break; }
                S->idx[(a * ng + b) * ng + c] = sh;
                if (sh >= 0) { sum[sh] += sqrt((double)(i * i + j * j + n * n)); cnt[sh] += 1; }
            }
    for (int s = 0; s < S->ns; ++s) S->K[s] = cnt[s] > 0 ? sum[s] / (double)cnt[s] : 0.0;
    return 0;
}

static double legendre_even(int l, double z)
{
    return assoc_legendre(l, 0, z);
}

/* Y_l0 of the direction of cube point (a, b, c) (k != 0) */
static double y_l0_at(int l, int ng, long a, long b, long c)
{
    long i = signed_freq(a, ng), j = signed_freq(b, ng), n = signed_freq(c, ng);
    double k = sqrt((double)(i * i + j * j + n * n));
    return ylm_norm(l, 0) * legendre_even(l, (double)n / k);
}

/* field sum_{k in s} w(k) e^{-ik.x} on the cube, w = value * Y_l0^power */
static void shell_field(const shells_t *S, const cplx *cube, int s, int l, int power, cplx *out)
{
    int ng = S->ng;
    long n3 = (long)ng * ng * ng;
    for (long p = 0; p < n3; ++p) {
        if (S->idx[p] != s) { out[p] = 0; continue; }
        long a = p / ((long)ng * ng), b = (p / ng) % ng, c = p % ng;
        double w = 1.0;
        for (int q = 0; q < power; ++q) w *= y_l0_at(l, ng, a, b, c);
        out[p] = (cube ? cube[p] : 1.0) * w;
    }
    dft3(out, ng);
}

/* Accepted triples and their sums.  tri[k][4] = s1, s2, s3, bin; ntri[k];
 * num/den [k][nl] (nl = l_max/2 + 1, l = 0, 2, ..).  delta may be NULL
 * (num left 0).  Returns the count (all of it, even beyond cap), or -1. */
long bo_shell_triples(const bo_desc *d, const double *delta, long cap, int *tri, double *ntri,
                      double *num, double *den)
{
    if (desc_check(d) || (d->l_max & 1)) return -1;
    set_threads(d->nthreads);
    shells_t S;
    if (shells_build(d->ng, &S)) return -1;
    int ng = d->ng, ns = S.ns, nl = d->l_max / 2 + 1;
    long n3 = (long)ng * ng * ng;
    cplx *cube = delta ? forward_cube(ng, d->box_len, delta) : NULL;
    long n = 0;
    if (d->mode == 0) {
        /* fields: D_s, F_{s,l} (l >= 2), I_s, G_{s,l} */
        cplx **D = calloc((size_t)ns, sizeof(cplx *)), **I1 = calloc((size_t)ns, sizeof(cplx *));
        cplx **F = calloc((size_t)ns * nl, sizeof(cplx *)), **G = calloc((size_t)ns * nl, sizeof(cplx *));
        for (int s = 1; s < ns; ++s) {
            I1[s] = malloc(sizeof(cplx) * (size_t)n3);
            shell_field(&S, NULL, s, 0, 0, I1[s]);
            for (int li = 0; li < nl; ++li) {
                G[s * nl + li] = malloc(sizeof(cplx) * (size_t)n3);
                shell_field(&S, NULL, s, 2 * li, 2, G[s * nl + li]);
            }
            if (cube) {
                D[s] = malloc(sizeof(cplx) * (size_t)n3);
                shell_field(&S, cube, s, 0, 0, D[s]);
                for (int li = 0; li < nl; ++li) {
                    F[s * nl + li] = malloc(sizeof(cplx) * (size_t)n3);
                    shell_field(&S, cube, s, 2 * li, 1, F[s * nl + li]);
                }
            }
        }
        for (int s1 = 1; s1 < ns; ++s1)
            for (int s2 = 1; s2 <= s1; ++s2)
                for (int s3 = 1; s3 <= s2; ++s3) {
                    geom_t g;
                    if (!combo_geometry(d, S.K[s1], S.K[s2], S.K[s3], 0, 0, 0, &g)) continue;
                    cplx t = 0;
                    for (long p = 0; p < n3; ++p) t += I1[s1][p] * I1[s2][p] * I1[s3][p];
                    double cnt = creal(t) / (double)n3;
                    if (!(cnt > 0.5)) continue;
                    if (n < cap) {
                        tri[4 * n] = s1; tri[4 * n + 1] = s2; tri[4 * n + 2] = s3; tri[4 * n + 3] = g.bin;
                        ntri[n] = floor(cnt + 0.5);
                        for (int li = 0; li < nl; ++li) {
                            cplx u = 0, v = 0;
                            for (long p = 0; p < n3; ++p) {
                                u += G[s1 * nl + li][p] * I1[s2][p] * I1[s3][p];
                                if (cube) v += F[s1 * nl + li][p] * D[s2][p] * D[s3][p];
                            }
                            den[n * nl + li] = creal(u) / (double)n3;
                            num[n * nl + li] = creal(v) / (double)n3;
                        }
                    }
                    ++n;
                }
        for (int s = 0; s < ns; ++s) {
            free(D[s]); free(I1[s]);
            for (int li = 0; li < nl; ++li) { free(F[s * nl + li]); free(G[s * nl + li]); }
        }
        free(D); free(I1); free(F); free(G);
    } else {
        /* direct: every ordered pair of modes (k1, k2), k3 = -k1 - k2 */
        long nt3 = (long)ns * ns * ns;
        double *acc_n = calloc((size_t)nt3 * nl, sizeof(double)), *acc_d = calloc((size_t)nt3 * nl, sizeof(double));
        double *acc_c = calloc((size_t)nt3, sizeof(double));
        for (long p1 = 0; p1 < n3; ++p1) {
            int s1 = S.idx[p1];
            if (s1 < 1) continue;
            long a1 = p1 / ((long)ng * ng), b1 = (p1 / ng) % ng, c1 = p1 % ng;
            long i1 = signed_freq(a1, ng), j1 = signed_freq(b1, ng), n1 = signed_freq(c1, ng);
            double y[8];
            for (int li = 0; li < nl; ++li) y[li] = y_l0_at(2 * li, ng, a1, b1, c1);
            for (long p2 = 0; p2 < n3; ++p2) {
                int s2 = S.idx[p2];
                if (s2 < 1 || s2 > s1) continue;
                long a2 = p2 / ((long)ng * ng), b2 = (p2 / ng) % ng, c2 = p2 % ng;
                long i3 = -i1 - signed_freq(a2, ng), j3 = -j1 - signed_freq(b2, ng), n3z = -n1 - signed_freq(c2, ng);
                long h = ng / 2;
                if (i3 < -h || i3 >= h || j3 < -h || j3 >= h || n3z < -h || n3z >= h) continue;
                long p3 = (((i3 + ng) % ng) * ng + (j3 + ng) % ng) * ng + (n3z + ng) % ng;
                int s3 = S.idx[p3];
                if (s3 < 1 || s3 > s2) continue;
                long t = ((long)s1 * ns + s2) * ns + s3;
                acc_c[t] += 1.0;
                cplx v = cube ? cube[p1] * cube[p2] * cube[p3] : 0;
                for (int li = 0; li < nl; ++li) {
                    acc_d[t * nl + li] += y[li] * y[li];
                    acc_n[t * nl + li] += y[li] * creal(v);
                }
            }
        }
        for (int s1 = 1; s1 < ns; ++s1)
            for (int s2 = 1; s2 <= s1; ++s2)
                for (int s3 = 1; s3 <= s2; ++s3) {
                    geom_t g;
                    long t = ((long)s1 * ns + s2) * ns + s3;
                    if (!combo_geometry(d, S.K[s1], S.K[s2], S.K[s3], 0, 0, 0, &g)) continue;
                    if (!(acc_c[t] > 0.5)) continue;
                    if (n < cap) {
                        tri[4 * n] = s1; tri[4 * n + 1] = s2; tri[4 * n + 2] = s3; tri[4 * n + 3] = g.bin;
                        ntri[n] = acc_c[t];
                        for (int li = 0; li < nl; ++li) {
                            den[n * nl + li] = acc_d[t * nl + li];
                            num[n * nl + li] = acc_n[t * nl + li];
                        }
                    }
                    ++n;
                }
        free(acc_n); free(acc_d); free(acc_c);
    }
    free(cube);
    free(S.idx);
    return n;
}

/* B_l^0 [n_k1][n_mu][n_t][nl] of the shell estimator (mode as above). */
long bo_shell_estimate(const bo_desc *d, const double *delta, double *B)
{
    long n = bo_shell_triples(d, delta, 0, NULL, NULL, NULL, NULL);
    if (n < 0) return -1;
    int nl = d->l_max / 2 + 1;
    int *tri = malloc(sizeof(int) * 4 * (size_t)(n > 0 ? n : 1));
    double *nt = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *num = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * nl);
    double *den = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * nl);
    bo_shell_triples(d, delta, n, tri, nt, num, den);
    long nbin = (long)d->n_k1 * d->n_mu * d->n_t;
    double *sn = calloc((size_t)nbin * nl, sizeof(double)), *sd = calloc((size_t)nbin * nl, sizeof(double));
    for (long k = 0; k < n; ++k)
        for (int li = 0; li < nl; ++li) {
            sn[(long)tri[4 * k + 3] * nl + li] += num[k * nl + li];
            sd[(long)tri[4 * k + 3] * nl + li] += den[k * nl + li];
        }
    double V = d->box_len * d->box_len * d->box_len;
    for (long b = 0; b < nbin; ++b)
        for (int li = 0; li < nl; ++li) {
            int l = 2 * li;
            double dn = sd[b * nl + li];
            B[b * nl + li] = dn > 0 ? sqrt((2.0 * l + 1.0) / (2.0 * BO_TWO_PI)) * sn[b * nl + li] / (V * dn) : NAN;
        }
    free(tri); free(nt); free(num); free(den); free(sn); free(sd);
    return n;
}
