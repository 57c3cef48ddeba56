// kernels.cu -- CUDA kernels of the bispectrum-multipole estimator
// (Gill & Bharadwaj, arXiv:2405.14513, Sec. II) for sm_103a.
//
//   k_fft_z_real    forward transform along the line of sight (real rows),
//                   keeping planes 0..N_g/3, written plane-major
//   k_fft_rows_T    batched row transforms written transposed (the y and x
//                   passes of the forward transform; second pass of Step I)
//   k_ring_gather   Step I first pass: ring mask (and fold onto the M x M
//                   reduction grid) fused into the load, transform along u_y
//   k_step2         Step II: partial triple sums sum_x D1 D2 D3 (Eq. fftbs)
//   k_reduce        partial sums -> S per combination, grid normalisation
//   k_epilogue      Y_lm weights, (k1, mu, t) binning and the ratio of
//                   Eq. bs_lm2_1; or the plan-time denominators
//   k_ntri          N_tri = M^-2 sum_y I1 I2 I3 on the unit fields (Eq. Ntri2)
//
// All transforms use exp(-i k.x), the sign of Eq. iFT.  Transform lengths
// are 2^q, 3 x 2^q, 5 x 2^q or 7 x 2^q (N_g and the reduction grids of the
// plan); the twiddle tables, computed on the host in double, are
// twF[k] = exp(-2 pi i k / (F x 2^lgF)), F = 1 (tw2), 3, 5, 7.
#include "kernels.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>

namespace bisp {

namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmk(double re, double im);
template <> __device__ __forceinline__ float2 cmk<float2>(double re, double im) { return make_float2(float(re), float(im)); }
template <> __device__ __forceinline__ double2 cmk<double2>(double re, double im) { return make_double2(re, im); }

// Field f = blockIdx.y of a batched launch: its buffers sit fs bytes apart.
template <typename T> __device__ __forceinline__ T *field_ptr(T *p, int64_t fs)
{
    return reinterpret_cast<T *>(reinterpret_cast<char *>(p) + int64_t(blockIdx.y) * fs);
}
template <typename T> __device__ __forceinline__ const T *field_ptr(const T *p, int64_t fs)
{
    return reinterpret_cast<const T *>(reinterpret_cast<const char *>(p) + int64_t(blockIdx.y) * fs);
}

// t = q d + r along t = t0, t0 + step, ...: quotient and remainder kept
// incrementally (one division per thread rather than one per element)
struct DivIter {
    int q, r, dq, dr, d;
    __device__ __forceinline__ DivIter(int t0, int step, int d_) : d(d_)
    {
        q = t0 / d;
        r = t0 - q * d;
        dq = step / d;
        dr = step - dq * d;
    }
    __device__ __forceinline__ void next()
    {
        q += dq;
        r += dr;
        if (r >= d) {
            r -= d;
            ++q;
        }
    }
};

// Shared-memory position of element i of a transform row: a padding slot
// after every 8 elements, so that the strided stores of the first radix-8
// stages (elements 8 and 64 apart) fall in different banks.  A row takes
// fft_stride(M) elements (kernels.cuh).
__device__ __forceinline__ int spos(int i) { return i + (i >> 3); }

// Stockham transform of nrows rows of length M = F x 2^q (F = 1, 3, 5 or 7)
// held in shared memory (row stride P), X_k = sum_j x_j exp(-2 pi i jk / M):
// one radix-F stage first when F > 1, then radix-8 stages and, for what is
// left of the power of two, one radix-4 or radix-2 stage.  Every thread of
// the block takes part; the caller synchronises before the call.  The result
// is in the returned buffer (a or b).  Every index split below is a shift, or
// a shift and a division by the constant F.
template <typename C, int F>
__device__ C *fft_smem_f(C *a, C *b, int M, int P, int nrows, const Twiddles<C> &tw)
{
    using Rr = decltype(a[0].x);
    const int p = __ffs(M) - 1;                 // M = F 2^p
    auto divF = [](int x) { return F == 1 ? x : int(unsigned(x) / unsigned(F)); };
    int Ns = 1;
    if (F == 3) {
        const int third = M / 3;
        const int total = nrows * third;
        const Rr h = Rr(0.86602540378443864676);   // sqrt(3)/2
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int row = t >> p, j = t & (third - 1);
            const C v0 = a[row * P + spos(j)], v1 = a[row * P + spos(j + third)], v2 = a[row * P + spos(j + 2 * third)];
            const Rr sx = v1.x + v2.x, sy = v1.y + v2.y, dx = v1.x - v2.x, dy = v1.y - v2.y;
            const Rr mx = v0.x - Rr(0.5) * sx, my = v0.y - Rr(0.5) * sy;
            C y0, y1, y2;
            y0.x = v0.x + sx; y0.y = v0.y + sy;
            y1.x = mx + h * dy; y1.y = my - h * dx;
            y2.x = mx - h * dy; y2.y = my + h * dx;
            b[row * P + spos(3 * j)] = y0;
            b[row * P + spos(3 * j + 1)] = y1;
            b[row * P + spos(3 * j + 2)] = y2;
        }
        __syncthreads();
        C *t2 = a;
        a = b;
        b = t2;
        Ns = 3;
    } else if (F == 5) {
        // 5-point DFT of v_k = x[j + k M/5], w = exp(-2 pi i/5):
        //   y_0 = v0 + s1 + s2,  s1 = v1 + v4,  s2 = v2 + v3,  d1 = v1 - v4,  d2 = v2 - v3,
        //   y_1, y_4 = v0 + c1 s1 + c2 s2 -/+ i (n1 d1 + n2 d2),
        //   y_2, y_3 = v0 + c2 s1 + c1 s2 -/+ i (n2 d1 - n1 d2),
        // c_m = cos(2 pi m/5), n_m = sin(2 pi m/5)
        const int fifth = M / 5;
        const int total = nrows * fifth;
        const Rr c1 = Rr(0.30901699437494742410), c2 = Rr(-0.80901699437494742410);
        const Rr n1 = Rr(0.95105651629515357212), n2 = Rr(0.58778525229247312917);
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int row = t >> p, j = t & (fifth - 1);
            const C *src = a + row * P;
            const C v0 = src[spos(j)], v1 = src[spos(j + fifth)], v2 = src[spos(j + 2 * fifth)], v3 = src[spos(j + 3 * fifth)],
                    v4 = src[spos(j + 4 * fifth)];
            const C s1 = cadd(v1, v4), s2 = cadd(v2, v3), d1 = csub(v1, v4), d2 = csub(v2, v3);
            C a1, a2, b1, b2;
            a1.x = v0.x + c1 * s1.x + c2 * s2.x; a1.y = v0.y + c1 * s1.y + c2 * s2.y;
            a2.x = v0.x + c2 * s1.x + c1 * s2.x; a2.y = v0.y + c2 * s1.y + c1 * s2.y;
            b1.x = n1 * d1.x + n2 * d2.x; b1.y = n1 * d1.y + n2 * d2.y;
            b2.x = n2 * d1.x - n1 * d2.x; b2.y = n2 * d1.y - n1 * d2.y;
            // -i b = (b.y, -b.x)
            C *dst = b + row * P;
            C y;
            y.x = v0.x + s1.x + s2.x; y.y = v0.y + s1.y + s2.y; dst[spos(5 * j)] = y;
            y.x = a1.x + b1.y; y.y = a1.y - b1.x; dst[spos(5 * j + 1)] = y;
            y.x = a2.x + b2.y; y.y = a2.y - b2.x; dst[spos(5 * j + 2)] = y;
            y.x = a2.x - b2.y; y.y = a2.y + b2.x; dst[spos(5 * j + 3)] = y;
            y.x = a1.x - b1.y; y.y = a1.y + b1.x; dst[spos(5 * j + 4)] = y;
        }
        __syncthreads();
        C *t2 = a;
        a = b;
        b = t2;
        Ns = 5;
    } else if (F == 7) {
        // 7-point DFT of v_k = x[j + k M/7], by the same pairing:
        //   s_k = v_k + v_{7-k},  d_k = v_k - v_{7-k}  (k = 1, 2, 3),
        //   y_m, y_{7-m} = v0 + sum_k cos(2 pi mk/7) s_k -/+ i sum_k sin(2 pi mk/7) d_k  (m = 1, 2, 3)
        const int sev = M / 7;
        const int total = nrows * sev;
        const Rr c1 = Rr(0.62348980185873353053), c2 = Rr(-0.22252093395631440429), c3 = Rr(-0.90096886790241912624);
        const Rr n1 = Rr(0.78183148246802980871), n2 = Rr(0.97492791218182360702), n3 = Rr(0.43388373911755812048);
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int row = t >> p, j = t & (sev - 1);
            const C *src = a + row * P;
            C v[7];
#pragma unroll
            for (int k = 0; k < 7; ++k) v[k] = src[spos(j + k * sev)];
            const C s1 = cadd(v[1], v[6]), s2 = cadd(v[2], v[5]), s3 = cadd(v[3], v[4]);
            const C d1 = csub(v[1], v[6]), d2 = csub(v[2], v[5]), d3 = csub(v[3], v[4]);
            C am[3], bm[3];
            am[0].x = v[0].x + c1 * s1.x + c2 * s2.x + c3 * s3.x; am[0].y = v[0].y + c1 * s1.y + c2 * s2.y + c3 * s3.y;
            am[1].x = v[0].x + c2 * s1.x + c3 * s2.x + c1 * s3.x; am[1].y = v[0].y + c2 * s1.y + c3 * s2.y + c1 * s3.y;
            am[2].x = v[0].x + c3 * s1.x + c1 * s2.x + c2 * s3.x; am[2].y = v[0].y + c3 * s1.y + c1 * s2.y + c2 * s3.y;
            bm[0].x = n1 * d1.x + n2 * d2.x + n3 * d3.x; bm[0].y = n1 * d1.y + n2 * d2.y + n3 * d3.y;
            bm[1].x = n2 * d1.x - n3 * d2.x - n1 * d3.x; bm[1].y = n2 * d1.y - n3 * d2.y - n1 * d3.y;
            bm[2].x = n3 * d1.x - n1 * d2.x + n2 * d3.x; bm[2].y = n3 * d1.y - n1 * d2.y + n2 * d3.y;
            C *dst = b + row * P;
            C y;
            y.x = v[0].x + s1.x + s2.x + s3.x; y.y = v[0].y + s1.y + s2.y + s3.y; dst[spos(7 * j)] = y;
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                // -i b = (b.y, -b.x)
                y.x = am[m].x + bm[m].y; y.y = am[m].y - bm[m].x; dst[spos(7 * j + m + 1)] = y;
                y.x = am[m].x - bm[m].y; y.y = am[m].y + bm[m].x; dst[spos(7 * j + 6 - m)] = y;
            }
        }
        __syncthreads();
        C *t2 = a;
        a = b;
        b = t2;
        Ns = 7;
    }
    const C *wt = F == 7 ? tw.tw7 : (F == 5 ? tw.tw5 : (F == 3 ? tw.tw3 : tw.tw2));
    const int lg = F == 7 ? tw.lg7 : (F == 5 ? tw.lg5 : (F == 3 ? tw.lg3 : tw.lg2));
    int s = 0;                                  // Ns = F 2^s
    while (Ns < M) {
        if (M / Ns >= 8) {
            // radix 8: v_r = x[j + r M/8] w^(rk), w = exp(-2 pi i / (8 Ns)),
            // out[q 8 Ns + k + m Ns] = sum_r v_r exp(-2 pi i rm / 8), as a
            // radix-2 step (pairs r, r + 4; the odd half turned by
            // exp(-2 pi i r / 8)) followed by two 4-point transforms
            const int eighth = M / 8;
            const int total = nrows * eighth;
            const int sh = lg - s - 3;
            const Rr r2 = Rr(0.70710678118654752440);   // 1/sqrt(2)
            for (int t = threadIdx.x; t < total; t += blockDim.x) {
                const int row = divF(t >> (p - 3));
                const int j = t - row * eighth;
                const int q = divF(j >> s);
                const int k = j - q * Ns;
                const C *src = a + row * P;
                C v[8];
                v[0] = src[spos(j)];
#pragma unroll
                for (int r = 1; r < 8; ++r) v[r] = cmul(src[spos(j + r * eighth)], __ldg(&wt[(r * k) << sh]));
                C e[4], o[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    e[r] = cadd(v[r], v[r + 4]);
                    o[r] = csub(v[r], v[r + 4]);
                }
                // o_1 exp(-i pi/4), o_2 (-i), o_3 exp(-3 i pi/4)
                {
                    const C t1 = o[1], t3 = o[3];
                    o[1].x = (t1.x + t1.y) * r2; o[1].y = (t1.y - t1.x) * r2;
                    const Rr x2 = o[2].x;
                    o[2].x = o[2].y; o[2].y = -x2;
                    o[3].x = (t3.y - t3.x) * r2; o[3].y = -(t3.x + t3.y) * r2;
                }
                C *dst = b + row * P;
                const int d0 = q * 8 * Ns + k;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const C *x = h ? o : e;
                    const C s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]), s13 = cadd(x[1], x[3]),
                            d13 = csub(x[1], x[3]);
                    C m1 = d02, m3 = d02;                 // d02 -/+ i d13
                    m1.x += d13.y; m1.y -= d13.x;
                    m3.x -= d13.y; m3.y += d13.x;
                    dst[spos(d0 + (0 + h) * Ns)] = cadd(s02, s13);
                    dst[spos(d0 + (2 + h) * Ns)] = m1;
                    dst[spos(d0 + (4 + h) * Ns)] = csub(s02, s13);
                    dst[spos(d0 + (6 + h) * Ns)] = m3;
                }
            }
            Ns *= 8;
            s += 3;
        } else if (M / Ns >= 4) {
            // radix 4: v_r = x[j + r M/4] w^(rk), w = exp(-2 pi i / (4 Ns)),
            // out[q 4 Ns + k + m Ns] = sum_r v_r (-i)^(rm)
            const int quarter = M / 4;
            const int total = nrows * quarter;
            const int sh = lg - s - 2;
            for (int t = threadIdx.x; t < total; t += blockDim.x) {
                const int row = divF(t >> (p - 2));
                const int j = t - row * quarter;
                const int q = divF(j >> s);
                const int k = j - q * Ns;
                const C *src = a + row * P;
                const C v0 = src[spos(j)];
                const C v1 = cmul(src[spos(j + quarter)], __ldg(&wt[k << sh]));
                const C v2 = cmul(src[spos(j + 2 * quarter)], __ldg(&wt[(2 * k) << sh]));
                const C v3 = cmul(src[spos(j + 3 * quarter)], __ldg(&wt[(3 * k) << sh]));
                const C s02 = cadd(v0, v2), d02 = csub(v0, v2), s13 = cadd(v1, v3), d13 = csub(v1, v3);
                C *dst = b + row * P;
                const int d0 = q * 4 * Ns + k;
                dst[spos(d0)] = cadd(s02, s13);
                dst[spos(d0 + 2 * Ns)] = csub(s02, s13);
                // -i d13 = (d13.y, -d13.x)
                C m1 = d02, m3 = d02;
                m1.x += d13.y; m1.y -= d13.x;
                m3.x -= d13.y; m3.y += d13.x;
                dst[spos(d0 + Ns)] = m1;
                dst[spos(d0 + 3 * Ns)] = m3;
            }
            Ns *= 4;
            s += 2;
        } else {
            const int half = M / 2;
            const int total = nrows * half;
            const int sh = lg - s - 1;
            for (int t = threadIdx.x; t < total; t += blockDim.x) {
                const int row = divF(t >> (p - 1));
                const int j = t - row * half;
                const int q = divF(j >> s);
                const int k = j - q * Ns;
                C v0 = a[row * P + spos(j)];
                C v1 = cmul(a[row * P + spos(j + half)], __ldg(&wt[k << sh]));
                const int idx = q * 2 * Ns + k;
                b[row * P + spos(idx)] = cadd(v0, v1);
                b[row * P + spos(idx + Ns)] = csub(v0, v1);
            }
            Ns *= 2;
            s += 1;
        }
        __syncthreads();
        C *t2 = a;
        a = b;
        b = t2;
    }
    return a;
}

// Transform of rows of length M = 2^q, 3 x 2^q, 5 x 2^q or 7 x 2^q
// (block-uniform dispatch)
template <typename C>
__device__ __forceinline__ C *fft_smem(C *a, C *b, int M, int P, int nrows, const Twiddles<C> &tw)
{
    const int odd = M >> (__ffs(M) - 1);
    if (odd == 7) return fft_smem_f<C, 7>(a, b, M, P, nrows, tw);
    if (odd == 5) return fft_smem_f<C, 5>(a, b, M, P, nrows, tw);
    if (odd == 3) return fft_smem_f<C, 3>(a, b, M, P, nrows, tw);
    return fft_smem_f<C, 1>(a, b, M, P, nrows, tw);
}

// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
k_fft_z_real(const R *__restrict__ in, typename Cx<R>::T *__restrict__ out, int M, int64_t rows,
             int nkeep, int rt, Twiddles<typename Cx<R>::T> tw, int64_t fs_in, int64_t fs_out)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    in = field_ptr(in, fs_in);
    out = field_ptr(out, fs_out);
    const int P = fft_stride(M);
    C *a = reinterpret_cast<C *>(smem_raw);
    C *b = a + rt * P;
    const int64_t row0 = int64_t(blockIdx.x) * rt;
    const int nrow = int(min(int64_t(rt), rows - row0));
    DivIter ld(threadIdx.x, blockDim.x, M);
    for (int t = threadIdx.x; t < nrow * M; t += blockDim.x, ld.next()) {
        const int r = ld.q, j = ld.r;
        a[r * P + spos(j)] = cmk<C>(double(in[(row0 + r) * M + j]), 0.0);
    }
    __syncthreads();
    const C *res = fft_smem(a, b, M, P, nrow, tw);
    DivIter st(threadIdx.x, blockDim.x, nrow);
    for (int t = threadIdx.x; t < nkeep * nrow; t += blockDim.x, st.next()) {
        const int k = st.q, r = st.r;
        out[int64_t(k) * rows + row0 + r] = res[r * P + spos(k)];
    }
}

template <typename R>
__global__ void __launch_bounds__(256)
k_fft_rows_T(const typename Cx<R>::T *__restrict__ in, typename Cx<R>::T *__restrict__ out, int M,
             int nrow, int ntile, const int64_t *__restrict__ out_off, R scale, int zero_dc, int rt,
             Twiddles<typename Cx<R>::T> tw, int64_t fs)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    in = field_ptr(in, fs);
    out = field_ptr(out, fs);
    const int P = fft_stride(M);
    C *a = reinterpret_cast<C *>(smem_raw);
    C *b = a + rt * P;
    const int64_t bt = blockIdx.x / ntile;
    const int tile = int(blockIdx.x - bt * ntile);
    const int row0 = tile * rt;
    const int nr = min(rt, nrow - row0);
    const C *src = in + bt * int64_t(M) * nrow;
    DivIter ld(threadIdx.x, blockDim.x, M);
    for (int t = threadIdx.x; t < nr * M; t += blockDim.x, ld.next()) {
        const int r = ld.q, j = ld.r;
        a[r * P + spos(j)] = src[int64_t(row0 + r) * M + j];
    }
    __syncthreads();
    const C *res = fft_smem(a, b, M, P, nr, tw);
    C *dst = out + (out_off ? out_off[bt] : bt * int64_t(M) * nrow);
    DivIter st(threadIdx.x, blockDim.x, nr);
    for (int t = threadIdx.x; t < M * nr; t += blockDim.x, st.next()) {
        const int k = st.q, r = st.r;
        C v = res[r * P + spos(k)];
        v.x *= scale;
        v.y *= scale;
        if (zero_dc && bt == 0 && row0 + r == 0 && k == 0) v = cmk<C>(0.0, 0.0);
        dst[int64_t(k) * nrow + row0 + r] = v;
    }
}

template <typename R, bool UNIT>
__global__ void __launch_bounds__(256)
k_ring_gather(const typename Cx<R>::T *__restrict__ planes, int ng, RingArg rings,
              const Job *__restrict__ jobs, int M, int ntile, int rt, typename Cx<R>::T *__restrict__ gt,
              Twiddles<typename Cx<R>::T> tw, int64_t fs)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    planes = field_ptr(planes, fs);
    gt = field_ptr(gt, fs);
    const int P = fft_stride(M);
    C *a = reinterpret_cast<C *>(smem_raw);
    C *b = a + rt * P;
    const int64_t jb = blockIdx.x / ntile;
    const int tile = int(blockIdx.x - jb * ntile);
    const Job J = jobs[jb];
    const C *pl = planes + int64_t(J.n) * ng * ng;
    const int64_t lo = rings.e3sq[J.r], hi = rings.e3sq[J.r + 1];
    const int mc = rings.maxc[J.r];
    const int row0 = tile * rt;
    const int nr = min(rt, M - row0);
    // rows i hold ring members only where |u_x| <= maxc for u_x = i or i - M;
    // a block of rows without members is zero after the transform too, and
    // the column pass reads such rows as zero without loading them
    if (row0 > mc && row0 + nr - 1 < M - mc) return;
    DivIter ld(threadIdx.x, blockDim.x, M);
    for (int t = threadIdx.x; t < nr * M; t += blockDim.x, ld.next()) {
        const int tr = ld.q, j = ld.r;
        const int i = row0 + tr;
        R vr = 0, vi = 0;
        // members u with u_x = i or i - M and u_y = j or j - M (mod M folding;
        // |u_x|, |u_y| <= maxc < M, so no other alias exists)
#pragma unroll
        for (int ca = 0; ca < 2; ++ca) {
            const int ux = ca ? i - M : i;
            if (ux > mc || ux < -mc) continue;
#pragma unroll
            for (int cb = 0; cb < 2; ++cb) {
                const int uy = cb ? j - M : j;
                if (uy > mc || uy < -mc) continue;
                const int64_t q9 = 9 * (int64_t(ux) * ux + int64_t(uy) * uy);
                if (q9 < lo || q9 >= hi) continue;
                if (UNIT) {
                    vr += R(1);
                } else {
                    const C v = pl[int64_t(ux < 0 ? ux + ng : ux) * ng + (uy < 0 ? uy + ng : uy)];
                    vr += v.x;
                    vi += v.y;
                }
            }
        }
        a[tr * P + spos(j)] = cmk<C>(double(vr), double(vi));
    }
    __syncthreads();
    const C *res = fft_smem(a, b, M, P, nr, tw);
    // rows of the job's M x M field in place (u_x, k_y), whole rows: coalesced
    C *dst = gt + jb * int64_t(M) * M + int64_t(row0) * M;
    DivIter st(threadIdx.x, blockDim.x, M);
    for (int t = threadIdx.x; t < M * nr; t += blockDim.x, st.next()) {
        const int r = st.q, k = st.r;
        dst[t] = res[r * P + spos(k)];
    }
}

// Step I second pass: transforms along the first axis of each job's M x M
// field (rows u_x of the gather's output), a strip of w columns k_y per
// block, read and written in place order (runs of w consecutive elements
// of every row), so the D field comes out as [k_x][k_y].
template <typename R>
__global__ void __launch_bounds__(256)
k_fft_cols(const typename Cx<R>::T *__restrict__ in, typename Cx<R>::T *__restrict__ out, int M, int ntile, int w,
           const int64_t *__restrict__ out_off, const Job *__restrict__ jobs, RingArg rings,
           Twiddles<typename Cx<R>::T> tw, int64_t fs)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    in = field_ptr(in, fs);
    out = field_ptr(out, fs);
    const int P = fft_stride(M);
    C *a = reinterpret_cast<C *>(smem_raw);
    C *b = a + w * P;
    const int64_t jb = blockIdx.x / ntile;
    const int c0 = int(blockIdx.x - jb * ntile) * w;
    const int nc = min(w, M - c0);
    const C *src = in + jb * int64_t(M) * M + c0;
    const int mc = rings.maxc[jobs[jb].r];      // rows mc < i < M - mc hold no ring member: zero
    DivIter ld(threadIdx.x, blockDim.x, nc);
    for (int t = threadIdx.x; t < M * nc; t += blockDim.x, ld.next()) {
        const int i = ld.q, c = ld.r;
        a[c * P + spos(i)] = (i <= mc || i >= M - mc) ? src[int64_t(i) * M + c] : cmk<C>(0.0, 0.0);
    }
    __syncthreads();
    const C *res = fft_smem(a, b, M, P, nc, tw);
    C *dst = out + out_off[jb] + c0;
    DivIter st(threadIdx.x, blockDim.x, nc);
    for (int t = threadIdx.x; t < M * nc; t += blockDim.x, st.next()) {
        const int k = st.q, c = st.r;
        dst[int64_t(k) * M + c] = res[c * P + spos(k)];
    }
}

// ---------------------------------------------------------------------------
// Step II (Eq. fftbs): S(r1, r2, r3) = sum over the M x M grid of
// D(r1, n1) D(r2, n2) D(r3, n3), for every combination of a plane pair.
//
// One block per unit: an x chunk of one group (plane pair and grid) and up
// to NW of its tiles, one tile per warp.  The block stages the unit's rings
// of the three planes for TX grid points at a time in shared memory
// ([slot][x], x contiguous), double-buffered with cp.async.  The lanes of a
// warp take consecutive grid points, so every shared-memory load is
// conflict free.  Per point a lane forms the 8 row products
// P_i = D(r1_i, n1) D(r2_i, n2) once and accumulates Re(P_i D(w0 + j, n3))
// for the 8 r3 of the tile's window: 64 sums in registers over the whole
// chunk, reduced across the warp at the end.  Negative planes enter through
// D(r, -n) = conj D(r, n) as sign factors.  Blocks of 4, 8 and 16 warps
// (unit classes) let small units share an SM.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

template <typename R, int NW>
__global__ void __launch_bounds__(32 * NW, (sizeof(R) == 8 ? 8 : 16) / NW)
k_step2(StepIIArgs args, int64_t unit0, const typename Cx<R>::T *__restrict__ dstore, int smem_bytes)
{
    dstore = field_ptr(dstore, args.fs);
    args.partials = field_ptr(args.partials, args.fs);
    using C = typename Cx<R>::T;
    constexpr int NT = 32 * NW;
    constexpr int PER16 = 16 / sizeof(C);     // complex values per 16-byte copy
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Unit U = args.units[unit0 + blockIdx.x];
    const Group G = args.groups[U.group];
    const int lev = G.lev;
    const int64_t M2 = int64_t(G.M) * G.M;
    const int64_t x0 = int64_t(U.chunk) * args.x_chunk;
    const int64_t x1 = min(M2, x0 + args.x_chunk);
    const int nq0 = U.rhi[0] - U.rlo[0] + 1, nq1 = U.rhi[1] - U.rlo[1] + 1, nq2 = U.rhi[2] - U.rlo[2] + 1;
    const int ns = nq0 + nq1 + nq2;

    int64_t *offs = reinterpret_cast<int64_t *>(smem_raw);
    const size_t off = (size_t(ns) * sizeof(int64_t) + 127) & ~size_t(127);
    C *buf = reinterpret_cast<C *>(smem_raw + off);
    // grid points per stage: as many as fit, a multiple of 64, at most 256
    int TX = int((size_t(smem_bytes) - off) / (2 * size_t(ns) * sizeof(C)));
    TX = min(256, TX & ~63);
    const size_t stage_elems = size_t(ns) * TX;

    for (int s = threadIdx.x; s < ns; s += NT) {
        const int q = s < nq0 ? 0 : (s < nq0 + nq1 ? 1 : 2);
        const int r = U.rlo[q] + s - (q == 0 ? 0 : (q == 1 ? nq0 : nq0 + nq1));
        const int n = q == 0 ? G.n1 : (q == 1 ? G.n2 : G.n3);
        offs[s] = r < args.nr ? args.doff[(size_t(lev) * args.nz1 + (n < 0 ? -n : n)) * kMaxRings + r] : -1;
    }
    __syncthreads();

    // sign factors of conj(D) for negative planes: with D1 -> (a.x, g1 a.y),
    // D2 -> (b.x, g2 b.y), D3 -> (c.x, g3 c.y):
    //   Re(P D3) = Pr c.x - g3 Pi c.y,  Pr = a.x b.x - g1 g2 a.y b.y,
    //   g3 Pi = g3 g2 a.x b.y + g3 g1 a.y b.x
    const R g1 = G.n1 < 0 ? R(-1) : R(1), g2 = G.n2 < 0 ? R(-1) : R(1), g3 = G.n3 < 0 ? R(-1) : R(1);
    const R k12 = -g1 * g2, k32 = g3 * g2, k31 = g3 * g1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool active = warp < U.nt;
    Tile T;
    if (active) T = args.tiles[U.t0 + warp];
    R a[kTileRows * kTileCols];
#pragma unroll
    for (int i = 0; i < kTileRows * kTileCols; ++i) a[i] = R(0);

    const int nstage = int((x1 - x0 + TX - 1) / TX);
    auto issue = [&](int st) {
        C *dst = buf + size_t(st & 1) * stage_elems;
        const int64_t xs = x0 + int64_t(st) * TX;
        const int nx = int(min(int64_t(TX), x1 - xs));
        const int per = TX / PER16;                   // 16-byte pieces per slot row
        for (int k = threadIdx.x; k < ns * per; k += NT) {
            const int s = k / per, c = (k - s * per) * PER16;
            C *d = dst + size_t(s) * TX + c;
            if (offs[s] >= 0 && c < nx) cp_async16(d, dstore + offs[s] + xs + c);
            else *reinterpret_cast<float4 *>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };
    issue(0);
    for (int st = 0; st < nstage; ++st) {
        if (st + 1 < nstage) {
            issue(st + 1);
            asm volatile("cp.async.wait_group 1;\n" ::);
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::);
        }
        __syncthreads();
        const C *b = buf + size_t(st & 1) * stage_elems;
        const int nx = int(min(int64_t(TX), x1 - (x0 + int64_t(st) * TX)));
        if (active) {
            // per-stage slot pointers (lane offset included); the x loop
            // advances them by 64 points and reads two points per lane
            const int o3 = T.s3 * TX + lane;
            int o1[kTileRows], o2[kTileRows];
#pragma unroll
            for (int i = 0; i < kTileRows; ++i) {
                o1[i] = T.s1[i] * TX + lane;
                o2[i] = T.s2[i] * TX + lane;
            }
            for (int xc = 0; xc < nx; xc += 64) {
#pragma unroll 1
                for (int h = 0; h < 2; ++h) {
                    const int x = xc + 32 * h;
                    C w[kTileCols];
#pragma unroll
                    for (int j = 0; j < kTileCols; ++j) w[j] = b[o3 + j * TX + x];
#pragma unroll
                    for (int i = 0; i < kTileRows; ++i) {
                        const C u = b[o1[i] + x];
                        const C v = b[o2[i] + x];
                        const R pr = fma(u.x, v.x, k12 * (u.y * v.y));
                        const R npi = -fma(k32 * u.x, v.y, k31 * (u.y * v.x));
#pragma unroll
                        for (int j = 0; j < kTileCols; ++j) {
                            R &acc = a[i * kTileCols + j];
                            acc = fma(pr, w[j].x, acc);
                            acc = fma(npi, w[j].y, acc);
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    if (!active) return;
    // butterfly reduction across the warp: after the step with offset o the
    // lane keeps the half of its sums selected by (lane & o); at the end lane
    // l holds the sums of tile entries 2 l and 2 l + 1
#pragma unroll
    for (int o = 16, n = kTileRows * kTileCols / 2; o >= 1; o >>= 1, n >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < kTileRows * kTileCols / 2; ++k) {
            if (k >= n) break;
            const R keep = up ? a[k + n] : a[k];
            const R give = up ? a[k] : a[k + n];
            a[k] = keep + __shfl_xor_sync(0xffffffffu, give, o);
        }
    }
    double *dst = args.partials + G.part0 + int64_t(U.chunk) * G.ncombo;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int idx = 2 * lane + k;
        if ((T.mask[idx >> 5] >> (idx & 31)) & 1u) dst[T.coff[idx / kTileCols] + (idx % kTileCols)] = double(a[k]);
    }
}

template <typename A>
__global__ void __launch_bounds__(256)
k_reduce(const Group *__restrict__ groups, const double *__restrict__ partials, int ng, double *__restrict__ S,
         int64_t fs)
{
    partials = field_ptr(partials, fs);
    S = field_ptr(S, fs);
    const Group G = groups[blockIdx.x];
    const double f = double(ng) / double(G.M);
    const A scale = A(f * f);
    for (int j = threadIdx.x; j < G.ncombo; j += blockDim.x) {
        A s = A(0);
        for (int k = 0; k < G.nchunk; ++k) s += A(partials[G.part0 + int64_t(k) * G.ncombo + j]);
        S[G.c0 + j] = double(s * scale);
    }
}

// Y_lm normalisation sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), and the prefactor
// sqrt((2l+1)/(4 pi)) of Eq. bs_lm2_1, set by set_ylm_constants.
__constant__ double c_nlm[9][9];
__constant__ double c_pref[9];
// Legendre recurrence ratios (2l+1)/(l+1-m) and (l+m)/(l+1-m), l, m <= 8
__constant__ double c_rec[2][9][9];

// W: type of the sums over records; Y: type the Y_lm of each record are
// computed in (FP32 for the FP32-transform paths, whose tolerance is 1e-4;
// FP64 for the FP64 path and the plan-time denominators).  The moments
// written are lm_lo .. (LMAX/2 + 1)^2 - 1 (even l from l_lo = 2 sqrt(lm_lo)),
// nlm_out = that count per bin, for out and den alike.
template <typename W, typename Y, int LMAX>
__global__ void __launch_bounds__(256)
k_epi_part(int mode, const Record *__restrict__ rec, const int64_t *__restrict__ chunk_lo,
           const int64_t *__restrict__ chunk_hi, int64_t nchunks, const double *__restrict__ value,
           double *__restrict__ partial, int64_t fs_in, int64_t fs_part)
{
    value = field_ptr(value, fs_in);
    partial = field_ptr(partial, fs_part);
    constexpr int NLM = (LMAX / 2 + 1) * (LMAX / 2 + 1);
    const int64_t ch = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (ch >= nchunks) return;   // whole warps leave together
    W acc[NLM];
#pragma unroll
    for (int i = 0; i < NLM; ++i) acc[i] = W(0);
    const int64_t k0 = chunk_lo[ch], k1 = chunk_hi[ch];
    for (int64_t k = k0 + lane; k < k1; k += 32) {
        const Record R = rec[k];
        const Y x = Y(R.pz), c = Y(R.cphi);
        const W mult = (R.flags & 1) ? W(1) : W(2);
        const W v = W(mode == 0 ? value[R.s_index] : value[k]) * mult;
        const bool deg = (R.flags & 2) != 0;
        const Y s = sqrt(max(Y(0), Y(1) - x * x));
        Y pmm = Y(1), tm1 = Y(1), tm2 = Y(1);   // P_m^m; cos(m phi), cos((m-1) phi)
#pragma unroll
        for (int m = 0; m <= LMAX; ++m) {
            Y tm;
            if (m == 0) tm = Y(1);
            else if (m == 1) tm = c;
            else tm = Y(2) * c * tm1 - tm2;
            if (m > 0) pmm *= -Y(2 * m - 1) * s;
            Y plm1 = Y(0), pl = pmm;                 // P_{l-1}^m, P_l^m at l = m
#pragma unroll
            for (int l = m; l <= LMAX; ++l) {
                if ((l & 1) == 0) {
                    const Y y = Y(c_nlm[l][m]) * pl;
                    const int idx = (l >> 1) * (l >> 1) + m;
                    if (mode == 0) {
                        const Y w = deg ? (m == 0 ? y : Y(0)) : y * tm;
                        acc[idx] += W(w) * v;
                    } else {
                        acc[idx] += W(y) * W(y) * v;
                    }
                }
                // P_{l+1}^m = ((2l+1) x P_l^m - (l+m) P_{l-1}^m) / (l+1-m), with
                // the two ratios from constant memory (no division per record)
                const Y pn = Y(c_rec[0][l][m]) * x * pl - Y(c_rec[1][l][m]) * plm1;
                plm1 = pl;
                pl = pn;
            }
            tm2 = tm1;
            tm1 = tm;
        }
    }
#pragma unroll
    for (int i = 0; i < NLM; ++i) {
        W v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) partial[ch * NLM + i] = double(v);
    }
}

// One thread per bin: its chunks' partial sums in chunk order, then (mode
// 0) the ratio of Eq. bs_lm2_1 or (mode 1) the sum itself.
template <int LMAX>
__global__ void __launch_bounds__(256)
k_epi_fin(int mode, const int64_t *__restrict__ bin_chunk, int64_t nbins, const double *__restrict__ partial,
          const double *__restrict__ den, double norm, double *__restrict__ out, int64_t fs_part, int64_t fs_out,
          int lm_lo, int nlm_out)
{
    partial = field_ptr(partial, fs_part);
    out = field_ptr(out, fs_out);
    constexpr int NLM = (LMAX / 2 + 1) * (LMAX / 2 + 1);
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    const int64_t c0 = bin_chunk[b], c1 = bin_chunk[b + 1];
    for (int i = lm_lo; i < NLM; ++i) {
        double v = 0.0;
        for (int64_t ch = c0; ch < c1; ++ch) v += partial[ch * NLM + i];
        const int64_t o = b * nlm_out + (i - lm_lo);
        if (mode == 0) {
            int l = 0;
            while ((l / 2 + 1) * (l / 2 + 1) <= i) l += 2;
            const double d = den[o];
            out[o] = d > 0.0 ? c_pref[l] * v * norm / d : __longlong_as_double(0x7ff8000000000000LL);
        } else {
            out[o] = v;
        }
    }
}

// Running statistics of estimates over fields: Welford's update (mean and
// sum of squared deviations, FP64) of element i with B[f][i], f < nf, in
// field order; non-finite values (empty bins) are skipped.
__global__ void __launch_bounds__(256)
k_stats_update(const double *__restrict__ B, int nf, int64_t n, int64_t *__restrict__ count,
               double *__restrict__ mean, double *__restrict__ m2)
{
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t c = count[i];
    double m = mean[i], s = m2[i];
    for (int f = 0; f < nf; ++f) {
        const double x = B[int64_t(f) * n + i];
        if (!isfinite(x)) continue;
        ++c;
        const double d = x - m;
        m += d / double(c);
        s += d * (x - m);
    }
    count[i] = c;
    mean[i] = m;
    m2[i] = s;
}

__global__ void __launch_bounds__(256)
k_ntri(const double2 *__restrict__ I, const int64_t *__restrict__ ioff, const int32_t *__restrict__ tri,
       GridArg grids, double *__restrict__ raw)
{
    __shared__ double red[8];
    const int r1 = tri[4 * blockIdx.x], r2 = tri[4 * blockIdx.x + 1], r3 = tri[4 * blockIdx.x + 2];
    const int lev = tri[4 * blockIdx.x + 3];
    const int64_t M2 = int64_t(grids.M[lev]) * grids.M[lev];
    const double2 *a = I + ioff[lev * kMaxRings + r1];
    const double2 *b = I + ioff[lev * kMaxRings + r2];
    const double2 *c = I + ioff[lev * kMaxRings + r3];
    double s = 0;
    for (int64_t y = threadIdx.x; y < M2; y += blockDim.x) {
        const double2 p = cmul(cmul(a[y], b[y]), c[y]);
        s += p.x;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
        raw[blockIdx.x] = t / double(M2);
    }
}

}  // namespace

size_t fft_rows_per_block(int M, size_t elem, size_t bytes)
{
    size_t rt = bytes / (size_t(M) * elem);
    if (rt < 1) rt = 1;
    if (rt > 256) rt = 256;
    return rt;
}

template <typename R>
cudaError_t launch_fft_z_real(const R *in, typename Cx<R>::T *out, int ng, int64_t rows, int nkeep,
                              const Twiddles<typename Cx<R>::T> &tw, const Batch &fb, cudaStream_t s, int rt)
{
    using C = typename Cx<R>::T;
    if (rt <= 0) rt = int(fft_rows_per_block(ng, sizeof(C)));
    const size_t smem = size_t(2) * rt * fft_stride(ng) * sizeof(C);
    const int64_t nblk = (rows + rt - 1) / rt;
    k_fft_z_real<R><<<dim3(unsigned(nblk), fb.nf), 256, smem, s>>>(in, out, ng, rows, nkeep, rt, tw, fb.fs_in,
                                                                   fb.fs_out);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fft_rows_T(const typename Cx<R>::T *in, typename Cx<R>::T *out, int M, int nrow,
                              int64_t nb, const int64_t *out_off, R scale, bool zero_dc,
                              const Twiddles<typename Cx<R>::T> &tw, const Batch &fb, cudaStream_t s, int rt)
{
    using C = typename Cx<R>::T;
    if (rt <= 0) rt = int(fft_rows_per_block(M, sizeof(C)));
    rt = std::min(rt, nrow);
    const size_t smem = size_t(2) * rt * fft_stride(M) * sizeof(C);
    const int ntile = (nrow + rt - 1) / rt;
    const int64_t nblk = nb * ntile;
    if (nblk == 0) return cudaSuccess;
    k_fft_rows_T<R><<<dim3(unsigned(nblk), fb.nf), 256, smem, s>>>(in, out, M, nrow, ntile, out_off, scale,
                                                                   zero_dc ? 1 : 0, rt, tw, fb.fs_in);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_ring_gather(const typename Cx<R>::T *planes, int ng, const RingArg &rings, const Job *jobs,
                               int64_t njobs, int M, bool unit, typename Cx<R>::T *gt,
                               const Twiddles<typename Cx<R>::T> &tw, const Batch &fb, cudaStream_t s, int rt)
{
    using C = typename Cx<R>::T;
    if (rt <= 0) rt = int(fft_rows_per_block(M, sizeof(C)));
    rt = std::min(rt, M);
    const size_t smem = size_t(2) * rt * fft_stride(M) * sizeof(C);
    const int ntile = (M + rt - 1) / rt;
    const int64_t nblk = njobs * ntile;
    if (nblk == 0) return cudaSuccess;
    const dim3 grid(unsigned(nblk), fb.nf);
    if (unit)
        k_ring_gather<R, true><<<grid, 256, smem, s>>>(planes, ng, rings, jobs, M, ntile, rt, gt, tw, fb.fs_in);
    else
        k_ring_gather<R, false><<<grid, 256, smem, s>>>(planes, ng, rings, jobs, M, ntile, rt, gt, tw, fb.fs_in);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fft_cols(const typename Cx<R>::T *in, typename Cx<R>::T *out, int M, int64_t njobs,
                            const int64_t *out_off, const Job *jobs, const RingArg &rings,
                            const Twiddles<typename Cx<R>::T> &tw, const Batch &fb, cudaStream_t s, int w)
{
    using C = typename Cx<R>::T;
    if (w <= 0) w = 8;
    w = std::min(w, M);
    const size_t smem = size_t(2) * w * fft_stride(M) * sizeof(C);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    const int ntile = (M + w - 1) / w;
    const int64_t nblk = njobs * ntile;
    if (nblk == 0) return cudaSuccess;
    k_fft_cols<R><<<dim3(unsigned(nblk), fb.nf), 256, smem, s>>>(in, out, M, ntile, w, out_off, jobs, rings, tw,
                                                                 fb.fs_in);
    return cudaGetLastError();
}

template <typename R, int NW>
cudaError_t launch_step2_class(const StepIIArgs &a, const typename Cx<R>::T *dstore, int64_t u0, int64_t n,
                               size_t smem, int nf, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_step2<R, NW><<<dim3(unsigned(n), nf), 32 * NW, smem, s>>>(a, u0, dstore, int(smem));
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_step2(const StepIIArgs &a, const typename Cx<R>::T *dstore, const int64_t *lo, const int64_t *hi,
                         int nf, cudaStream_t s)
{
    if constexpr (sizeof(R) == 4) {
        cudaError_t e = launch_step2_class<R, 4>(a, dstore, lo[2], hi[2] - lo[2], kStep2ClassSmem[2], nf, s);
        if (e == cudaSuccess)
            e = launch_step2_class<R, 8>(a, dstore, lo[3], hi[3] - lo[3], kStep2ClassSmem[3], nf, s);
        if (e == cudaSuccess)
            e = launch_step2_class<R, 16>(a, dstore, lo[4], hi[4] - lo[4], kStep2ClassSmem[4], nf, s);
        return e;
    }
    // FP64: register tiles, blocks of at most 8 warps (register file)
    cudaError_t e = launch_step2_class<R, 4>(a, dstore, lo[2], hi[2] - lo[2], kStep2ClassSmem[2], nf, s);
    if (e == cudaSuccess)
        e = launch_step2_class<R, 8>(a, dstore, lo[3], hi[3] - lo[3], kStep2ClassSmem[3], nf, s);
    if (e == cudaSuccess && hi[4] != lo[4]) e = cudaErrorInvalidValue;
    return e;
}

template <typename A>
cudaError_t launch_reduce_partials(const Group *groups, int64_t ngroups, const double *partials, int ng,
                                   double *S, const Batch &fb, cudaStream_t s)
{
    if (ngroups == 0) return cudaSuccess;
    k_reduce<A><<<dim3(unsigned(ngroups), fb.nf), 256, 0, s>>>(groups, partials, ng, S, fb.fs_in);
    return cudaGetLastError();
}

template <typename W, typename Y, int LMAX>
cudaError_t epilogue_l(int mode, const EpiArgs &e, const double *value, const double *den, double norm, double *out,
                       const Batch &fb, int lo, int n, cudaStream_t s)
{
    const dim3 g1(unsigned((e.nchunks * 32 + 255) / 256), fb.nf), g2(unsigned((e.nbins + 255) / 256), fb.nf);
    if (e.nchunks > 0)
        k_epi_part<W, Y, LMAX><<<g1, 256, 0, s>>>(mode, e.rec, e.chunk_lo, e.chunk_hi, e.nchunks, value, e.partial,
                                                  fb.fs_in, e.fs_part);
    k_epi_fin<LMAX><<<g2, 256, 0, s>>>(mode, e.bin_chunk, e.nbins, e.partial, den, norm, out, e.fs_part, fb.fs_out,
                                       lo, n);
    return cudaGetLastError();
}

template <typename W, typename Y>
cudaError_t epilogue_lmax(int mode, const EpiArgs &e, const double *value, int l_lo, int l_hi, const double *den,
                          double norm, double *out, const Batch &fb, cudaStream_t s)
{
    const int lo = (l_lo / 2) * (l_lo / 2), n = (l_hi / 2 + 1) * (l_hi / 2 + 1) - lo;
    switch (l_hi) {
    case 0: return epilogue_l<W, Y, 0>(mode, e, value, den, norm, out, fb, lo, n, s);
    case 2: return epilogue_l<W, Y, 2>(mode, e, value, den, norm, out, fb, lo, n, s);
    case 4: return epilogue_l<W, Y, 4>(mode, e, value, den, norm, out, fb, lo, n, s);
    case 6: return epilogue_l<W, Y, 6>(mode, e, value, den, norm, out, fb, lo, n, s);
    case 8: return epilogue_l<W, Y, 8>(mode, e, value, den, norm, out, fb, lo, n, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename W>
cudaError_t launch_epilogue(int mode, const EpiArgs &e, const double *value, int l_lo, int l_hi, const double *den,
                            double norm, double *out, const Batch &fb, cudaStream_t s, bool fp32_weights)
{
    if (e.nbins == 0) return cudaSuccess;
    if (l_lo < 0 || l_lo > l_hi || (l_lo & 1)) return cudaErrorInvalidValue;
    if (fp32_weights) return epilogue_lmax<W, float>(mode, e, value, l_lo, l_hi, den, norm, out, fb, s);
    return epilogue_lmax<W, W>(mode, e, value, l_lo, l_hi, den, norm, out, fb, s);
}

// Every kernel that takes more than 48 KB of dynamic shared memory is
// allowed the 227 KB maximum once, up front, so that the launches of an
// estimate are plain stream work (capturable in a CUDA graph).
cudaError_t init_kernel_attributes()
{
    const int mx = 227 * 1024;
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *f) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    };
    set((const void *)k_fft_z_real<float>);
    set((const void *)k_fft_z_real<double>);
    set((const void *)k_fft_rows_T<float>);
    set((const void *)k_fft_rows_T<double>);
    set((const void *)k_fft_cols<float>);
    set((const void *)k_fft_cols<double>);
    set((const void *)k_ring_gather<float, false>);
    set((const void *)k_ring_gather<float, true>);
    set((const void *)k_ring_gather<double, false>);
    set((const void *)k_ring_gather<double, true>);
    set((const void *)k_step2<float, 4>);
    set((const void *)k_step2<float, 8>);
    set((const void *)k_step2<float, 16>);
    set((const void *)k_step2<double, 4>);
    set((const void *)k_step2<double, 8>);
    return e;
}

cudaError_t launch_stats_update(const double *B, int nf, int64_t n, int64_t *count, double *mean, double *m2,
                                cudaStream_t s)
{
    if (n == 0 || nf == 0) return cudaSuccess;
    k_stats_update<<<unsigned((n + 255) / 256), 256, 0, s>>>(B, nf, n, count, mean, m2);
    return cudaGetLastError();
}

cudaError_t launch_ntri(const double2 *ifields, const int64_t *ioff, const int32_t *triples, int64_t ntriples,
                        const GridArg &grids, double *raw, cudaStream_t s)
{
    if (ntriples == 0) return cudaSuccess;
    k_ntri<<<unsigned(ntriples), 256, 0, s>>>(ifields, ioff, triples, grids, raw);
    return cudaGetLastError();
}

cudaError_t set_ylm_constants(const double nlm[9][9], const double pref[9], cudaStream_t s)
{
    double rec[2][9][9] = {};
    for (int l = 0; l <= 8; ++l)
        for (int m = 0; m <= l; ++m) {
            rec[0][l][m] = double(2 * l + 1) / double(l + 1 - m);
            rec[1][l][m] = double(l + m) / double(l + 1 - m);
        }
    cudaError_t e = cudaMemcpyToSymbolAsync(c_nlm, nlm, sizeof(double) * 81, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_pref, pref, sizeof(double) * 9, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(c_rec, rec, sizeof(rec), 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the tables above live on this stack
    return e;
}

// explicit instantiations
template cudaError_t launch_fft_z_real<float>(const float *, float2 *, int, int64_t, int, const Twiddles<float2> &, const Batch &, cudaStream_t, int);
template cudaError_t launch_fft_z_real<double>(const double *, double2 *, int, int64_t, int, const Twiddles<double2> &, const Batch &, cudaStream_t, int);
template cudaError_t launch_fft_rows_T<float>(const float2 *, float2 *, int, int, int64_t, const int64_t *, float, bool, const Twiddles<float2> &, const Batch &, cudaStream_t, int);
template cudaError_t launch_fft_rows_T<double>(const double2 *, double2 *, int, int, int64_t, const int64_t *, double, bool, const Twiddles<double2> &, const Batch &, cudaStream_t, int);
template cudaError_t launch_ring_gather<float>(const float2 *, int, const RingArg &, const Job *, int64_t, int, bool, float2 *, const Twiddles<float2> &, const Batch &, cudaStream_t, int);
template cudaError_t launch_ring_gather<double>(const double2 *, int, const RingArg &, const Job *, int64_t, int, bool, double2 *, const Twiddles<double2> &, const Batch &, cudaStream_t, int);
template cudaError_t launch_fft_cols<float>(const float2 *, float2 *, int, int64_t, const int64_t *, const Job *,
                                            const RingArg &, const Twiddles<float2> &,
                                            const Batch &, cudaStream_t, int);
template cudaError_t launch_fft_cols<double>(const double2 *, double2 *, int, int64_t, const int64_t *, const Job *,
                                             const RingArg &,
                                             const Twiddles<double2> &, const Batch &, cudaStream_t, int);
template cudaError_t launch_step2<float>(const StepIIArgs &, const float2 *, const int64_t *, const int64_t *, int,
                                         cudaStream_t);
template cudaError_t launch_step2<double>(const StepIIArgs &, const double2 *, const int64_t *, const int64_t *, int,
                                          cudaStream_t);
template cudaError_t launch_reduce_partials<float>(const Group *, int64_t, const double *, int, double *, const Batch &, cudaStream_t);
template cudaError_t launch_reduce_partials<double>(const Group *, int64_t, const double *, int, double *, const Batch &, cudaStream_t);
template cudaError_t launch_epilogue<float>(int, const EpiArgs &, const double *, int, int, const double *, double,
                                            double *, const Batch &, cudaStream_t, bool);
template cudaError_t launch_epilogue<double>(int, const EpiArgs &, const double *, int, int, const double *, double,
                                             double *, const Batch &, cudaStream_t, bool);

}  // namespace bisp
