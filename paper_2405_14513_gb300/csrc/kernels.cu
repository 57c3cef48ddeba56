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
// All transforms use exp(-i k.x), the sign of Eq. iFT, with twiddles
// tw[k] = exp(-2 pi i k / 2^lg_tw) computed on the host in double.
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

// Stockham radix-2 transform of nrows rows of length 2^lg held in shared
// memory (row stride P), X_k = sum_j x_j exp(-2 pi i jk / M).  Every thread
// of the block takes part; the caller synchronises before the call.  The
// result is in the returned buffer (a or b).
template <typename C>
__device__ C *fft_smem(C *a, C *b, int lg, int P, int nrows, const C *__restrict__ tw, int lg_tw)
{
    const int half = 1 << (lg - 1);
    const int total = nrows << (lg - 1);
    for (int s = 0; s < lg; ++s) {
        const int Ns = 1 << s;
        const int tws = lg_tw - s - 1;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            const int row = t >> (lg - 1);
            const int j = t & (half - 1);
            const int k = j & (Ns - 1);
            C v0 = a[row * P + j];
            C v1 = cmul(a[row * P + j + half], __ldg(&tw[k << tws]));
            const int idx = ((j >> s) << (s + 1)) + k;
            b[row * P + idx] = cadd(v0, v1);
            b[row * P + idx + Ns] = csub(v0, v1);
        }
        __syncthreads();
        C *t2 = a;
        a = b;
        b = t2;
    }
    return a;
}

// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256)
k_fft_z_real(const R *__restrict__ in, typename Cx<R>::T *__restrict__ out, int lg, int64_t rows,
             int nkeep, int rt, const typename Cx<R>::T *__restrict__ tw, int lg_tw)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = 1 << lg, P = M + 1;
    C *a = reinterpret_cast<C *>(smem_raw);
    C *b = a + rt * P;
    const int64_t row0 = int64_t(blockIdx.x) * rt;
    const int nrow = int(min(int64_t(rt), rows - row0));
    for (int t = threadIdx.x; t < nrow * M; t += blockDim.x) {
        const int r = t >> lg, j = t & (M - 1);
        a[r * P + j] = cmk<C>(double(in[(row0 + r) * M + j]), 0.0);
    }
    __syncthreads();
    const C *res = fft_smem(a, b, lg, P, nrow, tw, lg_tw);
    for (int t = threadIdx.x; t < nkeep * nrow; t += blockDim.x) {
        const int k = t / nrow, r = t - k * nrow;
        out[int64_t(k) * rows + row0 + r] = res[r * P + k];
    }
}

template <typename R>
__global__ void __launch_bounds__(256)
k_fft_rows_T(const typename Cx<R>::T *__restrict__ in, typename Cx<R>::T *__restrict__ out, int lg,
             int nrow, int ntile, const int64_t *__restrict__ out_off, R scale, int zero_dc, int rt,
             const typename Cx<R>::T *__restrict__ tw, int lg_tw)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = 1 << lg, P = M + 1;
    C *a = reinterpret_cast<C *>(smem_raw);
    C *b = a + rt * P;
    const int64_t bt = blockIdx.x / ntile;
    const int tile = int(blockIdx.x - bt * ntile);
    const int row0 = tile * rt;
    const int nr = min(rt, nrow - row0);
    const C *src = in + bt * int64_t(M) * nrow;
    for (int t = threadIdx.x; t < nr * M; t += blockDim.x) {
        const int r = t >> lg, j = t & (M - 1);
        a[r * P + j] = src[int64_t(row0 + r) * M + j];
    }
    __syncthreads();
    const C *res = fft_smem(a, b, lg, P, nr, tw, lg_tw);
    C *dst = out + (out_off ? out_off[bt] : bt * int64_t(M) * nrow);
    for (int t = threadIdx.x; t < M * nr; t += blockDim.x) {
        const int k = t / nr, r = t - k * nr;
        C v = res[r * P + k];
        v.x *= scale;
        v.y *= scale;
        if (zero_dc && bt == 0 && row0 + r == 0 && k == 0) v = cmk<C>(0.0, 0.0);
        dst[int64_t(k) * nrow + row0 + r] = v;
    }
}

template <typename R, bool UNIT>
__global__ void __launch_bounds__(256)
k_ring_gather(const typename Cx<R>::T *__restrict__ planes, int ng, RingArg rings,
              const Job *__restrict__ jobs, int lg, int ntile, int rt, typename Cx<R>::T *__restrict__ gt,
              const typename Cx<R>::T *__restrict__ tw, int lg_tw)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = 1 << lg, P = M + 1;
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
    for (int t = threadIdx.x; t < nr * M; t += blockDim.x) {
        const int i = row0 + (t >> lg), j = t & (M - 1);
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
        a[(t >> lg) * P + j] = cmk<C>(double(vr), double(vi));
    }
    __syncthreads();
    const C *res = fft_smem(a, b, lg, P, nr, tw, lg_tw);
    C *dst = gt + jb * int64_t(M) * M;
    for (int t = threadIdx.x; t < M * nr; t += blockDim.x) {
        const int k = t / nr, r = t - k * nr;
        dst[int64_t(k) * M + row0 + r] = res[r * P + k];
    }
}

// ---------------------------------------------------------------------------
// Step II.  One block per item (a group's x chunk).  The block stages the
// rings of its three planes for TX grid points at a time in shared memory
// (conjugated for negative planes, D(r,-n) = conj D(r,n)), and each thread
// takes segments: P = D(r1,n1) D(r2,n2) once per point, then
// Re(P D(r3+j, n3)) for up to eight r3.  A: per-tile sums; S: block sums.
template <typename R, typename A, typename S>
__global__ void __launch_bounds__(256)
k_step2(StepIIArgs args, const typename Cx<R>::T *__restrict__ dstore)
{
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Item it = args.items[blockIdx.x];
    const Group G = args.groups[it.group];
    const int lg = G.log2m;
    const int64_t M2 = int64_t(1) << (2 * lg);
    const int64_t x0 = int64_t(it.chunk) * args.x_chunk;
    const int64_t x1 = min(M2, x0 + args.x_chunk);
    const int nr0 = G.rhi[0] - G.rlo[0] + 1, nr1 = G.rhi[1] - G.rlo[1] + 1, nr2 = G.rhi[2] - G.rlo[2] + 1;
    const int ns = nr0 + nr1 + nr2;
    const int TX = args.tx, TXP = TX + 1;

    S *acc = reinterpret_cast<S *>(smem_raw);
    size_t off = (size_t(G.ncombo) * sizeof(S) + 15) & ~size_t(15);
    int64_t *offs = reinterpret_cast<int64_t *>(smem_raw + off);
    off += size_t(ns) * sizeof(int64_t);
    int *cj = reinterpret_cast<int *>(smem_raw + off);
    off = (off + size_t(ns) * sizeof(int) + 15) & ~size_t(15);
    C *tile = reinterpret_cast<C *>(smem_raw + off);

    for (int j = threadIdx.x; j < G.ncombo; j += blockDim.x) acc[j] = S(0);
    const int nabs[3] = {G.n1 < 0 ? -G.n1 : G.n1, G.n2 < 0 ? -G.n2 : G.n2, G.n3 < 0 ? -G.n3 : G.n3};
    const int nsg[3] = {G.n1 < 0, G.n2 < 0, G.n3 < 0};
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        int q = s < nr0 ? 0 : (s < nr0 + nr1 ? 1 : 2);
        int r = G.rlo[q] + s - (q == 0 ? 0 : (q == 1 ? nr0 : nr0 + nr1));
        offs[s] = args.doff[(size_t(lg) * args.nz1 + nabs[q]) * kMaxRings + r];
        cj[s] = nsg[q];
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int64_t xs = x0; xs < x1; xs += TX) {
        const int nx = int(min(int64_t(TX), x1 - xs));
        for (int s = warp; s < ns; s += nwarp) {
            const int64_t o = offs[s];
            const R sg = cj[s] ? R(-1) : R(1);
            for (int x = lane; x < nx; x += 32) {
                C v = cmk<C>(0.0, 0.0);
                if (o >= 0) {   // every staged field is stored; a missing one reads as zero
                    v = dstore[o + xs + x];
                    v.y *= sg;
                }
                tile[s * TXP + x] = v;
            }
        }
        __syncthreads();
        for (int g = threadIdx.x; g < G.nseg; g += blockDim.x) {
            const Segment q = args.segs[G.seg0 + g];
            const C *t1 = tile + (q.r1 - G.rlo[0]) * TXP;
            const C *t2 = tile + (nr0 + q.r2 - G.rlo[1]) * TXP;
            const C *t3 = tile + (nr0 + nr1 + q.r3a - G.rlo[2]) * TXP;
            const int n = q.n;
            A p[kSegLen];
#pragma unroll
            for (int j = 0; j < kSegLen; ++j) p[j] = A(0);
            for (int x = 0; x < nx; ++x) {
                const C u = t1[x], v = t2[x];
                const A pr = A(u.x) * A(v.x) - A(u.y) * A(v.y);
                const A pi = A(u.x) * A(v.y) + A(u.y) * A(v.x);
#pragma unroll
                for (int j = 0; j < kSegLen; ++j)
                    if (j < n) {
                        const C w = t3[j * TXP + x];
                        p[j] += pr * A(w.x) - pi * A(w.y);
                    }
            }
#pragma unroll
            for (int j = 0; j < kSegLen; ++j)
                if (j < n) acc[q.coff + j] += S(p[j]);
        }
        __syncthreads();
    }
    double *dst = args.partials + G.part0 + int64_t(it.chunk) * G.ncombo;
    for (int j = threadIdx.x; j < G.ncombo; j += blockDim.x) dst[j] = double(acc[j]);
}

template <typename A>
__global__ void __launch_bounds__(256)
k_reduce(const Group *__restrict__ groups, const double *__restrict__ partials, int ng, double *__restrict__ S)
{
    const Group G = groups[blockIdx.x];
    const double f = double(ng) / double(1 << G.log2m);
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

template <typename W>
__global__ void __launch_bounds__(256)
k_epilogue(int mode, const Record *__restrict__ rec, const int64_t *__restrict__ bin_start, int64_t nbins,
           const double *__restrict__ value, int l_max, const double *__restrict__ den, double norm,
           double *__restrict__ out)
{
    constexpr int kMaxLm = 25;
    const int64_t b = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nbins) return;   // whole warps leave together
    W acc[kMaxLm];
#pragma unroll
    for (int i = 0; i < kMaxLm; ++i) acc[i] = W(0);
    const int64_t k0 = bin_start[b], k1 = bin_start[b + 1];
    for (int64_t k = k0 + lane; k < k1; k += 32) {
        const Record R = rec[k];
        const W x = W(R.pz), c = W(R.cphi);
        const W mult = (R.flags & 1) ? W(1) : W(2);
        const W v = W(mode == 0 ? value[R.s_index] : value[k]) * mult;
        const bool deg = (R.flags & 2) != 0;
        const W s = sqrt(max(W(0), W(1) - x * x));
        W pmm = W(1), tm1 = W(1), tm2 = W(1);   // P_m^m; cos(m phi), cos((m-1) phi)
        for (int m = 0; m <= l_max; ++m) {
            W tm;
            if (m == 0) tm = W(1);
            else if (m == 1) tm = c;
            else tm = W(2) * c * tm1 - tm2;
            if (m > 0) pmm *= -W(2 * m - 1) * s;
            W plm1 = W(0), pl = pmm;                 // P_{l-1}^m, P_l^m at l = m
            for (int l = m; l <= l_max; ++l) {
                if ((l & 1) == 0) {
                    const W y = W(c_nlm[l][m]) * pl;
                    const int idx = (l >> 1) * (l >> 1) + m;
                    if (mode == 0) {
                        const W w = deg ? (m == 0 ? y : W(0)) : y * tm;
                        acc[idx] += w * v;
                    } else {
                        acc[idx] += y * y * v;
                    }
                }
                const W pn = (W(2 * l + 1) * x * pl - W(l + m) * plm1) / W(l + 1 - m);
                plm1 = pl;
                pl = pn;
            }
            tm2 = tm1;
            tm1 = tm;
        }
    }
    const int nlm = (l_max / 2 + 1) * (l_max / 2 + 1);
    for (int i = 0; i < nlm; ++i) {
        W v = acc[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) {
            if (mode == 0) {
                int l = 0;
                while ((l / 2 + 1) * (l / 2 + 1) <= i) l += 2;
                const double d = den[b * nlm + i];
                out[b * nlm + i] = d > 0.0 ? c_pref[l] * double(v) * norm / d : __longlong_as_double(0x7ff8000000000000LL);
            } else {
                out[b * nlm + i] = double(v);
            }
        }
    }
}

__global__ void __launch_bounds__(256)
k_ntri(const double2 *__restrict__ I, const int64_t *__restrict__ ioff, const int32_t *__restrict__ tri,
       double *__restrict__ raw)
{
    __shared__ double red[8];
    const int r1 = tri[4 * blockIdx.x], r2 = tri[4 * blockIdx.x + 1], r3 = tri[4 * blockIdx.x + 2];
    const int lg = tri[4 * blockIdx.x + 3];
    const int64_t M2 = int64_t(1) << (2 * lg);
    const double2 *a = I + ioff[lg * kMaxRings + r1];
    const double2 *b = I + ioff[lg * kMaxRings + r2];
    const double2 *c = I + ioff[lg * kMaxRings + r3];
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

template <typename F>
cudaError_t set_smem(F f, size_t bytes)
{
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    return cudaSuccess;
}

int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

}  // namespace

size_t fft_rows_per_block(int M, size_t elem)
{
    size_t rt = 65536 / (size_t(M) * elem);
    if (rt < 1) rt = 1;
    if (rt > 256) rt = 256;
    return rt;
}

template <typename R>
cudaError_t launch_fft_z_real(const R *in, typename Cx<R>::T *out, int ng, int64_t rows, int nkeep,
                              const typename Cx<R>::T *tw, int lg_tw, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    const int lg = ilog2(ng);
    const int rt = int(fft_rows_per_block(ng, sizeof(C)));
    const size_t smem = size_t(2) * rt * (ng + 1) * sizeof(C);
    cudaError_t e = set_smem(k_fft_z_real<R>, smem);
    if (e != cudaSuccess) return e;
    const int64_t nblk = (rows + rt - 1) / rt;
    k_fft_z_real<R><<<unsigned(nblk), 256, smem, s>>>(in, out, lg, rows, nkeep, rt, tw, lg_tw);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_fft_rows_T(const typename Cx<R>::T *in, typename Cx<R>::T *out, int M, int nrow,
                              int64_t nb, const int64_t *out_off, R scale, bool zero_dc,
                              const typename Cx<R>::T *tw, int lg_tw, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    const int lg = ilog2(M);
    const int rt = int(std::min<size_t>(fft_rows_per_block(M, sizeof(C)), size_t(nrow)));
    const size_t smem = size_t(2) * rt * (M + 1) * sizeof(C);
    cudaError_t e = set_smem(k_fft_rows_T<R>, smem);
    if (e != cudaSuccess) return e;
    const int ntile = (nrow + rt - 1) / rt;
    const int64_t nblk = nb * ntile;
    if (nblk == 0) return cudaSuccess;
    k_fft_rows_T<R><<<unsigned(nblk), 256, smem, s>>>(in, out, lg, nrow, ntile, out_off, scale, zero_dc ? 1 : 0,
                                                      rt, tw, lg_tw);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_ring_gather(const typename Cx<R>::T *planes, int ng, const RingArg &rings, const Job *jobs,
                               int64_t njobs, int M, bool unit, typename Cx<R>::T *gt,
                               const typename Cx<R>::T *tw, int lg_tw, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    const int lg = ilog2(M);
    const int rt = int(std::min<size_t>(fft_rows_per_block(M, sizeof(C)), size_t(M)));
    const size_t smem = size_t(2) * rt * (M + 1) * sizeof(C);
    const int ntile = (M + rt - 1) / rt;
    const int64_t nblk = njobs * ntile;
    if (nblk == 0) return cudaSuccess;
    cudaError_t e;
    if (unit) {
        e = set_smem(k_ring_gather<R, true>, smem);
        if (e != cudaSuccess) return e;
        k_ring_gather<R, true><<<unsigned(nblk), 256, smem, s>>>(planes, ng, rings, jobs, lg, ntile, rt, gt, tw, lg_tw);
    } else {
        e = set_smem(k_ring_gather<R, false>, smem);
        if (e != cudaSuccess) return e;
        k_ring_gather<R, false><<<unsigned(nblk), 256, smem, s>>>(planes, ng, rings, jobs, lg, ntile, rt, gt, tw, lg_tw);
    }
    return cudaGetLastError();
}

template <typename R, typename A, typename S>
cudaError_t launch_step2(const StepIIArgs &a, const typename Cx<R>::T *dstore, int64_t nitems, size_t smem,
                         cudaStream_t s)
{
    if (nitems == 0) return cudaSuccess;
    cudaError_t e = set_smem(k_step2<R, A, S>, smem);
    if (e != cudaSuccess) return e;
    k_step2<R, A, S><<<unsigned(nitems), 256, smem, s>>>(a, dstore);
    return cudaGetLastError();
}

template <typename A>
cudaError_t launch_reduce_partials(const Group *groups, int64_t ngroups, const double *partials, int ng,
                                   double *S, cudaStream_t s)
{
    if (ngroups == 0) return cudaSuccess;
    k_reduce<A><<<unsigned(ngroups), 256, 0, s>>>(groups, partials, ng, S);
    return cudaGetLastError();
}

template <typename W>
cudaError_t launch_epilogue(int mode, const Record *rec, const int64_t *bin_start, int64_t nbins,
                            const double *value, int l_max, const double *den, double norm, double *out,
                            cudaStream_t s)
{
    if (nbins == 0) return cudaSuccess;
    const int64_t nblk = (nbins * 32 + 255) / 256;
    k_epilogue<W><<<unsigned(nblk), 256, 0, s>>>(mode, rec, bin_start, nbins, value, l_max, den, norm, out);
    return cudaGetLastError();
}

cudaError_t launch_ntri(const double2 *ifields, const int64_t *ioff, const int32_t *triples, int64_t ntriples,
                        double *raw, cudaStream_t s)
{
    if (ntriples == 0) return cudaSuccess;
    k_ntri<<<unsigned(ntriples), 256, 0, s>>>(ifields, ioff, triples, raw);
    return cudaGetLastError();
}

cudaError_t set_ylm_constants(const double nlm[9][9], const double pref[9], cudaStream_t s)
{
    cudaError_t e = cudaMemcpyToSymbolAsync(c_nlm, nlm, sizeof(double) * 81, 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbolAsync(c_pref, pref, sizeof(double) * 9, 0, cudaMemcpyHostToDevice, s);
}

// explicit instantiations
template cudaError_t launch_fft_z_real<float>(const float *, float2 *, int, int64_t, int, const float2 *, int, cudaStream_t);
template cudaError_t launch_fft_z_real<double>(const double *, double2 *, int, int64_t, int, const double2 *, int, cudaStream_t);
template cudaError_t launch_fft_rows_T<float>(const float2 *, float2 *, int, int, int64_t, const int64_t *, float, bool, const float2 *, int, cudaStream_t);
template cudaError_t launch_fft_rows_T<double>(const double2 *, double2 *, int, int, int64_t, const int64_t *, double, bool, const double2 *, int, cudaStream_t);
template cudaError_t launch_ring_gather<float>(const float2 *, int, const RingArg &, const Job *, int64_t, int, bool, float2 *, const float2 *, int, cudaStream_t);
template cudaError_t launch_ring_gather<double>(const double2 *, int, const RingArg &, const Job *, int64_t, int, bool, double2 *, const double2 *, int, cudaStream_t);
template cudaError_t launch_step2<float, float, float>(const StepIIArgs &, const float2 *, int64_t, size_t, cudaStream_t);
template cudaError_t launch_step2<float, float, double>(const StepIIArgs &, const float2 *, int64_t, size_t, cudaStream_t);
template cudaError_t launch_step2<double, double, double>(const StepIIArgs &, const double2 *, int64_t, size_t, cudaStream_t);
template cudaError_t launch_reduce_partials<float>(const Group *, int64_t, const double *, int, double *, cudaStream_t);
template cudaError_t launch_reduce_partials<double>(const Group *, int64_t, const double *, int, double *, cudaStream_t);
template cudaError_t launch_epilogue<float>(int, const Record *, const int64_t *, int64_t, const double *, int, const double *, double, double *, cudaStream_t);
template cudaError_t launch_epilogue<double>(int, const Record *, const int64_t *, int64_t, const double *, int, const double *, double, double *, cudaStream_t);

}  // namespace bisp
