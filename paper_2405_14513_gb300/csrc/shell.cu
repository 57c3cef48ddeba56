// shell.cu -- the spherical-shell estimator of the m = 0 multipoles, a
// comparison for the m = 0 subset of the ring/plane estimator (Gill &
// Bharadwaj, arXiv:2405.14513).  The shell-based FFT estimators the paper
// builds on (Sec. I) bin modes in spherical shells and weight each mode
// with its own direction, which reaches the m = 0 moments only:
//
//   shells  s = {k : e_s <= |k| < e_{s+1}}, |k| in 3D, the ring edges e of
//           Sec. II (same width rule, cut at N_g/3); s = 0 holds k = 0 only
//           and is not used; K_s = mean |k| over the shell
//   triples s1 >= s2 >= s3 >= 1 (so K1 >= K2 >= K3), accepted and binned in
//           (k1, mu, t) from (K1, K2, K3) as a ring combination is, and kept
//           when N_tri > 0
//   sums    over closed triangles k1 + k2 + k3 = 0 with k_i in s_i:
//           num_l = sum Y_l0(k1) Delta(k1) Delta(k2) Delta(k3),
//           den_l = sum Y_l0(k1)^2, N_tri = sum 1, Y_l0 = sqrt((2l+1)/4pi)
//           P_l(k_z/|k|), taken on the N_g^3 grid as N_g^-3 sum_x of
//           products of shell fields (the 3D form of the identity behind
//           Eq. fftbs; every component is below N_g/3, so nothing aliases)
//   result  B_l^0 = sqrt((2l+1)/4pi) sum num_l / (V sum den_l) over the
//           triples of a bin (as Eq. bs_lm2_1 with each triangle's own
//           Y_l0), NaN where the denominator is 0.
//
// Plan: shell table, triples, and the field-independent N_tri and den_l
// from FP64 unit fields.  Estimate: the forward transform (the kernels of
// the main path), the weighted shell spectra of every shell, 3D transforms
// (three passes of the row transform, each a cyclic transpose), FP32
// fields, FP32 triple products summed in FP64, binning.  Lengths N_g <= 128
// (the plan's FP64 sums over N_g^3 points per triple grow as N_g^6).
#include "kernels.cuh"

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace bisp {
int record_error(int code, const char *msg);
void clear_error();
}  // namespace bisp

using namespace bisp;

namespace {

constexpr double kShellTwoPi = 6.283185307179586476925286766559;
constexpr int kShellMaxNg = 128;

// One field of a batch: shell s, kind 0: Delta, 1: Delta Y_l0, 2: 1, 3: Y_l0^2
struct ShellJob {
    int s, kind, l, pad;
};

// sqrt((2l+1)/4pi) P_l(z), l = 0, 2, 4, 6
__device__ __forceinline__ double y_l0(int l, double z)
{
    const double z2 = z * z;
    double p;
    switch (l) {
    case 0: p = 1.0; break;
    case 2: p = 0.5 * (3.0 * z2 - 1.0); break;
    case 4: p = 0.125 * ((35.0 * z2 - 30.0) * z2 + 3.0); break;
    default: p = 0.0625 * (((231.0 * z2 - 315.0) * z2 + 105.0) * z2 - 5.0); break;
    }
    return sqrt((2.0 * l + 1.0) / (2.0 * kShellTwoPi)) * p;
}

// Weighted shell spectra on the N_g^3 grid, [job][a][b][c] with (a, b, c)
// the FFT indices of (k_x, k_y, k_z); Delta from the kept planes n >= 0
// ([n][k_x][k_y]) and Delta(k_x, k_y, -n) = conj Delta(-k_x, -k_y, n).
template <typename C>
__global__ void __launch_bounds__(256)
k_shell_spectrum(const C *__restrict__ planes, int ng, const int64_t *__restrict__ e3sq,
                 const ShellJob *__restrict__ jobs, C *__restrict__ out)
{
    const ShellJob J = jobs[blockIdx.y];
    const int64_t n3 = int64_t(ng) * ng * ng;
    C *dst = out + int64_t(blockIdx.y) * n3;
    const int64_t lo = e3sq[J.s], hi = e3sq[J.s + 1];
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n3; p += int64_t(gridDim.x) * blockDim.x) {
        const int a = int(p / (int64_t(ng) * ng)), b = int((p / ng) % ng), c = int(p % ng);
        const int i = a < ng / 2 ? a : a - ng, j = b < ng / 2 ? b : b - ng, n = c < ng / 2 ? c : c - ng;
        const int64_t q9 = 9 * (int64_t(i) * i + int64_t(j) * j + int64_t(n) * n);
        C v;
        v.x = 0;
        v.y = 0;
        if (q9 >= lo && q9 < hi) {
            double w = 1.0;
            if (J.kind == 1 || J.kind == 3) {
                const double y = y_l0(J.l, double(n) / sqrt(double(int64_t(i) * i + int64_t(j) * j + int64_t(n) * n)));
                w = J.kind == 1 ? y : y * y;
            }
            if (J.kind <= 1) {
                C d;
                if (n >= 0) {
                    d = planes[(int64_t(n) * ng + a) * ng + b];
                } else {
                    d = planes[(int64_t(-n) * ng + (ng - a) % ng) * ng + (ng - b) % ng];
                    d.y = -d.y;
                }
                v.x = decltype(v.x)(double(d.x) * w);
                v.y = decltype(v.y)(double(d.y) * w);
            } else {
                v.x = decltype(v.x)(w);
            }
        }
        dst[p] = v;
    }
}

template <typename C, typename R>
__global__ void __launch_bounds__(256) k_real_part(const C *__restrict__ in, R *__restrict__ out, int64_t n)
{
    for (int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < n; p += int64_t(gridDim.x) * blockDim.x)
        out[p] = in[p].x;
}

// out[q] = scale sum_p A[p] B[p] C[p] for the field triple of product q
// (products in R, the sum in FP64), one block per product; outputs whose
// index is a multiple of every_first (if > 0) take scale_first instead.
template <typename R>
__global__ void __launch_bounds__(256)
k_triple_products(const R *__restrict__ fields, int64_t n3, const int4 *__restrict__ prods, double scale,
                  int every_first, double scale_first, double *__restrict__ out)
{
    __shared__ double red[8];
    const int4 P = prods[blockIdx.x];
    const R *A = fields + int64_t(P.x) * n3, *B = fields + int64_t(P.y) * n3, *Cf = fields + int64_t(P.z) * n3;
    double acc = 0;
    for (int64_t p = threadIdx.x; p < n3; p += blockDim.x) acc += double(A[p] * B[p] * Cf[p]);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
        out[P.w] = t * (every_first > 0 && P.w % every_first == 0 ? scale_first : scale);
    }
}

// B[bin][li] = sqrt((2l+1)/4pi) sum num / (V sum den) over the bin's triples
__global__ void __launch_bounds__(256)
k_shell_bin(const int64_t *__restrict__ bin_start, const int32_t *__restrict__ bin_tri, int64_t nbins, int nl,
            const double *__restrict__ num, const double *__restrict__ den, double inv_v, double *__restrict__ B)
{
    const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (q >= nbins * nl) return;
    const int64_t b = q / nl;
    const int li = int(q - b * nl);
    double sn = 0, sd = 0;
    for (int64_t k = bin_start[b]; k < bin_start[b + 1]; ++k) {
        const int32_t t = bin_tri[k];
        sn += num[int64_t(t) * nl + li];
        sd += den[int64_t(t) * nl + li];
    }
    const int l = 2 * li;
    B[q] = sd > 0.0 ? sqrt((2.0 * l + 1.0) / (2.0 * kShellTwoPi)) * sn * inv_v / sd
                    : __longlong_as_double(0x7ff8000000000000LL);
}

unsigned blocks_for(int64_t n) { return unsigned(std::min<int64_t>((n + 255) / 256, 152 * 16)); }

}  // namespace

struct bisp_shell_plan {
    bisp_desc desc{};
    std::vector<double> edges;
    int ng = 0, nz = 0, ns = 0, nl = 0;
    std::vector<int64_t> e3sq;            // (3 e_s)^2, ns + 1
    std::vector<double> K;                // mean |k| per shell, grid units
    std::vector<int32_t> tri;             // accepted triples [n][3]
    std::vector<int32_t> tri_bin;
    std::vector<double> ntri, den;        // [n], [n][nl]
    int64_t nbins = 0;
    // device
    int64_t *d_e3sq = nullptr;
    ShellJob *d_jobs = nullptr;           // estimate fields: D_s, F_{s,l} (l >= 2), s >= 1
    int njobs = 0;
    int4 *d_prods = nullptr;              // estimate products: (F_{s1,l}, D_{s2}, D_{s3}) -> num [t][li]
    double *d_den = nullptr;
    int64_t *d_bin_start = nullptr;
    int32_t *d_bin_tri = nullptr;
    float2 *tw2f = nullptr, *tw3f = nullptr;
    double2 *tw2d = nullptr, *tw3d = nullptr;
    Twiddles<float2> twf{};
    Twiddles<double2> twd{};
    // workspace layout (bytes)
    size_t off_a = 0, off_b = 0, off_spec = 0, off_spec2 = 0, off_fields = 0, off_num = 0, ws_bytes = 0;
    std::vector<void *> owned;
};

namespace {

int sfail(int code, const std::string &msg) { return record_error(code, msg.c_str()); }

#define SCK(x)                                                                                     \
    do {                                                                                           \
        cudaError_t e_ = (x);                                                                      \
        if (e_ != cudaSuccess)                                                                     \
            return sfail(e_ == cudaErrorMemoryAllocation ? BISP_OUT_OF_MEMORY : BISP_CUDA_ERROR,   \
                         std::string(#x) + ": " + cudaGetErrorString(e_));                         \
    } while (0)

template <typename T>
int sup(bisp_shell_plan *p, T **out, const std::vector<T> &v, cudaStream_t s)
{
    void *q = nullptr;
    SCK(cudaMalloc(&q, std::max<size_t>(v.size() * sizeof(T), 16)));
    p->owned.push_back(q);
    if (!v.empty()) SCK(cudaMemcpyAsync(q, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    *out = static_cast<T *>(q);
    return BISP_OK;
}

size_t al(size_t v) { return (v + 255) & ~size_t(255); }

// 3D transform of nb complex N^3 arrays: three passes of the row
// transform, each along the contiguous axis and written cyclically
// transposed, so the result is back in [x][y][z] order.  a -> b -> a -> b.
template <typename R>
cudaError_t fft3(typename Cx<R>::T *a, typename Cx<R>::T *b, int ng, int64_t nb,
                 const Twiddles<typename Cx<R>::T> &tw, cudaStream_t s)
{
    const int nrow = ng * ng;
    cudaError_t e = launch_fft_rows_T<R>(a, b, ng, nrow, nb, nullptr, R(1), false, tw, Batch{}, s);
    if (e == cudaSuccess) e = launch_fft_rows_T<R>(b, a, ng, nrow, nb, nullptr, R(1), false, tw, Batch{}, s);
    if (e == cudaSuccess) e = launch_fft_rows_T<R>(a, b, ng, nrow, nb, nullptr, R(1), false, tw, Batch{}, s);
    return e;
}

// the acceptance and (k1, mu, t) bin of a shell triple: the triangle of
// sides K1, K2, K3 (mean shell radii, grid units) shaped and binned like a
// ring combination with n1 = n2 = n3 = 0
bool triple_bin(const bisp_shell_plan &P, double kp1, double kp2, double kp3, int *bin)
{
    const bisp_desc &d = P.desc;
    TriShape sh;
    if (!triangle_shape(P.edges, kShellTwoPi / d.box_len, d.n_mu, d.n_t, kp1 * kp1, kp2 * kp2, kp3 * kp3, &sh))
        return false;
    *bin = sh.bin;
    return true;
}

int make_twiddles(bisp_shell_plan *p, cudaStream_t s)
{
    const int ng = p->ng;
    int lg2 = 0, lg3 = 0;
    while ((2 << lg2) <= ng) ++lg2;
    while (3 * (2 << lg3) <= ng) ++lg3;
    if (lg3 < 1) lg3 = 1;
    auto table = [&](int base, int count, float2 **f, double2 **d) -> int {
        std::vector<double2> vd(count);
        std::vector<float2> vf(count);
        for (int k = 0; k < count; ++k) {
            const double a = -kShellTwoPi * double(k) / double(base);
            vd[k] = make_double2(std::cos(a), std::sin(a));
            vf[k] = make_float2(float(vd[k].x), float(vd[k].y));
        }
        int st = sup(p, d, vd, s);
        return st ? st : sup(p, f, vf, s);
    };
    int st = table(1 << lg2, (7 * (1 << lg2) + 7) / 8, &p->tw2f, &p->tw2d);
    if (!st) st = table(3 << lg3, (7 * (3 << lg3) + 7) / 8, &p->tw3f, &p->tw3d);
    if (st) return st;
    p->twf = Twiddles<float2>{p->tw2f, p->tw3f, lg2, lg3};
    p->twd = Twiddles<double2>{p->tw2d, p->tw3d, lg2, lg3};
    return BISP_OK;
}

int build_shell_plan(bisp_shell_plan *p, const bisp_desc *d, cudaStream_t s)
{
    if (!d || !d->k1_edges) return sfail(BISP_INVALID_ARG, "NULL argument");
    if (!grid_size_supported(d->n_g) || d->n_g > kShellMaxNg)
        return sfail(BISP_UNSUPPORTED_SIZE, "the shell estimator takes N_g = 2^k or 3 x 2^k in [8, 128]");
    if (!(d->box_len > 0) || !std::isfinite(d->box_len) || d->n_k1 < 1 || d->n_mu < 1 || d->n_t < 1 ||
        d->n_mu > 4096 || d->n_t > 4096)
        return sfail(BISP_INVALID_ARG, "bad box length or bin counts");
    if (d->l_max < 0 || d->l_max > 6 || (d->l_max & 1)) return sfail(BISP_INVALID_ARG, "l_max must be 0, 2, 4 or 6");
    for (int b = 0; b < d->n_k1; ++b)
        if (!(d->k1_edges[b] < d->k1_edges[b + 1])) return sfail(BISP_INVALID_ARG, "k1_edges must ascend strictly");
    if (d->k1_edges[d->n_k1] > (d->n_g / 3.0) * (kShellTwoPi / d->box_len) * (1.0 + 1e-12))
        return sfail(BISP_INVALID_ARG, "k1_edges beyond (N_g/3) k_f alias");
    if (cudaError_t e = init_kernel_attributes(); e != cudaSuccess)
        return sfail(BISP_CUDA_ERROR, std::string("kernel attributes: ") + cudaGetErrorString(e));
    p->desc = *d;
    p->edges.assign(d->k1_edges, d->k1_edges + d->n_k1 + 1);
    p->desc.k1_edges = p->edges.data();
    p->desc.n_mu_l = p->desc.n_t_l = nullptr;
    const int ng = d->n_g;
    p->ng = ng;
    p->nz = ng / 3;
    p->nl = d->l_max / 2 + 1;
    p->nbins = int64_t(d->n_k1) * d->n_mu * d->n_t;
    Rings R;
    if (!build_rings(ng, R)) return sfail(BISP_UNSUPPORTED_SIZE, "shell table");
    p->ns = R.nr;
    const int ns = p->ns, nl = p->nl;
    p->e3sq.resize(ns + 1);
    for (int r = 0; r <= ns; ++r) p->e3sq[r] = R.e3[r] * R.e3[r];
    // mean |k| per shell, summed in FFT index order
    {
        std::vector<double> sum(ns, 0.0);
        std::vector<int64_t> cnt(ns, 0);
        for (int a = 0; a < ng; ++a)
            for (int b = 0; b < ng; ++b)
                for (int c = 0; c < ng; ++c) {
                    const int64_t i = a < ng / 2 ? a : a - ng, j = b < ng / 2 ? b : b - ng, n = c < ng / 2 ? c : c - ng;
                    const int64_t q9 = 9 * (i * i + j * j + n * n);
                    for (int r = 0; r < ns; ++r)
                        if (p->e3sq[r] <= q9 && q9 < p->e3sq[r + 1]) {
                            sum[r] += std::sqrt(double(i * i + j * j + n * n));
                            ++cnt[r];
                            break;
                        }
                }
        p->K.resize(ns);
        for (int r = 0; r < ns; ++r) p->K[r] = cnt[r] > 0 ? sum[r] / double(cnt[r]) : 0.0;
    }
    // candidate triples, binned
    std::vector<int32_t> cand, cbin;
    for (int s1 = 1; s1 < ns; ++s1)
        for (int s2 = 1; s2 <= s1; ++s2)
            for (int s3 = 1; s3 <= s2; ++s3) {
                int bin;
                if (!triple_bin(*p, p->K[s1], p->K[s2], p->K[s3], &bin)) continue;
                cand.insert(cand.end(), {s1, s2, s3});
                cbin.push_back(bin);
            }
    int st = make_twiddles(p, s);
    if (!st) st = sup(p, &p->d_e3sq, p->e3sq, s);
    if (st) return st;
    const int64_t n3 = int64_t(ng) * ng * ng;
    const int64_t nc = int64_t(cbin.size());
    // plan-time FP64 unit fields: I_s (kind 2) and Y_l0^2-weighted (kind 3), s >= 1
    {
        std::vector<ShellJob> uj;
        for (int sh = 1; sh < ns; ++sh) {
            uj.push_back(ShellJob{sh, 2, 0, 0});
            for (int li = 0; li < nl; ++li) uj.push_back(ShellJob{sh, 3, 2 * li, 0});
        }
        const int per = 1 + nl;
        const int64_t nu = int64_t(uj.size());
        ShellJob *d_uj = nullptr;
        double2 *sa = nullptr, *sb = nullptr;
        double *fld = nullptr, *sums = nullptr;
        int4 *d_up = nullptr;
        std::vector<int4> up;
        for (int64_t t = 0; t < nc; ++t) {
            const int s1 = cand[3 * t], s2 = cand[3 * t + 1], s3 = cand[3 * t + 2];
            auto f = [&](int sh, int k) { return (sh - 1) * per + k; };
            up.push_back(int4{f(s1, 0), f(s2, 0), f(s3, 0), int(t * (1 + nl))});
            for (int li = 0; li < nl; ++li)
                up.push_back(int4{f(s1, 1 + li), f(s2, 0), f(s3, 0), int(t * (1 + nl) + 1 + li)});
        }
        auto cleanup = [&]() {
            cudaFree(d_uj); cudaFree(sa); cudaFree(sb); cudaFree(fld); cudaFree(sums); cudaFree(d_up);
        };
        std::vector<double> h(size_t(std::max<int64_t>(nc, 1)) * (1 + nl));
        cudaError_t e = cudaMalloc(&d_uj, sizeof(ShellJob) * std::max<int64_t>(nu, 1));
        if (e == cudaSuccess) e = cudaMalloc(&sa, sizeof(double2) * std::max<int64_t>(nu * n3, 1));
        if (e == cudaSuccess) e = cudaMalloc(&sb, sizeof(double2) * std::max<int64_t>(nu * n3, 1));
        if (e == cudaSuccess) e = cudaMalloc(&fld, sizeof(double) * std::max<int64_t>(nu * n3, 1));
        if (e == cudaSuccess) e = cudaMalloc(&sums, sizeof(double) * h.size());
        if (e == cudaSuccess) e = cudaMalloc(&d_up, sizeof(int4) * std::max<size_t>(up.size(), 1));
        if (e == cudaSuccess && nu > 0) e = cudaMemcpyAsync(d_uj, uj.data(), sizeof(ShellJob) * nu, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !up.empty())
            e = cudaMemcpyAsync(d_up, up.data(), sizeof(int4) * up.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && nu > 0) {
            k_shell_spectrum<double2><<<dim3(blocks_for(n3), unsigned(nu)), 256, 0, s>>>(nullptr, ng, p->d_e3sq, d_uj, sa);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = fft3<double>(sa, sb, ng, nu, p->twd, s);
            if (e == cudaSuccess) {
                k_real_part<double2, double><<<blocks_for(nu * n3), 256, 0, s>>>(sb, fld, nu * n3);
                e = cudaGetLastError();
            }
        }
        if (e == cudaSuccess && !up.empty()) {
            k_triple_products<double><<<unsigned(up.size()), 256, 0, s>>>(fld, n3, d_up, 1.0 / double(n3), 0, 0.0,
                                                                          sums);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && nc > 0)
            e = cudaMemcpyAsync(h.data(), sums, sizeof(double) * nc * (1 + nl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cleanup();
        if (e != cudaSuccess) {
            cudaGetLastError();
            return sfail(e == cudaErrorMemoryAllocation ? BISP_OUT_OF_MEMORY : BISP_CUDA_ERROR,
                         std::string("shell plan sums: ") + cudaGetErrorString(e));
        }
        for (int64_t t = 0; t < nc; ++t) {
            const double cnt = h[t * (1 + nl)];
            const double rc = std::floor(cnt + 0.5);
            if (std::fabs(cnt - rc) > 1e-3) return sfail(BISP_INTERNAL, "shell triangle count not an integer");
            if (!(rc > 0.5)) continue;
            p->tri.insert(p->tri.end(), {cand[3 * t], cand[3 * t + 1], cand[3 * t + 2]});
            p->tri_bin.push_back(cbin[t]);
            p->ntri.push_back(rc);
            for (int li = 0; li < nl; ++li) p->den.push_back(h[t * (1 + nl) + 1 + li]);
        }
    }
    // estimate fields: D_s (kind 0) and F_{s,l} (kind 1, l >= 2), s >= 1;
    // field of (s, li): (s - 1) nl + li, li = 0 being D_s
    std::vector<ShellJob> jobs;
    for (int sh = 1; sh < ns; ++sh) {
        jobs.push_back(ShellJob{sh, 0, 0, 0});
        for (int li = 1; li < nl; ++li) jobs.push_back(ShellJob{sh, 1, 2 * li, 0});
    }
    p->njobs = int(jobs.size());
    const int64_t nt = int64_t(p->tri_bin.size());
    std::vector<int4> prods;
    for (int64_t t = 0; t < nt; ++t) {
        const int s1 = p->tri[3 * t], s2 = p->tri[3 * t + 1], s3 = p->tri[3 * t + 2];
        for (int li = 0; li < nl; ++li)
            prods.push_back(int4{(s1 - 1) * nl + li, (s2 - 1) * nl, (s3 - 1) * nl, int(t * nl + li)});
    }
    // bins: triples grouped by bin
    std::vector<int64_t> bs(p->nbins + 1, 0);
    for (int32_t b : p->tri_bin) ++bs[b + 1];
    for (int64_t b = 0; b < p->nbins; ++b) bs[b + 1] += bs[b];
    std::vector<int32_t> bt(std::max<int64_t>(nt, 1));
    {
        std::vector<int64_t> pos(bs.begin(), bs.end() - 1);
        for (int64_t t = 0; t < nt; ++t) bt[pos[p->tri_bin[t]]++] = int32_t(t);
    }
    st = sup(p, &p->d_jobs, jobs, s);
    if (!st) st = sup(p, &p->d_prods, prods, s);
    if (!st) st = sup(p, &p->d_den, p->den, s);
    if (!st) st = sup(p, &p->d_bin_start, bs, s);
    if (!st) st = sup(p, &p->d_bin_tri, bt, s);
    if (st) return st;
    // workspace
    const int64_t planes = int64_t(p->nz + 1) * ng * ng;
    size_t o = 0;
    p->off_a = o; o = al(o + size_t(planes) * sizeof(float2));
    p->off_b = o; o = al(o + size_t(planes) * sizeof(float2));
    p->off_spec = o; o = al(o + size_t(p->njobs) * n3 * sizeof(float2));
    p->off_spec2 = o; o = al(o + size_t(p->njobs) * n3 * sizeof(float2));
    p->off_fields = o; o = al(o + size_t(p->njobs) * n3 * sizeof(float));
    p->off_num = o; o = al(o + size_t(std::max<int64_t>(nt, 1)) * nl * sizeof(double));
    p->ws_bytes = o;
    SCK(cudaStreamSynchronize(s));
    return BISP_OK;
}

void free_shell_plan(bisp_shell_plan *p)
{
    if (!p) return;
    for (void *q : p->owned) cudaFree(q);
    delete p;
}

}  // namespace

extern "C" {

int estimator_shell_plan(bisp_shell_plan **out, const bisp_desc *desc, void *stream)
{
    clear_error();
    if (!out) return sfail(BISP_INVALID_ARG, "out is NULL");
    *out = nullptr;
    bisp_shell_plan *p = nullptr;
    int st;
    try {
        p = new bisp_shell_plan();
        st = build_shell_plan(p, desc, static_cast<cudaStream_t>(stream));
    } catch (const std::bad_alloc &) {
        st = sfail(BISP_OUT_OF_MEMORY, "host allocation failed while planning");
    }
    if (st) {
        free_shell_plan(p);
        return st;
    }
    *out = p;
    return BISP_OK;
}

int estimator_shell_info(const bisp_shell_plan *p, int *n_shells, int64_t *n_triples, size_t *workspace_bytes)
{
    if (!p) return sfail(BISP_INVALID_ARG, "NULL plan");
    if (n_shells) *n_shells = p->ns;
    if (n_triples) *n_triples = int64_t(p->tri_bin.size());
    if (workspace_bytes) *workspace_bytes = p->ws_bytes;
    return BISP_OK;
}

int estimator_shell_triples(const bisp_shell_plan *p, int32_t *tri, double *ntri, double *den)
{
    if (!p) return sfail(BISP_INVALID_ARG, "NULL plan");
    const size_t n = p->tri_bin.size();
    for (size_t t = 0; t < n; ++t) {
        if (tri) {
            tri[4 * t] = p->tri[3 * t];
            tri[4 * t + 1] = p->tri[3 * t + 1];
            tri[4 * t + 2] = p->tri[3 * t + 2];
            tri[4 * t + 3] = p->tri_bin[t];
        }
        if (ntri) ntri[t] = p->ntri[t];
    }
    if (den) std::copy(p->den.begin(), p->den.end(), den);
    return BISP_OK;
}

int estimator_shell_estimate(bisp_shell_plan *p, const float *delta, void *workspace, double *B, void *stream)
{
    clear_error();
    if (!p || !delta || !workspace || !B) return sfail(BISP_INVALID_ARG, "NULL argument");
    if (reinterpret_cast<uintptr_t>(workspace) % 256) return sfail(BISP_INVALID_ARG, "workspace not 256-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    const int ng = p->ng;
    const int64_t ng2 = int64_t(ng) * ng, n3 = ng2 * ng;
    float2 *A_ = reinterpret_cast<float2 *>(ws + p->off_a), *B_ = reinterpret_cast<float2 *>(ws + p->off_b);
    float2 *sa = reinterpret_cast<float2 *>(ws + p->off_spec), *sb = reinterpret_cast<float2 *>(ws + p->off_spec2);
    float *fld = reinterpret_cast<float *>(ws + p->off_fields);
    double *num = reinterpret_cast<double *>(ws + p->off_num);
    const double V = p->desc.box_len * p->desc.box_len * p->desc.box_len;
    // forward transform (planes 0..N_g/3 kept, scaled by V/N^3, Delta(0) = 0)
    SCK(launch_fft_z_real<float>(delta, A_, ng, ng2, p->nz + 1, p->twf, Batch{}, s));
    SCK(launch_fft_rows_T<float>(A_, B_, ng, ng, p->nz + 1, nullptr, 1.0f, false, p->twf, Batch{}, s));
    SCK(launch_fft_rows_T<float>(B_, A_, ng, ng, p->nz + 1, nullptr, float(V / double(n3)), true, p->twf, Batch{}, s));
    if (p->njobs > 0) {
        k_shell_spectrum<float2><<<dim3(blocks_for(n3), unsigned(p->njobs)), 256, 0, s>>>(A_, ng, p->d_e3sq, p->d_jobs, sa);
        SCK(cudaGetLastError());
        SCK(fft3<float>(sa, sb, ng, p->njobs, p->twf, s));
        k_real_part<float2, float><<<blocks_for(int64_t(p->njobs) * n3), 256, 0, s>>>(sb, fld, int64_t(p->njobs) * n3);
        SCK(cudaGetLastError());
    }
    const int64_t nprod = int64_t(p->tri_bin.size()) * p->nl;
    if (nprod > 0) {
        // l = 0 takes D_{s1} for F_{s1,0} = Y_00 D_{s1}: its sums are scaled by Y_00
        const double y00 = std::sqrt(1.0 / (2.0 * kShellTwoPi));
        k_triple_products<float><<<unsigned(nprod), 256, 0, s>>>(fld, n3, p->d_prods, 1.0 / double(n3), p->nl,
                                                                 y00 / double(n3), num);
        SCK(cudaGetLastError());
    }
    const int64_t nq = p->nbins * p->nl;
    if (nq > 0) {
        k_shell_bin<<<unsigned((nq + 255) / 256), 256, 0, s>>>(p->d_bin_start, p->d_bin_tri, p->nbins, p->nl, num,
                                                                p->d_den, 1.0 / V, B);
        SCK(cudaGetLastError());
    }
    return BISP_OK;
}

int estimator_shell_sums(const bisp_shell_plan *p, const void *workspace, double *num, void *stream)
{
    if (!p || !workspace || !num) return sfail(BISP_INVALID_ARG, "NULL argument");
    const size_t n = p->tri_bin.size() * size_t(p->nl);
    if (n == 0) return BISP_OK;
    SCK(cudaMemcpyAsync(num, static_cast<const unsigned char *>(workspace) + p->off_num, n * sizeof(double),
                        cudaMemcpyDeviceToHost, static_cast<cudaStream_t>(stream)));
    SCK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    return BISP_OK;
}

void estimator_shell_destroy(bisp_shell_plan *p) { free_shell_plan(p); }

}  // extern "C"
