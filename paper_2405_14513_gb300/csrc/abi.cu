// abi.cu -- the C ABI of include/bisp.h: plan construction, workspace layout
// and the stream-ordered estimate (forward transform, Step I, Step II,
// binning) of Gill & Bharadwaj, arXiv:2405.14513, Sec. II.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "bisp.h"
#include "kernels.cuh"
#include "plan.hpp"

using namespace bisp;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define CK(x)                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = (x);                                                                     \
        if (e_ != cudaSuccess)                                                                    \
            return fail(e_ == cudaErrorMemoryAllocation ? BISP_OUT_OF_MEMORY : BISP_CUDA_ERROR,   \
                        std::string(#x) + ": " + cudaGetErrorString(e_));                         \
    } while (0)

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int64_t kXChunk = 16384;        // grid points of one Step-II unit

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

int ilog2i(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

}  // namespace

namespace bisp {
// Record a failure message for estimator_last_error() from another
// translation unit of the library.
int record_error(int code, const char *msg) { return fail(code, msg); }
// Clear the calling thread's failure message (at the entry of a call).
void clear_error() { g_err.clear(); }
}  // namespace bisp

struct bisp_plan {
    HostPlan hp;
    int precision = BISP_PREC_MIXED;
    size_t celem = 8;                    // bytes of one complex field value
    int64_t x_chunk = 0;                 // grid points of one Step-II unit
    std::vector<void *> owned;           // device allocations of the plan
    Group *d_groups = nullptr;
    Tile *d_tiles = nullptr;
    Unit *d_units = nullptr;
    TcTile *d_tc_tiles = nullptr;        // tcgen05 Step II (MIXED_TC)
    TcRow *d_tc_rows = nullptr;
    int32_t *d_tc_slots = nullptr;
    TcUnit *d_tc_units = nullptr;
    int64_t *d_doff = nullptr;
    Record *d_rec = nullptr;
    int64_t *d_bin_start = nullptr;
    int64_t *d_chunk_lo = nullptr, *d_chunk_hi = nullptr, *d_bin_chunk = nullptr;   // binning chunks
    double *d_den = nullptr;
    std::vector<double> h_den;
    Twiddles<float2> tw_f{};             // transform twiddles (device tables)
    Twiddles<double2> tw_d{};
    GridArg grid_arg{};                  // reduction grid sides by level index
    RingArg ring_arg{};
    std::vector<Job *> d_jobs;           // per level in use
    std::vector<int64_t *> d_job_off;    // per level: output offsets of the jobs
    // one field's workspace region (offsets within it); field f of a batch
    // uses bytes [f region_bytes, (f + 1) region_bytes) of the workspace
    // off_status: one int, set by a Step-II block of this field whose bounded
    // wait ran out; cleared at the start of every estimate
    // off_epi: the binning's partial sums per chunk
    size_t off_a = 0, off_b = 0, off_gt = 0, off_dstore = 0, off_part = 0, off_S = 0, off_status = 0, off_epi = 0,
           region_bytes = 0;
    int wait_spins = kDefaultWaitSpins;  // bound of the tensor-core Step II's abortable waits
    int device = -1;                     // the device the plan's tables live on
    int last_field = 0;                  // field of the last estimate that introspection reads
    // transform rows per block picked by the plan's autotuner (0 = default rule)
    int rt_z = 0, rt_xy = 0;
    int rt_gather[kMaxLevels] = {}, rt_rows[kMaxLevels] = {};
    size_t resident = 0;
    // buffers of estimator_estimate_host
    void *own_ws = nullptr, *own_in = nullptr;
    double *own_out = nullptr;
    // streaming from host memory (estimator_host_submit / _wait): two slots,
    // each with its input and output buffers; the input copies run on a
    // stream of the plan's own, the estimates on the caller's stream
    struct HostPipe {
        cudaStream_t copy = nullptr;
        void *in[2] = {};
        double *out[2] = {};
        int *status_h = nullptr;                  // pinned: [2][max_batch] wait-status words
        cudaEvent_t in_ready[2] = {}, in_free[2] = {}, done[2] = {};
        int batch[2] = {};
        int head = 0, count = 0;                  // oldest slot in flight; submissions in flight
    } pipe;
    // stage timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Mark { int stage; cudaEvent_t a, b; int launches; };
    std::vector<Mark> pending;
    double stage_ms[BISP_N_STAGES] = {};
    int64_t stage_launches[BISP_N_STAGES] = {};
};

// The device of a plan, for the static-scratch entry point (noalloc.cu).
int bisp::plan_device(const bisp_plan *p) { return p ? p->device : -1; }

namespace {

template <typename T>
int dev_alloc(bisp_plan *p, T **out, size_t count)
{
    void *q = nullptr;
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BISP_OUT_OF_MEMORY, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                            cudaGetErrorString(e));
    }
    p->owned.push_back(q);
    p->resident += bytes;
    *out = static_cast<T *>(q);
    return BISP_OK;
}

template <typename T>
int upload(bisp_plan *p, T **out, const std::vector<T> &v, cudaStream_t s)
{
    int st = dev_alloc(p, out, v.size());
    if (st) return st;
    if (!v.empty()) CK(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return BISP_OK;
}

cudaEvent_t take_event(bisp_plan *p)
{
    if (!p->ev_pool.empty()) {
        cudaEvent_t e = p->ev_pool.back();
        p->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// Event pair around one stage on stream s, when timing is on.
struct StageMark {
    bisp_plan *p;
    int stage, launches;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    StageMark(bisp_plan *p_, int stage_, int launches_, cudaStream_t s_) : p(p_), stage(stage_), launches(launches_), s(s_)
    {
        if (p->timing && (a = take_event(p))) cudaEventRecord(a, s);
    }
    ~StageMark()
    {
        if (!a) return;
        cudaEvent_t b = take_event(p);
        if (!b) { p->ev_pool.push_back(a); return; }
        cudaEventRecord(b, s);
        p->pending.push_back(bisp_plan::Mark{stage, a, b, launches});
    }
};

int collect_times(bisp_plan *p)
{
    for (auto &m : p->pending) {
        CK(cudaEventSynchronize(m.b));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, m.a, m.b));
        p->stage_ms[m.stage] += ms;
        p->stage_launches[m.stage] += m.launches;
        p->ev_pool.push_back(m.a);
        p->ev_pool.push_back(m.b);
    }
    p->pending.clear();
    return BISP_OK;
}

void free_plan(bisp_plan *p)
{
    if (!p) return;
    for (auto &m : p->pending) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    for (void *q : p->owned) cudaFree(q);
    if (p->own_ws) cudaFree(p->own_ws);
    if (p->own_in) cudaFree(p->own_in);
    if (p->own_out) cudaFree(p->own_out);
    auto &h = p->pipe;
    for (int i = 0; i < 2; ++i) {
        if (h.in[i]) cudaFree(h.in[i]);
        if (h.out[i]) cudaFree(h.out[i]);
        if (h.in_ready[i]) cudaEventDestroy(h.in_ready[i]);
        if (h.in_free[i]) cudaEventDestroy(h.in_free[i]);
        if (h.done[i]) cudaEventDestroy(h.done[i]);
    }
    if (h.status_h) cudaFreeHost(h.status_h);
    if (h.copy) cudaStreamDestroy(h.copy);
    delete p;
}

int check_desc(const bisp_desc *d)
{
    if (!d) return fail(BISP_INVALID_ARG, "desc is NULL");
    if (!grid_size_supported(d->n_g))
        return fail(BISP_UNSUPPORTED_SIZE, "n_g must be 2^k or 3 x 2^k in [8, 1024]");
    if (!(d->box_len > 0) || !std::isfinite(d->box_len)) return fail(BISP_INVALID_ARG, "box_len must be > 0");
    if (d->n_k1 < 1 || !d->k1_edges) return fail(BISP_INVALID_ARG, "need n_k1 >= 1 and k1_edges");
    for (int b = 0; b < d->n_k1; ++b)
        if (!(d->k1_edges[b] < d->k1_edges[b + 1])) return fail(BISP_INVALID_ARG, "k1_edges must ascend strictly");
    if (!(d->k1_edges[0] >= 0)) return fail(BISP_INVALID_ARG, "k1_edges must be >= 0");
    const double kf = kTwoPi / d->box_len;
    if (d->k1_edges[d->n_k1] > (d->n_g / 3.0) * kf * (1.0 + 1e-12))
        return fail(BISP_INVALID_ARG, "k1_edges beyond (N_g/3) k_f alias");
    if (d->n_mu < 1 || d->n_t < 1 || d->n_mu > 4096 || d->n_t > 4096)
        return fail(BISP_INVALID_ARG, "n_mu and n_t must be in [1, 4096]");
    if (d->l_max < 0 || d->l_max > 8 || (d->l_max & 1)) return fail(BISP_INVALID_ARG, "l_max must be even, 0..8");
    if (!d->n_mu_l != !d->n_t_l) return fail(BISP_INVALID_ARG, "give both n_mu_l and n_t_l, or neither");
    if (d->n_mu_l)
        for (int i = 0; i <= d->l_max / 2; ++i)
            if (d->n_mu_l[i] < 1 || d->n_t_l[i] < 1 || d->n_mu_l[i] > 4096 || d->n_t_l[i] > 4096)
                return fail(BISP_INVALID_ARG, "per-l (mu, t) bins must be in [1, 4096]");
    if (d->precision < BISP_PREC_FP32 || d->precision > BISP_PREC_MIXED_TC)
        return fail(BISP_INVALID_ARG, "unknown precision");
    if (d->max_batch < 1 || d->max_batch > 65535) return fail(BISP_INVALID_ARG, "max_batch must be in [1, 65535]");
    return BISP_OK;
}

// N_tri of every ring triple by Eq. Ntri2 on the GPU in FP64: unit fields
// I(r) on each reduction grid, then M^-2 sum_y I1 I2 I3, rounded.
int compute_ntri(bisp_plan *p, cudaStream_t s)
{
    HostPlan &P = p->hp;
    const Rings &R = P.rings;
    const int nr = R.nr;
    std::vector<int32_t> tri;
    std::vector<uint8_t> need(size_t(kMaxLevels) * kMaxRings, 0);
    for (int a = 0; a < nr; ++a)
        for (int b = a; b < nr; ++b)
            for (int c = b; c < nr; ++c) {
                const int lv = triple_level(R, a, b, c);
                tri.insert(tri.end(), {a, b, c, lv});
                need[lv * kMaxRings + a] = need[lv * kMaxRings + b] = need[lv * kMaxRings + c] = 1;
            }
    std::vector<int64_t> ioff(size_t(kMaxLevels) * kMaxRings, -1);
    int64_t cur = 0, gtmax = 0;
    std::vector<std::vector<Job>> jobs(kMaxLevels);
    for (int lv = 0; lv < R.ngrid; ++lv) {
        const int64_t M2 = int64_t(R.grid[lv]) * R.grid[lv];
        for (int r = 0; r < nr; ++r)
            if (need[lv * kMaxRings + r]) {
                ioff[lv * kMaxRings + r] = cur;
                jobs[lv].push_back(Job{0, r, cur});
                cur += M2;
            }
        gtmax = std::max<int64_t>(gtmax, int64_t(jobs[lv].size()) * M2);
    }

    std::vector<void *> tmp;
    auto talloc = [&](size_t bytes) -> void * {
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        tmp.push_back(q);
        return q;
    };
    auto cleanup = [&]() { for (void *q : tmp) cudaFree(q); };
    double2 *I = (double2 *)talloc(size_t(cur) * sizeof(double2));
    double2 *gt = (double2 *)talloc(size_t(gtmax) * sizeof(double2));
    int64_t *d_ioff = (int64_t *)talloc(ioff.size() * sizeof(int64_t));
    int32_t *d_tri = (int32_t *)talloc(tri.size() * sizeof(int32_t));
    double *d_raw = (double *)talloc(tri.size() / 4 * sizeof(double));
    Job *d_jobs = (Job *)talloc(size_t(nr) * sizeof(Job));
    int64_t *d_joff = (int64_t *)talloc(size_t(nr) * sizeof(int64_t));
    if (!I || !gt || !d_ioff || !d_tri || !d_raw || !d_jobs || !d_joff) {
        cleanup();
        return fail(BISP_OUT_OF_MEMORY, "device memory for the triangle counts");
    }
    auto run = [&]() -> int {
        CK(cudaMemcpyAsync(d_ioff, ioff.data(), ioff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_tri, tri.data(), tri.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        for (int lv = 0; lv < R.ngrid; ++lv) {
            if (jobs[lv].empty()) continue;
            const int M = R.grid[lv];
            std::vector<int64_t> joff;
            for (auto &j : jobs[lv]) joff.push_back(j.out_off);
            CK(cudaMemcpyAsync(d_jobs, jobs[lv].data(), jobs[lv].size() * sizeof(Job), cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(d_joff, joff.data(), joff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
            CK(launch_ring_gather<double>(I, R.ng, p->ring_arg, d_jobs, int64_t(jobs[lv].size()), M, true, gt,
                                          p->tw_d, Batch{}, s));
            CK(launch_fft_cols<double>(gt, I, M, int64_t(jobs[lv].size()), d_joff, d_jobs, p->ring_arg, p->tw_d, Batch{},
                                        s));
            CK(cudaStreamSynchronize(s));   // the job tables are reused by the next grid
        }
        CK(launch_ntri(I, d_ioff, d_tri, int64_t(tri.size() / 4), p->grid_arg, d_raw, s));
        std::vector<double> raw(tri.size() / 4);
        CK(cudaMemcpyAsync(raw.data(), d_raw, raw.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        P.ntri.assign(size_t(nr) * nr * nr, 0);
        for (size_t t = 0; t < raw.size(); ++t) {
            const double v = raw[t], rv = std::nearbyint(v);
            if (!(std::fabs(v - rv) < 1e-3) || rv < 0)
                return fail(BISP_INTERNAL, "triangle count not an integer: " + std::to_string(v));
            const int a = tri[4 * t], b = tri[4 * t + 1], c = tri[4 * t + 2];
            const int64_t n = int64_t(rv);
            const int perm[6][3] = {{a, b, c}, {a, c, b}, {b, a, c}, {b, c, a}, {c, a, b}, {c, b, a}};
            for (auto &q : perm) P.ntri[(size_t(q[0]) * nr + q[1]) * nr + q[2]] = n;
        }
        return BISP_OK;
    };
    int st = run();
    cudaStreamSynchronize(s);
    cleanup();
    return st;
}

// Kernel attributes are per device; set them once per device in the process.
int init_attributes()
{
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (std::find(done.begin(), done.end(), dev) != done.end()) return BISP_OK;
    CK(init_kernel_attributes());
    CK(init_step2_tc_attributes());
    done.push_back(dev);
    return BISP_OK;
}

// Transform tile autotuner.  Each transform kernel holds rt rows (or, in
// Step I's second pass, w columns) of its length M in two shared-memory
// buffers; the best tile depends on M, the kernel and the GPU (large tiles
// leave one block per SM).  For the forward z pass, the forward row passes
// and each reduction grid's gather, candidate tiles of 4-64 KB per buffer,
// and for each grid's second pass strips of 2-32 columns, are timed on
// scratch buffers holding a sample of the plan's rows (16 planes, 64K z
// rows, and at most kTuneJobs fields of a grid, evenly spaced over its
// fields so that their rings, and the launch's size, are those of the
// estimate), and the fastest is kept.  Rows and columns are transformed
// independently, so the choice changes the speed, not the results.
constexpr int64_t kTuneJobs = 512;

template <typename R>
int autotune_transforms(bisp_plan *p, cudaStream_t s)
{
    using C = typename Cx<R>::T;
    const HostPlan &P = p->hp;
    const Rings &Rg = P.rings;
    const int ng = P.desc.n_g, nz1 = Rg.nz + 1;
    const int64_t ng2 = int64_t(ng) * ng;
    Twiddles<C> tw;
    if constexpr (sizeof(R) == 8) tw = p->tw_d; else tw = p->tw_f;
    const int64_t zrows = std::min<int64_t>(ng2, 65536);
    const int64_t npl = std::min<int64_t>(nz1, 16);
    // the sampled fields of every grid: every stride-th of its (plane, ring)
    // fields, in the estimate's order, at most kTuneJobs
    std::vector<std::vector<Job>> sample(P.levels.size());
    int64_t jmax = 0, nsamp = 0;
    for (size_t l = 0; l < P.levels.size(); ++l) {
        const Level &L = P.levels[l];
        const int64_t stride = (L.njobs + kTuneJobs - 1) / kTuneJobs;
        int64_t k = 0;
        for (int n = 0; n <= Rg.nz; ++n)
            for (int r = 0; r < Rg.nr; ++r)
                if (P.doff[(size_t(L.lev) * (Rg.nz + 1) + n) * kMaxRings + r] >= 0 && k++ % stride == 0)
                    sample[l].push_back(Job{n, r, 0});
        jmax = std::max(jmax, int64_t(sample[l].size()) * L.M * L.M);
        nsamp += int64_t(sample[l].size());
    }
    // scratch: z-pass input and output, the transformed planes (input of the
    // gathers), and two buffers for the row passes
    const size_t bz = size_t(zrows) * ng * sizeof(R);
    const size_t bplanes = size_t(nz1) * ng2 * sizeof(C);
    const size_t brows = std::max<size_t>(size_t(jmax), size_t(npl) * ng2) * sizeof(C);
    const size_t bout = std::max<size_t>(size_t(nz1) * zrows * sizeof(C), brows);
    std::vector<void *> tmp;
    auto talloc = [&](size_t b) -> void * {
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(b, 256)) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        tmp.push_back(q);
        return q;
    };
    auto cleanup = [&]() { for (void *q : tmp) cudaFree(q); };
    R *zin = static_cast<R *>(talloc(bz));
    C *planes = static_cast<C *>(talloc(bplanes));
    C *b0 = static_cast<C *>(talloc(bout));
    C *b1 = static_cast<C *>(talloc(brows));
    // the sampled jobs and their output offsets (job j of a grid at j M^2)
    int64_t *d_offs = static_cast<int64_t *>(talloc(sizeof(int64_t) * size_t(nsamp)));
    Job *d_samp = static_cast<Job *>(talloc(sizeof(Job) * size_t(nsamp)));
    std::vector<int64_t> h_offs;
    std::vector<Job> h_samp;
    std::vector<int64_t> samp0;
    for (size_t l = 0; l < P.levels.size(); ++l) {
        samp0.push_back(int64_t(h_samp.size()));
        for (size_t j = 0; j < sample[l].size(); ++j) {
            h_offs.push_back(int64_t(j) * P.levels[l].M * P.levels[l].M);
            h_samp.push_back(sample[l][j]);
        }
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!zin || !planes || !b0 || !b1 || !d_offs || !d_samp || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        if (e0) cudaEventDestroy(e0);
        return fail(BISP_OUT_OF_MEMORY, "device memory for the transform autotuner");
    }
    cudaMemsetAsync(zin, 0, bz, s);
    cudaMemsetAsync(planes, 0, bplanes, s);
    cudaMemsetAsync(b0, 0, bout, s);
    cudaMemsetAsync(b1, 0, brows, s);
    cudaMemcpyAsync(d_offs, h_offs.data(), h_offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_samp, h_samp.data(), h_samp.size() * sizeof(Job), cudaMemcpyHostToDevice, s);
    const size_t cand[] = {4096, 8192, 16384, 32768, 65536};
    // the fastest of the candidate rows per block for one launch
    auto pick = [&](int M, int cap, auto &&launch) -> int {
        int best = 0, last = -1;
        float best_ms = 1e30f;
        for (size_t bytes : cand) {
            const int rt = std::min(int(fft_rows_per_block(M, sizeof(C), bytes)), cap);
            if (rt == last) continue;
            last = rt;
            if (launch(rt) != cudaSuccess) return -1;
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3; ++r) launch(rt);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return -1;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) { best_ms = ms; best = rt; }
        }
        return best;
    };
    // the fastest strip width (columns per block) of a grid's second pass
    auto pick_w = [&](int M, auto &&launch) -> int {
        int best = 0;
        float best_ms = 1e30f;
        for (int w : {2, 4, 8, 16, 32}) {
            if (w > M || size_t(2) * w * fft_stride(M) * sizeof(C) > 227 * 1024) continue;
            if (launch(w) != cudaSuccess) return -1;
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3; ++r) launch(w);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return -1;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) { best_ms = ms; best = w; }
        }
        return best;
    };
    const Batch one{};
    int st = BISP_OK;
    p->rt_z = pick(ng, 256, [&](int rt) {
        return launch_fft_z_real<R>(zin, b0, ng, zrows, nz1, tw, one, s, rt);
    });
    p->rt_xy = pick(ng, ng, [&](int rt) {
        return launch_fft_rows_T<R>(b1, b0, ng, ng, npl, nullptr, R(1), false, tw, one, s, rt);
    });
    if (p->rt_z < 0 || p->rt_xy < 0) st = fail(BISP_CUDA_ERROR, "transform autotuner");
    for (size_t l = 0; l < P.levels.size() && !st; ++l) {
        const Level &L = P.levels[l];
        const int64_t nj = int64_t(sample[l].size());
        const int64_t *d_off = d_offs + samp0[l];
        const Job *d_j = d_samp + samp0[l];
        const int g = pick(L.M, L.M, [&](int rt) {
            return launch_ring_gather<R>(planes, ng, p->ring_arg, d_j, nj, L.M, false, b0, tw, one, s, rt);
        });
        const int r = pick_w(L.M, [&](int w) {
            return launch_fft_cols<R>(b0, b1, L.M, nj, d_off, d_j, p->ring_arg, tw, one, s, w);
        });
        if (g < 0 || r < 0) st = fail(BISP_CUDA_ERROR, "transform autotuner");
        p->rt_gather[L.lev] = std::max(g, 0);
        p->rt_rows[L.lev] = std::max(r, 0);
    }
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cleanup();
    return st;
}

int build_plan(bisp_plan *p, const bisp_desc *desc, cudaStream_t s)
{
    if (int st = init_attributes()) return st;
    HostPlan &P = p->hp;
    P.desc = *desc;
    P.k1_edges.assign(desc->k1_edges, desc->k1_edges + desc->n_k1 + 1);
    P.desc.k1_edges = P.k1_edges.data();
    // per-l grids: the plan's own n_mu x n_t (combination bins) is that of l = 0
    std::vector<int> mu_l, t_l;
    if (desc->n_mu_l) {
        mu_l.assign(desc->n_mu_l, desc->n_mu_l + desc->l_max / 2 + 1);
        t_l.assign(desc->n_t_l, desc->n_t_l + desc->l_max / 2 + 1);
        P.desc.n_mu = mu_l[0];
        P.desc.n_t = t_l[0];
    }
    P.desc.n_mu_l = P.desc.n_t_l = nullptr;    // caller memory is not kept
    P.kf = kTwoPi / desc->box_len;
    P.volume = desc->box_len * desc->box_len * desc->box_len;
    P.n_lm = (desc->l_max / 2 + 1) * (desc->l_max / 2 + 1);
    P.n_bins = int64_t(desc->n_k1) * P.desc.n_mu * P.desc.n_t;
    p->precision = desc->precision;
    p->celem = desc->precision == BISP_PREC_FP64 ? sizeof(double2) : sizeof(float2);
    if (!build_rings(desc->n_g, P.rings)) return fail(BISP_UNSUPPORTED_SIZE, "ring table");
    const Rings &R = P.rings;
    p->ring_arg.nr = R.nr;
    for (int r = 0; r <= R.nr; ++r) p->ring_arg.e3sq[r] = R.e3[r] * R.e3[r];
    for (int r = 0; r < R.nr; ++r) p->ring_arg.maxc[r] = R.maxc[r];

    for (int l = 0; l < R.ngrid; ++l) p->grid_arg.M[l] = R.grid[l];
    // twiddles in double: exp(-2 pi i k / (F x 2^lgF)), k < 7/8 of F x 2^lgF
    // (radix-8 stages reach seven eighths of the circle), for the lengths
    // F x 2^q <= N_g of the transforms, F = 1, 3, 5, 7
    {
        const int ng = desc->n_g;
        int lg2 = 0, lg3 = 0, lg5 = 0, lg7 = 0;
        while ((2 << lg2) <= ng) ++lg2;
        while (3 * (2 << lg3) <= ng) ++lg3;
        while (5 * (2 << lg5) <= ng) ++lg5;
        while (7 * (2 << lg7) <= ng) ++lg7;
        if (lg3 < 1) lg3 = 1;
        if (lg5 < 2) lg5 = 2;
        if (lg7 < 2) lg7 = 2;
        auto table = [&](int base, int count, float2 **df, double2 **dd) -> int {
            std::vector<double2> twd(count);
            std::vector<float2> twf(count);
            for (int k = 0; k < count; ++k) {
                const double a = -kTwoPi * double(k) / double(base);
                twd[k] = make_double2(std::cos(a), std::sin(a));
                twf[k] = make_float2(float(twd[k].x), float(twd[k].y));
            }
            int st = upload(p, dd, twd, s);
            return st ? st : upload(p, df, twf, s);
        };
        float2 *f2 = nullptr, *f3 = nullptr, *f5 = nullptr, *f7 = nullptr;
        double2 *d2 = nullptr, *d3 = nullptr, *d5 = nullptr, *d7 = nullptr;
        int st = table(1 << lg2, (7 * (1 << lg2) + 7) / 8, &f2, &d2);
        if (!st) st = table(3 << lg3, (7 * (3 << lg3) + 7) / 8, &f3, &d3);
        if (!st) st = table(5 << lg5, (7 * (5 << lg5) + 7) / 8, &f5, &d5);
        if (!st) st = table(7 << lg7, (7 * (7 << lg7) + 7) / 8, &f7, &d7);
        if (st) return st;
        p->tw_f = Twiddles<float2>{f2, f3, lg2, lg3, f5, lg5, f7, lg7};
        p->tw_d = Twiddles<double2>{d2, d3, lg2, lg3, d5, lg5, d7, lg7};
    }
    // Y_lm normalisations
    {
        double nlm[9][9] = {}, pref[9] = {};
        for (int l = 0; l <= 8; ++l) {
            pref[l] = std::sqrt((2.0 * l + 1.0) / (2.0 * kTwoPi));
            for (int m = 0; m <= l; ++m) {
                double r = 1.0;
                for (int k = l - m + 1; k <= l + m; ++k) r /= double(k);
                nlm[l][m] = std::sqrt((2.0 * l + 1.0) / (2.0 * kTwoPi) * r);
            }
        }
        CK(set_ylm_constants(nlm, pref, s));
    }
    int st = compute_ntri(p, s);
    if (st) return st;
    P.celem = p->celem;
    P.max_cls = desc->precision == BISP_PREC_FP64 ? 3 : 4;   // FP64 blocks have at most 8 warps
    P.tensor = desc->precision == BISP_PREC_MIXED_TC;       // Step II on tensor cores
    p->x_chunk = kXChunk;
    std::string err = enumerate(P, p->x_chunk);
    if (!err.empty()) return fail(BISP_INTERNAL, err);
    unit_costs(P, p->x_chunk);
    build_views(P, mu_l.empty() ? nullptr : mu_l.data(), t_l.empty() ? nullptr : t_l.data());
    sort_records(P);

    st = upload(p, &p->d_groups, P.groups, s);
    if (!st) st = upload(p, &p->d_tiles, P.tiles, s);
    if (!st) st = upload(p, &p->d_units, P.units, s);
    if (!st) st = upload(p, &p->d_tc_tiles, P.tc_tiles, s);
    if (!st) st = upload(p, &p->d_tc_rows, P.tc_rows, s);
    if (!st) st = upload(p, &p->d_tc_slots, P.tc_slots, s);
    if (!st) st = upload(p, &p->d_tc_units, P.tc_units, s);
    if (!st) st = upload(p, &p->d_doff, P.doff, s);
    if (!st) st = upload(p, &p->d_rec, P.records, s);
    if (!st) st = upload(p, &p->d_bin_start, P.bin_start, s);
    if (!st) st = upload(p, &p->d_chunk_lo, P.chunk_lo, s);
    if (!st) st = upload(p, &p->d_chunk_hi, P.chunk_hi, s);
    if (!st) st = upload(p, &p->d_bin_chunk, P.bin_chunk, s);
    if (!st) st = dev_alloc(p, &p->d_den, size_t(P.n_out));
    if (st) return st;
    const int64_t epi_nlm = int64_t(desc->l_max / 2 + 1) * (desc->l_max / 2 + 1);   // moments of l <= l_max
    // plan-time denominators of Eq. bs_lm2_1 (FP64)
    {
        double *d_nt = nullptr, *d_epi = nullptr;
        void *q = nullptr, *q2 = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(P.rec_ntri.size() * sizeof(double), 16)) != cudaSuccess ||
            cudaMalloc(&q2, std::max<size_t>(size_t(P.max_chunks * epi_nlm) * sizeof(double), 16)) != cudaSuccess) {
            cudaGetLastError();
            if (q) cudaFree(q);
            return fail(BISP_OUT_OF_MEMORY, "device memory for the denominators");
        }
        d_nt = static_cast<double *>(q);
        d_epi = static_cast<double *>(q2);
        cudaError_t e = cudaMemcpyAsync(d_nt, P.rec_ntri.data(), P.rec_ntri.size() * sizeof(double),
                                        cudaMemcpyHostToDevice, s);
        for (const View &v : P.views)
            if (e == cudaSuccess) {
                const EpiArgs ea{p->d_rec, p->d_chunk_lo + v.chunk_off, p->d_chunk_hi + v.chunk_off, v.n_chunks,
                                 p->d_bin_chunk + v.bc_off, v.n_bins, d_epi, 0};
                e = launch_epilogue<double>(1, ea, d_nt, v.l_lo, v.l_hi, nullptr, 1.0, p->d_den + v.out_off,
                                            Batch{}, s);
            }
        p->h_den.resize(size_t(P.n_out));
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->h_den.data(), p->d_den, p->h_den.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(d_nt);
        cudaFree(d_epi);
        if (e != cudaSuccess) return fail(BISP_CUDA_ERROR, std::string("denominators: ") + cudaGetErrorString(e));
        std::vector<double>().swap(P.rec_ntri);
    }
    // Step-I jobs per grid
    for (const Level &L : P.levels) {
        std::vector<Job> jobs;
        std::vector<int64_t> off;
        for (int n = 0; n <= R.nz; ++n)
            for (int r = 0; r < R.nr; ++r) {
                int64_t o = P.doff[(size_t(L.lev) * (R.nz + 1) + n) * kMaxRings + r];
                if (o >= 0) {
                    jobs.push_back(Job{n, r, o});
                    off.push_back(o);
                }
            }
        Job *dj = nullptr;
        int64_t *dof = nullptr;
        st = upload(p, &dj, jobs, s);
        if (!st) st = upload(p, &dof, off, s);
        if (st) return st;
        p->d_jobs.push_back(dj);
        p->d_job_off.push_back(dof);
    }
    // workspace layout
    const int64_t planes = int64_t(R.nz + 1) * desc->n_g * desc->n_g;
    size_t o = 0;
    p->off_a = o; o = align256(o + size_t(planes) * p->celem);
    p->off_b = o; o = align256(o + size_t(planes) * p->celem);
    p->off_gt = o; o = align256(o + size_t(P.gt_elems) * p->celem);
    p->off_dstore = o; o = align256(o + size_t(P.dstore_elems) * p->celem);
    p->off_part = o; o = align256(o + size_t(P.n_partials) * sizeof(double));
    p->off_S = o; o = align256(o + size_t(P.n_combos) * sizeof(double));
    p->off_status = o; o = align256(o + sizeof(int));
    p->off_epi = o; o = align256(o + size_t(P.max_chunks * epi_nlm) * sizeof(double));
    p->region_bytes = o;
    CK(cudaStreamSynchronize(s));
    return desc->precision == BISP_PREC_FP64 ? autotune_transforms<double>(p, s) : autotune_transforms<float>(p, s);
}

// Step-II launches of one estimate (one per non-empty block class)
int step2_launches(const int64_t *lo, const int64_t *hi)
{
    int n = 0;
    for (int c = 0; c < kClassSlots; ++c) n += hi[c] > lo[c];
    return n;
}

template <typename R, typename A, typename S, typename W>
int run_estimate(bisp_plan *p, const R *delta, int batch, unsigned char *ws, double *B, int share, int nshares,
                 cudaStream_t s)
{
    using C = typename Cx<R>::T;
    const HostPlan &P = p->hp;
    const Rings &Rg = P.rings;
    const int ng = P.desc.n_g;
    Twiddles<C> tw;
    if constexpr (sizeof(R) == 8) tw = p->tw_d; else tw = p->tw_f;
    C *A_ = reinterpret_cast<C *>(ws + p->off_a);
    C *B_ = reinterpret_cast<C *>(ws + p->off_b);
    C *gt = reinterpret_cast<C *>(ws + p->off_gt);
    C *dstore = reinterpret_cast<C *>(ws + p->off_dstore);
    double *part = reinterpret_cast<double *>(ws + p->off_part);
    double *Ssum = reinterpret_cast<double *>(ws + p->off_S);
    const int64_t ng2 = int64_t(ng) * ng;
    const R scale = R(P.volume / (double(ng2) * ng));
    const int64_t fs = int64_t(p->region_bytes);          // between the fields' workspace regions
    StepIIArgs a2{p->d_groups, p->d_tiles, p->d_units, p->d_doff, Rg.nz + 1, Rg.nr, p->x_chunk, part, fs};
    TcArgs atc{p->d_tc_tiles, p->d_tc_rows, p->d_tc_slots, p->d_tc_units, p->d_doff, Rg.nz + 1, Rg.nr, p->x_chunk,
               part, reinterpret_cast<int *>(ws + p->off_status), fs, p->wait_spins};
    // every stage runs once for all fields of the batch (gridDim.y = field)
    const unsigned nf = unsigned(batch);
    const Batch in_field{nf, int64_t(ng2) * ng * int64_t(sizeof(R)), fs};   // input field -> region
    const Batch region{nf, fs, fs};
    const Batch to_out{nf, fs, P.n_out * int64_t(sizeof(double))};
    // the wait status of each field starts clear
    CK(cudaMemset2DAsync(ws + p->off_status, size_t(fs), 0, sizeof(int), nf, s));
    {   // forward transform: z (real, planes 0..N_g/3 kept) -> y -> x, scaled by V/N_g^3, Delta(0) = 0
        StageMark m(p, BISP_STAGE_FORWARD, 3, s);
        CK(launch_fft_z_real<R>(delta, A_, ng, ng2, Rg.nz + 1, tw, in_field, s, p->rt_z));
        CK(launch_fft_rows_T<R>(A_, B_, ng, ng, Rg.nz + 1, nullptr, R(1), false, tw, region, s, p->rt_xy));
        CK(launch_fft_rows_T<R>(B_, A_, ng, ng, Rg.nz + 1, nullptr, scale, true, tw, region, s, p->rt_xy));
    }
    {   // Step I: D(r, n) on each reduction grid (Eq. iFT)
        StageMark m(p, BISP_STAGE_STEP1, int(2 * P.levels.size()), s);
        for (size_t l = 0; l < P.levels.size(); ++l) {
            const Level &L = P.levels[l];
            const int M = L.M;
            CK(launch_ring_gather<R>(A_, ng, p->ring_arg, p->d_jobs[l], L.njobs, M, false, gt, tw, region, s,
                                     p->rt_gather[L.lev]));
            CK(launch_fft_cols<R>(gt, dstore, M, L.njobs, p->d_job_off[l], p->d_jobs[l], p->ring_arg, tw, region, s,
                                  p->rt_rows[L.lev]));
        }
    }
    {   // Step II: triple sums (Eq. fftbs), all units or one share of them
        int64_t lo[kClassSlots], hi[kClassSlots];
        const int64_t *cb;
        const int ncls = unit_classes(P, &cb);
        for (int c = 0; c < kClassSlots; ++c) lo[c] = hi[c] = 0;
        if (nshares == 1) {
            for (int c = 0; c < ncls; ++c) { lo[c] = cb[c]; hi[c] = cb[c + 1]; }
        } else {
            part_ranges(P, share, nshares, lo, hi);
            // the partial sums of the other shares' units count as zero
            for (unsigned f = 0; f < nf; ++f)
                CK(cudaMemsetAsync(ws + int64_t(f) * fs + p->off_part, 0, size_t(P.n_partials) * sizeof(double), s));
        }
        StageMark m(p, BISP_STAGE_STEP2, step2_launches(lo, hi), s);
        if constexpr (sizeof(R) == 4) {
            if (P.tensor) {
                CK(launch_step2_tc(atc, dstore, lo, hi, int(nf), s));
            } else {
                CK(launch_step2<R>(a2, dstore, lo, hi, int(nf), s));
            }
        } else {
            CK(launch_step2<R>(a2, dstore, lo, hi, int(nf), s));
        }
    }
    {
        StageMark m(p, BISP_STAGE_REDUCE, 1, s);
        using RA = typename std::conditional<std::is_same<S, float>::value, float, double>::type;
        CK(launch_reduce_partials<RA>(p->d_groups, int64_t(P.groups.size()), part, ng, Ssum, region, s));
    }
    {   // binning and the ratio of Eq. bs_lm2_1
        StageMark m(p, BISP_STAGE_BIN, int(2 * P.views.size()), s);
        for (const View &v : P.views) {
            const EpiArgs ea{p->d_rec, p->d_chunk_lo + v.chunk_off, p->d_chunk_hi + v.chunk_off, v.n_chunks,
                             p->d_bin_chunk + v.bc_off, v.n_bins, reinterpret_cast<double *>(ws + p->off_epi), fs};
            CK(launch_epilogue<W>(0, ea, Ssum, v.l_lo, v.l_hi, p->d_den + v.out_off, 1.0 / (P.volume * double(ng2)),
                                  B + v.out_off, to_out, s, p->precision != BISP_PREC_FP64));
        }
    }
    p->last_field = batch - 1;
    return BISP_OK;
}

int dispatch_estimate(bisp_plan *p, const void *delta, int batch, void *ws, double *B, cudaStream_t s,
                      int part = 0, int nparts = 1)
{
    unsigned char *w = static_cast<unsigned char *>(ws);
    switch (p->precision) {
    case BISP_PREC_FP32:
        return run_estimate<float, float, float, float>(p, static_cast<const float *>(delta), batch, w, B, part,
                                                        nparts, s);
    case BISP_PREC_MIXED:
    case BISP_PREC_MIXED_TC:
        return run_estimate<float, float, double, double>(p, static_cast<const float *>(delta), batch, w, B, part,
                                                          nparts, s);
    default:
        return run_estimate<double, double, double, double>(p, static_cast<const double *>(delta), batch, w, B,
                                                            part, nparts, s);
    }
}

}  // namespace

extern "C" {

int estimator_plan(bisp_plan **out, const bisp_desc *desc, void *stream)
{
    g_err.clear();
    if (!out) return fail(BISP_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int st = check_desc(desc);
    if (st) return st;
    bisp_plan *p = nullptr;
    try {
        p = new bisp_plan();
        if (cudaGetDevice(&p->device) != cudaSuccess) p->device = -1;
        st = build_plan(p, desc, static_cast<cudaStream_t>(stream));
    } catch (const std::bad_alloc &) {
        st = fail(BISP_OUT_OF_MEMORY, "host allocation failed while planning");
    } catch (const std::exception &e) {
        st = fail(BISP_INTERNAL, e.what());
    }
    if (st) {
        free_plan(p);
        return st;
    }
    *out = p;
    return BISP_OK;
}

int estimator_plan_info(const bisp_plan *p, bisp_plan_info *info)
{
    if (!p || !info) return fail(BISP_INVALID_ARG, "NULL argument");
    const HostPlan &P = p->hp;
    info->n_g = P.desc.n_g;
    info->n_rings = P.rings.nr;
    info->n_planes = P.rings.nz + 1;
    info->l_max = P.desc.l_max;
    info->n_lm = P.n_lm;
    info->n_k1 = P.desc.n_k1;
    info->n_mu = P.desc.n_mu;
    info->n_t = P.desc.n_t;
    info->n_levels = int(P.levels.size());
    info->n_bins = P.n_bins;
    info->n_combos = P.n_combos;
    info->n_pairs = P.n_pairs;
    info->n_items = int64_t(P.tensor ? P.tc_units.size() : P.units.size());
    info->triple_products = P.triple_products;
    info->dstore_bytes = size_t(P.dstore_elems) * p->celem;
    info->workspace_bytes = p->region_bytes;
    info->resident_bytes = p->resident;
    info->n_views = int(P.views.size());
    info->out_doubles = P.n_out;
    info->pair_products = P.pair_products;
    info->tc_row_points = 0;
    info->tc_lane_points = 0;
    info->tc_mma_products = P.tensor ? P.tc_mma_products : 0;
    info->tc_staged_bytes = 0;
    if (P.tensor)
        for (const TcTile &T : P.tc_tiles) {
            const double m2 = double(T.M) * T.M;
            info->tc_row_points += double(T.nrow) * m2;
            info->tc_lane_points += double(kTcRows) * m2;
            // every stage stages each slot and window field (16 points, 8 bytes each)
            info->tc_staged_bytes += double(T.nslot + T.ncol) * m2 * 8.0;
        }
    return BISP_OK;
}

int estimator_view_info(const bisp_plan *p, int view, bisp_view_info *info)
{
    if (!p || !info) return fail(BISP_INVALID_ARG, "NULL argument");
    const HostPlan &P = p->hp;
    if (view < 0 || view >= int(P.views.size())) return fail(BISP_INVALID_ARG, "view out of range");
    const View &v = P.views[view];
    info->l_lo = v.l_lo;
    info->l_hi = v.l_hi;
    info->n_mu = v.n_mu;
    info->n_t = v.n_t;
    info->n_lm = v.n_lm;
    info->n_bins = v.n_bins;
    info->offset = v.out_off;
    return BISP_OK;
}

size_t estimator_workspace_bytes(const bisp_plan *p, int batch)
{
    if (!p || batch < 1 || batch > p->hp.desc.max_batch) return 0;
    return size_t(batch) * p->region_bytes;
}

int estimator_estimate(bisp_plan *p, const void *delta, int batch, void *workspace, double *B, void *stream)
{
    g_err.clear();
    if (!p || !delta || !workspace || !B) return fail(BISP_INVALID_ARG, "NULL argument");
    if (batch < 1 || batch > p->hp.desc.max_batch) return fail(BISP_INVALID_ARG, "batch out of range");
    if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(BISP_INVALID_ARG, "workspace not 256-byte aligned");
    return dispatch_estimate(p, delta, batch, workspace, B, static_cast<cudaStream_t>(stream));
}

int estimator_stats_update(const double *B, int batch, int64_t n, int64_t *count, double *mean, double *m2,
                           void *stream)
{
    g_err.clear();
    if (!B || !count || !mean || !m2) return fail(BISP_INVALID_ARG, "NULL argument");
    if (batch < 0 || n < 0) return fail(BISP_INVALID_ARG, "batch and n must be >= 0");
    CK(launch_stats_update(B, batch, n, count, mean, m2, static_cast<cudaStream_t>(stream)));
    return BISP_OK;
}

int estimator_estimate_part(bisp_plan *p, const void *delta, int batch, void *workspace, double *B_part, int part,
                            int nparts, void *stream)
{
    g_err.clear();
    if (!p || !delta || !workspace || !B_part) return fail(BISP_INVALID_ARG, "NULL argument");
    if (batch < 1 || batch > p->hp.desc.max_batch) return fail(BISP_INVALID_ARG, "batch out of range");
    if (nparts < 1 || part < 0 || part >= nparts) return fail(BISP_INVALID_ARG, "part must satisfy 0 <= part < nparts");
    if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(BISP_INVALID_ARG, "workspace not 256-byte aligned");
    return dispatch_estimate(p, delta, batch, workspace, B_part, static_cast<cudaStream_t>(stream), part, nparts);
}

int estimator_estimate_host(bisp_plan *p, const void *delta_host, int batch, double *B_host, void *stream)
{
    g_err.clear();
    if (!p || !delta_host || !B_host) return fail(BISP_INVALID_ARG, "NULL argument");
    if (batch < 1 || batch > p->hp.desc.max_batch) return fail(BISP_INVALID_ARG, "batch out of range");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const HostPlan &P = p->hp;
    const size_t field = size_t(P.desc.n_g) * P.desc.n_g * P.desc.n_g *
                         (p->precision == BISP_PREC_FP64 ? sizeof(double) : sizeof(float));
    const size_t outb = size_t(P.n_out) * sizeof(double);
    if (!p->own_ws) {
        CK(cudaMalloc(&p->own_ws, std::max<size_t>(size_t(P.desc.max_batch) * p->region_bytes, 256)));
        CK(cudaMalloc(&p->own_in, field * P.desc.max_batch));
        CK(cudaMalloc((void **)&p->own_out, outb * P.desc.max_batch));
    }
    CK(cudaMemcpyAsync(p->own_in, delta_host, field * batch, cudaMemcpyHostToDevice, s));
    int st = dispatch_estimate(p, p->own_in, batch, p->own_ws, p->own_out, s);
    if (st) return st;
    CK(cudaMemcpyAsync(B_host, p->own_out, outb * batch, cudaMemcpyDeviceToHost, s));
    return estimator_workspace_status(p, p->own_ws, batch, stream);
}

int estimator_host_submit(bisp_plan *p, const void *delta_host, int batch, double *B_host, void *stream)
{
    g_err.clear();
    if (!p || !delta_host || !B_host) return fail(BISP_INVALID_ARG, "NULL argument");
    if (batch < 1 || batch > p->hp.desc.max_batch) return fail(BISP_INVALID_ARG, "batch out of range");
    auto &h = p->pipe;
    if (h.count == 2) return fail(BISP_INVALID_ARG, "two submissions in flight: call estimator_host_wait first");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const HostPlan &P = p->hp;
    const int mb = P.desc.max_batch;
    const size_t field = size_t(P.desc.n_g) * P.desc.n_g * P.desc.n_g *
                         (p->precision == BISP_PREC_FP64 ? sizeof(double) : sizeof(float));
    const size_t outb = size_t(P.n_out) * sizeof(double);
    if (!h.copy) {
        if (!p->own_ws) CK(cudaMalloc(&p->own_ws, std::max<size_t>(size_t(mb) * p->region_bytes, 256)));
        CK(cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking));
        CK(cudaMallocHost((void **)&h.status_h, sizeof(int) * 2 * size_t(mb)));
        for (int i = 0; i < 2; ++i) {
            CK(cudaMalloc(&h.in[i], field * mb));
            CK(cudaMalloc((void **)&h.out[i], outb * mb));
            CK(cudaEventCreateWithFlags(&h.in_ready[i], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h.in_free[i], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h.done[i], cudaEventDisableTiming));
        }
    }
    const int k = (h.head + h.count) % 2;       // the slot of this submission
    // input copy on the plan's copy stream, once the estimate that last read
    // this slot's input is done (an event not yet recorded is no wait)
    CK(cudaStreamWaitEvent(h.copy, h.in_free[k], 0));
    CK(cudaMemcpyAsync(h.in[k], delta_host, field * batch, cudaMemcpyHostToDevice, h.copy));
    CK(cudaEventRecord(h.in_ready[k], h.copy));
    // the estimate, its wait status and the output copy on the caller's stream
    CK(cudaStreamWaitEvent(s, h.in_ready[k], 0));
    int st = dispatch_estimate(p, h.in[k], batch, p->own_ws, h.out[k], s);
    if (st) return st;
    CK(cudaEventRecord(h.in_free[k], s));
    CK(cudaMemcpy2DAsync(h.status_h + size_t(k) * mb, sizeof(int),
                         static_cast<unsigned char *>(p->own_ws) + p->off_status, p->region_bytes, sizeof(int),
                         size_t(batch), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(B_host, h.out[k], outb * batch, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(h.done[k], s));
    h.batch[k] = batch;
    ++h.count;
    return BISP_OK;
}

int estimator_host_wait(bisp_plan *p, void *stream)
{
    (void)stream;
    g_err.clear();
    if (!p) return fail(BISP_INVALID_ARG, "NULL plan");
    auto &h = p->pipe;
    if (h.count == 0) return fail(BISP_INVALID_ARG, "no submission in flight");
    const int k = h.head;
    CK(cudaEventSynchronize(h.done[k]));
    h.head = (h.head + 1) % 2;
    --h.count;
    int bad = 0;
    const int mb = p->hp.desc.max_batch;
    for (int f = 0; f < h.batch[k]; ++f) bad |= h.status_h[size_t(k) * mb + f] != 0;
    if (bad) return fail(BISP_TIMEOUT, "a tensor-core Step-II block gave up a bounded wait; its sums are NaN");
    return BISP_OK;
}

}  // extern "C"

struct bisp_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t own = nullptr;
};

extern "C" {

int estimator_graph_create(bisp_graph **out, bisp_plan *p, const void *delta, int batch, void *workspace,
                           double *B, void *stream)
{
    g_err.clear();
    if (!out) return fail(BISP_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!p || !delta || !workspace || !B) return fail(BISP_INVALID_ARG, "NULL argument");
    if (batch < 1 || batch > p->hp.desc.max_batch) return fail(BISP_INVALID_ARG, "batch out of range");
    if (reinterpret_cast<uintptr_t>(workspace) % 256) return fail(BISP_INVALID_ARG, "workspace not 256-byte aligned");
    bisp_graph *g = new (std::nothrow) bisp_graph();
    if (!g) return fail(BISP_OUT_OF_MEMORY, "host allocation failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto bail = [&](int st) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        if (g->own) cudaStreamDestroy(g->own);
        delete g;
        cudaGetLastError();
        return st;
    };
    if (!s) {
        if (cudaStreamCreateWithFlags(&g->own, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(BISP_CUDA_ERROR, "stream for capture"));
        s = g->own;
    }
    const bool timing = p->timing;
    p->timing = false;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        p->timing = timing;
        return bail(fail(BISP_CUDA_ERROR, std::string("begin capture: ") + cudaGetErrorString(e)));
    }
    const int st = dispatch_estimate(p, delta, batch, workspace, B, s);
    e = cudaStreamEndCapture(s, &g->graph);
    p->timing = timing;
    if (st) return bail(st);
    if (e != cudaSuccess) return bail(fail(BISP_CUDA_ERROR, std::string("end capture: ") + cudaGetErrorString(e)));
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) return bail(fail(BISP_CUDA_ERROR, std::string("instantiate: ") + cudaGetErrorString(e)));
    *out = g;
    return BISP_OK;
}

int estimator_graph_launch(bisp_graph *g, void *stream)
{
    if (!g || !g->exec) return fail(BISP_INVALID_ARG, "NULL graph");
    CK(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
    return BISP_OK;
}

void estimator_graph_destroy(bisp_graph *g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->own) cudaStreamDestroy(g->own);
    delete g;
}

int estimator_workspace_status(const bisp_plan *p, const void *workspace, int batch, void *stream)
{
    if (!p) return fail(BISP_INVALID_ARG, "NULL plan");
    if (batch < 1 || batch > p->hp.desc.max_batch) return fail(BISP_INVALID_ARG, "batch out of range");
    const unsigned char *ws = static_cast<const unsigned char *>(workspace);
    if (!ws) {
        void *a = nullptr;
        const int st = static_scratch_address(&a);
        if (st) return st;
        ws = static_cast<const unsigned char *>(a);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<int> h(size_t(batch), 0);
    CK(cudaMemcpy2DAsync(h.data(), sizeof(int), ws + p->off_status, p->region_bytes, sizeof(int), size_t(batch),
                         cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int bad = 0;
    for (int v : h) bad |= v != 0;
    if (!bad) return BISP_OK;
    CK(cudaMemset2DAsync(const_cast<unsigned char *>(ws) + p->off_status, p->region_bytes, 0, sizeof(int),
                         size_t(batch), s));
    CK(cudaStreamSynchronize(s));
    return fail(BISP_TIMEOUT, "a tensor-core Step-II block gave up a bounded wait; its sums are NaN");
}

int estimator_set_wait_limit(bisp_plan *p, int spins)
{
    if (!p) return fail(BISP_INVALID_ARG, "NULL plan");
    if (spins < 0) return fail(BISP_INVALID_ARG, "negative wait limit");
    p->wait_spins = spins == 0 ? kDefaultWaitSpins : spins;
    return BISP_OK;
}

void estimator_destroy(bisp_plan *p) { free_plan(p); }

int estimator_set_timing(bisp_plan *p, int on)
{
    if (!p) return fail(BISP_INVALID_ARG, "NULL plan");
    int st = collect_times(p);
    if (st) return st;
    p->timing = on != 0;
    if (p->timing)
        for (int i = 0; i < BISP_N_STAGES; ++i) { p->stage_ms[i] = 0; p->stage_launches[i] = 0; }
    return BISP_OK;
}

int estimator_stage_times(bisp_plan *p, double *ms, int64_t *launches)
{
    if (!p) return fail(BISP_INVALID_ARG, "NULL plan");
    int st = collect_times(p);
    if (st) return st;
    for (int i = 0; i < BISP_N_STAGES; ++i) {
        if (ms) ms[i] = p->stage_ms[i];
        if (launches) launches[i] = p->stage_launches[i];
    }
    return BISP_OK;
}

int estimator_stage_flops(const bisp_plan *p, double *flops)
{
    if (!p || !flops) return fail(BISP_INVALID_ARG, "NULL argument");
    const HostPlan &P = p->hp;
    const double ng = P.desc.n_g, lg = ilog2i(P.desc.n_g), planes = P.rings.nz + 1;
    // 5 N log2 N per complex transform of length N
    flops[BISP_STAGE_FORWARD] = 5.0 * ng * lg * (ng * ng + 2.0 * planes * ng);
    double s1 = 0;
    for (const Level &L : P.levels) {
        const double M = double(L.M);
        s1 += double(L.njobs) * 2.0 * M * 5.0 * M * std::log2(M);
    }
    flops[BISP_STAGE_STEP1] = s1;
    flops[BISP_STAGE_STEP2] = 4.0 * P.triple_products + 6.0 * P.pair_products;
    flops[BISP_STAGE_REDUCE] = double(P.n_partials);
    flops[BISP_STAGE_BIN] = 0;
    for (const View &v : P.views) flops[BISP_STAGE_BIN] += double(P.n_combos) * 4.0 * (v.l_hi / 2 + 1) * (v.l_hi / 2 + 1);
    return BISP_OK;
}

const char *estimator_status_string(int status)
{
    switch (status) {
    case BISP_OK: return "ok";
    case BISP_INVALID_ARG: return "invalid argument";
    case BISP_UNSUPPORTED_SIZE: return "unsupported grid size";
    case BISP_OUT_OF_MEMORY: return "out of memory";
    case BISP_CUDA_ERROR: return "CUDA error";
    case BISP_TIMEOUT: return "device wait timed out";
    case BISP_INTERNAL: return "internal error";
    default: return "unknown status";
    }
}

const char *estimator_last_error(void) { return g_err.c_str(); }

int estimator_denominator(const bisp_plan *p, double *den)
{
    if (!p || !den) return fail(BISP_INVALID_ARG, "NULL argument");
    std::memcpy(den, p->h_den.data(), p->h_den.size() * sizeof(double));
    return BISP_OK;
}

int64_t estimator_combo_table(const bisp_plan *p, int64_t cap, int32_t *ints, int64_t *ntri, int32_t *bin,
                              int32_t *grid)
{
    if (!p) return -1;
    const HostPlan &P = p->hp;
    const int nr = P.rings.nr;
    for (const Group &G : P.groups)
        for (int s = 0; s < G.nrow; ++s) {
            const Row &q = P.rows[G.row0 + s];
            for (int j = 0; j < q.n; ++j) {
                const int64_t k = G.c0 + q.coff + j;
                if (k >= cap) continue;
                const int r3 = q.r3a + j;
                if (ints) {
                    int32_t *o = ints + 6 * k;
                    o[0] = G.n1; o[1] = G.n2; o[2] = G.n3;
                    o[3] = q.r1; o[4] = q.r2; o[5] = r3;
                }
                if (ntri) ntri[k] = P.ntri[(size_t(q.r1) * nr + q.r2) * nr + r3];
                if (bin) bin[k] = P.combo_bin[k];
                if (grid) grid[k] = G.M;
            }
        }
    return P.n_combos;
}

int64_t estimator_combo_geometry(const bisp_plan *p, int64_t cap, double *geo)
{
    if (!p) return -1;
    if (geo) combo_shapes(p->hp, cap, geo);
    return p->hp.n_combos;
}

int estimator_combo_sums(const bisp_plan *p, const void *workspace, double *S, void *stream)
{
    if (!p || !workspace || !S) return fail(BISP_INVALID_ARG, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaMemcpyAsync(S, static_cast<const unsigned char *>(workspace) + size_t(p->last_field) * p->region_bytes + p->off_S,
                       size_t(p->hp.n_combos) * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return BISP_OK;
}

static int copy_complex_out(const bisp_plan *p, const unsigned char *src, int64_t n, double *out, cudaStream_t s)
{
    if (p->celem == sizeof(double2)) {
        CK(cudaMemcpyAsync(out, src, size_t(n) * 16, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    } else {
        std::vector<float> tmp(size_t(n) * 2);
        CK(cudaMemcpyAsync(tmp.data(), src, size_t(n) * 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (size_t i = 0; i < tmp.size(); ++i) out[i] = tmp[i];
    }
    return BISP_OK;
}

int estimator_dfield(const bisp_plan *p, const void *workspace, int M, int n, int r, double *out, void *stream)
{
    if (!p || !workspace || !out) return fail(BISP_INVALID_ARG, "NULL argument");
    const HostPlan &P = p->hp;
    int lv = -1;
    for (int l = 0; l < P.rings.ngrid; ++l)
        if (P.rings.grid[l] == M) lv = l;
    if (lv < 0 || n < 0 || n > P.rings.nz || r < 0 || r >= P.rings.nr)
        return fail(BISP_INVALID_ARG, "no such field");
    const int64_t o = P.doff[(size_t(lv) * (P.rings.nz + 1) + n) * kMaxRings + r];
    if (o < 0) return fail(BISP_INVALID_ARG, "field not stored on this grid");
    const unsigned char *src = static_cast<const unsigned char *>(workspace) + size_t(p->last_field) * p->region_bytes +
                               p->off_dstore + size_t(o) * p->celem;
    return copy_complex_out(p, src, int64_t(M) * M, out, static_cast<cudaStream_t>(stream));
}

int estimator_delta_plane(const bisp_plan *p, const void *workspace, int n, double *out, void *stream)
{
    if (!p || !workspace || !out) return fail(BISP_INVALID_ARG, "NULL argument");
    const HostPlan &P = p->hp;
    if (n < 0 || n > P.rings.nz) return fail(BISP_INVALID_ARG, "plane out of range");
    const int64_t ng2 = int64_t(P.desc.n_g) * P.desc.n_g;
    const unsigned char *src = static_cast<const unsigned char *>(workspace) + size_t(p->last_field) * p->region_bytes +
                               p->off_a + size_t(n) * ng2 * p->celem;
    return copy_complex_out(p, src, ng2, out, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
