// step2_tc.cu -- Step II of the estimator (the triple sums of Eq. fftbs,
// Gill & Bharadwaj, arXiv:2405.14513, Sec. II) on the tcgen05 tensor cores
// of sm_103a.
//
// A tile holds up to 128 rows (r1, r2), each of some plane pair (n1, n2),
// and a window of NC consecutive rings r3lo .. r3lo + NC - 1 of plane n3
// (all rows of a tile share the reduction grid and |n3|).  Its sums
//   S[row][c] = sum_x Re( P_row(x) D(r3lo + c, n3; x) ),  P_row = D(r1, n1) D(r2, n2),
// are a real matrix product over k = 2x + (0: real part, 1: imaginary part):
//   A[row][2x] = Re P,  A[row][2x + 1] = -g3 Im P,
//   B[c][2x]  = Re D3,  B[c][2x + 1]  = Im D3,
// with D3 the stored field of plane |n3| and g3 = -1 when n3 < 0 (the field
// of a negative plane is the conjugate of the stored one; likewise g1, g2 in
// P).  The CUDA cores form A and store it to tensor memory (lane = row); B
// is staged in shared memory in the K-major canonical layout (core matrices
// of 8 rows x 16 bytes, no swizzle); one thread issues the MMAs
// (M = 128, N = NC, K = 8, kind::tf32, FP32 accumulator in tensor memory).
//
// Precision.  A tf32 MMA reads the top 19 bits of each FP32 operand (it
// truncates), so every operand is split x = hi + lo with hi = x with its 13
// low mantissa bits cleared (the raw x is passed: the MMA drops those bits
// itself) and lo = x - hi, exact in FP32; the product is taken as
// hi hi' + lo hi' + hi lo' (lo lo' is below FP32 rounding), which keeps
// FP32 accuracy.  The tensor-memory accumulator (it also truncates when it
// accumulates) holds one stage of 16 grid points; every stage is added
// into FP32 registers, and each unit's sums go out as FP64 partials, as in
// the CUDA-core kernel.
#include "kernels.cuh"

#include <algorithm>

namespace bisp {

namespace {

constexpr int kTX = 16;                      // grid points per stage (K = 32)
constexpr int kSlotBytes = kTX * 8 + 16;     // one staged D1 / D2 field row, padded
constexpr uint32_t kTmemCols = 128;          // A hi [0, 32), A lo [32, 64), D [64, 64 + NC)
constexpr int kWaitSpins = 1 << 22;          // bound of a tensor-core completion wait

__device__ __forceinline__ uint32_t su32(const void *p) { return uint32_t(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

// Shared-memory matrix descriptor of tcgen05: start address, leading byte
// offset (next core matrix along K), stride byte offset (next 8 rows along
// M / N), all in 16-byte units; bits 46-47 = 1 (descriptor version); no
// swizzle, base offset 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return uint64_t((addr & 0x3FFFF) >> 4) | (uint64_t((lbo & 0x3FFFF) >> 4) << 16) |
           (uint64_t((sbo & 0x3FFFF) >> 4) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor: FP32 accumulator, A and B tf32, both K-major, N, M.
template <int N>
__host__ __device__ constexpr uint32_t idesc_tf32()
{
    return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
                 ::"r"(d), "r"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                   "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
                   "r"(v[15]) : "memory");
}

// 16 columns of this thread's lane; the wait is in the same statement so the
// registers are not read before the load completes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15])
                 : "r"(taddr) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity)
{
    for (int i = 0; i < kWaitSpins; ++i) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(mb), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

template <int NC>
__device__ __forceinline__ void add_accumulator(uint32_t tcol, float (&acc)[NC])
{
#pragma unroll
    for (int q = 0; q < NC / 16; ++q) {
        uint32_t v[16];
        tmem_ld16(tcol + 16 * q, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[16 * q + j] += __uint_as_float(v[j]);
    }
}

template <int NC>
__global__ void __launch_bounds__(128, 4)
k_step2_tc(TcArgs args, int64_t unit0, const float2 *__restrict__ dstore)
{
    constexpr int NB = NC / 8;                   // 8-row groups of B
    constexpr uint32_t LBO = NB * 128;           // next core matrix along K
    constexpr uint32_t SBO = 128;                // next 8 rows of B
    constexpr int BB = NC * kTX * 8;             // bytes of one stage of B
    constexpr uint32_t ID = idesc_tf32<NC>();
    extern __shared__ __align__(1024) unsigned char smem[];

    const TcUnit U = args.units[unit0 + blockIdx.x];
    const TcTile T = args.tiles[U.tile];
    const int t = threadIdx.x, warp = t >> 5;
    const int nslot = T.nslot, nf = nslot + NC;
    // shared memory: B stages [2][BB], B lo [BB], D1 / D2 stages
    // [2][nslot][kSlotBytes], field offsets [nf], mbarrier, tensor-memory address
    unsigned char *sB = smem;
    unsigned char *sLo = smem + 2 * BB;
    unsigned char *sS = smem + 3 * BB;
    int64_t *offs = reinterpret_cast<int64_t *>(sS + 2 * size_t(nslot) * kSlotBytes);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(offs + nf);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 1);

    for (int f = t; f < nf; f += 128) {
        int64_t o = -1;
        if (f < nslot) {
            const int32_t v = args.slots[T.slot0 + f];
            o = args.doff[(size_t(T.lev) * args.nz1 + (v >> 8)) * kMaxRings + (v & 255)];
        } else {
            const int r = T.r3lo + f - nslot;
            if (r < args.nr) o = args.doff[(size_t(T.lev) * args.nz1 + T.n3abs) * kMaxRings + r];
        }
        offs[f] = o;
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(su32(tslot)), "n"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    const bool live = t < T.nrow;
    TcRow R{};
    if (live) R = args.rows[T.row0 + t];
    const float g1 = (R.flags & 1) ? -1.f : 1.f, g2 = (R.flags & 2) ? -1.f : 1.f, g3 = (R.flags & 4) ? -1.f : 1.f;
    const float k12 = -g1 * g2, kb = -g3 * g2, ka = -g3 * g1;
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t tlane = tmem + (uint32_t(warp * 32) << 16);

    // fields that are not stored (past the last ring) read as zero in both stages
    for (int i = t; i < 2 * nf * 8; i += 128) {
        const int b = i / (nf * 8), rem = i - b * nf * 8, f = rem >> 3, p = rem & 7;
        if (offs[f] >= 0) continue;
        unsigned char *d = f < nslot ? sS + (size_t(b) * nslot + f) * kSlotBytes + p * 16
                                     : sB + b * BB + (p * NB + (f - nslot) / 8) * 128 + ((f - nslot) & 7) * 16;
        *reinterpret_cast<float4 *>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
    }

    const int64_t M2 = int64_t(T.M) * T.M;
    const int64_t x0 = int64_t(U.chunk) * args.x_chunk;
    const int64_t x1 = min(M2, x0 + args.x_chunk);
    const int nstage = int((x1 - x0) / kTX);
    // 16-byte piece p (grid points 2p, 2p + 1) of every field for stage st;
    // B pieces land in the canonical layout: core matrix (K block p, rows
    // 8 (c / 8) ..), row c % 8
    auto issue = [&](int st) {
        const int b = st & 1;
        const int64_t xs = x0 + int64_t(st) * kTX;
        for (int i = t; i < nf * 8; i += 128) {
            const int f = i >> 3, p = i & 7;
            const int64_t o = offs[f];
            if (o < 0) continue;
            const uint32_t d = f < nslot ? su32(sS + (size_t(b) * nslot + f) * kSlotBytes + p * 16)
                                         : su32(sB + b * BB + (p * NB + (f - nslot) / 8) * 128 + ((f - nslot) & 7) * 16);
            cp_async16(d, dstore + o + xs + 2 * p);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    float acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.f;
    const uint32_t mb = su32(mbar);
    int failed = 0;
    if (nstage > 0) issue(0);
    for (int st = 0; st < nstage; ++st) {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        // the previous stage's MMAs read B stage (st - 1) & 1, B lo and A, and wrote D
        int late = 0;
        if (st > 0 && t == 0) late = !mbar_wait(mb, uint32_t(st - 1) & 1);
        if (__syncthreads_or(late)) {
            failed = 1;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (st + 1 < nstage) issue(st + 1);
        if (st > 0) add_accumulator<NC>(tlane + 64, acc);
        const int b = st & 1;
        // low parts of B
        for (int i = t; i < NC * 8; i += 128) {
            const float4 v = *reinterpret_cast<const float4 *>(sB + b * BB + i * 16);
            *reinterpret_cast<float4 *>(sLo + i * 16) =
                make_float4(v.x - tf32_hi(v.x), v.y - tf32_hi(v.y), v.z - tf32_hi(v.z), v.w - tf32_hi(v.w));
        }
        // A: the row's pair products, high and low parts, to tensor memory
        {
            const unsigned char *p1 = sS + (size_t(b) * nslot + R.s1) * kSlotBytes;
            const unsigned char *p2 = sS + (size_t(b) * nslot + R.s2) * kSlotBytes;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 u = *reinterpret_cast<const float4 *>(p1 + (h * 4 + q) * 16);
                    const float4 v = *reinterpret_cast<const float4 *>(p2 + (h * 4 + q) * 16);
                    float e[4];
                    e[0] = fmaf(u.x, v.x, k12 * (u.y * v.y));
                    e[1] = fmaf(kb * u.x, v.y, ka * (u.y * v.x));
                    e[2] = fmaf(u.z, v.z, k12 * (u.w * v.w));
                    e[3] = fmaf(kb * u.z, v.w, ka * (u.w * v.z));
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float x = live ? e[j] : 0.f;
                        hi[4 * q + j] = __float_as_uint(x);
                        lo[4 * q + j] = __float_as_uint(x - tf32_hi(x));
                    }
                }
                tmem_st16(tlane + 16 * h, hi);
                tmem_st16(tlane + 32 + 16 * h, lo);
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t bh = su32(sB + b * BB), bl = su32(sLo), d = tmem + 64;
#pragma unroll
            for (int j = 0; j < 4; ++j) mma_tf32(d, tmem + 8 * j, smem_desc(bh + 2 * j * LBO, LBO, SBO), ID, j > 0);
#pragma unroll
            for (int j = 0; j < 4; ++j) mma_tf32(d, tmem + 32 + 8 * j, smem_desc(bh + 2 * j * LBO, LBO, SBO), ID, 1);
#pragma unroll
            for (int j = 0; j < 4; ++j) mma_tf32(d, tmem + 8 * j, smem_desc(bl + 2 * j * LBO, LBO, SBO), ID, 1);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                         ::"r"(mb) : "memory");
        }
    }
    if (!failed && nstage > 0) {
        int late = 0;
        if (t == 0) late = !mbar_wait(mb, uint32_t(nstage - 1) & 1);
        if (__syncthreads_or(late)) {
            failed = 1;
        } else {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            add_accumulator<NC>(tlane + 64, acc);
        }
    }
    if (live) {
        double *dst = args.partials + R.p0 + int64_t(U.chunk) * R.stride;
        const double nan = __longlong_as_double(0x7FF8000000000000LL);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int j = c - int(R.col0);
            if (j >= 0 && j < int(R.n)) dst[j] = failed ? nan : double(acc[c]);
        }
    }
    if (failed && t == 0) atomicExch(args.status, 1);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(kTmemCols) : "memory");
    }
}

template <int NC>
cudaError_t launch_class(const TcArgs &a, const float2 *dstore, int64_t u0, int64_t n, size_t smem, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_step2_tc<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    k_step2_tc<NC><<<unsigned(n), 128, smem, s>>>(a, u0, dstore);
    return cudaGetLastError();
}

}  // namespace

size_t step2_tc_smem(int cls, int nslot)
{
    const int nc = 16 * (cls + 1);
    const size_t need = size_t(3) * nc * kTX * 8 + size_t(2) * nslot * kSlotBytes + 8 * size_t(nslot + nc) + 16;
    // at least 56 KB so that at most four blocks (4 x 128 tensor-memory
    // columns) share an SM
    return std::max<size_t>(need, 56 * 1024);
}

cudaError_t launch_step2_tc(const TcArgs &a, const float2 *dstore, const int64_t *cb, const int *cs, cudaStream_t s)
{
    cudaError_t e = launch_class<16>(a, dstore, cb[0], cb[1] - cb[0], step2_tc_smem(0, cs[0]), s);
    if (e == cudaSuccess) e = launch_class<32>(a, dstore, cb[1], cb[2] - cb[1], step2_tc_smem(1, cs[1]), s);
    if (e == cudaSuccess) e = launch_class<48>(a, dstore, cb[2], cb[3] - cb[2], step2_tc_smem(2, cs[2]), s);
    if (e == cudaSuccess) e = launch_class<64>(a, dstore, cb[3], cb[4] - cb[3], step2_tc_smem(3, cs[3]), s);
    return e;
}

}  // namespace bisp
