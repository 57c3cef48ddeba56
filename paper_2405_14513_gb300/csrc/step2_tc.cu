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
// P).  The fields of a stage (16 grid points = 128 bytes each) are staged
// in shared memory by cp.async; the CUDA cores form A and store it to
// tensor memory (lane = row) and write B, split into high and low parts, in
// the K-major canonical layout (core matrices of 8 rows x 16 bytes, no
// swizzle); one thread issues the MMAs (M = 128, N = NC, K = 8, kind::tf32,
// FP32 accumulator in tensor memory).
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

constexpr int kTX = kTcTX;                   // grid points per stage (K = 32)
constexpr int kSlotBytes = kTcSlotBytes;     // a field's row of a ring buffer: two stages (+ padding)
constexpr uint32_t kTmemCols = 256;          // A[tc_abuf] (hi 32 + lo 32 columns each), then the accumulators
constexpr int kDrainSpins = kDefaultWaitSpins;  // bound of the wait for the block's own MMAs

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

// One MMA, issued by one elected lane of a converged warp whose lanes all
// hold the same operands.  Issued this way the operands stay warp-uniform,
// and a stage's twelve MMAs issue in ~15 cycles each; issued from a single
// lane (inside a lane test) they took ~48.
__device__ __forceinline__ void mma_tf32(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile("{\n.reg .pred p, e;\nsetp.ne.b32 p, %4, 0;\nelect.sync _|e, 0xffffffff;\n"
                 "@e tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
                 ::"r"(d), "r"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}

// tcgen05.commit of the warp's MMAs to mbarrier m, by one elected lane
__device__ __forceinline__ void mma_commit(uint32_t m)
{
    asm volatile("{\n.reg .pred e;\nelect.sync _|e, 0xffffffff;\n"
                 "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n"
                 ::"r"(m) : "memory");
}

// -hi(x): x with its 13 low mantissa bits cleared, negated (one logical operation)
__device__ __forceinline__ uint32_t tf32_neg_hi(float x) { return (__float_as_uint(x) & 0xFFFFE000u) ^ 0x80000000u; }

// (a, b) += (x, y): one packed FP32 addition (round to nearest, as two
// scalar additions would be)
__device__ __forceinline__ void add2(float &a, float &b, uint32_t x, uint32_t y)
{
    asm("{\n.reg .b64 p, q;\nmov.b64 p, {%0, %1};\nmov.b64 q, {%2, %3};\nadd.rn.f32x2 p, p, q;\nmov.b64 {%0, %1}, p;\n}\n"
        : "+f"(a), "+f"(b) : "r"(x), "r"(y));
}

// (lo(x), lo(y)) = (x - hi(x), y - hi(y)), exact
__device__ __forceinline__ void lo2(float x, float y, uint32_t &lx, uint32_t &ly)
{
    float a = x, b = y;
    add2(a, b, tf32_neg_hi(x), tf32_neg_hi(y));
    lx = __float_as_uint(a);
    ly = __float_as_uint(b);
}

// No memory clobber: tensor memory is not memory the compiler tracks, so
// shared-memory loads of the next points may be scheduled across the store
// (its order against tcgen05.wait::st and the fences, all volatile, stays).
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                   "r"(v[7]));
}

// The loads below keep the wait in the same statement, so the registers are
// not read before the load completes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 "tcgen05.wait::ld.sync.aligned;\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr) : "memory");
}

// acc[j] += accumulator column tcol + j, j < NH (NH a multiple of 8)
template <int NH>
__device__ __forceinline__ void add_accumulator(uint32_t tcol, float (&acc)[NH])
{
#pragma unroll
    for (int q = 0; q < NH / 8; ++q) {
        uint32_t v[8];
        tmem_ld8(tcol + 8 * q, v);
#pragma unroll
        for (int j = 0; j < 8; j += 2) add2(acc[8 * q + j], acc[8 * q + j + 1], v[j], v[j + 1]);
    }
}

// One block per unit (tile, x chunk), warp-specialised:
//   warps 0-7  form A and write B's high and low parts into buffer
//              st % NA of stage st (NA = tc_abuf(NC): 3 for NC <= 32, else
//              2; A in tensor-memory columns 64 a .. 64 a + 63); warps w and
//              w + 4 share tensor-memory lanes 32 (w % 4) .. (the tile's
//              rows, one per lane): warp w forms grid points 0-7 of a stage
//              and adds accumulator columns 0 .. NC/2 - 1 into FP32
//              registers, warp w + 4 points 8-15 and columns NC/2 .. NC - 1,
//              reading the accumulators of stage st - (NA - 1) after forming
//              stage st;
//   warp 8     issues the 12 MMAs of a stage (one elected lane) into
//              accumulator buffer st & 1 (tensor-memory columns from 64 NA,
//              NC apart with three A buffers, 64 apart with two).  The MMAs
//              of stage st wait for A(st) only: every compute thread read
//              stage st - 2's accumulators (the buffer they overwrite) before
//              it signalled A(st).  (A second issuer with an accumulator of its
//              own was slower: a second accumulator doubles the compute
//              warps' reads);
//   warps 9-10 stage the fields of each stage in shared memory (cp.async,
//              a ring of 2 to 4 buffers of two stages each: 32 grid points
//              a field row, waited for and released once per two stages).
// mbarriers (phase k of a barrier = its k-th use):
//   full[q]   the data of ring buffer q landed        (64 producer arrivals)
//   empty[q]  ring buffer q has been read             (1 arrival: the MMA warp,
//                                                      once it has seen A of
//                                                      the buffer's last stage,
//                                                      which every compute
//                                                      thread signals after its
//                                                      reads of the buffer)
//   aready[a] A and B (high, low) of buffer a written (256 compute arrivals)
//   mdone[b]  the MMAs into accumulator b are done    (commit)
//   drain     every MMA the block issued is done      (commit; before the
//             tensor memory is freed, also when the block gives up early)
// A barrier's next phase cannot complete before its waiters have seen the
// current one: A(st + NA) is formed only after the accumulators of stage st
// were read, which waited for mdone of stage st, and the MMAs of stage
// st + 2 wait for A(st + 2), signalled after that read.
constexpr int kThreads = 352;
constexpr int kCompute = 256;
constexpr int kProdFields = (kTcMaxSlots + kTcMaxCols + 7) / 8;   // fields per producer lane

struct TcSync {
    uint64_t full[kTcMaxRing], empty[kTcMaxRing], aready[3], mdone[2], drain;
    uint32_t tmem;
    int abort;
};
static_assert(sizeof(TcSync) <= 256, "barriers fit the fixed shared-memory allowance");

__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(m)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *m)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(su32(m)) : "memory");
}

// Bounded wait for phase `parity` of m; gives up (false) when the block is
// aborting or after `spins` polls, and then raises the abort flag.  A poll
// is a try_wait, which may suspend the thread for a while before it reports;
// under kTestPolls polls (a limit set to exercise the give-up path) it is a
// test_wait, which reports at once, so that such a limit really cuts the
// wait short.
constexpr int kTestPolls = 64;
__device__ __forceinline__ bool mbar_wait_abort(uint64_t *m, uint32_t parity, volatile int *abort, int spins)
{
    const uint32_t a = su32(m);
    const bool test = spins < kTestPolls;
    for (int i = 0; i < spins; ++i) {
        uint32_t ok;
        if (test)
            asm volatile("{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                         : "=r"(ok) : "r"(a), "r"(parity) : "memory");
        else
            asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                         : "=r"(ok) : "r"(a), "r"(parity) : "memory");
        if (ok) return true;
        if (*abort) return false;
    }
    *abort = 1;
    return false;
}

// Bounded wait for phase `parity` of m that does not stop at the abort flag
// (waits for the block's own tensor-core work; always the full bound).
__device__ __forceinline__ void mbar_wait_bounded(uint64_t *m, uint32_t parity)
{
    const uint32_t a = su32(m);
    for (int i = 0; i < kDrainSpins; ++i) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(a), "r"(parity) : "memory");
        if (ok) return;
    }
}

// The A columns of half a stage (grid points 8 half .. 8 half + 7) for this
// thread's row: P = D1' D2' with D' the stored field or its conjugate (G1,
// G2: n1 < 0, n2 < 0), and A = (Re P, -g3 Im P) (G3: n3 < 0), high parts at
// column a + 16 half, low parts at a + 32 + 16 half.  u8, v8: the row's two
// staged fields (16 points each).
template <bool G1, bool G2, bool G3>
__device__ __forceinline__ void form_a(const unsigned char *u8, const unsigned char *v8, uint32_t a, int half)
{
    // Re P = ux vx - g1 g2 uy vy;  -g3 Im P = s2 ux vy + s1 uy vx,
    // s2 = -g3 g2, s1 = -g3 g1
    constexpr bool NEG12 = (G1 == G2);            // the uy vy term enters with -
    constexpr bool NEG2 = !(G3 ^ G2);             // s2 = -1
    constexpr bool NEG1 = !(G3 ^ G1);             // s1 = -1
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {              // 4 grid points = 8 columns
        const int h = 2 * half + hh;
        uint32_t hi[8], lo[8];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float4 u = *reinterpret_cast<const float4 *>(u8 + (h * 2 + k) * 16);
            const float4 v = *reinterpret_cast<const float4 *>(v8 + (h * 2 + k) * 16);
            float e[4];
            const float t0 = u.y * v.y, t1 = u.y * v.x, t2 = u.w * v.w, t3 = u.w * v.z;
            e[0] = fmaf(u.x, v.x, NEG12 ? -t0 : t0);
            e[1] = fmaf(NEG2 ? -u.x : u.x, v.y, NEG1 ? -t1 : t1);
            e[2] = fmaf(u.z, v.z, NEG12 ? -t2 : t2);
            e[3] = fmaf(NEG2 ? -u.z : u.z, v.w, NEG1 ? -t3 : t3);
#pragma unroll
            for (int j = 0; j < 4; ++j) hi[4 * k + j] = __float_as_uint(e[j]);
            lo2(e[0], e[1], lo[4 * k], lo[4 * k + 1]);
            lo2(e[2], e[3], lo[4 * k + 2], lo[4 * k + 3]);
        }
        tmem_st8(a + 8 * h, hi);
        tmem_st8(a + 32 + 8 * h, lo);
    }
}

// What a compute warp's stage loop needs (see k_step2_tc).
struct CompArgs {
    unsigned char *sS, *sHi, *sLo;
    uint32_t tlane;            // tensor-memory address of lane 0 of this warp's quarter
    volatile int *abort;
    TcSync *sy;
    int rowb, nslot, S, nstage, spins, t, half, s1, s2;
};

// Tensor-memory column of accumulator buffer 0 and the distance to buffer 1
template <int NC> __device__ constexpr uint32_t acc_col0() { return 64u * tc_abuf(NC); }
template <int NC> __device__ constexpr uint32_t acc_step() { return tc_abuf(NC) == 3 ? uint32_t(NC) : 64u; }

// The stage loop of one compute thread: form A (its row's 8 points of the
// stage) and its share of B into buffer st % NA, and add the accumulators of
// stage st - (NA - 1).  With two buffers the sums of stage st - 1 are read
// after forming stage st (the MMAs of st - 1 run meanwhile); with three, the
// sums of stage st - 2 are read first, so that the MMAs of stage st (which
// overwrite that accumulator buffer, and wait only for A(st), signalled
// after the read) can start as soon as A(st) is written, and have the whole
// next stage to finish.  Returns false if a wait gave up.  B piece p
// (grid points 2p, 2p + 1) of column c goes to core matrix (K block p, rows
// 8 (c / 8) ..), row c % 8; this thread's pieces are i = t and t + 256
// (i = p NC + c), fixed for the tile, so their offsets are computed once.
template <int NC, bool G1, bool G2, bool G3>
__device__ __forceinline__ bool compute_loop(const CompArgs &ca, float (&acc)[NC / 2])
{
    constexpr int NH = NC / 2;
    constexpr int NB = NC / 8;
    constexpr int BB = NC * kTX * 8;
    constexpr int NP = (NC * 8 + kCompute - 1) / kCompute;    // B pieces per thread (at most 2)
    constexpr int NA = tc_abuf(NC), LAG = NA - 1;
    constexpr bool READ_FIRST = NA == 3;
    TcSync *sy = ca.sy;
    int src[NP], dst[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const int i = ca.t + k * kCompute;
        const int c = i % NC, p = i / NC;
        src[k] = i < NC * 8 ? (ca.nslot + c) * kSlotBytes + p * 16 : -1;
        dst[k] = (p * NB + c / 8) * 128 + (c % 8) * 16;
    }
    const int uoff = ca.s1 * kSlotBytes, voff = ca.s2 * kSlotBytes;
#pragma unroll
    for (int c = 0; c < NH; ++c) acc[c] = 0.f;
    int q = 0;                                   // ring buffer of stage st: (st / 2) % S
    uint32_t ph = 0;                             // its phase: (st / 2S) & 1
    const unsigned char *sq = ca.sS;             // ring buffer q
    int ia = 0;                                  // A / B buffer of stage st: st % NA
    // A and B of stage st (half st & 1 of ring buffer q) into buffer ia
    // (last read by the MMAs of stage st - NA, complete: their sums have
    // been read); the ring buffer is waited for at its first stage and left
    // after its second (or the last stage); the MMA warp releases it
    auto form = [&](int st) -> bool {
        const int h = (st & 1) * (kTX * 8);
        if (h == 0 && !mbar_wait_abort(&sy->full[q], ph, ca.abort, ca.spins)) return false;
        form_a<G1, G2, G3>(sq + uoff + h, sq + voff + h, ca.tlane + 64 * ia, ca.half);
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            if (src[k] < 0) continue;
            const float4 v = *reinterpret_cast<const float4 *>(sq + src[k] + h);
            const int o = ia * BB + dst[k];
            *reinterpret_cast<float4 *>(ca.sHi + o) = v;
            uint4 l;
            lo2(v.x, v.y, l.x, l.y);
            lo2(v.z, v.w, l.z, l.w);
            *reinterpret_cast<uint4 *>(ca.sLo + o) = l;
        }
        if (h != 0 || st + 1 == ca.nstage) {
            if (++q == ca.S) {
                q = 0;
                ph ^= 1u;
                sq = ca.sS;
            } else {
                sq += ca.rowb;
            }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        mbar_arrive(&sy->aready[ia]);
        if (++ia == NA) ia = 0;
        return true;
    };
    // the accumulators of stage s (buffer s & 1)
    auto read = [&](int s) -> bool {
        const int b = s & 1;
        if (!mbar_wait_abort(&sy->mdone[b], uint32_t(s >> 1) & 1, ca.abort, ca.spins)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // (ordered before this thread's next signal of A, which the MMAs that
        // overwrite buffer b wait for, by the fence that precedes it)
        add_accumulator<NH>(ca.tlane + acc_col0<NC>() + acc_step<NC>() * b + NH * ca.half, acc);
        return true;
    };
    for (int st = 0; st < ca.nstage + LAG; ++st) {
        if (READ_FIRST && st >= LAG && !read(st - LAG)) return false;
        if (st < ca.nstage && !form(st)) return false;
        if (!READ_FIRST && st >= LAG && !read(st - LAG)) return false;
    }
    return true;
}

// Two blocks per SM (sharing its 227 KB of shared memory and 512
// tensor-memory columns) hold 22 warps, 6 on some of the SM's four
// schedulers, whose register files are 16384 each: at most 80 registers a
// thread (an 88-register build ran one block per SM and was 45% slower).
template <int NC>
__global__ void __launch_bounds__(kThreads, 2)
k_step2_tc(TcArgs args, int64_t unit0, const float2 *__restrict__ dstore)
{
    constexpr int NB = NC / 8;                   // 8-row groups of B
    constexpr uint32_t LBO = NB * 128;           // next core matrix along K
    constexpr uint32_t SBO = 128;                // next 8 rows of B
    constexpr int BB = NC * kTX * 8;             // bytes of one stage of B
    constexpr int NA = tc_abuf(NC);              // A / B buffers
    constexpr uint32_t ID = idesc_tf32<NC>();
    extern __shared__ __align__(1024) unsigned char smem[];

    const TcUnit U = args.units[unit0 + blockIdx.x];
    const TcTile T = args.tiles[U.tile];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    // field blockIdx.y of a batch: its D store and partial sums
    dstore = reinterpret_cast<const float2 *>(reinterpret_cast<const char *>(dstore) + int64_t(blockIdx.y) * args.fs);
    args.partials = reinterpret_cast<double *>(reinterpret_cast<char *>(args.partials) + int64_t(blockIdx.y) * args.fs);
    args.status = reinterpret_cast<int *>(reinterpret_cast<char *>(args.status) + int64_t(blockIdx.y) * args.fs);
    const int spins = args.wait_spins;
    const int nslot = T.nslot, nf = nslot + NC;
    const int S = tc_ring(NC, nslot);            // ring buffers (>= 2; the plan checked)
    const int rowb = (nf + 1) * kSlotBytes;      // one ring buffer: nf fields and a zero row
    // shared memory: B high and low parts [NA][BB] each (canonical layout),
    // field offsets [nf], barriers, ring [S][nf + 1][kSlotBytes] (two stages of D1 / D2
    // slots, the B window, a zero row)
    unsigned char *sHi = smem;
    unsigned char *sLo = smem + NA * BB;
    int64_t *offs = reinterpret_cast<int64_t *>(smem + 2 * NA * BB);
    TcSync *sy = reinterpret_cast<TcSync *>(smem + 2 * NA * BB + 8 * size_t(nf));
    unsigned char *sS = smem + tc_fixed_smem(NC, nslot);

    for (int f = t; f < nf; f += kThreads) {
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
        for (int q = 0; q < S; ++q) {
            mbar_init(&sy->full[q], 64);
            mbar_init(&sy->empty[q], 1);
        }
        for (int b = 0; b < NA; ++b) mbar_init(&sy->aready[b], kCompute);
        for (int b = 0; b < 2; ++b) mbar_init(&sy->mdone[b], 1);
        mbar_init(&sy->drain, 1);
        sy->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(su32(&sy->tmem)), "n"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    __syncthreads();
    // fields that are not stored (past the last ring), and the zero row, read as zero
    for (int i = t; i < S * (nf + 1) * 16; i += kThreads) {
        const int q = i / ((nf + 1) * 16), rem = i - q * (nf + 1) * 16, f = rem >> 4, p = rem & 15;
        if (f < nf && offs[f] >= 0) continue;
        *reinterpret_cast<float4 *>(sS + q * rowb + f * kSlotBytes + p * 16) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = sy->tmem;
    volatile int *abort = &sy->abort;

    const int64_t M2 = int64_t(T.M) * T.M;
    const int64_t x0 = int64_t(U.chunk) * args.x_chunk;
    const int64_t x1 = min(M2, x0 + args.x_chunk);
    const int nstage = int((x1 - x0) / kTX);
    bool ok = true;

    if (warp >= 9) {
        // producers: lane l of the 64 copies piece p = l % 8 (grid points
        // 2p, 2p + 1) of fields l / 8, l / 8 + 8, ...; their offsets (in
        // 16-element units: every stored field starts at a multiple of 16)
        // are held in registers
        const int pl = t - 288, p = pl & 7, f0 = pl >> 3;
        // (all kProdFields copies are issued under a predicate: a loop
        // bound by the fields that exist was 6% slower)
        uint32_t o16[kProdFields];
#pragma unroll
        for (int k = 0; k < kProdFields; ++k) {
            const int f = f0 + 8 * k;
            const int64_t o = f < nf ? offs[f] : -1;
            o16[k] = o < 0 ? 0xFFFFFFFFu : uint32_t(o >> 4);
        }
        // A ring buffer holds two stages (32 grid points): the lane copies
        // piece p of each stage; the last buffer of an odd stage count holds
        // one
        int q = 0;                                   // ring buffer sb % S
        uint32_t ph = 0;                             // its phase: (sb / S) & 1
        const int nbuf = (nstage + 1) / 2;
        for (int sb = 0; sb < nbuf && ok; ++sb) {
            if (sb >= S) ok = mbar_wait_abort(&sy->empty[q], ph ^ 1u, abort, spins);
            if (!ok) break;
            const float2 *src = dstore + x0 + int64_t(sb) * (2 * kTX) + 2 * p;
            const uint32_t dst = su32(sS + q * rowb + f0 * kSlotBytes + p * 16);
            if (2 * sb + 1 < nstage) {
#pragma unroll
                for (int k = 0; k < kProdFields; ++k)
                    if (o16[k] != 0xFFFFFFFFu) {
                        cp_async16(dst + 8 * k * kSlotBytes, src + (int64_t(o16[k]) << 4));
                        cp_async16(dst + 8 * k * kSlotBytes + kTX * 8, src + (int64_t(o16[k]) << 4) + kTX);
                    }
            } else {
#pragma unroll
                for (int k = 0; k < kProdFields; ++k)
                    if (o16[k] != 0xFFFFFFFFu) cp_async16(dst + 8 * k * kSlotBytes, src + (int64_t(o16[k]) << 4));
            }
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(su32(&sy->full[q])) : "memory");
            if (++q == S) { q = 0; ph ^= 1u; }
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    } else if (warp == 8) {
        // MMA issue: high A x high B, low A x high B and high A x low B over
        // the four k-steps of the stage.  The whole warp runs the loop (all
        // lanes wait, one elected lane issues), so that its operands are
        // warp-uniform; a lane's wait that gives up stops the warp.
        {
            const uint64_t dh = smem_desc(su32(sHi), LBO, SBO), dl = smem_desc(su32(sLo), LBO, SBO);
            int ia = 0;                                         // A / B buffer of stage st
            uint32_t pa = 0;                                    // its phase: (st / NA) & 1
            int qr = 0;                                         // ring buffer of stage st
            for (int st = 0; st < nstage && ok; ++st) {
                const int b = st & 1;                           // accumulator buffer
                ok = mbar_wait_abort(&sy->aready[ia], pa, abort, spins);
                ok = __all_sync(0xFFFFFFFFu, ok);
                if (!ok) break;
                // A(st) signalled by every compute thread: at the last stage
                // of a ring buffer, all its reads are done (the MMAs do not
                // read the ring)
                if ((st & 1) || st + 1 == nstage) {
                    if (lane == 0) mbar_arrive(&sy->empty[qr]);
                    if (++qr == S) qr = 0;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t a = tmem + 64 * ia;
                const uint32_t d = tmem + acc_col0<NC>() + acc_step<NC>() * b;
                const uint64_t bo = uint64_t(ia * BB) >> 4;     // start-address field offset of buffer ia
                if (++ia == NA) { ia = 0; pa ^= 1u; }
                constexpr uint64_t kstep = (2 * LBO) >> 4;      // next k-step (two core matrices along K)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_tf32(d, a + 8 * j, dh + bo + j * kstep, ID, j > 0);
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_tf32(d, a + 32 + 8 * j, dh + bo + j * kstep, ID, 1);
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_tf32(d, a + 8 * j, dl + bo + j * kstep, ID, 1);
                mma_commit(su32(&sy->mdone[b]));
            }
            // the MMAs issued so far finish before the tensor memory is freed
            mma_commit(su32(&sy->drain));
            mbar_wait_bounded(&sy->drain, 0);
        }
        __syncwarp();
    } else {
        // compute warps: the thread owns tensor-memory lane (row) 32 (warp % 4)
        // + lane; rows past the tile's end read the zero row.  The loop is
        // instantiated per sign pattern (uniform over the tile; n1 >= 0)
        const int quarter = warp & 3, half = warp >> 2;
        const int row = quarter * 32 + lane;
        const bool live = row < T.nrow;
        TcRow R{};
        if (live) R = args.rows[T.row0 + row];
        CompArgs ca{sS, sHi, sLo, tmem + (uint32_t(quarter * 32) << 16), abort, sy, rowb, nslot, S, nstage, spins,
                    t, half, live ? int(R.s1) : nf, live ? int(R.s2) : nf};
        float acc[NC / 2];
        switch (T.flags) {
        case 0: ok = compute_loop<NC, false, false, false>(ca, acc); break;
        case 2: ok = compute_loop<NC, false, true, false>(ca, acc); break;
        case 4: ok = compute_loop<NC, false, false, true>(ca, acc); break;
        default: ok = compute_loop<NC, false, true, true>(ca, acc); break;
        }
        if (live) {
            double *dst = args.partials + R.p0 + int64_t(U.chunk) * R.stride;
            const double nan = __longlong_as_double(0x7FF8000000000000LL);
            constexpr int NH = NC / 2;
#pragma unroll
            for (int c = 0; c < NH; ++c) {
                const int j = c + NH * half - int(R.col0);
                if (j >= 0 && j < int(R.n)) dst[j] = ok ? double(acc[c]) : nan;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (t == 0 && *abort) atomicExch(args.status, 1);
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(kTmemCols) : "memory");
    }
}

template <int NC>
cudaError_t launch_class(const TcArgs &a, const float2 *dstore, int64_t u0, int64_t n, int nf, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_step2_tc<NC><<<dim3(unsigned(n), unsigned(nf)), kThreads, kTcSmem, s>>>(a, u0, dstore);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step2_tc(const TcArgs &a, const float2 *dstore, const int64_t *lo, const int64_t *hi, int nf,
                            cudaStream_t s)
{
    cudaError_t e = launch_class<16>(a, dstore, lo[0], hi[0] - lo[0], nf, s);
    if (e == cudaSuccess) e = launch_class<32>(a, dstore, lo[1], hi[1] - lo[1], nf, s);
    if (e == cudaSuccess) e = launch_class<48>(a, dstore, lo[2], hi[2] - lo[2], nf, s);
    if (e == cudaSuccess) e = launch_class<64>(a, dstore, lo[3], hi[3] - lo[3], nf, s);
    return e;
}

cudaError_t init_step2_tc_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k_step2_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTcSmem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTcSmem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2_tc<48>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTcSmem));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step2_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kTcSmem));
    return e;
}

}  // namespace bisp
