// kernels.cuh -- device kernels of the bispectrum-multipole estimator and
// their launch helpers.  Internal to libbisp.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "plan.hpp"

namespace bisp {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

// Ring table as a kernel argument (membership by the integer test of
// build_rings).
struct RingArg {
    int nr;
    int64_t e3sq[kMaxRings + 1];   // (3 e_r)^2
    int maxc[kMaxRings];
};

// Twiddle tables of the transforms: tw2[k] = exp(-2 pi i k / 2^lg2) for
// lengths 2^q <= 2^lg2, tw3[k] = exp(-2 pi i k / (3 x 2^lg3)) for lengths
// 3 x 2^q <= 3 x 2^lg3, and likewise tw5 and tw7 for lengths 5 x 2^q and
// 7 x 2^q (tw3, tw5, tw7 may be null when no such length is used).
template <typename C> struct Twiddles {
    const C *tw2;
    const C *tw3;
    int lg2, lg3;
    const C *tw5;
    int lg5;
    const C *tw7;
    int lg7;
};

// Side lengths of the plan's reduction grids, by level index.
struct GridArg {
    int M[kMaxLevels];
};

// Fields of a batched launch: gridDim.y = nf; field f reads its input fs_in
// bytes and writes its output fs_out bytes past field f - 1's (kernels whose
// buffers all lie in one per-field workspace region use fs_in for both).
struct Batch {
    unsigned nf = 1;
    int64_t fs_in = 0, fs_out = 0;
};

// Step-I job: one (plane, ring) field on one reduction grid.
struct Job {
    int32_t n, r;
    int64_t out_off;   // complex elements into the destination store
};

struct StepIIArgs {
    const Group *groups;
    const Tile *tiles;
    const Unit *units;
    const int64_t *doff;     // [kMaxLevels][nz+1][kMaxRings]
    int nz1;                 // planes stored: 0 .. nz1 - 1
    int nr;                  // rings per plane
    int64_t x_chunk;         // grid points of one unit
    double *partials;
    int64_t fs;              // bytes between the workspace regions of the fields of a batch
};

// --- launch helpers (kernels.cu); all return cudaGetLastError() --------------

// z pass of the forward 3D transform: real rows of length ng -> kept
// frequencies [0, nkeep) written transposed as out[k][row].
template <typename R>
cudaError_t launch_fft_z_real(const R *in, typename Cx<R>::T *out, int ng, int64_t rows, int nkeep,
                              const Twiddles<typename Cx<R>::T> &tw, const Batch &fb, cudaStream_t s, int rt = 0);

// Batched row transforms written transposed: in[b][nrow][M] -> out[b][M][nrow]
// (out at out_off[b] when out_off is not null, else b * M * nrow), times
// scale; zero_dc clears element [0][0] of batch 0.
template <typename R>
cudaError_t launch_fft_rows_T(const typename Cx<R>::T *in, typename Cx<R>::T *out, int M, int nrow,
                              int64_t nb, const int64_t *out_off, R scale, bool zero_dc,
                              const Twiddles<typename Cx<R>::T> &tw, const Batch &fb, cudaStream_t s,
                              int rt = 0);

// Step I, first pass: ring r of plane n of Delta (planes [nz+1][ng][ng]),
// folded onto the M x M grid, transformed along u_y, written in place order
// to gt[job][u_x][k_y].  unit = true uses Delta = 1 (the unit fields of
// Eq. 2FT).
template <typename R>
cudaError_t launch_ring_gather(const typename Cx<R>::T *planes, int ng, const RingArg &rings,
                               const Job *jobs, int64_t njobs, int M, bool unit,
                               typename Cx<R>::T *gt, const Twiddles<typename Cx<R>::T> &tw,
                               const Batch &fb, cudaStream_t s, int rt = 0);

// Step I second pass: for each of njobs M x M fields in gt ([u_x][k_y],
// the gather's output), transforms along u_x in strips of w columns and
// writes the field [k_x][k_y] at out + out_off[job].  Rows that hold no
// member of the job's ring (jobs[job].r, its largest |u_x| in rings) are
// taken as zero without being read (the gather does not write them).
template <typename R>
cudaError_t launch_fft_cols(const typename Cx<R>::T *in, typename Cx<R>::T *out, int M, int64_t njobs,
                            const int64_t *out_off, const Job *jobs, const RingArg &rings,
                            const Twiddles<typename Cx<R>::T> &tw, const Batch &fb, cudaStream_t s, int w = 0);

// Step II: partial triple sums of units, one block per unit, one launch per
// block class (units [lo[c], hi[c]) run in blocks of 2^c warps with
// kStep2ClassSmem[c] bytes of shared memory; a whole estimate passes
// lo = class_begin, hi = class_begin + 1).
template <typename R>
cudaError_t launch_step2(const StepIIArgs &a, const typename Cx<R>::T *dstore, const int64_t *lo, const int64_t *hi,
                         int nf, cudaStream_t s);

// Step II on tcgen05 (FP32 fields; step2_tc.cu).
struct TcArgs {
    const TcTile *tiles;
    const TcRow *rows;
    const int32_t *slots;
    const TcUnit *units;
    const int64_t *doff;     // [kMaxLevels][nz+1][kMaxRings]
    int nz1, nr;
    int64_t x_chunk;
    double *partials;
    int *status;             // field 0's status word, set to 1 by a block whose wait ran out
    int64_t fs;              // bytes between the workspace regions of the fields of a batch
    int wait_spins;          // polls before an abortable wait gives up
};

// Polls of an mbarrier before a tensor-core Step-II wait gives up (the plan's
// default; estimator_set_wait_limit lowers it to test the give-up path).
constexpr int kDefaultWaitSpins = 1 << 22;

// Device address of estimator_estimate_static's scratch array on the current
// device (noalloc.cu), and the device a plan lives on (abi.cu).
int static_scratch_address(void **out);
int plan_device(const bisp_plan *p);

// One launch per column class: units [lo[c], hi[c]), one block per unit
// with kTcSmem bytes of shared memory.
cudaError_t launch_step2_tc(const TcArgs &a, const float2 *dstore, const int64_t *lo, const int64_t *hi, int nf,
                            cudaStream_t s);

// Allow the kernels their dynamic shared memory once (kernels.cu and
// step2_tc.cu), so that estimates are plain stream work.
cudaError_t init_kernel_attributes();
cudaError_t init_step2_tc_attributes();

// S[c0 + j] = (ng/M)^2 sum_k partials[part0 + k ncombo + j]
template <typename A>
cudaError_t launch_reduce_partials(const Group *groups, int64_t ngroups, const double *partials,
                                   int ng, double *S, const Batch &fb, cudaStream_t s);

// Binning epilogue of Eq. bs_lm2_1 for the moments of even l_lo .. l_hi
// (out and den: [nbins][moments of those l]).  mode 0: B = sqrt((2l+1)/4pi)
// num / (V N_g^2 den) from S and den; mode 1: den from the triangle counts.
// fp32_weights: the Y_lm of each record in FP32 (sums stay in W).
// The records are walked in chunks of one bin each (one warp per chunk, FP64
// partial sums per moment in `partial` [nchunks][moments of l <= l_hi]),
// then each bin adds its chunks in order (one thread per bin).
struct EpiArgs {
    const Record *rec;
    const int64_t *chunk_lo, *chunk_hi;   // record range of each chunk
    int64_t nchunks;
    const int64_t *bin_chunk;             // [nbins + 1]: first chunk of each bin
    int64_t nbins;
    double *partial;                      // field 0's partial sums
    int64_t fs_part;                      // bytes between the fields' partial sums
};
template <typename W>
cudaError_t launch_epilogue(int mode, const EpiArgs &e, const double *value, int l_lo, int l_hi, const double *den,
                            double norm, double *out, const Batch &fb, cudaStream_t s, bool fp32_weights = false);

// Y_lm normalisations nlm[l][m] and the prefactors sqrt((2l+1)/(4 pi)).
cudaError_t set_ylm_constants(const double nlm[9][9], const double pref[9], cudaStream_t s);

// Welford update of per-element count, mean and squared deviations with
// nf fields B[f][0 .. n-1] (non-finite values skipped).
cudaError_t launch_stats_update(const double *B, int nf, int64_t n, int64_t *count, double *mean, double *m2,
                                cudaStream_t s);

// N_tri of unordered ring triples from the unit fields (Eq. Ntri2), FP64.
// triples[4 t .. 4 t + 3] = (r1, r2, r3, level index into grids.M).
cudaError_t launch_ntri(const double2 *ifields, const int64_t *ioff, const int32_t *triples,
                        int64_t ntriples, const GridArg &grids, double *raw, cudaStream_t s);

// Sizes of dynamic shared memory (bytes) of the transform kernels.
// Rows of length M a transform block holds: each of its two shared-memory
// buffers takes about `bytes` (1 .. 256 rows).  rt = 0 passed to the
// launchers above selects this with the default 16 KB; the plan's autotuner
// passes its own choice.
size_t fft_rows_per_block(int M, size_t elem, size_t bytes = 16384);
// Elements of one row of a transform's shared-memory buffers: M values with
// a padding slot after every 8, and one more so that consecutive rows start
// in different banks.
inline __host__ __device__ constexpr int fft_stride(int M) { return M + (M >> 3) + 1; }

}  // namespace bisp
