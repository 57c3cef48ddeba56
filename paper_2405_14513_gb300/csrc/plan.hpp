// plan.hpp -- host-side plan of the bispectrum-multipole estimator: ring
// table, combination enumeration, work decomposition and table layouts.
// Internal to libbisp; the public interface is include/bisp.h.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "bisp.h"

#if defined(__CUDACC__)
#define BISP_HD __host__ __device__
#else
#define BISP_HD
#endif

namespace bisp {

constexpr int kMaxRings = 64;     // N_r for N_g <= 1024 is 52
constexpr int kMaxLevels = 32;    // reduction grids: 2^k, 3, 5, 7 x 2^k from 8 to N_g (27 at 1024)
constexpr int kTileRows = 8;      // rows (r1, r2) of a Step-II register tile
constexpr int kTileCols = 8;      // consecutive r3 of a Step-II register tile

// Ring table (Sec. II, implementation paragraph): ring r holds the modes
// u = (i, j) with e_{r} <= |u| < e_{r+1}; e_0 = 0, widths 2^floor(r/10)
// (0-based r), the outer edge capped at N_g/3.  Edges are kept as 3 e_r,
// exact integers, so membership is the integer test
// (3 e_r)^2 <= 9 |u|^2 < (3 e_{r+1})^2.
struct Rings {
    int ng = 0, nr = 0, nz = 0;        // nz = floor(N_g/3): planes 0..nz
    int64_t e3[kMaxRings + 1] = {};
    double kperp[kMaxRings] = {};      // mode-averaged |u|, grid units
    int64_t count[kMaxRings] = {};
    int maxc[kMaxRings] = {};          // largest |u_x| of a member (= largest |u_y|)
    int ngrid = 0;                     // reduction grids, ascending: M = F x 2^k (F = 1, 3, 5, 7),
    int grid[kMaxLevels] = {};         // 8 <= M <= N_g
};

// Plane pair (n1, n2, n3 = -n1 - n2) on one reduction grid M: the set of
// ring triples whose triple sum runs on the M x M grid.  Its combinations
// are ordered by (r1, r2, r3).
struct Group {
    int32_t n1, n2, n3;        // signed planes
    int32_t lev;               // reduction grid index (Rings::grid)
    int32_t M;                 // reduction grid side
    int32_t row0, nrow;        // rows of this group
    int32_t ncombo;
    int64_t c0;                // index of the first combination (S order)
    int32_t nchunk;            // x chunks of the M^2 grid
    int32_t self_conj;         // 1 for n1 = n2 = 0 (counted once), else 0
    int64_t part0;             // partial sums [nchunk][ncombo] start here
};

// A run of consecutive r3 (r3a .. r3a + n - 1) accepted for (r1, r2): the
// combinations coff .. coff + n - 1 of its group.
struct Row {
    uint8_t r1, r2, r3a, n;
    int32_t coff;
};

// Step-II register tile: up to 8 rows (r1, r2) of one group times 8
// consecutive r3 (the window w0 .. w0 + 7).  Slots index the rings staged
// by the tile's unit in shared memory.
struct Tile {
    uint8_t s1[kTileRows];     // slot of D(r1, n1) of each row
    uint8_t s2[kTileRows];     // slot of D(r2, n2) of each row
    uint8_t s3;                // slot of D(w0, n3); the window is s3 .. s3 + 7
    uint8_t pad[3];
    uint32_t mask[2];          // bit 8 i + j: (row i, r3 = w0 + j) is a combination
    int32_t coff[kTileRows];   // combination (in the group) of (row i, w0); (i, j) -> coff[i] + j
    int32_t pad2;
};
static_assert(sizeof(Tile) == 64, "Tile is copied in 16-byte pieces");

// Tensor-core (tcgen05) Step II.  A tile is up to 128 rows (r1, r2) taken
// from groups that share the reduction grid and |n3|, times a window of NC
// consecutive r3 (r3lo .. r3lo + NC - 1) of plane |n3|; NC = 16, 32, 48 or
// 64.  The pair products D1 D2 of the rows form the MMA's A operand (one row
// per tensor-memory lane), the window's stored D3 fields its B operand.
constexpr int kTcRows = 128;
constexpr int kTcMaxCols = 64;
constexpr int kTcMaxSlots = 250;      // distinct D1 / D2 fields staged by a tile
constexpr int kTcClasses = 4;         // NC = 16 (class + 1)
constexpr int kTcTX = 16;             // grid points of one pipeline stage (one MMA step)
constexpr int kTcRingTX = 2 * kTcTX;  // grid points of one ring buffer (two stages)
constexpr int kTcSlotBytes = kTcRingTX * 8 + 16;   // one staged field row of a ring buffer (padded)
constexpr int kTcMinRing = 2;         // ring buffers
constexpr int kTcMaxRing = 4;
constexpr size_t kTcSmem = 110 * 1024;         // dynamic shared memory of a block (two per SM)
// Buffers of a stage's A and B operands: three for NC <= 32 (3 x 64 columns
// of A and two accumulators of NC columns fit the 256 tensor-memory columns
// of a block), two otherwise.
BISP_HD constexpr int tc_abuf(int ncol) { return ncol <= 32 ? 3 : 2; }
// Shared memory of a tcgen05 block other than its stage ring: B high and
// low parts (tc_abuf buffers each), field offsets, barriers; a multiple of
// 128 bytes, so that the ring that follows is aligned for 16-byte copies.
BISP_HD inline size_t tc_fixed_smem(int ncol, int nslot)
{
    return size_t(2 * tc_abuf(ncol)) * ncol * kTcTX * 8 + ((8 * size_t(nslot + ncol) + 256 + 127) & ~size_t(127));
}
// Buffers of the stage ring for a tile (0 if fewer than kTcMinRing fit):
// each holds two stages of the tile's nslot + ncol fields and one zero row.
BISP_HD inline int tc_ring(int ncol, int nslot)
{
    const size_t fixed = tc_fixed_smem(ncol, nslot);
    if (fixed >= kTcSmem) return 0;
    const size_t per = size_t(nslot + ncol + 1) * kTcSlotBytes;
    const int n = int((kTcSmem - fixed) / per);
    return n < kTcMinRing ? 0 : (n > kTcMaxRing ? kTcMaxRing : n);
}
struct TcRow {
    int64_t p0;                // partial sum of (x chunk 0, first combination of the run)
    int32_t stride;            // partial sums of one x chunk of the row's group (its ncombo)
    uint8_t s1, s2;            // staged slots of D(r1, |n1|) and D(r2, |n2|)
    uint8_t col0, n;           // combinations r3 = r3lo + col0 .. r3lo + col0 + n - 1
    uint8_t flags;             // bit 0: n1 < 0, bit 1: n2 < 0, bit 2: n3 < 0 (conjugated fields)
    uint8_t pad[7];
};
static_assert(sizeof(TcRow) == 24, "TcRow layout");
struct TcTile {
    int32_t lev, M;            // reduction grid
    int32_t row0, nrow;        // rows in tc_rows
    int32_t slot0, nslot;      // staged D1 / D2 fields in tc_slots: (plane << 8) | ring
    int32_t n3abs, r3lo;       // B window: rings r3lo .. r3lo + ncol - 1 of plane |n3|
    int32_t ncol, nchunk;      // NC; x chunks of the M^2 grid
    int32_t flags;             // the rows' flags (all rows of a tile share them)
    int32_t pad;
};
struct TcUnit {
    int32_t tile, chunk;
};

// One Step-II block: an x chunk of a group with up to 16 of its tiles (one
// per warp), and the ring ranges it stages per plane (plane 3 may reach
// past the last ring; those slots are zero).  cls: log2 of the warps of the
// block class it runs in (2, 3 or 4).
struct Unit {
    int32_t group, chunk;
    int32_t t0, nt;
    int16_t rlo[3], rhi[3];
    int32_t cls;
};

// Shared-memory bytes of a Step-II block staging ns rings, two stages of tx
// grid points of celem-byte values.
inline size_t step2_smem_need(int ns, int tx, size_t celem)
{
    return ((size_t(ns) * sizeof(int64_t) + 127) & ~size_t(127)) + 2 * size_t(ns) * size_t(tx) * celem;
}

// Dynamic shared memory of a block of each class (2, 3, 4 = 4, 8, 16 warps):
// 1, 2 or 4 blocks share the 227 KB of an SM.
constexpr size_t kStep2ClassSmem[5] = {0, 0, 55 * 1024, 111 * 1024, 222 * 1024};

// Per-combination data of the binning epilogue, in (k1, mu, t)-bin order.
struct Record {
    int32_t s_index;           // index into the S array (S order)
    int32_t flags;             // bit 0: counted once (self-conjugate pair);
                               // bit 1: linear triangle (azimuth averaged)
    double pz;                 // cos(theta) of p (Eq. orient)
    double cphi;               // cos(phi) of p
};

// A binning of the combinations (Eq. bs_lm2_1): the moments of even l
// l_lo .. l_hi on an n_mu x n_t grid of (mu, t) bins; one field's output
// block [n_k1][n_mu][n_t][n_lm] starts at out_off doubles, its records in
// (k1, mu, t)-bin order at rec_off of the plan's record array, its
// bin_start at bs_off of the plan's bin_start array (absolute record
// indices).  One view (every l on the caller's n_mu x n_t) unless per-l
// bins are asked for; then consecutive l with the same grid share a view.
// The binning runs over chunks of at most kBinChunk records of one bin (a
// bin's records cut in order), chunk_off .. chunk_off + n_chunks - 1 of the
// plan's chunk arrays, and bin b's chunks are bin_chunk[bc_off + b] ..
// bin_chunk[bc_off + b + 1] - 1.
struct View {
    int l_lo = 0, l_hi = 0, n_mu = 1, n_t = 1;
    int lm_lo = 0, n_lm = 1;           // first moment index (l_lo/2)^2, moments in the view
    int64_t n_bins = 0, out_off = 0, rec_off = 0, bs_off = 0;
    int64_t chunk_off = 0, n_chunks = 0, bc_off = 0;
};
constexpr int64_t kBinChunk = 2048;

struct Level {
    int lev = 0;               // index into Rings::grid
    int M = 0;                 // grid side
    int64_t njobs = 0;         // stored (plane, ring) fields on this grid
    int64_t dstore_off = 0;    // first element of this grid in the D store
};

// Everything the host knows about a plan.
struct HostPlan {
    bisp_desc desc{};
    std::vector<double> k1_edges;
    Rings rings;
    int n_lm = 0;
    int64_t n_bins = 0;
    double kf = 0, volume = 0;

    // triangle counts N_tri[r1][r2][r3]
    std::vector<int64_t> ntri;

    // combinations in S order
    std::vector<Group> groups;
    std::vector<Row> rows;
    std::vector<Tile> tiles;            // FP64 path: 8 x 8 register tiles
    bool tensor = false;                // build tcgen05 tiles (set before enumerate)
    std::vector<TcTile> tc_tiles;
    std::vector<TcRow> tc_rows;
    std::vector<int32_t> tc_slots;
    std::vector<TcUnit> tc_units;       // by class (NC), then grid, x chunk, tile
    int64_t tc_class_begin[kTcClasses + 1] = {};
    double tc_mma_products = 0;         // sum over tiles of 128 NC M^2 (lane-column-points)
    std::vector<Unit> units;            // Step-II blocks in launch order
    int max_slots = 0;                  // largest staged ring count of a unit
    int max_cls = 4;                    // largest block class (set before enumerate)
    size_t celem = 8;                   // bytes of a staged complex value (set before enumerate)
    int64_t class_begin[6] = {};        // units of class c: [class_begin[c], class_begin[c+1])
    std::vector<double> unit_cost;      // prefix sums of the Step-II units' costs, launch order (n + 1)
    int64_t n_combos = 0;
    int64_t n_partials = 0;
    int64_t n_pairs = 0;
    double triple_products = 0;          // sum over combinations of M^2 (M: its smallest exact grid)
    double pair_products = 0;            // sum over distinct (pair, r1, r2, smallest grid) of M^2
    std::vector<int32_t> combo_bin;      // S order
    std::vector<Record> records_s;      // S order (moved to bin order later)
    std::vector<double> ntri_s;         // N_tri per combination, S order

    // binnings: records of every view in its own bin order, one after another
    std::vector<View> views;
    int64_t n_out = 0;                  // doubles of one field's output (all views)
    std::vector<Record> records;
    std::vector<double> rec_ntri;
    std::vector<int64_t> bin_start;     // per view: n_bins + 1 absolute record indices
    std::vector<int64_t> chunk_lo, chunk_hi;   // record ranges of the binning chunks (all views)
    std::vector<int64_t> bin_chunk;     // per view: n_bins + 1 chunk indices (relative to chunk_off)
    int64_t max_chunks = 0;             // largest n_chunks of a view

    // D store: offset (in complex elements) of field (level, plane, ring),
    // -1 where not stored; [kMaxLevels][nz+1][kMaxRings]
    std::vector<int64_t> doff;
    std::vector<Level> levels;          // levels in use
    int64_t dstore_elems = 0;
    int64_t gt_elems = 0;               // largest per-level Step-I scratch
};

// N_g = 2^k or 3 x 2^k in [8, 1024] (the transform lengths the kernels handle).
bool grid_size_supported(int ng);

// Build the ring table; returns false for an unsupported N_g.
bool build_rings(int ng, Rings &R);

// Reduction grid of a ring triple: the index of the smallest grid M with
// M > maxc1 + maxc2 + maxc3 (the largest, N_g, if none).  On that grid no
// non-zero sum u + v + w of members aliases to zero, so the triple sum over
// the M x M grid is exactly (M/N_g)^2 times the sum on the N_g x N_g grid.
int triple_level(const Rings &R, int r1, int r2, int r3);

// Enumerate the accepted combinations of one half of the plane pairs and
// fill groups, rows, tiles, units, records and the D-store layout.
// Requires rings and ntri.  Returns "" or an error message.
std::string enumerate(HostPlan &P, int64_t x_chunk);

// Views of the plan (from desc n_mu, n_t, or the per-l grids n_mu_l, n_t_l
// for l = 0, 2, .., l_max), their output offsets and n_out.
void build_views(HostPlan &P, const int *n_mu_l, const int *n_t_l);

// Counting sort of the records by (k1, mu, t) bin, once per view.
// Shape of a triangle with squared sides q1 >= q2 >= q3 > 0 (grid units)
// and its (k1, mu, t) bin (Eq. shape; Sec. II, second-level binning): side
// lengths a_i = sqrt(q_i); accepted when K1 = kf a1 lies in a k1 bin and
// t = a2/a1 >= 1/2.  mu = -k1^.k2^ is the cosine of the triangle's angle
// between k1 and -k2 (opposite side 3), from the half-angle form of the
// cosine law, 1 - mu = 2 sin^2(gamma/2) = (a3 - a1 + a2)(a3 + a1 - a2) /
// (2 a1 a2), clamped to [1/2, 1] (where it lies for a1 >= a2 >= a3).
struct TriShape {
    double a1, a2, h, mu, t;   // h = 1 - mu
    int ib, bin;
};
bool triangle_shape(const std::vector<double> &k1_edges, double kf, int n_mu, int n_t, double q1, double q2,
                    double q3, TriShape *s);
// bin of x among n uniform bins of [1/2, 1] (top edge closed) and the flat
// (k1, mu, t) bin on an n_mu x n_t grid
int half_unit_bin(double x, int n);
int grid_bin(int ib, double mu, double t, int n_mu, int n_t);
void sort_records(HostPlan &P);
// mu, t, p_z, cos phi of every combination, in S order: out[4 k + 0..3]
void combo_shapes(const HostPlan &P, int64_t cap, double *out);

// Step-II block classes of the plan's kernel (tcgen05: NC = 16, 32, 48, 64;
// CUDA cores: 2^c warps, c = 2, 3, 4), as ranges of its launch-ordered units.
constexpr int kClassSlots = 6;
int unit_classes(const HostPlan &P, const int64_t **class_begin);

// Fill P.unit_cost: the cost of a unit is the grid points of its x chunk
// (tcgen05: one tile per block) times its register tiles (CUDA cores).
void unit_costs(HostPlan &P, int64_t x_chunk);

// Share `part` of `nparts` of the Step-II work: for every block class k,
// the units [lo[k], hi[k]), a contiguous run of the class with about
// 1/nparts of its cost.  The shares of parts 0 .. nparts - 1 partition
// every class.
void part_ranges(const HostPlan &P, int part, int nparts, int64_t *lo, int64_t *hi);

}  // namespace bisp
