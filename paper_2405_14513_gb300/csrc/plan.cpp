// plan.cpp -- host part of the plan: ring table (Sec. II), acceptance and
// geometry of each ring/plane combination (Eqs. shape, orient), bin index,
// work decomposition of the Step-II reduction and the D-store layout.
//
// Compiled with -ffp-contract=off: every floating-point operation below is
// the IEEE operation written, so bin decisions are reproducible on any host.
#include "plan.hpp"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

namespace bisp {

bool grid_size_supported(int ng)
{
    if (ng < 8 || ng > 1024) return false;
    const int m = ng % 3 == 0 ? ng / 3 : ng;
    return (m & (m - 1)) == 0;
}

bool build_rings(int ng, Rings &R)
{
    if (!grid_size_supported(ng)) return false;
    R = Rings{};
    R.ng = ng;
    R.nz = ng / 3;
    // 3 e_r: 0, then steps of 3 * 2^floor(r/10) grid units, capped at N_g
    int r = 0;
    R.e3[0] = 0;
    while (R.e3[r] < ng) {
        if (r >= kMaxRings) return false;
        int64_t w = int64_t(3) << (r / 10);
        R.e3[r + 1] = std::min<int64_t>(R.e3[r] + w, ng);
        ++r;
    }
    R.nr = r;
    // members: mode-averaged radius (summed over i, then j, ascending) and
    // the largest |u_x|
    const int h = ng / 2;
    double sum[kMaxRings] = {};
    for (int64_t i = -h; i < h; ++i)
        for (int64_t j = -h; j < h; ++j) {
            int64_t q9 = 9 * (i * i + j * j);
            if (q9 >= R.e3[R.nr] * R.e3[R.nr]) continue;
            int q = 0;
            while (!(q9 < R.e3[q + 1] * R.e3[q + 1])) ++q;
            sum[q] += std::sqrt(double(i * i + j * j));
            R.count[q] += 1;
            R.maxc[q] = std::max<int>(R.maxc[q], int(i < 0 ? -i : i));
        }
    for (int q = 0; q < R.nr; ++q)
        R.kperp[q] = R.count[q] > 0 ? sum[q] / double(R.count[q]) : 0.5 * double(R.e3[q] + R.e3[q + 1]) / 3.0;
    // reduction grids: 2^k, 3 x 2^k, 5 x 2^k and 7 x 2^k from 8 to N_g,
    // multiples of 4 (a grid's M^2 points are a whole number of 16-point
    // stages), ascending
    R.ngrid = 0;
    for (int m = 8; m <= ng; m *= 2)
        for (int f : {2, 3, 5, 7})
            if (f * m / 2 <= ng && R.ngrid < kMaxLevels) R.grid[R.ngrid++] = f * m / 2;
    std::sort(R.grid, R.grid + R.ngrid);
    return true;
}

int triple_level(const Rings &R, int r1, int r2, int r3)
{
    const int need = R.maxc[r1] + R.maxc[r2] + R.maxc[r3] + 1;
    for (int l = 0; l < R.ngrid; ++l)
        if (R.grid[l] >= need) return l;
    return R.ngrid - 1;
}

// Bin of x among n uniform bins of [1/2, 1] with the top edge closed: the
// number of interior edges 1/2 + j/(2n), j = 1 .. n - 1, lying at or below x
// (binary search over the edges).
int half_unit_bin(double x, int n)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int j = (lo + hi + 1) / 2;
        if (0.5 + double(j) / (2.0 * double(n)) <= x) lo = j;
        else hi = j - 1;
    }
    return lo;
}

// (k1, mu, t) bin of a shape on an n_mu x n_t grid of [1/2, 1]^2
int grid_bin(int ib, double mu, double t, int n_mu, int n_t)
{
    return (ib * n_mu + half_unit_bin(mu, n_mu)) * n_t + half_unit_bin(t, n_t);
}

// k1 bin of K1: the last edge at or below K1 (the top edge belongs to the
// last bin), -1 outside the edges
static int k1_bin(const std::vector<double> &edges, double K1)
{
    const int n = int(edges.size()) - 1;
    if (!(K1 >= edges[0]) || K1 > edges[n]) return -1;
    const int b = int(std::upper_bound(edges.begin(), edges.end(), K1) - edges.begin()) - 1;
    return b < n ? b : n - 1;
}

bool triangle_shape(const std::vector<double> &k1_edges, double kf, int n_mu, int n_t, double q1, double q2,
                    double q3, TriShape *s)
{
    if (!(q3 > 0.0 && q2 >= q3 && q1 >= q2)) return false;
    const double a1 = std::sqrt(q1), a2 = std::sqrt(q2), a3 = std::sqrt(q3);
    const int ib = k1_bin(k1_edges, kf * a1);
    if (ib < 0) return false;
    const double t = a2 / a1;
    if (t < 0.5) return false;
    double h = (a3 - a1 + a2) * (a3 + a1 - a2) / (2.0 * a1 * a2);
    h = std::min(0.5, std::max(0.0, h));
    s->a1 = a1;
    s->a2 = a2;
    s->h = h;
    s->mu = 1.0 - h;
    s->t = t;
    s->ib = ib;
    s->bin = grid_bin(ib, s->mu, t, n_mu, n_t);
    return true;
}

namespace {

struct Geo {
    int bin;                   // (k1, mu, t) bin on the plan's n_mu x n_t grid
    int degenerate;
    double pz, cphi;
    int ib;                    // k1 bin
    double mu, t;              // shape (mu clamped to [1/2, 1])
};

// Acceptance and geometry of one combination (planes n1, n2, n3, ring
// radii kp1..kp3; grid units), from the triangle it describes: sides
// a_i^2 = kp_i^2 + n_i^2, shape and bin by triangle_shape.  Orientation, in
// the frame of Eq. orient (e_z along k1, k2 in the (x, z) plane with x > 0):
//   k1 = a1 e_z,  k2 = a2 (-mu e_z + s e_x),  k3 = -k1 - k2,
// s = sqrt(1 - mu^2) = sqrt(h (2 - h)) with h = 1 - mu; the line of sight p
// obeys k_i . p = n_i (the plane index is the component along the line of
// sight).  Side 1 gives p_z = n1/a1 and side 3 p_x = ((a2 mu - a1) p_z - n3)
// / (a2 s) (side 2 then holds by closure); |p| = 1 gives
// p_y = +sqrt(max(0, 1 - p_z^2 - p_x^2)), and the azimuth cos phi =
// p_x / sqrt(1 - p_z^2), within [-1, 1] (1 where p_z = +-1: there the
// azimuth is undefined and P_l^m(p_z) = 0 for m > 0).  A linear triangle
// (mu >= 1 - 1e-12) is flagged `degenerate`: its azimuth is undefined.
bool combo_geometry(const HostPlan &P, double kp1, double kp2, double kp3, int n1, int n2, int n3,
                    Geo *g)
{
    const bisp_desc &d = P.desc;
    TriShape sh;
    if (!triangle_shape(P.k1_edges, P.kf, d.n_mu, d.n_t, kp1 * kp1 + double(n1) * n1,
                        kp2 * kp2 + double(n2) * n2, kp3 * kp3 + double(n3) * n3, &sh))
        return false;
    g->ib = sh.ib;
    g->mu = sh.mu;
    g->t = sh.t;
    g->bin = sh.bin;
    g->pz = double(n1) / sh.a1;
    g->degenerate = (sh.mu >= 1.0 - 1e-12);
    g->cphi = 1.0;
    if (!g->degenerate) {
        const double sperp = std::sqrt(sh.h * (2.0 - sh.h));
        const double px = ((sh.a2 * sh.mu - sh.a1) * g->pz - double(n3)) / (sh.a2 * sperp);
        const double rho2 = 1.0 - g->pz * g->pz;
        if (rho2 > 0.0) g->cphi = std::min(1.0, std::max(-1.0, px / std::sqrt(rho2)));
    }
    return true;
}

struct Acc {            // one accepted combination of a pair
    uint8_t r1, r2, r3, lev;
    Geo g;
};

struct PairOut {
    int n1, n2;
    std::vector<Acc> acc;   // (r1, r2, r3) ascending
};

void enumerate_pair(const HostPlan &P, int n1, int n2, PairOut &out)
{
    const Rings &R = P.rings;
    const int nr = R.nr;
    const int n3 = -(n1 + n2);
    out.n1 = n1;
    out.n2 = n2;
    for (int r1 = 0; r1 < nr; ++r1) {
        double k1sq = R.kperp[r1] * R.kperp[r1] + double(n1) * n1;
        double K1 = P.kf * std::sqrt(k1sq);
        if (K1 < P.k1_edges[0] || K1 > P.k1_edges[P.desc.n_k1]) continue;
        for (int r2 = 0; r2 < nr; ++r2) {
            double k2sq = R.kperp[r2] * R.kperp[r2] + double(n2) * n2;
            if (k2sq > k1sq) break;                  // radii increase with r
            for (int r3 = 0; r3 < nr; ++r3) {
                double k3sq = R.kperp[r3] * R.kperp[r3] + double(n3) * n3;
                if (k3sq > k2sq) break;
                if (P.ntri[(size_t(r1) * nr + r2) * nr + r3] <= 0) continue;
                Geo g;
                if (!combo_geometry(P, R.kperp[r1], R.kperp[r2], R.kperp[r3], n1, n2, n3, &g)) continue;
                out.acc.push_back(Acc{uint8_t(r1), uint8_t(r2), uint8_t(r3),
                                      uint8_t(triple_level(R, r1, r2, r3)), g});
            }
        }
    }
}

// tcgen05 tiles (see TcTile): the groups of each (grid, |n3|, signs of n1,
// n2, n3) in order of n1, their rows by the centre of their r3 run, cut
// greedily into tiles of at most 128 rows and a window of at most 64 r3
// whose fields fit kTcMinRing ring buffers of shared memory; then units (tile,
// x chunk) by class.
// Requires the groups' partial-sum layout.  Marks the fields the tiles read.
template <typename UsedFn>
std::string build_tc(HostPlan &P, int64_t x_chunk, UsedFn &&U_)
{
    const Rings &R = P.rings;
    const int nz = R.nz;
    P.tc_tiles.clear();
    P.tc_rows.clear();
    P.tc_slots.clear();
    P.tc_units.clear();
    P.tc_mma_products = 0;
    auto gflags = [](const Group &G) { return (G.n1 < 0 ? 1 : 0) | (G.n2 < 0 ? 2 : 0) | (G.n3 < 0 ? 4 : 0); };
    std::vector<std::vector<int32_t>> pool(size_t(R.ngrid) * (nz + 1) * 8);
    for (size_t g = 0; g < P.groups.size(); ++g) {
        const Group &G = P.groups[g];
        pool[(size_t(G.lev) * (nz + 1) + (G.n3 < 0 ? -G.n3 : G.n3)) * 8 + gflags(G)].push_back(int32_t(g));
    }
    struct Cur {
        std::vector<std::pair<int32_t, int32_t>> rows;   // (group, row index in P.rows)
        std::vector<int32_t> slots;
        int lo = 1 << 30, hi = -1;
    } cur;
    int cur_lev = 0, cur_n3 = 0, cur_flags = 0;
    auto slot_of = [&](std::vector<int32_t> &sl, int32_t key) {
        for (size_t i = 0; i < sl.size(); ++i)
            if (sl[i] == key) return int(i);
        return -1;
    };
    auto close = [&]() -> std::string {
        if (cur.rows.empty()) return "";
        TcTile T{};
        T.lev = cur_lev;
        T.M = R.grid[cur_lev];
        T.row0 = int32_t(P.tc_rows.size());
        T.nrow = int32_t(cur.rows.size());
        T.slot0 = int32_t(P.tc_slots.size());
        T.nslot = int32_t(cur.slots.size());
        T.n3abs = cur_n3;
        T.r3lo = cur.lo;
        T.ncol = ((cur.hi - cur.lo + 1 + 15) / 16) * 16;
        const int64_t M2 = int64_t(T.M) * T.M;
        T.nchunk = int32_t((M2 + x_chunk - 1) / x_chunk);
        T.flags = cur_flags;
        if (cur_flags & 1) return "tcgen05 tiles need n1 >= 0";
        if (T.ncol > kTcMaxCols || T.nslot > kTcMaxSlots || T.nrow > kTcRows || tc_ring(T.ncol, T.nslot) == 0)
            return "tcgen05 tile limits";
        // rows (tensor-memory lanes) in order of their D1 field, then D2
        // field, and the staged fields numbered in that order: lanes of one
        // shared-memory load phase then read the same D1 row (a broadcast) or
        // consecutive slots (different banks)
        auto keys = [&](const std::pair<int32_t, int32_t> &gr) {
            const Group &G = P.groups[gr.first];
            const Row &rw = P.rows[gr.second];
            const int a1 = G.n1 < 0 ? -G.n1 : G.n1, a2 = G.n2 < 0 ? -G.n2 : G.n2;
            return std::make_pair((a1 << 8) | rw.r1, (a2 << 8) | rw.r2);
        };
        std::stable_sort(cur.rows.begin(), cur.rows.end(),
                         [&](const auto &x, const auto &y) { return keys(x) < keys(y); });
        cur.slots.clear();
        for (auto &gr : cur.rows) {
            const auto k = keys(gr);
            if (slot_of(cur.slots, k.first) < 0) cur.slots.push_back(k.first);
            if (slot_of(cur.slots, k.second) < 0) cur.slots.push_back(k.second);
        }
        if (int(cur.slots.size()) != T.nslot) return "tcgen05 tile slots";
        // Bank groups: a 16-byte load of slot s falls in bank group s % 8
        // (slot stride 144 bytes), and the 8 lanes of a load phase that read
        // different slots of one group are served one after another.  Colour
        // the fields greedily (first appearance order) so that the distinct
        // D1 fields of each 8-row phase, and its distinct D2 fields, take
        // distinct colours where they can, and number them colour + 8 k;
        // numbers left free are padding slots that hold a field nothing
        // stores (they read as zero).  Kept only if the tile still fits.
        const int ns = T.nslot;
        std::vector<int> num(ns);
        {
            std::vector<std::vector<int>> adj(ns);
            for (size_t g0 = 0; g0 < cur.rows.size(); g0 += 8) {
                std::vector<int> U, V;
                for (size_t r = g0; r < std::min(cur.rows.size(), g0 + 8); ++r) {
                    const auto k = keys(cur.rows[r]);
                    const int f1 = slot_of(cur.slots, k.first), f2 = slot_of(cur.slots, k.second);
                    if (std::find(U.begin(), U.end(), f1) == U.end()) U.push_back(f1);
                    if (std::find(V.begin(), V.end(), f2) == V.end()) V.push_back(f2);
                }
                for (const auto *grp : {&U, &V})
                    for (int a : *grp)
                        for (int b : *grp)
                            if (a != b) adj[a].push_back(b);
            }
            std::vector<int> col(ns, -1), cnt(8, 0), next(8, 0);
            int top = 0;
            for (int f = 0; f < ns; ++f) {
                int use[8] = {0};
                for (int n : adj[f])
                    if (col[n] >= 0) ++use[col[n]];
                int best = 0;
                for (int c = 1; c < 8; ++c)
                    if (use[c] < use[best] || (use[c] == use[best] && cnt[c] < cnt[best])) best = c;
                col[f] = best;
                ++cnt[best];
                num[f] = best + 8 * next[best]++;
                top = std::max(top, num[f] + 1);
            }
            if (top <= kTcMaxSlots && tc_ring(T.ncol, top) > 0) {
                std::vector<int32_t> sl(size_t(top), (0 << 8) | R.nr);   // ring nr: never stored
                for (int f = 0; f < ns; ++f) sl[num[f]] = cur.slots[f];
                cur.slots.swap(sl);
                T.nslot = top;
            } else {
                for (int f = 0; f < ns; ++f) num[f] = f;
            }
        }
        for (auto &gr : cur.rows) {
            const Group &G = P.groups[gr.first];
            const Row &rw = P.rows[gr.second];
            TcRow t{};
            t.p0 = G.part0 + rw.coff;
            t.stride = G.ncombo;
            const int a1 = G.n1 < 0 ? -G.n1 : G.n1, a2 = G.n2 < 0 ? -G.n2 : G.n2;
            const auto k = keys(gr);
            t.s1 = uint8_t(slot_of(cur.slots, k.first));     // the field's number (its slot)
            t.s2 = uint8_t(slot_of(cur.slots, k.second));
            t.col0 = uint8_t(rw.r3a - cur.lo);
            t.n = rw.n;
            t.flags = uint8_t((G.n1 < 0 ? 1 : 0) | (G.n2 < 0 ? 2 : 0) | (G.n3 < 0 ? 4 : 0));
            P.tc_rows.push_back(t);
            U_(cur_lev, a1, rw.r1) = 1;
            U_(cur_lev, a2, rw.r2) = 1;
            for (int j = 0; j < rw.n; ++j) U_(cur_lev, cur_n3, rw.r3a + j) = 1;
        }
        P.tc_slots.insert(P.tc_slots.end(), cur.slots.begin(), cur.slots.end());
        P.tc_mma_products += double(kTcRows) * T.ncol * double(M2);
        P.tc_tiles.push_back(T);
        cur = Cur{};
        return "";
    };
    for (int lv = 0; lv < R.ngrid; ++lv)
        for (int n3 = 0; n3 <= nz; ++n3)
            for (int fl = 0; fl < 8; ++fl) {
            std::vector<int32_t> &gl = pool[(size_t(lv) * (nz + 1) + n3) * 8 + fl];
            if (gl.empty()) continue;
            std::stable_sort(gl.begin(), gl.end(), [&](int32_t a, int32_t b) {
                return P.groups[a].n1 < P.groups[b].n1;
            });
            std::string e = close();
            if (!e.empty()) return e;
            cur_lev = lv;
            cur_n3 = n3;
            cur_flags = fl;
            for (int32_t g : gl) {
                const Group &G = P.groups[g];
                std::vector<int32_t> order(G.nrow);
                for (int q = 0; q < G.nrow; ++q) order[q] = G.row0 + q;
                std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
                    const Row &X = P.rows[x], &Y = P.rows[y];
                    const int cx = 2 * X.r3a + X.n, cy = 2 * Y.r3a + Y.n;
                    return cx != cy ? cx < cy : X.r3a < Y.r3a;
                });
                const int a1 = G.n1 < 0 ? -G.n1 : G.n1, a2 = G.n2 < 0 ? -G.n2 : G.n2;
                for (int32_t ri : order) {
                    const Row &rw = P.rows[ri];
                    if (rw.n > kTcMaxCols) return "a row's r3 run is longer than a tcgen05 window";
                    const int k1 = (a1 << 8) | rw.r1, k2 = (a2 << 8) | rw.r2;
                    if (!cur.rows.empty()) {
                        const int lo = std::min(cur.lo, int(rw.r3a)), hi = std::max(cur.hi, rw.r3a + rw.n - 1);
                        const int add = (slot_of(cur.slots, k1) < 0) + (k2 != k1 && slot_of(cur.slots, k2) < 0);
                        const int ncol = ((hi - lo + 1 + 15) / 16) * 16;
                        const int ns = int(cur.slots.size()) + add;
                        if (int(cur.rows.size()) >= kTcRows || hi - lo + 1 > kTcMaxCols || ns > kTcMaxSlots ||
                            tc_ring(ncol, ns) == 0) {
                            e = close();
                            if (!e.empty()) return e;
                        }
                    }
                    if (slot_of(cur.slots, k1) < 0) cur.slots.push_back(k1);
                    if (slot_of(cur.slots, k2) < 0) cur.slots.push_back(k2);
                    cur.lo = std::min(cur.lo, int(rw.r3a));
                    cur.hi = std::max(cur.hi, rw.r3a + rw.n - 1);
                    cur.rows.emplace_back(g, ri);
                }
            }
        }
    std::string e = close();
    if (!e.empty()) return e;
    // units: class, then biggest grids first, x chunk, tile
    for (int c = 0; c < kTcClasses; ++c) {
        P.tc_class_begin[c] = int64_t(P.tc_units.size());
        for (int lv = R.ngrid - 1; lv >= 0; --lv) {
            int maxchunk = 0;
            for (const auto &T : P.tc_tiles)
                if (T.lev == lv && T.ncol / 16 - 1 == c) maxchunk = std::max(maxchunk, T.nchunk);
            for (int ch = 0; ch < maxchunk; ++ch)
                for (size_t t = 0; t < P.tc_tiles.size(); ++t) {
                    const TcTile &T = P.tc_tiles[t];
                    if (T.lev != lv || T.ncol / 16 - 1 != c || ch >= T.nchunk) continue;
                    P.tc_units.push_back(TcUnit{int32_t(t), ch});
                }
        }
    }
    P.tc_class_begin[kTcClasses] = int64_t(P.tc_units.size());
    return "";
}

}  // namespace

std::string enumerate(HostPlan &P, int64_t x_chunk)
{
    const Rings &R = P.rings;
    const int nz = R.nz, nr = R.nr;
    // half of the plane pairs: n1 > 0, or n1 == 0 and n2 >= 0
    std::vector<std::pair<int, int>> pairs;
    for (int n1 = 0; n1 <= nz; ++n1)
        for (int n2 = -nz; n2 <= nz; ++n2) {
            int n3 = -(n1 + n2);
            if (n3 < -nz || n3 > nz) continue;
            if (n1 == 0 && n2 < 0) continue;
            pairs.emplace_back(n1, n2);
        }
    std::vector<PairOut> outs(pairs.size());
    {
        std::atomic<size_t> next{0};
        unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
        std::vector<std::thread> th;
        for (unsigned t = 0; t < nt; ++t)
            th.emplace_back([&]() {
                for (;;) {
                    size_t k = next.fetch_add(1);
                    if (k >= pairs.size()) break;
                    enumerate_pair(P, pairs[k].first, pairs[k].second, outs[k]);
                }
            });
        for (auto &t : th) t.join();
    }

    // Work of the sums on each combination's smallest exact grid (the
    // algorithmic figures the plan reports): the grid points of every
    // combination, and of every distinct (pair, r1, r2, grid) product D1 D2.
    // acc is ordered by (r1, r2, r3), so the grids of one (r1, r2) are
    // collected in one run.
    P.triple_products = 0;
    P.pair_products = 0;
    for (const PairOut &po : outs)
        for (size_t i = 0; i < po.acc.size();) {
            uint32_t levs = 0;
            size_t j = i;
            for (; j < po.acc.size() && po.acc[j].r1 == po.acc[i].r1 && po.acc[j].r2 == po.acc[i].r2; ++j) {
                const double m = double(R.grid[po.acc[j].lev]);
                P.triple_products += m * m;
                levs |= 1u << po.acc[j].lev;
            }
            for (int lv = 0; lv < R.ngrid; ++lv)
                if (levs >> lv & 1u) P.pair_products += double(R.grid[lv]) * double(R.grid[lv]);
            i = j;
        }
    // tcgen05: the combinations of one (r1, r2) of a pair are summed on one
    // grid, the largest their r3 need.  On any grid above the bound the sum
    // is exact (see triple_level), and a row's pair product D1 D2 is then
    // formed once instead of once per grid; forming it, not the MMAs that
    // apply it to the r3 window, is what the tensor-core tiles spend their
    // time on.  The CUDA-core tiles do work per combination and keep the
    // smallest grid.
    if (P.tensor)
        for (PairOut &po : outs)
            for (size_t i = 0; i < po.acc.size();) {
                size_t j = i;
                uint8_t top = 0;
                for (; j < po.acc.size() && po.acc[j].r1 == po.acc[i].r1 && po.acc[j].r2 == po.acc[i].r2; ++j)
                    top = std::max(top, po.acc[j].lev);
                for (size_t q = i; q < j; ++q) po.acc[q].lev = top;
                i = j;
            }

    // used[l][n][r]: D fields to store
    std::vector<uint8_t> used(size_t(kMaxLevels) * (nz + 1) * kMaxRings, 0);
    auto U_ = [&](int lv, int n, int r) -> uint8_t & {
        return used[(size_t(lv) * (nz + 1) + n) * kMaxRings + r];
    };

    P.groups.clear();
    P.rows.clear();
    P.tiles.clear();
    P.units.clear();
    P.records_s.clear();
    P.ntri_s.clear();
    P.n_combos = 0;
    P.n_pairs = 0;
    P.max_slots = 0;
    std::vector<Unit> unit_tmpl;                 // per group: tile ranges and staged rings
    std::vector<int32_t> group_unit0(1, 0);      // first template of each group
    int64_t cidx = 0;
    for (size_t k = 0; k < outs.size(); ++k) {
        PairOut &po = outs[k];
        if (po.acc.empty()) continue;
        P.n_pairs++;
        const int n1 = po.n1, n2 = po.n2, n3 = -(n1 + n2);
        for (int lv = 0; lv < R.ngrid; ++lv) {
            Group G{};
            G.n1 = n1; G.n2 = n2; G.n3 = n3;
            G.lev = lv;
            G.M = R.grid[lv];
            G.row0 = int32_t(P.rows.size());
            G.c0 = cidx;
            G.self_conj = (n1 == 0 && n2 == 0) ? 1 : 0;
            int ncombo = 0;
            size_t i = 0;
            while (i < po.acc.size()) {
                if (po.acc[i].lev != lv) { ++i; continue; }
                // a run of consecutive r3 with the same (r1, r2) on this grid
                const Acc &a = po.acc[i];
                size_t j = i + 1;
                int r3 = a.r3;
                while (j < po.acc.size() && po.acc[j].lev == lv && po.acc[j].r1 == a.r1 &&
                       po.acc[j].r2 == a.r2 && po.acc[j].r3 == r3 + 1 && (j - i) < size_t(255)) {
                    ++j;
                    ++r3;
                }
                P.rows.push_back(Row{a.r1, a.r2, a.r3, uint8_t(j - i), ncombo});
                for (size_t q = i; q < j; ++q) {
                    const Acc &c = po.acc[q];
                    Record rec;
                    rec.s_index = int32_t(cidx + ncombo);
                    rec.flags = (G.self_conj ? 1 : 0) | (c.g.degenerate ? 2 : 0);
                    rec.pz = c.g.pz;
                    rec.cphi = c.g.cphi;
                    P.records_s.push_back(rec);
                    P.ntri_s.push_back(double(P.ntri[(size_t(c.r1) * nr + c.r2) * nr + c.r3]));
                    ++ncombo;
                }
                i = j;
            }
            if (ncombo == 0) continue;
            G.nrow = int32_t(P.rows.size()) - G.row0;
            G.ncombo = ncombo;
            const int64_t M2 = int64_t(G.M) * G.M;
            G.nchunk = int32_t((M2 + x_chunk - 1) / x_chunk);
            cidx += ncombo;

            if (P.tensor) {             // tcgen05 tiles span groups: built after the loop
                P.groups.push_back(G);
                group_unit0.push_back(int32_t(unit_tmpl.size()));
                continue;
            }
            // register tiles: rows ordered by the centre of their r3 run,
            // blocks of kTileRows rows, each block cut into windows of
            // kTileCols consecutive r3 covering the union of its runs
            std::vector<int> order(G.nrow);
            for (int q = 0; q < G.nrow; ++q) order[q] = q;
            const Row *rw = P.rows.data() + G.row0;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
                int cx = 2 * rw[x].r3a + rw[x].n, cy = 2 * rw[y].r3a + rw[y].n;
                return cx != cy ? cx < cy : rw[x].r3a < rw[y].r3a;
            });
            struct Raw { int rows[kTileRows]; int nr; int w0; };
            std::vector<Raw> raws;
            for (int b = 0; b < G.nrow; b += kTileRows) {
                Raw base{};
                base.nr = std::min(kTileRows, G.nrow - b);
                for (int q = 0; q < base.nr; ++q) base.rows[q] = order[b + q];
                std::vector<uint8_t> cov(kMaxRings + kTileCols, 0);
                for (int q = 0; q < base.nr; ++q)
                    for (int c = 0; c < rw[base.rows[q]].n; ++c) cov[rw[base.rows[q]].r3a + c] = 1;
                for (int c = 0; c < kMaxRings; ++c) {
                    if (!cov[c]) continue;
                    Raw t = base;
                    t.w0 = c;
                    raws.push_back(t);
                    for (int d = 0; d < kTileCols; ++d) cov[c + d] = 0;
                }
            }
            // units: runs of 16, 8 or 4 consecutive tiles (one per warp), each
            // staging the union of its tiles' rings
            size_t u0 = 0;
            while (u0 < raws.size()) {
                const size_t rem = raws.size() - u0;
                int cls = rem >= 16 ? 4 : (rem >= 8 ? 3 : 2);
                if (cls > P.max_cls) cls = P.max_cls;
                const size_t take = std::min(rem, size_t(1) << cls);
                const size_t u1 = u0 + take;
                Unit U{};
                U.t0 = int32_t(P.tiles.size());
                U.nt = int32_t(take);
                int lo[3] = {nr, nr, kMaxRings}, hi[3] = {-1, -1, -1};
                for (size_t t = u0; t < u1; ++t) {
                    const Raw &w = raws[t];
                    for (int q = 0; q < w.nr; ++q) {
                        const Row &r = rw[w.rows[q]];
                        lo[0] = std::min<int>(lo[0], r.r1); hi[0] = std::max<int>(hi[0], r.r1);
                        lo[1] = std::min<int>(lo[1], r.r2); hi[1] = std::max<int>(hi[1], r.r2);
                    }
                    lo[2] = std::min(lo[2], w.w0);
                    hi[2] = std::max(hi[2], w.w0 + kTileCols - 1);
                }
                for (int q = 0; q < 3; ++q) { U.rlo[q] = int16_t(lo[q]); U.rhi[q] = int16_t(hi[q]); }
                const int nq0 = hi[0] - lo[0] + 1, nq1 = hi[1] - lo[1] + 1, nq2 = hi[2] - lo[2] + 1;
                const int ns = nq0 + nq1 + nq2;
                if (ns > 255) return "too many staged rings in a Step-II unit";
                // a class whose shared memory holds two stages of 64 points
                while (cls < P.max_cls && step2_smem_need(ns, 64, P.celem) > kStep2ClassSmem[cls]) ++cls;
                if (step2_smem_need(ns, 64, P.celem) > kStep2ClassSmem[cls])
                    return "Step-II unit too large for shared memory";
                U.cls = cls;
                P.max_slots = std::max(P.max_slots, ns);
                for (size_t t = u0; t < u1; ++t) {
                    const Raw &w = raws[t];
                    Tile T{};
                    for (int q = 0; q < kTileRows; ++q) {
                        const Row &r = rw[w.rows[q < w.nr ? q : 0]];
                        T.s1[q] = uint8_t(r.r1 - lo[0]);
                        T.s2[q] = uint8_t(nq0 + r.r2 - lo[1]);
                        T.coff[q] = r.coff + (w.w0 - r.r3a);
                        if (q >= w.nr) continue;
                        for (int d = 0; d < kTileCols; ++d) {
                            const int r3 = w.w0 + d;
                            if (r3 >= r.r3a && r3 < r.r3a + r.n)
                                T.mask[(q * kTileCols + d) >> 5] |= 1u << ((q * kTileCols + d) & 31);
                        }
                    }
                    T.s3 = uint8_t(nq0 + nq1 + w.w0 - lo[2]);
                    P.tiles.push_back(T);
                }
                const int nsabs[3] = {n1 < 0 ? -n1 : n1, n2 < 0 ? -n2 : n2, n3 < 0 ? -n3 : n3};
                for (int q = 0; q < 3; ++q)
                    for (int r = lo[q]; r <= std::min(hi[q], nr - 1); ++r) U_(lv, nsabs[q], r) = 1;
                U.group = int32_t(P.groups.size());
                unit_tmpl.push_back(U);
                u0 = u1;
            }
            P.groups.push_back(G);
            group_unit0.push_back(int32_t(unit_tmpl.size()));
        }
        std::vector<Acc>().swap(po.acc);
    }
    P.n_combos = cidx;
    if (P.n_combos >= (int64_t(1) << 31) - 1) return "too many combinations for 32-bit indices";

    // partial sums [group][x chunk][combination]
    int64_t part = 0;
    for (auto &G : P.groups) {
        G.part0 = part;
        part += int64_t(G.nchunk) * G.ncombo;
    }
    P.n_partials = part;
    if (P.tensor) {
        std::string e = build_tc(P, x_chunk, U_);
        if (!e.empty()) return e;
    }

    // D-store layout, grid by grid, plane by plane, ring by ring
    P.doff.assign(size_t(kMaxLevels) * (nz + 1) * kMaxRings, -1);
    P.levels.clear();
    int64_t cursor = 0;
    P.gt_elems = 0;
    for (int lv = 0; lv < R.ngrid; ++lv) {
        Level L;
        L.lev = lv;
        L.M = R.grid[lv];
        L.dstore_off = cursor;
        const int64_t M2 = int64_t(L.M) * L.M;
        for (int n = 0; n <= nz; ++n)
            for (int r = 0; r < nr; ++r)
                if (U_(lv, n, r)) {
                    P.doff[(size_t(lv) * (nz + 1) + n) * kMaxRings + r] = cursor;
                    cursor += M2;
                    L.njobs++;
                }
        if (L.njobs) {
            P.levels.push_back(L);
            P.gt_elems = std::max(P.gt_elems, L.njobs * M2);
        }
    }
    P.dstore_elems = cursor;

    // Step-II units in launch order: biggest grids
    // first, then by x chunk, then by blocks of 8 x 8 plane pairs, so that
    // blocks running together share planes (and their rings) in L2
    if (P.tensor) return "";
    std::vector<int32_t> gorder(P.groups.size());
    for (size_t g = 0; g < gorder.size(); ++g) gorder[g] = int32_t(g);
    auto blk = [&](const Group &G) { return std::make_pair((G.n1) / 8, (G.n2 + nz) / 8); };
    std::stable_sort(gorder.begin(), gorder.end(), [&](int32_t a, int32_t b) {
        const Group &A = P.groups[a], &B = P.groups[b];
        if (A.lev != B.lev) return A.lev > B.lev;
        return blk(A) < blk(B);
    });
    // units grouped by block class; within a class: grid, x chunk, pair block
    for (int cls = 2; cls <= 4; ++cls) {
        P.class_begin[cls] = int64_t(P.units.size());
        for (int lv = R.ngrid - 1; lv >= 0; --lv) {
            int maxchunk = 0;
            for (auto &G : P.groups)
                if (G.lev == lv) maxchunk = std::max(maxchunk, G.nchunk);
            for (int c = 0; c < maxchunk; ++c)
                for (int32_t g : gorder) {
                    const Group &G = P.groups[g];
                    if (G.lev != lv || c >= G.nchunk) continue;
                    for (int32_t u = group_unit0[g]; u < group_unit0[g + 1]; ++u) {
                        if (unit_tmpl[u].cls != cls) continue;
                        Unit U = unit_tmpl[u];
                        U.chunk = c;
                        P.units.push_back(U);
                    }
                }
        }
    }
    P.class_begin[5] = int64_t(P.units.size());
    return "";
}

void build_views(HostPlan &P, const int *n_mu_l, const int *n_t_l)
{
    const bisp_desc &d = P.desc;
    P.views.clear();
    for (int l = 0; l <= d.l_max; l += 2) {
        const int nm = n_mu_l ? n_mu_l[l / 2] : d.n_mu, nt = n_t_l ? n_t_l[l / 2] : d.n_t;
        if (!P.views.empty() && P.views.back().n_mu == nm && P.views.back().n_t == nt) {
            P.views.back().l_hi = l;
            continue;
        }
        View v;
        v.l_lo = v.l_hi = l;
        v.n_mu = nm;
        v.n_t = nt;
        P.views.push_back(v);
    }
    int64_t off = 0, bs = 0;
    for (size_t i = 0; i < P.views.size(); ++i) {
        View &v = P.views[i];
        v.lm_lo = (v.l_lo / 2) * (v.l_lo / 2);
        v.n_lm = (v.l_hi / 2 + 1) * (v.l_hi / 2 + 1) - v.lm_lo;
        v.n_bins = int64_t(d.n_k1) * v.n_mu * v.n_t;
        v.out_off = off;
        v.bs_off = bs;
        off += v.n_bins * v.n_lm;
        bs += v.n_bins + 1;
    }
    P.n_out = off;
}

void combo_shapes(const HostPlan &P, int64_t cap, double *out)
{
    const Rings &R = P.rings;
    for (const auto &G : P.groups)
        for (int s = 0; s < G.nrow; ++s) {
            const Row &rw = P.rows[G.row0 + s];
            for (int j = 0; j < rw.n; ++j) {
                const int64_t k = G.c0 + rw.coff + j;
                if (k >= cap) continue;
                Geo g;
                combo_geometry(P, R.kperp[rw.r1], R.kperp[rw.r2], R.kperp[rw.r3a + j], G.n1, G.n2, G.n3, &g);
                out[4 * k] = g.mu;
                out[4 * k + 1] = g.t;
                out[4 * k + 2] = g.pz;
                out[4 * k + 3] = g.cphi;
            }
        }
}

void sort_records(HostPlan &P)
{
    // shape of each record, recomputed from S order through its group
    const size_t n = P.records_s.size();
    std::vector<int32_t> bin(n), kb(n);
    std::vector<double> mu(n), t(n);
    const Rings &R = P.rings;
    for (const auto &G : P.groups)
        for (int s = 0; s < G.nrow; ++s) {
            const Row &rw = P.rows[G.row0 + s];
            for (int j = 0; j < rw.n; ++j) {
                Geo g;
                combo_geometry(P, R.kperp[rw.r1], R.kperp[rw.r2], R.kperp[rw.r3a + j], G.n1, G.n2, G.n3, &g);
                const int64_t k = G.c0 + rw.coff + j;
                bin[k] = g.bin;
                kb[k] = g.ib;
                mu[k] = g.mu;
                t[k] = g.t;
            }
        }
    P.combo_bin = bin;
    size_t total_bs = 0;
    for (const View &v : P.views) total_bs += size_t(v.n_bins) + 1;
    P.records.resize(n * P.views.size());
    P.rec_ntri.resize(n * P.views.size());
    P.bin_start.assign(total_bs, 0);
    for (size_t vi = 0; vi < P.views.size(); ++vi) {
        View &v = P.views[vi];
        v.rec_off = int64_t(vi * n);
        for (size_t k = 0; k < n; ++k) bin[k] = grid_bin(kb[k], mu[k], t[k], v.n_mu, v.n_t);
        int64_t *bs = P.bin_start.data() + v.bs_off;
        bs[0] = v.rec_off;
        for (size_t k = 0; k < n; ++k) bs[bin[k] + 1]++;
        for (int64_t b = 0; b < v.n_bins; ++b) bs[b + 1] += bs[b];
        std::vector<int64_t> pos(bs, bs + v.n_bins);
        for (size_t k = 0; k < n; ++k) {
            const int64_t p = pos[bin[k]]++;
            P.records[p] = P.records_s[k];
            P.rec_ntri[p] = P.ntri_s[k];
        }
    }
    std::vector<Record>().swap(P.records_s);
    std::vector<double>().swap(P.ntri_s);
    // binning chunks: each bin's records in runs of at most kBinChunk, so no
    // warp of the binning walks a whole large bin alone
    P.chunk_lo.clear();
    P.chunk_hi.clear();
    P.bin_chunk.assign(total_bs, 0);
    P.max_chunks = 0;
    int64_t bc = 0;
    for (View &v : P.views) {
        const int64_t *bs = P.bin_start.data() + v.bs_off;
        v.chunk_off = int64_t(P.chunk_lo.size());
        v.bc_off = bc;
        for (int64_t b = 0; b < v.n_bins; ++b) {
            P.bin_chunk[bc + b] = int64_t(P.chunk_lo.size()) - v.chunk_off;
            for (int64_t k = bs[b]; k < bs[b + 1]; k += kBinChunk) {
                P.chunk_lo.push_back(k);
                P.chunk_hi.push_back(std::min(k + kBinChunk, bs[b + 1]));
            }
        }
        v.n_chunks = int64_t(P.chunk_lo.size()) - v.chunk_off;
        P.bin_chunk[bc + v.n_bins] = v.n_chunks;
        bc += v.n_bins + 1;
        P.max_chunks = std::max(P.max_chunks, v.n_chunks);
    }
}

int unit_classes(const HostPlan &P, const int64_t **class_begin)
{
    *class_begin = P.tensor ? P.tc_class_begin : P.class_begin;
    return P.tensor ? kTcClasses : 5;
}

void unit_costs(HostPlan &P, int64_t x_chunk)
{
    auto points = [&](int M, int chunk) {
        const int64_t m2 = int64_t(M) * M, x0 = int64_t(chunk) * x_chunk;
        return double(std::min(x_chunk, m2 - x0));
    };
    const size_t n = P.tensor ? P.tc_units.size() : P.units.size();
    P.unit_cost.assign(n + 1, 0.0);
    for (size_t u = 0; u < n; ++u) {
        double c;
        if (P.tensor) {
            const TcUnit &U = P.tc_units[u];
            c = points(P.tc_tiles[U.tile].M, U.chunk);
        } else {
            const Unit &U = P.units[u];
            c = points(P.groups[U.group].M, U.chunk) * U.nt;
        }
        P.unit_cost[u + 1] = P.unit_cost[u] + c;
    }
}

void part_ranges(const HostPlan &P, int part, int nparts, int64_t *lo, int64_t *hi)
{
    const int64_t *cb;
    const int ncls = unit_classes(P, &cb);
    const std::vector<double> &c = P.unit_cost;
    for (int k = 0; k < ncls; ++k) {
        const int64_t a = cb[k], b = cb[k + 1];
        // first unit of share p: the first whose preceding cost reaches p/nparts of the class
        auto cut = [&](int p) -> int64_t {
            if (p <= 0) return a;
            if (p >= nparts) return b;
            const double target = c[a] + (c[b] - c[a]) * double(p) / double(nparts);
            return int64_t(std::lower_bound(c.begin() + a, c.begin() + b, target) - c.begin());
        };
        lo[k] = cut(part);
        hi[k] = cut(part + 1);
    }
    for (int k = ncls; k < kClassSlots; ++k) lo[k] = hi[k] = 0;
}

}  // namespace bisp
