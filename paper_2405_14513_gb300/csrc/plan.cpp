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

bool build_rings(int ng, Rings &R)
{
    if (ng < 8 || ng > 1024 || (ng & (ng - 1))) return false;
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
    return true;
}

int triple_log2m(const Rings &R, int r1, int r2, int r3)
{
    int need = R.maxc[r1] + R.maxc[r2] + R.maxc[r3] + 1;
    int lg = kMinLog2M;
    while ((1 << lg) < need) ++lg;
    int lgmax = 0;
    while ((1 << lgmax) < R.ng) ++lgmax;
    return std::min(lg, lgmax);
}

namespace {

struct Geo {
    int bin;
    int degenerate;
    double pz, cphi;
};

// Acceptance and geometry of one combination (planes n1, n2, n3 with ring
// radii kp1..kp3 in grid units): K1 >= K2 >= K3 > 0 with
// K_i^2 = k_perp,i^2 + n_i^2; K1 in a k1 bin; t = K2/K1 >= 1/2;
// mu = (K1^2 + K2^2 - K3^2) / (2 K1 K2) clamped to [1/2, 1];
// p_z = mu_1, p_x = (mu_2 + mu mu_1)/sqrt(1 - mu^2) (inverse of Eq. orient),
// p_y = +sqrt(max(0, 1 - p_z^2 - p_x^2)), cos phi = p_x / |(p_x, p_y)|.
bool combo_geometry(const HostPlan &P, double kp1, double kp2, double kp3, int n1, int n2, int n3,
                    Geo *g)
{
    const bisp_desc &d = P.desc;
    double k1sq = kp1 * kp1 + double(n1) * n1;
    double k2sq = kp2 * kp2 + double(n2) * n2;
    double k3sq = kp3 * kp3 + double(n3) * n3;
    if (!(k1sq >= k2sq && k2sq >= k3sq && k3sq > 0.0)) return false;
    double s1 = std::sqrt(k1sq), s2 = std::sqrt(k2sq);
    double K1 = P.kf * s1;
    int ib = -1;
    for (int b = 0; b < d.n_k1; ++b)
        if (P.k1_edges[b] <= K1 && K1 < P.k1_edges[b + 1]) { ib = b; break; }
    if (ib < 0 && K1 == P.k1_edges[d.n_k1]) ib = d.n_k1 - 1;
    if (ib < 0) return false;
    double t = s2 / s1;
    double mu = (k1sq + k2sq - k3sq) / (2.0 * std::sqrt(k1sq * k2sq));
    if (mu > 1.0) mu = 1.0;
    if (mu < 0.5) mu = 0.5;
    if (t < 0.5) return false;
    int it = int(std::floor((t - 0.5) * (2.0 * d.n_t)));
    int im = int(std::floor((mu - 0.5) * (2.0 * d.n_mu)));
    if (it >= d.n_t) it = d.n_t - 1;
    if (im >= d.n_mu) im = d.n_mu - 1;
    g->bin = (ib * d.n_mu + im) * d.n_t + it;
    double mu1 = double(n1) / s1;
    double mu2 = double(n2) / s2;
    g->pz = mu1;
    g->degenerate = (mu >= 1.0 - 1e-12);
    if (g->degenerate) {
        g->cphi = 1.0;
    } else {
        double px = (mu2 + mu * mu1) / std::sqrt(1.0 - mu * mu);
        double q = 1.0 - g->pz * g->pz - px * px;
        double py = std::sqrt(q > 0.0 ? q : 0.0);
        double rho = std::sqrt(px * px + py * py);
        g->cphi = rho > 0.0 ? px / rho : 1.0;
    }
    return true;
}

struct Acc {            // one accepted combination of a pair
    uint8_t r1, r2, r3, lg;
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
                                      uint8_t(triple_log2m(R, r1, r2, r3)), g});
            }
        }
    }
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

    // used[l][n][r]: D fields to store
    const int lgmax = [&] { int l = 0; while ((1 << l) < R.ng) ++l; return l; }();
    std::vector<uint8_t> used(size_t(kMaxLevels) * (nz + 1) * kMaxRings, 0);
    auto U = [&](int lg, int n, int r) -> uint8_t & {
        return used[(size_t(lg) * (nz + 1) + n) * kMaxRings + r];
    };

    P.groups.clear();
    P.segs.clear();
    P.records_s.clear();
    P.ntri_s.clear();
    P.n_combos = 0;
    P.n_pairs = 0;
    P.triple_products = 0;
    int64_t cidx = 0;
    for (size_t k = 0; k < outs.size(); ++k) {
        PairOut &po = outs[k];
        if (po.acc.empty()) continue;
        P.n_pairs++;
        const int n1 = po.n1, n2 = po.n2, n3 = -(n1 + n2);
        for (int lg = kMinLog2M; lg <= lgmax; ++lg) {
            Group G{};
            G.n1 = n1; G.n2 = n2; G.n3 = n3;
            G.log2m = lg;
            G.seg0 = int32_t(P.segs.size());
            G.c0 = cidx;
            G.self_conj = (n1 == 0 && n2 == 0) ? 1 : 0;
            for (int q = 0; q < 3; ++q) { G.rlo[q] = nr; G.rhi[q] = -1; }
            int ncombo = 0;
            size_t i = 0;
            while (i < po.acc.size()) {
                if (po.acc[i].lg != lg) { ++i; continue; }
                // a run of consecutive r3 with the same (r1, r2) on this grid
                const Acc &a = po.acc[i];
                size_t j = i + 1;
                int r3 = a.r3;
                while (j < po.acc.size() && po.acc[j].lg == lg && po.acc[j].r1 == a.r1 &&
                       po.acc[j].r2 == a.r2 && po.acc[j].r3 == r3 + 1 && (j - i) < size_t(kSegLen)) {
                    ++j;
                    ++r3;
                }
                Segment s{a.r1, a.r2, a.r3, uint8_t(j - i), ncombo};
                P.segs.push_back(s);
                G.rlo[0] = std::min<int>(G.rlo[0], a.r1); G.rhi[0] = std::max<int>(G.rhi[0], a.r1);
                G.rlo[1] = std::min<int>(G.rlo[1], a.r2); G.rhi[1] = std::max<int>(G.rhi[1], a.r2);
                G.rlo[2] = std::min<int>(G.rlo[2], a.r3); G.rhi[2] = std::max<int>(G.rhi[2], r3);
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
                // skip the run (later entries of other grids stay)
                for (size_t q = i; q < j; ++q) po.acc[q].lg = 255;
                i = j;
            }
            if (ncombo == 0) continue;
            G.nseg = int32_t(P.segs.size()) - G.seg0;
            G.ncombo = ncombo;
            const int64_t M2 = int64_t(1) << (2 * lg);
            G.nchunk = int32_t((M2 + x_chunk - 1) / x_chunk);
            P.triple_products += double(ncombo) * double(M2);
            cidx += ncombo;
            const int ns[3] = {n1 < 0 ? -n1 : n1, n2 < 0 ? -n2 : n2, n3 < 0 ? -n3 : n3};
            for (int q = 0; q < 3; ++q)
                for (int r = G.rlo[q]; r <= G.rhi[q]; ++r) U(lg, ns[q], r) = 1;
            P.groups.push_back(G);
        }
        std::vector<Acc>().swap(po.acc);
    }
    P.n_combos = cidx;
    if (P.n_combos >= (int64_t(1) << 31) - 1) return "too many combinations for 32-bit indices";

    // D-store layout, grid by grid, plane by plane, ring by ring
    P.doff.assign(size_t(kMaxLevels) * (nz + 1) * kMaxRings, -1);
    P.levels.clear();
    int64_t cursor = 0;
    P.gt_elems = 0;
    for (int lg = kMinLog2M; lg <= lgmax; ++lg) {
        Level L;
        L.log2m = lg;
        L.dstore_off = cursor;
        const int64_t M2 = int64_t(1) << (2 * lg);
        for (int n = 0; n <= nz; ++n)
            for (int r = 0; r < nr; ++r)
                if (U(lg, n, r)) {
                    P.doff[(size_t(lg) * (nz + 1) + n) * kMaxRings + r] = cursor;
                    cursor += M2;
                    L.njobs++;
                }
        if (L.njobs) {
            P.levels.push_back(L);
            P.gt_elems = std::max(P.gt_elems, L.njobs * M2);
        }
    }
    P.dstore_elems = cursor;

    // partial-sum layout and Step-II items: biggest grids first, then by
    // chunk, then in pair order, so that concurrent blocks share planes
    int64_t part = 0;
    for (auto &G : P.groups) {
        G.part0 = part;
        part += int64_t(G.nchunk) * G.ncombo;
    }
    P.n_partials = part;
    P.items.clear();
    for (int lg = lgmax; lg >= kMinLog2M; --lg) {
        int maxchunk = 0;
        for (auto &G : P.groups)
            if (G.log2m == lg) maxchunk = std::max(maxchunk, G.nchunk);
        for (int c = 0; c < maxchunk; ++c)
            for (size_t g = 0; g < P.groups.size(); ++g)
                if (P.groups[g].log2m == lg && c < P.groups[g].nchunk)
                    P.items.push_back(Item{int32_t(g), int32_t(c)});
    }
    return "";
}

void sort_records(HostPlan &P)
{
    // bin of each record, recomputed from S order through its group
    const int64_t nb = P.n_bins;
    std::vector<int32_t> bin(P.records_s.size());
    const Rings &R = P.rings;
    for (const auto &G : P.groups)
        for (int s = 0; s < G.nseg; ++s) {
            const Segment &sg = P.segs[G.seg0 + s];
            for (int j = 0; j < sg.n; ++j) {
                Geo g;
                combo_geometry(P, R.kperp[sg.r1], R.kperp[sg.r2], R.kperp[sg.r3a + j], G.n1, G.n2, G.n3, &g);
                bin[G.c0 + sg.coff + j] = g.bin;
            }
        }
    P.combo_bin = bin;
    P.bin_start.assign(nb + 1, 0);
    for (auto b : bin) P.bin_start[b + 1]++;
    for (int64_t b = 0; b < nb; ++b) P.bin_start[b + 1] += P.bin_start[b];
    std::vector<int64_t> pos(P.bin_start.begin(), P.bin_start.end() - 1);
    P.records.resize(P.records_s.size());
    P.rec_ntri.resize(P.records_s.size());
    for (size_t k = 0; k < P.records_s.size(); ++k) {
        int64_t p = pos[bin[k]]++;
        P.records[p] = P.records_s[k];
        P.rec_ntri[p] = P.ntri_s[k];
    }
    std::vector<Record>().swap(P.records_s);
    std::vector<double>().swap(P.ntri_s);
}

}  // namespace bisp
