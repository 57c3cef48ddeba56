// plan_host_check.cpp -- builds the host part of an estimator plan on the CPU
// (the triangle counts N_tri are read from a file instead of being computed
// on the GPU) and writes what tests/test_plan_host.py checks:
//   <out>.combos  int32 [n][7]: n1, n2, n3, r1, r2, r3, M of every combination
//   <out>.groups  int64 [g][2]: partial-sum start and combination count of every group
//   <out>.tcrows  int64 [t][7]: p0, n, col0, ncol, nrow, nslot, ring buffers of every
//                               tensor-core tile row (tensor plans only)
//   stdout: one line "combos groups tcrows missing_fields"
// Usage: plan_host_check ng box_len n_k1 n_mu tensor ntri_file edges_file out_prefix
// (ntri_file: int64 [nr][nr][nr]; edges_file: double [n_k1 + 1], h/Mpc)
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "plan.hpp"

using namespace bisp;

int main(int argc, char **argv)
{
    if (argc != 9) return 2;
    const int ng = std::atoi(argv[1]), nk1 = std::atoi(argv[3]), nmu = std::atoi(argv[4]);
    const double L = std::atof(argv[2]);
    const bool tensor = std::atoi(argv[5]) != 0;
    HostPlan P;
    P.desc.n_g = ng;
    P.desc.box_len = L;
    P.desc.n_k1 = nk1;
    P.desc.n_mu = nmu;
    P.desc.n_t = nmu;
    P.desc.l_max = 6;
    P.desc.max_batch = 1;
    P.desc.precision = tensor ? BISP_PREC_MIXED_TC : BISP_PREC_MIXED;
    P.kf = 2.0 * M_PI / L;
    P.k1_edges.resize(size_t(nk1) + 1);
    FILE *fe = std::fopen(argv[7], "rb");
    if (!fe || std::fread(P.k1_edges.data(), sizeof(double), P.k1_edges.size(), fe) != P.k1_edges.size()) return 4;
    std::fclose(fe);
    P.desc.k1_edges = P.k1_edges.data();
    if (!build_rings(ng, P.rings)) return 3;
    const int nr = P.rings.nr;
    P.ntri.resize(size_t(nr) * nr * nr);
    FILE *f = std::fopen(argv[6], "rb");
    if (!f || std::fread(P.ntri.data(), sizeof(int64_t), P.ntri.size(), f) != P.ntri.size()) return 4;
    std::fclose(f);
    P.celem = 8;
    P.max_cls = 4;
    P.tensor = tensor;
    const std::string err = enumerate(P, 16384);
    if (!err.empty()) {
        std::fprintf(stderr, "enumerate: %s\n", err.c_str());
        return 5;
    }
    const std::string out = argv[8];
    std::vector<int32_t> combos;
    std::vector<int64_t> groups;
    int64_t missing = 0;
    for (const Group &G : P.groups) {
        groups.push_back(G.part0);
        groups.push_back(G.ncombo);
        for (int q = 0; q < G.nrow; ++q) {
            const Row &rw = P.rows[size_t(G.row0) + q];
            for (int j = 0; j < rw.n; ++j) {
                const int r3 = rw.r3a + j;
                combos.insert(combos.end(), {G.n1, G.n2, G.n3, int32_t(rw.r1), int32_t(rw.r2), r3, G.M});
                const int n[3] = {G.n1, G.n2, G.n3}, r[3] = {rw.r1, rw.r2, r3};
                for (int k = 0; k < 3; ++k) {
                    const int a = n[k] < 0 ? -n[k] : n[k];
                    if (P.doff[(size_t(G.lev) * (P.rings.nz + 1) + a) * kMaxRings + r[k]] < 0) ++missing;
                }
            }
        }
    }
    std::vector<int64_t> tcrows;
    for (const TcTile &T : P.tc_tiles)
        for (int q = 0; q < T.nrow; ++q) {
            const TcRow &R = P.tc_rows[size_t(T.row0) + q];
            tcrows.insert(tcrows.end(), {R.p0, int64_t(R.n), int64_t(R.col0), int64_t(T.ncol), int64_t(T.nrow),
                                         int64_t(T.nslot), int64_t(tc_ring(T.ncol, T.nslot))});
        }
    auto dump = [&](const char *ext, const void *data, size_t bytes) {
        FILE *o = std::fopen((out + ext).c_str(), "wb");
        if (!o) return false;
        const bool ok = std::fwrite(data, 1, bytes, o) == bytes;
        std::fclose(o);
        return ok;
    };
    if (!dump(".combos", combos.data(), combos.size() * sizeof(int32_t)) ||
        !dump(".groups", groups.data(), groups.size() * sizeof(int64_t)) ||
        !dump(".tcrows", tcrows.data(), tcrows.size() * sizeof(int64_t)))
        return 6;
    std::printf("%zu %zu %zu %lld\n", combos.size() / 7, groups.size() / 2, tcrows.size() / 7, (long long)missing);
    return 0;
}
