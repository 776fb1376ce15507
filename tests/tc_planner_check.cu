// Host-only checks of the tensor-core contraction planner (layout_plan): pair tiles, windows of singles, tensor-
// and shared-memory budgets, and the gather index of every output.  Built by the CPU test suite from the kernel
// source itself and linked against libpolybin for the few host helpers it references; it makes no CUDA call.
#include "contract_tc.cu"

#include <cstdio>
#include <map>
#include <random>
#include <set>
#include <tuple>

using namespace pb;
using namespace pb::tc;

static int n_fail = 0;
#define REQUIRE(cond, ...)                                      \
    do {                                                        \
        if (!(cond)) {                                          \
            ++n_fail;                                           \
            std::printf("FAIL %s: ", name);                     \
            std::printf(__VA_ARGS__);                           \
            std::printf("\n");                                  \
            return;                                             \
        }                                                       \
    } while (0)

// One layout with the given options: the default options must succeed; the autotuner's other candidates may be
// rejected by the planner (e.g. more than four row groups) but must satisfy every check when accepted.
static void check_one(const char* name, long ncell, int ng, int nh, int hsep, std::vector<NeedPair> need, int n_out,
                      int sing_g, const PlanOpts& opts, bool must) {
    std::map<int, std::tuple<int, int, int>> want;   // output -> (j, k, single)
    for (const NeedPair& p : need)
        for (auto& so : p.outs) want[so.second] = std::make_tuple(p.j, p.k, so.first);
    Plan pl;   // layout only: its device pointers stay null
    std::vector<short2> rows;
    std::vector<int> gidx;
    const char* msg = layout_plan(pl, ncell, 148, ng, nh, hsep, need, n_out, rows, gidx, sing_g, opts);
    if (msg && !must) return;
    REQUIRE(msg == nullptr, "layout_plan: %s", msg ? msg : "");
    const Params& P = pl.base;
    REQUIRE(pl.smem <= 227 * 1024, "shared memory %zu", pl.smem);
    REQUIRE(P.s_chunks <= 256 * kBloItems, "B_lo chunks %d", P.s_chunks);
    REQUIRE(P.slot_bytes % 1024 == 0 && P.off_b % 1024 == 0, "slot / B_lo stage not 1024-aligned");
    REQUIRE(pl.ngroups >= 1 && pl.ngroups <= kMaxGroups, "groups %d", pl.ngroups);
    // singles region: the h rows when they are separate (unless the singles are the g rows), else the g rows
    const int grows = (ng + 7) / 8 * 8;
    REQUIRE(P.s_off == ((hsep && !sing_g) ? grows * 128 : 0), "singles region offset %d", P.s_off);
    REQUIRE(P.slot_bytes == (grows + (hsep ? (nh + 7) / 8 * 8 : 0)) * 128, "slot bytes %d", P.slot_bytes);
    REQUIRE((long)pl.ncta * pl.cells_cta >= ncell && pl.cells_cta % kSlotCells == 0, "cell split");
    int units = 0;
    for (int gi = 0; gi < pl.ngroups; ++gi) {
        const GroupDesc& D = P.grp[gi];
        REQUIRE(D.ntiles >= 1 && D.ntiles <= kMaxTiles, "group %d: %d tiles", gi, D.ntiles);
        REQUIRE(D.nA >= 2 && D.nA <= kMaxAStages, "group %d: %d A stages", gi, D.nA);
        REQUIRE(kDBuf * D.d_cols + D.nA * 64 * D.ntiles <= 512, "group %d: tensor memory over 512 columns", gi);
        REQUIRE(D.a_col0 == kDBuf * D.d_cols, "group %d: A ring does not follow the accumulators", gi);
        REQUIRE(D.unit_base == units, "group %d: unit base", gi);
        int wsum = 0;
        std::vector<std::pair<int, int>> acc;
        for (int t = 0; t < D.ntiles; ++t) {
            const int W = D.tile_w[t];
            REQUIRE(W == 16 || W == 32, "tile width %d", W);
            REQUIRE(D.tile_s0[t] % 8 == 0 && D.tile_s0[t] >= 0, "window start %d", D.tile_s0[t]);
            REQUIRE(D.dm_col[t] % (2 * W) == 0, "accumulator of tile %d not aligned to its size", t);
            acc.push_back({D.dm_col[t], D.dm_col[t] + 2 * W});
            wsum += W;
        }
        std::sort(acc.begin(), acc.end());
        for (size_t i = 0; i + 1 < acc.size(); ++i) REQUIRE(acc[i].second <= acc[i + 1].first, "accumulators overlap");
        REQUIRE(acc.back().second <= D.d_cols && D.d_cols % 32 == 0, "accumulator columns");
        REQUIRE(D.nunits == wsum / 16 && D.nunits <= kMaxUnits, "units %d for windows %d", D.nunits, wsum);
        REQUIRE(D.bstage_bytes == P.s_chunks * 16, "B_lo stage size");
        units += D.nunits;
    }
    REQUIRE(units == pl.total_units, "total units");
    // every output exactly once, at a (unit, column, row) that holds its pair and single
    REQUIRE((int)gidx.size() >= n_out, "gather index size");
    std::set<int> seen;
    for (int o = 0; o < n_out; ++o) {
        const int g = gidx[o];
        REQUIRE(seen.insert(g).second, "output %d shares its slot", o);
        const int gu = g / 2048, col = (g / 128) % 16, r = g % 128;
        int gi = 0;
        while (gi + 1 < pl.ngroups && gu >= P.grp[gi + 1].unit_base) ++gi;
        const GroupDesc& D = P.grp[gi];
        const int u = gu - D.unit_base;
        REQUIRE(u >= 0 && u < D.nunits, "output %d: unit %d", o, u);
        const int t = D.unit_tile[u], cc = D.unit_c[u] + col;
        REQUIRE(cc < D.tile_w[t], "output %d: column %d beyond the window", o, cc);
        const short2 jk = rows[(size_t)(D.tile0 + t) * 128 + r];
        const int s = D.tile_s0[t] + cc;
        auto w = want.find(o);
        REQUIRE(w != want.end(), "output %d not requested", o);
        REQUIRE(jk.x == std::get<0>(w->second) && jk.y == std::get<1>(w->second) && s == std::get<2>(w->second),
                "output %d: row (%d, %d) single %d, wanted (%d, %d) single %d", o, jk.x, jk.y, s,
                std::get<0>(w->second), std::get<1>(w->second), std::get<2>(w->second));
        REQUIRE(s < (sing_g ? ng : nh), "output %d: single %d out of range", o, s);
        REQUIRE(jk.x < grows + (hsep ? (nh + 7) / 8 * 8 : 0) && jk.y < grows + (hsep ? (nh + 7) / 8 * 8 : 0),
                "output %d: pair row beyond the slot", o);
    }
}

static void check(const char* name, long ncell, int ng, int nh, int hsep, std::vector<NeedPair> need, int n_out,
                  int sing_g = 0) {
    check_one(name, ncell, ng, nh, hsep, need, n_out, sing_g, PlanOpts{}, true);
    for (int cost : {8, 24})
        for (int cap : {kMaxTiles, 1})
            for (int mode : {0, 1, 2}) {
                PlanOpts o;
                o.tile_cost = cost;
                o.group_cap = cap;
                o.cta_mode = mode;
                check_one(name, ncell, ng, nh, hsep, need, n_out, sing_g, o, false);
            }
}

// all pairs j <= k of ng maps against nh singles (the general contraction)
static void full(long ncell, int ng, int nh, int hsep) {
    std::vector<NeedPair> need;
    int p = 0;
    for (int j = 0; j < ng; ++j)
        for (int k = j; k < ng; ++k, ++p) {
            NeedPair np{j, k, 0, nh - 1, {}};
            for (int i = 0; i < nh; ++i) np.outs.push_back({i, p * nh + i});
            need.push_back(std::move(np));
        }
    char name[64];
    std::snprintf(name, sizeof name, "full ng=%d nh=%d hsep=%d", ng, nh, hsep);
    check(name, ncell, ng, nh, hsep, std::move(need), p * nh);
}

// closed triplets a <= b <= c (closure c <= a + b + gap) read from pair (b, c) and single a
static void triplets(long ncell, int nb, int gap, const std::vector<int>* keep = nullptr) {
    std::map<std::pair<int, int>, NeedPair> m;
    int nt = 0;
    for (int a = 0; a < nb; ++a)
        for (int b = a; b < nb; ++b)
            for (int c = b; c < nb && c <= a + b + gap; ++c) {
                if (keep && !(*keep)[(a * 31 + b * 7 + c) % keep->size()]) continue;
                auto f = m.find({b, c});
                if (f == m.end()) f = m.emplace(std::make_pair(b, c), NeedPair{b, c, a, a, {}}).first;
                f->second.lo = std::min(f->second.lo, a);
                f->second.hi = std::max(f->second.hi, a);
                f->second.outs.push_back({a, nt++});
            }
    std::vector<NeedPair> need;
    for (auto& kv : m) need.push_back(std::move(kv.second));
    char name[64];
    std::snprintf(name, sizeof name, "triplets nb=%d gap=%d%s", nb, gap, keep ? " (subset)" : "");
    if (need.empty()) return;
    check(name, ncell, nb, nb, 0, std::move(need), nt);
}

// closed triplets for a multipole: pair (g_b, h_c) with h_c at slot row h0 + c, single g_a (singles = g rows)
static void ell_triplets(long ncell, int nb, int gap) {
    const int h0 = (nb + 7) / 8 * 8;
    std::map<std::pair<int, int>, NeedPair> m;
    int nt = 0;
    for (int a = 0; a < nb; ++a)
        for (int b = a; b < nb; ++b)
            for (int c = b; c < nb && c <= a + b + gap; ++c) {
                auto f = m.find({b, c});
                if (f == m.end()) f = m.emplace(std::make_pair(b, c), NeedPair{b, h0 + c, a, a, {}}).first;
                f->second.lo = std::min(f->second.lo, a);
                f->second.hi = std::max(f->second.hi, a);
                f->second.outs.push_back({a, nt++});
            }
    std::vector<NeedPair> need;
    for (auto& kv : m) need.push_back(std::move(kv.second));
    char name[64];
    std::snprintf(name, sizeof name, "ell triplets nb=%d gap=%d", nb, gap);
    if (need.empty()) return;
    check(name, ncell, nb, nb, 1, std::move(need), nt, 1);
}

int main() {
    int cases = 0;
    for (long ncell : {32L * 32 * 32, 512L * 512 * 512, 96L * 96 * 96}) {
        // every shape the tensor-core path accepts (ng (ng + 1) / 2 <= 512 pairs, nh <= 32 singles)
        for (int ng = 1; ng * (ng + 1) / 2 <= 512; ++ng) {
            if (ng <= 32) { full(ncell, ng, ng, 0); ++cases; }
            for (int nh : {1, 7, 16, 17, 32}) { full(ncell, ng, nh, 1); ++cases; }
        }
        for (int nb = 2; nb <= 32; ++nb)
            for (int gap : {0, 1, 2}) { triplets(ncell, nb, gap); ell_triplets(ncell, nb, gap); cases += 2; }
        std::mt19937 rng(12345);
        for (int rep = 0; rep < 40; ++rep) {
            std::vector<int> keep(37);
            for (int& x : keep) x = (rng() % 4) != 0;
            triplets(ncell, 8 + (int)(rng() % 25), 1, &keep);
            ++cases;
        }
    }
    std::printf("%d cases, %d failures\n", cases, n_fail);
    return n_fail ? 1 : 0;
}
