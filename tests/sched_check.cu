// Host-only check of the tensor-core pass schedules (sched.cuh): for many pass shapes and CTA
// counts, every (unit, k-block) is processed exactly once, every CTA writes at most its two
// partial slots, and the fix-up's view (split_owners / split_slot) names exactly the CTAs and
// slots that hold each split unit's parts.  Exit status 0 when every shape passes.
//
//   nvcc -std=c++17 -O2 -I paper_1606_09402_gb300/csrc -o sched_check tests/sched_check.cu
//   ./sched_check
#include <cstdio>
#include <map>
#include <vector>

#include "sched.cuh"

using namespace qb;

static int g_fail = 0;
#define CHECK(cond, ...)                                   \
    do {                                                   \
        if (!(cond)) {                                     \
            if (g_fail < 20) {                             \
                std::printf("FAIL %s: ", #cond);           \
                std::printf(__VA_ARGS__);                  \
                std::printf("\n");                         \
            }                                              \
            ++g_fail;                                      \
        }                                                  \
    } while (0)

struct Part {
    int u, k0, k1;
};

static void check(int64_t M, int64_t N, int64_t K, int bn, int sms, int mode_count[3]) {
    const Sched s = make_sched(M, N, K, bn, sms);
    const int G = grid_size(s, sms);
    const int units = s.tiles_m * s.tiles_n;
    mode_count[s.streamk]++;
    CHECK(G >= 1, "M=%lld N=%lld K=%lld bn=%d sms=%d", (long long)M, (long long)N, (long long)K,
          bn, sms);
    if (s.streamk) CHECK(G <= TC_MAX_SK_CTAS, "split launch of %d CTAs", G);
    if (s.streamk == 2) {
        CHECK(G == std::min(sms, TC_MAX_SK_CTAS), "hybrid grid %d", G);
        CHECK(s.dp_units > 0 && s.dp_units % G == 0 && s.dp_units < units,
              "hybrid dp_units %d units %d G %d", s.dp_units, units, G);
    }
    std::vector<int> cover(size_t(units) * s.kb, 0);
    std::vector<int> direct(units, 0);
    std::map<std::pair<int, int>, Part> parts;   // (cta, slot) -> part
    for (int cta = 0; cta < G; ++cta) {
        SegWalk wk(s, cta, G);
        Seg sg;
        int guard = 0;
        while (wk.next(sg)) {
            CHECK(++guard <= units + 2, "walk does not end (cta %d)", cta);
            if (guard > units + 2) break;
            CHECK(sg.u >= 0 && sg.u < units && sg.k0 >= 0 && sg.k0 < sg.k1 && sg.k1 <= s.kb,
                  "segment u=%d k=[%d,%d) units=%d kb=%d", sg.u, sg.k0, sg.k1, units, s.kb);
            if (!(sg.u >= 0 && sg.u < units && sg.k0 >= 0 && sg.k1 <= s.kb)) continue;
            for (int k = sg.k0; k < sg.k1; ++k) cover[size_t(sg.u) * s.kb + k]++;
            if (sg.slot < 0) {
                CHECK(sg.k0 == 0 && sg.k1 == s.kb, "whole segment not whole");
                direct[sg.u]++;
            } else {
                CHECK(sg.slot <= 1, "slot %d", sg.slot);
                CHECK(!parts.count({cta, sg.slot}), "cta %d writes slot %d twice", cta, sg.slot);
                parts[{cta, sg.slot}] = Part{sg.u, sg.k0, sg.k1};
            }
        }
    }
    for (size_t i = 0; i < cover.size(); ++i)
        CHECK(cover[i] == 1, "unit %d k-block %d covered %d times (mode %d)", int(i / s.kb),
              int(i % s.kb), cover[i], s.streamk);
    // the fix-up's view
    const int u0 = s.streamk ? split_first_unit(s) : units;
    for (int u = 0; u < units; ++u) {
        if (u < u0) {
            CHECK(direct[u] == 1, "raster unit %d written %d times", u, direct[u]);
            continue;
        }
        const int64_t ur = u - u0;
        int64_t c_first;
        int count;
        split_owners(s, ur, G, c_first, count);
        int n_parts = 0;
        for (auto& kv : parts) n_parts += kv.second.u == u;
        if (count == 0) {
            CHECK(direct[u] == 1 && n_parts == 0, "unit %d: count 0, direct %d, parts %d", u,
                  direct[u], n_parts);
            continue;
        }
        CHECK(direct[u] == 0 && n_parts == count, "unit %d: count %d, direct %d, parts %d", u,
              count, direct[u], n_parts);
        int covered = 0;
        for (int t = 0; t < count; ++t) {
            const int64_t c = c_first + t;
            const int slot = split_slot(s, ur, c, G);
            auto it = parts.find({int(c), slot});
            CHECK(it != parts.end() && it->second.u == u, "unit %d: cta %lld slot %d missing", u,
                  (long long)c, slot);
            if (it != parts.end() && it->second.u == u) covered += it->second.k1 - it->second.k0;
        }
        CHECK(covered == s.kb, "unit %d: fix-up covers %d of %d k-blocks", u, covered, s.kb);
    }
    if (s.streamk) CHECK(split_units(s) == units - u0, "split units");
}

int main() {
    int modes[3] = {0, 0, 0};
    int shapes = 0;
    const int sms_list[] = {1, 2, 3, 8, 148, 152, 160, 192};
    const int bn_list[] = {64, 128, 256};
    const int64_t mn_list[] = {1, 64, 127, 128, 129, 640, 5000, 19999, 20000, 40000, 70000};
    const int64_t k_list[] = {1, 63, 64, 65, 1000, 20000, 40000};
    for (int sms : sms_list)
        for (int bn : bn_list)
            for (int64_t M : mn_list)
                for (int64_t N : {int64_t(1), int64_t(64), int64_t(200), int64_t(512),
                                  int64_t(3200)})
                    for (int64_t K : k_list) {
                        if (M * N > int64_t(3e8) && K > 1000) continue;   // keep it quick
                        check(M, N, K, bn, sms, modes);
                        ++shapes;
                    }
    // the passes of the 40000 x 20000 step, explicitly
    check(20000, 512, 40000, 128, 152, modes);   // H chunk: 628 units
    check(40000, 512, 20000, 256, 152, modes);   // sketch chunk
    check(20000, 512, 40000, 256, 152, modes);   // power-step transposed chunk
    shapes += 3;
    // Q^T [Q_i | Y_i] of a randQB_FP block (M = rank so far, N = 2 b_i, K = m; 128-wide tile when
    // N > 64), and the fixed-rank map's Gram-Schmidt products (M = j0, N = 64, K = m)
    for (int64_t M : {int64_t(1), int64_t(64), int64_t(200), int64_t(700), int64_t(1439)})
        for (int64_t N : {int64_t(40), int64_t(100), int64_t(128)}) {
            check(M, N, 40000, N > 64 ? 128 : 64, 152, modes);
            ++shapes;
        }
    for (int64_t M : {int64_t(64), int64_t(128), int64_t(192)}) {
        check(M, 64, 8192, 64, 152, modes);
        ++shapes;
    }
    std::printf("%d shapes: raster %d, stream-K %d, hybrid %d; %d failures\n", shapes, modes[0],
                modes[1], modes[2], g_fail);
    return g_fail == 0 && modes[2] > 0 ? 0 : 1;
}
