// Prints the work lists of the symmetric pair pass (sym_schedule.h) as JSON for
// tests/test_schedule_cpu.py.  usage: schedule_dump single N num_sms | schedule_dump part N num_sms part
// nparts | schedule_dump batch N0 N1 ... | schedule_dump noalloc max_N max_sms max_partial_elems fp64
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "grid_plan.h"
#include "sym_schedule.h"

static void dump(const char *name, const std::vector<int> &v, bool last = false)
{
    std::printf("\"%s\": [", name);
    for (size_t i = 0; i < v.size(); ++i) std::printf(i ? ",%d" : "%d", v[i]);
    std::printf("]%s", last ? "" : ", ");
}

int main(int argc, char **argv)
{
    const int tile = 128;
    if (argc >= 6 && std::strcmp(argv[1], "noalloc") == 0) {
        // noalloc max_N max_sms max_partial_elems fp64: every (N, SM count) plan, one line each when it
        // breaks a bound ("N sms splits chunk"), then "ok" or "bad"
        const long long maxN = std::atoll(argv[2]);
        const int maxs = std::atoi(argv[3]);
        const long long cap = std::atoll(argv[4]);
        const bool fp64 = std::atoi(argv[5]) != 0;
        long long bad = 0;
        for (long long N = 1; N <= maxN; ++N)
            for (int sms = 1; sms <= maxs; sms += (sms < 160 ? 1 : 37)) {
                int splits = 0;
                int64_t chunk = 0;
                rpb::noalloc_grid_plan(N, sms, fp64, tile, cap, &splits, &chunk);
                const bool ok = splits >= 1 && (long long)splits * 3 * N <= cap && chunk % (fp64 ? 4 : tile) == 0 &&
                                (long long)splits * chunk >= N && (long long)(splits - 1) * chunk < N;
                if (!ok && bad++ < 20) std::printf("%lld %d %d %lld\n", N, sms, splits, (long long)chunk);
            }
        std::printf(bad ? "bad\n" : "ok\n");
        return 0;
    }
    if (argc >= 6 && std::strcmp(argv[1], "part") == 0) {
        // part N num_sms part nparts: the schedule of one share of the triangle
        std::vector<int> cta4, seg4, row_seg, col_start, col_rows;
        int64_t u0, u1;
        const long long N = std::atoll(argv[2]);
        rpb::sym_part_units(N, tile, std::atoi(argv[4]), std::atoi(argv[5]), &u0, &u1);
        rpb::sym_schedule_range(N, std::atoi(argv[3]), tile, u0, u1, cta4, seg4, row_seg, col_start, col_rows);
        std::printf("{\"u0\": %lld, \"u1\": %lld, ", (long long)u0, (long long)u1);
        dump("cta4", cta4);
        dump("seg4", seg4);
        dump("row_seg", row_seg);
        dump("col_start", col_start);
        dump("col_rows", col_rows, true);
        std::printf("}\n");
        return 0;
    }
    if (argc >= 4 && std::strcmp(argv[1], "single") == 0) {
        std::vector<int> cta4, seg4, row_seg, col_start;
        rpb::sym_schedule(std::atoll(argv[2]), std::atoi(argv[3]), tile, cta4, seg4, row_seg, col_start);
        std::printf("{");
        dump("cta4", cta4);
        dump("seg4", seg4);
        dump("row_seg", row_seg);
        dump("col_start", col_start, true);
        std::printf("}\n");
        return 0;
    }
    if (argc >= 3 && std::strcmp(argv[1], "batch") == 0) {
        std::vector<int64_t> N;
        for (int i = 2; i < argc; ++i) N.push_back(std::atoll(argv[i]));
        rpb::BatchSchedule s;
        rpb::batch_sym_schedule((int)N.size(), N.data(), tile, 8, s);
        std::printf("{\"tile0\": [");
        for (size_t i = 0; i < s.tile0.size(); ++i) std::printf(i ? ",%d" : "%d", s.tile0[i]);
        std::printf("], \"n_src_slots\": %lld, \"ntiles\": %d, ", (long long)s.n_src_slots, s.ntiles);
        dump("seg4", s.seg4);
        dump("row_seg", s.row_seg);
        dump("col_start", s.col_start);
        dump("tile_inst", s.tile_inst);
        dump("cta_order", s.cta_order, true);
        std::printf("}\n");
        return 0;
    }
    std::fprintf(stderr, "usage: schedule_dump single N num_sms | schedule_dump batch N0 N1 ...\n");
    return 2;
}
