// sym_schedule.h -- host-side work lists of the symmetric pair pass (plain C++, no CUDA: the CPU tests
// compile it on its own).
//
// The symmetric pass evaluates every unordered pair of spheres once (Sec. II.B's mobility is
// reciprocal, M_ji = M_ij^T).  With the spheres in tiles of `tile`, the work is the upper triangle
// of (target tile b, source tile t >= b) units; a unit with t > b gives both target sums (row b) and
// source sums (column t), the diagonal unit b = t only target sums.
//   seg4:      (b, t0, t1, tag) per segment: row b, source tiles [t0, t1); segments of row b are
//              [row_seg[b], row_seg[b + 1]) and each writes one target partial
//   col_start: the source partial of unit (b, t), t > b, is slot col_start[t] + b
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace rpb {

// One suspension of N spheres, units [u0, u1) of the nb (nb + 1) / 2 in row-major order (all of them
// for the whole product; a contiguous share of them for one of several processes, each of which then
// holds a partial product): cut into runs of equal length L = ceil((u1 - u0) / (60 x SMs)) (the last
// one shorter), so at most 60 x SMs CTAs: about whole waves at 3 to 6 resident CTAs per SM; each run
// is split into segments at row ends.  cta4: (s0, s1, 0, 0) per CTA, segments [s0, s1); seg4 tags
// are 0; row_seg[b]: the first segment of a row >= b; col_start[t] = t (t - 1) / 2; col_rows[2t],
// col_rows[2t + 1]: the rows [r0, r1) whose source partials of column t the range writes (rows of a
// column come in increasing unit order, so they are contiguous; (0, t) for the whole triangle).
inline void sym_schedule_range(int64_t N, int num_sms, int tile, int64_t u0, int64_t u1, std::vector<int> &cta4,
                               std::vector<int> &seg4, std::vector<int> &row_seg, std::vector<int> &col_start,
                               std::vector<int> &col_rows)
{
    const int nb = (int)((N + tile - 1) / tile);
    const int64_t units = (int64_t)nb * (nb + 1) / 2;
    u0 = std::min(std::max<int64_t>(u0, 0), units);
    u1 = std::min(std::max(u1, u0), units);
    const int64_t nu = u1 - u0;
    const int64_t ncta = std::min<int64_t>(nu, 60 * (int64_t)num_sms);
    const int64_t L = ncta > 0 ? (nu + ncta - 1) / ncta : 0;
    cta4.clear();
    seg4.clear();
    row_seg.assign(nb + 1, 0);
    col_start.assign(nb, 0);
    col_rows.assign(2 * (size_t)nb, 0);
    for (int t = 0; t < nb; ++t) col_start[t] = (int)((int64_t)t * (t - 1) / 2);
    // (b, t) of unit u0: row b holds nb - b units
    int b = 0;
    int64_t rest = u0;
    while (b < nb && rest >= nb - b) {
        rest -= nb - b;
        ++b;
    }
    int t = b + (int)rest, nseg = 0;
    int64_t left = nu;
    while (left > 0) {
        int64_t k = std::min(L, left);
        left -= k;
        cta4.push_back(nseg);
        while (k > 0) {
            const int m = (int)std::min<int64_t>(k, nb - t);
            seg4.push_back(b);
            seg4.push_back(t);
            seg4.push_back(t + m);
            seg4.push_back(0);
            ++nseg;
            for (int c = std::max(t, b + 1); c < t + m; ++c) {
                if (col_rows[2 * c + 1] == 0) col_rows[2 * c] = b;
                col_rows[2 * c + 1] = b + 1;
            }
            t += m;
            k -= m;
            if (t == nb) {
                ++b;
                t = b;
            }
        }
        cta4.push_back(nseg);
        cta4.push_back(0);
        cta4.push_back(0);
    }
    for (int r = 0, q = 0; r <= nb; ++r) {
        while (q < nseg && seg4[4 * q] < r) ++q;
        row_seg[r] = q;
    }
}

// Units [u0, u1) of share `part` of `nparts` equal contiguous shares of the triangle of N spheres.
inline void sym_part_units(int64_t N, int tile, int part, int nparts, int64_t *u0, int64_t *u1)
{
    const int64_t nb = (N + tile - 1) / tile;
    const int64_t units = nb * (nb + 1) / 2;
    *u0 = units * part / nparts;
    *u1 = units * (part + 1) / nparts;
}

// The whole triangle (the single-process product).
inline void sym_schedule(int64_t N, int num_sms, int tile, std::vector<int> &cta4, std::vector<int> &seg4,
                         std::vector<int> &row_seg, std::vector<int> &col_start)
{
    std::vector<int> col_rows;
    sym_schedule_range(N, num_sms, tile, 0, INT64_MAX, cta4, seg4, row_seg, col_start, col_rows);
}

// Many suspensions packed one after another (suspension k at spheres [off_k, off_k + N_k), its tiles
// numbered from tile0_k).  Every suspension's rows are cut by a fixed rule, runs of at most seg_tiles
// tiles, so that the partial sums a suspension's result is made of do not depend on its companions;
// one CTA per run, longest runs first (cta_order).  The seg4 tag is the suspension; tile_inst maps a
// tile to its suspension; col_start[t] + b is the source-partial slot of unit (b, t) with the rows of
// a column counted from its suspension's first tile; n_src_slots is the number of those slots.
struct BatchSchedule {
    std::vector<int64_t> off;
    std::vector<int> n, tile0;
    std::vector<int> seg4, row_seg, col_start, tile_inst, cta_order;
    int64_t n_src_slots = 0;
    int ntiles = 0;
};

inline void batch_sym_schedule(int B, const int64_t *N, int tile, int seg_tiles, BatchSchedule &s)
{
    s = BatchSchedule();
    s.off.resize(B);
    s.n.resize(B);
    s.tile0.resize(B);
    int64_t off = 0;
    int g = 0;
    for (int k = 0; k < B; ++k) {
        const int nb = (int)((N[k] + tile - 1) / tile);
        s.off[k] = off;
        s.n[k] = (int)N[k];
        s.tile0[k] = g;
        for (int r = 0; r < nb; ++r) {
            s.row_seg.push_back((int)(s.seg4.size() / 4));
            s.tile_inst.push_back(k);
            for (int t0 = g + r; t0 < g + nb; t0 += seg_tiles) {
                s.seg4.push_back(g + r);
                s.seg4.push_back(t0);
                s.seg4.push_back(std::min(g + nb, t0 + seg_tiles));
                s.seg4.push_back(k);
            }
            s.col_start.push_back((int)(s.n_src_slots - g));  // slot of row b in column g + r: col_start + b
            s.n_src_slots += r;
        }
        off += N[k];
        g += nb;
    }
    const int nseg = (int)(s.seg4.size() / 4);
    s.row_seg.push_back(nseg);
    s.ntiles = g;
    s.cta_order.resize(nseg);
    for (int q = 0; q < nseg; ++q) s.cta_order[q] = q;
    const std::vector<int> &seg4 = s.seg4;
    std::stable_sort(s.cta_order.begin(), s.cta_order.end(), [&](int x, int y) {
        return seg4[4 * x + 2] - seg4[4 * x + 1] > seg4[4 * y + 2] - seg4[4 * y + 1];
    });
}

}  // namespace rpb
