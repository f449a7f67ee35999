// grid_plan.h -- source-chunk plans of the one-way pair kernels (host logic, no CUDA), so that the
// tests can compile and check them on the CPU.
//
// A one-way product splits the N sources of every target block into `splits` chunks of `chunk`
// sources on grid.y; each chunk writes one float64 partial per (chunk, target, component), which a
// reduce kernel adds in a fixed order (Sec. II.B's direct summation, spread over the whole GPU).
#pragma once

#include <algorithm>
#include <cstdint>

namespace rpb {

constexpr int64_t kMaxSplitsF32 = 16;  // source chunks of a float32 one-way product

inline int64_t target_blocks(int num_sms)
{
    return (int64_t)num_sms * 8;
}

// Split of a product over N spheres into source chunks.  fp64: chunks of any multiple of 4 sources,
// enough of them to spread even a small product over every SM (float64 runs at a small fraction of
// the float32 rate on this part).  float32: whole tiles of `tile` sources; with slots > 0 (the CTAs
// resident on the whole GPU at once) the split count minimising (waves) x (chunk length), a larger
// one only if it saves over 1%; otherwise about target_blocks CTAs.
inline void pair_grid_plan(int64_t N, int num_sms, bool fp64, int slots, int64_t tile, int *splits, int64_t *chunk)
{
    const int64_t tiles = (N + tile - 1) / tile;
    int64_t S = (target_blocks(num_sms) + tiles - 1) / tiles;
    if (fp64) {
        if (S > (N + 3) / 4) S = (N + 3) / 4;
        if (S < 1) S = 1;
        const int64_t ch = ((N + S - 1) / S + 3) / 4 * 4;
        *chunk = ch;
        *splits = (int)((N + ch - 1) / ch);
        return;
    }
    auto chunk_of = [&](int64_t s) { return std::max<int64_t>(tile, ((N + s - 1) / s + tile - 1) / tile * tile); };
    if (slots > 0) {
        auto cost = [&](int64_t s) {
            const int64_t ch = chunk_of(s), sp = (N + ch - 1) / ch;
            return (double)((tiles * sp + slots - 1) / slots) * (double)ch;
        };
        const int64_t smax = std::min<int64_t>(kMaxSplitsF32, tiles);
        S = 1;
        double best = cost(1);
        for (int64_t s2 = 2; s2 <= smax; ++s2) {
            const double l = cost(s2);
            if (l < 0.99 * best) {
                best = l;
                S = s2;
            }
        }
    } else {
        if (S > tiles) S = tiles;
        if (S < 1) S = 1;
    }
    *chunk = chunk_of(S);
    *splits = (int)((N + *chunk - 1) / *chunk);
}

// Split of a product restricted to nt target rows (all N sources): about target_blocks CTAs in all,
// source chunks of whole tiles (float32) or multiples of 4 sources (float64).
inline void rows_grid_plan(int64_t nt, int64_t N, int num_sms, bool fp64, int64_t tile, int *splits, int64_t *chunk)
{
    const int64_t tblocks = (nt + tile - 1) / tile;
    const int64_t q = fp64 ? 4 : tile;
    int64_t S = (target_blocks(num_sms) + tblocks - 1) / tblocks;
    const int64_t smax = (N + q - 1) / q;
    if (S > smax) S = smax;
    if (S < 1) S = 1;
    *chunk = ((N + S - 1) / S + q - 1) / q * q;
    *splits = (int)((N + *chunk - 1) / *chunk);
}

// The split of the allocation-free product: pair_grid_plan without occupancy slots, then at most
// max_partial_elems / (3N) chunks (its partial sums live in a fixed array of max_partial_elems
// doubles); chunks stay whole tiles.
inline void noalloc_grid_plan(int64_t N, int num_sms, bool fp64, int64_t tile, int64_t max_partial_elems,
                              int *splits, int64_t *chunk)
{
    pair_grid_plan(N, num_sms, fp64, 0, tile, splits, chunk);
    const int64_t max_splits = max_partial_elems / (3 * N);
    if (*splits > max_splits) {
        *chunk = ((N + max_splits - 1) / max_splits + tile - 1) / tile * tile;
        *splits = (int)((N + *chunk - 1) / *chunk);
    }
}

}  // namespace rpb
