// pair.cu -- the all-pairs Rotne-Prager-Blake product U = M_tt F + M_tr T (and the force kernel).
//
// Mobility (Sec. II.B Eq. mobilityDifferential / mobilityOverlap, Sec. III Eq.
// mobilityDifferentialTR, Appendix A Eq. effMob):
//   M_ij = s_i s_j Mtilde(q~_i, q~_j),  s = H0(z/a),  q~ = (x, y, max(z, a)),
//   Mtilde = free-space RPY (overlap branch for r < 2a) + wall correction.
// The wall correction is the Faxen-operated image system of Blake's half-space Green's function,
// written in closed form on the basis {I, e e, e z, z e, z z} (translation) and
// {T x e, T x z, e (z x e).T, z (z x e).T} (rotation), with R = x_i - x_j* (source mirrored in
// the wall), e = R/|R|, t = z~_j/|R|, s = a^2/|R|^2.  The coefficients were obtained by
// decomposing the Faxen-operated image tensors onto that basis; they reproduce the published
// near-wall self mobilities 1 - 9/(16h) + 1/(8h^3) - 1/(16h^5) and 1 - 9/(8h) + 1/(2h^3) - 1/(8h^5).
//
// Kernel design (GB300, CUDA cores -- the pair work is not a dense contraction):
//   - one target per thread, 128 targets per block, sources staged 128 at a time in shared
//     memory (every thread reads the same source: broadcast, no bank conflicts);
//   - the source range is split into chunks (grid.y) so that small N still fills all SMs; each
//     (target block, chunk) writes a float64 partial, summed in fixed order by the reduce kernel
//     (deterministic, no atomics);
//   - the self pair (j == i) is excluded from the pair loop (only the block's diagonal tile pays
//     for the test) and added in float64 by the reduce kernel, which also applies s_i/(8 pi eta);
//   - float32 mode: positions split x = x_hi + x_lo (two floats), so near-pair offsets keep float32
//     relative accuracy anywhere in a large box; per-tile float32 sums are added with Kahan
//     compensation.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <vector>

#include "grid_plan.h"
#include "pair_math.cuh"
#include "sym_schedule.h"

namespace rpb {

// ------------------------------------------------------------------ packing
__global__ void pack_f32_kernel(const double *__restrict__ pos, const double *__restrict__ F,
                                const double *__restrict__ T, int N, double a, int wall, SrcF32 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double x = pos[i], y = pos[N + i], z = pos[2 * N + i];
    const double s = wall ? H0(z / a) : 1.0;
    const float xh = (float)x, yh = (float)y;
    SrcF32 o;
    o.p = make_float4(xh, yh, (float)(x - (double)xh), (float)(y - (double)yh));
    o.f = make_float4((float)(wall ? fmax(z, a) : z), F ? (float)(s * F[i]) : 0.f, F ? (float)(s * F[N + i]) : 0.f,
                      F ? (float)(s * F[2 * N + i]) : 0.f);
    o.t = make_float4(T ? (float)(s * T[i]) : 0.f, T ? (float)(s * T[N + i]) : 0.f, T ? (float)(s * T[2 * N + i]) : 0.f,
                      0.f);
    out[i] = o;
}

// Second right-hand side of the two-RHS symmetric pass: s_j P_j as float32 (x, y, z, 0).
__global__ void pack_rhs2_kernel(const double *__restrict__ pos, const double *__restrict__ P, int N, double a,
                                 float4 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double s = H0(pos[2 * N + i] / a);
    out[i] = make_float4((float)(s * P[i]), (float)(s * P[N + i]), (float)(s * P[2 * N + i]), 0.f);
}

__global__ void pack_f64_kernel(const double *__restrict__ pos, const double *__restrict__ F,
                                const double *__restrict__ T, int N, double a, int wall, SrcF64 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double z = pos[2 * N + i];
    const double s = wall ? H0(z / a) : 1.0;
    SrcF64 o;
    o.p = make_double2(pos[i], pos[N + i]);
    o.q = make_double2(wall ? fmax(z, a) : z, F ? s * F[i] : 0.0);
    o.r = make_double2(F ? s * F[N + i] : 0.0, F ? s * F[2 * N + i] : 0.0);
    o.s = make_double2(T ? s * T[i] : 0.0, T ? s * T[N + i] : 0.0);
    o.u = make_double2(T ? s * T[2 * N + i] : 0.0, 0.0);
    out[i] = o;
}

// ------------------------------------------------------------------ pair kernels
// grid = (ceil(N/128), splits); block (bx, by) covers targets [128 bx, 128 bx + 128) and sources
// [by chunk, (by + 1) chunk); chunk is a multiple of 128, so the tile holding the block's own
// targets (where j == i can occur) is the one starting at 128 bx.
template <bool TORQUE, bool WALL = true>
__global__ void __launch_bounds__(kPairThreads) pair_f32_kernel(const SrcF32 *__restrict__ src, int N, int chunk,
                                                                 PairConsts<float> c, double *__restrict__ part)
{
    __shared__ float4 sp[kTile];
    __shared__ float4 sf[kTile];
    __shared__ float4 st[TORQUE ? kTile : 1];
    const int tid = threadIdx.x;
    const int i = blockIdx.x * kPairThreads + tid;
    const int j0 = blockIdx.y * chunk;
    const int j1 = min(N, j0 + chunk);
    float4 tp = make_float4(0.f, 0.f, 0.f, 0.f);
    float tz = 1.f;
    if (i < N) {
        tp = src[i].p;
        tz = src[i].f.x;
    }
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    const int diag = blockIdx.x * kTile;
    for (int base = j0; base < j1; base += kTile) {
        const int j = base + tid;
        if (j < j1) {
            sp[tid] = src[j].p;
            sf[tid] = src[j].f;
            if (TORQUE) st[tid] = src[j].t;
        }
        __syncthreads();
        const int cnt = min(kTile, j1 - base);
        float ux = 0.f, uy = 0.f, uz = 0.f;
        if (base != diag) {
#pragma unroll 4
            for (int k = 0; k < cnt; ++k) {
                const float4 p = sp[k];
                const float4 f = sf[k];
                const float4 q = TORQUE ? st[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float rx = (tp.x - p.x) + (tp.z - p.z);
                const float ry = (tp.y - p.y) + (tp.w - p.w);
                pair_velocity_f32<TORQUE, WALL>(rx, ry, tz, f.x, f.y, f.z, f.w, q.x, q.y, q.z, c, ux, uy, uz);
            }
        } else {
            for (int k = 0; k < cnt; ++k) {
                const float4 p = sp[k];
                const float4 f = sf[k];
                const float4 q = TORQUE ? st[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float rx = (tp.x - p.x) + (tp.z - p.z);
                const float ry = (tp.y - p.y) + (tp.w - p.w);
                float dx = 0.f, dy = 0.f, dz = 0.f;
                pair_velocity_f32<TORQUE, WALL>(rx, ry, tz, f.x, f.y, f.z, f.w, q.x, q.y, q.z, c, dx, dy, dz);
                if (k != tid) {
                    ux += dx;
                    uy += dy;
                    uz += dz;
                }
            }
        }
        // compensated (Kahan) accumulation of the tile sums
        {
            float yv = ux - cx, tv = sx + yv;
            cx = (tv - sx) - yv;
            sx = tv;
            yv = uy - cy;
            tv = sy + yv;
            cy = (tv - sy) - yv;
            sy = tv;
            yv = uz - cz;
            tv = sz + yv;
            cz = (tv - sz) - yv;
            sz = tv;
        }
        __syncthreads();
    }
    if (i < N) {
        const size_t o = (size_t)blockIdx.y * 3 * N;
        part[o + i] = (double)sx - (double)cx;
        part[o + N + i] = (double)sy - (double)cy;
        part[o + 2 * N + i] = (double)sz - (double)cz;
    }
}

// Float32 pair pass evaluating two sources per lane and iteration with packed float32x2 arithmetic.
// The shared tile holds the 128 sources as 64 interleaved pairs: float4 (x_hi[2p], x_hi[2p+1],
// y_hi[2p], y_hi[2p+1]), (x_lo.., y_lo..), (z~.., Fx..), (Fy.., Fz..), and for torques (Tx.., Ty..)
// and (Tz[2p], Tz[2p+1]).  Slots past the chunk's end hold a distant source with zero load, whose
// contribution is exactly zero, so every tile is a full 64 iterations.
// Targets t0 .. t0 + nt - 1 (t0 a multiple of kTile; nt < 0: all N), partials indexed by i - t0.
template <bool TORQUE>
__global__ void __launch_bounds__(kPairThreads, 6) pair_f32x2_kernel(const SrcF32 *__restrict__ src, int N, int chunk,
                                                                   X2Consts c, double *__restrict__ part, int t0 = 0,
                                                                   int nt = -1)
{
    constexpr int P = kTile / 2;
    __shared__ float4 sA[P], sB[P], sC[P], sD[P];
    __shared__ float4 sE[TORQUE ? P : 1];
    __shared__ float2 sG[TORQUE ? P : 1];
    if (nt < 0) nt = N;
    const int tid = threadIdx.x;
    const int li = blockIdx.x * kPairThreads + tid;
    const int i = t0 + li;
    const bool live = li < nt && i < N;
    const int j0 = blockIdx.y * chunk;
    const int j1 = min(N, j0 + chunk);
    float4 tp = make_float4(0.f, 0.f, 0.f, 0.f);
    float tz = 1.f;
    if (live) {
        tp = src[i].p;
        tz = src[i].f.x;
    }
    const float2 txh = make_float2(tp.x, tp.x), tyh = make_float2(tp.y, tp.y);
    const float2 txl = make_float2(tp.z, tp.z), tyl = make_float2(tp.w, tp.w);
    const float2 tz2 = make_float2(tz, tz);
    const float2 zero2 = make_float2(0.f, 0.f);
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    const int diag = t0 + blockIdx.x * kTile;
    const int pp = tid >> 1, hh = tid & 1;
    float *fA = reinterpret_cast<float *>(sA);
    float *fB = reinterpret_cast<float *>(sB);
    float *fC = reinterpret_cast<float *>(sC);
    float *fD = reinterpret_cast<float *>(sD);
    float *fE = reinterpret_cast<float *>(sE);
    float *fG = reinterpret_cast<float *>(sG);
    for (int base = j0; base < j1; base += kTile) {
        const int j = base + tid;
        float4 sp_ = make_float4(1e18f, 0.f, 0.f, 0.f), sf_ = make_float4(1.f, 0.f, 0.f, 0.f);
        float4 st_ = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < j1) {
            sp_ = src[j].p;
            sf_ = src[j].f;
            if (TORQUE) st_ = src[j].t;
        }
        fA[4 * pp + hh] = sp_.x;
        fA[4 * pp + 2 + hh] = sp_.y;
        fB[4 * pp + hh] = sp_.z;
        fB[4 * pp + 2 + hh] = sp_.w;
        fC[4 * pp + hh] = sf_.x;
        fC[4 * pp + 2 + hh] = sf_.y;
        fD[4 * pp + hh] = sf_.z;
        fD[4 * pp + 2 + hh] = sf_.w;
        if (TORQUE) {
            fE[4 * pp + hh] = st_.x;
            fE[4 * pp + 2 + hh] = st_.y;
            fG[2 * pp + hh] = st_.z;
        }
        __syncthreads();
        float2 ux = zero2, uy = zero2, uz = zero2;
        if (base != diag) {
#pragma unroll 2
            for (int k = 0; k < P; ++k) {
                const float4 a = sA[k], cc = sC[k], d = sD[k];
                const float4 e = TORQUE ? sE[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float2 g = TORQUE ? sG[k] : zero2;
                const float2 zj = make_float2(cc.x, cc.y);
                float2 rx, ry, rz, rho2, r2;
                const bool close = pair_offsets_x2(txh, tyh, txl, tyl, tz2, zj, a, &sB[k], c, rx, ry, rz, rho2, r2);
                pair_velocity_x2_geo<TORQUE>(rx, ry, rz, rho2, r2, close, tz2, zj, make_float2(cc.z, cc.w),
                                             make_float2(d.x, d.y), make_float2(d.z, d.w), make_float2(e.x, e.y),
                                             make_float2(e.z, e.w), g, c, ux, uy, uz);
            }
        } else {
            for (int k = 0; k < P; ++k) {
                const float4 a = sA[k], b = sB[k], cc = sC[k], d = sD[k];
                const float4 e = TORQUE ? sE[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float2 g = TORQUE ? sG[k] : zero2;
                const float2 rx = add2(sub2(txh, make_float2(a.x, a.y)), sub2(txl, make_float2(b.x, b.y)));
                const float2 ry = add2(sub2(tyh, make_float2(a.z, a.w)), sub2(tyl, make_float2(b.z, b.w)));
                float2 dx = zero2, dy = zero2, dz = zero2;
                pair_velocity_x2<TORQUE>(rx, ry, tz2, make_float2(cc.x, cc.y), make_float2(cc.z, cc.w),
                                         make_float2(d.x, d.y), make_float2(d.z, d.w), make_float2(e.x, e.y),
                                         make_float2(e.z, e.w), g, c, dx, dy, dz);
                if (k == pp) {  // source 2k + hh is this thread's own sphere
                    if (hh == 0) {
                        dx.x = 0.f;
                        dy.x = 0.f;
                        dz.x = 0.f;
                    } else {
                        dx.y = 0.f;
                        dy.y = 0.f;
                        dz.y = 0.f;
                    }
                }
                ux = add2(ux, dx);
                uy = add2(uy, dy);
                uz = add2(uz, dz);
            }
        }
        {
            const float tx = ux.x + ux.y, ty = uy.x + uy.y, tzs = uz.x + uz.y;
            float yv = tx - cx, tv = sx + yv;
            cx = (tv - sx) - yv;
            sx = tv;
            yv = ty - cy;
            tv = sy + yv;
            cy = (tv - sy) - yv;
            sy = tv;
            yv = tzs - cz;
            tv = sz + yv;
            cz = (tv - sz) - yv;
            sz = tv;
        }
        __syncthreads();
    }
    if (live) {
        const size_t o = (size_t)blockIdx.y * 3 * nt;
        part[o + li] = (double)sx - (double)cx;
        part[o + nt + li] = (double)sy - (double)cy;
        part[o + 2 * nt + li] = (double)sz - (double)cz;
    }
}

// ------------------------------------------------------------------ symmetric tt pass
// Translation-translation product evaluating each unordered pair once (reciprocity M_ji = M_ij^T).
// The work is the upper triangle of (target block b, source tile t >= b) units of 128 x 128 spheres,
// taken in row-major order and cut into runs of equal length, one per CTA, so that every CTA has the
// same amount of work; a run is split at row ends into segments (b, t0, t1).  Per segment the CTA
// keeps the 128 targets of block b in registers; the diagonal tile (t = b) is done one-directionally
// with the self pair excluded; every other tile gives both u_i (target side, registers) and v_j
// (source side): each lane evaluates four source pairs (eight sources) per step, and their v_j are
// combined across the warp by a reduce-scatter (three exchange levels, then two butterfly levels;
// the order in which a lane takes the pairs and a swapped copy of the tile make it select-free), the
// four warps' sums are added at the end of the tile, and the tile's source sums go to
// src_part[col_start[t] + b].  Each segment's target sums go to tgt_part[segment].  The reduce
// kernel adds, for each sphere, its row's segment partials and its column's source partials in a
// fixed order.  The translation-translation forms load the next tile's sources while a tile is
// evaluated.  The work lists come from sym_schedule.h.
struct SymCta {
    int s0, s1, pad0, pad1;  // segments [s0, s1)
};
struct SymSeg {
    int b, t0, t1, pad;
};

// both halves of a float2 from the lane lane ^ m
__device__ __forceinline__ float2 shfl_xor2(float2 v, int m)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// Periods of the pseudo-periodic mode for the float32 kernels: L = L_hi + L_lo, and 1 / L_hi.
struct PerLen {
    float xh, xl, yh, yl, ix, iy;
};
// Minimum image of an in-plane offset (positions folded into the unit cell: |d| < L).
__device__ __forceinline__ float min_image_f(float d, float Lh, float Ll, float inv)
{
    const float m = rintf(d * inv);
    return fmaf(-m, Ll, fmaf(-m, Lh, d));
}
__device__ __forceinline__ float2 min_image2(float2 d, float Lh, float Ll, float inv)
{
    return make_float2(min_image_f(d.x, Lh, Ll, inv), min_image_f(d.y, Lh, Ll, inv));
}
// d + n L for the image shift n in {-1, 0, 1}
__device__ __forceinline__ float2 shift2(float2 d, float n, float Lh, float Ll)
{
    return make_float2(fmaf(n, Ll, fmaf(n, Lh, d.x)), fmaf(n, Ll, fmaf(n, Lh, d.y)));
}

// RHS2: a second translation-translation right-hand side (src2: s_j P_j per sphere) evaluated with
// the same pair blocks; components 3..5 of the partials carry it.
// PER: pseudo-periodic boundaries (Appendix B): each pair's offset is taken at its minimum image and
// the block is summed over that image and its eight shifts by one period (reciprocity holds image by
// image: the reversed pair's image at -s is the transposed block); the sphere's own unshifted image
// is the self term of the reduce kernel.
// BATCH: the tiles belong to many suspensions packed one after another (sinst: one record per
// suspension; a segment's pad field names its suspension, whose tiles are numbered from tile0);
// segments of suspensions with active[] == 0 are skipped.
template <int MINB, bool TORQUE, bool RHS2 = false, bool PER = false, bool BATCH = false>
__global__ void __launch_bounds__(kPairThreads, MINB) pair_f32x2_sym_kernel(const SrcF32 *__restrict__ src, int N,
                                                                             const SymCta *__restrict__ ctas,
                                                                             const SymSeg *__restrict__ segs,
                                                                             X2Consts c,
                                                                             const int *__restrict__ col_start,
                                                                             double *__restrict__ tgt_part,
                                                                             float *__restrict__ src_part,
                                                                             const float4 *__restrict__ src2 = nullptr,
                                                                             PerLen pl = PerLen{},
                                                                             const SymInst *__restrict__ sinst = nullptr,
                                                                             const int *__restrict__ active = nullptr)
{
    constexpr int P = kTile / 2;
    constexpr int NC = RHS2 ? 6 : 3;
    constexpr int NS = PER ? 9 : 1;  // image shifts per pair
    static_assert(!(PER && RHS2), "the two-right-hand-side form has no pseudo-periodic variant");
    static_assert(!(BATCH && (PER || RHS2)), "the batched form is the plain or the torque form");
    // G source pairs (2G sources) are evaluated per step and then reduce-scattered over the warp
    // (G = 2 is kept as an option: every form measured faster with four).  Each source array holds
    // the tile's pairs (2p, 2p+1) at [p] and the same pairs swapped at [SW + p]; lanes with bit 3
    // (G = 2) or bit 2 (G = 4) set read the swapped copy, so that the element each lane keeps in the
    // reduce-scatter is always .x (SW puts the two copies in different banks for the 2G lane groups)
    constexpr int G = 4;
    constexpr int SW = G == 4 ? P + 4 : P + 2;
    __shared__ float4 sA[SW + P], sB[SW + P], sC[SW + P], sD[SW + P];
    __shared__ float4 sE[TORQUE ? SW + P : 1];
    __shared__ float4 sG[TORQUE ? SW + P : 1];  // (T_z, T_z', 6 z_j, 6 z_j')
    __shared__ float4 sZ[SW + P];                // (-2 z_j, -2 z_j', -4 z_j^2, -4 z_j'^2)
    __shared__ float4 sP[RHS2 ? SW + P : 1];
    __shared__ float2 sQ[RHS2 ? SW + P : 1];
    __shared__ float sv[4][NC][kTile];
    const SymCta cd = ctas[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float2 zero2 = make_float2(0.f, 0.f);
    const int pp = tid >> 1, hh = tid & 1;
    const bool bit4 = (lane >> 4) & 1, bit3 = (lane >> 3) & 1;
    // pk: the pair of a step this lane keeps in the reduce-scatter (it evaluates pairs in the order
    // h ^ pk, so v[0] is that pair and the pairs it sends come in the order its partners keep them);
    // swz: its copy of the source arrays
    const int pk = G == 4 ? ((2 * (int)bit4) ^ (int)bit3) : (int)bit4;
    const bool bsw = G == 4 ? (lane >> 2) & 1 : bit3;  // the lane reads the swapped copy
    const int swz = bsw ? SW : 0;
    // G = 2: offsets of the pair this lane keeps (k0) and of the pair it sends (k1)
    const int k0 = (int)bit4 + (bit3 ? SW : 0), k1 = 1 - (int)bit4 + (bit3 ? SW : 0);
    float *fA = reinterpret_cast<float *>(sA);
    float *fB = reinterpret_cast<float *>(sB);
    float *fC = reinterpret_cast<float *>(sC);
    float *fD = reinterpret_cast<float *>(sD);
    float *fE = reinterpret_cast<float *>(sE);
    float *fG = reinterpret_cast<float *>(sG);
    float *fZ = reinterpret_cast<float *>(sZ);
    float *fP = reinterpret_cast<float *>(sP);
    float *fQ = reinterpret_cast<float *>(sQ);
    for (int sg = cd.s0; sg < cd.s1; ++sg) {
    const SymSeg seg = segs[sg];
    long long off = 0;
    int Ni = N, tb = 0;
    if (BATCH) {
        if (active && !active[seg.pad]) continue;  // the same for the whole CTA
        const SymInst si = sinst[seg.pad];
        off = si.off;
        Ni = si.N;
        tb = si.tile0;
    }
    const int li = (seg.b - tb) * kTile + tid;
    const long long i = off + li;
    float4 tp = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 tf = make_float4(1.f, 0.f, 0.f, 0.f);
    float4 th = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 tq = make_float4(0.f, 0.f, 0.f, 0.f);
    if (li < Ni) {
        tp = src[i].p;
        tf = src[i].f;
        if (TORQUE) th = src[i].t;
        if (RHS2) tq = src2[i];
    }
    const float2 txh = make_float2(tp.x, tp.x), tyh = make_float2(tp.y, tp.y);
    const float2 txl = make_float2(tp.z, tp.z), tyl = make_float2(tp.w, tp.w);
    const float2 tz2 = make_float2(tf.x, tf.x);
    const float2 Gx = make_float2(tf.y, tf.y), Gy = make_float2(tf.z, tf.z), Gz = make_float2(tf.w, tf.w);
    const float2 Hx = make_float2(th.x, th.x), Hy = make_float2(th.y, th.y), Hz = make_float2(th.z, th.z);
    const float2 Qx = make_float2(tq.x, tq.x), Qy = make_float2(tq.y, tq.y), Qz = make_float2(tq.z, tq.z);
    const float2 six_zi = make_float2(6.f * tf.x, 6.f * tf.x);
    float ks[NC], kc[NC];  // compensated per-tile sums of the target side
#pragma unroll
    for (int q = 0; q < NC; ++q) ks[q] = kc[q] = 0.f;
    // translation-translation forms: the next tile's sources are loaded into registers while the
    // current tile is evaluated (the load latency is hidden behind the pair work)
    constexpr bool PF = !TORQUE && !RHS2 && !PER;
    float4 nsp = make_float4(1e18f, 0.f, 0.f, 0.f), nsf = make_float4(1.f, 0.f, 0.f, 0.f);
    if (PF && (seg.t0 - tb) * kTile + tid < Ni) {
        const long long j0 = off + (seg.t0 - tb) * kTile + tid;
        nsp = src[j0].p;
        nsf = src[j0].f;
    }
    for (int t = seg.t0; t < seg.t1; ++t) {
        const int lj = (t - tb) * kTile + tid;
        const long long j = off + lj;
        float4 sp_ = make_float4(1e18f, 0.f, 0.f, 0.f), sf_ = make_float4(1.f, 0.f, 0.f, 0.f);
        float4 st_ = make_float4(0.f, 0.f, 0.f, 0.f), sq_ = make_float4(0.f, 0.f, 0.f, 0.f);
        if (PF) {
            sp_ = nsp;
            sf_ = nsf;
        } else if (lj < Ni) {
            sp_ = src[j].p;
            sf_ = src[j].f;
            if (TORQUE) st_ = src[j].t;
            if (RHS2) sq_ = src2[j];
        }
#pragma unroll
        for (int cp = 0; cp < 2; ++cp) {
            const int o4 = 4 * (cp * SW + pp) + (hh ^ cp), o2 = 2 * (cp * SW + pp) + (hh ^ cp);
            fA[o4] = sp_.x;
            fA[o4 + 2] = sp_.y;
            fB[o4] = sp_.z;
            fB[o4 + 2] = sp_.w;
            fC[o4] = sf_.x;
            fC[o4 + 2] = sf_.y;
            fD[o4] = sf_.z;
            fD[o4 + 2] = sf_.w;
            fZ[o4] = -2.f * sf_.x;
            fZ[o4 + 2] = -4.f * (sf_.x * sf_.x);
            if (TORQUE) {
                fE[o4] = st_.x;
                fE[o4 + 2] = st_.y;
                fG[o4] = st_.z;
                fG[o4 + 2] = 6.f * sf_.x;
            }
            if (RHS2) {
                fP[o4] = sq_.x;
                fP[o4 + 2] = sq_.y;
                fQ[o2] = sq_.z;
            }
        }
        __syncthreads();
        if (PF) {
            nsp = make_float4(1e18f, 0.f, 0.f, 0.f);
            nsf = make_float4(1.f, 0.f, 0.f, 0.f);
            if (t + 1 < seg.t1 && lj + kTile < Ni) {
                nsp = src[j + kTile].p;
                nsf = src[j + kTile].f;
            }
        }
        // a batched suspension's last tile is ragged: the loops stop after its last live source (the
        // padding sources carry zero force, so what they would add is an exact zero; the column
        // partial slots of padding sources then hold stale values, which no output reads)
        const int nsrc = BATCH ? min(kTile, Ni - (t - tb) * kTile) : kTile;
        float2 u[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) u[q] = zero2;
        if (t == seg.b) {
            const int kend = BATCH ? (nsrc + 1) >> 1 : P;
            for (int k = 0; k < kend; ++k) {
                const float4 a = sA[k], b = sB[k], cc = sC[k], d = sD[k];
                const float4 e = TORQUE ? sE[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float2 g = TORQUE ? make_float2(sG[k].x, sG[k].y) : zero2;
                float2 rx0 = add2(sub2(txh, make_float2(a.x, a.y)), sub2(txl, make_float2(b.x, b.y)));
                float2 ry0 = add2(sub2(tyh, make_float2(a.z, a.w)), sub2(tyl, make_float2(b.z, b.w)));
                if (PER) {
                    rx0 = min_image2(rx0, pl.xh, pl.xl, pl.ix);
                    ry0 = min_image2(ry0, pl.yh, pl.yl, pl.iy);
                }
                for (int sh = 0; sh < NS; ++sh) {
                    const float2 rx = PER ? shift2(rx0, (float)(sh / 3 - 1), pl.xh, pl.xl) : rx0;
                    const float2 ry = PER ? shift2(ry0, (float)(sh % 3 - 1), pl.yh, pl.yl) : ry0;
                    float2 dd[NC];
#pragma unroll
                    for (int q = 0; q < NC; ++q) dd[q] = zero2;
                    pair_velocity_x2<TORQUE>(rx, ry, tz2, make_float2(cc.x, cc.y), make_float2(cc.z, cc.w),
                                             make_float2(d.x, d.y), make_float2(d.z, d.w), make_float2(e.x, e.y),
                                             make_float2(e.z, e.w), g, c, dd[0], dd[1], dd[2]);
                    if (RHS2) {
                        const float4 pv = sP[k];
                        pair_velocity_x2<false>(rx, ry, tz2, make_float2(cc.x, cc.y), make_float2(pv.x, pv.y),
                                                make_float2(pv.z, pv.w), sQ[k], zero2, zero2, zero2, c, dd[3 % NC],
                                                dd[4 % NC], dd[5 % NC]);
                    }
                    // source 2k + hh is this thread's own sphere: its unshifted image is the self term
                    if (k == pp && (!PER || sh == 4)) {
#pragma unroll
                        for (int q = 0; q < NC; ++q) {
                            if (hh == 0)
                                dd[q].x = 0.f;
                            else
                                dd[q].y = 0.f;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < NC; ++q) u[q] = add2(u[q], dd[q]);
                }
            }
        } else {
            const int kend = BATCH ? min(P, (nsrc + 2 * G - 1) / (2 * G) * G) : P;
            for (int k = 0; k < kend; k += G) {
                float2 v[G][NC];
#pragma unroll
                for (int h = 0; h < G; ++h) {
                    const int kh = G == 2 ? k + (h ? k1 : k0) : k + (h ^ pk) + swz;
                    const float4 a = sA[kh], cc = sC[kh], d = sD[kh];
                    const float4 e = TORQUE ? sE[kh] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 g4 = TORQUE ? sG[kh] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float2 g = make_float2(g4.x, g4.y), six_zj = make_float2(g4.z, g4.w);
                    const float4 zf = sZ[kh];
                    const float2 m2zj = make_float2(zf.x, zf.y), m4zj2 = make_float2(zf.z, zf.w);
                    const float4 pv = RHS2 ? sP[kh] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float2 pz = RHS2 ? sQ[kh] : zero2;
                    const float2 zj = make_float2(cc.x, cc.y);
                    if (!PER) {
                        float2 rx, ry, rz, rho2, r2;
                        const bool close =
                            pair_offsets_x2(txh, tyh, txl, tyl, tz2, zj, a, &sB[kh], c, rx, ry, rz, rho2, r2);
                        pair_sym_x2<TORQUE, RHS2>(rx, ry, rz, rho2, r2, close, tz2, zj, m2zj, m4zj2, six_zi, six_zj,
                                                  make_float2(cc.z, cc.w),
                                                  make_float2(d.x, d.y), make_float2(d.z, d.w), Gx, Gy, Gz,
                                                  make_float2(e.x, e.y), make_float2(e.z, e.w), g, Hx, Hy, Hz, c,
                                                  u[0], u[1], u[2], v[h][0], v[h][1], v[h][2],
                                                  make_float2(pv.x, pv.y), make_float2(pv.z, pv.w), pz, Qx, Qy, Qz,
                                                  RHS2 ? &u[3 % NC] : nullptr, RHS2 ? &v[h][3 % NC] : nullptr);
                    } else {
                        // minimum image from the full offsets, then the nine images summed both ways
                        const float4 bl = sB[kh];
                        const float2 rx0 = min_image2(add2(sub2(txh, make_float2(a.x, a.y)),
                                                           sub2(txl, make_float2(bl.x, bl.y))), pl.xh, pl.xl, pl.ix);
                        const float2 ry0 = min_image2(add2(sub2(tyh, make_float2(a.z, a.w)),
                                                           sub2(tyl, make_float2(bl.z, bl.w))), pl.yh, pl.yl, pl.iy);
                        const float2 rz = sub2(tz2, zj);
#pragma unroll
                        for (int q = 0; q < NC; ++q) v[h][q] = zero2;
                        for (int sh = 0; sh < 9; ++sh) {
                            const float2 rx = shift2(rx0, (float)(sh / 3 - 1), pl.xh, pl.xl);
                            const float2 ry = shift2(ry0, (float)(sh % 3 - 1), pl.yh, pl.yl);
                            const float2 rho2 = fma2(rx, rx, mul2(ry, ry));
                            const float2 r2 = fma2(rz, rz, rho2);
                            const bool close = __any_sync(0xffffffffu, r2.x < c.four_a2 || r2.y < c.four_a2);
                            float2 vx, vy, vz;
                            pair_sym_x2<TORQUE>(rx, ry, rz, rho2, r2, close, tz2, zj, m2zj, m4zj2, six_zi, six_zj,
                                                make_float2(cc.z, cc.w),
                                                make_float2(d.x, d.y), make_float2(d.z, d.w), Gx, Gy, Gz,
                                                make_float2(e.x, e.y), make_float2(e.z, e.w), g, Hx, Hy, Hz, c,
                                                u[0], u[1], u[2], vx, vy, vz);
                            v[h][0] = add2(v[h][0], vx);
                            v[h][1] = add2(v[h][1], vy);
                            v[h][2] = add2(v[h][2], vz);
                        }
                    }
                }
                // reduce-scatter of the 2G sources 2k .. 2k + 2G - 1 over the warp.  G = 2: lane L ends
                // with the sum for source 2(k + pk) + bit3(L), stored by lanes 0, 8, 16, 24; G = 4:
                // with source 2(k + pk) + bit2(L), stored by lanes 0, 4, .., 28
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    float w;
                    if (G == 2) {
                        const float2 w2 = add2(v[0][q], shfl_xor2(v[1 % G][q], 16));
                        w = w2.x + __shfl_xor_sync(0xffffffffu, w2.y, 8);
                    } else {
                        const float2 a0 = add2(v[0][q], shfl_xor2(v[2 % G][q], 16));
                        const float2 a1 = add2(v[1 % G][q], shfl_xor2(v[3 % G][q], 16));
                        const float2 x2 = add2(a0, shfl_xor2(a1, 8));
                        w = x2.x + __shfl_xor_sync(0xffffffffu, x2.y, 4);
                    }
                    if (G == 2) w += __shfl_xor_sync(0xffffffffu, w, 4);
                    w += __shfl_xor_sync(0xffffffffu, w, 2);
                    w += __shfl_xor_sync(0xffffffffu, w, 1);
                    // (the two-pair index is spelled 2k + 2 bit4 + bit3: the equal 2(k + pk) + bit3 cost the
                    // two-right-hand-side form, at its 128-register cap, 14% in time)
                    if ((lane & (G == 4 ? 3 : 7)) == 0) sv[warp][q][G == 4 ? 2 * (k + pk) + bsw : 2 * k + 2 * bit4 + bit3] = w;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            const float yv = (u[q].x + u[q].y) - kc[q];
            const float tv = ks[q] + yv;
            kc[q] = (tv - ks[q]) - yv;
            ks[q] = tv;
        }
        __syncthreads();
        if (t != seg.b) {
            float *o = src_part + (size_t)(col_start[t] + seg.b) * NC * kTile;
#pragma unroll
            for (int q = 0; q < NC; ++q) o[q * kTile + tid] = (sv[0][q][tid] + sv[1][q][tid]) + (sv[2][q][tid] + sv[3][q][tid]);
        }
        __syncthreads();
    }
    double *o = tgt_part + (size_t)sg * NC * kTile;
#pragma unroll
    for (int q = 0; q < NC; ++q) o[q * kTile + tid] = (double)ks[q] - (double)kc[q];
    }
}

// Row partials of the targets plus column partials of the sources, fixed order; float64 self term
// (with the torque's wall self coupling when T is given; left out when self_term is 0, for all but
// one share of a shared product); s_i / (8 pi eta).  col_rows: the rows [r0, r1) of each column that
// the schedule wrote (null: all rows above the diagonal).  NC = 6: the partials also
// carry a second translation-translation right-hand side P, written to U2 with its own self term.
// BATCH: tiles of many suspensions (tile_inst: the suspension of each tile; sinst as in the pair
// kernel); the column of tile b holds the rows tile0 .. b - 1 of its suspension, summed in an order
// relative to tile0 so that a suspension's result does not depend on its companions.
template <int NC, bool BATCH = false>
__global__ void __launch_bounds__(BATCH ? 384 : 768, BATCH ? 5 : 2) pair_sym_reduce_kernel(const double *__restrict__ tgt_part, const float *__restrict__ src_part,
                                       const int *__restrict__ row_seg, const int *__restrict__ col_start, int N,
                                       const double *__restrict__ pos, const double *__restrict__ F,
                                       const double *__restrict__ T, PairConsts<double> c, double a, double scale,
                                       double *__restrict__ U, const double *__restrict__ P = nullptr,
                                       double *__restrict__ U2 = nullptr,
                                       const SymInst *__restrict__ sinst = nullptr,
                                       const int *__restrict__ tile_inst = nullptr,
                                       const int *__restrict__ active = nullptr,
                                       const int *__restrict__ col_rows = nullptr, int self_term = 1)
{
    // one CTA of 768 threads (384 batched) per 128-sphere tile, the longest columns first; thread (half, q, l):
    // component q of sphere l, rows of its column congruent to `half` modulo HALVES
    // (a batched suspension's columns are at most a few tiles long: one thread per (q, l) there, so
    // that twice as many tiles are resident at once)
    constexpr int HALVES = BATCH ? 1 : 6 / NC;
    __shared__ double s[NC][kTile];
    __shared__ double s1[NC][kTile];
    const int nb = gridDim.x;
    const int b = BATCH ? (int)blockIdx.x : nb - 1 - (int)blockIdx.x;
    long long off = 0;
    int Ni = N, tb = 0;
    if (BATCH) {
        const int inst = tile_inst[b];
        if (active && !active[inst]) return;  // the same for the whole CTA
        const SymInst si = sinst[inst];
        off = si.off;
        Ni = si.N;
        tb = si.tile0;
    }
    const int half = threadIdx.x / (NC * kTile);
    const int r = threadIdx.x - half * NC * kTile;
    const int q = r / kTile, l = r - q * kTile;
    // column of float32 partials: four independent compensated float32 sums per thread (GB300's
    // float64 rate would make a float64 add per partial the bottleneck; one chain per thread would
    // leave the column latency-bound), converted once and added in a fixed order
    // rows [r0, r1) of the column (a share of the triangle writes only some of them)
    const int r0 = BATCH ? tb : (col_rows ? col_rows[2 * b] : 0);
    const int r1 = BATCH ? b : (col_rows ? col_rows[2 * b + 1] : b);
    const float *col = src_part + (size_t)col_start[b] * NC * kTile + q * kTile + l;
    float cs[4] = {0.f, 0.f, 0.f, 0.f}, cc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int bb = r0 + half; bb < r1; bb += 4 * HALVES) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int row = bb + HALVES * u;
            if (row < r1) {
                const float yv = col[(size_t)row * NC * kTile] - cc[u];
                const float tv = cs[u] + yv;
                cc[u] = (tv - cs[u]) - yv;
                cs[u] = tv;
            }
        }
    }
    double v = 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) v += (double)cs[u] - (double)cc[u];
    if (HALVES == 2 && half == 1) s1[q][l] = v;
    __syncthreads();
    if (half == 0) {
        double acc = 0.0;
        for (int k = row_seg[b]; k < row_seg[b + 1]; ++k) acc += tgt_part[((size_t)k * NC + q) * kTile + l];
        s[q][l] = acc + (HALVES == 2 ? v + s1[q][l] : v);
    }
    __syncthreads();
    const int lb = (b - tb) * kTile + l;
    if (half != 0 || lb >= Ni || (q != 0 && q != 3)) return;
    const long long i = off + lb;
    const double z = pos[2 * N + i];
    const double si = H0(z / a);
    const double zc = fmax(z, a);
    const double k = si * scale;
    if (q == 0) {
        double ux = s[0][l], uy = s[1][l], uz = s[2][l];
        if (!BATCH && !self_term)
            ;
        else if (T)
            self_velocity<true>(zc, si * F[i], si * F[N + i], si * F[2 * N + i], si * T[i], si * T[N + i], c, ux, uy,
                                uz);
        else
            self_velocity<false>(zc, si * F[i], si * F[N + i], si * F[2 * N + i], 0.0, 0.0, c, ux, uy, uz);
        U[i] = k * ux;
        U[N + i] = k * uy;
        U[2 * N + i] = k * uz;
    } else if (NC == 6) {
        double ux = s[3 % NC][l], uy = s[4 % NC][l], uz = s[5 % NC][l];
        if (BATCH || self_term)
            self_velocity<false>(zc, si * P[i], si * P[N + i], si * P[2 * N + i], 0.0, 0.0, c, ux, uy, uz);
        U2[i] = k * ux;
        U2[N + i] = k * uy;
        U2[2 * N + i] = k * uz;
    }
}

constexpr int kTtMinBlocks = 5;     // resident CTAs per SM of the translation-translation form (up to 102 registers:
                                    // four source pairs per step and the next tile's sources in flight fit in 96
                                    // with the polynomial coefficient form; 4 CTAs measured 2.6% slower)
constexpr int kFusedMinBlocks = 4;  // resident CTAs per SM of the form with torques
constexpr int kRhs2MinBlocks = 3;  // resident CTAs per SM of the two-right-hand-side form
constexpr int kPerMinBlocks = 4;   // resident CTAs per SM of the pseudo-periodic forms

// Capacity of the schedule: at most kSymMaxCtaPerSm x SMs CTAs and that many plus nb segments.
constexpr int kSymMaxCtaPerSm = 64;

size_t sym_src_part_bytes(int64_t max_N)
{
    const int64_t nb = (max_N + kTile - 1) / kTile;
    return (size_t)(nb * (nb - 1) / 2) * 3 * kTile * sizeof(float);
}

size_t sym_tgt_part_bytes(int64_t max_N, int num_sms)
{
    const int64_t nb = (max_N + kTile - 1) / kTile;
    return (size_t)(nb + (int64_t)kSymMaxCtaPerSm * num_sms + 1) * 3 * kTile * sizeof(double);
}

size_t sym_index_ints(int64_t max_N, int num_sms)
{
    const int64_t nb = (max_N + kTile - 1) / kTile;
    const int64_t maxcta = (int64_t)kSymMaxCtaPerSm * num_sms;
    return (size_t)(4 * maxcta + 4 * (maxcta + nb + 1) + 4 * (nb + 1));
}

// Schedule of the symmetric pass for N, share `part` of `nparts` (built and copied to the device when
// they change): the whole triangle in ws.sym, a share in ws.sym_part.
static int sym_prepare(rpb_ctx *ctx, int N, const SymSched **out, int part = 0, int nparts = 1)
{
    Workspace &w = ctx->ws;
    SymSched &sc = nparts == 1 ? w.sym : w.sym_part;
    *out = &sc;
    if (sc.N == N && sc.part == part && sc.nparts == nparts) return RPB_OK;
    sc.N = -1;
    cudaStream_t st = ctx->stream;
    std::vector<int> cta4, seg4, row_seg, col_start, col_rows;
    int64_t u0, u1;
    sym_part_units(N, kTile, part, nparts, &u0, &u1);
    sym_schedule_range(N, ctx->num_sms, kTile, u0, u1, cta4, seg4, row_seg, col_start, col_rows);
    const size_t need = cta4.size() + seg4.size() + row_seg.size() + col_start.size() + col_rows.size();
    if (need > w.sym_index_ints || seg4.size() / 4 * 3 * kTile * sizeof(double) > w.sym_tgt_bytes) {
        set_error("internal: symmetric schedule larger than its scratch (N=%d)", N);
        return RPB_EINVAL;
    }
    std::vector<int> host(need);
    size_t o = 0;
    for (const std::vector<int> *v : {&cta4, &seg4, &row_seg, &col_start, &col_rows}) {
        std::copy(v->begin(), v->end(), host.begin() + o);
        o += v->size();
    }
    sc.index = w.sym_index + (nparts == 1 ? 0 : w.sym_index_ints);
    int rc;
    if ((rc = cuda_fail(cudaMemcpyAsync(sc.index, host.data(), need * sizeof(int), cudaMemcpyHostToDevice, st),
                        "symmetric schedule copy")))
        return rc;
    if ((rc = cuda_fail(cudaStreamSynchronize(st), "symmetric schedule copy"))) return rc;
    sc.N = N;
    sc.part = part;
    sc.nparts = nparts;
    sc.ncta = (int)(cta4.size() / 4);
    sc.nseg = (int)(seg4.size() / 4);
    sc.seg_off = (int)cta4.size();
    sc.row_off = sc.seg_off + (int)seg4.size();
    sc.col_off = sc.row_off + (int)row_seg.size();
    sc.rows_off = sc.col_off + (int)col_start.size();
    return RPB_OK;
}

int pair_prepare(rpb_ctx *ctx, int64_t N)
{
    const SymSched *sc;
    if (ctx->sym_enabled && N >= 2 * kTile && N <= ctx->max_N) return sym_prepare(ctx, (int)N, &sc);
    return RPB_OK;
}

// Symmetric product (float32 pairs), translation-translation or, with T, the fused product;
// requires ctx->ws.sym_* scratch.  With nparts > 1: share `part` of the triangle's pairs, the self
// terms with share 0 only (the shares add up to the product).
static int mobility_sym(rpb_ctx *ctx, int N, const double *pos, const double *F, const double *T, double *U,
                        int part = 0, int nparts = 1)
{
    cudaStream_t st = ctx->stream;
    Workspace &w = ctx->ws;
    const SymSched *sc;
    int rc;
    if ((rc = sym_prepare(ctx, N, &sc, part, nparts))) return rc;
    const double a = ctx->p.a;
    SrcF32 *src = (SrcF32 *)w.src;
    const int pb = 256;
    pack_f32_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, F, T, N, a, 1, src);
    const SymCta *ctas = (const SymCta *)sc->index;
    const SymSeg *segs = (const SymSeg *)(sc->index + sc->seg_off);
    const X2Consts c = make_x2_consts(a);
    const int *cs = sc->index + sc->col_off;
    if (sc->ncta > 0) {
        if (T)
            pair_f32x2_sym_kernel<kFusedMinBlocks, true><<<sc->ncta, kPairThreads, 0, st>>>(src, N, ctas, segs, c, cs,
                                                                                            w.sym_tgt, w.sym_src);
        else
            pair_f32x2_sym_kernel<kTtMinBlocks, false><<<sc->ncta, kPairThreads, 0, st>>>(src, N, ctas, segs, c, cs,
                                                                                          w.sym_tgt, w.sym_src);
    }
    pair_sym_reduce_kernel<3><<<(N + kTile - 1) / kTile, 6 * kTile, 0, st>>>(
        w.sym_tgt, w.sym_src, sc->index + sc->row_off, cs, N, pos, F, T, make_consts<double>(a), a,
        1.0 / (8.0 * kPi * ctx->p.eta), U, nullptr, nullptr, nullptr, nullptr, nullptr, sc->index + sc->rows_off,
        part == 0);
    count_launches(sc->ncta > 0 ? 3 : 2);
    return cuda_fail(cudaGetLastError(), "symmetric pair kernels");
}

// The symmetric product in pseudo-periodic mode: positions already folded into the unit cell
// (pos_w; the self terms use the heights of pos, which the fold leaves unchanged); shares as above.
static int mobility_sym_periodic(rpb_ctx *ctx, int N, const double *pos_w, const double *pos, const double *F,
                                 const double *T, double *U, int part = 0, int nparts = 1)
{
    cudaStream_t st = ctx->stream;
    Workspace &w = ctx->ws;
    const SymSched *sc;
    int rc;
    if ((rc = sym_prepare(ctx, N, &sc, part, nparts))) return rc;
    const double a = ctx->p.a;
    SrcF32 *src = (SrcF32 *)w.src;
    const int pb = 256;
    pack_f32_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos_w, F, T, N, a, 1, src);
    const SymCta *ctas = (const SymCta *)sc->index;
    const SymSeg *segs = (const SymSeg *)(sc->index + sc->seg_off);
    const X2Consts c = make_x2_consts(a);
    const int *cs = sc->index + sc->col_off;
    PerLen pl;
    pl.xh = (float)ctx->Lx;
    pl.xl = (float)(ctx->Lx - (double)pl.xh);
    pl.yh = (float)ctx->Ly;
    pl.yl = (float)(ctx->Ly - (double)pl.yh);
    pl.ix = 1.f / pl.xh;
    pl.iy = 1.f / pl.yh;
    if (sc->ncta > 0) {
        if (T)
            pair_f32x2_sym_kernel<kPerMinBlocks, true, false, true><<<sc->ncta, kPairThreads, 0, st>>>(
                src, N, ctas, segs, c, cs, w.sym_tgt, w.sym_src, nullptr, pl);
        else
            pair_f32x2_sym_kernel<kPerMinBlocks, false, false, true><<<sc->ncta, kPairThreads, 0, st>>>(
                src, N, ctas, segs, c, cs, w.sym_tgt, w.sym_src, nullptr, pl);
    }
    pair_sym_reduce_kernel<3><<<(N + kTile - 1) / kTile, 6 * kTile, 0, st>>>(
        w.sym_tgt, w.sym_src, sc->index + sc->row_off, cs, N, pos, F, T, make_consts<double>(a), a,
        1.0 / (8.0 * kPi * ctx->p.eta), U, nullptr, nullptr, nullptr, nullptr, nullptr, sc->index + sc->rows_off,
        part == 0);
    count_launches(sc->ncta > 0 ? 3 : 2);
    return cuda_fail(cudaGetLastError(), "periodic symmetric pair kernels");
}

// ------------------------------------------------------------------ batched symmetric pass
// Each suspension's rows of tiles are cut by a fixed rule (runs of at most kBatchSegTiles tiles), so
// that the partial sums a suspension's result is made of do not depend on the other suspensions; one
// CTA per run, longest runs first.
constexpr int kBatchSegTiles = 8;
constexpr size_t kBatchSymScratchLimit = (size_t)4 << 30;

void batch_sym_free(BatchSymPlan &pl)
{
    void *d[] = {pl.index, pl.sinst, pl.tgt, pl.srcp};
    for (void *x : d)
        if (x) cudaFree(x);
    pl = BatchSymPlan();
}

static int grow(void **ptr, size_t *cap, size_t need, const char *what)
{
    if (need <= *cap) return RPB_OK;
    if (*ptr) cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
    if (cudaMalloc(ptr, need) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        set_error("cudaMalloc of %zu bytes (%s) failed", need, what);
        return RPB_ENOMEM;
    }
    *cap = need;
    return RPB_OK;
}

int batch_sym_plan(BatchSymPlan &pl, int B, const int64_t *N, cudaStream_t st, bool *ok, int seg_tiles)
{
    *ok = false;
    if (seg_tiles < 1) seg_tiles = kBatchSegTiles;
    std::vector<int64_t> sizes(N, N + B);
    if (pl.valid && sizes == pl.sizes && seg_tiles == pl.seg_tiles) {
        *ok = true;
        return RPB_OK;
    }
    pl.valid = false;
    BatchSchedule bs;
    batch_sym_schedule(B, N, kTile, seg_tiles, bs);
    std::vector<SymInst> si(B);
    for (int k = 0; k < B; ++k) si[k] = SymInst{(long long)bs.off[k], bs.n[k], bs.tile0[k]};
    const std::vector<int> &seg4 = bs.seg4, &row_seg = bs.row_seg, &col_start = bs.col_start,
                           &tile_inst = bs.tile_inst, &order = bs.cta_order;
    const int nseg = (int)(seg4.size() / 4);
    const int g = bs.ntiles;
    const size_t src_bytes = (size_t)bs.n_src_slots * 3 * kTile * sizeof(float);
    const size_t tgt_bytes = (size_t)nseg * 3 * kTile * sizeof(double);
    if (src_bytes + tgt_bytes > kBatchSymScratchLimit) return RPB_OK;  // one-way kernels instead
    std::vector<int> host;
    host.reserve(4 * nseg + seg4.size() + row_seg.size() + col_start.size() + tile_inst.size());
    for (int q : order) {
        host.push_back(q);
        host.push_back(q + 1);
        host.push_back(0);
        host.push_back(0);
    }
    const int seg_off = (int)host.size();
    host.insert(host.end(), seg4.begin(), seg4.end());
    const int row_off = (int)host.size();
    host.insert(host.end(), row_seg.begin(), row_seg.end());
    const int col_off = (int)host.size();
    host.insert(host.end(), col_start.begin(), col_start.end());
    const int inst_off = (int)host.size();
    host.insert(host.end(), tile_inst.begin(), tile_inst.end());
    int rc;
    size_t icap = pl.index_cap * sizeof(int), scap = (size_t)pl.sinst_cap * sizeof(SymInst);
    if ((rc = grow((void **)&pl.index, &icap, host.size() * sizeof(int), "batched symmetric schedule")) ||
        (rc = grow((void **)&pl.sinst, &scap, (size_t)B * sizeof(SymInst), "batched symmetric instances")) ||
        (rc = grow((void **)&pl.tgt, &pl.tgt_cap, tgt_bytes, "batched symmetric partials")) ||
        (rc = grow((void **)&pl.srcp, &pl.src_cap, std::max<size_t>(src_bytes, 16), "batched symmetric partials")))
        return rc;
    pl.index_cap = icap / sizeof(int);
    pl.sinst_cap = (int)(scap / sizeof(SymInst));
    if ((rc = cuda_fail(cudaMemcpyAsync(pl.index, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice, st),
                        "batched symmetric schedule copy")) ||
        (rc = cuda_fail(cudaMemcpyAsync(pl.sinst, si.data(), (size_t)B * sizeof(SymInst), cudaMemcpyHostToDevice, st),
                        "batched symmetric instances copy")) ||
        (rc = cuda_fail(cudaStreamSynchronize(st), "batched symmetric plan")))
        return rc;
    pl.ncta = nseg;
    pl.nseg = nseg;
    pl.ntiles = g;
    pl.seg_off = seg_off;
    pl.row_off = row_off;
    pl.col_off = col_off;
    pl.inst_off = inst_off;
    pl.sizes = sizes;
    pl.seg_tiles = seg_tiles;
    pl.valid = true;
    *ok = true;
    return RPB_OK;
}

int batch_sym_apply(const BatchSymPlan &pl, cudaStream_t st, const SrcF32 *src, int64_t total, const double *pos,
                    const double *F, const double *T, double *U, const int *active, double a, double eta)
{
    const SymCta *ctas = (const SymCta *)pl.index;
    const SymSeg *segs = (const SymSeg *)(pl.index + pl.seg_off);
    const int *cs = pl.index + pl.col_off;
    const X2Consts c = make_x2_consts(a);
    const int n = (int)total;
    if (T)
        pair_f32x2_sym_kernel<kFusedMinBlocks, true, false, false, true><<<pl.ncta, kPairThreads, 0, st>>>(
            src, n, ctas, segs, c, cs, pl.tgt, pl.srcp, nullptr, PerLen{}, pl.sinst, active);
    else if (pl.tt_minb == 4)
        pair_f32x2_sym_kernel<4, false, false, false, true><<<pl.ncta, kPairThreads, 0, st>>>(
            src, n, ctas, segs, c, cs, pl.tgt, pl.srcp, nullptr, PerLen{}, pl.sinst, active);
    else
        pair_f32x2_sym_kernel<5, false, false, false, true><<<pl.ncta, kPairThreads, 0, st>>>(
            src, n, ctas, segs, c, cs, pl.tgt, pl.srcp, nullptr, PerLen{}, pl.sinst, active);
    pair_sym_reduce_kernel<3, true><<<pl.ntiles, 3 * kTile, 0, st>>>(
        pl.tgt, pl.srcp, pl.index + pl.row_off, cs, n, pos, F, T, make_consts<double>(a), a, 1.0 / (8.0 * kPi * eta),
        U, nullptr, nullptr, pl.sinst, pl.index + pl.inst_off, active);
    count_launches(2);
    return cuda_fail(cudaGetLastError(), "batched symmetric kernels");
}

bool mobility_apply2_ok(const rpb_ctx *ctx, int64_t N)
{
    return !ctx->hook && ctx->sym_rhs2 && ctx->sym_enabled && ctx->p.wall && !(ctx->Lx > 0.0) && N >= 2 * kTile;
}

int mobility_apply2_impl(rpb_ctx *ctx, int64_t N64, const double *pos, const double *F, const double *T,
                         const double *P, double *U, double *U2)
{
    const int N = (int)N64;
    cudaStream_t st = ctx->stream;
    Workspace &w = ctx->ws;
    const SymSched *sc;
    int rc;
    if ((rc = sym_prepare(ctx, N, &sc))) return rc;
    if ((size_t)sc->nseg * 6 * kTile * sizeof(double) > w.sym_tgt_bytes ||
        sym_src_part_bytes(N) * 2 > w.sym_src_bytes) {
        set_error("internal: two-right-hand-side scratch too small (N=%d)", N);
        return RPB_EINVAL;
    }
    const double a = ctx->p.a;
    SrcF32 *src = (SrcF32 *)w.src;
    float4 *src2 = (float4 *)w.src2;
    const int pb = 256;
    pack_f32_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, F, T, N, a, 1, src);
    pack_rhs2_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, P, N, a, src2);
    const SymCta *ctas = (const SymCta *)sc->index;
    const SymSeg *segs = (const SymSeg *)(sc->index + sc->seg_off);
    const int *cs = sc->index + sc->col_off;
    pair_f32x2_sym_kernel<kRhs2MinBlocks, true, true><<<sc->ncta, kPairThreads, 0, st>>>(
        src, N, ctas, segs, make_x2_consts(a), cs, w.sym_tgt, w.sym_src, src2);
    pair_sym_reduce_kernel<6><<<(N + kTile - 1) / kTile, 6 * kTile, 0, st>>>(
        w.sym_tgt, w.sym_src, sc->index + sc->row_off, cs, N, pos, F, T, make_consts<double>(a), a,
        1.0 / (8.0 * kPi * ctx->p.eta), U, P, U2, nullptr, nullptr, nullptr, sc->index + sc->rows_off);
    count_launches(4);
    return cuda_fail(cudaGetLastError(), "two-right-hand-side symmetric kernels");
}

template <bool TORQUE, bool WALL = true>
__global__ void __launch_bounds__(kPairThreads) pair_f64_kernel(const SrcF64 *__restrict__ src, int N, int chunk,
                                                                 PairConsts<double> c, double *__restrict__ part,
                                                                 int t0 = 0, int nt = -1)
{
    __shared__ double2 sp[kTile];
    __shared__ double2 sq[kTile];
    __shared__ double2 sr[kTile];
    __shared__ double2 ss[TORQUE ? kTile : 1];
    __shared__ double2 su[TORQUE ? kTile : 1];
    if (nt < 0) nt = N;
    const int tid = threadIdx.x;
    const int li = blockIdx.x * kPairThreads + tid;
    const int i = t0 + li;
    const bool live = li < nt && i < N;
    const int j0 = blockIdx.y * chunk;
    const int j1 = min(N, j0 + chunk);
    double2 tp = make_double2(0.0, 0.0);
    double tz = 1.0;
    if (live) {
        tp = src[i].p;
        tz = src[i].q.x;
    }
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int base = j0; base < j1; base += kTile) {
        const int j = base + tid;
        if (j < j1) {
            sp[tid] = src[j].p;
            sq[tid] = src[j].q;
            sr[tid] = src[j].r;
            if (TORQUE) {
                ss[tid] = src[j].s;
                su[tid] = src[j].u;
            }
        }
        __syncthreads();
        const int cnt = min(kTile, j1 - base);
        const int self_k = i - base;  // this thread's own sphere is source self_k of the tile, if in [0, cnt)
        if (self_k < 0 || self_k >= cnt) {
#pragma unroll 2
            for (int k = 0; k < cnt; ++k) {
                const double2 p = sp[k], q = sq[k], r = sr[k];
                const double2 s = TORQUE ? ss[k] : make_double2(0.0, 0.0);
                const double2 u = TORQUE ? su[k] : make_double2(0.0, 0.0);
                pair_velocity_f64<TORQUE, WALL>(tp.x - p.x, tp.y - p.y, tz, q.x, q.y, r.x, r.y, s.x, s.y, u.x, c,
                                                    ux, uy, uz);
            }
        } else {
            for (int k = 0; k < cnt; ++k) {
                const double2 p = sp[k], q = sq[k], r = sr[k];
                const double2 s = TORQUE ? ss[k] : make_double2(0.0, 0.0);
                const double2 u = TORQUE ? su[k] : make_double2(0.0, 0.0);
                double dx = 0.0, dy = 0.0, dz = 0.0;
                pair_velocity_f64<TORQUE, WALL>(tp.x - p.x, tp.y - p.y, tz, q.x, q.y, r.x, r.y, s.x, s.y, u.x, c,
                                                    dx, dy, dz);
                if (k != self_k) {
                    ux += dx;
                    uy += dy;
                    uz += dz;
                }
            }
        }
        __syncthreads();
    }
    if (live) {
        const size_t o = (size_t)blockIdx.y * 3 * nt;
        part[o + li] = ux;
        part[o + nt + li] = uy;
        part[o + 2 * nt + li] = uz;
    }
}

// ------------------------------------------------------------------ pseudo-periodic boundaries
// Positions folded into the unit cell [0, Lx) x [0, Ly) (heights unchanged).
__global__ void wrap_kernel(const double *__restrict__ pos, int N, double Lx, double Ly, double *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double x = pos[i], y = pos[N + i];
    out[i] = x - Lx * floor(x / Lx);
    out[N + i] = y - Ly * floor(y / Ly);
    out[2 * N + i] = pos[2 * N + i];
}

// Appendix B: periodic in x and y; each source is taken at its minimum image and at the eight shifts of
// it by one period (the unit cell and its eight neighbour cells).  One-way kernels (the symmetric
// pass is not used in this mode).  The pack kernel has wrapped every position into the unit cell, so
// in-plane offsets lie in (-L, L) and the minimum-image correction is 0 or +-L.  The sphere's own
// unshifted image is the self term (added by the reduce kernel); its eight shifted images are pairs.
template <bool TORQUE, bool WALL>
__global__ void __launch_bounds__(kPairThreads) pair_periodic_f64_kernel(const SrcF64 *__restrict__ src, int N,
                                                                          int chunk, PairConsts<double> c, double Lx,
                                                                          double Ly, double *__restrict__ part)
{
    __shared__ SrcF64 ss[kTile];
    const int tid = threadIdx.x;
    const int i = blockIdx.x * kPairThreads + tid;
    const int j0 = blockIdx.y * chunk;
    const int j1 = min(N, j0 + chunk);
    double2 tp = make_double2(0.0, 0.0);
    double tz = 1.0;
    if (i < N) {
        tp = src[i].p;
        tz = src[i].q.x;
    }
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int base = j0; base < j1; base += kTile) {
        if (base + tid < j1) ss[tid] = src[base + tid];
        __syncthreads();
        const int cnt = min(kTile, j1 - base);
        for (int k = 0; k < cnt; ++k) {
            const SrcF64 s = ss[k];
            double dx = tp.x - s.p.x, dy = tp.y - s.p.y;
            dx -= Lx * rint(dx / Lx);
            dy -= Ly * rint(dy / Ly);
            const bool self = base + k == i;
            for (int nx = -1; nx <= 1; ++nx)
                for (int ny = -1; ny <= 1; ++ny) {
                    if (self && nx == 0 && ny == 0) continue;
                    pair_velocity_f64<TORQUE, WALL>(dx + nx * Lx, dy + ny * Ly, tz, s.q.x, s.q.y, s.r.x, s.r.y,
                                                        s.s.x, s.s.y, s.u.x, c, ux, uy, uz);
                }
        }
        __syncthreads();
    }
    if (i < N) {
        const size_t o = (size_t)blockIdx.y * 3 * N;
        part[o + i] = ux;
        part[o + N + i] = uy;
        part[o + 2 * N + i] = uz;
    }
}

// Float32 version; the period is split L = L_hi + L_lo like the positions.
template <bool TORQUE, bool WALL>
__global__ void __launch_bounds__(kPairThreads) pair_periodic_f32_kernel(const SrcF32 *__restrict__ src, int N,
                                                                          int chunk, PairConsts<float> c, float Lxh,
                                                                          float Lxl, float Lyh, float Lyl,
                                                                          double *__restrict__ part)
{
    __shared__ SrcF32 ss[kTile];
    const int tid = threadIdx.x;
    const int i = blockIdx.x * kPairThreads + tid;
    const int j0 = blockIdx.y * chunk;
    const int j1 = min(N, j0 + chunk);
    float4 tp = make_float4(0.f, 0.f, 0.f, 0.f);
    float tz = 1.f;
    if (i < N) {
        tp = src[i].p;
        tz = src[i].f.x;
    }
    const float ix = 1.f / Lxh, iy = 1.f / Lyh;
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int base = j0; base < j1; base += kTile) {
        if (base + tid < j1) ss[tid] = src[base + tid];
        __syncthreads();
        const int cnt = min(kTile, j1 - base);
        float ux = 0.f, uy = 0.f, uz = 0.f;
        for (int k = 0; k < cnt; ++k) {
            const SrcF32 s = ss[k];
            float dx = (tp.x - s.p.x) + (tp.z - s.p.z);
            float dy = (tp.y - s.p.y) + (tp.w - s.p.w);
            const float mx = rintf(dx * ix), my = rintf(dy * iy);
            dx = (dx - mx * Lxh) - mx * Lxl;
            dy = (dy - my * Lyh) - my * Lyl;
            const bool self = base + k == i;
            for (int nx = -1; nx <= 1; ++nx)
                for (int ny = -1; ny <= 1; ++ny) {
                    float ax = 0.f, ay = 0.f, az = 0.f;
                    pair_velocity_f32<TORQUE, WALL>((dx + nx * Lxh) + nx * Lxl, (dy + ny * Lyh) + ny * Lyl, tz, s.f.x,
                                                    s.f.y, s.f.z, s.f.w, s.t.x, s.t.y, s.t.z, c, ax, ay, az);
                    if (!(self && nx == 0 && ny == 0)) {
                        ux += ax;
                        uy += ay;
                        uz += az;
                    }
                }
        }
        sx += ux;
        sy += uy;
        sz += uz;
        __syncthreads();
    }
    if (i < N) {
        const size_t o = (size_t)blockIdx.y * 3 * N;
        part[o + i] = sx;
        part[o + N + i] = sy;
        part[o + 2 * N + i] = sz;
    }
}

// Sum the chunk partials in order, add the float64 self term, apply s_i / (8 pi eta).  Targets t0 ..
// t0 + nt - 1 (nt < 0: all N); U and the partials are indexed by i - t0, the partials with component
// stride nt, U with component stride ldu (ldu < 0: nt).
__global__ void pair_reduce_kernel(const double *__restrict__ part, int splits, int N, const double *__restrict__ pos,
                                   const double *__restrict__ F, const double *__restrict__ T, PairConsts<double> c,
                                   double a, double scale, double *__restrict__ U, int wall = 1, int t0 = 0,
                                   int nt = -1, int ldu = -1)
{
    if (nt < 0) nt = N;
    if (ldu < 0) ldu = nt;
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t0 + li;
    if (li >= nt || i >= N) return;
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int s = 0; s < splits; ++s) {
        const size_t o = (size_t)s * 3 * nt;
        ux += part[o + li];
        uy += part[o + nt + li];
        uz += part[o + 2 * nt + li];
    }
    const double z = pos[2 * N + i];
    const double si = wall ? H0(z / a) : 1.0;
    const double zc = wall ? fmax(z, a) : z;
    const double Fx = F ? si * F[i] : 0.0, Fy = F ? si * F[N + i] : 0.0, Fz = F ? si * F[2 * N + i] : 0.0;
    const double Tx = T ? si * T[i] : 0.0, Ty = T ? si * T[N + i] : 0.0;
    if (wall)
        self_velocity<true, true>(zc, Fx, Fy, Fz, Tx, Ty, c, ux, uy, uz);
    else
        self_velocity<true, false>(zc, Fx, Fy, Fz, Tx, Ty, c, ux, uy, uz);
    const double k = si * scale;
    U[li] = k * ux;
    U[ldu + li] = k * uy;
    U[2 * ldu + li] = k * uz;
}

// The same sum with one warp per target, for products split into many source chunks (small float64
// products): lane l adds chunks l, l + 32, ... and a butterfly adds the lanes in a fixed order, so the
// float64 additions spread over many warps instead of one dependent chain per target; lane 0 adds the
// self term and writes.  Four targets per 128-thread block.
__global__ void __launch_bounds__(128) pair_reduce_warp_kernel(const double *__restrict__ part, int splits, int N,
                                                               const double *__restrict__ pos,
                                                               const double *__restrict__ F,
                                                               const double *__restrict__ T, PairConsts<double> c,
                                                               double a, double scale, double *__restrict__ U,
                                                               int wall, int t0, int nt, int ldu)
{
    const int lane = threadIdx.x & 31;
    const int li = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int i = t0 + li;
    if (li >= nt || i >= N) return;  // the same for the whole warp
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int s = lane; s < splits; s += 32) {
        const size_t o = (size_t)s * 3 * nt;
        ux += part[o + li];
        uy += part[o + nt + li];
        uz += part[o + 2 * nt + li];
    }
    for (int m = 16; m > 0; m >>= 1) {
        ux += __shfl_xor_sync(0xffffffffu, ux, m);
        uy += __shfl_xor_sync(0xffffffffu, uy, m);
        uz += __shfl_xor_sync(0xffffffffu, uz, m);
    }
    if (lane != 0) return;
    const double z = pos[2 * N + i];
    const double si = wall ? H0(z / a) : 1.0;
    const double zc = wall ? fmax(z, a) : z;
    const double Fx = F ? si * F[i] : 0.0, Fy = F ? si * F[N + i] : 0.0, Fz = F ? si * F[2 * N + i] : 0.0;
    const double Tx = T ? si * T[i] : 0.0, Ty = T ? si * T[N + i] : 0.0;
    if (wall)
        self_velocity<true, true>(zc, Fx, Fy, Fz, Tx, Ty, c, ux, uy, uz);
    else
        self_velocity<true, false>(zc, Fx, Fy, Fz, Tx, Ty, c, ux, uy, uz);
    const double k = si * scale;
    U[li] = k * ux;
    U[ldu + li] = k * uy;
    U[2 * ldu + li] = k * uz;
}

// Chunk partials -> U (targets t0 .. t0 + nt - 1, nt < 0: all N; U's component stride ldu, ldu < 0:
// nt): a thread per target for few chunks (coalesced loads), a warp per target for many.
static void launch_pair_reduce(cudaStream_t st, const double *part, int splits, int N, const double *pos,
                               const double *F, const double *T, double a, double scale, double *U, int wall,
                               int t0 = 0, int nt = -1, int ldu = -1)
{
    if (nt < 0) nt = N;
    if (ldu < 0) ldu = nt;
    const PairConsts<double> c = make_consts<double>(a);
    if (splits >= 16) {
        pair_reduce_warp_kernel<<<(unsigned)((nt + 3) / 4), 128, 0, st>>>(part, splits, N, pos, F, T, c, a, scale, U,
                                                                          wall, t0, nt, ldu);
    } else {
        // 64-target CTAs: the float64 self terms of a small product then spread over several SMs
        const int rb = 64;
        pair_reduce_kernel<<<(unsigned)((nt + rb - 1) / rb), rb, 0, st>>>(part, splits, N, pos, F, T, c, a, scale, U,
                                                                          wall, t0, nt, ldu);
    }
}

void pair_grid(int64_t N, int num_sms, int precision, int slots, int *splits, int64_t *chunk)
{
    pair_grid_plan(N, num_sms, precision == RPB_FP64, slots, kTile, splits, chunk);
}

// Resident CTAs over the whole GPU of the float32 one-way kernels (translation only, with torques).
int pair_occupancy(rpb_ctx *ctx)
{
    int a = 0, b = 0;
    int rc;
    if ((rc = cuda_fail(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, pair_f32x2_kernel<false>, kPairThreads, 0),
                        "pair kernel occupancy")) ||
        (rc = cuda_fail(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, pair_f32x2_kernel<true>, kPairThreads, 0),
                        "pair kernel occupancy")))
        return rc;
    ctx->f32_slots[0] = std::max(1, a) * ctx->num_sms;
    ctx->f32_slots[1] = std::max(1, b) * ctx->num_sms;
    return RPB_OK;
}

size_t pair_partial_bytes(int64_t max_N, int num_sms)
{
    const int64_t tiles = (max_N + kTile - 1) / kTile;
    const int64_t f64 = (target_blocks(num_sms) + tiles + 1) * kTile;  // float64 splits x N bound
    const int64_t f32 = (int64_t)kMaxSplitsF32 * max_N;                 // float32 splits x N bound
    return (size_t)3 * sizeof(double) * (size_t)std::max(f64, f32);
}

// Rows t0 .. t1 - 1 of U = M_tt F + M_tr T (all N sources), written to U_rows with component stride
// ldu (ldu < 0: t1 - t0): the one-way kernels restricted to a range of targets (t0 a multiple of kTile).
int mobility_rows_impl(rpb_ctx *ctx, int64_t N64, const double *pos, const double *F, const double *T, int64_t t0,
                       int64_t t1, double *U_rows, int64_t ldu)
{
    const int N = (int)N64, nt = (int)(t1 - t0);
    cudaStream_t st = ctx->stream;
    const double a = ctx->p.a;
    const bool fp64 = ctx->p.precision == RPB_FP64;
    int splits;
    int64_t chunk;
    rows_grid_plan(nt, N64, ctx->num_sms, fp64, kTile, &splits, &chunk);
    if ((size_t)splits * 3 * nt * sizeof(double) > ctx->ws.partial_bytes) {
        set_error("internal: pair partial buffer too small for rows (nt=%d splits=%d)", nt, splits);
        return RPB_EINVAL;
    }
    double *part = (double *)ctx->ws.partial;
    const int pb = 256;
    const dim3 grid((unsigned)((nt + kPairThreads - 1) / kPairThreads), (unsigned)splits);
    const bool torque = T != nullptr;
    if (fp64) {
        SrcF64 *src = (SrcF64 *)ctx->ws.src;
        pack_f64_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, F, T, N, a, ctx->p.wall, src);
        const PairConsts<double> c = make_consts<double>(a);
        if (!ctx->p.wall) {
            if (torque)
                pair_f64_kernel<true, false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part, (int)t0, nt);
            else
                pair_f64_kernel<false, false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part, (int)t0, nt);
        } else if (torque) {
            pair_f64_kernel<true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part, (int)t0, nt);
        } else {
            pair_f64_kernel<false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part, (int)t0, nt);
        }
    } else {
        SrcF32 *src = (SrcF32 *)ctx->ws.src;
        pack_f32_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, F, T, N, a, 1, src);
        const X2Consts c = make_x2_consts(a);
        if (torque)
            pair_f32x2_kernel<true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part, (int)t0, nt);
        else
            pair_f32x2_kernel<false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part, (int)t0, nt);
    }
    launch_pair_reduce(st, part, splits, N, pos, F, T, a, 1.0 / (8.0 * kPi * ctx->p.eta), U_rows, ctx->p.wall,
                       (int)t0, nt, (int)ldu);
    count_launches(3);
    return cuda_fail(cudaGetLastError(), "row pair kernels");
}

static int mobility_direct(rpb_ctx *ctx, int64_t N64, const double *pos, const double *F, const double *T,
                           double *U);

int mobility_apply_impl(rpb_ctx *ctx, int64_t N64, const double *pos, const double *F, const double *T, double *U)
{
    if (ctx->hook && !ctx->in_hook) {  // the product is delegated (e.g. shared out among processes)
        ctx->in_hook = 1;
        const int rc = ctx->hook(ctx->hook_user, N64, pos, F, T, U);
        ctx->in_hook = 0;
        if (rc != RPB_OK && rpb_last_error()[0] == 0) set_error("product hook returned %d", rc);
        return rc;
    }
    return mobility_direct(ctx, N64, pos, F, T, U);
}

// Rows [r0, r1) of share `part` of `nparts`: whole 128-row tiles, as equal as the tiles allow.
static void part_rows(int64_t N, int part, int nparts, int64_t *r0, int64_t *r1)
{
    const int64_t tiles = (N + kTile - 1) / kTile;
    const int64_t base = tiles / nparts, extra = tiles % nparts;
    const int64_t t0 = part * base + std::min<int64_t>(part, extra);
    const int64_t t1 = t0 + base + (part < extra ? 1 : 0);
    *r0 = std::min(N, t0 * kTile);
    *r1 = std::min(N, t1 * kTile);
}

int mobility_part_impl(rpb_ctx *ctx, int64_t N64, const double *pos, const double *F, const double *T, int part,
                       int nparts, double *U)
{
    if (nparts == 1) return mobility_direct(ctx, N64, pos, F, T, U);
    const int N = (int)N64;
    cudaStream_t st = ctx->stream;
    const bool sym = ctx->sym_enabled && ctx->p.wall && F && N >= 2 * kTile && (!T || ctx->sym_fused);
    if (sym && !(ctx->Lx > 0.0)) return mobility_sym(ctx, N, pos, F, T, U, part, nparts);
    if (sym && ctx->p.precision == RPB_FP32) {
        const int pb = 256;
        wrap_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, N, ctx->Lx, ctx->Ly, ctx->ws.pos_w);
        count_launches(1);
        return mobility_sym_periodic(ctx, N, ctx->ws.pos_w, pos, F, T, U, part, nparts);
    }
    int rc;
    if ((rc = cuda_fail(cudaMemsetAsync(U, 0, (size_t)3 * N * sizeof(double), st), "part product zero fill")))
        return rc;
    // the pseudo-periodic one-way kernels and the float32 ones without the wall take all targets:
    // share 0 holds the product
    if (ctx->Lx > 0.0 || (ctx->p.precision == RPB_FP32 && !ctx->p.wall))
        return part == 0 && (F || T) ? mobility_direct(ctx, N64, pos, F, T, U) : RPB_OK;
    if (!F && !T) return RPB_OK;
    int64_t r0, r1;
    part_rows(N64, part, nparts, &r0, &r1);
    if (r1 <= r0) return RPB_OK;
    return mobility_rows_impl(ctx, N64, pos, F, T, r0, r1, U + r0, N64);
}

static int mobility_direct(rpb_ctx *ctx, int64_t N64, const double *pos, const double *F, const double *T,
                           double *U)
{
    const int N = (int)N64;
    if (ctx->sym_enabled && ctx->p.wall && !(ctx->Lx > 0.0) && F && N >= 2 * kTile && (!T || ctx->sym_fused))
        return mobility_sym(ctx, N, pos, F, T, U);
    cudaStream_t st = ctx->stream;
    const double a = ctx->p.a;
    int splits;
    int64_t chunk;
    pair_grid(N64, ctx->num_sms, ctx->p.precision, ctx->f32_slots[T != nullptr ? 1 : 0], &splits, &chunk);
    if ((size_t)splits * 3 * N * sizeof(double) > ctx->ws.partial_bytes) {
        set_error("internal: pair partial buffer too small (N=%d splits=%d)", N, splits);
        return RPB_EINVAL;
    }
    double *part = (double *)ctx->ws.partial;
    const int pb = 256;
    const dim3 grid((unsigned)((N + kPairThreads - 1) / kPairThreads), (unsigned)splits);
    const bool torque = T != nullptr;
    if (ctx->Lx > 0.0) {  // pseudo-periodic: wrap into the unit cell, pack, nine shifts per source
        const double Lx = ctx->Lx, Ly = ctx->Ly;
        wrap_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, N, Lx, Ly, ctx->ws.pos_w);
        const double *pw = ctx->ws.pos_w;
        if (ctx->p.precision == RPB_FP32 && ctx->sym_enabled && ctx->p.wall && F && N >= 2 * kTile &&
            (!T || ctx->sym_fused)) {
            count_launches(1);
            return mobility_sym_periodic(ctx, N, pw, pos, F, T, U);
        }
        if (ctx->p.precision == RPB_FP32) {
            SrcF32 *src = (SrcF32 *)ctx->ws.src;
            pack_f32_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pw, F, T, N, a, ctx->p.wall, src);
            const PairConsts<float> c = make_consts<float>(a);
            const float Lxh = (float)Lx, Lyh = (float)Ly;
            const float Lxl = (float)(Lx - (double)Lxh), Lyl = (float)(Ly - (double)Lyh);
            if (torque && ctx->p.wall)
                pair_periodic_f32_kernel<true, true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, Lxh, Lxl, Lyh, Lyl, part);
            else if (torque)
                pair_periodic_f32_kernel<true, false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, Lxh, Lxl, Lyh, Lyl, part);
            else if (ctx->p.wall)
                pair_periodic_f32_kernel<false, true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, Lxh, Lxl, Lyh, Lyl, part);
            else
                pair_periodic_f32_kernel<false, false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, Lxh, Lxl, Lyh, Lyl, part);
        } else {
            SrcF64 *src = (SrcF64 *)ctx->ws.src;
            pack_f64_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pw, F, T, N, a, ctx->p.wall, src);
            const PairConsts<double> c = make_consts<double>(a);
            if (torque && ctx->p.wall)
                pair_periodic_f64_kernel<true, true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, Lx, Ly, part);
            else if (torque)
                pair_periodic_f64_kernel<true, false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, Lx, Ly, part);
            else if (ctx->p.wall)
                pair_periodic_f64_kernel<false, true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, Lx, Ly, part);
            else
                pair_periodic_f64_kernel<false, false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, Lx, Ly, part);
        }
        launch_pair_reduce(st, part, splits, N, pos, F, T, a, 1.0 / (8.0 * kPi * ctx->p.eta), U, ctx->p.wall);
        count_launches(4);
        return cuda_fail(cudaGetLastError(), "periodic pair kernels");
    }
    if (ctx->p.precision == RPB_FP32) {
        SrcF32 *src = (SrcF32 *)ctx->ws.src;
        pack_f32_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, F, T, N, a, ctx->p.wall, src);
        if (!ctx->p.wall) {
            const PairConsts<float> c = make_consts<float>(a);
            if (torque)
                pair_f32_kernel<true, false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
            else
                pair_f32_kernel<false, false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
        } else if (ctx->fp32_variant == 1) {
            const X2Consts c = make_x2_consts(a);
            if (torque)
                pair_f32x2_kernel<true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
            else
                pair_f32x2_kernel<false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
        } else {
            const PairConsts<float> c = make_consts<float>(a);
            if (torque)
                pair_f32_kernel<true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
            else
                pair_f32_kernel<false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
        }
    } else {
        SrcF64 *src = (SrcF64 *)ctx->ws.src;
        pack_f64_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, F, T, N, a, ctx->p.wall, src);
        const PairConsts<double> c = make_consts<double>(a);
        if (!ctx->p.wall) {
            if (torque)
                pair_f64_kernel<true, false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
            else
                pair_f64_kernel<false, false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
        } else if (torque) {
            pair_f64_kernel<true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
        } else {
            pair_f64_kernel<false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
        }
    }
    launch_pair_reduce(st, part, splits, N, pos, F, T, a, 1.0 / (8.0 * kPi * ctx->p.eta), U, ctx->p.wall);
    count_launches(3);
    return cuda_fail(cudaGetLastError(), "pair kernels");
}

// ------------------------------------------------------------------ cell lists for the force pass
// Square cells of side h = the screen radius on an unbounded grid, hashed into G x G buckets by their
// coordinates modulo G (G ~ sqrt(N), a power of two in [64, kCellGrid]; far-away cells that share a
// bucket only add candidates, which the distance screen rejects); heights are not binned.  Buckets are filled by a
// counting sort and each bucket's list is then sorted by sphere index, so that every force is summed
// in a fixed order (buckets in a fixed order, spheres by index within a bucket).  A bucket with more
// than kCellMaxSorted spheres sets the overfull flag and the all-pairs kernel takes the product.
__device__ __forceinline__ void cell_coords(double x, double y, double inv_h, int &cx, int &cy)
{
    // clamped so that the conversion is defined for any input (non-finite positions land in one cell)
    const double fx = floor(fmin(fmax(x * inv_h, -1e9), 1e9)), fy = floor(fmin(fmax(y * inv_h, -1e9), 1e9));
    cx = fx == fx ? (int)fx : 0;
    cy = fy == fy ? (int)fy : 0;
}
// G x G buckets, G a power of two in [64, kCellGrid] chosen by N (cell_grid)
__device__ __forceinline__ int cell_bucket(int cx, int cy, int G)
{
    return (cy & (G - 1)) * G + (cx & (G - 1));
}

static int cell_grid(int64_t N)
{
    int G = 64;
    while (G < kCellGrid && (int64_t)G * G < N) G *= 2;
    return G;
}

__global__ void cell_count_kernel(const double *__restrict__ pos, int N, double inv_h, int G, int *__restrict__ count,
                                  int *__restrict__ cellof)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int cx, cy;
    cell_coords(pos[i], pos[N + i], inv_h, cx, cy);
    const int c = cell_bucket(cx, cy, G);
    cellof[i] = c;
    atomicAdd(&count[c], 1);
}

// Exclusive scan of the nb = G^2 counts by one block: 1024 threads, nb / 1024 (a multiple of 4)
// consecutive buckets each, read (twice: sums, then the running offsets) and written as int4.
__global__ void __launch_bounds__(1024) cell_scan_kernel(const int *__restrict__ count, int nb, int *__restrict__ start,
                                                         int *__restrict__ fill)
{
    const int per = nb / 1024;
    __shared__ int wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = tid * per;
    const int4 *in4 = reinterpret_cast<const int4 *>(count + c0);
    int s = 0;
#pragma unroll 4
    for (int k = 0; k < per / 4; ++k) {
        const int4 q = in4[k];
        s += (q.x + q.y) + (q.z + q.w);
    }
    int inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += u;
        }
        wsum[lane] = w;  // inclusive warp totals
    }
    __syncthreads();
    int run = inc - s + (warp > 0 ? wsum[warp - 1] : 0);
    int4 *s4 = reinterpret_cast<int4 *>(start + c0), *f4 = reinterpret_cast<int4 *>(fill + c0);
#pragma unroll 4
    for (int k = 0; k < per / 4; ++k) {
        const int4 q = in4[k];
        int4 o;
        o.x = run;
        o.y = o.x + q.x;
        o.z = o.y + q.y;
        o.w = o.z + q.z;
        run = o.w + q.w;
        s4[k] = o;
        f4[k] = o;
    }
    if (tid == 1023) start[nb] = run;
}

__global__ void cell_fill_kernel(int N, const int *__restrict__ cellof, int *__restrict__ fill, int *__restrict__ idx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    idx[atomicAdd(&fill[cellof[i]], 1)] = i;
}

__global__ void cell_sort_kernel(const double *__restrict__ pos, int N, int nb, const int *__restrict__ start,
                                 int *__restrict__ idx, float4 *__restrict__ posf, CellHeader *__restrict__ hdr)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nb) return;
    const int a0 = start[c], a1 = start[c + 1];
    if (a1 - a0 > kCellMaxSorted) {
        hdr->overfull = 1;  // every writer stores the same value
        return;
    }
    for (int m = a0 + 1; m < a1; ++m) {
        const int v = idx[m];
        int q = m - 1;
        while (q >= a0 && idx[q] > v) {
            idx[q + 1] = idx[q];
            --q;
        }
        idx[q + 1] = v;
    }
    for (int m = a0; m < a1; ++m) {
        const int j = idx[m];
        posf[m] = make_float4((float)pos[j], (float)pos[N + j], (float)pos[2 * N + j], __int_as_float(j));
    }
}

// Force pass over the buckets: threads take the spheres in bucket order (neighbouring threads search
// the same buckets); candidates are screened in float32 against the radius of the all-pairs kernel,
// queued per thread and evaluated in float64 after the search, in the same fixed order.
__global__ void __launch_bounds__(128) forces_cell_kernel(const double *__restrict__ pos, int N, double a,
                                                          double weight, double U0, double b, float cut2,
                                                          double inv_h, int G, const CellHeader *__restrict__ hdr,
                                                          const int *__restrict__ start, const int *__restrict__ idx,
                                                          const float4 *__restrict__ posf, double *__restrict__ F)
{
    if (cell_overfull(hdr)) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int i = idx[k];
    const double xi = pos[i], yi = pos[N + i], zi = pos[2 * N + i];
    const float xf = (float)xi, yf = (float)yi, zf = (float)zi;
    int cx, cy;
    cell_coords(xi, yi, inv_h, cx, cy);
    const double f0 = U0 / b;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    // the bucket loops have different lengths in different lanes, so the float64 work waits until
    // after them (all lanes flush together); a queue filled earlier (dense configurations) flushes
    // on its own
    constexpr int kQ = 64;
    int queue[kQ];
    int nq = 0;
    auto flush = [&]() {
        for (int q = 0; q < nq; ++q) {
            const int j = queue[q];
            const double dx = xi - pos[j], dy = yi - pos[N + j], dz = zi - pos[2 * N + j];
            const double mm = steric_pair_factor(dx * dx + dy * dy + dz * dz, 2.0 * a, f0, 1.0 / b);
            fx += mm * dx;
            fy += mm * dy;
            fz += mm * dz;
        }
        nq = 0;
    };
    for (int dyc = -1; dyc <= 1; ++dyc)
        for (int dxc = -1; dxc <= 1; ++dxc) {
            const int cc = cell_bucket(cx + dxc, cy + dyc, G);
            for (int m = start[cc]; m < start[cc + 1]; ++m) {
                const float4 pj = posf[m];
                const int j = __float_as_int(pj.w);
                const float ex = xf - pj.x, ey = yf - pj.y, ez = zf - pj.z;
                if (j != i && fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < cut2) {
                    queue[nq++] = j;
                    if (nq == kQ) flush();
                }
            }
        }
    flush();
    fz += (zi < a ? f0 : f0 * exp(-(zi - a) / b)) - weight;
    F[i] = fx;
    F[N + i] = fy;
    F[2 * N + i] = fz;
}

// ------------------------------------------------------------------ forces (Sec. III)
// F_i = -weight z + sum_j f(|r_ij|) r_ij/|r_ij| + f_wall(z_i) z with f = -dU/dr of Eq. (soft_potential).
// Pairs are screened in float32 against a cutoff with a generous margin; the ones inside are
// evaluated in float64.
// PER: pseudo-periodic boundaries (Appendix B), minimum image in x (period Lx) and y (period Ly); the
// positions are then the ones folded into the unit cell.
// gate: when given, the kernel runs only if the cell-list pass declined the configuration.
template <bool PER>
__global__ void __launch_bounds__(128) forces_kernel(const double *__restrict__ pos, int N, double a, double weight,
                                                     double U0, double b, float cut2, double *__restrict__ F,
                                                     double Lx = 0.0, double Ly = 0.0,
                                                     const CellHeader *gate = nullptr)
{
    if (gate && !cell_overfull(gate)) return;
    __shared__ float4 sp[64];  // float32 copies of the tile's positions, for the screen only
    const int tid = threadIdx.x;
    const int i = blockIdx.x * 128 + tid;
    double xi = 0.0, yi = 0.0, zi = 0.0;
    if (i < N) {
        xi = pos[i];
        yi = pos[N + i];
        zi = pos[2 * N + i];
    }
    const float xf = (float)xi, yf = (float)yi, zf = (float)zi;
    const double f0 = U0 / b;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    // Near pairs found by the float32 screen are queued per thread and evaluated in float64 together
    // after the screen (or when the queue is full), so a warp pays for the slowest lane's list rather
    // than for every lane's pairs one after another.
    constexpr int kQ = 32;
    int queue[kQ];
    int nq = 0;
    auto flush = [&]() {
        for (int q = 0; q < nq; ++q) {
            const int jj = queue[q];
            double dx = xi - pos[jj], dy = yi - pos[N + jj];
            const double dz = zi - pos[2 * N + jj];
            if (PER) {
                dx -= Lx * rint(dx / Lx);
                dy -= Ly * rint(dy / Ly);
            }
            const double m = steric_pair_factor(dx * dx + dy * dy + dz * dz, 2.0 * a, f0, 1.0 / b);
            fx += m * dx;
            fy += m * dy;
            fz += m * dz;
        }
        nq = 0;
    };
    // the tile as 64 interleaved pairs: sp[p] = (x[2p], x[2p+1], y[2p], y[2p+1]); z in sp2, so that two
    // sources are screened per lane with packed float32x2 arithmetic
    __shared__ float2 sz[64];
    float *fxy = reinterpret_cast<float *>(sp);
    float *fz2 = reinterpret_cast<float *>(sz);
    const float2 X = make_float2(xf, xf), Y = make_float2(yf, yf), Z = make_float2(zf, zf);
    const float fLx = (float)Lx, fLy = (float)Ly;
    const float fiLx = PER ? 1.f / fLx : 0.f, fiLy = PER ? 1.f / fLy : 0.f;
    const int pp = tid >> 1, hh = tid & 1;
    for (int base = 0; base < N; base += 128) {
        const int j = base + tid;
        // slots past N hold a point far above the wall (never inside the screen, also after the
        // minimum-image fold of x and y); the queue test re-checks the index
        const bool in = j < N;
        fxy[4 * pp + hh] = in ? (float)pos[j] : 0.f;
        fxy[4 * pp + 2 + hh] = in ? (float)pos[N + j] : 0.f;
        fz2[2 * pp + hh] = in ? (float)pos[2 * N + j] : 1e18f;
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 64; ++k) {
            const float4 p = sp[k];
            float2 dx = sub2(X, make_float2(p.x, p.y)), dy = sub2(Y, make_float2(p.z, p.w));
            const float2 dz = sub2(Z, sz[k]);
            if (PER) {
                dx.x -= fLx * rintf(dx.x * fiLx);
                dx.y -= fLx * rintf(dx.y * fiLx);
                dy.x -= fLy * rintf(dy.x * fiLy);
                dy.y -= fLy * rintf(dy.y * fiLy);
            }
            const float2 d2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
            if (d2.x < cut2 || d2.y < cut2) {  // rare: a near pair (or the sphere itself)
                const int j0 = base + 2 * k;
                if (d2.x < cut2 && j0 != i && j0 < N) {
                    queue[nq++] = j0;
                    if (nq == kQ) flush();
                }
                if (d2.y < cut2 && j0 + 1 != i && j0 + 1 < N) {
                    queue[nq++] = j0 + 1;
                    if (nq == kQ) flush();
                }
            }
        }
        __syncthreads();
    }
    flush();
    if (i < N) {
        fz += (zi < a ? f0 : f0 * exp(-(zi - a) / b)) - weight;
        F[i] = fx;
        F[N + i] = fy;
        F[2 * N + i] = fz;
    }
}

int forces_impl(rpb_ctx *ctx, int64_t N, const double *pos, const rpb_force_params *fp, double *F)
{
    const double a = ctx->p.a;
    const double r_cut = 2.0 * a + kForceCutoffB * fp->b;
    const double rcm = r_cut * 1.01 + 0.01 * a;
    const float cut2 = (float)(rcm * rcm);
    const int n = (int)N;
    cudaStream_t st = ctx->stream;
    if (ctx->Lx > 0.0) {
        const int pb = 256;
        wrap_kernel<<<(unsigned)((N + pb - 1) / pb), pb, 0, st>>>(pos, n, ctx->Lx, ctx->Ly, ctx->ws.pos_w);
        forces_kernel<true><<<(unsigned)((N + 127) / 128), 128, 0, st>>>(ctx->ws.pos_w, n, a, fp->weight, fp->U0,
                                                                         fp->b, cut2, F, ctx->Lx, ctx->Ly);
        count_launches(2);
        return cuda_fail(cudaGetLastError(), "forces kernel");
    }
    // buckets of cells of side = the screen radius, then the bucket force pass; the all-pairs kernel
    // runs instead when a bucket holds more than kCellMaxSorted spheres (it checks the flag itself)
    CellLists L = cell_lists(ctx->ws.cells, ctx->max_N);
    const double inv_h = 1.0 / rcm;
    const int G = cell_grid(N), nb = G * G;
    int rc;
    // the header (overfull flag) and the bucket counts are contiguous: one clear
    if ((rc = cuda_fail(cudaMemsetAsync(L.hdr, 0, 64 + sizeof(int) * (nb + 1), st), "clear cell counts")))
        return rc;
    cell_count_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(pos, n, inv_h, G, L.count, L.cellof);
    cell_scan_kernel<<<1, 1024, 0, st>>>(L.count, nb, L.start, L.fill);
    cell_fill_kernel<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(n, L.cellof, L.fill, L.idx);
    cell_sort_kernel<<<nb / 256, 256, 0, st>>>(pos, n, nb, L.start, L.idx, L.posf, L.hdr);
    // small systems in 32-sphere blocks: their float64 near pairs then spread over more SMs
    const int fb = N < 128 * ctx->num_sms ? 32 : 128;
    forces_cell_kernel<<<(unsigned)((N + fb - 1) / fb), fb, 0, st>>>(pos, n, a, fp->weight, fp->U0, fp->b, cut2, inv_h,
                                                                     G, L.hdr, L.start, L.idx, L.posf, F);
    forces_kernel<false><<<(unsigned)((N + 127) / 128), 128, 0, st>>>(pos, n, a, fp->weight, fp->U0, fp->b, cut2, F,
                                                                      0.0, 0.0, L.hdr);
    count_launches(6);
    return cuda_fail(cudaGetLastError(), "forces kernels");
}

}  // namespace rpb

// ------------------------------------------------------------------ allocation-free product
// rpb_mobility_apply_noalloc: the same pack / pair / reduce kernels as rpb_mobility_apply, with their
// scratch (packed sources, then the per-chunk partial sums) in a fixed array of the library's device
// image instead of a context's cudaMalloc'd workspace.  The array is created with the module on
// every device that loads the library and lives until the process exits.
#include <cuda.h>

#include <mutex>

namespace rpb {

constexpr int64_t kNoAllocSrcBytes = (int64_t)RPB_NOALLOC_MAX_N * (int64_t)sizeof(SrcF64);
constexpr int64_t kNoAllocPartialElems = (int64_t)16 * 3 * RPB_NOALLOC_MAX_N;  // 16 chunks at the maximum N
constexpr int64_t kNoAllocBytes = kNoAllocSrcBytes + kNoAllocPartialElems * (int64_t)sizeof(double);
static_assert(kNoAllocSrcBytes % 256 == 0, "partials must start 256-byte aligned");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
// Per device: the context the address was looked up in (its process-unique id), the address, the SM
// count.  A context destroyed and created again (cudaDeviceReset, or a primary context released and
// retained anew) loads the module again, and the array may then live elsewhere: the id tells.
struct NoAllocSlot {
    unsigned long long ctx_id;
    void *ptr;
    int sms;
};
static NoAllocSlot g_noalloc[kNoAllocMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Process-unique id of the calling thread's current CUDA context (driver entry points through the
// runtime, so the library needs no link against the driver library).  Called with g_noalloc_mu held.
static int current_ctx_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    int rc;
    if (!get_current || !get_id) {
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0 = cudaDriverEntryPointSymbolNotFound, q1 = q0;
        if ((rc = cuda_fail(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0),
                            "cudaGetDriverEntryPointByVersion(cuCtxGetCurrent)")))
            return rc;
        if ((rc = cuda_fail(cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1),
                            "cudaGetDriverEntryPointByVersion(cuCtxGetId)")))
            return rc;
        if (q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1) {
            set_error("the CUDA driver offers no cuCtxGetCurrent / cuCtxGetId");
            return RPB_ECUDA;
        }
        get_current = (CtxGetCurrentFn)f0;
        get_id = (CtxGetIdFn)f1;
    }
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || !c) {
        set_error("no current CUDA context");
        return RPB_ECUDA;
    }
    if (get_id(c, id) != CUDA_SUCCESS) {
        set_error("cuCtxGetId failed");
        return RPB_ECUDA;
    }
    return RPB_OK;
}

// Device address of the scratch array in the current context (looked up once per device and
// context).  The lookup is refused while `st` is being captured into a graph: it runs host-side
// runtime calls that have no place in a capture.
static int noalloc_setup(cudaStream_t st, void **ptr, int *sms)
{
    int dev = 0;
    int rc;
    if ((rc = cuda_fail(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("device ordinal %d outside [0, %d)", dev, kNoAllocMaxDevices);
        return RPB_EINVAL;
    }
    // (a runtime call on the stream: it also makes the device's context current if nothing has yet)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((rc = cuda_fail(cudaStreamIsCapturing(st, &cs), "cudaStreamIsCapturing"))) return rc;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);  // also guards the driver entry points' first lookup
    unsigned long long id = 0;
    if ((rc = current_ctx_id(&id))) return rc;
    NoAllocSlot &sl = g_noalloc[dev];
    if (!sl.ptr || sl.ctx_id != id) {
        if (cs != cudaStreamCaptureStatusNone) {
            set_error("rpb_mobility_apply_noalloc: the first call on a device (or after its context was "
                      "recreated) must not be made while the stream is being captured");
            return RPB_EINVAL;
        }
        void *p = nullptr;
        if ((rc = cuda_fail(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)"))) return rc;
        int n = 0;
        if ((rc = cuda_fail(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev), "SM count"))) return rc;
        sl.ctx_id = id;
        sl.ptr = p;
        sl.sms = n;
    }
    *ptr = sl.ptr;
    *sms = sl.sms;
    return RPB_OK;
}

}  // namespace rpb

extern "C" int rpb_mobility_apply_noalloc(int64_t N64, const double *pos, const double *F, const double *T, double *U,
                                          const rpb_params *p, void *stream)
{
    using namespace rpb;
    if (!p || !(p->a > 0.0) || !(p->eta > 0.0) || (p->precision != RPB_FP64 && p->precision != RPB_FP32) ||
        p->wall != 1) {
        set_error("rpb_mobility_apply_noalloc: missing or bad parameters (wall must be 1)");
        return RPB_EINVAL;
    }
    if (N64 <= 0 || N64 > RPB_NOALLOC_MAX_N) {
        set_error("rpb_mobility_apply_noalloc: N=%lld outside [1, %d] (the size of its fixed scratch)", (long long)N64,
                  RPB_NOALLOC_MAX_N);
        return RPB_EINVAL;
    }
    const void *ptrs[] = {pos, F, T, U};
    for (const void *q : ptrs)
        if (q && ((uintptr_t)q & 7u)) {
            set_error("rpb_mobility_apply_noalloc: pointer not 8-byte aligned");
            return RPB_EINVAL;
        }
    if (!pos || !U) {
        set_error("rpb_mobility_apply_noalloc: pos and U must not be null");
        return RPB_EINVAL;
    }
    if (U == pos || U == F || U == T) {
        set_error("rpb_mobility_apply_noalloc: U aliases an input");
        return RPB_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int N = (int)N64;
    if (!F && !T) return cuda_fail(cudaMemsetAsync(U, 0, 3 * N64 * sizeof(double), st), "memset U");
    void *base = nullptr;
    int sms = 0;
    int rc;
    if ((rc = noalloc_setup(st, &base, &sms))) return rc;
    int splits;
    int64_t chunk;
    noalloc_grid_plan(N64, sms, p->precision == RPB_FP64, kTile, kNoAllocPartialElems, &splits, &chunk);
    double *part = (double *)((unsigned char *)base + kNoAllocSrcBytes);
    const int pb = 256;
    const dim3 grid((unsigned)((N + kPairThreads - 1) / kPairThreads), (unsigned)splits);
    const double a = p->a;
    if (p->precision == RPB_FP32) {
        SrcF32 *src = (SrcF32 *)base;
        pack_f32_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, F, T, N, a, 1, src);
        const PairConsts<float> c = make_consts<float>(a);
        if (T)
            pair_f32_kernel<true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
        else
            pair_f32_kernel<false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
    } else {
        SrcF64 *src = (SrcF64 *)base;
        pack_f64_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, F, T, N, a, 1, src);
        const PairConsts<double> c = make_consts<double>(a);
        if (T)
            pair_f64_kernel<true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
        else
            pair_f64_kernel<false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
    }
    launch_pair_reduce(st, part, splits, N, pos, F, T, a, 1.0 / (8.0 * kPi * p->eta), U, 1);
    count_launches(3);
    return cuda_fail(cudaGetLastError(), "rpb_mobility_apply_noalloc kernels");
}
