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
#include <cmath>
#include <cstdio>

#include "pair_math.cuh"

namespace rpb {

// ------------------------------------------------------------------ packing
__global__ void pack_f32_kernel(const double *__restrict__ pos, const double *__restrict__ F,
                                const double *__restrict__ T, int N, double a, SrcF32 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double x = pos[i], y = pos[N + i], z = pos[2 * N + i];
    const double s = H0(z / a);
    const float xh = (float)x, yh = (float)y;
    SrcF32 o;
    o.p = make_float4(xh, yh, (float)(x - (double)xh), (float)(y - (double)yh));
    o.f = make_float4((float)fmax(z, a), F ? (float)(s * F[i]) : 0.f, F ? (float)(s * F[N + i]) : 0.f,
                      F ? (float)(s * F[2 * N + i]) : 0.f);
    o.t = make_float4(T ? (float)(s * T[i]) : 0.f, T ? (float)(s * T[N + i]) : 0.f, T ? (float)(s * T[2 * N + i]) : 0.f,
                      0.f);
    out[i] = o;
}

__global__ void pack_f64_kernel(const double *__restrict__ pos, const double *__restrict__ F,
                                const double *__restrict__ T, int N, double a, SrcF64 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double z = pos[2 * N + i];
    const double s = H0(z / a);
    SrcF64 o;
    o.p = make_double2(pos[i], pos[N + i]);
    o.q = make_double2(fmax(z, a), F ? s * F[i] : 0.0);
    o.r = make_double2(F ? s * F[N + i] : 0.0, F ? s * F[2 * N + i] : 0.0);
    o.s = make_double2(T ? s * T[i] : 0.0, T ? s * T[N + i] : 0.0);
    o.u = make_double2(T ? s * T[2 * N + i] : 0.0, 0.0);
    out[i] = o;
}

// ------------------------------------------------------------------ pair kernels
// grid = (ceil(N/128), splits); block (bx, by) covers targets [128 bx, 128 bx + 128) and sources
// [by chunk, (by + 1) chunk); chunk is a multiple of 128, so the tile holding the block's own
// targets (where j == i can occur) is the one starting at 128 bx.
template <bool TORQUE>
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
                pair_velocity_f32<TORQUE>(rx, ry, tz, f.x, f.y, f.z, f.w, q.x, q.y, q.z, c, ux, uy, uz);
            }
        } else {
            for (int k = 0; k < cnt; ++k) {
                const float4 p = sp[k];
                const float4 f = sf[k];
                const float4 q = TORQUE ? st[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float rx = (tp.x - p.x) + (tp.z - p.z);
                const float ry = (tp.y - p.y) + (tp.w - p.w);
                float dx = 0.f, dy = 0.f, dz = 0.f;
                pair_velocity_f32<TORQUE>(rx, ry, tz, f.x, f.y, f.z, f.w, q.x, q.y, q.z, c, dx, dy, dz);
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
template <bool TORQUE>
__global__ void __launch_bounds__(kPairThreads) pair_f32x2_kernel(const SrcF32 *__restrict__ src, int N, int chunk,
                                                                   X2Consts c, double *__restrict__ part)
{
    constexpr int P = kTile / 2;
    __shared__ float4 sA[P], sB[P], sC[P], sD[P];
    __shared__ float4 sE[TORQUE ? P : 1];
    __shared__ float2 sG[TORQUE ? P : 1];
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
    const float2 txh = make_float2(tp.x, tp.x), tyh = make_float2(tp.y, tp.y);
    const float2 txl = make_float2(tp.z, tp.z), tyl = make_float2(tp.w, tp.w);
    const float2 tz2 = make_float2(tz, tz);
    const float2 zero2 = make_float2(0.f, 0.f);
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    const int diag = blockIdx.x * kTile;
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
                const float4 a = sA[k], b = sB[k], cc = sC[k], d = sD[k];
                const float4 e = TORQUE ? sE[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float2 g = TORQUE ? sG[k] : zero2;
                const float2 rx = add2(sub2(txh, make_float2(a.x, a.y)), sub2(txl, make_float2(b.x, b.y)));
                const float2 ry = add2(sub2(tyh, make_float2(a.z, a.w)), sub2(tyl, make_float2(b.z, b.w)));
                pair_velocity_x2<TORQUE>(rx, ry, tz2, make_float2(cc.x, cc.y), make_float2(cc.z, cc.w),
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
    if (i < N) {
        const size_t o = (size_t)blockIdx.y * 3 * N;
        part[o + i] = (double)sx - (double)cx;
        part[o + N + i] = (double)sy - (double)cy;
        part[o + 2 * N + i] = (double)sz - (double)cz;
    }
}

template <bool TORQUE>
__global__ void __launch_bounds__(kPairThreads) pair_f64_kernel(const SrcF64 *__restrict__ src, int N, int chunk,
                                                                 PairConsts<double> c, double *__restrict__ part)
{
    __shared__ double2 sp[kTile];
    __shared__ double2 sq[kTile];
    __shared__ double2 sr[kTile];
    __shared__ double2 ss[TORQUE ? kTile : 1];
    __shared__ double2 su[TORQUE ? kTile : 1];
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
    const int diag = blockIdx.x * kTile;
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
        if (base != diag) {
#pragma unroll 2
            for (int k = 0; k < cnt; ++k) {
                const double2 p = sp[k], q = sq[k], r = sr[k];
                const double2 s = TORQUE ? ss[k] : make_double2(0.0, 0.0);
                const double2 u = TORQUE ? su[k] : make_double2(0.0, 0.0);
                pair_velocity<double, TORQUE>(tp.x - p.x, tp.y - p.y, tz, q.x, q.y, r.x, r.y, s.x, s.y, u.x, c, ux, uy,
                                              uz);
            }
        } else {
            for (int k = 0; k < cnt; ++k) {
                const double2 p = sp[k], q = sq[k], r = sr[k];
                const double2 s = TORQUE ? ss[k] : make_double2(0.0, 0.0);
                const double2 u = TORQUE ? su[k] : make_double2(0.0, 0.0);
                double dx = 0.0, dy = 0.0, dz = 0.0;
                pair_velocity<double, TORQUE>(tp.x - p.x, tp.y - p.y, tz, q.x, q.y, r.x, r.y, s.x, s.y, u.x, c, dx, dy,
                                              dz);
                if (k != tid) {
                    ux += dx;
                    uy += dy;
                    uz += dz;
                }
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

// Sum the chunk partials in order, add the float64 self term, apply s_i / (8 pi eta).
__global__ void pair_reduce_kernel(const double *__restrict__ part, int splits, int N, const double *__restrict__ pos,
                                   const double *__restrict__ F, const double *__restrict__ T, PairConsts<double> c,
                                   double a, double scale, double *__restrict__ U)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int s = 0; s < splits; ++s) {
        const size_t o = (size_t)s * 3 * N;
        ux += part[o + i];
        uy += part[o + N + i];
        uz += part[o + 2 * N + i];
    }
    const double z = pos[2 * N + i];
    const double si = H0(z / a);
    const double zc = fmax(z, a);
    const double Fx = F ? si * F[i] : 0.0, Fy = F ? si * F[N + i] : 0.0, Fz = F ? si * F[2 * N + i] : 0.0;
    if (T) {
        pair_velocity<double, true>(0.0, 0.0, zc, zc, Fx, Fy, Fz, si * T[i], si * T[N + i], si * T[2 * N + i], c, ux,
                                    uy, uz);
    } else {
        pair_velocity<double, false>(0.0, 0.0, zc, zc, Fx, Fy, Fz, 0.0, 0.0, 0.0, c, ux, uy, uz);
    }
    const double k = si * scale;
    U[i] = k * ux;
    U[N + i] = k * uy;
    U[2 * N + i] = k * uz;
}

static int target_blocks(int num_sms)
{
    return num_sms * 8;
}

void pair_grid(int64_t N, int num_sms, int precision, int *splits, int64_t *chunk)
{
    (void)precision;
    const int64_t tiles = (N + kTile - 1) / kTile;
    int64_t S = (target_blocks(num_sms) + tiles - 1) / tiles;
    if (S > tiles) S = tiles;
    if (S < 1) S = 1;
    int64_t ch = ((N + S - 1) / S + kTile - 1) / kTile * kTile;
    if (ch < kTile) ch = kTile;
    *chunk = ch;
    *splits = (int)((N + ch - 1) / ch);
}

size_t pair_partial_bytes(int64_t max_N, int num_sms)
{
    const int64_t tiles = (max_N + kTile - 1) / kTile;
    return (size_t)3 * sizeof(double) * (size_t)(target_blocks(num_sms) + tiles + 1) * kTile;
}

int mobility_apply_impl(rpb_ctx *ctx, int64_t N64, const double *pos, const double *F, const double *T, double *U)
{
    const int N = (int)N64;
    cudaStream_t st = ctx->stream;
    const double a = ctx->p.a;
    int splits;
    int64_t chunk;
    pair_grid(N64, ctx->num_sms, ctx->p.precision, &splits, &chunk);
    if ((size_t)splits * 3 * N * sizeof(double) > ctx->ws.partial_bytes) {
        set_error("internal: pair partial buffer too small (N=%d splits=%d)", N, splits);
        return RPB_EINVAL;
    }
    double *part = (double *)ctx->ws.partial;
    const int pb = 256;
    const dim3 grid((unsigned)((N + kPairThreads - 1) / kPairThreads), (unsigned)splits);
    const bool torque = T != nullptr;
    if (ctx->p.precision == RPB_FP32) {
        SrcF32 *src = (SrcF32 *)ctx->ws.src;
        pack_f32_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, F, T, N, a, src);
        if (ctx->fp32_variant == 1) {
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
        pack_f64_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, F, T, N, a, src);
        const PairConsts<double> c = make_consts<double>(a);
        if (torque)
            pair_f64_kernel<true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
        else
            pair_f64_kernel<false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
    }
    const PairConsts<double> cd = make_consts<double>(a);
    pair_reduce_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(part, splits, N, pos, F, T, cd, a,
                                                          1.0 / (8.0 * kPi * ctx->p.eta), U);
    count_launches(3);
    return cuda_fail(cudaGetLastError(), "pair kernels");
}

// ------------------------------------------------------------------ forces (Sec. III)
// F_i = -weight z + sum_j f(|r_ij|) r_ij/|r_ij| + f_wall(z_i) z with f = -dU/dr of Eq. (soft_potential).
// Pairs are screened in float32 against a cutoff with a generous margin; the ones inside are
// evaluated in float64.
__global__ void __launch_bounds__(128) forces_kernel(const double *__restrict__ pos, int N, double a, double weight,
                                                     double U0, double b, float cut2, double *__restrict__ F)
{
    __shared__ double sx[128], sy[128], sz[128];
    __shared__ float fxs[128], fys[128], fzs[128];
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
    for (int base = 0; base < N; base += 128) {
        const int j = base + tid;
        if (j < N) {
            sx[tid] = pos[j];
            sy[tid] = pos[N + j];
            sz[tid] = pos[2 * N + j];
            fxs[tid] = (float)sx[tid];
            fys[tid] = (float)sy[tid];
            fzs[tid] = (float)sz[tid];
        }
        __syncthreads();
        const int cnt = min(128, N - base);
        for (int k = 0; k < cnt; ++k) {
            const float dxf = xf - fxs[k], dyf = yf - fys[k], dzf = zf - fzs[k];
            if (dxf * dxf + dyf * dyf + dzf * dzf < cut2 && base + k != i) {
                const double dx = xi - sx[k], dy = yi - sy[k], dz = zi - sz[k];
                const double r = sqrt(dx * dx + dy * dy + dz * dz);
                if (r > 0.0) {
                    const double m = (r < 2.0 * a ? f0 : f0 * exp(-(r - 2.0 * a) / b)) / r;
                    fx += m * dx;
                    fy += m * dy;
                    fz += m * dz;
                }
            }
        }
        __syncthreads();
    }
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
    const double rc = 2.0 * a + 50.0 * fp->b;
    const double rcm = rc * 1.01 + 0.01 * a;
    const float cut2 = (float)(rcm * rcm);
    forces_kernel<<<(unsigned)((N + 127) / 128), 128, 0, ctx->stream>>>(pos, (int)N, a, fp->weight, fp->U0, fp->b,
                                                                          cut2, F);
    count_launches(1);
    return cuda_fail(cudaGetLastError(), "forces kernel");
}

}  // namespace rpb

// ------------------------------------------------------------------ allocation-free product
// rpb_mobility_apply_noalloc: the same pack / pair / reduce kernels as rpb_mobility_apply, with their
// scratch (packed sources, then the per-chunk partial sums) in a fixed array of the library's device
// image instead of a context's cudaMalloc'd workspace.  The array is created with the module on
// every device that loads the library and lives until the process exits.
#include <mutex>

namespace rpb {

constexpr int64_t kNoAllocSrcBytes = (int64_t)RPB_NOALLOC_MAX_N * (int64_t)sizeof(SrcF64);
constexpr int64_t kNoAllocPartialElems = (int64_t)16 * 3 * RPB_NOALLOC_MAX_N;  // 16 chunks at the maximum N
constexpr int64_t kNoAllocBytes = kNoAllocSrcBytes + kNoAllocPartialElems * (int64_t)sizeof(double);
static_assert(kNoAllocSrcBytes % 256 == 0, "partials must start 256-byte aligned");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[kNoAllocMaxDevices];
static int g_noalloc_sms[kNoAllocMaxDevices];

// Device address of the scratch array on the current device (looked up once per device).
static int noalloc_setup(void **ptr, int *sms)
{
    int dev = 0;
    int rc;
    if ((rc = cuda_fail(cudaGetDevice(&dev), "cudaGetDevice"))) return rc;
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("device ordinal %d outside [0, %d)", dev, kNoAllocMaxDevices);
        return RPB_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if ((rc = cuda_fail(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)"))) return rc;
        int n = 0;
        if ((rc = cuda_fail(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev), "SM count"))) return rc;
        g_noalloc_sms[dev] = n;
        g_noalloc_ptr[dev] = p;
    }
    *ptr = g_noalloc_ptr[dev];
    *sms = g_noalloc_sms[dev];
    return RPB_OK;
}

}  // namespace rpb

extern "C" int rpb_mobility_apply_noalloc(int64_t N64, const double *pos, const double *F, const double *T, double *U,
                                          const rpb_params *p, void *stream)
{
    using namespace rpb;
    if (!p || !(p->a > 0.0) || !(p->eta > 0.0) || (p->precision != RPB_FP64 && p->precision != RPB_FP32)) {
        set_error("rpb_mobility_apply_noalloc: missing or bad parameters");
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
    if ((rc = noalloc_setup(&base, &sms))) return rc;
    int splits;
    int64_t chunk;
    pair_grid(N64, sms, p->precision, &splits, &chunk);
    const int64_t max_splits = kNoAllocPartialElems / (3 * N64);
    if (splits > max_splits) {
        chunk = ((N64 + max_splits - 1) / max_splits + kTile - 1) / kTile * kTile;
        splits = (int)((N64 + chunk - 1) / chunk);
    }
    double *part = (double *)((unsigned char *)base + kNoAllocSrcBytes);
    const int pb = 256;
    const dim3 grid((unsigned)((N + kPairThreads - 1) / kPairThreads), (unsigned)splits);
    const double a = p->a;
    if (p->precision == RPB_FP32) {
        SrcF32 *src = (SrcF32 *)base;
        pack_f32_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, F, T, N, a, src);
        const PairConsts<float> c = make_consts<float>(a);
        if (T)
            pair_f32_kernel<true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
        else
            pair_f32_kernel<false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
    } else {
        SrcF64 *src = (SrcF64 *)base;
        pack_f64_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(pos, F, T, N, a, src);
        const PairConsts<double> c = make_consts<double>(a);
        if (T)
            pair_f64_kernel<true><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
        else
            pair_f64_kernel<false><<<grid, kPairThreads, 0, st>>>(src, N, (int)chunk, c, part);
    }
    pair_reduce_kernel<<<(N + pb - 1) / pb, pb, 0, st>>>(part, splits, N, pos, F, T, make_consts<double>(a), a,
                                                          1.0 / (8.0 * kPi * p->eta), U);
    count_launches(3);
    return cuda_fail(cudaGetLastError(), "rpb_mobility_apply_noalloc kernels");
}
