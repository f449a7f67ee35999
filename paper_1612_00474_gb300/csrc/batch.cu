// batch.cu -- one call advances many independent suspensions of different sizes (a ragged batch).
//
// The caller keeps each suspension's state in its own device buffers; a call gathers them into a
// packed structure-of-arrays layout (instance b occupies spheres [off_b, off_b + N_b)), runs every
// stage of the step for all instances at once, and scatters the results back.  Per-instance
// quantities (seed, step counter, Lanczos state, convergence) are kept separately, and the work of
// an instance (its target blocks, its source tiles, its reductions) is laid out the same way
// whatever else is in the batch, so an instance's result does not depend on its companions.
//
//   pair products : one 128-target block of one instance per CTA, all of that instance's sources
//                   in 128-source tiles; the float64 self term and s_i/(8 pi eta) in the epilogue.
//   Lanczos       : per-instance dot products / Gram-Schmidt (one CTA per instance), one warp per
//                   instance for the tridiagonal step, instances drop out as they converge.
//   noise         : Philox keyed by each instance's seed, counter (k/2, step_b, stream, 0) -- the
//                   same numbers the single-suspension path draws for that seed and step.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lanczos_math.cuh"
#include "pair_math.cuh"

namespace rpb {

struct InstDesc {
    int64_t off;      // first sphere in the packed layout
    int N;            // spheres
    int first;        // 1: first step of this instance (Euler-Maruyama)
    uint32_t seed_lo, seed_hi, step, pad;
    double *pos;      // caller's buffers (SoA, 3N), or null
    double *aux;      // U_prev (step) or F (product)
    double *aux2;     // T (product)
    double *out;      // U (product)
};

struct BlockDesc {
    int inst;
    int first;  // first target (instance-local) of this 128-target block
};

constexpr int kBThreads = 256;

// ------------------------------------------------------------------ layout kernels
__global__ void inst_of_kernel(const InstDesc *__restrict__ inst, int B, int *__restrict__ inst_of)
{
    const int b = blockIdx.x;
    if (b >= B) return;
    const InstDesc d = inst[b];
    for (int i = threadIdx.x; i < d.N; i += blockDim.x) inst_of[d.off + i] = b;
}

// Copy (or write back) three-component SoA vectors between the callers' buffers and the packed
// layout.  which: 0 = pos, 1 = aux, 2 = aux2, 3 = out.
__global__ void gather_kernel(const InstDesc *__restrict__ inst, const int *__restrict__ inst_of, int64_t total,
                              int which, double *__restrict__ packed, int to_caller)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < 3 * total; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = r / total, i = r - c * total;
        const InstDesc &d = inst[inst_of[i]];
        double *p = which == 0 ? d.pos : (which == 1 ? d.aux : (which == 2 ? d.aux2 : d.out));
        const int64_t k = c * d.N + (i - d.off);
        if (to_caller)
            p[k] = packed[r];
        else
            packed[r] = p ? p[k] : 0.0;
    }
}

// ------------------------------------------------------------------ pair products
template <bool TORQUE>
__global__ void __launch_bounds__(kPairThreads, 6) batch_pair_f32x2_kernel(
    const SrcF32 *__restrict__ src, const InstDesc *__restrict__ inst, const BlockDesc *__restrict__ blocks,
    const int *__restrict__ active, int64_t total, X2Consts c, PairConsts<double> cd, double a, double scale,
    const double *__restrict__ pos, const double *__restrict__ F, const double *__restrict__ T, double *__restrict__ U)
{
    constexpr int P = kTile / 2;
    __shared__ float4 sA[P], sB[P], sC[P], sD[P];
    __shared__ float4 sE[TORQUE ? P : 1];
    __shared__ float2 sG[TORQUE ? P : 1];
    const BlockDesc bd = blocks[blockIdx.x];
    if (active && !active[bd.inst]) return;
    const InstDesc d = inst[bd.inst];
    const int tid = threadIdx.x;
    const int il = bd.first + tid;
    const int64_t i = d.off + il;
    const bool valid = il < d.N;
    float4 tp = make_float4(0.f, 0.f, 0.f, 0.f);
    float tz = 1.f;
    if (valid) {
        tp = src[i].p;
        tz = src[i].f.x;
    }
    const float2 txh = make_float2(tp.x, tp.x), tyh = make_float2(tp.y, tp.y);
    const float2 txl = make_float2(tp.z, tp.z), tyl = make_float2(tp.w, tp.w);
    const float2 tz2 = make_float2(tz, tz);
    const float2 zero2 = make_float2(0.f, 0.f);
    float sx = 0.f, sy = 0.f, sz = 0.f, cx = 0.f, cy = 0.f, cz = 0.f;
    const int pp = tid >> 1, hh = tid & 1;
    float *fA = reinterpret_cast<float *>(sA);
    float *fB = reinterpret_cast<float *>(sB);
    float *fC = reinterpret_cast<float *>(sC);
    float *fD = reinterpret_cast<float *>(sD);
    float *fE = reinterpret_cast<float *>(sE);
    float *fG = reinterpret_cast<float *>(sG);
    for (int base = 0; base < d.N; base += kTile) {
        const int jl = base + tid;
        float4 sp_ = make_float4(1e18f, 0.f, 0.f, 0.f), sf_ = make_float4(1.f, 0.f, 0.f, 0.f);
        float4 st_ = make_float4(0.f, 0.f, 0.f, 0.f);
        if (jl < d.N) {
            sp_ = src[d.off + jl].p;
            sf_ = src[d.off + jl].f;
            if (TORQUE) st_ = src[d.off + jl].t;
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
        const bool diag = base == bd.first;
        for (int k = 0; k < P; ++k) {
            const float4 av = sA[k], bv = sB[k], cc = sC[k], dv = sD[k];
            const float4 e = TORQUE ? sE[k] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float2 g = TORQUE ? sG[k] : zero2;
            // instances are small (every warp iteration has some pair within 10a), so the low parts
            // of the positions are always added
            const float2 rx = add2(sub2(txh, make_float2(av.x, av.y)), sub2(txl, make_float2(bv.x, bv.y)));
            const float2 ry = add2(sub2(tyh, make_float2(av.z, av.w)), sub2(tyl, make_float2(bv.z, bv.w)));
            float2 dx = zero2, dy = zero2, dz = zero2;
            pair_velocity_x2<TORQUE>(rx, ry, tz2, make_float2(cc.x, cc.y), make_float2(cc.z, cc.w),
                                     make_float2(dv.x, dv.y), make_float2(dv.z, dv.w), make_float2(e.x, e.y),
                                     make_float2(e.z, e.w), g, c, dx, dy, dz);
            if (diag && k == pp) {  // source 2k + hh of the diagonal tile is this thread's sphere
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
    if (valid) {
        double ux = (double)sx - (double)cx, uy = (double)sy - (double)cy, uz = (double)sz - (double)cz;
        const double z = pos[2 * total + i];
        const double si = H0(z / a), zc = fmax(z, a);
        const double Fx = F ? si * F[i] : 0.0, Fy = F ? si * F[total + i] : 0.0, Fz = F ? si * F[2 * total + i] : 0.0;
        if (TORQUE)
            self_velocity<true>(zc, Fx, Fy, Fz, si * T[i], si * T[total + i], cd, ux, uy, uz);
        else
            self_velocity<false>(zc, Fx, Fy, Fz, 0.0, 0.0, cd, ux, uy, uz);
        const double k = si * scale;
        U[i] = k * ux;
        U[total + i] = k * uy;
        U[2 * total + i] = k * uz;
    }
}

template <bool TORQUE>
__global__ void __launch_bounds__(kPairThreads) batch_pair_f64_kernel(
    const SrcF64 *__restrict__ src, const InstDesc *__restrict__ inst, const BlockDesc *__restrict__ blocks,
    const int *__restrict__ active, int64_t total, PairConsts<double> c, double a, double scale,
    const double *__restrict__ pos, const double *__restrict__ F, const double *__restrict__ T, double *__restrict__ U)
{
    __shared__ double2 sp[kTile], sq[kTile], sr[kTile];
    __shared__ double2 ss[TORQUE ? kTile : 1], su[TORQUE ? kTile : 1];
    const BlockDesc bd = blocks[blockIdx.x];
    if (active && !active[bd.inst]) return;
    const InstDesc d = inst[bd.inst];
    const int tid = threadIdx.x;
    const int il = bd.first + tid;
    const int64_t i = d.off + il;
    const bool valid = il < d.N;
    double2 tp = make_double2(0.0, 0.0);
    double tz = 1.0;
    if (valid) {
        tp = src[i].p;
        tz = src[i].q.x;
    }
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int base = 0; base < d.N; base += kTile) {
        const int jl = base + tid;
        if (jl < d.N) {
            const SrcF64 s = src[d.off + jl];
            sp[tid] = s.p;
            sq[tid] = s.q;
            sr[tid] = s.r;
            if (TORQUE) {
                ss[tid] = s.s;
                su[tid] = s.u;
            }
        }
        __syncthreads();
        const int cnt = min(kTile, d.N - base);
        const bool diag = base == bd.first;
        for (int k = 0; k < cnt; ++k) {
            const double2 p = sp[k], q = sq[k], r = sr[k];
            const double2 s = TORQUE ? ss[k] : make_double2(0.0, 0.0);
            const double2 u = TORQUE ? su[k] : make_double2(0.0, 0.0);
            double dx = 0.0, dy = 0.0, dz = 0.0;
            pair_velocity_f64<TORQUE>(tp.x - p.x, tp.y - p.y, tz, q.x, q.y, r.x, r.y, s.x, s.y, u.x, c, dx, dy, dz);
            if (!(diag && k == tid)) {
                ux += dx;
                uy += dy;
                uz += dz;
            }
        }
        __syncthreads();
    }
    if (valid) {
        const double z = pos[2 * total + i];
        const double si = H0(z / a), zc = fmax(z, a);
        const double Fx = F ? si * F[i] : 0.0, Fy = F ? si * F[total + i] : 0.0, Fz = F ? si * F[2 * total + i] : 0.0;
        if (TORQUE)
            self_velocity<true>(zc, Fx, Fy, Fz, si * T[i], si * T[total + i], c, ux, uy, uz);
        else
            self_velocity<false>(zc, Fx, Fy, Fz, 0.0, 0.0, c, ux, uy, uz);
        const double k = si * scale;
        U[i] = k * ux;
        U[total + i] = k * uy;
        U[2 * total + i] = k * uz;
    }
}

// Forces of Sec. III within each instance (same screening as the single-suspension kernel).
// Pairs farther apart than 2a + kFarB b, whose repulsion is below e^-kFarB U0/b (~2e-9 U0/b), take it
// in float32 (IEEE square root and division, expf: a relative error of a few 1e-6 on a term that small
// is below 1e-14 U0/b) and are summed in float32 before their total joins the float64 sum; nearer
// pairs are evaluated in float64.  The two kinds are queued apart so that a warp runs the float64 loop
// only as long as its longest near queue (a float64 warp instruction costs the same whatever the
// number of active lanes).
constexpr float kFarB = 20.f;

__global__ void __launch_bounds__(128) batch_forces_kernel(const double *__restrict__ pos, const InstDesc *__restrict__ inst,
                                                           const BlockDesc *__restrict__ blocks, int64_t total, double a,
                                                           double weight, double U0, double b, float cut2,
                                                           float near2, double *__restrict__ F)
{
    // the screen of forces_kernel, within the block's own instance: the float32 screen takes two
    // sources per lane (packed); near pairs are queued from the front of one array, far pairs from its
    // back, and each kind is evaluated together, in index order
    __shared__ float4 sp[64];
    __shared__ float2 sz[64];
    const BlockDesc bd = blocks[blockIdx.x];
    const InstDesc d = inst[bd.inst];
    const int tid = threadIdx.x;
    const int il = bd.first + tid;
    const int64_t i = d.off + il;
    const bool valid = il < d.N;
    double xi = 0.0, yi = 0.0, zi = 0.0;
    if (valid) {
        xi = pos[i];
        yi = pos[total + i];
        zi = pos[2 * total + i];
    }
    const float xf = (float)xi, yf = (float)yi, zf = (float)zi;
    const double f0 = U0 / b, inv_b = 1.0 / b;
    const float f0f = (float)f0, inv_bf = (float)inv_b, two_af = (float)(2.0 * a);
    double fx = 0.0, fy = 0.0, fz = 0.0;
    float gx = 0.f, gy = 0.f, gz = 0.f;  // far pairs
    constexpr int kQ = 32;
    int queue[kQ];
    int nn = 0, nf = 0;  // near pairs at queue[0 .. nn), far pairs at queue[kQ - nf .. kQ)
    auto flush = [&]() {
        for (int q = 0; q < nn; ++q) {
            const int64_t j = d.off + queue[q];
            const double dx = xi - pos[j], dy = yi - pos[total + j], dz = zi - pos[2 * total + j];
            const double m = steric_pair_factor(dx * dx + dy * dy + dz * dz, 2.0 * a, f0, inv_b);
            fx += m * dx;
            fy += m * dy;
            fz += m * dz;
        }
        for (int q = kQ - nf; q < kQ; ++q) {
            const int64_t j = d.off + queue[q];
            const float dx = (float)(xi - pos[j]), dy = (float)(yi - pos[total + j]), dz = (float)(zi - pos[2 * total + j]);
            const float r = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
            const float m = f0f * expf((two_af - r) * inv_bf) / r;
            gx = fmaf(m, dx, gx);
            gy = fmaf(m, dy, gy);
            gz = fmaf(m, dz, gz);
        }
        nn = 0;
        nf = 0;
    };
    float *fxy = reinterpret_cast<float *>(sp);
    float *fz2 = reinterpret_cast<float *>(sz);
    const float2 X = make_float2(xf, xf), Y = make_float2(yf, yf), Z = make_float2(zf, zf);
    const int pp = tid >> 1, hh = tid & 1;
    for (int base = 0; base < d.N; base += 128) {
        const int jl = base + tid;
        const int64_t jt = d.off + jl;
        // slots past the instance's end hold a point far above the wall (never inside the screen)
        const bool in = jl < d.N;
        fxy[4 * pp + hh] = in ? (float)pos[jt] : 0.f;
        fxy[4 * pp + 2 + hh] = in ? (float)pos[total + jt] : 0.f;
        fz2[2 * pp + hh] = in ? (float)pos[2 * total + jt] : 1e18f;
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 64; ++k) {
            const float4 p = sp[k];
            const float2 dx = sub2(X, make_float2(p.x, p.y)), dy = sub2(Y, make_float2(p.z, p.w));
            const float2 dz = sub2(Z, sz[k]);
            const float2 d2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
            if (d2.x < cut2 || d2.y < cut2) {
                const int j0 = base + 2 * k;
                if (d2.x < cut2 && j0 != il && j0 < d.N) {
                    if (d2.x < near2)
                        queue[nn++] = j0;
                    else
                        queue[kQ - ++nf] = j0;
                    if (nn + nf == kQ) flush();
                }
                if (d2.y < cut2 && j0 + 1 != il && j0 + 1 < d.N) {
                    if (d2.y < near2)
                        queue[nn++] = j0 + 1;
                    else
                        queue[kQ - ++nf] = j0 + 1;
                    if (nn + nf == kQ) flush();
                }
            }
        }
        __syncthreads();
    }
    flush();
    if (valid) {
        fz += (zi < a ? f0 : f0 * exp(-(zi - a) / b)) - weight;
        F[i] = fx + (double)gx;
        F[total + i] = fy + (double)gy;
        F[2 * total + i] = fz + (double)gz;
    }
}

// ------------------------------------------------------------------ noise and elementwise steps
__device__ __forceinline__ uint4 philox4x32_10_b(uint4 c, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
        const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Element (c, i) of the packed vector: normal k = 3 il + c of instance inst_of[i] (il local index).
__global__ void batch_philox_kernel(const InstDesc *__restrict__ inst, const int *__restrict__ inst_of, int64_t total,
                                    uint32_t sid, double *__restrict__ out)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < 3 * total; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = r / total, i = r - c * total;
        const InstDesc &d = inst[inst_of[i]];
        const int64_t k = 3 * (i - d.off) + c;
        const uint4 w = philox4x32_10_b(make_uint4((uint32_t)(k >> 1), d.step, sid, 0u), d.seed_lo, d.seed_hi);
        const double two26 = 67108864.0, two_m53 = 1.1102230246251565e-16;
        const double u1 = ((double)(w.x >> 5) * two26 + (double)(w.y >> 6) + 1.0) * two_m53;
        const double u2 = ((double)(w.z >> 5) * two26 + (double)(w.w >> 6) + 1.0) * two_m53;
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        out[r] = sqrt(-2.0 * log(u1)) * ((k & 1) ? sn : cs);
    }
}

__global__ void batch_ab_update_kernel(const InstDesc *__restrict__ inst, const int *__restrict__ inst_of, int64_t total,
                                       double *__restrict__ pos, double *__restrict__ U_prev,
                                       const double *__restrict__ Un, const double *__restrict__ g,
                                       const double *__restrict__ drift, double dt, double noise_scale)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < 3 * total; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = r % total;
        const double un = Un[r];
        const double up = inst[inst_of[i]].first ? un : U_prev[r];
        pos[r] = pos[r] + dt * (1.5 * un - 0.5 * up) + noise_scale * g[r] + dt * drift[r];
        U_prev[r] = un;
    }
}

__global__ void batch_fill3_kernel(double *__restrict__ v, int64_t total, double x, double y, double z)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < 3 * total; r += (int64_t)gridDim.x * blockDim.x)
        v[r] = r < total ? x : (r < 2 * total ? y : z);
}

__global__ void batch_displace_kernel(const double *__restrict__ pos, const double *__restrict__ Wt, int64_t n, double h,
                                      double *__restrict__ plus, double *__restrict__ minus)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const double q = pos[r], dd = h * Wt[r];
        plus[r] = q + dd;
        minus[r] = q - dd;
    }
}

__global__ void batch_rfd_combine_kernel(double *__restrict__ up_drift, const double *__restrict__ um, int64_t n, double k)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        up_drift[r] = k * (up_drift[r] - um[r]);
}

// ------------------------------------------------------------------ batched Lanczos
__device__ __forceinline__ double block_sum_b(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    __syncthreads();
    return r;
}

// red[k * B + b] = <V[k], w> over instance b's 3 N_b rows; grid (B, nvec).
__global__ void __launch_bounds__(kBThreads) batch_dots_kernel(const double *__restrict__ V, size_t ld,
                                                               const double *__restrict__ w,
                                                               const InstDesc *__restrict__ inst,
                                                               const int *__restrict__ active, int64_t total, int B,
                                                               double *__restrict__ red)
{
    __shared__ double sh[kBThreads / 32];
    const int b = blockIdx.x;
    if (active && !active[b]) return;  // uniform per block
    const InstDesc d = inst[b];
    const double *v = V + (size_t)blockIdx.y * ld;
    double acc = 0.0;
    for (int c = 0; c < 3; ++c)
        for (int il = threadIdx.x; il < d.N; il += blockDim.x) {
            const int64_t r = c * total + d.off + il;
            acc = fma(v[r], w[r], acc);
        }
    acc = block_sum_b(acc, sh);
    if (threadIdx.x == 0) red[(size_t)blockIdx.y * B + b] = acc;
}

// w -= sum_k coef_k V[k] over instance b's rows (coef_k = red[k B + b]); block b also stores the
// coefficients in its state block (lz_b + coef_off) and, if norm_out, |w|^2 in norm_out[b].
__global__ void __launch_bounds__(kBThreads) batch_project_kernel(const double *__restrict__ V, size_t ld,
                                                                  double *__restrict__ w,
                                                                  const InstDesc *__restrict__ inst,
                                                                  const int *__restrict__ active, int64_t total, int B,
                                                                  int nvec, const double *__restrict__ red,
                                                                  double *__restrict__ lz, size_t lz_stride,
                                                                  size_t coef_off, double *__restrict__ norm_out)
{
    __shared__ double coef[kMaxIter + 1];
    __shared__ double sh[kBThreads / 32];
    const int b = blockIdx.x;
    if (active && !active[b]) return;
    const InstDesc d = inst[b];
    for (int k = threadIdx.x; k < nvec; k += blockDim.x) {
        coef[k] = red[(size_t)k * B + b];
        lz[(size_t)b * lz_stride + coef_off + k] = coef[k];
    }
    __syncthreads();
    double acc = 0.0;
    for (int c = 0; c < 3; ++c)
        for (int il = threadIdx.x; il < d.N; il += blockDim.x) {
            const int64_t r = c * total + d.off + il;
            double x = w[r];
            for (int k = 0; k < nvec; ++k) x -= coef[k] * V[(size_t)k * ld + r];
            w[r] = x;
            acc = fma(x, x, acc);
        }
    if (norm_out) {
        acc = block_sum_b(acc, sh);
        if (threadIdx.x == 0) norm_out[b] = acc;
    }
}

// |W_b| per instance from red[b] (the squared norms); v_0 scale factors; activity.
__global__ void batch_norm_init_kernel(const double *__restrict__ red, int B, double *__restrict__ lz, size_t lz_stride,
                                       size_t status_off, int *__restrict__ active)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
        double *st = lz + (size_t)b * lz_stride + status_off;
        const double nw = sqrt(red[b]);
        st[ST_NW] = nw;
        st[ST_INV_NW] = nw > 0.0 ? 1.0 / nw : 0.0;
        st[ST_EPS] = -1.0;
        st[ST_STOP] = nw > 0.0 ? 0.0 : 1.0;
        st[ST_BREAK] = 0.0;
        st[6] = 0.0;  // m (iterations used)
        st[7] = nw > 0.0 ? 0.0 : 1.0;  // converged flag
        active[b] = nw > 0.0 ? 1 : 0;
    }
}

// v[r] = w[r] * status_b[idx] for rows of active instances (all instances when active is null).
__global__ void batch_scale_kernel(const double *__restrict__ w, const InstDesc *__restrict__ inst,
                                   const int *__restrict__ inst_of, const int *__restrict__ active, int64_t total,
                                   const double *__restrict__ lz, size_t lz_stride, size_t status_off, int idx,
                                   double *__restrict__ v)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < 3 * total; r += (int64_t)gridDim.x * blockDim.x) {
        const int b = inst_of[r % total];
        if (active && !active[b]) continue;
        v[r] = w[r] * lz[(size_t)b * lz_stride + status_off + idx];
    }
}

// One warp per instance (4 per block): the tridiagonal step; converged instances leave the active set.
__global__ void __launch_bounds__(128) batch_tail_kernel(double *__restrict__ lz, size_t lz_stride, LzLayout L, int k,
                                                         double tol, const double *__restrict__ norm2, int B,
                                                         int *__restrict__ active, int *__restrict__ n_active)
{
    __shared__ double q0[4][kMaxIter];
    __shared__ double sl[4][kMaxIter];
    __shared__ double red[4][32];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * 4 + wid;
    if (b >= B || !active[b]) return;  // whole warp leaves together
    double *lzb = lz + (size_t)b * lz_stride;
    lanczos_tail_warp(lzb, L, k, tol, lzb[L.c1 + k] + lzb[L.c2 + k], sqrt(norm2[b]), q0[wid], sl[wid], red[wid]);
    __syncwarp();
    if (lane == 0) {
        double *st = lzb + L.status;
        st[6] = k + 1;
        if (st[ST_STOP] != 0.0) {
            st[7] = 1.0;
            active[b] = 0;
        } else {
            atomicAdd(n_active, 1);
        }
    }
}

// g[r] = sum_{k < m_b} y_b[k] V[k][r]
__global__ void batch_combine_kernel(const double *__restrict__ V, size_t ld, const int *__restrict__ inst_of,
                                     int64_t total, const double *__restrict__ lz, size_t lz_stride, LzLayout L,
                                     double *__restrict__ g)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < 3 * total; r += (int64_t)gridDim.x * blockDim.x) {
        const double *lzb = lz + (size_t)inst_of[r % total] * lz_stride;
        const int m = (int)lzb[L.status + 6];
        double acc = 0.0;
        for (int k = 0; k < m; ++k) acc = fma(lzb[L.y + k], V[(size_t)k * ld + r], acc);
        g[r] = acc;
    }
}

}  // namespace rpb

using namespace rpb;

struct rpb_batch {
    rpb_params p;
    int64_t max_total;
    int max_B;
    int max_iter;
    cudaStream_t stream;
    int num_sms;
    size_t lz_stride;
    // device
    InstDesc *d_inst = nullptr;
    BlockDesc *d_blocks = nullptr;
    int *d_inst_of = nullptr;
    int *d_active = nullptr;
    int *d_nactive = nullptr;
    void *src = nullptr;
    double *vec[12] = {};  // pos, Up, F, T, Un, W, Wt, g, drift, pos_a, pos_b, w
    double *V = nullptr;
    double *lz = nullptr;
    double *red = nullptr;
    double *norm2 = nullptr;
    // host (pinned)
    InstDesc *h_inst = nullptr;
    BlockDesc *h_blocks = nullptr;
    int *h_nactive = nullptr;
    double *h_lz = nullptr;
    int64_t total = 0;
    int B = 0;
    int nblocks = 0;
    // multi-step runs: a private stream to capture and replay the step graph on, joined to the
    // caller's stream by an event; a device counter of unconverged instance-steps
    cudaStream_t cap = nullptr;
    cudaStream_t loop = nullptr;  // the WHILE node's body (a step) is captured here
    int *d_left = nullptr;        // steps left in the run
    cudaEvent_t join = nullptr;
    unsigned long long *d_unconv = nullptr;
    unsigned long long *h_unconv = nullptr;
    // graph-replayed Lanczos: iterations after the first run inside conditional (IF) nodes of the
    // graph, captured on `body`; d_iter_runs[k] counts how often iteration k ran (for the launch
    // count), iter_launches[k] is the number of kernels of iteration k's body
    cudaStream_t body = nullptr;
    unsigned long long *d_iter_runs = nullptr;
    unsigned long long *h_iter_runs = nullptr;
    int iter_launches[kMaxIter] = {};
    // float32 products by the symmetric pass (both directions of a pair from one evaluation):
    // schedule and partial-sum scratch for the current batch sizes
    bool sym_enabled = false;
    bool sym_ok = false;
    BatchSymPlan sym;
    int seg_tiles = 8;  // run length of the symmetric pass's row cut (rpb_batch_set_tiles / rpb_batch_tune)
    int sym_env = 1;    // RPB_FP32_BATCH_SYM (the symmetric pass unless "0")
};

namespace rpb {

enum { V_POS, V_UP, V_F, V_T, V_UN, V_W, V_WT, V_G, V_DRIFT, V_PA, V_PB, V_WORK };

static void batch_free(rpb_batch *bt)
{
    void *dev[] = {bt->d_inst, bt->d_blocks, bt->d_inst_of, bt->d_active, bt->d_nactive, bt->src, bt->V, bt->lz, bt->red,
                   bt->norm2, bt->d_left};
    for (void *p : dev)
        if (p) cudaFree(p);
    for (double *p : bt->vec)
        if (p) cudaFree(p);
    void *host[] = {bt->h_inst, bt->h_blocks, bt->h_nactive, bt->h_lz, bt->h_unconv};
    for (void *p : host)
        if (p) cudaFreeHost(p);
    if (bt->d_unconv) cudaFree(bt->d_unconv);
    if (bt->d_iter_runs) cudaFree(bt->d_iter_runs);
    if (bt->h_iter_runs) cudaFreeHost(bt->h_iter_runs);
    if (bt->body) cudaStreamDestroy(bt->body);
    batch_sym_free(bt->sym);
    if (bt->join) cudaEventDestroy(bt->join);
    if (bt->cap) cudaStreamDestroy(bt->cap);
    if (bt->loop) cudaStreamDestroy(bt->loop);
}

static int grid_for(int64_t n, int sms)
{
    int64_t g = (n + 255) / 256;
    if (g > 16 * (int64_t)sms) g = 16 * sms;
    return g < 1 ? 1 : (int)g;
}

// Describe the batch on the host and copy the descriptors to the device.  Blocks are listed
// largest instance first so that the long CTAs start early.
static int batch_setup(rpb_batch *bt, int B, const int64_t *N, const int64_t *steps, const uint64_t *seeds,
                       double *const *pos, double *const *aux, const double *const *aux2, double *const *out)
{
    if (B < 1 || B > bt->max_B) {
        set_error("batch size B=%d outside [1, %d]", B, bt->max_B);
        return RPB_EINVAL;
    }
    int64_t total = 0;
    for (int b = 0; b < B; ++b) {
        if (N[b] <= 0 || N[b] > (int64_t)1 << 30) {
            set_error("instance %d: N=%lld invalid", b, (long long)N[b]);
            return RPB_EINVAL;
        }
        total += N[b];
    }
    if (total > bt->max_total) {
        set_error("batch of %lld spheres exceeds the context's max_total_N=%lld", (long long)total,
                  (long long)bt->max_total);
        return RPB_EINVAL;
    }
    int64_t off = 0;
    int nblk = 0;
    for (int b = 0; b < B; ++b) {
        InstDesc &d = bt->h_inst[b];
        d.off = off;
        d.N = (int)N[b];
        d.first = steps ? (steps[b] == 0) : 0;
        const uint64_t s = seeds ? seeds[b] : 0;
        d.seed_lo = (uint32_t)(s & 0xffffffffu);
        d.seed_hi = (uint32_t)(s >> 32);
        d.step = steps ? (uint32_t)steps[b] : 0u;
        d.pad = 0;
        d.pos = pos ? pos[b] : nullptr;
        d.aux = aux ? aux[b] : nullptr;
        d.aux2 = aux2 ? const_cast<double *>(aux2[b]) : nullptr;
        d.out = out ? out[b] : nullptr;
        off += N[b];
        nblk += (int)((N[b] + kTile - 1) / kTile);
    }
    std::vector<int> order(B);
    for (int b = 0; b < B; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return N[x] > N[y]; });
    int k = 0;
    for (int b : order)
        for (int64_t f = 0; f < N[b]; f += kTile) bt->h_blocks[k++] = BlockDesc{b, (int)f};
    bt->total = total;
    bt->B = B;
    bt->nblocks = nblk;
    int rc;
    if ((rc = cuda_fail(cudaMemcpyAsync(bt->d_inst, bt->h_inst, B * sizeof(InstDesc), cudaMemcpyHostToDevice, bt->stream),
                        "batch descriptors")))
        return rc;
    if ((rc = cuda_fail(cudaMemcpyAsync(bt->d_blocks, bt->h_blocks, nblk * sizeof(BlockDesc), cudaMemcpyHostToDevice,
                                        bt->stream),
                        "batch blocks")))
        return rc;
    inst_of_kernel<<<B, 256, 0, bt->stream>>>(bt->d_inst, B, bt->d_inst_of);
    count_launches(1);
    if ((rc = cuda_fail(cudaGetLastError(), "inst_of"))) return rc;
    bt->sym_ok = false;
    if (bt->sym_enabled && (rc = batch_sym_plan(bt->sym, B, N, bt->stream, &bt->sym_ok, bt->seg_tiles))) return rc;
    return RPB_OK;
}

static int batch_gather(rpb_batch *bt, int which, double *packed, int to_caller)
{
    gather_kernel<<<grid_for(3 * bt->total, bt->num_sms), 256, 0, bt->stream>>>(bt->d_inst, bt->d_inst_of, bt->total,
                                                                               which, packed, to_caller);
    count_launches(1);
    return cuda_fail(cudaGetLastError(), "batch gather");
}

// U = M_tt F + M_tr T over the packed layout; F or T may be null; active masks instances.
static int batch_product(rpb_batch *bt, const double *pos, const double *F, const double *T, double *U,
                         const int *active)
{
    const int64_t total = bt->total;
    const double a = bt->p.a;
    const double scale = 1.0 / (8.0 * kPi * bt->p.eta);
    const int pb = 256;
    const int gpack = (int)((total + pb - 1) / pb);
    if (bt->p.precision == RPB_FP32 && bt->sym_ok) {
        SrcF32 *src = (SrcF32 *)bt->src;
        pack_f32_kernel<<<gpack, pb, 0, bt->stream>>>(pos, F, T, (int)total, a, 1, src);
        count_launches(1);
        return batch_sym_apply(bt->sym, bt->stream, src, total, pos, F, T, U, active, a, bt->p.eta);
    } else if (bt->p.precision == RPB_FP32) {
        SrcF32 *src = (SrcF32 *)bt->src;
        pack_f32_kernel<<<gpack, pb, 0, bt->stream>>>(pos, F, T, (int)total, a, 1, src);
        const X2Consts c = make_x2_consts(a);
        const PairConsts<double> cd = make_consts<double>(a);
        if (T)
            batch_pair_f32x2_kernel<true><<<bt->nblocks, kPairThreads, 0, bt->stream>>>(
                src, bt->d_inst, bt->d_blocks, active, total, c, cd, a, scale, pos, F, T, U);
        else
            batch_pair_f32x2_kernel<false><<<bt->nblocks, kPairThreads, 0, bt->stream>>>(
                src, bt->d_inst, bt->d_blocks, active, total, c, cd, a, scale, pos, F, T, U);
    } else {
        SrcF64 *src = (SrcF64 *)bt->src;
        pack_f64_kernel<<<gpack, pb, 0, bt->stream>>>(pos, F, T, (int)total, a, 1, src);
        const PairConsts<double> c = make_consts<double>(a);
        if (T)
            batch_pair_f64_kernel<true><<<bt->nblocks, kPairThreads, 0, bt->stream>>>(
                src, bt->d_inst, bt->d_blocks, active, total, c, a, scale, pos, F, T, U);
        else
            batch_pair_f64_kernel<false><<<bt->nblocks, kPairThreads, 0, bt->stream>>>(
                src, bt->d_inst, bt->d_blocks, active, total, c, a, scale, pos, F, T, U);
    }
    count_launches(2);
    return cuda_fail(cudaGetLastError(), "batch pair kernels");
}

// Inside a replayed graph: count this run of iteration k and, unless it is the last one, let the
// conditional node of iteration k + 1 run only while some instance is still active.
__global__ void batch_iter_kernel(cudaGraphConditionalHandle next, int has_next, const int *__restrict__ n_active,
                                  unsigned long long *__restrict__ runs_k)
{
    *runs_k += 1ull;
    if (has_next) cudaGraphSetConditional(next, *n_active > 0 ? 1u : 0u);
}

// Lanczos for every instance at once; per-instance m, eps and convergence land in h_lz statuses.
// graph == false: the host reads the number of still-active instances after every iteration and stops
// when it reaches zero, then copies the per-instance statuses to h_lz.  graph == true (inside a CUDA
// graph capture): iteration 0 is captured as is and iterations 1 .. max_iter - 1 each inside a
// conditional node that runs only while some instance is still active (the previous iteration's
// last kernel sets its condition), so a replay does the iterations the step needs, at most max_iter;
// converged instances are masked out of every kernel, and nothing is read back.
static int batch_lanczos(rpb_batch *bt, const double *pos, const double *W, double *g, double tol, int max_iter,
                         bool graph = false)
{
    cudaStream_t main_st = bt->stream;
    const int B = bt->B;
    const int64_t total = bt->total;
    const size_t ld = (size_t)3 * bt->max_total;
    const LzLayout L(bt->max_iter);
    double *V = bt->V, *w = bt->vec[V_WORK];
    const int ge = grid_for(3 * total, bt->num_sms);
    int rc;
    cudaGraphConditionalHandle hnd[kMaxIter] = {};
    if (graph) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t cg = nullptr;
        if ((rc = cuda_fail(cudaStreamGetCaptureInfo(main_st, &cs, nullptr, &cg, nullptr, nullptr, nullptr),
                            "capture info")))
            return rc;
        CondSet cs_all = {};
        for (int k = 1; k < max_iter; ++k) {
            if ((rc = cuda_fail(cudaGraphConditionalHandleCreate(&hnd[k], cg, 0u, cudaGraphCondAssignDefault),
                                "conditional handle")))
                return rc;
            cs_all.h[k - 1] = hnd[k];
        }
        // the iterations' conditions start at 0 in every step (the graph runs the step in a loop)
        if (max_iter > 1) {
            graph_reset_conds_kernel<<<1, 64, 0, main_st>>>(cs_all, max_iter - 1);
            count_launches(1);
        }
    }
    batch_dots_kernel<<<dim3(B, 1), kBThreads, 0, main_st>>>(W, 0, W, bt->d_inst, nullptr, total, B, bt->red);
    batch_norm_init_kernel<<<(B + 127) / 128, 128, 0, main_st>>>(bt->red, B, bt->lz, bt->lz_stride, L.status,
                                                                bt->d_active);
    batch_scale_kernel<<<ge, 256, 0, main_st>>>(W, bt->d_inst, bt->d_inst_of, nullptr, total, bt->lz, bt->lz_stride,
                                                L.status, ST_INV_NW, V);
    count_launches(3);
    for (int k = 0; k < max_iter; ++k) {
        const bool cond = graph && k >= 1;
        if (cond) {
            if ((rc = graph_begin_if(main_st, bt->body, hnd[k]))) return rc;
            bt->stream = bt->body;
        }
        cudaStream_t st = bt->stream;
        const uint64_t before = rpb_launch_count();
        const double *vk = V + (size_t)k * ld;
        rc = batch_product(bt, pos, vk, nullptr, w, bt->d_active);
        const int nv = k + 1;
        if (!rc) {
            batch_dots_kernel<<<dim3(B, nv), kBThreads, 0, st>>>(V, ld, w, bt->d_inst, bt->d_active, total, B, bt->red);
            batch_project_kernel<<<B, kBThreads, 0, st>>>(V, ld, w, bt->d_inst, bt->d_active, total, B, nv, bt->red,
                                                          bt->lz, bt->lz_stride, L.c1, nullptr);
            batch_dots_kernel<<<dim3(B, nv), kBThreads, 0, st>>>(V, ld, w, bt->d_inst, bt->d_active, total, B, bt->red);
            batch_project_kernel<<<B, kBThreads, 0, st>>>(V, ld, w, bt->d_inst, bt->d_active, total, B, nv, bt->red,
                                                          bt->lz, bt->lz_stride, L.c2, bt->norm2);
            rc = cuda_fail(cudaMemsetAsync(bt->d_nactive, 0, sizeof(int), st), "memset");
        }
        if (!rc) {
            batch_tail_kernel<<<(B + 3) / 4, 128, 0, st>>>(bt->lz, bt->lz_stride, L, k, tol, bt->norm2, B,
                                                           bt->d_active, bt->d_nactive);
            count_launches(5);
            if (graph) {
                const bool has_next = k + 1 < max_iter;
                batch_iter_kernel<<<1, 1, 0, st>>>(has_next ? hnd[k + 1] : 0ull, has_next ? 1 : 0, bt->d_nactive,
                                                   bt->d_iter_runs + k);
                count_launches(1);
            } else {
                if ((rc = cuda_fail(cudaMemcpyAsync(bt->h_nactive, bt->d_nactive, sizeof(int),
                                                    cudaMemcpyDeviceToHost, st),
                                    "n_active copy")))
                    return rc;
                if ((rc = cuda_fail(cudaStreamSynchronize(st), "batch lanczos iteration"))) return rc;
                if (*bt->h_nactive == 0) break;
            }
            if (k + 1 < max_iter) {
                batch_scale_kernel<<<ge, 256, 0, st>>>(w, bt->d_inst, bt->d_inst_of, bt->d_active, total, bt->lz,
                                                       bt->lz_stride, L.status, ST_INV_BETA, V + (size_t)(k + 1) * ld);
                count_launches(1);
            }
            rc = cuda_fail(cudaGetLastError(), "batch lanczos kernels");
        }
        if (cond) {
            bt->iter_launches[k] = (int)(rpb_launch_count() - before);
            cudaGraph_t body_graph = nullptr;
            const int erc = cuda_fail(cudaStreamEndCapture(bt->body, &body_graph), "body capture end");
            bt->stream = main_st;
            if (!rc) rc = erc;
        }
        if (rc) return rc;
    }
    batch_combine_kernel<<<ge, 256, 0, main_st>>>(V, ld, bt->d_inst_of, total, bt->lz, bt->lz_stride, L, g);
    count_launches(1);
    if (graph) return cuda_fail(cudaGetLastError(), "batch lanczos kernels");
    if ((rc = cuda_fail(cudaMemcpyAsync(bt->h_lz, bt->lz, (size_t)B * bt->lz_stride * sizeof(double),
                                        cudaMemcpyDeviceToHost, main_st),
                        "status copy")))
        return rc;
    return cuda_fail(cudaStreamSynchronize(main_st), "batch lanczos");
}

// After a step replayed from a CUDA graph: advance every instance's step counter and count the
// instances whose Lanczos did not converge within the fixed iteration count.
__global__ void batch_advance_kernel(InstDesc *__restrict__ inst, int B, const int *__restrict__ active,
                                     unsigned long long *__restrict__ unconv)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    inst[b].step += 1u;
    inst[b].first = 0;
    if (active[b]) atomicAdd(unconv, 1ull);
}

// One AB step of the packed batch (state in vec[V_POS], vec[V_UP]).  graph: see batch_lanczos; the
// step then also advances the device-side step counters.
static int batch_step_body(rpb_batch *bt, double dt, double delta, double tol, int max_iter,
                           const rpb_force_params *fp, bool graph)
{
    cudaStream_t st = bt->stream;
    const int64_t total = bt->total, n = 3 * total;
    double **v = bt->vec;
    const int ge = grid_for(n, bt->num_sms);
    int rc;
    const double a = bt->p.a;
    const double rcut = (2.0 * a + kForceCutoffB * fp->b) * 1.01 + 0.01 * a;
    const double rnear = 2.0 * a + (double)kFarB * fp->b;
    batch_forces_kernel<<<bt->nblocks, 128, 0, st>>>(v[V_POS], bt->d_inst, bt->d_blocks, total, a, fp->weight, fp->U0,
                                                     fp->b, (float)(rcut * rcut), (float)(rnear * rnear), v[V_F]);
    batch_fill3_kernel<<<ge, 256, 0, st>>>(v[V_T], total, fp->torque[0], fp->torque[1], fp->torque[2]);
    count_launches(2);
    if ((rc = batch_product(bt, v[V_POS], v[V_F], v[V_T], v[V_UN], nullptr))) return rc;
    batch_philox_kernel<<<ge, 256, 0, st>>>(bt->d_inst, bt->d_inst_of, total, 0u, v[V_W]);
    batch_philox_kernel<<<ge, 256, 0, st>>>(bt->d_inst, bt->d_inst_of, total, 1u, v[V_WT]);
    count_launches(2);
    if ((rc = batch_lanczos(bt, v[V_POS], v[V_W], v[V_G], tol, max_iter, graph))) return rc;
    // RFD: two products at the displaced configurations, regularised anew
    batch_displace_kernel<<<ge, 256, 0, st>>>(v[V_POS], v[V_WT], n, 0.5 * delta, v[V_PA], v[V_PB]);
    count_launches(1);
    if ((rc = batch_product(bt, v[V_PA], v[V_WT], nullptr, v[V_DRIFT], nullptr))) return rc;
    if ((rc = batch_product(bt, v[V_PB], v[V_WT], nullptr, v[V_WORK], nullptr))) return rc;
    batch_rfd_combine_kernel<<<ge, 256, 0, st>>>(v[V_DRIFT], v[V_WORK], n, bt->p.kT / delta);
    batch_ab_update_kernel<<<ge, 256, 0, st>>>(bt->d_inst, bt->d_inst_of, total, v[V_POS], v[V_UP], v[V_UN], v[V_G],
                                               v[V_DRIFT], dt, sqrt(2.0 * bt->p.kT * dt));
    count_launches(2);
    if (graph) {
        batch_advance_kernel<<<(bt->B + 127) / 128, 128, 0, st>>>(bt->d_inst, bt->B, bt->d_active, bt->d_unconv);
        count_launches(1);
    }
    return cuda_fail(cudaGetLastError(), "batch step kernels");
}

// Per-instance statistics from the host copy of the Lanczos states; returns how many did not converge.
static int batch_read_stats(rpb_batch *bt, double tol, rpb_step_stats *stats)
{
    const LzLayout L(bt->max_iter);
    int noconv = 0;
    for (int b = 0; b < bt->B; ++b) {
        const double *stb = bt->h_lz + (size_t)b * bt->lz_stride + L.status;
        const int conv = stb[7] != 0.0;
        noconv += !conv && tol > 0.0;
        if (stats) {
            stats[b].lanczos_iters = (int)stb[6];
            stats[b].lanczos_err = stb[ST_EPS];
            stats[b].converged = conv;
        }
    }
    return noconv;
}

// nsteps AB steps of the batch: one gather, one launch of a CUDA graph whose WHILE node runs a step
// (fixed Lanczos iteration count, converged instances masked) nsteps times without host
// synchronisation, one scatter.
static int batch_run_impl(rpb_batch *bt, int B, const int64_t *N, double *const *pos, double *const *U_prev,
                          const int64_t *steps, const uint64_t *seeds, int nsteps, double dt, double delta, double tol,
                          int lanczos_iters, const rpb_force_params *fp, rpb_step_stats *stats, int64_t *unconverged)
{
    int rc;
    if ((rc = batch_setup(bt, B, N, steps, seeds, pos, U_prev, nullptr, nullptr))) return rc;
    cudaStream_t st = bt->stream;
    double **v = bt->vec;
    if ((rc = batch_gather(bt, 0, v[V_POS], 0)) || (rc = batch_gather(bt, 1, v[V_UP], 0))) return rc;
    if ((rc = cuda_fail(cudaMemsetAsync(bt->d_unconv, 0, sizeof(unsigned long long), st), "memset")) ||
        (rc = cuda_fail(cudaMemsetAsync(bt->d_iter_runs, 0, kMaxIter * sizeof(unsigned long long), st), "memset")))
        return rc;
    for (int k = 0; k < kMaxIter; ++k) bt->iter_launches[k] = 0;
    int per_step = 0;
    if (nsteps > 0) {
        // one graph launch for all nsteps: a WHILE node whose body is a step, counted down on the device
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        graph_loop_init_kernel<<<1, 1, 0, st>>>(bt->d_left, nsteps);
        count_launches(1);
        const uint64_t before = rpb_launch_count();
        if ((rc = cuda_fail(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture"))) return rc;
        cudaGraphConditionalHandle loop_h = 0;
        int brc = graph_begin_loop(st, bt->loop, &loop_h);
        if (!brc) {
            bt->stream = bt->loop;
            brc = batch_step_body(bt, dt, delta, tol, lanczos_iters, fp, true);
            if (!brc) {
                graph_loop_tail_kernel<<<1, 1, 0, bt->loop>>>(bt->d_left, loop_h);
                count_launches(1);
                brc = cuda_fail(cudaGetLastError(), "loop kernel");
            }
            bt->stream = st;
            cudaGraph_t loop_graph = nullptr;  // owned by the WHILE node
            const cudaError_t el = cudaStreamEndCapture(bt->loop, &loop_graph);
            if (!brc && el != cudaSuccess) brc = cuda_fail(el, "loop body capture end");
        }
        const cudaError_t ec = cudaStreamEndCapture(st, &graph);
        per_step = (int)(rpb_launch_count() - before);
        count_launches(-per_step);  // captured, not executed (counted below from the runs)
        if (brc) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return brc;
        }
        if ((rc = cuda_fail(ec, "end capture"))) return rc;
        if ((rc = cuda_fail(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate"))) {
            cudaGraphDestroy(graph);
            return rc;
        }
        rc = cuda_fail(cudaGraphLaunch(exec, st), "graph launch");
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (rc) return rc;
    }
    if ((rc = batch_gather(bt, 0, v[V_POS], 1)) || (rc = batch_gather(bt, 1, v[V_UP], 1))) return rc;
    if ((rc = cuda_fail(cudaMemcpyAsync(bt->h_lz, bt->lz, (size_t)B * bt->lz_stride * sizeof(double),
                                        cudaMemcpyDeviceToHost, st),
                        "status copy")) ||
        (rc = cuda_fail(cudaMemcpyAsync(bt->h_unconv, bt->d_unconv, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                                        st),
                        "count copy")) ||
        (rc = cuda_fail(cudaMemcpyAsync(bt->h_iter_runs, bt->d_iter_runs, kMaxIter * sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, st),
                        "iteration count copy")) ||
        (rc = cuda_fail(cudaStreamSynchronize(st), "batch run")))
        return rc;
    if (nsteps > 0) {  // kernels executed: the unconditional part every step, each iteration body per run
        int64_t cond_part = 0, executed = 0;
        for (int k = 1; k < kMaxIter; ++k) {
            cond_part += bt->iter_launches[k];
            executed += (int64_t)bt->iter_launches[k] * (int64_t)bt->h_iter_runs[k];
        }
        count_launches((int)((per_step - cond_part) * (int64_t)nsteps + executed));
    }
    batch_read_stats(bt, tol, stats);
    if (unconverged) *unconverged = (int64_t)*bt->h_unconv;
    if (*bt->h_unconv && tol > 0.0) {
        set_error("lanczos: %llu instance-step(s) did not converge in %d iterations", *bt->h_unconv, lanczos_iters);
        return RPB_ENOCONV;
    }
    return RPB_OK;
}

}  // namespace rpb

extern "C" {

int rpb_batch_create(rpb_batch **out, const rpb_params *p, int64_t max_total_N, int max_B, int max_iter, void *stream)
{
    if (!out || !p) {
        set_error("null argument to rpb_batch_create");
        return RPB_EINVAL;
    }
    *out = nullptr;
    if (!(p->a > 0.0) || !(p->eta > 0.0) || !(p->kT >= 0.0) || (p->precision != RPB_FP64 && p->precision != RPB_FP32) ||
        p->wall != 1) {
        set_error("bad parameters (batch contexts need precision RPB_FP64/RPB_FP32 and wall = 1)");
        return RPB_EINVAL;
    }
    if (max_total_N <= 0 || max_total_N > (int64_t)1 << 28 || max_B < 1 || max_B > (1 << 20) || max_iter < 1 ||
        max_iter > kMaxIter) {
        set_error("bad batch limits (max_total_N=%lld max_B=%d max_iter=%d)", (long long)max_total_N, max_B, max_iter);
        return RPB_EINVAL;
    }
    rpb_batch *bt = new (std::nothrow) rpb_batch();
    if (!bt) {
        set_error("host allocation failed");
        return RPB_ENOMEM;
    }
    bt->p = *p;
    bt->max_total = max_total_N;
    bt->max_B = max_B;
    bt->max_iter = max_iter;
    bt->stream = (cudaStream_t)stream;
    {
        // RPB_FP32_BATCH_SYM=0: float32 products by the one-way kernel instead of the symmetric pass
        const char *v = getenv("RPB_FP32_BATCH_SYM");
        bt->sym_env = !(v && strcmp(v, "0") == 0);
        bt->sym_enabled = p->precision == RPB_FP32 && bt->sym_env;
    }
    int dev = 0;
    if (cuda_fail(cudaGetDevice(&dev), "cudaGetDevice") ||
        cuda_fail(cudaDeviceGetAttribute(&bt->num_sms, cudaDevAttrMultiProcessorCount, dev), "SM count")) {
        delete bt;
        return RPB_ECUDA;
    }
    const LzLayout L(max_iter);
    bt->lz_stride = L.total;
    const size_t vb = (size_t)3 * max_total_N * sizeof(double);
    const int64_t max_blocks = max_total_N / kTile + max_B + 1;
    bool ok = cudaMalloc(&bt->d_inst, max_B * sizeof(InstDesc)) == cudaSuccess &&
              cudaMalloc(&bt->d_blocks, max_blocks * sizeof(BlockDesc)) == cudaSuccess &&
              cudaMalloc(&bt->d_inst_of, max_total_N * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&bt->d_active, max_B * sizeof(int)) == cudaSuccess &&
              cudaMalloc(&bt->d_nactive, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&bt->src, max_total_N * sizeof(SrcF64)) == cudaSuccess &&
              cudaMalloc(&bt->V, vb * (max_iter + 1)) == cudaSuccess &&
              cudaMalloc(&bt->lz, (size_t)max_B * L.total * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&bt->red, (size_t)(max_iter + 2) * max_B * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&bt->norm2, (size_t)max_B * sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&bt->h_inst, max_B * sizeof(InstDesc)) == cudaSuccess &&
              cudaMallocHost(&bt->h_blocks, max_blocks * sizeof(BlockDesc)) == cudaSuccess &&
              cudaMallocHost(&bt->h_nactive, sizeof(int)) == cudaSuccess &&
              cudaMallocHost(&bt->h_lz, (size_t)max_B * L.total * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&bt->d_unconv, sizeof(unsigned long long)) == cudaSuccess &&
              cudaMallocHost(&bt->h_unconv, sizeof(unsigned long long)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&bt->loop, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&bt->d_left, sizeof(int)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&bt->body, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&bt->d_iter_runs, kMaxIter * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMallocHost(&bt->h_iter_runs, kMaxIter * sizeof(unsigned long long)) == cudaSuccess &&
              cudaEventCreateWithFlags(&bt->join, cudaEventDisableTiming) == cudaSuccess;
    for (double *&v : bt->vec) ok = ok && cudaMalloc(&v, vb) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        set_error("batch scratch allocation failed (max_total_N=%lld, max_B=%d)", (long long)max_total_N, max_B);
        batch_free(bt);
        delete bt;
        return RPB_ENOMEM;
    }
    if (cuda_fail(cudaMemsetAsync(bt->lz, 0, (size_t)max_B * L.total * sizeof(double), bt->stream), "memset")) {
        batch_free(bt);
        delete bt;
        return RPB_ECUDA;
    }
    *out = bt;
    return RPB_OK;
}

int rpb_batch_destroy(rpb_batch *bt)
{
    if (!bt) return RPB_OK;
    const int rc = cuda_fail(cudaStreamSynchronize(bt->stream), "rpb_batch_destroy sync");
    batch_free(bt);
    delete bt;
    return rc;
}

int rpb_batch_set_stream(rpb_batch *bt, void *stream)
{
    if (!bt) {
        set_error("null batch");
        return RPB_EINVAL;
    }
    bt->stream = (cudaStream_t)stream;
    return RPB_OK;
}

int rpb_batch_set_tiles(rpb_batch *bt, const rpb_batch_tiles *t)
{
    if (!bt) {
        set_error("null batch context");
        return RPB_EINVAL;
    }
    rpb_batch_tiles d = {8, 5, bt->sym_env};
    if (!t) t = &d;
    if (t->seg_tiles < 1 || t->seg_tiles > 64 || (t->ctas_per_sm != 4 && t->ctas_per_sm != 5) ||
        (t->symmetric != 0 && t->symmetric != 1)) {
        set_error("bad tile schedule (seg_tiles=%d ctas_per_sm=%d symmetric=%d)", t->seg_tiles, t->ctas_per_sm,
                  t->symmetric);
        return RPB_EINVAL;
    }
    bt->seg_tiles = t->seg_tiles;
    bt->sym.tt_minb = t->ctas_per_sm;
    bt->sym_enabled = bt->p.precision == RPB_FP32 && t->symmetric;
    bt->sym_ok = false;  // planned again by the next call
    return RPB_OK;
}

int rpb_batch_get_tiles(rpb_batch *bt, rpb_batch_tiles *t)
{
    if (!bt || !t) {
        set_error("null argument to rpb_batch_get_tiles");
        return RPB_EINVAL;
    }
    t->seg_tiles = bt->seg_tiles;
    t->ctas_per_sm = bt->sym.tt_minb;
    t->symmetric = bt->sym_enabled ? 1 : 0;
    return RPB_OK;
}

int rpb_batch_tune(rpb_batch *bt, int B, const int64_t *N, const double *const *pos, int reps, rpb_batch_tiles *best,
                   int max_cand, rpb_batch_tiles *cand, double *cand_ms, int *ncand)
{
    if (!bt || !N || !pos || reps < 1) {
        set_error("bad argument to rpb_batch_tune");
        return RPB_EINVAL;
    }
    for (int b = 0; b < B && b < bt->max_B; ++b)
        if (!pos[b]) {
            set_error("instance %d: null pos", b);
            return RPB_EINVAL;
        }
    int rc;
    // candidates: the symmetric pass at every run length and occupancy, and the one-way kernel
    std::vector<rpb_batch_tiles> cs;
    if (bt->p.precision == RPB_FP32) {
        for (int seg : {4, 8, 16, 32})
            for (int minb : {4, 5}) cs.push_back(rpb_batch_tiles{seg, minb, 1});
        cs.push_back(rpb_batch_tiles{8, 5, 0});
    } else {
        cs.push_back(rpb_batch_tiles{8, 5, 0});  // float64: the one-way kernel only
    }
    if ((rc = rpb_batch_set_tiles(bt, &cs[0])) ||
        (rc = batch_setup(bt, B, N, nullptr, nullptr, const_cast<double *const *>(pos), nullptr, nullptr, nullptr)))
        return rc;
    cudaStream_t st = bt->stream;
    double **v = bt->vec;
    const int ge = grid_for(3 * bt->total, bt->num_sms);
    if ((rc = batch_gather(bt, 0, v[V_POS], 0))) return rc;
    batch_fill3_kernel<<<ge, 256, 0, st>>>(v[V_F], bt->total, 0.0, 0.0, -1.0);
    batch_fill3_kernel<<<ge, 256, 0, st>>>(v[V_T], bt->total, 0.0, 1.0, 0.0);
    count_launches(2);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((rc = cuda_fail(cudaEventCreate(&e0), "event")) || (rc = cuda_fail(cudaEventCreate(&e1), "event"))) {
        if (e0) cudaEventDestroy(e0);
        return rc;
    }
    double best_cost = -1.0;
    size_t best_k = 0;
    for (size_t k = 0; k < cs.size() && !rc; ++k) {
        if ((rc = rpb_batch_set_tiles(bt, &cs[k]))) break;
        if (bt->sym_enabled && (rc = batch_sym_plan(bt->sym, B, N, st, &bt->sym_ok, bt->seg_tiles))) break;
        // a step makes about ten translation-translation products per fused one
        float t_tt = 0.f, t_fu = 0.f;
        for (int pass = 0; pass < 2 && !rc; ++pass) {  // pass 0 warms up
            for (int which = 0; which < 2 && !rc; ++which) {
                const double *T = which ? v[V_T] : nullptr;
                cudaEventRecord(e0, st);
                for (int r = 0; r < reps && !rc; ++r) rc = batch_product(bt, v[V_POS], v[V_F], T, v[V_UN], nullptr);
                cudaEventRecord(e1, st);
                if (!rc) rc = cuda_fail(cudaEventSynchronize(e1), "tune timing");
                float ms = 0.f;
                if (!rc) rc = cuda_fail(cudaEventElapsedTime(&ms, e0, e1), "tune timing");
                if (pass == 1) (which ? t_fu : t_tt) = ms / reps;
            }
        }
        const double cost = 10.0 * t_tt + t_fu;
        if (cand && cand_ms && (int)k < max_cand) {
            cand[k] = cs[k];
            cand_ms[k] = cost;
        }
        if (!rc && (best_cost < 0.0 || cost < best_cost)) {
            best_cost = cost;
            best_k = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (ncand) *ncand = (int)cs.size();
    if (best) *best = cs[best_k];
    return rpb_batch_set_tiles(bt, &cs[best_k]);
}

int rpb_batch_mobility_apply(rpb_batch *bt, int B, const int64_t *N, const double *const *pos, const double *const *F,
                             const double *const *T, double *const *U)
{
    if (!bt || !N || !pos || !U) {
        set_error("null argument to rpb_batch_mobility_apply");
        return RPB_EINVAL;
    }
    for (int b = 0; b < B && b < bt->max_B; ++b)
        if (!pos[b] || !U[b]) {
            set_error("instance %d: null pos or U", b);
            return RPB_EINVAL;
        }
    int rc;
    if ((rc = batch_setup(bt, B, N, nullptr, nullptr, const_cast<double *const *>(pos), const_cast<double *const *>(F),
                          T, U)))
        return rc;
    double *P = bt->vec[V_POS], *Fp = F ? bt->vec[V_F] : nullptr, *Tp = T ? bt->vec[V_T] : nullptr, *Up = bt->vec[V_UN];
    if ((rc = batch_gather(bt, 0, P, 0))) return rc;
    if (Fp && (rc = batch_gather(bt, 1, Fp, 0))) return rc;
    if (Tp && (rc = batch_gather(bt, 2, Tp, 0))) return rc;
    if (!Fp && !Tp) {
        if ((rc = cuda_fail(cudaMemsetAsync(Up, 0, 3 * bt->total * sizeof(double), bt->stream), "memset"))) return rc;
    } else if ((rc = batch_product(bt, P, Fp, Tp, Up, nullptr))) {
        return rc;
    }
    return batch_gather(bt, 3, Up, 1);
}

int rpb_batch_ab_step(rpb_batch *bt, int B, const int64_t *N, double *const *pos, double *const *U_prev,
                      const int64_t *steps, const uint64_t *seeds, double dt, double delta, double tol, int max_iter,
                      const rpb_force_params *fp, rpb_step_stats *stats)
{
    if (!bt || !N || !pos || !U_prev || !steps || !seeds || !fp) {
        set_error("null argument to rpb_batch_ab_step");
        return RPB_EINVAL;
    }
    if (!(fp->b > 0.0) || !(dt > 0.0) || !(delta > 0.0) || max_iter < 1 || max_iter > bt->max_iter) {
        set_error("bad step arguments (dt=%g delta=%g max_iter=%d)", dt, delta, max_iter);
        return RPB_EINVAL;
    }
    for (int b = 0; b < B && b < bt->max_B; ++b)
        if (!pos[b] || !U_prev[b] || steps[b] < 0 || steps[b] > 0xffffffffLL) {
            set_error("instance %d: null buffer or bad step", b);
            return RPB_EINVAL;
        }
    int rc;
    if ((rc = batch_setup(bt, B, N, steps, seeds, pos, U_prev, nullptr, nullptr))) return rc;
    double **v = bt->vec;
    if ((rc = batch_gather(bt, 0, v[V_POS], 0)) || (rc = batch_gather(bt, 1, v[V_UP], 0))) return rc;
    if ((rc = batch_step_body(bt, dt, delta, tol, max_iter, fp, false))) return rc;
    if ((rc = batch_gather(bt, 0, v[V_POS], 1)) || (rc = batch_gather(bt, 1, v[V_UP], 1))) return rc;
    const int noconv = batch_read_stats(bt, tol, stats);
    if (noconv) {
        set_error("lanczos: %d instance(s) did not converge in %d iterations", noconv, max_iter);
        return RPB_ENOCONV;
    }
    return RPB_OK;
}

int rpb_batch_run(rpb_batch *bt, int B, const int64_t *N, double *const *pos, double *const *U_prev,
                  const int64_t *steps, const uint64_t *seeds, int nsteps, double dt, double delta, double tol,
                  int lanczos_iters, const rpb_force_params *fp, rpb_step_stats *stats, int64_t *unconverged)
{
    if (!bt || !N || !pos || !U_prev || !steps || !seeds || !fp) {
        set_error("null argument to rpb_batch_run");
        return RPB_EINVAL;
    }
    if (!(fp->b > 0.0) || !(dt > 0.0) || !(delta > 0.0) || lanczos_iters < 1 || lanczos_iters > bt->max_iter ||
        nsteps < 0) {
        set_error("bad run arguments (dt=%g delta=%g lanczos_iters=%d nsteps=%d)", dt, delta, lanczos_iters, nsteps);
        return RPB_EINVAL;
    }
    for (int b = 0; b < B && b < bt->max_B; ++b)
        if (!pos[b] || !U_prev[b] || steps[b] < 0 || steps[b] + nsteps > 0xffffffffLL) {
            set_error("instance %d: null buffer or bad step", b);
            return RPB_EINVAL;
        }
    // Everything runs on the batch's own capture stream, ordered after the caller's stream.
    cudaStream_t user = bt->stream;
    int rc;
    if ((rc = cuda_fail(cudaEventRecord(bt->join, user), "event record")) ||
        (rc = cuda_fail(cudaStreamWaitEvent(bt->cap, bt->join, 0), "stream wait")))
        return rc;
    bt->stream = bt->cap;
    rc = batch_run_impl(bt, B, N, pos, U_prev, steps, seeds, nsteps, dt, delta, tol, lanczos_iters, fp, stats,
                        unconverged);
    bt->stream = user;
    return rc;
}

}  // extern "C"
