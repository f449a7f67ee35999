// step.cu -- Philox noise, random-finite-difference drift and the Adams-Bashforth update.
#include <cmath>

#include "rpb_internal.cuh"

namespace rpb {

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror & Shaw (SC'11): ten rounds of two 32x32->64-bit multiplications of counter
// words 0 and 2, whose high halves are mixed with words 1 and 3 and the round key; the key is
// advanced by a Weyl increment between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
        const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Normals k = 2p and 2p + 1 of the particle-major index k = 3 i + c, stored SoA out[c N + i].
__global__ void philox_normal_kernel(int N, uint32_t k0, uint32_t k1, uint32_t step, uint32_t sid, uint32_t inst,
                                     double *__restrict__ out, const unsigned int *__restrict__ d_step)
{
    if (d_step) step = *d_step;
    const int64_t n = 3 * (int64_t)N;
    const int64_t npairs = (n + 1) / 2;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += (int64_t)gridDim.x * blockDim.x) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)p, step, sid, inst), k0, k1);
        const double two26 = 67108864.0, two_m53 = 1.1102230246251565e-16;
        const double u1 = ((double)(r.x >> 5) * two26 + (double)(r.y >> 6) + 1.0) * two_m53;
        const double u2 = ((double)(r.z >> 5) * two26 + (double)(r.w >> 6) + 1.0) * two_m53;
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        const int64_t ka = 2 * p, kb = 2 * p + 1;
        out[(ka % 3) * N + ka / 3] = rad * cs;
        if (kb < n) out[(kb % 3) * N + kb / 3] = rad * sn;
    }
}

int philox_impl(rpb_ctx *ctx, int64_t N, uint64_t seed, uint32_t step, uint32_t stream_id, uint32_t instance,
                double *out, const unsigned int *d_step)
{
    const int64_t npairs = (3 * N + 1) / 2;
    int grid = (int)((npairs + 255) / 256);
    if (grid > 8 * ctx->num_sms) grid = 8 * ctx->num_sms;
    philox_normal_kernel<<<grid, 256, 0, ctx->stream>>>((int)N, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32),
                                                        step, stream_id, instance, out, d_step);
    count_launches(1);
    return cuda_fail(cudaGetLastError(), "philox kernel");
}

// ------------------------------------------------------------------ RFD (Sec. II.A)
__global__ void displace_kernel(const double *__restrict__ pos, const double *__restrict__ Wt, int64_t n, double h,
                                double *__restrict__ plus, double *__restrict__ minus)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const double q = pos[r], d = h * Wt[r];
        plus[r] = q + d;
        minus[r] = q - d;
    }
}

__global__ void rfd_combine_kernel(double *__restrict__ up_drift, const double *__restrict__ um, int64_t n, double k)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        up_drift[r] = k * (up_drift[r] - um[r]);
}

static int elem_grid(int64_t n, int num_sms)
{
    int64_t g = (n + 255) / 256;
    if (g > 8 * (int64_t)num_sms) g = 8 * num_sms;
    return g < 1 ? 1 : (int)g;
}

int rfd_impl(rpb_ctx *ctx, int64_t N, const double *pos, const double *Wt, double delta, double *drift, int one_sided)
{
    const int64_t n = 3 * N;
    const int G = elem_grid(n, ctx->num_sms);
    // centred: q +- delta/2 W~; one-sided: q + delta W~ and q itself
    displace_kernel<<<G, 256, 0, ctx->stream>>>(pos, Wt, n, one_sided ? delta : 0.5 * delta, ctx->ws.pos_a,
                                                ctx->ws.pos_b);
    count_launches(1);
    int rc;
    if ((rc = cuda_fail(cudaGetLastError(), "rfd displace"))) return rc;
    if ((rc = mobility_apply_impl(ctx, N, ctx->ws.pos_a, Wt, nullptr, drift))) return rc;
    if ((rc = mobility_apply_impl(ctx, N, one_sided ? pos : ctx->ws.pos_b, Wt, nullptr, ctx->ws.w))) return rc;
    rfd_combine_kernel<<<G, 256, 0, ctx->stream>>>(drift, ctx->ws.w, n, ctx->p.kT / delta);
    count_launches(1);
    return cuda_fail(cudaGetLastError(), "rfd combine");
}

// ------------------------------------------------------------------ AB update (Eq. AB)
__global__ void ab_update_kernel(double *__restrict__ pos, double *__restrict__ U_prev, const double *__restrict__ Un,
                                 const double *__restrict__ g, const double *__restrict__ drift, int64_t n, double dt,
                                 double noise_scale, int first, const int *__restrict__ d_first)
{
    if (d_first && *d_first) first = 1;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const double un = Un[r];
        const double up = first ? un : U_prev[r];
        pos[r] = pos[r] + dt * (1.5 * un - 0.5 * up) + noise_scale * g[r] + dt * drift[r];
        U_prev[r] = un;
    }
}

__global__ void fill3_kernel(double *__restrict__ v, int N, double x, double y, double z)
{
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < 3 * (int64_t)N;
         r += (int64_t)gridDim.x * blockDim.x)
        v[r] = r < N ? x : (r < 2 * (int64_t)N ? y : z);
}

int ab_update_impl(rpb_ctx *ctx, int64_t N, double *pos, double *U_prev, const double *Un, const double *g,
                   const double *drift, double dt, double noise_scale, int first, const int *d_first)
{
    const int64_t n = 3 * N;
    ab_update_kernel<<<elem_grid(n, ctx->num_sms), 256, 0, ctx->stream>>>(pos, U_prev, Un, g, drift, n, dt,
                                                                            noise_scale, first, d_first);
    count_launches(1);
    return cuda_fail(cudaGetLastError(), "ab update");
}

int fill_torque(rpb_ctx *ctx, int64_t N, const double *t, double *T)
{
    fill3_kernel<<<elem_grid(3 * N, ctx->num_sms), 256, 0, ctx->stream>>>(T, (int)N, t[0], t[1], t[2]);
    count_launches(1);
    return cuda_fail(cudaGetLastError(), "fill torque");
}

}  // namespace rpb
