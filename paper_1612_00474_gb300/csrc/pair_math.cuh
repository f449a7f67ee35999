// pair_math.cuh -- device arithmetic of one Rotne-Prager-Blake pair (shared by the single-suspension
// and batched kernels).
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
#pragma once

#include "rpb_internal.cuh"

namespace rpb {

// Reciprocal square root of a float32 squared distance: the hardware approximation with subnormal
// inputs flushed to zero, one MUFU operation.  Squared distances below the smallest normal float are
// treated as coincident spheres by the callers (kMinNormal).
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kMinNormal = 1.17549435e-38f;

template <typename R>
__device__ __forceinline__ R rsq(R x);
template <>
__device__ __forceinline__ float rsq<float>(float x)
{
    return rsqrt_ftz(x);
}
template <>
__device__ __forceinline__ double rsq<double>(double x)
{
    return rsqrt(x);
}

// Velocity of the target from one source, in units of 1/(8 pi eta), before the target's s_i.
// rx, ry: in-plane offset target - source; zi, zj: clamped heights; F, T: source force and torque
// with s_j folded in.  Accumulates into (ux, uy, uz).  Valid for r = 0 (self pair: mu0 F + wall).
template <typename R, bool TORQUE, bool WALL = true>
__device__ __forceinline__ void pair_velocity(R rx, R ry, R zi, R zj, R Fx, R Fy, R Fz, R Tx, R Ty, R Tz,
                                              const PairConsts<R> &c, R &ux, R &uy, R &uz)
{
    // ---- free-space RPY
    const R rz = zi - zj;
    const R rho2 = rx * rx + ry * ry;
    const R r2 = rho2 + rz * rz;
    const R inv_r = r2 > R(0) ? rsq<R>(r2) : R(0);
    const R r = r2 * inv_r;
    const R inv_r2 = inv_r * inv_r;
    const bool far = r >= c.two_a;
    const R c1 = far ? inv_r * (R(1) + c.two_3_a2 * inv_r2) : c.near_c1 * (R(1) - c.near_r * r);
    const R c2 = far ? inv_r * inv_r2 * (R(1) - c.two_a2 * inv_r2) : c.near_c2 * inv_r;
    const R k2 = c2 * (rx * Fx + ry * Fy + rz * Fz);
    ux += c1 * Fx + k2 * rx;
    uy += c1 * Fy + k2 * ry;
    uz += c1 * Fz + k2 * rz;
    if (TORQUE) {
        const R ct = far ? inv_r * inv_r2 : c.near_tr * (R(1) - c.near_tr_r * r);
        ux += ct * (Ty * rz - Tz * ry);
        uy += ct * (Tz * rx - Tx * rz);
        uz += ct * (Tx * ry - Ty * rx);
    }
    if (!WALL) return;  // unbounded domain: free-space RPY only
    // ---- wall correction (image of the source below z = 0)
    const R Rz = zi + zj;
    const R invR = rsq<R>(rho2 + Rz * Rz);
    const R ex = rx * invR, ey = ry * invR, ez = Rz * invR;
    const R t = zj * invR;
    const R s = c.a2 * invR * invR;
    const R ez2 = ez * ez;
    const R t2 = t * t;
    const R et = ez * t;
    const R s2 = s * s;
    const R A = R(-1) - R(2) * et + R(2) * t2 + s * (R(2) * ez2 - R(2.0 / 3.0)) + s2 * (R(2.0 / 3.0) - R(10.0 / 3.0) * ez2);
    const R B = R(-1) + R(6) * et - R(6) * t2 + s * (R(2) - R(10) * ez2) + s2 * (R(70.0 / 3.0) * ez2 - R(10.0 / 3.0));
    const R C = t * (R(2) - R(12) * ez2) + R(12) * et * t +
                ez * (s * (R(20) * ez2 - R(4)) + s2 * (R(40.0 / 3.0) - R(140.0 / 3.0) * ez2));
    const R D = R(2) * t - R(20.0 / 3.0) * s2 * ez;
    const R E = R(-4) * t2 - R(4) * s * ez2 + s2 * (R(20) * ez2 - R(8.0 / 3.0));
    const R eF = ex * Fx + ey * Fy + ez * Fz;
    const R ke = (B * eF + C * Fz) * invR;
    const R kz = (D * eF + E * Fz) * invR;
    const R kA = A * invR;
    ux += kA * Fx + ke * ex;
    uy += kA * Fy + ke * ey;
    uz += kA * Fz + ke * ez + kz;
    if (TORQUE) {
        const R invR2 = invR * invR;
        const R cz = R(2) * (t + s * ez);                 // coefficient of T x z
        const R ce = R(6) * (ez - t) - R(10) * s * ez;   // coefficient of e (z x e).T
        const R w = ex * Ty - ey * Tx;                    // (z x e) . T
        ux += invR2 * (-(Ty * ez - Tz * ey) + cz * Ty + ce * w * ex);
        uy += invR2 * (-(Tz * ex - Tx * ez) - cz * Tx + ce * w * ey);
        uz += invR2 * (-(Tx * ey - Ty * ex) + (ce * ez + R(2) * s) * w);
    }
}

// Float64 target velocity from one source with the wall: the same block as pair_velocity, its wall
// coefficients evaluated as polynomials in s = 1/|R|^2 with height-only coefficients (see the
// packed float32 form below for the algebra): about half the float64 operations of the direct
// form, which matters where float64 runs at a small fraction of the float32 rate.  Valid for r = 0
// (the self pair, r2 = 0, takes the overlap branch).  Accumulates into (ux, uy, uz).
template <bool TORQUE>
__device__ __forceinline__ void pair_velocity_wall64(double rx, double ry, double zi, double zj, double Fx, double Fy,
                                                     double Fz, double Tx, double Ty, double Tz,
                                                     const PairConsts<double> &c, double &ux, double &uy, double &uz)
{
    const double a2 = c.a2, a4 = a2 * a2;
    const double rz = zi - zj;
    const double rho2 = fma(rx, rx, ry * ry);
    const double r2 = fma(rz, rz, rho2);
    const double ir = r2 > 0.0 ? rsqrt(r2) : 0.0;
    const double r = r2 * ir;
    const double Rz = zi + zj;
    const double Z = Rz * Rz;
    const double u = rsqrt(rho2 + Z);
    const double ir2 = ir * ir, ir3 = ir * ir2;
    const bool far = r >= c.two_a;
    const double c1mu = far ? fma(c.two_3_a2, ir3, ir - u) : fma(c.near_c1, fma(-c.near_r, r, 1.0), -u);
    const double c2 = far ? fma(-c.two_a2, ir3 * ir2, ir3) : c.near_c2 * ir;
    const double s = u * u, u3 = s * u, u5 = u3 * s, sZ = s * Z;
    const double p = fma(-2.0 * zj, zi, -(2.0 / 3.0) * a2);
    const double q = fma(c.two_a2, Z, (2.0 / 3.0) * a4);
    const double XA = fma(s, fma(sZ, (-10.0 / 3.0) * a4, q), p);
    const double XB2 = fma(s, fma(sZ, (140.0 / 3.0) * a4, fma(-20.0 * a2, Z, (-20.0 / 3.0) * a4)), -6.0 * p);
    const double Eh = fma(s, fma(sZ, 20.0 * a4, fma(-4.0 * a2, Z, (-8.0 / 3.0) * a4)), -4.0 * zj * zj);
    const double b2 = u5 * XB2;
    const double T2 = 2.0 * u3 * zj;
    const double u5Rz = u5 * Rz, u7Rz = u5Rz * s;
    const double cF = fma(u3, XA, c1mu);
    const double cFE = fma(u3, Eh, cF);
    const double B3 = fma(0.5, b2, -u3);
    const double C3 = fma(-Rz, b2, fma(u7Rz, (20.0 / 3.0) * a4, T2));
    const double D3 = fma(u7Rz, (-20.0 / 3.0) * a4, T2);
    const double pF = fma(rx, Fx, ry * Fy);
    const double w = fma(Rz, Fz, pF);
    const double k2 = c2 * fma(rz, Fz, pF);
    const double ke = fma(B3, w, C3 * Fz);
    const double kk = k2 + ke;
    ux = fma(cF, Fx, fma(kk, rx, ux));
    uy = fma(cF, Fy, fma(kk, ry, uy));
    uz = fma(cFE, Fz, fma(k2, rz, fma(ke, Rz, fma(D3, w, uz))));
    if (TORQUE) {
        const double ct = far ? ir3 : c.near_tr * fma(-c.near_tr_r, r, 1.0);
        const double dcp = ct - u3;
        const double m2 = fma(u5Rz, c.two_a2, dcp * rz);
        const double kt = fma(6.0 * zi, u5, -10.0 * a2 * u7Rz);
        const double zt = fma(-Rz, kt, fma(-c.two_a2, u5, dcp));
        const double tz3 = fma(Tx, ry, -(Ty * rx));
        const double dTz = dcp * Tz, ktz = kt * tz3;
        ux = fma(Ty, m2, fma(-dTz, ry, fma(-ktz, rx, ux)));
        uy = fma(-Tx, m2, fma(dTz, rx, fma(-ktz, ry, uy)));
        uz = fma(tz3, zt, uz);
    }
}

// The float64 pair of the kernels: the polynomial form with the wall, the free-space form without.
template <bool TORQUE, bool WALL = true>
__device__ __forceinline__ void pair_velocity_f64(double rx, double ry, double zi, double zj, double Fx, double Fy,
                                                  double Fz, double Tx, double Ty, double Tz,
                                                  const PairConsts<double> &c, double &ux, double &uy, double &uz)
{
    if (WALL)
        pair_velocity_wall64<TORQUE>(rx, ry, zi, zj, Fx, Fy, Fz, Tx, Ty, Tz, c, ux, uy, uz);
    else
        pair_velocity<double, TORQUE, false>(rx, ry, zi, zj, Fx, Fy, Fz, Tx, Ty, Tz, c, ux, uy, uz);
}

// Self term M_ii (F, T) in float64, in units of 1/(8 pi eta), F and T with s_i folded in, at the
// clamped height h: the r = 0 limit of pair_velocity in closed form.  With x = a/h the wall-corrected
// self mobilities are mu0 (1 - 9x/16 + x^3/8 - x^5/16) parallel and mu0 (1 - 9x/8 + x^3/2 - x^5/8)
// normal to the wall (the image sum of Sec. II.B at R = 2h e_z), and the translation-rotation self
// coupling is a^2/(8 h^4) e_z x T (Sec. III); mu0 = 4/(3a).  One division instead of the general
// pair's two float64 reciprocal square roots and its wall coefficients: float64 runs at a small
// fraction of the float32 rate on this GPU, and the epilogues that add this term are short.
template <bool TORQUE, bool WALL = true>
__device__ __forceinline__ void self_velocity(double h, double Fx, double Fy, double Fz, double Tx, double Ty,
                                              const PairConsts<double> &c, double &ux, double &uy, double &uz)
{
    const double mu0 = c.near_c1;
    if (!WALL) {
        ux += mu0 * Fx;
        uy += mu0 * Fy;
        uz += mu0 * Fz;
        return;
    }
    const double ih = 1.0 / h;
    const double x = 0.5 * c.two_a * ih;  // a / h
    const double x2 = x * x;
    const double x3 = x2 * x;
    const double x5 = x3 * x2;
    const double mpar = mu0 * (1.0 - 0.5625 * x + 0.125 * x3 - 0.0625 * x5);
    const double mperp = mu0 * (1.0 - 1.125 * x + 0.5 * x3 - 0.125 * x5);
    ux += mpar * Fx;
    uy += mpar * Fy;
    uz += mperp * Fz;
    if (TORQUE) {
        const double ih2 = ih * ih;
        const double ct = 0.125 * c.a2 * ih2 * ih2;
        ux += ct * Ty;
        uy -= ct * Tx;
    }
}

// Float32 form of pair_velocity for the hot loop, hand-fused and algebraically rearranged (same
// mathematics): the wall terms use the unnormalised image vector R, the free-space c1 and wall A/|R|
// share one multiply-add into F, r.F and R.F share their in-plane part, the free-space rotlet
// c_t T x r and the wall's -|R|^-3 T x R share their z component, and the overlap branch (r < 2a,
// rare) is evaluated only when some lane of the warp needs it.  Must be called by all 32 lanes.
template <bool TORQUE, bool WALL = true>
__device__ __forceinline__ void pair_velocity_f32(float rx, float ry, float zi, float zj, float Fx, float Fy,
                                                  float Fz, float Tx, float Ty, float Tz, const PairConsts<float> &c,
                                                  float &ux, float &uy, float &uz)
{
    // ---- free-space RPY, far branch by default
    const float rz = zi - zj;
    const float rho2 = fmaf(rx, rx, ry * ry);
    const float r2 = fmaf(rz, rz, rho2);
    const float inv_r = rsqrt_ftz(r2);
    const float inv_r2 = inv_r * inv_r;
    const float ir3 = inv_r * inv_r2;
    float c1 = inv_r * fmaf(c.two_3_a2, inv_r2, 1.f);
    float c2 = ir3 * fmaf(-c.two_a2, inv_r2, 1.f);
    float ct = ir3;
    const bool near = r2 < c.four_a2;
    if (__any_sync(0xffffffffu, near)) {
        if (near) {  // overlap branch; r = 0 (coincident spheres) gives the self form
            const float r = r2 >= kMinNormal ? r2 * inv_r : 0.f;
            const float ir = r2 >= kMinNormal ? inv_r : 0.f;
            c1 = c.near_c1 * fmaf(-c.near_r, r, 1.f);
            c2 = c.near_c2 * ir;
            ct = c.near_tr * fmaf(-c.near_tr_r, r, 1.f);
        }
    }
    if (!WALL) {  // unbounded domain: free-space RPY only
        const float k2 = c2 * fmaf(rz, Fz, fmaf(rx, Fx, ry * Fy));
        ux = fmaf(c1, Fx, fmaf(k2, rx, ux));
        uy = fmaf(c1, Fy, fmaf(k2, ry, uy));
        uz = fmaf(c1, Fz, fmaf(k2, rz, uz));
        if (TORQUE) {
            ux = fmaf(ct, Ty * rz - Tz * ry, ux);
            uy = fmaf(ct, Tz * rx - Tx * rz, uy);
            uz = fmaf(ct, Tx * ry - Ty * rx, uz);
        }
        return;
    }
    // ---- wall correction
    const float Rz = zi + zj;
    const float invR = rsqrt_ftz(fmaf(Rz, Rz, rho2));
    const float invR2 = invR * invR;
    const float ez = Rz * invR;
    const float t = zj * invR;
    const float s = c.a2 * invR2;
    const float ez2 = ez * ez, t2 = t * t, et = ez * t, s2 = s * s;
    const float d = t2 - et;
    const float A = fmaf(s2, fmaf(-10.f / 3.f, ez2, 2.f / 3.f), fmaf(s, fmaf(2.f, ez2, -2.f / 3.f), fmaf(2.f, d, -1.f)));
    const float B = fmaf(s2, fmaf(70.f / 3.f, ez2, -10.f / 3.f), fmaf(s, fmaf(-10.f, ez2, 2.f), fmaf(-6.f, d, -1.f)));
    const float C =
        fmaf(ez, fmaf(s2, fmaf(-140.f / 3.f, ez2, 40.f / 3.f), s * fmaf(20.f, ez2, -4.f)), t * fmaf(12.f, et - ez2, 2.f));
    const float D = fmaf(-20.f / 3.f, s2 * ez, t + t);
    const float E = fmaf(s2, fmaf(20.f, ez2, -8.f / 3.f), -4.f * fmaf(s, ez2, t2));
    const float pF = fmaf(rx, Fx, ry * Fy);
    const float q = fmaf(Rz, Fz, pF) * invR;          // e.F
    const float k2 = c2 * fmaf(rz, Fz, pF);           // free-space c2 (r.F)
    const float ke = fmaf(B, q, C * Fz) * invR2;      // multiplies R
    const float kz = fmaf(D, q, E * Fz) * invR;       // multiplies z_hat
    const float cF = fmaf(A, invR, c1);               // multiplies F
    const float kk = k2 + ke;
    ux = fmaf(cF, Fx, fmaf(kk, rx, ux));
    uy = fmaf(cF, Fy, fmaf(kk, ry, uy));
    uz = fmaf(cF, Fz, fmaf(k2, rz, fmaf(ke, Rz, uz + kz)));
    if (TORQUE) {
        // c_t T x r - p T x R + |R|^-2 [c_z T x z + (c_e e + 2 s z) (z x e).T],  p = |R|^-3
        const float p = invR2 * invR;
        const float dcp = ct - p;
        const float m1 = fmaf(ct, rz, -(p * Rz));
        const float tz3 = fmaf(Tx, ry, -(Ty * rx));   // (T x r)_z = (T x R)_z
        const float se = s * ez;
        const float m2 = fmaf(t + se, invR2 + invR2, m1);
        const float ce = fmaf(-10.f, se, 6.f * (ez - t));
        const float w = -tz3 * invR;                   // (z x e).T
        const float cw = ce * w * p;                   // multiplies R
        const float dTz = dcp * Tz;
        ux = fmaf(Ty, m2, fmaf(-dTz, ry, fmaf(cw, rx, ux)));
        uy = fmaf(-Tx, m2, fmaf(dTz, rx, fmaf(cw, ry, uy)));
        uz = fmaf(dcp, tz3, fmaf(cw, Rz, fmaf((s + s) * invR2, w, uz)));
    }
}

// ---- two pairs per lane with packed float32x2 arithmetic (FFMA2/FMUL2/FADD2 on sm_100+)
// Every quantity is a float2 whose halves belong to two independent pairs, so one packed instruction
// does the work of two scalar ones.  Constants are passed as float2 pairs in the kernel parameters.
//
// Coefficient form.  With u = 1/|R|, s = u^2, Z = R_z^2 and the closed form of pair_velocity, the wall
// coefficients are polynomials in s whose coefficients depend on the heights only:
//   A = -1 + s X_A,           X_A = p + s (q - (10/3) a^4 s Z),   p = -2 z_i z_j - 2a^2/3,  q = 2a^2 Z + 2a^4/3
//   B = -1 + s X_B,           2 X_B = -6 p + s (-20 a^2 Z - (20/3) a^4 + (140/3) a^4 s Z)
//   C = u (2 z_j + R_z s X_C), X_C = -2 X_B + (20/3) a^4 s
//   D = u (2 z_j - (20/3) a^4 R_z s^2)
//   E = s Ehat,               Ehat = -4 z_j^2 + s (-4 a^2 Z - (8/3) a^4 + 20 a^4 s Z)
// so the coefficients of the application (free-space c1, c2 included) are
//   c_F = c1 + A u = (c1 - u) + u^3 X_A,    B3 = B u^3 = u^5 X_B - u^3,
//   C3 = C u^2 = 2 u^3 z_j - u^5 R_z (2 X_B) + (20/3) a^4 u^7 R_z,   D3 = D u^2 = 2 u^3 z_j - (20/3) a^4 u^7 R_z,
//   E3 = E u = u^3 Ehat,  and the block is  M F = c_F F + c2 (r.F) r + (B3 w + C3 F_z) R + (D3 w + E3 F_z) z_hat,
// w = R.F (R and r share their in-plane part).  c_F + E3 multiplies F_z in the z component, so it is
// formed once (c_FE).  Per source, -2 z_j and -4 z_j^2 (and 6 z_j for the rotation coupling) come
// precomputed with the source.
//   Translation-rotation, with c_t the free-space rotlet coefficient (|r|^-3, or the overlap form) and
// dcp = c_t - u^3:  u += T_y m2 - dcp T_z r_y - kappa tz3 r_x,  u_y += -T_x m2 + dcp T_z r_x - kappa tz3 r_y,
// u_z += tz3 (dcp - 2a^2 u^5 - kappa R_z), where tz3 = T_x r_y - T_y r_x, m2 = dcp r_z + 2a^2 u^5 R_z and
// kappa = u^5 (6 z_i - 10 a^2 s R_z).  The reversed pair (source velocity from the target's torque) has
// r -> -r and z_i <-> z_j in m2 and kappa.
struct X2Consts {
    float2 two_3_a2, m_two_a2, two_a2;    // 2a^2/3, -2a^2, 2a^2
    float2 m2_3_a2, two_3_a4;             // -2a^2/3, 2a^4/3
    float2 m10_3_a4, c140_3_a4, m20_a2;   // -(10/3) a^4, (140/3) a^4, -20 a^2
    float2 m20_3_a4, c20_3_a4, m6;        // -(20/3) a^4, (20/3) a^4, -6
    float2 m4_a2, m8_3_a4, c20_a4;        // -4 a^2, -(8/3) a^4, 20 a^4
    float2 half, m10_a2;                  // 1/2, -10 a^2
    float lo_r2;  // squared distance below which the low parts of the positions are added (float32 kernels)
    float four_a2, near_c1, near_r, near_c2, near_tr, near_tr_r;
};

inline X2Consts make_x2_consts(double a)
{
    auto p = [](double v) { return make_float2((float)v, (float)v); };
    const double a2 = a * a, a4 = a2 * a2;
    X2Consts c;
    c.two_3_a2 = p(2.0 * a2 / 3.0);
    c.m_two_a2 = p(-2.0 * a2);
    c.two_a2 = p(2.0 * a2);
    c.m2_3_a2 = p(-2.0 * a2 / 3.0);
    c.two_3_a4 = p(2.0 * a4 / 3.0);
    c.m10_3_a4 = p(-10.0 * a4 / 3.0);
    c.c140_3_a4 = p(140.0 * a4 / 3.0);
    c.m20_a2 = p(-20.0 * a2);
    c.m20_3_a4 = p(-20.0 * a4 / 3.0);
    c.c20_3_a4 = p(20.0 * a4 / 3.0);
    c.m6 = p(-6.0);
    c.m4_a2 = p(-4.0 * a2);
    c.m8_3_a4 = p(-8.0 * a4 / 3.0);
    c.c20_a4 = p(20.0 * a4);
    c.half = p(0.5);
    c.m10_a2 = p(-10.0 * a2);
    c.four_a2 = (float)(4.0 * a2);
    c.near_c1 = (float)(4.0 / (3.0 * a));
    c.near_r = (float)(9.0 / (32.0 * a));
    c.near_c2 = (float)(1.0 / (8.0 * a2));
    c.near_tr = (float)(1.0 / (2.0 * a2 * a));
    c.near_tr_r = (float)(3.0 / (8.0 * a));
    c.lo_r2 = (float)(100.0 * a2);
    return c;
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c)
{
    return __ffma2_rn(a, b, c);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b)
{
    return __fmul2_rn(a, b);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b)
{
    return __fadd2_rn(a, b);
}
__device__ __forceinline__ float2 neg2(float2 a)
{
    return make_float2(-a.x, -a.y);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return __fadd2_rn(a, neg2(b));
}

// Overlap branch (r < 2a) of the free-space coefficients for one pair: c1 - u (u = 1/|R| of the
// image), c2 and the rotlet coefficient c_t.  r^2 below the smallest normal float is a coincident
// pair (the self form).
__device__ __forceinline__ void near_fix(float r2, float inv_r, float u, const X2Consts &c, float &c1mu, float &c2,
                                         float &ct)
{
    const float r = r2 >= kMinNormal ? r2 * inv_r : 0.f;
    const float ir = r2 >= kMinNormal ? inv_r : 0.f;
    c1mu = fmaf(c.near_c1, fmaf(-c.near_r, r, 1.f), -u);
    c2 = c.near_c2 * ir;
    ct = c.near_tr * fmaf(-c.near_tr_r, r, 1.f);
}

// Offsets of the target from two sources (packed), from the high parts of the positions; the low
// parts are added, for the whole warp, when some lane has a pair closer than sqrt(c.lo_r2) = 10a (the
// error of a high-part offset, up to ulp(|x|), is small against |r| beyond that).  Returns that
// warp-uniform flag, which also covers every overlapping pair (r < 2a).  Must be called by all 32
// lanes.  hi: (x_hi, x_hi', y_hi, y_hi') of the two sources; lo: their low parts, read only if needed.
__device__ __forceinline__ bool pair_offsets_x2(float2 txh, float2 tyh, float2 txl, float2 tyl, float2 zi, float2 zj,
                                                const float4 &hi, const float4 *lo, const X2Consts &c, float2 &rx,
                                                float2 &ry, float2 &rz, float2 &rho2, float2 &r2)
{
    rx = sub2(txh, make_float2(hi.x, hi.y));
    ry = sub2(tyh, make_float2(hi.z, hi.w));
    rz = sub2(zi, zj);
    rho2 = fma2(rx, rx, mul2(ry, ry));
    r2 = fma2(rz, rz, rho2);
    const bool close = __any_sync(0xffffffffu, r2.x < c.lo_r2 || r2.y < c.lo_r2);
    if (close) {
        const float4 l = *lo;
        rx = add2(rx, sub2(txl, make_float2(l.x, l.y)));
        ry = add2(ry, sub2(tyl, make_float2(l.z, l.w)));
        rho2 = fma2(rx, rx, mul2(ry, ry));
        r2 = fma2(rz, rz, rho2);
    }
    return close;
}

// Coefficients of a translation-translation pair block (packed pairs): M F = c_F F + c2 (r.F) r +
// (B3 w + C3 F_z) R + (D3 w + E3 F_z) z_hat with w = R.F, c_FE = c_F + E3.
struct TTBlock {
    float2 rx, ry, rz, Rz, c2, cF, cFE, B3, C3, D3;
};
// Direction-independent factors of the translation-rotation coupling: dcp = c_t - u^3; m2, kappa and
// the z factor (dcp - 2a^2 u^5 - kappa R_z) for the pair (t) and the reversed pair (s).
struct TRBlock {
    float2 dcp, m2t, m2s, kt, ks, zt, zs;
};

// The block of two pairs from their geometry: in-plane offset (rx, ry), rz = zi - zj, rho2 = rx^2 +
// ry^2, r2 = rho2 + rz^2; `close` true (warp-uniformly) when some lane may hold an overlapping pair
// (r < 2a), the overlap branch then being taken per pair.  m2zj = -2 z_j, m4zj2 = -4 z_j^2; six_zi,
// six_zj = 6 z_i, 6 z_j (read only with TORQUE; six_zj only for the reversed pair's factors).
template <bool TORQUE>
__device__ __forceinline__ void pair_block_x2(float2 rx, float2 ry, float2 rz, float2 rho2, float2 r2, bool close,
                                              float2 zi, float2 zj, float2 m2zj, float2 m4zj2, float2 six_zi,
                                              float2 six_zj, const X2Consts &c, TTBlock &m, TRBlock &tb)
{
    const float2 ir = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
    const float2 Rz = add2(zi, zj);
    const float2 Z = mul2(Rz, Rz);
    const float2 R2 = add2(rho2, Z);
    const float2 u = make_float2(rsqrt_ftz(R2.x), rsqrt_ftz(R2.y));
    const float2 ir2 = mul2(ir, ir);
    const float2 ir3 = mul2(ir, ir2);
    float2 c1mu = fma2(c.two_3_a2, ir3, sub2(ir, u));  // (1 + 2a^2/(3 r^2)) / r - u
    float2 c2 = fma2(c.m_two_a2, mul2(ir3, ir2), ir3);  // (1 - 2a^2/r^2) / r^3
    float2 ct = ir3;
    if (close) {
        if (r2.x < c.four_a2) near_fix(r2.x, ir.x, u.x, c, c1mu.x, c2.x, ct.x);
        if (r2.y < c.four_a2) near_fix(r2.y, ir.y, u.y, c, c1mu.y, c2.y, ct.y);
    }
    const float2 s = mul2(u, u);
    const float2 u3 = mul2(s, u);
    const float2 u5 = mul2(u3, s);
    const float2 sZ = mul2(s, Z);
    const float2 p = fma2(m2zj, zi, c.m2_3_a2);
    const float2 q = fma2(c.two_a2, Z, c.two_3_a4);
    const float2 XA = fma2(s, fma2(sZ, c.m10_3_a4, q), p);
    const float2 XB2 = fma2(s, fma2(sZ, c.c140_3_a4, fma2(c.m20_a2, Z, c.m20_3_a4)), mul2(c.m6, p));
    const float2 Eh = fma2(s, fma2(sZ, c.c20_a4, fma2(c.m4_a2, Z, c.m8_3_a4)), m4zj2);
    const float2 b2 = mul2(u5, XB2);
    const float2 T2 = neg2(mul2(u3, m2zj));  // 2 u^3 z_j
    const float2 u5Rz = mul2(u5, Rz);
    const float2 u7Rz = mul2(u5Rz, s);
    const float2 cF = fma2(u3, XA, c1mu);
    m.rx = rx;
    m.ry = ry;
    m.rz = rz;
    m.Rz = Rz;
    m.c2 = c2;
    m.cF = cF;
    m.cFE = fma2(u3, Eh, cF);
    m.B3 = fma2(b2, c.half, neg2(u3));
    m.C3 = fma2(neg2(Rz), b2, fma2(u7Rz, c.c20_3_a4, T2));
    m.D3 = fma2(u7Rz, c.m20_3_a4, T2);
    if (TORQUE) {
        const float2 dcp = sub2(ct, u3);
        const float2 dcprz = mul2(dcp, rz);
        const float2 w10 = mul2(c.m10_a2, u7Rz);
        const float2 d2 = fma2(c.m_two_a2, u5, dcp);
        tb.dcp = dcp;
        tb.m2t = fma2(u5Rz, c.two_a2, dcprz);
        tb.m2s = fma2(u5Rz, c.two_a2, neg2(dcprz));
        tb.kt = fma2(six_zi, u5, w10);
        tb.ks = fma2(six_zj, u5, w10);
        tb.zt = fma2(neg2(Rz), tb.kt, d2);
        tb.zs = fma2(neg2(Rz), tb.ks, d2);
    }
}

// target side: u += M_ij F_j
__device__ __forceinline__ void tt_apply_target(const TTBlock &m, float2 Fx, float2 Fy, float2 Fz, float2 &ux,
                                                float2 &uy, float2 &uz)
{
    const float2 pF = fma2(m.rx, Fx, mul2(m.ry, Fy));
    const float2 w = fma2(m.Rz, Fz, pF);
    const float2 k2 = mul2(m.c2, fma2(m.rz, Fz, pF));
    const float2 ke = fma2(m.B3, w, mul2(m.C3, Fz));
    const float2 kk = add2(k2, ke);
    ux = fma2(m.cF, Fx, fma2(kk, m.rx, ux));
    uy = fma2(m.cF, Fy, fma2(kk, m.ry, uy));
    uz = fma2(m.cFE, Fz, fma2(k2, m.rz, fma2(ke, m.Rz, fma2(m.D3, w, uz))));
}
// source side: v = M_ij^T G_i (C3 and D3 exchanged)
__device__ __forceinline__ void tt_apply_source(const TTBlock &m, float2 Gx, float2 Gy, float2 Gz, float2 &vx,
                                                float2 &vy, float2 &vz)
{
    const float2 pF = fma2(m.rx, Gx, mul2(m.ry, Gy));
    const float2 w = fma2(m.Rz, Gz, pF);
    const float2 k2 = mul2(m.c2, fma2(m.rz, Gz, pF));
    const float2 ke = fma2(m.B3, w, mul2(m.D3, Gz));
    const float2 kk = add2(k2, ke);
    vx = fma2(m.cF, Gx, mul2(kk, m.rx));
    vy = fma2(m.cF, Gy, mul2(kk, m.ry));
    vz = fma2(m.cFE, Gz, fma2(k2, m.rz, fma2(ke, m.Rz, mul2(m.C3, w))));
}
// target side of the translation-rotation coupling: u += M_tr(i, j) T_j
__device__ __forceinline__ void tr_apply_target(const TTBlock &m, const TRBlock &tb, float2 Tx, float2 Ty, float2 Tz,
                                                float2 &ux, float2 &uy, float2 &uz)
{
    const float2 tz3 = fma2(Tx, m.ry, neg2(mul2(Ty, m.rx)));
    const float2 dTz = mul2(tb.dcp, Tz);
    const float2 kt = mul2(tb.kt, tz3);
    ux = fma2(Ty, tb.m2t, fma2(neg2(dTz), m.ry, fma2(neg2(kt), m.rx, ux)));
    uy = fma2(neg2(Tx), tb.m2t, fma2(dTz, m.rx, fma2(neg2(kt), m.ry, uy)));
    uz = fma2(tz3, tb.zt, uz);
}
// source side: v += M_tr(j, i) H_i (the reversed pair: r -> -r, z_i <-> z_j)
__device__ __forceinline__ void tr_apply_source(const TTBlock &m, const TRBlock &tb, float2 Hx, float2 Hy, float2 Hz,
                                                float2 &vx, float2 &vy, float2 &vz)
{
    const float2 tau = fma2(Hx, m.ry, neg2(mul2(Hy, m.rx)));
    const float2 dHz = mul2(tb.dcp, Hz);
    const float2 ks = mul2(tb.ks, tau);
    vx = fma2(Hy, tb.m2s, fma2(dHz, m.ry, fma2(neg2(ks), m.rx, vx)));
    vy = fma2(neg2(Hx), tb.m2s, fma2(neg2(dHz), m.rx, fma2(neg2(ks), m.ry, vy)));
    vz = fma2(neg2(tau), tb.zs, vz);
}

// Target velocity of two sources (one-way), from the geometry of pair_offsets_x2 (close: some lane
// may overlap); the per-source factors are formed here.  In units of 1/(8 pi eta); F, T with s_j.
template <bool TORQUE>
__device__ __forceinline__ void pair_velocity_x2_geo(float2 rx, float2 ry, float2 rz, float2 rho2, float2 r2,
                                                     bool close, float2 zi, float2 zj, float2 Fx, float2 Fy,
                                                     float2 Fz, float2 Tx, float2 Ty, float2 Tz, const X2Consts &c,
                                                     float2 &ux, float2 &uy, float2 &uz)
{
    const float2 zj2 = add2(zj, zj);
    const float2 six = make_float2(6.f, 6.f);
    TTBlock m;
    TRBlock tb;
    pair_block_x2<TORQUE>(rx, ry, rz, rho2, r2, close, zi, zj, neg2(zj2), neg2(mul2(zj2, zj2)), mul2(six, zi),
                          make_float2(0.f, 0.f), c, m, tb);
    tt_apply_target(m, Fx, Fy, Fz, ux, uy, uz);
    if (TORQUE) tr_apply_target(m, tb, Tx, Ty, Tz, ux, uy, uz);
}

template <bool TORQUE>
__device__ __forceinline__ void pair_velocity_x2(float2 rx, float2 ry, float2 zi, float2 zj, float2 Fx, float2 Fy,
                                                 float2 Fz, float2 Tx, float2 Ty, float2 Tz, const X2Consts &c,
                                                 float2 &ux, float2 &uy, float2 &uz)
{
    const float2 rz = sub2(zi, zj);
    const float2 rho2 = fma2(rx, rx, mul2(ry, ry));
    const float2 r2 = fma2(rz, rz, rho2);
    const bool close = __any_sync(0xffffffffu, r2.x < c.four_a2 || r2.y < c.four_a2);
    pair_velocity_x2_geo<TORQUE>(rx, ry, rz, rho2, r2, close, zi, zj, Fx, Fy, Fz, Tx, Ty, Tz, c, ux, uy, uz);
}

// Both directions of a pair block, two pairs per lane (packed float32x2).  Reciprocity of the
// mobility (M_ji = M_ij^T) lets one evaluation of the pair geometry serve the target
// (u_i += M_ij F_j, accumulated) and the source (v_j = M_ji G_i, returned): the free-space
// translation block is symmetric, and the transposed wall block swaps the roles of C3 and D3.
// TORQUE adds the translation-rotation coupling both ways: u_i += M_tr(i,j) T_j and
// v_j += M_tr(j,i) H_i.  F, T: source loads; G, H: target loads.  Per-source factors m2zj = -2 z_j,
// m4zj2 = -4 z_j^2, six_zj = 6 z_j and the target's six_zi = 6 z_i come precomputed.
// RHS2: a second translation-translation right-hand side applied with the same block, P (sources)
// and Q (targets) -> u2 (target side, accumulated) and v2 (source side, returned).
template <bool TORQUE, bool RHS2 = false>
__device__ __forceinline__ void pair_sym_x2(float2 rx, float2 ry, float2 rz, float2 rho2, float2 r2, bool close,
                                            float2 zi, float2 zj, float2 m2zj, float2 m4zj2, float2 six_zi,
                                            float2 six_zj, float2 Fx, float2 Fy, float2 Fz, float2 Gx,
                                            float2 Gy, float2 Gz, float2 Tx, float2 Ty, float2 Tz, float2 Hx,
                                            float2 Hy, float2 Hz, const X2Consts &c, float2 &ux, float2 &uy,
                                            float2 &uz, float2 &vx, float2 &vy, float2 &vz, float2 Px = {},
                                            float2 Py = {}, float2 Pz = {}, float2 Qx = {}, float2 Qy = {},
                                            float2 Qz = {}, float2 *u2 = nullptr, float2 *v2 = nullptr)
{
    TTBlock m;
    TRBlock tb;
    pair_block_x2<TORQUE>(rx, ry, rz, rho2, r2, close, zi, zj, m2zj, m4zj2, six_zi, six_zj, c, m, tb);
    tt_apply_target(m, Fx, Fy, Fz, ux, uy, uz);
    tt_apply_source(m, Gx, Gy, Gz, vx, vy, vz);
    if (RHS2) {
        tt_apply_target(m, Px, Py, Pz, u2[0], u2[1], u2[2]);
        tt_apply_source(m, Qx, Qy, Qz, v2[0], v2[1], v2[2]);
    }
    if (TORQUE) {
        tr_apply_target(m, tb, Tx, Ty, Tz, ux, uy, uz);
        tr_apply_source(m, tb, Hx, Hy, Hz, vx, vy, vz);
    }
}

// Factor m of the pair steric force m (x_i - x_j) of Sec. III: U0/b inside contact (r < 2a),
// (U0/b) e^{-(r - 2a)/b} beyond, divided by r; zero for coincident centres.  f0 = U0/b, inv_b = 1/b.
// One float64 reciprocal square root gives r and 1/r (float64 runs at a small fraction of the
// float32 rate on this GPU, and a square root plus two divisions per near pair made the batched
// force pass float64-bound).
__device__ __forceinline__ double steric_pair_factor(double r2, double two_a, double f0, double inv_b)
{
    if (!(r2 > 0.0)) return 0.0;
    const double ir = rsqrt(r2);
    const double r = r2 * ir;
    return (r < two_a ? f0 : f0 * exp((two_a - r) * inv_b)) * ir;
}

__device__ __forceinline__ double H0(double x)
{
    return x > 1.0 ? 1.0 : (x >= 0.0 ? x : 0.0);
}

}  // namespace rpb
