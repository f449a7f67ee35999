/* mcmc.c -- Metropolis Monte Carlo sample of the Gibbs-Boltzmann distribution exp(-U/kT) of spheres
 * above a wall (Appendix B: the "exact" equilibrium that the Brownian dynamics must reproduce).
 *
 * TEST INFRASTRUCTURE ONLY: see oracle/__init__.py.
 *
 * Energy (Sec. III): gravity weight * z_i for every sphere, the soft potential of Eq. (soft_potential)
 *   U(r) = U0 + U0 (d - r)/b  for r < d,   U0 exp(-(r - d)/b)  for r >= d,
 * with the wall (d = a, r = the height) and between every pair (d = 2a, r = the centre distance).
 * With periods Lx, Ly > 0 the suspension is periodic in x and y and pairs interact through their
 * minimum image (Appendix B); with Lx = Ly = 0 it is unbounded in-plane.
 *
 * Moves: the standard single-particle Metropolis step (Allen & Tildesley, cited in Appendix B):
 * sphere i (taken in order) is displaced by a uniform vector in [-step, step]^3 and the move is
 * accepted with probability min(1, exp(-dU/kT)).  The random numbers come from the caller (four
 * uniforms in [0, 1) per move), so this file holds no generator.
 */
#include <math.h>
#include <stdint.h>

static double soft_energy(double r, double d, double U0, double b)
{
    if (r < d) return U0 + U0 * (d - r) / b;
    return U0 * exp(-(r - d) / b);
}

static double wrap_diff(double d, double L)
{
    return L > 0.0 ? d - L * nearbyint(d / L) : d;
}

static double one_body(double z, double a, double weight, double U0, double b)
{
    return weight * z + soft_energy(z, a, U0, b);
}

/* energy of sphere i at position p with all others (pairs only) */
static double pair_energy_of(int64_t N, const double *pos, int64_t i, const double *p, double a, double U0, double b,
                             double Lx, double Ly)
{
    double e = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        if (j == i) continue;
        const double dx = wrap_diff(p[0] - pos[3 * j], Lx), dy = wrap_diff(p[1] - pos[3 * j + 1], Ly);
        const double dz = p[2] - pos[3 * j + 2];
        e += soft_energy(sqrt(dx * dx + dy * dy + dz * dz), 2.0 * a, U0, b);
    }
    return e;
}

/* Total energy U (one-body terms plus every pair once). */
double oracle_mc_energy(int64_t N, const double *pos, double a, double weight, double U0, double b, double Lx,
                        double Ly)
{
    double e = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        e += one_body(pos[3 * i + 2], a, weight, U0, b);
        for (int64_t j = i + 1; j < N; ++j) {
            const double dx = wrap_diff(pos[3 * i] - pos[3 * j], Lx), dy = wrap_diff(pos[3 * i + 1] - pos[3 * j + 1], Ly);
            const double dz = pos[3 * i + 2] - pos[3 * j + 2];
            e += soft_energy(sqrt(dx * dx + dy * dy + dz * dz), 2.0 * a, U0, b);
        }
    }
    return e;
}

/* nsweeps sweeps (N moves each) in place; u: 4 N nsweeps uniforms in [0, 1).  Returns the number of
 * accepted moves.  Positions are folded back into [0, L) in periodic directions. */
int64_t oracle_mc_sweeps(int64_t N, double *pos, int64_t nsweeps, const double *u, double step, double kT, double a,
                         double weight, double U0, double b, double Lx, double Ly)
{
    int64_t acc = 0;
    for (int64_t s = 0; s < nsweeps; ++s)
        for (int64_t i = 0; i < N; ++i) {
            const double *r = &u[4 * (s * N + i)];
            const double *q = &pos[3 * i];
            double p[3] = {q[0] + step * (2.0 * r[0] - 1.0), q[1] + step * (2.0 * r[1] - 1.0),
                           q[2] + step * (2.0 * r[2] - 1.0)};
            const double dU = one_body(p[2], a, weight, U0, b) - one_body(q[2], a, weight, U0, b) +
                              pair_energy_of(N, pos, i, p, a, U0, b, Lx, Ly) -
                              pair_energy_of(N, pos, i, q, a, U0, b, Lx, Ly);
            if (dU <= 0.0 || r[3] < exp(-dU / kT)) {
                if (Lx > 0.0) p[0] -= Lx * floor(p[0] / Lx);
                if (Ly > 0.0) p[1] -= Ly * floor(p[1] / Ly);
                pos[3 * i] = p[0];
                pos[3 * i + 1] = p[1];
                pos[3 * i + 2] = p[2];
                ++acc;
            }
        }
    return acc;
}
