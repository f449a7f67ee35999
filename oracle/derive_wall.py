"""Symbolic derivation of the wall (image) part of the Rotne-Prager-Blake mobility.

TEST INFRASTRUCTURE ONLY: this file, and everything under oracle/, is the plain
CPU reference that the CUDA path is checked against.  Only tests/, the smoke
check and the CPU-baseline leg of the benchmark may use it.

What is derived (Sec. II.B, Eq. (mobilityDifferential) and Sec. III,
Eq. (mobilityDifferentialTR)):

    M_tt(q_i, q_j) = (I + a^2/6 lap_x) (I + a^2/6 lap_y) G(x, y)      at x=q_i, y=q_j
    M_tr(q_i, q_j) = (I + a^2/6 lap_x) (1/2 curl_y) G(x, y)           at x=q_i, y=q_j

G is the Green's function of Stokes flow above a no-slip wall at z=0 (Blake's
image solution, cited in Sec. II.B).  G = Oseen(x - y) + G_img(x, y); the
free-space Oseen part, together with the overlap branch of the Rotne-Prager-
Yamakawa tensor, is written by hand in rpb_oracle.c.  Here only the image part
is handled, mechanically: sympy builds G_img from its textbook form, applies
the Faxen operators literally (second and fourth derivatives, no hand
simplification) and prints C code with common-subexpression elimination.

Image part, with y* = (y1, y2, -y3) the mirror point of the source, R = x - y*,
h = y3, P = diag(1, 1, -1), S_ij(v) = delta_ij/|v| + v_i v_j/|v|^3:

    8 pi eta G_img_ij = -S_ij(R) + 2 h P_jk d/dR_k [ h R_i/|R|^3 - (delta_i3/|R| + R_i R_3/|R|^3) ]

(index i: velocity component at x; index j: force component at y; the R-derivative
is taken with h held fixed).  This form is not trusted: tests/test_oracle_wall.py
checks that Oseen + G_img vanishes on the wall, that it is divergence free in x,
and that the Faxen-operated blocks equal the sphere-surface averages of
Eq. (mobilityOverlap), which pins both the image system and the operator step.

The torque coupling uses u_i = 1/2 eps_{mkl} d/dy_k G_il T_m, i.e. the flow of a
point couple; it reduces to T x r / (8 pi eta |r|^3) for the Oseen tensor.

Run:  python oracle/derive_wall.py   (rewrites oracle/wall_image.c)
"""
import os
import sys
import time

import sympy as sp


def derive():
    x1, x2, x3, y1, y2, y3, a = sp.symbols("x1 x2 x3 y1 y2 y3 a", real=True)
    R1, R2, R3, H = sp.symbols("R1 R2 R3 H", real=True)
    Rv = [R1, R2, R3]
    Rn = sp.sqrt(R1**2 + R2**2 + R3**2)

    def S(v, n):
        return sp.Matrix(3, 3, lambda i, j: sp.KroneckerDelta(i, j) / n + v[i] * v[j] / n**3)

    P = sp.diag(1, 1, -1)
    # bracket_i = h R_i/|R|^3 - (delta_i3/|R| + R_i R_3/|R|^3)
    bracket = [H * Rv[i] / Rn**3 - (sp.KroneckerDelta(i, 2) / Rn + Rv[i] * Rv[2] / Rn**3) for i in range(3)]
    Gimg_R = sp.zeros(3, 3)
    SR = S(Rv, Rn)
    for i in range(3):
        for j in range(3):
            acc = -SR[i, j]
            for k in range(3):
                if P[j, k] != 0:
                    acc += 2 * H * P[j, k] * sp.diff(bracket[i], Rv[k])
            Gimg_R[i, j] = acc
    subs = {R1: x1 - y1, R2: x2 - y2, R3: x3 + y3, H: y3}
    Gimg = Gimg_R.subs(subs)

    X = [x1, x2, x3]
    Y = [y1, y2, y3]

    def lap(expr, vars_):
        return sum(sp.diff(expr, v, 2) for v in vars_)

    # translation-translation: (1 + a^2/6 lap_x)(1 + a^2/6 lap_y) G_img
    tt = sp.zeros(3, 3)
    for i in range(3):
        for j in range(3):
            g = Gimg[i, j]
            gy = g + a**2 / 6 * lap(g, Y)
            tt[i, j] = gy + a**2 / 6 * lap(gy, X)
    # translation-rotation: (1 + a^2/6 lap_x) (1/2 eps_{mkl} d/dy_k G_il); column m = torque component
    eps = sp.LeviCivita
    tr = sp.zeros(3, 3)
    for i in range(3):
        for m in range(3):
            c = 0
            for k in range(3):
                for l in range(3):
                    e = eps(m, k, l)
                    if e != 0:
                        c += sp.Rational(1, 2) * e * sp.diff(Gimg[i, l], Y[k])
            tr[i, m] = c + a**2 / 6 * lap(c, X)

    # express in (rx, ry, zi, zj): rx = x1 - y1, ry = x2 - y2, zi = x3 (target), zj = y3 (source)
    rx, ry, zi, zj = sp.symbols("rx ry zi zj", real=True)
    fin = {x1: y1 + rx, x2: y2 + ry, x3: zi, y3: zj}
    return (Gimg.subs(fin), tt.subs(fin), tr.subs(fin)), (rx, ry, zi, zj, a)


def emit_c(name, mat, args, out):
    syms = list(mat)
    reps, red = sp.cse(syms, symbols=sp.numbered_symbols("t"), optimizations="basic")
    lines = []
    argdecl = ", ".join("double " + str(s) for s in args)
    lines.append(f"void {name}({argdecl}, double *out)")
    lines.append("{")
    for s, e in reps:
        lines.append(f"    const double {s} = {sp.ccode(e)};")
    for idx, e in enumerate(red):
        lines.append(f"    out[{idx}] = {sp.ccode(e)};")
    lines.append("}")
    out.write("\n".join(lines) + "\n\n")


def main():
    t0 = time.time()
    (Gimg, tt, tr), (rx, ry, zi, zj, a) = derive()
    here = os.path.dirname(os.path.abspath(__file__))
    path = os.path.join(here, "wall_image.c")
    with open(path, "w") as f:
        f.write("/* GENERATED by oracle/derive_wall.py -- do not edit.  Oracle (test infrastructure) only.\n")
        f.write(" * Image (wall) part of the Rotne-Prager-Blake tensors, row-major 3x3, all in units of\n")
        f.write(" * 1/(8 pi eta).  rx, ry: in-plane target-minus-source offset; zi: target height; zj: source\n")
        f.write(" * height (both above the wall).  out[3*i + j]: velocity component i, force/torque component j.\n")
        f.write(" * blake_image_raw: 8 pi eta G_img (no Faxen operators).\n")
        f.write(" * wall_image_tt:   (I + a^2/6 lap_x)(I + a^2/6 lap_y) 8 pi eta G_img.\n")
        f.write(" * wall_image_tr:   (I + a^2/6 lap_x)(1/2 curl_y) 8 pi eta G_img. */\n")
        f.write("#include <math.h>\n\n")
        emit_c("blake_image_raw", Gimg, (rx, ry, zi, zj), f)
        emit_c("wall_image_tt", tt, (rx, ry, zi, zj, a), f)
        emit_c("wall_image_tr", tr, (rx, ry, zi, zj, a), f)
    print(f"wrote {path} in {time.time() - t0:.1f}s", file=sys.stderr)


if __name__ == "__main__":
    main()
