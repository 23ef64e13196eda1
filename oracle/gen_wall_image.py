"""Generate ``oracle/wall_image.py``: the regularised Blake image part of the
Rotne-Prager-Blake blob mobility.

TEST INFRASTRUCTURE ONLY: this file belongs to the CPU oracle.

What is derived (Sec. 2.3, Eq. RPY: the blob mobility is the double surface
average of the Green's function over the two blob surfaces; the no-slip wall
case uses the Green's function of a Stokeslet above a plane wall, Blake 1971,
as the paper's wall-corrected RPY reference does):

Blake's Green's function for a point force F at y (height h = y_3 > 0) above
the no-slip plane z = 0, evaluated at x, is

    8 pi eta u_i = F_j [ S_ij(r) - S_ij(R)
                         + 2 h D_jl d/dR_l ( h R_i / R^3 - delta_i3 / R
                                              - R_i R_3 / R^3 ) ]

with r = x - y, R = x - y*, y* = (y_1, y_2, -y_3), S_ij(v) = delta_ij/|v| +
v_i v_j/|v|^3 (the Oseen tensor) and D = diag(1, 1, -1).

Every term after S_ij(r) (the "image part") is, as a function of x, a Stokes
flow that is regular in the upper half space; by reciprocity of the full
Green's function it is also one as a function of y.  Its components are
therefore biharmonic in x and in y there, and the exact average over a sphere
of radius a of a biharmonic f is f + (a^2/6) lap f.  The double surface
average of the image part is thus exactly

    (1 + a^2/6 lap_x)(1 + a^2/6 lap_y) G_img(x, y) / (8 pi eta),

for any two blobs whose centres are higher than a.  This script forms that
expression symbolically with sympy (plain differentiation of the formula
above, no simplification beyond common-subexpression elimination) and writes
it out as straight-line numpy code of the variables

    Rx = x_1 - y_1, Ry = x_2 - y_2, Rz = x_3 + y_3, h = y_3, a

so the generated function is vectorised over pairs.  The free-space part
S_ij(r) is handled in ``oracle/mobility.py`` by the closed-form RPY tensor.

Run:  python oracle/gen_wall_image.py   (writes oracle/wall_image.py)
"""
import os
import sympy as sp


def blake_image_tensor(x, y):
    """8*pi*eta times the image part of Blake's Green's function, G_img[i][j]
    (i: velocity component at x, j: force component at y)."""
    h = y[2]
    R = sp.Matrix([x[0] - y[0], x[1] - y[1], x[2] + y[2]])
    Rn = sp.sqrt(R.dot(R))
    D = [1, 1, -1]
    G = [[None] * 3 for _ in range(3)]
    for i in range(3):
        di3 = 1 if i == 2 else 0
        # Phi_i(R) = h R_i / R^3 - delta_i3 / R - R_i R_3 / R^3
        phi_i = h * R[i] / Rn**3 - di3 / Rn - R[i] * R[2] / Rn**3
        for j in range(3):
            dij = 1 if i == j else 0
            oseen_image = dij / Rn + R[i] * R[j] / Rn**3
            # d/dR_l of Phi_i with h held fixed; R_l depends on x_l with unit
            # derivative, so differentiate with respect to x_l.
            dphi = sp.diff(phi_i, x[j])
            G[i][j] = -oseen_image + 2 * h * D[j] * dphi
    return G


def regularised(G, x, y, a):
    def lap(f, v):
        return sum(sp.diff(f, vk, 2) for vk in v)
    out = [[None] * 3 for _ in range(3)]
    for i in range(3):
        for j in range(3):
            g = G[i][j]
            lx = lap(g, x)
            ly = lap(g, y)
            lxy = lap(lx, y)
            out[i][j] = g + a**2 / 6 * (lx + ly) + a**4 / 36 * lxy
    return out


def main():
    x = sp.symbols("x1 x2 x3", real=True)
    y = sp.symbols("y1 y2 y3", real=True)
    a = sp.Symbol("a", positive=True)
    Rx, Ry, Rz, h = sp.symbols("Rx Ry Rz h", real=True)
    G = blake_image_tensor(x, y)
    W = regularised(G, x, y, a)
    subs = {x[0]: Rx + y[0], x[1]: Ry + y[1], x[2]: Rz - y[2]}
    exprs = []
    for i in range(3):
        for j in range(3):
            e = W[i][j].subs(subs).subs(y[2], h)
            exprs.append(e)
    assert all(e.free_symbols <= {Rx, Ry, Rz, h, a} for e in exprs)
    repl, reduced = sp.cse(exprs, symbols=sp.numbered_symbols("t"))
    lines = [
        '"""GENERATED by oracle/gen_wall_image.py -- do not edit.',
        "",
        "TEST INFRASTRUCTURE ONLY: part of the CPU oracle.",
        "",
        "Regularised image part of the Rotne-Prager-Blake blob mobility",
        "(Sec. 2.3, Eq. RPY with Blake's wall Green's function), times 8*pi*eta.",
        "Arguments are numpy float64 arrays (broadcast together):",
        "Rx, Ry, Rz = target minus image of source, h = source height, a = blob radius.",
        "Returns a (..., 3, 3) array W[..., i, j]: velocity i at the target from",
        "force j at the source.",
        '"""',
        "import numpy as np",
        "",
        "",
        "def wall_image_8pieta(Rx, Ry, Rz, h, a):",
        "    sqrt = np.sqrt",
    ]
    from sympy.printing.pycode import PythonCodePrinter
    printer = PythonCodePrinter({"fully_qualified_modules": False})

    def code(e):
        s = printer.doprint(e)
        return s.replace("math.sqrt", "sqrt")

    for sym, e in repl:
        lines.append(f"    {sym} = {code(e)}")
    lines.append("    W = np.empty(np.broadcast(Rx, Ry, Rz, h).shape + (3, 3))")
    for k, e in enumerate(reduced):
        i, j = divmod(k, 3)
        lines.append(f"    W[..., {i}, {j}] = {code(e)}")
    lines.append("    return W")
    lines.append("")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "wall_image.py")
    with open(path, "w") as f:
        f.write("\n".join(lines))
    print("wrote", path, "with", len(repl), "subexpressions")


if __name__ == "__main__":
    main()
