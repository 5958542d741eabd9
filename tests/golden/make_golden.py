"""Write tests/golden/linear_closed_form.json: exact values of the continuous
skew-symmetric advection operator for linear velocity fields.

The PW scheme (Sec. 2.2) is the centred discretisation of
    S(q) = -1/2 [ (u.grad) q + div(u q) ] = -(u.grad) q - 1/2 q div(u)
for q = u, v, w on an Arakawa-C grid.  For u_a(x) = A[a][0] + sum_b A[a][1+b] x_b
the operator is  S_a = -sum_b u_b A[a][1+b] - 1/2 u_a trace(B),  B = A[:, 1:],
and on a uniform grid the scheme reproduces it exactly at every level that is
neither the surface nor the lid.  This script evaluates that closed form in
exact rational arithmetic (fractions.Fraction) at the staggered points of a
4 x 4 x 4 grid with dx = 2, dy = 4, dz = 1; it calls neither the oracle nor the
CUDA library.  Positions: u(k,j,i) at (i dx, (j-1/2) dy, (k-3/2) dz),
v at ((i-1/2) dx, j dy, (k-3/2) dz), w at ((i-1/2) dx, (j-1/2) dy, (k-1) dz).
"""
import json
import os
from fractions import Fraction as F

NX = NY = NZ = 4
DX, DY, DZ = 2, 4, 1
A = [[3, 1, -2, 2], [-1, 2, 1, -3], [2, -1, 3, 1]]


def pos(q, k, j, i):
    h = F(1, 2)
    if q == 0:
        return (i * DX, (j - h) * DY, (k - 3 * h) * DZ)
    if q == 1:
        return ((i - h) * DX, j * DY, (k - 3 * h) * DZ)
    return ((i - h) * DX, (j - h) * DY, (k - 1) * DZ)


def vel(b, x):
    a = A[b]
    return a[0] + a[1] * x[0] + a[2] * x[1] + a[3] * x[2]


def S(q, x):
    tr = A[0][1] + A[1][2] + A[2][3]
    return -sum(vel(b, x) * A[q][1 + b] for b in range(3)) - F(1, 2) * vel(q, x) * tr


def main():
    out = {"citation": "Sec. 2.2 (PW scheme); closed form of the skew-symmetric operator for linear fields",
           "nx": NX, "ny": NY, "nz": NZ, "dx": DX, "dy": DY, "dz": DZ, "A": A}
    for q, name in enumerate(("su", "sv", "sw")):
        rows = []
        for k in range(2, NZ):
            for j in range(1, NY + 1):
                for i in range(1, NX + 1):
                    val = S(q, pos(q, k, j, i))
                    rows.append([[k, j, i], val.numerator, val.denominator])
        out[name] = rows
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "linear_closed_form.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=0)
    print(path)


if __name__ == "__main__":
    main()
