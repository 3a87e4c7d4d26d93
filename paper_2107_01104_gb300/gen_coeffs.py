"""Generate the interpolation-kernel coefficient tables used by the CUDA kernels.

Each kernel weight beta_i (Sec. 2.2, Eq. triple_sum) is a polynomial in the
normalised offset t = x_bar / delta in [0, 1].  The kernels evaluate it by
Horner's rule in the centred variable s = t - 1/2 (smaller powers, better
conditioned), so this script writes, for every supported (family, I, m),

    beta_i(t) = sum_d c[i][d] * (t - 1/2)^d,   i = 0..I-1  <->  node i + 1 - I/2.

All arithmetic is exact (fractions.Fraction); the table is rounded to float64
only when printed.

Families
--------
Lagrange (Sec. 2.2): beta_i is the Lagrange basis polynomial of node i on the
I nodes {1-I/2, ..., I/2}.

Spline (the family cited in Sec. 2.2): with I = 2n + 2 nodes {-n .. n+1}, the
interpolant on a cell is the degree-(2m+1) polynomial whose derivatives of
order 0..m at both cell ends equal those of the centred (2n+1)-point Lagrange
polynomial through that end node and its n neighbours on each side.
Adjacent cells share node derivatives, so the result is C^m.

Run ``python -m paper_2107_01104_gb300.gen_coeffs`` to rewrite
``csrc/coeffs.inc``.
"""
from __future__ import annotations

import os
from fractions import Fraction as F

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "csrc", "coeffs.inc")
MAX_I = 8
MAX_DEG = 10  # coefficients stored per row (degree <= 9)


def poly_mul(a, b):
    out = [F(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def poly_add(a, b):
    n = max(len(a), len(b))
    return [(a[i] if i < len(a) else F(0)) + (b[i] if i < len(b) else F(0)) for i in range(n)]


def poly_scale(a, c):
    return [x * c for x in a]


def lagrange_basis(xs, r):
    """Coefficients (increasing powers of x) of the Lagrange basis polynomial of node xs[r]."""
    p = [F(1)]
    for s, xv in enumerate(xs):
        if s == r:
            continue
        p = poly_mul(p, [-xv, F(1)])
        p = poly_scale(p, F(1) / (xs[r] - xv))
    return p


def shift_to_centre(p):
    """Given p(t) = sum a_d t^d, return q with q(s) = p(s + 1/2)."""
    half = F(1, 2)
    out = [F(0)] * len(p)
    for d, a in enumerate(p):
        # (s + 1/2)^d = sum_k C(d, k) s^k (1/2)^(d-k)
        binom = F(1)
        for k in range(d + 1):
            if k > 0:
                binom = binom * (d - k + 1) / k
            out[k] += a * binom * half ** (d - k)
    return out


def lagrange_weights(I):
    nodes = [F(j) for j in range(1 - I // 2, I // 2 + 1)]
    return [lagrange_basis(nodes, r) for r in range(I)]


def solve_exact(A, b):
    n = len(A)
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col] / M[col][col]
                M[r] = [x - f * y for x, y in zip(M[r], M[col])]
    return [M[i][n] / M[i][i] for i in range(n)]


def falling(s, q):
    out = 1
    for r in range(q):
        out *= (s - r)
    return out


def spline_weights(I, m):
    n = I // 2 - 1
    nodes = list(range(-n, n + 2))              # I nodes
    K = 2 * m + 2
    # derivative operators at node p: D_q(p) = sum_r coef[q][r] * y[p - n + r]
    xs = [F(r - n) for r in range(2 * n + 1)]   # centred stencil, relative to p
    basis = [lagrange_basis(xs, r) for r in range(2 * n + 1)]
    dop = [[falling(q, q) * (basis[r][q] if q < len(basis[r]) else F(0)) for r in range(2 * n + 1)]
           for q in range(m + 1)]
    # Hermite system: P^(q)(0) and P^(q)(1) for q = 0..m, P = sum_s h_s t^s
    A = []
    for q in range(m + 1):
        A.append([F(falling(s, q)) if s == q else F(0) for s in range(K)])
    for q in range(m + 1):
        A.append([F(falling(s, q)) if s >= q else F(0) for s in range(K)])
    weights = []
    for i in range(I):
        y = {nodes[k]: F(1 if k == i else 0) for k in range(I)}
        rhs = []
        for p in (0, 1):
            for q in range(m + 1):
                rhs.append(sum(dop[q][r] * y[p - n + r] for r in range(2 * n + 1)))
        # reorder rhs to match A (all t=0 rows, then all t=1 rows)
        b = rhs[: m + 1] + rhs[m + 1:]
        weights.append(solve_exact(A, b))
    return weights


def table(family, I, m):
    w = lagrange_weights(I) if family == 0 else spline_weights(I, m)
    w = [shift_to_centre(p) for p in w]
    deg = max(len(p) for p in w) - 1
    while deg > 0 and all((p[deg] if deg < len(p) else 0) == 0 for p in w):
        deg -= 1
    rows = [[(p[d] if d < len(p) else F(0)) for d in range(deg + 1)] for p in w]
    return deg, rows


def supported():
    out = [(0, I, 0) for I in (4, 6, 8)]
    out += [(1, I, m) for I in (4, 6, 8) for m in range(0, I // 2 + 1)]
    return out


def _rows_text(rows_by_table):
    out = ["{"]
    for rows in rows_by_table:
        out.append("  {")
        for r in range(MAX_I):
            vals = [repr(float(rows[r][d])) if (r < len(rows) and d < len(rows[r])) else "0.0" for d in range(MAX_DEG)]
            out.append("    { " + ", ".join(vals) + " },")
        out.append("  },")
    out.append("}")
    return " \\\n".join(out)


def render():
    tabs = supported()
    info, coef, dcoef = [], [], []
    for fam, I, m in tabs:
        deg, rows = table(fam, I, m)
        info.append(f"{{ {fam}, {I}, {m}, {deg} }}")
        coef.append(rows)
        # d beta / dt = d beta / ds: coefficients (d+1) c[d+1]
        dcoef.append([[(d + 1) * row[d + 1] for d in range(len(row) - 1)] for row in rows])
    lines = [
        "/* Generated by gen_coeffs.py from exact rational arithmetic.  Do not edit.",
        " * Table k describes kernel TRK_TABLE_INFO[k] = (family, I, m, degree); family 0 =",
        " * Lagrange, 1 = spline (C^m, degree 2m+1) (Sec. 2.2).  Coefficients:",
        " *   beta_i(t)  = sum_d TRK_COEF_INIT[k][i][d]  (t - 1/2)^d",
        " *   beta_i'(t) = sum_d TRK_DCOEF_INIT[k][i][d] (t - 1/2)^d",
        " * for node i + 1 - I/2, i = 0..I-1. */",
        f"#define TRK_NUM_TABLES {len(tabs)}",
        f"#define TRK_TAB_MAX_I {MAX_I}",
        f"#define TRK_TAB_MAX_DEG {MAX_DEG}",
        "#define TRK_TABLE_INFO { " + ", ".join(info) + " }",
        "#define TRK_COEF_INIT " + _rows_text(coef),
        "#define TRK_DCOEF_INIT " + _rows_text(dcoef),
    ]
    return "\n".join(lines) + "\n"


def main():
    with open(OUT, "w") as fh:
        fh.write(render())
    print(OUT)


if __name__ == "__main__":
    main()
