"""Generate bgk_tables.h: exact reference-element constants of the nodal DG sweep.

For an affine simplex K with outward area-weighted face normals N_i (face i opposite
vertex i) the gradient of the barycentric coordinate is grad l_i = -N_i / (d |K|), so
every cell matrix of the upwind DG local problem (Sec. 3.3, Eq. bgk-ss-inflow-outflow)
is a fixed combination of |K| and s_i = v . N_i:

  A / |K| = nu_s Mh + sum_i (s_i/|K|) (Dd_i + [s_i > 0] Eh_i)
  b / |K| = Mh src + sum_{s_i < 0} (-s_i/|K|) Eh_i y_up

with Mh = (1/|K|) int phi_a phi_b, Dd_i = (1/(d |K|)) int phi_b d phi_a / d l_i and
Eh_i = (1/|F_i|) int_{F_i} phi_a phi_b.  This script integrates the products exactly
with rational arithmetic (int over a k-simplex of prod l^e = k! |S| prod e! / (k+|e|)!)
and writes them as constexpr doubles.  Q1 parallelograms: see q1_tables.
Run: python gen_tables.py > bgk_tables.h
"""
from fractions import Fraction as Fr
from math import factorial


def basis(kind):
    """Polynomials in barycentric coordinates as {exponent tuple: coefficient}."""
    if kind == "p1tri":
        nv = 3
        return nv, [{tuple(1 if k == a else 0 for k in range(nv)): Fr(1)} for a in range(nv)]
    if kind == "p1tet":
        nv = 4
        return nv, [{tuple(1 if k == a else 0 for k in range(nv)): Fr(1)} for a in range(nv)]
    if kind == "p2tri":
        nv = 3
        out = []
        for a in range(3):
            e2 = tuple(2 if k == a else 0 for k in range(3))
            e1 = tuple(1 if k == a else 0 for k in range(3))
            out.append({e2: Fr(2), e1: Fr(-1)})
        for k in range(3):
            l = (k + 1) % 3
            e = [0, 0, 0]
            e[k] += 1
            e[l] += 1
            out.append({tuple(e): Fr(4)})
        return nv, out
    raise ValueError(kind)


def mul(p, q):
    r = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            r[e] = r.get(e, 0) + ca * cb
    return r


def dl(p, i):
    r = {}
    for e, c in p.items():
        if e[i]:
            e2 = list(e)
            e2[i] -= 1
            r[tuple(e2)] = r.get(tuple(e2), 0) + c * e[i]
    return r


def integ(p, k, skip=None):
    """(1/|S|) int over the k-simplex spanned by the coordinates other than `skip`."""
    s = Fr(0)
    for e, c in p.items():
        if skip is not None and e[skip]:
            continue
        ee = [x for i, x in enumerate(e) if i != skip]
        num = factorial(k)
        for x in ee:
            num *= factorial(x)
        s += c * Fr(num, factorial(k + sum(ee)))
    return s


def q1_tables():
    """Q1 on a parallelogram K = x0 + J [0,1]^2, nodes at the vertices in cell order
    (phi_0 = (1-s)(1-t), phi_1 = s(1-t), phi_2 = st, phi_3 = (1-s)t), face i from vertex i
    to vertex i+1.  The area-weighted outward normal of the face s = 1 (face 1) is
    N_1 = |K| J^-T e_s and that of t = 1 (face 2) is N_2 = |K| J^-T e_t, the opposite faces'
    are their negatives, so v . grad phi = (s_1 d_s + s_2 d_t) phi / |K| with s_i = v . N_i:

      -(1/|K|) int phi_b v.grad phi_a = -r_1 G_s[a][b] - r_2 G_t[a][b],   G_x = int_[0,1]^2 phi_b d_x phi_a

    written symmetrically over the opposite faces (r_3 = -r_1, r_0 = -r_2):
    Dd_1 = -G_s/2, Dd_3 = +G_s/2, Dd_2 = -G_t/2, Dd_0 = +G_t/2.  Mh = int phi_a phi_b over
    the unit square, Eh_i the edge mass over the unit edge."""
    # polynomials in (s, t) as {(p, q): coefficient}
    one = {(0, 0): Fr(1)}
    s_ = {(1, 0): Fr(1)}
    t_ = {(0, 1): Fr(1)}
    oms = {(0, 0): Fr(1), (1, 0): Fr(-1)}
    omt = {(0, 0): Fr(1), (0, 1): Fr(-1)}
    phi = [mul(oms, omt), mul(s_, omt), mul(s_, t_), mul(oms, t_)]
    del one

    def d(p, k):
        r = {}
        for e, c in p.items():
            if e[k]:
                e2 = list(e)
                e2[k] -= 1
                r[tuple(e2)] = r.get(tuple(e2), 0) + c * e[k]
        return r

    def sq(p):
        return sum(c * Fr(1, (e[0] + 1) * (e[1] + 1)) for e, c in p.items())

    def edge(p, i):
        # face i: (0) t=0, s from 0 to 1; (1) s=1; (2) t=1; (3) s=0 -- integrate over the unit edge
        tot = Fr(0)
        for e, c in p.items():
            if i == 0:
                tot += c * (Fr(1, e[0] + 1) if e[1] == 0 else 0)
            elif i == 1:
                tot += c * Fr(1, e[1] + 1)
            elif i == 2:
                tot += c * Fr(1, e[0] + 1)
            else:
                tot += c * (Fr(1, e[1] + 1) if e[0] == 0 else 0)
        return tot
    nd = 4
    Mh = [[sq(mul(phi[a], phi[b])) for b in range(nd)] for a in range(nd)]
    Gs = [[sq(mul(phi[b], d(phi[a], 0))) for b in range(nd)] for a in range(nd)]
    Gt = [[sq(mul(phi[b], d(phi[a], 1))) for b in range(nd)] for a in range(nd)]
    half = Fr(1, 2)
    Dd = [[[Gt[a][b] * half for b in range(nd)] for a in range(nd)],
          [[-Gs[a][b] * half for b in range(nd)] for a in range(nd)],
          [[-Gt[a][b] * half for b in range(nd)] for a in range(nd)],
          [[Gs[a][b] * half for b in range(nd)] for a in range(nd)]]
    Eh = [[[edge(mul(phi[a], phi[b]), i) for b in range(nd)] for a in range(nd)] for i in range(4)]
    fn = [[i, (i + 1) % 4] for i in range(4)]
    return 2, nd, 4, Mh, Dd, Eh, fn


def tables(kind):
    if kind == "q1quad":
        return q1_tables()
    nv, phi = basis(kind)
    d = nv - 1
    nd = len(phi)
    Mh = [[integ(mul(phi[a], phi[b]), d) for b in range(nd)] for a in range(nd)]
    Dd = [[[integ(mul(phi[b], dl(phi[a], i)), d) / d for b in range(nd)] for a in range(nd)] for i in range(nv)]
    Eh = [[[integ(mul(phi[a], phi[b]), d - 1, skip=i) for b in range(nd)] for a in range(nd)] for i in range(nv)]
    # local nodes on face i (opposite vertex i): vertices != i ascending, then the midpoint
    fn = []
    for i in range(nv):
        f = [a for a in range(nv) if a != i]
        if kind == "p2tri":
            f.append(3 + (i + 1) % 3)
        fn.append(f)
    return d, nd, nv, Mh, Dd, Eh, fn


def lit(x):
    return "T(%.17g)" % float(x)


def emit(name, kind):
    """Struct with sizes, the face-node map, and device routines in which every zero of
    the tables has been dropped at generation time."""
    d, nd, nf, Mh, Dd, Eh, fn = tables(kind)
    fd = len(fn[0])
    o = ["struct %s {" % name,
         "  static constexpr int D = %d, NDOF = %d, NF = %d, FD = %d;" % (d, nd, nf, fd),
         "  BGK_HD static constexpr int fn(int i, int k) {",
         "    return " + " : ".join("(i == %d && k == %d) ? %d" % (i, k, fn[i][k])
                                    for i in range(nf) for k in range(fd)) + " : -1;",
         "  }",
         "#ifdef __CUDACC__"]
    # A = nus*Mh + sum_i r_i Dd_i + sum_{i outflow} r_i Eh_i
    o.append("  template <typename T> __device__ static __forceinline__ void assemble("
             "T nus, const T (&r)[%d], unsigned outm, T (&A)[%d][%d]) {" % (nf, nd, nd))
    for a in range(nd):
        for b in range(nd):
            terms = []
            if Mh[a][b] != 0:
                terms.append("nus * %s" % lit(Mh[a][b]))
            for i in range(nf):
                if Dd[i][a][b] != 0:
                    terms.append("r[%d] * %s" % (i, lit(Dd[i][a][b])))
            o.append("    A[%d][%d] = %s;" % (a, b, " + ".join(terms) if terms else "T(0)"))
    for i in range(nf):
        nz = [(a, b) for a in range(nd) for b in range(nd) if Eh[i][a][b] != 0]
        o.append("    if (outm & %du) {" % (1 << i))
        for a, b in nz:
            o.append("      A[%d][%d] += r[%d] * %s;" % (a, b, i, lit(Eh[i][a][b])))
        o.append("    }")
    o.append("  }")
    # b = Mh src
    o.append("  template <typename T> __device__ static __forceinline__ void mass("
             "const T (&s)[%d], T (&b)[%d]) {" % (nd, nd))
    for a in range(nd):
        terms = ["s[%d] * %s" % (b, lit(Mh[a][b])) for b in range(nd) if Mh[a][b] != 0]
        o.append("    b[%d] = %s;" % (a, " + ".join(terms)))
    o.append("  }")
    # b += c * Eh_i y, y in face-local order
    o.append("  template <typename T> __device__ static __forceinline__ void inflow("
             "int i, T c, const T (&y)[%d], T (&b)[%d]) {" % (fd, nd))
    o.append("    switch (i) {")
    for i in range(nf):
        o.append("      case %d:" % i)
        for a in range(nd):
            terms = ["y[%d] * %s" % (k, lit(Eh[i][a][fn[i][k]])) for k in range(fd) if Eh[i][a][fn[i][k]] != 0]
            if terms:
                o.append("        b[%d] += c * (%s);" % (a, " + ".join(terms)))
        o.append("        break;")
    o.append("      default: break;")
    o.append("    }")
    o.append("  }")
    # the same with the face mass written as (1/den) x integers that are all signed powers
    # of two: b += (c/den) * sum_k n_k y_k, the products by n_k exact scalings (float pairs)
    den = 1
    for i in range(nf):
        for a in range(nd):
            for k in range(fd):
                x = Eh[i][a][fn[i][k]]
                den = den * x.denominator // _gcd(den, x.denominator)
    ints = all(_pow2(abs(Eh[i][a][fn[i][k]] * den)) for i in range(nf) for a in range(nd) for k in range(fd)
               if Eh[i][a][fn[i][k]] != 0)
    if ints:
        o.append("  static constexpr double inflow_den = %d.0;" % den)
        o.append("  template <typename T> __device__ static __forceinline__ void inflow_int("
                 "int i, T c_den, const T (&y)[%d], T (&b)[%d]) {" % (fd, nd))
        o.append("    switch (i) {")
        for i in range(nf):
            o.append("      case %d:" % i)
            for a in range(nd):
                terms = ["y[%d] * %.1ff" % (k, float(Eh[i][a][fn[i][k]] * den)) for k in range(fd)
                         if Eh[i][a][fn[i][k]] != 0]
                if terms:
                    o.append("        b[%d] += c_den * (%s);" % (a, " + ".join(terms)))
            o.append("        break;")
        o.append("      default: break;")
        o.append("    }")
        o.append("  }")
    o.append("#endif")
    o.append("};")
    return "\n".join(o)


def _gcd(a, b):
    while b:
        a, b = b, a % b
    return a


def _pow2(x):
    """x a positive integer power of two (Fraction or int)."""
    return x > 0 and x.denominator == 1 and (int(x) & (int(x) - 1)) == 0


if __name__ == "__main__":
    print("// Generated by gen_tables.py -- exact reference-element tables (see that file).")
    print("#pragma once")
    print("#ifndef __CUDACC__")
    print("#define BGK_HD")
    print("#else")
    print("#define BGK_HD __host__ __device__")
    print("#endif")
    for name, kind in (("ElemP1Tri", "p1tri"), ("ElemP2Tri", "p2tri"), ("ElemP1Tet", "p1tet"), ("ElemQ1Quad", "q1quad")):
        print(emit(name, kind))
