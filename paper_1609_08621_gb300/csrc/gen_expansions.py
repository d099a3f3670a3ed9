"""Generate ``expansions.cuh``: straight-line FP32 device code for the expansion operators.

Run ``python gen_expansions.py`` after editing; the generated header is committed so
that building needs only nvcc.

Green's function: Plummer, G(r) = (r.r + eps^2)^(-1/2) (the softened kernel of the
direct sum, used for every interaction so that the expansion converges to it).  It
depends on r only through s = r.r, so its derivative tensors are those of 1/r with
R = sqrt(r.r + eps^2) in place of |r| in the radial factors.

FP32 range.  For R near the softening length (~1e-4) the order-5 factor R^-11 would
overflow single precision, so every operator works with the unit-free vector
q = r / R and scaled derivatives

    Dhat^m(q) = R^(|m|+1) D^m G(r)
              = sum_{i,j,k} H(a,i) H(b,j) H(c,k) q^(m - 2(i,j,k)) c_(|m| - i - j - k),

with H(n,p) = n! / (2^p p! (n-2p)!) (ways to pick p index pairs) and
c_n = (-1)^n (2n-1)!!.  Moments enter scaled by R^-|n|, powers of 1/R are applied
order by order.

Multi-indices n = (a,b,c) are ordered by total order, then a descending, then b
descending.  Moment records hold [M, M2 (6), M3 (10), M4 (15)] -- raw moments
sum_j m_j y_j^n about the centre of mass (the dipole vanishes there) -- followed
by the traces used by the particle-cell kernel:
[trM2, trM3 (3), trM4 (6), trtrM4, pad]  (44 floats).
Local coefficients are L_k = D^k Phi(c), |k| <= 5 (56 floats), with
Phi(x) = sum_j m_j G(x - x_j), acceleration = grad Phi, potential = -Phi.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

ORDER_L = 5  # local expansion order (Sec. 3.1: "done to 5th order")
ORDER_M = 4  # multipole order (Sec. 3.1: "4th order moments")


def mindices(order):
    out = []
    for o in range(order + 1):
        for a in range(o, -1, -1):
            for b in range(o - a, -1, -1):
                out.append((a, b, o - a - b))
    return out


MI = mindices(ORDER_L)
IDX = {n: i for i, n in enumerate(MI)}
NL = len(MI)  # 56

# moment record slots
MOM = [(0, 0, 0)] + [n for n in MI if sum(n) in (2, 3, 4)]
MSLOT = {n: i for i, n in enumerate(MOM)}  # 32 slots
NMOM = len(MOM)
TR2 = 32
TR3 = {0: 33, 1: 34, 2: 35}
TR4 = {n: 36 + i for i, n in enumerate(n for n in MI if sum(n) == 2)}
TT4 = 42
NREC = 44


def add(n, m):
    return tuple(x + y for x, y in zip(n, m))


def sub(n, m):
    return tuple(x - y for x, y in zip(n, m))


E = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]


def nfact(n):
    return math.factorial(n[0]) * math.factorial(n[1]) * math.factorial(n[2])


def lit(v):
    """float literal"""
    if isinstance(v, Fraction):
        v = float(v)
    s = repr(float(v))
    if "e" not in s and "." not in s:
        s += ".0"
    return s + "f"


def herm(n, p):
    return Fraction(math.factorial(n), (2 ** p) * math.factorial(p) * math.factorial(n - 2 * p))


def cfac(n):
    # (-1)^n (2n-1)!!
    v = 1
    for k in range(1, 2 * n, 2):
        v *= k
    return (-1) ** n * v


def mono_name(n):
    return f"q{n[0]}{n[1]}{n[2]}"


def emit_monomials(var, order, names=None, decl="float"):
    """Code computing var-monomials up to order (prefix var), returns lines."""
    lines = []
    for o in range(1, order + 1):
        for n in mindices(o):
            if sum(n) != o:
                continue
            # build from a lower monomial
            for ax in range(3):
                if n[ax] > 0:
                    lo = list(n)
                    lo[ax] -= 1
                    lo = tuple(lo)
                    break
            comp = "xyz"[ax]
            if sum(lo) == 0:
                lines.append(f"    const {decl} {var}{n[0]}{n[1]}{n[2]} = {var}{comp};")
            else:
                lines.append(f"    const {decl} {var}{n[0]}{n[1]}{n[2]} = {var}{lo[0]}{lo[1]}{lo[2]} * {var}{comp};")
    return lines


def mono_ref(var, n):
    if sum(n) == 0:
        return None
    if sum(n) == 1:
        return var + "xyz"[n.index(1)]
    return f"{var}{n[0]}{n[1]}{n[2]}"


def gen_green_scaled():
    """Dhat[56] from q (|q| <= 1) and the scalars c_n."""
    L = ["__device__ __forceinline__ void fmm_green_scaled(float qx, float qy, float qz, float* __restrict__ D)", "{"]
    L += emit_monomials("q", ORDER_L)
    for n in MI:
        a, b, c = n
        terms = []
        for i in range(a // 2 + 1):
            for j in range(b // 2 + 1):
                for k in range(c // 2 + 1):
                    coef = herm(a, i) * herm(b, j) * herm(c, k) * cfac(a + b + c - i - j - k)
                    m = (a - 2 * i, b - 2 * j, c - 2 * k)
                    terms.append((coef, m))
        expr = []
        for coef, m in terms:
            r = mono_ref("q", m)
            expr.append(lit(coef) if r is None else f"{lit(coef)} * {r}")
        L.append(f"    D[{IDX[n]}] = " + " + ".join(expr) + ";")
    L.append("}")
    return L


def gen_p2m():
    L = ["/* moments about the centre: M[slot(n)] += m y^n, orders 0, 2, 3, 4 */",
         "__device__ __forceinline__ void fmm_p2m_acc(float m, float yx, float yy, float yz, float* __restrict__ M)",
         "{"]
    L += emit_monomials("y", ORDER_M)
    for n in MOM:
        r = mono_ref("y", n)
        L.append(f"    M[{MSLOT[n]}] += m" + ("" if r is None else f" * {r}") + ";")
    L.append("}")
    return L


def gen_m2m():
    """Shift child moments (about the child's centre) to the parent centre: y_p = y_c + t.
    M_n(p) += sum_{k<=n} C(n,k) t^(n-k) M_k(c); the child's dipole is zero."""
    L = ["/* child moments about its own centre -> parent centre, t = com_child - com_parent */",
         "__device__ __forceinline__ void fmm_m2m_acc(const float* __restrict__ Mc, float tx, float ty, float tz,",
         "                                            float* __restrict__ Mp)", "{"]
    L += emit_monomials("t", ORDER_M)
    for n in MOM:
        terms = []
        for k in MOM:
            if all(k[q] <= n[q] for q in range(3)):
                binom = math.comb(n[0], k[0]) * math.comb(n[1], k[1]) * math.comb(n[2], k[2])
                r = mono_ref("t", sub(n, k))
                t = f"Mc[{MSLOT[k]}]"
                if r is not None:
                    t = f"{r} * {t}"
                if binom != 1:
                    t = f"{lit(binom)} * {t}"
                terms.append(t)
        L.append(f"    Mp[{MSLOT[n]}] += " + " + ".join(terms) + ";")
    L.append("}")
    return L


def gen_traces():
    L = ["/* traces of the moment tensors for the particle-cell kernel */",
         "__device__ __forceinline__ void fmm_moment_traces(float* __restrict__ R)", "{"]
    L.append(f"    R[{TR2}] = " + " + ".join(f"R[{MSLOT[add(E[a], E[a])]}]" for a in range(3)) + ";")
    for i in range(3):
        L.append(f"    R[{TR3[i]}] = " + " + ".join(f"R[{MSLOT[add(E[i], add(E[a], E[a]))]}]" for a in range(3)) + ";")
    for m, s in TR4.items():
        L.append(f"    R[{s}] = " + " + ".join(f"R[{MSLOT[add(m, add(E[a], E[a]))]}]" for a in range(3)) + ";")
    L.append(f"    R[{TT4}] = " + " + ".join(f"R[{TR4[add(E[a], E[a])]}]" for a in range(3)) + ";")
    L.append(f"    R[{NREC - 1}] = 0.0f;")
    L.append("}")
    return L


def gen_norms():
    """Frobenius norms of the symmetric moment tensors of orders 2 and 4: sum over tensor
    components = sum over multi-indices of (|n|! / n!) M_n^2."""
    L = ["/* squared Frobenius norms of the order-2 and order-4 moment tensors of a record, each",
         "   component scaled (by s2, s4) before it is squared so that small cells do not underflow */",
         "__device__ __forceinline__ void fmm_moment_norms2(const float* __restrict__ R, float s2, float s4, float& n2,",
         "                                                  float& n4)", "{"]
    for o, var, sv in ((2, "n2", "s2"), (4, "n4", "s4")):
        terms = []
        for n in MOM:
            if sum(n) != o:
                continue
            w = math.factorial(o) // nfact(n)
            L.append(f"    const float t{MSLOT[n]} = R[{MSLOT[n]}] * {sv};")
            t = f"t{MSLOT[n]} * t{MSLOT[n]}"
            terms.append(t if w == 1 else f"{lit(w)} * {t}")
        L.append(f"    {var} = " + " + ".join(terms) + ";")
    L.append("}")
    return L


def gen_m2l():
    """L_k += R^-(|k|+1) sum_{|n|+|k|<=5} (-1)^|n|/n! (M_n R^-|n|) Dhat^(n+k)(q), r = c_sink - z_source."""
    L = ["/* multipole (moment record M about z) -> local coefficients about c; r = c - z */",
         "__device__ __forceinline__ void fmm_m2l_acc(const float* __restrict__ M, float rx, float ry, float rz,",
         "                                            float eps2, float* __restrict__ Lc)", "{",
         "    const float ir = fmm_rsqrt(fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, eps2))));",
         "    float D[56];",
         "    fmm_green_scaled(rx * ir, ry * ir, rz * ir, D);",
         "    const float ir2 = ir * ir, ir3 = ir2 * ir, ir4 = ir2 * ir2;"]
    sc = {0: None, 2: "ir2", 3: "ir3", 4: "ir4"}
    for n in MOM:
        s = Fraction((-1) ** sum(n), nfact(n))
        e = f"M[{MSLOT[n]}]"
        if sc[sum(n)]:
            e = f"{e} * {sc[sum(n)]}"
        L.append(f"    const float w{n[0]}{n[1]}{n[2]} = {lit(s)} * {e};")
    L.append("    float p = ir;")
    for o in range(ORDER_L + 1):
        for k in MI:
            if sum(k) != o:
                continue
            terms = []
            for n in MOM:
                if sum(n) + o > ORDER_L:
                    continue
                terms.append(f"w{n[0]}{n[1]}{n[2]} * D[{IDX[add(n, k)]}]")
            L.append(f"    Lc[{IDX[k]}] += p * (" + " + ".join(terms) + ");")
        if o < ORDER_L:
            L.append("    p *= ir;")
    L.append("}")
    return L


def gen_p2l():
    L = ["/* particle of mass m at z -> local coefficients about c; r = c - z */",
         "__device__ __forceinline__ void fmm_p2l_acc(float m, float rx, float ry, float rz, float eps2,",
         "                                            float* __restrict__ Lc)", "{",
         "    const float ir = fmm_rsqrt(fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, eps2))));",
         "    float D[56];",
         "    fmm_green_scaled(rx * ir, ry * ir, rz * ir, D);",
         "    float p = m * ir;"]
    for o in range(ORDER_L + 1):
        for k in MI:
            if sum(k) == o:
                L.append(f"    Lc[{IDX[k]}] = fmaf(p, D[{IDX[k]}], Lc[{IDX[k]}]);")
        if o < ORDER_L:
            L.append("    p *= ir;")
    L.append("}")
    return L


def gen_l2l():
    """L'_k = sum_{|j|<=5-|k|} t^j/j! L_(k+j), t = c_child - c_parent."""
    L = ["/* re-expand local coefficients about c at c + t */",
         "__device__ __forceinline__ void fmm_l2l(const float* __restrict__ Lp, float tx, float ty, float tz,",
         "                                        float* __restrict__ Lo)", "{"]
    L += emit_monomials("t", ORDER_L)
    for k in MI:
        terms = []
        for j in MI:
            if sum(j) + sum(k) > ORDER_L:
                continue
            f = Fraction(1, nfact(j))
            r = mono_ref("t", j)
            t = f"Lp[{IDX[add(k, j)]}]"
            if r is not None:
                t = f"{r} * {t}"
            if f != 1:
                t = f"{lit(f)} * {t}"
            terms.append(t)
        L.append(f"    Lo[{IDX[k]}] = " + " + ".join(terms) + ";")
    L.append("}")
    return L


def gen_l2p():
    L = ["/* local coefficients about c, evaluated at c + u: acceleration += grad Phi, phi -= Phi */",
         "__device__ __forceinline__ void fmm_l2p_acc(const float* __restrict__ Lc, float ux, float uy, float uz,",
         "                                            float& ax, float& ay, float& az, float& phi)", "{"]
    L += emit_monomials("u", ORDER_L)
    pot, acc = [], [[], [], []]
    for k in MI:
        f = Fraction(1, nfact(k))
        r = mono_ref("u", k)
        def term(idx):
            t = f"Lc[{idx}]"
            if r is not None:
                t = f"{r} * {t}"
            if f != 1:
                t = f"{lit(f)} * {t}"
            return t
        pot.append(term(IDX[k]))
        if sum(k) < ORDER_L:
            for q in range(3):
                acc[q].append(term(IDX[add(k, E[q])]))
    for q, c in enumerate("xyz"):
        L.append(f"    a{c} += " + " + ".join(acc[q]) + ";")
    L.append("    phi -= " + " + ".join(pot) + ";")
    L.append("}")
    return L


def gen_pc():
    """Field of one moment record at r = x - z (trace form, see module docstring of interact.cu).

    With q = r/R, ir = 1/R and contractions of the raw moment tensors with q:
      Phi = ir [M + ir^2 p2 + ir^3 p3 + ir^4 p4]
      a   = ir^2 [(-M + ir^2 s2 + ir^3 s3 + ir^4 s4) q + ir^2 v2 + ir^3 v3 + ir^4 v4]
    p2 = 3/2 C0 - 1/2 t2          s2 = -15/2 C0 + 3/2 t2          v2 = 3 C1
    p3 = 5/2 B0 - 3/2 u0          s3 = -35/2 B0 + 15/2 u0         v3 = 15/2 B1 - 3/2 trM3
    p4 = 35/8 A0 - 15/4 T0 + 3/8 tt4
                                  s4 = -315/8 A0 + 105/4 T0 - 15/8 tt4
                                  v4 = 35/2 A1 - 15/2 T1
    C1 = M2.q, C0 = M2:qq, t2 = tr M2; B1 = M3:qq, B0 = M3:qqq, u0 = trM3.q;
    A1 = M4:qqq, A0 = M4:qqqq, T1 = trM4.q, T0 = trM4:qq, tt4 = tr tr M4.
    """
    L = ["/* particle-cell: acceleration and potential at r = x - z of the record R (44 floats, smem) */",
         "__device__ __forceinline__ void fmm_pc_acc(const float* __restrict__ R, float rx, float ry, float rz,",
         "                                           float eps2, float& ax, float& ay, float& az, float& phi)", "{",
         "    const float ir = fmm_rsqrt(fmaf(rx, rx, fmaf(ry, ry, fmaf(rz, rz, eps2))));",
         "    const float qx = rx * ir, qy = ry * ir, qz = rz * ir;",
         "    const float ir2 = ir * ir;"]
    q = ["qx", "qy", "qz"]

    def contract(src, rank, name, load):
        """(T.q)[m] for |m| = rank-1, T given by load(n) for |n| = rank."""
        lines = []
        out = {}
        for m in mindices(rank - 1):
            if sum(m) != rank - 1:
                continue
            terms = [f"{load(add(m, E[a]))} * {q[a]}" for a in range(3)]
            v = f"{name}{m[0]}{m[1]}{m[2]}"
            lines.append(f"    const float {v} = " + " + ".join(terms) + ";")
            out[m] = v
        return lines, out

    rec = lambda n: f"R[{MSLOT[n]}]"
    # M4 chain
    l, A3 = contract(None, 4, "A3_", rec); L += l
    l, A2 = contract(None, 3, "A2_", lambda n: A3[n]); L += l
    l, A1 = contract(None, 2, "A1_", lambda n: A2[n]); L += l
    l, A0 = contract(None, 1, "A0_", lambda n: A1[n]); L += l
    # M3 chain
    l, B2 = contract(None, 3, "B2_", rec); L += l
    l, B1 = contract(None, 2, "B1_", lambda n: B2[n]); L += l
    l, B0 = contract(None, 1, "B0_", lambda n: B1[n]); L += l
    # M2 chain
    l, C1 = contract(None, 2, "C1_", rec); L += l
    l, C0 = contract(None, 1, "C0_", lambda n: C1[n]); L += l
    # traces
    l, T1 = contract(None, 2, "T1_", lambda n: f"R[{TR4[n]}]"); L += l
    l, T0 = contract(None, 1, "T0_", lambda n: T1[n]); L += l
    l, U0 = contract(None, 1, "U0_", lambda n: f"R[{TR3[n.index(1)]}]"); L += l
    a0, b0, c0, t0, u0 = A0[(0, 0, 0)], B0[(0, 0, 0)], C0[(0, 0, 0)], T0[(0, 0, 0)], U0[(0, 0, 0)]
    t2, tt4, M = f"R[{TR2}]", f"R[{TT4}]", "R[0]"
    L += [
        f"    const float p2 = 1.5f * {c0} - 0.5f * {t2};",
        f"    const float p3 = 2.5f * {b0} - 1.5f * {u0};",
        f"    const float p4 = 4.375f * {a0} - 3.75f * {t0} + 0.375f * {tt4};",
        f"    const float s2 = -7.5f * {c0} + 1.5f * {t2};",
        f"    const float s3 = -17.5f * {b0} + 7.5f * {u0};",
        f"    const float s4 = -39.375f * {a0} + 26.25f * {t0} - 1.875f * {tt4};",
        f"    const float S = -{M} + ir2 * (s2 + ir * (s3 + ir * s4));",
        f"    phi -= ir * ({M} + ir2 * (p2 + ir * (p3 + ir * p4)));",
    ]
    for a, c in enumerate("xyz"):
        m = E[a]
        L.append(f"    const float v{c} = 3.0f * {C1[m]} + ir * ((7.5f * {B1[m]} - 1.5f * R[{TR3[a]}])"
                 f" + ir * (17.5f * {A1[m]} - 7.5f * {T1[m]}));")
        L.append(f"    a{c} = fmaf(ir2, fmaf(S, q{c}, ir2 * v{c}), a{c});")
    L.append("}")
    return L


def gen_pc2():
    """gen_pc for two sinks at once (FP32x2): the same field of one record at r0 and r1, as
    float2 lanes.  Record values and constants are shared by both sinks; each multiply-add of the
    scalar body becomes one __ffma2_rn, so a pair of sinks costs the FP32 instructions of one.
    The potential is summed with the opposite sign (phip += ..., phi = -phip), so no negation is
    issued per pair."""
    f2 = lambda x: f"make_float2({x}, {x})"
    L = ["/* particle-cell for two sinks (FP32x2 lanes): field of the record R at r0 and r1; phip sums -phi */",
         "__device__ __forceinline__ void fmm_pc_acc2(const float* __restrict__ R, float2 rx, float2 ry, float2 rz,",
         "                                            float2 eps2, float2& ax, float2& ay, float2& az, float2& phip)",
         "{",
         "    const float2 r2 = __ffma2_rn(rx, rx, __ffma2_rn(ry, ry, __ffma2_rn(rz, rz, eps2)));",
         "    const float2 ir = make_float2(fmm_rsqrt(r2.x), fmm_rsqrt(r2.y));",
         "    const float2 qx = __fmul2_rn(rx, ir), qy = __fmul2_rn(ry, ir), qz = __fmul2_rn(rz, ir);",
         "    const float2 ir2 = __fmul2_rn(ir, ir);"]
    q = ["qx", "qy", "qz"]

    def contract(rank, name, load, scalar):
        lines, out = [], {}
        for m in mindices(rank - 1):
            if sum(m) != rank - 1:
                continue
            ops = [load(add(m, E[a])) for a in range(3)]
            if scalar:
                ops = [f2(o) for o in ops]
            v = f"{name}{m[0]}{m[1]}{m[2]}"
            lines.append(f"    const float2 {v} = __ffma2_rn({ops[2]}, {q[2]}, __ffma2_rn({ops[1]}, {q[1]}, "
                         f"__fmul2_rn({ops[0]}, {q[0]})));")
            out[m] = v
        return lines, out

    rec = lambda n: f"R[{MSLOT[n]}]"
    l, A3 = contract(4, "A3_", rec, True); L += l
    l, A2 = contract(3, "A2_", lambda n: A3[n], False); L += l
    l, A1 = contract(2, "A1_", lambda n: A2[n], False); L += l
    l, A0 = contract(1, "A0_", lambda n: A1[n], False); L += l
    l, B2 = contract(3, "B2_", rec, True); L += l
    l, B1 = contract(2, "B1_", lambda n: B2[n], False); L += l
    l, B0 = contract(1, "B0_", lambda n: B1[n], False); L += l
    l, C1 = contract(2, "C1_", rec, True); L += l
    l, C0 = contract(1, "C0_", lambda n: C1[n], False); L += l
    l, T1 = contract(2, "T1_", lambda n: f"R[{TR4[n]}]", True); L += l
    l, T0 = contract(1, "T0_", lambda n: T1[n], False); L += l
    l, U0 = contract(1, "U0_", lambda n: f"R[{TR3[n.index(1)]}]", True); L += l
    a0, b0, c0, t0, u0 = A0[(0, 0, 0)], B0[(0, 0, 0)], C0[(0, 0, 0)], T0[(0, 0, 0)], U0[(0, 0, 0)]
    t2, tt4, M = f"R[{TR2}]", f"R[{TT4}]", "R[0]"
    L += [
        f"    const float2 p2 = __ffma2_rn({f2('1.5f')}, {c0}, {f2(f'-0.5f * {t2}')});",
        f"    const float2 p3 = __ffma2_rn({f2('2.5f')}, {b0}, __fmul2_rn({f2('-1.5f')}, {u0}));",
        f"    const float2 p4 = __ffma2_rn({f2('4.375f')}, {a0}, __ffma2_rn({f2('-3.75f')}, {t0}, {f2(f'0.375f * {tt4}')}));",
        f"    const float2 s2 = __ffma2_rn({f2('-7.5f')}, {c0}, {f2(f'1.5f * {t2}')});",
        f"    const float2 s3 = __ffma2_rn({f2('-17.5f')}, {b0}, __fmul2_rn({f2('7.5f')}, {u0}));",
        f"    const float2 s4 = __ffma2_rn({f2('-39.375f')}, {a0}, __ffma2_rn({f2('26.25f')}, {t0}, {f2(f'-1.875f * {tt4}')}));",
        f"    const float2 S = __ffma2_rn(ir2, __ffma2_rn(ir, __ffma2_rn(ir, s4, s3), s2), {f2(f'-{M}')});",
        f"    phip = __ffma2_rn(ir, __ffma2_rn(ir2, __ffma2_rn(ir, __ffma2_rn(ir, p4, p3), p2), {f2(M)}), phip);",
    ]
    for a, c in enumerate("xyz"):
        m = E[a]
        L.append(f"    const float2 w{c} = __ffma2_rn({f2('17.5f')}, {A1[m]}, __fmul2_rn({f2('-7.5f')}, {T1[m]}));")
        L.append(f"    const float2 v{c} = __ffma2_rn({f2('3.0f')}, {C1[m]}, __fmul2_rn(ir, __ffma2_rn(ir, w{c}, "
                 f"__ffma2_rn({f2('7.5f')}, {B1[m]}, {f2(f'-1.5f * R[{TR3[a]}]')}))));")
        L.append(f"    a{c} = __ffma2_rn(ir2, __ffma2_rn(S, q{c}, __fmul2_rn(ir2, v{c})), a{c});")
    L.append("}")
    return L


def count_flops(lines):
    """FP32 flops of generated straight-line code: each binary '*', '+', '-' is 1 flop, fmaf is 2,
    an update 'x += e' / 'x -= e' adds 1; fmm_rsqrt is not counted (special-function unit)."""
    n = 0
    for ln in lines:
        st = ln.strip()
        if "=" not in st or st.startswith("/*") or st.startswith("float D[") or st.startswith("static"):
            continue
        lhs, rhs = st.split("=", 1)
        n += rhs.count("*") + rhs.count(" + ") + rhs.count(" - ") + 2 * rhs.count("fmaf(")
        if lhs.endswith("+") or lhs.endswith("-"):
            n += 1
        if "= -" in st:
            n += 1
    return n


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    parts = {
        "green": gen_green_scaled(), "p2m": gen_p2m(), "m2m": gen_m2m(), "traces": gen_traces(),
        "norms": gen_norms(),
        "m2l": gen_m2l(), "p2l": gen_p2l(), "l2l": gen_l2l(), "l2p": gen_l2p(), "pc": gen_pc(), "pc2": gen_pc2(),
    }
    out = ["// GENERATED by gen_expansions.py -- do not edit by hand.",
           "// Straight-line FP32 expansion operators for the Plummer-softened Green's function,",
           "// multipoles of order 4 about the centre of mass and local expansions of order 5 (Sec. 3.1).",
           "#pragma once", "",
           f"#define FMM_NL {NL}      /* local coefficients, |k| <= 5 */",
           f"#define FMM_NMOM {NMOM}    /* moment slots: M, M2, M3, M4 */",
           f"#define FMM_NREC {NREC}    /* moment record incl. traces */", "",
           "/* 1/sqrt(x) for x >= eps^2 > 0, which is never subnormal: the approximate reciprocal square",
           "   root instruction in its subnormal-flushing form, which needs no scaling of subnormal inputs",
           "   around the special-function unit (PTX ISA, rsqrt.approx.ftz.f32) */",
           "__device__ __forceinline__ float fmm_rsqrt(float x)",
           "{",
           "#ifdef __CUDA_ARCH__",
           "    float y;",
           '    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));',
           "    return y;",
           "#else  /* host builds of these operators (tests): 1 / sqrt(x) in single precision */",
           "    return 1.0f / sqrtf(x);",
           "#endif",
           "}", "",
           "/* multi-index table (a, b, c) of the local coefficients, in storage order */",
           "static const int fmm_multi_index_table[FMM_NL * 3] = {"]
    out.append("    " + ", ".join(f"{a}, {b}, {c}" for a, b, c in MI))
    out.append("};")
    out.append("/* moment slot -> multi-index */")
    out.append("static const int fmm_moment_index_table[FMM_NMOM * 3] = {")
    out.append("    " + ", ".join(f"{a}, {b}, {c}" for a, b, c in MOM))
    out.append("};")
    out.append("")
    for k, v in parts.items():
        out += v
        out.append("")
    flops = {k: count_flops(v) for k, v in parts.items() if k != "pc2"}  # pc2: the pc arithmetic, paired
    out.append("/* FP32 flops of the generated bodies (fmaf = 2): " +
               ", ".join(f"{k} {v}" for k, v in flops.items()) + " */")
    out.append(f"#define FMM_FLOPS_PC {flops['pc']}")
    with open(os.path.join(here, "expansions.cuh"), "w") as f:
        f.write("\n".join(out) + "\n")
    print(flops)


if __name__ == "__main__":
    main()
