"""Generate the Taylor coefficients used by the overlap branch of the D
assembly kernel (ewald_build.cu).

For an image closer than 2a the kernel evaluates M1 + M* (Eq. M1 plus the
overlap correction, Eq. cor5) in the cancellation-free form
Omega_B(r) - G(r), where G = Omega_A - M1 is the smooth part of the Ewald
split (Beenakker's real-space function removed from the RPY branch A).  With
s = alpha r and x = r/a:

  G_delta(r)     = a alpha A1(s) + a^3 alpha^3 B1(s)
  G_rr(r) / r^2  = a alpha^3 A2(s)/s^2 + a^3 alpha^5 B2(s)/s^2

and sqrt(pi) A1, B1, A2/s^2, B2/s^2 are even power series in s with rational
coefficients.  This script derives them with sympy and prints C literals of
the first NT coefficients (the kernel uses them for s <= 1, where 22 terms
reach double precision).  Run: python gen_overlap_series.py
"""
import sympy as sp

NT = 22


def series_coeffs():
    s = sp.symbols("s", positive=True)
    E = sp.exp(-s ** 2)
    P = sp.sqrt(sp.pi)
    # brackets of G = Omega_A - M1, Eq. (b1) minus Eq. (M1), in units of
    # a alpha and a^3 alpha^3
    A1 = sp.erf(s) * 3 / (4 * s) - E * (3 * s ** 2 - sp.Rational(9, 2)) / P
    B1 = sp.erf(s) / (2 * s ** 3) - E * (4 * s ** 4 - 20 * s ** 2 + 14 + 1 / s ** 2) / P
    A2 = sp.erf(s) * 3 / (4 * s) - E * (sp.Rational(3, 2) - 3 * s ** 2) / P
    B2 = -3 * sp.erf(s) / (2 * s ** 3) - E * (-4 * s ** 4 + 16 * s ** 2 - 2 - 3 / s ** 2) / P
    out = {}
    for name, f in (("A1", A1), ("B1", B1), ("A2s", A2 / s ** 2), ("B2s", B2 / s ** 2)):
        ser = sp.series(f * P, s, 0, 2 * NT + 2).removeO()
        poly = sp.Poly(sp.expand(ser), s)
        out[name] = [sp.nsimplify(poly.coeff_monomial(s ** (2 * j))) for j in range(NT)]
    return out


if __name__ == "__main__":
    for name, cs in series_coeffs().items():
        print(f"// {name}")
        print(",\n".join(f"    {float(c)!r}" for c in cs))
