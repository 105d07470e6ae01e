"""Symbolic re-derivation of the (r*, theta) equation from Eq. (1) of the paper.

Test helper.  It shares nothing with the oracle or the CUDA path: it types in
Eq. (1) (the Teukolsky master equation in Boyer-Lindquist coordinates), the
coordinate changes of Eqs. (2)-(3) and the ansatz of Eq. (4), and lets sympy do
the chain rule.  What comes out is what the oracle's S vector must reproduce.
"""
from __future__ import annotations

import functools

import sympy as sp

t, r, th, ph = sp.symbols("t r theta phi", real=True)
M, a, s, m = sp.symbols("M a s m", real=True)
X = sp.Function("X")(r)      # r*(r), Eq. (2): dX/dr = (r^2 + a^2)/Delta
G = sp.Function("G")(r)      # phi~ - phi,  Eq. (3): dG/dr = a/Delta
Delta = r**2 - 2 * M * r + a**2


def eq1_lhs(Psi):
    """Left-hand side of Eq. (1) applied to Psi(t, r, theta, phi)."""
    sn, cs = sp.sin(th), sp.cos(th)
    return (-((r**2 + a**2)**2 / Delta - a**2 * sn**2) * sp.diff(Psi, t, 2)
            - 4 * M * a * r / Delta * sp.diff(Psi, t, ph)
            - 2 * s * (r - M * (r**2 - a**2) / Delta + sp.I * a * cs) * sp.diff(Psi, t)
            + Delta**(-s) * sp.diff(Delta**(s + 1) * sp.diff(Psi, r), r)
            + 1 / sn * sp.diff(sn * sp.diff(Psi, th), th)
            + (1 / sn**2 - a**2 / Delta) * sp.diff(Psi, ph, 2)
            + 2 * s * (a * (r - M) / Delta + sp.I * cs / sn**2) * sp.diff(Psi, ph)
            - (s**2 * sp.cot(th)**2 - s) * Psi)


def _coordinate_subs(expr):
    """Replace derivatives of X and G by Eqs. (2)-(3).  G itself only enters through
    the overall factor e^{i m G}, which divides out, so it is then set to 0."""
    dX = (r**2 + a**2) / Delta
    dG = a / Delta
    expr = expr.subs({sp.Derivative(X, (r, 2)): sp.diff(dX, r),
                      sp.Derivative(G, (r, 2)): sp.diff(dG, r)})
    expr = expr.subs({sp.Derivative(X, r): dX, sp.Derivative(G, r): dG})
    return expr.subs(G, 0)


# jet coefficients of Phi at the expansion point (t0, x0, th0)
J = dict(zip(["c0", "ct", "ctt", "cx", "cxx", "ch", "chh", "ctx", "cth", "cxh"],
             sp.symbols("c0 c_t c_tt c_x c_xx c_h c_hh c_tx c_th c_xh")))
t0, x0, th0 = sp.symbols("t0 x0 th0", real=True)


@functools.lru_cache(maxsize=None)
def transformed_operator():
    """Eq. (1) LHS of Psi = e^{i m (phi + G)} r^3 Phi(t, X(r), theta), for a quadratic
    jet Phi, divided by -Sigma^2 e^{i m phi~} r^3 / Delta, as an expression in the jet
    coefficients (to be evaluated at t = t0, X = x0, theta = th0)."""
    T, xi, et = t - t0, X - x0, th - th0
    Phi = (J["c0"] + J["ct"] * T + J["ctt"] * T**2 / 2 + J["cx"] * xi + J["cxx"] * xi**2 / 2
           + J["ch"] * et + J["chh"] * et**2 / 2 + J["ctx"] * T * xi + J["cth"] * T * et
           + J["cxh"] * xi * et)
    Psi = sp.exp(sp.I * m * (ph + G)) * r**3 * Phi
    L = _coordinate_subs(eq1_lhs(Psi))
    Sig2 = (r**2 + a**2)**2 - a**2 * Delta * sp.sin(th)**2
    return L / (-Sig2 * sp.exp(sp.I * m * ph) * r**3 / Delta)


_KEYS = [("tt", "ctt"), ("t", "ct"), ("xx", "cxx"), ("x", "cx"), ("hh", "chh"), ("h", "ch"),
         ("0", "c0"), ("tx", "ctx"), ("th", "cth"), ("xh", "cxh")]


@functools.lru_cache(maxsize=None)
def coefficient_exprs(Mv, av, sv, mv):
    """Coefficient of each Phi derivative in the transformed equation, as sympy
    expressions in (r, theta) for numeric M, a, s, m:

      Phi_tt ('tt'), Phi_t ('t'), Phi_** ('xx'), Phi_* ('x'), Phi_thth ('hh'),
      Phi_th ('h'), Phi ('0') and the mixed derivatives ('tx', 'th', 'xh').

    The oracle's form  Phi_tt + c_t Phi_t - b^2 Phi_** - p* Phi_* - w (Phi_thth +
    cot Phi_th - V Phi) - q Phi  must match them term by term."""
    expr = transformed_operator()
    expr = expr.subs(X, x0).subs({t: t0, th: th0})
    expr = expr.subs({M: sp.Float(Mv, 50), a: sp.Float(av, 50), s: sp.Integer(sv),
                      m: sp.Integer(mv), ph: 0})
    expr = sp.expand(expr)
    out = {}
    for key, c in _KEYS:
        out[key] = expr.coeff(J[c]).subs(th0, th)
    return out


def coefficients_at(Mv, av, sv, mv, rv, thv, prec=30):
    """Numeric values of coefficient_exprs at (r, theta), as Python complex."""
    ex = coefficient_exprs(Mv, av, sv, mv)
    return {k: complex(sp.N(e.subs({r: sp.Float(rv, 50), th: sp.Float(thv, 50)}), prec))
            for k, e in ex.items()}


def mpmath_coefficients(Mv, av, sv, mv):
    """Callables (r, theta) -> mpc for each key of coefficient_exprs (mpmath precision)."""
    ex = coefficient_exprs(Mv, av, sv, mv)
    return {k: sp.lambdify((r, th), e, "mpmath") for k, e in ex.items()}


def mms_source(Mv, av, sv, mv, omega0, rc, ell):
    """tau for the manufactured solution Phi = e^{-i omega0 t} e^{-(r*-rc)^2/ell^2} sin^4(theta),
    obtained by applying Eq. (1) to Psi = e^{i m phi~} r^3 Phi and converting the
    right-hand side -4 pi (r^2 + a^2 cos^2) T to tau = 4 pi Delta (r^2 + a^2 cos^2)
    T / (Sigma^2 r^3).  Returns numpy callables Q(r, rstar, theta) with
    tau = e^{-i omega0 t} Q, and Phi_m(t, rstar, theta), Pi_m(t, r, rstar, theta)."""
    rs = sp.Symbol("rs", real=True)
    Phi = sp.exp(-sp.I * omega0 * t) * sp.exp(-(X - rc)**2 / ell**2) * sp.sin(th)**4
    Psi = sp.exp(sp.I * m * (ph + G)) * r**3 * Phi
    L = _coordinate_subs(eq1_lhs(Psi))
    Sig2 = (r**2 + a**2)**2 - a**2 * Delta * sp.sin(th)**2
    tau = -Delta * L / (Sig2 * r**3 * sp.exp(sp.I * m * ph))
    tau = tau.subs({M: Mv, a: av, s: sv, m: mv, ph: 0})
    # tau = e^{-i omega0 t} Q: evaluate at t = 0 to get Q
    Q = tau.subs(X, rs).subs(t, 0)
    b = ((r**2 + a**2) / sp.sqrt(Sig2)).subs({M: Mv, a: av})
    Phi_rs = Phi.subs(X, rs)
    Pi = sp.diff(Phi_rs, t) + b * sp.diff(Phi_rs, rs)
    fQ = sp.lambdify((r, rs, th), Q, "numpy")
    fPhi = sp.lambdify((t, rs, th), Phi_rs, "numpy")
    fPi = sp.lambdify((t, r, rs, th), Pi, "numpy")
    return fQ, fPhi, fPi


def tortoise_closed_form(Mv, av, rv):
    """r*(r) of Eq. (2) with the constant fixed by r* = r + 2M ln(r/2M - 1) at a = 0."""
    import mpmath as mp
    rp = Mv + mp.sqrt(Mv * Mv - av * av)
    return tortoise_of_x(Mv, av, mp.mpf(rv) - rp)


def tortoise_of_x(Mv, av, xv):
    """The same r*, written for r = r_+ + x (x > 0 given exactly, so near the horizon the
    logarithm's argument carries no cancellation)."""
    import mpmath as mp
    rp = Mv + mp.sqrt(Mv * Mv - av * av)
    rm = Mv - mp.sqrt(Mv * Mv - av * av)
    k = 2 * Mv / (rp - rm)
    xv = mp.mpf(xv)
    return rp + xv + k * rp * mp.log(xv / (2 * Mv)) - k * rm * mp.log((xv + rp - rm) / (2 * Mv))
