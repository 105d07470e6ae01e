"""Pins of the oracle's S vector against Eq. (1).

The matrices M, L, A of Eq. (8) are not printed in the paper.  The oracle uses
coefficients derived by hand from Eq. (1) with Eqs. (2)-(7).  Here sympy
re-derives them from Eq. (1) itself (typed in ``derive.py``), and the textbook
spin-weighted spherical harmonics pin the discrete angular operator."""
import math
import random

import mpmath as mp
import numpy as np
import pytest
import sympy as sp

import derive


def _points():
    rnd = random.Random(1001)
    pts = []
    for s in [-2, -1, 0, 1, 2]:
        for m in [-2, 0, 1, 2, 3]:
            a = rnd.choice([0.0, rnd.uniform(0.05, 0.99)])
            rp = 1.0 + math.sqrt(1.0 - a * a)
            r = rp + 10 ** rnd.uniform(-2, 1.7)
            th = rnd.uniform(0.05, math.pi - 0.05)
            pts.append((s, m, a, r, th))
    return pts


@pytest.mark.parametrize("s,m,a,r,th", _points()[::3])
def test_coefficients_rederived_from_eq1(orc, s, m, a, r, th):
    c = derive.coefficients_at(1.0, a, s, m, r, th, prec=40)
    p = orc.params(s=s, m=m, a=a)
    rp = 1.0 + math.sqrt(1.0 - a * a)
    k = orc.coeffs(p, r - rp, th)
    ct = k["ct_re"] + 1j * k["ct_im"]
    pst = k["pst_re"] + 1j * k["pst_im"]
    q = k["q_re"] + 1j * k["q_im"]

    def close(x, y, tol=1e-11):
        assert abs(x - y) <= tol * max(1.0, abs(y)), (x, y)

    close(c["tt"], 1.0)
    close(c["t"], ct)
    close(c["xx"], -k["b"] ** 2)
    close(c["x"], -pst)
    close(c["hh"], -k["w"])
    close(c["h"], -k["w"] / math.tan(th))
    close(c["0"], -q + k["w"] * k["V"])
    for mixed in ("tx", "th", "xh"):
        assert abs(c[mixed]) < 1e-12


@pytest.mark.parametrize("a,r,th", [(0.9, 2.6, 0.7), (0.7, 9.0, 1.3), (0.99, 1.2, 2.9),
                                    (0.5, 40.0, 0.2)])
def test_first_order_split_terms(orc, a, r, th):
    """b b_{,r*} by a numeric derivative of b = (r^2+a^2)/Sigma (Eqs. 6-7) and
    P* = c_t b + p* - b b_{,r*}, the Phi_* coefficient of the Pi equation."""
    p = orc.params(a=a)
    rp = 1.0 + math.sqrt(1.0 - a * a)
    k = orc.coeffs(p, r - rp, th)

    def b_of(rr):
        D = rr * rr - 2 * rr + a * a
        return (rr * rr + a * a) / mp.sqrt((rr * rr + a * a) ** 2 - a * a * D * mp.sin(th) ** 2)

    with mp.workdps(40):
        D = r * r - 2 * r + a * a
        bbr = b_of(mp.mpf(r)) * mp.diff(b_of, mp.mpf(r)) * D / (r * r + a * a)
        assert k["bbr"] == pytest.approx(float(bbr), rel=1e-10, abs=1e-15)
        assert k["b"] == pytest.approx(float(b_of(mp.mpf(r))), rel=1e-14)
    ct = k["ct_re"] + 1j * k["ct_im"]
    pst = k["pst_re"] + 1j * k["pst_im"]
    Pst = k["Pst_re"] + 1j * k["Pst_im"]
    assert abs(Pst - (ct * k["b"] + pst - k["bbr"])) < 1e-14 * max(1, abs(Pst))


# spin-weighted spherical harmonics sY_lm(theta): Theta[S] = -(l - s)(l + s + 1) S.
# Near either pole sY_lm ~ theta^|m+s|, so the pole rule d_theta Phi = 0 / Phi = 0 by
# the parity of |m + s| (the paper's even/odd |m| for its even s) fits every s; the odd
# s entries fail with the rule by |m| alone.
_C = sp.cos(derive.th)
_S = sp.sin(derive.th)
HARMONICS = [
    (-2, 2, 2, (1 + _C) ** 2),
    (-2, 1, 2, _S * (1 + _C)),
    (-2, 2, 3, (1 + _C) ** 2 * (3 * _C - 2)),
    (0, 0, 2, (3 * _C ** 2 - 1) / 2),
    (0, 1, 2, _S * _C),
    (0, 2, 2, _S ** 2),
    (2, 2, 2, (1 - _C) ** 2),
    (2, 1, 2, _S * (1 - _C)),
    (1, 0, 1, _S),
    (1, 1, 1, 1 - _C),
    (-1, 1, 1, 1 + _C),
    (-1, 0, 2, _S * _C),
]


@pytest.mark.parametrize("s,m,l,expr", HARMONICS)
def test_theta_operator_on_spin_weighted_harmonics(orc, s, m, l, expr):
    # the harmonic really is an eigenfunction of Theta with eigenvalue -(l-s)(l+s+1)
    th = derive.th
    Vc = (m + s * sp.cos(th)) ** 2 / sp.sin(th) ** 2 - s
    res = sp.diff(sp.sin(th) * sp.diff(expr, th), th) / sp.sin(th) - Vc * expr
    lam = (l - s) * (l + s + 1)
    assert sp.simplify(res + lam * expr) == 0
    f = sp.lambdify(th, expr, "numpy")
    # The oracle's centred Theta_h (with its pole ghosts) converges to it at second
    # order at fixed theta.  Near a pole the truncation of the cot(theta) F_theta term is
    # cot(theta) dtheta^2 F'''/6, which for odd |m| (F ~ theta) grows like
    # dtheta^2/theta.  So the error times the distance to the pole is second order
    # uniformly, and the sin(theta)-weighted L2 error is second order up to a log.
    inner, pole, wl2 = [], [], []
    for n in (32, 64, 128):
        p = orc.params(s=s, m=m, a=0.0, n_theta=n)
        tj = (np.arange(n) + 0.5) * math.pi / n
        F = f(tj) * (1 + 0.5j)
        err = np.abs(orc.theta_apply(p, F) + lam * F)
        away = (tj > 0.5) & (tj < math.pi - 0.5)
        inner.append(err[away].max())
        pole.append((err * np.minimum(tj, math.pi - tj)).max())
        wl2.append(np.sqrt((err ** 2 * np.sin(tj)).sum() * math.pi / n))
    for e in (inner, pole):
        r1, r2 = e[0] / e[1], e[1] / e[2]
        assert 3.4 < r1 < 4.6 and 3.4 < r2 < 4.6, e
    assert wl2[0] / wl2[1] > 3.2 and wl2[1] / wl2[2] > 3.2, wl2
