"""Pins of the oracle's staggered operators against the paper and mathematics.

- coefficients equal the values (and formulas) printed in eqs. (derivcoef),
  (interpcoef);
- polynomial exactness (derivative: degree <= 6, interpolation: degree <= 5),
  with degree 7 / 6 as negative controls;
- the closed-form Fourier symbols of the periodic operators;
- measured convergence order 6 on sinusoids;
- summation-by-parts transposes: sum up(f) g = sum f dn(g),
  sum ddup(f) g = -sum f dddn(g).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle.stagger as S

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def frac(s):
    return float(Fraction(s))


def test_coefficients_match_paper():
    d = GOLD["derivative"]
    assert S.DC == pytest.approx(frac(d["c"]), abs=0, rel=1e-15)
    assert S.DB == pytest.approx(frac(d["b"]), rel=1e-15)
    assert S.DA == pytest.approx(frac(d["a"]), rel=1e-15)
    c = eval(d["c_formula"])
    b = eval(d["b_formula"], {"c": c})
    a = eval(d["a_formula"], {"b": b, "c": c})
    assert (a, b, c) == pytest.approx((S.DA, S.DB, S.DC), rel=1e-14)
    i = GOLD["interpolation"]
    assert (S.IA, S.IB, S.IC) == pytest.approx((frac(i["a"]), frac(i["b"]), frac(i["c"])), rel=1e-15)
    assert eval(i["a_formula"], {"b": S.IB, "c": S.IC}) == pytest.approx(S.IA, rel=1e-15)


def test_rk_constants_match_paper():
    assert tuple(GOLD["rk3"]["alpha"]) == S.ALPHA
    assert tuple(GOLD["rk3"]["beta"]) == S.BETA


def _line(n, ax, values):
    shape = {"x": (1, 1, n), "y": (1, n, 1), "z": (n, 1, 1)}[ax]
    return torch.tensor(values, dtype=torch.float64).reshape(shape)


def _flat(t):
    return t.reshape(-1).numpy()


@pytest.mark.parametrize("ax", ["x", "y", "z"])
def test_polynomial_exactness(ax):
    n, h = 64, 0.37
    i = np.arange(n, dtype=np.float64)
    xc = i * h                      # sample positions of the input
    inner = slice(8, n - 8)         # away from the periodic wrap
    L = 16 * h                      # polynomial in t = (x - x0)/L, |t| <= 4
    x0 = 32 * h
    for deg in range(0, 8):
        f = _line(n, ax, ((xc - x0) / L) ** deg)
        up_exact = ((xc + 0.5 * h - x0) / L) ** deg
        dn_exact = ((xc - 0.5 * h - x0) / L) ** deg
        if deg:
            dd_up = deg / L * ((xc + 0.5 * h - x0) / L) ** (deg - 1)
            dd_dn = deg / L * ((xc - 0.5 * h - x0) / L) ** (deg - 1)
        else:
            dd_up = dd_dn = 0 * xc
        e_up = np.abs(_flat(S.up(f, ax)) - up_exact)[inner].max()
        e_dn = np.abs(_flat(S.dn(f, ax)) - dn_exact)[inner].max()
        e_du = np.abs(_flat(S.ddup(f, ax, h)) - dd_up)[inner].max()
        e_dd = np.abs(_flat(S.dddn(f, ax, h)) - dd_dn)[inner].max()
        if deg <= 5:
            assert e_up < 1e-11 and e_dn < 1e-11, (deg, e_up, e_dn)
        else:
            assert e_up > 1e-8, ("interpolation should not be exact for degree 6+", e_up)
        if deg <= 6:
            assert e_du < 1e-11 and e_dd < 1e-11, (deg, e_du, e_dd)
        else:
            assert e_du > 1e-8, ("derivative should not be exact for degree 7", e_du)


def D_symbol(th):
    return 2 * (S.DA * math.sin(th / 2) + S.DB * math.sin(3 * th / 2) + S.DC * math.sin(5 * th / 2))


def I_symbol(th):
    return 2 * (S.IA * math.cos(th / 2) + S.IB * math.cos(3 * th / 2) + S.IC * math.cos(5 * th / 2))


def test_symbol_closed_forms():
    # Values of the symbols fixed by the printed coefficients.
    assert D_symbol(math.pi) == pytest.approx(2 * (225 / 192 + 25 / 384 + 3 / 640), rel=1e-15)
    assert D_symbol(math.pi) == pytest.approx(2.48333, abs=5e-6)
    th = 2 * math.pi * 2 / 32
    assert D_symbol(th) / th == pytest.approx(0.9999975, abs=5e-8)
    assert I_symbol(th) == pytest.approx(0.9999825, abs=5e-8)
    # Low-order Taylor: D(th) = th + O(th^7), I(th) = 1 + O(th^6).
    t = 1e-2
    assert abs(D_symbol(t) - t) < 1e-14
    assert abs(I_symbol(t) - 1) < 1e-13


@pytest.mark.parametrize("ax", ["x", "y", "z"])
@pytest.mark.parametrize("m", [1, 3, 7])
def test_periodic_symbols(ax, m):
    n = 32
    h = 1.0 / n
    k = 2 * math.pi * m
    th = k * h
    x = np.arange(n) * h
    f = _line(n, ax, np.sin(k * x + 0.3))
    np.testing.assert_allclose(_flat(S.ddup(f, ax, h)), D_symbol(th) / h * np.cos(k * (x + h / 2) + 0.3), atol=1e-12 * n)
    np.testing.assert_allclose(_flat(S.dddn(f, ax, h)), D_symbol(th) / h * np.cos(k * (x - h / 2) + 0.3), atol=1e-12 * n)
    np.testing.assert_allclose(_flat(S.up(f, ax)), I_symbol(th) * np.sin(k * (x + h / 2) + 0.3), atol=1e-14)
    np.testing.assert_allclose(_flat(S.dn(f, ax)), I_symbol(th) * np.sin(k * (x - h / 2) + 0.3), atol=1e-14)


def test_convergence_order_six():
    errs_d, errs_i, hs = [], [], []
    for n in (16, 32, 64, 128):
        h = 1.0 / n
        x = np.arange(n) * h
        k = 2 * math.pi
        f = _line(n, "x", np.sin(k * x))
        errs_d.append(np.abs(_flat(S.ddup(f, "x", h)) - k * np.cos(k * (x + h / 2))).max())
        errs_i.append(np.abs(_flat(S.up(f, "x")) - np.sin(k * (x + h / 2))).max())
        hs.append(h)
    sd = np.polyfit(np.log(hs[:3]), np.log(errs_d[:3]), 1)[0]
    si = np.polyfit(np.log(hs[:3]), np.log(errs_i[:3]), 1)[0]
    assert 5.8 < sd < 6.2, sd
    assert 5.8 < si < 6.2, si


def test_summation_by_parts():
    g = torch.Generator().manual_seed(0)
    f = torch.randn(6, 7, 9, generator=g, dtype=torch.float64)
    q = torch.randn(6, 7, 9, generator=g, dtype=torch.float64)
    for ax in "xyz":
        assert float((S.up(f, ax) * q).sum()) == pytest.approx(float((f * S.dn(q, ax)).sum()), rel=1e-13)
        assert float((S.ddup(f, ax, 0.1) * q).sum()) == pytest.approx(float(-(f * S.dddn(q, ax, 0.1)).sum()), rel=1e-12)
        # dn is up shifted down by one cell.
        assert torch.equal(S.dn(f, ax), torch.roll(S.up(f, ax), 1, dims=S._AX[ax]))


def test_degenerate_axis_is_identity():
    f = torch.randn(1, 5, 6, dtype=torch.float64)
    assert torch.allclose(S.up(f, "z"), f, rtol=0, atol=1e-15)
    assert float(S.ddup(f, "z", 0.1).abs().max()) == 0.0
