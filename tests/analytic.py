"""Closed forms the paper prints, used to pin the oracle.

* heated microchannel with two superimposed layers (Sec. 4.1, Eqs. 47-59),
  written in the paper's coordinates: -h < y < 0 heavy layer, 0 < y < H light
  layer, walls at y = -h and y = H, period L in x;
* relative L2 error of Table 1's caption.
"""
import numpy as np


def microchannel_closed_form(x, y, L, H, h, T_h, T_c, T_0, lam_r, mu_r, sigma_T, mu_h, k=1):
    w = 2.0 * np.pi * k / L
    Ht, ht = H * w, h * w
    sh, ch = np.sinh, np.cosh
    f = 1.0 / (lam_r * sh(ht) * ch(Ht) + sh(Ht) * ch(ht))
    DH = sh(Ht) ** 2 - Ht ** 2
    Dh = sh(ht) ** 2 - ht ** 2
    C1H, C2H, C3H = sh(Ht) ** 2 / DH, -H * Ht / DH, (2 * Ht - sh(2 * Ht)) / (2 * DH)
    C1h, C2h, C3h = sh(ht) ** 2 / Dh, -h * ht / Dh, (sh(2 * ht) - 2 * ht) / (2 * Dh)
    g = sh(Ht) * f
    hfun = DH * Dh / (mu_r * Dh * (sh(2 * Ht) - 2 * Ht) + DH * (sh(2 * ht) - 2 * ht))
    Umax = -(T_0 * sigma_T / mu_h) * g * hfun

    den = H + lam_r * h
    TL = ((T_c - T_h) * y + lam_r * T_c * h + T_h * H) / den + T_0 * f * sh(Ht - w * y) * np.cos(w * x)
    TH = ((lam_r * (T_c - T_h) * y + lam_r * T_c * h + T_h * H) / den
          + T_0 * f * (sh(Ht) * ch(w * y) - lam_r * sh(w * y) * ch(Ht)) * np.cos(w * x))
    uxL = Umax * ((C1H + w * (C2H + C3H * y)) * ch(w * y) + (C3H + w * C1H * y) * sh(w * y)) * np.sin(w * x)
    uyL = -w * Umax * (C1H * y * ch(w * y) + (C2H + C3H * y) * sh(w * y)) * np.cos(w * x)
    uxH = Umax * ((C1h + w * (C2h + C3h * y)) * ch(w * y) + (C3h + w * C1h * y) * sh(w * y)) * np.sin(w * x)
    uyH = -w * Umax * (C1h * y * ch(w * y) + (C2h + C3h * y) * sh(w * y)) * np.cos(w * x)
    up = y >= 0
    return dict(T=np.where(up, TL, TH), ux=np.where(up, uxL, uxH), uy=np.where(up, uyL, uyH),
                Umax=Umax)


def rel_l2(num, ana):
    num = np.asarray(num, dtype=np.float64)
    ana = np.asarray(ana, dtype=np.float64)
    return float(np.sqrt(np.sum((num - ana) ** 2) / np.sum(ana ** 2)))
