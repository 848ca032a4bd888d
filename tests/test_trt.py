"""Pins of the two-relaxation-time (TRT) collision for the NS and thermal LBEs in the
FP64 oracle (CPU): it reduces to BGK when the magic parameter equals (tau - 1/2)^2,
its halfway bounce-back Poiseuille flow has the slip G (4 Lambda - 3/4) / (6 nu), which
vanishes at Lambda = 3/16, and its thermal diffusivity is set by tau- alone."""
import math

import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_2306_11320_gb300 import workloads as WL

CS2 = 1.0 / 3.0


def _run(p, f, nx, ny, steps):
    s = OracleSim(nx, ny, p)
    s.init(**f)
    s.step(steps)
    return s


def test_trt_with_matching_lambda_is_bgk():
    nx, ny = 24, 20
    p, f, _ = WL.random_state(nx, ny, seed=3, bc_x=0, bc_y=0, contrast=False)
    p.update(rho_l=1.0, rho_h=1.0, mu_l=0.1, mu_h=0.1, lambda_l=0.1, lambda_h=0.1, cp_l=1.0, cp_h=1.0)
    tau = 0.1 / CS2 + 0.5      # tau_g = tau_h = 0.8
    a = _run(p, f, nx, ny, 30).fields()
    b = _run(dict(p, collision=1, trt_lambda=(tau - 0.5) ** 2), f, nx, ny, 30).fields()
    for k in a:
        assert np.abs(a[k] - b[k]).max() <= 1e-12 * (1 + np.abs(a[k]).max()), k


@pytest.mark.parametrize("mu", [0.1, 0.5])
@pytest.mark.parametrize("lam", [3.0 / 16.0, 0.25, 1.0 / 12.0])
def test_trt_poiseuille_slip(mu, lam):
    nx, ny, G = 4, 24, 1e-6
    p = WL.base_params(mu_l=mu, mu_h=mu, Gx=G, sigma_ref=0.0, collision=1, trt_lambda=lam)
    z = np.zeros((ny, nx))
    s = _run(p, dict(phi=np.ones((ny, nx)), ux=z, uy=z, p=z, T=z), nx, ny, int(5 * ny * ny / mu))
    y = np.arange(ny) + 0.5
    ana = G / (2 * mu) * y * (ny - y) + G * (4 * lam - 0.75) / (6 * mu)
    assert np.abs(s.fields()["ux"][:, 0] - ana).max() / ana.max() < 1e-6


@pytest.mark.parametrize("lam", [0.25, 1.0 / 12.0])
def test_trt_thermal_diffusivity(lam):
    """Cosine mode at rest: T decays as exp(-lambda k^2 t / (rho c_p)) with the
    conductivity carried by tau- = lambda / cs2 + 1/2 whatever the magic parameter."""
    nx, ny, steps, kappa, rcp = 64, 4, 1500, 0.05, 1.0
    p = WL.base_params(lambda_l=kappa, lambda_h=kappa, bc_y=1, sigma_ref=0.0, collision=1, trt_lambda=lam)
    x = np.arange(nx)[None, :] + np.zeros((ny, 1))
    k = 2 * math.pi / nx
    fields = dict(phi=np.ones((ny, nx)), ux=np.zeros((ny, nx)), uy=np.zeros((ny, nx)),
                  p=np.zeros((ny, nx)), T=1.0 + 0.5 * np.cos(k * x))
    T = _run(p, fields, nx, ny, steps).fields()["T"][0] - 1.0
    z = (T * np.exp(-1j * k * np.arange(nx))).sum() * 2 / nx
    amp_exact = 0.5 * math.exp(-kappa / rcp * k * k * steps)
    assert abs(abs(z) - amp_exact) / amp_exact < 2e-3
