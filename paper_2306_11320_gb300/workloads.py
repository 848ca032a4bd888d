"""Seeded synthetic workloads: physical parameters and initial fields.

This module holds no lattice Boltzmann arithmetic.  It only builds the inputs
that both the CUDA path and the oracle consume: a parameter dictionary (lattice
units, dx = dt = 1, Sec. 4) and initial macroscopic fields (phi, ux, uy, p, T)
as float64 arrays of shape (ny, nx), row-major, y = 0 the bottom fluid row.

Geometry conventions shared by every workload:
  * halfway walls sit at y = -1/2 and y = ny - 1/2; a horizontal inlet at
    x = -1/2 and an outflow plane at x = nx - 1/2;
  * the heavy fluid has phi = +1, the light fluid phi = -1 (Sec. 2);
  * diffuse interfaces take the profile phi = tanh(d / (sqrt(2) W)) with d the
    signed distance (positive on the heavy side).  This is the profile that
    makes the chemical potential below Eq. 11 vanish and integrates the delta
    function of Eq. 10 to one; the printed 0.5 tanh(2d/W) of Eq. 3 belongs to
    a +-1/2 convention and is not used.

Parameter keys (all floats unless noted):
  rho_l rho_h mu_l mu_h lambda_l lambda_h cp_l cp_h   bulk properties (Eq. 45)
  W M_phi                                             interface width, mobility
  sigma_law (int: 0 linear Eq. 12, 1 parabolic Eq. 63) sigma_ref sigma_T sigma_TT T_ref
  Gx Gy                                               body-force density
  bc_x (int: 0 periodic, 1 inlet/outflow)  bc_y (int: 0 walls, 1 periodic)
  u_ave phi_in T_in                                   inlet data
  p_out                                               outflow pressure
  T_bot T_bot_amp T_bot_k T_bot_slope                 bottom wall T(x) = T_bot
                                                      + T_bot_amp cos(2 pi k x/nx) + slope x
  T_top T_top_slope                                   top wall T(x) = T_top + slope x
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_W = 4.0
DEFAULT_M_PHI = 0.1


def base_params(**kw) -> dict:
    p = dict(
        rho_l=1.0, rho_h=1.0, mu_l=0.1, mu_h=0.1, lambda_l=0.1, lambda_h=0.1,
        cp_l=1.0, cp_h=1.0, W=DEFAULT_W, M_phi=DEFAULT_M_PHI,
        sigma_law=0, sigma_ref=1e-3, sigma_T=0.0, sigma_TT=0.0, T_ref=0.0,
        Gx=0.0, Gy=0.0, bc_x=0, bc_y=0, u_ave=0.0, phi_in=1.0, T_in=0.0, p_out=0.0,
        T_bot=0.0, T_bot_amp=0.0, T_bot_k=1.0, T_bot_slope=0.0, T_top=0.0, T_top_slope=0.0,
    )
    p.update(kw)
    return p


def _profile(d, W):
    return np.tanh(d / (math.sqrt(2.0) * W))


def _grid(nx, ny):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    return x, y


# ---------------------------------------------------------------- microchannel

def microchannel(nx=128, ny=32, lam_r=0.5, W=DEFAULT_W, k=1, h_frac=0.5,
                 T_h=20.0, T_c=10.0, T_0=4.0, T_ref=10.0, sigma_ref=2.5e-2, sigma_T=-5e-4,
                 mu=0.2, lambda_h=0.2, M_phi=DEFAULT_M_PHI):
    """Heated microchannel with two superimposed layers (Sec. 4.1).

    Heavy layer of height h = h_frac * ny below a light layer of height H = ny - h;
    bottom wall T = T_h + T_0 cos(2 pi k x / nx), top wall T = T_c, periodic in x.
    Initial state: flat interface, fluid at rest, T linear between the wall means.
    """
    h = int(round(h_frac * ny))
    params = base_params(
        rho_l=1.0, rho_h=1.0, mu_l=mu, mu_h=mu, lambda_h=lambda_h, lambda_l=lam_r * lambda_h,
        cp_l=1.0, cp_h=1.0, W=W, M_phi=M_phi, sigma_law=0, sigma_ref=sigma_ref,
        sigma_T=sigma_T, T_ref=T_ref, bc_x=0, bc_y=0,
        T_bot=T_h, T_bot_amp=T_0, T_bot_k=float(k), T_top=T_c,
    )
    x, y = _grid(nx, ny)
    y_int = h - 0.5                      # interface between rows h-1 and h
    phi = _profile(y_int - y, W)         # heavy (+1) below
    T = T_h + (T_c - T_h) * (y + 0.5) / ny
    z = np.zeros_like(phi)
    fields = dict(phi=phi, ux=z.copy(), uy=z.copy(), p=z.copy(), T=T)
    meta = dict(name="microchannel", h=h, H=ny - h, L=nx, T_h=T_h, T_c=T_c, T_0=T_0,
                lam_r=lam_r, k=k)
    return params, fields, meta


# ----------------------------------------------------------------------- drop

def drop_migration(nx=256, ny=1024, R=32.0, Ma=0.1, Re=0.1, Ca=0.08, ratio=0.5,
                   gradT=0.1, T_c=16.0, mu_h=0.2, rho_h=1.0, lambda_h=None, W=DEFAULT_W,
                   M_phi=DEFAULT_M_PHI):
    """Thermocapillary drop migration in a channel with a vertical T gradient (Sec. 4.2).

    The drop (light, phi = -1) has viscosity, conductivity and heat-capacity ratios
    `ratio` to the matrix; density ratio 1.  The characteristic length is R and the
    velocity U = -sigma_T grad T R / mu_h (below Eq. 60); Re, Ma, Ca of Eq. 46 fix
    U, c_p,h, sigma_T and sigma_ref.  sigma(T_ref) = sigma_ref at the drop centre.
    lambda_h defaults to the larger of 0.2 and the value that makes the drop's heat
    capacitance rho c_p equal to one: the update of Eq. 28 weighs the old population
    by (1 - 1/(rho c_p)), which turns negative (and the scheme unstable) below one.
    """
    nu_h = mu_h / rho_h
    U = Re * nu_h / R
    sigma_T = -U * mu_h / (R * gradT)
    sigma_ref = U * mu_h / Ca
    if lambda_h is None:
        lambda_h = max(0.2, rho_h * R * U / (Ma * min(1.0, ratio)))
    cp_h = Ma * lambda_h / (rho_h * R * U)
    xc, yc = 0.5 * (nx - 1), 0.5 * (ny - 1)
    T_at_centre = T_c + gradT * (yc + 0.5)
    params = base_params(
        rho_l=rho_h, rho_h=rho_h, mu_l=ratio * mu_h, mu_h=mu_h,
        lambda_l=ratio * lambda_h, lambda_h=lambda_h, cp_l=ratio * cp_h, cp_h=cp_h,
        W=W, M_phi=M_phi, sigma_law=0, sigma_ref=sigma_ref, sigma_T=sigma_T,
        T_ref=T_at_centre, bc_x=0, bc_y=0, T_bot=T_c, T_top=T_c + gradT * ny,
    )
    x, y = _grid(nx, ny)
    r = np.hypot(x - xc, y - yc)
    phi = _profile(r - R, W)
    T = T_c + gradT * (y + 0.5)
    z = np.zeros_like(phi)
    fields = dict(phi=phi, ux=z.copy(), uy=z.copy(), p=z.copy(), T=T)
    mu_r = ratio
    lam_r = ratio
    U_ygb = 2.0 * U / ((2.0 + 3.0 * mu_r) * (2.0 + lam_r))
    meta = dict(name="drop", R=R, U=U, U_ygb=U_ygb, xc=xc, yc=yc, Ma=Ma, Re=Re, Ca=Ca)
    return params, fields, meta


def drop_density_ratio(rho_r, nx=160, ny=320, R=20.0, W=DEFAULT_W, M_phi=DEFAULT_M_PHI, T_c=16.0):
    """The high-density-ratio drop of Table 2 (Sec. 4.2), on the paper's 160 x 320 lattice
    (periodic in x, walls in y) with R = 20.

    Printed: sigma_ref = 2.5e-4, sigma_T = -1e-5, mu = 0.8, (rho c_p)_h = 5,
    (rho c_p)_l = 1, Re = 0.00625, Ma = 0.0125, Ca = 0.08.  The printed U_YGB column
    follows with U = 2.5e-5, lambda_r = 0.5 and mu_r = 1 / rho_r (the paper's "mu_l =
    mu_h" does not reproduce it); U = -sigma_T grad T R / mu_h then needs grad T = 0.1,
    Re = rho_h U R / mu_h needs rho_h = 10, so the drop has rho_l = 10 / rho_r and the
    same kinematic viscosity, and Ma = U R (rho c_p)_h / lambda_h gives lambda_h = 0.2.
    """
    mu_h, rho_h, sigma_T, sigma_ref, gradT = 0.8, 10.0, -1e-5, 2.5e-4, 0.1
    U = -sigma_T * gradT * R / mu_h
    lambda_h = U * R * 5.0 / 0.0125
    xc, yc = 0.5 * (nx - 1), 0.5 * (ny - 1)
    params = base_params(
        rho_l=rho_h / rho_r, rho_h=rho_h, mu_l=mu_h / rho_r, mu_h=mu_h,
        lambda_l=0.5 * lambda_h, lambda_h=lambda_h, cp_l=rho_r / rho_h, cp_h=5.0 / rho_h,
        W=W, M_phi=M_phi, sigma_law=0, sigma_ref=sigma_ref, sigma_T=sigma_T,
        T_ref=T_c + gradT * (yc + 0.5), bc_x=0, bc_y=0, T_bot=T_c, T_top=T_c + gradT * ny,
    )
    x, y = _grid(nx, ny)
    phi = _profile(np.hypot(x - xc, y - yc) - R, W)
    z = np.zeros_like(phi)
    fields = dict(phi=phi, ux=z.copy(), uy=z.copy(), p=z.copy(), T=T_c + gradT * (y + 0.5))
    U_ygb = young_speed(U, 1.0 / rho_r, 0.5)
    return params, fields, dict(name="drop_rho", R=R, U=U, U_ygb=U_ygb, rho_r=rho_r)


def young_speed(U, mu_r, lam_r):
    """Young-Goldstein-Block terminal speed, Eq. 60."""
    return 2.0 * U / ((2.0 + 3.0 * mu_r) * (2.0 + lam_r))


# --------------------------------------------------------------------- bubbles

def bubbles(nx=2048, ny=512, R1=40.0, R2=32.0, spacing=150.0, lead_x_frac=460.0 / 500.0,
            u_ave=2.5e-4, T_c=0.0, T_h=1.0, T_ref=0.5, sigma_ref=5e-3, sigma_TT=2e-2,
            nu_h=0.04, nu_l=0.2, rho_h=1.0, rho_l=0.1, cp=20.0, lambda_h=7.0, lambda_l=0.7,
            W=DEFAULT_W, M_phi=DEFAULT_M_PHI):
    """Two recalcitrant bubbles in a Poiseuille channel flow, parabolic sigma(T) (Sec. 4.3).

    Inlet at x = -1/2 with u_x(y) = 6 u_ave y (H - y) / H^2 (Eq. 62 along the channel),
    held at T_c; outflow at x = nx - 1/2; walls heated linearly in x from T_c to T_h.
    Bubbles (light, phi = -1) of radius R1 (leading) and R2 (trailing), centres on the
    mid-line, the leading one at lead_x_frac * nx, the trailing one `spacing` upstream.
    """
    slope = (T_h - T_c) / nx
    params = base_params(
        rho_l=rho_l, rho_h=rho_h, mu_l=nu_l * rho_l, mu_h=nu_h * rho_h,
        lambda_l=lambda_l, lambda_h=lambda_h, cp_l=cp, cp_h=cp, W=W, M_phi=M_phi,
        sigma_law=1, sigma_ref=sigma_ref, sigma_TT=sigma_TT, T_ref=T_ref,
        bc_x=1, bc_y=0, u_ave=u_ave, phi_in=1.0, T_in=T_c,
        T_bot=T_c + 0.5 * slope, T_bot_slope=slope, T_top=T_c + 0.5 * slope, T_top_slope=slope,
    )
    x, y = _grid(nx, ny)
    x1 = round(lead_x_frac * nx)
    x2 = x1 - spacing
    yc = 0.5 * (ny - 1)
    d1 = np.hypot(x - x1, y - yc) - R1
    d2 = np.hypot(x - x2, y - yc) - R2
    phi = _profile(np.minimum(d1, d2), W)
    z = np.zeros_like(phi)
    fields = dict(phi=phi, ux=z.copy(), uy=z.copy(), p=z.copy(), T=np.full_like(phi, T_c))
    meta = dict(name="bubbles", x1=x1, x2=x2, yc=yc, R1=R1, R2=R2)
    return params, fields, meta


# ---------------------------------------------------------------- small cases

def static_drop(n=80, R=16.0, sigma=1e-3, W=DEFAULT_W, mu=0.1, rho_l=1.0, rho_h=1.0):
    """Static drop in a fully periodic box (Laplace-law check)."""
    params = base_params(rho_l=rho_l, rho_h=rho_h, mu_l=mu, mu_h=mu, W=W,
                         sigma_law=0, sigma_ref=sigma, sigma_T=0.0, bc_x=0, bc_y=1)
    x, y = _grid(n, n)
    c = 0.5 * (n - 1)
    phi = _profile(np.hypot(x - c, y - c) - R, W)
    z = np.zeros_like(phi)
    return params, dict(phi=phi, ux=z.copy(), uy=z.copy(), p=z.copy(), T=z.copy()), dict(R=R)


def random_state(nx, ny, seed=0, bc_x=0, bc_y=0, sigma_law=0, amp_u=1e-2, contrast=True):
    """A drop plus smooth random perturbations, used for step-by-step parity.

    Properties differ between phases (when `contrast`) so that every closure,
    ratio and heat-capacitance path is exercised.
    """
    rng = np.random.default_rng(seed)
    x, y = _grid(nx, ny)
    R = 0.3 * min(nx, ny)
    xc, yc = 0.45 * nx, 0.55 * ny
    phi = _profile(np.hypot(x - xc, y - yc) - R, 2.0) + 0.05 * rng.standard_normal((ny, nx))

    def smooth(a):
        return (a + np.roll(a, 1, 0) + np.roll(a, -1, 0) + np.roll(a, 1, 1) + np.roll(a, -1, 1)) / 5

    ux = amp_u * smooth(rng.standard_normal((ny, nx)))
    uy = amp_u * smooth(rng.standard_normal((ny, nx)))
    p = 1e-3 * smooth(rng.standard_normal((ny, nx)))
    T = 1.0 + 0.3 * smooth(rng.standard_normal((ny, nx))) + 0.01 * x
    if contrast:
        params = base_params(rho_l=0.5, rho_h=1.0, mu_l=0.05, mu_h=0.12, lambda_l=0.08,
                             lambda_h=0.3, cp_l=3.0, cp_h=1.0, W=2.0)
    else:
        params = base_params(W=2.0)
    params.update(sigma_law=sigma_law, sigma_ref=5e-3, sigma_T=-1e-3, sigma_TT=4e-2, T_ref=1.0,
                  bc_x=bc_x, bc_y=bc_y, Gx=1e-6, Gy=-2e-6, u_ave=1e-2, phi_in=1.0, T_in=0.8,
                  T_bot=1.3, T_bot_amp=0.2, T_bot_k=1.0, T_bot_slope=0.002, T_top=0.7,
                  T_top_slope=-0.001)
    return params, dict(phi=phi, ux=ux, uy=uy, p=p, T=T), dict(seed=seed)


def fp16_scales(params):
    """Power-of-two scales of the float16 population storage: the stored deviations
    from the nodes' rest equilibria (of order 1e-3 for f and g, 1e-2 for h on these
    workloads) land well inside float16's normal range."""
    return dict(fp16_scale_f=1024.0, fp16_scale_g=1024.0, fp16_scale_h=64.0)


def ensemble(n=256, seed=0, nx_range=(64, 512), ny_range=(64, 256), round_to=8):
    """Parameter-sweep ensemble of uneven microchannel and drop instances.

    Sizes are log-uniform and rounded to `round_to`; Ma in [0.01, 50], viscosity
    and conductivity ratios in [0.1, 10], all log-uniform; types alternate.
    Returns a list of (params, fields, meta).
    """
    rng = np.random.default_rng(seed)

    def logu(lo, hi):
        return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))

    out = []
    for k in range(n):
        nx = int(round(logu(*nx_range) / round_to) * round_to)
        ny = int(round(logu(*ny_range) / round_to) * round_to)
        Ma = logu(0.01, 50.0)
        mu_r = logu(0.1, 10.0)
        lam_r = logu(0.1, 10.0)
        if k % 2 == 0:
            p, f, m = microchannel(nx=nx, ny=ny, lam_r=lam_r)
            p["mu_l"] = mu_r * p["mu_h"]
            # Ma = rho_h c_p,h L U / lambda_h with L = nx and U from the wall forcing;
            # rho c_p >= 1 (see drop_migration), lambda raised to keep Ma where needed
            U = abs(p["sigma_T"]) * 4.0 / nx * (ny // 2) / p["mu_h"]
            cp = max(1.0, Ma * p["lambda_h"] / (nx * U))
            p["cp_h"] = p["cp_l"] = cp
            p["lambda_h"] = cp * nx * U / Ma
            p["lambda_l"] = lam_r * p["lambda_h"]
        else:
            R = max(6.0, 0.2 * min(nx, ny))
            p, f, m = drop_migration(nx=nx, ny=ny, R=R, Ma=Ma, ratio=1.0, gradT=0.02)
            p["mu_l"] = mu_r * p["mu_h"]
            p["lambda_l"] = lam_r * p["lambda_h"]
        m.update(nx=nx, ny=ny, Ma=Ma, mu_r=mu_r, lam_r=lam_r)
        out.append((p, f, m))
    return out
