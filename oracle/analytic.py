"""Closed-form circular Couette profiles (oracle pins; test infrastructure only).

* Rigid rotation (Sec. VI.C.3): f = f_eq(n(R), u^phi = Omega R, T_w) solves the
  kinetic equation for every tau, with n(R) from Eq. (rigid_density) and
  N_tot = pi (R_out^2 - R_in^2).
* Navier-Stokes regime (Sec. VI.D.1): u^phi (Eq. NS_U), T^{R phi}
  (Eq. NS_TRph), T (Eq. NS_T), q^R (Eq. NS_QR), Q (Eq. NS_Q) and the position
  of the temperature maximum (Eq. NS_Rmax), for constant mu and kappa with
  mu / kappa = 2/5 (Eq. CE_tcoeff with m = 1).
"""
from __future__ import annotations

import math

import numpy as np


def rigid_density(R, omega, T_w, r_in, r_out):
    c = omega ** 2 / (4.0 * T_w)
    n_tot = math.pi * (r_out ** 2 - r_in ** 2)
    return n_tot * c / math.pi * np.exp(c * (2.0 * np.asarray(R) ** 2 - r_in ** 2 - r_out ** 2)) / math.sinh(c * (r_out ** 2 - r_in ** 2))


def ns_u_phi(R, omega_in, r_in, r_out):
    R = np.asarray(R, dtype=np.float64)
    return omega_in / (r_in ** -2 - r_out ** -2) / R - R * omega_in * r_in ** 2 / (r_out ** 2 - r_in ** 2)


def ns_T_Rphi(R, mu, omega_in, r_in, r_out):
    t_in = 2.0 * mu * omega_in * r_out ** 2 / (r_out ** 2 - r_in ** 2)
    return t_in * r_in ** 2 / np.asarray(R, dtype=np.float64) ** 2


def ns_T(R, mu_over_kappa, omega_in, T_w, r_in, r_out):
    R = np.asarray(R, dtype=np.float64)
    d = r_in ** -2 - r_out ** -2
    return T_w + mu_over_kappa * omega_in ** 2 / d * ((r_in ** -2 - R ** -2) / d - np.log(R / r_in) / math.log(r_out / r_in))


def ns_qR(R, mu, omega_in, r_in, r_out):
    R = np.asarray(R, dtype=np.float64)
    d = r_in ** -2 - r_out ** -2
    return -mu / R * omega_in ** 2 / d * (2.0 * R ** -2 / d - 1.0 / math.log(r_out / r_in))


def ns_Q(mu, omega_in, r_in, r_out):
    d = r_in ** -2 - r_out ** -2
    return mu * omega_in ** 2 / d * (1.0 / math.log(r_out / r_in) - 2.0 * r_in ** 2 / (r_out ** 2 - r_in ** 2))


def ns_R_Tmax(r_in, r_out):
    return math.sqrt(2.0 * math.log(r_out / r_in) / (r_in ** -2 - r_out ** -2))
