"""Exact linear wave solutions on flat space in the 27 state fields (numpy): a transverse-traceless
gravitational plane wave and the longitudinal gauge modes of the (modified) puncture gauge. Test
infrastructure shared by the oracle pins and the GPU tests; no method arithmetic beyond the
closed forms."""
import math

import numpy as np

import grf_inputs as gi


def tt_wave_state(b, amp, k, t):
    """Flat space with the transverse-traceless wave h_yy = -h_zz = a, h_yz = 0.7 a', a =
    amp sin(k (x - t)) (outgoing along +x), unit lapse, zero shift, K_ij = -d_t gamma_ij / 2, in the
    conformal variables (chi = det(gamma)^(-1/3), A_ij = chi (K_ij - gamma_ij K / 3)); Gamma-hat, K and
    the lapse perturbation are second order in amp and set to their flat values."""
    s = gi.flat_state(b)
    X, _, _ = b.coords()
    ph = k * (X - t)
    a, ad = amp * np.sin(ph), -amp * k * np.cos(ph)            # a and d_t a
    c, cd = 0.7 * amp * np.cos(ph), 0.7 * amp * k * np.sin(ph)  # the cross polarisation and d_t
    gyy, gzz, gyz = 1 + a, 1 - a, c
    det = gyy * gzz - gyz * gyz
    chi = det ** (-1.0 / 3.0)
    Kyy, Kzz, Kyz = -0.5 * ad, 0.5 * ad, -0.5 * cd
    # K = gamma^ij K_ij over the yz block (the x row is trivial)
    Ktr = (gzz * Kyy + gyy * Kzz - 2 * gyz * Kyz) / det
    s[0] = chi
    s[4], s[5], s[6] = chi * gyy, chi * gyz, chi * gzz          # h22, h23, h33
    s[1] = chi
    s[7] = Ktr
    s[8] = chi * (0.0 - Ktr / 3.0)
    s[11], s[12], s[13] = chi * (Kyy - gyy * Ktr / 3), chi * (Kyz - gyz * Ktr / 3), chi * (Kzz - gzz * Ktr / 3)
    return s


def gauge_wave_state(b, eps, k, t, a=0.0):
    """The exact linear gauge wave of the modified puncture gauge with F = 0 on flat space, from
    d_t alpha = -2 alpha K / (1 + a), d_t beta^i = -(a / (1 + a)) alpha chi h^ij d_j alpha,
    d_t K_ij = -d_i d_j alpha and d_t gamma_ij = -2 alpha K_ij + d_i beta_j + d_j beta_i (a metric
    perturbation gamma_xx(x) alone is pure gauge, so the curvature stays flat):
      alpha = 1 + eps sin(k x) cos(w t),  w = k sqrt(2 / (1 + a)),
      K = K_xx = ((1 + a) / 2) eps w sin(k x) sin(w t),
      beta^x = -(a / (1 + a)) eps (k / w) cos(k x) sin(w t),
      gamma_xx = 1 - eps sin(k x) (1 - cos(w t))
    (the shift's contribution to gamma_xx cancels part of the slicing's). Conformal variables to
    first order in eps; Gamma-hat = Gamma-tilde of the conformal metric."""
    s = gi.flat_state(b)
    X, _, _ = b.coords()
    w = k * math.sqrt(2.0 / (1.0 + a))
    sx, cx = np.sin(k * X), np.cos(k * X)
    s[18] = 1.0 + eps * sx * math.cos(w * t)
    s[19] = -(a / (1.0 + a)) * eps * (k / w) * cx * math.sin(w * t)
    Ktr = 0.5 * (1.0 + a) * eps * w * sx * math.sin(w * t)
    gxx = 1.0 - eps * sx * (1.0 - math.cos(w * t))
    dgxx = -eps * k * cx * (1.0 - math.cos(w * t))
    chi = gxx ** (-1.0 / 3.0)
    s[0] = chi
    s[1], s[4], s[6] = gxx ** (2.0 / 3.0), chi, chi
    s[7] = Ktr
    # A_ij = chi (K_ij - gamma_ij K / 3) with K_ij = K in the xx slot only
    s[8], s[11], s[13] = chi * (Ktr - gxx * Ktr / 3.0), -chi * Ktr / 3.0, -chi * Ktr / 3.0
    # Gamma-tilde^x = -d_x h^xx to first order (h^xx = gxx^(-2/3)): (2/3) d_x gxx
    s[15] = 2.0 / 3.0 * dgxx
    return s


def gamma_driver_wave_state(b, eps, k, t, a, F, eta):
    """The exact linear longitudinal gauge mode of the modified puncture gauge with the
    Gamma-driver on: alpha = 1 + A sin(kx), K = K_xx = Kh sin(kx), beta^x = Bs cos(kx),
    B^x = Bb cos(kx), gamma_xx = 1 + G sin(kx), Gamma-hat^x = (2/3) k G cos(kx), with the amplitudes
    y = (A, Kh, Bs, Bb, G) solving y' = M y (the linearised slicing, K, shift, B and metric
    equations below), y(0) = (eps, 0, 0, 0, 0), by the matrix exponential:
      A' = -2 Kh / (1 + a);  Kh' = k^2 A;  Bs' = F Bb / (1 + a) - (a / (1 + a)) k A;
      G' = -2 Kh - 2 k Bs;   Bb' = (Gamma-hat amplitude)' - eta Bb, (2/3) k G' = -(4/3) k Kh - (4/3) k^2 Bs."""
    from scipy.linalg import expm
    M = np.zeros((5, 5))
    M[0, 1] = -2.0 / (1.0 + a)
    M[1, 0] = k * k
    M[2, 3] = F / (1.0 + a)
    M[2, 0] = -(a / (1.0 + a)) * k
    M[4, 1] = -2.0
    M[4, 2] = -2.0 * k
    M[3, :] = (2.0 / 3.0) * k * M[4, :]
    M[3, 3] -= eta
    A, Kh, Bs, Bb, G = expm(M * t) @ np.array([eps, 0.0, 0.0, 0.0, 0.0])
    s = gi.flat_state(b)
    X, _, _ = b.coords()
    sx, cx = np.sin(k * X), np.cos(k * X)
    gxx = 1.0 + G * sx
    chi = gxx ** (-1.0 / 3.0)
    Ktr = Kh * sx
    s[0] = chi
    s[1], s[4], s[6] = gxx ** (2.0 / 3.0), chi, chi
    s[7] = Ktr
    s[8], s[11], s[13] = chi * (Ktr - gxx * Ktr / 3.0), -chi * Ktr / 3.0, -chi * Ktr / 3.0
    s[15] = (2.0 / 3.0) * k * G * cx
    s[18] = 1.0 + A * sx
    s[19] = Bs * cx
    s[22] = Bb * cx
    return s
