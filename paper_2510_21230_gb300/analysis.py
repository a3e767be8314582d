"""Post-processing of the observables of the validation runs (section 5).

* ``rdf``: g(r) from the library's pair-distance histogram (every pair once):
  g = counts / (samples * N/2 * rho * shell volume), at the bin centres.
* ``density_profile``: rho(z) at the bin centres from the density histogram.
* ``fit_interfaces``: the two planar interfaces of a liquid slab fitted, side
  by side, to the hyperbolic-tangent profile of Eq. tanh,
      rho(z) = (rho_l + rho_g) / 2 - (rho_l - rho_g) / 2 * tanh(2 (z - z0) / d).
  The printed equation has (rho_l + rho_g) in both terms, which would make
  the profile run from rho_l + rho_g to 0; the difference in the tanh term
  is the form that tends to rho_l inside the liquid and rho_g in the vapour.

Host arithmetic only (numpy; the fit uses scipy's least squares).
"""
import math

import numpy as np


def rdf(counts, samples, n, volume, r_max):
    """(r, g) at the bin centres of a histogram over [0, r_max)."""
    counts = np.asarray(counts, dtype=np.float64)
    nb = counts.shape[-1]
    edges = np.linspace(0.0, float(r_max), nb + 1)
    shell = 4.0 / 3.0 * math.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    rho = n / float(volume)
    g = counts / (max(samples, 1) * 0.5 * n * rho * shell)
    return 0.5 * (edges[1:] + edges[:-1]), g


def density_profile(counts, samples, box, axis=2):
    """(z, rho) at the bin centres of a density histogram along ``axis``."""
    counts = np.asarray(counts, dtype=np.float64)
    box = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    nb = counts.shape[-1]
    h = box[axis] / nb
    area = float(np.prod(box)) / box[axis]
    return (np.arange(nb) + 0.5) * h, counts / (max(samples, 1) * area * h)


def tanh_profile(z, rho_l, rho_g, z0, d):
    """Eq. tanh (difference reading): liquid below z0, vapour above for d > 0."""
    return 0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * np.tanh(2.0 * (z - z0) / d)


def _fit_side(u, rho, half):
    from scipy.optimize import least_squares
    hi = float(np.percentile(rho, 95))
    lo = float(np.percentile(rho, 5))
    x0 = np.array([hi, lo, 0.5 * half, 2.0])

    def res(p):
        return tanh_profile(u, p[0], p[1], p[2], p[3]) - rho

    fit = least_squares(res, x0, bounds=([0.0, 0.0, 0.0, 1e-3], [np.inf, np.inf, half, half]),
                        x_scale="jac")
    rl, rg, u0, d = fit.x
    return dict(rho_l=float(rl), rho_g=float(rg), u0=float(u0), d=float(d),
                rms=float(np.sqrt(np.mean(fit.fun ** 2))))


def fit_interfaces(z, rho, length):
    """Fit both interfaces of a periodic slab profile.

    The slab centre z_c is the circular mean of z weighted by rho - min(rho);
    the half above it is fitted as is, the half below it mirrored, each with
    Eq. tanh.  Returns {"centre": z_c, "right": {...}, "left": {...}} with
    rho_l, rho_g, the interface position z0 (box coordinates) and width d."""
    z = np.asarray(z, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    L = float(length)
    w = rho - rho.min()
    th = 2.0 * math.pi * z / L
    zc = (math.atan2(float((w * np.sin(th)).sum()), float((w * np.cos(th)).sum())) * L
          / (2.0 * math.pi)) % L
    u = (z - zc + 0.5 * L) % L - 0.5 * L
    out = {"centre": zc}
    for side, sel, sign in (("right", u >= 0.0, 1.0), ("left", u < 0.0, -1.0)):
        r = _fit_side(sign * u[sel], rho[sel], 0.5 * L)
        r["z0"] = (zc + sign * r.pop("u0")) % L
        out[side] = r
    return out
