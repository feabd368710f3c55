"""Manufactured solution of the paper's convergence tests (Sec. 3.1): p = prod sin(pi sin(pi x_a))
on [0,1]^d and f = p - Lap p from the continuous equation, evaluated at cell centres."""
import numpy as np


def _parts(n):
    x = (np.arange(n) + 0.5) / n
    g = np.pi * np.sin(np.pi * x)
    gp = np.pi ** 2 * np.cos(np.pi * x)
    gpp = -np.pi ** 3 * np.sin(np.pi * x)
    s = np.sin(g)
    spp = -np.sin(g) * gp ** 2 + np.cos(g) * gpp  # d^2/dx^2 sin(g(x))
    return s, spp


def exact_and_source(n, dim):
    s, spp = _parts(n)
    if dim == 2:
        p = s[:, None] * s[None, :]
        lap = spp[:, None] * s[None, :] + s[:, None] * spp[None, :]
    else:
        p = s[:, None, None] * s[None, :, None] * s[None, None, :]
        lap = (spp[:, None, None] * s[None, :, None] * s[None, None, :]
               + s[:, None, None] * spp[None, :, None] * s[None, None, :]
               + s[:, None, None] * s[None, :, None] * spp[None, None, :])
    return p, p - lap


def l2_error(u, p, n, dim):
    return (1.0 / n) ** (dim / 2.0) * float(np.sqrt(np.sum((u - p) ** 2)))
