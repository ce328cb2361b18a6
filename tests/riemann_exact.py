"""Exact solution of the 1D Euler Riemann problem (Toro, "Riemann Solvers and
Numerical Methods for Fluid Dynamics", ch. 4), written from the textbook's
pressure-function equations.  Test helper for the continuum-limit pin."""
import numpy as np
from scipy.optimize import brentq


def density(x, t, left, right, x0=0.5, g=5.0 / 3.0):
    rL, uL, pL = left
    rR, uR, pR = right
    aL, aR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)

    def fk(p, r, pk, a):
        if p > pk:  # shock branch
            A, B = 2.0 / ((g + 1) * r), (g - 1) / (g + 1) * pk
            return (p - pk) * np.sqrt(A / (p + B))
        return 2 * a / (g - 1) * ((p / pk) ** ((g - 1) / (2 * g)) - 1)  # rarefaction

    ps = brentq(lambda p: fk(p, rL, pL, aL) + fk(p, rR, pR, aR) + uR - uL, 1e-10, 100.0, xtol=1e-14)
    us = 0.5 * (uL + uR) + 0.5 * (fk(ps, rR, pR, aR) - fk(ps, rL, pL, aL))
    out = np.empty(len(x))
    for k, xi in enumerate(x):
        S = (xi - x0) / t
        if S <= us:
            if ps > pL:
                SL = uL - aL * np.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                out[k] = rL if S < SL else rL * (ps / pL + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pL + 1)
            else:
                SHL, STL = uL - aL, us - aL * (ps / pL) ** ((g - 1) / (2 * g))
                if S < SHL:
                    out[k] = rL
                elif S > STL:
                    out[k] = rL * (ps / pL) ** (1 / g)
                else:
                    out[k] = rL * (2 / (g + 1) + (g - 1) / ((g + 1) * aL) * (uL - S)) ** (2 / (g - 1))
        else:
            if ps > pR:
                SR = uR + aR * np.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                out[k] = rR if S > SR else rR * (ps / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pR + 1)
            else:
                SHR, STR = uR + aR, us + aR * (ps / pR) ** ((g - 1) / (2 * g))
                if S > SHR:
                    out[k] = rR
                elif S < STR:
                    out[k] = rR * (ps / pR) ** (1 / g)
                else:
                    out[k] = rR * (2 / (g + 1) - (g - 1) / ((g + 1) * aR) * (uR - S)) ** (2 / (g - 1))
    return out
