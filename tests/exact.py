"""Closed forms the tests pin the oracle (and the library) against.

Nothing here calls the oracle or the CUDA library:
  * integrals of monomials over arbitrary simplices by the Dirichlet formula on barycentric
    coordinates, int_T lambda^g = d! |T| prod(g_j!) / (|g| + d)!, after multinomial expansion;
  * the exact solution of the 1D Riemann problem for the Euler equations (Toro, "Riemann Solvers
    and Numerical Methods for Fluid Dynamics", ch. 4: pressure function, Newton iteration for the
    star pressure, sampling of the self-similar solution).
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def _compositions(total: int, parts: int):
    if parts == 1:
        yield (total,)
        return
    for k in range(total + 1):
        for rest in _compositions(total - k, parts - 1):
            yield (k,) + rest


def _multinomial(n, ks):
    out = math.factorial(n)
    for k in ks:
        out //= math.factorial(k)
    return out


def simplex_volume(verts: np.ndarray) -> float:
    d = verts.shape[1]
    J = (verts[1:] - verts[0]).T
    return abs(np.linalg.det(J)) / math.factorial(d)


def simplex_monomial_integral(verts: np.ndarray, exps) -> float:
    """int_T prod_j x_j^{e_j} dx over the simplex with vertices verts [(d+1), d]."""
    verts = np.asarray(verts, dtype=np.float64)
    d = verts.shape[1]
    nvt = d + 1
    vol = simplex_volume(verts)
    total = 0.0
    # expand each coordinate power over barycentric coordinates
    per_coord = []
    for j in range(d):
        terms = []
        for beta in _compositions(int(exps[j]), nvt):
            c = _multinomial(int(exps[j]), beta)
            for a in range(nvt):
                c *= verts[a, j] ** beta[a]
            terms.append((c, beta))
        per_coord.append(terms)
    for combo in itertools.product(*per_coord):
        coef = 1.0
        g = [0] * nvt
        for c, beta in combo:
            coef *= c
            for a in range(nvt):
                g[a] += beta[a]
        num = math.factorial(d)
        for ga in g:
            num *= math.factorial(ga)
        total += coef * num / math.factorial(sum(g) + d)
    return vol * total


def poly_eval(poly: dict, x: np.ndarray) -> np.ndarray:
    """poly: {exponent tuple: coefficient}; x [..., d]."""
    out = np.zeros(x.shape[:-1])
    for e, c in poly.items():
        term = np.full(x.shape[:-1], c, dtype=np.float64)
        for j, p in enumerate(e):
            term = term * x[..., j] ** p
        out = out + term
    return out


def poly_cell_average(poly: dict, verts: np.ndarray) -> float:
    return sum(c * simplex_monomial_integral(verts, e) for e, c in poly.items()) / simplex_volume(verts)


def all_exponents(d: int, r: int, min_deg: int = 0):
    out = []
    for t in range(min_deg, r + 1):
        for e in _compositions(t, d):
            out.append(e)
    return out


def random_poly(d: int, r: int, rng: np.random.Generator, scale: float = 1.0) -> dict:
    return {e: scale * rng.uniform(-1, 1) for e in all_exponents(d, r)}


# ---------------------------------------------------------------------------------------------
# Exact Riemann solver (Toro, ch. 4)
# ---------------------------------------------------------------------------------------------
def _fK(p, rho, pK, cK, g):
    if p > pK:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        f = (p - pK) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - (p - pK) / (2.0 * (B + p)))
    else:
        f = 2.0 * cK / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * cK) * (p / pK) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def riemann_exact(WL, WR, xi: np.ndarray, g: float = 1.4) -> np.ndarray:
    """Self-similar solution (rho, u, p) at xi = x/t of the Riemann problem WL | WR."""
    rL, uL, pL = WL
    rR, uR, pR = WR
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    p = max(1e-8, 0.5 * (pL + pR))
    for _ in range(100):
        fL, dL = _fK(p, rL, pL, cL, g)
        fR, dR = _fK(p, rR, pR, cR, g)
        pn = max(1e-12, p - (fL + fR + uR - uL) / (dL + dR))
        if abs(pn - p) < 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fK(p, rL, pL, cL, g)
    fR, _ = _fK(p, rR, pR, cR, g)
    us = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    out = np.empty((xi.size, 3))
    for k, s in enumerate(xi):
        if s <= us:  # left of contact
            if p > pL:
                rs = rL * ((p / pL + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pL + 1))
                SL = uL - cL * math.sqrt((g + 1) / (2 * g) * p / pL + (g - 1) / (2 * g))
                out[k] = (rL, uL, pL) if s <= SL else (rs, us, p)
            else:
                rs = rL * (p / pL) ** (1 / g)
                cs = cL * (p / pL) ** ((g - 1) / (2 * g))
                if s <= uL - cL:
                    out[k] = (rL, uL, pL)
                elif s >= us - cs:
                    out[k] = (rs, us, p)
                else:
                    u = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
                    c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    out[k] = (rL * (c / cL) ** (2 / (g - 1)), u, pL * (c / cL) ** (2 * g / (g - 1)))
        else:
            if p > pR:
                rs = rR * ((p / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * p / pR + 1))
                SR = uR + cR * math.sqrt((g + 1) / (2 * g) * p / pR + (g - 1) / (2 * g))
                out[k] = (rR, uR, pR) if s >= SR else (rs, us, p)
            else:
                rs = rR * (p / pR) ** (1 / g)
                cs = cR * (p / pR) ** ((g - 1) / (2 * g))
                if s >= uR + cR:
                    out[k] = (rR, uR, pR)
                elif s <= us + cs:
                    out[k] = (rs, us, p)
                else:
                    u = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
                    c = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    out[k] = (rR * (c / cR) ** (2 / (g - 1)), u, pR * (c / cR) ** (2 * g / (g - 1)))
    return out


def euler_flux(u: np.ndarray, n: np.ndarray, g: float = 1.4) -> np.ndarray:
    """Physical flux F(U).n of the Euler equations (eq. 1), conserved U."""
    d = n.size
    rho = u[0]
    vel = u[1:1 + d] / rho
    p = (g - 1) * (u[d + 1] - 0.5 * rho * vel @ vel)
    un = vel @ n
    F = np.empty(d + 2)
    F[0] = rho * un
    F[1:1 + d] = u[1:1 + d] * un + p * n
    F[d + 1] = (u[d + 1] + p) * un
    return F


def prim_to_cons(prim, g: float = 1.4) -> np.ndarray:
    prim = np.asarray(prim, dtype=np.float64)
    d = prim.size - 2
    rho, vel, p = prim[0], prim[1:1 + d], prim[-1]
    return np.concatenate([[rho], rho * vel, [p / (g - 1) + 0.5 * rho * vel @ vel]])
