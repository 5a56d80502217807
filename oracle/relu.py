"""Composite polynomial ReLU (HActivation, Sec. 2.4.2 / Alg. 1, activation step) for the oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

ReLU(x) = x (1 + sign(x)) / 2 with sign approximated by a composition of odd
polynomials (degrees 15, 15, 27 by default).  The paper takes its ReLU approximation
from the literature (Sec. 5, "poly approx") and does not print coefficients; the
reading here: each stage is the minimax odd polynomial of its degree for the constant 1
on [eps_k, 1] (a linear program on a fine grid, scipy's HiGHS), normalised by 1 + tau_k
so that it maps [-1, 1] into [-1, 1]; stage k+1 then works on [eps_{k+1}, 1] with
eps_{k+1} = (1 - tau_k) / (1 + tau_k).  The last stage is folded into g = (1 + p) / 2.
Stages are returned in the Chebyshev basis (what the evaluator takes).
"""
import numpy as np
from scipy.optimize import linprog

from .scheme import Oracle


def fit_odd_sign(deg, eps, npts=3000):
    """minimise t subject to |sum_k a_k x^(2k+1) - 1| <= t on [eps, 1]; returns (a, t)"""
    th = np.linspace(0.0, np.pi, npts)
    x = eps + (1.0 - eps) * (1.0 - np.cos(th)) / 2.0
    K = (deg + 1) // 2
    V = np.stack([x ** (2 * k + 1) for k in range(K)], axis=1)
    c = np.zeros(K + 1)
    c[-1] = 1.0
    A = np.vstack([np.hstack([V, -np.ones((npts, 1))]), np.hstack([-V, -np.ones((npts, 1))])])
    b = np.concatenate([np.ones(npts), -np.ones(npts)])
    r = linprog(c, A_ub=A, b_ub=b, bounds=[(None, None)] * K + [(0, None)], method="highs")
    assert r.success, r.message
    a = r.x[:K]
    # the LP bounds the error on its grid; report the error measured on a 20x finer grid
    xf = np.linspace(eps, 1.0, 20 * npts)
    pf = sum(a[k] * xf ** (2 * k + 1) for k in range(K))
    return a, float(np.abs(pf - 1.0).max())


def odd_power_to_cheb(a):
    """odd power-basis coefficients a_k of x^(2k+1) -> Chebyshev coefficients"""
    p = np.zeros(2 * len(a))
    p[1::2] = a
    return np.polynomial.chebyshev.poly2cheb(p)


def composite_relu_stages(degrees=(15, 15, 27), eps=2.0 ** -8):
    """Chebyshev coefficients of f_1, ..., f_{k-1}, g with ReLU(x) ~ x g(f_{k-1}(...f_1(x)))"""
    stages, info = [], []
    e = eps
    for i, deg in enumerate(degrees):
        a, t = fit_odd_sign(deg, e)
        info.append({"deg": deg, "eps": e, "tau": t})
        if i < len(degrees) - 1:
            stages.append(odd_power_to_cheb(a / (1.0 + t)))
            e = (1.0 - t) / (1.0 + t)
        else:
            g = 0.5 * odd_power_to_cheb(a)
            g[0] += 0.5
            stages.append(g)
    return [list(map(float, s)) for s in stages], info


def relu_poly_fp64(x, stages):
    """the FP64 network activation: x g(f_{k-1}(...f_1(x)))"""
    y = np.asarray(x, dtype=np.float64)
    for s in stages:
        y = np.polynomial.chebyshev.chebval(y, s)
    return np.asarray(x) * y


def relu_eval(orc: Oracle, ct, stages):
    """HActivation on a slot-encoded ciphertext: chained Chebyshev evaluations, then one
    HMult with the input brought down to the last stage's level"""
    y = ct
    for s in stages:
        y = orc.cheb_eval(y, s)
    lev = orc.prod_level(y.level)
    return orc.mul_relin_rescale(orc.level_down(ct, lev), orc.level_down(y, lev))
