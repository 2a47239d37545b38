"""High-precision restatements for tiny systems (n <= ~40), in Python ``decimal``.

TEST INFRASTRUCTURE (pins for the FP64 oracle, not an oracle of its own).

* ``cg_decimal``   -- textbook Hestenes-Stiefel CG, the method the paper
  reformulates (Sec. 1); exact up to ``prec`` digits.
* ``plcg_decimal`` -- Algorithm 1 (M = I) with full histories of every basis
  vector and of the whole matrix G (no rings, no band storage), so that the
  exact-arithmetic identity "p(l)-CG produces the CG iterates"
  (Sec. 2.1: it is a reformulation of CG via D-Lanczos) can be checked
  iterate for iterate.

Both take a dense matrix (list of lists of Decimal or floats) so they share
nothing with the oracle's operators.
"""
from __future__ import annotations

from decimal import Decimal, getcontext, localcontext


def _D(v):
    return v if isinstance(v, Decimal) else Decimal(repr(float(v)))


def _matvec(A, x):
    return [sum((a * xi for a, xi in zip(row, x)), Decimal(0)) for row in A]


def _dot(a, b):
    return sum((x * y for x, y in zip(a, b)), Decimal(0))


def cg_decimal(A, b, kmax, prec=60):
    """Textbook CG from x0 = 0.  Returns (xs, alphas, betas, rnorms) with
    xs[k] the k-th iterate; stops when r vanishes (relative 1e-(prec-10))."""
    with localcontext() as ctx:
        ctx.prec = prec
        A = [[_D(a) for a in row] for row in A]
        b = [_D(v) for v in b]
        n = len(b)
        x = [Decimal(0)] * n
        r = list(b)
        p = list(r)
        rr = _dot(r, r)
        tiny = rr * Decimal(10) ** (-(prec - 10))
        xs, alphas, betas, rnorms = [list(x)], [], [], [rr.sqrt()]
        for _ in range(kmax):
            if rr <= tiny:
                break
            q = _matvec(A, p)
            alpha = rr / _dot(p, q)
            x = [xi + alpha * pi for xi, pi in zip(x, p)]
            r = [ri - alpha * qi for ri, qi in zip(r, q)]
            rr_new = _dot(r, r)
            beta = rr_new / rr
            p = [ri + beta * pi for ri, pi in zip(r, p)]
            rr = rr_new
            xs.append(list(x))
            alphas.append(alpha)
            betas.append(beta)
            rnorms.append(rr.sqrt())
        return xs, alphas, betas, rnorms


def plcg_decimal(A, b, l, sigma, kmax, prec=60):
    """Algorithm 1 with M = I from x0 = 0, all 2l+1 dot products of K5,
    full histories.  Returns dict with xs (x_k), gamma, delta, zeta, G (dict
    keyed by (j, i)), Z (list over k of dict j -> vector).  Stops after kmax
    x-updates or at a (lucky) breakdown, where it stops without the extra
    update so that only well-defined CG iterates are compared."""
    with localcontext() as ctx:
        ctx.prec = prec
        A = [[_D(a) for a in row] for row in A]
        b = [_D(v) for v in b]
        sig = [_D(s) for s in sigma]
        n = len(b)
        zero = [Decimal(0)] * n
        r0 = list(b)                        # x0 = 0
        nu = _dot(r0, r0).sqrt()
        z0 = [v / nu for v in r0]
        Z = [{0: list(z0)} for _ in range(l + 1)]   # Z[k][j] = z^(k)_j
        G = {(0, 0): Decimal(1)}
        g = lambda j, i: G.get((j, i), Decimal(0)) if j >= 0 else Decimal(0)
        gamma, delta, eta, zeta = {}, {}, {}, {}
        x = [Decimal(0)] * n
        xs = [list(x)]
        p = None
        i = 0
        while True:
            # K1
            w = _matvec(A, Z[l][i])
            if i < l:
                w = [wi - sig[i] * zi for wi, zi in zip(w, Z[l][i])]
            Z[l][i + 1] = w
            if i < l - 1:
                for k in range(i + 1, l):
                    Z[k][i + 1] = list(w)
            if i >= l:
                c, m = i - l + 1, i - l
                lo = max(0, i - 3 * l + 1)
                for j in range(max(0, i - 2 * l + 2), i - l + 1):
                    s = g(j, c) - sum((g(k, j) * g(k, c) for k in range(lo, j)), Decimal(0))
                    G[(j, c)] = s / g(j, j)
                arg = g(c, c) - sum((g(k, c) ** 2 for k in range(lo, c)), Decimal(0))
                if arg <= 0:
                    break
                G[(c, c)] = arg.sqrt()
                dm1 = delta.get(m - 1, Decimal(0))
                if i < 2 * l:
                    gamma[m] = (g(m, c) + sig[m] * g(m, m) - g(m - 1, m) * dm1) / g(m, m)
                    delta[m] = g(c, c) / g(m, m)
                else:
                    gamma[m] = (g(m, m) * gamma[m - l] + g(m, c) * delta[m - l]
                                - g(m - 1, m) * dm1) / g(m, m)
                    delta[m] = g(c, c) * delta[m - l] / g(m, m)
                for k in range(l):
                    zp = Z[k].get(m + k - 1, zero)
                    Z[k][m + k + 1] = [(a + (sig[k] - gamma[m]) * bb - dm1 * cc) / delta[m]
                                       for a, bb, cc in zip(Z[k + 1][m + k + 1], Z[k][m + k], zp)]
                zp = Z[l].get(i - 1, zero)
                Z[l][i + 1] = [(a - gamma[m] * bb - dm1 * cc) / delta[m]
                               for a, bb, cc in zip(Z[l][i + 1], Z[l][i], zp)]
            # K5 (2l+1 dot products)
            u = Z[l][i + 1]
            for j in range(max(0, i - 2 * l + 1), i - l + 2):
                G[(j, i + 1)] = _dot(u, Z[0][j])
            for j in range(max(0, i - l + 2), i + 2):
                G[(j, i + 1)] = _dot(u, Z[l][j])
            # K6
            if i == l:
                eta[0] = gamma[0]
                zeta[0] = nu
                p = [v / eta[0] for v in Z[0][0]]
            elif i >= l + 1:
                m = i - l
                lam = delta[m - 1] / eta[m - 1]
                eta[m] = gamma[m] - lam * delta[m - 1]
                zeta[m] = -lam * zeta[m - 1]
                x = [xi + zeta[m - 1] * pi for xi, pi in zip(x, p)]
                p = [(v - delta[m - 1] * pi) / eta[m] for v, pi in zip(Z[0][m], p)]
                xs.append(list(x))
                if m >= kmax:
                    break
            i += 1
        return {"xs": xs, "gamma": gamma, "delta": delta, "zeta": zeta, "G": G, "Z": Z}
