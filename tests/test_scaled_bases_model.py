"""Host model of FP64 p(1)-CG with scaled bases (no GPU).

The GPU kernel for FP64 p(1)-CG on large systems stores its bases scaled,
Z_j = z^(1)_j / s_j and W_j = z^(0)_j / t_j (and the direction phat_m / t_m),
so that K4 needs no multiply; the K5 dots are multiplied back by their
scales before the scalar step, and a power of two is folded in whenever a
scale leaves its range.  This file restates the kernel's l = 1 iteration
(the scalar step and the sweep, M = I, a constant-coefficient stencil) in
numpy twice -- with unscaled bases, and with scaled bases whose range bound
is made tiny (2^-1 .. 2^1) so that almost every iteration rescales -- and
checks both against the FP64 oracle's iterates: the transformation is exact
up to rounding, and the power-of-two rescaling path is exercised densely.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1905_06850_gb300 import workloads as W


def _neighbour_sum(op, z):
    """nb with (A z) = center z + off nb (Dirichlet), lexicographic x fastest."""
    nx, ny, nz = op["nx"], op["ny"], op.get("nz", 1) if op["dim"] == 3 else 1
    g = z.reshape(nz, ny, nx)
    nb = np.zeros_like(g)
    nb[:, :, 1:] += g[:, :, :-1]
    nb[:, :, :-1] += g[:, :, 1:]
    nb[:, 1:, :] += g[:, :-1, :]
    nb[:, :-1, :] += g[:, 1:, :]
    if op["dim"] == 3:
        nb[1:, :, :] += g[:-1, :, :]
        nb[:-1, :, :] += g[1:, :, :]
    return nb.ravel()


def plcg1_model(op, b, sigma0, maxit, scaled, bound=1):
    """p(1)-CG as the kernel runs it (l + 1 dots, x0 = 0): x_maxit and the
    number of power-of-two rescales."""
    kc, kn = op["center"], op["off"]
    rn = np.linalg.norm(b)
    z1 = {0: b / rn}             # z^(1)_j (stored: Z_j)
    z0 = {0: b / rn}             # z^(0)_j (stored: W_j)
    x = np.zeros_like(b)
    p = None
    G = {0: [0.0, 0.0, 1.0]}     # G[c] = [g_{c-2,c}, g_{c-1,c}, g_{c,c}]; g_00 = 1
    G_inv = {0: 1.0}
    gam, dl, idl, eta, zeta, ieta = {}, {}, {}, {}, {}, {}
    s, t, i_s, i_t = {0: 1.0, 1: 1.0}, {0: 1.0}, {0: 1.0, 1: 1.0}, {0: 1.0}
    ikn = 1.0 / kn
    rescales = 0

    def g(j, cc):
        if j < 0 or j < cc - 2 or j > cc:
            return 0.0
        return G[cc][j - cc + 2]

    # sweep 0 (fill): z^(1)_1 = (A - sigma_0) z^(1)_0; dots with u_1 = z^(1)_1
    u = (kc - sigma0) * z1[0] + kn * _neighbour_sum(op, z1[0])
    z1[1] = u
    raw = [0.0, u @ z0[0], u @ u]
    i = 1
    while True:
        m, c = i - 1, i
        si = s[i] if scaled else 1.0
        col = []
        for q in range(3):
            v = raw[q] if c - 2 + q >= 0 else 0.0
            if scaled:
                v *= si * (si if q == 2 else t[m] if q == 1 else t.get(m - 1, 1.0))
            col.append(v)
        G[c] = col
        if c - 2 >= 0:                       # l + 1 dots: g_{c-2,c} = g_{c-1,c-1}
            col[0] = g(c - 1, c - 1)
        lo = max(c - 2, 0)
        arg = col[2] - sum(col[k - c + 2] ** 2 for k in range(lo, c))
        assert arg > 0
        rg = 1.0 / np.sqrt(arg)
        gmm, igmm = g(m, m), G_inv[m]
        gmc = col[m - c + 2]
        dm1 = dl.get(m - 1, 0.0)
        if m < 1:
            gm = (gmc + sigma0 * gmm) * igmm
        else:
            gm = (gmm * gam[m - 1] + gmc * dl[m - 1] - g(m - 1, m) * dm1) * igmm
        gam[m] = gm
        lam = em = iem = zm = 0.0
        if m >= 1:
            lam = dm1 * ieta[m - 1]
            em = gm - lam * dm1
            iem = 1.0 / em
            zm = -lam * zeta[m - 1]
        gcc = arg * rg
        col[2] = gcc
        G_inv[c] = rg
        invd = rg * gmm if m < 1 else rg * gmm * idl[m - 1]
        dm = gcc * igmm if m < 1 else gcc * dl[m - 1] * igmm
        dl[m], idl[m] = dm, invd
        tmm1 = t.get(m - 1, 1.0) if scaled else 1.0
        if scaled:
            bs, bt = invd * kn * si, invd * si
            e = 0 if 2.0 ** -bound <= abs(bs) <= 2.0 ** bound else -int(np.floor(np.log2(abs(bs))))
            f = 0 if 2.0 ** -bound <= abs(bt) <= 2.0 ** bound else -int(np.floor(np.log2(abs(bt))))
            pe, pf = 2.0 ** -e, 2.0 ** -f
            rescales += (e != 0) + (f != 0)
            s[i + 1], i_s[i + 1] = bs * 2.0 ** e, dm * ikn * i_s[i] * pe
            t[m + 1], i_t[m + 1] = bt * 2.0 ** f, dm * i_s[i] * pf
            ivk = pe * ikn
            uc, unb = (kc - gm) * ivk, pe
            bm = -dm1 * (s[i - 1] * i_s[i]) * ivk if m >= 1 else 0.0
            ak = (sigma0 - gm) * (t[m] * i_s[i]) * pf
            wu = pf
            wb = -dm1 * (t.get(m - 1, 1.0) * i_s[i]) * pf if m >= 1 else 0.0
        else:
            uc, unb = kc * invd - gm * invd, kn * invd
            bm = -dm1 * invd if m >= 1 else 0.0
            ak, wu, wb = (sigma0 - gm) * invd, invd, bm
        # K6 on phat_m / t_m
        if i == 1:
            eta[0], zeta[0], ieta[0] = gm, rn, 1.0 / gm
            k6, zx, pp = 1, 0.0, 0.0
        else:
            iep = ieta[m - 1]
            k6, zx, pp = 2, zeta[m - 1] * iep * tmm1, -dm1 * iep * (tmm1 * i_t[m] if scaled else 1.0)
            eta[m], ieta[m], zeta[m] = em, iem, zm
            if m >= maxit:                   # the final sweep: x_m = x_{m-1} + zx P_{m-1}
                return x + zx * p, rescales
        # sweep i
        Zi, Zp = z1[i], z1[i - 1]
        un = uc * Zi + unb * _neighbour_sum(op, Zi) + bm * Zp
        pk = z0[m - 1] if m >= 1 else np.zeros_like(b)
        nw = wu * Zi + ak * z0[m] + wb * pk
        if k6 == 1:
            p = z0[m].copy()
        else:
            x = x + zx * p
            p = pp * p + z0[m]
        z1[i + 1], z0[m + 1] = un, nw
        raw = [0.0, un @ nw, un @ un]
        i += 1


@pytest.mark.parametrize("scaled", [False, True])
@pytest.mark.parametrize("k", [1, 2, 7, 40])
@pytest.mark.parametrize("dims", [(12, 10, 1), (7, 6, 5)])
def test_scaled_bases_model_matches_oracle(scaled, k, dims):
    nx, ny, nz = dims
    op = W.stencil2d(nx, ny) if nz == 1 else W.stencil3d(nx, ny, nz)
    b = W.rhs(op, np.random.default_rng(nx * ny * nz).standard_normal(nx * ny * nz))
    interval = (0.0, 8.0) if nz == 1 else (0.0, 12.0)
    sig = O.chebyshev_shifts(1, *interval)
    ref = O.plcg(op, b, l=1, sigma=sig, rtol=1e-300, maxit=k, dots_2l1=False)
    assert ref.iters == k
    x, rescales = plcg1_model(op, b, sig[0], k, scaled)
    assert np.linalg.norm(x - ref.x) <= 1e-12 * np.linalg.norm(ref.x), (scaled, k, dims)
    if scaled and k >= 7:
        assert rescales >= k // 2   # the range bound 2^+-1 is left at most steps
