"""A host model of one p(l)-CG solve sharded over ranks (no GPU).

The paper's own setting (Sec. 3.1, Algorithm 2) is one solve distributed
over MPI ranks: every rank owns a block of rows, the SpMV needs the
neighbours' boundary values of z^(l)_i first (a halo exchange), and the dot
products of K5 are summed over ranks by an MPI_Iallreduce that the scalar
steps wait for l iterations later.  This module restates that layout in
numpy over torch.distributed (gloo, CPU), for a 3D 7-point Dirichlet
stencil split into slabs of whole z-planes:

* rank r owns planes [z0, z1) -- rows [z0 nx ny, z1 nx ny) in lexicographic
  order -- of every vector;
* before each application of A the rank sends its first plane to rank r-1
  and its last plane to rank r+1 and receives theirs (zeros at the domain's
  own boundary, Dirichlet);
* the 2l+1 (or l+1) dot products of K5 are local partial sums, started as an
  asynchronous all_reduce at iteration i and waited for at iteration i+l,
  when K2 finalises column i-l+1 of G (the overlap of Algorithm 2);
* every rank runs the O(l^2) scalar work (K2, K3, K6 scalars) on the same
  reduced values, so all ranks hold the same scalars without a broadcast.

The arithmetic is Algorithm 1 with M = I in the paper's order and notation,
with full histories (tiny systems), so that the tests can hold every
iterate x_k against the FP64 oracle's.  It is a model of the data flow for
a multi-GPU layout, not a product path.
"""
from __future__ import annotations

import numpy as np


class Slab:
    """Rank `rank`'s planes of an nx x ny x nz grid split over `world` ranks."""

    def __init__(self, nx: int, ny: int, nz: int, rank: int, world: int):
        planes = np.array_split(np.arange(nz), world)[rank]
        if planes.size == 0:
            raise ValueError("every rank needs at least one plane")
        self.nx, self.ny, self.nz = nx, ny, nz
        self.rank, self.world = rank, world
        self.z0, self.z1 = int(planes[0]), int(planes[-1]) + 1
        self.nxy = nx * ny
        self.nloc = (self.z1 - self.z0) * self.nxy
        self.rows = slice(self.z0 * self.nxy, self.z1 * self.nxy)

    def halo(self, v: np.ndarray):
        """The plane below z0 and the plane above z1 - 1 from the neighbours."""
        import torch
        import torch.distributed as dist
        below = torch.zeros(self.nxy, dtype=torch.float64)
        above = torch.zeros(self.nxy, dtype=torch.float64)
        reqs = []
        if self.rank > 0:
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(v[:self.nxy])), self.rank - 1))
            reqs.append(dist.irecv(below, self.rank - 1))
        if self.rank < self.world - 1:
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(v[-self.nxy:])), self.rank + 1))
            reqs.append(dist.irecv(above, self.rank + 1))
        for r in reqs:
            r.wait()
        return below.numpy(), above.numpy()

    def apply(self, v: np.ndarray, center: float, off: float) -> np.ndarray:
        """(A v) on this slab: center v + off * (sum of the 6 neighbours)."""
        below, above = self.halo(v)
        nzl = self.z1 - self.z0
        V = v.reshape(nzl, self.ny, self.nx)
        nb = np.zeros_like(V)
        nb[:, :, 1:] += V[:, :, :-1]
        nb[:, :, :-1] += V[:, :, 1:]
        nb[:, 1:, :] += V[:, :-1, :]
        nb[:, :-1, :] += V[:, 1:, :]
        nb[1:] += V[:-1]
        nb[:-1] += V[1:]
        nb[0] += below.reshape(self.ny, self.nx)
        nb[-1] += above.reshape(self.ny, self.nx)
        return (center * V + off * nb).ravel()


def allreduce_async(vals):
    import torch
    import torch.distributed as dist
    t = torch.tensor(vals, dtype=torch.float64)
    return t, dist.all_reduce(t, async_op=True)


def sharded_plcg(slab: Slab, center: float, off: float, b_loc: np.ndarray, l: int, sigma,
                 rtol: float, maxit: int, dots_2l1: bool = True):
    """Algorithm 1 (M = I, x0 = 0) on this rank's slab.  Returns the list of
    this rank's slabs of x_0, x_1, ..., the last iterate's index k and
    |zeta_k|; stops at |zeta_k| < rtol ||b||, at k = maxit or at a
    square-root breakdown (then without the extra update)."""
    import torch.distributed as dist
    import torch
    bb = torch.tensor([float(b_loc @ b_loc)], dtype=torch.float64)
    dist.all_reduce(bb)
    nrm_b = float(np.sqrt(bb.item()))
    nu = nrm_b                                   # x0 = 0: r0 = b
    z0 = b_loc / nu
    Z = [{0: z0.copy()} for _ in range(l + 1)]   # Z[k][j] = this rank's slab of z^(k)_j
    G = {(0, 0): 1.0}

    def g(j, i):
        return G.get((j, i), 0.0) if j >= 0 else 0.0

    gamma, delta, eta, zeta = {}, {}, {}, {}
    x = np.zeros_like(b_loc)
    xs = [x.copy()]
    p = None
    pending = {}                                  # iteration -> (values, work) of its all_reduce
    i = 0
    while True:
        # K1: A z^(l)_i (halo exchange inside), shifted in the fill phase
        w = slab.apply(Z[l][i], center, off)
        if i < l:
            w = w - sigma[i] * Z[l][i]
            Z[l][i + 1] = w
            for k in range(i + 1, l):
                Z[k][i + 1] = w.copy()
        else:
            # MPI_Wait of the reduction started l iterations ago: column c of G
            c, m = i - l + 1, i - l
            t, work = pending.pop(i - l)
            work.wait()
            vals = t.numpy()
            j0 = max(0, c - 2 * l)
            for q, j in enumerate(range(c - 2 * l, c + 1)):
                if j >= 0 and (dots_2l1 or j >= c - l):
                    G[(j, c)] = float(vals[q])
            if not dots_2l1:                      # Sec. 2.2: g_{j,c} = g_{c-l, j+l}
                for j in range(j0, c - l):
                    G[(j, c)] = g(c - l, j + l)
            lo = max(0, i - 3 * l + 1)
            # K2: finalise column c
            for j in range(max(0, i - 2 * l + 2), c):
                s = g(j, c) - sum(g(k, j) * g(k, c) for k in range(lo, j))
                G[(j, c)] = s / g(j, j)
            arg = g(c, c) - sum(g(k, c) ** 2 for k in range(lo, c))
            if arg <= 0.0:                        # breakdown: no further iterate
                for t, work in pending.values():
                    work.wait()
                return xs, len(xs) - 1, None
            G[(c, c)] = float(np.sqrt(arg))
            # K3
            dm1 = delta.get(m - 1, 0.0)
            if i < 2 * l:
                gamma[m] = (g(m, c) + sigma[m] * g(m, m) - g(m - 1, m) * dm1) / g(m, m)
                delta[m] = g(c, c) / g(m, m)
            else:
                gamma[m] = (g(m, m) * gamma[m - l] + g(m, c) * delta[m - l] - g(m - 1, m) * dm1) / g(m, m)
                delta[m] = g(c, c) * delta[m - l] / g(m, m)
            # K4: the l + 1 basis recurrences
            for k in range(l):
                zp = Z[k].get(m + k - 1, 0.0)
                Z[k][m + k + 1] = (Z[k + 1][m + k + 1] + (sigma[k] - gamma[m]) * Z[k][m + k] - dm1 * zp) / delta[m]
            zp = Z[l].get(i - 1, 0.0)
            Z[l][i + 1] = (w - gamma[m] * Z[l][i] - dm1 * zp) / delta[m]
        # K5: local partials of column i + 1, reduced asynchronously (Iallreduce)
        u = Z[l][i + 1]
        part = []
        for j in range(i - 2 * l + 1, i + 2):
            if j < 0 or (not dots_2l1 and j < i - l + 1):
                part.append(0.0)
            elif j <= i - l + 1:
                part.append(float(u @ Z[0][j]))
            else:
                part.append(float(u @ Z[l][j]))
        pending[i] = allreduce_async(part)
        # K6: the D-Lanczos update of x (Sec. 2.1)
        if i == l:
            eta[0] = gamma[0]
            zeta[0] = nu
            p = Z[0][0] / eta[0]
        elif i >= l + 1:
            m = i - l
            lam = delta[m - 1] / eta[m - 1]
            eta[m] = gamma[m] - lam * delta[m - 1]
            zeta[m] = -lam * zeta[m - 1]
            x = x + zeta[m - 1] * p
            p = (Z[0][m] - delta[m - 1] * p) / eta[m]
            xs.append(x.copy())
            if abs(zeta[m]) < rtol * nrm_b or m >= maxit:
                for t, work in pending.values():
                    work.wait()
                return xs, m, abs(zeta[m])
        i += 1
