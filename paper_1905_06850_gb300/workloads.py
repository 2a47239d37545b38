"""Seeded synthetic workloads for the p(l)-CG solver.

This module builds INPUTS only: operator descriptions, right-hand sides and
request streams.  It holds none of the solver's arithmetic and imports
neither the CUDA library nor the test oracle; both consume what it returns.

Operator descriptions are plain dicts:

* ``{"kind": "stencil", "dim": 2|3, "nx", "ny", "nz", "center", "off"}`` --
  Dirichlet 5-point (2D) / 7-point (3D) constant-coefficient stencil, unknowns
  in lexicographic order with x fastest.  ``center`` includes any diagonal
  shift ``c`` (the shifted Poisson systems of the batched workload).
* ``{"kind": "csr", "n", "rowptr" int64[n+1], "col" int32[nnz], "val"
  float64[nnz]}`` -- general sparse SPD matrix, column indices sorted per row.

The paper (Sec. 4) measures PETSc examples (a 2D 5-point Laplacian, a
diagonal matrix with the same spectrum, and an ice-sheet FE problem); the
workloads below are synthetic stand-ins with the shapes of those problems
and of the benchmark configurations:

1. 2D 5-point Laplacian 100x100, x* ~ U[-1,1] (seed 1), b = A x*.
2. 3D 7-point Laplacian 256^3, x* ~ N(0,1) (seed 2), b = A x*.
3. 27-point heterogeneous-diffusion operator on 128^3 in CSR, cell
   coefficients kappa = exp(N(0,1)) (seed 3), x* ~ N(0,1).
4. 4096 shifted 2D Poisson systems, side s ~ U{16..256}, shift c ~ U[0,1],
   b ~ N(0,1) per system.
5. A Poisson-arrival request stream (rate 2000/s, seed 5), n log-uniform in
   [1e3, 4e6], operator type uniform over {2D stencil, 3D stencil, random
   sparse SPD CSR}.
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# Operators
# ---------------------------------------------------------------------------


def stencil2d(nx: int, ny: int, center: float = 4.0, off: float = -1.0,
              shift: float = 0.0) -> dict:
    """2D Dirichlet 5-point stencil; the Laplacian is (4, -1)."""
    return {"kind": "stencil", "dim": 2, "nx": int(nx), "ny": int(ny), "nz": 1,
            "center": float(center) + float(shift), "off": float(off)}


def stencil3d(nx: int, ny: int, nz: int, center: float = 6.0, off: float = -1.0,
              shift: float = 0.0) -> dict:
    """3D Dirichlet 7-point stencil; the Laplacian is (6, -1)."""
    return {"kind": "stencil", "dim": 3, "nx": int(nx), "ny": int(ny), "nz": int(nz),
            "center": float(center) + float(shift), "off": float(off)}


def op_size(op: dict) -> int:
    if op["kind"] == "stencil":
        return int(op["nx"]) * int(op["ny"]) * (int(op["nz"]) if op["dim"] == 3 else 1)
    if op["kind"] == "var27":
        return int(op["nx"]) * int(op["ny"]) * int(op["nz"])
    return int(op["n"])


def stencil_spectrum_bounds(op: dict) -> tuple[float, float]:
    """Closed-form extreme eigenvalues of a constant-coefficient Dirichlet
    stencil: center + 2*off*cos(pi/(n_d+1)) summed over the axes, largest
    with the sign flipped (separable Kronecker sum)."""
    dims = [op["nx"], op["ny"]] + ([op["nz"]] if op["dim"] == 3 else [])
    c, o = op["center"], op["off"]
    lo = c + sum(2 * o * math.cos(math.pi / (d + 1)) for d in dims)
    hi = c - sum(2 * o * math.cos(math.pi / (d + 1)) for d in dims)
    return min(lo, hi), max(lo, hi)


def shift_interval(op: dict) -> tuple[float, float]:
    """The interval [lmin, lmax] the Chebyshev shifts are placed on.

    Stencils: [c, center + 2*dim*|off|] with c = the diagonal shift
    ([0, 8] for the 2D Laplacian, [0, 12] for the 3D one, [c, 8 + c] for the
    shifted systems).  CSR: [0, Gershgorin bound]."""
    if op["kind"] == "stencil":
        base = 4.0 if op["dim"] == 2 else 6.0
        shift = op["center"] - base
        return (max(0.0, shift), op["center"] + 2 * op["dim"] * abs(op["off"]))
    if op["kind"] == "var27":
        op = var27_to_csr(op)
    rowsum = np.add.reduceat(np.abs(op["val"]), op["rowptr"][:-1]) \
        if op["val"].size else np.zeros(op["n"])
    return (0.0, float(rowsum.max()))


def jacobi_shift_interval(op: dict) -> tuple[float, float]:
    """The shift interval for the Jacobi-preconditioned operator diag(A)^{-1} A:
    [0, max_i sum_j |a_ij| / a_ii] (Gershgorin; <= 2 for a diagonally
    dominant A, the [0, 2] of the paper's preconditioned experiments).
    Constant-coefficient stencils: shift_interval divided by the center."""
    if op["kind"] == "stencil":
        lo, hi = shift_interval(op)
        return lo / op["center"], hi / op["center"]
    if op["kind"] == "var27":
        op = var27_to_csr(op)
    val, rowptr = op["val"], op["rowptr"]
    n = op["n"]
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    diag = np.zeros(n)
    np.add.at(diag, rows[op["col"] == rows], val[op["col"] == rows])
    rowsum = np.add.reduceat(np.abs(val), rowptr[:-1]) if val.size else np.zeros(n)
    return 0.0, float((rowsum / diag).max())


# The 13 "forward" neighbour offsets (dz, dy, dx) of a 27-point stencil, in
# lexicographic order: the structured operator stores the weight to each of
# them per cell; the weight to c - d is the neighbour's weight to c (symmetry).
VAR27_FORWARD = [(0, 0, 1), (0, 1, -1), (0, 1, 0), (0, 1, 1),
                 (1, -1, -1), (1, -1, 0), (1, -1, 1), (1, 0, -1), (1, 0, 0), (1, 0, 1),
                 (1, 1, -1), (1, 1, 0), (1, 1, 1)]


def _hetero27_entries(nx: int, ny: int, nz: int, seed: int, sigma: float):
    """Entries of the 27-point heterogeneous-diffusion operator: for each of
    the 27 offsets (dz, dy, dx) the (nz, ny, nx) array of A[c, c + d] (the
    diagonal for (0, 0, 0)) and the mask of in-grid neighbours."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    kappa = np.exp(sigma * rng.standard_normal(n))
    k3 = kappa.reshape(nz, ny, nx)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    offsets = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    masks, entries = {}, {}
    diag = np.zeros((nz, ny, nx))
    for dz, dy, dx in offsets:
        if (dz, dy, dx) == (0, 0, 0):
            continue
        s = 1.0 / (abs(dz) + abs(dy) + abs(dx))
        valid = ((iz + dz >= 0) & (iz + dz < nz) & (iy + dy >= 0) & (iy + dy < ny)
                 & (ix + dx >= 0) & (ix + dx < nx))
        kd = np.roll(k3, shift=(-dz, -dy, -dx), axis=(0, 1, 2))
        kd = np.where(valid, kd, k3)
        w = s * 2.0 * (k3 * kd) / (k3 + kd)   # symmetric in (c, d) bit for bit
        diag += w
        masks[(dz, dy, dx)] = valid
        entries[(dz, dy, dx)] = -w
    masks[(0, 0, 0)] = np.ones((nz, ny, nx), dtype=bool)
    entries[(0, 0, 0)] = diag
    return offsets, masks, entries


def hetero27_csr(nx: int, ny: int, nz: int, seed: int = 3, sigma: float = 1.0) -> dict:
    """27-point heterogeneous-diffusion SPD operator in CSR.

    Cell coefficients kappa_c = exp(N(0, sigma^2)).  For each of the 26
    neighbours d of cell c the edge weight is w = s * 2 k_c k_d / (k_c + k_d)
    (harmonic mean) with s = 1, 1/2, 1/3 for face, edge and corner
    neighbours.  A_cd = -w; A_cc = the sum of all 26 weights, where a
    neighbour outside the grid takes k_d = k_c and stays on the diagonal
    only (Dirichlet).  The result is a symmetric, irreducibly diagonally
    dominant M-matrix, hence SPD."""
    n = nx * ny * nz
    offsets, masks, entries = _hetero27_entries(nx, ny, nz, seed, sigma)
    counts = sum(masks[o].astype(np.int64) for o in offsets).ravel()
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    nnz = int(rowptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    cursor = rowptr[:-1].copy()
    lin = np.arange(n, dtype=np.int64)
    for dz, dy, dx in offsets:
        mf = masks[(dz, dy, dx)].ravel()
        pos = cursor[mf]
        col[pos] = (lin[mf] + (dz * ny + dy) * nx + dx).astype(np.int32)
        val[pos] = entries[(dz, dy, dx)].ravel()[mf]
        cursor[mf] += 1
    return {"kind": "csr", "n": n, "rowptr": rowptr, "col": col, "val": val}


def hetero27_var27(nx: int, ny: int, nz: int, seed: int = 3, sigma: float = 1.0) -> dict:
    """The same operator as hetero27_csr (same seed: the same matrix, entry for
    entry) in the structured variable-coefficient layout: coef[0] = the
    diagonal, coef[1 + k] = A[c, c + VAR27_FORWARD[k]] (0 where that neighbour
    is outside the grid), each a length-n array in lexicographic order."""
    n = nx * ny * nz
    _, masks, entries = _hetero27_entries(nx, ny, nz, seed, sigma)
    coef = np.zeros((14, n))
    coef[0] = entries[(0, 0, 0)].ravel()
    for k, o in enumerate(VAR27_FORWARD):
        coef[1 + k] = np.where(masks[o], entries[o], 0.0).ravel()
    return {"kind": "var27", "nx": nx, "ny": ny, "nz": nz, "coef": coef}


def var27_to_csr(op: dict) -> dict:
    """CSR form of a structured 27-point operator (forward weights, their
    symmetric partners and the diagonal; entries to cells outside the grid
    dropped), columns sorted per row."""
    import scipy.sparse as sp
    nx, ny, nz = op["nx"], op["ny"], op["nz"]
    n = nx * ny * nz
    coef = op["coef"]
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    iz, iy, ix = iz.ravel(), iy.ravel(), ix.ravel()
    lin = np.arange(n)
    rows, cols, vals = [lin], [lin], [coef[0]]
    for k, (dz, dy, dx) in enumerate(VAR27_FORWARD):
        valid = ((iz + dz < nz) & (iy + dy >= 0) & (iy + dy < ny) & (ix + dx >= 0) & (ix + dx < nx))
        c = lin[valid]
        d = c + (dz * ny + dy) * nx + dx
        w = coef[1 + k][valid]
        rows += [c, d]
        cols += [d, c]
        vals += [w, w]
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    A.sort_indices()
    return {"kind": "csr", "n": n, "rowptr": A.indptr.astype(np.int64),
            "col": A.indices.astype(np.int32), "val": A.data.astype(np.float64)}


def random_spd_csr(n: int, seed: int, nnz_lo: int = 5, nnz_hi: int = 30) -> dict:
    """Random-sparsity SPD CSR: per row k ~ U{nnz_lo..nnz_hi} target nonzeros;
    (k-1)//2 random partner columns per row with values -U(0,1); the pattern
    and values are symmetrised (A_off + A_off^T, duplicates summed, self-loops
    dropped); the diagonal is the absolute off-diagonal row sum times
    (1 + U(0.05, 0.5)), so A is strictly diagonally dominant, hence SPD."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    k = rng.integers(nnz_lo, nnz_hi + 1, size=n)
    per = (k - 1) // 2
    rows = np.repeat(np.arange(n, dtype=np.int64), per)
    cols = rng.integers(0, n, size=rows.size, dtype=np.int64)
    vals = -rng.uniform(0.0, 1.0, size=rows.size)
    keep = rows != cols
    off = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n, n)).tocsr()
    off = (off + off.T).tocsr()
    off.sum_duplicates()
    rowabs = np.asarray(abs(off).sum(axis=1)).ravel()
    dvals = rowabs * (1.0 + rng.uniform(0.05, 0.5, size=n))
    dvals[dvals == 0] = 1.0
    A = (off + sp.diags(dvals)).tocsr()
    A.sort_indices()
    return {"kind": "csr", "n": n, "rowptr": A.indptr.astype(np.int64),
            "col": A.indices.astype(np.int32), "val": A.data.astype(np.float64)}


def fp32_rounded(op: dict) -> dict:
    """The operator the FP32 path solves with: every coefficient rounded to
    FP32 (and widened back to FP64 for the FP64 oracle)."""
    out = dict(op)
    if op["kind"] == "stencil":
        out["center"] = float(np.float32(op["center"]))
        out["off"] = float(np.float32(op["off"]))
    elif op["kind"] == "var27":
        out["coef"] = op["coef"].astype(np.float32).astype(np.float64)
    else:
        out["val"] = op["val"].astype(np.float32).astype(np.float64)
    return out


def to_scipy(op: dict):
    """A scipy.sparse CSR matrix of the operator (library construction:
    Kronecker sums for stencils), used to form right-hand sides."""
    import scipy.sparse as sp
    if op["kind"] == "var27":
        op = var27_to_csr(op)
    if op["kind"] == "csr":
        n = op["n"]
        return sp.csr_matrix((op["val"], op["col"], op["rowptr"]), shape=(n, n))

    def lap1(m):
        return sp.diags([np.ones(m - 1), np.ones(m - 1)], [-1, 1], format="csr")

    dims = [op["nx"], op["ny"]] + ([op["nz"]] if op["dim"] == 3 else [])
    n = int(np.prod(dims))
    S = sp.csr_matrix((n, n))
    for a, m in enumerate(dims):
        mats = [sp.identity(d, format="csr") for d in dims]
        mats[a] = lap1(m)
        K = mats[0]
        for M in mats[1:]:
            K = sp.kron(M, K, format="csr")   # x fastest: later axes are outer factors
        S = S + K
    return (op["off"] * S + op["center"] * sp.identity(n, format="csr")).tocsr()


def rhs(op: dict, xstar: np.ndarray) -> np.ndarray:
    """b = A x* in FP64 (scipy.sparse for CSR; array shifts for stencils)."""
    if op["kind"] in ("csr", "var27"):
        return to_scipy(op) @ xstar
    dims = (op["nz"], op["ny"], op["nx"]) if op["dim"] == 3 else (op["ny"], op["nx"])
    X = xstar.reshape(dims)
    Y = op["center"] * X
    nb = np.zeros_like(X)
    for ax in range(X.ndim):
        sl_lo = [slice(None)] * X.ndim
        sl_hi = [slice(None)] * X.ndim
        sl_lo[ax] = slice(0, -1)
        sl_hi[ax] = slice(1, None)
        nb[tuple(sl_lo)] += X[tuple(sl_hi)]
        nb[tuple(sl_hi)] += X[tuple(sl_lo)]
    return (Y + op["off"] * nb).ravel()


# ---------------------------------------------------------------------------
# Benchmark configurations
# ---------------------------------------------------------------------------


def config_2d(nx: int = 100, seed: int = 1) -> dict:
    """2D 5-point Laplacian, x* ~ U[-1,1], b = A x*, x0 = 0, shifts on [0, 8]."""
    op = stencil2d(nx, nx)
    xs = np.random.default_rng(seed).uniform(-1.0, 1.0, op_size(op))
    return {"op": op, "b": rhs(op, xs), "xstar": xs, "interval": (0.0, 8.0), "rtol": 1e-6}


def config_3d(nx: int = 256, seed: int = 2) -> dict:
    """3D 7-point Laplacian, x* ~ N(0,1), b = A x*, x0 = 0, shifts on [0, 12]."""
    op = stencil3d(nx, nx, nx)
    xs = np.random.default_rng(seed).standard_normal(op_size(op))
    return {"op": op, "b": rhs(op, xs), "xstar": xs, "interval": (0.0, 12.0), "rtol": 1e-8}


def config_hetero27(nx: int = 128, seed: int = 3) -> dict:
    """27-point heterogeneous CSR, FP32-rounded values, x* ~ N(0,1)."""
    op = fp32_rounded(hetero27_csr(nx, nx, nx, seed=seed))
    xs = np.random.default_rng(seed + 1000).standard_normal(op["n"])
    return {"op": op, "b": rhs(op, xs), "xstar": xs, "interval": shift_interval(op),
            "rtol": 1e-8}


def e3_diagonal(nx: int = 100, seed: int = 1) -> dict:
    """The paper's communication-bound toy (Sec. 4, Fig. "lapl", right): a
    diagonal ("one-point stencil") operator carrying the nx^2 eigenvalues of
    the 2D 5-point Laplacian, lambda_jk = 4 - 2 cos(j pi/(nx+1)) -
    2 cos(k pi/(nx+1)) in (k, j) = (y, x) order, with the right-hand side
    rotated into that eigenbasis: b_diag = Q^T b where Q is the orthonormal
    DST-I basis (scipy.fft.dstn, norm "ortho") and b = A x* of config_2d.  It
    has the Laplacian's spectrum and residual history, with an SpMV that is
    one multiply per row.  Returns op (CSR, one entry per row), b, the
    Laplacian's b, interval."""
    import scipy.fft
    lap = config_2d(nx=nx, seed=seed)
    j = np.arange(1, nx + 1)
    lam1 = 2.0 - 2.0 * np.cos(j * np.pi / (nx + 1))
    lam = (lam1[:, None] + lam1[None, :]).ravel()
    n = nx * nx
    op = {"kind": "csr", "n": n, "rowptr": np.arange(n + 1, dtype=np.int64),
          "col": np.arange(n, dtype=np.int32), "val": lam}
    bt = scipy.fft.dstn(lap["b"].reshape(nx, nx), type=1, norm="ortho").ravel()
    return {"op": op, "b": bt, "b_laplacian": lap["b"], "interval": (0.0, 8.0),
            "rtol": 1e-6}


def config_hetero27_var27(nx: int = 128, seed: int = 3) -> dict:
    """The 27-point heterogeneous operator of config_hetero27 (FP32-rounded
    values, the same x* and b) in the structured layout."""
    op = fp32_rounded(hetero27_var27(nx, nx, nx, seed=seed))
    xs = np.random.default_rng(seed + 1000).standard_normal(op_size(op))
    return {"op": op, "b": rhs(op, xs), "xstar": xs, "rtol": 1e-8}


def batched_systems(count: int = 4096, s_lo: int = 16, s_hi: int = 256, seed: int = 4):
    """The batched workload: ``count`` shifted 2D Poisson systems.  Returns a
    list of dicts with op (FP32-rounded coefficients), b, interval, side, c."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(s_lo, s_hi + 1, size=count)
    cs = rng.uniform(0.0, 1.0, size=count)
    return [_batched_one(seed, idx, int(sides[idx]), float(cs[idx])) for idx in range(count)]


def batched_system(index: int, count: int = 4096, s_lo: int = 16, s_hi: int = 256, seed: int = 4) -> dict:
    """System ``index`` of batched_systems(count, ...), built alone."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(s_lo, s_hi + 1, size=count)
    cs = rng.uniform(0.0, 1.0, size=count)
    return _batched_one(seed, index, int(sides[index]), float(cs[index]))


def _batched_one(seed: int, idx: int, side: int, c: float) -> dict:
    op = fp32_rounded(stencil2d(side, side, shift=c))
    b = np.random.default_rng([seed, idx]).standard_normal(op_size(op))
    return {"op": op, "b": b, "interval": (c, 8.0 + c), "side": side, "c": c}


def serving_stream(duration_s: float = 1.0, rate: float = 2000.0, n_lo: float = 1e3,
                   n_hi: float = 4e6, seed: int = 5, max_requests: int | None = None):
    """Poisson request stream: arrival times (s), and for each request a size
    n log-uniform in [n_lo, n_hi] and a type in {"2d", "3d", "csr"}.  The
    operator is realised lazily by ``serving_request`` so that the stream can
    be described without building every matrix."""
    rng = np.random.default_rng(seed)
    t, reqs = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration_s or (max_requests is not None and len(reqs) >= max_requests):
            break
        n = float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        kind = ("2d", "3d", "csr")[int(rng.integers(0, 3))]
        reqs.append({"t": t, "n_target": n, "type": kind, "seed": int(rng.integers(0, 2**31 - 1))})
    return reqs


def serving_request(req: dict) -> dict:
    """Build the operator and right-hand side of one request of the stream."""
    rng = np.random.default_rng(req["seed"])
    n = req["n_target"]
    if req["type"] == "2d":
        s = max(4, int(round(math.sqrt(n))))
        op = fp32_rounded(stencil2d(s, s))
    elif req["type"] == "3d":
        s = max(4, int(round(n ** (1.0 / 3.0))))
        op = fp32_rounded(stencil3d(s, s, s))
    else:
        op = fp32_rounded(random_spd_csr(max(16, int(round(n))), seed=req["seed"]))
    b = rng.standard_normal(op_size(op))
    return {"op": op, "b": b, "interval": shift_interval(op)}
