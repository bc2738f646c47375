"""Seeded synthetic inputs shaped like the simulated data of arXiv 2106.09382.

This module draws data only: a true precision matrix Omega0 and n samples
X ~ N(0, Omega0^{-1}).  It holds none of the estimator's arithmetic (no
standardization, no Gram, no coordinate descent), so both the CPU oracle and
the CUDA path consume exactly the same arrays.

Numbering: numpy ``default_rng(seed)``; draws are taken in a fixed order
(graph, edge values, Gaussian noise) so every array is reproducible.

Sampling: with Omega0 = L L^T (Cholesky, FP64) the rows x^T = z^T L^{-1} with
z ~ N(0, I) have covariance (L L^T)^{-1} = Omega0^{-1}.

Generators (Section 5 describes the paper's own AR(2) and scale-free designs;
the sizes and value ranges follow the workloads this library is measured on):

    random_graph   Erdos-Renyi edges with probability `edge_prob`, values
                   +-U[lo, hi], diagonal = row |sum| + margin (diagonally
                   dominant, hence positive definite).
    ar1_extra      AR(1) precision for rho (tridiagonal) plus `n_extra` random
                   non-band edges, each +-U[lo, hi] with |value| added to both
                   endpoint diagonals (each added term is PSD).
    ar2            the paper's AR(2) design (0.45 on the first, 0.4 on the
                   second off-diagonal, diagonal 1).
    scale_free     Barabasi-Albert graph (m edges per new vertex), values by
                   the paper's four steps (uniform on [-1,-0.5] U [0.5,1], row
                   scaling by 1.25 x the absolute row sum, symmetrization,
                   magnitude floor 0.1).
    block_diag     `n_blocks` blocks, within-block edge probability, values
                   +-U[lo, hi], diagonal dominance margin.
    joint_ar1      two related precision matrices for the joint estimator:
                   one AR(1) band, extra edges shared by both, and extra
                   edges of each population's own.
    power_law      Barabasi-Albert graph (m edges per new vertex), values
                   +-U[lo, hi], diagonal dominance margin; kept sparse (edge
                   lists) for large p, sampled by sample_sparse.

Large sparse sampling (sample_sparse): a diagonally dominant Omega0 is the
sum of one rank-one term per edge, |v| (e_i + sign(v) e_j)(e_i + sign(v)
e_j)^T, and the diagonal margin, so Omega0 = B B^T with B sparse; y = B z
(z ~ N(0, I)) has covariance Omega0 and x = Omega0^{-1} y has covariance
Omega0^{-1}.  The sparse system is solved by conjugate gradients to a
relative residual of 1e-13 (torch on the given device; this is sampling, not
the estimator).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def _signed_uniform(rng, size, lo, hi):
    mag = rng.uniform(lo, hi, size=size)
    sgn = np.where(rng.random(size) < 0.5, -1.0, 1.0)
    return sgn * mag


def random_graph(p: int, edge_prob: float = 0.05, lo: float = 0.3, hi: float = 0.6,
                 margin: float = 0.5, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(p, 1)
    keep = rng.random(iu.size) < edge_prob
    iu, ju = iu[keep], ju[keep]
    vals = _signed_uniform(rng, iu.size, lo, hi)
    Om = np.zeros((p, p))
    Om[iu, ju] = vals
    Om[ju, iu] = vals
    np.fill_diagonal(Om, np.abs(Om).sum(axis=1) + margin)
    return Om


def ar1_extra(p: int, rho: float = 0.5, n_extra: int | None = None, lo: float = 0.3,
              hi: float = 0.6, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    if n_extra is None:
        n_extra = int(round(0.01 * (p - 1)))
    c = 1.0 / (1.0 - rho * rho)
    Om = np.zeros((p, p))
    idx = np.arange(p)
    Om[idx, idx] = c * (1.0 + rho * rho)
    Om[0, 0] = c
    Om[p - 1, p - 1] = c
    Om[idx[:-1], idx[1:]] = -c * rho
    Om[idx[1:], idx[:-1]] = -c * rho
    chosen = set()
    while len(chosen) < n_extra:
        i, j = (int(v) for v in rng.integers(0, p, size=2))
        if i == j:
            continue
        a, b = min(i, j), max(i, j)
        if b - a <= 1 or (a, b) in chosen:
            continue
        chosen.add((a, b))
    for (a, b) in sorted(chosen):
        v = float(_signed_uniform(rng, 1, lo, hi)[0])
        Om[a, b] = v
        Om[b, a] = v
        Om[a, a] += abs(v)
        Om[b, b] += abs(v)
    return Om


def _extra_edges(rng, p: int, count: int, taken: set) -> list:
    """`count` distinct non-band pairs (a < b, b - a > 1) not in `taken`."""
    if count > (p - 1) * (p - 2) // 2 - len(taken):
        raise ValueError("p = %d has too few non-band pairs for %d more edges" % (p, count))
    out = []
    while len(out) < count:
        i, j = (int(v) for v in rng.integers(0, p, size=2))
        a, b = min(i, j), max(i, j)
        if b - a <= 1 or (a, b) in taken:
            continue
        taken.add((a, b))
        out.append((a, b))
    return out


def joint_ar1(p: int, rho: float = 0.5, n_shared: int | None = None,
              n_own: int | None = None, lo: float = 0.3, hi: float = 0.6, seed: int = 0):
    """Two precision matrices (Om1, Om2) with a common AR(1) band (as
    ar1_extra), n_shared extra edges present in both with the same value,
    and n_own extra edges in each one alone; every extra edge adds |value| to
    both endpoint diagonals (a PSD term), so both stay positive definite.
    Defaults: n_shared = n_own = round(0.01 (p - 1))."""
    rng = np.random.default_rng(seed)
    if n_shared is None:
        n_shared = int(round(0.01 * (p - 1)))
    if n_own is None:
        n_own = int(round(0.01 * (p - 1)))
    base = ar1_extra(p, rho, 0, lo, hi, seed)
    taken: set = set()
    shared = _extra_edges(rng, p, n_shared, taken)
    own = [_extra_edges(rng, p, n_own, taken) for _ in range(2)]
    out = []
    vs = _signed_uniform(rng, len(shared), lo, hi)
    for m in range(2):
        Om = base.copy()
        vo = _signed_uniform(rng, len(own[m]), lo, hi)
        for (a, b), v in list(zip(shared, vs)) + list(zip(own[m], vo)):
            Om[a, b] = Om[b, a] = v
            Om[a, a] += abs(v)
            Om[b, b] += abs(v)
        out.append(Om)
    return out[0], out[1]


def ar2(p: int) -> np.ndarray:
    Om = np.eye(p)
    i = np.arange(p)
    Om[i[:-1], i[1:]] = Om[i[1:], i[:-1]] = 0.45
    Om[i[:-2], i[2:]] = Om[i[2:], i[:-2]] = 0.4
    return Om


def barabasi_albert_edges(p: int, m: int, rng) -> list[tuple[int, int]]:
    """Preferential attachment: start from a clique on m+1 vertices, then every
    new vertex attaches to m distinct existing vertices drawn with probability
    proportional to degree."""
    edges = []
    targets_pool: list[int] = []
    for a in range(m + 1):
        for b in range(a + 1, m + 1):
            edges.append((a, b))
            targets_pool += [a, b]
    for v in range(m + 1, p):
        picked: set[int] = set()
        while len(picked) < m:
            picked.add(targets_pool[int(rng.integers(0, len(targets_pool)))])
        for u in sorted(picked):
            edges.append((u, v))
            targets_pool += [u, v]
    return edges


def scale_free(p: int, m: int = 2, seed: int = 0, margin: float = 0.1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    edges = barabasi_albert_edges(p, m, rng)
    T = np.eye(p)
    for (a, b) in edges:
        v = float(_signed_uniform(rng, 1, 0.5, 1.0)[0])
        T[a, b] = T[b, a] = v
    off = T - np.diag(np.diag(T))
    rowsum = np.abs(off).sum(axis=1)
    rowsum[rowsum == 0] = 1.0
    off = off / (1.25 * rowsum[:, None])
    Om = (off + off.T) / 2.0
    mask = Om != 0
    small = mask & (np.abs(Om) < 0.1)
    Om[small] = 0.1 * np.sign(Om[small])
    # the recipe's unit diagonal does not make the matrix positive definite
    # once hubs are symmetrised; raise it to diagonal dominance with `margin`
    diag = np.maximum(1.0, np.abs(Om).sum(axis=1) + margin)
    Om[np.diag_indices(p)] = diag
    return Om


def block_diag(p: int, n_blocks: int, edge_prob: float = 0.1, lo: float = 0.3,
               hi: float = 0.6, margin: float = 0.5, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    Om = np.zeros((p, p))
    bs = p // n_blocks
    for b in range(n_blocks):
        s = b * bs
        e = p if b == n_blocks - 1 else s + bs
        k = e - s
        iu, ju = np.triu_indices(k, 1)
        keep = rng.random(iu.size) < edge_prob
        vals = _signed_uniform(rng, int(keep.sum()), lo, hi)
        Om[s + iu[keep], s + ju[keep]] = vals
        Om[s + ju[keep], s + iu[keep]] = vals
    np.fill_diagonal(Om, np.abs(Om).sum(axis=1) + margin)
    return Om


def sample(Om0: np.ndarray, n: int, seed: int = 0) -> np.ndarray:
    """n rows x ~ N(0, Om0^{-1}) as an (n, p) float64 array."""
    rng = np.random.default_rng(seed + 1_000_003)
    p = Om0.shape[0]
    L = np.linalg.cholesky(Om0)
    Z = rng.standard_normal((n, p))
    # X = Z L^{-1}  <=>  L^T X^T = Z^T
    Xt = sla.solve_triangular(L, Z.T, trans="T", lower=True, check_finite=False)
    return np.ascontiguousarray(Xt.T)


# Named workloads -------------------------------------------------------------

def workload_small(seed: int = 0):
    """p=100, n=200, random graph (edge prob 0.05, +-U[0.3,0.6], margin 0.5),
    lambda=0.3, tol 1e-6."""
    Om0 = random_graph(100, 0.05, 0.3, 0.6, 0.5, seed)
    return dict(name="random-graph p=100 n=200", X=sample(Om0, 200, seed), Om0=Om0,
                lam=0.3, tol=1e-6)


def workload_ar1(p: int = 5000, n: int = 2000, seed: int = 0):
    """AR(1) rho=0.5 precision plus round(0.01 (p-1)) extra edges, lambda=0.2."""
    Om0 = ar1_extra(p, 0.5, None, 0.3, 0.6, seed)
    return dict(name="AR(1)+1%% extra p=%d n=%d" % (p, n), X=sample(Om0, n, seed), Om0=Om0,
                lam=0.2, tol=1e-5)


def workload_path(p: int = 1000, n: int = 800, seed: int = 0):
    """Regularisation-path / stability-selection workload: a scale-free
    (Barabasi-Albert, m = 2) precision matrix, n samples."""
    Om0 = scale_free(p, m=2, seed=seed)
    return {"Om0": Om0, "X": sample(Om0, n, seed=seed + 1), "p": p, "n": n}


def subsamples(n: int, count: int = 64, lo: int = 200, hi: int = 800, seed: int = 0):
    """`count` row subsets of range(n), sizes uniform on [lo, min(hi, n)],
    drawn without replacement, each sorted."""
    rng = np.random.default_rng(seed)
    hi = min(hi, n)
    sizes = rng.integers(lo, hi + 1, size=count)
    return [np.sort(rng.choice(n, size=int(m), replace=False)) for m in sizes]


def workload_joint(p: int = 1000, n: int = 500, seed: int = 0):
    """Joint two-population workload: joint_ar1(p) with n samples drawn
    independently from each population; lambda1 = 0.2, lambda2 = 0.05."""
    Om1, Om2 = joint_ar1(p, seed=seed)
    return {"Om0": (Om1, Om2), "X1": sample(Om1, n, seed), "X2": sample(Om2, n, seed + 11),
            "p": p, "n": n, "lam1": 0.2, "lam2": 0.05, "tol": 1e-5}


def workload_adjoint(p: int = 2000, n_train: int = 1000, n_val: int = 500, seed: int = 0):
    """Differentiable-solve workload: a block-diagonal precision matrix (20
    blocks, within-block edge probability 0.1, values +-U[0.3, 0.6], margin
    0.5), n_train training rows and n_val held-out rows drawn independently."""
    Om0 = block_diag(p, 20, 0.1, 0.3, 0.6, 0.5, seed)
    return {"Om0": Om0, "X": sample(Om0, n_train, seed), "X_val": sample(Om0, n_val, seed + 7),
            "p": p, "n": n_train, "n_val": n_val}


def power_law(p: int, m: int = 2, lo: float = 0.2, hi: float = 0.5, margin: float = 0.5,
              seed: int = 0):
    """Sparse power-law precision matrix: Barabasi-Albert edges (i < j), values
    +-U[lo, hi], diagonal = absolute row sum + margin.  Returns (i, j, v, diag)."""
    rng = np.random.default_rng(seed)
    edges = np.array(barabasi_albert_edges(p, m, rng), dtype=np.int64)
    ei, ej = np.minimum(edges[:, 0], edges[:, 1]), np.maximum(edges[:, 0], edges[:, 1])
    v = _signed_uniform(rng, len(ei), lo, hi)
    diag = np.full(p, float(margin))
    np.add.at(diag, ei, np.abs(v))
    np.add.at(diag, ej, np.abs(v))
    return ei, ej, v, diag


def sample_sparse(ei, ej, v, diag, n: int, seed: int = 0, device="cuda", dtype=None):
    """n rows x ~ N(0, Omega0^{-1}) for the sparse diagonally dominant Omega0
    given by its upper edges (ei < ej, values v) and diagonal; returns an
    (n, p) torch tensor on `device` (FP64 unless dtype is given)."""
    import torch
    p = len(diag)
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed) + 2_000_003)
    f64 = torch.float64
    ei_t = torch.as_tensor(ei, device=dev)
    ej_t = torch.as_tensor(ej, device=dev)
    v_t = torch.as_tensor(v, dtype=f64, device=dev)
    rest = torch.as_tensor(diag, dtype=f64, device=dev)
    rest = rest - torch.zeros(p, dtype=f64, device=dev).index_add_(0, ei_t, v_t.abs()) \
        .index_add_(0, ej_t, v_t.abs())
    # y = B z, columns of y are samples (p x n)
    Y = torch.randn((p, n), generator=g, dtype=f64, device=dev) * rest.clamp_min(0).sqrt()[:, None]
    ze = torch.randn((len(ei), n), generator=g, dtype=f64, device=dev) * v_t.abs().sqrt()[:, None]
    Y.index_add_(0, ei_t, ze)
    Y.index_add_(0, ej_t, ze * torch.sign(v_t)[:, None])
    del ze
    rows = torch.cat([ei_t, ej_t, torch.arange(p, device=dev)])
    cols = torch.cat([ej_t, ei_t, torch.arange(p, device=dev)])
    vals = torch.cat([v_t, v_t, torch.as_tensor(diag, dtype=f64, device=dev)])
    A = torch.sparse_coo_tensor(torch.stack([rows, cols]), vals, (p, p),
                                check_invariants=False).coalesce()
    # conjugate gradients on A X = Y, all columns at once (Jacobi preconditioner)
    dinv = 1.0 / torch.as_tensor(diag, dtype=f64, device=dev)[:, None]
    X = torch.zeros_like(Y)
    R = Y.clone()
    Zr = R * dinv
    P = Zr.clone()
    rz = (R * Zr).sum(0)
    ynorm = Y.norm(dim=0)
    for _ in range(10000):
        AP = torch.sparse.mm(A, P)
        alpha = rz / (P * AP).sum(0)
        X += alpha * P
        R -= alpha * AP
        if (R.norm(dim=0) <= 1e-13 * ynorm).all():
            break
        Zr = R * dinv
        rz_new = (R * Zr).sum(0)
        P = Zr + (rz_new / rz) * P
        rz = rz_new
    out = X.t().contiguous()
    return out if dtype is None else out.to(dtype)


def workload_large(p: int = 20000, n: int = 5000, seed: int = 0, device="cuda"):
    """Large sparse solve: power-law precision (Barabasi-Albert m = 2, average
    degree 4, +-U[0.2, 0.5], margin 0.5), n samples in FP32 on `device`,
    lambda = 0.15, tol 1e-5."""
    import torch
    ei, ej, v, diag = power_law(p, 2, 0.2, 0.5, 0.5, seed)
    X = sample_sparse(ei, ej, v, diag, n, seed, device, dtype=torch.float32)
    return {"X": X, "edges": (ei, ej, v), "diag": diag, "p": p, "n": n, "lam": 0.15, "tol": 1e-5}
