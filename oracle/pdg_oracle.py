"""FP64 CPU oracle of the per-iteration step of Preconditioned Deformation Grids
(arXiv 2509.18097).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this module;
it is used by `tests/`, by `__graft_entry__.smoke()` and by the `cpu_baseline` /
`--impl reference` legs of `bench.py`.  It shares no code with the CUDA path: it is a
plain, slow re-statement of what the paper defines, written in numpy float64, with
library primitives (scipy's k-d tree as a candidate generator, numpy reductions) used
only as steps whose result is then checked exactly.

Every function cites the passage it follows.  Where the paper is silent or garbled the
oracle takes one reading, stated at the function that depends on it: a 3-float
displacement payload per grid vertex (Sec. 3.1/3.3), levels whose vertices are aligned with
the domain corners and points clamped to the domain (Eq. 1), the free-boundary unit-weight
6-neighbour graph Laplacian (Sec. 3.2), the raw gradient preconditioned and then fed to
Adam (Sec. 3.2 Eq. 3 with Sec. 3.6), a differentiated robust weight (Sec. 3.4), the
lowest index winning a nearest-neighbour tie, sgn(0) = 0 at the isometry kink, and every
frame starting from zero grids and fresh Adam state.

Layout conventions (shared only as *conventions* with the CUDA path):
  * a level with n vertices per axis is an array [n, n, n, 3] indexed [z, y, x, channel],
    i.e. vertex (i, j, k) = (x, y, z) has flat index (k * n + j) * n + i;
  * the level's vertices sit at lo + (hi - lo) * i / (n - 1) (corners aligned);
  * points are [N, 3] arrays.
"""
from __future__ import annotations

import dataclasses

import numpy as np

F64 = np.float64

# ---------------------------------------------------------------------------------------
# hyper-parameters printed in the paper (Sec. 3.4 and Sec. 3.6)
# ---------------------------------------------------------------------------------------

ALPHA = 5.56  # robust Chamfer Gaussian weight, Sec. 3.4 (w_R)
W_ISO = 250.0  # isometry weight, Sec. 3.4 (total loss)
LR0 = 5e-3  # coarsest-level learning rate, Sec. 3.6
LR_GROWTH = 1.1  # +10 % per finer level, Sec. 3.6
LAMBDA0 = 0.25  # coarsest-level smoothness weight, Sec. 3.6
LAMBDA_GROWTH = 1.5  # +50 % per finer level, Sec. 3.6
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8  # Adam defaults, Sec. 3.6
NO_PRECOND_LR_FACTOR = 0.1  # ablation: lr x 0.1 without preconditioning, Sec. 4 (key components)


@dataclasses.dataclass
class Config:
    """Per-frame optimisation settings (defaults = the paper's values, Sec. 3.4/3.6)."""

    res: tuple = (8, 16, 32)  # vertices per axis per level, coarse -> fine
    lo: tuple = (-1.5, -1.5, -1.5)
    hi: tuple = (1.5, 1.5, 1.5)
    alpha: float = ALPHA
    w_chamfer_mesh: float = 1.0  # w_confidence of the mesh term (1 for a single frame)
    w_chamfer_pts: float = 1.0
    w_iso: float = W_ISO
    lr0: float = LR0
    lr_growth: float = LR_GROWTH
    lambda0: float = LAMBDA0
    lambda_growth: float = LAMBDA_GROWTH
    beta1: float = BETA1
    beta2: float = BETA2
    eps: float = EPS
    precondition: bool = True
    robust_weight_stopgrad: bool = False
    payload: str = "displacement"  # or "cayley": the 6-D rotation + translation of Sec. 3.3

    @property
    def channels(self) -> int:
        return 6 if self.payload == "cayley" else 3

    def lr(self, l: int) -> float:
        """Learning rate of level l (0 = coarsest), Sec. 3.6; x0.1 without preconditioning."""
        f = 1.0 if self.precondition else NO_PRECOND_LR_FACTOR
        return self.lr0 * self.lr_growth**l * f

    def lam(self, l: int) -> float:
        """Smoothness weight lambda of level l (0 = coarsest), Sec. 3.6."""
        return self.lambda0 * self.lambda_growth**l


# ---------------------------------------------------------------------------------------
# (a) multi-level trilinear evaluation, Sec. 3.1 Eq. 1
# ---------------------------------------------------------------------------------------


def level_coords(x, lo, hi, n):
    """Cell index and fractional offset of points x in a level with n vertices per axis.

    Eq. 1 interpolates trilinearly between the grid values around x.  Reading: the n
    vertices per axis span [lo, hi] with corners aligned; points outside are clamped to
    the border; the last cell is closed (i0 <= n - 2).  Returns (i0 int [N,3], f [N,3]).
    """
    x = np.asarray(x, F64)
    lo = np.asarray(lo, F64)
    hi = np.asarray(hi, F64)
    u = (x - lo) / (hi - lo) * (n - 1)
    u = np.clip(u, 0.0, n - 1)
    i0 = np.minimum(np.floor(u), max(n - 2, 0)).astype(np.int64)
    return i0, u - i0


def _corners(x, lo, hi, n):
    """The 8 (or 1, for n == 1) interpolation corners of each point: flat vertex index
    [N, K] and trilinear weight [N, K] (Eq. 1, w^{l,c})."""
    if n == 1:
        N = len(x)
        return np.zeros((N, 1), np.int64), np.ones((N, 1), F64)
    i0, f = level_coords(x, lo, hi, n)
    idx, wts = [], []
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                w = (f[:, 0] if dx else 1 - f[:, 0]) * (f[:, 1] if dy else 1 - f[:, 1]) * (f[:, 2] if dz else 1 - f[:, 2])
                v = ((i0[:, 2] + dz) * n + (i0[:, 1] + dy)) * n + (i0[:, 0] + dx)
                idx.append(v)
                wts.append(w)
    return np.stack(idx, 1), np.stack(wts, 1)


def eval_displacement(x, thetas, lo, hi):
    """u(x) = (1/L) sum_l sum_{c in N^l(x)} w^{l,c}(x) T^{l,c}   (Sec. 3.1, Eq. 1).

    Reading: levels are averaged (not residual), values live on grid vertices.  The payload
    has C channels: a 3-vector displacement (the default payload) or the 6-D Cayley
    rotation + translation of Sec. 3.3.
    thetas: list of [n, n, n, C] arrays.  Returns [N, C] float64.
    """
    x = np.asarray(x, F64)
    L = len(thetas)
    C = np.asarray(thetas[0]).shape[-1]
    u = np.zeros((len(x), C), F64)
    for th in thetas:
        n = th.shape[0]
        flat = np.asarray(th, F64).reshape(-1, C)
        idx, w = _corners(x, lo, hi, n)
        u += (w[:, :, None] * flat[idx]).sum(1)
    return u / L


def deform(x, thetas, lo, hi):
    """x_t = x_{t-1} + u_t(x_{t-1}): the recursive composition of Sec. 3.3 with a
    displacement payload (the rotation part is the identity)."""
    return np.asarray(x, F64) + eval_displacement(x, thetas, lo, hi)


def interp_adjoint(x, g_pts, res, lo, hi):
    """Adjoint of eval_displacement: dLoss/dT^l = (1/L) sum_p w^{l,c}(x_p) dLoss/du_p.

    Chain rule of Eq. 1 (the interpolation is linear in the grid values).
    Returns a list of [n, n, n, 3] arrays.
    """
    g_pts = np.asarray(g_pts, F64)
    L = len(res)
    C = g_pts.shape[1]
    out = []
    for n in res:
        idx, w = _corners(x, lo, hi, n)
        G = np.zeros((n * n * n, C), F64)
        for c in range(idx.shape[1]):
            np.add.at(G, idx[:, c], w[:, c : c + 1] * g_pts / L)
        out.append(G.reshape(n, n, n, C))
    return out


# ---------------------------------------------------------------------------------------
# the 6-D payload of Sec. 3.3: Cayley rotation + translation per grid vertex
# ---------------------------------------------------------------------------------------


def skew(z):
    """The skew-symmetric matrix Z of z (Sec. 3.3): rows (0, -z2, z1), (z2, 0, -z0),
    (-z1, z0, 0).  z: [..., 3] -> [..., 3, 3]."""
    z = np.asarray(z, F64)
    Z = np.zeros(z.shape[:-1] + (3, 3), F64)
    Z[..., 0, 1], Z[..., 0, 2] = -z[..., 2], z[..., 1]
    Z[..., 1, 0], Z[..., 1, 2] = z[..., 2], -z[..., 0]
    Z[..., 2, 0], Z[..., 2, 1] = -z[..., 1], z[..., 0]
    return Z


def cayley(z):
    """R(z) = (I + Z)(I - Z)^{-1}, the Cayley parameterisation of a rotation (Sec. 3.3).
    z: [..., 3] -> [..., 3, 3]."""
    Z = skew(z)
    I = np.broadcast_to(np.eye(3), Z.shape)
    return (I + Z) @ np.linalg.inv(I - Z)


def apply_transform(x, T):
    """M(T) x for the 4x4 homogeneous matrix [[R(z), t], [0, 1]] of T = [z, t] (Sec. 3.3),
    without the homogeneous coordinate: R(z) x + t.  Reading: the rotation acts about the
    world origin, as the matrix product is written.  x: [N, 3], T: [N, 6] -> [N, 3]."""
    x = np.asarray(x, F64)
    T = np.asarray(T, F64)
    return np.einsum("nij,nj->ni", cayley(T[:, :3]), x) + T[:, 3:]


def apply_transform_backward(x, T, g):
    """dLoss/dT given dLoss/dy = g for y = R(z) x + t: dLoss/dt = g and, by the product rule
    on R = (I + Z)(I - Z)^{-1} with dZ/dz_k = E_k (the skew matrix of the k-th unit vector),
    dR/dz_k = E_k (I - Z)^{-1} + (I + Z)(I - Z)^{-1} E_k (I - Z)^{-1}, so
    dLoss/dz_k = g . (dR/dz_k x).  Returns [N, 6]."""
    x = np.asarray(x, F64)
    T = np.asarray(T, F64)
    g = np.asarray(g, F64)
    Z = skew(T[:, :3])
    I = np.broadcast_to(np.eye(3), Z.shape)
    Ainv = np.linalg.inv(I - Z)
    R = (I + Z) @ Ainv
    out = np.zeros((len(x), 6), F64)
    for k in range(3):
        Ek = skew(np.eye(3)[k])
        dR = Ek @ Ainv + R @ Ek @ Ainv
        out[:, k] = np.einsum("ni,nij,nj->n", g, dR, x)
    out[:, 3:] = g
    return out


def deform_cayley(x, thetas, lo, hi):
    """x_t = M(T_t(x_{t-1})) x_{t-1}: one factor of the recursive product of Sec. 3.3, with
    T_t = (1/L) sum_l trilerp(G^l, x) the averaged 6-D payload (Eq. 1).  thetas: list of
    [n, n, n, 6] arrays (z first, then t)."""
    return apply_transform(x, eval_displacement(x, thetas, lo, hi))


# ---------------------------------------------------------------------------------------
# (b) exact nearest neighbours and the robust Chamfer distance, Sec. 3.4
# ---------------------------------------------------------------------------------------


def _sqdist(q, b):
    """Squared distance in difference form, (qx-bx)^2 + (qy-by)^2 + (qz-bz)^2."""
    d = q - b
    return d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2]


def nn_bruteforce(q, b, chunk: int = 512):
    """argmin_j ||q - b_j|| by exhaustive search (the argmin of the nearest-neighbour
    definitions in Sec. 3.4).  Ties go to the lowest index (reading; the paper is
    silent).  Returns (idx int64 [Nq], d2 float64 [Nq])."""
    q = np.asarray(q, F64)
    b = np.asarray(b, F64)
    idx = np.empty(len(q), np.int64)
    d2 = np.empty(len(q), F64)
    for s in range(0, len(q), chunk):
        D = _sqdist(q[s : s + chunk, None, :], b[None, :, :])
        j = np.argmin(D, axis=1)  # first minimum = lowest index
        idx[s : s + chunk] = j
        d2[s : s + chunk] = D[np.arange(len(j)), j]
    return idx, d2


def nn_exact(q, b, k: int = 8):
    """Exact nearest neighbours (lexicographic min of (d2, index)), Sec. 3.4.

    A k-d tree proposes the k closest candidates; their squared distances are recomputed
    in difference form and the lexicographic minimum is taken.  Queries for which the
    k-th candidate is not strictly farther than the best (a possible tie beyond the
    candidate list) are resolved by brute force.  Returns (idx, d2).
    """
    from scipy.spatial import cKDTree

    q = np.asarray(q, F64)
    b = np.asarray(b, F64)
    if len(b) == 0 or len(q) == 0:
        raise ValueError("empty point set")
    k = min(k, len(b))
    _, cand = cKDTree(b).query(q, k=k)
    cand = np.asarray(cand).reshape(len(q), k)
    D = _sqdist(q[:, None, :], b[cand])
    # lexicographic (d2, index) minimum over the candidates
    best = np.full(len(q), np.inf)
    bidx = np.full(len(q), np.iinfo(np.int64).max)
    for c in range(k):
        d, j = D[:, c], cand[:, c]
        better = (d < best) | ((d == best) & (j < bidx))
        best = np.where(better, d, best)
        bidx = np.where(better, j, bidx)
    if k < len(b):
        unsure = D.max(axis=1) <= best * (1 + 1e-9) + 1e-300
        if unsure.any():
            bi, bd = nn_bruteforce(q[unsure], b)
            bidx[unsure] = bi
            best[unsure] = bd
    return bidx, best


def nn_second_gap(q, b, idx, d2):
    """Relative gap between the best and the second-best squared distance of each query
    (inf for a single-point set).  Used to flag near-ties (gap < 1e-6)."""
    from scipy.spatial import cKDTree

    q = np.asarray(q, F64)
    b = np.asarray(b, F64)
    if len(b) < 2:
        return np.full(len(q), np.inf)
    _, cand = cKDTree(b).query(q, k=min(4, len(b)))
    D = _sqdist(q[:, None, :], b[cand])
    D = np.where(cand == idx[:, None], np.inf, D)
    second = D.min(1)
    return (second - d2) / np.maximum(second, 1e-300)


def robust_weight(d2, alpha):
    """w_R = exp(-alpha ||p - q||^2)  (Sec. 3.4)."""
    return np.exp(-alpha * np.asarray(d2, F64))


def robust_chamfer(A, B, alpha=ALPHA, stopgrad=False):
    """CD_R(A, B) and its gradient with respect to the points of A (Sec. 3.4).

    CD_R(A,B) = 1/|A| sum_a w_R(a, b_a) ||a - b_a||^2 + 1/|B| sum_b w_R(a_b, b) ||a_b - b||^2
    with b_a, a_b the nearest neighbours in the other set.  With s = ||a - b||^2 each term
    is phi(s) = s exp(-alpha s); its derivative is phi'(s) = exp(-alpha s)(1 - alpha s)
    (reading: the weight is differentiated; with `stopgrad` it is held constant,
    phi' = exp(-alpha s)).  d/da phi(||a-b||^2) = 2 phi'(s) (a - b).  B is data (no
    gradient).  Returns dict(loss, grad_A, nn_ab, d2_ab, nn_ba, d2_ba).
    """
    A = np.asarray(A, F64)
    B = np.asarray(B, F64)
    nab, sab = nn_exact(A, B)
    nba, sba = nn_exact(B, A)
    wab = robust_weight(sab, alpha)
    wba = robust_weight(sba, alpha)
    loss = (wab * sab).mean() + (wba * sba).mean()
    dab = wab if stopgrad else wab * (1 - alpha * sab)
    dba = wba if stopgrad else wba * (1 - alpha * sba)
    g = (2.0 / len(A)) * dab[:, None] * (A - B[nab])
    np.add.at(g, nba, (2.0 / len(B)) * dba[:, None] * (A[nba] - B))
    return dict(loss=loss, grad_A=g, nn_ab=nab, d2_ab=sab, nn_ba=nba, d2_ba=sba)


# ---------------------------------------------------------------------------------------
# (c) weak edge isometry, Sec. 3.4
# ---------------------------------------------------------------------------------------


def edge_lengths(x, edges):
    """||x_i - x_j|| for every edge (i, j)."""
    x = np.asarray(x, F64)
    e = np.asarray(edges, np.int64)
    d = x[e[:, 0]] - x[e[:, 1]]
    return np.sqrt((d * d).sum(1))


def isometry(y, edges, e_prev):
    """L_iso = 1/|E| sum_(i,j) | ||y_i - y_j|| - e_prev_ij |  and its gradient (Sec. 3.4).

    Per-frame form (T = 1).  Reading at the kink: the subgradient of |r| at r = 0 is 0,
    and a zero-length edge contributes no gradient.  Returns (loss, grad [V,3]).
    """
    y = np.asarray(y, F64)
    e = np.asarray(edges, np.int64)
    d = y[e[:, 0]] - y[e[:, 1]]
    ln = np.sqrt((d * d).sum(1))
    r = ln - np.asarray(e_prev, F64)
    E = len(e)
    loss = np.abs(r).sum() / E
    coef = np.where(ln > 0, np.sign(r) / np.where(ln > 0, ln, 1.0), 0.0) / E
    g = np.zeros_like(y)
    np.add.at(g, e[:, 0], coef[:, None] * d)
    np.add.at(g, e[:, 1], -coef[:, None] * d)
    return loss, g


# ---------------------------------------------------------------------------------------
# (e) grid Sobolev preconditioning, Sec. 3.2 Eq. 3, and Adam, Sec. 3.6
# ---------------------------------------------------------------------------------------


def grid_laplacian(g):
    """L g for the unit-weight 6-neighbour graph Laplacian of the vertex grid
    (degree minus adjacency, free boundary), applied per channel.

    Sec. 3.2 defines L^l as the Laplacian encoding adjacency between neighbouring grid
    cells; reading: axis neighbours only, unit weights, no spacing scaling.
    g: [n, n, n, C] (or [n, n, n]).
    """
    g = np.asarray(g, F64)
    out = np.zeros_like(g)
    for ax in range(3):
        n = g.shape[ax]
        if n < 2:
            continue
        hi_ = [slice(None)] * g.ndim
        lo_ = [slice(None)] * g.ndim
        hi_[ax] = slice(1, None)
        lo_[ax] = slice(0, n - 1)
        diff = g[tuple(hi_)] - g[tuple(lo_)]
        out[tuple(lo_)] -= diff
        out[tuple(hi_)] += diff
    return out


def _cg_shifted(b, lam, tol=1e-14, maxiter=2000):
    """Solve (I + lam L) h = b per channel by conjugate gradients to a relative residual
    of `tol`.  b: [n, n, n, C]."""
    b = np.asarray(b, F64)
    C = b.shape[-1]
    A = lambda v: v + lam * grid_laplacian(v)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    axes = (0, 1, 2)
    rr = (r * r).sum(axis=axes)
    bn = np.sqrt((b * b).sum(axis=axes))
    for _ in range(maxiter):
        if np.all(np.sqrt(rr) <= tol * np.maximum(bn, 1e-300)):
            break
        Ap = A(p)
        pAp = (p * Ap).sum(axis=axes)
        a = np.where(pAp > 0, rr / np.where(pAp > 0, pAp, 1.0), 0.0)
        x += a.reshape(1, 1, 1, C) * p
        r -= a.reshape(1, 1, 1, C) * Ap
        rr_new = (r * r).sum(axis=axes)
        beta = np.where(rr > 0, rr_new / np.where(rr > 0, rr, 1.0), 0.0)
        p = r + beta.reshape(1, 1, 1, C) * p
        rr = rr_new
    return x


def sobolev_precondition(g, lam, tol=1e-14):
    """(I + lam L)^{-2} g, applied per channel (Sec. 3.2, Eq. 3): two CG solves with the
    fixed grid Laplacian.  g: [n, n, n, 3]."""
    if lam == 0:
        return np.asarray(g, F64).copy()
    h = _cg_shifted(g, lam, tol)
    return _cg_shifted(h, lam, tol)


def sobolev_precondition_spectral(g, lam):
    """(I + lam L)^{-2} g per channel by the eigen-decomposition of L (Sec. 3.2, Eq. 3).

    Reading of the Laplacian as the free-boundary 6-neighbour graph Laplacian of the vertex
    grid: it is the Kronecker sum of three path-graph Laplacians, whose orthonormal
    eigenvectors are the DCT-II basis vectors with eigenvalues 4 sin^2(pi k / 2n).  So
    (I + lam L)^{-2} = C^T diag((1 + lam (mu_kx + mu_ky + mu_kz))^{-2}) C with C the
    orthonormal 3-D DCT-II, which scipy's dctn applies as a library step.  Same operator
    as sobolev_precondition (CG); used where a level is too large for CG to finish in
    seconds.  g: [nz, ny, nx, C]."""
    from scipy.fft import dctn, idctn

    g = np.asarray(g, F64)
    if lam == 0:
        return g.copy()
    mus = [4.0 * np.sin(np.pi * np.arange(n) / (2.0 * n)) ** 2 for n in g.shape[:3]]
    mu = mus[0][:, None, None] + mus[1][None, :, None] + mus[2][None, None, :]
    f = (1.0 + lam * mu) ** -2
    out = np.empty_like(g)
    for c in range(g.shape[3]):
        out[..., c] = idctn(f * dctn(g[..., c], type=2, norm="ortho"), type=2, norm="ortho")
    return out


def adam_update(theta, m, v, g, k, lr, beta1=BETA1, beta2=BETA2, eps=EPS):
    """One Adam step (Sec. 3.6: default hyper-parameters), PyTorch semantics:
    m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
    theta -= lr / (1 - b1^k) * m / (sqrt(v) / sqrt(1 - b2^k) + eps).
    k is the 1-based step count.  Returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    bc1 = 1 - beta1**k
    bc2 = 1 - beta2**k
    theta = theta - (lr / bc1) * m / (np.sqrt(v) / np.sqrt(bc2) + eps)
    return theta, m, v


# ---------------------------------------------------------------------------------------
# template-mesh optimisation, Sec. 3.4 (surface initialisation loss) and Sec. 3.6
# ---------------------------------------------------------------------------------------

MESH_LAMBDA = 16.0  # smoothness weight of the mesh preconditioner, Sec. 3.6
MESH_LR = 1e-4  # fixed learning rate of the mesh vertices, Sec. 3.6


def mesh_laplacian(n_verts, edges):
    """The combinatorial graph Laplacian (degree minus adjacency) of the mesh edges, as a
    scipy CSR matrix.  Reading: the paper preconditions the mesh vertices following Nicolet
    et al. (Sec. 3.2, last paragraph) without naming the Laplacian; this is the uniform-weight
    one, the mesh analogue of the grid Laplacian."""
    import scipy.sparse as sp

    e = np.asarray(edges, np.int64)
    A = sp.coo_matrix((np.ones(2 * len(e)), (np.concatenate([e[:, 0], e[:, 1]]), np.concatenate([e[:, 1], e[:, 0]]))),
                      shape=(n_verts, n_verts)).tocsr()
    deg = np.asarray(A.sum(1)).ravel()
    return (sp.diags(deg) - A).tocsr()


def mesh_precondition(g, edges, lam):
    """(I + lam L)^{-2} g per channel with L the mesh Laplacian: two sparse direct solves (a
    library step).  Reading: the same form as the grids' preconditioner (Sec. 3.2 Eq. 3 with
    the raw gradient then fed to Adam), with the mesh's Laplacian.  g: [V, C]."""
    import scipy.sparse as sp
    from scipy.sparse.linalg import factorized

    g = np.asarray(g, F64)
    if lam == 0:
        return g.copy()
    A = (sp.identity(len(g), format="csc") + lam * mesh_laplacian(len(g), edges)).tocsc()
    solve = factorized(A)
    out = np.empty_like(g)
    for c in range(g.shape[1]):
        out[:, c] = solve(solve(g[:, c]))
    return out


@dataclasses.dataclass
class MeshState:
    """Template-mesh fit: the vertices X_0 being optimised, the keyframe cloud P_0, the edges
    and Adam state (Sec. 3.4, L_mesh; Sec. 3.6)."""

    X: np.ndarray
    target: np.ndarray
    edges: np.ndarray
    m: np.ndarray
    v: np.ndarray
    k: int = 0


def mesh_begin(template, target, edges):
    X = np.asarray(template, F64).copy()
    return MeshState(X=X, target=np.asarray(target, F64), edges=np.asarray(edges, np.int64), m=np.zeros_like(X),
                     v=np.zeros_like(X))


def mesh_step(st: MeshState, lam=MESH_LAMBDA, lr=MESH_LR, alpha=ALPHA, update=True, cfg: Config | None = None):
    """One iteration of the template-mesh fit: L_mesh = CD_R(X_0, P_0) (Sec. 3.4) and its
    gradient with respect to the vertices, preconditioned by (I + lam L_mesh)^{-2}, then Adam
    with the fixed learning rate (Sec. 3.6).  Returns the loss, gradient and preconditioned
    gradient (before the update)."""
    c = cfg or Config()
    ch = robust_chamfer(st.X, st.target, alpha, c.robust_weight_stopgrad)
    pg = mesh_precondition(ch["grad_A"], st.edges, lam)
    out = dict(loss=ch["loss"], grad=ch["grad_A"], pgrad=pg, chamfer=ch, X=st.X.copy())
    if update:
        st.k += 1
        st.X, st.m, st.v = adam_update(st.X, st.m, st.v, pg, st.k, lr, c.beta1, c.beta2, c.eps)
    return out


# ---------------------------------------------------------------------------------------
# the whole per-iteration step and the per-frame fit
# ---------------------------------------------------------------------------------------


@dataclasses.dataclass
class FrameState:
    """State of one frame fit (Sec. 3.3/3.4): the fixed query points Q = X_{t-1} u P_{t-1}
    (template vertices first), the target P_t, edges, rest lengths, grids and Adam state."""

    x: np.ndarray  # [V+N, 3] float64
    n_verts: int
    target: np.ndarray  # [M, 3]
    edges: np.ndarray
    e_prev: np.ndarray
    thetas: list
    m: list
    v: list
    k: int = 0


def begin_frame(template_prev, source_prev, target, edges, cfg: Config, thetas=None) -> FrameState:
    """Per-frame set-up: Q = X_{t-1} u P_{t-1}; rest lengths from X_{t-1} (Sec. 3.4,
    isometry); grids zero (reading: each frame fits the motion t-1 -> t from zero) or the
    given values; fresh Adam state."""
    X = np.asarray(template_prev, F64)
    P = np.asarray(source_prev, F64)
    x = np.concatenate([X, P], 0)
    if thetas is None:
        thetas = [np.zeros((n, n, n, cfg.channels), F64) for n in cfg.res]
    else:
        thetas = [np.asarray(t, F64).copy() for t in thetas]
    return FrameState(
        x=x,
        n_verts=len(X),
        target=np.asarray(target, F64),
        edges=np.asarray(edges, np.int64),
        e_prev=edge_lengths(X, edges),
        thetas=thetas,
        m=[np.zeros_like(t) for t in thetas],
        v=[np.zeros_like(t) for t in thetas],
    )


def step(st: FrameState, cfg: Config, update: bool = True) -> dict:
    """One optimisation iteration (the hot path):
    (a) y = x + u(x) on Q (Eq. 1, Sec. 3.3), or y = R(z(x)) x + t(x) with the Cayley payload;
    (b) CD_R(X_hat, P_t) and CD_R(P_hat, P_t) with gradients (Sec. 3.4, L_transform with
        T = 1 and the confidence weight as the scalar w_chamfer_mesh);
    (c) w_iso * L_iso (Sec. 3.4);
    (d) adjoint of (a) into per-level grid gradients;
    (e) (I + lambda_l L_l)^{-2} per level (Eq. 3), then Adam with lr_l (Sec. 3.6).
    Returns a dict of every intermediate (for parity tests)."""
    V = st.n_verts
    if cfg.payload == "cayley":
        T = eval_displacement(st.x, st.thetas, cfg.lo, cfg.hi)
        y = apply_transform(st.x, T)
    else:
        y = deform(st.x, st.thetas, cfg.lo, cfg.hi)
    YX, PH = y[:V], y[V:]
    cm = robust_chamfer(YX, st.target, cfg.alpha, cfg.robust_weight_stopgrad)
    cp = robust_chamfer(PH, st.target, cfg.alpha, cfg.robust_weight_stopgrad)
    iso, giso = isometry(YX, st.edges, st.e_prev)
    loss = cfg.w_chamfer_mesh * cm["loss"] + cfg.w_chamfer_pts * cp["loss"] + cfg.w_iso * iso
    g_pts = np.concatenate([cfg.w_chamfer_mesh * cm["grad_A"] + cfg.w_iso * giso, cfg.w_chamfer_pts * cp["grad_A"]], 0)
    # with the Cayley payload the point gradients go through y = R(z) x + t first
    g_T = apply_transform_backward(st.x, T, g_pts) if cfg.payload == "cayley" else g_pts
    grads = interp_adjoint(st.x, g_T, cfg.res, cfg.lo, cfg.hi)
    pgrads = []
    for l, g in enumerate(grads):
        pgrads.append(sobolev_precondition(g, cfg.lam(l)) if cfg.precondition else g.copy())
    out = dict(y=y, loss=loss, cd_mesh=cm["loss"], cd_pts=cp["loss"], iso=iso, g_pts=g_pts, g_T=g_T, grads=grads,
               pgrads=pgrads, chamfer_mesh=cm, chamfer_pts=cp)
    if update:
        st.k += 1
        for l in range(len(st.thetas)):
            st.thetas[l], st.m[l], st.v[l] = adam_update(st.thetas[l], st.m[l], st.v[l], pgrads[l], st.k, cfg.lr(l),
                                                         cfg.beta1, cfg.beta2, cfg.eps)
    return out


def end_frame(st: FrameState, cfg: Config):
    """Frame end (Sec. 3.3): X_t = M(T_t(X_{t-1})) X_{t-1} with the final grids (for the
    displacement payload X_{t-1} + u_t(X_{t-1})); the target becomes the next frame's
    source.  Returns (X_t, P_t)."""
    xv = st.x[: st.n_verts]
    X = deform_cayley(xv, st.thetas, cfg.lo, cfg.hi) if cfg.payload == "cayley" else deform(xv, st.thetas, cfg.lo, cfg.hi)
    return X, st.target.copy()


def fit_frame(template_prev, source_prev, target, edges, cfg: Config, n_steps: int, thetas=None):
    """Fit one frame with n_steps iterations.  Returns (X_t, history, state)."""
    st = begin_frame(template_prev, source_prev, target, edges, cfg, thetas)
    hist = []
    for _ in range(n_steps):
        o = step(st, cfg)
        hist.append((o["loss"], o["cd_mesh"], o["cd_pts"], o["iso"]))
    X, _ = end_frame(st, cfg)
    return X, np.asarray(hist), st
