"""Plain FP64 CPU oracle for the spectral-element Poisson hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this module; only the
tests, the smoke check and the benchmark's CPU-baseline leg do.  It shares no
code with the CUDA path: the only common module is `synthetic`, which makes
seeded meshes and fields and holds none of the method's arithmetic.

What it computes (Karp et al., "A High-Fidelity Flow Solver for Unstructured
Meshes on FPGAs", HPC Asia 2022):
  * Section 3, Eqs. 1-4: Poisson problem, weak form, GLL tensor-product basis,
    local operator A^e = D^T G^e D, evaluated matrix-free (Section 3.1).
  * Section 3.1, Eq. 5: gather-scatter QQ^T (direct stiffness summation) on the
    replicated local representation u_L = Q u, plus Dirichlet masking.
  * Section 3.2, Algorithm 1: CG on the local representation with the
    multiplicity-weighted inner product <a, b, c>; here with z = M^-1 r added
    (Jacobi preconditioner, exact assembled diagonal).
  * Section 5.1: the rematerialised (on-the-fly) variant computes the same
    operator; the oracle computes G from the element vertices once.
The textbook pieces the paper cites (GLL nodes and weights, D, G^e written out)
follow Deville, Fischer and Mund, "High-Order Methods for Incompressible Fluid
Flow" (2002), the paper's SEM reference.

Readings where the paper is silent or garbled (each listed in the design notes):
  * Eq. 1 is printed as lap(u) = f, but the weak form Eq. 2 is that of
    -lap(u) = f; the oracle solves -lap(u) = f (symmetric positive operator).
  * G^e = w_i w_j w_k |det J| J^-1 J^-T with J_ab = dx_a/dxi_b (six unique entries,
    Section 4.2 counts six geometric factors per point).
  * Elements are trilinear hexahedra (Section 5.1: linearly deformed); vertex
    a + 2b + 4c sits at reference corner (2a-1, 2b-1, 2c-1).
  * c_i = 1 / multiplicity of the global node of local node i (Algorithm 1
    uses c without defining it).
  * Global numbering: order of first occurrence in the local traversal
    (element, k, j, i) of a key naming the topological entity and position.
  * A node is Dirichlet-masked iff it lies on a face that belongs to one
    element only (optionally: and whose four vertices are all flagged).
  * Preconditioned CG: r0 = b - A x0, z = M^-1 r, rho = <r, z, c>, stop when
    sqrt(<r, r, c> / <b, b, c>) <= rtol, checked after the r update.

Layout: local arrays are [E, Np, Np, Np] indexed (e, k, j, i), i fastest, with
Np = N + 1; flattened local index = ((e*Np + k)*Np + j)*Np + i.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# ---------------------------------------------------------------------------
# GLL nodes, weights and the derivative matrix (Section 3, Eq. 3; Deville et
# al. Appendix B).
# ---------------------------------------------------------------------------


def _legendre_and_derivs(N: int, x):
    """L_N(x), L_N'(x) by the three-term recurrence (x may be an array)."""
    p0 = np.ones_like(x)
    if N == 0:
        return p0, np.zeros_like(x)
    p1 = x.copy()
    d0, d1 = np.zeros_like(x), np.ones_like(x)
    for k in range(1, N):
        p2 = ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
        d2 = d0 + (2 * k + 1) * p1  # P'_{k+1} = P'_{k-1} + (2k+1) P_k
        p0, p1, d0, d1 = p1, p2, d1, d2
    return p1, d1


def gll_nodes_weights(N: int):
    """N+1 Gauss-Lobatto-Legendre nodes (ascending) and weights.

    Nodes: -1, +1 and the N-1 roots of L_N'; found by Newton on L_N' started
    from the Chebyshev-Gauss-Lobatto points, in extended precision.
    Weights: w_i = 2 / (N (N+1) L_N(xi_i)^2).
    """
    if N < 1:
        raise ValueError("N >= 1 required")
    ld = np.longdouble
    x = -np.cos(np.pi * np.arange(N + 1, dtype=ld) / ld(N))
    x[0], x[N] = ld(-1), ld(1)
    xi = x[1:N].copy()
    for _ in range(100):
        L, dL = _legendre_and_derivs(N, xi)
        # L_N'' from Legendre's equation: (1-x^2) L'' = 2x L' - N(N+1) L
        d2L = (2 * xi * dL - N * (N + 1) * L) / (1 - xi * xi)
        step = dL / d2L
        xi = xi - step
        if np.all(np.abs(step) < ld(1e-30)):
            break
    x[1:N] = xi
    L, _ = _legendre_and_derivs(N, x)
    w = ld(2) / (ld(N * (N + 1)) * L * L)
    return x.astype(np.float64), w.astype(np.float64)


def lagrange_derivative_matrix(xi: np.ndarray) -> np.ndarray:
    """D[i, j] = l_j'(xi_i) for the Lagrange basis through the nodes xi.

    Written from the definition l_j(x) = prod_{m != j} (x - xi_m)/(xi_j - xi_m):
      l_j'(xi_i) = prod_{m != i, j} (xi_i - xi_m) / prod_{m != j} (xi_j - xi_m)  (i != j)
      l_j'(xi_j) = sum_{m != j} 1 / (xi_j - xi_m).
    """
    n = len(xi)
    D = np.zeros((n, n))
    for j in range(n):
        den = 1.0
        for m in range(n):
            if m != j:
                den *= xi[j] - xi[m]
        for i in range(n):
            if i == j:
                D[i, j] = sum(1.0 / (xi[j] - xi[m]) for m in range(n) if m != j)
            else:
                num = 1.0
                for m in range(n):
                    if m != i and m != j:
                        num *= xi[i] - xi[m]
                D[i, j] = num / den
    return D


# ---------------------------------------------------------------------------
# Geometry of trilinear hexahedra: Jacobian, geometric factors G (six per point,
# Section 4.2), mass B, physical coordinates.
# ---------------------------------------------------------------------------

_CORNER = [(a, b, c) for c in range(2) for b in range(2) for a in range(2)]  # index a + 2b + 4c


def _phi(s, t):
    """Linear shape functions on [-1, 1]: phi_0 = (1-t)/2, phi_1 = (1+t)/2."""
    return 0.5 * (1.0 - t) if s == 0 else 0.5 * (1.0 + t)


def _dphi(s):
    return -0.5 if s == 0 else 0.5


def element_vertices(vert_xyz: np.ndarray, elem_verts: np.ndarray) -> np.ndarray:
    """X[e, v, :] = coordinates of local vertex v (tensor order a + 2b + 4c)."""
    return np.asarray(vert_xyz, dtype=np.float64)[np.asarray(elem_verts, dtype=np.int64)]


def coordinates(X: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """Physical coordinates x(xi_i, xi_j, xi_k) -> array [E, Np, Np, Np, 3] (e, k, j, i)."""
    Np = len(xi)
    out = np.zeros((X.shape[0], Np, Np, Np, 3))
    for v, (a, b, c) in enumerate(_CORNER):
        wgt = (_phi(c, xi)[:, None, None] * _phi(b, xi)[None, :, None] * _phi(a, xi)[None, None, :])
        out += wgt[None, :, :, :, None] * X[:, v, None, None, None, :]
    return out


def jacobian(X: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """J[e, k, j, i, alpha, beta] = d x_alpha / d xi_beta at the GLL points.

    beta = 0, 1, 2 are the reference directions (xi along i, eta along j,
    gamma along k); each derivative differentiates one linear factor.
    """
    Np = len(xi)
    J = np.zeros((X.shape[0], Np, Np, Np, 3, 3))
    one = np.ones_like(xi)
    for v, (a, b, c) in enumerate(_CORNER):
        fa, fb, fc = _phi(a, xi), _phi(b, xi), _phi(c, xi)
        ga, gb, gc = _dphi(a) * one, _dphi(b) * one, _dphi(c) * one
        d_xi = fc[:, None, None] * fb[None, :, None] * ga[None, None, :]
        d_eta = fc[:, None, None] * gb[None, :, None] * fa[None, None, :]
        d_gam = gc[:, None, None] * fb[None, :, None] * fa[None, None, :]
        for beta, wgt in enumerate((d_xi, d_eta, d_gam)):
            J[..., :, beta] += wgt[None, :, :, :, None] * X[:, v, None, None, None, :]
    return J


def weights3(w: np.ndarray) -> np.ndarray:
    """w_i w_j w_k as [Np, Np, Np] indexed (k, j, i)."""
    return w[:, None, None] * w[None, :, None] * w[None, None, :]


class MeshError(ValueError):
    pass


def geometric_factors(X: np.ndarray, xi: np.ndarray, w: np.ndarray):
    """G (six unique entries) and mass B at every GLL point (Eq. 4's G^e).

    G = w_i w_j w_k |det J| J^-1 J^-T, returned as [E, 6, Np, Np, Np] in the
    order (G11, G12, G13, G22, G23, G33); B = w_i w_j w_k |det J|.
    Raises MeshError if det J <= 0 anywhere (inverted or degenerate element).
    """
    J = jacobian(X, xi)
    det = np.linalg.det(J)
    if not np.all(det > 0):
        raise MeshError("det J <= 0 at some GLL point")
    Jinv = np.linalg.inv(J)
    M = Jinv @ np.swapaxes(Jinv, -1, -2)  # J^-1 J^-T
    scale = weights3(w)[None] * det
    Gfull = M * scale[..., None, None]
    G = np.stack([Gfull[..., 0, 0], Gfull[..., 0, 1], Gfull[..., 0, 2],
                  Gfull[..., 1, 1], Gfull[..., 1, 2], Gfull[..., 2, 2]], axis=1)
    return G, scale


# ---------------------------------------------------------------------------
# Local operator A_L (Eq. 4, Section 3.1), sum-factorised.
# ---------------------------------------------------------------------------


def ax_local(u: np.ndarray, G: np.ndarray, D: np.ndarray) -> np.ndarray:
    """w = A_L u = D^T G D u element by element.

    u : [E, Np, Np, Np] (e, k, j, i).  Forward derivatives along i, j, k:
      ur = (I x I x D) u, us = (I x D x I) u, ut = (D x I x I) u;
    G-weighting (v = G grad u with the symmetric 3x3 G);
    transposed derivatives summed: w = D^T-along-i vr + D^T-along-j vs + D^T-along-k vt.
    """
    ur = np.einsum("il,ekjl->ekji", D, u)
    us = np.einsum("jl,ekli->ekji", D, u)
    ut = np.einsum("kl,elji->ekji", D, u)
    G11, G12, G13, G22, G23, G33 = (G[:, m] for m in range(6))
    vr = G11 * ur + G12 * us + G13 * ut
    vs = G12 * ur + G22 * us + G23 * ut
    vt = G13 * ur + G23 * us + G33 * ut
    return (np.einsum("li,ekjl->ekji", D, vr)
            + np.einsum("lj,ekli->ekji", D, vs)
            + np.einsum("lk,elji->ekji", D, vt))


# ---------------------------------------------------------------------------
# Numbering, multiplicity, mask (Section 3.1: Q, u_L = Q u; Algorithm 1's c).
# ---------------------------------------------------------------------------


def _node_key(N, e, i, j, k, v):
    """Key of local node (i, j, k) of an element with vertex ids v[a + 2b + 4c]."""
    coords = (i, j, k)
    ends = [None if 0 < q < N else (q // N) for q in coords]
    free = [d for d in range(3) if ends[d] is None]
    if len(free) == 3:
        return ("I", e, i, j, k)

    def corner(sel):
        # sel: dict axis -> 0/1 for the free axes; fixed axes use their end value
        abc = [sel[d] if d in sel else ends[d] for d in range(3)]
        return int(v[abc[0] + 2 * abc[1] + 4 * abc[2]])

    if len(free) == 0:
        return ("V", corner({}))
    if len(free) == 1:
        d = free[0]
        lo, hi = corner({d: 0}), corner({d: 1})
        t = coords[d]
        return ("E", min(lo, hi), max(lo, hi), t if lo < hi else N - t)
    # face: free axes s-axis = free[0], t-axis = free[1]
    ds, dt = free
    c = {(a, b): corner({ds: a, dt: b}) for a in (0, 1) for b in (0, 1)}
    o = min(c, key=lambda ab: c[ab])
    n_s = (1 - o[0], o[1])  # neighbour of the origin along s
    n_t = (o[0], 1 - o[1])  # neighbour of the origin along t
    ps = coords[ds] if o[0] == 0 else N - coords[ds]
    pt = coords[dt] if o[1] == 0 else N - coords[dt]
    if c[n_s] < c[n_t]:
        p, q = ps, pt
    else:
        p, q = pt, ps
    return ("F", tuple(sorted(c.values())), p, q)


_FACES = [  # (axis, end) -> the face of the element where coordinate `axis` is at `end`
    (0, 0), (0, 1), (1, 0), (1, 1), (2, 0), (2, 1)]


@dataclass
class Numbering:
    glo_num: np.ndarray  # int64 [n]
    n_glob: int
    mult: np.ndarray     # int64 [n_glob]
    mask: np.ndarray     # uint8 [n]; 1 = Dirichlet node (zeroed)

    def c(self) -> np.ndarray:
        """Algorithm 1's weight c_i = 1 / multiplicity(glo_num[i])."""
        return 1.0 / self.mult[self.glo_num].astype(np.float64)


def number_nodes(N: int, elem_verts: np.ndarray, dirichlet_vertex_flags=None) -> Numbering:
    """Canonical global numbering, multiplicity and Dirichlet mask.

    Two local nodes are one global node iff they sit on the same topological
    entity (vertex; edge = sorted vertex pair, at the same distance from its
    lower-id end; face = sorted vertex 4-set, at the same position in the frame
    whose origin is the lowest-id corner and whose first axis points to that
    corner's lower-id neighbour).  Global id = order of first occurrence in the
    traversal (e, k, j, i).  Plain dictionary, one node at a time.
    """
    ev = np.asarray(elem_verts, dtype=np.int64)
    E = ev.shape[0]
    Np = N + 1
    for e in range(E):
        if len(set(ev[e].tolist())) != 8:
            raise MeshError(f"element {e} repeats a vertex id")
    ids: dict = {}
    glo = np.empty(E * Np ** 3, dtype=np.int64)
    pos = 0
    for e in range(E):
        v = ev[e]
        for k in range(Np):
            for j in range(Np):
                for i in range(Np):
                    key = _node_key(N, e, i, j, k, v)
                    g = ids.get(key)
                    if g is None:
                        g = len(ids)
                        ids[key] = g
                    glo[pos] = g
                    pos += 1
    n_glob = len(ids)
    mult = np.bincount(glo, minlength=n_glob).astype(np.int64)
    # boundary faces: faces (as vertex 4-sets) owned by exactly one element
    owners: dict = {}
    for e in range(E):
        for axis, end in _FACES:
            corners = []
            for c in range(2):
                for b in range(2):
                    for a in range(2):
                        abc = [a, b, c]
                        if abc[axis] == end:
                            corners.append(int(ev[e, a + 2 * b + 4 * c]))
            owners.setdefault(tuple(sorted(corners)), []).append((e, axis, end))
    flags = None if dirichlet_vertex_flags is None else np.asarray(dirichlet_vertex_flags)
    masked_glob = np.zeros(n_glob, dtype=bool)
    for fkey, own in owners.items():
        if len(own) > 2:
            raise MeshError("face shared by more than two elements")
        if len(own) != 1:
            continue
        if flags is not None and not all(flags[vid] for vid in fkey):
            continue
        e, axis, end = own[0]
        for k in range(Np):
            for j in range(Np):
                for i in range(Np):
                    if (i, j, k)[axis] == end * N:
                        masked_glob[glo[((e * Np + k) * Np + j) * Np + i]] = True
    mask = masked_glob[glo].astype(np.uint8)
    return Numbering(glo, n_glob, mult, mask)


# ---------------------------------------------------------------------------
# Gather-scatter QQ^T and masking (Eq. 5, Section 4.3; Algorithm 1 step 7).
# ---------------------------------------------------------------------------


def dssum(w_local: np.ndarray, glo_num: np.ndarray, mask=None, dtype=np.float64) -> np.ndarray:
    """QQ^T w: every local copy of a global node receives the sum of all copies.

    The copies of one global node are summed left to right in ascending local
    index (s = w_a, s = s + w_b, ...), in `dtype` arithmetic, so the result is
    fixed bit for bit.  With `mask`, masked copies are then set to zero.
    """
    w = np.asarray(w_local, dtype=dtype).ravel()
    glo = np.asarray(glo_num).ravel()
    order = np.argsort(glo, kind="stable")  # ascending local index within each global id
    g_sorted = glo[order]
    starts = np.flatnonzero(np.r_[True, g_sorted[1:] != g_sorted[:-1]])
    counts = np.diff(np.r_[starts, g_sorted.size])
    sums = w[order[starts]].copy()               # s = first copy
    for r in range(1, int(counts.max()) if counts.size else 0):
        has = counts > r
        sums[has] = sums[has] + w[order[starts[has] + r]]   # s = s + next copy
    total = np.empty(g_sorted.size and (int(g_sorted[-1]) + 1), dtype=dtype)
    total[g_sorted[starts]] = sums
    out = total[glo]
    if mask is not None:
        out = np.where(np.asarray(mask).ravel() != 0, dtype(0), out).astype(dtype)
    return out.reshape(np.shape(w_local))


def gather_global(w_local: np.ndarray, glo_num: np.ndarray, n_glob: int) -> np.ndarray:
    """Q^T w: sum of local copies into a global vector."""
    out = np.zeros(n_glob)
    np.add.at(out, np.asarray(glo_num).ravel(), np.asarray(w_local, dtype=np.float64).ravel())
    return out


def scatter_local(u_glob: np.ndarray, glo_num: np.ndarray) -> np.ndarray:
    """Q u: replicate global values to their local copies."""
    return np.asarray(u_glob)[np.asarray(glo_num)]


def glsc3(a, b, c) -> float:
    """Weighted inner product <a, b, c> = sum_i a_i b_i c_i (Algorithm 1)."""
    return float(np.sum(np.asarray(a).ravel() * np.asarray(b).ravel() * np.asarray(c).ravel()))


# ---------------------------------------------------------------------------
# Problem set-up: operator object, Jacobi diagonal, right-hand side.
# ---------------------------------------------------------------------------


class SemProblem:
    """Everything the oracle needs for one mesh at order N."""

    def __init__(self, N: int, vert_xyz, elem_verts, dirichlet_vertex_flags=None):
        self.N, self.Np = int(N), int(N) + 1
        self.xi, self.w = gll_nodes_weights(self.N)
        self.D = lagrange_derivative_matrix(self.xi)
        self.X = element_vertices(vert_xyz, elem_verts)
        self.E = self.X.shape[0]
        self.G, self.B = geometric_factors(self.X, self.xi, self.w)
        self.num = number_nodes(self.N, elem_verts, dirichlet_vertex_flags)
        self.glo_num, self.mask = self.num.glo_num, self.num.mask
        self.c = self.num.c()
        self.n = self.E * self.Np ** 3

    def shape(self):
        return (self.E, self.Np, self.Np, self.Np)

    def ax_local(self, u):
        return ax_local(np.asarray(u, dtype=np.float64).reshape(self.shape()), self.G, self.D)

    def ax(self, u, assemble=True):
        """Section 3.1's Ax = QQ^T A_L x, with the Dirichlet mask (Algorithm 1 steps 6-7)."""
        w = self.ax_local(u)
        if not assemble:
            return w
        return dssum(w, self.glo_num, self.mask)

    def jacobi_diagonal(self):
        """Diagonal of the assembled unmasked operator, on the local layout.

        Local diagonal of D^T G D at (i, j, k):
          sum_l D_li^2 G11(l,j,k) + sum_l D_lj^2 G22(i,l,k) + sum_l D_lk^2 G33(i,j,l)
          + 2 D_ii D_jj G12 + 2 D_ii D_kk G13 + 2 D_jj D_kk G23,
        then summed over the copies of each global node (QQ^T).
        """
        D = self.D
        G11, G12, G13, G22, G23, G33 = (self.G[:, m] for m in range(6))
        D2 = D * D
        dd = np.diag(D)
        d = (np.einsum("li,ekjl->ekji", D2, G11)
             + np.einsum("lj,ekli->ekji", D2, G22)
             + np.einsum("lk,elji->ekji", D2, G33)
             + 2 * dd[None, None, None, :] * dd[None, None, :, None] * G12
             + 2 * dd[None, None, None, :] * dd[None, :, None, None] * G13
             + 2 * dd[None, None, :, None] * dd[None, :, None, None] * G23)
        return dssum(d, self.glo_num)

    def jacobi_inverse(self):
        """M^-1 on the local layout: 1 / assembled diagonal, 0 on masked nodes."""
        d = self.jacobi_diagonal()
        return np.where(self.mask.reshape(self.shape()) != 0, 0.0, 1.0 / d)

    def coords(self):
        return coordinates(self.X, self.xi)

    def rhs(self, a=1, b=1, c=1):
        """b = mask(QQ^T (B f)) with f = (a^2+b^2+c^2) pi^2 sin(a pi x) sin(b pi y) sin(c pi z).

        f is -lap of the manufactured solution sin(a pi x) sin(b pi y) sin(c pi z).
        """
        x = self.coords()
        f = ((a * a + b * b + c * c) * math.pi ** 2 * np.sin(a * math.pi * x[..., 0])
             * np.sin(b * math.pi * x[..., 1]) * np.sin(c * math.pi * x[..., 2]))
        return dssum(self.B * f, self.glo_num, self.mask)

    def exact_solution(self, a=1, b=1, c=1):
        x = self.coords()
        return (np.sin(a * math.pi * x[..., 0]) * np.sin(b * math.pi * x[..., 1])
                * np.sin(c * math.pi * x[..., 2]))


# ---------------------------------------------------------------------------
# Conjugate gradient, Algorithm 1 (Section 3.2), with optional Jacobi z = M^-1 r.
# ---------------------------------------------------------------------------


@dataclass
class CGResult:
    x: np.ndarray
    iterations: int
    rel_res: float
    converged: bool
    history: list


def pcg(prob: SemProblem, b, x0=None, rtol=1e-10, max_iter=10000, precond=True) -> CGResult:
    """Algorithm 1 on the local representation.

    r = b - A x0; beta = 0; p = 0; rho = <r, z, c> with z = M^-1 r (z = r
    without preconditioning); then per iteration: p = z + beta p; w = QQ^T A_L p
    masked; alpha = rho / <p, w, c>; x += alpha p; r -= alpha w; z = M^-1 r;
    rho_new = <r, z, c>; stop when sqrt(<r, r, c> / <b, b, c>) <= rtol;
    beta = rho_new / rho.  `iterations` counts the operator applications in the loop.
    """
    shape = prob.shape()
    c = prob.c.reshape(shape)
    b = np.asarray(b, dtype=np.float64).reshape(shape)
    x = np.zeros(shape) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(shape).copy()
    Minv = prob.jacobi_inverse() if precond else np.where(prob.mask.reshape(shape) != 0, 0.0, 1.0)
    r = b - prob.ax(x)
    z = Minv * r
    beta = 0.0
    p = np.zeros(shape)
    rho = glsc3(r, z, c)
    bb = glsc3(b, b, c)
    rr = glsc3(r, r, c)
    hist = [math.sqrt(rr / bb) if bb > 0 else math.sqrt(rr)]
    if rr <= rtol * rtol * bb:
        return CGResult(x, 0, hist[-1], True, hist)
    for it in range(1, max_iter + 1):
        p = z + beta * p
        w = prob.ax(p)
        alpha = rho / glsc3(p, w, c)
        x = x + alpha * p
        r = r - alpha * w
        z = Minv * r
        rho_new = glsc3(r, z, c)
        rr = glsc3(r, r, c)
        hist.append(math.sqrt(rr / bb))
        if rr <= rtol * rtol * bb:
            return CGResult(x, it, hist[-1], True, hist)
        beta = rho_new / rho
        rho = rho_new
    return CGResult(x, max_iter, hist[-1], False, hist)


# ---------------------------------------------------------------------------
# Brute force: dense element matrices from explicit basis gradients.
# ---------------------------------------------------------------------------


def element_stiffness_dense(X1: np.ndarray, xi: np.ndarray, w: np.ndarray, D: np.ndarray) -> np.ndarray:
    """A^e[a, b] = sum_q w_q |det J_q| grad phi_a(q) . grad phi_b(q) for one element.

    X1 : [8, 3] vertices.  Reference gradients of the nodal basis at the GLL
    quadrature points are formed as explicit dense matrices (Kronecker products
    of D with identities), mapped with J^-T at each point; no sum factorisation
    and no geometric-factor tensor are used.
    """
    Np = len(xi)
    I = np.eye(Np)
    # rows: quadrature point (k, j, i); columns: basis function (c, b, a); i fastest
    Dxi = np.kron(I, np.kron(I, D))
    Deta = np.kron(I, np.kron(D, I))
    Dgam = np.kron(D, np.kron(I, I))
    J = jacobian(X1[None], xi)[0].reshape(-1, 3, 3)
    det = np.linalg.det(J)
    JinvT = np.swapaxes(np.linalg.inv(J), -1, -2)
    ref = np.stack([Dxi, Deta, Dgam], axis=1)            # [q, beta, basis]
    phys = np.einsum("qab,qbn->qan", JinvT, ref)         # [q, alpha, basis]
    wq = weights3(w).reshape(-1) * det
    return np.einsum("qan,q,qam->nm", phys, wq, phys)


def assembled_stiffness_dense(prob: SemProblem) -> np.ndarray:
    """K = sum_e Q_e^T A^e Q_e as a dense n_glob x n_glob matrix (small meshes only)."""
    n_glob = prob.num.n_glob
    P = prob.Np ** 3
    K = np.zeros((n_glob, n_glob))
    for e in range(prob.E):
        Ae = element_stiffness_dense(prob.X[e], prob.xi, prob.w, prob.D)
        g = prob.glo_num[e * P:(e + 1) * P]
        K[np.ix_(g, g)] += Ae
    return K
