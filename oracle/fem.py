"""FP64 oracle of the finite-element bending term of the hybrid membrane
(Section 3.1, Eq. 6-10).  Test infrastructure: only the tests, the smoke check
and the benchmark's CPU baseline use this module; the CUDA library shares no
code with it.

The surface is covered by quadratic six-node triangles (three corners and the
three edge midpoints); on each element a field u is interpolated from its
nodal values with the quadratic basis N_1..N_6 (Eq. 7).  Nodes are numbered
corners (xi, eta) = (0,0), (1,0), (0,1), then midpoints (1/2,0), (1/2,1/2),
(0,1/2).  In the order of Section 3.1:

1. the unit normal at every element node, from the tangents dX/dxi, dX/deta
   of the interpolated surface, averaged over the elements sharing the node
   (sum of unit normals, normalised);
2. Eq. 9 at every element node: the curvature tensor kappa solves
   dX/dxi . kappa = dn/dxi, dX/deta . kappa = dn/deta, n . kappa = 0, with
   n the nodal normals of step 1 interpolated by Eq. 7 and the third row the
   node's own normal; kappa is then averaged over the elements sharing the
   node (per node: the mean of its element values);
3. Eq. 10: mean curvature K = tr(kappa)/2; Gaussian curvature
   K_G = kappa_1 kappa_2 = ((tr kappa)^2 - tr(kappa kappa))/2;
4. the surface Laplacian of K: the surface gradient g of K solves the same
   system as step 2 with K in place of n (dX/dxi . g = dK/dxi, ...,
   n . g = 0), averaged per node; the surface divergence of g is the trace of
   the tensor that the same system gives for g's components, averaged per
   node;
5. the bending force at node i: F_i = A_i (k0/2) (Lap_S K + 2 K (K^2 - K_G)) n_i,
   the normal force density that follows from the energy of Eq. 6,
   H = (k0/2) int K^2 dS, by its first variation, times the node's area A_i
   (one third of each flat sub-triangle of the four that split every element
   and touch node i).

Readings (the paper is silent or garbled here):
  * the force after Eq. 10 is printed as (Lap_S K + 2 K^3) n: the first
    variation of Eq. 6 gives (k0/2)(Lap_S K + 2 K (K^2 - K_G)) n, which keeps
    a sphere force-free; that form is used;
  * Eq. 8's deformation gradient feeds the in-plane strain of the cited
    finite-element membrane; the hybrid model's in-plane elasticity is Eq. 2-5,
    so the bending term needs Eq. 9-10 only;
  * nodal averaging is the plain mean over the elements sharing the node;
  * the nodal area is the barycentric one of the flat sub-triangles.
"""
import numpy as np

# parametric coordinates of the six element nodes
NODE_XI = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [0.5, 0.0], [0.5, 0.5], [0.0, 0.5]])
# the four flat sub-triangles of an element, by local node
SUB_TRI = np.array([[0, 3, 5], [3, 1, 4], [5, 4, 2], [3, 4, 5]])


def shape(xi, eta):
    """Quadratic six-node basis (Eq. 7) and its parametric derivatives at
    (xi, eta): arrays N, dN/dxi, dN/deta of length 6."""
    z = 1.0 - xi - eta
    N = np.array([z * (2 * z - 1), xi * (2 * xi - 1), eta * (2 * eta - 1), 4 * xi * z, 4 * xi * eta, 4 * eta * z])
    dxi = np.array([-(4 * z - 1), 4 * xi - 1, 0.0, 4 * (z - xi), 4 * eta, -4 * eta])
    deta = np.array([-(4 * z - 1), 0.0, 4 * eta - 1, -4 * xi, 4 * xi, 4 * (z - eta)])
    return N, dxi, deta


def _node_derivative_matrices():
    Dxi = np.zeros((6, 6))
    Deta = np.zeros((6, 6))
    for j, (xi, eta) in enumerate(NODE_XI):
        _, Dxi[j], Deta[j] = shape(xi, eta)
    return Dxi, Deta


DXI, DETA = _node_derivative_matrices()   # [node j][basis k] at the element nodes


def node_mean(vals, elem6, n):
    """Mean over the elements sharing each node of per-element-node values
    vals[E, 6, ...]; nodes of no element get zero."""
    vals = np.asarray(vals, dtype=np.float64)
    out = np.zeros((n,) + vals.shape[2:])
    cnt = np.zeros(n)
    np.add.at(out, elem6.ravel(), vals.reshape((-1,) + vals.shape[2:]))
    np.add.at(cnt, elem6.ravel(), 1.0)
    nz = cnt > 0
    out[nz] /= cnt[nz].reshape((-1,) + (1,) * (out.ndim - 1))
    return out


def derivatives(u, elem6):
    """d/dxi and d/deta at the six element nodes of a nodal field u[n, ...]
    interpolated by Eq. 7: arrays [E, 6, ...]."""
    U = np.asarray(u, dtype=np.float64)[elem6]            # [E, 6(basis), ...]
    return np.einsum("jk,ek...->ej...", DXI, U), np.einsum("jk,ek...->ej...", DETA, U)


def element_normals(X, elem6):
    """Unit normal dX/dxi x dX/deta at every element node: [E, 6, 3]."""
    a_xi, a_eta = derivatives(X, elem6)
    nrm = np.cross(a_xi, a_eta)
    return nrm / np.linalg.norm(nrm, axis=-1, keepdims=True)


def nodal_normals(X, elem6):
    """Step 1: averaged unit normals [n, 3] (zero for nodes of no element)."""
    s = node_mean(element_normals(X, elem6), elem6, len(X))
    L = np.linalg.norm(s, axis=1, keepdims=True)
    return np.divide(s, L, out=np.zeros_like(s), where=L > 0)


def _systems(X, elem6, n_node):
    """The matrices [dX/dxi; dX/deta; n_j] of Eq. 9 at every element node."""
    a_xi, a_eta = derivatives(X, elem6)
    return np.stack([a_xi, a_eta, n_node[elem6]], axis=-2)   # [E, 6, 3, 3]


def _solve_tangential(M, d_xi, d_eta):
    """Solves M t = [d_xi; d_eta; 0] (right-hand sides stacked as rows)."""
    B = np.stack([d_xi, d_eta, np.zeros_like(d_xi)], axis=-2)
    return np.linalg.solve(M, B)


def curvature_tensors(X, elem6, n_node=None):
    """Step 2: kappa at every element node, [E, 6, 3, 3]."""
    if n_node is None:
        n_node = nodal_normals(X, elem6)
    dn_xi, dn_eta = derivatives(n_node, elem6)
    return _solve_tangential(_systems(X, elem6, n_node), dn_xi, dn_eta)


def curvatures(X, elem6, n_node=None):
    """Steps 2-3: nodal mean curvature K and Gaussian curvature K_G (the
    per-element values of Eq. 10 averaged per node)."""
    kap = curvature_tensors(X, elem6, n_node)
    tr = np.trace(kap, axis1=-2, axis2=-1)
    tr2 = np.trace(kap @ kap, axis1=-2, axis2=-1)
    K = node_mean(0.5 * tr, elem6, len(X))
    KG = node_mean(0.5 * (tr * tr - tr2), elem6, len(X))
    return K, KG


def surface_gradient(X, elem6, u, n_node=None):
    """Surface gradient of a nodal scalar u: [n, 3] (averaged per node)."""
    if n_node is None:
        n_node = nodal_normals(X, elem6)
    d_xi, d_eta = derivatives(u, elem6)
    M = _systems(X, elem6, n_node)
    B = np.stack([d_xi, d_eta, np.zeros_like(d_xi)], axis=-1)   # [E, 6, 3]
    g = np.linalg.solve(M, B[..., None])[..., 0]
    return node_mean(g, elem6, len(X))


def surface_divergence(X, elem6, v, n_node=None):
    """Surface divergence of a nodal vector field v[n, 3]: [n]."""
    if n_node is None:
        n_node = nodal_normals(X, elem6)
    d_xi, d_eta = derivatives(v, elem6)
    G = _solve_tangential(_systems(X, elem6, n_node), d_xi, d_eta)
    return node_mean(np.trace(G, axis1=-2, axis2=-1), elem6, len(X))


def laplace_beltrami(X, elem6, u, n_node=None):
    """Step 4 for any nodal scalar: div_S(grad_S u)."""
    if n_node is None:
        n_node = nodal_normals(X, elem6)
    return surface_divergence(X, elem6, surface_gradient(X, elem6, u, n_node), n_node)


def node_areas(X, elem6):
    """Barycentric nodal areas from the four flat sub-triangles of every
    element."""
    P = np.asarray(X, dtype=np.float64)[elem6]            # [E, 6, 3]
    A = np.zeros(len(X))
    for t in SUB_TRI:
        a = 0.5 * np.linalg.norm(np.cross(P[:, t[1]] - P[:, t[0]], P[:, t[2]] - P[:, t[0]]), axis=1)
        for k in t:
            np.add.at(A, elem6[:, k], a / 3.0)
    return A


def bending_fields(X, elem6):
    """All nodal fields of steps 1-5: dict of n (normals), K, KG, lapK, A."""
    X = np.asarray(X, dtype=np.float64)
    nn = nodal_normals(X, elem6)
    K, KG = curvatures(X, elem6, nn)
    lapK = laplace_beltrami(X, elem6, K, nn)
    return dict(n=nn, K=K, KG=KG, lapK=lapK, A=node_areas(X, elem6))


def bending_forces(X, elem6, k0):
    """Step 5: nodal bending forces [n, 3] of positions X[n, 3]."""
    f = bending_fields(X, elem6)
    dens = 0.5 * k0 * (f["lapK"] + 2.0 * f["K"] * (f["K"] ** 2 - f["KG"]))
    return (f["A"] * dens)[:, None] * f["n"]


def bending_energy(X, elem6, k0):
    """Eq. 6 on the nodal fields: (k0/2) sum_i K_i^2 A_i."""
    X = np.asarray(X, dtype=np.float64)
    K, _ = curvatures(X, elem6)
    return 0.5 * k0 * float(np.sum(K * K * node_areas(X, elem6)))


def forces_soa(X_soa, elem6, k0):
    """bending_forces for positions in the [3][n] layout of the solvers;
    returns the [3][n] force, flattened."""
    X = np.asarray(X_soa, dtype=np.float64).reshape(3, -1).T
    return np.ascontiguousarray(bending_forces(X, np.asarray(elem6).reshape(-1, 6), k0).T).ravel()
