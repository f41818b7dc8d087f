"""Q1 finite-element matrices and pattern assembly (inputs of the method, Eq. 1).

A pattern is a square (2D) or a cube (3D) of m x m (x m) equal Q1 elements of side h.
Nodes are numbered x-fastest: n = i + (m+1) * (j + (m+1) * k); dof = node * dpn + component.
This module only states the discretised problem K u = f that the method is given.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

GAUSS2 = (-1.0 / np.sqrt(3.0), 1.0 / np.sqrt(3.0))


def _corner_signs(dim):
    """Reference-element corner signs, corner index = i + 2 j (+ 4 k)."""
    return np.array([[2 * ((a >> d) & 1) - 1 for d in range(dim)] for a in range(2 ** dim)], dtype=float)


def _shape_grads(xi, dim):
    """d N_a / d xi_d at reference point xi for the 2^dim bilinear/trilinear shape functions."""
    s = _corner_signs(dim)
    g = np.empty((2 ** dim, dim))
    for a in range(2 ** dim):
        for d in range(dim):
            v = 0.5 ** dim * s[a, d]
            for e in range(dim):
                if e != d:
                    v *= 1.0 + s[a, e] * xi[e]
            g[a, d] = v
    return g


def q1_laplace(dim: int, h: float = 1.0, kappa: float = 1.0) -> np.ndarray:
    """Element conductivity matrix kappa * int grad N_a . grad N_b over a cube of side h (2x2(x2) Gauss)."""
    n = 2 ** dim
    K = np.zeros((n, n))
    jac = h / 2.0
    for xi in itertools.product(GAUSS2, repeat=dim):
        dN = _shape_grads(np.array(xi), dim) / jac
        K += kappa * dN @ dN.T * jac ** dim
    return K


def lame(E: float, nu: float):
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    return lam, mu


def elastic_D(E: float, nu: float) -> np.ndarray:
    """Isotropic 3D constitutive matrix, Voigt order (xx, yy, zz, yz, xz, xy), engineering shear strain."""
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def q1_elastic3d(h: float = 1.0, E: float = 1.0, nu: float = 0.3) -> np.ndarray:
    """24x24 trilinear hexahedron stiffness (full 2x2x2 Gauss), dof = corner * 3 + component."""
    D = elastic_D(E, nu)
    K = np.zeros((24, 24))
    jac = h / 2.0
    for xi in itertools.product(GAUSS2, repeat=3):
        dN = _shape_grads(np.array(xi), 3) / jac
        B = np.zeros((6, 24))
        for a in range(8):
            gx, gy, gz = dN[a]
            B[0, 3 * a + 0] = gx
            B[1, 3 * a + 1] = gy
            B[2, 3 * a + 2] = gz
            B[3, 3 * a + 1] = gz
            B[3, 3 * a + 2] = gy
            B[4, 3 * a + 0] = gz
            B[4, 3 * a + 2] = gx
            B[5, 3 * a + 0] = gy
            B[5, 3 * a + 1] = gx
        K += B.T @ D @ B * jac ** 3
    return K


def grid_nodes(dim: int, m: int, h: float) -> np.ndarray:
    """Coordinates of the (m+1)^dim nodes of a pattern, x-fastest."""
    ax = np.arange(m + 1) * h
    mesh = np.meshgrid(*([ax] * dim), indexing="ij")
    # x fastest: flatten in Fortran order over (x, y, z)
    return np.stack([c.flatten(order="F") for c in mesh], axis=1)


def element_connectivity(dim: int, m: int) -> np.ndarray:
    """(n_elem, 2^dim) node indices; corner index a = i + 2 j + 4 k as in _corner_signs."""
    n1 = m + 1
    if dim == 2:
        e_idx = np.array([(i, j) for j in range(m) for i in range(m)])
    else:
        e_idx = np.array([(i, j, k) for k in range(m) for j in range(m) for i in range(m)])
    conn = np.empty((len(e_idx), 2 ** dim), dtype=np.int64)
    for a in range(2 ** dim):
        off = [(a >> d) & 1 for d in range(dim)]
        node = np.zeros(len(e_idx), dtype=np.int64)
        stride = 1
        for d in range(dim):
            node += (e_idx[:, d] + off[d]) * stride
            stride *= n1
        conn[:, a] = node
    return conn


def assemble(conn: np.ndarray, Ke: np.ndarray, n_nodes: int, dpn: int) -> sp.csr_matrix:
    """Assemble identical element matrices (dof = corner * dpn + comp) into a CSR matrix."""
    n_e, n_c = conn.shape
    edofs = (conn[:, :, None] * dpn + np.arange(dpn)[None, None, :]).reshape(n_e, n_c * dpn)
    rows = np.repeat(edofs, n_c * dpn, axis=1).ravel()
    cols = np.tile(edofs, (1, n_c * dpn)).ravel()
    vals = np.tile(Ke.ravel(), n_e)
    K = sp.coo_matrix((vals, (rows, cols)), shape=(n_nodes * dpn, n_nodes * dpn)).tocsr()
    K.sum_duplicates()
    K.sort_indices()
    return K


def boundary_nodes(dim: int, m: int) -> np.ndarray:
    """Nodes on the surface of the square/cube, increasing order."""
    idx = np.stack(np.meshgrid(*([np.arange(m + 1)] * dim), indexing="ij"), axis=-1).reshape(-1, dim, order="F")
    on = np.any((idx == 0) | (idx == m), axis=1)
    return np.nonzero(on)[0].astype(np.int32)


@dataclass
class Pattern:
    """One meshed pattern: the free (floating) stiffness K in the pattern frame plus its trace set."""
    name: str
    dim: int
    m: int
    h: float
    dpn: int
    physics: str                 # "heat" or "elastic"
    material: dict
    coords: np.ndarray           # (n_nodes, dim)
    K: sp.csr_matrix             # (n_nodes*dpn)^2, symmetric, singular (floating)
    bnd_nodes: np.ndarray        # int32, nodes on the surface (those that may carry multipliers)
    kernel_dim: int              # 1 (heat) or 6 (3D elasticity)

    @property
    def n_nodes(self):
        return self.coords.shape[0]

    @property
    def n_dofs(self):
        return self.n_nodes * self.dpn

    @property
    def n_b(self):
        return len(self.bnd_nodes) * self.dpn


def heat_pattern(m: int, H: float = 1.0, kappa: float = 1.0, dim: int = 2, name: str = "") -> Pattern:
    h = H / m
    conn = element_connectivity(dim, m)
    coords = grid_nodes(dim, m, h)
    K = assemble(conn, q1_laplace(dim, h, kappa), coords.shape[0], 1)
    return Pattern(name or f"heat{dim}d_{m}_k{kappa:g}", dim, m, h, 1, "heat", {"kappa": kappa},
                   coords, K, boundary_nodes(dim, m), 1)


def elastic_pattern(m: int, H: float = 1.0, E: float = 1.0, nu: float = 0.3, name: str = "") -> Pattern:
    h = H / m
    conn = element_connectivity(3, m)
    coords = grid_nodes(3, m, h)
    K = assemble(conn, q1_elastic3d(h, E, nu), coords.shape[0], 3)
    return Pattern(name or f"elastic3d_{m}", 3, m, h, 3, "elastic", {"E": E, "nu": nu},
                   coords, K, boundary_nodes(3, m), 6)
