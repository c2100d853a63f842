"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only draws numbers and lays out element data: meshes (vertex
coordinates per element), per-element PDE coefficients, per-element degrees and
the scalar field coefficients of the nonlinear workload.  It holds none of the
integration method's arithmetic (no quadrature, basis, Jacobian or element
matrix code), so that the oracle and the CUDA path can both consume it without
sharing any of the method.

Random numbers come from a counter-based generator: SplitMix64's output
function (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to ``key + (n+1)*GOLDEN`` where ``key =
seed XOR (index * GOLDEN)``.  Every draw is addressed by (seed, index, n), so
any element's data can be regenerated alone (used for sampled parity checks on
full-size workloads).

Problem data follows Section 2 of the paper (coefficients c[iD][jD] constant
per element, as in the model problem of Section 5.1): a symmetric positive
definite diffusion tensor D, a convection vector b, a reaction c and a source
f per element.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_MESH = 1310
SEED_COEF = 1191
SEED_PMIX = 7
SEED_SURROGATE = 42

# coefficient rows of the SoA array [11][E]
COEF_ROWS = ("Dxx", "Dyy", "Dzz", "Dxy", "Dxz", "Dyz", "bx", "by", "bz", "c", "f")
N_COEF = len(COEF_ROWS)

# per-element degree weights of the mixed-degree mesh, p = 1..7
PMIX_WEIGHTS = (0.25, 0.2, 0.15, 0.15, 0.1, 0.1, 0.05)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def draw_u64(seed: int, index: np.ndarray, n: int) -> np.ndarray:
    """Draw number ``n`` (0-based) of the streams ``(seed, index)``; uint64."""
    with np.errstate(over="ignore"):
        idx = np.asarray(index, dtype=np.uint64)
        key = np.uint64(seed) ^ (idx * GOLDEN)
        return _mix64(key + np.uint64(n + 1) * GOLDEN)


def draw_uniform(seed: int, index: np.ndarray, n: int) -> np.ndarray:
    """Uniform in the open interval (0, 1): 53 random bits, offset by half an ulp."""
    z = draw_u64(seed, index, n)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def _jitter_vertices(grid_shape, h, seed, amp):
    """Vertex coordinates of a regular grid with interior vertices jittered.

    grid_shape = (nx+1, ny+1, nz+1) vertex counts; vertex id = ix + NX*(iy + NY*iz).
    Each coordinate of an interior vertex moves by U[-amp*h, amp*h]; boundary
    vertices stay put so the box stays a box.
    """
    NX, NY, NZ = grid_shape
    ix, iy, iz = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    ix = ix.transpose(2, 1, 0).ravel()  # vertex id order: ix fastest
    iy = iy.transpose(2, 1, 0).ravel()
    iz = iz.transpose(2, 1, 0).ravel()
    vid = ix + NX * (iy + NY * iz)
    xyz = np.stack([ix * h[0], iy * h[1], iz * h[2]], axis=1).astype(np.float64)
    interior = (ix > 0) & (ix < NX - 1) & (iy > 0) & (iy < NY - 1) & (iz > 0) & (iz < NZ - 1)
    if amp > 0:
        v = vid[interior]
        for c in range(3):
            u = draw_uniform(seed, v, c)
            xyz[interior, c] += (2.0 * u - 1.0) * amp * h[c]
    return xyz


def tet_mesh(n: int = 16, seed: int = SEED_MESH, jitter: float = 0.1) -> np.ndarray:
    """Unit cube, n^3 cells, each split into 6 Kuhn tetrahedra; coords [6 n^3][4][3].

    Cell (ix,iy,iz) -> cell id ix + n*(iy + n*iz); per cell the 6 tets follow the
    axis permutations (0,1,2),(0,2,1),(1,0,2),(1,2,0),(2,0,1),(2,1,0): vertices
    v0, v0+e_a, v0+e_a+e_b, v0+(1,1,1).  The signed volume of such a tet has the
    sign of the permutation, so for odd permutations local vertices 2 and 3 are
    swapped to keep every element positively oriented.
    """
    h = 1.0 / n
    xyz = _jitter_vertices((n + 1, n + 1, n + 1), (h, h, h), seed, jitter)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    odd = [False, True, True, False, False, True]
    N = n + 1
    cz, cy, cx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()  # cell id order: ix fastest
    base = np.stack([cx, cy, cz], axis=1)
    E = 6 * n ** 3
    conn = np.empty((n ** 3, 6, 4), dtype=np.int64)
    unit = np.eye(3, dtype=np.int64)

    def vid(ijk):
        return ijk[:, 0] + N * (ijk[:, 1] + N * ijk[:, 2])

    for k, (a, b, c) in enumerate(perms):
        v0 = base
        v1 = base + unit[a]
        v2 = v1 + unit[b]
        v3 = base + 1
        ids = [vid(v0), vid(v1), vid(v2), vid(v3)]
        if odd[k]:
            ids[2], ids[3] = ids[3], ids[2]
        conn[:, k, :] = np.stack(ids, axis=1)
    conn = conn.reshape(E, 4)
    return np.ascontiguousarray(xyz[conn])


def prism_grid_dims(E: int):
    """Hex grid nx = ny = ceil((E/2)^(1/3)), nz = ceil(E / (2 nx ny)), h = 1/nx."""
    nx = int(math.ceil((E / 2.0) ** (1.0 / 3.0) - 1e-9))
    nx = max(nx, 1)
    nz = max(int(math.ceil(E / (2.0 * nx * nx))), 1)
    return nx, nx, nz


def _vertex_coords(vid: np.ndarray, grid_shape, h, seed, amp) -> np.ndarray:
    """Coordinates of the given vertex ids of the jittered grid of
    _jitter_vertices (the same counter-based draws, addressed by vertex id)."""
    NX, NY, NZ = grid_shape
    ix, iy, iz = vid % NX, (vid // NX) % NY, vid // (NX * NY)
    xyz = np.stack([ix * h[0], iy * h[1], iz * h[2]], axis=1).astype(np.float64)
    interior = (ix > 0) & (ix < NX - 1) & (iy > 0) & (iy < NY - 1) & (iz > 0) & (iz < NZ - 1)
    if amp > 0:
        v = vid[interior]
        for c in range(3):
            u = draw_uniform(seed, v, c)
            xyz[interior, c] += (2.0 * u - 1.0) * amp * h[c]
    return xyz


def prism_mesh(E: int, seed: int = SEED_MESH, jitter: float = 0.1,
               dims=None, first: int = 0) -> np.ndarray:
    """Straight-edged 6-node prisms from a jittered hex grid; coords [E][6][3].

    Each hex (ix,iy,iz) (hex id ix + nx*(iy + ny*iz)) is cut along its xy
    diagonal into the prisms (v000, v100, v110 | same + z) and
    (v000, v110, v010 | same + z); local vertices 0..2 form the bottom
    triangle (counter-clockwise seen from +z) and 3..5 the top one.  The first
    E prisms are returned.  With jitter the quadrilateral side faces are not
    planar, so the map is bilinear in the vertical direction.

    ``first`` > 0 returns prisms first .. first+E-1 of the grid ``dims`` (a
    shard of a larger mesh, identical to slicing the whole mesh), computing
    only the vertices those prisms use.
    """
    if first > 0:
        if dims is None:
            raise ValueError("a shard (first > 0) needs the grid dims of the whole mesh")
        nx, ny, nz = dims
        if 2 * nx * ny * nz < first + E:
            raise ValueError("grid too small for the shard")
        h = 1.0 / nx
        NX, NY = nx + 1, ny + 1
        k = np.arange(first, first + E, dtype=np.int64)
        hid, side = k // 2, k % 2
        ix, iy, iz = hid % nx, (hid // nx) % ny, hid // (nx * ny)

        def vid(dx, dy, dz):
            return (ix + dx) + NX * ((iy + dy) + NY * (iz + dz))

        pa = np.stack([vid(0, 0, 0), vid(1, 0, 0), vid(1, 1, 0), vid(0, 0, 1), vid(1, 0, 1), vid(1, 1, 1)], axis=1)
        pb = np.stack([vid(0, 0, 0), vid(1, 1, 0), vid(0, 1, 0), vid(0, 0, 1), vid(1, 1, 1), vid(0, 1, 1)], axis=1)
        conn = np.where(side[:, None] == 0, pa, pb)
        xyz = _vertex_coords(conn.ravel(), (NX, NY, nz + 1), (h, h, h), seed, jitter)
        return np.ascontiguousarray(xyz.reshape(E, 6, 3))
    nx, ny, nz = dims if dims is not None else prism_grid_dims(E)
    if 2 * nx * ny * nz < E:
        raise ValueError("grid too small for E elements")
    h = 1.0 / nx
    NX, NY, NZ = nx + 1, ny + 1, nz + 1
    xyz = _jitter_vertices((NX, NY, NZ), (h, h, h), seed, jitter)
    nhex = (E + 1) // 2
    hid = np.arange(nhex, dtype=np.int64)
    ix = hid % nx
    iy = (hid // nx) % ny
    iz = hid // (nx * ny)

    def vid(dx, dy, dz):
        return (ix + dx) + NX * ((iy + dy) + NY * (iz + dz))

    v000, v100, v110, v010 = vid(0, 0, 0), vid(1, 0, 0), vid(1, 1, 0), vid(0, 1, 0)
    w000, w100, w110, w010 = vid(0, 0, 1), vid(1, 0, 1), vid(1, 1, 1), vid(0, 1, 1)
    pa = np.stack([v000, v100, v110, w000, w100, w110], axis=1)
    pb = np.stack([v000, v110, v010, w000, w110, w010], axis=1)
    conn = np.stack([pa, pb], axis=1).reshape(2 * nhex, 6)[:E]
    return np.ascontiguousarray(xyz[conn])


def prism_box_volume(E: int, dims=None) -> float:
    """Volume of the box of a full prism grid (valid when E = 2 nx ny nz)."""
    nx, ny, nz = dims if dims is not None else prism_grid_dims(E)
    h = 1.0 / nx
    return (nx * h) * (ny * h) * (nz * h)


# --------------------------------------------------------------------------
# coefficients
# --------------------------------------------------------------------------

def coefficients(E: int, seed: int = SEED_COEF, kind: str = "random",
                 first: int = 0) -> np.ndarray:
    """Per-element coefficients, SoA float64 [11][E] in COEF_ROWS order.

    kind="random": eigenvalues lam_k ~ U[0.1, 10] (draws 0..2), a rotation from
    the unit quaternion normalise(4 x N(0,1)) (draws 3..6, Box-Muller pairs),
    D = R diag(lam) R^T; b ~ U[-1,1]^3 (draws 7..9), c ~ U[0,1] (draw 10),
    f ~ U[-1,1] (draw 11).  kind="symmetric": same but b = 0.  kind="laplace":
    D = I, b = 0, c = 0, f = 1.  ``first`` offsets the element index, so any
    slice of a large workload can be regenerated on its own.
    """
    out = np.zeros((N_COEF, E), dtype=np.float64)
    if kind == "laplace":
        out[0:3] = 1.0
        out[10] = 1.0
        return out
    if kind not in ("random", "symmetric"):
        raise ValueError(kind)
    idx = np.arange(first, first + E, dtype=np.uint64)
    u = [draw_uniform(seed, idx, n) for n in range(12)]
    lam = [0.1 + 9.9 * u[k] for k in range(3)]
    r0 = np.sqrt(-2.0 * np.log(u[3]))
    r1 = np.sqrt(-2.0 * np.log(u[5]))
    qw = r0 * np.cos(2 * np.pi * u[4])
    qx = r0 * np.sin(2 * np.pi * u[4])
    qy = r1 * np.cos(2 * np.pi * u[6])
    qz = r1 * np.sin(2 * np.pi * u[6])
    nrm = np.sqrt(qw * qw + qx * qx + qy * qy + qz * qz)
    qw, qx, qy, qz = qw / nrm, qx / nrm, qy / nrm, qz / nrm
    R = np.empty((E, 3, 3))
    R[:, 0, 0] = 1 - 2 * (qy * qy + qz * qz)
    R[:, 0, 1] = 2 * (qx * qy - qz * qw)
    R[:, 0, 2] = 2 * (qx * qz + qy * qw)
    R[:, 1, 0] = 2 * (qx * qy + qz * qw)
    R[:, 1, 1] = 1 - 2 * (qx * qx + qz * qz)
    R[:, 1, 2] = 2 * (qy * qz - qx * qw)
    R[:, 2, 0] = 2 * (qx * qz - qy * qw)
    R[:, 2, 1] = 2 * (qy * qz + qx * qw)
    R[:, 2, 2] = 1 - 2 * (qx * qx + qy * qy)
    L = np.stack(lam, axis=1)
    D = np.matmul(R * L[:, None, :], R.transpose(0, 2, 1))
    out[0], out[1], out[2] = D[:, 0, 0], D[:, 1, 1], D[:, 2, 2]
    out[3], out[4], out[5] = D[:, 0, 1], D[:, 0, 2], D[:, 1, 2]
    if kind == "random":
        out[6] = 2 * u[7] - 1
        out[7] = 2 * u[8] - 1
        out[8] = 2 * u[9] - 1
    out[9] = u[10]
    out[10] = 2 * u[11] - 1
    return out


def mixed_degrees(E: int, seed: int = SEED_PMIX) -> np.ndarray:
    """Per-element degree p in 1..7 drawn with PMIX_WEIGHTS; int8 [E]."""
    u = draw_uniform(seed, np.arange(E, dtype=np.uint64), 0)
    cdf = np.cumsum(PMIX_WEIGHTS)
    cdf[-1] = 1.0
    return (np.searchsorted(cdf, u, side="right") + 1).clip(1, 7).astype(np.int8)


def field_coefficients(E: int, ns: int, seed: int = SEED_COEF + 1,
                       first: int = 0) -> np.ndarray:
    """Scalar field coefficients U_k ~ U[-1,1] per element; float64 [E][ns]."""
    idx = np.arange(first, first + E, dtype=np.uint64)
    return np.stack([2.0 * draw_uniform(seed, idx, 100 + k) - 1.0 for k in range(ns)], axis=1)


def dof_vectors(E: int, ns: int, seed: int = SEED_COEF + 3, first: int = 0) -> np.ndarray:
    """Per-element coefficient vectors x_e ~ U[-1,1]^ns that the element
    operators are applied to (the operator-apply workload); float64 [E][ns]."""
    return field_coefficients(E, ns, seed=seed, first=first)


def box_samples(n: int, box, seed: int = SEED_SURROGATE, first: int = 0) -> np.ndarray:
    """n points uniform in the box [u_min,u_max] x [g_min,g_max]; float64 [n][2]."""
    (u0, u1), (g0, g1) = box
    idx = np.arange(first, first + n, dtype=np.uint64)
    a = draw_uniform(seed, idx, 0)
    b = draw_uniform(seed, idx, 1)
    return np.stack([u0 + (u1 - u0) * a, g0 + (g1 - g0) * b], axis=1)


def elastic_coefficients(E: int, seed: int = SEED_COEF + 2, first: int = 0) -> np.ndarray:
    """Per-element isotropic material and body force, SoA float64 [5][E]:
    Young modulus U[1, 10], Poisson ratio U[0.05, 0.45], body force U[-1,1]^3."""
    idx = np.arange(first, first + E, dtype=np.uint64)
    u = [draw_uniform(seed, idx, n) for n in range(5)]
    out = np.empty((5, E))
    out[0] = 1.0 + 9.0 * u[0]
    out[1] = 0.05 + 0.4 * u[1]
    out[2] = 2 * u[2] - 1
    out[3] = 2 * u[3] - 1
    out[4] = 2 * u[4] - 1
    return out
