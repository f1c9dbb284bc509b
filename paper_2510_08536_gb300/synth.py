"""Seeded synthetic inputs for the repartitioning path.

This module stands in for the CFD application that sits *above* the library:
it generates a uniform hexahedral box mesh, decomposes it into ``k`` boxes
(one per CPU rank, like ``decomposePar``), and gives every rank the arrays an
OpenFOAM rank would hold after assembling a pressure equation:

* an LDU matrix: ``diag[n_r]``, ``upper[F_r]``, ``lower[F_r]`` over the
  owner/neighbour face addressing ``lower_addr`` / ``upper_addr`` (owner <
  neighbour, faces ordered by owner then neighbour);
* processor-interface entries ``(iface_row, iface_nbr_rank, iface_nbr_col)``
  with one coefficient each.

The mesh, its decomposition and the coefficient draws are the workload of
the paper's evaluation (Sec. 4: a uniform cubic grid, decomposed into equal
boxes), made synthetic. Nothing here repartitions, permutes or solves: the
module holds no arithmetic of the method, so both the CUDA path and the CPU
oracle can take their inputs from it.

Conventions (all seeded, all decomposition independent):

* cells are numbered lexicographically, x fastest, both globally and inside
  a rank's sub-box;
* global faces are numbered x-faces, then y-faces, then z-faces, then the
  Dirichlet boundary faces at x = 0; all coefficient draws follow this global
  order, so the assembled physical matrix does not depend on ``k``;
* the stored matrix is the SPD pressure operator: off-diagonal ``-a_f``,
  diagonal ``sum_f a_f + 2 a_b (cells at x = 0) + shift`` with
  ``shift = 1e-3``;
* the staging layout of one rank is ``[diag n_r | upper F_r | lower F_r |
  iface E_r]`` (``lower`` left out in symmetric mode); ranks follow each
  other in rank order.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DIAG_SHIFT = 1.0e-3


@dataclasses.dataclass
class RankLDU:
    """One CPU rank's LDU sparsity plus the mesh bookkeeping behind it."""

    n_cells: int
    lower_addr: np.ndarray      # int32 [F]  owner (local id)
    upper_addr: np.ndarray      # int32 [F]  neighbour (local id), > owner
    iface_row: np.ndarray       # int32 [E]  local row
    iface_nbr_rank: np.ndarray  # int32 [E]  rank owning the column
    iface_nbr_col: np.ndarray   # int32 [E]  column, local to that rank
    cell_gid: np.ndarray        # int64 [n]  global lexicographic cell id
    face_gid: np.ndarray        # int64 [F]  global face id of each face
    iface_face_gid: np.ndarray  # int64 [E]  global face id behind each entry

    @property
    def n_faces(self) -> int:
        return int(self.lower_addr.shape[0])

    @property
    def n_iface(self) -> int:
        return int(self.iface_row.shape[0])


@dataclasses.dataclass
class BoxMesh:
    """A uniform nx*ny*nz hex mesh decomposed into px*py*pz box ranks."""

    nx: int
    ny: int
    nz: int
    px: int
    py: int
    pz: int
    ranks: list

    @property
    def k(self) -> int:
        return len(self.ranks)

    @property
    def n_cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_fx(self) -> int:
        return (self.nx - 1) * self.ny * self.nz

    @property
    def n_fy(self) -> int:
        return self.nx * (self.ny - 1) * self.nz

    @property
    def n_fz(self) -> int:
        return self.nx * self.ny * (self.nz - 1)

    @property
    def n_internal_faces(self) -> int:
        return self.n_fx + self.n_fy + self.n_fz

    @property
    def n_boundary_faces(self) -> int:
        return self.ny * self.nz

    def merged_gid(self) -> np.ndarray:
        """Global cell id of every merged row (ranks concatenated)."""
        return np.concatenate([r.cell_gid for r in self.ranks])

    def staging_size(self, symmetric: bool = False) -> int:
        per = 1 if symmetric else 2
        return sum(r.n_cells + per * r.n_faces + r.n_iface for r in self.ranks)

    def nnz(self) -> int:
        return sum(r.n_cells + 2 * r.n_faces + r.n_iface for r in self.ranks)


def _bounds(n: int, p: int) -> list:
    return [(i * n) // p for i in range(p + 1)]


def box_mesh(nx: int, ny: int, nz: int, px: int = 1, py: int = 1, pz: int = 1) -> BoxMesh:
    """Build the mesh and its box decomposition.

    Rank id is ``rx + px*(ry + py*rz)``. Sub-box extents follow
    ``floor(i*n/p)`` bounds, so uneven splits are allowed.
    """
    if min(nx, ny, nz) < 1 or min(px, py, pz) < 1:
        raise ValueError("mesh and decomposition sizes must be positive")
    if px > nx or py > ny or pz > nz:
        raise ValueError("more ranks than cells along an axis")
    bx, by, bz = _bounds(nx, px), _bounds(ny, py), _bounds(nz, pz)
    fx = (nx - 1) * ny * nz
    fy = nx * (ny - 1) * nz

    def rank_id(rx, ry, rz):
        return rx + px * (ry + py * rz)

    ranks = []
    for rz in range(pz):
        for ry in range(py):
            for rx in range(px):
                x0, x1 = bx[rx], bx[rx + 1]
                y0, y1 = by[ry], by[ry + 1]
                z0, z1 = bz[rz], bz[rz + 1]
                sx, sy, sz = x1 - x0, y1 - y0, z1 - z0
                c, b, a = np.meshgrid(np.arange(sz), np.arange(sy), np.arange(sx), indexing="ij")
                a = a.ravel().astype(np.int64)
                b = b.ravel().astype(np.int64)
                c = c.ravel().astype(np.int64)
                lid = a + sx * (b + sy * c)
                gi, gj, gk = a + x0, b + y0, c + z0
                cell_gid = gi + nx * (gj + ny * gk)

                owners, nbrs, gids = [], [], []
                m = a + 1 < sx
                owners.append(lid[m]); nbrs.append(lid[m] + 1)
                gids.append(gi[m] + (nx - 1) * (gj[m] + ny * gk[m]))
                m = b + 1 < sy
                owners.append(lid[m]); nbrs.append(lid[m] + sx)
                gids.append(fx + gi[m] + nx * (gj[m] + (ny - 1) * gk[m]))
                m = c + 1 < sz
                owners.append(lid[m]); nbrs.append(lid[m] + sx * sy)
                gids.append(fx + fy + gi[m] + nx * (gj[m] + ny * gk[m]))
                owner = np.concatenate(owners)
                nbr = np.concatenate(nbrs)
                gid = np.concatenate(gids)
                order = np.lexsort((nbr, owner))  # upper-triangular face order

                # processor interfaces: one entry per face shared with another rank
                ent = []  # (nbr_rank, row, col, face gid)
                if rx > 0:
                    q = rank_id(rx - 1, ry, rz); sq = bx[rx] - bx[rx - 1]
                    m = a == 0
                    ent.append((q, lid[m], (sq - 1) + sq * (b[m] + sy * c[m]),
                                (gi[m] - 1) + (nx - 1) * (gj[m] + ny * gk[m])))
                if rx + 1 < px:
                    q = rank_id(rx + 1, ry, rz); sq = bx[rx + 2] - bx[rx + 1]
                    m = a == sx - 1
                    ent.append((q, lid[m], 0 + sq * (b[m] + sy * c[m]),
                                gi[m] + (nx - 1) * (gj[m] + ny * gk[m])))
                if ry > 0:
                    q = rank_id(rx, ry - 1, rz); sq = by[ry] - by[ry - 1]
                    m = b == 0
                    ent.append((q, lid[m], a[m] + sx * ((sq - 1) + sq * c[m]),
                                fx + gi[m] + nx * ((gj[m] - 1) + (ny - 1) * gk[m])))
                if ry + 1 < py:
                    q = rank_id(rx, ry + 1, rz); sq = by[ry + 2] - by[ry + 1]
                    m = b == sy - 1
                    ent.append((q, lid[m], a[m] + sx * (0 + sq * c[m]),
                                fx + gi[m] + nx * (gj[m] + (ny - 1) * gk[m])))
                if rz > 0:
                    q = rank_id(rx, ry, rz - 1); sq = bz[rz] - bz[rz - 1]
                    m = c == 0
                    ent.append((q, lid[m], a[m] + sx * (b[m] + sy * (sq - 1)),
                                fx + fy + gi[m] + nx * (gj[m] + ny * (gk[m] - 1))))
                if rz + 1 < pz:
                    q = rank_id(rx, ry, rz + 1)
                    m = c == sz - 1
                    ent.append((q, lid[m], a[m] + sx * (b[m] + sy * 0),
                                fx + fy + gi[m] + nx * (gj[m] + ny * gk[m])))
                ent.sort(key=lambda t: t[0])  # neighbour rank ascending, rows ascending inside
                if ent:
                    irow = np.concatenate([e[1] for e in ent])
                    irank = np.concatenate([np.full(e[1].shape[0], e[0], np.int64) for e in ent])
                    icol = np.concatenate([e[2] for e in ent])
                    igid = np.concatenate([e[3] for e in ent])
                else:
                    irow = irank = icol = igid = np.zeros(0, np.int64)
                ranks.append(RankLDU(
                    n_cells=int(sx * sy * sz),
                    lower_addr=owner[order].astype(np.int32),
                    upper_addr=nbr[order].astype(np.int32),
                    iface_row=irow.astype(np.int32),
                    iface_nbr_rank=irank.astype(np.int32),
                    iface_nbr_col=icol.astype(np.int32),
                    cell_gid=cell_gid,
                    face_gid=gid[order],
                    iface_face_gid=igid,
                ))
    return BoxMesh(nx, ny, nz, px, py, pz, ranks)


def face_coeffs(mesh: BoxMesh, sigma: float | None = None, seed: int = 100) -> np.ndarray:
    """Face coefficients a_f for every internal face, then every x=0 face.

    ``sigma=None`` gives the uniform case a_f = area/dist = 1 (unit spacing);
    otherwise a_f ~ lognormal(0, sigma) drawn in global face order from
    ``numpy.random.default_rng(seed)``.
    """
    total = mesh.n_internal_faces + mesh.n_boundary_faces
    if sigma is None:
        return np.ones(total, np.float64)
    rng = np.random.default_rng(seed)
    return rng.lognormal(0.0, sigma, size=total)


def global_diag(mesh: BoxMesh, a: np.ndarray, shift: float = DIAG_SHIFT) -> np.ndarray:
    """Assembled diagonal over global lexicographic cells (the application's
    pressure assembly: every face adds its coefficient to both cells, every
    Dirichlet face adds twice its coefficient, plus a constant shift)."""
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    fx, fy, fz = mesh.n_fx, mesh.n_fy, mesh.n_fz
    d = np.full((nz, ny, nx), shift, np.float64)
    ax = a[:fx].reshape(nz, ny, nx - 1)
    d[:, :, :-1] += ax
    d[:, :, 1:] += ax
    ay = a[fx:fx + fy].reshape(nz, ny - 1, nx)
    d[:, :-1, :] += ay
    d[:, 1:, :] += ay
    az = a[fx + fy:fx + fy + fz].reshape(nz - 1, ny, nx)
    d[:-1, :, :] += az
    d[1:, :, :] += az
    ab = a[fx + fy + fz:].reshape(nz, ny)
    d[:, :, 0] += 2.0 * ab
    return d.ravel()


class Assembler:
    """Turns face coefficients into the staging buffer in one gather.

    The index table maps every staging slot to an entry of
    ``[diag (global cells) | -a (global faces)]``; it is built once per mesh.
    """

    def __init__(self, mesh: BoxMesh, symmetric: bool = False):
        self.mesh = mesh
        self.symmetric = symmetric
        n = mesh.n_cells
        parts = []
        for r in mesh.ranks:
            parts.append(r.cell_gid)
            parts.append(n + r.face_gid)
            if not symmetric:
                parts.append(n + r.face_gid)
            parts.append(n + r.iface_face_gid)
        dtype = np.int32 if n + mesh.n_internal_faces + mesh.n_boundary_faces < 2**31 else np.int64
        self.index = np.concatenate(parts).astype(dtype)

    def staging(self, a: np.ndarray, shift: float = DIAG_SHIFT, out: np.ndarray | None = None) -> np.ndarray:
        ext = np.concatenate([global_diag(self.mesh, a, shift), -a])
        if out is None:
            return ext[self.index]
        np.take(ext, self.index, out=out)
        return out

    def rank_slices(self, staging: np.ndarray):
        """Split a staging buffer into per-rank (diag, upper, lower, iface) views."""
        out = []
        pos = 0
        for r in self.mesh.ranks:
            n, f, e = r.n_cells, r.n_faces, r.n_iface
            diag = staging[pos:pos + n]; pos += n
            upper = staging[pos:pos + f]; pos += f
            if self.symmetric:
                lower = None
            else:
                lower = staging[pos:pos + f]; pos += f
            iface = staging[pos:pos + e]; pos += e
            out.append((diag, upper, lower, iface))
        return out


# ---------------------------------------------------------------- momentum (non-symmetric) systems

MOMENTUM_U0 = 1.0   # velocity scale (cells per unit time)
MOMENTUM_CT = 0.1   # transient term V / dt on the diagonal


def _face_flux(mesh: BoxMesh, u0: float) -> np.ndarray:
    """Volume flux through every internal face (global face order, owner -> neighbour
    along +x / +y / +z, unit area) of the velocity field
    u = u0 (sin(pi X) cos(pi Y), -cos(pi X) sin(pi Y), sin(2 pi Z) / 4) at the face centre,
    with X, Y, Z the cell-unit coordinates scaled to [0, 1]: a cavity-like vortex."""
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx - 1), indexing="ij")
    X, Y = (i + 1.0) / nx, (j + 0.5) / ny
    fx = u0 * np.sin(np.pi * X) * np.cos(np.pi * Y)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny - 1), np.arange(nx), indexing="ij")
    X, Y = (i + 0.5) / nx, (j + 1.0) / ny
    fy = -u0 * np.cos(np.pi * X) * np.sin(np.pi * Y)
    k, j, i = np.meshgrid(np.arange(nz - 1), np.arange(ny), np.arange(nx), indexing="ij")
    Z = (k + 1.0) / nz
    fz = 0.25 * u0 * np.sin(2.0 * np.pi * Z) + 0.0 * i
    return np.concatenate([fx.ravel(), fy.ravel(), fz.ravel()])


def momentum_staging(mesh: BoxMesh, sigma: float = 0.5, seed: int = 100, u0: float = MOMENTUM_U0,
                     ct: float = MOMENTUM_CT) -> np.ndarray:
    """Staging buffer (general storage: [diag | upper | lower | iface] per rank) of an
    upwind convection-diffusion (momentum) matrix: per internal face, diffusion
    a_f ~ lognormal(0, sigma) (seeded, global face order) and flux F_f from
    ``_face_flux``; the owner row couples to the neighbour with -(a_f + max(-F_f, 0)),
    the neighbour row to the owner with -(a_f + max(F_f, 0)); the diagonal is ct plus
    the magnitudes of its row's off-diagonals (row sums = ct). Interface entries take
    the value of the side their row lies on."""
    n = mesh.n_cells
    nf = mesh.n_internal_faces
    a = np.random.default_rng(seed).lognormal(0.0, sigma, size=nf)
    F = _face_flux(mesh, u0)
    up = -(a + np.maximum(-F, 0.0))   # row = owner (low side), col = neighbour
    lo = -(a + np.maximum(F, 0.0))    # row = neighbour (high side), col = owner
    owner, nbr = _global_face_cells(mesh)
    diag = ct + np.bincount(owner, weights=-up, minlength=n) + np.bincount(nbr, weights=-lo, minlength=n)
    ext = np.concatenate([diag, up, lo])
    parts = []
    for r in mesh.ranks:
        parts.append(r.cell_gid)
        parts.append(n + r.face_gid)
        parts.append(n + nf + r.face_gid)
        if r.n_iface:
            row_g = r.cell_gid[r.iface_row]
            col_g = np.empty(r.n_iface, np.int64)
            for q in np.unique(r.iface_nbr_rank):
                m = r.iface_nbr_rank == q
                col_g[m] = mesh.ranks[q].cell_gid[r.iface_nbr_col[m]]
            low_side = row_g < col_g
            parts.append(np.where(low_side, n + r.iface_face_gid, n + nf + r.iface_face_gid))
    return ext[np.concatenate(parts)]


def _global_face_cells(mesh: BoxMesh):
    """Global owner (low side) and neighbour cell of every internal face."""
    nx, ny, nz = mesh.nx, mesh.ny, mesh.nz
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx - 1), indexing="ij")
    ox = (i + nx * (j + ny * k)).ravel()
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny - 1), np.arange(nx), indexing="ij")
    oy = (i + nx * (j + ny * k)).ravel()
    k, j, i = np.meshgrid(np.arange(nz - 1), np.arange(ny), np.arange(nx), indexing="ij")
    oz = (i + nx * (j + ny * k)).ravel()
    owner = np.concatenate([ox, oy, oz])
    nbr = np.concatenate([ox + 1, oy + nx, oz + nx * ny])
    return owner, nbr


def uniform_vector(mesh: BoxMesh, seed: int) -> np.ndarray:
    """U[-1, 1] over global cells (seeded), returned in merged row order."""
    g = np.random.default_rng(seed).uniform(-1.0, 1.0, size=mesh.n_cells)
    return g[mesh.merged_gid()]


def batch_shapes(count: int = 256, lo: int = 8000, hi: int = 300000, seed: int = 0):
    """Box dimensions of ``count`` independent systems.

    Cell counts are log-uniform in [lo, hi]; two aspect ratios are uniform in
    [1, 4]; the three extents are (c, c*r1, c*r2) with c = (N/(r1*r2))^(1/3),
    rounded (at least 2) and put in a random axis order.
    """
    rng = np.random.default_rng(seed)
    dims = []
    for _ in range(count):
        n = math.exp(rng.uniform(math.log(lo), math.log(hi)))
        r1, r2 = rng.uniform(1.0, 4.0, size=2)
        c = (n / (r1 * r2)) ** (1.0 / 3.0)
        d = [max(2, int(round(c))), max(2, int(round(c * r1))), max(2, int(round(c * r2)))]
        perm = rng.permutation(3)
        dims.append(tuple(int(d[i]) for i in perm))
    return dims


# Named workloads: (mesh extents, rank grid, coefficient sigma or None)
WORKLOADS = {
    "plain_fp64_32": dict(n=(32, 32, 32), p=(2, 2, 2), sigma=None),
    "update_128": dict(n=(128, 128, 128), p=(4, 4, 4), sigma=0.5),
    "mixed_256": dict(n=(256, 256, 256), p=(8, 4, 4), sigma=1.0),
    "adjoint_128": dict(n=(128, 128, 128), p=(4, 4, 4), sigma=0.5),
    # profiling size: every pass larger than L2, a few GB on the device
    "profile_192": dict(n=(192, 192, 192), p=(3, 3, 3), sigma=1.0),
    # non-symmetric momentum system on the headline mesh (momentum_staging)
    "momentum_256": dict(n=(256, 256, 256), p=(8, 4, 4), sigma=0.5),
}


def workload_mesh(name: str) -> BoxMesh:
    w = WORKLOADS[name]
    return box_mesh(*w["n"], *w["p"])


class Batch:
    """Independent box systems (one rank each, Dirichlet at each x = 0 face)
    for the batched form: shapes from ``batch_shapes``; every draw uses one
    generator per step, systems in order."""

    def __init__(self, count: int = 256, lo: int = 8000, hi: int = 300000, seed: int = 0):
        self.dims = batch_shapes(count, lo, hi, seed)
        self.meshes = [box_mesh(*d) for d in self.dims]
        self.systems = [m.ranks[0] for m in self.meshes]
        self.assemblers = [Assembler(m) for m in self.meshes]

    @property
    def n_rows(self) -> int:
        return sum(m.n_cells for m in self.meshes)

    def staging(self, sigma: float = 0.5, seed: int = 100) -> np.ndarray:
        rng = np.random.default_rng(seed)
        parts = []
        for m, asm in zip(self.meshes, self.assemblers):
            a = rng.lognormal(0.0, sigma, size=m.n_internal_faces + m.n_boundary_faces)
            parts.append(asm.staging(a))
        return np.concatenate(parts)

    def rhs(self, seed: int = 0) -> np.ndarray:
        rng = np.random.default_rng(seed)
        return np.concatenate([rng.uniform(-1.0, 1.0, size=m.n_cells)[m.merged_gid()] for m in self.meshes])
