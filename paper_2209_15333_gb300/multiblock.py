"""Splitting a periodic box into blocks with ghost layers (multi-block
domains on one GPU, cfd_set_halo_links).

Host-side bookkeeping only: which part of the box each block holds, its
extended grid (H = CFD_HALO_WIDTH ghost layers on every face of a split
direction), the boundary conditions (HALO on split faces, periodic
elsewhere) and the neighbour links.  Arrays are [var][k][j][i] (x fastest).
"""
import numpy as np

from ._lib import BC_HALO, BC_PERIODIC, HALO_WIDTH


def _cuts(n, parts):
    base, extra = divmod(n, parts)
    edges = [0]
    for p in range(parts):
        edges.append(edges[-1] + base + (1 if p < extra else 0))
    return edges


def decompose_box(shape, parts, H=HALO_WIDTH):
    """shape (nx, ny, nz) of a periodic box, parts (px, py, pz).  Returns a
    list of block dicts, in x-fastest block order:
      origin (i0, j0, k0) and size (interior nodes per direction),
      grid (nx, ny, nz) of the extended block, bc_lo / bc_hi,
      halo (ghost layers per direction: H if split else 0),
    and the links array [nblocks][3][2]."""
    n = list(shape)
    edges = [_cuts(n[d], parts[d]) for d in range(3)]
    for d in range(3):
        if parts[d] > 1 and min(np.diff(edges[d])) < H + 1:
            raise ValueError("blocks along direction %d are thinner than the ghost layers" % d)
    blocks = []
    index = {}
    for bk in range(parts[2]):
        for bj in range(parts[1]):
            for bi in range(parts[0]):
                bidx = (bi, bj, bk)
                origin = [edges[d][bidx[d]] for d in range(3)]
                size = [edges[d][bidx[d] + 1] - edges[d][bidx[d]] for d in range(3)]
                halo = [H if parts[d] > 1 else 0 for d in range(3)]
                grid = [size[d] + 2 * halo[d] for d in range(3)]
                bc = [BC_HALO if parts[d] > 1 else BC_PERIODIC for d in range(3)]
                index[bidx] = len(blocks)
                blocks.append(dict(pos=bidx, origin=origin, size=size, halo=halo, grid=tuple(grid),
                                   bc_lo=tuple(bc), bc_hi=tuple(bc)))
    links = -np.ones((len(blocks), 3, 2), dtype=np.int32)
    for b, blk in enumerate(blocks):
        for d in range(3):
            if parts[d] == 1:
                continue
            for side, step in ((0, -1), (1, 1)):
                nb = list(blk["pos"])
                nb[d] = (nb[d] + step) % parts[d]
                links[b, d, side] = index[tuple(nb)]
    return blocks, links


def _index(blk, shape):
    """periodic source indices of the extended block along each direction"""
    idx = []
    for d in range(3):
        lo = blk["origin"][d] - blk["halo"][d]
        idx.append(np.arange(lo, lo + blk["grid"][d]) % shape[d])
    return idx


def scatter(U, blocks):
    """Per-block extended arrays [5][nz][ny][nx] from the box field U (ghost
    layers filled with the periodic neighbours' values)."""
    shape = (U.shape[3], U.shape[2], U.shape[1])
    out = []
    for blk in blocks:
        ix, iy, iz = _index(blk, shape)
        out.append(np.ascontiguousarray(U[:, iz][:, :, iy][:, :, :, ix]))
    return out


def gather(parts_U, blocks, shape):
    """The box field from the blocks' interiors."""
    nx, ny, nz = shape
    U = np.empty((parts_U[0].shape[0], nz, ny, nx))
    for Ub, blk in zip(parts_U, blocks):
        (i0, j0, k0), (sx, sy, sz), (hx, hy, hz) = blk["origin"], blk["size"], blk["halo"]
        U[:, k0:k0 + sz, j0:j0 + sy, i0:i0 + sx] = Ub[:, hz:hz + sz, hy:hy + sy, hx:hx + sx]
    return U
