"""Host-side bookkeeping of multi-block domains (no GPU): splitting a
periodic box, ghost-layer contents and links."""
import numpy as np
import pytest

from paper_2209_15333_gb300 import multiblock as mb
from paper_2209_15333_gb300._lib import BC_HALO, BC_PERIODIC, HALO_WIDTH


def test_round_trip_and_ghost_contents():
    shape = (37, 26, 20)
    rng = np.random.default_rng(3)
    U = rng.standard_normal((5, shape[2], shape[1], shape[0]))
    blocks, links = mb.decompose_box(shape, (2, 1, 2))
    assert len(blocks) == 4
    parts = mb.scatter(U, blocks)
    assert np.array_equal(mb.gather(parts, blocks, shape), U)
    H = HALO_WIDTH
    for b, (blk, Ub) in enumerate(zip(blocks, parts)):
        assert Ub.shape == (5, blk["grid"][2], blk["grid"][1], blk["grid"][0])
        assert blk["bc_lo"] == (BC_HALO, BC_PERIODIC, BC_HALO)
        # the ghost layers a face receives equal the neighbour's interior layers
        # that the exchange copies: low face <- layers [n-2H, n-H), high face <- [H, 2H)
        for d, axis in ((0, 3), (2, 1)):
            for side in (0, 1):
                c = links[b, d, side]
                Uc = parts[c]
                nd = Ub.shape[axis]
                ncd = Uc.shape[axis]
                dst = np.take(Ub, range(0, H) if side == 0 else range(nd - H, nd), axis=axis)
                src = np.take(Uc, range(ncd - 2 * H, ncd - H) if side == 0 else range(H, 2 * H), axis=axis)
                assert np.array_equal(dst, src)


def test_links_periodic_neighbours():
    blocks, links = mb.decompose_box((40, 40, 40), (3, 2, 1))
    pos = {blk["pos"]: b for b, blk in enumerate(blocks)}
    assert links[pos[(0, 0, 0)], 0, 0] == pos[(2, 0, 0)]
    assert links[pos[(2, 1, 0)], 0, 1] == pos[(0, 1, 0)]
    assert links[pos[(1, 1, 0)], 1, 1] == pos[(1, 0, 0)]
    assert (links[:, 2, :] == -1).all()


def test_too_thin_blocks_rejected():
    with pytest.raises(ValueError):
        mb.decompose_box((16, 32, 32), (2, 1, 1))
