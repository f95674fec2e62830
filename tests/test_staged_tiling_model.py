"""A CPU model of the staged batch form's tiles (batch_staged.cu): a tile is a
stretch of 64 NC elements of one z-plane's interior rows, which lie
contiguously at the row pitch P; the producer passes the row and column of
the tile's first element, and each consumer thread carries its first element
over row ends.  The model checks, for ragged, narrow and multi-plane cells,
that every interior node is updated exactly once, that a thread's two nodes
lie in one row, and that every population's copy starts and ends on a
16-byte boundary inside the plane's ghost rows."""
import pytest


def pitch(nx):
    """The row pitch of the population layout (tlbm_bind_memory): 32 ceil((nx + 16) / 32)."""
    return 32 * ((nx + 16 + 31) // 32)


def tiles_of(nx, ny, nz, nc, elem):
    """(z, e0, length) of every tile of one instance, in launch order."""
    P = pitch(nx)
    run = ny * P
    tw = min(64 * nc, run)
    tpp = (run + tw - 1) // tw
    for z in range(nz):
        for k in range(tpp):
            e0 = k * tw
            yield z, e0, min(tw, run - e0), P, tw


@pytest.mark.parametrize("nx,ny,nz,nc,elem", [(33, 33, 1, 4, 2), (33, 33, 1, 8, 2), (1025, 7, 1, 4, 2),
                                               (1025, 5, 1, 8, 4), (129, 13, 1, 8, 2), (300, 5, 4, 4, 2),
                                               (9, 11, 7, 7, 2), (17, 8, 9, 4, 4), (385, 3, 2, 7, 2), (1, 3, 2, 4, 2)])
def test_tiles_cover_every_node_once(nx, ny, nz, nc, elem):
    A = 16 // elem
    seen = {}
    for z, e0, tw, P, tws in tiles_of(nx, ny, nz, nc, elem):
        assert tws % A == 0 and e0 % A == 0 and tw % 2 == 0
        y0 = e0 // P
        x0 = e0 - y0 * P
        for ex in (-1, 0, 1):
            lo = e0 - A if ex == 1 else e0
            end = (e0 + tw + (1 if ex == -1 else 0) + A - 1) // A * A
            assert lo % A == 0 and end % A == 0
            # inside the plane: ghost row y = -1 (P elements before) to ghost row y = ny
            assert -P <= lo and end <= ny * P + P
        for c in range(32 * nc):
            xr = 2 * c
            x, y = x0 + xr, y0
            while x >= P:
                x -= P
                y += 1
            active = xr < tw and x < nx
            both = xr + 1 < tw and x + 1 < nx
            assert not both or active
            if active:
                assert y * P + x == e0 + xr and 0 <= y < ny
                for xn in ((x, x + 1) if both else (x,)):
                    key = (xn, y, z)
                    assert key not in seen, key
                    seen[key] = True
    assert len(seen) == nx * ny * nz
