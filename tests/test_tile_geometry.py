"""Host-side model of the stencil kernels' tile geometry (csrc/pf_stencil.cuh, csrc/pf_internal.cuh): 32 x 8 tiles,
halo boxes x0-4 .. x0+35 / y0-1 .. y0+8, the stencil plane of (TX + 2) x (TY + 2) slots filled by the centre threads
and the halo slots, mirror images on the zero-flux x / y sides (Eq. 4), and the edge nodes that take the last column
and row of a 2^k + 1 grid into the tiles next to them.

For every grid shape the model checks that each node of an x-y plane is computed exactly once, that every stencil
plane slot an output reads holds the right neighbour (the node itself or its mirror image), and that every halo-box
offset the face data reads is inside the box and names the right node.  The constants and index formulas are the
kernels' own; a change to one of them must be made in both places."""
import pytest

TX, TY = 32, 8
PW, HBX, HBY, NTH = TX + 2, TX + 8, TY + 2, TX * TY
NHALO = 2 * (TX + 2) + 2 * TY


def edge_x(nx, edges):
    return edges and nx > TX and nx % TX == 1


def edge_y(ny, edges):
    return edges and ny > TY and ny % TY == 1


def tiles_x(nx, edges):
    return nx // TX if edge_x(nx, edges) else (nx + TX - 1) // TX


def tiles_y(ny, edges):
    return ny // TY if edge_y(ny, edges) else (ny + TY - 1) // TY


def mirror(g, n):
    if g < 0:
        return 1
    if g < n:
        return g
    if g == n:
        return n - 2
    return -1


def cs(lx, ly):
    return (ly + 1) * PW + (lx + 1)


def halo_pos(h):
    if h < TX + 2:
        return h - 1, -1
    h -= TX + 2
    if h < TX + 2:
        return h - 1, TY
    h -= TX + 2
    if h < TY:
        return -1, h
    return TX, h - TY


def box_off(gi, gj, x0, y0, nx, ny):
    mi, mj = mirror(gi, nx), mirror(gj, ny)
    if mi < 0 or mj < 0:
        return -1
    return (mj - y0 + 1) * HBX + (mi - x0 + 4)


def box_node(o, x0, y0):
    return (o % HBX) - 4 + x0, (o // HBX) - 1 + y0


def tile_outputs(nx, ny, x0, y0, edges):
    """(node, plane slot, neighbour offsets, box offset, side flags) of every output of one tile, and the plane."""
    ee = edge_x(nx, edges) and x0 + TX == nx - 1
    en = edge_y(ny, edges) and y0 + TY == ny - 1
    plane = {}
    for t in range(NTH):
        lx, ly = t % TX, t // TX
        o = box_off(x0 + lx, y0 + ly, x0, y0, nx, ny)
        plane[cs(lx, ly)] = box_node(o, x0, y0) if o >= 0 else None
    for h in range(NHALO):
        hx, hy = halo_pos(h)
        o = box_off(x0 + hx, y0 + hy, x0, y0, nx, ny)
        plane[cs(hx, hy)] = box_node(o, x0, y0) if o >= 0 else None
    outs = []
    for t in range(NTH):
        gi, gj = x0 + t % TX, y0 + t // TX
        if gi < nx and gj < ny:
            outs.append(((gi, gj), cs(t % TX, t // TX), (1, -1, PW, -PW), box_off(gi, gj, x0, y0, nx, ny),
                         (gi > 0, gj > 0, gi < nx - 1, gj < ny - 1)))
    if ee or en:
        for h in range(NHALO):
            hx, hy = halo_pos(h)
            es = -1
            if ee and hx == TX and 0 <= hy < TY and y0 + hy < ny:
                es = hy
            if en and hy == TY and hx >= 0 and (hx < TX or ee) and x0 + hx < nx:
                es = TY + hx
            if es < 0:
                continue
            assert 0 <= es < TY + TX + 1
            gi, gj = x0 + hx, y0 + hy
            west, south, east, north = gi > 0, gj > 0, gi < nx - 1, gj < ny - 1
            outs.append(((gi, gj), cs(hx, hy), (1 if east else -1, -1, PW if north else -PW, -PW),
                         box_off(gi, gj, x0, y0, nx, ny), (west, south, east, north)))
    return plane, outs


def check_grid(nx, ny, edges):
    count = {}
    for ty in range(tiles_y(ny, edges)):
        for tx in range(tiles_x(nx, edges)):
            x0, y0 = tx * TX, ty * TY
            plane, outs = tile_outputs(nx, ny, x0, y0, edges)
            assert len(plane) == PW * (TY + 2)
            for (gi, gj), pc, nb, o, (west, south, east, north) in outs:
                count[(gi, gj)] = count.get((gi, gj), 0) + 1
                assert plane[pc] == (gi, gj)
                want = [(mirror(gi + 1, nx), gj), (mirror(gi - 1, nx), gj), (gi, mirror(gj + 1, ny)),
                        (gi, mirror(gj - 1, ny))]
                for d, w in zip(nb, want):
                    assert 0 <= pc + d < PW * (TY + 2) and plane[pc + d] == w
                assert 0 <= o < HBX * HBY and box_node(o, x0, y0) == (gi, gj)
                for oo, w in [(o + 1 if east else o - 1, want[0]), (o - 1 if west else o + 1, want[1]),
                              (o + HBX if north else o - HBX, want[2]), (o - HBX if south else o + HBX, want[3])]:
                    assert 0 <= oo < HBX * HBY and box_node(oo, x0, y0) == w
    assert all(count.get((i, j), 0) == 1 for i in range(nx) for j in range(ny))


SIZES = [3, 9, 16, 17, 29, 32, 33, 34, 49, 63, 65, 97, 129, 257]


@pytest.mark.parametrize("edges", [0, 1])
def test_every_node_once_and_neighbours_right(edges):
    for nx in SIZES:
        for ny in SIZES:
            check_grid(nx, ny, edges)


def test_edge_tiles_drop_the_narrow_tiles():
    # 257 = 8 * 32 + 1 columns and 32 * 8 + 1 rows: 9 x 33 tiles without edge nodes, 8 x 32 with them
    assert (tiles_x(257, 0), tiles_y(257, 0)) == (9, 33)
    assert (tiles_x(257, 1), tiles_y(257, 1)) == (8, 32)
    assert (tiles_x(33, 1), tiles_y(33, 1)) == (1, 4)
    # nothing to take in when the extent is not one more than a multiple of the tile, or fits one tile
    assert (tiles_x(49, 1), tiles_y(50, 1), tiles_x(17, 1), tiles_y(9, 1)) == (2, 7, 1, 1)
