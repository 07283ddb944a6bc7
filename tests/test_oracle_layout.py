"""Pins of the interface-node layout (Sec. 3.1, 3.5)."""
import numpy as np
import pytest

from oracle.layout import interface_nodes, subdomains


@pytest.mark.parametrize("nx,ny,px,py", [(33, 33, 2, 2), (257, 257, 4, 4), (65, 129, 8, 2), (9, 9, 1, 4)])
def test_dirichlet_count_and_membership(nx, ny, px, py):
    nodes = interface_nodes(nx, ny, px, py, 0)
    M = (px - 1) * (ny - 2) + (py - 1) * (nx - 2) - (px - 1) * (py - 1)
    assert len(nodes) == M
    assert len({tuple(v) for v in nodes}) == M
    sx, sy = (nx - 1) // px, (ny - 1) // py
    for i, j in nodes:
        assert 0 < i < nx - 1 and 0 < j < ny - 1
        assert i % sx == 0 or j % sy == 0
    # every interior node on an interface line is listed
    want = {(i, j) for i in range(1, nx - 1) for j in range(1, ny - 1) if i % sx == 0 or j % sy == 0}
    assert want == {tuple(v) for v in nodes}


def test_known_counts():
    assert len(interface_nodes(33, 33, 2, 2, 0)) == 61
    assert len(interface_nodes(257, 257, 4, 4, 0)) == 1521
    assert len(interface_nodes(257, 257, 4, 4, 1)) == 2032


@pytest.mark.parametrize("nx,ny,px,py", [(33, 33, 2, 2), (257, 257, 4, 4), (17, 33, 4, 2)])
def test_periodic_count_and_membership(nx, ny, px, py):
    nodes = interface_nodes(nx, ny, px, py, 1)
    M = px * (ny - 1) + py * (nx - 1) - px * py
    assert len(nodes) == M and len({tuple(v) for v in nodes}) == M
    sx, sy = (nx - 1) // px, (ny - 1) // py
    want = {(i, j) for i in range(nx - 1) for j in range(ny - 1) if i % sx == 0 or j % sy == 0}
    assert want == {tuple(v) for v in nodes}


def test_order_vertical_lines_first():
    nodes = interface_nodes(9, 9, 2, 2, 0)
    assert [tuple(v) for v in nodes[:7]] == [(4, j) for j in range(1, 8)]
    assert [tuple(v) for v in nodes[7:]] == [(i, 4) for i in range(1, 8) if i != 4]


def test_subdomain_rims_are_interface_or_boundary():
    nx = ny = 17
    nodes = {tuple(v) for v in interface_nodes(nx, ny, 4, 2, 0)}
    subs = subdomains(nx, ny, 4, 2)
    assert len(subs) == 8
    covered = np.zeros((ny, nx), int)
    for (i0, i1, j0, j1) in subs:
        for i in range(i0, i1 + 1):
            for j in range(j0, j1 + 1):
                rim = i in (i0, i1) or j in (j0, j1)
                boundary = i in (0, nx - 1) or j in (0, ny - 1)
                if rim:
                    assert boundary or (i, j) in nodes
                else:
                    covered[j, i] += 1
    # interiors tile the non-interface interior exactly once
    for j in range(1, ny - 1):
        for i in range(1, nx - 1):
            assert covered[j, i] == (0 if (i, j) in nodes else 1)



@pytest.mark.parametrize("periodic", [0, 1])
@pytest.mark.parametrize("stride", [1, 2, 3, 5, 7])
def test_interface_sampling_reproduces_fields_linear_along_lines(periodic, stride):
    from oracle.layout import interface_sampling
    nx, ny, px, py, Lx, Ly = 33, 41, 4, 5, 2.0, 1.5
    sampled, fill = interface_sampling(nx, ny, px, py, periodic, stride, Lx, Ly)
    nodes = interface_nodes(nx, ny, px, py, periodic)
    # the identity mesh is linear along every line (with the period offset across the seam)
    est = np.stack([Lx * nodes[:, 0] / (nx - 1), Ly * nodes[:, 1] / (ny - 1)], 1)
    blank = est.copy()
    blank[~sampled] = np.nan
    assert np.allclose(fill(blank), est, atol=1e-14, rtol=0)
    if stride == 1:
        assert sampled.all()
    else:
        assert 0 < sampled.sum() < len(nodes)


def test_interface_sampling_counts_closed_form():
    from oracle.layout import interface_sampling
    # 33 x 33 split 4 x 4, stride 2: 3 vertical lines x 15 even rows (crossings are even) and
    # 3 horizontal lines x (15 even columns - 3 crossing columns)
    sampled, _ = interface_sampling(33, 33, 4, 4, 0, 2)
    assert sampled.sum() == 3 * 15 + 3 * 12
    # stride 3: rows 3, 6, .., 30 (10) plus the crossings 8 and 16 (24 is a multiple of 3) on
    # each vertical line; columns 3..30 step 3 (10) on each horizontal line, less the crossing
    # column 24 (crossings are listed on the vertical lines)
    sampled, _ = interface_sampling(33, 33, 4, 4, 0, 3)
    assert sampled.sum() == 3 * 12 + 3 * 9


def test_interface_sampling_brute_force_neighbours():
    """Every interpolated node equals the linear interpolation between the nearest sampled node
    (or boundary node) found by walking along its line in both directions."""
    from oracle.layout import interface_sampling
    nx, ny, px, py = 25, 17, 3, 2
    rng = np.random.default_rng(5)
    nodes = interface_nodes(nx, ny, px, py, 0)
    sampled, fill = interface_sampling(nx, ny, px, py, 0, 4)
    est = rng.normal(size=(len(nodes), 2))
    out = fill(est)
    ident = {(int(i), int(j)): m for m, (i, j) in enumerate(nodes)}
    vcols = {8, 16}
    for m, (i, j) in enumerate(nodes):
        if sampled[m]:
            assert np.array_equal(out[m], est[m])
            continue
        vertical = i in vcols
        def value(ii, jj):
            if (ii, jj) in ident and sampled[ident[(ii, jj)]]:
                return est[ident[(ii, jj)]]
            if ii in (0, nx - 1) or jj in (0, ny - 1):
                return np.array([ii / (nx - 1), jj / (ny - 1)])
            return None
        step = (0, 1) if vertical else (1, 0)
        lo, hi = 1, 1
        while value(i - lo * step[0], j - lo * step[1]) is None:
            lo += 1
        while value(i + hi * step[0], j + hi * step[1]) is None:
            hi += 1
        a = value(i - lo * step[0], j - lo * step[1])
        b = value(i + hi * step[0], j + hi * step[1])
        want = (hi * a + lo * b) / (lo + hi)
        assert np.allclose(out[m], want, atol=1e-14)


def test_uneven_split_lines_and_tiling():
    """41 nodes in 3 parts: lines at floor(40 I / 3) = 13, 26, parts of 13, 13 and 14 cells; the
    counts keep their closed forms and the subdomain interiors still tile the grid once."""
    from oracle.layout import split_line
    assert [split_line(I, 41, 3) for I in range(4)] == [0, 13, 26, 40]
    nodes = interface_nodes(41, 41, 3, 3, 0)
    assert len(nodes) == 2 * 39 + 2 * 39 - 4
    assert {int(i) for i, j in nodes[:2 * 39]} == {13, 26}
    per = interface_nodes(41, 41, 3, 3, 1)
    assert len(per) == 3 * 40 + 3 * 40 - 9
    subs = subdomains(41, 41, 3, 3)
    covered = np.zeros((41, 41), int)
    for (i0, i1, j0, j1) in subs:
        covered[j0 + 1:j1, i0 + 1:i1] += 1
    on_line = np.zeros((41, 41), bool)
    on_line[:, [0, 13, 26, 40]] = True
    on_line[[0, 13, 26, 40], :] = True
    assert np.array_equal(covered, (~on_line).astype(int))
    with pytest.raises(ValueError):
        interface_nodes(5, 5, 5, 1, 0)
