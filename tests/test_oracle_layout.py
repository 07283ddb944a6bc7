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
