"""The lane-to-link maps of the four-lanes-per-node kernels against the D3Q19 link table.

The D3Q19 order of the step: link 0 at rest; links 2p + 1 and 2p + 2 of pair p move along
+c_p and -c_p, with c_0..c_2 the axes and c_3..c_8 = x + y, x - y, x + z, x - z, y + z,
y - z (the order the moment sums of Eq. 10 use).

* Forward step (k_step_quad): lane j = 0, 1, 2 of a node holds axis pair j and the two
  diagonal pairs of the plane (a, b) = (x, y), (y, z), (x, z), i.e. pairs pd and pd + 1
  with pd = 3, 7, 5; lane 3 holds the rest link.  Slot directions: slots 0-1 +-e_j,
  slots 2-5 +(e_a + e_b), -(e_a + e_b), +(e_a - e_b), -(e_a - e_b).
* Reverse step (k_adj_step_ws): lane j takes pairs j, j + 4, j + 8, with each pair's
  direction read from bit masks over p.

Both maps are restated here as the kernels compute them and checked to cover each link
exactly once with its own direction; swapped planes or a flipped mask bit fail.  No GPU
code runs.
"""
DIRS = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
        (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
        (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]


def quad_forward_slots(j, pd_of=(3, 7, 5)):
    """(link, direction) of lane j's six slots, as the forward quad step builds them."""
    ai = j if j < 3 else 0
    da = 1 if j == 1 else 0
    db = 1 if j == 0 else 2
    pd = pd_of[j] if j < 3 else 3
    out = []
    for sl in range(6):
        if sl < 2:
            c = 1 if sl == 0 else -1
            d = (c if ai == 0 else 0, c if ai == 1 else 0, c if ai == 2 else 0)
            link = 2 * ai + 1 + sl
        else:
            sa = -1 if sl & 1 else 1
            sb = sa if sl < 4 else -sa
            d = (sa if da == 0 else 0, (sa if da == 1 else 0) + (sb if db == 1 else 0), sb if db == 2 else 0)
            link = 2 * pd + 1 + (sl - 2)
        if j == 3:
            link, d = 0, (0, 0, 0)
        out.append((link, d))
    return out


def pair_dir(p, masks=(0x079, 0x19A, 0x1E4)):
    cx = (masks[0] >> p) & 1
    cy = ((masks[1] >> p) & 1) * (-1 if p == 4 else 1)
    cz = ((masks[2] >> p) & 1) * (-1 if p in (6, 8) else 1)
    return (cx, cy, cz)


def test_forward_quad_lanes_cover_every_link_once():
    seen = {}
    for j in range(4):
        for link, d in quad_forward_slots(j):
            if j == 3:
                assert link == 0 and d == (0, 0, 0)
                continue
            assert link not in seen, link
            seen[link] = d
    assert sorted(seen) == list(range(1, 19))
    for link, d in seen.items():
        assert d == DIRS[link], (link, d)


def test_forward_quad_swapped_planes_fail():
    seen = {}
    for j in range(3):
        for link, d in quad_forward_slots(j, pd_of=(3, 5, 7)):
            seen[link] = d
    assert any(d != DIRS[link] for link, d in seen.items())


def test_reverse_pair_directions_match_the_link_table():
    for p in range(9):
        assert pair_dir(p) == DIRS[2 * p + 1], p
        assert tuple(-c for c in pair_dir(p)) == DIRS[2 * p + 2], p
    lanes = {j: [p for p in (j, j + 4, j + 8) if p <= 8] for j in range(4)}
    assert sorted(p for ps in lanes.values() for p in ps) == list(range(9))
    # a flipped mask bit breaks a direction
    assert any(pair_dir(p, masks=(0x079, 0x19B, 0x1E4)) != DIRS[2 * p + 1] for p in range(9))
