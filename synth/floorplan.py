"""Seeded synthetic occupancy maps (uint8, 1 = occupied, 0 = free), row-major [H][W].

Cell (j, i) is row j (+y) and column i (+x).  These maps stand in for the public floor
plans the paper evaluates on (Section IV); only their structure (rooms, corridors, thin
walls, doorways, clutter) is imitated.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def free_components(occ: np.ndarray) -> int:
    """Number of 4-connected components of free space."""
    from scipy import ndimage
    _, n = ndimage.label(occ == 0)
    return int(n)


def rooms_map(seed: int, size: int = 64, rooms: int = 4, door: int = 3,
              box_frac: float = 0.05) -> np.ndarray:
    """rooms x rooms rectangular rooms with 1-cell walls, one `door`-cell doorway per shared
    wall, plus random 1-3-cell square boxes until `box_frac` of the free cells is covered.

    Wall lines sit at multiples of size // rooms and at size - 1.  Boxes never touch a
    doorway (1-cell clearance) and never disconnect free space.
    """
    rng = _rng(seed)
    occ = np.zeros((size, size), np.uint8)
    step = size // rooms
    lines = [r * step for r in range(rooms)] + [size - 1]
    for l in lines:
        occ[l, :] = 1
        occ[:, l] = 1
    doors = np.zeros_like(occ, dtype=bool)
    # vertical shared walls (x = lines[1..rooms-1]) inside each room row, and horizontal ones
    for a in range(1, rooms):
        for b in range(rooms):
            lo, hi = lines[b] + 1, lines[b + 1] - 1          # interior span of the room row
            off = int(rng.integers(lo, hi - door + 2))
            occ[off:off + door, lines[a]] = 0
            doors[max(off - 1, 0):off + door + 1, max(lines[a] - 1, 0):lines[a] + 2] = True
            off = int(rng.integers(lo, hi - door + 2))
            occ[lines[a], off:off + door] = 0
            doors[max(lines[a] - 1, 0):lines[a] + 2, max(off - 1, 0):off + door + 1] = True
    n_free0 = int((occ == 0).sum())
    covered = 0
    tries = 0
    while covered < box_frac * n_free0 and tries < 10000:
        tries += 1
        s = int(rng.integers(1, 4))
        j = int(rng.integers(1, size - s - 1))
        i = int(rng.integers(1, size - s - 1))
        patch = occ[j:j + s, i:i + s]
        if patch.any() or doors[j - 1:j + s + 1, i - 1:i + s + 1].any():
            continue
        occ[j:j + s, i:i + s] = 1
        if free_components(occ) != 1:
            occ[j:j + s, i:i + s] = 0
            continue
        covered += s * s
    return occ


def office_map(seed: int, size: int = 512, cell: float = 0.05,
               corridor_m=(1.5, 2.5), room_m=(3.0, 8.0), wall_m: float = 0.1,
               door_m: float = 0.9) -> np.ndarray:
    """Office floor plan: a grid of corridors (width U(corridor_m)) whose blocks are split
    into rooms with sides U(room_m); walls are `wall_m` thick; every room has one door of
    at least `door_m` onto an adjacent corridor, so free space is connected.
    """
    rng = _rng(seed)
    c = lambda m: max(1, int(round(m / cell)))
    wall = c(wall_m)
    occ = np.ones((size, size), np.uint8)

    def bands(n):
        """Alternate corridor / block bands along one axis: [(start, end, is_corridor)]."""
        out, pos = [], wall
        is_corr = True
        while pos < n - wall:
            if is_corr:
                w = c(rng.uniform(*corridor_m))
            else:
                w = c(rng.uniform(2 * room_m[0], 2 * room_m[1]))
            end = min(pos + w, n - wall)
            if not is_corr and end - pos < c(room_m[0]) + 2 * wall:
                # too thin for a room: widen the previous corridor instead
                s, _, _ = out[-1]
                out[-1] = (s, end, True)
                pos = end
                continue
            out.append((pos, end, is_corr))
            pos = end
            is_corr = not is_corr
        if not out[-1][2]:
            # close with a corridor strip carved from the last block if possible
            s, e, _ = out[-1]
            cw = c(corridor_m[0])
            if e - s > cw + c(room_m[0]) + 2 * wall:
                out[-1] = (s, e - cw, False)
                out.append((e - cw, e, True))
        return out

    ybands, xbands = bands(size), bands(size)
    for (y0, y1, yc) in ybands:
        for (x0, x1, xc) in xbands:
            if yc or xc:
                occ[y0:y1, x0:x1] = 0
    door = c(door_m)
    for (y0, y1, yc) in ybands:
        if yc:
            continue
        for (x0, x1, xc) in xbands:
            if xc:
                continue
            # the block [y0,y1) x [x0,x1) is surrounded by corridors; split into room rows
            h = y1 - y0
            rows = [(y0, y1, 'both')]
            if h >= 2 * c(room_m[0]):
                cut = y0 + h // 2 + int(rng.integers(-h // 8, h // 8 + 1))
                rows = [(y0, cut, 'low'), (cut, y1, 'high')]
            for (ry0, ry1, face) in rows:
                cols, pos = [], x0
                while pos < x1:
                    w = c(rng.uniform(*room_m))
                    if x1 - (pos + w) < c(room_m[0]):
                        w = x1 - pos
                    cols.append((pos, pos + w))
                    pos += w
                for (rx0, rx1) in cols:
                    # interior: inset by one wall thickness on every side (walls between
                    # neighbouring rooms are then two wall thicknesses; the corridor side
                    # keeps one thickness of wall)
                    iy0, iy1, ix0, ix1 = ry0 + wall, ry1 - wall, rx0 + wall, rx1 - wall
                    if iy1 - iy0 < 2 or ix1 - ix0 < 2:
                        continue
                    occ[iy0:iy1, ix0:ix1] = 0
                    # door onto a corridor: the corridor side facing this room
                    sides = []
                    if face in ('low', 'both'):
                        sides.append('low')
                    if face in ('high', 'both'):
                        sides.append('high')
                    side = sides[int(rng.integers(len(sides)))]
                    span = ix1 - ix0
                    dl = min(door, span)
                    d0 = ix0 + int(rng.integers(0, span - dl + 1))
                    if side == 'low':
                        occ[ry0:iy0, d0:d0 + dl] = 0
                    else:
                        occ[iy1:ry1, d0:d0 + dl] = 0
    occ[:wall, :] = 1
    occ[-wall:, :] = 1
    occ[:, :wall] = 1
    occ[:, -wall:] = 1
    return occ


def crop(occ: np.ndarray, j0: int, i0: int, h: int, w: int) -> np.ndarray:
    """A sub-map with its own 1-cell occupied border, so it is a closed floor plan."""
    out = occ[j0:j0 + h, i0:i0 + w].copy()
    out[0, :] = 1
    out[-1, :] = 1
    out[:, 0] = 1
    out[:, -1] = 1
    return out
