"""Seeded synthetic inputs: conductor geometries and mesh parameters.

This module only builds inputs (boxes, mesh parameters, request streams).  It
holds none of the method's arithmetic, so that both the CUDA path and the CPU
oracle can take the same inputs from it.

Geometry is in micrometres.  A box is ``(lo[3], hi[3], conductor_id)``; mesh
parameters are ``dict(h=..., ratio=..., h_min=...)`` (maximum panel edge,
geometric grading ratio toward face edges, first cell size at an edge; ratio
1 means uniform).

Random draws use SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), so every workload is a pure
function of its seed.

The paper's own test case (Sec. 5, Table 2: two crossing 4x1x1 bars in a
grounded 40x40x10 box) is reproduced by ``paper_two_bars``; the paper used no
public dataset, so every other geometry is synthetic interconnect of the
shapes and sizes below.
"""
from __future__ import annotations

import math

EPS_R_SIO2 = 3.9
MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator: 64-bit state advanced by the golden-ratio
    increment, output through two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] inclusive."""
        return lo + int(self.uniform() * (hi - lo + 1)) if hi > lo else lo

    def exponential(self, rate: float) -> float:
        return -math.log(1.0 - self.uniform()) / rate


def _box(lo, hi, cid):
    return (tuple(float(v) for v in lo), tuple(float(v) for v in hi), int(cid))


# --------------------------------------------------------------------------
# Fixed structures
# --------------------------------------------------------------------------

def two_bars():
    """Two parallel 1.0 x 0.2 x 0.2 um bars, 0.1 um apart; uniform panels of
    at most 0.06 um: 17 x 4 cells on the long faces, 4 x 4 on the ends,
    304 panels per bar, N = 608."""
    boxes = [_box((0.0, 0.0, 0.0), (1.0, 0.2, 0.2), 0),
             _box((0.0, 0.3, 0.0), (1.0, 0.5, 0.2), 1)]
    return boxes, dict(h=0.06, ratio=1.0, h_min=0.0)


def crossing_bus_2x2(h: float = 0.03, ratio: float = 1.5, h_min: float = 0.005):
    """2x2 crossing bus: two 0.1 x 0.1 um wires along x on layer 1 (z in
    [0, 0.1]) crossing two along y on layer 2 (z in [0.3, 0.4]); widths and
    spacings 0.1 um, vertical gap 0.2 um, length 1.0 um, centred.  Panels are
    graded toward face edges (h_min 5 nm, ratio 1.5, h 30 nm): N = 6264."""
    boxes = []
    cid = 0
    for y0 in (-0.15, 0.05):
        boxes.append(_box((-0.5, y0, 0.0), (0.5, y0 + 0.1, 0.1), cid))
        cid += 1
    for x0 in (-0.15, 0.05):
        boxes.append(_box((x0, -0.5, 0.3), (x0 + 0.1, 0.5, 0.4), cid))
        cid += 1
    return boxes, dict(h=h, ratio=ratio, h_min=h_min)


def bus_3layer_5x5x5(seed: int = 20220323, h: float = 0.04, ratio: float = 1.5,
                     h_min: float = 0.008):
    """Three crossing layers (directions x, y, x) of five wires each; widths
    and spacings uniform in [0.08, 0.16] um from the seed; thickness 0.15 um;
    inter-layer gap 0.15 um; each wire spans the crossing layers plus a
    0.2 um overhang at both ends; panels graded toward face edges (h_min
    8 nm, ratio 1.5, h 40 nm).  15 conductors, N = 23172."""
    rng = SplitMix64(seed)
    t, gap, over = 0.15, 0.15, 0.2
    layers = []
    for _ in range(3):
        ws = [rng.uniform(0.08, 0.16) for _ in range(5)]
        ss = [rng.uniform(0.08, 0.16) for _ in range(4)]
        pos, x = [], 0.0
        for i in range(5):
            pos.append((x, x + ws[i]))
            x += ws[i] + (ss[i] if i < 4 else 0.0)
        span = x
        pos = [(a - span / 2, b - span / 2) for a, b in pos]
        layers.append((pos, span))
    boxes, cid = [], 0
    for li, (pos, _span) in enumerate(layers):
        z0 = li * (t + gap)
        cross = [layers[j][1] for j in range(3) if j != li]
        half = max(cross) / 2 + over
        for a, b in pos:
            if li % 2 == 0:   # along x
                boxes.append(_box((-half, a, z0), (half, b, z0 + t), cid))
            else:             # along y
                boxes.append(_box((a, -half, z0), (b, half, z0 + t), cid))
            cid += 1
    return boxes, dict(h=h, ratio=ratio, h_min=h_min)


def cube(a: float = 1.0, n: int = 4):
    """Isolated cube of side a, uniform n x n panels per face."""
    return [_box((0.0, 0.0, 0.0), (a, a, a), 0)], dict(h=a / n, ratio=1.0, h_min=0.0)


def parallel_plates(L: float = 1.0, t: float = 0.02, g: float = 0.1, h: float = 0.1):
    """Two square L x L plates of thickness t, gap g, stacked along z."""
    boxes = [_box((0.0, 0.0, 0.0), (L, L, t), 0),
             _box((0.0, 0.0, t + g), (L, L, 2 * t + g), 1)]
    return boxes, dict(h=h, ratio=1.0, h_min=0.0)


def paper_two_bars():
    """Sec. 5, single-dielectric case: net 1 from (-2,-0.5,1) to (2,0.5,2),
    net 2 from (-0.5,-2,3) to (0.5,2,4), inside a grounded box from
    (-20,-20,0) to (20,20,10) (um)."""
    return ([_box((-2.0, -0.5, 1.0), (2.0, 0.5, 2.0), 0),
             _box((-0.5, -2.0, 3.0), (0.5, 2.0, 4.0), 1)],
            _box((-20.0, -20.0, 0.0), (20.0, 20.0, 10.0), 2))


def voxel_sphere_panels(R: float, nvox: int, outer: bool):
    """Surface panels of a staircase body made of cubic voxels of side
    R / nvox: every voxel entirely inside the sphere of radius R (outer=False)
    or every voxel that meets the closed ball (outer=True).  Returns
    (axis list, geo list of (c, lo0, hi0, lo1, hi1), cond list), one panel per
    exposed voxel face."""
    v = R / nvox
    m = nvox + 1
    inside = set()
    for i in range(-m, m):
        for j in range(-m, m):
            for k in range(-m, m):
                lo = (i * v, j * v, k * v)
                hi = ((i + 1) * v, (j + 1) * v, (k + 1) * v)
                far2 = sum(max(abs(lo[d]), abs(hi[d])) ** 2 for d in range(3))
                near2 = sum((0.0 if lo[d] <= 0.0 <= hi[d] else min(abs(lo[d]), abs(hi[d]))) ** 2
                            for d in range(3))
                if (outer and near2 < R * R) or (not outer and far2 <= R * R):
                    inside.add((i, j, k))
    axis, geo, cond = [], [], []
    for (i, j, k) in sorted(inside):
        idx = (i, j, k)
        for d in range(3):
            for s in (-1, 1):
                nb = list(idx)
                nb[d] += s
                if tuple(nb) in inside:
                    continue
                p, q = [a for a in range(3) if a != d]
                c = (idx[d] + (1 if s > 0 else 0)) * v
                axis.append(d)
                geo.append((c, idx[p] * v, (idx[p] + 1) * v, idx[q] * v, (idx[q] + 1) * v))
                cond.append(0)
    return axis, geo, cond


# --------------------------------------------------------------------------
# Batches of small structures and request streams
# --------------------------------------------------------------------------

def random_bars(rng: SplitMix64, n_target: float):
    """2-6 bars, parallel (along x, side by side in y) or crossing (alternate
    layers along x and y); dimensions uniform in [0.05, 1.0] um (lengths)
    and [0.05, 0.3] um (cross sections); mesh size chosen so that the panel
    count is near n_target."""
    nb = rng.randint(2, 6)
    crossing = rng.uniform() < 0.5
    boxes = []
    area = 0.0
    y = 0.0
    z = 0.0
    for b in range(nb):
        L = rng.uniform(0.3, 1.0)
        w = rng.uniform(0.05, 0.3)
        t = rng.uniform(0.05, 0.3)
        s = rng.uniform(0.05, 0.3)
        if crossing and b % 2 == 1:
            lo, hi = (-w / 2 + y * 0.0, -L / 2, z), (w / 2, L / 2, z + t)
            z += t + s
        elif crossing:
            lo, hi = (-L / 2, -w / 2, z), (L / 2, w / 2, z + t)
            z += t + s
        else:
            lo, hi = (-L / 2, y, 0.0), (L / 2, y + w, t)
            y += w + s
        boxes.append(_box(lo, hi, b))
        area += 2 * (L * w + L * t + w * t)
    h = math.sqrt(area / n_target)
    return boxes, dict(h=h, ratio=1.0, h_min=0.0)


def batch_small_structures(seed: int = 4242, count: int = 512, n_lo: int = 200, n_hi: int = 3000):
    """``count`` independent structures with log-uniform target panel counts
    in [n_lo, n_hi]."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        n_target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        out.append(random_bars(rng, n_target))
    return out


def bus_structure(rng: SplitMix64, n_target: float):
    """Random 2-15 conductor bus: parallel wires on one layer, or two crossing
    layers; widths and spacings in [0.08, 0.16] um."""
    nc = rng.randint(2, 15)
    crossing = nc >= 4 and rng.uniform() < 0.5
    t = 0.1
    boxes = []
    area = 0.0
    if crossing:
        n1 = nc // 2
        groups = [(n1, 0), (nc - n1, 1)]
    else:
        groups = [(nc, 0)]
    cid = 0
    for count, layer in groups:
        pos = []
        x = 0.0
        for _ in range(count):
            w = rng.uniform(0.08, 0.16)
            pos.append((x, x + w))
            x += w + rng.uniform(0.08, 0.16)
        span = x
        L = max(1.0, span + 0.4)
        z0 = layer * 0.3
        for a, b in pos:
            a -= span / 2
            b -= span / 2
            if layer == 0:
                lo, hi = (-L / 2, a, z0), (L / 2, b, z0 + t)
            else:
                lo, hi = (a, -L / 2, z0), (b, L / 2, z0 + t)
            boxes.append(_box(lo, hi, cid))
            area += 2 * (L * (b - a) + L * t + (b - a) * t)
            cid += 1
    h = math.sqrt(area / n_target)
    return boxes, dict(h=h, ratio=1.0, h_min=0.0)


def serving_requests(seed: int = 777, count: int = 1000, rate_per_s: float = 50.0,
                     n_lo: int = 500, n_hi: int = 30000):
    """Poisson arrivals: list of (arrival time in s, boxes, mesh params)."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(rate_per_s)
        n_target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        boxes, params = bus_structure(rng, n_target)
        out.append((t, boxes, params))
    return out


def stack_3layer_5wires(h: float = 0.25, h_outer: float = 0.6):
    """A layered dielectric stack (Sec. 4; the paper's own six-conductor case
    is not public, so this one is synthetic): a 12 x 12 x 4 um enclosure with
    grounded bottom and top and insulating sides (the boundary conditions of
    the paper's multi-dielectric experiment, Sec. 5), three layers of
    eps_r 3.9 / 2.5 / 7.0 (oxide, low-k, nitride) split at z = 1 and 2.5, and
    five parallel 1 x 10 x 0.5 um wires at 2 um pitch inside the middle one.
    Returns a dict of the gbem_stack fields and the boxes; with the default
    cells the system has 5520 equations."""
    face_ground, face_neumann = -1, -2
    return {
        "lo": [-6.0, -6.0, 0.0], "hi": [6.0, 6.0, 4.0], "z": [0.0, 1.0, 2.5, 4.0], "eps_r": [3.9, 2.5, 7.0],
        "face_bc": [face_neumann] * 4 + [face_ground, face_ground],
        "boxes": [([-4.0 + 2 * i, -5.0, 1.5], [-3.0 + 2 * i, 5.0, 2.0], i) for i in range(5)],
        "h": h, "h_outer": h_outer,
    }


def icosphere(R: float = 1.0, level: int = 2, centre=(0.0, 0.0, 0.0)):
    """Flat triangles inscribed in a sphere of radius R: the icosahedron,
    each face split into four by its edge midpoints `level` times, the new
    vertices pushed out to the sphere.  Returns float64[20 * 4**level, 9]
    (each row the three vertices, counter-clockwise seen from outside)."""
    import numpy as np
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6),
         (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    tris = np.array([[v[a], v[b], v[c]] for a, b, c in f])
    for _ in range(level):
        a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
        ab, bc, ca = a + b, b + c, c + a
        ab /= np.linalg.norm(ab, axis=1, keepdims=True)
        bc /= np.linalg.norm(bc, axis=1, keepdims=True)
        ca /= np.linalg.norm(ca, axis=1, keepdims=True)
        tris = np.concatenate([np.stack([a, ab, ca], 1), np.stack([ab, b, bc], 1), np.stack([ca, bc, c], 1),
                               np.stack([ab, bc, ca], 1)])
    return (R * tris + np.asarray(centre, dtype=np.float64)).reshape(-1, 9)


def trapezoid_bar(x0: float, x1: float, w_bottom: float, w_top: float, z0: float, z1: float,
                  n_len: int = 8, n_w: int = 3, n_h: int = 3, y0: float = 0.0):
    """Flat triangles on the closed surface of a straight wire along x whose
    cross-section is a trapezoid (bottom width w_bottom at z0, top width w_top
    at z1, centred on y0), as etched interconnect is.  Every face is a grid of
    quadrilaterals (n_len along the wire, n_w across, n_h up the sides) cut
    into two triangles; vertices shared by faces are the same numbers, so
    touching triangles share them exactly.  Returns float64[n, 9]."""
    import numpy as np
    canon = {}

    def vert(x, y, z):
        key = (round(x, 12), round(y, 12), round(z, 12))
        return canon.setdefault(key, (float(x), float(y), float(z)))

    def lerp(a, b, t, n):
        return b if t == n else a + (b - a) * t / n

    def section(s, t):
        """Point (y, z) of the cross-section at width fraction s/n_w of the
        level t/n_h."""
        z = lerp(z0, z1, t, n_h)
        w = lerp(w_bottom, w_top, t, n_h)
        return lerp(y0 - 0.5 * w, y0 + 0.5 * w, s, n_w), z

    tris = []

    def quad(a, b, c, d):   # counter-clockwise seen from outside
        tris.append(a + b + c)
        tris.append(a + c + d)

    xs = [lerp(x0, x1, i, n_len) for i in range(n_len + 1)]
    # the four long faces, each a strip along x: bottom, right side, top, left side
    ring = ([section(s, 0) for s in range(n_w + 1)] + [section(n_w, t) for t in range(1, n_h + 1)] +
            [section(s, n_h) for s in range(n_w - 1, -1, -1)] + [section(0, t) for t in range(n_h - 1, 0, -1)])
    m = len(ring)
    for i in range(n_len):
        for r in range(m):
            (ya, za), (yb, zb) = ring[r], ring[(r + 1) % m]
            quad(vert(xs[i], ya, za), vert(xs[i], yb, zb), vert(xs[i + 1], yb, zb), vert(xs[i + 1], ya, za))
    # the two end caps: the trapezoid's grid
    for x, flip in ((x0, True), (x1, False)):
        for t in range(n_h):
            for s in range(n_w):
                (ya, za), (yb, zb) = section(s, t), section(s + 1, t)
                (yc, zc), (yd, zd) = section(s + 1, t + 1), section(s, t + 1)
                p = [vert(x, ya, za), vert(x, yb, zb), vert(x, yc, zc), vert(x, yd, zd)]
                if flip:
                    p = p[::-1]
                quad(*p)
    return np.array(tris, dtype=np.float64)
