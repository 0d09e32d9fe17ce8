"""Seeded synthetic scene generators (inputs only).

This module builds scene descriptions -- rigid/near-rigid box bodies and
the joints between them -- with the shapes, sizes and value distributions of
the paper's workloads (Sec. 6, Table 1).  It draws every random number the
inputs need from ``numpy.random.default_rng(seed)`` in a fixed consumption
order, and it performs none of the per-step arithmetic of the method: no
mass matrices, no rotations of the solver, no constraint rows.  Both the CPU
oracle and the CUDA path read the dictionaries produced here, and nothing
else is shared between them.

A scene is a plain dict of numpy arrays (M bodies, K joints):

  h (float), gravity (3,)
  mass (M,)            body mass [kg]
  second_moment (M,6)  Sigma = int rho xbar xbar^T about the centre of mass,
                       ordered xx, yy, zz, xy, xz, yz  [kg m^2]
  volume (M,), young (M,), poisson (M,)
  fixed (M,) int32     1 = the body never moves (joints to it are one-sided)
  q (M,12), qdot (M,12)  affine coordinates [vec(A) column-stacked; t]
  jtype (K,) int32     0 = ball (3 rows), 1 = hinge (5 rows)
  body_a, body_b (K,) int64   body_b may be WORLD (-1)
  anchor_a, anchor_b (K,3)    joint point in each body's rest frame
                              (anchor_b is a world point when body_b = WORLD)
  axis_a, axis_b (K,3)        hinge axis in each rest frame (world if WORLD)
  axis_len (K,)               distance of the second on-axis point

Box mass properties follow from the definition of the second moment of a
homogeneous box, Sigma = m/12 diag(a^2, b^2, c^2) (sides a, b, c).
"""
from __future__ import annotations

import numpy as np

WORLD = -1
BALL = 0
HINGE = 1
UNIVERSAL = 2
PRISMATIC = 3
ROWS = {BALL: 3, HINGE: 5}

_I9 = np.array([1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0])


def _empty_scene(M: int, K: int, h: float, gravity=(0.0, 0.0, -9.8)) -> dict:
    return {
        "h": float(h),
        "gravity": np.asarray(gravity, dtype=np.float64),
        "mass": np.zeros(M),
        "second_moment": np.zeros((M, 6)),
        "volume": np.zeros(M),
        "young": np.zeros(M),
        "poisson": np.zeros(M),
        "fixed": np.zeros(M, dtype=np.int32),
        "q": np.zeros((M, 12)),
        "qdot": np.zeros((M, 12)),
        "jtype": np.zeros(K, dtype=np.int32),
        "body_a": np.zeros(K, dtype=np.int64),
        "body_b": np.zeros(K, dtype=np.int64),
        "anchor_a": np.zeros((K, 3)),
        "anchor_b": np.zeros((K, 3)),
        "axis_a": np.tile(np.array([0.0, 1.0, 0.0]), (K, 1)),
        "axis_b": np.tile(np.array([0.0, 1.0, 0.0]), (K, 1)),
        "axis_len": np.ones(K),
    }


def _set_boxes(sc: dict, sides: np.ndarray, rho: np.ndarray, centres: np.ndarray,
               young: float, poisson: float = 0.3) -> None:
    sides = np.asarray(sides, dtype=np.float64)
    vol = sides[:, 0] * sides[:, 1] * sides[:, 2]
    m = rho * vol
    sc["mass"][:] = m
    sc["volume"][:] = vol
    sc["second_moment"][:, 0:3] = (m / 12.0)[:, None] * sides ** 2
    sc["second_moment"][:, 3:6] = 0.0
    sc["young"][:] = young
    sc["poisson"][:] = poisson
    sc["q"][:, 0:9] = _I9
    sc["q"][:, 9:12] = centres


def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotations (normalised Gaussian quaternions), shape (n,3,3)."""
    qv = _unit(rng.standard_normal((n, 4)))
    w, x, y, z = qv[:, 0], qv[:, 1], qv[:, 2], qv[:, 3]
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def axis_angle(axis, angle: float) -> np.ndarray:
    """Rotation matrix about a unit axis (Rodrigues); used to pose inputs."""
    a = _unit(np.asarray(axis, dtype=np.float64))
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(angle) * K + (1 - np.cos(angle)) * (K @ K)


# ---------------------------------------------------------------------------
# Workloads shaped like the paper's scenes (Sec. 6, Table 1)
# ---------------------------------------------------------------------------

def chain_cubes(M: int = 64, h: float = 1e-2, young: float = 1e8) -> dict:
    """Chain of M unit cubes (rho = 1000) joined by ball joints at shared face
    centres, body 0 pinned to the world at its -x face centre, starting
    horizontal along +x (the 64-body plain FP64 chain; seed unused)."""
    K = M
    sc = _empty_scene(M, K, h)
    sides = np.ones((M, 3))
    centres = np.zeros((M, 3))
    centres[:, 0] = np.arange(M) + 0.5
    _set_boxes(sc, sides, np.full(M, 1000.0), centres, young)
    sc["jtype"][:] = BALL
    sc["body_a"][0], sc["body_b"][0] = 0, WORLD
    sc["anchor_a"][0] = (-0.5, 0, 0)
    sc["anchor_b"][0] = (0, 0, 0)
    for k in range(1, K):
        sc["body_a"][k], sc["body_b"][k] = k - 1, k
        sc["anchor_a"][k] = (0.5, 0, 0)
        sc["anchor_b"][k] = (-0.5, 0, 0)
    return sc


def ring_chain(M: int = 1 << 20, seed: int = 1, h: float = 1e-2, young: float = 1e8) -> dict:
    """The pulley-cable chain closed into a loop (Sec. 5.4, Case III): M boxes
    with sides U[0.5,1.5]^3 and densities 10^U[2,4] laid along a horizontal
    circle, each box's x axis along its chord of a closed polygon whose edge
    lengths are the boxes' x sides, consecutive boxes touching at face
    centres; joint j (bodies j, j+1 mod M) is a ball for even j and a hinge
    with an axis uniform on the sphere for odd j; no world joints.  The
    polygon's radius solves sum_j 2 asin(L_j / 2R) = 2 pi (bisection)."""
    rng = np.random.default_rng(seed)
    sides = rng.uniform(0.5, 1.5, size=(M, 3))
    rho = 10.0 ** rng.uniform(2.0, 4.0, size=M)
    L = sides[:, 0]
    lo, hi = 0.5 * L.max(), L.sum()
    for _ in range(200):
        R = 0.5 * (lo + hi)
        if np.sum(2.0 * np.arcsin(np.minimum(1.0, L / (2.0 * R)))) > 2.0 * np.pi:
            lo = R
        else:
            hi = R
    R = 0.5 * (lo + hi)
    phi = np.cumsum(2.0 * np.arcsin(np.minimum(1.0, L / (2.0 * R))))
    P = np.stack([R * np.cos(phi), R * np.sin(phi), np.zeros(M)], axis=1)  # joint j's point
    Pm = np.roll(P, 1, axis=0)                                              # box j spans Pm[j] .. P[j]
    d = _unit(P - Pm)
    centres = 0.5 * (P + Pm)
    K = M
    sc = _empty_scene(M, K, h)
    _set_boxes(sc, sides, rho, centres, young)
    A = np.zeros((M, 3, 3))
    A[:, :, 0] = d
    A[:, :, 1] = np.stack([-d[:, 1], d[:, 0], np.zeros(M)], axis=1)
    A[:, 2, 2] = 1.0
    sc["q"][:, 0:9] = np.transpose(A, (0, 2, 1)).reshape(M, 9)  # q stacks A's columns
    j = np.arange(M)
    nxt = (j + 1) % M
    sc["body_a"][:] = j
    sc["body_b"][:] = nxt
    sc["anchor_a"][:, 0] = 0.5 * L
    sc["anchor_b"][:, 0] = -0.5 * L[nxt]
    is_h = (j % 2) == 1
    sc["jtype"][:] = np.where(is_h, HINGE, BALL)
    w = _unit(rng.standard_normal((M, 3)))
    sc["axis_a"][:] = np.einsum("kji,kj->ki", A, w)          # A_a^T w
    sc["axis_b"][:] = np.einsum("kji,kj->ki", A[nxt], w)     # A_b^T w
    return sc


def long_chain(M: int = 1 << 20, seed: int = 1, h: float = 1e-2,
               young: float = 1e8) -> dict:
    """Pulley-cable chain: M boxes with sides U[0.5,1.5]^3 and densities
    10^U[2,4] laid end to end along +x touching at face centres.  Internal
    joint i (bodies i, i+1) is a ball for even i and a hinge with an axis
    uniform on the sphere for odd i.  Both outer face centres are pinned to
    the world by ball joints at their initial positions.  Joint order:
    [left pin, internal 0 .. M-2, right pin]."""
    rng = np.random.default_rng(seed)
    sides = rng.uniform(0.5, 1.5, size=(M, 3))
    rho = 10.0 ** rng.uniform(2.0, 4.0, size=M)
    n_int = M - 1
    n_hinge = n_int // 2
    axes = _unit(rng.standard_normal((max(n_hinge, 1), 3)))[:n_hinge]
    half = 0.5 * sides[:, 0]
    cx = np.empty(M)
    cx[0] = half[0]
    if M > 1:
        cx[1:] = half[0] + np.cumsum(half[:-1] + half[1:])
    centres = np.zeros((M, 3))
    centres[:, 0] = cx
    K = n_int + 2
    sc = _empty_scene(M, K, h)
    _set_boxes(sc, sides, rho, centres, young)
    # left pin
    sc["body_a"][0], sc["body_b"][0] = 0, WORLD
    sc["anchor_a"][0] = (-half[0], 0, 0)
    sc["anchor_b"][0] = (0.0, 0, 0)
    # internal joints 1..M-1
    i = np.arange(n_int)
    k = i + 1
    sc["body_a"][k] = i
    sc["body_b"][k] = i + 1
    sc["anchor_a"][k, 0] = half[i]
    sc["anchor_b"][k, 0] = -half[i + 1]
    is_h = (i % 2) == 1
    sc["jtype"][k] = np.where(is_h, HINGE, BALL)
    hk = k[is_h]
    sc["axis_a"][hk] = axes
    sc["axis_b"][hk] = axes
    # right pin
    sc["body_a"][K - 1], sc["body_b"][K - 1] = M - 1, WORLD
    sc["anchor_a"][K - 1] = (half[M - 1], 0, 0)
    sc["anchor_b"][K - 1] = (cx[M - 1] + half[M - 1], 0, 0)
    return sc


def random_tree(M: int = 262144, seed: int = 2, h: float = 5e-3,
                max_depth: int = 64, mean_children: float = 1.8,
                young: float = 1e8, joint: str = "hinge") -> dict:
    """Random rooted tree grown breadth-first: each body draws Poisson(1.8)
    children (0 at depth max_depth), truncated when M bodies exist; if the
    frontier dies out early, the first body (in creation order) below the
    depth limit gets one extra child.  Boxes have sides U[0.2,1]^3, rho=1000.
    Children sit upright on the parent's +z face at evenly spaced x
    positions; hinge axes are uniform on the sphere.  The root is pinned to
    the world by a ball joint at its -z face centre.  Body ids are in
    creation (BFS) order; joint 0 is the root pin, joint j>0 is the parent
    joint of body j with body_a = parent."""
    rng = np.random.default_rng(seed)
    sides = rng.uniform(0.2, 1.0, size=(M, 3))
    parent = np.full(M, -1, dtype=np.int64)
    depth = np.zeros(M, dtype=np.int64)
    slot = np.zeros(M, dtype=np.int64)      # index among siblings
    nsib = np.zeros(M, dtype=np.int64)      # number of siblings incl. self
    count = 1
    head = 0
    children_of = [[] for _ in range(M)]
    while count < M:
        if head < count:
            p = head
            head += 1
            n = 0 if depth[p] >= max_depth else int(rng.poisson(mean_children))
        else:  # frontier died out: first body below the depth limit grows one
            p = int(np.argmax(depth < max_depth))
            n = 1
        n = min(n, M - count)
        for _ in range(n):
            c = count
            count += 1
            parent[c] = p
            depth[c] = depth[p] + 1
            children_of[p].append(c)
    for p in range(M):
        ch = children_of[p]
        for s, c in enumerate(ch):
            slot[c] = s
            nsib[c] = len(ch)
    centres = np.zeros((M, 3))
    off = np.zeros((M, 3))  # attachment point in the parent frame
    for c in range(1, M):
        p = parent[c]
        ax = sides[p, 0]
        xo = (slot[c] + 1.0) / (nsib[c] + 1.0) * ax - 0.5 * ax
        off[c] = (xo, 0.0, 0.5 * sides[p, 2])
        centres[c] = centres[p] + off[c] + (0.0, 0.0, 0.5 * sides[c, 2])
    K = M
    sc = _empty_scene(M, K, h)
    _set_boxes(sc, sides, np.full(M, 1000.0), centres, young)
    sc["body_a"][0], sc["body_b"][0] = 0, WORLD
    sc["anchor_a"][0] = (0, 0, -0.5 * sides[0, 2])
    sc["anchor_b"][0] = (0, 0, -0.5 * sides[0, 2])
    c = np.arange(1, M)
    sc["body_a"][c] = parent[c]
    sc["body_b"][c] = c
    sc["anchor_a"][c] = off[c]
    sc["anchor_b"][c] = np.stack([np.zeros(M - 1), np.zeros(M - 1),
                                  -0.5 * sides[c, 2]], axis=1)
    if joint == "hinge":
        axes = _unit(rng.standard_normal((M - 1, 3)))
        sc["jtype"][c] = HINGE
        sc["axis_a"][c] = axes
        sc["axis_b"][c] = axes
    elif joint == "mixed":
        axes = _unit(rng.standard_normal((M - 1, 3)))
        kind = rng.random(M - 1) < 0.5
        sc["jtype"][c] = np.where(kind, HINGE, BALL)
        sc["axis_a"][c] = axes
        sc["axis_b"][c] = axes
    return sc


def jittered_net(nx: int = 64, ny: int = 64, nz: int = 16, seed: int = 4,
                 p_keep: float = 0.7, sigma: float = 0.05, h: float = 1e-2,
                 young: float = 1e9) -> dict:
    """Irregular closed-loop network: unit cubes (rho=1000) at lattice points
    plus N(0, sigma^2) jitter; candidate neighbour pairs (all x pairs, then
    all y pairs, then all z pairs, each in lexicographic order of the lower
    cell) are kept with probability p_keep as ball joints at the midpoint of
    the two centres.  The bottom layer is fixed; fixed-fixed pairs are
    dropped after the draw.  Body id = i + nx*(j + ny*k)."""
    rng = np.random.default_rng(seed)
    M = nx * ny * nz
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx),
                             indexing="ij")
    lattice = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.float64)
    centres = lattice + sigma * rng.standard_normal((M, 3))

    def bid(i, j, k):
        return i + nx * (j + ny * k)

    pairs = []
    for d in range(3):
        n = np.array([nx, ny, nz])
        n[d] -= 1
        k3, j3, i3 = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]),
                                 indexing="ij")
        i3, j3, k3 = i3.ravel(), j3.ravel(), k3.ravel()
        # lexicographic order of the lower cell (i, j, k)
        order = np.lexsort((k3, j3, i3))
        i3, j3, k3 = i3[order], j3[order], k3[order]
        a = bid(i3, j3, k3)
        b = bid(i3 + (d == 0), j3 + (d == 1), k3 + (d == 2))
        pairs.append(np.stack([a, b], axis=1))
    pairs = np.concatenate(pairs, axis=0)
    keep = rng.random(len(pairs)) < p_keep
    fixed = (lattice[:, 2] == 0).astype(np.int32)
    both_fixed = (fixed[pairs[:, 0]] == 1) & (fixed[pairs[:, 1]] == 1)
    pairs = pairs[keep & ~both_fixed]
    K = len(pairs)
    sc = _empty_scene(M, K, h)
    _set_boxes(sc, np.ones((M, 3)), np.full(M, 1000.0), centres, young)
    sc["fixed"][:] = fixed
    a, b = pairs[:, 0], pairs[:, 1]
    mid = 0.5 * (centres[a] + centres[b])
    sc["body_a"][:] = a
    sc["body_b"][:] = b
    sc["anchor_a"][:] = mid - centres[a]
    sc["anchor_b"][:] = mid - centres[b]
    sc["jtype"][:] = BALL
    return sc


def assemblies(n: int = 4096, seed: int = 3, h: float = 2e-3, young: float = 1e8,
               min_links: int = 7, max_links: int = 64, mean_children: float = 1.3,
               spacing: float = 40.0) -> dict:
    """Independent articulated assemblies (the batched form): each has a link
    count uniform in [7, 64] and is a random tree grown breadth-first with
    Poisson(1.3) children (truncated at its link count; a body whose
    frontier died out gets one child); joints are hinges or balls with
    probability 1/2 and hinge axes are uniform on the sphere.  Links are
    boxes with sides U[0.1,0.5]^3 and masses 10^U[-1,1] kg.  Link 0 is a
    fixed base with a uniformly random pose, so every subtree hanging from
    it is an independent tree whose root joint is one-sided.  Assemblies
    sit on a square grid `spacing` metres apart.  Body ids are contiguous
    per assembly; joint j>0 of an assembly is the parent joint of its link j
    with body_a = the parent.

    Random numbers are drawn per assembly in this order: link count, the
    child counts, sides, log-masses, joint kinds, hinge axes, base pose."""
    rng = np.random.default_rng(seed)
    bodies_sides, bodies_mass, centres, rots, fixed = [], [], [], [], []
    jt, ja, jb, an_a, an_b, ax = [], [], [], [], [], []
    side_len = int(np.ceil(np.sqrt(n)))
    base_id = 0
    for a in range(n):
        L = int(rng.integers(min_links, max_links + 1))
        parent = np.full(L, -1, dtype=np.int64)
        count, head = 1, 0
        kids = [[] for _ in range(L)]
        while count < L:
            if head < count:
                p_ = head
                head += 1
                k = int(rng.poisson(mean_children))
            else:
                p_ = count - 1
                k = 1
            k = min(k, L - count)
            for _ in range(k):
                parent[count] = p_
                kids[p_].append(count)
                count += 1
        sides = rng.uniform(0.1, 0.5, size=(L, 3))
        mass = 10.0 ** rng.uniform(-1.0, 1.0, size=L)
        kind = rng.random(L - 1) < 0.5
        axes = _unit(rng.standard_normal((L - 1, 3)))
        Q = random_rotations(rng, 1)[0]
        # local layout: children upright on the parent's +z face
        loc = np.zeros((L, 3))
        off = np.zeros((L, 3))
        for p_ in range(L):
            ch = kids[p_]
            for si, c in enumerate(ch):
                axl = sides[p_, 0]
                xo = (si + 1.0) / (len(ch) + 1.0) * axl - 0.5 * axl
                off[c] = (xo, 0.0, 0.5 * sides[p_, 2])
                loc[c] = loc[p_] + off[c] + (0.0, 0.0, 0.5 * sides[c, 2])
        origin = np.array([spacing * (a % side_len), spacing * (a // side_len), 0.0])
        for j in range(L):
            bodies_sides.append(sides[j])
            bodies_mass.append(mass[j])
            centres.append(origin + Q @ loc[j])
            rots.append(Q)
            fixed.append(1 if j == 0 else 0)
        for j in range(1, L):
            jt.append(HINGE if kind[j - 1] else BALL)
            ja.append(base_id + parent[j])
            jb.append(base_id + j)
            an_a.append(off[j])
            an_b.append((0.0, 0.0, -0.5 * sides[j, 2]))
            ax.append(axes[j - 1])
        base_id += L
    M = base_id
    K = len(jt)
    sc = _empty_scene(M, K, h)
    sides = np.array(bodies_sides)
    mass = np.array(bodies_mass)
    vol = sides.prod(axis=1)
    _set_boxes(sc, sides, mass / vol, np.array(centres), young)
    R = np.array(rots)
    sc["q"][:, 0:9] = np.transpose(R, (0, 2, 1)).reshape(M, 9)  # columns of R stacked
    sc["fixed"][:] = np.array(fixed, dtype=np.int32)
    sc["jtype"][:] = jt
    sc["body_a"][:] = ja
    sc["body_b"][:] = jb
    sc["anchor_a"][:] = an_a
    sc["anchor_b"][:] = an_b
    sc["axis_a"][:] = ax
    sc["axis_b"][:] = ax
    return sc


# ---------------------------------------------------------------------------
# Small scenes for checks
# ---------------------------------------------------------------------------

def single_body(sides=(1.0, 1.0, 1.0), rho: float = 1000.0, h: float = 1e-2,
                young: float = 1e8, gravity=(0.0, 0.0, -9.8)) -> dict:
    sc = _empty_scene(1, 0, h, gravity)
    _set_boxes(sc, np.asarray([sides], dtype=np.float64), np.array([rho]),
               np.zeros((1, 3)), young)
    return sc


def pendulum(theta0: float, h: float = 1e-3, young: float = 1e8) -> dict:
    """Unit cube (rho = 1000) hanging from a world ball joint at the centre
    of its +z face (the pivot, at the origin), released at rest after a
    rotation theta0 about the world x axis."""
    sc = _empty_scene(1, 1, h)
    R = axis_angle((1.0, 0.0, 0.0), theta0)
    centre = R @ np.array([0.0, 0.0, -0.5])
    _set_boxes(sc, np.ones((1, 3)), np.array([1000.0]), centre[None, :], young)
    sc["q"][0, 0:9] = R.T.reshape(9)  # columns of R, stacked
    sc["body_a"][0], sc["body_b"][0] = 0, WORLD
    sc["anchor_a"][0] = (0.0, 0.0, 0.5)
    sc["anchor_b"][0] = (0.0, 0.0, 0.0)
    return sc


def random_small(topology: str, M: int, seed: int, h: float = 1e-2,
                 young: float = 1e8, pin: bool = True, hinge_frac: float = 0.5,
                 gap: float = 0.02, univ_frac: float = 0.0, prism_frac: float = 0.0) -> dict:
    """Small random scene with mixed ball/hinge joints.

    topology: 'chain' (path 0-1-...-M-1, optional world pins at both ends),
    with univ_frac > 0 joints between two bodies are universal joints with
    that probability (axes perpendicular at generation); with prism_frac > 0
    any joint is a prismatic joint with that probability (the same sliding
    axis and reference direction on both sides, the reference normal to the
    axis; the scene then carries 'ref_a' / 'ref_b');
    'tree' (random parent p < j, root pinned), 'loop' (ring), 'graph' (tree
    plus extra random edges), 'free' (tree with no world pins).  Bodies are
    boxes with sides U[0.3,1.2]^3 and densities 10^U[2.5,3.5]; each joint
    point lies near the midpoint of its two bodies, and the two anchors miss
    each other by up to `gap` per axis, so the joint residual c is non-zero."""
    rng = np.random.default_rng(seed)
    sides = rng.uniform(0.3, 1.2, size=(M, 3))
    rho = 10.0 ** rng.uniform(2.5, 3.5, size=M)
    centres = rng.uniform(-2.0, 2.0, size=(M, 3))
    edges = []
    if topology == "chain":
        edges = [(j - 1, j) for j in range(1, M)]
    elif topology in ("tree", "free"):
        for j in range(1, M):
            edges.append((int(rng.integers(0, j)), j))
    elif topology == "loop":
        edges = [(j - 1, j) for j in range(1, M)] + [(0, M - 1)]
    elif topology == "graph":
        for j in range(1, M):
            edges.append((int(rng.integers(0, j)), j))
        extra = max(1, M // 2)
        for _ in range(extra):
            a, b = rng.choice(M, size=2, replace=False)
            edges.append((int(min(a, b)), int(max(a, b))))
    else:
        raise ValueError(topology)
    world = []
    if pin and topology != "free":
        world.append(0)
        if topology == "chain" and M > 1:
            world.append(M - 1)
    K = len(edges) + len(world)
    sc = _empty_scene(M, K, h)
    if prism_frac > 0:
        sc["ref_a"] = np.zeros((K, 3))
        sc["ref_b"] = np.zeros((K, 3))
    _set_boxes(sc, sides, rho, centres, young)
    k = 0
    order = []
    if topology == "chain" and world:
        order = [("w", world[0])] + [("e", e) for e in edges] + \
                [("w", w) for w in world[1:]]
    else:
        order = [("w", w) for w in world] + [("e", e) for e in edges]
    for kind, val in order:
        # joint point near the bodies (A = I at generation), with a small gap
        if kind == "w":
            j = val
            sc["body_a"][k], sc["body_b"][k] = j, WORLD
            off = rng.uniform(-0.5, 0.5, 3) * sides[j]
            sc["anchor_a"][k] = off
            sc["anchor_b"][k] = centres[j] + off + rng.uniform(-gap, gap, 3)
        else:
            a, b = val
            sc["body_a"][k], sc["body_b"][k] = a, b
            x = 0.5 * (centres[a] + centres[b]) + rng.uniform(-0.3, 0.3, 3)
            sc["anchor_a"][k] = x - centres[a]
            sc["anchor_b"][k] = x - centres[b] + rng.uniform(-gap, gap, 3)
        is_h = rng.random() < hinge_frac
        sc["jtype"][k] = HINGE if is_h else BALL
        sc["axis_a"][k] = _unit(rng.standard_normal(3))
        sc["axis_b"][k] = _unit(rng.standard_normal(3))
        sc["axis_len"][k] = rng.uniform(0.5, 1.5)
        if univ_frac > 0 and kind == "e" and rng.random() < univ_frac:
            # universal joint (Sec. 4.4): beta's axis perpendicular to alpha's
            sc["jtype"][k] = UNIVERSAL
            sc["axis_b"][k] = _unit(np.cross(sc["axis_a"][k], sc["axis_b"][k]))
        if prism_frac > 0 and rng.random() < prism_frac:
            # prismatic joint (Sec. 4.5); bodies have A = I at generation
            sc["jtype"][k] = PRISMATIC
            sc["axis_b"][k] = sc["axis_a"][k]
            ref = _unit(np.cross(sc["axis_a"][k], rng.standard_normal(3)))
            sc["ref_a"][k] = ref
            sc["ref_b"][k] = ref
        k += 1
    return sc


def perturb_state(sc: dict, seed: int, rot: float = 0.3, vel: float = 0.5,
                  strain: float = 1e-5) -> tuple[np.ndarray, np.ndarray]:
    """A random state near the scene's pose: each body is turned about its own
    centre by a random rotation of angle up to `rot` (radians) composed with
    a small random symmetric stretch of size `strain`, and given random
    affine velocities of scale `vel`.  Returns (q, qdot) of shape (M,12)."""
    rng = np.random.default_rng(seed)
    M = len(sc["mass"])
    q = sc["q"].copy()
    axes = _unit(rng.standard_normal((M, 3)))
    ang = rng.uniform(-rot, rot, size=M)
    S = rng.standard_normal((M, 3, 3)) * strain
    S = 0.5 * (S + np.transpose(S, (0, 2, 1)))
    qd = rng.standard_normal((M, 12)) * vel
    for j in range(M):
        A = q[j, 0:9].reshape(3, 3).T  # columns stacked -> matrix
        A = axis_angle(axes[j], ang[j]) @ A @ (np.eye(3) + S[j])
        q[j, 0:9] = A.T.reshape(9)
    fixed = sc["fixed"] != 0
    q[fixed] = sc["q"][fixed]
    qd[fixed] = 0.0
    return q, qd


def rotate_scene(sc: dict, Q: np.ndarray) -> dict:
    """The same assembly turned rigidly by the rotation Q about the world
    origin (body poses, world anchor points and world axes); gravity is
    left unchanged."""
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    M = len(sc["mass"])
    for j in range(M):
        A = sc["q"][j, 0:9].reshape(3, 3).T
        out["q"][j, 0:9] = (Q @ A).T.reshape(9)
        out["q"][j, 9:12] = Q @ sc["q"][j, 9:12]
        Ad = sc["qdot"][j, 0:9].reshape(3, 3).T
        out["qdot"][j, 0:9] = (Q @ Ad).T.reshape(9)
        out["qdot"][j, 9:12] = Q @ sc["qdot"][j, 9:12]
    w = sc["body_b"] == WORLD
    out["anchor_b"][w] = sc["anchor_b"][w] @ Q.T
    out["axis_b"][w] = sc["axis_b"][w] @ Q.T
    if "ref_b" in sc:
        out["ref_b"][w] = sc["ref_b"][w] @ Q.T
    return out


def turn_rest_frames(sc: dict, seed: int) -> dict:
    """The same assembly described in rest frames turned off the principal
    axes: body j's rest coordinates become xbar' = Q_j xbar for a random
    rotation Q_j, so its second moment becomes Q_j Sigma Q_j^T (no longer
    diagonal), its affine matrix A Q_j^T (q and qdot), and the rest-frame
    anchors, axes and reference directions of its joints Q_j times the old
    ones.  World points and directions are unchanged; so is the motion."""
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    M = len(sc["mass"])
    Q = random_rotations(np.random.default_rng(seed), M)
    S = sc["second_moment"]
    for j in range(M):
        Sg = np.array([[S[j, 0], S[j, 3], S[j, 4]], [S[j, 3], S[j, 1], S[j, 5]], [S[j, 4], S[j, 5], S[j, 2]]])
        T = Q[j] @ Sg @ Q[j].T
        out["second_moment"][j] = [T[0, 0], T[1, 1], T[2, 2], T[0, 1], T[0, 2], T[1, 2]]
        for key in ("q", "qdot"):
            A = sc[key][j, 0:9].reshape(3, 3).T
            out[key][j, 0:9] = (A @ Q[j].T).T.reshape(9)
    for side, body in (("a", sc["body_a"]), ("b", sc["body_b"])):
        on = body != WORLD
        for key in ("anchor_", "axis_", "ref_"):
            k = key + side
            if k not in sc:
                continue
            v = sc[k].copy()
            v[on] = np.einsum("kij,kj->ki", Q[body[on]], sc[k][on])
            out[k] = v
    return out


def concat_scenes(parts: list[dict], spacing: float = 100.0) -> dict:
    """Disjoint union of scenes with the same h and gravity: part i is moved
    by i * spacing along x and its body and joint ids are offset."""
    out = {}
    h, g = parts[0]["h"], parts[0]["gravity"]
    boff = 0
    chunks: dict[str, list] = {}
    for i, sc in enumerate(parts):
        M = len(sc["mass"])
        c = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
        c["q"][:, 9] += i * spacing
        for key in ("body_a", "body_b"):
            v = c[key]
            c[key] = np.where(v == WORLD, WORLD, v + boff)
        w = c["body_b"] == WORLD
        c["anchor_b"][w, 0] += i * spacing
        for k, v in c.items():
            if isinstance(v, np.ndarray):
                chunks.setdefault(k, []).append(v)
        boff += M
    for k, vs in chunks.items():
        out[k] = np.concatenate(vs, axis=0)
    out["h"], out["gravity"] = h, g
    return out


def net_collection(n: int = 48, seed: int = 10, size_range=((4, 10), (4, 10), (3, 6))) -> dict:
    """n disjoint jittered nets of the closed-loop form (jittered_net) with
    sizes drawn uniformly from size_range and their own seeds: the training
    scenes of the learned preconditioner."""
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(n):
        dims = [int(rng.integers(lo, hi + 1)) for lo, hi in size_range]
        parts.append(jittered_net(*dims, seed=int(rng.integers(1 << 30))))
    return concat_scenes(parts)


# parameter layout of the learned preconditioner (sizes only; the network
# itself lives in the library and in the oracle)
LPC_SIZES = (("W1", (16, 64)), ("b1", (64,)), ("W2", (128, 64)), ("b2", (64,)),
             ("W3", (128, 64)), ("b3", (64,)), ("Wa", (64, 8)), ("Wb", (64, 8)),
             ("wd", (64,)), ("cd", (1,)), ("we", (2,)), ("ce", (1,)))


def lpc_param_count() -> int:
    return int(sum(np.prod(shape) for _, shape in LPC_SIZES))


def lpc_init_params(seed: int = 0) -> np.ndarray:
    """Random starting parameters (float32): layer weights N(0, 2/fan_in),
    biases 0, edge-head factors N(0, 0.01/64), scale head 0, edge gate
    offset ln(1/2) (alpha = 0.5 where the bilinear term is 0)."""
    rng = np.random.default_rng(seed)
    out = []
    for name, shape in LPC_SIZES:
        if name in ("W1", "W2", "W3"):
            v = rng.standard_normal(shape) * np.sqrt(2.0 / shape[0])
        elif name in ("Wa", "Wb"):
            v = rng.standard_normal(shape) * np.sqrt(0.01 / shape[0])
        elif name == "ce":
            v = np.full(shape, np.log(0.5))
        else:
            v = np.zeros(shape)
        out.append(np.asarray(v, dtype=np.float64).ravel())
    return np.concatenate(out).astype(np.float32)


def lpc_probe(nv: int, K: int, seed: int) -> np.ndarray:
    """Probe vectors [nv][K][3] (float32), uniform with unit variance."""
    rng = np.random.default_rng(seed)
    return (rng.uniform(-1.0, 1.0, size=(nv, K, 3)) * np.sqrt(3.0)).astype(np.float32)


JOINT_ROWS = {BALL: 3, HINGE: 5, UNIVERSAL: 4, PRISMATIC: 5}


def joint_rows(jtype) -> np.ndarray:
    """Constraint rows per joint: ball 3 (Eq. ball), hinge 5 (Eq. hinge),
    universal 4 (Eq. universal), prismatic 5 (Eq. prismatic)."""
    jt = np.asarray(jtype)
    out = np.full(jt.shape, 3, dtype=np.int64)
    out[(jt == HINGE) | (jt == PRISMATIC)] = 5
    out[jt == UNIVERSAL] = 4
    return out


def dual_rows(sc: dict) -> int:
    return int(joint_rows(sc["jtype"]).sum())


def workload(name: str, **kw) -> dict:
    """Named workloads: 'chain64', 'chain1m', 'tree256k', 'net64x64x16'
    (sizes overridable through keyword arguments)."""
    if name == "chain64":
        return chain_cubes(**kw)
    if name == "chain1m":
        return long_chain(**kw)
    if name == "tree256k":
        return random_tree(**kw)
    if name == "net64x64x16":
        return jittered_net(**kw)
    if name == "batch4096":
        return assemblies(**kw)
    raise KeyError(name)
