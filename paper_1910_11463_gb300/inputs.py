"""Seeded synthetic inputs for the S_N transport problems: PRNG, angular
quadrature, meshes and cross sections.

This module is the problem *definition* only.  It holds no arithmetic of the
method (no discretisation, no multigrid, no source iteration): it produces the
arrays that both the CUDA path and the CPU oracle take as inputs, so that both
see bit-identical data.

* PRNG: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014), u = (x >> 11) * 2^-53.
* Quadrature: level-symmetric S_N sets (Lewis & Miller tables), the angular
  quadrature of Eq. (angular_quad), phi = sum_m w_m psi_m, weights summing to
  4*pi.  The paper itself used a square Chebyshev-Legendre S4 set (Sec. 4);
  the workloads here use level-symmetric S2/S4/S8.
* Meshes: the unit cube split into n^3 axis-aligned hexahedra (Q1 DG, 8 DOFs
  per element, DOF = 8*e + a, e = ix + n*(iy + n*iz), a = ax + 2*ay + 4*az).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def splitmix64_stream(seed: int, count: int) -> np.ndarray:
    """The first `count` outputs of SplitMix64 started at state `seed`."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) with 53 random bits each, drawn in order."""
    z = splitmix64_stream(seed, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ---------------------------------------------------------------------------
# Level-symmetric quadrature
# ---------------------------------------------------------------------------

_LS_MU1 = {2: 1.0 / math.sqrt(3.0), 4: 0.3500212, 8: math.sqrt(1.0 / 21.0)}


def level_symmetric(order: int):
    """Level-symmetric S_N set for N in {2, 4, 8}.

    Returns (omega[M,3], w[M]) with M = N(N+2).  Octants are ordered by sign
    (x fastest, '+' first); inside an octant the points are the index triples
    (i, j, k), i + j + k = N/2 + 2, in lexicographic order, with direction
    cosines (mu_i, mu_j, mu_k), mu_i^2 = mu_1^2 + (i-1) 2 (1 - 3 mu_1^2)/(N-2).
    Weights: S2, S4 equal; S8 from the per-octant moment conditions
    sum w = 1, sum w mu^4 = 1/5, sum w mu^6 = 1/7 over the three point classes.
    The weights are scaled to sum to 4*pi.
    """
    if order not in _LS_MU1:
        raise ValueError("level_symmetric: order must be 2, 4 or 8")
    n_half = order // 2
    mu1 = _LS_MU1[order]
    if order == 2:
        mus = [mu1]
    else:
        step = 2.0 * (1.0 - 3.0 * mu1 * mu1) / (order - 2)
        mus = [math.sqrt(mu1 * mu1 + i * step) for i in range(n_half)]
    triples = [(i, j, k)
               for i in range(1, n_half + 1)
               for j in range(1, n_half + 1)
               for k in range(1, n_half + 1) if i + j + k == n_half + 2]
    if order == 8:
        classes = {(1, 1, 4): 0, (1, 2, 3): 1, (2, 2, 2): 2}
        # per-octant moment system: rows = moments 0, 4, 6 of mu_x
        A = np.zeros((3, 3))
        for t in triples:
            c = classes[tuple(sorted(t))]
            mx = mus[t[0] - 1]
            A[0, c] += 1.0
            A[1, c] += mx ** 4
            A[2, c] += mx ** 6
        wc = np.linalg.solve(A, np.array([1.0, 0.2, 1.0 / 7.0]))
        w_oct = [wc[classes[tuple(sorted(t))]] for t in triples]
    else:
        w_oct = [1.0 / len(triples)] * len(triples)
    omega, w = [], []
    scale = 4.0 * math.pi / 8.0
    for octant in range(8):
        sx = -1.0 if octant & 1 else 1.0
        sy = -1.0 if octant & 2 else 1.0
        sz = -1.0 if octant & 4 else 1.0
        for t, wt in zip(triples, w_oct):
            omega.append((sx * mus[t[0] - 1], sy * mus[t[1] - 1], sz * mus[t[2] - 1]))
            w.append(wt * scale)
    return np.ascontiguousarray(np.array(omega, dtype=np.float64)), np.array(w, dtype=np.float64)


# ---------------------------------------------------------------------------
# Problems
# ---------------------------------------------------------------------------

@dataclass
class HexProblem:
    """Unit cube, n^3 hexahedra, Q1 upwind DG, one energy group."""
    name: str
    n: int
    omega: np.ndarray          # (M, 3) direction cosines
    w: np.ndarray              # (M,) quadrature weights, sum 4*pi
    sigma_t: np.ndarray        # (E,) per element
    sigma_s: np.ndarray        # (E,)
    q: np.ndarray              # (E,) isotropic source strength (divided by 4*pi in the equation)
    meta: dict = field(default_factory=dict)

    @property
    def E(self) -> int:
        return self.n ** 3

    @property
    def N(self) -> int:
        return 8 * self.n ** 3

    @property
    def M(self) -> int:
        return self.omega.shape[0]


def element_index_grid(n: int):
    """(ix, iy, iz) of every element, e = ix + n*(iy + n*iz)."""
    e = np.arange(n ** 3)
    return e % n, (e // n) % n, e // (n * n)


def hex_uniform(n: int, order: int, sigma_t: float, ratio: float, q: float = 1.0,
                name: str = "hex_uniform") -> HexProblem:
    omega, w = level_symmetric(order)
    E = n ** 3
    st = np.full(E, float(sigma_t))
    return HexProblem(name, n, omega, w, st, st * ratio, np.full(E, float(q)),
                      {"order": order, "sigma": "uniform", "ratio": ratio})


def hex_random(n: int, order: int, ratio: float, seed: int = 1, lo: float = 0.5,
               hi: float = 2.0, log_uniform: bool = False, source_block=None,
               name: str = "hex_random") -> HexProblem:
    """sigma_t drawn per element in element order: U[lo,hi] -> lo + (hi-lo) u,
    log-U[lo,hi] -> 10^(log10 lo + (log10 hi - log10 lo) u); sigma_s = ratio*sigma_t.
    source_block = (a, b): q = 1 on elements with all indices in [a, b), else 0."""
    omega, w = level_symmetric(order)
    E = n ** 3
    u = uniform01(seed, E)
    if log_uniform:
        a, b = math.log10(lo), math.log10(hi)
        st = 10.0 ** (a + (b - a) * u)
    else:
        st = lo + (hi - lo) * u
    if source_block is None:
        q = np.ones(E)
    else:
        ix, iy, iz = element_index_grid(n)
        a, b = source_block
        inside = (ix >= a) & (ix < b) & (iy >= a) & (iy < b) & (iz >= a) & (iz < b)
        q = inside.astype(np.float64)
    return HexProblem(name, n, omega, w, st, st * ratio, q,
                      {"order": order, "seed": seed, "ratio": ratio,
                       "sigma": ("log-U" if log_uniform else "U") + f"[{lo},{hi}]"})


def detector_elements(n: int, lo: int = 0, hi: int = 4) -> np.ndarray:
    """Elements with all indices in [lo, hi) (a corner block)."""
    ix, iy, iz = element_index_grid(n)
    return ((ix >= lo) & (ix < hi) & (iy >= lo) & (iy < hi) & (iz >= lo) & (iz < hi))


def config(name: str) -> HexProblem:
    """The named synthetic workloads.

    hex8_s2     : 8^3 hex (4,096 DOFs/direction), S2 (8 directions), sigma_t = 1,
                  sigma_s = 0.5, q = 1, vacuum boundaries.
    hex32_s4    : 32^3 hex (262,144 DOFs/direction), S4 (24 directions),
                  sigma_t ~ U[0.5, 2] per element (seed 1), sigma_s = 0.8 sigma_t, q = 1.
    hex24_s4_adj: 24^3 hex (110,592 DOFs/direction), S4, sigma_t ~ U[0.5, 2],
                  sigma_s = 0.7 sigma_t, q = 1 in the central 8^3 block.
    hex64_s8    : 64^3 hex (2,097,152 DOFs/direction), S8 (80 directions),
                  sigma_t ~ log-U[0.1, 100], sigma_s = 0.95 sigma_t, q = 1.
    tet40_s8    : 40^3 cubes x 6 jittered Kuhn tets (1,536,000 DOFs/direction), S8,
                  sigma_t checkerboard {1, 100} over 4^3 regions (tet_checkerboard).
    tet16_s8    : the same construction on 16^3 cubes (98,304 DOFs/direction).
    """
    if name == "hex8_s2":
        return hex_uniform(8, 2, 1.0, 0.5, 1.0, name)
    if name == "hex32_s4":
        return hex_random(32, 4, 0.8, seed=1, name=name)
    if name == "hex24_s4_adj":
        return hex_random(24, 4, 0.7, seed=1, source_block=(8, 16), name=name)
    if name == "hex64_s8":
        return hex_random(64, 8, 0.95, seed=1, lo=0.1, hi=100.0, log_uniform=True, name=name)
    if name == "tet40_s8":
        return tet_checkerboard(40, 8, 4, 0.9, 0.2, 1, name)
    if name == "tet16_s8":
        return tet_checkerboard(16, 8, 4, 0.9, 0.2, 1, name)
    raise KeyError(name)


# ---------------------------------------------------------------------------
# Unstructured tetrahedra: Kuhn split of a jittered cube grid
# ---------------------------------------------------------------------------

# the six permutations of (x, y, z) in lexicographic order
_KUHN = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


@dataclass
class TetProblem:
    """Tetrahedral mesh of the unit cube, P1 upwind DG (4 DOFs per tet, DOF = 4 t + a)."""
    name: str
    n: int                     # cubes per axis
    verts: np.ndarray          # (V, 3) coordinates
    tets: np.ndarray           # (T, 4) vertex ids, local node a = column a
    nbr: np.ndarray            # (T, 4) tet across the face opposite local vertex f, -1 on the boundary
    omega: np.ndarray
    w: np.ndarray
    sigma_t: np.ndarray        # (T,)
    sigma_s: np.ndarray
    q: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def E(self) -> int:
        return self.tets.shape[0]

    @property
    def N(self) -> int:
        return 4 * self.tets.shape[0]

    @property
    def M(self) -> int:
        return self.omega.shape[0]


def kuhn_mesh(n: int, jitter: float = 0.2, seed: int = 1):
    """Vertices of the (n+1)^3 grid (v = vx + (n+1)(vy + (n+1) vz)); interior
    vertices moved by U[-jitter h, jitter h] per coordinate, three draws per
    vertex in vertex order (boundary vertices draw but do not move).  Cube
    c = cx + n (cy + n cz) is split into 6 tets, tet 6c + k = {v000,
    v000 + e_p0, v000 + e_p0 + e_p1, v111} for the k-th permutation p.
    Returns (verts, tets, nbr, cube_of_tet)."""
    h = 1.0 / n
    n1 = n + 1
    v = np.arange(n1 ** 3)
    vx, vy, vz = v % n1, (v // n1) % n1, v // (n1 * n1)
    verts = np.stack([vx, vy, vz], 1).astype(np.float64) * h
    if jitter > 0:
        u = uniform01(seed, 3 * n1 ** 3).reshape(-1, 3)
        interior = (vx > 0) & (vx < n) & (vy > 0) & (vy < n) & (vz > 0) & (vz < n)
        verts[interior] += (2.0 * u[interior] - 1.0) * (jitter * h)
    c = np.arange(n ** 3)
    cx, cy, cz = c % n, (c // n) % n, c // (n * n)
    base = np.stack([cx, cy, cz], 1)
    tets = np.zeros((6 * n ** 3, 4), np.int64)
    vid = lambda p: p[:, 0] + n1 * (p[:, 1] + n1 * p[:, 2])
    for k, perm in enumerate(_KUHN):
        p0 = base.copy()
        p1 = p0.copy(); p1[:, perm[0]] += 1
        p2 = p1.copy(); p2[:, perm[1]] += 1
        p3 = base + 1
        tets[k::6] = np.stack([vid(p0), vid(p1), vid(p2), vid(p3)], 1)
    # face neighbours: face f of tet t is the triangle without local vertex f
    T = tets.shape[0]
    faces = np.stack([np.delete(tets, f, axis=1) for f in range(4)], 1)   # (T, 4, 3)
    key = np.sort(faces, axis=2).reshape(-1, 3)
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0]))
    ks = key[order]
    same = np.all(ks[1:] == ks[:-1], axis=1)
    nbr = -np.ones(4 * T, np.int64)
    i = np.nonzero(same)[0]
    a, b = order[i], order[i + 1]
    nbr[a] = b // 4
    nbr[b] = a // 4
    return verts, tets.astype(np.int32), nbr.reshape(T, 4).astype(np.int32), np.repeat(c, 6)


def tet_checkerboard(n: int = 40, order: int = 8, regions: int = 4, ratio: float = 0.9, jitter: float = 0.2,
                     seed: int = 1, name: str = "tet40_s8") -> TetProblem:
    """Checkerboard of regions^3 blocks of cubes: sigma_t = 1 where the block
    parity (rx + ry + rz) is even, 100 where odd; sigma_s = ratio sigma_t; q = 1
    only where sigma_t = 1."""
    verts, tets, nbr, cube = kuhn_mesh(n, jitter, seed)
    omega, w = level_symmetric(order)
    per = n // regions
    cx, cy, cz = cube % n, (cube // n) % n, cube // (n * n)
    odd = ((cx // per + cy // per + cz // per) % 2) == 1
    st = np.where(odd, 100.0, 1.0)
    q = np.where(odd, 0.0, 1.0)
    return TetProblem(name, n, verts, tets, nbr, omega, w, st, st * ratio, q,
                      {"order": order, "regions": regions, "jitter": jitter, "seed": seed})


def small_tet(n: int = 3, order: int = 2, seed: int = 4, ratio: float = 0.5, jitter: float = 0.2) -> TetProblem:
    verts, tets, nbr, cube = kuhn_mesh(n, jitter, seed)
    omega, w = level_symmetric(order)
    u = uniform01(seed + 100, tets.shape[0])
    st = 0.5 + 1.5 * u
    return TetProblem(f"tet{n}_s{order}_seed{seed}", n, verts, tets, nbr, omega, w, st, st * ratio,
                      np.ones(tets.shape[0]), {"order": order, "seed": seed})


def node_coordinates(n: int):
    """(x, y, z) of every Q1 DOF 8e + a on the unit cube (node a = ax + 2 ay + 4 az at
    ((ix + ax) h, (iy + ay) h, (iz + az) h), h = 1/n), each an array of length 8 n^3."""
    ix, iy, iz = element_index_grid(n)
    a = np.arange(8)
    h = 1.0 / n
    x = ((ix[:, None] + (a & 1)[None, :]) * h).ravel()
    y = ((iy[:, None] + ((a >> 1) & 1)[None, :]) * h).ravel()
    z = ((iz[:, None] + ((a >> 2) & 1)[None, :]) * h).ravel()
    return x, y, z


def mms_hex(n: int, order: int = 4, sigma_t: float = 1.0, ratio: float = 0.5):
    """Manufactured solution of the paper's appendix on the unit cube (L = 1):
        psi(x, Omega) = Phi(x) Psi(x, Omega),
        Phi = sin(pi x) sin(pi y) sin(pi z),
        Psi = (1 + 2 mu (x - 1/2)) (1 + 2 eta (y - 1/2)) (1 + 2 xi (z - 1/2)).
    psi vanishes on the boundary (vacuum inflow).  For a level-symmetric set the odd
    moments of the weights vanish, so sum_m w_m Psi_m = 4 pi and the discrete scalar
    flux is phi = 4 pi Phi exactly; the scattering source sigma_s phi / (4 pi) is then
    sigma_s Phi, and the angular source of direction m is
        q_m = Omega_m . grad(Phi Psi_m) + sigma_t Phi Psi_m - sigma_s Phi
    (the appendix writes the scattering term with phi normalised as the angular
    average; with phi = integral of psi over the sphere it is sigma_s Phi).
    Returns (problem with q = 0, q_ang (M, 8 n^3) nodal values of q_m, phi_exact at
    the nodes)."""
    prob = hex_uniform(n, order, sigma_t, ratio, q=0.0, name=f"mms{n}_s{order}")
    x, y, z = node_coordinates(n)
    pi = np.pi
    sx, sy, sz = np.sin(pi * x), np.sin(pi * y), np.sin(pi * z)
    cx, cy, cz = np.cos(pi * x), np.cos(pi * y), np.cos(pi * z)
    Phi = sx * sy * sz
    q_ang = np.empty((prob.M, prob.N))
    for m, (mu, eta, xi) in enumerate(prob.omega):
        f, g, k = 1 + 2 * mu * (x - 0.5), 1 + 2 * eta * (y - 0.5), 1 + 2 * xi * (z - 0.5)
        Psi = f * g * k
        dx = pi * cx * sy * sz * Psi + Phi * 2 * mu * g * k
        dy = pi * sx * cy * sz * Psi + Phi * f * 2 * eta * k
        dz = pi * sx * sy * cz * Psi + Phi * f * g * 2 * xi
        q_ang[m] = mu * dx + eta * dy + xi * dz + sigma_t * Phi * Psi - sigma_t * ratio * Phi
    return prob, q_ang, 4 * pi * Phi


def small_hex(n: int, order: int = 2, seed: int = 7, ratio: float = 0.5) -> HexProblem:
    """Small seeded problem for parity tests (spans several tiles, ragged sizes)."""
    return hex_random(n, order, ratio, seed=seed, name=f"hex{n}_s{order}_seed{seed}")


def cyclic_block_operator(nb: int, ring: int, up: int = 3, down: int = 4, scale: float = 0.2, seed: int = 21):
    """A block-scaled operator whose element graph holds one cycle: an upstream
    chain of `up` elements feeds a ring of `ring` elements (ring element i reads
    ring element i - 1, the first reads the last and the end of the chain), and a
    downstream chain of `down` elements hangs off the ring.  Element ids are a
    seeded permutation, so id order is not upwind order.  Diagonal entries are
    1.0 (identity diagonal blocks, off-diagonal zeros not stored); every coupling
    is a dense nb x nb block of scale * U[-1, 1] values.  Returns CSR
    (rowptr, col, val) with ascending columns in every row, numpy int32/float64."""
    if ring == 1:
        raise ValueError("a ring has 0 (no cycle) or at least 2 elements")
    E = up + ring + down
    perm = (np.argsort(uniform01(seed, E), kind="stable")).astype(np.int64)
    chain_u = list(range(up))
    ring_ids = list(range(up, up + ring))
    chain_d = list(range(up + ring, E))
    reads = {k: [] for k in range(E)}
    for i in range(1, up):
        reads[chain_u[i]].append(chain_u[i - 1])
    for i, r in enumerate(ring_ids):
        reads[r].append(ring_ids[i - 1])
    if up and ring:
        reads[ring_ids[0]].append(chain_u[-1])
    prev = ring_ids[-1] if ring else (chain_u[-1] if up else None)
    for d in chain_d:
        if prev is not None:
            reads[d].append(prev)
        prev = d
    u = uniform01(seed + 1, E * 2 * nb * nb) * 2.0 - 1.0
    rows = [[] for _ in range(E * nb)]
    t = 0
    for k in range(E):
        e = int(perm[k])
        for a in range(nb):
            rows[e * nb + a].append((e * nb + a, 1.0))
        for src in reads[k]:
            f = int(perm[src])
            for a in range(nb):
                for b in range(nb):
                    rows[e * nb + a].append((f * nb + b, scale * u[t]))
                    t += 1
    rowptr = np.zeros(E * nb + 1, np.int32)
    col, val = [], []
    for r, ent in enumerate(rows):
        ent.sort()
        col += [c for c, _ in ent]
        val += [v for _, v in ent]
        rowptr[r + 1] = len(col)
    return rowptr, np.asarray(col, np.int32), np.asarray(val, np.float64)
