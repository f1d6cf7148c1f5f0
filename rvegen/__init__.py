"""Seeded synthetic fiber-network RVE inputs.

This module builds the inputs that both the CUDA path and the CPU oracle
consume: node coordinates, fiber connectivity, rest lengths, fiber
parameters, boundary flags, per-RVE offsets and deformation gradients.  It
holds none of the solver's arithmetic (no fiber law, no equilibrium, no
stress): it only draws random numbers and lays out arrays.

Geometry (reading of the paper's RVE description, Sec. 2 and Sec. 4.3; the
paper's RVE library is not available, jittered grids stand in for it):

* an n x n x n grid spanning the unit cube centred at the origin,
  X in [-1/2, 1/2]^3 (the RVE centroid sits at the macroscale material
  point, Eq. micro_coords), spacing s = 1/(n-1);
* each coordinate of a node is jittered by U(-0.3 s, 0.3 s) only along axes
  where the node is not on a face, so face nodes move in-plane, edge nodes
  along their edge and corners not at all;
* boundary nodes are all nodes on the six faces (affine BC, Eq. affine-bc);
* candidate fibers are the axis-neighbour bonds, 3 n^2 (n-1) of them, each
  kept with probability p; rest length L0 = |X_j - X_i| (stress free at F=I).

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator, so every platform draws the same bits.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise (wrapping uint64)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based SplitMix64 stream: draw k is mix(base + (k+1)*golden)."""

    def __init__(self, seed: int):
        self.base = _mix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        self.ctr = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.ctr + 1, self.ctr + 1 + n, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            return _mix64(self.base + k * _GOLDEN)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        """n doubles in [lo, hi) from the top 53 bits of each draw."""
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by the Box-Muller transform (two draws each)."""
        u1 = 1.0 - self.uniform(n)  # (0, 1]
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def rve_seed(config: int, index: int) -> int:
    """Per-RVE stream seed: 0x5EED0000 + config * 2^20 + index."""
    return 0x5EED0000 + config * (1 << 20) + index


@dataclass
class Network:
    """One RVE: reference coordinates, fibers and boundary flags."""

    X: np.ndarray            # (N, 3) float64 reference coordinates
    conn: np.ndarray         # (E, 2) int32 RVE-local node ids
    L0: np.ndarray           # (E,) float64 rest lengths
    EA: np.ndarray           # (E,) float64 axial stiffness
    B: np.ndarray            # (E,) float64 exponential nonlinearity
    is_boundary: np.ndarray  # (N,) uint8, 1 on the cube faces
    V0: float = 1.0          # reference RVE volume
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return self.X.shape[0]

    @property
    def n_fibers(self) -> int:
        return self.conn.shape[0]


def _candidate_bonds(n: int) -> np.ndarray:
    """All axis-neighbour pairs of an n^3 grid, axis 0 first, lexicographic."""
    idx = np.arange(n ** 3).reshape(n, n, n)
    pairs = [
        np.stack([idx[:-1, :, :].ravel(), idx[1:, :, :].ravel()], 1),
        np.stack([idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel()], 1),
        np.stack([idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel()], 1),
    ]
    return np.concatenate(pairs, 0).astype(np.int32)


def grid_network(n: int, p: float, stream: Stream, jitter: float = 0.3,
                 EA: float | str = 1.0, B: float = 10.0) -> Network:
    """Jittered n^3 grid with axis bonds kept with probability p.

    Draw order: jitter (3 n^3), bonds (3 n^2 (n-1)), then EA (one per kept
    fiber when EA == 'lognormal', i.e. log-normal mu=0, sigma=0.5).
    """
    if n < 2:
        raise ValueError("grid side must be >= 2")
    s = 1.0 / (n - 1)
    ijk = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1).reshape(-1, 3)
    X = ijk * s - 0.5
    interior_axis = (ijk > 0) & (ijk < n - 1)
    jit = stream.uniform(3 * n ** 3, -jitter * s, jitter * s).reshape(-1, 3)
    X = X + np.where(interior_axis, jit, 0.0)
    is_boundary = (~interior_axis.all(axis=1)).astype(np.uint8)
    cand = _candidate_bonds(n)
    keep = stream.uniform(cand.shape[0]) < p
    conn = cand[keep]
    L0 = np.linalg.norm(X[conn[:, 1]] - X[conn[:, 0]], axis=1)
    E = conn.shape[0]
    if EA == "lognormal":
        EAv = np.exp(0.5 * stream.normal(E))
    else:
        EAv = np.full(E, float(EA))
    Bv = np.full(E, float(B))
    return Network(X=X, conn=conn, L0=L0, EA=EAv, B=Bv, is_boundary=is_boundary,
                   V0=1.0, meta=dict(n=n, p=p))


def _quat_rotation(q: np.ndarray) -> np.ndarray:
    """Rotation matrix of a unit quaternion (w, x, y, z)."""
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def random_F(stream: Stream, strain_lo: float = -0.05, strain_hi: float = 0.15) -> np.ndarray:
    """F = R U: R Haar-random, U = Q diag(1+e) Q^T with e ~ U[lo, hi].

    Haar rotations come from normalised 4-D Gaussian quaternions.  Draw
    order: R's quaternion (4), Q's quaternion (4), principal strains (3).
    """
    R = _quat_rotation(stream.normal(4))
    Q = _quat_rotation(stream.normal(4))
    e = stream.uniform(3, strain_lo, strain_hi)
    U = Q @ np.diag(1.0 + e) @ Q.T
    return R @ U


F_UNIAXIAL_10 = np.array([[1.1, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


# ---------------------------------------------------------------- workloads

def config_single(seed_index: int = 0) -> tuple[list[Network], np.ndarray]:
    """Single 6^3 RVE, p = 0.6, EA = 1, B = 10 under F = I + 0.1 e1 (x) e1."""
    st = Stream(rve_seed(1, seed_index))
    net = grid_network(6, 0.6, st)
    return [net], F_UNIAXIAL_10[None].copy()


def config_uniform(n_rve: int = 1024, side: int = 10, p: float = 0.6,
                   first: int = 0, config_id: int = 2) -> tuple[list[Network], np.ndarray]:
    """n_rve jittered side^3 grids, p = 0.6, EA = 1, B = 10, random F = R U."""
    nets, Fs = [], []
    for r in range(first, first + n_rve):
        st = Stream(rve_seed(config_id, r))
        nets.append(grid_network(side, p, st))
        Fs.append(random_F(st))
    return nets, np.stack(Fs)


def config_uneven(n_rve: int = 4096, first: int = 0, side_lo: int = 6,
                  side_hi: int = 16) -> tuple[list[Network], np.ndarray]:
    """Uneven batch: side ~ U{lo..hi}, p ~ U[0.5, 0.8], EA log-normal(0, 0.5)
    per fiber, B ~ U[5, 20] per RVE, random F = R U.

    Draw order per RVE: side, p, B, then the grid, then F.
    """
    nets, Fs = [], []
    for r in range(first, first + n_rve):
        st = Stream(rve_seed(3, r))
        side = side_lo + int(st.uniform(1)[0] * (side_hi - side_lo + 1))
        p = float(st.uniform(1, 0.5, 0.8)[0])
        B = float(st.uniform(1, 5.0, 20.0)[0])
        nets.append(grid_network(side, p, st, EA="lognormal", B=B))
        Fs.append(random_F(st))
    return nets, np.stack(Fs)


def config_serving_network(rve_id: int, sides=(6, 8, 12, 16)) -> Network:
    """RVE of the serving pool: side drawn from `sides`, p = 0.6, EA = 1, B = 10."""
    st = Stream(rve_seed(5, rve_id))
    side = sides[int(st.uniform(1)[0] * len(sides)) % len(sides)]
    return grid_network(side, 0.6, st)


def serving_F(rve_id: int, request: int) -> np.ndarray:
    """Random F for request number `request` on pool RVE `rve_id`."""
    return random_F(Stream(rve_seed(6, (rve_id << 20) ^ request)))


# ------------------------------------------------------------------ packing

@dataclass
class Packed:
    """Batch of RVEs packed into flat arrays with per-RVE offsets (CRS-like)."""

    node_off: np.ndarray     # (n+1,) int64
    X: np.ndarray            # (3 N_total,) float64
    fiber_off: np.ndarray    # (n+1,) int64
    conn: np.ndarray         # (2 E_total,) int32, RVE-local node ids
    L0: np.ndarray
    EA: np.ndarray
    B: np.ndarray
    is_boundary: np.ndarray  # (N_total,) uint8
    V0: np.ndarray           # (n,) float64

    @property
    def n_rve(self) -> int:
        return self.node_off.shape[0] - 1


def pack(nets: list[Network]) -> Packed:
    node_off = np.zeros(len(nets) + 1, np.int64)
    fiber_off = np.zeros(len(nets) + 1, np.int64)
    node_off[1:] = np.cumsum([n.n_nodes for n in nets])
    fiber_off[1:] = np.cumsum([n.n_fibers for n in nets])
    cat = lambda xs, dt: (np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt))
    return Packed(
        node_off=node_off,
        X=np.ascontiguousarray(cat([n.X.ravel() for n in nets], np.float64)),
        fiber_off=fiber_off,
        conn=np.ascontiguousarray(cat([n.conn.ravel() for n in nets], np.int32)),
        L0=np.ascontiguousarray(cat([n.L0 for n in nets], np.float64)),
        EA=np.ascontiguousarray(cat([n.EA for n in nets], np.float64)),
        B=np.ascontiguousarray(cat([n.B for n in nets], np.float64)),
        is_boundary=np.ascontiguousarray(cat([n.is_boundary for n in nets], np.uint8)),
        V0=np.array([n.V0 for n in nets], np.float64),
    )


def unpack(pk: Packed, r: int) -> Network:
    a, b = pk.node_off[r], pk.node_off[r + 1]
    c, d = pk.fiber_off[r], pk.fiber_off[r + 1]
    return Network(X=pk.X[3 * a:3 * b].reshape(-1, 3), conn=pk.conn[2 * c:2 * d].reshape(-1, 2),
                   L0=pk.L0[c:d], EA=pk.EA[c:d], B=pk.B[c:d],
                   is_boundary=pk.is_boundary[a:b], V0=float(pk.V0[r]))
