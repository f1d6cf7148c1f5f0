"""Small hand-built networks for tests (inputs only, no solver arithmetic)."""
import numpy as np

import rvegen


def lattice(n, p=1.0, jitter=0.0, seed=0, EA=1.0, B=10.0):
    """n^3 grid; jitter=0 and p=1 gives the regular lattice."""
    st = rvegen.Stream(seed)
    return rvegen.grid_network(n, p, st, jitter=jitter, EA=EA, B=B)


def tiny(kind, seed=0):
    """Networks with 1-3 free nodes for brute-force checks."""
    rng = np.random.default_rng(seed)
    if kind == "one":
        Xb = np.array([[-.5, 0, 0], [.5, 0, 0], [0, -.5, 0], [0, .5, 0], [0, 0, -.5], [0, 0, .5]])
        Xf = rng.uniform(-.1, .1, (1, 3))
        X = np.vstack([Xf, Xb])
        conn = np.array([[0, k] for k in range(1, 7)])
    elif kind == "two":
        Xb = np.array([[-.5, .2, 0], [-.5, -.2, .1], [-.5, 0, -.3], [.5, .2, 0], [.5, -.2, .1], [.5, 0, -.3]])
        Xf = np.array([[-.15, 0, 0], [.15, 0, 0]]) + rng.uniform(-.05, .05, (2, 3))
        X = np.vstack([Xf, Xb])
        conn = np.array([[0, 1], [0, 2], [0, 3], [0, 4], [1, 5], [1, 6], [1, 7]])
    elif kind == "three":
        Xb = np.array([[-.5, 0, 0], [.5, 0, 0], [0, -.5, 0], [0, .5, 0], [0, 0, -.5], [0, 0, .5], [.4, .4, .4]])
        Xf = np.array([[-.15, 0, 0], [.15, 0, 0], [0, .15, .1]]) + rng.uniform(-.05, .05, (3, 3))
        X = np.vstack([Xf, Xb])
        conn = np.array([[0, 1], [1, 2], [2, 0], [0, 3], [0, 5], [0, 7], [1, 4], [1, 8], [1, 6],
                         [2, 6], [2, 8], [2, 9]])
    else:
        raise ValueError(kind)
    nb = np.zeros(X.shape[0], np.uint8)
    nb[{"one": 1, "two": 2, "three": 3}[kind]:] = 1
    L0 = np.linalg.norm(X[conn[:, 1]] - X[conn[:, 0]], axis=1)
    E = conn.shape[0]
    EA = rng.uniform(0.5, 2.0, E)
    B = rng.uniform(2.0, 15.0, E)
    return rvegen.Network(X=X, conn=conn.astype(np.int32), L0=L0, EA=EA, B=B, is_boundary=nb, V0=1.0)


def F_tension_shear():
    return np.array([[1.1, 0.05, 0.0], [0.0, 1.05, 0.02], [0.0, 0.0, 1.08]])
