"""D2Q9 and D3Q19 velocity sets (Sec. 2.1: 'The D2Q9 stencil and the D3Q19
stencil have been used').  Ordering is private to the oracle."""
import numpy as np

CS2 = 1.0 / 3.0  # lattice speed of sound squared, c_s = 1/sqrt(3) (Sec. 2.1)


def velocity_set(q: int):
    """Return (xi, w, opp): xi (q, 3) int, w (q,) float64, opp (q,) int."""
    if q == 9:
        xi = [(0, 0, 0)]
        xi += [(1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0)]
        xi += [(1, 1, 0), (-1, 1, 0), (-1, -1, 0), (1, -1, 0)]
        w = [4.0 / 9.0] + [1.0 / 9.0] * 4 + [1.0 / 36.0] * 4
    elif q == 19:
        xi = [(0, 0, 0)]
        xi += [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]
        for a, b in ((0, 1), (0, 2), (1, 2)):
            for sa in (1, -1):
                for sb in (1, -1):
                    v = [0, 0, 0]
                    v[a], v[b] = sa, sb
                    xi.append(tuple(v))
        w = [1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12
    else:
        raise ValueError("q must be 9 or 19")
    xi = np.array(xi, dtype=np.int64)
    w = np.array(w, dtype=np.float64)
    opp = np.array([int(np.nonzero((xi == -xi[i]).all(axis=1))[0][0]) for i in range(q)])
    return xi, w, opp


def dim_of(q: int) -> int:
    return 2 if q == 9 else 3
