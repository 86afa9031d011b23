"""The local-maximum tie rule of Sec. V.B, literally and exactly (test
infrastructure: only tests/ use it).

The paper breaks ToT ties by adding 0.001 times the pixel's position in the
data stream to its ToT, so that the later pixel wins. Taken literally, the
offset stops being a tie-break once positions reach 1000: it then outweighs a
whole ToT unit and a dimmer, later pixel beats a brighter, earlier neighbour.
The library and the oracle use the exact reading -- compare (ToT, position)
lexicographically -- which is what the rule intends and agrees with the
literal one whenever positions stay below 1000.
"""
from __future__ import annotations

import numpy as np


def maxima_literal(tot: np.ndarray, pos: np.ndarray, adj: np.ndarray) -> np.ndarray:
    """Local maxima with the literal key ToT + 0.001 * position (adj: the
    boolean adjacency matrix of the pixels, zero diagonal)."""
    key = np.asarray(tot, float) + 0.001 * np.asarray(pos, float)
    n = key.size
    return np.array([not any(adj[i, j] and key[j] > key[i] for j in range(n)) for i in range(n)])


def maxima_exact(tot: np.ndarray, pos: np.ndarray, adj: np.ndarray) -> np.ndarray:
    """Local maxima with the exact key (ToT, position), compared
    lexicographically."""
    n = len(tot)
    return np.array([not any(adj[i, j] and (tot[j], pos[j]) > (tot[i], pos[i]) for j in range(n))
                     for i in range(n)])
