"""CPU-rank simulation of the paper's transpose-free slab decomposition
(Sec. 2.2), as test infrastructure: p processes each hold n0/p planes of the
real array; after the local 2D transforms of their planes each sends to rank s
the block with k1 in [s*n1/p, (s+1)*n1/p) -- n0/p strided runs of (n1/p)*H
contiguous values at stride n1*H, the shape of an MPI vector type -- and lays
what it receives down contiguously, so that it holds n0 x (n1/p) x H with the
n0 axis outermost at stride (n1/p)*H, and transforms that axis in place at its
stride.  No local transpose anywhere.  The inverse runs the steps in reverse
order.  The local transforms use numpy.fft (an independent library); the
point under test is the data layout and the exchange.
"""
from __future__ import annotations

import numpy as np


def send_block(local: np.ndarray, s: int, p: int) -> np.ndarray:
    """The values of a rank's slab (n0/p, n1, H) destined for rank s, in the
    order a strided vector type (count n0/p, block (n1/p)*H, stride n1*H)
    picks them from the flat slab."""
    n0p, n1 = local.shape[0], local.shape[1]
    h = int(np.prod(local.shape[2:], dtype=int)) if local.ndim > 2 else 1
    b = n1 // p
    flat = local.reshape(-1)
    idx = (np.arange(n0p)[:, None] * (n1 * h) + s * b * h + np.arange(b * h)[None, :]).ravel()
    return flat[idx]


def place_received(blocks, n0p: int, b: int, tail) -> np.ndarray:
    """Contiguous receive: the block from rank q is rows [q*n0p, (q+1)*n0p) of
    the (n0, n1/p, ...) buffer."""
    return np.concatenate([np.asarray(x).reshape((n0p, b) + tuple(tail)) for x in blocks], axis=0)


def return_block(held: np.ndarray, q: int, p: int) -> np.ndarray:
    """Inverse exchange: the rows of the (n0, n1/p, H) buffer that rank q owns,
    a contiguous run."""
    n0p = held.shape[0] // p
    return held[q * n0p:(q + 1) * n0p].reshape(-1)


def place_returned(blocks, n0p: int, n1: int, p: int, tail) -> np.ndarray:
    """Strided receive of the inverse exchange: the block from rank s fills
    the k1 columns [s*n1/p, (s+1)*n1/p) of every local plane."""
    b = n1 // p
    out = np.empty((n0p, n1) + tuple(tail), dtype=np.asarray(blocks[0]).dtype)
    for s, x in enumerate(blocks):
        out[:, s * b:(s + 1) * b] = np.asarray(x).reshape((n0p, b) + tuple(tail))
    return out
