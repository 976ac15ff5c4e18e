"""Test-side helpers (numpy only): packing of +-1 hypervectors into words.

Packed layout of the library: bit d of a hypervector is bit (d % 32) of
32-bit word d // 32; a set bit is the element -1; words past the last
dimension are zero.  These helpers convert between that layout and the
oracle's one-byte-per-dimension arrays.  They hold none of the method's
arithmetic.
"""
import numpy as np


def words_for(D: int) -> int:
    """Words per packed row: ceil(D/32) rounded up to a multiple of 4."""
    w = (D + 31) // 32
    return (w + 3) // 4 * 4


def pack(bits: np.ndarray, W: int | None = None) -> np.ndarray:
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    n, D = bits.shape
    W = words_for(D) if W is None else W
    pad = np.zeros((n, W * 32), dtype=np.uint8)
    pad[:, :D] = bits
    by = np.packbits(pad.reshape(n, W * 4, 8), axis=2, bitorder="little").reshape(n, W * 4)
    return by.view("<u4").reshape(n, W).copy()


def unpack(words: np.ndarray, D: int) -> np.ndarray:
    words = np.ascontiguousarray(words, dtype="<u4")
    n, W = words.shape
    by = words.view(np.uint8).reshape(n, W * 4)
    bits = np.unpackbits(by, axis=1, bitorder="little")
    return bits[:, :D].copy()
