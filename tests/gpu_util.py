"""Helpers for the GPU tests: column-major uint32 matrices <-> device tensors.

A column-major m x n matrix with leading dimension m has the same bytes as a
row-major n x m array, so a device tensor of shape (n, m) (int32 view of the
words) holds it and element (i, j) is tensor[j, i].
"""
import numpy as np
import torch

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def to_dev(M: np.ndarray) -> torch.Tensor:
    """Column-major copy of a 2-D (or 1-D) uint32 array on the GPU."""
    M = np.asarray(M, dtype=np.uint32)
    if M.ndim == 1:
        return torch.from_numpy(M.view(np.int32).copy()).to(DEV)
    return torch.from_numpy(np.ascontiguousarray(M.T).view(np.int32)).to(DEV)


def from_dev(T: torch.Tensor, shape=None) -> np.ndarray:
    """Back to a (rows, cols) uint32 array from a (cols, rows) device tensor."""
    h = T.detach().cpu().numpy().view(np.uint32)
    if h.ndim == 1:
        return h.copy()
    return np.ascontiguousarray(h.T)


def words_to_dev(w: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(w, dtype=np.uint32).view(np.int32)).to(DEV)


def words_from_dev(T: torch.Tensor) -> np.ndarray:
    return T.detach().cpu().numpy().view(np.uint32).copy()


def mixed_words(rng: np.random.Generator, count: int) -> np.ndarray:
    """Posit words from several families: any word; |x| near 1; long
    regimes (tiny and huge magnitudes, incl. the exponent-truncated band);
    few fraction bits (exact results and ties); the special words."""
    fam = rng.integers(0, 4, size=count)
    w = rng.integers(0, 2 ** 32, size=count, dtype=np.uint64).astype(np.uint32)
    near1 = (w & np.uint32(0x8FFFFFFF)) | (rng.integers(2, 6, size=count).astype(np.uint32) << np.uint32(28))
    shift = rng.integers(1, 31, size=count).astype(np.uint32)
    body = (w & np.uint32(0x7FFFFFFF)) >> shift
    flip = rng.integers(0, 2, size=count).astype(bool)
    body = np.where(flip, np.uint32(0x7FFFFFFF) - body, body)
    body = np.maximum(body, np.uint32(1))
    longreg = np.where(w >> np.uint32(31) == 1, (~body + np.uint32(1)).astype(np.uint32), body)
    fewbits = (w & np.uint32(0xFFFC0000)) | ((w >> np.uint32(5)) & np.uint32(1))
    out = np.where(fam == 0, w, np.where(fam == 1, near1, np.where(fam == 2, longreg, fewbits)))
    out = out.astype(np.uint32)
    specials = np.array([0, 0x80000000, 0x40000000, 0xC0000000, 1, 0xFFFFFFFF,
                         0x7FFFFFFF, 0x80000001, 2, 3, 0x7FFFFFFE, 0x7FFFFFFD], np.uint32)
    out[: specials.size] = specials
    return out
