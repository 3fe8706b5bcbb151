"""Write tests/golden/factor8192.txt: the CPU oracle's Rgetrf and Rpotrf('L')
of the two n = 8192 workload matrices (Sec. 5.2 factors N = 8000-class
matrices; Table taball), stored as SHA-256 digests of the factors, pivots and
info, plus one CRC-32 per column so that a mismatch can be located.

Only the oracle (oracle/) and the seeded input generators
(paper_2401_14117_gb300.inputs) are used; nothing comes from the CUDA
library.  The oracle takes about half an hour per factorisation on 8 cores.

    python tests/golden/make_factor8192.py [--threads T]
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time
import zlib

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2401_14117_gb300 import inputs  # noqa: E402

N = 8192
LU_SEED = inputs.SEED_BASE + 3
CHOL_SEED = inputs.SEED_BASE + 5
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "factor8192.txt")


def lu_input() -> np.ndarray:
    """A uniform in [-1, 1], rounded to posit by the oracle's conversion."""
    return oracle.from_double_array(inputs.uniform((N, N), LU_SEED))


def chol_input() -> np.ndarray:
    """A = G G^T / n + I (exact in FP64 on any host), rounded to posit."""
    return oracle.from_double_array(inputs.spd(N, CHOL_SEED))


def sha(a: np.ndarray) -> str:
    """Digest of a matrix's column-major bytes (or of a vector's bytes)."""
    a = np.asarray(a)
    return hashlib.sha256(a.tobytes(order="F")).hexdigest()


def column_crcs(F: np.ndarray) -> list[int]:
    Ft = np.ascontiguousarray(np.asarray(F, dtype=np.uint32).T)
    return [zlib.crc32(Ft[j].tobytes()) for j in range(Ft.shape[0])]


def record(tag: str, A: np.ndarray, F: np.ndarray, ipiv, info: int) -> list[str]:
    lines = [f"{tag} n {N}", f"{tag} input_sha256 {sha(A)}", f"{tag} info {info}",
             f"{tag} factor_sha256 {sha(F)}"]
    if ipiv is not None:
        lines.append(f"{tag} ipiv_sha256 {sha(np.asarray(ipiv, dtype=np.int32))}")
    crcs = column_crcs(F)
    for c0 in range(0, N, 64):
        lines.append(f"{tag} crc32 {c0} " + " ".join(f"{c:08x}" for c in crcs[c0:c0 + 64]))
    return lines


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count())
    args = ap.parse_args()
    oracle.set_threads(args.threads)
    out = ["# The CPU oracle's factorisations of the n = 8192 workload matrices",
           "# (Sec. 5.2, Table taball): SHA-256 of the column-major factor words,",
           "# of the 1-based pivots and of the matrix that was factored, info, and",
           "# one CRC-32 per column (64 per line: first column, then the CRCs).",
           "# lu:   A uniform in [-1, 1], seed SEED_BASE + 3, unblocked Rgetrf",
           "# chol: A = G G^T / n + I, seed SEED_BASE + 5, unblocked Rpotrf('L')",
           "# written by: python tests/golden/make_factor8192.py (oracle/ only)"]
    t = time.time()
    A = lu_input()
    F, ipiv, info = oracle.rgetrf(A)
    out += record("lu", A, F, ipiv, info)
    print(f"lu: info {info}, {time.time() - t:.0f} s", flush=True)
    t = time.time()
    S = chol_input()
    Fs, info_s = oracle.rpotrf(S, uplo="L")
    out += record("chol", S, Fs, None, info_s)
    print(f"chol: info {info_s}, {time.time() - t:.0f} s", flush=True)
    with open(OUT + ".tmp", "w") as f:
        f.write("\n".join(out) + "\n")
    os.replace(OUT + ".tmp", OUT)
    print(OUT)


if __name__ == "__main__":
    main()
