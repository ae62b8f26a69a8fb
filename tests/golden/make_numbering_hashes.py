"""Writes numbering_hashes.txt: SHA-256 of the oracle's global numbering and Dirichlet
mask for the box meshes the full-size tests use (Section 3.1's Q; Algorithm 1 step 7).

Calls only oracle/ and synthetic/ (topology does not depend on the jitter).
Run: python tests/golden/make_numbering_hashes.py   (a few minutes of CPU)
"""
import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import sem_oracle as so  # noqa: E402
from synthetic import BoxMesh  # noqa: E402

CASES = [(32, 7), (20, 3), (9, 11)]  # (elements per direction, N)


def main():
    lines = ["# SHA-256 of the oracle's int64 glo_num bytes and uint8 mask bytes (little endian)",
             "# written by make_numbering_hashes.py; columns: n N n_glob sha_glo sha_mask"]
    for n, N in CASES:
        m = BoxMesh(n, n, n)
        num = so.number_nodes(N, m.elem_verts)
        hg = hashlib.sha256(num.glo_num.astype("<i8").tobytes()).hexdigest()
        hm = hashlib.sha256(num.mask.astype(np.uint8).tobytes()).hexdigest()
        lines.append(f"{n} {N} {num.n_glob} {hg} {hm}")
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "numbering_hashes.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
