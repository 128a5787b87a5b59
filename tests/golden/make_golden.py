"""Write the stored oracle solutions used by the full-size parity tests.

Calls only the CPU oracle (``oracle``) on the seeded inputs of
``workloads``; nothing here touches the CUDA library.  Each file records a
SHA-256 of the input bytes so that a test can confirm that the generator
rebuilt exactly the same problem before comparing against the stored x.

    python tests/golden/make_golden.py            # all files
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads  # noqa: E402


def input_digest(p) -> str:
    h = hashlib.sha256()
    for a in (p.row_ptr.astype(np.int64), p.col_idx.astype(np.int32), p.val.astype(np.float64),
              p.b.astype(np.float64)):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def write(name, prob, **kw):
    t = time.time()
    r = oracle.bpp_solve(prob, **kw)
    path = os.path.join(HERE, name)
    np.savez_compressed(path, x=r.x, y=r.y, inF=r.inF.astype(np.uint8), trace=r.trace,
                        digest=np.array(input_digest(prob)), seconds=np.array(time.time() - t))
    print(f"{name}: iters={r.iters} |F|={r.final_k} {time.time() - t:.1f}s")


if __name__ == "__main__":
    write("larger_sparse_20000x8000.npz", workloads.larger_sparse(), final_step=oracle.FINAL_LSQR)
