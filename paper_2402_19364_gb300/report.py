"""Structure report of an arrow decomposition (host only, no GPU).

For a synthetic workload it prints, as one JSON line, what the decomposition results of
Section 6 describe for the paper's datasets: the order l of the decomposition, every level's
active rows and entries, how the entries of each B_i split between the head rows/columns
(the part pruned towards the top and left corners) and the band, and the number of non-zero
b x b tiles summed over the levels against the tiles of the matrix in its own order (the
equally sized blocks of a 1.5D distribution).  With --predicate both it also decomposes
with the literal band of Section 1 (host-only there) to compare level counts and tiles.

    python -m paper_2402_19364_gb300.report --workload grid3d --size 100 --b 256
    python -m paper_2402_19364_gb300.report --workload rmat --size 18 --b 1024 --predicate both
"""
from __future__ import annotations

import argparse
import json
import math
import time


def _matrix(workload: str, size: int, seed: int):
    import workloads as w
    if workload == "grid3d":
        return w.grid3d(size, seed=seed), f"3D {size}^3 grid, 7-point stencil"
    if workload == "grid2d":
        return w.grid_stencil((size, size), seed=seed), f"2D {size}x{size} grid, 5-point stencil"
    if workload == "rmat":
        return w.rmat_gcn(size, 16, seed=seed), f"R-MAT scale {size}, edge factor 16, GCN-normalised"
    if workload == "rgg":
        return w.rgg(size, seed=seed), f"2D random-geometric graph, n = {size}, mean degree 8"
    raise SystemExit(f"unknown workload {workload}")


def report(A, b: int, predicate: str = "block", seed: int = 0, nthreads: int = 0) -> dict:
    """Decompose A (host only) and return its structure report."""
    from . import ArrowMatrix, count_tiles
    t0 = time.perf_counter()
    M = ArrowMatrix(A, b, seed=seed, predicate=predicate, host_only=True, nthreads=nthreads)
    secs = time.perf_counter() - t0
    rep = M.structure_report()
    rep["predicate"] = predicate
    rep["decompose_s"] = secs
    rep["tiles_input_order"] = count_tiles(A, b)
    M.close()
    return rep


def main(argv=None) -> None:
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--workload", default="grid3d", choices=["grid3d", "grid2d", "rmat", "rgg"])
    p.add_argument("--size", type=int, default=100)
    p.add_argument("--b", type=int, default=0, help="arrow width (0: ceil(sqrt(n)))")
    p.add_argument("--seed", type=int, default=3)
    p.add_argument("--predicate", default="block", choices=["block", "band", "both"])
    p.add_argument("--threads", type=int, default=0)
    a = p.parse_args(argv)
    A, desc = _matrix(a.workload, a.size, a.seed)
    b = a.b or int(math.ceil(math.sqrt(A.n)))
    preds = ["block", "band"] if a.predicate == "both" else [a.predicate]
    out = {"workload": desc, "n": int(A.n), "nnz": int(A.nnz), "b": b,
           "reports": [report(A, b, pr, seed=a.seed, nthreads=a.threads) for pr in preds]}
    for r in out["reports"]:
        del r["n"], r["nnz"], r["b"]
    print(json.dumps(out))


if __name__ == "__main__":
    main()
