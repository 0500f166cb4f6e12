"""Restart schedule of a full oracle solve of a named workload.

TEST INFRASTRUCTURE ONLY: runs the CPU oracle (single thread) on the seeded
workload to the binary64 target and prints its inner iterations, restart
cycles and CPU seconds as one JSON line.  bench.py's reference arm scales its
bounded per-cycle samples of the oracle to this schedule.  At 160^3 the solve
takes about 20 minutes.

    python -m oracle.schedule convdiff3d_160 mixed
"""
from __future__ import annotations

import json
import sys
import time


def main(argv=None):
    import oracle as O
    from paper_2011_01850_gb300 import inputs as I

    argv = sys.argv[1:] if argv is None else argv
    name, prec = argv[0], argv[1]
    A, b, spec = I.workload(name, seed=20110185)
    P = {"fp64": O.FP64, "mixed": O.MIXED, "mixed_bf16": O.MIXED_BF16,
         "mixed_fp16": O.MIXED_FP16}[prec]
    ortho = O.MGS if spec["ortho"] == "mgs" else O.CGSR
    t = time.time()
    _, info = O.gmres(A, b, m=spec["m"], tol=1e-10, ortho=ortho, prec=P, maxiter=100000)
    info["seconds"] = round(time.time() - t, 1)
    info.update(workload=name, prec=prec, m=spec["m"], ortho=spec["ortho"])
    print(json.dumps(info), flush=True)


if __name__ == "__main__":
    main()
