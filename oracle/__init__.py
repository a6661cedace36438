"""Plain FP64 CPU oracle of the hybrid pressure-correction sub-step (Fang, arXiv 2304.14690).

TEST INFRASTRUCTURE ONLY. This package exists to check the CUDA library against the paper.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it. The product path (``paper_2304_14690_gb300``) never imports, calls or links it,
and shares no code, table or constant generator with it; the only common module is the
seeded input generator ``paper_2304_14690_gb300.workloads``, which holds none of the
method's arithmetic.

Everything here is float64 numpy, written for a reader who checks it against the paper:

* ``grid``        - the staggered (MAC) pressure grid, its boundary kinds and the 2d+1-point
                    Laplacian with its ghost-cell rules (§2.1 Eq. 7, §3.3 wall workaround).
* ``knn``         - the linked-list (cell-list) neighbour search of §2.2.
* ``wls``         - the weighted-least-squares rows C^-1 A of §2.2 Eqs. 13-17, with the
                    f-unknown basis (Eq. 16) and the Gaussian weight (Eq. 17).
* ``poisson``     - the three-step transform solve of §2.3 written as an exact eigen-expansion
                    of the discrete Laplacian, axis by axis.
* ``projection``  - the whole sub-step: transfer, divergence source of the modified PPE
                    (§2.3 Eq. 20), solve, WLS gradient, correction with IB force (Eqs. 18-19).

Parity status of each function is stated in its module header; every function is pinned by
``tests/test_oracle_*.py`` except the comparison with the paper's flow results, which is
"parity unpinned" (they need the whole flow solver and data the paper does not publish).
"""
from . import grid, knn, wls, poisson, projection  # noqa: F401
