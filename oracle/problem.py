"""Convenience: build every oracle input of a ``workloads.ProblemSpec``.

Oracle (test infrastructure only).  Combines the oracle's own assembly,
partition and coarse interpolation modules.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import bpjd, coarse, fem, partition


@dataclass
class OracleProblem:
    spec: object
    K: sp.csr_matrix
    M: sp.csr_matrix
    P: sp.csr_matrix
    P0: sp.csr_matrix
    sub_ptr: np.ndarray
    sub_dofs: np.ndarray
    sub_color: np.ndarray
    n_colors: int

    def setup(self) -> bpjd.Setup:
        return bpjd.setup(self.K, self.M, self.P, self.sub_ptr, self.sub_dofs, self.spec.k,
                          P0=None if self.spec.tau == 0 else self.P0)


def build(spec) -> OracleProblem:
    spec.validate()
    K, M = fem.assemble(spec)
    P = coarse.prolongation(spec)
    P0 = P if spec.tau == 0 else coarse.prolongation(spec.initial_grid())
    if getattr(spec, "partition", "boxes") == "triangles":
        ptr, dofs, col, nc = partition.triangle_partition(spec.n[0], spec.nsub[0], spec.delta)
    else:
        ptr, dofs, col, nc = partition.box_partition(spec)
    return OracleProblem(spec, K, M, P, P0, ptr, dofs, col, nc)
