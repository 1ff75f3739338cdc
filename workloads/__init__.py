"""Seeded synthetic inputs for the HODLR/HSS matrix-times-block product.

This package is shared by the CPU oracle (``oracle/``), the tests and the
benchmark.  It only draws random numbers and writes down fixture generators
from closed formulas; it performs none of the matrix-vector arithmetic whose
correctness the oracle and the CUDA path are compared on.

Generator dictionaries (the layout every consumer in this repository uses):

* Cluster tree: the leaf-end vector ``c = [n_1, ..., n_{2^p}]`` of Sec. 3.7
  (0-based row ``g`` of leaf ``i`` satisfies ``c[i-1] <= g < c[i]``).
* Node ids are level order: level ``l`` (root = 0), position ``j`` (0-based)
  has id ``2**l - 1 + j``.  Internal nodes are ids ``0 .. L-2`` and leaves are
  ids ``L-1 .. 2L-2`` with ``L = 2**p``.
* HODLR (Def. 2.2 and the ``hodlr`` class of Sec. 2.1):
  ``{"kind": "hodlr", "D": [L], "U12": [L-1], "V12": [L-1], "U21": [L-1],
  "V21": [L-1]}``; for internal node q with children a (left), b (right):
  ``A(I_a, I_b) = U12[q] @ V12[q].T`` and ``A(I_b, I_a) = U21[q] @ V21[q].T``.
* HSS (Def. 2.3, Eq. 2.2 and the ``hss`` class of Sec. 2.2):
  ``{"kind": "hss", "D": [L], "U": [L], "V": [L], "RU": [2L-1], "RV": [2L-1],
  "B12": [L-1], "B21": [L-1]}``; ``RU[q] = [Rl; Rr]`` and ``RV[q] = [Wl; Wr]``
  for internal non-root q (``None`` elsewhere).
"""

from .synth import *  # noqa: F401,F403
