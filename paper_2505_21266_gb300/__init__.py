"""GB300-native Discrete Morse Sandwich hot path (arXiv 2505.21266).

order -> lower-star discrete gradient -> critical simplices -> D0/D2 pairs
(and D1 after them),
all in hand-written CUDA for sm_103a behind a C ABI (``include/dms.h``).
The CUDA library is loaded on first use; importing this package needs no GPU.
"""
from .api import (CRITICAL, PAIR_DTYPE, DiagramFn, Diagrams, Diagrams2d, DMSError, Gradient,
                  Gradient2d, Result, Result2d, backward, critical, critical2d, diagram,
                  diagram2d, diagram_d0d1, diagram_d0d2, diagram_d1, diagram_from_host, diagram_values,
                  diagrams_from_host,
                  gradient, gradient2d, order, order2d, pair_values, topological_loss)

__all__ = ["order", "gradient", "critical", "diagram_d0d2", "diagram_d1", "diagram",
           "diagram_from_host", "diagrams_from_host",
           "order2d", "gradient2d", "critical2d", "diagram_d0d1", "diagram2d", "Gradient2d",
           "Diagrams2d", "Result2d",
           "backward", "DiagramFn", "diagram_values", "pair_values", "topological_loss",
           "Gradient", "Diagrams", "Result", "DMSError", "PAIR_DTYPE", "CRITICAL"]
