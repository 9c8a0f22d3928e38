"""GB300-native Discrete Morse Sandwich hot path (arXiv 2505.21266).

order -> lower-star discrete gradient -> critical simplices -> D0/D2 pairs,
all in hand-written CUDA for sm_103a behind a C ABI (``include/dms.h``).
The CUDA library is loaded on first use; importing this package needs no GPU.
"""
from .api import (CRITICAL, PAIR_DTYPE, DiagramFn, Diagrams, DMSError, Gradient, Result,
                  backward, critical, diagram, diagram_d0d2, diagram_from_host, diagram_values,
                  gradient, order, pair_values, topological_loss)

__all__ = ["order", "gradient", "critical", "diagram_d0d2", "diagram", "diagram_from_host",
           "backward", "DiagramFn", "diagram_values", "pair_values", "topological_loss",
           "Gradient", "Diagrams", "Result", "DMSError", "PAIR_DTYPE", "CRITICAL"]
