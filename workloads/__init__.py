"""Seeded synthetic inputs for the satisfiability check of out-of-bounds queries.

This package builds *inputs only*: integer constraint sets (query IR) shaped like
the paper's worked examples (Figs. 1-5, Sec. IV-A/V-B) and uniform random 3-SAT
formulas. It holds none of the method's arithmetic: no bit-blasting, no
solving, no evaluation. Both the product encoder and the CPU oracle consume the
same serialized IR (``workloads.ir``), each with its own code.
"""
from .ir import IR, OP, IR_MAGIC, IR_VERSION  # noqa: F401
from .rng import SplitMix64  # noqa: F401
from . import queries  # noqa: F401
