"""CPU FP64 oracle for LU_PRRP: test infrastructure only.

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs (``cpu_baseline`` and
``--impl reference``) may import this package. The product package
``paper_1208_2451_gb300`` never imports it and shares no code with it.
"""
from .algorithm import (LUResult, NonFiniteError, PanelResult, SingularError, SwapLimitError,
                      eta, householder_qr, lu_prrp, lu_solve, qrcp, refine, selection_multipliers, strong_rrqr, unpack)
from .block_lu import BlockLUResult, block_lu_prrp, block_solve
from .calu import CALUResult, calu_growth_bound_log10, calu_prrp
from . import metrics

__all__ = ["LUResult", "NonFiniteError", "PanelResult", "SingularError", "SwapLimitError", "eta",
           "householder_qr", "lu_prrp", "lu_solve", "qrcp", "refine", "selection_multipliers",
           "strong_rrqr", "unpack", "CALUResult", "calu_prrp", "calu_growth_bound_log10",
           "BlockLUResult", "block_lu_prrp", "block_solve",
           "metrics"]
