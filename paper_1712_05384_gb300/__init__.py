"""GB300-native amplitudes of random grid circuits by complex graphical-model
variable elimination (Boixo, Isakov, Smelyanskiy, Neven, arXiv:1712.05384).

The product is the C-ABI library ``libqgm.so`` (``include/qgm.h``); this
package is its thin binding (``_lib``) plus the build step (``build``) and the
torch-facing helpers (``api``).
"""
from ._lib import (EXEC_AUTO, EXEC_COMPILED, EXEC_RESIDENT, EXEC_STEPWISE, OUT_BATCH, OUT_OPEN, ORDER_AUTO, ORDER_GIVEN, ORDER_MINFILL, ORDER_VERTICAL,
                   ORDER_VERTICAL_T, Circuit, Model, Plan, QgmError, lib)

__all__ = ["EXEC_AUTO", "EXEC_COMPILED", "EXEC_RESIDENT", "EXEC_STEPWISE", "Circuit", "Model", "Plan", "QgmError", "lib", "OUT_BATCH", "OUT_OPEN", "ORDER_AUTO",
           "ORDER_GIVEN", "ORDER_MINFILL", "ORDER_VERTICAL", "ORDER_VERTICAL_T"]
