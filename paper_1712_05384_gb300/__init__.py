"""GB300-native amplitudes of random grid circuits by complex graphical-model
variable elimination (Boixo, Isakov, Smelyanskiy, Neven, arXiv:1712.05384).

The product is the C-ABI library ``libqgm.so`` (``include/qgm.h``); this
package is its thin binding (``_lib``), the build step (``build``), the
torch.autograd wrapper of the amplitudes and their adjoint elimination
(``autograd``, imported on first use), bitstring sharding over ranks
(``shard``), observables (``observable``) and the ordering study (``study``).
"""
from ._lib import (EXEC_AUTO, EXEC_COMPILED, EXEC_RESIDENT, EXEC_STEPWISE, OUT_BATCH, OUT_OPEN, ORDER_AUTO, ORDER_GIVEN, ORDER_MINFILL, ORDER_VERTICAL,
                   ORDER_VERTICAL_T, Circuit, Model, Plan, QgmError, lib)

__all__ = ["EXEC_AUTO", "EXEC_COMPILED", "EXEC_RESIDENT", "EXEC_STEPWISE", "Circuit", "Model", "Plan", "QgmError", "lib", "OUT_BATCH", "OUT_OPEN", "ORDER_AUTO",
           "ORDER_GIVEN", "ORDER_MINFILL", "ORDER_VERTICAL", "ORDER_VERTICAL_T"]


def __getattr__(name):
    # torch-facing helpers, imported on first use
    if name == "autograd":
        import importlib
        return importlib.import_module(".autograd", __name__)
    raise AttributeError(name)
