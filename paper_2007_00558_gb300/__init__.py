"""GB300-native view synthesis (FVV Live, Sec. VI) behind the C ABI of
include/fvv.h.  ``fvv`` is the ctypes binding; ``build`` compiles libfvv.so."""
from . import build  # noqa: F401
from . import fvv  # noqa: F401
