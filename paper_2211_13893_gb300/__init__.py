"""GB300 (sm_103a) MS-GFEM local stage: C-ABI library libmsgfem and its binding."""
from .msgfem import MSGFEM, MsgfemError, Net, load_library, plan, LIB_PATH, EXPORTS  # noqa: F401
