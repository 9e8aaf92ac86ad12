"""GB300-native (sm_103a) single-chain slip-spring model (T. Uneyama, arXiv:1106.2899).

The product is the C-ABI library built from csrc/ (include/slipspring.h); this
package builds it (`build`) and binds it (`api.SlipSpring`).  Importing the
package does not load the library; creating a context does, and fails loudly if
it is missing.
"""
from .api import SlipSpring  # noqa: F401
