"""FP64 CPU oracle of the SG-splatting rasterizer -- test infrastructure only.

Only the tests, the smoke check and the bench's CPU-baseline leg may import it.
"""
from .sg_oracle import *  # noqa: F401,F403
from .sg_oracle import Decisions, ViewResult  # noqa: F401
from . import sg_admm_oracle as admm  # noqa: F401,E402
from . import sg_post_oracle as post  # noqa: F401,E402
from . import sg_sh_oracle as sh  # noqa: F401,E402
