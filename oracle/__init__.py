"""Plain FP64 CPU oracle for the rigid-aggregate FSD saddle-point solve.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The product path (the CUDA library and its Python binding) never
imports, links or executes anything in here, and this package never imports
the product package.
"""

from .fsd_oracle import *  # noqa: F401,F403
