"""FP64 CPU oracle of circulant-embedding conditional simulation.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package.  The CUDA library never calls it and shares no code with it.
"""
from .ce_oracle import *  # noqa: F401,F403
